"""Thin ctypes binding of the C ABI in include/mm.h (argument marshalling only).

Every computation runs in libmm.so's CUDA kernels; if the library is missing
or no CUDA device is usable, the calls raise -- there is no fallback.

Arrays: numpy float64 arrays are passed as host pointers; torch float64 CUDA
tensors are passed as device pointers (read or written in stream order on the
handle's stream, by default torch's current stream).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .inputs import Grid, Rates

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmm.so")

MM_FP64 = 0
MM_FP32_MIXED = 1
STATUS = {0: "MM_OK", 1: "MM_ERR_INVALID", 2: "MM_ERR_OOM", 3: "MM_ERR_CUDA",
          4: "MM_ERR_UNSUPPORTED", 5: "MM_ERR_TIMEOUT", 6: "MM_ERR_NONFINITE", 7: "MM_ERR_STATE"}
FIELD_NAMES = ("rho", "Px", "Py", "Qxx", "Qxy", "C", "Mf", "Fx", "Fy", "Sxx", "Sxy", "Syy")
SCALAR_NAMES = ("N_psi", "bound", "free", "motors", "polar_order", "mean_stress",
                "sum_psi_cos", "sum_psi_sin")


class MMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mm_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("ntheta", C.c_int), ("ns", C.c_int),
                ("L", C.c_double)]


class mm_rates(C.Structure):
    _fields_ = [("v_walk", C.c_double), ("k_on", C.c_double), ("k_off", C.c_double),
                ("glide", C.c_double), ("v_sp", C.c_double), ("force_scale", C.c_double),
                ("ell", C.c_double), ("cfl", C.c_double)]


class mm_moments_out(C.Structure):
    _fields_ = [("fields", C.c_void_p), ("fields_on_device", C.c_int),
                ("scalars", C.c_double * 8)]


class mm_batch_tune(C.Structure):
    _fields_ = [("tile_work", C.c_int), ("chunk_bytes", C.c_int), ("ms_per_substep", C.c_double),
                ("cells_per_warp", C.c_int)]


class mm_adjoint_seed(C.Structure):
    _fields_ = [("observable", C.c_int), ("dL_dpsi", C.c_void_p), ("dL_dnb", C.c_void_p),
                ("dL_dm1", C.c_void_p), ("dL_dmf", C.c_void_p), ("on_device", C.c_int),
                ("dL_dmb", C.c_void_p)]


class mm_adjoint_out(C.Structure):
    _fields_ = [("dL_du", C.c_void_p), ("du_capacity", C.c_int), ("dL_dpsi0", C.c_void_p),
                ("on_device", C.c_int),
                ("dL_drates", C.c_double * 3), ("value", C.c_double), ("n_velocities", C.c_int)]


OBSERVABLES = {"none": 0, "polar_order": 1, "mean_stress": 2}

# Every symbol include/mm.h declares, with its argument types.
_P = C.c_void_p
_H = C.c_void_p
PROTOTYPES = {
    "mm_create": ([C.POINTER(mm_grid), C.POINTER(mm_rates), C.c_int, _P, C.POINTER(C.c_void_p)], C.c_int),
    "mm_destroy": ([_H], C.c_int),
    "mm_set_stream": ([_H, _P], C.c_int),
    "mm_set_rates": ([_H, C.POINTER(mm_rates)], C.c_int),
    "mm_set_state": ([_H, _P, _P, _P, C.c_int], C.c_int),
    "mm_get_state": ([_H, _P, _P, _P, _P, C.c_int], C.c_int),
    "mm_set_velocity": ([_H, _P, C.c_int], C.c_int),
    "mm_snapshot_bytes": ([_H, C.POINTER(C.c_size_t)], C.c_int),
    "mm_save_snapshot": ([_H, _P, C.c_size_t, C.c_int], C.c_int),
    "mm_load_snapshot": ([_H, _P, C.c_size_t, C.c_int], C.c_int),
    "mm_get_dt": ([_H, C.POINTER(C.c_double)], C.c_int),
    "mm_set_dt": ([_H, C.c_double], C.c_int),
    "mm_micro_step": ([_H, C.c_int], C.c_int),
    "mm_moments": ([_H, C.POINTER(mm_moments_out)], C.c_int),
    "mm_set_checkpointing": ([_H, C.c_int, C.c_int], C.c_int),
    "mm_set_checkpointing_levels": ([_H, C.c_int, C.c_int, C.c_int], C.c_int),
    "mm_adjoint_step": ([_H, C.c_int, C.POINTER(mm_adjoint_seed), C.POINTER(mm_adjoint_out)],
                        C.c_int),
    "mm_sync": ([_H], C.c_int),
    "mm_diffuse": ([_H, C.c_double, C.c_double, C.c_double], C.c_int),
    "mm_motor_local": ([_H, C.c_double, _P, _P, C.c_int], C.c_int),
    "mm_set_anchors": ([_H, C.c_int], C.c_int),
    "mm_set_capture": ([_H, C.c_double], C.c_int),
    "mm_set_tangent": ([_H, _P], C.c_int),
    "mm_get_tangent": ([_H, _P, _P, _P, C.c_int], C.c_int),
    "mm_tangent_observable": ([_H, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
                              C.c_int),
    "mm_capture_template": ([_H, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int),
                             C.POINTER(C.c_int), C.POINTER(C.c_double)], C.c_int),
    "mm_fluid_setup": ([_H, C.c_double, C.c_double], C.c_int),
    "mm_fluid_solve": ([_H, _P, C.c_int, C.c_int, _P, C.c_int], C.c_int),
    "mm_fluid_response": ([_H, _P, C.c_int], C.c_int),
    "mm_debug_set": ([_H, C.c_uint, C.c_uint], C.c_int),
    "mm_get_launch_info": ([_H, C.POINTER(C.c_int), C.c_int], C.c_int),
    "mm_moments_static": ([C.POINTER(mm_grid), C.POINTER(mm_rates), _P, _P, _P, _P, _P, _P, _P],
                          C.c_int),
    "mm_create_batch": ([C.c_int, C.POINTER(mm_grid), C.POINTER(mm_rates), C.c_int, _P,
                         C.POINTER(_H)], C.c_int),
    "mm_batch_member": ([_H, C.c_int, C.POINTER(_H)], C.c_int),
    "mm_batch_autotune": ([_H, C.c_int, C.POINTER(mm_batch_tune), C.c_int,
                           C.POINTER(C.c_int)], C.c_int),
    "mm_last_error": ([_H], C.c_char_p),
    "mm_alu_peak": ([C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), _P], C.c_int),
    "mm_build_info": ([], C.c_char_p),
}

_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load libmm.so (raises if it has not been built). The environment
    variable MM_LIBRARY may name another build of the same library."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or os.environ.get("MM_LIBRARY") or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} is missing "
                                   "(run paper_1908_04279_gb300.build.build())")
            lib = C.CDLL(p)
            for name, (args, res) in PROTOTYPES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _ptr(a, what: str):
    """(pointer, on_device) for a numpy host array or a torch CUDA tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError(f"{what}: need a C-contiguous float64 array")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError(f"{what}: need a contiguous float64 tensor")
        if not a.is_cuda:
            return a.data_ptr(), 0
        return a.data_ptr(), 1
    raise TypeError(f"{what}: unsupported array type {type(a)}")


def _buf_ptr(a):
    """(pointer, on_device) of a uint8 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.uint8 or not a.flags.c_contiguous:
            raise TypeError("need a C-contiguous uint8 array")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise TypeError("need a contiguous tensor")
        return a.data_ptr(), int(bool(a.is_cuda))
    raise TypeError(f"unsupported buffer type {type(a)}")


def _buf_len(a) -> int:
    return int(a.nbytes) if isinstance(a, np.ndarray) else int(a.numel() * a.element_size())


def current_stream_handle() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # torch missing is fine: the legacy default stream is used
        pass
    return 0


class Simulation:
    """One simulation instance resident on the current CUDA device."""

    def __init__(self, grid: Grid, rates: Rates = Rates(), precision: str = "fp64",
                 stream: int | None = None, _member=None):
        self.lib = load_library()
        self.grid, self.rates = grid, rates
        self.precision = precision
        self._owned = _member is None
        if _member is not None:  # a batch member: the batch owns the handle
            self.h = _member
            return
        prec = {"fp64": MM_FP64, "fp32": MM_FP32_MIXED}[precision]
        h = C.c_void_p()
        st = self.lib.mm_create(C.byref(self._g()), C.byref(self._r(rates)), prec,
                                C.c_void_p(stream if stream is not None else current_stream_handle()),
                                C.byref(h))
        if st != 0:
            raise MMError(st, self.lib.mm_last_error(None).decode())
        self.h = h

    def _g(self):
        g = self.grid
        return mm_grid(g.nx, g.ny, g.ntheta, g.ns, g.L)

    @staticmethod
    def _r(r: Rates):
        return mm_rates(r.v_walk, r.k_on, r.k_off, r.glide, r.v_sp, r.force_scale, r.ell, r.cfl)

    def _check(self, st: int):
        if st != 0:
            raise MMError(st, self.lib.mm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                self.lib.mm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- state -------------------------------------------------------------
    def set_stream(self, stream: int):
        self._check(self.lib.mm_set_stream(self.h, C.c_void_p(stream)))

    def set_rates(self, rates: Rates):
        self.rates = rates
        self._check(self.lib.mm_set_rates(self.h, C.byref(self._r(rates))))

    def set_state(self, psi, mb=None, mtot=None):
        pp, d0 = _ptr(psi, "psi")
        pm, d1 = _ptr(mb, "mb")
        pt, d2 = _ptr(mtot, "mtot")
        flags = {d for d in (d0, d1, d2) if d is not None}
        if len(flags) > 1:
            raise TypeError("psi, mb and mtot must all be host arrays or all device tensors")
        self._check(self.lib.mm_set_state(self.h, pp, pm, pt, d0))

    def get_state(self):
        """Host copies: dict psi, mb, mf, c (float64); mb is [ny][nx][nconf]
        with a capture radius set (set_capture)."""
        g = self.grid
        tpl = getattr(self, "_capture", None)
        mshape = (g.ny, g.nx, tpl["nconf"]) if tpl else (g.ny, g.nx, g.ntheta, g.ns)
        out = dict(psi=np.empty((g.ny, g.nx, g.ntheta)), mb=np.empty(mshape),
                   mf=np.empty((g.ny, g.nx)), c=np.empty((g.ny, g.nx)))
        self._check(self.lib.mm_get_state(self.h, out["psi"].ctypes.data, out["mb"].ctypes.data,
                                          out["mf"].ctypes.data, out["c"].ctypes.data, 0))
        return out

    def get_state_into(self, psi=None, mb=None, mf=None, c=None):
        ptrs = [_ptr(a, n) for a, n in ((psi, "psi"), (mb, "mb"), (mf, "mf"), (c, "c"))]
        flags = {d for _, d in ptrs if d is not None}
        if len(flags) > 1:
            raise TypeError("outputs must all be host arrays or all device tensors")
        dev = flags.pop() if flags else 0
        self._check(self.lib.mm_get_state(self.h, *[p for p, _ in ptrs], dev))

    def set_velocity(self, u):
        p, d = _ptr(u, "u")
        self._check(self.lib.mm_set_velocity(self.h, p, d))

    @property
    def dt(self) -> float:
        v = C.c_double()
        self._check(self.lib.mm_get_dt(self.h, C.byref(v)))
        return v.value

    def set_dt(self, dt: float):
        self._check(self.lib.mm_set_dt(self.h, float(dt)))

    def step(self, n: int):
        self._check(self.lib.mm_micro_step(self.h, int(n)))

    def diffuse(self, D_t: float, D_r: float, dt: float):
        """One Crank-Nicolson step of filament diffusion (mm_diffuse)."""
        self._check(self.lib.mm_diffuse(self.h, float(D_t), float(D_r), float(dt)))

    def set_tangent(self, dparams=None):
        """Tangent-linear mode (mm_set_tangent): dparams = (d k_off, d v_walk,
        d k_on) switches it on (the tangent starts at zero), None off."""
        if dparams is None:
            self._check(self.lib.mm_set_tangent(self.h, None))
            return
        arr = (C.c_double * 3)(*[float(x) for x in dparams])
        self._check(self.lib.mm_set_tangent(self.h, C.cast(arr, C.c_void_p)))

    def get_tangent(self):
        """Host copies of the tangent: dict dpsi, dmb, dmf (float64)."""
        g = self.grid
        out = dict(dpsi=np.empty((g.ny, g.nx, g.ntheta)), dmb=np.empty((g.ny, g.nx, g.ntheta, g.ns)),
                   dmf=np.empty((g.ny, g.nx)))
        self._check(self.lib.mm_get_tangent(self.h, out["dpsi"].ctypes.data, out["dmb"].ctypes.data,
                                            out["dmf"].ctypes.data, 0))
        return out

    def tangent_observable(self, observable: str = "polar_order"):
        """(value, derivative along the tangent's direction) of a built-in
        observable of the current state (mm_tangent_observable)."""
        v, dv = C.c_double(), C.c_double()
        self._check(self.lib.mm_tangent_observable(self.h, OBSERVABLES[observable], C.byref(v),
                                                   C.byref(dv)))
        return v.value, dv.value

    def set_capture(self, r_c: float):
        """Finite capture radius (mm_set_capture): r_c >= 0 keeps the anchor
        axis of Mb (anchors within r_c of the motor head), r_c < 0 switches it
        off. Discards the motors. Returns the template (capture_template) or
        None."""
        self._check(self.lib.mm_set_capture(self.h, float(r_c)))
        self._capture = None
        if r_c >= 0:
            self._capture = self.capture_template()
        return self._capture

    def capture_template(self) -> dict:
        """{"lines": int [n][6] (k, dx, dy, j0, len, off), "nconf": int,
        "w": [ntheta][ns] = 1 / n_a} of the capture radius in effect."""
        g = self.grid
        nl, nconf = C.c_int(), C.c_int()
        self._check(self.lib.mm_capture_template(self.h, None, 0, C.byref(nl), C.byref(nconf),
                                                 None))
        lines = np.empty((nl.value, 6), dtype=np.int32)
        w = np.empty((g.ntheta, g.ns))
        self._check(self.lib.mm_capture_template(
            self.h, lines.ctypes.data_as(C.POINTER(C.c_int)), nl.value, C.byref(nl),
            C.byref(nconf), w.ctypes.data_as(C.POINTER(C.c_double))))
        return {"lines": lines, "nconf": nconf.value, "w": w}

    def set_anchors(self, enable: bool = True):
        """Non-local motor anchors (mm_set_anchors): each configuration anchored
        in the cell under its motor head, x + (l/L) s p with l/L = rates.ell."""
        self._check(self.lib.mm_set_anchors(self.h, 1 if enable else 0))

    def fluid_setup(self, eps: float, z0: float):
        """Thin-gap fluid solve of Eq. 7-9 (mm_fluid_setup): gap aspect eps,
        filament plane at z0 between no-slip plates at z = 0 and 1."""
        self._check(self.lib.mm_fluid_setup(self.h, float(eps), float(z0)))

    def fluid_solve(self, sigma=None, dipole: bool = False, u_out="host"):
        """u_2 on the filament plane from the motor force of the current state
        (plus -div sigma_a with dipole, plus div sigma of the caller's extra
        stress [3][ny][nx]); it becomes the velocity in effect. u_out: "host"
        returns a numpy [2][ny][nx], None returns nothing (no
        synchronisation), a float64 CUDA tensor receives it on the device."""
        g = self.grid
        sp, sd = _ptr(sigma, "sigma")
        if sigma is not None and tuple(sigma.shape) != (3, g.ny, g.nx):
            raise ValueError("sigma must have shape [3][ny][nx]")
        if isinstance(u_out, str):
            if u_out != "host":
                raise ValueError('u_out must be "host", None or a CUDA tensor')
            out = np.empty((2, g.ny, g.nx))
            self._check(self.lib.mm_fluid_solve(self.h, sp, sd or 0, int(bool(dipole)),
                                                out.ctypes.data, 0))
            return out
        up, ud = _ptr(u_out, "u_out")
        if u_out is not None and (not ud or tuple(u_out.shape) != (2, g.ny, g.nx)):
            raise TypeError("u_out must be a float64 CUDA tensor [2][ny][nx]")
        self._check(self.lib.mm_fluid_solve(self.h, sp, sd or 0, int(bool(dipole)), up, ud or 0))
        return None

    def fluid_response(self) -> np.ndarray:
        """The per-mode response table [ny][nx//2 + 1][2] (g_T, g_L)."""
        g = self.grid
        out = np.empty((g.ny, g.nx // 2 + 1, 2))
        self._check(self.lib.mm_fluid_response(self.h, out.ctypes.data, 0))
        return out

    def motor_local(self, T: float, nsteps=None):
        """Motor kinetics over T with psi frozen and a local substep per cell
        (mm_motor_local). nsteps (int array [ny][nx], optional) imposes the
        substeps per cell. Returns the substeps used per cell (host int32)."""
        g = self.grid
        out = np.empty((g.ny, g.nx), dtype=np.int32)
        nin = None
        if nsteps is not None:
            nin = np.ascontiguousarray(nsteps, dtype=np.int32)
            if nin.shape != (g.ny, g.nx):
                raise ValueError("nsteps must have shape [ny][nx]")
        self._check(self.lib.mm_motor_local(self.h, float(T),
                                            nin.ctypes.data if nin is not None else None,
                                            out.ctypes.data, 0))
        return out

    def motor_local_device(self, T: float, nsteps_out=None):
        """mm_motor_local with the counts (optional) written to an int32 CUDA
        tensor of ncells; stream-ordered, no synchronisation."""
        p = None
        if nsteps_out is not None:
            import torch
            if nsteps_out.dtype != torch.int32 or not nsteps_out.is_cuda:
                raise TypeError("nsteps_out must be an int32 CUDA tensor")
            p = nsteps_out.data_ptr()
        self._check(self.lib.mm_motor_local(self.h, float(T), None, p, 1))

    def sync(self):
        self._check(self.lib.mm_sync(self.h))

    # ---- adjoint -------------------------------------------------------------
    def set_checkpointing(self, K: int, max_substeps: int, K_inner: int | None = None):
        """Start an adjoint recording at the current state, with checkpoints
        every K substeps (and, with K_inner < K, inner checkpoints every
        K_inner substeps rebuilt during the reverse sweep). K = 0 ends it and
        frees its memory; set_state ends it and keeps the memory, which a new
        recording of the same shape reuses."""
        Ki = K if K_inner is None else K_inner
        self._check(self.lib.mm_set_checkpointing_levels(self.h, int(K), int(Ki),
                                                         int(max_substeps)))

    def adjoint(self, n_substeps: int, observable: str = "none", dL_dpsi=None, dL_dnb=None,
                dL_dm1=None, dL_dmf=None, n_velocities: int = 1, want_du: bool = True,
                want_dpsi0: bool = True, out_du=None, out_dpsi0=None, dL_dmb=None):
        """Reverse sweep over the recorded substeps. Seeds are float64 arrays
        (numpy, or CUDA tensors; psi-shaped for dL_dpsi/dL_dnb/dL_dm1, [ny][nx]
        for dL_dmf, [ny][nx][ntheta][ns] for dL_dmb) or a built-in observable. Returns a dict: value, dL_drates
        (k_off, v_walk, k_on), dL_du [n_velocities][2][ny][nx], dL_dpsi0.
        With out_du / out_dpsi0 (float64 CUDA tensors of those shapes) the
        gradients are written there on the device instead of to new host
        arrays."""
        g = self.grid
        seeds = [dL_dpsi, dL_dnb, dL_dm1, dL_dmf, dL_dmb]
        shapes = [(g.ny, g.nx, g.ntheta)] * 3 + [(g.ny, g.nx), (g.ny, g.nx, g.ntheta, g.ns)]
        for a, shp in zip(seeds, shapes):
            if a is not None and tuple(a.shape) != shp:
                raise ValueError(f"seed of shape {tuple(a.shape)}, expected {shp}")
        kept = [np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a
                for a in seeds]
        ptrs = [_ptr(a, "seed") for a in kept]
        devs = {d for _, d in ptrs if d is not None}
        if len(devs) > 1:
            raise TypeError("seeds must all be host arrays or all device tensors")
        sd = mm_adjoint_seed(OBSERVABLES[observable], *[p for p, _ in ptrs[:4]],
                             devs.pop() if devs else 0, ptrs[4][0])
        if out_du is not None or out_dpsi0 is not None:
            pu, du_dev = _ptr(out_du, "out_du")
            pp, dp_dev = _ptr(out_dpsi0, "out_dpsi0")
            if {d for d in (du_dev, dp_dev) if d is not None} != {1}:
                raise TypeError("out_du and out_dpsi0 must be CUDA tensors")
            cap = out_du.shape[0] if out_du is not None else 0
            if out_du is not None and tuple(out_du.shape) != (cap, 2, g.ny, g.nx):
                raise ValueError("out_du must have shape [n][2][ny][nx]")
            if out_dpsi0 is not None and tuple(out_dpsi0.shape) != (g.ny, g.nx, g.ntheta):
                raise ValueError("out_dpsi0 must have shape [ny][nx][ntheta]")
            out = mm_adjoint_out(pu, cap, pp, 1)
            self._check(self.lib.mm_adjoint_step(self.h, int(n_substeps), C.byref(sd),
                                                 C.byref(out)))
            return dict(value=out.value, dL_drates=np.array(list(out.dL_drates)), dL_du=out_du,
                        dL_dpsi0=out_dpsi0, n_velocities=out.n_velocities)
        du = np.empty((n_velocities, 2, g.ny, g.nx)) if want_du else None
        dp = np.empty((g.ny, g.nx, g.ntheta)) if want_dpsi0 else None
        out = mm_adjoint_out(du.ctypes.data if du is not None else None, n_velocities,
                             dp.ctypes.data if dp is not None else None, 0)
        self._check(self.lib.mm_adjoint_step(self.h, int(n_substeps), C.byref(sd), C.byref(out)))
        if du is not None:
            du = du[:out.n_velocities]
        return dict(value=out.value, dL_drates=np.array(list(out.dL_drates)), dL_du=du,
                    dL_dpsi0=dp, n_velocities=out.n_velocities)

    def snapshot_bytes(self) -> int:
        """Bytes of a snapshot of this handle (mm_snapshot_bytes)."""
        n = C.c_size_t()
        self._check(self.lib.mm_snapshot_bytes(self.h, C.byref(n)))
        return n.value

    def snapshot(self, out=None):
        """Bitwise snapshot of the state (mm_save_snapshot): into `out` (a
        uint8 numpy array or CUDA tensor of at least snapshot_bytes() bytes),
        or a new host uint8 array. Returns the buffer."""
        if out is None:
            out = np.empty(self.snapshot_bytes(), dtype=np.uint8)
        p, dev = _buf_ptr(out)
        self._check(self.lib.mm_save_snapshot(self.h, p, _buf_len(out), dev))
        return out

    def load_snapshot(self, buf):
        """Continue from a snapshot of a handle of the same grid and precision
        (mm_load_snapshot); buf as returned by snapshot()."""
        p, dev = _buf_ptr(buf)
        self._check(self.lib.mm_load_snapshot(self.h, p, _buf_len(buf), dev))

    def debug_set(self, wait_limit: int, flags: int = 0):
        self._check(self.lib.mm_debug_set(self.h, int(wait_limit), int(flags)))

    def launch_info(self) -> dict:
        arr = (C.c_int * 10)()
        self._check(self.lib.mm_get_launch_info(self.h, arr, 10))
        keys = ("grid", "block", "smem", "tma", "stages", "chunk_rows", "chunks_per_cell", "V",
                "seg", "sms")
        return dict(zip(keys, list(arr)))

    def moments(self, fields=True):
        """(fields dict name -> [ny][nx] or None, scalars dict). `fields` may be
        True (host numpy), False, or a float64 CUDA tensor of 12*ny*nx."""
        g = self.grid
        out = mm_moments_out()
        host = None
        if fields is True:
            host = np.empty((12, g.ny, g.nx))
            out.fields, out.fields_on_device = host.ctypes.data, 0
        elif fields is not False and fields is not None:
            p, d = _ptr(fields, "fields")
            out.fields, out.fields_on_device = p, d
        self._check(self.lib.mm_moments(self.h, C.byref(out)))
        sc = dict(zip(SCALAR_NAMES, list(out.scalars)))
        return (dict(zip(FIELD_NAMES, host)) if host is not None else None), sc


class Batch:
    """An ensemble of independent instances advanced together: one launch per
    substep over all members, the substeps of one step() call in one CUDA
    graph (mm_create_batch). members[i] is a Simulation view of instance i
    for its per-instance calls (set_state, set_velocity, moments, adjoint)."""

    def __init__(self, grids, rates, precision: str = "fp32", stream: int | None = None):
        self.lib = load_library()
        n = len(grids)
        if len(rates) != n:
            raise ValueError("one Rates per grid")
        ga = (mm_grid * n)(*[mm_grid(g.nx, g.ny, g.ntheta, g.ns, g.L) for g in grids])
        ra = (mm_rates * n)(*[Simulation._r(r) for r in rates])
        prec = {"fp64": MM_FP64, "fp32": MM_FP32_MIXED}[precision]
        h = C.c_void_p()
        st = self.lib.mm_create_batch(n, ga, ra, prec,
                                      C.c_void_p(stream if stream is not None
                                                 else current_stream_handle()), C.byref(h))
        if st != 0:
            raise MMError(st, self.lib.mm_last_error(None).decode())
        self.h = h
        self.members = []
        for i in range(n):
            m = C.c_void_p()
            self._check(self.lib.mm_batch_member(self.h, i, C.byref(m)))
            self.members.append(Simulation(grids[i], rates[i], precision, _member=m))

    def _check(self, st: int):
        if st != 0:
            raise MMError(st, self.lib.mm_last_error(self.h).decode())

    def step(self, n: int):
        self._check(self.lib.mm_micro_step(self.h, int(n)))

    def diffuse(self, D_t: float, D_r: float, dt: float):
        """One Crank-Nicolson step of filament diffusion (mm_diffuse)."""
        self._check(self.lib.mm_diffuse(self.h, float(D_t), float(D_r), float(dt)))

    def sync(self):
        self._check(self.lib.mm_sync(self.h))

    def debug_set(self, wait_limit: int, flags: int = 0):
        self._check(self.lib.mm_debug_set(self.h, int(wait_limit), int(flags)))

    def autotune(self, substeps: int = 5):
        """Time every (tile_work, chunk_bytes, cells per warp) candidate; keep
        the fastest. Returns the list of timings."""
        res = (mm_batch_tune * 64)()
        n = C.c_int()
        self._check(self.lib.mm_batch_autotune(self.h, int(substeps), res, 64, C.byref(n)))
        return [dict(tile_work=r.tile_work, chunk_bytes=r.chunk_bytes,
                     cells_per_warp=r.cells_per_warp, ms_per_substep=r.ms_per_substep)
                for r in res[:n.value]]

    def launch_info(self) -> dict:
        arr = (C.c_int * 12)()
        self._check(self.lib.mm_get_launch_info(self.h, arr, 12))
        keys = ("grid", "block", "smem", "tma", "stages", "stage_elems", "tiles", "V",
                "tile_work", "chunk_bytes", "tuned", "pair_cells")
        return dict(zip(keys, list(arr)))

    @property
    def cell_updates_per_substep(self) -> int:
        return sum(m.grid.micro_cells for m in self.members)

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            self.lib.mm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def moments_static(grid: Grid, rates: Rates, psi, mb, mf, c, fields, scalars, stream: int = 0):
    """Allocation-free moments of a caller-held float64 device state (see
    mm_moments_static in include/mm.h); all arrays are CUDA tensors."""
    lib = load_library()
    ptrs = [_ptr(a, n) for a, n in ((psi, "psi"), (mb, "mb"), (mf, "mf"), (c, "c"),
                                    (scalars, "scalars"))]
    if any(d != 1 for _, d in ptrs):
        raise TypeError("mm_moments_static takes device arrays only")
    fp, fd = _ptr(fields, "fields")
    if fields is not None and fd != 1:
        raise TypeError("fields must be a device array")
    g = mm_grid(grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L)
    r = Simulation._r(rates)
    st = lib.mm_moments_static(C.byref(g), C.byref(r), ptrs[0][0], ptrs[1][0], ptrs[2][0],
                               ptrs[3][0], fp, ptrs[4][0], C.c_void_p(stream))
    if st != 0:
        raise MMError(st, lib.mm_last_error(None).decode())


ALU_KINDS = {"fp64": 0, "fp32": 1, "fp32x2": 2}


def alu_peak(kind: str, stream: int = 0) -> dict:
    """Measured fused multiply-add rate of the current device (mm_alu_peak):
    kind "fp64", "fp32" or "fp32x2" (packed, each instruction counted as two).
    Returns {"fma_per_s", "ms_per_launch"}."""
    lib = load_library()
    rate, ms = C.c_double(), C.c_double()
    st = lib.mm_alu_peak(ALU_KINDS[kind], C.byref(rate), C.byref(ms), C.c_void_p(stream))
    if st != 0:
        raise MMError(st, lib.mm_last_error(None).decode())
    return {"fma_per_s": rate.value, "ms_per_launch": ms.value}


def build_info() -> str:
    return load_library().mm_build_info().decode()
