"""ctypes front end of the FP64 CPU oracle (mm_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. Nothing here is shared with the CUDA
path; the oracle library is compiled from its own C source with gcc
(-O2, no fast-math, no floating-point contraction, so x86 and Arm hosts give
the same results).

All arrays are float64 numpy arrays in the layouts of mm_oracle.c:
psi [ny][nx][nth], mb [ny][nx][nth][ns], u [2][ny][nx], mf/c/mtot [ny][nx].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library in-tree (oracle/_build/liboracle.so)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nth", C.c_int), ("ns", C.c_int),
                ("L", C.c_double), ("lx", C.c_double), ("ly", C.c_double)]


class _Rates(C.Structure):
    _fields_ = [("v_walk", C.c_double), ("k_on", C.c_double), ("k_off", C.c_double),
                ("glide", C.c_double), ("v_sp", C.c_double), ("force_scale", C.c_double),
                ("ell", C.c_double), ("cfl", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(C.c_double)
            G, R = C.POINTER(_Grid), C.POINTER(_Rates)
            lib.or_dt.argtypes = [G, R, P, P, P, P]
            lib.or_init_free.argtypes = [G, P, P, P, P, P]
            lib.or_substep.argtypes = [G, R, C.c_double, P, P, P, P, P, P]
            lib.or_run.argtypes = [G, R, C.c_double, P, P, P, P, P, P, C.c_int]
            lib.or_moments.argtypes = [G, R, P, P, P, P, P, P]
            lib.or_tangent_substep.argtypes = [G, R, C.c_double, P, P, P, P, P, P, P, P, P, P]
            lib.or_adjoint_substep.argtypes = [G, R, C.c_double, P, P, P, P, P, P, P, P, P, P]
            IP = C.POINTER(C.c_int)
            lib.or_motor_local.argtypes = [G, R, C.c_double, P, P, P, P, P, IP, IP]
            lib.or_init_free_anchor.argtypes = [G, R, P, P, P, P, P]
            lib.or_substep_anchor.argtypes = [G, R, C.c_double, P, P, P, P, P, P]
            lib.or_anchor_force.argtypes = [G, R, P, P, P]
            lib.or_anchor_offsets.argtypes = [G, R, IP, IP]
            D = C.c_double
            lib.or_rc_template.argtypes = [G, R, D, IP, C.c_int, IP, IP, P]
            lib.or_init_free_rc.argtypes = [G, R, D, P, P, P, P, P]
            lib.or_rc_rows.argtypes = [G, R, D, P, P, P]
            lib.or_substep_rc.argtypes = [G, R, D, D, P, P, P, P, P, P]
            lib.or_rc_force.argtypes = [G, R, D, P, P, P]
            lib.or_moments_rc.argtypes = [G, R, D, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _grid(g) -> _Grid:
    return _Grid(g.nx, g.ny, g.ntheta, g.ns, g.L, getattr(g, "lx", 1.0), getattr(g, "ly", 1.0))


@dataclass(frozen=True)
class PatchGrid:
    """Grid of a periodic patch cut out of a larger grid (same dx, dy)."""

    nx: int
    ny: int
    ntheta: int
    ns: int
    L: float
    lx: float
    ly: float


def _rates(r) -> _Rates:
    return _Rates(r.v_walk, r.k_on, r.k_off, r.glide, r.v_sp, r.force_scale, r.ell, r.cfl)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


FIELD_NAMES = ("rho", "Px", "Py", "Qxx", "Qxy", "C", "Mf", "Fx", "Fy", "Sxx", "Sxy", "Syy")
SCALAR_NAMES = ("N_psi", "bound", "free", "motors", "polar_order", "mean_stress",
                "sum_psi_cos", "sum_psi_sin")


@dataclass
class State:
    """Oracle state: psi, mb, mf, c and the fixed total motor density mtot."""

    grid: object
    psi: np.ndarray
    mb: np.ndarray
    mf: np.ndarray
    c: np.ndarray
    mtot: np.ndarray

    def copy(self) -> "State":
        return State(self.grid, self.psi.copy(), self.mb.copy(), self.mf.copy(), self.c.copy(),
                     self.mtot.copy())


def make_state(grid, psi, mb=None, mtot=None) -> State:
    """Set up a state: Mb (default 0), M (default 1), then C, the Alg. 2 clip
    and Mf = M - C."""
    g = grid
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(g.ny, g.nx, g.ntheta).copy()
    mb = (np.zeros((g.ny, g.nx, g.ntheta, g.ns)) if mb is None
          else np.ascontiguousarray(mb, dtype=np.float64).reshape(g.ny, g.nx, g.ntheta, g.ns).copy())
    mtot = (np.ones((g.ny, g.nx)) if mtot is None
            else np.ascontiguousarray(mtot, dtype=np.float64).reshape(g.ny, g.nx).copy())
    mf = np.empty((g.ny, g.nx))
    c = np.empty((g.ny, g.nx))
    _check(_load().or_init_free(C.byref(_grid(g)), _p(psi), _p(mb), _p(mtot), _p(mf), _p(c)),
           "init_free")
    return State(g, psi, mb, mf, c, mtot)


def dt(grid, rates, state: State, u: np.ndarray) -> float:
    out = C.c_double(0.0)
    u = np.ascontiguousarray(u, dtype=np.float64)
    _check(_load().or_dt(C.byref(_grid(grid)), C.byref(_rates(rates)), _p(state.psi),
                         _p(state.mb), _p(u), C.byref(out)), "dt")
    return out.value


def run(grid, rates, state: State, u: np.ndarray, dt_: float, nsub: int) -> State:
    """Advance nsub substeps in place; returns the same state object."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    _check(_load().or_run(C.byref(_grid(grid)), C.byref(_rates(rates)), float(dt_), _p(u),
                          _p(state.psi), _p(state.mb), _p(state.mf), _p(state.c),
                          _p(state.mtot), int(nsub)), "run")
    return state


def moments(grid, rates, state: State):
    """Returns (fields dict name -> [ny][nx], scalars dict)."""
    g = grid
    f = np.empty((12, g.ny, g.nx))
    s = np.empty(8)
    _check(_load().or_moments(C.byref(_grid(g)), C.byref(_rates(rates)), _p(state.psi),
                              _p(state.mb), _p(state.mf), _p(state.c), _p(f), _p(s)), "moments")
    return dict(zip(FIELD_NAMES, f)), dict(zip(SCALAR_NAMES, s))


def tangent_substep(grid, rates, dt_, u, du, dparams, state: State, dpsi, dmb, dmf):
    """Tangent of one substep at `state` (not modified); dpsi/dmb/dmf updated in place.
    dparams = (d k_off, d v_walk, d k_on)."""
    dp = np.ascontiguousarray(dparams, dtype=np.float64)
    _check(_load().or_tangent_substep(
        C.byref(_grid(grid)), C.byref(_rates(rates)), float(dt_),
        _p(np.ascontiguousarray(u, dtype=np.float64)), _p(np.ascontiguousarray(du, dtype=np.float64)),
        _p(dp), _p(state.psi), _p(state.mb), _p(state.mf), _p(state.mtot), _p(dpsi), _p(dmb),
        _p(dmf)), "tangent")


def adjoint_substep(grid, rates, dt_, u, state: State, lpsi, lmb, lmf, lu, lp):
    """Adjoint of one substep at `state` (state at step n, not modified).
    lpsi/lmb/lmf: adjoint at n+1 in, at n out. lu [2][ny][nx] and
    lp (k_off, v_walk, k_on) accumulate."""
    _check(_load().or_adjoint_substep(
        C.byref(_grid(grid)), C.byref(_rates(rates)), float(dt_),
        _p(np.ascontiguousarray(u, dtype=np.float64)), _p(state.psi), _p(state.mb), _p(state.mf),
        _p(state.mtot), _p(lpsi), _p(lmb), _p(lmf), _p(lu), _p(lp)), "adjoint")


def substep_states(grid, rates, state: State, u, dt_, nsub: int) -> list[State]:
    """States 0..nsub of a trajectory (for the adjoint sweep)."""
    out = [state.copy()]
    cur = state.copy()
    for _ in range(nsub):
        run(grid, rates, cur, u, dt_, 1)
        out.append(cur.copy())
    return out


def adjoint(grid, rates, state0: State, u, dt_, nsub: int, lpsi, lmb, lmf):
    """Reverse sweep over nsub substeps from state0 (all states stored).
    Returns (lpsi0, lmb0, lmf0, lu, lp)."""
    states = substep_states(grid, rates, state0, u, dt_, nsub)
    lpsi = np.array(lpsi, dtype=np.float64, copy=True)
    lmb = np.array(lmb, dtype=np.float64, copy=True)
    lmf = np.array(lmf, dtype=np.float64, copy=True)
    lu = np.zeros((2, grid.ny, grid.nx))
    lp = np.zeros(3)
    for n in range(nsub - 1, -1, -1):
        adjoint_substep(grid, rates, dt_, u, states[n], lpsi, lmb, lmf, lu, lp)
    return lpsi, lmb, lmf, lu, lp


def patch_substep(grid, rates, dt_, u, psi, mb, mf, mtot, cells):
    """One substep for selected cells only, each evaluated on the 3x3 periodic
    patch around it (one substep reads only a cell's 4 neighbours, so the
    patch centre equals the full-grid result). psi/mb/mf/mtot/u are the full
    float64 arrays (numpy, any layout-compatible view); cells is a list of
    (iy, ix). Returns a list of dicts psi [nth], mb [nth][ns], mf, c."""
    g = grid
    pg = PatchGrid(3, 3, g.ntheta, g.ns, g.L, 3.0 / g.nx, 3.0 / g.ny)
    out = []
    for iy, ix in cells:
        ys = [(iy + d) % g.ny for d in (-1, 0, 1)]
        xs = [(ix + d) % g.nx for d in (-1, 0, 1)]
        sel = np.ix_(ys, xs)
        st = State(pg, np.ascontiguousarray(psi[sel]), np.ascontiguousarray(mb[sel]),
                   np.ascontiguousarray(mf[sel]), np.zeros((3, 3)), np.ascontiguousarray(mtot[sel]))
        uu = np.ascontiguousarray(np.stack([u[0][sel], u[1][sel]]))
        run(pg, rates, st, uu, dt_, 1)
        out.append(dict(psi=st.psi[1, 1].copy(), mb=st.mb[1, 1].copy(), mf=float(st.mf[1, 1]),
                        c=float(st.c[1, 1])))
    return out


def _cn_factor(n: int, a: float) -> tuple[np.ndarray, np.ndarray]:
    """Dense matrices (I - a/2 L, I + a/2 L) of one Crank-Nicolson step along a
    periodic line of n points, L the periodic second difference
    (L psi)_i = psi_{i-1} - 2 psi_i + psi_{i+1} (indices mod n), a = D dt / h^2."""
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] -= 2.0
        L[i, (i - 1) % n] += 1.0
        L[i, (i + 1) % n] += 1.0
    eye = np.eye(n)
    return eye - 0.5 * a * L, eye + 0.5 * a * L


def diffuse(grid, psi, D_t: float, D_r: float, dt: float) -> np.ndarray:
    """One step of filament diffusion, the -D_t grad ln psi and
    -D_r d_theta ln psi fluxes of Eq. 2-3 (d_t psi = D_t lap_x psi +
    D_r d_theta^2 psi), by Crank-Nicolson (Sec. 2, Alg. 1: the diffusive terms
    of the psi update) applied one direction at a time -- theta, then x, then
    y -- each a periodic second difference (h = dtheta, dx = 1/nx, dy = 1/ny)
    solved exactly with a dense linear solve. psi is [ny][nx][nth]; returns
    the new array."""
    g = grid
    out = np.array(psi, dtype=np.float64, copy=True)
    for axis, n, h, D in ((2, g.ntheta, 2 * np.pi / g.ntheta, D_r), (1, g.nx, 1.0 / g.nx, D_t),
                          (0, g.ny, 1.0 / g.ny, D_t)):
        if D == 0.0:
            continue
        A, B = _cn_factor(n, D * dt / (h * h))
        lines = np.moveaxis(out, axis, -1)  # [..., n]
        flat = lines.reshape(-1, n)
        new = np.linalg.solve(A, B @ flat.T).T
        out = np.moveaxis(new.reshape(lines.shape), -1, axis)
    return np.ascontiguousarray(out)


def motor_local(grid, rates, state: State, T: float, nsteps=None) -> np.ndarray:
    """Motor kinetics over T with psi frozen and a local substep per cell
    (or_motor_local), in place; nsteps (int array [ny][nx], optional) imposes
    the substeps per cell. Returns the substeps used per cell."""
    out = np.zeros((grid.ny, grid.nx), dtype=np.int32)
    IP = C.POINTER(C.c_int)
    nin = None
    if nsteps is not None:
        nin = np.ascontiguousarray(nsteps, dtype=np.int32)
    _check(_load().or_motor_local(C.byref(_grid(grid)), C.byref(_rates(rates)), float(T),
                                  _p(state.psi), _p(state.mb), _p(state.mf), _p(state.c),
                                  _p(state.mtot),
                                  nin.ctypes.data_as(IP) if nin is not None else None,
                                  out.ctypes.data_as(IP)), "motor_local")
    return out


# ---- non-local motor anchors (next row f2)


def make_state_anchor(grid, rates, psi, mb=None, mtot=None) -> State:
    """make_state with the anchors kept: C at each anchor cell (the cell under
    the motor head x + (l/L) s p), the Alg. 2 scale-down per anchor, Mf."""
    g = grid
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(g.ny, g.nx, g.ntheta).copy()
    mb = (np.zeros((g.ny, g.nx, g.ntheta, g.ns)) if mb is None
          else np.ascontiguousarray(mb, dtype=np.float64).reshape(g.ny, g.nx, g.ntheta, g.ns).copy())
    mtot = (np.ones((g.ny, g.nx)) if mtot is None
            else np.ascontiguousarray(mtot, dtype=np.float64).reshape(g.ny, g.nx).copy())
    mf = np.empty((g.ny, g.nx))
    c = np.empty((g.ny, g.nx))
    _check(_load().or_init_free_anchor(C.byref(_grid(g)), C.byref(_rates(rates)), _p(psi), _p(mb),
                                       _p(mtot), _p(mf), _p(c)), "init_free_anchor")
    return State(g, psi, mb, mf, c, mtot)


def run_anchor(grid, rates, state: State, u: np.ndarray, dt_: float, nsub: int) -> State:
    """nsub substeps with the anchors kept (or_substep_anchor), in place."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    lib = _load()
    for _ in range(nsub):
        _check(lib.or_substep_anchor(C.byref(_grid(grid)), C.byref(_rates(rates)), float(dt_),
                                     _p(u), _p(state.psi), _p(state.mb), _p(state.mf),
                                     _p(state.c), _p(state.mtot)), "substep_anchor")
    return state


def anchor_force(grid, rates, state: State) -> np.ndarray:
    """Motor force of Eq. 10 acting at the anchors, [2][ny][nx]."""
    F = np.empty((2, grid.ny, grid.nx))
    _check(_load().or_anchor_force(C.byref(_grid(grid)), C.byref(_rates(rates)), _p(state.psi),
                                   _p(state.mb), _p(F)), "anchor_force")
    return F


def anchor_offsets(grid, rates):
    """(ox, oy) int arrays [ntheta][ns]: the anchor cell offsets."""
    ox = np.empty((grid.ntheta, grid.ns), dtype=np.int32)
    oy = np.empty((grid.ntheta, grid.ns), dtype=np.int32)
    IP = C.POINTER(C.c_int)
    _check(_load().or_anchor_offsets(C.byref(_grid(grid)), C.byref(_rates(rates)),
                                     ox.ctypes.data_as(IP), oy.ctypes.data_as(IP)), "anchor_offsets")
    return ox, oy


# ---- finite capture radius: the anchor axis of Mb (next row f2)


@dataclass
class RcTemplate:
    """The configurations of B_rc(r0), the same for every anchor r0: lines
    [n][6] = (k, dx, dy, j0, len, off) -- the motors of anchor r0 on a filament
    of orientation k centred at r0 - (dx, dy) cells, at nodes j0..j0+len-1,
    stored from entry off of mb[r0][] -- and w [ntheta][ns] = 1 / n_a."""

    lines: np.ndarray
    nconf: int
    w: np.ndarray


def rc_template(grid, rates, rc: float) -> RcTemplate:
    IP = C.POINTER(C.c_int)
    nl, nconf = C.c_int(0), C.c_int(0)
    w = np.empty((grid.ntheta, grid.ns))
    lib = _load()
    _check(lib.or_rc_template(C.byref(_grid(grid)), C.byref(_rates(rates)), float(rc), None, 0,
                              C.byref(nl), C.byref(nconf), _p(w)), "rc_template")
    lines = np.empty((nl.value, 6), dtype=np.int32)
    _check(lib.or_rc_template(C.byref(_grid(grid)), C.byref(_rates(rates)), float(rc),
                              lines.ctypes.data_as(IP), nl.value, C.byref(nl), C.byref(nconf),
                              _p(w)), "rc_template")
    return RcTemplate(lines, nconf.value, w)


def make_state_rc(grid, rates, rc: float, psi, mb=None, mtot=None) -> State:
    """A state of the capture-radius model: mb [ny][nx][nconf] (anchor-major,
    template order; default 0), then C, the scale-down and Mf per anchor."""
    g = grid
    nconf = rc_template(g, rates, rc).nconf
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(g.ny, g.nx, g.ntheta).copy()
    mb = (np.zeros((g.ny, g.nx, nconf)) if mb is None
          else np.ascontiguousarray(mb, dtype=np.float64).reshape(g.ny, g.nx, nconf).copy())
    mtot = (np.ones((g.ny, g.nx)) if mtot is None
            else np.ascontiguousarray(mtot, dtype=np.float64).reshape(g.ny, g.nx).copy())
    mf = np.empty((g.ny, g.nx))
    c = np.empty((g.ny, g.nx))
    _check(_load().or_init_free_rc(C.byref(_grid(g)), C.byref(_rates(rates)), float(rc), _p(psi),
                                   _p(mb), _p(mtot), _p(mf), _p(c)), "init_free_rc")
    return State(g, psi, mb, mf, c, mtot)


def run_rc(grid, rates, rc: float, state: State, u: np.ndarray, dt_: float, nsub: int) -> State:
    """nsub substeps of the capture-radius model (or_substep_rc), in place."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    lib = _load()
    for _ in range(nsub):
        _check(lib.or_substep_rc(C.byref(_grid(grid)), C.byref(_rates(rates)), float(rc),
                                 float(dt_), _p(u), _p(state.psi), _p(state.mb), _p(state.mf),
                                 _p(state.c), _p(state.mtot)), "substep_rc")
    return state


def rows_rc(grid, rates, rc: float, state: State):
    """(n_b, m1) per (x, theta) of a capture-radius state, [ny][nx][ntheta]."""
    nb = np.empty((grid.ny, grid.nx, grid.ntheta))
    m1 = np.empty((grid.ny, grid.nx, grid.ntheta))
    _check(_load().or_rc_rows(C.byref(_grid(grid)), C.byref(_rates(rates)), float(rc),
                              _p(state.mb), _p(nb), _p(m1)), "rc_rows")
    return nb, m1


def force_rc(grid, rates, rc: float, state: State) -> np.ndarray:
    """Motor force of Eq. 10 at the heads of a capture-radius state, [2][ny][nx]."""
    F = np.empty((2, grid.ny, grid.nx))
    _check(_load().or_rc_force(C.byref(_grid(grid)), C.byref(_rates(rates)), float(rc),
                               _p(state.psi), _p(state.mb), _p(F)), "rc_force")
    return F


def moments_rc(grid, rates, rc: float, state: State):
    """moments() of a capture-radius state (n_b, m1 over the anchors, the force
    at the heads)."""
    g = grid
    f = np.empty((12, g.ny, g.nx))
    s = np.empty(8)
    _check(_load().or_moments_rc(C.byref(_grid(g)), C.byref(_rates(rates)), float(rc),
                                 _p(state.psi), _p(state.mb), _p(state.mf), _p(state.c), _p(f),
                                 _p(s)), "moments_rc")
    return dict(zip(FIELD_NAMES, f)), dict(zip(SCALAR_NAMES, s))
