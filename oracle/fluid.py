"""Float64 CPU oracle of the thin-gap fluid solve (Eq. 7-9), numpy + scipy.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. Nothing here is shared with the CUDA
path.

The fluid fills the gap 0 <= z <= 1 between two no-slip plates and is periodic
in x and y over the unit square (Sec. 2). The filaments and bound motors lie on
the plane z = z0 near the bottom plate (Sec. 2: a Dirac delta in z about that
plane), so the right side of Eq. 7 is (F_2 + div_2 Sigma) delta(z - z0), with
F_2 the motor force of Eq. 10 and Sigma the in-plane extra stress
(Sigma = sigma_f S_f - sigma_t S_t; its constitutive law is not part of the
paper, it is an input here). The filaments are advected by u_2 on that plane.

Per Fourier mode k = (kx, ky) of |k| = kappa the transformed Eq. 7-9 split
into the part of u_2 across k (no pressure) and the part along k, coupled to w
and the pressure q. Both are linear ODE boundary value problems in z with
constant coefficients; they are solved here exactly (up to rounding) by
multiple shooting: the propagator of the first-order system over each short
interval is a matrix exponential (scipy.linalg.expm), and the interval states,
the jump at z0 and the wall conditions form one sparse linear system.

The z-grid of the paper (adaptive, fine near z0; Sec. 2) is replaced by this
exact solve, its limit under refinement.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg


def _shoot(M: np.ndarray, jump: np.ndarray, wall: list[int], z0: float, hmax: float,
           out: int) -> float:
    """Solve Y' = M Y on (0, z0) and (z0, 1) with Y(z0+) - Y(z0-) = jump and
    the components `wall` of Y zero at z = 0 and z = 1; returns Y(z0)[out]
    (a component continuous at z0).

    Unknowns: the states at the nodes of [0, z0] (n1 intervals) and of
    [z0, 1] (n2 intervals). Equations: Y_{j+1} = expm(M h) Y_j on every
    interval, the jump at z0, and the wall conditions."""
    d = M.shape[0]
    n1 = max(1, math.ceil(z0 / hmax))
    n2 = max(1, math.ceil((1.0 - z0) / hmax))
    E1 = scipy.linalg.expm(M * (z0 / n1))
    E2 = scipy.linalg.expm(M * ((1.0 - z0) / n2))
    nodes = (n1 + 1) + (n2 + 1)
    A = scipy.sparse.lil_matrix((nodes * d, nodes * d))
    b = np.zeros(nodes * d)
    row = 0
    eye = np.eye(d)

    def put(r, node, block):
        A[r:r + d, node * d:(node + 1) * d] = block

    for j in range(n1):  # lower interval: nodes 0..n1
        put(row, j + 1, eye)
        put(row, j, -E1)
        row += d
    for j in range(n2):  # upper interval: nodes n1+1..n1+1+n2
        put(row, n1 + 2 + j, eye)
        put(row, n1 + 1 + j, -E2)
        row += d
    put(row, n1 + 1, eye)  # Y(z0+) - Y(z0-) = jump
    put(row, n1, -eye)
    b[row:row + d] = jump
    row += d
    for c in wall:  # walls
        A[row, 0 * d + c] = 1.0
        row += 1
        A[row, (nodes - 1) * d + c] = 1.0
        row += 1
    assert row == nodes * d
    Y = scipy.sparse.linalg.spsolve(A.tocsc(), b)
    return float(Y[n1 * d + out])


def transverse_response(kappa: float, eps: float, z0: float) -> float:
    """u_2 . t at z0 per unit force t . F_2 on the plane (t across k).

    With no pressure term Eq. 7 reads -eps^-2 u'' + kappa^2 u = f delta(z - z0),
    u(0) = u(1) = 0. First-order form Y = (u, u'):
    u'' = eps^2 kappa^2 u away from z0, and [u'] = -eps^2 f across it."""
    M = np.array([[0.0, 1.0], [eps * eps * kappa * kappa, 0.0]])
    hmax = min(0.05, 1.0 / max(eps * kappa, 1.0))
    return _shoot(M, np.array([0.0, -eps * eps]), [0], z0, hmax, 0)


def longitudinal_response(kappa: float, eps: float, z0: float, P0: float = 1.0) -> float:
    """u_2 . k/kappa at z0 per unit force (k/kappa) . F_2 on the plane.

    Along k Eq. 7-9 read, with u the component of u_2 along k,
        -eps^-2 u'' + kappa^2 u + i kappa P0 q = f delta(z - z0)   (Eq. 7)
        -eps^-2 w'' + kappa^2 w + P0 q'         = 0                (Eq. 8)
         i kappa u + w'                         = 0                (Eq. 9)
    with u = w = 0 at both plates. For real f the solution has u real and w,
    q imaginary: w = i W, q = i Q. First-order form Y = (u, u', W, Q):
        u'' = eps^2 (kappa^2 u - kappa P0 Q)
        W'  = -kappa u
        Q'  = (-kappa eps^-2 u' - kappa^2 W) / P0       (Eq. 8 with W'' = -kappa u')
    and only u' jumps at z0: [u'] = -eps^2 f. Walls: u = W = 0.
    kappa = 0 has no direction; there the mode is the transverse one."""
    if kappa == 0.0:
        return transverse_response(0.0, eps, z0)
    e2, k = eps * eps, kappa
    M = np.array([[0.0, 1.0, 0.0, 0.0],
                  [e2 * k * k, 0.0, 0.0, -e2 * k * P0],
                  [-k, 0.0, 0.0, 0.0],
                  [0.0, -k / (e2 * P0), -k * k / P0, 0.0]])
    hmax = min(0.05, 1.0 / max(k, 1.0))
    return _shoot(M, np.array([0.0, -e2, 0.0, 0.0]), [0, 2], z0, hmax, 0)


@lru_cache(maxsize=None)
def mode_response(kappa: float, eps: float, z0: float) -> tuple[float, float]:
    """(g_T, g_L): the plane's in-plane response across and along k."""
    return transverse_response(kappa, eps, z0), longitudinal_response(kappa, eps, z0)


def _wavenumbers(n: int) -> list[list[float]]:
    """2 pi m for the DFT index j of a length-n periodic unit interval, m in
    (-n/2, n/2]. The index j = n/2 of an even n (Nyquist) stands for both
    +n/2 and -n/2; both are listed and the operator is averaged over them."""
    out = []
    for j in range(n):
        m = j if j <= n // 2 else j - n
        if n % 2 == 0 and j == n // 2:
            out.append([2.0 * math.pi * m, -2.0 * math.pi * m])
        else:
            out.append([2.0 * math.pi * m])
    return out


def velocity(eps: float, z0: float, F: np.ndarray, sigma: np.ndarray | None = None) -> np.ndarray:
    """u_2 [2][ny][nx] on the plane z0 from F [2][ny][nx] (x, y) and the extra
    stress sigma [3][ny][nx] (xx, xy, yy) or None, both concentrated on the
    plane; cell values on the uniform grid of the unit square.

    Per mode: f = F^ + i k . Sigma^ (the divergence), then
    u^ = g_T f + (g_L - g_T) (k/kappa)((k/kappa) . f); at a Nyquist index the
    map is the mean over the sign choices of that component (so the output is
    real); then the inverse DFT."""
    F = np.asarray(F, dtype=np.float64)
    _, ny, nx = F.shape
    Fh = np.fft.fft2(F, axes=(-2, -1))
    Sh = None if sigma is None else np.fft.fft2(np.asarray(sigma, dtype=np.float64), axes=(-2, -1))
    KX, KY = _wavenumbers(nx), _wavenumbers(ny)
    Uh = np.zeros((2, ny, nx), dtype=np.complex128)
    for jy in range(ny):
        for jx in range(nx):
            choices = [(kx, ky) for ky in KY[jy] for kx in KX[jx]]
            acc = np.zeros(2, dtype=np.complex128)
            for kx, ky in choices:
                f = Fh[:, jy, jx].copy()
                if Sh is not None:
                    sxx, sxy, syy = Sh[:, jy, jx]
                    f += 1j * np.array([kx * sxx + ky * sxy, kx * sxy + ky * syy])
                kappa = math.hypot(kx, ky)
                gT, gL = mode_response(kappa, eps, z0)
                if kappa == 0.0:
                    acc += gT * f
                else:
                    kh = np.array([kx, ky]) / kappa
                    acc += gT * f + (gL - gT) * kh * (kh @ f)
            Uh[:, jy, jx] = acc / len(choices)
    u = np.fft.ifft2(Uh, axes=(-2, -1))
    scale = max(np.abs(u).max(), 1e-300)
    assert np.abs(u.imag).max() <= 1e-12 * scale, "the mode map is not real-consistent"
    return np.ascontiguousarray(u.real)


def response_table(nx: int, ny: int, eps: float, z0: float) -> np.ndarray:
    """(g_T, g_L) [ny][nx//2 + 1][2] at |k| of the half spectrum (index jx in
    0..nx//2, jy in 0..ny-1, wavenumbers as in _wavenumbers)."""
    out = np.zeros((ny, nx // 2 + 1, 2))
    for jy in range(ny):
        my = jy if jy <= ny // 2 else jy - ny
        for jx in range(nx // 2 + 1):
            kappa = 2.0 * math.pi * math.hypot(jx, my)
            out[jy, jx] = mode_response(kappa, eps, z0)
    return out
