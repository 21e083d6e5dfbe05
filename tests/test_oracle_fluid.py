"""Pins of the float64 fluid oracle (oracle/fluid.py, Eq. 7-9) to facts that do
not come from it:
  - the mean mode (kappa = 0): -eps^-2 u'' = f delta(z - z0) with u(0) = u(1) = 0,
    u(z0) = eps^2 z0 (1 - z0) f;
  - across k: the Dirichlet Green's function of (eps^2 kappa^2 - d_zz), closed form;
  - along k, walls far away (eps kappa z0 >> 1): the free-space response of the
    anisotropic Stokes equations, eps^2 / (2 kappa (1 + eps)), from the Fourier
    integral over the z-wavenumber m of eps^2 m^2 / ((m^2 + eps^2 kappa^2)(m^2 + kappa^2)) / (2 pi);
  - along k at moderate kappa: a staggered finite-difference discretisation of
    Eq. 7-9 themselves (u, q at cell centres, w at nodes), Richardson-extrapolated;
  - symmetries: z0 -> 1 - z0, independence of P0;
  - the full-field solve against plane waves (force along and across k, a
    stress divergence, a uniform force) with the expected field written out,
    realness at Nyquist indices, translation invariance and positivity.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import fluid as FL


def green_transverse(kappa, eps, z0):
    mu = eps * kappa
    if mu == 0.0:
        return eps * eps * z0 * (1.0 - z0)
    return eps * eps * math.sinh(mu * z0) * math.sinh(mu * (1.0 - z0)) / (mu * math.sinh(mu))


@pytest.mark.parametrize("eps", [0.1, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("z0", [0.1, 0.3, 0.5])
def test_mean_mode_closed_form(eps, z0):
    gT, gL = FL.mode_response(0.0, eps, z0)
    ref = eps * eps * z0 * (1.0 - z0)
    assert abs(gT - ref) <= 1e-14 * ref and abs(gL - ref) <= 1e-14 * ref


@pytest.mark.parametrize("eps", [0.1, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("z0", [0.05, 0.3])
@pytest.mark.parametrize("kappa", [2 * math.pi, 20.0, 150.0])
def test_transverse_green_function(eps, z0, kappa):
    ref = green_transverse(kappa, eps, z0)
    assert abs(FL.transverse_response(kappa, eps, z0) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("eps", [0.1, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("kappa", [1500.0, 4000.0])
def test_longitudinal_free_space_limit(eps, kappa):
    z0 = 0.3
    assert eps * kappa * z0 > 40  # wall corrections ~ exp(-2 eps kappa z0): below rounding
    ref = eps * eps / (2.0 * kappa * (1.0 + eps))
    assert abs(FL.longitudinal_response(kappa, eps, z0) - ref) <= 1e-12 * ref
    # across k the same limit is eps / (2 kappa)
    assert abs(FL.transverse_response(kappa, eps, z0) - eps / (2 * kappa)) <= 1e-12 * eps / kappa


def fd_longitudinal(kappa, eps, z0, P0, j0):
    """Eq. 7-9 along k on a staggered grid of N cells, h = z0 / (j0 + 1/2) (z0 a
    cell centre): u and q at centres, w at the interior nodes (w = 0 at the
    plates), u = 0 at the plates by the mirror ghost u_{-1} = -u_0; the force
    f = 1 as 1/h in cell j0. Returns u at z0 (second order in h)."""
    h = z0 / (j0 + 0.5)
    N = round(1.0 / h)
    assert abs(N * h - 1.0) < 1e-9
    iu = lambda j: j  # noqa: E731
    iw = lambda j: N + j - 1  # noqa: E731
    iq = lambda j: 2 * N - 1 + j  # noqa: E731
    n = 3 * N - 1
    A = sp.lil_matrix((n, n), dtype=complex)
    b = np.zeros(n, dtype=complex)
    e2i = 1.0 / (eps * eps)
    r = 0
    for j in range(N):  # Eq. 7 at centres
        A[r, iu(j)] += 2 * e2i / h**2 + kappa**2
        for jj in (j - 1, j + 1):
            if 0 <= jj < N:
                A[r, iu(jj)] += -e2i / h**2
            else:
                A[r, iu(j)] += e2i / h**2
        A[r, iq(j)] += 1j * kappa * P0
        if j == j0:
            b[r] = 1.0 / h
        r += 1
    for j in range(1, N):  # Eq. 8 at interior nodes
        A[r, iw(j)] += 2 * e2i / h**2 + kappa**2
        for jj in (j - 1, j + 1):
            if 1 <= jj <= N - 1:
                A[r, iw(jj)] += -e2i / h**2
        A[r, iq(j)] += P0 / h
        A[r, iq(j - 1)] += -P0 / h
        r += 1
    for j in range(N):  # Eq. 9 at centres
        A[r, iu(j)] += 1j * kappa
        if j + 1 <= N - 1:
            A[r, iw(j + 1)] += 1.0 / h
        if j >= 1:
            A[r, iw(j)] += -1.0 / h
        r += 1
    x = spl.spsolve(A.tocsc(), b)
    return x[iu(j0)]


@pytest.mark.parametrize("kappa,eps,z0,P0", [(2 * math.pi, 0.5, 0.1, 1.0), (20.0, 0.3, 0.1, 3.0),
                                             (8.0, 2.0, 0.1, 1.0), (2 * math.pi * 3, 1.0, 0.25, 0.5)])
def test_longitudinal_against_finite_differences(kappa, eps, z0, P0):
    vals = [fd_longitudinal(kappa, eps, z0, P0, j0) for j0 in (13, 40, 121)]  # h / 3 each
    assert all(abs(v.imag) <= 1e-12 * abs(v) for v in vals)  # u real for a real force
    r1 = [(9 * vals[i + 1].real - vals[i].real) / 8 for i in range(2)]
    rich = (81 * r1[1] - r1[0]) / 80
    ref = FL.longitudinal_response(kappa, eps, z0, P0)
    assert abs(rich - ref) <= 1e-6 * ref, (rich, ref)
    # second order: the error shrinks about 9-fold per refinement
    errs = [abs(v.real - ref) for v in vals]
    assert 7 < errs[0] / errs[1] < 11 and 7 < errs[1] / errs[2] < 11


@pytest.mark.parametrize("kappa", [2 * math.pi, 30.0, 200.0])
def test_symmetries(kappa):
    eps = 0.4
    for z0 in (0.1, 0.27):
        a, b = FL.mode_response(kappa, eps, z0), FL.mode_response(kappa, eps, 1.0 - z0)
        assert abs(a[0] - b[0]) <= 1e-13 * a[0] and abs(a[1] - b[1]) <= 1e-12 * a[1]
    l1 = FL.longitudinal_response(kappa, eps, 0.2, 1.0)
    l7 = FL.longitudinal_response(kappa, eps, 0.2, 7.0)
    assert abs(l1 - l7) <= 1e-12 * l1  # P0 scales the pressure only
    gT, gL = FL.mode_response(kappa, eps, 0.2)
    assert 0 < gL < gT  # the pressure resists compression along k


def grid_x(n):
    return np.arange(n) / n


def test_plane_waves_along_and_across():
    eps, z0 = 0.3, 0.15
    ny, nx = 6, 8
    X, Y = np.meshgrid(grid_x(nx), grid_x(ny))
    mx, my = 1, 2
    k = 2 * math.pi * np.array([mx, my])
    kappa = float(np.linalg.norm(k))
    phase = np.cos(k[0] * X + k[1] * Y)
    gT, gL = FL.mode_response(kappa, eps, z0)
    along, across = k / kappa, np.array([-k[1], k[0]]) / kappa
    for d, g in ((along, gL), (across, gT)):
        F = np.stack([d[0] * phase, d[1] * phase])
        u = FL.velocity(eps, z0, F)
        ref = np.stack([g * d[0] * phase, g * d[1] * phase])
        assert np.abs(u - ref).max() <= 1e-14 * np.abs(ref).max()


def test_uniform_force_and_stress_divergence():
    eps, z0 = 0.2, 0.1
    ny, nx = 4, 10
    F = np.zeros((2, ny, nx))
    F[0] += 0.7
    F[1] -= 0.2
    u = FL.velocity(eps, z0, F)
    g0 = eps * eps * z0 * (1 - z0)
    assert np.allclose(u[0], 0.7 * g0, rtol=1e-14) and np.allclose(u[1], -0.2 * g0, rtol=1e-14)
    # Sigma_xx = cos(2 pi m x): div Sigma = (-2 pi m sin(2 pi m x), 0), along k = (2 pi m, 0)
    X, _ = np.meshgrid(grid_x(nx), grid_x(ny))
    m = 3
    sig = np.zeros((3, ny, nx))
    sig[0] = np.cos(2 * math.pi * m * X)
    u = FL.velocity(eps, z0, np.zeros((2, ny, nx)), sig)
    _, gL = FL.mode_response(2 * math.pi * m, eps, z0)
    ref = -2 * math.pi * m * np.sin(2 * math.pi * m * X) * gL
    assert np.abs(u[0] - ref).max() <= 1e-13 * np.abs(ref).max() and np.abs(u[1]).max() <= 1e-15
    # Sigma_xy = cos(2 pi m x): div Sigma = (0, -2 pi m sin(2 pi m x)), across k
    sig = np.zeros((3, ny, nx))
    sig[1] = np.cos(2 * math.pi * m * X)
    u = FL.velocity(eps, z0, np.zeros((2, ny, nx)), sig)
    gT, _ = FL.mode_response(2 * math.pi * m, eps, z0)
    ref = -2 * math.pi * m * np.sin(2 * math.pi * m * X) * gT
    assert np.abs(u[1] - ref).max() <= 1e-13 * np.abs(ref).max() and np.abs(u[0]).max() <= 1e-15


def test_nyquist_mode_and_realness():
    eps, z0 = 0.3, 0.2
    ny, nx = 4, 6
    alt = (-1.0) ** np.arange(nx)[None, :] * np.ones((ny, 1))
    F = np.stack([alt, np.zeros((ny, nx))])
    u = FL.velocity(eps, z0, F)  # k = (+-pi nx, 0): along x for both signs
    gT, gL = FL.mode_response(math.pi * nx, eps, z0)
    assert np.abs(u[0] - gL * alt).max() <= 1e-14 and np.abs(u[1]).max() <= 1e-15
    rng = np.random.default_rng(3)
    F = rng.standard_normal((2, ny, nx))
    S = rng.standard_normal((3, ny, nx))
    FL.velocity(eps, z0, F, S)  # asserts a real inverse transform


def test_translation_and_positivity():
    eps, z0 = 0.5, 0.25
    ny, nx = 5, 7
    rng = np.random.default_rng(11)
    F = rng.standard_normal((2, ny, nx))
    u = FL.velocity(eps, z0, F)
    u2 = FL.velocity(eps, z0, np.roll(F, (2, 3), axis=(1, 2)))
    assert np.abs(u2 - np.roll(u, (2, 3), axis=(1, 2))).max() <= 1e-14 * np.abs(u).max()
    # the Stokes operator is positive definite: the force does positive work
    assert float(np.sum(F * u)) > 0


def test_table_layout():
    eps, z0 = 0.2, 0.1
    tab = FL.response_table(6, 5, eps, z0)
    assert tab.shape == (5, 4, 2)
    kap = 2 * math.pi * math.hypot(3, -2)  # jy = 3 of ny = 5 is my = -2
    assert np.allclose(tab[3, 3], FL.mode_response(kap, eps, z0), rtol=0, atol=0)
