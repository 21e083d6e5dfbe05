"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test states the fact it pins and which plausible mistake in the oracle
would fail it. Expected values come from closed forms, invariants, symmetries
or an independent brute-force expansion -- never from the oracle itself.
"""
import math

import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, cellular_flow,
                                           psi_isotropic_perturbed, psi_uniform,
                                           random_divfree_flow)
from tests import brute_force

TWO_PI = 2.0 * math.pi


def _rand_state(O, g, seed, mb_scale=0.3, mtot=1.0):
    rng = SplitMix64(seed)
    psi = psi_isotropic_perturbed(g, seed, amp=0.3)
    mb = mb_scale * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    return O.make_state(g, psi, mb, np.full((g.ny, g.nx), mtot))


# --------------------------------------------------------------- invariants

def test_filament_number_conserved(oracle_mod):
    """Eq. 1 in flux form telescopes: sum psi is constant to round-off over
    200 substeps (fails for a face flux that differs between its two cells)."""
    O = oracle_mod
    g, r = Grid(32, 32, 16, 16), Rates()
    st = O.make_state(g, psi_isotropic_perturbed(g, 0))
    u = cellular_flow(g)
    N0 = st.psi.sum()
    O.run(g, r, st, u, O.dt(g, r, st, u), 200)
    assert abs(st.psi.sum() - N0) / N0 <= 1e-14


def test_motor_number_conserved(oracle_mod):
    """Eq. 5-6: free plus coarse-bound motors equal M in every cell, with the
    coarse density recomputed from the exported psi and Mb."""
    O = oracle_mod
    g, r = Grid(16, 16, 8, 8), Rates()
    st = O.make_state(g, psi_isotropic_perturbed(g, 3))
    u = random_divfree_flow(g, 5, 8, 0.1)
    O.run(g, r, st, u, O.dt(g, r, st, u), 100)
    dth, ds = TWO_PI / g.ntheta, g.L / g.ns
    C = np.einsum("yxk,yxkj->yx", st.psi, st.mb) * dth * ds
    assert np.abs(st.mf + C - st.mtot).max() <= 1e-14
    assert np.abs(C - st.c).max() <= 1e-15


@pytest.mark.parametrize("glide,v_sp", [(0.05, 0.0), (0.5, 0.3)])
def test_isotropic_uniform_state_stationary(oracle_mod, glide, v_sp):
    """Uniform isotropic psi with zero flow: every face velocity is the same on
    both sides of a cell, so psi stays bitwise unchanged and every cell's motor
    rows evolve identically."""
    O = oracle_mod
    g, r = Grid(8, 6, 8, 8), Rates(glide=glide, v_sp=v_sp)
    st = O.make_state(g, psi_uniform(g))
    psi0 = st.psi.copy()
    u = np.zeros((2, g.ny, g.nx))
    O.run(g, r, st, u, 0.01, 50)
    assert np.array_equal(st.psi, psi0)
    assert np.array_equal(st.mb, np.broadcast_to(st.mb[0, 0], st.mb.shape))
    assert st.mb.max() > 0.0


# -------------------------------------------------------------- closed forms

def test_bind_unbind_closed_form(oracle_mod):
    """Walking off, flow off, uniform psi (rho = 1): midpoint RK2 with Mf lagged
    gives M^{n+1} = A M^n + B Mf^n, A = 1 - k dt + (k dt)^2/2,
    B = k_on dt (1 - k dt/2), Mf^n = M - rho L M^n, so
    M^n = M_inf (1 - r^n), r = A - B rho L, M_inf = B M / (1 - A + B rho L).
    Fails for a wrong RK2 stage weight, a wrong reaction sign, or a wrong
    ds / dtheta normalisation of the coarse density."""
    O = oracle_mod
    g = Grid(2, 3, 4, 5, L=1.3)
    r = Rates(v_walk=0.0, k_on=1.0, k_off=0.5, glide=0.0)
    st = O.make_state(g, psi_uniform(g), mtot=np.full((g.ny, g.nx), 1.7))
    u = np.zeros((2, g.ny, g.nx))
    dt, k, kon, M, rho, L = 0.01, 0.5, 1.0, 1.7, 1.0, 1.3
    A = 1 - k * dt + 0.5 * (k * dt) ** 2
    B = kon * dt * (1 - 0.5 * k * dt)
    rr = A - B * rho * L
    Minf = B * M / (1 - A + B * rho * L)
    for n in range(1, 101):
        O.run(g, r, st, u, dt, 1)
        expect = Minf * (1 - rr ** n)
        assert np.allclose(st.mb, expect, rtol=1e-13, atol=0)
        assert np.allclose(st.mf, M - rho * L * expect, rtol=1e-13, atol=0)


def test_pure_decay_closed_form(oracle_mod):
    """k_on = 0, no walking: each RK2 step multiplies Mb by A = 1 - k dt + (k dt)^2/2
    (the midpoint rule applied to exponential decay)."""
    O = oracle_mod
    g = Grid(3, 2, 3, 4)
    r = Rates(v_walk=0.0, k_on=0.0, k_off=2.0, glide=0.0)
    st = O.make_state(g, psi_uniform(g), mb=np.full((2, 3, 3, 4), 0.7), mtot=np.full((2, 3), 10.0))
    u = np.zeros((2, g.ny, g.nx))
    dt = 0.05
    A = 1 - 2.0 * dt + 0.5 * (2.0 * dt) ** 2
    O.run(g, r, st, u, dt, 30)
    assert np.allclose(st.mb, 0.7 * A ** 30, rtol=1e-13, atol=0)


def test_translation_donor_cell_closed_form(oracle_mod):
    """Constant flow U > 0 in x, no gliding: one step is the first-order upwind
    update psi_i - dt U (psi_i - psi_{i-1}) / dx; with U < 0 it upwinds from
    the right. Fails for a reversed upwind side or a wrong face average."""
    O = oracle_mod
    g = Grid(7, 3, 4, 2)
    r = Rates(glide=0.0, v_walk=0.0, k_on=0.0, k_off=0.0)
    rng = SplitMix64(11)
    psi = 0.1 + rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta)
    for U in (0.37, -0.37):
        st = O.make_state(g, psi)
        u = np.zeros((2, g.ny, g.nx))
        u[0] = U
        dt = 0.1
        O.run(g, r, st, u, dt, 1)
        if U > 0:
            exp = psi - dt * U * (psi - np.roll(psi, 1, axis=1)) * g.nx
        else:
            exp = psi - dt * U * (np.roll(psi, -1, axis=1) - psi) * g.nx
        assert np.allclose(st.psi, exp, rtol=1e-14, atol=1e-15)


def test_gliding_direction_closed_form(oracle_mod):
    """Gliding speed V = v_sp > 0 with no flow moves filaments along -p
    (Eq. 2): the theta=0 population upwinds from the right in x, the
    theta=pi/2 population from the north neighbour in y."""
    O = oracle_mod
    g = Grid(5, 4, 4, 2)
    r = Rates(glide=0.0, v_sp=0.8, v_walk=0.0, k_on=0.0, k_off=0.0)
    rng = SplitMix64(12)
    psi = 0.1 + rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta)
    st = O.make_state(g, psi)
    dt = 0.05
    O.run(g, r, st, np.zeros((2, g.ny, g.nx)), dt, 1)
    V = 0.8
    e0 = psi[:, :, 0] + dt * V * (np.roll(psi[:, :, 0], -1, axis=1) - psi[:, :, 0]) * g.nx
    e1 = psi[:, :, 1] + dt * V * (np.roll(psi[:, :, 1], -1, axis=0) - psi[:, :, 1]) * g.ny
    assert np.allclose(st.psi[:, :, 0], e0, rtol=1e-13, atol=1e-15)
    # theta = pi/2: cos is 6e-17, not 0, so allow that much x-flux
    assert np.allclose(st.psi[:, :, 1], e1, rtol=1e-12, atol=1e-14)


def test_jeffery_rotation_closed_form(oracle_mod):
    """Uniform psi in the shear-like flow u = (a sin 2 pi y, 0): x and y fluxes
    cancel, and the theta update is psibar (1 + dt (w_{k+1/2} - w_{k-1/2}) ... )
    with Jeffery rate w(phi) = -G_xy sin^2 phi and the central difference
    G_xy = a (sin 2pi y_{j+1} - sin 2pi y_{j-1}) / (2 dy). Fails for a wrong
    rotation sign, a swapped gradient component or a misplaced theta face."""
    O = oracle_mod
    g = Grid(4, 8, 12, 2)
    r = Rates(glide=0.0, v_walk=0.0, k_on=0.0, k_off=0.0)
    a = 0.3
    y = (np.arange(g.ny) + 0.5) / g.ny
    u = np.zeros((2, g.ny, g.nx))
    u[0] = (a * np.sin(2 * math.pi * y))[:, None]
    st = O.make_state(g, psi_uniform(g))
    dt = 0.02
    O.run(g, r, st, u, dt, 1)
    dth = TWO_PI / g.ntheta
    pb = 1.0 / TWO_PI
    yp, ym = np.roll(y, -1), np.roll(y, 1)
    Gxy = a * (np.sin(2 * math.pi * yp) - np.sin(2 * math.pi * ym)) * g.ny / 2.0
    k = np.arange(g.ntheta)
    wp = -Gxy[:, None] * np.sin((k + 0.5) * dth) ** 2
    wm = -Gxy[:, None] * np.sin((k - 0.5) * dth) ** 2
    exp = pb - dt * pb * (wp - wm) / dth
    assert np.allclose(st.psi, np.broadcast_to(exp[:, None, :], st.psi.shape), rtol=1e-13, atol=1e-16)


def test_dt_rule_closed_forms(oracle_mod):
    """Adaptive substep (Sec. 2): cfl over the largest of walking v/ds,
    advection |ax|/dx + |ay|/dy, rotation |w|/dth and k_off + k_on L rho."""
    O = oracle_mod
    g, r = Grid(32, 32, 16, 16), Rates()
    st = O.make_state(g, psi_uniform(g))
    assert O.dt(g, r, st, np.zeros((2, 32, 32))) == pytest.approx(0.4 / 16.0, rel=1e-15)
    u = np.zeros((2, 32, 32))
    u[0] = 100.0
    assert O.dt(g, Rates(glide=0.0), st, u) == pytest.approx(0.4 / (100.0 * 32), rel=1e-15)
    r2 = Rates(k_off=50.0, k_on=3.0)
    assert O.dt(g, r2, st, np.zeros((2, 32, 32))) == pytest.approx(0.4 / (50.0 + 3.0), rel=1e-15)


def test_moments_closed_forms(oracle_mod):
    """psi = psibar (1 + eps cos(theta - theta0)) and linear rows Mb = a + b s:
    polar order eps/2, P = psibar eps pi (cos, sin)(theta0), rho = 1, Q = 0,
    n_b = a L, m1 = b (L^3/12 - L ds^2/12) (midpoint sum of s^2),
    F = F_m n_b P, tr sigma_a = F_m ell m1 rho, sigma_xx = sigma_yy."""
    O = oracle_mod
    g = Grid(3, 2, 16, 8, L=1.5)
    r = Rates(force_scale=1.7, ell=0.6)
    eps, th0, a, b = 0.2, 0.4, 0.3, 0.9
    k = np.arange(g.ntheta)
    pb = 1 / TWO_PI
    psi = np.broadcast_to(pb * (1 + eps * np.cos(k * TWO_PI / g.ntheta - th0)), (2, 3, 16)).copy()
    ds = g.L / g.ns
    s = -g.L / 2 + (np.arange(g.ns) + 0.5) * ds
    mb = np.broadcast_to(a + b * s, (2, 3, 16, 8)).copy()
    st = O.make_state(g, psi, mb, mtot=np.full((2, 3), 100.0))
    f, sc = O.moments(g, r, st)
    nb, m1 = a * g.L, b * (g.L ** 3 / 12 - g.L * ds ** 2 / 12)
    P = pb * eps * math.pi * np.array([math.cos(th0), math.sin(th0)])
    assert sc["polar_order"] == pytest.approx(eps / 2, rel=1e-13)
    assert np.allclose(f["rho"], 1.0, rtol=1e-14)
    assert np.allclose(f["Px"], P[0], rtol=1e-13) and np.allclose(f["Py"], P[1], rtol=1e-13)
    assert np.abs(f["Qxx"]).max() < 1e-15 and np.abs(f["Qxy"]).max() < 1e-15
    assert np.allclose(f["Fx"], 1.7 * nb * P[0], rtol=1e-13)
    assert np.allclose(f["Fy"], 1.7 * nb * P[1], rtol=1e-13)
    assert np.allclose(f["Sxx"] + f["Syy"], 1.7 * 0.6 * m1, rtol=1e-13)
    assert np.allclose(f["Sxx"], f["Syy"], rtol=1e-13)
    assert sc["mean_stress"] == pytest.approx(1.7 * 0.6 * m1, rel=1e-13)
    assert sc["N_psi"] == pytest.approx(1.0, rel=1e-14)


# ------------------------------------------------------------ walking in s

def _walk_only(O, ns, M0, nsteps, cfl=0.4, v=1.0):
    g = Grid(1, 1, 1, ns)
    r = Rates(v_walk=v, k_on=0.0, k_off=0.0, glide=0.0)
    st = O.make_state(g, np.full((1, 1, 1), 1 / TWO_PI), mb=np.asarray(M0).reshape(1, 1, 1, ns),
                      mtot=np.full((1, 1), 1e30))
    dt = cfl * (g.L / ns) / v
    hist = [st.mb.ravel().copy()]
    for _ in range(nsteps):
        O.run(g, r, st, np.zeros((2, 1, 1)), dt, 1)
        hist.append(st.mb.ravel().copy())
    return hist, dt


def test_walk_conserves_away_from_plus_end(oracle_mod):
    """A bump away from both ends: sum_j M_j ds is constant (flux form with
    zero inflow), to round-off."""
    O = oracle_mod
    ns = 64
    s = -0.5 + (np.arange(ns) + 0.5) / ns
    M0 = np.where(np.abs(s + 0.2) < 0.1, np.cos(math.pi * (s + 0.2) / 0.2) ** 2, 0.0)
    hist, _ = _walk_only(O, ns, M0, 20)
    assert abs(hist[-1].sum() - M0.sum()) <= 1e-14 * M0.sum()


def test_walk_outflow_at_plus_end(oracle_mod):
    """Uniform row M = 1, walking only, Courant number c = v dt / ds = 0.4.
    Worked by hand: stage 1 has zero slopes, so M*_0 = 1 - c/2 and the rest
    stay 1; stage 2 takes the Superbee branch sigma_0 = 2b = c at the first
    node, giving Phi_{1/2} = 1, and the plus-end outflow v M_{ns-1} = 1 equals
    the inflow to the last node. Hence M^1 = (1 - c, 1, ..., 1): nothing walks
    on at the minus end and the row loses exactly dt v through the plus end."""
    O = oracle_mod
    ns = 8
    hist, dt = _walk_only(O, ns, np.ones(ns), 1)
    c = 0.4
    exp = np.ones(ns)
    exp[0] = 1.0 - c
    assert np.allclose(hist[1], exp, rtol=1e-15, atol=1e-15)
    assert hist[1].sum() / ns == pytest.approx(1.0 - dt, rel=1e-15)


def test_walk_second_order_convergence(oracle_mod):
    """A smooth cos^2 bump translated at speed v: the L1 error against the exact
    translate drops at better than order 1.7 under refinement (Superbee MUSCL
    with midpoint RK2 is second order on smooth data), so a limiter that falls
    back to first-order upwinding (order 1) fails."""
    O = oracle_mod
    errs = []
    bump = lambda x: np.where(np.abs(x) < 0.25, np.cos(math.pi * x / 0.5) ** 2, 0.0)
    for ns in (128, 256, 512):
        ds = 1.0 / ns
        s = -0.5 + (np.arange(ns) + 0.5) * ds
        steps = int(round(0.2 / (0.4 * ds)))
        hist, dt = _walk_only(O, ns, bump(s + 0.15), steps)
        T = steps * dt
        errs.append(np.abs(hist[-1] - bump(s + 0.15 - T)).sum() * ds)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.7, (errs, orders)


def test_walk_total_variation_bounded(oracle_mod):
    """A square pulse walked for 150 steps stays within its initial range and
    its total variation never grows by more than round-off (the limiter keeps
    the scheme free of new extrema at cfl 0.4). Fails for an unlimited or
    sign-flipped slope."""
    O = oracle_mod
    ns = 100
    M0 = np.zeros(ns)
    M0[10:30] = 1.0
    hist, _ = _walk_only(O, ns, M0, 150)
    tv = lambda m: np.abs(np.diff(np.concatenate(([0.0], m)))).sum()
    for a, b in zip(hist, hist[1:]):
        assert tv(b) <= tv(a) + 1e-13
        assert b.min() >= -1e-14 and b.max() <= 1.0 + 1e-14


# ------------------------------------------------------------- symmetries

def _step(O, g, r, st, u, dt, n=1):
    s2 = st.copy()
    O.run(g, r, s2, u, dt, n)
    return s2


def test_periodic_shift_commutes(oracle_mod):
    """Shifting the periodic grid commutes with a substep, bitwise: no cell is
    special, so a boundary wrap error anywhere fails."""
    O = oracle_mod
    g, r = Grid(6, 5, 4, 6), Rates(v_sp=0.1, glide=0.4)
    st = _rand_state(O, g, 21)
    u = random_divfree_flow(g, 3, 4, 0.3)
    a = _step(O, g, r, st, u, 0.01, 3)
    sh = lambda x: np.roll(np.roll(x, 2, axis=0), -3, axis=1)
    st2 = O.State(g, sh(st.psi), sh(st.mb), sh(st.mf), sh(st.c), sh(st.mtot))
    b = _step(O, g, r, st2, np.stack([sh(u[0]), sh(u[1])]), 0.01, 3)
    assert np.array_equal(sh(a.psi), b.psi) and np.array_equal(sh(a.mb), b.mb)
    assert np.array_equal(sh(a.mf), b.mf)


def _rot90(st_psi, st_mb, u, g):
    """Rotate the square by +90 degrees about its centre: a point (i, j) goes to
    (n-1-j, i), a direction theta to theta + pi/2 (k -> k + nth/4), and the
    velocity vector (ux, uy) to (-uy, ux)."""
    n, q = g.nx, g.ntheta // 4
    # new[b, a] (row = y index b, column = x index a) = old[y = n-1-a, x = b]
    def sc(F):
        return np.array([[F[n - 1 - a, b] for a in range(n)] for b in range(n)])
    def rowsrc(F):
        out = np.empty_like(F)
        for b in range(n):
            for a in range(n):
                out[b, a] = np.roll(F[n - 1 - a, b], q, axis=0)
        return out
    ux, uy = sc(u[0]), sc(u[1])
    return rowsrc(st_psi), rowsrc(st_mb), np.stack([-uy, ux])


def test_rotation_by_quarter_turn_commutes(oracle_mod):
    """Rotating grid, orientations and flow by 90 degrees commutes with a
    substep to round-off. Fails for swapped x/y components, a transposed
    velocity gradient or a wrong sign in the rotation rate."""
    O = oracle_mod
    g, r = Grid(6, 6, 8, 5), Rates(v_sp=0.2, glide=0.5)
    st = _rand_state(O, g, 31)
    u = random_divfree_flow(g, 7, 6, 0.4)
    a = _step(O, g, r, st, u, 0.01, 2)
    p2, m2, u2 = _rot90(st.psi, st.mb, u, g)
    st2 = O.make_state(g, p2, m2)
    b = _step(O, g, r, st2, u2, 0.01, 2)
    pa, ma, _ = _rot90(a.psi, a.mb, u, g)
    assert np.allclose(pa, b.psi, rtol=1e-12, atol=1e-15)
    assert np.allclose(ma, b.mb, rtol=1e-12, atol=1e-15)


def test_mirror_reflection_commutes(oracle_mod):
    """Reflecting x -> -x maps theta to pi - theta (k -> nth/2 - k) and
    (ux, uy) to (-ux, uy); a substep commutes with it to round-off. The
    rotation rate changes sign under the reflection, so a sign error in
    Jeffery's term fails."""
    O = oracle_mod
    g, r = Grid(5, 4, 8, 4), Rates(v_sp=0.1, glide=0.3)
    st = _rand_state(O, g, 41)
    u = random_divfree_flow(g, 9, 6, 0.4)
    kk = (g.ntheta // 2 - np.arange(g.ntheta)) % g.ntheta

    def refl_state(psi, mb):
        return psi[:, ::-1, :][:, :, kk], mb[:, ::-1, :, :][:, :, kk, :]

    a = _step(O, g, r, st, u, 0.01, 2)
    p2, m2 = refl_state(st.psi, st.mb)
    u2 = np.stack([-u[0][:, ::-1], u[1][:, ::-1]])
    st2 = O.make_state(g, np.ascontiguousarray(p2), np.ascontiguousarray(m2))
    b = _step(O, g, r, st2, np.ascontiguousarray(u2), 0.01, 2)
    pa, ma = refl_state(a.psi, a.mb)
    assert np.allclose(pa, b.psi, rtol=1e-12, atol=1e-15)
    assert np.allclose(ma, b.mb, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------ clip (Alg. 2)

def test_scale_down_clip(oracle_mod):
    """Alg. 2: where the coarse bound density would exceed the total M, every
    Mb at that anchor is scaled by M / C so that the coarse density equals M
    and no motor is free. Forced with M = 0.1 and a binding rate large enough
    that one substep overshoots; the same substep with the clip out of reach
    (M huge, same free motors) gives the unscaled rows."""
    O = oracle_mod
    g = Grid(4, 4, 8, 8)
    r = Rates(k_on=3000.0, k_off=0.5)
    psi = psi_isotropic_perturbed(g, 2)
    u = cellular_flow(g)
    zero = np.zeros((4, 4, 8, 8))
    free = np.full((4, 4), 0.1)
    mtot = free.copy()
    mtot[0, 0] = 50.0  # this cell never clips
    clip = O.State(g, psi.copy(), zero.copy(), free.copy(), np.zeros((4, 4)), mtot)
    noclip = O.State(g, psi.copy(), zero.copy(), free.copy(), np.zeros((4, 4)), np.full((4, 4), 1e6))
    O.run(g, r, clip, u, 0.002, 1)
    O.run(g, r, noclip, u, 0.002, 1)
    dth, ds = TWO_PI / g.ntheta, g.L / g.ns
    Cpre = np.einsum("yxk,yxkj->yx", noclip.psi, noclip.mb) * dth * ds
    clipped = np.ones((4, 4), bool)
    clipped[0, 0] = False
    assert np.all(Cpre[clipped] > 0.1)
    scale = np.where(clipped, 0.1 / Cpre, 1.0)
    assert np.allclose(clip.mb, noclip.mb * scale[:, :, None, None], rtol=1e-14, atol=0)
    C = np.einsum("yxk,yxkj->yx", clip.psi, clip.mb) * dth * ds
    assert np.allclose(C[clipped], 0.1, rtol=1e-14)
    assert np.all(clip.mf[clipped] == 0.0) and np.all(clip.c[clipped] == 0.1)
    assert clip.mf[0, 0] == pytest.approx(50.0 - Cpre[0, 0], rel=1e-14)


# ---------------------------------------------------- brute-force expansion

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 6, 7)])
def test_brute_force_expansion_agrees(oracle_mod, dims):
    """Independent scatter-form, ratio-limiter expansion of one substep on tiny
    grids (including ragged sizes) agrees with the oracle to round-off."""
    O = oracle_mod
    g = Grid(*dims, L=1.1)
    r = Rates(v_walk=0.9, k_on=1.3, k_off=0.7, glide=0.4, v_sp=0.15)
    st = _rand_state(O, g, 51, mb_scale=0.5, mtot=1.0)
    u = random_divfree_flow(g, 13, 5, 0.5)
    dt = 0.02
    for _ in range(3):
        bp, bm, bf, bc = brute_force.substep(g, r, dt, u.tolist(), st.psi.tolist(), st.mb.tolist(),
                                             st.mf.tolist(), st.mtot.tolist())
        O.run(g, r, st, u, dt, 1)
        assert np.allclose(st.psi, np.array(bp), rtol=1e-13, atol=1e-16)
        assert np.allclose(st.mb, np.array(bm), rtol=1e-12, atol=1e-15)
        assert np.allclose(st.mf, np.array(bf), rtol=1e-13, atol=1e-15)
        assert np.allclose(st.c, np.array(bc), rtol=1e-13, atol=1e-15)


# ------------------------------------------------------- tangent and adjoint

def _perturb(g, seed):
    rng = SplitMix64(seed)
    d = lambda *sh: rng.uniforms(int(np.prod(sh))).reshape(sh) - 0.5
    return (d(g.ny, g.nx, g.ntheta), d(g.ny, g.nx, g.ntheta, g.ns), d(g.ny, g.nx),
            d(2, g.ny, g.nx), d(3))


def _forward_n(O, g, r, st, u, dt, n, params):
    rr = Rates(**{**r.__dict__, "k_off": params[0], "v_walk": params[1], "k_on": params[2]})
    s2 = st.copy()
    O.run(g, rr, s2, u, dt, n)
    return s2


@pytest.mark.parametrize("clip", [False, True])
def test_tangent_matches_central_differences(oracle_mod, clip):
    """The tangent of n substeps equals the central difference of the forward
    map (h = 1e-6) along a random direction in (psi, Mb, Mf, u, rates)."""
    O = oracle_mod
    g = Grid(4, 3, 6, 5)
    r = Rates(v_sp=0.1, glide=0.5, k_on=(300.0 if clip else 1.0))
    mt = 0.08 if clip else 1.0
    st = _rand_state(O, g, 61, mb_scale=0.02 if clip else 0.3, mtot=mt)
    u = random_divfree_flow(g, 17, 5, 0.4)
    dt, n = 0.01, 4
    dpsi, dmb, dmf, du, dp = _perturb(g, 62)
    p0 = np.array([r.k_off, r.v_walk, r.k_on])
    h = 1e-6

    def fwd(sign):
        s = O.State(g, st.psi + sign * h * dpsi, st.mb + sign * h * dmb, st.mf + sign * h * dmf,
                    st.c.copy(), st.mtot.copy())
        return _forward_n(O, g, r, s, u + sign * h * du, dt, n, p0 + sign * h * dp)

    fp, fm = fwd(1), fwd(-1)
    # tangent sweep
    cur = st.copy()
    tp, tm, tf = dpsi.copy(), dmb.copy(), dmf.copy()
    clipped_steps = 0
    for _ in range(n):
        O.tangent_substep(g, r, dt, u, du, dp, cur, tp, tm, tf)
        O.run(g, r, cur, u, dt, 1)
        clipped_steps += int(np.any(cur.mf == 0.0))
    fd_p, fd_m, fd_f = [(a - b) / (2 * h) for a, b in ((fp.psi, fm.psi), (fp.mb, fm.mb), (fp.mf, fm.mf))]
    for tl, fd in ((tp, fd_p), (tm, fd_m), (tf, fd_f)):
        assert np.linalg.norm(tl - fd) <= 1e-6 * max(np.linalg.norm(fd), 1e-12)
    assert (clipped_steps > 0) == clip


@pytest.mark.parametrize("clip", [False, True])
def test_adjoint_dot_product(oracle_mod, clip):
    """<w, J d> = <J^T w, d> over n substeps for random d (state, u, rates) and
    random w: the adjoint is the exact transpose of the tangent."""
    O = oracle_mod
    g = Grid(5, 4, 6, 7)
    r = Rates(v_sp=0.1, glide=0.5, k_on=(300.0 if clip else 1.0))
    mt = 0.08 if clip else 1.0
    st = _rand_state(O, g, 71, mb_scale=0.02 if clip else 0.3, mtot=mt)
    u = random_divfree_flow(g, 19, 5, 0.4)
    dt, n = 0.01, 5
    dpsi, dmb, dmf, du, dp = _perturb(g, 72)
    wpsi, wmb, wmf, _, _ = _perturb(g, 73)
    cur = st.copy()
    tp, tm, tf = dpsi.copy(), dmb.copy(), dmf.copy()
    clipped_steps = 0
    for _ in range(n):
        O.tangent_substep(g, r, dt, u, du, dp, cur, tp, tm, tf)
        O.run(g, r, cur, u, dt, 1)
        clipped_steps += int(np.any(cur.mf == 0.0))
    assert (clipped_steps > 0) == clip
    lhs = (wpsi * tp).sum() + (wmb * tm).sum() + (wmf * tf).sum()
    lpsi, lmb, lmf, lu, lp = O.adjoint(g, r, st, u, dt, n, wpsi, wmb, wmf)
    rhs = ((lpsi * dpsi).sum() + (lmb * dmb).sum() + (lmf * dmf).sum() + (lu * du).sum()
           + (lp * dp).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300)


def test_patch_substep_equals_full_grid(oracle_mod):
    """The 3x3 periodic patch (same dx, dy) reproduces the full-grid substep of
    its centre cell exactly: the basis of the sampled full-size GPU checks."""
    O = oracle_mod
    g, r = Grid(9, 7, 8, 6), Rates(v_sp=0.1, glide=0.5)
    st = _rand_state(O, g, 81)
    u = random_divfree_flow(g, 23, 6, 0.4)
    full = _step(O, g, r, st, u, 0.01)
    cells = [(0, 0), (3, 4), (6, 8), (2, 0)]
    res = O.patch_substep(g, r, 0.01, u, st.psi, st.mb, st.mf, st.mtot, cells)
    for (iy, ix), c in zip(cells, res):
        assert np.array_equal(c["psi"], full.psi[iy, ix])
        assert np.array_equal(c["mb"], full.mb[iy, ix])
        assert c["mf"] == full.mf[iy, ix] and c["c"] == full.c[iy, ix]


# ---- filament diffusion (next row f1): Crank-Nicolson per direction


def _mode_psi(g, mx, my, k, eps=0.1):
    x = (np.arange(g.nx) + 0.5) / g.nx
    y = (np.arange(g.ny) + 0.5) / g.ny
    th = np.arange(g.ntheta) * 2 * np.pi / g.ntheta
    return 1.0 + eps * (np.cos(2 * np.pi * my * y)[:, None, None] *
                        np.cos(2 * np.pi * mx * x)[None, :, None] * np.cos(k * th)[None, None, :])


def test_diffusion_fourier_mode_closed_form(oracle_mod):
    """A Fourier mode is an eigenvector of every periodic second difference:
    one step multiplies its amplitude by the product over directions of
    (1 - a (1 - cos kappa h)) / (1 + a (1 - cos kappa h)), a = D dt / h^2, and
    leaves the mean unchanged."""
    g = Grid(10, 12, 16, 4)
    D_t, D_r, dt = 0.003, 0.7, 0.05
    mx, my, k = 2, 3, 5
    psi = _mode_psi(g, mx, my, k)
    out = oracle_mod.diffuse(g, psi, D_t, D_r, dt)

    def amp(n, h, D, m):
        a = D * dt / h ** 2
        q = a * (1 - np.cos(2 * np.pi * m / n))
        return (1 - q) / (1 + q)
    fac = amp(g.nx, 1 / g.nx, D_t, mx) * amp(g.ny, 1 / g.ny, D_t, my) * amp(
        g.ntheta, 2 * np.pi / g.ntheta, D_r, k)
    expect = 1.0 + fac * (psi - 1.0)
    assert np.max(np.abs(out - expect)) <= 1e-14
    assert 0 < fac < 1


def test_diffusion_conserves_and_commutes(oracle_mod):
    """The periodic Crank-Nicolson step conserves sum psi to round-off, is the
    identity at zero diffusivity, and (the 1-D operators commute) does not
    depend on the order of the directions."""
    g = Grid(7, 9, 6, 4)
    psi = psi_isotropic_perturbed(g, 8, amp=0.4)
    out = oracle_mod.diffuse(g, psi, 0.01, 0.3, 0.2)
    assert abs(out.sum() - psi.sum()) <= 1e-13 * psi.sum()
    assert np.array_equal(oracle_mod.diffuse(g, psi, 0.0, 0.0, 0.2), psi)
    # the opposite order (y, then x, then theta) with the same 1-D operators
    Mt = np.linalg.solve(*oracle_mod._cn_factor(g.ntheta, 0.3 * 0.2 / (2 * np.pi / g.ntheta) ** 2))
    Mx = np.linalg.solve(*oracle_mod._cn_factor(g.nx, 0.01 * 0.2 * g.nx ** 2))
    My = np.linalg.solve(*oracle_mod._cn_factor(g.ny, 0.01 * 0.2 * g.ny ** 2))
    step = np.einsum("ab,bxk->axk", My, psi)
    step = np.einsum("ab,ybk->yak", Mx, step)
    step = np.einsum("ab,yxb->yxa", Mt, step)
    assert np.max(np.abs(step - out)) <= 1e-13


def test_diffusion_large_step_is_stable_and_smooths(oracle_mod):
    """Unconditional stability: a step far beyond the explicit limit keeps
    every Fourier amplitude below one in magnitude (the extreme value drops)."""
    g = Grid(8, 8, 8, 4)
    psi = psi_isotropic_perturbed(g, 9, amp=0.5)
    out = oracle_mod.diffuse(g, psi, 0.5, 5.0, 10.0)
    assert np.linalg.norm(out - out.mean()) < np.linalg.norm(psi - psi.mean())


# ---- local substeps with psi frozen (next row f4)


def test_motor_local_equals_global_substeps_for_uniform_psi(oracle_mod):
    """With the same psi everywhere every cell takes the same local step, and
    with no flow and no gliding psi stays put: the local-step motor update is
    bit for bit the global substep of the hot path with dt = T / n."""
    g = Grid(5, 4, 6, 12)
    r = Rates(k_on=1.7, k_off=0.6, v_walk=0.8, glide=0.0, v_sp=0.0)
    psi = psi_isotropic_perturbed(g, 61, amp=0.0)
    rng = np.random.default_rng(62)
    mb = 0.2 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    a = oracle_mod.make_state(g, psi, mb)
    b = a.copy()
    T = 0.37
    n = oracle_mod.motor_local(g, r, a, T)
    assert np.all(n == n[0, 0]) and n[0, 0] > 1
    oracle_mod.run(g, r, b, np.zeros((2, g.ny, g.nx)), T / n[0, 0], int(n[0, 0]))
    for k in ("mb", "mf", "c"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert np.array_equal(b.psi, psi)


def test_motor_local_bind_unbind_closed_form_per_cell(oracle_mod):
    """No walking: each cell relaxes by its own lagged bind/unbind recursion
    M^n = M_inf (1 - r^n) (as for the global step) with its own density rho_i,
    step count n_i = ceil(T (k_off + k_on L rho_i) / cfl) and dt_i = T / n_i."""
    g = Grid(4, 3, 8, 6)
    r = Rates(k_on=1.2, k_off=0.5, v_walk=0.0, glide=0.0)
    dens = 1.0 / (2 * np.pi) * (0.5 + np.arange(g.nx * g.ny).reshape(g.ny, g.nx) / 6.0)
    psi = np.repeat(dens[:, :, None], g.ntheta, axis=2)
    st = oracle_mod.make_state(g, psi)
    T = 0.9
    n = oracle_mod.motor_local(g, r, st, T)
    for iy in range(g.ny):
        for ix in range(g.nx):
            rho = dens[iy, ix] * 2 * np.pi
            ni = max(1, math.ceil(T * (r.k_off + r.k_on * g.L * rho) / r.cfl))
            assert n[iy, ix] == ni
            dt = T / ni
            A = 1 - r.k_off * dt + (r.k_off * dt) ** 2 / 2
            B = r.k_on * dt * (1 - r.k_off * dt / 2)
            rr = A - B * rho * g.L
            Minf = B * 1.0 / (1 - A + B * rho * g.L)
            expect = Minf * (1 - rr ** ni)
            assert np.max(np.abs(st.mb[iy, ix] - expect)) <= 1e-13 * max(1.0, abs(expect))
    # different densities, different step counts
    assert len(np.unique(n)) > 1
    np.testing.assert_allclose(st.mf + st.c, 1.0, rtol=0, atol=1e-14)


# ---- non-local motor anchors (next row f2)


def test_anchor_zero_length_is_the_local_substep(oracle_mod):
    """With l/L = 0 every configuration is anchored in its filament's own cell:
    the anchor substep, its set-up and its force equal the local ones."""
    g = Grid(6, 5, 8, 12)
    r = Rates(ell=0.0, k_on=1.3, glide=0.2)
    psi = psi_isotropic_perturbed(g, 101, amp=0.4)
    rng = np.random.default_rng(102)
    mb = 0.3 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    mtot = 0.3 + rng.random((g.ny, g.nx))
    u = random_divfree_flow(g, 103, 4, 0.2)
    a = oracle_mod.make_state_anchor(g, r, psi, mb, mtot)
    b = oracle_mod.make_state(g, psi, mb, mtot)
    for k in ("mb", "mf", "c"):
        np.testing.assert_allclose(getattr(a, k), getattr(b, k), rtol=1e-14, atol=1e-15)
    dt = oracle_mod.dt(g, r, b, u)
    oracle_mod.run_anchor(g, r, a, u, dt, 6)
    oracle_mod.run(g, r, b, u, dt, 6)
    for k in ("psi", "mb", "mf", "c"):
        np.testing.assert_allclose(getattr(a, k), getattr(b, k), rtol=1e-13, atol=1e-15)
    fl, _ = oracle_mod.moments(g, r, b)
    F = oracle_mod.anchor_force(g, r, b)
    np.testing.assert_allclose(F[0], fl["Fx"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F[1], fl["Fy"], rtol=1e-12, atol=1e-15)


def test_anchor_offsets_locate_the_head(oracle_mod):
    """The anchor offsets put the head x + (l/L) s p inside the anchor cell."""
    g = Grid(16, 12, 8, 10)
    r = Rates(ell=0.37)
    ox, oy = oracle_mod.anchor_offsets(g, r)
    for k in range(g.ntheta):
        th = k * 2 * np.pi / g.ntheta
        for j in range(g.ns):
            s = -0.5 * g.L + (j + 0.5) * g.L / g.ns
            hx = 0.5 + r.ell * s * np.cos(th) * g.nx  # head, in cells from the centre's cell
            hy = 0.5 + r.ell * s * np.sin(th) * g.ny
            assert ox[k, j] <= hx < ox[k, j] + 1 + 1e-12
            assert oy[k, j] <= hy < oy[k, j] + 1 + 1e-12
    assert len(np.unique(ox)) > 3 and len(np.unique(oy)) > 3
    # opposite orientations mirror the offsets (s -> -s)
    kh = g.ntheta // 2
    assert np.all(np.abs(ox[kh, ::-1] - ox[0]) <= 1)


def test_anchor_single_filament_closed_form(oracle_mod):
    """One filament density in one cell and orientation, no flow, no walking,
    no gliding: psi stays put, and the nodes sharing an anchor r relax together
    by the lagged bind/unbind recursion with rho L replaced by
    psi0 ds dth n_r (n_r = nodes of that row anchored at r)."""
    g = Grid(9, 7, 8, 12)
    r = Rates(v_walk=0.0, glide=0.0, v_sp=0.0, k_on=2.0, k_off=0.4, ell=0.45)
    psi = np.zeros((g.ny, g.nx, g.ntheta))
    i0y, i0x, k0 = 3, 4, 1
    psi0 = 30.0
    psi[i0y, i0x, k0] = psi0
    st = oracle_mod.make_state_anchor(g, r, psi)
    u = np.zeros((2, g.ny, g.nx))
    dt, n = 0.05, 40
    oracle_mod.run_anchor(g, r, st, u, dt, n)
    assert np.array_equal(st.psi, psi)
    ox, oy = oracle_mod.anchor_offsets(g, r)
    anchors = [((i0y + oy[k0, j]) % g.ny, (i0x + ox[k0, j]) % g.nx) for j in range(g.ns)]
    counts = {a: anchors.count(a) for a in anchors}
    assert len(counts) >= 3
    ds, dth = g.L / g.ns, 2 * np.pi / g.ntheta
    A = 1 - r.k_off * dt + (r.k_off * dt) ** 2 / 2
    B = r.k_on * dt * (1 - r.k_off * dt / 2)
    for j, a in enumerate(anchors):
        w = psi0 * ds * dth * counts[a]
        rr = A - B * w
        Minf = B * 1.0 / (1 - A + B * w)
        expect = Minf * (1 - rr ** n)
        assert abs(st.mb[i0y, i0x, k0, j] - expect) <= 1e-13 * expect, j
        assert abs(st.c[a] - w * expect) <= 1e-13 * w * expect
        assert abs(st.mf[a] - (1 - w * expect)) <= 1e-13
    # rows that carry no filaments bind against a full pool: M_inf = B / (1 - A)
    other = st.mb[0, 0, 5, 3]
    assert abs(other - B / (1 - A) * (1 - A ** n)) <= 1e-13 * other


def test_anchor_conservation_and_uniform_state(oracle_mod):
    """Bound plus free motors equal the total at every anchor, summed over the
    grid; a uniform state stays uniform."""
    g = Grid(8, 6, 8, 10)
    r = Rates(ell=0.3, k_on=3.0)
    psi = psi_isotropic_perturbed(g, 111, amp=0.5)
    rng = np.random.default_rng(112)
    mb = 0.4 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    st = oracle_mod.make_state_anchor(g, r, psi, mb)
    u = random_divfree_flow(g, 113, 4, 0.1)
    dt = oracle_mod.dt(g, r, st, u)
    oracle_mod.run_anchor(g, r, st, u, dt, 15)
    ds, dth = g.L / g.ns, 2 * np.pi / g.ntheta
    bound = np.sum(st.psi[..., None] * st.mb) * ds * dth
    assert abs(bound + st.mf.sum() - st.mtot.sum()) <= 1e-13 * st.mtot.sum()
    np.testing.assert_allclose(st.mf + st.c, st.mtot, rtol=0, atol=1e-14)
    # uniform: the same psi and rows everywhere, no flow
    psiu = psi_isotropic_perturbed(g, 114, amp=0.0)
    mbu = np.broadcast_to(0.2 * rng.random((g.ntheta, g.ns)), mb.shape).copy()
    su = oracle_mod.make_state_anchor(g, r, psiu, mbu)
    oracle_mod.run_anchor(g, r, su, np.zeros((2, g.ny, g.nx)), 0.01, 8)
    assert np.ptp(su.c) <= 1e-14 * su.c.max()
    assert np.max(np.ptp(su.mb, axis=(0, 1))) <= 1e-14 * su.mb.max()


@pytest.mark.parametrize("dims", [(4, 3, 4, 5), (3, 4, 6, 4)])
def test_anchor_brute_force_agrees(oracle_mod, dims):
    """An independent expansion (head located on the grid, binding per node,
    coarse density per anchor cell) on tiny grids, with flow, gliding and a
    forced scale-down, agrees with the anchor substep."""
    g = Grid(*dims)
    r = Rates(ell=0.43, k_on=9.0, glide=0.3)
    psi = psi_isotropic_perturbed(g, 121, amp=0.6)
    rng = np.random.default_rng(122)
    mb = 0.3 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    mtot = 0.25 + 0.5 * rng.random((g.ny, g.nx))
    u = random_divfree_flow(g, 123, 3, 0.3)
    st = oracle_mod.make_state_anchor(g, r, psi, mb, mtot)
    dt = oracle_mod.dt(g, r, st, u) * 4.0  # a long step: the binding overshoots in some cells
    before = st.copy()
    oracle_mod.run_anchor(g, r, st, u, dt, 1)
    bp, bm, bf, bc = brute_force.substep_anchor(g, r, dt, u.tolist(), before.psi.tolist(),
                                                before.mb.tolist(), before.mf.tolist(),
                                                before.mtot.tolist())
    np.testing.assert_allclose(st.psi, np.array(bp), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st.mb, np.array(bm), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st.mf, np.array(bf), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st.c, np.array(bc), rtol=1e-12, atol=1e-14)
    clipped = np.array(bc) == before.mtot
    assert np.any(clipped) and not np.all(clipped)  # the scale-down acted in some cells


@pytest.mark.parametrize("dims,ell", [((5, 4, 8, 6), 0.43), ((4, 6, 6, 9), 0.9),
                                      ((7, 5, 5, 7), 1.7)])
def test_anchor_force_brute_force_deposit(oracle_mod, dims, ell):
    """Eq. 10 with the delta at the head x + (l/L) s p: an independent deposit
    (each node's head located from its own geometry on the grid, not from the
    oracle's offset table) agrees with the anchored force at l/L > 0, on heads
    that cross several cells and, at l/L = 1.7, wrap around the periodic grid.
    Fails for a force put in the filament's own cell, for one anchor used for
    a whole row, or for swapped x and y offsets."""
    g = Grid(*dims)
    r = Rates(ell=ell, force_scale=0.7)
    rng = np.random.default_rng(sum(dims) + 131)
    psi = rng.random((g.ny, g.nx, g.ntheta))
    mb = rng.random((g.ny, g.nx, g.ntheta, g.ns))
    st = oracle_mod.make_state_anchor(g, r, psi, mb, np.full((g.ny, g.nx), 1e9))
    F = oracle_mod.anchor_force(g, r, st)
    B = np.array(brute_force.anchor_force(g, r, st.psi.tolist(), st.mb.tolist()))
    np.testing.assert_allclose(F, B, rtol=1e-13, atol=1e-15)
    # the heads really leave the filament's cell: the local force field differs
    fl, _ = oracle_mod.moments(g, r, st)
    assert np.max(np.abs(F[0] - fl["Fx"])) > 1e-3 * np.max(np.abs(fl["Fx"]))


def test_anchor_force_total_is_the_local_total(oracle_mod):
    """Moving each node's force to the cell under its head moves it but does
    not change it: summed over the grid the anchored force equals the sum of
    the local force field F_m sum_k p psi n_b dtheta (Eq. 10), at any l/L.
    Fails for a dropped node, a wrong sign of p or a missing ds or dtheta."""
    g = Grid(9, 7, 12, 10)
    rng = np.random.default_rng(141)
    psi = rng.random((g.ny, g.nx, g.ntheta))
    mb = rng.random((g.ny, g.nx, g.ntheta, g.ns))
    for ell in (0.0, 0.21, 0.66, 2.3):
        r = Rates(ell=ell, force_scale=1.3)
        st = oracle_mod.make_state_anchor(g, r, psi, mb, np.full((g.ny, g.nx), 1e9))
        F = oracle_mod.anchor_force(g, r, st)
        fl, _ = oracle_mod.moments(g, r, st)
        assert abs(F[0].sum() - fl["Fx"].sum()) <= 1e-13 * np.abs(fl["Fx"]).sum()
        assert abs(F[1].sum() - fl["Fy"].sum()) <= 1e-13 * np.abs(fl["Fy"]).sum()


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_anchor_force_single_filament_closed_form(oracle_mod, k):
    """One filament density psi0 in one cell with orientation theta_k = k pi/2
    and a linear row M_j = a + b s_j, on a 6 x 6 grid with 12 nodes and
    l/L = 1/2. The head sits 0.5 + 3 s_j cells along p from the cell's lower
    edge, so nodes 0-3 land one cell behind, 4-7 in the cell, 8-11 one cell
    ahead (no node on a cell edge). With s_j = -1/2 + (j + 1/2)/12 the node
    sums are sum_{0-3} s_j = -4/3, sum_{4-7} s_j = 0, sum_{8-11} s_j = 4/3, so
    the three cells get F_m psi0 ds dtheta p (4a - 4b/3), (4a), (4a + 4b/3)
    and every other cell nothing."""
    g = Grid(6, 6, 4, 12)
    r = Rates(ell=0.5, force_scale=0.7)
    a, b, psi0 = 0.3, 0.4, 2.5
    iy0, ix0 = 2, 3
    ds, dth = g.L / g.ns, TWO_PI / g.ntheta
    sj = -0.5 + (np.arange(g.ns) + 0.5) / g.ns
    psi = np.zeros((g.ny, g.nx, g.ntheta))
    psi[iy0, ix0, k] = psi0
    mb = np.zeros((g.ny, g.nx, g.ntheta, g.ns))
    mb[iy0, ix0, k] = a + b * sj
    st = oracle_mod.make_state_anchor(g, r, psi, mb, np.full((g.ny, g.nx), 1e9))
    F = oracle_mod.anchor_force(g, r, st)
    step = [(1, 0), (0, 1), (-1, 0), (0, -1)][k]  # p_k rounded to the grid
    w = r.force_scale * psi0 * ds * dth
    expect = np.zeros((2, g.ny, g.nx))
    for back_or_ahead, total in ((-1, 4 * a - 4 * b / 3), (0, 4 * a), (1, 4 * a + 4 * b / 3)):
        cy = (iy0 + back_or_ahead * step[1]) % g.ny
        cx = (ix0 + back_or_ahead * step[0]) % g.nx
        expect[0, cy, cx] = w * total * step[0]
        expect[1, cy, cx] = w * total * step[1]
    np.testing.assert_allclose(F, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dims", [(3, 2, 16, 8), (5, 4, 7, 5), (2, 3, 12, 11)])
def test_moments_brute_force(oracle_mod, dims):
    """Every moment field and global scalar on a random state with non-symmetric
    psi and rows, against its definition summed directly (numpy): rho, P, Q
    (xx, xy), C, Mf, F = F_m sum_k p psi n_b dtheta (Eq. 10 with anchors in the
    cell), sigma_a = F_m ell sum_k p p psi m1 dtheta with n_b = sum_j Mb ds and
    m1 = sum_j s_j Mb ds at s_j = -L/2 + (j + 1/2) ds, theta_k = k dtheta."""
    O = oracle_mod
    g = Grid(*dims, L=1.3)
    r = Rates(force_scale=0.8, ell=1.4)
    rng = np.random.default_rng(sum(dims))
    psi = rng.random((g.ny, g.nx, g.ntheta))
    mb = 0.1 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    st = O.make_state(g, psi, mb, mtot=rng.random((g.ny, g.nx)) + 0.5)
    f, sc = O.moments(g, r, st)
    dth, ds = TWO_PI / g.ntheta, g.L / g.ns
    th = np.arange(g.ntheta) * dth
    c, s = np.cos(th), np.sin(th)
    sj = -g.L / 2 + (np.arange(g.ns) + 0.5) * ds
    nb = st.mb.sum(-1) * ds
    m1 = (st.mb * sj).sum(-1) * ds
    P = st.psi
    ref = {
        "rho": P.sum(-1) * dth,
        "Px": (P * c).sum(-1) * dth, "Py": (P * s).sum(-1) * dth,
        "Qxx": (P * (c * c - 0.5)).sum(-1) * dth, "Qxy": (P * c * s).sum(-1) * dth,
        "C": st.c, "Mf": st.mf,
        "Fx": 0.8 * (P * nb * c).sum(-1) * dth, "Fy": 0.8 * (P * nb * s).sum(-1) * dth,
        "Sxx": 0.8 * 1.4 * (P * m1 * c * c).sum(-1) * dth,
        "Sxy": 0.8 * 1.4 * (P * m1 * c * s).sum(-1) * dth,
        "Syy": 0.8 * 1.4 * (P * m1 * s * s).sum(-1) * dth,
    }
    for k, v in ref.items():
        assert np.allclose(f[k], v, rtol=1e-12, atol=1e-15), k
    dA = 1.0 / (g.nx * g.ny)
    sum_cos, sum_sin = (P * c).sum(), (P * s).sum()
    ref_sc = {"N_psi": P.sum() * dth * dA, "bound": st.c.sum() * dA, "free": st.mf.sum() * dA,
              "motors": (st.c.sum() + st.mf.sum()) * dA,
              "polar_order": math.hypot(sum_cos, sum_sin) / P.sum(),
              "mean_stress": (ref["Sxx"] + ref["Syy"]).mean(),
              "sum_psi_cos": sum_cos, "sum_psi_sin": sum_sin}
    for k, v in ref_sc.items():
        assert sc[k] == pytest.approx(v, rel=1e-12, abs=1e-15), k
