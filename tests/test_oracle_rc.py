"""Pins of the oracle's finite capture radius (the anchor axis r0 of Mb kept,
Sec. 2's B_rc(r0), Eq. 4's capture indicator, Alg. 2 per r0).

Each test states what it pins and which slip it catches. Expected values come
from the one-anchor and local substeps (limits), closed forms, invariants, an
independent geometric membership test and an independent brute-force
expansion (tests/brute_force.py) -- never from the capture-radius oracle
itself.
"""
import math

import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, psi_isotropic_perturbed,
                                           random_divfree_flow)
from tests import brute_force

TWO_PI = 2.0 * math.pi


def _one_anchor_to_rc(mb, tpl):
    """Mb in the filament-major one-anchor layout [fy][fx][k][j] laid out on
    the template (anchor-major): entry (r0, line, q) = Mb[r0 - d][k][j0 + q]."""
    ny, nx = mb.shape[:2]
    out = np.zeros((ny, nx, tpl.nconf))
    for k, dx, dy, j0, ln, off in tpl.lines:
        for ay in range(ny):
            for ax in range(nx):
                out[ay, ax, off:off + ln] = mb[(ay - dy) % ny, (ax - dx) % nx, k, j0:j0 + ln]
    return out


def _rc_to_one_anchor(mbr, tpl, g):
    """Inverse of _one_anchor_to_rc where every node has one anchor."""
    out = np.zeros((g.ny, g.nx, g.ntheta, g.ns))
    for k, dx, dy, j0, ln, off in tpl.lines:
        for ay in range(g.ny):
            for ax in range(g.nx):
                out[(ay - dy) % g.ny, (ax - dx) % g.nx, k, j0:j0 + ln] = mbr[ay, ax, off:off + ln]
    return out


def test_rc_zero_length_zero_radius_is_the_local_substep(oracle_mod):
    """l/L = 0 and rc = 0: every head is at its filament's centre, the only
    anchor is the filament's own cell and each row is one walking line: the
    capture-radius substep equals the local substep bit for bit (flow,
    gliding, walking, a forced scale-down). Fails for a wrong line boundary,
    a binding weight other than 1, or a coarse sum over the wrong cells."""
    O = oracle_mod
    g = Grid(6, 5, 8, 12)
    r = Rates(ell=0.0, k_on=40.0, glide=0.3)
    tpl = O.rc_template(g, r, 0.0)
    assert tpl.nconf == g.ntheta * g.ns and np.all(tpl.lines[:, 1:3] == 0)
    psi = psi_isotropic_perturbed(g, 201, amp=0.4)
    rng = np.random.default_rng(202)
    mb = 0.1 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    mtot = 0.05 + 0.1 * rng.random((g.ny, g.nx))
    u = random_divfree_flow(g, 203, 4, 0.2)
    a = O.make_state_rc(g, r, 0.0, psi, mb.reshape(g.ny, g.nx, -1), mtot)
    b = O.make_state(g, psi, mb, mtot)
    dt = O.dt(g, r, b, u) * 3.0
    clipped = False
    for _ in range(5):
        O.run_rc(g, r, 0.0, a, u, dt, 1)
        O.run(g, r, b, u, dt, 1)
        clipped = clipped or bool(np.any(b.mf == 0.0))
        assert np.array_equal(a.psi, b.psi)
        assert np.array_equal(a.mb.reshape(b.mb.shape), b.mb)
        assert np.array_equal(a.mf, b.mf) and np.array_equal(a.c, b.c)
    assert clipped  # the scale-down acted


def test_rc_zero_radius_without_walking_is_the_one_anchor_path(oracle_mod):
    """rc = 0 with l/L > 0: each node's only anchor is the cell under its head
    (no head on a cell edge here), as on the rc -> 0 path. Without walking the
    two models are the same map (they differ only in whether a walking motor
    keeps its tail): equal to round-off after 8 substeps with flow, gliding
    and a forced scale-down. Fails for a swapped anchor offset sign or a
    coarse density gathered at the filament instead of the anchor."""
    O = oracle_mod
    g = Grid(9, 7, 8, 12)
    r = Rates(ell=0.37, k_on=40.0, glide=0.3, v_walk=0.0)
    tpl = O.rc_template(g, r, 0.0)
    assert np.all(tpl.w == 1.0)
    psi = psi_isotropic_perturbed(g, 211, amp=0.4)
    rng = np.random.default_rng(212)
    mb = 0.1 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    mtot = 0.05 + 0.1 * rng.random((g.ny, g.nx))
    u = random_divfree_flow(g, 213, 4, 0.2)
    a = O.make_state_rc(g, r, 0.0, psi, _one_anchor_to_rc(mb, tpl), mtot)
    b = O.make_state_anchor(g, r, psi, mb, mtot)
    np.testing.assert_allclose(a.c, b.c, rtol=1e-14, atol=1e-15)
    dt = O.dt(g, Rates(ell=0.37, k_on=40.0, glide=0.3), b, u) * 3.0
    clipped = False
    for _ in range(8):
        O.run_rc(g, r, 0.0, a, u, dt, 1)
        O.run_anchor(g, r, b, u, dt, 1)
        clipped = clipped or bool(np.any(b.mf == 0.0))
    np.testing.assert_allclose(a.psi, b.psi, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(_rc_to_one_anchor(a.mb, tpl, g), b.mb, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(a.mf, b.mf, rtol=1e-12, atol=1e-15)
    assert clipped
    # with walking the models differ: here a motor lets go where its head
    # leaves the anchor's cell
    rw = Rates(ell=0.37, k_on=40.0, glide=0.3, v_walk=1.0)
    a2 = O.make_state_rc(g, rw, 0.0, psi, _one_anchor_to_rc(mb, tpl), mtot)
    b2 = O.make_state_anchor(g, rw, psi, mb, mtot)
    O.run_rc(g, rw, 0.0, a2, u, dt, 3)
    O.run_anchor(g, rw, b2, u, dt, 3)
    assert np.max(np.abs(_rc_to_one_anchor(a2.mb, tpl, g) - b2.mb)) > 1e-6


@pytest.mark.parametrize("dims,ell,rc", [((16, 12, 8, 10), 0.37, 0.09), ((10, 14, 6, 7), 0.8, 0.0),
                                         ((12, 12, 12, 16), 0.05, 0.2)])
def test_rc_template_is_the_capture_set(oracle_mod, dims, ell, rc):
    """The template's configurations are exactly those whose anchor cell's
    square lies within rc of the head (measured here by clamping the head onto
    each cell's square, for every cell of the grid), every (node, anchor) in
    one line, lines are maximal runs of consecutive nodes, the cell under the
    head is always in reach, and w = 1 / (anchors in reach of the node)."""
    g = Grid(*dims)
    r = Rates(ell=ell)
    tpl = oracle_mod.rc_template(g, r, rc)
    dx, dy = 1.0 / g.nx, 1.0 / g.ny
    seen = {}
    for k, ox, oy, j0, ln, off in tpl.lines:
        for j in range(j0, j0 + ln):
            assert (k, j, ox, oy) not in seen
            seen[(k, j, ox, oy)] = True
    offs = sorted({(int(a), int(b)) for a, b in tpl.lines[:, 1:3]})
    box = range(-g.nx, g.nx + 1)
    for k in range(g.ntheta):
        th = k * TWO_PI / g.ntheta
        for j in range(g.ns):
            s = -0.5 * g.L + (j + 0.5) * g.L / g.ns
            hx, hy = 0.5 * dx + ell * s * math.cos(th), 0.5 * dy + ell * s * math.sin(th)
            n_a = 0
            for ox in box:
                for oy in range(-g.ny, g.ny + 1):
                    px = min(max(hx, ox * dx), (ox + 1) * dx)
                    py = min(max(hy, oy * dy), (oy + 1) * dy)
                    dist = math.hypot(hx - px, hy - py)
                    if abs(dist - rc) < 1e-12:
                        continue  # on the boundary of reach: either is right
                    inside = dist < rc or (rc == 0.0 and dist == 0.0)
                    assert inside == ((k, j, ox, oy) in seen), (k, j, ox, oy, dist)
                    n_a += inside
            assert (k, j, int(math.floor(hx / dx)), int(math.floor(hy / dy))) in seen
            assert tpl.w[k, j] == 1.0 / sum(1 for key in seen if key[0] == k and key[1] == j)
    # maximal runs: no two lines of one (k, offset) touch
    by = {}
    for k, ox, oy, j0, ln, off in tpl.lines:
        by.setdefault((k, ox, oy), []).append((j0, ln))
    for runs in by.values():
        runs.sort()
        for (a0, al), (b0, _) in zip(runs, runs[1:]):
            assert b0 > a0 + al
    assert offs


@pytest.mark.parametrize("ell,rc", [(0.3, 0.0), (0.25, 0.07), (0.6, 0.16)])
def test_rc_uniform_bind_unbind_closed_form(oracle_mod, ell, rc):
    """Uniform psi, no flow, no walking, no gliding: every anchor sees the
    same free motors, so each configuration relaxes as x^n / n_a(k, j) where
    x^n = M_inf (1 - r^n) is the lagged bind/unbind recursion of the local
    model (A = 1 - k_off dt + (k_off dt)^2 / 2, B = k_on dt (1 - k_off dt/2),
    r = A - B rho L): the binding is shared among the n_a anchors in reach
    and the n_a lines of a node add up to one local row. Fails for a binding
    weight of 1 (n_a times too much binding), or a coarse density that misses
    anchors."""
    O = oracle_mod
    g = Grid(10, 8, 8, 10)
    r = Rates(ell=ell, v_walk=0.0, glide=0.0, v_sp=0.0, k_on=1.7, k_off=0.6)
    tpl = O.rc_template(g, r, rc)
    psi = psi_isotropic_perturbed(g, 221, amp=0.0)
    st = O.make_state_rc(g, r, rc, psi)
    dt, n = 0.05, 30
    O.run_rc(g, r, rc, st, np.zeros((2, g.ny, g.nx)), dt, n)
    rho = psi[0, 0].sum() * TWO_PI / g.ntheta
    A = 1 - r.k_off * dt + (r.k_off * dt) ** 2 / 2
    B = r.k_on * dt * (1 - r.k_off * dt / 2)
    rr = A - B * rho * g.L
    x = B * 1.0 / (1 - A + B * rho * g.L) * (1 - rr ** n)
    for k, ox, oy, j0, ln, off in tpl.lines:
        expect = x * tpl.w[k, j0:j0 + ln]
        assert np.max(np.abs(st.mb[..., off:off + ln] - expect)) <= 1e-13 * x
    nb, _ = O.rows_rc(g, r, rc, st)
    np.testing.assert_allclose(nb, g.L * x, rtol=1e-13)
    np.testing.assert_allclose(st.c, rho * g.L * x, rtol=1e-13)
    if rc > 0.1:
        assert tpl.w.min() < 0.2  # several anchors per node


def test_rc_lines_of_a_centred_filament_split_the_local_row(oracle_mod):
    """l/L = 0 with rc > 0: every node of a row reaches the same 9 anchors
    (the cell and its 8 neighbours at rc = 1.3 cells), so every row has 9
    full-length lines, each bound with 1/9 of the binding. With a uniform
    state the free motors stay uniform, and since the walking flux is
    positively homogeneous each line is the local row / 9 at all times (with
    walking on), and the lines add up to it. Fails for lines walked with the
    wrong boundaries or a weight other than 1 / n_a."""
    O = oracle_mod
    g = Grid(8, 8, 8, 16)
    r = Rates(ell=0.0, glide=0.0, v_sp=0.0, k_on=1.3, k_off=0.4, v_walk=1.1)
    rc = 1.3 / 8
    tpl = O.rc_template(g, r, rc)
    assert len(tpl.lines) == 9 * g.ntheta and np.all(tpl.lines[:, 4] == g.ns)
    psi = psi_isotropic_perturbed(g, 231, amp=0.0)
    a = O.make_state_rc(g, r, rc, psi)
    b = O.make_state(g, psi)
    u = np.zeros((2, g.ny, g.nx))
    O.run_rc(g, r, rc, a, u, 0.02, 25)
    O.run(g, r, b, u, 0.02, 25)
    for k, ox, oy, j0, ln, off in tpl.lines:
        np.testing.assert_allclose(9.0 * a.mb[..., off:off + ln], b.mb[:, :, k, :],
                                   rtol=1e-12, atol=1e-16)
    nb, _ = O.rows_rc(g, r, rc, a)
    np.testing.assert_allclose(nb, b.mb.sum(-1) * g.L / g.ns, rtol=1e-13)
    np.testing.assert_allclose(a.mf, b.mf, rtol=1e-13)


def test_rc_conservation(oracle_mod):
    """With flow, gliding and walking: free plus coarse equals the total at
    every anchor, the coarse density recomputed from the exported state
    (sum over B_rc(r0) of psi Mb ds dth) equals C, and the filament number is
    conserved."""
    O = oracle_mod
    g = Grid(12, 10, 8, 10)
    r = Rates(ell=0.3, k_on=2.0, glide=0.2)
    rc = 0.11
    tpl = O.rc_template(g, r, rc)
    rng = np.random.default_rng(241)
    psi = psi_isotropic_perturbed(g, 242, amp=0.4)
    st = O.make_state_rc(g, r, rc, psi, 0.05 * rng.random((g.ny, g.nx, tpl.nconf)))
    u = random_divfree_flow(g, 243, 4, 0.2)
    dt = O.dt(g, r, O.make_state(g, psi), u)
    N0 = st.psi.sum()
    O.run_rc(g, r, rc, st, u, dt, 12)
    assert abs(st.psi.sum() - N0) <= 1e-14 * N0
    np.testing.assert_allclose(st.mf + st.c, st.mtot, rtol=0, atol=1e-15)
    ds, dth = g.L / g.ns, TWO_PI / g.ntheta
    C = np.zeros((g.ny, g.nx))
    for k, ox, oy, j0, ln, off in tpl.lines:
        filament_psi = np.roll(np.roll(st.psi[:, :, k], oy, axis=0), ox, axis=1)
        C += filament_psi * st.mb[..., off:off + ln].sum(-1) * ds * dth
    np.testing.assert_allclose(C, st.c, rtol=1e-13)


@pytest.mark.parametrize("dims,ell,rc", [((5, 4, 4, 5), 0.317, 0.1073), ((6, 6, 6, 6), 0.413, 0.1231)])
def test_rc_brute_force_agrees(oracle_mod, dims, ell, rc):
    """An independent expansion -- configurations found by measuring every
    head's distance to every cell's square, walking between members only,
    binding shared among the anchors in reach, coarse density, scale-down and
    free motors per anchor -- agrees with the oracle on its configuration set
    and, after one substep with flow, gliding, walking and a forced
    scale-down, on every value."""
    O = oracle_mod
    g = Grid(*dims)
    r = Rates(ell=ell, k_on=25.0, glide=0.3, v_walk=0.9)
    tpl = O.rc_template(g, r, rc)
    members = brute_force.capture_sets(g, r, rc)
    keys = []
    for k, ox, oy, j0, ln, off in tpl.lines:
        for ay in range(g.ny):
            for ax in range(g.nx):
                for q in range(ln):
                    keys.append((ax, ay, (ax - ox) % g.nx, (ay - oy) % g.ny, int(k), int(j0 + q)))
    assert len(keys) == len(set(keys)) == len(members)
    assert set(keys) == members
    rng = np.random.default_rng(sum(dims))
    psi = psi_isotropic_perturbed(g, 251, amp=0.5)
    mb = rng.random((g.ny, g.nx, tpl.nconf)) / tpl.nconf
    mtot = 0.01 + 0.05 * rng.random((g.ny, g.nx))
    u = random_divfree_flow(g, 252, 3, 0.3)
    st = O.make_state_rc(g, r, rc, psi, mb, mtot)
    before = st.copy()
    dt = O.dt(g, r, O.make_state(g, psi), u) * 4.0
    O.run_rc(g, r, rc, st, u, dt, 1)

    def key_index():
        idx = {}
        for k, ox, oy, j0, ln, off in tpl.lines:
            for ay in range(g.ny):
                for ax in range(g.nx):
                    for q in range(ln):
                        idx[(ax, ay, (ax - ox) % g.nx, (ay - oy) % g.ny, int(k), int(j0 + q))] = (
                            ay, ax, off + q)
        return idx

    idx = key_index()
    mbd = {key: before.mb[i] for key, i in idx.items()}
    bp, bm, bf, bc = brute_force.substep_rc(g, r, rc, dt, u.tolist(), before.psi.tolist(), mbd,
                                            before.mf.tolist(), before.mtot.tolist())
    np.testing.assert_allclose(st.psi, np.array(bp), rtol=1e-12, atol=1e-14)
    got = np.array([st.mb[idx[key]] for key in bm])
    np.testing.assert_allclose(got, np.array(list(bm.values())), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st.mf, np.array(bf), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st.c, np.array(bc), rtol=1e-12, atol=1e-14)
    clipped = np.array(bc) == before.mtot
    assert np.any(clipped) and not np.all(clipped)


@pytest.mark.parametrize("dims,ell,rc", [((5, 4, 8, 6), 0.23, 0.071), ((8, 9, 6, 9), 0.55, 0.093)])
def test_rc_force_at_the_heads(oracle_mod, dims, ell, rc):
    """Eq. 10 with the capture radius: every configuration's force acts in the
    cell under its head, whatever its anchor. Against an independent deposit
    (each head located from its geometry, the motors per node summed over its
    anchors first), and its grid total against the local force total
    F sum p psi n_b dth with n_b summed over the anchors; the moments' force
    fields are this force and the rest of the moments take n_b and m1 summed
    over the anchors."""
    O = oracle_mod
    g = Grid(*dims)
    r = Rates(ell=ell, force_scale=0.7)
    tpl = O.rc_template(g, r, rc)
    rng = np.random.default_rng(261)
    psi = rng.random((g.ny, g.nx, g.ntheta))
    st = O.make_state_rc(g, r, rc, psi, rng.random((g.ny, g.nx, tpl.nconf)),
                         np.full((g.ny, g.nx), 1e9))
    F = O.force_rc(g, r, rc, st)
    # motors per node (filament cell, k, j), summed over anchors
    per_node = np.zeros((g.ny, g.nx, g.ntheta, g.ns))
    for k, ox, oy, j0, ln, off in tpl.lines:
        for ay in range(g.ny):
            for ax in range(g.nx):
                per_node[(ay - oy) % g.ny, (ax - ox) % g.nx, k, j0:j0 + ln] += st.mb[ay, ax,
                                                                                     off:off + ln]
    B = np.array(brute_force.anchor_force(g, r, st.psi.tolist(), per_node.tolist()))
    np.testing.assert_allclose(F, B, rtol=1e-12, atol=1e-14)
    nb, m1 = O.rows_rc(g, r, rc, st)
    ds, dth = g.L / g.ns, TWO_PI / g.ntheta
    np.testing.assert_allclose(nb, per_node.sum(-1) * ds, rtol=1e-13)
    s = -0.5 * g.L + (np.arange(g.ns) + 0.5) * ds
    np.testing.assert_allclose(m1, (per_node * s).sum(-1) * ds, rtol=1e-12, atol=1e-14)
    th = np.arange(g.ntheta) * dth
    total = r.force_scale * np.array([(np.cos(th) * psi * nb).sum(), (np.sin(th) * psi * nb).sum()])
    np.testing.assert_allclose(F.sum(axis=(1, 2)), total * dth, rtol=1e-12)
    f, sc = O.moments_rc(g, r, rc, st)
    np.testing.assert_allclose(f["Fx"], F[0], rtol=0, atol=0)
    np.testing.assert_allclose(f["Fy"], F[1], rtol=0, atol=0)
    sxx = r.force_scale * r.ell * (np.cos(th) ** 2 * psi * m1).sum(-1) * dth
    np.testing.assert_allclose(f["Sxx"], sxx, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(sc["bound"], st.c.sum() / (g.nx * g.ny), rtol=1e-13)


def test_rc_refuses_a_reach_wider_than_the_grid(oracle_mod):
    """Two template offsets that name the same cell of a periodic grid would
    make one configuration two: refused."""
    with pytest.raises(RuntimeError):
        oracle_mod.rc_template(Grid(4, 4, 4, 8), Rates(ell=0.9), 0.3)
