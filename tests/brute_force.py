"""Deliberately naive pure-Python expansion of one substep, for tiny grids.

It is written independently of the oracle and in a different form, so that a
slip in either shows up as a disagreement:
  * psi transport is done in scatter form: every face flux is subtracted from
    the donor side and added to the receiving side;
  * the Superbee slope uses the ratio form phi(r) = max(0, min(2r,1), min(r,2))
    times the forward difference (equal to the division-free form wherever the
    forward difference is non-zero, and zero otherwise);
  * the RK2 midpoint stages are applied to the whole motor array at once;
  * every trigonometric value is recomputed where it is used.
Model: Eq. 1-6 of the paper with the readings listed in the oracle's header.
"""
from __future__ import annotations

import math


def _phi_superbee(r: float) -> float:
    return max(0.0, min(2.0 * r, 1.0), min(r, 2.0))


def _slope(back: float, fwd: float) -> float:
    if fwd == 0.0:
        return 0.0
    return _phi_superbee(back / fwd) * fwd


def substep(grid, rates, dt, u, psi, mb, mf, mtot):
    """One substep on nested Python lists; returns (psi, mb, mf, c) new lists.
    psi[iy][ix][k], mb[iy][ix][k][j], u[c][iy][ix], mf/mtot[iy][ix]."""
    nx, ny, nth, ns, L = grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L
    dx, dy, dth, ds = 1.0 / nx, 1.0 / ny, 2.0 * math.pi / nth, L / ns

    nb = [[[sum(mb[iy][ix][k][j] for j in range(ns)) * ds for k in range(nth)]
           for ix in range(nx)] for iy in range(ny)]

    def vel(ix, iy, k):
        V = rates.v_sp + rates.glide * nb[iy][ix][k]
        th = k * dth
        return (u[0][iy][ix] - V * math.cos(th), u[1][iy][ix] - V * math.sin(th))

    dpsi = [[[0.0] * nth for _ in range(nx)] for _ in range(ny)]

    def face(amount_vel, left, right, h):
        (lx, ly, lk), (rx, ry, rk) = left, right
        donor = psi[ly][lx][lk] if amount_vel > 0 else psi[ry][rx][rk]
        flux = amount_vel * donor
        dpsi[ly][lx][lk] -= dt * flux / h
        dpsi[ry][rx][rk] += dt * flux / h

    for iy in range(ny):
        for ix in range(nx):
            e = (ix + 1) % nx
            n = (iy + 1) % ny
            gxx = (u[0][iy][e] - u[0][iy][(ix - 1) % nx]) / (2 * dx)
            gxy = (u[0][n][ix] - u[0][(iy - 1) % ny][ix]) / (2 * dy)
            gyx = (u[1][iy][e] - u[1][iy][(ix - 1) % nx]) / (2 * dx)
            gyy = (u[1][n][ix] - u[1][(iy - 1) % ny][ix]) / (2 * dy)
            for k in range(nth):
                ax = 0.5 * (vel(ix, iy, k)[0] + vel(e, iy, k)[0])
                face(ax, (ix, iy, k), (e, iy, k), dx)
                ay = 0.5 * (vel(ix, iy, k)[1] + vel(ix, n, k)[1])
                face(ay, (ix, iy, k), (ix, n, k), dy)
                ph = (k + 0.5) * dth
                px, py = math.cos(ph), math.sin(ph)
                # p_perp . (G p), p_perp = (-py, px), (G p)_a = sum_b G_ab p_b
                om = -py * (gxx * px + gxy * py) + px * (gyx * px + gyy * py)
                face(om, (ix, iy, k), (ix, iy, (k + 1) % nth), dth)

    psi_new = [[[psi[iy][ix][k] + dpsi[iy][ix][k] for k in range(nth)] for ix in range(nx)]
               for iy in range(ny)]

    def rhs(M, mfree):
        out = []
        for j in range(ns):
            def flux_right(jj):
                if jj == ns - 1:
                    return rates.v_walk * M[jj]
                back = M[jj] - (M[jj - 1] if jj > 0 else 0.0)
                fwd = M[jj + 1] - M[jj]
                return rates.v_walk * (M[jj] + 0.5 * _slope(back, fwd))
            fin = flux_right(j - 1) if j > 0 else 0.0
            out.append(-(flux_right(j) - fin) / ds - rates.k_off * M[j] + rates.k_on * mfree)
        return out

    mb_new, c_new, mf_new = [], [], []
    for iy in range(ny):
        rowy_mb, rowy_c, rowy_mf = [], [], []
        for ix in range(nx):
            cell = []
            for k in range(nth):
                M = mb[iy][ix][k]
                k1 = rhs(M, mf[iy][ix])
                half = [M[j] + 0.5 * dt * k1[j] for j in range(ns)]
                k2 = rhs(half, mf[iy][ix])
                cell.append([M[j] + dt * k2[j] for j in range(ns)])
            coarse = sum(psi_new[iy][ix][k] * sum(cell[k]) * ds * dth for k in range(nth))
            if coarse > mtot[iy][ix]:
                scale = mtot[iy][ix] / coarse
                cell = [[v * scale for v in row] for row in cell]
                coarse = mtot[iy][ix]
            rowy_mb.append(cell)
            rowy_c.append(coarse)
            rowy_mf.append(mtot[iy][ix] - coarse)
        mb_new.append(rowy_mb)
        c_new.append(rowy_c)
        mf_new.append(rowy_mf)
    return psi_new, mb_new, mf_new, c_new


def head_cell(grid, rates, ix, iy, k, j):
    """(row, column) of the cell that holds the motor head of node j of a
    filament centred in cell (ix, iy) with orientation k: the centre plus
    (l/L) s_j p_k, located on the periodic grid by flooring its coordinates."""
    nx, ny, nth, ns, L = grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L
    s = -0.5 * L + (j + 0.5) * (L / ns)
    th = k * (2.0 * math.pi / nth)
    hx = (ix + 0.5) / nx + rates.ell * s * math.cos(th)
    hy = (iy + 0.5) / ny + rates.ell * s * math.sin(th)
    return int(math.floor(hy * ny)) % ny, int(math.floor(hx * nx)) % nx


def anchor_force(grid, rates, psi, mb):
    """Eq. 10 with the delta at the motor head: every node of every row puts
    its own force F p psi Mb_j ds dtheta into the cell under its own head.
    Returns [Fx, Fy] as nested lists [c][iy][ix]."""
    nx, ny, nth, ns, L = grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L
    dth, ds = 2.0 * math.pi / nth, L / ns
    F = [[[0.0] * nx for _ in range(ny)] for _ in range(2)]
    for iy in range(ny):
        for ix in range(nx):
            for k in range(nth):
                for j in range(ns):
                    hy, hx = head_cell(grid, rates, ix, iy, k, j)
                    w = rates.force_scale * psi[iy][ix][k] * mb[iy][ix][k][j] * ds * dth
                    F[0][hy][hx] += w * math.cos(k * dth)
                    F[1][hy][hx] += w * math.sin(k * dth)
    return F


def substep_anchor(grid, rates, dt, u, psi, mb, mf, mtot):
    """One substep with non-local motor anchors: a motor bound at node j of a
    filament in cell (ix, iy) with orientation k is anchored in the cell that
    contains its head, the filament centre plus (l/L) s_j p_k (found here by
    locating that point on the grid, periodic). Binding at node j takes the
    free motors of that cell; the coarse density, the scale-down and the free
    motors are formed per anchor cell. The psi transport is the one of
    substep() (anchors do not enter it)."""
    nx, ny, nth, ns, L = grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L
    dth, ds = 2.0 * math.pi / nth, L / ns
    # psi at the new time from the plain substep (its motor part is discarded)
    psi_new = substep(grid, rates, dt, u, psi, mb, mf, mtot)[0]

    def anchor(ix, iy, k, j):
        return head_cell(grid, rates, ix, iy, k, j)

    def rhs(M, mfree):
        out = []
        for j in range(ns):
            def flux_right(jj):
                if jj == ns - 1:
                    return rates.v_walk * M[jj]
                back = M[jj] - (M[jj - 1] if jj > 0 else 0.0)
                fwd = M[jj + 1] - M[jj]
                return rates.v_walk * (M[jj] + 0.5 * _slope(back, fwd))
            fin = flux_right(j - 1) if j > 0 else 0.0
            out.append(-(flux_right(j) - fin) / ds - rates.k_off * M[j] + rates.k_on * mfree[j])
        return out

    new = [[[None] * nth for _ in range(nx)] for _ in range(ny)]
    coarse = [[0.0] * nx for _ in range(ny)]
    for iy in range(ny):
        for ix in range(nx):
            for k in range(nth):
                M = mb[iy][ix][k]
                anc = [anchor(ix, iy, k, j) for j in range(ns)]
                mfree = [mf[ay][ax] for ay, ax in anc]
                k1 = rhs(M, mfree)
                half = [M[j] + 0.5 * dt * k1[j] for j in range(ns)]
                k2 = rhs(half, mfree)
                row = [M[j] + dt * k2[j] for j in range(ns)]
                new[iy][ix][k] = row
                for j, (ay, ax) in enumerate(anc):
                    coarse[ay][ax] += psi_new[iy][ix][k] * row[j] * ds * dth
    scale = [[1.0] * nx for _ in range(ny)]
    c_new = [[0.0] * nx for _ in range(ny)]
    mf_new = [[0.0] * nx for _ in range(ny)]
    for ay in range(ny):
        for ax in range(nx):
            cc = coarse[ay][ax]
            if cc > mtot[ay][ax]:
                scale[ay][ax] = mtot[ay][ax] / cc
                cc = mtot[ay][ax]
            c_new[ay][ax] = cc
            mf_new[ay][ax] = mtot[ay][ax] - cc
    for iy in range(ny):
        for ix in range(nx):
            for k in range(nth):
                new[iy][ix][k] = [v * scale[a][b] for v, (a, b) in
                                  zip(new[iy][ix][k], [anchor(ix, iy, k, j) for j in range(ns)])]
    return psi_new, new, mf_new, c_new


def _square_dist(hx, hy, ax, ay, grid):
    """Distance from the point (hx, hy) to the closed square of cell (ax, ay),
    over the periodic images of the unit square (nearest point by clamping)."""
    nx, ny = grid.nx, grid.ny
    best = math.inf
    for sx in (-1.0, 0.0, 1.0):
        for sy in (-1.0, 0.0, 1.0):
            x0, y0 = ax / nx + sx, ay / ny + sy
            px = min(max(hx, x0), x0 + 1.0 / nx)
            py = min(max(hy, y0), y0 + 1.0 / ny)
            best = min(best, math.hypot(hx - px, hy - py))
    return best


def capture_sets(grid, rates, rc):
    """{(ax, ay, fx, fy, k, j)}: every configuration of the capture-radius
    model -- anchor cell (ax, ay) within rc of the head of node j of a
    filament of orientation k centred in cell (fx, fy) -- found by measuring
    each head's distance to every cell's square directly."""
    nx, ny, nth, ns, L = grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L
    out = set()
    for fy in range(ny):
        for fx in range(nx):
            for k in range(nth):
                th = k * 2.0 * math.pi / nth
                for j in range(ns):
                    s = -0.5 * L + (j + 0.5) * (L / ns)
                    hx = (fx + 0.5) / nx + rates.ell * s * math.cos(th)
                    hy = (fy + 0.5) / ny + rates.ell * s * math.sin(th)
                    for ay in range(ny):
                        for ax in range(nx):
                            if _square_dist(hx, hy, ax, ay, grid) <= rc:
                                out.add((ax, ay, fx, fy, k, j))
    return out


def substep_rc(grid, rates, rc, dt, u, psi, mbd, mf, mtot):
    """One substep of the capture-radius model on a dict of configurations
    {(ax, ay, fx, fy, k, j): Mb} (every member of capture_sets present).
    psi by the plain substep; each motor keeps its anchor while it walks, so
    walking runs along j at fixed (anchor, filament, k) between members only
    (nothing walks in before a run, the last member of a run flows out);
    binding at a node is k_on Mf(anchor) divided by the number of anchors in
    reach of that node; then the coarse density, the scale-down and the free
    motors per anchor. Returns (psi, mbd, mf, c)."""
    nx, ny, nth, ns, L = grid.nx, grid.ny, grid.ntheta, grid.ns, grid.L
    dth, ds = 2.0 * math.pi / nth, L / ns
    nb = [[[0.0] * nth for _ in range(nx)] for _ in range(ny)]
    for (ax, ay, fx, fy, k, j), m in mbd.items():
        nb[fy][fx][k] += m * ds
    # psi at the new time from the plain substep, given these n_b (motor part
    # discarded): a one-node row per (cell, k) holding n_b / ds
    rows = [[[[nb[iy][ix][k] / ds] for k in range(nth)] for ix in range(nx)] for iy in range(ny)]
    g1 = type(grid)(nx, ny, nth, 1, ds)
    psi_new = substep(g1, rates, dt, u, psi, rows, mf, mtot)[0]
    count = {}
    for (ax, ay, fx, fy, k, j) in mbd:
        count[(fx, fy, k, j)] = count.get((fx, fy, k, j), 0) + 1

    def member(key):
        return key in mbd

    def rhs(vals):
        out = {}
        for key, m in vals.items():
            ax, ay, fx, fy, k, j = key
            left = (ax, ay, fx, fy, k, j - 1)
            right = (ax, ay, fx, fy, k, j + 1)

            def flux_right(kk):
                a_, b_, c_, d_, e_, jj = kk
                r_key = (a_, b_, c_, d_, e_, jj + 1)
                if not member(r_key):
                    return rates.v_walk * vals[kk]
                l_key = (a_, b_, c_, d_, e_, jj - 1)
                back = vals[kk] - (vals[l_key] if member(l_key) else 0.0)
                fwd = vals[r_key] - vals[kk]
                return rates.v_walk * (vals[kk] + 0.5 * _slope(back, fwd))

            fin = flux_right(left) if member(left) else 0.0
            out[key] = (-(flux_right(key) - fin) / ds - rates.k_off * m
                        + rates.k_on * mf[ay][ax] / count[(fx, fy, k, j)])
        return out

    k1 = rhs(mbd)
    half = {key: m + 0.5 * dt * k1[key] for key, m in mbd.items()}
    k2 = rhs(half)
    new = {key: m + dt * k2[key] for key, m in mbd.items()}
    coarse = [[0.0] * nx for _ in range(ny)]
    for (ax, ay, fx, fy, k, j), m in new.items():
        coarse[ay][ax] += psi_new[fy][fx][k] * m * ds * dth
    c_new = [[0.0] * nx for _ in range(ny)]
    mf_new = [[0.0] * nx for _ in range(ny)]
    scale = [[1.0] * nx for _ in range(ny)]
    for ay in range(ny):
        for ax in range(nx):
            cc = coarse[ay][ax]
            if cc > mtot[ay][ax]:
                scale[ay][ax] = mtot[ay][ax] / cc
                cc = mtot[ay][ax]
            c_new[ay][ax] = cc
            mf_new[ay][ax] = mtot[ay][ax] - cc
    new = {key: m * scale[key[1]][key[0]] for key, m in new.items()}
    return psi_new, new, mf_new, c_new
