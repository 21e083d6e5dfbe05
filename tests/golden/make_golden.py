"""Writes the oracle fixtures under tests/golden/ (run from the repository
root: python tests/golden/make_golden.py). Calls only oracle/ and the seeded
input generators; every value is the float64 oracle's, printed with 17
significant digits. The paper prints no worked example of the method's values,
so these fixtures pin the oracle against accidental change; its correctness is
pinned by tests/test_oracle_pins.py and tests/test_oracle_fluid.py.
"""
from __future__ import annotations

import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import fluid as FL  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64,  # noqa: E402
                                           psi_isotropic_perturbed, random_divfree_flow)


def fmt(a) -> str:
    return " ".join(f"{float(x):.17g}" for x in np.asarray(a, dtype=np.float64).ravel())


def substep_case():
    """Three substeps of the 4x4 x 4 x 4 seeded case (Eq. 1 and Alg. 2's RK2 of
    Eq. 4, then Eq. 5, the clip and Eq. 6), its dt and its moments (Eq. 10)."""
    g = Grid(4, 4, 4, 4)
    r = Rates(k_on=1.5, glide=0.1)
    psi = psi_isotropic_perturbed(g, 7, amp=0.3)
    mb = 0.2 * SplitMix64(8).uniforms(g.micro_cells).reshape(g.ny, g.nx, g.ntheta, g.ns)
    u = random_divfree_flow(g, 9, 4, 0.1)
    st = O.make_state(g, psi, mb)
    dt = O.dt(g, r, st, u)
    O.run(g, r, st, u, dt, 3)
    f, sc = O.moments(g, r, st)
    lines = ["# oracle: 3 substeps of Grid(4, 4, 4, 4), Rates(k_on=1.5, glide=0.1),",
             "# psi_isotropic_perturbed(g, 7, amp=0.3), mb = 0.2 SplitMix64(8) uniforms,",
             "# u = random_divfree_flow(g, 9, 4, 0.1); Eq. 1, Eq. 4 (Alg. 2), Eq. 5-6, Eq. 10",
             f"dt {dt:.17g}"]
    for k in ("psi", "mb", "mf", "c"):
        lines.append(f"{k} {fmt(getattr(st, k))}")
    for k in ("Fx", "Fy", "Sxx", "Sxy", "Syy"):
        lines.append(f"{k} {fmt(f[k])}")
    for k in ("N_psi", "polar_order", "mean_stress"):
        lines.append(f"{k} {sc[k]:.17g}")
    return "\n".join(lines) + "\n"


def fluid_case():
    """Per-mode responses of Eq. 7-9 (g_T, g_L at z0) and one velocity field."""
    lines = ["# oracle/fluid.py: (g_T, g_L) of Eq. 7-9 per |k|, force on the plane z = z0",
             "# kappa eps z0 g_T g_L"]
    for kappa in (0.0, 2 * math.pi, 20.0, 150.0):
        for eps, z0 in ((0.1, 0.1), (0.5, 0.3), (1.0, 0.25)):
            gT, gL = FL.mode_response(kappa, eps, z0)
            lines.append(f"mode {kappa:.17g} {eps:.17g} {z0:.17g} {gT:.17g} {gL:.17g}")
    rng = np.random.default_rng(13)
    F = rng.standard_normal((2, 4, 6))
    S = rng.standard_normal((3, 4, 6))
    u = FL.velocity(0.3, 0.2, F, S)
    lines.append("# velocity(eps=0.3, z0=0.2, F, S), F, S = default_rng(13) normals [2][4][6], [3][4][6]")
    lines.append(f"u {fmt(u)}")
    return "\n".join(lines) + "\n"


def main():
    O.build()
    with open(os.path.join(HERE, "oracle_substep_4x4x4x4.txt"), "w") as fh:
        fh.write(substep_case())
    with open(os.path.join(HERE, "oracle_fluid_modes.txt"), "w") as fh:
        fh.write(fluid_case())


if __name__ == "__main__":
    main()
