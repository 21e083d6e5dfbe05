"""The oracle against its stored fixtures (tests/golden/, written by
tests/golden/make_golden.py from the oracle itself): a change of the oracle's
arithmetic shows up here. Relative tolerance 1e-12 (libm and scipy may round
differently on another host)."""
import math
import os

import numpy as np
import pytest

from tests.golden.make_golden import fluid_case, substep_case

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse(text):
    out = {}
    for line in text.splitlines():
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out.setdefault(key, []).append(np.array([float(v) for v in vals]))
    return out


@pytest.mark.parametrize("name,make", [("oracle_substep_4x4x4x4.txt", substep_case),
                                       ("oracle_fluid_modes.txt", fluid_case)])
def test_oracle_reproduces_fixture(oracle_mod, name, make):
    stored = parse(open(os.path.join(HERE, name)).read())
    fresh = parse(make())
    assert stored.keys() == fresh.keys()
    for key in stored:
        for a, b in zip(stored[key], fresh[key]):
            assert a.shape == b.shape, key
            scale = max(np.abs(a).max(), 1e-300)
            assert np.abs(a - b).max() <= 1e-12 * scale, (key, np.abs(a - b).max() / scale)
    assert all(math.isfinite(v) for arr in stored.values() for row in arr for v in row)
