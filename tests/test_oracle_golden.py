"""The oracle against its regression anchors in tests/golden/ (written by
tests/golden/write_oracle_golden.py from the oracle itself; the external pins are the closed
forms of the other test_oracle_* files).  A failure means the oracle or the seeded input
generator changed: justify the change by the paper, then rewrite the anchors."""
import os

import numpy as np
import pytest

from tests.golden import write_oracle_golden as gold

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", sorted(gold.CASES))
def test_oracle_matches_its_anchor(name):
    approx, flavour = gold.CASES[name]
    want = np.loadtxt(os.path.join(HERE, name))
    co = gold.compute(approx, flavour)
    assert want.shape == (gold.STEPS, 6)
    got = np.column_stack([co.beta, co.gamma.real, co.gamma.imag, co.z.real, co.z.imag])
    scale = np.max(np.abs(want[:, 1:]), axis=0)
    # the ground state is rebuilt by LAPACK on whatever machine runs this: rounding-level
    # differences grow slowly along the recursion
    assert np.all(np.abs(got - want[:, 1:]) <= 1e-8 * scale + 1e-14)
