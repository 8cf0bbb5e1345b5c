"""Writes the oracle regression anchors under tests/golden/ (run from the repository root:
`python tests/golden/write_oracle_golden.py`).

Each file holds the first 40 Lanczos coefficients the FP64 oracle computes on the seeded
tiny cell (two-atom FCC, 4 Ry, 12^3 grid, 2x2x2 k-points, 4 bands): b_1 and T_{j+1,j},
T_{j,j+1} and z_j of the pseudo-Hermitian recursion under ALDA and of the non-Hermitian
recursion under RPA (Sec. 2.5; operators of Eqs. 24-28).  They are not external numbers:
the oracle's pins are the closed forms in tests/test_oracle_*.py.  The files guard the oracle
(and the input generator) against unnoticed changes; regenerate them only with a change of
the oracle that a passage of the paper justifies.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as w                      # noqa: E402
from oracle import lanczos                 # noqa: E402
from oracle.liouvillian import System      # noqa: E402

STEPS = 40
CASES = {"oracle_tiny_tddft_ph.txt": ("tddft", "ph"), "oracle_tiny_rpa_nh.txt": ("rpa", "nh")}


def compute(approx: str, flavour: str):
    sys_ = System(w.get_bundle(w.config_tiny()), approx)
    return lanczos.run(sys_, STEPS, flavour)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for name, (approx, flavour) in CASES.items():
        co = compute(approx, flavour)
        rows = np.column_stack([np.arange(STEPS), co.beta, co.gamma.real, co.gamma.imag, co.z.real, co.z.imag])
        head = (f"oracle regression anchor: tiny cell, {approx}, {flavour}, {STEPS} steps "
                f"(written by tests/golden/write_oracle_golden.py)\n"
                "columns: i, beta[i], Re gamma[i], Im gamma[i], Re z[i], Im z[i]  (index 0: b_1; Sec. 2.5)")
        np.savetxt(os.path.join(here, name), rows, fmt=["%d"] + ["%.17e"] * 5, header=head)


if __name__ == "__main__":
    main()
