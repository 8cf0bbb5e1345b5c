"""Lanczos coefficient files: the hand-off between the recursion (Sec. 3.2, which keeps the
coefficients beta_i, gamma_i and z_i) and the spectrum post-processing (Sec. 3.3).  A chain's
spectrum can then be evaluated later, extrapolated or not, or its coefficients inspected,
without the chain.

Format (text): one header line of key=value pairs, then one row per coefficient

    # ll-coefficients v1 omega_cell=<bohr^3> q=<qx>,<qy>,<qz> flavour=<ph|nh> approx=<name>
    i  beta_i  Re gamma_i  Im gamma_i  Re z_i  Im z_i

with index 0 holding b_1, as the arrays of ll_lanczos do.  Numbers are written with 17
significant digits, so a save/load round trip is exact.
"""
from __future__ import annotations

import numpy as np

MAGIC = "ll-coefficients v1"


def save(path, beta, gamma, z, omega_cell: float, q_cart, flavour: str = "ph", approx: str = "tddft"):
    """Writes the m coefficients (beta real [m], gamma and z complex [m]) of one chain."""
    b = np.asarray(beta, dtype=np.float64)
    g = np.asarray(gamma, dtype=np.complex128)
    zz = np.asarray(z, dtype=np.complex128)
    if not (b.ndim == g.ndim == zz.ndim == 1 and len(b) == len(g) == len(zz) and len(b) > 0):
        raise ValueError("beta, gamma and z must be 1-D arrays of the same non-zero length")
    q = np.asarray(q_cart, dtype=np.float64).reshape(3)
    for key, val in (("flavour", flavour), ("approx", approx)):
        if not val or any(c.isspace() or c == "=" for c in val):
            raise ValueError(f"{key} must be a single word")
    head = (f"{MAGIC} omega_cell={float(omega_cell):.17e} q={q[0]:.17e},{q[1]:.17e},{q[2]:.17e} "
            f"flavour={flavour} approx={approx}")
    rows = np.column_stack([np.arange(len(b)), b, g.real, g.imag, zz.real, zz.imag])
    np.savetxt(path, rows, fmt=["%d"] + ["%.17e"] * 5, header=head, comments="# ")


def load(path) -> dict:
    """Reads a file written by save: beta, gamma, z, omega_cell, q_cart, flavour, approx."""
    with open(path) as f:
        first = f.readline()
    if not first.startswith("# " + MAGIC):
        raise ValueError(f"{path}: not an {MAGIC} file")
    meta = dict(item.split("=", 1) for item in first[len("# " + MAGIC):].split())
    rows = np.loadtxt(path, comments="#", ndmin=2)
    if rows.shape[1] != 6 or not np.array_equal(rows[:, 0], np.arange(len(rows))):
        raise ValueError(f"{path}: malformed coefficient rows")
    return dict(beta=rows[:, 1].copy(), gamma=rows[:, 2] + 1j * rows[:, 3], z=rows[:, 4] + 1j * rows[:, 5],
                omega_cell=float(meta["omega_cell"]),
                q_cart=np.array([float(v) for v in meta["q"].split(",")]),
                flavour=meta["flavour"], approx=meta["approx"])
