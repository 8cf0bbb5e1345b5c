"""Extrapolation of the Lanczos coefficients (Sec. 2.5 end, Sec. 3.3, Appendix A), FP64.

Test infrastructure, like the rest of `oracle/`.  The paper extends the tridiagonal matrix
T_M computed in M Lanczos steps to a larger dimension M' at no cost by continuing its
off-diagonal coefficients, either with one constant ('constant') or with two constants that
alternate between odd and even positions ('osc', bi-constant), and leaves the method's details
to its references.  Readings used here (the paper is silent on them):

  - the constants are the means of the computed off-diagonal coefficients over the second
    half of the chain, positions h..M-1 with h = max(1, M // 2) in the array convention of
    `oracle.lanczos` (beta[0] = b_1 is the norm of the starting vector, not a matrix element,
    and is never averaged); 'osc' averages the even and the odd positions separately and
    continues each parity with its own mean;
  - gamma is continued the same way as beta (gamma = beta for the pseudo-Hermitian chain);
  - z_j = ((y, 0), v_j) is continued with zeros: the extra dimensions only reshape the
    resolvent's (j, 1) elements through the tail of T.
"""
from __future__ import annotations

import numpy as np

KINDS = ("no", "constant", "osc")


def _tail(a: np.ndarray, m: int, m_total: int, kind: str) -> np.ndarray:
    h = max(1, m // 2)
    idx = np.arange(m, m_total)
    if kind == "constant":
        return np.full(len(idx), np.mean(a[h:m]), dtype=a.dtype)
    pos = np.arange(h, m)
    even, odd = np.mean(a[h:m][pos % 2 == 0]), np.mean(a[h:m][pos % 2 == 1])
    return np.where(idx % 2 == 0, even, odd).astype(a.dtype)


def extrapolate(beta, gamma, z, kind: str, m_total: int):
    """(beta, gamma, z) continued from M = len(beta) to m_total entries (kind 'no': unchanged)."""
    if kind not in KINDS:
        raise ValueError(f"extrapolation must be one of {KINDS}")
    beta, gamma, z = np.asarray(beta), np.asarray(gamma), np.asarray(z)
    m = len(beta)
    if kind == "no" or m_total <= m:
        return beta, gamma, z
    if kind == "osc" and m < 4:
        raise ValueError("bi-constant extrapolation needs at least 4 coefficients")
    if m < 2:
        raise ValueError("extrapolation needs at least 2 coefficients")
    return (np.concatenate([beta, _tail(beta, m, m_total, kind)]),
            np.concatenate([gamma, _tail(gamma, m, m_total, kind)]),
            np.concatenate([z, np.zeros(m_total - m, dtype=z.dtype)]))
