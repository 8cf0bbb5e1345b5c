"""Slater exchange + Perdew-Zunger 1981 correlation, unpolarised, Hartree units.

The paper uses the LDA with the Perdew-Zunger parametrisation (Sec. 5) and the adiabatic
XC kernel (Eq. 12: kappa_XC independent of frequency).  In the ALDA the kernel is local,
kappa_XC(r, r') = f_xc(n(r)) delta(r - r'), with f_xc = d v_xc / dn = d^2 (n e_xc) / dn^2.

Readings: f_xc = 0 where n <= 1e-10 bohr^-3; at r_s = 1 exactly the r_s >= 1 branch.
"""
from __future__ import annotations

import numpy as np

GAMMA, BETA1, BETA2 = -0.1423, 1.0529, 0.3334          # r_s >= 1
A, B, C, D = 0.0311, -0.048, 0.0020, -0.0116           # r_s < 1
N_MIN = 1e-10
CX = 0.75 * (3.0 / np.pi) ** (1.0 / 3.0)               # e_x = -CX n^(1/3)


def rs_of_n(n):
    return (3.0 / (4.0 * np.pi * n)) ** (1.0 / 3.0)


def eps_c(rs):
    rs = np.asarray(rs, dtype=np.float64)
    hi = rs >= 1.0
    out = np.empty_like(rs)
    out[hi] = GAMMA / (1.0 + BETA1 * np.sqrt(rs[hi]) + BETA2 * rs[hi])
    r = rs[~hi]
    out[~hi] = A * np.log(r) + B + C * r * np.log(r) + D * r
    return out


def deps_c_drs(rs):
    rs = np.asarray(rs, dtype=np.float64)
    hi = rs >= 1.0
    out = np.empty_like(rs)
    s = np.sqrt(rs[hi])
    den = 1.0 + BETA1 * s + BETA2 * rs[hi]
    out[hi] = -GAMMA * (BETA1 / (2.0 * s) + BETA2) / den ** 2
    r = rs[~hi]
    out[~hi] = A / r + C * (np.log(r) + 1.0) + D
    return out


def d2eps_c_drs2(rs):
    rs = np.asarray(rs, dtype=np.float64)
    hi = rs >= 1.0
    out = np.empty_like(rs)
    s = np.sqrt(rs[hi])
    den = 1.0 + BETA1 * s + BETA2 * rs[hi]
    dden = BETA1 / (2.0 * s) + BETA2
    d2den = -BETA1 / (4.0 * s ** 3)
    out[hi] = -GAMMA * (d2den * den - 2.0 * dden ** 2) / den ** 3
    r = rs[~hi]
    out[~hi] = -A / r ** 2 + C / r
    return out


def exc(n):
    """Energy per electron e_xc(n)."""
    n = np.asarray(n, dtype=np.float64)
    return -CX * n ** (1.0 / 3.0) + eps_c(rs_of_n(n))


def vxc(n):
    """v_xc = d(n e_xc)/dn = e_xc - (r_s/3) d e_xc/d r_s."""
    n = np.asarray(n, dtype=np.float64)
    rs = rs_of_n(n)
    vx = -4.0 / 3.0 * CX * n ** (1.0 / 3.0)
    vc = eps_c(rs) - rs / 3.0 * deps_c_drs(rs)
    return vx + vc


def fxc(n):
    """f_xc = d v_xc / dn, with d r_s/dn = -r_s/(3n).

    d v_c/d r_s = (2/3) e_c' - (r_s/3) e_c''.  Zero where n <= N_MIN."""
    n = np.asarray(n, dtype=np.float64)
    out = np.zeros_like(n)
    m = n > N_MIN
    nm = n[m]
    rs = rs_of_n(nm)
    fx = -4.0 / 9.0 * CX * nm ** (-2.0 / 3.0)
    dvc = 2.0 / 3.0 * deps_c_drs(rs) - rs / 3.0 * d2eps_c_drs2(rs)
    fc = dvc * (-rs / (3.0 * nm))
    out[m] = fx + fc
    return out
