"""Post-processing of the Lanczos coefficients (Sec. 3.3; Eqs. 5, 30-33).

For each frequency, with omega -> omega + i eta (Lorentzian broadening, Sec. 3.3):
    ((omega + i eta) I - T_M) x = e_1          solved with LAPACK zgtsv
    chi(Q, omega) = (4 / Omega) b_1 sum_j z_j x_j
    eps^-1(Q, omega) = 1 + (4 pi / |Q|^2) chi   (Eq. 5, diagonal element)
    eps(Q, omega) = 1 / eps^-1                 (a scalar inverse, Sec. 2.1)
The factor 4/Omega turns ((y, 0), (omega - L)^-1 (0, y)), with the batch scalar product
that carries the 1/N_k k-weights, into the susceptibility per unit volume of a
spin-degenerate system (independent-particle check: one transition of weight |M|^2 and
energy Delta gives (4/Omega) w_k |M|^2 Delta / (omega^2 - Delta^2)).  No extrapolation of
the coefficients: T is truncated at M x M.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import lapack

from workloads import HA_EV


def tridiag_x(beta, gamma, w: complex) -> np.ndarray:
    """x = (w I - T)^-1 e_1 with T_{j+1,j} = beta[j], T_{j,j+1} = gamma[j] (j >= 1), zero diagonal."""
    m = len(beta)
    d = np.full(m, w, dtype=np.complex128)
    dl = -np.asarray(beta[1:], dtype=np.complex128)
    du = -np.asarray(gamma[1:], dtype=np.complex128)
    b = np.zeros(m, dtype=np.complex128)
    b[0] = 1.0
    _, _, _, x, info = lapack.zgtsv(dl.copy(), d, du.copy(), b)
    if info != 0:
        raise np.linalg.LinAlgError(f"zgtsv info={info}")
    return x


def chi_lanczos(beta, gamma, z, omega_ha: np.ndarray, eta_ha: float) -> np.ndarray:
    """b_1 sum_j z_j x_j(omega + i eta) -- the Lanczos estimate of ((y,0),(w - L)^-1 (0,y))."""
    b1 = float(np.real(beta[0]))
    return np.array([b1 * np.dot(z, tridiag_x(beta, gamma, w + 1j * eta_ha)) for w in omega_ha])


def spectrum(beta, gamma, z, omega_cell: float, q_cart, omega_ev: np.ndarray, eta_ev: float):
    """(chi, eps_inv, eps) on a frequency grid given in eV."""
    w = np.asarray(omega_ev, dtype=np.float64) / HA_EV
    chi = 4.0 / omega_cell * chi_lanczos(beta, gamma, z, w, eta_ev / HA_EV)
    q2 = float(np.dot(q_cart, q_cart))
    eps_inv = 1.0 + 4.0 * np.pi / q2 * chi
    return chi, eps_inv, 1.0 / eps_inv


def loss(eps_inv: np.ndarray) -> np.ndarray:
    return -np.imag(eps_inv)


def fsum_moment(omega_ev: np.ndarray, eps_inv: np.ndarray) -> float:
    """First frequency moment of the loss function, int omega (-Im eps^-1(omega)) d omega, by
    the trapezoid rule on the given grid (eV in, Ha^2 out).  The f-sum rule (Sec. 2.1) makes
    it (pi/2) omega_p^2 over all frequencies for a local potential."""
    w = np.asarray(omega_ev, dtype=np.float64) / HA_EV
    f = w * loss(np.asarray(eps_inv))
    return float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(w)))


def fsum_expected(nelec: float, omega_cell: float) -> float:
    """(pi/2) omega_p^2 with omega_p^2 = 4 pi n, n = nelec / Omega (Ha^2)."""
    return 0.5 * np.pi * 4.0 * np.pi * nelec / omega_cell


def default_grid() -> np.ndarray:
    """0-40 eV inclusive, 4001 points (0.01 eV step)."""
    return np.linspace(0.0, 40.0, 4001)
