"""Pins of the oracle's LDA (Slater + PZ81) against the mathematics that fixes it."""
import numpy as np

from oracle import xc
from workloads import lda_vxc


DENS = np.array([1e-4, 3e-3, 0.01, 0.03, 0.08, 0.2, 0.5, 2.0])


def _n_at_rs(rs):
    return 3.0 / (4.0 * np.pi * rs ** 3)


def test_vxc_is_derivative_of_energy_density():
    h = 1e-6
    e = lambda n: n * xc.exc(n)
    fd = (e(DENS * (1 + h)) - e(DENS * (1 - h))) / (2 * h * DENS)
    assert np.allclose(xc.vxc(DENS), fd, rtol=1e-7, atol=0)


def test_fxc_is_derivative_of_vxc():
    h = 1e-5
    fd = (xc.vxc(DENS * (1 + h)) - xc.vxc(DENS * (1 - h))) / (2 * h * DENS)
    assert np.allclose(xc.fxc(DENS), fd, rtol=1e-6, atol=0)


def test_exchange_closed_form():
    # Slater exchange: e_x = -(3/4)(3 n/pi)^(1/3); remove correlation by subtracting eps_c
    n = DENS
    ex = xc.exc(n) - xc.eps_c(xc.rs_of_n(n))
    assert np.allclose(ex, -0.75 * (3 * n / np.pi) ** (1 / 3), rtol=1e-14)
    # r_s form: e_x = -0.458165293283143 / r_s  (3/4 (9/(4 pi^2))^(1/3))
    assert np.allclose(ex * xc.rs_of_n(n), -0.75 * (9 / (4 * np.pi ** 2)) ** (1 / 3), rtol=1e-13)


def test_pz81_continuity_at_rs_1():
    lo, hi = xc.eps_c(np.array([1 - 1e-12])), xc.eps_c(np.array([1.0]))
    assert abs(lo[0] - hi[0]) < 1e-4          # the published parameters match to ~1e-5 Ha
    vlo = xc.vxc(np.array([_n_at_rs(1 - 1e-12)]))
    vhi = xc.vxc(np.array([_n_at_rs(1.0)]))
    assert abs(vlo[0] - vhi[0]) < 1e-4


def test_high_density_limit_coefficient():
    # r_s -> 0: e_c -> A ln r_s + B  (Gell-Mann-Brueckner), A = 0.0311
    rs = np.array([1e-6, 2e-6])
    slope = (xc.eps_c(rs[1:]) - xc.eps_c(rs[:1])) / np.log(2.0)
    assert abs(slope[0] - 0.0311) < 1e-6


def test_independent_vxc_implementations_agree():
    # the ground-state generator carries its own PZ81 potential
    assert np.allclose(lda_vxc(DENS), xc.vxc(DENS), rtol=1e-13, atol=1e-15)


def test_fxc_threshold():
    assert xc.fxc(np.array([0.0, 1e-11]))[0] == 0.0
    assert xc.fxc(np.array([1e-11]))[0] == 0.0
