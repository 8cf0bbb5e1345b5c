"""Pins of the coefficient extrapolation (oracle/extrapolation.py) against closed forms.

A semi-infinite chain with zero diagonal and constant hopping beta has the resolvent element
G(w) = (w - sqrt(w - 2 beta) sqrt(w + 2 beta)) / (2 beta^2); with hoppings alternating a, b,
a, b, ... (first hopping a), G1 = 1/(w - a^2 G2), G2 = 1/(w - b^2 G1) give the quadratic
w b^2 G1^2 - (w^2 - a^2 + b^2) G1 + w = 0 (the root with Im G1 < 0 for Im w > 0).  A chain
computed exactly for M steps and extrapolated to M' = 20000 must reproduce these within the
reflection from its far end, exp(-2 M' eta / v), negligible here.
"""
import numpy as np
import pytest

from oracle import spectrum
from oracle.extrapolation import extrapolate

W = np.linspace(-3.0, 3.0, 121)
ETA = 0.05


def _chain_g(beta, gamma, z):
    return spectrum.chi_lanczos(beta, gamma, z, W, ETA)


def test_constant_matches_semi_infinite_chain():
    b = 0.7
    m = 40
    beta = np.full(m, b)
    beta[0] = 1.0                      # b_1 = 1 so that chi_lanczos returns x_1
    z = np.zeros(m, dtype=complex)
    z[0] = 1.0
    be, ge, ze = extrapolate(beta, beta, z, "constant", 20000)
    w = W + 1j * ETA
    exact = (w - np.sqrt(w - 2 * b) * np.sqrt(w + 2 * b)) / (2 * b * b)
    assert np.max(np.abs(_chain_g(be, ge, ze) - exact)) < 1e-9
    # truncated at M the chain is visibly different inside the band
    assert np.max(np.abs(_chain_g(beta, beta, z) - exact)) > 1e-2


def test_osc_matches_alternating_chain():
    a, b = 0.6, 0.9
    m = 40
    beta = np.array([1.0] + [a if j % 2 == 1 else b for j in range(1, m)])
    z = np.zeros(m, dtype=complex)
    z[0] = 1.0
    be, ge, ze = extrapolate(beta, beta, z, "osc", 20000)
    w = W + 1j * ETA
    p = w * w - a * a + b * b
    disc = np.sqrt(p * p - 4 * w * w * b * b + 0j)
    roots = np.stack([(p - disc) / (2 * w * b * b), (p + disc) / (2 * w * b * b)])
    lower = roots.imag < 0
    assert np.all(lower.sum(axis=0) == 1)
    exact = np.where(lower[0], roots[0], roots[1])
    assert np.max(np.abs(_chain_g(be, ge, ze) - exact)) < 1e-9
    # a one-constant tail cannot represent the gap of the alternating chain
    bc, gc, zc = extrapolate(beta, beta, z, "constant", 20000)
    assert np.max(np.abs(_chain_g(bc, gc, zc) - exact)) > 1e-2


def test_averages_only_the_second_half():
    rng = np.random.default_rng(0)
    m = 30
    beta = np.concatenate([[2.0], rng.uniform(0.1, 3.0, m // 2 - 1), np.full(m - m // 2, 0.8)])
    be, _, ze = extrapolate(beta, beta, np.ones(m), "constant", m + 10)
    assert np.array_equal(be[:m], beta) and np.allclose(be[m:], 0.8, rtol=0, atol=1e-15)
    assert np.all(ze[m:] == 0) and np.all(ze[:m] == 1)
    # 'osc': each parity continues with its own mean
    beta2 = np.concatenate([[2.0], rng.uniform(0.1, 3.0, 13), np.tile([0.5, 1.5], 8)])
    bo, _, _ = extrapolate(beta2, beta2, np.ones(len(beta2)), "osc", len(beta2) + 6)
    tail = beta2[len(beta2) // 2:]
    pos = np.arange(len(beta2) // 2, len(beta2))
    ev, od = tail[pos % 2 == 0].mean(), tail[pos % 2 == 1].mean()
    idx = np.arange(len(beta2), len(beta2) + 6)
    assert np.allclose(bo[len(beta2):], np.where(idx % 2 == 0, ev, od), rtol=0, atol=1e-15)


def test_no_extrapolation_is_identity():
    beta = np.arange(1.0, 11.0)
    out = extrapolate(beta, beta, np.ones(10), "no", 100)
    assert all(len(x) == 10 for x in out)
    with pytest.raises(ValueError):
        extrapolate(beta, beta, np.ones(10), "linear", 100)
