"""Pins of the comparison windows of the parity tests (Sec. 2.5 recursions, Sec. 3.3
spectrum): how many Lanczos coefficients, and which spectrum, a rounding-level change of the
input leaves reproducible.

The oracle is rerun with the local potential scaled by (1 + 1e-14), a change the size of the
rounding differences between two correct arithmetics (another summation order, another
FFT).  A recursion that has converged on the discrete spectrum of a finite basis amplifies
such differences exponentially once the Krylov space stops growing, so a comparison of two
arithmetics is meaningful only inside the reproducible window:

  - tiny cell (2x2x2 k, ~1000 transitions): the first 40 coefficients agree to 1e-12, and the
    coefficients depart by more than 1e-10 before step 100;
  - small two-atom cell (4x4x4 k): the first 100 coefficients agree to 1e-12 and their loss
    function to 1e-10, while the loss function of all 300 coefficients moves by more than
    1e-4 -- eight orders of magnitude more -- so the 300-step loss function compares
    amplified rounding, not error;
  - the semimetal with smeared occupations (Sec. 2.6): rounding of FP32 size at every step
    (not a single input change) moves the oracle's own loss function of 100 coefficients by
    more than 1e-3 and that of 80 by less, so its FP32 window is 80 coefficients.
"""
import copy

import numpy as np
import pytest

import workloads as w
from oracle import lanczos, spectrum
from oracle.liouvillian import System

WGRID = np.linspace(0.0, 40.0, 4001)


def _perturbed(b, rel=1e-14):
    b2 = copy.copy(b)
    b2.vloc_r = b.vloc_r * (1.0 + rel)
    return b2


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


@pytest.mark.parametrize("approx", ["ipa", "rpa", "tddft"])
def test_tiny_cell_window(approx):
    b = w.get_bundle(w.config_tiny())
    a = lanczos.pseudo_hermitian(System(b, approx), 100)
    p = lanczos.pseudo_hermitian(System(_perturbed(b), approx), 100)
    r = _rel(p.beta, a.beta)
    assert r[:40].max() < 1e-12
    assert r.max() > 1e-10


def test_small_cell_window():
    b = w.get_bundle(w.config_small())
    a = lanczos.pseudo_hermitian(System(b), 300)
    p = lanczos.pseudo_hermitian(System(_perturbed(b)), 300)
    assert _rel(p.beta[:100], a.beta[:100]).max() < 1e-12

    def loss(co, m):
        _, ei, _ = spectrum.spectrum(co.beta[:m], co.gamma[:m], co.z[:m], b.spec.omega, b.spec.q_cart, WGRID, 0.1)
        return spectrum.loss(ei)

    d100 = np.max(np.abs(loss(a, 100) - loss(p, 100))) / np.max(np.abs(loss(a, 100)))
    d300 = np.max(np.abs(loss(a, 300) - loss(p, 300))) / np.max(np.abs(loss(a, 300)))
    assert d100 < 1e-10
    assert d300 > 1e-4


class _RoundedSteps(System):
    """The oracle with every new Lanczos vector perturbed elementwise by a relative complex
    noise of 6e-8 (the FP32 unit roundoff) before its projection: rounding of FP32 size at
    every step, as an FP32 recursion suffers it."""

    def __init__(self, b, seed, rel=6e-8):
        super().__init__(b)
        self._rng = np.random.default_rng(seed)
        self._rel = rel

    def project_c(self, x, ks=None):
        r = self._rng
        y = [xk * (1 + self._rel * (r.standard_normal(xk.shape) + 1j * r.standard_normal(xk.shape))) for xk in x]
        return super().project_c(y, ks)


def test_metal_fp32_window():
    """The semimetal (smeared occupations, Sec. 2.6) leaves a shorter window to an FP32
    recursion: with rounding of FP32 size at every step the oracle's own loss function of the
    first 80 coefficients moves by less than 1e-3 (measured 1e-5 to 1e-4 over two noise seeds),
    that of the first 100 by more than 1e-3 (measured 4e-3 to 2e-2), so FP32 parity on this
    cell is compared on the first 80 coefficients (for the insulating two-atom cell the same
    noise moves the 100-coefficient loss function by ~5e-4)."""
    from workloads.cells import config_metal
    b = w.get_bundle(config_metal())
    a = lanczos.pseudo_hermitian(System(b), 100)

    def loss(co, m):
        _, ei, _ = spectrum.spectrum(co.beta[:m], co.gamma[:m], co.z[:m], b.spec.omega, b.spec.q_cart, WGRID, 0.1)
        return spectrum.loss(ei)

    l80, l100 = loss(a, 80), loss(a, 100)
    for seed in (1, 2):
        p = lanczos.pseudo_hermitian(_RoundedSteps(b, seed), 100)
        assert np.max(np.abs(loss(p, 80) - l80)) / np.max(l80) < 1e-3
        assert np.max(np.abs(loss(p, 100) - l100)) / np.max(l100) > 1e-3
