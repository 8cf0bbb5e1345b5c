"""Parity of the CUDA path with the FP64 oracle on the benchmark workloads at full size, through
the C ABI:

  - the KB workload: two-atom cell + KB s/p projectors, 25 Ry, 32^3, 8x8x8 k-points, 4 bands
    (2048 response orbitals), both recursions (Sec. 2.5);
  - the sixteen-atom cell: 2x2x2 supercell + KB (64 projectors), 30 Ry, 48^3, 4x4x4 k-points,
    32 bands, pseudo-Hermitian; its per-k work takes the split path, whose P_c and KB
    projections run on the tensor cores in the FP32 path.

Reference coefficients: tests/golden/oracle_<case>.txt, written by the oracle alone
(tests/golden/write_workload_golden.py), used when this machine's ground-state bundle is the
very input they were computed on (same digest).  A bundle rebuilt here by another LAPACK
differs in its last bits; the oracle then runs here, on every core (oracle.pool), on that
bundle.

Criteria: FP64 path, the first 100 coefficients to 1e-10 relative; every path, the loss
function -Im eps^-1 of the first 100 coefficients to 1e-3 relative L-infinity of its peak
(0-40 eV, 4001 points, eta = 0.1 eV; the reproducible window, tests/test_oracle_window.py).
"""
from types import SimpleNamespace

import numpy as np
import pytest

import workloads as w
from oracle import pool, spectrum
from tests.golden import write_workload_golden as gold

from .helpers import chain_from_bundle

pytestmark = pytest.mark.gpu

WGRID = np.linspace(0.0, 40.0, 4001)
ETA = 0.1
M = 100


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    return ll


@pytest.fixture(scope="module")
def kb():
    return w.get_bundle(w.config_kb())


@pytest.fixture(scope="module")
def sc16():
    b = w.cached_bundle(w.config_sc16())
    if b is None:
        pytest.skip("sixteen-atom ground state not cached (workloads.get_bundle(config_sc16()): ~35 min of CPU)")
    return b


_REF = {}


def _reference(case, bundle, n, n_live=None):
    """The oracle's first n coefficients of `case` on `bundle`: the golden file when its digest
    matches, else the oracle run here (first n_live coefficients, default n)."""
    key = (case, n)
    if key not in _REF:
        g = gold.load(case)
        if g is not None and g[1] >= n and g[0] == w.bundle_digest(bundle):
            _REF[key] = SimpleNamespace(beta=g[2][:n], gamma=g[3][:n], z=g[4][:n], source="golden")
        else:
            mk, flavour, _ = gold.CASES[case]
            nl = n_live or n
            co, _, _ = pool.run(mk(), nl, flavour)
            _REF[key] = SimpleNamespace(beta=co.beta, gamma=co.gamma, z=co.z, source="live")
    return _REF[key]


def _coef_rel(got, want, n):
    n = min(n, len(want.beta))
    b = np.max(np.abs(got[0][:n] - want.beta[:n]) / np.abs(want.beta[:n]))
    g = np.max(np.abs(got[1][:n] - want.gamma[:n]) / np.abs(want.gamma[:n]))
    z = np.max(np.abs(got[2][:n] - want.z[:n])) / np.max(np.abs(want.z[:n]))
    return max(b, g, z)


def _loss_err(got, want, b, m):
    m = min(m, len(want.beta))
    s = b.spec
    _, eg, _ = spectrum.spectrum(got[0][:m], got[1][:m], got[2][:m], s.omega, s.q_cart, WGRID, ETA)
    _, ew, _ = spectrum.spectrum(want.beta[:m], want.gamma[:m], want.z[:m], s.omega, s.q_cart, WGRID, ETA)
    lg, lw = spectrum.loss(eg), spectrum.loss(ew)
    return np.max(np.abs(lg - lw)) / np.max(np.abs(lw))


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_kb_workload_fp64_first_100(lib, kb, flavour):
    ref = _reference("kb_" + flavour, kb, M)
    got = chain_from_bundle(kb, flavour=flavour, precision="fp64", max_steps=M).lanczos(M)
    assert _coef_rel(got, ref, M) < 1e-10, ref.source
    assert _loss_err(got, ref, kb, M) < 1e-3


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_kb_workload_fp32_spectrum(lib, kb, flavour):
    """The FP32 path (the benchmark's headline arithmetic) in both recursions."""
    ref = _reference("kb_" + flavour, kb, M)
    got = chain_from_bundle(kb, flavour=flavour, precision="fp32", max_steps=M).lanczos(M)
    assert _loss_err(got, ref, kb, M) < 1e-3, ref.source
    assert _coef_rel(got, ref, 10) < 1e-4


def test_sc16_fp64_first_coefficients(lib, sc16):
    ref = _reference("sc16_ph", sc16, M, n_live=30)
    n = len(ref.beta)
    got = chain_from_bundle(sc16, precision="fp64", max_steps=n).lanczos(n)
    assert _coef_rel(got, ref, n) < 1e-10, ref.source


def test_sc16_fp32_spectrum(lib, sc16):
    """FP32 FFTs, tensor-core BF16-split P_c and KB projections, FP64 scalars."""
    ref = _reference("sc16_ph", sc16, M, n_live=30)
    n = len(ref.beta)
    got = chain_from_bundle(sc16, precision="fp32", max_steps=n).lanczos(n)
    assert _loss_err(got, ref, sc16, n) < 1e-3, ref.source
    assert _coef_rel(got, ref, 10) < 1e-4


def _golden_or_skip(case, bundle, n):
    g = gold.load(case)
    if g is None or g[1] < n or g[0] != w.bundle_digest(bundle):
        pytest.skip(f"no golden {case} coefficients for this bundle (a live oracle run of {n} steps takes too long)")
    return SimpleNamespace(beta=g[2][:n], gamma=g[3][:n], z=g[4][:n])


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_kb_workload_fp64_first_300(lib, kb, flavour):
    """FP64 against the oracle's whole 1000-step chains: the first 300 coefficients to 1e-10
    (measured 3e-15 in both recursions) and their loss function to 1e-3."""
    ref = _golden_or_skip("kb_" + flavour, kb, 1000)
    got = chain_from_bundle(kb, flavour=flavour, precision="fp64", max_steps=300).lanczos(300)
    assert _coef_rel(got, ref, 300) < 1e-10
    assert _loss_err(got, ref, kb, 300) < 1e-3


def test_kb_workload_fp64_full_length_ph(lib, kb):
    """All 1000 pseudo-Hermitian steps of the configuration, FP64: the loss function of the
    whole chain to 1e-3 of the oracle's (measured 6.5e-5; beyond ~300 steps both arithmetics
    amplify their rounding, so the coefficients themselves are compared over 300 steps)."""
    ref = _golden_or_skip("kb_ph", kb, 1000)
    got = chain_from_bundle(kb, flavour="ph", precision="fp64", max_steps=1000).lanczos(1000)
    assert _loss_err(got, ref, kb, 1000) < 1e-3
