"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the same
seeded ground-state bundles.

Tolerances: FP64 path, single operator application 1e-12 relative (rounding-order only);
first 100 Lanczos coefficients 1e-10 relative; every path's loss function 1e-3 relative
L-infinity of the peak.  FP32 path: one application 2e-5 relative (float FFTs of length
<= 32 in three passes: a few ulps of 6e-8 times the line length).  Index maps bit-exact.

Spectra are compared on the coefficients of the reproducible part of the recursion (the
first 100 steps, the same window as the coefficient criterion): past ~145 steps the
recursion amplifies rounding (a 1e-14 relative change of the local potential moves the
oracle's own 300-step loss function by ~1e-3, eight orders of magnitude more than its
100-coefficient loss function; pinned in tests/test_oracle_window.py), so a pointwise
comparison of two arithmetics there measures amplified rounding noise, not error.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import workloads as w
from oracle import lanczos, spectrum
from oracle.liouvillian import System

from .helpers import chain_from_bundle, rel_batch

pytestmark = pytest.mark.gpu

WGRID = np.linspace(0.0, 40.0, 4001)
ETA = 0.1


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    return ll


@pytest.fixture(scope="module")
def tiny():
    return w.get_bundle(w.config_tiny())


@pytest.fixture(scope="module")
def small():
    return w.get_bundle(w.config_small())


def _rand(sys, seed):
    rng = np.random.default_rng(seed)
    x = [rng.normal(size=(sys.nbnd, len(m))) + 1j * rng.normal(size=(sys.nbnd, len(m))) for m in sys.mkq]
    return sys.project_c(x)


M_SPEC = 100


def _loss_err(co_a, co_b, omega_cell, q, m=M_SPEC):
    _, ea, _ = spectrum.spectrum(co_a[0][:m], co_a[1][:m], co_a[2][:m], omega_cell, q, WGRID, ETA)
    _, eb, _ = spectrum.spectrum(co_b[0][:m], co_b[1][:m], co_b[2][:m], omega_cell, q, WGRID, ETA)
    la, lb = spectrum.loss(ea), spectrum.loss(eb)
    return np.max(np.abs(la - lb)) / np.max(np.abs(lb))


@pytest.mark.parametrize("cfg", ["tiny", "small"])
def test_index_map_bit_exact(lib, cfg, tiny, small):
    b = tiny if cfg == "tiny" else small
    sys = System(b)
    ch = chain_from_bundle(b, max_steps=4)
    got = ch.index_map()
    for g, r in zip(got, sys.map_k_kq):
        assert np.array_equal(g, r)


def test_start_vector(lib, small):
    sys = System(small)
    ch = chain_from_bundle(small, max_steps=4)
    assert rel_batch(ch.start_vector(), sys.starting_vector()) < 1e-13


@pytest.mark.parametrize("approx", ["ipa", "rpa", "tddft"])
@pytest.mark.parametrize("upper", [False, True])
def test_single_application_fp64(lib, small, approx, upper):
    sys = System(small, approx)
    ch = chain_from_bundle(small, approx=approx, max_steps=4)
    x = _rand(sys, 7)
    got = ch.apply(x, upper)
    want = sys.apply_op(x, upper)
    assert rel_batch(got, want) < 1e-12


@pytest.mark.parametrize("upper", [False, True])
def test_single_application_fp32(lib, small, upper):
    sys = System(small, "tddft")
    ch = chain_from_bundle(small, precision="fp32", max_steps=4)
    x = _rand(sys, 8)
    assert rel_batch(ch.apply(x, upper), sys.apply_op(x, upper)) < 2e-5


def test_single_application_tiny_nh_chain(lib, tiny):
    """The two-vector (non-Hermitian) chain reuses the same operator on one vector."""
    sys = System(tiny, "tddft")
    ch = chain_from_bundle(tiny, flavour="nh", max_steps=4)
    x = _rand(sys, 9)
    assert rel_batch(ch.apply(x, True), sys.apply_op(x, True)) < 1e-12


def _coef_rel(got, want, n):
    b = np.max(np.abs(got[0][:n] - want.beta[:n]) / np.abs(want.beta[:n]))
    g = np.max(np.abs(got[1][:n] - want.gamma[:n]) / np.abs(want.gamma[:n]))
    zs = np.max(np.abs(want.z[:n]))
    z = np.max(np.abs(got[2][:n] - want.z[:n])) / zs
    return max(b, g, z)


_ORACLE_RUNS = {}


def _oracle(bundle, flavour, n, n_run=300):
    """The oracle's first n coefficients (beta, gamma, z) on a bundle, in its own approximation.
    Each recursion is sequential, so the first n coefficients of a longer run are those of an
    n-step run: one run per bundle and flavour, of max(n, n_run) steps, serves every test."""
    key = (id(bundle), flavour)
    hit = _ORACLE_RUNS.get(key)
    if hit is None or hit[0] is not bundle or len(hit[1].beta) < n:
        hit = (bundle, lanczos.run(System(bundle), max(n, n_run), flavour))
        _ORACLE_RUNS[key] = hit
    co = hit[1]
    return SimpleNamespace(beta=co.beta[:n], gamma=co.gamma[:n], z=co.z[:n])


def test_ph_coefficients_small_fp64(lib, small):
    """Plain method, FP64: 300 pseudo-Hermitian steps (the small two-atom workload)."""
    ref = _oracle(small, "ph", 300)
    ch = chain_from_bundle(small, max_steps=300)
    got = ch.lanczos(300)
    assert _coef_rel(got, ref, 100) < 1e-10
    assert np.array_equal(ch.alpha, np.zeros(300))   # T has a zero diagonal (one SBR half per vector)
    assert _loss_err(got, (ref.beta, ref.gamma, ref.z), small.spec.omega, small.spec.q_cart) < 1e-3


def test_ph_resume_matches_single_call(lib, small):
    ch1 = chain_from_bundle(small, max_steps=60)
    a = ch1.lanczos(60)
    ch2 = chain_from_bundle(small, max_steps=60)
    ch2.lanczos(25)
    b = ch2.lanczos(35)
    assert len(b[0]) == 60
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_nh_coefficients_small_fp64(lib, small):
    ref = _oracle(small, "nh", 120)
    ch = chain_from_bundle(small, flavour="nh", max_steps=120)
    got = ch.lanczos(120)
    assert _coef_rel(got, ref, 100) < 1e-10


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_fp32_spectrum_small(lib, small, flavour):
    ref = _oracle(small, flavour, 300)
    ch = chain_from_bundle(small, flavour=flavour, precision="fp32", max_steps=300)
    got = ch.lanczos(300)
    assert _loss_err(got, (ref.beta, ref.gamma, ref.z), small.spec.omega, small.spec.q_cart) < 1e-3


@pytest.mark.parametrize("approx", ["ipa", "rpa"])
def test_other_approximations_tiny(lib, tiny, approx):
    """The tiny cell's space (~1000 transitions) is small enough that rounding-level input
    changes make its coefficients depart by more than 1e-10 before step 100 (between steps 80
    and 90; tests/test_oracle_window.py); the first 40, reproducible to 1e-12, are compared."""
    sys = System(tiny, approx)
    ref = lanczos.pseudo_hermitian(sys, 40)
    got = chain_from_bundle(tiny, approx=approx, max_steps=40).lanczos(40)
    assert _coef_rel(got, ref, 40) < 1e-10


def test_device_spectrum_matches_oracle(lib, small):
    ref = _oracle(small, "ph", 200)
    ch = chain_from_bundle(small, max_steps=200)
    ch.lanczos(200)
    chi, ei, e = ch.spectrum(WGRID, ETA)
    rchi, rei, re = spectrum.spectrum(ref.beta, ref.gamma, ref.z, small.spec.omega, small.spec.q_cart, WGRID, ETA)
    assert np.max(np.abs(ei - rei)) / np.max(np.abs(rei - 1)) < 1e-8
    # caller-held coefficients through ll_spectrum give the oracle's numbers to rounding
    c2, e2, _ = lib.spectrum(ref.beta, ref.gamma, ref.z, small.spec.omega, small.spec.q_cart, WGRID, ETA)
    assert np.max(np.abs(c2 - rchi)) / np.max(np.abs(rchi)) < 1e-10


def test_indefinite_metric_reported(lib, tiny):
    """Occupied energies pushed above the conduction band make D indefinite: the
    pseudo-Hermitian set-up reports LL_ENOTPD (computed on the device, no fault)."""
    import copy
    b = copy.copy(tiny)
    b.eps_k = tiny.eps_k + 5.0
    with pytest.raises(lib.LLError) as e:
        chain_from_bundle(b, max_steps=4)
    assert e.value.code == lib.LL_ENOTPD


@pytest.fixture(scope="module")
def kb():
    return w.get_bundle(w.config_kb())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_kb_workload_single_application(lib, kb, precision, tol):
    """The benchmark workload at full size (2048 orbitals, 32^3, 8 KB projectors per k), in
    the launch configuration the benchmark times: both operator halves against the oracle."""
    sys = System(kb)
    ch = chain_from_bundle(kb, precision=precision, max_steps=4)
    x = _rand(sys, 11)
    for upper in (False, True):
        assert rel_batch(ch.apply(x, upper), sys.apply_op(x, upper)) < tol


def test_kb_workload_first_coefficients(lib, kb):
    """First 6 pseudo-Hermitian steps of the benchmark workload, FP64 and FP32 paths."""
    sys = System(kb)
    ref = lanczos.pseudo_hermitian(sys, 6)
    got64 = chain_from_bundle(kb, max_steps=6).lanczos(6)
    assert _coef_rel(got64, ref, 6) < 1e-10
    got32 = chain_from_bundle(kb, precision="fp32", max_steps=6).lanczos(6)
    assert _coef_rel(got32, ref, 6) < 1e-4


# ---- per-k work split over several CTAs per k-point (systems whose k blocks do not fit one
# CTA's shared memory; LL_SPLIT_PERK=1 forces it on the smaller cells) ----------------------

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_split_path_single_application(lib, small, kb, precision, tol, monkeypatch):
    """Forced split path, both operator halves against the oracle, with and without KB."""
    monkeypatch.setenv("LL_SPLIT_PERK", "1")
    for b in (small, kb):
        sys = System(b)
        ch = chain_from_bundle(b, precision=precision, max_steps=4)
        x = _rand(sys, 12)
        for upper in (False, True):
            assert rel_batch(ch.apply(x, upper), sys.apply_op(x, upper)) < tol


def test_split_path_coefficients_small(lib, small, monkeypatch):
    """Forced split path, 120 pseudo-Hermitian FP64 steps: the oracle's first 100 coefficients."""
    ref = _oracle(small, "ph", 120)
    monkeypatch.setenv("LL_SPLIT_PERK", "1")
    got = chain_from_bundle(small, max_steps=120).lanczos(120)
    assert _coef_rel(got, ref, 100) < 1e-10


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_split_path_fp32_tensor_cores(lib, small, flavour, monkeypatch):
    """FP32 on the forced split path, whose P_c and KB dot blocks run on the tensor cores
    (three-way BF16 split, FP32 accumulation): against the same path with the dot blocks on
    the CUDA cores (LL_TC=0), and the loss function of the first 100 coefficients against
    the oracle's."""
    ref = _oracle(small, flavour, 120)
    monkeypatch.setenv("LL_SPLIT_PERK", "1")
    got = chain_from_bundle(small, flavour=flavour, precision="fp32", max_steps=120).lanczos(120)
    monkeypatch.setenv("LL_TC", "0")
    cc = chain_from_bundle(small, flavour=flavour, precision="fp32", max_steps=120).lanczos(120)
    assert _coef_rel(got, SimpleNamespace(beta=cc[0], gamma=cc[1], z=cc[2]), 20) < 1e-5
    assert _coef_rel(got, ref, 20) < 1e-4
    assert _loss_err(got, (ref.beta, ref.gamma, ref.z), small.spec.omega, small.spec.q_cart) < 1e-3


@pytest.fixture(scope="module")
def cubic8():
    return w.get_bundle(w.config_cubic8())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_cubic8_single_application(lib, cubic8, precision, tol):
    """Eight-atom cell (16 bands, ~1630 plane waves, 1024 orbitals): 16 per-k CTAs per k-point."""
    sys = System(cubic8)
    ch = chain_from_bundle(cubic8, precision=precision, max_steps=4)
    x = _rand(sys, 13)
    for upper in (False, True):
        assert rel_batch(ch.apply(x, upper), sys.apply_op(x, upper)) < tol


def test_cubic8_first_coefficients(lib, cubic8):
    sys = System(cubic8)
    ref = lanczos.pseudo_hermitian(sys, 8)
    got64 = chain_from_bundle(cubic8, max_steps=8).lanczos(8)
    assert _coef_rel(got64, ref, 8) < 1e-10
    got32 = chain_from_bundle(cubic8, precision="fp32", max_steps=8).lanczos(8)
    assert _coef_rel(got32, ref, 8) < 1e-4


def test_cubic8_non_hermitian(lib, cubic8):
    """The non-Hermitian recursion on the eight-atom cell."""
    sys = System(cubic8)
    ref = lanczos.non_hermitian(sys, 5)
    got = chain_from_bundle(cubic8, flavour="nh", max_steps=5).lanczos(5)
    assert _coef_rel(got, ref, 5) < 1e-10


def test_split_path_non_hermitian_small(lib, small, monkeypatch):
    """Forced split path, 120 non-Hermitian FP64 steps: the oracle's first 100 coefficients."""
    ref = _oracle(small, "nh", 120)
    monkeypatch.setenv("LL_SPLIT_PERK", "1")
    got = chain_from_bundle(small, flavour="nh", max_steps=120).lanczos(120)
    assert _coef_rel(got, ref, 100) < 1e-10


@pytest.mark.parametrize("kind", ["constant", "osc"])
def test_extrapolated_spectrum(lib, small, kind):
    """Coefficients continued to 5000 (Sec. 3.3) on the device, from caller-held coefficients
    (ll_spectrum_x) and from the chain's own (ll_lanczos_spectrum_x), against the oracle's
    extrapolation and LAPACK solve on the same coefficients."""
    from oracle.extrapolation import extrapolate
    ref = _oracle(small, "ph", 200)
    s = small.spec
    eb, eg, ez = extrapolate(ref.beta, ref.gamma, ref.z, kind, 5000)
    rchi, _, _ = spectrum.spectrum(eb, eg, ez, s.omega, s.q_cart, WGRID, ETA)
    chi, _, _ = lib.spectrum(ref.beta, ref.gamma, ref.z, s.omega, s.q_cart, WGRID, ETA, extrapolation=kind,
                             m_total=5000)
    assert np.max(np.abs(chi - rchi)) / np.max(np.abs(rchi)) < 1e-10
    ch = chain_from_bundle(small, max_steps=200)
    got = ch.lanczos(200)
    chi2, _, _ = ch.spectrum(WGRID, ETA, extrapolation=kind, m_total=5000)
    gb, gg, gz = extrapolate(got[0], got[1], got[2], kind, 5000)
    rchi2, _, _ = spectrum.spectrum(gb, gg, gz, s.omega, s.q_cart, WGRID, ETA)
    assert np.max(np.abs(chi2 - rchi2)) / np.max(np.abs(rchi2)) < 1e-10


# ---- sixteen-atom cell (32 bands, 48^3, 64 KB projectors, ~6000 plane waves): its ground
# state takes ~30 minutes of CPU, so these run where the bundle has been built and cached ----

@pytest.fixture(scope="module")
def sc16():
    b = w.cached_bundle(w.config_sc16())
    if b is None:
        pytest.skip("sixteen-atom ground state not cached (workloads.get_bundle(config_sc16()))")
    return b


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_sc16_single_application(lib, sc16, precision, tol):
    sys = System(sc16)
    ch = chain_from_bundle(sc16, precision=precision, max_steps=4)
    x = _rand(sys, 14)
    for upper in (False, True):
        assert rel_batch(ch.apply(x, upper), sys.apply_op(x, upper)) < tol


def test_sc16_first_coefficients(lib, sc16):
    sys = System(sc16)
    ref = lanczos.pseudo_hermitian(sys, 3)
    got = chain_from_bundle(sc16, max_steps=3).lanczos(3)
    assert _coef_rel(got, ref, 3) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replayed_steps_match_eager(lib, small, precision):
    """On a stream other than the legacy default, the chain captures one pseudo-Hermitian step
    of each parity into a CUDA graph and replays it; the coefficients are those of the eager
    launches (default stream) bit for bit, over several calls (resume)."""
    torch = pytest.importorskip("torch")
    eager = chain_from_bundle(small, precision=precision, max_steps=80).lanczos(80)
    st = torch.cuda.Stream()
    ch = chain_from_bundle(small, precision=precision, max_steps=80, stream=st.cuda_stream)
    ch.lanczos(7)
    ch.lanczos(30)
    got = ch.lanczos(43)
    st.synchronize()
    for a, b in zip(eager, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_lane_pair_plane_pass_kb(lib, kb, precision, tol, monkeypatch):
    """The plane pass with every line transform split over a lane pair (LL_XY_PAIR=1; the
    default at N = 48 only) on the KB workload at N = 32: both operator halves against the
    oracle."""
    monkeypatch.setenv("LL_XY_PAIR", "1")
    sys = System(kb)
    ch = chain_from_bundle(kb, precision=precision, max_steps=4)
    x = _rand(sys, 15)
    for upper in (False, True):
        assert rel_batch(ch.apply(x, upper), sys.apply_op(x, upper)) < tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pruned_forward_lines_bit_identical(lib, kb, precision, monkeypatch):
    """The line transforms pruned to the spheres' extent (forward lines keep only the points a
    sphere keeps, inverse lines skip the adds of the zero inputs outside it) against the
    unpruned kernels.  At the N/4 bound (LL_PRUNE=1) the results are the same bit for bit.  At
    the tighter 3N/16 bound (the default here: the KB spheres reach |m| = 6 at N = 32) more
    butterflies are dropped and the compiled code of the remaining ones rounds differently at
    a few points (measured on GB300 in FP64), so that level is held to the single-application
    tolerance of the oracle parity tests instead."""
    sys = System(kb, "tddft")
    x = _rand(sys, 14)
    got = {}
    for prune in ("", "1", "0"):
        monkeypatch.setenv("LL_PRUNE", prune)
        ch = chain_from_bundle(kb, precision=precision, max_steps=4)
        got[prune] = (ch.apply(x, True), ch.apply(x, False))
        ch.close()
    for a, b in zip(got["1"], got["0"]):
        for ak, bk in zip(a, b):
            assert np.array_equal(ak, bk)
    tol = 1e-12 if precision == "fp64" else 2e-5
    for a, b in zip(got[""], got["0"]):
        for ak, bk in zip(a, b):
            assert np.max(np.abs(ak - bk)) <= tol * np.max(np.abs(bk))
