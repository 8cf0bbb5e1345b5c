"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on metals (Sec. 2.6:
the projector on empty states redefined per band, occupations as weights in the band sums).

The library iterates on z = Q^-1 S x, with S = diag(sqrt(f_vk)) (the band weight folded into
u_k) and Q the square root of the projector P_{c,v} (weight sqrt(c_mv) along the kept states
of k+Q): its operator is (Q^-1 S) L (Q^-1 S)^-1, symmetric in the plain scalar product.  One
application to z(x) is compared with z of the oracle's application to x, while the Lanczos
coefficients, which this similarity with the matching change of metric leaves unchanged, are
compared directly.

Tolerances as for the insulators: one FP64 application 1e-12 relative, FP32 2e-5; the first 100
FP64 coefficients 1e-10; the FP32 loss function 1e-3, over the first 80 coefficients (this
cell's FP32 window, pinned on the oracle in test_oracle_window.py).  The
metallic gas's spectrum (eight steps span its Krylov space) is compared with the Lindhard sum.
"""
import numpy as np
import pytest

import workloads as w
from workloads.cells import config_metal
from oracle import lanczos, spectrum, xc
from oracle.liouvillian import System

from .helpers import chain_from_bundle, rel_batch
from .test_oracle_metal import _lindhard_pairs, _metal_gas

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
def metal():
    return w.get_bundle(config_metal())


_ORACLE = {}


def _oracle(b, flavour, n=120):
    key = (b.spec.name, flavour)
    if key not in _ORACLE:
        _ORACLE[key] = lanczos.run(System(b), n, flavour)
    return _ORACLE[key]


def _to_z(b, sys, x):
    """z = Q^-1 S x: the band weights sqrt(f_v), then 1/sqrt(c_mv) along the kept states."""
    out = []
    for k, xk in enumerate(x):
        y = np.sqrt(b.occ_k[k])[:, None] * xk
        u, c = b.u_kq[k], sys.c[k]
        s = u.conj() @ y.T                                   # (m, v)
        f = np.where(c > 0, 1.0 / np.sqrt(np.where(c > 0, c, 1.0)) - 1.0, 0.0)
        out.append(y + (u.T @ (f * s)).T)
    return out


def _rand(sys, seed):
    rng = np.random.default_rng(seed)
    x = [rng.normal(size=(sys.nbnd, len(m))) + 1j * rng.normal(size=(sys.nbnd, len(m))) for m in sys.mkq]
    return sys.project_c(x)


def _coef_rel(got, want, n):
    b = np.max(np.abs(got[0][:n] - want.beta[:n]) / np.abs(want.beta[:n]))
    g = np.max(np.abs(got[1][:n] - want.gamma[:n]) / np.abs(want.gamma[:n]))
    z = np.max(np.abs(got[2][:n] - want.z[:n])) / np.max(np.abs(want.z[:n]))
    return max(b, g, z)


def _loss_err(got, want, b, m=100):
    _, ea, _ = spectrum.spectrum(got[0][:m], got[1][:m], got[2][:m], b.spec.omega, b.spec.q_cart, WGRID, ETA)
    _, eb, _ = spectrum.spectrum(want.beta[:m], want.gamma[:m], want.z[:m], b.spec.omega, b.spec.q_cart, WGRID, ETA)
    la, lb = spectrum.loss(ea), spectrum.loss(eb)
    return np.max(np.abs(la - lb)) / np.max(np.abs(lb))


def test_metal_cell_has_partial_bands(metal):
    """The semimetal's ground state: bands with fractional occupations at k and at k+Q."""
    assert ((metal.occ_k > 0) & (metal.occ_k < 1)).sum() > 100
    assert ((metal.occ_kq > 0) & (metal.occ_kq < 1)).sum() > 100


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("upper", [False, True])
def test_single_application_metal(lib, metal, precision, tol, upper):
    sys = System(metal)
    ch = chain_from_bundle(metal, precision=precision, max_steps=4)
    x = _rand(sys, 31)
    got = ch.apply(_to_z(metal, sys, x), upper)
    want = _to_z(metal, sys, sys.apply_op(x, upper))
    assert rel_batch(got, want) < tol


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_metal_coefficients_fp64(lib, metal, flavour):
    ref = _oracle(metal, flavour)
    ch = chain_from_bundle(metal, flavour=flavour, max_steps=120)
    got = ch.lanczos(120)
    assert _coef_rel(got, ref, 100) < 1e-10


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_metal_loss_function_fp32(lib, metal, flavour):
    """The FP32 window of this cell is 80 coefficients: FP32-sized rounding at every step moves
    the oracle's own 100-coefficient loss function by more than 1e-3 (test_oracle_window.py)."""
    ref = _oracle(metal, flavour)
    ch = chain_from_bundle(metal, flavour=flavour, precision="fp32", max_steps=120)
    got = ch.lanczos(120)
    assert _loss_err(got, ref, metal, m=80) < 1e-3


@pytest.mark.parametrize("flavour", ["ph", "nh"])
@pytest.mark.parametrize("approx", ["ipa", "tddft"])
def test_metal_gas_lindhard(lib, approx, flavour):
    """The metallic free-electron gas on the device: eps^-1 of its eight coefficients equals
    the Dyson form on the Lindhard sum of its smeared occupations."""
    b = _metal_gas(approx)
    spec = b.spec
    ch = chain_from_bundle(b, approx=approx, flavour=flavour, max_steps=8)
    beta, gamma, z = ch.lanczos(8)
    wev = np.linspace(0.0, 12.0, 241)
    eta = 0.15
    zz = (wev + 1j * eta) / w.HA_EV
    pairs = _lindhard_pairs(b)
    chi0 = 2.0 / spec.omega / b.nks * np.sum(pairs[None, :, 0] / (zz[:, None] - pairs[None, :, 1]), axis=1)
    q2 = float(spec.q_cart @ spec.q_cart)
    n = spec.nelec / spec.omega
    kern = 0.0 if approx == "ipa" else 4 * np.pi / q2 + float(xc.fxc(np.array(n)))
    want = 1.0 + 4 * np.pi / q2 * chi0 / (1.0 - kern * chi0)
    _, eps_inv, _ = spectrum.spectrum(beta, gamma, z, spec.omega, spec.q_cart, wev, eta)
    assert np.max(np.abs(eps_inv - want)) < 1e-10 * np.max(np.abs(want - 1.0))


def test_full_occupations_match_the_insulator(lib):
    """Every occupation 1 through the metallic tables: the insulator's coefficients."""
    b = w.get_bundle(w.config_tiny())
    ins = chain_from_bundle(b, max_steps=40).lanczos(40)
    b.occ_k = np.ones_like(b.eps_k)
    b.occ_kq = np.ones_like(b.eps_kq)
    met = chain_from_bundle(b, max_steps=40).lanczos(40)
    for a, c in zip(met, ins):
        assert np.max(np.abs(np.asarray(a) - np.asarray(c))) <= 1e-12 * np.max(np.abs(c))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("upper", [False, True])
def test_single_application_metal_split_path(lib, metal, precision, tol, upper, monkeypatch):
    """The split per-k path (forced; the large cells' path, tensor-core projections in FP32)
    with the metal's image and coefficients formed over plane-wave chunks."""
    monkeypatch.setenv("LL_SPLIT_PERK", "1")
    sys = System(metal)
    ch = chain_from_bundle(metal, precision=precision, max_steps=4)
    x = _rand(sys, 33)
    got = ch.apply(_to_z(metal, sys, x), upper)
    want = _to_z(metal, sys, sys.apply_op(x, upper))
    assert rel_batch(got, want) < tol


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_metal_split_path_coefficients(lib, metal, flavour, monkeypatch):
    """Split path: the first 100 FP64 coefficients (1e-10) and the FP32 loss function of the
    first 80 (1e-3) against the oracle, both recursions."""
    monkeypatch.setenv("LL_SPLIT_PERK", "1")
    ref = _oracle(metal, flavour)
    got = chain_from_bundle(metal, flavour=flavour, max_steps=120).lanczos(120)
    assert _coef_rel(got, ref, 100) < 1e-10
    got32 = chain_from_bundle(metal, flavour=flavour, precision="fp32", max_steps=120).lanczos(120)
    assert _loss_err(got32, ref, metal, m=80) < 1e-3


def test_metal_occupations_checked(lib, metal):
    """Occupations outside [0, 1] are refused at create."""
    from paper_2111_06623_gb300 import ll
    s = metal.spec
    base = dict(lattice=s.lattice, nfft=s.nfft, kcart=metal.kcart, miller_k=metal.miller_k,
                miller_kq=metal.miller_kq, u_k=metal.u_k, u_kq=metal.u_kq, eps_k=metal.eps_k,
                vloc_r=metal.vloc_r, rho_r=metal.rho_r, q_cart=s.q_cart, max_steps=4)
    bad = metal.occ_k.copy()
    bad[0, 0] = 1.5
    with pytest.raises(ll.LLError) as e:
        ll.Chain(**base, occ_k=bad, occ_kq=metal.occ_kq, eps_kq=metal.eps_kq)
    assert e.value.code == 1


def test_metal_job_through_the_request_loop(lib, metal):
    """A metal submitted to the request loop (occupations deep-copied at submit) beside an
    insulator gives the chain's own coefficients, bit for bit."""
    from .helpers import metal_args
    n = 60
    ref = chain_from_bundle(metal, precision="fp32", max_steps=n).lanczos(n)
    small = w.get_bundle(w.config_small())
    srv = lib.Server(hbm_budget_bytes=8 << 30, max_slots=2, chunk=16)

    def system(b, **extra):
        s = b.spec
        return dict(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq,
                    u_k=b.u_k, u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r, rho_r=b.rho_r, beta_kq=b.beta_kq,
                    dij=b.dij, q_cart=s.q_cart, approx=s.approx, precision="fp32", max_steps=n, **extra)

    wgrid = np.linspace(0.0, 40.0, 401)
    ids = [srv.submit(n, wgrid, 0.1, **system(metal, **metal_args(metal))), srv.submit(n, wgrid, 0.1, **system(small))]
    import time
    t0, res = time.time(), {}
    while len(res) < 2:
        for i in ids:
            if i not in res:
                st, r = srv.poll(i)
                if st in (lib.JOB_DONE, lib.JOB_FAILED):
                    res[i] = (st, r)
        assert time.time() - t0 < 300
        time.sleep(0.01)
    srv.close()
    st, out = res[ids[0]]
    assert st == lib.JOB_DONE and out["steps_done"] == n, out.get("error")
    assert np.array_equal(out["beta"], ref[0]) and np.array_equal(out["z"], ref[2])
