"""The C-ABI library builds, loads without a GPU and exports every declared entry point;
host-side input validation (no kernel runs) rejects malformed systems."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ll():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll as mod
    return mod


def test_exports_match_header(ll):
    hdr = open(os.path.join(ROOT, "include", "ll.h")).read()
    declared = set(re.findall(r"^\s*(?:int|const char\*)\s+(ll_\w+)\s*\(", hdr, flags=re.M))
    assert declared, "no declarations parsed"
    lib = ctypes.CDLL(ll.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(ll.EXPORTS)
    assert "sm_103a" in ll.version()


def _desc_args(b):
    s = b.spec
    return dict(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=list(b.miller_k),
                miller_kq=list(b.miller_kq), u_k=b.u_k, u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r,
                rho_r=b.rho_r, beta_kq=b.beta_kq, dij=b.dij, q_cart=s.q_cart, max_steps=10)


def test_rejects_unsorted_sphere(ll):
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    m = args["miller_kq"][0].copy()
    m[[0, 1]] = m[[1, 0]]
    args["miller_kq"][0] = m
    with pytest.raises(ll.LLError) as e:
        ll.Chain(**args)
    assert e.value.code == ll.LL_EINVAL and "lexicographic" in str(e.value)


def test_rejects_q_on_reciprocal_lattice(ll):
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    args["q_cart"] = b.spec.bvec[0].copy()
    with pytest.raises(ll.LLError) as e:
        ll.Chain(**args)
    assert e.value.code == ll.LL_EINVAL and "reciprocal" in str(e.value)


def test_rejects_unsupported_grid(ll):
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    args["nfft"] = 20
    with pytest.raises(ll.LLError) as e:
        ll.Chain(**args)
    assert e.value.code == ll.LL_EUNSUPPORTED


def test_rejects_sphere_too_large_for_grid(ll):
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    m = args["miller_k"][0].copy()
    m[-1, 2] = m[-1, 2] + 40
    args["miller_k"][0] = m
    with pytest.raises(ll.LLError) as e:
        ll.Chain(**args)
    assert e.value.code == ll.LL_EINVAL


def test_rejects_bad_extrapolation(ll):
    """Argument checks of ll_spectrum_x run on the host before any device work."""
    b = np.ones(10)
    g = np.ones(10, dtype=complex)
    w = np.linspace(0, 10, 5)
    for kind, m_total, beta in (("osc", 100, b[:3]), ("constant", 5, b), ("constant", 100, b[:1])):
        with pytest.raises(ll.LLError) as e:
            ll.spectrum(beta, g[:len(beta)], g[:len(beta)], 270.0, [0.06, 0, 0], w, 0.1,
                        extrapolation=kind, m_total=m_total)
        assert e.value.code == ll.LL_EINVAL
    with pytest.raises(KeyError):
        ll.spectrum(b, g, g, 270.0, [0.06, 0, 0], w, 0.1, extrapolation="linear", m_total=100)


@pytest.mark.parametrize("name,bad", [("eps_k", np.nan), ("kcart", np.nan), ("q_cart", np.nan), ("dij", np.inf)])
def test_rejects_non_finite_input(ll, name, bad):
    """The small host arrays are checked on the host before any device work (the large ones,
    u_k, u_kq, vloc_r, rho_r and beta_kq, on the device once staged: a GPU test covers them)."""
    _non_finite_refused(ll, name, bad)


def _non_finite_refused(ll, name, bad):
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    if name in ("beta_kq", "dij") and len(b.dij) == 0:
        pytest.skip("the cell has no KB projectors")
    v = args[name]
    if isinstance(v, list):                       # per-k arrays: spoil the last k-point's last entry
        v = [x.copy() for x in v]
        v[-1].flat[-1] = bad
    else:
        v = np.array(v, copy=True)
        v.flat[v.size // 2] = bad
    args[name] = v
    with pytest.raises(ll.LLError) as e:
        ll.Chain(**args)
    assert e.value.code == ll.LL_EINVAL and f"non-finite value in {name}" in str(e.value)


def test_rejects_bad_occupations(ll):
    """A metal's occupations and k+Q levels are host arrays checked before any device work."""
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    occ = np.ones_like(b.eps_k)
    for extra, what in ((dict(occ_k=occ, occ_kq=occ, eps_kq=np.full_like(b.eps_kq, np.nan)), "non-finite value in eps_kq"),
                        (dict(occ_k=occ * np.nan, occ_kq=occ, eps_kq=b.eps_kq), "non-finite value in occ_k")):
        with pytest.raises(ll.LLError) as e:
            ll.Chain(**args, **extra)
        assert e.value.code == ll.LL_EINVAL and what in str(e.value)


def test_footprint_bound_orders(ll):
    """ll_footprint on the host: it grows with the coefficient capacity, with FP64 orbitals over
    FP32 ones, and with the non-Hermitian chain's second vector; the KB workload's FP32 chain
    at 1000 steps is a few GB at most (it is admitted under budgets of that order)."""
    small = _desc_args(w.get_bundle(w.config_small()))
    fp = lambda **kw: ll.footprint(**{**small, **kw})
    assert fp(max_steps=100) < fp(max_steps=3000)
    assert fp(precision="fp32") < fp(precision="fp64")
    assert fp(flavour="ph") < fp(flavour="nh")
    kb = _desc_args(w.get_bundle(w.config_kb()))
    assert 1 << 20 < ll.footprint(**{**kb, "precision": "fp32", "max_steps": 1000}) < 8 << 30


def test_packed_host_arrays_checked(ll):
    """u_k, u_kq, beta_kq may come packed (1-D complex128 in the descriptor's layout, used in
    place); a packed array of the wrong length is refused before the library is called."""
    b = w.get_bundle(w.config_tiny())
    args = _desc_args(b)
    packed = np.concatenate([x.ravel() for x in b.u_k]).astype(np.complex128)
    d, keep = ll._make_desc(**dict(args, u_k=packed))
    assert keep["u_k"] is packed                     # no copy
    with pytest.raises(ValueError):
        ll._make_desc(**dict(args, u_k=packed[:-1]))
