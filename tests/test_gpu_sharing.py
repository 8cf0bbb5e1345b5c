"""Several momentum transfers on one ground state (ll_create_sharing): chains at other Q use
the u_{vk}(r) grids of a chain of the same ground state instead of building and storing their
own (Sec. 2.1, Q = q + G; Sec. 5, one recursion per Q).  Each sharing chain's coefficients are
those of a chain with its own grids, bit for bit, also after the lending chain is destroyed;
a chain of another ground state is refused."""
import numpy as np
import pytest

import workloads as w

from .helpers import chain_from_bundle

pytestmark = pytest.mark.gpu

QS = [np.array([0.13, 0.04, -0.02]), np.array([-0.07, 0.21, 0.05]), np.array([1.3, 0.2, 0.1])]


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    return ll


def _at_q(q):
    """The small cell's ground state at another Q: the k+Q states of that Q, and the ground
    state's own k-side (k-points, V_KS, n0, sphere(k), u_k, eps_k) taken from the base bundle, as one
    user holding one ground state does.  (A bundle at another Q built on another machine than
    the base bundle has its k-side states from that machine's LAPACK, different in the last
    bits, which the library rightly refuses to share.)"""
    base = w.get_bundle(w.config_small())
    spec = w.config_small()
    spec.q_cart = np.asarray(q, dtype=np.float64) * (2 * np.pi / w.A_LAT)
    spec.name = "fcc2_10ry_18_q" + "_".join("%+.3f" % c for c in q)
    b = w.get_bundle(spec)
    for name in ("kfrac", "kcart", "vloc_r", "rho_r", "miller_k", "u_k", "eps_k"):
        setattr(b, name, getattr(base, name))
    return b


def _system(b, **kw):
    s = b.spec
    d = dict(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq, u_k=b.u_k,
             u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r, rho_r=b.rho_r, beta_kq=b.beta_kq, dij=b.dij,
             q_cart=s.q_cart, approx=s.approx)
    d.update(kw)
    return d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sharing_chains_match_own_grids(lib, precision):
    base = w.get_bundle(w.config_small())
    others = [_at_q(q) for q in QS]
    lender = chain_from_bundle(base, precision=precision, max_steps=60)
    lender.lanczos(10)
    sharers = [lib.Chain(share=lender, **_system(b, precision=precision, max_steps=60)) for b in others]
    own = [chain_from_bundle(b, precision=precision, max_steps=60) for b in others]
    for sh, ow in zip(sharers, own):
        assert sh.bytes() < ow.bytes()
        a, b = sh.lanczos(30), ow.lanczos(30)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    lender.close()        # the grids live on with the chains that use them
    for sh, ow in zip(sharers, own):
        a, b = sh.lanczos(30), ow.lanczos(30)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        sh.close()
        ow.close()


def test_sharing_refuses_another_ground_state(lib):
    small = w.get_bundle(w.config_small())
    kb = w.get_bundle(w.config_kb())
    lender = chain_from_bundle(small, max_steps=4)
    with pytest.raises(lib.LLError) as e:
        lib.Chain(share=lender, **_system(kb, max_steps=4))
    assert e.value.code == lib.LL_EINVAL and "ground state differs" in str(e.value)
    with pytest.raises(lib.LLError) as e:
        lib.Chain(share=lender, **_system(small, precision="fp32", max_steps=4))
    assert e.value.code == lib.LL_EINVAL and "precision" in str(e.value)
