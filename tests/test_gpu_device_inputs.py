"""Device-resident inputs (ll_system_desc.where = LL_WHERE_DEVICE): the large arrays of the
ground state passed as device pointers (torch CUDA tensors' data_ptr()), read on the device
with no host round trip.  The chain they build is the one host inputs build, bit for bit; a
NaN in a device array and a host address flagged as device memory are refused with
LL_EINVAL before any set-up work."""
import ctypes as C

import numpy as np
import pytest

import workloads as w

from .helpers import chain_from_bundle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    return ll


def _packed(blocks):
    return torch.from_numpy(np.concatenate([np.ascontiguousarray(x, dtype=np.complex128).ravel() for x in blocks])).cuda()


def _device_system(b, **kw):
    s = b.spec
    d = dict(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq,
             u_k=_packed(b.u_k), u_kq=_packed(b.u_kq), eps_k=b.eps_k,
             vloc_r=torch.from_numpy(np.ascontiguousarray(b.vloc_r)).cuda(),
             rho_r=torch.from_numpy(np.ascontiguousarray(b.rho_r)).cuda(),
             beta_kq=_packed(b.beta_kq) if b.dij.size else None, dij=b.dij, q_cart=s.q_cart, approx=s.approx)
    d.update(kw)
    return d


@pytest.mark.parametrize("cell", ["small", "kb"])
@pytest.mark.parametrize("precision,flavour", [("fp64", "ph"), ("fp32", "ph"), ("fp32", "nh")])
def test_device_inputs_match_host_inputs(lib, cell, precision, flavour):
    b = w.get_bundle(w.config_small() if cell == "small" else w.config_kb())
    host = chain_from_bundle(b, precision=precision, flavour=flavour, max_steps=30).lanczos(30)
    ch = lib.Chain(**_device_system(b, precision=precision, flavour=flavour, max_steps=30))
    dev = ch.lanczos(30)
    ch.close()
    for a, c in zip(host, dev):
        assert np.array_equal(a, c)


def test_packed_host_inputs_match_lists(lib):
    """Host inputs already packed (pinned memory here) build the chain the per-k lists build."""
    b = w.get_bundle(w.config_kb())
    ref = chain_from_bundle(b, precision="fp32", max_steps=20).lanczos(20)
    packed = {}
    for name in ("u_k", "u_kq", "beta_kq"):
        blocks = getattr(b, name)
        n = sum(x.size for x in blocks)
        t = torch.empty(2 * n, dtype=torch.float64, pin_memory=True)
        a = t.numpy().view(np.complex128)
        a[:] = np.concatenate([x.ravel() for x in blocks])
        packed[name] = (a, t)
    s = b.spec
    ch = lib.Chain(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq,
                   u_k=packed["u_k"][0], u_kq=packed["u_kq"][0], eps_k=b.eps_k, vloc_r=b.vloc_r, rho_r=b.rho_r,
                   beta_kq=packed["beta_kq"][0], dij=b.dij, q_cart=s.q_cart, approx=s.approx, precision="fp32",
                   max_steps=20)
    got = ch.lanczos(20)
    ch.close()
    for a, c in zip(got, ref):
        assert np.array_equal(a, c)


def test_device_inputs_refused(lib):
    b = w.get_bundle(w.config_small())
    sysd = _device_system(b, max_steps=4)
    bad = sysd["u_kq"].clone()
    bad[17] = float("nan")
    with pytest.raises(lib.LLError) as e:
        lib.Chain(**dict(sysd, u_kq=bad))
    assert e.value.code == lib.LL_EINVAL and "u_kq" in str(e.value)
    # host arrays flagged as device memory
    s = b.spec
    d, keep = lib._make_desc(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k,
                             miller_kq=b.miller_kq, u_k=b.u_k, u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r,
                             rho_r=b.rho_r, beta_kq=b.beta_kq, dij=b.dij, q_cart=s.q_cart, max_steps=4)
    d.where = lib.LL_WHERE_DEVICE
    h = C.c_void_p()
    rc = lib._lib.ll_create(C.byref(d), None, C.byref(h))
    assert rc == lib.LL_EINVAL and "not a device pointer" in lib._lib.ll_last_error().decode()


@pytest.mark.parametrize("name,bad", [("u_k", np.nan), ("u_kq", np.inf), ("vloc_r", -np.inf), ("rho_r", np.nan),
                                      ("beta_kq", np.nan)])
def test_host_inputs_non_finite_refused(lib, name, bad):
    """Host inputs: the large arrays are checked on the device after their staging copy."""
    b = w.get_bundle(w.config_kb())
    s = b.spec
    args = dict(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=list(b.miller_k),
                miller_kq=list(b.miller_kq), u_k=b.u_k, u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r,
                rho_r=b.rho_r, beta_kq=b.beta_kq, dij=b.dij, q_cart=s.q_cart, max_steps=4)
    v = args[name]
    if isinstance(v, list):
        v = [x.copy() for x in v]
        v[-1].flat[-1] = bad
    else:
        v = np.array(v, copy=True)
        v.flat[v.size // 2] = bad
    args[name] = v
    with pytest.raises(lib.LLError) as e:
        lib.Chain(**args)
    assert e.value.code == lib.LL_EINVAL and f"non-finite value in {name}" in str(e.value)


def test_request_loop_takes_device_inputs(lib):
    b = w.get_bundle(w.config_small())
    wgrid = np.linspace(0.0, 40.0, 401)
    srv = lib.Server(hbm_budget_bytes=8 << 30, max_slots=2, chunk=16)
    i_host = srv.submit(40, wgrid, 0.1, **dict(lattice=b.spec.lattice, nfft=b.spec.nfft, kcart=b.kcart,
                                                  miller_k=b.miller_k, miller_kq=b.miller_kq, u_k=b.u_k,
                                                  u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r, rho_r=b.rho_r,
                                                  beta_kq=b.beta_kq, dij=b.dij, q_cart=b.spec.q_cart,
                                                  precision="fp32", max_steps=40))
    i_dev = srv.submit(40, wgrid, 0.1, **_device_system(b, precision="fp32", max_steps=40))
    res = {}
    import time
    t0 = time.time()
    while len(res) < 2 and time.time() - t0 < 120:
        for i in (i_host, i_dev):
            st, r = srv.poll(i)
            if st in (lib.JOB_DONE, lib.JOB_FAILED):
                res[i] = (st, r)
        time.sleep(0.01)
    srv.close()
    assert res[i_host][0] == lib.JOB_DONE and res[i_dev][0] == lib.JOB_DONE
    for key in ("beta", "gamma", "z", "eps_inv"):
        assert np.array_equal(res[i_host][1][key], res[i_dev][1][key])
