"""The request loop on the GPU: continuous batching, admission by HBM footprint, and
independence of each job's result from the jobs running beside it."""
import time

import numpy as np
import pytest

import workloads as w

from .helpers import chain_from_bundle

pytestmark = pytest.mark.gpu
WGRID = np.linspace(0.0, 40.0, 401)


@pytest.fixture(scope="module")
def ll():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll as mod
    return mod


def _system(b, **kw):
    s = b.spec
    d = dict(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq, u_k=b.u_k,
             u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r, rho_r=b.rho_r, beta_kq=b.beta_kq, dij=b.dij,
             q_cart=s.q_cart)
    d.update(kw)
    return d


def _jobs():
    tiny, small = w.get_bundle(w.config_tiny()), w.get_bundle(w.config_small())
    return [
        (tiny, dict(flavour="ph", precision="fp64"), 60),
        (small, dict(flavour="ph", precision="fp32"), 150),
        (tiny, dict(flavour="nh", precision="fp64", approx="rpa"), 40),
        (small, dict(flavour="ph", precision="fp64"), 90),
        (small, dict(flavour="nh", precision="fp32"), 70),
    ]


def _alone(b, opts, n):
    ch = chain_from_bundle(b, approx=opts.get("approx"), flavour=opts["flavour"], precision=opts["precision"],
                           max_steps=n)
    beta, gamma, z = ch.lanczos(n)
    chi, _, _ = ch.spectrum(WGRID, 0.1)
    ch.close()
    return beta, gamma, z, chi


def _wait(srv, ids, timeout=300):
    t0 = time.time()
    res = {}
    while len(res) < len(ids):
        for i in ids:
            if i not in res:
                st, r = srv.poll(i)
                if st in (2, 3):
                    res[i] = (st, r)
        assert time.time() - t0 < timeout, "the request loop did not finish"
        time.sleep(0.01)
    return res


def test_results_identical_alone_and_in_the_mix(ll):
    jobs = _jobs()
    ref = [_alone(b, o, n) for b, o, n in jobs]
    srv = ll.Server(hbm_budget_bytes=16 << 30, max_slots=4, chunk=16)
    ids = []
    for idx, (b, o, n) in enumerate(jobs):
        ids.append(srv.submit(n, WGRID, 0.1, **_system(b, max_steps=n, **o)))
        if idx == 1:
            time.sleep(0.05)   # later jobs arrive while the first ones run
    res = _wait(srv, ids)
    for (b, o, n), jid, r in zip(jobs, ids, ref):
        st, out = res[jid]
        assert st == 2 and out["status"] == 0 and out["steps_done"] == n, out.get("error")
        assert np.array_equal(out["beta"], r[0])
        assert np.array_equal(out["gamma"], r[1])
        assert np.array_equal(out["z"], r[2])
        assert np.array_equal(out["chi"], r[3])
    srv.close()


def test_admission_respects_budget(ll):
    small = w.get_bundle(w.config_small())
    probe = ll.Server(hbm_budget_bytes=64 << 30, max_slots=1)
    jid = probe.submit(10, None, 0.1, **_system(small, max_steps=10))
    _wait(probe, [jid])
    one = probe.stats()["peak"]
    probe.close()
    assert one > 0
    budget = int(2.5 * one)          # room for two chains at a time; five submitted at once
    srv = ll.Server(hbm_budget_bytes=budget, max_slots=8, chunk=8)
    ids = [srv.submit(40, WGRID, 0.1, **_system(small, max_steps=40)) for _ in range(5)]
    seen = 0
    t0 = time.time()
    while True:
        st = srv.stats()
        seen = max(seen, st["running"])
        if st["running"] == 0 and st["queued"] == 0 and all(srv.poll(i)[0] == 2 for i in ids):
            break
        assert time.time() - t0 < 300
        time.sleep(0.005)
    assert srv.stats()["peak"] <= budget
    assert 1 <= seen <= 2
    srv.close()


def test_malformed_job_fails_without_stopping_the_loop(ll):
    tiny = w.get_bundle(w.config_tiny())
    srv = ll.Server(hbm_budget_bytes=8 << 30, max_slots=2, chunk=8)
    bad = _system(tiny, max_steps=10)
    mk = [m.copy() for m in bad["miller_kq"]]
    mk[0][[0, 1]] = mk[0][[1, 0]]
    bad["miller_kq"] = mk
    j_bad = srv.submit(10, None, 0.1, **bad)
    j_ok = srv.submit(10, None, 0.1, **_system(tiny, max_steps=10))
    res = _wait(srv, [j_bad, j_ok])
    assert res[j_bad][0] == 3 and res[j_bad][1]["status"] == 1
    assert res[j_ok][0] == 2 and res[j_ok][1]["steps_done"] == 10
    srv.close()


def test_cancel_queued_and_running_jobs(ll):
    """A cancelled queued job ends at once with no steps; a cancelled running chain stops after
    its current round with the coefficients of the steps it finished (those of the same job
    run alone), its memory returns to the budget and the next job takes its slot."""
    small = w.get_bundle(w.config_small())
    opts = dict(flavour="ph", precision="fp64", approx="tddft")
    n_long = 20000
    srv = ll.Server(hbm_budget_bytes=16 << 30, max_slots=1, chunk=8)
    long_id = srv.submit(n_long, WGRID, 0.1, **_system(small, max_steps=n_long, **opts))
    queued_id = srv.submit(10, None, 0.1, **_system(small, max_steps=10, **opts))
    t0 = time.time()
    while True:
        st, r = srv.poll(long_id)
        if st == 1 and r["steps_done"] >= 16:
            break
        assert st in (0, 1) and time.time() - t0 < 120, r.get("error")
        time.sleep(0.002)
    srv.cancel(queued_id)
    st, r = srv.poll(queued_id)
    assert st == 3 and r["status"] == ll.LL_ECANCELED and r["steps_done"] == 0
    srv.cancel(long_id)
    st, r = _wait(srv, [long_id], timeout=120)[long_id]
    m = r["steps_done"]
    assert st == 3 and r["status"] == ll.LL_ECANCELED, r.get("error")
    assert 16 <= m < n_long and m % 8 == 0
    beta, gamma, z, _ = _alone(small, opts, m)
    assert np.array_equal(r["beta"], beta) and np.array_equal(r["gamma"], gamma) and np.array_equal(r["z"], z)
    assert np.all(np.isfinite(r["chi"])) and np.any(r["chi"] != 0)
    assert srv.stats()["used"] == 0
    nxt = srv.submit(10, None, 0.1, **_system(small, max_steps=10, **opts))
    st, r = _wait(srv, [nxt])[nxt]
    assert st == 2 and r["steps_done"] == 10, r.get("error")
    srv.cancel(nxt)                                # already ended: unchanged
    assert srv.poll(nxt)[0] == 2
    srv.close()


@pytest.mark.parametrize("cell", ["small", "kb", "cubic8"])
@pytest.mark.parametrize("flavour,precision", [("ph", "fp32"), ("nh", "fp64")])
def test_chain_bytes_within_footprint(ll, cell, flavour, precision):
    """The request loop admits by ll_footprint (plus the spectrum staging): the device bytes a
    chain really holds after its steps and its spectrum never exceed that bound."""
    b = {"small": w.config_small, "kb": w.config_kb, "cubic8": w.config_cubic8}[cell]()
    b = w.get_bundle(b)
    ch = chain_from_bundle(b, flavour=flavour, precision=precision, max_steps=12)
    ch.lanczos(12)
    wgrid = np.linspace(0.0, 40.0, 4001)
    ch.spectrum(wgrid, 0.1, extrapolation="osc", m_total=200)
    held = ch.bytes()
    bound = ch.footprint() + ll.spectrum_bytes(len(wgrid))
    ch.close()
    assert 0 < held <= bound, (held, bound)
