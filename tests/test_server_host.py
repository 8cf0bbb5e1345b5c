"""Host-side behaviour of the request loop that needs no GPU: refusals at submit, cancel."""
import time

import numpy as np
import pytest

import workloads as w


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
             q_cart=s.q_cart, max_steps=50)
    d.update(kw)
    return d


def test_over_budget_job_refused_at_submit(ll):
    b = w.get_bundle(w.config_tiny())
    srv = ll.Server(hbm_budget_bytes=1 << 16, max_slots=2)
    with pytest.raises(ll.LLError) as e:
        srv.submit(20, np.linspace(0, 40, 11), 0.1, **_system(b))
    assert e.value.code == ll.LL_ENOMEM and "budget" in str(e.value)
    srv.close()


def test_bad_step_count_and_unknown_job(ll):
    b = w.get_bundle(w.config_tiny())
    srv = ll.Server(hbm_budget_bytes=1 << 34, max_slots=2)
    with pytest.raises(ll.LLError) as e:
        srv.submit(80, None, 0.1, **_system(b, max_steps=50))
    assert e.value.code == ll.LL_EINVAL
    with pytest.raises(ll.LLError) as e:
        srv.poll(12345)
    assert e.value.code == ll.LL_ENOTFOUND
    srv.close()


def test_server_arguments(ll):
    with pytest.raises(ll.LLError):
        ll.Server(hbm_budget_bytes=0, max_slots=1)
    with pytest.raises(ll.LLError):
        ll.Server(hbm_budget_bytes=1 << 30, max_slots=0)


def test_cancel_unknown_and_ended_jobs(ll):
    """ll_cancel: LL_ENOTFOUND for an unknown id; a job that has ended keeps its outcome."""
    b = w.get_bundle(w.config_tiny())
    srv = ll.Server(hbm_budget_bytes=1 << 34, max_slots=2)
    with pytest.raises(ll.LLError) as e:
        srv.cancel(777)
    assert e.value.code == ll.LL_ENOTFOUND
    jid = srv.submit(5, None, 0.1, **_system(b))
    t0 = time.time()
    while srv.poll(jid)[0] not in (2, 3):       # without a GPU the job fails at admission
        assert time.time() - t0 < 60
        time.sleep(0.01)
    st, r = srv.poll(jid)
    srv.cancel(jid)
    st2, r2 = srv.poll(jid)
    assert (st2, r2["status"]) == (st, r["status"]) and r2["status"] != ll.LL_ECANCELED
    srv.close()


def test_non_finite_job_refused_at_submit(ll):
    b = w.get_bundle(w.config_tiny())
    srv = ll.Server(hbm_budget_bytes=1 << 34, max_slots=2)
    eps = np.array(b.eps_k, copy=True)
    eps[1, 2] = np.nan
    with pytest.raises(ll.LLError) as e:
        srv.submit(5, None, 0.1, **_system(b, eps_k=eps))
    assert e.value.code == ll.LL_EINVAL and "non-finite value in eps_k" in str(e.value)
    assert srv.stats()["queued"] == 0
    srv.close()


def test_release_ended_job(ll):
    """ll_release frees an ended job's record; its id is unknown afterwards."""
    b = w.get_bundle(w.config_tiny())
    srv = ll.Server(hbm_budget_bytes=1 << 34, max_slots=2)
    with pytest.raises(ll.LLError) as e:
        srv.release(4242)
    assert e.value.code == ll.LL_ENOTFOUND
    jid = srv.submit(5, None, 0.1, **_system(b))
    t0 = time.time()
    while True:
        try:
            srv.release(jid)                    # LL_PENDING until the job has ended
            break
        except ll.LLError as err:
            assert err.code == ll.LL_PENDING and time.time() - t0 < 60
            time.sleep(0.01)
    for call in (srv.poll, srv.cancel, srv.release):
        with pytest.raises(ll.LLError) as e:
            call(jid)
        assert e.value.code == ll.LL_ENOTFOUND
    srv.close()
