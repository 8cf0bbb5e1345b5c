"""Host-side pieces of the benchmark: the many-Q pool, the flop model, the profile digest."""
import numpy as np
import pytest

import bench
import workloads as w


def test_q_pool_is_seeded_and_in_range():
    a, b = bench.q_pool(), bench.q_pool()
    assert a.shape == (64, 3) and np.array_equal(a, b)
    mag = np.linalg.norm(a, axis=1) / (2 * np.pi / w.A_LAT)
    assert np.all((mag >= 0.05) & (mag <= 0.6))


def test_nominal_step_flops():
    """2P + 2 full FFTs for D + K and 2P for D, 5 N^3 log2 N^3 each, averaged over the pair."""
    b = w.get_bundle(w.config_small())
    nom, pru = bench._step_flops(b)
    n, p = b.spec.nfft, b.nks * b.spec.nbnd
    assert nom == pytest.approx(0.5 * (4 * p + 2) * 5 * n ** 3 * np.log2(n ** 3), rel=1e-12)
    assert 0 < pru < nom


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 500.0) == 8000.0
    assert bench.max_over_ranks(123.0, 1) == 123.0


def test_source_digest_is_stable():
    assert bench.source_digest() == bench.source_digest()
    assert len(bench.source_digest()) == 16


def test_committed_traffic_matches_the_sources():
    """The DRAM bytes per launch in profiles/roofline_traffic.txt were captured on the plane
    pass as it is now: a change to its code without a new capture fails here."""
    t = bench.profiled_traffic()
    assert t is not None and 3e8 < t < 4e8
