"""Multi-process paths on the CPU (gloo, 127.0.0.1).

1. The k-point split of a chain (each rank a block of k-points; the response density and
   the scalar products summed over ranks) reproduces the single-process recursions: the same
   coefficients up to the summation order of the k sums (1e-12 relative).  World sizes 2
   and 3 (8 k-points: blocks 4+4 and 3+3+2).
2. The benchmark's replica aggregation: the timed region is the slowest rank's, and the
   whole-job rate counts every rank's steps.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import workloads as w
from oracle import lanczos
from oracle.ksplit import KSplit, k_block
from oracle.liouvillian import System

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)


def _allreduce(a: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _ksplit_worker(rank, world, port, bundle, steps, outdir):
    _init(rank, world, port)
    try:
        ks = KSplit(System(bundle), rank, world, _allreduce)
        ph = lanczos.pseudo_hermitian(ks, steps[0])
        nh = lanczos.non_hermitian(ks, steps[1])
        if rank == 0:
            for tag, r in (("ph", ph), ("nh", nh)):
                np.save(os.path.join(outdir, f"{tag}.npy"), np.stack([r.beta, r.gamma, r.z]))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def tiny():
    return w.get_bundle(w.config_tiny())


def test_k_block_partition():
    for nks in (1, 7, 8, 64, 512):
        for world in (1, 2, 3, 5, 8):
            blocks = [k_block(nks, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == nks
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_ksplit_recursions_match_single_process(tiny, world):
    steps = (20, 10)
    sys1 = System(tiny)
    ref_ph = lanczos.pseudo_hermitian(sys1, steps[0])
    ref_nh = lanczos.non_hermitian(sys1, steps[1])
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_ksplit_worker, args=(world, _free_port(), tiny, steps, d), nprocs=world,
                           join=True, start_method="spawn")
        for tag, ref in (("ph", ref_ph), ("nh", ref_nh)):
            got = np.load(os.path.join(d, f"{tag}.npy"))
            for g, r in zip(got, (ref.beta, ref.gamma, ref.z)):
                assert np.max(np.abs(g - r)) <= 1e-12 * np.max(np.abs(r))


def _bench_worker(rank, world, port, outdir):
    _init(rank, world, port)
    try:
        import bench
        ms = [120.0, 150.0, 90.0][rank]
        tmax = bench.max_over_ranks(ms, world)
        if rank == 0:
            np.save(os.path.join(outdir, "agg.npy"), np.array([tmax, bench.whole_job_rate(1000, world, tmax)]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_replica_aggregation(world):
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_bench_worker, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        tmax, rate = np.load(os.path.join(d, "agg.npy"))
    want = max([120.0, 150.0, 90.0][:world])
    assert tmax == want
    assert rate == pytest.approx(world * 1000 / (want / 1e3))
