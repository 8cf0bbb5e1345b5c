"""The oracle's recursions on every host core: the k-point split of `oracle.ksplit` (the
paper's k-point pools, Sec. 4) run by W local processes that sum over gloo on 127.0.0.1.

Test and benchmark infrastructure, like the rest of `oracle/`: it runs the unchanged
recursions of `oracle.lanczos` on the k-blocks of `oracle.ksplit.KSplit` (the decomposition
pinned against the single-process recursions by the world-size 2 and 3 tests), one
single-threaded process per core.  It changes how the k sums are grouped, not what is
summed, so the coefficients agree with a single process to rounding.

Processes start with the `spawn` method: a process forked after CUDA has been initialised
in the parent would hang.  Each worker loads the ground-state bundle from the input
generator's cache (`workloads.get_bundle`), so the caller must have built it first.
"""
from __future__ import annotations

import os
import queue as queue_mod
import socket
import time

import numpy as np

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, spec, approx, flavour, nsteps, out):
    import torch
    import torch.distributed as dist

    import workloads as w
    from oracle import lanczos
    from oracle.ksplit import KSplit
    from oracle.liouvillian import System

    torch.set_num_threads(1)
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)

        def allreduce(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        bundle = w.get_bundle(spec)
        ks = KSplit(System(bundle, approx), rank, world, allreduce)
        dist.barrier()
        marks = {}
        t0 = time.perf_counter()
        co = lanczos.run(ks, nsteps, flavour, on_step=lambda j: marks.__setitem__(j, time.perf_counter() - t0))
        dist.barrier()
        if rank == 0:
            out.put(("ok", co.beta, co.gamma, co.z, co.applies, marks))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001  (reported to the caller, which raises)
        out.put(("error", f"rank {rank}: {type(e).__name__}: {e}"))


def default_world() -> int:
    return max(1, os.cpu_count() or 1)


def run(spec, nsteps: int, flavour: str, approx: str | None = None, world: int | None = None,
        timeout: float = 7200.0):
    """The oracle's first nsteps coefficients of one chain of `spec` over `world` processes.

    Returns (Coefficients, marks, world): marks[j] = seconds from the start of the recursion
    (after set-up) to the moment step j's coefficients were known."""
    import multiprocessing as mp

    from oracle.lanczos import Coefficients

    world = world or default_world()
    approx = approx or spec.approx
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        procs = [ctx.Process(target=_worker, args=(r, world, port, spec, approx, flavour, nsteps, out))
                 for r in range(world)]
        for p in procs:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    try:
        try:
            res = out.get(timeout=timeout)
        except queue_mod.Empty:
            raise RuntimeError(f"oracle pool: no result within {timeout} s") from None
        if res[0] != "ok":
            raise RuntimeError("oracle pool failed: " + res[1])
        _, beta, gamma, z, applies, marks = res
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
                p.join()
    return Coefficients(beta=beta, gamma=gamma, z=z, applies=applies, flavour=flavour), marks, world
