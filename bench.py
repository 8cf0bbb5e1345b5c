#!/usr/bin/env python3
"""Lanczos steps/s of the Liouville-Lanczos hot path on one GB300 (per rank).

Workload (the configuration the metric is quoted on): the two-atom FCC cell with
Kleinman-Bylander s/p projectors, 25 Ry, 32^3 FFT grid, 8x8x8 k-mesh, 4 bands (2048
response orbitals), Q = 0.1 (2 pi/a) x, TDDFT (RPA + ALDA) kernel, pseudo-Hermitian
recursion.  A step is one Lanczos step: the update of the Lanczos vectors and scalars plus
one application of the Liouvillian (D + K or D) to the whole batch.  `value` is the FP32
path (FP32 orbitals and FFTs, FP64 Lanczos scalars); the plain FP64 path is timed beside it
on the same steps, and the spectrum error of the FP32 path against it is reported.

Inputs: the seeded synthetic ground state of that cell (workloads/), built once and cached.
Device inputs stay resident; the per-step working set (orbital grids, column buffers,
vectors: ~0.6 GB in FP32) is larger than the 129 MB L2, so no flush is needed.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun every rank runs an independent chain on its own GPU (replicas; chains of
different momenta are independent problems) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lanczos steps/s (Liouvillian applies) FP32 vs FP64 @1e-3 err; p50/p99 latency"
WORKLOAD = ("fcc2kb_25ry_32: 2-atom FCC a=10.26 + KB s/p, 25 Ry, 32^3 FFT, 8x8x8 k, 4 bands, "
            "Q=0.1(2pi/a)x, RPA+ALDA, pseudo-Hermitian")
# every atom of the insulating cells also carries a repulsive KB s channel of 40 Ry: the local
# potential as specified binds a semimetal, which the insulator formalism cannot take
SCHANNEL = {"kb": "KB s channel D_s = 2 + 40 Ry per atom (40 Ry repulsive, added to open a gap: the cell "
                  "with the specified local potential alone is a semimetal); p channels D_p = -1 Ry",
            "cubic8": "repulsive KB s channel of 40 Ry per atom (gap opener); no other projectors"}
SCHANNEL["sc16"] = SCHANNEL["kb"]
SPEC_WINDOW = 100        # coefficients of the reproducible part of the recursion
FP32_PEAK_PER_SM_CLK = 128 * 2   # FP32 lanes per SM x 2 flops per FMA


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's timed region (ms); a host collective on the default group."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([ms], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps_per_rank: int, world: int, ms_max: float) -> float:
    """Steps/s of the whole job: every rank's steps over the slowest rank's time."""
    return world * steps_per_rank / (ms_max / 1e3)


def _bundle(workload: str = "kb"):
    import workloads as w
    if workload == "sc16":
        b = w.cached_bundle(w.config_sc16())
        if b is None:
            raise SystemExit("the sixteen-atom ground state is not cached (workloads.get_bundle(config_sc16()))")
        return b
    return w.get_bundle(w.config_cubic8() if workload == "cubic8" else w.config_kb())


def _pinned_packed(blocks):
    """A list of per-k complex arrays copied into one pinned, packed host buffer: (the numpy
    view, the torch tensor that owns the pinned memory)."""
    import torch
    n = sum(x.size for x in blocks)
    t = torch.empty(2 * max(n, 1), dtype=torch.float64, pin_memory=True)
    a = t.numpy().view(np.complex128)[:n]
    o = 0
    for x in blocks:
        a[o:o + x.size] = np.asarray(x).ravel()
        o += x.size
    return a, t


def _chain(b, precision, max_steps, stream, flavour="ph", packed=None):
    from paper_2111_06623_gb300 import ll
    s = b.spec
    p = packed or {}
    return ll.Chain(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq,
                    u_k=p.get("u_k", b.u_k), u_kq=p.get("u_kq", b.u_kq), eps_k=b.eps_k, vloc_r=b.vloc_r,
                    rho_r=b.rho_r, beta_kq=p.get("beta_kq", b.beta_kq),
                    dij=b.dij, q_cart=s.q_cart, approx="tddft", flavour=flavour, precision=precision,
                    max_steps=max_steps, stream=stream, kweight=b.kweight, sym=b.sym,
                    **({} if b.occ_k is None else dict(occ_k=b.occ_k, occ_kq=b.occ_kq, eps_kq=b.eps_kq)))


def _kb_wedge(b_full, stream, K, W):
    """The KB workload on the irreducible wedge of the small group of Q (Sec. 2.6: 164 of the
    512 k-points, star-size weights, the density averaged over the group): the same chain as
    the full mesh.  FP32 steps/s over K steps, and the loss function of its first 100
    coefficients against the oracle's full-mesh golden coefficients (when they match the
    full-mesh bundle)."""
    import workloads as w
    b = w.get_bundle(w.config_kb(True))
    ch, c, ms, _ = _time_chain(b, "fp32", K, W, stream, extra=64 + SPEC_WINDOW)
    if ch.steps < SPEC_WINDOW:
        ch.lanczos(SPEC_WINDOW - ch.steps)
    c = ch.lanczos(0)
    ch.close()
    ref = _golden(b_full, "kb_ph", SPEC_WINDOW)
    return {"workload": "fcc2kb_25ry_32 on the irreducible wedge of the small group of Q (C2v)",
            "kpoints": int(b.nks), "kpoints_full_mesh": int(np.sum(b.kweight)), "steps": K,
            "steps_per_s": K / (ms / 1e3), "ms_per_step": ms / K, "dtype": "f32",
            "loss_err_vs_full_mesh_oracle_100": None if ref is None else _loss_err(c, ref, b_full, SPEC_WINDOW)}


def _bundle_bytes(b) -> int:
    n = sum(a.nbytes for a in (b.kcart, b.eps_k, b.vloc_r, b.rho_r, b.dij))
    n += sum(m.nbytes for m in b.miller_k) + sum(m.nbytes for m in b.miller_kq)
    n += sum(u.nbytes for u in b.u_k) + sum(u.nbytes for u in b.u_kq) + sum(x.nbytes for x in b.beta_kq)
    return int(n)


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _xy_flops_per_apply(b, with_k: bool) -> float:
    """Algorithmic FP32 flops of the per-plane kernel for one operator application: for every
    orbital and plane, (rows + N) inverse and (N + rows) forward line FFTs of 5 N log2 N flops,
    the V(r) x(r) product (2 flops/point) and, with K, the density product (8 flops/point)."""
    n = b.spec.nfft
    line = 5.0 * n * np.log2(n)
    tot = 0.0
    for m in b.miller_kq:
        rows = len(np.unique(m[:, 1]))       # sphere rows: columns of equal m2
        per_plane = (2 * rows + 2 * n) * line + (2 + (8 if with_k else 0)) * n * n
        tot += b.spec.nbnd * n * per_plane
    return tot


def _small_cell(stream):
    import torch
    import workloads as w
    bs = w.get_bundle(w.config_small())
    ch, _, ms, _ = _time_chain(bs, "fp64", 300, 5, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ch.spectrum(np.linspace(0.0, 40.0, 4001), 0.1)
    e1.record()
    torch.cuda.synchronize()
    ch.close()
    return {"workload": "fcc2_10ry_18: 2-atom FCC, 10 Ry, 18^3, 4x4x4 k, 4 bands, RPA+ALDA, PH, FP64, "
                        "repulsive KB s channel of 40 Ry per atom (gap opener; no p channels)",
            "steps": 300, "steps_per_s": 300 / (ms / 1e3), "ms_per_step": ms / 300,
            "spectrum_ms": e0.elapsed_time(e1), "dtype": "f64"}


def _metal_cell(stream, steps: int = 300, window: int = 80):
    """The semimetal with smeared occupations (Sec. 2.6: two-atom cell with its bare local
    potential, 10 Ry, 18^3, 4x4x4 k, 6 bands with fractional occupations, RPA+ALDA, PH):
    FP32 and FP64 steps/s over 300 steps, the FP64 coefficients of the first 100 steps and the
    FP32 loss function of the first 80 (the cell's FP32 window) against the oracle's golden
    coefficients of the same bundle."""
    import workloads as w
    b = w.get_bundle(w.config_metal())
    out = {"workload": "fcc2metal_10ry_18: 2-atom semimetal, Gaussian smearing 0.04 Ry, 10 Ry, 18^3, "
                       "4x4x4 k, 6 bands, RPA+ALDA, PH", "steps": steps}
    ref = _golden(b, "metal_ph", 100)
    for prec in ("fp32", "fp64"):
        ch, c, ms, _ = _time_chain(b, prec, steps, 5, stream)
        ch.close()
        out[prec] = {"steps_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps}
        if ref is not None and prec == "fp32":
            out[prec]["loss_err_vs_oracle_80"] = _loss_err(c, ref, b, window)
        if ref is not None and prec == "fp64":
            out[prec]["coef_err_vs_oracle_100"] = float(np.max(np.abs(c[0][:100] - ref[0]) / np.abs(ref[0])))
    return out


def _step_flops(b) -> tuple[float, float]:
    """FFT flops of one pseudo-Hermitian step (the mean of a D+K and a D application):
    (nominal, pruned).  Nominal: 5 N^3 log2 N^3 per full 3D FFT, 2P + 2 FFTs for D+K and 2P
    for D (P orbitals).  Pruned (what the kernels compute): per orbital, the sphere's
    columns along axis 3 both ways, the per-plane passes of _xy_flops_per_apply, pass 2's
    (N + rows) forward lines per plane, and two full FFTs of the response density."""
    n = b.spec.nfft
    nb = b.spec.nbnd
    p = b.nks * nb
    full = 5.0 * n ** 3 * np.log2(n ** 3)
    nominal = 0.5 * ((2 * p + 2) + 2 * p) * full
    line = 5.0 * n * np.log2(n)
    axis3 = sum(nb * 2 * len({(a, c) for a, c in m[:, :2].tolist()}) * line for m in b.miller_kq)
    pass2 = sum(nb * n * ((n + len(np.unique(m[:, 1]))) * line + 6 * n * n) for m in b.miller_kq)
    dk = _xy_flops_per_apply(b, True) + pass2 + axis3 + 2 * full
    d = _xy_flops_per_apply(b, False) + axis3
    return nominal, 0.5 * (dk + d)


def _sc16(stream, steps: int = 2000):
    """The sixteen-atom cell (32 bands, 48^3, 64 KB projectors, 2048 orbitals of ~6000 plane
    waves; the split per-k path with tensor-core projections), the configured 2000 FP32
    pseudo-Hermitian steps, when its ground state is cached (building it takes ~90 minutes of
    CPU); with the loss function of the first 100 coefficients against the oracle's golden
    coefficients of the same bundle."""
    import workloads as w
    b = w.cached_bundle(w.config_sc16())
    if b is None:
        return {"skipped": "ground state not cached (workloads.get_bundle(config_sc16()) takes ~90 min of CPU)"}
    ch, c, ms, _ = _time_chain(b, "fp32", steps, 3, stream)
    ch.close()
    ref = _golden(b, "sc16_ph", SPEC_WINDOW)
    return {"workload": "sc16kb_30ry_48: 16-atom 2x2x2 supercell + KB s/p, 30 Ry, 48^3, 4x4x4 k, 32 bands, PH",
            "steps": steps, "steps_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps, "dtype": "f32",
            "loss_err_vs_oracle_100": None if ref is None else _loss_err(c, ref, b, SPEC_WINDOW)}


def source_digest() -> str:
    """sha256 of the code that sets the plane pass's DRAM traffic per launch: common.cuh,
    fft.cuh, the k_xy section of kernels.cuh and its batch sizes and launch in chain.cuh."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2111_06623_gb300", "csrc")

    def read(name):
        with open(os.path.join(csrc, name)) as fh:
            return fh.read()

    def between(text, start, end):
        i = text.index(start)
        return text[i:text.index(end, i)]

    k = read("kernels.cuh")
    c = read("chain.cuh")
    parts = [read("common.cuh"), read("fft.cuh"),
             between(k, "// Per-plane pass of one operator application.", "// Response potential of one density"),
             between(c, "template <int N, int MODE> struct BO", "};"),
             between(c, "  int xy_nm(", "  // mode 0: operator pass 1")]
    return hashlib.sha256("\0".join(parts).encode()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel class from the committed ncu summary
    (profiles/roofline_traffic.txt), or None when the sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_digest") != source_digest():
        return None
    try:
        return float(kv["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _time_chain(b, precision, steps, warmup, stream, profile=False, flavour="ph", extra=64):
    import torch
    ch = _chain(b, precision, warmup + steps + extra, stream, flavour)
    ch.lanczos(warmup)
    torch.cuda.synchronize()
    if profile:
        ch.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    coefs = ch.lanczos(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = ch.profile_read() if profile else None
    return ch, coefs, ms, prof


def _golden(b, case: str, n: int):
    """The oracle's first n coefficients of a workload from the committed golden file
    (tests/golden/oracle_<case>.txt, written by the oracle), when the bundle is the very input
    they were computed on (same digest); else None."""
    import workloads as w
    from tests.golden import write_workload_golden as gold
    g = gold.load(case)
    if g is None or g[1] < n or g[0] != w.bundle_digest(b):
        return None
    return g[2][:n], g[3][:n], g[4][:n]


def _loss_err(a, ref, b, m):
    la, lr = _loss(a, b, m), _loss(ref, b, m)
    return float(np.max(np.abs(la - lr)) / np.max(np.abs(lr)))


def _loss(coefs, b, m):
    from paper_2111_06623_gb300 import ll
    w = np.linspace(0.0, 40.0, 4001)
    beta, gamma, z = (c[:m] for c in coefs)
    _, ei, _ = ll.spectrum(beta, gamma, z, b.spec.omega, b.spec.q_cart, w, 0.1)
    return -ei.imag


def oracle_timing(spec, warm: int, timed: int, world: int | None = None):
    """The FP64 oracle on every host core: one pseudo-Hermitian chain of the whole workload
    (every k-point) through oracle.pool (the k-point split over one single-threaded process per
    core, gloo sums).  Returns (seconds per step over steps warm+1 .. warm+timed, processes,
    wall seconds including start-up)."""
    from oracle import pool
    t0 = time.perf_counter()
    _, marks, used = pool.run(spec, warm + timed, "ph", world=world)
    per = (marks[warm + timed] - marks[warm]) / timed
    return per, used, time.perf_counter() - t0


def oracle_sample_text(spec, warm, timed, used, nks):
    return (f"steps {warm + 1}-{warm + timed} (after {warm} untimed) of one pseudo-Hermitian chain of the whole "
            f"workload ({nks} k-points, FP64 NumPy/SciPy oracle), k-point split over {used} single-threaded "
            f"processes (one per host core); measured, not scaled")


def _serving(b_kb, n_jobs: int, seed: int = 7):
    """A Poisson stream (mean 20 jobs/s, arrivals from default_rng(seed)) of Lanczos jobs
    through the request loop under a 150 GB HBM budget: each job picks a configuration
    uniformly -- the small two-atom cell at one of four q of the many-Q pool, the KB workload,
    the sixteen-atom cell (the eight-atom cell at one of two q of the pool where the
    sixteen-atom ground state is not cached) -- and U[500, 3000] pseudo-Hermitian FP32 steps.
    Returns throughput and the p50/p99 time from submission to the finished spectrum."""
    import workloads as w
    from paper_2111_06623_gb300 import ll
    pools = _batch_bundles(4, 2)
    b16 = w.cached_bundle(w.config_sc16())
    third = [b16] if b16 is not None else pools["cubic8_20ry_32"]
    cells = [pools["fcc2_10ry_18"], [b_kb], third]
    rng = np.random.default_rng(seed)
    wgrid = np.linspace(0.0, 40.0, 4001)
    srv = ll.Server(hbm_budget_bytes=150 << 30, max_slots=16, chunk=32)
    t_arr = np.cumsum(rng.exponential(1.0 / 20.0, size=n_jobs))
    picks = rng.integers(0, len(cells), size=n_jobs)
    steps = rng.integers(500, 3001, size=n_jobs)
    which = rng.integers(0, 1 << 30, size=n_jobs)
    ids, t0 = [], time.perf_counter()
    for ta, pk, ns, wq in zip(t_arr, picks, steps, which):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.001)
        bb = cells[pk][wq % len(cells[pk])]
        s = bb.spec
        ids.append(srv.submit(int(ns), wgrid, 0.1, lattice=s.lattice, nfft=s.nfft, kcart=bb.kcart,
                              miller_k=bb.miller_k, miller_kq=bb.miller_kq, u_k=bb.u_k, u_kq=bb.u_kq, eps_k=bb.eps_k,
                              vloc_r=bb.vloc_r, rho_r=bb.rho_r, beta_kq=bb.beta_kq, dij=bb.dij, q_cart=s.q_cart,
                              approx="tddft", flavour="ph", precision="fp32", max_steps=int(ns)))
    lat, done = {}, 0
    while len(lat) < len(ids):
        for i in ids:
            if i not in lat:
                st, r = srv.poll(i)
                if st in (ll.JOB_DONE, ll.JOB_FAILED):
                    lat[i] = r["queue_s"] + r["run_s"]
                    done += r["steps_done"] if st == ll.JOB_DONE else 0
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    peak = srv.stats()["peak"]
    srv.close()
    v = np.array(list(lat.values()))
    per_cfg = {}
    for pk, ns in zip(picks, steps):
        c = per_cfg.setdefault(["fcc2_10ry_18", "fcc2kb_25ry_32", third[0].spec.name][pk], {"jobs": 0, "steps": 0})
        c["jobs"] += 1
        c["steps"] += int(ns)
    return {"jobs": n_jobs, "steps_per_s": done / wall, "p50_s": float(np.percentile(v, 50)),
            "p99_s": float(np.percentile(v, 99)), "wall_s": wall, "peak_hbm_gb": peak / 2 ** 30,
            "budget_gb": 150, "slots": 16, "per_config": per_cfg,
            "stream": (f"Poisson 20 jobs/s (seed 7), first {n_jobs} jobs of the stream; configuration "
                       f"U{{2-atom 10 Ry at 4 q, KB workload, {third[0].spec.name}}}; U[500, 3000] FP32 PH steps")}


def q_pool(n: int = 64) -> np.ndarray:
    """Momentum transfers of the many-Q batch: |q| ~ U(0.05, 0.6) 2 pi/a, direction a
    normalised Gaussian 3-vector, drawn from default_rng(4) (magnitudes first)."""
    import workloads as w
    rng = np.random.default_rng(4)
    mag = rng.uniform(0.05, 0.6, size=n) * (2 * np.pi / w.A_LAT)
    d = rng.normal(size=(n, 3))
    return mag[:, None] * d / np.linalg.norm(d, axis=1, keepdims=True)


def _batch_bundles(n_small: int, n_cubic: int):
    """Ground states of the first q of the pool on the two-atom cell (10 Ry, 18^3, 4^3 k) and
    on the eight-atom cubic cell (20 Ry, 32^3, 4^3 k, 16 bands); a q whose sphere puts a plane
    wave on the cut-off is skipped."""
    import workloads as w
    out = {"fcc2_10ry_18": [], "cubic8_20ry_32": []}
    for cell, n, mk in (("fcc2_10ry_18", n_small, lambda q: _with_q(w.config_small(), q)),
                        ("cubic8_20ry_32", n_cubic, w.config_cubic8)):
        for q in q_pool():
            if len(out[cell]) >= n:
                break
            try:
                spec = mk(q)
                spec.name = "%s_q%s" % (cell, "_".join("%+.4f" % c for c in q))
                out[cell].append(w.get_bundle(spec))
            except ValueError:
                continue
    return out


def _with_q(spec, q):
    spec.q_cart = np.asarray(q, dtype=np.float64)
    return spec


def _batch(n_small: int, n_cubic: int, steps: int = 1500, n_sc16: int = 1):
    """Many independent chains on one GPU at once: n_small momentum transfers of the pool on
    the two-atom cell, n_cubic on the eight-atom cell and (where its ground state is cached)
    the sixteen-atom cell at its configured q, all submitted together to the request loop (one
    stream per chain), steps FP32 pseudo-Hermitian steps each.  Returns the whole batch's
    steps/s and the wall time to the last spectrum."""
    import workloads as w
    from paper_2111_06623_gb300 import ll
    pools = _batch_bundles(n_small, n_cubic)
    if n_sc16 > 0:
        b16 = w.cached_bundle(w.config_sc16())
        pools["sc16kb_30ry_48"] = [b16] if b16 is not None else []
    jobs = [(cell, b) for cell, bs in pools.items() for b in bs]
    wgrid = np.linspace(0.0, 40.0, 4001)
    srv = ll.Server(hbm_budget_bytes=150 << 30, max_slots=len(jobs), chunk=32)
    ids, t0 = [], time.perf_counter()
    for cell, bb in jobs:
        s = bb.spec
        ids.append(srv.submit(steps, wgrid, 0.1, lattice=s.lattice, nfft=s.nfft, kcart=bb.kcart,
                              miller_k=bb.miller_k, miller_kq=bb.miller_kq, u_k=bb.u_k, u_kq=bb.u_kq, eps_k=bb.eps_k,
                              vloc_r=bb.vloc_r, rho_r=bb.rho_r, beta_kq=bb.beta_kq, dij=bb.dij, q_cart=s.q_cart,
                              approx="tddft", flavour="ph", precision="fp32", max_steps=steps))
    res = {}
    while len(res) < len(ids):
        for i, (cell, _) in zip(ids, jobs):
            if i not in res:
                st, r = srv.poll(i)
                if st in (ll.JOB_DONE, ll.JOB_FAILED):
                    res[i] = (cell, st, r)
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    peak = srv.stats()["peak"]
    srv.close()
    done = sum(r["steps_done"] for _, st, r in res.values() if st == ll.JOB_DONE)
    per_cell = {}
    for cell, st, r in res.values():
        c = per_cell.setdefault(cell, {"chains": 0, "failed": 0, "mean_run_s": 0.0})
        c["chains"] += 1
        c["failed"] += st != ll.JOB_DONE
        c["mean_run_s"] += r["run_s"]
    for c in per_cell.values():
        c["mean_run_s"] /= max(1, c["chains"])
    # one eight-atom chain alone (CUDA events, FP32): the per-chain speed of the larger cell
    single = None
    if pools["cubic8_20ry_32"]:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
        ch, _, ms, _ = _time_chain(pools["cubic8_20ry_32"][0], "fp32", 300, 5, stream)
        ch.close()
        single = {"cell": "cubic8_20ry_32", "steps": 300, "steps_per_s": 300 / (ms / 1e3), "ms_per_step": ms / 300}
    return {"chains": len(jobs), "steps_per_chain": steps, "steps_per_s": done / wall, "wall_s": wall,
            "single_chain": single,
            "peak_hbm_gb": peak / 2 ** 30, "cells": per_cell,
            "q_pool": "64 q, |q| ~ U(0.05, 0.6) 2pi/a, Gaussian directions, default_rng(4); first q of the pool per cell"}


REF_MAX_STEPS = 40      # timed oracle steps at most in one reference run (a few minutes of CPU)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.perf_counter()
    b = _bundle()
    warm = max(1, min(args.warmup, 10))
    timed = max(1, min(args.steps, REF_MAX_STEPS))
    per, used, _ = oracle_timing(b.spec, warm, timed)
    value = 1.0 / per
    sample = oracle_sample_text(b.spec, warm, timed, used, b.nks)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": timed, "warmup": warm, "ms_per_step": 1e3 * per, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "projectors": SCHANNEL["kb"], "kpoints": int(b.nks),
                       "orbitals": int(b.nks * b.spec.nbnd)},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=20, help="timed oracle steps of the CPU baseline (0: none)")
    ap.add_argument("--serving-jobs", type=int, default=16, help="jobs of the Poisson stream (400 in the paper-derived stream)")
    ap.add_argument("--workload", default="kb", choices=["kb", "cubic8", "sc16"],
                    help="cell of the timed chain with --headline-only (profiling); the benchmark line is the KB workload")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the FP32 chain on the KB workload only (no other legs): for profiling")
    ap.add_argument("--batch-small", type=int, default=64, help="chains of the two-atom cell in the many-Q batch")
    ap.add_argument("--batch-cubic", type=int, default=2, help="chains of the eight-atom cell in the many-Q batch")
    ap.add_argument("--batch-sc16", type=int, default=1, help="chains of the sixteen-atom cell in the batch (0 or 1)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.workload != "kb" and not args.headline_only:
        ap.error("--workload other than kb is for --headline-only profiling runs")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll

    b = _bundle(args.workload)
    # a dedicated stream: the chains capture their steps into CUDA graphs there (the legacy
    # default stream cannot be captured)
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream().cuda_stream
    K, W = args.steps, args.warmup

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # FP32 path: the headline, with per-kernel-class device time
    barrier()
    extra = 64 + SPEC_WINDOW + 64      # room for the spectrum check and the latency samples
    with Clocks(local) as clk:
        ch32, c32, ms32, _ = _time_chain(b, "fp32", K, W, stream, extra=extra)
    barrier()
    clocks = clk.summary()
    # the same steps again with per-kernel-class CUDA events (eager launches: a profiled step is
    # not replayed from its graph), for the class times and the roofline of the dominant kernel
    chp, _, ms32_prof, prof = _time_chain(b, "fp32", K, W, stream, profile=True)
    chp.close()
    if args.headline_only:   # the FP32 chain alone (for profiling the headline's kernels)
        ch64, c64, ms64 = ch32, c32, ms32
        nh = small = None
    else:
        # FP64 path on the same number of steps
        ch64, c64, ms64, _ = _time_chain(b, "fp64", K, W, stream, extra=extra)
        # the non-Hermitian recursion (two applications per step), FP32, same steps
        chnh, _, msnh, _ = _time_chain(b, "fp32", K, W, stream, flavour="nh")
        chnh.close()
        nh = {"value": world * K / (msnh / 1e3), "ms_per_step": msnh / K, "applies_per_step": 2, "dtype": "f32"}
        # the small two-atom cell (10 Ry, 18^3, 4^3 k, 256 orbitals): 300 FP64 pseudo-Hermitian
        # steps and the spectrum, on the device
        small = _small_cell(stream)
    sc16 = None if args.headline_only else _sc16(stream)
    wedge = None if args.headline_only else _kb_wedge(b, stream, K, W)
    metal = None if args.headline_only else _metal_cell(stream)
    # the spectrum check spans the first SPEC_WINDOW coefficients whatever K is: the chains run
    # on, untimed, to that many steps
    kt = len(c32[0])
    if not args.headline_only:
        for ch in (ch32, ch64):
            if ch.steps < SPEC_WINDOW:
                ch.lanczos(SPEC_WINDOW - ch.steps)
        c32, c64 = ch32.lanczos(0), ch64.lanczos(0)
    m = min(SPEC_WINDOW, len(c32[0]), len(c64[0]))
    spec_err = _loss_err(c32, c64, b, m)
    spec_err_full = _loss_err(tuple(c[:kt] for c in c32), tuple(c[:kt] for c in c64), b, kt)
    vs_oracle = None
    ref = None if args.headline_only else _golden(b, "kb_ph", m)
    if ref is not None:
        vs_oracle = {"coefficients": m, "source": "tests/golden/oracle_kb_ph.txt (same bundle digest)",
                     "loss_err_fp32": _loss_err(c32, ref, b, m), "loss_err_fp64": _loss_err(c64, ref, b, m),
                     "coef_err_fp64": float(np.max(np.abs(c64[0][:m] - ref[0]) / np.abs(ref[0])))}
    # per-step latency (single-step calls, host sync included)
    lat = []
    for _ in range(0 if args.headline_only else 50):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if ch32.steps >= ch32.max_steps:
            break
        e0.record()
        ch32.lanczos(1)
        e1.record()
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
    ch32.close()
    if ch64 is not ch32:
        ch64.close()

    # end to end through the C ABI with host buffers: create (H2D of the ground state and
    # set-up), K steps, spectrum, coefficients and spectrum back to the host
    e2e = None
    if not args.headline_only:
        # the inputs as a caller holds them for repeated runs: packed in the descriptor's
        # layout in pinned host memory (prepared before the timed region; the H2D copies of
        # the ground state are inside it, in ll_create)
        pinned = {name: _pinned_packed(getattr(b, name)) for name in ("u_k", "u_kq", "beta_kq")}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        che = _chain(b, "fp32", K, stream, packed={n: a for n, (a, _) in pinned.items()})
        ce = che.lanczos(K)
        wgrid = np.linspace(0.0, 40.0, 4001)
        chi, ei, eps = che.spectrum(wgrid, 0.1)
        che.close()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": K / t_e2e, "unit": "steps/s", "h2d_bytes_per_step": _bundle_bytes(b) / K,
               "d2h_bytes_per_step": (sum(c.nbytes for c in ce) + chi.nbytes + ei.nbytes + eps.nbytes) / K}

    # max over ranks of the timed region; the whole job's steps over that time
    tmax = max_over_ranks(ms32, world)
    value = whole_job_rate(K, world, tmax)

    ms_cls, launches, total = prof
    dom = max(ms_cls, key=ms_cls.get)
    n_dom = max(1, launches[dom])
    # one pass-1 launch per operator application; half of the K applications carry K
    flops = 0.5 * (_xy_flops_per_apply(b, True) + _xy_flops_per_apply(b, False))
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = 152 * FP32_PEAK_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    roofline = None
    if dom == "xy1":
        ach = flops / (ms_cls[dom] / n_dom / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": "k_xy (pass 1: per-plane 2D FFTs, V x, density)", "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": profiled_traffic(),
                    "traffic_unit": "bytes per launch (mean of the D+K and D launches)",
                    "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flops x max SM clock (derived)"}
    else:
        roofline = {"bound": "alu", "kernel": dom, "achieved": None, "peak": peak, "unit": "TFLOP/s",
                    "frac": None, "traffic": None}

    fma32 = fma64 = None
    if not args.headline_only:
        fma32 = ll.fma_peak("fp32", stream)
        fma64 = ll.fma_peak("fp64", stream)
    if roofline.get("achieved") and fma32:
        roofline["peak_measured_fma"] = fma32
        roofline["frac_of_measured_fma"] = roofline["achieved"] / fma32
    nom, pru = _step_flops(b)
    step_roofline = {"fft_gflop_per_step_nominal": nom / 1e9, "fft_gflop_per_step_pruned": pru / 1e9,
                     "achieved_tflops_nominal": nom * value / world / 1e12,
                     "achieved_tflops_pruned": pru * value / world / 1e12,
                     "frac_nominal": nom * value / world / 1e12 / peak, "frac_pruned": pru * value / world / 1e12 / peak,
                     "peak_tflops": peak, "bound": "alu",
                     "measured_fma_tflops": {"fp32": fma32, "fp64": fma64},
                     "frac_nominal_of_measured_fma": nom * value / world / 1e12 / fma32 if fma32 else None}
    serving = _serving(b, args.serving_jobs) if args.serving_jobs > 0 and not args.headline_only else None
    batch = (_batch(args.batch_small, args.batch_cubic, n_sc16=args.batch_sc16)
             if args.batch_small + args.batch_cubic > 0 and not args.headline_only else None)

    cpu = None
    if rank == 0 and not args.headline_only and args.cpu_steps > 0:
        per, used, wall = oracle_timing(b.spec, 10, args.cpu_steps)
        cpu = {"value": 1.0 / per, "unit": "steps/s", "cores": used, "kind": "oracle",
               "sample": oracle_sample_text(b.spec, 10, args.cpu_steps, used, b.nks), "wall_s": wall}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": tmax / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded LDA ground state, workloads/)",
            "config": {"workload": WORKLOAD if args.workload == "kb" else b.spec.name, "projectors": SCHANNEL[args.workload],
                       "orbitals": int(b.nks * b.spec.nbnd), "npw_avg": float(np.mean(b.npw_kq)),
                       "l2": "per-step working set ~0.6 GB > 129 MB L2 (no flush)", "parallelism": "replicas"},
            "fp64": None if args.headline_only else {"value": world * K / (ms64 / 1e3), "ms_per_step": ms64 / K,
                                                      "dtype": "f64"},
            "nh_fp32": nh, "small_cell": small, "sc16": sc16, "kb_wedge": wedge, "metal": metal,
            "speedup_fp32_vs_fp64": ms64 / ms32,
            "spectrum_err_fp32_vs_fp64": spec_err, "spectrum_window_steps": m,
            "spectrum_err_fp32_vs_fp64_timed_steps": spec_err_full, "spectrum_vs_oracle": vs_oracle,
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))} if lat else None,
            "kernel_ms": ms_cls, "kernel_launches": launches, "ms_per_step_eager_profiled": ms32_prof / K,
            "roofline": roofline, "step_roofline": step_roofline, "serving": serving, "batch": batch, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(total), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
