#!/usr/bin/env python
"""Benchmark of GPU visual matrix ordering: nnz ordered per second (recursive
BBD), one JSON line on stdout.

Workload (one step): the medium configuration — a 3D 7-point Laplacian on a
64^3 grid (262,144 rows, 1,810,432 nnz) and a seeded random symmetric
power-law matrix with 500,000 rows (~5.6M nnz) — each taken from a
device-resident CSR to device-resident permutations: hypergraph build,
multilevel layout in d = 3 (T = 100 steps per level), recursive BBD to depth
10.  Inputs are synthetic (seeded generators in ``workloads``).

Timing: W untimed warm-up steps, then K steps, each bracketed by a device
synchronisation and timed with CUDA events on the current stream; the L2 cache
(129 MB) is flushed by writing a 512 MB buffer before every timed step.  The
roofline of the step kernel comes from K more steps with CUDA events around
every step-kernel launch (not part of the value: per-launch events turn off
the library's CUDA-graph replay of the layout steps).

Further legs (under "modes"): batched — 4,096 matrices of the batch mix in one
batch against one-at-a-time calls; served — a Poisson request stream through
the request server with latency percentiles.
Under torchrun every rank orders its own replica (weak scaling, no
collective on the data path); the time is the max over ranks.

--impl reference times the CPU oracle (test infrastructure, FP64, single
thread) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "nnz ordered/sec (recursive BBD)"
# algorithmic FP32 operations per source interaction of the layout step kernel
# (differences, squared norm, reciprocal power, force accumulation), per d
FLOPS_PER_INTERACTION = {2: 10, 3: 18, 4: 23}


MEDIUM_NAME = "grid3d_64^3+powerlaw_500k"


def medium_workload():
    mats = [(W.grid_laplacian_3d(64), dict(d=3, max_depth=10)),
            (W.powerlaw_symmetric(500_000, seed=1), dict(d=3, max_depth=10))]
    return MEDIUM_NAME, mats


def cpu_sample(small: bool, single: bool = False):
    """Bounded sample of the medium workload for the oracle: the same two
    families with the same parameters, scaled down (single: the sample of the
    single-thread timing)."""
    if single:
        return "grid3d_16^3+powerlaw_2000", [(W.grid_laplacian_3d(16), dict(d=3, max_depth=10)),
                                              (W.powerlaw_symmetric(2000, seed=1), dict(d=3, max_depth=10))]
    if small:
        return "grid3d_12^3+powerlaw_1000", [(W.grid_laplacian_3d(12), dict(d=3, max_depth=10)),
                                               (W.powerlaw_symmetric(1000, seed=1), dict(d=3, max_depth=10))]
    return "grid3d_32^3+powerlaw_20000", [(W.grid_laplacian_3d(32), dict(d=3, max_depth=10)),
                                           (W.powerlaw_symmetric(20_000, seed=1), dict(d=3, max_depth=10))]


def host_cpu() -> dict:
    """Model name and core count of the host CPU (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    model = v
                    break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"cpu_model": model or "unknown", "cpu_cores": os.cpu_count() or 1, "arch": platform.machine()}


def oracle_step(mats, seed=1):
    import oracle
    nnz = 0
    for A, cfg in mats:
        hg = oracle.build_from_matrix("symmetric", A)
        x = oracle.layout_multilevel(hg, cfg["d"], seed)
        oracle.order(hg, cfg["d"], x.astype(np.float32), seed=seed, max_depth=cfg["max_depth"])
        nnz += A.nnz
    return nnz


def _oracle_order_one(A) -> int:
    """One matrix through the oracle's full pipeline (a worker of the all-core
    baseline, one thread: the pool gives one worker per core; touches no GPU)."""
    import oracle
    oracle.set_threads(1)
    return oracle_step([(A, dict(d=3, max_depth=62))])


def batch_cpu_all_cores(mats=None, count: int = 0, max_nnz: int = 15_000) -> dict:
    """The oracle on all host cores over independent matrices of the batch mix:
    a seeded sample of `count` (default: one per core; 128 in the default run)
    of the 4,096 matrices among those of at most `max_nnz` nonzeros, one
    matrix per task, a spawn process pool of one worker per core."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    mats = mats if mats is not None else W.batch_mix(4096, seed=1)
    small = [i for i, A in enumerate(mats) if A.nnz <= max_nnz]
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(24)
    pick = sorted(int(i) for i in rng.choice(small, size=min(count or cores, len(small)), replace=False))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        nnz = sum(pool.map(_oracle_order_one, [mats[i] for i in pick], chunksize=1))
    dt = time.perf_counter() - t0
    return {"value": nnz / dt, "unit": "nnz/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(pick)} matrices of the batch mix with <= {max_nnz} nnz (seeded), {nnz} nnz, oracle "
                      f"FP64 full pipeline (multilevel layout d=3, recursive BBD, min_part 64), one matrix per "
                      f"worker process, {dt:.1f} s", **host_cpu()}


def run_cpu_baseline(mats, sample_name):
    """The oracle on all host cores (OpenMP over the per-vertex loops) over a
    bounded sample, and single-threaded over a smaller one."""
    import oracle
    oracle.build()
    th = oracle.threads()  # the oracle's per-vertex loops run on this many OpenMP threads
    t0 = time.perf_counter()
    nnz = oracle_step(mats)
    dt = time.perf_counter() - t0
    s_name, s_mats = cpu_sample(small=False, single=True)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    s_nnz = oracle_step(s_mats)
    s_dt = time.perf_counter() - t1
    oracle.set_threads(th)
    return {"value": nnz / dt, "unit": "nnz/s", "cores": th, "kind": "oracle",
            "sample": f"{sample_name}: oracle FP64 as built (OpenMP over the per-vertex gradient loop, {th} "
                      f"threads), full pipeline (multilevel layout d=3, T=100 per level, recursive BBD depth 10), "
                      f"{nnz} nnz in {dt:.1f} s",
            "single_thread": {"value": s_nnz / s_dt, "unit": "nnz/s", "cores": 1,
                              "sample": f"{s_name}: the same oracle on one thread, {s_nnz} nnz in {s_dt:.1f} s"}}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"vmo_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def gpu_step(V, torch, mats, dev_csr, params):
    """Build + layout + recursive BBD of every matrix; returns nnz ordered."""
    nnz = 0
    for (A, cfg), (rp, ci) in zip(mats, dev_csr):
        hg = V.Hypergraph(rp, ci, A.m, A.n, "symmetric")
        p = V.Params(d=cfg["d"], max_depth=cfg["max_depth"], seed=params["seed"])
        hg.order(p, None, sbd=False, with_tree=True)
        nnz += A.nnz
        del hg
    return nnz


def batched_leg(V, torch, count: int, plain_sample: int, warmup: int, steps: int, flush, mats=None):
    """Config-4 distribution: `count` independent matrices ordered to BBD in one
    batch (vmo_batch_order) against one-at-a-time plain calls on the first
    `plain_sample` of them; both in nnz ordered per second."""
    mats = mats if mats is not None else W.batch_mix(count, seed=1)
    dev = [(torch.as_tensor(A.rowptr).cuda(), torch.as_tensor(A.colidx).cuda(), A.m) for A in mats]
    nnz = sum(A.nnz for A in mats)
    p = V.Params(d=3, seed=1)
    stream = torch.cuda.current_stream()
    for _ in range(max(warmup, 3)):
        V.batch_order(dev, p)
    t = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        V.batch_order(dev, p)
        b.record(stream)
        torch.cuda.synchronize()
        t += a.elapsed_time(b) / 1e3
    batched = nnz * steps / t
    sample = dev[:plain_sample]
    snnz = sum(A.nnz for A in mats[:plain_sample])
    for rp, ci, m in sample[:2]:
        V.Hypergraph(rp, ci, m, m).order_vertices(p)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for rp, ci, m in sample:
        V.Hypergraph(rp, ci, m, m).order_vertices(p)
    b.record(stream)
    torch.cuda.synchronize()
    plain = snnz / (a.elapsed_time(b) / 1e3)
    return {"workload": f"batch_mix x{count} (n log-uniform 200..20000, half 2D grids, half random symmetric "
                        f"3-30 nnz/row), d=3, min_part 64",
            "matrices": count, "rows": sum(A.m for A in mats), "nnz": nnz,
            "batched": {"value": batched, "unit": "nnz/s", "ms_per_batch": 1e3 * t / steps, "steps": steps},
            "plain_one_at_a_time": {"value": plain, "unit": "nnz/s", "sample_matrices": plain_sample,
                                    "sample_nnz": snnz},
            "batched_over_plain": batched / plain}


def step_roofline(V, torch, run_once, d: int, steps: int, peak: dict) -> dict:
    """Roofline of the layout step kernel over one workload: algorithmic flops
    per launch (interactions counted by the kernel in one untimed run, times
    FLOPS_PER_INTERACTION[d]) over the average launch time, measured with CUDA
    events around every step-kernel launch on its stream in `steps` further
    runs; against the measured FP32 peak of this GPU.  share_of_step: the
    kernel's event-timed share of those instrumented runs (per-launch events
    replace the graph replay there, so the runs are longer than plain ones)."""
    V.stats_reset(time_step_kernel=True, count_interactions=True)
    run_once()
    counted = V.stats()
    V.stats_reset(time_step_kernel=True, count_interactions=False)
    t0 = time.perf_counter()
    for _ in range(steps):
        run_once()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = V.stats()
    V.stats_reset(time_step_kernel=False, count_interactions=False)
    launches = max(counted["step_launches"], 1)
    flops_per_launch = counted["step_interactions"] * FLOPS_PER_INTERACTION[d] / launches
    avg_ms = st["step_ms"] / max(st["step_launches"], 1)
    achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": f"k_repulse_update<{d}> (layout step)", "achieved": achieved,
            "peak": peak["ffma2_tflops"], "unit": "TFLOP/s", "frac": achieved / peak["ffma2_tflops"],
            "peak_source": f"measured in this run (vmo_measure_alu_peaks): packed FP32 fma2 on all "
                           f"{peak['sms']} SMs, {peak['ffma2_tflops']:.1f} TFLOP/s (scalar fma "
                           f"{peak['ffma_tflops']:.1f}, rsqrt {peak['rsqrt_tops']:.2f} T/s)",
            "interactions_per_launch": counted["step_interactions"] / launches,
            "flops_per_interaction": FLOPS_PER_INTERACTION[d], "avg_launch_ms": avg_ms,
            "launches": st["step_launches"],
            "share_of_step": st["step_ms"] / 1e3 / wall,
            "timing": "CUDA events around every step-kernel launch on its stream"}


def owner_parts(k: int, perm: np.ndarray, tree: dict, sbd: bool) -> np.ndarray:
    """Final owner of every vertex: the index of its leaf record, or of the
    split node whose separator holds it (the parts of the cut metrics)."""
    part = np.full(k, -1, dtype=np.int32)
    off, n1, n2, ns = (tree[f].cpu().numpy() for f in ("offset", "n1", "n2", "nsep"))
    for i in range(len(off)):
        o, a, b, c = int(off[i]), int(n1[i]), int(n2[i]), int(ns[i])
        if b == 0 and c == 0:
            part[perm[o:o + a]] = i
        else:
            so = o + a if sbd else o + a + b
            part[perm[so:so + c]] = i
    return part


def config_leg(V, torch, name: str, A, model: str, d: int, sbd: bool, max_depth: int, min_part: int, steps: int,
               warmup: int, flush, peak: dict, cuts: bool = False) -> dict:
    """One configuration ordered plain (one matrix, device-resident CSR): build
    of the model + multilevel layout + recursive BBD/SBD per step, in nnz
    ordered per second, with its own step-kernel roofline; optionally the cut
    metrics of the final parts (cut-net and lambda - 1 over the row nets and
    the column nets)."""
    rp, ci = torch.as_tensor(A.rowptr).cuda(), torch.as_tensor(A.colidx).cuda()
    p = V.Params(d=d, max_depth=max_depth, min_part=min_part, seed=1)
    stream = torch.cuda.current_stream()

    def once(with_tree=False):
        hg = V.Hypergraph(rp, ci, A.m, A.n, model)
        out = hg.order_vertices(p, None, sbd=sbd) if with_tree else hg.order(p, None, sbd=sbd, with_tree=False)
        del hg
        return out

    for _ in range(max(warmup, 3)):
        once()
    t = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        once()
        b.record(stream)
        torch.cuda.synchronize()
        t += a.elapsed_time(b) / 1e3
    leg = {"workload": name, "m": A.m, "n": A.n, "nnz": int(A.nnz), "model": model, "d": d,
           "form": "SBD" if sbd else "BBD", "max_depth": max_depth, "min_part": min_part,
           "value": A.nnz * steps / t, "unit": "nnz/s", "ms_per_step": 1e3 * t / steps, "steps": steps,
           "roofline": step_roofline(V, torch, once, d, max(1, min(steps, 3)), peak)}
    if cuts:
        perm, tree = once(with_tree=True)
        part = owner_parts(A.m + A.n, perm.cpu().numpy(), tree, sbd)
        rows, cols = part[:A.m], part[A.m:]
        nparts = int(part.max()) + 1
        cn_r, l1_r = V.Hypergraph.from_matrix(A, "rownet").cut_size(torch.as_tensor(cols), nparts)
        cn_c, l1_c = V.Hypergraph.from_matrix(A, "colnet").cut_size(torch.as_tensor(rows), nparts)
        nsep = tree["nsep"].cpu().numpy()
        leg["cuts"] = {"parts": nparts, "leaves": int((nsep == 0).sum()), "sum_sep": int(nsep.sum()),
                       "max_sep": int(nsep.max()), "lambda_minus_1": l1_r + l1_c,
                       "lambda_minus_1_rownets": l1_r, "lambda_minus_1_colnets": l1_c, "cut_nets": cn_r + cn_c}
    return leg


def plain_over_requests(V, torch, reqs, count: int) -> dict:
    """The served mix one request at a time through the plain API (host CSR in,
    host permutation out, each call finished before the next), on the first
    `count` requests of the stream."""
    p = V.Params(d=3, seed=1)
    sample = reqs[:count]
    host = [(torch.as_tensor(A.rowptr).pin_memory(), torch.as_tensor(A.colidx).pin_memory(),
             torch.empty(A.m, dtype=torch.int32).pin_memory()) for A in sample]
    for (rp, ci, out), A in list(zip(host, sample))[:2]:
        V.Hypergraph(rp.cuda(), ci.cuda(), A.m, A.m).order(p, None, with_tree=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (rp, ci, out), A in zip(host, sample):
        hg = V.Hypergraph(rp.cuda(non_blocking=True), ci.cuda(non_blocking=True), A.m, A.m)
        perm, _, _ = hg.order(p, None, with_tree=False)
        out.copy_(perm)  # waits for the result, as a caller of the plain API would
        del hg
    dt = time.perf_counter() - t0
    nnz = sum(A.nnz for A in sample)
    return {"value": nnz / dt, "unit": "nnz/s", "requests": len(sample), "nnz": int(nnz),
            "large_requests": sum(1 for A in sample if A.m >= 1_000_000), "seconds": dt}


def max_over_ranks(seconds: float, world: int, device: str) -> float:
    """Largest elapsed time over the ranks (the job's time: every rank orders
    its own replica, so the job ends with the slowest)."""
    import torch
    if world <= 1:
        return float(seconds)
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, tmax: float) -> float:
    """Whole-job throughput of weak-scaled replicas: all ranks' units over the
    slowest rank's time."""
    return units_per_rank * world / tmax


def served_leg(V, rate: float, duration: float, large_every: int = 50, slots: int = 4, plain_sample: int = 0,
               torch=None):
    """Served mode: an open-loop Poisson stream of ordering requests (seeded),
    98% from the batch_mix size distribution and every `large_every`-th a
    27-point stencil on 100^3 (1,000,000 rows, 26,463,592 nnz), submitted from
    host memory to the request server (continuous batching, HBM-budget
    admission).  Reports offered and achieved nnz/s and latency percentiles
    from submission to the permutation in host memory."""
    import threading
    arrivals = W.poisson_arrivals(rate, duration, seed=5)
    nreq = len(arrivals)
    small = W.batch_mix(nreq, seed=5)
    large = W.stencil27(100)
    reqs = [large if (i % large_every == large_every - 1) else small[i] for i in range(nreq)]
    p = V.Params(d=3, seed=1)
    # warm the server path once (library, pool) outside the measured stream
    with V.Server(p, slots=slots) as srv:
        for A in small[:8]:
            srv.wait(srv.submit_matrix(A), 300.0)
    with V.Server(p, slots=slots) as srv:
        ids = [None] * nreq
        t0 = time.perf_counter()

        def producer():
            for i, A in enumerate(reqs):
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                ids[i] = srv.submit_matrix(A)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        infos = [srv.wait(r, 1800.0) for r in ids]
        st = srv.stats()
    done = [d for d in infos if d["state"] == "done"]
    lat = np.array([d["latency"] for d in done])
    lat_small = np.array([d["latency"] for d, A in zip(infos, reqs) if d["state"] == "done" and A is not large])
    lat_large = np.array([d["latency"] for d, A in zip(infos, reqs) if d["state"] == "done" and A is large])
    t_first = min(d["t_submit"] for d in infos)
    t_last = max(d["t_done"] for d in done)
    nnz_done = sum(d["nnz"] for d in done)
    nnz_all = sum(A.nnz for A in reqs)

    def pct(a, q):
        return float(np.percentile(a, q)) if len(a) else None

    plain = plain_over_requests(V, torch, reqs, plain_sample) if plain_sample > 0 else None
    return {"workload": f"Poisson arrivals {rate:g}/s for {duration:g} s (seed 5): batch_mix sizes, every "
                        f"{large_every}th request a 27-point stencil 100^3 (26.46M nnz); host CSR in, host "
                        f"permutation out; d=3, min_part 64",
            "requests": nreq, "large_requests": sum(1 for A in reqs if A is large), "completed": len(done),
            "offered_nnz_per_s": nnz_all / duration, "achieved_nnz_per_s": nnz_done / (t_last - t_first),
            "unit": "nnz/s", "p50_s": pct(lat, 50), "p99_s": pct(lat, 99), "p50_small_s": pct(lat_small, 50),
            "p99_small_s": pct(lat_small, 99), "p50_large_s": pct(lat_large, 50), "max_s": pct(lat, 100),
            "batches": st["batches"], "slots": slots, "budget_bytes": st["budget_bytes"],
            "peak_admitted_bytes": st["bytes_peak"], "pool_peak_bytes": st["pool_peak_bytes"],
            "drain_s": t_last - t_first,
            **({"plain_one_at_a_time": plain, "served_over_plain": (nnz_done / (t_last - t_first)) / plain["value"]}
               if plain else {})}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vmo", choices=["vmo", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=4096,
                    help="matrices of the batched leg (config-4 distribution; 0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=2000.0,
                    help="requests per second of the served leg (0 skips it)")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="length of the served arrival stream")
    ap.add_argument("--serve-plain", type=int, default=200,
                    help="requests of the served stream also ordered one at a time through the plain API")
    ap.add_argument("--no-config-legs", action="store_true",
                    help="skip the legs of the small 2D grid and the rectangular SBD workload")
    ap.add_argument("--serve-sweep", default="",
                    help="comma-separated request rates: run the served leg at each and report the highest rate "
                         "sustained (achieved >= 95%% of offered, p99 <= 2 s)")
    ap.add_argument("--autotune", type=int, default=0, metavar="N",
                    help="before the batched leg, tune the launch shapes (vmo_autotune) on the first N matrices "
                         "of the batch mix and report the setting and its times (the setting never changes a "
                         "result)")
    ap.add_argument("--profile", action="store_true",
                    help="one untimed step of the workload and exit (for ncu captures; no JSON line)")
    ap.add_argument("--profile-matrix", type=int, default=-1,
                    help="with --profile: order only this matrix of the workload (0 or 1)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="one untimed batched ordering of the first N matrices of the batch mix (after one "
                         "warm-up), for an ncu launch list of the batched path")
    ap.add_argument("--profile-small", action="store_true",
                    help="one untimed ordering of the 64x64 grid of the small workload (d=2, BBD to parts of <= 64 "
                         "rows, after one warm-up), for an ncu launch list of the small levels")
    ap.add_argument("--profile-large", type=int, default=0, metavar="SIDE",
                    help="a case larger than L2 for the memory-bound kernels (ncu captures, no JSON line): "
                         "SIDE^3 7-point grid, 4 layout steps from random coordinates at one level, then the "
                         "recursive BBD of the grid's own coordinates to depth 10")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        sample_name, mats = cpu_sample(small=True)
        import oracle
        oracle.build()
        th = oracle.threads()  # OpenMP threads of the oracle's per-vertex loops
        for _ in range(max(args.warmup, 0)):
            oracle_step(mats)
        t0 = time.perf_counter()
        nnz = 0
        for _ in range(args.steps):
            nnz += oracle_step(mats)
        dt = time.perf_counter() - t0
        val = nnz / dt
        print(json.dumps({"metric": METRIC, "value": val, "unit": "nnz/s", "impl": "reference", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": {"workload": MEDIUM_NAME, "model": "symmetric", "d": 3, "iters_per_level": 100,
                                     "max_depth": 10, "layout": "multilevel",
                                     "sample_per_step": f"{sample_name} (bounded sample of the workload)",
                                     "l2": "n/a (CPU)"},
                          "cpu_baseline": {"value": val, "unit": "nnz/s", "cores": th, "kind": "oracle",
                                           "sample": f"{sample_name} per step, oracle FP64 as built (OpenMP over "
                                                     f"the per-vertex gradient loop, {th} threads)",
                                           **host_cpu()},
                          "e2e": {"value": val, "unit": "nnz/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_1105_4490_gb300 as V
    V.load()

    if args.profile_batch:
        bm = W.batch_mix(4096, seed=1)[:args.profile_batch]
        dev = [(torch.as_tensor(A.rowptr).cuda(), torch.as_tensor(A.colidx).cuda(), A.m) for A in bm]
        for _ in range(2):
            V.batch_order(dev, V.Params(d=3, seed=1))
        torch.cuda.synchronize()
        print(f"profile-batch done: {len(bm)} matrices, {sum(A.nnz for A in bm)} nnz", file=sys.stderr)
        return

    if args.profile_small:
        A = W.grid_laplacian_2d(64)
        p = V.Params(d=2, max_depth=62, min_part=64, seed=1)
        for _ in range(2):
            V.Hypergraph.from_matrix(A).order(p, None, sbd=False, with_tree=False)
        torch.cuda.synchronize()
        print(f"profile-small done: 64x64 grid, {A.n} rows, {A.nnz} nnz", file=sys.stderr)
        return

    if args.profile_large:
        side = args.profile_large
        A = W.grid_laplacian_3d(side)
        hg = V.Hypergraph.from_matrix(A)
        p = V.Params(d=3, iters=4, seed=1)
        x0 = V.init_coords(A.n, 3, 1)
        hg.layout(p, x0.clone())
        ijk = torch.tensor(np.indices((side, side, side)).reshape(3, -1).T.astype(np.float32))
        xg = torch.zeros((A.n, 4), dtype=torch.float32)
        xg[:, :3] = ijk
        hg.order_vertices(V.Params(d=3, max_depth=10, seed=1), xg.cuda())
        torch.cuda.synchronize()
        print(f"profile-large done: {side}^3 grid, {A.n} rows, {A.nnz} nnz", file=sys.stderr)
        return

    name, mats = medium_workload()
    if args.profile and args.profile_matrix >= 0:
        mats = [mats[args.profile_matrix]]
    params = {"seed": 1}
    dev_csr = [(torch.as_tensor(A.rowptr).cuda(), torch.as_tensor(A.colidx).cuda()) for A, _ in mats]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    if args.profile:
        V.stats_reset(time_step_kernel=True, count_interactions=False)  # events only, no extra kernels
        gpu_step(V, torch, mats, dev_csr, params)
        torch.cuda.synchronize()
        st = V.stats()
        print(f"profile step done: {name} launches={st['launches']} step_launches={st['step_launches']}",
              file=sys.stderr)
        return

    for _ in range(max(args.warmup, 3)):
        gpu_step(V, torch, mats, dev_csr, params)

    # one untimed counting step: interactions and points of the step kernel
    V.stats_reset(time_step_kernel=True, count_interactions=True)
    gpu_step(V, torch, mats, dev_csr, params)
    counted = V.stats()
    V.stats_reset(time_step_kernel=False, count_interactions=False)

    def timed_steps():
        el, z = 0.0, 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            z += gpu_step(V, torch, mats, dev_csr, params)
            b.record(stream)
            barrier()
            el += a.elapsed_time(b) / 1e3
        return el, z

    # end to end through the public API: pinned host CSR -> permutations in
    # pinned host memory (one untimed warm-up pass, then K timed passes)
    host_csr = [(torch.as_tensor(A.rowptr).pin_memory(), torch.as_tensor(A.colidx).pin_memory()) for A, _ in mats]
    host_out = [(torch.empty(A.m, dtype=torch.int32).pin_memory(), torch.empty(A.n, dtype=torch.int32).pin_memory())
                for A, _ in mats]
    h2d = sum(r.numel() * 4 + c.numel() * 4 for r, c in host_csr)
    d2h = sum(r.numel() * 4 + c.numel() * 4 for r, c in host_out)

    def e2e_pass():
        for (A, cfg), (rp, ci), (ro, co) in zip(mats, host_csr, host_out):
            hg = V.Hypergraph(rp.cuda(non_blocking=True), ci.cuda(non_blocking=True), A.m, A.n, "symmetric")
            p = V.Params(d=cfg["d"], max_depth=cfg["max_depth"], seed=params["seed"])
            rperm, cperm, _ = hg.order(p, None, sbd=False, with_tree=False)
            ro.copy_(rperm, non_blocking=True)
            co.copy_(cperm, non_blocking=True)
            del hg

    def e2e_steps():
        el = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_pass()
            b.record(stream)
            barrier()
            el += a.elapsed_time(b) / 1e3
        return el

    e2e_pass()  # untimed warm-up of the host buffers and the pinned copies
    barrier()
    with ClockSampler(local) as clocks:
        # timed region: plain library calls (the layout steps of a level replay
        # a CUDA graph)
        V.stats_reset(time_step_kernel=False, count_interactions=False)
        elapsed, nnz = timed_steps()
        st_timed = V.stats()
        # the same K steps end to end (host buffers in and out), plain calls
        e2e_time = e2e_steps()
        # the same K steps again with CUDA events around every step-kernel
        # launch, for the kernel's roofline (per-launch events turn graph
        # replay off, so these steps are not part of `value`)
        V.stats_reset(time_step_kernel=True, count_interactions=False)
        elapsed_ev, _ = timed_steps()
        st = V.stats()
        V.stats_reset(time_step_kernel=False, count_interactions=False)  # plain library calls from here on
    tmax = max_over_ranks(elapsed, world, "cuda")
    value = replica_throughput(nnz, world, tmax)
    e2e_value = nnz * world / max_over_ranks(e2e_time, world, "cuda")

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    csum = clocks.summary()
    peak = V.vmo.measure_alu_peaks()  # this GPU's measured FP32 rates (a few ms; after the timed region)
    d = 3
    inter_per_step = counted["step_interactions"]
    launches_per_step = max(counted["step_launches"], 1)
    flops_per_launch = inter_per_step * FLOPS_PER_INTERACTION[d] / launches_per_step
    avg_ms = st["step_ms"] / max(st["step_launches"], 1)
    achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_repulse_update<3> (layout step)", "achieved": achieved,
                "peak": peak["ffma2_tflops"], "unit": "TFLOP/s", "frac": achieved / peak["ffma2_tflops"],
                "traffic": None,
                "traffic_note": "the per-launch mean over a step's 3,000 launches is not captured for the "
                                "current kernel (ncu captures are kept to single launches); one finest-level "
                                "launch of the 500k power-law read 31.9 MB from DRAM",
                "peak_source": f"measured in this run (vmo_measure_alu_peaks): packed FP32 fma2 on all "
                               f"{peak['sms']} SMs, {peak['ffma2_tflops']:.1f} TFLOP/s (scalar fma "
                               f"{peak['ffma_tflops']:.1f}, rsqrt {peak['rsqrt_tops']:.2f} T/s); nominal "
                               f"{peak['sms']} x 128 lanes x 2 x 2070 MHz = {peak['sms'] * 256 * 2.07e-3:.1f}",
                "interactions_per_launch": inter_per_step / launches_per_step,
                "flops_per_interaction": FLOPS_PER_INTERACTION[d],
                "avg_launch_ms": avg_ms, "launches": st["step_launches"],
                "share_of_step": st["step_ms"] / 1e3 / elapsed_ev,
                "timing": "CUDA events around every step-kernel launch on its stream, over K instrumented steps of "
                          "the same workload run right after the timed region"}

    modes = {}
    if args.autotune > 0 and world == 1:
        sample = W.batch_mix(args.batch_count or 4096, seed=1)[:args.autotune]
        dev = [(torch.as_tensor(A.rowptr).cuda(), torch.as_tensor(A.colidx).cuda(), A.m) for A in sample]
        best, best_ms, default_ms = V.autotune(dev, V.Params(d=3, seed=1), reps=3)
        modes["autotune"] = {"sample": f"first {args.autotune} matrices of the batch mix, vmo_batch_order, median of 3",
                             "setting": best, "best_ms": best_ms, "default_ms": default_ms}
    if args.batch_count > 0:
        bmats = W.batch_mix(args.batch_count, seed=1)
        modes["batched"] = batched_leg(V, torch, args.batch_count, 32, args.warmup, max(min(args.steps, 3), 1),
                                       flush, bmats)
    if not args.no_config_legs and world == 1:
        modes["config_grid2d_64"] = config_leg(
            V, torch, "2D 5-point Laplacian 64x64 (n 4,096), symmetric model, d=2, BBD to parts of <= 64 rows",
            W.grid_laplacian_2d(64), "symmetric", 2, False, 62, 64, max(args.steps, 5), args.warmup, flush, peak)
        modes["config_sbd_400k"] = config_leg(
            V, torch, "400,000 x 300,000 power-law (column degrees ~d^-2.5, mean ~16), bipartite model, d=2, "
                      "SBD to depth 6 (64 parts)",
            W.powerlaw_rectangular(400_000, 300_000, seed=1), "bipartite", 2, True, 6, 1, args.steps, args.warmup,
            flush, peak, cuts=True)
    if args.serve_rate > 0 and world == 1:
        modes["served"] = served_leg(V, args.serve_rate, args.serve_seconds, plain_sample=args.serve_plain,
                                     torch=torch)
    if args.serve_sweep and world == 1:
        sweep = []
        for rate in [float(r) for r in args.serve_sweep.split(",") if r]:
            leg = served_leg(V, rate, args.serve_seconds)
            leg["rate"] = rate
            leg["sustained"] = (leg["achieved_nnz_per_s"] >= 0.95 * leg["offered_nnz_per_s"] and
                                leg["p99_s"] is not None and leg["p99_s"] <= 2.0)
            sweep.append({k: leg[k] for k in ("rate", "offered_nnz_per_s", "achieved_nnz_per_s", "p50_s", "p99_s",
                                              "sustained")})
        ok = [r["rate"] for r in sweep if r["sustained"]]
        modes["served_sweep"] = {"rates": sweep, "max_sustained_rate": max(ok) if ok else None}

    if world == 1:
        # m-way k-means++ (Algorithm 5, 64 centres) of a million points, one call
        kpts = V.init_coords(1_000_000, 3, seed=3)
        kverts = torch.arange(1_000_000, dtype=torch.int32, device="cuda")
        V.kmeans(kpts, kverts, 64, seed=1, km_iters=20, d=3)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, _, ne = V.kmeans(kpts, kverts, 64, seed=1, km_iters=20, d=3)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        modes["kmeans_m64"] = {"workload": "1,000,000 points of a seeded uniform layout in d = 3, m = 64 centres, "
                                           "k-means++ seeding + at most 20 Lloyd rounds",
                               "ms_per_call": statistics.median(ts), "points_per_s": 1e6 / (statistics.median(ts) / 1e3),
                               "nonempty": ne}

    # phase split of one untimed step (build, layout = V, ordering = O)
    breakdown = {"build_ms": 0.0, "layout_ms": 0.0, "order_ms": 0.0}
    for (A, cfg), (rp, ci) in zip(mats, dev_csr):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        hg = V.Hypergraph(rp, ci, A.m, A.n, "symmetric")
        ev[1].record(stream)
        p = V.Params(d=cfg["d"], max_depth=cfg["max_depth"], seed=params["seed"])
        x = hg.layout(p)
        ev[2].record(stream)
        hg.order_vertices(p, x)
        ev[3].record(stream)
        torch.cuda.synchronize()
        breakdown["build_ms"] += ev[0].elapsed_time(ev[1])
        breakdown["layout_ms"] += ev[1].elapsed_time(ev[2])
        breakdown["order_ms"] += ev[2].elapsed_time(ev[3])
        del hg

    # the host-only oracle baselines last, after every GPU leg, so that their
    # processes and threads never share the host with a timed GPU leg
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        if "batched" in modes:
            modes["batched"]["cpu_oracle_all_cores"] = batch_cpu_all_cores(bmats, count=128)
            if "served" in modes:  # the served requests other than the 27-point ones follow the batch mix
                modes["served"]["cpu_oracle_all_cores"] = dict(
                    modes["batched"]["cpu_oracle_all_cores"],
                    note="the batched leg's subsample: the served stream's sizes other than its 27-point 100^3 "
                         "requests follow the batch mix; those are beyond the oracle's reach in a bounded run")
        sname, smats = cpu_sample(small=False)
        cpu = run_cpu_baseline(smats, sname)
        cpu.update(host_cpu())

    out = {"metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded generators; SuiteSparse matrices are not available)",
           "config": {"workload": name, "nnz_per_step": nnz // args.steps, "model": "symmetric", "d": 3,
                      "iters_per_level": 100, "max_depth": 10, "layout": "multilevel",
                      "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{world}"},
           "gpu_launches": st_timed["launches"], "clocks": csum, "roofline": roofline, "cpu_baseline": cpu,
           "modes": modes, "breakdown": breakdown,
           "e2e": {"value": e2e_value, "unit": "nnz/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
