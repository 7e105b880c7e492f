"""Benchmark of the APIC augury contact step (arXiv 2108.02259) on GB300.

One "step" is one full contact step through the C ABI: keys, sort, sparse
grid activation, mass P2G, then N + 1 fused transfer passes (the paper's
series with the Coulomb projection), on synthetic scenes resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line.  The metric is contact particle-iterations per second,
P * (N + 1) per step (each particle through each transfer pair).

Workloads (seeded, synthetic, shaped like the paper's bodies):
  eight_bodies  8 bodies, 4,000,000 nodes, h = 1/512, per-pair mu, N = 8, FP32
                (default).  The default line also carries the metric's other
                parts: "batched64" (the batched scenes below against the same
                scenes stepped one call each) and "served" (the serving loop
                below with 3 s per offered load: throughput, p50/p99 latency)
  four_bodies   4 bodies, 200,000 FE nodes, h = 1/256, mu = 0.3, N = 8, FP32
  two_cubes     2 cubes of 8^3 nodes, h = 1/32, mu = 0.3, N = 10, FP64
  batched64     64 independent scenes, 1k-200k nodes and 2-6 bodies each, h in
                {1/64, 1/128, 1/256}, mu = 0.3, N = 8, FP32, one batched call per
                step; also reports the same scenes stepped one call each
  served        256 resident simulations (2k-1M nodes each, 2-8 bodies, mu in
                [0, 0.5], N = 8) behind the serving loop; Poisson step requests
                at 0.5 / 0.8 / 0.95 of the measured batched capacity; reports
                throughput and p50/p99 request latency (value: load 0.8); one GPU
                (under torchrun only rank 0 runs it)

The CPU baseline (and the reference arm, --impl reference) is the FP64
oracle as it stands, on the host cores: one thread per independent bounded
sample of the workload, as many threads as cores (up to 16).

Multi-GPU (torchrun): every rank steps its own scene(s) of the workload's shape
and size, drawn from seed + 1000 * rank (independent problems: no collective
on the data path, only a barrier and a max-reduction of the time); value =
all ranks' particle-iterations / the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contact particle-iters/s"
UNIT = "particle-iters/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


RANK_SEED_STRIDE = 1000  # rank r draws its scenes from the workload's seed + 1000 r


def make_scene(name, rank=0):
    from paper_2108_02259_gb300 import scenes

    off = RANK_SEED_STRIDE * rank
    if name == "four_bodies":
        return scenes.four_bodies(seed=scenes.SEED_BASE + 2 + off), np.float32
    if name == "two_cubes":  # no random draw: every rank steps the same two cubes
        return scenes.two_cubes(mu=0.3, n_iter=10), np.float64
    if name == "eight_bodies":
        return scenes.eight_bodies(seed=scenes.SEED_BASE + 3 + off), np.float32
    raise SystemExit(f"unknown workload {name}")


def make_workload(name, rank=0):
    """(list of scenes, dtype, batched) of one rank.  Ranks step independent
    scenes of the same shape and size (seeds differ), so per-rank work is
    fixed as ranks are added (weak scaling) and no data crosses ranks."""
    from paper_2108_02259_gb300 import scenes

    if name == "batched64":
        return scenes.batch_of_scenes(64, seed=scenes.SEED_BASE + 4 + RANK_SEED_STRIDE * rank), np.float32, True
    s, dt = make_scene(name, rank)
    return [s], dt, False


def max_over_ranks(x: float, ws: int, device="cpu") -> float:
    """The largest x over all ranks (the slowest rank's time); x itself at
    one rank.  `device` is where the process group's backend reduces (a
    CUDA device for NCCL, the CPU for gloo)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(name, sc, dt):
    if len(sc) > 1:
        P = sum(s.n for s in sc)
        return {"workload": f"{name}: {len(sc)} independent scenes, {P} FE nodes in total "
                            f"({min(s.n for s in sc)}-{max(s.n for s in sc)} per scene, "
                            f"{min(s.n_bodies for s in sc)}-{max(s.n_bodies for s in sc)} bodies), "
                            f"h in {{1/64, 1/128, 1/256}}, N={sc[0].n_iter}, mu={sc[0].mu}, one batched call per step",
                "particles": P, "scenes": len(sc), "n_iter": sc[0].n_iter,
                "transfer_pairs_per_step": sc[0].n_iter + 1,
                "precision": "fp32 (fp64 node momentum at multi-body nodes)",
                "l2": "flushed before every timed step (256 MiB write)"}
    s = sc[0]
    return {
        "workload": f"{name}: {s.n_bodies} bodies, {s.n} FE nodes, h=1/{round(1 / s.h)}, N={s.n_iter}, "
                    + ("mu per body pair" if s.mu_pair is not None else f"mu={s.mu}"),
        "particles": s.n,
        "bodies": s.n_bodies,
        "h": s.h,
        "n_iter": s.n_iter,
        "transfer_pairs_per_step": s.n_iter + 1,
        "precision": "fp64" if dt == np.float64 else "fp32 (fp64 node momentum at multi-body nodes)",
        "l2": "flushed before every timed step (256 MiB write)",
    }


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def algorithmic_bytes_per_pass(P, G):
    """Bytes one fused transfer pass must move: per particle read the offset
    and mass (16 B), normal (12 B) and cell tag (4 B), read and write the
    12-float change Delta (96 B) = 128 B; per active node read v_i and
    accumulate p_i (24 B)."""
    return 128.0 * P + 24.0 * G


# Essential FP32 work of one fused pass per particle, an FMA counted as 2:
# G2P sum-factorised (x stage 64 nodes x 6 FMA, y-z stage 16 x 12) 1,152;
# P2G (64 nodes x 3 components x 2 FMA, plus 16 row factors) 1,104; weights,
# Delta update and two projections ~140.
FLOP_PER_PARTICLE_PASS = 2400.0
# GB300 FP32 peak: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz (maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Shared-memory peak: one 128-byte wavefront per SM per clock.
SMEM_PEAK_GWAVEFRONTS = 152 * 2.07


SAMPLE_PARTICLES = 60_000  # one oracle sample: about half a second of single-threaded FP64 work per step


def _sub_scene(s, keep):
    """The particles `keep` of scene s, body ids renumbered 0.. over the
    bodies present (with the matching block of a per-pair friction table)."""
    from paper_2108_02259_gb300 import scenes

    present = np.unique(s.body[keep])
    remap = np.full(s.n_bodies, -1, np.int32)
    remap[present] = np.arange(len(present), dtype=np.int32)
    mp = None if s.mu_pair is None else s.mu_pair[np.ix_(present, present)].copy()
    return scenes.Scene(s.x[keep], s.v[keep], s.C[keep], s.m[keep], s.nrm[keep], remap[s.body[keep]], len(present),
                        s.h, s.mu, s.n_iter, mp)


def oracle_samples(sc, max_samples=16):
    """Independent bounded samples of a workload for the oracle, each about
    SAMPLE_PARTICLES particles, with the contact the workload has:
      - a batch: its first scenes (whole), up to max_samples;
      - one small scene: the whole scene (each thread steps its own copy);
      - one large scene (the 4 M-node scene): per approaching pair of bodies
        (2k, 2k+1), the particles nearest the pair's contact plane x = 0.5,
        split into slabs along y, so that each sample holds both bodies
        where they meet."""
    if len(sc) > 1:
        out = [s for s in sc if s.n <= 4 * SAMPLE_PARTICLES][:max_samples]
        P = sum(s.n for s in out)
        return out, f"{len(out)} whole scenes of the batch ({P} particles)"
    s = sc[0]
    if s.n <= 4 * SAMPLE_PARTICLES:
        return [s], f"the whole scene ({s.n} particles)"
    pairs = s.n_bodies // 2
    per_pair = max(1, max_samples // max(pairs, 1))
    out = []
    for k in range(pairs):
        inp = (s.body == 2 * k) | (s.body == 2 * k + 1)
        idx = np.nonzero(inp)[0]
        d = np.abs(s.x[idx, 0] - 0.5)
        near = idx[np.argsort(d, kind="stable")[:per_pair * SAMPLE_PARTICLES]]
        ys = s.x[near, 1]
        cuts = np.quantile(ys, np.linspace(0, 1, per_pair + 1))
        for j in range(per_pair):
            lo, hi = cuts[j], cuts[j + 1]
            sel = near[(ys >= lo) & ((ys < hi) if j + 1 < per_pair else (ys <= hi))]
            keep = np.zeros(s.n, bool)
            keep[sel] = True
            out.append(_sub_scene(s, keep))
    P = sum(x.n for x in out)
    return out, (f"{len(out)} slabs of ~{SAMPLE_PARTICLES} particles across the contact planes of the scene's "
                 f"{pairs} approaching pairs ({P} of {s.n} particles)")


def run_oracle_steps(samples):
    """One oracle contact step of each sample, one host thread per sample
    (the oracle holds no global state, and ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    def one(s):
        oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                            mu_pair=s.mu_pair)
        return s.n * (s.n_iter + 1)

    if len(samples) == 1:
        return one(samples[0])
    with ThreadPoolExecutor(len(samples)) as ex:
        return sum(ex.map(one, samples))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(sc, budget_s=8.0):
    """The FP64 oracle as it stands, on the machine's host cores: one thread per
    independent sample, as many threads as cores (and samples), plus the
    same oracle on one thread for reference."""
    import oracle

    oracle.build()
    samples, what = oracle_samples(sc)
    cores = host_cores()
    threads = max(1, min(cores, 16))
    par = [samples[i % len(samples)] for i in range(threads)]

    def rate(batch):
        t0 = time.perf_counter()
        steps = units = 0
        while True:
            units += run_oracle_steps(batch)
            steps += 1
            el = time.perf_counter() - t0
            if el > budget_s or steps >= 8:
                return units / el, steps, el

    one_v, one_steps, one_el = rate(samples[:1])
    all_v, all_steps, all_el = rate(par)
    return {"value": all_v, "unit": UNIT, "cores": threads, "nproc": cores, "kind": "oracle",
            "sample": f"{all_steps} step(s) of {threads} independent samples in parallel threads "
                      f"(from {what}), N={samples[0].n_iter}, {all_el:.1f} s, FP64",
            "single_thread": {"value": one_v, "unit": UNIT, "cores": 1,
                              "sample": f"{one_steps} step(s) of the first sample ({samples[0].n} particles), "
                                        f"{one_el:.1f} s"}}


def run_reference(args):
    """The reference arm: the oracle (the only other implementation of the
    method) on the host cores, each step one oracle step of every bounded
    sample of the workload, one thread per sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    sc, dt, _ = make_workload(args.workload)
    samples, what = oracle_samples(sc)
    cores = host_cores()
    threads = max(1, min(cores, 16))
    par = [samples[i % len(samples)] for i in range(threads)]
    for _ in range(args.warmup):
        run_oracle_steps(par)
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units += run_oracle_steps(par)
    el = time.perf_counter() - t0
    value = units / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args.workload, sc, dt),
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads, "nproc": cores,
                         "sample": f"each step: {threads} independent samples in parallel threads (from {what}), "
                                   "FP64 oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200; 20 for --impl reference, whose steps are host-bound)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="eight_bodies",
                    choices=["four_bodies", "two_cubes", "eight_bodies", "batched64", "served"])
    ap.add_argument("--served-workers", type=int, default=2, help="served workload: server worker threads")
    ap.add_argument("--served-batch", type=int, default=64, help="served workload: most requests per batch")
    ap.add_argument("--served-seconds", type=float, default=6.0,
                    help="open-loop seconds per offered load (the served workload; 3 s in the default line's leg)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variant", type=int, default=-1,
                    help="fix the transfer-kernel variant (default: autotune for the workload)")
    ap.add_argument("--no-graphs", action="store_true", help="launch the transfer passes one by one")
    ap.add_argument("--deterministic", action="store_true",
                    help="APIC_DETERMINISTIC: bitwise-reproducible steps (fixed-point node sums, variant 0)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="launch each pass strictly after the grid before it (no programmatic dependent launch)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip every measurement beside the workload's own (normals, augury, batched and served legs)")
    args = ap.parse_args()
    if args.steps is None:
        # about a second of timed device work on the 4M-node scene, so that the
        # clock samples taken during it are several
        args.steps = 20 if args.impl == "reference" else 200
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "served":
        return run_served(args)

    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}" if ws > 1 else "cuda:0")
    torch.cuda.set_device(dev)

    from paper_2108_02259_gb300 import apic, build

    # one rank compiles (if anything is stale); the others wait for it
    if rank == 0:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = apic.Context(dev.index)
    sc, dt, batched = make_workload(args.workload, rank)
    m = measure(args, apic, ctx, sc, dt, batched, dev, stream, flush, ws, with_e2e=not args.no_e2e,
                with_clocks=True)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if dt == np.float64 else "f32", "data": "synthetic",
        "config": workload_config(args.workload, sc, dt),
    }
    line.update({k: m[k] for k in ("e2e", "gpu_launches", "kernel_variant", "cuda_graph", "dependent_launch",
                                   "deterministic", "sort_primitive_calls_per_step", "roofline", "roofline_fp32",
                                   "roofline_smem", "step_breakdown_ms", "momentum_check", "clocks")})
    if "plain_single_scene" in m:
        line["plain_single_scene"] = m["plain_single_scene"]
    if not args.no_extras:
        line["node_normals"] = bench_node_normals(apic, ctx, dev, stream, flush)
        line["augury_dynamics"] = bench_augury(apic, ctx, dev, stream)
    if not args.no_extras and args.workload == "eight_bodies" and ws == 1:
        # the metric's other two parts on the same line: batched scenes
        # against the plain single-scene path, and the served loop's p50/p99
        b_sc, b_dt, _ = make_workload("batched64", rank)
        b = measure(args, apic, ctx, b_sc, b_dt, True, dev, stream, flush, ws, with_e2e=not args.no_e2e,
                    with_clocks=False)
        line["batched64"] = {
            "what": "64 independent scenes in one batched call per step, against the same scenes "
                    "one apic_contact_step call each (plain single-scene path)",
            "config": workload_config("batched64", b_sc, b_dt), "value": b["value"], "unit": UNIT,
            "ms_per_step": b["ms_per_step"], "kernel_variant": b["kernel_variant"], "e2e": b["e2e"],
            "plain_single_scene": b["plain_single_scene"], "roofline": b["roofline"],
            "gpu_launches": b["gpu_launches"], "momentum_check": b["momentum_check"]}
        line["partitioned2"] = partitioned_measure(args, apic, ctx, sc[0], dev, stream, flush, m["ms_per_step"])
        ctx.close()
        ctx = None
        line["served"] = served_measure(args, seconds=3.0, squeezed=False)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc)
    print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def partitioned_measure(args, apic, ctx, s, dev, stream, flush, whole_ms):
    """The scene as two partitions (halves along x) in one APIC_PARTITIONED
    batched call: each keeps its own grid and the blocks both reach are
    summed across them after every particle-to-grid transfer, the exchange a
    split of one scene over two devices needs (here both on one GPU).  Times
    the step like the main leg and checks the outputs against one call on
    the whole scene."""
    import torch

    f = s.astype(np.float32)
    xm = float(np.median(s.x[:, 0]))
    parts = [np.flatnonzero(s.x[:, 0] < xm), np.flatnonzero(s.x[:, 0] >= xm)]

    def t(a, d):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=d).to(dev)

    batch = [apic.BatchScene(t(f.x[ix], torch.float64), t(f.v[ix], torch.float32), t(f.C[ix], torch.float32),
                             t(f.m[ix], torch.float32), t(f.nrm[ix], torch.float32), t(f.body[ix], torch.int32),
                             s.h, s.mu, n_bodies=s.n_bodies, mu_pair=s.mu_pair) for ix in parts]
    N = s.n_iter
    for _ in range(max(args.warmup, 3)):
        apic.contact_step_batched(ctx, batch, N, stream=stream, flags=apic.APIC_PARTITIONED)
    torch.cuda.synchronize(dev)
    steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.fill_(1.0)
        a.record(stream)
        apic.contact_step_batched(ctx, batch, N, stream=stream, flags=apic.APIC_PARTITIONED)
        b.record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    whole = apic.contact_step(ctx, t(f.x, torch.float64), t(f.v, torch.float32), t(f.C, torch.float32),
                              t(f.m, torch.float32), t(f.nrm, torch.float32), t(f.body, torch.int32), s.h, s.mu, N,
                              n_bodies=s.n_bodies, mu_pair=s.mu_pair, stream=stream)
    torch.cuda.synchronize(dev)
    v = np.zeros((s.n, 3), np.float32)
    for ix, b in zip(parts, batch):
        v[ix] = b.v_out.cpu().numpy().reshape(-1, 3)
    dv = float(np.abs(v - whole.v.cpu().numpy()).max() / np.abs(s.v).max())
    return {"what": "the same scene as two partitions (halves along x), each with its own grid, summed where "
                    "they share grid blocks after every particle-to-grid transfer (APIC_PARTITIONED)",
            "partitions": [int(len(ix)) for ix in parts], "value": s.n * (N + 1) / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms, "vs_whole_scene_step": ms / whole_ms,
            "max_dv_vs_whole_scene": dv, "l2": "flushed before every timed step"}


def measure(args, apic, ctx, sc, dt, batched, dev, stream, flush, ws, with_e2e=True, with_clocks=True):
    """Time K contact steps of one workload (device buffers, L2 flushed
    before each step), then the per-pass roofline from an untimed profiling
    run, the plain path for a batch, and the end-to-end host-buffer figure."""
    import torch

    tdt = torch.float32 if dt == np.float32 else torch.float64
    N = sc[0].n_iter
    P = sum(s.n for s in sc)

    def t(a, d):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=d).to(dev)

    bs = []
    for s in sc:
        f = s.astype(dt)
        bs.append(apic.BatchScene(t(f.x, torch.float64), t(f.v, tdt), t(f.C, tdt), t(f.m, tdt), t(f.nrm, tdt),
                                  t(f.body, torch.int32), s.h, s.mu, n_bodies=s.n_bodies, mu_pair=s.mu_pair))
    FL = apic.APIC_DETERMINISTIC if args.deterministic else 0

    def step_one(b):
        apic.contact_step(ctx, b.x, b.v, b.C, b.m, b.nrm, b.body, b.h, b.mu, N, n_bodies=b.n_bodies,
                          mu_pair=b.mu_pair, v_out=b.v_out, C_out=b.C_out, stream=stream, flags=FL)

    def step():
        if batched:
            apic.contact_step_batched(ctx, bs, N, stream=stream, flags=FL)
        else:
            step_one(bs[0])

    # pick the transfer-kernel variant for this size class (untimed), then
    # one checked step: the device's own momentum balance
    ctx.set_overlap(not args.no_overlap)
    if args.deterministic:
        variant = 0  # the mode runs the first variant, untuned
    elif args.variant >= 0:
        ctx.set_variant(args.variant)
        variant = args.variant
    else:
        variant = ctx.autotune(bs, N, stream=stream)
    ctx.set_graphs(not args.no_graphs)
    st = apic.contact_step_batched(ctx, bs, N, stream=stream, stats=True, flags=FL)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    def timed(fn, steps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            fn()
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends))

    clocks = None
    if with_clocks:
        try:  # nvidia-smi wants the physical GPU: address it by UUID
            clocks = Clocks("GPU-" + str(torch.cuda.get_device_properties(dev).uuid))
        except Exception:
            clocks = Clocks(dev.index)
    ctx.set_profiling(False)  # resets the launch counter; passes replay as a graph
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
    t_ms = timed(step, args.steps)
    if ws > 1:
        torch.distributed.barrier()
    ck = clocks.stop() if clocks else None
    launches = ctx.profile()["kernel_launches"]
    # per-pass kernel times for the roofline: a separate, untimed run with
    # an event pair around every pass (launched one by one)
    ctx.set_profiling(True)
    timed(step, max(2, min(args.steps, 5)))
    prof = ctx.profile()
    ctx.set_profiling(False)
    t_ms = max_over_ranks(t_ms, ws, dev)
    units = P * (N + 1) * args.steps * ws
    value = units / (t_ms / 1e3)
    out = {"value": value, "ms_per_step": t_ms / args.steps}

    # the same scenes one call each (the plain single-scene path)
    if batched:
        for b in bs:
            step_one(b)
        torch.cuda.synchronize(dev)
        k = max(2, args.steps // 4)
        t_plain = timed(lambda: [step_one(b) for b in bs], k)
        plain = P * (N + 1) * k / (t_plain / 1e3)
        out["plain_single_scene"] = {"value": plain, "unit": UNIT, "ms_per_step": t_plain / k,
                                     "what": "the same scenes, one apic_contact_step call each",
                                     "batched_over_plain": value / plain}

    # roofline of the fused transfer kernel (timed live with events on the launch stream)
    G = prof["active_nodes"]
    iter_avg_ms = prof["iter_ms"] / max(prof["iter_launches"], 1)
    alg = algorithmic_bytes_per_pass(P, G)
    peak, peak_kind = measured_peak_hbm()
    achieved = alg / (iter_avg_ms / 1e3) / 1e9
    traffic = wavefronts = None
    wl = args.workload if not batched or args.workload == "batched64" else "batched64"
    tfile = os.path.join(ROOT, "profiles", f"traffic_{wl}.json")
    if os.path.exists(tfile):
        try:
            tj = json.load(open(tfile))
            if tj.get("kernel_source_hash") == kernel_source_hash() and not args.deterministic:
                traffic = tj.get("dram_bytes_per_launch")
                wavefronts = tj.get("shared_wavefronts_per_launch")
        except Exception:
            traffic = wavefronts = None

    # end to end: the same step through the C ABI from pinned host buffers
    e2e = None
    if with_e2e:
        def pin(a, d):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=d).pin_memory().numpy()

        hs = []
        for s in sc:
            f = s.astype(dt)
            hs.append(apic.BatchScene(pin(f.x, torch.float64), pin(f.v, tdt), pin(f.C, tdt), pin(f.m, tdt),
                                      pin(f.nrm, tdt), pin(f.body, torch.int32), s.h, s.mu, n_bodies=s.n_bodies,
                                      mu_pair=s.mu_pair, v_out=pin(np.zeros_like(f.v), tdt),
                                      C_out=pin(np.zeros_like(f.C), tdt)))

        def host_step():
            if batched:
                apic.contact_step_batched(ctx, hs, N, stream=stream, flags=FL)
            else:
                h = hs[0]
                apic.contact_step(ctx, h.x, h.v, h.C, h.m, h.nrm, h.body, h.h, h.mu, N, n_bodies=h.n_bodies,
                                  mu_pair=h.mu_pair, v_out=h.v_out, C_out=h.C_out, stream=stream, flags=FL)

        for _ in range(2):
            host_step()
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        el = max_over_ranks(el, ws, dev)
        isz = np.dtype(dt).itemsize
        e2e = {"value": units / el, "unit": UNIT,
               "h2d_bytes_per_step": int(P * (24 + 4 + isz * (3 + 9 + 1 + 3))),
               "d2h_bytes_per_step": int(P * isz * (3 + 9))}

    sP = float(sum(np.sum(s.m * np.linalg.norm(s.v, axis=1)) for s in sc))
    drift = float(sum(np.abs(x["P_out"] - x["P_in"]).max() for x in st)) / sP
    out.update({
        "e2e": e2e,
        "gpu_launches": int(launches),
        "kernel_variant": apic.variants()[variant],
        "cuda_graph": not args.no_graphs,
        "dependent_launch": not args.no_overlap,
        "deterministic": bool(args.deterministic),
        "sort_primitive_calls_per_step": prof["sort_launches"] / max(prof["steps"], 1),
        "roofline": {"bound": "hbm", "kernel": "k_items (fused G2P + projection + P2G pass)",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg, "avg_launch_ms": iter_avg_ms,
                     "launches": int(prof["iter_launches"]), "active_nodes": int(G)},
        "roofline_fp32": {"bound": "alu", "kernel": "k_items (fused G2P + projection + P2G pass)",
                          "achieved": FLOP_PER_PARTICLE_PASS * P / (iter_avg_ms / 1e3) / 1e12,
                          "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": FLOP_PER_PARTICLE_PASS * P / (iter_avg_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                          "flop_per_particle_pass": FLOP_PER_PARTICLE_PASS,
                          "peak_from": "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"},
        # the unit that binds: shared-memory wavefronts of one launch (ncu,
        # same kernel source) over its live duration
        "roofline_smem": None if wavefronts is None else {
            "bound": "shared", "kernel": "k_items (fused G2P + projection + P2G pass)",
            "achieved": wavefronts / (iter_avg_ms / 1e3) / 1e9, "peak": SMEM_PEAK_GWAVEFRONTS,
            "unit": "G wavefronts/s", "frac": wavefronts / (iter_avg_ms / 1e3) / 1e9 / SMEM_PEAK_GWAVEFRONTS,
            "wavefronts_per_launch": wavefronts, "peak_from": "152 SMs x 1 wavefront/clock x 2.07 GHz",
            "wavefronts_from": f"profiles/traffic_{wl}.json (ncu)"},
        "step_breakdown_ms": step_breakdown(prof),
        "momentum_check": {"P_drift_rel": drift,
                           "multibody_nodes": int(sum(x["multibody_nodes"] for x in st)),
                           "active_blocks": int(sum(x["active_blocks"] for x in st)),
                           "work_items": int(sum(x["work_items"] for x in st)),
                           # generalised kinetic energy, outputs over inputs (contact dissipates)
                           "E_change_rel": float(sum(x["E_out"] - x["E_in"] for x in st)
                                                 / max(sum(x["E_in"] for x in st), 1e-300))},
        "clocks": ck,
    })
    return out


def run_served(args):
    """The served workload as the bench line itself (value: throughput at
    offered load 0.8)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0  # one server on one GPU: under torchrun the other ranks have nothing to do
    sv = served_measure(args, seconds=args.served_seconds, squeezed=True)
    mid = sv["loads"]["0.8"]
    line = {
        "metric": METRIC, "value": mid["throughput"], "unit": UNIT, "n_gpus": 1, "steps": mid["requests"],
        "warmup": args.warmup, "ms_per_step": mid["mean_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": sv.pop("config"),
        "served": sv,
        "e2e": {"value": mid["throughput"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "state is resident on the device; latency is submit to completion"},
        "roofline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def served_measure(args, seconds=6.0, squeezed=True):
    """Serving: 256 resident simulations behind the serving loop.  Capacity
    in a closed loop, then open-loop Poisson step requests at 0.5 / 0.8 /
    0.95 of that capacity (`seconds` each), throughput and p50/p99 request
    latency; optionally the same simulations against a budget of about half
    their resident state, to exercise admission."""
    import torch  # noqa: F401

    from paper_2108_02259_gb300 import apic, build, scenes

    build.build()
    sims = scenes.served_simulations()
    workers, batch = getattr(args, "served_workers", 2), getattr(args, "served_batch", 64)
    srv = apic.Server(0, hbm_budget_bytes=80 << 30, n_workers=workers, max_batch_scenes=batch)
    srv.set_policy(args.variant, not args.no_graphs)
    hs = []
    for s in sims:
        f = s.astype(np.float32)
        hs.append(srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies))
    dts = [0.1 * s.h / max(np.abs(s.v).max(), 1e-30) for s in sims]
    units = np.array([s.n * (s.n_iter + 1) for s in sims], np.float64)
    P = int(sum(s.n for s in sims))

    def round_all(k):
        ts = []
        for _ in range(k):
            ts += [h.submit(dt) for h, dt in zip(hs, dts)]
        for t in ts:
            srv.wait(t, 600.0)

    round_all(max(1, args.warmup // 3))  # warm-up: scratch grows to its working size
    srv.stats(reset=True)
    t0 = time.perf_counter()
    round_all(2)
    cap_s = time.perf_counter() - t0
    capacity = 2 * units.sum() / cap_s
    cap_stats = srv.stats(reset=True)

    loads = {}
    rng = np.random.default_rng(2108_0225 + 5)
    # an untimed open-loop phase first: the workers meet the small batches of
    # light load (new size classes to tune, new buffer sizes) before timing
    for rho in ("warm", 0.5, 0.8, 0.95):
        lam = (0.5 if rho == "warm" else rho) * capacity / units.sum()  # requests per second per simulation
        T = 1.0 if rho == "warm" else seconds
        events = []
        for i in range(len(sims)):
            t = 0.0
            while True:
                t += rng.exponential(1.0 / lam)
                if t >= T:
                    break
                events.append((t, i))
        events.sort()
        tickets = []
        srv.stats(reset=True)
        start = time.perf_counter()
        for t_ev, i in events:
            delay = start + t_ev - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(hs[i].submit(dts[i]))
        for t in tickets:
            srv.wait(t, 600.0)
        wall = time.perf_counter() - start
        st = srv.stats(reset=True)
        if rho == "warm":
            continue
        loads[str(rho)] = {"offered_particle_iters_per_s": rho * capacity,
                           "throughput": st["particle_iters"] / wall, "requests": st["completed"],
                           "failed": st["failed"], "p50_ms": st["latency_p50_ms"], "p99_ms": st["latency_p99_ms"],
                           "mean_ms": st["latency_mean_ms"], "mean_batch_scenes": st["mean_batch_scenes"],
                           "wall_s": wall}
    res = srv.stats()
    for h in hs:
        h.close()
    srv.close()
    resident = res["resident_bytes"]

    out = {"config": {"workload": f"served: {len(sims)} resident simulations, {P} FE nodes in total (2k-1M per "
                                  f"simulation, each size drawn on its own, 2-8 bodies, mu in [0, 0.5], "
                                  f"N = {sims[0].n_iter}), Poisson step requests, each step advects x by "
                                  f"0.1 h / max|v|, 80 GiB budget, {workers} workers, at most {batch} requests a batch",
                      "launch_policy": {"variant": args.variant, "graphs": not args.no_graphs},
                      "particles": P, "simulations": len(sims), "seconds_per_load": seconds,
                      "l2": f"working set far above L2 ({P / 1e6:.1f}M nodes)"},
           "capacity_closed_loop": capacity, "capacity_mean_batch_scenes": cap_stats["mean_batch_scenes"],
           "loads": loads, "resident_bytes": resident,
           "p50_ms_at_0.8": loads["0.8"]["p50_ms"], "p99_ms_at_0.8": loads["0.8"]["p99_ms"]}
    if squeezed:
        # the same simulations against a budget of about half their resident
        # state: admission refuses what does not fit; the admitted ones run a
        # closed-loop round
        budget = int(resident // 2)
        sq_out = {"budget_bytes": budget}
        with apic.Server(0, hbm_budget_bytes=budget, n_workers=2, max_batch_scenes=64) as sq:
            sq.set_policy(args.variant, not args.no_graphs)
            adm, refused = [], 0
            for s, dt_i in zip(sims, dts):
                f = s.astype(np.float32)
                try:
                    adm.append((sq.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter,
                                            n_bodies=s.n_bodies), dt_i, s.n * (s.n_iter + 1)))
                except apic.ApicError as e:
                    if e.code != apic.APIC_ERR_ADMISSION:
                        raise
                    refused += 1
            t0 = time.perf_counter()
            ts = [h.submit(dt_i) for h, dt_i, _ in adm]
            for t in ts:
                sq.wait(t, 600.0)
            wall = time.perf_counter() - t0
            st = sq.stats()
            sq_out.update({"admitted": len(adm), "refused": refused,
                           "admitted_particles": int(sum(u for _, _, u in adm) / (sims[0].n_iter + 1)),
                           "resident_bytes": st["resident_bytes"], "round_particle_iters_per_s":
                           sum(u for _, _, u in adm) / wall, "failed": st["failed"]})
            for h, _, _ in adm:
                h.close()
        out["budget_squeezed"] = sq_out
    return out


def bench_node_normals(apic, ctx, dev, stream, flush, reps=10):
    """apic_node_normals (Sec. 2.3 node normals) on the boundary of a
    100^3-node lattice block: 1,000,000 nodes, 117,612 triangles.  Device
    time per call (CUDA events, L2 flushed before each), against the bytes
    the operation must move: 12 B of ids per triangle; per node 24 B of x,
    24 B of FP64 sums written and read back, 12 B of normals."""
    import torch

    from paper_2108_02259_gb300 import scenes

    x, tri = scenes.box_lattice_surface(100, 100, 100, spacing=1 / 512)
    X = torch.as_tensor(x, device=dev)
    Tr = torch.as_tensor(tri, device=dev)
    out = torch.empty((len(x), 3), dtype=torch.float32, device=dev)
    for _ in range(3):
        apic.node_normals(ctx, X, Tr, out=out, stream=stream)
    ms = []
    for i in range(reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        apic.node_normals(ctx, X, Tr, out=out, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    alg = 12 * len(tri) + (24 + 48 + 12) * len(x)
    peak, kind = measured_peak_hbm()
    return {"mesh": "boundary of a 100^3-node lattice block", "nodes": len(x), "triangles": len(tri),
            "ms": t, "triangles_per_s": len(tri) / (t / 1e3), "nodes_per_s": len(x) / (t / 1e3),
            "algorithmic_bytes": alg, "achieved_gbs": alg / (t / 1e3) / 1e9, "frac_of_hbm_peak": alg / (t / 1e3) / 1e9 / peak}


def bench_augury(apic, ctx, dev, stream, steps=20):
    """apic_augury_steps (Sec. 2.2 augury dynamics, springs + contact) on two
    elastic lattice cubes of 40^3 nodes (128,000 nodes, 1,104,480 springs,
    N = 4), already in contact: device time per time step (CUDA events)."""
    import torch

    from paper_2108_02259_gb300 import scenes

    e = scenes.elastic_pair(n_side=40, spacing=1 / 256, gap_cells=0.5)
    s = e.scene

    def d(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=ty, device=dev)

    st = [d(s.x, torch.float64), d(s.v, torch.float32), d(np.zeros((s.n, 9)), torch.float32),
          d(np.zeros((s.n, 3)), torch.float32), d(np.zeros((s.n, 9)), torch.float32), d(s.m, torch.float32),
          d(s.body, torch.int32), d(e.springs, torch.int32), d(e.rest, torch.float64), d(e.stiffness, torch.float64),
          d(e.tri, torch.int32)]

    def run(k, init=False):
        apic.augury_steps(ctx, *st, s.h, s.mu, s.n_iter, e.dt, e.tau, k, n_bodies=2, init=init, stream=stream)

    run(3, init=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(stream)
    run(steps)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    return {"scene": "two elastic lattice cubes, 40^3 nodes each, in contact", "nodes": s.n,
            "springs": int(len(e.springs)), "n_iter": s.n_iter, "ms_per_time_step": ms,
            "node_steps_per_s": s.n / (ms / 1e3),
            "note": "each time step: normals from boundary triangles, spring forces, one contact step, two half kicks"}


def step_breakdown(prof):
    """Per-step device time by phase, from the profiling run (events on the
    launch stream; passes launched one by one)."""
    k = max(prof["steps"], 1)
    b = {"sort_and_grid_sizing": prof["prep_ms"] / k, "mass_p2g_and_normalise": prof["mass_ms"] / k,
         "transfer_passes": prof["iter_ms"] / k, "step": prof["step_ms"] / k}
    b["normalise_between_passes_host_sync_and_gaps"] = b["step"] - b["sort_and_grid_sizing"] - b["mass_p2g_and_normalise"] - b[
        "transfer_passes"]
    return b


def kernel_source_hash():
    """Hash of the fused transfer kernel's own source: kernels.cu up to the
    end of k_items, the shared types at the top of apic_internal.h and its
    variant table.  Traffic counters taken from an ncu capture count only
    while it is unchanged."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2108_02259_gb300", "csrc")
    k = open(os.path.join(csrc, "kernels.cu")).read()
    k = k[:k.index("// v_i = p_i / m_i (0 where m_i = 0)")]
    h = open(os.path.join(csrc, "apic_internal.h")).read()
    table = "".join(line for line in h.splitlines(True) if "kVariant" in line or "kNumVariants" in line)
    h = h[:h.index("// Cells, validation")] + table
    return hashlib.sha256((k + h).encode()).hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
