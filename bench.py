#!/usr/bin/env python
"""Benchmark: cutoff geodesic pair evaluations/s and MD steps/s on one GB300.

Workload (default): the large noisy sphere -- level-8 icosphere of radius 10 (1,310,720
faces) with vertices displaced radially by 0.02 N(0,1), 65536 active Brownian particles
(v0 = 1, D_r = 0.1), WCA with sigma = 0.2 and r_c = 2^(1/6) sigma, dt = 1e-3.  A "step"
is one full MD step through the C ABI: face bucketing, geodesic neighbours by window
propagation, forces, the face walk and the orientation update.  The headline precision is
the FP32 form (one persistent launch over all sources, the step replayed from a captured
CUDA graph); the FP64 form is measured beside it on the same workload.  The many-mesh
workload (64 tori of 2k-60k faces, 128-4096 particles each, NVE) is measured in the same
run and reported under "batched_tori64": the FP32 batched form (one persistent launch
over all meshes' sources) against the plain FP64 path (one call per mesh).

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the
library's stream, with a 256 MiB L2-flushing write between timed steps (outside the
events); barrier + synchronize around the timed region, max over ranks.  With
--gpus N > 1 (torchrun) every rank runs its own replica (the method does not shard
across GPUs in this build), "scaling": "weak".

--impl reference times the CPU oracle (plain FP64 C, OpenMP over sources) on the
same workload, each step a full oracle MD step of a bounded sample of the particles.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cutoff geodesic pair evals/s & MD steps/s, FP32-batched vs FP64, err≤1e-5"
UNIT = "pair evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FLOPS_PER_PROPAGATION = 150.0   # one window unfolding + child trimming (FP arithmetic)
FLOPS_PER_PAIR = 20.0           # one target evaluation
BYTES_PER_FACE = 64.0           # patch mesh data a source must read per face reached
BYTES_PER_WINDOW = 48.0         # one window record written and read back per propagation
BYTES_PER_PAIR = 20.0           # one FP32 output row entry (j, distance, tangent)
BYTES_PER_SOURCE = 24.0         # the source's force
DEFAULT_WORKLOAD = "noisy_ico8_n65536"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one first-pass launch of the
# FP32 neighbour kernel from an ncu capture, per workload: bytes, the sources that launch
# processed (the figure is scaled to a full launch by sources) and a digest of the kernel
# sources it was taken on; a kernel changed since then reports null
TRAFFIC = {
    # k_geodesic<float, 2, 0> (128-register variant, global tables, 8 warps per CTA, pool of 32768
    # windows) over 8192 of the 65536 sources on the same noisy L8 sphere: 5.829 GB read +
    # 2.419 GB written in 8.72 ms (one ncu pass, dram__bytes_read.sum + dram__bytes_write.sum)
    "noisy_ico8_n65536": {"bytes": 5828550400 + 2418572544, "sources": 8192, "kernel": "0c622ec7855f2012"},
}
KERNEL_SOURCES = ("paper_2404_19751_gb300/csrc/geodesic.cu", "paper_2404_19751_gb300/csrc/css_dev.cuh",
                  "paper_2404_19751_gb300/csrc/css_internal.h")


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch(name: str, n_sources: int):
    t = TRAFFIC.get(name)
    if not t or t["kernel"] != kernel_digest():
        return None
    return t["bytes"] * n_sources / t["sources"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the nested many-mesh measurement of the default workload")
    ap.add_argument("--sweep", choices=["n", "v", "vhm"], default=None,
                    help="time per MD step against particle count (n) or mesh size (v) on a torus, "
                         "with the fitted power-law exponents; vhm: the approximate solver against the "
                         "exact one, all pairs, on the same tori (not the benchmark line)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ------------------------------------------------------------------ the workload
def workload(name: str):
    import synth
    cfg = synth.make_config(name)
    return cfg


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


def cpu_baseline(cfg, budget_s: float = 12.0):
    """The CPU oracle as it stands on this host's cores: full neighbour passes over the
    workload's particles until about budget_s of wall time has been spent."""
    from oracle import oracle as O
    om = O.OracleMesh(cfg["mesh"])
    cores = os.cpu_count() or 1
    face, bary = cfg["face"], cfg["bary"]
    pairs = 0
    passes = 0
    stats = None
    t0 = time.perf_counter()
    while True:
        rs, j, d, t, st = om.neighbors(face, bary, cfg["r_c"], nthreads=cores, stats=True)
        pairs += int(rs[-1])
        passes += 1
        stats = st
        if time.perf_counter() - t0 > budget_s or passes >= 100000:
            break
    el = time.perf_counter() - t0
    # one thread (the paper's own CPU setup), over a bounded prefix of the sources
    n1 = max(1, min(len(face), 256))
    t1 = time.perf_counter()
    pairs1 = reps1 = 0
    while reps1 < 1 or time.perf_counter() - t1 < 2.0:
        rs1, *_ = om.neighbors(face, bary, cfg["r_c"], nthreads=1, sources=list(range(n1)))
        pairs1 += int(rs1[-1])
        reps1 += 1
    el1 = time.perf_counter() - t1
    return dict(value=pairs / el, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{passes} full neighbour passes ({len(face)} sources each, r_c={cfg['r_c']}) "
                       f"of the same workload, FP64, OpenMP over sources, {el:.1f} s",
                single_thread={"value": pairs1 / el1, "unit": UNIT, "cores": 1,
                               "sample": f"{reps1} x the rows of the first {n1} sources, {el1:.2f} s"}), stats, om


def run_reference(args, rank: int, world: int):
    """The oracle as it stands, on the host cores: full MD steps of the same workload
    (forces by window propagation from every particle, the face walk), one mesh after
    another for the many-mesh workload."""
    if rank != 0:
        return
    from oracle import oracle as O
    cfg = workload(args.workload)
    cores = os.cpu_count() or 1
    pot, integ, rc = cfg["pot"], cfg["integ"], cfg["r_c"]
    items = cfg["items"] if "items" in cfg else [cfg]
    states = []
    for it in items:
        om = O.OracleMesh(it["mesh"])
        F, _ = om.forces(it["face"], it["bary"], rc, pot, nthreads=cores)
        states.append((om, dict(face=it["face"], bary=it["bary"], vel=it.get("vel"), orient=it.get("orient"),
                                force=F)))

    def step(k):
        out = []
        for om, st in states:
            st = om.integrate(st["face"], st["bary"], st["vel"], st["orient"], st["force"], pot, integ, rc, 1,
                              nthreads=cores, seed=1, step0=k)
            out.append((om, st))
        return out
    for k in range(args.warmup):
        states = step(k)
    times, pairs = [], 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        states = step(args.warmup + k)
        times.append(time.perf_counter() - t0)
        for om, st in states:
            rs, *_ = om.neighbors(st["face"], st["bary"], rc, nthreads=cores)
            pairs += int(rs[-1])
    total = sum(times)
    v = pairs / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(describe(cfg, 1), l2="host run", precision="FP64 oracle"),
            "md_steps_per_s": args.steps / total,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle MD steps of the full workload after {args.warmup} "
                                       f"warm-up steps, OpenMP over sources"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(dist, t: float, device: str) -> float:
    """The slowest rank's time (every rank gets it); without a process group, t itself.
    The job's throughput is then (units processed by all ranks) / this time."""
    if not dist:
        return t
    import torch
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_throughput(world: int, units_per_rank: float, t_max: float) -> float:
    """Whole-job rate of `world` replicas that each processed units_per_rank in at most t_max."""
    return world * units_per_rank / t_max


POT_NAMES = {0: "harmonic (1-d/sigma)^2", 1: "WCA", 2: "Gaussian"}
INT_NAMES = {0: "NVE velocity Verlet", 1: "overdamped Brownian", 2: "active Brownian"}


def describe(cfg, world):
    """The config object of the JSON line, from the workload itself."""
    pot, integ, rc = cfg["pot"], cfg["integ"], cfg["r_c"]
    if "items" in cfg:
        nfs = [it["mesh"].nf for it in cfg["items"]]
        mesh = f"{len(nfs)} tori, {min(nfs)}-{max(nfs)} faces each ({sum(nfs)} total)"
        n = sum(len(it["face"]) for it in cfg["items"])
    else:
        m = cfg["mesh"]
        mesh = f"{m.name}, {m.nf} faces" + (", periodic" if m.period is not None else "")
        n = len(cfg["face"])
    return {"workload": cfg["name"], "mesh": mesh, "n_particles": n,
            "r_c": rc if math.isfinite(rc) else "all pairs",
            "potential": f"{POT_NAMES[pot['kind']]}, sigma={pot['sigma']:.4g}",
            "integrator": f"{INT_NAMES[integ['kind']]} dt={integ['dt']:g}",
            "l2": "256 MiB flush between timed steps", "parallelism": f"replicas x{world}"}


def counter_reader(ctx):
    """Reads what the last library call measured: its neighbour-kernel time and counts."""
    def read():
        c = ctx.last_counters()
        return ctx.last_kernel_ms(), c["pairs"], c["propagated"]
    return read


class Timer:
    """Per-step CUDA events on the library's stream, an L2-flushing write before each
    timed step (outside the events), clocks sampled during the timed region."""

    def __init__(self, torch, stream, flush, local, dist):
        self.torch, self.stream, self.flush, self.local, self.dist = torch, stream, flush, local, dist

    def run(self, step, steps, warmup, counters):
        torch = self.torch
        for _ in range(warmup):
            step()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kms, pairs, props = [], 0, 0
        torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(self.local) as clk:
            for k in range(steps):
                with torch.cuda.stream(self.stream):
                    self.flush.zero_()
                    ev[k][0].record(self.stream)
                r = step()
                with torch.cuda.stream(self.stream):
                    ev[k][1].record(self.stream)
                # a step may hand back a reader of its counters, so that reading them (bench
                # bookkeeping, not part of the step) happens after the end event
                km, pc, pp = r() if callable(r) else r
                kms.append(km)
                pairs += pc
                props += pp
            torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        t = max_over_ranks(self.dist, sum(a.elapsed_time(b) for a, b in ev) / 1e3, "cuda")
        return dict(t=t, steps=steps, kernel_ms=kms, pairs=pairs, props=props, clocks=clk.summary())


def csr_to_dict(rs, j, d, t):
    """{(i, j): (distance, tangent)} of a CSR neighbour result."""
    out = {}
    for i in range(len(rs) - 1):
        for q in range(rs[i], rs[i + 1]):
            out[(i, int(j[q]))] = (float(d[q]), t[q])
    return out


def accuracy(css, ctx, cases):
    """Max distance error of both forms against the oracle on (mesh handle, synth mesh,
    face, bary, r_c) cases, relative to each mesh's bounding-box diagonal."""
    import synth
    from oracle import oracle as O
    acc = {}
    for prec, nm in ((css.FP32, "fp32"), (css.FP64, "fp64")):
        worst, only = 0.0, 0
        worst_abs = 0.0
        for mesh, m, face, bary, rc, om in cases:
            om = om or O.OracleMesh(m)
            R = csr_to_dict(*om.neighbors(face, bary, rc))
            p2 = css.particles_set(ctx, mesh, face, bary)
            G = csr_to_dict(*css.geodesic_neighbors(p2, rc, prec))
            p2.free()
            common = set(G) & set(R)
            err = max((abs(G[k][0] - R[k][0]) for k in common), default=0.0)
            worst_abs = max(worst_abs, err)
            worst = max(worst, err / synth.bbox_diagonal(m))
            only += len(set(G) ^ set(R))
        acc[nm] = {"max_abs_dist_err": worst_abs, "max_err_over_diameter": worst, "pairs_only_one_side": only}
    return acc


def roofline(css, ctx, pk, props_per_src, n, pairs_per_launch, kern_s, kernel_name, traffic=None):
    """ALU roofline of the neighbour kernel (algorithmic FP32 flops per launch over the
    nominal FP32 peak) and its memory roofline (algorithmic bytes over measured HBM)."""
    fp32_peak_nominal = 152 * 128 * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    alg_flops = n * props_per_src * FLOPS_PER_PROPAGATION + pairs_per_launch * FLOPS_PER_PAIR
    achieved = alg_flops / kern_s
    faces_per_src = props_per_src / 2.0     # about two windows enter each face reached
    alg_bytes = (n * (faces_per_src * BYTES_PER_FACE + props_per_src * BYTES_PER_WINDOW + BYTES_PER_SOURCE) +
                 pairs_per_launch * BYTES_PER_PAIR)
    hbm = float(pk.get("hbm_gbs", 6800.0)) * 1e9
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak_nominal / 1e12,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak_nominal, "traffic": traffic,
            "kernel": kernel_name, "kernel_ms": kern_s * 1e3,
            "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock (nominal; no measured FP32 peak)",
            "fma_probe_tflops": {"fp32": ctx.fma_peak(css.FP32) / 1e12, "fp64": ctx.fma_peak(css.FP64) / 1e12},
            "algorithmic": {"propagations_per_source": props_per_src,
                            "flops_per_propagation": FLOPS_PER_PROPAGATION,
                            "flops_per_pair": FLOPS_PER_PAIR, "flops_per_launch": alg_flops}}
    mem = {"achieved_gbs": alg_bytes / kern_s / 1e9, "peak_gbs": hbm / 1e9, "peak_basis": "measured HBM copy",
           "frac": alg_bytes / kern_s / hbm, "bytes_per_launch": alg_bytes,
           "bytes_model": f"per source {BYTES_PER_FACE:g} B x faces reached (propagations / 2) + "
                          f"{BYTES_PER_WINDOW:g} B x windows propagated + {BYTES_PER_SOURCE:g} B force; "
                          f"{BYTES_PER_PAIR:g} B per pair",
           "traffic_over_algorithmic": (traffic / alg_bytes) if traffic else None}
    return roof, mem


def run_ours(args, rank: int, world: int):
    import torch
    import paper_2404_19751_gb300 as css
    from paper_2404_19751_gb300 import build as cbuild

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(cbuild.LIB):
        if rank == 0:
            cbuild.build()
        if dist:
            dist.barrier()
    css.load()
    cfg = workload(args.workload)
    stream = torch.cuda.Stream()
    ctx = css.create(local, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    timer = Timer(torch, stream, flush, local, dist)
    if "items" in cfg:
        line = run_batched(args, cfg, css, ctx, torch, stream, timer, rank, world)
    else:
        line = run_single(args, cfg, css, ctx, torch, stream, timer, rank, world)
        if args.workload == DEFAULT_WORKLOAD and not args.no_batched:
            # the many-mesh batched form, measured in the same run and nested in the line
            nested = run_batched(args, workload("tori64"), css, ctx, torch, stream, timer, rank, world,
                                 nested=True)
            if line is not None and nested is not None:
                line["batched_tori64"] = nested
    if rank == 0 and line:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_single(args, cfg, css, ctx, torch, stream, timer, rank, world):
    import numpy as np
    m = cfg["mesh"]
    pot, integ, rc = cfg["pot"], cfg["integ"], cfg["r_c"]
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    n = len(cfg["face"])

    def timed_run(prec, steps, warmup):
        parts = css.particles_set(ctx, mesh, cfg["face"], cfg["bary"], cfg["vel"], cfg["orient"], seed=1)
        # the library's autotuner picks the launch shape for this workload (outside the timing)
        shape, _ = ctx.autotune([parts], pot, rc, prec, reps=3, sample=min(n, 16384))

        counters = counter_reader(ctx)

        def step():
            css.integrate_step(parts, pot, integ, rc, prec, 1)
            return counters
        r = timer.run(step, steps, warmup, True)
        r["launch"] = shape
        parts.free()
        return r

    r32 = timed_run(css.FP32, args.steps, args.warmup)
    r64 = timed_run(css.FP64, max(3, args.steps // 2), max(3, args.warmup))
    ctx.set_launch(**r32["launch"])
    t32, t64, k32, k64 = r32["t"], r64["t"], r32["steps"], r64["steps"]
    # ---- end to end through the C ABI with host buffers: upload the state from pinned
    # host memory, one step, read the state back, every step
    parts = css.particles_set(ctx, mesh, cfg["face"], cfg["bary"], cfg["vel"], cfg["orient"], seed=1)
    # a host-driven loop: every step writes the state held in pinned host memory to the
    # device, steps, and reads the new state (and forces) back into the same buffers
    hf = torch.from_numpy(np.ascontiguousarray(cfg["face"], np.int32)).pin_memory()
    hb = torch.from_numpy(np.ascontiguousarray(cfg["bary"])).pin_memory()
    hv = torch.from_numpy(np.ascontiguousarray(cfg["vel"] if cfg["vel"] is not None else np.zeros((n, 3)))).pin_memory()
    oF = torch.empty((n, 3), dtype=torch.float64).pin_memory()

    def e2e_step():
        css.particles_update(parts, hf, hb, hv)
        css.integrate_step(parts, pot, integ, rc, css.FP32, 1)
        pc = ctx.last_counters()["pairs"]
        css.particles_get_into(parts, hf, hb, hv, None, oF)
        return pc
    e2e_t, e2e_pairs = e2e_time(torch, stream, e2e_step, args, timer.dist)
    parts.free()
    h2d = n * (4 + 24 + 24)
    d2h = n * (4 + 24 + 24 + 24)
    if rank != 0:
        mesh.free()
        return None
    pk = peaks()
    cb, ostats, om = (None, None, None)
    if not args.no_cpu_baseline and world == 1:
        cb, ostats, om = cpu_baseline(cfg)
    try:
        acc = accuracy(css, ctx, [(mesh, m, cfg["face"], cfg["bary"], rc, om)])
    except Exception as e:  # accuracy is informative; the parity tests are the gate
        acc = {"error": str(e)}
    # algorithmic work per launch: the oracle's (priority-ordered) propagation count per
    # source times the per-propagation flop figure, plus the pair evaluations
    if ostats:
        props_per_src = ostats["windows_propagated"] / max(1, ostats["sources"])
    else:
        props_per_src = r32["props"] / max(1, k32 * n)
    roof, mem = roofline(css, ctx, pk, props_per_src, n, r32["pairs"] / k32,
                         statistics.mean(r32["kernel_ms"]) / 1e3, "k_geodesic<float>",
                         traffic=traffic_per_launch(cfg["name"], n))
    line = {
        "metric": METRIC, "value": replica_throughput(world, r32["pairs"], t32), "unit": UNIT, "n_gpus": world, "steps": k32,
        "warmup": args.warmup, "ms_per_step": 1e3 * t32 / k32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(describe(cfg, world), precision="FP32 form", launch=r32["launch"]),
        "md_steps_per_s": world * k32 / t32,
        "pairs_per_step": r32["pairs"] / k32,
        "fp64": {"value": replica_throughput(world, r64["pairs"], t64), "unit": UNIT, "md_steps_per_s": world * k64 / t64,
                 "ms_per_step": 1e3 * t64 / k64, "kernel_ms": statistics.mean(r64["kernel_ms"]),
                 "clocks": r64["clocks"], "launch": r64["launch"]},
        "fp32_over_fp64": (r32["pairs"] / t32) / (r64["pairs"] / t64),
        "accuracy_vs_oracle": acc,
        "roofline": roof,
        "memory_roofline": mem,
        "e2e": {"value": replica_throughput(world, e2e_pairs, e2e_t), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        # per step: move (1) + bucketing (6: count, scan, scatter, rank) + neighbour/force first
        # and second pass (2) + kick or step counter (1)
        "gpu_launches": 10 * k32,
        "clocks": r32["clocks"],
        "kernel_digest": kernel_digest(),
    }
    if cb:
        line["cpu_baseline"] = cb
    mesh.free()
    return line


def e2e_time(torch, stream, step, args, dist):
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ee = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    pairs = 0
    with torch.cuda.stream(stream):
        ee[0].record(stream)
    for _ in range(args.steps):
        pairs += step()
    with torch.cuda.stream(stream):
        ee[1].record(stream)
    torch.cuda.synchronize()
    t = max_over_ranks(dist, ee[0].elapsed_time(ee[1]) / 1e3, "cuda")
    return t, pairs


def run_batched(args, cfg, css, ctx, torch, stream, timer, rank, world, nested=False):
    """Many independent meshes: the FP32 batched form (one persistent launch per step over
    every source of every mesh, inside a captured graph) against the plain FP64 path (one
    integrate call per mesh), both forms of both shown.  nested: the compact record that
    the default workload's line carries (FP32 batched vs FP64 plain, accuracy on three
    meshes, the same timing rules; no CPU baseline or end-to-end loop)."""
    import numpy as np
    items = cfg["items"]
    pot, integ, rc = cfg["pot"], cfg["integ"], cfg["r_c"]
    meshes = [css.mesh_upload(ctx, it["mesh"].verts, it["mesh"].faces) for it in items]
    n = sum(len(it["face"]) for it in items)

    def make_sets():
        return [css.particles_set(ctx, meshes[k], it["face"], it["bary"], it["vel"], None, seed=1)
                for k, it in enumerate(items)]

    default_shape = ctx.get_launch()

    def batched(prec, steps, warmup):
        sets = make_sets()
        b = css.batch_create(ctx, sets)
        # the autotuner picks warps, residency, table scale and work tile for the batch
        shape, _ = ctx.autotune(sets, pot, rc, prec, reps=3, sample=32768)

        counters = counter_reader(ctx)

        def step():
            css.batch_step(b, pot, integ, rc, prec, 1)
            return counters
        r = timer.run(step, steps, warmup, True)
        r["launch"] = shape
        b.free()
        for p in sets:
            p.free()
        return r

    def plain(prec, steps, warmup):
        ctx.set_launch(**default_shape)   # the plain path: default launch shape, one call per mesh
        sets = make_sets()

        def step():
            km = pc = pp = 0
            for p in sets:
                css.integrate_step(p, pot, integ, rc, prec, 1)
                c = ctx.last_counters()
                km += ctx.last_kernel_ms()
                pc += c["pairs"]
                pp += c["propagated"]
            return km, pc, pp
        r = timer.run(step, steps, warmup, True)
        for p in sets:
            p.free()
        return r

    saved_shape = ctx.get_launch()
    r32b = batched(css.FP32, args.steps, args.warmup)
    ks = max(3, args.steps // 2)
    r64p = plain(css.FP64, ks, max(3, args.warmup))

    def rate(r):
        return replica_throughput(world, r["pairs"], r["t"])

    def sub(r, what):
        return {"value": rate(r), "unit": UNIT, "what": what, "md_steps_per_s": world * r["steps"] / r["t"],
                "mesh_steps_per_s": world * len(items) * r["steps"] / r["t"],
                "ms_per_step": 1e3 * r["t"] / r["steps"], "kernel_ms": statistics.mean(r["kernel_ms"]),
                "clocks": r["clocks"]}
    if nested:
        ctx.set_launch(**saved_shape)
        out = None
        if rank == 0:
            order = np.argsort([len(it["face"]) for it in items], kind="stable")
            pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
            try:
                acc = accuracy(css, ctx, [(meshes[k], items[k]["mesh"], items[k]["face"], items[k]["bary"], rc, None)
                                          for k in pick])
                acc["sampled_meshes"] = pick
            except Exception as e:
                acc = {"error": str(e)}
            out = {"workload": cfg["name"], "config": dict(describe(cfg, world),
                                                           precision="FP32 form, batched (one launch over all meshes)",
                                                           launch=r32b["launch"]),
                   **sub(r32b, "FP32 form, batched: one persistent launch per step over all meshes"),
                   "steps": r32b["steps"], "pairs_per_step": r32b["pairs"] / r32b["steps"],
                   "particle_steps_per_s": world * n * r32b["steps"] / r32b["t"],
                   "fp64": sub(r64p, "plain FP64: one integrate call per mesh"),
                   "fp32_batched_over_fp64": rate(r32b) / rate(r64p), "accuracy_vs_oracle": acc,
                   "gpu_launches": 8 * r32b["steps"]}
        for mh in meshes:
            mh.free()
        return out
    r64b = batched(css.FP64, ks, max(3, args.warmup))
    r32p = plain(css.FP32, ks, max(3, args.warmup))
    ctx.set_launch(**r32b["launch"])
    # ---- end to end: every mesh's state up from pinned host memory, one batched step, all
    # states back, every step
    sets = make_sets()
    b = css.batch_create(ctx, sets)
    host = []
    for it in items:
        k = len(it["face"])
        host.append((torch.from_numpy(np.ascontiguousarray(it["face"], np.int32)).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(it["bary"])).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(it["vel"])).pin_memory(),
                     torch.empty((k, 3), dtype=torch.float64).pin_memory()))

    def e2e_step():
        for p, h in zip(sets, host):
            css.particles_update(p, h[0], h[1], h[2])
        css.batch_step(b, pot, integ, rc, css.FP32, 1)
        pc = ctx.last_counters()["pairs"]
        for p, h in zip(sets, host):
            css.particles_get_into(p, h[0], h[1], h[2], None, h[3])
        return pc
    e2e_t, e2e_pairs = e2e_time(torch, stream, e2e_step, args, timer.dist)
    b.free()
    for p in sets:
        p.free()
    if rank != 0:
        for mh in meshes:
            mh.free()
        return None
    pk = peaks()
    # the oracle on the host cores: full neighbour passes over every mesh, bounded
    cb, props_per_src = None, None
    oms = {}
    if not args.no_cpu_baseline and world == 1:
        from oracle import oracle as O
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        pairs = srcs = props = 0
        passes = 0
        while passes < 1 or time.perf_counter() - t0 < 12.0:
            for k, it in enumerate(items):
                om = oms.get(k) or O.OracleMesh(it["mesh"])
                oms[k] = om
                rs, j, d, t, st = om.neighbors(it["face"], it["bary"], rc, nthreads=cores, stats=True)
                pairs += int(rs[-1])
                srcs += st["sources"]
                props += st["windows_propagated"]
            passes += 1
        el = time.perf_counter() - t0
        props_per_src = props / max(1, srcs)
        cb = dict(value=pairs / el, unit=UNIT, cores=cores, kind="oracle",
                  sample=f"{passes} full neighbour pass(es) over all {len(items)} meshes ({n} sources, "
                         f"r_c={rc}), FP64, OpenMP over sources, {el:.1f} s, mesh setup included")
    if props_per_src is None:
        props_per_src = r32b["props"] / max(1, r32b["steps"] * n)
    order = np.argsort([len(it["face"]) for it in items], kind="stable")
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    try:
        acc = accuracy(css, ctx, [(meshes[k], items[k]["mesh"], items[k]["face"], items[k]["bary"], rc, oms.get(k))
                                  for k in pick])
        acc["sampled_meshes"] = pick
    except Exception as e:
        acc = {"error": str(e)}
    k32 = r32b["steps"]
    roof, mem = roofline(css, ctx, pk, props_per_src, n, r32b["pairs"] / k32,
                         statistics.mean(r32b["kernel_ms"]) / 1e3, "k_geodesic<float> (batched launch)")
    # per step, for all meshes at once: move (1) + bucketing (4: count, scan, scatter, rank) +
    # two passes (2) + kick or step counter (1)
    launches_per_step = 8
    line = {
        "metric": METRIC, "value": rate(r32b), "unit": UNIT, "n_gpus": world, "steps": k32,
        "warmup": args.warmup, "ms_per_step": 1e3 * r32b["t"] / k32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(describe(cfg, world), precision="FP32 form, batched (one launch over all meshes)",
                       launch=r32b["launch"]),
        "md_steps_per_s": world * k32 / r32b["t"],
        "mesh_steps_per_s": world * len(items) * k32 / r32b["t"],
        "particle_steps_per_s": world * n * k32 / r32b["t"],
        "pairs_per_step": r32b["pairs"] / k32,
        "fp64": sub(r64p, "plain FP64: one integrate call per mesh"),
        "fp64_batched": dict(sub(r64b, "FP64 form, batched"), launch=r64b["launch"]),
        "fp32_plain": sub(r32p, "FP32 form, one integrate call per mesh"),
        "fp32_over_fp64": rate(r32b) / rate(r64p),
        "accuracy_vs_oracle": acc,
        "roofline": roof,
        "memory_roofline": mem,
        "e2e": {"value": replica_throughput(world, e2e_pairs, e2e_t), "unit": UNIT, "h2d_bytes_per_step": n * (4 + 24 + 24),
                "d2h_bytes_per_step": n * (4 + 24 + 24 + 24)},
        "gpu_launches": launches_per_step * k32,
        "clocks": r32b["clocks"],
    }
    if cb:
        line["cpu_baseline"] = cb
    for mh in meshes:
        mh.free()
    return line


def run_sweep(args):
    """Time per MD step against N (torus r=1, R=3, ~4616 faces, range 1) or against the face
    count V (N = 100 on the same aspect-3 torus, range = one tenth of the span, and the
    whole mesh without cutoff), both forms, each point the median of `--steps` graph-replayed
    steps after `--warmup`; prints the points and the log-log slopes (the paper's Sec. 4
    reports exponents of about 1.4 in N and 2.07 / 1.73 in V for its CPU code)."""
    import numpy as np
    import torch
    import paper_2404_19751_gb300 as css
    import synth
    from synth.configs import torus_for_faces
    ctx = css.create(0)
    integ = dict(kind=css.INT_NVE, dt=1e-3, kT=0.0, lam=1.0, v0=0.0, Dr=0.0, mass=1.0, max_disp=math.inf)

    def step_ms(m, n, r_c, prec, seed):
        face, bary = synth.place_uniform(m, n, seed)
        mesh = css.mesh_upload(ctx, m.verts, m.faces)
        parts = css.particles_set(ctx, mesh, face, bary)
        sig = r_c if math.isfinite(r_c) else 1.0
        pot = dict(kind=css.POT_HARMONIC, eps=1.0, sigma=sig, r_cut=sig)
        css.integrate_step(parts, pot, integ, r_c, prec, max(1, args.warmup))
        t = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            css.integrate_step(parts, pot, integ, r_c, prec, 1)
            b.record()
            torch.cuda.synchronize()
            t.append(a.elapsed_time(b))
        parts.free()
        mesh.free()
        return float(np.median(t))

    pts = []
    if args.sweep == "n":
        m = torus_for_faces(4616, 3.0, 1.0)
        for n in (64, 128, 256, 512, 1024, 2048, 4096):
            pts.append(dict(N=n, faces=m.nf, r_c=1.0, ms_fp32=step_ms(m, n, 1.0, css.FP32, 7),
                            ms_fp64=step_ms(m, n, 1.0, css.FP64, 7)))
        xs = [p["N"] for p in pts]
        paper = {"submesh": 1.4, "full_mesh": 1.4}
    else:
        for F in (1000, 2000, 4000, 8000, 16000):
            m = torus_for_faces(F, 3.0, 1.0)
            span = 2 * (3.0 + 1.0)
            pts.append(dict(N=100, faces=m.nf, r_c=span / 10, ms_fp32=step_ms(m, 100, span / 10, css.FP32, 8),
                            ms_fp64=step_ms(m, 100, span / 10, css.FP64, 8),
                            full_ms_fp32=step_ms(m, 100, math.inf, css.FP32, 8)))
        xs = [p["faces"] for p in pts]
        paper = {"submesh": 1.73, "full_mesh": 2.07}

    def slope(key):
        ys = [p[key] for p in pts]
        return float(np.polyfit(np.log(xs), np.log(ys), 1)[0])
    out = {"sweep": args.sweep, "points": pts, "exponent_fp32": slope("ms_fp32"), "exponent_fp64": slope("ms_fp64"),
           "paper_exponents_cpu": paper}
    if args.sweep == "v":
        out["exponent_full_mesh_fp32"] = slope("full_ms_fp32")
    print(json.dumps(out), flush=True)
    ctx.close()


def run_vhm_sweep(args):
    """All-pairs neighbours on the V-sweep tori (100 particles, aspect 3) by the approximate
    solver (heat-method distances, vector-heat tangents, t = h^2) and by exact window
    propagation (FP64 and FP32): median time of `--steps` calls after `--warmup`, and the
    approximate solver's error against the exact FP64 distances and tangents."""
    import numpy as np
    import torch
    import paper_2404_19751_gb300 as css
    import synth
    from synth.configs import torus_for_faces
    ctx = css.create(0)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            out = fn()
        t = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            t.append(1e3 * (time.perf_counter() - t0))
        return float(np.median(t)), out

    pts = []
    for F in (1000, 2000, 4000, 8000, 16000):
        m = torus_for_faces(F, 3.0, 1.0)
        face, bary = synth.place_uniform(m, 100, 8)
        mesh = css.mesh_upload(ctx, m.verts, m.faces)
        parts = css.particles_set(ctx, mesh, face, bary)
        ms_a, a = timed(lambda: css.vhm_neighbors(parts, math.inf, 1.0))
        c = ctx.last_counters()
        ms_e, e = timed(lambda: css.geodesic_neighbors(parts, math.inf, css.FP64))
        ms_e32, _ = timed(lambda: css.geodesic_neighbors(parts, math.inf, css.FP32))
        rel = np.abs(a[2] - e[2]) / np.maximum(e[2], 1e-12)
        far = e[2] > 0.1 * np.max(e[2])
        ang = np.arccos(np.clip(np.sum(a[3] * e[3], axis=1), -1.0, 1.0))
        pts.append(dict(faces=m.nf, vertices=m.nv, pairs=int(len(e[2])), ms_vhm=ms_a, ms_exact_fp64=ms_e,
                        ms_exact_fp32=ms_e32, heat_sweeps=int(c["windows"]), cg_iterations=int(c["propagated"]),
                        rel_dist_err_mean=float(rel[far].mean()), rel_dist_err_p99=float(np.percentile(rel[far], 99)),
                        tangent_angle_err_median=float(np.median(ang[far])),
                        tangent_angle_err_p90=float(np.percentile(ang[far], 90))))
        parts.free()
        mesh.free()
    xs = [p["faces"] for p in pts]

    def slope(key):
        return float(np.polyfit(np.log(xs), np.log([p[key] for p in pts]), 1)[0])
    print(json.dumps({"sweep": "vhm", "what": "all pairs of 100 particles on aspect-3 tori, t = h^2; times are "
                      "wall ms per call (host outputs included)", "points": pts,
                      "exponent_vhm": slope("ms_vhm"), "exponent_exact_fp64": slope("ms_exact_fp64"),
                      "exponent_rel_err": slope("rel_dist_err_mean")}), flush=True)
    ctx.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.sweep == "vhm":
        run_vhm_sweep(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
