#!/usr/bin/env python
"""Benchmark: cutoff geodesic pair evaluations/s and MD steps/s on one GB300.

Workload (default): the icosphere workload -- level-5 icosphere of radius 1
(20480 faces), 1024 particles uniform on the surface, cutoff r_c = 0.15, harmonic
repulsion sigma = 0.15, velocity-Verlet NVE at dt = 0.002.  A "step" is one full MD
step through the C ABI: face bucketing, geodesic neighbours by window propagation,
forces, the face-walk drift and both kicks.  The headline precision is the FP32 form;
the FP64 form is measured beside it.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the
library's stream, with a 256 MiB L2-flushing write between timed steps (outside the
events); barrier + synchronize around the timed region, max over ranks.  With
--gpus N > 1 (torchrun) every rank runs its own replica (the method does not shard
across GPUs in this build), "scaling": "weak".

--impl reference times the CPU oracle (plain FP64 C, OpenMP over sources) on the
same workload, each step a full oracle MD step.
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ico5_n1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
        if time.perf_counter() - t0 > budget_s or passes >= 200:
            break
    el = time.perf_counter() - t0
    return dict(value=pairs / el, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{passes} full neighbour passes ({len(face)} sources each, r_c={cfg['r_c']}) "
                       f"of the same workload, FP64, OpenMP over sources, {el:.1f} s"), stats, om


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    cfg = workload(args.workload)
    om = O.OracleMesh(cfg["mesh"])
    cores = os.cpu_count() or 1
    face, bary, vel = cfg["face"], cfg["bary"], cfg["vel"]
    pot, integ, rc = cfg["pot"], cfg["integ"], cfg["r_c"]
    F, _ = om.forces(face, bary, rc, pot, nthreads=cores)
    state = dict(face=face, bary=bary, vel=vel, force=F)
    for _ in range(args.warmup):
        state = om.integrate(state["face"], state["bary"], state["vel"], None, state["force"], pot, integ, rc, 1,
                             nthreads=cores)
    times, pairs = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        state = om.integrate(state["face"], state["bary"], state["vel"], None, state["force"], pot, integ, rc, 1,
                             nthreads=cores)
        times.append(time.perf_counter() - t0)
        rs, *_ = om.neighbors(state["face"], state["bary"], rc, nthreads=cores)
        pairs += int(rs[-1])
    total = sum(times)
    v = pairs / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_particles": len(face), "faces": int(cfg["mesh"].nf),
                       "r_c": rc, "integrator": "NVE velocity Verlet", "l2": "host run"},
            "md_steps_per_s": args.steps / total,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle MD steps of the full workload after {args.warmup} "
                                       f"warm-up steps, OpenMP over sources"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank: int, world: int):
    import numpy as np
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
    m = cfg["mesh"]
    pot, integ, rc = cfg["pot"], cfg["integ"], cfg["r_c"]
    stream = torch.cuda.Stream()
    ctx = css.create(local, stream=stream.cuda_stream)
    mesh = css.mesh_upload(ctx, m.verts, m.faces, m.period)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    n = len(cfg["face"])

    def timed_run(prec, steps, warmup):
        parts = css.particles_set(ctx, mesh, cfg["face"], cfg["bary"], cfg["vel"], cfg["orient"], seed=1)
        for _ in range(warmup):
            css.integrate_step(parts, pot, integ, rc, prec, 1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kms, pairs, props = [], 0, 0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for k in range(steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                    ev[k][0].record(stream)
                css.integrate_step(parts, pot, integ, rc, prec, 1)
                with torch.cuda.stream(stream):
                    ev[k][1].record(stream)
                kms.append(ctx.last_kernel_ms())
                c = ctx.last_counters()
                pairs += c["pairs"]
                props += c["propagated"]
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        state = css.particles_get(parts)
        parts.free()
        return dict(step_ms=step_ms, kernel_ms=kms, pairs=pairs, props=props, clocks=clk.summary(), state=state)

    r32 = timed_run(css.FP32, args.steps, args.warmup)
    r64 = timed_run(css.FP64, max(3, args.steps // 2), max(3, args.warmup))

    def agg(r):
        t = sum(r["step_ms"]) / 1e3
        if dist:
            tt = torch.tensor([t], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t

    t32 = agg(r32)
    t64 = agg(r64)
    k32 = len(r32["step_ms"])
    k64 = len(r64["step_ms"])
    value = world * r32["pairs"] / t32
    # ---- end to end through the C ABI with host buffers: upload the state from pinned
    # host memory, one step, read the state back, every step
    parts = css.particles_set(ctx, mesh, cfg["face"], cfg["bary"], cfg["vel"], cfg["orient"], seed=1)
    hf = torch.from_numpy(np.ascontiguousarray(cfg["face"], np.int32)).pin_memory()
    hb = torch.from_numpy(np.ascontiguousarray(cfg["bary"])).pin_memory()
    hv = torch.from_numpy(np.ascontiguousarray(cfg["vel"] if cfg["vel"] is not None else np.zeros((n, 3)))).pin_memory()
    of = torch.empty(n, dtype=torch.int32).pin_memory()
    ob = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    ov = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    oF = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    for _ in range(max(3, args.warmup)):
        css.particles_update(parts, hf, hb, hv)
        css.integrate_step(parts, pot, integ, rc, css.FP32, 1)
        css.particles_get_into(parts, of, ob, ov, None, oF)
    torch.cuda.synchronize()
    e2e_steps = args.steps
    ee = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    e2e_pairs = 0
    with torch.cuda.stream(stream):
        ee[0].record(stream)
    for _ in range(e2e_steps):
        css.particles_update(parts, hf, hb, hv)
        css.integrate_step(parts, pot, integ, rc, css.FP32, 1)
        e2e_pairs += ctx.last_counters()["pairs"]
        css.particles_get_into(parts, of, ob, ov, None, oF)
    with torch.cuda.stream(stream):
        ee[1].record(stream)
    torch.cuda.synchronize()
    e2e_t = ee[0].elapsed_time(ee[1]) / 1e3
    parts.free()
    if dist:
        tt = torch.tensor([e2e_t], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
    h2d = n * (4 + 24 + 24)
    d2h = n * (4 + 24 + 24 + 24)
    if rank != 0:
        return
    # ---- accuracy of this run's first state against the oracle, roofline, CPU baseline
    pk = peaks()
    fp32_peak_nominal = 152 * 128 * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    fp32_probe = ctx.fma_peak(css.FP32)
    fp64_probe = ctx.fma_peak(css.FP64)
    cb, ostats, om = (None, None, None)
    if not args.no_cpu_baseline and world == 1:
        cb, ostats, om = cpu_baseline(cfg)
    acc = {}
    try:
        import synth
        from tests._common import csr_to_dict
        if om is None:
            from oracle import oracle as O
            om = O.OracleMesh(m)
        ref = om.neighbors(cfg["face"], cfg["bary"], rc)
        p2 = css.particles_set(ctx, mesh, cfg["face"], cfg["bary"])
        R = csr_to_dict(*ref)
        diam = synth.bbox_diagonal(m)
        for prec, nm in ((css.FP32, "fp32"), (css.FP64, "fp64")):
            G = csr_to_dict(*css.geodesic_neighbors(p2, rc, prec))
            common = set(G) & set(R)
            err = max((abs(G[k][0] - R[k][0]) for k in common), default=0.0)
            acc[nm] = {"max_abs_dist_err": err, "max_err_over_diameter": err / diam,
                       "pairs_only_one_side": len(set(G) ^ set(R))}
        p2.free()
    except Exception as e:  # accuracy is informative; the parity tests are the gate
        acc = {"error": str(e)}
    # algorithmic work per launch: the oracle's (priority-ordered) propagation count per
    # source times the per-propagation flop figure, plus the pair evaluations
    if ostats:
        props_per_src = ostats["windows_propagated"] / max(1, ostats["sources"])
    else:
        props_per_src = r32["props"] / max(1, k32 * n)
    pairs_per_launch = r32["pairs"] / k32
    alg_flops = n * props_per_src * FLOPS_PER_PROPAGATION + pairs_per_launch * FLOPS_PER_PAIR
    kern_s = statistics.mean(r32["kernel_ms"]) / 1e3
    achieved = alg_flops / kern_s
    faces_per_src = props_per_src / 2.0     # about two windows enter each face reached
    alg_bytes = n * faces_per_src * BYTES_PER_FACE + pairs_per_launch * 24.0
    hbm = float(pk.get("hbm_gbs", 6800.0)) * 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": k32, "warmup": args.warmup,
        "ms_per_step": 1e3 * t32 / k32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "mesh": f"icosphere level 5, radius 1, {m.nf} faces",
                   "n_particles": n, "r_c": rc, "potential": "harmonic (1-d/sigma)^2, sigma=0.15",
                   "integrator": "NVE velocity Verlet dt=0.002", "precision": "FP32 form",
                   "l2": "256 MiB flush between timed steps", "parallelism": f"replicas x{world}"},
        "md_steps_per_s": world * k32 / t32,
        "pairs_per_step": r32["pairs"] / k32,
        "fp64": {"value": world * r64["pairs"] / t64, "unit": UNIT, "md_steps_per_s": world * k64 / t64,
                 "ms_per_step": 1e3 * t64 / k64, "kernel_ms": statistics.mean(r64["kernel_ms"]),
                 "clocks": r64["clocks"]},
        "fp32_over_fp64": (r32["pairs"] / t32) / (r64["pairs"] / t64),
        "accuracy_vs_oracle": acc,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak_nominal / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak_nominal, "traffic": None,
                     "kernel": "k_geodesic<float>", "kernel_ms": kern_s * 1e3,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock",
                     "fma_probe_tflops": {"fp32": fp32_probe / 1e12, "fp64": fp64_probe / 1e12},
                     "algorithmic": {"propagations_per_source": props_per_src,
                                     "flops_per_propagation": FLOPS_PER_PROPAGATION,
                                     "flops_per_pair": FLOPS_PER_PAIR, "flops_per_launch": alg_flops}},
        "memory_roofline": {"achieved_gbs": alg_bytes / kern_s / 1e9, "peak_gbs": hbm / 1e9,
                            "frac": alg_bytes / kern_s / hbm, "bytes_per_launch": alg_bytes},
        "e2e": {"value": world * e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 8 * k32,
        "clocks": r32["clocks"],
    }
    if cb:
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    mesh.free()
    ctx.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
