#!/usr/bin/env python
"""Throughput of the FPPG relaxation path on GB300: particle-iterations/s.

Workload (default): icosphere r = 1 (level 5, 20,480 triangles) plus torus
R = 1, r = 0.3 (256 x 64 quads) at dx = 0.02, h = 1.3 dx -- two bodies,
~0.78 M particles, seeded synthetic lattices with +-0.25 dx jitter.  A step
is one replay of a 50-iteration CUDA graph of the batched form (every phase
of an iteration is one launch over both bodies); K = 10 steps are the 500
iterations of the workload.  L2 is flushed (a 256 MiB write) between steps,
outside the timed events.

Reported beside it: the plain form (each body relaxed with its own launches,
no graph), the end-to-end number through the C ABI with host buffers (pinned
host -> device copy of the particles, relaxation, device -> host copy of the
positions, every step), the force kernel against the FP32 ALU roofline, and
the FP64 CPU oracle on the host cores.  ``--impl reference`` times the
oracle alone (the CPU program the GPU path is checked against).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20
SMS, FP32_LANES = 152, 128        # GB300: SMs and FP32 lanes per SM
# DRAM bytes (read + write) of one k_force launch on the default workload
# (dx = 0.02), from the ncu capture summarised in
# profiles/k_force_icosphere_torus_dx002.md; None for other workloads and
# until the current kernel has been captured.
K_FORCE_DRAM_BYTES = {0.02: 26615040 + 3072}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--iters-per-step", type=int, default=50)
    p.add_argument("--dx", type=float, default=0.02)
    p.add_argument("--no-extras", action="store_true", help="skip plain / e2e / CPU legs")
    p.add_argument("--no-autotune", action="store_true", help="keep the default kernel configuration")
    p.add_argument("--config", default=None,
                   help="force variant,block,search CTAs per SM (e.g. 0,128,4) instead of the autotuner")
    return p.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float) -> float:
    """Largest value over the ranks of the default process group (itself
    when not distributed); CUDA tensors under NCCL, CPU tensors under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle(asm, iters=1):
    """The FP64 oracle on the host cores: `iters` iterations of every body."""
    import oracle
    bodies = [oracle.from_assembly(a) for a in asm]
    t0 = time.perf_counter()
    for o in bodies:
        o.relax(iters)
    dt = time.perf_counter() - t0
    n = sum(a.n for a in asm)
    return n * iters / dt, oracle.get_threads(), dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2501_03056_gb300 import workloads as W
    import oracle
    asm = W.sphere_torus_workload(dx=args.dx)
    bodies = [oracle.from_assembly(a) for a in asm]
    n = sum(a.n for a in asm)
    for _ in range(args.warmup):
        for o in bodies:
            o.relax(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for o in bodies:
            o.relax(1)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": "relaxation particle-iterations/s", "value": value,
        "unit": "particle-iterations/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"icosphere_l5+torus_256x64 dx={args.dx}", "bodies": 2, "particles": n,
                   "iterations_per_step": 1, "form": "FP64 CPU oracle, one iteration per step (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "particle-iterations/s", "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": "one FP64 iteration of both bodies per step"},
        "e2e": {"value": value, "unit": "particle-iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2501_03056_gb300 as pkg
    from paper_2501_03056_gb300 import workloads as W

    G, K, Wm = args.iters_per_step, args.steps, args.warmup
    asm = W.sphere_torus_workload(seed=1 + 10 * rank, dx=args.dx)    # weak scaling: one copy per rank
    n = sum(a.n for a in asm)
    stream = torch.cuda.current_stream()
    bodies = [pkg.Body.from_assembly(a, stream=stream) for a in asm]
    cand = pairs = tested = 0
    for b in bodies:
        c, p, t = b.work_counts()
        cand += c
        pairs += p
        tested += t
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed_steps(step_fn, reset_fn):
        reset_fn()
        for _ in range(Wm):
            step_fn()
        reset_fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        for s, e in ev:
            flush.zero_()
            s.record(stream)
            step_fn()
            e.record(stream)
        barrier()
        return [s.elapsed_time(e) for s, e in ev]

    # ---- batched form, CUDA graph of G iterations --------------------------
    batch = pkg.Batch(bodies, stream=stream)
    if args.config:
        v, tb, sc = (int(x) for x in args.config.split(","))
        batch.configure(v, tb, sc)
        tuned = {"force_variant": v, "force_block": tb, "search_ctas_per_sm": sc, "fixed": True}
    else:
        tuned = None if args.no_autotune else batch.autotune(G)   # trials as long as a timed step
    batch.set_graph_iters(G)
    clocks = Clocks(local)
    clocks.start()
    ms = timed_steps(lambda: batch.relax(G, use_graph=True), batch.load)
    clk = clocks.stop()
    # one more replay, with CUDA event records around the phases of every
    # iteration captured into the graph: live per-phase device times
    batch.time_force(True)
    batch.load()
    batch.relax(G, use_graph=True)
    phases = batch.phase_ms()
    force_ms = phases["force"]
    batch.time_force(False)
    tot_ms = max_over_ranks(sum(ms))
    value = n * world * G * K / (tot_ms / 1e3)
    kpi = batch.kernels_per_iter

    extras = {}
    if not args.no_extras:
        # ---- plain form: each body with its own launches, no graph ---------
        def plain_reset():
            for b, a in zip(bodies, asm):
                b.set_particles(a.xyz, a.cls)

        pms = timed_steps(lambda: [b.relax(G) for b in bodies], plain_reset)
        plain_value = n * G * K / (sum(pms) / 1e3)
        extras["plain"] = {"value": plain_value, "unit": "particle-iterations/s", "ms_per_step": sum(pms) / K,
                           "launches_per_iteration": kpi * len(bodies), "graph": False}
        extras["batched_over_plain"] = value / world / plain_value

        # ---- end to end through the C ABI with host buffers ------------------
        pinned = [(torch.from_numpy(np.ascontiguousarray(a.xyz)).pin_memory(),
                   torch.from_numpy(np.ascontiguousarray(a.cls)).pin_memory(),
                   torch.empty((a.n, 3), dtype=torch.float32).pin_memory()) for a in asm]

        def e2e_step():
            for b, (x, c, _) in zip(bodies, pinned):
                b.set_particles(x.numpy(), c.numpy())
            batch.load()
            batch.relax(G, use_graph=True)
            batch.store()
            for b, (_, _, out) in zip(bodies, pinned):
                b.get_positions_into(out.numpy())

        for _ in range(Wm):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            e2e_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        extras["e2e"] = {"value": n * world * G * K / e2e_s, "unit": "particle-iterations/s",
                         "h2d_bytes_per_step": int(n * 16), "d2h_bytes_per_step": int(n * 12)}

        # ---- the other configurations at full size: batched + graph and plain ---
        def config_leg(casm, steps=2):
            cb = [pkg.Body.from_assembly(a, stream=stream) for a in casm]
            cn = sum(b.n for b in cb)
            snap_c = [b.get_particles() for b in cb]

            def reset_c():
                for b, (x, c, cons) in zip(cb, snap_c):
                    b.set_particles(x, c)
                    b.set_constraints(cons)

            cbt = pkg.Batch(cb, stream=stream)
            ctuned = cbt.autotune(G)
            cbt.set_graph_iters(G)
            t_b, t_p = [], []
            for _ in range(steps + 1):
                cbt.load()
                flush.zero_()
                s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s_.record(stream)
                cbt.relax(G, use_graph=True)
                e_.record(stream)
                torch.cuda.synchronize()
                t_b.append(s_.elapsed_time(e_))
                reset_c()
                flush.zero_()
                s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s_.record(stream)
                for b in cb:
                    b.relax(G)
                e_.record(stream)
                torch.cuda.synchronize()
                t_p.append(s_.elapsed_time(e_))
                reset_c()
            cbt.close()
            for b in cb:
                b.close()
            vb_ = cn * G * steps / (sum(t_b[1:]) / 1e3)
            vp_ = cn * G * steps / (sum(t_p[1:]) / 1e3)
            return {"particles": cn, "iterations_per_step": G, "steps": steps, "warmup": 1,
                    "batched_graph": vb_, "plain": vp_, "batched_over_plain": vb_ / vp_,
                    "unit": "particle-iterations/s", "autotune": ctuned}

        extras["configs"] = {
            "cube (config 1, dx=0.05)": config_leg(W.cube_workload()),
            "spur gear (config 3, dx=0.004, generated)": config_leg(W.gear_workload()),
            "vehicle shell (config 5, 2.0 M triangles, dx=0.0068, generated)": config_leg(W.vehicle_workload(), 1),
        }

        # ---- generation (Sec. 3.2) on the GPU: config 3's gear ------------------
        ga = W.gear_workload()[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gb = pkg.Body(ga.verts, ga.tris, ga.dx, ga.h, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        gb.extract_features(ga.dihedral_deg)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        gn = gb.map_particles(**ga.meta["generate"])
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        extras["generation"] = {"workload": f"spur gear, {len(ga.tris)} triangles, dx={ga.dx:g}, band 2 + inner 1 cells",
                                "particles": gn, "mesh_build_ms": 1e3 * (t1 - t0),
                                "features_ms": 1e3 * (t2 - t1), "map_particles_ms": 1e3 * (t3 - t2),
                                "particles_per_s": gn / (t3 - t2), "timer": "host wall clock around synchronised calls"}
        gb.close()

        # ---- energy (A8): energy-descent relaxation and the backward ------------
        for b, a in zip(bodies, asm):
            b.set_particles(a.xyz, a.cls)
        Ge = 10
        for b in bodies:
            b.relax_energy(1)
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for b in bodies:
            b.relax_energy(Ge)
        ee.record(stream)
        torch.cuda.synchronize()
        e_relax = n * Ge / (es.elapsed_time(ee) / 1e3)
        tb, ta = bodies[1], asm[1]                      # the torus: surface particles through the projection
        y = torch.from_numpy(np.ascontiguousarray(tb.get_particles()[0])).cuda()
        verts = torch.from_numpy(np.ascontiguousarray(ta.verts)).cuda()
        gy, gv = torch.empty_like(y), torch.empty_like(verts)
        tb.energy_ptr(y.data_ptr(), verts.data_ptr(), gy.data_ptr(), gv.data_ptr())
        reps = 5
        es.record(stream)
        for _ in range(reps):
            tb.energy_ptr(y.data_ptr(), verts.data_ptr(), gy.data_ptr(), gv.data_ptr())
        ee.record(stream)
        torch.cuda.synchronize()
        extras["energy"] = {"relax_energy": {"value": e_relax, "unit": "particle-iterations/s",
                                             "iterations": Ge, "form": "plain, both bodies"},
                            "energy_and_backward_ms": es.elapsed_time(ee) / reps,
                            "backward_workload": f"torus body, {tb.n} particles, {len(ta.verts)} vertices: "
                                                 "E, dE/dy and dE/dverts through the frozen surface projection"}

        # ---- 64 bodies of uneven size with gear-shaft unions: batched + graph
        # against plain (single bodies one by one, each union as a 2-body
        # batch, no graph) ------------------------------------------------------
        basm = W.batch_union_workload(seed=3 + 10 * rank)
        bbodies = [pkg.Body.from_assembly(a, stream=stream) for a in basm]
        upairs = [(i, a.meta["union_with"]) for i, a in enumerate(basm) if a.meta.get("union_with", -1) > i]
        for i, j in upairs:
            pkg.union(bbodies[i], bbodies[j])
        in_pair = {k for p in upairs for k in p}
        singles = [b for k, b in enumerate(bbodies) if k not in in_pair]
        pair_batches = [pkg.Batch([bbodies[i], bbodies[j]], stream=stream) for i, j in upairs]
        nb = sum(b.n for b in bbodies)
        snap = [b.get_particles() for b in bbodies]

        def reset_bodies():
            for b, (x, c, cons) in zip(bbodies, snap):
                b.set_particles(x, c)
                b.set_constraints(cons)

        bb = pkg.Batch(bbodies, stream=stream)
        btuned = bb.autotune(G)
        bb.set_graph_iters(G)
        kb = 3
        ms_bb, ms_bp = [], []
        for _ in range(kb + 1):
            bb.load()
            flush.zero_()
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            bb.relax(G, use_graph=True)
            e_.record(stream)
            torch.cuda.synchronize()
            ms_bb.append(s_.elapsed_time(e_))
            reset_bodies()
            for pb in pair_batches:
                pb.load()
            flush.zero_()
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            for b in singles:
                b.relax(G)
            for pb in pair_batches:
                pb.relax(G, use_graph=False)
            e_.record(stream)
            torch.cuda.synchronize()
            ms_bp.append(s_.elapsed_time(e_))
            reset_bodies()
        vb = nb * G * kb / (sum(ms_bb[1:]) / 1e3)
        vp = nb * G * kb / (sum(ms_bp[1:]) / 1e3)
        bb.time_force(True)
        bb.load()
        bb.relax(G, use_graph=True)
        bphases = bb.phase_ms()
        bb.time_force(False)
        extras["batch64"] = {"workload": "64 bodies (cubes, cylinders, icospheres, gears; scales 0.1-1), dx=0.008, "
                                         f"{len(upairs)} gear-shaft Boolean unions",
                             "particles": nb, "iterations_per_step": G, "steps": kb, "warmup": 1,
                             "batched_graph": vb, "plain": vp, "batched_over_plain": vb / vp,
                             "unit": "particle-iterations/s", "autotune": btuned,
                             "phase_ms_per_iteration": bphases,
                             "launches_per_iteration": {"batched": bb.kernels_per_iter,
                                                        "plain": bb.kernels_per_iter * (len(singles) +
                                                                                        len(pair_batches))}}
        bb.close()
        for pb in pair_batches:
            pb.close()

    peaks, peak_kind = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = SMS * FP32_LANES * 2 * sm_max * 1e6 / 1e12     # TFLOP/s, FMA = 2
    flops = 8.0 * cand + 12.0 * pairs                           # per force launch (all bodies)
    achieved = flops / (force_ms / 1e3) / 1e12
    executed = (8.0 * tested + 12.0 * pairs) / (force_ms / 1e3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    useful_gbs = 56.0 * value / world / 1e9
    line = {
        "metric": "relaxation particle-iterations/s",
        "value": value, "unit": "particle-iterations/s", "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": tot_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"icosphere_l5+torus_256x64 dx={args.dx}", "bodies": len(asm), "particles": n,
                   "iterations_per_step": G, "form": "batched + CUDA graph",
                   "l2": "flushed between steps (256 MiB write), working set < L2"},
        "roofline": {"bound": "alu", "kernel": "k_force", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": K_FORCE_DRAM_BYTES.get(round(args.dx, 6)),
                     "peak_kind": f"FP32 {SMS} SMs x {FP32_LANES} lanes x 2 x {sm_max:.0f} MHz ({peak_kind} clock)",
                     "flops_per_launch": flops, "candidates": cand, "pairs": pairs, "force_ms": force_ms,
                     "tested": tested, "executed_TFLOPs": executed, "executed_frac": executed / fp32_peak},
        "hbm": {"useful_bytes_per_particle_iteration": 56, "useful_GBps": useful_gbs,
                "frac_of_measured": useful_gbs / hbm},
        "phase_ms_per_iteration": {**phases, "note": "one extra replay with event records in the graph"},
        "gpu_launches": kpi * G * K,
        "autotune": tuned,
        "clocks": clk,
    }
    line.update(extras)
    if not args.no_extras and rank == 0:
        cpu_v, cores, dt = cpu_oracle(asm, 1)
        line["cpu_baseline"] = {"value": cpu_v, "unit": "particle-iterations/s", "cores": cores, "kind": "oracle",
                                "sample": f"one FP64 iteration of both bodies ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
