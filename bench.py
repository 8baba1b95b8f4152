#!/usr/bin/env python
"""Throughput of the FPPG relaxation path on GB300: particle-iterations/s.

Workload (default, ``--workload vehicle``): the vehicle-like closed shell --
union of two rounded boxes and four wheel cylinders as a signed-distance
field, surface nets and two Loop subdivision steps (2,009,344 triangles),
seeded 1e-3 vertex noise, 30 degree features -- at dx = 0.0068, h = 1.3 dx,
with its initial particles (19.2 M feature, surface and volume particles)
generated on the GPU by the method's own generation (Sec. 3.2).  A step is
one replay of a 50-iteration CUDA graph of the batched form (every phase of
an iteration is one launch); K = 20 steps are the workload's 1000
iterations.  The working set (~2.4 GB of particle state) is larger than L2;
L2 is also flushed (a 256 MiB write) between steps, outside the timed
events.  ``--workload sphere_torus`` times the icosphere + torus pair at
dx = 0.02 (777 k particles) instead.

Reported beside it: the plain form (the body relaxed with its own launches,
no graph), the end-to-end number through the C ABI with host buffers (pinned
host -> device copy of the particles and their constraints, relaxation,
device -> host copy of the positions, every step), the force kernel against
the FP32 ALU roofline (lane instructions per candidate and per pair against
SMs x 128 lanes x clock), and the FP64 CPU oracle on the host cores on a
bounded crop of the same workload.  ``--impl reference`` times the oracle
alone (the CPU program the GPU path is checked against).
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
FP32_LANES = 128                  # FP32 lanes per SM (the SM count is read from the device)
# FP32 lane instructions of the force pass (Eq. 15): per candidate of the
# 27-cell search set (difference, squared distance, compare) and per
# accepted pair (root, Wendland C2 gradient, accumulation)
INSTR_PER_CANDIDATE, INSTR_PER_PAIR = 7.0, 25.0
# FP32 flops of the same (FMA = 2): 8 per candidate, 12 per accepted pair
FLOPS_PER_CANDIDATE, FLOPS_PER_PAIR = 8.0, 12.0
# DRAM bytes (read + write) of one k_force launch, from one ncu capture per
# workload of the current kernel (null until captured)
K_FORCE_DRAM_BYTES = {"sphere_torus": 26987520 + 6400, "vehicle": 653986304 + 286342400}
# bytes per particle-iteration: state in and out plus the mandated cell-list
# rebuild (useful), and the compulsory traffic of the whole pipeline
USEFUL_BYTES, PIPELINE_BYTES = 56.0, 224.0


def workload(name, rank=0, dx=0.02):
    """(assemblies, description) of a named workload; weak scaling gives each
    rank its own seeded copy."""
    from paper_2501_03056_gb300 import workloads as W
    if name == "vehicle":
        return W.vehicle_workload(), ("vehicle shell: rounded boxes + 4 wheels, surface nets + 2 Loop "
                                      "steps, 2,009,344 triangles, 1e-3 noise, 30 deg features, dx=0.0068, "
                                      "particles generated on the GPU (Sec. 3.2)")
    if name == "sphere_torus":
        return (W.sphere_torus_workload(seed=1 + 10 * rank, dx=dx),
                f"icosphere_l5+torus_256x64 dx={dx}")
    raise ValueError(name)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="vehicle", choices=["vehicle", "sphere_torus"])
    p.add_argument("--iters-per-step", type=int, default=50)
    p.add_argument("--dx", type=float, default=0.02, help="dx of the sphere_torus workload")
    p.add_argument("--no-extras", action="store_true", help="skip plain / e2e / CPU legs")
    p.add_argument("--no-autotune", action="store_true", help="keep the default kernel configuration")
    p.add_argument("--config", default=None,
                   help="force variant,block,search CTAs per SM[,incremental order 0/1[,row order 0/1]] "
                        "(e.g. 0,128,4,1) instead of the autotuner")
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


def oracle_crop(asm, frac):
    """FP64 oracle bodies on a bounded crop of the workload: every body with
    its full mesh and features, particles cut to the `frac` of each body
    with the smallest x (the oracle's own generation where the workload
    generates its particles).  Returns (bodies, particles, description)."""
    import oracle
    bodies, n = [], 0
    for a in asm:
        o = oracle.from_assembly(a)
        if frac < 1.0:
            x, _, _ = o.get_particles()
            keep = x[:, 0] <= np.quantile(x[:, 0], frac)
            oracle.keep_rows(o, keep)
        n += o.n
        bodies.append(o)
    return bodies, n, f"the {100 * frac:g} % of particles with the smallest x of each body, full meshes"


def cpu_baseline_leg(asm, workload):
    """The FP64 oracle on the host cores, on a bounded crop of the workload
    (about 10 s of CPU work), then on one thread on the 1/16 of that crop
    with the smallest x (the reference point of the paper's thread
    scaling, a few seconds)."""
    import oracle
    frac = 1.0 / 16 if workload == "vehicle" else 1.0
    obodies, on, sample = oracle_crop(asm, frac)
    iters = 30 if workload == "vehicle" else 1   # about 10 s of CPU work
    cores = oracle.get_threads()
    t0 = time.perf_counter()
    for o in obodies:
        o.relax(iters)
    dt = time.perf_counter() - t0
    out = {"value": on * iters / dt, "unit": "particle-iterations/s", "cores": cores, "kind": "oracle",
           "sample": f"{iters} FP64 iterations of {sample} ({on} particles, {dt:.1f} s)"}
    for o in obodies:
        x, _, _ = o.get_particles()
        if len(x):
            oracle.keep_rows(o, x[:, 0] <= np.quantile(x[:, 0], 1.0 / 16))
    n1 = sum(o.n for o in obodies)
    iters1 = 10 if workload == "vehicle" else 1
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        for o in obodies:
            o.relax(iters1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    one = n1 * iters1 / dt1
    out["single_thread"] = {"value": one, "unit": "particle-iterations/s", "cores": 1,
                            "sample": f"{iters1} FP64 iterations of the 1/16 of that crop with the smallest x "
                                      f"({n1} particles, {dt1:.1f} s)",
                            "cores_over_one": out["value"] / one}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    asm, desc = workload(args.workload, 0, args.dx)
    frac = 1.0 / 16 if args.workload == "vehicle" else 1.0
    bodies, n, sample = oracle_crop(asm, frac)
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
        "config": {"workload": desc, "bodies": len(asm), "particles": n, "iterations_per_step": 1,
                   "form": "FP64 CPU oracle, one iteration per step (bounded sample)", "sample": sample},
        "cpu_baseline": {"value": value, "unit": "particle-iterations/s", "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": f"one FP64 iteration per step of {sample}"},
        "e2e": {"value": value, "unit": "particle-iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def force_roofline(cand, pairs, tested, force_ms, sms, sm_mhz, peak_kind, traffic):
    """ALU roofline of the force pass: FP32 lane instructions per launch
    (7 per candidate of the 27-cell set + 25 per accepted pair) against
    SMs x 128 lanes x clock, with the flop form beside it."""
    lane_peak = sms * FP32_LANES * sm_mhz * 1e6 / 1e12                     # T lane-instr/s
    instr = INSTR_PER_CANDIDATE * cand + INSTR_PER_PAIR * pairs
    achieved = instr / (force_ms / 1e3) / 1e12
    flop_peak = 2.0 * lane_peak
    flops = FLOPS_PER_CANDIDATE * cand + FLOPS_PER_PAIR * pairs
    flops_exec = FLOPS_PER_CANDIDATE * tested + FLOPS_PER_PAIR * pairs
    return {"bound": "alu", "kernel": "k_force", "achieved": achieved, "peak": lane_peak,
            "unit": "T FP32 lane-instructions/s", "frac": achieved / lane_peak, "traffic": traffic,
            "peak_kind": f"{sms} SMs (from the device) x {FP32_LANES} FP32 lanes x {sm_mhz:.0f} MHz ({peak_kind} "
                         "max clock)",
            "lane_instructions_per_launch": instr, "candidates": cand, "pairs": pairs, "tested": tested,
            "tested_per_pair": tested / max(pairs, 1), "force_ms": force_ms,
            "flop_form": {"achieved_TFLOPs": flops / (force_ms / 1e3) / 1e12, "peak_TFLOPs": flop_peak,
                          "frac": flops / (force_ms / 1e3) / 1e12 / flop_peak,
                          "executed_frac": flops_exec / (force_ms / 1e3) / 1e12 / flop_peak}}


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
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peaks, peak_kind = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sms = pkg.device_sm_count()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def make_bodies(asm):
        """Bodies of the assemblies (generated on the GPU where the workload
        carries no particles) and a host snapshot of their initial state."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bodies = [pkg.Body.from_assembly(a, stream=stream) for a in asm]
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        snap = [b.get_particles() for b in bodies]
        return bodies, snap, gen_s

    def reset(bodies, snap):
        for b, (x, c, cons) in zip(bodies, snap):
            b.set_particles(x, c)
            b.set_constraints(cons)

    def timed(step_fn, reset_fn, steps, warm):
        """Device ms of `steps` steps after `warm` warm-up steps, the state
        reset before each group, L2 flushed before each step (outside the
        events)."""
        reset_fn()
        for _ in range(warm):
            step_fn()
        reset_fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        for s, e in ev:
            flush.zero_()
            s.record(stream)
            step_fn()
            e.record(stream)
        barrier()
        return [s.elapsed_time(e) for s, e in ev]

    def measure(asm, desc, steps, warm, tune=True, config=None, with_plain=False, plain_steps=2, clocks=None):
        """Batched + graph form of a workload (autotuned), its live phase
        times, work counts and force roofline; optionally the plain form."""
        bodies, snap, gen_s = make_bodies(asm)
        n = sum(b.n for b in bodies)
        cand = pairs = tested = 0
        for b in bodies:
            c, p, t = b.work_counts()
            cand += c
            pairs += p
            tested += t
        batch = pkg.Batch(bodies, stream=stream)
        if config:
            vals = [int(x) for x in config.split(",")]
            v, tb, sc = vals[:3]
            batch.configure(v, tb, sc)
            tuned = {"force_variant": v, "force_block": tb, "search_ctas_per_sm": sc, "fixed": True}
            if len(vals) > 3:
                batch.set_incremental(bool(vals[3]))
                tuned["incremental_order"] = vals[3]
            if len(vals) > 4:
                batch.set_cell_order(vals[4])
                tuned["cell_order"] = vals[4]
        else:
            tuned = batch.autotune(G) if tune else None     # trials as long as a timed step
        batch.set_graph_iters(G)
        if clocks:
            clocks.start()
        ms = timed(lambda: batch.relax(G, use_graph=True), batch.load, steps, warm)
        clk = clocks.stop() if clocks else None
        # one more replay, with CUDA event records around the phases of every
        # iteration captured into the graph: live per-phase device times
        batch.time_force(True)
        batch.load()
        batch.relax(G, use_graph=True)
        phases = batch.phase_ms()
        batch.time_force(False)
        r = {"bodies": bodies, "snap": snap, "batch": batch, "n": n, "ms": ms, "phases": phases, "tuned": tuned,
             "clocks": clk, "cand": cand, "pairs": pairs, "tested": tested, "gen_s": gen_s,
             "value": n * G * steps / (sum(ms) / 1e3), "desc": desc}
        if with_plain:
            pms = timed(lambda: [b.relax(G) for b in bodies], lambda: reset(bodies, snap), plain_steps, 1)
            r["plain"] = n * G * plain_steps / (sum(pms) / 1e3)
            r["plain_ms"] = sum(pms) / plain_steps
        return r

    # ---- the headline: batched form, CUDA graph of G iterations ----------------
    asm, desc = workload(args.workload, rank, args.dx)
    clocks = Clocks(local)
    H = measure(asm, desc, K, Wm, tune=not args.no_autotune, config=args.config, clocks=clocks)
    n, batch, bodies = H["n"], H["batch"], H["bodies"]
    tot_ms = max_over_ranks(sum(H["ms"]))
    value = n * world * G * K / (tot_ms / 1e3)
    kpi = batch.kernels_per_iter
    roof = force_roofline(H["cand"], H["pairs"], H["tested"], H["phases"]["force"], sms, sm_max, peak_kind,
                          K_FORCE_DRAM_BYTES.get(args.workload))
    it_ms = tot_ms / K / G
    line = {
        "metric": "relaxation particle-iterations/s",
        "value": value, "unit": "particle-iterations/s", "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": tot_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "bodies": len(asm), "particles": n, "iterations_per_step": G,
                   "iterations": G * K, "form": "batched + CUDA graph",
                   "l2": "working set larger than L2; L2 also flushed between steps (256 MiB write)"
                         if args.workload == "vehicle" else
                         "flushed between steps (256 MiB write), working set < L2"},
        "roofline": roof,
        "hbm": {"useful_bytes_per_particle_iteration": USEFUL_BYTES,
                "useful_GBps": USEFUL_BYTES * value / world / 1e9,
                "frac_of_measured": USEFUL_BYTES * value / world / 1e9 / hbm,
                "pipeline_bytes_per_particle_iteration": PIPELINE_BYTES,
                "pipeline_GBps": PIPELINE_BYTES * value / world / 1e9,
                "pipeline_frac_of_measured": PIPELINE_BYTES * value / world / 1e9 / hbm,
                "peak_GBps": hbm, "peak_kind": peak_kind},
        "phase_ms_per_iteration": {**H["phases"], "whole_iteration": it_ms,
                                   "note": "one extra replay with event records in the graph"},
        "gpu_launches": kpi * G * K,
        "kernels_per_iteration": kpi,
        "autotune": H["tuned"],
        "clocks": H["clocks"],
    }

    if not args.no_extras:
        # ---- plain form of the headline workload: no graph, own launches ------
        snap = H["snap"]
        ps = min(K, 4)
        pms = timed(lambda: [b.relax(G) for b in bodies], lambda: reset(bodies, snap), ps, 1)
        plain_value = n * G * ps / (sum(pms) / 1e3)
        line["plain"] = {"value": plain_value, "unit": "particle-iterations/s", "ms_per_step": sum(pms) / ps,
                         "steps": ps, "launches_per_iteration": kpi * len(bodies), "graph": False}
        line["batched_over_plain"] = value / world / plain_value

        # ---- end to end through the C ABI with host buffers ------------------
        pinned = [(torch.from_numpy(np.ascontiguousarray(x)).pin_memory(),
                   torch.from_numpy(np.ascontiguousarray(c)).pin_memory(),
                   torch.from_numpy(np.ascontiguousarray(cons)).pin_memory(),
                   torch.empty((len(x), 3), dtype=torch.float32).pin_memory()) for x, c, cons in snap]

        def e2e_step():
            for b, (x, c, cons, _) in zip(bodies, pinned):
                b.set_particles(x.numpy(), c.numpy())
                b.set_constraints(cons.numpy())
            batch.load()
            batch.relax(G, use_graph=True)
            batch.store()
            for b, (_, _, _, out) in zip(bodies, pinned):
                b.get_positions_into(out.numpy())

        for _ in range(Wm):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            e2e_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        line["e2e"] = {"value": n * world * G * K / e2e_s, "unit": "particle-iterations/s",
                       "h2d_bytes_per_step": int(n * 20), "d2h_bytes_per_step": int(n * 12),
                       "copies": "xyz (12 B) + class (4 B) + constraint (4 B) in, xyz (12 B) out, per particle"}
        line["generation_headline"] = {"particles": n, "seconds": H["gen_s"],
                                       "what": "mesh build, feature extraction and fppg_map_particles of the "
                                               "headline workload (host wall clock around synchronised calls)"}
        batch.close()

        # ---- the icosphere + torus workload as its own leg ------------------------
        if args.workload != "sphere_torus":
            st_asm, st_desc = workload("sphere_torus", rank, 0.02)
            S2 = measure(st_asm, st_desc, 10, 3, with_plain=True, plain_steps=4)
            line["sphere_torus"] = {
                "workload": st_desc, "particles": S2["n"], "iterations_per_step": G, "steps": 10,
                "batched_graph": S2["value"], "plain": S2["plain"], "batched_over_plain": S2["value"] / S2["plain"],
                "unit": "particle-iterations/s", "autotune": S2["tuned"], "phase_ms_per_iteration": S2["phases"],
                "roofline": force_roofline(S2["cand"], S2["pairs"], S2["tested"], S2["phases"]["force"], sms,
                                           sm_max, peak_kind, K_FORCE_DRAM_BYTES["sphere_torus"])}
            st_bodies = S2["bodies"]
            S2["batch"].close()
        else:
            st_asm, st_bodies = asm, bodies

        # ---- the other configurations at full size: batched + graph and plain ---
        def config_leg(casm, steps=2):
            R = measure(casm, "", steps, 1, with_plain=True, plain_steps=steps)
            R["batch"].close()
            for b in R["bodies"]:
                b.close()
            return {"particles": R["n"], "iterations_per_step": G, "steps": steps, "warmup": 1,
                    "batched_graph": R["value"], "plain": R["plain"], "batched_over_plain": R["value"] / R["plain"],
                    "unit": "particle-iterations/s", "autotune": R["tuned"], "phase_ms_per_iteration": R["phases"]}

        line["configs"] = {
            "unit cube (12 triangles, dx=0.05)": config_leg(W.cube_workload()),
            "spur gear (51,840 triangles, dx=0.004, generated)": config_leg(W.gear_workload()),
        }

        # ---- generation (Sec. 3.2) on the GPU: the spur gear ------------------
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
        line["generation"] = {"workload": f"spur gear, {len(ga.tris)} triangles, dx={ga.dx:g}, band 2 + inner 1 cells",
                              "particles": gn, "mesh_build_ms": 1e3 * (t1 - t0),
                              "features_ms": 1e3 * (t2 - t1), "map_particles_ms": 1e3 * (t3 - t2),
                              "particles_per_s": gn / (t3 - t2), "timer": "host wall clock around synchronised calls"}
        gb.close()

        # ---- the paper's sphere at ~1e8 particles: generation and relaxation --
        sa = W.sphere_1e8_workload()[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sb = pkg.Body(sa.verts, sa.tris, sa.dx, sa.h, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sb.extract_features(sa.dihedral_deg)
        sn = sb.map_particles(**sa.meta["generate"])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        sbatch = pkg.Batch([sb], stream=stream)
        tu = H["tuned"] or {}
        if "force_variant" in tu:       # the headline's tuned configuration (no trials at this size)
            sbatch.configure(tu["force_variant"], tu["force_block"], tu["search_ctas_per_sm"])
            sbatch.set_incremental(bool(tu.get("incremental_order", 0)))
        sbatch.set_graph_iters(G)
        sms_1e8 = timed(lambda: sbatch.relax(G, use_graph=True), sbatch.load, 2, 1)
        line["scale_1e8"] = {
            "workload": f"sphere 1x1x1 (icosphere level 7, {len(sa.tris)} triangles), dx={sa.dx:g}, surface + every "
                        "interior cell (Sec. 3.2)",
            "particles": sn, "mesh_build_ms": 1e3 * (t1 - t0), "features_and_map_ms": 1e3 * (t2 - t1),
            "generated_particles_per_s": sn / (t2 - t1),
            "relax": {"iterations_per_step": G, "steps": 2, "ms_per_step": sum(sms_1e8) / 2,
                      "value": sn * G * 2 / (sum(sms_1e8) / 1e3), "unit": "particle-iterations/s",
                      "configuration": "the headline's autotuned one"},
            "timer": "generation: host wall clock around synchronised calls; relaxation: CUDA events"}
        sbatch.close()
        sb.close()

        # ---- energy (A8): energy-descent relaxation and the backward ------------
        for b, a in zip(st_bodies, st_asm):
            b.set_particles(a.xyz, a.cls)
        st_n = sum(b.n for b in st_bodies)
        Ge = 10
        for b in st_bodies:
            b.relax_energy(1)
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for b in st_bodies:
            b.relax_energy(Ge)
        ee.record(stream)
        torch.cuda.synchronize()
        e_relax = st_n * Ge / (es.elapsed_time(ee) / 1e3)
        tb, ta = st_bodies[1], st_asm[1]                # the torus: surface particles through the projection
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
        line["energy"] = {"relax_energy": {"value": e_relax, "unit": "particle-iterations/s",
                                           "iterations": Ge, "form": "plain, icosphere + torus"},
                          "energy_and_backward_ms": es.elapsed_time(ee) / reps,
                          "backward_workload": f"torus body, {tb.n} particles, {len(ta.verts)} vertices: "
                                               "E, dE/dy and dE/dverts through the frozen surface projection"}
        for b in st_bodies:
            b.close()

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
        bsnap = [b.get_particles() for b in bbodies]
        bb = pkg.Batch(bbodies, stream=stream)
        btuned = bb.autotune(G)
        bb.set_graph_iters(G)
        kb = 3

        def plain64():
            for pb in pair_batches:
                pb.load()
            for b in singles:
                b.relax(G)
            for pb in pair_batches:
                pb.relax(G, use_graph=False)

        ms_bb = timed(lambda: bb.relax(G, use_graph=True), bb.load, kb, 1)
        ms_bp = timed(plain64, lambda: reset(bbodies, bsnap), kb, 1)
        vb = nb * G * kb / (sum(ms_bb) / 1e3)
        vp = nb * G * kb / (sum(ms_bp) / 1e3)
        bb.time_force(True)
        bb.load()
        bb.relax(G, use_graph=True)
        bphases = bb.phase_ms()
        bb.time_force(False)
        line["batch64"] = {"workload": "64 bodies (cubes, cylinders, icospheres, gears; scales 0.1-1), dx=0.008, "
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
        for b in bbodies:
            b.close()
    else:
        batch.close()

    if not args.no_extras and rank == 0:
        line["cpu_baseline"] = cpu_baseline_leg(asm, args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for b in bodies:
        b.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
