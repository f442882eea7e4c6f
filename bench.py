"""Benchmark of the coupled LB-MD step (one JSON line on stdout).

A step is one coupled lattice-Boltzmann / molecular-dynamics step of the whole
hot path: particle kernel (gather, MD cycle, spread) concurrently with the
fused stream-collide kernel, then the source pass.  The metric is MLUPS
(million lattice-site updates per second, all nx*ny*nz*n_real sites counted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl native|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
(its own seed); value = all ranks' site updates / max-over-ranks time
(weak scaling, no data-path collective).

Timing: each timed step is bracketed by CUDA events on the library's stream;
between timed steps a 256 MiB buffer is written to flush the 129 MB L2 (the
populations of the default workload, 2 x 40 MB, would otherwise stay in L2).
The roofline object reports the stream-collide kernel: algorithmic bytes
(19 x 4 B read + 19 x 4 B written per site in FP32, half that in FP16)
over its CUDA-event duration, against the measured HBM copy bandwidth.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import tempfile
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _traffic_record(sites: int):
    """DRAM bytes per launch of the stream-collide kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "stream_collide_traffic.json")
    src = os.path.join(ROOT, "paper_0711_2665_gb300", "csrc", "k_fluid.cu")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("k_fluid_sha256") != sha:
        return None
    return rec["dram_bytes_per_site"] * sites


class ClockSampler:
    """nvidia-smi samples every 20 ms while the timed regions run; entering
    waits (at most 3 s) for the first sample, so that sampling covers them."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"lbmd_clocks_{self.gpu}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            t_end = time.perf_counter() + 3.0
            while time.perf_counter() < t_end and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
            if self.path:
                self.fh.close()
                os.unlink(self.path)
                self.path = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _config_block(w, flush):
    return {"workload": w["name"], "lattice": [w["nx"], w["ny"], w["nz"]],
            "n_real": w.get("full_n_real", w["n_real"]),
            "beads": w["n_beads"], "tau": w["tau"], "precision": w["precision"],
            "md_substeps": [w["md_outer"], w["md_inner"]], "kappa_bend": w["kappa_bend"],
            "l2": ("flushed before every timed launch (256 MiB written, 256 MiB read); a launch is a "
                   "2-step graph") if flush else "inputs larger than L2",
            "parallelism": "realizations split across ranks" if "shard" in w else "replicas"}


def run_reference(args, w, world, rank):
    """The oracle (FP64, plain C, one host thread) on the same workload; each
    step is one oracle LB-MD step of realization 0."""
    if rank != 0:
        return
    import oracle
    from paper_0711_2665_gb300 import workloads
    oracle.build()
    inp = workloads.build_inputs(w)
    o1 = int(inp["offsets"][1])
    orc = oracle.OracleSim(workloads.oracle_params(w, 0, o1), inp["solid"])
    orc.set_beads(inp["r0"][:o1])
    for _ in range(args.warmup):
        orc.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(1)
    dt = time.perf_counter() - t0
    sites = w["nx"] * w["ny"] * w["nz"]
    mlups = sites * args.steps / dt / 1e6 * w["n_real"] / w["n_real"]
    sample = f"{args.steps} oracle steps of realization 0 ({sites} sites, {o1} beads)"
    line = {"impl": "reference", "metric": "coupled LB-MD MLUPS", "value": mlups, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config_block(w, False),
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, budget_s=15.0):
    """Oracle timed on a bounded sample of the workload (whole LB-MD steps of
    realization 0) on one host core."""
    import oracle
    from paper_0711_2665_gb300 import workloads
    oracle.build()
    inp = workloads.build_inputs(w)
    o1 = int(inp["offsets"][1])
    orc = oracle.OracleSim(workloads.oracle_params(w, 0, o1), inp["solid"])
    orc.set_beads(inp["r0"][:o1])
    orc.step(1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or n < 2:
        orc.step(1)
        n += 1
    dt = time.perf_counter() - t0
    sites = w["nx"] * w["ny"] * w["nz"]
    return {"value": sites * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{n} FP64 oracle steps of realization 0 ({sites} sites, {o1} beads), {dt:.1f} s"}


def _sc_roofline(sim, w, peak, peak_kind, steps=10):
    """Stream-collide roofline from per-launch CUDA events over a few eager
    steps: inside the step (sharing the GPU with the particle kernel) and
    alone (the particle kernel waited for); achieved/frac are the latter."""
    sites = w["nx"] * w["ny"] * w["nz"] * w["n_real"]
    b = (152 if w["precision"] == "fp32" else 76) * sites
    us = {}
    for overlap in (True, False):
        sim.set_overlap(overlap)
        sim.profile(True)
        sim.step(steps)
        kt = sim.kernel_times()
        sim.profile(False)
        n, ms = kt["stream_collide"]
        us["in_step" if overlap else "alone"] = 1e3 * ms / n
    sim.set_overlap(True)
    achieved = b / (us["alone"] * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "kernel": "k_stream_collide", "algorithmic_bytes_per_launch": b,
            "us_per_launch_alone": us["alone"], "us_per_launch_in_step": us["in_step"],
            "frac_in_step": b / (us["in_step"] * 1e-6) / 1e9 / peak}


def _variants(dev, lbmd, workloads, tiles, steps=100):
    """The method's variants on the headline workload (128x64x64, N = 400),
    each timed like the headline (2-step graph launches, L2 flushed before
    every launch), beside the default form: stochastic position Verlet
    (integrator 1), nearest-grid-point coupling (interp 1), both (the paper's
    own scheme), and the fluctuating fluid (lb_kT = kT = 1e-4)."""
    import torch
    flush_w = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    flush_r = torch.ones(64 << 20, dtype=torch.float32, device=dev)
    res = {}
    for name, ov in (("default", {}), ("spv", {"integrator": 1}), ("ngp", {"interp": 1}),
                     ("ngp_spv", {"interp": 1, "integrator": 1}), ("fluctuating", {"lb_kT": 1e-4})):
        w = workloads.get("plain_fp32", **ov)
        inp = workloads.build_inputs(w)
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=str(dev))
        if tiles:
            sim.set_tiles(*tiles)
        else:
            sim.autotune(8)
        st = sim.stream
        sim.set_graph(2)
        sim.step(6)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps // 2)]
        torch.cuda.synchronize(dev)
        for a, b in ev:
            with torch.cuda.stream(st):
                flush_w.zero_()
                flush_r.sum()
            a.record(st)
            sim.step(2)
            b.record(st)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / (2 * len(ev))
        sim.set_graph(0)
        sim.profile(True)
        sim.step(10)
        kt = sim.kernel_times()
        sim.profile(False)
        sim.check()
        sites = w["nx"] * w["ny"] * w["nz"]
        res[name] = {"value": sites / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
                     "us_particles": 1e3 * kt["particles"][1] / kt["particles"][0],
                     "us_stream_collide": 1e3 * kt["stream_collide"][1] / kt["stream_collide"][0],
                     "config": ov}
        sim.close()
    return res


def extra_measurements(dev, stream, peak, peak_kind, forms, tiles=None):
    """The other forms of the step, each timed on its own workload with CUDA
    events on the library's stream (inputs larger than L2, no flush needed):
    the batched ensemble and the FP16-deviation storage, each run of K steps
    one launch of the device-side step-loop graph, and the reverse sweep
    (forward + checkpointed adjoint of 200 steps)."""
    import numpy as np
    import torch
    from paper_0711_2665_gb300 import lbmd, workloads
    out = {}

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) * 1e-3

    # fp32_matched: the FP16 form's workload (256x128x128, N = 1000) stored in
    # FP32, the plain step at the 4.19 M sites of the ensemble and FP16 forms
    for name, K in (("ensemble_fp32", 100), ("fp16dev", 60), ("fp32_matched", 60)):
        if name not in forms:
            continue
        w = workloads.get("fp16dev", precision="fp32") if name == "fp32_matched" else workloads.get(name)
        inp = workloads.build_inputs(w)
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=str(dev))
        if tiles:
            sim.set_tiles(*tiles)
            by, zc = tiles
        else:
            by, zc = sim.autotune(8)
        sim.step_loop(20)  # captures the device-side loop graph
        t = timed(lambda: sim.step_loop(K))
        sites = w["nx"] * w["ny"] * w["nz"] * w["n_real"]
        rf = _sc_roofline(sim, w, peak, peak_kind)
        sim.check()
        out[name] = {"value": sites * K / t / 1e6, "unit": "MLUPS", "ms_per_step": 1e3 * t / K,
                     "steps_per_s": K / t, "realization_steps_per_s": K * w["n_real"] / t, "steps": K,
                     "lattice": [w["nx"], w["ny"], w["nz"]], "n_real": w["n_real"], "beads": int(inp["offsets"][-1]),
                     "precision": w["precision"], "tiles": [by, zc], "md_shape": list(sim.md_shape()), "md_exchange": sim.md_exchange(),
                     "md_bonded": sim.md_bonded(), "md_reserve": sim.md_reserve(),
                     "launch": "one CUDA-graph launch per run (device-side loop of two-step bodies)",
                     "roofline": rf}
        sim.close()
    if "fp32_matched" in out:
        base = out["fp32_matched"]["value"]
        out["speedups_vs_fp32_matched"] = {
            k: out[k]["value"] / base for k in ("ensemble_fp32", "fp16dev") if k in out}
    if "variants" in forms:
        out["variants"] = _variants(dev, lbmd, workloads, tiles)
    if "adjoint" not in forms:
        return out
    w = workloads.get("adjoint")
    inp = workloads.build_inputs(w)
    K, C = w["steps"], w["checkpoint_every"]
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=str(dev))
    if tiles:
        sim.set_tiles(*tiles)
    else:
        sim.autotune(8)
    sim.step(4)
    t_fwd = timed(lambda: sim.step(K))
    sim2 = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=str(dev))
    sim2.set_tiles(*sim.tiles())
    sim2.adjoint(K, C)  # warm-up: first launches, and the scratch block the timed call reuses
    sim3 = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=str(dev))
    sim3.set_tiles(*sim.tiles())
    res = {}
    t_adj = timed(lambda: res.update(sim3.adjoint(K, C)))
    sites = w["nx"] * w["ny"] * w["nz"]
    out["adjoint"] = {"value": K / t_adj, "unit": "steps/s", "forward_steps_per_s": K / t_fwd,
                      "ratio_to_forward": t_adj / t_fwd, "K": K, "checkpoint_every": C,
                      "lattice": [w["nx"], w["ny"], w["nz"]], "beads": int(inp["offsets"][-1]),
                      "mlups_equivalent": sites * K / t_adj / 1e6,
                      "grad_finite": bool(np.all(np.isfinite(res["dr0"]))),
                      "note": "forward sweep with checkpoints, segment replay recording the MD trajectory, and the "
                              "adjoint kernels; gradients of the centre-of-mass displacement w.r.t. gamma, E, r0"}
    for s_ in (sim, sim2, sim3):
        s_.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="plain_fp32")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="ensemble_fp32,fp16dev,fp32_matched,variants,adjoint",
                    help="comma list of the other forms to measure (ensemble_fp32, fp16dev, fp32_matched, "
                         "variants, adjoint), or none")
    ap.add_argument("--tiles", type=int, nargs=2, metavar=("BY", "ZC"), default=None,
                    help="fixed stream-collide tile shape instead of the autotuner (for profiling runs)")
    ap.add_argument("--md-shape", type=int, nargs=2, metavar=("T", "C"), default=None,
                    help="with --tiles: lanes per bead and blocks per chain of the particle kernel")
    ap.add_argument("--md-exchange", choices=["push", "pull"], default=None,
                    help="with --tiles: the particle kernel's chain exchange")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_0711_2665_gb300 import dist as pdist, workloads
    world, rank, local = pdist.env()
    # one lattice: every rank runs a replica with its own seed; an ensemble:
    # each rank runs its block of realizations (same noise streams as unsplit)
    w_full = workloads.get(args.workload)
    w = pdist.rank_workload(w_full, rank, world)

    if args.impl == "reference":
        return run_reference(args, w, world, rank)

    import numpy as np
    import torch
    from paper_0711_2665_gb300 import build as libbuild, lbmd

    libbuild.build_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    inp = pdist.rank_inputs(w, workloads.build_inputs)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=f"cuda:{local}")
    if args.tiles:
        sim.set_tiles(*args.tiles)
        if args.md_shape:
            sim.set_md_shape(*args.md_shape)
        if args.md_exchange:
            sim.set_md_exchange(args.md_exchange)
    else:
        sim.autotune(8)
    sites = w["nx"] * w["ny"] * w["nz"] * w["n_real"]
    flush = not args.no_flush
    # L2 flush between timed steps: write 256 MiB, then read another 256 MiB so
    # that the L2 ends up holding clean lines (the written lines' write-backs
    # happen during the read, not inside the next timed step)
    scratch_w = torch.empty(64 << 20, dtype=torch.float32, device=dev) if flush else None
    scratch_r = torch.ones(64 << 20, dtype=torch.float32, device=dev) if flush else None

    def flush_l2():
        scratch_w.zero_()
        scratch_r.sum()

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # Timed region 1 (the value): K coupled steps launched the library's
    # production way, as captured 2-step CUDA graphs, the L2 flushed before
    # every launch (an odd K ends with one kernel-by-kernel step).
    sim.set_graph(2)
    for _ in range(args.warmup):
        if flush:
            flush_l2()
        sim.step(2)
    barrier()
    units = [2] * (args.steps // 2) + [1] * (args.steps % 2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in units]
    launches0 = sim.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        for k, n in enumerate(units):
            if flush:
                flush_l2()
            ev[k][0].record(stream)
            sim.step(n)
            ev[k][1].record(stream)
        barrier()
        launches = sim.launch_count() - launches0
        total_ms = pdist.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
        sim.check()
        job_sites = pdist.sum_over_ranks(sites, world)
        value = job_sites * args.steps / (total_ms * 1e-3) / 1e6

        # Timed region 2 (kernel shares and the lattice kernel's roofline): the
        # same K steps launched kernel by kernel with a CUDA event pair around
        # every kernel on the stream it runs on.  The events lengthen the step,
        # so this pass does not give the value.
        sim.set_graph(0)
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        sim.profile(True)
        barrier()
        for k in range(args.steps):
            if flush:
                flush_l2()
            ev2[k][0].record(stream)
            sim.step(1)
            ev2[k][1].record(stream)
        barrier()
    ktimes = sim.kernel_times()
    sim.profile(False)
    profiled_ms = pdist.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev2), world)
    sim.check()

    # roofline of the stream-collide kernel (the lattice pass)
    peak, peak_kind = _peaks()
    n_sc, ms_sc = ktimes["stream_collide"]
    bytes_site = 152 if w["precision"] == "fp32" else 76
    achieved = bytes_site * sites / (ms_sc / n_sc * 1e-3) / 1e9 if n_sc else None
    traffic = _traffic_record(sites)
    # the step's own kernels: the particle kernel dominates a single chain's
    # step; it is latency-bound (100 cluster barriers per LB step) and has no
    # byte or flop roofline, so the roofline is the lattice kernel's and the
    # dominant kernel is named beside it with its share
    kern_ms = {k: ktimes[k][1] for k in ("gather", "particles", "stream_collide", "source") if k in ktimes}
    n_p = ktimes["particles"][0] if "particles" in ktimes else 0
    dominant = None
    if n_p:
        dominant = {"kernel": "k_particles", "bound": "latency",
                    "share_of_step_kernels": kern_ms["particles"] / sum(kern_ms.values()),
                    "us_per_launch": 1e3 * kern_ms["particles"] / n_p,
                    "us_per_md_substep": 1e3 * kern_ms["particles"] / n_p / (w["md_outer"] * w["md_inner"])}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "peak_kind": peak_kind, "kernel": "k_stream_collide",
                "algorithmic_bytes_per_launch": bytes_site * sites, "dominant_kernel": dominant}
    shares = {k: {"launches": n, "ms_total": ms, "ms_per_launch": ms / n if n else None}
              for k, (n, ms) in ktimes.items()}

    # end-to-end through the C ABI from pinned host buffers: upload the state,
    # K steps each reading back its diagnostics row, download the final state
    f_host = torch.empty(sim.n_real * 19 * sim.ns, dtype=torch.float32, pin_memory=True).numpy()
    r_host, v_host = sim.get_beads()
    f_host[:] = sim.get_populations().reshape(-1)
    # Host wall clock, summed over the timed intervals: the upload, every step
    # with its diagnostics read (the read synchronises), the download.  The
    # L2 flush before each step runs, and is waited for, between intervals.
    barrier()
    t0 = time.perf_counter()
    sim.set_populations(f_host)
    sim.set_beads(r_host, v_host)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    for _ in range(args.steps):
        if flush:
            flush_l2()
            torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sim.step(1)
        sim.diagnostics(1)
        wall += time.perf_counter() - t0
    t0 = time.perf_counter()
    f_back = sim.get_populations()
    r_back, _ = sim.get_beads()
    torch.cuda.synchronize(dev)
    wall += time.perf_counter() - t0
    e2e_s = pdist.max_over_ranks(wall, world)
    bi = f_host.nbytes + 2 * r_host.nbytes
    bo = args.steps * sim.n_real * ctypes.sizeof(lbmd.Diag) + f_back.nbytes + 2 * r_back.nbytes
    e2e = {"value": job_sites * args.steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": bi / args.steps, "d2h_bytes_per_step": bo / args.steps,
           "note": ("state uploaded once and downloaded once per K-step job; each step launched kernel by kernel "
                    "and its diagnostics row read back; host wall clock, L2 flush between the timed intervals")}

    if rank == 0:
        clocks = clk.summary()
        line = {"metric": "coupled LB-MD MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong" if "shard" in w else "weak", "vs_baseline": None,
                "dtype": "f32" if w["precision"] == "fp32" else "f16-storage/f32-math",
                "data": "synthetic", "config": dict(_config_block(w, flush), tiles=list(sim.tiles()),
                                                     md_shape=list(sim.md_shape()), md_exchange=sim.md_exchange(),
                                                     md_bonded=sim.md_bonded(), md_reserve=sim.md_reserve()),
                "launch": "captured 2-step CUDA graphs, L2 flushed before every launch",
                "roofline": roofline, "kernels": shares, "gpu_launches": launches,
                "kernel_timing": {"pass": "the same K steps kernel by kernel, CUDA events around every kernel",
                                  "ms_per_step": profiled_ms / args.steps},
                "clocks": clocks, "e2e": e2e}
        forms = [f for f in args.forms.split(",") if f and f != "none"]
        if forms and world == 1:
            line["forms"] = extra_measurements(dev, stream, peak, peak_kind, forms, args.tiles)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
