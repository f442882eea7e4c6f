"""Benchmark of the coupled LB-MD step (one JSON line on stdout).

A step is one coupled lattice-Boltzmann / molecular-dynamics step of the whole
hot path: gather, particle kernel (MD cycle and spread) and bead diagnostics
concurrently with the fused stream-collide kernel, then the source pass.  The
metric is MLUPS (million lattice-site updates per second, all
nx*ny*nz*n_real sites counted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl native|reference]

The default workload is the largest single-lattice configuration: 256x128x128
(4.19 M sites) with a 1000-bead chain, populations stored in FP32.

Under torchrun (N > 1) every rank runs an independent replica of the workload
(its own seed); value = all ranks' site updates / max-over-ranks time
(weak scaling, no data-path collective).

Timing: the K timed steps are one launch of the library's device-side
step-loop graph, bracketed by CUDA events on the library's stream.  The
populations (2 x 318 MB) are larger than the 129 MB L2; for a lattice small
enough to stay in L2 the steps are launched as 2-step graphs instead, with a
256 MiB buffer written and another read before each launch.
The roofline object reports the stream-collide kernel: algorithmic bytes
(19 x 4 B read + 19 x 4 B written per site in FP32, half that in FP16)
over its CUDA-event duration, against the measured HBM copy bandwidth;
`step_roofline` divides the same bytes by the whole step's time.
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


def _traffic_record(workload: str, sites: int):
    """DRAM bytes per launch of the stream-collide kernel on this workload from
    the committed ncu summary, if it was taken on the current kernel source;
    else None."""
    p = os.path.join(ROOT, "profiles", "stream_collide_traffic.json")
    src = os.path.join(ROOT, "paper_0711_2665_gb300", "csrc", "k_fluid.cu")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(workload)
    if not rec:
        return None
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


def _oracle_worker(job):
    """One oracle process: realization 0 of the workload, `warm` untimed
    steps, then whole LB-MD steps until `steps` are done (steps > 0) or
    `budget_s` seconds have passed.  Returns (steps, seconds)."""
    w, warm, steps, budget_s = job
    import oracle
    from paper_0711_2665_gb300 import workloads
    inp = workloads.build_inputs(w)
    o1 = int(inp["offsets"][1])
    orc = oracle.OracleSim(workloads.oracle_params(w, 0, o1), inp["solid"])
    orc.set_beads(inp["r0"][:o1])
    orc.step(max(warm, 1))
    n, t0 = 0, time.perf_counter()
    while (steps > 0 and n < steps) or (steps <= 0 and (time.perf_counter() - t0 < budget_s or n < 2)):
        orc.step(1)
        n += 1
    return n, time.perf_counter() - t0


def oracle_on_host_cores(w, warm=1, steps=0, budget_s=10.0):
    """The FP64 oracle, as it stands, on every host core: one spawned oracle
    process per core, each stepping its own copy of realization 0 (replicas,
    no shared work).  value = all processes' site updates / the slowest
    process's time; per_core = the mean process's rate."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(w, warm, steps, budget_s)] * cores)
    sites = w["nx"] * w["ny"] * w["nz"]
    total = sum(n for n, _ in res)
    t = max(dt for _, dt in res)
    per_core = statistics.mean(sites * n / dt / 1e6 for n, dt in res)
    beads = int(workloads_mod().bead_counts(w)[0])
    return {"value": sites * total / t / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "per_core": per_core,
            "sample": (f"{cores} oracle processes (one per host core), each {res[0][0]}+ FP64 steps of realization 0 "
                       f"({sites} sites, {beads} beads) after {max(warm, 1)} untimed; slowest {t:.1f} s")}


def workloads_mod():
    from paper_0711_2665_gb300 import workloads
    return workloads


def run_reference(args, w, world, rank):
    """The oracle (FP64, plain C) on the same workload, on every host core:
    each of K timed steps is one oracle LB-MD step of realization 0 in every
    core's process."""
    if rank != 0:
        return
    cb = oracle_on_host_cores(w, warm=args.warmup, steps=args.steps)
    mlups = cb["value"]
    sites = w["nx"] * w["ny"] * w["nz"]
    line = {"impl": "reference", "metric": "coupled LB-MD MLUPS", "value": mlups, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sites * cb["cores"] / (mlups * 1e6), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config_block(w, False), "cpu_baseline": cb,
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, budget_s=10.0):
    """The oracle timed on a bounded sample of the workload on every host core."""
    return oracle_on_host_cores(w, warm=1, steps=0, budget_s=budget_s)


def _lattice_kernel(sim):
    """The lattice-pass kernel the tiles select: one site per thread (by > 0),
    fed by tensor copies (by = 0) or two x sites per thread (by < 0)."""
    by = sim.tiles()[0]
    return "k_stream_collide" if by > 0 else ("k_stream_collide_tma" if by == 0 else "k_stream_collide_x2")


def _sc_roofline(sim, w, peak, peak_kind, steps=10, flush=None):
    """Stream-collide roofline from per-launch CUDA events over a few eager
    steps: inside the step (sharing the GPU with the particle kernel) and
    alone (the particle kernel waited for); achieved/frac are the latter.
    flush, if given, runs before every step (lattices that fit in L2)."""
    sites = w["nx"] * w["ny"] * w["nz"] * w["n_real"]
    b = (152 if w["precision"] == "fp32" else 76) * sites
    us = {}
    for overlap in (True, False):
        sim.set_overlap(overlap)
        sim.profile(True)
        for _ in range(steps):
            if flush:
                flush()
            sim.step(1)
        kt = sim.kernel_times()
        sim.profile(False)
        n, ms = kt["stream_collide"]
        us["in_step" if overlap else "alone"] = 1e3 * ms / n
    sim.set_overlap(True)
    achieved = b / (us["alone"] * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "kernel": _lattice_kernel(sim), "algorithmic_bytes_per_launch": b,
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


def extra_measurements(dev, stream, peak, peak_kind, forms, tiles=None, headline=None):
    """The other forms of the step, each timed on its own workload with CUDA
    events on the library's stream: the 128x64x64 plain step (its 80 MB of
    populations fit in L2, so it is launched as 2-step graphs with the L2
    flushed before each launch), the batched ensemble and the FP16-deviation
    storage (inputs larger than L2; each run of K steps one launch of the
    device-side step-loop graph), and the reverse sweep (forward +
    checkpointed adjoint of 200 steps).  The ensemble's and the FP16 form's
    speedups are over the headline's plain FP32 step on the same 4.19 M
    sites."""
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

    flush_w = flush_r = None
    for name, K in (("plain_fp32", 60), ("ensemble_fp32", 100), ("fp16dev", 60)):
        if name not in forms:
            continue
        w = workloads.get(name)
        inp = workloads.build_inputs(w)
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=str(dev))
        if tiles:
            sim.set_tiles(*tiles)
            by, zc = tiles
        else:
            by, zc = sim.autotune(8)
        sites = w["nx"] * w["ny"] * w["nz"] * w["n_real"]
        fits_l2 = sites * (152 if w["precision"] == "fp32" else 76) < 2 * L2_BYTES
        if fits_l2:
            if flush_w is None:
                flush_w = torch.empty(64 << 20, dtype=torch.float32, device=dev)
                flush_r = torch.ones(64 << 20, dtype=torch.float32, device=dev)

            def flush():
                with torch.cuda.stream(stream):
                    flush_w.zero_()
                    flush_r.sum()
            sim.set_graph(2)
            for _ in range(3):
                flush()
                sim.step(2)
            t = 0.0
            for _ in range(K // 2):
                flush()
                t += timed(lambda: sim.step(2))
            launch = "2-step CUDA graphs, L2 flushed before every launch"
        else:
            flush = None
            sim.step_loop(20)  # captures the device-side loop graph
            t = timed(lambda: sim.step_loop(K))
            launch = "one CUDA-graph launch per run (device-side loop of two-step bodies)"
        rf = _sc_roofline(sim, w, peak, peak_kind, flush=flush)
        sim.check()
        out[name] = {"value": sites * K / t / 1e6, "unit": "MLUPS", "ms_per_step": 1e3 * t / K,
                     "steps_per_s": K / t, "realization_steps_per_s": K * w["n_real"] / t, "steps": K,
                     "lattice": [w["nx"], w["ny"], w["nz"]], "n_real": w["n_real"], "beads": int(inp["offsets"][-1]),
                     "precision": w["precision"], "tiles": [by, zc], "md_shape": list(sim.md_shape()),
                     "md_exchange": sim.md_exchange(), "md_bonded": sim.md_bonded(), "md_reserve": sim.md_reserve(),
                     "launch": launch, "roofline": rf,
                     "step_frac": rf["algorithmic_bytes_per_launch"] / (t / K) / 1e9 / peak}
        sim.close()
    if headline and headline[0] == "lattice_4m_fp32":
        out["speedups_vs_headline_fp32"] = {
            k: out[k]["value"] / headline[1] for k in ("ensemble_fp32", "fp16dev") if k in out}
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


L2_BYTES = 129 * 1024 * 1024


def run_slabs(args, w_full, world, rank, local):
    """One lattice split into x-slabs over the ranks (one slab per rank and
    GPU): each step gathers, sums u_p over the ranks, advances and exchanges
    the slab faces with the neighbours (NCCL), then imports them.  value =
    the whole lattice's site updates / the slowest rank's time (strong
    scaling: the lattice is fixed as N grows)."""
    import torch
    import torch.distributed as dist
    from paper_0711_2665_gb300 import build as libbuild, dist as pdist, lbmd, workloads
    libbuild.build_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    w = pdist.slab_workload(w_full, rank, world)
    inp = workloads.build_inputs(w_full)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=f"cuda:{local}")
    sim.autotune(8)
    views = sim.slab_views()
    for _ in range(args.warmup):
        pdist.slab_step_dist(sim, views, rank, world)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        a.record(stream)
        for _ in range(args.steps):
            pdist.slab_step_dist(sim, views, rank, world)
        b.record(stream)
        barrier()
    total_ms = pdist.max_over_ranks(a.elapsed_time(b), world)
    sim.check()
    sites = w_full["nx"] * w_full["ny"] * w_full["nz"]
    value = sites * args.steps / (total_ms * 1e-3) / 1e6
    # end to end: upload this slab's state from pinned host memory, K steps,
    # read back the K diagnostics rows and the final state
    L = sim._lib
    f_in = torch.empty(sim.n_real * 19 * sim.ns, dtype=torch.float32, pin_memory=True)
    f_in.numpy()[:] = sim.get_populations().reshape(-1)
    r0h, v0h = sim.get_beads()
    r_in = torch.from_numpy(r0h.reshape(-1).copy()).pin_memory()
    v_in = torch.from_numpy(v0h.reshape(-1).copy()).pin_memory()
    diag = (lbmd.Diag * args.steps)()
    rows = ctypes.c_int32()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    barrier()
    t0 = time.perf_counter()
    ok = [L.lbmd_set_populations(sim._h, P(f_in)), L.lbmd_set_beads(sim._h, P(r_in), P(v_in))]
    for _ in range(args.steps):
        pdist.slab_step_dist(sim, views, rank, world)
    ok += [L.lbmd_diagnostics(sim._h, diag, args.steps, ctypes.byref(rows)),
           L.lbmd_get_populations(sim._h, P(f_in)), L.lbmd_get_beads(sim._h, P(r_in), P(v_in))]
    barrier()
    e2e_s = pdist.max_over_ranks(time.perf_counter() - t0, world)
    assert all(x == 0 for x in ok)
    nb = 2 * 8 * 3 * sim.total_beads
    if rank == 0:
        line = {"metric": "coupled LB-MD MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32" if w["precision"] == "fp32" else "f16-storage/f32-math", "data": "synthetic",
                "config": dict(_config_block(w, False), parallelism=f"x-slabs over {world} ranks",
                               slab_planes=[p for _, p in pdist.slab_partition(w_full["nx"], world)]),
                "launch": "per step: gather, u_p all-reduce, advance, face exchange (NCCL send/recv), import",
                "roofline": {"bound": "hbm", "achieved": None, "peak": _peaks()[0], "unit": "GB/s", "frac": None,
                             "traffic": None, "note": "see the single-lattice run"},
                "gpu_launches": sim.launch_count(), "clocks": clk.summary(),
                "e2e": {"value": sites * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                        "h2d_bytes_per_step": (f_in.numel() * 4 + nb) / args.steps,
                        "d2h_bytes_per_step": (rows.value * ctypes.sizeof(lbmd.Diag) + f_in.numel() * 4 + nb) / args.steps}}
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="lattice_4m_fp32")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="plain_fp32,ensemble_fp32,fp16dev,variants,adjoint",
                    help="comma list of the other forms to measure (plain_fp32, ensemble_fp32, fp16dev, "
                         "variants, adjoint), or none")
    ap.add_argument("--tiles", type=int, nargs=2, metavar=("BY", "ZC"), default=None,
                    help="fixed stream-collide tile shape instead of the autotuner (for profiling runs)")
    ap.add_argument("--md-shape", type=int, nargs=2, metavar=("T", "C"), default=None,
                    help="with --tiles: lanes per bead and blocks per chain of the particle kernel")
    ap.add_argument("--md-exchange", choices=["push", "pull"], default=None,
                    help="with --tiles: the particle kernel's chain exchange")
    ap.add_argument("--md-bonded", choices=["lanes", "warp"], default=None,
                    help="with --tiles: who evaluates the particle kernel's bonded terms")
    ap.add_argument("--md-reserve", choices=["share", "reserve"], default=None,
                    help="whether the particle kernel's blocks claim their SMs (else the autotuner's choice)")
    ap.add_argument("--slabs", action="store_true",
                    help="with N ranks: split the one lattice into N x-slabs (strong scaling) instead of "
                         "running N replicas")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_0711_2665_gb300 import dist as pdist, workloads
    world, rank, local = pdist.env()
    if args.slabs and args.impl == "native":
        return run_slabs(args, workloads.get(args.workload), world, rank, local)
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
    if args.md_reserve:
        sim.set_md_reserve(args.md_reserve)
    if args.tiles:
        sim.set_tiles(*args.tiles)
        if args.md_shape:
            sim.set_md_shape(*args.md_shape)
        if args.md_exchange:
            sim.set_md_exchange(args.md_exchange)
        if args.md_bonded:
            sim.set_md_bonded(args.md_bonded)
    else:
        sim.autotune(8)
    sites = w["nx"] * w["ny"] * w["nz"] * w["n_real"]
    bytes_site = 152 if w["precision"] == "fp32" else 76
    # the populations' two buffers against the L2: a lattice that fits is
    # launched as 2-step graphs with an L2 flush (write 256 MiB, then read
    # another 256 MiB, so that the L2 ends up holding clean lines) before each
    flush = sites * bytes_site < 2 * L2_BYTES
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
    # production way: one step-loop graph launch (or 2-step graphs with an L2
    # flush before each, for a lattice that fits in L2).
    if flush:
        sim.set_graph(2)
        for _ in range(args.warmup):
            flush_l2()
            sim.step(2)
        units = [2] * (args.steps // 2) + [1] * (args.steps % 2)
    else:
        sim.step_loop(args.warmup + (args.warmup & 1))  # captures the loop graph
        units = [args.steps]
    # the state (and step number) the timed steps start from: the end-to-end
    # jobs below start from it too, so they compute the very same steps
    L = sim._lib
    nf = sim.n_real * 19 * sim.ns
    nb3 = 3 * max(sim.total_beads, 1)
    f_in = torch.empty(nf, dtype=torch.float32, pin_memory=True)
    r_in = torch.empty(nb3, dtype=torch.float64, pin_memory=True)
    v_in = torch.empty(nb3, dtype=torch.float64, pin_memory=True)
    f_in.numpy()[:] = sim.get_populations().reshape(-1)
    if sim.total_beads:
        r0h, v0h = sim.get_beads()
        r_in.numpy()[:] = r0h.reshape(-1)
        v_in.numpy()[:] = v0h.reshape(-1)
    step0 = sim.step_count
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in units]
    launches0 = sim.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        for k, n in enumerate(units):
            if flush:
                flush_l2()
            ev[k][0].record(stream)
            if flush:
                sim.step(n)
            else:
                sim.step_loop(n)
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

    # roofline of the stream-collide kernel (the lattice pass): inside the
    # step (sharing the GPU with the particle kernel; the timed region) and
    # alone (the particle kernel waited for)
    peak, peak_kind = _peaks()
    n_sc, ms_sc = ktimes["stream_collide"]
    alg = bytes_site * sites
    achieved = alg / (ms_sc / n_sc * 1e-3) / 1e9 if n_sc else None
    alone = _sc_roofline(sim, w, peak, peak_kind, steps=min(args.steps, 10), flush=flush_l2 if flush else None)
    # the committed capture is of the one-site-per-thread kernel
    traffic = _traffic_record(w["name"], sites) if world == 1 and sim.tiles()[0] > 0 else None
    # the step's own kernels: the particle kernel sets a single chain's step;
    # it is latency-bound (100 cluster barriers per LB step) and has no byte
    # or flop roofline, so the roofline is the lattice kernel's and the
    # dominant kernel is named beside it with its share
    kern_ms = {k: ktimes[k][1] for k in ("gather", "particles", "stream_collide", "source", "bead_diag") if k in ktimes}
    n_p = ktimes["particles"][0] if "particles" in ktimes else 0
    dominant = None
    if n_p:
        dominant = {"kernel": "k_particles", "bound": "latency",
                    "share_of_step_kernels": kern_ms["particles"] / sum(kern_ms.values()),
                    "us_per_launch": 1e3 * kern_ms["particles"] / n_p,
                    "us_per_md_substep": 1e3 * kern_ms["particles"] / n_p / (w["md_outer"] * w["md_inner"])}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "peak_kind": peak_kind, "kernel": _lattice_kernel(sim), "algorithmic_bytes_per_launch": alg,
                "us_per_launch_in_step": 1e3 * ms_sc / n_sc if n_sc else None,
                "us_per_launch_alone": alone["us_per_launch_alone"], "frac_alone": alone["frac"],
                "dominant_kernel": dominant}
    ms_step = total_ms / args.steps
    step_roofline = {"bound": "hbm", "bytes_per_step": alg, "achieved": alg / (ms_step * 1e-3) / 1e9,
                     "peak": peak, "unit": "GB/s", "frac": alg / (ms_step * 1e-3) / 1e9 / peak,
                     "note": "the lattice pass's algorithmic bytes over the whole coupled step's time"}
    shares = {k: {"launches": n, "ms_total": ms, "ms_per_launch": ms / n if n else None}
              for k, (n, ms) in ktimes.items()}

    # End to end through the C ABI from pinned host buffers: upload the state
    # (populations and beads), K steps as one step-loop launch, read back the
    # K diagnostics rows, download the final state; host wall clock.
    f_out = torch.empty(nf, dtype=torch.float32, pin_memory=True)
    r_out = torch.empty(nb3, dtype=torch.float64, pin_memory=True)
    v_out = torch.empty(nb3, dtype=torch.float64, pin_memory=True)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    diag = (lbmd.Diag * (sim.n_real * args.steps))()
    rows = ctypes.c_int32()
    # the step-loop graph is captured once per configuration (the profiling
    # passes above dropped it); a caller's jobs reuse it, so capture it here
    sim.step_loop(2)
    # three identical jobs, each uploading the state and step number the
    # timed steps started from (so each computes those same K steps: the
    # particle kernel's cost follows the chain along its trajectory); the
    # median is reported, every job's time beside it: the copies share the
    # host's memory with whatever else runs on it, and one job can catch a
    # stall
    walls = []
    for _ in range(3):
        if flush:
            flush_l2()
        barrier()
        t0 = time.perf_counter()
        ok = [L.lbmd_set_populations(sim._h, P(f_in)), L.lbmd_set_beads(sim._h, P(r_in), P(v_in)),
              L.lbmd_set_step(sim._h, ctypes.c_int64(step0))]
        sim.step_loop(args.steps)
        ok += [L.lbmd_diagnostics(sim._h, diag, args.steps, ctypes.byref(rows)),
               L.lbmd_get_populations(sim._h, P(f_out)), L.lbmd_get_beads(sim._h, P(r_out), P(v_out))]
        walls.append(time.perf_counter() - t0)
        assert all(x == 0 for x in ok) and rows.value == args.steps, (ok, rows.value)
    wall = statistics.median(walls)
    e2e_s = pdist.max_over_ranks(wall, world)
    bi = f_in.numel() * 4 + 2 * 8 * 3 * sim.total_beads + 8
    bo = sim.n_real * rows.value * ctypes.sizeof(lbmd.Diag) + f_out.numel() * 4 + 2 * 8 * 3 * sim.total_beads
    e2e = {"value": job_sites * args.steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": bi / args.steps, "d2h_bytes_per_step": bo / args.steps,
           "jobs_ms": [round(1e3 * x, 3) for x in walls],
           "note": ("K-step jobs through the C ABI from pinned host buffers: state upload, one step-loop launch "
                    "(its graph captured before, as a caller's later jobs reuse it), the K diagnostics rows and the "
                    "final state read back; host wall clock, the median of three identical jobs, each from the state and step "
                    "the timed steps started from")}

    if rank == 0:
        clocks = clk.summary()
        line = {"metric": "coupled LB-MD MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "strong" if "shard" in w else "weak", "vs_baseline": None,
                "dtype": "f32" if w["precision"] == "fp32" else "f16-storage/f32-math",
                "data": "synthetic", "config": dict(_config_block(w, flush), tiles=list(sim.tiles()),
                                                     md_shape=list(sim.md_shape()), md_exchange=sim.md_exchange(),
                                                     md_bonded=sim.md_bonded(), md_reserve=sim.md_reserve()),
                "launch": ("captured 2-step CUDA graphs, L2 flushed before every launch" if flush else
                           "one launch of the device-side step-loop graph for the K steps"),
                "roofline": roofline, "step_roofline": step_roofline, "kernels": shares, "gpu_launches": launches,
                "kernel_timing": {"pass": "the same K steps kernel by kernel, CUDA events around every kernel",
                                  "ms_per_step": profiled_ms / args.steps},
                "clocks": clocks, "e2e": e2e}
        forms = [f for f in args.forms.split(",") if f and f != "none"]
        if forms and world == 1:
            line["forms"] = extra_measurements(dev, stream, peak, peak_kind, forms, args.tiles,
                                               headline=(w["name"], value))
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
