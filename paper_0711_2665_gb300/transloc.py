"""Translocation statistics of an ensemble of chains (Sec. IV.A, IV.B).

The particle kernel keeps one record per realization (lbmd_translocation):
the first step at which every bead of the chain had crossed the wall, and the
radii of gyration of the untranslocated part at the record's origin and of
the translocated part at that step.  This module turns the records of an
ensemble into the paper's statistics:

* the duration of each event, tau = t_x - t_origin (LB steps);
* a duration histogram per chain length N0; the distributions are skewed
  towards long times, so tau(N0) is the most probable duration, the centre of
  the histogram's highest bin, not the mean (Sec. IV.A);
* the exponent alpha of tau(N0) ~ N0^alpha, by least squares on
  log tau against log N0 (Sec. IV.A);
* lambda_R = R_T(t_X) / R_U(0) per event (Sec. IV.B).

Histogram bins follow the Freedman-Diaconis rule unless given: the paper
does not state its binning.  `run` drives one ensemble on the GPU;
``python -m paper_0711_2665_gb300.transloc`` prints its summary as JSON.
`precision_run` (``--precision-study WORKLOAD``) runs one chain in FP32 and
in FP16 population storage from the same seed and noise streams and reports
both translocation times.
"""
from __future__ import annotations

import json
import time

import numpy as np


def durations(rec) -> np.ndarray:
    """tau = t_x - t_origin of each record; NaN where the chain has not yet
    translocated completely."""
    t_x = np.asarray(rec["t_x"], dtype=np.int64)
    t0 = np.asarray(rec["t_origin"], dtype=np.int64)
    return np.where(t_x >= 0, (t_x - t0).astype(np.float64), np.nan)


def lambda_r(rec) -> np.ndarray:
    """R_T(t_X) / R_U(0) of each completed event (NaN elsewhere)."""
    ru = np.asarray(rec["rg_u_origin"], dtype=np.float64)
    rt = np.asarray(rec["rg_t_x"], dtype=np.float64)
    ok = (np.asarray(rec["t_x"]) >= 0) & (ru > 0)
    out = np.full(ru.shape, np.nan)
    out[ok] = rt[ok] / ru[ok]
    return out


def histogram(tau, bins="fd"):
    """Counts and bin edges of the finite durations in tau."""
    t = np.asarray(tau, dtype=np.float64)
    t = t[np.isfinite(t)]
    if t.size == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(1)
    if np.ptp(t) == 0:
        return np.array([t.size]), np.array([t[0] - 0.5, t[0] + 0.5])
    return np.histogram(t, bins=bins)


def most_probable(tau, bins="fd") -> float:
    """Centre of the highest histogram bin of the finite durations (the first
    such bin on a tie); NaN for an empty sample."""
    counts, edges = histogram(tau, bins)
    if counts.size == 0:
        return float("nan")
    k = int(np.argmax(counts))
    return 0.5 * float(edges[k] + edges[k + 1])


def scaling_exponent(n0, tau) -> dict:
    """Least-squares fit log tau = log c + alpha log N0 over the finite
    pairs: alpha, c and the standard error of alpha (NaN with two points)."""
    n = np.asarray(n0, dtype=np.float64)
    t = np.asarray(tau, dtype=np.float64)
    ok = np.isfinite(t) & (t > 0) & (n > 0)
    x, y = np.log(n[ok]), np.log(t[ok])
    if x.size < 2:
        raise ValueError("the exponent needs at least two chain lengths")
    A = np.stack([np.ones_like(x), x], axis=1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    se = float("nan")
    if x.size > 2:
        res = y - A @ coef
        s2 = float(res @ res) / (x.size - 2)
        se = float(np.sqrt(s2 / np.sum((x - x.mean()) ** 2)))
    return {"alpha": float(coef[1]), "prefactor": float(np.exp(coef[0])), "alpha_stderr": se}


def summarize(counts, rec, bins="fd") -> dict:
    """Per chain length: events, completed events, mean and most probable
    duration, mean lambda_R; and the exponent over the lengths with a
    most probable duration."""
    counts = np.asarray(counts)
    tau = durations(rec)
    lam = lambda_r(rec)
    per = {}
    for n in sorted(set(int(c) for c in counts)):
        sel = counts == n
        t = tau[sel]
        done = np.isfinite(t)
        per[n] = {"events": int(sel.sum()), "completed": int(done.sum()),
                  "tau_mean": float(np.mean(t[done])) if done.any() else None,
                  "tau_most_probable": most_probable(t, bins) if done.any() else None,
                  "lambda_r_mean": float(np.nanmean(lam[sel])) if done.any() else None}
    ns = [n for n, v in per.items() if v["tau_most_probable"] is not None]
    fit = None
    if len(ns) >= 2:
        fit = scaling_exponent(ns, [per[n]["tau_most_probable"] for n in ns])
    return {"by_length": per, "fit": fit}


def run(lengths, copies: int, max_steps: int, chunk: int = 200, overrides: dict | None = None,
        autotune: bool = True) -> dict:
    """Translocation experiment on the ensemble engine: copies realizations of
    every chain length (each its own starting conformation and noise stream)
    on the ensemble workload's lattice, stepped with the device-side graph
    loop until every chain has translocated or max_steps have run."""
    from . import lbmd, workloads
    counts = np.repeat(np.asarray(lengths, dtype=np.int64), copies)
    w = workloads.get("ensemble_fp32", n_real=int(counts.size), bead_counts=[int(c) for c in counts],
                      **(overrides or {}))
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    if autotune:
        sim.autotune(3)
    sim.reset_translocation()
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        n = min(chunk, max_steps - steps)
        sim.step_loop(n)
        steps += n
        rec = sim.translocation()
        if np.all(rec["t_x"] >= 0):
            break
    sim.check()
    wall = time.perf_counter() - t0
    rec = sim.translocation()
    sites = w["nx"] * w["ny"] * w["nz"] * counts.size
    return {"counts": counts, "records": rec, "steps": steps, "seconds": wall,
            "mlups": sites * steps / wall / 1e6, "workload": w}


def precision_run(name: str = "lattice_4m_fp32", precisions=("fp32", "fp16dev"), seed: int | None = None,
                  max_steps: int = 20000, chunk: int = 1000, every: int = 100, autotune: bool = True) -> dict:
    """One chain on one lattice, run from the same seeded start with the same
    noise streams in each population storage precision: its translocation
    time t_X (Sec. IV.A; -1 if the event has not completed in max_steps) and
    the translocated fraction of the chain every `every` steps, read from the
    per-step diagnostics rows."""
    from . import lbmd, workloads
    out = {}
    for prec in precisions:
        ov = {"precision": prec}
        if seed is not None:
            ov.update(seed=seed, chain_seed=seed)
        w = workloads.get(name, **ov)
        inp = workloads.build_inputs(w)
        n_beads = int(inp["offsets"][1])
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
        if autotune:
            sim.autotune(3)
        sim.reset_translocation()
        frac, steps, t0 = [], 0, time.perf_counter()
        rec = sim.translocation()[0]
        while steps < max_steps:
            n = min(chunk, max_steps - steps, 1000)
            sim.step_loop(n)
            rows = sim.diagnostics(n)[0]
            frac += [(int(r["step"]), float(r["n_translocated"]) / n_beads) for r in rows if r["step"] % every == 0]
            steps += n
            rec = sim.translocation()[0]
            if rec["t_x"] >= 0:
                break
        sim.check()
        out[prec] = {"t_x": int(rec["t_x"]), "steps": steps, "seconds": time.perf_counter() - t0,
                     "beads": n_beads, "fraction": frac}
        sim.close()
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--lengths", default="20,40,60,80,100,140,200")
    ap.add_argument("--copies", type=int, default=32)
    ap.add_argument("--max-steps", type=int, default=20000)
    ap.add_argument("--chunk", type=int, default=200)
    ap.add_argument("--E", type=float, default=None)
    ap.add_argument("--gamma", type=float, default=None)
    ap.add_argument("--kT", type=float, default=None)
    ap.add_argument("--box", type=int, default=None,
                    help="Nx of an Nx x Nx/2 x Nx/2 box with the wall at Nx/2 (Sec. IV: 80 up to 400 beads)")
    ap.add_argument("--interp", type=int, default=None, help="0 trilinear, 1 nearest grid point")
    ap.add_argument("--integrator", type=int, default=None, help="0 velocity Verlet, 1 stochastic position Verlet")
    ap.add_argument("--records", default=None, help="write the raw records (.npz) here")
    ap.add_argument("--precision-study", default=None, metavar="WORKLOAD",
                    help="instead: one chain of WORKLOAD in FP32 and in FP16 storage (same seed and noise): "
                         "t_X and the translocated fraction every 100 steps")
    ap.add_argument("--seed", type=int, default=None, help="with --precision-study: chain and noise seed")
    a = ap.parse_args(argv)
    if a.precision_study:
        print(json.dumps(precision_run(a.precision_study, seed=a.seed, max_steps=a.max_steps), default=float))
        return
    ov = {k: v for k, v in (("E", a.E), ("gamma", a.gamma), ("kT", a.kT), ("interp", a.interp),
                            ("integrator", a.integrator)) if v is not None}
    if a.box:
        ov.update(nx=a.box, ny=a.box // 2, nz=a.box // 2, wall_x=a.box // 2)
    lengths = [int(x) for x in a.lengths.split(",") if x]
    out = run(lengths, a.copies, a.max_steps, a.chunk, ov)
    summ = summarize(out["counts"], out["records"])
    w = out["workload"]
    line = {"workload": {k: w.get(k, 0) for k in ("nx", "ny", "nz", "wall_x", "pore_h", "E", "gamma", "kT", "tau",
                                                  "interp", "integrator")},
            "lengths": lengths, "copies": a.copies, "steps": out["steps"], "seconds": out["seconds"],
            "mlups": out["mlups"], **summ}
    if a.records:
        np.savez(a.records, counts=out["counts"], records=out["records"])
    print(json.dumps(line, default=float))


if __name__ == "__main__":
    main()
