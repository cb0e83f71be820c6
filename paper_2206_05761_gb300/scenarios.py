"""Runnable scenarios of the paper's tests on the GPU path.

    python -m paper_2206_05761_gb300.scenarios pseudo2d [--L 10] [--eps 1e-3]
        [--t-end 10] [--dt-sample 0.5] [--profile-window T0 T1] [--leaf-store]

pseudo2d: the pseudo-2D dam-break of Sec. 3.2 (50 m x 25 m flat channel,
6 m / 2 m, dam at x = 10 m, open sides) run with HWFV1 and with uniform FV1
from t = 0 to t_end; per interval of dt_sample the mean number of leaves,
the device time per step and the HWFV1 / uniform FV1 speed-up in simulated
seconds per second (the paper's speed-up as the flow goes from vigorous to
smooth).  --profile-window brackets the HWFV1 steps between T0 and T1 with
the CUDA profiler's start/stop (for ncu --profile-from-start off).
--leaf-store runs the HWFV1 side with the exact leaf-value store
(hwfv1_set_leaf_store: flat-bed subtrees stored at their deepest leaf level;
the same results).  Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json

import torch

from .sim import Simulation


def _series(p, f, uniform, t_end, dt_sample, precision, stream, window=None, leaf_store=False):
    sim = Simulation(p, f, precision, stream=stream)
    if leaf_store and not uniform:
        sim.set_leaf_store(True)
    sim.counters()                                # captures the step graph
    rows, tt = [], 0.0
    while tt < t_end - 1e-12:
        t1 = min(t_end, tt + dt_sample)
        prof = window is not None and not uniform and window[0] <= tt < window[1]
        c0 = sim.counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if prof:
            torch.cuda.profiler.start()
        e0.record(stream)
        while sim.time()[0] < t1:
            t, dt, _ = sim.time()
            k = max(1, min(2000, int((t1 - t) / dt) + 1))
            (sim.advance_uniform if uniform else sim.advance)(t_end=t1, max_steps=k)
        e1.record(stream)
        stream.synchronize()
        if prof:
            torch.cuda.profiler.stop()
        c1 = sim.counters()
        n = c1[0] - c0[0]
        rows.append({"t": t1, "steps": n, "ms": e0.elapsed_time(e1),
                     "mean_leaves": (c1[1] - c0[1]) / max(n, 1)})
        tt = t1
    sim.close()
    return rows


def pseudo2d(L=10, eps=1e-3, t_end=10.0, dt_sample=0.5, precision=64, window=None, leaf_store=False):
    import synth
    p, f = synth.pseudo_2d_dam_break(L=L, eps=eps)
    stream = torch.cuda.Stream()
    a = _series(p, f, False, t_end, dt_sample, precision, stream, window, leaf_store)
    u = _series(p, f, True, t_end, dt_sample, precision, stream)
    out = []
    for ra, ru in zip(a, u):
        out.append({"t": ra["t"], "hwfv1_mean_leaves": round(ra["mean_leaves"]),
                    "hwfv1_ms_per_step": ra["ms"] / max(ra["steps"], 1),
                    "uniform_ms_per_step": ru["ms"] / max(ru["steps"], 1),
                    "speedup": ru["ms"] / ra["ms"]})
    ms_a, ms_u = sum(r["ms"] for r in a), sum(r["ms"] for r in u)
    return {"workload": "pseudo-2D dam-break, 50 m x 25 m, 6 m / 2 m, L=%d (%dx%d), eps=%g, 0-%g s%s"
                        % (L, 1 << L, 1 << L, eps, t_end, ", exact leaf-value store" if leaf_store else ""),
            "finest_cells": 1 << (2 * L), "hwfv1_s": ms_a / 1e3, "uniform_s": ms_u / 1e3,
            "speedup": ms_u / ms_a, "series": out}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2206_05761_gb300.scenarios")
    ap.add_argument("scenario", choices=["pseudo2d"])
    ap.add_argument("--L", type=int, default=10)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--dt-sample", type=float, default=0.5)
    ap.add_argument("--precision", type=int, default=64, choices=[64, 32])
    ap.add_argument("--profile-window", type=float, nargs=2, default=None)
    ap.add_argument("--leaf-store", action="store_true")
    a = ap.parse_args(argv)
    r = pseudo2d(a.L, a.eps, a.t_end, a.dt_sample, a.precision, a.profile_window, a.leaf_store)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
