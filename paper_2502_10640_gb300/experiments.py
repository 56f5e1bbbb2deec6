"""The paper's own PP experiments on the GPU path (Sec. 2.1-2.2, Fig. 2).

The electron bunch is the cell-centred cube lattice of Sec. 2.1 (edge 0.1 mm, density
5e16 m^-3, at rest), run to 1e-8 s:
  * time-step sweep (Fig. 2a): N_p = 16^3, dt in {1e-13, 1e-12, 1e-11, 1e-10} s;
  * particle-number sweep (Fig. 2b): N_p in {4^3, 8^3, 16^3, 32^3}, dt = 1e-13 s;
recording the emittance of Eq. I and the moments of Figs. 5-6 along the way, and the
relative change of the total energy (kinetic + Coulomb potential) over each run.  The runs
use the hot path unchanged (pp_step) and only add diagnostics over time.

    python -m paper_2502_10640_gb300.experiments [--t-end 1e-8] [--records 200] [--out DIR]
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import time

import numpy as np

from . import capi, workloads as wl

EDGE = 1e-4          # m
DENSITY = 5e16       # m^-3
DT_SWEEP = (1e-13, 1e-12, 1e-11, 1e-10)
NP_SWEEP = (4, 8, 16, 32)
FIELDS = ("t", "step", "emit_x", "x_rms", "x_max", "vx_rms", "vx_max", "rms_radius", "ke")


def run_lattice(n_side: int, dt: float, t_end: float, records: int = 200,
                softening: float = 0.0) -> dict:
    """One lattice run; returns the diagnostics time series and the wall time."""
    n = n_side ** 3
    w = wl.lattice_weight(DENSITY, EDGE, n)
    pos = wl.cube_lattice(n_side, EDGE)
    steps = int(round(t_end / dt))
    every = max(1, steps // records)
    series = []
    with capi.Simulation(n, w, dt, softening, tune="cache") as sim:
        sim.load(pos)
        t0 = time.perf_counter()
        done = 0
        first = sim.diagnostics(with_pe=True)
        series.append(first)
        while done < steps:
            k = min(every, steps - done)
            sim.step(k)
            done += k
            series.append(sim.diagnostics(with_pe=done == steps))
        wall = time.perf_counter() - t0
        resident = bool(sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE))
    last = series[-1]
    e0, e1 = first["ke"] + first["pe"], last["ke"] + last["pe"]
    return {"n_side": n_side, "n": n, "w": w, "dt": dt, "steps": steps, "wall_s": wall,
            "pairs_per_s": float(n) * n * steps / wall, "resident": resident,
            "energy_drift": (e1 - e0) / abs(e0),
            "series": {k: [d[k] for d in series] for k in FIELDS}}


def write_csv(path: str, run: dict):
    with open(path, "w", newline="") as f:
        wr = csv.writer(f)
        wr.writerow(FIELDS)
        for row in zip(*(run["series"][k] for k in FIELDS)):
            wr.writerow(row)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--t-end", type=float, default=1e-8)
    ap.add_argument("--records", type=int, default=200)
    ap.add_argument("--out", default="experiments_out")
    ap.add_argument("--only", choices=["dt", "np", "all"], default="all")
    args = ap.parse_args(argv)
    os.makedirs(args.out, exist_ok=True)
    summary = []
    jobs = []
    if args.only in ("dt", "all"):
        jobs += [("dt", 16, dt) for dt in DT_SWEEP]
    if args.only in ("np", "all"):
        jobs += [("np", k, 1e-13) for k in NP_SWEEP if not (args.only == "all" and k == 16)]
    for sweep, k, dt in jobs:
        run = run_lattice(k, dt, args.t_end, args.records)
        name = f"lattice{k}_dt{dt:.0e}.csv"
        write_csv(os.path.join(args.out, name), run)
        row = {kk: run[kk] for kk in ("n_side", "n", "w", "dt", "steps", "wall_s", "pairs_per_s",
                                      "resident", "energy_drift")}
        ser = run["series"]
        row.update(sweep=sweep, file=name, final_emit_x=ser["emit_x"][-1],
                   x_rms_growth=ser["x_rms"][-1] / ser["x_rms"][0],
                   final_vx_max=ser["vx_max"][-1])
        summary.append(row)
        print(json.dumps(row), flush=True)
    with open(os.path.join(args.out, "summary.json"), "w") as f:
        json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
