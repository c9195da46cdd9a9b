"""Section 8's first-Hopf-bifurcation study through the C ABI.

A 100 x 100 box with diffusive Maxwell walls (the top one moving with
u0 = 0.1), entropic equilibria and the median entropy filter (delta = 1e-3);
the velocity of the control point (L/16, 13L/16) is recorded every step,
and the energy E_u of Eq. (energy) of the last 1% of the signal is computed
per Reynolds number; E_u^2 grows linearly with Re above the bifurcation and
the line's zero locates it (the paper reports Re = 7135 on this grid).

Readings: the box has n sites a side, the wall sites on its edges, and
L = n - 1 is the distance between opposite walls (Re = u0 L / nu); the
control point is the site nearest (L/16, 13L/16) from the bottom-left
corner; 5000 L / u0 steps.

    python -m paper_1110_0270_gb300.experiments --re 7000 7250 7500 7750 8000
"""
from __future__ import annotations

import argparse
import json
import time

from . import lbm
from .analysis import fit_onset, hopf_energy


def hopf_sweep(res, n: int = 100, u0: float = 0.1, steps: int | None = None, precision: str = "fp64",
               delta: float = 1e-3, frac: float = 0.01, chunk: int = 6400) -> dict:
    """One lattice per Reynolds number, each on its own CUDA stream so that
    the small, latency-bound lattices run concurrently; the probe keeps the
    last `frac` of the signal of the control point."""
    import numpy as np
    import torch
    L = n - 1
    steps = int(steps if steps is not None else 5000 * L / u0)
    keep = max(2, int(frac * steps))
    xp, yp = int(round(L / 16)), int(round(13 * L / 16))
    runs = []
    for re in res:
        cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="diffusive", lid_u=u0, nu=u0 * L / re, collision="median",
                   equilibrium="entropic", delta=delta, precision=precision)
        lat = lbm.Lattice(cfg)
        ones = np.ones((n, n))
        lat.init(ones, 0 * ones, 0 * ones)
        lat.probe(xp, yp, keep)
        runs.append((re, lat, torch.cuda.Stream()))
    torch.cuda.synchronize()
    t0 = time.time()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        for _, lat, s in runs:
            lat.step(k, stream=s)
        done += k
    torch.cuda.synchronize()
    seconds = time.time() - t0
    points = []
    for re, lat, _ in runs:
        sig = lat.probe_signal()
        st = lat.stats()
        E = hopf_energy(sig[:, 0], L, u0)
        points.append({"re": re, "E_u": E, "E_u2": E * E, "samples": int(sig.shape[0]),
                       "u_mean": float(sig[:, 0].mean()), "v_mean": float(sig[:, 1].mean()),
                       "diverged": int(st["diverged"]), "limited_total": int(st["limited_total"])})
    fit = fit_onset([p["re"] for p in points], [p["E_u2"] for p in points])
    return {"n": n, "L": L, "u0": u0, "steps": steps, "control_point": [xp, yp], "precision": precision,
            "seconds": round(seconds, 1), "points": points, "fit": fit}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--re", type=float, nargs="+", required=True)
    ap.add_argument("--n", type=int, default=100)
    ap.add_argument("--steps", type=int, default=None, help="default 5000 L / u0")
    ap.add_argument("--precision", default="fp64")
    args = ap.parse_args(argv)
    print(json.dumps(hopf_sweep(args.re, n=args.n, steps=args.steps, precision=args.precision)), flush=True)


if __name__ == "__main__":
    main()
