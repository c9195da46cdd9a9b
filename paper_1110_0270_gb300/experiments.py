"""Section 8's two lid-driven-cavity studies through the C ABI.

Stability: a 129 x 129 cavity with half-way bounce-back walls and the lid
at u_wall = 0.1, polynomial (product) equilibria, run for up to 10^7 steps
with six methods - LBGK, LBGK with Ehrenfest steps, LBGK with the MRT
limiter (at most 9 limited sites per step each), TRT, MRT with the TRT
third-order rate and s_e = 1.64, s_eps = 1.54, and MRT1 (s_q = 1.9,
s_e = 1.64, s_eps = 1.54) - recording which survive, their mean enstrophy
over the last 2 10^5 steps and the primary vortex of the final stream
function.

Hopf: a 100 x 100 box with diffusive Maxwell walls (the top one moving with
u0 = 0.1), entropic equilibria and the median entropy filter (delta = 1e-3);
the velocity of the control point (L/16, 13L/16) is recorded every step,
and the energy E_u of Eq. (energy) of the last 1% of the signal is computed
per Reynolds number; E_u^2 grows linearly with Re above the bifurcation and
the line's zero locates it (the paper reports Re = 7135 on this grid).

Readings: the box has n sites a side, the wall sites on its edges, and
L = n - 1 is the distance between opposite walls (Re = u0 L / nu); the
control point is the site nearest (L/16, 13L/16) from the bottom-left
corner; 5000 L / u0 steps.  The alternative placement (walls="outside")
reads "100 x 100" as the fluid sites: the lattice has n + 2 sites a side,
the wall sites around the n x n fluid, and L = n + 1.

Stability readings: L = n - 1 = 128 (Re = u_wall L / nu), Ehrenfest and
MRT-limiter threshold delta = 1e-3, survival = no non-finite or
non-positive density seen (checked every `check` steps).

    python -m paper_1110_0270_gb300.experiments hopf --re 7000 7250 7500 7750 8000 [--walls outside]
    python -m paper_1110_0270_gb300.experiments stability --re 1000 2500 5000 7500 10000
"""
from __future__ import annotations

import argparse
import json
import time

from . import lbm
from .analysis import dominant_frequency, fit_onset, hopf_energy, stream_function, vortex_summary


def hopf_sweep(res, n: int = 100, u0: float = 0.1, steps: int | None = None, precision: str = "fp64",
               delta: float = 1e-3, frac: float = 0.01, chunk: int = 6400, walls: str = "edge") -> dict:
    """One lattice per Reynolds number, each on its own CUDA stream so that
    the small, latency-bound lattices run concurrently; the probe keeps the
    last `frac` of the signal of the control point.  walls: "edge" (n sites
    a side including the wall sites) or "outside" (n x n fluid sites inside
    the wall sites)."""
    import numpy as np
    import torch
    if walls not in ("edge", "outside"):
        raise ValueError(f"walls must be 'edge' or 'outside', not {walls!r}")
    fluid = n
    n = n + 2 if walls == "outside" else n
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
        spec = dominant_frequency(sig[:, 0], L, u0)
        points.append({"re": re, "E_u": E, "E_u2": E * E, "samples": int(sig.shape[0]),
                       "f_dom": spec["f"], "omega_dom": spec["omega"], "peak_share": spec["peak_share"],
                       "u_mean": float(sig[:, 0].mean()), "v_mean": float(sig[:, 1].mean()),
                       "diverged": int(st["diverged"]), "limited_total": int(st["limited_total"])})
    fit = fit_onset([p["re"] for p in points], [p["E_u2"] for p in points])
    return {"n": n, "fluid_sites": fluid if walls == "outside" else n - 2, "walls": walls, "L": L, "u0": u0,
            "steps": steps, "control_point": [xp, yp], "precision": precision,
            "seconds": round(seconds, 1), "points": points, "fit": fit}


STABILITY_METHODS = ("bgk", "ehrenfest", "mrt_limiter", "trt", "mrt", "mrt1")


def stability_config(method: str, re: float, n: int = 129, u0: float = 0.1, precision: str = "fp64",
                     topk: int = 9, delta: float = 1e-3) -> dict:
    """The lattice configuration of one method of the stability study."""
    L = n - 1
    nu = u0 * L / re
    beta = 1.0 / (6.0 * nu + 1.0)
    cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="cavity", lid_u=u0, nu=nu, precision=precision)
    if method == "bgk":
        cfg["collision"] = "lbgk"
    elif method in ("ehrenfest", "mrt_limiter"):
        cfg.update(collision=method, topk=topk, delta=delta)
    elif method in ("trt", "mrt", "mrt1"):
        cfg.update(collision="mrt", **lbm.mrt_rates(method, beta))
    else:
        raise ValueError(f"unknown method {method!r}")
    return cfg


def stability_sweep(res, methods=STABILITY_METHODS, n: int = 129, u0: float = 0.1, steps: int = 10**7,
                    precision: str = "fp64", window: int = 200000, sample: int = 1000,
                    check: int = 100000, chunk: int = 6400) -> dict:
    """Every (method, Re) pair as its own lattice on its own CUDA stream,
    stepped round-robin `chunk` steps at a time.
    Runs are checked for divergence every `check` steps and dropped when
    they diverge; the survivors' enstrophy is sampled every `sample` steps
    over the last `window` steps."""
    import numpy as np
    import torch
    runs = []
    for re in res:
        for m in methods:
            lat = lbm.Lattice(stability_config(m, re, n=n, u0=u0, precision=precision))
            ones = np.ones((n, n))
            lat.init(ones, 0 * ones, 0 * ones)
            runs.append({"method": m, "re": re, "lat": lat, "stream": torch.cuda.Stream(),
                         "diverged_by": None, "ens": []})
    torch.cuda.synchronize()
    t0 = time.time()
    window = min(window, steps)
    done = 0
    while done < steps:
        if done < steps - window:
            k = min(check, steps - window - done)
        else:
            k = min(sample, steps - done)
        live = [r for r in runs if r["diverged_by"] is None]
        if not live:
            break
        for sub in range(0, k, chunk):  # round-robin keeps every stream's queue short
            for r in live:
                r["lat"].step(min(chunk, k - sub), stream=r["stream"])
        done += k
        for r in live:
            st = r["lat"].stats(stream=r["stream"])
            if st["diverged"]:
                r["diverged_by"] = done
            elif done > steps - window:  # a sample at the end of each window chunk
                r["ens"].append(r["lat"].enstrophy(stream=r["stream"]))
    torch.cuda.synchronize()
    seconds = time.time() - t0
    table = []
    for r in runs:
        st = r["lat"].stats()
        row = {"method": r["method"], "re": r["re"], "survived": r["diverged_by"] is None,
               "diverged_by": r["diverged_by"], "limited_total": int(st["limited_total"])}
        if r["diverged_by"] is None:
            ens = np.asarray(r["ens"])
            rho, u = r["lat"].macros()
            ux, uy = u[0].cpu().numpy(), u[1].cpu().numpy()
            row.update(enstrophy_mean=float(ens.mean()), enstrophy_min=float(ens.min()),
                       enstrophy_max=float(ens.max()), vortices=vortex_summary(stream_function(ux, uy)))
        table.append(row)
    survivors = {str(re): [r["method"] for r in table if r["re"] == re and r["survived"]] for re in res}
    return {"n": n, "L": n - 1, "u0": u0, "steps": steps, "precision": precision, "seconds": round(seconds, 1),
            "survivors": survivors, "runs": table}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="study", required=True)
    h = sub.add_parser("hopf", help="first Hopf bifurcation (100 x 100, diffusive walls, median)")
    h.add_argument("--re", type=float, nargs="+", required=True)
    h.add_argument("--n", type=int, default=100)
    h.add_argument("--steps", type=int, default=None, help="default 5000 L / u0")
    h.add_argument("--precision", default="fp64")
    h.add_argument("--walls", choices=["edge", "outside"], default="edge",
                   help="n sites a side with the walls on the edges, or n x n fluid sites inside them")
    s = sub.add_parser("stability", help="survival of six methods (129 x 129, bounce-back)")
    s.add_argument("--re", type=float, nargs="+", required=True)
    s.add_argument("--methods", nargs="+", default=list(STABILITY_METHODS))
    s.add_argument("--n", type=int, default=129)
    s.add_argument("--steps", type=int, default=10**7)
    s.add_argument("--precision", default="fp64")
    args = ap.parse_args(argv)
    if args.study == "hopf":
        out = hopf_sweep(args.re, n=args.n, steps=args.steps, precision=args.precision, walls=args.walls)
    else:
        out = stability_sweep(args.re, methods=args.methods, n=args.n, steps=args.steps,
                              precision=args.precision)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
