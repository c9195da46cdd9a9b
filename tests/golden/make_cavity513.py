"""Writes cavity513.npz: the FP64 oracle's D2Q9 lid-driven cavity 513 x 513
(U 0.05, nu = U 512 / Re; fluid at rest at t = 0) after 2000 steps, the
reduced-size run that stands for the 4097^2 bandwidth configuration when the
storage formats' error is measured.  Three runs:

  ehrenfest_re10000  Re 10000, the Ehrenfest limiter (k = 64, delta = 1e-3)
  median_re10000     Re 10000, the median filter (delta = 1e-3)
  lbgk_re1000        Re 1000, plain LBGK (a smooth flow: at Re 10000 plain
                     LBGK is no longer finite after 2000 steps on this grid,
                     the failure of BGK at high Re the limiters cure)

For each: rho, u_x and u_y at every 8th site in each direction (65 x 65
sites, the corners included) and the lattice totals of mass and
H = sum f ln(f / W).

Calls only the oracle (one process per run).

    python tests/golden/make_cavity513.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "cavity513.npz")
N, U, STEPS, STRIDE = 513, 0.05, 2000, 8
RUNS = {"ehrenfest_re10000": ("ehrenfest", 10000.0, dict(topk=64, delta=1e-3)),
        "median_re10000": ("median", 10000.0, dict(delta=1e-3)),
        "lbgk_re1000": ("lbgk", 1000.0, {})}


def config(name):
    collision, re, extra = RUNS[name]
    return dict(lattice="D2Q9", nx=N, ny=N, bc="cavity", lid_u=U, nu=U * (N - 1) / re, collision=collision,
                **extra)


def run(name):
    sys.path.insert(0, ROOT)
    import oracle as O
    cfg = config(name)
    ones = np.ones((N, N))
    f = O.init_equilibrium(cfg, ones, 0 * ones, 0 * ones)
    f = O.step(cfg, f, STEPS)
    rho, ux, uy = O.macros(cfg, f)
    sub = np.s_[::STRIDE, ::STRIDE]
    return name, rho[sub], ux[sub], uy[sub], float(f.sum()), O.total_h(cfg, f)


def main():
    with mp.get_context("spawn").Pool(len(RUNS)) as pool:
        res = pool.map(run, list(RUNS))
    out = {}
    for name, rho, ux, uy, mass, H in res:
        out[f"{name}_rho"], out[f"{name}_ux"], out[f"{name}_uy"] = rho, ux, uy
        out[f"{name}_mass"], out[f"{name}_H"] = np.array(mass), np.array(H)
        out[f"{name}_re"] = np.array(RUNS[name][1])
    np.savez_compressed(OUT, n=N, u=U, steps=STEPS, stride=STRIDE, runs=np.array(list(RUNS)), **out)
    print(OUT)


if __name__ == "__main__":
    main()
