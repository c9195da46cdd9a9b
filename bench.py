#!/usr/bin/env python3
"""Benchmark of the fused D2Q9 stream-and-collide step on one or more GB300s.

Workload (the bandwidth configuration): D2Q9 lid-driven cavity 4097 x 4097,
Re = 10000, U = 0.05 (nu = U (N - 1) / Re), started from rest, FP32
populations; headline step = LBGK with the Ehrenfest limiter (k = 64,
delta = 1e-3), i.e. load/stream, moments, equilibrium, Delta S screen,
collision, limiter selection and store in one pass over the lattice.

One bench step = one lattice time step.  The state (604 MB in FP32) is far
larger than L2 (126 MB), so no flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 4097
RE, LID_U = 10000.0, 0.05
TOPK, DELTA = 64, 1e-3
METRIC = "MLUPS and % HBM peak per collision variant; adjoint grad time vs forward, 1 GB300"
Q = 9
BYTES_PER_POP = {"fp64": 8, "fp32": 4, "bf16_dev": 2, "fp16_dev": 2}


def workload_cfg(collision="ehrenfest", precision="fp32", n=N_SIDE):
    from paper_1110_0270_gb300 import workloads as WL
    cfg, init = WL.cavity(n, RE, LID_U)
    cfg.update(collision=collision, precision=precision, topk=TOPK, delta=DELTA,
               s_e=1.64, s_eps=1.64, s_q=1.2, **LIMITER_PARAMS.get(collision, {}))
    return cfg, init


# Sections 4.2-4.4 limiters in the variants table
LIMITER_PARAMS = {"smooth": dict(lim_alpha=40.0, lim_k=1.0), "double_monotonic": dict(lim_dst=2e-3, lim_k=1.5),
                  "ensemble": dict(lim_alpha=1.0, lim_k=1.0), "ensemble_lagged": dict(lim_alpha=1.0, lim_k=1.0),
                  "threshold": dict(lim_delta0=0.01)}


# DRAM bytes (read + written) per launch of the headline step kernel, from a
# one-pass ncu launch list of the full-size workload; valid only for the
# kernel sources it was taken on (their hash).
TRAFFIC_CAPTURE = {"sources_sha256_16": "18720493904ca250", "collision": "ehrenfest",
                   "precision": "fp32", "side": 4097, "bytes_per_launch": 1157.9e6}
TRAFFIC_SOURCES = ["lbm_device.cuh", "lbm_kernels.cuh", "lbm_params.h", "lbm_kernels_f32.cu"]


def captured_traffic(collision, precision, side):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1110_0270_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    c = TRAFFIC_CAPTURE
    if (h.hexdigest()[:16] == c["sources_sha256_16"] and collision == c["collision"]
            and precision == c["precision"] and side == c["side"]):
        return c["bytes_per_launch"]
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 100 ms) with host timestamps, so that only
    the samples inside the timed window are kept."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self._proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        """Median SM clock and the throttle reasons seen during [t0, t1]; a
        timed window shorter than the sampling period may hold no sample,
        and then the samples within 0.3 s of it (warm-up and the per-kernel
        pass right after, the same kernels) stand in ("samples_near")."""
        inside = [r for t, r in self.rows if t0 <= t <= t1]
        near = [r for t, r in self.rows if t0 - 0.3 <= t <= t1 + 0.3]
        pool = inside or near or [r for _, r in self.rows]
        if not pool:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        sm = [float(r[1]) for r in pool if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in pool if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in pool for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside), "samples_near": len(near), "window_s": round(t1 - t0, 3)}


# --------------------------------------------------------------------------- GPU arm
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, dist=None, device="cuda"):
    """The slowest rank's time (ms): every rank's number is the max."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(ws, sites, steps, ms):
    """Site updates of all ranks (each advances its own lattice of `sites`)
    per second of the slowest rank, in millions."""
    return ws * sites * steps / (ms * 1e-3) / 1e6


def time_steps(lat, steps, warmup, dist=None, profile=False, sampler=None):
    """Warm up, then time exactly `steps` lattice steps on the current stream
    with CUDA events, barrier + synchronize on both sides."""
    import torch
    for _ in range(warmup):
        lat.step(1)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if profile:
        lat.profile(True)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(s)
    lat.step(steps)  # one call: lbm_step replays its step graphs
    e1.record(s)
    torch.cuda.synchronize()
    t1 = time.time()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = lat.profile_read() if profile else None
    if profile:
        lat.profile(False)
    return ms, prof, (t0, t1)


def run_variants(n_side, steps, warmup, fma_per_s=None):
    """MLUPS and fraction of HBM peak per collision x precision (one GPU).
    The FP64-bound ones (ELBM's root solve, FP64 storage) also get their cost
    in FP64 FMA issue slots per site at the measured FMA rate."""
    import torch
    from paper_1110_0270_gb300 import lbm
    hbm, _ = peaks()
    out = {}
    N = n_side * n_side
    for precision in ["fp32", "fp16_dev", "bf16_dev", "fp64"]:
        for coll in ["lbgk", "ehrenfest", "median", "positivity", "mrt", "elbm", "smooth", "double_monotonic",
                     "ensemble", "ensemble_lagged", "threshold", "mrt2", "mrt_limiter"]:
            cfg, init = workload_cfg(coll, precision, n_side)
            lat = lbm.Lattice(cfg)
            lat.init(init["rho"], init["ux"], init["uy"])
            k = max(5, steps // 10) if coll == "elbm" else steps
            # the step as lbm_step runs it (graph replay), then the same
            # number of steps again with per-kernel events for the split
            ms, _, _ = time_steps(lat, k, warmup)
            _, prof, _ = time_steps(lat, k, 2, profile=True)
            per = ms / k
            mlups = N / (per * 1e-3) / 1e6
            alg = 2 * Q * BYTES_PER_POP[precision] * N
            kstep = prof["step"][1] / max(1, prof["step"][0])
            out[f"{coll}/{precision}"] = {
                "mlups": round(mlups, 1), "ms_per_step": round(per, 4),
                "hbm_frac_step": round(alg / (per * 1e-3) / 1e9 / hbm, 4),
                "hbm_frac_step_kernel": round(alg / (kstep * 1e-3) / 1e9 / hbm, 4),
                "kernel_ms": round(kstep, 5), "steps": k}
            if prof["fixup"][0]:
                out[f"{coll}/{precision}"]["fixup_ms"] = round(prof["fixup"][1] / prof["fixup"][0], 5)
            if fma_per_s and (coll == "elbm" or precision == "fp64"):
                out[f"{coll}/{precision}"]["fp64_fma_slots_per_site"] = round(fma_per_s / (mlups * 1e6), 1)
            if coll == "elbm":
                # the root finder's work: FP64 parabola steps per solved site
                # (after the FP32 pre-iterations) and the share of each outcome
                st = lat.stats()
                tot = max(1, st["elbm_solved"] + st["elbm_skipped"] + st["elbm_fallbacks"])
                out[f"{coll}/{precision}"]["elbm"] = {
                    "fp64_steps_per_solved": round(st["elbm_iters_total"] / max(1, st["elbm_solved"]), 4),
                    "fp64_steps_max": st["elbm_iters_max"], "solved_frac": round(st["elbm_solved"] / tot, 4),
                    "skipped_frac": round(st["elbm_skipped"] / tot, 4),
                    "fallback_frac": round(st["elbm_fallbacks"] / tot, 6)}
            del lat
            torch.cuda.empty_cache()
    return out


def random_start(n, seed=7):
    """Equilibrium at a seeded random density and velocity field (rho
    1 +- 0.02, u components uniform in +-0.05): after the first streaming
    every site is out of equilibrium, so the per-site work the rest state
    skips (the ELBM root solve, the limiters' candidates) runs everywhere."""
    from paper_1110_0270_gb300 import workloads as WL
    return WL.random_fields(n, n, seed, 0.02, 0.05)


def run_elbm_loaded(n_side, steps=5):
    """ELBM with every site solved: the 4097^2 cavity started from the random
    velocity field of random_start (the variants table starts from rest,
    where the near-equilibrium skip takes most sites), FP32 and FP64 storage:
    MLUPS, FP64 parabola steps per solved site (after the FP32
    pre-iterations) and the share of solved / skipped / fallback sites."""
    import torch
    from paper_1110_0270_gb300 import lbm
    out = {}
    init = random_start(n_side)
    for precision in ["fp32", "fp64"]:
        cfg, _ = workload_cfg("elbm", precision, n_side)
        lat = lbm.Lattice(cfg)
        lat.init(init["rho"], init["ux"], init["uy"])
        lat.step(2)
        st0 = lat.stats()
        ms, _, _ = time_steps(lat, steps, 1)
        st = lat.stats()
        d = {k: st[k] - st0[k] for k in ("elbm_solved", "elbm_skipped", "elbm_fallbacks", "elbm_iters_total")}
        tot = max(1, d["elbm_solved"] + d["elbm_skipped"] + d["elbm_fallbacks"])
        out[precision] = {"mlups": round(n_side * n_side * steps / (ms * 1e-3) / 1e6, 1),
                          "ms_per_step": round(ms / steps, 3),
                          "fp64_steps_per_solved": round(d["elbm_iters_total"] / max(1, d["elbm_solved"]), 4),
                          "solved_frac": round(d["elbm_solved"] / tot, 4),
                          "skipped_frac": round(d["elbm_skipped"] / tot, 4),
                          "fallback_frac": round(d["elbm_fallbacks"] / tot, 6)}
        del lat
        torch.cuda.empty_cache()
    return out


def run_loaded_selection(n_side, hots=(300, 3000, 30000), reps=5):
    """The headline lattice (4097^2, FP32) one step after lbm_set_state of
    the cavity at rest with `hot` random sites perturbed (each population
    times exp(0.3 N(0, 1))): the Ehrenfest (k = 64) and median steps with
    hundreds to tens of thousands of screened sites, so that the grid-wide
    FP64 Delta S pass, the radix selection and the median windows are
    timed, not only the settled-in-FP32 few-candidate path of a flow
    started from rest.  Per case the median of `reps` single steps (step
    kernel and follow-up, CUDA events per kernel)."""
    import torch
    from paper_1110_0270_gb300 import lbm
    w = np.array([4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36], np.float32)
    base = np.broadcast_to(w[:, None, None], (9, n_side, n_side))
    rng = np.random.default_rng(17)
    out = {}
    for coll in ["ehrenfest", "median"]:
        cfg, _ = workload_cfg(coll, "fp32", n_side)
        lat = lbm.Lattice(cfg)
        rows = []
        for hot in hots:
            f = np.array(base)
            ys, xs = rng.integers(2, n_side - 2, hot), rng.integers(2, n_side - 2, hot)
            f[:, ys, xs] *= np.exp(0.3 * rng.standard_normal((9, hot))).astype(np.float32)
            ft = torch.from_numpy(f).cuda()
            del f
            times = []
            for _ in range(reps):
                lat.set_state(ft)
                torch.cuda.synchronize()
                lat.profile(True)
                lat.step(1)
                prof = lat.profile_read()
                lat.profile(False)
                times.append((prof["step"][1], prof["fixup"][1]))
            st = lat.stats()
            times.sort(key=lambda t: t[0] + t[1])
            k_ms, f_ms = times[len(times) // 2]
            rows.append({"hot_sites": hot, "screened": st["screened_last"], "candidates": st["candidates_last"],
                         "limited": st["limited_total"], "step_kernel_ms": round(k_ms, 5),
                         "followup_ms": round(f_ms, 5), "ms_per_step": round(k_ms + f_ms, 5),
                         "mlups": round(n_side * n_side / ((k_ms + f_ms) * 1e-3) / 1e6, 1)})
            del ft
        out[coll] = rows
        del lat
        torch.cuda.empty_cache()
    return out


GOLDEN_513 = os.path.join(ROOT, "tests", "golden", "cavity513.npz")


PRECISION_RUNS = {"ehrenfest_re10000": ("ehrenfest", dict(topk=64, delta=1e-3)),
                  "median_re10000": ("median", dict(delta=1e-3)), "lbgk_re1000": ("lbgk", {})}


def run_precision_error():
    """Storage-precision error of the bandwidth configuration against the
    FP64 oracle, on the reduced 513 x 513 run that stands for it (U 0.05,
    2000 steps from rest): each storage format's GPU run against the
    oracle's fields stored by tests/golden/make_cavity513.py (rho, u at every
    8th site, totals of mass and H), for Re 10000 with the Ehrenfest and
    median limiters (plain LBGK diverges there) and for plain LBGK at Re
    1000: rel-L2 of rho - 1 and of u on the sampled sites, relative errors of
    the total mass, of H = sum f ln(f / W) and of its Kullback form
    H_K = sum (f ln(f / W) - f + W) = H - (mass - N), which leaves out the
    mass term (the oracle's own FP64 mass rounding dominates H's error in
    FP64 storage).

    The rows "fp64_perturbed_<eps>" run FP64 storage from the same rest state
    with every initial population multiplied by (1 + eps z), z ~ N(0, 1)
    (seeded), eps = 1e-12 and 6e-8 (FP32's relative rounding): how the flow
    answers one small perturbation.  Under the Ehrenfest step at Re 10000 any
    perturbation changes the fields at O(1): the symmetric start has exact
    ties in Delta S, broken by site index, and a perturbation breaks them
    differently."""
    import torch
    from paper_1110_0270_gb300 import lbm
    from paper_1110_0270_gb300 import workloads as WL
    g = np.load(GOLDEN_513)
    n, u0, steps, stride = int(g["n"]), float(g["u"]), int(g["steps"]), int(g["stride"])
    out = {"reference": "FP64 oracle (tests/golden/cavity513.npz)", "lattice": f"{n}x{n}", "u": u0,
           "steps": steps, "sample_stride": stride}
    nrm = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    sub = np.s_[::stride, ::stride]
    variants = [(p, None) for p in ["fp64", "fp32", "fp16_dev", "bf16_dev"]]
    variants += [("fp64", eps) for eps in (1e-12, 6e-8)]
    for run, (coll, extra) in PRECISION_RUNS.items():
        re = float(g[f"{run}_re"])
        m_ref, H_ref = float(g[f"{run}_mass"]), float(g[f"{run}_H"])
        HK_ref = H_ref - (m_ref - n * n)
        rows = {"re": re, "collision": coll}
        for precision, eps in variants:
            cfg, init = WL.cavity(n, re, u0)
            cfg.update(collision=coll, precision=precision, **extra)
            lat = lbm.Lattice(cfg)
            lat.init(init["rho"], init["ux"], init["uy"])
            if eps is not None:
                f0 = lat.get_state(torch.float64)
                z = torch.from_numpy(WL.normal_noise(tuple(f0.shape), 2024, 1.0)).to(f0.device)
                lat.set_state(f0 * (1.0 + eps * z))
            lat.step(steps)
            rho, u = lat.macros(torch.float64)
            rho, u = rho.cpu().numpy(), u.cpu().numpy()
            mass = float(lat.get_state(torch.float64).sum())
            H = lat.entropy()
            HK = H - (mass - n * n)
            key = precision if eps is None else f"fp64_perturbed_{eps:g}"
            rows[key] = {
                "rho_dev_rel_l2": nrm(rho[sub] - 1.0, g[f"{run}_rho"] - 1.0),
                "u_rel_l2": nrm(np.stack([u[0][sub], u[1][sub]]), np.stack([g[f"{run}_ux"], g[f"{run}_uy"]])),
                "mass_rel": abs(mass - m_ref) / m_ref,
                "H_rel": abs(H - H_ref) / abs(H_ref),
                "HK_rel": abs(HK - HK_ref) / abs(HK_ref),
                "limited_total": lat.stats()["limited_total"]}
            del lat
        out[run] = rows
    return out


def run_shear_decay(res=(10, 30, 100, 300, 1000, 3000, 10000), Ls=(50, 100), u0=0.05):
    """Section 7's shear-decay experiment on the GPU (FP64 storage, textbook
    polynomial equilibrium): L + 1 periodic sites a side, u_y = u0 sin(2 pi x/L),
    L / u0 steps; lambda = -(L^2 / (nu t)) ln(a(t) / a(0)) from the amplitude a
    of the sin(2 pi x / L) component of u_y, for LBGK, the aggressive MRT A_2 and
    the A_1 MRT with the Lallemand-Luo rates (s_e 1.64, s_eps 1.54,
    s_q = 3 (2 - s_nu)/(3 - s_nu)).  The exact decay has lambda = 4 pi^2."""
    import numpy as np
    import torch
    from paper_1110_0270_gb300 import lbm
    from paper_1110_0270_gb300 import workloads as WL
    out = {"lambda_exact": round(4 * math.pi ** 2, 4), "steps": "L / u0", "table": {}}
    for name, coll in [("lbgk", "lbgk"), ("mrt_a2", "mrt2"), ("mrt_a1_ll", "mrt")]:
        rows = {}
        for L in Ls:
            vals = []
            for re in res:
                cfg, init = WL.shear_decay(L, re, u0)
                beta = 1.0 / (6.0 * cfg["nu"] + 1.0)
                cfg.update(collision=coll, precision="fp64", equilibrium="poly_std", beta=beta)
                if coll == "mrt":
                    cfg.update(lbm.mrt_rates("mrt_ll", beta))
                lat = lbm.Lattice(cfg)
                lat.init(init["rho"], init["ux"], init["uy"])
                n = cfg["nx"]
                s = np.sin(2 * math.pi * np.arange(n) / L)
                amp = lambda: float((lat.macros(torch.float64)[1][1].cpu().numpy().mean(0) * s).sum() / (s * s).sum())
                a0 = amp()
                T = int(round(L / u0))
                lat.step(T)
                ratio = amp() / a0
                # a non-positive or non-finite amplitude: the run went unstable
                lam = round(-(L * L) / (cfg["nu"] * T) * math.log(ratio), 3) if ratio > 0 and math.isfinite(ratio) else None
                vals.append([re, lam])
                del lat
            rows[str(L)] = vals
        out["table"][name] = rows
    out["columns"] = ["Re", "lambda"]
    return out


def batched_configs(precision="fp32", seed=0, n=512):
    """The batched configuration: n cavities with seeded sides (64..768) and
    Reynolds numbers (log-uniform 100..20000), lid speed 0.1, collisions
    cycling LBGK / ELBM / Ehrenfest (k = 64) / median."""
    from paper_1110_0270_gb300 import workloads as WL
    out = []
    for inst in WL.batched_cavities(n=n, seed=seed):
        cfg, _ = WL.cavity(inst["side"], inst["re"], 0.1)
        cfg.update(collision=inst["collision"], precision=precision, topk=TOPK, delta=DELTA)
        out.append(cfg)
    return out


def run_batched(steps, warmup, fp64_mlups=None, separate=True, tune=True):
    """The batched configuration (512 cavities, FP32): aggregate MLUPS of the
    persistent batched kernels with the default launch options and with the
    options the library's autotuner picks (its sweep recorded), the time and
    HBM fraction of each collision group advanced alone, and the same
    instances run as separate single-lattice contexts (one lbm_step per
    instance per step)."""
    import torch
    from paper_1110_0270_gb300 import lbm
    hbm, _ = peaks()
    cfgs = batched_configs()
    sites = sum(c["nx"] * c["ny"] for c in cfgs)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(opts):
        b = lbm.Batch(cfgs, opts=opts)
        b.init_uniform(1.0, 0.0, 0.0)
        b.step(warmup)
        torch.cuda.synchronize()
        e0.record(s)
        b.step(steps)
        e1.record(s)
        torch.cuda.synchronize()
        return b, e0.elapsed_time(e1) / steps

    b, ms = timed(None)
    status = b.step(0, status=True)
    group_sites = {}
    for c in cfgs:
        group_sites[c["collision"]] = group_sites.get(c["collision"], 0) + c["nx"] * c["ny"]
    gt = b.group_times(steps)
    groups = {}
    for k, t in gt.items():
        per = t / steps
        groups[k] = {"instances": sum(1 for c in cfgs if c["collision"] == k), "sites": group_sites[k],
                     "ms_per_step": round(per, 4), "mlups": round(group_sites[k] / (per * 1e-3) / 1e6, 1),
                     "hbm_frac": round(72 * group_sites[k] / (per * 1e-3) / 1e9 / hbm, 4)}
    out = {"instances": len(cfgs), "sites": sites, "steps": steps, "ms_per_step": round(ms, 4),
           "mlups": round(sites / (ms * 1e-3) / 1e6, 1),
           "hbm_frac_if_all_streaming": round(72 * sites / (ms * 1e-3) / 1e9 / hbm, 4),
           "diverged_instances": sum(1 for v in status if v != "LBM_OK"),
           "opts": b.opts, "groups": groups,
           "note": "persistent kernels (HBM-bound collisions; ELBM) on parallel branches of a CUDA graph; "
                   "groups: each collision's instances alone, HBM fraction at 72 B per site update"}
    del b
    torch.cuda.empty_cache()
    def tuned():
        t0 = time.perf_counter()
        opts, sweep = lbm.tune_batch(cfgs, steps=2)
        tb, tms = timed(opts)
        tg = tb.group_times(steps)
        del tb
        torch.cuda.empty_cache()
        return {"opts": opts, "ms_per_step": round(tms, 4), "mlups": round(sites / (tms * 1e-3) / 1e6, 1),
                "tune_s": round(time.perf_counter() - t0, 2),
                "groups_hbm_frac": {k: round(72 * group_sites[k] / (t / steps * 1e-3) / 1e9 / hbm, 4)
                                    for k, t in tg.items()},
                "sweep": [[o["tile_x"], o["tile_rows"], o["ctas_per_sm"], o["chunk"], o["order"], round(m, 4),
                           round(r, 4)] for o, m, r in sweep],
                "sweep_columns": ["tile_x", "tile_rows", "ctas_per_sm", "chunk", "order",
                                  "groups_ms_per_step_summed", "objective_mean_relative_group_time"]}

    if tune:
        guarded(out, "tuned", tuned)
    if separate:
        lats = []
        for c in cfgs:
            lat = lbm.Lattice(c)
            ny, nx = c["ny"], c["nx"]
            lat.init(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
            lats.append(lat)
        for lat in lats:
            lat.step(warmup)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(steps):
            for lat in lats:
                lat.step(1)
        e1.record(s)
        torch.cuda.synchronize()
        ms_sep = e0.elapsed_time(e1) / steps
        out["separate_ms_per_step"] = round(ms_sep, 4)
        out["speedup_vs_separate"] = round(ms_sep / ms, 3)
        del lats
        torch.cuda.empty_cache()
    if fp64_mlups:
        out["vs_fp64_lbgk_step"] = round(out["mlups"] / fp64_mlups, 3)
    return out


def run_small_configs(tube_steps=400, cavity_steps=2000):
    """The two small configurations, timed through lbm_step (which replays
    its two-step CUDA graph): the D1Q3 shock tube (800 sites, FP64, 400
    steps, mu s per step) and the 257^2 cavity (Re 5000, U 0.1, FP64 and
    FP32, MLUPS; its 2.4-4.8 MB state stays in L2)."""
    import torch
    from paper_1110_0270_gb300 import lbm
    from paper_1110_0270_gb300 import workloads as WL
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_steps(lat, n):
        lat.step(2)
        torch.cuda.synchronize()
        e0.record(s)
        lat.step(n)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {"tube_us_per_step": {}, "cavity257_mlups": {}}
    cfg, init = WL.shock_tube(800, 1e-9)
    for coll in ["lbgk", "elbm", "ehrenfest", "median", "mrt"]:
        lat = lbm.Lattice(dict(cfg, collision=coll, precision="fp64", topk=4, delta=1e-3))
        lat.init(init["rho"], init["ux"])
        out["tube_us_per_step"][coll] = round(timed_steps(lat, tube_steps) * 1e3 / tube_steps, 3)
    cfg, init = WL.cavity(257, 5000.0, 0.1)
    for prec in ["fp64", "fp32"]:
        for coll in ["lbgk", "elbm", "ehrenfest", "median", "mrt"]:
            lat = lbm.Lattice(dict(cfg, collision=coll, precision=prec, topk=64, delta=1e-3,
                                   s_e=1.64, s_eps=1.64, s_q=1.2))
            lat.init(init["rho"], init["ux"], init["uy"])
            n = cavity_steps if coll != "elbm" else cavity_steps // 4
            ms = timed_steps(lat, n)
            key = f"{coll}/{prec}"
            out["cavity257_mlups"][key] = round(257 * 257 * n / (ms * 1e-3) / 1e6, 1)
            if lat.stats()["diverged"]:
                out.setdefault("cavity257_diverged", []).append(key)
    return out


def run_adjoint(T=4000, K=100, n=513, fd=True, collision="ehrenfest"):
    """The adjoint configuration: D2Q9 cavity n^2, Re 1000, U 0.1, FP32, with
    the Ehrenfest limiter (k = 32) or the median filter (delta = 1e-3),
    f0 = equilibrium at rest + N(0, 1e-4) noise; gradient of the kinetic
    energy after T steps with respect to U, beta and f0, checkpoints every K
    steps.  Reports backward / forward time and the central differences
    (h = 1e-3, Richardson with h/2) of FP64 forward runs, with a flag when a
    perturbed run limited a different number of sites than the base run
    (the difference then crosses a selection boundary)."""
    import torch
    from paper_1110_0270_gb300 import lbm
    from paper_1110_0270_gb300 import workloads as WL
    cfg, init = WL.cavity(n, 1000.0, 0.1)
    cfg.update(collision=collision, topk=32, delta=1e-3, precision="fp32")
    beta = 1.0 / (6.0 * cfg["nu"] + 1.0)
    cfg["beta"] = beta
    lat = lbm.Lattice(cfg)
    lat.init(init["rho"], init["ux"], init["uy"])
    f0 = (lat.get_state(torch.float64) + torch.tensor(
        WL.normal_noise((9, n, n), 5, 1e-4), device="cuda")).float()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    work = lat.adjoint_work(T, K)
    lat.set_state(f0)
    lat.adjoint_forward(T, K, work)  # warm-up of both passes
    lat.adjoint_backward(T, K, work)
    lat.set_state(f0)
    (J, _), t_f = timed(lambda: lat.adjoint_forward(T, K, work))
    limited = lat.stats()["limited_total"]
    (g, gU, gB), t_b = timed(lambda: lat.adjoint_backward(T, K, work))
    lim = "Ehrenfest k=32" if collision == "ehrenfest" else "median filter delta=1e-3"
    out = {"config": f"D2Q9 cavity {n}^2, Re 1000, U 0.1, FP32, {lim}, T={T}, K={K}",
           "J": J, "dJ_dU": gU, "dJ_dbeta": gB, "forward_s": round(t_f, 4),
           "backward_s": round(t_b, 4), "backward_over_forward": round(t_b / t_f, 3),
           "work_bytes": int(work.numel()), "limited_sites": limited}
    if fd:
        f64 = f0.double()
        crossed = []

        def ke(**kw):
            l2 = lbm.Lattice(dict(cfg, precision="fp64", **kw))
            l2.set_state(f64)
            J2 = l2.adjoint_forward(T, T)[0]
            crossed.append(l2.stats()["limited_total"])
            return J2

        def cd(key, x0, h):
            d = lambda hh: (ke(**{key: x0 + hh}) - ke(**{key: x0 - hh})) / (2 * hh)
            return (4 * d(h / 2) - d(h)) / 3

        base = lbm.Lattice(dict(cfg, precision="fp64"))
        base.set_state(f64)
        base.adjoint_forward(T, T)
        lim0 = base.stats()["limited_total"]
        fdU, fdB = cd("lid_u", 0.1, 1e-3), cd("beta", beta, 1e-3)
        out.update(fd_dJ_dU=fdU, fd_dJ_dbeta=fdB, rel_err_U=abs(gU - fdU) / abs(fdU),
                   rel_err_beta=abs(gB - fdB) / abs(fdB),
                   fd_branch_crossing=any(c != lim0 for c in crossed))
    return out


def e2e_measure(cfg, init, jobs=6, inner=100, dist=None, ws=1):
    """End to end through the public API with host buffers: per job,
    lbm_init from pinned host rho/u (H2D), `inner` steps, lbm_macros and a
    D2H copy of rho and u into pinned host memory.  Two lattices on two CUDA
    streams take the jobs in turn, so that one job's copies overlap the other
    job's steps (as a caller running independent jobs would); the timed
    region covers `jobs` whole jobs, every copy included, after two untimed
    ones.  With several ranks every rank runs its own jobs at the same time;
    the time is the slowest rank's and the value counts the sites of all
    ranks."""
    import torch
    from paper_1110_0270_gb300 import lbm
    lats = [lbm.Lattice(cfg) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in init.items()}
    ny, nx = init["rho"].shape
    outs = [(torch.empty((ny, nx), dtype=torch.float32).pin_memory(),
             torch.empty((2, ny, nx), dtype=torch.float32).pin_memory()) for _ in range(2)]

    def job(k):
        s, lat, (out_rho, out_u) = streams[k % 2], lats[k % 2], outs[k % 2]
        with torch.cuda.stream(s):
            lat.init(host["rho"].numpy(), host["ux"].numpy(), host["uy"].numpy(), stream=s)
            lat.step(inner, stream=s)
            rho, u = lat.macros(torch.float32, stream=s)
            out_rho.copy_(rho, non_blocking=True)
            out_u.copy_(u, non_blocking=True)

    for k in range(2):  # warms the pinned buffers and both lattices
        job(k)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(jobs):
        job(k)
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t0) * 1e3, dist) * 1e-3
    N = nx * ny
    return {"value": round(whole_job_mlups(ws, N, inner * jobs, dt * 1e3), 1), "unit": "MLUPS",
            "h2d_bytes_per_step": int(3 * 8 * N), "d2h_bytes_per_step": int(3 * 4 * N),
            "steps_per_job": inner, "jobs": jobs,
            "note": "one e2e step = lbm_init from pinned host rho,u + 100 lattice steps + lbm_macros + D2H "
                    "of rho,u; two lattices on two streams take the jobs in turn (copies of one job overlap "
                    "the steps of the other)"}


def cpu_baseline(budget_s=12.0):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of
    the workload: a smaller cavity of the same Re and U, same collision."""
    import oracle as O
    n = 1025
    cfg, init = workload_cfg("ehrenfest", "fp64", n)
    f = O.init_equilibrium(cfg, init["rho"], init["ux"], init["uy"])
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        f = O.step(cfg, f, 1)
        steps += 1
    t = time.perf_counter() - t0
    return {"value": round(n * n * steps / t / 1e6, 3), "unit": "MLUPS", "cores": 1,
            "kind": "oracle",
            "sample": f"D2Q9 cavity {n}x{n} (1/16 of the 4097^2 sites), Re {RE:g}, U {LID_U}, "
                      f"Ehrenfest k={TOPK} delta={DELTA:g}, FP64, {steps} steps, "
                      f"{os.cpu_count()} host cores present, 1 used",
            "host": host_cpu(), "per_config": oracle_configs()}


def host_cpu():
    """CPU model line of this host (Linux /proc/cpuinfo), or the machine type."""
    import platform
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    v = line.split(":", 1)[1].strip()
                    v = {"0xd4f": "Neoverse V2 (0xd4f)"}.get(v, v)
                    return f"{platform.machine()} {v}, {os.cpu_count()} cores"
    except OSError:
        pass
    return f"{platform.machine()}, {os.cpu_count()} cores"


def oracle_configs(budget_s=2.0):
    """Single-thread oracle MLUPS on the shock tube (800 sites, LBGK), the
    257^2 cavity (Re 5000, U 0.1, LBGK) and the adjoint configuration's
    forward step (513^2, Re 1000, U 0.1, Ehrenfest k = 32), each for about
    budget_s seconds of steps."""
    import oracle as O
    from paper_1110_0270_gb300 import workloads as WL
    out = {}
    cases = [("tube_800_lbgk", *WL.shock_tube(800)), ("cavity_257_lbgk", *WL.cavity(257, 5000.0, 0.1)),
             ("adjoint_513_ehrenfest_forward", *WL.cavity(513, 1000.0, 0.1))]
    for name, cfg, init in cases:
        cfg = dict(cfg, precision="fp64", collision="ehrenfest" if "ehrenfest" in name else "lbgk",
                   topk=32, delta=1e-3)
        f = O.init_equilibrium(cfg, init["rho"], init["ux"], None if cfg["lattice"] == "D1Q3" else init["uy"])
        t0, steps = time.perf_counter(), 0
        while time.perf_counter() - t0 < budget_s:
            f = O.step(cfg, f, 10 if cfg["nx"] * cfg["ny"] < 10000 else 1)
            steps += 10 if cfg["nx"] * cfg["ny"] < 10000 else 1
        t = time.perf_counter() - t0
        out[name] = round(cfg["nx"] * cfg["ny"] * steps / t / 1e6, 3)
    out["unit"] = "MLUPS, FP64 oracle, 1 thread"
    return out


def gpu_arm(args):
    import torch
    from paper_1110_0270_gb300 import build as B
    from paper_1110_0270_gb300 import lbm

    ws, rank, local = dist_setup()
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    cfg, init = workload_cfg(args.collision, args.precision, args.side)
    if args.init == "random":
        init = random_start(args.side)
    N = args.side * args.side
    lat = lbm.Lattice(cfg)
    lat.init(init["rho"], init["ux"], init["uy"])
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    # the timed region replays lbm_step's graphs as a user's call does; the
    # per-kernel split (roofline) comes from the same number of steps right
    # after it, launched one kernel at a time between CUDA events
    ms, _, (t0, t1) = time_steps(lat, args.steps, args.warmup, dist)
    if sampler:
        time.sleep(0.25)
        sampler.stop()
    _, prof, _ = time_steps(lat, args.steps, 0, dist, profile=True)
    ms = max_over_ranks(ms, dist)
    st = lat.stats()
    per = ms / args.steps
    value = whole_job_mlups(ws, N, args.steps, ms)
    hbm, peak_kind = peaks()
    alg = 2 * Q * BYTES_PER_POP[args.precision] * N  # bytes per launch of the fused step kernel
    k_ms = prof["step"][1] / max(1, prof["step"][0])
    achieved = alg / (k_ms * 1e-3) / 1e9
    launches = prof["step"][0] + prof["fixup"][0]
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16_dev": "bf16", "fp16_dev": "f16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"D2Q9 lid-driven cavity {args.side}x{args.side}, Re {RE:g}, "
                               f"U {LID_U}, {args.precision} populations, collision {args.collision}"
                               f" (Ehrenfest/median: k={TOPK}, delta={DELTA:g}), started "
                               + ("from rest" if args.init == "rest" else "from a random velocity field"),
                   "sites": N, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (state 604 MB in FP32), no flush",
                   "limiter_sites_total": st["limited_total"],
                   "last_step_candidates": st["candidates_last"],
                   "last_step_screened": st["screened_last"]},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": captured_traffic(args.collision, args.precision, args.side),
                     "kernel": f"step_kernel<D2Q9, {args.precision}, {args.collision}>",
                     "algorithmic_bytes_per_launch": alg,
                     "kernel_ms": round(k_ms, 5), "peak_kind": f"{peak_kind} hbm_gbs",
                     "fixup_ms": round(prof["fixup"][1] / max(1, prof["fixup"][0]), 5)},
        "gpu_launches": launches,
    }
    if not args.no_e2e:  # every rank at once
        guarded(result, "e2e", lambda: e2e_measure(cfg, init, dist=dist, ws=ws))
    if rank == 0:
        result["clocks"] = sampler.summary(t0, t1) if sampler else None
        run_sections(args, result, init)
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def guarded(result, key, fn):
    """One optional section of the JSON line; a failure is recorded there
    instead of ending the run without the headline line."""
    try:
        result[key] = fn()
    except Exception as e:  # noqa: BLE001
        result[key] = {"error": f"{type(e).__name__}: {e}"}


def run_sections(args, result, init):
    from paper_1110_0270_gb300 import lbm
    if not args.no_variants:
        r = {}
        guarded(result, "fp64_probe", lambda: r.update(lbm.fp64_rates()) or {
            "dfma_tflops": round(r["dfma_flops"] / 1e12, 4), "log_gops": round(r["log_per_s"] / 1e9, 2),
            "note": "measured FP64 ceilings of the FP64-bound kernels"})
        guarded(result, "variants",
                lambda: run_variants(args.side, args.variant_steps, 3, r.get("dfma_flops", 0) / 2 or None))
    if not args.no_small:
        guarded(result, "small_configs", run_small_configs)
    if not args.no_variants:
        guarded(result, "loaded_selection", lambda: run_loaded_selection(args.side))
        guarded(result, "elbm_loaded", lambda: run_elbm_loaded(args.side))
    if args.precision_steps > 0 and os.path.exists(GOLDEN_513):
        guarded(result, "precision_error", run_precision_error)
    if not args.no_small:
        guarded(result, "shear_decay", run_shear_decay)
    if args.adjoint_steps > 0:
        guarded(result, "adjoint", lambda: run_adjoint(args.adjoint_steps, 100))
        guarded(result, "adjoint_median", lambda: run_adjoint(args.adjoint_steps, 100, collision="median"))
    if args.batch_steps > 0:
        fp64 = (result.get("variants") or {}).get("lbgk/fp64", {}).get("mlups")
        guarded(result, "batched", lambda: run_batched(args.batch_steps, 3, fp64))
    if not args.no_cpu:
        guarded(result, "cpu_baseline", lambda: cpu_baseline(args.cpu_budget))


# --------------------------------------------------------------------------- reference arm
def reference_arm(args):
    """The FP64 oracle on the host cores, same metric and unit; each step is
    one oracle step of a smaller cavity sized so that the whole run stays
    within about `budget` seconds."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O
    budget = args.ref_budget
    total = args.steps + args.warmup
    # the oracle's Ehrenfest FP64 step runs at roughly 0.7 MLUPS on one core
    sites = max(65 * 65, int(0.7e6 * budget / max(1, total)))
    n = int(min(args.side, max(65, int(sites ** 0.5))))
    cfg, init = workload_cfg("ehrenfest", "fp64", n)
    f = O.init_equilibrium(cfg, init["rho"], init["ux"], init["uy"])
    for _ in range(args.warmup):
        f = O.step(cfg, f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.step(cfg, f, 1)
    t = time.perf_counter() - t0
    value = n * n * args.steps / t / 1e6
    sample = (f"D2Q9 cavity {n}x{n} per step (a bounded sample of the {args.side}^2 workload), "
              f"Ehrenfest k={TOPK}, FP64 oracle, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"D2Q9 lid-driven cavity {args.side}x{args.side}, Re {RE:g}, "
                               f"U {LID_U}, LBGK + Ehrenfest limiter (k={TOPK}, delta={DELTA:g})"},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--side", type=int, default=N_SIDE)
    ap.add_argument("--collision", default="ehrenfest",
                    choices=["lbgk", "elbm", "ehrenfest", "positivity", "median", "mrt", "smooth",
                             "double_monotonic", "ensemble", "ensemble_lagged", "threshold", "mrt2",
                             "mrt_limiter"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16_dev", "bf16_dev"])
    ap.add_argument("--init", default="rest", choices=["rest", "random"],
                    help="start the timed lattice from rest (the workload) or from random_start (profiling)")
    ap.add_argument("--variant-steps", type=int, default=100)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the tube and 257^2 runs")
    ap.add_argument("--precision-steps", type=int, default=1,
                    help="0 skips the storage-precision comparison against the oracle's 513^2 fields")
    ap.add_argument("--adjoint-steps", type=int, default=4000,
                    help="T of the adjoint run (0 skips it)")
    ap.add_argument("--batch-steps", type=int, default=20,
                    help="steps of the 512-cavity batched run (0 skips it)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=90.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
