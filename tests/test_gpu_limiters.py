"""GPU-vs-oracle parity of the Section 4.2-4.4 limiters through the C ABI:
smooth (Eq. smoothReg), double monotonic (Eq. DoublMonSpec), ensemble
dependent (Eq. phiExamp, the lattice mean of Delta S from a pre-pass, or
lagged: the previous step's mean, accumulated by that step) and
the threshold limiter (Eqs. EntThresh, entrHom: step-wide sum of Delta S,
then Delta S_t from the candidates).  FP64 storage within 1e-12 rel-L2,
FP32 within 1e-5; the threshold limiter's corrected-site count is exact in
FP64."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}

CASES = {
    "cavity": dict(lattice="D2Q9", nx=37, ny=29, bc="cavity", lid_u=0.1),
    "periodic": dict(lattice="D2Q9", nx=33, ny=17, bc="periodic"),
    "wide": dict(lattice="D2Q9", nx=200, ny=12, bc="cavity", lid_u=0.1),
    "tube": dict(lattice="D1Q3", nx=301, ny=1, bc="ends"),
}

PARAMS = {
    "smooth": dict(lim_alpha=40.0, lim_k=1.0, beta=0.95),
    "double_monotonic": dict(lim_dst=2e-3, lim_k=1.5, beta=0.95),
    "ensemble": dict(lim_alpha=1.0, lim_k=1.0, beta=0.8),
    # E(Delta S) of the previous step (accumulated by the step kernel)
    "ensemble_lagged": dict(lim_alpha=1.0, lim_k=1.0, beta=0.8),
    "threshold": dict(lim_delta0=0.05, delta=1e-4, beta=0.95),
}


def state(cfg, seed=5):
    ny, nx = cfg["ny"], cfg["nx"]
    fl = WL.random_fields(ny, nx, seed, 0.05, 0.05)
    f = O.init_equilibrium(dict(cfg, collision="lbgk"), fl["rho"], fl["ux"],
                           None if cfg["lattice"] == "D1Q3" else fl["uy"])
    f = f * WL.lognormal_factors(f.shape, seed + 1, 0.01)
    return f * WL.lognormal_factors(f.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, 12, 0.4)[None])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("collision", list(PARAMS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_limiters_match_oracle(case, collision, precision):
    cfg = dict(CASES[case], collision=collision, precision=precision, **PARAMS[collision])
    f0 = state(cfg)
    if precision != "fp64":
        f0 = f0.astype(np.float32).astype(np.float64)
    n = 201
    lat = lbm.Lattice(cfg)
    dt = torch.float64 if precision == "fp64" else torch.float32
    lat.set_state(torch.tensor(f0, dtype=dt, device="cuda"))
    lat.step(n)
    g = lat.get_state(torch.float64).cpu().numpy()
    f, st = O.step(cfg, f0, n, stats=True)
    assert rel(g, f) < TOL[precision], rel(g, f)
    gs = lat.stats()
    assert gs["diverged"] == 0
    if collision == "threshold" and precision == "fp64":
        assert gs["limited_total"] == st["limited_sites"] > 0


@pytest.mark.parametrize("collision,params", [
    ("smooth", dict(lim_alpha=40.0, lim_k=1.3, beta=0.95)),
    ("smooth", dict(lim_alpha=5.0, lim_k=2.0, beta=0.95)),
    ("double_monotonic", dict(lim_dst=2e-3, lim_k=0.7, beta=0.95)),
    ("double_monotonic", dict(lim_dst=2e-3, lim_k=1.0, beta=0.95)),
    ("ensemble", dict(lim_alpha=1.0, lim_k=1.3, beta=0.8)),
    ("ensemble", dict(lim_alpha=1.0, lim_k=0.5, beta=0.8)),
])
def test_limiter_exponents_fp32(collision, params):
    """Exponents k off the exact FP32 forms of the limiter powers (the
    exp2 / log2 evaluation) and on them (k = 2; the ensemble's k - 1/2 = 0;
    the double-monotonic outer power -1/(2k) = -1/2), FP32 storage against
    the oracle over 201 steps."""
    cfg = dict(CASES["cavity"], collision=collision, precision="fp32", **params)
    f0 = state(cfg).astype(np.float32).astype(np.float64)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, dtype=torch.float32, device="cuda"))
    lat.step(201)
    g = lat.get_state(torch.float64).cpu().numpy()
    assert rel(g, O.step(cfg, f0, 201)) < TOL["fp32"]


def test_threshold_budget_and_delta_floor():
    """The threshold limiter in both regimes: Delta S_0 above delta (the
    budget delta0 sets the threshold) and below it (Delta S_t = delta), one
    step each, FP64, against the oracle; with delta0 = 0 and delta above
    every Delta S it is the LBGK step."""
    base = dict(CASES["cavity"], collision="threshold", precision="fp64", beta=0.95)
    f0 = state(base, seed=9)
    dS = O.delta_s_field(base, f0)
    for delta0, delta in [(0.05, 1e-5), (1e-6, 1e-3), (0.0, 1e3)]:
        cfg = dict(base, lim_delta0=delta0, delta=delta)
        d0 = O.threshold_dS0(dS, delta0, 0.95)
        lat = lbm.Lattice(cfg)
        lat.set_state(torch.tensor(f0, device="cuda"))
        lat.step(1)
        g = lat.get_state(torch.float64).cpu().numpy()
        assert rel(g, O.step(cfg, f0, 1)) < 1e-13, (delta0, delta, d0)
        if delta == 1e3:
            assert rel(g, O.step(dict(cfg, collision="lbgk"), f0, 1)) < 1e-13
            assert lat.stats()["limited_total"] == 0
        else:
            ds, site, sel = lat.last_candidates()
            dst = max(d0, delta)
            assert sorted(site[sel == 1].tolist()) == sorted(np.flatnonzero(dS.ravel() >= dst).tolist())


def test_threshold_many_candidates_radix_path():
    """delta = 0: every site is a candidate (the multi-CTA evaluation and the
    radix descent over thousands of values), FP64, against the oracle."""
    cfg = dict(lattice="D2Q9", nx=96, ny=80, bc="periodic", collision="threshold", precision="fp64",
               beta=0.9, lim_delta0=0.02, delta=0.0)
    f0 = state(cfg, seed=13)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, device="cuda"))
    lat.step(3)
    g = lat.get_state(torch.float64).cpu().numpy()
    f, st = O.step(cfg, f0, 3, stats=True)
    assert rel(g, f) < 1e-12
    assert lat.stats()["limited_total"] == st["limited_sites"] > 50


MRT2_CASES = {k: v for k, v in CASES.items() if v["lattice"] == "D2Q9"}


@pytest.mark.parametrize("case", list(MRT2_CASES))
@pytest.mark.parametrize("collision", ["mrt2", "mrt_limiter"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_a2_collisions_match_oracle(case, collision, precision):
    """Section 5's aggressive MRT A_2 at every site, and the MRT limiter (A_2 at
    the Ehrenfest selection, LBGK elsewhere): 201 steps against the oracle;
    the limiter's count of corrected sites is exact in FP64."""
    cfg = dict(MRT2_CASES[case], collision=collision, precision=precision, beta=0.95, topk=3, delta=2e-4)
    f0 = state(cfg)
    if precision != "fp64":
        f0 = f0.astype(np.float32).astype(np.float64)
    n = 201
    lat = lbm.Lattice(cfg)
    dt = torch.float64 if precision == "fp64" else torch.float32
    lat.set_state(torch.tensor(f0, dtype=dt, device="cuda"))
    lat.step(n)
    g = lat.get_state(torch.float64).cpu().numpy()
    f, st = O.step(cfg, f0, n, stats=True)
    assert rel(g, f) < TOL[precision], rel(g, f)
    if collision == "mrt_limiter" and precision == "fp64":
        assert lat.stats()["limited_total"] == st["limited_sites"] > 0


@pytest.mark.parametrize("collision", ["mrt2", "mrt_limiter"])
def test_a2_collisions_16bit_pair_kernel(collision):
    """The 16-bit pair kernel runs the A_2 collisions too: one even and one
    odd step against the oracle step of the decoded state (FP16 deviations:
    half a spacing of the format plus FP32 arithmetic)."""
    cfg = dict(CASES["wide"], collision=collision, precision="fp16_dev", beta=0.95, topk=3, delta=2e-4)
    f0 = state(cfg)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, dtype=torch.float32, device="cuda"))
    _, _, w = O.lattice("D2Q9")
    for _ in range(2):
        pre = lat.get_state(torch.float64).cpu().numpy()
        lat.step(1)
        post = lat.get_state(torch.float64).cpu().numpy()
        want = O.step(cfg, pre, 1)
        dev = np.abs(want - np.asarray(w)[:, None, None])
        dev[:, -1, :] += cfg["lid_u"] / 6.0
        bound = 0.5 * np.spacing(dev.astype(np.float16)).astype(np.float64) * (1 + 1e-3) + 2e-6
        assert (np.abs(post - want) <= bound).all()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_enstrophy_matches_oracle(precision, tol):
    """lbm_enstrophy (Section 8) on a developing cavity and a periodic
    lattice against the oracle's enstrophy of the oracle's state."""
    for cfg in [dict(CASES["cavity"], collision="lbgk", beta=0.95),
                dict(CASES["periodic"], collision="mrt", beta=0.9)]:
        cfg = dict(cfg, precision=precision)
        f0 = state(cfg, seed=3)
        if precision != "fp64":
            f0 = f0.astype(np.float32).astype(np.float64)
        lat = lbm.Lattice(cfg)
        lat.set_state(torch.tensor(f0, dtype=torch.float64 if precision == "fp64" else torch.float32,
                                   device="cuda"))
        lat.step(37)  # an odd step count: the A-A layout of odd steps
        want = O.enstrophy(cfg, O.step(cfg, f0, 37))
        assert lat.enstrophy() == pytest.approx(want, rel=tol)


@pytest.mark.parametrize("collision", ["lbgk", "mrt2", "mrt"])
def test_shear_decay_lambda_matches_oracle(collision):
    """Section 7's shear decay (L = 50, L + 1 periodic points, u0 = 0.05,
    textbook polynomial equilibrium, L / u0 steps): the decay constant lambda
    measured on the GPU equals the oracle's (FP64), and the MRT forms decay
    like LBGK (the section's observation), within 5% of 4 pi^2 at Re 10 and
    1000."""
    import math
    L, u0 = 50, 0.05
    lam = {}
    for re in (10, 1000):
        cfg, init = WL.shear_decay(L, re, u0)
        beta = 1.0 / (6.0 * cfg["nu"] + 1.0)
        cfg.update(collision=collision, equilibrium="poly_std", beta=beta, precision="fp64")
        if collision == "mrt":
            cfg.update(lbm.mrt_rates("mrt_ll", beta))
        n = cfg["nx"]
        s = np.sin(2 * math.pi * np.arange(n) / L)
        amp = lambda uy: float((uy.mean(0) * s).sum() / (s * s).sum())
        T = int(round(L / u0))
        lat = lbm.Lattice(cfg)
        lat.init(init["rho"], init["ux"], init["uy"])
        a0 = amp(lat.macros(torch.float64)[1][1].cpu().numpy())
        lat.step(T)
        g = -(L * L) / (cfg["nu"] * T) * math.log(amp(lat.macros(torch.float64)[1][1].cpu().numpy()) / a0)
        f = O.step(cfg, O.init_equilibrium(cfg, init["rho"], init["ux"], init["uy"]), T)
        o = -(L * L) / (cfg["nu"] * T) * math.log(amp(O.macros(cfg, f)[2]) / a0)
        assert g == pytest.approx(o, rel=1e-9)
        assert g == pytest.approx(4 * math.pi ** 2, rel=0.05)
        lam[re] = g
    ref = {10: 37.884, 1000: 39.778}  # LBGK's values of this set-up (oracle)
    for re in lam:
        assert lam[re] == pytest.approx(ref[re], rel=0.01)


DIFF_CASES = {"box": dict(lattice="D2Q9", nx=37, ny=29, bc="diffusive", lid_u=0.1),
              "wide_box": dict(lattice="D2Q9", nx=200, ny=12, bc="diffusive", lid_u=0.1)}


@pytest.mark.parametrize("case", list(DIFF_CASES))
@pytest.mark.parametrize("collision", ["lbgk", "median", "ehrenfest", "mrt", "ensemble", "threshold"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diffusive_walls_match_oracle(case, collision, precision):
    """Section 8's diffusive Maxwell walls (entropic equilibria, moving top
    wall): wall sites not collided, the rule at the start of each step,
    limiters and median windows on the fluid sites; 101 steps against the
    oracle."""
    cfg = dict(DIFF_CASES[case], collision=collision, precision=precision, equilibrium="entropic",
               beta=0.93, topk=3, delta=2e-4, lim_alpha=1.0, lim_k=1.0, lim_delta0=0.05)
    f0 = state(cfg)
    if precision != "fp64":
        f0 = f0.astype(np.float32).astype(np.float64)
    n = 101
    lat = lbm.Lattice(cfg)
    dt = torch.float64 if precision == "fp64" else torch.float32
    lat.set_state(torch.tensor(f0, dtype=dt, device="cuda"))
    lat.step(n)
    g = lat.get_state(torch.float64).cpu().numpy()
    f, st = O.step(cfg, f0, n, stats=True)
    assert rel(g, f) < TOL[precision], rel(g, f)
    if collision in ("median", "ehrenfest", "threshold") and precision == "fp64":
        assert lat.stats()["limited_total"] == st["limited_sites"]


def test_control_point_probe_records_the_velocity_each_step():
    """lbm_probe_set: the velocity of the control site in the state each step
    produces, in order, through a ring buffer smaller than the run; equal to
    the oracle's velocity of each intermediate state."""
    cfg = dict(DIFF_CASES["box"], collision="median", precision="fp64", equilibrium="entropic", beta=0.93,
               delta=2e-4)
    f = state(cfg)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f, device="cuda"))
    xp, yp = 3, 22
    lat.probe(xp, yp, 16)
    want = []
    for _ in range(40):
        f = O.step(cfg, f, 1)
        _, ux, uy = O.macros(cfg, f)
        want.append((ux[yp, xp], uy[yp, xp]))
    lat.step(40)
    sig = lat.probe_signal()
    assert sig.shape == (16, 2)
    assert np.allclose(sig, np.array(want[-16:]), rtol=1e-12, atol=1e-15)
    lat.probe(None, None, 0)
    lat.step(2)
