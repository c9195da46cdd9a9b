"""GPU-vs-oracle parity through the C ABI (CUDA kernels on sm_103a).

Each test runs the same seeded input through ``paper_1110_0270_gb300.lbm``
(the CUDA path) and through the FP64 oracle, and compares element by
element: rel-L2 <= 1e-12 for FP64 storage and <= 1e-5 for FP32 storage over
the stated number of steps (the accuracy targets of the FP64 and FP32 paths),
bit-exact for the integer limiter-site selection.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def perturbed_state(cfg, seed, amp=0.02, hot=0, hot_amp=0.4, u_amp=0.05):
    """Equilibrium of random moments (oracle) times lognormal noise, with an
    optional few strongly non-equilibrium sites."""
    ny, nx = cfg["ny"], cfg["nx"]
    fields = WL.random_fields(ny, nx, seed, 0.05, u_amp)
    if cfg["lattice"] == "D1Q3":
        fields["uy"] = None
    f = O.init_equilibrium(dict(cfg, collision="lbgk"), fields["rho"], fields["ux"], fields["uy"])
    f = f * WL.lognormal_factors(f.shape, seed + 1, amp)
    if hot:
        f = f * WL.lognormal_factors(f.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, hot, hot_amp)[None])
    return f


def gpu_run(cfg, f0, n, store=None):
    lat = lbm.Lattice(cfg)
    dt = torch.float64 if cfg.get("precision", "fp32") == "fp64" else torch.float32
    lat.set_state(torch.tensor(f0, dtype=dt, device="cuda"))
    lat.step(n)
    return lat.get_state(torch.float64).cpu().numpy(), lat


def as_stored(cfg, f0):
    """The state both sides start from: rounded to the storage format."""
    return f0.astype(np.float32).astype(np.float64) if cfg["precision"] != "fp64" else f0


CASES = {
    "cavity": dict(lattice="D2Q9", nx=37, ny=29, bc="cavity", lid_u=0.1),
    "periodic": dict(lattice="D2Q9", nx=33, ny=17, bc="periodic"),
    "channel": dict(lattice="D2Q9", nx=130, ny=5, bc="channel", lid_u=0.05),
    "tube": dict(lattice="D1Q3", nx=301, ny=1, bc="ends"),
    "ring": dict(lattice="D1Q3", nx=64, ny=1, bc="periodic"),
    # wide enough for whole warps of two-site threads away from the walls,
    # with a ragged last block (200 = 128 + 72) and an exact one (256)
    "wide": dict(lattice="D2Q9", nx=200, ny=12, bc="cavity", lid_u=0.1),
    "wide_periodic": dict(lattice="D2Q9", nx=256, ny=6, bc="periodic"),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("collision", ["lbgk", "mrt", "positivity", "elbm"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_local_collisions_match_oracle(case, collision, precision):
    cfg = dict(CASES[case], collision=collision, precision=precision, beta=0.95,
               s_e=1.64, s_eps=1.54, s_q=1.2)
    amp = 0.6 if collision == "positivity" else 0.02
    f0 = as_stored(cfg, perturbed_state(cfg, 11, amp=amp))
    n = 301 if collision == "elbm" else 1001
    g, lat = gpu_run(cfg, f0, n)
    f = O.step(cfg, f0, n)
    assert rel(g, f) < TOL[precision], rel(g, f)
    assert lat.stats()["diverged"] == 0


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("collision", ["ehrenfest", "median"])
def test_limiters_fp64_match_oracle(case, collision):
    cfg = dict(CASES[case], collision=collision, precision="fp64", beta=0.97, topk=3, delta=2e-4)
    f0 = perturbed_state(cfg, 5, amp=0.01, hot=12)
    n = 201
    g, lat = gpu_run(cfg, f0, n)
    f, st = O.step(cfg, f0, n, stats=True)
    assert rel(g, f) < TOL["fp64"], rel(g, f)
    gs = lat.stats()
    assert gs["limited_total"] == st["limited_sites"]
    assert st["limited_sites"] > 0


@pytest.mark.parametrize("collision", ["ehrenfest", "median"])
@pytest.mark.parametrize("case", ["cavity", "tube", "wide"])
def test_limiters_fp32_one_step_and_selection_replay(case, collision):
    """FP32 storage: one step from a common state, and the integer selection
    replayed on the CPU from the GPU's own FP64 Delta S keys (bit-exact) and
    from the oracle's Delta S of the same state."""
    cfg = dict(CASES[case], collision=collision, precision="fp32", beta=0.97, topk=3, delta=2e-4)
    f0 = as_stored(cfg, perturbed_state(cfg, 7, amp=0.01, hot=12))
    g, lat = gpu_run(cfg, f0, 1)
    f = O.step(cfg, f0, 1)
    assert rel(g, f) < 1e-6, rel(g, f)
    ds, site, sel = lat.last_candidates()
    dS_or = O.delta_s_field(cfg, f0).ravel()
    cand_or = np.flatnonzero(dS_or > cfg["delta"])
    assert sorted(site.tolist()) == cand_or.tolist()
    assert np.allclose(ds, dS_or[site], rtol=1e-13, atol=0)
    if collision == "ehrenfest":
        order = sorted(range(len(ds)), key=lambda j: (-ds[j], site[j]))
        replay = set(site[order[: cfg["topk"]]].tolist())
        assert set(site[sel == 1].tolist()) == replay
        mask, _ = O.select_topk(dS_or, cfg["topk"], cfg["delta"])
        assert set(np.flatnonzero(mask).tolist()) == replay


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("collision,topk", [("median", 2), ("ehrenfest", 2), ("ehrenfest", 8),
                                            ("mrt_limiter", 2), ("mrt_limiter", 16)])
def test_few_candidates_match_oracle(collision, topk, precision):
    """A periodic fluid at rest with two hot sites: a handful of candidates
    per step (the one-CTA paths of the median and selection kernels; with
    k = 2 the selection ranks more candidates than it takes, with k >= the
    count it takes them all, in FP32 without an FP64 evaluation when FP32
    settles every site's side of delta), then none.  The candidates the
    ABI reports after one step carry FP64 values either way."""
    cfg = dict(CASES["periodic"], collision=collision, precision=precision, beta=0.97, delta=2e-4, topk=topk)
    ny, nx = cfg["ny"], cfg["nx"]
    f0 = O.init_equilibrium(dict(cfg, collision="lbgk"), np.ones((ny, nx)), np.zeros((ny, nx)),
                            np.zeros((ny, nx)))
    f0 = f0 * WL.lognormal_factors(f0.shape, 4, 0.002)
    rng = np.random.default_rng(1)
    for y, x in [(5, 7), (11, 20)]:
        f0[:, y, x] *= np.exp(0.3 * rng.standard_normal(9))
    f0 = as_stored(cfg, f0)
    g, lat = gpu_run(cfg, f0, 30)
    f, st = O.step(cfg, f0, 30, stats=True)
    assert rel(g, f) < TOL[precision], rel(g, f)
    assert st["limited_sites"] > 0
    assert lat.stats()["limited_total"] == st["limited_sites"]
    f1 = O.step(cfg, f0, 1)
    g1, lat1 = gpu_run(cfg, f0, 1)
    assert rel(g1, f1) < TOL[precision]
    ds, site, sel = lat1.last_candidates()
    dS_or = O.delta_s_field(cfg, f0).ravel()
    assert sorted(site.tolist()) == np.flatnonzero(dS_or > cfg["delta"]).tolist()
    assert np.allclose(ds, dS_or[site], rtol=1e-13, atol=0)
    assert lat1.stats()["candidates_last"] == len(site)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("collision,topk", [("ehrenfest", 4), ("ehrenfest", 600), ("mrt_limiter", 4)])
def test_tens_to_hundreds_of_candidates_match_oracle(collision, topk, precision):
    """A periodic fluid at rest with 40 hot sites: 36 candidates in the first
    step, then hundreds (for up to 512 screened sites every CTA of the
    selection kernel settles the sides of delta in FP32, and the first takes
    all candidates without FP64 when at most k are above; else, and beyond
    512, the grid-wide FP64 pass), 12 steps; k = 4 ranks many candidates,
    k = 600 takes them all."""
    cfg = dict(CASES["periodic"], collision=collision, precision=precision, beta=0.97, delta=2e-4, topk=topk)
    ny, nx = cfg["ny"], cfg["nx"]
    f0 = O.init_equilibrium(dict(cfg, collision="lbgk"), np.ones((ny, nx)), np.zeros((ny, nx)),
                            np.zeros((ny, nx)))
    f0 = f0 * WL.lognormal_factors(f0.shape, 4, 0.002)
    rng = np.random.default_rng(2)
    for y, x in zip(rng.integers(0, ny, 40), rng.integers(0, nx, 40)):
        f0[:, y, x] *= np.exp(0.3 * rng.standard_normal(9))
    f0 = as_stored(cfg, f0)
    g, lat = gpu_run(cfg, f0, 12)
    f, st = O.step(cfg, f0, 12, stats=True)
    assert rel(g, f) < TOL[precision], rel(g, f)
    assert lat.stats()["limited_total"] == st["limited_sites"] > 0
    # the second step's candidates against the oracle's Delta S of the GPU's
    # own state after one step (the step's input)
    g1, lat1 = gpu_run(cfg, f0, 1)
    lat1.step(1)
    ds, site, sel = lat1.last_candidates()
    dS_or = O.delta_s_field(cfg, g1).ravel()
    assert sorted(site.tolist()) == np.flatnonzero(dS_or > cfg["delta"]).tolist()
    assert np.allclose(ds, dS_or[site], rtol=1e-12, atol=0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("beta", [0.52, 0.7])
def test_median_window_sources_match_oracle(precision, beta):
    """The median window's Delta S from the step's field (beta = 0.52, where
    1 - 2 beta is too small to recover the pre-collision state) and from the
    post-collision state (beta = 0.7), cavity with hot sites, 60 steps."""
    cfg = dict(CASES["cavity"], collision="median", precision=precision, beta=beta, delta=2e-4)
    f0 = as_stored(cfg, perturbed_state(cfg, 9, amp=0.01, hot=12))
    g, lat = gpu_run(cfg, f0, 60)
    f, st = O.step(cfg, f0, 60, stats=True)
    assert rel(g, f) < TOL[precision], rel(g, f)
    assert st["limited_sites"] > 0
    if precision == "fp64":
        assert lat.stats()["limited_total"] == st["limited_sites"]


@pytest.mark.parametrize("precision", ["fp32", "fp16_dev"])
def test_fp32_init_and_macros(precision):
    """lbm_init evaluates f* in the storage's arithmetic type and lbm_macros
    forms FP32 outputs in FP32 (opposite populations subtracted first): from
    random rho and u the initial state is the oracle's f*(rho, u) to a few
    FP32 units (plus the 16-bit rounding of f - W), and after 300 steps of a
    65^2 cavity from rest (speeds from ~1e-9 near the bottom to 0.1 at the
    lid) the FP32 rho and u of the GPU's own state equal the oracle's
    moments of that state to 1e-6 of their largest magnitude."""
    cfg, init = WL.cavity(65, 400.0, 0.1)
    cfg.update(collision="lbgk", precision=precision)
    lat = lbm.Lattice(cfg)
    fields = WL.random_fields(65, 65, 41, 0.05, 0.05)
    lat.init(fields["rho"], fields["ux"], fields["uy"])
    g = lat.get_state(torch.float64).cpu().numpy()
    f = O.init_equilibrium(cfg, fields["rho"], fields["ux"], fields["uy"])
    _, _, w = O.lattice("D2Q9")
    slack = 1e-6 * np.abs(f) if precision == "fp32" else np.spacing(
        np.abs(f - np.asarray(w)[:, None, None]).astype(np.float16)).astype(np.float64) + 1e-7
    assert (np.abs(g - f) <= slack).all(), float((np.abs(g - f) / slack).max())
    lat.init(init["rho"], init["ux"], init["uy"])
    lat.step(300)
    g = lat.get_state(torch.float64).cpu().numpy()
    rho, u = lat.macros(torch.float32)
    r0, ux0, uy0 = O.macros(cfg, g)
    assert np.abs(rho.double().cpu().numpy() - r0).max() < 1e-6 * np.abs(r0).max()
    umax = max(np.abs(ux0).max(), np.abs(uy0).max())
    assert np.abs(u[0].double().cpu().numpy() - ux0).max() < 1e-6 * umax
    assert np.abs(u[1].double().cpu().numpy() - uy0).max() < 1e-6 * umax


def test_cavity_from_rest_fp64_1000_steps_and_macros():
    cfg, init = WL.cavity(41, 400.0, 0.1)
    cfg.update(collision="lbgk", precision="fp64")
    lat = lbm.Lattice(cfg)
    lat.init(init["rho"], init["ux"], init["uy"])
    f = O.init_equilibrium(cfg, init["rho"], init["ux"], init["uy"])
    for n in (999, 1):  # odd then even parity
        lat.step(n)
        f = O.step(cfg, f, n)
        g = lat.get_state(torch.float64).cpu().numpy()
        assert rel(g, f) < 1e-12
        rho, u = lat.macros(torch.float64)
        r0, ux0, uy0 = O.macros(cfg, f)
        assert rel(rho.cpu().numpy(), r0) < 1e-12
        assert rel(u[0].cpu().numpy(), ux0) < 1e-12
        assert rel(u[1].cpu().numpy(), uy0) < 1e-12
        H, dS = lat.entropy(field=True)
        # H = sum f ln(f/W) is a sum of cancelling terms and moves by ~1 per
        # unit of mass, so its tolerance is relative to sum |terms| and to the
        # (rounding-level) mass difference of the two runs
        _, _, W = O.lattice("D2Q9")
        terms = np.abs(g * np.log(g / W[:, None, None])).sum()
        Hg = float((g * np.log(g / W[:, None, None])).sum())
        assert abs(H - Hg) < 1e-13 * terms
        assert abs(H - O.total_h(cfg, f)) < 1e-13 * terms + 2 * abs(g.sum() - f.sum())
        # Delta S near equilibrium amplifies differences by ~1/|x|: it is
        # checked on the GPU's own state, with an absolute slack of a few ulp
        # of the equilibrium per unit of sum |f - f*| (the two sides round f*
        # differently)
        dS_or = O.delta_s_field(cfg, g)
        neq = np.zeros_like(dS_or)
        for y in range(cfg["ny"]):
            for x in range(cfg["nx"]):
                r_, a_, b_ = O.moments("D2Q9", g[:, y, x])
                neq[y, x] = np.abs(g[:, y, x] - O.equilibrium("D2Q9", "poly", r_, a_, b_)).sum()
        assert np.all(np.abs(dS.cpu().numpy() - dS_or) <= 1e-12 * dS_or + 1e-15 * neq + 1e-30)


def test_shock_tube_all_collisions_400_steps():
    cfg, init = WL.shock_tube(800, 1e-9)
    for collision in ["lbgk", "elbm", "ehrenfest", "median", "mrt"]:
        c = dict(cfg, collision=collision, precision="fp64", topk=4, delta=1e-3)
        lat = lbm.Lattice(c)
        lat.init(init["rho"], init["ux"])
        lat.step(400)
        g = lat.get_state(torch.float64).cpu().numpy()
        f = O.step(c, O.init_equilibrium(c, init["rho"], init["ux"]), 400)
        assert rel(g, f) < 1e-12, (collision, rel(g, f))


def _spacing16(dev, precision):
    """Spacing of the 16-bit deviation format at dev (bf16: 8 significant
    bits, fp16: 11, with fp16's subnormal floor)."""
    a = np.abs(dev)
    if precision == "fp16_dev":
        return np.spacing(a.astype(np.float16)).astype(np.float64)
    e = np.floor(np.log2(np.maximum(a, 1e-38)))
    return 2.0 ** (e - 7)


def _median_window_recovery_bound(cfg, lat, pre, precision):
    """Extra error allowed at the populations a median-limited site streams
    out, when the filter's window Delta S comes from the stored 16-bit LBGK
    post-collision state (f = f* + (F - f*) / c, c = 1 - 2 beta): a stored
    F_i off by at most h_i (half a spacing at F_i - W_i) moves a window
    site's Delta S by at most B = sum |x_i| h_i / |c| + 1/2 sum h_i^2 / (c^2 f*_i)
    (x = (f - f*) / f*), the lower median by at most the window's largest B,
    phi = sqrt(M / C) by at most sqrt(B / C) and the limited populations by
    |c| sqrt(B / C) |f_i - f*_i|.  Added to the 3 x 3 block around the site
    (its populations land there, bounced back at walls)."""
    ny, nx = cfg["ny"], cfg["nx"]
    _, _, w = O.lattice("D2Q9")
    beta = cfg["beta"]
    c = 1.0 - 2.0 * beta
    lb = dict(cfg, collision="lbgk", nx=1, ny=1)
    extra = np.zeros_like(pre)
    _, site, sel = lat.last_candidates()
    for s_ in site[sel == 1]:
        y, x = divmod(int(s_), nx)
        B = 0.0
        for yy in range(max(0, y - 1), min(ny, y + 2)):
            for xx in range(max(0, x - 1), min(nx, x + 2)):
                f = pre[:, yy, xx]
                fe = O.equilibrium("D2Q9", "poly", *O.moments("D2Q9", f))
                F = O.collide_site(lb, f)
                h = 0.5 * _spacing16(np.abs(F - np.asarray(w)), precision) * (1 + 1e-3) + 2e-6
                xr = (f - fe) / fe
                B = max(B, float((np.abs(xr) * h).sum() / abs(c) + 0.5 * (h * h / (c * c * fe)).sum()))
        f = pre[:, y, x]
        fe = O.equilibrium("D2Q9", "poly", *O.moments("D2Q9", f))
        C = O.delta_s(f, fe)
        e = abs(c) * np.sqrt(B / C) * np.abs(f - fe).max()
        extra[:, max(0, y - 1):y + 2, max(0, x - 1):x + 2] += e
    return extra


@pytest.mark.parametrize("precision", ["fp16_dev", "bf16_dev"])
@pytest.mark.parametrize("collision", ["lbgk", "mrt", "positivity", "ehrenfest", "median"])
def test_reduced_precision_one_step_rounding(precision, collision):
    """16-bit deviation storage, one even and one odd step from a common
    state: each stored population is the oracle's post-step value of the
    decoded pre-step state, rounded once to the format (half a spacing of
    the deviation f_i - W_i, plus FP32 arithmetic).  In the layout after an
    even step the top row's wall links hold the bounced value before the
    moving-lid term 6 W_i |v_ix| U (at most U / 6) is added, so there the
    stored deviation may be larger by that much."""
    cfg = dict(CASES["wide"], collision=collision, precision=precision, beta=0.97, topk=3,
               delta=2e-4, s_e=1.64, s_eps=1.54, s_q=1.2)
    amp = 0.6 if collision == "positivity" else 0.01
    f0 = perturbed_state(cfg, 17, amp=amp, hot=12 if collision in ("ehrenfest", "median") else 0)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, dtype=torch.float32, device="cuda"))
    _, _, w = O.lattice("D2Q9")
    for parity in (0, 1):
        pre = lat.get_state(torch.float64).cpu().numpy()
        lat.step(1)
        post = lat.get_state(torch.float64).cpu().numpy()
        want = O.step(cfg, pre, 1)
        dev = np.abs(want - np.asarray(w)[:, None, None])
        dev[:, -1, :] += cfg["lid_u"] / 6.0
        bound = 0.5 * _spacing16(dev, precision) * (1 + 1e-3) + 2e-6
        if collision == "median":
            bound = bound + _median_window_recovery_bound(cfg, lat, pre, precision)
        err = np.abs(post - want)
        worst = np.unravel_index(int(np.argmax(err / bound)), err.shape)
        assert (err <= bound).all(), (parity, float((err / bound).max()), worst, post[worst], want[worst])


@pytest.mark.parametrize("precision,tol", [("fp16_dev", 3e-3), ("bf16_dev", 3e-2)])
def test_reduced_precision_storage_tracks_fp64(precision, tol):
    """16-bit deviation storage with FP32 math: error against the FP64 oracle
    after 200 steps of a 65^2 cavity stays within the stated bound."""
    cfg, init = WL.cavity(65, 1000.0, 0.1)
    cfg.update(collision="lbgk", precision=precision)
    lat = lbm.Lattice(cfg)
    lat.init(init["rho"], init["ux"], init["uy"])
    lat.step(200)
    f = O.step(cfg, O.init_equilibrium(cfg, init["rho"], init["ux"], init["uy"]), 200)
    g = lat.get_state(torch.float64).cpu().numpy()
    assert rel(g, f) < tol, rel(g, f)
    rho, u = lat.macros(torch.float64)
    r0, ux0, uy0 = O.macros(cfg, f)
    uerr = np.linalg.norm(u[0].cpu().numpy() - ux0) / np.linalg.norm(ux0)
    assert uerr < 20 * tol, uerr


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (33, 3), (129, 3), (513, 4),
                                   (514, 5), (1025, 3)])
def test_tiny_and_ragged_lattices(shape):
    """Degenerate and ragged shapes in FP64 and FP32 storage, including
    widths just past whole 128-site blocks (129, 513, 1025: the last column
    alone in the last block; 514: two columns)."""
    nx, ny = shape
    for bc in ["cavity", "periodic", "channel"]:
        for precision, tol in [("fp64", 1e-12), ("fp32", 1e-5)]:
            cfg = dict(lattice="D2Q9", nx=nx, ny=ny, bc=bc, lid_u=0.1, collision="lbgk",
                       precision=precision, beta=0.9)
            f0 = as_stored(cfg, perturbed_state(cfg, 3))
            g, _ = gpu_run(cfg, f0, 17)
            assert rel(g, O.step(cfg, f0, 17)) < tol, (shape, bc, precision)
    for nx1 in (1, 2, 3, 257):
        cfg = dict(lattice="D1Q3", nx=nx1, ny=1, bc="ends", collision="lbgk", precision="fp64", beta=0.9)
        f0 = perturbed_state(cfg, 4)
        g, _ = gpu_run(cfg, f0, 9)
        assert rel(g, O.step(cfg, f0, 9)) < 1e-12


def test_ehrenfest_selection_edge_cases():
    base = dict(lattice="D2Q9", nx=40, ny=30, bc="periodic", collision="ehrenfest",
                precision="fp64", beta=0.9)
    f0 = perturbed_state(base, 21, amp=0.03, hot=25)
    # delta = 0: every site is a candidate (large list, radix select path)
    for topk, delta in [(0, 1e-4), (5, 0.0), (10**6, 1e-4), (1, 1e-4), (37, 1e-9)]:
        cfg = dict(base, topk=topk, delta=delta)
        g, lat = gpu_run(cfg, f0, 3)
        f = O.step(cfg, f0, 3)
        assert rel(g, f) < 1e-12, (topk, delta, rel(g, f))
    # exact ties: identical hot spots in a uniform field; lower index wins
    cfg = dict(base, nx=16, ny=16, topk=3, delta=1e-5)
    f0 = O.init_equilibrium(cfg, np.ones((16, 16)), np.zeros((16, 16)), np.zeros((16, 16)))
    bump = np.array([1.3, 0.8, 1.1, 0.9, 1.2, 0.7, 1.05, 0.95, 1.0])
    for s in [(3, 3), (3, 9), (10, 4), (12, 12), (7, 7)]:
        f0[:, s[0], s[1]] *= bump
    g, lat = gpu_run(cfg, f0, 1)
    ds, site, sel = lat.last_candidates()
    assert len(site) == 5 and len(set(ds.tolist())) == 1
    assert sorted(site[sel == 1].tolist()) == sorted([3 * 16 + 3, 3 * 16 + 9, 7 * 16 + 7])
    assert rel(g, O.step(cfg, f0, 1)) < 1e-12


def test_full_size_4097_sampled_sites_and_mass():
    """The benchmark's lattice (4097^2, FP32, the same lbm_step launch):
    sampled interior sites after one step equal the oracle's collision of
    the source sites, f_i(x, t+1) = F_i(x - v_i, t); total mass is kept."""
    n = 4097
    for collision in ["lbgk", "mrt", "positivity"]:
        cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="cavity", lid_u=0.05, collision=collision,
                   precision="fp32", nu=0.05 * (n - 1) / 10000.0, s_e=1.64, s_eps=1.54, s_q=1.2)
        lat = lbm.Lattice(cfg)
        fields = WL.random_fields(n, n, 99, 0.05, 0.05)
        lat.init(fields["rho"], fields["ux"], fields["uy"])
        lat.step(1)  # a non-equilibrium state with the A-A layout of odd steps
        pre = lat.get_state(torch.float32)
        m0 = float(pre.double().sum())
        lat.step(1)
        post = lat.get_state(torch.float32)
        assert abs(float(post.double().sum()) - m0) < 1e-6 * m0
        rng = np.random.default_rng(5)
        xs, ys = rng.integers(1, n - 1, 400), rng.integers(1, n - 1, 400)
        cx, cy, _ = O.lattice("D2Q9")
        beta = 1.0 / (6 * cfg["nu"] + 1)
        ocfg = dict(cfg, nx=1, ny=1, beta=beta)
        for x, y in zip(xs, ys):
            for i in range(9):
                src = pre[:, y - cy[i], x - cx[i]].double().cpu().numpy()
                F = O.collide_site(ocfg, src)
                got = float(post[i, y, x])
                assert abs(got - F[i]) < 2e-6 * abs(F[i]) + 1e-7, (collision, x, y, i, got, F[i])
        del lat, pre, post
        torch.cuda.empty_cache()


@pytest.mark.parametrize("collision", ["ehrenfest", "median"])
def test_full_size_4097_limiters(collision):
    """The benchmark's lattice (4097^2, FP32, lbm_step's launch) with 300
    strongly perturbed sites, one step: the candidate set equals the
    oracle's (FP64 Delta S of the whole field), the selection is the
    oracle's (the k = 64 largest; the median rule), the populations that
    selected sites stream out equal the oracle's limited collision, sampled
    other sites equal its LBGK collision, and the mass is kept."""
    n, k, delta = 4097, 64, 1e-3
    cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="cavity", lid_u=0.05, collision=collision, precision="fp32",
               nu=0.05 * (n - 1) / 10000.0, topk=k, delta=delta)
    beta = 1.0 / (6 * cfg["nu"] + 1)
    fields = WL.random_fields(n, n, 7, 0.05, 0.05)
    f0 = O.init_equilibrium(dict(cfg, collision="lbgk"), fields["rho"], fields["ux"], fields["uy"])
    rng = np.random.default_rng(11)
    hx, hy = rng.integers(2, n - 2, 300), rng.integers(2, n - 2, 300)
    f0[:, hy, hx] *= np.exp(0.3 * rng.standard_normal((9, 300)))
    pre = f0.astype(np.float32)
    del f0
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.from_numpy(pre).cuda())
    lat.step(1)
    post = lat.get_state(torch.float32).cpu().numpy()
    pre64 = pre.astype(np.float64)
    assert abs(float(post.astype(np.float64).sum()) - float(pre64.sum())) < 1e-6 * float(pre64.sum())
    dS = O.delta_s_field(cfg, pre64)
    cand = np.flatnonzero(dS.ravel() > delta)
    ds, site, sel = lat.last_candidates()
    assert sorted(site.tolist()) == cand.tolist()
    assert np.allclose(ds, dS.ravel()[site], rtol=1e-12, atol=0)
    if collision == "ehrenfest":
        mask, _ = O.select_topk(dS, k, delta)
        want = np.flatnonzero(mask)
    else:
        med = O.median_field("D2Q9", dS).ravel()
        want = cand[med[cand] < dS.ravel()[cand]]
    got = np.sort(site[sel == 1])
    assert got.tolist() == want.tolist()
    assert 0 < len(want) and (collision == "median" or len(want) == k)
    cx, cy, _ = O.lattice("D2Q9")
    lb = dict(cfg, collision="lbgk", nx=1, ny=1, beta=beta)
    med_all = None if collision == "ehrenfest" else O.median_field("D2Q9", dS)

    def expected(y, x):
        f = pre64[:, y, x]
        if y * n + x not in chosen:
            return O.collide_site(lb, f)
        r, ux, uy = O.moments("D2Q9", f)
        fe = O.equilibrium("D2Q9", "poly", r, ux, uy)
        if collision == "ehrenfest":
            return fe
        phi = np.sqrt(med_all[y, x] / dS[y, x])
        return fe + (1 - 2 * beta) * phi * (f - fe)

    chosen = set(want.tolist())
    checks = [(s // n, s % n) for s in want if 1 <= s // n < n - 1 and 1 <= s % n < n - 1]
    checks += list(zip(rng.integers(1, n - 1, 300), rng.integers(1, n - 1, 300)))
    for y, x in checks:
        F = expected(y, x)
        for i in range(9):  # F_i(x) streams to x + v_i
            got_i = float(post[i, y + cy[i], x + cx[i]])
            assert abs(got_i - F[i]) < 2e-6 * abs(F[i]) + 1e-7, (collision, x, y, i, got_i, F[i])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_init_from_device_arrays_equals_host_init(precision):
    """lbm_init_device (device rho, u) produces the same state as lbm_init
    from host arrays, which is the oracle's equilibrium; D1Q3 takes no u_y."""
    for cfg in [dict(CASES["cavity"], collision="lbgk", precision=precision, beta=0.9),
                dict(CASES["tube"], collision="lbgk", precision=precision, beta=0.9)]:
        ny, nx = cfg["ny"], cfg["nx"]
        fl = WL.random_fields(ny, nx, 21, 0.05, 0.05)
        uy = None if cfg["lattice"] == "D1Q3" else fl["uy"]
        a = lbm.Lattice(cfg)
        a.init(fl["rho"], fl["ux"], uy)
        b = lbm.Lattice(cfg)
        dev = [torch.tensor(v, dtype=torch.float64, device="cuda") if v is not None else None
               for v in (fl["rho"], fl["ux"], uy)]
        b.init_device(*dev)
        ga, gb = a.get_state(torch.float64), b.get_state(torch.float64)
        assert torch.equal(ga, gb)
        want = as_stored(cfg, O.init_equilibrium(cfg, fl["rho"], fl["ux"], uy))
        assert rel(ga.cpu().numpy(), want) < TOL[precision]


def test_profile_counts_every_kernel_launch():
    """lbm_profile_enable: each step is timed kernel by kernel (one step and
    one selection launch per Ehrenfest step, positive times); with the
    profile off again lbm_step replays its graphs and the state continues
    identically to an unprofiled run."""
    cfg = dict(CASES["cavity"], collision="ehrenfest", precision="fp64", beta=0.97, topk=3, delta=2e-4)
    f0 = perturbed_state(cfg, 5, amp=0.01, hot=12)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, device="cuda"))
    lat.profile(True)
    lat.step(7)
    prof = lat.profile_read()
    lat.profile(False)
    lat.step(6)
    assert prof["step"][0] == 7 and prof["fixup"][0] == 7
    assert prof["step"][1] > 0 and prof["fixup"][1] > 0
    g, _ = gpu_run(cfg, f0, 13)
    assert np.array_equal(lat.get_state(torch.float64).cpu().numpy(), g)
    assert rel(g, O.step(cfg, f0, 13)) < TOL["fp64"]
