"""Batched form (lbm_batch_*): persistent kernels over mixed batches of D2Q9
cavities, channels and periodic boxes and D1Q3 tubes.  Every instance must
match the FP64 oracle run of that instance alone, and the single-lattice
path in FP32; divergence is reported per instance; a bounded wait that runs
out returns LBM_ERR_TIMEOUT and leaves the batch usable after
re-initialisation; the per-group timing advances the instances exactly as
plain steps do; the autotuner returns valid options and caches them."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu


def instances(precision):
    base = dict(lattice="D2Q9", precision=precision, s_e=1.64, s_eps=1.54, s_q=1.2)
    tube = dict(lattice="D1Q3", ny=1, precision=precision)
    return [
        dict(base, nx=37, ny=29, bc="cavity", lid_u=0.1, collision="lbgk", beta=0.95),
        dict(base, nx=33, ny=17, bc="periodic", collision="mrt", beta=0.9),
        dict(base, nx=40, ny=30, bc="cavity", lid_u=0.1, collision="ehrenfest", beta=0.97,
             topk=3, delta=2e-4),
        dict(base, nx=31, ny=31, bc="cavity", lid_u=0.05, collision="median", beta=0.97,
             delta=2e-4),
        dict(base, nx=130, ny=5, bc="channel", lid_u=0.05, collision="positivity", beta=0.99),
        dict(base, nx=20, ny=20, bc="cavity", lid_u=0.1, collision="elbm", beta=0.9),
        dict(base, nx=129, ny=3, bc="periodic", collision="lbgk", beta=0.8),
        dict(tube, nx=301, bc="ends", collision="lbgk", beta=0.97),
        dict(tube, nx=600, bc="ends", collision="ehrenfest", beta=0.99, topk=4, delta=1e-4),
        dict(tube, nx=257, bc="periodic", collision="median", beta=0.97, delta=1e-4),
        dict(tube, nx=90, bc="ends", collision="elbm", beta=0.95),
    ]


def state(cfg, seed):
    ny, nx = cfg["ny"], cfg["nx"]
    fields = WL.random_fields(ny, nx, seed, 0.05, 0.05)
    kind = "entropic" if cfg["collision"] == "elbm" else "poly"
    uy = None if cfg["lattice"] == "D1Q3" else fields["uy"]
    f = O.init_equilibrium(dict(cfg, collision="lbgk", equilibrium=kind), fields["rho"], fields["ux"], uy)
    f = f * WL.lognormal_factors(f.shape, seed + 1, 0.01)
    return f * WL.lognormal_factors(f.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, 8, 0.4)[None])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


OPTS = {
    "default": None,
    # narrow tiles, one item per claim, tile j of every instance in turn,
    # four steps per graph launch
    "narrow_interleaved": dict(tile_x=32, chunk=1, order=1, graph_steps=4),
    "wide_chunked": dict(tile_x=256, chunk=16, ctas_per_sm=2, graph_steps=8),
}


@pytest.mark.parametrize("opts", list(OPTS))
@pytest.mark.parametrize("nsteps", [11, 20])
def test_batch_fp64_matches_oracle_per_instance(nsteps, opts):
    cfgs = instances("fp64")
    b = lbm.Batch(cfgs, opts=OPTS[opts])
    b.init_uniform(1.0, 0.0, 0.0)
    f0 = [state(c, 40 + i) for i, c in enumerate(cfgs)]
    for i, f in enumerate(f0):
        b.set_state(i, torch.tensor(f, device="cuda"))
    status = b.step(nsteps, status=True)
    assert status == ["LBM_OK"] * len(cfgs)
    for i, c in enumerate(cfgs):
        g = b.get_state(i).cpu().numpy()
        f, st = O.step(c, f0[i], nsteps, stats=True)
        assert rel(g, f) < 1e-12, (i, c["collision"], rel(g, f))
        if c["collision"] in ("ehrenfest", "median"):
            assert b.stats(i)["limited_total"] == st["limited_sites"] > 0, i


def test_batch_fp32_matches_single_lattice_path():
    cfgs = instances("fp32")
    b = lbm.Batch(cfgs)
    f0 = [state(c, 60 + i).astype(np.float32) for i, c in enumerate(cfgs)]
    for i, f in enumerate(f0):
        b.set_state(i, torch.tensor(f, device="cuda"))
    b.step(7)
    b.step(6)
    for i, c in enumerate(cfgs):
        lat = lbm.Lattice(c)
        lat.set_state(torch.tensor(f0[i], device="cuda"))
        lat.step(13)
        ref = lat.get_state(torch.float64).cpu().numpy()
        g = b.get_state(i).cpu().numpy()
        assert rel(g, ref) < 1e-6, (i, c["collision"], rel(g, ref))
        assert b.stats(i)["limited_total"] == lat.stats()["limited_total"]


@pytest.mark.parametrize("precision", ["fp16_dev", "bf16_dev"])
def test_batch_16bit_matches_single_lattice_path_bit_for_bit(precision):
    """16-bit storage: the batched kernels and the single-lattice kernels
    compute every site alike (the deviation form), so after 9 steps the
    decoded states are equal."""
    cfgs = [c for c in instances(precision) if c["collision"] != "median"]
    b = lbm.Batch(cfgs)
    f0 = [state(c, 80 + i).astype(np.float32) for i, c in enumerate(cfgs)]
    for i, f in enumerate(f0):
        b.set_state(i, torch.tensor(f, device="cuda"))
    b.step(9)
    for i, c in enumerate(cfgs):
        lat = lbm.Lattice(c)
        lat.set_state(torch.tensor(f0[i], device="cuda"))
        lat.step(9)
        assert torch.equal(b.get_state(i, torch.float32), lat.get_state(torch.float32)), (i, c["collision"])


@pytest.mark.parametrize("precision", ["fp16_dev", "bf16_dev"])
def test_batch_16bit_screened_pairs_match_bit_for_bit(precision):
    """Wide 16-bit lattices, where the single-lattice step runs two sites per
    thread and a pair with a screened site (Ehrenfest) or a negative
    population (positivity rule) is run again through the one-site form:
    the batched kernels, one site per thread throughout, give the same bits
    after 9 steps, and the same limiter counts."""
    base = dict(lattice="D2Q9", precision=precision, nx=200, ny=12)
    cfgs = [dict(base, bc="cavity", lid_u=0.1, collision="ehrenfest", beta=0.97, topk=3, delta=2e-4),
            dict(base, bc="channel", lid_u=0.05, collision="positivity", beta=0.99)]
    f0 = []
    for i, c in enumerate(cfgs):
        f = state(c, 120 + i)
        if c["collision"] == "positivity":
            f = f * WL.lognormal_factors(f.shape, 130, 0.6)
        f0.append(f.astype(np.float32))
    b = lbm.Batch(cfgs)
    for i, f in enumerate(f0):
        b.set_state(i, torch.tensor(f, device="cuda"))
    b.step(9)
    for i, c in enumerate(cfgs):
        lat = lbm.Lattice(c)
        lat.set_state(torch.tensor(f0[i], device="cuda"))
        lat.step(9)
        assert torch.equal(b.get_state(i, torch.float32), lat.get_state(torch.float32)), (i, c["collision"])
        assert b.stats(i)["limited_total"] == lat.stats()["limited_total"] > 0, (i, c["collision"])


def test_batch_reports_divergence_per_instance():
    cfgs = instances("fp32")[:4]
    b = lbm.Batch(cfgs)
    b.init_uniform(1.0, 0.0, 0.0)
    bad = state(cfgs[2], 7).astype(np.float32)
    bad[:, 5, 5] = np.nan  # a poisoned site in instance 2 only (host-side fault)
    b.set_state(2, torch.tensor(bad, device="cuda"))
    status = b.step(2, status=True)
    assert status == ["LBM_OK", "LBM_OK", "LBM_ERR_DIVERGED", "LBM_OK"]


def test_batch_bounded_wait_times_out_and_recovers():
    """An instance held one step behind (a step generation nothing will
    publish): its next step's wait runs into wait_ms, the launch stops and
    the status check returns LBM_ERR_TIMEOUT; re-initialised, the batch steps
    normally again."""
    cfgs = instances("fp32")[:3] + instances("fp32")[7:8]
    b = lbm.Batch(cfgs, opts=dict(wait_ms=20.0))
    b.init_uniform(1.0, 0.0, 0.0)
    assert b.step(2, status=True) == ["LBM_OK"] * 4
    b.debug_hold(1)
    assert b.step_status(2) == 5  # LBM_ERR_TIMEOUT
    b.init_uniform(1.0, 0.0, 0.0)
    assert b.step(3, status=True) == ["LBM_OK"] * 4
    ref = lbm.Batch(cfgs)
    ref.init_uniform(1.0, 0.0, 0.0)
    ref.step(3)
    for i in range(4):
        assert torch.equal(b.get_state(i), ref.get_state(i))


def test_batch_group_times_advance_like_steps():
    cfgs = instances("fp32")
    f0 = [state(c, 90 + i).astype(np.float32) for i, c in enumerate(cfgs)]
    a, b = lbm.Batch(cfgs), lbm.Batch(cfgs)
    for i, f in enumerate(f0):
        a.set_state(i, torch.tensor(f, device="cuda"))
        b.set_state(i, torch.tensor(f, device="cuda"))
    ms = a.group_times(6)
    assert set(ms) == {"lbgk", "mrt", "ehrenfest", "median", "positivity", "elbm"}
    assert all(v > 0 for v in ms.values())
    a.step(4)
    b.step(10)
    for i in range(len(cfgs)):
        assert torch.equal(a.get_state(i), b.get_state(i)), i
        assert a.stats(i)["limited_total"] == b.stats(i)["limited_total"]


def test_autotuner_returns_valid_options_and_caches(tmp_path):
    cfgs = [dict(lattice="D2Q9", nx=n, ny=n, bc="cavity", lid_u=0.1, collision=k, beta=0.9, precision="fp32",
                 topk=4, delta=1e-3) for n, k in [(200, "lbgk"), (150, "ehrenfest"), (90, "median")]]
    cfgs.append(dict(lattice="D1Q3", nx=800, ny=1, bc="ends", collision="lbgk", beta=0.9, precision="fp32"))
    cache = str(tmp_path / "tune.json")
    opts, sweep = lbm.tune_batch(cfgs, steps=2, cache=cache)
    assert opts["tile_x"] in (32, 64, 128, 256) and opts["chunk"] in (1, 4, 16)
    assert len(sweep) >= 8 and all(ms > 0 and obj > 0 for _, ms, obj in sweep)
    assert sweep[0][2] == 1.0  # the objective is relative to the starting options
    data = json.load(open(cache))
    assert len(data) == 1 and list(data.values())[0]["opts"] == opts
    again, _ = lbm.tune_batch(cfgs, steps=2, cache=cache)  # from the cache
    assert again == opts
    b = lbm.Batch(cfgs, opts=opts)
    b.init_uniform(1.0, 0.0, 0.0)
    assert b.step(4, status=True) == ["LBM_OK"] * 4
    assert os.path.getsize(cache) > 0
