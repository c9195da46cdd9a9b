"""Batched form (lbm_batch_*): every instance of a mixed batch must match
the FP64 oracle run of that instance alone, and the single-lattice path in
FP32; divergence is reported per instance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu


def instances(precision):
    base = dict(lattice="D2Q9", precision=precision, s_e=1.64, s_eps=1.54, s_q=1.2)
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
    ]


def state(cfg, seed):
    ny, nx = cfg["ny"], cfg["nx"]
    fields = WL.random_fields(ny, nx, seed, 0.05, 0.05)
    kind = "entropic" if cfg["collision"] == "elbm" else "poly"
    f = O.init_equilibrium(dict(cfg, collision="lbgk", equilibrium=kind), fields["rho"],
                           fields["ux"], fields["uy"])
    f = f * WL.lognormal_factors(f.shape, seed + 1, 0.01)
    return f * WL.lognormal_factors(f.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, 8, 0.4)[None])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nsteps", [11, 20])
def test_batch_fp64_matches_oracle_per_instance(nsteps):
    cfgs = instances("fp64")
    b = lbm.Batch(cfgs)
    b.init_uniform(1.0, 0.0, 0.0)
    f0 = [state(c, 40 + i) for i, c in enumerate(cfgs)]
    for i, f in enumerate(f0):
        b.set_state(i, torch.tensor(f, device="cuda"))
    status = b.step(nsteps, status=True)
    assert status == ["LBM_OK"] * len(cfgs)
    for i, c in enumerate(cfgs):
        g = b.get_state(i).cpu().numpy()
        f = O.step(c, f0[i], nsteps)
        assert rel(g, f) < 1e-12, (i, c["collision"], rel(g, f))


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


def test_batch_reports_divergence_per_instance():
    cfgs = instances("fp32")[:4]
    b = lbm.Batch(cfgs)
    b.init_uniform(1.0, 0.0, 0.0)
    bad = state(cfgs[2], 7).astype(np.float32)
    bad[:, 5, 5] = np.nan  # a poisoned site in instance 2 only (host-side fault)
    b.set_state(2, torch.tensor(bad, device="cuda"))
    status = b.step(2, status=True)
    assert status == ["LBM_OK", "LBM_OK", "LBM_ERR_DIVERGED", "LBM_OK"]
