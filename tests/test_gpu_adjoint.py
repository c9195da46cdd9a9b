"""Hand-written adjoint (lbm_adjoint_*): FP64 against the oracle's FP64 tape
adjoint, FP32 against central differences of FP64 forward runs, and the
torch.autograd.Function built on it.  Collisions: LBGK, the Ehrenfest step
(Section 4), the median filter (Section 4.4, Eq. entrHom) and the positivity
rule (Section 4, Eq. StrLine); through the limiters the selected branch is
differentiated with the selection of each step held fixed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu


def start_state(cfg, seed, amp=0.02, hot=4, hot_amp=None):
    ny, nx = cfg["ny"], cfg["nx"]
    fl = WL.random_fields(ny, nx, seed, 0.05, 0.05)
    f0 = O.init_equilibrium(dict(cfg, collision="lbgk"), fl["rho"], fl["ux"],
                            None if cfg["lattice"] == "D1Q3" else fl["uy"])
    f0 = f0 * WL.lognormal_factors(f0.shape, seed + 1, amp)
    # hot sites strong enough that the positivity rule fires
    if hot_amp is None:
        hot_amp = 1.2 if cfg.get("collision") == "positivity" else 0.4
    return f0 * WL.lognormal_factors(f0.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, hot, hot_amp)[None])


def gpu_adjoint(cfg, f0, T, K):
    lat = lbm.Lattice(cfg)
    dt = torch.float64 if cfg["precision"] == "fp64" else torch.float32
    lat.set_state(torch.tensor(f0, dtype=dt, device="cuda"))
    J, work = lat.adjoint_forward(T, K)
    g, gU, gB = lat.adjoint_backward(T, K, work)
    return J, g.cpu().numpy(), gU, gB, lat


CASES = {
    "cavity_lbgk": dict(lattice="D2Q9", nx=33, ny=29, bc="cavity", lid_u=0.1, collision="lbgk", beta=0.9),
    "cavity_ehrenfest": dict(lattice="D2Q9", nx=33, ny=29, bc="cavity", lid_u=0.1,
                             collision="ehrenfest", beta=0.95, topk=3, delta=1e-4),
    "tube": dict(lattice="D1Q3", nx=64, ny=1, bc="ends", collision="lbgk", beta=0.97),
    "periodic_entropic": dict(lattice="D2Q9", nx=24, ny=20, bc="periodic", collision="ehrenfest",
                              beta=0.92, topk=2, delta=1e-4, equilibrium="entropic"),
    "cavity_median": dict(lattice="D2Q9", nx=33, ny=29, bc="cavity", lid_u=0.1, collision="median",
                          beta=0.9, delta=1e-4),
    "periodic_median": dict(lattice="D2Q9", nx=24, ny=20, bc="periodic", collision="median", beta=0.95,
                            delta=5e-5, equilibrium="entropic"),
    "tube_median": dict(lattice="D1Q3", nx=64, ny=1, bc="ends", collision="median", beta=0.97, delta=1e-4),
    "cavity_positivity": dict(lattice="D2Q9", nx=33, ny=29, bc="cavity", lid_u=0.1, collision="positivity",
                              beta=0.99),
    "tube_positivity": dict(lattice="D1Q3", nx=64, ny=1, bc="ends", collision="positivity", beta=0.99),
}


@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_fp64_matches_oracle_tape(case):
    cfg = dict(CASES[case], precision="fp64")
    f0 = start_state(cfg, 12)
    T, K = 60, 16  # four segments, the last one partial
    if cfg["collision"] in ("median", "positivity"):
        _, st = O.step(cfg, f0, T, stats=True)
        assert st["limited_sites"] > 0  # the limiter branch is exercised
    J, g, gU, gB, lat = gpu_adjoint(cfg, f0, T, K)
    Jo, go, gUo, gBo = O.adjoint_ke(cfg, f0, T)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert np.linalg.norm(g - go) <= 1e-10 * np.linalg.norm(go)
    assert abs(gB - gBo) <= 1e-10 * abs(gBo) + 1e-14
    if cfg["bc"] == "cavity":
        assert abs(gU - gUo) <= 1e-10 * abs(gUo)
    # the context holds f_T afterwards
    fT = lat.get_state(torch.float64).cpu().numpy()
    assert np.linalg.norm(fT - O.step(cfg, f0, T)) <= 1e-12 * np.linalg.norm(fT)


@pytest.mark.parametrize("case", ["cavity_ehrenfest", "cavity_median", "cavity_positivity"])
def test_adjoint_gradient_does_not_depend_on_the_segment_length(case):
    """Full segments replay a captured graph (one per starting lambda
    buffer: with an odd K two of them alternate) and a partial segment, or
    K = 1, launches its kernels one by one; a segment that starts at an odd
    step is recomputed with the even-step kernels.  The gradient is the same
    for every K (to the order of the FP64 atomic sums)."""
    cfg = dict(CASES[case], precision="fp64")
    f0 = start_state(cfg, 13)
    T = 45
    J1, g1, gU1, gB1, _ = gpu_adjoint(cfg, f0, T, 1)
    for K in (7, 10, 45):
        J, g, gU, gB, _ = gpu_adjoint(cfg, f0, T, K)
        assert abs(J - J1) <= 1e-14 * abs(J1), K
        assert np.linalg.norm(g - g1) <= 1e-13 * np.linalg.norm(g1), K
        assert abs(gU - gU1) <= 1e-13 * abs(gU1) and abs(gB - gB1) <= 1e-13 * abs(gB1) + 1e-16, K


def _ke_fp64(cfg, f0, T):
    lat = lbm.Lattice(dict(cfg, precision="fp64"))
    lat.set_state(torch.tensor(f0, dtype=torch.float64, device="cuda"))
    J, _ = lat.adjoint_forward(T, T)
    return J


def _fp32_copy(collision):
    """A 65^2 copy of the adjoint configuration (Re 1000, U 0.1) with the
    given limiter: Ehrenfest k = 32 or the median filter at delta = 1e-3 from
    the resting state with N(0, 1e-4) noise; the positivity rule from a
    random state with strong hot sites (beta 0.99)."""
    n = 65
    cfg, init = WL.cavity(n, 1000.0, 0.1)
    cfg.update(collision=collision, topk=32, delta=1e-3, precision="fp32")
    beta = 1.0 / (6.0 * cfg["nu"] + 1.0)
    if collision == "positivity":
        beta = 0.99
        cfg["beta"] = beta
        f0 = start_state(cfg, 31, hot=40)
    else:
        cfg["beta"] = beta
        f0 = O.init_equilibrium(cfg, init["rho"], init["ux"], init["uy"])
        f0 = f0 + WL.normal_noise(f0.shape, 4, 1e-4)
    return cfg, beta, f0.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("collision", ["ehrenfest", "median", "positivity"])
def test_adjoint_fp32_against_central_differences_and_oracle(collision):
    """FP32 adjoint on a 65^2 cavity against central differences of FP64
    forward runs (U, beta, a random direction in f0) and against the oracle's
    FP64 tape adjoint, within 1e-4 relative.  In the first steps the
    Ehrenfest copy has up to 118 candidates for 32 slots, so a step of 1e-3
    moves sites across the selection boundary (the finite difference then
    measures a jump, not the derivative of either branch); h = 1e-6 stays on
    the branch, as it does for the median's window sites and the positivity
    rule's binding populations."""
    cfg, beta, f0 = _fp32_copy(collision)
    # the positivity rule fires at a few sites in every step; where it binds
    # near its boundary the FP32 and FP64 trajectories separate after 100 to
    # 300 steps (GPU FP32 against the oracle: 4e-7 at T = 100, 5e-4 at
    # T = 300; GPU FP64 1e-12 at both), so its FP32 check runs 100 steps
    T, K = (100, 25) if collision == "positivity" else (300, 50)
    _, st = O.step(cfg, f0, T, stats=True)
    assert st["limited_sites"] > 0
    J, g, gU, gB, _ = gpu_adjoint(cfg, f0, T, K)
    # the median's window sites can lie within 1e-5 of each other in Delta S:
    # the smaller step keeps their order (FP64 forward noise stays ~1e-7)
    h = 1e-7 if collision == "median" else 1e-6
    cd = lambda key, x0: (_ke_fp64(dict(cfg, **{key: x0 + h}), f0, T) -
                          _ke_fp64(dict(cfg, **{key: x0 - h}), f0, T)) / (2 * h)
    fdU, fdB = cd("lid_u", 0.1), cd("beta", beta)
    assert abs(gU - fdU) <= 1e-4 * abs(fdU), (gU, fdU)
    assert abs(gB - fdB) <= 1e-4 * abs(fdB), (gB, fdB)
    # every population moves at once here, so a smaller step keeps all 300
    # selections unchanged
    v, hv = WL.normal_noise(f0.shape, 9, 1.0), 1e-8
    dv = (_ke_fp64(cfg, f0 + hv * v, T) - _ke_fp64(cfg, f0 - hv * v, T)) / (2 * hv)
    assert abs((g * v).sum() - dv) <= 1e-4 * abs(dv), ((g * v).sum(), dv)
    Jo, go, gUo, gBo = O.adjoint_ke(cfg, f0, T)
    assert abs(gU - gUo) <= 1e-4 * abs(gUo) and abs(gB - gBo) <= 1e-4 * abs(gBo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_autograd_function_uses_the_adjoint():
    cfg = dict(CASES["cavity_ehrenfest"], precision="fp64")
    f0 = start_state(cfg, 21)
    T, K = 40, 12
    f0t = torch.tensor(f0, device="cuda", requires_grad=True)
    U = torch.tensor(0.1, dtype=torch.float64, device="cuda", requires_grad=True)
    B = torch.tensor(cfg["beta"], dtype=torch.float64, device="cuda", requires_grad=True)
    J = lbm.kinetic_energy(f0t, U, B, cfg, T, K)
    (2.0 * J).backward()
    Jo, go, gUo, gBo = O.adjoint_ke(cfg, f0, T)
    assert abs(J.item() - Jo) <= 1e-12 * abs(Jo)
    assert np.linalg.norm(f0t.grad.cpu().numpy() - 2 * go) <= 1e-10 * np.linalg.norm(2 * go)
    assert abs(U.grad.item() - 2 * gUo) <= 1e-10 * abs(2 * gUo)
    assert abs(B.grad.item() - 2 * gBo) <= 1e-10 * abs(2 * gBo)
