"""Section 8's cavity studies (paper_1110_0270_gb300.experiments): the
method configurations of the stability study (host), and both runners at
small sizes against the oracle stepping the same lattices (GPU, FP64)."""
import numpy as np
import pytest

from paper_1110_0270_gb300 import experiments as X
from paper_1110_0270_gb300 import lbm
from paper_1110_0270_gb300.analysis import (dominant_frequency, hopf_energy, stream_function,
                                            vortex_summary)


def test_stability_configs_follow_section_8():
    """Six methods; L = n - 1, nu = u_wall L / Re; limiters capped at 9
    sites; TRT / MRT / MRT1 rates from the presets of the section."""
    cfgs = {m: X.stability_config(m, 5000.0) for m in X.STABILITY_METHODS}
    assert set(cfgs) == {"bgk", "ehrenfest", "mrt_limiter", "trt", "mrt", "mrt1"}
    for c in cfgs.values():
        assert (c["nx"], c["ny"], c["bc"], c["lid_u"]) == (129, 129, "cavity", 0.1)
        assert c["nu"] == pytest.approx(0.1 * 128 / 5000.0, rel=1e-15)
        lbm.LBMConfig.from_dict(c)  # every key is a config field
    assert cfgs["bgk"]["collision"] == "lbgk"
    for m in ("ehrenfest", "mrt_limiter"):
        assert cfgs[m]["collision"] == m and cfgs[m]["topk"] == 9 and cfgs[m]["delta"] == 1e-3
    snu = 2.0 / (6.0 * cfgs["trt"]["nu"] + 1.0)
    assert cfgs["trt"]["s_e"] == cfgs["trt"]["s_eps"] == pytest.approx(snu, rel=1e-15)
    # TRT's third-order rate keeps (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16
    assert (1 / snu - 0.5) * (1 / cfgs["trt"]["s_q"] - 0.5) == pytest.approx(3 / 16, rel=1e-12)
    assert (cfgs["mrt"]["s_e"], cfgs["mrt"]["s_eps"]) == (1.64, 1.54)
    assert cfgs["mrt"]["s_q"] == cfgs["trt"]["s_q"]
    assert (cfgs["mrt1"]["s_e"], cfgs["mrt1"]["s_eps"], cfgs["mrt1"]["s_q"]) == (1.64, 1.54, 1.9)
    with pytest.raises(ValueError):
        X.stability_config("elbm", 1000.0)


@pytest.mark.gpu
def test_stability_runner_matches_oracle():
    """A 17 x 17 cavity, Re 100 and 400, all six methods, 1200 steps with
    the enstrophy sampled at steps 1000 and 1200.  LBGK at Re 400 diverges
    in the oracle (density below zero after step 829 on this grid): the
    runner reports it in the chunk that holds the step reading that state
    (steps 800-1000).  Every other run survives, with the oracle's mean
    enstrophy and the vortices of the oracle's final stream function
    (clockwise primary vortex)."""
    import oracle as O
    n, steps = 17, 1200
    out = X.stability_sweep([100.0, 400.0], n=n, steps=steps, window=400, sample=200, check=400)
    assert out["steps"] == steps and len(out["runs"]) == 12
    chunk_ends = [400, 800, 1000, 1200]
    for r in out["runs"]:
        cfg = X.stability_config(r["method"], r["re"], n=n)
        f = O.init_equilibrium(cfg, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
        ens, bad = [], None
        for s in range(1, steps + 1):
            f = O.step(cfg, f, 1)
            rho = O.macros(cfg, f)[0]
            if not (np.isfinite(rho).all() and (rho > 0).all()):
                bad = s
                break
            if s in (1000, 1200):
                ens.append(O.enstrophy(cfg, f))
        if bad is not None:
            assert (r["method"], r["re"]) == ("bgk", 400.0)
            assert not r["survived"]
            assert r["diverged_by"] == min(e for e in chunk_ends if e >= bad + 1), (r, bad)
            continue
        assert r["survived"] and r["diverged_by"] is None, r
        assert r["enstrophy_mean"] == pytest.approx(np.mean(ens), rel=1e-10)
        assert r["enstrophy_min"] == pytest.approx(min(ens), rel=1e-10)
        _, ux, uy = O.macros(cfg, f)
        want = vortex_summary(stream_function(ux, uy))
        assert r["vortices"]["primary"]["psi"] < 0
        for k in ("primary", "secondary"):
            assert r["vortices"][k]["psi"] == pytest.approx(want[k]["psi"], rel=1e-9, abs=1e-14)
            assert (r["vortices"][k]["x"], r["vortices"][k]["y"]) == (want[k]["x"], want[k]["y"])
    assert out["survivors"]["400.0"] == ["ehrenfest", "mrt_limiter", "trt", "mrt", "mrt1"]


@pytest.mark.gpu
def test_hopf_runner_matches_oracle():
    """A 20 x 20 box with diffusive walls and the median filter, 600 steps
    keeping the last half of the control-point signal: E_u and the dominant
    frequency equal those of the oracle's signal at the same site."""
    import oracle as O
    n, steps, re = 20, 600, 300.0
    out = X.hopf_sweep([re], n=n, steps=steps, frac=0.5, chunk=256)
    p = out["points"][0]
    L = n - 1
    xp, yp = out["control_point"]
    assert (xp, yp) == (round(L / 16), round(13 * L / 16))
    cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="diffusive", lid_u=0.1, nu=0.1 * L / re, collision="median",
               equilibrium="entropic", delta=1e-3, precision="fp64")
    f = O.init_equilibrium(cfg, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    sig = []
    for _ in range(steps):
        f = O.step(cfg, f, 1)
        _, ux, _ = O.macros(cfg, f)
        sig.append(ux[yp, xp])
    sig = np.array(sig[steps // 2:])
    assert p["samples"] == sig.size and p["diverged"] == 0
    assert p["E_u"] == pytest.approx(hopf_energy(sig, L, 0.1), rel=1e-8)
    assert p["f_dom"] == pytest.approx(dominant_frequency(sig, L, 0.1)["f"], rel=1e-12)


@pytest.mark.gpu
def test_hopf_outside_walls_is_the_box_two_sites_larger():
    """walls="outside" reads n as the fluid sites: 18 x 18 fluid sites inside
    the wall sites is the 20-site box of the edge reading (L = 19, the same
    control point), so both give the same signal."""
    a = X.hopf_sweep([300.0], n=18, steps=400, frac=0.5, chunk=256, walls="outside")
    b = X.hopf_sweep([300.0], n=20, steps=400, frac=0.5, chunk=256)
    assert (a["n"], a["L"], a["fluid_sites"], a["walls"]) == (20, 19, 18, "outside")
    assert (b["fluid_sites"], b["walls"]) == (18, "edge")
    assert a["control_point"] == b["control_point"]
    assert a["points"][0]["E_u"] == b["points"][0]["E_u"]
    with pytest.raises(ValueError):
        X.hopf_sweep([300.0], n=18, steps=10, walls="inside")
