"""The allocation-free Ehrenfest step (lbm_ehrenfest_step_noalloc).

Some callers cannot allocate device memory where they step (a host framework
that owns a fixed device pool and passes only the population buffer, or a
loop that must not call cudaMalloc because it can synchronise the device).
This entry point serves them with scratch held in a file-scope device array
of the library.  The tests check, through the C ABI, that two calls in a row
give bit for bit what the regular lbm_step gives on the same state (the same
kernels and per-site arithmetic on a dense instead of a padded layout), for
FP32, FP64 and 16-bit storage, odd and even widths and a D1Q3 line, and that
an oversized lattice is refused.  It lives in a file of its own that pytest
collects last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu

W9 = [4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36]  # rest, E, SE, S, SW, W, NW, N, NE
W3 = [1 / 6, 2 / 3, 1 / 6]
STORE = {"fp64": torch.float64, "fp32": torch.float32, "fp16_dev": torch.float16, "bf16_dev": torch.bfloat16}


def _state(cfg, seed):
    ny, nx = cfg["ny"], cfg["nx"]
    fields = WL.random_fields(ny, nx, seed, 0.05, 0.05)
    uy = None if cfg["lattice"] == "D1Q3" else fields["uy"]
    f = O.init_equilibrium(dict(cfg, collision="lbgk"), fields["rho"], fields["ux"], uy)
    f = f * WL.lognormal_factors(f.shape, seed + 1, 0.01)
    f = f * WL.lognormal_factors(f.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, 20, 0.4)[None])
    return f


def _weights(cfg):
    w = W3 if cfg["lattice"] == "D1Q3" else W9
    return torch.tensor(w, dtype=torch.float32, device="cuda")[:, None, None]


def _encode(cfg, f):
    """The caller's dense array in the storage format (16-bit: f_i - W_i in
    FP32, rounded to nearest even, as the library stores it)."""
    prec = cfg["precision"]
    if prec in ("fp64", "fp32"):
        return f.to(STORE[prec]).contiguous()
    return (f.float() - _weights(cfg)).to(STORE[prec]).contiguous()


def _decode(cfg, d):
    if cfg["precision"] in ("fp64", "fp32"):
        return d
    return d.float() + _weights(cfg)


CASES = {
    "d2q9_fp32_odd": dict(lattice="D2Q9", nx=129, ny=97, bc="cavity", lid_u=0.1, precision="fp32"),
    "d2q9_fp32_even": dict(lattice="D2Q9", nx=128, ny=96, bc="cavity", lid_u=0.1, precision="fp32"),
    "d2q9_fp64_even": dict(lattice="D2Q9", nx=128, ny=96, bc="periodic", precision="fp64"),
    "d2q9_fp16_even": dict(lattice="D2Q9", nx=128, ny=96, bc="cavity", lid_u=0.1, precision="fp16_dev"),
    "d2q9_bf16_odd": dict(lattice="D2Q9", nx=129, ny=97, bc="channel", lid_u=0.05, precision="bf16_dev"),
    "d1q3_fp64": dict(lattice="D1Q3", nx=301, ny=1, bc="ends", precision="fp64"),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_step_matches_lbm_step_on_two_calls(case):
    """Two calls of 4 steps each; after every call the caller's dense array
    equals lbm_step's state bit for bit (the selected sites are rewritten to
    f*, so equal states mean equal selections), and the limiter acted."""
    cfg = dict(CASES[case], collision="ehrenfest", beta=0.97, topk=5, delta=2e-4)
    f0 = _state(cfg, 31)
    wide = torch.float64 if cfg["precision"] == "fp64" else torch.float32
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, dtype=wide, device="cuda"))
    dense = _encode(cfg, lat.get_state(wide))
    assert torch.equal(_decode(cfg, dense), lat.get_state(wide))  # same starting state
    c = lbm.LBMConfig.from_dict(cfg).to_c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        lat.step(4)
        rc = lbm.lib().lbm_ehrenfest_step_noalloc(C.byref(c), C.c_void_p(dense.data_ptr()), 4, stream)
        assert rc == 0, lbm.STATUS.get(rc, rc)
        ref = lat.get_state(wide)
        got = _decode(cfg, dense)
        diff = int((got != ref).sum())
        assert diff == 0, (case, call, diff)
    assert lat.stats()["limited_total"] > 0  # the limiter acted on this state


def test_noalloc_rejects_lattices_beyond_its_scratch():
    big = lbm.LBMConfig.from_dict(dict(lattice="D2Q9", nx=4097, ny=4097, collision="ehrenfest",
                                       precision="fp32", beta=0.9)).to_c()
    dummy = torch.zeros(1, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lbm.lib().lbm_ehrenfest_step_noalloc(C.byref(big), C.c_void_p(dummy.data_ptr()), 2, stream)
    assert rc == 3  # LBM_ERR_OOM: the static scratch is too small for this lattice
    odd = lbm.LBMConfig.from_dict(dict(lattice="D2Q9", nx=8, ny=8, collision="ehrenfest",
                                       precision="fp32", beta=0.9)).to_c()
    assert lbm.lib().lbm_ehrenfest_step_noalloc(C.byref(odd), C.c_void_p(dummy.data_ptr()), 3,
                                                stream) == 1  # odd step count
    bad = lbm.LBMConfig.from_dict(dict(lattice="D2Q9", nx=8, ny=8, collision="ehrenfest",
                                       precision="fp32", beta=0.9, lid_u=float("inf"))).to_c()
    assert lbm.lib().lbm_ehrenfest_step_noalloc(C.byref(bad), C.c_void_p(dummy.data_ptr()), 2,
                                                stream) == 1  # the checks of lbm_create
