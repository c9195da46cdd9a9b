"""The allocation-free Ehrenfest step (lbm_ehrenfest_step_noalloc).

Some callers cannot allocate device memory where they step (a host framework
that owns a fixed device pool and passes only the population buffer, or a
loop that must not call cudaMalloc because it can synchronise the device).
This entry point serves them with scratch held in a file-scope device array
of the library.  The test checks, through the C ABI, that two calls in a row
give what the regular lbm_step gives on the same state, within the FP32
tolerance of the parity tests, and that an oversized lattice is refused.
It lives in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1110_0270_gb300 import lbm  # noqa: E402
from paper_1110_0270_gb300 import workloads as WL  # noqa: E402

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5  # rel-L2 bound of the FP32 parity tests


def _state(cfg, seed):
    ny, nx = cfg["ny"], cfg["nx"]
    fields = WL.random_fields(ny, nx, seed, 0.05, 0.05)
    f = O.init_equilibrium(dict(cfg, collision="lbgk"), fields["rho"], fields["ux"], fields["uy"])
    f = f * WL.lognormal_factors(f.shape, seed + 1, 0.01)
    f = f * WL.lognormal_factors(f.shape, seed + 2, 1.0) ** (WL.hot_spots(ny, nx, seed + 3, 20, 0.4)[None])
    return f


def test_noalloc_step_matches_lbm_step_on_two_calls():
    cfg = dict(lattice="D2Q9", nx=129, ny=97, bc="cavity", lid_u=0.1, collision="ehrenfest",
               precision="fp32", beta=0.97, topk=5, delta=2e-4)
    f0 = _state(cfg, 31).astype(np.float32)
    lat = lbm.Lattice(cfg)
    lat.set_state(torch.tensor(f0, device="cuda"))
    dense = torch.tensor(f0, device="cuda").contiguous()
    c = lbm.LBMConfig.from_dict(cfg).to_c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        lat.step(4)
        ref = lat.get_state(torch.float32).double().cpu().numpy()
        rc = lbm.lib().lbm_ehrenfest_step_noalloc(C.byref(c), C.c_void_p(dense.data_ptr()), 4, stream)
        assert rc == 0, lbm.STATUS.get(rc, rc)
        got = dense.double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= FP32_TOL, err
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
