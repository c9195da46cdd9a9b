"""Host-side checks of the C ABI library (no GPU needed): it loads, exports
every function include/lbm.h declares, and validates configurations."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1110_0270_gb300 import build as B
from paper_1110_0270_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 16
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lbm_\w+)", out))
    assert set(names) <= exported, set(names) - exported
    assert set(names) == set(lbm.EXPORTS)
    for n in names:
        assert hasattr(lib, n)


def test_abi_version_and_status_strings(lib):
    assert lib.lbm_abi_version() == lbm.ABI_VERSION == 2
    assert lib.lbm_status_string(0) == b"LBM_OK"
    assert lib.lbm_status_string(4) == b"LBM_ERR_DIVERGED"


def test_required_bytes_and_config_validation(lib):
    c = lbm.lbm_config()
    assert lib.lbm_config_default(C.byref(c)) == 0
    n = C.c_size_t()
    assert lib.lbm_required_bytes(C.byref(c), C.byref(n)) == 0
    # populations: 9 planes of 16 x 32 (pitch) floats, plus aligned scratch
    assert n.value >= 9 * 16 * 32 * 4
    base = lbm.required_bytes(dict(lattice="D2Q9", nx=100, ny=50, precision="fp32", beta=0.9))
    ehr = lbm.required_bytes(dict(lattice="D2Q9", nx=100, ny=50, precision="fp32", beta=0.9,
                                  collision="ehrenfest", topk=4))
    assert ehr > base  # candidate list
    f64 = lbm.required_bytes(dict(lattice="D2Q9", nx=100, ny=50, precision="fp64", beta=0.9))
    assert f64 > base
    bad = [dict(lattice="D1Q3", nx=10, ny=2, beta=0.9),
           dict(lattice="D2Q9", nx=0, ny=5, beta=0.9),
           dict(lattice="D2Q9", nx=5, ny=5, beta=1.5),
           dict(lattice="D2Q9", nx=5, ny=5, beta=0.0, nu=0.0),
           dict(lattice="D2Q9", nx=5, ny=5, beta=0.9, topk=-1),
           dict(lattice="D1Q3", nx=5, ny=1, beta=0.9, bc="channel")]
    for d in bad:
        with pytest.raises(lbm.LBMError):
            lbm.required_bytes(d)
    # nu converts to beta inside the library
    assert lbm.required_bytes(dict(lattice="D2Q9", nx=5, ny=5, beta=0.0, nu=0.01)) > 0


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    c = lbm.LBMConfig(nx=8, ny=8, beta=0.9).to_c()
    h = C.c_void_p()
    # NULL and misaligned device pointers are rejected before any CUDA call
    assert lib.lbm_create(C.byref(c), None, 1 << 20, C.byref(h)) == 1
    assert lib.lbm_create(C.byref(c), C.c_void_p(0x1001), 1 << 20, C.byref(h)) == 1
    assert lib.lbm_create(C.byref(c), C.c_void_p(0x100000), 16, C.byref(h)) == 3  # too small


def test_batch_validation_is_host_side(lib):
    ok = [dict(lattice="D2Q9", nx=10, ny=12, beta=0.9, precision="fp32"),
          dict(lattice="D2Q9", nx=64, ny=8, beta=0.9, precision="fp32", collision="ehrenfest", topk=2)]
    n = lbm.batch_required_bytes(ok)
    assert n >= lbm.required_bytes(ok[0])
    for bad in ([dict(lattice="D2Q9", nx=10, ny=12, beta=0.9, precision="fp32"),
                 dict(lattice="D2Q9", nx=10, ny=12, beta=0.9, precision="fp64")],
                [dict(lattice="D1Q3", nx=10, ny=1, beta=0.9)]):
        with pytest.raises(lbm.LBMError):
            lbm.batch_required_bytes(bad)


def test_limiter_config_defaults_and_validation(lib):
    """The Section 4.2-4.4 limiter fields: defaults from lbm_config_default
    match the binding's, and out-of-range values are rejected."""
    c = lbm.lbm_config()
    assert lib.lbm_config_default(C.byref(c)) == 0
    py = lbm.LBMConfig()
    assert (c.lim_alpha, c.lim_k, c.lim_dst, c.lim_delta0) == (py.lim_alpha, py.lim_k, py.lim_dst, py.lim_delta0)
    n = C.c_size_t()
    for coll, field, bad in [(6, "lim_alpha", 0.0), (6, "lim_k", -1.0), (7, "lim_dst", 0.0),
                             (7, "lim_k", 0.0), (8, "lim_alpha", -2.0), (9, "lim_delta0", -0.1)]:
        c2 = lbm.lbm_config()
        lib.lbm_config_default(C.byref(c2))
        c2.collision = coll
        assert lib.lbm_required_bytes(C.byref(c2), C.byref(n)) == 0, coll
        setattr(c2, field, bad)
        assert lib.lbm_required_bytes(C.byref(c2), C.byref(n)) == 1, (coll, field)
    c.collision = 13
    assert lib.lbm_required_bytes(C.byref(c), C.byref(n)) == 1
    # Section 5's A_2 collisions exist for D2Q9 only
    for coll in (10, 11):
        c.collision = coll
        assert lib.lbm_required_bytes(C.byref(c), C.byref(n)) == 0
        c.lattice, c.ny = 1, 1
        assert lib.lbm_required_bytes(C.byref(c), C.byref(n)) == 1
        c.lattice, c.ny = 2, 16
    # the threshold limiter carries a candidate list and reduction slots
    c.collision = 0
    lib.lbm_required_bytes(C.byref(c), C.byref(n))
    base = n.value
    c.collision = 9
    lib.lbm_required_bytes(C.byref(c), C.byref(n))
    assert n.value > base


def test_mrt_presets_follow_sections_5_7_8(lib):
    """lbm_mrt_preset writes the MRT rates of each preset (s_nu = 2 beta):
    TRT (Section 5) s_e = s_eps = s_nu and the magic s_q = 8 (2 - s_nu)/(8 - s_nu);
    MRT and MRT1 (Section 8); the Lallemand-Luo A_1 rates of Section 7; beta
    may come from nu; unknown presets and beta outside (0, 1] are refused."""
    for beta in (0.55, 0.8, 0.97):
        snu = 2 * beta
        magic = 8 * (2 - snu) / (8 - snu)
        want = {"trt": (snu, snu, magic), "mrt": (1.64, 1.54, magic), "mrt1": (1.64, 1.54, 1.9),
                "mrt_ll": (1.64, 1.54, 3 * (2 - snu) / (3 - snu))}
        for name, (se, seps, sq) in want.items():
            r = lbm.mrt_rates(name, beta)
            assert r["s_e"] == pytest.approx(se, rel=1e-15)
            assert r["s_eps"] == pytest.approx(seps, rel=1e-15)
            assert r["s_q"] == pytest.approx(sq, rel=1e-15)
    # the TRT magic relation: (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16
    r = lbm.mrt_rates("trt", 0.9)
    assert (1 / 1.8 - 0.5) * (1 / r["s_q"] - 0.5) == pytest.approx(3 / 16, rel=1e-14)
    c = lbm.LBMConfig(beta=0.0, nu=0.01).to_c()
    assert lib.lbm_mrt_preset(C.byref(c), 0) == 0
    assert c.s_e == pytest.approx(2 / (6 * 0.01 + 1), rel=1e-15)
    assert lib.lbm_mrt_preset(C.byref(c), 7) == 1
    bad = lbm.LBMConfig(beta=1.5).to_c()
    assert lib.lbm_mrt_preset(C.byref(bad), 0) == 1
    assert lib.lbm_mrt_preset(None, 0) == 1
    with pytest.raises(ValueError):
        lbm.mrt_rates("nope", 0.9)
