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
    c.collision = 12
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
