"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the lattice Boltzmann path runs in
the CUDA kernels of ``_lib/liblbm.so``.  PyTorch supplies the device
allocation and the current stream.  Importing this module fails loudly when
the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm.so")

LATTICES = {"D1Q3": 1, "D2Q9": 2}
COLLISIONS = {"lbgk": 0, "elbm": 1, "ehrenfest": 2, "positivity": 3, "median": 4, "mrt": 5,
              "smooth": 6, "double_monotonic": 7, "ensemble": 8, "threshold": 9, "mrt2": 10,
              "mrt_limiter": 11, "ensemble_lagged": 12}
EQUILIBRIA = {"poly": 0, "entropic": 1, "poly_std": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16_dev": 2, "fp16_dev": 3}
BCS = {"cavity": 0, "ends": 1, "periodic": 2, "channel": 3, "diffusive": 4}
NORMS = {"entropic": 0, "l1": 1}
FALLBACKS = {"positivity": 0, "ehrenfest": 1}
DTYPE_F64, DTYPE_F32 = 0, 1
ABI_VERSION = 2  # LBM_ABI_VERSION of include/lbm.h (lbm_config layout)
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM",
          4: "LBM_ERR_DIVERGED", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}

# every symbol declared in include/lbm.h
EXPORTS = ["lbm_config_default", "lbm_required_bytes", "lbm_create", "lbm_destroy", "lbm_init",
           "lbm_init_device", "lbm_set_state", "lbm_get_state", "lbm_step", "lbm_macros",
           "lbm_entropy", "lbm_stats_get", "lbm_last_candidates", "lbm_last_error",
           "lbm_status_string", "lbm_abi_version", "lbm_profile_enable", "lbm_profile_read",
           "lbm_ehrenfest_step_noalloc", "lbm_batch_required_bytes", "lbm_batch_create",
           "lbm_batch_destroy", "lbm_batch_init_uniform", "lbm_batch_set_state",
           "lbm_batch_get_state", "lbm_batch_step", "lbm_batch_stats", "lbm_batch_last_error",
           "lbm_adjoint_required_bytes", "lbm_adjoint_forward", "lbm_adjoint_backward",
           "lbm_fp64_rates", "lbm_enstrophy", "lbm_probe_set", "lbm_probe_count",
           "lbm_mrt_preset", "lbm_batch_opts_default", "lbm_batch_required_bytes_ex",
           "lbm_batch_create_ex", "lbm_batch_get_opts", "lbm_batch_group_times", "lbm_batch_tune_bytes",
           "lbm_batch_tune", "lbm_batch_debug_hold"]


class lbm_config(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("collision", C.c_int),
        ("equilibrium", C.c_int), ("precision", C.c_int), ("bc", C.c_int),
        ("beta", C.c_double), ("nu", C.c_double), ("lid_u", C.c_double),
        ("topk", C.c_int), ("delta", C.c_double),
        ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
        ("elbm_eps", C.c_double), ("elbm_max_iter", C.c_int), ("elbm_norm", C.c_int),
        ("elbm_fallback", C.c_int),
        ("lim_alpha", C.c_double), ("lim_k", C.c_double), ("lim_dst", C.c_double),
        ("lim_delta0", C.c_double),
    ]


class lbm_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "steps", "candidates_last", "limited_total", "elbm_solved", "elbm_skipped",
        "elbm_fallbacks", "elbm_iters_total", "elbm_iters_max", "diverged", "overflow",
        "screened_last")]


class lbm_batch_opts(C.Structure):
    _fields_ = [("tile_x", C.c_int), ("ctas_per_sm", C.c_int), ("chunk", C.c_int), ("order", C.c_int),
                ("graph_steps", C.c_int), ("wait_ms", C.c_double), ("tile_rows", C.c_int)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class lbm_batch_tune_record(C.Structure):
    _fields_ = [("opts", lbm_batch_opts), ("ms_per_step", C.c_double), ("objective", C.c_double)]


BATCH_KINDS = ["lbgk", "elbm", "ehrenfest", "positivity", "median", "mrt"]  # LBM_LBGK ... LBM_MRT


class LBMError(RuntimeError):
    pass


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    p, i, sz = C.c_void_p, C.c_int, C.c_size_t
    sig = {
        "lbm_config_default": (i, [C.POINTER(lbm_config)]),
        "lbm_required_bytes": (i, [C.POINTER(lbm_config), C.POINTER(sz)]),
        "lbm_mrt_preset": (i, [C.POINTER(lbm_config), i]),
        "lbm_create": (i, [C.POINTER(lbm_config), p, sz, C.POINTER(p)]),
        "lbm_destroy": (None, [p]),
        "lbm_init": (i, [p, p, p, p, p]),
        "lbm_init_device": (i, [p, p, p, p, p]),
        "lbm_set_state": (i, [p, p, i, p]),
        "lbm_get_state": (i, [p, p, i, p]),
        "lbm_step": (i, [p, i, p]),
        "lbm_macros": (i, [p, p, p, i, p]),
        "lbm_entropy": (i, [p, C.POINTER(C.c_double), p, p]),
        "lbm_stats_get": (i, [p, C.POINTER(lbm_stats), p]),
        "lbm_last_candidates": (i, [p, p, p, p, i, C.POINTER(i), p]),
        "lbm_last_error": (C.c_char_p, [p]),
        "lbm_status_string": (C.c_char_p, [i]),
        "lbm_abi_version": (i, []),
        "lbm_profile_enable": (i, [p, i]),
        "lbm_profile_read": (i, [p, C.POINTER(i), C.POINTER(C.c_double)]),
        "lbm_ehrenfest_step_noalloc": (i, [C.POINTER(lbm_config), p, i, p]),
        "lbm_fp64_rates": (i, [C.POINTER(C.c_double), C.POINTER(C.c_double), p]),
        "lbm_enstrophy": (i, [p, C.POINTER(C.c_double), p]),
        "lbm_probe_set": (i, [p, i, i, p, i]),
        "lbm_probe_count": (i, [p, C.POINTER(C.c_uint64), p]),
        "lbm_batch_required_bytes": (i, [C.POINTER(lbm_config), i, C.POINTER(sz)]),
        "lbm_batch_create": (i, [C.POINTER(lbm_config), i, p, sz, C.POINTER(p)]),
        "lbm_batch_destroy": (None, [p]),
        "lbm_batch_init_uniform": (i, [p, C.c_double, C.c_double, C.c_double, p]),
        "lbm_batch_set_state": (i, [p, i, p, i, p]),
        "lbm_batch_get_state": (i, [p, i, p, i, p]),
        "lbm_batch_step": (i, [p, i, C.POINTER(i), p]),
        "lbm_batch_stats": (i, [p, i, C.POINTER(lbm_stats), p]),
        "lbm_batch_last_error": (C.c_char_p, [p]),
        "lbm_batch_opts_default": (i, [C.POINTER(lbm_batch_opts)]),
        "lbm_batch_required_bytes_ex": (i, [C.POINTER(lbm_config), i, C.POINTER(lbm_batch_opts),
                                            C.POINTER(sz)]),
        "lbm_batch_create_ex": (i, [C.POINTER(lbm_config), i, C.POINTER(lbm_batch_opts), p, sz,
                                    C.POINTER(p)]),
        "lbm_batch_get_opts": (i, [p, C.POINTER(lbm_batch_opts)]),
        "lbm_batch_group_times": (i, [p, i, C.POINTER(C.c_double), p]),
        "lbm_batch_tune_bytes": (i, [C.POINTER(lbm_config), i, C.POINTER(sz)]),
        "lbm_batch_tune": (i, [C.POINTER(lbm_config), i, p, sz, i, C.POINTER(lbm_batch_opts),
                               C.POINTER(lbm_batch_tune_record), i, C.POINTER(i), C.POINTER(C.c_double), p]),
        "lbm_batch_debug_hold": (i, [p, i, p]),
        "lbm_adjoint_required_bytes": (i, [C.POINTER(lbm_config), i, i, C.POINTER(sz)]),
        "lbm_adjoint_forward": (i, [p, i, i, p, sz, C.POINTER(C.c_double), p]),
        "lbm_adjoint_backward": (i, [p, i, i, p, i, p, i, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), p, sz, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.lbm_abi_version() != ABI_VERSION:
        raise LBMError(f"{path}: ABI version {lib.lbm_abi_version()}, this binding needs {ABI_VERSION} "
                       "(rebuild with paper_1110_0270_gb300.build)")
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


@dataclasses.dataclass
class LBMConfig:
    """Python mirror of ``lbm_config``; accepts the names used by the
    workload generators (``nu`` instead of ``beta`` where given)."""
    lattice: str = "D2Q9"
    nx: int = 16
    ny: int = 16
    collision: str = "lbgk"
    equilibrium: str = "poly"
    precision: str = "fp32"
    bc: str = "cavity"
    beta: float = 0.0
    nu: float = 0.0
    lid_u: float = 0.0
    topk: int = 0
    delta: float = 1e-3
    s_e: float = 1.64
    s_eps: float = 1.54
    s_q: float = 1.9
    elbm_eps: float = 1e-15
    elbm_max_iter: int = 20
    elbm_norm: str = "entropic"
    elbm_fallback: str = "positivity"
    lim_alpha: float = 1.0
    lim_k: float = 1.0
    lim_dst: float = 1e-3
    lim_delta0: float = 0.01

    @classmethod
    def from_dict(cls, d: dict) -> "LBMConfig":
        names = {f.name for f in dataclasses.fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in names})

    @property
    def Q(self) -> int:
        return 3 if self.lattice == "D1Q3" else 9

    def to_c(self) -> lbm_config:
        return lbm_config(LATTICES[self.lattice], int(self.nx), int(self.ny),
                          COLLISIONS[self.collision], EQUILIBRIA[self.equilibrium],
                          PRECISIONS[self.precision], BCS[self.bc], float(self.beta),
                          float(self.nu), float(self.lid_u), int(self.topk), float(self.delta),
                          float(self.s_e), float(self.s_eps), float(self.s_q),
                          float(self.elbm_eps), int(self.elbm_max_iter), NORMS[self.elbm_norm],
                          FALLBACKS[self.elbm_fallback], float(self.lim_alpha), float(self.lim_k),
                          float(self.lim_dst), float(self.lim_delta0))


def required_bytes(cfg) -> int:
    cfg = cfg if isinstance(cfg, LBMConfig) else LBMConfig.from_dict(cfg)
    c = cfg.to_c()
    n = C.c_size_t()
    rc = lib().lbm_required_bytes(C.byref(c), C.byref(n))
    if rc != 0:
        raise LBMError(f"lbm_required_bytes: {STATUS.get(rc, rc)} for {cfg}")
    return n.value


def _stream(stream=None) -> C.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class Lattice:
    """One lattice on the current CUDA device, backed by a torch uint8 tensor.

    All methods enqueue on the current torch stream unless `stream` is given.
    """

    def __init__(self, cfg, device=None):
        import torch
        self.cfg = cfg if isinstance(cfg, LBMConfig) else LBMConfig.from_dict(cfg)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.Q = self.cfg.Q
        self._c = self.cfg.to_c()
        self.nbytes = required_bytes(self.cfg)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().lbm_create(C.byref(self._c), _ptr(self.mem), self.nbytes, C.byref(h))
        if rc != 0:
            msg = lib().lbm_last_error(None)
            raise LBMError(f"lbm_create: {STATUS.get(rc, rc)}: {msg.decode() if msg else ''}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.lbm_destroy(h)
            self._h = None

    # -- helpers
    def _check(self, rc: int, what: str):
        if rc != 0:
            msg = lib().lbm_last_error(self._h)
            raise LBMError(f"{what}: {STATUS.get(rc, rc)}: {msg.decode() if msg else ''}")

    @property
    def shape(self):
        return (self.Q, self.cfg.ny, self.cfg.nx)

    # -- ABI calls
    def init(self, rho, ux, uy=None, stream=None):
        """f = f*(rho, u) from host arrays (numpy float64, [ny][nx])."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux)]
        arrs.append(np.ascontiguousarray(uy, dtype=np.float64) if uy is not None else None)
        p = [a.ctypes.data_as(C.c_void_p) if a is not None else None for a in arrs]
        self._check(lib().lbm_init(self._h, *p, _stream(stream)), "lbm_init")

    def init_device(self, rho, ux, uy=None, stream=None):
        p = [_ptr(a) if a is not None else None for a in (rho, ux, uy)]
        self._check(lib().lbm_init_device(self._h, *p, _stream(stream)), "lbm_init_device")

    def set_state(self, f, stream=None):
        import torch
        assert f.is_cuda and f.is_contiguous() and tuple(f.shape) == self.shape
        dt = DTYPE_F64 if f.dtype == torch.float64 else DTYPE_F32
        assert f.dtype in (torch.float64, torch.float32)
        self._check(lib().lbm_set_state(self._h, _ptr(f), dt, _stream(stream)), "lbm_set_state")

    def get_state(self, dtype=None, out=None, stream=None):
        import torch
        dtype = dtype or torch.float64
        out = out if out is not None else torch.empty(self.shape, dtype=dtype, device=self.device)
        dt = DTYPE_F64 if out.dtype == torch.float64 else DTYPE_F32
        self._check(lib().lbm_get_state(self._h, _ptr(out), dt, _stream(stream)), "lbm_get_state")
        return out

    def step(self, n: int = 1, stream=None):
        self._check(lib().lbm_step(self._h, int(n), _stream(stream)), "lbm_step")

    def macros(self, dtype=None, stream=None):
        import torch
        dtype = dtype or torch.float64
        rho = torch.empty((self.cfg.ny, self.cfg.nx), dtype=dtype, device=self.device)
        u = torch.empty((2 if self.Q == 9 else 1, self.cfg.ny, self.cfg.nx), dtype=dtype,
                        device=self.device)
        dt = DTYPE_F64 if dtype == torch.float64 else DTYPE_F32
        self._check(lib().lbm_macros(self._h, _ptr(rho), _ptr(u), dt, _stream(stream)), "lbm_macros")
        return rho, u

    def entropy(self, field: bool = False, stream=None):
        import torch
        H = C.c_double()
        dS = torch.empty((self.cfg.ny, self.cfg.nx), dtype=torch.float64,
                         device=self.device) if field else None
        self._check(lib().lbm_entropy(self._h, C.byref(H), _ptr(dS) if field else None,
                                      _stream(stream)), "lbm_entropy")
        return (H.value, dS) if field else H.value

    def probe(self, x: int, y: int, cap: int):
        """Record the velocity of site (x, y) at every following step into a
        device ring buffer of cap samples (None for x turns it off)."""
        import torch
        if x is None:
            self._probe = None
            self._check(lib().lbm_probe_set(self._h, 0, 0, None, 0), "lbm_probe_set")
            return
        self._probe = torch.zeros((cap, 2), dtype=torch.float64, device=self.device)
        self._check(lib().lbm_probe_set(self._h, int(x), int(y), _ptr(self._probe), int(cap)), "lbm_probe_set")

    def probe_signal(self):
        """The recorded samples in time order (the last cap of them) as a
        host array [n, 2] of (u_x, u_y)."""
        n = C.c_uint64()
        self._check(lib().lbm_probe_count(self._h, C.byref(n), None), "lbm_probe_count")
        cap = self._probe.shape[0]
        buf = self._probe.cpu().numpy()
        k = int(n.value)
        if k <= cap:
            return buf[:k].copy()
        start = k % cap
        return np.concatenate([buf[start:], buf[:start]])

    def enstrophy(self, stream=None) -> float:
        """Section 8's enstrophy: mean over sites of the vorticity squared."""
        E = C.c_double()
        self._check(lib().lbm_enstrophy(self._h, C.byref(E), _stream(stream)), "lbm_enstrophy")
        return E.value

    def stats(self, stream=None) -> dict:
        st = lbm_stats()
        self._check(lib().lbm_stats_get(self._h, C.byref(st), _stream(stream)), "lbm_stats_get")
        return {n: int(getattr(st, n)) for n, _ in lbm_stats._fields_}

    def profile(self, enable: bool = True):
        """Start (or stop) per-kernel CUDA-event timing of step()."""
        self._check(lib().lbm_profile_enable(self._h, int(enable)), "lbm_profile_enable")

    def profile_read(self) -> dict:
        """{kind: (launches, total_ms)} for the 'step' and 'fixup' kernels."""
        n = (C.c_int * 2)()
        ms = (C.c_double * 2)()
        self._check(lib().lbm_profile_read(self._h, n, ms), "lbm_profile_read")
        return {"step": (n[0], ms[0]), "fixup": (n[1], ms[1])}

    # -- reverse mode
    def adjoint_work(self, T: int, K: int):
        import torch
        n = C.c_size_t()
        rc = lib().lbm_adjoint_required_bytes(C.byref(self._c), int(T), int(K), C.byref(n))
        if rc != 0:
            raise LBMError(f"lbm_adjoint_required_bytes: {STATUS.get(rc, rc)}")
        return torch.empty(n.value, dtype=torch.uint8, device=self.device)

    def adjoint_forward(self, T: int, K: int, work=None, stream=None):
        """T steps with checkpoints every K; returns (J, work)."""
        work = work if work is not None else self.adjoint_work(T, K)
        J = C.c_double()
        self._check(lib().lbm_adjoint_forward(self._h, int(T), int(K), _ptr(work), work.numel(),
                                              C.byref(J), _stream(stream)), "lbm_adjoint_forward")
        return J.value, work

    def adjoint_backward(self, T: int, K: int, work, seed=None, stream=None):
        """(dJ/df0 as a float64 tensor, dJ/dU, dJ/dbeta) after adjoint_forward."""
        import torch
        g = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        gU, gB = C.c_double(), C.c_double()
        sdt = DTYPE_F64 if seed is None or seed.dtype == torch.float64 else DTYPE_F32
        self._check(lib().lbm_adjoint_backward(
            self._h, int(T), int(K), _ptr(seed) if seed is not None else None, sdt, _ptr(g),
            DTYPE_F64, C.byref(gU), C.byref(gB), _ptr(work), work.numel(), _stream(stream)),
            "lbm_adjoint_backward")
        return g, gU.value, gB.value

    def last_candidates(self, cap: int | None = None, stream=None):
        """(delta_s float64, site int32, selected int32) of the last step."""
        cap = cap if cap is not None else self.cfg.nx * self.cfg.ny
        ds = np.zeros(cap, np.float64)
        site = np.zeros(cap, np.int32)
        sel = np.zeros(cap, np.int32)
        n = C.c_int()
        self._check(lib().lbm_last_candidates(
            self._h, ds.ctypes.data_as(C.c_void_p), site.ctypes.data_as(C.c_void_p),
            sel.ctypes.data_as(C.c_void_p), cap, C.byref(n), _stream(stream)), "lbm_last_candidates")
        m = min(n.value, cap)
        return ds[:m], site[:m], sel[:m]


MRT_PRESETS = {"trt": 0, "mrt": 1, "mrt1": 2, "mrt_ll": 3}


def mrt_rates(preset: str, beta: float) -> dict:
    """MRT relaxation rates (s_e, s_eps, s_q) of a preset, from the library's
    lbm_mrt_preset (Sections 5, 7 and 8; s_nu = 2 beta): 'trt', 'mrt',
    'mrt1' or 'mrt_ll' (LBM_MRT_PRESET_TRT / _MRT / _MRT1 / _LL).  Use with
    collision="mrt"."""
    if preset not in MRT_PRESETS:
        raise ValueError(f"unknown MRT preset {preset!r}")
    c = LBMConfig(beta=float(beta)).to_c()
    rc = lib().lbm_mrt_preset(C.byref(c), MRT_PRESETS[preset])
    if rc != 0:
        raise LBMError(f"lbm_mrt_preset: {STATUS.get(rc, rc)} for {preset!r}, beta={beta}")
    return {"s_e": c.s_e, "s_eps": c.s_eps, "s_q": c.s_q}


def fp64_rates(stream=None) -> dict:
    """Measured FP64 FMA rate (FLOP/s) and FP64 log() rate (1/s) of the
    current GPU: the ceilings of the FP64-bound step kernels."""
    fl, lg = C.c_double(0.0), C.c_double(0.0)
    rc = lib().lbm_fp64_rates(C.byref(fl), C.byref(lg), _stream(stream))
    if rc != 0:
        raise LBMError(f"lbm_fp64_rates: {STATUS.get(rc, rc)}")
    return {"dfma_flops": fl.value, "log_per_s": lg.value}


def batch_opts(**kw) -> lbm_batch_opts:
    """lbm_batch_opts with the library's defaults, overridden by kw."""
    o = lbm_batch_opts()
    lib().lbm_batch_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _configs(cfgs):
    cs = [c if isinstance(c, LBMConfig) else LBMConfig.from_dict(c) for c in cfgs]
    return cs, (lbm_config * len(cs))(*[c.to_c() for c in cs])


def batch_required_bytes(cfgs, opts=None) -> int:
    cs, arr = _configs(cfgs)
    n = C.c_size_t()
    rc = lib().lbm_batch_required_bytes_ex(arr, len(cs), C.byref(opts) if opts is not None else None,
                                           C.byref(n))
    if rc != 0:
        raise LBMError(f"lbm_batch_required_bytes: {STATUS.get(rc, rc)}")
    return n.value


def _tune_key(cs) -> str:
    """The tuner's cache key: precision, lattice x collision mix, and the
    size class (log2 of the total and of the largest instance's sites)."""
    import math
    mix = sorted({f"{c.lattice}/{c.collision}" for c in cs})
    sites = [c.nx * c.ny for c in cs]
    return "|".join([cs[0].precision, ",".join(mix), f"total2^{int(math.log2(sum(sites)))}",
                     f"max2^{int(math.log2(max(sites)))}", f"n{len(cs)}"])


def tune_batch(cfgs, steps: int = 4, cache: str | None = None, device=None) -> tuple[dict, list]:
    """The library's autotuner (lbm_batch_tune) for this batch: returns the
    chosen options and the timed sweep [(opts, summed group ms per step,
    objective)].  With a cache
    path the choice is read from / stored in a JSON file keyed by
    precision, lattice and collision mix and size class."""
    import json
    import torch
    cs, arr = _configs(cfgs)
    key = _tune_key(cs)
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            data = json.load(fh)
        if key in data:
            return data[key]["opts"], data[key]["sweep"]
    n = C.c_size_t()
    rc = lib().lbm_batch_tune_bytes(arr, len(cs), C.byref(n))
    if rc != 0:
        raise LBMError(f"lbm_batch_tune_bytes: {STATUS.get(rc, rc)}")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    mem = torch.empty(n.value, dtype=torch.uint8, device=dev)
    best = batch_opts()
    recs = (lbm_batch_tune_record * 64)()
    nrec, best_ms = C.c_int(), C.c_double()
    with torch.cuda.device(dev):
        rc = lib().lbm_batch_tune(arr, len(cs), _ptr(mem), n.value, int(steps), C.byref(best), recs, 64,
                                  C.byref(nrec), C.byref(best_ms), _stream(None))
    if rc != 0:
        raise LBMError(f"lbm_batch_tune: {STATUS.get(rc, rc)}")
    sweep = [(recs[k].opts.as_dict(), recs[k].ms_per_step, recs[k].objective) for k in range(min(nrec.value, 64))]
    out = best.as_dict()
    if cache:
        data = {}
        if os.path.exists(cache):
            with open(cache) as fh:
                data = json.load(fh)
        data[key] = {"opts": out, "objective": best_ms.value, "sweep": sweep}
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as fh:
            json.dump(data, fh, indent=1)
    return out, sweep


class Batch:
    """Many independent lattices (D2Q9 and D1Q3) advanced together by the
    library's persistent batched kernels (lbm_batch_*).  `opts`: a dict of
    lbm_batch_opts fields (None: the library's defaults)."""

    def __init__(self, cfgs, device=None, opts=None):
        import torch
        self.cfgs, self._arr = _configs(cfgs)
        self.n = len(self.cfgs)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self._opts = batch_opts(**(opts or {}))
        self.nbytes = batch_required_bytes(self.cfgs, self._opts)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().lbm_batch_create_ex(self._arr, self.n, C.byref(self._opts), _ptr(self.mem), self.nbytes,
                                           C.byref(h))
        if rc != 0:
            raise LBMError(f"lbm_batch_create: {STATUS.get(rc, rc)}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.lbm_batch_destroy(h)
            self._h = None

    def _check(self, rc, what):
        if rc != 0:
            msg = lib().lbm_batch_last_error(self._h)
            raise LBMError(f"{what}: {STATUS.get(rc, rc)}: {msg.decode() if msg else ''}")

    @property
    def opts(self) -> dict:
        o = lbm_batch_opts()
        self._check(lib().lbm_batch_get_opts(self._h, C.byref(o)), "lbm_batch_get_opts")
        return o.as_dict()

    def shape(self, i):
        return (self.cfgs[i].Q, self.cfgs[i].ny, self.cfgs[i].nx)

    def init_uniform(self, rho=1.0, ux=0.0, uy=0.0, stream=None):
        self._check(lib().lbm_batch_init_uniform(self._h, rho, ux, uy, _stream(stream)),
                    "lbm_batch_init_uniform")

    def set_state(self, i, f, stream=None):
        import torch
        assert f.is_cuda and f.is_contiguous() and tuple(f.shape) == self.shape(i)
        dt = DTYPE_F64 if f.dtype == torch.float64 else DTYPE_F32
        self._check(lib().lbm_batch_set_state(self._h, i, _ptr(f), dt, _stream(stream)),
                    "lbm_batch_set_state")

    def get_state(self, i, dtype=None, stream=None):
        import torch
        dtype = dtype or torch.float64
        out = torch.empty(self.shape(i), dtype=dtype, device=self.device)
        dt = DTYPE_F64 if dtype == torch.float64 else DTYPE_F32
        self._check(lib().lbm_batch_get_state(self._h, i, _ptr(out), dt, _stream(stream)),
                    "lbm_batch_get_state")
        return out

    def step(self, n=1, status=False, stream=None):
        st = (C.c_int * self.n)() if status else None
        self._check(lib().lbm_batch_step(self._h, int(n), st, _stream(stream)), "lbm_batch_step")
        return [STATUS[v] for v in st] if status else None

    def step_status(self, n=1, stream=None) -> int:
        """lbm_batch_step with status; returns the raw lbm_status code."""
        st = (C.c_int * self.n)()
        return lib().lbm_batch_step(self._h, int(n), st, _stream(stream))

    def group_times(self, n: int, stream=None) -> dict:
        """{collision: ms} of each collision group advanced alone n steps."""
        ms = (C.c_double * 6)()
        self._check(lib().lbm_batch_group_times(self._h, int(n), ms, _stream(stream)), "lbm_batch_group_times")
        return {k: ms[j] for j, k in enumerate(BATCH_KINDS) if ms[j] > 0.0}

    def debug_hold(self, i: int, stream=None):
        self._check(lib().lbm_batch_debug_hold(self._h, int(i), _stream(stream)), "lbm_batch_debug_hold")

    def stats(self, i, stream=None) -> dict:
        st = lbm_stats()
        self._check(lib().lbm_batch_stats(self._h, i, C.byref(st), _stream(stream)), "lbm_batch_stats")
        return {n: int(getattr(st, n)) for n, _ in lbm_stats._fields_}


def _kinetic_energy_function():
    import torch

    class KineticEnergy(torch.autograd.Function):
        """J = 1/2 sum rho |u|^2 after T steps of the configured LBGK or
        Ehrenfest step, as a differentiable function of the initial
        populations f0 [Q, ny, nx], the lid velocity and beta (0-d tensors).
        Forward runs the CUDA step with checkpoints every K steps; backward
        runs the hand-written adjoint kernels (lbm_adjoint_backward)."""

        @staticmethod
        def forward(ctx, f0, lid_u, beta, cfg, T, K):
            c = LBMConfig.from_dict(dict(cfg, lid_u=float(lid_u), beta=float(beta)))
            lat = Lattice(c, device=f0.device)
            dt = torch.float64 if c.precision == "fp64" else torch.float32
            lat.set_state(f0.detach().to(dt).contiguous())
            J, work = lat.adjoint_forward(T, K)
            ctx.lat, ctx.work, ctx.T, ctx.K = lat, work, T, K
            ctx.dtypes = (f0.dtype, lid_u.dtype, beta.dtype)
            return torch.tensor(J, dtype=torch.float64, device=f0.device)

        @staticmethod
        def backward(ctx, gJ):
            g, gU, gB = ctx.lat.adjoint_backward(ctx.T, ctx.K, ctx.work)
            df0, dU, dB = ctx.dtypes
            dev = g.device
            f64 = torch.float64
            return ((gJ * g).to(df0), (gJ * torch.tensor(gU, dtype=f64, device=dev)).to(dU),
                    (gJ * torch.tensor(gB, dtype=f64, device=dev)).to(dB), None, None, None)

    return KineticEnergy


def kinetic_energy(f0, lid_u, beta, cfg, T: int, K: int):
    """Differentiable kinetic energy after T steps (see KineticEnergy)."""
    return _kinetic_energy_function().apply(f0, lid_u, beta, cfg, T, K)
