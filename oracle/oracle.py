"""ctypes marshalling for the FP64 oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy
float64 in the natural layout ``f[i, y, x]`` (pre-collision, post-stream),
velocity numbering as in Section 5 of the paper (rest, E, SE, S, SW, W, NW,
N, NE) for D2Q9 and (-1, 0, +1) for D1Q3.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblbm_oracle.so")

LATTICES = {"D1Q3": 1, "D2Q9": 2}
COLLISIONS = {"lbgk": 0, "elbm": 1, "ehrenfest": 2, "positivity": 3, "median": 4, "mrt": 5,
              "smooth": 6, "double_monotonic": 7, "ensemble": 8, "threshold": 9, "mrt2": 10,
              "mrt_limiter": 11, "ensemble_lagged": 12}
EQUILIBRIA = {"poly": 0, "entropic": 1, "poly_std": 2}
BCS = {"cavity": 0, "ends": 1, "periodic": 2, "channel": 3, "diffusive": 4}
NORMS = {"entropic": 0, "l1": 1}
FALLBACKS = {"positivity": 0, "ehrenfest": 1}


class _Cfg(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("collision", C.c_int), ("equilibrium", C.c_int), ("bc", C.c_int),
        ("beta", C.c_double), ("lid_u", C.c_double), ("topk", C.c_int),
        ("delta", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double),
        ("s_q", C.c_double), ("elbm_eps", C.c_double), ("elbm_max_iter", C.c_int),
        ("elbm_norm", C.c_int), ("elbm_fallback", C.c_int),
        ("lim_alpha", C.c_double), ("lim_k", C.c_double), ("lim_dst", C.c_double),
        ("lim_delta0", C.c_double),
    ]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in (
        "limited_sites", "candidates", "elbm_solved", "elbm_skipped",
        "elbm_fallbacks", "elbm_iters_total", "elbm_iters_max", "elbm_corrected")]


@dataclasses.dataclass
class OracleConfig:
    """Parameters of one lattice; field names follow the paper's symbols."""
    lattice: str = "D2Q9"
    nx: int = 16
    ny: int = 16
    collision: str = "lbgk"
    equilibrium: str = "poly"
    bc: str = "cavity"
    beta: float = 0.9
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
    def from_dict(cls, d: dict) -> "OracleConfig":
        """Accepts either beta or a kinematic viscosity nu.  Reading of the
        beta-nu relation of Section 2: nu = c_s^2 (1/beta - 1) / 2 with
        c_s^2 = 1/3, i.e. beta = 1 / (6 nu + 1)."""
        names = {f.name for f in dataclasses.fields(cls)}
        kw = {k: v for k, v in d.items() if k in names}
        if "beta" not in d and d.get("nu") is not None:
            kw["beta"] = 1.0 / (6.0 * float(d["nu"]) + 1.0)
        return cls(**kw)

    @property
    def Q(self) -> int:
        return 3 if self.lattice == "D1Q3" else 9

    def _c(self) -> _Cfg:
        return _Cfg(LATTICES[self.lattice], int(self.nx), int(self.ny),
                    COLLISIONS[self.collision], EQUILIBRIA[self.equilibrium], BCS[self.bc],
                    float(self.beta), float(self.lid_u), int(self.topk), float(self.delta),
                    float(self.s_e), float(self.s_eps), float(self.s_q),
                    float(self.elbm_eps), int(self.elbm_max_iter),
                    NORMS[self.elbm_norm], FALLBACKS[self.elbm_fallback],
                    float(self.lim_alpha), float(self.lim_k), float(self.lim_dst),
                    float(self.lim_delta0))


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` with the host C compiler (portable C99)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, p = C.c_double, C.c_int, C.c_void_p
            sig = {
                "orc_q": (i, [i]),
                "orc_lattice": (None, [i, p, p, p]),
                "orc_opposite": (i, [i, i]),
                "orc_eq1d_poly": (None, [d, p]),
                "orc_eq1d_entropic": (None, [d, p]),
                "orc_equilibrium": (None, [i, i, d, d, d, p]),
                "orc_moments": (None, [i, p, p, p, p]),
                "orc_gfun": (d, [d]),
                "orc_delta_s": (d, [i, p, p]),
                "orc_delta_s_direct": (d, [i, p, p]),
                "orc_entropy": (d, [i, p]),
                "orc_entropy_d1q3_paper": (d, [p]),
                "orc_elbm_alpha": (i, [p, p, p, p, p, p]),
                "orc_elbm_sf": (None, [i, p, p, d, p, p, p]),
                "orc_mrt_basis": (None, [i, p]),
                "orc_mrt_matrix": (None, [p, p]),
                "orc_mrt2_basis": (None, [p]),
                "orc_mrt2_matrix": (None, [p, p]),
                "orc_collide_site": (None, [p, p, p, p]),
                "orc_select_topk": (C.c_longlong, [p, C.c_longlong, i, d, p]),
                "orc_median_field": (None, [i, i, i, i, i, p, p]),
                "orc_phi_smooth": (d, [d, d, d]),
                "orc_phi_double_monotonic": (d, [d, d, d]),
                "orc_phi_ensemble": (d, [d, d, d, d]),
                "orc_threshold_dS0": (d, [p, C.c_longlong, d, d]),
                "orc_init_equilibrium": (None, [p, p, p, p, p]),
                "orc_macros": (None, [p, p, p, p, p]),
                "orc_delta_s_field": (None, [p, p, p]),
                "orc_total_h": (d, [p, p]),
                "orc_enstrophy": (d, [p, p]),
                "orc_step": (i, [p, p, i, p]),
                "orc_stream": (None, [p, p, p]),
                "orc_diffusive_rule": (None, [p, p]),
                "orc_kinetic_energy": (d, [p, p]),
                "orc_adjoint_ke": (i, [p, p, i, p, p, p, p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _cfg(cfg) -> OracleConfig:
    return cfg if isinstance(cfg, OracleConfig) else OracleConfig.from_dict(cfg)


# --------------------------------------------------------------------------- lattice
def lattice(name: str):
    """(cx, cy, W) of the named lattice in the oracle's numbering."""
    Q = 3 if name == "D1Q3" else 9
    cx = np.zeros(Q, np.int32)
    cy = np.zeros(Q, np.int32)
    W = np.zeros(Q)
    _L().orc_lattice(LATTICES[name], _ptr(cx), _ptr(cy), _ptr(W))
    return cx, cy, W


def opposite(name: str, i: int) -> int:
    return _L().orc_opposite(LATTICES[name], i)


def eq1d(u: float, kind: str = "poly") -> np.ndarray:
    out = np.zeros(3)
    (_L().orc_eq1d_entropic if kind == "entropic" else _L().orc_eq1d_poly)(float(u), _ptr(out))
    return out


def equilibrium(name: str, kind: str, rho: float, ux: float, uy: float = 0.0) -> np.ndarray:
    Q = 3 if name == "D1Q3" else 9
    out = np.zeros(Q)
    _L().orc_equilibrium(LATTICES[name], EQUILIBRIA[kind], float(rho), float(ux), float(uy), _ptr(out))
    return out


def moments(name: str, f) -> tuple:
    f = _f64(f)
    r, a, b = C.c_double(), C.c_double(), C.c_double()
    _L().orc_moments(LATTICES[name], _ptr(f), C.byref(r), C.byref(a), C.byref(b))
    return r.value, a.value, b.value


def gfun(x: float) -> float:
    return _L().orc_gfun(float(x))


def delta_s(f, feq) -> float:
    f, feq = _f64(f), _f64(feq)
    return _L().orc_delta_s(len(f), _ptr(f), _ptr(feq))


def delta_s_direct(f, feq) -> float:
    f, feq = _f64(f), _f64(feq)
    return _L().orc_delta_s_direct(len(f), _ptr(f), _ptr(feq))


def entropy(name: str, f) -> float:
    f = _f64(f)
    return _L().orc_entropy(LATTICES[name], _ptr(f))


def entropy_d1q3_paper(f) -> float:
    f = _f64(f)
    return _L().orc_entropy_d1q3_paper(_ptr(f))


def elbm_alpha(cfg, f, feq):
    """Returns (alpha, code, iterations, corrected); code 0 root, 1 skip, 2 fallback."""
    cfg = _cfg(cfg)
    c = cfg._c()
    f, feq = _f64(f), _f64(feq)
    a, it, co = C.c_double(), C.c_int(), C.c_int()
    rc = _L().orc_elbm_alpha(C.byref(c), _ptr(f), _ptr(feq), C.byref(a), C.byref(it), C.byref(co))
    return a.value, rc, it.value, co.value


def elbm_sf(f, feq, alpha: float):
    f, feq = _f64(f), _f64(feq)
    s0, s1, s2 = C.c_double(), C.c_double(), C.c_double()
    _L().orc_elbm_sf(len(f), _ptr(f), _ptr(feq), float(alpha), C.byref(s0), C.byref(s1), C.byref(s2))
    return s0.value, s1.value, s2.value


def mrt_basis(name: str) -> np.ndarray:
    Q = 3 if name == "D1Q3" else 9
    M = np.zeros((Q, Q))
    _L().orc_mrt_basis(LATTICES[name], _ptr(M))
    return M


def mrt_matrix(cfg) -> np.ndarray:
    cfg = _cfg(cfg)
    c = cfg._c()
    A = np.zeros((cfg.Q, cfg.Q))
    _L().orc_mrt_matrix(C.byref(c), _ptr(A))
    return A


def diffusive_rule(cfg, f) -> np.ndarray:
    """Section 8's diffusive Maxwell rule applied to the wall sites of f."""
    cfg = _cfg(cfg)
    c = cfg._c()
    out = _f64(f).copy()
    _L().orc_diffusive_rule(C.byref(c), _ptr(out))
    return out


def enstrophy(cfg, f) -> float:
    """Section 8's enstrophy: mean over sites of the vorticity squared."""
    cfg = _cfg(cfg)
    c = cfg._c()
    return _L().orc_enstrophy(C.byref(c), _ptr(_f64(f)))


def mrt2_basis() -> np.ndarray:
    """M_2 of Section 5 in this oracle's velocity numbering."""
    M = np.zeros((9, 9))
    _L().orc_mrt2_basis(_ptr(M))
    return M


def mrt2_matrix(cfg) -> np.ndarray:
    """A_2 = M_2^-1 C_2 M_2 with s_nu = 2 beta."""
    cfg = _cfg(cfg)
    c = cfg._c()
    A = np.zeros((9, 9))
    _L().orc_mrt2_matrix(C.byref(c), _ptr(A))
    return A


def collide_site(cfg, f) -> np.ndarray:
    cfg = _cfg(cfg)
    c = cfg._c()
    f = _f64(f)
    F = np.zeros_like(f)
    st = _Stats()
    _L().orc_collide_site(C.byref(c), _ptr(f), _ptr(F), C.byref(st))
    return F


def select_topk(dS, k: int, delta: float):
    dS = _f64(dS).ravel()
    mask = np.zeros(dS.size, np.uint8)
    nc = _L().orc_select_topk(_ptr(dS), dS.size, int(k), float(delta), _ptr(mask))
    return mask.astype(bool), int(nc)


def phi_smooth(dS: float, alpha: float, k: float) -> float:
    """Eq. smoothReg's example limiter function 1 / (1 + alpha Delta S^k)."""
    return _L().orc_phi_smooth(float(dS), float(alpha), float(k))


def phi_double_monotonic(dS: float, dst: float, k: float) -> float:
    """Eq. DoublMonSpec: (1 + (Delta S / Delta S_t)^k)^(-1/(2k))."""
    return _L().orc_phi_double_monotonic(float(dS), float(dst), float(k))


def phi_ensemble(dS: float, alpha: float, k: float, E: float) -> float:
    """Eq. phiExamp with the lattice mean E of Delta S."""
    return _L().orc_phi_ensemble(float(dS), float(alpha), float(k), float(E))


def threshold_dS0(dS, delta0: float, beta: float) -> float:
    """Delta S_0 of Eq. EntThresh for the empirical distribution of dS."""
    dS = _f64(dS).ravel()
    return _L().orc_threshold_dS0(_ptr(dS), dS.size, float(delta0), float(beta))


def median_field(name: str, dS, periodic_x=False, periodic_y=False) -> np.ndarray:
    dS = _f64(dS)
    ny, nx = (1, dS.size) if dS.ndim == 1 else dS.shape
    med = np.zeros_like(dS)
    _L().orc_median_field(LATTICES[name], nx, ny, int(periodic_x), int(periodic_y), _ptr(dS), _ptr(med))
    return med


# --------------------------------------------------------------------------- fields
def _shape(cfg: OracleConfig):
    return (cfg.Q, cfg.ny, cfg.nx)


def init_equilibrium(cfg, rho, ux, uy=None) -> np.ndarray:
    cfg = _cfg(cfg)
    c = cfg._c()
    rho, ux = _f64(rho), _f64(ux)
    uyp = None
    if uy is not None:
        uy = _f64(uy)
        uyp = _ptr(uy)
    f = np.zeros(_shape(cfg))
    _L().orc_init_equilibrium(C.byref(c), _ptr(rho), _ptr(ux), uyp, _ptr(f))
    return f


def macros(cfg, f):
    cfg = _cfg(cfg)
    c = cfg._c()
    f = _f64(f)
    rho = np.zeros((cfg.ny, cfg.nx))
    ux = np.zeros_like(rho)
    uy = np.zeros_like(rho)
    _L().orc_macros(C.byref(c), _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def delta_s_field(cfg, f) -> np.ndarray:
    cfg = _cfg(cfg)
    c = cfg._c()
    f = _f64(f)
    dS = np.zeros((cfg.ny, cfg.nx))
    _L().orc_delta_s_field(C.byref(c), _ptr(f), _ptr(dS))
    return dS


def total_h(cfg, f) -> float:
    cfg = _cfg(cfg)
    c = cfg._c()
    f = _f64(f)
    return _L().orc_total_h(C.byref(c), _ptr(f))


def stream(cfg, F) -> np.ndarray:
    cfg = _cfg(cfg)
    c = cfg._c()
    F = _f64(F)
    out = np.zeros_like(F)
    _L().orc_stream(C.byref(c), _ptr(F), _ptr(out))
    return out


def step(cfg, f, nsteps: int = 1, stats: bool = False):
    """Advance ``nsteps`` collide-then-stream steps; returns a new array."""
    cfg = _cfg(cfg)
    c = cfg._c()
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    assert out.shape == _shape(cfg), (out.shape, _shape(cfg))
    st = _Stats()
    rc = _L().orc_step(C.byref(c), _ptr(out), int(nsteps), C.byref(st))
    if rc != 0:
        raise ValueError(f"oracle step failed with code {rc}")
    if stats:
        return out, {n: getattr(st, n) for n, _ in _Stats._fields_}
    return out


def kinetic_energy(cfg, f) -> float:
    cfg = _cfg(cfg)
    c = cfg._c()
    f = _f64(f)
    return _L().orc_kinetic_energy(C.byref(c), _ptr(f))


def adjoint_ke(cfg, f0, T: int):
    """(J, dJ/df0, dJ/dU, dJ/dbeta) of J = 1/2 sum rho |u|^2 after T steps."""
    cfg = _cfg(cfg)
    c = cfg._c()
    f0 = _f64(f0)
    g = np.zeros_like(f0)
    J, gU, gB = C.c_double(), C.c_double(), C.c_double()
    rc = _L().orc_adjoint_ke(C.byref(c), _ptr(f0), int(T), C.byref(J), _ptr(g), C.byref(gU),
                             C.byref(gB))
    if rc != 0:
        raise ValueError(f"oracle adjoint failed with code {rc}")
    return J.value, g, gU.value, gB.value


__all__ = ["kinetic_energy", "adjoint_ke", 
    "OracleConfig", "build", "lattice", "opposite", "eq1d", "equilibrium", "moments", "gfun",
    "delta_s", "delta_s_direct", "entropy", "entropy_d1q3_paper", "elbm_alpha", "elbm_sf",
    "mrt_basis", "mrt_matrix", "collide_site", "select_topk", "median_field",
    "phi_smooth", "phi_double_monotonic", "phi_ensemble", "threshold_dS0", "mrt2_basis", "mrt2_matrix", "enstrophy", "diffusive_rule",
    "init_equilibrium", "macros", "delta_s_field", "total_h", "stream", "step",
]
