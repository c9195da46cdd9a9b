"""Post-processing of recorded signals (host NumPy; no step of the lattice
Boltzmann path runs here).

Section 8's first-Hopf-bifurcation statistic: the energy of Eq. (energy) of
the last part of a control-point velocity signal, and the straight-line fit
of E_u^2 against Re whose zero locates the bifurcation (E_u^2 grows in
proportion to Re - Re_c for a standard Hopf bifurcation).
"""
from __future__ import annotations

import numpy as np


def hopf_energy(u_sig, L: float, u0: float) -> float:
    """E_u = || sqrt(L / (u0 |u_sig|)) (u_sig - mean(u_sig)) ||_2 with |u_sig|
    the number of samples (Eq. energy)."""
    u = np.asarray(u_sig, dtype=np.float64)
    return float(np.sqrt(L / (u0 * u.size)) * np.linalg.norm(u - u.mean()))


def fit_onset(re, e2, floor: float = 0.05) -> dict:
    """Least-squares line E_u^2 = a (Re - Re_c) through the points whose E_u^2
    is at least `floor` times the largest (the oscillating side; below the
    onset E_u^2 is numerical noise).  Returns a, Re_c and the points used."""
    re = np.asarray(re, dtype=np.float64)
    e2 = np.asarray(e2, dtype=np.float64)
    use = e2 >= floor * e2.max()
    if use.sum() < 2:
        return {"slope": None, "re_c": None, "used": use.tolist()}
    a, b = np.polyfit(re[use], e2[use], 1)
    return {"slope": float(a), "re_c": float(-b / a), "used": use.tolist()}


def dominant_frequency(u_sig, L: float, u0: float) -> dict:
    """Dominant frequency of a control-point signal sampled once per step:
    the peak of the one-sided amplitude spectrum of u_sig - mean(u_sig)
    (Section 8 reports omega = 0.525 at Re = 7375).  Returns the peak's
    frequency f in cycles per convective time L / u0, omega = 2 pi f, and
    the share of the signal's power in the peak and its two neighbours
    (near 1 for a clean oscillation, small for broadband noise).  The
    resolution is one cycle per signal length."""
    u = np.asarray(u_sig, dtype=np.float64)
    u = u - u.mean()
    n = u.size
    p = np.abs(np.fft.rfft(u)) ** 2
    p[0] = 0.0
    total = p.sum()
    if n < 4 or total <= 0.0:
        return {"f": None, "omega": None, "peak_share": 0.0}
    k = int(np.argmax(p))
    share = float(p[max(k - 1, 1):k + 2].sum() / total)
    f = k / n * (L / u0)  # cycles per step times steps per convective time
    return {"f": float(f), "omega": float(2.0 * np.pi * f), "peak_share": share}


def _cumulative_simpson(g, h: float, axis: int):
    """Running integral of samples g (spacing h) from index 0 along `axis`:
    composite Simpson at even indices; at odd indices the last interval is
    integrated over the parabola through it and its neighbour (exact for
    quadratic integrands at every index)."""
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, 0)
    n = g.shape[0]
    out = np.zeros_like(g)
    if n < 2:
        return np.moveaxis(out, 0, axis)
    if n == 2:
        out[1] = 0.5 * h * (g[0] + g[1])
        return np.moveaxis(out, 0, axis)
    for j in range(2, n, 2):
        out[j] = out[j - 2] + h / 3.0 * (g[j - 2] + 4.0 * g[j - 1] + g[j])
    for j in range(1, n, 2):
        if j + 1 < n:  # parabola through j-1, j, j+1
            out[j] = out[j - 1] + h / 12.0 * (5.0 * g[j - 1] + 8.0 * g[j] - g[j + 1])
        else:          # parabola through j-2, j-1, j
            out[j] = out[j - 1] + h / 12.0 * (-g[j - 2] + 8.0 * g[j - 1] + 5.0 * g[j])
    return np.moveaxis(out, 0, axis)


def stream_function(ux, uy, h: float = 1.0):
    """Stream function psi of a 2D velocity field [ny][nx] (u_x = dpsi/dy,
    u_y = -dpsi/dx) by Simpson integration first along x on the bottom row,
    then along y up every column (Section 8), with psi = 0 at site (0, 0)."""
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    psi_bottom = -_cumulative_simpson(uy[0], h, 0)           # along x, y = 0
    return psi_bottom[None, :] + _cumulative_simpson(ux, h, 0)  # along y


def vortex_summary(psi) -> dict:
    """The primary vortex (extreme of psi of the larger magnitude) and the
    extreme of the other sign, each with its site (x, y)."""
    psi = np.asarray(psi, dtype=np.float64)
    lo, hi = np.unravel_index(np.argmin(psi), psi.shape), np.unravel_index(np.argmax(psi), psi.shape)
    a = {"psi": float(psi[lo]), "x": int(lo[1]), "y": int(lo[0])}
    b = {"psi": float(psi[hi]), "x": int(hi[1]), "y": int(hi[0])}
    return {"primary": a, "secondary": b} if abs(a["psi"]) >= abs(b["psi"]) else {"primary": b, "secondary": a}
