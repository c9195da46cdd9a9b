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
