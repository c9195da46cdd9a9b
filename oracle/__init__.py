"""FP64 CPU oracle for the LBM add-ons (ELBM, entropic limiters, MRT).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; the
product path (``paper_1110_0270_gb300``) never imports it.  The numerics live
in ``lbm_oracle.c`` (plain single-threaded C, double precision); this module
only builds it and marshals numpy arrays through ctypes.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, OracleConfig  # noqa: F401
