"""GB300-native (sm_103a) lattice Boltzmann stream-and-collide with the
add-ons of Brownlee, Levesley, Packwood and Gorban: LBGK, ELBM, Ehrenfest
top-k, positivity rule, median entropy filter and MRT, for D1Q3 and D2Q9.

The compute path is the C-ABI library ``_lib/liblbm.so`` (declared in
``include/lbm.h``); ``lbm.py`` is a thin ctypes binding over it.
"""
