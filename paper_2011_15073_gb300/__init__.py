"""GB300-native (sm_103a) fused MRT lattice Boltzmann step for natural
convection of a power-law fluid in a porous cavity.

The product is the C-ABI library ``libmrtlbm.so`` (declared in
``include/lbm.h``); :mod:`.lbm` is its thin ctypes binding and :mod:`.inputs`
the seeded synthetic workloads.  Nothing here computes on the CPU.
"""
from . import inputs  # noqa: F401
from .lbm import (BF16D, F16D, F32, F32D, F64, Cavity, LBMError, default_opts, destroy,  # noqa: F401
                  fields, get_lattice, get_state, get_state_f64, init, lib, nusselt, residual,
                  run_to_steady, set_state, set_state_f64, state_bytes, step, strerror, synchronize)
