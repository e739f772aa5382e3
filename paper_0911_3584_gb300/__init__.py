"""GB300-native range-truncated block-sparse products for the LNV method.

Bowler & Miyazaki (CONQUEST), Sec. 2: K = 3LSL - 2LSLSL (Eq. 3), N_e = 2 Tr[KS],
band energy E = 2 Tr[KH], their gradients with respect to the range-truncated
auxiliary density matrix L, and the minimisation of E over L.  The computation
runs in liblnv (CUDA, sm_103a) behind the C ABI of include/lnv.h; this package
is its Python binding.
"""
from .lnv import (  # noqa: F401
    FP32,
    FP64,
    Context,
    LnvError,
    Pattern,
    Plan,
    System,
    launch_count,
    lib,
    trace_product,
    vec_axpby,
    vec_dot,
    version,
)
from .autograd import LNVEnergy, lnv_energy  # noqa: F401
