"""GB300 (sm_103a) chi0 library: pair matrix elements + Hermitian polarizability contraction.

The compute path is the CUDA library ``libgwchi0.so`` (C ABI in include/gw_chi0.h);
this package only marshals arguments to it.
"""
from .chi0 import Chi0, Chi0Fn, GwError, contract_noalloc, create, from_problem  # noqa: F401
from . import _lib  # noqa: F401
