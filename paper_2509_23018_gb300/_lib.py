"""ctypes loader for libgwchi0.so (the C ABI of include/gw_chi0.h).

Marshalling only: every step of the chi0 path runs in the CUDA library.  There is
no CPU fallback; if the library is missing or cannot load, this raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

GW_OK, GW_ERR_ARG, GW_ERR_STATE, GW_ERR_OOM, GW_ERR_CUDA, GW_ERR_UNSUPPORTED, GW_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "GW_OK", 1: "GW_ERR_ARG", 2: "GW_ERR_STATE", 3: "GW_ERR_OOM", 4: "GW_ERR_CUDA",
                5: "GW_ERR_UNSUPPORTED", 6: "GW_ERR_TIMEOUT"}
GW_PREC_FP64, GW_PREC_OZAKI_BF16 = 0, 1
GW_MTXEL_FP64, GW_MTXEL_TWOFLOAT = 0, 1
# gw_probe_kind
PROBES = {"ffma": 0, "ffma2": 1, "fadd2": 2, "dfma": 3, "dmma_m8n8k4": 4, "dmma_m16n8k16": 5,
          "bf16_mma_sync": 6, "int8_mma_sync": 7, "tcgen05_n64": 8, "tcgen05_n128": 9, "tcgen05_n256": 10}

# Every entry point declared in include/gw_chi0.h, with its ctypes signature.
P, I, I64, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nq", I), ("prec", I), ("nslices", I), ("pair_chunk", I64),
                ("mem_budget_bytes", SZ), ("device", I), ("mtxel_prec", I), ("single_stream", I)]


SIGNATURES = {
    "gw_chi0_create": ([ctypes.POINTER(P), ctypes.POINTER(Desc), P], I),
    "gw_chi0_destroy": ([P], None),
    "gw_chi0_last_error": ([P], ctypes.c_char_p),
    "gw_chi0_set_stream": ([P, P], I),
    "gw_chi0_set_bands": ([P, I, I, I, I, P, P, P], I),
    "gw_chi0_set_gsphere": ([P, I, I, P], I),
    "gw_chi0_compute": ([P, I, P, I, P, P, P], I),
    "gw_chi0_compute_batch": ([P, I, P, I, P, P, P], I),
    "gw_chi0_tuning": ([P, P, P, P], I),
    "gw_chi0_pair_elements": ([P, I, I64, I64, P], I),
    "gw_chi0_pair_elements_block": ([P, I, I, I, P], I),
    "gw_chi0_contract": ([P, I, I, P, P, I, P, I, P, P], I),
    "gw_chi0_adjoint": ([P, I, D, P, P, P, P, P, P], I),
    "gw_chi0_subspace_basis": ([P, I, P, I, P, P], I),
    "gw_chi0_compute_subspace": ([P, I, I, P, I, P, P], I),
    "gw_chi0_epsilon_inverse": ([P, I, I, P, P, P], I),
    "gw_chi0_sigma_gpp": ([P, I, I, I, I, P, P, P, P, P, I, P, P], I),
    "gw_chi0_compute_real": ([P, I, I, P, D, P], I),
    "gw_chi0_jvp": ([P, I, I, P, P, P, P, P, P], I),
    "gw_chi0_streams": ([P, I], I),
    "gw_chi0_keep_pair_elements": ([P, I], I),
    "gw_chi0_sync": ([P], I),
    "gw_chi0_check_watchdog": ([P, ctypes.c_longlong], I),
    "gw_chi0_set_timing": ([P, I], I),
    "gw_chi0_timing": ([P, I, P, P, P, I], I),
    "gw_chi0_device_bytes": ([P], SZ),
    "gw_chi0_contract_noalloc": ([I, I, P, P, I, P, I, P, P, P], I),
    "gw_chi0_probe": ([I, ctypes.c_longlong, P, P, ctypes.POINTER(D)], I),
}


def library_path() -> str:
    return _build.LIB_DEBUG if os.environ.get("GW_CHI0_DEBUG") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Load libgwchi0.so (the bounds-checked build with GW_CHI0_DEBUG=1); build it first if it is
    missing or stale and nvcc exists."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if os.environ.get("GW_CHI0_DEBUG") == "1":
            if build_if_missing and not os.path.exists(path):
                _build.build(debug=True)
        elif build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib
