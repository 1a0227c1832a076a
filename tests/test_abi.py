"""The C-ABI library builds, loads without a GPU and exports every symbol the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gw_chi0.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"GW_API[^;(]*?\b(gw_chi0_\w+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = declared()
    for n in ("gw_chi0_create", "gw_chi0_destroy", "gw_chi0_set_bands", "gw_chi0_set_gsphere",
              "gw_chi0_compute", "gw_chi0_contract", "gw_chi0_pair_elements", "gw_chi0_adjoint"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2509_23018_gb300 import _lib
    lib = _lib.load()
    for n in declared():
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_binding_covers_only_declared_symbols():
    from paper_2509_23018_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared())


def test_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_23018_gb300 import _lib
    lib = _lib.load()
    d = _lib.Desc()
    d.n[0] = d.n[1] = d.n[2] = 24
    d.nq = 1
    h = ctypes.c_void_p()
    st = lib.gw_chi0_create(ctypes.byref(h), ctypes.byref(d), None)
    assert st != 0 and not h.value


def test_create_rejects_bad_descriptors():
    from paper_2509_23018_gb300 import _lib
    lib = _lib.load()
    for grid, nq, prec, ns in [((24, 24, 7), 1, 0, 0), ((24, 24, 24), 0, 0, 0), ((24, 24, 24), 1, 9, 0),
                               ((24, 24, 24), 1, 2, 7),  # no third (integer-sliced) precision
                               ((24, 24, 24), 1, 1, 2), ((256, 24, 24), 1, 0, 0)]:
        d = _lib.Desc()
        for a in range(3):
            d.n[a] = grid[a]
        d.nq, d.prec, d.nslices = nq, prec, ns
        h = ctypes.c_void_p()
        assert lib.gw_chi0_create(ctypes.byref(h), ctypes.byref(d), None) == _lib.GW_ERR_ARG
        assert not h.value


def test_noalloc_binding_rejects_host_tensors():
    """The binding refuses tensors that are not on the current CUDA device before any call."""
    torch = pytest.importorskip("torch")
    import paper_2509_23018_gb300 as gw
    ev = torch.full((2,), -5.0, dtype=torch.float64)
    ec = torch.full((3,), 5.0, dtype=torch.float64)
    M = torch.zeros((6, 4), dtype=torch.complex128)
    with pytest.raises(ValueError):
        gw.contract_noalloc(ev, ec, M, [0.0], torch.zeros((1, 4, 4), dtype=torch.complex128))
