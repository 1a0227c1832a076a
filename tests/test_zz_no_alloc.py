"""gw_chi0_contract_noalloc: the contraction without any device allocation inside the call.

Some callers cannot allocate device memory: a plugin whose host framework owns every
allocation through its own pool, or a service whose hot path forbids allocator calls
(cudaMalloc and cudaFree can synchronise the device and take unbounded time).  They use
this entry point, whose scratch is a fixed array inside the library.  Its chi must match
the oracle's, and the regular entry point's, on two calls in a row that share that
scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gwgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11  # the FP64 path's bar against the oracle


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def test_noalloc_matches_oracle_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2509_23018_gb300 as gw
    cases = [(gwgen.make_problem((24, 24, 24), 16, 64, 600, 200, seed=gwgen.BASE_SEED), [0.0, 3.5]),
             (gwgen.make_problem((16, 15, 18), 5, 41, 150, 77, seed=17), [1.25])]
    h = gw.Chi0((8, 8, 8))
    for p, om in cases:  # two calls in a row on the shared scratch
        M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
        ev, ec, Md = dev(p.ev), dev(p.ec), dev(M)
        regular = h.contract(ev, ec, Md, om).cpu().numpy()
        out = torch.full((len(om), M.shape[1], M.shape[1]), float("nan"), dtype=torch.complex128, device="cuda")
        got = gw.contract_noalloc(ev, ec, Md, om, out).cpu().numpy()
        torch.cuda.synchronize()
        for i, w in enumerate(om):
            ref = oracle.chi0(M, oracle.delta(p.ev, p.ec, w))
            assert rel(got[i], ref) < TOL
            assert rel(got[i], regular[i]) < TOL
            assert np.array_equal(got[i], got[i].conj().T)
    h.sync()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2509_23018_gb300 import _lib
    lib = _lib.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    om = (ctypes.c_double * 1)(0.0)
    # 1024 x 1024 pairs = 1048576 > 524288
    st = lib.gw_chi0_contract_noalloc(1024, 1024, p, p, 4, p, 1, om, p, None)
    assert st == _lib.GW_ERR_ARG


def test_noalloc_binding_rejects_mismatched_tensors():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2509_23018_gb300 as gw
    ev = torch.full((2,), -5.0, dtype=torch.float64, device="cuda")
    ec = torch.full((3,), 5.0, dtype=torch.float64, device="cuda")
    M = torch.zeros((6, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):  # out too small: the kernels would write past it
        gw.contract_noalloc(ev, ec, M, [0.0], torch.zeros((1, 4, 3), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):  # M has fewer rows than nv * nc
        gw.contract_noalloc(ev, ec, M[:5], [0.0], torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):  # a host tensor
        gw.contract_noalloc(ev, ec, M.cpu(), [0.0], torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda"))
