"""The bench's error figure (bench.block_error): the relative Frobenius error of the whole
N_G x N_G chi estimated from the oracle's sampled block, its diagonal and off-diagonal entries
weighted by their shares of the whole matrix.  Checked on the CPU against the exact whole-matrix
error where the estimate must be exact (each stratum with one relative error and one magnitude),
and on a matrix shaped like chi (a dominant diagonal), where the block's plain relative error
understates the whole matrix's and the estimate does not."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _full_rel(chi, ref):
    return float(np.linalg.norm(chi - ref) / np.linalg.norm(ref))


def test_stratified_estimate_is_exact_for_uniform_strata():
    b = _bench()
    rng = np.random.default_rng(1)
    ng, n = 300, 12
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, (ng, ng)))
    ref = 0.01 * ph
    np.fill_diagonal(ref, 5.0)
    err = 0.01 * 1e-9 * np.exp(1j * rng.uniform(0, 2 * np.pi, (ng, ng)))  # off-diagonal: rel. 1e-9 each
    np.fill_diagonal(err, 5.0 * 3e-13)                                   # diagonal: rel. 3e-13 each
    chi = ref + err
    idx = np.sort(rng.choice(ng, n, replace=False))
    got = b.block_error(chi, (idx, ref[np.ix_(idx, idx)], ng))
    assert abs(got["rel_frobenius_vs_oracle"] / _full_rel(chi, ref) - 1) < 1e-6
    assert abs(got["offdiag_rel"] / 1e-9 - 1) < 1e-6 and abs(got["diag_rel"] / 3e-13 - 1) < 1e-3


def test_stratified_estimate_tracks_the_whole_matrix():
    b = _bench()
    rng = np.random.default_rng(2)
    ng, n = 400, 24
    X = rng.standard_normal((3000, ng)) + 1j * rng.standard_normal((3000, ng))
    ref = -(X.conj().T @ X) / 3000                                       # Hermitian, dominant diagonal
    err = (rng.standard_normal((ng, ng)) + 1j * rng.standard_normal((ng, ng))) * 1e-12
    err = err + err.conj().T
    chi = ref + err
    full = _full_rel(chi, ref)
    idx = np.sort(rng.choice(ng, n, replace=False))
    got = b.block_error(chi, (idx, ref[np.ix_(idx, idx)], ng))
    assert got["block_rel"] < 0.5 * full                                 # the block alone understates it
    assert 0.6 < got["rel_frobenius_vs_oracle"] / full < 1.6
