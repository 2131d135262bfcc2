"""Pins of the Kronecker-sketch oracle (oracle/rhkron.py, the rHKron comparison
method of Sec. 3.3): the sketch against the explicit Kronecker test matrix, the
Gaussians' keying, the complete-sketch case that reduces to T-HOSVD, exact
recovery of exact multilinear rank, the best-approximation lower bound, and the
identity between the reduced-core and the projected core."""

import numpy as np
import pytest

import synth
from oracle import brute, rhkron, rng, tucker


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_sketch_is_unfolding_times_kronecker_matrix():
    X = _rand((3, 4, 5, 2), 1)
    ell = [2, 3, 2, 2]
    Om = [rhkron.kron_omega(n, l, 7, j) for j, (n, l) in enumerate(zip(X.shape, ell))]
    for k in range(4):
        others = [Om[j] for j in range(4) if j != k]
        K = others[0]
        for M in others[1:]:
            K = np.kron(K, M)
        ref = tucker.unfold(X, k) @ K
        assert np.allclose(rhkron.kron_sketch(X, Om, k), ref, rtol=1e-13, atol=1e-13)


def test_gaussians_are_keyed_by_mode_row_and_column():
    A = rhkron.kron_omega(300, 5, 11, 2)
    assert A.shape == (300, 5)
    assert np.array_equal(A[17, 3], rng.gaussian(17, 3, 11, 2, stream=rng.STREAM_KRON))
    assert not np.allclose(A, rhkron.kron_omega(300, 5, 11, 1))        # another mode
    assert not np.allclose(A, rng.gaussian(np.arange(300)[:, None], np.arange(5)[None, :], 11, 2))  # stream 2
    big = rhkron.kron_omega(20000, 10, 3, 0).ravel()
    assert abs(big.mean()) < 0.02 and abs(big.var() - 1.0) < 0.02


@pytest.mark.parametrize("shape,ell,r", [((4, 4, 4), (2, 2, 2), (2, 3, 2)),
                                         ((4, 4, 4, 8), (2, 2, 2, 1), (3, 2, 2, 4))])
def test_complete_sketch_reduces_to_t_hosvd(shape, ell, r):
    # prod_{j != k} l_j = n_k for every k: Q_k spans R^{n_k}, C is X in rotated
    # coordinates, and its T-HOSVD is the T-HOSVD of X
    X = _rand(shape, 2)
    got = rhkron.rhkron(X, r, ell, seed=5)
    ref = brute.t_hosvd(X, r)
    for k in range(len(shape)):
        assert np.abs(got["U"][k] - ref["U"][k]).max() < 1e-10
    assert np.abs(got["G"] - ref["G"]).max() < 1e-10


def test_exact_multilinear_rank_is_recovered():
    X = synth.tucker_tensor((10, 12, 9), (3, 3, 3), noise=0.0, data_seed=4, dtype="f64")
    got = rhkron.rhkron(X, (3, 3, 3), (2, 2, 2), seed=1)
    err = tucker.relerr(X, tucker.reconstruct(got["G"], got["U"]))
    assert err < 1e-12
    for U in got["U"]:
        assert np.abs(U.T @ U - np.eye(3)).max() < 1e-13


def test_error_respects_the_best_approximation_bound():
    # no multilinear-rank-r Tucker approximation beats the tail of any unfolding
    X = synth.tucker_tensor((14, 12, 10), (4, 4, 4), noise=1e-2, data_seed=8, dtype="f64")
    r = (4, 4, 4)
    got = rhkron.rhkron(X, r, (3, 3, 3), seed=2)
    err = tucker.relerr(X, tucker.reconstruct(got["G"], got["U"]))
    nx = np.linalg.norm(X)
    tails = [np.sqrt((brute.unfolding_singular_values(X, k)[r[k]:] ** 2).sum()) / nx for k in range(3)]
    assert err >= max(tails) * (1 - 1e-12)


def test_reduced_core_identity():
    # G = X x_k U_k^T equals the reduced core C x_k W_k^T up to the sign rule's flips
    X = _rand((9, 10, 11), 3)
    got = rhkron.rhkron(X, (2, 3, 2), (3, 3, 3), seed=4)
    GC = got["C"]
    for k in range(3):
        Wk = got["W"][k]
        s = np.sign(np.sum((got["Q"][k] @ Wk) * got["U"][k], axis=0))
        GC = tucker.ttm(GC, (Wk * s).T, k)
    assert np.abs(GC - got["G"]).max() < 1e-12


def test_size_rules():
    X = _rand((4, 5, 6), 0)
    with pytest.raises(ValueError):
        rhkron.rhkron(X, (2, 2, 2), (3, 3, 3))   # prod of the others' l (9) > n_0 = 4
    with pytest.raises(ValueError):
        rhkron.rhkron(X, (5, 2, 2), (2, 2, 2))   # r_0 = 5 > L_0 = 4
