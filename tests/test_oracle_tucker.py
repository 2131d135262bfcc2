"""Pins of the Sub-R-HOSVD oracle (Alg. 1) against what the paper and the
mathematics fix: brute-force definitions on tiny inputs, the exact special
case that reduces to T-HOSVD, exact recovery, orthonormality, the
deterministic error sandwich and the expected-error bound of Sec. 3.2, and the
counts the paper prints (tests/golden)."""

import itertools
import os

import numpy as np
import pytest

import synth
from oracle import brute, rng, tucker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------- paper's numbers
def test_golden_unfolding_column_counts():
    for label, d, n, printed, tol, cite in _rows("paper_counts.txt"):
        d, n, printed, tol = int(d), int(n), float(printed), float(tol)
        X_shape = (n,) * d
        N = int(np.prod(X_shape)) // n  # n_{!=k}
        assert abs(N - printed) <= tol * printed, (label, cite)


def test_golden_sampling_fractions():
    for label, d, n, s, pct, digits, cite in _rows("paper_fractions.txt"):
        d, n, s, pct = int(d), int(n), int(s), float(pct)
        N = n ** (d - 1)
        got = 100.0 * s / N
        # the paper prints one significant digit, rounded up
        unit = 10.0 ** np.floor(np.log10(pct))
        assert pct - unit < got <= pct, (label, got, cite)


# ------------------------------------------------------- Sec. 2.2 definitions
def test_multi_ttm_matches_elementwise_definition():
    rs = np.random.default_rng(1)
    X = rs.standard_normal((3, 4, 5))
    U = [rs.standard_normal((3, 2)), rs.standard_normal((4, 3)), rs.standard_normal((5, 2))]
    G = tucker.multi_ttm_t(X, U)
    ref = np.zeros((2, 3, 2))
    for a, b, c in itertools.product(range(2), range(3), range(2)):
        for i, j, k in itertools.product(range(3), range(4), range(5)):
            ref[a, b, c] += X[i, j, k] * U[0][i, a] * U[1][j, b] * U[2][k, c]
    assert np.allclose(G, ref, rtol=1e-13, atol=1e-13)
    Xh = tucker.reconstruct(ref, U)
    ref2 = np.zeros((3, 4, 5))
    for i, j, k in itertools.product(range(3), range(4), range(5)):
        for a, b, c in itertools.product(range(2), range(3), range(2)):
            ref2[i, j, k] += ref[a, b, c] * U[0][i, a] * U[1][j, b] * U[2][k, c]
    assert np.allclose(Xh, ref2, rtol=1e-13, atol=1e-13)


def test_ttm_unfolding_identity():
    # (A x_k U)^(k) = U A^(k)  (Sec. 2.2)
    rs = np.random.default_rng(2)
    A = rs.standard_normal((3, 4, 5, 2))
    for k in range(4):
        U = rs.standard_normal((6, A.shape[k]))
        assert np.allclose(tucker.unfold(tucker.ttm(A, U, k), k), U @ tucker.unfold(A, k))


def test_unfolding_index_is_natural_order():
    # X^(k)(i_k, j) = X(i), j the C-order linear index of the other modes
    rs = np.random.default_rng(3)
    X = rs.standard_normal((2, 3, 4))
    X1 = tucker.unfold(X, 1)
    for i0, i1, i2 in itertools.product(range(2), range(3), range(4)):
        assert X1[i1, i0 * 4 + i2] == X[i0, i1, i2]
    XS = tucker.set_unfold(X, 1, 2)
    for i0, i1, i2 in itertools.product(range(2), range(3), range(4)):
        assert XS[i1 * 4 + i2, i0] == X[i0, i1, i2]


def test_gather_fibers_equals_columns_of_unfolding():
    rs = np.random.default_rng(4)
    X = rs.standard_normal((3, 5, 2, 4))
    for a in range(4):
        for b in range(a, 4):
            if (a, b) == (0, 3):
                continue
            XS = tucker.set_unfold(X, a, b)
            pi = rng.fiber_indices(XS.shape[1], min(XS.shape[1], 7), 11, a * 4 + b)
            assert np.array_equal(tucker.gather_fibers(X, a, b, pi), XS[:, pi])


# --------------------------------------------------------------- Sec. 3.1
def test_sketch_equals_dense_sampling_times_dense_gaussian():
    # Y_k Omega_k = X^(k) E_k Omega_k with E_k the 0/1 sampling matrix and
    # Omega_k = E_k^T Omega_dense, Omega_dense the n_{!=k} x (r+p) Gaussian
    rs = np.random.default_rng(5)
    X = rs.standard_normal((6, 5, 7))
    r, p, seed = 2, 2, 17
    out = tucker.sub_r_hosvd(X, r, p, s=[9, 8, 10], seed=seed)
    for k in range(3):
        Xk = tucker.unfold(X, k)
        N = Xk.shape[1]
        pi = out["modes"][k]["pi"]
        E = np.zeros((N, len(pi)))
        E[pi, np.arange(len(pi))] = 1.0
        Om_dense = rng.gaussian(np.arange(N, dtype=np.uint64)[:, None],
                                np.arange(r + p, dtype=np.uint64)[None, :], seed, k)
        Z = Xk @ E @ (E.T @ Om_dense)
        assert np.allclose(out["modes"][k]["Z"], Z, rtol=1e-13, atol=1e-13)
        assert np.array_equal(out["modes"][k]["Y"], Xk @ E)


def test_exact_case_reduces_to_truncated_hosvd():
    # s_k = n_{!=k} and r_k + p = n_k: Range(Y_k Omega_k) = R^{n_k}, so
    # U_k = dominant r_k left singular vectors of X^(k) (T-HOSVD, Sec. 3)
    rs = np.random.default_rng(6)
    # one p for all modes: sizes and ranks with n_k - r_k = p for every k
    X = rs.standard_normal((6, 7, 8))
    r = [2, 3, 4]
    p = 4
    s = [56, 48, 42]
    out = tucker.sub_r_hosvd(X, r, p, s=s, seed=3)
    ref = brute.t_hosvd(X, r)
    for k in range(3):
        assert np.abs(out["U"][k] - ref["U"][k]).max() < 1e-10
    assert np.abs(out["G"] - ref["G"]).max() < 1e-10


def _exact_rank_tensor(shape, ranks, seed):
    X, C, A = synth.tucker_tensor(shape, ranks, noise=0.0, data_seed=seed, core="gauss",
                                  dtype="f64", with_parts=True)
    return X, A


def test_exact_recovery_of_low_multilinear_rank():
    X, A = _exact_rank_tensor((20, 18, 22, 16), (3, 4, 2, 3), 7)
    out = tucker.sub_r_hosvd(X, [3, 4, 2, 3], p=4, seed=9)
    Xh = tucker.reconstruct(out["G"], out["U"])
    assert tucker.relerr(X, Xh) < 1e-12
    for k in range(4):
        # principal angles between Range(U_k) and Range(A_k)
        sv = np.linalg.svd(out["U"][k].T @ A[k], compute_uv=False)
        assert np.arccos(np.clip(sv.min(), -1, 1)) < 1e-7
        assert np.abs(1 - sv).max() < 1e-12


def test_orthonormal_factors_and_sign_rule():
    X = synth.tucker_tensor((17, 19, 23), (5, 4, 6), noise=1e-3, data_seed=8, dtype="f64")
    out = tucker.sub_r_hosvd(X, [5, 4, 6], p=3, seed=4)
    for U in out["U"]:
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-13
        i = np.argmax(np.abs(U), axis=0)
        assert np.all(U[i, np.arange(U.shape[1])] > 0)


def test_deterministic_error_sandwich():
    # max_k ||Sigma_2^(k)||_F <= ||X - Xh||_F <= (sum_k ||(I - U_k U_k^T) X^(k)||_F^2)^(1/2)
    # (upper: first step of the proof of the Sub-R-HOSVD bound, Sec. 3.2;
    #  lower: Eckart-Young, rank(Xh^(k)) <= r_k)
    X = synth.tucker_tensor((15, 16, 14, 13), (5, 5, 5, 5), noise=3e-2, data_seed=9, dtype="f64")
    r = [4, 4, 4, 4]
    out = tucker.sub_r_hosvd(X, r, p=4, s=60, seed=2)
    err = np.linalg.norm(X - tucker.reconstruct(out["G"], out["U"]))
    lower = max(np.sqrt((brute.unfolding_singular_values(X, k)[r[k]:] ** 2).sum()) for k in range(4))
    upper = np.sqrt(sum(np.linalg.norm(tucker.unfold(X, k) - out["U"][k] @ (out["U"][k].T @ tucker.unfold(X, k))) ** 2
                        for k in range(4)))
    assert lower <= err * (1 + 1e-12)
    assert err <= upper * (1 + 1e-12)
    assert err > 1.01 * lower  # the tensor is not exactly low rank


@pytest.mark.slow
def test_expected_error_bound_sec32():
    # E_B ||X - Xh||^2 <= sum_k (1 + 3^{3/2} r_k (1+eta_k)(r_k+p) / ((1-delta_k)(p+1))) ||Sigma_2^(k)||^2
    # with delta_k, eta_k taken as the worst values seen over the 25 seeds (so
    # every draw lies in the event B of Sec. 3.2); checked on the mean over the
    # paper's 25 independent runs (Sec. 3.3).
    X = synth.tucker_tensor((12, 13, 11), (4, 4, 4), noise=5e-2, data_seed=10, dtype="f64")
    r, p, s = [3, 3, 3], 4, [40, 40, 40]
    Vs = []
    for k in range(3):
        _, S, Vt = np.linalg.svd(tucker.unfold(X, k), full_matrices=False)
        Vs.append((Vt.T, S))
    errs2, deltas, etas = [], np.zeros(3), np.zeros(3)
    for seed in range(25):
        out = tucker.sub_r_hosvd(X, r, p, s=s, seed=seed)
        errs2.append(np.linalg.norm(X - tucker.reconstruct(out["G"], out["U"])) ** 2)
        for k in range(3):
            V, _ = Vs[k]
            m = tucker.unfold(X, k).shape[1]
            VE = V[out["modes"][k]["pi"], :].T  # V^T E
            sr = np.linalg.svd(VE[:r[k]], compute_uv=False)[-1]
            s1 = np.linalg.svd(VE[r[k]:], compute_uv=False)[0]
            deltas[k] = max(deltas[k], 1 - sr ** 2 * m / s[k])
            etas[k] = max(etas[k], s1 ** 2 * m / s[k] - 1)
    bound = sum((1 + 3 ** 1.5 * r[k] * (1 + etas[k]) * (r[k] + p) / ((1 - deltas[k]) * (p + 1)))
                * (Vs[k][1][r[k]:] ** 2).sum() for k in range(3))
    assert np.mean(errs2) <= bound
    assert np.all(deltas < 1)


def test_argument_rules():
    X = np.zeros((4, 5, 6))
    with pytest.raises(ValueError):
        tucker.sub_r_hosvd(X, 4, p=1)  # r + p > n_1
    with pytest.raises(ValueError):
        tucker.sub_r_hosvd(X, 2, p=1, s=[2, 20, 20])  # s < r + p
    with pytest.raises(ValueError):
        tucker.sub_r_hosvd(X, 2, p=1, s=[31, 20, 20])  # s > n_{!=1} = 30


def test_bfloat16_rounding_matches_torch_and_its_definition():
    # round to nearest even at 8 significant bits: torch's own conversion as the
    # independent reference, exact values unchanged, a tie rounded to even
    torch = pytest.importorskip("torch")
    rs = np.random.default_rng(5)
    a = np.concatenate([rs.standard_normal(20000) * 10.0 ** rs.integers(-6, 6, 20000),
                        [0.0, 1.0, -2.5, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0]])
    want = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()
    got = tucker.round_bf16(a)
    assert np.array_equal(got, want)
    assert tucker.round_bf16([1.0 + 2 ** -8])[0] == 1.0                 # tie -> even
    assert tucker.round_bf16([1.0 + 3 * 2 ** -8])[0] == 1.0 + 2 ** -6   # tie -> even (up)
    assert np.all(np.abs(got - a.astype(np.float32)) <= 2 ** -8 * np.abs(a.astype(np.float32)))


def test_bf16_sketch_form_without_rounding_error_is_the_plain_form():
    # data that bfloat16 represents exactly: the BF16 sketch form changes nothing
    rs = np.random.default_rng(7)
    X = tucker.round_bf16(rs.integers(-64, 64, size=(9, 8, 7)).astype(np.float64) / 8.0).reshape(9, 8, 7)
    a = tucker.sub_r_hosvd(X, [3, 3, 3], 2, seed=4, with_core=False)
    b = tucker.sub_r_hosvd(X, [3, 3, 3], 2, seed=4, with_core=False, sketch_bf16=True)
    for k in range(3):
        Zr = a["modes"][k]["Y"] @ tucker.round_bf16(a["modes"][k]["Omega"])
        assert np.allclose(b["modes"][k]["Z"], Zr, rtol=1e-13, atol=1e-13)
