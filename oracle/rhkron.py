"""Randomized HOSVD with Kronecker-structured Gaussian test matrices, in plain
float64 NumPy: the rHKron comparison method of Sec. 3.3 (Minster et al.).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Steps, in the order the paper describes the method:

1. one small Gaussian Omega_j (n_j x l_j) per mode, drawn from the counter-based
   stream 3 of ``oracle/rng.py`` (entry (i, a) keyed by row i and column a, node j);
2. for each mode k the tensor is sketched along every other mode,
   S_k = X x_{j != k} Omega_j^T, and unfolded along k:
   Z_k = X^(k) (Omega_0 (x) ... (x) Omega_{k-1} (x) Omega_{k+1} (x) ... (x) Omega_{d-1}),
   n_k x L_k with L_k = prod_{j != k} l_j (the columns in natural order of the
   other modes, as every unfolding here) -- one Kronecker-structured test matrix
   per mode, built from the same d small Gaussians, so a single pass over X
   can form every Z_k;
3. Q_k = orthonormal factor of the thin QR of Z_k (Householder, diag(R) > 0);
4. the reduced tensor C = X x_1 Q_1^T ... x_d Q_d^T (L_1 x ... x L_d);
5. C is factored at multilinear rank r: the paper takes an ST-HOSVD there; this
   oracle, like the CUDA path, factors every mode of C independently (T-HOSVD:
   W_k = dominant r_k left singular vectors of C^(k)), which keeps the d
   factorisations mode-parallel (Sec. 3.3.3);
6. U_k = Q_k W_k with the column-sign rule, G = X x_1 U_1^T ... x_d U_d^T
   (= C x_k W_k^T).
"""

import numpy as np

from . import rng
from .tucker import multi_ttm_t, sign_rule, ttm, unfold


def kron_omega(n, ell, seed, j):
    """Omega_j (n x ell): entry (i, a) = g(seed, node j, m = i, c = a) of stream 3."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    a = np.arange(ell, dtype=np.uint64)[None, :]
    return rng.gaussian(i, a, seed, j, stream=rng.STREAM_KRON)


def kron_sketch(X, Om, k):
    """Z_k = unfolding along k of X x_{j != k} Omega_j^T (n_k x prod_{j != k} l_j)."""
    S = np.asarray(X, dtype=np.float64)
    for j in range(S.ndim):
        if j != k:
            S = ttm(S, Om[j].T, j)
    return unfold(S, k)


def check_sizes(shape, r, ell):
    d = len(shape)
    for k in range(d):
        L = int(np.prod([ell[j] for j in range(d) if j != k]))
        if not (1 <= r[k] <= L <= shape[k]):
            raise ValueError("mode %d: need r_k <= prod_{j != k} l_j <= n_k" % k)


def rhkron(X, r, ell, seed=0):
    """Tucker factors and core of X at multilinear rank r by steps 1-6 above."""
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    r = [int(v) for v in r]
    ell = [int(v) for v in ell]
    check_sizes(X.shape, r, ell)
    Om = [kron_omega(X.shape[j], ell[j], seed, j) for j in range(d)]
    Z, Q = [], []
    for k in range(d):
        Zk = kron_sketch(X, Om, k)
        Qk, Rk = np.linalg.qr(Zk)          # LAPACK Householder
        s = np.sign(np.diag(Rk))
        s[s == 0] = 1.0
        Z.append(Zk)
        Q.append(Qk * s)
    C = multi_ttm_t(X, Q)
    W, sig = [], []
    for k in range(d):
        Wf, sk, _ = np.linalg.svd(unfold(C, k), full_matrices=False)
        W.append(Wf[:, :r[k]])
        sig.append(sk)
    U = [sign_rule(Q[k] @ W[k]) for k in range(d)]
    G = multi_ttm_t(X, U)
    return dict(Omega=Om, Z=Z, Q=Q, C=C, W=W, sigma=sig, U=U, G=G)
