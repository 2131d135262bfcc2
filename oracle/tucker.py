"""Sub-R-HOSVD (Alg. 1) in plain float64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (the paper leaves the linear index L of Sec. 2.2 free; its
footnote allows natural or reverse lexicographic order):

* tensors are NumPy arrays in C order (last mode fastest);
* modes are numbered 0..d-1 here (the paper numbers them 1..d);
* the mode-k unfolding X^(k) (Sec. 2.2, Def. 2.1) has rows i_k and columns the
  natural (C-order) linear index of the remaining modes; the set unfolding
  X^(S) of a contiguous mode range S = {a..b} has rows the C-order index over
  S and columns the C-order index over the complement.
"""

import numpy as np

from . import rng


# ----------------------------------------------------------------- Sec. 2.2
def unfold(X, k):
    """Mode-k matricization X^(k), n_k x n_{!=k} (Sec. 2.2, Def. 2.1)."""
    return np.moveaxis(X, k, 0).reshape(X.shape[k], -1)


def set_unfold(X, a, b):
    """Set matricization X^(S), S = {a..b} contiguous, n_S x n_{notin S} (Sec. 2.2)."""
    S = list(range(a, b + 1))
    nS = int(np.prod([X.shape[j] for j in S]))
    return np.moveaxis(X, S, list(range(len(S)))).reshape(nS, -1)


def complement_shape(shape, a, b):
    """Mode sizes of the complement of {a..b}, in natural order."""
    return tuple(shape[:a]) + tuple(shape[b + 1:])


def ttm(A, U, k):
    """TTM A x_k U for U of size m x n_k (Sec. 2.2, Def. 2.2):
    B(i_1..j..i_d) = sum_{i_k} A(i) U(j, i_k)."""
    B = np.tensordot(U, A, axes=([1], [k]))  # new mode first
    return np.moveaxis(B, 0, k)


def multi_ttm_t(X, U):
    """Core S = (U_1^T, ..., U_d^T) X = X x_1 U_1^T ... x_d U_d^T (Alg. 1, core step).

    Each step contracts the current leading mode with U_k and appends the
    rank index at the end, so after d steps the axes are (r_1, ..., r_d).
    """
    G = X
    for Uk in U:
        G = np.tensordot(G, Uk, axes=([0], [0]))
    return G


def reconstruct(G, U):
    """Tucker tensor (U_1, ..., U_d) G = G x_1 U_1 ... x_d U_d (Sec. 3, Tucker format)."""
    Xh = G
    for Uk in U:
        Xh = np.tensordot(Xh, Uk, axes=([0], [1]))
    return Xh


def relerr(X, Xh):
    """Relative reconstruction error ||X - Xh||_F / ||X||_F, formed explicitly."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm((X - Xh).ravel()) / np.linalg.norm(X.ravel()))


# ----------------------------------------------------------------- Sec. 3.1
def gather_fibers(X, a, b, pi):
    """Y = X^(S) E for S = {a..b}: the columns pi of the set unfolding (Sec. 3.1).

    The columns are read from X by index transformation (decode each linear
    index pi(j) into the complement multi-index, natural order), without
    forming the unfolding.  For a single mode a = b = k this is Y_k = X^(k) E_k.
    """
    shape = X.shape
    cshape = complement_shape(shape, a, b)
    S = list(range(a, b + 1))
    nS = int(np.prod([shape[j] for j in S]))
    pi = np.asarray(pi, dtype=np.int64)
    if len(cshape) == 0:  # S is every mode: the single column is vec(X)
        return X.reshape(nS, 1)[:, np.zeros(len(pi), dtype=np.int64)]
    idx = np.unravel_index(pi, cshape)
    Xs = np.moveaxis(X, S, list(range(len(S))))  # view, rows-modes first
    Y = Xs[(slice(None),) * len(S) + tuple(idx)]
    return np.asarray(Y, dtype=np.float64).reshape(nS, len(pi))


def sign_rule(U):
    """Column signs fixed so each column's largest-magnitude entry is positive
    (ties: lowest row index).  U_k is otherwise unique only up to column sign."""
    U = np.array(U, dtype=np.float64, copy=True)
    if U.size == 0:
        return U
    i = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[i, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s


def round_bf16(a):
    """Round to bfloat16 (8 significant bits, round to nearest, ties to even) by way of
    float32, returned as float64: the rounding of the BF16 sketch form."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    b = x.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def range_finder(Y, pi, r, p, seed, node, sketch_bf16=False):
    """The range finder of the loop body of Alg. 1 (and of the per-node body of
    Alg. 2) on a sampled matrix Y (n x s):
      Omega  = Gaussian s x (r+p) test matrix (keyed by the sampled indices pi),
      Q      = orthonormal basis of Range(Y Omega): Householder thin QR with
               diag(R) > 0,
      W      = dominant r left singular vectors of Q^T Y,
      U      = Q W  (then the column-sign rule).
    ``sketch_bf16``: the BF16 sketch form, Z from Y and Omega rounded to bfloat16
    (the W-step keeps Y as given).
    """
    Omega = rng.sketch_matrix(pi, r + p, seed, node)
    Z = (round_bf16(Y) @ round_bf16(Omega)) if sketch_bf16 else Y @ Omega
    Q, R = np.linalg.qr(Z)  # LAPACK Householder (geqrf/orgqr)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    Q = Q * d
    R = d[:, None] * R
    B = Q.T @ Y
    Wf, sig, _ = np.linalg.svd(B, full_matrices=False)
    W = Wf[:, :r]
    U = sign_rule(Q @ W)
    return dict(Omega=Omega, Z=Z, Q=Q, R=R, B=B, sigma=sig, W=W, U=U)


def default_samples(shape):
    """s_k = min(10 n_k, n_{!=k}): the paper's rule of thumb s_k >= 10 n_k (Sec. 3.2)."""
    N = int(np.prod(shape))
    return [min(10 * nk, N // nk) for nk in shape]


def sub_r_hosvd(X, r, p, s=None, seed=0, with_core=True, nodes=None, sketch_bf16=False):
    """[S, {U_k}] = Sub-R-HOSVD(X, r, p, s) (Alg. 1).

    For every mode k (independently: the loop is mode-parallel):
      pick s_k mode-k fibers uniformly without repetition -> Y_k (n_k x s_k),
      draw Omega_k, Q_k = orth(Y_k Omega_k), W_k = top-r_k left singular vectors
      of Q_k^T Y_k, U_k = Q_k W_k.
    Then S = (U_1^T, ..., U_d^T) X.

    ``nodes[k]`` is the stream id of mode k (default k; the H-Tucker leaves use
    their dimension-tree node id).  Returns a dict with G (the core S), U and
    the per-mode intermediates.
    """
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    r = [int(v) for v in (r if np.ndim(r) else [r] * d)]
    s = default_samples(X.shape) if s is None else [int(v) for v in (s if np.ndim(s) else [s] * d)]
    nodes = list(range(d)) if nodes is None else list(nodes)
    modes = []
    for k in range(d):
        nk = X.shape[k]
        N = X.size // nk
        check_sizes(nk, N, r[k], p, s[k])
        pi = rng.fiber_indices(N, s[k], seed, nodes[k])
        Y = gather_fibers(X, k, k, pi)
        out = range_finder(Y, pi, r[k], p, seed, nodes[k], sketch_bf16=sketch_bf16)
        out.update(pi=pi, Y=Y)
        modes.append(out)
    U = [m["U"] for m in modes]
    G = multi_ttm_t(X, U) if with_core else None
    return dict(G=G, U=U, modes=modes, r=r, s=s, p=p)


def check_sizes(n, N, r, p, s):
    """Argument rules of Alg. 1 and the Sub-R-HOSVD error-bound theorem (Sec. 3.2):
    r+p <= min(n, N) and r+p <= s <= N."""
    if r < 1 or p < 0:
        raise ValueError("need r >= 1 and p >= 0")
    if r + p > n or r + p > N:
        raise ValueError("need r + p <= min(n_k, n_{!=k})")
    if s < r + p or s > N:
        raise ValueError("need r + p <= s <= n_{!=k}")
