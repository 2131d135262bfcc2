"""Deterministic T-HOSVD and RtL-HT by full SVDs, float64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

These are the comparison algorithms the randomized method reduces to in its
exact special cases; the tests use them only to pin the randomized oracle on
tiny inputs:

* T-HOSVD (Sec. 3): U_k = dominant r_k left singular vectors of X^(k),
  S = (U_1^T, ..., U_d^T) X.  Sub-R-HOSVD with s_k = n_{!=k} (every fiber) and
  r_k + p = n_k (Q_k square orthogonal) returns exactly these factors.
* RtL-HT (Sec. 4): U_S = dominant r_S left singular vectors of X^(S) at every
  non-root node, transfer tensors by the same inner products as Alg. 2.
"""

import numpy as np

from .tucker import unfold, set_unfold, multi_ttm_t, sign_rule
from .htucker import balanced_tree, transfer_tensor, root_transfer


def t_hosvd(X, r):
    X = np.asarray(X, dtype=np.float64)
    U = []
    for k in range(X.ndim):
        Uf, _, _ = np.linalg.svd(unfold(X, k), full_matrices=False)
        U.append(sign_rule(Uf[:, :r[k]]))
    return dict(G=multi_ttm_t(X, U), U=U)


def unfolding_singular_values(X, k):
    return np.linalg.svd(unfold(np.asarray(X, dtype=np.float64), k), compute_uv=False)


def rtl_ht(X, ranks, tree=None):
    X = np.asarray(X, dtype=np.float64)
    nodes = balanced_tree(X.ndim) if tree is None else tree
    US = [None] * len(nodes)
    for nd in nodes:
        if nd.id == 0:
            continue
        Uf, _, _ = np.linalg.svd(set_unfold(X, nd.a, nd.b), full_matrices=False)
        US[nd.id] = sign_rule(Uf[:, :ranks[nd.id]])
    B = [None] * len(nodes)
    for nd in nodes:
        if nd.is_leaf:
            continue
        B[nd.id] = (root_transfer(X, US[nd.left], US[nd.right]) if nd.id == 0
                    else transfer_tensor(US[nd.id], US[nd.left], US[nd.right]))
    leaves = sorted((nd for nd in nodes if nd.is_leaf), key=lambda nd: nd.a)
    return dict(U=[US[nd.id] for nd in leaves], B=B, US=US, tree=nodes)
