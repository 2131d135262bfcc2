"""Sub-R-RtL-HT (Alg. 2) in plain float64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Dimension tree (Sec. 4, definition of a dimension tree): binary, root {0..d-1}, singleton leaves,
each internal node the disjoint union of its two children.  The balanced tree
used here splits a node {a..b} into a left child holding the first
ceil(len/2) modes and a right child holding the rest, and numbers the nodes
level by level, left to right (for d = 8 this is the heap numbering of the
paper's dimension-tree figure: 0 = root, 1..2, 3..6, leaves 7..14).

Every node is a contiguous mode range, so its set unfolding X^(S) has rows
in natural order over S with the left child's modes slower, which is the
row order of the Kronecker product U_{S_l} (x) U_{S_r} in the nestedness
relation U_S = (U_{S_l} (x) U_{S_r}) (B_S^(1))^T (Sec. 4).
"""

import numpy as np

from . import rng
from .tucker import gather_fibers, range_finder, complement_shape


class Node:
    __slots__ = ("id", "a", "b", "left", "right", "parent", "level")

    def __init__(self, id, a, b, parent, level):
        self.id, self.a, self.b = id, a, b
        self.left = self.right = None
        self.parent, self.level = parent, level

    @property
    def is_leaf(self):
        return self.a == self.b


def balanced_tree(d):
    """Balanced dimension tree on modes 0..d-1, nodes numbered breadth-first."""
    if d < 2:
        raise ValueError("need d >= 2")
    nodes = [Node(0, 0, d - 1, -1, 0)]
    q = 0
    while q < len(nodes):
        nd = nodes[q]
        q += 1
        if nd.is_leaf:
            continue
        mid = nd.a + (nd.b - nd.a + 1 + 1) // 2  # left child: first ceil(len/2) modes
        for (a, b) in ((nd.a, mid - 1), (mid, nd.b)):
            ch = Node(len(nodes), a, b, nd.id, nd.level + 1)
            nodes.append(ch)
            if nd.left is None:
                nd.left = ch.id
            else:
                nd.right = ch.id
    return nodes


def tree_from_children(children):
    """Dimension tree from a child table: children[i] = (left, right) node ids of
    node i, (-1, -1) for a leaf, node 0 the root.  The leaves are the single modes
    0..d-1 taken left to right, so each node is the contiguous range of the leaves
    below it, its left child's modes first (any binary tree over the modes in
    their natural order, Sec. 4's definition of a dimension tree with natural
    unfolding order).  Node ids are the table's indices."""
    nn = len(children)
    nodes = [None] * nn
    leaves = []

    def visit(i, parent, level):
        l, r = children[i]
        if l < 0:
            nodes[i] = Node(i, len(leaves), len(leaves), parent, level)
            leaves.append(i)
            return
        visit(l, i, level + 1)
        visit(r, i, level + 1)
        nd = Node(i, nodes[l].a, nodes[r].b, parent, level)
        nd.left, nd.right = l, r
        nodes[i] = nd

    visit(0, -1, 0)
    if any(nd is None for nd in nodes) or nn != 2 * len(leaves) - 1:
        raise ValueError("not a binary dimension tree")
    return nodes


def children_of(tree):
    """Child table [(left, right), ...] of a tree given as a list of Nodes."""
    return [(-1, -1) if nd.is_leaf else (nd.left, nd.right) for nd in tree]


def node_rows(shape, nd):
    return int(np.prod(shape[nd.a:nd.b + 1]))


def node_cols(shape, nd):
    return int(np.prod(complement_shape(shape, nd.a, nd.b))) if (nd.a, nd.b) != (0, len(shape) - 1) else 1


def transfer_tensor(US, Ul, Ur):
    """B_S(i, j, k) = <U_S(:, i), U_{S_l}(:, j) (x) U_{S_r}(:, k)> (Sec. 4, transfer-tensor eq.).

    With C-order rows, (v (x) w)[a n_r + b] = v[a] w[b], so column i of U_S
    reshaped to M_i (n_l x n_r) gives B_S(i, j, k) = (U_l^T M_i U_r)[j, k].
    """
    nl, nr = Ul.shape[0], Ur.shape[0]
    M = US.T.reshape(US.shape[1], nl, nr)
    return np.einsum("iab,aj,bk->ijk", M, Ul, Ur)


def root_transfer(X, Ul, Ur):
    """B_R(1, j, k) = <vec X, U_{R_l}(:, j) (x) U_{R_r}(:, k)> (Sec. 4, root eq.).

    vec X in C order is X^(R_l) viewed as an n_{R_l} x n_{R_r} matrix, so
    B_R(1, :, :) = U_{R_l}^T X^(R_l) U_{R_r}.
    """
    Xm = np.asarray(X, dtype=np.float64).reshape(Ul.shape[0], Ur.shape[0])
    return (Ul.T @ Xm @ Ur)[None, :, :]


def default_ranks(nodes, r):
    return [1 if nd.id == 0 else int(r) for nd in nodes]


def default_w(shape, nodes):
    """w_S = min(20 max_k n_k, n_{notin S}) (the paper takes 20 n fibers at every
    node in its parallel H-Tucker experiment, Sec. 4.2)."""
    n = max(shape)
    return [0 if nd.id == 0 else min(20 * n, node_cols(shape, nd)) for nd in nodes]


def alpha_w(shape, nodes, alpha):
    """w_S = min(floor(alpha^(d-2) n_S), n_{notin S}) at every non-root node: the
    sampling rule of the paper's serial H-Tucker tests (Sec. 4.2), n_S the rows of
    the node's unfolding; the root takes none (0)."""
    d = len(shape)
    scale = float(alpha) ** (d - 2)
    return [0 if nd.id == 0 else min(int(np.floor(scale * node_rows(shape, nd))), node_cols(shape, nd))
            for nd in nodes]


def sub_r_rtl_ht(X, rank, p, w=None, seed=0, tree=None, with_root=True):
    """[{U_k}, {B_S}] = Sub-R-RtL-HT(X, T, r, w, p) (Alg. 2).

    Every non-root node S (leaves included) gets U_S from the range finder on
    w_S sampled columns of X^(S) (all nodes are independent in the RtL scheme,
    Sec. 4.1 remark); every internal non-root node gets its transfer tensor;
    the root transfer tensor is taken from vec X.  ``rank`` is one rank per
    node (the root's is 1) or a scalar.  Returns leaf factors, transfer tensors
    (indexed by node id; None for leaves), the node bases U_S and intermediates.
    X keeps its stored precision here: the sampled columns and the root are
    promoted to float64 where they are formed.  ``with_root=False`` leaves
    B[0] = None (for callers that form the root from X themselves).
    """
    X = np.asarray(X)
    shape = X.shape
    nodes = balanced_tree(X.ndim) if tree is None else tree
    ranks = default_ranks(nodes, rank) if np.ndim(rank) == 0 else [int(v) for v in rank]
    ranks[0] = 1
    w = default_w(shape, nodes) if w is None else [int(v) for v in (w if np.ndim(w) else [w] * len(nodes))]
    US = [None] * len(nodes)
    info = [None] * len(nodes)
    for nd in nodes:
        if nd.id == 0:
            continue
        nS, N = node_rows(shape, nd), node_cols(shape, nd)
        if ranks[nd.id] + p > min(nS, N) or not (ranks[nd.id] + p <= w[nd.id] <= N):
            raise ValueError("node %d: need r+p <= min(n_S, n_notin_S) and r+p <= w <= n_notin_S" % nd.id)
        pi = rng.fiber_indices(N, w[nd.id], seed, nd.id)
        Y = gather_fibers(X, nd.a, nd.b, pi)
        out = range_finder(Y, pi, ranks[nd.id], p, seed, nd.id)
        out.update(pi=pi, Y=Y)
        US[nd.id] = out["U"]
        info[nd.id] = out
    B = [None] * len(nodes)
    for nd in nodes:
        if nd.is_leaf:
            continue
        if nd.id == 0:
            if with_root:
                B[0] = root_transfer(X, US[nd.left], US[nd.right])
        else:
            B[nd.id] = transfer_tensor(US[nd.id], US[nd.left], US[nd.right])
    leaves = sorted((nd for nd in nodes if nd.is_leaf), key=lambda nd: nd.a)
    U_leaf = [US[nd.id] for nd in leaves]
    return dict(U=U_leaf, B=B, US=US, tree=nodes, ranks=ranks, w=w, info=info)


def reconstruct(U_leaf, B, tree, shape):
    """Full tensor of an H-Tucker format: U_hat(leaf k) = U_k,
    U_hat(S) = (U_hat(S_l) (x) U_hat(S_r)) (B_S^(1))^T for internal S, and
    X = U_hat(R_l) B_R(1, :, :) U_hat(R_r)^T reshaped to the tensor shape."""
    Uh = [None] * len(tree)
    for nd in tree:
        if nd.is_leaf:
            Uh[nd.id] = U_leaf[nd.a]
    for nd in sorted(tree, key=lambda n: -n.level):
        if nd.is_leaf or nd.id == 0:
            continue
        Ul, Ur = Uh[nd.left], Uh[nd.right]
        # column i: vec(U_l B_S[i] U_r^T), C-order rows (left index slower)
        Uh[nd.id] = np.einsum("aj,ijk,bk->abi", Ul, B[nd.id], Ur).reshape(Ul.shape[0] * Ur.shape[0], -1)
    root = tree[0]
    Xm = Uh[root.left] @ B[0][0] @ Uh[root.right].T
    return Xm.reshape(shape)
