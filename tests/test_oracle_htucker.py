"""Pins of the Sub-R-RtL-HT oracle (Alg. 2): the paper's order-8 dimension tree
(tests/golden), the transfer-tensor and root definitions written with explicit
Kronecker products, the full-sampling case that reduces to deterministic RtL-HT
and its error window (Sec. 4 quasi-optimality), exact recovery of tensors of
known hierarchical rank, nestedness, and the float32 input generator of the
1/||x|| workload."""

import itertools
import os

import numpy as np
import pytest

import synth
from oracle import brute, htucker, tucker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_tree_matches_paper_figure_d8():
    with open(os.path.join(GOLDEN, "dimtree_d8.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    tree = htucker.balanced_tree(8)
    assert len(tree) == len(rows) == 15
    for (nid, modes, bname), nd in zip(rows, tree):
        want = [int(m) - 1 for m in modes.split(",")]
        assert int(nid) == nd.id
        assert list(range(nd.a, nd.b + 1)) == want
        assert (bname != "-") == (not nd.is_leaf)
    # 14 node bases, 7 transfer tensors (Sec. 4.2.2)
    assert sum(1 for nd in tree if nd.id != 0) == 14
    assert sum(1 for nd in tree if not nd.is_leaf) == 7
    for nd in tree:
        if not nd.is_leaf:
            l, r = tree[nd.left], tree[nd.right]
            assert (l.a, r.b) == (nd.a, nd.b) and l.b + 1 == r.a


def test_tree_definition_properties_other_orders():
    for d in range(2, 12):
        tree = htucker.balanced_tree(d)
        leaves = sorted(nd.a for nd in tree if nd.is_leaf)
        assert leaves == list(range(d)) and len(tree) == 2 * d - 1
        depth = max(nd.level for nd in tree)
        assert depth == int(np.ceil(np.log2(d)))  # z = ceil(log2 d), Sec. 4


def test_transfer_and_root_tensors_match_kronecker_definition():
    rs = np.random.default_rng(1)
    Ul, Ur = rs.standard_normal((3, 2)), rs.standard_normal((4, 3))
    US = rs.standard_normal((12, 2))
    B = htucker.transfer_tensor(US, Ul, Ur)
    for i, j, k in itertools.product(range(2), range(2), range(3)):
        assert np.isclose(B[i, j, k], US[:, i] @ np.kron(Ul[:, j], Ur[:, k]), rtol=1e-13, atol=1e-13)
    X = rs.standard_normal((3, 2, 2, 2))  # R_l = modes {0,1} (6 rows), R_r = {2,3} (4)
    Vl, Vr = rs.standard_normal((6, 2)), rs.standard_normal((4, 3))
    BR = htucker.root_transfer(X, Vl, Vr)
    for j, k in itertools.product(range(2), range(3)):
        assert np.isclose(BR[0, j, k], X.ravel() @ np.kron(Vl[:, j], Vr[:, k]), rtol=1e-13, atol=1e-13)


def test_full_sampling_reduces_to_deterministic_rtl_ht():
    # w_S = n_{notin S} and r_S + p = n_S at every node: each U_S is the dominant
    # left singular basis of X^(S), i.e. deterministic RtL-HT (Sec. 4)
    rs = np.random.default_rng(2)
    X = rs.standard_normal((3, 4, 3, 4))
    tree = htucker.balanced_tree(4)
    p = 1
    ranks = [1] + [htucker.node_rows(X.shape, nd) - p for nd in tree[1:]]
    w = [0] + [htucker.node_cols(X.shape, nd) for nd in tree[1:]]
    out = htucker.sub_r_rtl_ht(X, ranks, p, w=w, seed=5)
    ref = brute.rtl_ht(X, ranks)
    for nd in tree[1:]:
        assert np.abs(out["US"][nd.id] - ref["US"][nd.id]).max() < 1e-10
    for nd in tree:
        if not nd.is_leaf:
            assert np.abs(out["B"][nd.id] - ref["B"][nd.id]).max() < 1e-10


def test_full_sampling_error_within_rtl_ht_bounds():
    # Sec. 4 (RtL-HT quasi-optimality, sqrt(2d-3) times the best error): with every
    # column sampled and r_S + p = min(n_S, n_notin_S), each U_S is the dominant left
    # singular basis of X^(S) and the format is the RtL-HT truncation, whose error
    # squared is at most the sum over the non-root nodes but one child of the root of
    # the discarded squared singular values of X^(S); no format of these ranks does
    # better than the largest single-node tail.  Low hierarchical rank plus noise, so
    # a wrong transfer tensor or reconstruction step lands far outside the window.
    for trial in range(12):
        rs = np.random.default_rng(300 + trial)
        shape = tuple(int(v) for v in rs.integers(3, 7, size=int(rs.integers(3, 6))))
        X = _random_ht_tensor(shape, 2, 300 + trial)
        X = X / np.linalg.norm(X) + 1e-2 * rs.standard_normal(shape) / np.sqrt(X.size)
        tree = htucker.balanced_tree(len(shape))
        p = int(rs.integers(1, 3))
        ranks = [1] + [min(htucker.node_rows(shape, nd), htucker.node_cols(shape, nd)) - p for nd in tree[1:]]
        if min(ranks[1:]) < 2:
            continue
        w = [0] + [htucker.node_cols(shape, nd) for nd in tree[1:]]
        out = htucker.sub_r_rtl_ht(X, ranks, p, w=w, seed=trial)
        err = np.linalg.norm(X - htucker.reconstruct(out["U"], out["B"], out["tree"], shape))
        tails = {}
        for nd in tree[1:]:
            rows = int(np.prod(shape[nd.a:nd.b + 1]))
            M = np.moveaxis(X, list(range(nd.a, nd.b + 1)), list(range(nd.b - nd.a + 1))).reshape(rows, -1)
            sv = np.linalg.svd(M, compute_uv=False)
            tails[nd.id] = float(np.sum(sv[ranks[nd.id]:] ** 2))
        lo = np.sqrt(max(tails.values()))
        hi = np.sqrt(sum(v for k, v in tails.items() if k != tree[0].right))
        assert lo * (1 - 1e-12) <= err <= hi * (1 + 1e-12), (shape, lo, err, hi)
        assert len(tails) == 2 * len(shape) - 2


def _random_ht_tensor(shape, r, seed, tree=None):
    """Tensor built from a random H-Tucker format of hierarchical rank <= r."""
    rs = np.random.default_rng(seed)
    tree = htucker.balanced_tree(len(shape)) if tree is None else tree
    U = [synth.haar(n, r, rs) for n in shape]
    B = [None] * len(tree)
    for nd in tree:
        if nd.is_leaf:
            continue
        rout = 1 if nd.id == 0 else r
        B[nd.id] = rs.standard_normal((rout, r, r))
    return htucker.reconstruct(U, B, tree, shape)


def test_exact_recovery_of_known_hierarchical_rank():
    shape = (5, 6, 4, 5, 6)
    X = _random_ht_tensor(shape, 2, 3)
    out = htucker.sub_r_rtl_ht(X, 2, p=2, seed=7)
    Xh = htucker.reconstruct(out["U"], out["B"], out["tree"], shape)
    assert tucker.relerr(X, Xh) < 1e-10
    # nestedness Range(U_S) in Range(U_l (x) U_r) (Sec. 4)
    for nd in out["tree"]:
        if nd.is_leaf or nd.id == 0:
            continue
        K = np.kron(out["US"][nd.left], out["US"][nd.right])
        res = out["US"][nd.id] - K @ (K.T @ out["US"][nd.id])
        assert np.abs(res).max() < 1e-10
    for nd in out["tree"][1:]:
        U = out["US"][nd.id]
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-13


def test_full_rank_format_reconstructs_exactly():
    rs = np.random.default_rng(4)
    X = rs.standard_normal((2, 3, 2, 2))
    tree = htucker.balanced_tree(4)
    ranks = [1] + [htucker.node_rows(X.shape, nd) for nd in tree[1:]]
    ref = brute.rtl_ht(X, ranks)
    Xh = htucker.reconstruct(ref["U"], ref["B"], tree, X.shape)
    assert np.abs(Xh - X).max() < 1e-12


def test_inv_norm_generator_matches_definition():
    # X(i) = (sum_j x_{i_j}^2)^{-1/2} on the uniform grid over [1, 2]^d (Sec. 4.2.1)
    n, d = 5, 4
    X = synth.inv_norm_tensor(n, d)
    x = np.linspace(1.0, 2.0, n)
    for i in itertools.product(range(n), repeat=d):
        want = 1.0 / np.sqrt(sum(x[v] ** 2 for v in i))
        assert abs(float(X[i]) - want) <= 6e-8 * want
    # entries at arbitrary indices agree bit-for-bit with the full tensor
    rs = np.random.default_rng(0)
    idx = tuple(rs.integers(0, n, size=50) for _ in range(d))
    assert np.array_equal(synth.inv_norm_entries(idx, n), X[idx])


def test_inv_norm_torch_generator_is_bit_identical():
    # the torch generator (used for the 17 GB 16^8 tensor on the device) makes the
    # same bytes as the numpy definition above
    torch = pytest.importorskip("torch")
    for n, d in [(5, 4), (16, 3), (3, 7)]:
        a = synth.inv_norm_tensor(n, d)
        b = synth.inv_norm_tensor_torch(n, d)
        assert b.dtype == torch.float32 and tuple(b.shape) == (n,) * d
        assert np.array_equal(a, b.numpy())


def test_root_transfer_is_linear_in_row_blocks():
    # the full-size H-Tucker test forms B_R from row blocks of X^(R_l); the sum of
    # the blocks' root transfers is the root transfer of the whole matrix
    rs = np.random.default_rng(4)
    X = rs.standard_normal((12, 10))
    Ul, Ur = rs.standard_normal((12, 3)), rs.standard_normal((10, 2))
    whole = htucker.root_transfer(X, Ul, Ur)
    parts = sum(htucker.root_transfer(X[a:a + 5], Ul[a:a + 5], Ur) for a in range(0, 12, 5))
    assert np.allclose(whole, parts, rtol=1e-14, atol=1e-14)
    assert whole.shape == (1, 3, 2)


def test_sub_r_rtl_ht_without_root_matches():
    X = synth.inv_norm_tensor(5, 4)
    a = htucker.sub_r_rtl_ht(X, 2, 1, seed=3)
    b = htucker.sub_r_rtl_ht(X, 2, 1, seed=3, with_root=False)
    assert b["B"][0] is None
    for nd in a["tree"][1:]:
        assert np.array_equal(a["US"][nd.id], b["US"][nd.id])


def test_inv_norm_workload_ht_runs_and_is_accurate():
    # small restriction of the 1/||x|| workload; the paper reports no bound for
    # Sub-R-RtL-HT (Sec. 4), so only sanity: error well below 1e-2 at rank 5
    X = synth.inv_norm_tensor(8, 6).astype(np.float64)
    out = htucker.sub_r_rtl_ht(X, 5, p=3, seed=3)
    Xh = htucker.reconstruct(out["U"], out["B"], out["tree"], X.shape)
    assert tucker.relerr(X, Xh) < 1e-2


def test_alpha_sampling_rule():
    # Sec. 4.2: min(alpha^(d-2) n_S, n_notin_S) fibers at node S, n_S its unfolding's rows.
    # 3 x 4 x 5 x 6, alpha = 2 (scale 4), worked by hand: {0,1} 12 rows -> min(48, 30);
    # {2,3} 30 rows -> min(120, 12); leaves 3, 4, 5, 6 rows -> 12, 16, 20, 24
    shape = (3, 4, 5, 6)
    nodes = htucker.balanced_tree(4)
    assert htucker.alpha_w(shape, nodes, 2) == [0, 30, 12, 12, 16, 20, 24]
    # the binding's helper (host arithmetic, no GPU) follows the same rule on the same tree
    import paper_2603_21379_gb300 as rt
    assert rt.ht_alpha_w(shape, 2) == [0, 30, 12, 12, 16, 20, 24]
    for shape, alpha in [((2, 3, 4, 5, 6), 1.5), ((16,) * 8, 1.2), ((7, 5, 9), 3.0)]:
        nodes = htucker.balanced_tree(len(shape))
        assert rt.ht_alpha_w(shape, alpha) == htucker.alpha_w(shape, nodes, alpha)


# ----------------------------------------------------------------- general trees
def caterpillar(d):
    """Child table of the caterpillar tree {0..d-1} -> {0}, {1..d-1} -> {1}, {2..d-1} ...:
    node 0 the root, internal node 2j has children 2j+1 (the leaf {j}) and 2j+2."""
    ch = []
    for j in range(d - 1):
        ch.append((2 * j + 1, 2 * j + 2))
        ch.append((-1, -1))
    ch.append((-1, -1))
    return ch


def left_heavy(d):
    """Child table with the root's right child a leaf: {0..d-2} on the left (balanced
    below it, ids shifted), {d-1} on the right."""
    sub = htucker.children_of(htucker.balanced_tree(d - 1))
    ch = [(1, 2 * d - 2)]
    for (l, r) in sub:
        ch.append((-1, -1) if l < 0 else (l + 1, r + 1))
    ch.append((-1, -1))
    return ch


def test_tree_from_children_reproduces_balanced_tree():
    for d in range(2, 12):
        a = htucker.balanced_tree(d)
        b = htucker.tree_from_children(htucker.children_of(a))
        assert [(n.id, n.a, n.b, n.left, n.right, n.level) for n in a] == \
            [(n.id, n.a, n.b, n.left, n.right, n.level) for n in b]


def test_tree_from_children_general_shapes():
    t = htucker.tree_from_children(caterpillar(5))
    # the leaves hold modes 0..4 in order; internal node 2j is {j..4}
    assert [(n.a, n.b) for n in t] == [(0, 4), (0, 0), (1, 4), (1, 1), (2, 4), (2, 2), (3, 4), (3, 3), (4, 4)]
    assert max(n.level for n in t) == 4
    t = htucker.tree_from_children(left_heavy(5))
    root = t[0]
    assert (t[root.left].a, t[root.left].b, t[root.right].a, t[root.right].b) == (0, 3, 4, 4)
    for bad in ([(1, 2), (-1, -1)], [(1, 1), (-1, -1), (-1, -1)], [(1, 2), (-1, -1), (0, 1)]):
        with pytest.raises((ValueError, RecursionError, IndexError, TypeError)):
            htucker.tree_from_children(bad)


@pytest.mark.parametrize("make", [caterpillar, left_heavy])
def test_general_tree_full_sampling_error_within_rtl_ht_bounds(make):
    # the RtL-HT window of Sec. 4 (largest node tail <= error <= sum of the node
    # tails but one child of the root) on trees other than the balanced one
    for trial in range(6):
        rs = np.random.default_rng(500 + trial)
        d = int(rs.integers(3, 6))
        shape = tuple(int(v) for v in rs.integers(3, 6, size=d))
        tree = htucker.tree_from_children(make(d))
        X = _random_ht_tensor(shape, 2, 500 + trial, tree=tree)
        X = X / np.linalg.norm(X) + 1e-2 * rs.standard_normal(shape) / np.sqrt(X.size)
        p = 1
        ranks = [1] + [min(htucker.node_rows(shape, nd), htucker.node_cols(shape, nd)) - p for nd in tree[1:]]
        if min(ranks[1:]) < 1:
            continue
        w = [0] + [htucker.node_cols(shape, nd) for nd in tree[1:]]
        out = htucker.sub_r_rtl_ht(X, ranks, p, w=w, seed=trial, tree=tree)
        ref = brute.rtl_ht(X, ranks, tree=tree)
        for nd in tree[1:]:
            assert np.abs(out["US"][nd.id] - ref["US"][nd.id]).max() < 1e-9
        err = np.linalg.norm(X - htucker.reconstruct(out["U"], out["B"], tree, shape))
        tails = {}
        for nd in tree[1:]:
            M = tucker.set_unfold(X, nd.a, nd.b)
            sv = np.linalg.svd(M, compute_uv=False)
            tails[nd.id] = float(np.sum(sv[ranks[nd.id]:] ** 2))
        lo = np.sqrt(max(tails.values()))
        hi = np.sqrt(sum(v for k, v in tails.items() if k != tree[0].right))
        assert lo * (1 - 1e-12) <= err <= hi * (1 + 1e-12), (shape, lo, err, hi)


@pytest.mark.parametrize("make", [caterpillar, left_heavy])
def test_general_tree_exact_recovery(make):
    shape = (4, 5, 3, 6, 4)
    tree = htucker.tree_from_children(make(5))
    X = _random_ht_tensor(shape, 2, 11, tree=tree)
    out = htucker.sub_r_rtl_ht(X, 2, p=1, seed=2, tree=tree)
    assert tucker.relerr(X, htucker.reconstruct(out["U"], out["B"], tree, shape)) < 1e-10
    # nestedness on this tree: Range(U_S) inside Range(U_l (x) U_r)
    for nd in tree:
        if nd.is_leaf or nd.id == 0:
            continue
        K = np.kron(out["US"][nd.left], out["US"][nd.right])
        assert np.abs(out["US"][nd.id] - K @ (K.T @ out["US"][nd.id])).max() < 1e-10


def test_binding_tree_helper_matches_oracle():
    import paper_2603_21379_gb300 as rt
    for ch in (caterpillar(5), left_heavy(5), caterpillar(3), htucker.children_of(htucker.balanced_tree(7))):
        a = rt.ht_tree_from_children(ch)
        b = htucker.tree_from_children(ch)
        assert [tuple(x) for x in a] == [(n.a, n.b, -1 if n.is_leaf else n.left, -1 if n.is_leaf else n.right,
                                          n.level) for n in b]
    with pytest.raises(ValueError):
        rt.ht_tree_from_children([(1, 2), (-1, -1)])
