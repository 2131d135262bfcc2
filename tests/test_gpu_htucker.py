"""GPU parity of the Sub-R-RtL-HT path (S8-S10) against the float64 oracle:
node bases U_S up to column sign (well-separated columns element-wise,
clusters through projectors), transfer tensors on the determined columns
(signs aligned), and the relative error of the whole format."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import brute, htucker, tucker  # noqa: E402
from parity_util import GAP_MIN, RELERR_TOL, U_TOL, clusters, compare_factor, orthonormality, to_np  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_21379_gb300 import build
    build.build()
    import paper_2603_21379_gb300 as m
    m.load_library()
    return m


def _strict_cols(sigma, r, gap_min=GAP_MIN):
    cl, tail_ok = clusters(sigma, r, gap_min)
    out = []
    for ci, c in enumerate(cl):
        if ci == len(cl) - 1 and not tail_ok:
            continue
        if len(c) == 1:
            out.append(c[0])
    return out


def _check_nodes(ref, U_leaf, B, Un, root_ref=None, gap_min=GAP_MIN):
    """Node bases, leaf factors and transfer tensors of a GPU result against an
    oracle result ``ref``; the root transfer tensor against ``root_ref`` (default
    ref["B"][0])."""
    tree = ref["tree"]
    signs, strict = {}, {}
    for nd in tree[1:]:
        sig = ref["info"][nd.id]["sigma"]
        Ug = to_np(Un[nd.id])
        s, dev, _, _ = compare_factor(Ug, ref["US"][nd.id], sig, gap_min=gap_min)
        assert dev <= U_TOL, (nd.id, dev)
        assert orthonormality(Ug) < 1e-5
        signs[nd.id] = s
        strict[nd.id] = _strict_cols(sig, ref["ranks"][nd.id], gap_min)
    for k, nd in enumerate(sorted((n for n in tree if n.is_leaf), key=lambda n: n.a)):
        assert np.array_equal(to_np(U_leaf[k]), to_np(Un[nd.id]))
    for nd in tree:
        if nd.is_leaf:
            continue
        Bg = to_np(B[nd.id])
        Br = (ref["B"][0] if root_ref is None else root_ref) if nd.id == 0 else ref["B"][nd.id]
        si = np.ones(1) if nd.id == 0 else signs[nd.id]
        Bg = Bg * si[:, None, None] * signs[nd.left][None, :, None] * signs[nd.right][None, None, :]
        ii = [0] if nd.id == 0 else strict[nd.id]
        jj, kk = strict[nd.left], strict[nd.right]
        if ii and jj and kk:
            sub_g = Bg[np.ix_(ii, jj, kk)]
            sub_r = Br[np.ix_(ii, jj, kk)]
            assert np.abs(sub_g - sub_r).max() <= 1e-4 * max(1.0, np.abs(Br).max()), nd.id


def _compare_ht(rt, X, rank, p, w=None, seed=0, x_oracle=None, gap_min=GAP_MIN, tree=None):
    """GPU against oracle on the dimension tree ``tree`` (child table; None =
    balanced), through rhtucker_decompose and rhtucker_relerr."""
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    U_leaf, B, Un = rt.rhtucker_decompose(Xd, rank, p, w=w, seed=seed, return_nodes=True, tree=tree)
    torch.cuda.synchronize()
    Xo = np.asarray(X if x_oracle is None else x_oracle, dtype=np.float64)
    otree = None if tree is None else htucker.tree_from_children(tree)
    ref = htucker.sub_r_rtl_ht(Xo, rank, p, w=w, seed=seed, tree=otree)
    _check_nodes(ref, U_leaf, B, Un, gap_min=gap_min)
    eg = rt.rhtucker_relerr(Xd, U_leaf, B, rank, tree=tree)
    er = tucker.relerr(Xo, htucker.reconstruct(ref["U"], ref["B"], ref["tree"], Xo.shape))
    assert abs(eg - er) <= RELERR_TOL, (eg, er)
    return eg, er


def test_inv_norm_d6(rt):
    X = synth.inv_norm_tensor(8, 6)
    eg, er = _compare_ht(rt, X, 5, 3, seed=3)
    assert er < 1e-5


def test_inv_norm_d8_n6(rt):
    X = synth.inv_norm_tensor(6, 8)
    _compare_ht(rt, X, 4, 2, seed=1)


def test_root_stream_ragged_rows(rt):
    # root of a (5, 7, 8, 8) tensor: X^(R_l) is 35 x 64, so the streaming root pass
    # runs one partial 64-row block over two 32-column stages
    rs = np.random.default_rng(8)
    X = rs.standard_normal((5, 7, 8, 8)).astype(np.float32)
    _compare_ht(rt, X, 3, 2, seed=4)


def test_root_stream_ragged_columns(rt):
    # 6 x 5 x 6 x 6: X^(R_l) is 30 x 36, so the streaming root pass runs two 32-column
    # stages, the second overhanging the rows by 28 zero-filled columns, against a copy
    # of U_r padded to 64 rows
    rs = np.random.default_rng(12)
    X = rs.standard_normal((6, 5, 6, 6)).astype(np.float32)
    _compare_ht(rt, X, 3, 2, seed=8)


def test_root_stream_wide(rt):
    # 12 x 10 x 16 x 40: X^(R_l) is 120 x 640 (two row blocks, 20 column stages), ranks 7
    rs = np.random.default_rng(9)
    X = rs.standard_normal((12, 10, 16, 40)).astype(np.float32)
    _compare_ht(rt, X, 7, 3, seed=6)


@pytest.mark.parametrize("rank", [7, 8])
def test_root_stream_rank8_rows(rt, rank):
    # 16^3 x 40: X^(R_l) is 256 x 640 (20 column stages, more than the 8-slot ring twice
    # over) with U_r rows of 8 floats (rank 8, and rank 7 padded to 8): the case where
    # ring slots read with plain shared loads were read again after their release
    rs = np.random.default_rng(21)
    X = rs.standard_normal((16, 16, 16, 40)).astype(np.float32)
    _compare_ht(rt, X, rank, 2, seed=2)


def test_exact_hierarchical_rank_recovery(rt):
    rs = np.random.default_rng(3)
    shape = (5, 6, 4, 5, 6)
    tree = htucker.balanced_tree(5)
    U = [synth.haar(n, 2, rs) for n in shape]
    B = [None] * len(tree)
    for nd in tree:
        if not nd.is_leaf:
            B[nd.id] = rs.standard_normal((1 if nd.id == 0 else 2, 2, 2))
    X = htucker.reconstruct(U, B, tree, shape).astype(np.float32)
    eg, er = _compare_ht(rt, X, 2, 2, seed=7)
    assert eg < 1e-5


def test_wide_ranks(rt):
    # hierarchical ranks 54 at the two inner nodes (r + p = 64, the largest supported
    # width; 1600-row node unfoldings: a two-level TSQR tree of Z, and B^T chunks
    # factored from row-block partials) and 30 at the leaves of a 40^4 tensor built in the format (Gaussian
    # transfer tensors, Haar leaves) plus 1e-4 noise: 54 x 30 x 30 transfer tensors and
    # a 54 x 54 root.  Sampled singular values ~1e-3 of sigma_1 apart: columns closer
    # than 5e-3 are compared as subspaces.
    rs = np.random.default_rng(34)
    shape, ranks, p = (40, 40, 40, 40), [1, 54, 54, 30, 30, 30, 30], 10
    tree = htucker.balanced_tree(4)
    U = [synth.haar(n, 30, rs) for n in shape]
    B = [None] * len(tree)
    for nd in tree:
        if not nd.is_leaf:
            B[nd.id] = rs.standard_normal((1 if nd.id == 0 else 54, ranks[nd.left], ranks[nd.right]))
    X = htucker.reconstruct(U, B, tree, shape)
    X = (X / np.abs(X).max() + 1e-4 * rs.standard_normal(shape)).astype(np.float32)
    eg, er = _compare_ht(rt, X, ranks, p, seed=5, gap_min=5e-3)
    assert er < 5e-3


def test_mixed_transfer_forms_and_chunked_root(rt):
    # node {0,1} rank 8 (grouped transfer kernel) beside node {2,3} rank 20 with rank-14
    # children (general form), and a root right-child rank of 20: two chunks of 10
    # columns of U_r, each a streaming root pass (n_r = 1024).  The format is built with
    # these ranks, so node {2,3} has 8 determined directions (the root's two children
    # share one rank); its other 12 are noise and not compared column by column.
    rs = np.random.default_rng(55)
    shape, ranks, p = (8, 9, 32, 32), [1, 8, 20, 3, 3, 14, 14], 3
    tree = htucker.balanced_tree(4)
    U = [synth.haar(n, r, rs) for n, r in zip(shape, ranks[3:])]
    B = [None] * len(tree)
    for nd in tree:
        if not nd.is_leaf:
            B[nd.id] = rs.standard_normal((1 if nd.id == 0 else ranks[nd.id], ranks[nd.left], ranks[nd.right]))
    X = htucker.reconstruct(U, B, tree, shape)
    X = (X / np.abs(X).max() + 1e-4 * rs.standard_normal(shape)).astype(np.float32)
    _compare_ht(rt, X, ranks, p, seed=5, gap_min=5e-3)


def test_order_16_balanced_tree(rt):
    # d = 16: 31 nodes (16 leaves of 2 rows, 4 levels of internal nodes), a 256 x 256
    # root unfolding; rank 1 at every node of a rank-one tensor plus noise
    X = synth.tucker_tensor((2,) * 16, (1,) * 16, noise=1e-3, data_seed=41)
    _compare_ht(rt, X, 1, 1, seed=2)


def test_full_sampling_matches_rtl_ht(rt):
    rs = np.random.default_rng(2)
    X = rs.standard_normal((3, 4, 3, 4)).astype(np.float32)
    tree = htucker.balanced_tree(4)
    p = 1
    ranks = [1] + [htucker.node_rows(X.shape, nd) - p for nd in tree[1:]]
    w = [1] + [htucker.node_cols(X.shape, nd) for nd in tree[1:]]
    _compare_ht(rt, X, ranks, p, w=w, seed=5)
    ref = brute.rtl_ht(X.astype(np.float64), ranks)
    Xd = torch.from_numpy(X).cuda()
    _, _, Un = rt.rhtucker_decompose(Xd, ranks, p, w=w, seed=5, return_nodes=True)
    for nd in tree[1:]:
        Ug = to_np(Un[nd.id])
        sg = np.sign((Ug * ref["US"][nd.id]).sum(axis=0))
        assert np.abs(Ug * sg - ref["US"][nd.id]).max() <= U_TOL


def test_tall_node_tsqr_path(rt):
    # node {0,1,2} of a 16^6 tensor has 4096 rows: two-level TSQR of Z
    X = synth.inv_norm_tensor(16, 6)
    _compare_ht(rt, X, 6, 3, seed=2)


def test_inv_norm_16_8_full_size(rt):
    # the paper's H-Tucker workload at full size: f = 1/||x|| on a 16^8 grid (17.2 GB
    # float32), balanced tree, rank 10 at every node, p = 5, w = 320 columns per node.
    # All 14 node bases and 6 transfer tensors are compared with the oracle (which
    # needs only the sampled columns); the root, B_R = U_l^T X^(R_l) U_r, with the
    # oracle's root transfer summed over row blocks of X^(R_l).
    cfg = synth.INVNORM_16_8
    n, d = cfg["n"], cfg["d"]
    Xd = synth.inv_norm_tensor_torch(n, d, cfg["lo"], cfg["hi"], device="cuda")
    rs = np.random.default_rng(0)
    idx = tuple(rs.integers(0, n, size=2000) for _ in range(d))
    assert np.array_equal(Xd[idx].cpu().numpy(), synth.inv_norm_entries(idx, n, cfg["lo"], cfg["hi"]))
    U_leaf, B, Un = rt.rhtucker_decompose(Xd, cfg["rank"], cfg["p"], w=cfg["w"], seed=cfg["seed"],
                                          return_nodes=True)
    torch.cuda.synchronize()
    Xh = Xd.cpu().numpy()
    del Xd
    ref = htucker.sub_r_rtl_ht(Xh, cfg["rank"], cfg["p"], w=cfg["w"], seed=cfg["seed"], with_root=False)
    root = ref["tree"][0]
    Ul, Ur = ref["US"][root.left], ref["US"][root.right]
    Xm = Xh.reshape(Ul.shape[0], Ur.shape[0])
    blk = 4096
    BR = sum(htucker.root_transfer(Xm[a:a + blk], Ul[a:a + blk], Ur) for a in range(0, Xm.shape[0], blk))
    _check_nodes(ref, U_leaf, B, Un, root_ref=BR)


def test_graph_replay_matches_direct_launches(rt):
    rs = np.random.default_rng(10)
    X = torch.from_numpy(rs.standard_normal((6, 7, 8, 9, 5)).astype(np.float32)).cuda()
    Ul0, B0 = rt.rhtucker_decompose(X, 3, 2, seed=4)
    Ul1, B1 = rt.rhtucker_decompose(X, 3, 2, seed=5)
    flat_u = torch.cat([u.reshape(-1) for u in Ul0]).clone()
    flat_b = torch.cat([b.reshape(-1) for b in B0.values()]).clone()
    out = (torch.empty_like(flat_u), torch.empty_like(flat_b))
    for seed, (Ul, B) in ((4, (Ul0, B0)), (4, (Ul0, B0)), (5, (Ul1, B1))):   # capture, replay, other seed
        Ug, Bg = rt.rhtucker_decompose(X, 3, 2, seed=seed, graph=True, out=out)
        torch.cuda.synchronize()
        for a, b in zip(Ug, Ul):
            assert torch.equal(a, b)
        for k in B:
            assert torch.equal(Bg[k], B[k])


# ----------------------------------------------------------------- other dimension trees
def _caterpillar(d):
    ch = []
    for j in range(d - 1):
        ch.append((2 * j + 1, 2 * j + 2))
        ch.append((-1, -1))
    ch.append((-1, -1))
    return ch


def test_caterpillar_tree_d5(rt):
    # Alg. 2 on the caterpillar tree {0..4} -> {0}, {1..4} -> {1}, ...: node bases of
    # 8, 8^4 = 4096 ... rows, four transfer tensors, the root's left child a leaf
    X = synth.inv_norm_tensor(8, 5)
    _compare_ht(rt, X, 4, 3, seed=6, tree=_caterpillar(5))


def test_tree_with_leaf_right_child_of_root(rt):
    # root {0..4} -> {0..3}, {4}: the root pass takes X as 4096 x 8 (U_{R_r} of a leaf);
    # ids below the left child are the balanced tree of 4 modes shifted by one
    ch = [(1, 8), (2, 3), (4, 5), (6, 7), (-1, -1), (-1, -1), (-1, -1), (-1, -1), (-1, -1)]
    rs = np.random.default_rng(21)
    X = (synth.inv_norm_tensor(8, 5) + 1e-3 * rs.standard_normal((8,) * 5)).astype(np.float32)
    _compare_ht(rt, X, 4, 2, seed=7, tree=ch)


def test_alpha_sampling_rule_on_the_gpu(rt):
    # w_S = min(floor(alpha^(d-2) n_S), n_notin_S) at every node (Sec. 4.2), from the
    # binding's helper; the oracle takes its own restatement of the rule
    X = synth.inv_norm_tensor(6, 6)
    shape = X.shape
    w = rt.ht_alpha_w(shape, 1.5)
    wo = htucker.alpha_w(shape, htucker.balanced_tree(6), 1.5)
    assert w == wo
    _compare_ht(rt, X, 4, 2, w=w, seed=9)


def test_bad_trees_are_rejected(rt):
    X = torch.from_numpy(synth.inv_norm_tensor(4, 4)).cuda()
    lib = rt.load_library()
    import ctypes
    h = rt._handle(X.device.index)
    n = (ctypes.c_int64 * 4)(4, 4, 4, 4)
    rk = (ctypes.c_int32 * 7)(*([2] * 7))
    U = torch.empty(64, device="cuda")
    B = torch.empty(64, device="cuda")
    for tab in ([(1, 2), (3, 4), (5, 6), (-1, -1), (-1, -1), (-1, -1), (1, -1)],     # one child
                [(1, 2), (3, 4), (3, 6), (-1, -1), (-1, -1), (-1, -1), (-1, -1)],    # node 3 twice
                [(1, 2), (3, 4), (5, 0), (-1, -1), (-1, -1), (-1, -1), (-1, -1)],    # root as a child
                [(1, 2), (-1, -1), (-1, -1), (-1, -1), (-1, -1), (-1, -1), (-1, -1)]):  # too many leaves
        flat = (ctypes.c_int32 * 14)(*[v for lr in tab for v in lr])
        st = lib.rhtucker_decompose(h, ctypes.c_void_p(X.data_ptr()), 0, 4, n, flat, rk, 1, None,
                                    ctypes.c_uint64(1), None, ctypes.c_void_p(U.data_ptr()),
                                    ctypes.c_void_p(B.data_ptr()), None)
        assert st == 1, tab
