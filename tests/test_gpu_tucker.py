"""GPU parity of the Sub-R-HOSVD path (S1-S7) against the float64 oracle.

Every call goes through the C ABI (ctypes binding).  Bars: sampled indices
bit-exact; sketches within 1e-5 of max|Z|; factors equal up to column sign
within 1e-4 (well-separated columns element-wise, clusters of close singular
values through their projectors); |relerr_gpu - relerr_oracle| <= 1e-5.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import brute, rng, tucker  # noqa: E402
from parity_util import (RELERR_TOL, U_TOL, compare_factor, flip_core, orthonormality,  # noqa: E402
                         to_np)

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


def _run_and_compare(rt, X, r, p, s=None, seed=0, check_core=True, x_for_oracle=None, min_covered=None,
                     qr="auto"):
    """Decomposition through the C ABI against the oracle.  check_core: True compares
    G with the oracle's core (signs aligned); "projection" compares G element-wise
    with the float64 projection of X on the GPU's own factors, X x_k U_k^T, at 1e-5
    of max|G| (exact for the core kernels, indifferent to rotations inside clusters
    of close singular values).  min_covered: columns per mode that must be compared
    (default: all r_k)."""
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    G, U = rt.rtucker_decompose(Xd, list(r), p, s=s, seed=seed, qr=qr)
    rt.sync()          # raises if a kernel reported a device-side failure
    _, sig = rt.rtucker_factors(Xd, list(r), p, s=s, seed=seed, with_sigma=True, qr=qr)
    rt.sync()
    Xo = np.asarray(X if x_for_oracle is None else x_for_oracle, dtype=np.float64)
    ref = tucker.sub_r_hosvd(Xo, list(r), p, s=s, seed=seed, with_core=(check_core is True))
    signs = []
    for k in range(Xo.ndim):
        need = r[k] if min_covered is None else min_covered
        sg, dev, strict, covered = compare_factor(to_np(U[k]), ref["U"][k], ref["modes"][k]["sigma"],
                                                  min_covered=need)
        assert dev <= U_TOL, ("mode", k, dev)
        assert orthonormality(to_np(U[k])) < 1e-5
        s_ref = ref["modes"][k]["sigma"]
        assert np.abs(to_np(sig[k]) - s_ref).max() <= 1e-5 * s_ref[0] + 1e-30
        signs.append(sg)
    err_gpu = rt.rtucker_relerr(Xd, G, U)
    Gref = ref["G"] if check_core is True else tucker.multi_ttm_t(Xo, ref["U"])
    err_ref = tucker.relerr(Xo, tucker.reconstruct(Gref, ref["U"]))
    del Gref
    assert abs(err_gpu - err_ref) <= RELERR_TOL, (err_gpu, err_ref)
    if check_core is True:
        Gg = flip_core(to_np(G), signs)
        assert np.abs(Gg - ref["G"]).max() <= 1e-4 * np.abs(ref["G"]).max()
    elif check_core == "projection":
        Gp = tucker.multi_ttm_t(Xo, [to_np(u) for u in U])
        assert np.abs(to_np(G) - Gp).max() <= 1e-5 * np.abs(Gp).max(), np.abs(to_np(G) - Gp).max()
    return G, U, ref, err_gpu, err_ref


def test_indices_bit_exact(rt):
    for n, s, seed in [((128, 128, 128, 128), (1280,) * 4, 1),
                       ((64, 64, 64), (640, 640, 640), 0),
                       ((7, 5, 3), (15, 21, 35), 123456789),
                       ((2, 3), (3, 2), 2**63 + 5)]:
        got = rt.rtucker_indices(list(n), list(s), seed=seed)
        N = int(np.prod(n))
        for k in range(len(n)):
            want = rng.fiber_indices(N // n[k], s[k], seed, k)
            assert np.array_equal(got[k].cpu().numpy(), want), (n, k)


def test_sketch_matches_oracle(rt):
    X = synth.tucker_tensor((40, 36, 150), (4, 5, 6), noise=1e-4, data_seed=5, dtype="f32")
    Xd = torch.from_numpy(X).cuda()
    r, p, seed = [4, 5, 6], 3, 11
    Z = rt.rtucker_sketch(Xd, r, p, seed=seed)
    ref = tucker.sub_r_hosvd(X.astype(np.float64), r, p, seed=seed, with_core=False)
    for k in range(3):
        Zr = ref["modes"][k]["Z"]
        assert np.abs(to_np(Z[k]) - Zr).max() <= 1e-5 * np.abs(Zr).max()


def test_small_order3_ragged_tiles(rt):
    X = synth.tucker_tensor((40, 36, 150), (4, 5, 6), noise=1e-4, data_seed=5, dtype="f32")
    _run_and_compare(rt, X, (4, 5, 6), 3, seed=11)


def test_order4_ragged(rt):
    X = synth.tucker_tensor((33, 29, 17, 70), (5, 4, 3, 7), noise=1e-5, data_seed=6, dtype="f32")
    _run_and_compare(rt, X, (5, 4, 3, 7), 4, seed=3)


def test_order3_float64_storage_64cube(rt):
    cfg = synth.ORDER3_F64
    X = synth.named(cfg)
    assert X.dtype == np.float64
    _, _, _, eg, er = _run_and_compare(rt, X, cfg["ranks"], cfg["p"], seed=cfg["seed"])
    assert er < 1e-6


def test_order4_graded_core_reduced(rt):
    X = synth.tucker_tensor((48, 48, 48, 48), (12, 12, 12, 12), noise=1e-6, data_seed=7, core="graded")
    _run_and_compare(rt, X, (12,) * 4, 6, seed=2)


def test_matrix_d2(rt):
    X = synth.tucker_tensor((300, 200), (10, 10), noise=1e-3, data_seed=8)
    _run_and_compare(rt, X, (10, 10), 5, seed=4, min_covered=9)   # sigma_10, sigma_11 closer than 1e-3 sigma_1


@pytest.mark.parametrize("shape,data_seed,s", [((70, 48, 48), 10, None), ((20000, 18, 18), 42, None),
                                                ((120, 90, 90), 65, [8000, 900, 900])])
def test_widest_sketch(rt, shape, data_seed, s):
    # r + p = 64, the largest supported width.  70 rows: one QR block, B^T formed and
    # factored in one kernel.  20000 rows: 125 row blocks of 160, so the TSQR of Z
    # runs a three-level tree (fan-in 5) with two combine passes, and B^T is reduced
    # over 40 row blocks before each 256-sample chunk is factored.  8000 samples: 32
    # chunk factors, more than the W-step stacks (5), reduced by a two-level R tree
    # (32 -> 7 -> 2) first.  The 54 sampled singular values sit ~1e-3 of sigma_1
    # apart, so columns closer than 5e-3 are compared as subspaces and the core is
    # checked as the projection of X on the returned factors.
    X = synth.tucker_tensor(shape, (54, 8, 8), noise=1e-4, data_seed=data_seed)
    r, p, seed = [54, 8, 8], 10, 12
    Xd = torch.from_numpy(X).cuda()
    G, U = rt.rtucker_decompose(Xd, r, p, s=s, seed=seed)
    _, sig = rt.rtucker_factors(Xd, r, p, s=s, seed=seed, with_sigma=True)
    rt.sync()
    Xo = X.astype(np.float64)
    ref = tucker.sub_r_hosvd(Xo, r, p, s=s, seed=seed, with_core=False)
    Un = [to_np(u) for u in U]
    for k in range(3):
        s_ref = ref["modes"][k]["sigma"]
        _, dev, _, _ = compare_factor(Un[k], ref["U"][k], s_ref, gap_min=5e-3)
        assert dev <= U_TOL, ("mode", k, dev)
        assert orthonormality(Un[k]) < 1e-5
        assert np.abs(to_np(sig[k]) - s_ref).max() <= 1e-5 * s_ref[0]
    Gp = tucker.multi_ttm_t(Xo, Un)
    assert np.abs(to_np(G) - Gp).max() <= 1e-5 * np.abs(Gp).max()
    er = tucker.relerr(Xo, tucker.reconstruct(tucker.multi_ttm_t(Xo, ref["U"]), ref["U"]))
    assert abs(rt.rtucker_relerr(Xd, G, U) - er) <= RELERR_TOL


def test_rp_equals_n_and_p_zero(rt):
    X = synth.tucker_tensor((8, 30, 25), (5, 6, 6), noise=1e-3, data_seed=9)
    _run_and_compare(rt, X, (5, 6, 6), 3, seed=5)       # r_0 + p = n_0
    _run_and_compare(rt, X, (5, 6, 6), 0, seed=6)       # no oversampling


def test_full_sampling_is_truncated_hosvd(rt):
    rs = np.random.default_rng(6)
    X = rs.standard_normal((6, 7, 8)).astype(np.float32)
    r, p = [2, 3, 4], 4
    s = [56, 48, 42]
    G, U, ref, _, _ = _run_and_compare(rt, X, r, p, s=s, seed=3)
    hs = brute.t_hosvd(X.astype(np.float64), r)
    for k in range(3):
        Ug = to_np(U[k])
        sg = np.sign((Ug * hs["U"][k]).sum(axis=0))
        assert np.abs(Ug * sg - hs["U"][k]).max() <= U_TOL


def test_tall_mode_uses_tsqr(rt):
    X = synth.tucker_tensor((3000, 8, 9), (6, 3, 3), noise=1e-4, data_seed=10)
    _run_and_compare(rt, X, (6, 3, 3), 2, seed=8)


def test_bf16_storage(rt):
    X = synth.tucker_tensor((40, 50, 60), (5, 5, 5), noise=1e-3, data_seed=11)
    Xb = torch.from_numpy(X).to(torch.bfloat16)
    Xo = Xb.float().numpy()  # the oracle sees the same (rounded) values
    Xd = Xb.cuda()
    G, U = rt.rtucker_decompose(Xd, [5, 5, 5], 3, seed=9)
    ref = tucker.sub_r_hosvd(Xo.astype(np.float64), [5, 5, 5], 3, seed=9)
    for k in range(3):
        _, dev, _, _ = compare_factor(to_np(U[k]), ref["U"][k], ref["modes"][k]["sigma"])
        assert dev <= U_TOL
    eg = rt.rtucker_relerr(Xd, G, U)
    er = tucker.relerr(Xo, tucker.reconstruct(ref["G"], ref["U"]))
    assert abs(eg - er) <= RELERR_TOL


def test_bf16_compute_form(rt):
    # float32 X rounded to one bfloat16 term in the tensor-core pass (factors keep two
    # terms): the factors are those of the float32 form (the range finder is float32)
    # and the relative error still meets the float32 criterion against the oracle
    X = synth.tucker_tensor((48, 40, 64, 32), (6, 5, 8, 8), noise=1e-3, data_seed=13)
    Xd = torch.from_numpy(X).cuda()
    r, p, seed = [6, 5, 8, 8], 4, 21
    G32, U32 = rt.rtucker_decompose(Xd, r, p, seed=seed, core="tc")
    G16, U16 = rt.rtucker_decompose(Xd, r, p, seed=seed, prec="bf16", core="tc")
    for a, b in zip(U32, U16):
        assert torch.equal(a, b)
    ref = tucker.sub_r_hosvd(X.astype(np.float64), r, p, seed=seed)
    er = tucker.relerr(X.astype(np.float64), tucker.reconstruct(ref["G"], ref["U"]))
    e16 = rt.rtucker_relerr(Xd, G16, U16)
    assert abs(e16 - er) <= RELERR_TOL, (e16, er)
    # the bf16 rounding of X is visible in G, at the level of its 2^-9 relative step
    dg = (G16 - G32).abs().max().item() / G32.abs().max().item()
    assert 0 < dg < 4e-3
    # the core entry point (pass over X on the final factors) and the decomposition
    # (pass on the QR factors, then the W contractions) round differently
    Gc = rt.rtucker_core(Xd, U32, prec="bf16", core="tc")
    assert (Gc - G16).abs().max().item() <= 2e-5 * G16.abs().max().item()


@pytest.mark.parametrize("shape,ranks", [((6, 40, 96, 64), (4, 6, 12, 16)), ((5, 9, 33, 16), (3, 4, 7, 5))])
def test_bf16_storage_tensor_core_pass(rt, shape, ranks):
    # bfloat16 X through the tensor-core pass (MMA1 reads X from the TMA stage) must
    # give the core of its exact float32 copy (whose lo terms are then zero); the
    # second shape has an odd slab height (33 rows of the 128-row MMA tile)
    rs = np.random.default_rng(14)
    Xb = torch.from_numpy(rs.standard_normal(shape).astype(np.float32)).to(torch.bfloat16).cuda()
    U = [np.linalg.qr(rs.standard_normal((n, k)))[0].astype(np.float32) for n, k in zip(shape, ranks)]
    Ud = [torch.from_numpy(u).cuda() for u in U]
    Gb = rt.rtucker_core(Xb, Ud, core="tc")
    Gf = rt.rtucker_core(Xb.float(), Ud, core="tc")
    Gr = tucker.multi_ttm_t(Xb.float().cpu().numpy().astype(np.float64), [u.astype(np.float64) for u in U])
    scale = np.abs(Gr).max()
    assert np.abs(to_np(Gf) - Gr).max() <= 1e-5 * scale
    assert np.abs(to_np(Gb) - Gr).max() <= 1e-5 * scale


def test_core_entry_point_and_evaluator(rt):
    X = synth.tucker_tensor((30, 40, 50), (4, 4, 4), noise=1e-3, data_seed=12)
    Xd = torch.from_numpy(X).cuda()
    rs = np.random.default_rng(1)
    U = [np.linalg.qr(rs.standard_normal((n, 4)))[0] for n in X.shape]
    Ud = [torch.from_numpy(u.astype(np.float32)).cuda() for u in U]
    G = rt.rtucker_core(Xd, Ud)
    Uf = [u.astype(np.float32).astype(np.float64) for u in U]
    Gr = tucker.multi_ttm_t(X.astype(np.float64), Uf)
    assert np.abs(to_np(G) - Gr).max() <= 1e-5 * np.abs(Gr).max()
    # evaluator against a host float64 reconstruction of the same G, U
    eg = rt.rtucker_relerr(Xd, G, Ud)
    eh = tucker.relerr(X, tucker.reconstruct(to_np(G), Uf))
    assert abs(eg - eh) <= 1e-9


@pytest.mark.parametrize("shape,ranks", [((300, 20000), (5, 12)), ((30, 40, 8000), (3, 4, 5))])
def test_evaluator_general_form(rt, shape, ranks):
    # r_{d-2} n_{d-1} doubles above 200 KB: mode d-2 expanded as well, then rows of
    # n_{d-1} against U_{d-1}; against a host float64 reconstruction of the same G, U
    rs = np.random.default_rng(len(shape))
    X = rs.standard_normal(shape).astype(np.float32)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [(rs.standard_normal((n, k)) / np.sqrt(n)).astype(np.float32) for n, k in zip(shape, ranks)]
    eg = rt.rtucker_relerr(torch.from_numpy(X).cuda(), torch.from_numpy(G).cuda(), [torch.from_numpy(u).cuda() for u in U])
    eh = tucker.relerr(X.astype(np.float64), tucker.reconstruct(G.astype(np.float64), [u.astype(np.float64) for u in U]))
    assert abs(eg - eh) <= 1e-9, (eg, eh)


def test_core_tensor_core_pass_odd_slab_height(rt):
    # float32 X, slabs of 33 x 12: odd n_{d-1} on the tensor-core pass, r = 5 and 7
    rs = np.random.default_rng(15)
    shape, ranks = (7, 6, 33, 12), (3, 4, 5, 7)
    X = rs.standard_normal(shape).astype(np.float32)
    U = [np.linalg.qr(rs.standard_normal((n, k)))[0].astype(np.float32) for n, k in zip(shape, ranks)]
    G = rt.rtucker_core(torch.from_numpy(X).cuda(), [torch.from_numpy(u).cuda() for u in U], core="tc")
    Gr = tucker.multi_ttm_t(X.astype(np.float64), [u.astype(np.float64) for u in U])
    assert np.abs(to_np(G) - Gr).max() <= 1e-5 * np.abs(Gr).max()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_core_tensor_core_pass_ranks_up_to_64(rt, dtype):
    # the tensor-core pass with r_{d-1} = 50 (M = 64 accumulator rows) and r_d = 60
    # (64-column T, one D2 buffer reused over many batches, four X stages)
    rs = np.random.default_rng(16)
    shape, ranks = (40, 40, 100, 96), (3, 4, 50, 60)
    X = rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    if dtype == "bf16":
        Xd = Xd.to(torch.bfloat16)
        X = Xd.float().cpu().numpy()
    U = [np.linalg.qr(rs.standard_normal((n, k)))[0].astype(np.float32) for n, k in zip(shape, ranks)]
    G = rt.rtucker_core(Xd, [torch.from_numpy(u).cuda() for u in U], core="tc")
    rt.sync()
    Gr = tucker.multi_ttm_t(X.astype(np.float64), [u.astype(np.float64) for u in U])
    assert np.abs(to_np(G) - Gr).max() <= 1e-5 * np.abs(Gr).max()


def test_core_wide_rho_ragged_tiles(rt):
    # order 4: the tensor-core pass contracts modes 3, 4 (P has 12*12 = 144 trailing
    # entries per slab), then the tensor-core one-mode contraction runs twice with ragged
    # 128-column tiles (144 and 7*144 = 1008), K below 128 (45, 37) and 5 and 7 rows of U
    rs = np.random.default_rng(5)
    shape, ranks = (37, 45, 24, 20), (5, 7, 12, 12)
    X = rs.standard_normal(shape).astype(np.float32)
    U = [np.linalg.qr(rs.standard_normal((n, k)))[0] for n, k in zip(shape, ranks)]
    Ud = [torch.from_numpy(u.astype(np.float32)).cuda() for u in U]
    G = rt.rtucker_core(torch.from_numpy(X).cuda(), Ud, core="tc")
    Uf = [u.astype(np.float32).astype(np.float64) for u in U]
    Gr = tucker.multi_ttm_t(X.astype(np.float64), Uf)
    assert G.shape == tuple(ranks)
    assert np.abs(to_np(G) - Gr).max() <= 1e-4 * np.abs(Gr).max()


@pytest.mark.parametrize("shape,ranks", [
    ((20, 128, 64, 64), (50, 64, 8, 8)),        # tensor-core contractions: n = 128 and r = 64
                                                # (four TMEM lane quadrants), then n = 20, r = 50
    ((150, 72, 64, 64), (9, 33, 6, 10)),        # n = 72 on the tensor cores, then n = 150 > 128:
                                                # the FFMA contraction for the last one
])
def test_core_tensor_core_contraction_shapes(rt, shape, ranks):
    rs = np.random.default_rng(sum(shape))
    X = rs.standard_normal(shape).astype(np.float32)
    U = [np.linalg.qr(rs.standard_normal((n, k)))[0].astype(np.float32) for n, k in zip(shape, ranks)]
    G = rt.rtucker_core(torch.from_numpy(X).cuda(), [torch.from_numpy(u).cuda() for u in U], core="tc")
    rt.sync()
    Gr = tucker.multi_ttm_t(X.astype(np.float64), [u.astype(np.float64) for u in U])
    assert np.abs(to_np(G) - Gr).max() <= 1e-5 * np.abs(Gr).max()


@pytest.mark.parametrize("shape,ranks,dtype", [
    ((7, 6, 33, 12), (3, 4, 5, 7), "f32"),      # two two-mode passes (R = 1, then R = 35)
    ((3,) * 8, (2,) * 8, "f32"),                 # four two-mode passes
    ((5, 6, 7), (2, 3, 4), "f64"),               # two-mode pass on float64 X, then one mode
    ((9, 10, 11, 13), (4, 5, 6, 7), "bf16"),     # bfloat16 X
    ((4, 5, 150, 90), (3, 3, 9, 8), "f32"),      # slab 150 x 90 > shared memory: one-mode chain
])
def test_core_two_mode_ffma_passes(rt, shape, ranks, dtype):
    # small slabs take k_slab2 (two modes per read); its results against the float64
    # definition for every kernel choice
    rs = np.random.default_rng(sum(shape))
    X = rs.standard_normal(shape)
    Xd = torch.from_numpy(X).cuda()
    Xd = Xd.to({"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[dtype])
    Xo = Xd.double().cpu().numpy()
    U = [np.linalg.qr(rs.standard_normal((n, k)))[0].astype(np.float32) for n, k in zip(shape, ranks)]
    Ud = [torch.from_numpy(u).cuda() for u in U]
    Gr = tucker.multi_ttm_t(Xo, [u.astype(np.float64) for u in U])
    for core in ("auto", "ffma", "tc"):
        G = rt.rtucker_core(Xd, Ud, core=core)
        rt.sync()
        assert np.abs(to_np(G) - Gr).max() <= 1e-5 * np.abs(Gr).max(), core


@pytest.mark.parametrize("shape,ranks", [((7, 6, 33, 12), (3, 4, 5, 7)), ((6, 40, 96, 64), (4, 6, 12, 16))])
def test_core_tuned_choice(rt, shape, ranks):
    # core="tune" times the tensor-core pass and the FFMA kernels on the first call for
    # a shape and keeps the faster: its core is bit-identical to one of the two, on the
    # core entry point and inside a decomposition, and stays so on later calls
    rs = np.random.default_rng(sum(shape) + 1)
    X = synth.tucker_tensor(shape, ranks, 1e-3, 77)
    Xd = torch.from_numpy(X).cuda()
    U = [torch.from_numpy(np.linalg.qr(rs.standard_normal((n, k)))[0].astype(np.float32)).cuda()
         for n, k in zip(shape, ranks)]
    fixed = [rt.rtucker_core(Xd, U, core=c) for c in ("tc", "ffma")]
    for _ in range(2):
        Gt = rt.rtucker_core(Xd, U, core="tune")
        rt.sync()
        assert any(torch.equal(Gt, f) for f in fixed)
    p = 2
    dec = [rt.rtucker_decompose(Xd, list(ranks), p, seed=5, core=c)[0] for c in ("tc", "ffma")]
    for _ in range(2):
        Gd, _ = rt.rtucker_decompose(Xd, list(ranks), p, seed=5, core="tune")
        rt.sync()
        assert any(torch.equal(Gd, f) for f in dec)


def test_invalid_arguments_raise(rt):
    X = torch.zeros((4, 5, 6), device="cuda")
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_decompose(X, [4, 2, 2], 1)       # r_0 + p > n_0
    assert e.value.status == 1
    with pytest.raises(rt.RtError):
        rt.rtucker_decompose(X, [2, 2, 2], 1, s=[2, 20, 20])  # s < r + p
    with pytest.raises(rt.RtError):
        rt.rtucker_decompose(X, [2, 2, 2], 1, s=[31, 20, 20])  # s > n_{!=k}
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_decompose(X, [2, 2, 2], 70)     # r + p > 64
    assert e.value.status in (1, 7)


def test_order_16_the_largest_supported(rt):
    # d = 16: every per-problem mode array is full; ragged last modes (3, 4) keep the
    # core on the FFMA chain
    X = synth.tucker_tensor((2,) * 14 + (3, 4), (1,) * 16, noise=1e-3, data_seed=40)
    _run_and_compare(rt, X, (1,) * 16, 1, seed=3)


def test_degenerate_shapes_are_rejected(rt):
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_decompose(torch.zeros((4, 0, 6), device="cuda"), [1, 1, 1], 0)   # empty mode
    assert e.value.status == 1
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_decompose(torch.zeros((1,) * 17, device="cuda"), [1] * 17, 0)    # d > 16
    assert e.value.status == 1
    with pytest.raises((rt.RtError, ValueError)):
        rt.rtucker_decompose(torch.zeros((8,), device="cuda"), [1], 0)              # d < 2
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_decompose(torch.zeros((4, 5, 6), device="cuda"), [0, 1, 1], 1)   # r_k = 0
    assert e.value.status == 1


def test_host_memory_entry_point(rt):
    X = synth.tucker_tensor((40, 36, 50), (4, 5, 6), noise=1e-4, data_seed=13)
    Xh = torch.from_numpy(X).pin_memory()
    G, U = rt.rtucker_decompose_host(Xh, [4, 5, 6], 3, seed=2)
    Gd, Ud = rt.rtucker_decompose(Xh.cuda(), [4, 5, 6], 3, seed=2)
    torch.cuda.synchronize()
    assert np.array_equal(G.numpy(), Gd.cpu().numpy())
    for a, b in zip(U, Ud):
        assert np.array_equal(a.numpy(), b.cpu().numpy())


def test_pipelined_host_entry_point(rt):
    # a stream of tensors (two shapes, so the device slots grow once; one
    # pageable input) through the pipelined host call: each result equals the
    # synchronous device call on the same tensor
    shapes = [(40, 36, 50), (40, 36, 50), (64, 48, 40), (40, 36, 50), (64, 48, 40)]
    ranks = [4, 5, 6]
    Xs = [torch.from_numpy(synth.tucker_tensor(sh, ranks, 1e-4, 300 + i)) for i, sh in enumerate(shapes)]
    Xs = [x.pin_memory() if i != 3 else x for i, x in enumerate(Xs)]
    outs = [rt.rtucker_decompose_host_async(x, ranks, 3, seed=10 + i) for i, x in enumerate(Xs)]
    rt.sync()
    for i, (x, (G, U)) in enumerate(zip(Xs, outs)):
        Gd, Ud = rt.rtucker_decompose(x.cuda(), ranks, 3, seed=10 + i)
        torch.cuda.synchronize()
        assert np.array_equal(G.numpy(), Gd.cpu().numpy()), i
        for a, b in zip(U, Ud):
            assert np.array_equal(a.numpy(), b.cpu().numpy()), i
    # an argument error leaves the pipeline usable
    with pytest.raises(rt.RtError):
        rt.rtucker_decompose_host_async(Xs[0], ranks, 70)
    G, U = rt.rtucker_decompose_host_async(Xs[1], ranks, 3, seed=11)
    rt.sync()
    assert np.array_equal(G.numpy(), outs[1][0].numpy())


def test_batched_matches_single_and_oracle(rt):
    shapes, ranks = synth.batched_shapes(T=12, data_seed=55)
    Xs = [synth.tucker_tensor(sh, rk, 1e-6, 9000 + t) for t, (sh, rk) in enumerate(zip(shapes, ranks))]
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    seeds = [100 + t for t in range(12)]
    outs = rt.rtucker_decompose_batched(Xd, [list(r) for r in ranks], 5, seeds)
    torch.cuda.synchronize()
    for t in range(12):
        G1, U1 = rt.rtucker_decompose(Xd[t], list(ranks[t]), 5, seed=seeds[t])
        Gb, Ub = outs[t]
        # same range finder (grouped) -> identical factors; the core takes the grouped
        # FFMA contractions in the batch and per-shape kernels alone
        for k in range(3):
            assert torch.equal(Ub[k], U1[k])
        assert np.abs(to_np(Gb) - to_np(G1)).max() <= 1e-5 * np.abs(to_np(G1)).max()
        ref = tucker.sub_r_hosvd(Xs[t].astype(np.float64), list(ranks[t]), 5, seed=seeds[t])
        for k in range(3):
            _, dev, _, _ = compare_factor(to_np(Ub[k]), ref["U"][k], ref["modes"][k]["sigma"])
            assert dev <= U_TOL
        eg = rt.rtucker_relerr(Xd[t], Gb, Ub)
        er = tucker.relerr(Xs[t], tucker.reconstruct(ref["G"], ref["U"]))
        assert abs(eg - er) <= RELERR_TOL


def test_batched_full_size_256(rt):
    # the batch the benchmark times (256 order-3 tensors, n_k ~ U{32..160}, one grouped
    # call): every 32nd tensor against the oracle (factors as subspaces where sampled
    # singular values sit within 5e-3 of sigma_1, the error of the format), and every
    # factor of the batch orthonormal
    cfg = synth.BATCHED_256
    Xh, shapes, ranks = synth.batched_tensors(cfg["T"], cfg["nmin"], cfg["nmax"], cfg["rmin"], cfg["rmax"],
                                              cfg["noise"], cfg["data_seed"])
    Xd = [torch.from_numpy(x).cuda() for x in Xh]
    seeds = [cfg["seed"] + t for t in range(cfg["T"])]
    outs = rt.BatchedDecomposition(Xd, ranks, cfg["p"], seeds).run().results()
    rt.sync()
    for t in range(cfg["T"]):
        for u in outs[t][1]:
            assert orthonormality(to_np(u)) < 1e-5, t
    for t in range(0, cfg["T"], 32):
        Gb, Ub = outs[t]
        ref = tucker.sub_r_hosvd(Xh[t].astype(np.float64), list(ranks[t]), cfg["p"], seed=seeds[t])
        for k in range(3):
            _, dev, _, _ = compare_factor(to_np(Ub[k]), ref["U"][k], ref["modes"][k]["sigma"], gap_min=5e-3)
            assert dev <= U_TOL, (t, k, dev)
        eg = rt.rtucker_relerr(Xd[t], Gb, Ub)
        er = tucker.relerr(Xh[t].astype(np.float64), tucker.reconstruct(ref["G"], ref["U"]))
        assert abs(eg - er) <= RELERR_TOL, (t, eg, er)


@pytest.mark.parametrize("shape,r,p", [((40, 36, 48, 64), (6, 5, 12, 20), 4), ((128, 128, 128, 128), None, None)])
def test_overlapped_core_schedule(rt, shape, r, p):
    # the pass over X on the QR factors beside the SVD part of the range finder,
    # then the W contractions: same factors (bit for bit) and the same core up to
    # rounding as the default schedule; parity with the oracle through the relerr
    if r is None:
        cfg = synth.ORDER4_128
        X = synth.named(cfg)
        r, p, seed = list(cfg["ranks"]), cfg["p"], cfg["seed"]
    else:
        X = synth.tucker_tensor(shape, r, noise=1e-3, data_seed=17)
        r, seed = list(r), 23
    Xd = torch.from_numpy(X).cuda()
    G0, U0 = rt.rtucker_decompose(Xd, r, p, seed=seed)
    G1, U1 = rt.rtucker_decompose(Xd, r, p, seed=seed, overlap=True)
    rt.sync()
    for a, b in zip(U0, U1):
        assert torch.equal(a, b)
    assert (G1 - G0).abs().max().item() <= 2e-5 * G0.abs().max().item()
    ref = tucker.sub_r_hosvd(X.astype(np.float64), r, p, seed=seed, with_core=False)
    er = tucker.relerr(X.astype(np.float64),
                       tucker.reconstruct(tucker.multi_ttm_t(X.astype(np.float64), ref["U"]), ref["U"]))
    assert abs(rt.rtucker_relerr(Xd, G1, U1) - er) <= RELERR_TOL


def test_order4_96_full_size(rt):
    cfg = synth.ORDER4_96
    X = synth.named(cfg)
    _run_and_compare(rt, X, cfg["ranks"], cfg["p"], seed=cfg["seed"], check_core="projection")


def _bf16_core_bound(Xo, U):
    """Element-wise bound on the core error of the BF16 compute form, which rounds
    float32 X to one bfloat16 term (unit roundoff 2^-8) and keeps the factors as two
    terms (2^-16) with float32 accumulation: |dG| <= (2^-8 + 2^-15) (|X| x_k |U_k|^T)."""
    A = tucker.multi_ttm_t(np.abs(Xo), [np.abs(u) for u in U])
    return (2.0 ** -8 + 2.0 ** -15) * A


def test_order4_128_full_size(rt):
    # the benchmark's workload and launch configuration: every column of every factor
    # compared (the 32 sampled singular values are separated), the core G of the
    # tensor-core pass compared element-wise with the float64 projection on its factors
    cfg = synth.ORDER4_128
    X = synth.named(cfg)
    G, U, ref, eg, er = _run_and_compare(rt, X, cfg["ranks"], cfg["p"], seed=cfg["seed"],
                                         check_core="projection")
    assert 5e-4 < er < 5e-3
    del G, U
    # BF16 compute form on the same tensor meets the same relerr criterion; its core is
    # the projection on its own factors within the rounding bound of one bfloat16 term
    Xd = torch.from_numpy(X).cuda()
    G16, U16 = rt.rtucker_decompose(Xd, cfg["ranks"], cfg["p"], seed=cfg["seed"], prec="bf16")
    assert abs(rt.rtucker_relerr(Xd, G16, U16) - er) <= RELERR_TOL
    Xo = np.asarray(X, dtype=np.float64)
    U16n = [to_np(u) for u in U16]
    dG = np.abs(to_np(G16) - tucker.multi_ttm_t(Xo, U16n))
    bound = _bf16_core_bound(Xo, U16n)
    assert (dG <= bound).all(), float((dG / bound).max())
    del G16, U16, dG, bound
    # bfloat16-stored X: the factors are fitted to the rounded data, which moves the
    # error against the float32 X well beyond 1e-5 on this tensor (the rounding, 1.7e-3
    # relative, is above the noise under the smallest kept directions); parity is with
    # the oracle run on the same rounded tensor, both measured against the float32 X
    Xb = Xd.to(torch.bfloat16)
    Gb, Ub = rt.rtucker_decompose(Xb, cfg["ranks"], cfg["p"], seed=cfg["seed"])
    eb = rt.rtucker_relerr(Xd, Gb, Ub)
    Xbo = Xb.float().cpu().numpy().astype(np.float64)
    refb = tucker.sub_r_hosvd(Xbo, cfg["ranks"], cfg["p"], seed=cfg["seed"])
    Gbp = tucker.multi_ttm_t(Xbo, [to_np(u) for u in Ub])
    assert np.abs(to_np(Gb) - Gbp).max() <= 1e-5 * np.abs(Gbp).max()
    del Xbo, Gbp
    ebr = tucker.relerr(Xo, tucker.reconstruct(refb["G"], refb["U"]))
    assert abs(eb - ebr) <= RELERR_TOL, (eb, ebr)


def test_decompositions_in_flight_on_several_streams(rt):
    # the benchmark's timed run: decompositions of the 128^4 workload on four CUDA
    # streams at once (one library handle, input copy and output per stream, graph
    # replay), round robin; every result equals the one-at-a-time result bit for bit,
    # and that result is the oracle's (test_order4_128_full_size)
    cfg = synth.ORDER4_128
    X = torch.from_numpy(synth.named(cfg)).cuda()
    r, p, seed = list(cfg["ranks"]), cfg["p"], cfg["seed"]
    n = list(X.shape)
    nu = sum(a * b for a, b in zip(n, r))
    G0, U0 = rt.rtucker_decompose(X, r, p, seed=seed)
    U0 = torch.cat([u.reshape(-1) for u in U0])
    P = 4
    streams = [torch.cuda.Stream() for _ in range(P)]
    Xs = [X.clone() for _ in range(P)]
    outs = [(torch.empty(nu, device="cuda"), torch.empty(r, device="cuda")) for _ in range(P)]
    torch.cuda.synchronize()
    for i in range(3 * P):
        k = i % P
        with torch.cuda.stream(streams[k]):
            rt.rtucker_decompose(Xs[k], r, p, seed=seed, out=outs[k], graph=True)
    torch.cuda.synchronize()
    for k in range(P):
        with torch.cuda.stream(streams[k]):
            rt.sync()
        assert torch.equal(outs[k][0], U0) and torch.equal(outs[k][1], G0), k


def test_repeated_calls_reuse_tables_safely(rt):
    # identical calls may skip re-uploading the problem tables; any other use of the
    # workspace in between (another decomposition, a core or gradient call) must not
    # leave stale tables behind
    X = synth.tucker_tensor((48, 40, 56), (5, 4, 6), 1e-4, 21)
    Xd = torch.from_numpy(X).cuda()
    r = [5, 4, 6]
    G0, U0 = rt.rtucker_decompose(Xd, r, 3, seed=7)
    G1, U1 = rt.rtucker_decompose(Xd, r, 3, seed=7)           # same tables
    Gs, _ = rt.rtucker_decompose(Xd, r, 3, seed=8)            # other seed: other tables
    G2, U2 = rt.rtucker_decompose(Xd, r, 3, seed=7)
    Y = torch.from_numpy(synth.tucker_tensor((30, 33, 31), (3, 3, 3), 1e-4, 22)).cuda()
    rt.rtucker_core(Y, [u[:m, :3].contiguous() for u, m in zip(U0, (30, 33, 31))])
    rt.rtucker_loss_grad(Xd, G0, U0)
    G3, U3 = rt.rtucker_decompose(Xd, r, 3, seed=7)
    rt.sync()
    for G, U in ((G1, U1), (G2, U2), (G3, U3)):
        assert torch.equal(G, G0)
        for a, b in zip(U, U0):
            assert torch.equal(a, b)
    assert not torch.equal(Gs, G0)


def _clone(G, U):
    return G.clone(), [u.clone() for u in U]


def _same(a, b):
    assert torch.equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("overlap", [False, True])
def test_graph_replay_matches_direct_launches(rt, overlap):
    # rt_options.use_graph: the first call captures the kernel sequence, later calls
    # with the same buffers and shapes replay it; each call still uploads its own
    # tables, so another seed or new contents of X give that call's result.  Same
    # kernels, same launch shapes: bit-identical to direct launches.
    shape, r, p = (40, 36, 64), [5, 4, 6], 3
    Xd = torch.from_numpy(synth.tucker_tensor(shape, tuple(r), 1e-4, 23)).cuda()
    out = (torch.empty(sum(n * k for n, k in zip(shape, r)), device="cuda"), torch.empty(r, device="cuda"))
    direct = {sd: _clone(*rt.rtucker_decompose(Xd, r, p, seed=sd, overlap=overlap)) for sd in (7, 8)}
    g1 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=7, out=out, overlap=overlap, graph=True))   # capture
    g2 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=7, out=out, overlap=overlap, graph=True))   # replay
    g3 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=8, out=out, overlap=overlap, graph=True))   # other tables
    rt.sync()
    _same(g1, direct[7])
    _same(g2, direct[7])
    _same(g3, direct[8])
    # new contents of X, replayed; then another shape (captured anew) and back
    Xd.copy_(torch.from_numpy(synth.tucker_tensor(shape, tuple(r), 1e-4, 24)).cuda())
    d2 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=7, overlap=overlap))
    g4 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=7, out=out, overlap=overlap, graph=True))
    Y = torch.from_numpy(synth.tucker_tensor((30, 33, 31), (3, 3, 3), 1e-4, 25)).cuda()
    dy = _clone(*rt.rtucker_decompose(Y, [3, 3, 3], 2, seed=1))
    gy = _clone(*rt.rtucker_decompose(Y, [3, 3, 3], 2, seed=1, graph=True))
    g5 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=7, out=out, overlap=overlap, graph=True))
    rt.sync()
    _same(g4, d2)
    _same(gy, dy)
    _same(g5, d2)
    # stage timing turns capture off; the result is the same
    rt.set_timing(True)
    g6 = _clone(*rt.rtucker_decompose(Xd, r, p, seed=7, out=out, overlap=overlap, graph=True))
    rt.sync()
    rt.get_timing(reset=True)
    rt.set_timing(False)
    _same(g6, d2)


def test_batched_tuned_schedules(rt):
    # rt_options.core = 3 on a batch: each contraction level's schedule picked by timing
    # (grouped tiles or one row per lane with 1..16 row blocks per CTA), cached per set of
    # shapes; the cores equal the default schedules' to rounding (the row form with any
    # block count is bit-identical, the tiles sum in another order)
    shapes, ranks = synth.batched_shapes(T=24, data_seed=57)
    Xs = [torch.from_numpy(synth.tucker_tensor(s, r, 1e-4, 60 + i)).cuda() for i, (s, r) in enumerate(zip(shapes, ranks))]
    seeds = list(range(24))
    ref = rt.BatchedDecomposition(Xs, [list(r) for r in ranks], 3, seeds).run()
    want = _clone_all(ref.results())
    assert ref.schedule() == [8, 0, 0]          # defaults: rows (8 blocks) for the last mode, tiles after
    bt = rt.BatchedDecomposition(Xs, [list(r) for r in ranks], 3, seeds, core="tune")
    for _ in range(2):                          # tuned, then the cached choice
        got = bt.run().results()
        rt.sync()
        sch = bt.schedule()
        assert len(sch) == 3 and sch[0] in (0, 1, 2, 4, 8, 16) and sch[1] == 0 and sch[2] == 0
        for (Ga, Ua), (Gb, Ub) in zip(got, want):
            assert torch.allclose(Ga, Gb, rtol=1e-5, atol=1e-5 * float(Gb.abs().max()))
            for a, b in zip(Ua, Ub):
                assert torch.equal(a, b)


def _clone_all(res):
    return [(G.clone(), [u.clone() for u in U]) for G, U in res]


def test_graph_replay_batched(rt):
    shapes = [(20, 24, 28), (33, 17, 40), (16, 16, 16, 16)]
    ranks = [(3, 4, 5), (4, 3, 6), (3, 3, 3, 3)]
    Xs = [torch.from_numpy(synth.tucker_tensor(s, k, 1e-4, 30 + i)).cuda() for i, (s, k) in enumerate(zip(shapes, ranks))]
    direct = rt.BatchedDecomposition(Xs, ranks, 3, [5, 6, 7]).run().results()
    want = [_clone(G, U) for G, U in direct]
    bd = rt.BatchedDecomposition(Xs, ranks, 3, [5, 6, 7], graph=True)
    for _ in range(3):                       # capture, then replays
        got = bd.run().results()
        rt.sync()
        for a, b in zip(got, want):
            _same(a, b)


# ----------------------------------------------------------------- factorisation forms (rt_options.qr)
_QR_CASES = {
    "small": lambda: (synth.tucker_tensor((40, 36, 150), (4, 5, 6), noise=1e-4, data_seed=5, dtype="f32"),
                      (4, 5, 6), 3, 11),
    "graded48": lambda: (synth.tucker_tensor((48, 48, 48, 48), (12, 12, 12, 12), noise=1e-6, data_seed=7,
                                             core="graded"), (12,) * 4, 6, 2),
    "widest70": lambda: (synth.tucker_tensor((70, 48, 48), (54, 8, 8), noise=1e-4, data_seed=10), (54, 8, 8), 10, 12),
    "tall": lambda: (synth.tucker_tensor((3000, 8, 9), (6, 3, 3), noise=1e-4, data_seed=10), (6, 3, 3), 2, 8),
    "illcond": lambda: _illconditioned(),
}


def _illconditioned():
    # sum of 10 rank-1 terms with weights 10^(-0.6 j): every unfolding has singular
    # values 1 ... 10^-5.4, so the sketch Z (r + p = 10 columns) has cond(Z) ~ 2.5e5,
    # beyond the 2^12 a float32 CholeskyQR2 covers and within the 2^24 of the shifted form
    rs = np.random.default_rng(44)
    A = [synth.haar(n, 10, rs) for n in (60, 50, 40)]
    w = 10.0 ** (-0.6 * np.arange(10))
    X = np.einsum("j,aj,bj,cj->abc", w, *A) + 1e-9 * rs.standard_normal((60, 50, 40))
    return X.astype(np.float32), (5, 5, 5), 5, 3


@pytest.mark.parametrize("qr", ["householder", "cholesky", "shifted_cholesky3"])
@pytest.mark.parametrize("case", sorted(_QR_CASES))
def test_factorisation_forms_match_oracle(rt, qr, case):
    # S5 and the W-step's R factor by Householder QR / TSQR, or by the Cholesky form
    # (mixed-precision CholeskyQR2 of Z, or shifted CholeskyQR3; Cholesky of the
    # double-float Gram of B); the 3000-row mode takes Householder under every setting
    X, r, p, seed = _QR_CASES[case]()
    gap = 5e-3 if case == "widest70" else None
    if gap:
        Xd = torch.from_numpy(X).cuda()
        G, U = rt.rtucker_decompose(Xd, list(r), p, seed=seed, qr=qr)
        _, sig = rt.rtucker_factors(Xd, list(r), p, seed=seed, with_sigma=True, qr=qr)
        rt.sync()
        Xo = X.astype(np.float64)
        ref = tucker.sub_r_hosvd(Xo, list(r), p, seed=seed, with_core=False)
        for k in range(3):
            s_ref = ref["modes"][k]["sigma"]
            _, dev, _, _ = compare_factor(to_np(U[k]), ref["U"][k], s_ref, gap_min=gap)
            assert dev <= U_TOL, (k, dev)
            assert orthonormality(to_np(U[k])) < 1e-5
            assert np.abs(to_np(sig[k]) - s_ref).max() <= 1e-5 * s_ref[0]
        Gp = tucker.multi_ttm_t(Xo, [to_np(u) for u in U])
        assert np.abs(to_np(G) - Gp).max() <= 1e-5 * np.abs(Gp).max()
    else:
        _run_and_compare(rt, X, r, p, seed=seed, qr=qr)


def test_cholesky_form_falls_back_on_rank_deficient_sketch(rt):
    # an exact multilinear-rank-2 tensor with r + p = 7: Z = Y Omega has rank 2, so the
    # CholeskyQR of Z meets zero pivots and the kernel takes Householder instead; the two
    # determined columns per mode match the oracle and every factor is orthonormal
    X = synth.tucker_tensor((40, 36, 50), (2, 2, 2), noise=0.0, data_seed=13, dtype="f32")
    Xd = torch.from_numpy(X).cuda()
    G, U = rt.rtucker_decompose(Xd, [2, 2, 2], 5, seed=4, qr="cholesky")
    rt.sync()
    ref = tucker.sub_r_hosvd(X.astype(np.float64), [2, 2, 2], 5, seed=4)
    for k in range(3):
        _, dev, _, cov = compare_factor(to_np(U[k]), ref["U"][k], ref["modes"][k]["sigma"], min_covered=2)
        assert dev <= U_TOL
        assert orthonormality(to_np(U[k])) < 1e-5
    assert rt.rtucker_relerr(Xd, G, U) < 1e-5


def test_bench_shape_householder_form(rt):
    # the benchmark's workload with the Householder / TSQR factorisations (qr = 1)
    cfg = synth.ORDER4_128
    X = synth.named(cfg)
    _run_and_compare(rt, X, cfg["ranks"], cfg["p"], seed=cfg["seed"], check_core="projection", qr="householder")


@pytest.mark.parametrize("case", ["graded48", "bench128"])
def test_bf16_sketch_form_matches_its_oracle(rt, case):
    # rt_options.sketch = 1: Z from bfloat16-rounded fibers and Omega (float32 sums),
    # CholeskyQR2 of Z; the oracle rounds the same values (round to nearest even) and
    # forms Z in float64.  Factors within 1e-4, core = projection on the factors, and
    # the relative error that of the oracle's BF16 sketch form.
    if case == "bench128":
        cfg = synth.ORDER4_128
        X, r, p, seed = synth.named(cfg), list(cfg["ranks"]), cfg["p"], cfg["seed"]
    else:
        X, r, p, seed = synth.tucker_tensor((48, 48, 48, 48), (12,) * 4, noise=1e-6, data_seed=7, core="graded"), \
            [12] * 4, 6, 2
    Xd = torch.from_numpy(X).cuda()
    G, U = rt.rtucker_decompose(Xd, r, p, seed=seed, sketch="bf16")
    rt.sync()
    Xo = np.asarray(X, dtype=np.float64)
    ref = tucker.sub_r_hosvd(Xo, r, p, seed=seed, with_core=False, sketch_bf16=True)
    Un = [to_np(u) for u in U]
    for k in range(len(r)):
        _, dev, _, _ = compare_factor(Un[k], ref["U"][k], ref["modes"][k]["sigma"], min_covered=r[k] // 2)
        assert dev <= U_TOL, (k, dev)
        assert orthonormality(Un[k]) < 1e-5
    Gp = tucker.multi_ttm_t(Xo, Un)
    assert np.abs(to_np(G) - Gp).max() <= 1e-5 * np.abs(Gp).max()
    er = tucker.relerr(Xo, tucker.reconstruct(tucker.multi_ttm_t(Xo, ref["U"]), ref["U"]))
    assert abs(rt.rtucker_relerr(Xd, G, U) - er) <= RELERR_TOL
