"""GPU parity of the float8 storage form (RT_F8E4M3): X packed as E4M3 codes
with one power-of-two scale per slab of the last two modes.

* The packing (rt_quantize_fp8) is integer work: codes and scales must equal
  the oracle's (oracle/fp8.py) bit for bit, ties to even included.
* The decomposition of a packed tensor is the Sub-R-HOSVD (Alg. 1) of its
  stored values code x scale, so it is compared with the float64 oracle run on
  those values at the plain form's bars: factors within 1e-4 after the sign rule,
  sigma within 1e-5 of sigma_1, the core element-wise within 1e-5 of max|G|
  against the float64 projection on the GPU's factors, relerr within 1e-5.
* What the storage itself costs (the rounding of X to the E4M3 grid) is
  reported by bench.py, not asserted here; only its stated bound is.
Every call goes through the C ABI."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import fp8, tucker  # noqa: E402
from parity_util import RELERR_TOL, U_TOL, compare_factor, orthonormality, to_np  # noqa: E402

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


_TDT = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}


def _spread_tensor(shape, seed):
    """Gaussian slabs with magnitudes spread over 2^-30..2^30, one all-zero slab and
    values that land exactly halfway between two E4M3 neighbours."""
    rs = np.random.default_rng(seed)
    X = rs.standard_normal(shape) * np.exp2(rs.integers(-30, 30, shape[:-2] + (1, 1)))
    flat = X.reshape(-1, shape[-2], shape[-1])
    flat[1] = 0.0
    # slab 2: max |x| = 1 exactly, so scale = 2^-7 and x / scale = 17, -19 (spacing 2 there)
    # and 1.5 * 2^-9 (subnormal spacing 2^-9) are ties
    flat[2] = 0.0
    flat[2].flat[:6] = np.array([128.0, 17.0, -19.0, 40.5, 1.5 * 2.0 ** -9, 9.0]) / 128.0
    return X


@pytest.mark.parametrize("dt", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("shape", [(3, 2, 12, 20), (5, 7, 33, 48), (120, 208)])
def test_quantize_bit_exact(rt, dt, shape):
    X = _spread_tensor(shape, 3) if len(shape) > 2 else np.random.default_rng(4).standard_normal(shape)
    Xd = torch.from_numpy(X).to(_TDT[dt]).cuda()
    Xs = Xd.cpu().double().numpy()                # the values as stored in dtype dt
    q = rt.quantize_fp8(Xd)
    rt.sync()
    codes, scales = fp8.quantize(Xs)
    assert np.array_equal(q.codes.cpu().numpy(), codes)
    assert np.array_equal(q.scales.cpu().numpy(), scales)


def _decompose_and_compare(rt, X, r, p, seed, min_covered=None):
    Xq = rt.quantize_fp8(torch.from_numpy(np.ascontiguousarray(X)).cuda())
    G, U = rt.rtucker_decompose(Xq, list(r), p, seed=seed)
    rt.sync()
    _, sig = rt.rtucker_factors(Xq, list(r), p, seed=seed, with_sigma=True)
    rt.sync()
    Xs = fp8.dequantize(q_codes := Xq.codes.cpu().numpy(), Xq.scales.cpu().numpy())
    assert np.array_equal(q_codes, fp8.quantize(X)[0])
    ref = tucker.sub_r_hosvd(Xs, list(r), p, seed=seed, with_core=False)
    for k in range(X.ndim):
        need = r[k] if min_covered is None else min_covered
        _, dev, _, _ = compare_factor(to_np(U[k]), ref["U"][k], ref["modes"][k]["sigma"], min_covered=need)
        assert dev <= U_TOL, ("mode", k, dev)
        assert orthonormality(to_np(U[k])) < 1e-5
        s_ref = ref["modes"][k]["sigma"]
        assert np.abs(to_np(sig[k]) - s_ref).max() <= 1e-5 * s_ref[0] + 1e-30
    Gp = tucker.multi_ttm_t(Xs, [to_np(u) for u in U])
    assert np.abs(to_np(G) - Gp).max() <= 1e-5 * np.abs(Gp).max(), np.abs(to_np(G) - Gp).max()
    err_gpu = rt.rtucker_relerr(Xq, G, U)
    err_ref = tucker.relerr(Xs, tucker.reconstruct(tucker.multi_ttm_t(Xs, ref["U"]), ref["U"]))
    assert abs(err_gpu - err_ref) <= RELERR_TOL, (err_gpu, err_ref)
    return G, U, Xs, err_gpu


@pytest.mark.parametrize("shape,r,p,seed", [
    ((6, 40, 100, 48), (3, 4, 6, 5), 3, 5),       # 100-row slabs (ragged MMA tile), r_2 = 5
    ((8, 9, 128, 144), (3, 4, 12, 12), 4, 6),     # 144 columns: two stages per slab, ragged K chunk
    ((12, 10, 64, 128), (4, 5, 10, 32), 4, 7),    # r_2 = 32, the widest rank tile of the form
    ((9, 96, 80), (5, 8, 9), 3, 8),               # order 3
    ((120, 208), (10, 10), 5, 4),                 # d = 2: the whole matrix is one slab
])
def test_decompose_matches_oracle_on_stored_values(rt, shape, r, p, seed):
    X = synth.tucker_tensor(shape, r, noise=1e-4, data_seed=seed + 20)
    _decompose_and_compare(rt, X, r, p, seed, min_covered=min(r) - 1)


def test_bench_shape_fp8(rt):
    # the 128^4 workload in float8 storage: parity on the stored values, and the
    # storage error within its bound (half an E4M3 spacing, 2^-4 relative)
    cfg = synth.ORDER4_128
    X = synth.named(cfg)
    G, U, Xs, err = _decompose_and_compare(rt, X, cfg["ranks"], cfg["p"], cfg["seed"], min_covered=31)
    ex = np.abs(Xs - X.astype(np.float64))
    assert ex.max() <= 2.0 ** -4 * np.abs(X).max()
    store = float(np.linalg.norm(ex) / np.linalg.norm(X))
    assert store < 2.0 ** -4
    Xd = torch.from_numpy(X).cuda()
    err_x = rt.rtucker_relerr(Xd, G, U)            # against the float32 tensor itself
    assert err_x <= err + store + 1e-6


def test_unsupported_shapes_and_entry_points(rt):
    X = torch.from_numpy(synth.tucker_tensor((6, 20, 40), (3, 3, 3), noise=1e-4, data_seed=1)).cuda()
    q = rt.quantize_fp8(X)                          # packing takes any shape
    with pytest.raises(rt.RtError) as e:            # n_{d-1} = 40: not a multiple of 16
        rt.rtucker_decompose(q, [3, 3, 3], 2)
    assert e.value.status == 7
    X2 = torch.from_numpy(synth.tucker_tensor((6, 20, 48), (3, 3, 3), noise=1e-4, data_seed=1)).cuda()
    q2 = rt.quantize_fp8(X2)
    for call in (lambda: rt.rtucker_decompose(q2, [3, 3, 40], 2),               # r_{d-1} > 32
                 lambda: rt.rtucker_decompose(q2, [3, 3, 3], 2, core="ffma"),   # the FFMA chain
                 lambda: rt.rhtucker_decompose(q2, [1, 3, 3, 3, 3], 2)):         # not an H-Tucker input
        with pytest.raises(rt.RtError) as e:
            call()
        assert e.value.status == 7
    # the gradient entry points do not take the packed form (C ABI, dtype 3)
    lib = rt.load_library()
    h = ctypes.c_void_p()
    assert lib.rt_create(ctypes.byref(h), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    try:
        n = (ctypes.c_int64 * 3)(6, 20, 48)
        rk = (ctypes.c_int32 * 3)(3, 3, 3)
        z = torch.zeros(6 * 3 + 20 * 3 + 48 * 3 + 27, device="cuda")
        p = ctypes.c_void_p(z.data_ptr())
        assert lib.rtucker_loss_grad(h, ctypes.c_void_p(q2.data_ptr()), 3, 3, n, rk, p, p, None, None, p,
                                     None) == 7
    finally:
        lib.rt_destroy(h)
    G, U = rt.rtucker_decompose(q2, [3, 3, 3], 2)   # and the supported call still runs
    rt.sync()
    assert torch.isfinite(G).all()
