"""GPU parity of the Kronecker-structured sketch and of randomized HOSVD with
Kronecker test matrices (the rHKron comparison method, Sec. 3.3) against the
float64 oracle (oracle/rhkron.py), through the C ABI.

Bars: every sketch entry within 1e-5 of the same sketch of |X| with |Omega_j|
(the scale of its rounding error); factors within 1e-4 after the sign rule
(clusters of close singular values of C^(k) through projectors); the core
element-wise within 1e-5 of max|G| against the float64 projection of X on the
GPU's factors; |relerr_gpu - relerr_oracle| <= 1e-5."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import rhkron, tucker  # noqa: E402
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


def _check_sketch(rt, X, ell, seed, dt="f32"):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(_TDT[dt]).cuda()
    Z = rt.rtucker_kron_sketch(Xd, ell, seed=seed)
    rt.sync()
    Xs = Xd.cpu().double().numpy()
    Om = [rhkron.kron_omega(n, l, seed, j) for j, (n, l) in enumerate(zip(X.shape, ell))]
    Oa = [np.abs(o) for o in Om]
    for k in range(X.ndim):
        ref = rhkron.kron_sketch(Xs, Om, k)
        scale = rhkron.kron_sketch(np.abs(Xs), Oa, k)
        err = np.abs(to_np(Z[k]) - ref)
        assert not (err > 1e-5 * scale + 1e-30).any(), (k, float((err / np.maximum(scale, 1e-30)).max()))


@pytest.mark.parametrize("shape,ell", [
    ((30, 64, 96), (3, 2, 4)),                 # order 3
    ((6, 40, 100, 48), (2, 2, 3, 2)),          # ragged slab chunks (100 rows, 12 float4 columns)
    ((4, 5, 6, 32, 40), (2, 2, 1, 3, 2)),      # order 5, a width-1 mode
])
def test_kron_sketch_matches_oracle(rt, shape, ell):
    X = np.random.default_rng(sum(shape)).standard_normal(shape).astype(np.float32)
    _check_sketch(rt, X, ell, seed=7)


@pytest.mark.parametrize("dt", ["f64", "bf16"])
def test_kron_sketch_other_storage_types(rt, dt):
    X = np.random.default_rng(5).standard_normal((7, 36, 44)).astype(np.float32)
    _check_sketch(rt, X, (2, 3, 2), seed=3, dt=dt)


def test_kron_sketch_bench_shape(rt):
    # 128^4 with l = 4: every sketch 128 x 64, the registers' full share (8192 entries)
    cfg = synth.ORDER4_128
    _check_sketch(rt, synth.named(cfg), (4, 4, 4, 4), seed=cfg["seed"])


def _rhkron_compare(rt, X, r, ell, seed, gap_min=1e-3, min_covered=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    G, U = rt.rtucker_rhkron(Xd, list(r), list(ell), seed=seed)
    rt.sync()
    Xo = X.astype(np.float64)
    ref = rhkron.rhkron(Xo, r, ell, seed=seed)
    Un = [to_np(u) for u in U]
    for k in range(X.ndim):
        need = r[k] if min_covered is None else min_covered
        _, dev, _, _ = compare_factor(Un[k], ref["U"][k], ref["sigma"][k], gap_min=gap_min, min_covered=need)
        assert dev <= U_TOL, (k, dev)
        assert orthonormality(Un[k]) < 1e-5
        # the sign rule on U_k itself
        idx = np.argmax(np.abs(Un[k]), axis=0)
        assert (Un[k][idx, np.arange(r[k])] > 0).all()
    Gp = tucker.multi_ttm_t(Xo, Un)
    assert np.abs(to_np(G) - Gp).max() <= 1e-5 * np.abs(Gp).max(), np.abs(to_np(G) - Gp).max()
    eg = rt.rtucker_relerr(Xd, G, U)
    er = tucker.relerr(Xo, tucker.reconstruct(ref["G"], ref["U"]))
    assert abs(eg - er) <= RELERR_TOL, (eg, er)
    return eg, er


@pytest.mark.parametrize("shape,r,ell", [
    ((50, 60, 64), (5, 6, 7), (3, 3, 3)),
    ((40, 36, 48, 64), (4, 4, 4, 4), (2, 2, 2, 2)),
])
def test_rhkron_matches_oracle(rt, shape, r, ell):
    # (with a few sketch columns beyond r the Kronecker test matrix mixes all of the
    # noise into every column, so the error sits well above the noise level; the
    # oracle reaches the same one)
    X = synth.tucker_tensor(shape, r, noise=1e-4, data_seed=sum(shape))
    _rhkron_compare(rt, X, r, ell, seed=3)


def test_rhkron_bench_shape(rt):
    cfg = synth.ORDER4_128
    X = synth.named(cfg)
    _rhkron_compare(rt, X, cfg["ranks"], (4, 4, 4, 4), cfg["seed"], gap_min=1e-3, min_covered=28)


def test_kron_sketch_rejects_unsupported_shapes(rt):
    X = torch.zeros((8, 16, 30), device="cuda")            # n_{d-1} = 30: not a multiple of 4
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_kron_sketch(X, (2, 2, 2))
    assert e.value.status == 7
    X = torch.zeros((64, 256, 256), device="cuda")         # n_{d-2} K l_{d-1} = 256 * 8 * 8 > 8192
    with pytest.raises(rt.RtError) as e:
        rt.rtucker_kron_sketch(X, (8, 8, 8))
    assert e.value.status == 7
    X = torch.zeros((20, 16, 32), device="cuda")
    with pytest.raises(rt.RtError) as e:                   # L_0 = 36 > n_0 = 20
        rt.rtucker_rhkron(X, (2, 2, 2), (2, 6, 6))
    assert e.value.status == 1
