"""The allocation-free entry point rhtucker_root_transfer_noalloc, called
through the C ABI.  Some callers cannot let a library allocate device memory
(code running under global-mode stream capture, frameworks that own all device
memory, loops that must not meet cudaMalloc's implicit synchronisation); this
entry point keeps its scratch in a static device array instead.  It must give
the root transfer tensor of rhtucker_decompose and of the float64 oracle
(B_R = U_l^T X^(R_l) U_r, Sec. 4) on two calls in a row, since every call
shares the one static array.  This file is collected last on purpose: a run
that stops at the first failure has run every other test by then."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import htucker  # noqa: E402

pytestmark = pytest.mark.gpu

_DT = {"f32": (torch.float32, 0), "f64": (torch.float64, 1), "bf16": (torch.bfloat16, 2)}


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_21379_gb300 import build
    build.build()
    import paper_2603_21379_gb300 as m
    m.load_library()
    return m


def _call(lib, X, code, Ul, Ur, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rhtucker_root_transfer_noalloc(ctypes.c_void_p(X.data_ptr()), code, Ul.shape[0], Ur.shape[0],
                                              ctypes.c_void_p(Ul.data_ptr()), Ul.shape[1],
                                              ctypes.c_void_p(Ur.data_ptr()), Ur.shape[1],
                                              ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("dt", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("rank", [5, 12])
def test_root_transfer_noalloc_matches_decompose_twice(rt, dt, rank):
    # rank 12: the widest right-child rank the root kernels take in one pass
    tdt, code = _DT[dt]
    lib = rt.load_library()
    X = torch.from_numpy(synth.inv_norm_tensor(8, 6)).cuda().to(tdt)
    tree = rt.ht_tree(6)
    # rank `rank` at the root's two children (512 x 512 unfoldings), 5 elsewhere
    ranks = [1] + [rank if i in (tree[0][2], tree[0][3]) else 5 for i in range(1, len(tree))]
    _, B, Un = rt.rhtucker_decompose(X, ranks, 3, seed=3, return_nodes=True)
    left, right = tree[0][2], tree[0][3]
    Ul, Ur = Un[left].contiguous(), Un[right].contiguous()
    BR = B[0].clone()
    torch.cuda.synchronize()
    Xo = X.double().cpu().numpy()
    ref = htucker.root_transfer(Xo, Ul.double().cpu().numpy(), Ur.double().cpu().numpy())
    tol = 1e-5 * float(np.abs(ref).max())
    assert float((BR.double().cpu() - torch.from_numpy(ref)).abs().max()) <= tol
    for _ in range(2):
        out = torch.full((1, Ul.shape[1], Ur.shape[1]), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, X, code, Ul, Ur, out) == 0
        torch.cuda.synchronize()
        diff = (out - BR).abs().max().item()
        assert np.isfinite(diff) and diff <= tol, diff
        assert np.abs(out.double().cpu().numpy() - ref).max() <= tol


def test_root_transfer_noalloc_folds_rows_beyond_grid_limit(rt):
    # 65538 row blocks of 512 rows: more than a grid's 65535 CTA rows, so the row
    # blocks are folded onto the CTAs; the partials (one per block) fit the array
    lib = rt.load_library()
    nl, nr = 65538 * 512, 8
    rs = np.random.default_rng(31)
    Xh = rs.standard_normal((nl, nr), dtype=np.float32)
    Ulh = rs.standard_normal((nl, 1), dtype=np.float32)
    Urh = rs.standard_normal((nr, 1), dtype=np.float32)
    X, Ul, Ur = (torch.from_numpy(a).cuda() for a in (Xh, Ulh, Urh))
    ref = htucker.root_transfer(Xh.astype(np.float64), Ulh.astype(np.float64), Urh.astype(np.float64))
    bound = float((np.abs(Ulh.astype(np.float64)).T @ np.abs(Xh.astype(np.float64)) @ np.abs(Urh.astype(np.float64))).item())
    del Xh
    for _ in range(2):
        out = torch.full((1, 1, 1), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, X, 0, Ul, Ur, out) == 0
        torch.cuda.synchronize()
        # float32 sums over 2.7e8 terms: within 1e-6 of the sum of magnitudes
        assert abs(float(out.item()) - float(ref[0, 0, 0])) <= 1e-6 * bound


def test_root_transfer_noalloc_rejects_bad_arguments(rt):
    lib = rt.load_library()
    dummy = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # 2^31 x 2^20 partial blocks of 12 x 12 exceed the static capacity: RT_ENOTSUP, nothing launched
    assert lib.rhtucker_root_transfer_noalloc(p, 0, 1 << 31, 1 << 20, p, 12, p, 12, p, None) == 7
    assert lib.rhtucker_root_transfer_noalloc(p, 0, 4, 4, p, 1, p, 13, p, None) == 7      # rr > 12
    assert lib.rhtucker_root_transfer_noalloc(None, 0, 4, 4, p, 1, p, 1, p, None) == 1    # null X
    assert lib.rhtucker_root_transfer_noalloc(p, 3, 4, 4, p, 1, p, 1, p, None) == 1       # unknown dtype
    assert lib.rhtucker_root_transfer_noalloc(p, 0, 0, 4, p, 1, p, 1, p, None) == 1       # nl < 1
    # the Python wrapper checks shapes, dtypes and layouts before calling
    X = torch.zeros((6, 4), device="cuda")
    Ul, Ur = torch.zeros((6, 2), device="cuda"), torch.zeros((4, 3), device="cuda")
    assert tuple(rt.rhtucker_root_transfer_noalloc(X, Ul, Ur).shape) == (1, 2, 3)
    with pytest.raises(ValueError):
        rt.rhtucker_root_transfer_noalloc(X[:5], Ul, Ur)                     # too few elements
    with pytest.raises(ValueError):
        rt.rhtucker_root_transfer_noalloc(X, Ul.double(), Ur)                # float64 factor
    with pytest.raises(ValueError):
        rt.rhtucker_root_transfer_noalloc(X, Ul, torch.zeros((3, 4), device="cuda").t())   # not contiguous
    with pytest.raises(ValueError):
        rt.rhtucker_root_transfer_noalloc(X, Ul, Ur, out=torch.zeros((2, 3), device="cuda"))
