"""The allocation-free entry point rhtucker_root_transfer_noalloc, called
through the C ABI, must reproduce the root transfer tensor that
rhtucker_decompose computes, on two calls in a row (its static scratch is
shared between calls).  This file is collected last on purpose."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_root_transfer_noalloc_matches_decompose_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_21379_gb300 import build
    build.build()
    import paper_2603_21379_gb300 as rt
    lib = rt.load_library()
    X = torch.from_numpy(synth.inv_norm_tensor(8, 6)).cuda()
    rank, p = 5, 3
    _, B, Un = rt.rhtucker_decompose(X, rank, p, seed=3, return_nodes=True)
    tree = rt.ht_tree(6)
    left, right = tree[0][2], tree[0][3]
    Ul, Ur = Un[left].contiguous(), Un[right].contiguous()
    BR = B[0].clone()
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = 1e-5 * float(BR.abs().max())
    for _ in range(2):
        out = torch.full((1, Ul.shape[1], Ur.shape[1]), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.rhtucker_root_transfer_noalloc(ctypes.c_void_p(X.data_ptr()), 0, Ul.shape[0], Ur.shape[0],
                                                ctypes.c_void_p(Ul.data_ptr()), Ul.shape[1],
                                                ctypes.c_void_p(Ur.data_ptr()), Ur.shape[1],
                                                ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize()
        diff = (out - BR).abs().max().item()
        assert np.isfinite(diff) and diff <= tol, diff


def test_root_transfer_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_21379_gb300 as rt
    lib = rt.load_library()
    dummy = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # 2^31 x 2^20 partial blocks of 12 x 12 exceed the static capacity: RT_ENOTSUP, nothing launched
    st = lib.rhtucker_root_transfer_noalloc(p, 0, 1 << 31, 1 << 20, p, 12, p, 12, p, None)
    assert st == 7
    assert lib.rhtucker_root_transfer_noalloc(None, 0, 4, 4, p, 1, p, 1, p, None) == 1
