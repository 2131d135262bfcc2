"""Failure paths of the library, exercised without faulting or hanging the GPU:
a bounded device wait that runs out (RT_ETIMEOUT through rt_sync, the context
and the handle usable afterwards) and a device workspace allocation that fails
(RT_ENOMEM, outputs untouched, the next call fine).  Both go through the C ABI."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import tucker  # noqa: E402
from parity_util import U_TOL, compare_factor, to_np  # noqa: E402

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


def _small_case():
    X = synth.tucker_tensor((40, 36, 150), (4, 5, 6), noise=1e-4, data_seed=5, dtype="f32")
    return X, [4, 5, 6], 3, 11


def _check_against_oracle(X, r, p, seed, G, U):
    ref = tucker.sub_r_hosvd(X.astype(np.float64), r, p, seed=seed)
    for k in range(3):
        _, dev, _, cov = compare_factor(to_np(U[k]), ref["U"][k], ref["modes"][k]["sigma"], min_covered=r[k])
        assert dev <= U_TOL


def test_bounded_wait_times_out_and_handle_recovers(rt):
    rt.sync()
    try:
        rt.set_wait_limit(2000)
        rt.selftest_wait()
        with pytest.raises(rt.RtError) as e:
            rt.sync()
        assert e.value.status == 4            # RT_ETIMEOUT
        rt.sync()                              # the status word was cleared
    finally:
        rt.set_wait_limit(0)
    # a normal decomposition on the same handle and context, the tensor-core pass
    # (its TMA pipeline uses the same bounded waits) included
    X, r, p, seed = _small_case()
    G, U = rt.rtucker_decompose(torch.from_numpy(X).cuda(), r, p, seed=seed, core="tc")
    rt.sync()
    _check_against_oracle(X, r, p, seed, G, U)
    X4 = synth.tucker_tensor((6, 8, 64, 96), (3, 3, 5, 6), noise=1e-4, data_seed=3)
    G4, U4 = rt.rtucker_decompose(torch.from_numpy(X4).cuda(), [3, 3, 5, 6], 2, seed=4, core="tc")
    rt.sync()
    Gp = tucker.multi_ttm_t(X4.astype(np.float64), [to_np(u) for u in U4])
    assert np.abs(to_np(G4) - Gp).max() <= 1e-5 * np.abs(Gp).max()


def test_workspace_allocation_failure_leaves_outputs_untouched(rt):
    lib = rt.load_library()
    X, r, p, seed = _small_case()
    Xd = torch.from_numpy(X).cuda()
    h = ctypes.c_void_p()
    assert lib.rt_create(ctypes.byref(h), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    try:
        n = (ctypes.c_int64 * 3)(*X.shape)
        rk = (ctypes.c_int32 * 3)(*r)
        U = torch.full((sum(a * b for a, b in zip(X.shape, r)),), 7.0, device="cuda")
        G = torch.full((int(np.prod(r)),), 7.0, device="cuda")

        def call():
            return lib.rtucker_decompose(h, ctypes.c_void_p(Xd.data_ptr()), 0, 3, n, rk, p, None,
                                         ctypes.c_uint64(seed), None, ctypes.c_void_p(U.data_ptr()),
                                         ctypes.c_void_p(G.data_ptr()))
        assert lib.rt_inject_fault(h, 1, 1) == 0
        assert call() == 2                                   # RT_ENOMEM
        assert b"allocation" in lib.rt_last_error(h)
        assert lib.rt_sync(h) == 0
        assert bool((U == 7.0).all()) and bool((G == 7.0).all())
        assert lib.rt_workspace_bytes(h) == 0
        assert call() == 0                                   # the injection was used up
        assert lib.rt_sync(h) == 0
        Gw, Uw = rt.rtucker_decompose(Xd, r, p, seed=seed)
        rt.sync()
        assert torch.equal(G, Gw.reshape(-1))
        assert torch.equal(U, torch.cat([u.reshape(-1) for u in Uw]))
        assert lib.rt_inject_fault(h, 9, 1) == 1             # unknown kind
    finally:
        lib.rt_destroy(h)
