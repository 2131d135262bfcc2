"""torch.autograd.Function wrappers of the differentiable Tucker path
(paper_2603_21379_gb300.autograd) against the float64 oracle of the gradients
(oracle/tucker_grad.py), and the prefix-recomputation mode of the gradient
kernels.  Every value is computed through the C ABI; the bar is the one of the
direct gradient tests: each element within 4e-5 of its rounding-error scale (the
same contraction on absolute values)."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import tucker_grad as tg  # noqa: E402
from oracle.tucker import reconstruct, unfold  # noqa: E402

pytestmark = pytest.mark.gpu

REL = 4e-5


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_21379_gb300 import build
    build.build()
    import paper_2603_21379_gb300 as m
    m.load_library()
    return m


def _check(got, ref, scale, what):
    got = np.asarray(got.detach().double().cpu().numpy() if torch.is_tensor(got) else got, np.float64)
    err = np.abs(got - ref)
    assert not (err > REL * scale + 1e-30).any(), (what, float((err / np.maximum(scale, 1e-30)).max()))


def _problem(shape, ranks, seed):
    rs = np.random.default_rng(seed)
    X = rs.standard_normal(shape).astype(np.float32)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    W = rs.standard_normal(ranks).astype(np.float32)
    return X, U, W


def _leaf(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().requires_grad_(True)


@pytest.mark.parametrize("shape,ranks", [((20, 24, 28, 16), (4, 5, 6, 3)), ((33, 17, 40), (5, 4, 7))])
def test_project_backward_matches_oracle(rt, shape, ranks):
    from paper_2603_21379_gb300.autograd import tucker_project
    X, U, W = _problem(shape, ranks, 1)
    Xd, Ud = _leaf(X), [_leaf(u) for u in U]
    G = tucker_project(Xd, Ud)
    (G * torch.from_numpy(W).cuda()).sum().backward()
    Xo, Uo, Wo = X.astype(np.float64), [u.astype(np.float64) for u in U], W.astype(np.float64)
    Gref = tg.core_projection(Xo, Uo)
    Ua = [np.abs(u) for u in Uo]
    _check(G, Gref, tg.core_projection(np.abs(Xo), Ua), "G")
    xb, ub = tg.core_projection_adjoint(Xo, Uo, Wo)
    _check(Xd.grad, xb, reconstruct(np.abs(Wo), Ua), "Xbar")
    for n in range(len(U)):
        sc = unfold(tg.partial_projection(np.abs(Xo), Ua, n), n) @ unfold(np.abs(Wo), n).T
        _check(Ud[n].grad, ub[n], sc, ("Ubar", n))


def test_reconstruct_forward_and_backward_match_oracle(rt):
    from paper_2603_21379_gb300.autograd import tucker_reconstruct
    shape, ranks = (20, 24, 28, 16), (4, 5, 6, 3)
    rs = np.random.default_rng(2)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    Z = rs.standard_normal(shape).astype(np.float32)
    Gd, Ud = _leaf(G), [_leaf(u) for u in U]
    Xh = tucker_reconstruct(Gd, Ud)
    (Xh * torch.from_numpy(Z).cuda()).sum().backward()
    Go, Uo, Zo = G.astype(np.float64), [u.astype(np.float64) for u in U], Z.astype(np.float64)
    Ua = [np.abs(u) for u in Uo]
    _check(Xh, reconstruct(Go, Uo), reconstruct(np.abs(Go), Ua), "Xhat")
    _check(Gd.grad, tg.core_projection(Zo, Uo), tg.core_projection(np.abs(Zo), Ua), "Gbar")
    _, ub = tg.core_projection_adjoint(Zo, Uo, Go)
    for n in range(len(U)):
        sc = unfold(tg.partial_projection(np.abs(Zo), Ua, n), n) @ unfold(np.abs(Go), n).T
        _check(Ud[n].grad, ub[n], sc, ("Ubar", n))


def test_misfit_autograd_equals_fused_kernels_and_oracle(rt):
    # the misfit's gradients from one fused call, scaled by the upstream gradient;
    # and the same misfit composed from tucker_reconstruct and torch's own ops
    from paper_2603_21379_gb300.autograd import tucker_misfit, tucker_reconstruct
    cfg = synth.ORDER4_96
    X = synth.named(cfg)[:48, :40, :36, :30].copy()
    rs = np.random.default_rng(3)
    ranks = (16, 16, 16, 16)
    U = [np.linalg.qr(rs.standard_normal((n, r)))[0].astype(np.float32) for n, r in zip(X.shape, ranks)]
    G = tg.core_projection(X.astype(np.float64), U).astype(np.float32) + 1e-3 * rs.standard_normal(ranks).astype(
        np.float32)
    Xd, Gd, Ud = _leaf(X), _leaf(G), [_leaf(u) for u in U]
    L = tucker_misfit(Xd, Gd, Ud)
    (3.0 * L).backward()
    Lr, dXr, dGr, dUr = tg.misfit_grads(X, G, U)
    Xo, Go, Uo = X.astype(np.float64), G.astype(np.float64), [u.astype(np.float64) for u in U]
    Ua = [np.abs(u) for u in Uo]
    A = np.abs(Xo) + reconstruct(np.abs(Go), Ua)
    assert abs(float(L.item()) - Lr) <= 1e-6 * Lr + REL * float(np.sum(A * np.abs(dXr)))
    _check(Xd.grad, 3.0 * dXr, 3.0 * A, "dX")
    _check(Gd.grad, 3.0 * dGr, 3.0 * tg.core_projection(A, Ua), "dG")
    for n in range(len(U)):
        sc = unfold(tg.partial_projection(A, Ua, n), n) @ unfold(np.abs(Go), n).T
        _check(Ud[n].grad, 3.0 * dUr[n], 3.0 * sc, ("dU", n))
    # composed: 1/2 ||X - reconstruct(G, U)||^2 through torch's autograd
    Gd2, Ud2 = _leaf(G), [_leaf(u) for u in U]
    R = Xd.detach() - tucker_reconstruct(Gd2, Ud2)
    (0.5 * (R * R).sum()).backward()
    _check(Gd2.grad, dGr, tg.core_projection(A, Ua), "composed dG")
    for n in range(len(U)):
        sc = unfold(tg.partial_projection(A, Ua, n), n) @ unfold(np.abs(Go), n).T
        _check(Ud2[n].grad, dUr[n], sc, ("composed dU", n))


def test_prefix_recompute_mode_is_identical_and_smaller(rt):
    # rt_set_grad_recompute: the partial projections recompute P_m instead of keeping
    # the prefixes; the same kernels run in the same order per chain, so the results
    # are bit-identical, and a fresh handle needs less workspace
    lib = rt.load_library()
    cfg = synth.ORDER4_96
    X = torch.from_numpy(synth.named(cfg)).cuda()
    r = list(cfg["ranks"])
    G, U = rt.rtucker_decompose(X, r, cfg["p"], seed=cfg["seed"])
    Uf = torch.cat([u.reshape(-1) for u in U])
    n = (ctypes.c_int64 * 4)(*X.shape)
    rk = (ctypes.c_int32 * 4)(*r)
    out = {}
    for mode in (0, 1):
        h = ctypes.c_void_p()
        assert lib.rt_create(ctypes.byref(h), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
        try:
            assert lib.rt_set_grad_recompute(h, mode) == 0
            loss = torch.empty((), dtype=torch.float64, device="cuda")
            dG = torch.empty_like(G)
            dU = torch.empty_like(Uf)
            Ub = torch.empty_like(Uf)
            p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
            assert lib.rtucker_loss_grad(h, p(X), 0, 4, n, rk, p(Uf), p(G), p(loss), None, p(dG), p(dU)) == 0
            assert lib.rtucker_core_adjoint(h, p(X), 0, 4, n, rk, p(Uf), p(G), None, p(Ub)) == 0
            assert lib.rt_sync(h) == 0
            out[mode] = (loss.clone(), dG.clone(), dU.clone(), Ub.clone(), lib.rt_workspace_bytes(h))
        finally:
            lib.rt_destroy(h)
    for a, b in zip(out[0][:4], out[1][:4]):
        assert torch.equal(a, b)
    assert out[1][4] < out[0][4], (out[1][4], out[0][4])
    assert lib.rt_set_grad_recompute(None, 1) == 1
