"""GPU parity of the differentiable Tucker extension (rtucker_loss_grad,
rtucker_core_adjoint) against the float64 oracle (oracle/tucker_grad.py).

Every call goes through the C ABI.  Bar: each output element within
4e-5 x its rounding-error scale, the same contraction applied to absolute
values (|X| + |G| x_k |U_k| for the residual, then |U_k| and |G|): the worst-case
forward error of the float32 chains (sums of at most ~300 terms) stays below
2e-5 x that scale, while a wrong term or index is off by O(1) of it.  The loss
within 1e-6 relative plus the residual's rounding scale.
"""

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


def _scales(X, G, U):
    """Rounding-error scales of dX, dG and dU_n: the same contractions on absolute
    values, starting from |X| + |G| x_k |U_k| (the sum of |terms| behind each
    element of Xhat, which bounds its float32 rounding)."""
    Ua = [np.abs(u) for u in U]
    A = np.abs(X) + reconstruct(np.abs(np.asarray(G, np.float64)), [np.asarray(u, np.float64) for u in Ua])
    sG = tg.core_projection(A, Ua)
    sU = [unfold(tg.partial_projection(A, Ua, n), n) @ unfold(np.abs(G), n).T for n in range(len(U))]
    return A, sG, sU


def _check(got, ref, scale, what):
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref)
    bad = err > REL * scale + 1e-30
    assert not bad.any(), (what, float((err / np.maximum(scale, 1e-30)).max()))


def _run_grad(rt, X, G, U):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Gd = torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()
    Ud = [torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda() for u in U]
    loss, dX, dG, dU = rt.rtucker_loss_grad(Xd, Gd, Ud)
    rt.sync()
    return loss.item(), dX.cpu().numpy(), dG.cpu().numpy(), [u.cpu().numpy() for u in dU]


CASES = [((13, 9, 11), (3, 4, 5)), ((7, 9, 11, 13), (2, 3, 4, 5)), ((40, 33), (6, 5)),
         ((5, 6, 4, 3, 7), (2, 3, 2, 3, 4)), ((70, 66, 65), (16, 9, 1))]


@pytest.mark.parametrize("shape,ranks", CASES)
def test_loss_grad_random_model(rt, shape, ranks):
    rs = np.random.default_rng(sum(shape))
    X = rs.standard_normal(shape).astype(np.float32)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    L, dX, dG, dU = _run_grad(rt, X, G, U)
    Lr, dXr, dGr, dUr = tg.misfit_grads(X, G, U)
    A, sG, sU = _scales(X, G, U)
    _check(dX, dXr, A, "dX")
    _check(dG, dGr, sG, "dG")
    for n in range(len(U)):
        _check(dU[n], dUr[n], sU[n], "dU%d" % n)
    assert abs(L - Lr) <= 1e-6 * Lr + REL * float(np.sum(A * np.abs(dXr)))


# Shapes whose last two modes take the general form (mode d-2 expanded, then the last
# mode by rows): one large slab (d = 2); slabs too large for shared memory.
GENERAL = [((600, 500), (8, 12)), ((3, 700, 1100), (2, 20, 30))]


@pytest.mark.parametrize("shape,ranks", GENERAL)
def test_loss_grad_general_last_modes(rt, shape, ranks):
    rs = np.random.default_rng(sum(shape))
    X = rs.standard_normal(shape).astype(np.float32)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    L, dX, dG, dU = _run_grad(rt, X, G, U)
    Lr, dXr, dGr, dUr = tg.misfit_grads(X, G, U)
    A, sG, sU = _scales(X, G, U)
    _check(dX, dXr, A, "dX")
    _check(dG, dGr, sG, "dG")
    for n in range(len(U)):
        _check(dU[n], dUr[n], sU[n], "dU%d" % n)
    bound = REL * float(np.sum(A * np.abs(dXr)))
    assert abs(L - Lr) <= 1e-6 * Lr + bound
    # the loss alone (no residual stored) and the core adjoint's Xbar (no X) on the same path
    Xd = torch.from_numpy(X).cuda()
    Gd = torch.from_numpy(G).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    only = rt.rtucker_loss_grad(Xd, Gd, Ud, dX=False, dG=False, dU=False)
    xb, _ = rt.rtucker_core_adjoint(Xd, Ud, Gd, Ubar=False)
    rt.sync()
    assert abs(only[0].item() - Lr) <= 1e-6 * Lr + bound
    Xbr, _ = tg.core_projection_adjoint(X, U, G)
    _check(xb.cpu().numpy(), Xbr, np.abs(reconstruct(np.abs(G).astype(np.float64), [np.abs(u) for u in U])),
           "Xbar")


def test_loss_grad_general_many_large_slabs(rt):
    # 152 slabs of 260 x 300 with r = 64 in the last two modes: more slabs than SMs,
    # each too large for shared memory; dX compared on sampled entries
    shape, ranks = (19, 8, 260, 300), (2, 2, 64, 64)
    rs = np.random.default_rng(21)
    X = rs.standard_normal(shape).astype(np.float32)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    L, dX, dG, dU = _run_grad(rt, X, G, U)
    Lr, dXr, dGr, dUr = tg.misfit_grads(X, G, U)
    A, sG, sU = _scales(X, G, U)
    idx = tuple(rs.integers(0, n, size=20000) for n in shape)
    _check(dX[idx], dXr[idx], A[idx], "dX")
    _check(dG, dGr, sG, "dG")
    for n in range(4):
        _check(dU[n], dUr[n], sU[n], "dU%d" % n)
    assert abs(L - Lr) <= 1e-6 * Lr + REL * float(np.sum(A * np.abs(dXr)))


def test_loss_only_and_partial_outputs(rt):
    rs = np.random.default_rng(3)
    shape, ranks = (20, 17, 19), (4, 3, 5)
    X = rs.standard_normal(shape).astype(np.float32)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [rs.standard_normal((n, r)).astype(np.float32) for n, r in zip(shape, ranks)]
    Xd = torch.from_numpy(X).cuda()
    Gd = torch.from_numpy(G).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    full = rt.rtucker_loss_grad(Xd, Gd, Ud)
    only = rt.rtucker_loss_grad(Xd, Gd, Ud, dX=False, dG=False, dU=False)
    no_dx = rt.rtucker_loss_grad(Xd, Gd, Ud, dX=False)
    rt.sync()
    assert only[1] is None and only[2] is None and only[3] is None
    assert only[0].item() == full[0].item()
    assert torch.equal(no_dx[2], full[2])
    for a, b in zip(no_dx[3], full[3]):
        assert torch.equal(a, b)


def test_core_adjoint_random(rt):
    rs = np.random.default_rng(11)
    for shape, ranks in CASES[:4]:
        X = rs.standard_normal(shape).astype(np.float32)
        U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
        Gb = rs.standard_normal(ranks).astype(np.float32)
        Xd = torch.from_numpy(X).cuda()
        xb, ub = rt.rtucker_core_adjoint(Xd, [torch.from_numpy(u).cuda() for u in U], torch.from_numpy(Gb).cuda())
        rt.sync()
        Xbr, Ubr = tg.core_projection_adjoint(X, U, Gb)
        Ua = [np.abs(u) for u in U]
        _check(xb.cpu().numpy(), Xbr, np.abs(reconstruct(np.abs(Gb).astype(np.float64), Ua)), "Xbar")
        for n in range(len(U)):
            s = unfold(tg.partial_projection(np.abs(X), Ua, n), n) @ unfold(np.abs(Gb), n).T
            _check(ub[n].cpu().numpy(), Ubr[n], s, "Ubar%d" % n)


def test_core_adjoint_bf16_and_f64_input(rt):
    rs = np.random.default_rng(12)
    shape, ranks = (12, 10, 14), (3, 4, 2)
    X64 = rs.standard_normal(shape)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    Gb = rs.standard_normal(ranks).astype(np.float32)
    Ud = [torch.from_numpy(u).cuda() for u in U]
    for Xd in (torch.from_numpy(X64).cuda(), torch.from_numpy(X64).to(torch.bfloat16).cuda()):
        _, ub = rt.rtucker_core_adjoint(Xd, Ud, torch.from_numpy(Gb).cuda(), Xbar=False)
        rt.sync()
        Xo = Xd.double().cpu().numpy()     # the values the kernels read
        _, Ubr = tg.core_projection_adjoint(Xo, U, Gb)
        Ua = [np.abs(u) for u in U]
        for n in range(3):
            s = unfold(tg.partial_projection(np.abs(Xo), Ua, n), n) @ unfold(np.abs(Gb), n).T
            _check(ub[n].cpu().numpy(), Ubr[n], s, "Ubar%d" % n)


def test_rejects_bad_arguments(rt):
    X = torch.zeros((4, 5, 6), device="cuda")
    G = torch.zeros((2, 2, 2), device="cuda")
    U = [torch.zeros((n, 2), device="cuda") for n in (4, 5, 6)]
    with pytest.raises(ValueError):
        rt.rtucker_loss_grad(X, G, U[:2])
    with pytest.raises(rt.RtError):
        rt.rtucker_loss_grad(X, torch.zeros((2, 2, 70), device="cuda"),
                             [torch.zeros((n, r), device="cuda") for n, r in zip((4, 5, 6), (2, 2, 70))])


def test_order4_96_at_the_decomposition(rt):
    # the differentiable workload at full size: 96^4 float32 (Gaussian 16^4 core, Haar
    # factors, 1e-4 noise), gradients at the Sub-R-HOSVD result (r = 16, p = 8)
    cfg = synth.ORDER4_96
    X = synth.named(cfg)
    Xd = torch.from_numpy(X).cuda()
    G, U = rt.rtucker_decompose(Xd, list(cfg["ranks"]), cfg["p"], seed=cfg["seed"])
    loss, dX, dG, dU = rt.rtucker_loss_grad(Xd, G, U)
    rt.sync()
    Gn, Un = G.cpu().numpy(), [u.cpu().numpy() for u in U]
    Lr, dXr, dGr, dUr = tg.misfit_grads(X, Gn, Un)
    A, sG, sU = _scales(X, Gn, Un)
    assert abs(loss.item() - Lr) <= 1e-6 * Lr + REL * float(np.sum(A * np.abs(dXr)))
    rs = np.random.default_rng(0)
    idx = tuple(rs.integers(0, 96, size=20000) for _ in range(4))
    _check(dX.cpu().numpy()[idx], dXr[idx], A[idx], "dX")
    _check(dG.cpu().numpy(), dGr, sG, "dG")
    for n in range(4):
        _check(dU[n].cpu().numpy(), dUr[n], sU[n], "dU%d" % n)
    # the core from the projection is (to float32 rounding) the best core for these U
    assert np.abs(dGr).max() <= 1e-4 * np.abs(Gn).max()


def test_loss_grad_bf16_and_f64_input(rt):
    # X stored as bfloat16 / float64 (read through the scalar path of the residual
    # kernel); the oracle gets the values the kernels read
    rs = np.random.default_rng(13)
    shape, ranks = (18, 21, 15), (4, 3, 5)
    X64 = rs.standard_normal(shape)
    G = rs.standard_normal(ranks).astype(np.float32)
    U = [(rs.standard_normal((n, r)) / np.sqrt(n)).astype(np.float32) for n, r in zip(shape, ranks)]
    Gd = torch.from_numpy(G).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    for Xd in (torch.from_numpy(X64).cuda(), torch.from_numpy(X64).to(torch.bfloat16).cuda()):
        loss, dX, dG, dU = rt.rtucker_loss_grad(Xd, Gd, Ud)
        rt.sync()
        Xo = Xd.double().cpu().numpy()
        Lr, dXr, dGr, dUr = tg.misfit_grads(Xo, G, U)
        A, sG, sU = _scales(Xo, G, U)
        _check(dX.cpu().numpy(), dXr, A, "dX")
        _check(dG.cpu().numpy(), dGr, sG, "dG")
        for n in range(3):
            _check(dU[n].cpu().numpy(), dUr[n], sU[n], "dU%d" % n)
        assert abs(loss.item() - Lr) <= 1e-6 * Lr + REL * float(np.sum(A * np.abs(dXr)))
