"""Pins of the float64 gradient oracle (oracle/tucker_grad.py) against what the
mathematics fixes, independently of its formulas: central finite differences of
the misfit and of <Gbar, core projection>, an autograd evaluation of the same
functions (torch, float64, CPU), and the normal equations of the projected core
(dL/dG = 0 at G = X x_k U_k^T for orthonormal U)."""
import numpy as np
import pytest
import torch

from oracle import tucker_grad as tg
from oracle.tucker import reconstruct

SHAPES = [((5, 6, 7), (2, 3, 4)), ((3, 4, 5, 6), (2, 2, 3, 3)), ((6, 5), (3, 2)), ((2, 3, 2, 3, 2), (1, 2, 2, 1, 2))]


def _problem(shape, ranks, seed):
    rs = np.random.default_rng(seed)
    X = rs.standard_normal(shape)
    G = rs.standard_normal(ranks)
    U = [rs.standard_normal((n, r)) for n, r in zip(shape, ranks)]
    return X, G, U


def _torch_misfit(X, G, U):
    Xh = G
    for Uk in U:
        Xh = torch.tensordot(Xh, Uk, dims=([0], [1]))
    R = X - Xh
    return 0.5 * (R * R).sum()


def _torch_phi(X, U, Gbar):
    Y = X
    for Uk in U:
        Y = torch.tensordot(Y, Uk, dims=([0], [0]))
    return (Gbar * Y).sum()


@pytest.mark.parametrize("shape,ranks", SHAPES)
def test_misfit_grads_match_autograd(shape, ranks):
    X, G, U = _problem(shape, ranks, 1)
    L, dX, dG, dU = tg.misfit_grads(X, G, U)
    tX = torch.tensor(X, requires_grad=True)
    tG = torch.tensor(G, requires_grad=True)
    tU = [torch.tensor(u, requires_grad=True) for u in U]
    tl = _torch_misfit(tX, tG, tU)
    tl.backward()
    assert abs(L - tl.item()) <= 1e-12 * max(1.0, abs(L))
    assert np.allclose(dX, tX.grad.numpy(), rtol=0, atol=1e-12 * np.abs(dX).max())
    assert np.allclose(dG, tG.grad.numpy(), rtol=0, atol=1e-11 * np.abs(dG).max())
    for a, b in zip(dU, tU):
        assert np.allclose(a, b.grad.numpy(), rtol=0, atol=1e-11 * np.abs(a).max())


@pytest.mark.parametrize("shape,ranks", SHAPES)
def test_misfit_grads_central_differences(shape, ranks):
    X, G, U = _problem(shape, ranks, 2)
    _, dX, dG, dU = tg.misfit_grads(X, G, U)
    rs = np.random.default_rng(3)
    h = 1e-5

    def fd(f, base, dirn):
        return (f(base + h * dirn) - f(base - h * dirn)) / (2 * h)

    Dx = rs.standard_normal(X.shape)
    got = fd(lambda x: tg.misfit(x, G, U), X, Dx)
    assert abs(got - np.sum(dX * Dx)) <= 1e-7 * max(1.0, abs(got))
    Dg = rs.standard_normal(G.shape)
    got = fd(lambda g: tg.misfit(X, g, U), G, Dg)
    assert abs(got - np.sum(dG * Dg)) <= 1e-7 * max(1.0, abs(got))
    for n in range(len(U)):
        Du = rs.standard_normal(U[n].shape)

        def f(u, n=n):
            V = list(U)
            V[n] = u
            return tg.misfit(X, G, V)
        got = fd(f, U[n], Du)
        assert abs(got - np.sum(dU[n] * Du)) <= 1e-6 * max(1.0, abs(got)), n


@pytest.mark.parametrize("shape,ranks", SHAPES)
def test_core_adjoint_matches_autograd_and_differences(shape, ranks):
    X, _, U = _problem(shape, ranks, 4)
    Gbar = np.random.default_rng(5).standard_normal(ranks)
    Xbar, Ubar = tg.core_projection_adjoint(X, U, Gbar)
    tX = torch.tensor(X, requires_grad=True)
    tU = [torch.tensor(u, requires_grad=True) for u in U]
    _torch_phi(tX, tU, torch.tensor(Gbar)).backward()
    assert np.allclose(Xbar, tX.grad.numpy(), rtol=0, atol=1e-12 * np.abs(Xbar).max())
    for a, b in zip(Ubar, tU):
        assert np.allclose(a, b.grad.numpy(), rtol=0, atol=1e-11 * np.abs(a).max())
    # directional derivative of phi along a random U_0 direction
    h = 1e-5
    D = np.random.default_rng(6).standard_normal(U[0].shape)

    def phi(u0):
        return float(np.sum(Gbar * tg.core_projection(X, [u0] + list(U[1:]))))
    got = (phi(U[0] + h * D) - phi(U[0] - h * D)) / (2 * h)
    assert abs(got - np.sum(Ubar[0] * D)) <= 1e-7 * max(1.0, abs(got))


def test_projected_core_is_stationary():
    # for orthonormal factors the best core is the projection: dL/dG = 0 there,
    # and L equals 1/2 (||X||^2 - ||G||^2)
    rs = np.random.default_rng(7)
    shape, ranks = (7, 8, 9), (3, 4, 2)
    X = rs.standard_normal(shape)
    U = [np.linalg.qr(rs.standard_normal((n, r)))[0] for n, r in zip(shape, ranks)]
    G = tg.core_projection(X, U)
    L, _, dG, _ = tg.misfit_grads(X, G, U)
    assert np.abs(dG).max() <= 1e-12 * np.abs(X).max()
    assert abs(L - 0.5 * (np.sum(X * X) - np.sum(G * G))) <= 1e-10 * np.sum(X * X)


def test_exact_tucker_has_zero_gradient():
    rs = np.random.default_rng(8)
    ranks, shape = (2, 3, 2), (5, 6, 4)
    G = rs.standard_normal(ranks)
    U = [rs.standard_normal((n, r)) for n, r in zip(shape, ranks)]
    X = reconstruct(G, U)
    L, dX, dG, dU = tg.misfit_grads(X, G, U)
    assert L <= 1e-25 * np.sum(X * X)
    assert np.abs(dG).max() <= 1e-12 and all(np.abs(u).max() <= 1e-12 for u in dU)
