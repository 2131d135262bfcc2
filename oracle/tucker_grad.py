"""Gradients of the Tucker reconstruction misfit and the adjoint of the core
projection, in plain float64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The Tucker format (Sec. 3) approximates X by Xhat = G x_1 U_1 ... x_d U_d; the
core step of Alg. 1 projects X onto given factors, G = X x_1 U_1^T ... x_d U_d^T.
Differentiating through either (the direction the paper's conclusion leaves
open; not itself in the paper) needs, for the misfit

    L(X, G, U) = 1/2 ||X - Xhat||_F^2,     R = X - Xhat,

the gradients

    dL/dX   = R
    dL/dG   = -R x_1 U_1^T ... x_d U_d^T
    dL/dU_n = -[R x_{m != n} U_m^T]_(n) G_(n)^T

and, for phi(X, U) = <Gbar, X x_1 U_1^T ... x_d U_d^T> (an upstream gradient Gbar
pulled back through the core projection),

    dphi/dX   = Gbar x_1 U_1 ... x_d U_d
    dphi/dU_n = [X x_{m != n} U_m^T]_(n) Gbar_(n)^T .

Both follow from d(A x_k M) = A x_k dM and <A, B x_k M> = <A x_k M^T, B>.
Unfoldings are the mode-n matricizations of Sec. 2.2 (C order over the other
modes).  Parity pinned by central finite differences, an independent autograd
evaluation and the stationarity of the projected core (tests/test_oracle_grad.py).
"""

import numpy as np

from .tucker import reconstruct, ttm, unfold


def partial_projection(X, U, n):
    """X x_{m != n} U_m^T (mode n keeps its size n_n, mode m becomes r_m)."""
    Y = np.asarray(X, dtype=np.float64)
    for m, Um in enumerate(U):
        if m != n:
            Y = ttm(Y, np.asarray(Um, dtype=np.float64).T, m)
    return Y


def core_projection(X, U):
    """G = X x_1 U_1^T ... x_d U_d^T (Alg. 1, core step), modes in order."""
    Y = np.asarray(X, dtype=np.float64)
    for m, Um in enumerate(U):
        Y = ttm(Y, np.asarray(Um, dtype=np.float64).T, m)
    return Y


def misfit(X, G, U):
    """L = 1/2 ||X - G x_1 U_1 ... x_d U_d||_F^2."""
    R = np.asarray(X, dtype=np.float64) - reconstruct(np.asarray(G, dtype=np.float64),
                                                      [np.asarray(u, dtype=np.float64) for u in U])
    return 0.5 * float(np.sum(R * R))


def misfit_grads(X, G, U):
    """(L, dL/dX, dL/dG, [dL/dU_n]) of the misfit at (X, G, U)."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    U = [np.asarray(u, dtype=np.float64) for u in U]
    R = X - reconstruct(G, U)
    L = 0.5 * float(np.sum(R * R))
    dG = -core_projection(R, U)
    dU = [-(unfold(partial_projection(R, U, n), n) @ unfold(G, n).T) for n in range(len(U))]
    return L, R, dG, dU


def core_projection_adjoint(X, U, Gbar):
    """(dphi/dX, [dphi/dU_n]) for phi(X, U) = <Gbar, X x_1 U_1^T ... x_d U_d^T>."""
    X = np.asarray(X, dtype=np.float64)
    Gbar = np.asarray(Gbar, dtype=np.float64)
    U = [np.asarray(u, dtype=np.float64) for u in U]
    Xbar = reconstruct(Gbar, U)
    Ubar = [unfold(partial_projection(X, U, n), n) @ unfold(Gbar, n).T for n in range(len(U))]
    return Xbar, Ubar
