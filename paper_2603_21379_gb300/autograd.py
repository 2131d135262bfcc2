"""torch.autograd.Function wrappers of the differentiable Tucker path.

The Tucker format of Sec. 3 approximates X by Xhat = G x_1 U_1 ... x_d U_d, and the
core step of Alg. 1 projects X on given factors, G = X x_1 U_1^T ... x_d U_d^T.
Training through a decomposition needs both directions; the gradients follow from
d(A x_k M) = A x_k dM and <A, B x_k M> = <A x_k M^T, B>:

  tucker_project(X, U)      G = X x_k U_k^T;  backward Gbar -> (Gbar x_k U_k,
                            [X x_{m!=n} U_m^T]_(n) Gbar_(n)^T)   (rtucker_core_adjoint)
  tucker_reconstruct(G, U)  Xhat = G x_k U_k; backward Zbar -> (Zbar x_k U_k^T,
                            [Zbar x_{m!=n} U_m^T]_(n) G_(n)^T)   (rtucker_core,
                            rtucker_core_adjoint with Zbar in the place of X)
  tucker_misfit(X, G, U)    L = 1/2 ||X - Xhat||_F^2 (float64) with dL/dX, dL/dG,
                            dL/dU_n from one rtucker_loss_grad call in the forward,
                            scaled by the upstream gradient in the backward.

Every value is computed by this library's CUDA kernels through the C ABI; torch
allocates the outputs and chains the gradients.  Factors and cores are float32; X
may be float32, float64 or bfloat16 (its gradient is returned in X's dtype).
set_grad_recompute(True) makes the partial projections recompute their prefix
contractions instead of keeping them (less workspace, more passes).
"""

import torch

from . import rtucker_core, rtucker_core_adjoint, rtucker_loss_grad, tucker_reconstruct_into


def _f32(t):
    return t.detach().to(torch.float32).contiguous()


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, *U):
        Xc = X.detach().contiguous()
        Uc = [_f32(u) for u in U]
        ctx.save_for_backward(Xc, *Uc)
        return rtucker_core(Xc, Uc)

    @staticmethod
    def backward(ctx, Gbar):
        X, *U = ctx.saved_tensors
        need_x = ctx.needs_input_grad[0]
        need_u = any(ctx.needs_input_grad[1:])
        if not (need_x or need_u):
            return (None,) * (1 + len(U))
        xb, ub = rtucker_core_adjoint(X, U, _f32(Gbar), Xbar=need_x, Ubar=need_u)
        out = [xb.to(X.dtype) if need_x else None]
        out += [ub[k] if (need_u and ctx.needs_input_grad[1 + k]) else None for k in range(len(U))]
        return tuple(out)


class _Reconstruct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G, *U):
        Gc = _f32(G)
        Uc = [_f32(u) for u in U]
        ctx.save_for_backward(Gc, *Uc)
        Xh = torch.empty([u.shape[0] for u in Uc], dtype=torch.float32, device=Gc.device)
        return tucker_reconstruct_into(Gc, Uc, Xh)

    @staticmethod
    def backward(ctx, Zbar):
        G, *U = ctx.saved_tensors
        Z = _f32(Zbar)
        need_g = ctx.needs_input_grad[0]
        need_u = any(ctx.needs_input_grad[1:])
        gG = rtucker_core(Z, U) if need_g else None
        gU = rtucker_core_adjoint(Z, U, G, Xbar=False, Ubar=True)[1] if need_u else None
        out = [gG]
        out += [gU[k] if (need_u and ctx.needs_input_grad[1 + k]) else None for k in range(len(U))]
        return tuple(out)


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, G, *U):
        need_x, need_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        need_u = any(ctx.needs_input_grad[2:])
        loss, gX, gG, gU = rtucker_loss_grad(X.detach().contiguous(), _f32(G), [_f32(u) for u in U],
                                             dX=need_x, dG=need_g, dU=need_u)
        ctx.xdtype = X.dtype
        ctx.nu = len(U)
        ctx.save_for_backward(*([t for t in (gX, gG) if t is not None] + (list(gU) if gU is not None else [])))
        ctx.has = (gX is not None, gG is not None, gU is not None)
        return loss

    @staticmethod
    def backward(ctx, gl):
        saved = list(ctx.saved_tensors)
        hx, hg, hu = ctx.has
        gX = saved.pop(0) if hx else None
        gG = saved.pop(0) if hg else None
        gU = saved if hu else None
        s = gl.to(torch.float32)
        out = [(gX * s).to(ctx.xdtype) if hx else None, gG * s if hg else None]
        out += [gU[k] * s if (hu and ctx.needs_input_grad[2 + k]) else None for k in range(ctx.nu)]
        return tuple(out)


def tucker_project(X, U):
    """G = X x_1 U_1^T ... x_d U_d^T with the hand-written backward (see module doc)."""
    return _Project.apply(X, *U)


def tucker_reconstruct(G, U):
    """Xhat = G x_1 U_1 ... x_d U_d (float32) with the hand-written backward."""
    return _Reconstruct.apply(G, *U)


def tucker_misfit(X, G, U):
    """L = 1/2 ||X - G x_1 U_1 ... x_d U_d||_F^2 (0-d float64 tensor) whose gradients
    come from the fused rtucker_loss_grad kernels."""
    return _Misfit.apply(X, G, *U)
