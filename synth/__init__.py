"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds the input generators only - none of the decomposition's
arithmetic.  Tests, the benchmark and the oracle all draw their tensors from
here, so the oracle and the CUDA library see the same bytes.

Workloads (the paper's own core function and its meteorological dataset are not
available; these seeded stand-ins keep the structure of its experiments:
low-multilinear-rank tensors with orthonormalized Gaussian factors, Sec. 3.3.1,
and the function f(x) = 1/||x|| on a uniform grid, Sec. 4.2.1):

* ``tucker_tensor``      X = C x_1 A_1 ... x_d A_d + noise, A_k Haar-orthonormal
                         (QR of a Gaussian with diag(R) > 0), C a Gaussian core
                         or the graded core C(i) = 10^{-(i_1+..+i_d)/16} xi_i.
* ``inv_norm_tensor``    X(i) = 1 / sqrt(sum_j x_{i_j}^2), x_i = lo + i (hi-lo)/(n-1),
                         evaluated in float64 with plain IEEE +, *, /, sqrt in a
                         fixed order, then rounded to float32 (bit-reproducible).
* ``inv_norm_tensor_torch``  the same tensor built with torch (float64 elementwise
                         ops, one kernel per operation, so no fused multiply-add),
                         slab by slab over the first mode, on any device: the
                         way to make the 16^8 (17 GB) tensor without a host copy.
* ``batched_shapes``     sizes/ranks of the batched workload (n_k ~ U{32..160},
                         r_k ~ U{4..min(24, n_k // 4)}).
"""

import numpy as np

# Named workloads: (shape, ranks, oversampling p, method seed, data seed, noise)
ORDER3_F64 = dict(shape=(64, 64, 64), ranks=(8, 8, 8), p=5, seed=0, data_seed=100,
                  noise=1e-8, core="gauss", core_ranks=(8, 8, 8), dtype="f64")
ORDER4_128 = dict(shape=(128, 128, 128, 128), ranks=(32, 32, 32, 32), p=10, seed=1,
                  data_seed=101, noise=1e-6, core="graded", core_ranks=(32, 32, 32, 32), dtype="f32")
ORDER4_96 = dict(shape=(96, 96, 96, 96), ranks=(16, 16, 16, 16), p=8, seed=4, data_seed=104,
                 noise=1e-4, core="gauss", core_ranks=(16, 16, 16, 16), dtype="f32")
INVNORM_16_8 = dict(n=16, d=8, lo=1.0, hi=2.0, rank=10, p=5, w=320, seed=3)
BATCHED_256 = dict(T=256, nmin=32, nmax=160, rmin=4, rmax=24, p=5, seed=2, data_seed=102,
                   noise=1e-6)
# The paper's single-node scaling workloads (its parallel experiments), one GPU:
# Tucker of order-8 low-rank tensors, rank 5, n = 16..20, s = 10^4 fibers per mode;
# H-Tucker of f = 1/||x|| on n^8 grids, rank 6, 20 n fibers per node.
SCALING_TUCKER = dict(d=8, ns=(16, 18, 20), rank=5, p=5, s=10000, seed=1, noise=1e-6)
SCALING_HT = dict(d=8, ns=(16, 18, 20), lo=1.0, hi=2.0, rank=6, p=5, w_per_n=20, seed=3)


def haar(n, r, rs):
    """n x r matrix with orthonormal columns, Haar distributed: Q of a Gaussian
    with the signs of diag(R) moved into Q."""
    Q, R = np.linalg.qr(rs.standard_normal((n, r)))
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def core_tensor(ranks, kind, rs):
    if kind == "gauss":
        return rs.standard_normal(tuple(ranks))
    if kind == "graded":
        # C(i) = 10^{-(i_1+...+i_d)/16} xi_i, i 0-based, xi_i ~ N(0,1)
        grids = np.meshgrid(*[np.arange(r) for r in ranks], indexing="ij")
        expo = sum(g.astype(np.float64) for g in grids)
        return 10.0 ** (-expo / 16.0) * rs.standard_normal(tuple(ranks))
    raise ValueError(kind)


def tucker_tensor(shape, core_ranks, noise=0.0, data_seed=0, core="gauss", dtype="f32",
                  with_parts=False):
    """X = C x_1 A_1 ... x_d A_d + noise * N(0,1), in float64 then cast to ``dtype``."""
    rs = np.random.default_rng(data_seed)
    C = core_tensor(core_ranks, core, rs)
    A = [haar(n, r, rs) for n, r in zip(shape, core_ranks)]
    X = C
    for Ak in A:  # contract the leading core mode, append the size-n mode
        X = np.tensordot(X, Ak, axes=([0], [1]))
    if noise:
        X = X + noise * rs.standard_normal(X.shape)
    X = np.ascontiguousarray(X.astype(np.float64 if dtype == "f64" else np.float32))
    if with_parts:
        return X, C, A
    return X


def named(cfg, with_parts=False):
    return tucker_tensor(cfg["shape"], cfg["core_ranks"], cfg["noise"], cfg["data_seed"],
                         cfg["core"], cfg["dtype"], with_parts=with_parts)


def inv_norm_grid(n, lo=1.0, hi=2.0):
    """Grid points x_i = lo + i (hi - lo)/(n - 1), i = 0..n-1 (endpoints included)."""
    i = np.arange(n, dtype=np.float64)
    return lo + i * ((hi - lo) / (n - 1))


def inv_norm_entries(idx, n, lo=1.0, hi=2.0):
    """X(i) for multi-indices ``idx`` (tuple of d integer arrays), float32.

    Sum of squares accumulated mode 0 first with separate IEEE multiply and add
    (no fused multiply-add), then sqrt and 1/(.) in float64, then one rounding
    to float32."""
    x = inv_norm_grid(n, lo, hi)
    acc = np.zeros(np.broadcast(*idx).shape, dtype=np.float64)
    for ij in idx:
        xi = x[ij]
        acc = acc + xi * xi
    return (1.0 / np.sqrt(acc)).astype(np.float32)


def inv_norm_tensor(n, d, lo=1.0, hi=2.0):
    """Full n^d tensor of f(x) = 1/||x|| on the grid (host; small d or n only)."""
    grids = np.meshgrid(*[np.arange(n)] * d, indexing="ij", sparse=True)
    return np.ascontiguousarray(inv_norm_entries(tuple(grids), n, lo, hi))


def inv_norm_tensor_torch(n, d, lo=1.0, hi=2.0, device="cpu"):
    """``inv_norm_tensor(n, d, lo, hi)`` as a contiguous torch float32 tensor on
    ``device``, bit-identical to the numpy version: the same float64 grid, the
    sum of squares accumulated mode 0 first with separate multiply and add
    kernels, then sqrt and 1/(.) in float64 (IEEE-rounded), then one rounding
    to float32.  Built one slab of the first mode at a time."""
    import torch
    x = torch.from_numpy(inv_norm_grid(n, lo, hi)).to(device)
    sq = x * x                                      # x_i^2, float64, rounded once
    out = torch.empty((n,) * d, dtype=torch.float32, device=device)
    rest = (n,) * (d - 1)
    for i0 in range(n):
        acc = sq[i0].expand(rest).clone()           # mode 0 term first
        for j in range(1, d):
            shape = [1] * (d - 1)
            shape[j - 1] = n
            acc = acc + sq.view(shape)              # modes 1..d-1 in order
        out[i0] = (1.0 / torch.sqrt(acc)).to(torch.float32)
    return out


def tucker_tensor_torch(shape, core_ranks, noise=0.0, data_seed=0, device="cpu"):
    """X = C x_1 A_1 ... x_d A_d + noise * N(0,1) as a contiguous float32 torch tensor
    built on ``device`` (for tensors too large for the host): Gaussian core, factors
    the Q of Gaussian n x r matrices, drawn from torch's generator seeded with
    ``data_seed``; the modes are expanded last to first, one batched matrix product
    each, and the noise is added one slab of the first mode at a time."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(data_seed))
    d = len(shape)
    Y = torch.randn(tuple(core_ranks), generator=g, device=device, dtype=torch.float32)
    A = [torch.linalg.qr(torch.randn((n, r), generator=g, device=device, dtype=torch.float64))[0].float()
         for n, r in zip(shape, core_ranks)]
    for k in range(d - 1, -1, -1):     # Y(..., a_k, i_{k+1}, ...) -> Y(..., i_k, i_{k+1}, ...)
        left = 1
        for j in range(k):
            left *= core_ranks[j]
        right = Y.numel() // (left * core_ranks[k])
        Y = torch.matmul(A[k], Y.reshape(left, core_ranks[k], right))
    X = Y.reshape(tuple(shape))
    if noise:
        for i0 in range(shape[0]):
            X[i0].add_(torch.randn(tuple(shape[1:]), generator=g, device=device, dtype=torch.float32),
                       alpha=noise)
    return X.contiguous()


def batched_shapes(T=256, nmin=32, nmax=160, rmin=4, rmax=24, data_seed=102):
    """Per-tensor mode sizes and ranks of the batched order-3 workload."""
    rs = np.random.default_rng(data_seed)
    shapes, ranks = [], []
    for _ in range(T):
        n = rs.integers(nmin, nmax + 1, size=3)
        r = [int(rs.integers(rmin, min(rmax, nk // 4) + 1)) for nk in n]
        shapes.append(tuple(int(v) for v in n))
        ranks.append(tuple(r))
    return shapes, ranks


def batched_tensors(T=256, nmin=32, nmax=160, rmin=4, rmax=24, noise=1e-6, data_seed=102):
    """T order-3 float32 tensors with Gaussian cores, Haar factors, and noise;
    tensor t uses data seed data_seed * 1000 + t."""
    shapes, ranks = batched_shapes(T, nmin, nmax, rmin, rmax, data_seed)
    Xs = [tucker_tensor(sh, rk, noise, data_seed * 1000 + t, "gauss", "f32")
          for t, (sh, rk) in enumerate(zip(shapes, ranks))]
    return Xs, shapes, ranks
