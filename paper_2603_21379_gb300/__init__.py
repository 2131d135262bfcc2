"""GB300-native subsampled randomized Tucker / H-Tucker (arXiv 2603.21379).

Thin ctypes binding over the C ABI of ``librtucker.so`` (``include/rtucker.h``).
Functions carry the C names and only marshal arguments: PyTorch supplies device
memory and the current CUDA stream, and every step of the decomposition runs
in the library's CUDA kernels.  There is no CPU fallback: if the library is
missing, calls raise.

Conventions: tensors are C-order CUDA tensors (float32, float64 or bfloat16);
factors come back as float32 ``n_k x r_k`` matrices, cores as float32 C-order
``r_1 x ... x r_d`` tensors.
"""

import ctypes
import os

import torch

__all__ = [
    "load_library", "library_path", "RtError", "sync",
    "rtucker_indices", "rtucker_sketch", "rtucker_factors", "rtucker_core", "rtucker_decompose",
    "rtucker_decompose_host", "rtucker_decompose_host_async", "rtucker_decompose_batched", "rtucker_relerr",
    "rhtucker_decompose", "rhtucker_relerr", "ht_tree", "ht_tree_from_children", "ht_alpha_w", "last_launch_count", "workspace_bytes",
    "set_timing", "get_timing", "STAGES", "rhtucker_root_transfer_noalloc", "BatchedDecomposition",
    "rtucker_loss_grad", "rtucker_core_adjoint", "set_wait_limit", "selftest_wait", "inject_fault",
    "set_grad_recompute", "tucker_reconstruct_into", "Fp8Tensor", "quantize_fp8", "rtucker_kron_sketch",
    "rtucker_rhkron", "kron_widths",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIBNAME = "librtucker.so"

RT_F32, RT_F64, RT_BF16, RT_F8E4M3 = 0, 1, 2, 3
_DT = {torch.float32: RT_F32, torch.float64: RT_F64, torch.bfloat16: RT_BF16}


class RtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("rtucker status %d: %s" % (status, msg))
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("overlap", ctypes.c_int32),
                ("core", ctypes.c_int32), ("qr", ctypes.c_int32), ("sketch", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


_QR = {"auto": 0, "householder": 1, "cholesky": 2, "shifted_cholesky3": 3}


_lib = None


def library_path():
    return os.path.join(_PKG, _LIBNAME)


def load_library():
    """Load librtucker.so (built by ``paper_2603_21379_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("librtucker.so is not built (run: python -m paper_2603_21379_gb300.build); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    P64 = ctypes.POINTER(ctypes.c_int64)
    P32 = ctypes.POINTER(ctypes.c_int32)
    PU64 = ctypes.POINTER(ctypes.c_uint64)
    PD = ctypes.POINTER(ctypes.c_double)
    PO = ctypes.POINTER(_Options)
    sig = {
        "rt_create": (ctypes.c_int, [ctypes.POINTER(vp), vp]),
        "rt_destroy": (ctypes.c_int, [vp]),
        "rt_set_stream": (ctypes.c_int, [vp, vp]),
        "rt_sync": (ctypes.c_int, [vp]),
        "rt_last_error": (ctypes.c_char_p, [vp]),
        "rt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "rt_version": (ctypes.c_int, []),
        "rt_last_launch_count": (ctypes.c_int, [vp]),
        "rt_workspace_bytes": (ctypes.c_size_t, [vp]),
        "rt_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "rt_get_timing": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), P64, ctypes.c_int, ctypes.c_int]),
        "rtucker_indices": (ctypes.c_int, [vp, ctypes.c_int, P64, P64, u64, vp]),
        "rtucker_sketch": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, i32, P64, u64, PO, vp]),
        "rtucker_factors": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, i32, P64, u64, PO, vp, vp]),
        "rtucker_core": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, vp, PO, vp]),
        "rtucker_decompose": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, i32, P64, u64, PO, vp, vp]),
        "rtucker_decompose_host": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, i32, P64, u64, PO,
                                                  vp, vp]),
        "rtucker_decompose_host_async": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, i32, P64, u64,
                                                        PO, vp, vp]),
        "rtucker_decompose_batched": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, P32,
                                                     ctypes.POINTER(P64), ctypes.POINTER(P32), i32,
                                                     ctypes.POINTER(P64), PU64, PO, ctypes.POINTER(vp),
                                                     ctypes.POINTER(vp)]),
        "rtucker_relerr": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, vp, vp, PD]),
        "rtucker_loss_grad": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, vp, vp, vp, vp, vp,
                                             vp]),
        "rtucker_core_adjoint": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, vp, vp, vp, vp]),
        "rhtucker_decompose": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, P32, i32, P64, u64,
                                              PO, vp, vp, vp]),
        "rhtucker_relerr": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, P32, vp, vp, PD]),
        "rhtucker_root_transfer_noalloc": (ctypes.c_int, [vp, ctypes.c_int, i64, i64, vp, i32, vp, i32, vp, vp]),
        "rt_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_uint32]),
        "rt_selftest_wait": (ctypes.c_int, [vp]),
        "rt_inject_fault": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "rt_set_grad_recompute": (ctypes.c_int, [vp, ctypes.c_int]),
        "rt_fp8_bytes": (ctypes.c_size_t, [ctypes.c_int, P64]),
        "rt_fp8_scale_offset": (ctypes.c_size_t, [ctypes.c_int, P64]),
        "rt_quantize_fp8": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, vp]),
        "rt_last_schedule": (ctypes.c_int, [vp, P32, ctypes.c_int]),
        "rtucker_kron_sketch": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, u64, PO, vp]),
        "rtucker_rhkron": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P64, P32, P32, u64, PO, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ------------------------------------------------------------------ handles
_handles = {}


def _handle(device=None):
    """Handle bound to the current CUDA stream of ``device`` (cached)."""
    lib = load_library()
    if device is None:
        device = torch.cuda.current_device()
    stream = torch.cuda.current_stream(device)
    key = (device, stream.cuda_stream)
    h = _handles.get(key)
    if h is None:
        with torch.cuda.device(device):
            hp = ctypes.c_void_p()
            st = lib.rt_create(ctypes.byref(hp), ctypes.c_void_p(stream.cuda_stream))
            if st != 0:
                raise RtError(st, "rt_create failed")
        h = hp
        _handles[key] = h
    return h


def _check(h, st):
    if st != 0:
        raise RtError(st, load_library().rt_last_error(h).decode())


def sync(device=None):
    """Wait for the library's work on the current stream and raise RtError if a
    kernel reported a device-side failure (bounded wait ran out, numerical
    breakdown, failed check) since the last sync."""
    h = _handle(device)
    try:
        _check(h, load_library().rt_sync(h))
    finally:
        _in_flight.pop(h.value, None)


def _i64(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int64 * len(vals))(*vals)


def _i32(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int32 * len(vals))(*vals)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _as_list(v, d):
    if isinstance(v, (list, tuple)):
        return [int(x) for x in v]
    return [int(v)] * d


class Fp8Tensor:
    """A tensor in the library's float8 storage (RT_F8E4M3, made by
    ``quantize_fp8``): ``data`` is the packed device buffer (uint8, E4M3 codes in
    C order, then one float32 power-of-two scale per slab of the last two modes),
    ``shape`` the tensor's sizes.  Accepted wherever the header lists RT_F8E4M3."""

    def __init__(self, data, shape):
        self.data = data
        self.shape = tuple(int(v) for v in shape)
        self.is_cuda = data.is_cuda
        self.device = data.device

    def data_ptr(self):
        return self.data.data_ptr()

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return True

    @property
    def codes(self):
        """The E4M3 codes, uint8, in the tensor's shape (a view of ``data``)."""
        return self.data[:_prod(self.shape)].view(self.shape)

    @property
    def scales(self):
        """The per-slab scales, float32 (a view of ``data``)."""
        off = int(load_library().rt_fp8_scale_offset(len(self.shape), _i64(self.shape)))
        nslab = _prod(self.shape[:-2])
        return self.data[off:off + 4 * nslab].view(torch.float32)


def quantize_fp8(X):
    """Pack a CUDA tensor (float32 / float64 / bfloat16, C order) into float8 storage
    (rt_quantize_fp8): per slab of the last two modes a power-of-two scale 2^(e-8)
    with max |x| = f 2^e, 0.5 <= f < 1, and the nearest E4M3 code of x / scale."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    if dt == 3:
        return X
    nbytes = int(lib.rt_fp8_bytes(d, _i64(n)))
    if nbytes == 0:
        raise ValueError("invalid sizes for float8 storage")
    data = torch.empty(nbytes, dtype=torch.uint8, device=X.device)
    h = _handle(X.device.index)
    _check(h, lib.rt_quantize_fp8(h, _ptr(X), dt, d, _i64(n), _ptr(data)))
    return Fp8Tensor(data, n)


def _tensor_args(X):
    if isinstance(X, Fp8Tensor):
        return 3, len(X.shape), list(X.shape)
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor")
    if X.dtype not in _DT:
        raise ValueError("X must be float32, float64 or bfloat16")
    if not X.is_contiguous():
        raise ValueError("X must be C-contiguous")
    return _DT[X.dtype], X.dim(), list(X.shape)


def _split(flat, rows, cols):
    out, off = [], 0
    for n, r in zip(rows, cols):
        out.append(flat[off:off + n * r].view(n, r))
        off += n * r
    return out


def last_launch_count(device=None):
    """Kernel launches enqueued by the last call on the current stream's handle."""
    return int(load_library().rt_last_launch_count(_handle(device)))


def workspace_bytes(device=None):
    return int(load_library().rt_workspace_bytes(_handle(device)))


STAGES = ("range_finder", "core_x_pass", "core_rest", "ht_transfer", "ht_root_pass", "range_finder_tail")


def set_timing(enable, device=None):
    """Record CUDA events around the library's stages on the current stream."""
    h = _handle(device)
    _check(h, load_library().rt_set_timing(h, 1 if enable else 0))


def get_timing(reset=True, device=None):
    """{stage: (total ms, intervals)} accumulated since the last reset."""
    h = _handle(device)
    ms = (ctypes.c_double * len(STAGES))()
    cnt = (ctypes.c_int64 * len(STAGES))()
    _check(h, load_library().rt_get_timing(h, ms, cnt, len(STAGES), 1 if reset else 0))
    return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}


# ------------------------------------------------------------------ Sub-R-HOSVD
def rtucker_indices(n, s=None, seed=0, device=None):
    """S1: concatenated sampled column indices pi_k (int64, on the device)."""
    lib = load_library()
    d = len(n)
    sv = [min(10 * n[k], _prod(n) // n[k]) for k in range(d)] if s is None else _as_list(s, d)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    idx = torch.empty(sum(sv), dtype=torch.int64, device=dev)
    h = _handle(dev.index)
    _check(h, lib.rtucker_indices(h, d, _i64(n), _i64(sv), ctypes.c_uint64(seed), _ptr(idx)))
    return list(torch.split(idx, sv))


def _prod(v):
    out = 1
    for x in v:
        out *= int(x)
    return out


def rtucker_sketch(X, r, p, s=None, seed=0):
    """S1-S4: sketches Z_k = Y_k Omega_k (n_k x (r_k + p)), float32."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    r = _as_list(r, d)
    Z = torch.empty(sum(nk * (rk + p) for nk, rk in zip(n, r)), dtype=torch.float32, device=X.device)
    h = _handle(X.device.index)
    sp = _i64(_as_list(s, d)) if s is not None else None
    _check(h, lib.rtucker_sketch(h, _ptr(X), dt, d, _i64(n), _i32(r), int(p), sp, ctypes.c_uint64(seed), None,
                                 _ptr(Z)))
    return _split(Z, n, [rk + p for rk in r])


def rtucker_factors(X, r, p, s=None, seed=0, with_sigma=False, qr="auto"):
    """S1-S6: factors U_k (n_k x r_k) with the column-sign rule; optionally the
    singular values of Q_k^T Y_k.  ``qr`` picks the range finder's factorisations
    (rt_options.qr: "auto", "householder", "cholesky", "shifted_cholesky3")."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    r = _as_list(r, d)
    U = torch.empty(sum(nk * rk for nk, rk in zip(n, r)), dtype=torch.float32, device=X.device)
    sig = torch.empty(sum(rk + p for rk in r), dtype=torch.float32, device=X.device) if with_sigma else None
    h = _handle(X.device.index)
    sp = _i64(_as_list(s, d)) if s is not None else None
    _check(h, lib.rtucker_factors(h, _ptr(X), dt, d, _i64(n), _i32(r), int(p), sp, ctypes.c_uint64(seed),
                                  _opts("fp32", qr=qr), _ptr(U), _ptr(sig)))
    Us = _split(U, n, r)
    if with_sigma:
        return Us, list(torch.split(sig, [rk + p for rk in r]))
    return Us


_PREC = {"fp32": 0, "bf16": 1}
_CORE = {"auto": 0, "tc": 1, "ffma": 2, "tune": 3}


def _opts(prec, overlap=False, graph=False, core="auto", qr="auto", sketch="fp32"):
    """rt_options for a precision form (the overlapped core schedule, CUDA-graph
    replay, the core kernels: "auto", "tc", "ffma" or "tune"; the range finder's
    factorisations: "auto", "householder", "cholesky" or "shifted_cholesky3"), or None (defaults)."""
    if prec not in _PREC:
        raise ValueError("prec must be 'fp32' or 'bf16'")
    if core not in _CORE:
        raise ValueError("core must be 'auto', 'tc', 'ffma' or 'tune'")
    if qr not in _QR:
        raise ValueError("qr must be 'auto', 'householder', 'cholesky' or 'shifted_cholesky3'")
    if sketch not in ("fp32", "bf16"):
        raise ValueError("sketch must be 'fp32' or 'bf16'")
    if prec == "fp32" and not overlap and not graph and core == "auto" and qr == "auto" and sketch == "fp32":
        return None
    o = _Options()
    o.prec = _PREC[prec]
    o.overlap = 1 if overlap else 0
    o.use_graph = 1 if graph else 0
    o.core = _CORE[core]
    o.qr = _QR[qr]
    o.sketch = 1 if sketch == "bf16" else 0
    return ctypes.byref(o)


def _cat_u(U):
    return torch.cat([u.reshape(-1).to(torch.float32) for u in U]).contiguous()


def rtucker_core(X, U, prec="fp32", core="auto"):
    """S7: core G = X x_1 U_1^T ... x_d U_d^T (float32 result; prec="bf16" rounds a
    float32 X to one bfloat16 term in the tensor-core pass; ``core`` selects the
    kernels, see rt_options.core)."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    r = [int(u.shape[1]) for u in U]
    Uc = _cat_u(U)
    G = torch.empty(r, dtype=torch.float32, device=X.device)
    h = _handle(X.device.index)
    _check(h, lib.rtucker_core(h, _ptr(X), dt, d, _i64(n), _i32(r), _ptr(Uc), _opts(prec, core=core), _ptr(G)))
    return G


def rtucker_decompose(X, r, p, s=None, seed=0, out=None, prec="fp32", overlap=False, graph=False, core="auto",
                      qr="auto", sketch="fp32"):
    """S1-S7: Sub-R-HOSVD; returns (G, [U_k]).  ``out`` = (Uflat, G) reuses buffers;
    ``prec`` "fp32" (default) or "bf16" (the BF16 compute form of the core pass);
    ``overlap`` runs the pass over X on the QR factors beside the SVD part of the
    range finder (see rt_options.overlap); ``graph`` replays the kernel sequence as
    a CUDA graph for repeated calls with the same buffers and shapes
    (rt_options.use_graph; pass ``out`` so that the output pointers repeat); ``qr``
    the range finder's factorisations (rt_options.qr); ``sketch`` "bf16" the
    bfloat16 sketch (rt_options.sketch)."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    r = _as_list(r, d)
    if out is None:
        U = torch.empty(sum(nk * rk for nk, rk in zip(n, r)), dtype=torch.float32, device=X.device)
        G = torch.empty(r, dtype=torch.float32, device=X.device)
    else:
        U, G = out
    h = _handle(X.device.index)
    sp = _i64(_as_list(s, d)) if s is not None else None
    _check(h, lib.rtucker_decompose(h, _ptr(X), dt, d, _i64(n), _i32(r), int(p), sp, ctypes.c_uint64(seed),
                                    _opts(prec, overlap, graph, core, qr, sketch), _ptr(U), _ptr(G)))
    return G, _split(U, n, r)


def rtucker_decompose_host(X, r, p, s=None, seed=0, out=None, prec="fp32"):
    """Sub-R-HOSVD of a HOST tensor (pinned memory recommended); copies in,
    decomposes, copies U and G back to host tensors; synchronous."""
    lib = load_library()
    if X.is_cuda or X.dtype not in _DT or not X.is_contiguous():
        raise ValueError("X must be a contiguous host tensor of float32/float64/bfloat16")
    d, n = X.dim(), list(X.shape)
    r = _as_list(r, d)
    if out is None:
        U = torch.empty(sum(nk * rk for nk, rk in zip(n, r)), dtype=torch.float32, pin_memory=True)
        G = torch.empty(r, dtype=torch.float32, pin_memory=True)
    else:
        U, G = out
    h = _handle()
    sp = _i64(_as_list(s, d)) if s is not None else None
    _check(h, lib.rtucker_decompose_host(h, _ptr(X), _DT[X.dtype], d, _i64(n), _i32(r), int(p), sp,
                                         ctypes.c_uint64(seed), _opts(prec), _ptr(U), _ptr(G)))
    return G, _split(U, n, r)


# host tensors of rtucker_decompose_host_async calls not yet synchronised, per handle
_in_flight = {}


def rtucker_decompose_host_async(X, r, p, s=None, seed=0, out=None, prec="fp32", graph=False):
    """Pipelined Sub-R-HOSVD of a HOST tensor: enqueues the copy of X into one of
    two device slots, the decomposition and the copies of U and G back to host
    tensors, and returns (G, [U_k]) before they are written.  The copy of the
    next call's X overlaps this call's decomposition; the results are valid
    after ``sync()``, and X must not be modified until then.  X and the outputs
    are kept alive here until that ``sync()``."""
    lib = load_library()
    if X.is_cuda or X.dtype not in _DT or not X.is_contiguous():
        raise ValueError("X must be a contiguous host tensor of float32/float64/bfloat16")
    d, n = X.dim(), list(X.shape)
    r = _as_list(r, d)
    if out is None:
        U = torch.empty(sum(nk * rk for nk, rk in zip(n, r)), dtype=torch.float32, pin_memory=True)
        G = torch.empty(r, dtype=torch.float32, pin_memory=True)
    else:
        U, G = out
    h = _handle()
    sp = _i64(_as_list(s, d)) if s is not None else None
    _check(h, lib.rtucker_decompose_host_async(h, _ptr(X), _DT[X.dtype], d, _i64(n), _i32(r), int(p), sp,
                                               ctypes.c_uint64(seed), _opts(prec, graph=graph), _ptr(U), _ptr(G)))
    _in_flight.setdefault(h.value, []).append((X, U, G))
    return G, _split(U, n, r)


def _flat_factors(U, n, r, device):
    if len(U) != len(n):
        raise ValueError("one factor per mode")
    for u, nk, rk in zip(U, n, r):
        if tuple(u.shape) != (nk, rk) or u.dtype != torch.float32 or u.device != device:
            raise ValueError("U_k must be float32 n_k x r_k tensors on X's device")
    return torch.cat([u.reshape(-1) for u in U])


def rtucker_loss_grad(X, G, U, dX=True, dG=True, dU=True):
    """Misfit L = 1/2 ||X - G x_1 U_1 ... x_d U_d||_F^2 of a Tucker model and its
    gradients (device float32): returns (loss as a 0-d float64 device tensor, dL/dX,
    dL/dG, [dL/dU_k]); a gradient not asked for is None."""
    lib = load_library()
    if not X.is_cuda or X.dtype not in _DT or not X.is_contiguous():
        raise ValueError("X must be a contiguous CUDA tensor of float32/float64/bfloat16")
    d, n = X.dim(), list(X.shape)
    r = list(G.shape)
    if len(r) != d or G.dtype != torch.float32 or not G.is_contiguous() or G.device != X.device:
        raise ValueError("G must be a contiguous float32 r_1 x ... x r_d tensor on X's device")
    Uf = _flat_factors(U, n, r, X.device)
    loss = torch.empty((), dtype=torch.float64, device=X.device)
    gX = torch.empty_like(X, dtype=torch.float32) if dX else None
    gG = torch.empty_like(G) if dG else None
    gU = torch.empty_like(Uf) if dU else None
    h = _handle()
    _check(h, lib.rtucker_loss_grad(h, _ptr(X), _DT[X.dtype], d, _i64(n), _i32(r), _ptr(Uf), _ptr(G), _ptr(loss),
                                    _ptr(gX), _ptr(gG), _ptr(gU)))
    return loss, gX, gG, (_split(gU, n, r) if dU else None)


def rtucker_core_adjoint(X, U, Gbar, Xbar=True, Ubar=True):
    """Adjoint of the core projection G = X x_1 U_1^T ... x_d U_d^T for an upstream
    gradient Gbar: returns (Xbar = Gbar x_k U_k, [Ubar_k]) (device float32); a result
    not asked for is None."""
    lib = load_library()
    if not X.is_cuda or X.dtype not in _DT or not X.is_contiguous():
        raise ValueError("X must be a contiguous CUDA tensor of float32/float64/bfloat16")
    d, n = X.dim(), list(X.shape)
    r = list(Gbar.shape)
    if len(r) != d or Gbar.dtype != torch.float32 or not Gbar.is_contiguous() or Gbar.device != X.device:
        raise ValueError("Gbar must be a contiguous float32 r_1 x ... x r_d tensor on X's device")
    Uf = _flat_factors(U, n, r, X.device)
    xb = torch.empty(n, dtype=torch.float32, device=X.device) if Xbar else None
    ub = torch.empty_like(Uf) if Ubar else None
    h = _handle()
    _check(h, lib.rtucker_core_adjoint(h, _ptr(X), _DT[X.dtype], d, _i64(n), _i32(r), _ptr(Uf), _ptr(Gbar),
                                       _ptr(xb), _ptr(ub)))
    return xb, (_split(ub, n, r) if Ubar else None)


def tucker_reconstruct_into(G, U, out):
    """out = G x_1 U_1 ... x_d U_d (the Tucker reconstruction, Sec. 3), out a
    contiguous float32 n_1 x ... x n_d device tensor: the Xbar part of
    rtucker_core_adjoint with Gbar = G (out stands in for X, which is not read
    when Ubar is not asked for)."""
    lib = load_library()
    if out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous float32 CUDA tensor")
    d, n = out.dim(), list(out.shape)
    r = list(G.shape)
    if len(r) != d or G.dtype != torch.float32 or not G.is_contiguous() or G.device != out.device:
        raise ValueError("G must be a contiguous float32 r_1 x ... x r_d tensor on out's device")
    Uf = _flat_factors(U, n, r, out.device)
    h = _handle()
    _check(h, lib.rtucker_core_adjoint(h, _ptr(out), 0, d, _i64(n), _i32(r), _ptr(Uf), _ptr(G), _ptr(out), None))
    return out


def set_grad_recompute(enable=True, device=None):
    """rt_set_grad_recompute: the partial projections of the gradient path recompute
    their prefix contractions instead of keeping them (less workspace)."""
    h = _handle(device)
    _check(h, load_library().rt_set_grad_recompute(h, 1 if enable else 0))


class BatchedDecomposition:
    """A batch of Sub-R-HOSVD problems with its argument arrays and outputs set up
    once: ``run()`` is a single call of ``rtucker_decompose_batched`` (one grouped
    launch per stage for all (tensor, mode) problems, one per contraction level of
    the cores), so repeated batches of the same shapes pay no per-call Python
    marshalling.  The tensors in ``Xs`` may be overwritten between runs.  U and G
    of all tensors live in two flat float32 buffers (``U_flat``, ``G_flat``);
    ``results()`` gives the per-tensor (G, [U_k]) views."""

    def __init__(self, Xs, ranks, p, seeds, s=None, prec="fp32", graph=False, qr="auto", core="auto"):
        self.lib = load_library()
        T = len(Xs)
        dts = {X.dtype for X in Xs}
        if len(dts) != 1:
            raise ValueError("all tensors of a batch share one dtype")
        self.dt = _DT[Xs[0].dtype]
        dev = Xs[0].device
        self.Xs = list(Xs)
        self.T, self.p = T, int(p)
        ds, ns, rs, shapes, rks = [], [], [], [], []
        for X, r in zip(Xs, ranks):
            _, d, n = _tensor_args(X)
            r = _as_list(r, d)
            ds.append(d)
            ns.append(_i64(n))
            rs.append(_i32(r))
            shapes.append(n)
            rks.append(r)
        self.shapes, self.ranks = shapes, rks
        usz = [sum(nk * rk for nk, rk in zip(n, r)) for n, r in zip(shapes, rks)]
        gsz = [_prod(r) for r in rks]
        self.U_flat = torch.empty(sum(usz), dtype=torch.float32, device=dev)
        self.G_flat = torch.empty(sum(gsz), dtype=torch.float32, device=dev)
        uoff = [0]
        for v in usz:
            uoff.append(uoff[-1] + v)
        goff = [0]
        for v in gsz:
            goff.append(goff[-1] + v)
        self._uoff, self._goff = uoff, goff
        P64 = ctypes.POINTER(ctypes.c_int64)
        P32 = ctypes.POINTER(ctypes.c_int32)
        self._keep = (ns, rs)
        self.n_arr = (P64 * T)(*[ctypes.cast(a, P64) for a in ns])
        self.r_arr = (P32 * T)(*[ctypes.cast(a, P32) for a in rs])
        self.s_arr = None
        if s is not None:
            self._s_keep = [_i64(_as_list(sv, dd)) for sv, dd in zip(s, ds)]
            self.s_arr = (P64 * T)(*[ctypes.cast(a, P64) for a in self._s_keep])
        self.d_arr = _i32(ds)
        self.X_arr = (ctypes.c_void_p * T)(*[X.data_ptr() for X in Xs])
        ub, gb = self.U_flat.data_ptr(), self.G_flat.data_ptr()
        self.U_arr = (ctypes.c_void_p * T)(*[ub + 4 * uoff[t] for t in range(T)])
        self.G_arr = (ctypes.c_void_p * T)(*[gb + 4 * goff[t] for t in range(T)])
        self.seed_arr = (ctypes.c_uint64 * T)(*[int(v) for v in seeds])
        self._opt_keep = _opts(prec, graph=graph, qr=qr, core=core)
        self.h = _handle(dev.index)

    def run(self):
        _check(self.h, self.lib.rtucker_decompose_batched(self.h, self.T, self.X_arr, self.dt, self.d_arr, self.n_arr,
                                                          self.r_arr, self.p, self.s_arr, self.seed_arr,
                                                          self._opt_keep, self.U_arr, self.G_arr))
        return self

    def schedule(self):
        """Per-level schedules of the last run's core contractions (rt_last_schedule):
        0 = grouped tiles, b > 0 = one row per lane with b 128-row blocks per CTA.
        ``core="tune"`` picks them by timing on the first run."""
        out = (ctypes.c_int32 * 16)()
        nlev = self.lib.rt_last_schedule(self.h, out, 16)
        return [int(out[k]) for k in range(max(0, min(nlev, 16)))]

    def results(self):
        out = []
        for t in range(self.T):
            n, r = self.shapes[t], self.ranks[t]
            G = self.G_flat[self._goff[t]:self._goff[t + 1]].view(r)
            U = self.U_flat[self._uoff[t]:self._uoff[t + 1]]
            out.append((G, _split(U, n, r)))
        return out


def rtucker_decompose_batched(Xs, ranks, p, seeds, s=None, prec="fp32"):
    """Batched Sub-R-HOSVD: one grouped launch per stage for all (tensor, mode)
    problems.  Returns a list of (G, [U_k]).  For repeated batches (and CUDA-graph
    replay, ``graph=True``) keep a ``BatchedDecomposition``."""
    return BatchedDecomposition(Xs, ranks, p, seeds, s=s, prec=prec).run().results()


def rtucker_relerr(X, G, U):
    """||X - (U_1..U_d) G||_F / ||X||_F, float64 on the device (evaluator)."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    r = [int(u.shape[1]) for u in U]
    Uc = _cat_u(U)
    Gc = G.to(torch.float32).contiguous()
    out = ctypes.c_double()
    h = _handle(X.device.index)
    _check(h, lib.rtucker_relerr(h, _ptr(X), dt, d, _i64(n), _i32(r), _ptr(Uc), _ptr(Gc), ctypes.byref(out)))
    return out.value


# ------------------------------------------------------------------ Kronecker-structured sketches
def _kron_L(ell):
    d = len(ell)
    return [_prod([ell[j] for j in range(d) if j != k]) for k in range(d)]


def kron_widths(shape, r, p=10):
    """Per-mode widths l_j for rtucker_rhkron: the smallest common l with
    l^(d-1) >= max_k r_k + p, capped so that every L_k = l^(d-1) stays within n_k
    and 64 where that is possible."""
    d = len(shape)
    rmax = max(_as_list(r, d))
    ell = 1
    while ell ** (d - 1) < rmax + p:
        ell += 1
    return [ell] * d


def rtucker_kron_sketch(X, ell, seed=0):
    """The Kronecker-structured sketches Z_k = X^(k) (kron_{j != k} Omega_j) of every
    mode from one pass over X (rHKron, Sec. 3.3); returns [Z_k] (n_k x L_k)."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    ell = _as_list(ell, d)
    L = _kron_L(ell)
    Z = torch.empty(sum(nk * lk for nk, lk in zip(n, L)), dtype=torch.float32, device=X.device)
    h = _handle(X.device.index)
    _check(h, lib.rtucker_kron_sketch(h, _ptr(X), dt, d, _i64(n), _i32(ell), ctypes.c_uint64(seed), None, _ptr(Z)))
    return _split(Z, n, L)


def rtucker_rhkron(X, r, ell, seed=0, qr="auto", core="auto"):
    """Randomized HOSVD with Kronecker-structured test matrices (rHKron, Sec. 3.3):
    one-pass sketches, their QR, the reduced core X x_k Q_k^T and its mode-wise
    factorisation; returns (G, [U_k])."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    r = _as_list(r, d)
    ell = _as_list(ell, d)
    U = torch.empty(sum(nk * rk for nk, rk in zip(n, r)), dtype=torch.float32, device=X.device)
    G = torch.empty(r, dtype=torch.float32, device=X.device)
    h = _handle(X.device.index)
    _check(h, lib.rtucker_rhkron(h, _ptr(X), dt, d, _i64(n), _i32(r), _i32(ell), ctypes.c_uint64(seed),
                                 _opts("fp32", core=core, qr=qr), _ptr(U), _ptr(G)))
    return G, _split(U, n, r)


# ------------------------------------------------------------------ Sub-R-RtL-HT
def ht_tree(d):
    """Balanced dimension tree: list of (a, b, left, right, level), node 0 the root."""
    nodes = [[0, d - 1, -1, -1, 0]]
    q = 0
    while q < len(nodes):
        a, b, _, _, lev = nodes[q]
        if a != b:
            mid = a + (b - a + 2) // 2
            nodes[q][2] = len(nodes)
            nodes.append([a, mid - 1, -1, -1, lev + 1])
            nodes[q][3] = len(nodes)
            nodes.append([mid, b, -1, -1, lev + 1])
        q += 1
    return [tuple(x) for x in nodes]


def ht_tree_from_children(children):
    """Dimension tree from a child table [(left, right), ...] (node 0 the root, (-1, -1)
    for a leaf), as the C ABI takes it: list of (a, b, left, right, level), the leaves
    holding the modes 0..d-1 in left-to-right order.  Raises ValueError for a table
    that is not a binary tree over 2d-1 nodes."""
    nn = len(children)
    if nn < 3 or nn % 2 == 0:
        raise ValueError("a dimension tree has 2d-1 >= 3 nodes")
    out = [[-1, -1, int(l), int(r), 0] for (l, r) in children]
    seen = set()

    def walk(i, lev, mode):
        if i in seen or not 0 <= i < nn:
            raise ValueError("not a tree")
        seen.add(i)
        out[i][4] = lev
        l, r = out[i][2], out[i][3]
        if (l < 0) != (r < 0):
            raise ValueError("node %d has one child" % i)
        if l < 0:
            out[i][0] = out[i][1] = mode
            return mode + 1
        m = walk(l, lev + 1, mode)
        m = walk(r, lev + 1, m)
        out[i][0], out[i][1] = out[l][0], out[r][1]
        return m

    walk(0, 0, 0)
    if len(seen) != nn:
        raise ValueError("not every node is reachable from the root")
    return [tuple(x) for x in out]


def _tree_args(d, tree):
    """(node tuples, child-table pointer for the C ABI or None) of ``tree``: None for
    the balanced tree, else a child table [(left, right), ...]."""
    if tree is None:
        return ht_tree(d), None
    nodes = ht_tree_from_children(tree)
    if len(nodes) != 2 * d - 1:
        raise ValueError("the tree must have 2d-1 = %d nodes" % (2 * d - 1))
    return nodes, _i32([v for lr in tree for v in lr])


def ht_alpha_w(shape, alpha, tree=None):
    """Samples per node by the alpha rule, w_S = min(floor(alpha^(d-2) n_S), n_{notin S})
    (n_S rows of the node's unfolding; the root entry is 0), for the ``w`` argument of
    ``rhtucker_decompose`` (balanced tree, or the child table ``tree``)."""
    d = len(shape)
    total = _prod(shape)
    scale = float(alpha) ** (d - 2)
    out = []
    nodes, _ = _tree_args(d, tree)
    for i, (a, b, _, _, _) in enumerate(nodes):
        rows = _prod(shape[a:b + 1])
        out.append(0 if i == 0 else min(int(scale * rows), total // rows))
    return out


def _ht_ranks(d, rank):
    nn = 2 * d - 1
    rk = _as_list(rank, nn) if isinstance(rank, (list, tuple)) else [int(rank)] * nn
    rk[0] = 1
    return rk


def rhtucker_decompose(X, rank, p, w=None, seed=0, return_nodes=False, graph=False, out=None, tree=None,
                       qr="auto"):
    """Sub-R-RtL-HT (Alg. 2) on the dimension tree ``tree`` (a child table
    [(left, right), ...], node 0 the root, (-1, -1) for leaves; None = the balanced
    tree).  Returns (U_leaf list, B dict node -> transfer tensor) and, with
    ``return_nodes``, the node bases U_S.  ``graph`` replays the kernel sequence as a
    CUDA graph for repeated calls with the same buffers and shapes
    (rt_options.use_graph); ``out`` = (U_leaf flat, B flat[, U_nodes flat]) reuses
    output buffers so that their pointers repeat."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    nodes, tab = _tree_args(d, tree)
    rk = _ht_ranks(d, rank)
    nrows = [_prod(n[a:b + 1]) for (a, b, _, _, _) in nodes]
    leaves = sorted((i for i, t in enumerate(nodes) if t[0] == t[1]), key=lambda i: nodes[i][0])
    internal = [i for i, t in enumerate(nodes) if t[0] != t[1]]
    Bsz = [rk[i] * rk[nodes[i][2]] * rk[nodes[i][3]] for i in internal]
    Un = None
    if out is not None:
        Ul, B = out[0], out[1]
        if return_nodes:
            Un = out[2]
    else:
        Ul = torch.empty(sum(n[nodes[i][0]] * rk[i] for i in leaves), dtype=torch.float32, device=X.device)
        B = torch.empty(sum(Bsz), dtype=torch.float32, device=X.device)
        if return_nodes:
            Un = torch.empty(sum(nrows[i] * rk[i] for i in range(1, len(nodes))), dtype=torch.float32,
                             device=X.device)
    h = _handle(X.device.index)
    wp = _i64(_as_list(w, len(nodes))) if w is not None else None
    _check(h, lib.rhtucker_decompose(h, _ptr(X), dt, d, _i64(n), tab, _i32(rk), int(p), wp,
                                     ctypes.c_uint64(seed), _opts("fp32", graph=graph, qr=qr), _ptr(Ul), _ptr(B),
                                     _ptr(Un)))
    U_leaf = _split(Ul, [n[nodes[i][0]] for i in leaves], [rk[i] for i in leaves])
    Bd, off = {}, 0
    for i, sz in zip(internal, Bsz):
        Bd[i] = B[off:off + sz].view(rk[i], rk[nodes[i][2]], rk[nodes[i][3]])
        off += sz
    if return_nodes:
        Ud = dict(zip(range(1, len(nodes)), _split(Un, nrows[1:], rk[1:])))
        return U_leaf, Bd, Ud
    return U_leaf, Bd


def rhtucker_relerr(X, U_leaf, B, rank, tree=None):
    """Relative error of an H-Tucker result (on the same ``tree`` as its
    decomposition) against X, float64 on the device."""
    lib = load_library()
    dt, d, n = _tensor_args(X)
    nodes, tab = _tree_args(d, tree)
    rk = _ht_ranks(d, rank)
    internal = [i for i, t in enumerate(nodes) if t[0] != t[1]]
    Uc = _cat_u(U_leaf)
    Bc = torch.cat([B[i].reshape(-1) for i in internal]).to(torch.float32).contiguous()
    out = ctypes.c_double()
    h = _handle(X.device.index)
    _check(h, lib.rhtucker_relerr(h, _ptr(X), dt, d, _i64(n), tab, _i32(rk), _ptr(Uc), _ptr(Bc),
                                  ctypes.byref(out)))
    return out.value


def rhtucker_root_transfer_noalloc(X, Ul, Ur, out=None):
    """Root transfer tensor U_l^T X_mat U_r (1 x r_l x r_r) without any device
    allocation by the library (its scratch is a fixed static device array).
    ``out`` must be preallocated by callers that cannot allocate either.  X is
    viewed as an n_l x n_r matrix (n_l, n_r the rows of Ul and Ur)."""
    lib = load_library()
    dt, _, _ = _tensor_args(X)
    if Ul.dim() != 2 or Ur.dim() != 2:
        raise ValueError("Ul and Ur must be matrices")
    nl, rl = int(Ul.shape[0]), int(Ul.shape[1])
    nr, rr = int(Ur.shape[0]), int(Ur.shape[1])
    if X.numel() != nl * nr:
        raise ValueError("X has %d elements, Ul and Ur need n_l * n_r = %d" % (X.numel(), nl * nr))
    for name, t in (("Ul", Ul), ("Ur", Ur)):
        if t.dtype != torch.float32 or not t.is_contiguous() or t.device != X.device:
            raise ValueError("%s must be a contiguous float32 tensor on X's device" % name)
    if out is None:
        out = torch.empty((1, rl, rr), dtype=torch.float32, device=X.device)
    elif (out.dtype != torch.float32 or not out.is_contiguous() or out.device != X.device
          or tuple(out.shape) != (1, rl, rr)):
        raise ValueError("out must be a contiguous float32 tensor of shape (1, %d, %d) on X's device" % (rl, rr))
    st = lib.rhtucker_root_transfer_noalloc(_ptr(X), dt, nl, nr, _ptr(Ul), rl, _ptr(Ur), rr, _ptr(out),
                                            ctypes.c_void_p(torch.cuda.current_stream(X.device).cuda_stream))
    if st != 0:
        raise RtError(st, lib.rt_status_string(st).decode())
    return out


# ----------------------------------------------------------------- failure handling
FAULT_ALLOC = 1


def set_wait_limit(polls=0, device=None):
    """Poll limit of the library's bounded mbarrier waits on ``device`` (0 = default)."""
    h = _handle(device)
    _check(h, load_library().rt_set_wait_limit(h, int(polls)))


def selftest_wait(device=None):
    """Enqueue the bounded-wait self-test (a wait nothing ends); ``sync()`` then
    raises RtError with status RT_ETIMEOUT once the poll limit has run out."""
    h = _handle(device)
    _check(h, load_library().rt_selftest_wait(h))


def inject_fault(kind=FAULT_ALLOC, count=1, device=None):
    """The handle's next ``count`` workspace growths fail as a failed cudaMalloc."""
    h = _handle(device)
    _check(h, load_library().rt_inject_fault(h, int(kind), int(count)))
