/*
 * rtucker.h - C ABI of the GB300 (sm_103a) library for the subsampled
 * randomized Tucker and H-Tucker decompositions of arXiv 2603.21379
 * ("A practical mode-parallel implementation of the (H-)Tucker decomposition
 * via randomization").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Tensors are dense and in C order (last mode fastest).  Modes are numbered
 *   0..d-1 (the paper numbers them 1..d).  The mode-k unfolding X^(k) of
 *   Sec. 2.2 uses the natural (C-order) linear index of the other modes for its
 *   columns; the set unfolding X^(S) of a contiguous mode range S has the
 *   C-order index over S as rows.
 * - Pointers named X, Z, U, G, B, idx are DEVICE pointers owned by the caller;
 *   size arrays (n, r, s, w, rank) are HOST arrays.  Outputs are float32,
 *   row-major.  X must be aligned to its element size.
 * - Calls are asynchronous on the handle's stream.  The returned status covers
 *   argument checks and launches.  Errors found on the device (a bounded loop
 *   that ran out, a numerical breakdown) are recorded in a device status word
 *   and returned by rt_sync() or by the next call on the handle.
 * - Workspace: the handle owns one device workspace (cudaMalloc), grown on
 *   demand and freed by rt_destroy().  A failed allocation returns RT_ENOMEM
 *   and leaves the outputs untouched.  There is no CPU fallback: every step of
 *   the computation runs in the library's CUDA kernels.
 * - Random streams: fiber indices and Gaussian test matrices are drawn from a
 *   64-bit seed with Philox4x32-10 (Salmon et al., SC'11): the sample of
 *   column indices is a keyed Feistel permutation of [0, N) restricted by
 *   cycle-walking (uniform without repetition, Sec. 3.1), and entry (j, c) of
 *   Omega is the Box-Muller normal keyed by the sampled column index pi(j) and
 *   c.  Stream id "node" = mode k for Tucker, the dimension-tree node id for
 *   H-Tucker.
 */
#ifndef RTUCKER_H
#define RTUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_EINVAL = 1,    /* an argument is out of range (message in rt_last_error) */
  RT_ENOMEM = 2,    /* device workspace allocation failed                      */
  RT_ECUDA = 3,     /* a CUDA runtime call or launch failed                    */
  RT_ETIMEOUT = 4,  /* a bounded device loop ran out (status word)             */
  RT_EDEVICE = 5,   /* a device-side check failed (status word)                */
  RT_ENUMERIC = 6,  /* numerical breakdown (non-finite value) on the device     */
  RT_ENOTSUP = 7    /* valid but unsupported combination                       */
} rt_status;

/* Storage type of X.  RT_F8E4M3 is a packed float8 form made by rt_quantize_fp8:
 * one E4M3 byte per element (C order; 1 sign, 4 exponent bits with bias 7,
 * 3 mantissa bits, no infinity) followed, at byte offset rt_fp8_scale_offset,
 * by one float32 scale per slab of the last two modes (X[i_0..i_{d-3}, :, :],
 * slab index in C order; the whole matrix when d = 2).  Element value = code
 * value x its slab's scale.  The buffer is rt_fp8_bytes long and 16-byte
 * aligned.  Entry points that take it: rtucker_sketch, rtucker_factors,
 * rtucker_core, rtucker_decompose and rtucker_relerr, for shapes the tensor-core
 * pass over X takes (n_{d-2} <= 128, n_{d-1} a multiple of 16, r_{d-2} <= 64,
 * r_{d-1} <= 32); RT_ENOTSUP for other shapes and other entry points. */
typedef enum { RT_F32 = 0, RT_F64 = 1, RT_BF16 = 2, RT_F8E4M3 = 3 } rt_dtype;

typedef enum {
  RT_PREC_FP32 = 0, /* float32-accurate arithmetic throughout (default)         */
  RT_PREC_BF16 = 1  /* BF16 compute form: in the tensor-core pass over a float32
                       X, X is rounded to one bfloat16 term (the factors and the
                       intermediate keep two terms; float32 accumulate).  The
                       range finder still computes in float32.  Tucker entry
                       points only; shapes the tensor-core pass cannot take run
                       in float32.  rhtucker_* return RT_ENOTSUP.             */
} rt_prec;

typedef struct rt_handle_s* rt_handle;

typedef struct {
  int32_t prec;        /* rt_prec                                              */
  int32_t use_graph;   /* 1: run the call's kernel sequence as a CUDA graph.
                          The sequence is captured on a stream of the handle's
                          own (so the caller's stream may be the legacy default
                          stream), instantiated and launched on the handle's
                          stream; later calls whose launch-shaping arguments
                          match (pointers, shapes, ranks, p, sample counts,
                          workspace) replay it.  The problem tables, seeds
                          included, are uploaded by every call.  Up to 4
                          sequences are cached per handle; stage timing
                          (rt_set_timing) turns capture off.  rtucker_decompose,
                          rtucker_factors, rtucker_decompose_batched,
                          rhtucker_decompose.  0 (default): direct launches.
                          Other values: RT_EINVAL.                              */
  int32_t overlap;     /* rtucker_decompose only: 1 runs the pass over X on the
                          QR factors Q of the last two modes (U_k = Q_k W_k) on
                          the tensor cores while the SVD / W / U part of their
                          range finder runs beside it on a second stream, then
                          contracts with W; 0 (default) waits for U.  Same
                          result up to rounding.  Shapes the tensor-core pass
                          cannot take ignore it.                                 */
  int32_t core;        /* kernels of the core contraction (rtucker_decompose,
                          rtucker_core): 0 (default) auto: the tensor-core pass
                          over X for slabs of at least 64 x 64 (last two modes),
                          after it the remaining one-mode contractions on the
                          tensor cores too where n_k <= 128 and r_k <= 64;
                          two-mode FFMA passes over small slabs that fit shared
                          memory, one-mode FFMA contractions otherwise; 1 the
                          tensor-core pass whenever the shape allows it; 2 FFMA
                          kernels only; 3 tune: on the first call for a shape
                          (d, n, r, dtype, prec) choices 1 and 2 are each timed
                          with CUDA events on the call's own buffers (the call
                          synchronises its stream once) and the faster is kept
                          in the handle for later calls.  Same result up to
                          rounding.  rtucker_decompose_batched: 3 times each
                          contraction level's schedules instead (grouped tiles,
                          or one row per lane with 1..16 row blocks per CTA;
                          see rt_last_schedule); other values its defaults.    */
  int32_t qr;          /* factorisations of the range finder (S5 and the W-step
                          of S6, Alg. 1 / Alg. 2).  For unfoldings of at most 256
                          rows with (n_S | 1)(r + p) <= 12288: 1 Householder QR
                          of Z and a TSQR of B^T = Y^T Q; 2 Cholesky form of
                          both: Z = Q R by CholeskyQR2 whose first Gram Z^T Z is
                          summed in double-float (two float32 words; GB300's
                          float64 rate is ~1/64 of float32), falling back to
                          Householder when Z is rank-deficient to rounding, and
                          the R factor of B^T from the Cholesky factor of the
                          Gram B B^T (compensated float32 sums of the rounded
                          products); 3 as 2 with Z = Q R by shifted CholeskyQR3
                          (Fukaya et al., SIAM J. Sci. Comput. 2020): a first
                          pass on Z^T Z + s I, s = 11 (m c + c (c + 1)) 2^-24
                          ||Z||_F^2 (m rows, c = r + p columns), which cannot
                          break down for cond(Z) up to about 2^24, then two
                          CholeskyQR passes (the Householder fallback stays for
                          a Z that is rank-deficient to rounding); 0 (default)
                          Householder QR of Z with the Cholesky form of the
                          W-step (the fastest measured).
                          Larger unfoldings always take 1.  The one-sided Jacobi
                          SVD of R^T is the same in all; same factors to
                          rounding.                                            */
  int32_t sketch;      /* 0 (default) float32 sketch Z = Y Omega; 1 BF16 sketch:
                          Y and Omega rounded to bfloat16 (float32 accumulate)
                          for Z only (the W-step and the core use the float32
                          fibers), with Z's QR by the CholeskyQR2 of qr = 2
                          unless qr = 1.  The rounding (2^-8 relative) can hide
                          directions whose share of the sampled fibers lies
                          below it; the benchmark reports its error.  Tucker
                          entry points.                                        */
  int32_t reserved[2]; /* must be zero                                          */
} rt_options;

/* ----------------------------------------------------------- handle
 * rt_create: new handle bound to `stream` (a cudaStream_t; NULL = legacy
 * default stream) on the current device.  rt_destroy waits for the handle's
 * work and frees its workspace, staging buffers and captured graphs.
 * rt_set_stream: later calls enqueue on `stream` (the caller orders it after
 * any earlier work of the handle).  rt_sync waits for the stream and returns
 * the device status word (then clears it).  rt_last_error: message of the last
 * failure on this handle (owned by the handle, valid until its next call). */
rt_status rt_create(rt_handle* h, void* stream);
rt_status rt_destroy(rt_handle h);
rt_status rt_set_stream(rt_handle h, void* stream);
rt_status rt_sync(rt_handle h);
const char* rt_last_error(rt_handle h);
const char* rt_status_string(rt_status s);
int rt_version(void);
/* Number of kernel launches the last rtucker_ / rhtucker_ call enqueued. */
int rt_last_launch_count(rt_handle h);
/* Bytes of device workspace currently held by the handle. */
size_t rt_workspace_bytes(rt_handle h);
/* Stage timing.  While enabled, the library records CUDA events on the
 * handle's stream around the stages of every call and accumulates the elapsed
 * times.  rt_get_timing synchronises the stream and writes, for stage
 * i < min(nmax, RT_NSTAGES), the total milliseconds ms[i] and the number of
 * timed intervals count[i] since the last reset (reset = 1 clears them).
 * Stages: 0 range finder (S1-S6; S1-S5 and the B-step of S6 when stage 5 is
 * split off), 1 first contraction of the core (the pass over X), 2 remaining
 * core contractions, 3 H-Tucker transfer tensors, 4 H-Tucker root pass (the
 * pass over X), 5 SVD/W/U part of S6 when it runs on the handle's second stream
 * beside the pass over X (timed on that stream; overlaps stage 1). */
#define RT_NSTAGES 6
rt_status rt_set_timing(rt_handle h, int enable);
rt_status rt_get_timing(rt_handle h, double* ms, int64_t* count, int nmax, int reset);

/* ----------------------------------------------------------- failure handling
 * Not part of the paper's method: the library's own failure paths, made
 * testable without faulting or hanging a GPU.
 *
 * rt_set_wait_limit: poll limit of every bounded mbarrier wait in the library's
 * TMA pipelines (the tensor-core pass over X, the streaming root pass), for the
 * device of `h` and every handle on it (0 = the default, 2^22 polls).  A wait
 * that runs out records RT_ETIMEOUT in the handle's status word (returned by
 * rt_sync or the next call), its CTA stops and frees what it holds, and the
 * context stays usable.  Synchronous; not while a call of another handle on
 * the device is running.
 * rt_selftest_wait: enqueues one CTA that waits, through that bounded wait, on a
 * barrier nothing arrives on: rt_sync(h) then returns RT_ETIMEOUT (after the
 * limit's polls; use a small limit) and clears the status word.
 * rt_inject_fault(h, RT_FAULT_ALLOC, count): the handle's next `count` device
 * workspace growths fail exactly as a failed cudaMalloc does (RT_ENOMEM, the
 * outputs untouched, nothing enqueued); count 0 clears.  The environment
 * variable RT_FAULT=alloc[:count] sets the same for every new handle. */
#define RT_FAULT_ALLOC 1
rt_status rt_set_wait_limit(rt_handle h, uint32_t polls);
rt_status rt_selftest_wait(rt_handle h);
rt_status rt_inject_fault(rt_handle h, int kind, int count);

/* ----------------------------------------------------------- Sub-R-HOSVD
 * Shared arguments (Alg. 1 inputs):
 *   X      device, d-way C-order tensor of sizes n[0..d-1], storage `dtype`;
 *   d      order, 2 <= d <= 16;  n[k] >= 1, prod n < 2^62;
 *   r      ranks r[k] >= 1 (host);   p  oversampling >= 0;
 *   s      samples per mode (host) or NULL for s_k = min(10 n_k, n_{!=k})
 *          (the paper's rule of thumb s_k >= 10 n_k, Sec. 3.2);
 *   seed   64-bit seed of the random streams;  opt  NULL = defaults.
 * Rules (Alg. 1 and the Sub-R-HOSVD error bound, Sec. 3.2): r_k + p <= n_k,
 * r_k + p <= n_{!=k}, r_k + p <= s_k <= n_{!=k}; else RT_EINVAL.
 */

/* S1 - fiber sample (Sec. 3.1): idx = concat_k pi_k[0..s_k-1], int64, the
 * sampled column indices of X^(k) (distinct, in [0, n_{!=k})).  No X needed. */
rt_status rtucker_indices(rt_handle h, int d, const int64_t* n, const int64_t* s, uint64_t seed,
                          int64_t* idx);

/* S1-S4 - sketch Z_k = Y_k Omega_k = X^(k) E_k Omega_k (Sec. 3.1, Alg. 1):
 * Z = concat_k of n_k x (r_k + p) row-major blocks. */
rt_status rtucker_sketch(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                         const int32_t* r, int32_t p, const int64_t* s, uint64_t seed,
                         const rt_options* opt, float* Z);

/* S1-S6 - factors U_k = Q_k W_k (Alg. 1): Q_k the orthonormal factor of the
 * thin QR of Z_k with diag(R) > 0, W_k the dominant r_k left singular vectors
 * of Q_k^T Y_k.  U = concat_k of n_k x r_k row-major blocks; each column's
 * largest-magnitude entry is positive (ties: lowest row).  sigma (optional,
 * may be NULL): concat_k of the r_k + p singular values of Q_k^T Y_k. */
rt_status rtucker_factors(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                          const int32_t* r, int32_t p, const int64_t* s, uint64_t seed,
                          const rt_options* opt, float* U, float* sigma);

/* S7 - core G = X x_1 U_1^T ... x_d U_d^T (Alg. 1, core step): U as returned
 * by rtucker_factors (any n_k x r_k blocks), G the r_0 x ... x r_{d-1} C-order
 * core. */
rt_status rtucker_core(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                       const int32_t* r, const float* U, const rt_options* opt, float* G);

/* S1-S7 - the whole Sub-R-HOSVD (Alg. 1): factors then core in one call. */
rt_status rtucker_decompose(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                            const int32_t* r, int32_t p, const int64_t* s, uint64_t seed,
                            const rt_options* opt, float* U, float* G);

/* Same as rtucker_decompose (Alg. 1) with X, U and G in HOST memory (pinned
 * memory recommended): X is copied to device workspace, the decomposition
 * runs, and U and G are copied back; the call returns after the copies
 * completed. */
rt_status rtucker_decompose_host(rt_handle h, const void* X_host, rt_dtype dtype, int d,
                                 const int64_t* n, const int32_t* r, int32_t p, const int64_t* s,
                                 uint64_t seed, const rt_options* opt, float* U_host, float* G_host);

/* Pipelined form of rtucker_decompose_host for a stream of tensors.  The call
 * enqueues the copy of X_host into one of two device input slots on the
 * handle's copy stream, the decomposition on the handle's stream after that
 * copy, and the copies of U and G into U_host / G_host after it, and returns
 * without waiting, so the copy of the next call's X runs while this call
 * decomposes.  X_host, U_host and G_host must stay allocated and X_host
 * unmodified until rt_sync(h) returns (after an error return X_host is no
 * longer read); with pageable memory the copies are
 * correct but do not overlap (pinned memory recommended).  Argument checks
 * are those of rtucker_decompose; device-side failures are reported by
 * rt_sync.  The two slots (2 x the tensor's bytes) and the outputs live in a
 * handle-owned device allocation that grows on demand (RT_ENOMEM if it
 * cannot). */
rt_status rtucker_decompose_host_async(rt_handle h, const void* X_host, rt_dtype dtype, int d,
                                       const int64_t* n, const int32_t* r, int32_t p, const int64_t* s,
                                       uint64_t seed, const rt_options* opt, float* U_host, float* G_host);

/* Batched Sub-R-HOSVD (Alg. 1 for each tensor; the modes of all tensors are
 * independent problems, as the modes of one are in Sec. 3.3): T independent
 * tensors (tensor t: X[t], order d[t], sizes n[t][.], ranks r[t][.], samples
 * s[t] or s == NULL / s[t] == NULL for the default, seed seeds[t]) decomposed
 * with one grouped launch per stage for all (tensor, mode) problems and one per
 * contraction level of the cores.  X, U, G: HOST arrays of DEVICE pointers
 * (U[t] and G[t] laid out as for rtucker_decompose); argument errors of any
 * tensor fail the whole call before anything is enqueued. */
rt_status rtucker_decompose_batched(rt_handle h, int T, const void* const* X, rt_dtype dtype,
                                    const int32_t* d, const int64_t* const* n,
                                    const int32_t* const* r, int32_t p,
                                    const int64_t* const* s, const uint64_t* seeds,
                                    const rt_options* opt, float* const* U, float* const* G);

/* ----------------------------------------------------- differentiable Tucker
 * Gradients of the Tucker format (Sec. 3: X ~ Xhat = G x_1 U_1 ... x_d U_d) for
 * training through a decomposition; an extension of the paper (not in it).
 *
 * rtucker_loss_grad: the misfit L = 1/2 ||X - Xhat||_F^2 and its gradients
 *   dX = R = X - Xhat                          (n_1 x ... x n_d, C order)
 *   dG = -R x_1 U_1^T ... x_d U_d^T            (r_1 x ... x r_d, C order)
 *   dU = concat_n -[R x_{m != n} U_m^T]_(n) G_(n)^T   (n_n x r_n row-major each)
 * X: DEVICE tensor (float32 / float64 / bfloat16); U (concat n_k x r_k) and G:
 * DEVICE float32, e.g. the outputs of rtucker_decompose.  Outputs (DEVICE,
 * caller-owned, each may be NULL): loss (one float64), dX, dG, dU (float32).
 * Without dX the residual lives in handle workspace (prod n floats) while dG
 * or dU are formed.  1 <= r_k <= 64.  Asynchronous on the handle's stream.
 * Arithmetic: float32 with the residual's squared norm summed in float32 per
 * thread and tile and in float64 across tiles and CTAs. */
rt_status rtucker_loss_grad(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                            const int32_t* r, const float* U, const float* G, double* loss, float* dX,
                            float* dG, float* dU);

/* Adjoint of the core projection G = X x_1 U_1^T ... x_d U_d^T (the core step of
 * Alg. 1): for an upstream gradient Gbar (r_1 x ... x r_d, DEVICE float32),
 *   Xbar = Gbar x_1 U_1 ... x_d U_d                    (n_1 x ... x n_d)
 *   Ubar = concat_n [X x_{m != n} U_m^T]_(n) Gbar_(n)^T  (n_n x r_n each)
 * Xbar and Ubar: DEVICE float32, caller-owned, either may be NULL.  Other
 * arguments and conventions as rtucker_loss_grad. */
rt_status rtucker_core_adjoint(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                               const int32_t* r, const float* U, const float* Gbar, float* Xbar,
                               float* Ubar);

/* rt_last_schedule: the per-level schedules of the core contractions of the last
 * rtucker_decompose_batched call on h (level k contracts mode d_t - 1 - k of every
 * tensor): 0 = generic grouped tiles (32 output rows x 128 columns), b > 0 = one row
 * per lane, b 128-row blocks per CTA.  With rt_options.core = 3 the batched call picks
 * each level's schedule among these by timing them once per set of shapes on its own
 * buffers (cached in the handle); otherwise the defaults are 8 row blocks where the
 * row form applies (every job a last-mode contraction of <= 256 rows into <= 32
 * columns) and the tiles elsewhere.  Writes min(levels, cap) entries to out (HOST)
 * and returns the number of levels (0 before any batched call, -1 for a null h). */
int rt_last_schedule(rt_handle h, int32_t* out, int cap);

/* rt_set_grad_recompute(h, 1): rtucker_loss_grad and rtucker_core_adjoint (for dU /
 * Ubar) recompute the prefix contractions P_m = T x_0 U_0^T ... x_{m-1} U_{m-1}^T of
 * every partial projection instead of keeping them in workspace: the handle's
 * workspace drops by sum_k P_k (about r_0 / n_0 of the tensor for the largest), at
 * the cost of d (d - 1) / 2 instead of d - 1 prefix contractions (re-reading T).
 * Same results up to rounding order (identical here: the same kernels in the same
 * order per chain).  0 (default) keeps them.  RT_EINVAL for other values. */
rt_status rt_set_grad_recompute(rt_handle h, int enable);

/* ------------------------------------------------------- float8 storage of X
 * The FP8 form of the pass over X (an extension of Alg. 1, which computes in the
 * input's precision): X stored as E4M3 bytes with one power-of-two scale per slab
 * of the last two modes, a quarter of float32's bytes.  The decomposition of the
 * packed tensor is that of its stored values (code x scale), computed with the
 * float32-level arithmetic of the plain form; the storage error itself is the
 * rounding of X to the E4M3 grid (at most 2^-4 relative for elements above 2^-14
 * of their slab's largest magnitude).
 *
 * rt_fp8_bytes: size in bytes of the packed buffer of a tensor of order d and
 * sizes n (0 for invalid sizes).  rt_fp8_scale_offset: byte offset of its scales
 * (the element count rounded up to 256). */
size_t rt_fp8_bytes(int d, const int64_t* n);
size_t rt_fp8_scale_offset(int d, const int64_t* n);

/* rt_quantize_fp8: pack the DEVICE tensor X (float32 / float64 / bfloat16, C
 * order) into the DEVICE buffer Xq (rt_fp8_bytes, 16-byte aligned, caller-owned).
 * Per slab: amax = max |x|, written amax = f 2^e with 0.5 <= f < 1 (e = 0 for an
 * all-zero slab); the scale is 2^(e-8), so |x| / scale < 256; each code is the
 * E4M3 value nearest to x / scale, ties to the even mantissa (the division by a
 * power of two is exact, so the rounding decision is exact).  X must be finite.
 * Asynchronous on the handle's stream; allocates nothing. */
rt_status rt_quantize_fp8(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, void* Xq);

/* -------------------------------------------- Kronecker-structured sketches
 * The rHKron comparison method of Sec. 3.3 (Minster et al.): randomized HOSVD
 * whose mode-k test matrix is the Kronecker product of small per-mode Gaussians,
 * so that one pass over X forms every mode's sketch.
 *
 * rtucker_kron_sketch: Omega_j (n_j x l_j, j = 0..d-1) Gaussian, entry (i, a) the
 * Box-Muller normal of Philox4x32-10 counter (i, a, (3 << 16) | j) with the seed as
 * key; Z_k = X^(k) (Omega_0 (x) .. (x) Omega_{k-1} (x) Omega_{k+1} (x) .. (x) Omega_{d-1}),
 * the unfolding along k of X x_{j != k} Omega_j^T, n_k x L_k with L_k =
 * prod_{j != k} l_j, columns in natural (C) order of the other modes.  Z =
 * concat_k of the n_k x L_k row-major blocks (DEVICE float32).  One read of X (the
 * slabs of its last two modes) forms all d sketches.  ell: HOST int32[d], 1 <= l_j
 * <= n_j.  Supported (else RT_ENOTSUP): d >= 3, l_{d-2}, l_{d-1} <= 8, n_{d-1} a
 * multiple of 4, n_{d-2}, n_{d-1} <= 1024, n_{d-2} L_{d-2} and n_{d-1} L_{d-1} at
 * most 8192, the slab (plus its double buffer) within shared memory.  float32 X
 * must be 16-byte aligned.  Arithmetic: float32 FMAs; the CTAs' partial sums are
 * added in a fixed order (deterministic). */
rt_status rtucker_kron_sketch(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                              const int32_t* ell, uint64_t seed, const rt_options* opt, float* Z);

/* rtucker_rhkron: Tucker factors U (concat n_k x r_k, DEVICE float32, the
 * column-sign rule applied) and core G (r_0 x .. x r_{d-1}, C order) by
 *   1. the sketches Z_k of rtucker_kron_sketch;
 *   2. Q_k = orthonormal factor of the thin QR of Z_k (diag(R) > 0);
 *   3. the reduced tensor C = X x_0 Q_0^T .. x_{d-1} Q_{d-1}^T (L_0 x .. x L_{d-1});
 *   4. W_k = dominant r_k left singular vectors of C^(k) for every mode at once
 *      (the paper's rHKron takes an ST-HOSVD of C; the modes are factored
 *      independently here, as in T-HOSVD, so that they run in parallel);
 *   5. U_k = Q_k W_k and G = C x_k W_k^T (= X x_k U_k^T).
 * Needs r_k <= L_k <= min(n_k, 64) and the shapes rtucker_kron_sketch takes.
 * rt_options: qr applies to step 4; core to steps 3 and 5. */
rt_status rtucker_rhkron(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                         const int32_t* ell, uint64_t seed, const rt_options* opt, float* U, float* G);

/* Relative reconstruction error ||X - (U_1..U_d) G||_F / ||X||_F computed on
 * the device in float64 (evaluator; not part of the decomposition; Sec. 3.3
 * reports this measure).  G (r_1 x ... x r_d, C order) and the concatenated
 * U_k (n_k x r_k row-major) are device float32.  The last two modes are formed
 * per slab when r_{d-1} n_d doubles fit 200 KB, else mode d-1 is expanded as
 * well and the rows of n_d are measured against U_d (r_d <= 64; RT_ENOTSUP
 * beyond).  The result is written to *out (HOST) after the call synchronises
 * the stream. */
rt_status rtucker_relerr(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                         const int32_t* r, const float* U, const float* G, double* out);

/* ----------------------------------------------------------- Sub-R-RtL-HT
 * rhtucker_decompose: Sub-R-RtL-HT(X, T, r, w, p) (Alg. 2) on the dimension
 * tree T (Sec. 4: a binary tree whose root holds every mode, whose leaves are
 * single modes, and whose internal nodes are the disjoint union of their two
 * children).  The tree has 2d-1 nodes.
 *   tree        host child table of 2 (2d-1) int32: tree[2i], tree[2i+1] are the
 *               left and right child ids of node i, both -1 for a leaf; node 0 is
 *               the root.  The leaves hold the modes 0..d-1 in left-to-right
 *               order, so every node is a contiguous mode range {a..b} whose left
 *               child holds the first modes (natural order: the rows of the set
 *               unfolding X^(S) and of U_{S_l} (x) U_{S_r} are C-order with the
 *               left child slower).  Node ids are free otherwise; the id is the
 *               node's random-stream id.  RT_EINVAL for a table that is not such
 *               a tree.  NULL: the balanced tree (node {a..b} splits into its
 *               first ceil(len/2) modes and the rest; nodes numbered level by
 *               level, left to right: for d = 8 the paper's heap numbering, root
 *               0, leaves 7..14).
 *   rank[node]  rank per node (host, 2d-1 entries; rank[0] is ignored: the
 *               root rank is 1);  p oversampling;
 *   w[node]     samples per node (host) or NULL for
 *               w_S = min(20 max_k n_k, n_{notin S}) (the paper's 20 n fibers
 *               per node, Sec. 4.2);
 *   U_leaf      device, concat over leaves (mode order) of n_k x rank_k;
 *   B           device, concat over internal nodes in id order of the
 *               transfer tensors r_S x r_{S_l} x r_{S_r} (C order), the root's
 *               first (1 x r_{R_l} x r_{R_r});
 *   U_nodes     device or NULL: concat over non-root nodes in id order of the
 *               node bases U_S (n_S x r_S).
 * Rules: r_S + p <= min(n_S, n_{notin S}), r_S + p <= w_S <= n_{notin S}
 * and r_S + p <= 64 (RT_EINVAL / RT_ENOTSUP otherwise).  Transfer tensors whose
 * ranks are all at most 12 (the paper uses 10) take one grouped kernel that
 * keeps r x r x r blocks on chip; wider ones take two mode contractions and a
 * permutation.  A root right-child rank above 12 costs one pass over X per
 * chunk of at most 12 columns of U_{R_r} (ceil(r / 12) passes). */
rt_status rhtucker_decompose(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                             const int32_t* tree, const int32_t* rank, int32_t p, const int64_t* w,
                             uint64_t seed, const rt_options* opt, float* U_leaf, float* B, float* U_nodes);

/* Relative error ||X - X_hat||_F / ||X||_F of the H-Tucker format (U_leaf, B,
 * laid out as rhtucker_decompose writes them for the same `tree`, NULL =
 * balanced) against X, with X_hat rebuilt through the nested node bases
 * (Sec. 4); float64 on the device; *out (HOST) written after the call
 * synchronises.  Ranks 1..64. */
rt_status rhtucker_relerr(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                          const int32_t* tree, const int32_t* rank, const float* U_leaf, const float* B,
                          double* out);

/* ----------------------------------------------------------- without allocation
 * rhtucker_root_transfer_noalloc: the root transfer tensor of an H-Tucker
 * format, BR(0, j, k) = sum_{a,b} X[a nr + b] Ul[a][j] Ur[b][k] (X viewed as an
 * nl x nr matrix; Ul nl x rl, Ur nr x rr row-major; BR 1 x rl x rr), for
 * callers that cannot allocate device memory (stream capture in global mode,
 * frameworks that own all device memory, loops that must avoid the implicit
 * synchronisation of cudaMalloc/cudaFree).  The paper has no counterpart: it
 * is this library's allocation-free form of the root pass of
 * rhtucker_decompose.  It runs the tiled root kernel of rhtucker_decompose (which
 * streams float32 X through TMA where the shape allows); results agree with
 * rhtucker_decompose to float32 rounding.
 *   - Allocates nothing: no handle, no workspace.  Its scratch is a static
 *     device array of RT_ROOT_NOALLOC_MAX_PARTIALS floats (4 MiB) that every
 *     GPU loading the library holds until the process exits.  The call needs
 *     ceil(nr / 8192) * ceil(nl / 512) * rl * rr of them; larger problems, or
 *     rr > 12, return RT_ENOTSUP.  Null pointers, an unknown dtype or sizes out
 *     of range (nl, nr, rl, rr < 1; nl > 2^31; nr > 2^40) return RT_EINVAL.
 *   - X (nl * nr elements of `dtype`, C order), Ul, Ur (float32) and BR
 *     (float32, rl * rr) are device pointers owned by the caller; `stream` is a
 *     cudaStream_t (NULL = legacy default stream).  Asynchronous on `stream`.
 *   - RT_ECUDA if a CUDA call of its own fails (the error stays pending in the
 *     runtime; errors pending before the call are neither reported nor cleared).
 *   - The first call on a device resolves the device address of the static
 *     array (cudaGetSymbolAddress) with that device current; make that first
 *     call before any stream capture.
 *   - Every call shares the one array: calls whose kernels overlap on the GPU
 *     (other streams, other host threads) race on it. */
#define RT_ROOT_NOALLOC_MAX_PARTIALS (1u << 20)
rt_status rhtucker_root_transfer_noalloc(const void* X, rt_dtype dtype, int64_t nl, int64_t nr,
                                         const float* Ul, int32_t rl, const float* Ur, int32_t rr,
                                         float* BR, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RTUCKER_H */
