// rt_common.cuh - shared device-side definitions of the rtucker CUDA library.
//
// A "range-finder problem" (RFProb) is one application of the loop body of
// Alg. 1 (one mode k of one tensor) or of the per-node body of Alg. 2 (one
// node S of the dimension tree): sample w columns of the set unfolding X^(S)
// for a contiguous mode range S, sketch, orthonormalise, W-step.  Every stage
// kernel takes the whole table of problems and maps its CTAs onto them, so one
// launch serves all modes of all tensors (or all nodes of a tree) at once.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace rt {

constexpr int MAXD = 16;
constexpr int TS_MAXLEV = 6;   // stack levels of the TSQR tree of Z above its row blocks

// device status word codes (first error wins)
enum : int { ST_OK = 0, ST_TIMEOUT = 1, ST_DEVICE = 2, ST_NUMERIC = 3 };

__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

enum : int { DT_F32 = 0, DT_F64 = 1, DT_BF16 = 2, DT_F8 = 3 };

// Value of an E4M3 code (1 sign, 4 exponent bits with bias 7, 3 mantissa bits;
// exponent field 0: subnormals m 2^-9), from the bit fields.  The NaN code
// S.1111.111 is never stored by the quantiser (its magnitudes stay below 256) and
// decodes as 480 here.
__device__ __forceinline__ float e4m3_value(uint32_t c) {
  const uint32_t ef = (c >> 3) & 15u, m = c & 7u;
  const float v = ef ? __uint_as_float(((ef + 120u) << 23) | (m << 20)) : (float)m * 0x1p-9f;
  return (c & 0x80u) ? -v : v;
}

// Nearest E4M3 code to y, ties to the even mantissa, magnitudes beyond 448 saturated
// (the conversion instruction's round-to-nearest-even, satfinite form).
__device__ __forceinline__ uint32_t e4m3_code(float y) {
  unsigned short r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(0.f), "f"(y));
  return r & 0xFFu;
}

struct RFProb {
  // input tensor and the geometry of the set unfolding X^(S), S = {a..b}
  const void* X;
  int32_t dtype;
  int32_t ncm;             // number of complement modes
  int64_t nS;              // rows of X^(S)
  int64_t N;               // columns of X^(S) = n_{notin S}
  int64_t rowstride;       // element stride in X of the C-order row index over S
  int64_t csize[MAXD];     // complement mode sizes (natural order)
  int64_t cstride[MAXD];   // their element strides in X
  // method parameters
  int32_t r, c;            // rank and r + p
  int64_t s;               // number of sampled columns
  uint64_t seed;
  uint32_t node;           // stream id (mode k or tree node id)
  int32_t fh;              // half width of the Feistel domain (bits)
  // workspace (device pointers) and tiling counts
  int64_t* idx;            // [s]      sampled column indices pi(j)
  int64_t* off;            // [s]      element offset in X of column pi(j)
  float* Om;               // [s][c]   Gaussian test matrix rows
  float* Yt;               // [s][nS]  sampled columns (fiber j contiguous)
  float* Zp;               // [nzc][nS][c] partial sketches per sample chunk; chunk 0
                           // holds Z itself once the gather/sketch kernel is done
  int32_t* zcnt;           // [nrt] finished-chunk counters per row tile of the sketch
  int32_t nzc;             // number of sample chunks of the sketch
  int32_t nrb;             // row blocks of the TSQR of Z (1 = single block)
  int32_t rbrows;          // rows per TSQR row block
  int32_t nbi;             // row blocks of the reduction B^T = Y^T Q
  float* Q;                // [nS][c]  orthonormal factor of Z
  float* Rb;               // [nrb][c][c] TSQR first-level R factors
  float* Q2;               // [nrb*c][c] TSQR level-0 Q (member slices; combined in place)
  int32_t nlev;            // stack levels of the TSQR tree (0: one row block)
  int32_t fan;             // R factors stacked per group at every level
  int32_t lev_n[TS_MAXLEV + 1];  // factors entering level l (lev_n[0] = nrb); lev_n[nlev] = 1
  float* tsR;              // R of the groups of levels 0 .. nlev-2 (inputs of levels 1 ..)
  float* tsQ;              // Q member slices of levels 1 .. nlev-1
  float* Bp;               // [nbi][s][c] partial B^T
  float* Rc;               // [nsc][c][c] R factors of the sample chunks of B^T
  int32_t nsc;             // number of sample chunks of B^T
  int32_t scrows;          // rows (samples) per chunk of B^T
  int32_t wlev;            // levels of the R tree over the chunk factors before the W-step
  int32_t wfan;            // chunk factors stacked per group in that tree
  int32_t wn[TS_MAXLEV + 1];  // factors entering level l (wn[0] = nsc)
  float* wsR;              // R of the tree's groups (levels 1 .. wlev)
  const float* Rw;         // the stack the W-step factors: Rc, or the tree's last level
  int32_t nrw;             // number of c x c factors in it
  float* W;                // [c][c]   left singular vectors of R^T, sorted (cols)
  float* Wsg;              // [c][r]   W(:, :r) with the sign rule's column signs (U = Q Wsg)
  float* sigma;            // [c]      singular values of Q^T Y, descending
  unsigned long long* keys;// [r]      sign-rule argmax keys
  float* U;                // [nS][r]  output factor
  float* sigma_out;        // optional copy of sigma for the caller (or null)
  // Cholesky form: double-float Grams of the B-step's sample chunks
  float* Cp;               // [nbg][c][c][2] hi/lo words (upper triangles)
  int32_t nbg;             // number of sample chunks of the B-step Gram
  int32_t skbf16;          // BF16 form: the sketch Z = Y Omega from bfloat16-rounded Y and
                           // Omega (float32 accumulate); Y itself stays float32
  // float8 storage of X (dtype DT_F8): element e = code x xsc[e / xslab]
  const float* xsc;        // per-slab scales
  int64_t xslab;           // elements per slab (the last two modes)
  int32_t zshift;          // S5 by shifted CholeskyQR3 (rt_options.qr = 3)
};

// Problem lookup: blocks (or threads) are numbered consecutively over the
// problems; prefix[p] = first unit of problem p, prefix[nprob] = total.
__device__ __forceinline__ int find_prob(const int64_t* prefix, int nprob, int64_t unit) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= unit) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float load_x(const void* X, int dtype, int64_t e) {
  if (dtype == DT_F32) return __ldg(reinterpret_cast<const float*>(X) + e);
  if (dtype == DT_F64) return (float)__ldg(reinterpret_cast<const double*>(X) + e);
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[e]);
}

// Element e of a problem's tensor for the fiber gathers, float8 storage included (the
// product of an E4M3 value and a power-of-two scale is exact in float32).  float32 X
// is read with ld.global.cg (cached in L2 only): a scattered 4-byte read then costs one
// 32-byte L2 sector instead of a 128-byte L1 line fill.
__device__ __forceinline__ float load_xq(const RFProb& q, int64_t e) {
  if (q.dtype == DT_F32) return __ldcg(reinterpret_cast<const float*>(q.X) + e);
  if (q.dtype == DT_F8)
    return e4m3_value(__ldg(reinterpret_cast<const unsigned char*>(q.X) + e)) * __ldg(q.xsc + e / q.xslab);
  return load_x(q.X, q.dtype, e);
}

// Compensated float32 sums (GB300's float64 rate is ~1/64 of float32).
// hi + lo += a b with the product's and the sum's rounding errors kept (TwoProd by
// fma, TwoSum).  Explicit _rn intrinsics: the compiler must not contract or reorder.
__device__ __forceinline__ void df_acc(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
// Kahan (compensated) sum s, k: s + k tracks the sum of the added values to about one
// rounding of each value (the values themselves rounded products here: a Gram entry's
// error stays within u sqrt(G_ii G_jj), the scale the Cholesky and Jacobi steps need).
__device__ __forceinline__ void kahan_add(float& s, float& k, float v) {
  const float y = __fsub_rn(v, k);
  const float t = __fadd_rn(s, y);
  k = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float bhi, float blo) {
  const float s = __fadd_rn(hi, bhi);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bhi, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, blo));
}

// Single-instruction approximations (flush-to-zero) used where a few ulp do not matter:
// the rotation parameters of the Jacobi SVD, whose orthogonality comes from cs^2 + sn^2
// = 1, not from the exact angle.
// Pairs of float32 in one 64-bit register pair for the packed FMA of sm_100-class
// GPUs: fma.rn.f32x2 rounds each lane exactly as a scalar fmaf does, so a kernel that
// packs two independent accumulators gives bit-identical results with half the FMA
// instructions.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; `red` is shared scratch of >= 32 floats.  All threads get the sum.
__device__ __forceinline__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = (threadIdx.x < (unsigned)nw) ? red[threadIdx.x] : 0.f;
  if (wid == 0) {
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  float out = red[0];
  __syncthreads();
  return out;
}

}  // namespace rt
