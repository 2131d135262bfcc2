// ht_kernels.cu - transfer tensors of the subsampled randomized RtL-HT (Alg. 2).
//
//  * internal node S (Sec. 4, transfer-tensor inner products):
//        B_S(i, j, k) = <U_S(:, i), U_{S_l}(:, j) (x) U_{S_r}(:, k)>
//                     = (U_l^T M_i U_r)(j, k),  M_i(a, b) = U_S(a n_r + b, i)
//    (C-order rows of the set unfolding: the left child's index is slower).
//  * root (Sec. 4, root inner products; the pass over all of X):
//        B_R(1, j, k) = <vec X, U_{R_l}(:, j) (x) U_{R_r}(:, k)> = (U_l^T X_mat U_r)(j, k)
//    with X_mat the n_{R_l} x n_{R_r} view of X.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "rt_common.cuh"
#include "rt_host.h"

namespace rt {

// ------------------------------------------------------------------ internal nodes
// k_transfer_part: CTA c of job q (q.cta0 <= c < q.cta0 + ceil(n_l / TR_A)) takes the
// left-child rows a in [a0, a0 + TR_A):
//     T(a, i, k) = sum_b U_S(a n_r + b, i) U_r(b, k)      (rows of U_S read contiguously)
//     part_c(i, j, k) = sum_a U_l(a, j) T(a, i, k)
// k_transfer_sum: B_S = sum over the job's CTAs of part_c, fixed order, float64.
constexpr int TR_A = 4, TR_B = 64, TR_MAX = 12, TR_TH = 256;
static_assert(TR_MAX == TRANSFER_RMAX, "grouped transfer kernel width");

__global__ void __launch_bounds__(TR_TH) k_transfer_part(const TransferJob* __restrict__ jobs, int njobs,
                                                         float* __restrict__ part) {
  __shared__ float us[TR_A * TR_B * TR_MAX];
  __shared__ float ur[TR_B * TR_MAX];
  __shared__ float tt[TR_A * TR_MAX * TR_MAX];
  int q = 0;
  while (q + 1 < njobs && (int64_t)blockIdx.x >= jobs[q + 1].cta0) ++q;
  const TransferJob jb = jobs[q];
  const int64_t a0 = ((int64_t)blockIdx.x - jb.cta0) * TR_A;
  const int na = (int)min((int64_t)TR_A, jb.nl - a0);
  const int rS = jb.rS, rl = jb.rl, rr = jb.rr;
  const int nT = TR_A * rS * rr;                 // outputs T(a, i, k), a < TR_A
  float acc[(TR_A * TR_MAX * TR_MAX + TR_TH - 1) / TR_TH];
#pragma unroll
  for (int u = 0; u < (int)(sizeof(acc) / sizeof(float)); ++u) acc[u] = 0.f;
  for (int64_t b0 = 0; b0 < jb.nr; b0 += TR_B) {
    const int nb = (int)min((int64_t)TR_B, jb.nr - b0);
    __syncthreads();
    for (int e = threadIdx.x; e < TR_A * nb * rS; e += TR_TH) {
      const int a = e / (nb * rS), rem = e % (nb * rS);
      us[e] = (a < na) ? __ldg(jb.US + ((a0 + a) * jb.nr + b0) * rS + rem) : 0.f;
    }
    for (int e = threadIdx.x; e < nb * rr; e += TR_TH) ur[e] = __ldg(jb.Ur + b0 * rr + e);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < (int)(sizeof(acc) / sizeof(float)); ++u) {
      const int o = threadIdx.x + u * TR_TH;
      if (o < nT) {
        const int a = o / (rS * rr), i = (o / rr) % rS, k = o % rr;
        const float* up = us + a * nb * rS + i;
        float v = acc[u];
        for (int b = 0; b < nb; ++b) v = fmaf(up[b * rS], ur[b * rr + k], v);
        acc[u] = v;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < (int)(sizeof(acc) / sizeof(float)); ++u) {
    const int o = threadIdx.x + u * TR_TH;
    if (o < nT) tt[o] = acc[u];
  }
  __syncthreads();
  float* pc = part + (size_t)blockIdx.x * TR_MAX * TR_MAX * TR_MAX;
  for (int o = threadIdx.x; o < rS * rl * rr; o += TR_TH) {
    const int i = o / (rl * rr), j = (o / rr) % rl, k = o % rr;
    float v = 0.f;
    for (int a = 0; a < na; ++a) v = fmaf(__ldg(jb.Ul + (a0 + a) * rl + j), tt[(a * rS + i) * rr + k], v);
    pc[o] = v;
  }
}

__global__ void __launch_bounds__(TR_TH) k_transfer_sum(const TransferJob* __restrict__ jobs,
                                                        const float* __restrict__ part) {
  const TransferJob jb = jobs[blockIdx.y];
  const int o = blockIdx.x * TR_TH + threadIdx.x;
  if (o >= jb.rS * jb.rl * jb.rr) return;
  const int64_t nc = (jb.nl + TR_A - 1) / TR_A;
  double v = 0.0;
  for (int64_t c = 0; c < nc; ++c) v += (double)part[(size_t)(jb.cta0 + c) * TR_MAX * TR_MAX * TR_MAX + o];
  jb.B[o] = (float)v;
}

// General form of one transfer tensor, for ranks above TR_MAX (up to 64): two mode
// contractions, T1(a, k, i) = sum_b U_r(b, k) U_S(a n_r + b, i) and
// T2(j, k, i) = sum_a U_l(a, j) T1(a, k, i), then B_S(i, j, k) = T2(j, k, i).
__global__ void k_perm_jki(const float* __restrict__ T2, int rS, int rl, int rr, float* __restrict__ B) {
  const int tot = rS * rl * rr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int i = e / (rl * rr), j = (e / rr) % rl, k = e % rr;
    B[e] = T2[((size_t)j * rr + k) * rS + i];
  }
}

size_t transfer_general_floats(int64_t nl, int rS, int rl, int rr) {
  return (size_t)nl * rr * rS + (size_t)rl * rr * rS + 4;
}

int launch_transfer_general(const TransferJob& jb, float* scratch, cudaStream_t st) {
  float* T1 = scratch;
  float* T2 = scratch + (((size_t)jb.nl * jb.rr * jb.rS + 3) & ~(size_t)3);
  int n = launch_ttm_t(jb.US, DT_F32, jb.nl, jb.nr, jb.rS, jb.Ur, jb.rr, T1, st);
  n += launch_ttm_t(T1, DT_F32, 1, jb.nl, (int64_t)jb.rr * jb.rS, jb.Ul, jb.rl, T2, st);
  const int tot = jb.rS * jb.rl * jb.rr;
  k_perm_jki<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(T2, jb.rS, jb.rl, jb.rr, jb.B);
  return n + 1;
}

int64_t transfer_ctas(int64_t nl) { return (nl + TR_A - 1) / TR_A; }
size_t transfer_part_floats(int64_t total_ctas) { return (size_t)total_ctas * TR_MAX * TR_MAX * TR_MAX; }

int launch_transfer(const TransferJob* jobs_dev, const TransferJob* jobs_host, int njobs, float* part,
                    cudaStream_t st) {
  if (njobs < 1) return 0;
  const int64_t total = jobs_host[njobs - 1].cta0 + transfer_ctas(jobs_host[njobs - 1].nl);
  int omax = 1;
  for (int q = 0; q < njobs; ++q) omax = std::max(omax, jobs_host[q].rS * jobs_host[q].rl * jobs_host[q].rr);
  k_transfer_part<<<(unsigned)total, TR_TH, 0, st>>>(jobs_dev, njobs, part);
  k_transfer_sum<<<dim3((unsigned)((omax + TR_TH - 1) / TR_TH), (unsigned)njobs), TR_TH, 0, st>>>(jobs_dev, part);
  return 2;
}

// ------------------------------------------------------------------ root pass
// CTA: rows [a0, a0 + RT_RA) x columns [b0, b0 + RT_CB).  Thread t owns rows
// a0 + t + RT_TH*q (q < 4).  X tiles of RT_CBT columns are staged in shared
// memory (row stride RT_CBT + 1), U_r rows in shared memory (padded to 12).
// Row sums t(a, k) accumulate per stage, then Kahan-add into the totals.
// Output: partial P[blk](j, k) = sum_{a in block} U_l(a, j) t(a, k), blk =
// by * gridDim.x + bx.  There are gy = ceil(nl / RT_RA) row blocks; a grid of
// fewer than gy rows of CTAs (grid.y is limited to 65535) walks them with
// stride gridDim.y.
constexpr int RT_TH = 128, RT_RPT = 4, RT_RA = RT_TH * RT_RPT, RT_CBT = 32, RT_CB = 8192, RT_KMAX = 12;
constexpr int RT_SMEM = RT_RA * (RT_CBT + 1) * 4;

template <typename T>
__device__ __forceinline__ float ldx(const T* p, int64_t e);
template <> __device__ __forceinline__ float ldx<float>(const float* p, int64_t e) { return __ldg(p + e); }
template <> __device__ __forceinline__ float ldx<double>(const double* p, int64_t e) { return (float)__ldg(p + e); }
template <> __device__ __forceinline__ float ldx<__nv_bfloat16>(const __nv_bfloat16* p, int64_t e) {
  return __bfloat162float(p[e]);
}

template <typename T, int RR>
__global__ void __launch_bounds__(RT_TH) k_root(const T* __restrict__ X, int64_t nl, int64_t nr,
                                                const float* __restrict__ Ul, int rl,
                                                const float* __restrict__ Ur, float* __restrict__ part) {
  extern __shared__ __align__(16) float Xs[];  // RT_RA * (RT_CBT + 1)
  __shared__ __align__(16) float Us[RT_CBT * RT_KMAX];
  __shared__ float red[RT_TH];
  const int tid = threadIdx.x;
  const int64_t gy = (nl + RT_RA - 1) / RT_RA;
  for (int64_t by = blockIdx.y; by < gy; by += gridDim.y) {
  const int64_t a0 = by * RT_RA;
  const int64_t b0 = (int64_t)blockIdx.x * RT_CB;
  const int64_t b1 = min(nr, b0 + RT_CB);
  float tot[RT_RPT][RR], cmp[RT_RPT][RR];
#pragma unroll
  for (int q = 0; q < RT_RPT; ++q)
#pragma unroll
    for (int k = 0; k < RR; ++k) tot[q][k] = cmp[q][k] = 0.f;
  for (int64_t bs = b0; bs < b1; bs += RT_CBT) {
    const int nb = (int)min((int64_t)RT_CBT, b1 - bs);
    __syncthreads();
    // X tile: RT_RA rows x RT_CBT columns; a warp reads whole 128-byte rows
    for (int e = tid; e < RT_RA * RT_CBT; e += RT_TH) {
      const int ra = e / RT_CBT, cb = e % RT_CBT;
      const int64_t a = a0 + ra, b = bs + cb;
      Xs[ra * (RT_CBT + 1) + cb] = (a < nl && cb < nb) ? ldx<T>(X, a * nr + b) : 0.f;
    }
    for (int e = tid; e < RT_CBT * RT_KMAX; e += RT_TH) {
      const int cb = e / RT_KMAX, k = e % RT_KMAX;
      Us[e] = (cb < nb && k < RR) ? __ldg(Ur + (bs + cb) * RR + k) : 0.f;
    }
    __syncthreads();
    float st[RT_RPT][RR];
#pragma unroll
    for (int q = 0; q < RT_RPT; ++q)
#pragma unroll
      for (int k = 0; k < RR; ++k) st[q][k] = 0.f;
#pragma unroll 4
    for (int cb = 0; cb < RT_CBT; ++cb) {
      float u[RT_KMAX];
      const float4* u4 = reinterpret_cast<const float4*>(Us + cb * RT_KMAX);
#pragma unroll
      for (int v = 0; v < RT_KMAX / 4; ++v) {
        const float4 w = u4[v];
        u[4 * v] = w.x; u[4 * v + 1] = w.y; u[4 * v + 2] = w.z; u[4 * v + 3] = w.w;
      }
#pragma unroll
      for (int q = 0; q < RT_RPT; ++q) {
        const float x = Xs[(tid + RT_TH * q) * (RT_CBT + 1) + cb];
#pragma unroll
        for (int k = 0; k < RR; ++k) st[q][k] = fmaf(x, u[k], st[q][k]);
      }
    }
#pragma unroll
    for (int q = 0; q < RT_RPT; ++q)
#pragma unroll
      for (int k = 0; k < RR; ++k) {  // Kahan: tot += st
        const float y = st[q][k] - cmp[q][k];
        const float s = tot[q][k] + y;
        cmp[q][k] = (s - tot[q][k]) - y;
        tot[q][k] = s;
      }
  }
  // partial(j, k) = sum over the block's rows of U_l(a, j) t(a, k)
  for (int j = 0; j < rl; ++j) {
    float ul[RT_RPT];
#pragma unroll
    for (int q = 0; q < RT_RPT; ++q) {
      const int64_t a = a0 + tid + RT_TH * q;
      ul[q] = (a < nl) ? __ldg(Ul + a * rl + j) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < RT_RPT; ++q) v = fmaf(ul[q], tot[q][k], v);
      v = block_sum(v, red);
      if (tid == 0) part[((size_t)by * gridDim.x + blockIdx.x) * rl * RR + j * RR + k] = v;
    }
  }
  }
}

// Sum of the per-CTA partials in float64 (fixed order: deterministic).
__global__ void k_root_reduce(const float* __restrict__ part, int64_t nblk, int rl, int rr, float* BR) {
  const int e = blockIdx.x;  // one CTA per entry (j, k)
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) acc += (double)part[b * rl * rr + e];
  __shared__ double red[32];
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    BR[e] = (float)s;
  }
}

size_t root_scratch_floats(int64_t nl, int64_t nr, int rl, int rr) {
  const int64_t gx = (nr + RT_CB - 1) / RT_CB, gy = (nl + RT_RA - 1) / RT_RA;
  return (size_t)(gx * gy) * rl * rr;
}

// Launches return their error directly (cudaLaunchKernel), so that a caller can tell
// a failure of these launches from an earlier error pending in the runtime.
template <typename T>
static cudaError_t root_dispatch(const T* X, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur,
                                 int rr, float* part, dim3 grid, cudaStream_t st) {
  void* args[] = {&X, &nl, &nr, &Ul, &rl, &Ur, &part};
  const void* fn = nullptr;
  switch (rr) {
#define RT_CASE(K)                                    \
  case K:                                             \
    fn = reinterpret_cast<const void*>(k_root<T, K>); \
    break;
    RT_CASE(1) RT_CASE(2) RT_CASE(3) RT_CASE(4) RT_CASE(5) RT_CASE(6)
    RT_CASE(7) RT_CASE(8) RT_CASE(9) RT_CASE(10) RT_CASE(11) RT_CASE(12)
#undef RT_CASE
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, RT_SMEM);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel(fn, grid, dim3(RT_TH), args, RT_SMEM, st);
}

void launch_root_reduce(const float* part, int64_t nblk, int rl, int rr, float* BR, cudaStream_t st) {
  k_root_reduce<<<(unsigned)(rl * rr), 256, 0, st>>>(part, nblk, rl, rr, BR);
}

constexpr int64_t RT_GRID_Y_MAX = 65535;

int launch_root_tiled(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl,
                      const float* Ur, int rr, float* BR, float* scratch, cudaStream_t st, cudaError_t* err) {
  const int64_t gx = (nr + RT_CB - 1) / RT_CB, gy = (nl + RT_RA - 1) / RT_RA;
  dim3 grid((unsigned)gx, (unsigned)std::min(gy, RT_GRID_Y_MAX));
  cudaError_t e;
  if (dtype == DT_F32) e = root_dispatch(static_cast<const float*>(X), nl, nr, Ul, rl, Ur, rr, scratch, grid, st);
  else if (dtype == DT_F64) e = root_dispatch(static_cast<const double*>(X), nl, nr, Ul, rl, Ur, rr, scratch, grid, st);
  else e = root_dispatch(static_cast<const __nv_bfloat16*>(X), nl, nr, Ul, rl, Ur, rr, scratch, grid, st);
  if (e == cudaSuccess) {
    int64_t nblk = gx * gy;
    int irl = rl, irr = rr;
    void* args[] = {&scratch, &nblk, &irl, &irr, &BR};
    e = cudaLaunchKernel(reinterpret_cast<const void*>(k_root_reduce), dim3((unsigned)(rl * rr)), dim3(256), args,
                         0, st);
  }
  if (err) *err = e;
  return 2;
}

size_t root_pass_scratch_floats(int64_t nl, int64_t nr, int rl, int rr) {
  return std::max(root_scratch_floats(nl, nr, rl, rr), root_stream_scratch_floats(nl, nr, rl, rr));
}

// dst[row][d0 + c] = src[row][c0 + c], c < nc (column blocks of row-major matrices).
__global__ void k_copy_cols(const float* __restrict__ src, int64_t rows, int lds, int c0, int nc,
                            float* __restrict__ dst, int ldd, int d0) {
  const int64_t tot = rows * nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / nc;
    const int c = (int)(e % nc);
    dst[r * ldd + d0 + c] = src[r * lds + c0 + c];
  }
}

static unsigned copy_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

static size_t pad4(size_t n) { return (n + 3) & ~(size_t)3; }

size_t root_any_scratch_floats(int64_t nl, int64_t nr, int rl, int rr) {
  if (rr <= RT_KMAX) return root_pass_scratch_floats(nl, nr, rl, rr);
  return pad4((size_t)nr * RT_KMAX) + pad4((size_t)rl * RT_KMAX) + root_pass_scratch_floats(nl, nr, rl, RT_KMAX);
}

int launch_root_any(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur,
                    int rr, float* BR, float* scratch, int* status, cudaStream_t st) {
  if (rr <= RT_KMAX) return launch_root(X, dtype, nl, nr, Ul, rl, Ur, rr, BR, scratch, status, st);
  // r_r above the root kernels' register width: one pass over X per chunk of at most
  // RT_KMAX columns of U_r (chunks of near-equal width), each on the root pass above.
  float* Urc = scratch;
  float* BRc = Urc + pad4((size_t)nr * RT_KMAX);
  float* rs = BRc + pad4((size_t)rl * RT_KMAX);
  const int nch = (rr + RT_KMAX - 1) / RT_KMAX;
  int n = 0;
  for (int ch = 0, k0 = 0; ch < nch; ++ch) {
    const int kc = (rr - k0) / (nch - ch);
    k_copy_cols<<<copy_grid(nr * kc), 256, 0, st>>>(Ur, nr, rr, k0, kc, Urc, kc, 0);
    n += 1 + launch_root(X, dtype, nl, nr, Ul, rl, Urc, kc, BRc, rs, status, st);
    k_copy_cols<<<copy_grid((int64_t)rl * kc), 256, 0, st>>>(BRc, rl, kc, 0, kc, BR, rr, k0);
    ++n;
    k0 += kc;
  }
  return n;
}

int launch_root(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur, int rr,
                float* BR, float* scratch, int* status, cudaStream_t st) {
  if (dtype == DT_F32) {
    const int n = launch_root_stream(static_cast<const float*>(X), nl, nr, Ul, rl, Ur, rr, BR, scratch, status, st);
    if (n > 0) return n;
  }
  return launch_root_tiled(X, dtype, nl, nr, Ul, rl, Ur, rr, BR, scratch, st);
}

}  // namespace rt
