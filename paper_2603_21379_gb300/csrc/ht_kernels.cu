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
// grid: (job, i).  Dynamic smem: T[nl][rr] (float)
__global__ void __launch_bounds__(256) k_transfer(const TransferJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* T = reinterpret_cast<float*>(smem_raw);
  const TransferJob jb = jobs[blockIdx.y];
  const int i = blockIdx.x;
  if (i >= jb.rS) return;
  // T(a, k) = sum_b M_i(a, b) U_r(b, k)
  for (int64_t e = threadIdx.x; e < jb.nl * jb.rr; e += blockDim.x) {
    const int64_t a = e / jb.rr;
    const int k = (int)(e % jb.rr);
    float acc = 0.f;
    for (int64_t b = 0; b < jb.nr; ++b)
      acc = fmaf(__ldg(jb.US + (a * jb.nr + b) * jb.rS + i), __ldg(jb.Ur + b * jb.rr + k), acc);
    T[e] = acc;
  }
  __syncthreads();
  // B(i, j, k) = sum_a U_l(a, j) T(a, k)
  for (int e = threadIdx.x; e < jb.rl * jb.rr; e += blockDim.x) {
    const int j = e / jb.rr, k = e % jb.rr;
    float acc = 0.f;
    for (int64_t a = 0; a < jb.nl; ++a) acc = fmaf(__ldg(jb.Ul + a * jb.rl + j), T[a * jb.rr + k], acc);
    jb.B[((int64_t)i * jb.rl + j) * jb.rr + k] = acc;
  }
}

int launch_transfer(const TransferJob* jobs_dev, const TransferJob* jobs_host, int njobs, cudaStream_t st) {
  if (njobs <= 0) return 0;
  int rmax = 1;
  size_t smax = 0;
  for (int q = 0; q < njobs; ++q) {
    rmax = rmax > jobs_host[q].rS ? rmax : jobs_host[q].rS;
    const size_t sz = (size_t)jobs_host[q].nl * jobs_host[q].rr * sizeof(float);
    smax = smax > sz ? smax : sz;
  }
  cudaFuncSetAttribute(k_transfer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
  k_transfer<<<dim3((unsigned)rmax, (unsigned)njobs), 256, smax, st>>>(jobs_dev);
  return 1;
}

// ------------------------------------------------------------------ root pass
// CTA: rows [a0, a0 + RT_RA) x columns [b0, b0 + RT_CB).  Thread t owns rows
// a0 + t + RT_TH*q (q < 4).  X tiles of RT_CBT columns are staged in shared
// memory (row stride RT_CBT + 1), U_r rows in shared memory (padded to 12).
// Row sums t(a, k) accumulate per stage, then Kahan-add into the totals.
// Output: partial P[blk](j, k) = sum_{a in block} U_l(a, j) t(a, k).
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
  const int64_t a0 = (int64_t)blockIdx.y * RT_RA;
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
      if (tid == 0) part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * rl * RR + j * RR + k] = v;
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

template <typename T>
static void root_dispatch(const T* X, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur,
                          int rr, float* part, dim3 grid, cudaStream_t st) {
  switch (rr) {
#define RT_CASE(K)                                                                          \
  case K:                                                                                   \
    cudaFuncSetAttribute(k_root<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, RT_SMEM); \
    k_root<T, K><<<grid, RT_TH, RT_SMEM, st>>>(X, nl, nr, Ul, rl, Ur, part);                 \
    break;
    RT_CASE(1) RT_CASE(2) RT_CASE(3) RT_CASE(4) RT_CASE(5) RT_CASE(6)
    RT_CASE(7) RT_CASE(8) RT_CASE(9) RT_CASE(10) RT_CASE(11) RT_CASE(12)
#undef RT_CASE
    default: break;
  }
}

void launch_root_reduce(const float* part, int64_t nblk, int rl, int rr, float* BR, cudaStream_t st) {
  k_root_reduce<<<(unsigned)(rl * rr), 256, 0, st>>>(part, nblk, rl, rr, BR);
}

int launch_root_tiled(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl,
                      const float* Ur, int rr, float* BR, float* scratch, cudaStream_t st) {
  const int64_t gx = (nr + RT_CB - 1) / RT_CB, gy = (nl + RT_RA - 1) / RT_RA;
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (dtype == DT_F32) root_dispatch(static_cast<const float*>(X), nl, nr, Ul, rl, Ur, rr, scratch, grid, st);
  else if (dtype == DT_F64) root_dispatch(static_cast<const double*>(X), nl, nr, Ul, rl, Ur, rr, scratch, grid, st);
  else root_dispatch(static_cast<const __nv_bfloat16*>(X), nl, nr, Ul, rl, Ur, rr, scratch, grid, st);
  launch_root_reduce(scratch, gx * gy, rl, rr, BR, st);
  return 2;
}

size_t root_pass_scratch_floats(int64_t nl, int64_t nr, int rl, int rr) {
  return std::max(root_scratch_floats(nl, nr, rl, rr), root_stream_scratch_floats(nl, rl, rr));
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
