// core_kernels.cu - core projection S = X x_1 U_1^T ... x_d U_d^T (Alg. 1, core
// step) as a chain of single-mode contractions (TTM, Sec. 2.2).
//
// One contraction with U (n x r) of a tensor viewed as A(L, n, R) (L the
// product of the leading modes, R of the trailing, already contracted, ones):
//     out(l, a, rho) = sum_i U[i][a] A(l, i, rho),
// i.e. the GEMM  out(a, col) = U^T(a, i) B(i, col)  with col = l R + rho.
// Modes are contracted last-to-first, so the pass over X is the R = 1 case
// (rows of X contiguous) and later passes work on the shrinking intermediate.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"

namespace rt {

constexpr int TT_BM = 32, TT_BN = 128, TT_BK = 16;

template <typename T>
__device__ __forceinline__ float ldf(const T* p, int64_t e);
template <> __device__ __forceinline__ float ldf<float>(const float* p, int64_t e) { return __ldg(p + e); }
template <> __device__ __forceinline__ float ldf<double>(const double* p, int64_t e) { return (float)__ldg(p + e); }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p, int64_t e) {
  return __bfloat162float(p[e]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_ttm_t(const T* __restrict__ A, int64_t L, int64_t n, int64_t R,
                                               const float* __restrict__ U, int r,
                                               float* __restrict__ out) {
  __shared__ __align__(16) float Us[TT_BK][TT_BM];
  __shared__ __align__(16) float Bs[TT_BK][TT_BN];
  const int tid = threadIdx.x;
  const int64_t ncol = L * R;
  const int64_t n0 = (int64_t)blockIdx.x * TT_BN;
  const int a0 = blockIdx.y * TT_BM;
  const int tm = tid >> 5, tn = tid & 31;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int64_t k0 = 0; k0 < n; k0 += TT_BK) {
    // U tile: Us[kk][mm] = U[(k0+kk) r + a0 + mm]
    for (int e = tid; e < TT_BK * TT_BM; e += 256) {
      const int kk = e / TT_BM, mm = e % TT_BM;
      const int64_t i = k0 + kk;
      const int a = a0 + mm;
      Us[kk][mm] = (i < n && a < r) ? __ldg(U + i * r + a) : 0.f;
    }
    if (R == 1) {  // B(i, col) = A[col n + i]: i contiguous
      for (int e = tid; e < TT_BK * TT_BN; e += 256) {
        const int nn = e / TT_BK, kk = e % TT_BK;
        const int64_t col = n0 + nn, i = k0 + kk;
        Bs[kk][nn] = (col < ncol && i < n) ? ldf<T>(A, col * n + i) : 0.f;
      }
    } else {       // B(i, col) = A[(l n + i) R + rho]: rho contiguous
      for (int e = tid; e < TT_BK * TT_BN; e += 256) {
        const int kk = e / TT_BN, nn = e % TT_BN;
        const int64_t col = n0 + nn, i = k0 + kk;
        float v = 0.f;
        if (col < ncol && i < n) {
          const int64_t l = col / R, rho = col - l * R;
          v = ldf<T>(A, (l * n + i) * R + rho);
        }
        Bs[kk][nn] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TT_BK; ++kk) {
      const float4 u = *reinterpret_cast<const float4*>(&Us[kk][tm * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tn * 4]);
      const float ua[4] = {u.x, u.y, u.z, u.w};
      const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(ua[x], bb[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int64_t col = n0 + tn * 4 + y;
    if (col >= ncol) continue;
    const int64_t l = col / R, rho = col - l * R;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int a = a0 + tm * 4 + x;
      if (a < r) out[(l * r + a) * R + rho] = acc[x][y];
    }
  }
}

int launch_ttm_t(const void* A, int dtype, int64_t L, int64_t n, int64_t R, const float* U, int r,
                 float* out, cudaStream_t st) {
  const int64_t ncol = L * R;
  dim3 grid((unsigned)((ncol + TT_BN - 1) / TT_BN), (unsigned)((r + TT_BM - 1) / TT_BM));
  if (dtype == DT_F32)
    k_ttm_t<float><<<grid, 256, 0, st>>>(static_cast<const float*>(A), L, n, R, U, r, out);
  else if (dtype == DT_F64)
    k_ttm_t<double><<<grid, 256, 0, st>>>(static_cast<const double*>(A), L, n, R, U, r, out);
  else
    k_ttm_t<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(A), L, n, R, U, r, out);
  return 1;
}

cudaError_t core_init_attributes() { return cudaSuccess; }

}  // namespace rt
