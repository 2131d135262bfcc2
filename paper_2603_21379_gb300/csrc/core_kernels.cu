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

// One 32 (a) x 128 (col) output tile of out(l, a, rho) = sum_i U[i][a] A(l, i, rho),
// col = l R + rho, starting at column n0 and row a0 of U^T.
template <typename T>
__device__ __forceinline__ void ttm_tile(const T* __restrict__ A, int64_t L, int64_t n, int64_t R,
                                         const float* __restrict__ U, int r, float* __restrict__ out, int64_t n0,
                                         int a0) {
  __shared__ __align__(16) float Us[TT_BK][TT_BM];
  __shared__ __align__(16) float Bs[TT_BK][TT_BN];
  const int tid = threadIdx.x;
  const int64_t ncol = L * R;
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

template <typename T>
__global__ void __launch_bounds__(256) k_ttm_t(const T* __restrict__ A, int64_t L, int64_t n, int64_t R,
                                               const float* __restrict__ U, int r,
                                               float* __restrict__ out) {
  ttm_tile<T>(A, L, n, R, U, r, out, (int64_t)blockIdx.x * TT_BN, blockIdx.y * TT_BM);
}

// Many contractions (one per tensor of a batch) in one launch: CTA b works on job
// j with pre[j] <= b < pre[j + 1], tile (b - pre[j]) of its tiles_x x tiles_y grid.
template <typename T>
__global__ void __launch_bounds__(256) k_ttm_grouped(const TTMJob* __restrict__ jobs, const int64_t* __restrict__ pre,
                                                     int njobs) {
  const int j = find_prob(pre, njobs, blockIdx.x);
  const TTMJob& q = jobs[j];
  const int64_t local = (int64_t)blockIdx.x - pre[j];
  const int64_t tx = local % q.tiles_x, ty = local / q.tiles_x;
  ttm_tile<T>(static_cast<const T*>(q.A), q.L, q.n, q.R, q.U, q.r, q.out, tx * TT_BN, (int)ty * TT_BM);
}

// ---------------------------------------------------------------- FP32, rho-contiguous form
// out(l, a, rho) = sum_i U[i][a] A(l, i, rho) for float A with R % 4 == 0.  One CTA owns
// all 32 a (of a 32-row block of U^T) and TN consecutive rho of one l; each thread keeps an
// 8 x 8 block of outputs in registers: 8 a times two runs of 4 rho, TN/2 apart, so that
// the 16-byte shared loads of consecutive lanes are consecutive (no bank conflicts).  A and U tiles of TK rows of i are staged in
// shared memory by 16-byte / 4-byte cp.async in a TS-deep ring, so the loads of tile
// t + TS - 1 overlap the FMAs of tile t.
constexpr int TF_TS = 3;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// AW: width of the block's slice of a (32, or 16 for r <= 16, which halves the
// products); TK: rows of A and U per pipeline stage (16 with the narrow slice, which
// halves the shared memory; for AW = 32, TK = 16 measured slower than 32).
template <int TN, int AW, int TK>
constexpr size_t ttm_f32_smem() { return (size_t)TF_TS * TK * (TN + AW) * sizeof(float); }

template <int TN, int AW, int TK>
__global__ void __launch_bounds__(AW * TN / 64) k_ttm_f32(const float* __restrict__ A, int64_t n, int64_t R,
                                                    int64_t tiles_per_l, const float* __restrict__ U, int r,
                                                    float* __restrict__ out) {
  constexpr int NT = AW * TN / 64;         // threads: AW/8 a-groups x TN/8 rho-groups
  extern __shared__ __align__(16) float tsm[];
  float* As = tsm;                          // [TS][TK][TN]
  float* Us = tsm + TF_TS * TK * TN;        // [TS][TK][AW]
  const int tid = threadIdx.x;
  const int64_t l = blockIdx.x / tiles_per_l;
  const int64_t rho0 = (blockIdx.x - l * tiles_per_l) * TN;
  const int a0 = blockIdx.y * AW;
  const int ta = tid / (TN / 8), tr = tid % (TN / 8);
  const float* Al = A + l * n * R;
  const int nk = (int)((n + TK - 1) / TK);

  auto issue = [&](int kt) {
    const int stg = kt % TF_TS;
    float* as = As + stg * TK * TN;
    float* us = Us + stg * TK * AW;
    const int64_t i0 = (int64_t)kt * TK;
#pragma unroll
    for (int e = tid; e < TK * TN / 4; e += NT) {
      const int kk = e / (TN / 4), c4 = (e % (TN / 4)) * 4;
      const int64_t i = i0 + kk, rho = rho0 + c4;
      const bool ok = i < n && rho < R;
      cp_async16(as + kk * TN + c4, ok ? (const void*)(Al + i * R + rho) : (const void*)A, ok ? 16 : 0);
    }
#pragma unroll
    for (int e = tid; e < TK * AW; e += NT) {
      const int kk = e / AW, aa = e % AW;
      const int64_t i = i0 + kk;
      const bool ok = i < n && a0 + aa < r;
      cp_async4(us + kk * AW + aa, ok ? (const void*)(U + i * r + a0 + aa) : (const void*)U, ok ? 4 : 0);
    }
  };

  float acc[8][8];
#pragma unroll
  for (int x = 0; x < 8; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;

#pragma unroll
  for (int s = 0; s < TF_TS - 1; ++s) {
    if (s < nk) issue(s);
    cp_async_commit();
  }
  for (int kt = 0; kt < nk; ++kt) {
    cp_async_wait<TF_TS - 2>();
    __syncthreads();
    if (kt + TF_TS - 1 < nk) issue(kt + TF_TS - 1);
    cp_async_commit();
    const float* as = As + (kt % TF_TS) * TK * TN + tr * 4;
    const float* us = Us + (kt % TF_TS) * TK * AW + ta * 8;
#pragma unroll 8
    for (int kk = 0; kk < TK; ++kk) {
      const float4 u0 = *reinterpret_cast<const float4*>(us + kk * AW);
      const float4 u1 = *reinterpret_cast<const float4*>(us + kk * AW + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(as + kk * TN);
      const float4 b1 = *reinterpret_cast<const float4*>(as + kk * TN + TN / 2);
      const float ua[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(ua[x], bb[y], acc[x][y]);
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t rho = rho0 + h * (TN / 2) + tr * 4;
    if (rho >= R) continue;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int a = a0 + ta * 8 + x;
      if (a >= r) continue;
      float* o = out + (l * r + a) * R + rho;
      if (rho + 4 <= R) {
        *reinterpret_cast<float4*>(o) = make_float4(acc[x][4 * h], acc[x][4 * h + 1], acc[x][4 * h + 2], acc[x][4 * h + 3]);
      } else {
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if (rho + y < R) o[y] = acc[x][4 * h + y];
      }
    }
  }
}

// Last-mode contraction out(l, a) = sum_i U[i][a] A(l, i) (R = 1): one thread per row
// l reads its n contiguous floats (16-byte loads when n % 4 == 0), U sits in shared
// memory and is read as 16-byte broadcasts along a; RW >= r partial sums per thread.
constexpr int TL_THREADS = 128;
template <int RW>
__global__ void __launch_bounds__(TL_THREADS) k_ttm_last(const float* __restrict__ A, int64_t L, int n,
                                                         const float* __restrict__ U, int r,
                                                         float* __restrict__ out) {
  extern __shared__ __align__(16) float us[];   // [n][RW], zero beyond r
  for (int e = threadIdx.x; e < n * RW; e += TL_THREADS) {
    const int i = e / RW, a = e % RW;
    us[e] = a < r ? U[i * r + a] : 0.f;
  }
  __syncthreads();
  const int64_t l = (int64_t)blockIdx.x * TL_THREADS + threadIdx.x;
  if (l >= L) return;
  const float* row = A + l * n;
  float acc[RW];
#pragma unroll
  for (int a = 0; a < RW; ++a) acc[a] = 0.f;
  const bool v4 = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  for (int i0 = 0; i0 < n; i0 += 4) {
    float x[4];
    if (v4) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(row + i0));
      x[0] = f.x; x[1] = f.y; x[2] = f.z; x[3] = f.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = i0 + q < n ? __ldg(row + i0 + q) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (i0 + q >= n) break;
      const float* ui = us + (i0 + q) * RW;
#pragma unroll
      for (int a = 0; a < RW; a += 4) {
        const float4 u = *reinterpret_cast<const float4*>(ui + a);
        acc[a] = fmaf(x[q], u.x, acc[a]);
        acc[a + 1] = fmaf(x[q], u.y, acc[a + 1]);
        acc[a + 2] = fmaf(x[q], u.z, acc[a + 2]);
        acc[a + 3] = fmaf(x[q], u.w, acc[a + 3]);
      }
    }
  }
  float* o = out + l * r;
#pragma unroll
  for (int a = 0; a < RW; ++a)
    if (a < r) o[a] = acc[a];
}

// Grouped last-mode contractions (R = 1) of a batch: job q contracts the last mode of
// its L x n tensor with U_q (n x r <= RW), one thread per row.  pre[j] counts CTAs of
// TL_THREADS rows before job j.  A's element type T (the batch's X type at the first
// level); 16-byte loads for float rows with n % 4 == 0.
template <typename T, int RW>
__global__ void __launch_bounds__(TL_THREADS) k_ttm_last_grouped(const TTMJob* __restrict__ jobs,
                                                                 const int64_t* __restrict__ pre, int njobs) {
  extern __shared__ __align__(16) float us[];   // [n][RW], zero beyond r
  const int j = find_prob(pre, njobs, blockIdx.x);
  const TTMJob& q = jobs[j];
  const int n = (int)q.n, r = q.r;
  for (int e = threadIdx.x; e < n * RW; e += TL_THREADS) {
    const int i = e / RW, a = e % RW;
    us[e] = a < r ? q.U[i * r + a] : 0.f;
  }
  __syncthreads();
  const int64_t l = ((int64_t)blockIdx.x - pre[j]) * TL_THREADS + threadIdx.x;
  if (l >= q.L) return;
  const T* row = static_cast<const T*>(q.A) + l * n;
  float acc[RW];
#pragma unroll
  for (int a = 0; a < RW; ++a) acc[a] = 0.f;
  const bool v4 = sizeof(T) == 4 && (n % 4) == 0 && (reinterpret_cast<uintptr_t>(q.A) & 15) == 0;
  for (int i0 = 0; i0 < n; i0 += 4) {
    float x[4];
    if (v4) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(row + i0));
      x[0] = f.x; x[1] = f.y; x[2] = f.z; x[3] = f.w;
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) x[t] = i0 + t < n ? ldf<T>(row, i0 + t) : 0.f;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (i0 + t >= n) break;
      const float* ui = us + (i0 + t) * RW;
#pragma unroll
      for (int a = 0; a < RW; a += 4) {
        const float4 u = *reinterpret_cast<const float4*>(ui + a);
        acc[a] = fmaf(x[t], u.x, acc[a]);
        acc[a + 1] = fmaf(x[t], u.y, acc[a + 1]);
        acc[a + 2] = fmaf(x[t], u.z, acc[a + 2]);
        acc[a + 3] = fmaf(x[t], u.w, acc[a + 3]);
      }
    }
  }
  float* o = q.out + l * r;
#pragma unroll
  for (int a = 0; a < RW; ++a)
    if (a < r) o[a] = acc[a];
}

static int g_num_sms = 0;

int launch_ttm_t(const void* A, int dtype, int64_t L, int64_t n, int64_t R, const float* U, int r,
                 float* out, cudaStream_t st) {
  const int64_t ncol = L * R;
  if (dtype == DT_F32 && R == 1 && n <= 256 && r <= 32 && L <= ((int64_t)1 << 40)) {
    const unsigned blocks = (unsigned)((L + TL_THREADS - 1) / TL_THREADS);
    const float* Af = static_cast<const float*>(A);
    if (r <= 16)
      k_ttm_last<16><<<blocks, TL_THREADS, (size_t)n * 16 * 4, st>>>(Af, L, (int)n, U, r, out);
    else
      k_ttm_last<32><<<blocks, TL_THREADS, (size_t)n * 32 * 4, st>>>(Af, L, (int)n, U, r, out);
    return 1;
  }
  if (dtype == DT_F32 && R >= 64 && R % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    // rho-contiguous FP32 form; the narrower tile when the wide one leaves SMs idle or
    // R is shorter than it (the tail of a tile is masked)
    const int64_t t256 = (R + 255) / 256, t128 = (R + 127) / 128;
    const float* Af = static_cast<const float*>(A);
    if (r <= 16) {
      if (R >= 256 && L * t256 >= 2 * (int64_t)g_num_sms)
        k_ttm_f32<256, 16, 16><<<dim3((unsigned)(L * t256), 1), 64, ttm_f32_smem<256, 16, 16>(), st>>>(Af, n, R, t256, U, r,
                                                                                               out);
      else
        k_ttm_f32<128, 16, 16><<<dim3((unsigned)(L * t128), 1), 32, ttm_f32_smem<128, 16, 16>(), st>>>(Af, n, R, t128, U, r,
                                                                                               out);
      return 1;
    }
    const unsigned gy = (unsigned)((r + 31) / 32);
    if (R >= 256 && L * t256 * gy >= 2 * (int64_t)g_num_sms)
      k_ttm_f32<256, 32, 32><<<dim3((unsigned)(L * t256), gy), 128, ttm_f32_smem<256, 32, 32>(), st>>>(Af, n, R, t256, U, r,
                                                                                               out);
    else
      k_ttm_f32<128, 32, 32><<<dim3((unsigned)(L * t128), gy), 64, ttm_f32_smem<128, 32, 32>(), st>>>(Af, n, R, t128, U, r,
                                                                                              out);
    return 1;
  }
  dim3 grid((unsigned)((ncol + TT_BN - 1) / TT_BN), (unsigned)((r + TT_BM - 1) / TT_BM));
  if (dtype == DT_F32)
    k_ttm_t<float><<<grid, 256, 0, st>>>(static_cast<const float*>(A), L, n, R, U, r, out);
  else if (dtype == DT_F64)
    k_ttm_t<double><<<grid, 256, 0, st>>>(static_cast<const double*>(A), L, n, R, U, r, out);
  else
    k_ttm_t<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(A), L, n, R, U, r, out);
  return 1;
}

int64_t ttm_last_job_ctas(const TTMJob& q) { return (q.L + TL_THREADS - 1) / TL_THREADS; }

int launch_ttm_last_grouped(const TTMJob* jobs_dev, const int64_t* pre_dev, int njobs, int64_t total_ctas,
                            int dtype, int nmax, int rmax, cudaStream_t st) {
  if (njobs < 1 || total_ctas < 1 || nmax > 256 || rmax > 32) return 0;
  const int rw = rmax <= 8 ? 8 : rmax <= 16 ? 16 : rmax <= 24 ? 24 : 32;
  const size_t smem = (size_t)nmax * rw * 4;
  const unsigned grid = (unsigned)total_ctas;
#define RT_TLG(T, RWV)                                                                       \
  k_ttm_last_grouped<T, RWV><<<grid, TL_THREADS, smem, st>>>(jobs_dev, pre_dev, njobs)
#define RT_TLG_RW(T)                                                                          \
  if (rw == 8) RT_TLG(T, 8); else if (rw == 16) RT_TLG(T, 16); else if (rw == 24) RT_TLG(T, 24); else RT_TLG(T, 32)
  if (dtype == DT_F32) { RT_TLG_RW(float); }
  else if (dtype == DT_F64) { RT_TLG_RW(double); }
  else { RT_TLG_RW(__nv_bfloat16); }
#undef RT_TLG_RW
#undef RT_TLG
  return 1;
}

int64_t ttm_job_tiles(TTMJob& q) {
  q.tiles_x = (q.L * q.R + TT_BN - 1) / TT_BN;
  return q.tiles_x * ((q.r + TT_BM - 1) / TT_BM);
}

int launch_ttm_grouped(const TTMJob* jobs_dev, const int64_t* pre_dev, int njobs, int64_t total_tiles, int dtype,
                       cudaStream_t st) {
  if (njobs < 1 || total_tiles < 1) return 0;
  const unsigned grid = (unsigned)total_tiles;
  if (dtype == DT_F32) k_ttm_grouped<float><<<grid, 256, 0, st>>>(jobs_dev, pre_dev, njobs);
  else if (dtype == DT_F64) k_ttm_grouped<double><<<grid, 256, 0, st>>>(jobs_dev, pre_dev, njobs);
  else k_ttm_grouped<__nv_bfloat16><<<grid, 256, 0, st>>>(jobs_dev, pre_dev, njobs);
  return 1;
}

cudaError_t core_init_attributes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
#define RT_TTM_ATTR(TN, AW, TK)                                                                          \
  if (e == cudaSuccess)                                                                                    \
    e = cudaFuncSetAttribute(k_ttm_f32<TN, AW, TK>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                             (int)ttm_f32_smem<TN, AW, TK>());
  RT_TTM_ATTR(256, 32, 32) RT_TTM_ATTR(128, 32, 32) RT_TTM_ATTR(256, 16, 16) RT_TTM_ATTR(128, 16, 16)
#undef RT_TTM_ATTR
  return e;
}

}  // namespace rt
