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

#include <algorithm>

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

  // acc2[x][m] holds outputs (x, 2m) and (x, 2m + 1): one packed fma.rn.f32x2 per pair
  uint64_t acc2[8][4];
#pragma unroll
  for (int x = 0; x < 8; ++x)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc2[x][m] = 0ull;

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
      const uint64_t bb[4] = {f2_pack(b0.x, b0.y), f2_pack(b0.z, b0.w), f2_pack(b1.x, b1.y), f2_pack(b1.z, b1.w)};
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const uint64_t uu = f2_pack(ua[x], ua[x]);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc2[x][m] = f2_fma(uu, bb[m], acc2[x][m]);
      }
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
      float v[4];
      f2_unpack(acc2[x][2 * h], v[0], v[1]);
      f2_unpack(acc2[x][2 * h + 1], v[2], v[3]);
      if (rho + 4 <= R) {
        *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if (rho + y < R) o[y] = v[y];
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

// The last two modes of float32 X in one read, for small slabs (n1 <= TL_THREADS rows
// of n2 values): a CTA owns spc = TL_THREADS / n1 whole slabs.  Thread per row l:
// T(l, b) = sum_j U2[j][b] X(l, j) in registers (as k_ttm_last, U2 zero-padded to RW
// columns in shared memory), written to shared memory; then the slabs' outputs
// P(s, a, b) = sum_i U1[i][a] T(s n1 + i, b), one per thread and step, written
// contiguously.  float32 products and sums, j then i in order.
// Dynamic smem: us[n2][RW] | Ts[spc n1][RW + 1] | U1s[n1][r1]
template <int RW>
__global__ void __launch_bounds__(TL_THREADS) k_last2(const float* __restrict__ A, int64_t S, int n1, int n2,
                                                      const float* __restrict__ U1, int r1,
                                                      const float* __restrict__ U2, int r2,
                                                      float* __restrict__ out) {
  extern __shared__ __align__(16) float l2m[];
  constexpr int LDT = RW + 1;                    // odd stride: row-wise stores are conflict-free
  const int spc = TL_THREADS / n1;
  float* us = l2m;
  float* Ts = us + n2 * RW;
  float* U1s = Ts + spc * n1 * LDT;
  for (int e = threadIdx.x; e < n2 * RW; e += TL_THREADS) {
    const int j = e / RW, b = e % RW;
    us[e] = b < r2 ? U2[j * r2 + b] : 0.f;
  }
  for (int e = threadIdx.x; e < n1 * r1; e += TL_THREADS) U1s[e] = U1[e];
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * spc;
  const int nsl = (int)min((int64_t)spc, S - s0);
  const int t = threadIdx.x;
  if (t < nsl * n1) {
    const float* row = A + (s0 * n1 + t) * n2;
    float acc[RW];
#pragma unroll
    for (int b = 0; b < RW; ++b) acc[b] = 0.f;
    const bool v4 = (n2 % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    for (int j0 = 0; j0 < n2; j0 += 4) {
      float x[4];
      if (v4) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(row + j0));
        x[0] = f.x; x[1] = f.y; x[2] = f.z; x[3] = f.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = j0 + q < n2 ? __ldg(row + j0 + q) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (j0 + q >= n2) break;
        const float* uj = us + (j0 + q) * RW;
#pragma unroll
        for (int b = 0; b < RW; b += 4) {
          const float4 u = *reinterpret_cast<const float4*>(uj + b);
          acc[b] = fmaf(x[q], u.x, acc[b]);
          acc[b + 1] = fmaf(x[q], u.y, acc[b + 1]);
          acc[b + 2] = fmaf(x[q], u.z, acc[b + 2]);
          acc[b + 3] = fmaf(x[q], u.w, acc[b + 3]);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < RW; ++b) Ts[t * LDT + b] = acc[b];
  }
  __syncthreads();
  const int osz = r1 * r2;
  float* dst = out + s0 * osz;
  for (int o = t; o < nsl * osz; o += TL_THREADS) {
    const int b = o % r2, a = (o / r2) % r1, s = o / osz;
    const float* tp = Ts + s * n1 * LDT + b;
    float acc = 0.f;
    for (int i = 0; i < n1; ++i) acc = fmaf(U1s[i * r1 + a], tp[i * LDT], acc);
    dst[o] = acc;
  }
}

// Grouped last-mode contractions (R = 1) of a batch: job q contracts the last mode of
// its L x n tensor with U_q (n x r <= RW), one thread per row.  pre[j] counts CTAs of
// TL_THREADS rows before job j.  A's element type T (the batch's X type at the first
// level); 16-byte loads for float rows with n % 4 == 0.
// Rows [lb0, lb0 + rb TL_THREADS) of one job, RWJ >= r output columns: U in us
// ([n][RWJ], zero beyond r).  Each warp walks its 32-row groups in 32-column chunks:
// a chunk is read by 32 coalesced row loads into registers one chunk ahead (so the
// loads of the next chunk are in flight while this one is computed), transposed
// through the warp's 32 x 33 tile, and lane i takes row i.
template <typename T, int RWJ>
__device__ __forceinline__ void last_rows(const TTMJob& q, const float* us, float* tile, int64_t lb0, int rbn) {
  const int n = (int)q.n, r = q.r;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (n + 31) >> 5;
  int nrb = 0;                                   // this warp's row groups
  while (nrb < rbn && lb0 + (int64_t)nrb * TL_THREADS + warp * 32 < q.L) ++nrb;
  const int nchunk = nrb * nk;
  float v[32];
  auto fetch = [&](int c) {
    const int rb = c / nk, k0 = (c % nk) * 32;
    const int64_t l0 = lb0 + (int64_t)rb * TL_THREADS + warp * 32;
    const int nrow = (int)(q.L - l0 < 32 ? q.L - l0 : 32);
    const T* base = static_cast<const T*>(q.A) + l0 * n;
    const bool col = k0 + lane < n;
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = (i < nrow && col) ? ldf<T>(base + (int64_t)i * n, k0 + lane) : 0.f;
  };
  if (nchunk > 0) fetch(0);
  float acc[RWJ];
#pragma unroll
  for (int a = 0; a < RWJ; ++a) acc[a] = 0.f;
  for (int c = 0; c < nchunk; ++c) {
#pragma unroll
    for (int i = 0; i < 32; ++i) tile[i * 33 + lane] = v[i];
    __syncwarp();
    if (c + 1 < nchunk) fetch(c + 1);
    const int rb = c / nk, k0 = (c % nk) * 32, kw = min(32, n - k0);
    for (int kk = 0; kk < kw; ++kk) {
      const float x = tile[lane * 33 + kk];
      const float* ui = us + (k0 + kk) * RWJ;
#pragma unroll
      for (int a = 0; a < RWJ; a += 4) {
        const float4 u = *reinterpret_cast<const float4*>(ui + a);
        acc[a] = fmaf(x, u.x, acc[a]);
        acc[a + 1] = fmaf(x, u.y, acc[a + 1]);
        acc[a + 2] = fmaf(x, u.z, acc[a + 2]);
        acc[a + 3] = fmaf(x, u.w, acc[a + 3]);
      }
    }
    __syncwarp();
    if (k0 + 32 >= n) {                          // the row group is complete
      const int64_t l0 = lb0 + (int64_t)rb * TL_THREADS + warp * 32;
      if (l0 + lane < q.L) {
        float* o = q.out + (l0 + lane) * r;
#pragma unroll
        for (int a = 0; a < RWJ; ++a)
          if (a < r) o[a] = acc[a];
      }
#pragma unroll
      for (int a = 0; a < RWJ; ++a) acc[a] = 0.f;
    }
  }
}

template <typename T, int RWJ>
__device__ __forceinline__ void last_job(const TTMJob& q, float* us, int64_t lb0, int rbn) {
  const int n = (int)q.n, r = q.r;
  for (int e = threadIdx.x; e < n * RWJ; e += TL_THREADS) {
    const int i = e / RWJ, a = e % RWJ;
    us[e] = a < r ? q.U[i * r + a] : 0.f;
  }
  __syncthreads();
  float* tile = us + (((n * RWJ) + 3) & ~3) + (threadIdx.x >> 5) * (32 * 33);
  last_rows<T, RWJ>(q, us, tile, lb0, rbn);
}

// One launch for the last-mode contraction of many jobs (out[l][a] = sum_i A[l][i] U[i][a],
// row-major A of L x n): CTAs mapped onto jobs by prefix, rbn 128-row blocks each (the
// batched autotuner's choice), U of the job staged once per CTA at the job's own rank
// width (8, 16, 24 or 32 <= RW).
template <typename T, int RW>
__global__ void __launch_bounds__(TL_THREADS) k_ttm_last_grouped(const TTMJob* __restrict__ jobs,
                                                                 const int64_t* __restrict__ pre, int njobs,
                                                                 int rbn) {
  extern __shared__ __align__(16) float us[];   // [n][RWJ] | per warp a 32 x 33 tile
  const int j = find_prob(pre, njobs, blockIdx.x);
  const TTMJob& q = jobs[j];
  const int64_t lb0 = ((int64_t)blockIdx.x - pre[j]) * (TL_THREADS * (int64_t)rbn);
  if (q.r <= 8) last_job<T, 8>(q, us, lb0, rbn);
  else if (RW >= 16 && q.r <= 16) last_job<T, (RW >= 16 ? 16 : 8)>(q, us, lb0, rbn);
  else if (RW >= 24 && q.r <= 24) last_job<T, (RW >= 24 ? 24 : 8)>(q, us, lb0, rbn);
  else if (RW >= 32) last_job<T, (RW >= 32 ? 32 : 8)>(q, us, lb0, rbn);
}

// ---------------------------------------------------------------- two modes of small slabs
// out(l, a, b, rho) = sum_{i,j} U1[i][a] U2[j][b] A(l, i, j, rho) for A of (L, n1, n2, R):
// two neighbouring modes contracted in one read of A when a slab (n1 n2 R values) fits
// in shared memory, for the small slabs that the tensor-core pass tiles poorly (its
// M = 128 rows per slab).  A CTA takes batches of nb consecutive slabs (contiguous in
// A): it forms T(s, i, b, rho) = sum_j U2[j][b] A(s, i, j, rho), then the outputs, one
// output per thread and step, and writes the batch's outputs (contiguous in out).
// float32 A is staged by cp.async into two buffers, the next batch's copies in flight
// while the current one is contracted; other dtypes are converted on a plain load.
// float32 products and sums, j then i in order.
// Dynamic smem: As[2][nb n1 n2 R] (one buffer for non-float32 A) | Ts[nb n1 r2 R] |
//               U1s[n1 r1] | U2s[n2 r2]
constexpr int S2_THREADS = 256, S2_MAXA = 12288, S2_FILL = 6144, S2_MAXT = 4096, S2_MAXU = 2048;

__device__ __forceinline__ void slab2_contract(const float* __restrict__ As, float* __restrict__ Ts,
                                               const float* __restrict__ U1s, const float* __restrict__ U2s,
                                               int cnt, int n1, int n2, int R, int r1, int r2,
                                               float* __restrict__ dst) {
  const int tsz = n1 * r2 * R, osz = r1 * r2 * R;
  for (int o = threadIdx.x; o < cnt * tsz; o += S2_THREADS) {   // o = ((s n1 + i) r2 + b) R + rho
    const int rho = o % R, b = (o / R) % r2, si = o / (R * r2);
    const float* a = As + (size_t)si * n2 * R + rho;
    float acc = 0.f;
    for (int j = 0; j < n2; ++j) acc = fmaf(U2s[j * r2 + b], a[j * R], acc);
    Ts[o] = acc;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < cnt * osz; o += S2_THREADS) {   // o = ((s r1 + a) r2 + b) R + rho
    const int rho = o % R, b = (o / R) % r2, a = (o / (R * r2)) % r1, s = o / osz;
    const float* t = Ts + (size_t)s * tsz + b * R + rho;
    float acc = 0.f;
    for (int i = 0; i < n1; ++i) acc = fmaf(U1s[i * r1 + a], t[i * r2 * R], acc);
    dst[o] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(S2_THREADS) k_slab2(const T* __restrict__ A, int64_t L, int n1, int n2, int R,
                                                      int nb, const float* __restrict__ U1, int r1,
                                                      const float* __restrict__ U2, int r2, float* __restrict__ out) {
  extern __shared__ __align__(16) float s2m[];
  constexpr bool F32 = sizeof(T) == 4;
  const int slab = n1 * n2 * R, osz = r1 * r2 * R;
  float* As = s2m;
  float* Ts = As + (F32 ? 2 : 1) * nb * slab;
  float* U1s = Ts + nb * n1 * r2 * R;
  float* U2s = U1s + n1 * r1;
  for (int e = threadIdx.x; e < n1 * r1; e += S2_THREADS) U1s[e] = U1[e];
  for (int e = threadIdx.x; e < n2 * r2; e += S2_THREADS) U2s[e] = U2[e];
  const int64_t nbatch = (L + nb - 1) / nb;
  if constexpr (F32) {
    const float* Af = reinterpret_cast<const float*>(A);
    const bool v4 = (slab % 4) == 0 && (reinterpret_cast<uintptr_t>(Af) & 15) == 0;
    // copies of batch bt into buffer q, one commit group per batch (empty past the end)
    auto issue = [&](int64_t bt, int q) {
      if (bt < nbatch) {
        const int64_t l0 = bt * nb;
        const int tot = (int)min((int64_t)nb, L - l0) * slab;
        const float* src = Af + l0 * slab;
        float* dst = As + q * nb * slab;
        if (v4) {
          for (int e = threadIdx.x; e < tot / 4; e += S2_THREADS) cp_async16(dst + 4 * e, src + 4 * e, 16);
        } else {
          for (int e = threadIdx.x; e < tot; e += S2_THREADS) cp_async4(dst + e, src + e, 4);
        }
      }
      cp_async_commit();
    };
    int q = 0;
    issue(blockIdx.x, 0);
    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, q ^= 1) {
      issue(bt + gridDim.x, q ^ 1);          // the next batch streams in meanwhile
      cp_async_wait<1>();                    // this batch's copies (all but the newest group)
      __syncthreads();
      const int64_t l0 = bt * nb;
      const int cnt = (int)min((int64_t)nb, L - l0);
      slab2_contract(As + q * nb * slab, Ts, U1s, U2s, cnt, n1, n2, R, r1, r2, out + l0 * osz);
      __syncthreads();                       // buffer q and Ts are free for the next round
    }
    cp_async_wait<0>();
  } else {
    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
      const int64_t l0 = bt * nb;
      const int cnt = (int)min((int64_t)nb, L - l0);
      const T* src = A + l0 * slab;
      __syncthreads();
      for (int e = threadIdx.x; e < cnt * slab; e += S2_THREADS) As[e] = ldf<T>(src, e);
      __syncthreads();
      slab2_contract(As, Ts, U1s, U2s, cnt, n1, n2, R, r1, r2, out + l0 * osz);
    }
  }
}

static int slab2_batch(int n1, int n2, int64_t R, int r1, int r2) {
  if (n1 < 1 || n2 < 1 || R < 1 || r1 < 1 || r2 < 1) return 0;
  const int64_t slab = (int64_t)n1 * n2 * R, tsz = (int64_t)n1 * r2 * R;
  if (slab > S2_MAXA || tsz > S2_MAXT || (int64_t)n1 * r1 + (int64_t)n2 * r2 > S2_MAXU) return 0;
  return (int)std::max<int64_t>(1, std::min(S2_FILL / slab, S2_MAXT / tsz));
}

static size_t slab2_smem() { return (size_t)(2 * S2_MAXA + S2_MAXT + S2_MAXU) * 4; }

static int g_num_sms = 0;

constexpr int L2_MAXN2 = 256, L2_MAXR1 = 32;
template <int RW>
static size_t last2_smem_max() {
  return ((size_t)L2_MAXN2 * RW + (size_t)TL_THREADS * (RW + 1) + (size_t)TL_THREADS * L2_MAXR1) * 4;
}

bool last2_fits(int64_t n1, int64_t n2, int r1, int r2) {
  return n1 >= 1 && n1 <= TL_THREADS && n2 >= 1 && n2 <= L2_MAXN2 && r1 >= 1 && r1 <= L2_MAXR1 && r2 >= 1 &&
         r2 <= 32;
}

int launch_last2(const float* X, int64_t S, int64_t n1, int64_t n2, const float* U1, int r1, const float* U2, int r2,
                 float* out, cudaStream_t st) {
  if (!last2_fits(n1, n2, r1, r2) || S < 1) return 0;
  const int spc = TL_THREADS / (int)n1;
  const int64_t blocks = (S + spc - 1) / spc;
  if (blocks >= ((int64_t)1 << 31)) return 0;
  const int rw = r2 <= 8 ? 8 : r2 <= 16 ? 16 : 32;
  const size_t sm = ((size_t)n2 * rw + (size_t)spc * n1 * (rw + 1) + (size_t)n1 * r1) * 4;
  if (rw == 8)
    k_last2<8><<<(unsigned)blocks, TL_THREADS, sm, st>>>(X, S, (int)n1, (int)n2, U1, r1, U2, r2, out);
  else if (rw == 16)
    k_last2<16><<<(unsigned)blocks, TL_THREADS, sm, st>>>(X, S, (int)n1, (int)n2, U1, r1, U2, r2, out);
  else
    k_last2<32><<<(unsigned)blocks, TL_THREADS, sm, st>>>(X, S, (int)n1, (int)n2, U1, r1, U2, r2, out);
  return 1;
}

bool slab2_fits(int64_t n1, int64_t n2, int64_t R, int r1, int r2) {
  return n1 <= 65536 && n2 <= 65536 && slab2_batch((int)n1, (int)n2, R, r1, r2) > 0;
}

int launch_slab2(const void* A, int dtype, int64_t L, int64_t n1, int64_t n2, int64_t R, const float* U1, int r1,
                 const float* U2, int r2, float* out, cudaStream_t st) {
  if (!slab2_fits(n1, n2, R, r1, r2) || L < 1) return 0;
  const int nb = slab2_batch((int)n1, (int)n2, R, r1, r2);
  const int64_t nbatch = (L + nb - 1) / nb;
  const int64_t cap = (int64_t)std::max(1, g_num_sms) * 8;
  const unsigned grid = (unsigned)std::min(nbatch, cap);
  const size_t sm = ((size_t)(dtype == DT_F32 ? 2 : 1) * nb * n1 * n2 * R + (size_t)nb * n1 * r2 * R + n1 * r1 +
                     n2 * r2) * 4;
  if (dtype == DT_F32)
    k_slab2<float><<<grid, S2_THREADS, sm, st>>>(static_cast<const float*>(A), L, (int)n1, (int)n2, (int)R, nb, U1,
                                                 r1, U2, r2, out);
  else if (dtype == DT_F64)
    k_slab2<double><<<grid, S2_THREADS, sm, st>>>(static_cast<const double*>(A), L, (int)n1, (int)n2, (int)R, nb,
                                                  U1, r1, U2, r2, out);
  else
    k_slab2<__nv_bfloat16><<<grid, S2_THREADS, sm, st>>>(static_cast<const __nv_bfloat16*>(A), L, (int)n1,
                                                         (int)n2, (int)R, nb, U1, r1, U2, r2, out);
  return 1;
}

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

int64_t ttm_last_job_ctas(const TTMJob& q, int rbn) {
  return (q.L + (int64_t)TL_THREADS * rbn - 1) / ((int64_t)TL_THREADS * rbn);
}

int launch_ttm_last_grouped(const TTMJob* jobs_dev, const int64_t* pre_dev, int njobs, int64_t total_ctas,
                            int dtype, int nmax, int rmax, int rbn, cudaStream_t st) {
  if (njobs < 1 || total_ctas < 1 || nmax > 256 || rmax > 32 || rbn < 1) return 0;
  const int rw = rmax <= 8 ? 8 : rmax <= 16 ? 16 : rmax <= 24 ? 24 : 32;
  const size_t smem = (((size_t)nmax * rw + 3) & ~(size_t)3) * 4 + (size_t)(TL_THREADS / 32) * 32 * 33 * 4;
  const unsigned grid = (unsigned)total_ctas;
#define RT_TLG(T, RWV)                                                                                     \
  do {                                                                                                     \
    cudaFuncSetAttribute(k_ttm_last_grouped<T, RWV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k_ttm_last_grouped<T, RWV><<<grid, TL_THREADS, smem, st>>>(jobs_dev, pre_dev, njobs, rbn);              \
  } while (0)
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
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_last2<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)last2_smem_max<8>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_last2<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)last2_smem_max<16>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_last2<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)last2_smem_max<32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_slab2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab2_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_slab2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab2_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_slab2<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)slab2_smem());
  return e;
}

}  // namespace rt
