// rf_kernels.cu - range finder of the subsampled randomized HOSVD / RtL-HT.
//
// For every problem (mode k of a tensor, Alg. 1; or node S of the dimension
// tree, Alg. 2) the stages are:
//   S1  sample  : pi(j), column offsets in X, Gaussian rows Omega(j, :)  (Sec. 3.1)
//   S2+S4 gather/sketch : Y = X^(S) E (kept as Y^T), Z = Y Omega (partials per
//         sample chunk)                                                  (Sec. 3.1)
//   S5  qr      : Z = Q R, Householder in shared memory, diag(R) > 0; tall Z
//         by a two-level TSQR                                     (Alg. 1, Q_k)
//   S6  W-step  : B = Q^T Y; TSQR of B^T -> R; one-sided Jacobi on R^T gives
//         the left singular vectors W of B (B B^T = R^T R); U = Q W(:, :r) with
//         each column's largest-magnitude entry made positive     (Alg. 1, W_k, U_k)
// All arithmetic is float32.  GB300's float64 rate is ~1/64 of float32, so the
// small factorisations use backward-stable float32 algorithms (Householder,
// one-sided Jacobi) instead of float64 Gram/eigen solves: the singular vectors
// then carry errors of order u ||B|| / gap rather than u ||B||^2 / gap^2.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rt_common.cuh"
#include "rt_host.h"
#include "rt_rng.cuh"
#include "rf_svd.cuh"

namespace rt {

// ------------------------------------------------------------------ S1
__global__ void __launch_bounds__(256) k_sample(const RFProb* __restrict__ P,
                                                const int64_t* __restrict__ pre, int np,
                                                int* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pre[np]) return;
  const int p = find_prob(pre, np, t);
  const RFProb& q = P[p];
  const int64_t j = t - pre[p];
  const PhiloxKey key = philox_key(q.seed);
  const uint64_t m = sample_index((uint64_t)j, (uint64_t)q.N, q.fh, key, q.node, status);
  q.idx[j] = (int64_t)m;
  uint64_t rem = m;
  int64_t off = 0;
  for (int t2 = q.ncm - 1; t2 >= 0; --t2) {
    const uint64_t sz = (uint64_t)q.csize[t2];
    off += (int64_t)(rem % sz) * q.cstride[t2];
    rem /= sz;
  }
  q.off[j] = off;
}

// ------------------------------------------------------------------ S2 + S4
// One CTA: rows [i0, i0+TI) x samples [j0, j0+TJ) of Y = X^(S) E.
// Dynamic smem: Ys[TJ][TI] | Os[TJ][CMAX] | offs[TJ] (int64)
__global__ void __launch_bounds__(256) k_gather_sketch(const RFProb* __restrict__ P,
                                                       const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);
  float* Os = Ys + SK_TJ * SK_TI;
  int64_t* offs = reinterpret_cast<int64_t*>(Os + SK_TJ * CMAX);
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int64_t local = (int64_t)blockIdx.x - pre[p];
  const int64_t nrt = (q.nS + SK_TI - 1) / SK_TI;
  const int64_t chunk = local / nrt, rtile = local % nrt;
  const int64_t i0 = rtile * SK_TI, j0 = chunk * SK_TJ;
  const int c = q.c, cp = (c + 3) & ~3;
  const int tid = threadIdx.x;
  if (tid < SK_TJ) offs[tid] = (j0 + tid < q.s) ? q.off[j0 + tid] : (int64_t)-1;
  __syncthreads();
  const int64_t nS = q.nS, rs = q.rowstride;
  // All loads of this thread are issued before any store, so the strided gathers (one
  // DRAM sector each for all but the last mode) overlap instead of waiting on one another.
  constexpr int PER = SK_TI * SK_TJ / 256;
  static_assert(SK_TI * SK_TJ % 256 == 0 && 256 % SK_TI == 0, "gather tiling");
  const int ii = tid % SK_TI;
  const int64_t i = i0 + ii;
  float v[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int jj = tid / SK_TI + t * (256 / SK_TI);
    const int64_t o = offs[jj];
    v[t] = (i < nS && o >= 0) ? load_xq(q, o + i * rs) : 0.f;
  }
  const bool bf = q.skbf16 != 0;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int jj = tid / SK_TI + t * (256 / SK_TI);
    if (i < nS && offs[jj] >= 0) q.Yt[(j0 + jj) * nS + i] = v[t];
    Ys[jj * SK_TI + ii] = bf ? __bfloat162float(__float2bfloat16_rn(v[t])) : v[t];
  }
  for (int e = tid; e < SK_TJ * cp; e += 256) {
    const int jj = e / cp, cc = e % cp;
    const float o = (j0 + jj < q.s && cc < c) ? q.Om[(j0 + jj) * c + cc] : 0.f;
    Os[jj * CMAX + cc] = bf ? __bfloat162float(__float2bfloat16_rn(o)) : o;
  }
  __syncthreads();
  const int ncg = cp >> 2;
  float* zp = q.Zp + chunk * nS * c;
  for (int t = tid; t < (SK_TI / 4) * ncg; t += 256) {
    const int rg = t % (SK_TI / 4), cg = t / (SK_TI / 4);
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 8
    for (int jj = 0; jj < SK_TJ; ++jj) {
      const float4 y = *reinterpret_cast<const float4*>(Ys + jj * SK_TI + rg * 4);
      const float4 o = *reinterpret_cast<const float4*>(Os + jj * CMAX + cg * 4);
      const float ya[4] = {y.x, y.y, y.z, y.w};
      const float ob[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ya[a], ob[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + rg * 4 + a;
      if (i >= nS) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int col = cg * 4 + b;
        if (col < c) zp[i * c + col] = acc[a][b];
      }
    }
  }
  if (q.nzc == 1) return;
  // The last CTA of this row tile to finish sums the nzc partial sketches of the tile,
  // in chunk order, into the chunk-0 slot (deterministic; no second pass over Zp).
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(q.zcnt + rtile, 1) == q.nzc - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int64_t zsz = nS * c;
  const int rows = (int)min((int64_t)SK_TI, nS - i0);
  for (int e = tid; e < rows * c; e += 256) {
    const float* src = q.Zp + i0 * c + e;
    float acc = 0.f;
    for (int ch0 = 0; ch0 < q.nzc; ch0 += 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = (ch0 + u < q.nzc) ? __ldcg(src + (int64_t)(ch0 + u) * zsz) : 0.f;
#pragma unroll
      for (int u = 0; u < 16; ++u) acc += v[u];
    }
    q.Zp[i0 * c + e] = acc;
  }
  if (tid == 0) q.zcnt[rtile] = 0;
}

// Z (reduced into the chunk-0 slot by the gather/sketch kernel) to the caller (test path).
__global__ void k_sketch_sum(const RFProb* __restrict__ P, const int64_t* __restrict__ pre, int np,
                             float* const* __restrict__ Zout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pre[np]) return;
  const int p = find_prob(pre, np, t);
  const RFProb& q = P[p];
  const int64_t e = t - pre[p];
  Zout[p][e] = q.Zp[e];
}

// ------------------------------------------------------------------ Householder QR in smem
// A is column-major (A[col * ld + row]), m x c.  On exit the columns hold the
// Householder vectors v_k (v_k[k] stored at A[k*ld+k]), the strict upper part
// holds R, rdiag[k] = R_kk and tau[k] the reflector scales, H_k = I - tau v v^T.
//
// Warp w owns the columns j with j % nwarps == w.  In step k every warp applies
// H_k to its columns j > k; the owner of column k+1 updates that column first
// and forms H_{k+1} from it right away, so each step needs one block barrier.

// Reflector of column k (rows k..m-1), formed by one warp.
__device__ __forceinline__ void hh_make(float* A, int ld, int m, int k, float* tau, float* rdiag) {
  const int lane = threadIdx.x & 31;
  float* a = A + (size_t)k * ld;
  float part = 0.f;
  for (int i = k + lane; i < m; i += 32) part = fmaf(a[i], a[i], part);
  const float nrm2 = warp_sum(part);
  if (lane == 0) {
    const float x0 = a[k];
    const float nrm = sqrtf(nrm2);
    if (nrm == 0.f) {
      tau[k] = 0.f;
      rdiag[k] = 0.f;
    } else {
      const float alpha = (x0 >= 0.f) ? -nrm : nrm;
      tau[k] = 1.f / (nrm * (nrm + fabsf(x0)));   // 2 / (v^T v)
      rdiag[k] = alpha;
      a[k] = x0 - alpha;
    }
  }
  __syncwarp();
}

__device__ void hh_factor(float* A, int ld, int m, int c, float* tau, float* rdiag, float* /*red*/) {
  const int K = min(m, c);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (K <= 0) return;
  if (warp == 0) hh_make(A, ld, m, 0, tau, rdiag);
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    const float tk = tau[k];
    const float* v = A + (size_t)k * ld;
    int j = k + 1 + ((warp - (k + 1)) % nw + nw) % nw;   // smallest owned column > k
    for (; j < c; j += nw) {
      float* aj = A + (size_t)j * ld;
      if (tk != 0.f) {
        float w = 0.f;
        for (int i = k + lane; i < m; i += 32) w = fmaf(v[i], aj[i], w);
        w = warp_sum(w) * tk;
        for (int i = k + lane; i < m; i += 32) aj[i] = fmaf(-w, v[i], aj[i]);
        __syncwarp();
      }
      if (j == k + 1 && k + 1 < K) hh_make(A, ld, m, k + 1, tau, rdiag);
    }
    __syncthreads();
  }
}

// Qm (column-major, ld) = H_0 ... H_{K-1} [I; 0], then the signs making diag(R) > 0.
__device__ void hh_form_q(const float* A, float* Qm, int ld, int m, int c, const float* tau,
                          const float* rdiag, bool fix_sign) {
  const int K = min(m, c);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int j = e / m, i = e % m;
    Qm[(size_t)j * ld + i] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  for (int k = K - 1; k >= 0; --k) {
    const float tk = tau[k];
    if (tk != 0.f) {
      const float* v = A + (size_t)k * ld;
      for (int j = k + warp; j < c; j += nw) {
        float* qj = Qm + (size_t)j * ld;
        float w = 0.f;
        for (int i = k + lane; i < m; i += 32) w = fmaf(v[i], qj[i], w);
        w = warp_sum(w) * tk;
        for (int i = k + lane; i < m; i += 32) qj[i] = fmaf(-w, v[i], qj[i]);
      }
    }
    __syncthreads();
  }
  if (fix_sign) {
    for (int e = threadIdx.x; e < m * K; e += blockDim.x) {
      const int j = e / m, i = e % m;
      if (rdiag[j] < 0.f) Qm[(size_t)j * ld + i] = -Qm[(size_t)j * ld + i];
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int odd_ld(int m) { return m | 1; }

// ------------------------------------------------------------------ register-resident Householder
// Same factorisation as hh_factor / hh_form_q for m <= 32*MR rows and
// c <= JPW*nwarps columns, with column j held in the registers of warp
// j % nwarps (lane l: rows l + 32 t).  Step k: the owner of column k forms
// H_k and publishes v_k through a double-buffered shared vector; one block
// barrier; every warp applies H_k to its own columns.  A is read at entry and
// written back (R above the diagonal, v_k at and below it) at exit.
template <int MR, int JPW>
__device__ void hh_factor_reg(float* A, int ld, int m, int c, float* tau, float* rdiag, float* vbuf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int K = min(m, c);
  float col[JPW][MR];
#pragma unroll
  for (int u = 0; u < JPW; ++u) {
    const int j = warp + u * nw;
#pragma unroll
    for (int t = 0; t < MR; ++t) {
      const int i = lane + 32 * t;
      col[u][t] = (j < c && i < m) ? A[(size_t)j * ld + i] : 0.f;
    }
  }
  for (int k = 0; k < K; ++k) {
    float* vb = vbuf + (k & 1) * (32 * MR);
    if (warp == k % nw) {
      const int uk = k / nw;
      float s2 = 0.f, xk = 0.f;
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        if (u != uk) continue;
#pragma unroll
        for (int t = 0; t < MR; ++t) {
          const int i = lane + 32 * t;
          const float x = col[u][t];
          if (i >= k && i < m) s2 = fmaf(x, x, s2);
          if (t == (k >> 5)) xk = x;
        }
      }
      s2 = warp_sum(s2);
      const float x0 = __shfl_sync(0xffffffffu, xk, k & 31);
      const float nrm = sqrtf(s2);
      const float alpha = (x0 >= 0.f) ? -nrm : nrm;
      const float tk = (nrm == 0.f) ? 0.f : 1.f / (nrm * (nrm + fabsf(x0)));
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        if (u != uk) continue;
#pragma unroll
        for (int t = 0; t < MR; ++t) {
          const int i = lane + 32 * t;
          float v = (i > k && i < m) ? col[u][t] : 0.f;
          if (i == k && nrm != 0.f) {
            v = x0 - alpha;
            col[u][t] = v;
          }
          vb[i] = (i == k && nrm == 0.f) ? 0.f : v;
        }
      }
      if (lane == 0) {
        tau[k] = tk;
        rdiag[k] = (nrm == 0.f) ? 0.f : alpha;
      }
    }
    __syncthreads();
    const float tk = tau[k];
    if (tk != 0.f) {
      float vr[MR];
#pragma unroll
      for (int t = 0; t < MR; ++t) vr[t] = vb[lane + 32 * t];
      float w[JPW];
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        w[u] = 0.f;
#pragma unroll
        for (int t = 0; t < MR; ++t) w[u] = fmaf(vr[t], col[u][t], w[u]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < JPW; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        const int j = warp + u * nw;
        if (j > k && j < c) {
          const float s = w[u] * tk;
#pragma unroll
          for (int t = 0; t < MR; ++t) col[u][t] = fmaf(-s, vr[t], col[u][t]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < JPW; ++u) {
    const int j = warp + u * nw;
    if (j >= c) continue;
#pragma unroll
    for (int t = 0; t < MR; ++t) {
      const int i = lane + 32 * t;
      if (i < m) A[(size_t)j * ld + i] = col[u][t];
    }
  }
  __syncthreads();
}

// As hh_factor_reg, with the owner of column k tracked by counters instead of k % nw
// and warps whose columns are all finished skipping the update.  Faster where the
// block holds only the QR (k_qr1, k_wsvd); inside k_bt_fused the original schedules
// better.
template <int MR, int JPW>
__device__ void hh_factor_reg_ct(float* A, int ld, int m, int c, float* tau, float* rdiag, float* vbuf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int K = min(m, c);
  float col[JPW][MR];
#pragma unroll
  for (int u = 0; u < JPW; ++u) {
    const int j = warp + u * nw;
#pragma unroll
    for (int t = 0; t < MR; ++t) {
      const int i = lane + 32 * t;
      col[u][t] = (j < c && i < m) ? A[(size_t)j * ld + i] : 0.f;
    }
  }
  int kw = 0, ku = 0;                  // k = ku * nw + kw: owner warp and register slot of column k
  for (int k = 0; k < K; ++k) {
    float* vb = vbuf + (k & 1) * (32 * MR);
    if (warp == kw) {
      const int uk = ku;
      float s2 = 0.f, xk = 0.f;
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        if (u != uk) continue;
#pragma unroll
        for (int t = 0; t < MR; ++t) {
          const int i = lane + 32 * t;
          const float x = col[u][t];
          if (i >= k && i < m) s2 = fmaf(x, x, s2);
          if (t == (k >> 5)) xk = x;
        }
      }
      s2 = warp_sum(s2);
      const float x0 = __shfl_sync(0xffffffffu, xk, k & 31);
      const float nrm = sqrtf(s2);
      const float alpha = (x0 >= 0.f) ? -nrm : nrm;
      const float tk = (nrm == 0.f) ? 0.f : 1.f / (nrm * (nrm + fabsf(x0)));
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        if (u != uk) continue;
#pragma unroll
        for (int t = 0; t < MR; ++t) {
          const int i = lane + 32 * t;
          float v = (i > k && i < m) ? col[u][t] : 0.f;
          if (i == k && nrm != 0.f) {
            v = x0 - alpha;
            col[u][t] = v;
          }
          vb[i] = (i == k && nrm == 0.f) ? 0.f : v;
        }
      }
      if (lane == 0) {
        tau[k] = tk;
        rdiag[k] = (nrm == 0.f) ? 0.f : alpha;
      }
    }
    if (++kw == nw) { kw = 0; ++ku; }
    __syncthreads();
    const float tk = tau[k];
    // a warp whose columns are all done skips the step
    if (tk != 0.f && warp + (JPW - 1) * nw > k) {
      float vr[MR];
#pragma unroll
      for (int t = 0; t < MR; ++t) vr[t] = vb[lane + 32 * t];
      float w[JPW];
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        w[u] = 0.f;
#pragma unroll
        for (int t = 0; t < MR; ++t) w[u] = fmaf(vr[t], col[u][t], w[u]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < JPW; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
#pragma unroll
      for (int u = 0; u < JPW; ++u) {
        const int j = warp + u * nw;
        if (j > k && j < c) {
          const float s = w[u] * tk;
#pragma unroll
          for (int t = 0; t < MR; ++t) col[u][t] = fmaf(-s, vr[t], col[u][t]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < JPW; ++u) {
    const int j = warp + u * nw;
    if (j >= c) continue;
#pragma unroll
    for (int t = 0; t < MR; ++t) {
      const int i = lane + 32 * t;
      if (i < m) A[(size_t)j * ld + i] = col[u][t];
    }
  }
  __syncthreads();
}

// Qm = H_0 ... H_{K-1} [I; 0] (signs fixed so that diag(R) > 0 when asked):
// warp w builds its own columns by applying every reflector, no barriers.
template <int MR, int JPW>
__device__ void hh_form_q_reg(const float* A, float* Qm, int ld, int m, int c, const float* tau, const float* rdiag,
                              bool fix_sign) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int K = min(m, c);
  float q[JPW][MR];
#pragma unroll
  for (int u = 0; u < JPW; ++u) {
    const int j = warp + u * nw;
#pragma unroll
    for (int t = 0; t < MR; ++t) q[u][t] = (lane + 32 * t == j) ? 1.f : 0.f;
  }
  const int jmax = min(c - 1, warp + (JPW - 1) * nw);
  for (int k = min(K - 1, jmax); k >= 0; --k) {
    const float tk = tau[k];
    if (tk == 0.f) continue;
    const float* v = A + (size_t)k * ld;
    float vr[MR];
#pragma unroll
    for (int t = 0; t < MR; ++t) {
      const int i = lane + 32 * t;
      vr[t] = (i >= k && i < m) ? v[i] : 0.f;
    }
    float w[JPW];
#pragma unroll
    for (int u = 0; u < JPW; ++u) {
      w[u] = 0.f;
#pragma unroll
      for (int t = 0; t < MR; ++t) w[u] = fmaf(vr[t], q[u][t], w[u]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < JPW; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
#pragma unroll
    for (int u = 0; u < JPW; ++u) {
      const int j = warp + u * nw;
      if (j >= k && j < c) {
        const float s = w[u] * tk;
#pragma unroll
        for (int t = 0; t < MR; ++t) q[u][t] = fmaf(-s, vr[t], q[u][t]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < JPW; ++u) {
    const int j = warp + u * nw;
    if (j >= c) continue;
    const float sg = (fix_sign && j < K && rdiag[j] < 0.f) ? -1.f : 1.f;
#pragma unroll
    for (int t = 0; t < MR; ++t) {
      const int i = lane + 32 * t;
      if (i < m) Qm[(size_t)j * ld + i] = sg * q[u][t];
    }
  }
  __syncthreads();
}

// Qm = H_0 ... H_{K-1} [I; 0] with one 8-lane group per column: group g (needs
// blockDim >= 8 c) holds column g of Q in registers (lane l: rows l + 8 t, m <= 8 RPL)
// and applies H_k for k = min(K-1, g) .. 0 (H_k leaves e_g alone for k > g); the
// groups never wait for one another, and each reflector costs one 3-level reduction.
template <int RPL>
__device__ void hh_form_q_g8(const float* A, float* Qm, int ld, int m, int c, const float* tau, const float* rdiag,
                             bool fix_sign) {
  const int g = threadIdx.x >> 3, l8 = threadIdx.x & 7;
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  const int K = min(m, c);
  if (g < c) {
    float q[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) q[t] = (l8 + 8 * t == g) ? 1.f : 0.f;
    for (int k = min(K - 1, g); k >= 0; --k) {
      const float tk = tau[k];
      if (tk == 0.f) continue;
      const float* vc = A + (size_t)k * ld;
      float v[RPL];
      float d = 0.f;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int i = l8 + 8 * t;
        v[t] = (i >= k && i < m) ? vc[i] : 0.f;
        d = fmaf(v[t], q[t], d);
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) d += __shfl_xor_sync(gm, d, o);
      const float sc = d * tk;
#pragma unroll
      for (int t = 0; t < RPL; ++t) q[t] = fmaf(-sc, v[t], q[t]);
    }
    const float sg = (fix_sign && g < K && rdiag[g] < 0.f) ? -1.f : 1.f;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = l8 + 8 * t;
      if (i < m) Qm[(size_t)g * ld + i] = sg * q[t];
    }
  }
  __syncthreads();
}

// Dispatch on the row count (m <= 512: registers; larger: shared memory).
template <int JPW, bool CT = true, bool TALL = false>
__device__ void qr_factor(float* A, int ld, int m, int c, float* tau, float* rdiag, float* vbuf) {
  if (CT) {
    if (m <= 32) hh_factor_reg_ct<1, JPW>(A, ld, m, c, tau, rdiag, vbuf);
    else if (m <= 64) hh_factor_reg_ct<2, JPW>(A, ld, m, c, tau, rdiag, vbuf);
    else if (m <= 128) hh_factor_reg_ct<4, JPW>(A, ld, m, c, tau, rdiag, vbuf);
    else if (m <= 256) hh_factor_reg_ct<8, JPW>(A, ld, m, c, tau, rdiag, vbuf);
    else if (m <= 512) hh_factor_reg_ct<16, JPW>(A, ld, m, c, tau, rdiag, vbuf);
    // tall stacks with at most one column per warp (small r + p): 48 rows per lane;
    // vbuf must then hold 2 x 32 x 48 floats
    else if (TALL && m <= 1536 && c <= (int)(blockDim.x >> 5)) hh_factor_reg_ct<48, 1>(A, ld, m, c, tau, rdiag, vbuf);
    else hh_factor(A, ld, m, c, tau, rdiag, nullptr);
    return;
  }
  if (m <= 32) hh_factor_reg<1, JPW>(A, ld, m, c, tau, rdiag, vbuf);
  else if (m <= 64) hh_factor_reg<2, JPW>(A, ld, m, c, tau, rdiag, vbuf);
  else if (m <= 128) hh_factor_reg<4, JPW>(A, ld, m, c, tau, rdiag, vbuf);
  else if (m <= 256) hh_factor_reg<8, JPW>(A, ld, m, c, tau, rdiag, vbuf);
  else if (m <= 512) hh_factor_reg<16, JPW>(A, ld, m, c, tau, rdiag, vbuf);
  else hh_factor(A, ld, m, c, tau, rdiag, nullptr);
}
template <int JPW, bool TALL = false>
__device__ void qr_form_q(const float* A, float* Qm, int ld, int m, int c, const float* tau, const float* rdiag,
                          bool fix_sign) {
  if ((int)blockDim.x >= 8 * c && m <= 128) {
    if (m <= 32) hh_form_q_g8<4>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
    else if (m <= 64) hh_form_q_g8<8>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
    else hh_form_q_g8<16>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  } else if (m <= 32) hh_form_q_reg<1, JPW>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  else if (m <= 64) hh_form_q_reg<2, JPW>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  else if (m <= 128) hh_form_q_reg<4, JPW>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  else if (m <= 256) hh_form_q_reg<8, JPW>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  else if (m <= 512) hh_form_q_reg<16, JPW>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  else if (TALL && m <= 1536 && c <= (int)(blockDim.x >> 5)) hh_form_q_reg<48, 1>(A, Qm, ld, m, c, tau, rdiag, fix_sign);
  else hh_form_q(A, Qm, ld, m, c, tau, rdiag, fix_sign);
}



// S5 level 1: QR of one row block of Z (sum of sketch partials).  Single-block
// problems finish here (signs fixed); tall problems also write R_b.
// Dynamic smem: A[ld*c] | Qm[ld*c] | tau[CMAX] | rdiag[CMAX] | vbuf[1024]
constexpr int QR_THREADS = 512;
constexpr int QR_JPW = CMAX / (QR_THREADS / 32);
__global__ void __launch_bounds__(QR_THREADS) k_qr1(const RFProb* __restrict__ P,
                                                    const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int b = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c;
  const int64_t row0 = (int64_t)b * q.rbrows;
  const int m = (int)min((int64_t)q.rbrows, q.nS - row0);
  const int ld = odd_ld(m);
  float* A = reinterpret_cast<float*>(smem_raw);
  float* Qm = A + (size_t)ld * c;
  float* tau = Qm + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* vbuf = rdiag + CMAX;
#pragma unroll 2
  for (int e = threadIdx.x; e < m * c; e += QR_THREADS) {
    const int i = e / c, j = e % c;
    A[(size_t)j * ld + i] = q.Zp[(row0 + i) * c + j];
  }
  __syncthreads();
  qr_factor<QR_JPW>(A, ld, m, c, tau, rdiag, vbuf);
  const bool single = (q.nrb == 1);
  if (!single) {  // R_b (c x c, zero below the diagonal and beyond row K)
    float* Rb = q.Rb + (size_t)b * c * c;
    for (int e = threadIdx.x; e < c * c; e += QR_THREADS) {
      const int k = e / c, j = e % c;
      float v = 0.f;
      if (k < m && j >= k) v = (j == k) ? rdiag[k] : A[(size_t)j * ld + k];
      Rb[e] = v;
    }
  }
  qr_form_q<QR_JPW>(A, Qm, ld, m, c, tau, rdiag, single);
  for (int e = threadIdx.x; e < m * c; e += QR_THREADS) {
    const int i = e / c, j = e % c;
    q.Q[(row0 + i) * c + j] = Qm[(size_t)j * ld + i];
  }
}

// TSQR tree of a tall Z: level l stacks the R factors entering it (lev_n[l] of
// them, c x c each; level 0 takes the row blocks' R_b) in groups of `fan`.  Level
// l's R inputs and Q member slices:
__device__ __forceinline__ size_t ts_level_off(const RFProb& q, int l) {
  size_t o = 0;
  for (int j = 1; j < l; ++j) o += (size_t)q.lev_n[j];
  return o * q.c * q.c;
}
__device__ __forceinline__ const float* ts_rin(const RFProb& q, int l) {
  return l == 0 ? q.Rb : q.tsR + ts_level_off(q, l);
}
__device__ __forceinline__ float* ts_q(const RFProb& q, int l) { return l == 0 ? q.Q2 : q.tsQ + ts_level_off(q, l); }

// S5, level `lev` of the TSQR tree: QR of one group's stacked R factors, (cnt c) x c.
// Below the top its R goes to the next level's inputs (signs as they come, matching
// its Q); at the top Q has diag(R) > 0, which fixes the overall factor.
__global__ void __launch_bounds__(QR_THREADS) k_qr2(const RFProb* __restrict__ P,
                                             const int64_t* __restrict__ pre, int np, int lev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int g = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c;
  const int b0 = g * q.fan;
  const int cnt = min(q.fan, q.lev_n[lev] - b0);
  const int m = cnt * c;
  const int ld = odd_ld(m);
  const bool top = (lev == q.nlev - 1);
  float* A = reinterpret_cast<float*>(smem_raw);
  float* Qm = A + (size_t)ld * c;
  float* tau = Qm + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* red = rdiag + CMAX;
  const float* Rin = ts_rin(q, lev) + (size_t)b0 * c * c;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    A[(size_t)j * ld + i] = Rin[e];
  }
  __syncthreads();
  qr_factor<QR_JPW, true, true>(A, ld, m, c, tau, rdiag, red + 32);
  if (!top) {
    float* Rout = const_cast<float*>(ts_rin(q, lev + 1)) + (size_t)g * c * c;
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
      const int k = e / c, j = e % c;
      float v = 0.f;
      if (j >= k) v = (j == k) ? rdiag[k] : A[(size_t)j * ld + k];
      Rout[e] = v;
    }
  }
  qr_form_q<QR_JPW, true>(A, Qm, ld, m, c, tau, rdiag, top);
  float* Qout = ts_q(q, lev) + (size_t)b0 * c * c;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    Qout[e] = Qm[(size_t)j * ld + i];
  }
}

// S5, combine pass t of the TSQR tree (top-down): at level l = nlev - 2 - t, member
// b's Q slice times its group's slice one level up (already combined), in place,
// so that level 0 ends with the slices of the whole tree's Q.
// Static smem: two c x c slices.
__global__ void __launch_bounds__(256) k_qrc(const RFProb* __restrict__ P, const int64_t* __restrict__ pre,
                                             int np, int t) {
  __shared__ float Sb[CMAX * CMAX], Sg[CMAX * CMAX];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int b = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c;
  const int l = q.nlev - 2 - t;
  float* Qb = ts_q(q, l) + (size_t)b * c * c;
  const float* Qg = ts_q(q, l + 1) + (size_t)(b / q.fan) * c * c;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    Sb[e] = Qb[e];
    Sg[e] = Qg[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    float acc = 0.f;
    for (int k = 0; k < c; ++k) acc = fmaf(Sb[i * c + k], Sg[k * c + j], acc);
    Qb[e] = acc;
  }
}

// S5 level 3 (tall Z): Q[block b] = Q_b * Q2[b c : b c + c, :].
// Dynamic smem: Qb[rbrows*c] | Q2b[c*c]
__global__ void __launch_bounds__(256) k_qr3(const RFProb* __restrict__ P,
                                             const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int b = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c;
  const int64_t row0 = (int64_t)b * q.rbrows;
  const int m = (int)min((int64_t)q.rbrows, q.nS - row0);
  float* Qb = reinterpret_cast<float*>(smem_raw);
  float* Q2b = Qb + (size_t)q.rbrows * c;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) Qb[e] = q.Q[row0 * c + e];
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) Q2b[e] = q.Q2[(size_t)b * c * c + e];
  __syncthreads();
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    float acc = 0.f;
    for (int t = 0; t < c; ++t) acc = fmaf(Qb[i * c + t], Q2b[t * c + j], acc);
    q.Q[(row0 + i) * c + j] = acc;
  }
}

// ------------------------------------------------------------------ S6: B^T = Y^T Q
// Partial over rows [ib*BT_IB, ...) for samples [sc*scrows, ...): 4x4 register
// micro-tiles over (sample, column).
// Dynamic smem: Ys[32][BT_LDY] (row ii, sample jj) | Qs[32][CMAX]
constexpr int BT_LDY = BT_SC + 4;
__global__ void __launch_bounds__(256) k_bt_partial(const RFProb* __restrict__ P,
                                                    const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);
  float* Qs = Ys + 32 * BT_LDY;
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int64_t local = (int64_t)blockIdx.x - pre[p];
  const int sc = (int)(local / q.nbi), ib = (int)(local % q.nbi);
  const int c = q.c, cp = (c + 3) & ~3;
  const int64_t j0 = (int64_t)sc * q.scrows;
  const int mj = (int)min((int64_t)q.scrows, q.s - j0);
  const int64_t iA = (int64_t)ib * BT_IB, iB = min(q.nS, iA + BT_IB);
  const int ntile = (BT_SC / 4) * (cp / 4);
  constexpr int TPT = (BT_SC / 4) * (CMAX / 4) / 256;   // 4x4 tiles per thread (at most)
  float acc[TPT][4][4];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[u][a][b] = 0.f;
  for (int64_t it = iA; it < iB; it += 32) {
    const int mi = (int)min((int64_t)32, iB - it);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * BT_SC; e += 256) {
      const int jj = e / 32, ii = e % 32;
      Ys[ii * BT_LDY + jj] = (jj < mj && ii < mi) ? q.Yt[(j0 + jj) * q.nS + it + ii] : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * cp; e += 256) {
      const int ii = e / cp, cc = e % cp;
      Qs[ii * CMAX + cc] = (ii < mi && cc < c) ? q.Q[(it + ii) * c + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = threadIdx.x + 256 * u;
      if (t < ntile) {
        const int jg = t % (BT_SC / 4), cg = t / (BT_SC / 4);
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
          const float4 y = *reinterpret_cast<const float4*>(Ys + ii * BT_LDY + jg * 4);
          const float4 o = *reinterpret_cast<const float4*>(Qs + ii * CMAX + cg * 4);
          const float ya[4] = {y.x, y.y, y.z, y.w};
          const float ob[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[u][a][b] = fmaf(ya[a], ob[b], acc[u][a][b]);
        }
      }
    }
  }
  float* out = q.Bp + ((size_t)ib * q.s + j0) * c;
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + 256 * u;
    if (t < ntile) {
      const int jg = t % (BT_SC / 4), cg = t / (BT_SC / 4);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int jj = jg * 4 + a;
        if (jj >= mj) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int cc = cg * 4 + b;
          if (cc < c) out[(size_t)jj * c + cc] = acc[u][a][b];
        }
      }
    }
  }
}

// S6 (rows of Y fit one block): B^T chunk = Y_chunk^T Q accumulated over all
// rows, kept in shared memory and factorised right away -> R_chunk.
// Dynamic smem: Ys[32][BT_LDY] | Qs[32][CMAX] | A[ld*c] | tau | rdiag
__global__ void __launch_bounds__(QR_THREADS) k_bt_fused(const RFProb* __restrict__ P,
                                                  const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);
  float* Qs = Ys + 32 * BT_LDY;
  float* A = Qs + 32 * CMAX;
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int sc = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c, cp = (c + 3) & ~3;
  const int64_t j0 = (int64_t)sc * q.scrows;
  const int mj = (int)min((int64_t)q.scrows, q.s - j0);
  const int ld = odd_ld(mj);
  float* tau = A + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* vbuf = rdiag + CMAX;
  const int ntile = (BT_SC / 4) * (cp / 4);
  constexpr int TPT = (BT_SC / 4) * (CMAX / 4) / QR_THREADS;   // 4x4 tiles per thread (at most)
  float acc[TPT][4][4];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[u][a][b] = 0.f;
  for (int64_t it = 0; it < q.nS; it += 32) {
    const int mi = (int)min((int64_t)32, q.nS - it);
    __syncthreads();
#pragma unroll
    for (int e = threadIdx.x; e < 32 * BT_SC; e += QR_THREADS) {
      const int jj = e / 32, ii = e % 32;
      Ys[ii * BT_LDY + jj] = (jj < mj && ii < mi) ? q.Yt[(j0 + jj) * q.nS + it + ii] : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * cp; e += QR_THREADS) {
      const int ii = e / cp, cc = e % cp;
      Qs[ii * CMAX + cc] = (ii < mi && cc < c) ? q.Q[(it + ii) * c + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = threadIdx.x + QR_THREADS * u;
      if (t < ntile) {
        const int jg = t % (BT_SC / 4), cg = t / (BT_SC / 4);
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
          const float4 y = *reinterpret_cast<const float4*>(Ys + ii * BT_LDY + jg * 4);
          const float4 o = *reinterpret_cast<const float4*>(Qs + ii * CMAX + cg * 4);
          const float ya[4] = {y.x, y.y, y.z, y.w};
          const float ob[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[u][a][b] = fmaf(ya[a], ob[b], acc[u][a][b]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + QR_THREADS * u;
    if (t < ntile) {
      const int jg = t % (BT_SC / 4), cg = t / (BT_SC / 4);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int jj = jg * 4 + a;
        if (jj >= mj) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int cc = cg * 4 + b;
          if (cc < c) A[(size_t)cc * ld + jj] = acc[u][a][b];
        }
      }
    }
  }
  __syncthreads();
  qr_factor<QR_JPW, false>(A, ld, mj, c, tau, rdiag, vbuf);
  float* Rc = q.Rc + (size_t)sc * c * c;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int k = e / c, j = e % c;
    float v = 0.f;
    if (k < mj && j >= k) v = (j == k) ? rdiag[k] : A[(size_t)j * ld + k];
    Rc[e] = v;
  }
}

// S6: QR of one sample chunk of B^T (sum of the row-block partials) -> R_chunk.
// Dynamic smem: A[ld*c] | tau | rdiag | red
__global__ void __launch_bounds__(QR_THREADS) k_bt_qr(const RFProb* __restrict__ P,
                                               const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int sc = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c;
  const int64_t j0 = (int64_t)sc * q.scrows;
  const int m = (int)min((int64_t)q.scrows, q.s - j0);
  const int ld = odd_ld(m);
  float* A = reinterpret_cast<float*>(smem_raw);
  float* tau = A + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* red = rdiag + CMAX;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    float acc = 0.f;
    for (int ib = 0; ib < q.nbi; ++ib) acc += q.Bp[((size_t)ib * q.s + j0 + i) * c + j];
    A[(size_t)j * ld + i] = acc;
  }
  __syncthreads();
  qr_factor<QR_JPW>(A, ld, m, c, tau, rdiag, red + 32);
  float* Rc = q.Rc + (size_t)sc * c * c;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int k = e / c, j = e % c;
    float v = 0.f;
    if (k < m && j >= k) v = (j == k) ? rdiag[k] : A[(size_t)j * ld + k];
    Rc[e] = v;
  }
}

// S6, many sample chunks: level `lev` of an R tree over the chunk factors R_c.  A
// group of up to wfan stacked c x c factors is replaced by the R of its QR.  Only R
// is kept: the W-step needs the left singular vectors of R^T, which an orthogonal
// factor applied to R from the left leaves unchanged.
// Dynamic smem: A[ld*c] | tau | rdiag | red | vbuf[3072]
__device__ __forceinline__ size_t wt_off(const RFProb& q, int l) {
  size_t o = 0;
  for (int j = 1; j < l; ++j) o += (size_t)q.wn[j];
  return o * q.c * q.c;
}
__global__ void __launch_bounds__(QR_THREADS) k_wtree(const RFProb* __restrict__ P,
                                               const int64_t* __restrict__ pre, int np, int lev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int g = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c;
  const int b0 = g * q.wfan;
  const int cnt = min(q.wfan, q.wn[lev] - b0);
  const int m = cnt * c;
  const int ld = odd_ld(m);
  float* A = reinterpret_cast<float*>(smem_raw);
  float* tau = A + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* red = rdiag + CMAX;
  const float* Rin = (lev == 0 ? q.Rc : q.wsR + wt_off(q, lev)) + (size_t)b0 * c * c;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    A[(size_t)j * ld + i] = Rin[e];
  }
  __syncthreads();
  qr_factor<QR_JPW, true, true>(A, ld, m, c, tau, rdiag, red + 32);
  float* Rout = q.wsR + wt_off(q, lev + 1) + (size_t)g * c * c;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int k = e / c, j = e % c;
    float v = 0.f;
    if (j >= k) v = (j == k) ? rdiag[k] : A[(size_t)j * ld + k];
    Rout[e] = v;
  }
}

// S6: R of the stacked chunk factors, then one-sided Jacobi (Hestenes) on the
// columns of R^T: R^T V = W Sigma, W = left singular vectors of B.  Columns
// are processed in round-robin order, one 16-lane group per pair, until a sweep
// makes no rotation or leaves every pair below sqrt(tol) / 2 before rotation (at
// most WS_MAX_SWEEPS, else ST_NUMERIC).  W is stored sorted by descending sigma.
// Dynamic smem: A[ld*c] | tau | rdiag | red | AT[CMAX*WS_LDT] | sig[CMAX] | flag[2], dmax[2] | vbuf
static_assert(QR_THREADS / 16 >= CMAX / 2, "one 16-lane group per Jacobi pair");
static_assert(WS_LDT >= CMAX && WS_LDT % 32 == 16, "Jacobi column stride");
__global__ void __launch_bounds__(QR_THREADS) k_wsvd(const RFProb* __restrict__ P,
                                               const int64_t* __restrict__ pre, int np,
                                               int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int c = q.c;
  const int m = q.nrw * c;
  const int ld = odd_ld(m);
  float* A = reinterpret_cast<float*>(smem_raw);
  float* tau = A + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* red = rdiag + CMAX;
  float* AT = red + 32;                  // column q of R^T at AT[q*WS_LDT + i], zero-padded to CMAX rows
  float* sig = AT + CMAX * WS_LDT;
  int* flag = reinterpret_cast<int*>(sig + CMAX);
  constexpr int LDT = WS_LDT;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    A[(size_t)j * ld + i] = q.Rw[e];
  }
  if (threadIdx.x < q.r) q.keys[threadIdx.x] = 0ull;
  if (threadIdx.x < 2) flag[threadIdx.x] = 0;
  __syncthreads();
  qr_factor<QR_JPW>(A, ld, m, c, tau, rdiag, sig + CMAX + 8);
  // AT[qc][i] = R[qc][i]  (column qc of R^T is row qc of R); rows c..CMAX-1 stay zero so
  // that every pair below runs the same fixed-length, fully unrolled loop.
  for (int e = threadIdx.x; e < CMAX * CMAX; e += blockDim.x) {
    const int qc = e / CMAX, i = e % CMAX;
    float v = 0.f;
    if (qc < c && qc < m && i < c && i >= qc) v = (i == qc) ? rdiag[qc] : A[(size_t)i * ld + qc];
    AT[qc * LDT + i] = v;
  }
  __syncthreads();
  jacobi_columns(AT, c, flag, status);
  store_sorted(q, AT, c, sig, status);
}

// ------------------------------------------------------------------ U = Q W(:, :r), sign rule
__device__ __forceinline__ float qw_entry(const float* __restrict__ Qrow, const float* Ws, int c,
                                          int col, int ldw) {
  float acc = 0.f;
  for (int t = 0; t < c; ++t) acc = fmaf(Qrow[t], Ws[t * ldw + col], acc);
  return acc;
}

// Dynamic smem: Ws[CMAX*CMAX] | Qs[QW_TI*CMAX] | keys[CMAX] (u64)
__global__ void __launch_bounds__(256) k_qw(const RFProb* __restrict__ P,
                                            const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ws = reinterpret_cast<float*>(smem_raw);
  float* Qs = Ws + CMAX * CMAX;
  unsigned long long* kb = reinterpret_cast<unsigned long long*>(Qs + QW_TI * CMAX);
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int64_t row0 = ((int64_t)blockIdx.x - pre[p]) * QW_TI;
  const int m = (int)min((int64_t)QW_TI, q.nS - row0);
  const int c = q.c, r = q.r;
  for (int e = threadIdx.x; e < c * r; e += blockDim.x) Ws[(e / r) * CMAX + e % r] = q.W[(e / r) * c + e % r];
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) Qs[e] = q.Q[row0 * c + e];
  if (threadIdx.x < r) kb[threadIdx.x] = 0ull;
  __syncthreads();
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int i = e / r, col = e % r;
    const float u = qw_entry(Qs + i * c, Ws, c, col, CMAX);
    q.U[(row0 + i) * r + col] = u;
    atomicMax(&kb[col], sign_key(u, row0 + i));
  }
  __syncthreads();
  if (threadIdx.x < r) atomicMax(&q.keys[threadIdx.x], kb[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_flip(const RFProb* __restrict__ P,
                                              const int64_t* __restrict__ pre, int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ws = reinterpret_cast<float*>(smem_raw);
  float* sg = Ws + CMAX * CMAX;
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int64_t row0 = ((int64_t)blockIdx.x - pre[p]) * QW_TI;
  const int m = (int)min((int64_t)QW_TI, q.nS - row0);
  const int c = q.c, r = q.r;
  for (int e = threadIdx.x; e < c * r; e += blockDim.x) Ws[(e / r) * CMAX + e % r] = q.W[(e / r) * c + e % r];
  __syncthreads();
  if (threadIdx.x < r) {
    const int col = threadIdx.x;
    const unsigned long long key = q.keys[col];
    const int64_t rstar = (int64_t)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
    const float u = qw_entry(q.Q + rstar * c, Ws, c, col, CMAX);
    sg[col] = (u < 0.f) ? -1.f : 1.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int col = e % r;
    if (sg[col] < 0.f) q.U[row0 * r + e] = -q.U[row0 * r + e];
  }
  if (row0 == 0)
    for (int e = threadIdx.x; e < c * r; e += blockDim.x) q.Wsg[e] = sg[e % r] * Ws[(e / r) * CMAX + e % r];
}

// U = Q W(:, :r) and the sign rule in one CTA per problem with n_S <= QWF_MAX rows.
// Dynamic smem: Ws[CMAX*CMAX] | Qt[CMAX*QWF_MAX] | Us[QWF_MAX*CMAX] | sg[CMAX]
__global__ void __launch_bounds__(512) k_qwf(const RFProb* __restrict__ P, const int64_t* __restrict__ pre,
                                             int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  qw_sign(P[p], reinterpret_cast<float*>(smem_raw));
}

// ================================================================== Cholesky form (qr = 2)
// For problems whose unfolding has at most QWF_MAX rows, S5 and the factorisation
// in S6 run as Cholesky factorisations of Gram matrices instead of Householder QRs:
//   S5: Z = Q R by CholeskyQR2 with a double-float first Gram (the mixed-precision
//       CholeskyQR2 of Yamazaki, Tomov and Dongarra, 2015): G = Z^T Z summed in
//       double-float (two float32 words, about 2^-48 relative), rounded to float32,
//       G = R1^T R1, Q1 = Z R1^-1 by substitution; then a float32 pass on Q1 (its Gram
//       is close to I) restores orthogonality to float32 rounding.
//   S6: B^T = Y^T Q per chunk of samples with its Gram C_chunk = B_chunk B_chunk^T in
//       double-float; the chunks summed in a fixed order, rounded to float32, and
//       C = R^T R: R is the R factor of B^T (B B^T = R^T R) up to row signs, so the
//       one-sided Jacobi SVD of R^T gives the left singular vectors W of B as before;
//       then U = Q W(:, :r) and the sign rule in the same CTA.
// Each stage is one CTA per problem (S5, W-step) or per sample chunk (B-step Gram);
// GB300's float64 rate is ~1/64 of float32, so the double-float sums run on the
// float32 pipes.

// G[i*ldg + j] (j >= i) = sum_{t < m} A[t*lda + i] A[t*lda + j], in double-float (dd) or
// float32, rounded to float32.  One thread per entry with four independent partial
// sums (rows t = 4 u + v) combined at the end; consecutive threads take consecutive
// j, so the column reads of a warp are conflict-free for odd lda.
__device__ void gram_upper(const float* A, int lda, int m, int c, float* G, int ldg, bool dd) {
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    if (j < i) continue;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    int t = 0;
    if (dd) {
      for (; t + 3 < m; t += 4) {
#pragma unroll
        for (int v = 0; v < 4; ++v) df_acc(hi[v], lo[v], A[(t + v) * lda + i], A[(t + v) * lda + j]);
      }
      for (; t < m; ++t) df_acc(hi[0], lo[0], A[t * lda + i], A[t * lda + j]);
      df_add(hi[0], lo[0], hi[1], lo[1]);
      df_add(hi[2], lo[2], hi[3], lo[3]);
      df_add(hi[0], lo[0], hi[2], lo[2]);
    } else {
      for (; t + 3 < m; t += 4) {
#pragma unroll
        for (int v = 0; v < 4; ++v) hi[v] = fmaf(A[(t + v) * lda + i], A[(t + v) * lda + j], hi[v]);
      }
      for (; t < m; ++t) hi[0] = fmaf(A[t * lda + i], A[t * lda + j], hi[0]);
      hi[0] = (hi[0] + hi[1]) + (hi[2] + hi[3]);
    }
    G[i * ldg + j] = hi[0] + lo[0];
  }
}

// Cholesky G = R^T R of the upper triangle of G (c x c), R upper triangular into R
// (zero below the diagonal); G is overwritten.  One barrier per step.  The upper
// triangle's entries (i, j) are listed once in ij (shared, c (c + 1) / 2 shorts
// pairs) by decreasing i, so the trailing entries of step k (i > k) are the first
// (c - 1 - k)(c - k) / 2 of the list and spread evenly over the threads; every
// thread reads pivot row k.  A pivot at or below thr (a column dependent on the
// earlier ones to rounding) gets R_kk = rzero and a zero row, and no trailing update;
// *nzero counts them (shared).
__device__ void chol_upper(float* G, int ldg, int c, float* R, int ldr, float thr, float rzero, int* nzero,
                           uint32_t* ij) {
  for (int e = threadIdx.x; e < c * ldr; e += blockDim.x) R[e] = 0.f;
  for (int i = (int)threadIdx.x; i < c; i += blockDim.x) {   // row i after the (c-1-i)(c-i)/2 entries of rows > i
    const int o = (c - 1 - i) * (c - i) / 2;
    for (int j = i; j < c; ++j) ij[o + (j - i)] = ((uint32_t)i << 16) | (uint32_t)j;
  }
  __syncthreads();
  for (int k = 0; k < c; ++k) {
    const float d = G[k * ldg + k];
    const bool zero = !(d > thr);
    const float rk = zero ? rzero : sqrtf(d);
    const float ik = zero ? 0.f : __frcp_rn(rk);
    for (int j = k + (int)threadIdx.x; j < c; j += blockDim.x) R[k * ldr + j] = (j == k) ? rk : G[k * ldg + j] * ik;
    if (!zero) {
      const int nt = (c - 1 - k) * (c - k) / 2;
      for (int e = threadIdx.x; e < nt; e += blockDim.x) {
        const uint32_t w = ij[e];
        const int i = (int)(w >> 16), j = (int)(w & 0xffffu);
        G[i * ldg + j] = fmaf(-(G[k * ldg + i] * ik), G[k * ldg + j] * ik, G[i * ldg + j]);
      }
    }
    if (zero && threadIdx.x == 0) atomicAdd(nzero, 1);
    __syncthreads();
  }
}

// A <- A R^-1 for R upper triangular (rinv[j] = 1 / R_jj): row i of the result solves
// x R = a_i by forward substitution.  Four lanes per row split each partial sum over
// k < j (k = 4 u + lane4) and combine it with two shuffles; the row's lanes then all
// hold x_j.  m rows in groups of blockDim / 4.
__device__ void trsm_rows(float* A, int lda, int m, int c, const float* R, int ldr, const float* rinv) {
  const int l4 = threadIdx.x & 3;
  const int rows_per_pass = (int)(blockDim.x >> 2);
  for (int i0 = 0; i0 < m; i0 += rows_per_pass) {
    const int i = i0 + (int)(threadIdx.x >> 2);
    const bool on = i < m;
    float* a = A + (on ? i : 0) * lda;
    for (int j = 0; j < c; ++j) {
      float s = 0.f;
      if (on)
        for (int k = l4; k < j; k += 4) s = fmaf(a[k], R[k * ldr + j], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (on && l4 == 0) a[j] = (a[j] - s) * rinv[j];
      __syncwarp();
    }
  }
}

constexpr int QZ_LD = CMAX + 1;   // odd row stride of Z / Q in shared memory
constexpr int GR_LD = CMAX + 1;   // row stride of the Gram and R matrices

// S5, Cholesky form: Q of Z (n_S <= QWF_MAX rows) by mixed-precision CholeskyQR2, or
// (q.zshift) by shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Zhang, Yamamoto,
// SIAM J. Sci. Comput. 2020): the first pass factors Z^T Z + s I with
// s = 11 (m c + c (c + 1)) u ||Z||_F^2, u = 2^-24 the unit roundoff of the float32
// Cholesky (||Z||_F^2 >= ||Z||_2^2), which keeps every pivot positive for cond(Z) up to
// about 1/u and leaves Z R^-1 with a condition number CholeskyQR2 then handles; the
// factor R of Z is the product of the three, Q = Z R^-1 the same Q.  A zero pivot
// (Z numerically rank-deficient) falls back to the Householder QR of the same Z in the
// same CTA.
// Dynamic smem: max(A[QWF_MAX*QZ_LD] | G[CMAX*GR_LD] | R[CMAX*GR_LD] | rinv[CMAX] | nzero,
//                   the Householder QR's A | Qm | tau | rdiag | vbuf)
__global__ void __launch_bounds__(QR_THREADS) k_qz(const RFProb* __restrict__ P, const int64_t* __restrict__ pre,
                                                   int np, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int c = q.c, m = (int)q.nS;
  const int lda = c | 1;
  float* A = reinterpret_cast<float*>(smem_raw);
  float* G = A + QWF_MAX * QZ_LD;
  float* R = G + CMAX * GR_LD;
  float* rinv = R + CMAX * GR_LD;
  int* nzero = reinterpret_cast<int*>(rinv + CMAX);
  uint32_t* ij = reinterpret_cast<uint32_t*>(nzero + 4);
  if (threadIdx.x == 0) *nzero = 0;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) A[(e / c) * lda + e % c] = q.Zp[e];
  __syncthreads();
  const int npass = q.zshift ? 3 : 2;
  for (int pass = 0; pass < npass; ++pass) {
    gram_upper(A, lda, m, c, G, GR_LD, pass == 0);
    __syncthreads();
    float dmax = 0.f, tr = 0.f;
    for (int k = 0; k < c; ++k) {
      dmax = fmaxf(dmax, G[k * GR_LD + k]);
      tr += G[k * GR_LD + k];
    }
    if (!(dmax < INFINITY)) {            // non-finite sketch
      if (threadIdx.x == 0) set_status(status, ST_NUMERIC);
      dmax = 0.f;
      tr = 0.f;
    }
    if (q.zshift && pass == 0) {
      const float shift = 11.f * (float)(m * c + c * (c + 1)) * 0x1p-24f * tr;
      __syncthreads();
      for (int k = threadIdx.x; k < c; k += blockDim.x) G[k * GR_LD + k] += shift;
      __syncthreads();
    }
    chol_upper(G, GR_LD, c, R, GR_LD, dmax * (float)(c * 3.6e-15), 0.f, nzero, ij);
    if (*nzero) break;
    for (int j = threadIdx.x; j < c; j += blockDim.x) rinv[j] = 1.f / R[j * GR_LD + j];
    __syncthreads();
    trsm_rows(A, lda, m, c, R, GR_LD, rinv);
    __syncthreads();
  }
  if (*nzero == 0) {
    for (int e = threadIdx.x; e < m * c; e += blockDim.x) q.Q[e] = A[(e / c) * lda + e % c];
    return;
  }
  // Householder fallback (as k_qr1 for a single row block)
  __syncthreads();
  const int ld = odd_ld(m);
  float* H = reinterpret_cast<float*>(smem_raw);
  float* Qm = H + (size_t)ld * c;
  float* tau = Qm + (size_t)ld * c;
  float* rdiag = tau + CMAX;
  float* vbuf = rdiag + CMAX;
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) H[(size_t)(e % c) * ld + e / c] = q.Zp[e];
  __syncthreads();
  qr_factor<QR_JPW>(H, ld, m, c, tau, rdiag, vbuf);
  qr_form_q<QR_JPW>(H, Qm, ld, m, c, tau, rdiag, true);
  for (int e = threadIdx.x; e < m * c; e += blockDim.x) q.Q[e] = Qm[(size_t)(e % c) * ld + e / c];
}

// S6, Cholesky form, per sample chunk sc: B^T_chunk = Y_chunk^T Q (BG_SC x c, in shared
// memory) and its Gram C_chunk = B_chunk B_chunk^T by compensated sums of the rounded
// products, written as sum / correction words to Cp[sc][i][j] (upper triangle).
// Dynamic smem: Ys[32][BG_LDY] | Qs[32][CMAX] | Bs[BG_SC][CMAX | 1]
constexpr int BG_LDY = BG_SC + 4;
__global__ void __launch_bounds__(256) k_btg(const RFProb* __restrict__ P, const int64_t* __restrict__ pre,
                                             int np) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);
  float* Qs = Ys + 32 * BG_LDY;
  float* Bs = Qs + 32 * CMAX;
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int sc = (int)((int64_t)blockIdx.x - pre[p]);
  const int c = q.c, cp = (c + 3) & ~3, ldb = c | 1;
  const int64_t j0 = (int64_t)sc * BG_SC;
  const int mj = (int)min((int64_t)BG_SC, q.s - j0);
  const int ntile = (BG_SC / 4) * (cp / 4);
  constexpr int TPT = (BG_SC / 4) * (CMAX / 4) / 256;
  float acc[TPT][4][4];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[u][a][b] = 0.f;
  for (int64_t it = 0; it < q.nS; it += 32) {
    const int mi = (int)min((int64_t)32, q.nS - it);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * BG_SC; e += 256) {
      const int jj = e / 32, ii = e % 32;
      Ys[ii * BG_LDY + jj] = (jj < mj && ii < mi) ? q.Yt[(j0 + jj) * q.nS + it + ii] : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * cp; e += 256) {
      const int ii = e / cp, cc = e % cp;
      Qs[ii * CMAX + cc] = (ii < mi && cc < c) ? q.Q[(it + ii) * c + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = threadIdx.x + 256 * u;
      if (t < ntile) {
        const int jg = t % (BG_SC / 4), cg = t / (BG_SC / 4);
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
          const float4 y = *reinterpret_cast<const float4*>(Ys + ii * BG_LDY + jg * 4);
          const float4 o = *reinterpret_cast<const float4*>(Qs + ii * CMAX + cg * 4);
          const float ya[4] = {y.x, y.y, y.z, y.w};
          const float ob[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[u][a][b] = fmaf(ya[a], ob[b], acc[u][a][b]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + 256 * u;
    if (t < ntile) {
      const int jg = t % (BG_SC / 4), cg = t / (BG_SC / 4);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int cc = cg * 4 + b;
          if (cc < c) Bs[(jg * 4 + a) * ldb + cc] = acc[u][a][b];   // rows >= mj hold zeros
        }
    }
  }
  __syncthreads();
  float* out = q.Cp + (size_t)sc * c * c * 2;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    if (j < i) continue;
    float s0 = 0.f, k0 = 0.f, s1 = 0.f, k1 = 0.f;   // two independent sums (even, odd t)
    int t = 0;
#pragma unroll 2
    for (; t + 1 < mj; t += 2) {
      kahan_add(s0, k0, __fmul_rn(Bs[t * ldb + i], Bs[t * ldb + j]));
      kahan_add(s1, k1, __fmul_rn(Bs[(t + 1) * ldb + i], Bs[(t + 1) * ldb + j]));
    }
    if (t < mj) kahan_add(s0, k0, __fmul_rn(Bs[t * ldb + i], Bs[t * ldb + j]));
    float hi = s0, lo = -k0;
    df_add(hi, lo, s1, -k1);
    out[2 * e] = hi;
    out[2 * e + 1] = lo;
  }
}

// S6, Cholesky form, one CTA per problem: C = sum of the chunk Grams (double-float,
// chunk order), C = R^T R, one-sided Jacobi on the columns of R^T, W sorted, then
// U = Q W(:, :r) with the sign rule.
// Dynamic smem: max(G[CMAX*GR_LD] | R[CMAX*GR_LD] | AT[CMAX*WS_LDT] | sig | flag[4] | nzero,
//                   the U = Q W stage: CMAX*CMAX + 2*QWF_MAX*CMAX + CMAX floats)
__global__ void __launch_bounds__(QR_THREADS) k_wsvd2(const RFProb* __restrict__ P,
                                                      const int64_t* __restrict__ pre, int np, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = find_prob(pre, np, blockIdx.x);
  const RFProb& q = P[p];
  const int c = q.c;
  float* Qt = reinterpret_cast<float*>(smem_raw);       // Q^T for U = Q W, staged first
  float* Ws = Qt + CMAX * QWF_MAX;
  float* sg = Ws + CMAX * CMAX;
  float* G = sg + CMAX;                                   // then G | R | AT | sig | flags,
  float* R = G + CMAX * GR_LD;                            // reused as Us by U = Q W
  float* AT = R + CMAX * GR_LD;
  float* sig = AT + CMAX * WS_LDT;
  int* flag = reinterpret_cast<int*>(sig + CMAX);
  int* nzero = flag + 4;
  uint32_t* ij = reinterpret_cast<uint32_t*>(flag + 8);
  if (threadIdx.x < 4) flag[threadIdx.x] = 0;
  if (threadIdx.x == 0) *nzero = 0;
  qw_stage_q(q, Qt);
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    if (j < i) continue;
    // chunk partials loaded eight at a time (independent loads in flight), added in order
    float hi = 0.f, lo = 0.f;
    for (int s0 = 0; s0 < q.nbg; s0 += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (s0 + u < q.nbg) ? __ldcg(reinterpret_cast<const float2*>(q.Cp + ((size_t)(s0 + u) * c * c + e) * 2))
                                : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) df_add(hi, lo, v[u].x, v[u].y);
    }
    G[i * GR_LD + j] = hi + lo;
  }
  __syncthreads();
  float dmax = 0.f;
  for (int k = 0; k < c; ++k) dmax = fmaxf(dmax, G[k * GR_LD + k]);
  if (!(dmax < INFINITY)) {
    if (threadIdx.x == 0) set_status(status, ST_NUMERIC);
    dmax = 0.f;
  }
  // dependent columns (B rank-deficient to rounding) keep a rounding-level diagonal, so
  // that the Jacobi step still returns an orthonormal W
  chol_upper(G, GR_LD, c, R, GR_LD, dmax * (float)(c * 3.6e-15), sqrtf(dmax) * 6e-8f, nzero, ij);
  // AT[qc][i] = R[qc][i]: column qc of R^T is row qc of R; rows c .. CMAX-1 zero
  for (int e = threadIdx.x; e < CMAX * CMAX; e += blockDim.x) {
    const int qc = e / CMAX, i = e % CMAX;
    AT[qc * WS_LDT + i] = (qc < c && i < c) ? R[qc * GR_LD + i] : 0.f;
  }
  __syncthreads();
  jacobi_columns(AT, c, flag, status);
  store_sorted(q, AT, c, sig, status, Ws);
  qw_core(q, Ws, Qt, G, sg);
}

// S1 + S3 with one thread per sample (pi(j), its fiber offset and row j of Omega):
// the form for many samples (batches), where one thread per sample already fills
// the GPU and the warp form below would walk each Feistel cycle 32 times.
__global__ void __launch_bounds__(128) k_sample_omega_t(const RFProb* __restrict__ P,
                                                        const int64_t* __restrict__ pre, int np, int* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pre[np]) return;
  const int p = find_prob(pre, np, t);
  const RFProb& q = P[p];
  const int64_t j = t - pre[p];
  const PhiloxKey key = philox_key(q.seed);
  const uint64_t m = sample_index((uint64_t)j, (uint64_t)q.N, q.fh, key, q.node, status);
  q.idx[j] = (int64_t)m;
  uint64_t rem = m;
  int64_t off = 0;
  for (int t2 = q.ncm - 1; t2 >= 0; --t2) {
    const uint64_t sz = (uint64_t)q.csize[t2];
    off += (int64_t)(rem % sz) * q.cstride[t2];
    rem /= sz;
  }
  q.off[j] = off;
  float* om = q.Om + j * q.c;
  for (int c = 0; c < q.c; ++c) om[c] = gauss_entry(m, (uint32_t)c, key, q.node);
  const int64_t nrt = (q.nS + SK_TI - 1) / SK_TI;
  for (int64_t e2 = j; e2 < nrt; e2 += q.s) q.zcnt[e2] = 0;
}

// S1 + S3 with one warp per sample, the form for few samples (a single tensor), where
// spreading the Gaussians over lanes and SMs shortens the stage: warp j computes pi(j)
// (every lane walks the same Feistel cycle, so the value is warp-uniform) and lane 0 its
// fiber offset; the lanes then share row j of Omega (Box-Muller of Philox counters
// (pi(j), c), one entry per lane and column).  Lane 0 also clears the sketch's
// per-row-tile counters.  Both forms write the same values.
__global__ void __launch_bounds__(128) k_sample_omega(const RFProb* __restrict__ P,
                                                      const int64_t* __restrict__ pre, int np, int* status) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= pre[np]) return;
  const int p = find_prob(pre, np, w);
  const RFProb& q = P[p];
  const int64_t j = w - pre[p];
  const PhiloxKey key = philox_key(q.seed);
  const uint64_t m = sample_index((uint64_t)j, (uint64_t)q.N, q.fh, key, q.node, status);
  float* om = q.Om + j * q.c;
  for (int c = lane; c < q.c; c += 32) om[c] = gauss_entry(m, (uint32_t)c, key, q.node);
  if (lane == 0) {
    q.idx[j] = (int64_t)m;
    uint64_t rem = m;
    int64_t off = 0;
    for (int t2 = q.ncm - 1; t2 >= 0; --t2) {
      const uint64_t sz = (uint64_t)q.csize[t2];
      off += (int64_t)(rem % sz) * q.cstride[t2];
      rem /= sz;
    }
    q.off[j] = off;
    const int64_t nrt = (q.nS + SK_TI - 1) / SK_TI;
    for (int64_t e2 = j; e2 < nrt; e2 += q.s) q.zcnt[e2] = 0;
  }
}

// ------------------------------------------------------------------ host launchers
// Samples up to which S1 + S3 take one warp per sample (beyond: one thread per sample).
constexpr int64_t SO_WARP_MAX = 32768;

static size_t smem_gs() { return (size_t)(SK_TJ * SK_TI + SK_TJ * CMAX) * 4 + SK_TJ * 8; }
static size_t smem_qr() { return (size_t)(2 * QR_MAXF + 2 * CMAX + 1024) * 4 + 64; }
static size_t smem_qr2() { return (size_t)(2 * QR2_MAXF + 2 * CMAX + 32 + 3072) * 4 + 64; }
static size_t smem_qr3() { return (size_t)(QR_MAXF + CMAX * CMAX) * 4; }
static size_t smem_btp() { return (size_t)(32 * BT_LDY + 32 * CMAX) * 4; }
static size_t smem_btf() {
  return (size_t)(32 * BT_LDY + 32 * CMAX + (BT_SC + 1) * CMAX + 2 * CMAX + 1024) * 4 + 64;
}
// k_bt_qr factors one whole chunk: up to (BT_SC | 1) x CMAX floats, then the register
// Householder's two 32 x MR vectors (MR = 16 rows per lane covers chunks up to 512).
static_assert(BT_SC <= 512, "B^T chunk must stay within the register Householder");
static size_t smem_wt() { return (size_t)(QR2_MAXF + 2 * CMAX + 32 + 3072) * 4 + 64; }
static size_t smem_btq() { return (size_t)((BT_SC | 1) * CMAX + 2 * CMAX + 32 + 1024) * 4 + 64; }
static size_t smem_wsvd() {
  return (size_t)(WS_MAXF + 2 * CMAX + 32 + CMAX * WS_LDT + CMAX + 8 + 1024) * 4 + 64;
}
static size_t smem_qw() { return (size_t)(CMAX * CMAX + QW_TI * CMAX) * 4 + CMAX * 8; }
static size_t smem_flip() { return (size_t)(CMAX * CMAX + CMAX) * 4; }
static size_t smem_qwf() { return (size_t)(CMAX * CMAX + 2 * QWF_MAX * CMAX + CMAX) * 4; }
constexpr int IJ_MAX = CMAX * (CMAX + 1) / 2;   // entries of the Cholesky step list
static size_t smem_qz() {
  return std::max((size_t)(QWF_MAX * QZ_LD + 2 * CMAX * GR_LD + CMAX + 4 + IJ_MAX) * 4, smem_qr());
}
static size_t smem_btg() { return (size_t)(32 * BG_LDY + 32 * CMAX + BG_SC * (CMAX | 1)) * 4; }
static size_t smem_wsvd2() {
  return (size_t)(CMAX * QWF_MAX + CMAX * CMAX + CMAX +
                  std::max(2 * CMAX * GR_LD + CMAX * WS_LDT + CMAX + 8 + IJ_MAX, QWF_MAX * CMAX)) * 4;
}

cudaError_t rf_init_attributes() {
  cudaError_t e;
#define RT_ATTR(k, sz)                                                                       \
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sz))) != \
      cudaSuccess)                                                                           \
    return e;
  RT_ATTR(k_gather_sketch, smem_gs());
  RT_ATTR(k_qr1, smem_qr());
  RT_ATTR(k_qr2, smem_qr2());
  RT_ATTR(k_qr3, smem_qr3());
  RT_ATTR(k_bt_partial, smem_btp());
  RT_ATTR(k_bt_qr, smem_btq());
  RT_ATTR(k_wtree, smem_wt());
  RT_ATTR(k_bt_fused, smem_btf());
  RT_ATTR(k_wsvd, smem_wsvd());
  RT_ATTR(k_qw, smem_qw());
  RT_ATTR(k_flip, smem_flip());
  RT_ATTR(k_qwf, smem_qwf());
  RT_ATTR(k_qz, smem_qz());
  RT_ATTR(k_btg, smem_btg());
  RT_ATTR(k_wsvd2, smem_wsvd2());
#undef RT_ATTR
  return cudaSuccess;
}

static inline unsigned grid_of(int64_t units) { return (unsigned)units; }

// S1-S5 and the B-step of S6 (up to the R factors of B^T).
// S5 of every problem of a group: the Cholesky form, or Householder QR of single-block
// sketches and the TSQR tree of tall ones.  The sketches are read from chunk 0 of Zp.
int launch_rf_qr(const RFGroup& g, cudaStream_t st, int* status) {
  const int np = g.nprob;
  const int64_t* pre = g.pre;
  const int64_t stride = np + 1;
  int n = 0;
  if (g.total[STG_QZ] > 0) {                    // Cholesky form of S5
    k_qz<<<grid_of(g.total[STG_QZ]), QR_THREADS, smem_qz(), st>>>(g.probs, pre + STG_QZ * stride, np, status);
    ++n;
  }
  if (g.total[STG_QR1] > 0) {
    k_qr1<<<grid_of(g.total[STG_QR1]), QR_THREADS, smem_qr(), st>>>(g.probs, pre + STG_QR1 * stride, np);
    ++n;
  }
  if (g.total[STG_QR2] > 0) {
    for (int j = 0; j < g.lmax; ++j) {          // the tree's levels, bottom-up
      const int sj = stg_qr2(j);
      if (g.total[sj] == 0) continue;
      k_qr2<<<grid_of(g.total[sj]), QR_THREADS, smem_qr2(), st>>>(g.probs, pre + sj * stride, np, j);
      ++n;
    }
    for (int t = 0; t + 1 < g.lmax; ++t) {      // Q slices combined top-down
      const int stc = stg_qrc(t);
      if (g.total[stc] == 0) continue;
      k_qrc<<<grid_of(g.total[stc]), 256, 0, st>>>(g.probs, pre + stc * stride, np, t);
      ++n;
    }
    k_qr3<<<grid_of(g.total[STG_QR3]), 256, smem_qr3(), st>>>(g.probs, pre + STG_QR3 * stride, np);
    ++n;
  }
  return n;
}

int launch_rf_head(const RFGroup& g, cudaStream_t st, int* status) {
  const int np = g.nprob;
  const int64_t* pre = g.pre;
  const int64_t stride = np + 1;
  int n = 0;
  if (g.total[STG_SAMPLE] > 0) {
    if (g.total[STG_SAMPLE] <= SO_WARP_MAX)
      k_sample_omega<<<(unsigned)((g.total[STG_SAMPLE] * 32 + 127) / 128), 128, 0, st>>>(
          g.probs, pre + STG_SAMPLE * stride, np, status);
    else
      k_sample_omega_t<<<(unsigned)((g.total[STG_SAMPLE] + 127) / 128), 128, 0, st>>>(
          g.probs, pre + STG_SAMPLE * stride, np, status);
    n += 1;
  }
  if (g.total[STG_GS] > 0) {
    k_gather_sketch<<<grid_of(g.total[STG_GS]), 256, smem_gs(), st>>>(g.probs, pre + STG_GS * stride, np);
    ++n;
  }
  n += launch_rf_qr(g, st, status);
  if (g.total[STG_BTG] > 0) {                   // Cholesky form: B-step Grams
    k_btg<<<grid_of(g.total[STG_BTG]), 256, smem_btg(), st>>>(g.probs, pre + STG_BTG * stride, np);
    ++n;
  }
  if (g.total[STG_BTQ] > 0) {
    if (g.total[STG_BTP] == g.total[STG_BTQ]) {   // every problem reduces B^T over one row block
      k_bt_fused<<<grid_of(g.total[STG_BTQ]), QR_THREADS, smem_btf(), st>>>(g.probs, pre + STG_BTQ * stride, np);
      n += 1;
    } else {
      k_bt_partial<<<grid_of(g.total[STG_BTP]), 256, smem_btp(), st>>>(g.probs, pre + STG_BTP * stride, np);
      k_bt_qr<<<grid_of(g.total[STG_BTQ]), QR_THREADS, smem_btq(), st>>>(g.probs, pre + STG_BTQ * stride, np);
      n += 2;
    }
  }
  for (int j = 0; j < g.wmax; ++j) {            // R tree over many chunk factors
    const int sj = stg_wt(j);
    if (g.total[sj] == 0) continue;
    k_wtree<<<grid_of(g.total[sj]), QR_THREADS, smem_wt(), st>>>(g.probs, pre + sj * stride, np, j);
    ++n;
  }
  return n;
}

// S6 after the B-step: the SVD of R, W, U = Q W and the sign rule (also W with signs).
int launch_rf_tail(const RFGroup& g, cudaStream_t st, int* status) {
  const int np = g.nprob;
  const int64_t* pre = g.pre;
  const int64_t stride = np + 1;
  int n = 0;
  if (g.total[STG_WSVD] > 0) {
    k_wsvd<<<grid_of(g.total[STG_WSVD]), QR_THREADS, smem_wsvd(), st>>>(g.probs, pre + STG_WSVD * stride, np,
                                                                   status);
    n += 1;
  }
  if (g.total[STG_WSV2] > 0) {                  // Cholesky form of the W-step, U = Q W, signs
    k_wsvd2<<<grid_of(g.total[STG_WSV2]), QR_THREADS, smem_wsvd2(), st>>>(g.probs, pre + STG_WSV2 * stride, np,
                                                                     status);
    n += 1;
  }
  if (g.total[STG_QWF] > 0) {
    k_qwf<<<grid_of(g.total[STG_QWF]), 512, smem_qwf(), st>>>(g.probs, pre + STG_QWF * stride, np);
    ++n;
  }
  if (g.total[STG_QW] > 0) {
    k_qw<<<grid_of(g.total[STG_QW]), 256, smem_qw(), st>>>(g.probs, pre + STG_QW * stride, np);
    k_flip<<<grid_of(g.total[STG_FLIP]), 256, smem_flip(), st>>>(g.probs, pre + STG_FLIP * stride, np);
    n += 2;
  }
  return n;
}

int launch_range_finder(const RFGroup& g, cudaStream_t st, int* status) {
  return launch_rf_head(g, st, status) + launch_rf_tail(g, st, status);
}

int launch_sample_only(const RFGroup& g, cudaStream_t st, int* status) {
  if (g.total[STG_SAMPLE] <= 0) return 0;
  k_sample<<<(unsigned)((g.total[STG_SAMPLE] + 255) / 256), 256, 0, st>>>(
      g.probs, g.pre + STG_SAMPLE * (g.nprob + 1), g.nprob, status);
  return 1;
}

int launch_sketch_sum(const RFGroup& g, float* const* Zout, cudaStream_t st) {
  const int64_t stride = g.nprob + 1;
  k_sketch_sum<<<(unsigned)((g.total[STG_ZSUM] + 255) / 256), 256, 0, st>>>(
      g.probs, g.pre + STG_ZSUM * stride, g.nprob, Zout);
  return 1;
}

}  // namespace rt
