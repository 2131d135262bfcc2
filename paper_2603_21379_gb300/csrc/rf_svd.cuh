// rf_svd.cuh - device steps shared by the W-step kernels of the range finder: the
// one-sided Jacobi SVD of a c x c matrix held by columns in shared memory, the
// sorted singular values and left singular vectors it gives (W-step of Alg. 1: the
// dominant left singular vectors of B = Q^T Y), and U = Q W(:, :r) with the column
// sign rule.  Included by the translation units that run these steps; every
// function must be called by all threads of the CTA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"

namespace rt {

// One-sided Jacobi (Hestenes) on the c columns of A, column qc at AT[qc * WS_LDT + i]
// for i < CMAX (rows c .. CMAX-1 zero): rotates column pairs in round-robin order
// until the columns are orthogonal, A V = W Sigma.  Columns are processed one
// 16-lane group per pair, until a sweep makes no rotation or leaves every pair below
// sqrt(tol) / 2 before rotation (at most WS_MAX_SWEEPS, else ST_NUMERIC).  flag: 2 ints
// and 2 unsigned of shared scratch.  Needs blockDim.x >= 8 CMAX.
__device__ __noinline__ void jacobi_columns(float* AT, int c, int* flag, int* status) {
  constexpr int LDT = WS_LDT;
  const int ne = c + (c & 1);           // even number of players (dummy = c)
  // Convergence threshold on |a_p . a_q| / (|a_p| |a_q|): about twice the worst rounding
  // error of the 16-term tree dot product below, so a converged pair is not rotated again
  // on noise alone.
  const float tol = 2e-6f;
  // Round-robin (circle) ordering: pair pr meets columns pa, qa; each round the players
  // other than column 0 move one seat.  One pair per 16-lane group; lane l16 holds rows
  // l16 + 16 k.  Column stride LDT = 80 puts the two groups of a warp on opposite bank
  // halves (their columns differ in parity).
  const int pr = threadIdx.x >> 4, l16 = threadIdx.x & 15;
  const int kc = (c + 15) >> 4;
  const unsigned gm = 0xffffu << (threadIdx.x & 16);
  // Stop after a sweep in which no pair rotated, or in which every pair's relative
  // off-diagonal |a_p.a_q| / (|a_p||a_q|) was below sqrt(tol) / 2: cyclic Jacobi
  // converges quadratically, so such a sweep leaves every pair below tol and the next
  // sweep would rotate nothing.
  const float quad_stop = 0.5f * sqrtf(tol);
  unsigned* dmax = reinterpret_cast<unsigned*>(flag + 2);   // per sweep, as float bits (>= 0)
  if (threadIdx.x < 2) dmax[threadIdx.x] = 0u;
  __syncthreads();
  bool converged = false;
  for (int sweep = 0; sweep < WS_MAX_SWEEPS && !converged; ++sweep) {
    int t = pr - 1, u = ne - 2 - pr;
    int rotated = 0;
    float dloc = 0.f;
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      const int pa = (pr == 0) ? 0 : 1 + t;
      const int qa = 1 + u;
      if (pr < ne / 2 && pa < c && qa < c) {
        float* ap = AT + pa * LDT + l16;
        float* aq = AT + qa * LDT + l16;
        float x[CMAX / 16], y[CMAX / 16];
#pragma unroll
        for (int k = 0; k < CMAX / 16; ++k) {
          x[k] = (k < kc) ? ap[16 * k] : 0.f;
          y[k] = (k < kc) ? aq[16 * k] : 0.f;
        }
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int k = 0; k < CMAX / 16; ++k) {
          al = fmaf(x[k], x[k], al);
          be = fmaf(y[k], y[k], be);
          ga = fmaf(x[k], y[k], ga);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(gm, al, o);
          be += __shfl_xor_sync(gm, be, o);
          ga += __shfl_xor_sync(gm, ga, o);
        }
        const float rel = (ga != 0.f) ? fabsf(ga) * rsqrt_approx(al) * rsqrt_approx(be) : 0.f;
        dloc = fmaxf(dloc, rel);
        if (ga != 0.f && rel > tol) {
          // tangent of the angle that makes the pair orthogonal, smaller root
          const float zeta = (be - al) * rcp_approx(2.f * ga);
          const float az = fabsf(zeta);
          float tt;
          if (az > 1e18f) {
            tt = 0.5f * rcp_approx(zeta);
          } else {
            const float s1 = fmaf(zeta, zeta, 1.f);
            tt = copysignf(rcp_approx(az + s1 * rsqrt_approx(s1)), zeta);
          }
          const float cs = rsqrt_approx(fmaf(tt, tt, 1.f)), sn = cs * tt;
#pragma unroll
          for (int k = 0; k < CMAX / 16; ++k) {
            if (k < kc) {
              ap[16 * k] = cs * x[k] - sn * y[k];
              aq[16 * k] = sn * x[k] + cs * y[k];
            }
          }
          rotated = 1;
        }
      }
      if (++t == ne - 1) t = 0;
      if (++u == ne - 1) u = 0;
      __syncthreads();
    }
    // flag[sweep & 1] is set by any pair that rotated; the other slot is cleared for the
    // next sweep (it was last read before the previous barrier).
    if (rotated) flag[sweep & 1] = 1;
    const unsigned dw = __reduce_max_sync(0xffffffffu, __float_as_uint(dloc));
    if ((threadIdx.x & 31) == 0 && dw) atomicMax(&dmax[sweep & 1], dw);
    __syncthreads();
    const int f = flag[sweep & 1];
    const float dm = __uint_as_float(dmax[sweep & 1]);
    if (threadIdx.x == 0) { flag[(sweep + 1) & 1] = 0; dmax[(sweep + 1) & 1] = 0u; }
    __syncthreads();
    converged = !f || dm < quad_stop;
  }
  if (!converged && threadIdx.x == 0) set_status(status, ST_NUMERIC);
}

// Singular values (column norms of the converged A V) in descending order into
// q.sigma (and q.sigma_out), the normalised columns into q.W (c x c row-major, column
// k = k-th largest).  sig: c floats of shared scratch.
// Ws (optional): W(:, :r) also into Ws[t * CMAX + col], columns r .. multiple of 4 zero.
__device__ __noinline__ void store_sorted(const RFProb& q, const float* AT, int c, float* sig, int* status,
                                          float* Ws = nullptr) {
  constexpr int LDT = WS_LDT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // singular values (column norms) and descending order
  for (int qc = warp; qc < c; qc += nw) {
    float s2 = 0.f;
    for (int i = lane; i < c; i += 32) s2 = fmaf(AT[qc * LDT + i], AT[qc * LDT + i], s2);
    s2 = warp_sum(s2);
    if (lane == 0) sig[qc] = sqrtf(s2);
  }
  __syncthreads();
  if (threadIdx.x < c) {
    const int qc = threadIdx.x;
    const float sq = sig[qc];
    if (!(sq == sq)) set_status(status, ST_NUMERIC);
    int rank = 0;
    for (int t = 0; t < c; ++t) rank += (sig[t] > sq) || (sig[t] == sq && t < qc);
    q.sigma[rank] = sq;
    if (q.sigma_out) q.sigma_out[rank] = sq;
    const float inv = (sq > 0.f) ? 1.f / sq : 0.f;
    for (int i = 0; i < c; ++i) q.W[i * c + rank] = AT[qc * LDT + i] * inv;
    if (Ws && rank < q.r)
      for (int i = 0; i < c; ++i) Ws[i * CMAX + rank] = AT[qc * LDT + i] * inv;
  }
  if (Ws) {
    const int r = q.r, rp = (r + 3) & ~3;
    for (int e = threadIdx.x; e < c * (rp - r); e += blockDim.x) Ws[(e / (rp - r)) * CMAX + r + e % (rp - r)] = 0.f;
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long sign_key(float v, int64_t row) {
  return ((unsigned long long)__float_as_uint(fabsf(v)) << 32) |
         (unsigned long long)(0xffffffffu - (uint32_t)row);
}

// Q of a problem with n_S <= QWF_MAX rows staged transposed: Qt[t][i] = Q[i][t] (rows
// padded to a multiple of 4 with zeros).  No barrier.
__device__ __forceinline__ void qw_stage_q(const RFProb& q, float* Qt) {
  const int m = (int)q.nS, c = q.c, mp = (m + 3) & ~3;
  for (int e = threadIdx.x; e < mp * c; e += blockDim.x) {
    const int i = e / c, t = e % c;
    Qt[t * QWF_MAX + i] = i < m ? q.Q[e] : 0.f;
  }
}

// U = Q W(:, :r) and the sign rule for a problem with n_S <= QWF_MAX rows, by one CTA,
// from the staged Qt and Ws[t][col] = W[t][col] (columns r .. multiple of 4 zero).
// A thread's 4 x 4 tile of U takes one 16-byte load of Q and one of W per t; every
// entry is the same sequential fma chain over t.  The sign rule's key (|u|, lowest
// row) of each column is a warp max-reduction over the U tile in shared memory.
// Writes q.U and q.Wsg (W(:, :r) with the columns' signs).  Us: QWF_MAX*CMAX floats,
// sg: CMAX floats of shared memory.
__device__ __noinline__ void qw_core(const RFProb& q, const float* Ws, const float* Qt, float* Us, float* sg) {
  const int m = (int)q.nS;
  const int c = q.c, r = q.r;
  const int mp = (m + 3) & ~3, rp = (r + 3) & ~3;
  __syncthreads();
  const int nrg = mp >> 2, ncg = rp >> 2;
  for (int tile = threadIdx.x; tile < nrg * ncg; tile += blockDim.x) {
    const int rg = tile % nrg, cg = tile / nrg;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int t = 0; t < c; ++t) {
      const float4 qv = *reinterpret_cast<const float4*>(Qt + t * QWF_MAX + 4 * rg);
      const float4 wv = *reinterpret_cast<const float4*>(Ws + t * CMAX + 4 * cg);
      const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
      const float wb[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(qa[a], wb[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Us[(4 * rg + a) * CMAX + 4 * cg + b] = acc[a][b];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int col = warp; col < r; col += nw) {
    unsigned long long best = 0ull;
    for (int i = lane; i < m; i += 32) {
      const unsigned long long k = sign_key(Us[i * CMAX + col], i);
      best = k > best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long k = __shfl_xor_sync(0xffffffffu, best, o);
      best = k > best ? k : best;
    }
    if (lane == 0) {
      const int rstar = (int)(0xffffffffu - (uint32_t)(best & 0xffffffffull));
      sg[col] = (Us[rstar * CMAX + col] < 0.f) ? -1.f : 1.f;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) q.U[e] = sg[e % r] * Us[(e / r) * CMAX + e % r];
  for (int e = threadIdx.x; e < c * r; e += blockDim.x) q.Wsg[e] = sg[e % r] * Ws[(e / r) * CMAX + e % r];
  __syncthreads();
}

// U = Q W(:, :r) and the sign rule with Q and W read from global memory.
// smem: Ws[CMAX*CMAX] | Qt[CMAX*QWF_MAX] | Us[QWF_MAX*CMAX] | sg[CMAX] floats.
__device__ __noinline__ void qw_sign(const RFProb& q, float* smem) {
  float* Ws = smem;
  float* Qt = Ws + CMAX * CMAX;
  float* Us = Qt + QWF_MAX * CMAX;
  float* sg = Us + QWF_MAX * CMAX;
  const int c = q.c, r = q.r, rp = (r + 3) & ~3;
  for (int e = threadIdx.x; e < c * rp; e += blockDim.x) {
    const int t = e / rp, col = e % rp;
    Ws[t * CMAX + col] = col < r ? q.W[t * c + col] : 0.f;
  }
  qw_stage_q(q, Qt);
  qw_core(q, Ws, Qt, Us, sg);
}

}  // namespace rt
