// kron_kernels.cu - the Kronecker-structured sketch of the rHKron comparison
// method (Sec. 3.3): one small Gaussian Omega_j (n_j x l_j) per mode and, for
// every mode k, Z_k = X^(k) (Omega_0 (x) .. (x) Omega_{k-1} (x) Omega_{k+1} (x) ..),
// the unfolding of X x_{j != k} Omega_j^T (n_k x L_k, L_k = prod_{j != k} l_j).
//
// All d sketches come from one read of X.  With X viewed as S slabs M_s of its
// last two modes (n1 x n2, s the C-order index of the leading d-2 modes) and
// w_s(kappa) = prod_{j < d-2} Omega_j(i_j(s), a_j) the Kronecker weight of the
// slab's leading indices (kappa = C-order index of (a_0 .. a_{d-3})):
//     A_s  = M_s Omega_{d-1}            (n1 x l_b)
//     Bt_s = Omega_{d-2}^T M_s          (l_a x n2)
//     T_s  = Omega_{d-2}^T A_s          (l_a x l_b)
//     Z_{d-2}(i, (kappa, b)) = sum_s w_s(kappa) A_s(i, b)
//     Z_{d-1}(j, (kappa, a)) = sum_s w_s(kappa) Bt_s(a, j)
//     Z_m(i_m, (kappa', a, b)) = sum_{s : i_m(s) = i_m} w_s^{(not m)}(kappa') T_s(a, b)   (m < d-2)
// The pass (k_kron_sketch) streams the slabs through shared memory (double-
// buffered cp.async), forms A_s, Bt_s and T_s with float32 FMAs (about 2 (l_a +
// l_b) per element of X: a few per byte, under the FFMA rate at the HBM rate),
// keeps each CTA's share of Z_{d-2} and Z_{d-1} in registers, and writes T_s;
// k_kron_reduce sums the CTAs' shares in a fixed order and k_kron_lead forms
// the leading modes' sketches from the T_s.  The rest of the method (QR of
// each Z_k, the reduced core, its factorisation) runs on the library's range-
// finder and core kernels; k_kron_qw and k_kron_sign finish U_k = Q_k W_k and
// the column-sign rule.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"
#include "rt_rng.cuh"

namespace rt {

constexpr int KS_THREADS = 256;
constexpr int KS_Q = KRON_ZMAX / KS_THREADS;   // register partials per thread and sketch

// Omega_j (n_j x l_j) of every mode, concatenated, entry (i, a) = Gaussian of stream 3
// keyed by row i and column a of node j.
__global__ void k_kron_omega(KronArgs a, uint64_t seed) {
  const PhiloxKey key = philox_key(seed);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.om_total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int j = 0;
    while (j + 1 < a.d && e >= a.om_off[j + 1]) ++j;
    const int64_t loc = e - a.om_off[j];
    const int64_t i = loc / a.ell[j];
    const int c = (int)(loc % a.ell[j]);
    a.om[e] = gauss_entry((uint64_t)i, (uint32_t)c, key, (uint32_t)j, 3u);
  }
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Kronecker weights of every slab: Wt[s][kappa] = prod_{j < d-2} Omega_j(i_j(s), a_j(kappa)).
__global__ void k_kron_weights(KronArgs a) {
  const int64_t tot = a.S * a.K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rs = e / a.K;
    int rk = (int)(e % a.K);
    float v = 1.f;
    for (int j = a.d - 3; j >= 0; --j) {     // leading modes, last fastest
      const int64_t ij = rs % a.n[j];
      rs /= a.n[j];
      const int aj = rk % a.ell[j];
      rk /= a.ell[j];
      v *= __ldg(a.om + a.om_off[j] + ij * a.ell[j] + aj);
    }
    a.Wt[e] = v;
  }
}

// Slab s of X into Ms (n1 rows, padded stride ld) and its K weights into w: 16-byte
// cp.async for float32 X, element loads otherwise; 4-byte cp.async for the weights.
__device__ __forceinline__ void load_slab(const KronArgs& a, int64_t s, float* Ms, int ld, float* w) {
  const int n1 = a.n1, n2 = a.n2, nq = n2 >> 2;
  if (a.dtype == DT_F32) {
    const float* src = static_cast<const float*>(a.X) + s * (int64_t)n1 * n2;
    for (int e = threadIdx.x; e < n1 * nq; e += KS_THREADS) {
      const int i = e / nq, q = e - i * nq;
      cp_async16(Ms + i * ld + 4 * q, src + (int64_t)i * n2 + 4 * q);
    }
  } else {
    for (int e = threadIdx.x; e < n1 * n2; e += KS_THREADS) {
      const int i = e / n2, j = e % n2;
      Ms[i * ld + j] = load_x(a.X, a.dtype, (s * n1 + i) * (int64_t)n2 + j);
    }
  }
  for (int k = threadIdx.x; k < a.K; k += KS_THREADS) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(w + k);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(a.Wt + s * a.K + k) : "memory");
  }
}

// Dynamic smem (floats): Ms[2][n1][ld] | w[2][Kp] | Ob[n2][LP] | Oa[n1][LP] | Ap[HA][n1][LP] |
// Bp[HB][LP][n2] | Af[n1][LP] | Btf[LP][n2]
// Register shares: thread t owns row i = t % n1 of Z_{d-2} for the weights kappa of its
// group t / n1 (and column j = t % n2 of Z_{d-1} likewise), all LP columns b (a), so the
// updates need no index arithmetic.
template <int LP>
__global__ void __launch_bounds__(KS_THREADS, 1) k_kron_sketch(KronArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int n1 = a.n1, n2 = a.n2, la = a.la, lb = a.lb, K = a.K;
  const int ld = n2 + 4, nq = n2 >> 2, Kp = (K + 3) & ~3;
  const int HA = a.ha, HB = a.hb;
  float* Ms0 = sm;
  float* w0 = Ms0 + 2 * n1 * ld;
  float* Ob = w0 + 2 * Kp;
  float* Oa = Ob + n2 * LP;
  float* Ap = Oa + n1 * LP;
  float* Bp = Ap + HA * n1 * LP;
  float* Af = Bp + HB * LP * n2;
  float* Btf = Af + n1 * LP;
  const int tid = threadIdx.x;
  const float* Oma = a.om + a.om_off[a.d - 2];
  const float* Omb = a.om + a.om_off[a.d - 1];
  for (int e = tid; e < n2 * LP; e += KS_THREADS) {
    const int j = e / LP, c = e % LP;
    Ob[e] = c < lb ? Omb[(int64_t)j * lb + c] : 0.f;
  }
  for (int e = tid; e < n1 * LP; e += KS_THREADS) {
    const int i = e / LP, c = e % LP;
    Oa[e] = c < la ? Oma[(int64_t)i * la + c] : 0.f;
  }
  constexpr int KPT = KS_Q / LP;               // weights per thread and sketch
  const int g1n = KS_THREADS / n1, g2n = KS_THREADS / n2;
  const int i_own = tid % n1, g1 = tid / n1;
  const int j_own = tid % n2, g2 = tid / n2;
  const int kc1 = (K + g1n - 1) / g1n, kc2 = (K + g2n - 1) / g2n;
  const int k10 = g1 < g1n ? g1 * kc1 : K, k11 = min(K, k10 + kc1);
  const int k20 = g2 < g2n ? g2 * kc2 : K, k21 = min(K, k20 + kc2);
  float z1[KS_Q], z2[KS_Q];
#pragma unroll
  for (int q = 0; q < KS_Q; ++q) { z1[q] = 0.f; z2[q] = 0.f; }
  const int cwq = (nq + HA - 1) / HA;          // float4 columns per chunk of A
  const int rh = (n1 + HB - 1) / HB;           // rows per chunk of Bt
  const int64_t S = a.S;
  int64_t s = blockIdx.x;
  if (s < S) load_slab(a, s, Ms0, ld, w0);
  cp_async_commit();
  for (int64_t t = 0; s < S; ++t, s += gridDim.x) {
    float* Ms = Ms0 + (t & 1) * n1 * ld;
    const float* w = w0 + (t & 1) * Kp;
    const int64_t sn = s + gridDim.x;
    if (sn < S) load_slab(a, sn, Ms0 + ((t + 1) & 1) * n1 * ld, ld, w0 + ((t + 1) & 1) * Kp);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    // partials of A = M Omega_b: row i, column chunk h
    for (int e = tid; e < n1 * HA; e += KS_THREADS) {
      const int i = e % n1, h = e / n1;
      const int q0 = h * cwq, q1 = min(nq, q0 + cwq);
      float acc[LP];
#pragma unroll
      for (int c = 0; c < LP; ++c) acc[c] = 0.f;
      for (int q = q0; q < q1; ++q) {
        const float4 m = *reinterpret_cast<const float4*>(Ms + i * ld + 4 * q);
        const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int c = 0; c < LP; c += 4) {
            const float4 o = *reinterpret_cast<const float4*>(Ob + (4 * q + u) * LP + c);
            acc[c] = fmaf(mv[u], o.x, acc[c]);
            acc[c + 1] = fmaf(mv[u], o.y, acc[c + 1]);
            acc[c + 2] = fmaf(mv[u], o.z, acc[c + 2]);
            acc[c + 3] = fmaf(mv[u], o.w, acc[c + 3]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < LP; c += 4)
        *reinterpret_cast<float4*>(Ap + (h * n1 + i) * LP + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
    }
    // partials of Bt = Omega_a^T M: four columns 4 jq .. 4 jq + 3, row chunk h
    for (int e = tid; e < nq * HB; e += KS_THREADS) {
      const int jq = e % nq, h = e / nq;
      const int i0 = h * rh, i1 = min(n1, i0 + rh);
      float acc[LP][4];
#pragma unroll
      for (int c = 0; c < LP; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[c][u] = 0.f;
      for (int i = i0; i < i1; ++i) {
        const float4 m = *reinterpret_cast<const float4*>(Ms + i * ld + 4 * jq);
#pragma unroll
        for (int c = 0; c < LP; c += 4) {
          const float4 o = *reinterpret_cast<const float4*>(Oa + i * LP + c);
          const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            acc[c + v][0] = fmaf(ov[v], m.x, acc[c + v][0]);
            acc[c + v][1] = fmaf(ov[v], m.y, acc[c + v][1]);
            acc[c + v][2] = fmaf(ov[v], m.z, acc[c + v][2]);
            acc[c + v][3] = fmaf(ov[v], m.w, acc[c + v][3]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < LP; ++c)
        *reinterpret_cast<float4*>(Bp + (h * LP + c) * n2 + 4 * jq) =
            make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
    }
    __syncthreads();
    // A, Bt: partials summed in chunk order
    for (int e = tid; e < n1 * LP; e += KS_THREADS) {
      float v = 0.f;
      for (int h = 0; h < HA; ++h) v += Ap[h * n1 * LP + e];
      Af[e] = v;
    }
    for (int e = tid; e < LP * n2; e += KS_THREADS) {
      float v = 0.f;
      for (int h = 0; h < HB; ++h) v += Bp[h * LP * n2 + e];
      Btf[e] = v;
    }
    __syncthreads();
    // T_s = Omega_a^T A (one warp per entry, lanes over rows)
    {
      const int wp = tid >> 5, lane = tid & 31;
      for (int o = wp; o < la * lb; o += KS_THREADS / 32) {
        const int ca = o / lb, cb = o % lb;
        float v = 0.f;
        for (int i = lane; i < n1; i += 32) v = fmaf(Oa[i * LP + ca], Af[i * LP + cb], v);
        v = warp_sum(v);
        if (lane == 0) a.Ts[s * (int64_t)(la * lb) + o] = v;
      }
    }
    // this CTA's shares of Z_{d-2} (row i_own) and Z_{d-1} (column j_own)
    {
      float av[LP], bv[LP];
#pragma unroll
      for (int c = 0; c < LP; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(Af + i_own * LP + c);
        av[c] = v.x; av[c + 1] = v.y; av[c + 2] = v.z; av[c + 3] = v.w;
      }
#pragma unroll
      for (int c = 0; c < LP; ++c) bv[c] = Btf[c * n2 + j_own];
#pragma unroll
      for (int kk = 0; kk < KPT; ++kk) {
        const float w1 = (k10 + kk < k11) ? w[k10 + kk] : 0.f;
        const float w2 = (k20 + kk < k21) ? w[k20 + kk] : 0.f;
#pragma unroll
        for (int c = 0; c < LP; ++c) {
          z1[kk * LP + c] = fmaf(w1, av[c], z1[kk * LP + c]);
          z2[kk * LP + c] = fmaf(w2, bv[c], z2[kk * LP + c]);
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  const int tot1 = n1 * K * lb, tot2 = n2 * K * la;
#pragma unroll
  for (int kk = 0; kk < KPT; ++kk) {
#pragma unroll
    for (int c = 0; c < LP; ++c) {
      if (k10 + kk < k11 && c < lb)
        a.part1[(int64_t)blockIdx.x * tot1 + ((int64_t)i_own * K + k10 + kk) * lb + c] = z1[kk * LP + c];
      if (k20 + kk < k21 && c < la)
        a.part2[(int64_t)blockIdx.x * tot2 + ((int64_t)j_own * K + k20 + kk) * la + c] = z2[kk * LP + c];
    }
  }
}

// Z_{d-2} and Z_{d-1}: the CTAs' shares summed in CTA order.
__global__ void k_kron_reduce(KronArgs a, int nblk) {
  const int tot1 = a.n1 * a.K * a.lb, tot2 = a.n2 * a.K * a.la;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot1 + tot2; e += gridDim.x * blockDim.x) {
    float v = 0.f;
    if (e < tot1) {
      for (int g = 0; g < nblk; ++g) v += a.part1[(int64_t)g * tot1 + e];
      a.z[a.d - 2][e] = v;
    } else {
      const int f = e - tot1;
      for (int g = 0; g < nblk; ++g) v += a.part2[(int64_t)g * tot2 + f];
      a.z[a.d - 1][f] = v;
    }
  }
}

// Z_m for the leading modes m < d-2 from the slabs' T_s: eight lanes per entry
// (i_m, (kappa', a, b)) split the sum over the S / n_m slabs with that i_m and
// combine it by shuffles (32-bit index arithmetic: S l_a l_b < 2^31).
__global__ void k_kron_lead(KronArgs a) {
  const int nl = a.d - 2, lab = a.la * a.lb;
  const int sub = threadIdx.x & 7;
  const int gid = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3);
  const int gstride = (int)(((int64_t)gridDim.x * blockDim.x) >> 3);
  for (int m = 0; m < nl; ++m) {
    const int Km = a.K / a.ell[m];
    const int cols = Km * lab, tot = (int)a.n[m] * cols;
    const int inner = (int)(a.S / a.n[m]);
    const int iters = (tot + gstride - 1) / gstride;
    for (int it = 0; it < iters; ++it) {     // the eight lanes of an entry stay together
      const int e = gid + it * gstride;
      const bool on = e < tot;
      const int ee = on ? e : 0;
      const int im = ee / cols, col = ee - im * cols;
      const int kp = col / lab, ab = col - kp * lab;
      float acc = 0.f;
      for (int t = sub; on && t < inner; t += 8) {
        // leading multi-index with i_m fixed, the others from t (C order), and the
        // Kronecker weight of the other leading modes' columns from kappa'
        int rt = t, s = 0, stride = 1, rk = kp;
        float wv = 1.f;
        for (int j = nl - 1; j >= 0; --j) {
          int ij;
          if (j == m) {
            ij = im;
          } else {
            const int nj = (int)a.n[j], lj = a.ell[j];
            ij = rt % nj;
            rt /= nj;
            const int aj = rk % lj;
            rk /= lj;
            wv *= __ldg(a.om + a.om_off[j] + ij * lj + aj);
          }
          s += ij * stride;
          stride *= (int)a.n[j];
        }
        acc = fmaf(wv, __ldg(a.Ts + (int64_t)s * lab + ab), acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      if (on && sub == 0) a.z[m][e] = acc;
    }
  }
}

// U_k = Q_k W_k for every mode (Q_k: n_k x L_k, W_k: L_k x r_k, row-major).
__global__ void k_kron_qw(KronFinish f) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < f.utotal;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < f.d && e >= f.uoff[k + 1]) ++k;
    const int64_t loc = e - f.uoff[k];
    const int r = f.r[k], L = f.L[k];
    const int64_t i = loc / r;
    const int c = (int)(loc % r);
    const float* q = f.Q + f.qoff[k] + i * L;
    const float* wk = f.W + f.woff[k] + c;
    float v = 0.f;
    for (int l = 0; l < L; ++l) v = fmaf(q[l], wk[(int64_t)l * r], v);
    f.U[e] = v;
  }
}

// Column-sign rule of U_k (largest-magnitude entry positive, ties: lowest row), one
// warp per column of every mode; flips the column and records the sign.
__global__ void k_kron_sign(KronFinish f) {
  const int lane = threadIdx.x & 31;
  const int col = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (col >= f.rtotal) return;
  int k = 0, c = col;
  while (c >= f.r[k]) { c -= f.r[k]; ++k; }
  const int r = f.r[k];
  float* u = f.U + f.uoff[k] + c;
  const int64_t n = f.n[k];
  float best = -1.f;
  int64_t bi = 0;
  for (int64_t i = lane; i < n; i += 32) {
    const float v = fabsf(u[i * r]);
    if (v > best) { best = v; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const float sg = u[bi * r] < 0.f ? -1.f : 1.f;
  if (sg < 0.f)
    for (int64_t i = lane; i < n; i += 32) u[i * r] = -u[i * r];
  if (lane == 0) f.sign[col] = sg;
}

// G(i_0, .., i_{d-1}) *= prod_k sign_k(i_k).
__global__ void k_kron_flip_core(KronFinish f) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < f.gtotal;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rest = e;
    float sg = 1.f;
    for (int k = f.d - 1; k >= 0; --k) {
      const int ik = (int)(rest % f.r[k]);
      rest /= f.r[k];
      sg *= f.sign[f.roff[k] + ik];
    }
    f.G[e] *= sg;
  }
}

// Gram M_k = C^(k) C^(k)^T of every mode unfolding of the reduced tensor C (float32,
// C order, L_0 x .. x L_{d-1}, L_k <= 64), for the W-step's Cholesky form: column chunks
// of 128 (x, y) pairs staged in shared memory (element (a, col) at x L_k B_k + a B_k + y,
// col = x B_k + y); each thread owns a 4 x 4 block of the upper triangle, sums a chunk's
// rounded-product FMAs in float32 and adds the chunk total to a Kahan sum; the CTAs'
// partials are then added in double-float in CTA order (k_mode_gram_reduce), written as
// the (sum, correction) words the W-step reads.
constexpr int MG_CH = 128;
constexpr int MG_LD = 68;          // a chunk column (64 entries) + 4: 16-byte aligned rows
// Chunk ch of C^(k) into Cs[cc][a] (4-byte cp.async): consecutive threads take
// consecutive global addresses (along y when B_k > 1, along a when B_k = 1, where a
// column is contiguous).
__device__ __forceinline__ void mg_load(const ModeGram& g, int c, int B, int LB, int N, int ch, float* Cs) {
  const int c0 = ch * MG_CH, cw = min(MG_CH, N - c0);
  for (int e = threadIdx.x; e < c * MG_CH; e += 256) {
    int a, cc;
    if (B == 1) { cc = e / c; a = e - cc * c; } else { a = e / MG_CH; cc = e - a * MG_CH; }
    if (cc < cw) {
      const int col = c0 + cc, x = col / B, y = col - x * B;
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(Cs + cc * MG_LD + a);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(g.C + (int64_t)x * LB + (int64_t)a * B + y)
                   : "memory");
    }
  }
}

__global__ void __launch_bounds__(256, 2) k_mode_gram(ModeGram g) {
  extern __shared__ __align__(16) float mgs[];   // two chunk buffers of MG_CH x MG_LD
  const int k = blockIdx.x / g.ctas, cta = blockIdx.x % g.ctas;
  const int c = g.L[k], nb = (c + 3) / 4;
  int bi = -1, bj = -1;
  {
    int t = threadIdx.x;
    for (int i = 0; i < nb; ++i) {
      const int cnt = nb - i;
      if (t < cnt) { bi = i; bj = i + t; break; }
      t -= cnt;
    }
  }
  constexpr int BUF = MG_CH * MG_LD;
  for (int e = threadIdx.x; e < 2 * BUF; e += 256) mgs[e] = 0.f;   // entries a >= c stay zero
  __syncthreads();
  float hs[4][4], ks[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { hs[i][j] = 0.f; ks[i][j] = 0.f; }
  const int N = g.N[k], B = g.B[k], LB = c * g.B[k];
  const int nch = (N + MG_CH - 1) / MG_CH;
  if (cta < nch) mg_load(g, c, B, LB, N, cta, mgs);
  cp_async_commit();
  int t = 0;
  for (int ch = cta; ch < nch; ch += g.ctas, ++t) {
    const int cw = min(MG_CH, N - ch * MG_CH);
    const float* Cs = mgs + (t & 1) * BUF;
    if (ch + g.ctas < nch) mg_load(g, c, B, LB, N, ch + g.ctas, mgs + ((t + 1) & 1) * BUF);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if (bi >= 0) {
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      const float* pu = Cs + 4 * bi;
      const float* pv = Cs + 4 * bj;
#pragma unroll 4
      for (int cc = 0; cc < cw; ++cc) {
        const float4 u4 = *reinterpret_cast<const float4*>(pu + cc * MG_LD);
        const float4 v4 = *reinterpret_cast<const float4*>(pv + cc * MG_LD);
        const float u[4] = {u4.x, u4.y, u4.z, u4.w}, v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(u[i], v[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) kahan_add(hs[i][j], ks[i][j], acc[i][j]);
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  if (bi >= 0) {
    float* part = g.part + g.poff[k] + (int64_t)cta * c * c * 2;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int row = 4 * bi + i, col = 4 * bj + j;
        if (row < c && col < c && col >= row) {
          part[(row * c + col) * 2] = hs[i][j];
          part[(row * c + col) * 2 + 1] = -ks[i][j];
        }
      }
  }
}

// The CTAs' partial Grams added in order (double-float) into the W-step's Gram words,
// and Q = I for the W-step's U = Q W (the reduced tensor's rows are its own basis).
__global__ void k_mode_gram_reduce(ModeGram g) {
  const int k = blockIdx.y, c = g.L[k];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
    const int i = e / c, j = e - i * c;
    g.qeye[k][e] = (i == j) ? 1.f : 0.f;
    if (j < i) continue;
    float hi = 0.f, lo = 0.f;
    for (int t = 0; t < g.ctas; ++t) {
      const float* p = g.part + g.poff[k] + ((int64_t)t * c * c + e) * 2;
      df_add(hi, lo, p[0], p[1]);
    }
    g.cp[k][2 * e] = hi;
    g.cp[k][2 * e + 1] = lo;
  }
}

int launch_mode_gram(const ModeGram& g, cudaStream_t st) {
  const int smem = 2 * MG_CH * MG_LD * (int)sizeof(float);
  cudaFuncSetAttribute(k_mode_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_mode_gram<<<g.d * g.ctas, 256, smem, st>>>(g);
  k_mode_gram_reduce<<<dim3(16, g.d), 256, 0, st>>>(g);
  return 2;
}

int kron_lp(const KronArgs& a) { return (a.la > 4 || a.lb > 4) ? 8 : 4; }

size_t kron_sketch_smem(const KronArgs& a) {
  const int LP = kron_lp(a);
  const size_t fl = 2 * (size_t)a.n1 * (a.n2 + 4) + 2 * (size_t)((a.K + 3) & ~3) + (size_t)a.n2 * LP +
                    (size_t)a.n1 * LP + (size_t)a.ha * a.n1 * LP + (size_t)a.hb * LP * a.n2 + (size_t)a.n1 * LP +
                    (size_t)LP * a.n2;
  return fl * sizeof(float);
}

// Whether the register shares fit: n1, n2 <= 256 and ceil(K / (256 / n)) LP <= 32.
bool kron_shares_fit(const KronArgs& a) {
  const int LP = kron_lp(a);
  if (a.n1 > KS_THREADS || a.n2 > KS_THREADS) return false;
  const int g1 = KS_THREADS / a.n1, g2 = KS_THREADS / a.n2;
  return ((a.K + g1 - 1) / g1) * LP <= KS_Q && ((a.K + g2 - 1) / g2) * LP <= KS_Q;
}

int launch_kron_omega(const KronArgs& a, uint64_t seed, cudaStream_t st) {
  const int64_t b = (a.om_total + 255) / 256;
  k_kron_omega<<<(unsigned)(b < 1024 ? b : 1024), 256, 0, st>>>(a, seed);
  return 1;
}

int launch_kron_sketch(const KronArgs& a, int grid, cudaStream_t st) {
  const size_t smem = kron_sketch_smem(a);
  int n = 0;
  const int64_t bw = (a.S * a.K + 255) / 256;
  k_kron_weights<<<(unsigned)(bw < 8192 ? bw : 8192), 256, 0, st>>>(a);
  ++n;
  if (a.la > 4 || a.lb > 4) {
    cudaFuncSetAttribute(k_kron_sketch<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_kron_sketch<8><<<grid, KS_THREADS, smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_kron_sketch<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_kron_sketch<4><<<grid, KS_THREADS, smem, st>>>(a);
  }
  ++n;
  const int tot = a.n1 * a.K * a.lb + a.n2 * a.K * a.la;
  k_kron_reduce<<<(tot + 255) / 256, 256, 0, st>>>(a, grid);
  ++n;
  if (a.d > 2) {
    int64_t mx = 0;
    for (int m = 0; m < a.d - 2; ++m) mx = std::max<int64_t>(mx, a.n[m] * (int64_t)(a.K / a.ell[m]) * a.la * a.lb);
    const int64_t b = (8 * mx + 255) / 256;
    k_kron_lead<<<(unsigned)(b < 8192 ? b : 8192), 256, 0, st>>>(a);
    ++n;
  }
  return n;
}

int launch_kron_finish(const KronFinish& f, cudaStream_t st) {
  const int64_t b = (f.utotal + 255) / 256;
  k_kron_qw<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(f);
  k_kron_sign<<<(f.rtotal * 32 + 255) / 256, 256, 0, st>>>(f);
  const int64_t bg = (f.gtotal + 255) / 256;
  k_kron_flip_core<<<(unsigned)(bg < 4096 ? bg : 4096), 256, 0, st>>>(f);
  return 3;
}

}  // namespace rt
