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

// Slab s of X into Ms (n1 rows, padded stride ld): 16-byte cp.async for float32 X,
// element loads otherwise.
__device__ __forceinline__ void load_slab(const KronArgs& a, int64_t s, float* Ms, int ld) {
  const int n1 = a.n1, n2 = a.n2, nq = n2 >> 2;
  if (a.dtype == DT_F32) {
    const float* src = static_cast<const float*>(a.X) + s * (int64_t)n1 * n2;
    for (int e = threadIdx.x; e < n1 * nq; e += KS_THREADS) {
      const int i = e / nq, q = e % nq;
      cp_async16(Ms + i * ld + 4 * q, src + (int64_t)i * n2 + 4 * q);
    }
  } else {
    for (int e = threadIdx.x; e < n1 * n2; e += KS_THREADS) {
      const int i = e / n2, j = e % n2;
      Ms[i * ld + j] = load_x(a.X, a.dtype, (s * n1 + i) * (int64_t)n2 + j);
    }
  }
}

// Dynamic smem (floats): Ms[2][n1][ld] | Ob[n2][LP] | Oa[n1][LP] | Ap[HA][n1][LP] |
// Bp[HB][LP][n2] | Af[n1][LP] | Btf[LP][n2] | w[K]
template <int LP>
__global__ void __launch_bounds__(KS_THREADS, 1) k_kron_sketch(KronArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int n1 = a.n1, n2 = a.n2, la = a.la, lb = a.lb, K = a.K;
  const int ld = n2 + 4, nq = n2 >> 2;
  const int HA = a.ha, HB = a.hb;
  float* Ms0 = sm;
  float* Ob = Ms0 + 2 * n1 * ld;
  float* Oa = Ob + n2 * LP;
  float* Ap = Oa + n1 * LP;
  float* Bp = Ap + HA * n1 * LP;
  float* Af = Bp + HB * LP * n2;
  float* Btf = Af + n1 * LP;
  float* w = Btf + LP * n2;
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
  float z1[KS_Q], z2[KS_Q];
#pragma unroll
  for (int q = 0; q < KS_Q; ++q) { z1[q] = 0.f; z2[q] = 0.f; }
  const int tot1 = n1 * K * lb, tot2 = n2 * K * la;
  const int cwq = (nq + HA - 1) / HA;          // float4 columns per chunk of A
  const int rh = (n1 + HB - 1) / HB;           // rows per chunk of Bt
  const int64_t S = a.S;
  int64_t s = blockIdx.x;
  if (s < S) load_slab(a, s, Ms0, ld);
  cp_async_commit();
  for (int64_t t = 0; s < S; ++t, s += gridDim.x) {
    float* Ms = Ms0 + (t & 1) * n1 * ld;
    const int64_t sn = s + gridDim.x;
    if (sn < S) load_slab(a, sn, Ms0 + ((t + 1) & 1) * n1 * ld, ld);
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
    // A, Bt (partials summed in chunk order) and the slab's Kronecker weights
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
    for (int kap = tid; kap < K; kap += KS_THREADS) {
      float v = 1.f;
      int64_t rs = s;
      int rk = kap;
      for (int j = a.d - 3; j >= 0; --j) {     // leading modes, last fastest
        const int64_t ij = rs % a.n[j];
        rs /= a.n[j];
        const int aj = rk % a.ell[j];
        rk /= a.ell[j];
        v *= __ldg(a.om + a.om_off[j] + ij * a.ell[j] + aj);
      }
      w[kap] = v;
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
    // this CTA's shares of Z_{d-2} and Z_{d-1}
#pragma unroll
    for (int q = 0; q < KS_Q; ++q) {
      const int e1 = tid + q * KS_THREADS;
      if (e1 < tot1) {
        const int i = e1 / (K * lb), rem = e1 % (K * lb);
        z1[q] = fmaf(w[rem / lb], Af[i * LP + rem % lb], z1[q]);
      }
      const int e2 = tid + q * KS_THREADS;
      if (e2 < tot2) {
        const int j = e2 / (K * la), rem = e2 % (K * la);
        z2[q] = fmaf(w[rem / la], Btf[(rem % la) * n2 + j], z2[q]);
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
#pragma unroll
  for (int q = 0; q < KS_Q; ++q) {
    const int e1 = tid + q * KS_THREADS;
    if (e1 < tot1) a.part1[(int64_t)blockIdx.x * tot1 + e1] = z1[q];
    const int e2 = tid + q * KS_THREADS;
    if (e2 < tot2) a.part2[(int64_t)blockIdx.x * tot2 + e2] = z2[q];
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

// Z_m for the leading modes m < d-2 from the slabs' T_s: one thread per entry
// (i_m, (kappa', a, b)), a sum over the S / n_m slabs with that i_m.
__global__ void k_kron_lead(KronArgs a) {
  const int nl = a.d - 2, lab = a.la * a.lb;
  for (int m = 0; m < nl; ++m) {
    const int Km = a.K / a.ell[m];
    const int64_t rows = a.n[m], cols = (int64_t)Km * lab, tot = rows * cols;
    const int64_t inner = a.S / a.n[m];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t im = e / cols;
      const int col = (int)(e % cols);
      const int kp = col / lab, ab = col % lab;
      float acc = 0.f;
      for (int64_t t = 0; t < inner; ++t) {
        // leading multi-index with i_m fixed, the others from t (C order), and the
        // Kronecker weight of the other leading modes' columns from kappa'
        int64_t rt = t, s = 0, stride = 1;
        int rk = kp;
        float wv = 1.f;
        for (int j = nl - 1; j >= 0; --j) {
          int64_t ij;
          if (j == m) {
            ij = im;
          } else {
            ij = rt % a.n[j];
            rt /= a.n[j];
            const int aj = rk % a.ell[j];
            rk /= a.ell[j];
            wv *= __ldg(a.om + a.om_off[j] + ij * a.ell[j] + aj);
          }
          s += ij * stride;
          stride *= a.n[j];
        }
        acc = fmaf(wv, __ldg(a.Ts + s * lab + ab), acc);
      }
      a.z[m][e] = acc;
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

size_t kron_sketch_smem(const KronArgs& a) {
  const int LP = (a.la > 4 || a.lb > 4) ? 8 : 4;
  const size_t fl = 2 * (size_t)a.n1 * (a.n2 + 4) + (size_t)a.n2 * LP + (size_t)a.n1 * LP +
                    (size_t)a.ha * a.n1 * LP + (size_t)a.hb * LP * a.n2 + (size_t)a.n1 * LP + (size_t)LP * a.n2 + a.K;
  return fl * sizeof(float);
}

int launch_kron_omega(const KronArgs& a, uint64_t seed, cudaStream_t st) {
  const int64_t b = (a.om_total + 255) / 256;
  k_kron_omega<<<(unsigned)(b < 1024 ? b : 1024), 256, 0, st>>>(a, seed);
  return 1;
}

int launch_kron_sketch(const KronArgs& a, int grid, cudaStream_t st) {
  const size_t smem = kron_sketch_smem(a);
  int n = 0;
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
    const int64_t b = (mx + 255) / 256;
    k_kron_lead<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(a);
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
