// grad_kernels.cu - kernels of the differentiable Tucker extension: the
// reconstruction Xhat = G x_1 U_1 ... x_d U_d of the Tucker format (Sec. 3),
// fused with the residual R = X - Xhat and its squared norm, and the unfolded
// contractions [Y]_(n) C_(n)^T that turn partial projections into factor
// gradients.  The partial projections themselves are TTM chains
// (core_kernels.cu); the order of the steps is in api.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"

namespace rt {
namespace {

__device__ __forceinline__ float ldx(const void* X, int dtype, int64_t e) {
  if (dtype == DT_F32) return __ldg(reinterpret_cast<const float*>(X) + e);
  if (dtype == DT_F64) return (float)__ldg(reinterpret_cast<const double*>(X) + e);
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[e]);
}

// out(l, i, rho) = sum_a U[i][a] A(l, a, rho): one leading mode of the core expanded.
__global__ void k_expand_f32(const float* __restrict__ A, int64_t L, int r, int64_t R,
                             const float* __restrict__ U, int64_t n, float* __restrict__ out) {
  const int64_t tot = L * n * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rho = e % R, li = e / R;
    const int64_t i = li % n, l = li / n;
    const float* a = A + l * r * R + rho;
    const float* u = U + i * r;
    float acc = 0.f;
    for (int q = 0; q < r; ++q) acc = fmaf(__ldg(u + q), a[(int64_t)q * R], acc);
    out[e] = acc;
  }
}

constexpr int SO_THREADS = 256;

// Per slab s of the leading d-2 modes (H_s = H[s], r1 x r2):
//   out(s, i, j) = alpha X(s, i, j) + beta sum_a U1[i][a] sum_b H_s[a][b] U2[j][b].
// U1 and U2 stay in shared memory, transposed (U1t[a][i], U2t[b][j]), for the whole
// kernel.  Per slab: T = H_s U2^T (r1 x n2) in shared memory, one thread per column
// j computing all r1 entries (U2t read along j, H_s^T as 16-byte broadcasts); then
// out = U1 T by 4 x 4 groups (one 16-byte load of T and one of U1t per a feed 16
// products), X prefetched and out stored as 16-byte accesses on the float32 path.
// part[blockIdx.x] = the CTA's sum of out^2 (float per thread and slab, float64
// across slabs and threads).  X may be null (alpha ignored); out may be null (only
// the sum of squares).  Row and column extents are padded to multiples of 4 (p
// suffix).  Dynamic smem: U1t[r1*n1p] | U2t[r2*n2p] | HsT[r2*r1p] | T[r1*n2p].
__global__ void __launch_bounds__(SO_THREADS) k_tucker_slab_out(
    const void* __restrict__ X, int dtype, float alpha, float beta, const float* __restrict__ H, int64_t nslab,
    int n1, int r1, int n2, int r2, const float* __restrict__ U1, const float* __restrict__ U2,
    float* __restrict__ out, double* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  const int n1p = (n1 + 3) & ~3, n2p = (n2 + 3) & ~3, r1p = (r1 + 3) & ~3;
  float* U1t = sm;                      // [r1][n1p]
  float* U2t = U1t + r1 * n1p;          // [r2][n2p]
  float* HsT = U2t + r2 * n2p;          // [r2][r1p]
  float* T = HsT + r2 * r1p;            // [r1][n2p]
  __shared__ double red[SO_THREADS / 32];
  for (int e = threadIdx.x; e < r1 * n1p; e += SO_THREADS) {
    const int a = e / n1p, i = e % n1p;
    U1t[e] = i < n1 ? U1[i * r1 + a] : 0.f;
  }
  for (int e = threadIdx.x; e < r2 * n2p; e += SO_THREADS) {
    const int b = e / n2p, j = e % n2p;
    U2t[e] = j < n2 ? U2[j * r2 + b] : 0.f;
  }
  // float32 fast path: 16-byte X loads and out stores (n2 % 4 == 0, aligned bases)
  const bool vec = (X == nullptr || dtype == DT_F32) && (n2 % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  const int nrg = n1p / 4, ncg = n2p / 4;
  double sqd = 0.0;
  for (int64_t s = blockIdx.x; s < nslab; s += gridDim.x) {
    __syncthreads();
    for (int e = threadIdx.x; e < r2 * r1p; e += SO_THREADS) {
      const int b = e / r1p, a = e % r1p;
      HsT[e] = a < r1 ? H[(s * r1 + a) * r2 + b] : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n2p; j += SO_THREADS) {
      for (int a0 = 0; a0 < r1; a0 += 4) {
        uint64_t t01 = 0ull, t23 = 0ull;          // (a0, a0 + 1), (a0 + 2, a0 + 3), packed
        for (int b = 0; b < r2; ++b) {
          const float u = U2t[b * n2p + j];
          const uint64_t uu = f2_pack(u, u);
          const float4 hv = *reinterpret_cast<const float4*>(HsT + b * r1p + a0);
          t01 = f2_fma(f2_pack(hv.x, hv.y), uu, t01);
          t23 = f2_fma(f2_pack(hv.z, hv.w), uu, t23);
        }
        float t4[4];
        f2_unpack(t01, t4[0], t4[1]);
        f2_unpack(t23, t4[2], t4[3]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (a0 + q < r1) T[(a0 + q) * n2p + j] = t4[q];
      }
    }
    __syncthreads();
    float sq = 0.f;
    const int64_t base = s * (int64_t)n1 * n2;
    for (int g = threadIdx.x; g < nrg * ncg; g += SO_THREADS) {
      const int rg = g / ncg, cg = g % ncg;
      const int i0 = 4 * rg, j0 = 4 * cg;
      float xv[4][4], acc[4][4];
      uint64_t acc2[4][2];                        // columns (j0, j0 + 1), (j0 + 2, j0 + 3), packed
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        const int64_t e = base + (int64_t)i * n2 + j0;
        if (vec) {
          float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
          if (X && i < n1) f = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(X) + e));
          xv[u][0] = f.x; xv[u][1] = f.y; xv[u][2] = f.z; xv[u][3] = f.w;
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) xv[u][v] = (X && i < n1 && j0 + v < n2) ? ldx(X, dtype, e + v) : 0.f;
        }
        acc2[u][0] = acc2[u][1] = 0ull;
      }
      for (int a = 0; a < r1; ++a) {
        const float4 t = *reinterpret_cast<const float4*>(T + a * n2p + j0);
        const float4 uu = *reinterpret_cast<const float4*>(U1t + a * n1p + i0);
        const float ur[4] = {uu.x, uu.y, uu.z, uu.w};
        const uint64_t t01 = f2_pack(t.x, t.y), t23 = f2_pack(t.z, t.w);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint64_t uw = f2_pack(ur[u], ur[u]);
          acc2[u][0] = f2_fma(uw, t01, acc2[u][0]);
          acc2[u][1] = f2_fma(uw, t23, acc2[u][1]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        f2_unpack(acc2[u][0], acc[u][0], acc[u][1]);
        f2_unpack(acc2[u][1], acc[u][2], acc[u][3]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i >= n1) continue;
        float val[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) val[v] = X ? fmaf(alpha, xv[u][v], beta * acc[u][v]) : beta * acc[u][v];
        const int64_t e = base + (int64_t)i * n2 + j0;
        if (vec) {
          if (out) *reinterpret_cast<float4*>(out + e) = make_float4(val[0], val[1], val[2], val[3]);
#pragma unroll
          for (int v = 0; v < 4; ++v) sq = fmaf(val[v], val[v], sq);
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            if (j0 + v >= n2) continue;
            if (out) out[e + v] = val[v];
            sq = fmaf(val[v], val[v], sq);
          }
        }
      }
    }
    sqd += (double)sq;
  }
  sqd = warp_sum_d(sqd);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sqd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < SO_THREADS / 32; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// General form of the last two modes, for slabs too large for shared memory or too
// few to fill the GPU: Hp = H x_{d-2} U1 is expanded beforehand (M = L n1 rows of
// r2), and here
//   out(l, j) = alpha X(l, j) + beta sum_b Hp[l][b] U2[j][b],   l < M, j < n2.
// Tiles of LO_R rows x LO_J columns; tile g = tj * ntr + tr, so that a CTA walking
// g, g + gridDim.x, ... keeps its column chunk of U2 (transposed in shared memory,
// reloaded only when tj changes) over many row tiles.  Thread (rh, j): column j of
// the chunk for LO_R / 2 rows.  part[blockIdx.x] = the CTA's sum of out^2 (float
// per thread and tile, float64 across tiles and threads).
constexpr int LO_THREADS = 256, LO_J = 128, LO_R = 32, LO_RT = LO_R / (LO_THREADS / LO_J);
constexpr int LO_LDU = LO_J + 1;     // odd stride: the transposing store is conflict-free
__global__ void __launch_bounds__(LO_THREADS) k_last_out(const void* __restrict__ X, int dtype, float alpha,
                                                         float beta, const float* __restrict__ Hp, int64_t M,
                                                         int r2, int64_t n2, const float* __restrict__ U2,
                                                         float* __restrict__ out, double* __restrict__ part) {
  __shared__ float U2t[CMAX * LO_LDU];               // [b][jj]
  __shared__ __align__(16) float Hs[LO_R * CMAX];    // [row][b]
  __shared__ double red[LO_THREADS / 32];
  const int64_t ntr = (M + LO_R - 1) / LO_R, ntj = (n2 + LO_J - 1) / LO_J;
  const int jj = threadIdx.x % LO_J, rh = threadIdx.x / LO_J;
  int64_t cur_tj = -1;
  double sqd = 0.0;
  for (int64_t g = blockIdx.x; g < ntr * ntj; g += gridDim.x) {
    const int64_t tj = g / ntr, tr = g % ntr;
    const int64_t j0 = tj * LO_J, l0 = tr * LO_R;
    __syncthreads();
    if (tj != cur_tj) {
      for (int e = threadIdx.x; e < r2 * LO_J; e += LO_THREADS) {
        const int b = e % r2, c = e / r2;     // consecutive threads read consecutive b of row j0 + c
        U2t[b * LO_LDU + c] = (j0 + c < n2) ? __ldg(U2 + (j0 + c) * r2 + b) : 0.f;
      }
      cur_tj = tj;
    }
    for (int e = threadIdx.x; e < LO_R * r2; e += LO_THREADS) {
      const int rr = e / r2, b = e % r2;
      Hs[rr * CMAX + b] = (l0 + rr < M) ? Hp[(l0 + rr) * r2 + b] : 0.f;
    }
    __syncthreads();
    float acc[LO_RT];
#pragma unroll
    for (int u = 0; u < LO_RT; ++u) acc[u] = 0.f;
    const float* hrow = Hs + rh * LO_RT * CMAX;
    for (int b = 0; b < r2; ++b) {
      const float u2 = U2t[b * LO_LDU + jj];
#pragma unroll
      for (int u = 0; u < LO_RT; ++u) acc[u] = fmaf(hrow[u * CMAX + b], u2, acc[u]);
    }
    const int64_t j = j0 + jj;
    float sq = 0.f;
    if (j < n2) {
#pragma unroll
      for (int u = 0; u < LO_RT; ++u) {
        const int64_t l = l0 + rh * LO_RT + u;
        if (l >= M) break;
        const int64_t e = l * n2 + j;
        const float val = X ? fmaf(alpha, ldx(X, dtype, e), beta * acc[u]) : beta * acc[u];
        if (out) out[e] = val;
        sq = fmaf(val, val, sq);
      }
    }
    sqd += (double)sq;
  }
  sqd = warp_sum_d(sqd);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sqd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < LO_THREADS / 32; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// out[0] = scale * sum of part[0..nblk) in a fixed order.
__global__ void k_sum_parts(const double* __restrict__ part, int nblk, double scale, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) a += part[q];
  a = warp_sum_d(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    out[0] = scale * t;
  }
}

// out[i][a] = scale * sum_{p, q} Y(p, i, q) C(p, a, q) for Y of (P, n, Q) and C of
// (P, r, Q): the mode-n unfoldings' product [Y]_(n) [C]_(n)^T.  CTA (ib, ks) takes
// rows ib*UC_ROWS .. + UC_ROWS and the ks-th chunk of UC_K terms k = p Q + q: the
// chunk of C (UC_K x r) is staged in shared memory once and serves all its rows;
// thread (row, k-lane) keeps r <= 64 partial sums over its terms, reduced across
// the k-lanes of the row into part[i][ks][a]; k_unfold_reduce adds the chunks in
// order (deterministic).
constexpr int UC_THREADS = 256, UC_K = 128, UC_ROWS = 8, UC_LANES = UC_THREADS / UC_ROWS;
__global__ void __launch_bounds__(UC_THREADS) k_unfold_contract(const float* __restrict__ Y,
                                                                const float* __restrict__ C, int64_t P,
                                                                int64_t n, int r, int64_t Q,
                                                                float* __restrict__ part) {
  __shared__ __align__(16) float cs[CMAX * UC_K];    // [a][kk]
  const int KS = gridDim.y;
  const int64_t K = P * Q, nchunk = (K + UC_K - 1) / UC_K;
  const int row = threadIdx.x / UC_LANES, kl = threadIdx.x % UC_LANES;
  const int64_t i = (int64_t)blockIdx.x * UC_ROWS + row;
  float acc[CMAX];
#pragma unroll
  for (int a = 0; a < CMAX; ++a) acc[a] = 0.f;
  for (int64_t ch = blockIdx.y; ch < nchunk; ch += KS) {   // chunks ks, ks + KS, ...
    const int64_t k0 = ch * UC_K;
    const int kn = (int)min((int64_t)UC_K, K - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kn * r; e += UC_THREADS) {
      // C(p, a, q) for k = k0 + kk: consecutive threads take consecutive q (then a)
      const int kk = e % kn, a = e / kn;
      const int64_t k = k0 + kk, p = k / Q, q = k % Q;
      cs[a * UC_K + kk] = C[(p * r + a) * Q + q];
    }
    __syncthreads();
    if (i < n) {
      for (int kk = kl; kk < kn; kk += UC_LANES) {
        const int64_t k = k0 + kk, p = k / Q, q = k % Q;
        const float y = __ldg(Y + (p * n + i) * Q + q);
        const float* c = cs + kk;
#pragma unroll
        for (int a = 0; a < CMAX; ++a)
          if (a < r) acc[a] = fmaf(y, c[a * UC_K], acc[a]);
      }
    }
  }
  const int ks = blockIdx.y;
  // the UC_LANES (= 32) k-lanes of a row are one warp
#pragma unroll
  for (int a = 0; a < CMAX; ++a) {
    if (a >= r) break;
    const float v = warp_sum(acc[a]);
    if (kl == 0 && i < n) part[(i * KS + ks) * r + a] = v;
  }
}

__global__ void k_unfold_reduce(const float* __restrict__ part, int64_t n, int r, int KS, float scale,
                                float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * r) return;
  const int64_t i = t / r;
  const int a = (int)(t % r);
  float s = 0.f;
  for (int ks = 0; ks < KS; ++ks) s += part[(i * KS + ks) * r + a];
  out[t] = scale * s;
}

__global__ void k_scale_f32(float* __restrict__ x, int64_t n, float s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] *= s;
}

unsigned grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 65535 * 16 ? (b > 0 ? b : 1) : 65535 * 16);
}

}  // namespace

constexpr int GR_SLAB_BLOCKS = 1216;   // 8 x 152 SMs

size_t expand_partial_doubles() { return GR_SLAB_BLOCKS + 8; }

int launch_expand_f32(const float* A, int64_t L, int r, int64_t R, const float* U, int64_t n, float* out,
                      cudaStream_t st) {
  k_expand_f32<<<grid_for(L * n * R, 256), 256, 0, st>>>(A, L, r, R, U, n, out);
  return 1;
}

int launch_tucker_slab_out(const void* X, int dtype, float alpha, float beta, const float* H, int64_t nslab,
                           int64_t n1, int r1, int64_t n2, int r2, const float* U1, const float* U2, float* out,
                           double* part, double* sumsq_scaled, double scale, cudaStream_t st) {
  if (!slab_out_fits(n1, r1, n2, r2)) return 0;
  const int64_t n1p = (n1 + 3) & ~(int64_t)3, n2p = (n2 + 3) & ~(int64_t)3, r1p = (r1 + 3) & ~3;
  const size_t smem = (size_t)(r1 * n1p + r2 * n2p + r2 * r1p + r1 * n2p) * 4;
  cudaFuncSetAttribute(k_tucker_slab_out, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nb = (int)(nslab < GR_SLAB_BLOCKS ? nslab : GR_SLAB_BLOCKS);
  k_tucker_slab_out<<<nb, SO_THREADS, smem, st>>>(X, dtype, alpha, beta, H, nslab, (int)n1, r1, (int)n2, r2, U1,
                                                   U2, out, part);
  int nl = 1;
  if (sumsq_scaled) {
    k_sum_parts<<<1, 1024, 0, st>>>(part, nb, scale, sumsq_scaled);
    ++nl;
  }
  return nl;
}

bool slab_out_fits(int64_t n1, int r1, int64_t n2, int r2) {
  if (n1 > 65536 || n2 > 65536) return false;
  const int64_t n1p = (n1 + 3) & ~(int64_t)3, n2p = (n2 + 3) & ~(int64_t)3, r1p = (r1 + 3) & ~3;
  return (r1 * n1p + r2 * n2p + r2 * r1p + r1 * n2p) * 4 <= 200 * 1024;
}

bool last_modes_general(int64_t L, int64_t n1, int r1, int64_t n2, int r2) {
  return !slab_out_fits(n1, r1, n2, r2) || (L < GR_SLAB_BLOCKS / 8 && n1 * n2 > 65536);
}

int launch_last_out(const void* X, int dtype, float alpha, float beta, const float* Hp, int64_t M, int r2,
                    int64_t n2, const float* U2, float* out, double* part, double* sumsq_scaled, double scale,
                    cudaStream_t st) {
  if (r2 < 1 || r2 > CMAX || M < 1 || n2 < 1) return 0;
  const int64_t tiles = ((M + LO_R - 1) / LO_R) * ((n2 + LO_J - 1) / LO_J);
  const int nb = (int)(tiles < GR_SLAB_BLOCKS ? tiles : GR_SLAB_BLOCKS);
  k_last_out<<<nb, LO_THREADS, 0, st>>>(X, dtype, alpha, beta, Hp, M, r2, n2, U2, out, part);
  int nl = 1;
  if (sumsq_scaled) {
    k_sum_parts<<<1, 1024, 0, st>>>(part, nb, scale, sumsq_scaled);
    ++nl;
  }
  return nl;
}

constexpr int UC_MAX_SPLIT = 4096;   // CTAs per row group along K

size_t unfold_scratch_floats(int64_t n, int r, int64_t K) {
  const int64_t ks = (K + UC_K - 1) / UC_K;
  return (size_t)n * (ks < UC_MAX_SPLIT ? ks : UC_MAX_SPLIT) * r;
}

int launch_unfold_contract(const float* Y, const float* C, int64_t P, int64_t n, int r, int64_t Q, float scale,
                           float* out, float* scratch, cudaStream_t st) {
  if (r > CMAX || n < 1 || n > (int64_t)0x7fffffff) return 0;
  const int64_t K = P * Q;
  int64_t KS = (K + UC_K - 1) / UC_K;
  if (KS > UC_MAX_SPLIT) KS = UC_MAX_SPLIT;     // a CTA then takes every KS-th chunk
  k_unfold_contract<<<dim3((unsigned)((n + UC_ROWS - 1) / UC_ROWS), (unsigned)KS), UC_THREADS, 0, st>>>(
      Y, C, P, n, r, Q, scratch);
  k_unfold_reduce<<<grid_for(n * r, 256), 256, 0, st>>>(scratch, n, r, (int)KS, scale, out);
  return 2;
}

int launch_scale_f32(float* x, int64_t n, float s, cudaStream_t st) {
  k_scale_f32<<<grid_for(n, 256), 256, 0, st>>>(x, n, s);
  return 1;
}

}  // namespace rt
