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
constexpr int SO_TR = 32, SO_TC = 64;            // output tile: 32 rows x 64 columns, 2 x 4 per thread

// Per slab s of the leading d-2 modes (H_s = H[s], r1 x r2):
//   out(s, i, j) = alpha X(s, i, j) + beta sum_a U1[i][a] sum_b H_s[a][b] U2[j][b].
// U1 and U2 (transposed) stay in shared memory for the whole kernel; per slab T = H_s U2^T
// (r1 x n2) goes to shared memory, then out = U1 T by 32 x 64 tiles, each thread a
// 2 x 4 register tile (rows ty + 16 u, columns 4 tx .. + 3), T read as float4.
// part[blockIdx.x] = the CTA's sum of out^2 (float per thread and slab, float64
// across slabs and threads).  X may be null (alpha ignored); out may be null (only
// the sum of squares).  Dynamic smem: U1[n1*r1] | U2^T[r2*n2] | H_s[r1*r2] | T[r1*n2p],
// n2p = n2 rounded up to a multiple of SO_TC.
__global__ void __launch_bounds__(SO_THREADS) k_tucker_slab_out(
    const void* __restrict__ X, int dtype, float alpha, float beta, const float* __restrict__ H, int64_t nslab,
    int n1, int r1, int n2, int r2, const float* __restrict__ U1, const float* __restrict__ U2,
    float* __restrict__ out, double* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  const int n2p = (n2 + SO_TC - 1) / SO_TC * SO_TC;
  float* U1s = sm;
  float* U2s = U1s + ((n1 * r1 + 3) & ~3);
  float* Hs = U2s + ((n2 * r2 + 3) & ~3);
  float* T = Hs + ((r1 * r2 + 3) & ~3);
  __shared__ double red[SO_THREADS / 32];
  for (int e = threadIdx.x; e < n1 * r1; e += SO_THREADS) U1s[e] = U1[e];
  // U2 transposed (U2s[b][j]): the T products below read it along j, conflict-free
  for (int e = threadIdx.x; e < n2 * r2; e += SO_THREADS) U2s[(e % r2) * n2 + e / r2] = U2[e];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  // float32 fast path: 16-byte X loads and out stores (rows of n2 % 4 == 0 floats,
  // 16-byte aligned bases; column groups of 4 never straddle n2)
  const bool vec = (X == nullptr || dtype == DT_F32) && (n2 % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  double sqd = 0.0;
  for (int64_t s = blockIdx.x; s < nslab; s += gridDim.x) {
    __syncthreads();
    for (int e = threadIdx.x; e < r1 * r2; e += SO_THREADS) Hs[e] = H[s * r1 * r2 + e];
    __syncthreads();
    for (int e = threadIdx.x; e < r1 * n2p; e += SO_THREADS) {
      const int a = e / n2p, j = e % n2p;
      float acc = 0.f;
      if (j < n2)
        for (int b = 0; b < r2; ++b) acc = fmaf(Hs[a * r2 + b], U2s[b * n2 + j], acc);
      T[e] = acc;
    }
    __syncthreads();
    float sq = 0.f;
    const int64_t base = s * (int64_t)n1 * n2;
    for (int i0 = 0; i0 < n1; i0 += SO_TR) {
      for (int j0 = 0; j0 < n2; j0 += SO_TC) {
        float acc[2][4], xv[2][4];
        const int ia = i0 + ty, ib = i0 + ty + 16;
        const int ja = ia < n1 ? ia : 0, jb = ib < n1 ? ib : 0;
        // X of the thread's 2 x 4 outputs, loaded before the products so that the
        // DRAM latency overlaps them (16-byte loads on the float32 fast path)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int i = u ? ib : ia;
          const int j = j0 + 4 * tx;
          const int64_t e = base + (int64_t)i * n2 + j;
          if (vec) {
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (X && i < n1 && j < n2) f = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(X) + e));
            xv[u][0] = f.x; xv[u][1] = f.y; xv[u][2] = f.z; xv[u][3] = f.w;
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) xv[u][v] = (X && i < n1 && j + v < n2) ? ldx(X, dtype, e + v) : 0.f;
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        }
        for (int a = 0; a < r1; ++a) {
          const float4 t = *reinterpret_cast<const float4*>(T + a * n2p + j0 + 4 * tx);
          const float ua = U1s[ja * r1 + a], ub = U1s[jb * r1 + a];
          acc[0][0] = fmaf(ua, t.x, acc[0][0]); acc[0][1] = fmaf(ua, t.y, acc[0][1]);
          acc[0][2] = fmaf(ua, t.z, acc[0][2]); acc[0][3] = fmaf(ua, t.w, acc[0][3]);
          acc[1][0] = fmaf(ub, t.x, acc[1][0]); acc[1][1] = fmaf(ub, t.y, acc[1][1]);
          acc[1][2] = fmaf(ub, t.z, acc[1][2]); acc[1][3] = fmaf(ub, t.w, acc[1][3]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int i = u ? ib : ia;
          if (i >= n1) continue;
          float val[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) val[v] = X ? fmaf(alpha, xv[u][v], beta * acc[u][v]) : beta * acc[u][v];
          const int j = j0 + 4 * tx;
          const int64_t e = base + (int64_t)i * n2 + j;
          if (vec && j < n2) {
            if (out) *reinterpret_cast<float4*>(out + e) = make_float4(val[0], val[1], val[2], val[3]);
#pragma unroll
            for (int v = 0; v < 4; ++v) sq = fmaf(val[v], val[v], sq);
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              if (j + v >= n2) continue;
              if (out) out[e + v] = val[v];
              sq = fmaf(val[v], val[v], sq);
            }
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
// (P, r, Q): the mode-n unfoldings' product [Y]_(n) [C]_(n)^T.  CTA (i, ks) takes
// the ks-th chunk of the P Q terms (q fastest, so Y and C are read along q); its
// threads keep r <= 64 partial sums, reduced across the CTA into part[i][ks][a];
// k_unfold_reduce then adds the chunks in order (deterministic).
constexpr int UC_THREADS = 256;
__global__ void __launch_bounds__(UC_THREADS) k_unfold_contract(const float* __restrict__ Y,
                                                                const float* __restrict__ C, int64_t P,
                                                                int64_t n, int r, int64_t Q, int64_t kchunk,
                                                                float* __restrict__ part) {
  __shared__ float red[UC_THREADS / 32][CMAX];
  const int64_t i = blockIdx.x;
  const int ks = blockIdx.y, KS = gridDim.y;
  float acc[CMAX];
#pragma unroll
  for (int a = 0; a < CMAX; ++a) acc[a] = 0.f;
  const int64_t K = P * Q;
  const int64_t k1 = min(K, (int64_t)(ks + 1) * kchunk);
  for (int64_t k = (int64_t)ks * kchunk + threadIdx.x; k < k1; k += UC_THREADS) {
    const int64_t p = k / Q, q = k % Q;
    const float y = __ldg(Y + (p * n + i) * Q + q);
    const float* c = C + p * r * Q + q;
#pragma unroll
    for (int a = 0; a < CMAX; ++a)
      if (a < r) acc[a] = fmaf(y, __ldg(c + (int64_t)a * Q), acc[a]);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < CMAX; ++a) {
    if (a >= r) break;
    const float v = warp_sum(acc[a]);
    if (lane == 0) red[w][a] = v;
  }
  __syncthreads();
  if (threadIdx.x < r) {
    float t = 0.f;
    for (int q = 0; q < UC_THREADS / 32; ++q) t += red[q][threadIdx.x];
    part[(i * KS + ks) * r + threadIdx.x] = t;
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
  if (n1 > 4096 || n2 > 4096) return 0;
  const int64_t n2p = (n2 + SO_TC - 1) / SO_TC * SO_TC;
  auto up4 = [](int64_t x) { return (x + 3) & ~(int64_t)3; };
  const size_t smem = (size_t)(up4(n1 * r1) + up4(n2 * r2) + up4((int64_t)r1 * r2) + (int64_t)r1 * n2p) * 4;
  if (smem > 200 * 1024) return 0;
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

constexpr int UC_MAX_SPLIT = 64;

size_t unfold_scratch_floats(int64_t n, int r) { return (size_t)n * UC_MAX_SPLIT * r; }

int launch_unfold_contract(const float* Y, const float* C, int64_t P, int64_t n, int r, int64_t Q, float scale,
                           float* out, float* scratch, cudaStream_t st) {
  if (r > CMAX || n < 1 || n > (int64_t)0x7fffffff) return 0;
  const int64_t K = P * Q;
  int64_t KS = (K + 2047) / 2048;                  // about 8 terms per thread per chunk
  if (KS < 1) KS = 1;
  if (KS > UC_MAX_SPLIT) KS = UC_MAX_SPLIT;
  const int64_t kchunk = (K + KS - 1) / KS;
  k_unfold_contract<<<dim3((unsigned)n, (unsigned)KS), UC_THREADS, 0, st>>>(Y, C, P, n, r, Q, kchunk, scratch);
  k_unfold_reduce<<<grid_for(n * r, 256), 256, 0, st>>>(scratch, n, r, (int)KS, scale, out);
  return 2;
}

int launch_scale_f32(float* x, int64_t n, float s, cudaStream_t st) {
  k_scale_f32<<<grid_for(n, 256), 256, 0, st>>>(x, n, s);
  return 1;
}

}  // namespace rt
