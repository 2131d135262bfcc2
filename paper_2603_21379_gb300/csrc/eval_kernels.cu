// eval_kernels.cu - relative reconstruction error ||X - Xhat||_F / ||X||_F of a
// Tucker (Sec. 3, Tucker format) or H-Tucker (Sec. 4, nested bases) result,
// in float64 on the device.  Not part of the decomposition; used to report the
// error the decomposition reached.
//
// Tucker: H = G x_1 U_1 ... x_{d-2} U_{d-2} (float64), then per slab s of the
// leading d-2 modes Xhat_s = U_{d-1} H_s U_d^T, compared with X_s.
// H-Tucker: U_hat(S) = (U_hat(S_l) (x) U_hat(S_r)) B_S^(1)T bottom-up, then
// Xhat = U_hat(R_l) B_R U_hat(R_r)^T tile by tile against X.
// Sums of squares are reduced per CTA and then in a fixed order (deterministic).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "rt_common.cuh"
#include "rt_host.h"

namespace rt {

__device__ __forceinline__ double ldxd(const void* X, int dtype, int64_t e) {
  if (dtype == DT_F32) return (double)__ldg(reinterpret_cast<const float*>(X) + e);
  if (dtype == DT_F8) return (double)e4m3_value(__ldg(reinterpret_cast<const unsigned char*>(X) + e));
  if (dtype == DT_F64) return __ldg(reinterpret_cast<const double*>(X) + e);
  return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[e]);
}

// out(l, i, rho) = sum_a U[i][a] A(l, a, rho); A float64 or float32 (Af)
__global__ void k_expand_f64(const double* __restrict__ A, const float* __restrict__ Af, int64_t L,
                             int r, int64_t R, const float* __restrict__ U, int64_t n,
                             double* __restrict__ out) {
  const int64_t tot = L * n * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rho = e % R, li = e / R;
    const int64_t i = li % n, l = li / n;
    double acc = 0.0;
    for (int a = 0; a < r; ++a) {
      const double av = A ? A[(l * r + a) * R + rho] : (double)Af[(l * r + a) * R + rho];
      acc = fma((double)__ldg(U + i * r + a), av, acc);
    }
    out[e] = acc;
  }
}

// Slab stage: for slab s, T = H_s U_d^T (r1 x n2) in smem, then
// xhat(i, j) = sum_a U_{d-1}[i][a] T[a][j].  Dynamic smem: T[r1 * n2] doubles.
__global__ void __launch_bounds__(256) k_tucker_slab_err(
    const void* __restrict__ X, int dtype, const double* __restrict__ H, const float* __restrict__ Hf,
    int64_t nslab, int64_t n1, int r1, int64_t n2, int r2, const float* __restrict__ U1,
    const float* __restrict__ U2, double* __restrict__ part, const float* __restrict__ xsc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* T = reinterpret_cast<double*>(smem_raw);
  __shared__ double red[64];
  double se = 0.0, sx = 0.0;
  for (int64_t s = blockIdx.x; s < nslab; s += gridDim.x) {
    const double xs = xsc ? (double)__ldg(xsc + s) : 1.0;   // float8 storage: the slab's scale
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)r1 * n2; e += blockDim.x) {
      const int a = (int)(e / n2);
      const int64_t j = e % n2;
      double acc = 0.0;
      for (int b = 0; b < r2; ++b) {
        const int64_t hidx = (s * r1 + a) * r2 + b;
        const double h = H ? H[hidx] : (double)Hf[hidx];
        acc = fma(h, (double)__ldg(U2 + j * r2 + b), acc);
      }
      T[e] = acc;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n1 * n2; e += blockDim.x) {
      const int64_t i = e / n2, j = e % n2;
      double xh = 0.0;
      for (int a = 0; a < r1; ++a) xh = fma((double)__ldg(U1 + i * r1 + a), T[a * n2 + j], xh);
      const double x = ldxd(X, dtype, s * n1 * n2 + e) * xs;
      se = fma(x - xh, x - xh, se);
      sx = fma(x, x, sx);
    }
  }
  se = warp_sum_d(se);
  sx = warp_sum_d(sx);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[w] = se; red[32 + w] = sx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[q]; b += red[32 + q]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_reduce_pairs(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double red[64];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) { a += part[2 * q]; b += part[2 * q + 1]; }
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[w] = a; red[32 + w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { s += red[q]; t += red[32 + q]; }
    out[0] = s;
    out[1] = t;
  }
}

constexpr int EV_BLOCKS = 1216;  // 8 x 152 SMs

// The last two modes per slab in shared memory (r_{d-2} x n_{d-1} doubles), else the
// general form: mode d-2 expanded as well, then the rows of n_{d-1} against U_{d-1}.
static bool relerr_slab_fits(int d, const int64_t* n, const int32_t* r) {
  return (size_t)r[d - 2] * n[d - 1] * 8 <= 200 * 1024;
}

bool tucker_relerr_slab_fits(int d, const int64_t* n, const int32_t* r) { return relerr_slab_fits(d, n, r); }

bool tucker_relerr_supported(int d, const int64_t* n, const int32_t* r) {
  return relerr_slab_fits(d, n, r) || r[d - 1] <= CMAX;
}

// largest expansion buffer (doubles): the leading d-2 modes, and mode d-2 as well in
// the general form
static size_t relerr_half(int d, const int64_t* n, const int32_t* r) {
  size_t cur = 1;
  for (int k = 0; k < d; ++k) cur *= (size_t)r[k];
  size_t best = cur;
  for (int k = 0; k + 2 < d; ++k) {
    cur = cur / (size_t)r[k] * (size_t)n[k];
    if (cur > best) best = cur;
  }
  if (!relerr_slab_fits(d, n, r)) best = std::max(best, cur / (size_t)r[d - 2] * (size_t)n[d - 2]);
  return best;
}

size_t tucker_relerr_scratch(int d, const int64_t* n, const int32_t* r) {
  // two ping-pong buffers for the expansions + per-CTA partials (+ U_{d-1} in float64)
  const size_t extra = relerr_slab_fits(d, n, r) ? 0 : (size_t)n[d - 1] * r[d - 1];
  return 2 * relerr_half(d, n, r) + 2 * EV_BLOCKS + 16 + extra;
}

static int launch_rows_err(const void* X, int dtype, int64_t M, int64_t n2, const double* V, const float* U2,
                           double* U64, int r2, double* part, double* result2, cudaStream_t st);

int launch_tucker_relerr(const void* X, int dtype, int d, const int64_t* n, const int32_t* r,
                         const float* const* U, const float* G, double* scratch, size_t scratch_doubles,
                         double* result2, cudaStream_t st, const float* xsc) {
  (void)scratch_doubles;
  int nl = 0;
  const size_t half = relerr_half(d, n, r);
  double* bufA = scratch;
  double* bufB = scratch + half;
  double* part = scratch + 2 * half;
  const double* H = nullptr;
  const float* Hf = G;
  // expand modes 0 .. d-3 in place order: current tensor (n_0..n_{k-1}, r_k, ..., r_{d-1})
  int64_t L = 1;
  for (int k = 0; k + 2 < d; ++k) {
    int64_t R = 1;
    for (int j = k + 1; j < d; ++j) R *= r[j];
    double* out = (k % 2 == 0) ? bufA : bufB;
    const int64_t tot = L * n[k] * R;
    const unsigned blocks = (unsigned)((tot + 255) / 256 < 65535 * 8 ? (tot + 255) / 256 : 65535 * 8);
    k_expand_f64<<<blocks, 256, 0, st>>>(H, Hf, L, r[k], R, U[k], n[k], out);
    ++nl;
    H = out;
    Hf = nullptr;
    L *= n[k];
  }
  if (!relerr_slab_fits(d, n, r)) {
    double* out = (H == bufA) ? bufB : bufA;
    const int64_t R = r[d - 1], tot = L * n[d - 2] * R;
    const unsigned blocks = (unsigned)((tot + 255) / 256 < 65535 * 8 ? (tot + 255) / 256 : 65535 * 8);
    k_expand_f64<<<blocks, 256, 0, st>>>(H, Hf, L, r[d - 2], R, U[d - 2], n[d - 2], out);
    return nl + 1 + launch_rows_err(X, dtype, L * n[d - 2], n[d - 1], out, U[d - 1], part + 2 * EV_BLOCKS + 16,
                                    r[d - 1], part, result2, st);
  }
  const int64_t n1 = n[d - 2], n2 = n[d - 1];
  const int r1 = r[d - 2], r2 = r[d - 1];
  const size_t smem = (size_t)r1 * n2 * sizeof(double);
  cudaFuncSetAttribute(k_tucker_slab_err, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nb = (int)(L < EV_BLOCKS ? L : EV_BLOCKS);
  k_tucker_slab_err<<<nb, 256, smem, st>>>(X, dtype, H, Hf, L, n1, r1, n2, r2, U[d - 2], U[d - 1], part, xsc);
  k_reduce_pairs<<<1, 1024, 0, st>>>(part, nb, result2);
  return nl + 2;
}

// ---------------------------------------------------------------- H-Tucker
__global__ void k_f32_to_f64(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

int launch_f32_to_f64(const float* in, double* out, int64_t n, cudaStream_t st) {
  const int64_t b = (n + 255) / 256;
  k_f32_to_f64<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(in, out, n);
  return 1;
}

// Uout[(a nr + b)][i] = sum_{j,k} Ul[a][j] B[i][j][k] Ur[b][k]
__global__ void k_ht_expand(const double* __restrict__ Ul, int64_t nl, int rl,
                            const double* __restrict__ Ur, int64_t nr, int rr,
                            const float* __restrict__ B, int rS, double* __restrict__ Uout) {
  const int64_t tot = nl * nr * rS;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rS);
    const int64_t ab = e / rS;
    const int64_t a = ab / nr, b = ab % nr;
    double acc = 0.0;
    for (int j = 0; j < rl; ++j) {
      double t = 0.0;
      for (int k = 0; k < rr; ++k) t = fma((double)B[((int64_t)i * rl + j) * rr + k], Ur[b * rr + k], t);
      acc = fma(Ul[a * rl + j], t, acc);
    }
    Uout[e] = acc;
  }
}

int launch_ht_expand(const double* Ul, int64_t nl, int rl, const double* Ur, int64_t nr, int rr,
                     const float* B, int rS, double* Uout, cudaStream_t st) {
  const int64_t tot = nl * nr * rS;
  const int64_t b = (tot + 255) / 256;
  k_ht_expand<<<(unsigned)(b < 8192 ? b : 8192), 256, 0, st>>>(Ul, nl, rl, Ur, nr, rr, B, rS, Uout);
  return 1;
}

// V = Ul * BR (nl x rr), float64
__global__ void k_ht_v(const double* __restrict__ Ul, int64_t nl, int rl, const float* __restrict__ BR,
                       int rr, double* __restrict__ V) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nl * rr;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / rr;
    const int k = (int)(e % rr);
    double acc = 0.0;
    for (int j = 0; j < rl; ++j) acc = fma(Ul[a * rl + j], (double)BR[j * rr + k], acc);
    V[e] = acc;
  }
}

// xhat(a, b) = sum_k V[a][k] Ur[b][k]; tiles of 32 rows x 256 columns; r_r <= CMAX
constexpr int HE_RA = 32, HE_CB = 256;
__global__ void __launch_bounds__(256) k_ht_err(const void* __restrict__ X, int dtype, int64_t nl, int64_t nr,
                                                const double* __restrict__ V, const double* __restrict__ Ur,
                                                int rr, double* __restrict__ part) {
  __shared__ double Vs[HE_RA * CMAX];
  __shared__ double red[64];
  double se = 0.0, sx = 0.0;
  const int64_t ntr = (nl + HE_RA - 1) / HE_RA, ntc = (nr + HE_CB - 1) / HE_CB;
  for (int64_t t = blockIdx.x; t < ntr * ntc; t += gridDim.x) {
    const int64_t a0 = (t / ntc) * HE_RA, b = (t % ntc) * HE_CB + threadIdx.x;
    __syncthreads();
    for (int e = threadIdx.x; e < HE_RA * rr; e += blockDim.x) {
      const int64_t a = a0 + e / rr;
      Vs[(e / rr) * CMAX + e % rr] = (a < nl) ? V[a * rr + e % rr] : 0.0;
    }
    __syncthreads();
    if (b < nr) {
      double u[CMAX];
      for (int k = 0; k < rr; ++k) u[k] = Ur[b * rr + k];
      for (int ra = 0; ra < HE_RA && a0 + ra < nl; ++ra) {
        double xh = 0.0;
        for (int k = 0; k < rr; ++k) xh = fma(Vs[ra * CMAX + k], u[k], xh);
        const double x = ldxd(X, dtype, (a0 + ra) * nr + b);
        se = fma(x - xh, x - xh, se);
        sx = fma(x, x, sx);
      }
    }
  }
  se = warp_sum_d(se);
  sx = warp_sum_d(sx);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[w] = se; red[32 + w] = sx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[q]; c += red[32 + q]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = c;
  }
}

// err over the M x n2 matrix X against V U2^T (V: M x r2 float64; U2 converted first)
static int launch_rows_err(const void* X, int dtype, int64_t M, int64_t n2, const double* V, const float* U2,
                           double* U64, int r2, double* part, double* result2, cudaStream_t st) {
  const int64_t nu = n2 * r2;
  k_f32_to_f64<<<(unsigned)((nu + 255) / 256 < 4096 ? (nu + 255) / 256 : 4096), 256, 0, st>>>(U2, U64, nu);
  k_ht_err<<<EV_BLOCKS, 256, 0, st>>>(X, dtype, M, n2, V, U64, r2, part);
  k_reduce_pairs<<<1, 1024, 0, st>>>(part, EV_BLOCKS, result2);
  return 3;
}

size_t ht_relerr_scratch(int64_t nl, int64_t nr) { (void)nr; return (size_t)nl * CMAX + 2 * EV_BLOCKS + 16; }

int launch_ht_relerr(const void* X, int dtype, int64_t nl, int64_t nr, const double* Ul, int rl,
                     const float* BR, const double* Ur, int rr, double* scratch, double* result2,
                     cudaStream_t st) {
  double* V = scratch;
  double* part = scratch + (size_t)nl * CMAX;
  k_ht_v<<<1024, 256, 0, st>>>(Ul, nl, rl, BR, rr, V);
  k_ht_err<<<EV_BLOCKS, 256, 0, st>>>(X, dtype, nl, nr, V, Ur, rr, part);
  k_reduce_pairs<<<1, 1024, 0, st>>>(part, EV_BLOCKS, result2);
  return 3;
}

}  // namespace rt
