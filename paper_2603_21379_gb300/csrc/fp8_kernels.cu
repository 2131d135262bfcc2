// fp8_kernels.cu - packing a tensor into float8 (E4M3) storage with one
// power-of-two scale per slab of its last two modes.
//
// Per slab: amax = max |x|, amax = f 2^e with 0.5 <= f < 1 (e = 0 for an
// all-zero slab); scale = 2^(e - 8); code = nearest E4M3 value to x / scale,
// ties to the even mantissa.  Dividing by a power of two is exact (ldexpf), so
// the rounding decision is taken on the exact quotient.
//
// Three launches: the per-slab maxima (atomicMax on the bit patterns of |x|,
// which order like the values for non-negative floats) into the scale slots,
// the codes (each reads its slab's maximum), and the conversion of the slots
// from maxima to scales.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"

namespace rt {

constexpr int Q8_CHUNK = 4096;   // elements per CTA

__device__ __forceinline__ int slab_exponent(float amax) {
  int e = 0;
  if (amax > 0.f) frexpf(amax, &e);
  return e;
}

__global__ void __launch_bounds__(256) k_fp8_amax(const void* __restrict__ X, int dtype, int64_t slab, int64_t cps,
                                                  unsigned int* __restrict__ amax) {
  const int64_t s = blockIdx.x / cps, c = blockIdx.x % cps;
  const int64_t e0 = c * Q8_CHUNK, e1 = min(slab, e0 + Q8_CHUNK);
  unsigned int m = 0u;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += 256) m = max(m, __float_as_uint(fabsf(load_x(X, dtype, s * slab + e))));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(amax + s, m);
}

__global__ void __launch_bounds__(256) k_fp8_codes(const void* __restrict__ X, int dtype, int64_t slab, int64_t cps,
                                                   const unsigned int* __restrict__ amax,
                                                   unsigned char* __restrict__ q) {
  const int64_t s = blockIdx.x / cps, c = blockIdx.x % cps;
  const int64_t e0 = c * Q8_CHUNK, e1 = min(slab, e0 + Q8_CHUNK);
  const int sh = 8 - slab_exponent(__uint_as_float(amax[s]));
  for (int64_t e = e0 + threadIdx.x; e < e1; e += 256)
    q[s * slab + e] = (unsigned char)e4m3_code(ldexpf(load_x(X, dtype, s * slab + e), sh));
}

__global__ void k_fp8_scales(float* __restrict__ sc, int64_t S) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
    sc[s] = ldexpf(1.f, slab_exponent(sc[s]) - 8);   // the slot holds amax until here
}

int launch_quantize_fp8(const void* X, int dtype, int64_t S, int64_t slab, unsigned char* q, float* scales,
                        cudaStream_t st) {
  const int64_t cps = (slab + Q8_CHUNK - 1) / Q8_CHUNK;
  const int64_t blocks = S * cps;
  if (blocks >= ((int64_t)1 << 31)) return -1;
  if (cudaMemsetAsync(scales, 0, (size_t)S * sizeof(float), st) != cudaSuccess) return -1;
  unsigned int* am = reinterpret_cast<unsigned int*>(scales);
  k_fp8_amax<<<(unsigned)blocks, 256, 0, st>>>(X, dtype, slab, cps, am);
  k_fp8_codes<<<(unsigned)blocks, 256, 0, st>>>(X, dtype, slab, cps, am, q);
  const int64_t b3 = (S + 255) / 256;
  k_fp8_scales<<<(unsigned)(b3 < 4096 ? b3 : 4096), 256, 0, st>>>(scales, S);
  return 3;
}

}  // namespace rt
