// rt_rng.cuh - counter-based random streams of the method, device side.
//
// The paper samples s_k fibers uniformly without repetition and draws a
// Gaussian test matrix Omega_k (Sec. 3.1, Alg. 1), but fixes no generator.
// Both are realised here from one published counter-based generator:
//  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
//    (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
//    the key advanced by the Weyl constants before every round but the first;
//  * a 4-round balanced Feistel network on [0, 2^b) (round function: word 0 of
//    one Philox draw on counter (R, t, 0, (1<<16)|node)), restricted to [0, N)
//    by cycle-walking (Black & Rogaway, CT-RSA 2002): pi(j) for j < s are s
//    distinct column indices of X^(S);
//  * Box-Muller: with (u0, u1) the first two words of Philox on counter
//    (m_lo, m_hi, c, (2<<16)|node), a = (u0 + 1/2) 2^-32, b = (u1 + 1/2) 2^-32,
//    Omega(j, c) = sqrt(-2 ln a) cos(2 pi b) for the sampled column m = pi(j).
//    Evaluated in float32: ln a through log1p(-(1-a)) when a > 1/2, where
//    1 - a = (~u0 + 1/2) 2^-32 is formed exactly from the integer, and
//    cos(2 pi b) = -cos(pi (2b - 1)) with 2b - 1 formed from the signed integer
//    u1 - 2^31; the result agrees with the real-valued definition to a few
//    float32 ulps.
#pragma once

#include <stdint.h>

namespace rt {

struct PhiloxKey { uint32_t k0, k1; };

__device__ __forceinline__ PhiloxKey philox_key(uint64_t seed) {
  return PhiloxKey{(uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32)};
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t k0 = k.k0, k1 = k.k1;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// One pass of the keyed Feistel bijection of [0, 2^(2h)).
__device__ __forceinline__ uint64_t feistel(uint64_t x, int h, PhiloxKey key, uint32_t node) {
  const uint64_t hmask = (h >= 64) ? ~0ull : ((1ull << h) - 1ull);
  uint64_t L = x >> h, R = x & hmask;
  const uint32_t w3 = (1u << 16) | node;
#pragma unroll
  for (uint32_t t = 0; t < 4; ++t) {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)R, t, 0u, w3), key);
    const uint64_t nl = R;
    R = L ^ ((uint64_t)o.x & hmask);
    L = nl;
  }
  return (L << h) | R;
}

// pi(j): cycle-walk the Feistel permutation until it lands in [0, N).  The
// walk is a permutation of [0, N) so it always ends; `limit` bounds it anyway
// (exceeding it sets the status word and returns j mod N).
__device__ __forceinline__ uint64_t sample_index(uint64_t j, uint64_t N, int h, PhiloxKey key,
                                                 uint32_t node, int* status) {
  uint64_t y = feistel(j, h, key, node);
  int it = 0;
  const int limit = 1 << 20;
  while (y >= N) {
    y = feistel(y, h, key, node);
    if (++it > limit) {
      set_status(status, ST_TIMEOUT);
      return j % N;
    }
  }
  return y;
}

// N(0,1) entry keyed by (m, col) in stream `stream` (2: the sketch's Omega; 3: the
// per-mode Gaussians of the Kronecker-structured sketch) of node `node`.
__device__ __forceinline__ float gauss_entry(uint64_t m, uint32_t col, PhiloxKey key, uint32_t node,
                                             uint32_t stream = 2u) {
  const uint4 o = philox4x32_10(
      make_uint4((uint32_t)(m & 0xffffffffull), (uint32_t)(m >> 32), col, (stream << 16) | node), key);
  const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
  float lna;
  if (o.x & 0x80000000u) {          // a > 1/2: ln a = log1p(-(1 - a))
    const float t = ((float)(~o.x) + 0.5f) * two_m32;
    lna = log1pf(-t);
  } else {
    lna = logf(((float)o.x + 0.5f) * two_m32);
  }
  const float rad = sqrtf(-2.0f * lna);
  // 2b - 1 = (u1 - 2^31 + 1/2) 2^-31, cos(2 pi b) = -cos(pi (2b - 1))
  const int32_t v = (int32_t)(o.y ^ 0x80000000u);
  const float x = ((float)v + 0.5f) * 4.6566128730773926e-10f;  // 2^-31
  return -rad * cospif(x);
}

}  // namespace rt
