// ttm_tc.cu - a one-mode contraction of a float32 intermediate on the tensor cores:
//     out(l, a, b) = sum_{i < n} U[i][a] A(l, i, b)        (a < r, b < R),
// the contractions of the core G = X x_1 U_1^T ... x_d U_d^T (Alg. 1, core step)
// that remain after the tensor-core pass over X has contracted the last two modes.
//
// Per tile (one l, 128 consecutive b) the CTA forms D (128 x 128, float32 in TMEM)
// = A_U B over K = i:
//   A_U  K-major, 128 rows: row 2a + t holds term t (hi, lo) of column a of U as
//        bf16, so that one MMA forms the products of both terms of U at once;
//   B    the tile A(l, :, b0 .. b0 + 127) split into bf16 hi and lo terms, MN-major
//        (b contiguous), 128-byte swizzle;
// two MMAs per 16-row K step (the two terms of B) give all four term products
// (float32-level accuracy, about 2^-16 relative per product, float32 accumulate),
// and out(l, a, b) = D(2a, b) + D(2a + 1, b).
//
// Warps of a CTA (persistent, one per SM, tiles strided by the grid; 12 warps so that
// no SM sub-partition holds more than three and each may use 152 registers):
//   warps 0-7   converters: each thread loads 8 consecutive float32 of 8 rows of the
//               tile with 16-byte loads (the next tile's loads in flight while this
//               one is split), splits them and stores both terms into one of the
//               two B buffers;
//   warps 8-11  epilogue: D from TMEM, the two rows of each a added by a lane-pair
//               shuffle, 16-byte stores of out; warp 8 also allocates the TMEM and
//               its lane 0 issues the MMAs.
// Every mbarrier wait is bounded; on expiry the CTA records the timeout in the
// status word, stops, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rt_common.cuh"
#include "rt_host.h"
#include "tma_util.cuh"
#include "tc_util.cuh"

namespace rt {
namespace tc {
namespace {

using namespace tma;

constexpr int TT_N = 128;                       // b columns per tile (MMA N)
constexpr int TT_K = 128;                       // largest n (MMA K, 8 steps of 16)
constexpr int TT_CONV = 8;                      // converter warps
constexpr int TT_W_EPI0 = TT_CONV;              // warps 0-7 converters, 8-11 epilogue
constexpr int TT_THREADS = (TT_W_EPI0 + 4) * 32;          // 384: three warps per SM sub-partition
constexpr int TT_AU_BYTES = 128 * TT_K * 2;               // A_U: 128 rows x 128 K, bf16
constexpr int TT_TERM = TT_K * TT_N * 2;                  // one term of B: 32 KB
constexpr int TT_NATOM = (TT_K / 8) * 1024;               // bytes between 64-column groups of B
constexpr int TT_TMEM_COLS = 2 * TT_N;                    // two D buffers
constexpr int TT_TASKS = TT_K * (TT_N / 8) / (TT_CONV * 32);   // 8-column chunks per converter thread

constexpr size_t ttm_tc_smem() { return 1024 + TT_AU_BYTES + 4 * (size_t)TT_TERM + 8 * 9 + 16; }

__global__ void __launch_bounds__(TT_THREADS, 1) k_ttm_tc(const float* __restrict__ A, int64_t L, int n, int64_t R,
                                                          const float* __restrict__ U, int r,
                                                          float* __restrict__ out, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* AU = base;
  unsigned char* Bs = AU + TT_AU_BYTES;                    // [2 buffers][2 terms][32 KB]
  uint64_t* bfull = reinterpret_cast<uint64_t*>(Bs + 4 * TT_TERM);
  uint64_t* bempty = bfull + 2;
  uint64_t* dfull = bempty + 2;
  uint64_t* dempty = dfull + 2;
  uint64_t* fin = dempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntb = (R + TT_N - 1) / TT_N;
  const int64_t ntiles = L * ntb;
  const int64_t nmine = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bfull[i], TT_CONV);
      mbar_init(&bempty[i], 1);
      mbar_init(&dfull[i], 1);
      mbar_init(&dempty[i], 4);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A_U: row 2a + t = term t of U(:, a), K-major, swizzled; rows a >= r and i >= n zero.
  // Every load of a thread is issued before the first split (a loop of dependent
  // load-then-store steps would pay the load latency once per element).
  {
    constexpr int PER = (TT_K * 64 + TT_THREADS - 1) / TT_THREADS;
    float uv[PER];
#pragma unroll
    for (int q2 = 0; q2 < PER; ++q2) {
      const int e = threadIdx.x + q2 * TT_THREADS;
      const int i = e / 64, a = e % 64;
      uv[q2] = (e < TT_K * 64 && i < n && a < r) ? __ldg(U + (int64_t)i * r + a) : 0.f;
    }
#pragma unroll
    for (int q2 = 0; q2 < PER; ++q2) {
      const int e = threadIdx.x + q2 * TT_THREADS;
      if (e >= TT_K * 64) break;
      const int i = e / 64, a = e % 64;
      unsigned short hi, lo;
      split1_bf16(uv[q2], hi, lo);
      *reinterpret_cast<unsigned short*>(AU + sw_off16(2 * a, i, 128)) = hi;
      *reinterpret_cast<unsigned short*>(AU + sw_off16(2 * a + 1, i, 128)) = lo;
    }
  }
  if (warp == TT_W_EPI0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"((uint32_t)TT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < TT_W_EPI0) {
    // ---------------------------------------------------------------- converters
    // task q of a tile: row i = e / 16, columns 8 (e % 16) .. + 7 (e = ct + 256 q).  The
    // loads of tile j + 1 are issued before tile j is split and stored (two register
    // sets), so the DRAM latency of one tile overlaps the work on the previous one.
    const int ct = threadIdx.x;                                        // 0 .. 255
    auto load = [&](float4 (&v)[TT_TASKS][2], int64_t j) {
      const int64_t tile = blockIdx.x + j * gridDim.x;
      const int64_t l = tile / ntb, b0 = (tile % ntb) * TT_N;
#pragma unroll
      for (int q = 0; q < TT_TASKS; ++q) {
        const int e = ct + q * (TT_CONV * 32);
        const int i = e >> 4;
        const int64_t b = b0 + (e & 15) * 8;
        v[q][0] = v[q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n) {
          const float* src = A + (l * n + i) * R + b;
          if (b + 4 <= R) v[q][0] = __ldg(reinterpret_cast<const float4*>(src));
          if (b + 8 <= R) v[q][1] = __ldg(reinterpret_cast<const float4*>(src + 4));
        }
      }
    };
    auto store = [&](const float4 (&v)[TT_TASKS][2], int64_t j) -> bool {
      const int buf = (int)(j & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(&bempty[buf], (uint32_t)(((j >> 1) & 1) ^ 1), abort_flag, status)))
        return false;
      unsigned char* hiB = Bs + (buf * 2) * TT_TERM;
      unsigned char* loB = hiB + TT_TERM;
#pragma unroll
      for (int q = 0; q < TT_TASKS; ++q) {
        const int e = ct + q * (TT_CONV * 32);
        const int i = e >> 4, c = (e & 15) * 8;
        uint32_t hi[4], lo[4];
        split_bf16(v[q][0].x, v[q][0].y, hi[0], lo[0]);
        split_bf16(v[q][0].z, v[q][0].w, hi[1], lo[1]);
        split_bf16(v[q][1].x, v[q][1].y, hi[2], lo[2]);
        split_bf16(v[q][1].z, v[q][1].w, hi[3], lo[3]);
        // MN-major, 128-byte swizzle: 64-column groups TT_NATOM apart, 8-row groups
        // 1 KB apart, 16-byte chunk (c % 64) / 8 of row i at chunk ^ (i % 8)
        const int off = (c >> 6) * TT_NATOM + (i >> 3) * 1024 + (i & 7) * 128 + ((((c & 63) >> 3) ^ (i & 7)) << 4);
        *reinterpret_cast<uint4*>(hiB + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(loB + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bfull[buf]);
      return true;
    };
    float4 va[TT_TASKS][2], vb[TT_TASKS][2];
    if (nmine > 0) load(va, 0);
    for (int64_t j = 0; j < nmine; j += 2) {
      if (j + 1 < nmine) load(vb, j + 1);
      if (!store(va, j)) break;
      if (j + 1 >= nmine) break;
      if (j + 2 < nmine) load(va, j + 2);
      if (!store(vb, j + 1)) break;
    }
  } else {
    // ---------------------------------------------------------------- epilogue + issuer
    // D row m in TMEM lane m: warp q holds rows 32 q + lane, i.e. a = 16 q + lane / 2 with
    // the hi term of U in the even lane and the lo term in the odd one; both lanes of a
    // pair form the same sum and each stores half of a 32-column chunk.  Lane 0 of the
    // first epilogue warp also issues the MMAs: the MMAs of tile j, then that warp's part
    // of the epilogue of tile j - 1 while they run.
    const int q = warp & 3;
    const int a = 16 * q + (lane >> 1);
    const int half = (lane & 1) * 16;
    auto issue = [&](int64_t j) -> bool {
      bool ok = true;
      if (lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(128, TT_N) | (1u << 16);   // B MN-major
        const int nk = (n + 15) / 16;                                    // K steps with rows i < n
        const int buf = (int)(j & 1);
        const uint32_t ph = (uint32_t)((j >> 1) & 1);
        ok = mbar_wait(&bfull[buf], ph, abort_flag, status) && mbar_wait(&dempty[buf], ph ^ 1, abort_flag, status);
        if (ok) {
          fence_after();
          const uint32_t dcol = tmem + buf * TT_N;
          for (int kk = 0; kk < nk; ++kk) {
            const uint64_t adesc = sw128_desc(saddr(AU + (kk >> 2) * 128 * 128 + (kk & 3) * 32));
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              const uint32_t baddr = saddr(Bs + (buf * 2 + t) * TT_TERM + kk * 2048);
              mma_bf16_ss(dcol, adesc, mn128_desc(baddr, TT_NATOM, 1024), idesc, (kk | t) ? 1u : 0u);
            }
          }
          mma_commit(&bempty[buf]);
          mma_commit(&dfull[buf]);
        }
      }
      return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    };
    auto epilogue = [&](int64_t j) -> bool {
      const int64_t tile = blockIdx.x + j * gridDim.x;
      const int64_t l = tile / ntb, b0 = (tile % ntb) * TT_N;
      const int buf = (int)(j & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(&dfull[buf], (uint32_t)((j >> 1) & 1), abort_flag, status)))
        return false;
      fence_after();
      if (16 * q < r) {
#pragma unroll 1
        for (int c0 = 0; c0 < TT_N; c0 += 32) {
          uint32_t d[32];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
            tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + buf * TT_N + c0 + cc * 8, d + 8 * cc);
          tmem_wait_ld();
          float w[16];
#pragma unroll
          for (int b = 0; b < 32; ++b) {
            const float x = __uint_as_float(d[b]);
            const float y = x + __shfl_xor_sync(0xffffffffu, x, 1);
            if ((b < 16) == ((lane & 1) == 0)) w[b & 15] = y;
          }
          const int64_t bb = b0 + c0 + half;
          if (a < r) {
            float* o = out + (l * r + a) * R + bb;
#pragma unroll
            for (int u = 0; u < 16; u += 4)
              if (bb + u < R) *reinterpret_cast<float4*>(o + u) = make_float4(w[u], w[u + 1], w[u + 2], w[u + 3]);
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dempty[buf]);
      return true;
    };
    if (warp == TT_W_EPI0) {
      bool ok = true;
      for (int64_t j = 0; j < nmine && ok; ++j) {
        ok = issue(j);
        if (ok && j >= 1) ok = epilogue(j - 1);
      }
      if (ok && nmine >= 1) epilogue(nmine - 1);
      if (lane == 0) {
        mma_commit(fin);
        for (uint32_t it = 0; it < (1u << 20); ++it)
          if (mbar_test(fin, 0)) break;
      }
      __syncwarp();
    } else {
      for (int64_t j = 0; j < nmine; ++j)
        if (!epilogue(j)) break;
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == TT_W_EPI0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TT_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace
}  // namespace tc

// Tensor-core form of the one-mode contraction for float32 A with n <= 128, r <= 64,
// R % 4 == 0 and 16-byte aligned A and out.  Returns the number of launches (1), or 0
// when the shape does not qualify (the caller then uses the FFMA kernels).
int launch_ttm_tc(const float* A, int64_t L, int64_t n, int64_t R, const float* U, int r, float* out, int* status,
                  cudaStream_t st) {
  using namespace tc;
  if (n < 1 || n > TT_K || r < 1 || r > 64 || R < 4 || (R % 4) != 0 || L < 1) return 0;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(out) & 15u)) return 0;
  const int64_t tiles = L * ((R + TT_N - 1) / TT_N);
  if (tiles >= ((int64_t)1 << 31)) return 0;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(tiles, nsm);
  if (cudaFuncSetAttribute(k_ttm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ttm_tc_smem()) != cudaSuccess)
    return 0;
  k_ttm_tc<<<grid, TT_THREADS, ttm_tc_smem(), st>>>(A, L, (int)n, R, U, r, out, status);
  return 1;
}

}  // namespace rt
