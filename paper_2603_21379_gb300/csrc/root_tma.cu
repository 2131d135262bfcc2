// root_tma.cu - the root pass of Sub-R-RtL-HT (Alg. 2, root transfer tensor),
//     B_R(0, j, k) = sum_{a, b} U_l(a, j) X(a, b) U_r(b, k),
// X = X^(R_l) the n_l x n_r matricization of the whole tensor (row-major), as
// one streaming read of X:
//
//   k_root_rows   T(a, k) = sum_b X(a, b) U_r(b, k) for every row a.
//                 Persistent, two CTAs per SM.  In each CTA a producer warp
//                 streams 64-row x 32-column boxes of X (TMA, 128-byte swizzle)
//                 and the matching 32 x r_r rows of U_r (bulk copy) through a
//                 ring of RS_NS shared-memory stages; four consumer warps own the
//                 64 rows of the current block, each thread 4 rows x 4 columns of
//                 every stage (so one read of its 4 x r_r slice of U_r serves 4
//                 rows), accumulating 16 stages (64 products) in registers and
//                 adding those partials into a running total (two-level sum:
//                 worst-case relative error about (64 + nst / 16) u of the sum
//                 of |terms|; Kahan compensation at the second level cost 18 %
//                 of the pass for no visible change in B_R).  Each warp holds half of the
//                 columns of 32 rows; at the end of the block its 4 column groups
//                 are combined with warp shuffles and the half is written to T.
//   k_root_left   per CTA of 256 rows: sum_a U_l(a, j) T(a, k).
//   k_root_reduce (ht_kernels.cu): fixed-order float64 sum of the partials.
//
// The bytes that count are X's (17.2 GB for the 16^8 tensor): U_r (n_r r_r
// floats) is re-read from L2 once per 64-row block, T (two column halves) and
// the partials are 2 n_l r_r and (n_l / 256) r_l r_r floats.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rt_common.cuh"
#include "rt_host.h"
#include "tma_util.cuh"

namespace rt {
namespace {

using namespace tma;


constexpr int RS_ROWS = 64;                  // rows of X per work item
constexpr int RS_COLS = 32;                  // columns per stage (128 bytes of float32)
constexpr int RS_NS = 8;                     // stages in the ring (8 KB of X each)
constexpr int RS_CONS = 4;                   // consumer warps
constexpr int RS_THREADS = (RS_CONS + 1) * 32;
constexpr int RS_CTAS_PER_SM = 2;
constexpr int RS_XBYTES = RS_ROWS * RS_COLS * 4;
constexpr int RS_UMAX = 12;                  // largest r_r
constexpr int RS_UBYTES = RS_COLS * RS_UMAX * 4;

constexpr int RS_FOLD = 16;                  // stages summed in registers before the running total
constexpr int RL_ROWS = 256;                 // rows per CTA of k_root_left

constexpr size_t rs_smem() { return 1024 + (size_t)RS_NS * (RS_XBYTES + RS_UBYTES) + 8 * (2 * RS_NS) + 16; }

template <int RR>
__global__ void __launch_bounds__(RS_THREADS, RS_CTAS_PER_SM) k_root_rows(const __grid_constant__ CUtensorMap tmap,
                                                             const float* __restrict__ Ur, int64_t nl, int64_t nr,
                                                             float* __restrict__ T, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xs = base;                                   // [RS_NS][64 rows][128 B], swizzled
  float* us = reinterpret_cast<float*>(base + RS_NS * RS_XBYTES);  // [RS_NS][32][RE]
  uint64_t* full = reinterpret_cast<uint64_t*>(base + RS_NS * (RS_XBYTES + RS_UBYTES));
  uint64_t* empty = full + RS_NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + RS_NS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nitems = (nl + RS_ROWS - 1) / RS_ROWS;
  const int64_t nst = nr / RS_COLS;        // stages per item (nr: columns padded to a multiple of 32)
  constexpr int RE = RR + (RR & 1), RP = RE / 2;   // U_r columns padded to pairs
  const uint32_t ubytes = (uint32_t)(RS_COLS * RE * 4);
  if (threadIdx.x == 0) {
    for (int i = 0; i < RS_NS; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], RS_CONS); }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == RS_CONS) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t c = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        for (int64_t s = 0; s < nst; ++s, ++c) {
          const int slot = (int)(c % RS_NS);
          if (!(ok = mbar_wait(&empty[slot], (uint32_t)(((c / RS_NS) & 1) ^ 1), abort_flag, status))) break;
          mbar_arrive_tx(&full[slot], (uint32_t)RS_XBYTES + ubytes);
          tma_load_2d(saddr(xs + slot * RS_XBYTES), &tmap, (int)(s * RS_COLS), (int)(it * RS_ROWS), &full[slot]);
          bulk_load(saddr(us + slot * (RS_UBYTES / 4)), Ur + s * RS_COLS * RE, ubytes, &full[slot]);
        }
      }
      // the CTA may exit only when no copy into its shared memory is in flight
      for (int64_t q = c - 1; q >= 0 && q >= c - RS_NS; --q)
        for (uint32_t w = 0; w < (1u << 22); ++w)
          if (mbar_test(&full[q % RS_NS], (uint32_t)((q / RS_NS) & 1))) break;
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  // thread = (row group rs, column group g): rows rs + 16 h (h < 4), columns 4g..4g+3.
  // Warp w covers row groups 8 (w & 1) .. + 7 and column groups 4 (w >> 1) .. + 3, so
  // the four U_r slices a warp reads start 40 floats apart (distinct banks) and its X
  // reads are 8 rows x 64 bytes (4 wavefronts under the 128-byte swizzle).
  constexpr int NCG = 8;                                        // column groups
  constexpr int CPT = RS_COLS / NCG;                            // columns per thread
  constexpr int RPT = RS_ROWS * NCG / (RS_CONS * 32);           // rows per thread
  constexpr int RSTEP = RS_ROWS / RPT;
  static_assert(RS_CONS == 4 && RPT == 4 && RSTEP == 16, "lane map below assumes 4 warps of 8 x 4 threads");
  const int rs = 8 * (warp & 1) + (lane >> 2), g = 4 * (warp >> 1) + (lane & 3);
  int64_t c = 0;
  // Accumulators hold the pairs (k, k + 1) of U_r columns in one packed register pair:
  // one fma.rn.f32x2 does the two scalar FMAs, rounded the same way.
  const uint64_t one2 = f2_pack(1.f, 1.f);
  for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    uint64_t acc[RPT][RP], tot[RPT][RP];
#pragma unroll
    for (int h = 0; h < RPT; ++h)
#pragma unroll
      for (int m = 0; m < RP; ++m) acc[h][m] = tot[h][m] = 0ull;
    bool ok = true;
    for (int64_t s = 0; s < nst; ++s, ++c) {
      const int slot = (int)(c % RS_NS);
      if (!(ok = __all_sync(0xffffffffu, mbar_wait(&full[slot], (uint32_t)((c / RS_NS) & 1), abort_flag, status))))
        break;
      uint64_t u2[CPT * RP];            // u2[cc RP + m] = (U_r(col, 2m), U_r(col, 2m + 1))
      const float4* u4 = reinterpret_cast<const float4*>(us + slot * (RS_UBYTES / 4) + CPT * g * RE);
#pragma unroll
      for (int v = 0; v < CPT * RE / 4; ++v) {
        const float4 w = lds128_slot(u4 + v);
        u2[2 * v] = f2_pack(w.x, w.y);
        u2[2 * v + 1] = f2_pack(w.z, w.w);
      }
#pragma unroll
      for (int h = 0; h < RPT; ++h) {
        const int row = rs + RSTEP * h;
        const unsigned char* rp = xs + slot * RS_XBYTES + row * 128;
        float x[CPT];
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
          const float4 xv = lds128_slot(rp + ((((CPT / 4) * g + q) ^ (row & 7)) << 4));
          x[4 * q] = xv.x; x[4 * q + 1] = xv.y; x[4 * q + 2] = xv.z; x[4 * q + 3] = xv.w;
        }
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const uint64_t xx = f2_pack(x[cc], x[cc]);
#pragma unroll
          for (int m = 0; m < RP; ++m) acc[h][m] = f2_fma(xx, u2[cc * RP + m], acc[h][m]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if ((s % RS_FOLD) == RS_FOLD - 1 || s == nst - 1) {
#pragma unroll
        for (int h = 0; h < RPT; ++h)
#pragma unroll
          for (int m = 0; m < RP; ++m) {
            tot[h][m] = f2_fma(acc[h][m], one2, tot[h][m]);   // tot + acc, one rounding
            acc[h][m] = 0ull;
          }
      }
    }
    if (!ok) break;
    // T(a, half, k): sum over the 4 column groups of this warp (lanes 4m .. 4m + 3); the
    // other half of the columns is in warp w ^ 2 and has its own slot (k_root_left adds
    // the two), so the consumer warps never wait on one another
    const int half = warp >> 1;
#pragma unroll
    for (int h = 0; h < RPT; ++h) {
      const int64_t a = it * RS_ROWS + rs + RSTEP * h;
#pragma unroll
      for (int m = 0; m < RP; ++m) {
        float tv[2];
        f2_unpack(tot[h][m], tv[0], tv[1]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = 2 * m + e;
          if (k >= RR) continue;
          float v = tv[e];
          v += __shfl_xor_sync(0xffffffffu, v, 1);
          v += __shfl_xor_sync(0xffffffffu, v, 2);
          if ((lane & 3) == 0 && a < nl) T[(a * 2 + half) * RR + k] = v;
        }
      }
    }
  }
}

// part[blk](j, k) = sum over the CTA's rows a of U_l(a, j) T(a, k), with T(a, k) the
// sum of the two column halves written by k_root_rows.
__global__ void __launch_bounds__(RL_ROWS) k_root_left(const float* __restrict__ Ul, int rl,
                                                       const float* __restrict__ T, int rr, int64_t nl,
                                                       float* __restrict__ part) {
  __shared__ float ul[RL_ROWS * RS_UMAX], ts[RL_ROWS * RS_UMAX];
  const int64_t a0 = (int64_t)blockIdx.x * RL_ROWS;
  const int rows = (int)min((int64_t)RL_ROWS, nl - a0);
  for (int e = threadIdx.x; e < rows * rl; e += blockDim.x) ul[e] = Ul[a0 * rl + e];
  for (int e = threadIdx.x; e < rows * rr; e += blockDim.x) {
    const int a = e / rr, k = e % rr;
    ts[e] = T[((a0 + a) * 2) * rr + k] + T[((a0 + a) * 2 + 1) * rr + k];
  }
  __syncthreads();
  const int p = threadIdx.x;
  if (p < rl * rr) {
    // four interleaved float32 partial sums of 64 products each; the partials of all
    // CTAs are added in float64 by k_root_reduce
    const int j = p / rr, k = p % rr;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < rows; ++a) acc[a & 3] = fmaf(ul[a * rl + j], ts[a * rr + k], acc[a & 3]);
    part[(size_t)blockIdx.x * rl * rr + p] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
}

template <int RR>
int launch_rows(const CUtensorMap& map, const float* Ur, int64_t nl, int64_t nr, float* T, int* status,
                cudaStream_t st) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nitems = (nl + RS_ROWS - 1) / RS_ROWS;
  const int grid = (int)std::min<int64_t>(nitems, (int64_t)nsm * RS_CTAS_PER_SM);
  cudaFuncSetAttribute(k_root_rows<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem());
  k_root_rows<RR><<<grid, RS_THREADS, rs_smem(), st>>>(map, Ur, nl, nr, T, status);
  return 1;
}

}  // namespace

static int64_t cols_padded(int64_t nr) { return (nr + RS_COLS - 1) / RS_COLS * RS_COLS; }

// T and the partial sums, then (ragged n_r) the padded U_r at a 16-byte boundary
static size_t stream_base_floats(int64_t nl, int rl, int rr) {
  return ((size_t)nl * 2 * rr + (size_t)((nl + RL_ROWS - 1) / RL_ROWS) * rl * rr + 3) & ~(size_t)3;
}

cudaError_t root_tma_set_wait_limit(uint32_t polls) { return tma::set_wait_limit(polls); }

// U_r goes through a zero-padded copy when n_r is not a multiple of the 32-column stage
// or r_r is odd (the kernel reads U_r rows of r_r + (r_r & 1) floats: column pairs).
static bool needs_upad(int64_t nr, int rr) { return (nr % RS_COLS) != 0 || (rr & 1) != 0; }

size_t root_stream_scratch_floats(int64_t nl, int64_t nr, int rl, int rr) {
  const size_t upad = needs_upad(nr, rr) ? (size_t)cols_padded(nr) * (rr + (rr & 1)) : 0;
  return stream_base_floats(nl, rl, rr) + upad;
}

// Streaming root pass for float32 X with n_r % 4 == 0 (16-byte row stride), 16-byte
// aligned X and U_r and r_l, r_r <= 12.  When n_r is not a multiple of the 32-column
// stage, the last stage's TMA box overhangs the rows (the copy fills those columns
// with zeros) and U_r is first copied into a zero-padded buffer of ceil(n_r / 32) * 32
// rows, so that every stage's bulk copy of U_r stays inside it; for odd r_r the copy
// also gets a zero column (rows of r_r + 1 floats).  Returns the number
// of launches, or 0 when the shape does not qualify (the caller then uses the tiled
// kernel).  `scratch` holds root_stream_scratch_floats() floats; `reduce` launches the
// final float64 sum.
int launch_root_stream(const float* X, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur, int rr,
                       float* BR, float* scratch, int* status, cudaStream_t st) {
  if (nr % 4 != 0 || rr < 1 || rr > RS_UMAX || rl < 1 || rl > RS_UMAX) return 0;
  if (nl < 1 || nl >= ((int64_t)1 << 31) || cols_padded(nr) >= ((int64_t)1 << 31)) return 0;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) || (reinterpret_cast<uintptr_t>(Ur) & 15u)) return 0;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return 0;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)nr, (cuuint64_t)nl};
  const cuuint64_t gstride[1] = {(cuuint64_t)nr * 4};
  const cuuint32_t box[2] = {(cuuint32_t)RS_COLS, (cuuint32_t)RS_ROWS};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 0;
  float* T = scratch;
  float* part = scratch + (size_t)nl * 2 * rr;
  const int64_t ncols = cols_padded(nr);
  const float* Urs = Ur;
  int n = 0;
  if (needs_upad(nr, rr)) {
    const int re = rr + (rr & 1);
    float* Urp = scratch + stream_base_floats(nl, rl, rr);
    if ((reinterpret_cast<uintptr_t>(Urp) & 15u) ||
        cudaMemsetAsync(Urp, 0, (size_t)ncols * re * 4, st) != cudaSuccess ||
        cudaMemcpy2DAsync(Urp, (size_t)re * 4, Ur, (size_t)rr * 4, (size_t)rr * 4, (size_t)nr,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return 0;
    Urs = Urp;
  }
  switch (rr) {
#define RS_CASE(K) \
  case K: n = launch_rows<K>(map, Urs, nl, ncols, T, status, st); break;
    RS_CASE(1) RS_CASE(2) RS_CASE(3) RS_CASE(4) RS_CASE(5) RS_CASE(6)
    RS_CASE(7) RS_CASE(8) RS_CASE(9) RS_CASE(10) RS_CASE(11) RS_CASE(12)
#undef RS_CASE
    default: return 0;
  }
  const int64_t nblk = (nl + RL_ROWS - 1) / RL_ROWS;
  k_root_left<<<(unsigned)nblk, RL_ROWS, 0, st>>>(Ul, rl, T, rr, nl, part);
  launch_root_reduce(part, nblk, rl, rr, BR, st);
  return n + 2;
}

}  // namespace rt
