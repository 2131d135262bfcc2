// core_tc.cu - the pass over X of the core projection on the 5th-generation
// tensor cores (tcgen05, TMEM accumulators, TMA-fed).
//
// For X viewed as S slabs of n1 x n2 (the last two modes; S = product of the
// leading modes) it computes, per slab s,
//     P_s = U_1^T X_s U_2          (r1 x r2),
// i.e. the last two contractions of S = X x_1 U_1^T ... x_d U_d^T (Alg. 1,
// core step) fused in one read of X.  The remaining modes are contracted on
// P afterwards (core_kernels.cu).
//
// Arithmetic: every operand is split into bf16 terms, x = hi(x) + lo(x), and
// the MMAs (kind::f16, float32 accumulate) form the products of all terms, so
// the result carries float32-level accuracy (about 2^-16 relative per
// product).  X modes: 0 = float32 X split into hi + lo (default); 1 = bfloat16
// X as stored (one term); 2 = float32 X rounded to one bf16 term (the BF16
// compute form); 3 = E4M3 codes with one power-of-two scale per slab (the FP8
// storage form).  U_1 and the intermediate T are always split in two bf16
// terms; U_2 too, except in mode 3, where MMA1 is kind::f8f6f4 (K = 32 per
// instruction, A = the codes straight from the stage) and U_2 is four E4M3
// terms u = sigma (t_1 + t_2 / 32 + t_3 / 32^2 + t_4 / 32^3), each term the
// nearest E4M3 value to what the previous ones left (about 2^-16 relative in
// all, as two bf16 terms); the code values are exact, so each product is exact
// and only the float32 accumulation rounds.
//
// Data path per CTA (persistent, one per SM, warp-specialised, 14 warps):
//   warp 0      TMA producer: 128-byte-wide boxes (32 float32 or 64 bf16
//               columns) of one slab into a ring of NS3 shared-memory stages,
//               128-byte swizzle.
//   warp 1      TMEM allocator and MMA issuer.  MMA1 per K step:
//               D1 (n1 x 2 r2p) += X_s [hi(U_2) | lo(U_2)], A = X terms from
//               TMEM (float32 X) or from the stage (bf16 X).  MMA2 per batch
//               of 128 / r2p slabs: D2 (128 x 128) = A_U T, where row 2a + t of
//               A_U is term t (hi, lo) of column a of U_1 (K-major A) and T of
//               the batch (MN-major B, 128 columns) is split in bf16 terms: two
//               MMAs per K step (T's terms) give all four term products, and
//               P = D2 row 2a + D2 row 2a + 1.
//   warps 2-9   converters (float32 X): two groups of four quadrant warps take
//               alternate stages; each thread splits one row into bf16 terms
//               and stores them to a TMEM A buffer (tcgen05.st).
//   warps 10-13 epilogue: T = D1_hi + D1_lo from TMEM, each thread writes its
//               row of T as bf16 hi/lo terms with 16-byte stores; after MMA2,
//               the two rows of each a are added (lane pairs) and P_s rows
//               written to global memory.
// Every mbarrier wait is bounded; on expiry the CTA records the timeout in the
// status word, stops issuing work, drains and frees its TMEM, and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"
#include "tma_util.cuh"
#include "tc_util.cuh"

namespace rt {
namespace tc {

using namespace tma;

constexpr int ROWS = 128;        // rows per tile (M)
constexpr int KC = 32;           // columns per K-chunk (one 128-byte swizzle span)
constexpr int STAGE_BYTES = ROWS * KC * 4;


struct Core2Args {
  const void* X;     // only for the element type; data comes through the tensor map
  const float* U1;   // n1 x r1
  const float* U2;   // n2 x r2
  float* P;          // S x r1 x r2
  const float* xscale;  // mode 3: one scale per slab
  int64_t S;
  int n1, n2, r1, r2;
  int* status;
};


constexpr int NCONV = 8;                       // converter warps: two groups of four quadrants
constexpr int W_CONV0 = 2, W_EPI0 = W_CONV0 + NCONV;
constexpr int NWARPS = W_EPI0 + 4;
constexpr int NTHREADS_V2 = NWARPS * 32;       // 448
// Converter group g takes the chunks c with c % 2 == g.  Parity waits are only
// safe when one consumer group owns every use of a barrier (a second group
// could otherwise test a phase two behind and pass), so the number of stages
// and of TMEM A buffers must be even: stage c % NS and buffer c % NA then
// always belong to the same group.

template <int R2P, int XM>
struct Layout {
  static constexpr bool XBF16 = (XM == 1);      // X stored as bf16: MMA1 reads the stage
  static constexpr bool XF8 = (XM == 3);        // E4M3 codes: kind::f8f6f4 MMA1 reads the stage
  static constexpr bool XSMEM = XBF16 || XF8;   // A operand of MMA1 in shared memory
  static constexpr int NUT = XF8 ? 4 : 2;       // terms of U_2
  static constexpr int N1 = NUT * R2P;          // MMA1: X_s [terms of U2], M = 128 rows of the slab
  static constexpr int KCX = XF8 ? 128 : XBF16 ? 64 : 32;  // X columns per stage (128 bytes)
  static constexpr int KB = XF8 ? 128 : 64;     // K elements per 128-byte chunk of B1
  static_assert(!XF8 || R2P <= 32, "FP8 form: r_2 <= 32 (TMEM columns)");
  static constexpr int SPB = 128 / R2P;        // slabs per MMA2 batch (N = 128 columns of T)
  static constexpr int N2 = 128;               // MMA2: A_U [T of SPB slabs], M = 128 (2 terms x a < 64)
  static constexpr int NA = 4;                 // TMEM A buffers of 32 columns (float32 X only)
  static_assert(NA % 2 == 0, "A buffers must be even");
  static constexpr int A_COL = 0;
  static constexpr int D1_COL = XSMEM ? 0 : NA * 32;
  static constexpr int D2_COL = D1_COL + 2 * N1;
  static constexpr int ND2 = (D2_COL + 2 * N2 <= 512) ? 2 : 1;   // D2 buffers
  static constexpr int TMEM_USED = D2_COL + ND2 * N2;
  static constexpr int NS = (R2P == 64) ? 4 : 6;                 // X stages (shared-memory budget)
  static_assert(NS % 2 == 0, "stages must be even");
  static constexpr int TCH = XF8 ? (R2P < 16 ? R2P : 16) : (R2P < 32 ? R2P : 32);   // T columns per epilogue round
  static constexpr int TMEM_COLS = TMEM_USED <= 128 ? 128 : TMEM_USED <= 256 ? 256 : 512;
  // T of a batch as the MN-major B operand of MMA2: K = 128 rows (i) x N = 128 columns
  // (slab j, column b), 128-byte swizzle, atoms of 8 rows x 64 columns; the 16 row
  // atoms of a 64-column group are contiguous (1 KB apart), the two groups 16 KB apart.
  static constexpr int BT_TERM = 128 * 128 * 2;
  static constexpr int BT_NATOM = 16 * 1024;
  // A_U, the K-major A operand of MMA2: 128 rows (2a + term) x K = 128 (i), two 64-wide
  // K chunks of 16 KB
  static constexpr int AU_BYTES = 128 * 128 * 2;
  static_assert(TMEM_USED <= 512, "TMEM columns");
};

// Dynamic shared memory (1024-aligned):
//   BT[2 terms][2 groups][16 atoms][8][64 bf16] | B1[nkb][N1][64 bf16] | AU[2 chunks][128 rows 2a+t][64 bf16] |
//   stages[NS3][16 KB] | bars
template <int R2P, int XM>
__global__ void __launch_bounds__(NTHREADS_V2, 1) k_core2_tc(const __grid_constant__ CUtensorMap tmap, Core2Args args) {
  using LY = Layout<R2P, XM>;
  constexpr int NS3 = LY::NS, ND2 = LY::ND2, NA = LY::NA;
  constexpr bool XSMEM = LY::XSMEM, XF8 = LY::XF8;
  constexpr bool XLO = (XM == 0);                  // float32 X keeps its lo term
  constexpr int N1 = LY::N1, N2 = LY::N2, KCX = LY::KCX, SPB = LY::SPB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nkc = (args.n2 + KCX - 1) / KCX;       // stages per slab
  const int nkb = (args.n2 + LY::KB - 1) / LY::KB; // 128-byte K chunks of B1
  unsigned char* BT = base;
  unsigned char* B1 = BT + 2 * LY::BT_TERM;
  unsigned char* AU = B1 + (size_t)nkb * N1 * 128;
  unsigned char* stages = AU + LY::AU_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + NS3 * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = full + NS3;
  uint64_t* afull = empty + NS3;
  uint64_t* aempty = afull + NA;
  uint64_t* d1full = aempty + NA;
  uint64_t* d1empty = d1full + 2;
  uint64_t* tready = d1empty + 2;
  uint64_t* d2full = tready + 2;
  uint64_t* d2empty = d2full + 2;
  uint64_t* fin = d2empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n1 = args.n1, n2 = args.n2, r1 = args.r1, r2 = args.r2;
  const int64_t S = args.S;
  const int64_t nmine = (S > blockIdx.x) ? (S - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t nchunks = nmine * nkc;
  const int64_t nbatch = (nmine + SPB - 1) / SPB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS3; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], XSMEM ? 1 : 4); }
    for (int i = 0; i < NA; ++i) { mbar_init(&afull[i], 4); mbar_init(&aempty[i], 1); }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&d1full[i], 1); mbar_init(&d1empty[i], 4);
      mbar_init(&tready[i], 4);
      mbar_init(&d2full[i], 1); mbar_init(&d2empty[i], 4);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B1 = [hi(U2) | lo(U2)] (rows n < R2P: hi), AU = hi(U1)^T, lo(U1)^T (rows a >= r1 zero),
  // bf16, K-major, swizzled.  FP8 form: B1 = [t_1 | t_2 | t_3 | t_4] of U2 / sigma, E4M3.
  __shared__ unsigned int s_umax;
  float usig = 1.f;
  if constexpr (XF8) {
    if (threadIdx.x == 0) s_umax = 0u;
    __syncthreads();
    unsigned int m = 0u;
    for (int e = threadIdx.x; e < n2 * r2; e += NTHREADS_V2) m = max(m, __float_as_uint(fabsf(__ldg(args.U2 + e))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(&s_umax, m);
    __syncthreads();
    // max |U2| = f 2^ex with 0.5 <= f < 1: sigma = 2^(ex - 8) keeps every |u| / sigma below 256
    int ex = 0;
    const float umax = __uint_as_float(s_umax);
    if (umax > 0.f) frexpf(umax, &ex);
    usig = ldexpf(1.f, ex - 8);
    for (int e = threadIdx.x; e < nkb * 128 * R2P; e += NTHREADS_V2) {
      const int k = e / R2P, col = e % R2P;
      float v = (k < n2 && col < r2) ? ldexpf(__ldg(args.U2 + (int64_t)k * r2 + col), 8 - ex) : 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        // the residual of a nearest E4M3 value is exact in float32 and at most 2^-4 of |v|,
        // so 32 x residual stays within the 256 bound of the next term
        const uint32_t code = e4m3_code(v);
        B1[sw_off8(t * R2P + col, k, N1)] = (unsigned char)code;
        v = (v - e4m3_value(code)) * 32.f;
      }
    }
  } else {
    // (eight loads of a thread in flight per round: a loop of dependent load-then-store
    // steps would pay the load latency once per element before the first X stage)
    const int tot2 = nkb * 64 * R2P;
    for (int e0 = threadIdx.x; e0 < tot2; e0 += 8 * NTHREADS_V2) {
      float uv[8];
#pragma unroll
      for (int q2 = 0; q2 < 8; ++q2) {
        const int e = e0 + q2 * NTHREADS_V2, k = e / R2P, col = e % R2P;
        uv[q2] = (e < tot2 && k < n2 && col < r2) ? __ldg(args.U2 + (int64_t)k * r2 + col) : 0.f;
      }
#pragma unroll
      for (int q2 = 0; q2 < 8; ++q2) {
        const int e = e0 + q2 * NTHREADS_V2, k = e / R2P, col = e % R2P;
        if (e >= tot2) break;
        unsigned short hi, lo;
        split1_bf16(uv[q2], hi, lo);
        *reinterpret_cast<unsigned short*>(B1 + sw_off16(col, k, N1)) = hi;
        *reinterpret_cast<unsigned short*>(B1 + sw_off16(R2P + col, k, N1)) = lo;
      }
    }
  }
  for (int e0 = threadIdx.x; e0 < 128 * 64; e0 += 8 * NTHREADS_V2) {
    float uv[8];
#pragma unroll
    for (int q2 = 0; q2 < 8; ++q2) {
      const int e = e0 + q2 * NTHREADS_V2, i = e / 64, a = e % 64;
      uv[q2] = (e < 128 * 64 && i < n1 && a < r1) ? __ldg(args.U1 + (int64_t)i * r1 + a) : 0.f;
    }
#pragma unroll
    for (int q2 = 0; q2 < 8; ++q2) {
      const int e = e0 + q2 * NTHREADS_V2, i = e / 64, a = e % 64;
      if (e >= 128 * 64) break;
      unsigned short hi, lo;
      split1_bf16(uv[q2], hi, lo);
      *reinterpret_cast<unsigned short*>(AU + sw_off16(2 * a, i, 128)) = hi;
      *reinterpret_cast<unsigned short*>(AU + sw_off16(2 * a + 1, i, 128)) = lo;
    }
  }
  // T starts at zero: rows i >= n1 and the columns of a partial batch stay zero
  for (int e = threadIdx.x; e < 2 * LY::BT_TERM / 16; e += NTHREADS_V2)
    reinterpret_cast<uint4*>(BT)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"((uint32_t)LY::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t box_bytes = (uint32_t)n1 * 128;
  constexpr uint32_t idesc1 = XF8 ? idesc_e4m3(128, N1) : idesc_bf16(128, N1);
  constexpr uint32_t idesc2 = idesc_bf16(128, N2) | (1u << 16);  // B (T) MN-major

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      for (int64_t c = 0; c < nchunks; ++c) {
        const int st = (int)(c % NS3);
        if (!mbar_wait(&empty[st], (uint32_t)(((c / NS3) & 1) ^ 1), abort_flag, args.status)) break;
        const int64_t s = blockIdx.x + (c / nkc) * gridDim.x;
        const int kc = (int)(c % nkc);
        mbar_arrive_tx(&full[st], box_bytes);
        tma_load_2d(saddr(stages + st * STAGE_BYTES), &tmap, kc * KCX, (int)(s * n1), &full[st]);
      }
      for (int64_t c = nchunks - 1; c >= 0 && c >= nchunks - NS3; --c)
        for (uint32_t it = 0; it < (1u << 16); ++it)
          if (mbar_test(&full[c % NS3], (uint32_t)((c / NS3) & 1))) break;
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      bool ok = true;
      auto mma2 = [&](int64_t g) -> bool {   // P of batch g: D2 = A_U (hi T + lo T)
        // T of batch g is announced on tready[g & 1] (two barriers, by batch parity); the
        // accumulator uses buffer g % ND2
        if (!mbar_wait(&tready[g & 1], (uint32_t)((g >> 1) & 1), abort_flag, args.status)) return false;
        const int b = (int)(g % ND2);
        const uint32_t ph = (uint32_t)((g / ND2) & 1);
        if (!mbar_wait(&d2empty[b], ph ^ 1, abort_flag, args.status)) return false;
        fence_after();
        const uint32_t dcol = tmem + LY::D2_COL + b * N2;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {     // K = 128 in steps of 16
          const uint64_t adesc = sw128_desc(saddr(AU + (kk >> 2) * 128 * 128 + (kk & 3) * 32));
#pragma unroll
          for (int tb = 0; tb < 2; ++tb) {   // hi T, lo T (both terms of U_1 in the rows of A_U)
            const uint32_t baddr = saddr(BT + tb * LY::BT_TERM + kk * 2048);
            mma_bf16_ss(dcol, adesc, mn128_desc(baddr, LY::BT_NATOM, 1024), idesc2, (kk | tb) ? 1u : 0u);
          }
        }
        mma_commit(&d2full[b]);
        return true;
      };
      int64_t c = 0;
      for (int64_t t = 0; t < nmine && ok; ++t) {
        const int db = (int)(t & 1);
        if (!(ok = mbar_wait(&d1empty[db], (uint32_t)(((t >> 1) & 1) ^ 1), abort_flag, args.status))) break;
        fence_after();
        const uint32_t dcol = tmem + LY::D1_COL + db * N1;
        for (int kc = 0; kc < nkc; ++kc, ++c) {
          if (XSMEM) {
            const int st = (int)(c % NS3);
            if (!(ok = mbar_wait(&full[st], (uint32_t)((c / NS3) & 1), abort_flag, args.status))) break;
            fence_after();
            const uint32_t sbase = saddr(stages + st * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const int kg = kc * 4 + kk;    // global 16-wide K step
              const uint32_t baddr = saddr(B1 + (kg >> 2) * N1 * 128 + (kg & 3) * 32);
              if (XF8) mma_f8_ss(dcol, sw128_desc(sbase + kk * 32), sw128_desc(baddr), idesc1, (kc | kk) ? 1u : 0u);
              else mma_bf16_ss(dcol, sw128_desc(sbase + kk * 32), sw128_desc(baddr), idesc1, (kc | kk) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
          } else {
            const int ab = (int)(c % NA);
            if (!(ok = mbar_wait(&afull[ab], (uint32_t)((c / NA) & 1), abort_flag, args.status))) break;
            fence_after();
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const int kg = kc * 2 + kk;
              const uint64_t bdesc = sw128_desc(saddr(B1 + (kg >> 2) * N1 * 128 + (kg & 3) * 32));
              const uint32_t a = tmem + LY::A_COL + ab * 32 + kk * 8;
              mma_bf16_ts(dcol, a, bdesc, idesc1, (kc | kk) ? 1u : 0u);   // hi(X)
              if (XLO) mma_bf16_ts(dcol, a + 16, bdesc, idesc1, 1u);       // lo(X)
            }
            mma_commit(&aempty[ab]);
          }
        }
        if (!ok) break;
        mma_commit(&d1full[db]);
        // MMA2 of the previous batch once the first slab of the next batch is queued
        if (t % SPB == 0 && t >= SPB && !(ok = mma2(t / SPB - 1))) break;
      }
      if (ok && nbatch >= 1) mma2(nbatch - 1);
      mma_commit(fin);
      for (uint32_t it = 0; it < (1u << 20); ++it)
        if (mbar_test(fin, 0)) break;
    }
  } else if (warp < W_EPI0) {
    // ---------------------------------------------------------------- converters (float32 X)
    if (!XSMEM) {
      const int grp = (warp - W_CONV0) >> 2;
      const int q = warp & 3;
      const int row = q * 32 + lane;
      for (int64_t c = grp; c < nchunks; c += 2) {
        const int st = (int)(c % NS3), ab = (int)(c % NA);
        bool ok = __all_sync(0xffffffffu, mbar_wait(&full[st], (uint32_t)((c / NS3) & 1), abort_flag, args.status));
        if (!ok) break;
        uint32_t v[32];   // 16 columns hi, 16 columns lo
        const unsigned char* rowp = stages + st * STAGE_BYTES + row * 128;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < n1) f = lds128_slot(rowp + ((j ^ (row & 7)) << 4));
          if (XLO) {
            split_bf16(f.x, f.y, v[2 * j], v[16 + 2 * j]);
            split_bf16(f.z, f.w, v[2 * j + 1], v[16 + 2 * j + 1]);
          } else {
            v[2 * j] = pack_bf16(f.x, f.y);
            v[2 * j + 1] = pack_bf16(f.z, f.w);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        ok = __all_sync(0xffffffffu, mbar_wait(&aempty[ab], (uint32_t)(((c / NA) & 1) ^ 1), abort_flag, args.status));
        if (!ok) break;
        fence_after();
        if (XLO) tmem_st32(tmem + ((uint32_t)(q * 32) << 16) + LY::A_COL + ab * 32, v);
        else tmem_st16(tmem + ((uint32_t)(q * 32) << 16) + LY::A_COL + ab * 32, v);
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&afull[ab]);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;
    const int i = q * 32 + lane;                    // slab row = K index of MMA2
    auto read_p = [&](int64_t g) -> bool {          // P of the slabs of batch g
      const int bb = (int)(g % ND2);
      const uint32_t ph = (uint32_t)((g / ND2) & 1);
      bool ok = __all_sync(0xffffffffu, mbar_wait(&d2full[bb], ph, abort_flag, args.status));
      if (!ok) return false;
      fence_after();
      // M = 128 accumulator: row m in TMEM lane m, so warp q holds rows 32 q + lane, i.e.
      // a = 16 q + lane / 2 with the hi term of U_1 in the even lane and the lo term in the
      // odd one; column n = j R2P + b of slab j.  Both lanes of a pair form the same sum
      // and each writes half of the columns.
      if (16 * q < r1) {
        const int a = 16 * q + (lane >> 1);
        const int half = (lane & 1) * (LY::TCH / 2);
#pragma unroll
        for (int j = 0; j < SPB; ++j) {
          const int64_t t = g * SPB + j;
#pragma unroll
          for (int b0 = 0; b0 < R2P; b0 += LY::TCH) {
            uint32_t d[LY::TCH];
#pragma unroll
            for (int cc = 0; cc < LY::TCH / 8; ++cc)
              tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + LY::D2_COL + bb * N2 + j * R2P + b0 + cc * 8, d + 8 * cc);
            tmem_wait_ld();
            float v[LY::TCH / 2];
#pragma unroll
            for (int b = 0; b < LY::TCH; ++b) {
              const float x = __uint_as_float(d[b]);
              const float y = x + __shfl_xor_sync(0xffffffffu, x, 1);
              if ((b < LY::TCH / 2) == ((lane & 1) == 0)) v[b % (LY::TCH / 2)] = y;
            }
            if (a < r1 && t < nmine) {
              float* Pout = args.P + ((blockIdx.x + t * gridDim.x) * (int64_t)r1 + a) * r2 + b0 + half;
              if ((r2 & 3) == 0) {
#pragma unroll
                for (int b = 0; b < LY::TCH / 2; b += 4)
                  if (b0 + half + b < r2)
                    *reinterpret_cast<float4*>(Pout + b) = make_float4(v[b], v[b + 1], v[b + 2], v[b + 3]);
              } else {
#pragma unroll
                for (int b = 0; b < LY::TCH / 2; ++b)
                  if (b0 + half + b < r2) Pout[b] = v[b];
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d2empty[bb]);
      return true;
    };
    bool ok = true;
    for (int64_t t = 0; t < nmine && ok; ++t) {
      const int db = (int)(t & 1);
      ok = __all_sync(0xffffffffu, mbar_wait(&d1full[db], (uint32_t)((t >> 1) & 1), abort_flag, args.status));
      if (!ok) break;
      fence_after();
      const int j = (int)(t % SPB);
      const int64_t g = t / SPB;
      // Row i of T (columns b of slab j) into the MN-major B operand, TCH columns per
      // round: T = D1_hi + D1_lo, 8 consecutive columns per 16-byte store, hi and lo
      // terms.  Rows i >= n1 stay zero (for bf16 X those D1 rows come from stage rows
      // the TMA box does not cover).  The first slab of a batch first reads P of the
      // previous batch (which frees T).
      bool first = true;
      // FP8 form: T = scale_s sigma (D_1 + D_2 / 32 + D_3 / 32^2 + D_4 / 32^3)
      const float tsc = XF8 ? __ldg(args.xscale + blockIdx.x + t * gridDim.x) * usig : 1.f;
#pragma unroll
      for (int h0 = 0; h0 < R2P; h0 += LY::TCH) {
        uint32_t dh[LY::TCH], dl[LY::TCH];
#pragma unroll
        for (int cc = 0; cc < LY::TCH / 8; ++cc) {
          tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + LY::D1_COL + db * N1 + h0 + cc * 8, dh + 8 * cc);
          tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + LY::D1_COL + db * N1 + R2P + h0 + cc * 8, dl + 8 * cc);
        }
        if constexpr (XF8) {
          uint32_t d3[LY::TCH], d4[LY::TCH];
#pragma unroll
          for (int cc = 0; cc < LY::TCH / 8; ++cc) {
            tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + LY::D1_COL + db * N1 + 2 * R2P + h0 + cc * 8, d3 + 8 * cc);
            tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + LY::D1_COL + db * N1 + 3 * R2P + h0 + cc * 8, d4 + 8 * cc);
          }
          tmem_wait_ld();
          // fold the four term sums into dh (dl = 0), Horner in powers of 1/32 (exact scalings)
#pragma unroll
          for (int b = 0; b < LY::TCH; ++b) {
            float v = __uint_as_float(d4[b]) * 0.03125f + __uint_as_float(d3[b]);
            v = v * 0.03125f + __uint_as_float(dl[b]);
            v = v * 0.03125f + __uint_as_float(dh[b]);
            dh[b] = __float_as_uint(v * tsc);
            dl[b] = 0u;
          }
        } else {
          tmem_wait_ld();
        }
        if (h0 + LY::TCH >= R2P) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&d1empty[db]);
        }
        if (first) {
          first = false;
          if (j == 0 && g >= 1 && !(ok = read_p(g - 1))) break;
        }
        if (i < n1) {
          const int atom = (i >> 3) * 1024 + (i & 7) * 128;
#pragma unroll
          for (int b0 = 0; b0 < LY::TCH; b0 += 8) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              split_bf16(__uint_as_float(dh[b0 + 2 * e]) + __uint_as_float(dl[b0 + 2 * e]),
                         __uint_as_float(dh[b0 + 2 * e + 1]) + __uint_as_float(dl[b0 + 2 * e + 1]), hi[e], lo[e]);
            const int n = j * R2P + h0 + b0;
            const int off = (n >> 6) * LY::BT_NATOM + atom + ((((n & 63) >> 3) ^ (i & 7)) << 4);
            *reinterpret_cast<uint4*>(BT + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(BT + LY::BT_TERM + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      }
      if (!ok) break;
      if (j == SPB - 1 || t == nmine - 1) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tready[g & 1]);
      }
    }
    if (ok && nbatch >= 1) read_p(nbatch - 1);
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)LY::TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------ host side
template <int R2P, int XM>
static size_t smem_bytes(int nkb) {
  using LY = Layout<R2P, XM>;
  return 1024 + 2 * (size_t)LY::BT_TERM + (size_t)nkb * LY::N1 * 128 + (size_t)LY::AU_BYTES +
         (size_t)LY::NS * STAGE_BYTES + 8 * (2 * LY::NS + 2 * LY::NA + 11) + 16;
}

template <int R2P, int XM>
static int launch_v3(const CUtensorMap& map, const Core2Args& a, int grid, cudaStream_t st) {
  const int nkb = (a.n2 + Layout<R2P, XM>::KB - 1) / Layout<R2P, XM>::KB;
  const size_t sm = smem_bytes<R2P, XM>(nkb);
  if (sm > 227 * 1024) return -1;
  cudaFuncSetAttribute(k_core2_tc<R2P, XM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_core2_tc<R2P, XM><<<grid, NTHREADS_V2, sm, st>>>(map, a);
  return 1;
}

}  // namespace tc

// Returns the number of launches (1), or 0 when the shape is not supported
// by the tensor-core path (the caller then uses the FFMA chain).
// xmode: 0 float32 X split into two bf16 terms, 1 bfloat16 X, 2 float32 X
// rounded to one bf16 term, 3 E4M3 codes with per-slab scales (xscale).
cudaError_t core_tc_set_wait_limit(uint32_t polls) { return tma::set_wait_limit(polls); }

int launch_core2_tc(int xmode, const void* X, int64_t S, int n1, int n2, const float* U1, int r1, const float* U2,
                    int r2, float* P, int* status, cudaStream_t st, int max_ctas, const float* xscale) {
  using namespace tc;
  if (xmode < 0 || xmode > 3) return 0;
  const bool xbf16 = (xmode == 1), xf8 = (xmode == 3);
  const int esz = xf8 ? 1 : xbf16 ? 2 : 4;
  if (n1 < 1 || n1 > ROWS || n2 < 1 || ((int64_t)n2 * esz) % 16 != 0 || r1 < 1 || r1 > 64 || r2 < 1 || r2 > 64)
    return 0;
  if (xf8 && (r2 > 32 || !xscale)) return 0;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0) return 0;
  if (S * (int64_t)n1 >= ((int64_t)1 << 31)) return 0;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return 0;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)n2, (cuuint64_t)(S * n1)};
  const cuuint64_t gstride[1] = {(cuuint64_t)n2 * esz};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)n1};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&map,
          xf8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
              : xbf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
          2, const_cast<void*>(X),
          gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 0;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = std::min<int64_t>(S, nsm);
  if (max_ctas > 0) grid = std::min<int64_t>(grid, max_ctas);
  Core2Args a{X, U1, U2, P, xscale, S, n1, n2, r1, r2, status};
  const int r2p = r2 <= 8 ? 8 : r2 <= 16 ? 16 : r2 <= 32 ? 32 : 64;
  int rc = 0;
#define RT_TC_CASE(B)                                                            \
  if (r2p == B) {                                                                \
    rc = xmode == 1   ? launch_v3<B, 1>(map, a, (int)grid, st)                   \
         : xmode == 2 ? launch_v3<B, 2>(map, a, (int)grid, st)                   \
         : xmode == 3 ? launch_v3<B, 3>(map, a, (int)grid, st)                   \
                      : launch_v3<B, 0>(map, a, (int)grid, st);                  \
    return rc < 0 ? 0 : rc;                                                      \
  }
  RT_TC_CASE(8) RT_TC_CASE(16) RT_TC_CASE(32)
#undef RT_TC_CASE
  if (r2p == 64) {
    rc = xmode == 1 ? launch_v3<64, 1>(map, a, (int)grid, st)
         : xmode == 2 ? launch_v3<64, 2>(map, a, (int)grid, st)
         : xmode == 0 ? launch_v3<64, 0>(map, a, (int)grid, st) : -1;
    return rc < 0 ? 0 : rc;
  }
  return 0;
}

}  // namespace rt
