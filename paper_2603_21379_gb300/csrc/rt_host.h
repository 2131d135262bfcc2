// rt_host.h - host-side interfaces between the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"

namespace rt {

// Tile sizes of the range-finder stages (shared by planner and kernels).
constexpr int SK_TI = 32;          // rows per gather/sketch tile (small: spreads the
                                   // scattered fiber loads over many SMs)
constexpr int SK_TJ = 128;         // samples per sketch chunk
constexpr int CMAX = 64;           // largest r + p supported
constexpr int QR_MAXF = 12288;     // floats per smem array in the block QR
constexpr int QR2_MAXF = 24576;    // floats per smem array in the TSQR second level
constexpr int BT_SC = 256;         // samples per chunk of B^T = Y^T Q
constexpr int BT_IB = 512;         // rows per reduction block of B^T (more, shorter CTAs for tall nodes)
constexpr int WS_MAXF = 24576;     // floats of the stacked R factors in the W-step
constexpr int WS_LDT = 80;         // column stride of R^T in the Jacobi SVD (CMAX + 16)
constexpr int WS_MAX_SWEEPS = 40;  // one-sided Jacobi sweeps before ST_NUMERIC
constexpr int QW_TI = 32;          // rows per tile of U = Q W
constexpr int QWF_MAX = 256;       // rows up to which U = Q W and its signs take one CTA
constexpr int BG_SC = 64;          // samples per chunk of the B-step Gram (Cholesky form)

// Stages.  The Cholesky form (qr = 2) of a problem runs STG_QZ, STG_BTG and STG_WSV2
// in place of STG_QR1 .. STG_QWF; a problem has units in one set or the other.
enum Stage : int {
  STG_SAMPLE = 0, STG_GS, STG_QR1, STG_QR2, STG_QR3, STG_BTP, STG_BTQ, STG_WSVD, STG_QW, STG_FLIP,
  STG_ZSUM, STG_QWF, STG_QZ, STG_BTG, STG_WSV2, STG_COUNT
};
// Stages of the TSQR tree beyond its first level: the QR of level j >= 1 and the
// combine passes t = 0 .. (top-down); their prefix rows follow the fixed ones and
// are uploaded only for groups with a problem of two or more levels (or an R tree
// in front of its W-step).
// The levels j of the R tree in front of the W-step follow them.
constexpr int STG_ALL = STG_COUNT + 2 * (TS_MAXLEV - 1) + TS_MAXLEV;
inline int stg_qr2(int j) { return j == 0 ? (int)STG_QR2 : STG_COUNT + j - 1; }
inline int stg_qrc(int t) { return STG_COUNT + TS_MAXLEV - 1 + t; }
inline int stg_wt(int j) { return STG_COUNT + 2 * (TS_MAXLEV - 1) + j; }

// Device-side view of a planned group of range-finder problems.
struct RFGroup {
  const RFProb* probs;   // device table [nprob]
  const int64_t* pre;    // device prefixes [nst][nprob + 1]
  int nprob;
  int nst;               // prefix rows: STG_COUNT, or STG_ALL when lmax > 1 or wmax > 0
  int lmax;              // largest TSQR tree depth of the group's problems
  int wmax;              // largest W-step R tree depth
  int64_t total[STG_ALL];  // host copy of the unit totals per stage (0 beyond nst)
};

// Enqueue every stage of the range finder for the group (Alg. 1 loop body /
// Alg. 2 node body).  Returns the number of kernel launches enqueued.
int launch_range_finder(const RFGroup& g, cudaStream_t st, int* status);
int launch_rf_head(const RFGroup& g, cudaStream_t st, int* status);   // S1-S5, B-step of S6
int launch_rf_tail(const RFGroup& g, cudaStream_t st, int* status);   // SVD of R, W, U = Q W, signs
// Sampling stage alone (S1), for rtucker_indices.
int launch_sample_only(const RFGroup& g, cudaStream_t st, int* status);
// Z = sum of the partial sketches (for rtucker_sketch).
int launch_sketch_sum(const RFGroup& g, float* const* Zout, cudaStream_t st);
// Shared-memory opt-ins; call once per device.
cudaError_t rf_init_attributes();

// ---- multi-TTM (core_kernels.cu)
// out(L, r, R) = sum_i U[i][a] A(L, n, R): mode contraction with U^T.
int launch_ttm_t(const void* A, int dtype, int64_t L, int64_t n, int64_t R, const float* U, int r,
                 float* out, cudaStream_t st);
// The same for float32 A on the tensor cores (ttm_tc.cu; bf16 hi/lo terms of A and U,
// float32 accumulate): n <= 128, r <= 64, R % 4 == 0, 16-byte aligned A and out.
// Returns the number of launches, or 0 when the shape does not qualify.
int launch_ttm_tc(const float* A, int64_t L, int64_t n, int64_t R, const float* U, int r, float* out, int* status,
                  cudaStream_t st);
// One mode contraction out(l, a, rho) = sum_i U[i][a] A(l, i, rho) of a grouped launch
// (A's element type is the launch's dtype).
struct TTMJob {
  const void* A;
  int64_t L, n, R;
  const float* U;
  int32_t r;
  float* out;
  int64_t tiles_x;
};
int64_t ttm_job_tiles(TTMJob& q);  // sets tiles_x, returns the job's CTA count
int launch_ttm_grouped(const TTMJob* jobs_dev, const int64_t* pre_dev, int njobs, int64_t total_tiles, int dtype,
                       cudaStream_t st);
// Grouped last-mode contractions (every job R = 1, n <= 256, r <= 32): pre counts
// ttm_last_job_ctas per job; returns 0 when a job does not fit.
int64_t ttm_last_job_ctas(const TTMJob& q, int rbn);   // rbn 128-row blocks per CTA
// Two neighbouring modes of small slabs in one read: out(l, a, b, rho) =
// sum_{i,j} U1[i][a] U2[j][b] A(l, i, j, rho), A (L, n1, n2, R) of the launch's dtype.
// slab2_fits: whether a slab (n1 n2 R values) and its partial products fit shared
// memory; launch_slab2 returns 0 when they do not.
bool slab2_fits(int64_t n1, int64_t n2, int64_t R, int r1, int r2);
// The last two modes of float32 X (R = 1) of S slabs n1 x n2 (n1 <= 128, n2 <= 256,
// r1, r2 <= 32): one thread per row, then the slab outputs; 0 when not applicable.
bool last2_fits(int64_t n1, int64_t n2, int r1, int r2);
int launch_last2(const float* X, int64_t S, int64_t n1, int64_t n2, const float* U1, int r1, const float* U2, int r2,
                 float* out, cudaStream_t st);
int launch_slab2(const void* A, int dtype, int64_t L, int64_t n1, int64_t n2, int64_t R, const float* U1, int r1,
                 const float* U2, int r2, float* out, cudaStream_t st);
int launch_ttm_last_grouped(const TTMJob* jobs_dev, const int64_t* pre_dev, int njobs, int64_t total_ctas,
                            int dtype, int nmax, int rmax, int rbn, cudaStream_t st);
cudaError_t core_init_attributes();
// Poll limit of the bounded mbarrier waits (0 = default) in each unit that has them.
cudaError_t core_tc_set_wait_limit(uint32_t polls);
cudaError_t root_tma_set_wait_limit(uint32_t polls);
cudaError_t diag_set_wait_limit(uint32_t polls);
// One CTA waiting on an mbarrier that nothing arrives on: the bounded wait runs out
// and records ST_TIMEOUT in *status (the bounded-wait failure path, exercised).
int launch_wait_selftest(int* status, cudaStream_t st);
// ---- differentiable Tucker (grad_kernels.cu)
// out(l, i, rho) = sum_a U[i][a] A(l, a, rho) (one core mode expanded, float32).
int launch_expand_f32(const float* A, int64_t L, int r, int64_t R, const float* U, int64_t n, float* out,
                      cudaStream_t st);
// out(s, i, j) = alpha X(s, i, j) + beta (U1 H_s U2^T)(i, j) for nslab slabs (X may be
// null); when sumsq_scaled is non-null it receives scale * ||out||_F^2 (part: per-CTA
// float64 partials, expand_partial_doubles() entries).  Returns 0 if r1, r2 are too large.
size_t expand_partial_doubles();
int launch_tucker_slab_out(const void* X, int dtype, float alpha, float beta, const float* H, int64_t nslab,
                           int64_t n1, int r1, int64_t n2, int r2, const float* U1, const float* U2, float* out,
                           double* part, double* sumsq_scaled, double scale, cudaStream_t st);
// Whether launch_tucker_slab_out takes slabs of n1 x n2 with ranks r1, r2.
bool slab_out_fits(int64_t n1, int r1, int64_t n2, int r2);
// Whether the last two modes of L slabs take the general form (launch_last_out after
// one more expansion): slabs too large for launch_tucker_slab_out, or large slabs
// fewer than the SMs.
bool last_modes_general(int64_t L, int64_t n1, int r1, int64_t n2, int r2);
// out(l, j) = alpha X(l, j) + beta sum_b Hp[l][b] U2[j][b] for M rows of n2 (the last
// mode; Hp holds the other modes already expanded), with the same sum of squares.
int launch_last_out(const void* X, int dtype, float alpha, float beta, const float* Hp, int64_t M, int r2,
                    int64_t n2, const float* U2, float* out, double* part, double* sumsq_scaled, double scale,
                    cudaStream_t st);
// out[i][a] = scale * sum_{p,q} Y(p, i, q) C(p, a, q) (Y of P x n x Q, C of P x r x Q);
// scratch: unfold_scratch_floats(n, r, P * Q) floats.
size_t unfold_scratch_floats(int64_t n, int r, int64_t K);
int launch_unfold_contract(const float* Y, const float* C, int64_t P, int64_t n, int r, int64_t Q, float scale,
                           float* out, float* scratch, cudaStream_t st);
int launch_scale_f32(float* x, int64_t n, float s, cudaStream_t st);
// Fused pass over X on tensor cores: P[s] = U1^T X[s] U2 for S slabs of
// n1 x n2.  xmode 0: float32 X as two bf16 terms; 1: bfloat16 X; 2: float32 X
// rounded to one bf16 term; 3: E4M3 codes with one float32 scale per slab
// (xscale).  Returns 0 when the shape is unsupported.
int launch_core2_tc(int xmode, const void* X, int64_t S, int n1, int n2, const float* U1, int r1, const float* U2,
                    int r2, float* P, int* status, cudaStream_t st, int max_ctas = 0, const float* xscale = nullptr);

// ---- float8 storage (fp8_kernels.cu): codes q (S slabs of `slab` elements) and one
// power-of-two scale per slab; 3 launches, or -1 when the grid would be too large.
int launch_quantize_fp8(const void* X, int dtype, int64_t S, int64_t slab, unsigned char* q, float* scales,
                        cudaStream_t st);

// ---- Kronecker-structured sketch (kron_kernels.cu)
constexpr int KRON_ZMAX = 8192;   // entries of Z_{d-2} (and of Z_{d-1}) one CTA accumulates
constexpr int KRON_LMAX = 8;      // l_{d-2}, l_{d-1} at most
struct KronArgs {
  const void* X;
  int dtype;
  int d;
  int64_t n[MAXD];
  int ell[MAXD];
  int64_t S;                  // slabs: product of the leading d-2 sizes
  int n1, n2;                 // n_{d-2}, n_{d-1}
  int la, lb;                 // l_{d-2}, l_{d-1}
  int K;                      // product of the leading l_j
  int ha, hb;                 // column chunks of A, row chunks of Bt per slab
  float* om;                  // Omega_j concatenated (n_j x l_j each)
  int64_t om_off[MAXD + 1];
  int64_t om_total;
  float* part1;               // [grid][n1 K l_b]
  float* part2;               // [grid][n2 K l_a]
  float* Ts;                  // [S][l_a l_b]
  float* Wt;                  // [S][K] Kronecker weights of the slabs
  float* z[MAXD];             // outputs Z_k (n_k x L_k)
};
struct KronFinish {
  int d;
  int64_t n[MAXD];
  int r[MAXD], L[MAXD];
  const float* Q;  int64_t qoff[MAXD];      // Q_k (n_k x L_k)
  const float* W;  int64_t woff[MAXD];      // W_k (L_k x r_k)
  float* U;        int64_t uoff[MAXD + 1];  // U_k (n_k x r_k)
  int64_t utotal;
  float* G;        int64_t gtotal;
  float* sign;     int roff[MAXD];          // column signs
  int rtotal;
};
struct ModeGram {            // Grams of the mode unfoldings of the reduced tensor C
  const float* C;
  int d;
  int L[MAXD];                // sizes of C (<= 64 each)
  int N[MAXD], B[MAXD];       // columns of C^(k); product of the sizes after mode k
  int ctas;                   // CTAs per mode
  float* part;                // partial Grams [ctas][L_k][L_k][2] per mode, at poff[k]
  int64_t poff[MAXD];
  float* cp[MAXD];            // the W-step's Gram words of mode k
  float* qeye[MAXD];          // the W-step's Q of mode k (set to I)
};
int launch_mode_gram(const ModeGram& g, cudaStream_t st);
size_t kron_sketch_smem(const KronArgs& a);
bool kron_shares_fit(const KronArgs& a);
int launch_kron_omega(const KronArgs& a, uint64_t seed, cudaStream_t st);
int launch_kron_sketch(const KronArgs& a, int grid, cudaStream_t st);   // sketch, reduce, leading modes
int launch_kron_finish(const KronFinish& f, cudaStream_t st);           // U = Q W, signs, core flips
int launch_rf_qr(const RFGroup& g, cudaStream_t st, int* status);       // S5 of a group only

// ---- H-Tucker (ht_kernels.cu)
struct TransferJob {     // B_S(i, j, k) = sum_{a,b} U_S[a n_r + b][i] U_l[a][j] U_r[b][k]
  const float* US; const float* Ul; const float* Ur; float* B;
  int64_t nl, nr; int rS, rl, rr;
  int64_t cta0;          // first CTA of this job in the partial-sum launch
};
int64_t transfer_ctas(int64_t nl);               // CTAs of one job
size_t transfer_part_floats(int64_t total_ctas); // partial-sum scratch
// ranks up to TRANSFER_RMAX; part holds transfer_part_floats(total CTAs of all jobs)
constexpr int TRANSFER_RMAX = 12;
int launch_transfer(const TransferJob* jobs_dev, const TransferJob* jobs_host, int njobs, float* part,
                    cudaStream_t st);
// One job with any ranks up to 64 (host-side job; cta0 unused): two mode contractions
// and a permutation; scratch holds transfer_general_floats() floats.
size_t transfer_general_floats(int64_t nl, int rS, int rl, int rr);
int launch_transfer_general(const TransferJob& jb, float* scratch, cudaStream_t st);
// B_R(0, j, k) = sum_{a,b} X[a nr + b] Ul[a][j] Ur[b][k]
// Root pass B_R = U_l^T X^(R_l) U_r: the streaming (TMA) kernel for float32 X when the
// shape allows, else the tiled kernel; scratch holds root_pass_scratch_floats().
int launch_root(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur, int rr,
                float* BR, float* scratch, int* status, cudaStream_t st);
// Any r_r up to 64: above the root kernels' width, one root pass per chunk of U_r's
// columns; scratch holds root_any_scratch_floats().
size_t root_any_scratch_floats(int64_t nl, int64_t nr, int rl, int rr);
int launch_root_any(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur,
                    int rr, float* BR, float* scratch, int* status, cudaStream_t st);
// The tiled kernel alone (no waits, no status word); scratch of root_scratch_floats().
// Any n_l: row blocks beyond the grid's y limit are folded onto the CTAs.  *err (if
// given) receives the first error of its own launches, without touching errors that
// were pending in the runtime before the call.
int launch_root_tiled(const void* X, int dtype, int64_t nl, int64_t nr, const float* Ul, int rl,
                      const float* Ur, int rr, float* BR, float* scratch, cudaStream_t st,
                      cudaError_t* err = nullptr);
int launch_root_stream(const float* X, int64_t nl, int64_t nr, const float* Ul, int rl, const float* Ur, int rr,
                       float* BR, float* scratch, int* status, cudaStream_t st);
void launch_root_reduce(const float* part, int64_t nblk, int rl, int rr, float* BR, cudaStream_t st);
size_t root_stream_scratch_floats(int64_t nl, int64_t nr, int rl, int rr);
size_t root_pass_scratch_floats(int64_t nl, int64_t nr, int rl, int rr);
size_t root_scratch_floats(int64_t nl, int64_t nr, int rl, int rr);

// ---- evaluators (eval_kernels.cu), float64
int launch_tucker_relerr(const void* X, int dtype, int d, const int64_t* n, const int32_t* r,
                         const float* const* U, const float* G, double* scratch, size_t scratch_doubles,
                         double* result2, cudaStream_t st, const float* xsc = nullptr);
bool tucker_relerr_slab_fits(int d, const int64_t* n, const int32_t* r);
bool tucker_relerr_supported(int d, const int64_t* n, const int32_t* r);
size_t tucker_relerr_scratch(int d, const int64_t* n, const int32_t* r);
int launch_ht_relerr(const void* X, int dtype, int64_t nl, int64_t nr, const double* Ul, int rl,
                     const float* BR, const double* Ur, int rr, double* scratch, double* result2,
                     cudaStream_t st);
// Expand U_S = (U_l (x) U_r) B_S^(1)T in float64: Uout[(a nr + b)][i] = sum_jk Ul[a][j] B[i][j][k] Ur[b][k]
int launch_ht_expand(const double* Ul, int64_t nl, int rl, const double* Ur, int64_t nr, int rr,
                     const float* B, int rS, double* Uout, cudaStream_t st);
int launch_f32_to_f64(const float* in, double* out, int64_t n, cudaStream_t st);
size_t ht_relerr_scratch(int64_t nl, int64_t nr);

}  // namespace rt
