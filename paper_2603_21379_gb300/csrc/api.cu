// api.cu - C ABI of the rtucker library (declared in include/rtucker.h).
//
// Host orchestration only: argument checks, planning the grouped problem
// tables, the device workspace, and the launch sequence.  Every step of the
// decomposition runs in this library's CUDA kernels; there is no CPU path.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <cstdlib>

#include <algorithm>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "../../include/rtucker.h"
#include "rt_common.cuh"
#include "rt_host.h"

using namespace rt;

// One table upload: `words` 8-byte words from staging offset `src` to `dst`.
struct StageSeg {
  uint64_t* dst;
  size_t src;
  int64_t words;
};

namespace {

// Table uploads are read by a kernel straight from the mapped pinned staging
// buffer instead of being copied by the copy engine: a decomposition that
// waits behind a large host-to-device copy of the next tensor (the pipelined
// host call) would otherwise wait for that copy before its first kernel.
constexpr int UP_MAX = 16;            // segments per launch
constexpr int UP_CHUNK = 256 * 4;     // words per CTA (4 independent loads per thread)

struct UploadBatch {
  int nseg;
  int cta0[UP_MAX + 1];               // first CTA of each segment
  uint64_t* dst[UP_MAX];
  const uint64_t* src[UP_MAX];
  int64_t words[UP_MAX];
};

__global__ void __launch_bounds__(256) k_stage_copy(const UploadBatch b) {
  int sg = 0;
  while (sg + 1 < b.nseg && (int)blockIdx.x >= b.cta0[sg + 1]) ++sg;
  const int64_t w0 = (int64_t)(blockIdx.x - b.cta0[sg]) * UP_CHUNK;
  const int64_t nw = b.words[sg];
  const uint64_t* __restrict__ src = b.src[sg];
  uint64_t* __restrict__ dst = b.dst[sg];
  uint64_t v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t w = w0 + j * 256 + threadIdx.x;
    v[j] = w < nw ? __ldcv(src + w) : 0;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t w = w0 + j * 256 + threadIdx.x;
    if (w < nw) dst[w] = v[j];
  }
}

}  // namespace

// A captured kernel sequence (rt_options.use_graph) and the launch-shaping arguments
// it was captured for.  Stage-timing intervals recorded during the capture are event
// record nodes of the graph; each launch points them at fresh events.
struct TimedNodes {
  int stage;
  cudaGraphNode_t na, nb;
  cudaEvent_t a0, b0;    // the events recorded at capture (owned by the entry)
};
struct GraphEntry {
  std::vector<uint64_t> key;
  cudaGraph_t graph = nullptr;      // kept: its nodes address the executable's event nodes
  cudaGraphExec_t exec = nullptr;
  std::vector<TimedNodes> timed;
  int launches = 0;
  uint64_t used = 0;
};
constexpr size_t GRAPH_CACHE = 4;   // captured sequences kept per handle (least recently used replaced)

struct rt_handle_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  char* ws = nullptr;          // device workspace
  size_t ws_bytes = 0;
  int* d_status = nullptr;     // device status word
  int* h_status = nullptr;     // pinned copy of the status word
  cudaEvent_t ev_status = nullptr;
  bool status_pending = false;
  char* h_stage = nullptr;     // pinned staging of the problem tables
  char* d_stage = nullptr;     // the same buffer as the device addresses it
  size_t h_stage_bytes = 0;
  std::vector<StageSeg> stage_segs;  // uploads not yet enqueued
  // the last table upload: skipped when the next one is identical and nothing else
  // used the workspace in between (ws_epoch counts workspace users)
  uint64_t ws_epoch = 0, commit_epoch = ~0ull;
  std::vector<StageSeg> last_segs;
  std::vector<uint64_t> last_words;
  cudaEvent_t ev_stage = nullptr;
  bool stage_pending = false;
  std::string err;
  int launches = 0;
  char* hc_buf = nullptr;      // device buffers of rtucker_decompose_host
  size_t hc_bytes = 0;
  // rtucker_decompose_host_async: two device input slots filled on a copy
  // stream (slot k is reused once the decomposition that read it has run),
  // one device output area read back on the handle's stream
  cudaStream_t cstream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  char* pipe_buf = nullptr;
  size_t pipe_slot = 0, pipe_out = 0;
  int pipe_next = 0;
  // second stream for work that overlaps the pass over X, with fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // core kernels picked by timing (rt_options.core = 3), per shape
  std::map<std::vector<int64_t>, int> core_tuned;
  std::map<std::vector<int64_t>, std::vector<int>> batched_tuned;   // per-level schedules
  std::vector<int> last_schedule;   // the last batched call's per-level schedules
  // CUDA-graph replay: capture stream and cache
  cudaStream_t gstream = nullptr;
  bool capturing = false;            // a graph capture is running (stage timing records nodes)
  std::vector<GraphEntry> graphs;
  uint64_t graph_tick = 0;
  // stage timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;              // free events
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_open;  // recorded intervals
  double stage_ms[RT_NSTAGES] = {0};
  int64_t stage_cnt[RT_NSTAGES] = {0};
  // injected host-side failures (rt_inject_fault, environment RT_FAULT=alloc[:count])
  int fault_alloc = 0;         // the next this many workspace growths fail as a failed cudaMalloc
  int grad_recompute = 0;      // rt_set_grad_recompute: partial projections without kept prefixes
};

namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

rt_status fail(rt_handle h, rt_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

rt_status cuda_fail(rt_handle h, cudaError_t e, const char* where) {
  return fail(h, RT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RT_CUDA(h, call)                                  \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #call); \
  } while (0)

cudaEvent_t pool_event(rt_handle h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets the launches enqueued between begin() and end() with two events.
struct StageTimer {
  rt_handle h;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageTimer(rt_handle hh, int s, cudaStream_t stream = nullptr) : h(hh), stage(s), st(stream ? stream : hh->stream) {
    if (h->timing) {
      a = pool_event(h);
      record(a);
    }
  }
  ~StageTimer() {
    if (a) {
      cudaEvent_t b = pool_event(h);
      record(b);
      h->ev_open.push_back({stage, {a, b}});
    }
  }
  // under graph capture the record becomes an event-record node of the graph
  void record(cudaEvent_t e) {
    if (h->capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
};

void drain_timing(rt_handle h) {
  for (auto& it : h->ev_open) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, it.second.first, it.second.second) == cudaSuccess) {
      h->stage_ms[it.first] += ms;
      h->stage_cnt[it.first] += 1;
    }
    h->ev_pool.push_back(it.second.first);
    h->ev_pool.push_back(it.second.second);
  }
  h->ev_open.clear();
}

int dtype_size(rt_dtype t) { return t == RT_F64 ? 8 : t == RT_BF16 ? 2 : t == RT_F8E4M3 ? 1 : 4; }

// Packed float8 storage: codes (prod n bytes), then at the element count rounded up
// to 256 bytes one float32 scale per slab of the last two modes.
size_t fp8_scale_offset(int d, const int64_t* n) {
  size_t t = 1;
  for (int k = 0; k < d; ++k) t *= (size_t)n[k];
  return (t + 255) & ~(size_t)255;
}

int64_t fp8_slabs(int d, const int64_t* n) {
  int64_t S = 1;
  for (int k = 0; k + 2 < d; ++k) S *= n[k];
  return S;
}

const float* fp8_scales(const void* X, int d, const int64_t* n) {
  return reinterpret_cast<const float*>(static_cast<const char*>(X) + fp8_scale_offset(d, n));
}

bool mul_ok(int64_t a, int64_t b, int64_t* out) {
  if (a <= 0 || b <= 0) return false;
  if (a > (int64_t)(((uint64_t)1 << 62) / (uint64_t)b)) return false;
  *out = a * b;
  return true;
}

int feistel_half(int64_t N) {
  // smallest even b >= 2 with 2^b >= N; returns b / 2
  int b = 0;
  uint64_t v = (uint64_t)(N - 1);
  while (v) { ++b; v >>= 1; }
  if (b < 2) b = 2;
  b += (b & 1);
  return b / 2;
}

inline int odd(int m) { return m | 1; }

// Bump allocator over the device workspace.
struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  }
};

// --- range-finder problem planning ------------------------------------------
struct ProbSpec {
  const void* X;
  rt_dtype dtype;
  int d;
  int64_t n[MAXD];
  int a, b;           // contiguous mode range S
  int r, p;
  int64_t s;
  uint64_t seed;
  uint32_t node;
  float* U;           // output (device) or null -> workspace
  float* sigma_out;
  int64_t* idx_out;   // sampled indices straight to the caller (or null)
  int qr;             // rt_options.qr: 0 auto, 1 Householder / TSQR, 2 Cholesky form
  int sketch;         // rt_options.sketch: 1 = bfloat16 sketch
};

struct ProbPlan {
  RFProb q;
  size_t o_idx, o_off, o_Om, o_Yt, o_Zp, o_zcnt, o_Q, o_Rb, o_Q2, o_tsR, o_tsQ, o_Bp, o_Rc, o_W, o_Wsg, o_sig,
      o_keys, o_U, o_wsR, o_Cp;
  int64_t units[STG_ALL];
};

rt_status plan_problem(rt_handle h, const ProbSpec& ps, Bump& bump, ProbPlan& pp) {
  RFProb& q = pp.q;
  memset(&q, 0, sizeof(q));
  for (int64_t& u : pp.units) u = 0;
  const int d = ps.d;
  int64_t stride[MAXD];
  stride[d - 1] = 1;
  for (int j = d - 2; j >= 0; --j) stride[j] = stride[j + 1] * ps.n[j + 1];
  int64_t nS = 1, N = 1;
  for (int j = ps.a; j <= ps.b; ++j) nS *= ps.n[j];
  q.ncm = 0;
  for (int j = 0; j < d; ++j) {
    if (j >= ps.a && j <= ps.b) continue;
    q.csize[q.ncm] = ps.n[j];
    q.cstride[q.ncm] = stride[j];
    ++q.ncm;
    N *= ps.n[j];
  }
  const int c = ps.r + ps.p;
  if (ps.r < 1 || ps.p < 0) return fail(h, RT_EINVAL, "need r >= 1 and p >= 0");
  if (c > nS || c > N) return fail(h, RT_EINVAL, "need r + p <= min(n_S, n_notin_S) (node " + std::to_string(ps.node) + ")");
  if (ps.s < c || ps.s > N) return fail(h, RT_EINVAL, "need r + p <= s <= n_notin_S (node " + std::to_string(ps.node) + ")");
  if (c > CMAX) return fail(h, RT_ENOTSUP, "r + p > 64 is not supported");
  if (nS >= ((int64_t)1 << 31)) return fail(h, RT_ENOTSUP, "unfolding with 2^31 or more rows");
  q.X = ps.X;
  q.dtype = (int)ps.dtype;
  if (ps.dtype == RT_F8E4M3) {
    q.xsc = fp8_scales(ps.X, d, ps.n);
    q.xslab = ps.n[d - 2] * ps.n[d - 1];
  }
  q.nS = nS;
  q.N = N;
  q.rowstride = stride[ps.b];
  q.r = ps.r;
  q.c = c;
  q.s = ps.s;
  q.seed = ps.seed;
  q.node = ps.node;
  q.fh = feistel_half(N);
  q.nzc = (int)((ps.s + SK_TJ - 1) / SK_TJ);
  q.skbf16 = ps.sketch == 1 ? 1 : 0;
  // Cholesky form of S5 / S6 (rt_options.qr): unfoldings of at most QWF_MAX rows whose
  // Z also fits the single-block Householder QR it falls back to
  const bool chol = ps.qr != 1 && nS <= QWF_MAX && (int64_t)odd((int)nS) * c <= QR_MAXF;   // W-step
  // S5 by CholeskyQR2 when asked, and in the BF16 form (its second pass restores the
  // orthogonality the bfloat16 sketch does not need to carry)
  const bool chol_z = chol && (ps.qr == 2 || ps.qr == 3 || (ps.qr == 0 && ps.sketch == 1));
  q.zshift = (chol_z && ps.qr == 3) ? 1 : 0;
  // TSQR of Z
  int rb = (QR_MAXF / c - 1) & ~31;
  if (rb < 32) rb = 32;
  if (odd((int)std::min<int64_t>(nS, 1 << 30)) * (int64_t)c <= QR_MAXF) {
    q.nrb = 1;
    q.rbrows = (int)nS;
  } else {
    q.rbrows = rb;
    if ((nS + rb - 1) / rb > (1 << 30)) return fail(h, RT_ENOTSUP, "unfolding too tall for the TSQR");
    q.nrb = (int)((nS + rb - 1) / rb);
    // TSQR tree: groups of up to `fan` stacked R factors per level (the largest
    // stack the level kernel holds), until one group is left
    int fan = 1;
    while ((int64_t)odd((fan + 1) * c) * c <= QR2_MAXF) ++fan;
    q.fan = fan;
    q.lev_n[0] = q.nrb;
    int64_t cnt = q.nrb;
    while (cnt > 1) {
      if (q.nlev == TS_MAXLEV) return fail(h, RT_ENOTSUP, "unfolding too tall for the TSQR tree");
      cnt = (cnt + fan - 1) / fan;
      q.lev_n[++q.nlev] = (int)cnt;
    }
  }
  q.scrows = BT_SC;
  q.nsc = chol ? 0 : (int)((ps.s + BT_SC - 1) / BT_SC);
  q.nbi = chol ? 0 : (int)((nS + BT_IB - 1) / BT_IB);
  q.nbg = chol ? (int)((ps.s + BG_SC - 1) / BG_SC) : 0;
  // more chunk factors than the W-step stacks: an R tree over them first
  int wf = 1, tf = 1;
  while ((int64_t)odd((wf + 1) * c) * c <= WS_MAXF) ++wf;
  while ((int64_t)odd((tf + 1) * c) * c <= QR2_MAXF) ++tf;
  q.wfan = tf;
  q.wn[0] = q.nsc;
  int64_t wcnt = q.nsc;
  while (!chol && wcnt > wf) {
    if (q.wlev == TS_MAXLEV) return fail(h, RT_ENOTSUP, "too many samples for the W-step");
    wcnt = (wcnt + tf - 1) / tf;
    q.wn[++q.wlev] = (int)wcnt;
  }
  q.nrw = (int)wcnt;
  const int64_t s = ps.s;
  pp.o_idx = ps.idx_out ? (size_t)-1 : bump.take(s * 8);
  pp.o_off = bump.take(s * 8);
  pp.o_Om = bump.take(s * c * 4);
  pp.o_Yt = bump.take((size_t)s * nS * 4);
  pp.o_Zp = bump.take((size_t)q.nzc * nS * c * 4);
  pp.o_zcnt = bump.take((size_t)((nS + SK_TI - 1) / SK_TI) * 4);
  pp.o_Q = bump.take((size_t)nS * c * 4);
  pp.o_Rb = bump.take(q.nrb > 1 ? (size_t)q.nrb * c * c * 4 : 4);
  pp.o_Q2 = bump.take(q.nrb > 1 ? (size_t)q.nrb * c * c * 4 : 4);
  size_t upper = 0;   // factors entering levels 1 .. nlev-1
  for (int j = 1; j < q.nlev; ++j) upper += (size_t)q.lev_n[j];
  pp.o_tsR = bump.take(upper ? upper * c * c * 4 : 4);
  pp.o_tsQ = bump.take(upper ? upper * c * c * 4 : 4);
  pp.o_Bp = bump.take(std::max<size_t>(4, (size_t)q.nbi * s * c * 4));
  pp.o_Rc = bump.take(std::max<size_t>(4, (size_t)q.nsc * c * c * 4));
  pp.o_Cp = bump.take(std::max<size_t>(4, (size_t)q.nbg * c * c * 2 * 4));
  size_t wup = 0;   // factors produced by the R tree's levels
  for (int j = 1; j <= q.wlev; ++j) wup += (size_t)q.wn[j];
  pp.o_wsR = bump.take(wup ? wup * c * c * 4 : 4);
  pp.o_W = bump.take((size_t)c * c * 4);
  pp.o_Wsg = bump.take((size_t)c * ps.r * 4);
  pp.o_sig = bump.take((size_t)c * 4);
  pp.o_keys = bump.take((size_t)ps.r * 8);
  pp.o_U = ps.U ? (size_t)-1 : bump.take((size_t)nS * ps.r * 4);
  q.U = ps.U;
  q.sigma_out = ps.sigma_out;
  q.idx = ps.idx_out;
  const int64_t nrt = (nS + SK_TI - 1) / SK_TI;
  pp.units[STG_SAMPLE] = s;
  pp.units[STG_GS] = nrt * q.nzc;
  pp.units[STG_QR1] = chol_z ? 0 : q.nrb;
  for (int j = 0; j < q.nlev; ++j) pp.units[stg_qr2(j)] = q.lev_n[j + 1];      // groups of level j
  for (int t = 0; t + 1 < q.nlev; ++t) pp.units[stg_qrc(t)] = q.lev_n[q.nlev - 2 - t];   // members
  for (int j = 0; j < q.wlev; ++j) pp.units[stg_wt(j)] = q.wn[j + 1];                    // groups
  pp.units[STG_QR3] = q.nrb > 1 ? q.nrb : 0;
  pp.units[STG_BTP] = (int64_t)q.nsc * q.nbi;
  pp.units[STG_BTQ] = q.nsc;
  pp.units[STG_WSVD] = chol ? 0 : 1;
  const bool qw_fused = nS <= QWF_MAX;
  pp.units[STG_QW] = (chol || qw_fused) ? 0 : (nS + QW_TI - 1) / QW_TI;
  pp.units[STG_FLIP] = pp.units[STG_QW];
  pp.units[STG_QWF] = (!chol && qw_fused) ? 1 : 0;
  pp.units[STG_QZ] = chol_z ? 1 : 0;
  pp.units[STG_BTG] = q.nbg;
  pp.units[STG_WSV2] = chol ? 1 : 0;
  pp.units[STG_ZSUM] = nS * c;
  return RT_OK;
}

void bind_problem(ProbPlan& pp, char* ws) {
  RFProb& q = pp.q;
  if (pp.o_idx != (size_t)-1) q.idx = reinterpret_cast<int64_t*>(ws + pp.o_idx);
  q.off = reinterpret_cast<int64_t*>(ws + pp.o_off);
  q.Om = reinterpret_cast<float*>(ws + pp.o_Om);
  q.Yt = reinterpret_cast<float*>(ws + pp.o_Yt);
  q.Zp = reinterpret_cast<float*>(ws + pp.o_Zp);
  q.zcnt = reinterpret_cast<int32_t*>(ws + pp.o_zcnt);
  q.Q = reinterpret_cast<float*>(ws + pp.o_Q);
  q.Rb = reinterpret_cast<float*>(ws + pp.o_Rb);
  q.Q2 = reinterpret_cast<float*>(ws + pp.o_Q2);
  q.tsR = reinterpret_cast<float*>(ws + pp.o_tsR);
  q.tsQ = reinterpret_cast<float*>(ws + pp.o_tsQ);
  q.Bp = reinterpret_cast<float*>(ws + pp.o_Bp);
  q.Rc = reinterpret_cast<float*>(ws + pp.o_Rc);
  q.Cp = reinterpret_cast<float*>(ws + pp.o_Cp);
  q.wsR = reinterpret_cast<float*>(ws + pp.o_wsR);
  if (q.wlev == 0) {
    q.Rw = q.Rc;
  } else {
    size_t o = 0;
    for (int j = 1; j < q.wlev; ++j) o += (size_t)q.wn[j];
    q.Rw = q.wsR + o * q.c * q.c;
  }
  q.W = reinterpret_cast<float*>(ws + pp.o_W);
  q.Wsg = reinterpret_cast<float*>(ws + pp.o_Wsg);
  q.sigma = reinterpret_cast<float*>(ws + pp.o_sig);
  q.keys = reinterpret_cast<unsigned long long*>(ws + pp.o_keys);
  if (!q.U) q.U = reinterpret_cast<float*>(ws + pp.o_U);
}

// Grows the workspace to at least `bytes` (synchronising the stream first).
rt_status ensure_ws(rt_handle h, size_t bytes) {
  ++h->ws_epoch;
  if (bytes <= h->ws_bytes) return RT_OK;
  RT_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  const size_t want = align_up(bytes + bytes / 8);
  cudaError_t e = cudaErrorMemoryAllocation;
  if (h->fault_alloc > 0)
    --h->fault_alloc;      // injected: fails like cudaMalloc, with the old workspace already freed
  else
    e = cudaMalloc(&h->ws, want);
  if (e != cudaSuccess) {
    if (h->ws) cudaGetLastError();   // a real failure: clear its sticky-free error state
    h->ws = nullptr;
    return fail(h, RT_ENOMEM, "device workspace allocation of " + std::to_string(want) + " bytes failed");
  }
  h->ws_bytes = want;
  return RT_OK;
}

rt_status ensure_stage(rt_handle h, size_t bytes) {
  h->stage_segs.clear();  // left over from a call that failed before its commit
  if (h->stage_pending) {
    RT_CUDA(h, cudaEventSynchronize(h->ev_stage));
    h->stage_pending = false;
  }
  if (bytes <= h->h_stage_bytes) return RT_OK;
  if (h->h_stage) cudaFreeHost(h->h_stage);
  h->h_stage = nullptr;
  h->h_stage_bytes = 0;
  h->d_stage = nullptr;
  const size_t want = align_up(bytes * 2);
  RT_CUDA(h, cudaMallocHost(&h->h_stage, want));
  void* dv = nullptr;
  RT_CUDA(h, cudaHostGetDevicePointer(&dv, h->h_stage, 0));
  h->d_stage = static_cast<char*>(dv);
  h->h_stage_bytes = want;
  return RT_OK;
}

// Queues the upload of `bytes` (a multiple of 8) from `src` inside the staging
// buffer to device address `dst` (8-byte aligned).
rt_status stage_put(rt_handle h, void* dst, const void* src, size_t bytes) {
  const size_t off = static_cast<size_t>(static_cast<const char*>(src) - h->h_stage);
  if (bytes % 8 || off % 8 || reinterpret_cast<uintptr_t>(dst) % 8 || off + bytes > h->h_stage_bytes)
    return fail(h, RT_EINVAL, "internal: misaligned table upload");
  if (bytes) h->stage_segs.push_back({static_cast<uint64_t*>(dst), off, (int64_t)(bytes / 8)});
  return RT_OK;
}

// Enqueues the queued uploads on the handle's stream (one launch per UP_MAX
// segments, counted in *nl) and marks the staging buffer busy until they ran.
rt_status stage_commit(rt_handle h, int* nl) {
  std::vector<StageSeg> segs;
  segs.swap(h->stage_segs);
  // identical tables into an untouched workspace: the device copy is still current
  std::vector<uint64_t> words;
  for (const StageSeg& g : segs) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(h->h_stage + g.src);
    words.insert(words.end(), src, src + g.words);
  }
  bool same = h->commit_epoch == h->ws_epoch - 1 && segs.size() == h->last_segs.size() && words == h->last_words;
  for (size_t i = 0; same && i < segs.size(); ++i)
    same = segs[i].dst == h->last_segs[i].dst && segs[i].words == h->last_segs[i].words;
  h->commit_epoch = h->ws_epoch;
  if (same) {
    h->stage_pending = false;   // nothing reads the staging buffer
    return RT_OK;
  }
  h->last_segs = segs;
  h->last_words.swap(words);
  for (size_t i0 = 0; i0 < segs.size(); i0 += UP_MAX) {
    UploadBatch b{};
    b.nseg = (int)std::min<size_t>(UP_MAX, segs.size() - i0);
    int ctas = 0;
    for (int j = 0; j < b.nseg; ++j) {
      const StageSeg& g = segs[i0 + j];
      b.cta0[j] = ctas;
      b.dst[j] = g.dst;
      b.src[j] = reinterpret_cast<const uint64_t*>(h->d_stage + g.src);
      b.words[j] = g.words;
      ctas += (int)((g.words + UP_CHUNK - 1) / UP_CHUNK);
    }
    b.cta0[b.nseg] = ctas;
    k_stage_copy<<<ctas, 256, 0, h->stream>>>(b);
    ++*nl;
  }
  RT_CUDA(h, cudaEventRecord(h->ev_stage, h->stream));
  h->stage_pending = true;
  return RT_OK;
}

rt_status check_prior_status(rt_handle h) {
  if (h->status_pending && cudaEventQuery(h->ev_status) == cudaSuccess) {
    h->status_pending = false;
    const int s = *h->h_status;
    if (s != ST_OK) {
      *h->h_status = 0;
      cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
      if (s == ST_TIMEOUT) return fail(h, RT_ETIMEOUT, "a bounded device loop ran out in an earlier call");
      if (s == ST_NUMERIC) return fail(h, RT_ENUMERIC, "numerical breakdown on the device in an earlier call");
      return fail(h, RT_EDEVICE, "device-side check failed in an earlier call");
    }
  }
  return RT_OK;
}

void post_status_copy(rt_handle h) {
  if (cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
      cudaEventRecord(h->ev_status, h->stream) == cudaSuccess)
    h->status_pending = true;
}

// A grouped range-finder plan with its tables uploaded into the workspace.
struct Group {
  std::vector<ProbPlan> pp;
  size_t o_tab = 0, o_pre = 0;
  RFGroup g{};
};

// Prefix rows a group needs: the fixed stages, plus the tree stages when one of its
// problems has a TSQR tree of two or more levels or an R tree before its W-step.
int group_rows(const Group& G, int* lmax, int* wmax = nullptr) {
  int l = 0, w = 0;
  for (const ProbPlan& p : G.pp) {
    l = std::max(l, (int)p.q.nlev);
    w = std::max(w, (int)p.q.wlev);
  }
  if (lmax) *lmax = l;
  if (wmax) *wmax = w;
  return (l > 1 || w > 0) ? STG_ALL : STG_COUNT;
}

void group_layout(Group& G, Bump& bump) {
  const int np = (int)G.pp.size();
  G.o_tab = bump.take(sizeof(RFProb) * np);
  G.o_pre = bump.take(sizeof(int64_t) * group_rows(G, nullptr) * (np + 1));
}

// Writes the tables into staging and queues their upload; fills G.g.
rt_status group_upload(rt_handle h, Group& G, char* stage, size_t stage_off) {
  const int np = (int)G.pp.size();
  RFProb* tab = reinterpret_cast<RFProb*>(stage + stage_off);
  int64_t* pre = reinterpret_cast<int64_t*>(stage + stage_off + align_up(sizeof(RFProb) * np));
  for (int i = 0; i < np; ++i) {
    bind_problem(G.pp[i], h->ws);
    tab[i] = G.pp[i].q;
  }
  int lmax = 0, wmax = 0;
  const int nst = group_rows(G, &lmax, &wmax);
  for (int st = 0; st < STG_ALL; ++st) {
    int64_t acc = 0;
    for (int i = 0; i < np; ++i) {
      if (st < nst) pre[st * (np + 1) + i] = acc;
      acc += G.pp[i].units[st];
    }
    if (st < nst) pre[st * (np + 1) + np] = acc;
    G.g.total[st] = st < nst ? acc : 0;
  }
  G.g.nst = nst;
  G.g.lmax = lmax;
  G.g.wmax = wmax;
  rt_status st;
  if ((st = stage_put(h, h->ws + G.o_tab, tab, sizeof(RFProb) * np)) != RT_OK) return st;
  if ((st = stage_put(h, h->ws + G.o_pre, pre, sizeof(int64_t) * nst * (np + 1))) != RT_OK) return st;
  G.g.probs = reinterpret_cast<const RFProb*>(h->ws + G.o_tab);
  G.g.pre = reinterpret_cast<const int64_t*>(h->ws + G.o_pre);
  G.g.nprob = np;
  return RT_OK;
}

size_t group_stage_bytes(const Group& G) {
  const int np = (int)G.pp.size();
  return align_up(sizeof(RFProb) * np) + align_up(sizeof(int64_t) * group_rows(G, nullptr) * (np + 1));
}

rt_status check_tensor(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, int64_t* total,
                       bool allow_f8 = false) {
  if (!h) return RT_EINVAL;
  if (!X) return fail(h, RT_EINVAL, "X is null");
  if (dtype == RT_F8E4M3 && !allow_f8)
    return fail(h, RT_ENOTSUP, "float8 storage is taken by rtucker_sketch/factors/core/decompose/relerr only");
  if (dtype != RT_F32 && dtype != RT_F64 && dtype != RT_BF16 && dtype != RT_F8E4M3)
    return fail(h, RT_EINVAL, "unknown dtype");
  if (d < 2 || d > MAXD) return fail(h, RT_EINVAL, "need 2 <= d <= 16");
  if (!n) return fail(h, RT_EINVAL, "n is null");
  int64_t t = 1;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1) return fail(h, RT_EINVAL, "need n_k >= 1");
    if (!mul_ok(t, n[k], &t)) return fail(h, RT_EINVAL, "tensor too large (prod n >= 2^62)");
  }
  if (((uintptr_t)X) % (uintptr_t)(dtype == RT_F8E4M3 ? 16 : dtype_size(dtype)))
    return fail(h, RT_EINVAL, "X is misaligned");
  if (total) *total = t;
  return RT_OK;
}

// Shapes whose float8 storage the library takes: those of the tensor-core pass over X
// (its FP8 form reads the codes with TMA and contracts them with kind::f8f6f4 MMAs).
rt_status check_fp8_shape(rt_handle h, int d, const int64_t* n, const int32_t* r) {
  if (!r) return fail(h, RT_EINVAL, "r is null");
  if (n[d - 2] > 128 || n[d - 1] % 16 != 0 || r[d - 2] > 64 || r[d - 1] > 32 || r[d - 2] < 1 || r[d - 1] < 1)
    return fail(h, RT_ENOTSUP,
                "float8 storage needs n_{d-2} <= 128, n_{d-1} a multiple of 16, r_{d-2} <= 64, r_{d-1} <= 32");
  if (fp8_slabs(d, n) * n[d - 2] >= ((int64_t)1 << 31)) return fail(h, RT_ENOTSUP, "float8 storage: too many rows");
  return RT_OK;
}

rt_status check_opts(rt_handle h, const rt_options* opt) {
  if (!opt) return RT_OK;
  if (opt->prec != RT_PREC_FP32 && opt->prec != RT_PREC_BF16) return fail(h, RT_EINVAL, "unknown precision");
  if (opt->use_graph != 0 && opt->use_graph != 1) return fail(h, RT_EINVAL, "use_graph must be 0 or 1");
  if (opt->core < 0 || opt->core > 3) return fail(h, RT_EINVAL, "core must be 0, 1, 2 or 3");
  if (opt->qr < 0 || opt->qr > 3) return fail(h, RT_EINVAL, "qr must be 0, 1, 2 or 3");
  if (opt->sketch != 0 && opt->sketch != 1) return fail(h, RT_EINVAL, "sketch must be 0 or 1");
  for (int i = 0; i < 2; ++i)
    if (opt->reserved[i]) return fail(h, RT_EINVAL, "reserved option fields must be zero");
  return RT_OK;
}

int64_t default_s(const int64_t* n, int d, int k) {
  int64_t N = 1;
  for (int j = 0; j < d; ++j)
    if (j != k) N *= n[j];
  return std::min<int64_t>(10 * n[k], N);
}

// Tucker problems of one tensor appended to G.
rt_status add_tucker_problems(rt_handle h, Group& G, Bump& bump, const void* X, rt_dtype dtype, int d,
                              const int64_t* n, const int32_t* r, int32_t p, const int64_t* s,
                              uint64_t seed, float* U, float* sigma, int qr, int sketch) {
  size_t uoff = 0, soff = 0;
  for (int k = 0; k < d; ++k) {
    ProbSpec ps{};
    ps.X = X;
    ps.dtype = dtype;
    ps.d = d;
    for (int j = 0; j < d; ++j) ps.n[j] = n[j];
    ps.a = ps.b = k;
    ps.r = r[k];
    ps.p = p;
    ps.s = s ? s[k] : default_s(n, d, k);
    ps.seed = seed;
    ps.node = (uint32_t)k;
    ps.qr = qr;
    ps.sketch = sketch;
    ps.U = U ? U + uoff : nullptr;
    ps.sigma_out = sigma ? sigma + soff : nullptr;
    ProbPlan pp;
    rt_status st = plan_problem(h, ps, bump, pp);
    if (st != RT_OK) return st;
    G.pp.push_back(pp);
    uoff += (size_t)n[k] * r[k];
    soff += (size_t)(r[k] + p);
  }
  return RT_OK;
}

// Core chain sizes: contraction of mode k on (L_k, n_k, R_k) for k = d-1..0.
size_t core_buffer_floats(int d, const int64_t* n, const int32_t* r) {
  size_t best = 0;
  for (int k = d - 1; k >= 1; --k) {  // output of the mode-k step (k >= 1)
    size_t L = 1, R = 1;
    for (int j = 0; j < k; ++j) L *= (size_t)n[j];
    for (int j = k; j < d; ++j) R *= (size_t)r[j];
    best = std::max(best, L * R);
  }
  return best;
}

// Core kernel selection (environment variable RT_CORE_MODE): 1 = tensor-core pass
// over X when the shape allows (default), 0 = FFMA chain only.
int core_mode() {
  static int mode = [] {
    const char* e = getenv("RT_CORE_MODE");
    return e ? atoi(e) : 1;
  }();
  return mode;
}

int prec_of(const rt_options* opt) { return opt ? opt->prec : RT_PREC_FP32; }

int core_of(const rt_options* opt) { return opt ? opt->core : 0; }

int qr_of(const rt_options* opt) { return opt ? opt->qr : 0; }

int sketch_of(const rt_options* opt) { return opt ? opt->sketch : 0; }

// Contractions of the core G = X x_1 U_1^T ... x_d U_d^T, last modes first.  core
// (rt_options.core): 0 auto, 1 tensor-core pass whenever the shape allows, 2 FFMA only
// (also RT_CORE_MODE=0).  Auto takes the tensor-core pass over X for slabs of at least
// TC_MIN_SIDE x TC_MIN_SIDE (its MMA tiles are 128 rows; smaller slabs leave most of
// each tile empty); then, from the last remaining modes down, two modes at a time
// with k_slab2 where a slab fits shared memory, else one mode (after the tensor-core
// pass, on the tensor cores too where the shape allows: k_ttm_tc).  prec RT_PREC_BF16
// rounds float32 X to one bf16 term in the tensor-core pass (the factors and the
// intermediate keep two terms); the FFMA kernels compute in float32.
constexpr int64_t TC_MIN_SIDE = 64;

int enqueue_core(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                 const float* U, float* G, float* bufA, float* bufB, int prec, int core) {
  cudaStream_t st = h->stream;
  int nl = 0;
  size_t uoff[MAXD];
  size_t acc = 0;
  for (int k = 0; k < d; ++k) { uoff[k] = acc; acc += (size_t)n[k] * r[k]; }
  const void* A = X;
  int adt = (int)dtype;
  int ping = 0;
  int k = d - 1;
  bool tc_core = false;     // the tensor-core pass ran: the later one-mode contractions too
  if (core_mode() == 0) core = 2;
  // the last two modes in one tensor-core pass over X, when the shape allows
  const bool tc_pref = core == 1 || (core == 0 && n[d - 2] >= TC_MIN_SIDE && n[d - 1] >= TC_MIN_SIDE) ||
                       (core == 0 && !slab2_fits(n[d - 2], n[d - 1], 1, r[d - 2], r[d - 1]));
  if (dtype == RT_F8E4M3) core = 1;   // the float8 codes are read by the tensor-core pass only
  if (core != 2 && (tc_pref || dtype == RT_F8E4M3) && (dtype == RT_F32 || dtype == RT_BF16 || dtype == RT_F8E4M3) &&
      d >= 2) {
    int64_t S = 1;
    for (int j = 0; j < d - 2; ++j) S *= n[j];
    float* out = (d == 2) ? G : bufA;
    int got = 0;
    {
      StageTimer tm(h, 1);
      const int xmode = (dtype == RT_F8E4M3) ? 3 : (dtype == RT_BF16) ? 1 : (prec == RT_PREC_BF16 ? 2 : 0);
      got = launch_core2_tc(xmode, X, S, (int)n[d - 2], (int)n[d - 1], U + uoff[d - 2],
                            r[d - 2], U + uoff[d - 1], r[d - 1], out, h->d_status, st, 0,
                            dtype == RT_F8E4M3 ? fp8_scales(X, d, n) : nullptr);
    }
    if (got == 0 && dtype == RT_F8E4M3) return -1;   // no other kernel reads the codes
    if (got > 0) {
      nl += got;
      A = out;
      adt = DT_F32;
      ping = 1;
      k = d - 3;
      tc_core = true;
    }
  }
  if (A == X && k == d - 1 && dtype == RT_F32 && last2_fits(n[d - 2], n[d - 1], r[d - 2], r[d - 1])) {
    // the last two modes of float32 X with small slabs: one thread per row, one read
    int64_t S = 1;
    for (int j = 0; j < d - 2; ++j) S *= n[j];
    float* out = (d == 2) ? G : bufA;
    int got = 0;
    {
      StageTimer tm(h, 1);
      got = launch_last2(static_cast<const float*>(X), S, n[d - 2], n[d - 1], U + uoff[d - 2], r[d - 2],
                         U + uoff[d - 1], r[d - 1], out, st);
    }
    if (got > 0) {
      nl += got;
      A = out;
      adt = DT_F32;
      ping = 1;
      k = d - 3;
    }
  }
  while (k >= 0) {
    int64_t R = 1;
    for (int j = k + 1; j < d; ++j) R *= r[j];
    if (k >= 1 && slab2_fits(n[k - 1], n[k], R, r[k - 1], r[k])) {   // modes k-1 and k together
      int64_t L = 1;
      for (int j = 0; j < k - 1; ++j) L *= n[j];
      float* out = (k == 1) ? G : (ping ? bufB : bufA);
      {
        StageTimer tm(h, A == X ? 1 : 2);
        nl += launch_slab2(A, adt, L, n[k - 1], n[k], R, U + uoff[k - 1], r[k - 1], U + uoff[k], r[k], out, st);
      }
      A = out;
      adt = DT_F32;
      ping ^= 1;
      k -= 2;
      continue;
    }
    int64_t L = 1;
    for (int j = 0; j < k; ++j) L *= n[j];
    float* out = (k == 0) ? G : (ping ? bufB : bufA);
    {
      StageTimer tm(h, A == X ? 1 : 2);
      int got = 0;
      if (tc_core && adt == DT_F32)
        got = launch_ttm_tc(static_cast<const float*>(A), L, n[k], R, U + uoff[k], r[k], out, h->d_status, st);
      nl += got > 0 ? got : launch_ttm_t(A, adt, L, n[k], R, U + uoff[k], r[k], out, st);
    }
    A = out;
    adt = DT_F32;
    ping ^= 1;
    --k;
  }
  return nl;
}

// rt_options.core = 3: the core kernels for this shape picked by timing.  On the
// first call for (d, n, r, dtype, prec) each fixed choice (1 tensor-core pass where
// the shape allows, 2 FFMA kernels) runs once to warm up and twice timed with CUDA
// events on the call's own buffers (U may hold anything then: only the time counts;
// G is rewritten by the call itself afterwards); the faster is kept for the handle.
// Stage timing is paused meanwhile.  Returns the choice to use (1 or 2).
rt_status tune_core(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                    const float* U, float* G, float* bufA, float* bufB, int prec, int* choice) {
  std::vector<int64_t> key = {d, (int64_t)dtype, prec};
  for (int k = 0; k < d; ++k) key.push_back(n[k]);
  for (int k = 0; k < d; ++k) key.push_back(r[k]);
  auto it = h->core_tuned.find(key);
  if (it != h->core_tuned.end()) {
    *choice = it->second;
    return RT_OK;
  }
  const bool timing = h->timing;
  h->timing = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.f;
  int pick = 2;
  rt_status st = RT_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = fail(h, RT_ECUDA, "core tuning: event creation");
  } else {
    for (int cand = 1; cand <= 2 && st == RT_OK; ++cand) {
      enqueue_core(h, X, dtype, d, n, r, U, G, bufA, bufB, prec, cand);
      cudaEventRecord(e0, h->stream);
      for (int rep = 0; rep < 2; ++rep) enqueue_core(h, X, dtype, d, n, r, U, G, bufA, bufB, prec, cand);
      cudaEventRecord(e1, h->stream);
      float ms = 0.f;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        st = cuda_fail(h, e, "core tuning");
      } else if (cand == 1 || ms < best) {
        best = ms;
        pick = cand;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->timing = timing;
  if (st != RT_OK) return st;
  h->core_tuned[key] = pick;
  *choice = pick;
  return RT_OK;
}

rt_status ensure_side(rt_handle h) {
  if (h->side) return RT_OK;
  RT_CUDA(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  RT_CUDA(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  RT_CUDA(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  return RT_OK;
}

// The pass over X can run on the QR factors Q_{d-2}, Q_{d-1} (c = r + p columns):
// U_k = Q_k W_k (W_k with the sign rule's signs), so
//     X x_{d-2} U^T x_{d-1} U^T = (X x_{d-2} Q^T x_{d-1} Q^T) x_{d-2} W^T x_{d-1} W^T,
// and the SVD/W/U part of the range finder runs beside it on a second stream.
bool overlap_core_ok(const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r, int32_t p) {
  if (core_mode() < 1 || d < 2) return false;
  if (dtype != RT_F32 && dtype != RT_BF16) return false;
  const int esz = dtype == RT_BF16 ? 2 : 4;
  const int64_t n1 = n[d - 2], n2 = n[d - 1];
  const int c1 = r[d - 2] + p, c2 = r[d - 1] + p;
  int64_t S = 1;
  for (int j = 0; j < d - 2; ++j) S *= n[j];
  if (n1 > 128 || (n2 * esz) % 16 != 0 || c1 > 64 || c2 > 64) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0) return false;
  return S * n1 < ((int64_t)1 << 31);
}

// Buffer floats of the overlapped core: P' (S c1 c2) and every later intermediate.
size_t overlap_buffer_floats(int d, const int64_t* n, const int32_t* r, int32_t p) {
  const size_t c1 = r[d - 2] + p, c2 = r[d - 1] + p;
  size_t L = 1;
  for (int j = 0; j < d - 2; ++j) L *= (size_t)n[j];
  size_t best = L * c1 * c2;
  size_t R = c1 * c2;
  for (int k = d - 3; k >= 0; --k) {   // output of the mode-k contraction
    L /= (size_t)n[k];
    R *= (size_t)r[k];
    best = std::max(best, L * R);
  }
  best = std::max(best, R / c2 * (size_t)r[d - 1]);   // after W_{d-1}
  return best;
}

// Core on the overlapped path: the X pass on Q (already launched by the caller) left
// P' in bufA; contract the leading modes with U, then the last two with W (signed).
int enqueue_core_rest_overlap(rt_handle h, int d, const int64_t* n, const int32_t* r, int32_t p, const float* U,
                              const float* Wsg1, const float* Wsg2, float* G, float* bufA, float* bufB) {
  cudaStream_t st = h->stream;
  int nl = 0;
  size_t uoff[MAXD];
  size_t acc = 0;
  for (int k = 0; k < d; ++k) { uoff[k] = acc; acc += (size_t)n[k] * r[k]; }
  const int64_t c1 = r[d - 2] + p, c2 = r[d - 1] + p;
  const float* A = bufA;
  float* bufs[2] = {bufB, bufA};
  int ping = 0;
  int64_t R = c1 * c2;
  for (int k = d - 3; k >= 0; --k) {
    int64_t L = 1;
    for (int j = 0; j < k; ++j) L *= n[j];
    float* out = bufs[ping];
    nl += launch_ttm_t(A, DT_F32, L, n[k], R, U + uoff[k], r[k], out, st);
    A = out;
    ping ^= 1;
    R *= r[k];
  }
  int64_t Lr = R / (c1 * c2);     // product of r_0 .. r_{d-3}
  float* out = bufs[ping];
  nl += launch_ttm_t(A, DT_F32, Lr * c1, c2, 1, Wsg2, r[d - 1], out, st);   // mode d-1
  nl += launch_ttm_t(out, DT_F32, Lr, c1, r[d - 1], Wsg1, r[d - 2], G, st);  // mode d-2
  return nl;
}

// --- dimension tree (Sec. 4): node {a..b} splits into its first ceil(len/2)
// modes and the rest; nodes numbered level by level, left to right.
struct TNode {
  int a, b, left, right, level;
};

std::vector<TNode> balanced_tree(int d) {
  std::vector<TNode> t;
  t.push_back(TNode{0, d - 1, -1, -1, 0});
  for (size_t q = 0; q < t.size(); ++q) {
    if (t[q].a == t[q].b) continue;
    const int len = t[q].b - t[q].a + 1;
    const int mid = t[q].a + (len + 1) / 2;
    const TNode l{t[q].a, mid - 1, -1, -1, t[q].level + 1};
    const TNode r{mid, t[q].b, -1, -1, t[q].level + 1};
    t[q].left = (int)t.size();
    t.push_back(l);
    t[q].right = (int)t.size();
    t.push_back(r);
  }
  return t;
}

// A dimension tree given as a child table (Alg. 2's input T): tab[2i], tab[2i+1] are
// the left and right children of node i (both -1 for a leaf), node 0 is the root,
// 2d - 1 nodes.  Leaves take the modes 0..d-1 in left-to-right order, so every node
// is a contiguous mode range with its left child's modes first (the row order of
// the set unfoldings and of the Kronecker products in the nestedness relation,
// Sec. 4).  NULL gives the balanced tree.
rt_status tree_of(rt_handle h, int d, const int32_t* tab, std::vector<TNode>& out) {
  if (!tab) {
    out = balanced_tree(d);
    return RT_OK;
  }
  const int nn = 2 * d - 1;
  std::vector<int> parents(nn, 0);
  int nleaf = 0;
  for (int i = 0; i < nn; ++i) {
    const int l = tab[2 * i], r = tab[2 * i + 1];
    if ((l < 0) != (r < 0)) return fail(h, RT_EINVAL, "tree: node " + std::to_string(i) + " has one child");
    if (l < 0) {
      if (l != -1 || r != -1) return fail(h, RT_EINVAL, "tree: a leaf's children must be -1");
      ++nleaf;
      continue;
    }
    if (l >= nn || r >= nn || l == 0 || r == 0 || l == r)
      return fail(h, RT_EINVAL, "tree: children of node " + std::to_string(i) + " out of range");
    ++parents[l];
    ++parents[r];
  }
  if (nleaf != d) return fail(h, RT_EINVAL, "tree: need d leaves");
  for (int i = 1; i < nn; ++i)
    if (parents[i] != 1) return fail(h, RT_EINVAL, "tree: node " + std::to_string(i) + " needs one parent");
  if (d == 1 || tab[0] < 0) return fail(h, RT_EINVAL, "tree: the root must have two children");
  // in-order walk from the root: leaves numbered by mode, ranges and levels
  out.assign(nn, TNode{-1, -1, -1, -1, 0});
  std::vector<int> state(nn, 0), stack{0};
  int mode = 0, visited = 0;
  while (!stack.empty()) {
    const int i = stack.back();
    const int l = tab[2 * i], r = tab[2 * i + 1];
    if (state[i] == 0) {
      ++visited;
      out[i].left = l;
      out[i].right = r;
      if (l < 0) {
        out[i].a = out[i].b = mode++;
        stack.pop_back();
        continue;
      }
      state[i] = 1;
      out[l].level = out[r].level = out[i].level + 1;
      stack.push_back(r);
      stack.push_back(l);
    } else {
      out[i].a = out[l].a;
      out[i].b = out[r].b;
      stack.pop_back();
    }
    if ((int)stack.size() > nn) break;
  }
  if (visited != nn || mode != d) return fail(h, RT_EINVAL, "tree: not every node is reachable from the root");
  return RT_OK;
}

int64_t range_prod(const int64_t* n, int a, int b) {
  int64_t v = 1;
  for (int j = a; j <= b; ++j) v *= n[j];
  return v;
}

bool g_attrs_done[64] = {false};

rt_status init_device_attrs(rt_handle h) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && g_attrs_done[dev]) return RT_OK;
  RT_CUDA(h, rf_init_attributes());
  RT_CUDA(h, core_init_attributes());
  if (dev >= 0 && dev < 64) g_attrs_done[dev] = true;
  return RT_OK;
}

rt_status finish(rt_handle h, int launches) {
  h->launches = launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
  post_status_copy(h);
  return RT_OK;
}

// Launch-shaping arguments of a call, as words: a captured sequence is replayed only
// for calls whose words match (pointers, shapes, stage unit totals, workspace base
// and layout).  Everything else the kernels read (the problem tables: seeds, sample
// indices' parameters) is uploaded by each call before its sequence runs.
struct GraphKey {
  std::vector<uint64_t> w;
  void add(uint64_t v) { w.push_back(v); }
  void ptr(const void* p) { w.push_back((uint64_t)(uintptr_t)p); }
  template <typename T>
  void arr(const T* a, int n) {
    w.push_back((uint64_t)n);
    for (int i = 0; i < n; ++i) w.push_back((uint64_t)a[i]);
  }
  void group(const RFGroup& g) {
    add((uint64_t)g.nprob);
    add((uint64_t)g.nst);
    add((uint64_t)g.lmax);
    add((uint64_t)g.wmax);
    ptr(g.probs);
    ptr(g.pre);
    for (int i = 0; i < STG_ALL; ++i) add((uint64_t)g.total[i]);
  }
};

void release_graph(rt_handle h, GraphEntry& ge) {
  if (ge.exec) cudaGraphExecDestroy(ge.exec);
  if (ge.graph) cudaGraphDestroy(ge.graph);
  for (TimedNodes& t : ge.timed) {
    h->ev_pool.push_back(t.a0);
    h->ev_pool.push_back(t.b0);
  }
  ge = GraphEntry{};
}

rt_status launch_graph(rt_handle h, GraphEntry& ge) {
  for (const TimedNodes& t : ge.timed) {
    cudaEvent_t a = pool_event(h), b = pool_event(h);
    RT_CUDA(h, cudaGraphExecEventRecordNodeSetEvent(ge.exec, t.na, a));
    RT_CUDA(h, cudaGraphExecEventRecordNodeSetEvent(ge.exec, t.nb, b));
    h->ev_open.push_back({t.stage, {a, b}});
  }
  RT_CUDA(h, cudaGraphLaunch(ge.exec, h->stream));
  ge.used = ++h->graph_tick;
  return RT_OK;
}

// Runs enqueue(&launches) on the handle's stream, directly or (use_graph) as a CUDA
// graph: a cached one when the key matches, else captured on a private stream (so
// that the caller's stream may be the legacy default stream), instantiated and
// launched on the handle's stream.
template <class F>
rt_status run_kernels(rt_handle h, bool use_graph, GraphKey key, int* nl, F&& enqueue) {
  if (!use_graph) {
    int n = 0;
    const rt_status st = enqueue(&n);
    *nl += n;
    return st;
  }
  key.add(h->timing ? 1 : 0);
  for (GraphEntry& ge : h->graphs)
    if (ge.key == key.w) {
      rt_status st;
      if ((st = launch_graph(h, ge)) != RT_OK) return st;
      *nl += ge.launches;
      return RT_OK;
    }
  if (!h->gstream) RT_CUDA(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
  const size_t ev0 = h->ev_open.size();
  RT_CUDA(h, cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed));
  cudaStream_t user = h->stream;
  h->stream = h->gstream;
  h->capturing = true;
  int n = 0;
  const rt_status st = enqueue(&n);
  h->capturing = false;
  h->stream = user;
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->gstream, &g);
  // the stage intervals opened during the capture belong to the graph
  GraphEntry ne;
  for (size_t i = ev0; i < h->ev_open.size(); ++i)
    ne.timed.push_back({h->ev_open[i].first, nullptr, nullptr, h->ev_open[i].second.first,
                        h->ev_open[i].second.second});
  h->ev_open.resize(ev0);
  ne.graph = g;
  if (st != RT_OK || ec != cudaSuccess || !g) {
    release_graph(h, ne);
    cudaGetLastError();
    return st != RT_OK ? st : cuda_fail(h, ec != cudaSuccess ? ec : cudaErrorUnknown, "graph capture");
  }
  if (!ne.timed.empty()) {
    size_t cnt = 0;
    RT_CUDA(h, cudaGraphGetNodes(g, nullptr, &cnt));
    std::vector<cudaGraphNode_t> nodes(cnt);
    RT_CUDA(h, cudaGraphGetNodes(g, nodes.data(), &cnt));
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      RT_CUDA(h, cudaGraphNodeGetType(nd, &ty));
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev = nullptr;
      RT_CUDA(h, cudaGraphEventRecordNodeGetEvent(nd, &ev));
      for (TimedNodes& t : ne.timed) {
        if (t.a0 == ev) t.na = nd;
        if (t.b0 == ev) t.nb = nd;
      }
    }
    for (const TimedNodes& t : ne.timed)
      if (!t.na || !t.nb) {
        release_graph(h, ne);
        return fail(h, RT_ECUDA, "graph capture: stage-timing events not found");
      }
  }
  const cudaError_t ei = cudaGraphInstantiate(&ne.exec, g, 0);
  if (ei != cudaSuccess) {
    ne.exec = nullptr;
    release_graph(h, ne);
    return cuda_fail(h, ei, "graph instantiate");
  }
  ne.key = key.w;
  ne.launches = n;
  GraphEntry* slot = nullptr;
  if (h->graphs.size() < GRAPH_CACHE) {
    h->graphs.push_back(GraphEntry{});
    slot = &h->graphs.back();
  } else {
    slot = &h->graphs[0];
    for (GraphEntry& ge : h->graphs)
      if (ge.used < slot->used) slot = &ge;
    release_graph(h, *slot);
  }
  *slot = std::move(ne);
  rt_status sl;
  if ((sl = launch_graph(h, *slot)) != RT_OK) return sl;
  *nl += n;
  return RT_OK;
}

// Full Tucker pipeline for one tensor: tables, range finder, optional core.
rt_status tucker_run(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                     int32_t p, const int64_t* s, uint64_t seed, const rt_options* opt, float* U,
                     float* sigma, float* G, float* Zout) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, nullptr, true)) != RT_OK) return st;
  if ((st = check_opts(h, opt)) != RT_OK) return st;
  if (!r) return fail(h, RT_EINVAL, "r is null");
  if (dtype == RT_F8E4M3 && (st = check_fp8_shape(h, d, n, r)) != RT_OK) return st;
  if (dtype == RT_F8E4M3 && core_of(opt) == 2) return fail(h, RT_ENOTSUP, "float8 storage needs the tensor-core pass");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  if ((st = init_device_attrs(h)) != RT_OK) return st;
  Group Gp;
  Bump bump;
  st = add_tucker_problems(h, Gp, bump, X, dtype, d, n, r, p, s, seed, U, sigma, qr_of(opt), sketch_of(opt));
  if (st != RT_OK) return st;
  group_layout(Gp, bump);
  size_t o_zp = 0;
  if (Zout) o_zp = bump.take(sizeof(float*) * d);
  size_t o_bufA = 0, o_bufB = 0;
  const bool overlap = opt && opt->overlap && G && U && !Zout && overlap_core_ok(X, dtype, d, n, r, p);
  if (G) {
    size_t cb = core_buffer_floats(d, n, r);
    if (overlap) cb = std::max(cb, overlap_buffer_floats(d, n, r, p));
    o_bufA = bump.take(cb * 4);
    o_bufB = bump.take(cb * 4);
  }
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  const size_t sb = group_stage_bytes(Gp) + align_up(sizeof(float*) * d);
  if ((st = ensure_stage(h, sb)) != RT_OK) return st;
  if ((st = group_upload(h, Gp, h->h_stage, 0)) != RT_OK) return st;
  int nl = 0;
  if (Zout) {
    float** zp = reinterpret_cast<float**>(h->h_stage + group_stage_bytes(Gp));
    size_t off = 0;
    for (int k = 0; k < d; ++k) { zp[k] = Zout + off; off += (size_t)n[k] * (r[k] + p); }
    if ((st = stage_put(h, h->ws + o_zp, zp, sizeof(float*) * d)) != RT_OK) return st;
  }
  if ((st = stage_commit(h, &nl)) != RT_OK) return st;
  if (overlap && (st = ensure_side(h)) != RT_OK) return st;
  if (G && !U) return fail(h, RT_EINVAL, "U is required with G");
  int core = core_of(opt);
  if (core == 3 && dtype == RT_F8E4M3) core = 1;
  if (core == 3) {
    if (G && !overlap) {
      if ((st = tune_core(h, X, dtype, d, n, r, U, G, reinterpret_cast<float*>(h->ws + o_bufA),
                          reinterpret_cast<float*>(h->ws + o_bufB), prec_of(opt), &core)) != RT_OK)
        return st;
    } else {
      core = 0;
    }
  }
  const bool graph = opt && opt->use_graph;
  GraphKey key;
  if (graph) {
    key.add(1);
    key.add((uint64_t)h->device);
    key.ptr(h->ws);
    key.add(bump.off);
    key.ptr(X);
    key.add((uint64_t)dtype);
    key.arr(n, d);
    key.arr(r, d);
    key.add((uint64_t)p);
    key.ptr(U);
    key.ptr(sigma);
    key.ptr(G);
    key.ptr(Zout);
    key.add((uint64_t)prec_of(opt));
    key.add((uint64_t)core_of(opt));
    key.add(overlap ? 1 : 0);
    key.add(o_zp);
    key.add(o_bufA);
    key.add(o_bufB);
    key.group(Gp.g);
  }
  st = run_kernels(h, graph, key, &nl, [&](int* nk) -> rt_status {
    if (overlap) {
      {
        StageTimer tm(h, 0);
        *nk += launch_rf_head(Gp.g, h->stream, h->d_status);
      }
      RT_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
      RT_CUDA(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      {
        StageTimer tm(h, 5, h->side);
        *nk += launch_rf_tail(Gp.g, h->side, h->d_status);
      }
      RT_CUDA(h, cudaEventRecord(h->ev_join, h->side));
      const RFProb& q1 = Gp.pp[d - 2].q;
      const RFProb& q2 = Gp.pp[d - 1].q;
      int64_t S = 1;
      for (int j = 0; j < d - 2; ++j) S *= n[j];
      int nsm = 148;
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
      const int xmode = (dtype == RT_BF16) ? 1 : (prec_of(opt) == RT_PREC_BF16 ? 2 : 0);
      float* bufA = reinterpret_cast<float*>(h->ws + o_bufA);
      float* bufB = reinterpret_cast<float*>(h->ws + o_bufB);
      int got = 0;
      {
        StageTimer tm(h, 1);
        // leave one SM per problem to the SVD part running beside the pass
        got = launch_core2_tc(xmode, X, S, (int)n[d - 2], (int)n[d - 1], q1.Q, q1.c, q2.Q, q2.c, bufA,
                              h->d_status, h->stream, std::max(1, nsm - d));
      }
      RT_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
      if (got > 0) {
        *nk += got;
        StageTimer tm(h, 2);
        *nk += enqueue_core_rest_overlap(h, d, n, r, p, U, q1.Wsg, q2.Wsg, G, bufA, bufB);
      } else {
        *nk += enqueue_core(h, X, dtype, d, n, r, U, G, bufA, bufB, prec_of(opt), core);
      }
      return RT_OK;
    }
    {
      StageTimer tm(h, 0);
      *nk += launch_range_finder(Gp.g, h->stream, h->d_status);
    }
    if (Zout) *nk += launch_sketch_sum(Gp.g, reinterpret_cast<float* const*>(h->ws + o_zp), h->stream);
    if (G) {
      const int got = enqueue_core(h, X, dtype, d, n, r, U, G, reinterpret_cast<float*>(h->ws + o_bufA),
                                   reinterpret_cast<float*>(h->ws + o_bufB), prec_of(opt), core);
      if (got < 0) return fail(h, RT_ENOTSUP, "float8 storage: the tensor-core pass did not take the shape");
      *nk += got;
    }
    return RT_OK;
  });
  if (st != RT_OK) return st;
  return finish(h, nl);
}

// Kronecker-structured sketch (rHKron, Sec. 3.3): checks, launch shape and workspace.
struct KronPlan {
  KronArgs a{};
  int grid = 0;
  size_t o_om = 0, o_p1 = 0, o_p2 = 0, o_ts = 0, o_wt = 0;
  int64_t L[MAXD];
};

rt_status plan_kron(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* ell,
                    Bump& bump, KronPlan& kp) {
  if (!ell) return fail(h, RT_EINVAL, "ell is null");
  if (d < 3) return fail(h, RT_ENOTSUP, "the Kronecker sketch needs d >= 3");
  KronArgs& a = kp.a;
  a.X = X;
  a.dtype = (int)dtype;
  a.d = d;
  int64_t K = 1, S = 1;
  a.om_off[0] = 0;
  for (int j = 0; j < d; ++j) {
    if (ell[j] < 1 || ell[j] > n[j]) return fail(h, RT_EINVAL, "need 1 <= l_j <= n_j");
    a.n[j] = n[j];
    a.ell[j] = ell[j];
    a.om_off[j + 1] = a.om_off[j] + n[j] * ell[j];
    if (j < d - 2) {
      K *= ell[j];
      S *= n[j];
    }
  }
  for (int k = 0; k < d; ++k) {
    kp.L[k] = 1;
    for (int j = 0; j < d; ++j)
      if (j != k) kp.L[k] *= ell[j];
  }
  a.om_total = a.om_off[d];
  a.S = S;
  a.n1 = (int)n[d - 2];
  a.n2 = (int)n[d - 1];
  a.la = ell[d - 2];
  a.lb = ell[d - 1];
  if (a.la > KRON_LMAX || a.lb > KRON_LMAX) return fail(h, RT_ENOTSUP, "l_{d-2} and l_{d-1} must be at most 8");
  if (n[d - 1] % 4 != 0 || n[d - 2] > 1024 || n[d - 1] > 1024)
    return fail(h, RT_ENOTSUP, "the Kronecker sketch needs n_{d-1} a multiple of 4 and n_{d-2}, n_{d-1} <= 1024");
  a.K = (int)std::min<int64_t>(K, 1 << 20);
  if (K > 1024 || n[d - 2] > 256 || n[d - 1] > 256 || !kron_shares_fit(a))
    return fail(h, RT_ENOTSUP,
                "the Kronecker sketch needs n_{d-2}, n_{d-1} <= 256 and ceil(K / (256 / n)) max(4, l) <= 32 for "
                "n = n_{d-2}, n_{d-1}, K the product of the leading l_j");
  if (dtype == RT_F32 && ((uintptr_t)X & 15u)) return fail(h, RT_EINVAL, "float32 X must be 16-byte aligned");
  a.K = (int)K;
  const int nq = a.n2 / 4;
  a.ha = std::max(1, std::min(256 / std::max(1, a.n1), nq));
  a.hb = std::max(1, std::min(256 / std::max(1, nq), a.n1));
  if (kron_sketch_smem(a) > 227 * 1024) return fail(h, RT_ENOTSUP, "the Kronecker sketch's slab does not fit shared memory");
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (S * K >= ((int64_t)1 << 31) || S * a.la * a.lb >= ((int64_t)1 << 31))
    return fail(h, RT_ENOTSUP, "the Kronecker sketch: too many slabs");
  kp.grid = (int)std::min<int64_t>(S, nsm);
  kp.o_om = bump.take((size_t)a.om_total * 4);
  kp.o_p1 = bump.take((size_t)kp.grid * a.n1 * K * a.lb * 4);
  kp.o_p2 = bump.take((size_t)kp.grid * a.n2 * K * a.la * 4);
  kp.o_ts = bump.take((size_t)S * a.la * a.lb * 4);
  kp.o_wt = bump.take((size_t)S * K * 4);
  return RT_OK;
}

void bind_kron(KronPlan& kp, char* ws) {
  kp.a.om = reinterpret_cast<float*>(ws + kp.o_om);
  kp.a.part1 = reinterpret_cast<float*>(ws + kp.o_p1);
  kp.a.part2 = reinterpret_cast<float*>(ws + kp.o_p2);
  kp.a.Ts = reinterpret_cast<float*>(ws + kp.o_ts);
  kp.a.Wt = reinterpret_cast<float*>(ws + kp.o_wt);
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

int rt_version(void) { return 2; }

const char* rt_status_string(rt_status s) {
  switch (s) {
    case RT_OK: return "ok";
    case RT_EINVAL: return "invalid argument";
    case RT_ENOMEM: return "out of device memory";
    case RT_ECUDA: return "CUDA error";
    case RT_ETIMEOUT: return "device loop bound exceeded";
    case RT_EDEVICE: return "device-side check failed";
    case RT_ENUMERIC: return "numerical breakdown";
    case RT_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

rt_status rt_create(rt_handle* out, void* stream) {
  if (!out) return RT_EINVAL;
  *out = nullptr;
  rt_handle h = new rt_handle_s();
  h->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&h->device);
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return RT_ENOMEM;
  }
  if (cudaMallocHost(&h->h_status, sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_status, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_stage, cudaEventDisableTiming) != cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rt_destroy(h);
    return RT_ECUDA;
  }
  *h->h_status = 0;
  // RT_FAULT=alloc[:count]: the handle's next `count` (default 1) workspace growths fail
  if (const char* f = std::getenv("RT_FAULT")) {
    if (strncmp(f, "alloc", 5) == 0) h->fault_alloc = (f[5] == ':') ? std::max(0, atoi(f + 6)) : 1;
  }
  *out = h;
  return RT_OK;
}

rt_status rt_inject_fault(rt_handle h, int kind, int count) {
  if (!h || count < 0) return RT_EINVAL;
  if (kind != RT_FAULT_ALLOC) return fail(h, RT_EINVAL, "unknown fault kind");
  h->fault_alloc = count;
  return RT_OK;
}

rt_status rt_set_wait_limit(rt_handle h, uint32_t polls) {
  if (!h) return RT_EINVAL;
  int cur = 0;
  RT_CUDA(h, cudaGetDevice(&cur));
  if (cur != h->device) RT_CUDA(h, cudaSetDevice(h->device));
  cudaError_t e = core_tc_set_wait_limit(polls);
  if (e == cudaSuccess) e = root_tma_set_wait_limit(polls);
  if (e == cudaSuccess) e = diag_set_wait_limit(polls);
  if (cur != h->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_fail(h, e, "rt_set_wait_limit");
  return RT_OK;
}

rt_status rt_set_grad_recompute(rt_handle h, int enable) {
  if (!h || (enable != 0 && enable != 1)) return RT_EINVAL;
  h->grad_recompute = enable;
  return RT_OK;
}

size_t rt_fp8_scale_offset(int d, const int64_t* n) {
  if (d < 2 || d > MAXD || !n) return 0;
  int64_t t = 1;
  for (int k = 0; k < d; ++k)
    if (n[k] < 1 || !mul_ok(t, n[k], &t)) return 0;
  return fp8_scale_offset(d, n);
}

size_t rt_fp8_bytes(int d, const int64_t* n) {
  const size_t off = rt_fp8_scale_offset(d, n);
  if (!off) return 0;
  return (off + 4 * (size_t)fp8_slabs(d, n) + 15) & ~(size_t)15;
}

rt_status rt_quantize_fp8(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, void* Xq) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, nullptr)) != RT_OK) return st;
  if (!Xq || ((uintptr_t)Xq & 15u)) return fail(h, RT_EINVAL, "Xq must be a 16-byte aligned device pointer");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  const int64_t S = fp8_slabs(d, n), slab = n[d - 2] * n[d - 1];
  float* sc = reinterpret_cast<float*>(static_cast<char*>(Xq) + fp8_scale_offset(d, n));
  const int nl = launch_quantize_fp8(X, (int)dtype, S, slab, static_cast<unsigned char*>(Xq), sc, h->stream);
  if (nl < 0) return fail(h, RT_ENOTSUP, "float8 packing: too many slab chunks");
  return finish(h, nl);
}

int rt_last_schedule(rt_handle h, int32_t* out, int cap) {
  if (!h) return -1;
  const int nlev = (int)h->last_schedule.size();
  for (int k = 0; k < nlev && k < cap && out; ++k) out[k] = h->last_schedule[k];
  return nlev;
}

rt_status rt_selftest_wait(rt_handle h) {
  if (!h) return RT_EINVAL;
  rt_status st;
  if ((st = check_prior_status(h)) != RT_OK) return st;
  return finish(h, launch_wait_selftest(h->d_status, h->stream));
}

rt_status rt_destroy(rt_handle h) {
  if (!h) return RT_EINVAL;
  cudaStreamSynchronize(h->stream);
  if (h->ws) cudaFree(h->ws);
  if (h->hc_buf) cudaFree(h->hc_buf);
  if (h->d_status) cudaFree(h->d_status);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  if (h->ev_status) cudaEventDestroy(h->ev_status);
  if (h->ev_stage) cudaEventDestroy(h->ev_stage);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->cstream) {
    cudaStreamSynchronize(h->cstream);
    cudaStreamDestroy(h->cstream);
  }
  for (int k = 0; k < 2; ++k) {
    if (h->ev_copied[k]) cudaEventDestroy(h->ev_copied[k]);
    if (h->ev_used[k]) cudaEventDestroy(h->ev_used[k]);
  }
  if (h->pipe_buf) cudaFree(h->pipe_buf);
  for (GraphEntry& ge : h->graphs) release_graph(h, ge);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  drain_timing(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return RT_OK;
}

rt_status rt_set_stream(rt_handle h, void* stream) {
  if (!h) return RT_EINVAL;
  cudaStreamSynchronize(h->stream);
  h->stream = static_cast<cudaStream_t>(stream);
  return RT_OK;
}

rt_status rt_sync(rt_handle h) {
  if (!h) return RT_EINVAL;
  RT_CUDA(h, cudaStreamSynchronize(h->stream));
  int s = 0;
  RT_CUDA(h, cudaMemcpy(&s, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  h->status_pending = false;
  if (s != ST_OK) {
    RT_CUDA(h, cudaMemset(h->d_status, 0, sizeof(int)));
    if (s == ST_TIMEOUT) return fail(h, RT_ETIMEOUT, "a bounded device loop ran out");
    if (s == ST_NUMERIC) return fail(h, RT_ENUMERIC, "numerical breakdown on the device");
    return fail(h, RT_EDEVICE, "device-side check failed");
  }
  return RT_OK;
}

const char* rt_last_error(rt_handle h) { return h ? h->err.c_str() : "null handle"; }

rt_status rt_set_timing(rt_handle h, int enable) {
  if (!h) return RT_EINVAL;
  h->timing = enable != 0;
  return RT_OK;
}

rt_status rt_get_timing(rt_handle h, double* ms, int64_t* count, int nmax, int reset) {
  if (!h) return RT_EINVAL;
  RT_CUDA(h, cudaStreamSynchronize(h->stream));
  drain_timing(h);
  for (int i = 0; i < nmax && i < RT_NSTAGES; ++i) {
    if (ms) ms[i] = h->stage_ms[i];
    if (count) count[i] = h->stage_cnt[i];
  }
  if (reset)
    for (int i = 0; i < RT_NSTAGES; ++i) { h->stage_ms[i] = 0.0; h->stage_cnt[i] = 0; }
  return RT_OK;
}
int rt_last_launch_count(rt_handle h) { return h ? h->launches : 0; }
size_t rt_workspace_bytes(rt_handle h) { return h ? h->ws_bytes : 0; }

rt_status rtucker_indices(rt_handle h, int d, const int64_t* n, const int64_t* s, uint64_t seed, int64_t* idx) {
  if (!h) return RT_EINVAL;
  if (!idx) return fail(h, RT_EINVAL, "idx is null");
  // the sample needs no tensor; idx only stands in for X in the size checks
  rt_status st = check_tensor(h, reinterpret_cast<const void*>(idx), RT_F32, d, n, nullptr);
  if (st != RT_OK) return st;
  if ((st = check_prior_status(h)) != RT_OK) return st;
  if ((st = init_device_attrs(h)) != RT_OK) return st;
  Group Gp;
  Bump bump;
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    ProbSpec ps{};
    ps.X = idx;
    ps.dtype = RT_F32;
    ps.d = d;
    for (int j = 0; j < d; ++j) ps.n[j] = n[j];
    ps.a = ps.b = k;
    ps.r = 1;
    ps.p = 0;
    ps.s = s ? s[k] : default_s(n, d, k);
    ps.seed = seed;
    ps.node = (uint32_t)k;
    ps.idx_out = idx + off;
    ProbPlan pp;
    if ((st = plan_problem(h, ps, bump, pp)) != RT_OK) return st;
    Gp.pp.push_back(pp);
    off += (size_t)ps.s;
  }
  group_layout(Gp, bump);
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  if ((st = ensure_stage(h, group_stage_bytes(Gp))) != RT_OK) return st;
  if ((st = group_upload(h, Gp, h->h_stage, 0)) != RT_OK) return st;
  int nl = 0;
  if ((st = stage_commit(h, &nl)) != RT_OK) return st;
  nl += launch_sample_only(Gp.g, h->stream, h->d_status);
  return finish(h, nl);
}

rt_status rtucker_sketch(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                         int32_t p, const int64_t* s, uint64_t seed, const rt_options* opt, float* Z) {
  if (!h) return RT_EINVAL;
  if (!Z) return fail(h, RT_EINVAL, "Z is null");
  return tucker_run(h, X, dtype, d, n, r, p, s, seed, opt, nullptr, nullptr, nullptr, Z);
}

rt_status rtucker_factors(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                          int32_t p, const int64_t* s, uint64_t seed, const rt_options* opt, float* U,
                          float* sigma) {
  if (!h) return RT_EINVAL;
  if (!U) return fail(h, RT_EINVAL, "U is null");
  return tucker_run(h, X, dtype, d, n, r, p, s, seed, opt, U, sigma, nullptr, nullptr);
}

rt_status rtucker_decompose(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                            const int32_t* r, int32_t p, const int64_t* s, uint64_t seed, const rt_options* opt,
                            float* U, float* G) {
  if (!h) return RT_EINVAL;
  if (!U || !G) return fail(h, RT_EINVAL, "U and G are required");
  return tucker_run(h, X, dtype, d, n, r, p, s, seed, opt, U, nullptr, G, nullptr);
}

rt_status rtucker_core(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                       const float* U, const rt_options* opt, float* G) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, nullptr, true)) != RT_OK) return st;
  if ((st = check_opts(h, opt)) != RT_OK) return st;
  if (!r || !U || !G) return fail(h, RT_EINVAL, "r, U and G are required");
  for (int k = 0; k < d; ++k)
    if (r[k] < 1) return fail(h, RT_EINVAL, "need r_k >= 1");
  if (dtype == RT_F8E4M3 && (st = check_fp8_shape(h, d, n, r)) != RT_OK) return st;
  if (dtype == RT_F8E4M3 && core_of(opt) == 2) return fail(h, RT_ENOTSUP, "float8 storage needs the tensor-core pass");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  if ((st = init_device_attrs(h)) != RT_OK) return st;
  Bump bump;
  const size_t cb = core_buffer_floats(d, n, r);
  const size_t oA = bump.take(cb * 4), oB = bump.take(cb * 4);
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  float* bufA = reinterpret_cast<float*>(h->ws + oA);
  float* bufB = reinterpret_cast<float*>(h->ws + oB);
  int core = core_of(opt);
  if (core == 3 && dtype == RT_F8E4M3) core = 1;
  if (core == 3 && (st = tune_core(h, X, dtype, d, n, r, U, G, bufA, bufB, prec_of(opt), &core)) != RT_OK)
    return st;
  const int nl = enqueue_core(h, X, dtype, d, n, r, U, G, bufA, bufB, prec_of(opt), core);
  if (nl < 0) return fail(h, RT_ENOTSUP, "float8 storage: the tensor-core pass did not take the shape");
  return finish(h, nl);
}

// --- differentiable Tucker ----------------------------------------------------
namespace {

// Largest intermediate of the expansion of the leading d-2 modes of an
// r_0 x ... x r_{d-1} core (mode k: r_k -> n_k, k < d-2), and of mode d-2 as well
// when the last two modes take the general form.
size_t expand_buffer_floats(int d, const int64_t* n, const int32_t* r) {
  size_t cur = 1;
  for (int k = 0; k < d; ++k) cur *= (size_t)r[k];
  size_t best = cur;
  int64_t L = 1;
  for (int k = 0; k + 2 < d; ++k) {
    cur = cur / (size_t)r[k] * (size_t)n[k];
    best = std::max(best, cur);
    L *= n[k];
  }
  if (last_modes_general(L, n[d - 2], r[d - 2], n[d - 1], r[d - 1]))
    best = std::max(best, cur / (size_t)r[d - 2] * (size_t)n[d - 2]);
  return best;
}

// out = alpha X + beta C x_0 U_0 ... x_{d-1} U_{d-1} (X may be null): the leading
// d-2 modes of C expanded into H (two ping-pong buffers), then the last two per
// slab of H, or (slabs too large or too few) mode d-2 expanded as well and the
// last mode by rows; sumsq (device, may be null) receives scale * ||out||_F^2.
// Returns the launches made, 0 if the shape is unsupported.
int enqueue_expand(rt_handle h, const float* C, int d, const int64_t* n, const int32_t* r, const float* U,
                   const size_t* uoff, const void* X, int dtype, float alpha, float beta, float* out, float* bufA,
                   float* bufB, double* part, double* sumsq, double scale) {
  cudaStream_t st = h->stream;
  const float* A = C;
  int64_t L = 1;
  int nl = 0;
  for (int k = 0; k + 2 < d; ++k) {
    int64_t R = 1;
    for (int j = k + 1; j < d; ++j) R *= r[j];
    float* o = (k % 2 == 0) ? bufA : bufB;
    nl += launch_expand_f32(A, L, r[k], R, U + uoff[k], n[k], o, st);
    A = o;
    L *= n[k];
  }
  int got;
  if (last_modes_general(L, n[d - 2], r[d - 2], n[d - 1], r[d - 1])) {
    float* o = (A == bufA) ? bufB : bufA;
    nl += launch_expand_f32(A, L, r[d - 2], r[d - 1], U + uoff[d - 2], n[d - 2], o, st);
    got = launch_last_out(X, dtype, alpha, beta, o, L * n[d - 2], r[d - 1], n[d - 1], U + uoff[d - 1], out, part,
                          sumsq, scale, st);
  } else {
    got = launch_tucker_slab_out(X, dtype, alpha, beta, A, L, n[d - 2], r[d - 2], n[d - 1], r[d - 1],
                                 U + uoff[d - 2], U + uoff[d - 1], out, part, sumsq, scale, st);
  }
  return got > 0 ? nl + got : 0;
}

// Plan of the partial projections Y_n = T x_{m != n} U_m^T of an n_0 x ... x n_{d-1}
// tensor T: the prefixes P_k = T x_0 U_0^T ... x_{k-1} U_{k-1}^T (k = 1 .. d-1) are
// kept, and Y_n continues from P_n (P_0 = T) over modes n+1 .. d-1.  Leading modes
// go first so that every contraction of a large tensor has a long contiguous
// trailing extent (the fast TTM form); only reduced tensors see a last-mode step.
struct PartialPlan {
  size_t prefix_floats[MAXD + 1] = {0};  // size of P_k
  size_t chain_floats = 1;               // largest intermediate of a continuation
  size_t y_floats = 1;                   // largest Y_n
};

PartialPlan plan_partials(int d, const int64_t* n, const int32_t* r) {
  PartialPlan pl;
  for (int k = 1; k < d; ++k) {
    size_t s = 1;
    for (int j = 0; j < k; ++j) s *= (size_t)r[j];
    for (int j = k; j < d; ++j) s *= (size_t)n[j];
    pl.prefix_floats[k] = s;
  }
  for (int m = 0; m < d; ++m) {
    int64_t sh[MAXD];
    for (int j = 0; j < d; ++j) sh[j] = (j < m) ? r[j] : n[j];
    for (int j = m + 1; j < d; ++j) {
      sh[j] = r[j];
      size_t s = 1;
      for (int q = 0; q < d; ++q) s *= (size_t)sh[q];
      if (j < d - 1) pl.chain_floats = std::max(pl.chain_floats, s);
      else pl.y_floats = std::max(pl.y_floats, s);
    }
  }
  return pl;
}

// outU (concatenated n_n x r_n, may be null) = scale [T x_{m != n} U_m^T]_(n) C_(n)^T
// for every n, and outCore (may be null) = scale T x_k U_k^T.  T has element type
// dtype; prefix[k] hold P_k, chainA/B the continuations, ybuf the finished Y_n.
int enqueue_partials(rt_handle h, const void* T, int dtype, int d, const int64_t* n, const int32_t* r,
                     const float* U, const size_t* uoff, const float* C, float scale, float* outU, float* outCore,
                     float* const* prefix, float* chainA, float* chainB, float* ybuf, float* uscratch) {
  cudaStream_t st = h->stream;
  int nl = 0;
  // prefix == nullptr: recompute mode, every P_m is formed again from T in the
  // ping-pong chain buffers instead of being kept
  const bool keep = prefix != nullptr;
  // P_m into `dst` (or, recomputing, into a chain buffer; *ping tracks the one used)
  auto prefix_chain = [&](int m, int* ping) -> const void* {
    const void* A = T;
    int adt = dtype;
    for (int k = 1; k <= m; ++k) {
      int64_t L = 1, R = 1;
      for (int j = 0; j < k - 1; ++j) L *= r[j];
      for (int j = k; j < d; ++j) R *= n[j];
      float* o = *ping ? chainB : chainA;
      nl += launch_ttm_t(A, adt, L, n[k - 1], R, U + uoff[k - 1], r[k - 1], o, st);
      A = o;
      adt = DT_F32;
      *ping ^= 1;
    }
    return A;
  };
  if (keep) {
    const void* A = T;
    int adt = dtype;
    for (int k = 1; k < d; ++k) {        // P_k = P_{k-1} x_{k-1} U_{k-1}^T
      int64_t L = 1, R = 1;
      for (int j = 0; j < k - 1; ++j) L *= r[j];
      for (int j = k; j < d; ++j) R *= n[j];
      nl += launch_ttm_t(A, adt, L, n[k - 1], R, U + uoff[k - 1], r[k - 1], prefix[k], st);
      A = prefix[k];
      adt = DT_F32;
    }
  }
  if (outCore) {                       // P_{d-1} x_{d-1} U_{d-1}^T
    int64_t L = 1;
    for (int j = 0; j < d - 1; ++j) L *= r[j];
    int ping = 0;
    const void* Pd = keep ? prefix[d - 1] : prefix_chain(d - 1, &ping);
    nl += launch_ttm_t(Pd, DT_F32, L, n[d - 1], 1, U + uoff[d - 1], r[d - 1], outCore, st);
    if (scale != 1.f) nl += launch_scale_f32(outCore, L * r[d - 1], scale, st);
  }
  if (!outU) return nl;
  for (int m = 0; m < d; ++m) {
    int ping = 0;
    const void* Y = (m == 0) ? T : (keep ? (const void*)prefix[m] : prefix_chain(m, &ping));
    int ydt = (m == 0) ? dtype : DT_F32;
    int64_t sh[MAXD];
    for (int j = 0; j < d; ++j) sh[j] = (j < m) ? r[j] : n[j];
    for (int j = m + 1; j < d; ++j) {
      int64_t L = 1, R = 1;
      for (int q = 0; q < j; ++q) L *= sh[q];
      for (int q = j + 1; q < d; ++q) R *= sh[q];
      float* o = (j == d - 1) ? ybuf : (ping ? chainB : chainA);
      nl += launch_ttm_t(Y, ydt, L, sh[j], R, U + uoff[j], r[j], o, st);
      sh[j] = r[j];
      Y = o;
      ydt = DT_F32;
      ping ^= 1;
    }
    if (ydt != DT_F32) return -1;      // only for d = 1, excluded by the argument checks
    int64_t P = 1, Q = 1;
    for (int j = 0; j < m; ++j) P *= r[j];
    for (int j = m + 1; j < d; ++j) Q *= r[j];
    const int got = launch_unfold_contract(static_cast<const float*>(Y), C, P, n[m], r[m], Q, scale,
                                           outU + uoff[m], uscratch, st);
    if (got <= 0) return -1;
    nl += got;
  }
  return nl;
}

rt_status check_grad_args(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                          const float* U, const float* C, int64_t* total) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, total)) != RT_OK) return st;
  if (!r || !U || !C) return fail(h, RT_EINVAL, "r, U and the core are required");
  for (int k = 0; k < d; ++k)
    if (r[k] < 1 || r[k] > CMAX) return fail(h, RT_EINVAL, "need 1 <= r_k <= 64");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  return init_device_attrs(h);
}

}  // namespace

rt_status rtucker_loss_grad(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                            const float* U, const float* G, double* loss, float* dX, float* dG, float* dU) {
  int64_t total = 0;
  rt_status st = check_grad_args(h, X, dtype, d, n, r, U, G, &total);
  if (st != RT_OK) return st;
  size_t uoff[MAXD];
  size_t acc = 0;
  for (int k = 0; k < d; ++k) { uoff[k] = acc; acc += (size_t)n[k] * r[k]; }
  const bool grads = dG || dU;
  Bump bump;
  const size_t eb = expand_buffer_floats(d, n, r);
  const size_t oEA = bump.take(eb * 4), oEB = bump.take(eb * 4);
  const size_t oPart = bump.take(expand_partial_doubles() * 8);
  const size_t oR = (!dX && grads) ? bump.take((size_t)total * 4) : 0;
  PartialPlan pl = plan_partials(d, n, r);
  size_t oS[MAXD + 1] = {0};
  size_t oCA = 0, oCB = 0, oY = 0, oUS = 0;
  if (grads) {
    // recompute mode keeps no prefixes; its chain buffers also hold the largest P_k
    size_t chain = pl.chain_floats;
    if (h->grad_recompute) {
      for (int k = 1; k < d; ++k) chain = std::max(chain, pl.prefix_floats[k]);
    } else {
      for (int k = 1; k < d; ++k) oS[k] = bump.take(pl.prefix_floats[k] * 4);
    }
    oCA = bump.take(chain * 4);
    oCB = bump.take(chain * 4);
    oY = bump.take(pl.y_floats * 4);
    size_t us = 1;
    for (int m = 0; m < d; ++m) {
      int64_t K = 1;
      for (int j = 0; j < d; ++j)
        if (j != m) K *= r[j];
      us = std::max(us, unfold_scratch_floats(n[m], r[m], K));
    }
    oUS = bump.take(us * 4);
  }
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  char* ws = h->ws;
  float* R = dX ? dX : reinterpret_cast<float*>(ws + oR);
  int nl = 0;
  if (dX || grads || loss) {
    float* out = (dX || grads) ? R : nullptr;   // loss only: the residual is not stored
    const int got = enqueue_expand(h, G, d, n, r, U, uoff, X, dtype, 1.f, -1.f, out,
                                   reinterpret_cast<float*>(ws + oEA), reinterpret_cast<float*>(ws + oEB),
                                   reinterpret_cast<double*>(ws + oPart), loss, 0.5);
    if (got <= 0) return fail(h, RT_ENOTSUP, "ranks too large for the reconstruction kernel");
    nl += got;
    R = out;
  }
  if (grads) {
    float* prefix[MAXD + 1] = {nullptr};
    for (int k = 1; k < d; ++k) prefix[k] = reinterpret_cast<float*>(ws + oS[k]);
    const int got = enqueue_partials(h, R, DT_F32, d, n, r, U, uoff, G, -1.f, dU, dG,
                                     h->grad_recompute ? nullptr : prefix,
                                     reinterpret_cast<float*>(ws + oCA), reinterpret_cast<float*>(ws + oCB),
                                     reinterpret_cast<float*>(ws + oY), reinterpret_cast<float*>(ws + oUS));
    if (got < 0) return fail(h, RT_EINVAL, "internal: partial projection plan");
    nl += got;
  }
  return finish(h, nl);
}

rt_status rtucker_core_adjoint(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                               const int32_t* r, const float* U, const float* Gbar, float* Xbar, float* Ubar) {
  int64_t total = 0;
  rt_status st = check_grad_args(h, X, dtype, d, n, r, U, Gbar, &total);
  if (st != RT_OK) return st;
  size_t uoff[MAXD];
  size_t acc = 0;
  for (int k = 0; k < d; ++k) { uoff[k] = acc; acc += (size_t)n[k] * r[k]; }
  Bump bump;
  const size_t eb = expand_buffer_floats(d, n, r);
  const size_t oEA = bump.take(eb * 4), oEB = bump.take(eb * 4);
  const size_t oPart = bump.take(expand_partial_doubles() * 8);
  PartialPlan pl = plan_partials(d, n, r);
  size_t oS[MAXD + 1] = {0};
  size_t oCA = 0, oCB = 0, oY = 0, oUS = 0;
  if (Ubar) {
    // recompute mode keeps no prefixes; its chain buffers also hold the largest P_k
    size_t chain = pl.chain_floats;
    if (h->grad_recompute) {
      for (int k = 1; k < d; ++k) chain = std::max(chain, pl.prefix_floats[k]);
    } else {
      for (int k = 1; k < d; ++k) oS[k] = bump.take(pl.prefix_floats[k] * 4);
    }
    oCA = bump.take(chain * 4);
    oCB = bump.take(chain * 4);
    oY = bump.take(pl.y_floats * 4);
    size_t us = 1;
    for (int m = 0; m < d; ++m) {
      int64_t K = 1;
      for (int j = 0; j < d; ++j)
        if (j != m) K *= r[j];
      us = std::max(us, unfold_scratch_floats(n[m], r[m], K));
    }
    oUS = bump.take(us * 4);
  }
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  char* ws = h->ws;
  int nl = 0;
  if (Xbar) {
    const int got = enqueue_expand(h, Gbar, d, n, r, U, uoff, nullptr, (int)dtype, 0.f, 1.f, Xbar,
                                   reinterpret_cast<float*>(ws + oEA), reinterpret_cast<float*>(ws + oEB),
                                   reinterpret_cast<double*>(ws + oPart), nullptr, 1.0);
    if (got <= 0) return fail(h, RT_ENOTSUP, "ranks too large for the reconstruction kernel");
    nl += got;
  }
  if (Ubar) {
    float* prefix[MAXD + 1] = {nullptr};
    for (int k = 1; k < d; ++k) prefix[k] = reinterpret_cast<float*>(ws + oS[k]);
    const int got = enqueue_partials(h, X, (int)dtype, d, n, r, U, uoff, Gbar, 1.f, Ubar, nullptr,
                                     h->grad_recompute ? nullptr : prefix,
                                     reinterpret_cast<float*>(ws + oCA), reinterpret_cast<float*>(ws + oCB),
                                     reinterpret_cast<float*>(ws + oY), reinterpret_cast<float*>(ws + oUS));
    if (got < 0) return fail(h, RT_EINVAL, "internal: partial projection plan");
    nl += got;
  }
  return finish(h, nl);
}

rt_status rtucker_decompose_host(rt_handle h, const void* X_host, rt_dtype dtype, int d, const int64_t* n,
                                 const int32_t* r, int32_t p, const int64_t* s, uint64_t seed,
                                 const rt_options* opt, float* U_host, float* G_host) {
  if (!h) return RT_EINVAL;
  int64_t total = 0;
  rt_status st = check_tensor(h, X_host, dtype, d, n, &total);
  if (st != RT_OK) return st;
  if (!r || !U_host || !G_host) return fail(h, RT_EINVAL, "r, U and G are required");
  size_t usz = 0, gsz = 1;
  for (int k = 0; k < d; ++k) { usz += (size_t)n[k] * r[k]; gsz *= (size_t)r[k]; }
  // Device copies live in a separate allocation owned by the handle so that
  // the decomposition's own workspace planning is unchanged.
  const size_t xb = align_up((size_t)total * dtype_size(dtype));
  const size_t need = xb + align_up(usz * 4) + align_up(gsz * 4);
  if (need > h->hc_bytes) {
    RT_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->hc_buf) cudaFree(h->hc_buf);
    h->hc_buf = nullptr;
    h->hc_bytes = 0;
    if (cudaMalloc(&h->hc_buf, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, RT_ENOMEM, "device buffers for the host-memory call");
    }
    h->hc_bytes = need;
  }
  char* base = h->hc_buf;
  void* dX = base;
  float* dU = reinterpret_cast<float*>(base + xb);
  float* dG = reinterpret_cast<float*>(base + xb + align_up(usz * 4));
  RT_CUDA(h, cudaMemcpyAsync(dX, X_host, (size_t)total * dtype_size(dtype), cudaMemcpyHostToDevice, h->stream));
  st = rtucker_decompose(h, dX, dtype, d, n, r, p, s, seed, opt, dU, dG);
  if (st != RT_OK) return st;
  const int nl = h->launches;
  RT_CUDA(h, cudaMemcpyAsync(U_host, dU, usz * 4, cudaMemcpyDeviceToHost, h->stream));
  RT_CUDA(h, cudaMemcpyAsync(G_host, dG, gsz * 4, cudaMemcpyDeviceToHost, h->stream));
  st = rt_sync(h);
  h->launches = nl;
  return st;
}

rt_status rtucker_decompose_host_async(rt_handle h, const void* X_host, rt_dtype dtype, int d, const int64_t* n,
                                       const int32_t* r, int32_t p, const int64_t* s, uint64_t seed,
                                       const rt_options* opt, float* U_host, float* G_host) {
  if (!h) return RT_EINVAL;
  int64_t total = 0;
  rt_status st = check_tensor(h, X_host, dtype, d, n, &total);
  if (st != RT_OK) return st;
  if (!r || !U_host || !G_host) return fail(h, RT_EINVAL, "r, U and G are required");
  size_t usz = 0, gsz = 1;
  for (int k = 0; k < d; ++k) { usz += (size_t)n[k] * r[k]; gsz *= (size_t)r[k]; }
  const size_t xbytes = (size_t)total * dtype_size(dtype);
  const size_t xb = align_up(xbytes), ob = align_up(usz * 4) + align_up(gsz * 4);
  if (!h->cstream) {
    RT_CUDA(h, cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      RT_CUDA(h, cudaEventCreateWithFlags(&h->ev_copied[k], cudaEventDisableTiming));
      RT_CUDA(h, cudaEventCreateWithFlags(&h->ev_used[k], cudaEventDisableTiming));
    }
  }
  if (xb > h->pipe_slot || ob > h->pipe_out) {
    // both streams idle before the buffers move
    RT_CUDA(h, cudaStreamSynchronize(h->cstream));
    RT_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->pipe_buf) cudaFree(h->pipe_buf);
    h->pipe_buf = nullptr;
    h->pipe_slot = h->pipe_out = 0;
    const size_t slot = std::max(xb, h->pipe_slot), out = std::max(ob, h->pipe_out);
    if (cudaMalloc(&h->pipe_buf, 2 * slot + out) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, RT_ENOMEM, "device buffers for the pipelined host-memory call");
    }
    h->pipe_slot = slot;
    h->pipe_out = out;
  }
  const int k = h->pipe_next;
  char* dX = h->pipe_buf + (size_t)k * h->pipe_slot;
  float* dU = reinterpret_cast<float*>(h->pipe_buf + 2 * h->pipe_slot);
  float* dG = reinterpret_cast<float*>(h->pipe_buf + 2 * h->pipe_slot + align_up(usz * 4));
  // copy stream: slot k is free once the decomposition that last read it ran
  RT_CUDA(h, cudaStreamWaitEvent(h->cstream, h->ev_used[k], 0));
  RT_CUDA(h, cudaMemcpyAsync(dX, X_host, xbytes, cudaMemcpyHostToDevice, h->cstream));
  RT_CUDA(h, cudaEventRecord(h->ev_copied[k], h->cstream));
  RT_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_copied[k], 0));
  st = rtucker_decompose(h, dX, dtype, d, n, r, p, s, seed, opt, dU, dG);
  if (st != RT_OK) {
    cudaStreamSynchronize(h->cstream);  // X_host is no longer read when the call returns
    return st;
  }
  RT_CUDA(h, cudaEventRecord(h->ev_used[k], h->stream));
  // the next call's decomposition writes dU/dG after these reads on the same stream
  RT_CUDA(h, cudaMemcpyAsync(U_host, dU, usz * 4, cudaMemcpyDeviceToHost, h->stream));
  RT_CUDA(h, cudaMemcpyAsync(G_host, dG, gsz * 4, cudaMemcpyDeviceToHost, h->stream));
  h->pipe_next = k ^ 1;
  return RT_OK;
}

rt_status rtucker_decompose_batched(rt_handle h, int T, const void* const* X, rt_dtype dtype, const int32_t* d,
                                    const int64_t* const* n, const int32_t* const* r, int32_t p,
                                    const int64_t* const* s, const uint64_t* seeds, const rt_options* opt,
                                    float* const* U, float* const* G) {
  if (!h) return RT_EINVAL;
  if (T < 1 || !X || !d || !n || !r || !seeds || !U || !G) return fail(h, RT_EINVAL, "null batched argument");
  rt_status st;
  if ((st = check_opts(h, opt)) != RT_OK) return st;
  for (int t = 0; t < T; ++t)
    if ((st = check_tensor(h, X[t], dtype, d[t], n[t], nullptr)) != RT_OK) return st;
  if ((st = check_prior_status(h)) != RT_OK) return st;
  if ((st = init_device_attrs(h)) != RT_OK) return st;
  Group Gp;
  Bump bump;
  for (int t = 0; t < T; ++t) {
    st = add_tucker_problems(h, Gp, bump, X[t], dtype, d[t], n[t], r[t], p, s ? s[t] : nullptr, seeds[t], U[t],
                             nullptr, qr_of(opt), sketch_of(opt));
    if (st != RT_OK) return st;
  }
  group_layout(Gp, bump);
  // per-tensor core buffers
  std::vector<size_t> oA(T), oB(T);
  int dmax = 0;
  for (int t = 0; t < T; ++t) {
    const size_t cb = core_buffer_floats(d[t], n[t], r[t]);
    oA[t] = bump.take(cb * 4);
    oB[t] = bump.take(cb * 4);
    dmax = std::max(dmax, (int)d[t]);
  }
  // The core of every tensor as grouped contractions: level k contracts mode
  // d_t - 1 - k of every tensor with d_t > k, last mode first, one launch per level.
  std::vector<int> njob(dmax, 0);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < d[t]; ++k) ++njob[k];
  // Schedules of a level (rt_options.core = 3 times them): candidate 0 the generic grouped
  // tiles, candidate c >= 1 the one-row-per-lane form with kRowBlocks[c - 1] 128-row blocks
  // per CTA (levels whose jobs all contract a last mode of <= 256 rows into <= 32 columns).
  static const int kRowBlocks[] = {1, 2, 4, 8, 16};
  constexpr int NCAND = 6, CAND_DEFAULT_ROWS = 4;   // default: 8 row blocks
  std::vector<size_t> o_jobs(dmax);
  std::vector<std::array<size_t, NCAND>> o_lpre(dmax);
  size_t job_bytes = 0;
  for (int k = 0; k < dmax; ++k) {
    o_jobs[k] = bump.take(sizeof(TTMJob) * njob[k]);
    job_bytes += align_up(sizeof(TTMJob) * njob[k]);
    for (int c = 0; c < NCAND; ++c) {
      o_lpre[k][c] = bump.take(sizeof(int64_t) * (njob[k] + 1));
      job_bytes += align_up(sizeof(int64_t) * (njob[k] + 1));
    }
  }
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  const size_t gsb = group_stage_bytes(Gp);
  if ((st = ensure_stage(h, gsb + job_bytes)) != RT_OK) return st;
  if ((st = group_upload(h, Gp, h->h_stage, 0)) != RT_OK) return st;
  // job tables (workspace addresses are final once it is sized), staged after the
  // range-finder tables and uploaded with them
  std::vector<std::array<int64_t, NCAND>> ltiles(dmax);
  std::vector<char> last_rows(dmax, 0);
  std::vector<int> lnmax(dmax, 0), lrmax(dmax, 0);
  {
    size_t so = gsb;
    for (int k = 0; k < dmax; ++k) {
      TTMJob* js = reinterpret_cast<TTMJob*>(h->h_stage + so);
      so += align_up(sizeof(TTMJob) * njob[k]);
      int64_t* ps[NCAND];
      for (int c = 0; c < NCAND; ++c) {
        ps[c] = reinterpret_cast<int64_t*>(h->h_stage + so);
        so += align_up(sizeof(int64_t) * (njob[k] + 1));
      }
      int q_i = 0;
      int64_t acc[NCAND] = {0, 0, 0, 0, 0, 0};
      // a level whose jobs all contract a last mode of <= 256 rows into <= 32 columns
      // takes the one-thread-per-row form (CTAs counted per job by rows)
      bool rows = true;
      for (int t = 0; t < T && rows; ++t)
        if (d[t] > k) {
          const int m = d[t] - 1 - k;
          int64_t R = 1;
          for (int j = m + 1; j < d[t]; ++j) R *= r[t][j];
          rows = R == 1 && n[t][m] <= 256 && r[t][m] <= 32;
        }
      last_rows[k] = rows;
      for (int t = 0; t < T; ++t) {
        if (d[t] <= k) continue;
        const int m = d[t] - 1 - k;
        float* bufA = reinterpret_cast<float*>(h->ws + oA[t]);
        float* bufB = reinterpret_cast<float*>(h->ws + oB[t]);
        TTMJob q{};
        q.A = (k == 0) ? X[t] : static_cast<const void*>((k & 1) ? bufA : bufB);
        q.out = (m == 0) ? G[t] : ((k & 1) ? bufB : bufA);
        q.L = 1;
        q.R = 1;
        for (int j = 0; j < m; ++j) q.L *= n[t][j];
        for (int j = m + 1; j < d[t]; ++j) q.R *= r[t][j];
        q.n = n[t][m];
        q.r = r[t][m];
        int64_t uo = 0;
        for (int j = 0; j < m; ++j) uo += n[t][j] * r[t][j];
        q.U = U[t] + uo;
        for (int c = 0; c < NCAND; ++c) ps[c][q_i] = acc[c];
        acc[0] += ttm_job_tiles(q);   // also sets tiles_x
        if (rows) {
          for (int c = 1; c < NCAND; ++c) acc[c] += ttm_last_job_ctas(q, kRowBlocks[c - 1]);
          lnmax[k] = std::max<int>(lnmax[k], (int)q.n);
          lrmax[k] = std::max<int>(lrmax[k], q.r);
        }
        js[q_i++] = q;
      }
      for (int c = 0; c < NCAND; ++c) {
        ps[c][q_i] = acc[c];
        ltiles[k][c] = acc[c];
      }
      if ((st = stage_put(h, h->ws + o_jobs[k], js, sizeof(TTMJob) * njob[k])) != RT_OK) return st;
      for (int c = 0; c < NCAND; ++c)
        if ((st = stage_put(h, h->ws + o_lpre[k][c], ps[c], sizeof(int64_t) * (njob[k] + 1))) != RT_OK) return st;
    }
  }
  int nl = 0;
  if ((st = stage_commit(h, &nl)) != RT_OK) return st;
  auto launch_level = [&](int k, int c) -> int {
    const int dt = k == 0 ? (int)dtype : DT_F32;
    const TTMJob* jd = reinterpret_cast<const TTMJob*>(h->ws + o_jobs[k]);
    const int64_t* pd = reinterpret_cast<const int64_t*>(h->ws + o_lpre[k][c]);
    if (c == 0) return launch_ttm_grouped(jd, pd, njob[k], ltiles[k][0], dt, h->stream);
    return launch_ttm_last_grouped(jd, pd, njob[k], ltiles[k][c], dt, lnmax[k], lrmax[k], kRowBlocks[c - 1],
                                   h->stream);
  };
  // per-level schedule: fixed defaults, or (core = 3) the fastest candidate, timed once per
  // set of shapes on the call's own buffers (the values the candidates read and write do
  // not matter for the time; the decomposition below recomputes everything)
  std::vector<int> sched(dmax);
  for (int k = 0; k < dmax; ++k) sched[k] = last_rows[k] ? CAND_DEFAULT_ROWS : 0;
  if (core_of(opt) == 3) {
    std::vector<int64_t> tk = {(int64_t)dtype, T};
    for (int t = 0; t < T; ++t) {
      tk.push_back(d[t]);
      for (int k = 0; k < d[t]; ++k) { tk.push_back(n[t][k]); tk.push_back(r[t][k]); }
    }
    auto it = h->batched_tuned.find(tk);
    if (it != h->batched_tuned.end()) {
      sched = it->second;
    } else {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(h, RT_ECUDA, "batched tuning: event creation");
      }
      const bool timing = h->timing;
      h->timing = false;
      cudaError_t ce = cudaSuccess;
      for (int k = 0; k < dmax && ce == cudaSuccess; ++k) {
        float best = 0.f;
        for (int c = 0; c < (last_rows[k] ? NCAND : 1) && ce == cudaSuccess; ++c) {
          launch_level(k, c);
          cudaEventRecord(e0, h->stream);
          for (int rep = 0; rep < 2; ++rep) launch_level(k, c);
          cudaEventRecord(e1, h->stream);
          float ms = 0.f;
          ce = cudaEventSynchronize(e1);
          if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
          if (ce == cudaSuccess) ce = cudaGetLastError();
          if (ce == cudaSuccess && (c == 0 || ms < best)) {
            best = ms;
            sched[k] = c;
          }
        }
      }
      h->timing = timing;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ce != cudaSuccess) return cuda_fail(h, ce, "batched tuning");
      h->batched_tuned[tk] = sched;
    }
  }
  h->last_schedule.assign(dmax, 0);
  for (int k = 0; k < dmax; ++k) h->last_schedule[k] = sched[k] == 0 ? 0 : kRowBlocks[sched[k] - 1];
  const bool graph = opt && opt->use_graph;
  GraphKey key;
  if (graph) {
    key.add(2);
    key.add((uint64_t)h->device);
    key.ptr(h->ws);
    key.add(bump.off);
    key.add((uint64_t)T);
    key.add((uint64_t)dtype);
    key.add((uint64_t)p);
    for (int t = 0; t < T; ++t) {   // the job tables are uploaded per call; their launch shapes:
      key.ptr(X[t]);
      key.arr(n[t], d[t]);
      key.arr(r[t], d[t]);
      key.ptr(U[t]);
      key.ptr(G[t]);
    }
    for (int k = 0; k < dmax; ++k) {
      key.add((uint64_t)njob[k]);
      key.add((uint64_t)sched[k]);
      key.add((uint64_t)ltiles[k][sched[k]]);
      key.add((uint64_t)lnmax[k]);
      key.add((uint64_t)lrmax[k]);
      key.add(o_jobs[k]);
      key.add(o_lpre[k][sched[k]]);
    }
    key.group(Gp.g);
  }
  st = run_kernels(h, graph, key, &nl, [&](int* nk) -> rt_status {
    {
      StageTimer tm(h, 0);
      *nk += launch_range_finder(Gp.g, h->stream, h->d_status);
    }
    for (int k = 0; k < dmax; ++k) {
      StageTimer tm(h, k == 0 ? 1 : 2);
      *nk += launch_level(k, sched[k]);
    }
    return RT_OK;
  });
  if (st != RT_OK) return st;
  return finish(h, nl);
}

rt_status rtucker_kron_sketch(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                              const int32_t* ell, uint64_t seed, const rt_options* opt, float* Z) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, nullptr)) != RT_OK) return st;
  if ((st = check_opts(h, opt)) != RT_OK) return st;
  if (!Z) return fail(h, RT_EINVAL, "Z is null");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  Bump bump;
  KronPlan kp;
  if ((st = plan_kron(h, X, dtype, d, n, ell, bump, kp)) != RT_OK) return st;
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  bind_kron(kp, h->ws);
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    kp.a.z[k] = Z + off;
    off += (size_t)n[k] * kp.L[k];
  }
  int nl = 0;
  {
    StageTimer tm(h, 0);
    nl += launch_kron_omega(kp.a, seed, h->stream);
    nl += launch_kron_sketch(kp.a, kp.grid, h->stream);
  }
  return finish(h, nl);
}

rt_status rtucker_rhkron(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                         const int32_t* ell, uint64_t seed, const rt_options* opt, float* U, float* G) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, nullptr)) != RT_OK) return st;
  if ((st = check_opts(h, opt)) != RT_OK) return st;
  if (!r || !ell || !U || !G) return fail(h, RT_EINVAL, "r, ell, U and G are required");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  if ((st = init_device_attrs(h)) != RT_OK) return st;
  Bump bump;
  KronPlan kp;
  if ((st = plan_kron(h, X, dtype, d, n, ell, bump, kp)) != RT_OK) return st;
  int32_t L32[MAXD];
  for (int k = 0; k < d; ++k) {
    if (r[k] < 1 || r[k] > kp.L[k] || kp.L[k] > n[k])
      return fail(h, RT_EINVAL, "need r_k <= L_k = prod_{j != k} l_j <= n_k");
    if (kp.L[k] > CMAX) return fail(h, RT_ENOTSUP, "L_k above 64 is not supported");
    L32[k] = (int32_t)kp.L[k];
  }
  // S5 of every sketch: problems with r + p = L_k whose sketch the Kronecker pass writes
  Group G1;
  for (int k = 0; k < d; ++k) {
    ProbSpec ps{};
    ps.X = X;
    ps.dtype = dtype;
    ps.d = d;
    for (int j = 0; j < d; ++j) ps.n[j] = n[j];
    ps.a = ps.b = k;
    ps.r = L32[k];
    ps.p = 0;
    ps.s = kp.L[k];
    ps.seed = seed;
    ps.node = (uint32_t)k;
    ps.qr = 1;
    ProbPlan pp;
    if ((st = plan_problem(h, ps, bump, pp)) != RT_OK) return st;
    G1.pp.push_back(pp);
  }
  group_layout(G1, bump);
  size_t qoff[MAXD], woff[MAXD], qtot = 0, wtot = 0, ctot = 1;
  int roff[MAXD], rtot = 0;
  for (int k = 0; k < d; ++k) {
    qoff[k] = qtot;
    qtot += (size_t)n[k] * kp.L[k];
    woff[k] = wtot;
    wtot += (size_t)kp.L[k] * r[k];
    roff[k] = rtot;
    rtot += r[k];
    ctot *= (size_t)kp.L[k];
  }
  const size_t o_q = bump.take(qtot * 4), o_c = bump.take(ctot * 4), o_w = bump.take(wtot * 4);
  const size_t o_sg = bump.take((size_t)rtot * 4);
  const size_t cb = std::max(core_buffer_floats(d, n, L32), core_buffer_floats(d, kp.L, r));
  const size_t o_bA = bump.take(cb * 4), o_bB = bump.take(cb * 4);
  if (ctot >= ((size_t)1 << 31)) return fail(h, RT_ENOTSUP, "reduced tensor of 2^31 or more entries");
  // the reduced tensor C = X x_k Q_k^T factored mode by mode by the W-step's Cholesky
  // form on the exact Gram C^(k) C^(k)^T (k_mode_gram) with Q = I: W_k = the dominant
  // r_k left singular vectors of C^(k).  The problems are planned with the fewest
  // samples (one Gram chunk); only their W-step kernel runs.
  ModeGram mg{};
  mg.d = d;
  mg.ctas = 1;
  {
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    mg.ctas = std::max(1, 2 * nsm / d);
  }
  size_t ptot = 0;
  for (int k = 0; k < d; ++k) {
    mg.L[k] = L32[k];
    int64_t Bk = 1;
    for (int j = k + 1; j < d; ++j) Bk *= kp.L[j];
    mg.B[k] = (int)Bk;
    mg.N[k] = (int)(ctot / (size_t)kp.L[k]);
    mg.poff[k] = (int64_t)ptot;
    ptot += (size_t)mg.ctas * kp.L[k] * kp.L[k] * 2;
  }
  const size_t o_mg = bump.take(ptot * 4);
  Group G2;
  for (int k = 0; k < d; ++k) {
    ProbSpec ps{};
    ps.X = nullptr;
    ps.dtype = RT_F32;
    ps.d = d;
    int64_t N = 1;
    for (int j = 0; j < d; ++j) {
      ps.n[j] = kp.L[j];
      if (j != k) N *= kp.L[j];
    }
    ps.a = ps.b = k;
    ps.r = r[k];
    ps.p = L32[k] - r[k];
    ps.s = std::min<int64_t>(N, L32[k]);
    ps.seed = seed;
    ps.node = (uint32_t)k;
    ps.qr = 0;
    ProbPlan pp;
    if ((st = plan_problem(h, ps, bump, pp)) != RT_OK) return st;
    G2.pp.push_back(pp);
  }
  group_layout(G2, bump);
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  bind_kron(kp, h->ws);
  float* Qc = reinterpret_cast<float*>(h->ws + o_q);
  float* C = reinterpret_cast<float*>(h->ws + o_c);
  float* Wc = reinterpret_cast<float*>(h->ws + o_w);
  float* bufA = reinterpret_cast<float*>(h->ws + o_bA);
  float* bufB = reinterpret_cast<float*>(h->ws + o_bB);
  for (int k = 0; k < d; ++k) {
    kp.a.z[k] = reinterpret_cast<float*>(h->ws + G1.pp[k].o_Zp);
    G2.pp[k].q.X = C;
    G2.pp[k].q.U = Wc + woff[k];
  }
  const size_t sb = group_stage_bytes(G1) + group_stage_bytes(G2);
  if ((st = ensure_stage(h, sb)) != RT_OK) return st;
  if ((st = group_upload(h, G1, h->h_stage, 0)) != RT_OK) return st;
  if ((st = group_upload(h, G2, h->h_stage, group_stage_bytes(G1))) != RT_OK) return st;
  int nl = 0;
  if ((st = stage_commit(h, &nl)) != RT_OK) return st;
  {
    StageTimer tm(h, 0);
    nl += launch_kron_omega(kp.a, seed, h->stream);
    nl += launch_kron_sketch(kp.a, kp.grid, h->stream);
    nl += launch_rf_qr(G1.g, h->stream, h->d_status);
    for (int k = 0; k < d; ++k)
      RT_CUDA(h, cudaMemcpyAsync(Qc + qoff[k], G1.pp[k].q.Q, (size_t)n[k] * kp.L[k] * 4, cudaMemcpyDeviceToDevice,
                                 h->stream));
  }
  const int core = core_of(opt) == 3 ? 0 : core_of(opt);
  int got = enqueue_core(h, X, dtype, d, n, L32, Qc, C, bufA, bufB, RT_PREC_FP32, core);
  if (got < 0) return fail(h, RT_ENOTSUP, "reduced core");
  nl += got;
  mg.C = C;
  mg.part = reinterpret_cast<float*>(h->ws + o_mg);
  for (int k = 0; k < d; ++k) {
    if (G2.pp[k].q.nbg != 1 || G2.pp[k].units[STG_WSV2] != 1)
      return fail(h, RT_ENOTSUP, "internal: reduced-tensor W-step plan");
    mg.cp[k] = G2.pp[k].q.Cp;
    mg.qeye[k] = G2.pp[k].q.Q;
  }
  {
    StageTimer tm(h, 0);
    nl += launch_mode_gram(mg, h->stream);
    nl += launch_rf_tail(G2.g, h->stream, h->d_status);
  }
  got = enqueue_core(h, C, RT_F32, d, kp.L, r, Wc, G, bufA, bufB, RT_PREC_FP32, core);
  if (got < 0) return fail(h, RT_ENOTSUP, "core of the reduced tensor");
  nl += got;
  KronFinish f{};
  f.d = d;
  f.Q = Qc;
  f.W = Wc;
  f.U = U;
  f.G = G;
  f.sign = reinterpret_cast<float*>(h->ws + o_sg);
  f.uoff[0] = 0;
  f.gtotal = 1;
  for (int k = 0; k < d; ++k) {
    f.n[k] = n[k];
    f.r[k] = r[k];
    f.L[k] = L32[k];
    f.qoff[k] = (int64_t)qoff[k];
    f.woff[k] = (int64_t)woff[k];
    f.roff[k] = roff[k];
    f.uoff[k + 1] = f.uoff[k] + n[k] * r[k];
    f.gtotal *= r[k];
  }
  f.utotal = f.uoff[d];
  f.rtotal = rtot;
  {
    StageTimer tm(h, 0);
    nl += launch_kron_finish(f, h->stream);
  }
  return finish(h, nl);
}

rt_status rtucker_relerr(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n, const int32_t* r,
                         const float* U, const float* G, double* out) {
  rt_status st;
  if ((st = check_tensor(h, X, dtype, d, n, nullptr, true)) != RT_OK) return st;
  if (!r || !U || !G || !out) return fail(h, RT_EINVAL, "r, U, G and out are required");
  if (dtype == RT_F8E4M3 && !tucker_relerr_slab_fits(d, n, r))
    return fail(h, RT_ENOTSUP, "evaluator: float8 storage needs r_{d-2} n_{d-1} doubles within 200 KB");
  const size_t sd = tucker_relerr_scratch(d, n, r);
  Bump bump;
  const size_t o = bump.take(sd * 8);
  const size_t o_res = bump.take(16);
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  const float* Uk[MAXD];
  size_t off = 0;
  for (int k = 0; k < d; ++k) { Uk[k] = U + off; off += (size_t)n[k] * r[k]; }
  if (!tucker_relerr_supported(d, n, r)) return fail(h, RT_ENOTSUP, "evaluator: r_d above 64 with a large slab");
  double* res = reinterpret_cast<double*>(h->ws + o_res);
  const int nl = launch_tucker_relerr(X, (int)dtype, d, n, r, Uk, G, reinterpret_cast<double*>(h->ws + o), sd, res,
                                      h->stream, dtype == RT_F8E4M3 ? fp8_scales(X, d, n) : nullptr);
  h->launches = nl;
  RT_CUDA(h, cudaGetLastError());
  double hr[2];
  RT_CUDA(h, cudaMemcpyAsync(hr, res, 16, cudaMemcpyDeviceToHost, h->stream));
  RT_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = (hr[1] > 0) ? sqrt(hr[0] / hr[1]) : 0.0;
  return RT_OK;
}

rt_status rhtucker_decompose(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                             const int32_t* tree_tab, const int32_t* rank, int32_t p, const int64_t* w,
                             uint64_t seed, const rt_options* opt, float* U_leaf, float* B, float* U_nodes) {
  rt_status st;
  int64_t total = 0;
  if ((st = check_tensor(h, X, dtype, d, n, &total)) != RT_OK) return st;
  if ((st = check_opts(h, opt)) != RT_OK) return st;
  if (prec_of(opt) != RT_PREC_FP32) return fail(h, RT_ENOTSUP, "the H-Tucker path computes in float32 only");
  if (!rank || !U_leaf || !B) return fail(h, RT_EINVAL, "rank, U_leaf and B are required");
  if ((st = check_prior_status(h)) != RT_OK) return st;
  if ((st = init_device_attrs(h)) != RT_OK) return st;
  std::vector<TNode> tree;
  if ((st = tree_of(h, d, tree_tab, tree)) != RT_OK) return st;
  const int nn = (int)tree.size();
  std::vector<int> rk(nn);
  for (int i = 0; i < nn; ++i) rk[i] = (i == 0) ? 1 : rank[i];
  int64_t nmax = 0;
  for (int k = 0; k < d; ++k) nmax = std::max(nmax, n[k]);
  // output offsets
  std::vector<size_t> o_unode(nn, 0), o_leaf(nn, 0), o_B(nn, 0);
  size_t acc = 0;
  for (int i = 1; i < nn; ++i) { o_unode[i] = acc; acc += (size_t)range_prod(n, tree[i].a, tree[i].b) * rk[i]; }
  acc = 0;
  for (int k = 0; k < d; ++k)
    for (int i = 1; i < nn; ++i)
      if (tree[i].a == k && tree[i].b == k) { o_leaf[i] = acc; acc += (size_t)n[k] * rk[i]; }
  acc = 0;
  for (int i = 0; i < nn; ++i)
    if (tree[i].a != tree[i].b) { o_B[i] = acc; acc += (size_t)rk[i] * rk[tree[i].left] * rk[tree[i].right]; }
  Group Gp;
  Bump bump;
  std::vector<int> prob_of(nn, -1);
  for (int i = 1; i < nn; ++i) {
    const TNode& nd = tree[i];
    const bool leaf = nd.a == nd.b;
    ProbSpec ps{};
    ps.X = X;
    ps.dtype = dtype;
    ps.d = d;
    for (int j = 0; j < d; ++j) ps.n[j] = n[j];
    ps.a = nd.a;
    ps.b = nd.b;
    ps.r = rk[i];
    ps.p = p;
    const int64_t N = total / range_prod(n, nd.a, nd.b);
    ps.s = w ? w[i] : std::min<int64_t>(20 * nmax, N);
    ps.seed = seed;
    ps.node = (uint32_t)i;
    ps.qr = qr_of(opt);
    ps.U = U_nodes ? U_nodes + o_unode[i] : (leaf ? U_leaf + o_leaf[i] : nullptr);
    ProbPlan pp;
    if ((st = plan_problem(h, ps, bump, pp)) != RT_OK) return st;
    prob_of[i] = (int)Gp.pp.size();
    Gp.pp.push_back(pp);
  }
  group_layout(Gp, bump);
  // transfer jobs (internal non-root nodes): ranks up to TRANSFER_RMAX in one grouped
  // launch, wider ones one by one in the general form; and the root
  std::vector<int> internal, wide;
  size_t gen_floats = 4;
  for (int i = 1; i < nn; ++i) {
    if (tree[i].a == tree[i].b) continue;
    const int rl_i = rk[tree[i].left], rr_i = rk[tree[i].right];
    if (rk[i] <= TRANSFER_RMAX && rl_i <= TRANSFER_RMAX && rr_i <= TRANSFER_RMAX) {
      internal.push_back(i);
    } else {
      wide.push_back(i);
      gen_floats = std::max(gen_floats, transfer_general_floats(range_prod(n, tree[tree[i].left].a,
                                                                           tree[tree[i].left].b),
                                                                rk[i], rl_i, rr_i));
    }
  }
  const size_t o_jobs = bump.take(sizeof(TransferJob) * std::max<size_t>(1, internal.size()));
  const size_t o_tgen = bump.take(gen_floats * 4);
  const TNode& root = tree[0];
  const int64_t nl = range_prod(n, root.a, tree[root.left].b), nr = total / nl;
  const int rl = rk[root.left], rr = rk[root.right];
  const size_t o_rootp = bump.take(root_any_scratch_floats(nl, nr, rl, rr) * 4);
  int64_t tr_ctas = 0;
  for (int i : internal) tr_ctas += transfer_ctas(range_prod(n, tree[tree[i].left].a, tree[tree[i].left].b));
  const size_t o_tpart = bump.take(transfer_part_floats(std::max<int64_t>(1, tr_ctas)) * 4);
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  const size_t sb = group_stage_bytes(Gp) + align_up(sizeof(TransferJob) * std::max<size_t>(1, internal.size()));
  if ((st = ensure_stage(h, sb)) != RT_OK) return st;
  if ((st = group_upload(h, Gp, h->h_stage, 0)) != RT_OK) return st;
  auto Uof = [&](int i) { return Gp.pp[prob_of[i]].q.U; };
  TransferJob* jobs = reinterpret_cast<TransferJob*>(h->h_stage + group_stage_bytes(Gp));
  for (size_t q = 0; q < internal.size(); ++q) {
    const int i = internal[q];
    const TNode& nd = tree[i];
    TransferJob jb;
    jb.US = Uof(i);
    jb.Ul = Uof(nd.left);
    jb.Ur = Uof(nd.right);
    jb.B = B + o_B[i];
    jb.nl = range_prod(n, tree[nd.left].a, tree[nd.left].b);
    jb.nr = range_prod(n, tree[nd.right].a, tree[nd.right].b);
    jb.rS = rk[i];
    jb.rl = rk[nd.left];
    jb.rr = rk[nd.right];
    jb.cta0 = q == 0 ? 0 : jobs[q - 1].cta0 + transfer_ctas(jobs[q - 1].nl);
    jobs[q] = jb;
  }
  if ((st = stage_put(h, h->ws + o_jobs, jobs, sizeof(TransferJob) * internal.size())) != RT_OK) return st;
  int nlaunch = 0;
  if ((st = stage_commit(h, &nlaunch)) != RT_OK) return st;
  const bool graph = opt && opt->use_graph;
  GraphKey key;
  if (graph) {
    key.add(3);
    key.add((uint64_t)h->device);
    key.ptr(h->ws);
    key.add(bump.off);
    key.ptr(X);
    key.add((uint64_t)dtype);
    key.arr(n, d);
    key.arr(rk.data(), nn);
    for (const TNode& t : tree) {
      key.add((uint64_t)(uint32_t)t.left);
      key.add((uint64_t)(uint32_t)t.right);
    }
    key.add((uint64_t)p);
    if (w) key.arr(w, nn);
    key.ptr(U_leaf);
    key.ptr(B);
    key.ptr(U_nodes);
    key.add(o_jobs);
    key.add(o_tgen);
    key.add(o_tpart);
    key.add(o_rootp);
    key.group(Gp.g);
  }
  st = run_kernels(h, graph, key, &nlaunch, [&](int* nk) -> rt_status {
    {
      StageTimer tm(h, 0);
      *nk += launch_range_finder(Gp.g, h->stream, h->d_status);
    }
    if (U_nodes) {
      for (int i = 1; i < nn; ++i)
        if (tree[i].a == tree[i].b)
          RT_CUDA(h, cudaMemcpyAsync(U_leaf + o_leaf[i], U_nodes + o_unode[i], (size_t)n[tree[i].a] * rk[i] * 4,
                                     cudaMemcpyDeviceToDevice, h->stream));
    }
    {
      StageTimer tm(h, 3);
      *nk += launch_transfer(reinterpret_cast<const TransferJob*>(h->ws + o_jobs), jobs, (int)internal.size(),
                             reinterpret_cast<float*>(h->ws + o_tpart), h->stream);
      for (int i : wide) {
        const TNode& nd = tree[i];
        TransferJob jb{};
        jb.US = Uof(i);
        jb.Ul = Uof(nd.left);
        jb.Ur = Uof(nd.right);
        jb.B = B + o_B[i];
        jb.nl = range_prod(n, tree[nd.left].a, tree[nd.left].b);
        jb.nr = range_prod(n, tree[nd.right].a, tree[nd.right].b);
        jb.rS = rk[i];
        jb.rl = rk[nd.left];
        jb.rr = rk[nd.right];
        *nk += launch_transfer_general(jb, reinterpret_cast<float*>(h->ws + o_tgen), h->stream);
      }
    }
    {
      StageTimer tm(h, 4);
      *nk += launch_root_any(X, (int)dtype, nl, nr, Uof(root.left), rl, Uof(root.right), rr, B + o_B[0],
                             reinterpret_cast<float*>(h->ws + o_rootp), h->d_status, h->stream);
    }
    return RT_OK;
  });
  if (st != RT_OK) return st;
  return finish(h, nlaunch);
}

rt_status rhtucker_relerr(rt_handle h, const void* X, rt_dtype dtype, int d, const int64_t* n,
                          const int32_t* tree_tab, const int32_t* rank, const float* U_leaf, const float* B,
                          double* out) {
  rt_status st;
  int64_t total = 0;
  if ((st = check_tensor(h, X, dtype, d, n, &total)) != RT_OK) return st;
  if (!rank || !U_leaf || !B || !out) return fail(h, RT_EINVAL, "rank, U_leaf, B and out are required");
  std::vector<TNode> tree;
  if ((st = tree_of(h, d, tree_tab, tree)) != RT_OK) return st;
  const int nn = (int)tree.size();
  std::vector<int> rk(nn);
  for (int i = 0; i < nn; ++i) rk[i] = (i == 0) ? 1 : rank[i];
  const TNode& root = tree[0];
  for (int i = 1; i < nn; ++i)
    if (rk[i] < 1 || rk[i] > CMAX) return fail(h, RT_EINVAL, "need 1 <= rank <= 64 at every node");
  std::vector<size_t> o_u(nn, 0), o_leaf(nn, 0), o_B(nn, 0);
  Bump bump;
  for (int i = 1; i < nn; ++i) o_u[i] = bump.take((size_t)range_prod(n, tree[i].a, tree[i].b) * rk[i] * 8);
  size_t acc = 0;
  for (int k = 0; k < d; ++k)
    for (int i = 1; i < nn; ++i)
      if (tree[i].a == k && tree[i].b == k) { o_leaf[i] = acc; acc += (size_t)n[k] * rk[i]; }
  acc = 0;
  for (int i = 0; i < nn; ++i)
    if (tree[i].a != tree[i].b) { o_B[i] = acc; acc += (size_t)rk[i] * rk[tree[i].left] * rk[tree[i].right]; }
  const int64_t nl = range_prod(n, root.a, tree[root.left].b), nr = total / nl;
  const size_t o_scr = bump.take(ht_relerr_scratch(nl, nr) * 8);
  const size_t o_res = bump.take(16);
  if ((st = ensure_ws(h, bump.off)) != RT_OK) return st;
  auto U64 = [&](int i) { return reinterpret_cast<double*>(h->ws + o_u[i]); };
  int nlaunch = 0;
  for (int i = 1; i < nn; ++i)
    if (tree[i].a == tree[i].b)
      nlaunch += launch_f32_to_f64(U_leaf + o_leaf[i], U64(i), n[tree[i].a] * rk[i], h->stream);
  int maxlev = 0;
  for (int i = 0; i < nn; ++i) maxlev = std::max(maxlev, tree[i].level);
  for (int lev = maxlev; lev >= 1; --lev)
    for (int i = 1; i < nn; ++i) {
      const TNode& nd = tree[i];
      if (nd.level != lev || nd.a == nd.b) continue;
      nlaunch += launch_ht_expand(U64(nd.left), range_prod(n, tree[nd.left].a, tree[nd.left].b), rk[nd.left],
                                  U64(nd.right), range_prod(n, tree[nd.right].a, tree[nd.right].b), rk[nd.right],
                                  B + o_B[i], rk[i], U64(i), h->stream);
    }
  double* res = reinterpret_cast<double*>(h->ws + o_res);
  nlaunch += launch_ht_relerr(X, (int)dtype, nl, nr, U64(root.left), rk[root.left], B + o_B[0], U64(root.right),
                              rk[root.right], reinterpret_cast<double*>(h->ws + o_scr), res, h->stream);
  h->launches = nlaunch;
  RT_CUDA(h, cudaGetLastError());
  double hr[2];
  RT_CUDA(h, cudaMemcpyAsync(hr, res, 16, cudaMemcpyDeviceToHost, h->stream));
  RT_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = (hr[1] > 0) ? sqrt(hr[0] / hr[1]) : 0.0;
  return RT_OK;
}

}  // extern "C"
