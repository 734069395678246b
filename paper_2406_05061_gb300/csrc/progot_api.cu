// Host orchestration of the ProgOT hot path and its C ABI (include/progot.h).
//
// The Sinkhorn loop of Alg. 1 runs without a host round trip per iteration: every
// f-sweep measures the row-marginal error of the current (f, g) in its epilogue and the
// stop test runs on the device (SolverState): in the f-sweep's last CTA, or, in
// tensor-core loops, in the g-sweep that follows (SweepParams::lag). Later sweeps of a
// stopped loop return at entry, so the host enqueues iterations in growing chunks and
// reads the state back (pinned memory, one event per chunk) while the next chunk is
// already queued. The tensor-core operands are centred (prep_tc) and the large-n
// sweeps split whole row blocks in bands (tc::Split).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/progot.h"
#include "progot_internal.h"

namespace progot {

static std::atomic<int64_t> g_launches{0};
static std::atomic<int32_t> g_stall_window{512};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local std::string t_last_error;
void set_last_error_message(const char* msg) { t_last_error = msg ? msg : ""; }

// Opt-in per-kernel timing (progot_profile): CUDA events recorded on the launching
// stream. Inside a Sinkhorn loop the events bracket each enqueued chunk of sweeps (an
// event between two sweeps would break their programmatic overlap), and a chunk counts
// only when all of its launches did work (launches after the loop's stop return at
// entry); other sweeps (map passes, metrics) are sampled launch by launch.
enum ProfKind { kProfLse = 0, kProfMap = 1, kProfKinds = 2 };
struct ProfRec {
  cudaEvent_t a, b;
  int kind;
  double pairs;
  bool counted;
  int64_t seq;     // sequence number of the launch among all profiled-kernel launches
  int64_t nl = 1;  // launches bracketed by the two events
};
struct Profiler {
  bool on = false;
  int64_t period = 1;                   // events around every period-th launch of a kind
  int64_t seq[kProfKinds] = {0, 0};     // launches of each kind seen while on
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  double ms[kProfKinds] = {0, 0};
  double pairs[kProfKinds] = {0, 0};
  int64_t launches[kProfKinds] = {0, 0};
  int64_t worked[kProfKinds] = {0, 0};  // launches that did work, sampled or not
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
static thread_local Profiler t_prof;

// True when this launch is sampled (events recorded around it).
static bool prof_begin(ProfRec& r, cudaStream_t s, int kind) {
  if (!t_prof.on) return false;
  r.seq = t_prof.seq[kind]++;
  if (r.seq % t_prof.period != 0) return false;
  r.a = t_prof.get();
  r.b = t_prof.get();
  cudaEventRecord(r.a, s);
  return true;
}
static void prof_end(ProfRec& r, cudaStream_t s, int kind, double pairs) {
  cudaEventRecord(r.b, s);
  r.kind = kind;
  r.pairs = pairs;
  r.counted = true;
  t_prof.recs.push_back(r);
}
// Fold finished records into the totals (synchronises on their events).
static void prof_collect() {
  for (ProfRec& r : t_prof.recs) {
    if (r.counted) {
      float ms = 0.f;
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&ms, r.a, r.b);
      t_prof.ms[r.kind] += ms;
      t_prof.pairs[r.kind] += r.pairs;
      t_prof.launches[r.kind] += r.nl;
    } else {
      cudaEventSynchronize(r.b);
    }
    t_prof.pool.push_back(r.a);
    t_prof.pool.push_back(r.b);
  }
  t_prof.recs.clear();
}

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(PROGOT_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static int num_sms() {
  static thread_local int cached = 0;
  if (cached) return cached;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
  cached = sms;
  return sms;
}

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Column splits of a sweep of nA rows against nB columns. Each CTA covers one 128-row
// block and `tiles_per_split` 128-column tiles; about kWaves waves of CTAs on the GPU's
// resident slots (ctas_per_sm per SM) let the hardware scheduler balance the SMs, and
// a CTA never gets fewer than one tile. Returns the split count.
constexpr int64_t kWaves = 6;
static int plan_splits(int64_t nA, int64_t nB, int ctas_per_sm, int extra_mult = 1) {
  const int64_t rb = cdiv(nA, fp32_tile_rows()) * extra_mult;
  const int64_t ct = cdiv(nB, fp32_tile_cols());
  const int64_t slots = (int64_t)num_sms() * ctas_per_sm;
  int64_t tps = (rb * ct) / (slots * kWaves);
  if (tps < 1) tps = 1;
  if (tps > ct) tps = ct;
  return (int)cdiv(ct, tps);
}

// Device workspace carved from the caller's buffer.
struct Workspace {
  float* xn;        // nmax
  float* yn;        // nmax
  float* f0;        // nmax
  float* f1;        // nmax
  float* gaux;      // nmax
  float* L;         // nmax
  float* T;         // nmax * d
  float2* partial;  // partial_elems
  float* wpart;     // partial_elems (tilted sums of the coupling-metrics sweep)
  float* cpart;     // partial_elems (cross-cloud cost sums of the coupling-metrics sweep)
  double* metpart;  // kMetricSums * (rbmax + 2)
  double* metout;   // 2 * kMetricSums + 2: reduced metric sums (row sweep, column sweep), mean cost
  double* errpart;  // rbmax + 2
  unsigned* cnt;    // rbmax + 2
  unsigned* mcnt;   // rbmax + 2
  SolverState* state;  // [2]
  double* rpart;    // parts * (d + 1)
  double* rout;     // 2 * (d + 1)
  float* Opart;     // opart_elems
  float* Rpart;     // rpart_elems
  void* xh;         // bf16 hi/lo operands of the tensor-core sweeps: nmax x dp each
  void* xl;
  void* yh;
  void* yl;
  void* xb;         // bf16 bias rows (x side, rows padded to 128) x 16
  void* yb;
  float* mu;        // d: centre of the tensor-core operands
  float* xnc;       // nmax: |x_i - mu|^2
  float* ync;       // nmax: |y_j - mu|^2
  int32_t* fault;   // set by a tensor-core CTA whose bounded wait expired
  // persistent tensor-core Sinkhorn loop
  void* xb2;        // second bias-row buffers (the loop alternates xb / xb2 and yb / yb2)
  void* yb2;
  uint32_t* lflag;  // ready flags: x row blocks [rbmax], y row blocks [rbmax]
  unsigned long long* lcnt;  // arrivals: x row blocks [rbmax], y row blocks [rbmax], done_x, done_y
  float2* lpart;    // (max, sum) slots: f-update bank, then g-update bank (lslots each)
  int64_t lslots;
  int64_t lrb;      // rbmax of the carve (row-block capacity of lcnt and lerr)
  int4* ltab_segs;  // work-split tables of both sides: segments [2][lslots], contributor slots
  int32_t* ltab_cslot;  // [2][lslots], contributor offsets [2][rbmax + 1], segment counts [2][sms]
  int32_t* ltab_cptr;
  int32_t* ltab_nseg;
  double* lerr;     // [2][rbmax] error partials by iteration parity
  size_t bytes;
};

struct WsDims {
  int64_t nmax, rbmax, partial_elems, opart_elems, rpart_elems;
  int32_t d, dp;
  bool tc;
};

static int32_t pad64(int32_t d) { return (d + 63) / 64 * 64; }

static WsDims ws_dims(int64_t n, int64_t m, int32_t d, int32_t precision = PROGOT_FP32) {
  WsDims w;
  w.tc = precision != PROGOT_FP32;
  w.dp = pad64(d);
  w.nmax = std::max<int64_t>(std::max<int64_t>(n, m), 1);
  w.d = d;
  w.rbmax = cdiv(w.nmax, fp32_tile_rows());
  // Bound on splits * nA for both sweep directions. With X = rb ct / (slots W):
  // X < 1 gives tps = 1 and splits = ct, so splits * nA <= rb ct BM < slots W BM;
  // X >= 1 gives tps = floor(X) >= X / 2 and splits <= ct / tps + 1 <= 2 slots W / rb + 1,
  // so splits * nA <= (2 slots W + rb) BM.
  const int64_t BMr = fp32_tile_rows();
  const int64_t slots = (int64_t)num_sms() * 2;
  w.partial_elems = (2 * slots * kWaves + w.rbmax + 1) * BMr + w.nmax;
  const int64_t dch = cdiv(d, map_dchunk());
  const int64_t mslots = (int64_t)num_sms();
  const int64_t rows_cap = (2 * mslots * kWaves / dch + w.rbmax + 1) * BMr + w.nmax;
  w.opart_elems = rows_cap * d;
  w.rpart_elems = rows_cap;
  if (w.tc && w.dp <= 256) {
    // tensor-core map steps: G * maxseg <= R + 3 G partial slots of 128 rows x dp
    const int64_t slots = w.rbmax + 3 * (int64_t)num_sms();
    w.opart_elems = std::max<int64_t>(w.opart_elems, slots * BMr * w.dp);
    w.rpart_elems = std::max<int64_t>(w.rpart_elems, slots * BMr);
  }
  return w;
}

static size_t ws_layout(const WsDims& w, Workspace* out, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  Workspace ws;
  ws.xn = (float*)take(sizeof(float) * w.nmax);
  ws.yn = (float*)take(sizeof(float) * w.nmax);
  ws.f0 = (float*)take(sizeof(float) * w.nmax);
  ws.f1 = (float*)take(sizeof(float) * w.nmax);
  ws.gaux = (float*)take(sizeof(float) * w.nmax);
  ws.L = (float*)take(sizeof(float) * w.nmax);
  ws.T = (float*)take(sizeof(float) * w.nmax * (size_t)w.d);
  ws.partial = (float2*)take(sizeof(float2) * w.partial_elems);
  ws.wpart = (float*)take(sizeof(float) * w.partial_elems);
  ws.cpart = (float*)take(sizeof(float) * w.partial_elems);
  ws.metpart = (double*)take(sizeof(double) * kMetricSums * (w.rbmax + 2));
  ws.metout = (double*)take(sizeof(double) * (2 * kMetricSums + 2));
  ws.errpart = (double*)take(sizeof(double) * (w.rbmax + 2));
  ws.cnt = (unsigned*)take(sizeof(unsigned) * (w.rbmax + 2));
  ws.mcnt = (unsigned*)take(sizeof(unsigned) * (w.rbmax + 2));
  ws.state = (SolverState*)take(2 * sizeof(SolverState));  // [2]: see SweepParams::lag
  ws.rpart = (double*)take(sizeof(double) * reduce_parts() * (size_t)(w.d + 1));
  ws.rout = (double*)take(sizeof(double) * 2 * (size_t)(w.d + 1));
  ws.Opart = (float*)take(sizeof(float) * w.opart_elems);
  ws.Rpart = (float*)take(sizeof(float) * w.rpart_elems);
  const size_t opb = w.tc ? 2 * (size_t)w.nmax * (size_t)w.dp : 0;
  ws.xh = take(opb);
  ws.xl = take(opb);
  ws.yh = take(opb);
  ws.yl = take(opb);
  const size_t bb = w.tc ? 32 * (size_t)(cdiv(w.nmax, 256) * 256) : 0;
  ws.xb = take(bb);
  ws.yb = take(bb);
  ws.mu = (float*)take(w.tc ? sizeof(float) * (size_t)w.dp : 0);
  ws.xnc = (float*)take(w.tc ? sizeof(float) * w.nmax : 0);
  ws.ync = (float*)take(w.tc ? sizeof(float) * w.nmax : 0);
  ws.fault = (int32_t*)take(sizeof(int32_t));
  ws.xb2 = take(bb);
  ws.yb2 = take(bb);
  ws.lflag = (uint32_t*)take(w.tc ? sizeof(uint32_t) * 2 * (size_t)w.rbmax : 0);
  ws.lcnt = (unsigned long long*)take(w.tc ? sizeof(unsigned long long) * (2 * (size_t)w.rbmax + 2) : 0);
  // G * maxseg <= R + 2 G slots of 128 rows per bank (each CTA's segments: its whole row
  // blocks, plus at most two partial ones of the contiguous remainder)
  ws.lslots = w.tc ? w.rbmax + 3 * (int64_t)num_sms() : 0;
  // (max, sum) per slot, LSE warpgroup and row; one bank per update direction
  ws.lpart = (float2*)take(sizeof(float2) * 2 * (size_t)ws.lslots * 2 * 128);
  ws.lrb = w.rbmax;
  ws.ltab_segs = (int4*)take(sizeof(int4) * 2 * (size_t)ws.lslots);
  ws.ltab_cslot = (int32_t*)take(sizeof(int32_t) * 2 * (size_t)ws.lslots);
  ws.ltab_cptr = (int32_t*)take(w.tc ? sizeof(int32_t) * 2 * ((size_t)w.rbmax + 1) : 0);
  ws.ltab_nseg = (int32_t*)take(w.tc ? sizeof(int32_t) * 2 * (size_t)num_sms() : 0);
  ws.lerr = (double*)take(w.tc ? sizeof(double) * 2 * (size_t)w.rbmax : 0);
  ws.bytes = off;
  if (out) *out = ws;
  return off;
}

static int carve(int64_t n, int64_t m, int32_t d, void* workspace, size_t ws_bytes, Workspace* ws,
                 int32_t precision = PROGOT_FP32) {
  if (workspace == nullptr) return fail(PROGOT_ERR_WORKSPACE, "workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(PROGOT_ERR_WORKSPACE, "workspace is not 256-byte aligned");
  const WsDims w = ws_dims(n, m, d, precision);
  const size_t need = ws_layout(w, ws, (char*)workspace);
  if (ws_bytes < need)
    return fail(PROGOT_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, need);
  return PROGOT_OK;
}

// Pinned host mirror of the solver state, one pair per host thread.
struct HostMirror {
  SolverState* hs = nullptr;  // [2], pinned
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double* hd = nullptr;  // pinned doubles for reductions
  bool ok = false;
  int init() {
    if (ok) return PROGOT_OK;
    CK(cudaHostAlloc((void**)&hs, 2 * sizeof(SolverState), cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&hd, 1024 * sizeof(double), cudaHostAllocDefault));
    CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    ok = true;
    return PROGOT_OK;
  }
};
static thread_local HostMirror t_host;

// Tensor-core map step for d <= 64 on the tensor-core path (progot_set_map_tc).
static std::atomic<int> g_map_tc{1};
// Persistent tensor-core Sinkhorn loop (progot_set_loop_tc) and the bounded-wait limit of
// the tensor-core kernels (progot_set_wait_limit_ns).
static std::atomic<int> g_loop_tc{1};
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;
static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
// Test hook (progot_test_withhold_initial_betas): the persistent loop starts without the
// initial betas of g, so its first tiles wait on words that no sweep writes.
static std::atomic<int> g_withhold_betas{0};

static int check_common(const float* x, int64_t n, const float* y, int64_t m, int32_t d, int32_t precision) {
  if (x == nullptr || y == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "x and y must not be NULL");
  if (n <= 0 || m <= 0 || d <= 0) return fail(PROGOT_ERR_INVALID_ARG, "n, m, d must be positive (got %lld, %lld, %d)",
                                              (long long)n, (long long)m, d);
  if (n > (int64_t)1 << 31 || m > (int64_t)1 << 31)
    return fail(PROGOT_ERR_INVALID_ARG, "n and m must be below 2^31");
  if (precision != PROGOT_FP32 && precision != PROGOT_BF16X3 && precision != PROGOT_BF16)
    return fail(PROGOT_ERR_INVALID_ARG, "unknown precision %d", precision);
  return PROGOT_OK;
}

// ---------------------------------------------------------------- tensor-core operands
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// 2-D bf16 tensor map over a (rows x dp) row-major buffer with boxes of box_rows rows:
// 64-wide boxes with 128-byte swizzle for operands (dp a multiple of 64), or 16-wide
// boxes with 32-byte swizzle for bias rows (dp = 16).
static int make_map(CUtensorMap* map, void* base, int64_t rows, int32_t dp, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return fail(PROGOT_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const bool bias = dp == 16;
  cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
  cuuint32_t box[2] = {bias ? 16u : 64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, bias ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PROGOT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PROGOT_OK;
}

int encode_operand_map(void* map, void* base, int64_t rows, int32_t dp, int box_rows) {
  return make_map(reinterpret_cast<CUtensorMap*>(map), base, rows, dp, box_rows);
}
int32_t stall_window_setting() { return g_stall_window.load(); }
unsigned long long wait_limit_setting() { return g_wait_ns.load(); }
int device_sm_count() { return num_sms(); }
int fail_message(int code, const char* msg) { return fail(code, "%s", msg); }

struct TcOps {
  // operand maps in the A role (128-row boxes) and the B role (bn-row boxes), bias maps
  // (bn-row boxes); CUtensorMap is 64-byte aligned by its own declaration
  CUtensorMap xh_a, xl_a, yh_a, yl_a, xh_b, xl_b, yh_b, yl_b, xb, yb;
  // tensor-core map step (dp = 64): y-side bias rows in 128-row boxes
  CUtensorMap yb128;
  // tensor-core map step for 64 < d <= 256: y operand and bias rows in 32-row boxes
  CUtensorMap yh_m32, yl_m32, yb_m32;
  // centre mu of the operands and the squared norms |x_i - mu|^2, |y_j - mu|^2 that
  // the tensor-core sweeps use in place of |x_i|^2, |y_j|^2
  const float* mu = nullptr;
  const float* xnc = nullptr;
  const float* ync = nullptr;
  int nkb = 0;
  int split3 = 0;
  int bn = 128;
  bool on = false;
  // ws.L holds the row log-sum-exps of t against the y-side bias rows (the map step's
  // stabiliser), written by the persistent loop from its last f-update
  bool lse_ready = false;
};

// Split sqrt(2 log2(e) / eps) (X - mu) and (Y - mu) into bf16 hi/lo and describe them
// for TMA; write the bias rows of both sides from the current potentials (f on x, g on
// y) and the centred squared norms. mu is the midpoint of the two clouds' means: the
// cost |x - y|^2 = |x~|^2 + |y~|^2 - 2 x~ . y~ holds for any common centre, and the
// bf16x3 products and their float32 accumulation lose accuracy in proportion to
// |x~| |y~|, which centring keeps near the clouds' spread rather than their distance
// from the origin. The potentials are the same for every centre.
static int prep_tc(const float* x, int64_t n, const float* y, int64_t m, int32_t d, double eps, int32_t precision,
                   const Workspace& ws, TcOps* ops, cudaStream_t s, const float* f_cur = nullptr,
                   const float* g_cur = nullptr) {
  ops->on = precision != PROGOT_FP32;
  ops->lse_ready = false;
  if (!ops->on) return PROGOT_OK;
  const int32_t dp = pad64(d);
  ops->nkb = dp / 64;
  ops->split3 = precision == PROGOT_BF16X3 ? 1 : 0;
  if (tc_stages(ops->nkb, ops->split3) < 2)
    return fail(PROGOT_ERR_INVALID_ARG, "d = %d is too large for the tensor-core sweep", d);
  const float sc = (float)std::sqrt(2.0 * kLog2e / eps);
  CK(launch_center(x, n, y, m, d, ws.rpart, ws.mu, s));
  ops->mu = ws.mu;
  ops->xnc = ws.xnc;
  ops->ync = ws.ync;
  CK(launch_split_bf16(x, n, d, dp, sc, ws.xh, ops->split3 ? ws.xl : nullptr, s, ws.mu, ws.xnc));
  CK(launch_split_bf16(y, m, d, dp, sc, ws.yh, ops->split3 ? ws.yl : nullptr, s, ws.mu, ws.ync));
  ops->bn = tc_tile_cols(ops->nkb, ops->split3);
  void* xl = ops->split3 ? ws.xl : ws.xh;
  void* yl = ops->split3 ? ws.yl : ws.yh;
  int rc = make_map(&ops->xh_a, ws.xh, n, dp, 128);
  if (!rc) rc = make_map(&ops->xl_a, xl, n, dp, 128);
  if (!rc) rc = make_map(&ops->yh_a, ws.yh, m, dp, 128);
  if (!rc) rc = make_map(&ops->yl_a, yl, m, dp, 128);
  if (!rc) rc = make_map(&ops->xh_b, ws.xh, n, dp, ops->bn);
  if (!rc) rc = make_map(&ops->xl_b, xl, n, dp, ops->bn);
  if (!rc) rc = make_map(&ops->yh_b, ws.yh, m, dp, ops->bn);
  if (!rc) rc = make_map(&ops->yl_b, yl, m, dp, ops->bn);
  if (!rc) rc = make_map(&ops->xb, ws.xb, cdiv(n, 256) * 256, 16, ops->bn);
  if (!rc) rc = make_map(&ops->yb, ws.yb, cdiv(m, 256) * 256, 16, ops->bn);
  if (!rc && dp == 64) {
    rc = make_map(&ops->yb128, ws.yb, cdiv(m, 256) * 256, 16, 128);
  }
  if (!rc && dp > 64 && map_tc_onepass_supported(ops->nkb)) {
    const int bt = map_tc_onepass_tile_cols();
    rc = make_map(&ops->yh_m32, ws.yh, m, dp, bt);
    if (!rc) rc = make_map(&ops->yl_m32, yl, m, dp, bt);
    if (!rc) rc = make_map(&ops->yb_m32, ws.yb, cdiv(m, 256) * 256, 16, bt);
  }
  if (rc) return rc;
  const float bscale = (float)(kLog2e / eps);
  if (g_cur != nullptr) CK(launch_bias_prep(g_cur, ws.ync, m, cdiv(m, 256) * 256, bscale, ws.yb, s));
  if (f_cur != nullptr) CK(launch_bias_prep(f_cur, ws.xnc, n, cdiv(n, 256) * 256, bscale, ws.xb, s));
  return PROGOT_OK;
}

// One sweep description for "update the potential of A from the potential of B".
static SweepParams make_sweep(const float* A, int64_t nA, const float* B, int64_t nB, int32_t d, const float* An,
                              const float* Bn, double eps, const Workspace& ws, int ctas_per_sm = 2) {
  SweepParams p;
  memset(&p, 0, sizeof(p));
  p.A = A;
  p.B = B;
  p.An = An;
  p.Bn = Bn;
  p.nA = nA;
  p.nB = nB;
  p.d = d;
  p.splits = plan_splits(nA, nB, ctas_per_sm);
  const int64_t ct = cdiv(nB, fp32_tile_cols());
  p.tiles_per_split = (int)cdiv(ct, p.splits);
  p.splits = (int)cdiv(ct, p.tiles_per_split);  // drop empty splits
  p.scale = (float)(2.0 * kLog2e / eps);
  p.bscale = (float)(kLog2e / eps);
  p.eps = eps;
  p.inv_eps_f = (float)(1.0 / eps);
  p.inv_nA = 1.0 / (double)nA;
  p.log_w_uniform = std::log(1.0 / (double)nA);
  p.partial = ws.partial;
  p.wpart = ws.wpart;
  p.metpart = ws.metpart;
  p.errpart = ws.errpart;
  p.cnt = ws.cnt;
  p.stall_window = g_stall_window.load();
  return p;
}

// The ground cost of a sweep: the squared Euclidean cost (default) or the p-norm cost
// h(z) = (1/p) sum_k |z_k|^p of the coupling experiments (Sec. 5.2), float32 CUDA cores.
struct Cost {
  int32_t kind = kCostSqEuclid;
  float p = 2.f;
  bool pnorm() const { return kind != kCostSqEuclid; }
};

static int pnorm_cost(double p, Cost* c) {
  if (!(p > 1.0) || !(p <= 8.0))
    return fail(PROGOT_ERR_INVALID_ARG, "the p-norm cost needs 1 < p <= 8 (got %g)", p);
  c->kind = (p == 1.5) ? kCostP15 : kCostPGeneral;
  c->p = (float)p;
  return PROGOT_OK;
}

// Switch a sweep built by make_sweep to the p-norm cost: t_ij = (potB_j - h(a_i - b_j))
// log2(e) / eps, i.e. scale = -log2(e) / (eps p) on sum_k |a_ik - b_jk|^p and no norms.
static void apply_cost(SweepParams& sp, const Cost& c, double eps) {
  if (!c.pnorm()) return;
  sp.cost = c.kind;
  sp.cost_p = c.p;
  sp.scale = (float)(-kLog2e / (eps * (double)c.p));
  sp.An = nullptr;
  sp.Bn = nullptr;
}

// Launch one log-sum-exp sweep: float32 CUDA cores, or tcgen05 on the prepared split
// operands (a_is_x: rows of the sweep are the x cloud).
static int lse_sweep(const SweepParams& p, int32_t precision, cudaStream_t s, const TcOps* ops = nullptr,
                     bool a_is_x = true, const Workspace* ws = nullptr, bool in_loop = false) {
  ProfRec r;
  const bool rec = !in_loop && prof_begin(r, s, kProfLse);
  if (precision != PROGOT_FP32 && ops != nullptr && ops->on) {
    const CUtensorMap* ah = a_is_x ? &ops->xh_a : &ops->yh_a;
    const CUtensorMap* al = a_is_x ? &ops->xl_a : &ops->yl_a;
    const CUtensorMap* bh = a_is_x ? &ops->yh_b : &ops->xh_b;
    const CUtensorMap* bl = a_is_x ? &ops->yl_b : &ops->xl_b;
    const CUtensorMap* bb = a_is_x ? &ops->yb : &ops->xb;
    void* bias_out = (p.mode == kModePotential && ws) ? (a_is_x ? ws->xb : ws->yb) : nullptr;
    int G = 0, maxseg = 0;
    tc_plan(p.nA, p.nB, ops->bn, num_sms(), &G, &maxseg);
    SweepParams q = p;
    q.splits = G;  // not used by the persistent kernel beyond bookkeeping
    // the operands are centred: the row constants of the epilogue are the centred norms
    if (q.An != nullptr) q.An = a_is_x ? ops->xnc : ops->ync;
    if (q.Bn != nullptr) q.Bn = a_is_x ? ops->ync : ops->xnc;
    CK(launch_lse_sweep_tc(q, ah, al, bh, bl, bb, ops->nkb, ops->split3, ops->bn, G, maxseg,
                           ws ? ws->fault : nullptr, bias_out, s));
  } else {
    CK(launch_lse_sweep_fp32(p, s));
  }
  if (rec) prof_end(r, s, kProfLse, (double)p.nA * (double)p.nB);
  if (t_prof.on && p.state == nullptr) t_prof.worked[kProfLse] += 1;
  return PROGOT_OK;
}

// Sinkhorn loop (Alg. 1) as one persistent tensor-core launch (loop_tc.cu): the bias rows
// of each update's potential pass between the GPU's CTAs behind per-row-block ready
// flags, the stop test runs inside the kernel. pf and pg are the f- and g-update
// descriptions built by sinkhorn_core; ops describes the prepared operands, whose bias
// rows (ws.xb from f, ws.yb from g) prep_tc has written. On return the current f is in
// f_a, g in g, and the y-side bias rows (ws.yb) hold g for a map step at the same eps.
static int sinkhorn_loop_persistent(SweepParams pf, SweepParams pg, int64_t n, int64_t m, int32_t max_iter,
                                    double tau, float* f_a, float* f_b, float* g, const Workspace& ws,
                                    TcOps& ops, int32_t* iters_out, double* err_out, cudaStream_t s) {
  pf.An = ops.xnc;
  pf.Bn = ops.ync;
  pg.An = ops.ync;
  pg.Bn = ops.xnc;
  const int64_t rb = ws.lrb;
  // the second bias buffers: their padding rows (-inf) matter, the others are written
  // by the sweeps before any tile reads them
  CK(launch_bias_prep(f_a, ops.xnc, n, cdiv(n, 256) * 256, pf.bscale, ws.xb2, s));
  CK(launch_bias_prep(g, ops.ync, m, cdiv(m, 256) * 256, pf.bscale, ws.yb2, s));
  // ready flags: nothing published, then the initial g's row blocks (in ws.yb) as flag 1,
  // which the first f-update waits for. The test hook leaves them unpublished, so the
  // first f-update's bounded wait expires.
  CK(cudaMemsetAsync(ws.lflag, 0, sizeof(uint32_t) * 2 * (size_t)rb, s));
  if (!g_withhold_betas.load()) CK(launch_fill_u32(ws.lflag + rb, cdiv(m, 128), 1u, s));
  CK(cudaMemsetAsync(ws.lcnt, 0, sizeof(unsigned long long) * (2 * (size_t)rb + 2), s));
  CK(launch_init_state(ws.state, s));
  CUtensorMap xb2_map, yb2_map;
  int rc = make_map(&xb2_map, ws.xb2, cdiv(n, 256) * 256, 16, ops.bn);
  if (!rc) rc = make_map(&yb2_map, ws.yb2, cdiv(m, 256) * 256, 16, ops.bn);
  if (rc) return rc;
  LoopLaunch L;
  memset(&L, 0, sizeof(L));
  LoopSideLaunch& F = L.side[0];
  LoopSideLaunch& Gs = L.side[1];
  F.p = pf;
  F.out0 = f_a;
  F.out1 = f_b;
  F.bias_out[0] = ws.xb;
  F.bias_out[1] = ws.xb2;
  F.flag_out = ws.lflag;
  F.flag_in = ws.lflag + rb;
  F.cnt = ws.lcnt;
  F.done = ws.lcnt + 2 * rb;
  F.partial = ws.lpart;
  F.segs = ws.ltab_segs;
  F.cslot = ws.ltab_cslot;
  F.cptr = ws.ltab_cptr;
  F.nseg = ws.ltab_nseg;
  F.table_slots = ws.lslots;
  Gs.p = pg;
  Gs.out0 = g;
  Gs.out1 = nullptr;
  Gs.bias_out[0] = ws.yb;
  Gs.bias_out[1] = ws.yb2;
  Gs.flag_out = ws.lflag + rb;
  Gs.flag_in = ws.lflag;
  Gs.cnt = ws.lcnt + rb;
  Gs.done = ws.lcnt + 2 * rb + 1;
  Gs.partial = ws.lpart + ws.lslots * 2 * 128;
  Gs.segs = ws.ltab_segs + ws.lslots;
  Gs.cslot = ws.ltab_cslot + ws.lslots;
  Gs.cptr = ws.ltab_cptr + (rb + 1);
  Gs.nseg = ws.ltab_nseg + num_sms();
  Gs.table_slots = ws.lslots;
  const CUtensorMap* maps[12] = {&ops.xh_a, &ops.xl_a, &ops.yh_a, &ops.yl_a, &ops.xh_b, &ops.xl_b,
                                 &ops.yh_b, &ops.yl_b, &ops.xb,   &xb2_map,   &ops.yb,   &yb2_map};
  for (int q = 0; q < 12; ++q) L.maps[q] = maps[q];
  L.errpart = ws.lerr;
  L.state = ws.state;
  L.fault = ws.fault;
  L.wait_ns = g_wait_ns.load();
  L.nkb = ops.nkb;
  L.split3 = ops.split3;
  L.bn = ops.bn;
  loop_tc_plan(n, m, ops.bn, num_sms(), &L.G, &L.maxseg);
  if ((int64_t)L.G * L.maxseg > ws.lslots)
    return fail(PROGOT_ERR_WORKSPACE, "persistent loop needs %lld partial slots, the workspace has %lld",
                (long long)L.G * L.maxseg, (long long)ws.lslots);
  L.seq0 = 0;
  // max_iter + 1 f-updates always reach the stop test's max_iter branch; the tags of
  // sweep k are 2 k + 1 and 2 k + 2, so iterations stay below 2^30
  L.niter = (int)std::min<int64_t>((int64_t)max_iter + 1, (int64_t)1 << 30);
  ProfRec pr;
  if (t_prof.on) {
    pr.a = t_prof.get();
    pr.b = t_prof.get();
    pr.kind = kProfLse;
    pr.seq = t_prof.seq[kProfLse];
    CK(cudaEventRecord(pr.a, s));
  }
  CK(launch_sinkhorn_loop_tc(L, s));
  if (t_prof.on) CK(cudaEventRecord(pr.b, s));
  rc = t_host.init();
  if (rc) return rc;
  int32_t fault = 0;
  CK(cudaMemcpyAsync(&t_host.hs[0], ws.state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&fault, ws.fault, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const SolverState fin = t_host.hs[0];
  if (fault) return fail(PROGOT_ERR_TIMEOUT, "the persistent Sinkhorn loop hit its bounded wait and aborted");
  // every iteration up to the stop ran both sweeps (the last g-update without writes)
  const int64_t sweeps = 2 * ((int64_t)fin.it + 1);
  if (t_prof.on) {
    pr.nl = sweeps;
    pr.pairs = (double)sweeps * (double)n * (double)m;
    pr.counted = true;
    t_prof.recs.push_back(pr);
    t_prof.seq[kProfLse] += sweeps;
    t_prof.worked[kProfLse] += sweeps;
  }
  // The loop stops after an f-update whose result it does not adopt (f stays the iterate
  // the stop test measured, g is unchanged): that update formed f_new from exactly the
  // t_ij = c x~.y~ + beta(g) of a map step that follows, so its row log-sum-exps, read
  // back from f_new, are the map step's L and spare it a sweep.
  if (fin.status != kNumeric) {
    CK(launch_lse_from_potential(fin.fcur == 0 ? f_b : f_a, ops.xnc, pf.wA, pf.log_w_uniform, pf.eps, n, ws.L, s));
    ops.lse_ready = true;
  }
  if (fin.fcur == 1) CK(cudaMemcpyAsync(f_a, f_b, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  // the map step that may follow reads g through the y-side bias rows
  CK(launch_bias_prep(g, ops.ync, m, cdiv(m, 256) * 256, pf.bscale, ws.yb, s));
  if (iters_out) *iters_out = fin.it;
  if (err_out) *err_out = fin.err;
  switch (fin.status) {
    case kConverged:
      return PROGOT_OK;
    case kNumeric:
      return fail(PROGOT_ERR_NUMERIC, "non-finite marginal error after %d iterations", fin.it);
    case kStalled:
      return fail(PROGOT_ERR_NOT_CONVERGED, "marginal error %.3e stalled above tau %.3e after %d iterations", fin.err,
                  tau, fin.it);
    default:
      return fail(PROGOT_ERR_NOT_CONVERGED, "marginal error %.3e above tau %.3e after %d iterations", fin.err, tau,
                  fin.it);
  }
}

// Sinkhorn loop (Alg. 1) on device-resident state. f lives in {f_a, f_b} (ping-pong);
// on return the current f is copied into f_a. Norms xn, yn must be ready.
// ops_out (optional) receives the tensor-core operand descriptions, valid for a map
// step on the same (x, y, eps) right after the loop (the y-side bias rows then hold g).
// symmetric: self-transport (y = x, b = a) by the averaged fixed point
// f <- (f + f_new) / 2 with one sweep per iteration (potB = f); the symmetric coupling
// P_ij = exp((f_i + f_j - C_ij)/eps) then has both marginals equal, and on return g
// (when not NULL) receives f.
static int sinkhorn_core(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                         int32_t d, double eps, double tau, int32_t max_iter, int32_t precision, float* f_a, float* f_b,
                         float* g, const float* xn, const float* yn, const Workspace& ws, int32_t* iters_out,
                         double* err_out, cudaStream_t s, TcOps* ops_out = nullptr, bool symmetric = false,
                         const Cost& cost = Cost()) {
  int rc = t_host.init();
  if (rc) return rc;
  TcOps ops_local;
  TcOps& ops = ops_out ? *ops_out : ops_local;
  if (cost.pnorm()) {
    ops.on = false;  // the p-norm cost runs on CUDA cores (float32)
    precision = PROGOT_FP32;
  } else {
    rc = prep_tc(x, n, y, m, d, eps, precision, ws, &ops, s, f_a, symmetric ? f_a : g);
    if (rc) return rc;
  }
  const int cps = ops.on ? 1 : 2;
  CK(launch_init_state(ws.state, s));
  SweepParams pf = make_sweep(x, n, y, m, d, xn, yn, eps, ws, cps);
  pf.wA = a;
  pf.potB = symmetric ? f_a : g;
  pf.potB_alt = symmetric ? f_b : nullptr;
  pf.out = f_a;
  pf.out_alt = f_b;
  pf.mode = kModePotential;
  pf.role = symmetric ? 3 : 1;
  pf.state = ws.state;
  pf.tau = tau;
  pf.max_iter = max_iter;
  apply_cost(pf, cost, eps);
  SweepParams pg = make_sweep(y, m, x, n, d, yn, xn, eps, ws, cps);
  pg.wA = b;
  pg.potB = f_a;
  pg.potB_alt = f_b;
  pg.out = g;
  pg.mode = kModePotential;
  pg.role = 2;
  pg.state = ws.state;
  pg.tau = tau;
  pg.max_iter = max_iter;
  apply_cost(pg, cost, eps);
  // tensor-core loops run the stop test of an f-update in the g-update that follows it
  // (SweepParams::lag): the f-update's last row block then ends the sweep without a
  // sweep-level arrival and finish
  const bool lag = ops.on && !symmetric;
  pf.lag = pg.lag = lag ? 1 : 0;
  if (lag && g_loop_tc.load() && loop_tc_supported(ops.bn, ops.nkb, ops.split3)) {
    pf.lag = pg.lag = 0;
    return sinkhorn_loop_persistent(pf, pg, n, m, max_iter, tau, f_a, f_b, g, ws, ops, iters_out, err_out, s);
  }

  int64_t sym_sweeps = 0;
  int64_t launched = 0;  // iterations enqueued so far
  auto enqueue = [&](int iters) -> int {
    for (int i = 0; i < iters; ++i) {
      if (symmetric) {
        // alternate the operand roles so that the tensor-core sweep reads the bias rows
        // of the current f from one side's buffer while it writes the next f's rows
        // into the other side's buffer (x and y are the same cloud)
        int r = lse_sweep(pf, precision, s, &ops, (sym_sweeps & 1) == 0, &ws, true);
        if (r) return r;
        ++sym_sweeps;
        continue;
      }
      pf.seq = pg.seq = (int32_t)(launched + i);
      int r = lse_sweep(pf, precision, s, &ops, true, &ws, true);
      if (r) return r;
      r = lse_sweep(pg, precision, s, &ops, false, &ws, true);
      if (r) return r;
    }
    return PROGOT_OK;
  };
  const int64_t need = (int64_t)max_iter + 1;  // f-sweeps that guarantee a stop
  const int per_iter = symmetric ? 1 : 2;      // sweep launches per iteration
  int chunk = 2;
  int cur = 0;
  std::vector<ProfRec> chunk_recs;  // events around each enqueued chunk (profiling on)
  auto issue = [&](int slot, int iters) -> int {
    ProfRec pr;
    if (t_prof.on) {
      pr.a = t_prof.get();
      pr.b = t_prof.get();
      pr.seq = launched * per_iter;
      pr.nl = (int64_t)iters * per_iter;
      pr.kind = kProfLse;
      pr.pairs = (double)pr.nl * (double)n * (double)m;
      CK(cudaEventRecord(pr.a, s));
    }
    int r = enqueue(iters);
    if (r) return r;
    if (t_prof.on) {
      CK(cudaEventRecord(pr.b, s));
      chunk_recs.push_back(pr);
    }
    launched += iters;
    // after iteration launched - 1 the state is in state[launched & 1] (lagged) or state[0]
    const SolverState* st_dev = ws.state + (lag ? (launched & 1) : 0);
    CK(cudaMemcpyAsync(&t_host.hs[slot], st_dev, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(t_host.ev[slot], s));
    return PROGOT_OK;
  };
  rc = issue(cur, (int)std::min<int64_t>(chunk, need));
  if (rc) return rc;
  SolverState fin;
  // Chunk sizing: double until a completed chunk's state is known, then aim at the
  // iteration count predicted from the observed linear convergence rate of the error,
  // so that few launches after the stop return at entry.
  bool have_prev = false;
  SolverState prev_state;
  int next_chunk = chunk * 2;
  for (;;) {
    bool pending = false;
    if (launched < need) {
      rc = issue(cur ^ 1, (int)std::min<int64_t>(std::min(next_chunk, 64), need - launched));
      if (rc) return rc;
      pending = true;
    }
    CK(cudaEventSynchronize(t_host.ev[cur]));
    const SolverState now = t_host.hs[cur];
    if (now.done) {
      fin = now;
      if (pending) CK(cudaEventSynchronize(t_host.ev[cur ^ 1]));
      break;
    }
    if (!pending) return fail(PROGOT_ERR_CUDA, "Sinkhorn loop did not stop after max_iter + 1 sweeps");
    // iterations already queued beyond the state just read
    const int64_t queued = launched - (int64_t)now.it - 1;
    int64_t want = 2 * (int64_t)next_chunk;
    if (have_prev && now.it > prev_state.it && now.err > 0.0 && prev_state.err > now.err && tau > 0.0) {
      const double rate = std::pow(now.err / prev_state.err, 1.0 / (double)(now.it - prev_state.it));
      const double left = std::log(tau / now.err) / std::log(rate);  // iterations still needed
      want = (int64_t)std::ceil(left * 1.1) + 1 - queued;
    }
    next_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(want, 64));
    prev_state = now;
    have_prev = true;
    cur ^= 1;
  }
  if (t_prof.on) {
    // sweeps f_0, g_0, ..., g_{it-1}, f_it did work (f_0 .. f_it when symmetric); later
    // launches returned at entry. A chunk is timed only when all its launches worked.
    const int64_t working = (int64_t)per_iter * (int64_t)fin.it + 1;
    for (ProfRec& rr : chunk_recs) {
      rr.counted = rr.seq + rr.nl <= working;
      t_prof.recs.push_back(rr);
    }
    t_prof.worked[kProfLse] += working;
  }
  if (fin.fcur == 1) CK(cudaMemcpyAsync(f_a, f_b, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  if (symmetric && g != nullptr) CK(cudaMemcpyAsync(g, f_a, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  if (iters_out) *iters_out = fin.it;
  if (err_out) *err_out = fin.err;
  if (ops.on) {
    int32_t fault = 0;
    CK(cudaMemcpyAsync(&fault, ws.fault, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (fault) return fail(PROGOT_ERR_TIMEOUT, "a tensor-core sweep hit its bounded wait (2 s) and aborted");
  }
  switch (fin.status) {
    case kConverged:
      return PROGOT_OK;
    case kNumeric:
      return fail(PROGOT_ERR_NUMERIC, "non-finite marginal error after %d iterations", fin.it);
    case kStalled:
      return fail(PROGOT_ERR_NOT_CONVERGED, "marginal error %.3e stalled above tau %.3e after %d iterations", fin.err,
                  tau, fin.it);
    default:
      return fail(PROGOT_ERR_NOT_CONVERGED, "marginal error %.3e above tau %.3e after %d iterations", fin.err, tau,
                  fin.it);
  }
}

// One barycentric displacement X <- X + alpha (T(X) - X) (Alg. 2 / Alg. 3), in place on X.
// The log-sum-exp pass runs on the tensor cores when `ops` describes X, Y and the y-side
// bias rows of g at this eps; the map sweep itself normalises by its own row sums, so
// L only has to be close to the row's log-sum-exp.
static int map_step(float* X, int64_t n, const float* y, int64_t m, int32_t d, const float* g, const float* yn,
                    double eps, double alpha, int32_t precision, const Workspace& ws, cudaStream_t s,
                    const TcOps* ops = nullptr, const Cost& cost = Cost()) {
  const bool tc = !cost.pnorm() && ops != nullptr && ops->on;
  SweepParams pl = make_sweep(X, n, y, m, d, nullptr, yn, eps, ws, tc ? 1 : 2);
  pl.potB = g;
  pl.out = ws.L;
  pl.mode = kModeLse;
  apply_cost(pl, cost, eps);
  // the persistent loop that produced g may already have left L in ws.L
  int rc = (tc && ops->lse_ready) ? PROGOT_OK
           : tc                   ? lse_sweep(pl, precision, s, ops, true, &ws)
                                  : lse_sweep(pl, PROGOT_FP32, s);
  if (rc) return rc;
  if (tc && ops->nkb == 1 && g_map_tc.load()) {
    // d <= 64: S and P Y both on the tensor cores (P Y reuses the centred, scaled y operand)
    int G = 0, maxseg = 0;
    tc_plan(n, m, 128, num_sms(), &G, &maxseg);
    ProfRec r;
    const bool rec = prof_begin(r, s, kProfMap);
    CK(launch_map_sweep_tc(X, X, ws.L, n, m, d, (float)alpha, &ops->xh_a, &ops->xl_a, &ops->yh_a, &ops->yl_a,
                           &ops->yb128, (float)std::sqrt(eps / (2.0 * kLog2e)), ops->mu, ws.Opart, ws.Rpart,
                           ws.mcnt, G, maxseg, ops->split3, ws.fault, s));
    if (rec) prof_end(r, s, kProfMap, (double)n * (double)m);
    if (t_prof.on) t_prof.worked[kProfMap] += 1;
    return PROGOT_OK;
  }
  if (tc && ops->nkb > 1 && map_tc_onepass_supported(ops->nkb) && g_map_tc.load()) {
    // 64 < d <= 256: one launch, S once per tile, all output coordinates in TMEM
    int G = 0, maxseg = 0;
    tc_plan(n, m, map_tc_onepass_tile_cols(), num_sms(), &G, &maxseg);
    ProfRec r;
    const bool rec = prof_begin(r, s, kProfMap);
    CK(launch_map_sweep_tc_onepass(X, X, ws.L, n, m, d, ops->nkb, (float)alpha, &ops->xl_a,
                                   &ops->yh_m32, &ops->yl_m32, &ops->yb_m32, (float)std::sqrt(eps / (2.0 * kLog2e)),
                                   ops->mu, ws.xh, ws.Opart, ws.Rpart, ws.mcnt, G, maxseg, ops->split3, ws.fault, s));
    if (rec) prof_end(r, s, kProfMap, (double)n * (double)m);
    if (t_prof.on) t_prof.worked[kProfMap] += 1;
    return PROGOT_OK;
  }
  if (tc) {
    // the float32 map sweep below forms t_ij from the uncentred X and Y: move L there
    CK(launch_lse_uncenter(ws.L, X, n, d, ops->mu, (float)(kLog2e / eps), s));
  }
  MapParams mp;
  memset(&mp, 0, sizeof(mp));
  mp.A = X;
  mp.B = y;
  mp.Bn = yn;
  mp.potB = g;
  mp.L = ws.L;
  mp.out = X;
  mp.Opart = ws.Opart;
  mp.Rpart = ws.Rpart;
  mp.cnt = ws.mcnt;
  mp.nA = n;
  mp.nB = m;
  mp.d = d;
  mp.dchunks = (int)cdiv(d, map_dchunk());
  mp.splits = plan_splits(n, m, 1, mp.dchunks);
  const int64_t ct = cdiv(m, fp32_tile_cols());
  mp.tiles_per_split = (int)cdiv(ct, mp.splits);
  mp.splits = (int)cdiv(ct, mp.tiles_per_split);
  mp.scale = (float)(2.0 * kLog2e / eps);
  mp.bscale = (float)(kLog2e / eps);
  mp.alpha = (float)alpha;
  if (cost.pnorm()) {
    mp.cost = cost.kind;
    mp.cost_p = cost.p;
    mp.scale = (float)(-kLog2e / (eps * (double)cost.p));
  }
  ProfRec r;
  const bool rec = prof_begin(r, s, kProfMap);
  if (cost.pnorm())
    CK(launch_map_sweep_pnorm(mp, s));
  else
    CK(launch_map_sweep_fp32(mp, s));
  if (rec) prof_end(r, s, kProfMap, (double)n * (double)m);
  if (t_prof.on) t_prof.worked[kProfMap] += 1;
  return PROGOT_OK;
}

static int zero_counters(const Workspace& ws, int64_t rbmax, cudaStream_t s) {
  CK(cudaMemsetAsync(ws.cnt, 0, sizeof(unsigned) * (rbmax + 2), s));
  CK(cudaMemsetAsync(ws.mcnt, 0, sizeof(unsigned) * (rbmax + 2), s));
  CK(cudaMemsetAsync(ws.fault, 0, sizeof(int32_t), s));  // raised by a tensor-core kernel's expired wait
  return PROGOT_OK;
}

// PROGOT_ERR_TIMEOUT when a tensor-core kernel of this call raised the fault flag
// (synchronises the stream).
static int check_fault(const Workspace& ws, cudaStream_t s) {
  int32_t fault = 0;
  CK(cudaMemcpyAsync(&fault, ws.fault, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (fault) return fail(PROGOT_ERR_TIMEOUT, "a tensor-core kernel hit its bounded wait (2 s) and aborted");
  return PROGOT_OK;
}

// Coupling metrics (Sec. 5.2) of P = exp((f (+) g - C)/eps): a row sweep and a column
// sweep in kModeMetrics, each followed by a fixed-order float64 reduction of its
// per-row-block sums into ws.metout. ws.xn, ws.yn must hold |x|^2 and |y|^2 and the
// arrival counters must be zero.
static int metrics_core(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                        int32_t d, const float* f, const float* g, double eps, const Workspace& ws, cudaStream_t s,
                        progot_coupling_metrics* out, const Cost& cost = Cost(), const float* x_cost = nullptr) {
  int rc = t_host.init();
  if (rc) return rc;
  SweepParams pr = make_sweep(x, n, y, m, d, ws.xn, ws.yn, eps, ws);
  pr.wA = a;
  pr.potB = g;
  pr.potA_old = f;
  pr.mode = kModeMetrics;
  apply_cost(pr, cost, eps);
  if (x_cost != nullptr) {
    // integrate the cost from x_cost (its squared norms in ws.L) against P on x
    if (!cost.pnorm()) CK(launch_row_sqnorm(x_cost, n, d, ws.L, s));
    pr.Ac = x_cost;
    pr.Acn = cost.pnorm() ? nullptr : ws.L;
    pr.cpart = ws.cpart;
  }
  CK(launch_lse_sweep_fp32(pr, s));
  CK(launch_sum_parts(ws.metpart, (int)cdiv(n, fp32_tile_rows()), kMetricSums, ws.metout, s));
  SweepParams pc = make_sweep(y, m, x, n, d, ws.yn, ws.xn, eps, ws);
  pc.wA = b;
  pc.potB = f;
  pc.potA_old = g;
  pc.mode = kModeMetrics;
  apply_cost(pc, cost, eps);
  CK(launch_lse_sweep_fp32(pc, s));
  CK(launch_sum_parts(ws.metpart, (int)cdiv(m, fp32_tile_rows()), kMetricSums, ws.metout + kMetricSums, s));
  CK(cudaMemcpyAsync(t_host.hd, ws.metout, sizeof(double) * 2 * kMetricSums, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double* R = t_host.hd;                // row sweep: pot = f, w = a
  const double* Cs = t_host.hd + kMetricSums;  // column sweep: pot = g, w = b
  out->mass = R[kSumMass];
  out->err_row = R[kSumErr];
  out->err_col = Cs[kSumErr];
  out->entropy = R[kSumMass] - R[kSumPlogP];
  out->transport_cost = x_cost != nullptr ? R[kSumPC] : R[kSumPotR] + Cs[kSumPotR] - eps * R[kSumPlogP];
  out->dual = R[kSumPotW] + Cs[kSumPotW] - eps * R[kSumMass];
  if (!std::isfinite(out->transport_cost) || !std::isfinite(out->entropy) || !std::isfinite(out->dual))
    return fail(PROGOT_ERR_NUMERIC, "non-finite coupling metric");
  return PROGOT_OK;
}

// Mean cost of (x, y) in closed form from float64 first moments, computed on the device;
// the y moments must already sit at ws.rout + (d + 1) when y_ready.
static int mean_cost_dev(const float* x, int64_t n, const float* y, int64_t m, int32_t d, const Workspace& ws,
                         bool y_ready, cudaStream_t s, double* out, const Cost& cost = Cost()) {
  int rc = t_host.init();
  if (rc) return rc;
  if (cost.pnorm()) {
    // no closed form: sum h over all n m pairs on the CUDA cores
    double* dst = ws.metout + 2 * kMetricSums;
    CK(launch_pairwise_cost_sum(x, n, y, m, d, cost.kind, cost.p, ws.rpart, dst, s));
    CK(cudaMemcpyAsync(t_host.hd, dst, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = t_host.hd[0] / ((double)cost.p * (double)n * (double)m);
    return PROGOT_OK;
  }
  CK(launch_moments(x, n, d, ws.rpart, reduce_parts(), ws.rout, s));
  if (!y_ready) CK(launch_moments(y, m, d, ws.rpart, reduce_parts(), ws.rout + (d + 1), s));
  double* dst = ws.metout + 2 * kMetricSums;
  CK(launch_mean_cost_closed(ws.rout, ws.rout + (d + 1), n, m, d, dst, s));
  CK(cudaMemcpyAsync(t_host.hd, dst, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = t_host.hd[0];
  return PROGOT_OK;
}

// Alg. 2 with eps_k from `eps` (host, K) or, when eps is NULL, from the theta rule
// eps_k = theta mean cost(X^(k), Y) / 20 on the cloud each solve transports.
static int solve_impl(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                      int32_t K, const double* alpha, const double* eps, double theta, const double* tau,
                      int32_t max_iter, int32_t precision, float* x_out, float* g_all, float* f_last, float* x_last,
                      int32_t* iters, double* errs, double* eps_out, void* workspace, size_t ws_bytes,
                      cudaStream_t s, const Cost& cost = Cost()) {
  Workspace ws;
  int rc = carve(n, m, d, workspace, ws_bytes, &ws, precision);
  if (rc) return rc;
  rc = zero_counters(ws, ws_dims(n, m, d).rbmax, s);
  if (rc) return rc;
  if (x_out != x) CK(cudaMemcpyAsync(x_out, x, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, s));
  CK(launch_row_sqnorm(y, m, d, ws.yn, s));
  CK(cudaMemsetAsync(ws.f0, 0, sizeof(float) * n, s));
  if (eps == nullptr && !cost.pnorm()) CK(launch_moments(y, m, d, ws.rpart, reduce_parts(), ws.rout + (d + 1), s));
  int worst = PROGOT_OK;
  std::string worst_msg;
  for (int k = 0; k < K; ++k) {
    float* gk = g_all + (int64_t)k * m;
    if (k == 0) {
      CK(cudaMemsetAsync(gk, 0, sizeof(float) * m, s));
    } else {
      // warm start of Alg. 2: (1 - alpha_k) f, (1 - alpha_k) g^(k-1)
      const float c = (float)(1.0 - alpha[k]);
      CK(cudaMemcpyAsync(gk, gk - m, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
      CK(launch_scale(gk, m, c, s));
      CK(launch_scale(ws.f0, n, c, s));
    }
    if (x_last != nullptr && k == K - 1)
      CK(cudaMemcpyAsync(x_last, x_out, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, s));
    double eps_k = 0.0;
    if (eps != nullptr) {
      eps_k = eps[k];
    } else {
      double cbar = 0.0;
      rc = mean_cost_dev(x_out, n, y, m, d, ws, true, s, &cbar, cost);
      if (rc) return rc;
      eps_k = theta * cbar / 20.0;
      if (!(eps_k > 0.0) || !std::isfinite(eps_k))
        return fail(PROGOT_ERR_NUMERIC, "step %d: theta rule gave eps = %g (mean cost %g)", k + 1, eps_k, cbar);
    }
    if (eps_out) eps_out[k] = eps_k;
    CK(launch_row_sqnorm(x_out, n, d, ws.xn, s));
    int32_t it = 0;
    double err = 0.0;
    TcOps ops;
    rc = sinkhorn_core(x_out, a, n, y, b, m, d, eps_k, tau[k], max_iter, precision, ws.f0, ws.f1, gk, ws.xn, ws.yn,
                       ws, &it, &err, s, &ops, false, cost);
    if (iters) iters[k] = it;
    if (errs) errs[k] = err;
    if (rc == PROGOT_ERR_NOT_CONVERGED) {
      if (worst == PROGOT_OK) {
        worst = rc;
        worst_msg = "step " + std::to_string(k + 1) + ": " + t_last_error;
      }
    } else if (rc) {
      return rc;
    }
    rc = map_step(x_out, n, y, m, d, gk, ws.yn, eps_k, alpha[k], precision, ws, s, &ops, cost);
    if (rc) return rc;
  }
  if (f_last) CK(cudaMemcpyAsync(f_last, ws.f0, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  rc = check_fault(ws, s);  // synchronises the stream
  if (rc) return rc;
  if (worst) {
    t_last_error = worst_msg;
    return worst;
  }
  t_last_error.clear();
  return PROGOT_OK;
}

}  // namespace progot

using namespace progot;

extern "C" {

const char* progot_last_error_string(void) { return t_last_error.c_str(); }

const char* progot_version(void) { return "0.1.0"; }

size_t progot_workspace_size(int64_t n, int64_t m, int32_t d, int32_t precision) {
  if (n <= 0 || m <= 0 || d <= 0) return 0;
  return ws_layout(ws_dims(n, m, d, precision), nullptr, nullptr);
}

int progot_set_map_tc(int32_t on) {
  g_map_tc.store(on ? 1 : 0);
  return PROGOT_OK;
}

int progot_set_loop_tc(int32_t on) {
  g_loop_tc.store(on ? 1 : 0);
  return PROGOT_OK;
}

int progot_set_wait_limit_ns(uint64_t ns) {
  g_wait_ns.store(ns == 0 ? kDefaultWaitNs : (unsigned long long)ns);
  return PROGOT_OK;
}

int progot_test_withhold_initial_betas(int32_t on) {
  g_withhold_betas.store(on ? 1 : 0);
  return PROGOT_OK;
}

int progot_set_stall_window(int32_t iters) {
  if (iters < 0) return fail(PROGOT_ERR_INVALID_ARG, "stall window must be >= 0");
  g_stall_window.store(iters);
  return PROGOT_OK;
}

int64_t progot_launch_count(int32_t reset) {
  return reset ? g_launches.exchange(0) : g_launches.load();
}

int progot_profile(int32_t enable) {
  prof_collect();
  t_prof.on = enable != 0;
  t_prof.period = enable > 1 ? enable : 1;
  t_prof.seq[0] = t_prof.seq[1] = 0;
  for (int k = 0; k < kProfKinds; ++k) {
    t_prof.ms[k] = 0.0;
    t_prof.pairs[k] = 0.0;
    t_prof.launches[k] = 0;
    t_prof.worked[k] = 0;
  }
  return PROGOT_OK;
}

int progot_profile_read(int32_t kernel, int64_t* sampled, double* total_ms, double* pairs, int64_t* worked) {
  if (kernel < 0 || kernel >= kProfKinds) return fail(PROGOT_ERR_INVALID_ARG, "unknown kernel id %d", kernel);
  prof_collect();
  if (sampled) *sampled = t_prof.launches[kernel];
  if (total_ms) *total_ms = t_prof.ms[kernel];
  if (pairs) *pairs = t_prof.pairs[kernel];
  if (worked) *worked = t_prof.worked[kernel];
  return PROGOT_OK;
}

int sinkhorn_potentials(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                        int32_t d, double eps, double tau, int32_t max_iter, int32_t precision, float* f, float* g,
                        int32_t init_zero, int32_t* iters_out, double* err_out, void* workspace, size_t ws_bytes,
                        progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, precision);
  if (rc) return rc;
  if (f == nullptr || g == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "f and g must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  if (!(tau >= 0.0)) return fail(PROGOT_ERR_INVALID_ARG, "tau must be >= 0");
  if (max_iter < 0) return fail(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws, precision);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = zero_counters(ws, ws_dims(n, m, d).rbmax, s);
  if (rc) return rc;
  if (init_zero) {
    CK(cudaMemsetAsync(f, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(g, 0, sizeof(float) * m, s));
  }
  CK(launch_row_sqnorm(x, n, d, ws.xn, s));
  CK(launch_row_sqnorm(y, m, d, ws.yn, s));
  return sinkhorn_core(x, a, n, y, b, m, d, eps, tau, max_iter, precision, f, ws.f1, g, ws.xn, ws.yn, ws, iters_out,
                       err_out, s);
}

int entropic_map_apply(const float* xq, int64_t nq, const float* y, int64_t m, int32_t d, int32_t K,
                       const float* g_all, const double* eps, const double* alpha, int32_t precision, float* out,
                       void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(xq, nq, y, m, d, precision);
  if (rc) return rc;
  if (K <= 0 || g_all == nullptr || eps == nullptr || alpha == nullptr || out == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and non-NULL g_all, eps, alpha, out are required");
  for (int k = 0; k < K; ++k) {
    if (!(eps[k] > 0.0) || !std::isfinite(eps[k])) return fail(PROGOT_ERR_INVALID_ARG, "eps[%d] must be positive", k);
    if (k < K - 1 && !(alpha[k] > 0.0 && alpha[k] <= 1.0))
      return fail(PROGOT_ERR_INVALID_ARG, "alpha[%d] must lie in (0, 1]", k);
  }
  Workspace ws;
  rc = carve(nq, m, d, workspace, ws_bytes, &ws, precision);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = zero_counters(ws, ws_dims(nq, m, d).rbmax, s);
  if (rc) return rc;
  if (out != xq) CK(cudaMemcpyAsync(out, xq, sizeof(float) * nq * d, cudaMemcpyDeviceToDevice, s));
  CK(launch_row_sqnorm(y, m, d, ws.yn, s));
  for (int k = 0; k < K; ++k) {
    const double al = (k == K - 1) ? 1.0 : alpha[k];
    const float* gk = g_all + (int64_t)k * m;
    TcOps ops;
    rc = prep_tc(out, nq, y, m, d, eps[k], precision, ws, &ops, s, nullptr, gk);
    if (rc) return rc;
    rc = map_step(out, nq, y, m, d, gk, ws.yn, eps[k], al, precision, ws, s, &ops);
    if (rc) return rc;
  }
  return precision == PROGOT_FP32 ? PROGOT_OK : check_fault(ws, s);
}

int coupling_marginals(const float* x, int64_t n, const float* y, int64_t m, int32_t d, const float* f,
                       const float* g, double eps, int32_t precision, float* row, float* col, const float* a,
                       const float* b, double* err_l1_out, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, precision);
  if (rc) return rc;
  if (f == nullptr || g == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "f and g must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  rc = t_host.init();
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const WsDims w = ws_dims(n, m, d);
  rc = zero_counters(ws, w.rbmax, s);
  if (rc) return rc;
  CK(launch_row_sqnorm(x, n, d, ws.xn, s));
  CK(launch_row_sqnorm(y, m, d, ws.yn, s));
  SweepParams pr = make_sweep(x, n, y, m, d, ws.xn, ws.yn, eps, ws);
  pr.wA = a;
  pr.potB = g;
  pr.potA_old = f;
  pr.out = row;
  pr.mode = kModeMarginal;
  rc = lse_sweep(pr, precision, s);
  if (rc) return rc;
  const int64_t rbr = cdiv(n, fp32_tile_rows());
  CK(cudaMemcpyAsync(&t_host.hd[0], ws.errpart + rbr, sizeof(double), cudaMemcpyDeviceToHost, s));
  SweepParams pc = make_sweep(y, m, x, n, d, ws.yn, ws.xn, eps, ws);
  pc.wA = b;
  pc.potB = f;
  pc.potA_old = g;
  pc.out = col;
  pc.mode = kModeMarginal;
  rc = lse_sweep(pc, precision, s);
  if (rc) return rc;
  const int64_t rbc = cdiv(m, fp32_tile_rows());
  CK(cudaMemcpyAsync(&t_host.hd[1], ws.errpart + rbc, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err_l1_out) *err_l1_out = t_host.hd[0] + t_host.hd[1];
  return PROGOT_OK;
}

int progot_solve(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                 int32_t K, const double* alpha, const double* eps, const double* tau, int32_t max_iter,
                 int32_t precision, float* x_out, float* g_all, float* f_last, float* x_last, int32_t* iters,
                 double* errs, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, precision);
  if (rc) return rc;
  if (K <= 0 || alpha == nullptr || eps == nullptr || tau == nullptr || x_out == nullptr || g_all == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and non-NULL alpha, eps, tau, x_out, g_all are required");
  if (max_iter < 0) return fail(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  for (int k = 0; k < K; ++k) {
    if (!(eps[k] > 0.0) || !std::isfinite(eps[k])) return fail(PROGOT_ERR_INVALID_ARG, "eps[%d] must be positive", k);
    if (!(alpha[k] > 0.0 && alpha[k] <= 1.0)) return fail(PROGOT_ERR_INVALID_ARG, "alpha[%d] must lie in (0, 1]", k);
    if (!(tau[k] >= 0.0)) return fail(PROGOT_ERR_INVALID_ARG, "tau[%d] must be >= 0", k);
  }
  return solve_impl(x, a, n, y, b, m, d, K, alpha, eps, 0.0, tau, max_iter, precision, x_out, g_all, f_last, x_last,
                    iters, errs, nullptr, workspace, ws_bytes, (cudaStream_t)stream);
}

int progot_solve_theta(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                       int32_t d, int32_t K, const double* alpha, double theta, const double* tau, int32_t max_iter,
                       int32_t precision, float* x_out, float* g_all, float* f_last, float* x_last, int32_t* iters,
                       double* errs, double* eps_out, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, precision);
  if (rc) return rc;
  if (K <= 0 || alpha == nullptr || tau == nullptr || x_out == nullptr || g_all == nullptr || eps_out == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and non-NULL alpha, tau, x_out, g_all, eps_out are required");
  if (!(theta > 0.0) || !std::isfinite(theta)) return fail(PROGOT_ERR_INVALID_ARG, "theta must be positive and finite");
  if (max_iter < 0) return fail(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  for (int k = 0; k < K; ++k) {
    if (!(alpha[k] > 0.0 && alpha[k] <= 1.0)) return fail(PROGOT_ERR_INVALID_ARG, "alpha[%d] must lie in (0, 1]", k);
    if (!(tau[k] >= 0.0)) return fail(PROGOT_ERR_INVALID_ARG, "tau[%d] must be >= 0", k);
  }
  return solve_impl(x, a, n, y, b, m, d, K, alpha, nullptr, theta, tau, max_iter, precision, x_out, g_all, f_last,
                    x_last, iters, errs, eps_out, workspace, ws_bytes, (cudaStream_t)stream);
}

int progot_schedule_tau(int32_t K, double tau_first, double tau_last, double* out) {
  t_last_error.clear();
  if (K <= 0 || out == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and out required");
  if (!(tau_first >= 0.0) || !(tau_last >= 0.0) || !std::isfinite(tau_first) || !std::isfinite(tau_last))
    return fail(PROGOT_ERR_INVALID_ARG, "tau_first and tau_last must be finite and >= 0");
  if (K == 1) {
    out[0] = tau_last;
    return PROGOT_OK;
  }
  for (int k = 0; k < K; ++k) out[k] = tau_first + (tau_last - tau_first) * (double)k / (double)(K - 1);
  out[K - 1] = tau_last;
  return PROGOT_OK;
}

int coupling_metrics(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                     const float* f, const float* g, const float* x_cost, double eps, progot_coupling_metrics* out,
                     void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  if (f == nullptr || g == nullptr || out == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "f, g and out must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = zero_counters(ws, ws_dims(n, m, d).rbmax, s);
  if (rc) return rc;
  CK(launch_row_sqnorm(x, n, d, ws.xn, s));
  CK(launch_row_sqnorm(y, m, d, ws.yn, s));
  return metrics_core(x, a, n, y, b, m, d, f, g, eps, ws, s, out, Cost(), x_cost);
}

int sinkhorn_divergence(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                        int32_t d, double eps, double tau, int32_t max_iter, int32_t precision, double* value,
                        double* ot_parts, int32_t* iters, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, precision);
  if (rc) return rc;
  if (value == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "value must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  if (!(tau >= 0.0)) return fail(PROGOT_ERR_INVALID_ARG, "tau must be >= 0");
  if (max_iter < 0) return fail(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  const int64_t nmax = std::max<int64_t>(n, m);
  Workspace ws;
  rc = carve(nmax, nmax, d, workspace, ws_bytes, &ws, precision);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  struct Side {
    const float* p;
    const float* w;
    int64_t k;
  };
  const Side pairs[3][2] = {{{x, a, n}, {y, b, m}}, {{x, a, n}, {x, a, n}}, {{y, b, m}, {y, b, m}}};
  double ot[3] = {0.0, 0.0, 0.0};
  int worst = PROGOT_OK;
  std::string worst_msg;
  for (int q = 0; q < 3; ++q) {
    const Side& A = pairs[q][0];
    const Side& B = pairs[q][1];
    rc = zero_counters(ws, ws_dims(nmax, nmax, d).rbmax, s);
    if (rc) return rc;
    CK(launch_row_sqnorm(A.p, A.k, d, ws.xn, s));
    CK(launch_row_sqnorm(B.p, B.k, d, ws.yn, s));
    CK(cudaMemsetAsync(ws.f0, 0, sizeof(float) * A.k, s));
    CK(cudaMemsetAsync(ws.gaux, 0, sizeof(float) * B.k, s));
    int32_t it = 0;
    // the self terms OT(X, X), OT(Y, Y) use the symmetric fixed point, which reaches
    // the same maximiser of eq. (5) in far fewer iterations than alternating updates
    rc = sinkhorn_core(A.p, A.w, A.k, B.p, B.w, B.k, d, eps, tau, max_iter, precision, ws.f0, ws.f1, ws.gaux, ws.xn,
                       ws.yn, ws, &it, nullptr, s, nullptr, q != 0);
    if (iters) iters[q] = it;
    if (rc == PROGOT_ERR_NOT_CONVERGED) {
      if (worst == PROGOT_OK) {
        worst = rc;
        worst_msg = std::string(q == 0 ? "OT(X, Y)" : (q == 1 ? "OT(X, X)" : "OT(Y, Y)")) + ": " + t_last_error;
      }
    } else if (rc) {
      return rc;
    }
    progot_coupling_metrics met;
    rc = metrics_core(A.p, A.w, A.k, B.p, B.w, B.k, d, ws.f0, ws.gaux, eps, ws, s, &met);
    if (rc) return rc;
    ot[q] = met.dual;
  }
  *value = ot[0] - 0.5 * (ot[1] + ot[2]);
  if (ot_parts)
    for (int q = 0; q < 3; ++q) ot_parts[q] = ot[q];
  if (worst) {
    t_last_error = worst_msg;
    return worst;
  }
  t_last_error.clear();
  return PROGOT_OK;
}

int coupling_diagonal(const float* x, const float* y, int64_t n, int32_t d, const float* f, const float* g, double eps,
                      float* log_diag, double* trace, double* kl, void* workspace, size_t ws_bytes,
                      progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, n, d, PROGOT_FP32);
  if (rc) return rc;
  if (f == nullptr || g == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "f and g must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  Workspace ws;
  rc = carve(n, n, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  rc = t_host.init();
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_diag(x, y, f, g, n, d, eps, log_diag, ws.rpart, reduce_parts(), ws.rout, s));
  CK(cudaMemcpyAsync(t_host.hd, ws.rout, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (trace) *trace = t_host.hd[0];
  if (kl) *kl = -std::log((double)n) - t_host.hd[1] / (double)n;
  return PROGOT_OK;
}

int sinkhorn_potentials_pnorm(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                              int32_t d, double p, double eps, double tau, int32_t max_iter, float* f, float* g,
                              int32_t init_zero, int32_t* iters_out, double* err_out, void* workspace,
                              size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  Cost cost;
  rc = pnorm_cost(p, &cost);
  if (rc) return rc;
  if (f == nullptr || g == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "f and g must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  if (!(tau >= 0.0)) return fail(PROGOT_ERR_INVALID_ARG, "tau must be >= 0");
  if (max_iter < 0) return fail(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = zero_counters(ws, ws_dims(n, m, d).rbmax, s);
  if (rc) return rc;
  if (init_zero) {
    CK(cudaMemsetAsync(f, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(g, 0, sizeof(float) * m, s));
  }
  return sinkhorn_core(x, a, n, y, b, m, d, eps, tau, max_iter, PROGOT_FP32, f, ws.f1, g, ws.xn, ws.yn, ws, iters_out,
                       err_out, s, nullptr, false, cost);
}

int progot_solve_pnorm(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                       double p, int32_t K, const double* alpha, const double* eps, double theta, const double* tau,
                       int32_t max_iter, float* x_out, float* g_all, float* f_last, float* x_last, int32_t* iters,
                       double* errs, double* eps_out, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  Cost cost;
  rc = pnorm_cost(p, &cost);
  if (rc) return rc;
  if (K <= 0 || alpha == nullptr || tau == nullptr || x_out == nullptr || g_all == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and non-NULL alpha, tau, x_out, g_all are required");
  if (eps == nullptr && (!(theta > 0.0) || !std::isfinite(theta)))
    return fail(PROGOT_ERR_INVALID_ARG, "without an eps schedule theta must be positive and finite");
  if (max_iter < 0) return fail(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  for (int k = 0; k < K; ++k) {
    if (eps != nullptr && (!(eps[k] > 0.0) || !std::isfinite(eps[k])))
      return fail(PROGOT_ERR_INVALID_ARG, "eps[%d] must be positive", k);
    if (!(alpha[k] > 0.0 && alpha[k] <= 1.0)) return fail(PROGOT_ERR_INVALID_ARG, "alpha[%d] must lie in (0, 1]", k);
    if (!(tau[k] >= 0.0)) return fail(PROGOT_ERR_INVALID_ARG, "tau[%d] must be >= 0", k);
  }
  return solve_impl(x, a, n, y, b, m, d, K, alpha, eps, theta, tau, max_iter, PROGOT_FP32, x_out, g_all, f_last,
                    x_last, iters, errs, eps_out, workspace, ws_bytes, (cudaStream_t)stream, cost);
}

int entropic_map_apply_pnorm(const float* xq, int64_t nq, const float* y, int64_t m, int32_t d, double p, int32_t K,
                             const float* g_all, const double* eps, const double* alpha, float* out, void* workspace,
                             size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(xq, nq, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  Cost cost;
  rc = pnorm_cost(p, &cost);
  if (rc) return rc;
  if (K <= 0 || g_all == nullptr || eps == nullptr || alpha == nullptr || out == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and non-NULL g_all, eps, alpha, out are required");
  for (int k = 0; k < K; ++k) {
    if (!(eps[k] > 0.0) || !std::isfinite(eps[k])) return fail(PROGOT_ERR_INVALID_ARG, "eps[%d] must be positive", k);
    if (k < K - 1 && !(alpha[k] > 0.0 && alpha[k] <= 1.0))
      return fail(PROGOT_ERR_INVALID_ARG, "alpha[%d] must lie in (0, 1]", k);
  }
  Workspace ws;
  rc = carve(nq, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = zero_counters(ws, ws_dims(nq, m, d).rbmax, s);
  if (rc) return rc;
  if (out != xq) CK(cudaMemcpyAsync(out, xq, sizeof(float) * nq * d, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < K; ++k) {
    const double al = (k == K - 1) ? 1.0 : alpha[k];
    rc = map_step(out, nq, y, m, d, g_all + (int64_t)k * m, ws.yn, eps[k], al, PROGOT_FP32, ws, s, nullptr, cost);
    if (rc) return rc;
  }
  return PROGOT_OK;
}

int coupling_metrics_pnorm(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                           int32_t d, double p, const float* f, const float* g, const float* x_cost, double eps,
                           progot_coupling_metrics* out, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  Cost cost;
  rc = pnorm_cost(p, &cost);
  if (rc) return rc;
  if (f == nullptr || g == nullptr || out == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "f, g and out must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = zero_counters(ws, ws_dims(n, m, d).rbmax, s);
  if (rc) return rc;
  return metrics_core(x, a, n, y, b, m, d, f, g, eps, ws, s, out, cost, x_cost);
}

int progot_mean_cost_pnorm(const float* x, int64_t n, const float* y, int64_t m, int32_t d, double p, double* out,
                           void* workspace, size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  Cost cost;
  rc = pnorm_cost(p, &cost);
  if (rc) return rc;
  if (out == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "out must not be NULL");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  return mean_cost_dev(x, n, y, m, d, ws, false, (cudaStream_t)stream, out, cost);
}

int progot_schedule_alpha(int32_t K, int32_t kind, double* out) {
  t_last_error.clear();
  if (K <= 0 || out == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "K > 0 and out required");
  if (kind == PROGOT_ALPHA_DECELERATED) {
    for (int k = 0; k < K; ++k) out[k] = 1.0 / std::exp(1.0);
  } else if (kind == PROGOT_ALPHA_CONSTANT || kind == PROGOT_ALPHA_ACCELERATED) {
    auto t = [&](int k) {
      const double r = (double)k / (double)K;
      return kind == PROGOT_ALPHA_CONSTANT ? r : r * r;
    };
    for (int k = 1; k <= K; ++k) out[k - 1] = (t(k) - t(k - 1)) / (1.0 - t(k - 1));
  } else {
    return fail(PROGOT_ERR_INVALID_ARG, "unknown alpha schedule %d", kind);
  }
  out[K - 1] = 1.0;
  return PROGOT_OK;
}

int progot_mean_cost(const float* x, int64_t n, const float* y, int64_t m, int32_t d, double* out, void* workspace,
                     size_t ws_bytes, progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, PROGOT_FP32);
  if (rc) return rc;
  if (out == nullptr) return fail(PROGOT_ERR_INVALID_ARG, "out must not be NULL");
  Workspace ws;
  rc = carve(n, m, d, workspace, ws_bytes, &ws);
  if (rc) return rc;
  return mean_cost_dev(x, n, y, m, d, ws, false, (cudaStream_t)stream, out);
}

int progot_schedule_eps(const float* x, int64_t n, const float* y, const float* b, int64_t m, const float* y_test,
                        int64_t mt, int32_t d, int32_t K, const double* alpha, const double* s_grid, int32_t P,
                        double beta0, double tau, int32_t max_iter, int32_t precision, double* eps_out,
                        double* errors_out, int32_t* p_star_out, void* workspace, size_t ws_bytes,
                        progot_stream_t stream) {
  t_last_error.clear();
  int rc = check_common(x, n, y, m, d, precision);
  if (rc) return rc;
  if (y_test == nullptr || mt <= 0 || K <= 0 || alpha == nullptr || s_grid == nullptr || P <= 0 ||
      eps_out == nullptr)
    return fail(PROGOT_ERR_INVALID_ARG, "y_test, mt > 0, K > 0, alpha, s_grid, P > 0 and eps_out are required");
  const int64_t nmax = std::max<int64_t>(std::max<int64_t>(n, m), mt);
  Workspace ws;
  rc = carve(nmax, nmax, d, workspace, ws_bytes, &ws, precision);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  double mc_xy = 0.0, mc_yy = 0.0;
  rc = progot_mean_cost(x, n, y, m, d, &mc_xy, workspace, ws_bytes, stream);
  if (rc) return rc;
  rc = progot_mean_cost(y, m, y, m, d, &mc_yy, workspace, ws_bytes, stream);
  if (rc) return rc;
  const double eps0 = mc_xy / 20.0, sigma = mc_yy / 20.0;
  rc = zero_counters(ws, ws_dims(nmax, nmax, d).rbmax, s);
  if (rc) return rc;
  CK(launch_row_sqnorm(y, m, d, ws.yn, s));
  std::vector<double> errors(P);
  for (int p = 0; p < P; ++p) {
    const double eps = s_grid[p] * sigma;
    CK(cudaMemsetAsync(ws.f0, 0, sizeof(float) * m, s));
    CK(cudaMemsetAsync(ws.gaux, 0, sizeof(float) * m, s));
    rc = sinkhorn_core(y, b, m, y, b, m, d, eps, tau, max_iter, precision, ws.f0, ws.f1, ws.gaux, ws.yn, ws.yn, ws,
                       nullptr, nullptr, s);
    if (rc && rc != PROGOT_ERR_NOT_CONVERGED) return rc;
    CK(cudaMemcpyAsync(ws.T, y_test, sizeof(float) * mt * d, cudaMemcpyDeviceToDevice, s));
    // tensor-core operands of the held-out points against Y, with the y-side bias of g
    TcOps ops;
    rc = prep_tc(ws.T, mt, y, m, d, eps, precision, ws, &ops, s, nullptr, ws.gaux);
    if (rc) return rc;
    rc = map_step(ws.T, mt, y, m, d, ws.gaux, ws.yn, eps, 1.0, precision, ws, s, &ops);
    if (rc) return rc;
    CK(launch_sq_error(y_test, ws.T, mt, d, ws.rpart, reduce_parts(), ws.rout, s));
    rc = t_host.init();
    if (rc) return rc;
    CK(cudaMemcpyAsync(t_host.hd, ws.rout, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    errors[p] = t_host.hd[0];
  }
  int pstar = 0;
  for (int p = 1; p < P; ++p)
    if (errors[p] < errors[pstar]) pstar = p;
  const double epsK = s_grid[pstar] * sigma;
  double prod = 1.0;
  for (int k = 0; k < K; ++k) {
    prod *= (1.0 - alpha[k]);
    const double t = 1.0 - prod;
    eps_out[k] = (1.0 - t) * beta0 * eps0 + t * epsK;
  }
  if (errors_out)
    for (int p = 0; p < P; ++p) errors_out[p] = errors[p];
  if (p_star_out) *p_star_out = pstar;
  t_last_error.clear();
  return PROGOT_OK;
}

}  // extern "C"
