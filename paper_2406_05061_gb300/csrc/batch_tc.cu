// Many independent ProgOT problems (Alg. 2, each with its own Sinkhorn loops, Alg. 1)
// in one persistent tensor-core launch.
//
// Work list. Every problem is a chain of phases, each phase a set of tasks on 128-row
// blocks:
//   MOM    (x and y row blocks)  column sums of both clouds; the phase's finisher sets the
//                                problem's centre mu = (mean x + mean y) / 2 and copies x
//                                into the working cloud X (= x_out);
//   SPLIT  (x and y row blocks)  step k's operands: c_k (x - mu) as bf16 hi/lo (K padded
//                                to 64) and |x - mu|^2, (y - mu) and |y - mu|^2 at the
//                                first step only, the warm start (1 - alpha_k) f,
//                                g^(k) = (1 - alpha_k) g^(k-1), and the bias rows of g;
//   FUP    (x row block, column segment)   the f-update of Alg. 1, its row-marginal
//                                error measured at the current f; the finisher applies the
//                                stop test (err <= tau, max_iter, a stall, a non-finite
//                                error);
//   GUP    (y row block, column segment)   the g-update;
//   MAP    (x row block)         the barycentric displacement x <- x + alpha_k (T(x) - x)
//                                with T_i = sum_j 2^{t_ij - L_i} y_j / sum_j 2^{t_ij - L_i}
//                                and L_i from the last f-update (whose g is the final g).
// The last task of a phase (an arrival counter) runs the phase's finish and appends the
// next phase's tasks to a device-wide queue of eight priority levels (rings of task slots
// with per-slot sequence words, reserved with atomics), at the level of the problem's
// estimated remaining chain, so that the problems that need the most iterations are not
// held up behind the others. Persistent CTAs, one per SM, pop the most urgent task. A task never waits for another CTA: what it reads was written by an earlier
// phase of its own problem, published through the queue (release on the slot's sequence
// word, acquire by the popping CTA, proxy fences around the TMA reads). The problems'
// phases interleave, so while one problem waits for its phase's last task the other
// problems' tasks keep the SMs busy; the column segmentation of the sweep tasks
// (segments per row block, set per problem from a tuned target of tasks per phase) lets
// the last large problems spread over the GPU.
//
// Arithmetic per task follows the single-problem tensor-core path: t_ij = c (x~_i . y~_j)
// + beta_j in log2 units from three bf16 products of centred hi/lo operands (here the
// scale c = 2 log2(e) / eps_k sits in the x operand alone, so the y operand is split once
// per problem) plus one K = 16 product of ones with the three-way bf16 split of beta_j,
// float32 online log-sum-exp per row, a deterministic combine of the column segments in
// segment order, the potential f_i = eps log w_i + |x~_i|^2 - eps ln2 L_i in float32 FMAs
// on a hi/lo split of eps ln2, and P Y~ on the tensor cores for the map. A problem's
// results depend only on its own sizes and its segmentation, not on the rest of the
// batch or on which CTA ran which task. The centre is fixed per problem (the midpoint
// of the two clouds' means at the start), where the single-problem path re-centres at
// every step.
//
// CTA = 12 warps: 0 task fetch and TMA producer, 1 TMEM owner and MMA issuer, 2-9 two
// LSE warpgroups alternating tiles (and the CUDA-core tasks MOM and SPLIT), 10-11 task
// epilogues (segment combine, potentials, bias rows, arrivals, phase finish, enqueue).
// The roles read the same task sequence from a small ring in shared memory. Every wait
// is bounded: an expired wait raises the CTA's abort flag and the grid's fault word, the
// queue's consumers stop, every role winds down (copies and products drained, TMEM
// freed) and the host reports PROGOT_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/progot.h"
#include "progot_internal.h"
#include "tc_common.cuh"

namespace progot {
namespace tc {
namespace bat {

constexpr int NTHREADS = 384;
constexpr int EPI_TID0 = 320;
constexpr int NST = 3;          // operand stages
constexpr int NTQ = 2;          // task ring: the producer holds at most one task beyond the ones in work
constexpr int TMEM_COLS = 512;  // S buffers at [0, 128) and [128, 256), map accumulator O at [256, 320)
constexpr uint32_t O_COL = 256;
constexpr int SW_BN = 128;      // sweep tile columns
constexpr int MP_BN = 64;       // map tile columns
constexpr int kMaxSegs = 8;
constexpr int kLevels = 8;      // priority levels of the task queue (0 = most urgent)
// Limit of the idle waits (a CTA waiting for the next task to exist): a CTA can sit idle
// for as long as the last phases of the slowest problem take, so this limit is longer
// than the pipeline waits' (which a task's own work bounds).
constexpr unsigned long long kIdleNs = 30000000000ull;

constexpr uint32_t A_HALF = 128 * 64 * 2;         // 16 KB: 128 rows x 64 bf16
constexpr uint32_t OFF_ONES = 4 * A_HALF;         // after two A buffers (hi, lo each)
constexpr uint32_t OFF_ST = OFF_ONES + 4096;      // stages: B hi, B lo, bias rows
constexpr uint32_t ST_LO = 16384, ST_BIAS = 32768, ST_BYTES = 36864;
constexpr uint32_t OFF_P = OFF_ST + NST * ST_BYTES;  // map P tile: hi, lo (128 x 64 bf16 each)
constexpr uint32_t P_LO = 16384;
constexpr uint32_t OFF_CTRL = OFF_P + 2 * P_LO;
static_assert(OFF_ST % 1024 == 0 && ST_BYTES % 1024 == 0 && OFF_P % 1024 == 0, "swizzled tiles on 1 KB");

enum TaskKind : int32_t { kExit = 0, kMom = 1, kSplit = 2, kFup = 3, kGup = 4, kMap = 5 };
// tensor maps of a problem: operands in 128-row boxes, bias rows in 128-row boxes, the
// y operand and bias rows in 64-row boxes for the map tiles
enum MapIdx : int32_t { kXh = 0, kXl, kYh, kYl, kXb, kYb, kYh64, kYl64, kYb64, kNumMaps };

// Constants of step k of one problem (host-computed from eps_k, alpha_k, tau_k).
struct StepC {
  double tau;
  float c;             // c = 2 log2(e) / eps, the scale of the x operand
  float bscale;         // log2(e) / eps
  float inv_eps_f;      // 1 / eps
  float c_hi, c_lo;     // eps ln2 = c_hi + c_lo
  float e_hi, e_lo;     // eps = e_hi + e_lo
  float w_hi[2], w_lo[2];  // eps log(1 / n), eps log(1 / m)
  float alpha;          // alpha_k
  float keep;           // 1 - alpha_k (the warm start factor; unused at k = 0)
};

// Mutable per-problem state, written only by phase finishers (one phase at a time).
struct PState {
  int32_t k, it, status, fcur, best_it, done, pad0, pad1;
  double err, best_err;
};

struct Prob {
  const float* x;
  const float* y;
  const float* a;   // weights or nullptr (uniform)
  const float* b;
  float* X;         // n x d working cloud (the caller's x_out)
  float* g_all;     // K x m
  float* f_last;    // n or nullptr
  float* f[2];      // potential buffers (state.fcur selects the current one)
  float* xn;        // |x_i - mu|^2
  float* yn;
  float* L;         // n: log2-sum-exp of the last f-update
  float* mu;        // 64: centre (zero beyond d)
  __nv_bfloat16 *xh, *xl, *yh, *yl;  // operands (rows x 64)
  __nv_bfloat16 *xb, *yb;            // bias rows (row blocks x 128 x 16)
  float2* part;     // [row block][segment][128] (max, sum) partials
  double* errpart;  // [Rx]
  double* mom;      // [Rx + Ry][64] column sums
  unsigned* cnt;    // [max(Rx, Ry)] segment arrivals per row block
  unsigned* phase;  // arrivals of the current phase
  PState* st;
  const StepC* sc;  // [K]
  int32_t* iters;   // [K] outputs
  double* errs;
  int32_t* stat;
  const CUtensorMap* maps;  // [kNumMaps]
  int64_t n, m;
  int32_t d, K, Rx, Ry, Tx, Ty, Tm, segs_f, segs_g, max_iter, stall_window, pad;
};

struct Params {
  const Prob* probs;
  int4* qslots;              // [kLevels][Q] task = (problem, kind, row block, segment or side)
  unsigned long long* qseq;  // [kLevels][Q] per-slot sequence words
  unsigned long long* qctl;  // level l: head at [64 l], tail at [64 l + 16], count of published
                             // unclaimed tasks (signed) at [64 l + 32], each on its own 128-byte line
  unsigned long long qmask;  // ring size Q - 1 (a power of two)
  unsigned* remaining;       // problems not finished
  int32_t* fault;
  unsigned long long wait_ns;
  int32_t split3;
};

struct Shared {
  uint64_t full[NST], empty[NST];
  uint64_t tmem_full[2], tmem_empty[2];
  uint64_t a_full[2], a_empty[2];
  uint64_t p_full, p_empty;    // map P tile written (4 warps) / consumed (commit)
  uint64_t o_full, o_empty;    // map accumulator complete / read out (4 warps)
  uint64_t task_full[NTQ], task_empty[NTQ];
  uint64_t seg_full[2], seg_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort_flag;
  int32_t e_last, p_last;
  int4 tq[NTQ];
  float ered[4];
  float2 ms[2][128];
  float2 seg[2][128];
  float mu_s[64];   // the centre for the map task's update (written after a barrier of the task)
  float mu_sp[64];  // the centre for the split task (its own array: written before the task's first barrier)
};
static_assert(offsetof(Shared, tq) % 16 == 0, "task slots");
constexpr size_t SMEM_TOTAL = OFF_CTRL + sizeof(Shared) + 1024;
static_assert(SMEM_TOTAL <= 227 * 1024, "shared memory");

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ bool grid_fault(const Params& P) { return *reinterpret_cast<volatile int32_t*>(P.fault) != 0; }

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int32_t* abort_flag,
                                         const Params& P, bool ignore_abort = false, bool idle = false) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  const unsigned long long lim = idle ? kIdleNs : (ignore_abort ? kWaitNs : P.wait_ns);
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15) == 0) {
      if (!ignore_abort && *abort_flag) return false;
      if (global_ns() - t0 > lim) {
        *abort_flag = 1;
        atomicExch(P.fault, 1);
        return false;
      }
    }
  }
}
__device__ __forceinline__ bool warp_wait_bar(uint64_t* bar, uint32_t parity, volatile int32_t* abort_flag,
                                              const Params& P, bool ignore_abort = false, bool idle = false) {
  const bool ok = wait_bar(bar, parity, abort_flag, P, ignore_abort, idle);
  return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ unsigned long long ld_acq_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_sub_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(0u - v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_proxy_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ void umma_rt(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The stage's K-major y tile read as an MN-major B operand (rows of 128 B along K = j, 64
// coordinates each, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(1024 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ uint64_t pack2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ float2 combine_fast(float2 p, float2 q) {
  const float M = fmaxf(p.x, q.x);
  if (M == -INFINITY) return make_float2(-INFINITY, 0.f);
  return make_float2(M, p.y * fast_exp2(p.x - M) + q.y * fast_exp2(q.x - M));
}

// beta split into three bf16 terms (hi, mid, lo) in the first three of 16 slots (-inf in
// the first slot for a non-finite beta).
__device__ __forceinline__ void write_bias16(__nv_bfloat16* row16, float beta) {
  __nv_bfloat16 h1, h2, h3;
  if (isfinite(beta)) {
    h1 = __float2bfloat16_rn(beta);
    const float r1 = beta - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r1);
    h3 = __float2bfloat16_rn(r1 - __bfloat162float(h2));
  } else {
    h1 = __float2bfloat16_rn(-INFINITY);
    h2 = __float2bfloat16_rn(0.f);
    h3 = __float2bfloat16_rn(0.f);
  }
  uint4 lo4;
  lo4.x = (uint32_t)__bfloat16_as_ushort(h1) | ((uint32_t)__bfloat16_as_ushort(h2) << 16);
  lo4.y = (uint32_t)__bfloat16_as_ushort(h3);
  lo4.z = 0u;
  lo4.w = 0u;
  uint4* dst = reinterpret_cast<uint4*>(row16);
  dst[0] = lo4;
  dst[1] = make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
    h[e] = bf2_bits(hh);
    l[e] = bf2_bits(ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Named barriers: 1 = both LSE warpgroups (256), 2 = LSE warpgroup 0 (128), 3 = epilogue warps (64).
__device__ __forceinline__ void bar_lse_all() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void bar_epi() { asm volatile("bar.sync 3, 64;" ::: "memory"); }
__device__ __forceinline__ void bar_wg0() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// Column tiles [t0, t1) of a sweep or map task.
__device__ __forceinline__ void task_tiles(const Prob& pr, int4 t, int* t0, int* t1) {
  if (t.y == kMap) {
    *t0 = 0;
    *t1 = pr.Tm;
    return;
  }
  const bool g = t.y == kGup;
  const int T = g ? pr.Tx : pr.Ty, segs = g ? pr.segs_g : pr.segs_f;
  *t0 = (int)((int64_t)t.w * T / segs);
  *t1 = (int)((int64_t)(t.w + 1) * T / segs);
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Pop the next task (one lane). Each level counts its published, unclaimed tasks; a
// consumer claims one by decrementing the count of the most urgent level that shows
// some (undoing the decrement if it lost the race), and only then reserves the level's
// next position with one atomic add, so no consumer ever holds a position without a
// task and no compare-and-swap retries pile up on one word. The slot goes back to the
// producers one ring length later. Bounded (kIdleNs) and left early when the grid has
// faulted.
__device__ bool queue_pop(const Params& P, int4* t, volatile int32_t* abort_flag) {
  const unsigned long long Q = P.qmask + 1ull;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    long long av[kLevels];
#pragma unroll
    for (int l = 0; l < kLevels; ++l) av[l] = (long long)ld_relaxed_u64(P.qctl + 64 * l + 32);
    int lv = -1;
#pragma unroll
    for (int l = kLevels - 1; l >= 0; --l)
      if (av[l] > 0) lv = l;
    if (lv >= 0) {
      unsigned long long* avail = P.qctl + 64 * lv + 32;
      if ((long long)atomicAdd(avail, ~0ull) > 0) {
        const unsigned long long pos = atomicAdd(P.qctl + 64 * lv, 1ull);
        const unsigned long long idx = (unsigned long long)lv * Q + (pos & P.qmask);
        unsigned long long* seq = P.qseq + idx;
        // a claimed position's task is published (by its enqueuer, which never waits) at
        // the latest shortly after the count announced it
        const unsigned long long tw = global_ns();
        for (uint32_t j = 0; ld_acq_u64(seq) != pos + 1ull; ++j) {
          if ((j & 15) == 15 && global_ns() - tw > P.wait_ns) {
            *abort_flag = 1;
            atomicExch(P.fault, 1);
            return false;
          }
        }
        *t = __ldcg(P.qslots + idx);
        st_rel_u64(seq, pos + Q);
        return true;
      }
      atomicAdd(avail, 1ull);  // lost the race for the last one: undo and look again
      continue;
    }
    if ((i & 7) == 7) {
      if (*abort_flag || grid_fault(P)) {
        *abort_flag = 1;
        return false;
      }
      if (global_ns() - t0 > kIdleNs) {
        *abort_flag = 1;
        atomicExch(P.fault, 1);
        return false;
      }
    }
    __nanosleep(64);
  }
}

// Append n tasks (a full warp): lane 0 reserves positions, each lane publishes its
// tasks. The ring holds every task that can be outstanding, so a slot is always free;
// the wait for it is bounded all the same.
template <class F>
__device__ bool enqueue_warp(const Params& P, int level, int n, F make, volatile int32_t* abort_flag) {
  const int lane = threadIdx.x & 31;
  const unsigned long long base = (unsigned long long)level * (P.qmask + 1ull);
  unsigned long long pos0 = 0;
  if (lane == 0) pos0 = atomicAdd(P.qctl + 64 * level + 16, (unsigned long long)n);
  pos0 = __shfl_sync(0xffffffffu, pos0, 0);
  bool ok = true;
  for (int i = lane; i < n && ok; i += 32) {
    const unsigned long long pos = pos0 + (unsigned long long)i;
    unsigned long long* seq = P.qseq + base + (pos & P.qmask);
    if (ld_acq_u64(seq) != pos) {
      const unsigned long long t0 = global_ns();
      for (uint32_t it = 1;; ++it) {
        if (ld_acq_u64(seq) == pos) break;
        if ((it & 15) == 0 && global_ns() - t0 > P.wait_ns) {
          *abort_flag = 1;
          atomicExch(P.fault, 1);
          ok = false;
          break;
        }
      }
      if (!ok) break;
    }
    P.qslots[base + (pos & P.qmask)] = make(i);
    st_rel_u64(seq, pos + 1);
  }
  ok = __all_sync(0xffffffffu, ok) != 0;
  // announce the tasks once all are published
  if (lane == 0 && ok) atomicAdd(P.qctl + 64 * level + 32, (unsigned long long)n);
  return ok;
}

// Task of ring position idx, read by a whole warp (lane 0 hands the slot back).
__device__ __forceinline__ int4 ring_get(Shared& sh, int idx, volatile int32_t* abort_flag, const Params& P) {
  const int qi = idx % NTQ;
  int4 t = make_int4(-1, kExit, 0, 0);
  if (warp_wait_bar(&sh.task_full[qi], (uint32_t)((idx / NTQ) & 1), abort_flag, P, true, true)) t = sh.tq[qi];
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&sh.task_empty[qi]);
  return t;
}

// The stop test of Alg. 1 after an f-update whose row-marginal error is err.
__device__ __forceinline__ void stop_test(PState& st, double err, double tau, int max_iter, int stall_window) {
  st.err = err;
  const int it = st.it;
  if (!isfinite(err)) {
    st.status = kNumeric;
    st.done = 1;
  } else if (err <= tau) {
    st.status = kConverged;
    st.done = 1;
  } else if (it >= max_iter) {
    st.status = kMaxIter;
    st.done = 1;
  } else {
    if (err < 0.99 * st.best_err) {
      st.best_err = err;
      st.best_it = it;
    } else if (stall_window > 0 && it - st.best_it >= stall_window) {
      st.status = kStalled;
      st.done = 1;
    }
    if (!st.done) {
      st.fcur ^= 1;
      st.it += 1;
    }
  }
}

// ------------------------------------------------------------------ CUDA-core tasks (LSE warps)
// MOM: column sums of 128 rows of x (side 0, also copied into X) or y (side 1).
__device__ void task_mom(const Prob& pr, int rb, int side, unsigned char* smem) {
  const int ltid = threadIdx.x - 64, lw = ltid >> 5, lane = threadIdx.x & 31;
  const int d = pr.d;
  const int64_t rows = side ? pr.m : pr.n;
  const float* src = side ? pr.y : pr.x;
  // all loads of the warp's 16 rows first (they are independent), then sums and copies
  float v0[16], v1[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int64_t row = (int64_t)rb * BM + lw + 8 * q;
    const bool ok = row < rows;
    v0[q] = ok && lane < d ? src[row * d + lane] : 0.f;
    v1[q] = ok && lane + 32 < d ? src[row * d + lane + 32] : 0.f;
  }
  double a0 = 0.0, a1 = 0.0;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    a0 += (double)v0[q];
    a1 += (double)v1[q];
  }
  if (side == 0) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int64_t row = (int64_t)rb * BM + lw + 8 * q;
      if (row < rows) {
        if (lane < d) pr.X[row * d + lane] = v0[q];
        if (lane + 32 < d) pr.X[row * d + lane + 32] = v1[q];
      }
    }
  }
  // the map P tile's memory holds the reduction: warpgroup 0 reaches this barrier only
  // after the previous map task's last P Y~ products (which read the P tile) completed
  bar_lse_all();
  double* red = reinterpret_cast<double*>(smem + OFF_P);
  red[lw * 64 + lane] = a0;
  red[lw * 64 + lane + 32] = a1;
  bar_lse_all();
  if (ltid < 64) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w * 64 + ltid];
    pr.mom[(int64_t)(side ? pr.Rx + rb : rb) * 64 + ltid] = s;
  }
}

// Squared norm sum_c u_c^2 of up to 32 values in float32 without rounding loss: each
// square's exact value is p + e (p = u u rounded, e = fma(u, u, -p)), and the terms are
// accumulated as an unevaluated float pair with Knuth's TwoSum (about 48 bits, more than
// the float32 norm keeps), which the float64 pipe, a small fraction of the float32 rate
// on this GPU, would otherwise have to do.
__device__ __forceinline__ void sq_sum_pair(const float* u, int nv, float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    if (c < nv) {
      const float pr = u[c] * u[c];
      const float er = fmaf(u[c], u[c], -pr);
      const float sm = hi + pr;
      const float bb = sm - hi;
      const float ts = (hi - (sm - bb)) + (pr - bb);
      hi = sm;
      lo += ts + er;
    }
  }
}

// SPLIT: step k's operands, thread = (row, half of the 64 coordinates). x side, every
// step: c_k (x - mu) as bf16 hi/lo (K padded to 64), |x - mu|^2, the warm start
// (1 - alpha_k) f. y side: (y - mu) as bf16 hi/lo and |y - mu|^2 once (k = 0; neither
// depends on eps, the scale c_k sits in the x operand), every step the warm start
// g^(k) = (1 - alpha_k) g^(k-1) and the bias rows of g. Bias rows of padding rows are -inf.
__device__ void task_split(const Prob& pr, int rb, int side, int split3, float* mu_s, double* nrm_s) {
  const int ltid = threadIdx.x - 64;
  const int r = ltid & 127, h = ltid >> 7;
  const int d = pr.d;
  const int k = __ldcg(&pr.st->k);
  const StepC& C = pr.sc[k];
  const int64_t rows = side ? pr.m : pr.n;
  const int64_t rows_pad = (int64_t)(side ? pr.Ry : pr.Rx) * BM;
  const int64_t row = (int64_t)rb * BM + r;
  const bool operands = side == 0 || k == 0;
  if (operands && ltid < 64) mu_s[ltid] = __ldcg(pr.mu + ltid);
  // after this barrier the map task before (if any) has finished its products, so the
  // P tile's memory may hold the half-row norms below
  bar_lse_all();
  float* nrm = side ? pr.yn : pr.xn;
  if (operands) {
    const float* src = side ? pr.y : pr.X;
    __nv_bfloat16* hi = side ? pr.yh : pr.xh;
    __nv_bfloat16* lo = side ? pr.yl : pr.xl;
    const float scale = side ? 1.f : C.c;
    const int c0 = 32 * h;
    const int nv = min(32, max(0, d - c0));  // coordinates of this half inside the cloud
    float u[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) u[c] = (row < rows && c < nv) ? __ldcg(src + row * d + c0 + c) : 0.f;
#pragma unroll
    for (int c = 0; c < 32; ++c) u[c] = c < nv ? u[c] - mu_s[c0 + c] : 0.f;
    float shi, slo;
    sq_sum_pair(u, nv, shi, slo);
    if (row < rows) {
      uint32_t hw[16], lw[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(u[2 * e] * scale, u[2 * e + 1] * scale);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(u[2 * e] * scale - hf.x, u[2 * e + 1] * scale - hf.y);
        hw[e] = bf2_bits(hh);
        lw[e] = bf2_bits(ll);
      }
      uint4* dh = reinterpret_cast<uint4*>(hi + row * 64 + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dh[q] = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
      if (split3) {
        uint4* dl = reinterpret_cast<uint4*>(lo + row * 64 + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) dl[q] = make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
      }
    }
    if (h == 1) nrm_s[r] = (double)shi + (double)slo;
    bar_lse_all();
    if (h == 0 && row < rows) nrm[row] = (float)(((double)shi + (double)slo) + nrm_s[r]);
  }
  if (h == 0) {
    if (row < rows) {
      if (side) {
        const float gk = k ? C.keep * __ldcg(pr.g_all + (int64_t)(k - 1) * pr.m + row) : 0.f;
        pr.g_all[(int64_t)k * pr.m + row] = gk;
        // the norm: this thread's own store above, or an earlier step's
        const float nr = __ldcg(nrm + row);
        write_bias16(pr.yb + row * 16, (gk - nr) * C.bscale);
      } else {
        float* fc = pr.f[__ldcg(&pr.st->fcur)];
        fc[row] = k ? C.keep * __ldcg(fc + row) : 0.f;
      }
    } else if (row < rows_pad) {
      write_bias16((side ? pr.yb : pr.xb) + row * 16, -INFINITY);
    }
  }
}

// ------------------------------------------------------------------ phase finish (one warp)
__device__ void phase_finish(const Params& P, const Prob& pr, int pi, int kind, volatile int32_t* abort_flag) {
  const int lane = threadIdx.x & 31;
  PState* st = pr.st;
  int next = kExit;  // kExit here: the problem is done
  if (lane == 0) *pr.phase = 0;
  if (kind == kMom) {
    for (int c = lane; c < 64; c += 32) {
      double sx = 0.0, sy = 0.0;
      for (int r = 0; r < pr.Rx; ++r) sx += __ldcg(pr.mom + (int64_t)r * 64 + c);
      for (int r = 0; r < pr.Ry; ++r) sy += __ldcg(pr.mom + (int64_t)(pr.Rx + r) * 64 + c);
      pr.mu[c] = c < pr.d ? (float)(0.5 * (sx / (double)pr.n + sy / (double)pr.m)) : 0.f;
    }
    next = kSplit;
  } else if (kind == kSplit) {
    if (lane == 0) {
      st->it = 0;
      st->status = kRunning;
      st->done = 0;
      st->best_it = 0;
      st->err = 0.0;
      st->best_err = INFINITY;
    }
    next = kFup;
  } else if (kind == kFup) {
    double err = 0.0;
    for (int r = lane; r < pr.Rx; r += 32) err += __ldcg(pr.errpart + r);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) err += __shfl_xor_sync(0xffffffffu, err, off);
    int dec = 0;
    if (lane == 0) {
      PState s;
      s.k = __ldcg(&st->k);
      s.it = __ldcg(&st->it);
      s.status = __ldcg(&st->status);
      s.fcur = __ldcg(&st->fcur);
      s.best_it = __ldcg(&st->best_it);
      s.done = 0;
      s.err = __ldcg(&st->err);
      s.best_err = __ldcg(&st->best_err);
      stop_test(s, err, pr.sc[s.k].tau, pr.max_iter, pr.stall_window);
      st->it = s.it;
      st->status = s.status;
      st->fcur = s.fcur;
      st->best_it = s.best_it;
      st->done = s.done;
      st->err = s.err;
      st->best_err = s.best_err;
      if (s.done) {
        pr.iters[s.k] = s.it;
        pr.errs[s.k] = s.err;
        pr.stat[s.k] = s.status;
      }
      dec = s.done ? (s.status == kNumeric ? 2 : 1) : 0;
    }
    dec = __shfl_sync(0xffffffffu, dec, 0);
    next = dec == 0 ? kGup : (dec == 1 ? kMap : kExit);
  } else if (kind == kGup) {
    next = kFup;
  } else if (kind == kMap) {
    int kn = 0;
    if (lane == 0) {
      kn = __ldcg(&st->k) + 1;
      if (kn < pr.K) st->k = kn;
    }
    kn = __shfl_sync(0xffffffffu, kn, 0);
    next = kn < pr.K ? kSplit : kExit;
  }
  // queue level of the next phase from the problem's estimated remaining chain (what
  // decides when it finishes): the phases left (the steps left at the mean iteration
  // count of its finished steps, a guess before the first, and the rest of the current
  // step, which once past the mean is taken to need as many iterations again; two
  // sweeps per iteration and three more phases per step) times a phase's latency (a
  // fixed part plus the column tiles of one sweep task), one level per factor of two
  int level = kLevels - 1;
  if (next != kExit) {
    if (lane == 0) {
      const int kc = __ldcg(&st->k), itc = __ldcg(&st->it);
      double sum = 0.0;
      for (int q = 0; q < kc; ++q) sum += (double)__ldcg(pr.iters + q);
      const double avg = kc > 0 ? sum / kc : 24.0;
      const double cur = fmax(fmax(avg - itc, (double)itc), 1.0);
      const double phases = (double)(pr.K - kc - 1) * (2.0 * avg + 3.0) + 2.0 * cur + 2.0;
      const double tiles = fmax((double)pr.Ty / pr.segs_f, (double)pr.Tx / pr.segs_g);
      const double us = phases * (10.0 + 0.6 * tiles);
      level = min(kLevels - 1, max(0, 14 - ilogb(fmax(us, 1.0))));
    }
    level = __shfl_sync(0xffffffffu, level, 0);
  }
  __threadfence();
  __syncwarp();
  if (next == kSplit) {
    const int nx = pr.Rx;
    enqueue_warp(P, level, pr.Rx + pr.Ry,
                 [&](int i) { return i < nx ? make_int4(pi, kSplit, i, 0) : make_int4(pi, kSplit, i - nx, 1); },
                 abort_flag);
  } else if (next == kFup) {
    const int s = pr.segs_f;
    enqueue_warp(P, level, pr.Rx * s, [&](int i) { return make_int4(pi, kFup, i / s, i % s); }, abort_flag);
  } else if (next == kGup) {
    const int s = pr.segs_g;
    enqueue_warp(P, level, pr.Ry * s, [&](int i) { return make_int4(pi, kGup, i / s, i % s); }, abort_flag);
  } else if (next == kMap) {
    enqueue_warp(P, level, pr.Rx, [&](int i) { return make_int4(pi, kMap, i, 0); }, abort_flag);
  } else {
    // the problem is done; the last one releases every CTA with an exit task
    unsigned prev = 0;
    if (lane == 0) prev = atom_sub_acq_rel_u32(P.remaining, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev == 1u)
      enqueue_warp(P, kLevels - 1, (int)gridDim.x, [&](int) { return make_int4(-1, kExit, 0, 0); }, abort_flag);
  }
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(NTHREADS, 1) progot_batch_tc(const Params P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Shared& sh = *reinterpret_cast<Shared*>(smem + OFF_CTRL);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int32_t* abort_flag = &sh.abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.tmem_full[b], 1);
      mbar_init(&sh.tmem_empty[b], 4);
      mbar_init(&sh.a_full[b], 1);
      mbar_init(&sh.a_empty[b], 1);
      mbar_init(&sh.seg_full[b], 128);
      mbar_init(&sh.seg_empty[b], 64);
    }
    mbar_init(&sh.p_full, 4);
    mbar_init(&sh.p_empty, 1);
    mbar_init(&sh.o_full, 1);
    mbar_init(&sh.o_empty, 4);
    for (int q = 0; q < NTQ; ++q) {
      mbar_init(&sh.task_full[q], 1);
      mbar_init(&sh.task_empty[q], 11);  // MMA warp, 8 LSE warps, 2 epilogue warps
    }
    mbar_init(&sh.drain, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    // A side of the bias product: all ones (bf16 0x3F80)
    uint32_t* ones = reinterpret_cast<uint32_t*>(smem + OFF_ONES);
    for (int i = threadIdx.x; i < 1024; i += NTHREADS) ones[i] = 0x3F803F80u;
    fence_async_smem();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = sh.tmem_base;
  const int split3 = P.split3;

  if (warp == 0) {
    // ------------------------------------------------------------ task fetch and TMA producer
    bool ok = true;
    int tq_i = 0, ka = 0, u = 0;
    for (;;) {
      int4 t = make_int4(-1, kExit, 0, 0);
      if (ok && !*abort_flag) {
        int okp = 1;
        if (lane == 0) okp = queue_pop(P, &t, abort_flag) ? 1 : 0;
        okp = __shfl_sync(0xffffffffu, okp, 0);
        t.x = __shfl_sync(0xffffffffu, t.x, 0);
        t.y = __shfl_sync(0xffffffffu, t.y, 0);
        t.z = __shfl_sync(0xffffffffu, t.z, 0);
        t.w = __shfl_sync(0xffffffffu, t.w, 0);
        if (!okp) {
          ok = false;
          t = make_int4(-1, kExit, 0, 0);
        }
      }
      const int qi = tq_i % NTQ;
      warp_wait_bar(&sh.task_empty[qi], (uint32_t)(((tq_i / NTQ) & 1) ^ 1), abort_flag, P, true);
      if (lane == 0) {
        sh.tq[qi] = t;
        mbar_arrive(&sh.task_full[qi]);
      }
      __syncwarp();
      ++tq_i;
      if (t.y == kExit) break;
      if (!ok || (t.y != kFup && t.y != kGup && t.y != kMap)) continue;
      const Prob& pr = P.probs[t.x];
      const bool map = t.y == kMap, g = t.y == kGup;
      const CUtensorMap* M = pr.maps;
      const CUtensorMap* mAh = g ? M + kYh : M + kXh;
      const CUtensorMap* mAl = g ? M + kYl : M + kXl;
      const CUtensorMap* mBh = map ? M + kYh64 : (g ? M + kXh : M + kYh);
      const CUtensorMap* mBl = map ? M + kYl64 : (g ? M + kXl : M + kYl);
      const CUtensorMap* mBb = map ? M + kYb64 : (g ? M + kXb : M + kYb);
      const int bn = map ? MP_BN : SW_BN;
      const uint32_t b_bytes = (uint32_t)bn * 128u * (split3 ? 2u : 1u) + (uint32_t)bn * 32u;
      int t0, t1;
      task_tiles(pr, t, &t0, &t1);
      // the operands and bias rows were written by generic stores of earlier phases
      if (lane == 0) fence_proxy_global();
      __syncwarp();
      const int ai = ka & 1;
      ok = warp_wait_bar(&sh.a_empty[ai], (uint32_t)(((ka >> 1) & 1) ^ 1), abort_flag, P);
      if (!ok) continue;
      unsigned char* abuf = smem + ai * 2 * A_HALF;
      if (elect_one()) {
        mbar_arrive_expect_tx(&sh.a_full[ai], split3 ? 2 * A_HALF : A_HALF);
        tma_load_2d(abuf, mAh, &sh.a_full[ai], 0, t.z * BM);
        if (split3) tma_load_2d(abuf + A_HALF, mAl, &sh.a_full[ai], 0, t.z * BM);
      }
      __syncwarp();
      ++ka;
      for (int q = t0; q < t1; ++q, ++u) {
        const int s = u % NST;
        ok = warp_wait_bar(&sh.empty[s], (uint32_t)(((u / NST) & 1) ^ 1), abort_flag, P);
        if (!ok) break;
        unsigned char* stg = smem + OFF_ST + s * ST_BYTES;
        if (elect_one()) {
          mbar_arrive_expect_tx(&sh.full[s], b_bytes);
          tma_load_2d(stg, mBh, &sh.full[s], 0, q * bn);
          if (split3) tma_load_2d(stg + ST_LO, mBl, &sh.full[s], 0, q * bn);
          tma_load_2d(stg + ST_BIAS, mBb, &sh.full[s], 0, q * bn);
        }
        __syncwarp();
      }
    }
    // copies still in flight land before shared memory is released
    if (*abort_flag) {
      for (int k = max(0, ka - 2); k < ka; ++k)
        warp_wait_bar(&sh.a_full[k & 1], (uint32_t)((k >> 1) & 1), abort_flag, P, true);
      for (int v = max(0, u - NST); v < u; ++v)
        warp_wait_bar(&sh.full[v % NST], (uint32_t)((v / NST) & 1), abort_flag, P, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint64_t ones = desc_sw32(smem_u32(smem + OFF_ONES));
    const uint32_t id_sw = make_idesc(BM, SW_BN), id_mp = make_idesc(BM, MP_BN);
    const uint32_t id_py = make_idesc(BM, MP_BN) | (1u << 16);  // B MN-major
    const uint32_t p0 = smem_u32(smem + OFF_P);
    bool ok = true;
    int tq_i = 0, ka = 0, u = 0, tl = 0, pq = 0, mt = 0;
    int buse[2] = {0, 0};  // tiles issued into each TMEM buffer (the tile counter skips at task starts)
    // O += P Y~ of one map tile from the P tile and the tile's held stage; the stage and
    // the P tile go back after it
    auto issue_py = [&](int stage, bool first, bool last) -> bool {
      if (first && mt > 0 && !warp_wait_bar(&sh.o_empty, (uint32_t)((mt - 1) & 1), abort_flag, P)) return false;
      if (!warp_wait_bar(&sh.p_full, (uint32_t)(pq & 1), abort_flag, P)) return false;
      tc_fence_after();
      const uint32_t stg = smem_u32(smem + OFF_ST + stage * ST_BYTES);
      const uint64_t ah = desc_sw128(p0), al = desc_sw128(p0 + P_LO);
      const uint64_t bh = desc_mn(stg), bl = desc_mn(stg + ST_LO);
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 2), bdv = (uint64_t)(kk * 128);
          umma_rt(tmem_base + O_COL, ah + adv, bh + bdv, id_py, (first && kk == 0) ? 0u : 1u);
          if (split3) {
            umma_rt(tmem_base + O_COL, ah + adv, bl + bdv, id_py, 1u);
            umma_rt(tmem_base + O_COL, al + adv, bh + bdv, id_py, 1u);
          }
        }
        umma_commit(&sh.p_empty);
        umma_commit(&sh.empty[stage]);
        if (last) umma_commit(&sh.o_full);
      }
      __syncwarp();
      ++pq;
      return true;
    };
    for (;;) {
      const int4 t = ring_get(sh, tq_i++, abort_flag, P);
      if (t.y == kExit) break;
      if (!ok || (t.y != kFup && t.y != kGup && t.y != kMap)) continue;
      const Prob& pr = P.probs[t.x];
      const bool map = t.y == kMap;
      int t0, t1;
      task_tiles(pr, t, &t0, &t1);
      const int ai = ka & 1;
      ok = warp_wait_bar(&sh.a_full[ai], (uint32_t)((ka >> 1) & 1), abort_flag, P);
      ++ka;
      if (!ok) continue;
      tc_fence_after();
      const uint32_t a_hi = smem_u32(smem + ai * 2 * A_HALF), a_lo = a_hi + A_HALF;
      const uint64_t ah = desc_sw128(a_hi), al = desc_sw128(a_lo);
      const uint32_t idesc = map ? id_mp : id_sw;
      int pend = -1;
      bool pend_first = false;
      tl = (tl + 1) & ~1;  // a task's first tile goes to TMEM buffer 0 (LSE warpgroup 0)
      for (int q = t0; q < t1 && ok; ++q, ++tl, ++u) {
        const int b = tl & 1, s = u % NST;
        ok = warp_wait_bar(&sh.tmem_empty[b], (uint32_t)((buse[b] & 1) ^ 1), abort_flag, P);
        if (!ok) break;
        ++buse[b];
        ok = warp_wait_bar(&sh.full[s], (uint32_t)((u / NST) & 1), abort_flag, P);
        if (!ok) break;
        tc_fence_after();
        const uint32_t stg = smem_u32(smem + OFF_ST + s * ST_BYTES);
        const uint64_t bh = desc_sw128(stg), bl = desc_sw128(stg + ST_LO);
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * 128);
        if (elect_one()) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // +32 bytes per K = 16 step inside the 128-byte swizzle atom (encoded >> 4)
            const uint64_t adv = (uint64_t)(kk * 2);
            umma_rt(d_tmem, ah + adv, bh + adv, idesc, kk > 0 ? 1u : 0u);
            if (split3) {
              umma_rt(d_tmem, ah + adv, bl + adv, idesc, 1u);
              umma_rt(d_tmem, al + adv, bh + adv, idesc, 1u);
            }
          }
          // t_ij = c (a_i . b_j) + beta_j
          umma_rt(d_tmem, ones, desc_sw32(stg + ST_BIAS), idesc, 1u);
          if (!map) umma_commit(&sh.empty[s]);  // a map tile's stage is read again by P Y~
          umma_commit(&sh.tmem_full[b]);
        }
        __syncwarp();
        if (map) {
          // P Y~ of the previous tile after S of this one: its exponentials overlap these products
          if (pend >= 0) ok = issue_py(pend, pend_first, false);
          pend = s;
          pend_first = (q == t0);
        }
      }
      if (map) {
        if (ok && pend >= 0) ok = issue_py(pend, pend_first, true);
        ++mt;
      }
      if (elect_one()) umma_commit(&sh.a_empty[ai]);
      __syncwarp();
    }
    if (elect_one()) umma_commit(&sh.drain);
    __syncwarp();
    warp_wait_bar(&sh.drain, 0, abort_flag, P, true);
  } else if (threadIdx.x < EPI_TID0) {
    // ------------------------------------------------------------ LSE warps (and CUDA-core tasks)
    const int wg = (warp - 2) >> 2;
    const int quarter = warp & 3;
    const int row_local = quarter * 32 + lane;
    unsigned char* prow = smem + OFF_P + (row_local >> 3) * 1024 + (row_local & 7) * 128;
    int tq_i = 0, tl = 0, jt = 0, pq = 0, mt = 0, kt = 0;
    bool dead = false;
    for (;;) {
      const int4 t = ring_get(sh, tq_i++, abort_flag, P);
      if (t.y == kExit) break;
      const Prob& pr = P.probs[t.x];
      float2 hand = make_float2(0.f, 0.f);
      if (t.y == kFup || t.y == kGup) {
        int t0, t1;
        task_tiles(pr, t, &t0, &t1);
        float m_run = -INFINITY, s_run = 0.f;
        // tile q of the task goes to warpgroup (q - t0) & 1 whatever this CTA ran before, so
        // that the float32 partial sums (and the result) depend only on the task
        tl = (tl + 1) & ~1;
        for (int q = t0; q < t1; ++q, ++tl) {
          if ((tl & 1) != wg) continue;
          const uint32_t ph = (uint32_t)(jt & 1);
          ++jt;
          if (dead) continue;
          int okv = 0;
          if (lane == 0) okv = wait_bar(&sh.tmem_full[wg], ph, abort_flag, P) ? 1 : 0;
          if (__shfl_sync(0xffffffffu, okv, 0) == 0) {
            dead = true;
            continue;
          }
          __syncwarp();
          tc_fence_after();
          const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * 128);
          float v[4][32];
          PROGOT_TMEM_LD32(taddr + 0, v[0]);
          PROGOT_TMEM_LD32(taddr + 32, v[1]);
          PROGOT_TMEM_LD32(taddr + 64, v[2]);
          PROGOT_TMEM_LD32(taddr + 96, v[3]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.tmem_empty[wg]);
          float mx[8];
#pragma unroll
          for (int qq = 0; qq < 8; ++qq) mx[qq] = v[qq >> 1][(qq & 1) * 16];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
#pragma unroll
            for (int i = 1; i < 16; i += 2) {
              mx[cc * 2] = max3(mx[cc * 2], v[cc][i], v[cc][i + 1 < 16 ? i + 1 : i]);
              mx[cc * 2 + 1] = max3(mx[cc * 2 + 1], v[cc][16 + i], v[cc][16 + (i + 1 < 16 ? i + 1 : i)]);
            }
          const float tmax = max3(max3(mx[0], mx[1], mx[2]), max3(mx[3], mx[4], mx[5]), fmaxf(mx[6], mx[7]));
          const float mnew = fmaxf(m_run, tmax);
          if (mnew != -INFINITY) {
            const uint64_t negm = pack2(-mnew, -mnew);
            uint64_t acc[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) acc[qq] = 0ull;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
#pragma unroll
              for (int i = 0; i < 32; i += 2) {
                float a0, a1;
                unpack2(add2(pack2(v[cc][i], v[cc][i + 1]), negm), a0, a1);
                acc[(i >> 1) & 3] = add2(acc[(i >> 1) & 3], pack2(fast_exp2(a0), fast_exp2(a1)));
              }
            float s0, s1, s2, s3, s4, s5, s6, s7;
            unpack2(acc[0], s0, s1);
            unpack2(acc[1], s2, s3);
            unpack2(acc[2], s4, s5);
            unpack2(acc[3], s6, s7);
            s_run = s_run * fast_exp2(m_run - mnew) + (((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7)));
            m_run = mnew;
          }
        }
        if (dead) {
          m_run = NAN;
          s_run = NAN;
        }
        if (wg == 1) sh.ms[kt & 1][row_local] = make_float2(m_run, s_run);
        bar_lse_all();
        if (wg == 0) {
          const float2 o = sh.ms[kt & 1][row_local];
          const float2 mrg = lse_combine(make_float2(m_run, s_run), o);
          const bool bad = isnan(o.y) || isnan(s_run);
          hand = bad ? make_float2(NAN, NAN) : mrg;
        }
      } else if (t.y == kMap) {
        const int64_t i = (int64_t)t.z * BM + row_local;
        const bool row_ok = i < pr.n;
        const float Lr = row_ok ? __ldcg(pr.L + i) : 0.f;
        float rs = 0.f;
        tl = (tl + 1) & ~1;
        for (int q = 0; q < pr.Tm; ++q, ++tl, ++pq) {
          if ((tl & 1) != wg) continue;
          const uint32_t ph = (uint32_t)(jt & 1);
          ++jt;
          if (dead) continue;
          if (!warp_wait_bar(&sh.tmem_full[wg], ph, abort_flag, P)) {
            dead = true;
            continue;
          }
          tc_fence_after();
          const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * 128);
          float v[2][32];
          PROGOT_TMEM_LD32(taddr, v[0]);
          PROGOT_TMEM_LD32(taddr + 32, v[1]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.tmem_empty[wg]);
          // P_ij = 2^{t_ij - L_i} (0 on rows past the cloud)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const float pv = row_ok ? fast_exp2(v[cc][e] - Lr) : 0.f;
              v[cc][e] = pv;
              rs += pv;
            }
          // the P tile is free once the previous map tile's P Y~ has read it
          if (!warp_wait_bar(&sh.p_empty, (uint32_t)((pq & 1) ^ 1), abort_flag, P)) {
            dead = true;
            continue;
          }
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            uint4 h4, l4;
            split8(&v[ch >> 2][(ch & 3) * 8], h4, l4);
            const int pos = (ch ^ (row_local & 7)) * 16;
            *reinterpret_cast<uint4*>(prow + pos) = h4;
            *reinterpret_cast<uint4*>(prow + P_LO + pos) = l4;
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.p_full);
        }
        if (wg == 1) sh.ms[kt & 1][row_local] = make_float2(rs, 0.f);
        bar_lse_all();
        if (wg == 0) {
          rs += sh.ms[kt & 1][row_local].x;
          // the centre in shared memory (its reads below cannot alias the stores of x)
          if (row_local < 64) sh.mu_s[row_local] = __ldcg(pr.mu + row_local);
          bar_wg0();
          float o[2][32];
          const bool okv = !dead && warp_wait_bar(&sh.o_full, (uint32_t)(mt & 1), abort_flag, P);
          if (okv) {
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + O_COL;
            PROGOT_TMEM_LD32(taddr, o[0]);
            PROGOT_TMEM_LD32(taddr + 32, o[1]);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.o_empty);
          } else {
            dead = true;
          }
          if (okv && row_ok) {
            // x <- x + alpha (T - x), T = O / R + mu (the y operand of P Y~ is y - mu);
            // each half's loads before its stores
            const int k = __ldcg(&pr.st->k);
            const StepC& C = pr.sc[k];
            const int d = pr.d;
            float* xr = pr.X + i * d;
            const float inv_rs = 1.f / rs;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float xv[32];
#pragma unroll
              for (int e = 0; e < 32; ++e) xv[e] = 32 * h + e < d ? __ldcg(xr + 32 * h + e) : 0.f;
#pragma unroll
              for (int e = 0; e < 32; ++e) {
                const int c = 32 * h + e;
                if (c < d) {
                  const float tx = fmaf(o[h][e], inv_rs, sh.mu_s[c]);
                  xr[c] = fmaf(C.alpha, tx - xv[e], xv[e]);
                }
              }
            }
            if (k == pr.K - 1 && pr.f_last != nullptr) pr.f_last[i] = __ldcg(pr.f[__ldcg(&pr.st->fcur)] + i);
          }
        }
        ++mt;
      } else {
        // MOM / SPLIT on the CUDA cores
        if (t.y == kMom) task_mom(pr, t.z, t.w, smem);
        else task_split(pr, t.z, t.w, split3, sh.mu_sp, reinterpret_cast<double*>(smem + OFF_P));
        fence_proxy_global();  // the operand and bias rows are read by TMA in later phases
        bar_lse_all();
      }
      // hand the task's result (or its completion) to the epilogue warps
      if (wg == 0) {
        const int sl = kt & 1;
        wait_bar(&sh.seg_empty[sl], (uint32_t)(((kt >> 1) & 1) ^ 1), abort_flag, P, true);
        sh.seg[sl][row_local] = hand;
        mbar_arrive(&sh.seg_full[sl]);
      }
      ++kt;
    }
  } else {
    // ------------------------------------------------------------ task epilogues and phase finishes
    const int etid = threadIdx.x - EPI_TID0;  // 0..63
    int tq_i = 0, kt = 0;
    for (;;) {
      const int4 t = ring_get(sh, tq_i++, abort_flag, P);
      if (t.y == kExit) break;
      const Prob& pr = P.probs[t.x];
      const int sl = kt & 1;
      const int kind = t.y;
      bool fin = true;
      int target = pr.Rx + pr.Ry;
      if (kind == kFup || kind == kGup) {
        const int sd = kind == kGup ? 1 : 0;
        const int k = __ldcg(&pr.st->k), fcur = __ldcg(&pr.st->fcur);
        const StepC& C = pr.sc[k];
        const int64_t nA = sd ? pr.m : pr.n;
        const int rb = t.z, seg = t.w, segs = sd ? pr.segs_g : pr.segs_f;
        const float* an_arr = sd ? pr.yn : pr.xn;
        const float* w_arr = sd ? pr.b : pr.a;
        const float* pot_cur = pr.f[fcur];
        float an[2], pot[2], w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t i = (int64_t)rb * BM + etid + 64 * h;
          an[h] = 0.f;
          pot[h] = 0.f;
          w[h] = 0.f;
          if (i < nA) {
            an[h] = __ldcg(an_arr + i);
            pot[h] = sd ? 0.f : __ldcg(pot_cur + i);
            w[h] = w_arr ? w_arr[i] : 0.f;
          }
        }
        const bool okw = wait_bar(&sh.seg_full[sl], (uint32_t)((kt >> 1) & 1), abort_flag, P, true);
        float2 mv[2];
        mv[0] = okw ? sh.seg[sl][etid] : make_float2(NAN, NAN);
        mv[1] = okw ? sh.seg[sl][etid + 64] : make_float2(NAN, NAN);
        mbar_arrive(&sh.seg_empty[sl]);
        float2 acc[2] = {mv[0], mv[1]};
        if (segs > 1) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int rl = etid + 64 * h;
            if ((int64_t)rb * BM + rl < nA) pr.part[((int64_t)rb * segs + seg) * BM + rl] = mv[h];
          }
          bar_epi();  // every row's partial is stored before the arrival
          if (etid == 0) {
            const unsigned prev = atomic_add_acq_rel_gpu(pr.cnt + rb, 1u);
            sh.e_last = (prev + 1u == (unsigned)segs);
          }
          bar_epi();
          fin = sh.e_last != 0;
          if (fin) {
            // the row block's segments in segment order (this task's own from registers)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int rl = etid + 64 * h;
              float2 a2 = make_float2(-INFINITY, 0.f);
              if ((int64_t)rb * BM + rl < nA)
                for (int s2 = 0; s2 < segs; ++s2)
                  a2 = combine_fast(a2, s2 == seg ? mv[h] : __ldcg(pr.part + ((int64_t)rb * segs + s2) * BM + rl));
              acc[h] = a2;
            }
          }
        }
        if (fin) {
          float e[2] = {0.f, 0.f};
          __nv_bfloat16* bias = sd ? pr.yb : pr.xb;  // bias rows of this side's potential
          float* out = sd ? pr.g_all + (int64_t)k * pr.m : pr.f[fcur ^ 1];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int64_t i = (int64_t)rb * BM + etid + 64 * h;
            if (i >= nA) continue;
            const float Lr = acc[h].x + __log2f(acc[h].y);
            // f_i = eps log w_i + |a_i|^2 - eps ln2 L (float32 FMAs on eps ln2 = c_hi + c_lo)
            float tt = fmaf(-C.c_hi, Lr, an[h]);
            tt = fmaf(-C.c_lo, Lr, tt);
            float fnew;
            if (w_arr) {
              const float lw = __logf(w[h]);
              fnew = tt + fmaf(C.e_hi, lw, C.e_lo * lw);
            } else {
              fnew = (tt + C.w_lo[sd]) + C.w_hi[sd];
            }
            out[i] = fnew;
            write_bias16(bias + i * 16, (fnew - an[h]) * C.bscale);
            if (sd == 0) {
              pr.L[i] = Lr;
              // a_i |exp((f_old - f_new)/eps) - 1|, the exponent capped at 80
              float dl = (pot[h] - fnew) * C.inv_eps_f;
              if (dl > 80.f) dl = 80.f;
              const float wi = w_arr ? w[h] : (float)(1.0 / (double)pr.n);
              e[h] = wi * fabsf(expm1f(dl));
            }
          }
          fence_proxy_global();  // the bias rows are read by TMA in the next phase
          if (sd == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float v = e[h];
#pragma unroll
              for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
              if ((etid & 31) == 0) sh.ered[(etid + 64 * h) >> 5] = v;
            }
          }
          bar_epi();
          if (etid == 0) {
            if (sd == 0) pr.errpart[rb] = (double)((sh.ered[0] + sh.ered[1]) + (sh.ered[2] + sh.ered[3]));
            if (segs > 1) pr.cnt[rb] = 0u;
          }
          target = sd ? pr.Ry : pr.Rx;
        }
      } else {
        wait_bar(&sh.seg_full[sl], (uint32_t)((kt >> 1) & 1), abort_flag, P, true);
        mbar_arrive(&sh.seg_empty[sl]);
        if (kind == kMap) target = pr.Rx;
      }
      if (fin) {
        if (etid == 0) {
          const unsigned prev = atomic_add_acq_rel_gpu(pr.phase, 1u);
          sh.p_last = (prev + 1u == (unsigned)target) && !*abort_flag;
        }
        bar_epi();
        if (sh.p_last && etid < 32) phase_finish(P, pr, t.x, kind, abort_flag);
        bar_epi();
      }
      ++kt;
    }
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if (sh.abort_flag != 0 && threadIdx.x == 0) atomicExch(P.fault, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// Queue and per-problem state at the start of a run.
__global__ void batch_init_kernel(Params P, const int4* __restrict__ init, int64_t n_init, PState* states, int count) {
  const int64_t q = (int64_t)P.qmask + 1;
  // level 0 starts with the initial tasks, the other levels empty
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < kLevels * q; s += (int64_t)gridDim.x * blockDim.x) {
    const bool pre = s < n_init;
    P.qseq[s] = (unsigned long long)(pre ? s % q + 1 : s % q);
    if (pre) P.qslots[s] = init[s];
  }
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += (int64_t)gridDim.x * blockDim.x) {
    PState z;
    z.k = 0;
    z.it = 0;
    z.status = kRunning;
    z.fcur = 0;
    z.best_it = 0;
    z.done = 0;
    z.pad0 = z.pad1 = 0;
    z.err = 0.0;
    z.best_err = INFINITY;
    states[p] = z;
  }
  if (blockIdx.x == 0 && threadIdx.x < kLevels) {
    P.qctl[64 * threadIdx.x] = 0ull;
    P.qctl[64 * threadIdx.x + 16] = threadIdx.x == 0 ? (unsigned long long)n_init : 0ull;
    P.qctl[64 * threadIdx.x + 32] = threadIdx.x == 0 ? (unsigned long long)n_init : 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *P.remaining = (unsigned)count;
    *P.fault = 0;
  }
}

}  // namespace bat
}  // namespace tc
}  // namespace progot

// ---------------------------------------------------------------- host side
using progot::tc::bat::Params;
using progot::tc::bat::Prob;
using progot::tc::bat::PState;
using progot::tc::bat::StepC;

struct progot_batch_plan {
  int32_t count = 0, precision = 0, max_iter = 0, G = 0, Kmax = 0;
  int32_t target = 8;             // tasks per sweep phase the column segmentation aims at
  std::vector<Prob> probs;        // host image of the device descriptors
  Prob* d_probs = nullptr;
  Params P;
  int4* d_init = nullptr;
  int64_t n_init = 0;
  PState* d_states = nullptr;
  unsigned* d_counters = nullptr;
  size_t counters_bytes = 0;
  int32_t* d_stat = nullptr;      // count x Kmax step statuses (-1: step not run)
  int32_t* d_iters = nullptr;
  double* d_errs = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace progot {
namespace {

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }
int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct Dims {
  int64_t n, m;
  int32_t d, K, Rx, Ry, Tx, Ty, Tm;
};

Dims dims_of(const progot_problem& p) {
  Dims q;
  q.n = p.n;
  q.m = p.m;
  q.d = p.d;
  q.K = p.K;
  q.Rx = (int32_t)cdiv64(p.n, 128);
  q.Ry = (int32_t)cdiv64(p.m, 128);
  q.Tx = (int32_t)cdiv64(p.n, tc::bat::SW_BN);
  q.Ty = (int32_t)cdiv64(p.m, tc::bat::SW_BN);
  q.Tm = (int32_t)cdiv64(p.m, tc::bat::MP_BN);
  return q;
}

// Bytes of one problem's device region (every piece 256-byte aligned).
size_t problem_bytes(const Dims& q) {
  const size_t rmax = (size_t)std::max(q.Rx, q.Ry);
  size_t b = al256(tc::bat::kNumMaps * sizeof(CUtensorMap));
  b += 2 * al256((size_t)q.Rx * 128 * 64 * 2) + 2 * al256((size_t)q.Ry * 128 * 64 * 2);  // operands
  b += al256((size_t)q.Rx * 128 * 32) + al256((size_t)q.Ry * 128 * 32);                  // bias rows
  b += 4 * al256((size_t)q.n * 4) + al256((size_t)q.m * 4);                               // f0 f1 xn L, yn
  b += al256(64 * 4);                                                                      // mu
  b += al256(rmax * tc::bat::kMaxSegs * 128 * sizeof(float2));                             // partials
  b += al256((size_t)q.Rx * 8) + al256((size_t)(q.Rx + q.Ry) * 64 * 8);                   // errpart, mom
  b += al256((size_t)q.K * sizeof(StepC));
  return b;
}

struct Totals {
  size_t bytes = 0, counters = 0;
  int64_t n_init = 0, qsize = 0;
  int32_t Kmax = 0;
};

Totals totals_of(const progot_problem* probs, int32_t count, int sms) {
  Totals t;
  int64_t outstanding = 0;
  for (int i = 0; i < count; ++i) {
    const Dims q = dims_of(probs[i]);
    t.bytes += problem_bytes(q);
    t.counters += (size_t)std::max(q.Rx, q.Ry) + 1;
    t.n_init += q.Rx + q.Ry;
    t.Kmax = std::max(t.Kmax, q.K);
    outstanding += (int64_t)std::max(q.Rx, q.Ry) * tc::bat::kMaxSegs + q.Rx + q.Ry;
  }
  // a ring that holds every task that can be outstanding at once: one phase per
  // problem, the initial tasks, the exits and the positions idle CTAs reserve
  const int64_t need = outstanding + t.n_init + 4 * (int64_t)sms + 64;
  t.qsize = 1024;
  while (t.qsize < need) t.qsize <<= 1;
  t.bytes += al256((size_t)count * sizeof(Prob));
  t.bytes += al256((size_t)tc::bat::kLevels * t.qsize * sizeof(int4)) + al256((size_t)tc::bat::kLevels * t.qsize * 8);
  t.bytes += 512 * tc::bat::kLevels + 256;                      // heads, tails, counts; remaining, fault
  t.bytes += al256((size_t)t.n_init * sizeof(int4));
  t.bytes += al256((size_t)count * sizeof(PState));
  t.bytes += al256(t.counters * 4);
  t.bytes += al256((size_t)count * t.Kmax * 4) * 2 + al256((size_t)count * t.Kmax * 8);  // stat, iters, errs
  t.bytes += 256;                                               // base alignment
  return t;
}

int check_batch_problem(const progot_problem& p) {
  if (p.x == nullptr || p.y == nullptr || p.x_out == nullptr || p.g_all == nullptr || p.alpha == nullptr ||
      p.eps == nullptr || p.tau == nullptr)
    return fail_message(PROGOT_ERR_INVALID_ARG, "a batched problem has a NULL required pointer");
  if (p.n <= 0 || p.m <= 0 || p.d <= 0 || p.K <= 0)
    return fail_message(PROGOT_ERR_INVALID_ARG, "a batched problem has a non-positive size");
  if (p.d > 64)
    return fail_message(PROGOT_ERR_INVALID_ARG, "the persistent batched engine takes d <= 64");
  if (p.n > (int64_t)1 << 24 || p.m > (int64_t)1 << 24)
    return fail_message(PROGOT_ERR_INVALID_ARG, "the persistent batched engine takes n, m <= 2^24");
  for (int k = 0; k < p.K; ++k) {
    if (!(p.eps[k] > 0.0) || !std::isfinite(p.eps[k]))
      return fail_message(PROGOT_ERR_INVALID_ARG, "eps_k must be positive and finite");
    if (!(p.alpha[k] > 0.0 && p.alpha[k] <= 1.0))
      return fail_message(PROGOT_ERR_INVALID_ARG, "alpha_k must lie in (0, 1]");
    if (!(p.tau[k] >= 0.0)) return fail_message(PROGOT_ERR_INVALID_ARG, "tau_k must be >= 0");
  }
  return PROGOT_OK;
}

void set_segments(progot_batch_plan* pl) {
  for (Prob& pr : pl->probs) {
    auto segs = [&](int R, int T) {
      int s = (int)cdiv64(pl->target, R);
      return std::max(1, std::min(s, std::min(tc::bat::kMaxSegs, T)));
    };
    pr.segs_f = segs(pr.Rx, pr.Ty);
    pr.segs_g = segs(pr.Ry, pr.Tx);
  }
}

cudaError_t enqueue_run(progot_batch_plan* pl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pl->d_counters, 0, pl->counters_bytes, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(pl->d_stat, 0xFF, sizeof(int32_t) * (size_t)pl->count * pl->Kmax, s);
  if (e != cudaSuccess) return e;
  tc::bat::batch_init_kernel<<<64, 256, 0, s>>>(pl->P, pl->d_init, pl->n_init, pl->d_states, pl->count);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tc::bat::progot_batch_tc<<<pl->G, tc::bat::NTHREADS, tc::bat::SMEM_TOTAL, s>>>(pl->P);
  count_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace progot

using namespace progot;

extern "C" {

size_t progot_batch_plan_workspace_size(const progot_problem* problems, int32_t count, int32_t precision) {
  (void)precision;
  if (problems == nullptr || count <= 0) return 0;
  return totals_of(problems, count, device_sm_count()).bytes;
}

int progot_batch_plan_create(const progot_problem* problems, int32_t count, int32_t max_iter, int32_t precision,
                             void* workspace, size_t ws_bytes, progot_batch_plan** out) {
  set_last_error_message("");
  if (out == nullptr || problems == nullptr || count <= 0)
    return fail_message(PROGOT_ERR_INVALID_ARG, "problems, count > 0 and an output handle are required");
  *out = nullptr;
  if (precision != PROGOT_BF16X3 && precision != PROGOT_BF16)
    return fail_message(PROGOT_ERR_INVALID_ARG, "the persistent batched engine runs the bf16x3 and bf16 precisions");
  if (max_iter < 0) return fail_message(PROGOT_ERR_INVALID_ARG, "max_iter must be >= 0");
  for (int i = 0; i < count; ++i) {
    const int rc = check_batch_problem(problems[i]);
    if (rc) return rc;
  }
  const int sms = device_sm_count();
  const Totals tot = totals_of(problems, count, sms);
  if (workspace == nullptr || ws_bytes < tot.bytes)
    return fail_message(PROGOT_ERR_WORKSPACE, "batch workspace too small (see progot_batch_plan_workspace_size)");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tc::bat::progot_batch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc::bat::SMEM_TOTAL);
    if (e != cudaSuccess) return fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
    attr_set = true;
  }
  progot_batch_plan* pl = new (std::nothrow) progot_batch_plan();
  if (pl == nullptr) return fail_message(PROGOT_ERR_OOM, "host allocation failed");
  pl->count = count;
  pl->precision = precision;
  pl->max_iter = max_iter;
  pl->G = sms;
  pl->Kmax = tot.Kmax;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
  char* cur = base;
  auto take = [&](size_t bytes) {
    char* r = cur;
    cur += al256(bytes);
    return r;
  };
  pl->d_probs = reinterpret_cast<Prob*>(take((size_t)count * sizeof(Prob)));
  int4* qslots = reinterpret_cast<int4*>(take((size_t)tc::bat::kLevels * tot.qsize * sizeof(int4)));
  unsigned long long* qseq = reinterpret_cast<unsigned long long*>(take((size_t)tc::bat::kLevels * tot.qsize * 8));
  char* qctl = take(512 * tc::bat::kLevels);
  char* ctl = take(256);
  pl->d_init = reinterpret_cast<int4*>(take((size_t)tot.n_init * sizeof(int4)));
  pl->n_init = tot.n_init;
  pl->d_states = reinterpret_cast<PState*>(take((size_t)count * sizeof(PState)));
  pl->d_counters = reinterpret_cast<unsigned*>(take(tot.counters * 4));
  pl->counters_bytes = tot.counters * 4;
  pl->d_stat = reinterpret_cast<int32_t*>(take((size_t)count * tot.Kmax * 4));
  pl->d_iters = reinterpret_cast<int32_t*>(take((size_t)count * tot.Kmax * 4));
  pl->d_errs = reinterpret_cast<double*>(take((size_t)count * tot.Kmax * 8));
  Params& P = pl->P;
  P.probs = pl->d_probs;
  P.qslots = qslots;
  P.qseq = qseq;
  P.qctl = reinterpret_cast<unsigned long long*>(qctl);
  P.remaining = reinterpret_cast<unsigned*>(ctl);
  P.fault = reinterpret_cast<int32_t*>(ctl + 4);
  P.qmask = (unsigned long long)tot.qsize - 1ull;
  P.wait_ns = wait_limit_setting();
  P.split3 = precision == PROGOT_BF16X3 ? 1 : 0;

  // per-problem regions, descriptors, tensor maps and step constants
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::vector<int4> init;
  init.reserve((size_t)tot.n_init);
  unsigned* cnt_cur = pl->d_counters;
  pl->probs.resize(count);
  int rc = PROGOT_OK;
  for (int i = 0; i < count && rc == PROGOT_OK; ++i) {
    const progot_problem& p = problems[i];
    const Dims q = dims_of(p);
    Prob pr;
    memset(&pr, 0, sizeof(pr));
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(take(tc::bat::kNumMaps * sizeof(CUtensorMap)));
    pr.xh = reinterpret_cast<__nv_bfloat16*>(take((size_t)q.Rx * 128 * 64 * 2));
    pr.xl = reinterpret_cast<__nv_bfloat16*>(take((size_t)q.Rx * 128 * 64 * 2));
    pr.yh = reinterpret_cast<__nv_bfloat16*>(take((size_t)q.Ry * 128 * 64 * 2));
    pr.yl = reinterpret_cast<__nv_bfloat16*>(take((size_t)q.Ry * 128 * 64 * 2));
    pr.xb = reinterpret_cast<__nv_bfloat16*>(take((size_t)q.Rx * 128 * 32));
    pr.yb = reinterpret_cast<__nv_bfloat16*>(take((size_t)q.Ry * 128 * 32));
    pr.f[0] = reinterpret_cast<float*>(take((size_t)q.n * 4));
    pr.f[1] = reinterpret_cast<float*>(take((size_t)q.n * 4));
    pr.xn = reinterpret_cast<float*>(take((size_t)q.n * 4));
    pr.L = reinterpret_cast<float*>(take((size_t)q.n * 4));
    pr.yn = reinterpret_cast<float*>(take((size_t)q.m * 4));
    pr.mu = reinterpret_cast<float*>(take(64 * 4));
    pr.part = reinterpret_cast<float2*>(take((size_t)std::max(q.Rx, q.Ry) * tc::bat::kMaxSegs * 128 * sizeof(float2)));
    pr.errpart = reinterpret_cast<double*>(take((size_t)q.Rx * 8));
    pr.mom = reinterpret_cast<double*>(take((size_t)(q.Rx + q.Ry) * 64 * 8));
    StepC* sc = reinterpret_cast<StepC*>(take((size_t)q.K * sizeof(StepC)));
    pr.x = p.x;
    pr.y = p.y;
    pr.a = p.a;
    pr.b = p.b;
    pr.X = p.x_out;
    pr.g_all = p.g_all;
    pr.f_last = p.f_last;
    pr.cnt = cnt_cur;
    pr.phase = cnt_cur + std::max(q.Rx, q.Ry);
    cnt_cur += std::max(q.Rx, q.Ry) + 1;
    pr.st = pl->d_states + i;
    pr.sc = sc;
    pr.stat = pl->d_stat + (size_t)i * tot.Kmax;
    pr.iters = pl->d_iters + (size_t)i * tot.Kmax;
    pr.errs = pl->d_errs + (size_t)i * tot.Kmax;
    pr.maps = maps;
    pr.n = q.n;
    pr.m = q.m;
    pr.d = q.d;
    pr.K = q.K;
    pr.Rx = q.Rx;
    pr.Ry = q.Ry;
    pr.Tx = q.Tx;
    pr.Ty = q.Ty;
    pr.Tm = q.Tm;
    pr.max_iter = max_iter;
    pr.stall_window = stall_window_setting();
    // tensor maps (operands: rows = n or m, zero fill past the cloud; bias rows: whole row blocks)
    CUtensorMap hm[tc::bat::kNumMaps];
    void* xl = P.split3 ? (void*)pr.xl : (void*)pr.xh;
    void* yl = P.split3 ? (void*)pr.yl : (void*)pr.yh;
    rc = encode_operand_map(&hm[tc::bat::kXh], pr.xh, q.n, 64, 128);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kXl], xl, q.n, 64, 128);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kYh], pr.yh, q.m, 64, 128);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kYl], yl, q.m, 64, 128);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kXb], pr.xb, (int64_t)q.Rx * 128, 16, 128);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kYb], pr.yb, (int64_t)q.Ry * 128, 16, 128);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kYh64], pr.yh, q.m, 64, 64);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kYl64], yl, q.m, 64, 64);
    if (!rc) rc = encode_operand_map(&hm[tc::bat::kYb64], pr.yb, (int64_t)q.Ry * 128, 16, 64);
    if (rc) break;
    std::vector<StepC> hs((size_t)q.K);
    for (int k = 0; k < q.K; ++k) {
      const double eps = p.eps[k];
      StepC& c = hs[k];
      memset(&c, 0, sizeof(c));
      c.tau = p.tau[k];
      c.c = (float)(2.0 * kLog2e / eps);
      c.bscale = (float)(kLog2e / eps);
      c.inv_eps_f = (float)(1.0 / eps);
      const double cl = eps * kLn2;
      c.c_hi = (float)cl;
      c.c_lo = (float)(cl - (double)c.c_hi);
      c.e_hi = (float)eps;
      c.e_lo = (float)(eps - (double)c.e_hi);
      const double wl[2] = {eps * std::log(1.0 / (double)q.n), eps * std::log(1.0 / (double)q.m)};
      for (int s2 = 0; s2 < 2; ++s2) {
        c.w_hi[s2] = (float)wl[s2];
        c.w_lo[s2] = (float)(wl[s2] - (double)c.w_hi[s2]);
      }
      c.alpha = (float)p.alpha[k];
      c.keep = (float)(1.0 - p.alpha[k]);
    }
    cudaError_t e = cudaMemcpy(maps, hm, sizeof(hm), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sc, hs.data(), sizeof(StepC) * hs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
    pl->probs[i] = pr;
  }
  if (rc) {
    delete pl;
    return rc;
  }
  // initial tasks: the MOM phase of every problem, largest problems first
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const double wa = (double)problems[a].n * (double)problems[a].m, wb = (double)problems[b].n * (double)problems[b].m;
    return wa != wb ? wa > wb : a < b;
  });
  for (int i : order) {
    const Prob& pr = pl->probs[i];
    for (int r = 0; r < pr.Rx; ++r) init.push_back(make_int4(i, tc::bat::kMom, r, 0));
    for (int r = 0; r < pr.Ry; ++r) init.push_back(make_int4(i, tc::bat::kMom, r, 1));
  }
  set_segments(pl);
  cudaError_t e = cudaMemcpy(pl->d_init, init.data(), sizeof(int4) * init.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_probs, pl->probs.data(), sizeof(Prob) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete pl;
    return fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = pl;
  return PROGOT_OK;
}

int progot_batch_plan_run(progot_batch_plan* pl, int32_t use_graph, progot_stream_t stream) {
  if (pl == nullptr) return fail_message(PROGOT_ERR_INVALID_ARG, "no plan");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!use_graph) {
    const cudaError_t e = enqueue_run(pl, s);
    return e == cudaSuccess ? PROGOT_OK : fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
  }
  if (pl->exec == nullptr) {
    cudaError_t e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t er = enqueue_run(pl, pl->cap);
      e = cudaStreamEndCapture(pl->cap, &pl->graph);
      if (e == cudaSuccess) e = er;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    if (e != cudaSuccess) return fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
  } else {
    count_launch();  // the graph's two kernels (init and the persistent solve)
    count_launch();
  }
  const cudaError_t e = cudaGraphLaunch(pl->exec, s);
  return e == cudaSuccess ? PROGOT_OK : fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
}

int progot_batch_plan_collect(progot_batch_plan* pl, progot_problem* problems, progot_stream_t stream) {
  if (pl == nullptr || problems == nullptr) return fail_message(PROGOT_ERR_INVALID_ARG, "no plan or problems");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  const size_t nk = (size_t)pl->count * pl->Kmax;
  std::vector<int32_t> st(nk), it(nk);
  std::vector<double> er(nk);
  int32_t fault = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&fault, pl->P.fault, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), pl->d_stat, nk * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(it.data(), pl->d_iters, nk * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(er.data(), pl->d_errs, nk * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
  if (fault) {
    for (int i = 0; i < pl->count; ++i) problems[i].status = PROGOT_ERR_TIMEOUT;
    return fail_message(PROGOT_ERR_TIMEOUT, "the persistent batched solve hit its bounded wait and aborted");
  }
  int worst = PROGOT_OK;
  for (int i = 0; i < pl->count; ++i) {
    progot_problem& p = problems[i];
    int code = PROGOT_OK;
    for (int k = 0; k < p.K; ++k) {
      const size_t o = (size_t)i * pl->Kmax + k;
      const int32_t sk = st[o];
      if (p.iters) p.iters[k] = sk < 0 ? 0 : it[o];
      if (p.errs) p.errs[k] = sk < 0 ? NAN : er[o];
      if (sk < 0 || sk == kNumeric) code = PROGOT_ERR_NUMERIC;
      else if ((sk == kMaxIter || sk == kStalled) && code == PROGOT_OK) code = PROGOT_ERR_NOT_CONVERGED;
    }
    p.status = code;
    if (code == PROGOT_ERR_NUMERIC) worst = PROGOT_ERR_NUMERIC;
    else if (code == PROGOT_ERR_NOT_CONVERGED && worst == PROGOT_OK) worst = code;
  }
  if (worst == PROGOT_ERR_NUMERIC) return fail_message(worst, "a batched problem's marginal error became non-finite");
  if (worst == PROGOT_ERR_NOT_CONVERGED) return fail_message(worst, "a batched problem did not reach its tau");
  set_last_error_message("");
  return PROGOT_OK;
}

int progot_batch_plan_set_target(progot_batch_plan* pl, int32_t target) {
  if (pl == nullptr || target < 1) return fail_message(PROGOT_ERR_INVALID_ARG, "target must be >= 1");
  pl->target = target;
  set_segments(pl);
  const cudaError_t e = cudaMemcpy(pl->d_probs, pl->probs.data(), sizeof(Prob) * pl->count, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PROGOT_OK : fail_message(PROGOT_ERR_CUDA, cudaGetErrorString(e));
}

int progot_batch_plan_autotune(progot_batch_plan* pl, int32_t* target_out, double* ms_out, progot_stream_t stream) {
  if (pl == nullptr) return fail_message(PROGOT_ERR_INVALID_ARG, "no plan");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  static const int32_t cand[] = {1, 4, 16, 64, 256};
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return fail_message(PROGOT_ERR_CUDA, "cudaEventCreate failed");
  int32_t best = pl->target;
  double best_ms = INFINITY;
  int rc = PROGOT_OK;
  for (int32_t c : cand) {
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      rc = fail_message(PROGOT_ERR_CUDA, "stream synchronisation failed");
      break;
    }
    rc = progot_batch_plan_set_target(pl, c);
    if (!rc) rc = progot_batch_plan_run(pl, 1, stream);  // warm-up
    double ms = INFINITY;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      cudaEventRecord(a, s);
      rc = progot_batch_plan_run(pl, 1, stream);
      cudaEventRecord(b, s);
      float t = 0.f;
      if (!rc && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess)
        ms = std::min(ms, (double)t);
    }
    if (rc) break;
    int32_t fault = 0;
    cudaMemcpy(&fault, pl->P.fault, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (fault) {
      rc = fail_message(PROGOT_ERR_TIMEOUT, "the persistent batched solve hit its bounded wait during tuning");
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  rc = progot_batch_plan_set_target(pl, best);
  if (rc) return rc;
  if (target_out) *target_out = best;
  if (ms_out) *ms_out = best_ms;
  return PROGOT_OK;
}

void progot_batch_plan_destroy(progot_batch_plan* pl) {
  if (pl == nullptr) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  delete pl;
}

}  // extern "C"
