// Persistent tensor-core Sinkhorn loop (Alg. 1): one cooperative launch runs the
// (f-update, g-update) iterations of a solve, the stop test included, without returning
// to the host between sweeps.
//
// Every sweep is the log-sum-exp of lse_sweep_tc: for the rows a_i of one cloud,
//   L_i = log2 sum_j 2^{t_ij},  t_ij = c (a_i . b_j) + beta_j,  c = 2 log2(e) / eps,
//   beta_j = (pot_j - |b_j|^2) log2(e) / eps,
// with both clouds centred, scaled by sqrt(c) and split into bf16 hi/lo ("bf16x3"), so
// that the tensor cores accumulate c (a_i . b_j) in float32 TMEM; one more K = 16 MMA
// (ones against the three-way bf16 split of beta_j) adds the bias, so the LSE warps read
// t_ij directly.
//
// Data flow between sweeps. The row-block finisher of a sweep (the last CTA to arrive on
// the row block) writes the new potential and the bias rows of its 128 rows into a buffer
// chosen by the iteration's parity, then publishes the row block's ready flag (the index
// of the sweep that wrote it, plus one) with a release store. The producer warp of a CTA
// loads a column tile's operands as soon as a stage is free, and its bias rows once the
// flags of the row blocks under that tile carry the expected value. So a tile waits for
// exactly the row blocks it reads, the operand products of the next sweep's first tile
// run while the previous sweep finishes, and no grid-wide barrier sits between sweeps.
//
// Stop test (Alg. 1: error <= tau, max_iter, a stall, a non-finite error). The f-update
// of iteration k measures the row-marginal error of the current (f, g) and writes
// per-row-block partials; once all row blocks of that f-update are done (a monotonic
// counter), one warp per CTA sums the partials in a fixed order and applies the test
// (every CTA computes the same state). The g-update of iteration k runs meanwhile; when
// the test stops the loop, that g-update writes nothing and the loop ends after it.
//
// Warps: 0 TMA producer (A row block, B hi/lo stages, bias rows), 1 TMEM owner and MMA
// issuer, 2-9 two LSE warpgroups (alternate tiles), 10-11 segment epilogues (publish,
// arrive, combine on the last arrival, potentials, bias rows, flags, error partials)
// and the stop decision. All waits are bounded: an mbarrier wait, a flag poll or a
// counter poll that runs past the wait limit raises the CTA's abort flag and the grid's
// fault word; every role then winds down (copies and products in flight drained, TMEM
// freed) and the host returns PROGOT_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstddef>
#include <vector>

#include "progot_internal.h"
#include "sweep_epilogue.cuh"
#include "tc_common.cuh"

namespace progot {
namespace tc {
namespace loop {

constexpr int NTHREADS = 384;
constexpr int EPI_TID0 = 320;
constexpr int TMEM_COLS = 512;
constexpr int A_TILE_BYTES = BM * KB * 2;
constexpr int A_BIAS_BYTES = BM * 32;  // 128 rows x 16 bf16 of ones (32-byte swizzle)
constexpr int BIAS_SLOTS = 2;          // bias-row ring, one slot per tile
constexpr int SEG_RING = 8;            // segments the LSE warps may be ahead of the epilogue warps

struct Shared {
  uint64_t full[8];
  uint64_t empty[8];
  uint64_t bias_full[2];    // a tile's bias rows landed (loaded once the producer saw their flags)
  uint64_t bias_empty[2];
  uint64_t tmem_full[2];
  uint64_t tmem_empty[2];
  uint64_t a_full[2];
  uint64_t a_empty[2];
  uint64_t drain;
  uint64_t seg_full[SEG_RING];   // a segment's partials are in global memory (256 LSE threads)
  uint64_t seg_empty[SEG_RING];
  uint64_t dec_full;        // one phase per iteration: the stop decision is in dec_stop
  uint32_t tmem_base;
  int32_t abort_flag;
  int32_t e_last;
  int32_t dec_stop[2];      // by iteration parity
  int32_t entry_done;
  alignas(16) SolverState st;  // the stop test's state as this CTA computed it (copied in 16-byte pieces)
  float ered[4];
  int32_t cslot[8];         // partial slots of the row block's first eight contributors (combine order)
  int32_t cbase, ccount;    // the row block's contributor list in the tables and its length
};

static_assert(offsetof(Shared, st) % 16 == 0, "the state is copied into shared memory in 16-byte pieces");
static_assert(sizeof(Shared) % 16 == 0, "the control block follows 16-byte aligned buffers");

struct Layout {
  uint32_t a0, a_stride, a_lo_off, a_bias, bias0, bias_slot, stage0, stage_bytes, b_lo_off, ctrl, total;
};

// A buffers, the ones of the bias product, the bias-row ring, then the stages (B hi, B lo).
__host__ __device__ inline Layout layout(int bn, int nkb, int split3, int stages, int a_bufs) {
  Layout L;
  uint32_t off = 0;
  L.a0 = off;
  L.a_lo_off = nkb * A_TILE_BYTES;
  L.a_stride = nkb * A_TILE_BYTES * (split3 ? 2 : 1);
  off += a_bufs * L.a_stride;
  L.a_bias = off;
  off += A_BIAS_BYTES;
  L.bias0 = off;
  L.bias_slot = (uint32_t)bn * 32;
  off += BIAS_SLOTS * L.bias_slot;
  off = (off + 1023) & ~1023u;  // 128-byte swizzled stages start on 1024-byte boundaries
  L.stage0 = off;
  L.b_lo_off = (uint32_t)bn * KB * 2;
  L.stage_bytes = L.b_lo_off * (split3 ? 2 : 1);
  off += stages * L.stage_bytes;
  L.ctrl = off;
  off += (uint32_t)sizeof(Shared);
  L.total = off + 1024;
  return L;
}

// One sweep direction: rows of A (whose potential is updated) against the columns of B.
struct Side {
  SweepParams p;            // mode = potential, role 1 (f) or 2 (g), centred norms, weights, eps
  float* out0;              // f-update: the two f buffers (state.fcur selects the current one);
  float* out1;              //   g-update: out0 = g
  __nv_bfloat16* bias_out[2];  // bias rows of A (rows x 16 bf16), by iteration parity
  uint32_t* flag_out;          // [R] ready flags of A's row blocks (sweep index + 1)
  const uint32_t* flag_in;     // ready flags of B's row blocks
  int32_t RB;                  // row blocks of B
  // float32 pieces of the potential's constants: eps ln2 = c_hi + c_lo, eps = e_hi + e_lo,
  // eps log(1 / nA) = w_hi + w_lo (uniform weights)
  float c_hi, c_lo, e_hi, e_lo, w_hi, w_lo;
  unsigned long long* cnt;  // [R] arrivals per row block (monotonic over the loop)
  unsigned long long* done; // finished row blocks (monotonic over the loop)
  float2* partial;          // [G * maxseg][2][128] (max, sum) per segment slot, LSE warpgroup and row
  // the work split (host-built): CTA c's segments segs[c maxseg + k] = (row block, first
  // tile, end tile), k < nseg[c]; row block r's contributors are the partial slots
  // cslot[cptr[r] .. cptr[r + 1]) (slot = CTA * maxseg + segment), in combine order
  const int4* segs;
  const int32_t* nseg;
  const int32_t* cptr;
  const int32_t* cslot;
  int32_t R, T;
  int64_t nA, nB;
};

struct Params {
  Side side[2];  // 0: f-update (A = X, B = Y), 1: g-update (A = Y, B = X)
  double* errpart;          // [2][R_x] row-marginal error partials by iteration parity
  SolverState* state;       // read at entry, written by CTA 0 after every stop test
  int32_t* fault;           // grid-wide abort / fault word
  unsigned long long wait_ns;
  int32_t nkb, split3, stages, a_bufs, G, maxseg;
  int32_t seq0, niter;      // iterations seq0 .. seq0 + niter - 1 of the loop
};

// ------------------------------------------------------------------ waits
__device__ __forceinline__ bool grid_aborted(const Params& P) {
  return *reinterpret_cast<volatile int32_t*>(P.fault) != 0;
}

// Bounded mbarrier wait; false on expiry (then the CTA's abort flag and the grid's
// fault word are raised) or when the CTA already aborted (unless ignore_abort).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int32_t* abort_flag,
                                         const Params& P, bool ignore_abort = false) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  const unsigned long long lim = ignore_abort ? kWaitNs : P.wait_ns;
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
                                              const Params& P, bool ignore_abort = false) {
  const bool ok = wait_bar(bar, parity, abort_flag, P, ignore_abort);
  return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Poll a monotonic counter until it reaches `target` (acquire); bounded.
__device__ __forceinline__ bool wait_counter(const unsigned long long* c, unsigned long long target,
                                             volatile int32_t* abort_flag, const Params& P) {
  if (ld_acquire_u64(c) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (ld_acquire_u64(c) >= target) return true;
    if ((i & 15) == 0) {
      if (*abort_flag || grid_aborted(P)) {
        *abort_flag = 1;
        return false;
      }
      if (global_ns() - t0 > P.wait_ns) {
        *abort_flag = 1;
        atomicExch(P.fault, 1);
        return false;
      }
    }
  }
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

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// beta split into three bf16 terms (hi, mid, lo) in the first three of 16 slots
// (-inf in the first slot for a non-finite beta).
__device__ __forceinline__ void write_bias_row(__nv_bfloat16* row16, float beta) {
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

// Poll the ready flags of row blocks [r0, r1) until each is at least `want` (acquire);
// bounded. Called by one lane.
// Whole warp: lane l polls the ready flag of row block r0 + l (r1 - r0 <= 32), so the
// flags under a tile are read in parallel rather than one after another; returns once
// every flag carries want (the lanes' acquires are ordered before the caller's later
// accesses by the warp barrier at the end), false on abort or past the wait limit.
__device__ __forceinline__ bool wait_flags_warp(const uint32_t* flags, int r0, int r1, uint32_t want,
                                                volatile int32_t* abort_flag, const Params& P) {
  const int lane = threadIdx.x & 31;
  const bool mine = r0 + lane < r1;
  bool seen = !mine || ld_acquire_u32(flags + r0 + lane) >= want;
  bool ok = true;
  if (!__all_sync(0xffffffffu, seen)) {
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
      if (!seen) seen = ld_acquire_u32(flags + r0 + lane) >= want;
      if (__all_sync(0xffffffffu, seen)) break;
      if ((i & 15) == 0) {
        int stop = 0;
        if (lane == 0) {
          if (*abort_flag || grid_aborted(P)) {
            *abort_flag = 1;
            stop = 1;
          } else if (global_ns() - t0 > P.wait_ns) {
            *abort_flag = 1;
            atomicExch(P.fault, 1);
            stop = 1;
          }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) {
          ok = false;
          break;
        }
      }
    }
  }
  __syncwarp();
  return ok;
}

// New potential of row i from its log2-sum-exp L (Alg. 1's update, the row constant
// |a_i|^2 included): f_i = eps log w_i + |a_i|^2 - eps ln2 L, in float32 with the
// product eps ln2 L folded into FMAs on a hi/lo split of eps ln2, so that |a_i|^2 - eps
// ln2 L is rounded once (GB300's float64 pipe is narrow and this is the sweep's critical
// path). L itself is float32 (relative error 2^-24 of a value ~ |a_i|^2 / (eps ln2)),
// which bounds the result's absolute error to a few float32 ulps of |a_i|^2 either way.
// Writes out[i]; returns the f-update's marginal-error term w_i |exp((f_old - f_new)/eps) - 1|
// (the exponent capped at 80, as in the per-sweep kernels) or 0 for the g-update.
__device__ __forceinline__ float loop_row_potential(const Side& Sd, int sd, int64_t i, float L, const RowIn& in,
                                                    float* out, float* val) {
  float t = fmaf(-Sd.c_hi, L, in.an);
  t = fmaf(-Sd.c_lo, L, t);
  float fnew;
  if (Sd.p.wA) {
    const float lw = __logf(in.w);
    fnew = t + fmaf(Sd.e_hi, lw, Sd.e_lo * lw);
  } else {
    fnew = (t + Sd.w_lo) + Sd.w_hi;
  }
  out[i] = fnew;
  *val = fnew;
  if (sd != 0) return 0.f;
  float dlt = (in.pot - fnew) * Sd.p.inv_eps_f;
  if (dlt > 80.f) dlt = 80.f;
  return in.w * fabsf(expm1f(dlt));
}

// Combine of two partial (max, sum) pairs in log2 units with the hardware exp2.
__device__ __forceinline__ float2 combine_fast(float2 p, float2 q) {
  const float M = fmaxf(p.x, q.x);
  if (M == -INFINITY) return make_float2(-INFINITY, 0.f);
  return make_float2(M, p.y * fast_exp2(p.x - M) + q.y * fast_exp2(q.x - M));
}

// Named barriers: 3 = epilogue warps (64), 4 + wg = LSE warpgroup wg (128).
__device__ __forceinline__ void bar_epi() { asm volatile("bar.sync 3, 64;" ::: "memory"); }
__device__ __forceinline__ void bar_wg(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(4 + wg) : "memory"); }

// Flag value published by sweep sigma (sigma = 2 k for the f-update of iteration k,
// 2 k + 1 for its g-update): sigma + 2, and sweep sigma waits for flags >= sigma + 1 on
// the other side. Flags start at 0 ("nothing published"); the host publishes the initial
// g's row blocks with 1.
__device__ __forceinline__ uint32_t flag_of(int it, int side) { return (uint32_t)(2 * it + side + 2); }
__device__ __forceinline__ uint32_t flag_wanted(int it, int side) { return (uint32_t)(2 * it + side + 1); }

__device__ __forceinline__ Seg seg_at(const Side& Sd, int c, int k, int maxseg) {
  const int4 v = __ldg(Sd.segs + (int64_t)c * maxseg + k);
  Seg sg;
  sg.r = v.x;
  sg.t0 = v.y;
  sg.t1 = v.z;
  return sg;
}


// ------------------------------------------------------------------ kernel
// NKB: the operands' K blocks when fixed at compile time (1: d <= 64, the MMA warp's issue
// path then has no runtime K loop), 0 when read from P.nkb.
template <int BN, int NKB>
__global__ void __launch_bounds__(NTHREADS, 1)
    sinkhorn_loop_tc(const __grid_constant__ CUtensorMap mXh_a, const __grid_constant__ CUtensorMap mXl_a,
                     const __grid_constant__ CUtensorMap mYh_a, const __grid_constant__ CUtensorMap mYl_a,
                     const __grid_constant__ CUtensorMap mXh_b, const __grid_constant__ CUtensorMap mXl_b,
                     const __grid_constant__ CUtensorMap mYh_b, const __grid_constant__ CUtensorMap mYl_b,
                     const __grid_constant__ CUtensorMap mXb0, const __grid_constant__ CUtensorMap mXb1,
                     const __grid_constant__ CUtensorMap mYb0, const __grid_constant__ CUtensorMap mYb1,
                     const Params P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Layout L = layout(BN, P.nkb, P.split3, P.stages, P.a_bufs);
  Shared& sh = *reinterpret_cast<Shared*>(smem + L.ctrl);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = NKB > 0 ? NKB : P.nkb;
  const int c = blockIdx.x, S = P.stages, NA = P.a_bufs;
  volatile int32_t* abort_flag = &sh.abort_flag;
  constexpr uint32_t B_TILE_BYTES = (uint32_t)BN * KB * 2, BIAS_TILE_BYTES = (uint32_t)BN * 32;
  constexpr int RB_PER_TILE = BN / BM;  // row blocks of B under one column tile
  constexpr int NC = BN / 64;           // 32-column TMEM loads of one LSE warpgroup per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int s = 0; s < BIAS_SLOTS; ++s) {
      mbar_init(&sh.bias_full[s], 1);
      mbar_init(&sh.bias_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.tmem_full[b], 1);
      mbar_init(&sh.tmem_empty[b], 8);  // every LSE warp reads its columns of each tile
      mbar_init(&sh.a_full[b], 1);
      mbar_init(&sh.a_empty[b], 1);
    }
    for (int b = 0; b < SEG_RING; ++b) {
      mbar_init(&sh.seg_full[b], 256);
      mbar_init(&sh.seg_empty[b], 64);
    }
    mbar_init(&sh.drain, 1);
    mbar_init(&sh.dec_full, 1);
    sh.abort_flag = 0;
    // the state this launch starts from (written by the initialiser or an earlier launch)
    {
      const int4* src = reinterpret_cast<const int4*>(P.state);
      int4* dst = reinterpret_cast<int4*>(&sh.st);
      for (int q = 0; q < (int)(sizeof(SolverState) / 16); ++q) dst[q] = __ldcg(src + q);
    }
    sh.entry_done = sh.st.done;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A side of the bias product: all ones (bf16 0x3F80), so that the K = 16 step adds
  // beta_hi + beta_mid + beta_lo whatever the order of the 16-byte chunks in a row
  {
    uint32_t* ab = reinterpret_cast<uint32_t*>(smem + L.a_bias);
    for (int i = threadIdx.x; i < A_BIAS_BYTES / 4; i += NTHREADS) ab[i] = 0x3F803F80u;
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
  const int it_end = sh.entry_done ? P.seq0 : P.seq0 + P.niter;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    int u = 0, ka = 0, ub = 0;  // stage units, A segments, bias tiles issued
    int s_cur = 0;              // ring position of unit u (kept without division)
    uint32_t s_par = 0;         // parity of that stage's fills so far
    bool ok = true;
    for (int it = P.seq0; it < it_end && ok; ++it) {
      if (it > P.seq0) {
        // the next f-update runs only if the stop test of iteration it - 1 let it
        warp_wait_bar(&sh.dec_full, (uint32_t)((it - 1 - P.seq0) & 1), abort_flag, P, true);
        if (sh.dec_stop[(it - 1) & 1] || *abort_flag) break;
      }
      for (int sd = 0; sd < 2 && ok; ++sd) {
        const Side& Sd = P.side[sd];
        const CUtensorMap* mAh = sd == 0 ? &mXh_a : &mYh_a;
        const CUtensorMap* mAl = sd == 0 ? &mXl_a : &mYl_a;
        const CUtensorMap* mBh = sd == 0 ? &mYh_b : &mXh_b;
        const CUtensorMap* mBl = sd == 0 ? &mYl_b : &mXl_b;
        // bias rows of B: f-update: g of the previous g-update; g-update: this iteration's f
        const CUtensorMap* mBb = sd == 0 ? ((it & 1) ? &mYb1 : &mYb0) : ((it & 1) ? &mXb1 : &mXb0);
        const uint32_t want = flag_wanted(it, sd);
        const int nseg = __ldg(Sd.nseg + c);
        for (int k = 0; k < nseg && ok; ++k, ++ka) {
          const Seg sg = seg_at(Sd, c, k, P.maxseg);
          const int ai = ka % NA;
          ok = warp_wait_bar(&sh.a_empty[ai], (uint32_t)(((ka / NA) & 1) ^ 1), abort_flag, P);
          if (!ok) break;
          unsigned char* abuf = smem + L.a0 + ai * L.a_stride;
          if (elect_one()) {
            mbar_arrive_expect_tx(&sh.a_full[ai], L.a_stride);
            for (int kb = 0; kb < nkb; ++kb) {
              tma_load_2d(abuf + kb * A_TILE_BYTES, mAh, &sh.a_full[ai], kb * KB, sg.r * BM);
              if (P.split3) tma_load_2d(abuf + L.a_lo_off + kb * A_TILE_BYTES, mAl, &sh.a_full[ai], kb * KB, sg.r * BM);
            }
          }
          __syncwarp();
          for (int t = sg.t0; t < sg.t1 && ok; ++t) {
            for (int kb = 0; kb < nkb; ++kb, ++u) {
              const int s = s_cur;
              ok = warp_wait_bar(&sh.empty[s], s_par ^ 1u, abort_flag, P);
              if (!ok) break;
              if (++s_cur == S) {
                s_cur = 0;
                s_par ^= 1u;
              }
              unsigned char* st = smem + L.stage0 + s * L.stage_bytes;
              if (elect_one()) {
                mbar_arrive_expect_tx(&sh.full[s], B_TILE_BYTES * (P.split3 ? 2u : 1u));
                tma_load_2d(st, mBh, &sh.full[s], kb * KB, t * BN);
                if (P.split3) tma_load_2d(st + L.b_lo_off, mBl, &sh.full[s], kb * KB, t * BN);
              }
              __syncwarp();
            }
            if (!ok) break;
            // the tile's bias rows, once the row blocks of B under it are ready
            const int bs = ub % BIAS_SLOTS;
            ok = warp_wait_bar(&sh.bias_empty[bs], (uint32_t)(((ub / BIAS_SLOTS) & 1) ^ 1), abort_flag, P);
            if (!ok) break;
            const int r0 = t * RB_PER_TILE, r1 = min(Sd.RB, r0 + RB_PER_TILE);
            ok = wait_flags_warp(Sd.flag_in, r0, r1, want, abort_flag, P);
            if (!ok) break;
            if (lane == 0) {
              mbar_arrive_expect_tx(&sh.bias_full[bs], BIAS_TILE_BYTES);
              asm volatile("fence.proxy.async.global;" ::: "memory");
              tma_load_2d(smem + L.bias0 + bs * L.bias_slot, mBb, &sh.bias_full[bs], 0, t * BN);
            }
            __syncwarp();
            ++ub;
          }
        }
      }
    }
    // drain this CTA's own copies still in flight before shared memory is released
    if (!ok || *abort_flag) {
      for (int k = max(0, ka - NA); k < ka; ++k)
        warp_wait_bar(&sh.a_full[k % NA], (uint32_t)((k / NA) & 1), abort_flag, P, true);
      for (int v = max(0, u - S); v < u; ++v) warp_wait_bar(&sh.full[v % S], (uint32_t)((v / S) & 1), abort_flag, P, true);
      for (int v = max(0, ub - BIAS_SLOTS); v < ub; ++v)
        warp_wait_bar(&sh.bias_full[v % BIAS_SLOTS], (uint32_t)((v / BIAS_SLOTS) & 1), abort_flag, P, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // One thread runs the whole issue loop (a product is issued by a single thread): no
    // per-wait votes or elections between tiles, whose bookkeeping sits between one
    // tile's last product and the next tile's first; the other lanes wait at the end.
    if (lane == 0) {
      const uint64_t abias = desc_sw32(smem_u32(smem + L.a_bias));
      bool ok = true;
      int tl = 0, ka = 0;
      int s_cur = 0;          // stage of the next B block (ring position, kept without division)
      uint32_t s_par = 0;     // the parity of its fill
      for (int it = P.seq0; it < it_end && ok; ++it) {
        if (it > P.seq0) {
          wait_bar(&sh.dec_full, (uint32_t)((it - 1 - P.seq0) & 1), abort_flag, P, true);
          if (sh.dec_stop[(it - 1) & 1] || *abort_flag) break;
        }
        for (int sd = 0; sd < 2 && ok; ++sd) {
          const Side& Sd = P.side[sd];
          const int nseg = __ldg(Sd.nseg + c);
          for (int k = 0; k < nseg && ok; ++k, ++ka) {
            const Seg sg = seg_at(Sd, c, k, P.maxseg);
            const int ai = ka % NA;
            ok = wait_bar(&sh.a_full[ai], (uint32_t)((ka / NA) & 1), abort_flag, P);
            if (!ok) break;
            tc_fence_after();
            const uint32_t a_hi = smem_u32(smem + L.a0 + ai * L.a_stride);
            const uint32_t a_lo = a_hi + L.a_lo_off;
            for (int t = sg.t0; t < sg.t1 && ok; ++t, ++tl) {
              const int b = tl & 1;
              ok = wait_bar(&sh.tmem_empty[b], (uint32_t)(((tl >> 1) & 1) ^ 1), abort_flag, P);
              if (!ok) break;
              tc_fence_after();
              const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
              for (int kb = 0; kb < nkb; ++kb) {
                const int s = s_cur;
                ok = wait_bar(&sh.full[s], s_par, abort_flag, P);
                if (++s_cur == S) {
                  s_cur = 0;
                  s_par ^= 1u;
                }
                if (!ok) break;
                tc_fence_after();
                const uint32_t st = smem_u32(smem + L.stage0 + s * L.stage_bytes);
                const uint64_t bh = desc_sw128(st), bl = desc_sw128(st + L.b_lo_off);
                const uint64_t ah = desc_sw128(a_hi + kb * A_TILE_BYTES), al = desc_sw128(a_lo + kb * A_TILE_BYTES);
#pragma unroll
                for (int kk = 0; kk < KB / 16; ++kk) {
                  // +32 bytes per K = 16 step inside the 128-byte swizzle atom (encoded >> 4)
                  const uint64_t adv = (uint64_t)(kk * 2);
                  umma<BN>(d_tmem, ah + adv, bh + adv, (kb > 0 || kk > 0) ? 1u : 0u);
                  if (P.split3) {
                    umma<BN>(d_tmem, ah + adv, bl + adv, 1u);
                    umma<BN>(d_tmem, al + adv, bh + adv, 1u);
                  }
                }
                umma_commit(&sh.empty[s]);
              }
              if (!ok) break;
              // bias: t_ij = c (a_i . b_j) + beta_j, once the producer has the row blocks' bias rows
              const int bs = tl % BIAS_SLOTS;  // one bias slot per tile, in tile order
              ok = wait_bar(&sh.bias_full[bs], (uint32_t)((tl / BIAS_SLOTS) & 1), abort_flag, P);
              if (!ok) break;
              tc_fence_after();
              umma<BN>(d_tmem, abias, desc_sw32(smem_u32(smem + L.bias0 + bs * L.bias_slot)), 1u);
              umma_commit(&sh.bias_empty[bs]);
              umma_commit(&sh.tmem_full[b]);
            }
            if (!ok) break;
            umma_commit(&sh.a_empty[ai]);
          }
        }
      }
      umma_commit(&sh.drain);
      wait_bar(&sh.drain, 0, abort_flag, P, true);
    }
    __syncwarp();
  } else if (threadIdx.x < EPI_TID0) {
    // ------------------------------------------------------------ LSE warps
    const int wg = (warp - 2) >> 2;
    const int quarter = warp & 3;
    const int row_local = quarter * 32 + lane;
    int tl = 0, kseg = 0;
    bool dead = false;
    for (int it = P.seq0; it < it_end; ++it) {
      if (it > P.seq0) {
        // every LSE warp reads the same decision after the same wait (the decider always
        // arrives), so all of them leave at the same iteration
        wait_bar(&sh.dec_full, (uint32_t)((it - 1 - P.seq0) & 1), abort_flag, P, true);
        __syncwarp();
        if (sh.dec_stop[(it - 1) & 1]) break;
      }
      for (int sd = 0; sd < 2; ++sd) {
        const Side& Sd = P.side[sd];
        const int nseg = __ldg(Sd.nseg + c);
        for (int k = 0; k < nseg; ++k, ++kseg) {
          const Seg sg = seg_at(Sd, c, k, P.maxseg);
          float m_run = -INFINITY, s_run = 0.f;
          for (int t = sg.t0; t < sg.t1; ++t, ++tl) {
            // both warpgroups take every tile, warpgroup wg its columns wg BN / 2 ..: the
            // accumulator goes back to the MMA warp as soon as both halves are in
            // registers, and the exponentials overlap the next tile's products
            const uint32_t ph = (uint32_t)((tl >> 1) & 1);
            if (dead) continue;
            int okv = 0;
            if (lane == 0) okv = wait_bar(&sh.tmem_full[tl & 1], ph, abort_flag, P) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, okv, 0) == 0) {
              dead = true;
              continue;
            }
            __syncwarp();
            tc_fence_after();
            const uint32_t taddr =
                tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((tl & 1) * BN + wg * (BN / 2));
            float v[NC][32];
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) PROGOT_TMEM_LD32(taddr + 32 * cc, v[cc]);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.tmem_empty[tl & 1]);
            float mx[2 * NC];
#pragma unroll
            for (int q = 0; q < 2 * NC; ++q) mx[q] = v[q >> 1][(q & 1) * 16];
#pragma unroll
            for (int cc = 0; cc < NC; ++cc)
#pragma unroll
              for (int i = 1; i < 16; i += 2) {
                mx[cc * 2] = max3(mx[cc * 2], v[cc][i], v[cc][i + 1 < 16 ? i + 1 : i]);
                mx[cc * 2 + 1] = max3(mx[cc * 2 + 1], v[cc][16 + i], v[cc][16 + (i + 1 < 16 ? i + 1 : i)]);
              }
            float tmax = mx[0];
#pragma unroll
            for (int q = 1; q < 2 * NC; ++q) tmax = fmaxf(tmax, mx[q]);
            const float mnew = fmaxf(m_run, tmax);
            if (mnew != -INFINITY) {
              const uint64_t negm = pack2(-mnew, -mnew);
              uint64_t acc[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[q] = 0ull;
#pragma unroll
              for (int cc = 0; cc < NC; ++cc)
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
          // both warpgroups write their part of the segment to its partial slot (the row
          // block's finisher merges them) and count the segment as handed over, so that
          // neither waits for the other and the epilogue warps only count arrivals
          const int sl = kseg % SEG_RING;
          if ((int64_t)sg.r * BM + row_local < Sd.nA)
            Sd.partial[(((int64_t)c * P.maxseg + k) * 2 + wg) * BM + row_local] = make_float2(m_run, s_run);
          wait_bar(&sh.seg_empty[sl], (uint32_t)(((kseg / SEG_RING) & 1) ^ 1), abort_flag, P);
          mbar_arrive(&sh.seg_full[sl]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue warps and stop decision
    const int etid = threadIdx.x - EPI_TID0;  // 0..63
    int kseg = 0;
    // ---- stop test of iteration it (warp 10), once every row block of the f-update is done
    auto decide = [&](int it) {
      if (etid < 32) {
        bool okc = true;
        if (etid == 0) {
          okc = wait_counter(P.side[1].done, (unsigned long long)it * (unsigned long long)P.side[1].R, abort_flag,
                             P) &&
                wait_counter(P.side[0].done, (unsigned long long)(it + 1) * (unsigned long long)P.side[0].R,
                             abort_flag, P);
          __threadfence();
        }
        okc = __shfl_sync(0xffffffffu, okc ? 1 : 0, 0) != 0;
        __syncwarp();  // the other lanes' loads below follow lane 0's acquire
        const double err =
            okc ? sum_errpart_warp(P.errpart + (int64_t)(it & 1) * P.side[0].R, P.side[0].R) : (double)NAN;
        if (etid == 0) {
          SolverState st = sh.st;
          if (okc) {
            f_update_transition(st, err, P.side[0].p);
          } else {
            st.done = 1;
            st.status = kNumeric;  // reported as PROGOT_ERR_TIMEOUT by the host (fault word)
          }
          sh.st = st;
          sh.dec_stop[it & 1] = st.done;
          if (c == 0) *P.state = st;
          mbar_arrive(&sh.dec_full);
        }
      }
      bar_epi();  // both epilogue warps see the decision
    };

    for (int it = P.seq0; it < it_end; ++it) {
      for (int sd = 0; sd < 2; ++sd) {
        const Side& Sd = P.side[sd];
        const SweepParams& p = Sd.p;
        const int nseg = __ldg(Sd.nseg + c);
        const int fcur = sh.st.fcur;
        const float* pot_cur = (sd == 0) ? (fcur == 0 ? Sd.out0 : Sd.out1) : nullptr;
        float* out = (sd == 0) ? (fcur == 0 ? Sd.out1 : Sd.out0) : Sd.out0;
        __nv_bfloat16* bout = Sd.bias_out[sd == 0 ? (it & 1) : ((it + 1) & 1)];
        const uint32_t flag = flag_of(it, sd);
        for (int k = 0; k < nseg; ++k, ++kseg) {
          const Seg sg = seg_at(Sd, c, k, P.maxseg);
          const int sl = kseg % SEG_RING;
          // the rows' epilogue inputs do not depend on the sweep: load them while the LSE
          // warps finish the segment
          RowIn rin[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int64_t i = (int64_t)sg.r * BM + etid + 64 * h;
            rin[h].an = 0.f;
            rin[h].pot = 0.f;
            rin[h].w = 0.f;
            if (i < Sd.nA) rin[h] = row_inputs(p, i, pot_cur);
          }
          // the row block's contributors and their partial slots, once per segment, from the
          // split's tables; the previous segment's readers passed the barrier at its end
          if (etid < 8) {
            const int p0 = __ldg(Sd.cptr + sg.r), p1 = __ldg(Sd.cptr + sg.r + 1);
            if (p0 + etid < p1) sh.cslot[etid] = __ldg(Sd.cslot + p0 + etid);
            if (etid == 0) {
              sh.cbase = p0;
              sh.ccount = p1 - p0;
            }
          }
          // the segment's partials are in global memory once the LSE warps arrived (their
          // stores precede the arrival; the release of the arrival atomic below covers them)
          wait_bar(&sh.seg_full[sl], (uint32_t)((kseg / SEG_RING) & 1), abort_flag, P);
          mbar_arrive(&sh.seg_empty[sl]);
          if (etid == 0) {
            const unsigned long long prev = atom_add_acq_rel_u64(&Sd.cnt[sg.r], 1ull);
            sh.e_last = (prev + 1 == (unsigned long long)(it + 1) * (unsigned long long)sh.ccount);
          }
          bar_epi();
          const int ncc = sh.ccount;
          if (sh.e_last) {
            const bool skip = sd == 1 && sh.st.done != 0;  // the stop test ended the loop: g stays
            // the contributors' partials of both rows (each contributor: the two LSE
            // warpgroups' parts, merged as one segment), four contributors' loads issued
            // together, combined in the tables' order
            float2 acc[2];
            acc[0] = make_float2(-INFINITY, 0.f);
            acc[1] = make_float2(-INFINITY, 0.f);
            for (int q0 = 0; q0 < ncc; q0 += 4) {
              float2 pa[2][4], pb[2][4];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int q = q0 + j;
                if (q < ncc) {
                  const int slot = q < 8 ? sh.cslot[q] : __ldg(Sd.cslot + sh.cbase + q);
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    const int rl = etid + 64 * h;
                    pa[h][j] = __ldcg(&Sd.partial[((int64_t)slot * 2 + 0) * BM + rl]);
                    pb[h][j] = __ldcg(&Sd.partial[((int64_t)slot * 2 + 1) * BM + rl]);
                  }
                }
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (q0 + j < ncc) {
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    const float2 mrg = lse_combine(pa[h][j], pb[h][j]);
                    const float2 v = (isnan(pa[h][j].y) || isnan(pb[h][j].y)) ? make_float2(NAN, NAN) : mrg;
                    acc[h] = combine_fast(acc[h], v);
                  }
                }
              }
            }
            float e[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              e[h] = 0.f;
              const int rl = etid + 64 * h;
              const int64_t i = (int64_t)sg.r * BM + rl;
              if (i < Sd.nA) {
                const float Lr = acc[h].x + __log2f(acc[h].y);
                if (!skip) {
                  float val;
                  e[h] = loop_row_potential(Sd, sd, i, Lr, rin[h], out, &val);
                  write_bias_row(bout + i * 16, (val - rin[h].an) * p.bscale);
                }
              }
            }
            if (sd == 0) {
              // row-block sum of the error terms in a fixed order
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
              if (sd == 0)
                P.errpart[(int64_t)(it & 1) * Sd.R + sg.r] =
                    (double)((sh.ered[0] + sh.ered[1]) + (sh.ered[2] + sh.ered[3]));
              // the bias rows are read by TMA (async proxy) once the flag is seen
              asm volatile("fence.proxy.async.global;" ::: "memory");
              if (!skip) st_release_u32(Sd.flag_out + sg.r, flag);
              red_add_release_u64(Sd.done, 1ull);
            }
          }
          bar_epi();
        }
        if (sd == 0) decide(it);
      }
      if (sh.st.done) break;
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

__global__ void fill_u32_kernel(uint32_t* __restrict__ p, int64_t n, uint32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace loop
}  // namespace tc

// ---------------------------------------------------------------- host side
// Pipeline shape of the persistent loop: two resident A buffers and as many B stages
// (2..8) as fit in 227 KB; 0 stages when no shape fits (the per-sweep kernel serves it).
static void loop_shape(int bn, int nkb, int split3, int* stages, int* a_bufs) {
  *stages = 0;
  *a_bufs = 2;
  for (int na = 2; na >= 1; --na) {
    int best = 0;
    for (int s = 2; s <= 8; ++s)
      if (tc::loop::layout(bn, nkb, split3, s, na).total <= 227 * 1024) best = s;
    if (best >= 2) {
      *stages = best;
      *a_bufs = na;
      return;
    }
  }
}

cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  tc::loop::fill_u32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
  count_launch();
  return cudaGetLastError();
}

bool loop_tc_supported(int bn, int nkb, int split3) {
  int s, na;
  loop_shape(bn, nkb, split3, &s, &na);
  return s >= 2 && (bn == 128 || bn == 256);
}

// ---- work split of the loop (host-built tables): the (row block, column tile) grid of
// a sweep cut over the CTAs as in the per-update kernel (tc::Split), laid out for the
// kernel as per-CTA segment lists and per-row-block contributor lists (in CTA order, the
// order of the combine), so that no 64-bit division of the split runs on the GPU.
struct SideTables {
  std::vector<int4> segs;
  std::vector<int32_t> nseg, cptr, cslot;
  int maxseg = 0;
};

// ms_force: segment stride of the tables (the larger maxseg of both sides), 0 = own.
static void side_tables(int R, int T, int G, SideTables* out, int ms_force = 0) {
  const tc::Split sp = tc::make_split(R, T, G);
  int ms = 1;
  for (int c = 0; c < G; ++c) ms = std::max(ms, tc::num_segments(sp, c));
  out->maxseg = ms;
  if (ms_force >= ms) ms = ms_force;
  out->segs.assign((size_t)G * ms, make_int4(0, 0, 0, 0));
  out->nseg.assign((size_t)G, 0);
  std::vector<std::vector<int32_t>> by_row((size_t)R);
  for (int c = 0; c < G; ++c) {
    const int ns = tc::num_segments(sp, c);
    out->nseg[c] = ns;
    for (int k = 0; k < ns; ++k) {
      const tc::Seg sg = tc::segment(sp, c, k);
      out->segs[(size_t)c * ms + k] = make_int4(sg.r, sg.t0, sg.t1, 0);
      by_row[sg.r].push_back(c * ms + k);  // CTAs in increasing order
    }
  }
  out->cptr.assign((size_t)R + 1, 0);
  out->cslot.clear();
  for (int r = 0; r < R; ++r) {
    out->cptr[r + 1] = out->cptr[r] + (int32_t)by_row[r].size();
    out->cslot.insert(out->cslot.end(), by_row[r].begin(), by_row[r].end());
  }
}

void loop_tc_plan(int64_t n, int64_t m, int bn, int sms, int* G, int* maxseg) {
  const int64_t Rx = (n + tc::BM - 1) / tc::BM, Ry = (m + tc::BM - 1) / tc::BM;
  const int64_t Tx = (n + bn - 1) / bn, Ty = (m + bn - 1) / bn;
  const int g = (int)std::min<int64_t>(std::min<int64_t>(Rx * Ty, Ry * Tx), sms);
  SideTables a, b;
  side_tables((int)Rx, (int)Ty, g, &a);
  side_tables((int)Ry, (int)Tx, g, &b);
  *G = g;
  *maxseg = std::max(a.maxseg, b.maxseg);
}

size_t loop_tc_smem(int bn, int nkb, int split3) {
  int s, na;
  loop_shape(bn, nkb, split3, &s, &na);
  return tc::loop::layout(bn, nkb, split3, s, na).total;
}

template <int BN, int NKB>
static cudaError_t launch_loop(const tc::loop::Params& P, size_t smem, const void* const* maps, cudaStream_t stream) {
  static thread_local size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(tc::loop::sinkhorn_loop_tc<BN, NKB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.G);
  cfg.blockDim = dim3(tc::loop::NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // CTAs wait on one another: all must be resident
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const CUtensorMap* m[12];
  for (int q = 0; q < 12; ++q) m[q] = reinterpret_cast<const CUtensorMap*>(maps[q]);
  return cudaLaunchKernelEx(&cfg, tc::loop::sinkhorn_loop_tc<BN, NKB>, *m[0], *m[1], *m[2], *m[3], *m[4], *m[5],
                            *m[6], *m[7], *m[8], *m[9], *m[10], *m[11], P);
}

cudaError_t launch_sinkhorn_loop_tc(const LoopLaunch& Lq, cudaStream_t stream) {
  int stages, a_bufs;
  loop_shape(Lq.bn, Lq.nkb, Lq.split3, &stages, &a_bufs);
  if (stages < 2 || (Lq.bn != 128 && Lq.bn != 256)) return cudaErrorInvalidValue;
  tc::loop::Params P;
  memset(&P, 0, sizeof(P));
  for (int sd = 0; sd < 2; ++sd) {
    const LoopSideLaunch& s = Lq.side[sd];
    tc::loop::Side& d = P.side[sd];
    d.p = s.p;
    d.out0 = s.out0;
    d.out1 = s.out1;
    d.bias_out[0] = (__nv_bfloat16*)s.bias_out[0];
    d.bias_out[1] = (__nv_bfloat16*)s.bias_out[1];
    d.flag_out = s.flag_out;
    d.flag_in = s.flag_in;
    d.cnt = s.cnt;
    d.done = s.done;
    d.partial = s.partial;
    d.nA = s.p.nA;
    d.nB = s.p.nB;
    d.R = (int)((s.p.nA + tc::BM - 1) / tc::BM);
    d.T = (int)((s.p.nB + Lq.bn - 1) / Lq.bn);
    d.RB = (int)((s.p.nB + tc::BM - 1) / tc::BM);
    const double cl = s.p.eps * kLn2, wl = s.p.eps * s.p.log_w_uniform;
    d.c_hi = (float)cl;
    d.c_lo = (float)(cl - (double)d.c_hi);
    d.e_hi = (float)s.p.eps;
    d.e_lo = (float)(s.p.eps - (double)d.e_hi);
    d.w_hi = (float)wl;
    d.w_lo = (float)(wl - (double)d.w_hi);
  }
  // the work split's tables (the same as loop_tc_plan's), copied to the workspace
  {
    SideTables tab[2];
    for (int sd = 0; sd < 2; ++sd) {
      side_tables(P.side[sd].R, P.side[sd].T, Lq.G, &tab[sd], Lq.maxseg);
      if (tab[sd].maxseg > Lq.maxseg) return cudaErrorInvalidValue;
      const LoopSideLaunch& ls = Lq.side[sd];
      if ((int64_t)tab[sd].segs.size() > ls.table_slots || (int64_t)tab[sd].cslot.size() > ls.table_slots)
        return cudaErrorInvalidValue;
      cudaError_t e = cudaMemcpyAsync(ls.segs, tab[sd].segs.data(), sizeof(int4) * tab[sd].segs.size(),
                                      cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ls.nseg, tab[sd].nseg.data(), sizeof(int32_t) * tab[sd].nseg.size(),
                            cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ls.cptr, tab[sd].cptr.data(), sizeof(int32_t) * tab[sd].cptr.size(),
                            cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ls.cslot, tab[sd].cslot.data(), sizeof(int32_t) * tab[sd].cslot.size(),
                            cudaMemcpyHostToDevice, stream);
      if (e != cudaSuccess) return e;
      P.side[sd].segs = reinterpret_cast<const int4*>(ls.segs);
      P.side[sd].nseg = ls.nseg;
      P.side[sd].cptr = ls.cptr;
      P.side[sd].cslot = ls.cslot;
    }
  }
  P.errpart = Lq.errpart;
  P.state = Lq.state;
  P.fault = Lq.fault;
  P.wait_ns = Lq.wait_ns;
  P.nkb = Lq.nkb;
  P.split3 = Lq.split3;
  P.stages = stages;
  P.a_bufs = a_bufs;
  P.G = Lq.G;
  P.maxseg = Lq.maxseg;
  P.seq0 = Lq.seq0;
  P.niter = Lq.niter;
  const size_t smem = tc::loop::layout(Lq.bn, Lq.nkb, Lq.split3, stages, a_bufs).total;
  cudaError_t e = Lq.bn == 128 ? launch_loop<128, 0>(P, smem, Lq.maps, stream)
                  : Lq.nkb == 1 ? launch_loop<256, 1>(P, smem, Lq.maps, stream)
                                : launch_loop<256, 0>(P, smem, Lq.maps, stream);
  count_launch();
  return e;
}

}  // namespace progot
