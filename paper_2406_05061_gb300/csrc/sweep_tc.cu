// Tensor-core (tcgen05) log-sum-exp sweep of the ProgOT hot path.
//
// For every row a_i of A: L_i = log2 sum_j 2^{t_ij},
//   t_ij = c (a_i . b_j) + beta_j,   c = 2 log2(e) / eps,   beta_j = (potB_j - |b_j|^2) log2(e) / eps,
// the soft-min of Sec. 2 (Alg. 1's f- or g-update) with the row constant |a_i|^2 factored out.
//
// Both operands arrive pre-scaled by sqrt(c) and split into bf16 hi/lo parts
// (v = hi + lo to ~16 bits), K-padded to a multiple of 64, so that the tensor cores
// accumulate t_ij - beta_j = sum_k (ah bh + ah bl + al bh) in float32 (3 products per
// element: "bf16x3"), or ah bh only ("bf16"). beta_j enters the same accumulator as
// one more K = 16 MMA step: the A side holds ones, the B side [beta_hi, beta_mid,
// beta_lo, 0, ...] (a three-way bf16 split of the float32 beta), so TMEM holds t_ij
// directly and the cost matrix is never formed.
//
// Persistent CTAs of 12 warps; each owns a contiguous range of (128-row block,
// BN-column tile) work units, cut at row-block boundaries into segments:
//   warp 0: TMA producer (the A operand of a segment, B hi/lo and bias-row stages);
//   warp 1: TMEM owner and MMA issuer (one lane), two BN-column fp32 accumulators so
//           that the MMAs of tile t + 1 overlap the LSE of tile t;
//   warps 2-9: two LSE warpgroups taking alternate tiles, one TMEM lane (= one row)
//           per thread; tcgen05.ld the tile's values and fold them into an online
//           (max, sum) in log2 units;
//   warps 10-11: epilogue of the segments that end before the CTA's last one, so that
//           the LSE warps go straight on to the next row block.
// Column splits are combined in CTA order by the last CTA to finish a row block, whose
// epilogue is shared with the float32 kernel (Sinkhorn update + marginal error,
// raw L, or coupling marginal). Every mbarrier wait is bounded (2 s of global time);
// on expiry the CTA records a fault, drains its own TMA and MMA work, frees TMEM and
// produces NaN partials so the host sees an error instead of a hang.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "progot_internal.h"
#include "sweep_epilogue.cuh"
#include "tc_common.cuh"

namespace progot {
namespace tc {

constexpr int NTHREADS = 384;    // 12 warps: producer, MMA, two LSE warpgroups, two epilogue warps
constexpr int EPI_TID0 = 320;    // first thread of the epilogue warps
constexpr int TMEM_COLS = 512;   // two accumulators of up to 256 columns
constexpr int A_TILE_BYTES = BM * KB * 2;    // 16 KB: 128 rows x 64 bf16
constexpr int A_BIAS_BYTES = BM * 32;        // 4 KB: 128 rows x 16 bf16 (32-byte swizzle)
// Per column-tile width BN (128 or 256, a template parameter of the kernel):
//   B operand tile BN rows x 64 bf16, bias tile BN rows x 16 bf16.

struct TcShared {
  uint64_t full[8];       // operand tiles of a stage landed
  uint64_t bias_full[8];  // the stage's bias rows landed (plain arrival for stages without bias)
  uint64_t empty[8];
  uint64_t tmem_full[2];
  uint64_t tmem_empty[2];
  uint64_t a_full[2];
  uint64_t a_empty[2];
  uint64_t drain;
  uint64_t seg_full[2];   // a segment's merged (max, sum) handed to the epilogue warps
  uint64_t seg_empty[2];  // ... and read by them
  uint32_t tmem_base;
  int32_t abort_flag;
  int32_t s_last, s_fin;  // segment epilogue flags of LSE warpgroup 0
  int32_t e_last, e_fin;  // ... and of the epilogue warps
  int32_t stop;           // the previous sweep already stopped the Sinkhorn loop
  float red[4];
  float ered[4];
  float2 ms[2][128];   // (max, sum) of LSE warpgroup 1 by segment parity, merged by warpgroup 0
  float2 seg[2][128];  // merged (max, sum) of a handed-off segment, by segment parity
};


// Parameters beyond SweepParams. The CTAs are persistent and split the (row block,
// column tile) grid as tc::Split describes (whole row blocks in bands of G, then a
// contiguous split of the rest), each CTA's share cut into segments of one row block;
// a segment's (max, sum) partial goes to slot (c * maxseg + k), k = its index within
// the CTA.
struct TcParams {
  SweepParams p;
  int32_t nkb;        // K blocks of 64
  int32_t split3;     // 1: bf16x3 (hi and lo operands), 0: bf16 (hi only)
  int32_t stages;     // B pipeline depth (units of one K block of one tile)
  int32_t a_bufs;     // 1 or 2 resident A-operand buffers, or 0: A K blocks stream with B
  int32_t G;          // CTAs
  int32_t T;          // column tiles per row block
  int32_t R;          // row blocks
  int32_t maxseg;     // partial slots per CTA
  int32_t* fault;     // set to 1 by a CTA whose bounded wait expired
  __nv_bfloat16* bias_out;  // potential mode: beta rows of the updated side (rows x 16), or nullptr
};

struct SmemLayout {
  uint32_t a0, a_stride, a_lo_off, a_bias, stage0, stage_bytes, b_lo_off, bias_off, a_stage_off, ctrl, total;
};

__host__ __device__ inline SmemLayout smem_layout(int bn, int nkb, int split3, int stages, int a_bufs) {
  SmemLayout L;
  const uint32_t b_tile = (uint32_t)bn * KB * 2, bias_tile = (uint32_t)bn * 32;
  uint32_t off = 0;
  L.a0 = off;
  L.a_lo_off = nkb * A_TILE_BYTES;
  L.a_stride = nkb * A_TILE_BYTES * (split3 ? 2 : 1);
  off += a_bufs * L.a_stride;
  L.a_bias = off;
  off += A_BIAS_BYTES;
  L.stage0 = off;
  L.b_lo_off = b_tile;
  L.bias_off = b_tile * (split3 ? 2 : 1);
  // streamed A (a_bufs = 0): the A K block (hi, then lo) follows the bias rows in the stage
  L.a_stage_off = L.bias_off + bias_tile;
  L.stage_bytes = L.a_stage_off + (a_bufs == 0 ? A_TILE_BYTES * (split3 ? 2u : 1u) : 0u);
  off += stages * L.stage_bytes;
  L.ctrl = off;
  off += sizeof(TcShared);
  L.total = off + 1024;  // alignment slack for the dynamic base
  return L;
}


// Named barriers: 1 = both LSE warpgroups (256 threads), 2 = LSE warpgroup 0 (128),
// 3 = the epilogue warps (64).
__device__ __forceinline__ void lse_bar_all() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
template <int NT>
__device__ __forceinline__ void seg_bar() {
  static_assert(NT == 128 || NT == 64, "segment epilogue groups");
  if (NT == 128)
    asm volatile("bar.sync 2, 128;" ::: "memory");
  else
    asm volatile("bar.sync 3, 64;" ::: "memory");
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

// beta_j split into three bf16 terms (hi, mid, lo) in the first three of 16 slots.
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

static_assert(sizeof(SolverState) % 16 == 0, "the solver state is loaded in 16-byte pieces");

// The Sinkhorn state this sweep runs under, read from L2 after griddepcontrol.wait; called
// by a whole warp. For the g-update of a lagged loop it is the f-update's stop test
// applied to state[seq & 1] with the f-update's error partials (every warp that needs
// it computes the same value from the same loads in the same order).
__device__ __forceinline__ SolverState sweep_state(const SweepParams& p) {
  SolverState st;
  const int4* src = reinterpret_cast<const int4*>(p.state + (p.lag ? (p.seq & 1) : 0));
  int4* dst = reinterpret_cast<int4*>(&st);
#pragma unroll
  for (int q = 0; q < (int)(sizeof(SolverState) / 16); ++q) dst[q] = __ldcg(src + q);
  if (p.lag && p.role == 2) {
    const double err = sum_errpart_warp(p.errpart, (int)((p.nB + BM - 1) / BM));
    if (!st.done) f_update_transition(st, err, p);
  }
  return st;
}

// Epilogue of segment k of CTA c, run by NT threads (LSE warpgroup 0 with NT = 128 for
// the CTA's last segment, the epilogue warps with NT = 64 for the others); thread tid
// owns rows row0 + NT h of the row block. Publishes the segment's (max, sum) partials,
// arrives on the row block's counter and, on the last arrival, combines the row
// block's partials in CTA order, writes the rows' epilogue (and bias rows) and the
// block's error term, summed in the same float32 tree for either NT (a shuffle sum per
// 32 rows, then (q0 + q1) + (q2 + q3)); the last row block of the sweep finishes it.
// The g-update of a Sinkhorn loop (role 2) measures no error and changes no solver
// state, so its row blocks skip the sweep-level arrival altogether.
template <int NT>
__device__ __forceinline__ void segment_epilogue(const TcParams& tp, int c, int k, const Seg& sg, const Split& sp,
                                                 int tid, int row0, const float2 (&mv)[BM / NT], int fcur,
                                                 int32_t& s_last, int32_t& s_fin, float* red) {
  constexpr int RPT = BM / NT;
  const SweepParams& p = tp.p;
  const float* potA_cur = p.potA_old;
  float* out_target = p.out;
  if (p.role == 1 || p.role == 3) {
    potA_cur = (fcur == 0) ? p.out : p.out_alt;
    out_target = (fcur == 0) ? p.out_alt : p.out;
  }
  // the rows' epilogue inputs are loaded now, overlapping the arrival below
  RowIn rin[RPT];
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    const int rl = row0 + NT * h;
    const int64_t i = (int64_t)sg.r * BM + rl;
    rin[h].an = 0.f;
    rin[h].pot = 0.f;
    rin[h].w = 0.f;
    if (i < p.nA) {
      p.partial[((int64_t)c * tp.maxseg + k) * BM + rl] = mv[h];
      rin[h] = row_inputs(p, i, potA_cur);
    }
  }
  int c_first, c_last;
  contributors(sp, sg.r, &c_first, &c_last);
  seg_bar<NT>();  // the partial stores of all rows happen before the arrival below
  if (tid == 0) {
    const unsigned prev = atomic_add_acq_rel_gpu(&p.cnt[sg.r], 1u);
    s_last = (prev == (unsigned)(c_last - c_first));
  }
  seg_bar<NT>();  // ... and the other CTAs' partials are visible after it
  if (!s_last) return;
  float e[RPT];
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    e[h] = 0.f;
    const int rl = row0 + NT * h;
    const int64_t i = (int64_t)sg.r * BM + rl;
    if (i < p.nA) {
      // issue the partial loads back to back, then combine them in CTA order
      constexpr int kMaxC = 8;
      const int nc = c_last - c_first + 1;
      float2 pv[kMaxC];
#pragma unroll
      for (int q = 0; q < kMaxC; ++q) {
        if (q < nc) {
          const int cc = c_first + q;
          pv[q] = __ldcg(&p.partial[((int64_t)cc * tp.maxseg + seg_of(sp, sg.r, cc)) * BM + rl]);
        }
      }
      float2 acc = make_float2(-INFINITY, 0.f);
#pragma unroll
      for (int q = 0; q < kMaxC; ++q)
        if (q < nc) acc = lse_combine(acc, pv[q]);
      for (int cc = c_first + kMaxC; cc <= c_last; ++cc)
        acc = lse_combine(acc, __ldcg(&p.partial[((int64_t)cc * tp.maxseg + seg_of(sp, sg.r, cc)) * BM + rl]));
      const float Lr = acc.x + __log2f(acc.y);
      float val;
      e[h] = row_epilogue(p, i, Lr, rin[h], out_target, &val);
      if (tp.bias_out != nullptr && p.mode == kModePotential)
        write_bias_row(tp.bias_out + i * 16, (val - rin[h].an) * p.bscale);
    }
  }
  if (p.role == 2) {
    if (tid == 0) p.cnt[sg.r] = 0;
    return;  // the counter is read again only by the next sweep, after this grid ends
  }
  // block sum of the error terms, in a fixed order
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    float v = e[h];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) red[(row0 + NT * h) >> 5] = v;
  }
  seg_bar<NT>();
  if (tid == 0) {
    const float tot = (red[0] + red[1]) + (red[2] + red[3]);
    p.errpart[sg.r] = (double)tot;
    p.cnt[sg.r] = 0;
    s_fin = 0;
    // a lagged loop's stop test runs in the next sweep, which reads the error partials
    // once this grid has ended
    if (!(p.lag && p.role == 1)) {
      const unsigned prev = atomic_add_acq_rel_gpu(&p.cnt[tp.R], 1u);
      s_fin = (prev == (unsigned)(tp.R - 1));
    }
  }
  seg_bar<NT>();
  if (s_fin && tid < 32) {
    finish_sweep_warp(p, tp.R);
    if (tid == 0) p.cnt[tp.R] = 0;
  }
  seg_bar<NT>();
}

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    lse_sweep_tc(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
                 const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl,
                 const __grid_constant__ CUtensorMap mapBbias, TcParams tp) {
  const SweepParams& p = tp.p;
  // Programmatic dependent launch: let the next sweep's CTAs be scheduled as soon as
  // SMs free up; this kernel's own reads of the previous sweep's results wait below.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const SmemLayout L = smem_layout(BN, tp.nkb, tp.split3, tp.stages, tp.a_bufs);
  constexpr uint32_t B_TILE_BYTES = (uint32_t)BN * KB * 2, BIAS_TILE_BYTES = (uint32_t)BN * 32;
  TcShared& sh = *reinterpret_cast<TcShared*>(smem + L.ctrl);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x, G = tp.G, T = tp.T;
  const Split sp = make_split(tp.R, T, G);
  const int nseg = num_segments(sp, c);
  const int nkb = tp.nkb, S = tp.stages, NA = tp.a_bufs;
  volatile int32_t* abort_flag = &sh.abort_flag;

  // ---------------------------------------------------------------- set-up
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.bias_full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.tmem_full[b], 1);
      mbar_init(&sh.tmem_empty[b], 4);
      mbar_init(&sh.a_full[b], 1);
      mbar_init(&sh.a_empty[b], 1);
    }
    mbar_init(&sh.drain, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.seg_full[b], 128);
      mbar_init(&sh.seg_empty[b], 64);
    }
    sh.abort_flag = 0;
    sh.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A-side bias operand: all ones (bf16 0x3F80), so that the K = 16 bias step adds
  // beta_hi + beta_mid + beta_lo whatever the order of the 16-byte chunks in a row.
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
  // The operand tiles do not depend on the previous sweep in the stream, so the producer
  // loads the first stages and the MMA warp runs their operand products before the
  // previous sweep has finished; only the bias rows (its new potential) and the LSE
  // warps' reads of potentials and solver state wait for it (griddepcontrol.wait in the
  // producer and in the LSE warps). When the previous sweep stopped the loop, the
  // producer raises sh.stop through the pending bias barriers and every role winds down.

  if (warp == 0) {
    // ------------------------------------------------------------ producer (whole warp, one lane issues)
    int u = 0;  // B stage units issued
    bool ok = true;
    const uint32_t abytes = (uint32_t)L.a_stride;
    const uint32_t bbytes = B_TILE_BYTES * (tp.split3 ? 2u : 1u);
    // streamed A: each stage also carries the A K block (hi and lo) of its tile
    const uint32_t sabytes = NA == 0 ? A_TILE_BYTES * (tp.split3 ? 2u : 1u) : 0u;
    int a_issued = 0;
    bool waited = false, stopped = false;
    int pend_s[8], pend_t[8], npend = 0;  // stages whose bias rows wait for the previous sweep
    // wait for the previous sweep, then load the pending bias rows (or, when it stopped
    // the loop, release the MMA warp through the pending bias barriers)
    auto resolve = [&]() {
      asm volatile("griddepcontrol.wait;" ::: "memory");
      waited = true;
      stopped = p.state != nullptr && sweep_state(p).done != 0;
      if (elect_one()) {
        if (stopped) sh.stop = 1;
        for (int q = 0; q < npend; ++q) {
          if (stopped) {
            mbar_arrive(&sh.bias_full[pend_s[q]]);
          } else {
            unsigned char* st = smem + L.stage0 + pend_s[q] * L.stage_bytes;
            mbar_arrive_expect_tx(&sh.bias_full[pend_s[q]], BIAS_TILE_BYTES);
            tma_load_2d(st + L.bias_off, &mapBbias, &sh.bias_full[pend_s[q]], 0, pend_t[q] * BN);
          }
        }
      }
      __syncwarp();
    };
    for (int k = 0; k < nseg && ok && !stopped; ++k) {
      const Seg sg = segment(sp, c, k);
      if (NA > 0) {
        const int ai = k % NA;
        // reusing an A buffer waits for the MMA warp, which waits for the pending bias
        // rows: they must be on their way first (as before reusing a stage below)
        if (!waited && k >= NA) {
          resolve();
          if (stopped) break;
        }
        ok = warp_wait(&sh.a_empty[ai], (uint32_t)(((k / NA) & 1) ^ 1), abort_flag);
        if (!ok) break;
        unsigned char* abuf = smem + L.a0 + ai * L.a_stride;
        if (elect_one()) {
          mbar_arrive_expect_tx(&sh.a_full[ai], abytes);
          for (int kb = 0; kb < nkb; ++kb) {
            tma_load_2d(abuf + kb * A_TILE_BYTES, &mapAh, &sh.a_full[ai], kb * KB, sg.r * BM);
            if (tp.split3)
              tma_load_2d(abuf + L.a_lo_off + kb * A_TILE_BYTES, &mapAl, &sh.a_full[ai], kb * KB, sg.r * BM);
          }
        }
        __syncwarp();
        a_issued = k + 1;
      }
      for (int t = sg.t0; t < sg.t1 && ok && !stopped; ++t) {
        for (int kb = 0; kb < nkb; ++kb, ++u) {
          const int s = u % S;
          if (!waited && u == S) {  // a stage is about to be reused: its bias must be on its way
            resolve();
            if (stopped) break;
          }
          ok = warp_wait(&sh.empty[s], (uint32_t)(((u / S) & 1) ^ 1), abort_flag);
          if (!ok) break;
          unsigned char* st = smem + L.stage0 + s * L.stage_bytes;
          if (elect_one()) {
            // after the wait the bias rows travel with the operands on full[s]; before it
            // they follow later on bias_full[s]. bias_full[s] completes once per use of
            // the stage either way (a plain arrival when it carries nothing).
            const bool bias_now = waited && kb == 0;
            mbar_arrive_expect_tx(&sh.full[s], bbytes + sabytes + (bias_now ? BIAS_TILE_BYTES : 0u));
            tma_load_2d(st, &mapBh, &sh.full[s], kb * KB, t * BN);
            if (tp.split3) tma_load_2d(st + L.b_lo_off, &mapBl, &sh.full[s], kb * KB, t * BN);
            if (bias_now) tma_load_2d(st + L.bias_off, &mapBbias, &sh.full[s], 0, t * BN);
            if (NA == 0) {
              tma_load_2d(st + L.a_stage_off, &mapAh, &sh.full[s], kb * KB, sg.r * BM);
              if (tp.split3) tma_load_2d(st + L.a_stage_off + A_TILE_BYTES, &mapAl, &sh.full[s], kb * KB, sg.r * BM);
            }
            if (waited || kb != 0) mbar_arrive(&sh.bias_full[s]);
          }
          if (kb == 0 && !waited) {
            pend_s[npend] = s;
            pend_t[npend] = t;
            ++npend;
          }
          __syncwarp();
        }
      }
    }
    if (ok && !waited) resolve();  // fewer units than stages
    if (!ok || stopped) {
      // drain this CTA's own copies still in flight before shared memory is released
      if (NA > 0)
        for (int k = max(0, a_issued - NA); k < a_issued; ++k)
          warp_wait(&sh.a_full[k % NA], (uint32_t)((k / NA) & 1), abort_flag, true);
      for (int v = max(0, u - S); v < u; ++v) warp_wait(&sh.full[v % S], (uint32_t)((v / S) & 1), abort_flag, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (whole warp, one lane issues)
    const uint64_t abias = desc_sw32(smem_u32(smem + L.a_bias));
    bool ok = true;
    int u = 0, tl = 0;
    for (int k = 0; k < nseg && ok; ++k) {
      const Seg sg = segment(sp, c, k);
      const int ai = NA > 0 ? k % NA : 0;
      if (NA > 0) {
        ok = warp_wait(&sh.a_full[ai], (uint32_t)((k / NA) & 1), abort_flag);
        if (!ok) break;
        tc_fence_after();
      }
      const uint32_t a_hi = smem_u32(smem + L.a0 + ai * L.a_stride);
      const uint32_t a_lo = a_hi + L.a_lo_off;
      for (int t = sg.t0; t < sg.t1 && ok; ++t, ++tl) {
        const int b = tl & 1;
        ok = warp_wait(&sh.tmem_empty[b], (uint32_t)(((tl >> 1) & 1) ^ 1), abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
        for (int kb = 0; kb < nkb; ++kb, ++u) {
          const int s = u % S;
          ok = warp_wait(&sh.full[s], (uint32_t)((u / S) & 1), abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t st = smem_u32(smem + L.stage0 + s * L.stage_bytes);
          const uint64_t bh = desc_sw128(st), bl = desc_sw128(st + L.b_lo_off);
          const uint32_t sa = st + L.a_stage_off;  // streamed A block of this stage
          const uint64_t ah = NA > 0 ? desc_sw128(a_hi + kb * A_TILE_BYTES) : desc_sw128(sa);
          const uint64_t al = NA > 0 ? desc_sw128(a_lo + kb * A_TILE_BYTES) : desc_sw128(sa + A_TILE_BYTES);
          const uint64_t bb = desc_sw32(st + L.bias_off);
          if (elect_one()) {
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk) {
              // +32 bytes per K = 16 step inside the 128-byte swizzle atom (encoded >> 4)
              const uint64_t adv = (uint64_t)(kk * 2);
              umma<BN>(d_tmem, ah + adv, bh + adv, (kb > 0 || kk > 0) ? 1u : 0u);
              if (tp.split3) {
                umma<BN>(d_tmem, ah + adv, bl + adv, 1u);
                umma<BN>(d_tmem, al + adv, bh + adv, 1u);
              }
            }
          }
          __syncwarp();
          if (u < S) {
            // the first stages were loaded before the previous sweep finished: their bias
            // rows (its new potential) may follow on bias_full[s]; later stages carry them
            // on full[s]
            ok = warp_wait(&sh.bias_full[s], (uint32_t)((u / S) & 1), abort_flag);
            if (!ok) break;
            if (*reinterpret_cast<volatile int32_t*>(&sh.stop) != 0) {
              ok = false;  // the loop had already stopped: wind down (not a fault)
              break;
            }
            tc_fence_after();
          }
          if (elect_one()) {
            if (kb == 0) umma<BN>(d_tmem, abias, bb, 1u);
            umma_commit(&sh.empty[s]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (elect_one()) umma_commit(&sh.tmem_full[b]);
        __syncwarp();
      }
      if (!ok) break;
      if (NA > 0 && elect_one()) umma_commit(&sh.a_empty[ai]);
      __syncwarp();
    }
    // make sure no MMA is still writing TMEM when the CTA moves on
    if (elect_one()) umma_commit(&sh.drain);
    __syncwarp();
    warp_wait(&sh.drain, 0, abort_flag, true);
  } else if (threadIdx.x < EPI_TID0) {
    // ------------------------------------------------------------ LSE warps
    // Two warpgroups: warpgroup wg reads TMEM buffer wg, i.e. the tiles with
    // (tile counter & 1) == wg, so two tiles are folded at once.
    const int wg = (warp - 2) >> 2;
    const int quarter = warp & 3;  // TMEM lane quarter this warp may access
    const int row_local = quarter * 32 + lane;
    const int ltid = threadIdx.x - 64;  // 0..127 in warpgroup 0
    int tl = 0, jt = 0;
    // potentials, weights and the solver state below are the previous sweep's results
    asm volatile("griddepcontrol.wait;" ::: "memory");
    SolverState st0{};
    if (p.state != nullptr) st0 = sweep_state(p);
    const bool stopped = st0.done != 0;
    const int fcur = st0.fcur;
    // A warp whose bounded wait failed turns "dead": it skips tile work but keeps
    // executing every named barrier below, so the other LSE warps never block on it.
    bool dead = false;
    for (int k = 0; k < (stopped ? 0 : nseg); ++k) {
      const Seg sg = segment(sp, c, k);
      float m_run = -INFINITY, s_run = 0.f;
      for (int t = sg.t0; t < sg.t1; ++t, ++tl) {
        if ((tl & 1) != wg) continue;
        const uint32_t ph = (uint32_t)(jt & 1);
        ++jt;
        if (dead) continue;
        int okv = 0;
        if (lane == 0) okv = mbar_wait(&sh.tmem_full[wg], ph, abort_flag) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, okv, 0) == 0) {  // warp-uniform: the TMEM loads are .sync.aligned
          dead = true;
          continue;
        }
        __syncwarp();
        tc_fence_after();
        const uint32_t taddr0 = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * BN);
#pragma unroll 1
        for (int half = 0; half < BN / 128; ++half) {
          const uint32_t taddr = taddr0 + (uint32_t)(half * 128);
          float v[4][32];
          PROGOT_TMEM_LD32(taddr + 0, v[0]);
          PROGOT_TMEM_LD32(taddr + 32, v[1]);
          PROGOT_TMEM_LD32(taddr + 64, v[2]);
          PROGOT_TMEM_LD32(taddr + 96, v[3]);
          tmem_wait_ld();
          if (half == BN / 128 - 1) {
            // the whole accumulator is in registers: hand the TMEM buffer back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.tmem_empty[wg]);
          }
          // maximum: 8 independent chains of three-input max
          float mx[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) mx[q] = v[q >> 1][(q & 1) * 16];
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
            for (int q = 0; q < 4; ++q) acc[q] = 0ull;
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
      }
      if (dead) {
        m_run = NAN;
        s_run = NAN;
      }
      // merge warpgroup 1's (max, sum) into warpgroup 0
      // (slots alternate by segment parity: warpgroup 1 can only reuse slot k & 1 after
      // the next 256-thread barrier, which warpgroup 0 reaches after reading it)
      if (wg == 1) sh.ms[k & 1][row_local] = make_float2(m_run, s_run);
      lse_bar_all();
      if (wg == 1) continue;
      {
        const float2 o = sh.ms[k & 1][row_local];
        const float2 mrg = lse_combine(make_float2(m_run, s_run), o);
        m_run = (isnan(o.y) || isnan(s_run)) ? NAN : mrg.x;
        s_run = (isnan(o.y) || isnan(s_run)) ? NAN : mrg.y;
      }
      // ---- segment done
      if (k + 1 < nseg) {
        // hand it to the epilogue warps and go on with the next segment's tiles (slot
        // k & 1 was last read for segment k - 2)
        const int sl = k & 1;
        mbar_wait(&sh.seg_empty[sl], (uint32_t)(((k >> 1) & 1) ^ 1), abort_flag);
        sh.seg[sl][row_local] = make_float2(m_run, s_run);
        mbar_arrive(&sh.seg_full[sl]);
        continue;
      }
      const float2 mv[1] = {make_float2(m_run, s_run)};
      segment_epilogue<128>(tp, c, k, sg, sp, ltid, row_local, mv, fcur, sh.s_last, sh.s_fin, sh.red);
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    // Segments before the CTA's last one: publish, arrive, and combine the row block on
    // the last arrival, while the LSE warps work on the next segment.
    const int etid = threadIdx.x - EPI_TID0;  // 0..63
    asm volatile("griddepcontrol.wait;" ::: "memory");
    SolverState st0{};
    if (p.state != nullptr) st0 = sweep_state(p);
    const bool stopped = st0.done != 0;
    const int fcur = st0.fcur;
    // the g-update of a lagged loop records the f-update's stop test for the next sweeps
    // (also when it is itself a no-op); no other CTA of this grid reads state[(seq + 1) & 1]
    if (p.state != nullptr && p.lag && p.role == 2 && c == 0 && etid == 0) p.state[(p.seq + 1) & 1] = st0;
    for (int k = 0; k + 1 < (stopped ? 0 : nseg); ++k) {
      const Seg sg = segment(sp, c, k);
      const int sl = k & 1;
      const bool okw = mbar_wait(&sh.seg_full[sl], (uint32_t)((k >> 1) & 1), abort_flag);
      float2 mv[2];
      mv[0] = okw ? sh.seg[sl][etid] : make_float2(NAN, NAN);
      mv[1] = okw ? sh.seg[sl][etid + 64] : make_float2(NAN, NAN);
      mbar_arrive(&sh.seg_empty[sl]);
      segment_epilogue<64>(tp, c, k, sg, sp, etid, etid, mv, fcur, sh.e_last, sh.e_fin, sh.ered);
    }
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if (sh.abort_flag != 0 && threadIdx.x == 0 && tp.fault) atomicExch(tp.fault, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// beta_j = (potB_j - |b_j|^2) log2(e)/eps for j < nB, -inf for nB <= j < nB_pad.
__global__ void bias_prep_kernel(const float* __restrict__ potB, const float* __restrict__ Bn, int64_t nB,
                                 int64_t nB_pad, float bscale, __nv_bfloat16* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nB_pad) return;
  const float beta = (j < nB) ? (potB[j] - Bn[j]) * bscale : -INFINITY;
  write_bias_row(out + j * 16, beta);
}

// ---------------------------------------------------------------- operand prep
// One warp per row: hi/lo bf16 split of sqrt(c) (x_i - mu) (mu = 0 when NULL), K padded
// with zeros to dp (a multiple of 64), and (when norm is not NULL) |x_i - mu|^2 summed in
// float64 from the float32 differences.
__global__ void split_bf16_kernel(const float* __restrict__ X, int64_t n, int32_t d, int32_t dp, float scale,
                                  const float* __restrict__ mu, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, float* __restrict__ norm) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  double s = 0.0;
  for (int k = lane; k < dp; k += 32) {
    const float u = (k < d) ? X[r * d + k] - (mu ? mu[k] : 0.f) : 0.f;
    s += (double)u * (double)u;
    const float v = u * scale;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[r * dp + k] = h;
    if (lo) lo[r * dp + k] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
  if (norm == nullptr) return;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) norm[r] = (float)s;
}

}  // namespace tc

// ---------------------------------------------------------------- host side
// Pipeline shape for a tile width bn and a K depth of nkb blocks: the A operand of a row
// block resident in shared memory (two buffers when at least three B stages still fit
// in 227 KB, else one), or, when no resident A leaves room for two B stages (large d),
// streamed with B one K block per stage (a_bufs = 0); as many stages (<= 8) as fit.
static void tc_shape(int bn, int nkb, int split3, int* stages, int* a_bufs) {
  *stages = 0;
  *a_bufs = 1;
  for (int na = 2; na >= 0; --na) {
    int best = 0;
    for (int s = 2; s <= 8; ++s)
      if (tc::smem_layout(bn, nkb, split3, s, na).total <= 227 * 1024) best = s;
    if (best >= (na == 2 ? 3 : 2)) {
      *stages = best;
      *a_bufs = na;
      return;
    }
  }
}

// Column-tile width: 256 (one N = 256 MMA per K step) when two B stages fit next to a
// resident A, else 128 with a resident A; for K depths where neither fits, 256 with A
// streamed (or 128 when even that does not fit).
int tc_tile_cols(int nkb, int split3) {
  int s, na;
  tc_shape(256, nkb, split3, &s, &na);
  if (s >= 2 && na > 0) return 256;
  tc_shape(128, nkb, split3, &s, &na);
  if (s >= 2 && na > 0) return 128;
  tc_shape(256, nkb, split3, &s, &na);
  return s >= 2 ? 256 : 128;
}

int tc_stages(int nkb, int split3) {
  int s, na;
  tc_shape(tc_tile_cols(nkb, split3), nkb, split3, &s, &na);
  return s;
}

cudaError_t launch_split_bf16(const float* X, int64_t n, int32_t d, int32_t dp, float scale, void* hi, void* lo,
                              cudaStream_t s, const float* mu, float* norm) {
  if (n <= 0) return cudaSuccess;
  tc::split_bf16_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(X, n, d, dp, scale, mu, (__nv_bfloat16*)hi,
                                                                (__nv_bfloat16*)lo, norm);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bias_prep(const float* potB, const float* Bn, int64_t nB, int64_t nB_pad, float bscale, void* out,
                             cudaStream_t s) {
  tc::bias_prep_kernel<<<(unsigned)((nB_pad + 255) / 256), 256, 0, s>>>(potB, Bn, nB, nB_pad, bscale,
                                                                        (__nv_bfloat16*)out);
  count_launch();
  return cudaGetLastError();
}

// Number of persistent CTAs and partial slots per CTA for a sweep of nA x nB with
// column tiles of width bn.
void tc_plan(int64_t nA, int64_t nB, int bn, int sms, int* G, int* maxseg) {
  const int64_t R = (nA + tc::BM - 1) / tc::BM, T = (nB + bn - 1) / bn;
  const int g = (int)std::min<int64_t>(R * T, sms);
  const tc::Split sp = tc::make_split((int)R, (int)T, g);
  int ms = 1;
  for (int c = 0; c < g; ++c) ms = std::max(ms, tc::num_segments(sp, c));
  *G = g;
  *maxseg = ms;
}

template <int BN>
static cudaError_t launch_tc(const tc::TcParams& tp, size_t smem, const void* mapAh, const void* mapAl,
                             const void* mapBh, const void* mapBl, const void* mapBbias, cudaStream_t stream) {
  static thread_local size_t attr_bytes = 0;  // per host thread, see launch_map_sweep_fp32
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(tc::lse_sweep_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tp.G);
  cfg.blockDim = dim3(tc::NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc::lse_sweep_tc<BN>, *reinterpret_cast<const CUtensorMap*>(mapAh),
                            *reinterpret_cast<const CUtensorMap*>(mapAl), *reinterpret_cast<const CUtensorMap*>(mapBh),
                            *reinterpret_cast<const CUtensorMap*>(mapBl),
                            *reinterpret_cast<const CUtensorMap*>(mapBbias), tp);
}

cudaError_t launch_lse_sweep_tc(const SweepParams& p, const void* mapAh, const void* mapAl, const void* mapBh,
                                const void* mapBl, const void* mapBbias, int nkb, int split3, int bn, int G,
                                int maxseg, int32_t* fault, void* bias_out, cudaStream_t stream) {
  int stages, a_bufs;
  tc_shape(bn, nkb, split3, &stages, &a_bufs);
  if (stages < 2 || (bn != 128 && bn != 256)) return cudaErrorInvalidValue;
  const size_t smem = tc::smem_layout(bn, nkb, split3, stages, a_bufs).total;
  tc::TcParams tp;
  tp.p = p;
  tp.nkb = nkb;
  tp.split3 = split3;
  tp.stages = stages;
  tp.a_bufs = a_bufs;
  tp.G = G;
  tp.R = (int)((p.nA + tc::BM - 1) / tc::BM);
  tp.T = (int)((p.nB + bn - 1) / bn);
  tp.maxseg = maxseg;
  tp.fault = fault;
  tp.bias_out = (__nv_bfloat16*)bias_out;
  cudaError_t e = (bn == 256) ? launch_tc<256>(tp, smem, mapAh, mapAl, mapBh, mapBl, mapBbias, stream)
                              : launch_tc<128>(tp, smem, mapAh, mapAl, mapBh, mapBl, mapBbias, stream);
  count_launch();
  return e;
}

}  // namespace progot
