// Tensor-core (tcgen05) barycentric displacement of Alg. 2 / Alg. 3 for clouds with
// d <= 64:
//   T_i = sum_j 2^{t_ij - L_i} y_j / sum_j 2^{t_ij - L_i},   x_i <- x_i + alpha (T_i - x_i),
// with t_ij = c (x_i . y_j) + beta_j in log2 units (the LSE sweep's t) and L_i from that
// sweep or from the Sinkhorn loop's last f-update (the same t; the kernel normalises by its
// own row sums, so L only stabilises the exponentials). Both products run on the tensor
// cores:
//   S = X Y^T as in the LSE sweep (bf16 hi/lo operands pre-scaled by sqrt(c), three
//     products, beta added by one more K = 16 step) into one of two TMEM buffers;
//   O += P Y~ with P_ij = 2^{t_ij - L_i} written by the LSE warps into shared memory as
//     bf16 hi/lo (K-major, 128-byte swizzle), three products Ph Yh + Ph Yl + Pl Yh,
//     M = 128 rows, N = 64 coordinates, K = 128 columns of the tile, into a third TMEM
//     region. The B operand is the tile's own S operand Y~ = sqrt(c) (y - mu) (bf16
//     hi/lo) read a second time as an MN-major matrix (its 128-byte rows are the K index
//     j, each holding the 64 coordinates), so a stage is released only after the tile's
//     P Y~ products; T_i = (O_i / R_i) / sqrt(c) + mu. With hi parts only (split3 = 0)
//     each product is the single Xh Yh or Ph Yh term and the lo tiles are not loaded.
// CTA = 10 warps: warp 0 TMA producer (A row block once per segment; per tile the
// B hi/lo tiles with their bias rows into one of three stages), warp 1 MMA issuer (S of
// tile q + 1 is issued before P Y~ of tile q, so the exponentials of tile q overlap the
// tensor cores), warps 2-9 two LSE warpgroups alternating tiles (one TMEM lane = one
// row per thread: tcgen05.ld, exp2, row sums, the P tile in two 64-column halves). At
// the end of a segment warpgroup 0 reads O out of TMEM into a per-CTA partial slot;
// the last CTA of a row block sums the slots in CTA order (deterministic) and writes
// x + alpha (T - x). Persistent CTAs and segments as in the LSE sweep. Every
// mbarrier wait is bounded (2 s): on expiry the CTA raises a fault flag, drains its
// copies and products, frees TMEM and leaves.
#include <cuda.h>
#include <cuda_bf16.h>

#include "progot_internal.h"
#include "tc_common.cuh"

namespace progot {
namespace tc {

constexpr int MT_BN = 128;                 // columns per tile
constexpr int MT_NTHREADS = 320;
constexpr int MT_TMEM_COLS = 512;          // S buffers at [0, 256), O at [256, 320)
constexpr uint32_t MT_O_COL = 256;
constexpr uint32_t MT_TILE = 128 * 64 * 2;  // 16 KB: 128 rows x 64 bf16 (A, B or P half)
constexpr uint32_t MT_BIAS = 128 * 32;      // 4 KB: 128 rows x 16 bf16
constexpr int MT_NST = 3;                   // operand stages (a stage lives from S(q) to P Y~(q))

// Shared-memory layout (offsets from the 1024-aligned base).
constexpr uint32_t MT_OFF_A = 0;                          // A hi, A lo
constexpr uint32_t MT_OFF_ONES = 2 * MT_TILE;             // 32 KB
constexpr uint32_t MT_OFF_ST = MT_OFF_ONES + 4096;        // 36 KB: stages of B hi, B lo, bias
constexpr uint32_t MT_ST_BYTES = 2 * MT_TILE + MT_BIAS;   // 36 KB
constexpr uint32_t MT_OFF_P = MT_OFF_ST + MT_NST * MT_ST_BYTES;  // 144 KB: P halves 0 and 1, each hi + lo
constexpr uint32_t MT_P_BYTES = 2 * MT_TILE;                     // 32 KB per half
constexpr uint32_t MT_OFF_CTRL = MT_OFF_P + 2 * MT_P_BYTES;      // 208 KB

struct MtShared {
  uint64_t full[MT_NST], empty[MT_NST];  // operand stages
  uint64_t tmem_full[2], tmem_empty[2];
  uint64_t a_full, a_empty;
  uint64_t p_full[2];            // P half h of the current tile written (4 warps arrive)
  uint64_t p_empty[2][2];        // [warpgroup][half]: half h consumed, signalled to the warpgroup
                                 // whose tile uses that buffer next
  uint64_t o_full, o_empty;      // O of a segment complete / read out
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort_flag;
  int32_t s_last;
  float rs[2][128];  // row sums of warpgroup 1 by segment parity
  float den[128];    // combined row sums of the row block being finished
  int32_t slot[8];   // partial slots of the row block's CTAs (first eight)
};

constexpr size_t MT_SMEM_TOTAL = MT_OFF_CTRL + sizeof(MtShared) + 1024;

struct MapTcParams {
  const float* X;    // nA x d points (read in the epilogue; out may alias it)
  float* out;        // nA x d
  const float* L;    // nA row log-sum-exps of t (log2 units)
  float* Opart;      // [G * maxseg][128][64] partial sums of P Y
  float* Rpart;      // [G * maxseg][128] partial row sums of P
  unsigned* cnt;     // [R] arrival counters (zero between launches)
  int32_t* fault;
  int64_t nA, nB;
  int32_t d;
  int32_t G, T, R, maxseg;
  float alpha;
  float inv_sc;      // 1 / sqrt(c): the B operand is sqrt(c) (y - mu)
  const float* mu;   // d: centre of the operands
  int32_t split3;    // 1: hi/lo operands, three products; 0: hi parts only, one product
};

__device__ __forceinline__ void mt_bar_all() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void mt_bar_wg0() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// The B operand of P Y~: the stage's K-major S operand read as MN-major (rows of 128 B
// along K = j, 64 coordinates each, 8-row groups 1024 B apart; with N = 64 there is one
// group along N, so the leading offset is unused and set to the same 1024 B).
__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(1024 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}
// M = 128, N = 64, bf16 x bf16 -> fp32, A K-major, B MN-major.
__device__ __forceinline__ void umma_py(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  constexpr uint32_t kIdesc = make_idesc(BM, 64) | (1u << 16);
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// bf16 hi/lo pair of 8 consecutive values as two 16-byte chunks (paired conversions).
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

__global__ void __launch_bounds__(MT_NTHREADS, 1)
    map_sweep_tc(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
                 const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl,
                 const __grid_constant__ CUtensorMap mapBbias, MapTcParams mp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  MtShared& sh = *reinterpret_cast<MtShared*>(smem + MT_OFF_CTRL);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x, G = mp.G, T = mp.T;
  const Split sp = make_split(mp.R, T, G);
  const int nseg = num_segments(sp, c);
  volatile int32_t* abort_flag = &sh.abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MT_NST; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sh.tmem_full[s], 1);
      mbar_init(&sh.tmem_empty[s], 4);
      mbar_init(&sh.p_full[s], 4);
      mbar_init(&sh.p_empty[0][s], 1);
      mbar_init(&sh.p_empty[1][s], 1);
    }
    mbar_init(&sh.a_full, 1);
    mbar_init(&sh.a_empty, 1);
    mbar_init(&sh.o_full, 1);
    mbar_init(&sh.o_empty, 4);
    mbar_init(&sh.drain, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    // A side of the bias step: all ones (bf16 0x3F80)
    uint32_t* ones = reinterpret_cast<uint32_t*>(smem + MT_OFF_ONES);
    for (int i = threadIdx.x; i < 1024; i += MT_NTHREADS) ones[i] = 0x3F803F80u;
    fence_async_smem();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(MT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = sh.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    bool ok = true;
    int q = 0, a_issued = 0, n_st = 0;  // tiles started; A and stage loads issued
    for (int k = 0; k < nseg && ok; ++k) {
      const Seg sg = segment(sp, c, k);
      ok = warp_wait(&sh.a_empty, (uint32_t)((k & 1) ^ 1), abort_flag);
      if (!ok) break;
      if (elect_one()) {
        mbar_arrive_expect_tx(&sh.a_full, mp.split3 ? 2 * MT_TILE : MT_TILE);
        tma_load_2d(smem + MT_OFF_A, &mapAh, &sh.a_full, 0, sg.r * BM);
        if (mp.split3) tma_load_2d(smem + MT_OFF_A + MT_TILE, &mapAl, &sh.a_full, 0, sg.r * BM);
      }
      __syncwarp();
      a_issued = k + 1;
      for (int t = sg.t0; t < sg.t1 && ok; ++t, ++q) {
        const int s = q % MT_NST;
        ok = warp_wait(&sh.empty[s], (uint32_t)(((q / MT_NST) & 1) ^ 1), abort_flag);
        if (!ok) break;
        unsigned char* st = smem + MT_OFF_ST + s * MT_ST_BYTES;
        if (elect_one()) {
          mbar_arrive_expect_tx(&sh.full[s], (mp.split3 ? 2 * MT_TILE : MT_TILE) + MT_BIAS);
          tma_load_2d(st, &mapBh, &sh.full[s], 0, t * MT_BN);
          if (mp.split3) tma_load_2d(st + MT_TILE, &mapBl, &sh.full[s], 0, t * MT_BN);
          tma_load_2d(st + 2 * MT_TILE, &mapBbias, &sh.full[s], 0, t * MT_BN);
        }
        __syncwarp();
        n_st = q + 1;
      }
    }
    if (!ok) {
      // drain the copies this CTA still has in flight before shared memory is released
      if (a_issued > 0) warp_wait(&sh.a_full, (uint32_t)((a_issued - 1) & 1), abort_flag, true);
      for (int v = (n_st > MT_NST ? n_st - MT_NST : 0); v < n_st; ++v)
        warp_wait(&sh.full[v % MT_NST], (uint32_t)((v / MT_NST) & 1), abort_flag, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint64_t ones = desc_sw32(smem_u32(smem + MT_OFF_ONES));
    const int split3 = mp.split3;
    const uint32_t a_hi = smem_u32(smem + MT_OFF_A), a_lo = a_hi + MT_TILE;
    const uint32_t p0 = smem_u32(smem + MT_OFF_P);
    bool ok = true;
    int q = 0, oseg = 0;
    int pend = -1;
    bool pend_first = false, pend_last = false;
    // P Y~ of tile qq: two halves of 64 columns (two P buffers), each 4 K steps x 3
    // products into O; B is the tile's stage read as MN-major (K step = 16 rows =
    // 2048 B), and the stage goes back to the producer after the second half
    auto issue_py = [&](int qq, bool first, bool last) -> bool {
      if (first && oseg > 0 && !warp_wait(&sh.o_empty, (uint32_t)((oseg - 1) & 1), abort_flag)) return false;
      const int s = qq % MT_NST;
      const uint32_t st = smem_u32(smem + MT_OFF_ST + s * MT_ST_BYTES);
      for (int h = 0; h < 2; ++h) {
        if (!warp_wait(&sh.p_full[h], (uint32_t)(qq & 1), abort_flag)) return false;
        tc_fence_after();
        const uint64_t ah = desc_sw128(p0 + h * MT_P_BYTES), al = desc_sw128(p0 + h * MT_P_BYTES + MT_TILE);
        const uint64_t bh = desc_sw128_mn(st + h * 8192), bl = desc_sw128_mn(st + MT_TILE + h * 8192);
        if (elect_one()) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 2), bdv = (uint64_t)(kk * 128);
            umma_py(tmem_base + MT_O_COL, ah + adv, bh + bdv, (first && h == 0 && kk == 0) ? 0u : 1u);
            if (split3) {
              umma_py(tmem_base + MT_O_COL, ah + adv, bl + bdv, 1u);
              umma_py(tmem_base + MT_O_COL, al + adv, bh + bdv, 1u);
            }
          }
          // buffer h is next used by tile qq + 1, i.e. by the other warpgroup: each
          // warpgroup waits on its own barriers, so neither mistakes the other's release
          umma_commit(&sh.p_empty[(qq + 1) & 1][h]);
          if (h == 1) {
            umma_commit(&sh.empty[s]);
            if (last) umma_commit(&sh.o_full);
          }
        }
        __syncwarp();
      }
      if (last) ++oseg;
      return true;
    };
    for (int k = 0; k < nseg && ok; ++k) {
      const Seg sg = segment(sp, c, k);
      ok = warp_wait(&sh.a_full, (uint32_t)(k & 1), abort_flag);
      if (!ok) break;
      tc_fence_after();
      for (int t = sg.t0; t < sg.t1 && ok; ++t, ++q) {
        const int b = q & 1, s = q % MT_NST;
        ok = warp_wait(&sh.tmem_empty[b], (uint32_t)(((q >> 1) & 1) ^ 1), abort_flag);
        if (!ok) break;
        ok = warp_wait(&sh.full[s], (uint32_t)((q / MT_NST) & 1), abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + MT_OFF_ST + s * MT_ST_BYTES);
        const uint64_t ah = desc_sw128(a_hi), al = desc_sw128(a_lo);
        const uint64_t bh = desc_sw128(st), bl = desc_sw128(st + MT_TILE), bb = desc_sw32(st + 2 * MT_TILE);
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * MT_BN);
        if (elect_one()) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 2);
            umma<MT_BN>(d_tmem, ah + adv, bh + adv, kk > 0 ? 1u : 0u);
            if (split3) {
              umma<MT_BN>(d_tmem, ah + adv, bl + adv, 1u);
              umma<MT_BN>(d_tmem, al + adv, bh + adv, 1u);
            }
          }
          umma<MT_BN>(d_tmem, ones, bb, 1u);
          umma_commit(&sh.tmem_full[b]);
          if (t == sg.t1 - 1) umma_commit(&sh.a_empty);
        }
        __syncwarp();
        if (pend >= 0) {
          ok = issue_py(pend, pend_first, pend_last);
          if (!ok) break;
        }
        pend = q;
        pend_first = (t == sg.t0);
        pend_last = (t == sg.t1 - 1);
      }
    }
    if (ok && pend >= 0) ok = issue_py(pend, pend_first, pend_last);
    if (elect_one()) umma_commit(&sh.drain);
    __syncwarp();
    warp_wait(&sh.drain, 0, abort_flag, true);
  } else {
    // ------------------------------------------------------------ LSE warps
    const int wg = (warp - 2) >> 2;
    const int quarter = warp & 3;  // TMEM lane quarter this warp may access
    const int row_local = quarter * 32 + lane;
    const int ltid = threadIdx.x - 64;  // 0..127 in warpgroup 0
    unsigned char* prow = smem + MT_OFF_P + (row_local >> 3) * 1024 + (row_local & 7) * 128;
    int tl = 0, jt = 0;  // tiles seen, own tiles
    bool dead = false;  // a failed wait: skip work, keep executing the named barriers
    for (int k = 0; k < nseg; ++k) {
      const Seg sg = segment(sp, c, k);
      const int64_t i = (int64_t)sg.r * BM + row_local;
      const bool row_ok = i < mp.nA;
      const float Lr = row_ok ? mp.L[i] : 0.f;
      float rs = 0.f;
      for (int t = sg.t0; t < sg.t1; ++t, ++tl) {
        if ((tl & 1) != wg) continue;
        const uint32_t ph = (uint32_t)(jt & 1);
        ++jt;
        if (dead) continue;
        if (!warp_wait(&sh.tmem_full[wg], ph, abort_flag)) {
          dead = true;
          continue;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * MT_BN);
        // own tile n (jt - 1) needs buffer h released by the previous tile: warpgroup 0's
        // first tile has no predecessor, warpgroup 1's first needs release 0
        const int n_own = jt - 1;
        const uint32_t par = (uint32_t)(wg == 0 ? ((n_own & 1) ^ 1) : (n_own & 1));
        // two halves of 64 columns: load, exponentiate, write the P half (64 registers live)
        for (int h = 0; h < 2 && !dead; ++h) {
          float v[2][32];
          PROGOT_TMEM_LD32(taddr + h * 64, v[0]);
          PROGOT_TMEM_LD32(taddr + h * 64 + 32, v[1]);
          tmem_wait_ld();
          if (h == 1) {
            // the whole accumulator has been read: hand the buffer back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.tmem_empty[wg]);
          }
          // P_ij = 2^{t_ij - L_i} (0 on rows past the cloud)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const float pv = row_ok ? fast_exp2(v[cc][e] - Lr) : 0.f;
              v[cc][e] = pv;
              rs += pv;
            }
          if (!warp_wait(&sh.p_empty[wg][h], par, abort_flag)) {
            dead = true;
            break;
          }
          unsigned char* prow_hi = prow + h * MT_P_BYTES;
          unsigned char* prow_lo = prow_hi + MT_TILE;
          // 8 chunks of 8 columns; chunk ch of row r sits at chunk position ch ^ (r & 7)
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            uint4 hi, lo;
            split8(&v[ch >> 2][(ch & 3) * 8], hi, lo);
            const int pos = (ch ^ (row_local & 7)) * 16;
            *reinterpret_cast<uint4*>(prow_hi + pos) = hi;
            *reinterpret_cast<uint4*>(prow_lo + pos) = lo;
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.p_full[h]);
        }
      }
      // ---- segment done: row sums of both warpgroups, O out of TMEM, partial slot
      if (wg == 1) sh.rs[k & 1][row_local] = rs;
      mt_bar_all();
      if (wg == 1) continue;
      rs += sh.rs[k & 1][row_local];
      float o[2][32];
      bool okv = !dead && warp_wait(&sh.o_full, (uint32_t)(k & 1), abort_flag);
      if (okv) {
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + MT_O_COL;
        PROGOT_TMEM_LD32(taddr + 0, o[0]);
        PROGOT_TMEM_LD32(taddr + 32, o[1]);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.o_empty);
      } else {
        dead = true;
#pragma unroll
        for (int e = 0; e < 32; ++e) o[0][e] = o[1][e] = NAN;
        rs = NAN;
      }
      const int64_t slot = (int64_t)c * mp.maxseg + k;
      if (row_ok) {
        float4* dst = reinterpret_cast<float4*>(mp.Opart + (slot * BM + row_local) * 64);
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[e] = make_float4(o[0][4 * e], o[0][4 * e + 1], o[0][4 * e + 2], o[0][4 * e + 3]);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          dst[8 + e] = make_float4(o[1][4 * e], o[1][4 * e + 1], o[1][4 * e + 2], o[1][4 * e + 3]);
        mp.Rpart[slot * BM + row_local] = rs;
      }
      mt_bar_wg0();  // the slot stores of all 128 rows happen before the arrival
      if (ltid == 0) {
        int c_first, c_last;
        contributors(sp, sg.r, &c_first, &c_last);
        const unsigned prev = atomic_add_acq_rel_gpu(&mp.cnt[sg.r], 1u);
        sh.s_last = (prev == (unsigned)(c_last - c_first));
      }
      mt_bar_wg0();
      if (sh.s_last) {
        // the row block's CTAs c_first..c_last hold one partial slot each; sum them in CTA
        // order, first the row sums (one thread per row), then the 128 x d block of P Y
        // with consecutive threads on consecutive coordinates (coalesced, independent loads)
        int c_first, c_last;
        contributors(sp, sg.r, &c_first, &c_last);
        const int nc = c_last - c_first + 1;
        if (ltid < 8 && ltid < nc) {
          const int cc = c_first + ltid;
          sh.slot[ltid] = cc * mp.maxseg + seg_of(sp, sg.r, cc);
        }
        {
          float den = 0.f;
          for (int cc = c_first; cc <= c_last; ++cc)
            den += __ldcg(mp.Rpart + ((int64_t)cc * mp.maxseg + seg_of(sp, sg.r, cc)) * BM + row_local);
          sh.den[row_local] = den;
        }
        mt_bar_wg0();
        const int64_t rem = mp.nA - (int64_t)sg.r * BM;
        const int rows = rem < BM ? (int)rem : BM;
        const int dd = mp.d;
        const int64_t r0 = (int64_t)sg.r * BM;
        // Thread ltid owns the float4 groups f = ltid + 128 j of the 128 x 64 block (rows
        // f / 16, coordinates 4 (f % 16) .. + 3, the same four for every j). Each pass
        // issues the loads of eight groups together, contributor by contributor (the sums
        // keep the CTA order), then all eight groups' x before any store: out aliases x,
        // so a store between loads would serialise them.
        const int c0 = (ltid & 15) * 4;
        float muv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) muv[u] = (c0 + u < dd) ? mp.mu[c0 + u] : 0.f;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
          float4 acc[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int q2 = 0; q2 < nc; ++q2) {
            int64_t sl;
            if (q2 < 8) {
              sl = sh.slot[q2];
            } else {
              const int cc = c_first + q2;
              sl = (int64_t)cc * mp.maxseg + seg_of(sp, sg.r, cc);
            }
            const float4* src = reinterpret_cast<const float4*>(mp.Opart + sl * BM * 64);
            float4 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __ldcg(src + ltid + 128 * (pass * 8 + j));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              acc[j].x += v[j].x;
              acc[j].y += v[j].y;
              acc[j].z += v[j].z;
              acc[j].w += v[j].w;
            }
          }
          float xs[8][4];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int row = (ltid + 128 * (pass * 8 + j)) >> 4;
#pragma unroll
            for (int u = 0; u < 4; ++u)
              xs[j][u] = (row < rows && c0 + u < dd) ? mp.X[(r0 + row) * dd + c0 + u] : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int row = (ltid + 128 * (pass * 8 + j)) >> 4;
            if (row >= rows) continue;
            const float den = sh.den[row];
            const float num[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (c0 + u < dd) {
                const float tx = fmaf(num[u] / den, mp.inv_sc, muv[u]);
                mp.out[(r0 + row) * dd + c0 + u] = fmaf(mp.alpha, tx - xs[j][u], xs[j][u]);
              }
            }
          }
        }
        mt_bar_wg0();
        if (ltid == 0) mp.cnt[sg.r] = 0;
      }
    }
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if (sh.abort_flag != 0 && threadIdx.x == 0 && mp.fault) atomicExch(mp.fault, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(MT_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace tc

size_t map_sweep_tc_smem() { return tc::MT_SMEM_TOTAL; }

cudaError_t launch_map_sweep_tc(const float* X, float* out, const float* L, int64_t nA, int64_t nB, int32_t d,
                                float alpha, const void* mapAh, const void* mapAl, const void* mapBh,
                                const void* mapBl, const void* mapBbias, float inv_sc, const float* mu,
                                float* Opart, float* Rpart, unsigned* cnt, int G, int maxseg, int32_t split3,
                                int32_t* fault, cudaStream_t stream) {
  static thread_local bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tc::map_sweep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc::MT_SMEM_TOTAL);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  tc::MapTcParams mp;
  mp.X = X;
  mp.out = out;
  mp.L = L;
  mp.Opart = Opart;
  mp.Rpart = Rpart;
  mp.cnt = cnt;
  mp.fault = fault;
  mp.nA = nA;
  mp.nB = nB;
  mp.d = d;
  mp.G = G;
  mp.T = (int)((nB + tc::MT_BN - 1) / tc::MT_BN);
  mp.R = (int)((nA + tc::BM - 1) / tc::BM);
  mp.maxseg = maxseg;
  mp.alpha = alpha;
  mp.inv_sc = inv_sc;
  mp.mu = mu;
  mp.split3 = split3;
  tc::map_sweep_tc<<<G, tc::MT_NTHREADS, tc::MT_SMEM_TOTAL, stream>>>(
      *reinterpret_cast<const CUtensorMap*>(mapAh), *reinterpret_cast<const CUtensorMap*>(mapAl),
      *reinterpret_cast<const CUtensorMap*>(mapBh), *reinterpret_cast<const CUtensorMap*>(mapBl),
      *reinterpret_cast<const CUtensorMap*>(mapBbias), mp);
  count_launch();
  return cudaGetLastError();
}

}  // namespace progot
