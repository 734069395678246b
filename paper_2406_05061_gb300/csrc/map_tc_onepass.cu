// Tensor-core (tcgen05) barycentric displacement of Alg. 2 / Alg. 3 for 64 < d <= 256 in
// one pass over the target cloud:
//   T_i = sum_j 2^{t_ij - L_i} y_j / sum_j 2^{t_ij - L_i},   x_i <- x_i + alpha (T_i - x_i),
// with t_ij = c (x_i . y_j) + beta_j in log2 units and L_i a stabiliser close to the row's
// log-sum-exp (from a log-sum-exp pass, or from the Sinkhorn loop's last f-update, which
// used the same g), as in the d <= 64 kernel (map_tc.cu):
//   S = X Y~^T over all K blocks of the operands (bf16 hi/lo pre-scaled by sqrt(c), three
//     products, beta added by one more K = 16 step) into one of two 32-column TMEM
//     buffers (tiles of 32 columns j);
//   O += P Y~ over all d coordinates at once (N = 64 nkb <= 256), with P_ij =
//     2^{t_ij - L_i} written by the LSE warps into shared memory as bf16 hi/lo (K-major,
//     64-byte swizzle, K = 32 columns of the tile), three products; the B operand is the
//     tile's K blocks of Y~, the very blocks S read, read again as one MN-major matrix
//     whose 64-coordinate column groups are the K blocks; O takes up to 256 TMEM columns.
// With hi parts only (split3 = 0) each product is the single hi x hi term and the lo
// blocks are not loaded. So S is formed once per (row, column) pair, where a map run
// chunk by chunk forms it once per chunk.
// Operands in place: the X row block's hi part sits in TMEM (the A operand of the Xh Yh
// and Xh Yl products, written by warpgroup 1 from the bf16 operand rows at each
// segment's start), its lo part in shared memory (TMA); so four stages fit, each holding
// a tile's K blocks (hi and lo) and bias rows from the S products until its P Y~
// products, and three tiles' copies are in flight while a fourth is in use. The MMA
// warp issues S and P Y~ in whichever order their inputs arrive (S at most one tile
// ahead), so the exponentials of tile q overlap the products of tile q + 1 and P Y~(q)
// does not wait for a later copy.
// CTA = 10 warps: producer, MMA issuer, two LSE warpgroups alternating tiles (one P
// buffer shared in tile order); at a segment's end warpgroup 0 moves O to a per-CTA
// partial slot and the last CTA of a row block combines the slots in CTA order
// (deterministic) and writes x + alpha (T - x). Every mbarrier wait is bounded (2 s): on
// expiry the CTA raises a fault flag, drains its copies and products, frees TMEM and
// leaves.
#include <cuda.h>
#include <cuda_bf16.h>

#include "progot_internal.h"
#include "tc_common.cuh"

namespace progot {
namespace tc {

constexpr int OP_BN = 32;                      // columns j per tile
constexpr int OP_NTHREADS = 320;
constexpr int OP_TMEM_COLS = 512;              // S buffers [0, 64), X hi [64, 64 + 32 nkb), O [256, 256 + 64 nkb)
constexpr uint32_t OP_X_COL = 64;
constexpr uint32_t OP_O_COL = 256;
constexpr uint32_t OP_A_TILE = 128 * 64 * 2;   // 16 KB: one K block of the X row block (hi or lo)
constexpr uint32_t OP_B_TILE = 32 * 64 * 2;    // 4 KB: one K block of a 32-row Y tile (hi or lo)
constexpr uint32_t OP_BIAS = 32 * 32;          // 1 KB: 32 bias rows x 16 bf16
constexpr uint32_t OP_P_HALF = 128 * 32 * 2;   // 8 KB: the P tile (hi or lo), 128 rows x 32 bf16
constexpr int OP_NST = 4;                      // operand stages
constexpr int OP_MAXKB = 4;                    // d <= 256

struct OpLayout {
  uint32_t ones, st, st_bytes, st_lo, st_bias, p, ctrl, total;
};

struct OpShared {
  uint64_t full[OP_NST], empty[OP_NST];
  uint64_t tmem_full[2], tmem_empty[2];
  uint64_t a_full, a_empty;  // X lo copied / the segment's S products done (X hi, X lo free)
  uint64_t x_full;           // X hi written to TMEM (the 4 warps of warpgroup 1 arrive)
  uint64_t p_full, p_empty;  // the P buffer written (4 warps arrive) / consumed (commit)
  uint64_t o_full, o_empty;
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort_flag;
  int32_t s_last;
  float rs[2][128];
  float den[128];
  int32_t slot[8];
};

// X lo (the K blocks of the row block), the ones of the bias product, the stages (K
// blocks hi, K blocks lo, bias rows), the P tile (hi, lo), the control block; offsets
// from a 1024-aligned base.
__host__ __device__ inline OpLayout op_layout(int nkb) {
  OpLayout L;
  L.ones = (uint32_t)nkb * OP_A_TILE;
  L.st = L.ones + 4096;
  L.st_lo = (uint32_t)nkb * OP_B_TILE;
  L.st_bias = 2 * L.st_lo;
  L.st_bytes = (L.st_bias + OP_BIAS + 1023) & ~1023u;
  L.p = L.st + OP_NST * L.st_bytes;
  L.ctrl = L.p + 2 * OP_P_HALF;
  L.total = L.ctrl + (uint32_t)sizeof(OpShared) + 1024;
  return L;
}

struct MapOnepassParams {
  const float* X;
  float* out;
  const float* L;
  float* Opart;      // [G * maxseg][128][d rounded up to 64]
  float* Rpart;      // [G * maxseg][128]
  unsigned* cnt;     // [R] arrival counters (zero between launches)
  int32_t* fault;
  int64_t nA, nB;
  int32_t d, nkb;
  int32_t G, T, R, maxseg;
  float alpha;
  float inv_sc;
  const float* mu;
  const uint32_t* xh;  // bf16 hi rows of the X operand (nA x 64 nkb, pairs packed in 32-bit words)
  int32_t split3;    // 1: hi/lo operands, three products; 0: hi parts only, one product
};

__device__ __forceinline__ void op_bar_all() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void op_bar_wg0() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// K-major tile with 64-byte swizzle: rows of 64 B (32 bf16), 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t op_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;  // 64-byte swizzle
  return d;
}
// The stage's K-major Y blocks read as one MN-major matrix: rows of 128 B along K = j
// (64 coordinates each, 8-row groups 1024 B apart), the next 64 coordinates in the next
// K block, OP_B_TILE bytes on (the leading offset between 64-wide column groups).
__device__ __forceinline__ uint64_t op_desc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(OP_B_TILE >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void op_umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Non-blocking test of the phase with the given parity (mbarrier.test_wait: no suspend,
// so one role's barrier does not hold up the check of the other's).
__device__ __forceinline__ bool op_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same with A read from TMEM (K-major: lane = row, two bf16 per 32-bit column).
__device__ __forceinline__ void op_umma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 32 lanes x 32 columns of 32 bits from registers (one row per thread).
__device__ __forceinline__ void op_tmem_st32(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}
__device__ __forceinline__ uint32_t op_bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ void op_split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
    h[e] = op_bf2_bits(hh);
    l[e] = op_bf2_bits(ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__global__ void __launch_bounds__(OP_NTHREADS, 1)
    map_sweep_tc_onepass(const __grid_constant__ CUtensorMap mapAl,
                         const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl,
                         const __grid_constant__ CUtensorMap mapBbias, MapOnepassParams mp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const OpLayout Lo = op_layout(mp.nkb);
  OpShared& sh = *reinterpret_cast<OpShared*>(smem + Lo.ctrl);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x, G = mp.G, T = mp.T, nkb = mp.nkb;
  const int dw = nkb * 64;  // coordinates held in O and in a partial slot's row
  const Split sp = make_split(mp.R, T, G);
  const int nseg = num_segments(sp, c);
  volatile int32_t* abort_flag = &sh.abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OP_NST; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sh.tmem_full[s], 1);
      mbar_init(&sh.tmem_empty[s], 4);
    }
    mbar_init(&sh.p_full, 4);
    mbar_init(&sh.p_empty, 1);
    mbar_init(&sh.a_full, 1);
    mbar_init(&sh.a_empty, 1);
    mbar_init(&sh.x_full, 4);
    mbar_init(&sh.o_full, 1);
    mbar_init(&sh.o_empty, 4);
    mbar_init(&sh.drain, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    uint32_t* ones = reinterpret_cast<uint32_t*>(smem + Lo.ones);
    for (int i = threadIdx.x; i < 1024; i += OP_NTHREADS) ones[i] = 0x3F803F80u;
    fence_async_smem();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(OP_TMEM_COLS)
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
    int u = 0, a_issued = 0;  // stage units (tiles) and A loads issued
    const uint32_t nh = mp.split3 ? 2u : 1u;  // hi, or hi and lo
    const uint32_t st_tx = nh * (uint32_t)nkb * OP_B_TILE + OP_BIAS;
    for (int k = 0; k < nseg && ok; ++k) {
      const Seg sg = segment(sp, c, k);
      ok = warp_wait(&sh.a_empty, (uint32_t)((k & 1) ^ 1), abort_flag);
      if (!ok) break;
      if (elect_one()) {
        // X lo into shared memory (X hi goes to TMEM through warpgroup 1); with hi parts
        // only the barrier still completes, with no bytes
        mbar_arrive_expect_tx(&sh.a_full, mp.split3 ? (uint32_t)nkb * OP_A_TILE : 0u);
        if (mp.split3)
          for (int kb = 0; kb < nkb; ++kb) tma_load_2d(smem + kb * OP_A_TILE, &mapAl, &sh.a_full, kb * KB, sg.r * BM);
      }
      __syncwarp();
      a_issued = k + 1;
      for (int t = sg.t0; t < sg.t1 && ok; ++t, ++u) {
        const int s = u % OP_NST;
        ok = warp_wait(&sh.empty[s], (uint32_t)(((u / OP_NST) & 1) ^ 1), abort_flag);
        if (!ok) break;
        unsigned char* st = smem + Lo.st + s * Lo.st_bytes;
        if (elect_one()) {
          mbar_arrive_expect_tx(&sh.full[s], st_tx);
          for (int kb = 0; kb < nkb; ++kb) {
            tma_load_2d(st + kb * OP_B_TILE, &mapBh, &sh.full[s], kb * KB, t * OP_BN);
            if (mp.split3) tma_load_2d(st + Lo.st_lo + kb * OP_B_TILE, &mapBl, &sh.full[s], kb * KB, t * OP_BN);
          }
          tma_load_2d(st + Lo.st_bias, &mapBbias, &sh.full[s], 0, t * OP_BN);
        }
        __syncwarp();
      }
    }
    if (!ok) {
      // drain the copies this CTA still has in flight before shared memory is released
      if (a_issued > 0) warp_wait(&sh.a_full, (uint32_t)((a_issued - 1) & 1), abort_flag, true);
      for (int v = (u > OP_NST ? u - OP_NST : 0); v < u; ++v)
        warp_wait(&sh.full[v % OP_NST], (uint32_t)((v / OP_NST) & 1), abort_flag, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // Two streams over the CTA's tiles in order, S(q) and P Y~(q), issued in whichever
    // order their inputs arrive, S at most one tile ahead of the oldest tile still
    // without P Y~: so S(q + 1) runs while the exponentials of tile q are computed, and
    // an LSE warpgroup never waits on the P buffer's barrier more than one phase ahead
    // of it (a parity wait two phases early would pass on the older phase and overwrite
    // P before its products read it). The copies run up to three tiles ahead through
    // the four stages. S and P Y~ write different TMEM columns, so the order of issue
    // changes no result.
    const uint64_t ones = desc_sw32(smem_u32(smem + Lo.ones));
    const int split3 = mp.split3;
    const uint32_t a_lo = smem_u32(smem);
    const uint32_t p0 = smem_u32(smem + Lo.p);
    const uint32_t id_s = make_idesc(BM, OP_BN);
    const uint32_t id_py = make_idesc(BM, 64 * nkb) | (1u << 16);  // N = every coordinate, B MN-major
    int total = 0;
    for (int k = 0; k < nseg; ++k) {
      const Seg sg = segment(sp, c, k);
      total += sg.t1 - sg.t0;
    }
    bool ok = true;
    // S stream: segment, its tiles, the tile's column index and CTA tile index
    int ks = 0, qs = 0;
    Seg sgs = segment(sp, c, 0);
    int ts = sgs.t0;
    bool a_pending = true;  // the segment's A row block not yet seen
    // P Y~ stream
    int kp = 0, qp = 0, oseg = 0;
    Seg sgp = sgs;
    int tpp = sgp.t0;
    unsigned long long t_idle = 0;
    uint32_t spins = 0;
    while (ok && qp < total) {
      bool progressed = false;
      if (qs < total && qs <= qp + 1) {
        bool r = !a_pending ||
                 (op_test_wait(&sh.a_full, (uint32_t)(ks & 1)) && op_test_wait(&sh.x_full, (uint32_t)(ks & 1)));
        r = r && op_test_wait(&sh.tmem_empty[qs & 1], (uint32_t)(((qs >> 1) & 1) ^ 1));
        r = r && op_test_wait(&sh.full[qs % OP_NST], (uint32_t)((qs / OP_NST) & 1));
        if (__all_sync(0xffffffffu, r)) {
          tc_fence_after();
          const int b = qs & 1;
          const uint32_t st = smem_u32(smem + Lo.st + (qs % OP_NST) * Lo.st_bytes);
          const uint32_t d_tmem = tmem_base + (uint32_t)(b * OP_BN);
          const bool seg_end = (ts == sgs.t1 - 1);
          if (elect_one()) {
            for (int kb = 0; kb < nkb; ++kb) {
              const uint64_t bh = desc_sw128(st + kb * OP_B_TILE), bl = desc_sw128(st + Lo.st_lo + kb * OP_B_TILE);
              const uint64_t al = desc_sw128(a_lo + kb * OP_A_TILE);
#pragma unroll
              for (int kk = 0; kk < KB / 16; ++kk) {
                // K = 16 step: 8 TMEM columns of X hi, +32 bytes in the 128-byte swizzle atom
                const uint32_t ax = tmem_base + OP_X_COL + (uint32_t)(kb * 32 + kk * 8);
                const uint64_t adv = (uint64_t)(kk * 2);
                op_umma_ta(d_tmem, ax, bh + adv, id_s, (kb > 0 || kk > 0) ? 1u : 0u);
                if (split3) {
                  op_umma_ta(d_tmem, ax, bl + adv, id_s, 1u);
                  op_umma(d_tmem, al + adv, bh + adv, id_s, 1u);
                }
              }
            }
            op_umma(d_tmem, ones, desc_sw32(st + Lo.st_bias), id_s, 1u);
            umma_commit(&sh.tmem_full[b]);
            if (seg_end) umma_commit(&sh.a_empty);
          }
          __syncwarp();
          a_pending = false;
          ++qs;
          if (++ts == sgs.t1 && ++ks < nseg) {
            sgs = segment(sp, c, ks);
            ts = sgs.t0;
            a_pending = true;
          }
          progressed = true;
        }
      }
      if (qp < qs) {
        // O += P Y~ over every coordinate, from the P buffer and the tile's stage (its K
        // blocks are the B operand's column groups); the stage and P go back after it
        const bool first = (tpp == sgp.t0), last = (tpp == sgp.t1 - 1);
        bool r = !(first && oseg > 0) || op_test_wait(&sh.o_empty, (uint32_t)((oseg - 1) & 1));
        r = r && op_test_wait(&sh.p_full, (uint32_t)(qp & 1));
        if (__all_sync(0xffffffffu, r)) {
          tc_fence_after();
          const int stage = qp % OP_NST;
          const uint32_t st = smem_u32(smem + Lo.st + stage * Lo.st_bytes);
          const uint64_t ah = op_desc_sw64(p0), al = op_desc_sw64(p0 + OP_P_HALF);
          if (elect_one()) {
            const uint64_t bh = op_desc_mn(st), bl = op_desc_mn(st + Lo.st_lo);
            const uint32_t d_o = tmem_base + OP_O_COL;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              // +32 bytes per K = 16 step in P's 64-byte rows; +16 rows (2048 bytes) of the Y blocks
              const uint64_t adv = (uint64_t)(kk * 2), bdv = (uint64_t)(kk * 128);
              op_umma(d_o, ah + adv, bh + bdv, id_py, (first && kk == 0) ? 0u : 1u);
              if (split3) {
                op_umma(d_o, ah + adv, bl + bdv, id_py, 1u);
                op_umma(d_o, al + adv, bh + bdv, id_py, 1u);
              }
            }
            umma_commit(&sh.p_empty);
            umma_commit(&sh.empty[stage]);
            if (last) umma_commit(&sh.o_full);
          }
          __syncwarp();
          if (last) ++oseg;
          ++qp;
          if (++tpp == sgp.t1 && ++kp < nseg) {
            sgp = segment(sp, c, kp);
            tpp = sgp.t0;
          }
          progressed = true;
        }
      }
      if (progressed) {
        spins = 0;
      } else if ((++spins & 255) == 0) {
        // bounded: no input for kWaitNs, or another role gave up
        const unsigned long long now = global_ns();
        if (spins == 256) t_idle = now;
        if (*abort_flag) ok = false;
        else if (now - t_idle > kWaitNs) {
          *abort_flag = 1;
          ok = false;
        }
        ok = __all_sync(0xffffffffu, ok) != 0;
      }
    }
    if (elect_one()) umma_commit(&sh.drain);
    __syncwarp();
    warp_wait(&sh.drain, 0, abort_flag, true);
  } else {
    // ------------------------------------------------------------ LSE warps
    const int wg = (warp - 2) >> 2;
    const int quarter = warp & 3;
    const int row_local = quarter * 32 + lane;
    const int ltid = threadIdx.x - 64;
    // row r of the 64-byte-swizzled P tile: 8-row groups of 512 B, rows of 64 B
    unsigned char* prow = smem + Lo.p + (row_local >> 3) * 512 + (row_local & 7) * 64;
    const int pswz = (row_local >> 1) & 3;
    int tl = 0, jt = 0;
    bool dead = false;
    for (int k = 0; k < nseg; ++k) {
      const Seg sg = segment(sp, c, k);
      const int64_t i = (int64_t)sg.r * BM + row_local;
      const bool row_ok = i < mp.nA;
      if (wg == 1 && !dead) {
        // X hi of this row block into TMEM once the previous segment's S products are
        // done (one row per thread, 32 columns = 64 bf16 per store; zeros past the cloud)
        if (!warp_wait(&sh.a_empty, (uint32_t)((k & 1) ^ 1), abort_flag)) {
          dead = true;
        } else {
          tc_fence_after();
          const uint4* src = reinterpret_cast<const uint4*>(mp.xh + i * (int64_t)(nkb * 32));
          for (int kb = 0; kb < nkb; ++kb) {
            uint32_t w[32];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const uint4 u4 = row_ok ? __ldg(src + kb * 8 + e) : make_uint4(0u, 0u, 0u, 0u);
              w[4 * e] = u4.x;
              w[4 * e + 1] = u4.y;
              w[4 * e + 2] = u4.z;
              w[4 * e + 3] = u4.w;
            }
            op_tmem_st32(tmem_base + ((uint32_t)(quarter * 32) << 16) + OP_X_COL + (uint32_t)(kb * 32), w);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.x_full);
        }
      }
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
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * OP_BN);
        float v[32];
        PROGOT_TMEM_LD32(taddr, v);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.tmem_empty[wg]);
        // P_ij = 2^{t_ij - L_i} (0 on rows past the cloud)
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const float pv = row_ok ? fast_exp2(v[e] - Lr) : 0.f;
          v[e] = pv;
          rs += pv;
        }
        // the P buffer is free once the previous tile's P Y~ has read it
        if (!warp_wait(&sh.p_empty, (uint32_t)((tl & 1) ^ 1), abort_flag)) {
          dead = true;
          continue;
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          uint4 hi, lo;
          op_split8(&v[ch * 8], hi, lo);
          const int pos = (ch ^ pswz) * 16;
          *reinterpret_cast<uint4*>(prow + pos) = hi;
          *reinterpret_cast<uint4*>(prow + OP_P_HALF + pos) = lo;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.p_full);
      }
      // ---- segment done: row sums of both warpgroups, O out of TMEM, partial slot
      if (wg == 1) sh.rs[k & 1][row_local] = rs;
      op_bar_all();
      if (wg == 1) continue;
      rs += sh.rs[k & 1][row_local];
      const int64_t slot = (int64_t)c * mp.maxseg + k;
      const bool okv = !dead && warp_wait(&sh.o_full, (uint32_t)(k & 1), abort_flag);
      if (okv) tc_fence_after();
      for (int oc = 0; oc < nkb; ++oc) {
        float o[2][32];
        if (okv) {
          const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + OP_O_COL + (uint32_t)(oc * 64);
          PROGOT_TMEM_LD32(taddr + 0, o[0]);
          PROGOT_TMEM_LD32(taddr + 32, o[1]);
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) o[0][e] = o[1][e] = NAN;
        }
        if (row_ok) {
          float4* dst = reinterpret_cast<float4*>(mp.Opart + (slot * BM + row_local) * dw + oc * 64);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            dst[e] = make_float4(o[0][4 * e], o[0][4 * e + 1], o[0][4 * e + 2], o[0][4 * e + 3]);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            dst[8 + e] = make_float4(o[1][4 * e], o[1][4 * e + 1], o[1][4 * e + 2], o[1][4 * e + 3]);
        }
      }
      if (okv) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.o_empty);
      } else {
        dead = true;
        rs = NAN;
      }
      if (row_ok) mp.Rpart[slot * BM + row_local] = rs;
      op_bar_wg0();
      if (ltid == 0) {
        int c_first, c_last;
        contributors(sp, sg.r, &c_first, &c_last);
        const unsigned prev = atomic_add_acq_rel_gpu(&mp.cnt[sg.r], 1u);
        sh.s_last = (prev == (unsigned)(c_last - c_first));
      }
      op_bar_wg0();
      if (sh.s_last) {
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
        op_bar_wg0();
        const int64_t rem = mp.nA - (int64_t)sg.r * BM;
        const int rows = rem < BM ? (int)rem : BM;
        const int dd = mp.d;
        const int64_t r0 = (int64_t)sg.r * BM;
        // thread ltid owns the float4 groups f = ltid + 128 j of each chunk's 128 x 64 block
        // (rows f / 16, chunk coordinates 4 (f % 16) .. + 3); per pass all loads, contributor
        // by contributor in CTA order, then all x, then the stores (out may alias x)
        const int cl = (ltid & 15) * 4;
#pragma unroll 1
        for (int oc = 0; oc < nkb; ++oc) {
          const int cg0 = oc * 64 + cl;
          float muv[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) muv[w] = (cg0 + w < dd) ? mp.mu[cg0 + w] : 0.f;
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
              float4 vv[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int f = ltid + 128 * (pass * 8 + j);
                const int row = f >> 4;
                vv[j] = __ldcg(reinterpret_cast<const float4*>(mp.Opart + (sl * BM + row) * dw + oc * 64 + (f & 15) * 4));
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                acc[j].x += vv[j].x;
                acc[j].y += vv[j].y;
                acc[j].z += vv[j].z;
                acc[j].w += vv[j].w;
              }
            }
            float xs[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int row = (ltid + 128 * (pass * 8 + j)) >> 4;
#pragma unroll
              for (int w = 0; w < 4; ++w)
                xs[j][w] = (row < rows && cg0 + w < dd) ? mp.X[(r0 + row) * dd + cg0 + w] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int row = (ltid + 128 * (pass * 8 + j)) >> 4;
              if (row >= rows) continue;
              const float den = sh.den[row];
              const float num[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
#pragma unroll
              for (int w = 0; w < 4; ++w) {
                if (cg0 + w < dd) {
                  const float tx = fmaf(num[w] / den, mp.inv_sc, muv[w]);
                  mp.out[(r0 + row) * dd + cg0 + w] = fmaf(mp.alpha, tx - xs[j][w], xs[j][w]);
                }
              }
            }
          }
        }
        op_bar_wg0();
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(OP_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace tc

bool map_tc_onepass_supported(int nkb) {
  return nkb >= 2 && nkb <= tc::OP_MAXKB && tc::op_layout(nkb).total <= 227 * 1024;
}

int map_tc_onepass_tile_cols() { return tc::OP_BN; }

cudaError_t launch_map_sweep_tc_onepass(const float* X, float* out, const float* L, int64_t nA, int64_t nB,
                                        int32_t d, int32_t nkb, float alpha, const void* mapAl,
                                        const void* mapBh, const void* mapBl, const void* mapBbias, float inv_sc,
                                        const float* mu, const void* xh, float* Opart, float* Rpart, unsigned* cnt,
                                        int G, int maxseg, int32_t split3, int32_t* fault, cudaStream_t stream) {
  if (!map_tc_onepass_supported(nkb)) return cudaErrorInvalidValue;
  const size_t smem = tc::op_layout(nkb).total;
  static thread_local size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(tc::map_sweep_tc_onepass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  tc::MapOnepassParams mp;
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
  mp.nkb = nkb;
  mp.G = G;
  mp.T = (int)((nB + tc::OP_BN - 1) / tc::OP_BN);
  mp.R = (int)((nA + tc::BM - 1) / tc::BM);
  mp.maxseg = maxseg;
  mp.alpha = alpha;
  mp.inv_sc = inv_sc;
  mp.mu = mu;
  mp.split3 = split3;
  mp.xh = reinterpret_cast<const uint32_t*>(xh);
  tc::map_sweep_tc_onepass<<<G, tc::OP_NTHREADS, smem, stream>>>(
      *reinterpret_cast<const CUtensorMap*>(mapAl),
      *reinterpret_cast<const CUtensorMap*>(mapBh), *reinterpret_cast<const CUtensorMap*>(mapBl),
      *reinterpret_cast<const CUtensorMap*>(mapBbias), mp);
  count_launch();
  return cudaGetLastError();
}

}  // namespace progot
