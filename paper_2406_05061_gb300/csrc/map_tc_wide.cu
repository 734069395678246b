// Tensor-core (tcgen05) barycentric displacement of Alg. 2 / Alg. 3 for 64 < d <= 256:
//   T_i = sum_j 2^{t_ij - L_i} y_j / sum_j 2^{t_ij - L_i},   x_i <- x_i + alpha (T_i - x_i),
// with t_ij = c (x_i . y_j) + beta_j in log2 units and L_i from a log-sum-exp pass, as in
// the d <= 64 kernel (map_tc.cu), one launch per chunk of 64 output coordinates:
//   S = X Y~^T over all K blocks of the operands (bf16 hi/lo pre-scaled by sqrt(c), three
//     products, beta added by one more K = 16 step) into one of two 64-column TMEM
//     buffers (tiles of 64 columns j);
//   O += P Y~[:, chunk] with P_ij = 2^{t_ij - L_i} written by the LSE warps into shared
//     memory as bf16 hi/lo (K-major, 128-byte swizzle), M = 128 rows, N = 64
//     coordinates, K = 64 columns of the tile, three products; the B operand is the
//     tile's K block of the chunk, the stage S read, read again as an MN-major matrix.
// The X row block (all K blocks, hi and lo) stays resident for a segment; a tile's K
// blocks arrive in the order chunk + 1, ..., chunk: all but the last through two
// alternating streaming stages, the chunk's own block (which P Y~ reads again) through a
// third, held stage. The MMA warp issues S(q + 1) up to its last block, then P Y~(q)
// (which frees the held stage), then the last block of S(q + 1), so the exponentials of
// tile q overlap the products of tile q + 1. S is recomputed for every chunk; the chunk
// writes only its own coordinates of out (which may alias X: the products read the bf16
// operands prepared before the first chunk).
// CTA = 10 warps: producer, MMA issuer, two LSE warpgroups alternating tiles (one P
// buffer shared in tile order); at a segment's end warpgroup 0 moves O to a per-CTA
// partial slot and the last CTA of a row block combines the slots in CTA order. Every
// mbarrier wait is bounded (2 s): on expiry the CTA raises a fault flag, drains its
// copies and products, frees TMEM and leaves.
#include <cuda.h>
#include <cuda_bf16.h>

#include "progot_internal.h"
#include "tc_common.cuh"

namespace progot {
namespace tc {

constexpr int MW_BN = 64;                    // columns j per tile
constexpr int MW_NTHREADS = 320;
constexpr int MW_TMEM_COLS = 256;            // S buffers at [0, 128), O at [128, 192)
constexpr uint32_t MW_O_COL = 128;
constexpr uint32_t MW_A_TILE = 128 * 64 * 2;   // 16 KB: 128 rows x 64 bf16 (one K block of A, hi or lo)
constexpr uint32_t MW_B_TILE = 64 * 64 * 2;    // 8 KB: 64 rows x 64 bf16 (one K block of a B tile)
constexpr uint32_t MW_BIAS = 64 * 32;          // 2 KB: 64 rows x 16 bf16
constexpr int MW_NST = 3;                      // operand stages
constexpr int MW_MAXKB = 4;                    // d <= 256
constexpr uint32_t MW_ST_BYTES = 2 * MW_B_TILE + MW_BIAS;  // B hi, B lo, bias rows (18 KB, 1024-aligned)

// Shared-memory layout (offsets from the 1024-aligned base), for nkb K blocks.
struct MwLayout {
  uint32_t a_lo, ones, st, p, ctrl, total;
};
__host__ __device__ inline MwLayout mw_layout(int nkb);

struct MwShared {
  uint64_t full[MW_NST], empty[MW_NST];
  uint64_t tmem_full[2], tmem_empty[2];
  uint64_t a_full, a_empty;
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

__host__ __device__ inline MwLayout mw_layout(int nkb) {
  MwLayout L;
  L.a_lo = (uint32_t)nkb * MW_A_TILE;
  L.ones = 2 * L.a_lo;
  L.st = L.ones + 4096;
  L.p = L.st + MW_NST * MW_ST_BYTES;
  L.ctrl = L.p + 2 * (128 * 64 * 2);  // P hi, P lo: 128 rows x 64 bf16 each
  L.total = L.ctrl + (uint32_t)sizeof(MwShared) + 1024;
  return L;
}

struct MapWideParams {
  const float* X;
  float* out;
  const float* L;
  float* Opart;      // [G * maxseg][128][64]
  float* Rpart;      // [G * maxseg][128]
  unsigned* cnt;     // [R] arrival counters (zero between launches)
  int32_t* fault;
  int64_t nA, nB;
  int32_t d, nkb, oc;  // coordinates, K blocks, output chunk (coordinates 64 oc .. 64 oc + 63)
  int32_t G, T, R, maxseg;
  float alpha;
  float inv_sc;
  const float* mu;
};

__device__ __forceinline__ void mw_bar_all() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void mw_bar_wg0() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// The stage's K-major B tile read as MN-major (rows of 128 B along K = j, 64 coordinates
// each, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t mw_desc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(1024 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// M = 128, N = 64, bf16 x bf16 -> fp32; A K-major; B K-major (S) or MN-major (P Y~).
template <bool kBmn>
__device__ __forceinline__ void mw_umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  constexpr uint32_t kIdesc = make_idesc(BM, 64) | (kBmn ? (1u << 16) : 0u);
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ uint32_t mw_bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ void mw_split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
    h[e] = mw_bf2_bits(hh);
    l[e] = mw_bf2_bits(ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// K block of position j in a tile's order: chunk + 1, ..., nkb - 1, 0, ..., chunk.
__device__ __forceinline__ int mw_kb(int j, int oc, int nkb) { return (oc + 1 + j) % nkb; }

__global__ void __launch_bounds__(MW_NTHREADS, 1)
    map_sweep_tc_wide(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
                      const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl,
                      const __grid_constant__ CUtensorMap mapBbias, MapWideParams mp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const MwLayout Lw = mw_layout(mp.nkb);
  MwShared& sh = *reinterpret_cast<MwShared*>(smem + Lw.ctrl);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x, G = mp.G, T = mp.T, nkb = mp.nkb, oc = mp.oc;
  const Split sp = make_split(mp.R, T, G);
  const int nseg = num_segments(sp, c);
  volatile int32_t* abort_flag = &sh.abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MW_NST; ++s) {
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
    mbar_init(&sh.o_full, 1);
    mbar_init(&sh.o_empty, 4);
    mbar_init(&sh.drain, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    uint32_t* ones = reinterpret_cast<uint32_t*>(smem + Lw.ones);
    for (int i = threadIdx.x; i < 1024; i += MW_NTHREADS) ones[i] = 0x3F803F80u;
    fence_async_smem();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(MW_TMEM_COLS)
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
    int us = 0, uh = 0, a_issued = 0;  // streaming and held stage units issued, A loads issued
    for (int k = 0; k < nseg && ok; ++k) {
      const Seg sg = segment(sp, c, k);
      ok = warp_wait(&sh.a_empty, (uint32_t)((k & 1) ^ 1), abort_flag);
      if (!ok) break;
      if (elect_one()) {
        mbar_arrive_expect_tx(&sh.a_full, 2u * (uint32_t)nkb * MW_A_TILE);
        for (int kb = 0; kb < nkb; ++kb) {
          tma_load_2d(smem + kb * MW_A_TILE, &mapAh, &sh.a_full, kb * KB, sg.r * BM);
          tma_load_2d(smem + Lw.a_lo + kb * MW_A_TILE, &mapAl, &sh.a_full, kb * KB, sg.r * BM);
        }
      }
      __syncwarp();
      a_issued = k + 1;
      for (int t = sg.t0; t < sg.t1 && ok; ++t) {
        for (int j = 0; j < nkb && ok; ++j) {
          const bool held = (j == nkb - 1);
          const int s = held ? 2 : (us & 1);
          const uint32_t par = held ? (uint32_t)((uh & 1) ^ 1) : (uint32_t)(((us >> 1) & 1) ^ 1);
          const int kb = mw_kb(j, oc, nkb);
          ok = warp_wait(&sh.empty[s], par, abort_flag);
          if (!ok) break;
          unsigned char* st = smem + Lw.st + s * MW_ST_BYTES;
          if (elect_one()) {
            mbar_arrive_expect_tx(&sh.full[s], 2 * MW_B_TILE + (j == 0 ? MW_BIAS : 0u));
            tma_load_2d(st, &mapBh, &sh.full[s], kb * KB, t * MW_BN);
            tma_load_2d(st + MW_B_TILE, &mapBl, &sh.full[s], kb * KB, t * MW_BN);
            if (j == 0) tma_load_2d(st + 2 * MW_B_TILE, &mapBbias, &sh.full[s], 0, t * MW_BN);
          }
          __syncwarp();
          if (held) ++uh;
          else ++us;
        }
      }
    }
    if (!ok) {
      // drain the copies this CTA still has in flight before shared memory is released
      if (a_issued > 0) warp_wait(&sh.a_full, (uint32_t)((a_issued - 1) & 1), abort_flag, true);
      for (int v = (us > 2 ? us - 2 : 0); v < us; ++v)
        warp_wait(&sh.full[v & 1], (uint32_t)((v >> 1) & 1), abort_flag, true);
      if (uh > 0) warp_wait(&sh.full[2], (uint32_t)((uh - 1) & 1), abort_flag, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint64_t ones = desc_sw32(smem_u32(smem + Lw.ones));
    const uint32_t a_hi = smem_u32(smem), a_lo = a_hi + Lw.a_lo;
    const uint32_t p0 = smem_u32(smem + Lw.p);
    bool ok = true;
    int q = 0, us = 0, uh = 0, oseg = 0;
    int pend = -1;
    bool pend_first = false, pend_last = false;
    // P Y~[:, chunk] of tile qq from the P buffer and the held stage (the chunk's K block
    // of the tile); the held stage and the P buffer go back after it
    auto issue_py = [&](int qq, bool first, bool last) -> bool {
      if (first && oseg > 0 && !warp_wait(&sh.o_empty, (uint32_t)((oseg - 1) & 1), abort_flag)) return false;
      if (!warp_wait(&sh.p_full, (uint32_t)(qq & 1), abort_flag)) return false;
      tc_fence_after();
      const uint32_t st = smem_u32(smem + Lw.st + 2 * MW_ST_BYTES);
      const uint64_t ah = desc_sw128(p0), al = desc_sw128(p0 + 128 * 64 * 2);
      const uint64_t bh = mw_desc_mn(st), bl = mw_desc_mn(st + MW_B_TILE);
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 2), bdv = (uint64_t)(kk * 128);
          mw_umma<true>(tmem_base + MW_O_COL, ah + adv, bh + bdv, (first && kk == 0) ? 0u : 1u);
          mw_umma<true>(tmem_base + MW_O_COL, ah + adv, bl + bdv, 1u);
          mw_umma<true>(tmem_base + MW_O_COL, al + adv, bh + bdv, 1u);
        }
        umma_commit(&sh.p_empty);
        umma_commit(&sh.empty[2]);
        if (last) umma_commit(&sh.o_full);
      }
      __syncwarp();
      if (last) ++oseg;
      return true;
    };
    for (int k = 0; k < nseg && ok; ++k) {
      const Seg sg = segment(sp, c, k);
      ok = warp_wait(&sh.a_full, (uint32_t)(k & 1), abort_flag);
      if (!ok) break;
      tc_fence_after();
      for (int t = sg.t0; t < sg.t1 && ok; ++t, ++q) {
        const int b = q & 1;
        ok = warp_wait(&sh.tmem_empty[b], (uint32_t)(((q >> 1) & 1) ^ 1), abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * MW_BN);
        for (int j = 0; j < nkb && ok; ++j) {
          const bool held = (j == nkb - 1);
          if (held && pend >= 0) {
            // the previous tile's P Y~ frees the held stage this tile's last block needs
            ok = issue_py(pend, pend_first, pend_last);
            pend = -1;
            if (!ok) break;
          }
          const int s = held ? 2 : (us & 1);
          const uint32_t par = held ? (uint32_t)(uh & 1) : (uint32_t)((us >> 1) & 1);
          const int kb = mw_kb(j, oc, nkb);
          ok = warp_wait(&sh.full[s], par, abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t st = smem_u32(smem + Lw.st + s * MW_ST_BYTES);
          const uint64_t bh = desc_sw128(st), bl = desc_sw128(st + MW_B_TILE);
          const uint64_t ah = desc_sw128(a_hi + kb * MW_A_TILE), al = desc_sw128(a_lo + kb * MW_A_TILE);
          if (elect_one()) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t adv = (uint64_t)(kk * 2);
              mw_umma<false>(d_tmem, ah + adv, bh + adv, (j > 0 || kk > 0) ? 1u : 0u);
              mw_umma<false>(d_tmem, ah + adv, bl + adv, 1u);
              mw_umma<false>(d_tmem, al + adv, bh + adv, 1u);
            }
            if (j == 0) mw_umma<false>(d_tmem, ones, desc_sw32(st + 2 * MW_B_TILE), 1u);
            if (!held) umma_commit(&sh.empty[s]);  // the held block goes back after P Y~
            if (held) {
              umma_commit(&sh.tmem_full[b]);
              if (t == sg.t1 - 1) umma_commit(&sh.a_empty);
            }
          }
          __syncwarp();
          if (held) ++uh;
          else ++us;
        }
        if (!ok) break;
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
    const int quarter = warp & 3;
    const int row_local = quarter * 32 + lane;
    const int ltid = threadIdx.x - 64;
    unsigned char* prow = smem + Lw.p + (row_local >> 3) * 1024 + (row_local & 7) * 128;
    int tl = 0, jt = 0;
    bool dead = false;
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
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * MW_BN);
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
        // the P buffer is free once the previous tile's P Y~ has read it
        if (!warp_wait(&sh.p_empty, (uint32_t)((tl & 1) ^ 1), abort_flag)) {
          dead = true;
          continue;
        }
        unsigned char* prow_hi = prow;
        unsigned char* prow_lo = prow + 128 * 64 * 2;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          uint4 hi, lo;
          mw_split8(&v[ch >> 2][(ch & 3) * 8], hi, lo);
          const int pos = (ch ^ (row_local & 7)) * 16;
          *reinterpret_cast<uint4*>(prow_hi + pos) = hi;
          *reinterpret_cast<uint4*>(prow_lo + pos) = lo;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.p_full);
      }
      // ---- segment done: row sums of both warpgroups, O out of TMEM, partial slot
      if (wg == 1) sh.rs[k & 1][row_local] = rs;
      mw_bar_all();
      if (wg == 1) continue;
      rs += sh.rs[k & 1][row_local];
      float o[2][32];
      bool okv = !dead && warp_wait(&sh.o_full, (uint32_t)(k & 1), abort_flag);
      if (okv) {
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + MW_O_COL;
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
      mw_bar_wg0();
      if (ltid == 0) {
        int c_first, c_last;
        contributors(sp, sg.r, &c_first, &c_last);
        const unsigned prev = atomic_add_acq_rel_gpu(&mp.cnt[sg.r], 1u);
        sh.s_last = (prev == (unsigned)(c_last - c_first));
      }
      mw_bar_wg0();
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
        mw_bar_wg0();
        const int64_t rem = mp.nA - (int64_t)sg.r * BM;
        const int rows = rem < BM ? (int)rem : BM;
        const int dd = mp.d;
        const int64_t r0 = (int64_t)sg.r * BM;
        // thread ltid owns the float4 groups f = ltid + 128 j of the 128 x 64 block (rows
        // f / 16, chunk coordinates 4 (f % 16) .. + 3); all loads of a pass, contributor by
        // contributor in CTA order, then all x, then the stores (out may alias x)
        const int cl = (ltid & 15) * 4;       // coordinate within the chunk
        const int cg0 = mp.oc * 64 + cl;      // coordinate of the cloud
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
            const float4* src = reinterpret_cast<const float4*>(mp.Opart + sl * BM * 64);
            float4 vv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) vv[j] = __ldcg(src + ltid + 128 * (pass * 8 + j));
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
        mw_bar_wg0();
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(MW_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace tc

bool map_tc_wide_supported(int nkb) {
  return nkb >= 2 && nkb <= tc::MW_MAXKB && tc::mw_layout(nkb).total <= 227 * 1024;
}

cudaError_t launch_map_sweep_tc_wide(const float* X, float* out, const float* L, int64_t nA, int64_t nB, int32_t d,
                                     int32_t nkb, int32_t oc, float alpha, const void* mapAh, const void* mapAl,
                                     const void* mapBh, const void* mapBl, const void* mapBbias, float inv_sc,
                                     const float* mu, float* Opart, float* Rpart, unsigned* cnt, int G, int maxseg,
                                     int32_t* fault, cudaStream_t stream) {
  if (!map_tc_wide_supported(nkb)) return cudaErrorInvalidValue;
  const size_t smem = tc::mw_layout(nkb).total;
  static thread_local size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(tc::map_sweep_tc_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  tc::MapWideParams mp;
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
  mp.oc = oc;
  mp.G = G;
  mp.T = (int)((nB + tc::MW_BN - 1) / tc::MW_BN);
  mp.R = (int)((nA + tc::BM - 1) / tc::BM);
  mp.maxseg = maxseg;
  mp.alpha = alpha;
  mp.inv_sc = inv_sc;
  mp.mu = mu;
  tc::map_sweep_tc_wide<<<G, tc::MW_NTHREADS, smem, stream>>>(
      *reinterpret_cast<const CUtensorMap*>(mapAh), *reinterpret_cast<const CUtensorMap*>(mapAl),
      *reinterpret_cast<const CUtensorMap*>(mapBh), *reinterpret_cast<const CUtensorMap*>(mapBl),
      *reinterpret_cast<const CUtensorMap*>(mapBbias), mp);
  count_launch();
  return cudaGetLastError();
}

}  // namespace progot
