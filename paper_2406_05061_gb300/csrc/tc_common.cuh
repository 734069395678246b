// tcgen05 / TMA / mbarrier building blocks shared by the tensor-core kernels
// (sm_103a): bounded mbarrier waits, elected-lane issue, 2-D tiled TMA loads,
// shared-memory matrix descriptors, kind::f16 MMAs with float32 accumulation in TMEM
// and TMEM loads.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace progot {
namespace tc {

constexpr int BM = 128;  // rows per CTA (TMEM lanes, M of every MMA)
constexpr int KB = 64;   // bf16 K elements per 128-byte swizzle atom
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded-wait limit per CTA

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity; false when the CTA aborted or the wait
// ran past kWaitNs (then the abort flag is raised for the whole CTA).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int32_t* abort_flag,
                                       bool ignore_abort = false) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 0) {
      if (!ignore_abort && *abort_flag) return false;
      if (global_ns() - t0 > kWaitNs) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// One lane of a converged warp (the lowest), chosen by elect.sync: issuing TMA and
// tcgen05 instructions from warp-uniform code keeps their operands in uniform
// registers.
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "elect.sync _|P, 0xffffffff;\n\t"
      "selp.b32 %0, 1, 0, P;\n\t}"
      : "=r"(pred));
  return pred != 0;
}

// Bounded wait by every lane of a warp; the warp proceeds only if all lanes saw the phase.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int32_t* abort_flag,
                                          bool ignore_abort = false) {
  const bool ok = mbar_wait(bar, parity, abort_flag, ignore_abort);
  return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
// K-major tile with 32-byte swizzle: rows of 32 B (16 bf16), 8-row groups 256 B apart.
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;             // 32-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: bf16 x bf16 -> fp32, K-major A and B, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
template <int BN>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  constexpr uint32_t kIdesc = make_idesc(BM, BN);
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define PROGOT_TMEM_LD32(taddr, v)                                                                                   \
  asm volatile(                                                                                                      \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"   \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                                 \
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]), \
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),      \
        "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),     \
        "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])                   \
      : "r"(taddr))

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Persistent work split of the (row block, column tile) grid, R x T, over G CTAs.
// Bands: the first nb G row blocks (nb = floor(R / G)) go whole to one CTA each, row
// block b G + c to CTA c as its segment b, so that within a band all CTAs walk the
// column tiles in the same order and a B tile that one CTA reads from HBM the others
// read from L2 (for clouds whose operands exceed L2). Remainder: the W = (R - nb G) T
// units of the last row blocks in row-major order, spread over the first Gr = min(W, G)
// CTAs, CTA c owning [c W / Gr, (c + 1) W / Gr), cut at row-block boundaries into the
// segments nb, nb + 1, ... With R < G (nb = 0) this is a plain contiguous split.
struct Seg {
  int r, t0, t1;
};
struct Split {
  int R, T, G, nb, Gr;
  int64_t W;  // remainder units
};
__host__ __device__ inline Split make_split(int R, int T, int G) {
  Split s;
  s.R = R;
  s.T = T;
  s.G = G;
  s.nb = R / G;
  s.W = (int64_t)(R - s.nb * G) * T;
  s.Gr = (int)(s.W < (int64_t)G ? s.W : (int64_t)G);
  return s;
}
__host__ __device__ inline int64_t work_begin(const Split& s, int c) {
  return c >= s.Gr ? s.W : (int64_t)c * s.W / s.Gr;
}
// CTA owning remainder unit w (0 <= w < W): the largest c with floor(c W / Gr) <= w.
__host__ __device__ inline int cta_of(const Split& s, int64_t w) { return (int)(((w + 1) * s.Gr - 1) / s.W); }
__host__ __device__ inline int num_segments(const Split& s, int c) {
  const int64_t w0 = work_begin(s, c), w1 = work_begin(s, c + 1);
  return s.nb + (w1 <= w0 ? 0 : (int)((w1 - 1) / s.T - w0 / s.T + 1));
}
__host__ __device__ inline Seg segment(const Split& s, int c, int k) {
  Seg sg;
  if (k < s.nb) {
    sg.r = k * s.G + c;
    sg.t0 = 0;
    sg.t1 = s.T;
    return sg;
  }
  const int64_t w0 = work_begin(s, c), w1 = work_begin(s, c + 1);
  const int64_t rr = w0 / s.T + (k - s.nb);
  const int64_t rb0 = rr * s.T;
  sg.r = s.nb * s.G + (int)rr;
  sg.t0 = (int)((w0 > rb0 ? w0 : rb0) - rb0);
  sg.t1 = (int)((w1 < rb0 + s.T ? w1 : rb0 + s.T) - rb0);
  return sg;
}
// The CTAs whose segments cover row block r are c_first .. c_last (in CTA order); the
// segment index of CTA cc in row block r is seg_of(s, r, cc).
__host__ __device__ inline void contributors(const Split& s, int r, int* c_first, int* c_last) {
  if (r < s.nb * s.G) {
    *c_first = *c_last = r % s.G;
    return;
  }
  const int64_t rr = r - s.nb * s.G;
  *c_first = cta_of(s, rr * s.T);
  *c_last = cta_of(s, rr * s.T + s.T - 1);
}
__host__ __device__ inline int seg_of(const Split& s, int r, int cc) {
  if (r < s.nb * s.G) return r / s.G;
  return s.nb + (r - s.nb * s.G) - (int)(work_begin(s, cc) / s.T);
}

// Named barriers: 1 = both LSE warpgroups (256 threads), 2 = LSE warpgroup 0 (128).
// Arrival on a grid-wide counter with acquire-release semantics at GPU scope: orders
// this CTA's prior writes (made visible to the calling thread by a CTA barrier) before
// the increment, and the other arrivals' writes before this thread's later reads.
__device__ __forceinline__ unsigned atomic_add_acq_rel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

}  // namespace tc
}  // namespace progot
