// CUDA-core (float32 FMA) sweeps of the ProgOT hot path.
//
// lse_sweep_fp32: for every row a_i of A, L_i = log2 sum_j 2^{t_ij} with
//   t_ij = (2 a_i . b_j + potB_j - |b_j|^2) * log2(e) / eps,
// i.e. the soft-min of Sec. 2 over the squared Euclidean cost with the row constant
// |a_i|^2 factored out. The cost matrix is never stored: each CTA owns BM = 128 rows
// and streams BN = 128 columns at a time through shared memory, computing the 128 x 128
// tile of dot products with a register-blocked (8 x 8 per thread) float32 FMA loop and
// folding it into an online (max, sum) per row. Columns are split over gridDim.y; the
// last CTA to finish a row block combines the splits in split order (deterministic)
// and applies the epilogue (Sinkhorn update with the fused marginal-error term of
// Alg. 1, raw L, or the coupling marginal).
//
// map_sweep_fp32: the barycentric projection of Alg. 2 / Alg. 3: with L_i known,
//   T_i = sum_j 2^{t_ij - L_i} y_j / sum_j 2^{t_ij - L_i},
//   x_i <- x_i + alpha (T_i - x_i).
#include "progot_common.cuh"
#include "progot_internal.h"
#include "sweep_epilogue.cuh"

namespace progot {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;
constexpr int DCH = 64;  // columns of d handled per CTA by the map sweep

// Load one BK-wide chunk of `rows` rows (starting at r0) of a row-major (nrows x d)
// matrix into registers; zero outside [0, nrows) x [0, d).
struct ChunkLoader {
  float4 v[2];
  // Element e = threadIdx.x + NT * q maps to row r = e % BM and 4-wide k group
  // kq = e / BM, so that consecutive threads store consecutive rows of the transposed
  // shared tile (conflict-free stores).
  __device__ __forceinline__ void load(const float* __restrict__ M, int64_t nrows, int d, int64_t r0, int k0,
                                       bool vec_ok) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = threadIdx.x + NT * q;  // 0..511
      const int r = e & (BM - 1), kq = e / BM;
      const int64_t gr = r0 + r;
      const int k = k0 + kq * 4;
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < nrows) {
        const float* src = M + gr * (int64_t)d + k;
        if (vec_ok) {
          if (k < d) val = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          if (k + 0 < d) val.x = __ldg(src + 0);
          if (k + 1 < d) val.y = __ldg(src + 1);
          if (k + 2 < d) val.z = __ldg(src + 2);
          if (k + 3 < d) val.w = __ldg(src + 3);
        }
      }
      v[q] = val;
    }
  }
  // store transposed: S[k][row]
  __device__ __forceinline__ void store(float (*S)[BM]) const {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = threadIdx.x + NT * q;
      const int r = e & (BM - 1), kq = e / BM;
      S[kq * 4 + 0][r] = v[q].x;
      S[kq * 4 + 1][r] = v[q].y;
      S[kq * 4 + 2][r] = v[q].z;
      S[kq * 4 + 3][r] = v[q].w;
    }
  }
};

struct GemmSmem {
  float As[2][BK][BM];
  float Bs[2][BK][BN];
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One coordinate's contribution to the pair term of the sweep: a . b for the squared
// Euclidean cost (the norms enter through the bias), |a - b|^p for the p-norm costs.
template <int kCost>
__device__ __forceinline__ float pair_term(float a, float b, float acc, float cp) {
  if constexpr (kCost == kCostSqEuclid) {
    return fmaf(a, b, acc);
  } else if constexpr (kCost == kCostP15) {
    const float z = fabsf(a - b);
    return fmaf(z, sqrt_approx(z), acc);
  } else {
    const float z = fabsf(a - b);  // |z|^p = 2^(p log2 |z|); z = 0 gives 2^-inf = 0
    return acc + fast_exp2(cp * __log2f(z));
  }
}

// acc[r][c] = sum_k pair_term(a_row(r)_k, b_col(c)_k) for the thread's 8 x 8 block of a
// 128 x 128 tile (a_row . b_col for the squared Euclidean cost). Rows of the thread:
// ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns likewise with tx. Coordinates beyond d
// are zero on both sides and add nothing.
template <int kCost>
__device__ __forceinline__ void tile_accumulate(GemmSmem& sm, const float* __restrict__ A, int64_t nA,
                                                const float* __restrict__ B, int64_t nB, int d, int64_t row0,
                                                int64_t col0, bool vec_ok, float cp, float (&acc)[8][8]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  const int nk = (d + BK - 1) / BK;
  ChunkLoader la, lb;
  la.load(A, nA, d, row0, 0, vec_ok);
  lb.load(B, nB, d, col0, 0, vec_ok);
  __syncthreads();  // previous users of buffer 0 are done
  la.store(sm.As[0]);
  lb.store(sm.Bs[0]);
  __syncthreads();
  for (int kc = 0; kc < nk; ++kc) {
    const int buf = kc & 1;
    if (kc + 1 < nk) {
      la.load(A, nA, d, row0, (kc + 1) * BK, vec_ok);
      lb.load(B, nB, d, col0, (kc + 1) * BK, vec_ok);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&sm.As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&sm.As[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kk][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = pair_term<kCost>(av[r], bv[c], acc[r][c], cp);
    }
    if (kc + 1 < nk) {
      la.store(sm.As[buf ^ 1]);
      lb.store(sm.Bs[buf ^ 1]);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void tile_dots(GemmSmem& sm, const float* __restrict__ A, int64_t nA,
                                          const float* __restrict__ B, int64_t nB, int d, int64_t row0,
                                          int64_t col0, bool vec_ok, float (&acc)[8][8]) {
  tile_accumulate<kCostSqEuclid>(sm, A, nA, B, nB, d, row0, col0, vec_ok, 0.f, acc);
}

__device__ __forceinline__ int thread_row(int r) {  // 0..127
  const int ty = threadIdx.x >> 4;
  return (r < 4) ? ty * 4 + r : 64 + ty * 4 + (r - 4);
}
__device__ __forceinline__ int thread_col(int c) {
  const int tx = threadIdx.x & 15;
  return (c < 4) ? tx * 4 + c : 64 + tx * 4 + (c - 4);
}

// (max, sum, tilted sum) of one row's exponentials in log2 units: with M the max,
// S = sum_j 2^{t_j - M} and W = sum_j 2^{t_j - M} (t_j - M), so that the 2^t-weighted
// mean of t is M + W / S. Combining two triples rescales both to the larger max.
__device__ __forceinline__ float3 tilt_combine(float3 p, float3 q) {
  const float M = fmaxf(p.x, q.x);
  if (M == -INFINITY) return make_float3(-INFINITY, 0.f, 0.f);
  float s = 0.f, w = 0.f;
  if (p.x != -INFINITY) {
    const float c = exp2f(p.x - M);
    s += p.y * c;
    w += c * fmaf(p.y, p.x - M, p.z);
  }
  if (q.x != -INFINITY) {
    const float c = exp2f(q.x - M);
    s += q.y * c;
    w += c * fmaf(q.y, q.x - M, q.z);
  }
  return make_float3(M, s, w);
}

// Rescale a plain weighted sum from the max mp to the max M of a combine (0 when empty).
__device__ __forceinline__ float rescaled(float w, float mp, float M) {
  return (mp == -INFINITY) ? 0.f : w * exp2f(mp - M);
}

// kTilt adds the tilted sum W per row (coupling metrics) and, when p.Ac is given, the
// plain sum V = sum_j 2^{t_ij - M} c(ac_i, b_j) of the cost from another cloud (the
// cost tile is computed first and parked in dynamic shared memory, one entry per
// thread-owned pair); otherwise the plain sweep.
// kCost selects the pair term (the squared Euclidean dot product or a p-norm cost).
template <bool kTilt, int kCost>
__global__ void __launch_bounds__(NT, kTilt ? 1 : 2) lse_sweep_fp32(SweepParams p) {
  if (p.state != nullptr && p.state->done) return;
  __shared__ GemmSmem sm;
  __shared__ float beta_s[BN];
  __shared__ float bn_s[BN];
  __shared__ double red[NT / 32];
  __shared__ int s_last;
  extern __shared__ float cost_tile[];  // [BN][BM] in the cross-cloud metrics mode
  const bool cross = kTilt && p.Ac != nullptr;

  const int fcur = p.state ? p.state->fcur : 0;
  const float* potB = (p.potB_alt && fcur == 1) ? p.potB_alt : p.potB;
  const int tx = threadIdx.x & 15;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int ntiles = (int)((p.nB + BN - 1) / BN);
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int t_end = min(ntiles, t_begin + p.tiles_per_split);
  const bool vec_ok = ((p.d & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.A) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(p.B) & 15) == 0);

  float m_run[8], s_run[8], w_run[8], v_run[8], acn[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    m_run[r] = -INFINITY;
    s_run[r] = 0.f;
    w_run[r] = 0.f;
    v_run[r] = 0.f;
    acn[r] = 0.f;
    if constexpr (kTilt && kCost == kCostSqEuclid) {
      const int64_t i = row0 + thread_row(r);
      if (cross && i < p.nA) acn[r] = p.Acn[i];
    }
  }
  float acc[8][8];
  for (int tile = t_begin; tile < t_end; ++tile) {
    const int64_t col0 = (int64_t)tile * BN;
    __syncthreads();  // beta_s of the previous tile is no longer read
    if (threadIdx.x < BN) {
      const int64_t j = col0 + threadIdx.x;
      float bn = 0.f;  // |b_j|^2 enters only the squared Euclidean bias (Bn is NULL otherwise)
      if constexpr (kCost == kCostSqEuclid) {
        if (j < p.nB) bn = p.Bn[j];
      }
      beta_s[threadIdx.x] = (j < p.nB) ? (potB[j] - bn) * p.bscale : -INFINITY;
      bn_s[threadIdx.x] = bn;
    }
    if constexpr (kTilt) {
      if (cross) {
        // cost of the cost cloud against this tile, each thread keeping its own 8 x 8
        tile_accumulate<kCost>(sm, p.Ac, p.nA, p.B, p.nB, p.d, row0, col0, vec_ok, p.cost_p, acc);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float cv = (kCost == kCostSqEuclid) ? fmaf(-2.f, acc[r][c], acn[r] + bn_s[thread_col(c)])
                                                      : acc[r][c] / p.cost_p;
            cost_tile[thread_col(c) * BM + thread_row(r)] = cv;
          }
      }
    }
    tile_accumulate<kCost>(sm, p.A, p.nA, p.B, p.nB, p.d, row0, col0, vec_ok, p.cost_p, acc);  // ends with a sync
    float bcol[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) bcol[c] = beta_s[thread_col(c)];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float t[8];
      float tmax = -INFINITY;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        t[c] = fmaf(acc[r][c], p.scale, bcol[c]);
        tmax = fmaxf(tmax, t[c]);
      }
      const float mnew = fmaxf(m_run[r], tmax);
      if (mnew != -INFINITY) {
        const float resc = fast_exp2(m_run[r] - mnew);  // 0 while the row is still empty
        float s = s_run[r] * resc;
        if constexpr (kTilt) {
          float w = (m_run[r] == -INFINITY) ? 0.f : resc * fmaf(s_run[r], m_run[r] - mnew, w_run[r]);
          float v = v_run[r] * resc;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float e = fast_exp2(t[c] - mnew);
            s += e;
            // padded columns have t = -inf and e = 0; the clamp keeps 0 * (-inf) out
            w = fmaf(e, fmaxf(t[c] - mnew, -256.f), w);
            // padded columns: e = 0 and a finite cost entry
            if (cross) v = fmaf(e, cost_tile[thread_col(c) * BM + thread_row(r)], v);
          }
          w_run[r] = w;
          v_run[r] = v;
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) s += fast_exp2(t[c] - mnew);
        }
        s_run[r] = s;
        m_run[r] = mnew;
      }
    }
  }
  // reduce over the 16 threads that share rows (lanes tx = 0..15 of a half warp)
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if constexpr (kTilt) {
      float3 v = make_float3(m_run[r], s_run[r], w_run[r]);
      float vc = v_run[r];
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) {
        float3 o;
        o.x = __shfl_xor_sync(0xffffffffu, v.x, off);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, off);
        o.z = __shfl_xor_sync(0xffffffffu, v.z, off);
        const float oc = __shfl_xor_sync(0xffffffffu, vc, off);
        const float3 mrg = tilt_combine(v, o);
        vc = rescaled(vc, v.x, mrg.x) + rescaled(oc, o.x, mrg.x);
        v = mrg;
      }
      if (tx == 0) {
        const int64_t i = row0 + thread_row(r);
        if (i < p.nA) {
          p.partial[(int64_t)blockIdx.y * p.nA + i] = make_float2(v.x, v.y);
          p.wpart[(int64_t)blockIdx.y * p.nA + i] = v.z;
          if (cross) p.cpart[(int64_t)blockIdx.y * p.nA + i] = vc;
        }
      }
    } else {
      float2 v = make_float2(m_run[r], s_run[r]);
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v.x, off);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, off);
        v = lse_combine(v, o);
      }
      if (tx == 0) {
        const int64_t i = row0 + thread_row(r);
        if (i < p.nA) p.partial[(int64_t)blockIdx.y * p.nA + i] = v;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&p.cnt[blockIdx.x], 1u);
    s_last = (prev == (unsigned)(p.splits - 1));
  }
  __syncthreads();
  if (!s_last) return;

  // ---- last CTA of this row block: combine splits in order, epilogue
  const float* potA_cur = p.potA_old;
  float* out_target = p.out;
  if (p.role == 1 || p.role == 3) {
    potA_cur = (fcur == 0) ? p.out : p.out_alt;
    out_target = (fcur == 0) ? p.out_alt : p.out;
  }
  double e = 0.0;
  if constexpr (kTilt) {
    // coupling metrics of the rows of this block: with base_i = (pot_i - |a_i|^2) / eps,
    // log P_ij = base_i + ln2 t_ij, so r_i = exp(base_i + ln2 L_i) and
    // sum_j P_ij log P_ij = r_i (base_i + ln2 tbar_i), tbar_i = M + W / S
    double q[kMetricSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (threadIdx.x < BM) {
      const int64_t i = row0 + threadIdx.x;
      if (i < p.nA) {
        const RowIn in = row_inputs(p, i, potA_cur);
        float3 v = make_float3(-INFINITY, 0.f, 0.f);
        float vc = 0.f;
        for (int s = 0; s < p.splits; ++s) {
          const float2 ms = __ldcg(&p.partial[(int64_t)s * p.nA + i]);
          const float3 in3 = make_float3(ms.x, ms.y, __ldcg(&p.wpart[(int64_t)s * p.nA + i]));
          const float3 mrg = tilt_combine(v, in3);
          if (cross) vc = rescaled(vc, v.x, mrg.x) + rescaled(__ldcg(&p.cpart[(int64_t)s * p.nA + i]), in3.x, mrg.x);
          v = mrg;
        }
        double r = 0.0, plogp = 0.0, pc = 0.0;
        if (v.y > 0.f) {
          const double base = ((double)in.pot - (double)in.an) / p.eps;
          const double L = (double)v.x + (double)__log2f(v.y);
          r = (double)expf((float)(base + kLn2 * L));
          const double tbar = (double)v.x + (double)v.z / (double)v.y;
          plogp = r * (base + kLn2 * tbar);
          pc = r * (double)vc / (double)v.y;
        }
        if (out_target) out_target[i] = (float)r;
        q[kSumErr] = fabs(r - (double)in.w);
        q[kSumMass] = r;
        q[kSumPotR] = (double)in.pot * r;
        q[kSumPlogP] = plogp;
        q[kSumPotW] = (double)in.pot * (double)in.w;
        q[kSumPC] = pc;
      }
    }
    e = q[kSumErr];
#pragma unroll
    for (int k = 0; k < kMetricSums; ++k) {
      const double t = block_sum_f64<NT>(q[k], red);
      if (threadIdx.x == 0) p.metpart[(int64_t)blockIdx.x * kMetricSums + k] = t;
    }
  } else {
    if (threadIdx.x < BM) {
      const int64_t i = row0 + threadIdx.x;
      if (i < p.nA) {
        const RowIn in = row_inputs(p, i, potA_cur);
        float2 v = make_float2(-INFINITY, 0.f);
        for (int s = 0; s < p.splits; ++s) v = lse_combine(v, __ldcg(&p.partial[(int64_t)s * p.nA + i]));
        const float L = v.x + __log2f(v.y);
        float val;
        e = row_epilogue(p, i, L, in, out_target, &val);
      }
    }
  }
  const double tot = block_sum_f64<NT>(e, red);
  if (threadIdx.x == 0) {
    p.errpart[blockIdx.x] = tot;
    p.cnt[blockIdx.x] = 0;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&p.cnt[gridDim.x], 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x < 32) {
    __threadfence();
    finish_sweep_warp(p, gridDim.x);
    if (threadIdx.x == 0) p.cnt[gridDim.x] = 0;
  }
}

// ---------------------------------------------------------------- map sweep
struct MapSmem {
  GemmSmem g;
  float Ps[BN][BM];   // P tile stored transposed: Ps[c][r]
  float Ys[BN][DCH];  // d-chunk of the B tile for the P . Y product
};

size_t map_sweep_fp32_smem() { return sizeof(MapSmem); }

__global__ void __launch_bounds__(NT, 1) map_sweep_fp32(MapParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MapSmem& sm = *reinterpret_cast<MapSmem*>(smem_raw);
  __shared__ float beta_s[BN];
  __shared__ float Lrow[BM];
  __shared__ float den[BM];
  __shared__ int s_last;

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int dch0 = blockIdx.z * DCH;
  const int ntiles = (int)((p.nB + BN - 1) / BN);
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int t_end = min(ntiles, t_begin + p.tiles_per_split);
  const bool vec_ok = ((p.d & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.A) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(p.B) & 15) == 0);
  if (threadIdx.x < BM) {
    const int64_t i = row0 + threadIdx.x;
    Lrow[threadIdx.x] = (i < p.nA) ? p.L[i] : 0.f;
  }
  float o[8][4];
  float rs[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    rs[r] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) o[r][c] = 0.f;
  }
  float acc[8][8];
  for (int tile = t_begin; tile < t_end; ++tile) {
    const int64_t col0 = (int64_t)tile * BN;
    __syncthreads();  // the previous tile's Ps / Ys / beta_s are no longer read
    if (threadIdx.x < BN) {
      const int64_t j = col0 + threadIdx.x;
      beta_s[threadIdx.x] = (j < p.nB) ? (p.potB[j] - p.Bn[j]) * p.bscale : -INFINITY;
    }
    for (int e = threadIdx.x; e < BN * DCH; e += NT) {
      const int c = e / DCH, k = e % DCH;
      const int64_t j = col0 + c;
      const int kk = dch0 + k;
      sm.Ys[c][k] = (j < p.nB && kk < p.d) ? __ldg(p.B + j * (int64_t)p.d + kk) : 0.f;
    }
    tile_dots(sm.g, p.A, p.nA, p.B, p.nB, p.d, row0, col0, vec_ok, acc);  // syncs at entry and exit
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int rr = thread_row(r);
      const float Lr = Lrow[rr];
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = thread_col(c);
        const float pv = fast_exp2(fmaf(acc[r][c], p.scale, beta_s[cc]) - Lr);
        sm.Ps[cc][rr] = pv;
        part += pv;
      }
      rs[r] += part;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < BN; ++c) {
      const float4 p0 = *reinterpret_cast<const float4*>(&sm.Ps[c][ty * 4]);
      const float4 p1 = *reinterpret_cast<const float4*>(&sm.Ps[c][64 + ty * 4]);
      const float4 yv = *reinterpret_cast<const float4*>(&sm.Ys[c][tx * 4]);
      const float pr[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
      const float yk[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) o[r][k] = fmaf(pr[r], yk[k], o[r][k]);
    }
  }
  // row sums of P over this split: sum the 16 column groups of a half warp
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float v = rs[r];
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    rs[r] = v;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = row0 + thread_row(r);
    if (i >= p.nA) continue;
    float* dst = p.Opart + ((int64_t)blockIdx.y * p.nA + i) * p.d;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int kk = dch0 + tx * 4 + k;
      if (kk < p.d) dst[kk] = o[r][k];
    }
    if (blockIdx.z == 0 && tx == 0) p.Rpart[(int64_t)blockIdx.y * p.nA + i] = rs[r];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&p.cnt[blockIdx.x], 1u);
    s_last = (prev == (unsigned)(p.splits * p.dchunks - 1));
  }
  __syncthreads();
  if (!s_last) return;
  // ---- last CTA of this row block: T_i = sum_s O_s / sum_s R_s, x <- x + alpha (T - x)
  if (threadIdx.x < BM) {
    const int64_t i = row0 + threadIdx.x;
    float dsum = 0.f;
    if (i < p.nA)
      for (int s = 0; s < p.splits; ++s) dsum += __ldcg(p.Rpart + (int64_t)s * p.nA + i);
    den[threadIdx.x] = dsum;
  }
  __syncthreads();
  const int64_t rem = p.nA - row0;
  const int rows = rem < BM ? (int)rem : BM;
  // eight elements per thread per round: x first, then the split sums with the loads of
  // a split issued together, then the stores (out aliases x: a store between loads
  // would serialise them); the splits are added in split order as before
  const int total = rows * p.d;
  for (int e0 = threadIdx.x; e0 < total; e0 += NT * 8) {
    float num[8], xs[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      num[u] = 0.f;
      xs[u] = 0.f;
      const int e = e0 + NT * u;
      if (e < total) xs[u] = p.A[row0 * (int64_t)p.d + e];
    }
    for (int s = 0; s < p.splits; ++s) {
      const float* src = p.Opart + ((int64_t)s * p.nA + row0) * p.d;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + NT * u;
        if (e < total) num[u] += __ldcg(src + e);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + NT * u;
      if (e >= total) continue;
      const int r = e / p.d, k = e % p.d;
      const float x = xs[u];
      const float T = num[u] / den[r];
      p.out[row0 * (int64_t)p.d + e] = fmaf(p.alpha, T - x, x);
      (void)k;
    }
  }
  if (threadIdx.x == 0) p.cnt[blockIdx.x] = 0;
}

// ---------------------------------------------------------------- launchers
// ------------------------------------------------------- p-norm map and cost sum
// grad h of the p-norm cost, one coordinate: sign(z) |z|^(p-1).
template <int kCost>
__device__ __forceinline__ float grad_h_coord(float z, float cp) {
  const float az = fabsf(z);
  if constexpr (kCost == kCostP15) {
    return copysignf(sqrt_approx(az), z);
  } else {
    return copysignf(fast_exp2((cp - 1.f) * __log2f(az)), z);
  }
}

// grad h* of the p-norm cost, one coordinate: sign(w) |w|^(1/(p-1)).
template <int kCost>
__device__ __forceinline__ float grad_h_star_coord(float w, float cp) {
  const float aw = fabsf(w);
  if constexpr (kCost == kCostP15) {
    return w * aw;
  } else {
    return copysignf(exp2f(__log2f(aw) / (cp - 1.f)), w);
  }
}

// The barycentric displacement of Alg. 2 / Alg. 3 for the p-norm cost: with L_i known,
// Q_ij = 2^{t_ij - L_i} / sum_j 2^{t_ij - L_i}, t_ij = (g_j - h(x_i - y_j)) log2(e) / eps,
//   Z_i = grad h*(sum_j Q_ij grad h(x_i - y_j)),  x_i <- x_i - alpha Z_i.
// Unlike the squared Euclidean map the inner sum is not a product with Y: each thread
// evaluates grad h(x_ik - y_jk) for its 8 rows x 4 coordinates against every column of
// the tile (CUDA cores, one square root per term for p = 1.5). The cost tile, the P
// tile, the column splits and the last-CTA combine follow map_sweep_fp32.
template <int kCost>
__global__ void __launch_bounds__(NT, 1) map_sweep_pnorm(MapParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MapSmem& sm = *reinterpret_cast<MapSmem*>(smem_raw);
  __shared__ float beta_s[BN];
  __shared__ float Lrow[BM];
  __shared__ float den[BM];
  __shared__ int s_last;

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int dch0 = blockIdx.z * DCH;
  const int ntiles = (int)((p.nB + BN - 1) / BN);
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int t_end = min(ntiles, t_begin + p.tiles_per_split);
  const bool vec_ok = ((p.d & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.A) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(p.B) & 15) == 0);
  if (threadIdx.x < BM) {
    const int64_t i = row0 + threadIdx.x;
    Lrow[threadIdx.x] = (i < p.nA) ? p.L[i] : 0.f;
  }
  // this thread's coordinates of its rows (zero outside the cloud and beyond d)
  float xv[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = row0 + thread_row(r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int kk = dch0 + tx * 4 + k;
      xv[r][k] = (i < p.nA && kk < p.d) ? p.A[i * (int64_t)p.d + kk] : 0.f;
    }
  }
  float o[8][4];
  float rs[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    rs[r] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) o[r][c] = 0.f;
  }
  float acc[8][8];
  for (int tile = t_begin; tile < t_end; ++tile) {
    const int64_t col0 = (int64_t)tile * BN;
    __syncthreads();  // the previous tile's Ps / Ys / beta_s are no longer read
    if (threadIdx.x < BN) {
      const int64_t j = col0 + threadIdx.x;
      beta_s[threadIdx.x] = (j < p.nB) ? p.potB[j] * p.bscale : -INFINITY;
    }
    for (int e = threadIdx.x; e < BN * DCH; e += NT) {
      const int c = e / DCH, k = e % DCH;
      const int64_t j = col0 + c;
      const int kk = dch0 + k;
      sm.Ys[c][k] = (j < p.nB && kk < p.d) ? __ldg(p.B + j * (int64_t)p.d + kk) : 0.f;
    }
    tile_accumulate<kCost>(sm.g, p.A, p.nA, p.B, p.nB, p.d, row0, col0, vec_ok, p.cost_p, acc);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int rr = thread_row(r);
      const float Lr = Lrow[rr];
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = thread_col(c);
        const float pv = fast_exp2(fmaf(acc[r][c], p.scale, beta_s[cc]) - Lr);
        sm.Ps[cc][rr] = pv;
        part += pv;
      }
      rs[r] += part;
    }
    __syncthreads();
#pragma unroll 2
    for (int c = 0; c < BN; ++c) {
      const float4 p0 = *reinterpret_cast<const float4*>(&sm.Ps[c][ty * 4]);
      const float4 p1 = *reinterpret_cast<const float4*>(&sm.Ps[c][64 + ty * 4]);
      const float4 yv = *reinterpret_cast<const float4*>(&sm.Ys[c][tx * 4]);
      const float pr[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
      const float yk[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) o[r][k] = fmaf(pr[r], grad_h_coord<kCost>(xv[r][k] - yk[k], p.cost_p), o[r][k]);
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float v = rs[r];
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    rs[r] = v;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = row0 + thread_row(r);
    if (i >= p.nA) continue;
    float* dst = p.Opart + ((int64_t)blockIdx.y * p.nA + i) * p.d;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int kk = dch0 + tx * 4 + k;
      if (kk < p.d) dst[kk] = o[r][k];
    }
    if (blockIdx.z == 0 && tx == 0) p.Rpart[(int64_t)blockIdx.y * p.nA + i] = rs[r];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&p.cnt[blockIdx.x], 1u);
    s_last = (prev == (unsigned)(p.splits * p.dchunks - 1));
  }
  __syncthreads();
  if (!s_last) return;
  // ---- last CTA of this row block: Z_i = grad h*(sum_s O_s / sum_s R_s), x <- x - alpha Z
  if (threadIdx.x < BM) {
    const int64_t i = row0 + threadIdx.x;
    float dsum = 0.f;
    if (i < p.nA)
      for (int s = 0; s < p.splits; ++s) dsum += __ldcg(p.Rpart + (int64_t)s * p.nA + i);
    den[threadIdx.x] = dsum;
  }
  __syncthreads();
  const int64_t rem = p.nA - row0;
  const int rows = rem < BM ? (int)rem : BM;
  // eight elements per thread per round: x first, then the split sums with the loads of
  // a split issued together, then the stores (out aliases x: a store between loads
  // would serialise them); the splits are added in split order as before
  const int total = rows * p.d;
  for (int e0 = threadIdx.x; e0 < total; e0 += NT * 8) {
    float num[8], xs[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      num[u] = 0.f;
      xs[u] = 0.f;
      const int e = e0 + NT * u;
      if (e < total) xs[u] = p.A[row0 * (int64_t)p.d + e];
    }
    for (int s = 0; s < p.splits; ++s) {
      const float* src = p.Opart + ((int64_t)s * p.nA + row0) * p.d;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + NT * u;
        if (e < total) num[u] += __ldcg(src + e);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + NT * u;
      if (e >= total) continue;
      const int r = e / p.d, k = e % p.d;
      const float x = xs[u];
      const float Z = grad_h_star_coord<kCost>(num[u] / den[r], p.cost_p);
      p.out[row0 * (int64_t)p.d + e] = fmaf(-p.alpha, Z, x);
      (void)k;
    }
  }
  if (threadIdx.x == 0) p.cnt[blockIdx.x] = 0;
}

// Sum over all pairs of sum_k |x_ik - y_jk|^p (float64 per thread and per CTA, fixed
// order): gridDim.x CTAs stride over the 128 x 128 tiles.
template <int kCost>
__global__ void __launch_bounds__(NT, 2) pairwise_cost_sum(const float* __restrict__ X, int64_t n,
                                                           const float* __restrict__ Y, int64_t m, int32_t d,
                                                           float cp, double* __restrict__ partial) {
  __shared__ GemmSmem sm;
  __shared__ double red[NT / 32];
  const int64_t rb = (n + BM - 1) / BM, ct = (m + BN - 1) / BN;
  const bool vec_ok = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);
  double tot = 0.0;
  float acc[8][8];
  for (int64_t w = blockIdx.x; w < rb * ct; w += gridDim.x) {
    const int64_t row0 = (w / ct) * BM, col0 = (w % ct) * BN;
    tile_accumulate<kCost>(sm, X, n, Y, m, d, row0, col0, vec_ok, cp, acc);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t i = row0 + thread_row(r);
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t j = col0 + thread_col(c);
        if (i < n && j < m) part += acc[r][c];
      }
      tot += (double)part;
    }
  }
  const double b = block_sum_f64<NT>(tot, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

cudaError_t launch_lse_sweep_fp32(const SweepParams& p, cudaStream_t stream) {
  const int rb = (int)((p.nA + BM - 1) / BM);
  dim3 grid(rb, p.splits);
  const bool tilt = p.mode == kModeMetrics;
  // the cross-cloud metrics mode parks one cost tile in dynamic shared memory
  const size_t dyn = (tilt && p.Ac != nullptr) ? sizeof(float) * BN * BM : 0;
  if (tilt) {
    auto k = p.cost == kCostP15        ? lse_sweep_fp32<true, kCostP15>
             : p.cost == kCostPGeneral ? lse_sweep_fp32<true, kCostPGeneral>
                                       : lse_sweep_fp32<true, kCostSqEuclid>;
    if (dyn > 0) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
    }
    k<<<grid, NT, dyn, stream>>>(p);
  } else if (p.cost == kCostP15) {
    lse_sweep_fp32<false, kCostP15><<<grid, NT, 0, stream>>>(p);
  } else if (p.cost == kCostPGeneral) {
    lse_sweep_fp32<false, kCostPGeneral><<<grid, NT, 0, stream>>>(p);
  } else {
    lse_sweep_fp32<false, kCostSqEuclid><<<grid, NT, 0, stream>>>(p);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_map_sweep_fp32(const MapParams& p, cudaStream_t stream) {
  // per-thread flag: the attribute call is cheap and idempotent, so each host thread
  // sets it once without shared mutable state
  static thread_local bool attr_set = false;
  const size_t smem = sizeof(MapSmem);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(map_sweep_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int rb = (int)((p.nA + BM - 1) / BM);
  dim3 grid(rb, p.splits, p.dchunks);
  map_sweep_fp32<<<grid, NT, smem, stream>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int kCost>
static cudaError_t launch_map_pnorm_k(const MapParams& p, cudaStream_t stream) {
  static thread_local bool attr_set = false;
  const size_t smem = sizeof(MapSmem);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(map_sweep_pnorm<kCost>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int rb = (int)((p.nA + BM - 1) / BM);
  dim3 grid(rb, p.splits, p.dchunks);
  map_sweep_pnorm<kCost><<<grid, NT, smem, stream>>>(p);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_map_sweep_pnorm(const MapParams& p, cudaStream_t stream) {
  return p.cost == kCostP15 ? launch_map_pnorm_k<kCostP15>(p, stream) : launch_map_pnorm_k<kCostPGeneral>(p, stream);
}

cudaError_t launch_pairwise_cost_sum(const float* X, int64_t n, const float* Y, int64_t m, int32_t d, int32_t cost,
                                     float cost_p, double* partial, double* out, cudaStream_t s) {
  const int parts = reduce_parts();
  if (cost == kCostP15)
    pairwise_cost_sum<kCostP15><<<parts, NT, 0, s>>>(X, n, Y, m, d, cost_p, partial);
  else
    pairwise_cost_sum<kCostPGeneral><<<parts, NT, 0, s>>>(X, n, Y, m, d, cost_p, partial);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_parts(partial, parts, 1, out, s);
}

int fp32_tile_rows() { return BM; }
int fp32_tile_cols() { return BN; }
int map_dchunk() { return DCH; }

}  // namespace progot
