// Epilogue shared by the log-sum-exp sweep kernels: per-row outputs after the
// deterministic combine of the column splits, the block-wide float64 error sum and
// the device-side Sinkhorn stop decision.
#pragma once

#include "progot_common.cuh"

namespace progot {

// Block-wide float64 sum (deterministic order). Returns the total in thread 0.
template <int kThreads>
__device__ __forceinline__ double block_sum_f64(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
  return tot;
}

// Sum of the per-row-block error partials in a fixed order by one full warp (lane l
// takes blocks l, l + 32, ... in order, then a fixed shuffle tree); every lane returns
// the same total.
__device__ __forceinline__ double sum_errpart_warp(const double* errpart, int nblocks) {
  const int lane = threadIdx.x & 31;
  double err = 0.0;
  for (int b = lane; b < nblocks; b += 32) err += __ldcg(errpart + b);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) err += __shfl_xor_sync(0xffffffffu, err, off);
  return err;
}

// The stop test of Alg. 1 after an f-update whose row-marginal error is err: a
// non-finite error, err <= tau, max_iter or a stall stop the loop; otherwise the new f
// becomes current and the iteration (the f-update and the g-update that follows it,
// which changes no state) is counted.
__device__ __forceinline__ void f_update_transition(SolverState& st, double err, const SweepParams& p) {
  st.err = err;
  const int it = st.it;
  if (!isfinite(err)) {
    st.status = kNumeric;
    st.done = 1;
  } else if (err <= p.tau) {
    st.status = kConverged;
    st.done = 1;
  } else if (it >= p.max_iter) {
    st.status = kMaxIter;
    st.done = 1;
  } else {
    if (err < 0.99 * st.best_err) {
      st.best_err = err;
      st.best_it = it;
    } else if (p.stall_window > 0 && it - st.best_it >= p.stall_window) {
      st.status = kStalled;
      st.done = 1;
    }
    if (!st.done) {
      st.fcur ^= 1;
      st.it += 1;
    }
  }
}

// Called by one full warp of the last CTA of the whole sweep: sum the error partials
// and, for an f-update (roles 1 and 3), advance the device-side Sinkhorn state (lane 0).
__device__ __forceinline__ void finish_sweep_warp(const SweepParams& p, int nblocks) {
  const double err = sum_errpart_warp(p.errpart, nblocks);
  if ((threadIdx.x & 31) != 0) return;
  p.errpart[nblocks] = err;
  if (p.state == nullptr || !(p.role == 1 || p.role == 3)) return;
  SolverState st = *p.state;
  f_update_transition(st, err, p);
  *p.state = st;
}

// Per-row inputs of the epilogue, loaded before the split combine so that their
// latency overlaps it.
struct RowIn {
  float an;    // |a_i|^2 (potential and marginal modes)
  float pot;   // current potential of row i (f-update error, marginal mode)
  float w;     // weight a_i
};

__device__ __forceinline__ RowIn row_inputs(const SweepParams& p, int64_t i, const float* potA_cur) {
  RowIn r;
  r.an = (p.mode != kModeLse && p.An) ? p.An[i] : 0.f;
  r.pot = (potA_cur != nullptr && (p.mode == kModeMarginal || p.mode == kModeMetrics || p.role == 1 || p.role == 3))
              ? potA_cur[i]
              : 0.f;
  r.w = p.wA ? p.wA[i] : (float)p.inv_nA;
  return r;
}

// Epilogue for one row given L = log2 sum_j 2^{t_ij}. Writes the row's output, returns
// its error term and the written value in *val. The error terms are float32 (they only
// feed the stop test against tau): on GB300 every float64 instruction of this epilogue
// sits on the sweep's critical path at a small fraction of the float32 rate.
//   potential: f_i = eps log w_i + |a_i|^2 - eps ln2 L, assembled in float64 adds and
//              multiplies; error a_i |exp((f_old - f_new)/eps) - 1| with expm1 of the
//              small float32 difference; the symmetric update (role 3) stores the
//              average (f_old + f_new) / 2 and measures the error at f_old;
//   marginal:  r_i = exp((pot_i - |a_i|^2)/eps + ln2 L), the exponent formed in float64
//              (it is a difference of large terms) and exponentiated in float32.
__device__ __forceinline__ float row_epilogue(const SweepParams& p, int64_t i, float L, const RowIn& in,
                                              float* out_target, float* val) {
  if (p.mode == kModePotential) {
    const double logw = p.wA ? (double)__logf(in.w) : p.log_w_uniform;
    const float fnew = (float)(p.eps * logw + (double)in.an - p.eps * kLn2 * (double)L);
    const float fout = (p.role == 3) ? 0.5f * (in.pot + fnew) : fnew;
    out_target[i] = fout;
    *val = fout;
    if (p.role == 1 || p.role == 3) {
      // a_i exp(d) is the row sum of P at the current f; far from feasibility (a warm
      // start at small eps) it overflows float32. Such a term only has to exceed tau,
      // so d is capped at 80 (the term stays below 1e35); a NaN stays NaN.
      float d = (in.pot - fnew) * p.inv_eps_f;
      if (d > 80.f) d = 80.f;
      return in.w * fabsf(expm1f(d));
    }
    return 0.f;
  }
  if (p.mode == kModeLse) {
    out_target[i] = L;
    *val = L;
    return 0.f;
  }
  // marginal
  const double arg = ((double)in.pot - (double)in.an) / p.eps + kLn2 * (double)L;
  const float r = expf((float)arg);
  if (out_target) out_target[i] = r;
  *val = r;
  return fabsf(r - in.w);
}

}  // namespace progot
