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

// Called by the last CTA of the whole sweep (thread 0): sum the per-row-block error
// partials in order and advance the device-side Sinkhorn state.
__device__ __forceinline__ void finish_sweep(const SweepParams& p, int nblocks) {
  double err = 0.0;
  for (int b = 0; b < nblocks; ++b) err += __ldcg(p.errpart + b);
  p.errpart[nblocks] = err;
  SolverState* st = p.state;
  if (st == nullptr) return;
  if (p.role == 1) {
    st->err = err;
    const int it = st->it;
    if (!isfinite(err)) {
      st->status = kNumeric;
      st->done = 1;
    } else if (err <= p.tau) {
      st->status = kConverged;
      st->done = 1;
    } else if (it >= p.max_iter) {
      st->status = kMaxIter;
      st->done = 1;
    } else {
      if (err < 0.99 * st->best_err) {
        st->best_err = err;
        st->best_it = it;
      } else if (p.stall_window > 0 && it - st->best_it >= p.stall_window) {
        st->status = kStalled;
        st->done = 1;
      }
      if (!st->done) st->fcur ^= 1;  // the new f becomes current
    }
  } else if (p.role == 2) {
    st->it += 1;
  }
}

// Epilogue for one row given L (log2 units). Returns the row's error term.
__device__ __forceinline__ double row_epilogue(const SweepParams& p, int64_t i, float L, const float* potA_cur,
                                               float* out_target) {
  const double w = p.wA ? (double)p.wA[i] : p.inv_nA;
  if (p.mode == kModePotential) {
    const float fnew = (float)(p.eps * log(w) + (double)p.An[i] - p.eps * kLn2 * (double)L);
    out_target[i] = fnew;
    if (p.role == 1) {
      const double fold = (double)potA_cur[i];
      return w * fabs(exp((fold - (double)fnew) / p.eps) - 1.0);
    }
    return 0.0;
  }
  if (p.mode == kModeLse) {
    out_target[i] = L;
    return 0.0;
  }
  // marginal
  const double r = exp(((double)potA_cur[i] - (double)p.An[i]) / p.eps + kLn2 * (double)L);
  if (out_target) out_target[i] = (float)r;
  return fabs(r - w);
}

}  // namespace progot
