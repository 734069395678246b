// Shared device-side definitions of the ProgOT kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace progot {

constexpr double kLog2e = 1.4426950408889634;  // log2(e)
constexpr double kLn2 = 0.6931471805599453;    // ln(2)

// Epilogue of a row log-sum-exp sweep, applied once per row after the
// deterministic combine of the column splits. L_i = log2 sum_j 2^{t_ij}.
enum SweepMode : int32_t {
  kModePotential = 0,  // out_i = eps log w_i + |a_i|^2 - eps ln2 L_i (Sinkhorn update)
  kModeLse = 1,        // out_i = L_i (log2 units)
  kModeMarginal = 2,   // out_i = exp((pot_i - |a_i|^2)/eps + ln2 L_i)  (row sums of P)
  kModeMetrics = 3,    // marginal plus the per-row-block sums of the coupling metrics
};

// Per-row-block float64 sums written by a kModeMetrics sweep (metpart[block * kMetricSums + q]).
enum MetricSum : int32_t {
  kSumErr = 0,    // sum_i |r_i - w_i|
  kSumMass = 1,   // sum_i r_i
  kSumPotR = 2,   // sum_i pot_i r_i
  kSumPlogP = 3,  // sum_i sum_j P_ij log P_ij
  kSumPotW = 4,   // sum_i pot_i w_i
  kSumPC = 5,     // sum_i sum_j P_ij c(ac_i, b_j) against the cost cloud Ac (when given)
  kMetricSums = 6,
};

// Solver state kept on the device so that the Sinkhorn loop runs without a host
// round trip per iteration. All fields are written only by the last CTA of a sweep.
struct SolverState {
  int32_t it;         // completed (f, g) iterations
  int32_t done;       // nonzero: later sweeps return at entry
  int32_t status;     // kRunning / kConverged / kMaxIter / kNumeric / kStalled
  int32_t fcur;       // which of the two f buffers holds the current f
  int32_t best_it;    // iteration at which best_err last improved by 1%
  int32_t pad_[3];
  double err;         // last measured row-marginal L1 error
  double best_err;    // best error seen (stall detection)
};

enum SolverStatus : int32_t { kRunning = 0, kConverged = 1, kMaxIter = 2, kNumeric = 3, kStalled = 4 };

// Parameters of one sweep "rows of A against all rows of B".
struct SweepParams {
  const float* A;      // nA x d rows (the side whose potential is updated)
  const float* B;      // nB x d rows (summed over)
  const float* An;     // |a_i|^2, nA (float32 of a float64 sum)
  const float* Bn;     // |b_j|^2, nB
  const float* wA;     // weights of A (nA) or nullptr for uniform
  const float* potB;   // potential on B (g for the f-update), nB
  const float* potB_alt;  // second buffer of potB when it is chosen at run time (state->fcur)
  const float* potA_old;  // current potential on A (for the error / marginal), or nullptr
  const float* potA_alt;  // second buffer (state->fcur selects)
  float* out;          // nA outputs (see SweepMode)
  float* out_alt;      // second output buffer (state->fcur selects), or nullptr
  float2* partial;     // [splits][nA] (max, sum) in log2 units
  float* wpart;        // [splits][nA] tilted sums sum_j 2^{t_ij - max} (t_ij - max) (kModeMetrics)
  double* metpart;     // [row blocks][kMetricSums] (kModeMetrics)
  const float* Ac;     // kModeMetrics: nA x d cloud whose cost to B is integrated against P, or nullptr
  const float* Acn;    // |ac_i|^2 (squared Euclidean cost)
  float* cpart;        // [splits][nA] sums_j 2^{t_ij - max} c(ac_i, b_j) (when Ac is given)
  double* errpart;     // [row blocks] float64 error partials
  unsigned int* cnt;   // [row blocks + 1] arrival counters (zero between launches)
  SolverState* state;  // nullptr when the sweep is not part of a Sinkhorn loop
  int64_t nA, nB;
  int32_t d;
  int32_t splits;      // column splits (gridDim.y)
  int32_t tiles_per_split;
  int32_t mode;        // SweepMode
  int32_t role;        // 0 none, 1 f-update of a Sinkhorn loop (error + stop; it++ when the
                       //   loop goes on), 2 g-update (no state change),
                       // 3 symmetric self-transport update (A = B, potB = f): error + stop,
                       //   f <- (f + f_new) / 2 and it++
  int32_t max_iter;
  int32_t stall_window;
  // Stop test one sweep later (tensor-core Sinkhorn loops): the f-update of iteration
  // seq writes its error partials but no state; the g-update of iteration seq reads
  // state[seq & 1] and those partials, applies the f-update's stop test and writes
  // state[(seq + 1) & 1] (a no-op g-update when the loop has stopped). 0: the last CTA
  // of the f-update applies the test and state[0] is the only state.
  int32_t lag;
  int32_t seq;         // iteration of this sweep in its Sinkhorn loop (lag = 1)
  float scale;         // 2 log2(e) / eps: multiplies x . y
  float bscale;        // log2(e) / eps: multiplies (potB_j - |b_j|^2)
  double eps;
  float inv_eps_f;     // 1 / eps in float32 (the per-row error terms)
  double tau;
  double inv_nA;       // uniform weight 1/nA
  double log_w_uniform;  // log(1/nA)
  int32_t cost;        // CostKind: kCostSqEuclid uses scale * (a . b) + bscale (potB - |b|^2);
                       // the p-norm costs use scale * sum_k |a_k - b_k|^p + bscale potB
  float cost_p;        // p of the p-norm cost
};

// Cost of the sweeps. kCostSqEuclid: |x - y|^2 through the dot product (tensor cores or
// float32 FMAs); the p-norm cost h(z) = (1/p) sum_k |z_k|^p (Sec. 5.2) on CUDA cores,
// with p = 1.5 (|z| sqrt|z|) specialised.
enum CostKind : int32_t { kCostSqEuclid = 0, kCostP15 = 1, kCostPGeneral = 2 };

// Combine two partial log-sum-exps (max, sum) in log2 units.
__device__ __forceinline__ float2 lse_combine(float2 p, float2 q) {
  float M = fmaxf(p.x, q.x);
  if (M == -INFINITY) return make_float2(-INFINITY, 0.f);
  float s = p.y * exp2f(p.x - M) + q.y * exp2f(q.x - M);
  return make_float2(M, s);
}

__device__ __forceinline__ float fast_exp2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

}  // namespace progot
