// Internal (C++) interfaces between the host orchestration and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "progot_common.cuh"

namespace progot {

// Parameters of the barycentric-projection sweep (map step of Alg. 2 / Alg. 3).
struct MapParams {
  const float* A;      // nA x d current points (may alias out)
  const float* B;      // nB x d target points
  const float* Bn;     // |b_j|^2
  const float* potB;   // g
  const float* L;      // per-row log2-sum-exp of t_ij (from an LSE sweep)
  float* out;          // nA x d: x + alpha (T(x) - x)
  float* Opart;        // [splits][nA][d] partial numerators
  float* Rpart;        // [splits][nA] partial row sums of P
  unsigned int* cnt;   // [row blocks] arrival counters (zero between launches)
  int64_t nA, nB;
  int32_t d;
  int32_t splits, tiles_per_split, dchunks;
  float scale, bscale;
  float alpha;
  int32_t cost;        // CostKind (the p-norm map moves x by grad h*(sum_j Q_ij grad h(x - y_j)))
  float cost_p;
};

void count_launch();
// Text returned by progot_last_error_string() on the calling thread.
void set_last_error_message(const char* msg);

// float32 CUDA-core sweeps (sweep_fp32.cu)
cudaError_t launch_lse_sweep_fp32(const SweepParams& p, cudaStream_t stream);
cudaError_t launch_map_sweep_fp32(const MapParams& p, cudaStream_t stream);
// p-norm cost: barycentric displacement x <- x - alpha grad h*(sum_j Q_ij grad h(x_i - y_j))
cudaError_t launch_map_sweep_pnorm(const MapParams& p, cudaStream_t stream);
// out[0] = sum_ij h(x_i - y_j) for the p-norm cost (float64, fixed order; partial holds
// reduce_parts() doubles)
cudaError_t launch_pairwise_cost_sum(const float* X, int64_t n, const float* Y, int64_t m, int32_t d, int32_t cost,
                                     float cost_p, double* partial, double* out, cudaStream_t s);
int fp32_tile_rows();
int fp32_tile_cols();
int map_dchunk();

// small kernels (prep.cu)
cudaError_t launch_row_sqnorm(const float* X, int64_t n, int32_t d, float* out, cudaStream_t s);
// mu = (mean of the rows of X + mean of the rows of Y) / 2 (fixed-order float64 sums);
// partial: reduce_parts() * 2 * d doubles of scratch.
cudaError_t launch_center(const float* X, int64_t n, const float* Y, int64_t m, int32_t d, double* partial, float* mu,
                          cudaStream_t s);
// L_i = (eps log w_i + |a_i|^2 - f_i) / (eps ln2) from a potential an f-update wrote
// (w = NULL: log w_i = log_w_uniform).
cudaError_t launch_lse_from_potential(const float* f, const float* an, const float* w, double log_w_uniform,
                                      double eps, int64_t n, float* L, cudaStream_t s);
cudaError_t launch_lse_uncenter(float* L, const float* X, int64_t n, int32_t d, const float* mu, float bscale,
                                cudaStream_t s);
cudaError_t launch_scale(float* v, int64_t n, float factor, cudaStream_t s);
cudaError_t launch_init_state(SolverState* st, cudaStream_t s);
// out[0] = sum_i |x_i|^2, out[1 + k] = sum_i x_ik (float64; partial buffer of
// `parts` x (d + 1) doubles, deterministic two-pass reduction)
cudaError_t launch_moments(const float* X, int64_t n, int32_t d, double* partial, int parts, double* out,
                           cudaStream_t s);
// out[0] = sum_i ||a_i - b_i||^2 (float64, deterministic)
cudaError_t launch_sq_error(const float* A, const float* B, int64_t n, int32_t d, double* partial, int parts,
                            double* out, cudaStream_t s);
int reduce_parts();
// out[0] = sum_i P_ii, out[1] = sum_i log P_ii for n = m, log P_ii = (f_i + g_i - |x_i - y_i|^2)/eps;
// logd (optional) receives log P_ii in float32; partial holds parts x 2 doubles
cudaError_t launch_diag(const float* X, const float* Y, const float* f, const float* g, int64_t n, int32_t d, double eps,
                        float* logd, double* partial, int parts, double* out, cudaStream_t s);
// *out = mean_ij |x_i - y_j|^2 from launch_moments outputs mx (of X, n rows) and my (of Y, m rows)
cudaError_t launch_mean_cost_closed(const double* mx, const double* my, int64_t n, int64_t m, int32_t d, double* out,
                                    cudaStream_t s);
// out[k] = sum_b partial[b * width + k], b = 0..parts-1 in order
cudaError_t launch_sum_parts(const double* partial, int parts, int width, double* out, cudaStream_t s);

// tcgen05 sweeps (sweep_tc.cu): operands pre-scaled by sqrt(2 log2(e) / eps), split into
// bf16 hi/lo with K padded to a multiple of 64; map* point at CUtensorMap objects.
cudaError_t launch_split_bf16(const float* X, int64_t n, int32_t d, int32_t dp, float scale, void* hi, void* lo,
                              cudaStream_t s, const float* mu = nullptr, float* norm = nullptr);
// mapBbias: (nB padded to 128) x 16 bf16 rows [beta_hi, beta_mid, beta_lo, 0...] of the
// B side; bias_out (optional): the same rows for the A side, written from the updated
// potential in potential mode (the next sweep's B bias).
cudaError_t launch_lse_sweep_tc(const SweepParams& p, const void* mapAh, const void* mapAl, const void* mapBh,
                                const void* mapBl, const void* mapBbias, int nkb, int split3, int bn, int G,
                                int maxseg, int32_t* fault, void* bias_out, cudaStream_t stream);
cudaError_t launch_bias_prep(const float* potB, const float* Bn, int64_t nB, int64_t nB_pad, float bscale, void* out,
                             cudaStream_t s);
void tc_plan(int64_t nA, int64_t nB, int bn, int sms, int* G, int* maxseg);
// Barycentric displacement on the tensor cores for d <= 64 (map_tc.cu): x <- x + alpha
// (T(x) - x) in place (out may alias X), L from a log-sum-exp pass of the same t; the
// A / B / bias maps use 128-row boxes; the B operand sqrt(c) (y - mu) also serves the
// P Y product, whose result is mapped back with inv_sc = 1 / sqrt(c) and mu (d floats).
cudaError_t launch_map_sweep_tc(const float* X, float* out, const float* L, int64_t nA, int64_t nB, int32_t d,
                                float alpha, const void* mapAh, const void* mapAl, const void* mapBh,
                                const void* mapBl, const void* mapBbias, float inv_sc, const float* mu,
                                float* Opart, float* Rpart, unsigned* cnt, int G, int maxseg, int32_t split3,
                                int32_t* fault, cudaStream_t stream);
size_t map_sweep_tc_smem();
// The same for 64 < d <= 256 in one pass (map_tc_onepass.cu): tiles of 32 columns (B maps
// and bias rows in 32-row boxes) whose K blocks all stay in one stage, S formed once per
// tile and every chunk of 64 output coordinates accumulated in TMEM; Opart slots hold
// 128 rows x 64 nkb floats. xh is the bf16 hi operand of X (nA x 64 nkb, the buffer the
// A maps describe), read directly into TMEM.
bool map_tc_onepass_supported(int nkb);
int map_tc_onepass_tile_cols();
cudaError_t launch_map_sweep_tc_onepass(const float* X, float* out, const float* L, int64_t nA, int64_t nB,
                                        int32_t d, int32_t nkb, float alpha, const void* mapAl,
                                        const void* mapBh, const void* mapBl, const void* mapBbias, float inv_sc,
                                        const float* mu, const void* xh, float* Opart, float* Rpart, unsigned* cnt,
                                        int G, int maxseg, int32_t split3, int32_t* fault, cudaStream_t stream);
int tc_stages(int nkb, int split3);
int tc_tile_cols(int nkb, int split3);  // 128 or 256

// Persistent tensor-core Sinkhorn loop (loop_tc.cu). Side 0 is the f-update (rows of X
// against Y), side 1 the g-update. A finisher publishes its row block's bias rows, then
// the row block's ready flag (the index of the sweep that wrote it, plus one).
struct LoopSideLaunch {
  SweepParams p;             // potential mode; An / Bn the centred norms; role 1 (f) or 2 (g)
  float* out0;               // f-update: f buffers 0 and 1 (the state's fcur selects); g-update: g
  float* out1;
  void* bias_out[2];         // bias rows (rows x 16 bf16) of this side's rows, by iteration parity
  uint32_t* flag_out;        // [row blocks] ready flags of this side, zero at the loop's start
  const uint32_t* flag_in;   // the other side's flags
  unsigned long long* cnt;   // [row blocks] arrival counters, zero at the loop's start
  unsigned long long* done;  // finished row blocks, zero at the loop's start
  float2* partial;           // (max, sum) slots of this side's sweeps
  // device buffers for the work split's tables (filled by the launch): segs (int4) and
  // cslot hold table_slots entries each, cptr row blocks + 1, nseg one entry per CTA
  void* segs;
  int32_t* nseg;
  int32_t* cptr;
  int32_t* cslot;
  int64_t table_slots;
};
struct LoopLaunch {
  LoopSideLaunch side[2];
  // CUtensorMap: X hi, X lo, Y hi, Y lo (128-row boxes); X hi, X lo, Y hi, Y lo (bn-row
  // boxes); bias rows X[0], X[1], Y[0], Y[1] (bn-row boxes)
  const void* maps[12];
  double* errpart;           // [2][row blocks of X]
  SolverState* state;
  int32_t* fault;
  unsigned long long wait_ns;
  int nkb, split3, bn, G, maxseg, seq0, niter;
};
cudaError_t launch_sinkhorn_loop_tc(const LoopLaunch& L, cudaStream_t stream);

// Library settings and helpers shared with the batched engine (progot_api.cu).
// encode_operand_map: 2-D bf16 tensor map (CUtensorMap*) over a rows x dp row-major
// buffer, 64-wide 128-byte-swizzled boxes (dp a multiple of 64) or 16-wide 32-byte
// swizzled bias boxes (dp = 16), box_rows rows per box.
int encode_operand_map(void* map, void* base, int64_t rows, int32_t dp, int box_rows);
int32_t stall_window_setting();
unsigned long long wait_limit_setting();
int device_sm_count();
int fail_message(int code, const char* msg);  // sets the last-error text, returns code
cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t v, cudaStream_t s);
bool loop_tc_supported(int bn, int nkb, int split3);

void loop_tc_plan(int64_t n, int64_t m, int bn, int sms, int* G, int* maxseg);
size_t loop_tc_smem(int bn, int nkb, int split3);

}  // namespace progot
