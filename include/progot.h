/*
 * progot.h - C ABI of the GB300 (sm_103a) ProgOT hot path.
 *
 * ProgOT (arXiv 2406.05061) estimates an optimal-transport coupling and map between a
 * source cloud X (n x d) and a target cloud Y (m x d) by K warm-started entropic
 * (Sinkhorn) solves, each followed by a partial move of X along the entropic map
 * (Alg. 2). The cost is the squared Euclidean distance c(x, y) = ||x - y||^2
 * (h = ||.||^2 in Sec. 2) and is never stored: every row or column log-sum-exp over it
 * is computed tile by tile from x . y, |x|^2 and |y|^2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Point clouds are row-major float32 arrays with leading dimension d (point i at
 *   x[i*d .. i*d+d-1]). Weights a (n) and b (m) are float32 probability vectors, or
 *   NULL for the uniform weights 1/n and 1/m.
 * - Arrays named as "device" are device pointers (cudaMalloc / torch CUDA tensors on the
 *   current device); they are caller-allocated and caller-owned and the library never
 *   frees them. Arrays named as "host" are host memory.
 * - Potentials follow the dual convention of eq. (5): the coupling is
 *   P_ij = exp((f_i + g_j - c(x_i, y_j)) / eps); g absorbs eps log b_j.
 * - workspace / ws_bytes: device scratch owned by the caller, at least
 *   progot_workspace_size(...) bytes, 256-byte aligned. Its contents need not be
 *   initialised and are garbage after the call. Two calls in flight at the same time
 *   must not share a workspace.
 * - stream: a cudaStream_t (NULL = legacy default stream). Entry points that return
 *   host results (iteration counts, errors) synchronise that stream before
 *   returning; the others are asynchronous.
 * - precision: PROGOT_FP32 evaluates the cross term x . y with float32 FMAs on CUDA
 *   cores; PROGOT_BF16X3 uses tcgen05 tensor cores on a bf16 hi/lo split of both
 *   operands (x.y ~ xh.yh + xh.yl + xl.yh, float32 accumulation); PROGOT_BF16 uses the
 *   hi parts only. Log-sum-exps and potentials are float32 in every mode; squared norms
 *   and the marginal-error reduction accumulate in float64.
 * - Return value: PROGOT_OK or an error code below. progot_last_error_string()
 *   describes the last error on the calling thread. On PROGOT_ERR_NOT_CONVERGED all
 *   outputs are still written (the last iterate).
 */
#ifndef PROGOT_H
#define PROGOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* progot_stream_t; /* a cudaStream_t */

enum progot_status {
  PROGOT_OK = 0,
  PROGOT_ERR_INVALID_ARG = 1,   /* n, m, d <= 0, eps <= 0, alpha outside (0, 1], NULL required pointer, misaligned */
  PROGOT_ERR_NOT_CONVERGED = 2, /* marginal error still above tau after max_iter iterations (or stalled) */
  PROGOT_ERR_NUMERIC = 3,       /* NaN or Inf in the marginal-error reduction */
  PROGOT_ERR_OOM = 4,           /* a host-side allocation failed */
  PROGOT_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  PROGOT_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired */
  PROGOT_ERR_WORKSPACE = 7      /* workspace NULL, too small or not 256-byte aligned */
};

typedef enum { PROGOT_FP32 = 0, PROGOT_BF16X3 = 1, PROGOT_BF16 = 2 } progot_precision;

typedef enum { PROGOT_ALPHA_CONSTANT = 0, PROGOT_ALPHA_ACCELERATED = 1, PROGOT_ALPHA_DECELERATED = 2 } progot_alpha_kind;

/* Text of the last error on the calling thread ("" when none). Never NULL. */
const char* progot_last_error_string(void);

/* Library version, e.g. "0.1.0". */
const char* progot_version(void);

/* Bytes of device workspace that every entry point below needs for a problem with at
 * most n rows, m columns and dimension d (for entropic_map_apply pass nq as n). */
size_t progot_workspace_size(int64_t n, int64_t m, int32_t d, int32_t precision);

/*
 * sinkhorn_potentials - Sink(a, X, b, Y, eps, tau, f_init, g_init) of Alg. 1.
 *
 * While the row-marginal error ||P 1 - a||_1 exceeds tau, alternate
 *   f_i <- eps log a_i - eps log sum_j exp((g_j - c(x_i, y_j)) / eps)
 *   g_j <- eps log b_j - eps log sum_i exp((f_i - c(x_i, y_j)) / eps)
 * (the soft-min updates of Alg. 1 with the sign of the paper's min_eps term read as +).
 * The error is checked before each iteration, so the returned (f, g) is the last pair
 * whose error was measured; after the g-update the column marginal is exact.
 *
 * x (device, n x d), a (device, n, or NULL), y (device, m x d), b (device, m, or NULL).
 * eps > 0, tau >= 0, max_iter >= 0.
 * f (device, n) and g (device, m): in = initial potentials unless init_zero != 0 (then
 *   zero); out = the final potentials.
 * iters_out (host, may be NULL): completed (f, g) iterations. err_out (host, may be
 *   NULL): the last measured row-marginal L1 error (float64).
 * Returns PROGOT_ERR_NOT_CONVERGED when tau was not met within max_iter iterations or
 * the error stopped decreasing (see progot_set_stall_window).
 */
int sinkhorn_potentials(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                        int32_t d, double eps, double tau, int32_t max_iter, int32_t precision, float* f, float* g,
                        int32_t init_zero, int32_t* iters_out, double* err_out, void* workspace, size_t ws_bytes,
                        progot_stream_t stream);

/*
 * entropic_map_apply - T_Prog[b, Y, (g^(k), eps_k, alpha_k)_k] of Alg. 3 on nq points.
 *
 * For k = 1..K: p_j = softmax_j((g^(k)_j - c(z, y_j)) / eps_k),
 *   z <- (1 - alpha_k) z + alpha_k sum_j p_j y_j,
 * which is Alg. 3's z <- z - alpha_k grad h*(p^T [grad h(z - y_j)]_j) for h = ||.||^2.
 * With K = 1 and alpha = 1 this is the entropic map of eq. (7).
 * alpha_K is taken as 1 whatever alpha[K-1] holds (Alg. 3 resets it).
 *
 * xq (device, nq x d) query points; y (device, m x d); g_all (device, K x m) the stored
 * g^(k); eps (host, K) and alpha (host, K) float64; out (device, nq x d) may alias xq.
 */
int entropic_map_apply(const float* xq, int64_t nq, const float* y, int64_t m, int32_t d, int32_t K,
                       const float* g_all, const double* eps, const double* alpha, int32_t precision, float* out,
                       void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * coupling_marginals - r = P 1_m and c = P^T 1_n of P_ij = exp((f_i + g_j - c(x_i, y_j))/eps)
 * (the coupling returned by Alg. 1 / Alg. 2), and the marginal constraint violation
 * ||r - a||_1 + ||c - b||_1 reported with the coupling metrics of Sec. 5.2.
 *
 * row (device, n) and col (device, m) may be NULL (not written). a, b (device) may be
 * NULL for uniform weights. err_l1_out (host, may be NULL) is accumulated in float64.
 */
int coupling_marginals(const float* x, int64_t n, const float* y, int64_t m, int32_t d, const float* f,
                       const float* g, double eps, int32_t precision, float* row, float* col, const float* a,
                       const float* b, double* err_l1_out, void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * coupling_marginals_noalloc - coupling_marginals without a workspace and without any
 * allocation (the paper has no counterpart: this is an interface for callers that
 * cannot allocate device memory).
 *
 * Who needs it: callers that cannot call cudaMalloc or provide a scratch buffer, such
 * as code running inside a framework or inference-engine callback whose device memory
 * is planned ahead and where allocation calls are not allowed, code that must not incur
 * the implicit device-wide synchronisation of cudaFree, or code whose device memory
 * belongs to another allocator with a fixed budget. The caller still passes every input
 * and output exactly as for coupling_marginals (same meaning, layout and ownership);
 * the library's scratch is a fixed ~1.1 MB device array inside libprogot.so that every
 * GPU loading the library holds until the process exits. The call makes no cudaMalloc,
 * cudaFree or other allocating call.
 *
 * Limits and behaviour:
 * - n and m must each be at most 65536; larger sizes return PROGOT_ERR_INVALID_ARG with
 *   an explanatory progot_last_error_string(). Only PROGOT_FP32 is accepted.
 * - The first call on a device looks up the device address of the array (a one-time
 *   set-up per device, repeated only when the device's context was reset, e.g. by
 *   cudaDeviceReset); make that first call before any stream capture.
 * - All calls share the one array, which keeps the last call's contents (the arrival
 *   counters are cleared at the start of every call). Calls whose GPU work overlaps
 *   (other streams, other host threads on the same device) race on it: serialise them.
 * - err_l1_out (host, may be NULL): ||r - a||_1 + ||c - b||_1; when given, the stream is
 *   synchronised; otherwise the call is asynchronous.
 */
int coupling_marginals_noalloc(const float* x, int64_t n, const float* y, int64_t m, int32_t d, const float* f,
                               const float* g, double eps, int32_t precision, float* row, float* col, const float* a,
                               const float* b, double* err_l1_out, progot_stream_t stream);

/*
 * progot_solve - ProgOT(a, X, b, Y, (eps_k, alpha_k, tau_k)_k) of Alg. 2, K solves.
 *
 * f = 0, g^(0) = 0. For k = 1..K: warm start f, g <- (1 - alpha_k) f, (1 - alpha_k) g^(k-1);
 * (f, g^(k)) <- Sinkhorn at (eps_k, tau_k); Q = diag(1 / P 1) P;
 * x_i <- (1 - alpha_k) x_i + alpha_k sum_j Q_ij y_j (the barycentric displacement
 * X <- X - alpha_k Z with Z_i = grad h*(sum_j Q_ij grad h(x_i - y_j))).
 *
 * x (device, n x d) is not modified. alpha, eps, tau (host, K, float64); alpha_K should be
 * 1 so that x_out = T_Prog(x_i) (Def. 1). max_iter bounds each solve.
 * x_out (device, n x d): the displaced cloud after step K.
 * g_all (device, K x m): g^(k) of every step (the map-estimator state of Alg. 3).
 * f_last (device, n, may be NULL): f of the last solve; with x_last (device, n x d, may
 *   be NULL: the cloud X^(K) the last solve ran on) and g_all[K-1] it defines the
 *   returned coupling P.
 * iters (host, K, may be NULL), errs (host, K, may be NULL): per-step iteration counts and
 *   final row-marginal errors.
 * Returns PROGOT_ERR_NOT_CONVERGED if any step did not reach its tau (all outputs are
 * still written).
 */
int progot_solve(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                 int32_t K, const double* alpha, const double* eps, const double* tau, int32_t max_iter,
                 int32_t precision, float* x_out, float* g_all, float* f_last, float* x_last, int32_t* iters,
                 double* errs, void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * progot_problem - one ProgOT problem for progot_solve_batched (device pointers) or
 * for the server (host pointers). Meanings, layouts and lengths as in progot_solve;
 * alpha, eps, tau (host, K); iters, errs (host, K, may be NULL); f_last may be NULL;
 * status receives the problem's own return code.
 */
typedef struct progot_problem {
  const float* x;
  const float* a;
  int64_t n;
  const float* y;
  const float* b;
  int64_t m;
  int32_t d;
  int32_t K;
  const double* alpha;
  const double* eps;
  const double* tau;
  float* x_out;
  float* g_all;
  float* f_last;
  int32_t* iters;
  double* errs;
  int32_t status;
} progot_problem;

/*
 * progot_solve_batched - Alg. 2 on `count` independent problems of uneven sizes (the
 * batched workload of many small ProgOT problems); the call returns when every problem
 * is done. With the persistent engine (progot_set_batch_engine, the default where every
 * problem fits it) the batch runs as one persistent launch on `stream` (see
 * progot_batch_plan below; n_streams is then unused). Otherwise the problems run
 * through progot_solve on n_streams internal CUDA streams, each driven by a host worker
 * thread, largest problems first; the internal streams wait for `stream` at entry and
 * `stream` waits for them at exit, and results are bit-identical to solving each
 * problem alone (launch shapes depend only on a problem's sizes). workspace: at least
 * progot_batched_workspace_size(...) bytes (which covers the engine in use).
 * Returns the first hard error of any problem, else PROGOT_ERR_NOT_CONVERGED if any
 * problem did not reach its tau, else PROGOT_OK; per-problem codes in problems[i].status.
 */
size_t progot_batched_workspace_size(const progot_problem* problems, int32_t count, int32_t precision,
                                     int32_t n_streams);
int progot_solve_batched(progot_problem* problems, int32_t count, int32_t max_iter, int32_t precision,
                         int32_t n_streams, void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * progot_set_batch_engine - how progot_solve_batched runs a batch: 1 (default) = one
 * persistent launch over all problems (the progot_batch_plan engine below) when every
 * problem has d <= 64 and the precision is bf16x3 or bf16, else, and with 0, the
 * per-problem solves on host-driven streams described above (bit-identical to solving
 * each problem alone). The persistent engine's results match the single-problem path
 * within the mixed-precision tolerances but not bit for bit (its centre of the operands
 * is fixed per problem, its column tiles and segments differ); they depend only on the
 * problem itself, not on the rest of the batch. This library setting has no counterpart
 * in the paper.
 */
int progot_set_batch_engine(int32_t engine);

/*
 * Persistent batched engine: Alg. 2 (and each step's Alg. 1 loop) for many independent
 * problems in one persistent launch, tasks of (problem, phase, row block, column
 * segment) drawn from a device-side work queue by one CTA per SM; a problem's phases
 * (centre, operand split with warm start, f-updates, g-updates, map step) follow one
 * another through the queue, different problems interleave.
 *
 * progot_batch_plan_workspace_size - device bytes a plan over these problems needs
 *   (operands, bias rows, potentials, partials, queue; 256-byte aligned internally).
 * progot_batch_plan_create - validates the problems (device pointers x, y, a, b, x_out,
 *   g_all, f_last as in progot_solve; host alpha, eps, tau of length K; 1 <= d <= 64;
 *   n, m <= 2^24; precision PROGOT_BF16X3 or PROGOT_BF16), carves the caller's workspace
 *   (caller-owned, must stay valid until destroy), encodes the tensor maps and copies
 *   the descriptors and step constants to the device (synchronous host-to-device
 *   copies). The problems' device buffers must stay valid for the plan's life; the host
 *   arrays are read only here. *plan receives the handle.
 * progot_batch_plan_run - enqueues one solve of the whole batch on `stream`: a counter
 *   reset, a queue initialisation and the persistent kernel; with use_graph != 0 these
 *   are captured once into a CUDA graph that every later call replays. Outputs (x_out,
 *   g_all, f_last) are written by the time the stream reaches the end of the run.
 * progot_batch_plan_collect - synchronises `stream` and copies the per-step iteration
 *   counts and errors into problems[i].iters / errs (host, may be NULL) and each
 *   problem's code into problems[i].status; returns PROGOT_ERR_TIMEOUT if a bounded
 *   device wait expired, else the first PROGOT_ERR_NUMERIC, else
 *   PROGOT_ERR_NOT_CONVERGED if any step missed its tau, else PROGOT_OK.
 * progot_batch_plan_set_target - column segmentation of the sweep tasks: each problem's
 *   f- and g-updates are cut into at least `target` tasks (segments of a row block's
 *   column tiles, at most 8 and at most the number of tiles). Not while a run is in
 *   flight.
 * progot_batch_plan_autotune - times complete runs of the batch for the targets 1, 4,
 *   16, 64 and 256 (one warm-up and two timed runs each, on `stream`) and keeps the
 *   fastest; *target_out and *ms_out (may be NULL) receive it and its time.
 * progot_batch_plan_destroy - frees the host-side plan and its graph (not the workspace).
 * This engine is a serving-side device; the paper has no counterpart.
 */
typedef struct progot_batch_plan progot_batch_plan;
size_t progot_batch_plan_workspace_size(const progot_problem* problems, int32_t count, int32_t precision);
int progot_batch_plan_create(const progot_problem* problems, int32_t count, int32_t max_iter, int32_t precision,
                             void* workspace, size_t ws_bytes, progot_batch_plan** plan);
int progot_batch_plan_run(progot_batch_plan* plan, int32_t use_graph, progot_stream_t stream);
int progot_batch_plan_collect(progot_batch_plan* plan, progot_problem* problems, progot_stream_t stream);
int progot_batch_plan_set_target(progot_batch_plan* plan, int32_t target);
int progot_batch_plan_autotune(progot_batch_plan* plan, int32_t* target_out, double* ms_out, progot_stream_t stream);
void progot_batch_plan_destroy(progot_batch_plan* plan);

/*
 * Continuous-batching server. progot_server_create allocates one device arena of
 * budget_bytes (the device-memory budget) and starts n_workers host threads, each with
 * its own CUDA stream. progot_server_submit queues a request (host pointers, which must
 * stay valid until progot_server_wait returns for it) and returns its id (>= 0) or a
 * negated error code (-PROGOT_ERR_OOM when the request alone exceeds the budget).
 * Requests are admitted in arrival order as soon as a worker is free and the request's
 * memory (inputs, outputs, solve workspace) fits in the arena (first-fit sub-allocator);
 * the worker copies the inputs in, runs progot_solve with the server's precision and
 * max_iter, copies x_out, g_all (and f_last, iters, errs) back and releases the memory,
 * so requests that arrive while others run are admitted as memory frees up and their
 * work overlaps on the device. progot_server_wait blocks until a request finished and
 * returns its status and its latency from submission (ms). progot_server_stats reports
 * completed and in-flight requests and the arena's current and peak use.
 * progot_server_destroy finishes the queued requests and frees the arena.
 */
typedef struct progot_server progot_server;
progot_server* progot_server_create(size_t budget_bytes, int32_t n_workers, int32_t precision, int32_t max_iter);
int64_t progot_server_submit(progot_server* server, const progot_problem* request);
int progot_server_wait(progot_server* server, int64_t id, double* latency_ms);
int progot_server_stats(progot_server* server, int64_t* completed, int64_t* in_flight, size_t* bytes_in_use,
                        size_t* peak_bytes);
void progot_server_destroy(progot_server* server);

/*
 * progot_schedule_alpha - alpha_1..alpha_K of the step-length schedules of Sec. 4
 * (Table 7), with alpha_K = 1. Each alpha_k is the fraction of the remaining path that
 * step k covers: alpha_k = (t_k - t_{k-1}) / (1 - t_{k-1}) for the target progress
 * t_k = k/K (constant speed) or (k/K)^2 (accelerated); decelerated uses alpha_k = 1/e.
 * out (host, K).
 */
int progot_schedule_alpha(int32_t K, int32_t kind, double* out);

/*
 * progot_mean_cost - (1/(n m)) sum_ij ||x_i - y_j||^2, the mean of the cost matrix used
 * for eps0 and sigma in Alg. 4, in closed form
 * mean ||x||^2 + mean ||y||^2 - 2 xbar . ybar (float64 sums on the device).
 * out (host). Synchronises the stream.
 */
int progot_mean_cost(const float* x, int64_t n, const float* y, int64_t m, int32_t d, double* out, void* workspace,
                     size_t ws_bytes, progot_stream_t stream);

/*
 * progot_schedule_eps - the epsilon scheduler of Alg. 4.
 *
 * eps0 = mean cost(X, Y) / 20, sigma = mean cost(Y, Y) / 20. For each s_p of s_grid
 * (host, P): solve Sink(b, Y, b, Y, s_p sigma, tau) on the device, map y_test
 * (device, mt x d) with (g, s_p sigma, alpha = 1) and score sum ||y~ - T(y~)||^2 (float64).
 * eps_K = s_{p*} sigma for the first minimiser p*; eps_out (host, K) receives
 * (1 - t_k) beta0 eps0 + t_k eps_K with t_k = 1 - prod_{l<=k}(1 - alpha_l) from alpha
 * (host, K). errors_out (host, P, may be NULL) receives the scores; p_star_out (host,
 * may be NULL) the chosen index. workspace must cover (max(n, m, mt), max(m, n), d).
 */
int progot_schedule_eps(const float* x, int64_t n, const float* y, const float* b, int64_t m,
                        const float* y_test, int64_t mt, int32_t d, int32_t K, const double* alpha,
                        const double* s_grid, int32_t P, double beta0, double tau, int32_t max_iter, int32_t precision,
                        double* eps_out, double* errors_out, int32_t* p_star_out, void* workspace, size_t ws_bytes,
                        progot_stream_t stream);

/*
 * progot_schedule_tau - the Sinkhorn threshold schedule of Sec. 4 ("Setting threshold
 * schedule"): tau_k falls linearly in k from tau_first (k = 1) to tau_last (k = K), so
 * early solves stop loose and the last one meets tau_last. K = 1 gives tau_last.
 * tau_first, tau_last >= 0. out (host, K).
 */
int progot_schedule_tau(int32_t K, double tau_first, double tau_last, double* out);

/*
 * progot_solve_theta - Alg. 2 with the iterate-dependent regularisation of the coupling
 * experiments (Sec. 5.2 and the experiment details of the appendix): solve k uses
 * eps_k = theta cbar_k, where cbar_k = sum_ij ||x^(k)_i - y_j||^2 / (20 n m) is the mean
 * cost of the cloud X^(k) that solve k transports (X^(1) = X), divided by 20. cbar_k is
 * computed on the device in closed form from float64 first moments before each solve.
 * theta > 0 (the paper's default 2^-4). eps_out (host, K, required) receives eps_k (the
 * map estimator of Alg. 3 needs them). Every other argument, output and return code is
 * that of progot_solve. Synchronises the stream once per step (eps_k is a host scalar
 * of the sweeps).
 */
int progot_solve_theta(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                       int32_t d, int32_t K, const double* alpha, double theta, const double* tau, int32_t max_iter,
                       int32_t precision, float* x_out, float* g_all, float* f_last, float* x_last, int32_t* iters,
                       double* errs, double* eps_out, void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * Coupling metrics of Sec. 5.2 for P_ij = exp((f_i + g_j - ||x_i - y_j||^2) / eps):
 *   transport_cost = <P, C> = sum_ij P_ij ||x_i - y_j||^2
 *   entropy        = E(P) = -sum_ij P_ij (log P_ij - 1)
 *   dual           = <f, a> + <g, b> - eps sum_ij P_ij   (the objective of eq. (5))
 *   mass           = sum_ij P_ij
 *   err_row        = ||P 1 - a||_1,  err_col = ||P^T 1 - b||_1
 */
typedef struct progot_coupling_metrics {
  double transport_cost;
  double entropy;
  double dual;
  double mass;
  double err_row;
  double err_col;
} progot_coupling_metrics;

/*
 * coupling_metrics - the metrics above from two float32 CUDA-core sweeps (one over rows,
 * one over columns) that never store P. The row sweep carries, besides the row
 * log-sum-exp, the 2^t-weighted mean of t_ij (t_ij = log2 of the row's terms), which
 * gives sum_j P_ij log P_ij per row; then <P, C> = <f, P 1> + <g, P^T 1> - eps
 * sum P log P. All reductions are float64 in a fixed order (deterministic).
 * x (device, n x d), y (device, m x d), f (device, n), g (device, m), a, b (device or
 * NULL = uniform). x_cost (device, n x d, may be NULL): when given, transport_cost is
 * sum_ij P_ij ||xc_i - y_j||^2 with P still defined on x. ProgOT's final coupling lives on
 * the displaced cloud X^(K) (x_last of progot_solve) but couples the original points row
 * for row, so Sec. 5.2 measures its cost against the original X: pass x = x_last and
 * x_cost = the original X. The row sweep then also computes the cost tile of x_cost and
 * keeps sum_j 2^(t_ij - max) c(xc_i, y_j) per row. out (host). workspace:
 * progot_workspace_size(n, m, d, PROGOT_FP32). Synchronises the stream.
 */
int coupling_metrics(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                     const float* f, const float* g, const float* x_cost, double eps, progot_coupling_metrics* out,
                     void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * sinkhorn_divergence - the Sinkhorn divergence of eq. (8):
 *   D_eps(X, Y) = OT_eps(X, Y) - (OT_eps(X, X) + OT_eps(Y, Y)) / 2,
 * where OT_eps is the eq. (5) objective at the potentials of a Sinkhorn solve (Alg. 1,
 * zero start, threshold tau, at most max_iter iterations, given precision) and is
 * evaluated by coupling_metrics. The paper takes eps = 5% of the target's mean intra cost
 * (0.05 x progot_mean_cost(y, y)). value (host); ot_parts (host, 3, may be NULL):
 * OT(X, Y), OT(X, X), OT(Y, Y); iters (host, 3, may be NULL). workspace:
 * progot_workspace_size(max(n, m), max(n, m), d, precision). Returns
 * PROGOT_ERR_NOT_CONVERGED if a solve missed tau (value still written).
 */
int sinkhorn_divergence(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                        int32_t d, double eps, double tau, int32_t max_iter, int32_t precision, double* value,
                        double* ot_parts, int32_t* iters, void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * coupling_diagonal - the identity-coupling check of Sec. 5.3 / Prop. 3 for n = m
 * (point i of Y is the image of point i of X): log P_ii = (f_i + g_i - ||x_i - y_i||^2)
 * / eps, trace = sum_i P_ii and kl = KL(Id/n || P) = -log n - (1/n) sum_i log P_ii
 * (float64 sums, fixed order). log_diag (device, n, may be NULL) receives log P_ii.
 * trace, kl (host, may be NULL). workspace: progot_workspace_size(n, n, d, PROGOT_FP32).
 * Synchronises the stream.
 */
int coupling_diagonal(const float* x, const float* y, int64_t n, int32_t d, const float* f, const float* g, double eps,
                      float* log_diag, double* trace, double* kl, void* workspace, size_t ws_bytes,
                      progot_stream_t stream);

/*
 * The p-norm cost of the coupling experiments (Sec. 5.2): c(x, y) = h(x - y) with
 * h(z) = (1/p) sum_k |z_k|^p, 1 < p <= 8 (the paper uses p = 1.5, which has a
 * specialised kernel; other p go through 2^(p log2 |z|)). There is no product form, so
 * these entry points run on float32 CUDA cores: every pair term is summed coordinate by
 * coordinate, and the map step evaluates grad h(z)_k = sign(z_k) |z_k|^(p-1) for every
 * pair and coordinate and moves x by grad h*(w)_k = sign(w_k) |w_k|^(1/(p-1)):
 *   Z_i = grad h*(sum_j Q_ij grad h(x_i - y_j)), x_i <- x_i - alpha_k Z_i   (Alg. 2, Alg. 3).
 * The potentials follow the same eq. (5) convention, P_ij = exp((f_i + g_j - c_ij)/eps).
 * Arguments, layouts, outputs and errors are those of the squared Euclidean entry
 * points named in each comment, with p added and no precision argument; workspaces as
 * progot_workspace_size(..., PROGOT_FP32). p outside (1, 8] gives PROGOT_ERR_INVALID_ARG.
 */
/* As sinkhorn_potentials. */
int sinkhorn_potentials_pnorm(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                              int32_t d, double p, double eps, double tau, int32_t max_iter, float* f, float* g,
                              int32_t init_zero, int32_t* iters_out, double* err_out, void* workspace,
                              size_t ws_bytes, progot_stream_t stream);
/* As progot_solve with the eps schedule eps (host, K), or, when eps is NULL, as
 * progot_solve_theta with eps_k = theta * mean_ij h(x^(k)_i - y_j) / 20, the mean taken
 * over all n m pairs on the device; eps_out (host, K, may be NULL) receives eps_k. */
int progot_solve_pnorm(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m, int32_t d,
                       double p, int32_t K, const double* alpha, const double* eps, double theta, const double* tau,
                       int32_t max_iter, float* x_out, float* g_all, float* f_last, float* x_last, int32_t* iters,
                       double* errs, double* eps_out, void* workspace, size_t ws_bytes, progot_stream_t stream);
/* As entropic_map_apply (Alg. 3). */
int entropic_map_apply_pnorm(const float* xq, int64_t nq, const float* y, int64_t m, int32_t d, double p, int32_t K,
                             const float* g_all, const double* eps, const double* alpha, float* out, void* workspace,
                             size_t ws_bytes, progot_stream_t stream);
/* As coupling_metrics: <P, C> with C_ij = h(x_i - y_j) (or h(xc_i - y_j) with x_cost),
 * E(P), the eq. (5) objective. */
int coupling_metrics_pnorm(const float* x, const float* a, int64_t n, const float* y, const float* b, int64_t m,
                           int32_t d, double p, const float* f, const float* g, const float* x_cost, double eps,
                           progot_coupling_metrics* out, void* workspace, size_t ws_bytes, progot_stream_t stream);
/* (1/(n m)) sum_ij h(x_i - y_j), summed over all pairs (float64 per CTA, fixed order). out (host). */
int progot_mean_cost_pnorm(const float* x, int64_t n, const float* y, int64_t m, int32_t d, double p, double* out,
                           void* workspace, size_t ws_bytes, progot_stream_t stream);

/*
 * progot_set_stall_window - Sinkhorn stops with PROGOT_ERR_NOT_CONVERGED when its
 * marginal error has not fallen below 0.99 x its best value for `iters` consecutive
 * iterations (float32 potentials reach a rounding floor). 0 disables the check.
 * Default 512. Process-wide setting.
 */
int progot_set_stall_window(int32_t iters);

/*
 * progot_set_map_tc - choose the kernel of the map step (Alg. 2 / Alg. 3) on the
 * tensor-core paths (PROGOT_BF16X3, PROGOT_BF16) for d <= 256: 1 (default) runs S = X Y^T
 * and P Y on tcgen05 (P and the centred, scaled Y in bf16 hi/lo, three products with
 * PROGOT_BF16X3 and one with PROGOT_BF16, float32 accumulation in TMEM; for 64 < d <= 256
 * in one pass over Y with every output coordinate in TMEM); 0 runs P Y on float32 CUDA
 * cores after the tensor-core LSE pass (the path for d > 256 and PROGOT_FP32).
 * Process-wide setting.
 */
int progot_set_map_tc(int32_t on);

/*
 * progot_set_loop_tc - choose how the tensor-core paths run a Sinkhorn loop (Alg. 1):
 * 1 (default) as one persistent cooperative launch that runs every f- and g-update and
 * the stop test on the device (each update's bias rows pass between the GPU's CTAs
 * behind per-row-block ready flags, so a tile of the next update waits only for the
 * row blocks it reads); 0 as one launch per update (the host enqueues chunks of
 * iterations). Both compute the same iteration of Alg. 1 and stop at the same test.
 * Shapes the persistent kernel cannot hold in shared memory use the per-update kernel.
 * Process-wide setting.
 */
int progot_set_loop_tc(int32_t on);

/*
 * progot_set_wait_limit_ns - the bounded-wait limit of the persistent Sinkhorn loop's
 * waits (on its own pipeline, on another CTA's row blocks, on the stop test), in
 * nanoseconds of GPU global time; 0 restores the default of 2 s. A wait that runs past
 * it makes the launch abort: every CTA stops issuing work, retires the copies and
 * products it has in flight (those drains keep the 2 s limit), frees its tensor memory
 * and returns, and the entry point returns PROGOT_ERR_TIMEOUT; the CUDA context stays
 * usable. Process-wide setting.
 */
int progot_set_wait_limit_ns(uint64_t ns);

/*
 * progot_test_withhold_initial_betas - test hook for the timeout path: with on = 1 the
 * persistent Sinkhorn loops that start afterwards never publish the initial g's betas
 * (their row blocks' ready flags stay at "nothing published"), so the first f-update
 * waits for words that no sweep provides until the bounded wait
 * (progot_set_wait_limit_ns) expires and the entry point returns PROGOT_ERR_TIMEOUT.
 * Nothing faults or hangs; the context stays usable. 0 (default) restores normal
 * operation. Process-wide setting.
 */
int progot_test_withhold_initial_betas(int32_t on);

/* Number of kernels this library launched since the last call (process-wide counter);
 * used to report launches inside a timed region. */
int64_t progot_launch_count(int32_t reset);

/*
 * progot_profile - enable (enable >= 1) or disable (0) per-kernel timing on the calling
 * thread and reset its totals. While enabled, the log-sum-exp sweeps of a Sinkhorn loop
 * are timed by CUDA events around each chunk of sweeps the loop enqueues (an event
 * between two sweeps would break their programmatic overlap and inflate the figure);
 * a chunk counts when all its launches did work (launches after the loop's stop return
 * at entry). Other sweep and map launches are sampled one by one, every enable-th
 * launch (all of them for enable = 1).
 * progot_profile_read - totals since the last progot_profile call for kernel 0 (the
 * row/column log-sum-exp sweep) or 1 (the map sweep): timed launches, their summed
 * device time in ms and summed point pairs (rows x columns), and the number of
 * launches that did work (timed or not). Reading synchronises on the recorded events.
 * Any output pointer may be NULL.
 */
int progot_profile(int32_t enable);
int progot_profile_read(int32_t kernel, int64_t* sampled, double* total_ms, double* pairs, int64_t* worked);

#ifdef __cplusplus
}
#endif

#endif /* PROGOT_H */
