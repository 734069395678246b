// coupling_marginals_noalloc: the coupling-marginal computation of coupling_marginals
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand over a workspace: code that runs inside a
// host framework or inference-engine callback whose device memory is planned up front
// and where allocation calls are not allowed, code that must not trigger the implicit
// device-wide synchronisation of cudaFree, or code whose device memory is owned by
// another allocator under a fixed budget. This entry point needs nothing but its
// inputs and outputs: its scratch (squared norms, split partials, error partials and
// arrival counters) lives in the file-scope device array below, which every GPU that
// loads the library holds until the process exits.
//
// The array is sized for at most kNoAllocMaxPoints points on either side; larger
// problems are rejected with PROGOT_ERR_INVALID_ARG. Every call shares the one array
// and it keeps the previous call's contents, so the arrival counters are cleared at
// the start of each call; two calls whose work overlaps on the GPU (different streams,
// or different host threads on one device) race on the array and must be serialised by
// the caller.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/progot.h"
#include "progot_internal.h"

namespace progot {

constexpr int64_t kNoAllocMaxPoints = 65536;
constexpr int64_t kNoAllocMaxRowBlocks = kNoAllocMaxPoints / 128;
constexpr int64_t kNoAllocPartials = kNoAllocMaxPoints + 128;  // float2 (max, sum) per (split, row)

constexpr size_t round256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffXn = 0;
constexpr size_t kOffYn = kOffXn + round256(sizeof(float) * kNoAllocMaxPoints);
constexpr size_t kOffPartial = kOffYn + round256(sizeof(float) * kNoAllocMaxPoints);
constexpr size_t kOffErrRow = kOffPartial + round256(sizeof(float2) * kNoAllocPartials);
constexpr size_t kOffErrCol = kOffErrRow + round256(sizeof(double) * (kNoAllocMaxRowBlocks + 2));
constexpr size_t kOffCntRow = kOffErrCol + round256(sizeof(double) * (kNoAllocMaxRowBlocks + 2));
constexpr size_t kOffCntCol = kOffCntRow + round256(sizeof(unsigned) * (kNoAllocMaxRowBlocks + 2));
constexpr size_t kNoAllocBytes = kOffCntCol + round256(sizeof(unsigned) * (kNoAllocMaxRowBlocks + 2));

// About 1.1 MB of scratch, resident on every device that loads this library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up once per device
// (host code must not use the symbol itself: on the host it is only a stand-in). The
// lookup is keyed on the device's current CUDA context too: after cudaDeviceReset the
// module is loaded again at another address, and the next call looks it up again.
constexpr int kMaxDevices = 64;
static unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
static void* g_scratch_ctx[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

typedef int (*CtxGetCurrentFn)(void**);
static void* current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    looked = true;
  }
  void* ctx = nullptr;
  if (fn == nullptr || fn(&ctx) != 0) return nullptr;
  return ctx;
}

static int scratch_for_current_device(unsigned char** out, const char** why) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *why = "cudaGetDevice failed";
    return PROGOT_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *why = "device ordinal out of range";
    return PROGOT_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  void* ctx = current_context();
  if (g_scratch_addr[dev] == nullptr || ctx == nullptr || ctx != g_scratch_ctx[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      *why = cudaGetErrorString(e);
      return PROGOT_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
    g_scratch_ctx[dev] = current_context();  // the lookup made the device's context current
  }
  *out = g_scratch_addr[dev];
  return PROGOT_OK;
}

static int noalloc_fail(int code, const char* msg) {
  set_last_error_message(msg);
  return code;
}

static int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
  return sms;
}

// The scratch layout assumes the float32 sweep's 128 x 128 tiles (one error partial per
// 128-row block, at most kNoAllocPartials split partials); a kernel built with other tile
// sizes must not run on it.
static bool tiles_match_layout() { return fp32_tile_rows() == 128 && fp32_tile_cols() == 128; }

// One marginal sweep "rows of A against rows of B" on the static scratch.
static SweepParams noalloc_sweep(const float* A, int64_t nA, const float* B, int64_t nB, int32_t d, const float* An,
                                 const float* Bn, double eps, float2* partial, double* errpart, unsigned* cnt) {
  SweepParams p;
  memset(&p, 0, sizeof(p));
  p.A = A;
  p.B = B;
  p.An = An;
  p.Bn = Bn;
  p.nA = nA;
  p.nB = nB;
  p.d = d;
  const int64_t BMr = fp32_tile_rows(), BNc = fp32_tile_cols();
  const int64_t rb = (nA + BMr - 1) / BMr;
  const int64_t ct = (nB + BNc - 1) / BNc;
  int64_t s = (int64_t)sm_count() * 2 / rb;
  if (s < 1) s = 1;
  if (s > ct) s = ct;
  while (s > 1 && s * nA > kNoAllocPartials) --s;  // stay inside the static partial buffer
  const int64_t tps = (ct + s - 1) / s;
  p.tiles_per_split = (int)tps;
  p.splits = (int)((ct + tps - 1) / tps);
  p.scale = (float)(2.0 * kLog2e / eps);
  p.bscale = (float)(kLog2e / eps);
  p.eps = eps;
  p.inv_eps_f = (float)(1.0 / eps);
  p.inv_nA = 1.0 / (double)nA;
  p.log_w_uniform = std::log(1.0 / (double)nA);
  p.partial = partial;
  p.errpart = errpart;
  p.cnt = cnt;
  p.mode = kModeMarginal;
  return p;
}

}  // namespace progot

using namespace progot;

extern "C" int coupling_marginals_noalloc(const float* x, int64_t n, const float* y, int64_t m, int32_t d,
                                          const float* f, const float* g, double eps, int32_t precision, float* row,
                                          float* col, const float* a, const float* b, double* err_l1_out,
                                          progot_stream_t stream) {
  set_last_error_message("");
  if (x == nullptr || y == nullptr || f == nullptr || g == nullptr)
    return noalloc_fail(PROGOT_ERR_INVALID_ARG, "x, y, f and g must not be NULL");
  if (n <= 0 || m <= 0 || d <= 0) return noalloc_fail(PROGOT_ERR_INVALID_ARG, "n, m, d must be positive");
  if (n > kNoAllocMaxPoints || m > kNoAllocMaxPoints)
    return noalloc_fail(PROGOT_ERR_INVALID_ARG,
                        "coupling_marginals_noalloc supports at most 65536 points per side (static scratch); "
                        "use coupling_marginals with a workspace for larger problems");
  if (precision != PROGOT_FP32) return noalloc_fail(PROGOT_ERR_INVALID_ARG, "only PROGOT_FP32 is supported");
  if (!(eps > 0.0) || !std::isfinite(eps)) return noalloc_fail(PROGOT_ERR_INVALID_ARG, "eps must be positive and finite");
  if (!tiles_match_layout())
    return noalloc_fail(PROGOT_ERR_INVALID_ARG, "the float32 sweep's tile sizes do not match the static scratch layout");
  unsigned char* base = nullptr;
  const char* why = "";
  int rc = scratch_for_current_device(&base, &why);
  if (rc) return noalloc_fail(rc, why);
  cudaStream_t s = (cudaStream_t)stream;
  float* xn = reinterpret_cast<float*>(base + kOffXn);
  float* yn = reinterpret_cast<float*>(base + kOffYn);
  float2* partial = reinterpret_cast<float2*>(base + kOffPartial);
  double* err_row = reinterpret_cast<double*>(base + kOffErrRow);
  double* err_col = reinterpret_cast<double*>(base + kOffErrCol);
  unsigned* cnt_row = reinterpret_cast<unsigned*>(base + kOffCntRow);
  unsigned* cnt_col = reinterpret_cast<unsigned*>(base + kOffCntCol);
  // the counters must start at zero; the rest of the scratch is written before it is read
  if (cudaMemsetAsync(cnt_row, 0, sizeof(unsigned) * (kNoAllocMaxRowBlocks + 2), s) != cudaSuccess ||
      cudaMemsetAsync(cnt_col, 0, sizeof(unsigned) * (kNoAllocMaxRowBlocks + 2), s) != cudaSuccess)
    return noalloc_fail(PROGOT_ERR_CUDA, "clearing the scratch counters failed");
  if (launch_row_sqnorm(x, n, d, xn, s) != cudaSuccess || launch_row_sqnorm(y, m, d, yn, s) != cudaSuccess)
    return noalloc_fail(PROGOT_ERR_CUDA, "squared-norm kernel launch failed");
  SweepParams pr = noalloc_sweep(x, n, y, m, d, xn, yn, eps, partial, err_row, cnt_row);
  pr.wA = a;
  pr.potB = g;
  pr.potA_old = f;
  pr.out = row;
  if (launch_lse_sweep_fp32(pr, s) != cudaSuccess) return noalloc_fail(PROGOT_ERR_CUDA, "row sweep launch failed");
  SweepParams pc = noalloc_sweep(y, m, x, n, d, yn, xn, eps, partial, err_col, cnt_col);
  pc.wA = b;
  pc.potB = f;
  pc.potA_old = g;
  pc.out = col;
  if (launch_lse_sweep_fp32(pc, s) != cudaSuccess) return noalloc_fail(PROGOT_ERR_CUDA, "column sweep launch failed");
  if (err_l1_out != nullptr) {
    double er = 0.0, ec = 0.0;
    const int64_t rbr = (n + fp32_tile_rows() - 1) / fp32_tile_rows(), rbc = (m + fp32_tile_rows() - 1) / fp32_tile_rows();
    if (cudaMemcpyAsync(&er, err_row + rbr, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&ec, err_col + rbc, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return noalloc_fail(PROGOT_ERR_CUDA, "reading the marginal error failed");
    *err_l1_out = er + ec;
  }
  return PROGOT_OK;
}
