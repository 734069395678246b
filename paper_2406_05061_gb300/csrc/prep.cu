// Small O((n + m) d) kernels: squared norms (float64 accumulation), potential scaling
// for the warm start of Alg. 2, state initialisation, deterministic float64 reductions
// (first moments for the closed-form mean cost of Alg. 4 and of the theta rule, the
// centre of the tensor-core operands, squared error for the Alg. 4 score, the coupling
// diagonal of Prop. 3) and the move of a centred log-sum-exp back to uncentred form.
#include <algorithm>

#include "progot_internal.h"

namespace progot {

constexpr int kParts = 304;  // partial sums of the two-pass reductions

int reduce_parts() { return kParts; }

// One warp per row: |x_i|^2 summed in float64, stored as float32.
__global__ void row_sqnorm_kernel(const float* __restrict__ X, int64_t n, int32_t d, float* __restrict__ out) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* x = X + row * (int64_t)d;
  double s = 0.0;
  for (int k = lane; k < d; k += 32) {
    const double v = (double)x[k];
    s += v * v;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[row] = (float)s;
}

__global__ void scale_kernel(float* v, int64_t n, float factor) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] *= factor;
}

// Both solver states (the second is used by loops that run the stop test one sweep later).
__global__ void init_state_kernel(SolverState* st) {
  for (int q = 0; q < 2; ++q) {
    st[q].it = 0;
    st[q].done = 0;
    st[q].status = kRunning;
    st[q].fcur = 0;
    st[q].best_it = 0;
    st[q].err = 0.0;
    st[q].best_err = INFINITY;
  }
}

// Pass 1: block b sums rows b, b + parts, ... of (|x|^2, x_1 .. x_d) into partial[b].
__global__ void moments_pass1(const float* __restrict__ X, int64_t n, int32_t d, double* __restrict__ partial) {
  extern __shared__ double acc[];  // d + 1 per warp
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < warps * (d + 1); k += blockDim.x) acc[k] = 0.0;
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * warps + warp; row < n; row += (int64_t)gridDim.x * warps) {
    const float* x = X + row * (int64_t)d;
    double s = 0.0;
    for (int k = lane; k < d; k += 32) {
      const double v = (double)x[k];
      s += v * v;
      acc[warp * (d + 1) + 1 + k] += v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) acc[warp * (d + 1)] += s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d + 1; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < warps; ++w) t += acc[w * (d + 1) + k];
    partial[(int64_t)blockIdx.x * (d + 1) + k] = t;
  }
}

// Pass 2: out[k] = sum_b partial[b][k], in block order.
__global__ void sum_parts(const double* __restrict__ partial, int parts, int width, double* __restrict__ out) {
  for (int k = threadIdx.x; k < width; k += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < parts; ++b) t += partial[(int64_t)b * width + k];
    out[k] = t;
  }
}

__global__ void sq_error_pass1(const float* __restrict__ A, const float* __restrict__ B, int64_t n, int32_t d,
                               double* __restrict__ partial) {
  __shared__ double red[32];
  double s = 0.0;
  const int64_t total = n * (int64_t)d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)A[e] - (double)B[e];
    s += v * v;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// Pass 1 of the coupling diagonal (n = m): log P_ii = (f_i + g_i - |x_i - y_i|^2) / eps
// with the squared distance summed in float64 from the differences; block b sums
// P_ii and log P_ii over rows b, b + parts, ... (one warp per row).
__global__ void diag_pass1(const float* __restrict__ X, const float* __restrict__ Y, const float* __restrict__ f,
                           const float* __restrict__ g, int64_t n, int32_t d, double inv_eps,
                           float* __restrict__ logd, double* __restrict__ partial) {
  __shared__ double red[2][32];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double sp = 0.0, sl = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * warps + warp; row < n; row += (int64_t)gridDim.x * warps) {
    const float* x = X + row * (int64_t)d;
    const float* y = Y + row * (int64_t)d;
    double c = 0.0;
    for (int k = lane; k < d; k += 32) {
      const double v = (double)x[k] - (double)y[k];
      c += v * v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) {
      const double lp = ((double)f[row] + (double)g[row] - c) * inv_eps;
      if (logd) logd[row] = (float)lp;
      sp += exp(lp);
      sl += lp;
    }
  }
  if (lane == 0) {
    red[0][warp] = sp;
    red[1][warp] = sl;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < warps; ++w) t += red[threadIdx.x][w];
    partial[(int64_t)blockIdx.x * 2 + threadIdx.x] = t;
  }
}

// Closed-form mean cost over all pairs from first moments (exact for h = |.|^2):
// mean |x|^2 + mean |y|^2 - 2 xbar . ybar, with mx = (sum |x_i|^2, sum x_i), my likewise.
__global__ void mean_cost_closed(const double* __restrict__ mx, const double* __restrict__ my, int64_t n, int64_t m,
                                 int32_t d, double* __restrict__ out) {
  __shared__ double red[32];
  double dot = 0.0;
  for (int k = threadIdx.x; k < d; k += blockDim.x) dot += (mx[1 + k] / (double)n) * (my[1 + k] / (double)m);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = mx[0] / (double)n + my[0] / (double)m - 2.0 * t;
  }
}

cudaError_t launch_row_sqnorm(const float* X, int64_t n, int32_t d, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int rows_per_block = 8;
  const int64_t blocks = (n + rows_per_block - 1) / rows_per_block;
  row_sqnorm_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, n, d, out);
  count_launch();
  return cudaGetLastError();
}

// Per-coordinate column sums of X (blockIdx.y = 0) and Y (blockIdx.y = 1) in float64, in a
// fixed order: warp w of block b sums rows b W + w + k gridDim.x W (W warps per block),
// then the block adds its warps' sums in warp order.
__global__ void center_pass1(const float* __restrict__ X, int64_t n, const float* __restrict__ Y, int64_t m,
                             int32_t d, double* __restrict__ partial) {
  extern __shared__ double acc[];  // d per warp
  const float* Z = blockIdx.y ? Y : X;
  const int64_t rows = blockIdx.y ? m : n;
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < warps * d; k += blockDim.x) acc[k] = 0.0;
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * warps + warp; row < rows; row += (int64_t)gridDim.x * warps)
    for (int k = lane; k < d; k += 32) acc[warp * d + k] += (double)Z[row * (int64_t)d + k];
  __syncthreads();
  double* out = partial + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * d;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < warps; ++w) t += acc[w * d + k];
    out[k] = t;
  }
}

// mu_k = (sum_x_k / n + sum_y_k / m) / 2 from the block partials: one warp per
// coordinate, lane l summing blocks l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void center_finish(const double* __restrict__ partial, int parts, int64_t n, int64_t m, int32_t d,
                              float* __restrict__ mu) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= d) return;
  double sx = 0.0, sy = 0.0;
  for (int b = lane; b < parts; b += 32) {
    sx += partial[(int64_t)b * d + k];
    sy += partial[((int64_t)parts + b) * d + k];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
  }
  if (lane == 0) mu[k] = (float)(0.5 * (sx / (double)n + sy / (double)m));
}

cudaError_t launch_center(const float* X, int64_t n, const float* Y, int64_t m, int32_t d, double* partial, float* mu,
                          cudaStream_t s) {
  const size_t per_warp = sizeof(double) * (size_t)d;
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / per_warp));
  const size_t smem = per_warp * (size_t)warps;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;  // d above 25,600
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(center_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int parts = kParts / 2;
  center_pass1<<<dim3(parts, 2), 32 * warps, smem, s>>>(X, n, Y, m, d, partial);
  count_launch();
  center_finish<<<(d + 7) / 8, 256, 0, s>>>(partial, parts, n, m, d, mu);
  count_launch();
  return cudaGetLastError();
}

// L_i += bscale (|x_i|^2 - |x_i - mu|^2) = bscale (2 x_i . mu - |mu|^2): moves a row
// log-sum-exp taken on centred operands to the uncentred form t_ij = scale x_i . y_j +
// (g_j - |y_j|^2) bscale (one warp per row, float64 sums).
__global__ void lse_uncenter_kernel(float* __restrict__ L, const float* __restrict__ X, int64_t n, int32_t d,
                                    const float* __restrict__ mu, float bscale) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* x = X + row * (int64_t)d;
  double s = 0.0;
  for (int k = lane; k < d; k += 32) {
    const double u = (double)mu[k];
    s += (2.0 * (double)x[k] - u) * u;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) L[row] = (float)((double)L[row] + (double)bscale * s);
}

cudaError_t launch_lse_uncenter(float* L, const float* X, int64_t n, int32_t d, const float* mu, float bscale,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  lse_uncenter_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(L, X, n, d, mu, bscale);
  count_launch();
  return cudaGetLastError();
}

// L_i = (eps log w_i + |a_i|^2 - f_i) / (eps ln2): the row log-sum-exp (log2 units) that
// an f-update wrote as the potential f_i = eps log w_i + |a_i|^2 - eps ln2 L_i, recovered
// from f in float64 (w = NULL: uniform weights, log w_i = log_w_uniform).
__global__ void lse_from_potential_kernel(const float* __restrict__ f, const float* __restrict__ an,
                                          const float* __restrict__ w, double log_w_uniform, double eps, int64_t n,
                                          float* __restrict__ L) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double logw = w ? log((double)w[i]) : log_w_uniform;
  L[i] = (float)((eps * logw + (double)an[i] - (double)f[i]) / (eps * 0.69314718055994530942));
}

cudaError_t launch_lse_from_potential(const float* f, const float* an, const float* w, double log_w_uniform,
                                      double eps, int64_t n, float* L, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  lse_from_potential_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, an, w, log_w_uniform, eps, n, L);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale(float* v, int64_t n, float factor, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  scale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, n, factor);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_init_state(SolverState* st, cudaStream_t s) {
  init_state_kernel<<<1, 1, 0, s>>>(st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_moments(const float* X, int64_t n, int32_t d, double* partial, int parts, double* out,
                           cudaStream_t s) {
  // up to 8 warps, each with its own d + 1 float64 accumulators in shared memory
  const size_t per_warp = sizeof(double) * (size_t)(d + 1);
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / per_warp));
  const int threads = 32 * warps;
  const size_t smem = per_warp * (size_t)warps;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;  // d above 25,598
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(moments_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  moments_pass1<<<parts, threads, smem, s>>>(X, n, d, partial);
  count_launch();
  sum_parts<<<1, 256, 0, s>>>(partial, parts, d + 1, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sq_error(const float* A, const float* B, int64_t n, int32_t d, double* partial, int parts,
                            double* out, cudaStream_t s) {
  sq_error_pass1<<<parts, 256, 0, s>>>(A, B, n, d, partial);
  count_launch();
  sum_parts<<<1, 32, 0, s>>>(partial, parts, 1, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_diag(const float* X, const float* Y, const float* f, const float* g, int64_t n, int32_t d, double eps,
                        float* logd, double* partial, int parts, double* out, cudaStream_t s) {
  diag_pass1<<<parts, 256, 0, s>>>(X, Y, f, g, n, d, 1.0 / eps, logd, partial);
  count_launch();
  sum_parts<<<1, 32, 0, s>>>(partial, parts, 2, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mean_cost_closed(const double* mx, const double* my, int64_t n, int64_t m, int32_t d, double* out,
                                    cudaStream_t s) {
  mean_cost_closed<<<1, 256, 0, s>>>(mx, my, n, m, d, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sum_parts(const double* partial, int parts, int width, double* out, cudaStream_t s) {
  sum_parts<<<1, 32, 0, s>>>(partial, parts, width, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace progot
