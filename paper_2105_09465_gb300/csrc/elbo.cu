// Likelihood and ELBO terms of one reparameterised draw (Sec. 3.3 generative
// model, Sec. 3.6 ELBO, Sec. 3.7 mean-field proposal, Sec. 4.2 partial
// multivariate-normal proposal). All of it is elementwise, HBM-bound work
// with a few scalar sums. Per-element values are FP32 (logf, FP32
// reciprocals: FP64 transcendentals run at a small fraction of the FP32 rate
// on this part); the sums accumulate in FP64, in an order fixed by the
// problem size alone (per-thread strided partials, a fixed tree per block,
// and the last block to finish summing the block partials in block order),
// so results are bit-reproducible run to run.
#include <math.h>

#include "host.cuh"

namespace lr {

constexpr int kRedThreads = 256;
constexpr int kRedBlocksMax = 1216;
constexpr int kMvnDMax = 32;
constexpr double kLog2Pi = 1.8378770664093454836;

static int red_blocks(int64_t n) {
  const int64_t b = (n + kRedThreads - 1) / kRedThreads;
  return (int)(b < 1 ? 1 : (b > kRedBlocksMax ? kRedBlocksMax : b));
}

// Workspace: a completion counter, then kRedBlocksMax x K block partials.
struct RedWs {
  unsigned* counter;
  double* part;
};

static RedWs red_ws(void* ws) {
  char* w = static_cast<char*>(ws);
  return RedWs{reinterpret_cast<unsigned*>(w), reinterpret_cast<double*>(w + 256)};
}

static size_t red_ws_bytes(int K) { return 256 + align256(sizeof(double) * K * kRedBlocksMax); }

// Sum v[0..K) over the block in a fixed tree; the result is valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sh[K][kRedThreads];
#pragma unroll
  for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k][0];
  __syncthreads();
}

// Publish this block's sums; returns true in every thread of the last block
// to arrive, whose `v` then holds the totals over all blocks (block order).
template <int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], RedWs w) {
  __shared__ bool last;
  block_sum<K>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) w.part[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    last = atomicAdd(w.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kRedThreads) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(w.part + (size_t)b * K + k);
  }
  block_sum<K>(acc);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = acc[k];
  if (threadIdx.x == 0) *w.counter = 0u;
  return true;
}

// ---------------------------------------------------------------- likelihood
struct NllArgs {
  const float* f;
  const float* data;
  const float* sigma;
  float sigma0;
  int32_t nx, ny, ss;
  float* g;
  float* model;
  double* nll;
};

__global__ void __launch_bounds__(kRedThreads) nll_kernel(const __grid_constant__ NllArgs A, RedWs w) {
  const int64_t P = (int64_t)A.nx * A.ny;
  const int64_t W = (int64_t)A.nx * A.ss;
  const double inv_ss2 = 1.0 / ((double)A.ss * A.ss);
  double acc[1] = {0.0};
  for (int64_t p = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; p < P; p += (int64_t)gridDim.x * kRedThreads) {
    const int64_t r = p / A.nx, c = p - r * A.nx;
    const int64_t base = r * A.ss * W + c * A.ss;
    double m = 0.0;
    for (int a = 0; a < A.ss; ++a)
      for (int b = 0; b < A.ss; ++b) m += (double)A.f[base + a * W + b];
    m *= inv_ss2;
    const float s = A.sigma ? A.sigma[p] : A.sigma0;
    const double res = m - (double)A.data[p];
    const double is2 = (double)(1.0f / (s * s));
    acc[0] += 0.5 * res * res * is2 + (double)logf(s);
    if (A.model) A.model[p] = (float)m;
    if (A.g) {
      const float gv = (float)(res * is2 * inv_ss2);
      for (int a = 0; a < A.ss; ++a)
        for (int b = 0; b < A.ss; ++b) A.g[base + a * W + b] = gv;
    }
  }
  if (grid_sum<1>(acc, w) && threadIdx.x == 0) *A.nll = acc[0] + 0.5 * (double)P * kLog2Pi;
}

// ---------------------------------------------------------------- diagonal normal proposal
struct DiagArgs {
  const float* mu;
  const float* sd;
  const float* eps;
  int64_t m;
  float alpha;
  float* y;           // draw
  double* terms;      // [-ln p(y | alpha), ln q(y)]
  const float* d_y;   // vjp: upstream gradient
  double w_prior, w_q;
  float* d_mu;
  float* d_sd;
  double* d_alpha;
};

__global__ void __launch_bounds__(kRedThreads) diag_draw_kernel(const __grid_constant__ DiagArgs A, RedWs w) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < A.m; i += (int64_t)gridDim.x * kRedThreads) {
    const float e = A.eps[i], s = A.sd[i];
    const float y = fmaf(s, e, A.mu[i]);
    A.y[i] = y;
    acc[0] += (double)y * y;
    acc[1] += (double)fmaf(-0.5f * e, e, -logf(s));
  }
  if (grid_sum<2>(acc, w) && threadIdx.x == 0) {
    const double a = A.alpha, M = (double)A.m;
    A.terms[0] = acc[0] / (2.0 * a * a) + M * log(a) + 0.5 * M * kLog2Pi;
    A.terms[1] = acc[1] - 0.5 * M * kLog2Pi;
  }
}

__global__ void __launch_bounds__(kRedThreads) diag_vjp_kernel(const __grid_constant__ DiagArgs A, RedWs w) {
  const float wp_ia2 = (float)(A.w_prior / ((double)A.alpha * A.alpha)), wq = (float)A.w_q;
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < A.m; i += (int64_t)gridDim.x * kRedThreads) {
    const float e = A.eps[i], s = A.sd[i];
    const float y = fmaf(s, e, A.mu[i]);
    const float t = fmaf(wp_ia2, y, A.d_y[i]);
    A.d_mu[i] = t;
    A.d_sd[i] = fmaf(t, e, -wq / s);
    acc[0] += (double)y * y;
  }
  if (grid_sum<1>(acc, w) && threadIdx.x == 0) {
    const double a = A.alpha;
    *A.d_alpha = A.w_prior * ((double)A.m / a - acc[0] / (a * a * a));
  }
}

// ---------------------------------------------------------------- partial MVN proposal
struct MvnArgs {
  const float* mu;   // D + M
  const float* L;    // D x D row-major, lower triangle read
  const float* C;    // M x D row-major
  const float* sd;   // M
  const float* eps;  // D + M
  int32_t D;
  int64_t M;
  float* x;          // D + M
  double* logq;
  const float* d_x;  // vjp
  double w_q;
  float* d_mu;
  float* d_L;
  float* d_C;
  float* d_sd;
};

__global__ void __launch_bounds__(kRedThreads) mvn_draw_kernel(const __grid_constant__ MvnArgs A, RedWs w) {
  __shared__ float e1[kMvnDMax];
  const int D = A.D;
  if ((int)threadIdx.x < D) e1[threadIdx.x] = A.eps[threadIdx.x];
  __syncthreads();
  if (blockIdx.x == 0 && (int)threadIdx.x < D) {
    const int i = threadIdx.x;
    double s = A.mu[i];
    for (int j = 0; j <= i; ++j) s += (double)A.L[i * D + j] * e1[j];
    A.x[i] = (float)s;
  }
  double acc[1] = {0.0};
  for (int64_t j = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; j < A.M; j += (int64_t)gridDim.x * kRedThreads) {
    const float* c = A.C + j * D;
    double s = A.mu[D + j];
    for (int l = 0; l < D; ++l) s += (double)c[l] * e1[l];
    const float e2 = A.eps[D + j], sdv = A.sd[j];
    A.x[D + j] = (float)(s + (double)sdv * e2);
    acc[0] += (double)fmaf(-0.5f * e2, e2, -logf(sdv));
  }
  if (grid_sum<1>(acc, w) && threadIdx.x == 0) {
    double lens = 0.0;
    for (int i = 0; i < D; ++i) lens += (double)fmaf(-0.5f * e1[i], e1[i], -logf(A.L[i * D + i]));
    *A.logq = acc[0] + lens - 0.5 * (double)(D + A.M) * kLog2Pi;
  }
}

__global__ void __launch_bounds__(kRedThreads) mvn_vjp_kernel(const __grid_constant__ MvnArgs A) {
  __shared__ float e1[kMvnDMax];
  const int D = A.D;
  if ((int)threadIdx.x < D) e1[threadIdx.x] = A.eps[threadIdx.x];
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kRedThreads + threadIdx.x, stride = (int64_t)gridDim.x * kRedThreads;
  for (int64_t k = t0; k < (int64_t)D * D; k += stride) {
    const int i = (int)(k / D), j = (int)(k - (int64_t)i * D);
    float g = j <= i ? A.d_x[i] * e1[j] : 0.f;
    if (i == j) g -= (float)A.w_q / A.L[i * D + i];
    A.d_L[k] = g;
  }
  for (int64_t k = t0; k < (int64_t)D + A.M; k += stride) A.d_mu[k] = A.d_x[k];
  for (int64_t k = t0; k < A.M * D; k += stride) {
    const int64_t j = k / D;
    const int l = (int)(k - j * D);
    A.d_C[k] = A.d_x[D + j] * e1[l];
  }
  const float wq = (float)A.w_q;
  for (int64_t j = t0; j < A.M; j += stride) A.d_sd[j] = fmaf(A.d_x[D + j], A.eps[D + j], -wq / A.sd[j]);
}

static lr_status red_check(void* ws, size_t bytes, int K, const char* what) {
  LR_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255u) == 0 && bytes >= red_ws_bytes(K),
             "%s: workspace of %zu bytes (256-byte aligned) needed", what, red_ws_bytes(K));
  return LR_OK;
}

}  // namespace lr

using namespace lr;

extern "C" size_t lr_elbo_workspace_size(void) { return red_ws_bytes(2); }

extern "C" lr_status gp_gaussian_nll(const float* f, int64_t n, const lr_grid* grid, const float* data,
                                     const float* sigma, float sigma0, float* g_out, float* model_out,
                                     double* nll_out, void* workspace, size_t workspace_bytes, lr_stream stream) {
  NllArgs A{};
  if (grid) {
    LR_REQUIRE(grid->nx > 0 && grid->ny > 0 && grid->ss > 0, "gp_gaussian_nll: bad grid");
    LR_REQUIRE((int64_t)grid->nx * grid->ss * grid->ny * grid->ss == n, "gp_gaussian_nll: n != grid points");
    A.nx = grid->nx;
    A.ny = grid->ny;
    A.ss = grid->ss;
  } else {
    LR_REQUIRE(n > 0 && n < (int64_t(1) << 31), "gp_gaussian_nll: n out of range");
    A.nx = (int32_t)n;
    A.ny = 1;
    A.ss = 1;
  }
  LR_REQUIRE(f && data && nll_out, "gp_gaussian_nll: NULL f, data or nll_out");
  LR_REQUIRE(sigma != nullptr || (isfinite(sigma0) && sigma0 > 0.f), "gp_gaussian_nll: sigma0 must be > 0");
  lr_status st = red_check(workspace, workspace_bytes, 1, "gp_gaussian_nll");
  if (st != LR_OK) return st;
  A.f = f;
  A.data = data;
  A.sigma = sigma;
  A.sigma0 = sigma0;
  A.g = g_out;
  A.model = model_out;
  A.nll = nll_out;
  RedWs w = red_ws(workspace);
  cudaStream_t s = as_cuda(stream);
  LR_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned), s));
  nll_kernel<<<red_blocks((int64_t)A.nx * A.ny), kRedThreads, 0, s>>>(A, w);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status gp_diag_normal_draw(const float* mu, const float* sd, const float* eps, int64_t m, float alpha,
                                         float* y_out, double* terms_out, void* workspace, size_t workspace_bytes,
                                         lr_stream stream) {
  LR_REQUIRE(m > 0 && mu && sd && eps && y_out && terms_out, "gp_diag_normal_draw: NULL pointer or m <= 0");
  LR_REQUIRE(isfinite(alpha) && alpha > 0.f, "gp_diag_normal_draw: alpha must be > 0");
  lr_status st = red_check(workspace, workspace_bytes, 2, "gp_diag_normal_draw");
  if (st != LR_OK) return st;
  DiagArgs A{};
  A.mu = mu;
  A.sd = sd;
  A.eps = eps;
  A.m = m;
  A.alpha = alpha;
  A.y = y_out;
  A.terms = terms_out;
  RedWs w = red_ws(workspace);
  cudaStream_t s = as_cuda(stream);
  LR_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned), s));
  diag_draw_kernel<<<red_blocks(m), kRedThreads, 0, s>>>(A, w);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status gp_diag_normal_vjp(const float* mu, const float* sd, const float* eps, int64_t m, float alpha,
                                        const float* d_y, double w_prior, double w_q, float* d_mu, float* d_sd,
                                        double* d_alpha, void* workspace, size_t workspace_bytes, lr_stream stream) {
  LR_REQUIRE(m > 0 && mu && sd && eps && d_y && d_mu && d_sd && d_alpha, "gp_diag_normal_vjp: NULL pointer or m <= 0");
  LR_REQUIRE(isfinite(alpha) && alpha > 0.f, "gp_diag_normal_vjp: alpha must be > 0");
  lr_status st = red_check(workspace, workspace_bytes, 1, "gp_diag_normal_vjp");
  if (st != LR_OK) return st;
  DiagArgs A{};
  A.mu = mu;
  A.sd = sd;
  A.eps = eps;
  A.m = m;
  A.alpha = alpha;
  A.d_y = d_y;
  A.w_prior = w_prior;
  A.w_q = w_q;
  A.d_mu = d_mu;
  A.d_sd = d_sd;
  A.d_alpha = d_alpha;
  RedWs w = red_ws(workspace);
  cudaStream_t s = as_cuda(stream);
  LR_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned), s));
  diag_vjp_kernel<<<red_blocks(m), kRedThreads, 0, s>>>(A, w);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status gp_partial_mvn_draw(const float* mu, const float* L, const float* C, const float* sd,
                                         const float* eps, int32_t D, int64_t M, float* x_out, double* logq_out,
                                         void* workspace, size_t workspace_bytes, lr_stream stream) {
  LR_REQUIRE(D >= 1 && D <= kMvnDMax && M >= 0, "gp_partial_mvn_draw: need 1 <= D <= %d, M >= 0", kMvnDMax);
  LR_REQUIRE(mu && L && eps && x_out && logq_out && (M == 0 || (C && sd)), "gp_partial_mvn_draw: NULL pointer");
  lr_status st = red_check(workspace, workspace_bytes, 1, "gp_partial_mvn_draw");
  if (st != LR_OK) return st;
  MvnArgs A{};
  A.mu = mu;
  A.L = L;
  A.C = C;
  A.sd = sd;
  A.eps = eps;
  A.D = D;
  A.M = M;
  A.x = x_out;
  A.logq = logq_out;
  RedWs w = red_ws(workspace);
  cudaStream_t s = as_cuda(stream);
  LR_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned), s));
  mvn_draw_kernel<<<red_blocks(M), kRedThreads, 0, s>>>(A, w);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status gp_partial_mvn_vjp(const float* L, const float* sd, const float* eps, int32_t D, int64_t M,
                                        const float* d_x, double w_q, float* d_mu, float* d_L, float* d_C,
                                        float* d_sd, lr_stream stream) {
  LR_REQUIRE(D >= 1 && D <= kMvnDMax && M >= 0, "gp_partial_mvn_vjp: need 1 <= D <= %d, M >= 0", kMvnDMax);
  LR_REQUIRE(L && eps && d_x && d_mu && d_L && (M == 0 || (sd && d_C && d_sd)), "gp_partial_mvn_vjp: NULL pointer");
  MvnArgs A{};
  A.L = L;
  A.sd = sd;
  A.eps = eps;
  A.D = D;
  A.M = M;
  A.d_x = d_x;
  A.w_q = w_q;
  A.d_mu = d_mu;
  A.d_L = d_L;
  A.d_C = d_C;
  A.d_sd = d_sd;
  const int64_t work = M * D > (int64_t)D * D ? M * D : (int64_t)D * D;
  mvn_vjp_kernel<<<red_blocks(work), kRedThreads, 0, as_cuda(stream)>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
