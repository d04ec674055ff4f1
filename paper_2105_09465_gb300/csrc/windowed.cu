// Pixel windows and the windowed (non-stationary) transmission reduction of
// the paper's image-plane model (Sec. 3.2 window-function and window-kernel
// equations, Sec. 3.4 transmission equation):
//   Z_i = (a_i a_i^T + b_i b_i^T) / (4 pi)   from the projected pixel grid,
//   out_i = sum_k G(p_i - q_k, Z_i + (l^2/2) I) v_k,
//   G(d, C) = exp(-d^T C^-1 d / 2) / (2 pi sqrt(det C)),
// with the transmission weights A_k folded into v_k by the caller. Each
// query row carries its own window constants, prepared once with C and
// det C in FP64 (launch_window_prep): the Cholesky factor (a, b, c) of C^-1
// pre-scaled for exp2 and the normalisation; per pair the exponent is
// -((a dx + b dy)^2 + (c dy)^2). Grid sources: the grid tiling, chunking and
// fixed-order merge of the stationary reduction (windowed_kernel). Explicit
// sources (the image-plane layers, the pixels against themselves): the
// culled sweep of cull.cu, which leaves out the pairs whose exponent is below
// -126 by bounding boxes.
#include <math.h>

#include "cull.cuh"
#include "host.cuh"
#include "problems.cuh"

namespace lr {

constexpr int kWnThreads = 128;
constexpr int kWnR = 4;
constexpr int kWnRows = kWnThreads * kWnR;
constexpr int kWnTile = 256;
constexpr int kWnPairs = kWnTile / 2;
static_assert(kWnPairs == kWnThreads, "one source pair per thread when staging");
constexpr int kWnSeg = 16;  // grid sub-segment (columns) of the tile-local abscissae

__global__ void pixel_shapes_kernel(const float2* __restrict__ p, int32_t W, int32_t H, float* __restrict__ z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)W * H) return;
  const int32_t r = (int32_t)(i / W), c = (int32_t)(i - (int64_t)r * W);
  const int64_t cl = c > 0 ? i - 1 : i, cr = c + 1 < W ? i + 1 : i;
  const int64_t rd = r > 0 ? i - W : i, ru = r + 1 < H ? i + W : i;
  const float sa = (cr - cl == 2) ? 0.5f : 1.0f, sb = (ru - rd == 2 * (int64_t)W) ? 0.5f : 1.0f;
  const float2 pl = p[cl], pr = p[cr], pd = p[rd], pu = p[ru];
  const float ax = sa * (pr.x - pl.x), ay = sa * (pr.y - pl.y);
  const float bx = sb * (pu.x - pd.x), by = sb * (pu.y - pd.y);
  const float k = 0.0795774715459477f;  // 1 / (4 pi)
  z[3 * i] = k * fmaf(ax, ax, bx * bx);
  z[3 * i + 1] = k * fmaf(ax, ay, bx * by);
  z[3 * i + 2] = k * fmaf(ay, ay, by * by);
}

struct WnArgs {
  const float2* p;
  const float4* wcoef;  // the rows' window constants (launch_window_prep)
  int64_t n;
  GridDev g;        // the source grid
  int64_t m;
  int32_t segs, n_tiles, chunks;
  const float* v;
  float* out;
  float* partial;
};

__device__ __forceinline__ float2 wf2(float a, float b) { return make_float2(a, b); }

// Source tile t: a 256-column segment of one grid row.
__device__ __forceinline__ void wn_tile(const WnArgs& A, int t, int64_t& j0, int& cnt, int& grow) {
  grow = t / A.segs;
  const int c0 = (t - grow * A.segs) * kWnTile;
  cnt = min(kWnTile, A.g.W - c0);
  j0 = (int64_t)grow * A.g.W + c0;
}

__device__ __forceinline__ void wn_load(const WnArgs& A, int t, int p, float4& P, float2& V) {
  int64_t j0;
  int cnt, grow;
  wn_tile(A, t, j0, cnt, grow);
  const int a = 2 * p, b = 2 * p + 1;
  // abscissae relative to the centre column of their 16-column sub-segment
  const int c0 = (int)(j0 - (int64_t)grow * A.g.W);
  const float o = grid_x(A.g, c0 + kWnSeg * (a / kWnSeg) + kWnSeg / 2);
  P = make_float4((a < cnt) ? grid_x(A.g, c0 + a) - o : 0.f, (b < cnt) ? grid_x(A.g, c0 + b) - o : 0.f, 0.f, 0.f);
  V = wf2((a < cnt) ? __ldg(A.v + j0 + a) : 0.f, (b < cnt) ? __ldg(A.v + j0 + b) : 0.f);
}

__global__ void __launch_bounds__(kWnThreads) windowed_kernel(const __grid_constant__ WnArgs A) {
  __shared__ __align__(16) float4 sP[2][kWnPairs];
  __shared__ __align__(16) float2 sV[2][kWnPairs];
  __shared__ float ksum[kWnR][kWnThreads], kcomp[kWnR][kWnThreads];
  const int rb = blockIdx.x / A.chunks;
  const int chunk = blockIdx.x - rb * A.chunks;
  const int t0 = (int)((int64_t)chunk * A.n_tiles / A.chunks);
  const int t1 = (int)((int64_t)(chunk + 1) * A.n_tiles / A.chunks);
  const int tid = threadIdx.x;
  // per row: the scaled Cholesky factor (a, b, c) of C^-1 and N (window
  // constants prepared with C and det C in FP64: cull.cuh), so that the
  // exponent is -((a dx + b dy)^2 + (c dy)^2) with d = x_i - y_j
  float2 xq[kWnR], yq[kWnR], acc[kWnR];
  float ca[kWnR], boa[kWnR], cc[kWnR], norm[kWnR];
#pragma unroll
  for (int r = 0; r < kWnR; ++r) {
    int64_t i = (int64_t)rb * kWnRows + r * kWnThreads + tid;
    if (i >= A.n) i = A.n - 1;
    const float2 pp = __ldg(A.p + i);
    const float4 wc = A.wcoef[i];
    xq[r] = wf2(pp.x, pp.x);
    yq[r] = wf2(pp.y, pp.y);
    ca[r] = wc.x;
    boa[r] = wc.y / wc.x;
    cc[r] = wc.z;
    norm[r] = wc.w;
    acc[r] = wf2(0.f, 0.f);
    ksum[r][tid] = 0.f;
    kcomp[r][tid] = 0.f;
  }
  float4 P;
  float2 V;
  if (t0 < t1) {
    wn_load(A, t0, tid, P, V);
    sP[0][tid] = P;
    sV[0][tid] = V;
  }
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    if (t + 1 < t1) wn_load(A, t + 1, tid, P, V);
    int64_t j0;
    int cnt, grow;
    wn_tile(A, t, j0, cnt, grow);
    {
      // Uniform y on a grid row: the Cholesky form is a completed square in
      // dx, t = a^2 (dx + (b/a) dy)^2 + (c dy)^2, so with
      // w = a ((x_i - o) + (b/a) dy) - a (x_j - o) the pair needs one packed
      // FMA for w of two pairs, one for t = w^2 + (c dy)^2, the exp2 of -t
      // and one packed FMA to accumulate.
      const float yt = grid_y(A.g, grow);
      const int c0 = (int)(j0 - (int64_t)grow * A.g.W);
      float kdy[kWnR], sr[kWnR];
      float2 t0[kWnR], ns[kWnR];
#pragma unroll
      for (int r = 0; r < kWnR; ++r) {
        const float dy = yq[r].x - yt, cdy = cc[r] * dy;
        sr[r] = ca[r];
        kdy[r] = boa[r] * dy;
        t0[r] = wf2(cdy * cdy, cdy * cdy);
        ns[r] = wf2(-sr[r], -sr[r]);
      }
      const int nsg = (cnt + kWnSeg - 1) / kWnSeg;
      for (int sg = 0; sg < nsg; ++sg) {
        const float o = grid_x(A.g, c0 + kWnSeg * sg + kWnSeg / 2);
        float2 qc[kWnR];
#pragma unroll
        for (int r = 0; r < kWnR; ++r) {
          const float q = sr[r] * ((xq[r].x - o) + kdy[r]);  // small terms first: no large-ulp rounding
          qc[r] = wf2(q, q);
        }
#pragma unroll
        for (int pp = 0; pp < kWnSeg / 2; ++pp) {
          const int p = sg * (kWnSeg / 2) + pp;
          const float4 Q = sP[buf][p];
          const float2 W = sV[buf][p];
          const float2 X = wf2(Q.x, Q.y);
#pragma unroll
          for (int r = 0; r < kWnR; ++r) {
            const float2 w = __ffma2_rn(ns[r], X, qc[r]);
            const float2 t = __ffma2_rn(w, w, t0[r]);
            const float2 k = wf2(ex2_approx(-t.x), ex2_approx(-t.y));
            acc[r] = __ffma2_rn(k, W, acc[r]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kWnR; ++r) {
      const float y = (acc[r].x + acc[r].y) - kcomp[r][tid];
      const float s = ksum[r][tid] + y;
      kcomp[r][tid] = (s - ksum[r][tid]) - y;
      ksum[r][tid] = s;
      acc[r] = wf2(0.f, 0.f);
    }
    if (t + 1 < t1) {
      sP[buf ^ 1][tid] = P;
      sV[buf ^ 1][tid] = V;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kWnR; ++r) {
    const int64_t i = (int64_t)rb * kWnRows + r * kWnThreads + tid;
    if (i < A.n) {
      const float total = norm[r] * (ksum[r][tid] - kcomp[r][tid]);
      if (A.chunks == 1)
        A.out[i] = total;
      else
        A.partial[(int64_t)chunk * A.n + i] = total;
    }
  }
}

__global__ void windowed_merge_kernel(const float* __restrict__ partial, int chunks, int64_t n,
                                      float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f, c = 0.f;
  for (int k = 0; k < chunks; ++k) {
    const float y = partial[(int64_t)k * n + i] - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  out[i] = s - c;
}

// nll += c (the likelihood's constant terms), one thread.
__global__ void add_const_kernel(double* __restrict__ x, double c) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *x += c;
}

struct WnPlan {
  int32_t n_tiles, segs, chunks, row_blocks;  // grid sources
  int32_t culled;                             // explicit sources: the culled sweep
  CullPlan C;
  size_t off_wcoef, off_wreach;               // the rows' window constants
  size_t bytes;
};

// The query layout, when given, must describe exactly the n query points.
static lr_status check_layout(const lr_grid* layout, int64_t n, const char* what) {
  if (!layout) return LR_OK;
  LR_REQUIRE(layout->nx > 0 && layout->ny > 0 && layout->ss > 0 &&
                 (int64_t)layout->nx * layout->ss * layout->ny * layout->ss == n,
             "%s: the layout (%d x %d x %d^2) does not hold the %lld query points", what, layout->nx, layout->ny,
             layout->ss, (long long)n);
  return LR_OK;
}

static lr_status plan_windowed(int64_t n, const lr_grid* layout, const lr_points* s, WnPlan* P) {
  lr_status st = validate_points(s, "gp_windowed_matvec(source)", false);
  if (st != LR_OK) return st;
  LR_REQUIRE(!has_lens(s), "gp_windowed_matvec: sources must not carry a lens");
  LR_REQUIRE(n >= 0 && n < (int64_t(1) << 31), "gp_windowed_matvec: n out of range");
  if ((st = check_layout(layout, n, "gp_windowed_matvec")) != LR_OK) return st;
  WnPlan p{};
  if (s->xy != nullptr) {
    p.culled = 1;
    st = plan_cull(kCullWin, 1, n, layout, s->n, query_layout(s), &p.C);
    if (st != LR_OK) return st;
    p.off_wcoef = align256(p.C.bytes);
    p.off_wreach = p.off_wcoef + align256(16 * (size_t)n);
    p.bytes = p.off_wreach + align256(4 * (size_t)n);
    *P = p;
    return LR_OK;
  }
  const int W = s->grid.nx * s->grid.ss;
  p.segs = (W + kWnTile - 1) / kWnTile;
  p.n_tiles = (int32_t)((int64_t)p.segs * s->grid.ny * s->grid.ss);
  p.row_blocks = (int32_t)((n + kWnRows - 1) / kWnRows);
  int dev = 0, n_sm = 1, occ = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, windowed_kernel, kWnThreads, 0));
  p.chunks = plan_chunks(p.row_blocks, p.n_tiles, occ, n_sm);
  p.off_wcoef = p.chunks > 1 ? align256(4 * (size_t)p.chunks * (size_t)n) : 0;
  p.off_wreach = p.off_wcoef + align256(16 * (size_t)n);
  p.bytes = p.off_wreach + align256(4 * (size_t)n);
  *P = p;
  return LR_OK;
}

}  // namespace lr

using namespace lr;

extern "C" lr_status gp_pixel_shapes(const float* p, int32_t W, int32_t H, float* z, lr_stream stream) {
  LR_REQUIRE(W >= 1 && H >= 1 && (int64_t)W * H < (int64_t(1) << 31), "gp_pixel_shapes: bad grid %d x %d", W, H);
  LR_REQUIRE(p != nullptr && z != nullptr, "gp_pixel_shapes: NULL pointer");
  LR_REQUIRE(((uintptr_t)p & 7u) == 0 && ((uintptr_t)z & 3u) == 0, "gp_pixel_shapes: misaligned pointer");
  const int64_t n = (int64_t)W * H;
  pixel_shapes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, as_cuda(stream)>>>(reinterpret_cast<const float2*>(p),
                                                                                  W, H, z);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status lr_windowed_workspace_size(int64_t n, const lr_grid* layout, const lr_points* source,
                                                size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_windowed_workspace_size: bytes is NULL");
  WnPlan P;
  lr_status st = plan_windowed(n, layout, source, &P);
  if (st != LR_OK) return st;
  *bytes = P.bytes;
  return LR_OK;
}

extern "C" lr_status gp_windowed_matvec(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                        const lr_points* source, const float* v, float lengthscale, float* out,
                                        void* workspace, size_t workspace_bytes, lr_stream stream) {
  WnPlan P;
  lr_status st = plan_windowed(n, layout, source, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "gp_windowed_matvec: lengthscale must be > 0");
  LR_REQUIRE(n == 0 || (p != nullptr && z != nullptr && out != nullptr), "gp_windowed_matvec: NULL pointer");
  LR_REQUIRE(((uintptr_t)p & 7u) == 0 && ((uintptr_t)z & 3u) == 0, "gp_windowed_matvec: misaligned p or z");
  LR_REQUIRE(v != nullptr || source->n == 0, "gp_windowed_matvec: v is NULL");
  LR_REQUIRE(workspace_bytes >= P.bytes && (P.bytes == 0 || workspace != nullptr),
             "gp_windowed_matvec: workspace of %zu bytes, %zu needed", workspace_bytes, P.bytes);
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0, "gp_windowed_matvec: workspace must be 256-byte aligned");
  cudaStream_t s = as_cuda(stream);
  if (n == 0) return LR_OK;
  if (source->n == 0) {
    LR_CHECK_CUDA(cudaMemsetAsync(out, 0, 4 * (size_t)n, s));
    return LR_OK;
  }
  char* ws = static_cast<char*>(workspace);
  float4* wcoef = reinterpret_cast<float4*>(ws + P.off_wcoef);
  float* wreach = reinterpret_cast<float*>(ws + P.off_wreach);
  if ((st = launch_window_prep(z, n, lengthscale, wcoef, wreach, s)) != LR_OK) return st;
  if (P.culled) {
    st = launch_cull_prep(P.C, reinterpret_cast<const float2*>(source->xy), 0.f, v, nullptr, 1, 0, ws, s);
    if (st != LR_OK) return st;
    CullArgs A{};
    A.x = reinterpret_cast<const float2*>(p);
    A.n = n;
    A.nrhs = 1;
    A.stride = 1;
    A.wcoef = wcoef;
    A.wreach = wreach;
    A.out = out;
    return launch_cull_sweep(P.C, A, ws, LR_KT_WINDOWED, s);
  }
  WnArgs A{};
  A.p = reinterpret_cast<const float2*>(p);
  A.wcoef = wcoef;
  A.n = n;
  A.g = grid_dev(source->grid);
  A.m = source->n;
  A.segs = P.segs;
  A.n_tiles = P.n_tiles;
  A.chunks = P.chunks;
  A.v = v;
  A.out = out;
  A.partial = reinterpret_cast<float*>(ws);
  const unsigned grid = (unsigned)((int64_t)P.row_blocks * P.chunks);
  ktimer_begin(LR_KT_WINDOWED, s);
  windowed_kernel<<<grid, kWnThreads, 0, s>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_WINDOWED, s);
  if (P.chunks > 1) {
    windowed_merge_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A.partial, P.chunks, n, out);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

extern "C" lr_status gp_windowed_matvec_nll(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                            const lr_points* source, const float* v, float lengthscale,
                                            const float* f_in, const float* data, float sigma, float* out, float* g,
                                            double* nll, void* workspace, size_t workspace_bytes, lr_stream stream) {
  WnPlan P;
  lr_status st = plan_windowed(n, layout, source, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(P.culled, "gp_windowed_matvec_nll: sources must be explicit points");
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "gp_windowed_matvec_nll: lengthscale must be > 0");
  LR_REQUIRE(isfinite(sigma) && sigma > 0.f, "gp_windowed_matvec_nll: sigma must be > 0");
  LR_REQUIRE(nll != nullptr && ((uintptr_t)nll & 7u) == 0, "gp_windowed_matvec_nll: nll is NULL or misaligned");
  LR_REQUIRE(n == 0 || (p && z && data && out && g), "gp_windowed_matvec_nll: NULL pointer");
  LR_REQUIRE(((uintptr_t)p & 7u) == 0 && ((uintptr_t)z & 3u) == 0, "gp_windowed_matvec_nll: misaligned p or z");
  LR_REQUIRE(v != nullptr || source->n == 0, "gp_windowed_matvec_nll: v is NULL");
  LR_REQUIRE(workspace_bytes >= P.bytes && (P.bytes == 0 || workspace != nullptr),
             "gp_windowed_matvec_nll: workspace of %zu bytes, %zu needed", workspace_bytes, P.bytes);
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0, "gp_windowed_matvec_nll: workspace must be 256-byte aligned");
  cudaStream_t s = as_cuda(stream);
  LR_CHECK_CUDA(cudaMemsetAsync(nll, 0, sizeof(double), s));
  if (n == 0) return LR_OK;
  char* ws = static_cast<char*>(workspace);
  float4* wcoef = reinterpret_cast<float4*>(ws + P.off_wcoef);
  float* wreach = reinterpret_cast<float*>(ws + P.off_wreach);
  if ((st = launch_window_prep(z, n, lengthscale, wcoef, wreach, s)) != LR_OK) return st;
  st = launch_cull_prep(P.C, reinterpret_cast<const float2*>(source->xy), 0.f, v, nullptr, 1, 0, ws, s);
  if (st != LR_OK) return st;
  CullArgs A{};
  A.x = reinterpret_cast<const float2*>(p);
  A.n = n;
  A.nrhs = 1;
  A.stride = 1;
  A.wcoef = wcoef;
  A.wreach = wreach;
  A.out = out;
  A.f_in = f_in;
  A.lik_data = data;
  A.lik_isig2 = (float)(1.0 / ((double)sigma * (double)sigma));
  A.lik_g = g;
  double* part = reinterpret_cast<double*>(ws + P.C.off_scal);
  A.scal_part = part;
  if ((st = launch_cull_sweep(P.C, A, ws, LR_KT_WINDOWED, s)) != LR_OK) return st;
  if ((st = launch_cull_scalar_final(part, P.C.scal_blocks, nll, nullptr, s)) != LR_OK) return st;
  // the constant terms: n ln sigma + (n / 2) ln 2 pi
  add_const_kernel<<<1, 32, 0, s>>>(nll, (double)n * (log((double)sigma) + 0.91893853320467274));
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
