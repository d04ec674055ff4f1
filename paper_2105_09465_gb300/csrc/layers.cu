// Multi-layer kernel reduction (Sec. 3.1, the sum of RBF layers):
//   out_i = sum_l var_l sum_j exp(-|x_i - y_j|^2 / (2 l_l^2)) v_{l,j}
// over ONE set of query and source points (the paper's image-plane GP uses
// several layers on the same ray-traced points). The squared distance of a
// pair is formed once and shared by the layers; each layer costs one scale
// (a packed multiply), one exp2 per pair and one accumulation. Same tiling,
// chunking and fixed-order merging as the single-layer reduction.
#include <math.h>

#include "host.cuh"
#include "problems.cuh"

namespace lr {

constexpr int kLyMax = 4;
constexpr int kLyMaxRhs = 4;
constexpr int kLyThreads = 128;
constexpr int kLyTile = 256;
constexpr int kLyPairs = kLyTile / 2;
static_assert(kLyPairs == kLyThreads, "one source pair per thread when staging");

// Query rows per thread: 4, or 2 with more than two right-hand sides.
__host__ __device__ constexpr int ly_rows_per_thread(int nrhs) { return nrhs <= 2 ? 4 : 2; }

struct LyArgs {
  const float2* x;
  int64_t n;
  const float2* y;  // explicit sources, or NULL for the grid
  GridDev g;
  int64_t m;
  int32_t segs, n_tiles, chunks, L, nrhs;
  const float* v;          // [L][m][nrhs]
  float neg_c0;            // -log2(e)/(2 l_0^2)
  float ratio[kLyMax];     // (l_0 / l_l)^2
  float var[kLyMax];
  float* out;              // [n][nrhs] when chunks == 1
  float* partial;          // [chunks][n][nrhs]
};

__device__ __forceinline__ float2 lf2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void ly_tile(const LyArgs& A, int t, int64_t& j0, int& cnt, int& grow) {
  if (A.y) {
    j0 = (int64_t)t * kLyTile;
    const int64_t rem = A.m - j0;
    cnt = rem < kLyTile ? (int)rem : kLyTile;
    grow = 0;
  } else {
    grow = t / A.segs;
    const int c0 = (t - grow * A.segs) * kLyTile;
    cnt = min(kLyTile, A.g.W - c0);
    j0 = (int64_t)grow * A.g.W + c0;
  }
}

// Pair p of tile t: negated coordinates and, per layer and right-hand side,
// the weights scaled by the layer's variance.
template <int L, int H>
__device__ __forceinline__ void ly_load(const LyArgs& A, int t, int p, float4& P, float2 (&V)[L][H]) {
  int64_t j0;
  int cnt, grow;
  ly_tile(A, t, j0, cnt, grow);
  const int a = 2 * p, b = 2 * p + 1;
  float2 pa, pb;
  if (A.y) {
    pa = (a < cnt) ? __ldg(A.y + j0 + a) : lf2(0.f, 0.f);
    pb = (b < cnt) ? __ldg(A.y + j0 + b) : lf2(0.f, 0.f);
  } else {
    const int c0 = (int)(j0 - (int64_t)grow * A.g.W);
    const float yy = grid_y(A.g, grow);
    pa = lf2((a < cnt) ? grid_x(A.g, c0 + a) : 0.f, yy);
    pb = lf2((b < cnt) ? grid_x(A.g, c0 + b) : 0.f, yy);
  }
  P = make_float4(-pa.x, -pb.x, -pa.y, -pb.y);
#pragma unroll
  for (int l = 0; l < L; ++l)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float* vl = A.v + ((int64_t)l * A.m + j0) * H + h;
      V[l][h] = lf2((a < cnt) ? A.var[l] * __ldg(vl + (int64_t)a * H) : 0.f,
                    (b < cnt) ? A.var[l] * __ldg(vl + (int64_t)b * H) : 0.f);
    }
}

template <int L, int H>
__global__ void __launch_bounds__(kLyThreads) layers_kernel(const __grid_constant__ LyArgs A) {
  constexpr int R = ly_rows_per_thread(H), ROWS = kLyThreads * R;
  __shared__ __align__(16) float4 sP[2][kLyPairs];
  __shared__ __align__(16) float2 sV[2][L][H][kLyPairs];
  __shared__ float ksum[R][H][kLyThreads], kcomp[R][H][kLyThreads];
  const int rb = blockIdx.x / A.chunks;
  const int chunk = blockIdx.x - rb * A.chunks;
  const int t0 = (int)((int64_t)chunk * A.n_tiles / A.chunks);
  const int t1 = (int)((int64_t)(chunk + 1) * A.n_tiles / A.chunks);
  const int tid = threadIdx.x;

  float2 xq[R], yq[R], acc[R][H];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int64_t i = (int64_t)rb * ROWS + r * kLyThreads + tid;
    if (i >= A.n) i = A.n - 1;
    const float2 p = __ldg(A.x + i);
    xq[r] = lf2(p.x, p.x);
    yq[r] = lf2(p.y, p.y);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      acc[r][h] = lf2(0.f, 0.f);
      ksum[r][h][tid] = 0.f;
      kcomp[r][h][tid] = 0.f;
    }
  }
  const float2 nc = lf2(A.neg_c0, A.neg_c0);
  float4 P;
  float2 V[L][H];
  if (t0 < t1) {
    ly_load<L, H>(A, t0, tid, P, V);
    sP[0][tid] = P;
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int h = 0; h < H; ++h) sV[0][l][h][tid] = V[l][h];
  }
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    if (t + 1 < t1) ly_load<L, H>(A, t + 1, tid, P, V);
    int64_t j0;
    int cnt, grow;
    ly_tile(A, t, j0, cnt, grow);
    const int np = (cnt + 1) >> 1;
#pragma unroll 2
    for (int p = 0; p < np; ++p) {
      const float4 Q = sP[buf][p];
      float2 W[L][H];
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int h = 0; h < H; ++h) W[l][h] = sV[buf][l][h][p];
      const float2 nx = lf2(Q.x, Q.y), ny = lf2(Q.z, Q.w);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 dx = __fadd2_rn(xq[r], nx);
        const float2 dy = __fadd2_rn(yq[r], ny);
        const float2 e0 = __fmul2_rn(__ffma2_rn(dy, dy, __fmul2_rn(dx, dx)), nc);  // layer-0 exponent
#pragma unroll
        for (int l = 0; l < L; ++l) {
          // one exp2 per pair and layer, shared by the right-hand sides
          const float2 e = (l == 0) ? e0 : __fmul2_rn(e0, lf2(A.ratio[l], A.ratio[l]));
          const float2 k = lf2(ex2_approx(e.x), ex2_approx(e.y));
#pragma unroll
          for (int h = 0; h < H; ++h) acc[r][h] = __ffma2_rn(k, W[l][h], acc[r][h]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const float y = (acc[r][h].x + acc[r][h].y) - kcomp[r][h][tid];
        const float s = ksum[r][h][tid] + y;
        kcomp[r][h][tid] = (s - ksum[r][h][tid]) - y;
        ksum[r][h][tid] = s;
        acc[r][h] = lf2(0.f, 0.f);
      }
    if (t + 1 < t1) {
      sP[buf ^ 1][tid] = P;
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int h = 0; h < H; ++h) sV[buf ^ 1][l][h][tid] = V[l][h];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = (int64_t)rb * ROWS + r * kLyThreads + tid;
    if (i < A.n)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const float total = ksum[r][h][tid] - kcomp[r][h][tid];
        if (A.chunks == 1)
          A.out[i * H + h] = total;
        else
          A.partial[((int64_t)chunk * A.n + i) * H + h] = total;
      }
  }
}

// Fixed-order (Kahan) merge of the chunk partials [chunks][n * nrhs].
__global__ void layers_merge_kernel(const float* __restrict__ partial, int chunks, int64_t count,
                                    float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.f, c = 0.f;
  for (int k = 0; k < chunks; ++k) {
    const float y = partial[(int64_t)k * count + i] - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  out[i] = s - c;
}

struct LyPlan {
  int64_t n, m;
  bool q_raytrace, q_grid, self, s_grid;
  int32_t n_tiles, segs, chunks, row_blocks, nrhs;
  size_t off_q, off_partial, bytes;
};

static const void* layers_kernel_ptr(int nrhs) {
  switch (nrhs) {
    case 1: return reinterpret_cast<const void*>(&layers_kernel<kLyMax, 1>);
    case 2: return reinterpret_cast<const void*>(&layers_kernel<kLyMax, 2>);
    case 3: return reinterpret_cast<const void*>(&layers_kernel<kLyMax, 3>);
    default: return reinterpret_cast<const void*>(&layers_kernel<kLyMax, 4>);
  }
}

static lr_status plan_layers(const lr_points* q, const lr_points* s, int32_t L, int32_t nrhs, bool have_beta_out,
                             LyPlan* P) {
  lr_status st = validate_points(q, "gp_kernel_matvec_layers(query)", false);
  if (st != LR_OK) return st;
  if (s) {
    if ((st = validate_points(s, "gp_kernel_matvec_layers(source)", false)) != LR_OK) return st;
    LR_REQUIRE(!has_lens(s), "gp_kernel_matvec_layers: sources must not be ray-traced (use a self-kernel)");
  }
  LR_REQUIRE(L >= 1 && L <= kLyMax, "gp_kernel_matvec_layers: n_layers = %d outside [1, %d]", L, kLyMax);
  LR_REQUIRE(nrhs >= 1 && nrhs <= kLyMaxRhs, "gp_kernel_matvec_layers: nrhs = %d outside [1, %d]", nrhs, kLyMaxRhs);
  LyPlan p{};
  p.n = q->n;
  p.self = s == nullptr;
  p.m = p.self ? q->n : s->n;
  p.q_raytrace = has_lens(q);
  p.q_grid = !p.q_raytrace && q->xy == nullptr;
  p.s_grid = !p.self && s->xy == nullptr;
  if (p.s_grid) {
    const int W = s->grid.nx * s->grid.ss;
    p.segs = (W + kLyTile - 1) / kLyTile;
    p.n_tiles = (int32_t)((int64_t)p.segs * s->grid.ny * s->grid.ss);
  } else {
    p.n_tiles = (int32_t)((p.m + kLyTile - 1) / kLyTile);
  }
  const int64_t rows = (int64_t)kLyThreads * ly_rows_per_thread(nrhs);
  p.nrhs = nrhs;
  p.row_blocks = (int32_t)((p.n + rows - 1) / rows);
  int dev = 0, n_sm = 1, occ = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, layers_kernel_ptr(nrhs), kLyThreads, 0));
  p.chunks = plan_chunks(p.row_blocks, p.n_tiles, occ, n_sm);
  size_t off = 0;
  p.off_q = off;
  if ((p.q_raytrace || p.q_grid) && !have_beta_out) off += align256(8 * (size_t)p.n);
  p.off_partial = off;
  if (p.chunks > 1) off += align256(4 * (size_t)p.chunks * (size_t)p.n * (size_t)nrhs);
  p.bytes = off;
  *P = p;
  return LR_OK;
}

template <int L>
static void launch_layers(const LyArgs& A, unsigned grid, cudaStream_t s) {
  switch (A.nrhs) {
    case 1: layers_kernel<L, 1><<<grid, kLyThreads, 0, s>>>(A); break;
    case 2: layers_kernel<L, 2><<<grid, kLyThreads, 0, s>>>(A); break;
    case 3: layers_kernel<L, 3><<<grid, kLyThreads, 0, s>>>(A); break;
    default: layers_kernel<L, 4><<<grid, kLyThreads, 0, s>>>(A); break;
  }
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_matvec_layers_workspace_size(const lr_points* query, const lr_points* source, int32_t n_layers,
                                                     int32_t nrhs, size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_matvec_layers_workspace_size: bytes is NULL");
  LyPlan P;
  lr_status st = plan_layers(query, source, n_layers, nrhs, false, &P);
  if (st != LR_OK) return st;
  *bytes = P.bytes;
  return LR_OK;
}

extern "C" lr_status gp_kernel_matvec_layers(const lr_points* query, const lr_points* source, int32_t n_layers,
                                             const float* lengthscales, const float* variances, const float* v,
                                             int32_t nrhs, float* out, float* beta_out, void* workspace,
                                             size_t workspace_bytes, lr_stream stream) {
  LyPlan P;
  lr_status st = plan_layers(query, source, n_layers, nrhs, beta_out != nullptr, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(lengthscales != nullptr && variances != nullptr, "gp_kernel_matvec_layers: NULL hyperparameters");
  for (int l = 0; l < n_layers; ++l) {
    LR_REQUIRE(isfinite(lengthscales[l]) && lengthscales[l] > 0.f, "gp_kernel_matvec_layers: lengthscale %d <= 0", l);
    LR_REQUIRE(isfinite(variances[l]), "gp_kernel_matvec_layers: variance %d not finite", l);
  }
  LR_REQUIRE(out != nullptr || P.n == 0, "gp_kernel_matvec_layers: out is NULL");
  LR_REQUIRE(v != nullptr || P.m == 0, "gp_kernel_matvec_layers: v is NULL");
  LR_REQUIRE(workspace_bytes >= P.bytes, "gp_kernel_matvec_layers: workspace of %zu bytes, %zu needed",
             workspace_bytes, P.bytes);
  LR_REQUIRE(P.bytes == 0 || workspace != nullptr, "gp_kernel_matvec_layers: workspace is NULL");
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0 && ((uintptr_t)beta_out & 7u) == 0,
             "gp_kernel_matvec_layers: misaligned workspace or beta_out");
  cudaStream_t s = as_cuda(stream);
  if (P.n == 0) return LR_OK;
  if (P.m == 0) {
    LR_CHECK_CUDA(cudaMemsetAsync(out, 0, 4 * (size_t)P.n * (size_t)nrhs, s));
    return LR_OK;
  }
  char* ws = static_cast<char*>(workspace);
  const float2* xq = reinterpret_cast<const float2*>(query->xy);
  if (P.q_raytrace || P.q_grid) {
    float2* qb = beta_out ? reinterpret_cast<float2*>(beta_out) : reinterpret_cast<float2*>(ws + P.off_q);
    st = P.q_raytrace ? launch_raytrace(query, qb, nullptr, s) : launch_grid_points(query->grid, qb, s);
    if (st != LR_OK) return st;
    xq = qb;
  }
  LyArgs A{};
  A.x = xq;
  A.n = P.n;
  A.y = P.self ? xq : (P.s_grid ? nullptr : reinterpret_cast<const float2*>(source->xy));
  A.g = P.s_grid ? grid_dev(source->grid) : GridDev{};
  A.m = P.m;
  A.segs = P.segs;
  A.n_tiles = P.n_tiles;
  A.chunks = P.chunks;
  A.L = n_layers;
  A.nrhs = nrhs;
  A.v = v;
  const double l0 = lengthscales[0];
  A.neg_c0 = (float)(-1.4426950408889634 / (2.0 * l0 * l0));
  for (int l = 0; l < kLyMax; ++l) {
    const double ll = l < n_layers ? (double)lengthscales[l] : l0;
    A.ratio[l] = (float)((l0 * l0) / (ll * ll));
    A.var[l] = l < n_layers ? variances[l] : 0.f;
  }
  A.out = out;
  A.partial = reinterpret_cast<float*>(ws + P.off_partial);
  const unsigned grid = (unsigned)((int64_t)P.row_blocks * P.chunks);
  switch (n_layers) {
    case 1: launch_layers<1>(A, grid, s); break;
    case 2: launch_layers<2>(A, grid, s); break;
    case 3: launch_layers<3>(A, grid, s); break;
    default: launch_layers<4>(A, grid, s); break;
  }
  LR_CHECK_CUDA(cudaGetLastError());
  if (P.chunks > 1) {
    const int64_t count = P.n * nrhs;
    layers_merge_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(A.partial, P.chunks, count, out);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}
