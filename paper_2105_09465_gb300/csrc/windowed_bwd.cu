// Backward of the windowed transmission reduction (Sec. 3.4 transmission
// equation with the pixel windows of Sec. 3.2), recompute-only. For
// Loss = sum_i g_i out_i, out_i = sum_k G(p_i - q_k, C_i) v_k,
// C_i = Z_i + (l^2/2) I, with d = p_i - q_k, M = C_i^-1 and u = M d:
//   dG/dp_i = -G u,  dG/dq_k = G u,  dG/dC_i = G (u u^T - M) / 2,  dC_i/dl = l I.
// Two culled sweeps over the pairs (cull.cu, explicit sources):
//   rows:    per query row, sum_k v G [1, u, u u^T]     -> d_p, d_Z, d_l
//   columns: per source,    sum_i g G [1, u]            -> d_v, d_q
// Inside a sweep the exponent uses u' = M' d with M' = -(log2 e / 2) M, so
// that G = N 2^(d . u') and u = -2 ln2 u'; N = 1/(2 pi sqrt(det C)) is applied
// per row. The sweeps leave their sums per group range; the merges here add
// them in fixed order (Kahan) and form the gradients, the length-scale sum in
// FP64, so results are deterministic.
#include <math.h>

#include "cull.cuh"
#include "host.cuh"
#include "problems.cuh"

namespace lr {

constexpr float kTwoLn2 = 1.3862943611198906f;

__device__ __forceinline__ void wb_kahan(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// ---- merges
struct WbMergeArgs {
  const float* partial;
  int32_t chunks;
  int64_t n;
  const float4* wcoef;  // rows: window constants (a, b, c, N), k R = [[a, b], [0, c]], R^T R = C^-1
  const float* g;
  const float* v;  // columns: source weights
  float ell;
  float* d_a;      // rows: d_p [n][2]; columns: d_v [m]
  float* d_b;      // rows: d_z [n][3]; columns: d_q [m][2]
  double* scal;    // rows: per-block d_l partials
};

__device__ __forceinline__ float wb_merge(const float* partial, int chunks, int K, int k, int64_t n, int64_t i) {
  float s = 0.f, c = 0.f;
  for (int ch = 0; ch < chunks; ++ch) wb_kahan(s, c, partial[((int64_t)ch * K + k) * n + i]);
  return s - c;
}

__global__ void __launch_bounds__(256) wn_rows_merge_kernel(const __grid_constant__ WbMergeArgs M) {
  __shared__ double red[8];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double dl = 0.0;
  if (i < M.n) {
    float s[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = wb_merge(M.partial, M.chunks, 6, k, M.n, i);
    // C^-1 = R^T R = (2 ln 2) [[a^2, a b], [a b, b^2 + c^2]] (k^2 = 1 / (2 ln 2)):
    // products and a sum of squares, no cancellation
    const float4 wc = M.wcoef[i];
    const float ixx = kTwoLn2 * (wc.x * wc.x), ixy = kTwoLn2 * (wc.x * wc.y),
                iyy = kTwoLn2 * fmaf(wc.y, wc.y, wc.z * wc.z);
    const float gn = M.g[i] * wc.w;
    // d_p = g N (2 ln 2) P';  D = g N ((2 ln 2)^2 Q' - S C^-1) / 2
    if (M.d_a) {
      M.d_a[2 * i] = gn * kTwoLn2 * s[1];
      M.d_a[2 * i + 1] = gn * kTwoLn2 * s[2];
    }
    const float k2 = kTwoLn2 * kTwoLn2, h = 0.5f * gn;
    const float Dxx = h * fmaf(k2, s[3], -s[0] * ixx);
    const float Dxy = h * fmaf(k2, s[4], -s[0] * ixy);
    const float Dyy = h * fmaf(k2, s[5], -s[0] * iyy);
    if (M.d_b) {
      M.d_b[3 * i] = Dxx;
      M.d_b[3 * i + 1] = 2.0f * Dxy;
      M.d_b[3 * i + 2] = Dyy;
    }
    dl = (double)M.ell * ((double)Dxx + (double)Dyy);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dl;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    M.scal[blockIdx.x] = t;
  }
}

__global__ void wn_scalar_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 256) s += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *out = t;
  }
}

__global__ void wn_cols_merge_kernel(const __grid_constant__ WbMergeArgs M) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.n) return;
  const float T = wb_merge(M.partial, M.chunks, 3, 0, M.n, k);
  if (M.d_a) M.d_a[k] = T;
  if (M.d_b) {
    // d_q = v (2 ln 2) U with u' evaluated at q - p
    const float vk = kTwoLn2 * M.v[k];
    M.d_b[2 * k] = vk * wb_merge(M.partial, M.chunks, 3, 1, M.n, k);
    M.d_b[2 * k + 1] = vk * wb_merge(M.partial, M.chunks, 3, 2, M.n, k);
  }
}

// ---- pixel windows: dL/dp from dL/dZ (a gather over the neighbours whose
// window vectors include p_j)
__device__ __forceinline__ void window_vec_grad(const float2* __restrict__ p, const float* __restrict__ dz, int32_t W,
                                                int32_t H, int64_t i, float2& da, float2& db, float& sa, float& sb,
                                                int64_t& cl, int64_t& cr, int64_t& rd, int64_t& ru) {
  const int32_t r = (int32_t)(i / W), c = (int32_t)(i - (int64_t)r * W);
  cl = c > 0 ? i - 1 : i;
  cr = c + 1 < W ? i + 1 : i;
  rd = r > 0 ? i - W : i;
  ru = r + 1 < H ? i + W : i;
  sa = (cr - cl == 2) ? 0.5f : 1.0f;
  sb = (ru - rd == 2 * (int64_t)W) ? 0.5f : 1.0f;
  const float2 pl = p[cl], pr = p[cr], pd = p[rd], pu = p[ru];
  const float ax = sa * (pr.x - pl.x), ay = sa * (pr.y - pl.y);
  const float bx = sb * (pu.x - pd.x), by = sb * (pu.y - pd.y);
  const float k = 0.0795774715459477f;  // 1 / (4 pi)
  const float gxx = dz[3 * i], gxy = dz[3 * i + 1], gyy = dz[3 * i + 2];
  da = make_float2(k * fmaf(2.0f * gxx, ax, gxy * ay), k * fmaf(gxy, ax, 2.0f * gyy * ay));
  db = make_float2(k * fmaf(2.0f * gxx, bx, gxy * by), k * fmaf(gxy, bx, 2.0f * gyy * by));
}

__global__ void pixel_shapes_vjp_kernel(const float2* __restrict__ p, const float* __restrict__ dz, int32_t W,
                                        int32_t H, float2* __restrict__ dp) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int64_t)W * H) return;
  const int32_t r = (int32_t)(j / W), c = (int32_t)(j - (int64_t)r * W);
  float gx = 0.f, gy = 0.f;
  // every pixel i within one step of j along either axis may use p_j
  for (int di = -1; di <= 1; ++di)
    for (int dc = -1; dc <= 1; ++dc) {
      if ((di != 0) && (dc != 0)) continue;
      const int32_t rr = r + di, cc = c + dc;
      if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      const int64_t i = (int64_t)rr * W + cc;
      float2 da, db;
      float sa, sb;
      int64_t cl, cr, rd, ru;
      window_vec_grad(p, dz, W, H, i, da, db, sa, sb, cl, cr, rd, ru);
      if (cr == j) { gx = fmaf(sa, da.x, gx); gy = fmaf(sa, da.y, gy); }
      if (cl == j) { gx = fmaf(-sa, da.x, gx); gy = fmaf(-sa, da.y, gy); }
      if (ru == j) { gx = fmaf(sb, db.x, gx); gy = fmaf(sb, db.y, gy); }
      if (rd == j) { gx = fmaf(-sb, db.x, gx); gy = fmaf(-sb, db.y, gy); }
    }
  dp[j] = make_float2(gx, gy);
}

}  // namespace lr

namespace lr {

struct WbPlan {
  CullPlan R, C;    // row sweep (rows: the query points), column sweep (rows: the sources)
  int64_t merge_blocks;
  size_t off_rows, off_scal, off_cols, off_wcoef, off_wreach, bytes;
};

static lr_status plan_windowed_bwd(int64_t n, const lr_grid* layout, const lr_points* s, WbPlan* P) {
  lr_status st = validate_points(s, "gp_windowed_matvec_bwd(source)", false);
  if (st != LR_OK) return st;
  LR_REQUIRE(!has_lens(s) && s->xy != nullptr, "gp_windowed_matvec_bwd: sources must be explicit points");
  LR_REQUIRE(n >= 0 && n < (int64_t(1) << 31), "gp_windowed_matvec_bwd: n out of range");
  if (layout)
    LR_REQUIRE(layout->nx > 0 && layout->ny > 0 && layout->ss > 0 &&
                   (int64_t)layout->nx * layout->ss * layout->ny * layout->ss == n,
               "gp_windowed_matvec_bwd: the layout does not hold the %lld query points", (long long)n);
  const int64_t m = s->n;
  const lr_grid* sl = query_layout(s);
  WbPlan p{};
  if ((st = plan_cull(kCullWinRows, 1, n, layout, m, sl, &p.R)) != LR_OK) return st;
  if ((st = plan_cull(kCullWinCols, 1, m, sl, n, layout, &p.C)) != LR_OK) return st;
  p.merge_blocks = (n + 255) / 256;
  size_t o = 0;
  p.off_rows = o;
  o += align256(p.R.bytes);
  p.off_scal = o;
  o += align256(sizeof(double) * (size_t)(p.merge_blocks + 1));
  p.off_cols = o;
  o += align256(p.C.bytes);
  p.off_wcoef = o;
  o += align256(16 * (size_t)n);
  p.off_wreach = o;
  o += align256(4 * (size_t)n);
  p.bytes = o;
  *P = p;
  return LR_OK;
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_windowed_bwd_workspace_size(int64_t n, const lr_grid* layout, const lr_points* source,
                                                    size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_windowed_bwd_workspace_size: bytes is NULL");
  WbPlan P;
  lr_status st = plan_windowed_bwd(n, layout, source, &P);
  if (st != LR_OK) return st;
  *bytes = P.bytes;
  return LR_OK;
}

extern "C" lr_status gp_windowed_matvec_bwd(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                            const lr_points* source, const float* v, float lengthscale,
                                            const float* g, float* d_v, float* d_p, float* d_q, float* d_z,
                                            double* d_lengthscale, void* workspace, size_t workspace_bytes,
                                            lr_stream stream) {
  WbPlan P;
  lr_status st = plan_windowed_bwd(n, layout, source, &P);
  if (st != LR_OK) return st;
  const int64_t m = source->n;
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "gp_windowed_matvec_bwd: lengthscale must be > 0");
  LR_REQUIRE(n == 0 || (p && z && g), "gp_windowed_matvec_bwd: NULL p, z or g");
  LR_REQUIRE(m == 0 || v, "gp_windowed_matvec_bwd: v is NULL");
  LR_REQUIRE(((uintptr_t)p & 7u) == 0 && ((uintptr_t)d_p & 7u) == 0 && ((uintptr_t)d_q & 7u) == 0 &&
                 ((uintptr_t)d_lengthscale & 7u) == 0,
             "gp_windowed_matvec_bwd: misaligned pointer");
  LR_REQUIRE(workspace_bytes >= P.bytes && workspace != nullptr && ((uintptr_t)workspace & 255u) == 0,
             "gp_windowed_matvec_bwd: workspace of %zu bytes (256-byte aligned) needed", P.bytes);
  cudaStream_t s = as_cuda(stream);
  char* ws = static_cast<char*>(workspace);
  if (n == 0 || m == 0) {
    if (d_v && m) LR_CHECK_CUDA(cudaMemsetAsync(d_v, 0, 4 * (size_t)m, s));
    if (d_q && m) LR_CHECK_CUDA(cudaMemsetAsync(d_q, 0, 8 * (size_t)m, s));
    if (d_p && n) LR_CHECK_CUDA(cudaMemsetAsync(d_p, 0, 8 * (size_t)n, s));
    if (d_z && n) LR_CHECK_CUDA(cudaMemsetAsync(d_z, 0, 12 * (size_t)n, s));
    if (d_lengthscale) LR_CHECK_CUDA(cudaMemsetAsync(d_lengthscale, 0, 8, s));
    return LR_OK;
  }
  const float2* pp = reinterpret_cast<const float2*>(p);
  const float2* qq = reinterpret_cast<const float2*>(source->xy);
  float4* wcoef = reinterpret_cast<float4*>(ws + P.off_wcoef);
  float* wreach = reinterpret_cast<float*>(ws + P.off_wreach);
  if ((st = launch_window_prep(z, n, lengthscale, wcoef, wreach, s)) != LR_OK) return st;
  if (d_p || d_z || d_lengthscale) {
    char* wr = ws + P.off_rows;
    if ((st = launch_cull_prep(P.R, qq, 0.f, v, nullptr, 1, 0, wr, s)) != LR_OK) return st;
    CullArgs A{};
    A.x = pp;
    A.n = n;
    A.nrhs = 1;
    A.stride = 1;
    A.wcoef = wcoef;
    A.wreach = wreach;
    if ((st = launch_cull_sweep(P.R, A, wr, -1, s)) != LR_OK) return st;
    WbMergeArgs M{};
    M.partial = reinterpret_cast<const float*>(wr + P.R.off_partial);
    M.chunks = P.R.splits;
    M.n = n;
    M.wcoef = wcoef;
    M.g = g;
    M.ell = lengthscale;
    M.d_a = d_p;
    M.d_b = d_z;
    M.scal = reinterpret_cast<double*>(ws + P.off_scal);
    wn_rows_merge_kernel<<<(unsigned)P.merge_blocks, 256, 0, s>>>(M);
    LR_CHECK_CUDA(cudaGetLastError());
    if (d_lengthscale) {
      wn_scalar_final_kernel<<<1, 256, 0, s>>>(M.scal, (int)P.merge_blocks, d_lengthscale);
      LR_CHECK_CUDA(cudaGetLastError());
    }
  }
  if (d_v || d_q) {
    char* wc = ws + P.off_cols;
    if ((st = launch_cull_prep(P.C, pp, 0.f, g, nullptr, 1, 0, wc, s, wcoef, wreach)) != LR_OK) return st;
    CullArgs A{};
    A.x = qq;
    A.n = m;
    A.nrhs = 1;
    A.stride = 1;
    if ((st = launch_cull_sweep(P.C, A, wc, -1, s)) != LR_OK) return st;
    WbMergeArgs M{};
    M.partial = reinterpret_cast<const float*>(wc + P.C.off_partial);
    M.chunks = P.C.splits;
    M.n = m;
    M.v = v;
    M.d_a = d_v;
    M.d_b = d_q;
    wn_cols_merge_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(M);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

extern "C" lr_status lr_windowed_pairs_evaluated(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                                 const lr_points* source, float lengthscale, int32_t sweep,
                                                 int64_t* pairs, int64_t* slots, lr_stream stream) {
  WbPlan P;
  lr_status st = plan_windowed_bwd(n, layout, source, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(pairs != nullptr, "lr_windowed_pairs_evaluated: pairs is NULL");
  LR_REQUIRE(sweep >= 0 && sweep <= 2, "lr_windowed_pairs_evaluated: sweep = %d (0, 1 or 2)", sweep);
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "lr_windowed_pairs_evaluated: lengthscale must be > 0");
  LR_REQUIRE(n == 0 || (p && z), "lr_windowed_pairs_evaluated: NULL p or z");
  LR_REQUIRE(((uintptr_t)p & 7u) == 0 && ((uintptr_t)z & 3u) == 0, "lr_windowed_pairs_evaluated: misaligned p or z");
  const int64_t m = source->n;
  *pairs = 0;
  if (slots) *slots = 0;
  if (n == 0 || m == 0) return LR_OK;
  cudaStream_t s = as_cuda(stream);
  CullPlan C;
  if (sweep == 2) {
    C = P.C;
  } else {
    const int kind = sweep == 0 ? kCullWin : kCullWinRows;
    if ((st = plan_cull(kind, 1, n, layout, m, query_layout(source), &C)) != LR_OK) return st;
  }
  // temporaries: zero weights, window constants, the sweep's workspace, the counters
  const size_t b_w = align256(4 * (size_t)(n > m ? n : m)), b_c = align256(16 * (size_t)n),
               b_r = align256(4 * (size_t)n);
  char* buf = nullptr;
  LR_CHECK_CUDA(cudaMalloc(&buf, b_w + b_c + b_r + C.bytes + 256));
  auto done = [&](lr_status r) {
    cudaFree(buf);
    return r;
  };
  float* w = reinterpret_cast<float*>(buf);
  float4* wcoef = reinterpret_cast<float4*>(buf + b_w);
  float* wreach = reinterpret_cast<float*>(buf + b_w + b_c);
  char* ws = buf + b_w + b_c + b_r;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ws + C.bytes);
  if (cudaMemsetAsync(w, 0, b_w, s) != cudaSuccess || cudaMemsetAsync(cnt, 0, 16, s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "cudaMemsetAsync"));
  if ((st = launch_window_prep(z, n, lengthscale, wcoef, wreach, s)) != LR_OK) return done(st);
  const float2* pp = reinterpret_cast<const float2*>(p);
  const float2* qq = reinterpret_cast<const float2*>(source->xy);
  CullArgs A{};
  A.nrhs = 1;
  A.stride = 1;
  A.count = cnt;
  if (sweep == 2) {
    st = launch_cull_prep(C, pp, 0.f, w, nullptr, 1, 0, ws, s, wcoef, wreach);
    A.x = qq;
    A.n = m;
  } else {
    st = launch_cull_prep(C, qq, 0.f, w, nullptr, 1, 0, ws, s);
    A.x = pp;
    A.n = n;
    A.wcoef = wcoef;
    A.wreach = wreach;
  }
  if (st != LR_OK) return done(st);
  if ((st = launch_cull_sweep(C, A, ws, -1, s)) != LR_OK) return done(st);
  unsigned long long h[2] = {0, 0};
  if (cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "lr_windowed_pairs_evaluated"));
  *pairs = (int64_t)h[0];
  if (slots) *slots = (int64_t)h[1];
  return done(LR_OK);
}

extern "C" lr_status gp_pixel_shapes_vjp(const float* p, int32_t W, int32_t H, const float* dz, float* dp,
                                         lr_stream stream) {
  LR_REQUIRE(W >= 1 && H >= 1 && (int64_t)W * H < (int64_t(1) << 31), "gp_pixel_shapes_vjp: bad grid %d x %d", W, H);
  LR_REQUIRE(p && dz && dp, "gp_pixel_shapes_vjp: NULL pointer");
  LR_REQUIRE(((uintptr_t)p & 7u) == 0 && ((uintptr_t)dp & 7u) == 0 && ((uintptr_t)dz & 3u) == 0,
             "gp_pixel_shapes_vjp: misaligned pointer");
  const int64_t n = (int64_t)W * H;
  pixel_shapes_vjp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, as_cuda(stream)>>>(
      reinterpret_cast<const float2*>(p), dz, W, H, reinterpret_cast<float2*>(dp));
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
