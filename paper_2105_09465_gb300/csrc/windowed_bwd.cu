// Backward of the windowed transmission reduction (Sec. 3.4 transmission
// equation with the pixel windows of Sec. 3.2), recompute-only. For
// Loss = sum_i g_i out_i, out_i = sum_k G(p_i - q_k, C_i) v_k,
// C_i = Z_i + (l^2/2) I, with d = p_i - q_k, M = C_i^-1 and u = M d:
//   dG/dp_i = -G u,  dG/dq_k = G u,  dG/dC_i = G (u u^T - M) / 2,  dC_i/dl = l I.
// Two sweeps over the pairs (explicit sources):
//   rows:    per query row, sum_k v G [1, u, u u^T]     -> d_p, d_Z, d_l
//   columns: per source,    sum_i g G [1, u]            -> d_v, d_q
// Inside a sweep the exponent uses u' = M' d with M' = -(log2 e / 2) M, so
// that G = N 2^(d . u') and u = -2 ln2 u'; N = 1/(2 pi sqrt(det C)) is applied
// per row. Chunk partials are merged in fixed order (Kahan), the length-scale
// sum in FP64, so results are deterministic.
#include <math.h>

#include "host.cuh"
#include "problems.cuh"

namespace lr {

constexpr int kWbThreads = 128;
constexpr int kWbR = 4;
constexpr int kWbRows = kWbThreads * kWbR;
constexpr int kWbTile = 256;
constexpr int kWbPairs = kWbTile / 2;
static_assert(kWbPairs == kWbThreads, "one pair of staged points per thread");
constexpr float kTwoLn2 = 1.3862943611198906f;

__device__ __forceinline__ float2 bf2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void wb_kahan(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Per-row window constants: M' = -(log2 e / 2) C^-1 (xx, xy, yy) and N.
__device__ __forceinline__ void window_consts(const float* __restrict__ z, int64_t i, float half_s, float& mxx,
                                              float& mxy, float& myy, float& norm) {
  const float cxx = __ldg(z + 3 * i) + half_s, cxy = __ldg(z + 3 * i + 1), cyy = __ldg(z + 3 * i + 2) + half_s;
  const float det = fmaf(cxx, cyy, -cxy * cxy);
  const float s = -0.72134752044448170f / det;  // -log2(e) / (2 det)
  mxx = s * cyy;
  mxy = -s * cxy;
  myy = s * cxx;
  norm = 0.15915494309189535f * rsqrtf(det);  // 1 / (2 pi sqrt(det))
}

struct WbArgs {
  const float2* p;   // query points [n]
  const float* z;    // windows [n][3]
  const float* g;    // dL/dout [n]
  int64_t n;
  const float2* q;   // sources [m]
  const float* v;    // [m]
  int64_t m;
  float half_s;      // l^2 / 2
  int32_t chunks, n_tiles;
  float* partial;    // rows: [chunks][6][n]; columns: [chunks][3][m]
};

// ---- rows: S = sum v G', P = sum v G' u', Q = sum v G' u' u'^T (G' = 2^(d.u'))
struct WbRowSmem {
  float4 sQ[2][kWbPairs];  // (-qa.x, -qb.x, -qa.y, -qb.y)
  float2 sV[2][kWbPairs];
  float ksum[6][kWbR][kWbThreads], kcomp[6][kWbR][kWbThreads];
};

__global__ void __launch_bounds__(kWbThreads) wn_rows_kernel(const __grid_constant__ WbArgs A) {
  __shared__ __align__(16) WbRowSmem sm;
  const int rb = blockIdx.x / A.chunks, chunk = blockIdx.x - rb * A.chunks;
  const int t0 = (int)((int64_t)chunk * A.n_tiles / A.chunks);
  const int t1 = (int)((int64_t)(chunk + 1) * A.n_tiles / A.chunks);
  const int tid = threadIdx.x;
  float2 xq[kWbR], yq[kWbR], mxx[kWbR], mxy[kWbR], myy[kWbR];
#pragma unroll
  for (int r = 0; r < kWbR; ++r) {
    int64_t i = (int64_t)rb * kWbRows + r * kWbThreads + tid;
    if (i >= A.n) i = A.n - 1;
    const float2 pp = __ldg(A.p + i);
    float a, b, c, nrm;
    window_consts(A.z, i, A.half_s, a, b, c, nrm);
    xq[r] = bf2(pp.x, pp.x);
    yq[r] = bf2(pp.y, pp.y);
    mxx[r] = bf2(a, a);
    mxy[r] = bf2(b, b);
    myy[r] = bf2(c, c);
#pragma unroll
    for (int k = 0; k < 6; ++k) sm.ksum[k][r][tid] = sm.kcomp[k][r][tid] = 0.f;
  }
  auto load = [&](int t, float4& Q, float2& V) {
    const int64_t j0 = (int64_t)t * kWbTile;
    const int a = 2 * tid, b = a + 1;
    const bool ia = j0 + a < A.m, ib = j0 + b < A.m;
    const float2 qa = ia ? __ldg(A.q + j0 + a) : bf2(0.f, 0.f), qb = ib ? __ldg(A.q + j0 + b) : bf2(0.f, 0.f);
    Q = make_float4(-qa.x, -qb.x, -qa.y, -qb.y);
    V = bf2(ia ? __ldg(A.v + j0 + a) : 0.f, ib ? __ldg(A.v + j0 + b) : 0.f);
  };
  float4 Q;
  float2 V;
  if (t0 < t1) {
    load(t0, Q, V);
    sm.sQ[0][tid] = Q;
    sm.sV[0][tid] = V;
  }
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    if (t + 1 < t1) load(t + 1, Q, V);
    const int64_t rem = A.m - (int64_t)t * kWbTile;
    const int np = ((rem < kWbTile ? (int)rem : kWbTile) + 1) >> 1;
    float2 acc[kWbR][6];
#pragma unroll
    for (int r = 0; r < kWbR; ++r)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[r][k] = bf2(0.f, 0.f);
#pragma unroll 2
    for (int pidx = 0; pidx < np; ++pidx) {
      const float4 S = sm.sQ[buf][pidx];
      const float2 W = sm.sV[buf][pidx];
      const float2 nx = bf2(S.x, S.y), ny = bf2(S.z, S.w);
#pragma unroll
      for (int r = 0; r < kWbR; ++r) {
        const float2 dx = __fadd2_rn(xq[r], nx), dy = __fadd2_rn(yq[r], ny);
        const float2 ux = __ffma2_rn(mxx[r], dx, __fmul2_rn(mxy[r], dy));
        const float2 uy = __ffma2_rn(mxy[r], dx, __fmul2_rn(myy[r], dy));
        const float2 e = __ffma2_rn(dx, ux, __fmul2_rn(dy, uy));
        const float2 kv = __fmul2_rn(bf2(ex2_approx(e.x), ex2_approx(e.y)), W);
        const float2 kx = __fmul2_rn(kv, ux), ky = __fmul2_rn(kv, uy);
        acc[r][0] = __fadd2_rn(acc[r][0], kv);
        acc[r][1] = __fadd2_rn(acc[r][1], kx);
        acc[r][2] = __fadd2_rn(acc[r][2], ky);
        acc[r][3] = __ffma2_rn(kx, ux, acc[r][3]);
        acc[r][4] = __ffma2_rn(kx, uy, acc[r][4]);
        acc[r][5] = __ffma2_rn(ky, uy, acc[r][5]);
      }
    }
#pragma unroll
    for (int r = 0; r < kWbR; ++r)
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float su = sm.ksum[k][r][tid], co = sm.kcomp[k][r][tid];
        wb_kahan(su, co, acc[r][k].x + acc[r][k].y);
        sm.ksum[k][r][tid] = su;
        sm.kcomp[k][r][tid] = co;
      }
    if (t + 1 < t1) {
      sm.sQ[buf ^ 1][tid] = Q;
      sm.sV[buf ^ 1][tid] = V;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kWbR; ++r) {
    const int64_t i = (int64_t)rb * kWbRows + r * kWbThreads + tid;
    if (i < A.n)
#pragma unroll
      for (int k = 0; k < 6; ++k)
        A.partial[((int64_t)chunk * 6 + k) * A.n + i] = sm.ksum[k][r][tid] - sm.kcomp[k][r][tid];
  }
}

// ---- columns: T = sum_i g N G', U = sum_i g N G' u'  (u' evaluated with d = q - p)
struct WbColSmem {
  float4 sA[2][kWbPairs];  // (-pa.x, -pb.x, -pa.y, -pb.y)
  float4 sB[2][kWbPairs];  // (mxx_a, mxx_b, mxy_a, mxy_b)
  float4 sC[2][kWbPairs];  // (myy_a, myy_b, gN_a, gN_b)
  float ksum[3][kWbR][kWbThreads], kcomp[3][kWbR][kWbThreads];
};

__global__ void __launch_bounds__(kWbThreads) wn_cols_kernel(const __grid_constant__ WbArgs A) {
  __shared__ __align__(16) WbColSmem sm;
  const int rb = blockIdx.x / A.chunks, chunk = blockIdx.x - rb * A.chunks;
  const int t0 = (int)((int64_t)chunk * A.n_tiles / A.chunks);
  const int t1 = (int)((int64_t)(chunk + 1) * A.n_tiles / A.chunks);
  const int tid = threadIdx.x;
  float2 xs[kWbR], ys[kWbR];
#pragma unroll
  for (int r = 0; r < kWbR; ++r) {
    int64_t k = (int64_t)rb * kWbRows + r * kWbThreads + tid;
    if (k >= A.m) k = A.m - 1;
    const float2 qq = __ldg(A.q + k);
    xs[r] = bf2(qq.x, qq.x);
    ys[r] = bf2(qq.y, qq.y);
#pragma unroll
    for (int c = 0; c < 3; ++c) sm.ksum[c][r][tid] = sm.kcomp[c][r][tid] = 0.f;
  }
  auto load = [&](int t, float4& P1, float4& P2, float4& P3) {
    const int64_t j0 = (int64_t)t * kWbTile;
    const int a = 2 * tid, b = a + 1;
    float pa[2] = {0.f, 0.f}, pb[2] = {0.f, 0.f}, ma[4] = {0.f, 0.f, 0.f, 0.f}, mb[4] = {0.f, 0.f, 0.f, 0.f};
    if (j0 + a < A.n) {
      const float2 pp = __ldg(A.p + j0 + a);
      pa[0] = pp.x;
      pa[1] = pp.y;
      window_consts(A.z, j0 + a, A.half_s, ma[0], ma[1], ma[2], ma[3]);
      ma[3] *= __ldg(A.g + j0 + a);
    }
    if (j0 + b < A.n) {
      const float2 pp = __ldg(A.p + j0 + b);
      pb[0] = pp.x;
      pb[1] = pp.y;
      window_consts(A.z, j0 + b, A.half_s, mb[0], mb[1], mb[2], mb[3]);
      mb[3] *= __ldg(A.g + j0 + b);
    }
    P1 = make_float4(-pa[0], -pb[0], -pa[1], -pb[1]);
    P2 = make_float4(ma[0], mb[0], ma[1], mb[1]);
    P3 = make_float4(ma[2], mb[2], ma[3], mb[3]);  // padding rows carry gN = 0
  };
  float4 P1, P2, P3;
  if (t0 < t1) {
    load(t0, P1, P2, P3);
    sm.sA[0][tid] = P1;
    sm.sB[0][tid] = P2;
    sm.sC[0][tid] = P3;
  }
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    if (t + 1 < t1) load(t + 1, P1, P2, P3);
    const int64_t rem = A.n - (int64_t)t * kWbTile;
    const int np = ((rem < kWbTile ? (int)rem : kWbTile) + 1) >> 1;
    float2 acc[kWbR][3];
#pragma unroll
    for (int r = 0; r < kWbR; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[r][c] = bf2(0.f, 0.f);
#pragma unroll 2
    for (int pidx = 0; pidx < np; ++pidx) {
      const float4 a1 = sm.sA[buf][pidx], a2 = sm.sB[buf][pidx], a3 = sm.sC[buf][pidx];
      const float2 nx = bf2(a1.x, a1.y), ny = bf2(a1.z, a1.w);
      const float2 mxx = bf2(a2.x, a2.y), mxy = bf2(a2.z, a2.w), myy = bf2(a3.x, a3.y), gn = bf2(a3.z, a3.w);
#pragma unroll
      for (int r = 0; r < kWbR; ++r) {
        const float2 dx = __fadd2_rn(xs[r], nx), dy = __fadd2_rn(ys[r], ny);
        const float2 ux = __ffma2_rn(mxx, dx, __fmul2_rn(mxy, dy));
        const float2 uy = __ffma2_rn(mxy, dx, __fmul2_rn(myy, dy));
        const float2 e = __ffma2_rn(dx, ux, __fmul2_rn(dy, uy));
        const float2 kg = __fmul2_rn(bf2(ex2_approx(e.x), ex2_approx(e.y)), gn);
        acc[r][0] = __fadd2_rn(acc[r][0], kg);
        acc[r][1] = __ffma2_rn(kg, ux, acc[r][1]);
        acc[r][2] = __ffma2_rn(kg, uy, acc[r][2]);
      }
    }
#pragma unroll
    for (int r = 0; r < kWbR; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float su = sm.ksum[c][r][tid], co = sm.kcomp[c][r][tid];
        wb_kahan(su, co, acc[r][c].x + acc[r][c].y);
        sm.ksum[c][r][tid] = su;
        sm.kcomp[c][r][tid] = co;
      }
    if (t + 1 < t1) {
      sm.sA[buf ^ 1][tid] = P1;
      sm.sB[buf ^ 1][tid] = P2;
      sm.sC[buf ^ 1][tid] = P3;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kWbR; ++r) {
    const int64_t k = (int64_t)rb * kWbRows + r * kWbThreads + tid;
    if (k < A.m)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        A.partial[((int64_t)chunk * 3 + c) * A.m + k] = sm.ksum[c][r][tid] - sm.kcomp[c][r][tid];
  }
}

// ---- merges
struct WbMergeArgs {
  const float* partial;
  int32_t chunks;
  int64_t n;
  const float* z;
  const float* g;
  const float* v;  // columns: source weights
  float half_s, ell;
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
    const float cxx = M.z[3 * i] + M.half_s, cxy = M.z[3 * i + 1], cyy = M.z[3 * i + 2] + M.half_s;
    const float det = fmaf(cxx, cyy, -cxy * cxy), idet = 1.0f / det;
    const float gn = M.g[i] * 0.15915494309189535f * rsqrtf(det);
    // d_p = g N (2 ln 2) P';  D = g N ((2 ln 2)^2 Q' - S M) / 2
    if (M.d_a) {
      M.d_a[2 * i] = gn * kTwoLn2 * s[1];
      M.d_a[2 * i + 1] = gn * kTwoLn2 * s[2];
    }
    const float k2 = kTwoLn2 * kTwoLn2, h = 0.5f * gn;
    const float Dxx = h * fmaf(k2, s[3], -s[0] * cyy * idet);
    const float Dxy = h * fmaf(k2, s[4], s[0] * cxy * idet);
    const float Dyy = h * fmaf(k2, s[5], -s[0] * cxx * idet);
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
  int32_t rows_chunks, rows_blocks, rows_tiles, cols_chunks, cols_blocks, cols_tiles;
  int64_t merge_blocks;
  size_t off_rows, off_scal, off_cols, bytes;
};

static lr_status plan_windowed_bwd(int64_t n, const lr_points* s, WbPlan* P) {
  lr_status st = validate_points(s, "gp_windowed_matvec_bwd(source)", false);
  if (st != LR_OK) return st;
  LR_REQUIRE(!has_lens(s) && s->xy != nullptr, "gp_windowed_matvec_bwd: sources must be explicit points");
  LR_REQUIRE(n >= 0 && n < (int64_t(1) << 31), "gp_windowed_matvec_bwd: n out of range");
  const int64_t m = s->n;
  WbPlan p{};
  int dev = 0, n_sm = 1, occ_r = 1, occ_c = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_r, wn_rows_kernel, kWbThreads, 0));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, wn_cols_kernel, kWbThreads, 0));
  p.rows_blocks = (int32_t)((n + kWbRows - 1) / kWbRows);
  p.rows_tiles = (int32_t)((m + kWbTile - 1) / kWbTile);
  p.rows_chunks = (n > 0 && m > 0) ? plan_chunks(p.rows_blocks, p.rows_tiles, occ_r, n_sm) : 1;
  p.cols_blocks = (int32_t)((m + kWbRows - 1) / kWbRows);
  p.cols_tiles = (int32_t)((n + kWbTile - 1) / kWbTile);
  p.cols_chunks = (n > 0 && m > 0) ? plan_chunks(p.cols_blocks, p.cols_tiles, occ_c, n_sm) : 1;
  p.merge_blocks = (n + 255) / 256;
  size_t o = 0;
  p.off_rows = o;
  o += align256(sizeof(float) * 6 * (size_t)p.rows_chunks * (size_t)n);
  p.off_scal = o;
  o += align256(sizeof(double) * (size_t)(p.merge_blocks + 1));
  p.off_cols = o;
  o += align256(sizeof(float) * 3 * (size_t)p.cols_chunks * (size_t)m);
  p.bytes = o;
  *P = p;
  return LR_OK;
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_windowed_bwd_workspace_size(int64_t n, const lr_points* source, size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_windowed_bwd_workspace_size: bytes is NULL");
  WbPlan P;
  lr_status st = plan_windowed_bwd(n, source, &P);
  if (st != LR_OK) return st;
  *bytes = P.bytes;
  return LR_OK;
}

extern "C" lr_status gp_windowed_matvec_bwd(const float* p, const float* z, int64_t n, const lr_points* source,
                                            const float* v, float lengthscale, const float* g, float* d_v, float* d_p,
                                            float* d_q, float* d_z, double* d_lengthscale, void* workspace,
                                            size_t workspace_bytes, lr_stream stream) {
  WbPlan P;
  lr_status st = plan_windowed_bwd(n, source, &P);
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
  WbArgs A{};
  A.p = reinterpret_cast<const float2*>(p);
  A.z = z;
  A.g = g;
  A.n = n;
  A.q = reinterpret_cast<const float2*>(source->xy);
  A.v = v;
  A.m = m;
  A.half_s = 0.5f * lengthscale * lengthscale;
  if (d_p || d_z || d_lengthscale) {
    A.chunks = P.rows_chunks;
    A.n_tiles = P.rows_tiles;
    A.partial = reinterpret_cast<float*>(ws + P.off_rows);
    wn_rows_kernel<<<(unsigned)((int64_t)P.rows_blocks * P.rows_chunks), kWbThreads, 0, s>>>(A);
    LR_CHECK_CUDA(cudaGetLastError());
    WbMergeArgs M{};
    M.partial = A.partial;
    M.chunks = P.rows_chunks;
    M.n = n;
    M.z = z;
    M.g = g;
    M.half_s = A.half_s;
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
    A.chunks = P.cols_chunks;
    A.n_tiles = P.cols_tiles;
    A.partial = reinterpret_cast<float*>(ws + P.off_cols);
    wn_cols_kernel<<<(unsigned)((int64_t)P.cols_blocks * P.cols_chunks), kWbThreads, 0, s>>>(A);
    LR_CHECK_CUDA(cudaGetLastError());
    WbMergeArgs M{};
    M.partial = A.partial;
    M.chunks = P.cols_chunks;
    M.n = m;
    M.v = v;
    M.d_a = d_v;
    M.d_b = d_q;
    wn_cols_merge_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(M);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
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
