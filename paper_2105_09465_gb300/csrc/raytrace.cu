// Pixel-grid generation and the lens ray-trace beta = xi - alpha(xi).
//
// One thread per image-plane point. The SPLE and shear terms are evaluated in
// registers from per-lens constants passed as a kernel parameter; the
// subhalo records are staged into shared memory in chunks by a bulk
// asynchronous copy (the TMA engine's 1-D form) and reused by every point of
// the CTA. Stores are coalesced float2 writes.
#include <math.h>

#include "host.cuh"
#include "problems.cuh"
#include "lens.cuh"
#include "subs.cuh"

namespace lr {

constexpr int kRtThreads = 256;
constexpr int kSubChunk = 256;  // subhalos staged per chunk (multiple of 4)

__global__ void grid_points_kernel(GridDev g, int64_t n, float2* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = grid_point(g, i);
}

constexpr int kRtFold = 8;  // subhalos summed plainly before a Kahan fold

__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Deflection of the staged subhalos at (x, y), added to the Kahan sums
// (sx, cx), (sy, cy). Blocks of kRtFold subhalos are summed plainly in two
// packed lanes (even and odd subhalos) and folded into the Kahan sums; the
// fold order is fixed, so every kernel that calls this gets the same bits.
template <int PROFILE>
__device__ __forceinline__ void add_subs(const SubRec2* recs2, int cnt, float x, float y, float& sx, float& cx,
                                         float& sy, float& cy) {
  const float2 X = f2(x), Y = f2(y);
  for (int t0 = 0; t0 < cnt; t0 += kRtFold) {
    const int t1 = min(cnt, t0 + kRtFold);
    float2 ax = f2(0.f), ay = f2(0.f);
    int t = t0;
    if (PROFILE == LR_PROFILE_TNFW) {
      // two subhalos per step on the packed far-side form (the rare near
      // pairs are redone by the general form, which gives the same bits for
      // far pairs)
      for (; t + 1 < t1; t += 2) {
        const SubRec2 H = recs2[t >> 1];
        const float2 dx = sub2(X, H.xh), dy = sub2(Y, H.yh);
        const float2 R2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
        const float2 x2 = __fmul2_rn(R2, H.its2);
        float2 m = tnfw_m_far2(H, x2);
        if (!tnfw_is_far(x2.x)) m.x = tnfw_m(sub_lane(H, 0), R2.x);
        if (!tnfw_is_far(x2.y)) m.y = tnfw_m(sub_lane(H, 1), R2.y);
        ax = __ffma2_rn(m, dx, ax);
        ay = __ffma2_rn(m, dy, ay);
      }
    }
    for (; t < t1; ++t) {
      const SubRec h = sub_lane(recs2[t >> 1], t & 1);
      const float dx = __fsub_rn(x, h.xh), dy = __fsub_rn(y, h.yh);
      const float R2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
      const float m = (PROFILE == LR_PROFILE_POINT_MASS) ? pointmass_m(h, R2) : tnfw_m(h, R2);
      if (t & 1) {
        ax.y = __fmaf_rn(m, dx, ax.y);
        ay.y = __fmaf_rn(m, dy, ay.y);
      } else {
        ax.x = __fmaf_rn(m, dx, ax.x);
        ay.x = __fmaf_rn(m, dy, ay.x);
      }
    }
    kahan(sx, cx, __fadd_rn(ax.x, ax.y));
    kahan(sy, cy, __fadd_rn(ay.x, ay.y));
  }
}

struct RtSmem {
  float raw[5 * kSubChunk];
  SubRec2 recs2[kSubChunk / 2];
  uint64_t bar;
};

template <int PROFILE>
__device__ __forceinline__ void raytrace_body(const LensConst& L, const GridDev& g, const float2* __restrict__ xi,
                                              int64_t n, const float* __restrict__ sub, int n_sub, int bulk_ok,
                                              float2* __restrict__ beta, float2* __restrict__ alpha_out, int* fault,
                                              int64_t blk, RtSmem& sm) {
  const int64_t i = blk * kRtThreads + threadIdx.x;
  const bool valid = i < n;
  const int64_t ii = valid ? i : (n - 1);
  const float2 p = xi ? xi[ii] : grid_point(g, ii);

  float ax, ay;
  sple_alpha(L, p.x, p.y, ax, ay);
  // external shear about the origin
  ax = fmaf(L.g1, p.x, fmaf(L.g2, p.y, ax));
  ay = fmaf(L.g2, p.x, fmaf(-L.g1, p.y, ay));

  if (n_sub > 0) {
    if (threadIdx.x == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
    for (int h0 = 0; h0 < n_sub; h0 += kSubChunk) {
      const int cnt = min(kSubChunk, n_sub - h0);
      if (!stage_subs2(sub, h0, cnt, PROFILE, sm.raw, sm.recs2, &sm.bar, phase, bulk_ok != 0, fault)) return;
      add_subs<PROFILE>(sm.recs2, cnt, p.x, p.y, sx, cx, sy, cy);
      __syncthreads();
    }
    ax += sx - cx;
    ay += sy - cy;
  }
  if (valid) {
    beta[i] = make_float2(p.x - ax, p.y - ay);
    if (alpha_out) alpha_out[i] = make_float2(ax, ay);
  }
}

template <int PROFILE>
__global__ void __launch_bounds__(kRtThreads) raytrace_kernel(const __grid_constant__ LensConst L, GridDev g,
                                                              const float2* __restrict__ xi, int64_t n,
                                                              const float* __restrict__ sub, int n_sub, int bulk_ok,
                                                              float2* __restrict__ beta,
                                                              float2* __restrict__ alpha_out, int* fault) {
  __shared__ __align__(16) RtSmem sm;
  raytrace_body<PROFILE>(L, g, xi, n, sub, n_sub, bulk_ok, beta, alpha_out, fault, blockIdx.x, sm);
}

__global__ void __launch_bounds__(kRtThreads) raytrace_batched_kernel(const __grid_constant__ Batch<RtP> B,
                                                                      int* fault) {
  __shared__ __align__(16) RtSmem sm;
  const int k = batch_find(B, blockIdx.x);
  const RtP& P = B.p[k];
  const int64_t blk = blockIdx.x - B.start[k];
  if (P.profile == LR_PROFILE_POINT_MASS)
    raytrace_body<LR_PROFILE_POINT_MASS>(P.L, P.g, P.xi, P.n, P.sub, P.n_sub, P.bulk_ok, P.beta, P.alpha, fault,
                                         blk, sm);
  else
    raytrace_body<LR_PROFILE_TNFW>(P.L, P.g, P.xi, P.n, P.sub, P.n_sub, P.bulk_ok, P.beta, P.alpha, fault, blk,
                                   sm);
}

lr_status launch_raytrace_batched(const RtP* p, int count, cudaStream_t s) {
  int* fault = fault_ptr();
  LR_REQUIRE(fault != nullptr, "could not resolve the device fault word");
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<RtP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += (p[b0 + k].n + kRtThreads - 1) / kRtThreads;
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    raytrace_batched_kernel<<<(unsigned)tot, kRtThreads, 0, s>>>(B, fault);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Host side

static bool finitef(float v) { return isfinite(v); }

lr_status make_lens_const(const lr_lens* lens, LensConst* out) {
  LR_REQUIRE(lens != nullptr, "lens is NULL");
  const float* f = &lens->x0;
  for (int k = 0; k < 8; ++k) LR_REQUIRE(finitef(f[k]), "lens parameter %d is not finite", k);
  LR_REQUIRE(lens->q > 0.f && lens->q <= 1.f, "lens q = %g outside (0, 1]", (double)lens->q);
  LR_REQUIRE(lens->gamma > 1.f && lens->gamma < 3.f, "lens gamma = %g outside (1, 3)", (double)lens->gamma);
  LR_REQUIRE(lens->theta_e >= 0.f, "lens theta_e = %g < 0", (double)lens->theta_e);
  const double q = lens->q, gam = lens->gamma, te = lens->theta_e, phi = lens->phi;
  LensConst L;
  memset(&L, 0, sizeof L);
  L.x0 = lens->x0;
  L.y0 = lens->y0;
  L.c = (float)cos(phi);
  L.s = (float)sin(phi);
  L.sq = (float)sqrt(q);
  L.isq = (float)(1.0 / sqrt(q));
  L.pre = (float)(pow(te, gam - 1.0) * 2.0 * sqrt(q) / (1.0 + q));
  L.half_expo = (float)(0.5 * (1.0 - gam));
  L.g1 = lens->g1;
  L.g2 = lens->g2;
  // 2F1(1, a; b; -f w) = sum_n c_n (-f)^n w^n, c_n = prod_{k<=n} (a+k-1)/(b+k-1)
  const double a = 0.5 * (gam - 1.0), b = 0.5 * (5.0 - gam), fq = (1.0 - q) / (1.0 + q);
  double c = 1.0, fn = 1.0;
  int n = 0;
  L.d[0] = 1.0f;
  for (n = 1; n < kMaxSeriesTerms; ++n) {
    // tail bound: |d_n| f / (1 - f) (coefficient ratios are below 1 for gamma < 3)
    if (fq == 0.0 || fabs(c * fn) * fq / (1.0 - fq) < 1e-9) break;
    c *= (a + n - 1.0) / (b + n - 1.0);
    fn *= -fq;
    L.d[n] = (float)(c * fn);
  }
  LR_REQUIRE(fq == 0.0 || fabs(c * fn) * fq / (1.0 - fq) < 1e-9,
             "lens q = %g too small: the deflection series needs more than %d terms", q, kMaxSeriesTerms);
  L.nterms = n;
  *out = L;
  return LR_OK;
}

int64_t grid_count(const lr_grid& g) { return (int64_t)g.nx * g.ss * (int64_t)g.ny * g.ss; }

lr_status validate_points(const lr_points* p, const char* what, bool need_lens) {
  LR_REQUIRE(p != nullptr, "%s: point set is NULL", what);
  LR_REQUIRE(p->n >= 0, "%s: n = %lld < 0", what, (long long)p->n);
  LR_REQUIRE(p->n < (int64_t(1) << 31), "%s: n = %lld exceeds 2^31 - 1", what, (long long)p->n);
  if (p->n == 0) {
    // empty set: positions are never read (an empty tensor has a NULL data pointer)
  } else if (p->xy == nullptr) {
    const lr_grid& g = p->grid;
    LR_REQUIRE(g.nx > 0 && g.ny > 0 && g.ss > 0, "%s: grid dimensions must be positive", what);
    LR_REQUIRE(isfinite(g.pix) && g.pix > 0.f && isfinite(g.cx) && isfinite(g.cy), "%s: bad grid geometry", what);
    LR_REQUIRE((int64_t)g.nx * g.ss < (1 << 24) && (int64_t)g.ny * g.ss < (1 << 24),
               "%s: grid side exceeds 2^24 points", what);
    LR_REQUIRE(grid_count(g) == p->n, "%s: grid has %lld points but n = %lld", what, (long long)grid_count(g),
               (long long)p->n);
  } else {
    LR_REQUIRE(((uintptr_t)p->xy & 7u) == 0, "%s: xy must be 8-byte aligned", what);
  }
  if (need_lens) LR_REQUIRE(p->lens != nullptr, "%s: a lens is required", what);
  if (p->lens) {
    LR_REQUIRE(p->n_sub >= 0, "%s: n_sub < 0", what);
    LR_REQUIRE(p->n_sub == 0 || p->sub != nullptr, "%s: sub is NULL with n_sub = %d", what, p->n_sub);
    LR_REQUIRE(p->sub == nullptr || ((uintptr_t)p->sub & 3u) == 0, "%s: sub must be 4-byte aligned", what);
    LR_REQUIRE(p->profile == LR_PROFILE_TNFW || p->profile == LR_PROFILE_POINT_MASS, "%s: unknown profile %d",
               what, p->profile);
  }
  return LR_OK;
}

lr_status launch_grid_points(const lr_grid& g, float2* out, cudaStream_t s) {
  const int64_t n = grid_count(g);
  if (n == 0) return LR_OK;
  grid_points_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(grid_dev(g), n, out);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

lr_status launch_raytrace(const lr_points* p, float2* beta, float2* alpha, cudaStream_t s) {
  LensConst L;
  lr_status st = make_lens_const(p->lens, &L);
  if (st != LR_OK) return st;
  if (p->n == 0) return LR_OK;
  int* fault = fault_ptr();
  LR_REQUIRE(fault != nullptr, "could not resolve the device fault word");
  const GridDev g = p->xy ? GridDev{} : grid_dev(p->grid);
  const int bulk_ok = (((uintptr_t)p->sub & 15u) == 0) ? 1 : 0;
  const unsigned blocks = (unsigned)((p->n + kRtThreads - 1) / kRtThreads);
  const float2* xi = reinterpret_cast<const float2*>(p->xy);
  const int ns = p->n_sub;
  ktimer_begin(LR_KT_RAYTRACE, s);
  if (p->profile == LR_PROFILE_POINT_MASS)
    raytrace_kernel<LR_PROFILE_POINT_MASS><<<blocks, kRtThreads, 0, s>>>(L, g, xi, p->n, p->sub, ns, bulk_ok, beta,
                                                                         alpha, fault);
  else
    raytrace_kernel<LR_PROFILE_TNFW><<<blocks, kRtThreads, 0, s>>>(L, g, xi, p->n, p->sub, ns, bulk_ok, beta, alpha,
                                                                   fault);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_RAYTRACE, s);
  return LR_OK;
}

lr_status make_rt_problem(const lr_points* p, float2* beta, float2* alpha, RtP* R) {
  RtP r{};
  lr_status st = make_lens_const(p->lens, &r.L);
  if (st != LR_OK) return st;
  r.g = p->xy ? GridDev{} : grid_dev(p->grid);
  r.xi = reinterpret_cast<const float2*>(p->xy);
  r.n = p->n;
  r.sub = p->sub;
  r.n_sub = p->n_sub;
  r.bulk_ok = (((uintptr_t)p->sub & 15u) == 0) ? 1 : 0;
  r.profile = p->profile;
  r.beta = beta;
  r.alpha = alpha;
  *R = r;
  return LR_OK;
}

}  // namespace lr

extern "C" lr_status lens_raytrace(const lr_points* pts, float* beta_out, float* alpha_out, lr_stream stream) {
  lr_status st = lr::validate_points(pts, "lens_raytrace", true);
  if (st != LR_OK) return st;
  LR_REQUIRE(beta_out != nullptr || pts->n == 0, "lens_raytrace: beta_out is NULL");
  LR_REQUIRE(((uintptr_t)beta_out & 7u) == 0 && ((uintptr_t)alpha_out & 7u) == 0,
             "lens_raytrace: outputs must be 8-byte aligned");
  return lr::launch_raytrace(pts, reinterpret_cast<float2*>(beta_out), reinterpret_cast<float2*>(alpha_out),
                             lr::as_cuda(stream));
}
