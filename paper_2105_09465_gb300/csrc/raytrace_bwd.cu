// Ray-trace backward (vector-Jacobian product of the deflection sum): given G = dL/dbeta
// for every image-plane point, returns dL/d(x0, y0, q, phi, theta_e, g1, g2)
// of the lens and dL/d(x_h, y_h, kappa_s | theta_pm, theta_s) of every
// subhalo, with dL/dp = -sum_i G_i . dalpha_i/dp (beta = xi - alpha).
//
// The grid has at most one CTA per resident slot; CTA b takes the contiguous
// point range [b n / nblk, (b + 1) n / nblk), so every CTA does the same work
// to within one point and no wave is left partly empty. Points and their G
// are staged through shared memory in tiles; each thread OWNS one subhalo
// (threads loop over subhalo groups when there are more) and sweeps the
// tile's points, reading each point as a shared-memory broadcast, so the
// subhalo sums need no cross-thread reduction at all. The lens and shear
// terms are per point: the thread that stages a point also evaluates them.
// Per-CTA partials (FP64 lens terms, Kahan-compensated FP32 subhalo terms)
// are added in fixed order by a final kernel, so results are deterministic.
#include <math.h>

#include "host.cuh"
#include "problems.cuh"

namespace lr {

constexpr int kVjThreads = 128;
constexpr int kVjTile = kVjThreads;  // points staged per tile (one per thread)
constexpr int kVjWarps = kVjThreads / 32;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct VjSmem {
  float4 pts[2][kVjTile];  // (x, y, G_x, G_y)
  double lred[kVjWarps][7];
};

// One tNFW pair's terms of the four subhalo sums (with explicit roundings,
// so every caller and every kernel that inlines it sums the same values).
__device__ __forceinline__ void vj_accum(const SubRec& rec, float2 ex, float dx, float dy, float gx, float gy,
                                         float R2, float Gt, float Ht, float& a0, float& a1, float& a2, float& a3) {
  const float dg = fmaf(dx, gx, __fmul_rn(dy, gy));
  const float hg = fmaf(-2.0f, Gt, Ht);
  const float q = __fmul_rn(__fmul_rn(hg, dg), frcp(R2));
  a0 = fmaf(rec.A, fmaf(Gt, gx, __fmul_rn(q, dx)), a0);
  a1 = fmaf(rec.A, fmaf(Gt, gy, __fmul_rn(q, dy)), a1);
  a2 = fmaf(-__fmul_rn(ex.x, Gt), dg, a2);
  a3 = fmaf(__fmul_rn(__fmul_rn(rec.A, hg), dg), ex.y, a3);
}

__device__ __forceinline__ void vj_kahan(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <int PROFILE>
__device__ __forceinline__ void vjp_body(const LensConst& L, const LensGradConst& LG, const GridDev& g,
                                         const float2* __restrict__ xi, int64_t n, const float* __restrict__ sub,
                                         int n_sub, const float2* __restrict__ dbeta, double* __restrict__ lens_part,
                                         float* __restrict__ sub_part, int64_t blk, int64_t nblk, VjSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p0 = blk * n / nblk, p1 = (blk + 1) * n / nblk;
  const int ntiles = (int)((p1 - p0 + kVjTile - 1) / kVjTile);
  float la[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int ngroups = n_sub > 0 ? (n_sub + kVjThreads - 1) / kVjThreads : 1;

  // stage point p0 + k kVjTile + tid; the first subhalo group also takes the
  // point's lens and shear terms
  auto load = [&](int k, bool lens_terms) -> float4 {
    const int64_t i = p0 + (int64_t)k * kVjTile + tid;
    if (i >= p1) return make_float4(0.f, 0.f, 0.f, 0.f);  // zero gradient: contributes nothing
    const float2 p = xi ? xi[i] : grid_point(g, i);
    const float2 d = dbeta[i];
    if (lens_terms) {
      float o5[5];
      sple_vjp(L, LG, p.x, p.y, d.x, d.y, o5);
#pragma unroll
      for (int t = 0; t < 5; ++t) la[t] += o5[t];
      la[5] -= fmaf(d.x, p.x, -d.y * p.y);  // dalpha/dg1 = (x, -y)
      la[6] -= fmaf(d.x, p.y, d.y * p.x);   // dalpha/dg2 = (y, x)
    }
    return make_float4(p.x, p.y, d.x, d.y);
  };

  for (int grp = 0; grp < ngroups; ++grp) {
    const int h = grp * kVjThreads + tid;
    const bool own = h < n_sub;
    SubRec rec{};
    float2 ex = make_float2(0.f, 0.f);  // tNFW: (4T, 1/theta_s); point mass: (0, theta_pm)
    if (own) {
      const float* r = sub + 5 * (int64_t)h;
      rec = prep_sub(r, PROFILE);
      if (PROFILE == LR_PROFILE_POINT_MASS) {
        ex = make_float2(0.f, __ldg(r + 2));
      } else {
        const float tau = __ldg(r + 4), t2 = tau * tau;
        ex = make_float2(4.0f * t2 / ((t2 + 1.0f) * (t2 + 1.0f)), 1.0f / __ldg(r + 3));
      }
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
    float4 P = ntiles > 0 ? load(0, grp == 0) : make_float4(0.f, 0.f, 0.f, 0.f);
    sm.pts[0][tid] = P;
    __syncthreads();
    for (int k = 0; k < ntiles; ++k) {
      const int buf = k & 1;
      if (k + 1 < ntiles) P = load(k + 1, grp == 0);
      const int cnt = (int)min((int64_t)kVjTile, p1 - p0 - (int64_t)k * kVjTile);
      if (own) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int j = 0;
        if (PROFILE == LR_PROFILE_TNFW) {
          // two points per step on the straight-line far-side form (the rare
          // near pairs are redone by the general form); same sums, same order
          for (; j + 1 < cnt; j += 2) {
            const float4 Qa = sm.pts[buf][j], Qb = sm.pts[buf][j + 1];
            const float dxa = Qa.x - rec.xh, dya = Qa.y - rec.yh, dxb = Qb.x - rec.xh, dyb = Qb.y - rec.yh;
            const float R2a = fmaf(dxa, dxa, dya * dya), R2b = fmaf(dxb, dxb, dyb * dyb);
            const float x2a = R2a * rec.its2, x2b = R2b * rec.its2;
            float Ga, Ha, Gb, Hb;
            tnfw_GH_far(rec, x2a, Ga, Ha);
            tnfw_GH_far(rec, x2b, Gb, Hb);
            if (!tnfw_is_far(x2a)) tnfw_GH(rec, R2a, Ga, Ha);
            if (!tnfw_is_far(x2b)) tnfw_GH(rec, R2b, Gb, Hb);
            if (R2a > 1e-30f) vj_accum(rec, ex, dxa, dya, Qa.z, Qa.w, R2a, Ga, Ha, a0, a1, a2, a3);
            if (R2b > 1e-30f) vj_accum(rec, ex, dxb, dyb, Qb.z, Qb.w, R2b, Gb, Hb, a0, a1, a2, a3);
          }
        }
        for (; j < cnt; ++j) {
          const float4 Q = sm.pts[buf][j];
          const float dx = Q.x - rec.xh, dy = Q.y - rec.yh;
          const float R2 = fmaf(dx, dx, dy * dy);
          if (!(R2 > 1e-30f)) continue;
          if (PROFILE == LR_PROFILE_TNFW) {
            float Gt, Ht;
            tnfw_GH(rec, R2, Gt, Ht);
            vj_accum(rec, ex, dx, dy, Q.z, Q.w, R2, Gt, Ht, a0, a1, a2, a3);
            continue;
          }
          // point mass
          const float dg = fmaf(dx, Q.z, dy * Q.w);
          const float iR2 = frcp(R2);
          const float m = rec.its2 * iR2;
          const float q = 2.0f * dg * iR2;
          a0 += m * fmaf(-q, dx, Q.z);
          a1 += m * fmaf(-q, dy, Q.w);
          a2 -= 2.0f * ex.y * dg * iR2;
        }
        vj_kahan(s0, c0, a0);
        vj_kahan(s1, c1, a1);
        vj_kahan(s2, c2, a2);
        vj_kahan(s3, c3, a3);
      }
      if (k + 1 < ntiles) sm.pts[buf ^ 1][tid] = P;
      __syncthreads();
    }
    if (own) {
      float* o = sub_part + (blk * n_sub + h) * 4;
      o[0] = s0 - c0;
      o[1] = s1 - c1;
      o[2] = s2 - c2;
      o[3] = s3 - c3;
    }
  }

  // lens terms: warp shuffles then the warps in fixed order, FP64
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    const double v = warp_sum_d((double)la[t]);
    if (lane == 0) sm.lred[warp][t] = v;
  }
  __syncthreads();
  if (tid < 7) {
    double v = 0.0;
    for (int w = 0; w < kVjWarps; ++w) v += sm.lred[w][tid];
    lens_part[blk * 7 + tid] = v;
  }
}

template <int PROFILE>
__global__ void __launch_bounds__(kVjThreads) raytrace_vjp_kernel(const __grid_constant__ LensConst L,
                                                                  const __grid_constant__ LensGradConst LG, GridDev g,
                                                                  const float2* __restrict__ xi, int64_t n,
                                                                  const float* __restrict__ sub, int n_sub,
                                                                  const float2* __restrict__ dbeta,
                                                                  double* __restrict__ lens_part,
                                                                  float* __restrict__ sub_part) {
  __shared__ __align__(16) VjSmem sm;
  vjp_body<PROFILE>(L, LG, g, xi, n, sub, n_sub, dbeta, lens_part, sub_part, blockIdx.x, gridDim.x, sm);
}

__global__ void __launch_bounds__(kVjThreads) vjp_batched_kernel(const __grid_constant__ Batch<VjpP> B) {
  __shared__ __align__(16) VjSmem sm;
  const int k = batch_find(B, blockIdx.x);
  const VjpP& P = B.p[k];
  const int64_t blk = blockIdx.x - B.start[k];
  const int64_t nblk = B.start[k + 1] - B.start[k];
  if (P.profile == LR_PROFILE_POINT_MASS)
    vjp_body<LR_PROFILE_POINT_MASS>(P.L, P.LG, P.g, P.xi, P.n, P.sub, P.n_sub, P.dbeta, P.lens_part, P.sub_part,
                                    blk, nblk, sm);
  else
    vjp_body<LR_PROFILE_TNFW>(P.L, P.LG, P.g, P.xi, P.n, P.sub, P.n_sub, P.dbeta, P.lens_part, P.sub_part, blk,
                              nblk, sm);
}

// CTAs of the VJP for n points: one per resident slot of the device at most
// (and at most one per kVjTile points), so a launch is a single full wave.
int64_t vjp_blocks(int64_t n) {
  if (n <= 0) return 0;
  static int slots[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (slots[dev] == 0) {
    int n_sm = 1, occ = 1;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, raytrace_vjp_kernel<LR_PROFILE_TNFW>, kVjThreads, 0) !=
        cudaSuccess)
      occ = 1;
    slots[dev] = (occ > 0 ? occ : 1) * n_sm;
  }
  const int64_t nb = (n + kVjTile - 1) / kVjTile;
  return nb < slots[dev] ? nb : slots[dev];
}

// Fixed-order FP64 sum of the per-CTA partials: one warp per output value
// (7 lens values, then 4 per subhalo); lane l sums CTAs l, l + 32, ...; the
// warp reduces by xor-shuffle.
__device__ __forceinline__ void vjp_final_body(const double* __restrict__ lens_part,
                                               const float* __restrict__ sub_part, int nblk, int n_sub,
                                               double* __restrict__ d_lens, double* __restrict__ d_sub, int64_t blk) {
  const int o = (int)((blk * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (o >= 7 + 4 * n_sub) return;
  double s = 0.0;
  if (o < 7) {
    for (int b = lane; b < nblk; b += 32) s += lens_part[(int64_t)b * 7 + o];
  } else {
    const int t = o - 7;
    for (int b = lane; b < nblk; b += 32) s += (double)sub_part[(int64_t)b * n_sub * 4 + t];
  }
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if (lane == 0) {
    if (o < 7) {
      if (d_lens) d_lens[o] = s;
    } else if (d_sub) {
      d_sub[o - 7] = s;
    }
  }
}

__global__ void vjp_final_kernel(const double* __restrict__ lens_part, const float* __restrict__ sub_part, int nblk,
                                 int n_sub, double* __restrict__ d_lens, double* __restrict__ d_sub) {
  vjp_final_body(lens_part, sub_part, nblk, n_sub, d_lens, d_sub, blockIdx.x);
}

__global__ void vjp_final_batched_kernel(const __grid_constant__ Batch<VjpFinalP> B) {
  const int k = batch_find(B, blockIdx.x);
  const VjpFinalP& P = B.p[k];
  vjp_final_body(P.lens_part, P.sub_part, P.nblk, P.n_sub, P.d_lens, P.d_sub, blockIdx.x - B.start[k]);
}

lr_status launch_vjp_batched(const VjpP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<VjpP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += vjp_blocks(p[b0 + k].n);
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    vjp_batched_kernel<<<(unsigned)tot, kVjThreads, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

lr_status launch_vjp_final_batched(const VjpFinalP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<VjpFinalP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += ((7 + 4 * (int64_t)p[b0 + k].n_sub) * 32 + 255) / 256;
    }
    B.start[B.count] = (int32_t)tot;
    vjp_final_batched_kernel<<<(unsigned)tot, 256, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Host side

lr_status make_lens_grad_const(const lr_lens* lens, LensGradConst* out) {
  const double q = lens->q, gam = lens->gamma, te = lens->theta_e;
  LensGradConst G;
  memset(&G, 0, sizeof G);
  G.e = (float)(0.5 * (1.0 - gam));
  const double f = (1.0 - q) / (1.0 + q);
  G.f = (float)f;
  G.dlnpre_dq = (float)(0.5 / q - 1.0 / (1.0 + q));
  G.df_dq = (float)(-2.0 / ((1.0 + q) * (1.0 + q)));
  G.inv2q = (float)(0.5 / q);
  G.dlnte = te > 0.0 ? (float)((gam - 1.0) / te) : 0.f;
  // h_n = (n+1) c_{n+1} (-f)^n, c_n = prod_{k<=n} (a+k-1)/(b+k-1)
  const double a = 0.5 * (gam - 1.0), b = 0.5 * (5.0 - gam);
  double c = 1.0, fn = 1.0;  // c_{n+1}, (-f)^n
  int n = 0;
  for (n = 0; n < kMaxSeriesTerms; ++n) {
    c *= (a + n) / (b + n);  // c_{n+1}
    const double hn = (n + 1.0) * c * fn;
    G.hco[n] = (float)hn;
    // tail bound for sum_{k>n} |h_k|: |h_n| f (n+2)/(n+1) / (1 - f)^2
    if (f == 0.0 || fabs(hn) * f * (n + 2.0) / (n + 1.0) / ((1.0 - f) * (1.0 - f)) < 1e-9) {
      ++n;
      break;
    }
    fn *= -f;
  }
  LR_REQUIRE(n <= kMaxSeriesTerms, "lens q = %g too small for the gradient series", q);
  G.nterms = n < 1 ? 1 : n;
  *out = G;
  return LR_OK;
}

size_t raytrace_vjp_ws(int64_t n, int32_t n_sub) {
  const int64_t nblk = vjp_blocks(n);
  return align256(sizeof(double) * 7 * (size_t)nblk) + align256(sizeof(float) * 4 * (size_t)n_sub * (size_t)nblk);
}

lr_status launch_raytrace_vjp(const lr_points* p, const float2* dbeta, double* d_lens, double* d_sub, void* ws,
                              cudaStream_t s) {
  LensConst L;
  lr_status st = make_lens_const(p->lens, &L);
  if (st != LR_OK) return st;
  LensGradConst G;
  st = make_lens_grad_const(p->lens, &G);
  if (st != LR_OK) return st;
  const int64_t nblk = vjp_blocks(p->n);
  if (nblk == 0) {
    if (d_lens) LR_CHECK_CUDA(cudaMemsetAsync(d_lens, 0, 7 * sizeof(double), s));
    if (d_sub && p->n_sub) LR_CHECK_CUDA(cudaMemsetAsync(d_sub, 0, 4 * sizeof(double) * p->n_sub, s));
    return LR_OK;
  }
  double* lens_part = static_cast<double*>(ws);
  float* sub_part = reinterpret_cast<float*>(static_cast<char*>(ws) + align256(sizeof(double) * 7 * (size_t)nblk));
  const GridDev g = p->xy ? GridDev{} : grid_dev(p->grid);
  const float2* xi = reinterpret_cast<const float2*>(p->xy);
  if (p->profile == LR_PROFILE_POINT_MASS)
    raytrace_vjp_kernel<LR_PROFILE_POINT_MASS><<<(unsigned)nblk, kVjThreads, 0, s>>>(
        L, G, g, xi, p->n, p->sub, p->n_sub, dbeta, lens_part, sub_part);
  else
    raytrace_vjp_kernel<LR_PROFILE_TNFW><<<(unsigned)nblk, kVjThreads, 0, s>>>(
        L, G, g, xi, p->n, p->sub, p->n_sub, dbeta, lens_part, sub_part);
  LR_CHECK_CUDA(cudaGetLastError());
  const int64_t warps = 7 + 4 * (int64_t)p->n_sub;
  vjp_final_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(lens_part, sub_part, (int)nblk, p->n_sub,
                                                                        d_lens, p->n_sub ? d_sub : nullptr);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

// Problem descriptors for the ray-trace VJP; ws (raytrace_vjp_ws bytes) holds
// the per-CTA partials.
lr_status make_vjp_problem(const lr_points* p, const float2* dbeta, double* d_lens, double* d_sub, void* ws, VjpP* V,
                           VjpFinalP* F) {
  VjpP v{};
  lr_status st = make_lens_const(p->lens, &v.L);
  if (st != LR_OK) return st;
  st = make_lens_grad_const(p->lens, &v.LG);
  if (st != LR_OK) return st;
  const int64_t nblk = vjp_blocks(p->n);
  v.g = p->xy ? GridDev{} : grid_dev(p->grid);
  v.xi = reinterpret_cast<const float2*>(p->xy);
  v.n = p->n;
  v.sub = p->sub;
  v.n_sub = p->n_sub;
  v.profile = p->profile;
  v.dbeta = dbeta;
  v.lens_part = static_cast<double*>(ws);
  v.sub_part = reinterpret_cast<float*>(static_cast<char*>(ws) + align256(sizeof(double) * 7 * (size_t)nblk));
  *V = v;
  F->lens_part = v.lens_part;
  F->sub_part = v.sub_part;
  F->nblk = (int32_t)nblk;
  F->n_sub = p->n_sub;
  F->d_lens = d_lens;
  F->d_sub = p->n_sub ? d_sub : nullptr;
  return LR_OK;
}

}  // namespace lr

extern "C" lr_status lr_raytrace_vjp_workspace_size(const lr_points* pts, size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_raytrace_vjp_workspace_size: bytes is NULL");
  lr_status st = lr::validate_points(pts, "lr_raytrace_vjp_workspace_size", true);
  if (st != LR_OK) return st;
  *bytes = lr::raytrace_vjp_ws(pts->n, pts->n_sub);
  return LR_OK;
}

extern "C" lr_status lens_raytrace_vjp(const lr_points* pts, const float* d_beta, double* d_lens, double* d_sub,
                                       void* workspace, size_t workspace_bytes, lr_stream stream) {
  lr_status st = lr::validate_points(pts, "lens_raytrace_vjp", true);
  if (st != LR_OK) return st;
  LR_REQUIRE(d_beta != nullptr || pts->n == 0, "lens_raytrace_vjp: d_beta is NULL");
  LR_REQUIRE(((uintptr_t)d_beta & 7u) == 0, "lens_raytrace_vjp: d_beta must be 8-byte aligned");
  LR_REQUIRE(((uintptr_t)d_lens & 7u) == 0 && ((uintptr_t)d_sub & 7u) == 0,
             "lens_raytrace_vjp: gradient outputs must be 8-byte aligned");
  const size_t need = lr::raytrace_vjp_ws(pts->n, pts->n_sub);
  LR_REQUIRE(workspace_bytes >= need, "lens_raytrace_vjp: workspace of %zu bytes, %zu needed", workspace_bytes, need);
  LR_REQUIRE(need == 0 || workspace != nullptr, "lens_raytrace_vjp: workspace is NULL");
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0, "lens_raytrace_vjp: workspace must be 256-byte aligned");
  return lr::launch_raytrace_vjp(pts, reinterpret_cast<const float2*>(d_beta), d_lens, d_sub, workspace,
                                 lr::as_cuda(stream));
}
