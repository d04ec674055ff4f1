// Pixel-grid generation and the lens ray-trace beta = xi - alpha(xi).
//
// Two image-plane points per thread; a CTA takes a 16 x 16 tile of a pixel
// grid (or 256 consecutive explicit points). The SPLE and shear terms are
// evaluated in registers from per-lens constants passed as a kernel
// parameter; the subhalo records are staged into shared memory in chunks by a
// bulk asynchronous copy (the TMA engine's 1-D form) and reused by every
// point of the CTA. Each chunk is sorted by the degree of the far-field
// series that serves the whole tile (rt_degree, fewest terms first), and each
// degree's run is swept without per-pair tests; the rest take a per-pair
// choice of series, far-side closed form or general form. Stores are
// coalesced float2 writes.
#include <math.h>

#include "host.cuh"
#include "problems.cuh"
#include "lens.cuh"
#include "subs.cuh"

namespace lr {

constexpr int kRtThreads = 128;
constexpr int kRtPts = 2;                        // points per thread
constexpr int kRtPoints = kRtThreads * kRtPts;   // points per CTA
constexpr int kRtTile = 16;  // grid input: a CTA takes a kRtTile x kRtTile tile of pixels
static_assert(kRtTile * kRtTile == kRtPoints, "the CTA's points are one tile");
constexpr int kSubChunk = 256;  // subhalos staged per chunk (multiple of 4)

__global__ void grid_points_kernel(GridDev g, int64_t n, float2* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = grid_point(g, i);
}

constexpr int kRtFold = 8;        // subhalos summed plainly before a Kahan fold (closed forms)
constexpr int kRtFoldPairs = 16;  // staged pairs summed plainly before a Kahan fold (series runs)

__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Staged subhalos, as consecutive pairs (a, b), field by field as packed
// pairs. The hot words are all the series needs:
//   [0] (xh, yh)  [1] (its2, A)  [2] (xT2, q0)  [3..6] (q2, q3) .. (q8, q9);
// the cold words the closed forms: [0] (tau, tau2)  [1] (t2m1_l, C).
constexpr int kRtHot = 7, kRtCold = 2;

struct RtSmem {
  float raw[5 * kSubChunk];
  float4 hot[kSubChunk / 2][kRtHot];
  float4 cold[kSubChunk / 2][kRtCold];
  int order[kSubChunk];  // staged position -> subhalo of the chunk
  unsigned char deg[kSubChunk];  // series degree for the CTA's points of each subhalo of the chunk (0: none)
  int ndeg[5];                   // staged subhalos served by the series to y^3, y^4, y^5, y^7, y^9
  int wcnt[kRtThreads / 32][6];  // per warp's quarter of the chunk: subhalos by degree class
  float box[4];          // the CTA's points: x_lo, y_lo, x_hi, y_hi
  int nfar;
  uint64_t bar;
};

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

__device__ __forceinline__ SubRec2 rec_from(const float4* hot, const float4* cold) {
  SubRec2 r;
  r.xh = make_float2(hot[0].x, hot[0].y);
  r.yh = make_float2(hot[0].z, hot[0].w);
  r.its2 = lo2(hot[1]);
  r.A = hi2(hot[1]);
  r.tau = lo2(cold[0]);
  r.tau2 = hi2(cold[0]);
  r.t2m1_l = lo2(cold[1]);
  r.C = hi2(cold[1]);
  return r;
}

__device__ __forceinline__ SubSer ser_from(const float4* hot, int k) {
  SubSer s;
  s.xT2 = k ? hot[2].y : hot[2].x;
  s.q[0] = k ? hot[2].w : hot[2].z;
  s.q[1] = 0.f;
#pragma unroll
  for (int j = 2; j < kSerTerms; ++j) {
    const float4 w = hot[3 + (j - 2) / 2];
    s.q[j] = (j & 1) ? (k ? w.w : w.z) : (k ? w.y : w.x);
  }
  return s;
}

// The degree K of the deflection's far-field series (prep_series) that
// serves every pair of a subhalo with points at x^2 >= x2min, with m =
// max(tau^2, 4): the terms up to y^K from x = r_K max(tau, 2) on, K = 9 from
// r = 6, 7 from 8, 5 from 18, 4 from 32, 3 from 80 (the truncated terms fall
// as (tau / x)^(K + 1); against the closed form in extended precision within
// 5e-10 relative for K = 9 and 1.4e-8 for the others, tau in [0.5, 30]).
// 0 below 6 max(tau, 2).
__device__ __forceinline__ int rt_degree(float x2min, float m) {
  return x2min >= 6400.0f * m   ? 3
         : x2min >= 1024.0f * m ? 4
         : x2min >= 324.0f * m  ? 5
         : x2min >= 64.0f * m   ? 7
         : x2min >= 36.0f * m   ? 9
                                : 0;
}

// Stages subhalos [h0, h0 + cnt). Subhalos whose centre is beyond the series
// radius from the whole box of the CTA's points (every pair of them takes the
// series) come first, ordered by the degree that serves the whole box
// (rt_degree, fewest terms first), each degree in index order; sm.ndeg
// counts them by degree and sm.nfar in all. Returns false (all threads) if
// the bulk-copy wait timed out.
__device__ __forceinline__ bool stage_rt(const float* __restrict__ sub, int h0, int cnt, int profile, RtSmem& sm,
                                         uint32_t& phase, bool bulk_ok, int* fault) {
  if (!stage_raw(sub, h0, cnt, sm.raw, &sm.bar, phase, bulk_ok, fault)) return false;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const SubRec h = prep_sub(sm.raw + 5 * t, profile);
    const SubSer q = prep_series(h, profile);
    const float dx = fmaxf(fmaxf(sm.box[0] - h.xh, h.xh - sm.box[2]), 0.f);
    const float dy = fmaxf(fmaxf(sm.box[1] - h.yh, h.yh - sm.box[3]), 0.f);
    sm.deg[t] = isinf(q.xT2) ? 0
                             : (unsigned char)rt_degree(__fmul_rn(fmaf(dx, dx, dy * dy), h.its2), fmaxf(h.tau2, 4.0f));
  }
  __syncthreads();
  // stable partition by degree class: 3, 4, 5, 7, 9, then 0 (not far). Warp
  // w takes the chunk's positions [w q, (w + 1) q), q = kSubChunk / warps:
  // it counts its subhalos per class, then scatters them after the classes
  // before theirs and the warps before it.
  constexpr int kW = kRtThreads / 32, kQ = kSubChunk / kW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int pass = 0; pass < 6; ++pass) {
    const int want = pass == 5 ? 0 : (pass < 3 ? 3 + pass : 2 * pass + 1);
    int nc = 0;
    for (int b = warp * kQ; b < (warp + 1) * kQ; b += 32)
      nc += __popc(__ballot_sync(0xffffffffu, b + lane < cnt && sm.deg[b + lane] == want));
    if (lane == 0) sm.wcnt[warp][pass] = nc;
  }
  __syncthreads();
  int nf = 0;  // this warp's first position of the class
#pragma unroll 1
  for (int pass = 0; pass < 6; ++pass) {
    const int want = pass == 5 ? 0 : (pass < 3 ? 3 + pass : 2 * pass + 1);
    int tot = 0, before = 0;
    for (int w = 0; w < kW; ++w) {
      tot += sm.wcnt[w][pass];
      if (w < warp) before += sm.wcnt[w][pass];
    }
    if (threadIdx.x == 0) {
      if (pass < 5) sm.ndeg[pass] = tot;
      if (pass == 5) sm.nfar = nf;  // thread 0 is in warp 0: nf is the count of all far classes
    }
    int pos = nf + before;
    for (int b = warp * kQ; b < (warp + 1) * kQ; b += 32) {
      const bool f = b + lane < cnt && sm.deg[b + lane] == want;
      const unsigned m = __ballot_sync(0xffffffffu, f);
      if (f) sm.order[pos + __popc(m & ((1u << lane) - 1u))] = b + lane;
      pos += __popc(m);
    }
    nf += tot;
  }
  __syncthreads();
  for (int k = threadIdx.x; 2 * k < cnt; k += blockDim.x) {
    const SubRec a = prep_sub(sm.raw + 5 * sm.order[2 * k], profile);
    const bool hb = 2 * k + 1 < cnt;
    const SubRec b = hb ? prep_sub(sm.raw + 5 * sm.order[2 * k + 1], profile) : SubRec{};
    const SubSer sa = prep_series(a, profile), sb = prep_series(b, hb ? profile : LR_PROFILE_POINT_MASS);
    float4* hot = sm.hot[k];
    hot[0] = make_float4(a.xh, b.xh, a.yh, b.yh);
    hot[1] = make_float4(a.its2, b.its2, a.A, b.A);
    hot[2] = make_float4(sa.xT2, sb.xT2, sa.q[0], sb.q[0]);
#pragma unroll
    for (int w = 0; w < 4; ++w)
      hot[3 + w] = make_float4(sa.q[2 + 2 * w], sb.q[2 + 2 * w], sa.q[3 + 2 * w], sb.q[3 + 2 * w]);
    sm.cold[k][0] = make_float4(a.tau, b.tau, a.tau2, b.tau2);
    sm.cold[k][1] = make_float4(a.t2m1_l, b.t2m1_l, a.C, b.C);
  }
  __syncthreads();
  return true;
}

// m = A y^2 Q(y) of two subhalos (or one twice) by the series to y^K: q[j]
// for j = 2 .. K (explicitly rounded; K = 9 is tnfw_m_series2).
template <int K>
__device__ __forceinline__ float2 rt_series2(float2 A, float2 q0, const float2* q, float2 x2) {
  const float2 y = frsqrt2(x2), y2 = __fmul2_rn(y, y);
  float2 p = q[K];
#pragma unroll
  for (int j = K - 1; j >= 2; --j) p = __ffma2_rn(p, y, q[j]);
  return __fmul2_rn(A, __fmul2_rn(y2, __ffma2_rn(p, y2, q0)));
}

// The series coefficients q[2 .. K] of a staged pair.
template <int K>
__device__ __forceinline__ void rt_coeffs(const float4* hot, float2 (&q)[kSerTerms]) {
#pragma unroll
  for (int j = 2; j <= K; ++j) {
    const float4 c = hot[3 + (j - 2) / 2];
    q[j] = (j & 1) ? hi2(c) : lo2(c);
  }
}

// Staged pairs kp and kp + 1 (four subhalos, all far from every point of the
// CTA) by the series to y^K: four independent chains per thread, added in
// order.
template <int K>
__device__ __forceinline__ void rt_far4(const RtSmem& sm, int kp, const float2 (&X)[kRtPts],
                                        const float2 (&Y)[kRtPts], float2 (&ax)[kRtPts], float2 (&ay)[kRtPts]) {
  float2 m[2][kRtPts], dxs[2][kRtPts], dys[2][kRtPts];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const float4* hot = sm.hot[kp + u];
    const float4 w0 = hot[0], w1 = hot[1], w2 = hot[2];
    float2 q[kSerTerms];
    rt_coeffs<K>(hot, q);
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) {
      dxs[u][j] = sub2(X[j], make_float2(w0.x, w0.y));
      dys[u][j] = sub2(Y[j], make_float2(w0.z, w0.w));
      const float2 R2 = __ffma2_rn(dxs[u][j], dxs[u][j], __fmul2_rn(dys[u][j], dys[u][j]));
      m[u][j] = rt_series2<K>(hi2(w1), hi2(w2), q, __fmul2_rn(R2, lo2(w1)));
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) {
      ax[j] = __ffma2_rn(m[u][j], dxs[u][j], ax[j]);
      ay[j] = __ffma2_rn(m[u][j], dys[u][j], ay[j]);
    }
  }
}

// Staged pair kp (both subhalos far from every point of the CTA) by the
// series to y^K.
template <int K>
__device__ __forceinline__ void rt_far2(const RtSmem& sm, int kp, const float2 (&X)[kRtPts],
                                        const float2 (&Y)[kRtPts], float2 (&ax)[kRtPts], float2 (&ay)[kRtPts]) {
  const float4* hot = sm.hot[kp];
  const float4 w0 = hot[0], w1 = hot[1], w2 = hot[2];
  float2 q[kSerTerms];
  rt_coeffs<K>(hot, q);
#pragma unroll
  for (int j = 0; j < kRtPts; ++j) {
    const float2 dx = sub2(X[j], make_float2(w0.x, w0.y)), dy = sub2(Y[j], make_float2(w0.z, w0.w));
    const float2 R2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
    const float2 m = rt_series2<K>(hi2(w1), hi2(w2), q, __fmul2_rn(R2, lo2(w1)));
    ax[j] = __ffma2_rn(m, dx, ax[j]);
    ay[j] = __ffma2_rn(m, dy, ay[j]);
  }
}

__device__ __forceinline__ void fold(const float2 (&ax)[kRtPts], const float2 (&ay)[kRtPts], float (&sx)[kRtPts],
                                     float (&cx)[kRtPts], float (&sy)[kRtPts], float (&cy)[kRtPts]) {
#pragma unroll
  for (int j = 0; j < kRtPts; ++j) {
    kahan(sx[j], cx[j], __fadd_rn(ax[j].x, ax[j].y));
    kahan(sy[j], cy[j], __fadd_rn(ay[j].x, ay[j].y));
  }
}

// Staged pairs [ka, kb), every subhalo of them far from the whole CTA and
// served by the series to y^K (a pair that straddles two degrees takes the
// larger): two pairs per step, kRtFoldPairs pairs summed plainly per fold.
template <int K>
__device__ __forceinline__ void rt_far_run(const RtSmem& sm, int ka, int kb, const float2 (&X)[kRtPts],
                                           const float2 (&Y)[kRtPts], float (&sx)[kRtPts], float (&cx)[kRtPts],
                                           float (&sy)[kRtPts], float (&cy)[kRtPts]) {
  for (int k = ka; k < kb;) {
    const int kend = min(kb, k + kRtFoldPairs);
    float2 ax[kRtPts], ay[kRtPts];
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) ax[j] = ay[j] = f2(0.f);
    for (; k + 1 < kend; k += 2) rt_far4<K>(sm, k, X, Y, ax, ay);
    if (k < kend) {
      rt_far2<K>(sm, k, X, Y, ax, ay);
      ++k;
    }
    fold(ax, ay, sx, cx, sy, cy);
  }
}

// Deflection of the staged subhalos at the thread's kRtPts points (x[j],
// y[j]), added to the Kahan sums (sx, cx), (sy, cy) of each point. The
// subhalos far from the whole CTA come first, in runs of one series degree
// (rt_far_run); the rest in blocks of kRtFold subhalos. Each block is summed
// plainly in two packed lanes and folded into the Kahan sums; the order is
// fixed, so a point's bits do not depend on the other points of its thread.
// Each staged record is read once for all of the thread's points.
template <int PROFILE>
__device__ __forceinline__ void add_subs(const RtSmem& sm, int cnt, const float (&x)[kRtPts],
                                         const float (&y)[kRtPts], float (&sx)[kRtPts], float (&cx)[kRtPts],
                                         float (&sy)[kRtPts], float (&cy)[kRtPts]) {
  float2 X[kRtPts], Y[kRtPts];
#pragma unroll
  for (int j = 0; j < kRtPts; ++j) {
    X[j] = f2(x[j]);
    Y[j] = f2(y[j]);
  }
  int tfar = 0;  // staged subhalos [0, tfar): pairs far from every point of the CTA
  if (PROFILE == LR_PROFILE_TNFW) {
    // the run of pairs whose larger degree is K: [c_{<K} / 2, c_{<=K} / 2)
    // with c the staged counts by degree (both rounded down)
    int c = 0;
#pragma unroll
    for (int di = 0; di < 5; ++di) {
      const int ka = c >> 1;
      c += sm.ndeg[di];
      const int kb = c >> 1;
      if (kb > ka) {
        if (di == 0) rt_far_run<3>(sm, ka, kb, X, Y, sx, cx, sy, cy);
        if (di == 1) rt_far_run<4>(sm, ka, kb, X, Y, sx, cx, sy, cy);
        if (di == 2) rt_far_run<5>(sm, ka, kb, X, Y, sx, cx, sy, cy);
        if (di == 3) rt_far_run<7>(sm, ka, kb, X, Y, sx, cx, sy, cy);
        if (di == 4) rt_far_run<9>(sm, ka, kb, X, Y, sx, cx, sy, cy);
      }
    }
    tfar = c & ~1;
  }
  for (int t0 = tfar; t0 < cnt; t0 += kRtFold) {
    const int t1 = min(cnt, t0 + kRtFold);
    float2 ax[kRtPts], ay[kRtPts];
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) ax[j] = ay[j] = f2(0.f);
    int t = t0;
    if (PROFILE == LR_PROFILE_TNFW) {
      for (; t + 1 < t1; t += 2) {
        {
          const float4* hot = sm.hot[t >> 1];
          const float4 w0 = hot[0], w1 = hot[1], w2 = hot[2];
          float2 q[kSerTerms];
          rt_coeffs<kSerTerms - 1>(hot, q);
          // the series where x^2 reaches its radius, else the packed far-side
          // closed form, and the rare near pairs the general form (which
          // gives the same bits for far pairs)
          const SubRec2 H = rec_from(hot, sm.cold[t >> 1]);
#pragma unroll
          for (int j = 0; j < kRtPts; ++j) {
            const float2 dx = sub2(X[j], make_float2(w0.x, w0.y)), dy = sub2(Y[j], make_float2(w0.z, w0.w));
            const float2 R2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            const float2 x2 = __fmul2_rn(R2, lo2(w1));
            const bool sa = x2.x >= w2.x, sb = x2.y >= w2.y;
            float2 em1;
            float2 m = tnfw_m_far2(H, x2, em1);
            const bool na = !tnfw_is_far_em1(em1.x), nb = !tnfw_is_far_em1(em1.y);
            if (na || nb) {  // rare: one branch for both lanes
              if (na) m.x = tnfw_m(sub_lane(H, 0), R2.x);
              if (nb) m.y = tnfw_m(sub_lane(H, 1), R2.y);
            }
            if (sa || sb) {
              const float2 ms = tnfw_m_series2(hi2(w1), hi2(w2), q, x2);
              if (sa) m.x = ms.x;
              if (sb) m.y = ms.y;
            }
            ax[j] = __ffma2_rn(m, dx, ax[j]);
            ay[j] = __ffma2_rn(m, dy, ay[j]);
          }
        }
      }
    }
    for (; t < t1; ++t) {
      const float4* hot = sm.hot[t >> 1];
      const SubRec h = sub_lane(rec_from(hot, sm.cold[t >> 1]), t & 1);
#pragma unroll
      for (int j = 0; j < kRtPts; ++j) {
        const float dx = __fsub_rn(x[j], h.xh), dy = __fsub_rn(y[j], h.yh);
        const float R2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        const float m = (PROFILE == LR_PROFILE_POINT_MASS) ? pointmass_m(h, R2)
                                                           : tnfw_m_any(h, ser_from(hot, t & 1), R2);
        if (t & 1) {
          ax[j].y = __fmaf_rn(m, dx, ax[j].y);
          ay[j].y = __fmaf_rn(m, dy, ay[j].y);
        } else {
          ax[j].x = __fmaf_rn(m, dx, ax[j].x);
          ay[j].x = __fmaf_rn(m, dy, ay[j].x);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) {
      kahan(sx[j], cx[j], __fadd_rn(ax[j].x, ax[j].y));
      kahan(sy[j], cy[j], __fadd_rn(ay[j].x, ay[j].y));
    }
  }
}

template <int PROFILE>
__device__ __forceinline__ void raytrace_body(const LensConst& L, const GridDev& g, const float2* __restrict__ xi,
                                              int64_t n, const float* __restrict__ sub, int n_sub, int bulk_ok,
                                              float2* __restrict__ beta, float2* __restrict__ alpha_out, int* fault,
                                              int64_t blk, RtSmem& sm) {
  // explicit points: kRtPoints consecutive ones; grid: a 2-D tile, so that
  // the CTA's points are compact (padding points repeat an edge point).
  // Thread t takes the CTA's points t + j kRtThreads (j < kRtPts).
  int64_t i[kRtPts];
  bool valid[kRtPts];
  float px[kRtPts], py[kRtPts], ax[kRtPts], ay[kRtPts];
#pragma unroll
  for (int j = 0; j < kRtPts; ++j) {
    const int w = (int)threadIdx.x + j * kRtThreads;
    int64_t ii;
    if (xi) {
      i[j] = blk * kRtPoints + w;
      valid[j] = i[j] < n;
      ii = valid[j] ? i[j] : (n - 1);
    } else {
      const int tw = (g.W + kRtTile - 1) / kRtTile;
      const int ty = (int)(blk / tw), tx = (int)(blk - (int64_t)ty * tw);
      const int row = ty * kRtTile + w / kRtTile, col = tx * kRtTile + w % kRtTile;
      valid[j] = row < g.H && col < g.W;
      i[j] = (int64_t)row * g.W + col;
      ii = (int64_t)min(row, g.H - 1) * g.W + min(col, g.W - 1);
    }
    const float2 p = xi ? xi[ii] : grid_point(g, ii);
    px[j] = p.x;
    py[j] = p.y;
    sple_alpha(L, p.x, p.y, ax[j], ay[j]);
    // external shear about the origin
    ax[j] = fmaf(L.g1, p.x, fmaf(L.g2, p.y, ax[j]));
    ay[j] = fmaf(L.g2, p.x, fmaf(-L.g1, p.y, ay[j]));
  }

  if (n_sub > 0) {
    // the box of the CTA's points (the padding points repeat an edge point)
    float b0 = px[0], b1 = py[0], b2 = px[0], b3 = py[0];
#pragma unroll
    for (int j = 1; j < kRtPts; ++j) {
      b0 = fminf(b0, px[j]);
      b1 = fminf(b1, py[j]);
      b2 = fmaxf(b2, px[j]);
      b3 = fmaxf(b3, py[j]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      b0 = fminf(b0, __shfl_xor_sync(0xffffffffu, b0, o));
      b1 = fminf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
      b2 = fmaxf(b2, __shfl_xor_sync(0xffffffffu, b2, o));
      b3 = fmaxf(b3, __shfl_xor_sync(0xffffffffu, b3, o));
    }
    if ((threadIdx.x & 31) == 0) {
      float* wb = sm.raw + 4 * (threadIdx.x >> 5);  // the raw records are staged only later
      wb[0] = b0;
      wb[1] = b1;
      wb[2] = b2;
      wb[3] = b3;
    }
    if (threadIdx.x == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      float c0 = sm.raw[0], c1 = sm.raw[1], c2 = sm.raw[2], c3 = sm.raw[3];
      for (int w = 1; w < kRtThreads / 32; ++w) {
        c0 = fminf(c0, sm.raw[4 * w]);
        c1 = fminf(c1, sm.raw[4 * w + 1]);
        c2 = fmaxf(c2, sm.raw[4 * w + 2]);
        c3 = fmaxf(c3, sm.raw[4 * w + 3]);
      }
      sm.box[0] = c0;
      sm.box[1] = c1;
      sm.box[2] = c2;
      sm.box[3] = c3;
    }
    __syncthreads();
    uint32_t phase = 0;
    float sx[kRtPts], cx[kRtPts], sy[kRtPts], cy[kRtPts];
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) sx[j] = cx[j] = sy[j] = cy[j] = 0.f;
    for (int h0 = 0; h0 < n_sub; h0 += kSubChunk) {
      const int cnt = min(kSubChunk, n_sub - h0);
      if (!stage_rt(sub, h0, cnt, PROFILE, sm, phase, bulk_ok != 0, fault)) return;
      add_subs<PROFILE>(sm, cnt, px, py, sx, cx, sy, cy);
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kRtPts; ++j) {
      ax[j] += sx[j] - cx[j];
      ay[j] += sy[j] - cy[j];
    }
  }
#pragma unroll
  for (int j = 0; j < kRtPts; ++j) {
    if (valid[j]) {
      beta[i[j]] = make_float2(px[j] - ax[j], py[j] - ay[j]);
      if (alpha_out) alpha_out[i[j]] = make_float2(ax[j], ay[j]);
    }
  }
}

template <int PROFILE>
__global__ void __launch_bounds__(kRtThreads, 5) raytrace_kernel(const __grid_constant__ LensConst L, GridDev g,
                                                              const float2* __restrict__ xi, int64_t n,
                                                              const float* __restrict__ sub, int n_sub, int bulk_ok,
                                                              float2* __restrict__ beta,
                                                              float2* __restrict__ alpha_out, int* fault) {
  __shared__ __align__(16) RtSmem sm;
  raytrace_body<PROFILE>(L, g, xi, n, sub, n_sub, bulk_ok, beta, alpha_out, fault, blockIdx.x, sm);
}

// The same with the lens read from a device record (lr_lens_prepare); an
// invalid record is reported in the fault word.
template <int PROFILE>
__global__ void __launch_bounds__(kRtThreads, 5) raytrace_rec_kernel(const LensRecord* __restrict__ rec, GridDev g,
                                                                  const float2* __restrict__ xi, int64_t n,
                                                                  const float* __restrict__ sub, int n_sub,
                                                                  int bulk_ok, float2* __restrict__ beta,
                                                                  float2* __restrict__ alpha_out, int* fault) {
  __shared__ __align__(16) RtSmem sm;
  if (rec->status != 0 && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(fault, kFaultBadLens);
  raytrace_body<PROFILE>(rec->L, g, xi, n, sub, n_sub, bulk_ok, beta, alpha_out, fault, blockIdx.x, sm);
}

__global__ void lens_prepare_kernel(const float* __restrict__ theta7, float gamma, LensRecord* __restrict__ rec) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float p[8] = {theta7[0], theta7[1], theta7[2], theta7[3], theta7[4], gamma, theta7[5], theta7[6]};
  LensRecord r;
  r.status = lens_constants(p, &r.L, &r.G);
  if (r.status != 0) {
    // rejected parameters: a lens that deflects nothing, so that every loop
    // over the series coefficients stays within its arrays
    for (int k = 0; k < kMaxSeriesTerms; ++k) r.L.d[k] = r.G.hco[k] = 0.f;
    r.L.x0 = r.L.y0 = r.L.s = r.L.pre = r.L.half_expo = r.L.g1 = r.L.g2 = 0.f;
    r.L.c = r.L.sq = r.L.isq = 1.f;
    r.L.nterms = r.G.nterms = 1;
    r.L.pad_ = r.G.pad_ = 0;
    r.G.e = r.G.f = r.G.dlnpre_dq = r.G.df_dq = r.G.inv2q = r.G.dlnte = 0.f;
  }
  r.pad_[0] = r.pad_[1] = r.pad_[2] = 0;
  *rec = r;
}

__global__ void __launch_bounds__(kRtThreads, 5) raytrace_batched_kernel(const __grid_constant__ Batch<RtP> B,
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

// CTAs of the ray-trace: kRtPoints points each, or one per grid tile.
static int64_t rt_blocks(bool explicit_points, const GridDev& g, int64_t n) {
  if (explicit_points) return (n + kRtPoints - 1) / kRtPoints;
  return (int64_t)((g.W + kRtTile - 1) / kRtTile) * ((g.H + kRtTile - 1) / kRtTile);
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
      tot += rt_blocks(p[b0 + k].xi != nullptr, p[b0 + k].g, p[b0 + k].n);
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
  const int st = lens_constants(f, out, nullptr);
  LR_REQUIRE(st == 0, "lens q = %g too small: the deflection series needs more than %d terms", (double)lens->q,
             kMaxSeriesTerms);
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
  if (need_lens) LR_REQUIRE(has_lens(p), "%s: a lens is required", what);
  LR_REQUIRE(((uintptr_t)p->lens_record & 15u) == 0, "%s: lens_record must be 16-byte aligned", what);
  if (has_lens(p)) {
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
  const auto* rec = static_cast<const LensRecord*>(p->lens_record);
  if (!rec) {
    lr_status st = make_lens_const(p->lens, &L);
    if (st != LR_OK) return st;
  }
  if (p->n == 0) return LR_OK;
  int* fault = fault_ptr();
  LR_REQUIRE(fault != nullptr, "could not resolve the device fault word");
  const GridDev g = p->xy ? GridDev{} : grid_dev(p->grid);
  const int bulk_ok = (((uintptr_t)p->sub & 15u) == 0) ? 1 : 0;
  const unsigned blocks = (unsigned)rt_blocks(p->xy != nullptr, g, p->n);
  const float2* xi = reinterpret_cast<const float2*>(p->xy);
  const int ns = p->n_sub;
  ktimer_begin(LR_KT_RAYTRACE, s);
  if (rec && p->profile == LR_PROFILE_POINT_MASS)
    raytrace_rec_kernel<LR_PROFILE_POINT_MASS><<<blocks, kRtThreads, 0, s>>>(rec, g, xi, p->n, p->sub, ns, bulk_ok,
                                                                             beta, alpha, fault);
  else if (rec)
    raytrace_rec_kernel<LR_PROFILE_TNFW><<<blocks, kRtThreads, 0, s>>>(rec, g, xi, p->n, p->sub, ns, bulk_ok, beta,
                                                                       alpha, fault);
  else if (p->profile == LR_PROFILE_POINT_MASS)
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
  LR_REQUIRE(p->lens_record == nullptr, "batched ray-trace problems take a host lens");
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

extern "C" lr_status lr_grid_points(const lr_grid* grid, float* out, lr_stream stream) {
  LR_REQUIRE(grid != nullptr, "lr_grid_points: grid is NULL");
  LR_REQUIRE(grid->nx >= 0 && grid->ny >= 0 && grid->ss >= 1, "lr_grid_points: invalid grid");
  LR_REQUIRE(out != nullptr || lr::grid_count(*grid) == 0, "lr_grid_points: out is NULL");
  LR_REQUIRE(((uintptr_t)out & 7u) == 0, "lr_grid_points: out must be 8-byte aligned");
  return lr::launch_grid_points(*grid, reinterpret_cast<float2*>(out), lr::as_cuda(stream));
}

extern "C" size_t lr_lens_record_bytes(void) { return sizeof(lr::LensRecord); }

extern "C" lr_status lr_lens_prepare(const float* theta7, float gamma, void* record, lr_stream stream) {
  LR_REQUIRE(theta7 != nullptr && record != nullptr, "lr_lens_prepare: NULL argument");
  LR_REQUIRE(((uintptr_t)theta7 & 3u) == 0 && ((uintptr_t)record & 15u) == 0,
             "lr_lens_prepare: misaligned pointer (theta7: 4 bytes, record: 16 bytes)");
  LR_REQUIRE(gamma > 1.f && gamma < 3.f, "lr_lens_prepare: gamma = %g outside (1, 3)", (double)gamma);
  lr::lens_prepare_kernel<<<1, 32, 0, lr::as_cuda(stream)>>>(theta7, gamma, static_cast<lr::LensRecord*>(record));
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
