// Ray-trace backward (vector-Jacobian product of the deflection sum): given G = dL/dbeta
// for every image-plane point, returns dL/d(x0, y0, q, phi, theta_e, g1, g2)
// of the lens and dL/d(x_h, y_h, kappa_s | theta_pm, theta_s) of every
// subhalo, with dL/dp = -sum_i G_i . dalpha_i/dp (beta = xi - alpha).
//
// The points are cut into tiles, one CTA each, of equal point counts to
// within one image row: explicit points into contiguous index ranges; pixel
// grids into bands of image rows whose tiles split the band's points in
// column-major order (vjp_bands), so that a tile's points are compact and
// far from most subhalos. Below a full wave of the resident CTA slots there
// is a tile per kVjThreads points; above it whole waves, up to kVjWaves
// (vjp_tiles), because tiles inside the subhalo population cost several
// times the average: with more tiles than slots the CTA scheduler balances
// them, and a plan (vjp_plan_kernel, vjp_rank_kernel) launches them
// heaviest first. The CTA stages its
// points and their G in shared memory (kVjChunk at a time; one chunk at the
// usual sizes) and the thread that stages a point also evaluates its lens and
// shear terms. The subhalo sums are split into slots (h, phase): with P
// phases, slot (h, r) sums subhalo h over the staged points j = r (mod P).
// Threads own slots, so a slot's sums need no cross-thread reduction and,
// once the points are staged, a thread sweeps without block barriers. Points
// are staged as packed pairs (2k, 2k + 1), so a slot evaluates two points per
// step in f32x2 arithmetic; slot (h, r) takes the point pairs k = r (mod P).
// P is chosen on the host so that n_sub * P fills the CTA's threads nearly
// evenly. At the end the CTA adds each subhalo's P slot sums in phase order.
// Per-tile partials (FP64 lens terms, Kahan-compensated FP32 slot sums) are
// added in fixed order (the lens terms by tile, the subhalo sums by launch
// position) by a final kernel, so results are deterministic.
//
// tNFW subhalos whose far-field series radius (x >= 8 max(tau, 2)) clears
// the bounding box of all of a tile's points sum by the series of G and of
// x dG/dx (1 rsqrt and two short polynomials per pair) with no per-pair
// test, with as few terms as the box's distance allows (vj_degree). Where
// the tile is also small against its distance from the subhalo (half-
// diagonal within 0.08 of it) and a tile is swept in one phase, the same
// series is summed by its local expansion about the tile's centre
// (vj_expand): the tile's gradient moments are formed once (vj_moments), and
// each such subhalo costs a fixed 36 terms instead of a pass over the points.
// The others take the far-side closed form per pair and the general form for
// the rare near pairs. The subhalos of a tile are ordered by that choice,
// the expansion first and the closed forms last (vj_sort, by the plan or by
// the CTA itself), so that whole warps take one path.
#include <math.h>

#include "host.cuh"
#include "problems.cuh"
#include "tma.cuh"

namespace lr {

constexpr int kVjThreads = 128;
constexpr int kVjWarps = kVjThreads / 32;
constexpr int kVjChunk = 2048;    // points staged in shared memory at once
constexpr int kVjMaxPhases = 8;
constexpr int kVjFold = 32;       // point pairs summed plainly per slot before a Kahan fold
constexpr int kVjMaxOrd = 4096;   // subhalo counts up to which a CTA orders its slots by class (vj_sort)
constexpr int kVjWaves = 8;       // large inputs: tiles per resident CTA slot
constexpr int kVjTilePts = 512;   // ... while every tile keeps at least this many points
constexpr int kVjExpN = kExpN;     // local expansion: terms delta^k conj(delta)^l with k + l <= kVjExpN
constexpr int kVjExpTerms = (kVjExpN + 1) * (kVjExpN + 2) / 2;
constexpr float kVjExpRatio2 = kExpRatio2;  // (tile half-diagonal / distance)^2 up to which it serves (0.08^2)
constexpr int kVjExpFlag = 16;           // class code: series degree | flag, the expansion serves the tile

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct VjSmem {
  float4 pos[kVjChunk / 2];   // point pair k: (x_2k, x_2k+1, y_2k, y_2k+1)
  float4 grad[kVjChunk / 2];  // (G_x, G_x, G_y, G_y) of the same two points
  double lred[kVjWarps][7];
  unsigned short ord[kVjMaxOrd];  // slot subhalo -> subhalo, in the order of vj_sort
  unsigned char deg[kVjMaxOrd];   // class of each subhalo for the tile (vj_class)
  float wbox[kVjWarps][4];        // per-warp bounds of the CTA's points
  float box[4];                   // x_lo, y_lo, x_hi, y_hi of the CTA's points
  float2 wm[3][kVjExpTerms];      // the tile's moments for the local expansion (vj_moments): W, W_x, W_y
};

// The optional plan of a launch (vjp_plan_kernel, vjp_rank_kernel): CTA b
// takes tile perm[b] (the tiles heaviest first), whose subhalos in the
// order of vj_sort are ord[tile n_sub ..]. Both NULL: CTA b takes tile b and
// orders its subhalos itself.
struct VjPlan {
  const int* perm;
  const unsigned short* ord;
};

// One tNFW pair's terms of the four subhalo sums, for two points at once
// (packed f32x2; ix2 = 1/x^2 = theta_s^2 / R^2), without the subhalo's
// constant factors: with dg = d.G and hg = H - 2G (= x dG/dx),
//   sum 0 = G G_x + q dx, sum 1 = G G_y + q dy (q = hg dg / R^2),
//   sum 2 = G dg, sum 3 = hg dg.
// The q terms are kept apart (b0, b1, with hg dg / x^2 in place of q) and
// join sums 0 and 1 with the factor 1/theta_s^2 once per fold; the slot's
// sums are scaled once by (A, A, -4T, A / theta_s) (vj_scale).
__device__ __forceinline__ void vj_accum2(float2 dx, float2 dy, float2 gx, float2 gy, float2 ix2, float2 Gt,
                                          float2 hg, float2& a0, float2& a1, float2& a2, float2& a3, float2& b0,
                                          float2& b1) {
  const float2 dg = __ffma2_rn(dx, gx, __fmul2_rn(dy, gy));
  const float2 q = __fmul2_rn(__fmul2_rn(hg, dg), ix2);
  b0 = __ffma2_rn(q, dx, b0);
  b1 = __ffma2_rn(q, dy, b1);
  a0 = __ffma2_rn(Gt, gx, a0);
  a1 = __ffma2_rn(Gt, gy, a1);
  a2 = __ffma2_rn(Gt, dg, a2);
  a3 = __ffma2_rn(hg, dg, a3);
}

// The constant factors of a tNFW slot's four sums (1 for a point mass, whose
// terms are accumulated whole).
template <int PROFILE>
__device__ __forceinline__ float vj_scale(const SubRec& rec, float2 ex, int v) {
  if (PROFILE != LR_PROFILE_TNFW) return 1.0f;
  return v == 0 || v == 1 ? rec.A : (v == 2 ? -ex.x : __fmul_rn(rec.A, ex.y));
}

__device__ __forceinline__ void vj_kahan(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Sums of one slot over the staged point pairs k = r, r + P, ... < npairs.
// The rare near points of a tNFW step: the general form for the lanes with
// x^2 - 1 < 0.05, and a zero gradient for a point on the subhalo centre (a
// zero gradient makes every term 0; R^2 <= 1e-30 is a near pair for any
// theta_s above 1e-15, since x^2 = R^2 / theta_s^2 < 1.05, so the test lives
// here).
__device__ __forceinline__ void vj_fix_near(const SubRec& rec, float2 R2, float2 em1, float2& gx, float2& gy,
                                            float2& Gt, float2& Ht, float2& ix2) {
  const bool na = !tnfw_is_far_em1(em1.x), nb = !tnfw_is_far_em1(em1.y);
  if (na || nb) {  // rare: one branch for both lanes
    if (na) tnfw_GH(rec, R2.x, Gt.x, Ht.x, ix2.x);
    if (nb) tnfw_GH(rec, R2.y, Gt.y, Ht.y, ix2.y);
    gx = make_float2(R2.x > 1e-30f ? gx.x : 0.f, R2.y > 1e-30f ? gx.y : 0.f);
    gy = make_float2(R2.x > 1e-30f ? gy.x : 0.f, R2.y > 1e-30f ? gy.y : 0.f);
  }
}

// The far field of a tNFW subhalo for the gradient: with y = 1/x and the
// deflection's series G = y^2 Q(y), Q = q0 + sum_{j>=2} q_j y^j (prep_series),
//   hg = x dG/dx = -y^2 (2 Q + y Q'(y)) = y^2 (s0 + sum_{j>=2} s_j y^j),
//   s0 = -2 q0, s_j = -(j + 2) q_j.
// The terms up to y^K serve from x = r_K max(tau, 2) on:
//   K = 7 from r = 8, K = 5 from 18, K = 4 from 32, K = 3 from 80.
// Against the closed form in extended precision both G and hg are then
// within 1.4e-8 relative for tau in [0.5, 30] (the truncated terms fall as
// (tau / x)^(K + 1)), a quarter of the FP32 unit roundoff.
template <int K>
struct VjSer {
  float2 q0, s0;
  float2 q[K - 1], s[K - 1];  // index j - 2, j = 2 .. K
};

template <int K>
__device__ __forceinline__ VjSer<K> vj_series_coeffs(const SubSer& c) {
  VjSer<K> v;
  v.q0 = f2(c.q[0]);
  v.s0 = f2(-2.0f * c.q[0]);
#pragma unroll
  for (int j = 2; j <= K; ++j) {
    v.q[j - 2] = f2(c.q[j]);
    v.s[j - 2] = f2(-(float)(j + 2) * c.q[j]);
  }
  return v;
}

// The series degree K that serves every pair of a subhalo with points at
// x^2 >= x2min (m = max(tau^2, 4)); 0 where x is below 8 max(tau, 2).
__device__ __forceinline__ int vj_degree(float x2min, float m) {
  return x2min >= 6400.0f * m ? 3 : x2min >= 1024.0f * m ? 4 : x2min >= 324.0f * m ? 5 : x2min >= 64.0f * m ? 7 : 0;
}

// G, hg and 1/x^2 = y^2 of two points by the series of degree K.
template <int K>
__device__ __forceinline__ void vj_series2(const VjSer<K>& c, float2 x2, float2& Gt, float2& hg, float2& ix2) {
  const float2 y = frsqrt2(x2), y2 = __fmul2_rn(y, y);
  float2 r = c.q[K - 2], t = c.s[K - 2];
#pragma unroll
  for (int j = K - 3; j >= 0; --j) {
    r = __ffma2_rn(r, y, c.q[j]);
    t = __ffma2_rn(t, y, c.s[j]);
  }
  Gt = __fmul2_rn(y2, __ffma2_rn(r, y2, c.q0));
  hg = __fmul2_rn(y2, __ffma2_rn(t, y2, c.s0));
  ix2 = y2;
}

// K > 0: every staged point of the CTA is at or beyond the radius of the
// gradient's series of degree K (tNFW only), so that series serves every
// pair without a test; K = 0: the closed forms. P1: one phase (P = 1), so
// that consecutive steps read neighbouring point pairs.
template <int PROFILE, int K, bool P1>
__device__ __forceinline__ void vj_sweep(const SubRec& rec, float2 ex, const SubSer& q,
                                         const float4* __restrict__ pos, const float4* __restrict__ grad, int npairs,
                                         int r, int Pr, float* s, float* c) {
  const int P = P1 ? 1 : Pr;  // the slot's stride over the point pairs
  const SubRec2 H = sub_pair(rec, rec);
  constexpr bool kSeries = PROFILE == LR_PROFILE_TNFW && K > 0;
  const VjSer<kSeries ? K : 3> ser = vj_series_coeffs<kSeries ? K : 3>(q);
  for (int k = r; k < npairs;) {
    const int kend = min(npairs, k + P * kVjFold);
    float2 a0 = f2(0.f), a1 = f2(0.f), a2 = f2(0.f), a3 = f2(0.f), b0 = f2(0.f), b1 = f2(0.f);
    if constexpr (kSeries) {
      for (; k + P < kend; k += 2 * P) {
        float2 dx[2], dy[2], gx[2], gy[2], Gt[2], hg[2], ix2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float4 Q = pos[k + u * P], D = grad[k + u * P];
          dx[u] = sub2(make_float2(Q.x, Q.y), H.xh);
          dy[u] = sub2(make_float2(Q.z, Q.w), H.yh);
          gx[u] = make_float2(D.x, D.y);
          gy[u] = make_float2(D.z, D.w);
          const float2 R2 = __ffma2_rn(dx[u], dx[u], __fmul2_rn(dy[u], dy[u]));
          vj_series2(ser, __fmul2_rn(R2, H.its2), Gt[u], hg[u], ix2[u]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
          vj_accum2(dx[u], dy[u], gx[u], gy[u], ix2[u], Gt[u], hg[u], a0, a1, a2, a3, b0, b1);
      }
      if (k < kend) {
        const float4 Q = pos[k], D = grad[k];
        const float2 dx = sub2(make_float2(Q.x, Q.y), H.xh), dy = sub2(make_float2(Q.z, Q.w), H.yh);
        const float2 R2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
        float2 Gt, hg, ix2;
        vj_series2(ser, __fmul2_rn(R2, H.its2), Gt, hg, ix2);
        vj_accum2(dx, dy, make_float2(D.x, D.y), make_float2(D.z, D.w), ix2, Gt, hg, a0, a1, a2, a3, b0, b1);
        k += P;
      }
    } else if (PROFILE == LR_PROFILE_TNFW) {
      // two steps at a time: both far-side forms first (independent chains
      // that can interleave), then the near fixes and the sums in step order
      for (; k + P < kend; k += 2 * P) {
        float2 dx[2], dy[2], gx[2], gy[2], R2[2], Gt[2], Ht[2], ix2[2], em1[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float4 Q = pos[k + u * P], D = grad[k + u * P];
          dx[u] = sub2(make_float2(Q.x, Q.y), H.xh);
          dy[u] = sub2(make_float2(Q.z, Q.w), H.yh);
          gx[u] = make_float2(D.x, D.y);
          gy[u] = make_float2(D.z, D.w);
          R2[u] = __ffma2_rn(dx[u], dx[u], __fmul2_rn(dy[u], dy[u]));
          tnfw_GH_far2(H, __fmul2_rn(R2[u], H.its2), Gt[u], Ht[u], ix2[u], em1[u]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          vj_fix_near(rec, R2[u], em1[u], gx[u], gy[u], Gt[u], Ht[u], ix2[u]);
          vj_accum2(dx[u], dy[u], gx[u], gy[u], ix2[u], Gt[u], __ffma2_rn(f2(-2.0f), Gt[u], Ht[u]), a0, a1, a2, a3,
                    b0, b1);
        }
      }
    }
    for (; k < kend; k += P) {
      const float4 Q = pos[k], D = grad[k];
      const float2 dx = sub2(make_float2(Q.x, Q.y), H.xh), dy = sub2(make_float2(Q.z, Q.w), H.yh);
      float2 gx = make_float2(D.x, D.y), gy = make_float2(D.z, D.w);
      const float2 R2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
      if (PROFILE == LR_PROFILE_TNFW) {
        // the far-side form for both points; the rare near ones are redone
        // by the general form (the same bits where both apply)
        float2 Gt, Ht, ix2, em1;
        tnfw_GH_far2(H, __fmul2_rn(R2, H.its2), Gt, Ht, ix2, em1);
        vj_fix_near(rec, R2, em1, gx, gy, Gt, Ht, ix2);
        vj_accum2(dx, dy, gx, gy, ix2, Gt, __ffma2_rn(f2(-2.0f), Gt, Ht), a0, a1, a2, a3, b0, b1);
      } else {
        // point mass: alpha = theta^2 d / R^2 (its2 = theta^2, ex.y = theta)
        float2 iR2 = make_float2(R2.x > 1e-30f ? frcp(R2.x) : 0.f, R2.y > 1e-30f ? frcp(R2.y) : 0.f);
        const float2 dg = __ffma2_rn(dx, gx, __fmul2_rn(dy, gy));
        const float2 m = __fmul2_rn(H.its2, iR2);
        const float2 q = __fmul2_rn(__fmul2_rn(f2(-2.0f), dg), iR2);
        a0 = __ffma2_rn(m, __ffma2_rn(q, dx, gx), a0);
        a1 = __ffma2_rn(m, __ffma2_rn(q, dy, gy), a1);
        a2 = __ffma2_rn(f2(-2.0f * ex.y), __fmul2_rn(dg, iR2), a2);
      }
    }
    if (PROFILE == LR_PROFILE_TNFW) {
      a0.x = __fmaf_rn(rec.its2, __fadd_rn(b0.x, b0.y), a0.x);
      a1.x = __fmaf_rn(rec.its2, __fadd_rn(b1.x, b1.y), a1.x);
    }
    vj_kahan(s[0], c[0], __fadd_rn(a0.x, a0.y));
    vj_kahan(s[1], c[1], __fadd_rn(a1.x, a1.y));
    vj_kahan(s[2], c[2], __fadd_rn(a2.x, a2.y));
    vj_kahan(s[3], c[3], __fadd_rn(a3.x, a3.y));
  }
}

// The series degree (vj_degree) that serves every point of the box (x_lo,
// y_lo, x_hi, y_hi): x^2 of the box's nearest point. 0 where the deflection's
// series is not in use for the subhalo.
__device__ __forceinline__ int vj_degree_box(const SubRec& h, const SubSer& q, const float* box) {
  if (isinf(q.xT2)) return 0;
  const float dx = fmaxf(fmaxf(box[0] - h.xh, h.xh - box[2]), 0.f);
  const float dy = fmaxf(fmaxf(box[1] - h.yh, h.yh - box[3]), 0.f);
  return vj_degree(__fmul_rn(fmaf(dx, dx, dy * dy), h.its2), fmaxf(h.tau2, 4.0f));
}

// ---------------------------------------------------------------------------
// Local expansion of a far subhalo's deflection about a tile's centre.
//
// With z = xi - xi_h as a complex number, the far-field series gives
//   alpha(z) = A sum_j q_j theta_s^(j+2) |z|^-(j+2) z
//            = A theta_s^2 sum_j q_j (theta_s / |c|)^j conj(c)^-1
//              (1 + delta/c)^(-j/2) (1 + conj(delta)/conj(c))^(-(j+2)/2)
// about the tile's centre, z = c + delta. The binomial series of the two
// factors converge for |delta| < |c|; truncated at k + l <= kVjExpN they
// give alpha as a polynomial in delta and conj(delta) whose coefficients
// depend on the subhalo alone:
//   alpha(c + delta) = A theta_s^2 sum_{k,l} c_kl u^k conj(u)^(l+1) delta^k conj(delta)^l,
//   c_kl = sum_j q_j (theta_s / |c|)^j C(-j/2, k) C(-(j+2)/2, l), u = 1/c.
// The four gradient sums over the tile's points then need only the tile's
// moments W_kl = sum_i conj(G_i) delta_i^k conj(delta_i)^l (vj_moments):
//   sum_i G_i . alpha_i = Re sum_kl M_kl W_kl, with M_kl the coefficients,
//   and d/dxi_x, d/dxi_y of delta^k conj(delta)^l give the moments
//   W_x = k W_(k-1,l) + l W_(k,l-1), W_y = i (k W_(k-1,l) - l W_(k,l-1)).
// The order of the truncation follows the ratio of the tile's half-diagonal
// to |c|: 4 up to 0.01, 5 up to 0.03, 6 up to 0.05, 7 (kVjExpN) up to 0.08.
// Each keeps the truncation below 5e-9 of the sums of absolute terms
// (checked against the analytic FP64 gradients for theta_s from 0.015 to
// 0.2 arcsec and series degrees 3 to 7).

// Term index of delta^k conj(delta)^l: by total order s = k + l, then k.
__device__ __forceinline__ int vj_term(int k, int l) { return (k + l) * (k + l + 1) / 2 + k; }

// The class of a subhalo for a tile: its series degree (vj_degree_box), with
// kVjExpFlag added where exp_ok and the tile's half-diagonal is within 0.08
// of the distance from its centre.
__device__ __forceinline__ int vj_class(const SubRec& h, const SubSer& q, const float* box, bool exp_ok) {
  const int d = vj_degree_box(h, q, box);
  if (d == 0 || !exp_ok) return d;
  const float hx = 0.5f * (box[2] - box[0]), hy = 0.5f * (box[3] - box[1]);
  const float cx = 0.5f * (box[0] + box[2]) - h.xh, cy = 0.5f * (box[1] + box[3]) - h.yh;
  return fmaf(hx, hx, hy * hy) <= kVjExpRatio2 * fmaf(cx, cx, cy * cy) ? (d | kVjExpFlag) : d;
}

// The tile's moments about cen over its staged points (one chunk of cnt
// points): W into sm.wm[0], W_x into sm.wm[1], W_y into sm.wm[2]. All
// threads of the CTA take part; three threads per term sum a third of the
// points each (Kahan-compensated), and the thirds are added in order.
__device__ __forceinline__ void vj_moments(VjSmem& sm, int cnt, float2 cen) {
  const int t = threadIdx.x;
  if (t < 3 * kVjExpTerms) {
    const int m = t % kVjExpTerms, part = t / kVjExpTerms;
    int s = 0;
    while ((s + 1) * (s + 2) / 2 <= m) ++s;
    const int k = m - s * (s + 1) / 2, l = s - k;
    float2 acc = make_float2(0.f, 0.f), cmp = make_float2(0.f, 0.f);
    for (int i = part; i < cnt; i += 3) {
      const float4 P = sm.pos[i >> 1], D = sm.grad[i >> 1];
      const bool b = i & 1;
      const float2 d = make_float2((b ? P.y : P.x) - cen.x, (b ? P.w : P.z) - cen.y);
      float2 pw = make_float2(1.f, 0.f);
      for (int a = 0; a < k; ++a) pw = c2mul(pw, d);
      for (int a = 0; a < l; ++a) pw = c2mul(pw, make_float2(d.x, -d.y));
      const float2 term = c2mul(make_float2(b ? D.y : D.x, -(b ? D.w : D.z)), pw);
      vj_kahan(acc.x, cmp.x, term.x);
      vj_kahan(acc.y, cmp.y, term.y);
    }
    sm.wm[part][m] = make_float2(acc.x - cmp.x, acc.y - cmp.y);
  }
  __syncthreads();
  if (t < kVjExpTerms) {
    const float2 a = sm.wm[0][t], b = sm.wm[1][t], c = sm.wm[2][t];
    sm.wm[0][t] = make_float2(a.x + b.x + c.x, a.y + b.y + c.y);
  }
  __syncthreads();
  if (t < kVjExpTerms) {
    int s = 0;
    while ((s + 1) * (s + 2) / 2 <= t) ++s;
    const int k = t - s * (s + 1) / 2, l = s - k;
    const float2 wa = k > 0 ? sm.wm[0][vj_term(k - 1, l)] : make_float2(0.f, 0.f);
    const float2 wb = l > 0 ? sm.wm[0][vj_term(k, l - 1)] : make_float2(0.f, 0.f);
    const float fk = (float)k, fl = (float)l;
    sm.wm[1][t] = make_float2(fmaf(fk, wa.x, fl * wb.x), fmaf(fk, wa.y, fl * wb.y));
    // i (k W_(k-1,l) - l W_(k,l-1))
    sm.wm[2][t] = make_float2(-fmaf(fk, wa.y, -fl * wb.y), fmaf(fk, wa.x, -fl * wb.x));
  }
  __syncthreads();
}

// The tile's four subhalo sums by the local expansion: dL/d(x_h, y_h,
// kappa_s, theta_s) of one tNFW subhalo (K: its series degree for the tile),
// from the tile's moments about cen. The term loops stay rolled: unrolled
// inside the sweep's kernel they spill, and a separate (not inlined) unrolled
// function measured slower.
__device__ __forceinline__ float4 vj_expand(const SubRec& rec, const SubSer& q, float kappa, float ts, int K,
                                            float2 cen, float hd2, const VjSmem& sm) {
  const float2 c = make_float2(cen.x - rec.xh, cen.y - rec.yh);
  const float r2 = fmaf(c.x, c.x, c.y * c.y), ir2 = 1.0f / r2;
  // the truncation order for (half-diagonal / |c|)^2 = hd2 / r2
  const int nmax = exp_order(hd2, r2);
  const float2 u = make_float2(c.x * ir2, -c.y * ir2), ub = make_float2(u.x, -u.y);
  const float yc = ts * sqrtf(ir2);
  float qy[8];
  float yj = 1.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    qy[j] = (j == 1 || j > K) ? 0.f : q.q[j] * yj;
    yj *= yc;
  }
  // Q = u^k conj(u)^(l+1) for the terms of total order s = k + l: from
  // conj(u)^(s+1) at k = 0, each step in k times u / conj(u) = conj(c)^2 / |c|^2
  const float2 rot = make_float2((c.x * c.x - c.y * c.y) * ir2, -2.0f * c.x * c.y * ir2);
  float2 us = ub;  // conj(u)^(s+1)
  float L = 0.f, Lt = 0.f, X = 0.f, Y = 0.f;
#pragma unroll 1
  for (int s = 0; s <= nmax; ++s) {
    float2 Q = us;
#pragma unroll 1
    for (int k = 0; k <= s; ++k) {
      const int l = s - k, m = s * (s + 1) / 2 + k;
      float ckl = 0.f, ctl = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j == 1) continue;
        const float w = qy[j] * (kExpBin.a[j][k] * kExpBin.b[j][l]);
        ckl += w;
        ctl = fmaf(w, (float)(j + 2), ctl);
      }
      const float2 W = sm.wm[0][m], Wx = sm.wm[1][m], Wy = sm.wm[2][m];
      const float rw = fmaf(Q.x, W.x, -Q.y * W.y);
      L = fmaf(ckl, rw, L);
      Lt = fmaf(ctl, rw, Lt);
      X = fmaf(ckl, fmaf(Q.x, Wx.x, -Q.y * Wx.y), X);
      Y = fmaf(ckl, fmaf(Q.x, Wy.x, -Q.y * Wy.y), Y);
      Q = c2mul(Q, rot);
    }
    us = c2mul(us, ub);
  }
  const float sc = rec.A * ts * ts;
  return make_float4(sc * X, sc * Y, -sc * L / kappa, -sc * Lt / ts);
}

// The CTA's points: u in [u0, u1) indexes explicit points directly; on a
// pixel grid it indexes the points of the band of rows [row0, row0 + rows)
// in column-major order.
struct VjMap {
  int64_t u0, u1;
  int32_t row0, rows;
};

__device__ __forceinline__ VjMap vj_map(const GridDev& g, bool grid, int64_t n, int bands, int64_t blk,
                                        int64_t nblk) {
  VjMap m;
  if (!grid) {
    m.u0 = blk * n / nblk;
    m.u1 = (blk + 1) * n / nblk;
    m.row0 = m.rows = 0;
    return m;
  }
  const int64_t per = nblk / bands;  // CTAs per band
  const int64_t b = blk / per, c = blk - b * per;
  m.row0 = (int32_t)(b * g.H / bands);
  m.rows = (int32_t)((b + 1) * g.H / bands) - m.row0;
  const int64_t nb = (int64_t)m.rows * g.W;
  m.u0 = c * nb / per;
  m.u1 = (c + 1) * nb / per;
  return m;
}

// Index of the CTA's point u (explicit points: u itself).
__device__ __forceinline__ int64_t vj_index(const GridDev& g, const VjMap& m, bool grid, int64_t u) {
  if (!grid) return u;
  const int32_t col = (int32_t)(u / m.rows);
  const int32_t row = m.row0 + (int32_t)(u - (int64_t)col * m.rows);
  return (int64_t)row * g.W + col;
}

// The bounding box (x_lo, y_lo, x_hi, y_hi) of the tile's points into box,
// by all of the CTA's threads (wbox: per-warp scratch).
__device__ __forceinline__ void vj_box(const GridDev& g, const float2* __restrict__ xi, const VjMap& mp,
                                       float (*wbox)[4], float* box) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float b0 = INFINITY, b1 = INFINITY, b2 = -INFINITY, b3 = -INFINITY;
  for (int64_t u = mp.u0 + tid; u < mp.u1; u += kVjThreads) {
    const float2 p = xi ? xi[u] : grid_point(g, vj_index(g, mp, true, u));
    b0 = fminf(b0, p.x);
    b1 = fminf(b1, p.y);
    b2 = fmaxf(b2, p.x);
    b3 = fmaxf(b3, p.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    b0 = fminf(b0, __shfl_xor_sync(0xffffffffu, b0, o));
    b1 = fminf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
    b2 = fmaxf(b2, __shfl_xor_sync(0xffffffffu, b2, o));
    b3 = fmaxf(b3, __shfl_xor_sync(0xffffffffu, b3, o));
  }
  if (lane == 0) {
    wbox[warp][0] = b0;
    wbox[warp][1] = b1;
    wbox[warp][2] = b2;
    wbox[warp][3] = b3;
  }
  __syncthreads();
  if (tid < 4) {
    float v = wbox[0][tid];
    for (int w = 1; w < kVjWarps; ++w) v = tid < 2 ? fminf(v, wbox[w][tid]) : fmaxf(v, wbox[w][tid]);
    box[tid] = v;
  }
  __syncthreads();
}

// The sort key of a class: every expansion class (any series degree) alike.
__device__ __forceinline__ int vj_cls_key(int c) { return (c & kVjExpFlag) ? kVjExpFlag : c; }

// FP32 lanes per point of a subhalo's sums for a tile of npts points, by its
// class (vj_class): the series of degree K, the closed forms (0), or the
// local expansion (up to about 1,600 lanes per tile): the weight of a tile's
// work.
__device__ __forceinline__ float vj_cost(int cls, int npts) {
  if (cls & kVjExpFlag) return 1600.0f / (float)max(npts, 1);
  return cls ? 20.3f + 2.0f * (float)(cls - 2) : 50.3f;
}

// The tNFW subhalos (n_sub <= kVjMaxOrd) by their class for the tile's box
// (vj_class): those served by the local expansion first, then by the series
// of degree 3, 4, 5, 7, each class in index order, those that need the
// closed forms last: ord[rank] = subhalo (shared or global memory). cls:
// per-subhalo scratch in shared memory. Returns the thread's share of the
// tile's work per point (sum of vj_cost over its subhalos).
__device__ __forceinline__ float vj_sort(const float* __restrict__ sub, int n_sub, const float* box, bool exp_ok,
                                         int npts, unsigned char* cls, unsigned short* ord) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float cost = 0.f;
  for (int h = tid; h < n_sub; h += kVjThreads) {
    const SubRec r = prep_sub(sub + 5 * (int64_t)h, LR_PROFILE_TNFW);
    const int d = vj_class(r, prep_series(r, LR_PROFILE_TNFW), box, exp_ok);
    cls[h] = (unsigned char)d;
    cost += vj_cost(d, npts);
  }
  __syncthreads();
  // stable counting sort by class: the expansion (any series degree), then
  // the series of degree 3, 4, 5, 7, then 0. Warp w takes the
  // subhalos [w q, (w + 1) q), q = n_sub / warps rounded up to 32: it counts
  // its subhalos per class, then scatters them after the classes before
  // theirs and the warps before it.
  constexpr int kClasses = 6;
  const int qn = (n_sub + kVjWarps * 32 - 1) / (kVjWarps * 32) * 32;
  const int h0 = warp * qn, h1 = min(n_sub, h0 + qn);
  __shared__ int wcnt[kVjWarps][kClasses];
#pragma unroll 1
  for (int pass = 0; pass < kClasses; ++pass) {
    const int want = pass == 0 ? kVjExpFlag : (pass < 4 ? 2 + pass : (pass == 4 ? 7 : 0));
    int nc = 0;
    for (int b = h0; b < h1; b += 32)
      nc += __popc(__ballot_sync(0xffffffffu, b + lane < h1 && vj_cls_key(cls[b + lane]) == want));
    if (lane == 0) wcnt[warp][pass] = nc;
  }
  __syncthreads();
  int nf = 0;
#pragma unroll 1
  for (int pass = 0; pass < kClasses; ++pass) {
    const int want = pass == 0 ? kVjExpFlag : (pass < 4 ? 2 + pass : (pass == 4 ? 7 : 0));
    int tot = 0, before = 0;
    for (int w = 0; w < kVjWarps; ++w) {
      tot += wcnt[w][pass];
      if (w < warp) before += wcnt[w][pass];
    }
    int pos = nf + before;
    for (int b = h0; b < h1; b += 32) {
      const bool f = b + lane < h1 && vj_cls_key(cls[b + lane]) == want;
      const unsigned m = __ballot_sync(0xffffffffu, f);
      if (f) ord[pos + __popc(m & ((1u << lane) - 1u))] = (unsigned short)(b + lane);
      pos += __popc(m);
    }
    nf += tot;
  }
  __syncthreads();
  return cost;
}

template <int PROFILE>
__device__ __forceinline__ void vjp_body(const LensConst& L, const LensGradConst& LG, const GridDev& g,
                                         const float2* __restrict__ xi, int64_t n, const float* __restrict__ sub,
                                         int n_sub, int P, int bands, const VjPlan& plan,
                                         const float2* __restrict__ dbeta, double* __restrict__ lens_part,
                                         float* __restrict__ sub_part, float* __restrict__ slot_part, int64_t blk,
                                         int64_t nblk, VjSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool grid = xi == nullptr;
  // the lens partials are indexed by tile, the subhalo and slot partials by
  // launch position: CTAs that run together write neighbouring words
  const int64_t tile = plan.perm ? (int64_t)plan.perm[blk] : blk;
  const VjMap mp = vj_map(g, grid, n, bands, tile, nblk);
  const int64_t p0 = mp.u0, p1 = mp.u1;
  const int nchunks = (int)((p1 - p0 + kVjChunk - 1) / kVjChunk);
  const int slots = n_sub * P;
  const int ngroups = slots > 0 ? (slots + kVjThreads - 1) / kVjThreads : 1;
  float la[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int staged = -1;
  // tNFW: the subhalos in the order of their classes for the tile's box
  // (vj_sort), from the plan or sorted here; more than kVjMaxOrd subhalos:
  // index order. Each slot finds its subhalo's class itself (vj_class). The
  // local expansion needs one phase and one staged chunk.
  const bool ordered = PROFILE == LR_PROFILE_TNFW && n_sub > 0 && n_sub <= kVjMaxOrd;
  const bool exp_ok = ordered && P == 1 && nchunks == 1;
  const unsigned short* ord = plan.ord ? plan.ord + tile * n_sub : sm.ord;
  if (PROFILE == LR_PROFILE_TNFW) {
    vj_box(g, xi, mp, sm.wbox, sm.box);
    if (ordered && !plan.ord) vj_sort(sub, n_sub, sm.box, exp_ok, (int)(p1 - p0), sm.deg, sm.ord);
  }
  const float2 cen = make_float2(0.5f * (sm.box[0] + sm.box[2]), 0.5f * (sm.box[1] + sm.box[3]));
  const float hx = 0.5f * (sm.box[2] - sm.box[0]), hy = 0.5f * (sm.box[3] - sm.box[1]);
  const float hd2 = fmaf(hx, hx, hy * hy);  // the tile's half-diagonal squared

  for (int grp = 0; grp < ngroups; ++grp) {
    const int slot = grp * kVjThreads + tid;
    const bool own = slot < slots;
    const int hs = own ? slot / P : 0;  // the slot's subhalo in the CTA's order
    const int r = own ? slot - hs * P : 0;
    const int h = ordered ? (int)ord[hs] : hs;
    SubRec rec{};
    SubSer q{};
    int deg = 0;  // class for the tile (vj_class): series degree, 0 the closed forms, | kVjExpFlag
    float2 ex = make_float2(0.f, 0.f);  // tNFW: (4T, 1/theta_s); point mass: (0, theta_pm)
    if (own) {
      const float* rr = sub + 5 * (int64_t)h;
      rec = prep_sub(rr, PROFILE);
      if (PROFILE == LR_PROFILE_TNFW) {
        q = prep_series(rec, PROFILE);
        deg = vj_class(rec, q, sm.box, exp_ok);
      }
      if (PROFILE == LR_PROFILE_POINT_MASS) {
        ex = make_float2(0.f, __ldg(rr + 2));
      } else {
        const float tau = __ldg(rr + 4), t2 = tau * tau;
        ex = make_float2(4.0f * t2 / ((t2 + 1.0f) * (t2 + 1.0f)), 1.0f / __ldg(rr + 3));
      }
    }
    float sc[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ch = 0; ch < nchunks; ++ch) {
      const int64_t c0 = p0 + (int64_t)ch * kVjChunk;
      const int cnt = (int)min((int64_t)kVjChunk, p1 - c0);
      if (ch != staged) {  // uniform over the CTA
        __syncthreads();   // the previous chunk's readers are done
        for (int k = tid; k < cnt; k += kVjThreads) {
          const int64_t i = vj_index(g, mp, grid, c0 + k);
          const float2 p = xi ? xi[i] : grid_point(g, i);
          const float2 d = dbeta[i];
          if (grp == 0) {  // each chunk is staged once in group 0: the point's lens and shear terms
            float o5[5];
            sple_vjp(L, LG, p.x, p.y, d.x, d.y, o5);
#pragma unroll
            for (int t = 0; t < 5; ++t) la[t] += o5[t];
            la[5] -= fmaf(d.x, p.x, -d.y * p.y);  // dalpha/dg1 = (x, -y)
            la[6] -= fmaf(d.x, p.y, d.y * p.x);   // dalpha/dg2 = (y, x)
          }
          float* ps = reinterpret_cast<float*>(&sm.pos[k >> 1]);
          float* gs = reinterpret_cast<float*>(&sm.grad[k >> 1]);
          const int lane2 = k & 1;
          ps[lane2] = p.x;
          ps[2 + lane2] = p.y;
          gs[lane2] = d.x;
          gs[2 + lane2] = d.y;
          if (k == cnt - 1 && lane2 == 0) {  // odd count: a zero-gradient partner at the same position
            ps[1] = p.x;
            ps[3] = p.y;
            gs[1] = 0.f;
            gs[3] = 0.f;
          }
        }
        __syncthreads();
        staged = ch;
        if (exp_ok && grp == 0) vj_moments(sm, cnt, cen);  // uniform over the CTA
      }
      if (own && (deg & kVjExpFlag)) {
        // the local expansion about the tile's centre: the four sums whole
        const float* rr = sub + 5 * (int64_t)h;
        const float kap = __ldg(rr + 2), ts = __ldg(rr + 3);
        const float4 e = vj_expand(rec, q, kap, ts, deg & (kVjExpFlag - 1), cen, hd2, sm);
        sc[0] = e.x;
        sc[1] = e.y;
        sc[2] = e.z;
        sc[3] = e.w;
      } else if (own) {
        const int np = (cnt + 1) >> 1;
        if (P == 1) {
          switch (deg) {
            case 3:
              vj_sweep<PROFILE, 3, true>(rec, ex, q, sm.pos, sm.grad, np, r, 1, sc, cc);
              break;
            case 4:
              vj_sweep<PROFILE, 4, true>(rec, ex, q, sm.pos, sm.grad, np, r, 1, sc, cc);
              break;
            case 5:
              vj_sweep<PROFILE, 5, true>(rec, ex, q, sm.pos, sm.grad, np, r, 1, sc, cc);
              break;
            case 7:
              vj_sweep<PROFILE, 7, true>(rec, ex, q, sm.pos, sm.grad, np, r, 1, sc, cc);
              break;
            default:
              vj_sweep<PROFILE, 0, true>(rec, ex, q, sm.pos, sm.grad, np, r, 1, sc, cc);
          }
        } else {
          switch (deg) {
            case 3:
              vj_sweep<PROFILE, 3, false>(rec, ex, q, sm.pos, sm.grad, np, r, P, sc, cc);
              break;
            case 4:
              vj_sweep<PROFILE, 4, false>(rec, ex, q, sm.pos, sm.grad, np, r, P, sc, cc);
              break;
            case 5:
              vj_sweep<PROFILE, 5, false>(rec, ex, q, sm.pos, sm.grad, np, r, P, sc, cc);
              break;
            case 7:
              vj_sweep<PROFILE, 7, false>(rec, ex, q, sm.pos, sm.grad, np, r, P, sc, cc);
              break;
            default:
              vj_sweep<PROFILE, 0, false>(rec, ex, q, sm.pos, sm.grad, np, r, P, sc, cc);
          }
        }
      }
    }
    if (own) {
      const bool expd = (deg & kVjExpFlag) != 0;  // sc holds the expansion's sums, already scaled
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float x = expd ? sc[v] : __fmul_rn(sc[v] - cc[v], vj_scale<PROFILE>(rec, ex, v));
        if (P == 1)
          sub_part[((int64_t)h * 4 + v) * nblk + blk] = x;  // [value][CTA], h the subhalo itself
        else
          slot_part[(blk * slots + slot) * 4 + v] = x;
      }
    }
  }
  if (P > 1) {
    // each subhalo's P slots in phase order (written by this CTA's threads:
    // visible to the whole CTA after the barrier)
    __syncthreads();
    for (int t = tid; t < 4 * n_sub; t += kVjThreads) {
      const int hh = t >> 2, v = t & 3;  // hh: the CTA's order
      const float* q = slot_part + (blk * slots + (int64_t)hh * P) * 4 + v;
      float a = 0.f, c = 0.f;
      for (int rr = 0; rr < P; ++rr) vj_kahan(a, c, q[4 * rr]);
      const int64_t hreal = ordered ? (int64_t)ord[hh] : (int64_t)hh;
      sub_part[(hreal * 4 + v) * nblk + blk] = a - c;
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
    lens_part[tile * 7 + tid] = v;
  }
}

template <int PROFILE>
__global__ void __launch_bounds__(kVjThreads, 4) raytrace_vjp_kernel(const __grid_constant__ LensConst L,
                                                                  const __grid_constant__ LensGradConst LG, GridDev g,
                                                                  const float2* __restrict__ xi, int64_t n,
                                                                  const float* __restrict__ sub, int n_sub, int P,
                                                                  int bands, const VjPlan plan,
                                                                  const float2* __restrict__ dbeta,
                                                                  double* __restrict__ lens_part,
                                                                  float* __restrict__ sub_part,
                                                                  float* __restrict__ slot_part) {
  __shared__ __align__(16) VjSmem sm;
  vjp_body<PROFILE>(L, LG, g, xi, n, sub, n_sub, P, bands, plan, dbeta, lens_part, sub_part, slot_part,
                    blockIdx.x, gridDim.x, sm);
}

// The same with the lens read from a device record (lr_lens_prepare).
template <int PROFILE>
__global__ void __launch_bounds__(kVjThreads, 4) raytrace_vjp_rec_kernel(const LensRecord* __restrict__ rec, GridDev g,
                                                                      const float2* __restrict__ xi, int64_t n,
                                                                      const float* __restrict__ sub, int n_sub, int P,
                                                                      int bands, const VjPlan plan,
                                                                      const float2* __restrict__ dbeta,
                                                                      double* __restrict__ lens_part,
                                                                      float* __restrict__ sub_part,
                                                                      float* __restrict__ slot_part, int* fault) {
  __shared__ __align__(16) VjSmem sm;
  if (rec->status != 0 && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(fault, kFaultBadLens);
  vjp_body<PROFILE>(rec->L, rec->G, g, xi, n, sub, n_sub, P, bands, plan, dbeta, lens_part, sub_part, slot_part,
                    blockIdx.x, gridDim.x, sm);
}

// The plan of a tNFW launch with more tiles than resident CTA slots: one
// CTA per tile sorts the subhalos by their class for the tile's box
// (vj_sort) into ord, and writes the tile's work (FP32 lanes over its
// point-subhalo pairs, the expansion's per tile) to weight.
__global__ void __launch_bounds__(kVjThreads) vjp_plan_kernel(GridDev g, const float2* __restrict__ xi, int64_t n,
                                                              const float* __restrict__ sub, int n_sub, int P,
                                                              int bands, int64_t ntiles,
                                                              unsigned short* __restrict__ ord,
                                                              float* __restrict__ weight) {
  __shared__ float wbox[kVjWarps][4], box[4], wsum[kVjWarps];
  __shared__ unsigned char cls[kVjMaxOrd];
  const int64_t tile = blockIdx.x;
  const VjMap mp = vj_map(g, xi == nullptr, n, bands, tile, ntiles);
  vj_box(g, xi, mp, wbox, box);
  const int npts = (int)(mp.u1 - mp.u0);
  // the same choice as the sweep's (vjp_body): one phase and one staged chunk
  const bool exp_ok = P == 1 && npts > 0 && npts <= kVjChunk;
  float c = vj_sort(sub, n_sub, box, exp_ok, npts, cls, ord + tile * n_sub);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kVjWarps; ++w) t += wsum[w];
    weight[tile] = t * (float)(mp.u1 - mp.u0);
  }
}

// perm[rank] = tile, the tiles by weight, heaviest first (ties by index):
// one warp per tile counts the heavier tiles. Dynamic shared memory: the
// ntiles weights.
__global__ void __launch_bounds__(128) vjp_rank_kernel(const float* __restrict__ weight, int ntiles,
                                                       int* __restrict__ perm) {
  extern __shared__ float wsh[];
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) wsh[t] = weight[t];
  __syncthreads();
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  const float wt = wsh[t];
  int r = 0;
  for (int u = lane; u < ntiles; u += 32) {
    const float wu = wsh[u];
    r += (wu > wt || (wu == wt && u < t)) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if (lane == 0) perm[r] = t;
}

__global__ void __launch_bounds__(kVjThreads, 4) vjp_batched_kernel(const __grid_constant__ Batch<VjpP> B) {
  __shared__ __align__(16) VjSmem sm;
  const int k = batch_find(B, blockIdx.x);
  const VjpP& P = B.p[k];
  const int64_t blk = blockIdx.x - B.start[k];
  const int64_t nblk = B.start[k + 1] - B.start[k];
  if (P.profile == LR_PROFILE_POINT_MASS)
    vjp_body<LR_PROFILE_POINT_MASS>(P.L, P.LG, P.g, P.xi, P.n, P.sub, P.n_sub, P.phases, P.bands, VjPlan{},
                                    P.dbeta, P.lens_part, P.sub_part, P.slot_part, blk, nblk, sm);
  else
    vjp_body<LR_PROFILE_TNFW>(P.L, P.LG, P.g, P.xi, P.n, P.sub, P.n_sub, P.phases, P.bands, VjPlan{}, P.dbeta,
                              P.lens_part, P.sub_part, P.slot_part, blk, nblk, sm);
}

// Resident CTA slots of the VJP kernels on the current device.
static int64_t vjp_slots() {
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
  return slots[dev];
}

// Tiles (one CTA each) of the VJP for n points: one per kVjThreads points
// below a full wave of the resident slots; above it whole waves, up to
// kVjWaves of them while every tile keeps kVjTilePts points, so that the
// CTA scheduler can balance tiles of uneven work (a plan launches them
// heaviest first).
int64_t vjp_tiles(int64_t n) {
  if (n <= 0) return 0;
  const int64_t slots = vjp_slots();
  const int64_t nb = (n + kVjThreads - 1) / kVjThreads;
  if (nb < slots) return nb;
  int64_t w = n / (slots * kVjTilePts);
  w = w < 1 ? 1 : (w > kVjWaves ? kVjWaves : w);
  return w * slots;
}

// Whether the workspace holds a plan: subhalos that a CTA can order (at most
// kVjMaxOrd), more than one wave of tiles, and their weights within the
// rank kernel's shared memory.
static bool plan_fits(int64_t ntiles, int32_t n_sub) {
  return n_sub > 0 && n_sub <= kVjMaxOrd && ntiles > vjp_slots() && ntiles <= 12288;
}

// Whether a launch over ntiles tiles takes a plan: tNFW subhalos and a
// workspace that holds it.
static bool vjp_planned(int64_t ntiles, const lr_points* p) {
  return p->profile == LR_PROFILE_TNFW && plan_fits(ntiles, p->n_sub);
}

// Phases P of the subhalo sums: 1 when n_sub slots waste at most 5 % of the
// last group of kVjThreads (one phase sweeps with a constant stride and
// allows the local expansion), else the P in [1, kVjMaxPhases] whose slot
// count n_sub P wastes the fewest threads of the last group (the smallest
// such P), keeping at least 128 points per slot.
int vjp_phases(int64_t n, int32_t n_sub) {
  if (n_sub <= 0 || n <= 0) return 1;
  const int64_t per_cta = (n + vjp_tiles(n) - 1) / vjp_tiles(n);
  const int64_t pad1 = ((int64_t)n_sub + kVjThreads - 1) / kVjThreads * kVjThreads;
  if ((double)pad1 <= 1.05 * (double)n_sub) return 1;
  int best = 1;
  double best_w = 1e30;
  for (int P = 1; P <= kVjMaxPhases; ++P) {
    if (P > 1 && per_cta / P < 128) break;
    const int64_t sl = (int64_t)n_sub * P;
    const int64_t padded = (sl + kVjThreads - 1) / kVjThreads * kVjThreads;
    const double w = (double)padded / (double)sl;
    if (w < best_w - 1e-9) {
      best_w = w;
      best = P;
    }
  }
  return best;
}

// Bands of image rows for the CTAs of a pixel grid of W x H points: the
// divisor R of nblk (R <= H) whose tiles, H / R rows by W R / nblk columns,
// are closest to square, preferring bands of equal height; the nblk / R CTAs
// of a band split its points evenly in column-major order. 1 for explicit
// points (unused).
int vjp_bands(int64_t nblk, const lr_points* p) {
  if (p->xy || nblk <= 0) return 1;
  const GridDev g = grid_dev(p->grid);
  int best = 1;
  double best_s = 1e300;
  for (int64_t R = 1; R <= nblk && R <= g.H; ++R) {
    if (nblk % R) continue;
    const double th = (double)g.H / (double)R, tw = (double)g.W * (double)R / (double)nblk;
    const double uneven = (double)((g.H + R - 1) / R) / th - 1.0;
    const double sc = fabs(log(th / tw)) + 2.0 * uneven;
    if (sc < best_s) {
      best_s = sc;
      best = (int)R;
    }
  }
  return best;
}

// Fixed-order sum of the per-CTA partials: one warp per output value
// (7 lens values, then 4 per subhalo); lane l sums CTAs l, l + 32, ... (the
// subhalo partials are stored [value][CTA], so the warp reads contiguous
// memory); the warp reduces by xor-shuffle.
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
    // the lane's share in FP32 with Kahan compensation (FP64 arithmetic is
    // slow on this GPU), the lanes in FP64
    const float* q = sub_part + (int64_t)(o - 7) * nblk;
    float fs = 0.f, fc = 0.f;
    for (int b = lane; b < nblk; b += 32) vj_kahan(fs, fc, q[b]);
    s = (double)fs - (double)fc;
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
      tot += vjp_tiles(p[b0 + k].n);
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
  LR_REQUIRE(lens != nullptr, "lens is NULL");
  const int st = lens_constants(&lens->x0, nullptr, out);
  LR_REQUIRE(st == 0, "lens q = %g outside its domain or too small for the gradient series", (double)lens->q);
  return LR_OK;
}

// Workspace: per-tile lens partials [tile][7] (FP64), subhalo partials
// [4 n_sub][CTA], with P > 1 the slot sums [CTA][n_sub P][4], and where a
// plan fits (plan_fits) its subhalo orders [tile][n_sub] (16 bit), tile
// weights and the permutation of the tiles.
struct VjWs {
  double* lens_part;
  float* sub_part;
  float* slot_part;
  unsigned short* ord;
  float* weight;
  int* perm;
  size_t bytes;
};

static VjWs vjp_ws_layout(void* ws, int64_t n, int32_t n_sub) {
  const int64_t nt = vjp_tiles(n);
  const int P = vjp_phases(n, n_sub);
  const bool plan = plan_fits(nt, n_sub);
  const size_t b_lens = align256(sizeof(double) * 7 * (size_t)nt);
  const size_t b_sub = align256(sizeof(float) * 4 * (size_t)n_sub * (size_t)nt);
  const size_t b_slot = P > 1 ? align256(sizeof(float) * 4 * (size_t)n_sub * P * (size_t)nt) : 0;
  const size_t b_ord = plan ? align256(sizeof(unsigned short) * (size_t)n_sub * (size_t)nt) : 0;
  const size_t b_w = plan ? align256(sizeof(float) * (size_t)nt) : 0;
  const size_t b_perm = plan ? align256(sizeof(int) * (size_t)nt) : 0;
  char* c = static_cast<char*>(ws);
  size_t off = 0;
  auto at = [&](size_t bytes) -> char* {
    char* r = (c && bytes) ? c + off : nullptr;
    off += bytes;
    return r;
  };
  VjWs w;
  w.lens_part = reinterpret_cast<double*>(at(b_lens));
  w.sub_part = reinterpret_cast<float*>(at(b_sub));
  w.slot_part = reinterpret_cast<float*>(at(b_slot));
  w.ord = reinterpret_cast<unsigned short*>(at(b_ord));
  w.weight = reinterpret_cast<float*>(at(b_w));
  w.perm = reinterpret_cast<int*>(at(b_perm));
  w.bytes = off;
  return w;
}

size_t raytrace_vjp_ws(int64_t n, int32_t n_sub) { return vjp_ws_layout(nullptr, n, n_sub).bytes; }

lr_status launch_raytrace_vjp(const lr_points* p, const float2* dbeta, double* d_lens, double* d_sub, void* ws,
                              cudaStream_t s) {
  LensConst L{};
  LensGradConst G{};
  const auto* rec = static_cast<const LensRecord*>(p->lens_record);
  if (!rec) {
    lr_status st = make_lens_const(p->lens, &L);
    if (st != LR_OK) return st;
    st = make_lens_grad_const(p->lens, &G);
    if (st != LR_OK) return st;
  }
  const int64_t nblk = vjp_tiles(p->n);
  if (nblk == 0) {
    if (d_lens) LR_CHECK_CUDA(cudaMemsetAsync(d_lens, 0, 7 * sizeof(double), s));
    if (d_sub && p->n_sub) LR_CHECK_CUDA(cudaMemsetAsync(d_sub, 0, 4 * sizeof(double) * p->n_sub, s));
    return LR_OK;
  }
  const VjWs w = vjp_ws_layout(ws, p->n, p->n_sub);
  double* lens_part = w.lens_part;
  float* sub_part = w.sub_part;
  const GridDev g = p->xy ? GridDev{} : grid_dev(p->grid);
  const float2* xi = reinterpret_cast<const float2*>(p->xy);
  const int P = vjp_phases(p->n, p->n_sub);
  const int bands = vjp_bands(nblk, p);
  int* fault = fault_ptr();
  LR_REQUIRE(fault != nullptr, "could not resolve the device fault word");
  VjPlan plan{};
  if (vjp_planned(nblk, p)) {
    vjp_plan_kernel<<<(unsigned)nblk, kVjThreads, 0, s>>>(g, xi, p->n, p->sub, p->n_sub, P, bands, nblk, w.ord,
                                                          w.weight);
    LR_CHECK_CUDA(cudaGetLastError());
    vjp_rank_kernel<<<(unsigned)((nblk + 3) / 4), 128, sizeof(float) * (size_t)nblk, s>>>(w.weight, (int)nblk,
                                                                                          w.perm);
    LR_CHECK_CUDA(cudaGetLastError());
    plan = VjPlan{w.perm, w.ord};
  }
  ktimer_begin(LR_KT_RAYTRACE_VJP, s);
  if (rec && p->profile == LR_PROFILE_POINT_MASS)
    raytrace_vjp_rec_kernel<LR_PROFILE_POINT_MASS><<<(unsigned)nblk, kVjThreads, 0, s>>>(
        rec, g, xi, p->n, p->sub, p->n_sub, P, bands, plan, dbeta, lens_part, sub_part, w.slot_part, fault);
  else if (rec)
    raytrace_vjp_rec_kernel<LR_PROFILE_TNFW><<<(unsigned)nblk, kVjThreads, 0, s>>>(
        rec, g, xi, p->n, p->sub, p->n_sub, P, bands, plan, dbeta, lens_part, sub_part, w.slot_part, fault);
  else if (p->profile == LR_PROFILE_POINT_MASS)
    raytrace_vjp_kernel<LR_PROFILE_POINT_MASS><<<(unsigned)nblk, kVjThreads, 0, s>>>(
        L, G, g, xi, p->n, p->sub, p->n_sub, P, bands, plan, dbeta, lens_part, sub_part, w.slot_part);
  else
    raytrace_vjp_kernel<LR_PROFILE_TNFW><<<(unsigned)nblk, kVjThreads, 0, s>>>(
        L, G, g, xi, p->n, p->sub, p->n_sub, P, bands, plan, dbeta, lens_part, sub_part, w.slot_part);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_RAYTRACE_VJP, s);
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
  LR_REQUIRE(p->lens_record == nullptr, "batched ray-trace VJP problems take a host lens");
  VjpP v{};
  lr_status st = make_lens_const(p->lens, &v.L);
  if (st != LR_OK) return st;
  st = make_lens_grad_const(p->lens, &v.LG);
  if (st != LR_OK) return st;
  const int64_t nblk = vjp_tiles(p->n);
  v.g = p->xy ? GridDev{} : grid_dev(p->grid);
  v.xi = reinterpret_cast<const float2*>(p->xy);
  v.n = p->n;
  v.sub = p->sub;
  v.n_sub = p->n_sub;
  v.profile = p->profile;
  v.phases = vjp_phases(p->n, p->n_sub);
  v.bands = vjp_bands(nblk, p);
  v.dbeta = dbeta;
  const VjWs w = vjp_ws_layout(ws, p->n, p->n_sub);
  v.lens_part = w.lens_part;
  v.sub_part = w.sub_part;
  v.slot_part = w.slot_part;
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
