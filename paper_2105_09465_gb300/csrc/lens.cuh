// Device-side lens model: SPLE main deflector (series form of the
// hypergeometric deflection), external shear, and truncated-NFW / point-mass
// subhalos, all in FP32. Host-side preparation of the per-lens constants
// lives in raytrace.cu.
#pragma once
#include "common.cuh"

namespace lr {

constexpr int kMaxSeriesTerms = 96;
constexpr float kPi = 3.14159265358979f;

// Per-lens constants, passed by value as a kernel parameter.
//  (u, v) = Rot(phi) (xi - xi0),  R_x = sqrt(q) u,  R_y = v / sqrt(q)
//  alpha' = pre * R^(1-gamma) * F(w) * (R_x + i R_y),  w = e^{2 i phi_e}
//  with pre = theta_e^(gamma-1) 2 sqrt(q)/(1+q) and
//  F(w) = 2F1(1, (gamma-1)/2; (5-gamma)/2; -f w) = sum_n d_n w^n, the factor
//  (-f)^n, f = (1-q)/(1+q), folded into the coefficients d_n.
struct LensConst {
  float x0, y0, c, s;      // centre, cos/sin of the orientation
  float sq, isq;           // sqrt(q), 1/sqrt(q)
  float pre, half_expo;    // prefactor, (1 - gamma)/2 (exponent applied to R^2)
  float g1, g2;            // external shear
  int nterms;              // number of series coefficients in use
  int pad_;
  float d[kMaxSeriesTerms];
};

// Subhalo record after per-CTA preparation (8 floats, 32 B).
//  tNFW: x_h, y_h, 1/theta_s^2, A = 4 kappa_s tau^2/(tau^2+1)^2, tau, tau^2,
//        (tau^2-1)/tau * ln(2)/2, C = tau pi + (tau^2-1) ln tau
//        (the ln(2)/2 turns log2 of x^2/(tau + st)^2 into ln(x/(tau + st)))
//  point mass: x_h, y_h, theta_pm^2, 0...
struct SubRec {
  float xh, yh, its2, A, tau, tau2, t2m1_l, C;
};

// R2^e in FP32 with the exponent product split into an integer part (applied
// exactly by ldexpf) and a remainder of magnitude < ~1.5, so that the
// rounding of e * log2(R2) does not scale with |log2(R2)|.
__device__ __forceinline__ float pow_split(float R2, float e) {
  int k;
  const float m = frexpf(R2, &k);  // R2 = m 2^k, m in [0.5, 1)
  const float kf = (float)k;
  const float lf = log2f(m);       // in [-1, 0)
  const float ek = e * kf;
  const float ek_err = fmaf(e, kf, -ek);
  const float n = rintf(ek);
  const float r = (ek - n) + fmaf(e, lf, ek_err);
  return ldexpf(exp2f(r), (int)n);
}

// SPLE deflection at (x, y).
__device__ __forceinline__ void sple_alpha(const LensConst& L, float x, float y, float& ax, float& ay) {
  const float dx = x - L.x0, dy = y - L.y0;
  const float u = fmaf(L.c, dx, L.s * dy);
  const float v = fmaf(L.c, dy, -L.s * dx);
  const float Rx = L.sq * u, Ry = L.isq * v;
  const float R2 = fmaf(Rx, Rx, Ry * Ry);
  if (!(R2 > 1e-24f)) {  // singular centre (or NaN input): no deflection
    ax = 0.f;
    ay = 0.f;
    return;
  }
  const float inv = 1.0f / R2;
  const float wr = (Rx * Rx - Ry * Ry) * inv;
  const float wi = 2.0f * Rx * Ry * inv;
  // Horner in w = e^{2 i phi_e}
  float Fr = L.d[L.nterms - 1], Fi = 0.f;
  for (int n = L.nterms - 2; n >= 0; --n) {
    const float nr = fmaf(wr, Fr, fmaf(-wi, Fi, L.d[n]));
    const float ni = fmaf(wr, Fi, wi * Fr);
    Fr = nr;
    Fi = ni;
  }
  const float scale = L.pre * pow_split(R2, L.half_expo);
  const float apx = scale * fmaf(Fr, Rx, -Fi * Ry);
  const float apy = scale * fmaf(Fr, Ry, Fi * Rx);
  ax = fmaf(L.c, apx, -L.s * apy);
  ay = fmaf(L.s, apx, L.c * apy);
}

// Fast FP32 helpers for the subhalo terms (hardware reciprocal, reciprocal
// square root and log2; each within a few ulp, far inside the 1e-6 arcsec
// deflection budget of a subhalo whose deflection is at most ~0.1 arcsec).
// The .ftz forms flush subnormal inputs, which none of these arguments are
// (they are squared distances and ratios of order 1e-20 and up), and so skip
// the subnormal handling the non-ftz forms carry.
__device__ __forceinline__ float frsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fsqrt_pos(float x) { return x * frsqrt(x); }  // x > 0
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float frcp(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}
// ln x = log2(x) ln 2
__device__ __forceinline__ float flog(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * 0.69314718055994531f;
}
// ln(x) / 2 = log2(x) ln(2) / 2
constexpr float kHalfLn2 = 0.34657359027997265f;
__device__ __forceinline__ float flg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// arctan(s) / s for s > 0, given is = 1/s. With t = min(s, 1/s) and u = t^2,
// arctan(t) = t P(u), where P is a degree-8 polynomial fitted for this
// library to arctan(sqrt(u))/sqrt(u) on [0, 1] (least squares in the
// monomial basis, iteratively reweighted toward equal relative ripple:
// relative error 1.5e-8 in exact arithmetic, ~2e-7 after FP32 rounding);
// arctan(s) = pi/2 - arctan(1/s) for s > 1.
// Every operation is an explicitly rounded intrinsic (never contracted), so
// atan_over2 below, the same steps on packed f32x2 pairs, gives the same bits.
__device__ constexpr float kAtanP[9] = {2.849667566e-03f, -1.606774889e-02f, 4.269010574e-02f, -7.504177094e-02f,
                             1.064087972e-01f, -1.420363039e-01f, 1.999261826e-01f,  -3.333307207e-01f,
                             1.0f};
constexpr float kHalfPi = 1.57079632679f;

__device__ __forceinline__ float atan_over(float s, float is) {
  const float t = fminf(s, is);
  const float u = __fmul_rn(t, t);
  float p = kAtanP[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) p = __fmaf_rn(p, u, kAtanP[k]);
  const float at = __fmul_rn(t, p);
  return __fmul_rn(s <= 1.0f ? at : __fsub_rn(kHalfPi, at), is);
}

// ---- packed f32x2 forms: each lane rounds exactly as the scalar
// intrinsic it mirrors (a - b is b * (-1) + a with one rounding)
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 frsqrt2(float2 x) { return make_float2(frsqrt(x.x), frsqrt(x.y)); }
__device__ __forceinline__ float2 frcp2(float2 x) { return make_float2(frcp(x.x), frcp(x.y)); }

__device__ __forceinline__ float2 atan_over2(float2 s, float2 is) {
  const float2 t = make_float2(fminf(s.x, is.x), fminf(s.y, is.y));
  const float2 u = __fmul2_rn(t, t);
  float2 p = f2(kAtanP[0]);
#pragma unroll
  for (int k = 1; k < 9; ++k) p = __ffma2_rn(p, u, f2(kAtanP[k]));
  const float2 at = __fmul2_rn(t, p);
  const float2 alt = sub2(f2(kHalfPi), at);
  return __fmul2_rn(make_float2(s.x <= 1.0f ? at.x : alt.x, s.y <= 1.0f ? at.y : alt.y), is);
}

// F(x) of the NFW family as a function of x^2 (x = R / theta_s):
//   arccosh(1/x)/sqrt(1-x^2) for x < 1, arccos(1/x)/sqrt(x^2-1) for x > 1,
// with its series sum_n (-eps)^n/(2n+1), eps = x^2 - 1, near x = 1.
// Also returns s = sqrt(|1 - x^2|).
__device__ __forceinline__ float nfw_F(float x2, float xx, float& s) {
  const float eps = x2 - 1.0f;
  s = fsqrt_pos(fmaxf(fabsf(eps), 1e-30f));
  if (fabsf(eps) < 0.05f) {
    const float m = -eps;
    float p = 1.0f / 15.0f;
    p = fmaf(p, m, 1.0f / 13.0f);
    p = fmaf(p, m, 1.0f / 11.0f);
    p = fmaf(p, m, 1.0f / 9.0f);
    p = fmaf(p, m, 1.0f / 7.0f);
    p = fmaf(p, m, 1.0f / 5.0f);
    p = fmaf(p, m, 1.0f / 3.0f);
    return fmaf(p, m, 1.0f);
  }
  const float is = frcp(s);
  if (eps < 0.f) return flog((1.0f + s) * frcp(xx)) * is;  // arccosh(1/x) = ln((1 + s)/x)
  return atan_over(s, is);                                 // arccos(1/x) = arctan(s)
}

// Truncated-NFW deflection per unit offset: alpha = m * (dx, dy) with
// m = A * B(x)/x^2 where B is the bracket of the enclosed-mass function.
// For x < 0.5 the bracket is evaluated in a rearranged form whose terms are
// all O(x^2) (the direct form cancels catastrophically as x -> 0):
//   B/x^2 = -pi/(tau+st) + 2F + (tau^2-1) [F/(1+s) + log1p(dl)/x^2 + L/(tau (tau+st))],
//   dl = -x^2 [tau/(1+s) + 1/(tau+st)]/(tau+st),  st = sqrt(tau^2+x^2),
// otherwise B = (tau^2-1+2x^2) F + C + st (-pi + (tau^2-1)/tau L).
__device__ __forceinline__ float tnfw_m_far(const SubRec& h, float x2);
__device__ __forceinline__ bool tnfw_is_far(float x2);

__device__ __forceinline__ float tnfw_m(const SubRec& h, float R2) {
  const float x2 = __fmul_rn(R2, h.its2);
  if (tnfw_is_far(x2)) return tnfw_m_far(h, x2);
  if (!(x2 > 1e-20f)) return 0.f;
  const float xx = fsqrt_pos(x2);
  float s;
  const float F = nfw_F(x2, xx, s);
  const float st = fsqrt_pos(h.tau2 + x2);
  const float tp = h.tau + st;
  const float itp = frcp(tp);
  const float l2 = flg2(xx * itp);  // ln(x/(tau + st)) = l2 ln 2
  float G;
  if (x2 < 0.25f) {
    const float L = l2 * 0.69314718055994531f;
    const float is1 = frcp(1.0f + s);
    const float dlx2 = -fmaf(h.tau, is1, itp) * itp;
    const float dl = dlx2 * x2;
    const float ratio = (dl != 0.f) ? fdiv(log1pf(dl), dl) : 1.0f;
    const float t2m1 = h.tau2 - 1.0f;
    G = fmaf(t2m1, fmaf(F, is1, fmaf(dlx2, ratio, __fmul_rn(__fmul_rn(L, frcp(h.tau)), itp))),
             fmaf(2.0f, F, __fmul_rn(-kPi, itp)));
  } else {
    const float t2m1 = h.tau2 - 1.0f;
    const float B = fmaf(st, fmaf(2.0f * h.t2m1_l, l2, -kPi), fmaf(fmaf(2.0f, x2, t2m1), F, h.C));
    G = B * frcp(x2);
  }
  return h.A * G;
}

// Point mass: alpha = theta_pm^2 (dx, dy) / R^2.
__device__ __forceinline__ float pointmass_m(const SubRec& h, float R2) {
  return (R2 > 1e-30f) ? h.its2 * frcp(R2) : 0.f;
}

// The far side of the tNFW profile, x^2 - 1 >= 0.05 (arccos form of F,
// direct bracket), as straight-line code so that several pairs can be
// interleaved. tnfw_m and tnfw_GH return exactly these values for far x^2
// (they call the same code), so a pair gives the same bits on either path.
// Other x^2 give a finite value (the packed *2 forms: any value, NaN for
// x^2 < 1) that the caller replaces.
//
// Four MUFU operations per pair: one reciprocal square root gives both
// s = sqrt(eps) and 1/s (and 1/eps = (1/s)^2), one gives st = sqrt(tau^2 + x^2)
// and 1/st, one reciprocal of x^2 (tau + st) gives both 1/(tau + st) and
// 1/x^2, and ln(x/(tau + st)) = log2(x^2/(tau + st)^2) ln(2)/2 needs no
// sqrt(x^2) (L holds the log2; the record's (tau^2-1)/tau carries ln(2)/2).
// Valid while x^2 (tau + st) stays finite in FP32 (x^2 < ~1e24).
__device__ __forceinline__ bool tnfw_is_far_em1(float em1) { return em1 >= 0.05f; }
__device__ __forceinline__ bool tnfw_is_far(float x2) { return tnfw_is_far_em1(__fadd_rn(x2, -1.0f)); }

// Every step below is an explicitly rounded intrinsic, and the *2 forms
// repeat the same steps on packed f32x2 pairs, so a pair gives the same bits
// whether it is evaluated alone or packed with another. x2 must itself come
// from __fmul_rn (not a contractible product).
struct TnfwFar {
  float F, is, st, ist, ix2, L;
};

__device__ __forceinline__ TnfwFar tnfw_far_terms(const SubRec& h, float x2) {
  TnfwFar t;
  const float eps = fmaxf(__fadd_rn(x2, -1.0f), 0.05f);
  t.is = frsqrt(eps);
  const float s = __fmul_rn(eps, t.is);
  t.F = atan_over(s, t.is);
  const float u = __fadd_rn(h.tau2, x2);
  t.ist = frsqrt(u);
  t.st = __fmul_rn(u, t.ist);
  const float tp = __fadd_rn(h.tau, t.st);
  const float r = frcp(__fmul_rn(x2, tp));
  const float itp = __fmul_rn(x2, r);
  t.ix2 = __fmul_rn(tp, r);
  t.L = flg2(__fmul_rn(__fmul_rn(x2, itp), itp));  // log2(x^2/(tau + st)^2)
  return t;
}

__device__ __forceinline__ float tnfw_m_far(const SubRec& h, float x2) {
  const TnfwFar t = tnfw_far_terms(h, x2);
  const float t2m1 = __fadd_rn(h.tau2, -1.0f);
  const float B = __fmaf_rn(t.st, __fmaf_rn(h.t2m1_l, t.L, -kPi),
                            __fmaf_rn(__fmaf_rn(2.0f, x2, t2m1), t.F, h.C));
  return __fmul_rn(h.A, __fmul_rn(B, t.ix2));
}

// Two records (or one record twice) with every field as a packed pair.
struct SubRec2 {
  float2 xh, yh, its2, A, tau, tau2, t2m1_l, C;
};

__device__ __forceinline__ SubRec2 sub_pair(const SubRec& a, const SubRec& b) {
  SubRec2 r;
  r.xh = make_float2(a.xh, b.xh);
  r.yh = make_float2(a.yh, b.yh);
  r.its2 = make_float2(a.its2, b.its2);
  r.A = make_float2(a.A, b.A);
  r.tau = make_float2(a.tau, b.tau);
  r.tau2 = make_float2(a.tau2, b.tau2);
  r.t2m1_l = make_float2(a.t2m1_l, b.t2m1_l);
  r.C = make_float2(a.C, b.C);
  return r;
}

__device__ __forceinline__ SubRec sub_lane(const SubRec2& r, int k) {
  SubRec h;
  h.xh = k ? r.xh.y : r.xh.x;
  h.yh = k ? r.yh.y : r.yh.x;
  h.its2 = k ? r.its2.y : r.its2.x;
  h.A = k ? r.A.y : r.A.x;
  h.tau = k ? r.tau.y : r.tau.x;
  h.tau2 = k ? r.tau2.y : r.tau2.x;
  h.t2m1_l = k ? r.t2m1_l.y : r.t2m1_l.x;
  h.C = k ? r.C.y : r.C.x;
  return h;
}

struct TnfwFar2 {
  float2 F, is, st, ist, ix2, L, em1;  // em1 = x^2 - 1, the bits tnfw_is_far tests
};

__device__ __forceinline__ TnfwFar2 tnfw_far_terms2(const SubRec2& h, float2 x2) {
  TnfwFar2 t;
  const float2 e = __fadd2_rn(x2, f2(-1.0f));
  t.em1 = e;
  const float2 eps = e;  // no clamp: a near lane's value (NaN for x^2 < 1) is replaced by the caller
  t.is = frsqrt2(eps);
  const float2 s = __fmul2_rn(eps, t.is);
  t.F = atan_over2(s, t.is);
  const float2 u = __fadd2_rn(h.tau2, x2);
  t.ist = frsqrt2(u);
  t.st = __fmul2_rn(u, t.ist);
  const float2 tp = __fadd2_rn(h.tau, t.st);
  const float2 r = frcp2(__fmul2_rn(x2, tp));
  const float2 itp = __fmul2_rn(x2, r);
  t.ix2 = __fmul2_rn(tp, r);
  const float2 a = __fmul2_rn(__fmul2_rn(x2, itp), itp);
  t.L = make_float2(flg2(a.x), flg2(a.y));
  return t;
}

// em1 receives x^2 - 1 (tnfw_is_far_em1 tells the far lanes).
__device__ __forceinline__ float2 tnfw_m_far2(const SubRec2& h, float2 x2, float2& em1) {
  const TnfwFar2 t = tnfw_far_terms2(h, x2);
  em1 = t.em1;
  const float2 t2m1 = __fadd2_rn(h.tau2, f2(-1.0f));
  const float2 B = __ffma2_rn(t.st, __ffma2_rn(h.t2m1_l, t.L, f2(-kPi)),
                              __ffma2_rn(__ffma2_rn(f2(2.0f), x2, t2m1), t.F, h.C));
  return __fmul2_rn(h.A, __fmul2_rn(B, t.ix2));
}

// ---------------------------------------------------------------------------
// Local expansions of a far subhalo's series about a tile's centre (both
// ray-trace kernels): with z = c + delta,
//   |z|^-(j+2) z = |c|^-j conj(c)^-1 (1 + delta/c)^(-j/2) (1 + conj(delta)/conj(c))^(-(j+2)/2),
// whose two binomial series converge for |delta| < |c|.
constexpr int kExpN = 7;  // the highest total order k + l of delta^k conj(delta)^l

// Generalised binomial coefficients C(-j/2, k) and C(-(j+2)/2, k), j < 8.
struct ExpBin {
  float a[8][kExpN + 1];
  float b[8][kExpN + 1];
};

constexpr ExpBin exp_make_bin() {
  ExpBin t{};
  for (int j = 0; j < 8; ++j) {
    double ca = 1.0, cb = 1.0;
    for (int k = 0; k <= kExpN; ++k) {
      t.a[j][k] = (float)ca;
      t.b[j][k] = (float)cb;
      ca *= (-0.5 * j - k) / (k + 1.0);
      cb *= (-0.5 * (j + 2) - k) / (k + 1.0);
    }
  }
  return t;
}

static __constant__ ExpBin kExpBin = exp_make_bin();

__device__ __forceinline__ float2 c2mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// The truncation order of an expansion for (tile half-diagonal / |c|)^2 =
// hd2 / r2: 4 up to a ratio of 0.01, 5 up to 0.03, 6 up to 0.05, 7 up to
// 0.08 (the largest served). Each keeps the truncation below 5e-9 of the
// sums of absolute terms.
constexpr float kExpRatio2 = 0.0064f;
__device__ __forceinline__ int exp_order(float hd2, float r2) {
  return hd2 <= 1e-4f * r2 ? 4 : hd2 <= 9e-4f * r2 ? 5 : hd2 <= 2.5e-3f * r2 ? 6 : kExpN;
}

// Converts a raw subhalo record (5 floats) into the prepared form.
__device__ __forceinline__ SubRec prep_sub(const float* r, int profile) {
  SubRec h;
  h.xh = r[0];
  h.yh = r[1];
  if (profile == LR_PROFILE_POINT_MASS) {
    h.its2 = r[2] * r[2];
    h.A = h.tau = h.tau2 = h.t2m1_l = h.C = 0.f;
  } else {
    const float ks = r[2], ts = r[3], tau = r[4];
    const float t2 = tau * tau;
    h.its2 = 1.0f / (ts * ts);
    h.A = 4.0f * ks * t2 / ((t2 + 1.0f) * (t2 + 1.0f));
    h.tau = tau;
    h.tau2 = t2;
    h.t2m1_l = (t2 - 1.0f) / tau * kHalfLn2;
    h.C = fmaf(t2 - 1.0f, logf(tau), __fmul_rn(tau, kPi));  // explicit rounding: the same in every kernel
  }
  return h;
}

// ---------------------------------------------------------------------------
// Far field of the tNFW profile as a series in y = 1/x.
//
// Expanding the closed form for large x (with ln(x/(tau + sqrt(tau^2 + x^2)))
// = -asinh(tau/x) and arccos(1/x)/sqrt(x^2 - 1) both expanded in 1/x) gives
//   G = B(x)/x^2 = y^2 Q(y),  Q(y) = sum_{j=0}^{9} q_j y^j,
// with T = tau^2 and C the record's constant:
//   q0 = C - T - 1,             q1 = 0,
//   q2 = -(T + 1)^2 / 3,        q3 = pi (T + 1)^2 / 8,
//   q4 = 2 (T^3 - T^2 - 5T - 3) / 15,   q5 = pi (-T^3 + 3T + 2) / 16,
//   q6 = 8 (-T^4 + T^3 - 7T - 5) / 105, q7 = 5 pi (T^4 + 4T + 3) / 128,
//   q8 = 16 (T^5 - T^4 - 9T - 7) / 315, q9 = 7 pi (-T^5 + 5T + 4) / 256.
// For x >= 6 max(tau, 2) the truncation error, measured against the closed
// form in FP64, is below 1e-8 relative; the closed form in FP32 loses more
// than that to the cancellation of its O(x) terms. The forward ray-trace
// takes the series for every pair whose x^2 reaches xT2.
constexpr int kSerTerms = 10;

struct SubSer {
  float xT2;  // x^2 from which the series is used (+inf: never)
  float q[kSerTerms];
};

__device__ __forceinline__ SubSer prep_series(const SubRec& h, int profile) {
  SubSer s;
  const float T = h.tau2, T1 = T + 1.0f, T12 = T1 * T1;
  const float T2 = T * T, T3 = T2 * T, T4 = T3 * T, T5 = T4 * T;
  s.q[0] = h.C - T1;
  s.q[1] = 0.f;
  s.q[2] = -T12 * (1.0f / 3.0f);
  s.q[3] = kPi * T12 * 0.125f;
  s.q[4] = (2.0f / 15.0f) * (T3 - T2 - 5.0f * T - 3.0f);
  s.q[5] = kPi * (-T3 + 3.0f * T + 2.0f) * 0.0625f;
  s.q[6] = (8.0f / 105.0f) * (-T4 + T3 - 7.0f * T - 5.0f);
  s.q[7] = 5.0f * kPi * (T4 + 4.0f * T + 3.0f) * (1.0f / 128.0f);
  s.q[8] = (16.0f / 315.0f) * (T5 - T4 - 9.0f * T - 7.0f);
  s.q[9] = 7.0f * kPi * (-T5 + 5.0f * T + 4.0f) * (1.0f / 256.0f);
  bool ok = profile == LR_PROFILE_TNFW;
#pragma unroll
  for (int j = 0; j < kSerTerms; ++j) ok = ok && isfinite(s.q[j]);
  s.xT2 = ok ? 36.0f * fmaxf(T, 4.0f) : INFINITY;
  return s;
}

// m = A G from the series (x2 >= s.xT2), evaluated as
// Q = q0 + y^2 R(y), R = q2 + y (q3 + ... + y q9) (q1 = 0). Explicitly rounded,
// so the packed form gives the same bits per lane.
__device__ __forceinline__ float tnfw_m_series(const SubRec& h, const SubSer& s, float x2) {
  const float y = frsqrt(x2), y2 = __fmul_rn(y, y);
  float p = s.q[kSerTerms - 1];
#pragma unroll
  for (int j = kSerTerms - 2; j >= 2; --j) p = __fmaf_rn(p, y, s.q[j]);
  return __fmul_rn(h.A, __fmul_rn(y2, __fmaf_rn(p, y2, s.q[0])));
}

// The packed form for two subhalos (or one twice): A, q0 and q[j], j >= 2, as
// pairs (q[0] and q[1] are not read).
__device__ __forceinline__ float2 tnfw_m_series2(float2 A, float2 q0, const float2* q, float2 x2) {
  const float2 y = frsqrt2(x2), y2 = __fmul2_rn(y, y);
  float2 p = q[kSerTerms - 1];
#pragma unroll
  for (int j = kSerTerms - 2; j >= 2; --j) p = __ffma2_rn(p, y, q[j]);
  return __fmul2_rn(A, __fmul2_rn(y2, __ffma2_rn(p, y2, q0)));
}

// The deflection factor of any pair: the series, the far-side closed form
// or the general form, by x^2 (the choice depends on the pair alone).
__device__ __forceinline__ float tnfw_m_any(const SubRec& h, const SubSer& s, float R2) {
  const float x2 = __fmul_rn(R2, h.its2);
  if (x2 >= s.xT2) return tnfw_m_series(h, s, x2);
  return tnfw_m(h, R2);
}

// ---------------------------------------------------------------------------
// Gradients (ray-trace backward). With beta = xi - alpha and G = dL/dbeta,
// dL/dp = -G . dalpha/dp for every lens or subhalo parameter p.

// tNFW brackets: Gt = B(x)/x^2 (alpha = A Gt d, A = 4 kappa_s tau^2/(tau^2+1)^2)
// and Ht = g'(x)/(x T) with T = tau^2/(tau^2+1)^2, from
//   g'(x)/x = T [2F + (tau^2+1)(1-F)/eps - pi/st + (tau^2-1) L/(tau st)],
// eps = x^2 - 1, (1-F)/eps by its series 1/3 - eps/5 + eps^2/7 - ... near x = 1.
// Then dalpha/dxi = A [Gt I + (Ht - 2Gt) n n^T] and
// dalpha/dtheta_s = -A (Ht - 2Gt) d / theta_s.
__device__ __forceinline__ void tnfw_GH_far(const SubRec& h, float x2, float& Gt, float& Ht, float& ix2);

// Also returns ix2 = 1/x^2 (0 at x = 0).
__device__ __forceinline__ void tnfw_GH(const SubRec& h, float R2, float& Gt, float& Ht, float& ix2) {
  const float x2 = __fmul_rn(R2, h.its2);
  if (tnfw_is_far(x2)) {
    tnfw_GH_far(h, x2, Gt, Ht, ix2);
    return;
  }
  if (!(x2 > 1e-20f)) {
    Gt = 0.f;
    Ht = 0.f;
    ix2 = 0.f;
    return;
  }
  ix2 = frcp(x2);
  const float xx = fsqrt_pos(x2);
  float s;
  const float F = nfw_F(x2, xx, s);
  const float st = fsqrt_pos(h.tau2 + x2);
  const float tp = h.tau + st;
  const float itp = frcp(tp);
  const float l2 = flg2(xx * itp);  // ln(x/(tau + st)) = l2 ln 2
  const float lp = fmaf(2.0f * h.t2m1_l, l2, -kPi);
  const float t2m1 = h.tau2 - 1.0f;
  if (x2 < 0.25f) {
    const float L = l2 * 0.69314718055994531f;
    const float is1 = frcp(1.0f + s);
    const float dlx2 = -fmaf(h.tau, is1, itp) * itp;
    const float dl = dlx2 * x2;
    const float ratio = (dl != 0.f) ? fdiv(log1pf(dl), dl) : 1.0f;
    Gt = fmaf(t2m1, fmaf(F, is1, fmaf(dlx2, ratio, __fmul_rn(__fmul_rn(L, frcp(h.tau)), itp))),
              fmaf(2.0f, F, __fmul_rn(-kPi, itp)));
  } else {
    const float B = fmaf(st, lp, fmaf(fmaf(2.0f, x2, t2m1), F, h.C));
    Gt = B * ix2;
  }
  const float eps = x2 - 1.0f;
  float omf;  // (1 - F) / eps
  if (fabsf(eps) < 0.05f) {
    float p = 1.0f / 15.0f;
    p = fmaf(p, -eps, 1.0f / 13.0f);
    p = fmaf(p, -eps, 1.0f / 11.0f);
    p = fmaf(p, -eps, 1.0f / 9.0f);
    p = fmaf(p, -eps, 1.0f / 7.0f);
    p = fmaf(p, -eps, 1.0f / 5.0f);
    omf = fmaf(p, -eps, 1.0f / 3.0f);
  } else {
    omf = (1.0f - F) * frcp(eps);
  }
  const float ist = frcp(st);
  Ht = fmaf(ist, lp, fmaf(2.0f, F, __fmul_rn(h.tau2 + 1.0f, omf)));
}

// tnfw_GH on the far side (see tnfw_m_far), with 1/eps = (1/s)^2.
__device__ __forceinline__ void tnfw_GH_far(const SubRec& h, float x2, float& Gt, float& Ht, float& ix2) {
  const TnfwFar t = tnfw_far_terms(h, x2);
  const float t2m1 = __fadd_rn(h.tau2, -1.0f);
  const float lp = __fmaf_rn(h.t2m1_l, t.L, -kPi);
  const float B = __fmaf_rn(t.st, lp, __fmaf_rn(__fmaf_rn(2.0f, x2, t2m1), t.F, h.C));
  Gt = __fmul_rn(B, t.ix2);
  ix2 = t.ix2;
  // (tau^2 + 1)(1 - F)/eps as c - F c with c = (tau^2 + 1)/eps
  const float c = __fmul_rn(__fmul_rn(t.is, t.is), __fadd_rn(h.tau2, 1.0f));
  Ht = __fmaf_rn(t.ist, lp, __fmaf_rn(2.0f, t.F, __fmaf_rn(-t.F, c, c)));
}

__device__ __forceinline__ void tnfw_GH_far2(const SubRec2& h, float2 x2, float2& Gt, float2& Ht, float2& ix2,
                                             float2& em1) {
  const TnfwFar2 t = tnfw_far_terms2(h, x2);
  em1 = t.em1;
  const float2 t2m1 = __fadd2_rn(h.tau2, f2(-1.0f));
  const float2 lp = __ffma2_rn(h.t2m1_l, t.L, f2(-kPi));
  const float2 B = __ffma2_rn(t.st, lp, __ffma2_rn(__ffma2_rn(f2(2.0f), x2, t2m1), t.F, h.C));
  Gt = __fmul2_rn(B, t.ix2);
  ix2 = t.ix2;
  const float2 c = __fmul2_rn(__fmul2_rn(t.is, t.is), __fadd2_rn(h.tau2, f2(1.0f)));
  Ht = __ffma2_rn(t.ist, lp, __ffma2_rn(f2(2.0f), t.F, __ffma2_rn(make_float2(-t.F.x, -t.F.y), c, c)));
}

// Per-lens constants for the SPLE gradient (host-prepared).
//  h_n = (n+1) c_{n+1} (-f)^n so that W F'(W) = -f W H(W), dF/df = -W H(W).
struct LensGradConst {
  float e;            // (1 - gamma)/2
  float f;            // (1 - q)/(1 + q)
  float dlnpre_dq;    // d ln(pre)/dq = 1/(2q) - 1/(1+q)
  float df_dq;        // -2/(1+q)^2
  float inv2q;        // 1/(2q)
  float dlnte;        // (gamma - 1)/theta_e (0 when theta_e == 0)
  int nterms;
  int pad_;
  float hco[kMaxSeriesTerms];
};

// Both constant sets from the 8 lens parameters (x0, y0, q, phi, theta_e,
// gamma, g1, g2) in FP64, on the host or on the device: returns 0, 1 when a
// parameter is outside its domain or not finite, 2 when q is too small for
// the deflection series (more than kMaxSeriesTerms terms), 3 for the
// gradient series. Either output may be NULL.
__host__ __device__ inline int lens_constants(const float* p, LensConst* Lout, LensGradConst* Gout) {
  for (int k = 0; k < 8; ++k)
    if (!(p[k] == p[k]) || p[k] - p[k] != 0.0f) return 1;  // NaN or infinite
  const double q = p[2], phi = p[3], te = p[4], gam = p[5];
  if (!(q > 0.0 && q <= 1.0) || !(gam > 1.0 && gam < 3.0) || !(te >= 0.0)) return 1;
  const double a = 0.5 * (gam - 1.0), b = 0.5 * (5.0 - gam), fq = (1.0 - q) / (1.0 + q);
  if (Lout) {
    LensConst L;
    for (int k = 0; k < kMaxSeriesTerms; ++k) L.d[k] = 0.f;
    L.x0 = p[0];
    L.y0 = p[1];
    L.c = (float)cos(phi);
    L.s = (float)sin(phi);
    L.sq = (float)sqrt(q);
    L.isq = (float)(1.0 / sqrt(q));
    L.pre = (float)(pow(te, gam - 1.0) * 2.0 * sqrt(q) / (1.0 + q));
    L.half_expo = (float)(0.5 * (1.0 - gam));
    L.g1 = p[6];
    L.g2 = p[7];
    L.pad_ = 0;
    // 2F1(1, a; b; -f w) = sum_n c_n (-f)^n w^n, c_n = prod_{k<=n} (a+k-1)/(b+k-1)
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
    if (!(fq == 0.0 || fabs(c * fn) * fq / (1.0 - fq) < 1e-9)) return 2;
    L.nterms = n;
    *Lout = L;
  }
  if (Gout) {
    LensGradConst G;
    for (int k = 0; k < kMaxSeriesTerms; ++k) G.hco[k] = 0.f;
    G.e = (float)(0.5 * (1.0 - gam));
    G.f = (float)fq;
    G.dlnpre_dq = (float)(0.5 / q - 1.0 / (1.0 + q));
    G.df_dq = (float)(-2.0 / ((1.0 + q) * (1.0 + q)));
    G.inv2q = (float)(0.5 / q);
    G.dlnte = te > 0.0 ? (float)((gam - 1.0) / te) : 0.f;
    G.pad_ = 0;
    // h_n = (n+1) c_{n+1} (-f)^n, c_n = prod_{k<=n} (a+k-1)/(b+k-1)
    double c = 1.0, fn = 1.0;  // c_{n+1}, (-f)^n
    int n = 0;
    for (n = 0; n < kMaxSeriesTerms; ++n) {
      c *= (a + n) / (b + n);  // c_{n+1}
      const double hn = (n + 1.0) * c * fn;
      G.hco[n] = (float)hn;
      // tail bound for sum_{k>n} |h_k|: |h_n| f (n+2)/(n+1) / (1 - f)^2
      if (fq == 0.0 || fabs(hn) * fq * (n + 2.0) / (n + 1.0) / ((1.0 - fq) * (1.0 - fq)) < 1e-9) {
        ++n;
        break;
      }
      fn *= -fq;
    }
    if (n > kMaxSeriesTerms) return 3;
    G.nterms = n < 1 ? 1 : n;
    *Gout = G;
  }
  return 0;
}

// A lens prepared on the device from device-resident parameters (the
// lr_lens_prepare entry point): both constant sets and the status of
// lens_constants (nonzero: the parameters were outside their domain and the
// constants are not to be used).
struct LensRecord {
  LensConst L;
  LensGradConst G;
  int32_t status;
  int32_t pad_[3];
};

struct cf {
  float re, im;
};
__device__ __forceinline__ cf cmul(cf a, cf b) { return {fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re)}; }
__device__ __forceinline__ cf cadd(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf cscale(cf a, float s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ cf cconj(cf a) { return {a.re, -a.im}; }
// Re(conj(g) z)
__device__ __forceinline__ float cdot(cf g, cf z) { return fmaf(g.re, z.re, g.im * z.im); }

// SPLE deflection and the contraction of G = dL/dbeta with -dalpha/dp for
// p = (x0, y0, q, phi, theta_e). Wirtinger form: alpha' = P F(W) w with
// w = R_x + i R_y, W = w / conj(w), P = pre (w conj(w))^e; for a real
// parameter with dw/dp = t: dalpha' = A_w t + A_wb conj(t) (+ explicit terms),
//   A_w = P ((e+1) F - M),  A_wb = P W (e F + M),  M = f W H(W);
// alpha = e^{i phi} alpha'.
__device__ __forceinline__ void sple_vjp(const LensConst& L, const LensGradConst& G, float x, float y, float gx,
                                         float gy, float out[5]) {
  const float dx = x - L.x0, dy = y - L.y0;
  const float u = fmaf(L.c, dx, L.s * dy);
  const float v = fmaf(L.c, dy, -L.s * dx);
  const float Rx = L.sq * u, Ry = L.isq * v;
  const float R2 = fmaf(Rx, Rx, Ry * Ry);
  if (!(R2 > 1e-24f)) {
    for (int k = 0; k < 5; ++k) out[k] = 0.f;
    return;
  }
  const float inv = 1.0f / R2;
  const cf W = {(Rx * Rx - Ry * Ry) * inv, 2.0f * Rx * Ry * inv};
  cf F = {L.d[L.nterms - 1], 0.f}, H = {G.hco[G.nterms - 1], 0.f};
  for (int n = L.nterms - 2; n >= 0; --n) F = cadd(cmul(W, F), cf{L.d[n], 0.f});
  for (int n = G.nterms - 2; n >= 0; --n) H = cadd(cmul(W, H), cf{G.hco[n], 0.f});
  const float P = L.pre * pow_split(R2, L.half_expo);
  const cf w = {Rx, Ry};
  const cf Fw = cmul(F, w);
  const cf ap = cscale(Fw, P);                    // alpha' (rotated frame)
  const cf M = cscale(cmul(W, H), G.f);
  const cf Aw = cscale(cadd(cscale(F, G.e + 1.0f), cscale(M, -1.0f)), P);
  const cf Awb = cscale(cmul(W, cadd(cscale(F, G.e), M)), P);
  const cf rot = {L.c, L.s};                      // e^{i phi}
  const cf g = {gx, gy};
  const cf gr = cmul(cconj(rot), g);              // conj(e^{i phi})... applied as Re(conj(g) e^{i phi} z) = Re(conj(gr) z)
  // Re(conj(g) e^{i phi} z) = Re(conj(e^{-i phi} g) z)
  auto dalpha = [&](cf t) { return cadd(cmul(Aw, t), cmul(Awb, cconj(t))); };
  const cf tx = {L.sq * L.c, -L.isq * L.s};       // dw/dxi_x
  const cf ty = {L.sq * L.s, L.isq * L.c};        // dw/dxi_y
  // x0, y0: dalpha/dx0 = -dalpha/dxi_x, and dL/dp = -Re(conj(g) dalpha/dp)
  out[0] = cdot(gr, dalpha(tx));
  out[1] = cdot(gr, dalpha(ty));
  // q: explicit prefactor and series-coefficient dependence plus dw/dq = conj(w)/(2q)
  const cf tq = cscale(cconj(w), G.inv2q);
  const cf dFdf_term = cscale(cmul(cmul(W, H), w), -P * G.df_dq);  // P w dF/df df/dq, dF/df = -W H
  const cf daq = cadd(cadd(cscale(ap, G.dlnpre_dq), dFdf_term), dalpha(tq));
  out[2] = -cdot(gr, daq);
  // phi: dalpha/dphi = i alpha + e^{i phi} dalpha'(dw/dphi), dw/dphi = sq v - i isq u
  const cf tphi = {L.sq * v, -L.isq * u};
  const cf daphi = cadd(cf{-ap.im, ap.re}, dalpha(tphi));
  out[3] = -cdot(gr, daphi);
  // theta_e: dalpha/dtheta_e = (gamma-1)/theta_e alpha
  out[4] = -G.dlnte * cdot(gr, ap);
}

// SPLE deflection Jacobian d alpha / d xi at (x, y), row-major
// (J[0] = d ax/dx, J[1] = d ax/dy, J[2] = d ay/dx, J[3] = d ay/dy), from the
// Wirtinger derivatives used by sple_vjp: d alpha = e^{i phi} (A_w t + A_wb conj(t)).
__device__ __forceinline__ void sple_jacobian(const LensConst& L, const LensGradConst& G, float x, float y,
                                              float J[4]) {
  const float dx = x - L.x0, dy = y - L.y0;
  const float u = fmaf(L.c, dx, L.s * dy);
  const float v = fmaf(L.c, dy, -L.s * dx);
  const float Rx = L.sq * u, Ry = L.isq * v;
  const float R2 = fmaf(Rx, Rx, Ry * Ry);
  if (!(R2 > 1e-24f)) {
    J[0] = J[1] = J[2] = J[3] = 0.f;
    return;
  }
  const float inv = 1.0f / R2;
  const cf W = {(Rx * Rx - Ry * Ry) * inv, 2.0f * Rx * Ry * inv};
  cf F = {L.d[L.nterms - 1], 0.f}, H = {G.hco[G.nterms - 1], 0.f};
  for (int n = L.nterms - 2; n >= 0; --n) F = cadd(cmul(W, F), cf{L.d[n], 0.f});
  for (int n = G.nterms - 2; n >= 0; --n) H = cadd(cmul(W, H), cf{G.hco[n], 0.f});
  const float P = L.pre * pow_split(R2, L.half_expo);
  const cf M = cscale(cmul(W, H), G.f);
  const cf Aw = cscale(cadd(cscale(F, G.e + 1.0f), cscale(M, -1.0f)), P);
  const cf Awb = cscale(cmul(W, cadd(cscale(F, G.e), M)), P);
  const cf rot = {L.c, L.s};
  const cf tx = {L.sq * L.c, -L.isq * L.s};
  const cf ty = {L.sq * L.s, L.isq * L.c};
  const cf jx = cmul(rot, cadd(cmul(Aw, tx), cmul(Awb, cconj(tx))));
  const cf jy = cmul(rot, cadd(cmul(Aw, ty), cmul(Awb, cconj(ty))));
  J[0] = jx.re;
  J[1] = jy.re;
  J[2] = jx.im;
  J[3] = jy.im;
}

}  // namespace lr
