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
//        (tau^2-1)/tau, C = tau pi + (tau^2-1) ln tau
//  point mass: x_h, y_h, theta_pm^2, 0...
struct SubRec {
  float xh, yh, its2, A, tau, tau2, t2m1_t, C;
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

// a2: SPLE deflection at (x, y).
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

// F(x) of the NFW family as a function of x^2 (x = R / theta_s):
//   arccosh(1/x)/sqrt(1-x^2) for x < 1, arccos(1/x)/sqrt(x^2-1) for x > 1,
// with its series sum_n (-eps)^n/(2n+1), eps = x^2 - 1, near x = 1.
// Also returns s = sqrt(|1 - x^2|).
__device__ __forceinline__ float nfw_F(float x2, float xx, float& s) {
  const float eps = x2 - 1.0f;
  s = sqrtf(fabsf(eps));
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
  if (eps < 0.f) return logf((1.0f + s) / xx) / s;  // arccosh(1/x) = ln((1 + s)/x)
  return atanf(s) / s;                              // arccos(1/x) = arctan(s)
}

// a4: truncated-NFW deflection per unit offset: alpha = m * (dx, dy) with
// m = A * B(x)/x^2 where B is the bracket of the enclosed-mass function.
// For x < 0.5 the bracket is evaluated in a rearranged form whose terms are
// all O(x^2) (the direct form cancels catastrophically as x -> 0):
//   B/x^2 = -pi/(tau+st) + 2F + (tau^2-1) [F/(1+s) + log1p(dl)/x^2 + L/(tau (tau+st))],
//   dl = -x^2 [tau/(1+s) + 1/(tau+st)]/(tau+st),  st = sqrt(tau^2+x^2),
// otherwise B = (tau^2-1+2x^2) F + C + st (-pi + (tau^2-1)/tau L).
__device__ __forceinline__ float tnfw_m(const SubRec& h, float R2) {
  const float x2 = R2 * h.its2;
  if (!(x2 > 1e-20f)) return 0.f;
  const float xx = sqrtf(x2);
  float s;
  const float F = nfw_F(x2, xx, s);
  const float st = sqrtf(h.tau2 + x2);
  const float tp = h.tau + st;
  const float L = logf(xx / tp);
  float G;
  if (x2 < 0.25f) {
    const float dlx2 = -(h.tau / (1.0f + s) + 1.0f / tp) / tp;
    const float dl = dlx2 * x2;
    const float ratio = (dl != 0.f) ? log1pf(dl) / dl : 1.0f;
    const float t2m1 = h.tau2 - 1.0f;
    G = fmaf(2.0f, F, -kPi / tp) +
        t2m1 * (F / (1.0f + s) + dlx2 * ratio + L / (h.tau * tp));
  } else {
    const float t2m1 = h.tau2 - 1.0f;
    const float B = fmaf(fmaf(2.0f, x2, t2m1), F, h.C) + st * fmaf(h.t2m1_t, L, -kPi);
    G = B / x2;
  }
  return h.A * G;
}

// Point mass: alpha = theta_pm^2 (dx, dy) / R^2.
__device__ __forceinline__ float pointmass_m(const SubRec& h, float R2) {
  return (R2 > 1e-30f) ? h.its2 / R2 : 0.f;
}

}  // namespace lr
