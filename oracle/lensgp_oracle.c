/*
 * lensgp ORACLE — plain, slow, FP64 CPU implementation of the lens ray-trace
 * and Gaussian-kernel reduction of Karchev, Coogan & Weniger (arXiv:2105.09465).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. The CUDA library never calls
 * it and shares no code, header, table or constant with it.
 *
 * Every function states the passage of the paper it follows. Arithmetic is
 * FP64 throughout; sums over many terms use Neumaier (improved Kahan)
 * compensation. Parallelism is OpenMP over independent output rows only, so
 * results do not depend on the thread count.
 *
 * Subhalos are not part of the paper (Sec. 2.2 leaves substructure out). They
 * follow the truncated NFW profile of Baltz, Marshall & Oguri (2009),
 *   rho(r) = rho_s / [(r/r_s)(1 + r/r_s)^2] * tau^2 / (tau^2 + (r/r_s)^2),
 * with angular parameters (x_h, y_h, kappa_s, theta_s, tau), kappa_s =
 * rho_s r_s / Sigma_cr and theta_s = r_s / D_l. A point mass (deflection
 * theta_pm^2 d/|d|^2) is the second supported profile.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

static const double PI = 3.14159265358979323846264338327950288;

/* Image-plane grid (Sec. 2, Table 1: P are pixel centres; S x S
 * supersampling of an nx x ny grid of spacing pix is the (nx S) x (ny S) grid
 * of spacing pix/S). Positions are FP32 values: the FP32 rounding of
 * cx + (col - (nx S - 1)/2) * h with h = float(pix / S). */
typedef struct {
  int32_t nx, ny, ss;
  float pix, cx, cy;
} orc_grid;

/* Lens parameters in the order of Sec. 2.2: centre (x0, y0), axis ratio q,
 * orientation phi (radians), Einstein radius theta_e, 3-D slope gamma, and
 * external shear (g1, g2). */
typedef struct {
  double x0, y0, q, phi, theta_e, gamma, g1, g2;
} orc_lens;

/* ------------------------------------------------------------------------ */
/* Compensated summation (Neumaier).                                          */
typedef struct {
  double s, c;
} nsum;
static inline void ns_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double ns_val(const nsum* a) { return a->s + a->c; }

/* exp(-a) is exactly 0.0 in FP64 once a > 745.14 (below the smallest
 * subnormal); a pair whose kernel exponent is past EXP_ZERO therefore adds
 * exactly nothing to any sum below (a Neumaier sum is unchanged by adding
 * +0 or -0), and the loops skip it without changing a single result bit. */
#define EXP_ZERO 750.0

/* ------------------------------------------------------------------------ */
/* Forward-mode dual numbers: value plus derivatives with respect to up to
 * ND parameters. Used for the analytic parameter gradients of the ray-trace. */
#define ND 8
typedef struct {
  double v, d[ND];
} dn;

static inline dn dn_const(double v) {
  dn r;
  memset(&r, 0, sizeof r);
  r.v = v;
  return r;
}
static inline dn dn_var(double v, int k) {
  dn r = dn_const(v);
  r.d[k] = 1.0;
  return r;
}
static inline dn dn_add(dn a, dn b) {
  for (int k = 0; k < ND; ++k) a.d[k] += b.d[k];
  a.v += b.v;
  return a;
}
static inline dn dn_sub(dn a, dn b) {
  for (int k = 0; k < ND; ++k) a.d[k] -= b.d[k];
  a.v -= b.v;
  return a;
}
static inline dn dn_mul(dn a, dn b) {
  dn r;
  r.v = a.v * b.v;
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
static inline dn dn_scale(dn a, double s) {
  a.v *= s;
  for (int k = 0; k < ND; ++k) a.d[k] *= s;
  return a;
}
static inline dn dn_addc(dn a, double c) {
  a.v += c;
  return a;
}
/* f(a) with f(a.v) = fv and f'(a.v) = fp. */
static inline dn dn_chain(dn a, double fv, double fp) {
  dn r;
  r.v = fv;
  for (int k = 0; k < ND; ++k) r.d[k] = fp * a.d[k];
  return r;
}
static inline dn dn_div(dn a, dn b) {
  dn r;
  r.v = a.v / b.v;
  for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
  return r;
}
static inline dn dn_recip(dn a) { return dn_chain(a, 1.0 / a.v, -1.0 / (a.v * a.v)); }
static inline dn dn_sqrt(dn a) {
  double s = sqrt(a.v);
  return dn_chain(a, s, 0.5 / s);
}
static inline dn dn_log(dn a) { return dn_chain(a, log(a.v), 1.0 / a.v); }
static inline dn dn_powc(dn a, double e) {
  /* a^0 is the constant 1 (also at a = 0, where e a^(e-1) would be 0 * inf) */
  if (e == 0.0) return dn_const(1.0);
  return dn_chain(a, pow(a.v, e), e * pow(a.v, e - 1.0));
}
static inline dn dn_cos(dn a) { return dn_chain(a, cos(a.v), -sin(a.v)); }
static inline dn dn_sin(dn a) { return dn_chain(a, sin(a.v), cos(a.v)); }
static inline dn dn_acosh(dn a) { return dn_chain(a, acosh(a.v), 1.0 / sqrt(a.v * a.v - 1.0)); }
static inline dn dn_acos(dn a) { return dn_chain(a, acos(a.v), -1.0 / sqrt(1.0 - a.v * a.v)); }

/* Complex dual: (re, im), each a dual. */
typedef struct {
  dn re, im;
} cdn;
static inline cdn cdn_mul(cdn a, cdn b) {
  cdn r;
  r.re = dn_sub(dn_mul(a.re, b.re), dn_mul(a.im, b.im));
  r.im = dn_add(dn_mul(a.re, b.im), dn_mul(a.im, b.re));
  return r;
}
static inline cdn cdn_add(cdn a, cdn b) {
  cdn r = {dn_add(a.re, b.re), dn_add(a.im, b.im)};
  return r;
}
static inline cdn cdn_scale(cdn a, dn s) {
  cdn r = {dn_mul(a.re, s), dn_mul(a.im, s)};
  return r;
}
static inline cdn cdn_scalec(cdn a, double s) {
  cdn r = {dn_scale(a.re, s), dn_scale(a.im, s)};
  return r;
}

/* ------------------------------------------------------------------------ */
/* Pixel centres (Sec. 2 / Table 1).                                       */
ORC_API void orc_grid_points(const orc_grid* g, float* xi /* [n][2] */) {
  const int64_t W = (int64_t)g->nx * g->ss, H = (int64_t)g->ny * g->ss;
  const float h = g->pix / (float)g->ss;
  const float c0x = 0.5f * (float)(W - 1), c0y = 0.5f * (float)(H - 1);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < H; ++r)
    for (int64_t c = 0; c < W; ++c) {
      xi[2 * (r * W + c) + 0] = fmaf((float)c - c0x, h, g->cx);
      xi[2 * (r * W + c) + 1] = fmaf((float)r - c0y, h, g->cy);
    }
}

/* ------------------------------------------------------------------------ */
/* SPLE deflection (Sec. 2.2, eq. for the SPLE displacement).
 *  (u, v) = Rot(phi) (xi - xi0); R_x = sqrt(q) u, R_y = v / sqrt(q);
 *  e^{i phi_e} = (R_x + i R_y) / R;  z = -(1-q)/(1+q) e^{2 i phi_e};
 *  alpha' = theta_e 2 sqrt(q)/(1+q) (theta_e/R)^(gamma-2) 2F1(1, (gamma-1)/2;
 *           (5-gamma)/2; z) e^{i phi_e}, expressed in the (u, v) frame and
 *  rotated back by Rot(phi)^T.
 * 2F1(1, a; b; z) = sum_n (a)_n / (b)_n z^n, summed until the term falls
 * below 1e-17 |F|. The derivative slots of the inputs propagate through.
 * Returns 0 deflection when R < 1e-12 arcsec (the profile is singular there). */
static void sple_dual(dn x, dn y, dn x0, dn y0, dn q, dn phi, dn te, double gamma, dn* ax, dn* ay) {
  dn c = dn_cos(phi), s = dn_sin(phi);
  dn dx = dn_sub(x, x0), dy = dn_sub(y, y0);
  dn u = dn_add(dn_mul(c, dx), dn_mul(s, dy));
  dn v = dn_sub(dn_mul(c, dy), dn_mul(s, dx));
  dn sq = dn_sqrt(q);
  dn Rx = dn_mul(sq, u), Ry = dn_div(v, sq);
  dn R = dn_sqrt(dn_add(dn_mul(Rx, Rx), dn_mul(Ry, Ry)));
  if (R.v < 1e-12) {
    *ax = dn_const(0.0);
    *ay = dn_const(0.0);
    return;
  }
  cdn e = {dn_div(Rx, R), dn_div(Ry, R)};
  dn f = dn_div(dn_addc(dn_scale(q, -1.0), 1.0), dn_addc(q, 1.0)); /* (1-q)/(1+q) */
  cdn z = cdn_scale(cdn_mul(e, e), dn_scale(f, -1.0));
  const double a = 0.5 * (gamma - 1.0), b = 0.5 * (5.0 - gamma);
  cdn F = {dn_const(1.0), dn_const(0.0)};
  cdn term = F;
  for (int n = 1; n < 5000; ++n) {
    term = cdn_scalec(cdn_mul(term, z), (a + n - 1.0) / (b + n - 1.0));
    F = cdn_add(F, term);
    double tm = hypot(term.re.v, term.im.v), fm = hypot(F.re.v, F.im.v);
    if (tm < 1e-17 * fm) break;
  }
  /* prefactor theta_e * 2 sqrt(q)/(1+q) * (theta_e / R)^(gamma - 2) */
  dn pre = dn_mul(te, dn_div(dn_scale(sq, 2.0), dn_addc(q, 1.0)));
  pre = dn_mul(pre, dn_powc(dn_div(te, R), gamma - 2.0));
  cdn ap = cdn_scale(cdn_mul(F, e), pre);
  /* rotate back: alpha = Rot^T alpha' */
  *ax = dn_sub(dn_mul(c, ap.re), dn_mul(s, ap.im));
  *ay = dn_add(dn_mul(s, ap.re), dn_mul(c, ap.im));
}

/* SPLE convergence, Sec. 2.2: kappa = (3 - gamma)/2 (theta_e / R)^(gamma - 1)
 * with R the elliptical radius above. Used by the divergence pin. */
ORC_API double orc_sple_kappa(double x, double y, const orc_lens* L) {
  double c = cos(L->phi), s = sin(L->phi);
  double u = c * (x - L->x0) + s * (y - L->y0), v = -s * (x - L->x0) + c * (y - L->y0);
  double R = sqrt(L->q * u * u + v * v / L->q);
  return 0.5 * (3.0 - L->gamma) * pow(L->theta_e / R, L->gamma - 1.0);
}

/* ------------------------------------------------------------------------ */
/* Truncated NFW deflection (Baltz, Marshall & Oguri 2009), in units of
 * the scale radius: x = R / theta_s,
 *   g(x) = tau^2/(tau^2+1)^2 [ (tau^2 + 1 + 2(x^2-1)) F(x) + tau pi
 *          + (tau^2-1) ln tau + sqrt(tau^2+x^2) (-pi + (tau^2-1)/tau L(x)) ],
 *   F(x) = arccosh(1/x)/sqrt(1-x^2) (x<1), arccos(1/x)/sqrt(x^2-1) (x>1),
 *   L(x) = ln(x / (sqrt(tau^2+x^2) + tau)),
 * |alpha| = 4 kappa_s theta_s g(x) / x, directed along xi - xi_h.
 * Near x = 1 F uses its series in eps = x^2 - 1: sum_n (-eps)^n / (2n+1). */
static dn tnfw_F(dn x) {
  dn eps = dn_addc(dn_mul(x, x), -1.0);
  if (fabs(eps.v) < 1e-3) {
    dn acc = dn_const(0.0), pw = dn_const(1.0), meps = dn_scale(eps, -1.0);
    for (int n = 0; n < 12; ++n) {
      acc = dn_add(acc, dn_scale(pw, 1.0 / (2.0 * n + 1.0)));
      pw = dn_mul(pw, meps);
    }
    return acc;
  }
  if (x.v < 1.0) return dn_div(dn_acosh(dn_recip(x)), dn_sqrt(dn_scale(eps, -1.0)));
  return dn_div(dn_acos(dn_recip(x)), dn_sqrt(eps));
}

static void tnfw_dual(dn x, dn y, dn xh, dn yh, dn ks, dn ts, double tau, dn* ax, dn* ay) {
  dn dx = dn_sub(x, xh), dy = dn_sub(y, yh);
  dn R = dn_sqrt(dn_add(dn_mul(dx, dx), dn_mul(dy, dy)));
  if (R.v < 1e-15) {
    *ax = dn_const(0.0);
    *ay = dn_const(0.0);
    return;
  }
  dn X = dn_div(R, ts);
  const double t2 = tau * tau;
  dn st = dn_sqrt(dn_addc(dn_mul(X, X), t2));
  dn Lx = dn_log(dn_div(X, dn_addc(st, tau)));
  dn Fx = tnfw_F(X);
  dn term1 = dn_mul(dn_addc(dn_scale(dn_mul(X, X), 2.0), t2 - 1.0), Fx); /* (tau^2+1+2(x^2-1)) F */
  dn term2 = dn_const(tau * PI + (t2 - 1.0) * log(tau));
  dn term3 = dn_mul(st, dn_addc(dn_scale(Lx, (t2 - 1.0) / tau), -PI));
  dn g = dn_scale(dn_add(dn_add(term1, term2), term3), t2 / ((t2 + 1.0) * (t2 + 1.0)));
  /* alpha = 4 kappa_s theta_s g / x * d / R = 4 kappa_s g / x^2 * d */
  dn m = dn_div(dn_scale(dn_mul(ks, g), 4.0), dn_mul(X, X));
  *ax = dn_mul(m, dx);
  *ay = dn_mul(m, dy);
}

static void pointmass_dual(dn x, dn y, dn xh, dn yh, dn tpm, dn* ax, dn* ay) {
  dn dx = dn_sub(x, xh), dy = dn_sub(y, yh);
  dn r2 = dn_add(dn_mul(dx, dx), dn_mul(dy, dy));
  if (r2.v < 1e-30) {
    *ax = dn_const(0.0);
    *ay = dn_const(0.0);
    return;
  }
  dn m = dn_div(dn_mul(tpm, tpm), r2);
  *ax = dn_mul(m, dx);
  *ay = dn_mul(m, dy);
}

/* Deflection of subhalo h at (x, y): profile 0 = tNFW record (x, y, kappa_s,
 * theta_s, tau); profile 1 = point mass record (x, y, theta_pm, -, -).
 * Derivative slots 0..3 are (x_h, y_h, kappa_s or theta_pm, theta_s) when
 * `with_grad`. */
static void sub_dual(double x, double y, const double* rec, int profile, int with_grad, dn* ax, dn* ay) {
  dn X = dn_const(x), Y = dn_const(y);
  dn xh = with_grad ? dn_var(rec[0], 0) : dn_const(rec[0]);
  dn yh = with_grad ? dn_var(rec[1], 1) : dn_const(rec[1]);
  dn p2 = with_grad ? dn_var(rec[2], 2) : dn_const(rec[2]);
  dn p3 = with_grad ? dn_var(rec[3], 3) : dn_const(rec[3]);
  if (profile == 1)
    pointmass_dual(X, Y, xh, yh, p2, ax, ay);
  else
    tnfw_dual(X, Y, xh, yh, p2, p3, rec[4], ax, ay);
}

/* ------------------------------------------------------------------------ */
/* Ray-trace (eq. for the raytracing equation, Sec. 2.1):
 *   beta = xi - alpha(xi), alpha = alpha_SPLE + alpha_shear + sum_h alpha_h.
 * External shear (Sec. 2.2): alpha = [[g1, g2], [g2, -g1]] xi about the origin.
 * Outputs alpha and beta for n points xi (all FP64; FP32 inputs are widened
 * exactly by the caller). */
ORC_API void orc_raytrace(const double* xi, int64_t n, const orc_lens* L, const double* sub, int32_t n_sub,
                          int32_t profile, double* alpha /*[n][2] or NULL*/, double* beta /*[n][2] or NULL*/) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    const double x = xi[2 * i], y = xi[2 * i + 1];
    nsum sx = {0, 0}, sy = {0, 0};
    dn ax, ay;
    sple_dual(dn_const(x), dn_const(y), dn_const(L->x0), dn_const(L->y0), dn_const(L->q), dn_const(L->phi),
              dn_const(L->theta_e), L->gamma, &ax, &ay);
    ns_add(&sx, ax.v);
    ns_add(&sy, ay.v);
    ns_add(&sx, L->g1 * x + L->g2 * y);
    ns_add(&sy, L->g2 * x - L->g1 * y);
    for (int32_t h = 0; h < n_sub; ++h) {
      sub_dual(x, y, sub + 5 * (int64_t)h, profile, 0, &ax, &ay);
      ns_add(&sx, ax.v);
      ns_add(&sy, ay.v);
    }
    const double axv = ns_val(&sx), ayv = ns_val(&sy);
    if (alpha) {
      alpha[2 * i] = axv;
      alpha[2 * i + 1] = ayv;
    }
    if (beta) {
      beta[2 * i] = x - axv;
      beta[2 * i + 1] = y - ayv;
    }
  }
}

/* Ray-trace vector-Jacobian product: given d_beta = dLoss/dbeta_i, returns
 *   d_lens[7] = dLoss/d(x0, y0, q, phi, theta_e, g1, g2)   (slope held fixed,
 *               as in the paper's fits, Sec. 4.2),
 *   d_sub[S][4] = dLoss/d(x_h, y_h, kappa_s | theta_pm, theta_s),
 * with dLoss/dtheta = -sum_i (dalpha_i/dtheta)^T d_beta_i, from forward-mode
 * dual numbers through the same expressions as orc_raytrace. */
ORC_API void orc_raytrace_vjp(const double* xi, int64_t n, const orc_lens* L, const double* sub, int32_t n_sub,
                              int32_t profile, const double* d_beta, double* d_lens /*[7]*/,
                              double* d_sub /*[S][4] or NULL*/, double* d_lens_abs /*[7] or NULL*/,
                              double* d_sub_abs /*[S][4] or NULL*/) {
  nsum acc[7], aacc[7];
  memset(acc, 0, sizeof acc);
  memset(aacc, 0, sizeof aacc);
#pragma omp parallel
  {
    nsum loc[7], aloc[7];
    memset(loc, 0, sizeof loc);
    memset(aloc, 0, sizeof aloc);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const double x = xi[2 * i], y = xi[2 * i + 1];
      dn ax, ay;
      sple_dual(dn_const(x), dn_const(y), dn_var(L->x0, 0), dn_var(L->y0, 1), dn_var(L->q, 2), dn_var(L->phi, 3),
                dn_var(L->theta_e, 4), L->gamma, &ax, &ay);
      const double gx = d_beta[2 * i], gy = d_beta[2 * i + 1];
      double t[7];
      for (int k = 0; k < 5; ++k) t[k] = -(ax.d[k] * gx + ay.d[k] * gy);
      /* shear: dalpha/dg1 = (x, -y), dalpha/dg2 = (y, x) */
      t[5] = -(x * gx - y * gy);
      t[6] = -(y * gx + x * gy);
      for (int k = 0; k < 7; ++k) {
        ns_add(&loc[k], t[k]);
        ns_add(&aloc[k], fabs(t[k]));
      }
    }
#pragma omp critical
    for (int k = 0; k < 7; ++k) {
      ns_add(&acc[k], loc[k].s);
      ns_add(&acc[k], loc[k].c);
      ns_add(&aacc[k], aloc[k].s);
      ns_add(&aacc[k], aloc[k].c);
    }
  }
  for (int k = 0; k < 7; ++k) {
    d_lens[k] = ns_val(&acc[k]);
    if (d_lens_abs) d_lens_abs[k] = ns_val(&aacc[k]);
  }
  if (!d_sub) return;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t h = 0; h < n_sub; ++h) {
    nsum a4[4], b4[4];
    memset(a4, 0, sizeof a4);
    memset(b4, 0, sizeof b4);
    for (int64_t i = 0; i < n; ++i) {
      dn ax, ay;
      sub_dual(xi[2 * i], xi[2 * i + 1], sub + 5 * (int64_t)h, profile, 1, &ax, &ay);
      const double gx = d_beta[2 * i], gy = d_beta[2 * i + 1];
      for (int k = 0; k < 4; ++k) {
        const double t = -(ax.d[k] * gx + ay.d[k] * gy);
        ns_add(&a4[k], t);
        ns_add(&b4[k], fabs(t));
      }
    }
    for (int k = 0; k < 4; ++k) {
      d_sub[4 * (int64_t)h + k] = ns_val(&a4[k]);
      if (d_sub_abs) d_sub_abs[4 * (int64_t)h + k] = ns_val(&b4[k]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Lens Jacobian and magnification (Sec. 2.1, lens-Jacobian and magnification
 * equations): A = d beta / d xi = I - d alpha / d xi, mu = 1 / det A.
 * d alpha / d xi comes from forward-mode dual numbers in (x, y) through the
 * same deflection expressions as orc_raytrace (slots 0 and 1).
 * jac: [n][4] = (A_xx, A_xy, A_yx, A_yy) with A_xy = d beta_x / d y. */
ORC_API void orc_lens_jacobian(const double* xi, int64_t n, const orc_lens* L, const double* sub, int32_t n_sub,
                               int32_t profile, double* jac /*[n][4]*/, double* mu /*[n] or NULL*/) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    const double x = xi[2 * i], y = xi[2 * i + 1];
    dn X = dn_var(x, 0), Y = dn_var(y, 1);
    nsum a[4];
    memset(a, 0, sizeof a);
    dn ax, ay;
    sple_dual(X, Y, dn_const(L->x0), dn_const(L->y0), dn_const(L->q), dn_const(L->phi), dn_const(L->theta_e),
              L->gamma, &ax, &ay);
    ns_add(&a[0], ax.d[0]);
    ns_add(&a[1], ax.d[1]);
    ns_add(&a[2], ay.d[0]);
    ns_add(&a[3], ay.d[1]);
    /* shear: d alpha / d xi = [[g1, g2], [g2, -g1]] */
    ns_add(&a[0], L->g1);
    ns_add(&a[1], L->g2);
    ns_add(&a[2], L->g2);
    ns_add(&a[3], -L->g1);
    for (int32_t h = 0; h < n_sub; ++h) {
      const double* rec = sub + 5 * (int64_t)h;
      dn hx, hy;
      if (profile == 1)
        pointmass_dual(X, Y, dn_const(rec[0]), dn_const(rec[1]), dn_const(rec[2]), &hx, &hy);
      else
        tnfw_dual(X, Y, dn_const(rec[0]), dn_const(rec[1]), dn_const(rec[2]), dn_const(rec[3]), rec[4], &hx, &hy);
      ns_add(&a[0], hx.d[0]);
      ns_add(&a[1], hx.d[1]);
      ns_add(&a[2], hy.d[0]);
      ns_add(&a[3], hy.d[1]);
    }
    const double j00 = 1.0 - ns_val(&a[0]), j01 = -ns_val(&a[1]), j10 = -ns_val(&a[2]), j11 = 1.0 - ns_val(&a[3]);
    jac[4 * i] = j00;
    jac[4 * i + 1] = j01;
    jac[4 * i + 2] = j10;
    jac[4 * i + 3] = j11;
    if (mu) mu[i] = 1.0 / (j00 * j11 - j01 * j10);
  }
}

/* ------------------------------------------------------------------------ */
/* Gaussian RBF kernel reduction (eq. for the Gaussian RBF, Sec. 3.1, with
 * isotropic kernel Sigma = l^2 I; Sec. 3.3 evaluates T y as this lazily
 * reduced sum):
 *   out_i    = sum_j var * exp(-|x_i - y_j|^2 / (2 l^2)) v_j,
 *   absout_i = sum_j |var exp(...) v_j|           (scale of the parity tolerance)
 *   sens_i   = sum_j |var exp(...) v_j| |x_i - y_j| / l^2
 *              (bound on |d out_i / d x| per unit displacement of any point:
 *               scales the tolerance when the points themselves carry error)
 * x: n points, y: m points, v: m values (one right-hand side), all FP64.
 * `rows` (optional) restricts the evaluation to those row indices; outputs
 * then have n_rows entries. absout and sens may be NULL. */
static void matvec_row(const double* x, int64_t i, const double* y, int64_t m, const double* v, double inv2l2,
                       double invl2, double variance, double* out, double* absout, double* sens) {
  const double xi = x[2 * i], yi = x[2 * i + 1];
  nsum s = {0, 0}, a = {0, 0}, g = {0, 0};
  for (int64_t j = 0; j < m; ++j) {
    const double dx = xi - y[2 * j], dy = yi - y[2 * j + 1];
    const double d2 = dx * dx + dy * dy;
    if (d2 * inv2l2 > EXP_ZERO) continue;
    const double kv = variance * exp(-d2 * inv2l2) * v[j];
    ns_add(&s, kv);
    ns_add(&a, fabs(kv));
    ns_add(&g, fabs(kv) * sqrt(d2) * invl2);
  }
  *out = ns_val(&s);
  if (absout) *absout = ns_val(&a);
  if (sens) *sens = ns_val(&g);
}

ORC_API void orc_kernel_matvec(const double* x, int64_t n, const double* y, int64_t m, const double* v,
                               double lengthscale, double variance, const int64_t* rows, int64_t n_rows, double* out,
                               double* absout, double* sens) {
  const double inv2l2 = 1.0 / (2.0 * lengthscale * lengthscale), invl2 = 1.0 / (lengthscale * lengthscale);
  const int64_t cnt = rows ? n_rows : n;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < cnt; ++r) {
    const int64_t i = rows ? rows[r] : r;
    matvec_row(x, i, y, m, v, inv2l2, invl2, variance, out + r, absout ? absout + r : NULL, sens ? sens + r : NULL);
  }
}

/* ------------------------------------------------------------------------ */
/* Pixel windows (Sec. 3.2, the window-kernel equation and its footnote): the
 * projected pixel centres p form a W x H grid (row-major over grid y). The
 * axes of pixel i are a_i = half the vector between the two centres adjacent
 * along grid x, b_i the same along grid y; at the border of the grid, where
 * one neighbour is missing, the vector to the single neighbour. The window
 * covariance is Z_i = (a a^T + b b^T) / (4 pi); output (Zxx, Zxy, Zyy). */
ORC_API void orc_pixel_shapes(const double* p, int32_t W, int32_t H, double* z) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < H; ++r)
    for (int64_t c = 0; c < W; ++c) {
      const int64_t i = r * W + c;
      const int64_t cl = c > 0 ? i - 1 : i, cr = c + 1 < W ? i + 1 : i;
      const int64_t rd = r > 0 ? i - W : i, ru = r + 1 < H ? i + W : i;
      const double sa = (cr - cl == 2) ? 0.5 : 1.0, sb = (ru - rd == 2 * W) ? 0.5 : 1.0;
      const double ax = sa * (p[2 * cr] - p[2 * cl]), ay = sa * (p[2 * cr + 1] - p[2 * cl + 1]);
      const double bx = sb * (p[2 * ru] - p[2 * rd]), by = sb * (p[2 * ru + 1] - p[2 * rd + 1]);
      const double k = 1.0 / (4.0 * PI);
      z[3 * i] = k * (ax * ax + bx * bx);
      z[3 * i + 1] = k * (ax * ay + bx * by);
      z[3 * i + 2] = k * (ay * ay + by * by);
    }
}

/* Windowed transmission (Sec. 3.4, the transmission equation, with
 * Sigma = l^2 I): T_ik = A_k G(p_i - q_k, Z_i + Sigma / 2), reduced as
 *   out_i = sum_k G(p_i - q_k, Z_i + Sigma / 2) v_k,
 * G(d, C) = exp(-d^T C^-1 d / 2) / (2 pi sqrt(det C)); the caller folds the
 * weights A_k into v_k. absout_i = sum_k |G v_k|. With T != NULL (tiny
 * sizes only) also writes the dense G matrix [n][m]. */
ORC_API void orc_windowed_matvec(const double* p, const double* z, int64_t n, const double* q, int64_t m,
                                 const double* v, double lengthscale, double* out, double* absout, double* T) {
  const double half_s = 0.5 * lengthscale * lengthscale;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    const double cxx = z[3 * i] + half_s, cxy = z[3 * i + 1], cyy = z[3 * i + 2] + half_s;
    const double det = cxx * cyy - cxy * cxy;
    const double ixx = cyy / det, ixy = -cxy / det, iyy = cxx / det;
    const double norm = 1.0 / (2.0 * PI * sqrt(det));
    nsum s = {0, 0}, a = {0, 0};
    for (int64_t k = 0; k < m; ++k) {
      const double dx = p[2 * i] - q[2 * k], dy = p[2 * i + 1] - q[2 * k + 1];
      const double g = norm * exp(-0.5 * (ixx * dx * dx + 2.0 * ixy * dx * dy + iyy * dy * dy));
      if (T) T[i * m + k] = g;
      if (v) {
        ns_add(&s, g * v[k]);
        ns_add(&a, fabs(g * v[k]));
      }
    }
    if (out) out[i] = ns_val(&s);
    if (absout) absout[i] = ns_val(&a);
  }
}

/* Gradients of Loss = sum_i g_i out_i through the windowed transmission
 * reduction (out_i = sum_k G(p_i - q_k, C_i) v_k, C_i = Z_i + (l^2/2) I), by
 * differentiating each Gaussian term: with d = p_i - q_k, M = C_i^-1 and
 * u = M d,
 *   dG/dp_i = -G u,  dG/dq_k = G u,  dG/dC_i = G (u u^T - M) / 2,
 * and dC_i/dl = l I. Outputs (each may be NULL):
 *   d_v[m], d_p[n][2], d_q[m][2], d_z[n][3] (dL/d(Zxx, Zxy, Zyy), the
 *   off-diagonal entry counted in both symmetric positions), d_len[1];
 * abs_* (same shapes, optional) receive the sums of absolute terms. */
ORC_API void orc_windowed_vjp(const double* p, const double* z, int64_t n, const double* q, int64_t m,
                              const double* v, double lengthscale, const double* g, double* d_v, double* d_p,
                              double* d_q, double* d_z, double* d_len, double* abs_v, double* abs_p, double* abs_q,
                              double* abs_z, double* abs_len) {
  const double half_s = 0.5 * lengthscale * lengthscale;
  double* dq_acc = (double*)calloc((size_t)(3 * m + 1), sizeof(double));
  double* dq_abs = (double*)calloc((size_t)(3 * m + 1), sizeof(double));
  nsum len = {0, 0}, len_a = {0, 0};
  for (int64_t i = 0; i < n; ++i) {
    const double cxx = z[3 * i] + half_s, cxy = z[3 * i + 1], cyy = z[3 * i + 2] + half_s;
    const double det = cxx * cyy - cxy * cxy;
    const double mxx = cyy / det, mxy = -cxy / det, myy = cxx / det;
    const double norm = 1.0 / (2.0 * PI * sqrt(det));
    nsum px = {0, 0}, py = {0, 0}, zxx = {0, 0}, zxy = {0, 0}, zyy = {0, 0};
    double apx = 0, apy = 0, azxx = 0, azxy = 0, azyy = 0;
    for (int64_t k = 0; k < m; ++k) {
      const double dx = p[2 * i] - q[2 * k], dy = p[2 * i + 1] - q[2 * k + 1];
      const double ux = mxx * dx + mxy * dy, uy = mxy * dx + myy * dy;
      const double G = norm * exp(-0.5 * (dx * ux + dy * uy));
      const double gG = g[i] * G, gGv = gG * v[k];
      /* row role */
      ns_add(&px, -gGv * ux);
      ns_add(&py, -gGv * uy);
      apx += fabs(gGv * ux);
      apy += fabs(gGv * uy);
      const double cx = 0.5 * gGv * (ux * ux - mxx), cxy2 = 0.5 * gGv * (ux * uy - mxy),
                   cy = 0.5 * gGv * (uy * uy - myy);
      ns_add(&zxx, cx);
      ns_add(&zxy, 2.0 * cxy2);
      ns_add(&zyy, cy);
      /* scales: both parts of u u^T - M, which nearly cancel for a pair at
       * d^T M d ~ 1 */
      const double hg = 0.5 * fabs(gGv);
      const double sx = hg * (ux * ux + fabs(mxx)), sxy = hg * (fabs(ux * uy) + fabs(mxy)),
                   sy = hg * (uy * uy + fabs(myy));
      azxx += sx;
      azxy += 2.0 * sxy;
      azyy += sy;
      ns_add(&len, lengthscale * (cx + cy));
      ns_add(&len_a, lengthscale * (sx + sy));
      /* column role (sequential over i: fixed order) */
      dq_acc[k] += gG;
      dq_acc[m + k] += gGv * ux;
      dq_acc[2 * m + k] += gGv * uy;
      dq_abs[k] += fabs(gG);
      dq_abs[m + k] += fabs(gGv * ux);
      dq_abs[2 * m + k] += fabs(gGv * uy);
    }
    if (d_p) {
      d_p[2 * i] = ns_val(&px);
      d_p[2 * i + 1] = ns_val(&py);
    }
    if (abs_p) {
      abs_p[2 * i] = apx;
      abs_p[2 * i + 1] = apy;
    }
    if (d_z) {
      d_z[3 * i] = ns_val(&zxx);
      d_z[3 * i + 1] = ns_val(&zxy);
      d_z[3 * i + 2] = ns_val(&zyy);
    }
    if (abs_z) {
      abs_z[3 * i] = azxx;
      abs_z[3 * i + 1] = azxy;
      abs_z[3 * i + 2] = azyy;
    }
  }
  for (int64_t k = 0; k < m; ++k) {
    if (d_v) d_v[k] = dq_acc[k];
    if (abs_v) abs_v[k] = dq_abs[k];
    if (d_q) {
      d_q[2 * k] = dq_acc[m + k];
      d_q[2 * k + 1] = dq_acc[2 * m + k];
    }
    if (abs_q) {
      abs_q[2 * k] = dq_abs[m + k];
      abs_q[2 * k + 1] = dq_abs[2 * m + k];
    }
  }
  if (d_len) *d_len = ns_val(&len);
  if (abs_len) *abs_len = ns_val(&len_a);
  free(dq_acc);
  free(dq_abs);
}

/* Rounding sensitivities of the windowed reduction and its gradients, for
 * the tolerance of an FP32 evaluation (test infrastructure, not the method).
 * An FP32 pair evaluation rounds the difference d = p_i - q_k and the
 * window constants (each to relative error u), so the upper Cholesky factor
 * R of M = C_i^-1 (M = R^T R) applied to d, w = R d, is off by at most
 * 2u w^ with w^ = (|r11 dx| + |r12 dy|, |r22 dy|). With q = |w|^2 the
 * Gaussian factor exp(-q/2) is then off by a relative
 *   rho = 2 (|w1| w^1 + |w2| w^2) + q   (in units of u; q for the roundings
 * of the squares and their sum), and u = M d = R^T w by
 *   du_x = 2 |r11| w^1,  du_y = 2 (|r12| w^1 + |r22| w^2).
 * For a window elongated by a condition number kappa, rho grows like
 * q sqrt(kappa): far pairs of narrow windows carry the largest error. The
 * outputs (each may be NULL) sum, over the terms of each output, |term| rho
 * plus the terms' share through du:
 *   s_out[n]:   sum_k |G v| rho
 *   s_v[m]:     sum_i |g G| rho
 *   s_p[n][2], s_q[m][2]: sum |g G v| (|u| rho + du)
 *   s_z[n][3]:  (1/2) sum |g G v| ((u u^T + |M|) rho + d(u u^T)), the
 *               off-diagonal entry twice as in orc_windowed_vjp
 *   s_len[1]:   l sum_i (s_z[i][0] + s_z[i][2]). */
ORC_API void orc_windowed_rounding(const double* p, const double* z, int64_t n, const double* q, int64_t m,
                                   const double* v, double lengthscale, const double* g, double* s_out,
                                   double* s_v, double* s_p, double* s_q, double* s_z, double* s_len) {
  const double half_s = 0.5 * lengthscale * lengthscale;
  double* col = (double*)calloc((size_t)(3 * m + 1), sizeof(double));
  double len = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double cxx = z[3 * i] + half_s, cxy = z[3 * i + 1], cyy = z[3 * i + 2] + half_s;
    const double det = cxx * cyy - cxy * cxy;
    const double mxx = cyy / det, mxy = -cxy / det, myy = cxx / det;
    const double r11 = sqrt(cyy / det), r12 = -cxy / sqrt(cyy * det), r22 = 1.0 / sqrt(cyy);
    const double norm = 1.0 / (2.0 * PI * sqrt(det));
    const double gi = g ? fabs(g[i]) : 0.0;
    double so = 0, spx = 0, spy = 0, szx = 0, szxy = 0, szy = 0;
    for (int64_t k = 0; k < m; ++k) {
      const double dx = p[2 * i] - q[2 * k], dy = p[2 * i + 1] - q[2 * k + 1];
      const double w1 = r11 * dx + r12 * dy, w2 = r22 * dy;
      const double h1 = fabs(r11 * dx) + fabs(r12 * dy), h2 = fabs(r22 * dy);
      const double qq = w1 * w1 + w2 * w2;
      const double rho = 2.0 * (fabs(w1) * h1 + fabs(w2) * h2) + qq;
      const double G = norm * exp(-0.5 * qq);
      const double ux = mxx * dx + mxy * dy, uy = mxy * dx + myy * dy;
      const double dux = 2.0 * fabs(r11) * h1, duy = 2.0 * (fabs(r12) * h1 + fabs(r22) * h2);
      const double av = v ? fabs(v[k]) : 0.0;
      const double t = fabs(G) * av, tg = gi * t;
      so += t * rho;
      const double px = tg * (fabs(ux) * rho + dux), py = tg * (fabs(uy) * rho + duy);
      spx += px;
      spy += py;
      szx += 0.5 * tg * ((ux * ux + fabs(mxx)) * rho + 2.0 * fabs(ux) * dux);
      szxy += tg * ((fabs(ux * uy) + fabs(mxy)) * rho + fabs(ux) * duy + fabs(uy) * dux);
      szy += 0.5 * tg * ((uy * uy + fabs(myy)) * rho + 2.0 * fabs(uy) * duy);
      col[k] += gi * fabs(G) * rho;
      col[m + k] += px;
      col[2 * m + k] += py;
    }
    if (s_out) s_out[i] = so;
    if (s_p) {
      s_p[2 * i] = spx;
      s_p[2 * i + 1] = spy;
    }
    if (s_z) {
      s_z[3 * i] = szx;
      s_z[3 * i + 1] = szxy;
      s_z[3 * i + 2] = szy;
    }
    len += lengthscale * (szx + szy);
  }
  for (int64_t k = 0; k < m; ++k) {
    if (s_v) s_v[k] = col[k];
    if (s_q) {
      s_q[2 * k] = col[m + k];
      s_q[2 * k + 1] = col[2 * m + k];
    }
  }
  if (s_len) *s_len = len;
  free(col);
}

/* Gradient of Loss through the pixel windows: given dL/dZ (n x 3, the
 * off-diagonal entry counted in both positions as above), returns dL/dp
 * (n x 2) for the W x H grid of projected centres of orc_pixel_shapes, by
 * differentiating Z_i = (a a^T + b b^T)/(4 pi) and scattering the window
 * vectors' gradients onto the neighbours they are differences of. */
ORC_API void orc_pixel_shapes_vjp(const double* p, int32_t W, int32_t H, const double* dz, double* dp,
                                  double* dp_abs) {
  (void)p;
  memset(dp, 0, sizeof(double) * 2 * (size_t)W * (size_t)H);
  if (dp_abs) memset(dp_abs, 0, sizeof(double) * 2 * (size_t)W * (size_t)H);
  for (int64_t r = 0; r < H; ++r)
    for (int64_t c = 0; c < W; ++c) {
      const int64_t i = r * W + c;
      const int64_t cl = c > 0 ? i - 1 : i, cr = c + 1 < W ? i + 1 : i;
      const int64_t rd = r > 0 ? i - W : i, ru = r + 1 < H ? i + W : i;
      const double sa = (cr - cl == 2) ? 0.5 : 1.0, sb = (ru - rd == 2 * W) ? 0.5 : 1.0;
      const double ax = sa * (p[2 * cr] - p[2 * cl]), ay = sa * (p[2 * cr + 1] - p[2 * cl + 1]);
      const double bx = sb * (p[2 * ru] - p[2 * rd]), by = sb * (p[2 * ru + 1] - p[2 * rd + 1]);
      const double k = 1.0 / (4.0 * PI);
      const double gxx = dz[3 * i], gxy = dz[3 * i + 1], gyy = dz[3 * i + 2];
      /* Zxy = k (ax ay + bx by); its gradient gxy already counts both positions */
      const double dax = k * (2.0 * gxx * ax + gxy * ay), day = k * (gxy * ax + 2.0 * gyy * ay);
      const double dbx = k * (2.0 * gxx * bx + gxy * by), dby = k * (gxy * bx + 2.0 * gyy * by);
      dp[2 * cr] += sa * dax;
      dp[2 * cr + 1] += sa * day;
      dp[2 * cl] -= sa * dax;
      dp[2 * cl + 1] -= sa * day;
      dp[2 * ru] += sb * dbx;
      dp[2 * ru + 1] += sb * dby;
      dp[2 * rd] -= sb * dbx;
      dp[2 * rd + 1] -= sb * dby;
      if (dp_abs) {
        /* scales: the absolute terms of the same scatter */
        const double ax_ = k * (2.0 * fabs(gxx * ax) + fabs(gxy * ay)), ay_ = k * (fabs(gxy * ax) + 2.0 * fabs(gyy * ay));
        const double bx_ = k * (2.0 * fabs(gxx * bx) + fabs(gxy * by)), by_ = k * (fabs(gxy * bx) + 2.0 * fabs(gyy * by));
        const int64_t js[4] = {cr, cl, ru, rd};
        const double wx[4] = {sa * ax_, sa * ax_, sb * bx_, sb * bx_}, wy[4] = {sa * ay_, sa * ay_, sb * by_, sb * by_};
        for (int t = 0; t < 4; ++t) {
          dp_abs[2 * js[t]] += wx[t];
          dp_abs[2 * js[t] + 1] += wy[t];
        }
      }
    }
}

/* Inducing-point density (Sec. 3.4, footnote to the factorisation of the
 * covariance): rho(q_k) = k / (pi r_k^2) with r_k the distance from q_k to the
 * k-th closest OTHER point of the set (the point itself excluded by index;
 * coincident points count at distance 0). Writes r_k^2 for the rows listed
 * in `rows` (all m points when rows == NULL). Plain definition: every
 * squared distance in FP64, then the k-th smallest by repeated selection of
 * a bounded sorted list. */
ORC_API void orc_knn_r2(const double* q, int64_t m, int32_t k, const int64_t* rows, int64_t n_rows, double* r2) {
  const int64_t n = rows ? n_rows : m;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < n; ++t) {
    const int64_t i = rows ? rows[t] : t;
    double best[64];
    int32_t have = 0;
    for (int64_t j = 0; j < m; ++j) {
      if (j == i) continue;
      const double dx = q[2 * i] - q[2 * j], dy = q[2 * i + 1] - q[2 * j + 1];
      const double d2 = dx * dx + dy * dy;
      if (have == k && d2 >= best[k - 1]) continue;
      int32_t pos = have < k ? have++ : k - 1;
      while (pos > 0 && best[pos - 1] > d2) {
        best[pos] = best[pos - 1];
        --pos;
      }
      best[pos] = d2;
    }
    r2[t] = have == k ? best[k - 1] : INFINITY;
  }
}

/* ------------------------------------------------------------------------ */
/* Gradients of Loss = sum_i g_i out_i through the reduction, by
 * differentiating the RBF sum term by term (k_ij includes var):
 *   d_v_j   = sum_i g_i k_ij
 *   d_x_i   = g_i sum_j k_ij v_j (y_j - x_i) / l^2
 *   d_y_j   = sum_i g_i k_ij v_j (x_i - y_j) / l^2
 *   d_len   = sum_ij g_i v_j k_ij |x_i - y_j|^2 / l^3
 *   d_var   = sum_ij g_i v_j k_ij / var
 * For a self-kernel (x and y the same point set, `self` != 0) the point
 * gradient is the sum of both roles and is returned in d_x (d_y unused).
 * `scale` (optional, 10 arrays) receives the matching sums of absolute terms
 * (the scales of the parity tolerances): |d_v|, |d_x| (per component, both
 * roles), |d_y|, |d_len|, |d_var| in the order
 *   scale[0] = d_v_abs[m], scale[1] = d_x_abs[n][2], scale[2] = d_y_abs[m][2],
 *   scale[3] = d_len_abs[1], scale[4] = d_var_abs[1],
 * then the input-error sensitivities of the same outputs, scale[5..9]: if
 * every point moves by at most delta per coordinate, so that each pair
 * distance vector changes by at most D = 2 sqrt(2) delta, each output moves
 * by at most D times its sensitivity (to first order in D). Per pair, with
 * d = |d_ij| and k = var exp(-d^2 / (2 l^2)), |dk/dd| = k d / l^2, so
 *   k w d_c  changes by at most |w| k D (1 + d |d_c| / l^2),
 *   k w d^2  changes by at most |w| k D (2 d + d^3 / l^2),
 *   k w      changes by at most |w| k D d / l^2;
 * the sensitivities are these bounds without D, summed like the outputs.
 * Every output pointer may be NULL. */
ORC_API void orc_kernel_matvec_vjp(const double* x, int64_t n, const double* y, int64_t m, const double* v,
                                   double lengthscale, double variance, const double* g, int32_t self, double* d_v,
                                   double* d_x /*[n][2]*/, double* d_y /*[m][2]*/, double* d_len, double* d_var,
                                   double* const* scale /* [10] or NULL */) {
  const double l2 = lengthscale * lengthscale, inv2l2 = 1.0 / (2.0 * l2);
  double* s_dv = scale ? scale[0] : NULL;
  double* s_dx = scale ? scale[1] : NULL;
  double* s_dy = scale ? scale[2] : NULL;
  double* e_dv = scale ? scale[5] : NULL;
  double* e_dx = scale ? scale[6] : NULL;
  double* e_dy = scale ? scale[7] : NULL;
  nsum tl = {0, 0}, tv = {0, 0}, tla = {0, 0}, tva = {0, 0}, tle = {0, 0}, tve = {0, 0};
  /* row pass: d_x (row role), d_len, d_var */
#pragma omp parallel
  {
    nsum ll = {0, 0}, lv = {0, 0}, lla = {0, 0}, lva = {0, 0}, lle = {0, 0}, lve = {0, 0};
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      const double xi = x[2 * i], yi = x[2 * i + 1];
      nsum sx = {0, 0}, sy = {0, 0}, sl = {0, 0}, sv = {0, 0}, ax = {0, 0}, ay = {0, 0}, al = {0, 0}, av = {0, 0};
      nsum ex = {0, 0}, ey = {0, 0}, el = {0, 0}, ev = {0, 0};
      for (int64_t j = 0; j < m; ++j) {
        const double dx = y[2 * j] - xi, dy = y[2 * j + 1] - yi;
        const double d2 = dx * dx + dy * dy;
        if (d2 * inv2l2 > EXP_ZERO) continue;
        const double d = sqrt(d2);
        const double kv = variance * exp(-d2 * inv2l2) * v[j];
        ns_add(&sx, kv * dx);
        ns_add(&sy, kv * dy);
        ns_add(&sl, kv * d2);
        ns_add(&sv, kv);
        ns_add(&ax, fabs(kv * dx));
        ns_add(&ay, fabs(kv * dy));
        ns_add(&al, fabs(kv) * d2);
        ns_add(&av, fabs(kv));
        ns_add(&ex, fabs(kv) * (1.0 + d * fabs(dx) / l2));
        ns_add(&ey, fabs(kv) * (1.0 + d * fabs(dy) / l2));
        ns_add(&el, fabs(kv) * (2.0 * d + d * d2 / l2));
        ns_add(&ev, fabs(kv) * d / l2);
      }
      if (d_x) {
        d_x[2 * i] = g[i] * ns_val(&sx) / l2;
        d_x[2 * i + 1] = g[i] * ns_val(&sy) / l2;
      }
      if (s_dx) {
        s_dx[2 * i] = fabs(g[i]) * ns_val(&ax) / l2;
        s_dx[2 * i + 1] = fabs(g[i]) * ns_val(&ay) / l2;
      }
      if (e_dx) {
        e_dx[2 * i] = fabs(g[i]) * ns_val(&ex) / l2;
        e_dx[2 * i + 1] = fabs(g[i]) * ns_val(&ey) / l2;
      }
      ns_add(&ll, g[i] * ns_val(&sl) / (l2 * lengthscale));
      ns_add(&lv, g[i] * ns_val(&sv) / variance);
      ns_add(&lla, fabs(g[i]) * ns_val(&al) / (l2 * lengthscale));
      ns_add(&lva, fabs(g[i]) * ns_val(&av) / fabs(variance));
      ns_add(&lle, fabs(g[i]) * ns_val(&el) / (l2 * lengthscale));
      ns_add(&lve, fabs(g[i]) * ns_val(&ev) / fabs(variance));
    }
#pragma omp critical
    {
      ns_add(&tl, ll.s);
      ns_add(&tl, ll.c);
      ns_add(&tv, lv.s);
      ns_add(&tv, lv.c);
      ns_add(&tla, lla.s);
      ns_add(&tla, lla.c);
      ns_add(&tva, lva.s);
      ns_add(&tva, lva.c);
      ns_add(&tle, lle.s);
      ns_add(&tle, lle.c);
      ns_add(&tve, lve.s);
      ns_add(&tve, lve.c);
    }
  }
  if (d_len) *d_len = ns_val(&tl);
  if (d_var) *d_var = ns_val(&tv);
  if (scale && scale[3]) *scale[3] = ns_val(&tla);
  if (scale && scale[4]) *scale[4] = ns_val(&tva);
  if (scale && scale[8]) *scale[8] = ns_val(&tle);
  if (scale && scale[9]) *scale[9] = ns_val(&tve);
  /* column pass: d_v, d_y (column role) */
  double* col = (double*)calloc((size_t)(6 * m), sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < m; ++j) {
    const double yj = y[2 * j], zj = y[2 * j + 1];
    nsum s = {0, 0}, sx = {0, 0}, sy = {0, 0}, as = {0, 0}, ax = {0, 0}, ay = {0, 0};
    nsum es = {0, 0}, ex = {0, 0}, ey = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
      const double dx = x[2 * i] - yj, dy = x[2 * i + 1] - zj;
      const double d2 = dx * dx + dy * dy;
      if (d2 * inv2l2 > EXP_ZERO) continue;
      const double d = sqrt(d2);
      const double gk = g[i] * variance * exp(-d2 * inv2l2);
      ns_add(&s, gk);
      ns_add(&sx, gk * dx);
      ns_add(&sy, gk * dy);
      ns_add(&as, fabs(gk));
      ns_add(&ax, fabs(gk * dx));
      ns_add(&ay, fabs(gk * dy));
      ns_add(&es, fabs(gk) * d / l2);
      ns_add(&ex, fabs(gk) * (1.0 + d * fabs(dx) / l2));
      ns_add(&ey, fabs(gk) * (1.0 + d * fabs(dy) / l2));
    }
    if (d_v) d_v[j] = ns_val(&s);
    if (s_dv) s_dv[j] = ns_val(&as);
    if (e_dv) e_dv[j] = ns_val(&es);
    col[6 * j] = v[j] * ns_val(&sx) / l2;
    col[6 * j + 1] = v[j] * ns_val(&sy) / l2;
    col[6 * j + 2] = fabs(v[j]) * ns_val(&ax) / l2;
    col[6 * j + 3] = fabs(v[j]) * ns_val(&ay) / l2;
    col[6 * j + 4] = fabs(v[j]) * ns_val(&ex) / l2;
    col[6 * j + 5] = fabs(v[j]) * ns_val(&ey) / l2;
  }
  if (self) {
    for (int64_t i = 0; i < n; ++i) {
      if (d_x) {
        d_x[2 * i] += col[6 * i];
        d_x[2 * i + 1] += col[6 * i + 1];
      }
      if (s_dx) {
        s_dx[2 * i] += col[6 * i + 2];
        s_dx[2 * i + 1] += col[6 * i + 3];
      }
      if (e_dx) {
        e_dx[2 * i] += col[6 * i + 4];
        e_dx[2 * i + 1] += col[6 * i + 5];
      }
    }
  } else {
    for (int64_t j = 0; j < m; ++j) {
      if (d_y) {
        d_y[2 * j] = col[6 * j];
        d_y[2 * j + 1] = col[6 * j + 1];
      }
      if (s_dy) {
        s_dy[2 * j] = col[6 * j + 2];
        s_dy[2 * j + 1] = col[6 * j + 3];
      }
      if (e_dy) {
        e_dy[2 * j] = col[6 * j + 4];
        e_dy[2 * j + 1] = col[6 * j + 5];
      }
    }
  }
  free(col);
}

/* The self-kernel gradients of orc_kernel_matvec_vjp (x = y, both roles) on
 * the listed rows only, for sampled parity at sizes where the full n x n
 * sweep is out of reach. For each listed row i, with k_ij = var
 * exp(-|x_i - x_j|^2 / (2 l^2)) and d_ij = x_j - x_i:
 *   out[r]  = sum_j k_ij v_j          (the forward reduction, with s_out = sum |k v|)
 *   d_v[r]  = sum_j k_ij g_j
 *   d_x[r]  = [g_i sum_j k_ij v_j d_ij + v_i sum_j k_ij g_j d_ij] / l^2
 * (the row role plus the column role of point i), the sums of absolute terms
 * (s_dv, s_dx) and the input-error sensitivities (e_dv, e_dx) defined as for
 * orc_kernel_matvec_vjp. Any output may be NULL. */
ORC_API void orc_self_vjp_rows(const double* x, int64_t n, const double* v, const double* g, double lengthscale,
                               double variance, const int64_t* rows, int64_t n_rows, double* out, double* s_out,
                               double* d_v, double* d_x, double* s_dv, double* s_dx, double* e_dv, double* e_dx) {
  const double l2 = lengthscale * lengthscale, inv2l2 = 1.0 / (2.0 * l2);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t r = 0; r < n_rows; ++r) {
    const int64_t i = rows[r];
    const double xi = x[2 * i], yi = x[2 * i + 1];
    nsum kg = {0, 0}, akg = {0, 0}, ekg = {0, 0}, kvs = {0, 0}, akv = {0, 0};
    nsum rx = {0, 0}, ry = {0, 0}, cx = {0, 0}, cy = {0, 0};
    nsum arx = {0, 0}, ary = {0, 0}, acx = {0, 0}, acy = {0, 0};
    nsum erx = {0, 0}, ery = {0, 0}, ecx = {0, 0}, ecy = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      const double dx = x[2 * j] - xi, dy = x[2 * j + 1] - yi;
      const double d2 = dx * dx + dy * dy;
      if (d2 * inv2l2 > EXP_ZERO) continue;
      const double d = sqrt(d2);
      const double k = variance * exp(-d2 * inv2l2);
      const double kv = k * v[j], kgj = k * g[j];
      const double fx = 1.0 + d * fabs(dx) / l2, fy = 1.0 + d * fabs(dy) / l2;
      ns_add(&kvs, kv);
      ns_add(&akv, fabs(kv));
      ns_add(&kg, kgj);
      ns_add(&akg, fabs(kgj));
      ns_add(&ekg, fabs(kgj) * d / l2);
      ns_add(&rx, kv * dx);
      ns_add(&ry, kv * dy);
      ns_add(&cx, kgj * dx);
      ns_add(&cy, kgj * dy);
      ns_add(&arx, fabs(kv * dx));
      ns_add(&ary, fabs(kv * dy));
      ns_add(&acx, fabs(kgj * dx));
      ns_add(&acy, fabs(kgj * dy));
      ns_add(&erx, fabs(kv) * fx);
      ns_add(&ery, fabs(kv) * fy);
      ns_add(&ecx, fabs(kgj) * fx);
      ns_add(&ecy, fabs(kgj) * fy);
    }
    const double gi = g[i], vi = v[i];
    if (out) out[r] = ns_val(&kvs);
    if (s_out) s_out[r] = ns_val(&akv);
    if (d_v) d_v[r] = ns_val(&kg);
    if (s_dv) s_dv[r] = ns_val(&akg);
    if (e_dv) e_dv[r] = ns_val(&ekg);
    if (d_x) {
      d_x[2 * r] = (gi * ns_val(&rx) + vi * ns_val(&cx)) / l2;
      d_x[2 * r + 1] = (gi * ns_val(&ry) + vi * ns_val(&cy)) / l2;
    }
    if (s_dx) {
      s_dx[2 * r] = (fabs(gi) * ns_val(&arx) + fabs(vi) * ns_val(&acx)) / l2;
      s_dx[2 * r + 1] = (fabs(gi) * ns_val(&ary) + fabs(vi) * ns_val(&acy)) / l2;
    }
    if (e_dx) {
      e_dx[2 * r] = (fabs(gi) * ns_val(&erx) + fabs(vi) * ns_val(&ecx)) / l2;
      e_dx[2 * r + 1] = (fabs(gi) * ns_val(&ery) + fabs(vi) * ns_val(&ecy)) / l2;
    }
  }
}

/* Threads of the oracle's OpenMP loops from here on (the benchmark's
 * one-core timing sets 1, then restores the default). */
ORC_API void orc_set_num_threads(int32_t n) { omp_set_num_threads(n > 0 ? n : 1); }

/* Number of OpenMP threads the oracle runs with (reported by the benchmark). */
ORC_API int32_t orc_num_threads(void) {
  int32_t t = 1;
#pragma omp parallel
  {
#pragma omp single
    {
      t = (int32_t)omp_get_num_threads();
    }
  }
  return t;
}
