/*
 * lensgp — C ABI of the GB300 (sm_103a) lens ray-trace and Gaussian-kernel
 * reduction library.
 *
 * Method: Karchev, Coogan & Weniger, "Strong-lensing source reconstruction
 * with variationally optimised Gaussian processes" (arXiv:2105.09465).
 *
 * Conventions shared by every entry point
 *  - Array arguments are DEVICE pointers owned by the caller unless stated
 *    otherwise; the library never frees them and keeps no reference after the
 *    call returns.
 *  - Compute entry points are stream-ordered and asynchronous: they enqueue
 *    work on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *    return without synchronising. Results are valid once the stream reaches
 *    that point.
 *  - Every argument is validated on the host before anything is enqueued; a
 *    call that returns anything but LR_OK has enqueued nothing. No C++
 *    exception crosses the ABI. lr_last_error() returns a message describing
 *    the most recent failure on the calling thread.
 *  - Angles (positions, Einstein radii, length scales) are in arcseconds.
 */
#ifndef LENSGP_H
#define LENSGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lr_status;
enum {
  LR_OK = 0,
  LR_ERR_INVALID_ARG = 1,   /* bad pointer, size, or parameter outside its domain */
  LR_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed        */
  LR_ERR_OUT_OF_MEMORY = 3, /* device allocation failed or admission budget hit   */
  LR_ERR_TIMEOUT = 4,       /* a bounded wait ran out                            */
  LR_PENDING = 5,           /* result not ready yet (polling)                    */
  LR_ERR_NOT_FOUND = 6,     /* unknown ticket / handle                           */
  LR_ERR_BUSY = 7           /* no free slot right now                            */
};

/* A CUDA stream (cudaStream_t / CUstream); NULL = the legacy default stream. */
typedef struct CUstream_st* lr_stream;

/* Message for the most recent failure on this thread ("" if none). */
const char* lr_last_error(void);
/* Symbolic name of a status code, e.g. "LR_ERR_INVALID_ARG". */
const char* lr_status_name(lr_status s);

/*
 * Measures, on `device`, the FP32 FMA lanes (scalar FFMA and packed FFMA2)
 * and MUFU.EX2 results that one SM retires per SM clock (median over SMs),
 * and reports the SM count. These are the denominators of the ALU roofline
 * that pair-evaluation throughput is quoted against. Synchronous; allocates
 * and frees a few KB of device memory; takes a few milliseconds.
 */
lr_status lr_probe_pipe_rates(int32_t device, double* ffma_lanes_per_clk,
                              double* ffma2_lanes_per_clk, double* ex2_per_clk,
                              int32_t* sm_count);

/*
 * Reads (and with clear != 0 resets) the device fault word of the current
 * device. Kernels never trap: a bounded wait that runs out records a nonzero
 * code here (1 = an mbarrier wait for a bulk copy timed out) and the kernel
 * returns early. Synchronous.
 */
lr_status lr_fault_status(int32_t* code, int32_t clear);

/*
 * Self-test of the bounded waits (no paper counterpart): launches one thread
 * that arms an mbarrier for a bulk-copy transaction that never comes and
 * waits for it with a budget of `budget_cycles` SM clocks (0 < budget <= 2e9).
 * The wait runs out, the kernel records kFaultBarrierTimeout (1) in the
 * fault word (read it with lr_fault_status) and returns; *code = 1 says it
 * returned after giving up (2 would mean the wait completed). Nothing is in
 * flight when it gives up, so the context stays usable. Synchronous;
 * allocates 4 bytes of device memory.
 */
lr_status lr_selftest_bounded_wait(int64_t budget_cycles, int32_t* code);

/*
 * Launch timer: device time of the library's pair-sweep kernels alone,
 * without the pre-pass and merge launches of the same entry point (the
 * denominator of a per-kernel roofline). lr_kernel_timer_enable(1) makes the
 * current device the timed one and clears earlier records; from then on each
 * launch of a kernel below, from any single-problem entry point on that
 * device, records a CUDA event before and after it on its stream (not while
 * the stream is capturing a graph, and not past 8192 launches: those count as
 * dropped). lr_kernel_timer_enable(0) stops recording and keeps the records.
 * lr_kernel_timer_read waits for the recorded events of `kernel` and returns
 * the launch count and the summed milliseconds (and, if `dropped` is not NULL,
 * the number of launches that were not recorded). Host-thread safe; timing is
 * for profiling runs, since each record adds two event records to the stream.
 */
enum {
  LR_KT_MATVEC = 0,       /* gp_kernel_matvec pair sweep (matvec_kernel)                */
  LR_KT_TRAIN_ROWS = 1,   /* gp_kernel_matvec_train pair sweep (out + row moments)      */
  LR_KT_BWD_ROWS = 2,     /* gp_kernel_matvec_bwd row sweep without moments             */
  LR_KT_DV_ROWS = 3,      /* gp_kernel_matvec_bwd d_v sweep (grid sources)              */
  LR_KT_RAYTRACE = 4,     /* lens_raytrace                                              */
  LR_KT_RAYTRACE_VJP = 5, /* lens_raytrace_vjp                                          */
  LR_KT_WINDOWED = 6,     /* gp_windowed_matvec pair sweep                              */
  LR_KT_COUNT = 7
};
lr_status lr_kernel_timer_enable(int32_t enable);
lr_status lr_kernel_timer_read(int32_t kernel, int64_t* launches, double* total_ms, int64_t* dropped);

/*
 * Exact skipping of far pairs in the reductions over explicit sources
 * (gp_kernel_matvec, gp_kernel_matvec_bwd). A pair whose exponent is below
 * -126 contributes exactly 0 (the hardware exp2 flushes it), so a row block
 * leaves out every source chunk that is that far from all its rows.
 * lr_set_pair_culling(0) makes those entry points evaluate every pair, in
 * the same order; the results are bitwise the same, which is what it is for
 * (checking that the skipping is exact). Process-wide, read at each call;
 * on (1) by default.
 */
lr_status lr_set_pair_culling(int32_t enable);

/* ------------------------------------------------------------------------ */
/* Geometry and lens parameters                                               */

/*
 * Image-plane pixel grid (the pixel centres P of the paper's Table 1).
 * S x S supersampling of an nx x ny grid of spacing `pix` is the
 * (nx*ss) x (ny*ss) grid of spacing h = pix/ss (FP32 division). Point k,
 * with row = k / (nx*ss) and col = k % (nx*ss), sits at the FP32 value
 *   x = fmaf(col - (nx*ss - 1)/2, h, cx),  y = fmaf(row - (ny*ss - 1)/2, h, cy).
 * Also used for regular grids of inducing points in the source plane.
 */
typedef struct {
  int32_t nx, ny, ss;
  float pix, cx, cy;
} lr_grid;

/*
 * Lens parameters in the paper's order (Sec. 2.2): SPLE centre (x0, y0),
 * axis ratio q in (0, 1], orientation phi [rad], Einstein radius theta_e,
 * 3-D density slope gamma in (1, 3) (2 = isothermal), external shear
 * (g1, g2) acting about the origin. The SPLE deflection is the
 * hypergeometric closed form of Sec. 2.2, evaluated as its power series in
 * e^{2 i phi_e}; axis ratios below ~0.12 need more than 96 terms and are
 * rejected with LR_ERR_INVALID_ARG.
 */
typedef struct {
  float x0, y0, q, phi, theta_e, gamma, g1, g2;
} lr_lens;

/*
 * Subhalo profiles. Records are float[5] per subhalo, device memory,
 * 16-byte aligned base for the fast staging path (any 4-byte aligned base
 * works, more slowly):
 *  LR_PROFILE_TNFW:       (x_h, y_h, kappa_s, theta_s, tau) — truncated NFW
 *                         of Baltz, Marshall & Oguri (2009), kappa_s =
 *                         rho_s r_s / Sigma_cr, theta_s = r_s / D_l,
 *                         tau = r_t / r_s. Substructure is not part of the
 *                         paper (Sec. 2.2 defers it); this is the standard
 *                         profile for it.
 *  LR_PROFILE_POINT_MASS: (x_h, y_h, theta_pm, unused, unused) — deflection
 *                         theta_pm^2 d / |d|^2.
 */
enum { LR_PROFILE_TNFW = 0, LR_PROFILE_POINT_MASS = 1 };

/*
 * A point set: explicit FP32 positions or a grid, optionally ray-traced
 * through a lens (then the set is the source-plane positions
 * beta = xi - alpha(xi) of the image-plane points xi, eq. for the raytracing
 * equation, Sec. 2.1).
 *   xy      device float[n][2], or NULL to use `grid`
 *   grid    used when xy == NULL (then n must equal its point count)
 *   lens    host pointer; NULL = no ray-trace (positions used as given)
 *           unless lens_record is set
 *   sub, n_sub, profile   subhalos, used only when lens != NULL
 */
typedef struct {
  const float* xy;
  lr_grid grid;
  int64_t n;
  const lr_lens* lens;
  const float* sub;
  int32_t n_sub;
  int32_t profile;
  const void* lens_record; /* or: a DEVICE lens record (lr_lens_prepare) in place of `lens` */
} lr_points;

/*
 * Device-resident lens parameters (a lens drawn on the device, e.g. by
 * gp_partial_mvn_draw, never copied to the host). lr_lens_prepare computes,
 * on `stream`, the lens constants of the ray-trace and of its gradient from
 * theta7 (device float[7]: x0, y0, q, phi, theta_e, g1, g2, the slope held
 * fixed at `gamma`) into `record` (device memory of lr_lens_record_bytes()
 * bytes, 16-byte aligned, owned by the caller). A point set with
 * lens_record = record is then ray-traced (lens_raytrace, gp_kernel_matvec*,
 * gp_kernel_matvec_bwd, lens_raytrace_vjp) with that lens and no host
 * synchronisation. Parameters outside their domain (q not in (0, 1], slope
 * not in (1, 3), theta_e < 0, a non-finite value, or q too small for the
 * series) cannot be rejected when the call is made: the record is marked
 * invalid, the ray-trace kernels record fault code 2 in the device fault
 * word (lr_fault_status), and their outputs, finite but not to be used, are
 * those of a main deflector and shear that deflect nothing.
 */
size_t lr_lens_record_bytes(void);
lr_status lr_lens_prepare(const float* theta7, float gamma, void* record, lr_stream stream);

/* ------------------------------------------------------------------------ */
/* Ray-trace (Sec. 2.1 raytracing equation; Sec. 2.2 lens model)              */

/*
 * beta_i = xi_i - alpha(xi_i) for every point of `pts` (which must carry a
 * lens), alpha = alpha_SPLE + alpha_shear + sum_h alpha_h. The subhalo sum is
 * Kahan-compensated in FP32.
 *   beta_out   device float[n][2] (required)
 *   alpha_out  device float[n][2] or NULL
 * Errors: LR_ERR_INVALID_ARG for NULL/misaligned pointers, n < 0, a grid
 * whose size differs from n, lens parameters outside their domain or
 * non-finite. n == 0 is a no-op.
 */
lr_status lens_raytrace(const lr_points* pts, float* beta_out, float* alpha_out, lr_stream stream);

/*
 * The FP32 points of a grid (the pixel centres P of Table 1, supersampled as
 * lr_grid defines them) into out (device float[n][2], row-major). Exactly
 * the points every entry point generates for a grid argument, e.g. for
 * splitting an image's rows across GPUs.
 */
lr_status lr_grid_points(const lr_grid* grid, float* out, lr_stream stream);

/*
 * Lens Jacobian and magnification (Sec. 2.1, lens-Jacobian and magnification
 * equations): for every point of `pts` (which must carry a lens),
 *   jac_out[i] = d beta / d xi = I - d alpha / d xi, row-major float[4]
 *                (A_xx, A_xy, A_yx, A_yy), A_xy = d beta_x / d y,
 *   mu_out[i]  = 1 / det(jac) (signed; infinite on critical curves).
 * Either output may be NULL. jac_out must be 16-byte aligned.
 */
lr_status lens_jacobian(const lr_points* pts, float* jac_out, float* mu_out, lr_stream stream);

/* ------------------------------------------------------------------------ */
/* Gaussian-kernel reduction (Sec. 3.1 RBF kernel; Sec. 3.3 lazy T y)         */

/*
 * out_i = sum_j variance * exp(-|x_i - y_j|^2 / (2 lengthscale^2)) v_j
 * (the RBF covariance of Sec. 3.1 with isotropic kernel Sigma = l^2 I,
 * reduced lazily without storing the n x m matrix, Sec. 3.3).
 *   query   the x_i; ray-traced first when query->lens != NULL
 *   source  the y_j, or NULL for a self-kernel (y = x after ray-tracing)
 *   v       device float[m][nrhs]: nrhs = 1..4 right-hand sides reduced in
 *           one pass (one exponential per pair, nrhs FMA); with grid sources
 *           and nrhs > 1 the grid's points are written to the workspace and
 *           reduced like explicit sources
 *   out     device float[n][nrhs]
 *   beta_out device float[n][2] or NULL: receives the ray-traced query points
 *   workspace/workspace_bytes: caller-owned device scratch of at least
 *           lr_matvec_workspace_size() bytes (may be NULL when that is 0)
 * FP32 arithmetic: distances by FMA, exp through the hardware exp2, per-tile
 * partial sums merged with Kahan compensation. Deterministic: the same inputs
 * give bit-identical outputs. Pairs far enough apart that their FP32 kernel
 * value is exactly 0 are left out (see lr_set_pair_culling); points that
 * carry an image layout (a grid query, or explicit points whose lr_points
 * grid matches their count, e.g. ray-traced pixels) are grouped by image
 * tiles, which is what makes the skipping effective.
 * Errors: LR_ERR_INVALID_ARG (pointers, sizes, lengthscale <= 0, variance
 * not finite, workspace too small), LR_ERR_CUDA (launch failure).
 */
lr_status gp_kernel_matvec(const lr_points* query, const lr_points* source, const float* v, int32_t nrhs,
                           float lengthscale, float variance, float* out, float* beta_out, void* workspace,
                           size_t workspace_bytes, lr_stream stream);

/*
 * Multi-layer reduction (Sec. 3.1, sum of RBF layers with fixed length
 * scales and per-layer variances): with L = n_layers in [1, 4] and nrhs in
 * [1, 4] right-hand sides (e.g. several draws of the layers' weights),
 *   out[i][h] = sum_l variances[l] sum_j exp(-|x_i - y_j|^2 / (2 lengthscales[l]^2)) v[l][j][h].
 * The pair distance is formed once for all layers, and each layer's exp2
 * once for all right-hand sides. lengthscales and variances are HOST
 * float[L]; v is device float[L][m][nrhs] (layer-major), out device
 * float[n][nrhs]. Sources may be explicit or a grid, or NULL for a
 * self-kernel (the paper's image-plane GP); they may not carry a lens.
 * Other arguments as gp_kernel_matvec; workspace of
 * lr_matvec_layers_workspace_size() bytes.
 */
lr_status gp_kernel_matvec_layers(const lr_points* query, const lr_points* source, int32_t n_layers,
                                  const float* lengthscales, const float* variances, const float* v, int32_t nrhs,
                                  float* out, float* beta_out, void* workspace, size_t workspace_bytes,
                                  lr_stream stream);
lr_status lr_matvec_layers_workspace_size(const lr_points* query, const lr_points* source, int32_t n_layers,
                                          int32_t nrhs, size_t* bytes);

/* ------------------------------------------------------------------------ */
/* Pixel windows (Sec. 3.2) and the windowed transmission (Sec. 3.4)          */

/*
 * Window covariances of a W x H grid of projected pixel centres p (device
 * float[W*H][2], row-major over grid y, e.g. lens_raytrace of an lr_grid):
 * a_i / b_i = half the vector between the two centres adjacent along grid
 * x / y (the vector to the single neighbour at the border), and
 *   z[i] = (Zxx, Zxy, Zyy) of Z_i = (a_i a_i^T + b_i b_i^T) / (4 pi)
 * (window-kernel equation). z: device float[W*H][3].
 */
lr_status gp_pixel_shapes(const float* p, int32_t W, int32_t H, float* z, lr_stream stream);

/*
 * Windowed (non-stationary) transmission reduction (transmission equation
 * with Sigma = l^2 I):
 *   out_i = sum_k G(p_i - q_k, Z_i + (l^2/2) I) v_k,
 *   G(d, C) = exp(-d^T C^-1 d / 2) / (2 pi sqrt(det C)),
 * for n query points p (device float[n][2]) with window covariances z
 * (device float[n][3], from gp_pixel_shapes; zeros give point pixels) and
 * sources q (explicit or grid, no lens). The caller folds the transmission
 * weights A_k into v_k. Workspace of lr_windowed_workspace_size() bytes.
 *   layout  NULL, or the image grid the n query points come from (row-major,
 *           nx*ss x ny*ss == n; only its shape is read): the sweeps then take
 *           the rows in compact image tiles. Explicit sources are ordered the
 *           same way when source->grid describes them (lr_points).
 * Explicit sources: pairs whose exponent is below -126 (they contribute
 * exactly 0 in FP32) are skipped by bounding boxes, with the reach of each
 * row's widest window direction; lr_set_pair_culling(0) evaluates them all,
 * with bitwise the same results.
 */
lr_status gp_windowed_matvec(const float* p, const float* z, int64_t n, const lr_grid* layout,
                             const lr_points* source, const float* v, float lengthscale, float* out, void* workspace,
                             size_t workspace_bytes, lr_stream stream);
lr_status lr_windowed_workspace_size(int64_t n, const lr_grid* layout, const lr_points* source, size_t* bytes);

/*
 * The windowed reduction with the Gaussian pixel likelihood (Sec. 3.3) in its
 * epilogue, for the last layer of the model: with one value per pixel,
 *   out_i = f_in_i + sum_k G(p_i - q_k, Z_i + (l^2/2) I) v_k   (f_in may be NULL: 0),
 *   g_i   = (out_i - data_i) / sigma^2                          (dL/dout),
 *   nll   = sum_i (out_i - data_i)^2 / (2 sigma^2) + n ln sigma + (n/2) ln 2 pi
 * (device double[1]; FP32 per row, FP64 across rows, fixed order). The rows'
 * terms are formed where the reduction finishes each row, so the model total
 * is never re-read. Explicit sources only; other arguments, the workspace
 * (lr_windowed_workspace_size) and the skipping of exact zeros as for
 * gp_windowed_matvec. out, g: device float[n]; data device float[n].
 */
lr_status gp_windowed_matvec_nll(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                 const lr_points* source, const float* v, float lengthscale, const float* f_in,
                                 const float* data, float sigma, float* out, float* g, double* nll, void* workspace,
                                 size_t workspace_bytes, lr_stream stream);

/*
 * Gradients of Loss = sum_i g_i out_i through gp_windowed_matvec
 * (recompute-only). With d = p_i - q_k, C_i = Z_i + (l^2/2) I, M = C_i^-1,
 * u = M d and G = G(d, C_i):
 *   d_p[i] = -g_i sum_k v_k G u,          d_q[k] = v_k sum_i g_i G u,
 *   d_v[k] = sum_i g_i G,
 *   d_z[i] = g_i sum_k v_k G (u u^T - M)/2 as (xx, 2 xy, yy): the gradient
 *            with respect to (Zxx, Zxy, Zyy), the off-diagonal entry
 *            counted in both symmetric positions,
 *   d_lengthscale = l sum_i tr(d_z-matrix_i)  (device double[1]).
 * Sources must be explicit points (grid sources: use the stationary
 * reduction, which is what the windowed form reduces to without windows).
 * For an image-plane layer with q = p the total gradient of a point is
 * d_p + d_q + gp_pixel_shapes_vjp(d_z). Every output may be NULL; the row
 * sweep runs for d_p, d_z or d_lengthscale, the column sweep for d_v or d_q.
 * `layout` and the skipping of exact zeros as for gp_windowed_matvec (both
 * sweeps). Workspace of lr_windowed_bwd_workspace_size() bytes, 256-byte
 * aligned.
 */
lr_status gp_windowed_matvec_bwd(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                 const lr_points* source, const float* v, float lengthscale, const float* g,
                                 float* d_v, float* d_p, float* d_q, float* d_z, double* d_lengthscale,
                                 void* workspace, size_t workspace_bytes, lr_stream stream);
lr_status lr_windowed_bwd_workspace_size(int64_t n, const lr_grid* layout, const lr_points* source, size_t* bytes);

/*
 * Diagnostic: the pairs the windowed sweeps over explicit sources evaluate
 * (sweep 0: gp_windowed_matvec; 1: the backward's row sweep; 2: its column
 * sweep), counted like lr_cull_pairs_evaluated. Synchronises the stream;
 * allocates and frees its own temporary device memory.
 */
lr_status lr_windowed_pairs_evaluated(const float* p, const float* z, int64_t n, const lr_grid* layout,
                                      const lr_points* source, float lengthscale, int32_t sweep, int64_t* pairs,
                                      int64_t* slots, lr_stream stream);

/*
 * Gradient through gp_pixel_shapes: dp (device float[W*H][2], overwritten)
 * = dL/dp given dz = dL/d(Zxx, Zxy, Zyy) (device float[W*H][3], off-diagonal
 * counted in both positions) for the W x H grid of projected centres p.
 */
lr_status gp_pixel_shapes_vjp(const float* p, int32_t W, int32_t H, const float* dz, float* dp, lr_stream stream);

/*
 * Inducing-point density (Sec. 3.4, footnote to the covariance factorisation)
 * and the transmission weights it sets, for m points q (device float[m][2]):
 *   r2_out[i] = r_k(q_i)^2, the squared distance to the k-th closest OTHER
 *               point of q (the point itself excluded by index; coincident
 *               points count at distance 0), FP32;
 *   a_out[i]  = A_i = |2 pi Sigma|^(1/4) / sqrt(rho_i) with rho_i = k / (pi r2_i)
 *               and Sigma = lengthscale^2 I, i.e. pi l sqrt(2 r2_i / k).
 * Either output may be NULL (not both); lengthscale is read only for a_out.
 * 1 <= k <= 32 and m >= k + 1, else LR_ERR_INVALID_ARG. Workspace of
 * lr_knn_workspace_size(m) bytes, 256-byte aligned, owned by the caller.
 * Cost grows with the number of points per occupied cell of a uniform grid
 * over the bounding box: far outliers that stretch the box make it slower,
 * never wrong.
 */
lr_status gp_knn_density(const float* q, int64_t m, int32_t k, float lengthscale, float* r2_out, float* a_out,
                         void* workspace, size_t workspace_bytes, lr_stream stream);
lr_status lr_knn_workspace_size(int64_t m, size_t* bytes);

/* ------------------------------------------------------------------------ */
/* Likelihood and ELBO terms (Sec. 3.3 generative model, Sec. 3.6 ELBO,       */
/* Sec. 3.7 mean-field proposal, Sec. 4.2 partial MVN proposal)               */
/*
 * The loss of one reparameterised draw is
 *   nll(d | f) - ln p(y | alpha) + ln q(y)          (minus the ELBO estimate).
 * Every scalar below is an FP64 sum taken in an order fixed by the sizes
 * alone (bit-reproducible). Scalars are written to DEVICE memory. The
 * functions taking a workspace need lr_elbo_workspace_size() bytes, 256-byte
 * aligned; one workspace serves one call at a time on a stream.
 */
size_t lr_elbo_workspace_size(void);

/*
 * Gaussian pixel likelihood of supersampled model fluxes f (device float[n]):
 * the model of pixel p is the mean of its ss x ss subpixels (grid != NULL,
 * f in grid-point order, n = (nx ss)(ny ss); grid == NULL: one value per
 * pixel), and
 *   nll = sum_p (m_p - d_p)^2 / (2 s_p^2) + ln s_p  +  (P/2) ln 2 pi,
 * s_p = sigma[p] (device float[P]) or sigma0 when sigma == NULL.
 * Optional outputs: g_out[n] = d nll / d f = (m_p - d_p) / (s_p^2 ss^2) for
 * every subpixel of p, model_out[P] = m_p. nll_out: device double[1].
 */
lr_status gp_gaussian_nll(const float* f, int64_t n, const lr_grid* grid, const float* data, const float* sigma,
                          float sigma0, float* g_out, float* model_out, double* nll_out, void* workspace,
                          size_t workspace_bytes, lr_stream stream);

/*
 * Diagonal-normal proposal of m source parameters (Sec. 3.7) with prior
 * y ~ N(0, alpha^2 I) (Sec. 3.3): y_out = mu + sd * eps and
 *   terms_out[0] = -ln p(y | alpha) = sum y^2 / (2 alpha^2) + m ln alpha + (m/2) ln 2 pi,
 *   terms_out[1] = ln q(y) = sum (-eps^2 / 2 - ln sd) - (m/2) ln 2 pi.
 * All arrays device float[m]; terms_out device double[2].
 */
lr_status gp_diag_normal_draw(const float* mu, const float* sd, const float* eps, int64_t m, float alpha,
                              float* y_out, double* terms_out, void* workspace, size_t workspace_bytes,
                              lr_stream stream);

/*
 * Gradients of  Loss = L(y) + w_prior (-ln p(y | alpha)) + w_q ln q(y)  with
 * dL/dy = d_y, through y = mu + sd eps at fixed eps:
 *   d_mu = d_y + w_prior y / alpha^2,   d_sd = d_mu * eps - w_q / sd,
 *   d_alpha (device double[1]) = w_prior (m / alpha - sum y^2 / alpha^3).
 */
lr_status gp_diag_normal_vjp(const float* mu, const float* sd, const float* eps, int64_t m, float alpha,
                             const float* d_y, double w_prior, double w_q, float* d_mu, float* d_sd,
                             double* d_alpha, void* workspace, size_t workspace_bytes, lr_stream stream);

/*
 * Partial multivariate-normal proposal over D lens parameters and M
 * source-plane parameters (Sec. 4.2): x = mu + L_full eps with
 *   L_full = [[L, 0], [C, diag(sd)]],
 * L device float[D][D] row-major (lower triangle read, positive diagonal),
 * C device float[M][D], sd device float[M], mu, eps, x_out device float[D+M];
 *   logq_out (device double[1]) = ln N(x | mu, L_full L_full^T)
 *            = -|eps|^2 / 2 - sum ln L_ii - sum ln sd - ((D+M)/2) ln 2 pi.
 * 1 <= D <= 32.
 */
lr_status gp_partial_mvn_draw(const float* mu, const float* L, const float* C, const float* sd, const float* eps,
                              int32_t D, int64_t M, float* x_out, double* logq_out, void* workspace,
                              size_t workspace_bytes, lr_stream stream);

/*
 * Gradients of Loss = L(x) + w_q ln q(x) with dL/dx = d_x (device float[D+M])
 * at fixed eps: d_mu = d_x; d_L[i][j] = d_x[i] eps[j] for j <= i (0 above the
 * diagonal) minus w_q / L_ii on it; d_C[j][l] = d_x[D+j] eps[l];
 * d_sd[j] = d_x[D+j] eps[D+j] - w_q / sd[j]. No workspace.
 */
lr_status gp_partial_mvn_vjp(const float* L, const float* sd, const float* eps, int32_t D, int64_t M,
                             const float* d_x, double w_q, float* d_mu, float* d_L, float* d_C, float* d_sd,
                             lr_stream stream);

/*
 * Diagnostic: the number of (query, source) pairs the grid-source kernels
 * actually evaluate for query points x (device float[n][2]; ray-traced points
 * of query_grid, or explicit points when query_grid is NULL) against
 * source_grid with this length scale, for row blocks of rows_per_cta rows
 * (1024: gp_kernel_matvec and the d_v sweep; 512: gp_kernel_matvec_train).
 * Pairs left out are exactly those whose FP32 exp2 flushes to 0, so every
 * result equals the full n x m evaluation. Synchronises the stream; allocates
 * a small temporary buffer.
 */
lr_status lr_grid_pairs_evaluated(const float* x, int64_t n, const lr_grid* query_grid, const lr_grid* source_grid,
                                  float lengthscale, int32_t rows_per_cta, int64_t* pairs, lr_stream stream);

/*
 * Diagnostic: the pairs the culled sweeps over explicit, ray-traced or self
 * sources evaluate for these point sets and this length scale; sweep 0 is the
 * forward (gp_kernel_matvec), 1 the backward (gp_kernel_matvec_bwd, whose row
 * blocks are smaller). *pairs counts valid (query, source) pairs; *slots
 * (may be NULL) the pair slots the kernels compute, padding rows of a row
 * block and empty slots of a source chunk included. Pairs left out are those
 * whose FP32 exp2 flushes to exactly 0. Synchronises the stream; allocates
 * and frees its own temporary device memory.
 */
lr_status lr_cull_pairs_evaluated(const lr_points* query, const lr_points* source, float lengthscale, int32_t sweep,
                                  int64_t* pairs, int64_t* slots, lr_stream stream);

/* Scratch bytes gp_kernel_matvec needs for these point sets on the current device. */
lr_status lr_matvec_workspace_size(const lr_points* query, const lr_points* source, int32_t nrhs, size_t* bytes);

/* ------------------------------------------------------------------------ */
/* Backward (gradients through the reduction and the ray-trace)               */

/*
 * Gradient outputs of gp_kernel_matvec_bwd. Every pointer is device memory
 * owned by the caller, or NULL when that gradient is not wanted; requested
 * outputs are overwritten (not accumulated).
 *   d_v            float[m]     dL/dv
 *   d_x            float[n][2]  dL/d(query points after ray-tracing); for a
 *                               self-kernel both roles of each point
 *   d_y            float[m][2]  dL/d(source points): explicit, non-self only
 *   d_lengthscale  double[1]    dL/dl
 *   d_variance     double[1]    dL/dvariance
 *   d_lens         double[7]    dL/d(x0, y0, q, phi, theta_e, g1, g2) of the
 *                               query's lens (slope held fixed)
 *   d_sub          double[S][4] dL/d(x_h, y_h, kappa_s | theta_pm, theta_s)
 * and two optional INPUTS:
 *   beta_in        float[n][2]  the query's ray-traced points as the forward
 *                               pass produced them (gp_kernel_matvec's
 *                               beta_out); when given they are used instead of
 *                               being recomputed
 *   moments_in     float[4][n]  the row moments gp_kernel_matvec_train wrote
 *                               for the same query, source, v and length
 *                               scale (non-self sources only); when given the
 *                               row sums are not recomputed and only the
 *                               column sums for d_v (and d_y) sweep the pairs
 * and a mode for a self-kernel split by rows (one rank's share of the pairs
 * when the rows are partitioned across GPUs):
 *   source_rows    nonzero: the query points are the points
 *                  [row0, row0 + n) of the explicit source set, i.e. rows
 *                  of the self-kernel of the sources. g_out and v then cover
 *                  the whole source set ([m][nrhs]); d_x receives both roles
 *                  of the query points (as for a self-kernel), d_v the
 *                  query rows only ([n][nrhs]: d_v_i = var sum_j k_ij g_j),
 *                  and d_lengthscale, d_variance the query rows' share.
 *                  Summing the shares of a partition of the rows (and
 *                  gathering the rows' d_v, d_x) gives the whole
 *                  self-kernel's gradients; the query's lens gradients are
 *                  the query rows' share too. Not with moments_in or d_y.
 *   row0           first row of the query in the source set
 */
typedef struct {
  float* d_v;
  float* d_x;
  float* d_y;
  double* d_lengthscale;
  double* d_variance;
  double* d_lens;
  double* d_sub;
  const float* beta_in;
  const float* moments_in;
  int32_t source_rows;
  int32_t reserved;
  int64_t row0;
} lr_grads;

/*
 * Forward pass of a training step: out exactly as gp_kernel_matvec computes
 * it, plus the per-row sums the backward pass needs that do not depend on
 * dL/dout, written to moments_out (device float[4][n], owned by the caller):
 *   A_i = sum_j k_ij v_j,  B_i = sum_j k_ij v_j (x_i - y_j)  (two rows, in the
 *   library's internal coordinate scaling),  C_i = sum_j k_ij v_j d_ij^2
 *   (internal scaling).
 * Pass them unchanged as grads->moments_in to gp_kernel_matvec_bwd with the
 * same arguments. The pair sweep costs a few more FP32 operations per pair
 * than gp_kernel_matvec and saves the backward's row sweep. Sources: grid or
 * explicit, not a self-kernel (source != NULL) and not ray-traced. nrhs must
 * be 1 (LR_ERR_INVALID_ARG otherwise): this is the one-draw training path;
 * several draws share each pair's exp2 through gp_kernel_matvec and
 * gp_kernel_matvec_bwd with nrhs up to 4. Workspace of
 * lr_matvec_train_workspace_size() bytes, 256-byte aligned.
 */
lr_status gp_kernel_matvec_train(const lr_points* query, const lr_points* source, const float* v, int32_t nrhs,
                                 float lengthscale, float variance, float* out, float* beta_out, float* moments_out,
                                 void* workspace, size_t workspace_bytes, lr_stream stream);
lr_status lr_matvec_train_workspace_size(const lr_points* query, const lr_points* source, int32_t nrhs,
                                         size_t* bytes);

/*
 * Vector-Jacobian product of gp_kernel_matvec for Loss = sum_i g_out_i out_i
 * (g_out: device float[n]), recompute-only: the kernel values are evaluated
 * again, nothing of size n x m is stored, and the ray-traced points are
 * recomputed from the lens. Per pair (k_ij = exp(-d_ij^2/(2 l^2))):
 *   d_v_j = var sum_i k_ij g_i,  d_x_i = var/l^2 g_i sum_j k_ij v_j (y_j - x_i)
 *   (+ the column role for a self-kernel), d_l = var/l^3 sum g_i v_j k_ij d_ij^2,
 *   d_var = sum g_i v_j k_ij; then through beta = xi - alpha(xi) to the lens
 *   and subhalo parameters. Pair sums are FP32 with Kahan-merged tiles;
 *   parameter and hyperparameter sums are FP64. Deterministic.
 * Same arguments and conventions as gp_kernel_matvec; workspace of at least
 * lr_matvec_bwd_workspace_size() bytes, 256-byte aligned. With nrhs > 1
 * (1..4, not with moments_in) v, g_out and d_v are [.][nrhs]; d_x, d_y,
 * d_lengthscale, d_variance and the lens gradients sum over the right-hand
 * sides. A self-kernel shares each pair's exp2 across the columns; the d_v
 * sweep of other sources does too (grid sources are then written out as
 * points), while their d_x row moments take one sweep per column.
 * Errors: LR_ERR_INVALID_ARG also when d_y is requested for grid or
 * self-kernel sources, lens gradients without a ray-traced query, or a
 * ray-traced source set distinct from the query.
 */
lr_status gp_kernel_matvec_bwd(const lr_points* query, const lr_points* source, const float* v, int32_t nrhs,
                               float lengthscale, float variance, const float* g_out, const lr_grads* grads,
                               void* workspace, size_t workspace_bytes, lr_stream stream);

/* Scratch bytes gp_kernel_matvec_bwd needs for these point sets and requested gradients. */
lr_status lr_matvec_bwd_workspace_size(const lr_points* query, const lr_points* source, int32_t nrhs,
                                       const lr_grads* grads, size_t* bytes);

/*
 * Ray-trace backward alone (the vector-Jacobian product of the raytracing
 * equation beta = xi - alpha(xi), Sec. 2.1, with the deflectors of Sec. 2.2):
 * given d_beta = dL/dbeta (device float[n][2]) for the points of `pts` (which
 * must carry a lens), writes d_lens (double[7], dL/d(x0, y0, q, phi, theta_e,
 * g1, g2)) and d_sub (double[S][4], dL/d(x_h, y_h, kappa_s, theta_s), or
 * (x_h, y_h, theta_pm, -) for point masses); either may be NULL. Workspace of
 * lr_raytrace_vjp_workspace_size() bytes, 256-byte aligned, caller-owned.
 * The points are cut into tiles; a tNFW subhalo far from a tile is summed by
 * its far-field series, or by that series' local expansion about the tile's
 * centre, within 5e-9 of the sums of absolute terms, and per-tile partials
 * are added in a fixed order (deterministic). Asynchronous on `stream`;
 * LR_ERR_INVALID_ARG for a missing lens, misaligned or short buffers.
 */
lr_status lens_raytrace_vjp(const lr_points* pts, const float* d_beta, double* d_lens, double* d_sub,
                            void* workspace, size_t workspace_bytes, lr_stream stream);
lr_status lr_raytrace_vjp_workspace_size(const lr_points* pts, size_t* bytes);

/* ------------------------------------------------------------------------ */
/* Elementwise steps of a training step composed from the library (weight     */
/* folding A y, Sec. 3.4; the sum of the layers, Sec. 3.1; dL/dbeta summed    */
/* over the layers and the prior gradient, Sec. 3.6). Device arrays,          */
/* stream-ordered, FP32 unless stated; out may alias an input.                */

/* out = a x + b y (y may be NULL: out = a x), n elements. */
lr_status lr_vec_axpby(int64_t n, float a, const float* x, float b, const float* y, float* out, lr_stream stream);
/* out = a * b elementwise, n elements. */
lr_status lr_vec_mul(int64_t n, const float* a, const float* b, float* out, lr_stream stream);
/* out[0:nh] = (float)head (FP64), out[nh:nh+nt] = tail. */
lr_status lr_vec_pack(const double* head, int32_t nh, const float* tail, int64_t nt, float* out, lr_stream stream);
/* *out = sum of the n (<= 16) device doubles *parts[k] (parts: a HOST array
 * of device pointers), in that order. */
lr_status lr_sum_scalars(const double* const* parts, int32_t n, double* out, lr_stream stream);

/* ------------------------------------------------------------------------ */
/* Serving: device-resident request loop with continuous batching             */

/*
 * A session owns a worker thread, a CUDA stream and a device memory pool on
 * one GPU. Requests (lens systems) are submitted from host memory and
 * admitted, first come first served, while fewer than max_slots requests are
 * active and their device state fits in hbm_budget_bytes (state is held from
 * admission until the result is polled). Each admitted request runs `iters`
 * iterations of: ray-trace its image grid, out = K(beta, y) v over its
 * inducing grid, residual g = out - data, the full backward pass of
 * L = 0.5 |out - data|^2 (dL/dv, dL/dbeta, lens, subhalo, length-scale and
 * variance gradients), and v <- v - step dL/dv. Between iterations the
 * worker admits new requests; one iteration of ALL active requests is one
 * batched kernel launch per stage, so requests of different sizes share
 * launches and overlap on the device. A request is summed in an order fixed
 * by its own sizes: its results are bit-identical alone or in any mix.
 */
typedef struct lr_session lr_session;

typedef struct {
  size_t hbm_budget_bytes; /* device memory admitted requests may hold; 0 = 120 GiB */
  int32_t max_slots;       /* requests iterating at once (1 = one at a time) */
  int32_t device;          /* CUDA device ordinal */
  int64_t fill_pairs;      /* 0, or admit a request only while the active requests' pairs per
                              iteration (n x m each) stay within fill_pairs, or none is active:
                              requests that fill the GPU alone run alone, small ones share it */
} lr_session_cfg;

typedef struct {
  lr_grid grid;         /* image-plane grid, ray-traced through `lens` */
  lr_lens lens;
  const float* sub;     /* HOST float[n_sub][5] subhalo records (copied at submit) */
  int32_t n_sub;
  int32_t profile;      /* LR_PROFILE_TNFW or LR_PROFILE_POINT_MASS */
  lr_grid ygrid;        /* source-plane inducing grid */
  const float* v0;      /* HOST float[m]: initial source weights (copied) */
  const float* data;    /* HOST float[n]: observed fluxes (copied) */
  float lengthscale, variance;
  float step;           /* gradient step on v */
  int32_t iters;        /* >= 1 */
} lr_request;

typedef struct {
  float* out;           /* HOST float[n] or NULL: K v of the last iteration */
  float* v;             /* HOST float[m] or NULL: v after the last update */
  double* d_lens;       /* HOST double[7] or NULL: lens gradient of the last iteration */
  double* d_sub;        /* HOST double[n_sub][4] or NULL */
  double d_lengthscale; /* filled in */
  double d_variance;
  double loss;          /* 0.5 |out - data|^2 of the last iteration */
  double t_submit_s, t_admit_s, t_done_s; /* session clock (s): submit, admission, GPU completion */
} lr_result;

typedef struct {
  int64_t pending, active, held; /* held: finished, result not yet polled */
  size_t used_bytes;
  uint64_t iterations;           /* batched iterations run */
  uint64_t launches;             /* batched kernel launches issued */
  int64_t active_pairs;          /* pairs per iteration (n x m) of the active requests */
  int64_t peak_active_pairs;     /* the largest active_pairs since the session began */
} lr_session_stats;

lr_status solve_session_create(const lr_session_cfg* cfg, lr_session** out);
/* Copies the request in and queues it; *ticket identifies it. LR_ERR_OUT_OF_MEMORY
 * if its device state alone exceeds the budget; LR_ERR_INVALID_ARG on bad input. */
lr_status solve_session_submit(lr_session* s, const lr_request* req, uint64_t* ticket);
/* Waits up to timeout_us for the ticket (0: do not wait). LR_OK: result
 * copied into *out and the request's device state released; LR_PENDING (no
 * wait) or LR_ERR_TIMEOUT: not finished; LR_ERR_NOT_FOUND: unknown ticket;
 * any other status: the request failed (message in lr_last_error). One
 * poller per ticket. */
lr_status solve_session_poll(lr_session* s, uint64_t ticket, lr_result* out, int64_t timeout_us);
/* Removes a request that has not been admitted yet (LR_ERR_BUSY otherwise). */
lr_status solve_session_cancel(lr_session* s, uint64_t ticket);
/* Host-side fault injection: the next batched iteration is abandoned as if a
 * launch had failed; its requests fail with LR_ERR_CUDA, the session goes on. */
lr_status solve_session_inject_fault(lr_session* s);
lr_status solve_session_stats(lr_session* s, lr_session_stats* out);
/* Stops the worker after its current iteration and frees everything. */
lr_status solve_session_destroy(lr_session* s);

/*
 * gp_kernel_matvec for callers that cannot allocate device memory (an
 * application whose device memory is all held by its own pool or budget, a
 * latency-critical loop that must not hit cudaMalloc's implicit device
 * synchronisation, a plugin without access to its host's allocator). The
 * paper has no counterpart: this is a deployment variant of the same
 * reduction, with the same arguments minus the workspace.
 *  - Scratch is a static device array of lr_static_scratch_bytes() bytes
 *    (48 MiB) that every GPU loading this library holds until the process
 *    exits. Problems whose workspace requirement (lr_matvec_workspace_size)
 *    exceeds it are rejected with LR_ERR_INVALID_ARG; nothing else is
 *    allocated (no cudaMalloc, cudaFree or allocating library call).
 *  - Every call resolves the array's device address in the current
 *    device's context (cudaGetSymbolAddress, with that device current); the
 *    first call on a device may load the library's device code, so make it
 *    before any stream capture. Nothing is cached across calls, so a context
 *    destroyed and created again (cudaDeviceReset) is served from its own
 *    copy of the array.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents. Calls whose kernels overlap on the GPU (different streams, or
 *    host threads racing) corrupt each other's scratch: serialise them, for
 *    example on one stream.
 */
lr_status gp_kernel_matvec_static_scratch(const lr_points* query, const lr_points* source, const float* v,
                                          int32_t nrhs, float lengthscale, float variance, float* out,
                                          float* beta_out, lr_stream stream);

/* Size in bytes of the static scratch used by gp_kernel_matvec_static_scratch. */
size_t lr_static_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* LENSGP_H */
