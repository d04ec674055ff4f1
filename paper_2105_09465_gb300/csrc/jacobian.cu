// Lens Jacobian and magnification (Sec. 2.1, lens-Jacobian and magnification
// equations): A = d beta / d xi = I - d alpha / d xi per image-plane point and
// mu = 1 / det A. Same layout as the ray-trace: one thread per point,
// subhalo records staged in shared memory by bulk copy; the SPLE part uses
// the analytic Wirtinger derivatives of the series, the subhalo parts the
// closed-form Jacobians A [G I + (H - 2G) n n^T] (tNFW) and
// theta^2 (I - 2 n n^T) / R^2 (point mass).
#include <math.h>

#include "host.cuh"
#include "problems.cuh"
#include "subs.cuh"

namespace lr {

constexpr int kJThreads = 256;
constexpr int kJChunk = 256;

template <int PROFILE>
__global__ void __launch_bounds__(kJThreads) lens_jacobian_kernel(const __grid_constant__ LensConst L,
                                                                  const __grid_constant__ LensGradConst LG,
                                                                  GridDev g, const float2* __restrict__ xi,
                                                                  int64_t n, const float* __restrict__ sub, int n_sub,
                                                                  int bulk_ok, float4* __restrict__ jac,
                                                                  float* __restrict__ mu, int* fault) {
  __shared__ __align__(16) float raw[5 * kJChunk];
  __shared__ __align__(16) SubRec recs[kJChunk];
  __shared__ __align__(8) uint64_t bar;
  const int64_t i = (int64_t)blockIdx.x * kJThreads + threadIdx.x;
  const bool valid = i < n;
  const int64_t ii = valid ? i : (n - 1);
  const float2 p = xi ? xi[ii] : grid_point(g, ii);
  float J[4];
  sple_jacobian(L, LG, p.x, p.y, J);
  // external shear: d alpha / d xi = [[g1, g2], [g2, -g1]]
  J[0] += L.g1;
  J[1] += L.g2;
  J[2] += L.g2;
  J[3] -= L.g1;
  if (n_sub > 0) {
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (int h0 = 0; h0 < n_sub; h0 += kJChunk) {
      const int cnt = min(kJChunk, n_sub - h0);
      if (!stage_subs(sub, h0, cnt, PROFILE, raw, recs, &bar, phase, bulk_ok != 0, fault)) return;
      for (int t = 0; t < cnt; ++t) {
        const SubRec h = recs[t];
        const float dx = p.x - h.xh, dy = p.y - h.yh;
        const float R2 = fmaf(dx, dx, dy * dy);
        if (!(R2 > 1e-30f)) continue;
        const float iR2 = frcp(R2);
        if (PROFILE == LR_PROFILE_POINT_MASS) {
          const float m = h.its2 * iR2, q = -2.0f * m * iR2;
          J[0] += fmaf(q, dx * dx, m);
          J[1] += q * dx * dy;
          J[2] += q * dx * dy;
          J[3] += fmaf(q, dy * dy, m);
        } else {
          float Gt, Ht;
          float ix2_unused;
          tnfw_GH(h, R2, Gt, Ht, ix2_unused);
          const float a = h.A * Gt, q = h.A * (Ht - 2.0f * Gt) * iR2;
          J[0] += fmaf(q, dx * dx, a);
          J[1] += q * dx * dy;
          J[2] += q * dx * dy;
          J[3] += fmaf(q, dy * dy, a);
        }
      }
      __syncthreads();
    }
  }
  if (valid) {
    const float a00 = 1.0f - J[0], a01 = -J[1], a10 = -J[2], a11 = 1.0f - J[3];
    if (jac) jac[i] = make_float4(a00, a01, a10, a11);
    if (mu) mu[i] = 1.0f / fmaf(a00, a11, -a01 * a10);
  }
}

}  // namespace lr

extern "C" lr_status lens_jacobian(const lr_points* pts, float* jac_out, float* mu_out, lr_stream stream) {
  lr_status st = lr::validate_points(pts, "lens_jacobian", true);
  if (st != LR_OK) return st;
  LR_REQUIRE(((uintptr_t)jac_out & 15u) == 0 && ((uintptr_t)mu_out & 3u) == 0,
             "lens_jacobian: jac_out must be 16-byte and mu_out 4-byte aligned");
  lr::LensConst L;
  LR_REQUIRE(pts->lens != nullptr, "lens_jacobian: takes a host lens (lr_lens), not a device lens record");
  if ((st = lr::make_lens_const(pts->lens, &L)) != LR_OK) return st;
  lr::LensGradConst G;
  if ((st = lr::make_lens_grad_const(pts->lens, &G)) != LR_OK) return st;
  if (pts->n == 0) return LR_OK;
  int* fault = lr::fault_ptr();
  LR_REQUIRE(fault != nullptr, "could not resolve the device fault word");
  const lr::GridDev g = pts->xy ? lr::GridDev{} : lr::grid_dev(pts->grid);
  const int bulk_ok = (((uintptr_t)pts->sub & 15u) == 0) ? 1 : 0;
  const unsigned blocks = (unsigned)((pts->n + lr::kJThreads - 1) / lr::kJThreads);
  const float2* xi = reinterpret_cast<const float2*>(pts->xy);
  float4* jac = reinterpret_cast<float4*>(jac_out);
  cudaStream_t s = lr::as_cuda(stream);
  if (pts->profile == LR_PROFILE_POINT_MASS)
    lr::lens_jacobian_kernel<LR_PROFILE_POINT_MASS><<<blocks, lr::kJThreads, 0, s>>>(
        L, G, g, xi, pts->n, pts->sub, pts->n_sub, bulk_ok, jac, mu_out, fault);
  else
    lr::lens_jacobian_kernel<LR_PROFILE_TNFW><<<blocks, lr::kJThreads, 0, s>>>(L, G, g, xi, pts->n, pts->sub,
                                                                               pts->n_sub, bulk_ok, jac, mu_out, fault);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
