// Elementwise vector steps of the method's training step (the weight folding
// A y of the transmission, Sec. 3.4; the sum of the layers' fluxes, Sec. 3.1;
// the accumulation of dL/dbeta over the layers and the prior gradient of the
// ELBO, Sec. 3.6), so that a driver composing a step from the library does
// none of the arithmetic itself. All stream-ordered; FP32 unless stated.
#include "host.cuh"

namespace lr {
namespace {

__global__ void axpby_kernel(int64_t n, float a, const float* __restrict__ x, float b, const float* __restrict__ y,
                             float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = y ? fmaf(a, x[i], b * y[i]) : a * x[i];
}

__global__ void mul_kernel(int64_t n, const float* __restrict__ a, const float* __restrict__ b,
                           float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

__global__ void pack_kernel(const double* __restrict__ head, int32_t nh, const float* __restrict__ tail, int64_t nt,
                            float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nh + nt; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < nh ? (float)head[i] : tail[i - nh];
}

constexpr int kMaxScalars = 16;
struct ScalarList {
  const double* p[kMaxScalars];
  int32_t n;
};

__global__ void sum_scalars_kernel(const __grid_constant__ ScalarList L, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < L.n; ++k) s += *L.p[k];  // fixed order
  *out = s;
}

unsigned vec_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace
}  // namespace lr

using namespace lr;

extern "C" lr_status lr_vec_axpby(int64_t n, float a, const float* x, float b, const float* y, float* out,
                                  lr_stream stream) {
  LR_REQUIRE(n >= 0, "lr_vec_axpby: n < 0");
  if (n == 0) return LR_OK;
  LR_REQUIRE(x != nullptr && out != nullptr, "lr_vec_axpby: x or out is NULL");
  axpby_kernel<<<vec_blocks(n), 256, 0, as_cuda(stream)>>>(n, a, x, b, y, out);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status lr_vec_mul(int64_t n, const float* a, const float* b, float* out, lr_stream stream) {
  LR_REQUIRE(n >= 0, "lr_vec_mul: n < 0");
  if (n == 0) return LR_OK;
  LR_REQUIRE(a != nullptr && b != nullptr && out != nullptr, "lr_vec_mul: NULL argument");
  mul_kernel<<<vec_blocks(n), 256, 0, as_cuda(stream)>>>(n, a, b, out);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status lr_vec_pack(const double* head, int32_t nh, const float* tail, int64_t nt, float* out,
                                 lr_stream stream) {
  LR_REQUIRE(nh >= 0 && nt >= 0, "lr_vec_pack: negative length");
  if (nh + nt == 0) return LR_OK;
  LR_REQUIRE((head != nullptr || nh == 0) && (tail != nullptr || nt == 0) && out != nullptr,
             "lr_vec_pack: NULL argument");
  pack_kernel<<<vec_blocks(nh + nt), 256, 0, as_cuda(stream)>>>(head, nh, tail, nt, out);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

extern "C" lr_status lr_sum_scalars(const double* const* parts, int32_t n, double* out, lr_stream stream) {
  LR_REQUIRE(n >= 0 && n <= kMaxScalars, "lr_sum_scalars: n = %d outside [0, %d]", n, kMaxScalars);
  LR_REQUIRE(out != nullptr && (parts != nullptr || n == 0), "lr_sum_scalars: NULL argument");
  ScalarList L{};
  L.n = n;
  for (int k = 0; k < n; ++k) {
    LR_REQUIRE(parts[k] != nullptr && ((uintptr_t)parts[k] & 7u) == 0, "lr_sum_scalars: part %d is NULL or misaligned",
               k);
    L.p[k] = parts[k];
  }
  sum_scalars_kernel<<<1, 32, 0, as_cuda(stream)>>>(L, out);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
