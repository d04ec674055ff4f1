// Pipe-rate probe: measures, on the running GPU, how many FP32 FMA lanes
// (scalar FFMA and packed f32x2 FFMA2) and how many MUFU.EX2 results one SM
// retires per SM clock. These measured rates are the denominators of the
// ALU roofline that the kernel-reduction and ray-trace throughput is quoted
// against (one exp2 and a handful of FP32 operations per kernel pair).
#include "common.cuh"

namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kThreads = 1024;  // 32 warps: 8 per SM sub-partition

// OP 0: MUFU.EX2   a <- 2^(-a)        (fixed point in (0,1), never underflows)
// OP 1: FFMA       a <- a*m + b
// OP 2: FFMA2      (a0,a1) <- (a0,a1)*(m,m) + (b,b)
template <int OP>
__global__ void __launch_bounds__(kThreads, 1)
probe_kernel(float* sink, int iters, unsigned long long* cycles, float m, float b) {
  float a[2 * kChains];
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) a[k] = 0.25f + 1e-4f * (threadIdx.x & 31) + 1e-3f * k;
  __syncthreads();
  unsigned long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) {
        a[k] = lr::ex2_approx(-a[k]);
      } else if (OP == 1) {
        a[k] = fmaf(a[k], m, b);
      } else {
        float2 x = make_float2(a[2 * k], a[2 * k + 1]);
        x = __ffma2_rn(x, make_float2(m, m), make_float2(b, b));
        a[2 * k] = x.x;
        a[2 * k + 1] = x.y;
      }
    }
  }
  __syncthreads();
  unsigned long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) s += a[k];
  if (s == 12345.f) sink[threadIdx.x] = s;  // keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
lr_status run_one(int n_sm, int iters, float* sink, unsigned long long* d_cyc,
                  unsigned long long* h_cyc, double* rate) {
  // Dynamic shared memory above half the SM's capacity pins one CTA per SM.
  int smem = 120 * 1024;
  LR_CHECK_CUDA(cudaFuncSetAttribute(probe_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  for (int rep = 0; rep < 2; ++rep) {  // first launch warms up clocks and caches
    probe_kernel<OP><<<n_sm, kThreads, smem>>>(sink, iters, d_cyc, 0.999f, 1e-3f);
    LR_CHECK_CUDA(cudaGetLastError());
    LR_CHECK_CUDA(cudaDeviceSynchronize());
  }
  LR_CHECK_CUDA(cudaMemcpy(h_cyc, d_cyc, sizeof(unsigned long long) * n_sm, cudaMemcpyDeviceToHost));
  // Median over SMs of lanes retired per SM clock.
  double lanes_per_op = (OP == 2) ? 2.0 : 1.0;
  double ops = double(kThreads) * iters * kChains * lanes_per_op;
  double* r = new double[n_sm];
  for (int i = 0; i < n_sm; ++i) r[i] = ops / double(h_cyc[i]);
  for (int i = 1; i < n_sm; ++i)
    for (int j = i; j > 0 && r[j - 1] > r[j]; --j) { double t = r[j]; r[j] = r[j - 1]; r[j - 1] = t; }
  *rate = r[n_sm / 2];
  delete[] r;
  return LR_OK;
}

}  // namespace

extern "C" lr_status lr_probe_pipe_rates(int32_t device, double* ffma_lanes_per_clk,
                                         double* ffma2_lanes_per_clk, double* ex2_per_clk,
                                         int32_t* sm_count) {
  LR_REQUIRE(ffma_lanes_per_clk && ffma2_lanes_per_clk && ex2_per_clk && sm_count,
             "lr_probe_pipe_rates: NULL output pointer");
  LR_CHECK_CUDA(cudaSetDevice(device));
  int n_sm = 0;
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
  float* sink = nullptr;
  unsigned long long* d_cyc = nullptr;
  LR_CHECK_CUDA(cudaMalloc(&sink, kThreads * sizeof(float)));
  LR_CHECK_CUDA(cudaMalloc(&d_cyc, n_sm * sizeof(unsigned long long)));
  unsigned long long* h_cyc = new unsigned long long[n_sm];
  lr_status st = run_one<0>(n_sm, 4096, sink, d_cyc, h_cyc, ex2_per_clk);
  if (st == LR_OK) st = run_one<1>(n_sm, 8192, sink, d_cyc, h_cyc, ffma_lanes_per_clk);
  if (st == LR_OK) st = run_one<2>(n_sm, 8192, sink, d_cyc, h_cyc, ffma2_lanes_per_clk);
  delete[] h_cyc;
  cudaFree(sink);
  cudaFree(d_cyc);
  *sm_count = n_sm;
  return st;
}
