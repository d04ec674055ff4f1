// Error reporting for the C ABI: every entry point returns an lr_status and
// leaves a human-readable message in a thread-local buffer.
#include <stdarg.h>
#include <string.h>
#include "common.cuh"
#include "tma.cuh"

namespace lr {

static thread_local char g_msg[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
}

lr_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LR_ERR_OUT_OF_MEMORY : LR_ERR_CUDA;
}

}  // namespace lr

extern "C" const char* lr_last_error(void) { return lr::g_msg; }

extern "C" const char* lr_status_name(lr_status s) {
  switch (s) {
    case LR_OK: return "LR_OK";
    case LR_ERR_INVALID_ARG: return "LR_ERR_INVALID_ARG";
    case LR_ERR_CUDA: return "LR_ERR_CUDA";
    case LR_ERR_OUT_OF_MEMORY: return "LR_ERR_OUT_OF_MEMORY";
    case LR_ERR_TIMEOUT: return "LR_ERR_TIMEOUT";
    case LR_PENDING: return "LR_PENDING";
    case LR_ERR_NOT_FOUND: return "LR_ERR_NOT_FOUND";
    case LR_ERR_BUSY: return "LR_ERR_BUSY";
    default: return "LR_UNKNOWN_STATUS";
  }
}

// ---------------------------------------------------------------------------
// Device fault word: kernels that give up a bounded wait record a code here
// (instead of trapping), and the host reads it back with lr_fault_status().
__device__ int g_lr_fault;

namespace lr {

int* fault_ptr() {
  static thread_local int cached_dev = -1;
  static thread_local int* cached = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (dev != cached_dev) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lr_fault) != cudaSuccess) return nullptr;
    cached = static_cast<int*>(p);
    cached_dev = dev;
  }
  return cached;
}

}  // namespace lr

extern "C" lr_status lr_fault_status(int32_t* code, int32_t clear) {
  LR_REQUIRE(code != nullptr, "lr_fault_status: code is NULL");
  int* p = lr::fault_ptr();
  if (!p) return lr::cuda_status(cudaGetLastError(), "cudaGetSymbolAddress(g_lr_fault)");
  int v = 0;
  LR_CHECK_CUDA(cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost));
  *code = v;
  if (clear) LR_CHECK_CUDA(cudaMemset(p, 0, sizeof(int)));
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded wait: one thread arms an mbarrier for 16 bytes of
// transactions that never come (no copy is issued), waits with the given
// budget, and returns after recording the time-out. Nothing is in flight when
// it gives up, so the context stays usable.
namespace {

__global__ void bounded_wait_selftest_kernel(long long budget, int* fault, int* returned) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  lr::mbar_init(&bar, 1);
  lr::mbar_expect_tx(&bar, 16);  // arrive, and expect 16 bytes that no copy delivers
  const bool ok = lr::mbar_wait_bounded(&bar, 0, fault, budget);
  *returned = ok ? 2 : 1;
}

}  // namespace

extern "C" lr_status lr_selftest_bounded_wait(int64_t budget_cycles, int32_t* code) {
  LR_REQUIRE(code != nullptr, "lr_selftest_bounded_wait: code is NULL");
  LR_REQUIRE(budget_cycles > 0 && budget_cycles <= 2000000000LL,
             "lr_selftest_bounded_wait: budget of %lld cycles outside (0, 2e9]", (long long)budget_cycles);
  int* fault = lr::fault_ptr();
  LR_REQUIRE(fault != nullptr, "could not resolve the device fault word");
  int* ret = nullptr;
  LR_CHECK_CUDA(cudaMalloc(&ret, sizeof(int)));
  lr_status st = LR_OK;
  int h = 0;
  if (cudaMemset(ret, 0, sizeof(int)) != cudaSuccess) st = lr::cuda_status(cudaGetLastError(), "cudaMemset");
  if (st == LR_OK) {
    bounded_wait_selftest_kernel<<<1, 32>>>((long long)budget_cycles, fault, ret);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = lr::cuda_status(e, "bounded_wait_selftest_kernel");
  }
  if (st == LR_OK && cudaMemcpy(&h, ret, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = lr::cuda_status(cudaGetLastError(), "cudaMemcpy");
  cudaFree(ret);
  // 1: the kernel gave up the wait and returned; the fault word says why
  *code = h;
  return st;
}
