// Error reporting for the C ABI: every entry point returns an lr_status and
// leaves a human-readable message in a thread-local buffer.
#include <stdarg.h>
#include <string.h>
#include "common.cuh"

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
