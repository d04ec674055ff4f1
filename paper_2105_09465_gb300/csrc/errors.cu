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
