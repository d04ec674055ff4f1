// Internal helpers shared by the CUDA translation units of liblensgp.
// Not part of the public C ABI (include/lensgp.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include "../../include/lensgp.h"

namespace lr {

// Thread-local last-error message, read back through lr_last_error().
void set_error(const char* fmt, ...);

// Map a CUDA error to LR_ERR_CUDA, recording the failing call.
lr_status cuda_status(cudaError_t e, const char* what);

// Device address of the library's fault word on the current device.
int* fault_ptr();

// Launch timer (lr_kernel_timer_enable): events on stream s before and after
// one launch of kernel id (an LR_KT_* value). No-ops while the timer is off or
// s is capturing a graph.
void ktimer_begin(int id, cudaStream_t s);
void ktimer_end(int id, cudaStream_t s);

// Fork and join: fork_begin makes a per-device side stream wait for the work
// enqueued on s so far (f->side is s itself when no side stream exists);
// fork_end makes s wait for the side stream's work since. Under stream
// capture the two become graph edges. Every fork_begin that returned LR_OK
// must be followed by fork_end, also on error paths.
struct Fork {
  cudaStream_t side;
  cudaEvent_t join;
};
lr_status fork_begin(cudaStream_t s, Fork* f);
lr_status fork_end(cudaStream_t s, Fork* f);

// Streams cross the ABI as lr_stream (an opaque CUstream_st*).
inline cudaStream_t as_cuda(lr_stream s) { return reinterpret_cast<cudaStream_t>(s); }

#define LR_CHECK_CUDA(call)                                        \
  do {                                                             \
    cudaError_t _e = (call);                                       \
    if (_e != cudaSuccess) return ::lr::cuda_status(_e, #call);    \
  } while (0)

#define LR_REQUIRE(cond, ...)                                      \
  do {                                                             \
    if (!(cond)) {                                                 \
      ::lr::set_error(__VA_ARGS__);                                \
      return LR_ERR_INVALID_ARG;                                   \
    }                                                              \
  } while (0)

// Hardware exp2 (MUFU.EX2 with flush-to-zero): 2^x, underflows to +0.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace lr
