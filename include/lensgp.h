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

#ifdef __cplusplus
}
#endif
#endif /* LENSGP_H */
