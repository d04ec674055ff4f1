// Staging of subhalo records into shared memory: a bulk asynchronous copy
// (TMA engine, 1-D) of the raw float[5] records completed through an
// mbarrier with a bounded wait, then conversion to the prepared form.
#pragma once
#include "lens.cuh"
#include "tma.cuh"

namespace lr {

// Copies the raw records [h0, h0 + cnt) into shared memory. Returns false
// (all threads) if the bulk-copy wait timed out.
__device__ __forceinline__ bool stage_raw(const float* __restrict__ sub, int h0, int cnt, float* raw, uint64_t* bar,
                                          uint32_t& phase, bool bulk_ok, int* fault) {
  const float* src = sub + 5 * (int64_t)h0;
  const uint32_t bytes = 20u * (uint32_t)cnt;
  const uint32_t bulk_bytes = bulk_ok ? (bytes & ~15u) : 0u;
  if (threadIdx.x == 0 && bulk_bytes > 0) {
    // order this CTA's earlier generic-proxy accesses of `raw` before the async write
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bulk_bytes);
    bulk_g2s(raw, src, bulk_bytes, bar);
  }
  // the ragged tail (< 16 B) or everything when unaligned: plain loads
  for (uint32_t w = bulk_bytes / 4 + threadIdx.x; w < bytes / 4; w += blockDim.x) raw[w] = __ldg(src + w);
  bool ok = true;
  if (bulk_bytes > 0) ok = mbar_wait_bounded(bar, phase, fault);
  phase ^= (bulk_bytes > 0) ? 1u : 0u;
  __syncthreads();
  return !__syncthreads_or(!ok);
}

// Stages subhalo records [h0, h0 + cnt) into shared memory as SubRec.
// Returns false (all threads) if the bulk-copy wait timed out.
__device__ __forceinline__ bool stage_subs(const float* __restrict__ sub, int h0, int cnt, int profile, float* raw, SubRec* recs,
                           uint64_t* bar, uint32_t& phase, bool bulk_ok, int* fault) {
  if (!stage_raw(sub, h0, cnt, raw, bar, phase, bulk_ok, fault)) return false;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) recs[t] = prep_sub(raw + 5 * t, profile);
  __syncthreads();
  return true;
}

}  // namespace lr
