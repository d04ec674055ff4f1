// Batched launches: one kernel launch serves up to kMaxBatch independent
// problems (lens systems of different sizes). The problem descriptors and
// the prefix sums of their CTA counts travel in the kernel parameter itself
// (__grid_constant__, no device-side table to upload); CTA b finds its
// problem by scanning the prefix sums.
#pragma once
#include "common.cuh"

namespace lr {

constexpr int kMaxBatch = 16;

template <typename P>
struct Batch {
  int32_t count;
  int32_t start[kMaxBatch + 1];  // start[k] = first CTA of problem k; start[count] = total CTAs
  P p[kMaxBatch];
};

template <typename P>
__device__ __forceinline__ int batch_find(const Batch<P>& B, int t) {
  int k = 0;
  while (k + 1 < B.count && t >= B.start[k + 1]) ++k;
  return k;
}

}  // namespace lr
