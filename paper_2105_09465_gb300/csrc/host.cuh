// Host-side helpers shared by the translation units of liblensgp.
#pragma once
#include "common.cuh"
#include "grid.cuh"
#include "lens.cuh"

namespace lr {

lr_status make_lens_const(const lr_lens* lens, LensConst* out);
lr_status validate_points(const lr_points* p, const char* what, bool need_lens);
int64_t grid_count(const lr_grid& g);
lr_status launch_grid_points(const lr_grid& g, float2* out, cudaStream_t s);
lr_status launch_raytrace(const lr_points* p, float2* beta, float2* alpha, cudaStream_t s);
lr_status make_lens_grad_const(const lr_lens* lens, LensGradConst* out);
size_t raytrace_vjp_ws(int64_t n, int32_t n_sub);
lr_status launch_raytrace_vjp(const lr_points* p, const float2* dbeta, double* d_lens, double* d_sub, void* ws,
                              cudaStream_t s);

// A point set is ray-traced when it carries a lens, host struct or device record.
inline bool has_lens(const lr_points* p) { return p->lens != nullptr || p->lens_record != nullptr; }

// Rounds a byte count up to a multiple of 256 (workspace sub-allocation).
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Image-grid layout of a query point set, or NULL: the grid itself for a
// grid query, and for explicit points the grid they carry when its point
// count matches (points laid out row-major on that grid, e.g. ray-traced
// pixels). Only the order of rows in row blocks depends on it.
inline const lr_grid* query_layout(const lr_points* q) {
  const lr_grid& g = q->grid;
  if (q->xy == nullptr) return &g;
  if (g.nx > 0 && g.ny > 0 && g.ss > 0 && (int64_t)g.nx * g.ss * g.ny * g.ss == q->n) return &g;
  return nullptr;
}

}  // namespace lr
