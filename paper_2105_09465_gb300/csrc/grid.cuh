// Regular point grids (image-plane pixel centres, source-plane inducing
// points): point k of an lr_grid is generated from its index, never loaded.
#pragma once
#include "common.cuh"

namespace lr {

struct GridDev {
  int32_t W, H;       // points per row, rows
  float h, c0x, c0y;  // spacing (FP32 division pix / ss) and centre offsets
  float cx, cy;
};

inline GridDev grid_dev(const lr_grid& g) {
  GridDev d;
  d.W = g.nx * g.ss;
  d.H = g.ny * g.ss;
  d.h = g.pix / (float)g.ss;
  d.c0x = 0.5f * (float)(d.W - 1);
  d.c0y = 0.5f * (float)(d.H - 1);
  d.cx = g.cx;
  d.cy = g.cy;
  return d;
}

__device__ __forceinline__ float grid_x(const GridDev& g, int32_t col) { return fmaf((float)col - g.c0x, g.h, g.cx); }
__device__ __forceinline__ float grid_y(const GridDev& g, int32_t row) { return fmaf((float)row - g.c0y, g.h, g.cy); }

__device__ __forceinline__ float2 grid_point(const GridDev& g, int64_t k) {
  const int32_t row = (int32_t)(k / g.W);
  const int32_t col = (int32_t)(k - (int64_t)row * g.W);
  return make_float2(grid_x(g, col), grid_y(g, row));
}

}  // namespace lr
