// Row blocks of the grid-source reductions, and the pairs they can skip.
//
// Query rows that come from an image grid (ray-traced or not) are handed to
// the CTAs in 2-D image tiles (tw x th pixels per row block) instead of
// raster order: the lens map is continuous, so a tile's ray-traced points
// stay compact and a row block's bounding box is small.
//
// Skipping is exact. In the grid paths the weight of a pair is 2^-t with
// t = sc^2 d^2 (unsplit form), or 2^(bracket) v~ with
// bracket = x'^2 - t <= 30.25 (split form). When every pair between a row
// block and a source sub-segment has t > kSkipT = 170 (measured from the
// row block's bounding box to the sub-segment's abscissa range and row), both
// exponent arguments are below -126, where the flush-to-zero exp2 returns
// exactly 0. So leaving those pairs out changes no result bit.
// The 14-unit margin over 156 absorbs the FP32 rounding of either distance.
#pragma once
#include "grid.cuh"

namespace lr {

constexpr float kSkipT = 170.f;
constexpr int kRowTileW = 32;  // image-tile width of a row block (pixels)

struct RowMap {
  int32_t W, H;    // image grid of the query rows; W == 0: rows in index order
  int32_t tw, th;  // image tile of one row block (tw * th = rows per CTA)
  int32_t TW, TH;  // tiles per image row / column
};

// Per row block: bounding box of its rows and the range of source tiles that
// can hold a contributing pair ([t_lo, t_hi), empty when t_lo >= t_hi).
struct RowBlockInfo {
  float xlo, ylo, xhi, yhi;
  int32_t t_lo, t_hi, pad0, pad1;
};

inline RowMap make_row_map(const lr_grid* qgrid, int rows_per_cta) {
  RowMap m{};
  if (qgrid) {
    m.W = qgrid->nx * qgrid->ss;
    m.H = qgrid->ny * qgrid->ss;
    m.tw = kRowTileW;
    m.th = rows_per_cta / kRowTileW;
    m.TW = (m.W + m.tw - 1) / m.tw;
    m.TH = (m.H + m.th - 1) / m.th;
  }
  return m;
}

inline int64_t row_block_count(const RowMap& m, int64_t n, int rows_per_cta) {
  return m.W ? (int64_t)m.TW * m.TH : (n + rows_per_cta - 1) / rows_per_cta;
}

// Index of row w (0 <= w < rows per CTA) of row block rb, or -1 (padding).
__device__ __forceinline__ int64_t map_row(const RowMap& m, int64_t n, int rows_per_cta, int64_t rb, int w) {
  if (m.W == 0) {
    const int64_t i = rb * rows_per_cta + w;
    return i < n ? i : -1;
  }
  const int64_t ty = rb / m.TW, tx = rb - ty * m.TW;
  const int wy = w / m.tw, wx = w - wy * m.tw;
  const int64_t r = ty * m.th + wy, c = tx * m.tw + wx;
  return (r < m.H && c < m.W) ? r * m.W + c : -1;
}

// True when every pair between the box and the source segment
// [xa, xb] x {y} has sc^2 d^2 > kSkipT.
__device__ __forceinline__ bool seg_far(const RowBlockInfo& B, float xa, float xb, float y, float sc) {
  const float dx = fmaxf(fmaxf(B.xlo - xb, xa - B.xhi), 0.f);
  const float dy = fmaxf(fmaxf(B.ylo - y, y - B.yhi), 0.f);
  const float sx = sc * dx, sy = sc * dy;
  return fmaf(sx, sx, sy * sy) > kSkipT;
}

// Tile-local columns [lo, hi] of a source grid row at ordinate y that can
// hold a pair with sc^2 d^2 <= kSkipT for some point of the box: every column
// outside is far from the whole box (so are all columns when the row itself is
// out of reach: then lo > hi). The tile covers columns c0 .. c0 + cnt - 1.
// The bound is computed in FP32; one column of margin on each side absorbs its
// rounding, and the threshold's own 14-unit margin covers the kernels'
// rounding of the distances.
__device__ __forceinline__ void reach_cols(const RowBlockInfo& B, const GridDev& g, float y, float sc, int c0, int cnt,
                                           int& lo, int& hi) {
  lo = 0x3fffffff;
  hi = -1;
  if (!(B.xlo <= B.xhi)) return;  // a row block without rows
  const float dy = fmaxf(fmaxf(B.ylo - y, y - B.yhi), 0.f);
  const float sy = sc * dy;
  const float rem = kSkipT - sy * sy;
  if (!(rem > 0.f)) return;
  const float w = sqrtf(rem) / sc;  // reach along the row
  const float cl = (B.xlo - w - g.cx) / g.h + g.c0x;
  const float ch = (B.xhi + w - g.cx) / g.h + g.c0x;
  // clamp in float first: the bounds can be far outside the int range
  const float fl = fmaxf(floorf(cl) - 1.0f - (float)c0, 0.0f);
  const float fh = fminf(ceilf(ch) + 1.0f - (float)c0, (float)(cnt - 1));
  if (!(fl <= fh)) return;
  lo = (int)fl;
  hi = (int)fh;
}

// reach_cols with the divisions replaced by the reciprocals inv_sc = 1/sc and
// inv_h = 1/h (their extra rounding is far inside the one-column margin).
__device__ __forceinline__ void reach_cols_fast(const RowBlockInfo& B, const GridDev& g, float y, float sc,
                                                float inv_sc, float inv_h, int c0, int cnt, int& lo, int& hi) {
  lo = 0x3fffffff;
  hi = -1;
  if (!(B.xlo <= B.xhi)) return;  // a row block without rows
  const float dy = fmaxf(fmaxf(B.ylo - y, y - B.yhi), 0.f);
  const float sy = sc * dy;
  const float rem = kSkipT - sy * sy;
  if (!(rem > 0.f)) return;
  const float w = sqrtf(rem) * inv_sc;  // reach along the row
  const float cl = fmaf(B.xlo - w - g.cx, inv_h, g.c0x);
  const float ch = fmaf(B.xhi + w - g.cx, inv_h, g.c0x);
  const float fl = fmaxf(floorf(cl) - 1.0f - (float)c0, 0.0f);
  const float fh = fminf(ceilf(ch) + 1.0f - (float)c0, (float)(cnt - 1));
  if (!(fl <= fh)) return;
  lo = (int)fl;
  hi = (int)fh;
}

// The source pairs [pp_lo, pp_hi) of the sub-segment that starts at tile-local
// column s0 (pair p = columns s0 + 2p, s0 + 2p + 1; SEG / 2 pairs) that meet
// the reachable columns [lo, hi], widened to whole quarters of the
// sub-segment (2 pairs, 4 columns): the kernels evaluate a quarter or skip
// it as a block. Empty when pp_lo >= pp_hi.
constexpr int kQuarterPairs = 2;

template <int SEG>
__device__ __forceinline__ void seg_pair_range(int lo, int hi, int s0, int& pp_lo, int& pp_hi) {
  const int a = lo - s0, b = hi - s0;
  pp_lo = a <= 0 ? 0 : (a >> 1) & ~(kQuarterPairs - 1);
  pp_hi = b < 0 ? 0 : min(SEG / 2, ((b >> 1) + kQuarterPairs) & ~(kQuarterPairs - 1));
}

// One CTA (kRowPrepThreads) per row block: bounding box of its rows and the
// active source-tile range (grid rows whose whole abscissa range is not far).
constexpr int kRowPrepThreads = 128;

__device__ __forceinline__ void row_block_info_body(const float2* __restrict__ x, int64_t n, const RowMap& map,
                                                    int rows_per_cta, const GridDev& g, int32_t segs, float sc,
                                                    int64_t rb, RowBlockInfo* __restrict__ info) {
  __shared__ float red[4][kRowPrepThreads / 32];
  __shared__ int ired[2][kRowPrepThreads / 32];
  __shared__ RowBlockInfo B;
  float xlo = INFINITY, ylo = INFINITY, xhi = -INFINITY, yhi = -INFINITY;
  for (int w = threadIdx.x; w < rows_per_cta; w += kRowPrepThreads) {
    const int64_t i = map_row(map, n, rows_per_cta, rb, w);
    if (i < 0) continue;
    const float2 p = x[i];
    xlo = fminf(xlo, p.x);
    xhi = fmaxf(xhi, p.x);
    ylo = fminf(ylo, p.y);
    yhi = fmaxf(yhi, p.y);
  }
  for (int o = 16; o; o >>= 1) {
    xlo = fminf(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
    ylo = fminf(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
    xhi = fmaxf(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
    yhi = fmaxf(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wp] = xlo;
    red[1][wp] = ylo;
    red[2][wp] = xhi;
    red[3][wp] = yhi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kRowPrepThreads / 32; ++k) {
      red[0][0] = fminf(red[0][0], red[0][k]);
      red[1][0] = fminf(red[1][0], red[1][k]);
      red[2][0] = fmaxf(red[2][0], red[2][k]);
      red[3][0] = fmaxf(red[3][0], red[3][k]);
    }
    B.xlo = red[0][0];
    B.ylo = red[1][0];
    B.xhi = red[2][0];
    B.yhi = red[3][0];
  }
  __syncthreads();
  // grid rows within reach of the box (a row block without rows reaches none)
  int lo = 0x7fffffff, hi = -1;
  const bool any = B.xlo <= B.xhi;
  for (int r = threadIdx.x; r < g.H; r += kRowPrepThreads) {
    if (any && !seg_far(B, grid_x(g, 0), grid_x(g, g.W - 1), grid_y(g, r), sc)) {
      lo = min(lo, r);
      hi = max(hi, r);
    }
  }
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    ired[0][wp] = lo;
    ired[1][wp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kRowPrepThreads / 32; ++k) {
      ired[0][0] = min(ired[0][0], ired[0][k]);
      ired[1][0] = max(ired[1][0], ired[1][k]);
    }
    RowBlockInfo o = B;
    o.t_lo = ired[1][0] >= 0 ? ired[0][0] * segs : 0;
    o.t_hi = ired[1][0] >= 0 ? (ired[1][0] + 1) * segs : 0;
    o.pad0 = o.pad1 = 0;
    info[rb] = o;
  }
}

}  // namespace lr
