// Problem descriptors of the kernels, shared by the single-problem entry
// points and the batched launches of the serving engine, plus the host-side
// launch helpers for batches.
#pragma once
#include "batch.cuh"
#include "grid.cuh"
#include "lens.cuh"
#include "rowmap.cuh"

namespace lr {

// ---- exponent splitting of grid-source tiles (matvec.cu, matvec_bwd.cu)
// A grid tile is cut into sub-segments of kSplitSeg columns with scaled
// abscissae x' = sc (x_j - o) about each sub-segment's centre o. Splitting
// the exponent as [2 q x' - q^2 - dy'^2] - x'^2 is exact in real arithmetic;
// in FP32 it needs |x'| bounded, which holds when the length scale is not
// much below the grid spacing (l >= 1.24 h). Otherwise the kernels use the
// unsplit form.
constexpr int kSplitSeg = 16;
constexpr float kSplitXMax = 5.5f;
inline int32_t grid_split_ok(const GridDev& g, float sc) {
  return sc * g.h * (float)(kSplitSeg / 2) <= kSplitXMax ? 1 : 0;
}

// ---- row-block boxes for grid sources (rowmap.cu)
struct RowInfoP {
  const float2* x;  // query points
  int64_t n;
  RowMap map;
  int32_t rows_per_cta, segs;
  GridDev g;        // source grid
  float sc;
  RowBlockInfo* info;  // [row blocks]
};
lr_status launch_row_info(const RowInfoP& P, cudaStream_t s);
lr_status launch_row_info_batched(const RowInfoP* p, int count, cudaStream_t s);
inline size_t row_info_bytes(const RowMap& m, int64_t n, int rows_per_cta) {
  const size_t b = sizeof(RowBlockInfo) * (size_t)(row_block_count(m, n, rows_per_cta) + 1);
  return (b + 255) & ~size_t(255);
}

// ---- forward reduction (matvec.cu)
constexpr int kMvThreads = 128;
constexpr int kMvR = 8;                         // query rows per thread
constexpr int kRowsPerCta = kMvThreads * kMvR;  // 1024
constexpr int kTile = 256;                      // source points per tile
constexpr int kPairs = kTile / 2;               // = kMvThreads: one pair per loader thread

struct SrcDesc {
  const float2* xy;  // explicit source points, or NULL for a grid
  GridDev g;         // grid description when xy == NULL
  int64_t m;         // number of source points
  int32_t segs;      // grid: tiles per grid row
  int32_t n_tiles;   // total tiles
};

struct MvArgs {
  const float2* x;   // query points [n]
  int64_t n;
  SrcDesc src;
  const float* v;    // [m]
  float neg_c;       // -log2(e) / (2 l^2)
  float sc;          // sqrt(log2(e) / (2 l^2)): scale of the tile-local grid coordinates
  int32_t split;     // grid sources: split exponent (grid_split_ok)
  float variance;
  int32_t chunks;    // column chunks per row block
  RowMap map;        // order of the query rows in row blocks
  const RowBlockInfo* info;  // grid sources: per-row-block box and active tiles, or NULL (no skipping)
  float* out;        // [n] when chunks == 1
  float* partial;    // [chunks][n] when chunks > 1
};

struct MergeP {
  const float* partial;
  int32_t chunks;
  int64_t n;
  float variance;
  float* out;
};


// ---- backward row pass (matvec_bwd.cu)
constexpr int kBwThreads = 128;
constexpr int kBwR = 4;                     // rows per thread
constexpr int kBwRows = kBwThreads * kBwR;  // 512 rows per CTA
constexpr int kBwRdv = 8;                   // rows per thread with the fused d_v reduction
constexpr int kBwRgrid = 4;                 // rows per thread, grid sources without d_v (training forward)
constexpr int kBwTile = 256;
constexpr int kBwPairs = kBwTile / 2;
constexpr int kMergeThreads = 256;

struct BwSrc {
  const float2* xy;  // explicit sources, or NULL for a grid
  GridDev g;
  int64_t m;
  int32_t segs, n_tiles;
};

struct BwArgs {
  const float2* x;  // query points [n]
  int64_t n;
  BwSrc src;
  const float* v;   // [m] source weights
  const float* gs;  // [m] source-side g (self-kernel only: g of the same points)
  float neg_c;      // -log2(e)/(2 l^2)
  float sc;         // sqrt(log2(e)/(2 l^2)): scale of the tile-local grid coordinates
  int32_t split;    // grid sources: split exponent (grid_split_ok)
  int32_t chunks;
  RowMap map;       // order of the query rows in row blocks
  const RowBlockInfo* info;  // grid sources: per-row-block box and active tiles, or NULL (no skipping)
  int32_t K;        // quantities per row: 4, or 7 for a self-kernel
  int32_t rows_per_cta;  // kBwThreads x (kBwR, or kBwRdv with the fused d_v)
  float* partial;   // [chunks][K][n]
  // grid sources only: fused column reduction for dL/dv
  const float* grow;  // [n] g of the query rows, or NULL (no fused d_v)
  float* dv_part;     // [row blocks][m] per-row-block sums of k_ij g_i
};

// Fixed-order merge of the fused d_v partials: d_v_j = var sum_rb dv_part[rb][j].
struct DvMergeP {
  const float* dv_part;
  int32_t row_blocks;
  int64_t m;
  float var;
  float* d_v;
  const RowBlockInfo* info;  // row blocks' active tile ranges, or NULL (every row block wrote every source)
  int32_t W, segs;           // source grid width and tiles per grid row (with info)
};

// training forward: merge of the row-pass partials into out and the moments
struct MomMergeP {
  const float* partial;  // [chunks][4][n]
  int32_t chunks;
  int64_t n;
  float var;
  float* out;            // [n]
  float* mom;            // [4][n]
};

struct MergeArgs {
  const float* partial;
  int32_t chunks, K;
  int64_t n;
  const float* g;      // [n] dL/dout
  const float* vrow;   // [n] v of the query points (self-kernel column role)
  float var, inv_l2, dl_scale;  // d_x scale var/l^2 and d_len scale (sign per accumulation form)
  float b_scale;                // 1, or 1/sc when B was accumulated in scaled grid coordinates
  float2* d_x;         // [n] or NULL
  float* d_v;          // [n] (self-kernel) or NULL
  double* scal_part;   // [blocks][2]: d_len, d_var partials
};

struct ScalP {
  const double* part;
  int32_t nblk;
  double* d_len;
  double* d_var;
};

// ---- ray-trace and its backward (raytrace.cu, raytrace_bwd.cu)
struct RtP {
  LensConst L;
  GridDev g;
  const float2* xi;  // explicit points, or NULL for the grid
  int64_t n;
  const float* sub;
  int32_t n_sub, bulk_ok, profile;
  float2* beta;
  float2* alpha;
};

struct VjpP {
  LensConst L;
  LensGradConst LG;
  GridDev g;
  const float2* xi;
  int64_t n;
  const float* sub;
  int32_t n_sub, profile;
  int32_t phases;  // slots per subhalo (see vjp_phases)
  int32_t bands;   // grid points: bands of image rows of the CTAs' tiles (see vjp_bands)
  const float2* dbeta;
  double* lens_part;
  float* sub_part;   // [4 n_sub][CTA]
  float* slot_part;  // [CTA][n_sub phases][4] when phases > 1
};

struct VjpFinalP {
  const double* lens_part;
  const float* sub_part;
  int32_t nblk, n_sub;
  double* d_lens;
  double* d_sub;
};

// out[i] = a[i] - alpha * b[i]
struct AxpyP {
  const float* a;
  const float* b;
  float* out;
  int64_t n;
  float alpha;
};

// Batched launch helpers: each splits `count` problems into launches of at
// most kMaxBatch problems, all on stream s.
lr_status launch_raytrace_batched(const RtP* p, int count, cudaStream_t s);
lr_status launch_bwd_rows_batched(const BwArgs* p, int count, cudaStream_t s);
lr_status launch_bwd_merge_batched(const MergeArgs* p, int count, cudaStream_t s);
lr_status launch_scalar_batched(const ScalP* p, int count, cudaStream_t s);
lr_status launch_dv_merge_batched(const DvMergeP* p, int count, cudaStream_t s);
lr_status launch_dv_rows_batched(const BwArgs* p, int count, cudaStream_t s);
lr_status launch_moments_merge_batched(const MomMergeP* p, int count, cudaStream_t s);
// Training-step problems against grid sources (gp_kernel_matvec_train and
// gp_kernel_matvec_bwd with moments plan them the same way). With ws == NULL
// only *bytes is filled in.
lr_status make_train_problem(const float2* x, int64_t n, const lr_grid* qgrid, const float2* ys, const lr_grid* yg,
                             int64_t m, const float* v, float ell, float var, float* out, float* mom, char* ws,
                             BwArgs* A, MomMergeP* MM, RowInfoP* RI, size_t* bytes);
lr_status make_moment_rows_problem(const float* mom, int64_t n, bool grid, const float* g, const float* v, float ell,
                                   float var, float2* dx, double* d_len, double* d_var, char* ws, MergeArgs* M,
                                   ScalP* S, size_t* bytes);
lr_status make_dv_problem(const float2* x, int64_t n, const lr_grid* qgrid, const lr_grid* yg, const float* g,
                          float ell, float var, float* d_v, char* ws, BwArgs* A, DvMergeP* D, RowInfoP* RI,
                          size_t* bytes);
lr_status launch_vjp_batched(const VjpP* p, int count, cudaStream_t s);
lr_status launch_vjp_final_batched(const VjpFinalP* p, int count, cudaStream_t s);

// Problem constructors (planned exactly as the single-problem entry points).

lr_status make_rows_problem(const float2* x, int64_t n, const lr_grid* qgrid, const float2* ys, const lr_grid* yg,
                            int64_t m, const float* v, const float* g, float ell, float var, float2* dx, double* d_len,
                            double* d_var, float* d_v, char* ws, BwArgs* A, MergeArgs* M, ScalP* S, DvMergeP* D,
                            RowInfoP* RI, size_t* bytes);
lr_status make_rt_problem(const lr_points* p, float2* beta, float2* alpha, RtP* R);
lr_status make_vjp_problem(const lr_points* p, const float2* dbeta, double* d_lens, double* d_sub, void* ws, VjpP* V,
                           VjpFinalP* F);

// Column chunks for a reduction of row_blocks x n_tiles tasks: enough that
// every resident CTA slot (occupancy x SMs) receives about 8 tasks. Depends
// only on the problem's own sizes, so a problem is summed in the same order
// alone or inside a batch.
// Column chunks per row block so that there are about `waves` tasks per
// resident CTA slot. Grid sources that leave out exactly-zero pairs have
// smaller tasks, so they plan fewer (kSkipWaves).
constexpr int kChunkWaves = 8;
constexpr int kSkipWaves = 3;
int32_t plan_chunks(int64_t row_blocks, int64_t n_tiles, int occupancy, int n_sm, int waves = kChunkWaves);

}  // namespace lr
