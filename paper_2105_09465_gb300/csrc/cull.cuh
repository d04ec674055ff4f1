// Culled reduction over explicit point sets (sources given as points, including
// the self-kernel of the ray-traced pixels against themselves).
//
// Chunked point sets. The sources are cut into chunks of kChunkPts points and
// the chunks into groups of kGroupChunks. When the points carry an image layout
// (ray-traced pixels) a chunk is an 8 x 4 block of pixels and a group an 8 x 8
// block of chunks; the lens map is continuous, so a chunk's points stay close
// together in the source plane. Without a layout chunks are consecutive indices.
// A prepare kernel writes, per chunk, its bounding box and a record block:
//   float4 box       (xlo, ylo, xhi, yhi)
//   float4 head      (points in the chunk, smallest reach scale s of its
//                    windowed points (kCullWinCols), 0, 0)
//   float4 xy[16]    source pair p = points (2p, 2p+1): (xa, xb, ya, yb)
//   float2 w[NW][16] the pairs' weights
// Positions are stored as they are: the sweeps form x_j - x_i directly, which
// FP32 rounds correctly (relative error at most 2^-24 of the difference, and
// none at all for points within a factor of two of each other), and only
// then scale it: t = c |x_j - x_i|^2, c = log2(e) / (2 l^2), k = 2^-t. Offsets
// from a chunk origin, or pre-scaled coordinates, would each carry a rounding
// error proportional to the offset, which for a row whose sum is made of far
// pairs (t ~ 30 to 100) grows past the 2e-5 relative bound.
//
// Exact skipping. A pair with t > 126 has an exponent below -126, where the
// flush-to-zero exp2 returns exactly 0. A row block (or one warp of it) leaves
// out every group and chunk whose box is farther than sqrt(kSkipT) =
// sqrt(170) scaled units from its own box; the margin over 126 absorbs the
// FP32 rounding of both distances. A left-out chunk's partial sums are exact
// zeros, and the kernels fold a chunk's sums into the row totals only when
// they are nonzero (the forward) or add them plainly (the moments, where
// adding +0 changes nothing), so culled and unculled sweeps give the same
// bits.
//
// Windowed kinds (the image-plane transmission, Sec. 3.4): the pair's
// exponent is -(log2 e / 2) d^T C_i^-1 d with the covariance C_i = Z_i +
// (l^2/2) I of the windowed point i, at most -s_i^2 |d|^2 with
// s_i = sqrt(log2(e) / (2 lambda_max(C_i))). The same box test then runs with
// the smallest s_i of the points involved: of the rows (a warp's or a CTA's)
// when the rows carry the windows, of the chunk (stored with its box) when
// the sources do.
//
// Window precision. At the paper's narrow image-plane kernels (2 to 10 mas)
// the windows of magnified pixels are thin ellipses: C_i has a condition
// number kappa of order 100. Forming det C_i or the quadratic form
// mxx dx^2 + 2 mxy dx dy + myy dy^2 in FP32 loses about u kappa |exponent|,
// past the 2e-5 bound. So a prepare kernel forms C_i = Z_i + (l^2/2) I and
// det C_i in FP64 (the sums and the one cancelling difference; the rest is
// well-conditioned in FP32) and writes, per point, the upper Cholesky factor
// R of C_i^-1 scaled by
// k = sqrt(log2(e) / 2), (a, b, c) = k (r11, r12, r22), the normalisation
// N_i = 1 / (2 pi sqrt(det C_i)) and s_i. A pair then evaluates
// w = (a dx + b dy, c dy), exponent -|w|^2 (a sum of squares: error about
// u sqrt(kappa) |exponent|), and k^2 C^-1 d = R^T w = (a w1, b w1 + c w2).
#pragma once
#include "rowmap.cuh"
#include "tma.cuh"

namespace lr {

constexpr int kCullThreads = 128;
constexpr int kChunkPts = 32;
constexpr int kChunkPairs = kChunkPts / 2;
constexpr int kGroupChunks = 64;
constexpr int kChunkW = 8, kChunkH = 4;  // chunk of an image layout (pixels)
constexpr int kGroupW = 8, kGroupH = 8;  // group of an image layout (chunks)
constexpr int kCullTileW = 16;           // row blocks: 16-pixel-wide image tiles
constexpr int kRecHead = 32;             // box + head
constexpr int kRecXY = 16 * kChunkPairs;  // float4 per source pair

__host__ __device__ constexpr int rec_bytes(int nw) { return kRecHead + kRecXY + 8 * kChunkPairs * nw; }

struct ChunkLayout {
  int32_t W, H;    // image layout (W * H == n), or W == 0: index order
  int32_t GW, GH;  // groups per layout row / column
  int64_t n;
  int32_t n_chunks, n_groups;
};

inline ChunkLayout make_chunk_layout(const lr_grid* layout, int64_t n) {
  ChunkLayout L{};
  L.n = n;
  if (layout) {
    L.W = layout->nx * layout->ss;
    L.H = layout->ny * layout->ss;
    L.GW = (L.W + kChunkW * kGroupW - 1) / (kChunkW * kGroupW);
    L.GH = (L.H + kChunkH * kGroupH - 1) / (kChunkH * kGroupH);
    L.n_groups = L.GW * L.GH;
  } else {
    const int64_t chunks = (n + kChunkPts - 1) / kChunkPts;
    L.n_groups = (int32_t)((chunks + kGroupChunks - 1) / kGroupChunks);
  }
  L.n_chunks = L.n_groups * kGroupChunks;
  return L;
}

// Index of the point in slot s of chunk c, or -1 (an empty slot).
__device__ __forceinline__ int64_t chunk_point(const ChunkLayout& L, int c, int s) {
  if (L.W == 0) {
    const int64_t i = (int64_t)c * kChunkPts + s;
    return i < L.n ? i : -1;
  }
  const int g = c / kGroupChunks, lc = c - g * kGroupChunks;
  const int gy = g / L.GW, gx = g - gy * L.GW;
  const int ly = lc / kGroupW, lx = lc - ly * kGroupW;
  const int col = (gx * kGroupW + lx) * kChunkW + (s % kChunkW);
  const int row = (gy * kGroupH + ly) * kChunkH + (s / kChunkW);
  return (col < L.W && row < L.H) ? (int64_t)row * L.W + col : -1;
}

// True when every pair between the two boxes (raw coordinates) has scaled
// squared distance above kSkipT. An empty box (lo > hi) is far from anything.
__device__ __forceinline__ bool boxes_far(float4 a, float4 b, float sc) {
  const float dx = fmaxf(fmaxf(a.x - b.z, b.x - a.z), 0.f);
  const float dy = fmaxf(fmaxf(a.y - b.w, b.y - a.w), 0.f);
  const float sx = sc * dx, sy = sc * dy;
  return !(fmaf(sx, sx, sy * sy) <= kSkipT);
}

// What a sweep computes and its chunk records' weights hold.
enum CullKind : int32_t {
  kCullOut = 0,      // nrhs weights: the columns of v   (forward)
  kCullMom = 1,      // one weight a                     (row moments of a)
  kCullSelf = 2,     // a (v) and b (g), nrhs columns each  (self-kernel backward)
  kCullWin = 3,      // windowed forward: rows carry windows, weight v
  kCullWinRows = 4,  // windowed backward, row sums: rows carry windows, weight v
  kCullWinCols = 5,  // windowed backward, column sums: the sources (the
                     // windowed points) carry their window constants (a, b, c)
                     // and g N as their four weights
};

__host__ __device__ constexpr int cull_nw(int kind, int nrhs) {
  return kind == kCullOut ? nrhs
                          : (kind == kCullSelf ? 2 * nrhs : (kind == kCullWinCols ? 4 : 1));
}

// Sums per row of a sweep.
__host__ __device__ constexpr int cull_k(int kind, int nw) {
  return kind == kCullOut ? nw
                          : kind == kCullMom ? 4
                          : kind == kCullSelf ? 7 * (nw / 2)
                          : kind == kCullWin ? 1
                          : kind == kCullWinRows ? 6 : 3;
}

// Per-point window constants (see "Window precision" above): wcoef[i] =
// (a, b, c, N) and wreach[i] = s_i from the windows z [n][3] and l.
lr_status launch_window_prep(const float* z, int64_t n, float lengthscale, float4* wcoef, float* wreach,
                             cudaStream_t s);

struct CullPrepP {
  const float2* pts;  // [n] source points
  ChunkLayout L;
  float sc;
  int32_t kind, nw;
  const float* a;     // kOut: v [n][stride]; kMom / kSelf: column `col` of a [n][stride]
  const float* b;     // kSelf: column `col` of b [n][stride]
  int32_t stride, col;
  char* rec;          // [n_chunks][rec_bytes(nw)]
  float4* cbox;       // [n_chunks]
  float4* gbox;       // [n_groups]
  // kCullWinCols: the points' window constants (launch_window_prep; a = g);
  // the chunks' and groups' smallest reach scales
  const float4* wcoef;
  const float* wreach;
  float* csc;         // [n_chunks]
  float* gsc;         // [n_groups]
};

// Outputs of a culled sweep, by kind:
//  kCullOut:  out[i][r] = var * sum_j k_ij v_j[r]
//  kCullMom:  row moments of a over the sources:
//             A = sum k a, Bx/By = sum k a (x_j - x_i), C = sum k a d^2;
//             with g == NULL they are written to mom [4][n] (and out = var A);
//             else the row gradients d_x = var/l^2 g_i (Bx, By) and the
//             scalar partials (d_l, d_var) of g_i C, g_i A
//  kCullSelf: self-kernel backward for nrhs right-hand sides in one sweep
//             (the pair's exp2 shared): d_v = var sum_j k g_j per column,
//             d_x both roles summed over the columns, scalar partials.
//  kCullWin:  out[i] = N_i sum_j G'_ij v_j, G' = 2^(-|R_i d|^2 k^2)
//  kCullWinRows: per row, with d = x_i - y_j and u = k^2 C_i^-1 d, the six
//             sums S = sum v G', P = sum v G' u, Q = sum v G' u u^T (xx, xy, yy)
//  kCullWinCols: per row (a source of the windowed reduction), with
//             d = x_i - y_j and u = k^2 C_j^-1 d, T = sum gN G', U = sum gN G' u
//             The two backward kinds write partial[split][K][n] whatever the
//             split count; the windowed backward merges them.
struct CullArgs {
  const float2* x;   // [n] query points
  int64_t n;
  RowMap map;        // row blocks (image tiles of kCullTileW columns, or index order)
  int32_t rows_per_cta;
  float sc;          // sqrt(c): the skipping test's scale
  float c;           // log2(e) / (2 l^2)
  int32_t cull;      // 0: evaluate every chunk (same order, same bits)
  const char* rec;
  const float4* cbox;
  const float4* gbox;
  int32_t n_chunks, n_groups;
  int32_t splits;    // group ranges per row block (> 1: partials + merge)
  int32_t nrhs;      // kCullOut: weights per source
  float var;
  float dx_scale;    // var / l^2
  float dl_scale;    // var / l^3
  float* out;        // kCullOut: [n][nrhs]; kCullMom store: [n]
  float* mom;        // kCullMom store: [4][n]
  const float* g;    // kCullMom grad, kCullSelf: g of the rows, column col of [n][stride]
  const float* vrow; // kCullSelf: v of the rows, same layout
  int32_t stride, col;
  float2* d_x;       // row gradients (NULL: not wanted)
  int32_t dx_accumulate;  // add into d_x (later right-hand sides)
  float* d_v;        // kCullSelf: [n][stride] at column col
  double* scal_part; // [partial blocks][2]: d_l, d_var partials
  float* partial;    // splits > 1: [splits][K][n]
  const float4* wcoef;  // kCullWin, kCullWinRows: the rows' window constants (a, b, c, N)
  const float* wreach;  // and reach scales (launch_window_prep)
  // kCullWin with a Gaussian likelihood in the epilogue (lik_data != NULL):
  // out = f_in (or 0) + this reduction, lik_g = (out - data) / sigma^2, and
  // the rows' (out - data)^2 / (2 sigma^2) summed into scal_part
  const float* f_in;
  const float* lik_data;
  float lik_isig2;      // 1 / sigma^2
  float* lik_g;
  const float* csc;  // kCullWinCols: reach scales of the chunks and groups
  const float* gsc;
  int* fault;        // device fault word (a bulk-copy wait that ran out)
  unsigned long long* count;  // diagnostic: [0] valid pairs, [1] pair slots evaluated
                              // (non-NULL: count only, no outputs written)
};

// Plan of one culled sweep: source chunks, query row blocks, group ranges per
// row block and the workspace offsets (records, boxes, partials, scalars).
struct CullPlan {
  int32_t kind, nw, K;
  ChunkLayout L;
  RowMap map;
  int32_t rows_per_cta;
  int64_t row_blocks;
  int32_t splits;
  int64_t scal_blocks;  // blocks that write scalar partials
  size_t off_rec, off_cbox, off_gbox, off_csc, off_gsc, off_partial, off_scal, bytes;
};

// 1 unless lr_set_pair_culling(0) switched exact skipping off.
int cull_enabled();
// Plans a sweep of n query points (image layout qlayout or NULL) against m
// sources (layout slayout or NULL) with nrhs right-hand sides (kCullOut).
lr_status plan_cull(int kind, int nrhs, int64_t n, const lr_grid* qlayout, int64_t m, const lr_grid* slayout,
                    CullPlan* P);
// Writes the source chunks' boxes and records into ws (offsets of P):
// kCullOut weights a [m][stride] (all nrhs columns), kCullMom column col of a,
// kCullSelf column col of a and of b, kCullWin / kCullWinRows a [m],
// kCullWinCols the points' window constants (wcoef, wreach) and g = a [m].
lr_status launch_cull_prep(const CullPlan& P, const float2* pts, float sc, const float* a, const float* b,
                           int32_t stride, int32_t col, char* ws, cudaStream_t s, const float4* wcoef = nullptr,
                           const float* wreach = nullptr);
// The sweep (and merge when P.splits > 1); A carries the kind's outputs.
// timer_id: an LR_KT_* launch-timer id, or -1.
lr_status launch_cull_sweep(const CullPlan& P, CullArgs A, char* ws, int timer_id, cudaStream_t s);
// d_len, d_var from nblk scalar partials (fixed order, FP64).
lr_status launch_cull_scalar_final(const double* part, int64_t nblk, double* d_len, double* d_var, cudaStream_t s);

}  // namespace lr
