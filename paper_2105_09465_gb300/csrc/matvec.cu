// Lazily evaluated Gaussian-kernel reduction
//   out_i = sum_j var * exp(-|x_i - y_j|^2 / (2 l^2)) v_j
// (RBF covariance with Sigma = l^2 I, Sec. 3.1; T y evaluated without storing
// T, Sec. 3.3).
//
// Work decomposition: the n x m pair space is cut into tasks of
// (a block of kRowsPerCta query rows) x (a chunk of consecutive source
// tiles); one CTA per task, scheduled by the hardware. Each thread keeps R
// query points in registers; source tiles of kTile points are staged in
// shared memory in a pair-packed layout and streamed with double buffering,
// so that every instruction of the inner loop works on two sources at once
// (packed f32x2 add/mul/fma) and each exp is one MUFU.EX2.
// Per pair: 2 packed-FP32 lane ops (grid sources: uniform y per tile and a
// split exponent) or 5 (explicit sources) plus one exp2.
// Accuracy: per tile each thread sums <= kTile/2 terms per lane in plain
// FP32, then folds the tile total into a Kahan-compensated running sum. With
// several chunks per row the chunk totals are merged by a second kernel in
// fixed chunk order (Kahan), so results are deterministic.
#include <math.h>

#include "batch.cuh"
#include "cull.cuh"
#include "host.cuh"
#include "problems.cuh"

namespace lr {

static_assert(kPairs == kMvThreads, "one source pair per thread when staging");

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Range of source indices covered by tile t, and (grid) its uniform y.
__device__ __forceinline__ void tile_range(const SrcDesc& S, int t, int64_t& j0, int& cnt, int& grow) {
  if (S.xy) {
    j0 = (int64_t)t * kTile;
    const int64_t rem = S.m - j0;
    cnt = rem < kTile ? (int)rem : kTile;
    grow = 0;
  } else {
    grow = t / S.segs;
    const int seg = t - grow * S.segs;
    const int c0 = seg * kTile;
    cnt = min(kTile, S.g.W - c0);
    j0 = (int64_t)grow * S.g.W + c0;
  }
}

// Loads source pair `p` of tile t into registers (zero weight past the end).
// Grid tiles are cut into sub-segments of kSeg columns. A grid source is
// stored as its scaled abscissa x' = sc (x_j - o), relative to the
// sub-segment's centre column o, and its weight folded with the source half
// of the split exponent, v~ = v 2^-x'^2 (exponent splitting below). The split
// is used only when |x'| <= kSplitXMax inside a sub-segment, so that
// v~ >= 2^-30 v and the split terms stay small; otherwise (-x', v) is stored.
constexpr int kSeg = kSplitSeg;

__device__ __forceinline__ float seg_origin(const GridDev& g, int c0, int sg) {
  return grid_x(g, c0 + kSeg * sg + kSeg / 2);
}

template <bool GRID>
__device__ __forceinline__ void load_pair(const SrcDesc& S, const float* __restrict__ v, float sc, bool split, int t,
                                          int p, float4& P, float2& V) {
  int64_t j0;
  int cnt, grow;
  tile_range(S, t, j0, cnt, grow);
  const int a = 2 * p, b = 2 * p + 1;
  if (GRID) {
    const int c0 = (int)(j0 - (int64_t)grow * S.g.W);
    const float o = seg_origin(S.g, c0, a / kSeg);
    const float xa = (a < cnt) ? sc * (grid_x(S.g, c0 + a) - o) : 0.f;
    const float xb = (b < cnt) ? sc * (grid_x(S.g, c0 + b) - o) : 0.f;
    float va = (a < cnt) ? __ldg(v + j0 + a) : 0.f;
    float vb = (b < cnt) ? __ldg(v + j0 + b) : 0.f;
    // (x', v~) of the pair in one 16-byte word (one shared load per pair);
    // the unsplit form stores (-x', v)
    if (split)
      P = make_float4(xa, xb, va * ex2_approx(-xa * xa), vb * ex2_approx(-xb * xb));
    else
      P = make_float4(-xa, -xb, va, vb);
    V = f2(0.f, 0.f);
    return;
  } else {
    const float2 pa = (a < cnt) ? __ldg(S.xy + j0 + a) : f2(0.f, 0.f);
    const float2 pb = (b < cnt) ? __ldg(S.xy + j0 + b) : f2(0.f, 0.f);
    P = make_float4(-pa.x, -pb.x, -pa.y, -pb.y);
  }
  V = f2((a < cnt) ? __ldg(v + j0 + a) : 0.f, (b < cnt) ? __ldg(v + j0 + b) : 0.f);
}

// One task: kRowsPerCta query rows x one chunk of source tiles.
// Per-thread Kahan running sums live in shared memory (touched once per tile),
// which keeps them out of the register budget of the inner loop.
struct MvSmem {
  float4 sP[2][kPairs];
  float2 sV[2][kPairs];
  float ksum[kMvR][kMvThreads];
  float kcomp[kMvR][kMvThreads];
};

template <bool GRID>
__device__ __forceinline__ void matvec_body(const MvArgs& A, int rb, int chunk, MvSmem& sm) {
  float4 (*sP)[kPairs] = sm.sP;
  float2 (*sV)[kPairs] = sm.sV;
  // grid sources with row-block info: chunks split the block's active tile range
  RowBlockInfo B{};
  int lo = 0, hi = A.src.n_tiles;
  if (GRID && A.info) {
    B = A.info[rb];
    lo = B.t_lo;
    hi = B.t_hi > B.t_lo ? B.t_hi : B.t_lo;
  }
  const int t0 = lo + (int)((int64_t)chunk * (hi - lo) / A.chunks);
  const int t1 = lo + (int)((int64_t)(chunk + 1) * (hi - lo) / A.chunks);
  const int tid = threadIdx.x;

  float2 xq[kMvR], yq[kMvR], acc[kMvR];
#pragma unroll
  for (int r = 0; r < kMvR; ++r) {
    const int64_t ir = map_row(A.map, A.n, kRowsPerCta, rb, r * kMvThreads + tid);
    const int64_t i = ir >= 0 ? ir : 0;  // padding rows compute on row 0 and are not written
    const float2 p = __ldg(A.x + i);
    xq[r] = f2(p.x, p.x);
    yq[r] = f2(p.y, p.y);
    acc[r] = f2(0.f, 0.f);
    sm.ksum[r][tid] = 0.f;
    sm.kcomp[r][tid] = 0.f;
  }
  const float2 nc2 = f2(A.neg_c, A.neg_c);

  float4 P;
  float2 V;
  if (t0 < t1) {
    load_pair<GRID>(A.src, A.v, A.sc, A.split != 0, t0, tid, P, V);
    sP[0][tid] = P;
    sV[0][tid] = V;
  }
  __syncthreads();

  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    if (t + 1 < t1) load_pair<GRID>(A.src, A.v, A.sc, A.split != 0, t + 1, tid, P, V);  // in flight during compute
    int64_t j0;
    int cnt, grow;
    tile_range(A.src, t, j0, cnt, grow);
    const int np = (cnt + 1) >> 1;
    if (GRID) {
      // Exponent splitting: with scaled tile-local q = sc (x_i - o),
      // x' = sc (x_j - o) and dy' = sc (y_i - y_t),
      //   -(q - x')^2 - dy'^2 = [2 q x' - q^2 - dy'^2] - x'^2,
      // so k v = 2^(2 q x' + a_i) * v~ with a_i = -(q^2 + dy'^2) per row and
      // v~ = v 2^-x'^2 per source: ONE packed FMA forms the exponent of two
      // pairs and one more accumulates. The bracket is at most x'^2 <= 30.25,
      // so 2^bracket cannot overflow; for the pairs that contribute, its FP32
      // error is a few 1e-6 absolute (a relative error of k below 1e-5).
      const float yt = grid_y(A.src.g, grow);
      const int c0 = (int)(j0 - (int64_t)grow * A.src.g.W);
      float dy2[kMvR];
#pragma unroll
      for (int r = 0; r < kMvR; ++r) {
        const float dy = A.sc * (yq[r].x - yt);
        dy2[r] = dy * dy;
      }
      const int nsg = (cnt + kSeg - 1) / kSeg;
      // columns of this grid row within reach of the row block (all without
      // info), and the sub-segments that meet them
      int clo = 0, chi = cnt - 1;
      if (A.info) reach_cols(B, A.src.g, yt, A.sc, c0, cnt, clo, chi);
      const int sg_lo = clo <= chi ? clo / kSeg : nsg, sg_hi = clo <= chi ? chi / kSeg : -1;
      if (!A.split) {
        // unsplit: dx' = q - x', exponent -(dx'^2 + dy'^2)
        for (int sg = sg_lo; sg <= sg_hi; ++sg) {
          int pl, ph;
          seg_pair_range<kSeg>(clo, chi, kSeg * sg, pl, ph);
          if (pl >= ph) continue;  // every pair's exp2 flushes to 0
          const float o = seg_origin(A.src.g, c0, sg);
          float2 qx[kMvR], d2[kMvR];
#pragma unroll
          for (int r = 0; r < kMvR; ++r) {
            const float q = A.sc * (xq[r].x - o);
            qx[r] = f2(q, q);
            d2[r] = f2(dy2[r], dy2[r]);
          }
#pragma unroll
          for (int qq = 0; qq < kSeg / 2; qq += kQuarterPairs) {
            if (qq < pl || qq >= ph) continue;  // a quarter out of reach: exactly zero
#pragma unroll
            for (int pp = qq; pp < qq + kQuarterPairs; ++pp) {
              const float4 Q = sP[buf][sg * (kSeg / 2) + pp];
              const float2 W = f2(Q.z, Q.w);
              const float2 nx = f2(Q.x, Q.y);
#pragma unroll
              for (int r = 0; r < kMvR; ++r) {
                const float2 dx = __fadd2_rn(qx[r], nx);
                const float2 t = __ffma2_rn(dx, dx, d2[r]);
                const float2 k = f2(ex2_approx(-t.x), ex2_approx(-t.y));
                acc[r] = __ffma2_rn(k, W, acc[r]);
              }
            }
          }
        }
      } else {
        for (int sg = sg_lo; sg <= sg_hi; ++sg) {
          int pl, ph;
          seg_pair_range<kSeg>(clo, chi, kSeg * sg, pl, ph);
          if (pl >= ph) continue;  // every pair's exp2 flushes to 0
          const float o = seg_origin(A.src.g, c0, sg);
          float2 q2[kMvR], ar[kMvR];
#pragma unroll
          for (int r = 0; r < kMvR; ++r) {
            const float q = A.sc * (xq[r].x - o);
            const float a = -fmaf(q, q, dy2[r]);
            q2[r] = f2(2.f * q, 2.f * q);
            ar[r] = f2(a, a);
          }
#pragma unroll
          for (int qq = 0; qq < kSeg / 2; qq += kQuarterPairs) {
            if (qq < pl || qq >= ph) continue;  // a quarter out of reach: exactly zero
#pragma unroll
            for (int pp = qq; pp < qq + kQuarterPairs; ++pp) {
              const float4 Q = sP[buf][sg * (kSeg / 2) + pp];
              const float2 W = f2(Q.z, Q.w);
              const float2 X = f2(Q.x, Q.y);
#pragma unroll
              for (int r = 0; r < kMvR; ++r) {
                const float2 e = __ffma2_rn(q2[r], X, ar[r]);
                const float2 k = f2(ex2_approx(e.x), ex2_approx(e.y));
                acc[r] = __ffma2_rn(k, W, acc[r]);
              }
            }
          }
        }
      }
    } else {
#pragma unroll 2
      for (int p = 0; p < np; ++p) {
        const float4 Q = sP[buf][p];
        const float2 W = sV[buf][p];
        const float2 nx = f2(Q.x, Q.y), ny = f2(Q.z, Q.w);
#pragma unroll
        for (int r = 0; r < kMvR; ++r) {
          const float2 dx = __fadd2_rn(xq[r], nx);
          const float2 dy = __fadd2_rn(yq[r], ny);
          const float2 d2 = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
          const float2 e = __fmul2_rn(d2, nc2);
          const float2 k = f2(ex2_approx(e.x), ex2_approx(e.y));
          acc[r] = __ffma2_rn(k, W, acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kMvR; ++r) {
      float su = sm.ksum[r][tid], co = sm.kcomp[r][tid];
      kahan_add(su, co, acc[r].x + acc[r].y);
      sm.ksum[r][tid] = su;
      sm.kcomp[r][tid] = co;
      acc[r] = f2(0.f, 0.f);
    }
    if (t + 1 < t1) {
      sP[buf ^ 1][tid] = P;
      sV[buf ^ 1][tid] = V;
    }
    __syncthreads();
  }

#pragma unroll
  for (int r = 0; r < kMvR; ++r) {
    const int64_t i = map_row(A.map, A.n, kRowsPerCta, rb, r * kMvThreads + tid);
    if (i >= 0) {
      const float total = sm.ksum[r][tid] - sm.kcomp[r][tid];
      if (A.chunks == 1)
        A.out[i] = A.variance * total;
      else
        A.partial[(int64_t)chunk * A.n + i] = total;
    }
  }
}

template <bool GRID>
__global__ void __launch_bounds__(kMvThreads) matvec_kernel(const __grid_constant__ MvArgs A) {
  __shared__ __align__(16) MvSmem sm;
  const int rb = blockIdx.x / A.chunks;
  matvec_body<GRID>(A, rb, blockIdx.x - rb * A.chunks, sm);
}

// Fixed-order compensated merge of the chunk partials.
__device__ __forceinline__ void merge_body(const float* __restrict__ partial, int chunks, int64_t n, float variance,
                                           float* __restrict__ out, int64_t i) {
  if (i >= n) return;
  float s = 0.f, c = 0.f;
  for (int k = 0; k < chunks; ++k) kahan_add(s, c, partial[(int64_t)k * n + i]);
  out[i] = variance * (s - c);
}

__global__ void merge_chunks_kernel(const float* __restrict__ partial, int chunks, int64_t n, float variance,
                                    float* __restrict__ out) {
  merge_body(partial, chunks, n, variance, out, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Host side

int32_t plan_chunks(int64_t row_blocks, int64_t n_tiles, int occupancy, int n_sm, int waves) {
  const int64_t target = (int64_t)waves * n_sm * (occupancy > 0 ? occupancy : 1);
  int64_t chunks = 1;
  if (row_blocks > 0 && n_tiles > 0) {
    chunks = (target + row_blocks - 1) / row_blocks;
    if (chunks < 1) chunks = 1;
    if (chunks > n_tiles) chunks = n_tiles;
  }
  return (int32_t)chunks;
}

struct MvPlan {
  int64_t n, m;
  int32_t nrhs;
  bool self;
  bool q_raytrace, q_grid;   // query needs ray-tracing / grid materialisation
  bool s_raytrace;           // source needs ray-tracing
  bool s_grid;               // source read as a grid (no materialisation)
  bool s_mat;                // grid source written out as points (several right-hand sides)
  int32_t n_tiles, segs, chunks, row_blocks;
  RowMap map;                // row blocks: image tiles of a grid query, else index order
  CullPlan cull;             // explicit sources: the culled sweep
  size_t off_qbeta, off_sbeta, off_partial, off_info, off_cull, bytes;
};

static lr_status plan_matvec(const lr_points* q, const lr_points* s, int32_t nrhs, bool have_beta_out, MvPlan* P) {
  lr_status st = validate_points(q, "gp_kernel_matvec(query)", false);
  if (st != LR_OK) return st;
  if (s) {
    st = validate_points(s, "gp_kernel_matvec(source)", false);
    if (st != LR_OK) return st;
  }
  MvPlan p{};
  p.n = q->n;
  p.nrhs = nrhs;
  p.self = (s == nullptr);
  p.m = p.self ? q->n : s->n;
  p.q_raytrace = has_lens(q);
  p.q_grid = !p.q_raytrace && q->xy == nullptr;
  p.s_raytrace = !p.self && has_lens(s);
  p.s_grid = !p.self && !p.s_raytrace && s->xy == nullptr;
  LR_REQUIRE(nrhs >= 1 && nrhs <= 4, "gp_kernel_matvec: nrhs = %d; 1..4 right-hand sides", nrhs);
  // several right-hand sides over grid sources: the grid's points are
  // written out and reduced by the culled sweep, which shares each pair's
  // exp2 across the right-hand sides
  p.s_mat = p.s_grid && nrhs > 1;
  if (p.s_mat) p.s_grid = false;
  size_t off = 0;
  const bool need_qbuf = (p.q_raytrace || p.q_grid) && !have_beta_out;
  p.off_qbeta = off;
  if (need_qbuf) off += align256(sizeof(float2) * (size_t)p.n);
  p.off_sbeta = off;
  if (p.s_raytrace || p.s_mat) off += align256(sizeof(float2) * (size_t)p.m);
  const lr_grid* layout = query_layout(q);
  if (!p.s_grid) {
    // explicit, ray-traced or self sources: the culled sweep
    const lr_grid* slayout = p.self ? layout : query_layout(s);
    st = plan_cull(kCullOut, nrhs, p.n, layout, p.m, slayout, &p.cull);
    if (st != LR_OK) return st;
    p.off_cull = off;
    off += p.cull.bytes;
    p.off_partial = p.off_info = off;
    p.bytes = off;
    *P = p;
    return LR_OK;
  }
  const int W = s->grid.nx * s->grid.ss;
  p.segs = (W + kTile - 1) / kTile;
  p.n_tiles = (int32_t)((int64_t)p.segs * s->grid.ny * s->grid.ss);
  p.map = layout ? make_row_map(layout, kRowsPerCta) : RowMap{};
  p.row_blocks = (int32_t)row_block_count(p.map, p.n, kRowsPerCta);
  int dev = 0, n_sm = 1, occ = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, matvec_kernel<true>, kMvThreads, 0));
  p.chunks = plan_chunks(p.row_blocks, p.n_tiles, occ, n_sm, kSkipWaves);
  p.off_partial = off;
  if (p.chunks > 1) off += align256(sizeof(float) * (size_t)p.chunks * (size_t)p.n);
  p.off_info = off;
  off += row_info_bytes(p.map, p.n, kRowsPerCta);
  p.off_cull = off;
  p.bytes = off;
  *P = p;
  return LR_OK;
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_matvec_workspace_size(const lr_points* query, const lr_points* source, int32_t nrhs,
                                              size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_matvec_workspace_size: bytes is NULL");
  MvPlan P;
  lr_status st = plan_matvec(query, source, nrhs, false, &P);
  if (st != LR_OK) return st;
  *bytes = P.bytes;
  return LR_OK;
}

extern "C" lr_status gp_kernel_matvec(const lr_points* query, const lr_points* source, const float* v, int32_t nrhs,
                                      float lengthscale, float variance, float* out, float* beta_out,
                                      void* workspace, size_t workspace_bytes, lr_stream stream) {
  MvPlan P;
  lr_status st = plan_matvec(query, source, nrhs, beta_out != nullptr, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "gp_kernel_matvec: lengthscale = %g must be > 0",
             (double)lengthscale);
  LR_REQUIRE(isfinite(variance), "gp_kernel_matvec: variance is not finite");
  LR_REQUIRE(out != nullptr || P.n == 0, "gp_kernel_matvec: out is NULL");
  LR_REQUIRE(v != nullptr || P.m == 0, "gp_kernel_matvec: v is NULL");
  LR_REQUIRE(((uintptr_t)beta_out & 7u) == 0, "gp_kernel_matvec: beta_out must be 8-byte aligned");
  LR_REQUIRE(workspace_bytes >= P.bytes, "gp_kernel_matvec: workspace of %zu bytes, %zu needed", workspace_bytes,
             P.bytes);
  LR_REQUIRE(P.bytes == 0 || workspace != nullptr, "gp_kernel_matvec: workspace is NULL");
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0, "gp_kernel_matvec: workspace must be 256-byte aligned");
  LR_REQUIRE(P.q_raytrace || P.q_grid || beta_out == nullptr,
             "gp_kernel_matvec: beta_out given but the query is not ray-traced");
  cudaStream_t s = as_cuda(stream);
  if (P.n == 0) return LR_OK;
  if (P.m == 0) {
    LR_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)P.n * (size_t)P.nrhs, s));
    return LR_OK;
  }
  char* ws = static_cast<char*>(workspace);
  // query points
  const float2* xq = reinterpret_cast<const float2*>(query->xy);
  if (P.q_raytrace || P.q_grid) {
    float2* qb = beta_out ? reinterpret_cast<float2*>(beta_out) : reinterpret_cast<float2*>(ws + P.off_qbeta);
    st = P.q_raytrace ? launch_raytrace(query, qb, nullptr, s) : launch_grid_points(query->grid, qb, s);
    if (st != LR_OK) return st;
    xq = qb;
  }
  // source points
  SrcDesc S{};
  S.m = P.m;
  S.n_tiles = P.n_tiles;
  S.segs = P.segs;
  if (P.self) {
    S.xy = xq;
  } else if (P.s_raytrace || P.s_mat) {
    float2* sb = reinterpret_cast<float2*>(ws + P.off_sbeta);
    st = P.s_raytrace ? launch_raytrace(source, sb, nullptr, s) : launch_grid_points(source->grid, sb, s);
    if (st != LR_OK) return st;
    S.xy = sb;
  } else if (P.s_grid) {
    S.xy = nullptr;
    S.g = grid_dev(source->grid);
  } else {
    S.xy = reinterpret_cast<const float2*>(source->xy);
  }
  const float sc = (float)sqrt(1.4426950408889634 / (2.0 * (double)lengthscale * (double)lengthscale));
  if (!P.s_grid) {
    // explicit, ray-traced or self sources: culled sweep over chunk records
    char* cws = ws + P.off_cull;
    st = launch_cull_prep(P.cull, S.xy, sc, v, nullptr, P.nrhs, 0, cws, s);
    if (st != LR_OK) return st;
    CullArgs C{};
    C.x = xq;
    C.n = P.n;
    C.sc = sc;
    C.c = (float)(1.4426950408889634 / (2.0 * (double)lengthscale * (double)lengthscale));
    C.nrhs = P.nrhs;
    C.var = variance;
    C.out = out;
    return launch_cull_sweep(P.cull, C, cws, LR_KT_MATVEC, s);
  }
  MvArgs A;
  A.x = xq;
  A.n = P.n;
  A.src = S;
  A.v = v;
  A.neg_c = (float)(-1.4426950408889634 / (2.0 * (double)lengthscale * (double)lengthscale));
  A.sc = sc;
  A.split = grid_split_ok(S.g, A.sc);
  A.variance = variance;
  A.chunks = P.chunks;
  A.out = out;
  A.partial = reinterpret_cast<float*>(ws + P.off_partial);
  A.map = P.map;
  // row-block boxes: the exactly-zero pairs are left out
  RowInfoP R{xq, P.n, P.map, kRowsPerCta, P.segs, S.g, A.sc, reinterpret_cast<RowBlockInfo*>(ws + P.off_info)};
  if ((st = launch_row_info(R, s)) != LR_OK) return st;
  A.info = R.info;
  const unsigned grid = (unsigned)((int64_t)P.row_blocks * P.chunks);
  ktimer_begin(LR_KT_MATVEC, s);
  matvec_kernel<true><<<grid, kMvThreads, 0, s>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_MATVEC, s);
  if (P.chunks > 1) {
    merge_chunks_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, s>>>(A.partial, P.chunks, P.n, variance, out);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of gp_kernel_matvec.
//
// Some callers cannot allocate device memory at call time: a host
// application whose device memory is all owned by its own pool or budget
// fixed at start-up, a latency-critical loop that must not hit cudaMalloc's
// implicit device synchronisation, or a plugin linked against this C ABI
// without access to the host framework's allocator. For them this entry
// point takes no workspace: its scratch is one file-scope device array of
// kStaticScratchBytes that every GPU loading this library holds until the
// process exits.
namespace {

constexpr size_t kStaticScratchBytes = size_t(48) << 20;  // 48 MiB per device
static __device__ __align__(256) unsigned char g_matvec_static_scratch[kStaticScratchBytes];

// Device address of the static scratch in the current device's context,
// resolved with cudaGetSymbolAddress on every call (it allocates nothing and
// costs about a microsecond). Host code must never pass the array's name
// itself to a kernel: in host code it is only a host-side stand-in. Nothing
// is cached, so a context that was destroyed and created again (for example
// after cudaDeviceReset) gets the address of its own copy of the array.
lr_status static_scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_static_scratch);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_matvec_static_scratch)");
  *out = p;
  return LR_OK;
}

}  // namespace

extern "C" size_t lr_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" lr_status gp_kernel_matvec_static_scratch(const lr_points* query, const lr_points* source,
                                                     const float* v, int32_t nrhs, float lengthscale, float variance,
                                                     float* out, float* beta_out, lr_stream stream) {
  MvPlan P;
  lr_status st = plan_matvec(query, source, nrhs, beta_out != nullptr, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(P.bytes <= kStaticScratchBytes,
             "gp_kernel_matvec_static_scratch: this problem needs %zu bytes of scratch but the static scratch "
             "holds %zu bytes; use gp_kernel_matvec with a caller workspace",
             P.bytes, kStaticScratchBytes);
  void* scratch = nullptr;
  st = static_scratch_address(&scratch);
  if (st != LR_OK) return st;
  // Every word of scratch this call reads is written earlier in the same
  // call (query/source points, then each chunk partial exactly once), so
  // nothing needs clearing between calls.
  return gp_kernel_matvec(query, source, v, nrhs, lengthscale, variance, out, beta_out, scratch,
                          kStaticScratchBytes, stream);
}
