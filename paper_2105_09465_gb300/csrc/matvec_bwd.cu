// Backward of the Gaussian-kernel reduction, recompute-only (k is never
// stored). For Loss = sum_i g_i out_i with out_i = sum_j var k_ij v_j,
// k_ij = exp(-|x_i - y_j|^2 / (2 l^2)):
//   d_x_i = var/l^2 * g_i sum_j k_ij v_j (y_j - x_i)            (row role)
//         + var/l^2 * v_i sum_j k_ij g_j (y_j - x_i)            (column role, self-kernel)
//   d_v_j = var sum_i k_ij g_i
//   d_y_j = var/l^2 * v_j sum_i k_ij g_i (x_i - y_j)            (explicit, non-self sources)
//   d_l   = var/l^3 * sum_ij g_i v_j k_ij |x_i - y_j|^2
//   d_var = sum_ij g_i v_j k_ij
// The row pass runs one sweep over the pairs with the query block in
// registers (same tiling as the forward pass) and accumulates, per row,
// A = sum k v, B = sum k v (x_i - y_j), C = sum k v e (e = -log2(e) d^2/(2 l^2))
// and, for a self-kernel, D = sum k g, E = sum k g (x_i - x_j). Chunk partials
// are merged in fixed order (Kahan), scalars are reduced in FP64. d_v and d_y
// of non-self sources are the same reductions with the roles of the two point
// sets swapped.
#include <math.h>

#include "host.cuh"
#include "cull.cuh"
#include "problems.cuh"

namespace lr {

static_assert(kBwPairs == kBwThreads, "one source pair per thread when staging");
constexpr int kBwSeg = 16;  // grid sub-segment (columns) of the tile-local coordinates

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Warp reduce-scatter of the kBwSeg per-lane sums kgs[] of one sub-segment:
// after the halving stages lane L holds the warp total of source (L >> 1) & 15,
// which the even lanes store to dvred_w[source].
__device__ __forceinline__ void warp_reduce_scatter(float (&kgs)[kBwSeg], int lane, float* dvred_w) {
#pragma unroll
  for (int h = kBwSeg / 2, m = 16; h >= 1; h >>= 1, m >>= 1) {
    const bool upper = (lane & m) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float lo = kgs[i], hi = kgs[i + h];
      const float send = upper ? lo : hi;
      const float keep = upper ? hi : lo;
      kgs[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  kgs[0] += __shfl_xor_sync(0xffffffffu, kgs[0], 1);
  if ((lane & 1) == 0) dvred_w[(lane >> 1) & 15] = kgs[0];
}

// The same reduction for kgs filled in the lane-permuted order of dv_pairs_perm
// (slot pp of lane l holds source pair pp ^ ((l >> 2) & 7)): at every halving
// the half a lane keeps is already its lower half, so only the last pair needs
// a select. The lanes combine in the same tree as above, so the sums are the
// same bits.
__device__ __forceinline__ void warp_reduce_scatter_perm(float (&kgs)[kBwSeg], int lane, float* dvred_w) {
#pragma unroll
  for (int h = kBwSeg / 2, m = 16; h >= 2; h >>= 1, m >>= 1) {
#pragma unroll
    for (int i = 0; i < h; ++i) kgs[i] += __shfl_xor_sync(0xffffffffu, kgs[i + h], m);
  }
  const bool upper = (lane & 2) != 0;
  const float send = upper ? kgs[0] : kgs[1];
  const float keep = upper ? kgs[1] : kgs[0];
  kgs[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  kgs[0] += __shfl_xor_sync(0xffffffffu, kgs[0], 1);
  if ((lane & 1) == 0) dvred_w[(lane >> 1) & 15] = kgs[0];
}

__device__ __forceinline__ void bw_tile_range(const BwSrc& S, int t, int64_t& j0, int& cnt, int& grow) {
  if (S.xy) {
    j0 = (int64_t)t * kBwTile;
    const int64_t rem = S.m - j0;
    cnt = rem < kBwTile ? (int)rem : kBwTile;
    grow = 0;
  } else {
    grow = t / S.segs;
    const int c0 = (t - grow * S.segs) * kBwTile;
    cnt = min(kBwTile, S.g.W - c0);
    j0 = (int64_t)grow * S.g.W + c0;
  }
}

template <bool GRID, bool SELF, bool SPLIT>
__device__ __forceinline__ void bw_load_pair(const BwArgs& A, int t, int p, float4& P, float2& V, float2& Gp) {
  int64_t j0;
  int cnt, grow;
  bw_tile_range(A.src, t, j0, cnt, grow);
  const int a = 2 * p, b = 2 * p + 1;
  if (GRID) {
    // scaled tile-local abscissae (see the forward pass)
    const int c0 = (int)(j0 - (int64_t)grow * A.src.g.W);
    const float o = grid_x(A.src.g, c0 + kBwSeg * (a / kBwSeg) + kBwSeg / 2);
    const float xa = (a < cnt) ? A.sc * (grid_x(A.src.g, c0 + a) - o) : 0.f;
    const float xb = (b < cnt) ? A.sc * (grid_x(A.src.g, c0 + b) - o) : 0.f;
    if (SPLIT) {
      // split exponent: v~ = v 2^-x'^2 and its first two x' moments
      const float va = (a < cnt) ? __ldg(A.v + j0 + a) * ex2_approx(-xa * xa) : 0.f;
      const float vb = (b < cnt) ? __ldg(A.v + j0 + b) * ex2_approx(-xb * xb) : 0.f;
      P = make_float4(xa, xb, va, vb);
      V = f2(va * xa, vb * xb);
      Gp = f2(va * xa * xa, vb * xb * xb);
      return;
    }
    P = make_float4(-xa, -xb, 0.f, 0.f);
  } else {
    const float2 pa = (a < cnt) ? __ldg(A.src.xy + j0 + a) : f2(0.f, 0.f);
    const float2 pb = (b < cnt) ? __ldg(A.src.xy + j0 + b) : f2(0.f, 0.f);
    P = make_float4(-pa.x, -pb.x, -pa.y, -pb.y);
  }
  V = f2((a < cnt) ? __ldg(A.v + j0 + a) : 0.f, (b < cnt) ? __ldg(A.v + j0 + b) : 0.f);
  if (SELF) Gp = f2((a < cnt) ? __ldg(A.gs + j0 + a) : 0.f, (b < cnt) ? __ldg(A.gs + j0 + b) : 0.f);
}

template <int R, int K>
struct BwSmem {
  union {
    struct {
      float4 sP[2][kBwPairs];
      float2 sV[2][kBwPairs];
      float2 sG[2][kBwPairs];
    };
    // the training forward's pair records: pair p at 2p (x'_a, x'_b, v~_a,
    // v~_b) and 2p + 1 (v~u_a, v~u_b, v~u^2_a, v~u^2_b), one address per pair
    float4 sT[2][2 * kBwPairs];
  };
  float dvred[kBwThreads / 32][kBwTile];  // fused d_v: per-warp sums of k g per source
  float ksum[R][K][kBwThreads];            // per-thread Kahan running sums (touched once per tile)
  float kcomp[R][K][kBwThreads];
};

template <bool GRID, bool SELF, bool DV>
struct BwCfg {
  static constexpr int R = DV ? kBwRdv : (GRID ? kBwRgrid : kBwR);
  static constexpr int K = SELF ? 7 : 4;
  static constexpr int ROWS = kBwThreads * R;
  using Smem = BwSmem<R, K>;
};

template <bool GRID, bool SELF, bool DV, bool SPLIT>
__device__ __forceinline__ void bwd_rows_body(const BwArgs& A, int rb, int chunk,
                                              typename BwCfg<GRID, SELF, DV>::Smem& sm) {
  constexpr int kBwR = BwCfg<GRID, SELF, DV>::R;
  constexpr int kBwRows = BwCfg<GRID, SELF, DV>::ROWS;
  constexpr int K = BwCfg<GRID, SELF, DV>::K;
  float4 (*sP)[kBwPairs] = sm.sP;
  float2 (*sV)[kBwPairs] = sm.sV;
  float2 (*sG)[kBwPairs] = sm.sG;
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

  float2 xq[kBwR], yq[kBwR], gq[kBwR];
  float2 acc[kBwR][K];
#pragma unroll
  for (int r = 0; r < kBwR; ++r) {
    const int64_t ir = map_row(A.map, A.n, kBwRows, rb, r * kBwThreads + tid);
    const int64_t i = ir >= 0 ? ir : 0;  // padding rows compute on row 0 and are not written
    const float2 p = __ldg(A.x + i);
    xq[r] = f2(p.x, p.x);
    yq[r] = f2(p.y, p.y);
    {
      // padding rows carry g = 0 so that they add nothing to the fused d_v
      const float gv = (DV && ir >= 0) ? __ldg(A.grow + ir) : 0.f;
      gq[r] = f2(gv, gv);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      acc[r][k] = f2(0.f, 0.f);
      sm.ksum[r][k][tid] = 0.f;
      sm.kcomp[r][k][tid] = 0.f;
    }
  }
  const float2 nc2 = f2(A.neg_c, A.neg_c);

  float4 P;
  float2 V, Gp = f2(0.f, 0.f);
  if (t0 < t1) {
    bw_load_pair<GRID, SELF, SPLIT>(A, t0, tid, P, V, Gp);
    sP[0][tid] = P;
    sV[0][tid] = V;
    if (SELF || SPLIT) sG[0][tid] = Gp;
  }
  __syncthreads();

  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    if (t + 1 < t1) bw_load_pair<GRID, SELF, SPLIT>(A, t + 1, tid, P, V, Gp);
    int64_t j0;
    int cnt, grow;
    bw_tile_range(A.src, t, j0, cnt, grow);
    const int np = (cnt + 1) >> 1;
    float dyr[kBwR];
    if (GRID) {
      // t = sc^2 d^2 = dx'^2 + dy'^2 in scaled tile-local coordinates, k = 2^-t;
      // B accumulates k v dx' (= sc k v dx) and C accumulates k v t (= c k v d^2)
      const float yt = grid_y(A.src.g, grow);
      const int c0 = (int)(j0 - (int64_t)grow * A.src.g.W);
      float2 dy2[kBwR];
#pragma unroll
      for (int r = 0; r < kBwR; ++r) {
        dyr[r] = yq[r].x - yt;
        const float d = A.sc * dyr[r];
        dy2[r] = f2(d * d, d * d);
      }
      constexpr bool fuse_dv = DV;
      const int nsg = (cnt + kBwSeg - 1) / kBwSeg;
      // columns of this grid row within reach of the row block (all without
      // info), and the sub-segments that meet them
      int clo = 0, chi = cnt - 1;
      if (A.info) reach_cols(B, A.src.g, yt, A.sc, c0, cnt, clo, chi);
      const int sg_lo = clo <= chi ? clo / kBwSeg : nsg, sg_hi = clo <= chi ? chi / kBwSeg : -1;
      if (SPLIT) {
      for (int sg = sg_lo; sg <= sg_hi; ++sg) {
        int pl, ph;
        seg_pair_range<kBwSeg>(clo, chi, kBwSeg * sg, pl, ph);
        if (pl >= ph) {
          // every pair's exp2 flushes to 0: nothing to add, zero column sums
          if (fuse_dv && (tid & 31) < kBwSeg) sm.dvred[tid >> 5][sg * kBwSeg + (tid & 31)] = 0.f;
          continue;
        }
        // Split exponent (see the forward pass): k v = 2^(2 q x' + a_i) v~.
        // Per pair one packed FMA forms the exponent and three accumulate the
        // x' moments S0 = sum k~ v~, S1 = sum k~ v~ x', S2 = sum k~ v~ x'^2 of
        // the sub-segment, from which, with dx' = q - x',
        //   sum k v = S0, sum k v dx' = q S0 - S1,
        //   sum k v (dx'^2 + dy'^2) = (q^2 + dy'^2) S0 - 2 q S1 + S2;
        // the fused d_v sums k~ g and scales by 2^-x'^2 per source at the end.
        const float o = grid_x(A.src.g, c0 + kBwSeg * sg + kBwSeg / 2);
        float2 q2[kBwR], ar[kBwR], S0[kBwR], S1[kBwR], S2[kBwR];
#pragma unroll
        for (int r = 0; r < kBwR; ++r) {
          const float q = A.sc * (xq[r].x - o);
          const float a = -fmaf(q, q, dy2[r].x);
          q2[r] = f2(2.f * q, 2.f * q);
          ar[r] = f2(a, a);
          S0[r] = S1[r] = S2[r] = f2(0.f, 0.f);
        }
        float kgs[kBwSeg];
#pragma unroll
        for (int qq = 0; qq < kBwSeg / 2; qq += kQuarterPairs) {
          if (qq < pl || qq >= ph) {  // a quarter out of reach: exactly zero
#pragma unroll
            for (int c = 2 * qq; c < 2 * (qq + kQuarterPairs); ++c) kgs[c] = 0.f;
            continue;
          }
#pragma unroll
          for (int pp = qq; pp < qq + kQuarterPairs; ++pp) {
            const int p = sg * (kBwSeg / 2) + pp;
            const float4 Q = sP[buf][p];
            const float2 X = f2(Q.x, Q.y), W0 = f2(Q.z, Q.w);
            const float2 W1 = sV[buf][p], W2 = sG[buf][p];
            float2 kg = f2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < kBwR; ++r) {
              const float2 e = __ffma2_rn(q2[r], X, ar[r]);
              const float2 k = f2(ex2_approx(e.x), ex2_approx(e.y));
              S0[r] = __ffma2_rn(k, W0, S0[r]);
              S1[r] = __ffma2_rn(k, W1, S1[r]);
              S2[r] = __ffma2_rn(k, W2, S2[r]);
              if (fuse_dv) kg = __ffma2_rn(k, gq[r], kg);
            }
            kgs[2 * pp] = kg.x;
            kgs[2 * pp + 1] = kg.y;
          }
        }
#pragma unroll
        for (int r = 0; r < kBwR; ++r) {
          const float q = 0.5f * q2[r].x;
          const float s0 = S0[r].x + S0[r].y, s1 = S1[r].x + S1[r].y, s2 = S2[r].x + S2[r].y;
          acc[r][0].x += s0;
          acc[r][1].x += fmaf(q, s0, -s1);
          acc[r][3].x += fmaf(fmaf(q, q, dy2[r].x), s0, fmaf(-2.f * q, s1, s2));
        }
        if (fuse_dv) warp_reduce_scatter(kgs, tid & 31, &sm.dvred[tid >> 5][sg * kBwSeg]);
      }
      } else {
      for (int sg = sg_lo; sg <= sg_hi; ++sg) {
        int pl, ph;
        seg_pair_range<kBwSeg>(clo, chi, kBwSeg * sg, pl, ph);
        if (pl >= ph) {
          if (fuse_dv && (tid & 31) < kBwSeg) sm.dvred[tid >> 5][sg * kBwSeg + (tid & 31)] = 0.f;
          continue;
        }
        const float o = grid_x(A.src.g, c0 + kBwSeg * sg + kBwSeg / 2);
        float2 qx[kBwR];
#pragma unroll
        for (int r = 0; r < kBwR; ++r) {
          const float q = A.sc * (xq[r].x - o);
          qx[r] = f2(q, q);
        }
        float kgs[kBwSeg];  // fused d_v: per-thread sums of k g over its rows, per source of the sub-segment
#pragma unroll
        for (int qq = 0; qq < kBwSeg / 2; qq += kQuarterPairs) {
          if (qq < pl || qq >= ph) {  // a quarter out of reach: exactly zero
#pragma unroll
            for (int c = 2 * qq; c < 2 * (qq + kQuarterPairs); ++c) kgs[c] = 0.f;
            continue;
          }
#pragma unroll
          for (int pp = qq; pp < qq + kQuarterPairs; ++pp) {
            const int p = sg * (kBwSeg / 2) + pp;
            const float4 Q = sP[buf][p];
            const float2 W = sV[buf][p];
            const float2 nx = f2(Q.x, Q.y);
            float2 kg = f2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < kBwR; ++r) {
              const float2 dx = __fadd2_rn(qx[r], nx);
              const float2 t = __ffma2_rn(dx, dx, dy2[r]);
              const float2 k = f2(ex2_approx(-t.x), ex2_approx(-t.y));
              const float2 kv = __fmul2_rn(k, W);
              acc[r][0] = __fadd2_rn(acc[r][0], kv);
              acc[r][1] = __ffma2_rn(kv, dx, acc[r][1]);
              acc[r][3] = __ffma2_rn(kv, t, acc[r][3]);
              if (fuse_dv) kg = __ffma2_rn(k, gq[r], kg);
            }
            kgs[2 * pp] = kg.x;
            kgs[2 * pp + 1] = kg.y;
          }
        }
        if (fuse_dv) warp_reduce_scatter(kgs, tid & 31, &sm.dvred[tid >> 5][sg * kBwSeg]);
      }
      }
      if (fuse_dv) {
        __syncthreads();
        // combine the warps in order; row block rb owns these columns of
        // dv_part (exact zeros outside the sub-segments in reach)
        float* dst = A.dv_part + (int64_t)rb * A.src.m + j0;
        for (int j = tid; j < cnt; j += kBwThreads) {
          if (j < sg_lo * kBwSeg || j >= (sg_hi + 1) * kBwSeg) {
            dst[j] = 0.f;
            continue;
          }
          float sdv = sm.dvred[0][j];
#pragma unroll
          for (int w = 1; w < kBwThreads / 32; ++w) sdv += sm.dvred[w][j];
          if (SPLIT) {
            const float4 Q = sP[buf][j >> 1];
            const float xj = (j & 1) ? Q.y : Q.x;
            sdv *= ex2_approx(-xj * xj);
          }
          dst[j] = sdv;
        }
      }
    } else {
#pragma unroll 2
      for (int p = 0; p < np; ++p) {
        const float4 Q = sP[buf][p];
        const float2 W = sV[buf][p];
        const float2 nx = f2(Q.x, Q.y), ny = f2(Q.z, Q.w);
        float2 Gq;
        if (SELF) Gq = sG[buf][p];
#pragma unroll
        for (int r = 0; r < kBwR; ++r) {
          const float2 dx = __fadd2_rn(xq[r], nx);
          const float2 dy = __fadd2_rn(yq[r], ny);
          const float2 e = __fmul2_rn(__ffma2_rn(dy, dy, __fmul2_rn(dx, dx)), nc2);
          const float2 k = f2(ex2_approx(e.x), ex2_approx(e.y));
          const float2 kv = __fmul2_rn(k, W);
          acc[r][0] = __fadd2_rn(acc[r][0], kv);
          acc[r][1] = __ffma2_rn(kv, dx, acc[r][1]);
          acc[r][2] = __ffma2_rn(kv, dy, acc[r][2]);
          acc[r][3] = __ffma2_rn(kv, e, acc[r][3]);
          if (SELF) {
            const float2 kg = __fmul2_rn(k, Gq);
            acc[r][4] = __fadd2_rn(acc[r][4], kg);
            acc[r][5] = __ffma2_rn(kg, dx, acc[r][5]);
            acc[r][6] = __ffma2_rn(kg, dy, acc[r][6]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kBwR; ++r) {
      if (GRID) acc[r][2] = f2(dyr[r] * acc[r][0].x, dyr[r] * acc[r][0].y);  // uniform y on a grid row
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float su = sm.ksum[r][k][tid], co = sm.kcomp[r][k][tid];
        kahan(su, co, acc[r][k].x + acc[r][k].y);
        sm.ksum[r][k][tid] = su;
        sm.kcomp[r][k][tid] = co;
        acc[r][k] = f2(0.f, 0.f);
      }
    }
    if (t + 1 < t1) {
      sP[buf ^ 1][tid] = P;
      sV[buf ^ 1][tid] = V;
      if (SELF || SPLIT) sG[buf ^ 1][tid] = Gp;
    }
    __syncthreads();
  }

#pragma unroll
  for (int r = 0; r < kBwR; ++r) {
    const int64_t i = map_row(A.map, A.n, kBwRows, rb, r * kBwThreads + tid);
    if (i >= 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) A.partial[((int64_t)chunk * K + k) * A.n + i] = sm.ksum[r][k][tid] - sm.kcomp[r][k][tid];
    }
  }
}

// ---------------------------------------------------------------------------
// Row pass for grid sources with the split exponent and no fused d_v (the
// training forward, and the backward's row gradients without d_v): the row
// sums A, B_x, B_y, C of row block rb over one chunk of its active tiles.
//
// Moments about the row block's centre: with x_c the centre of the block's
// box, q0 = sc (x_i - x_c) per row and, for a source of sub-segment s,
// u = sc (x_j - x_c) = x' + delta_s (delta_s = sc (o_s - x_c)), a pair's
// dx' = q0 - u. So over a whole tile
//   A = S0, B_x = q0 S0 - S1, B_y = dy S0, C = (q0^2 + dy'^2) S0 - 2 q0 S1 + S2
// with S0 = sum k~ v~, S1 = sum k~ v~ u, S2 = sum k~ v~ u^2. The exponent
// keeps the sub-segment form 2 q_s x' + a_s (q_s = q0 - delta_s,
// a_s = -(q_s^2 + dy'^2), |x'| <= 5.5), so every sub-segment adds into the
// same packed sums and the conversion to A, B, C runs once per row and tile.
// The per-tile sums are added plainly for kTrainFold tiles, then folded into
// Kahan sums kept in shared memory.
//
// The form needs a compact row block: q0 and u stay small only when the
// block's box is narrow (image-tile row order). A wider box (rows in index
// order of scattered points) takes the per-sub-segment form (bwd_rows_body),
// whose exponent and moments are all relative to the sub-segment centre.
constexpr int kTrainFold = 16;
constexpr float kTrainCompact = 8.f;  // widest box, in scaled units sc x width

__device__ __forceinline__ bool train_compact(const BwArgs& A, int rb) {
  if (!A.info) return false;
  const RowBlockInfo& B = A.info[rb];
  return !(B.xlo <= B.xhi) || (B.xhi - B.xlo) * A.sc <= kTrainCompact;
}

// A tile of a grid-source sweep (the training forward and the d_v sweep):
// grid row `grow`, columns c0 .. c0 + cnt - 1,
// the columns [clo, chi] within reach of the row block (empty: clo > chi),
// and cs, the tile-local column where the tile's records start: clo rounded
// down to a quarter (4 columns). The sub-segments are laid from cs on, so
// all but the last one in reach are whole.
struct GridTile {
  int grow, c0, cnt, clo, chi, cs;
  float yt;
};

__device__ __forceinline__ GridTile grid_tile(const BwArgs& A, const RowBlockInfo& B, int grow, int seg,
                                              float inv_sc, float inv_h) {
  GridTile T;
  T.grow = grow;
  T.c0 = seg * kBwTile;
  T.cnt = min(kBwTile, A.src.g.W - T.c0);
  T.yt = grid_y(A.src.g, grow);
  T.clo = 0;
  T.chi = T.cnt - 1;
  if (A.info) reach_cols_fast(B, A.src.g, T.yt, A.sc, inv_sc, inv_h, T.c0, T.cnt, T.clo, T.chi);
  T.cs = T.clo <= T.chi ? (T.clo & ~(2 * kQuarterPairs - 1)) : 0;
  return T;
}

// What the sweep of a tile needs: its quarters in reach from cs on (every
// column outside is exactly zero), the grid column of cs, and the row's y.
struct TileRun {
  int nq, ccs;
  float yt;
};

__device__ __forceinline__ TileRun tile_run(const GridTile& T) {
  return TileRun{T.clo <= T.chi ? (T.chi - T.cs) / (2 * kQuarterPairs) + 1 : 0, T.c0 + T.cs, T.yt};
}

// Pair p of tile T's records: columns cs + 2p and cs + 2p + 1 (zero past the
// row's end), x' about the centre of their sub-segment.
__device__ __forceinline__ void train_load_pair(const BwArgs& A, const GridTile& T, int p, float xc, float4& P,
                                                float4& VG) {
  const int64_t j0 = (int64_t)T.grow * A.src.g.W + T.c0 + T.cs;
  const int a = 2 * p, b = 2 * p + 1;
  const int c = T.c0 + T.cs;
  const float o = grid_x(A.src.g, c + kBwSeg * (a / kBwSeg) + kBwSeg / 2);
  const float gxa = grid_x(A.src.g, c + a), gxb = grid_x(A.src.g, c + b);
  const bool ina = T.cs + a < T.cnt, inb = T.cs + b < T.cnt;
  const float xa = ina ? A.sc * (gxa - o) : 0.f;
  const float xb = inb ? A.sc * (gxb - o) : 0.f;
  const float va = ina ? __ldg(A.v + j0 + a) * ex2_approx(-xa * xa) : 0.f;
  const float vb = inb ? __ldg(A.v + j0 + b) * ex2_approx(-xb * xb) : 0.f;
  const float ua = A.sc * (gxa - xc), ub = A.sc * (gxb - xc);
  P = make_float4(xa, xb, va, vb);
  VG = make_float4(va * ua, vb * ub, va * ua * ua, vb * ub * ub);
}

// NP consecutive source pairs (records T[0 .. 2 NP)) against the thread's R
// rows: exponent, exp2 and the three packed moment sums.
template <int R, int NP>
__device__ __forceinline__ void train_pairs(const float4* __restrict__ T, const float2 (&q2)[R],
                                            const float2 (&ar)[R], float2 (&S0)[R], float2 (&S1)[R],
                                            float2 (&S2)[R]) {
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) {
    const float4 Q = T[2 * pp], U = T[2 * pp + 1];
    const float2 X = f2(Q.x, Q.y), W0 = f2(Q.z, Q.w);
    const float2 W1 = f2(U.x, U.y), W2 = f2(U.z, U.w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float2 e = __ffma2_rn(q2[r], X, ar[r]);
      const float2 k = f2(ex2_approx(e.x), ex2_approx(e.y));
      S0[r] = __ffma2_rn(k, W0, S0[r]);
      S1[r] = __ffma2_rn(k, W1, S1[r]);
      S2[r] = __ffma2_rn(k, W2, S2[r]);
    }
  }
}

template <int R>
__device__ __forceinline__ void train_rows_body(const BwArgs& A, int rb, int chunk, BwSmem<R, 4>& sm) {
  constexpr int kRows = kBwThreads * R;
  RowBlockInfo B{};
  int lo = 0, hi = A.src.n_tiles;
  float xc = 0.f;
  if (A.info) {
    B = A.info[rb];
    lo = B.t_lo;
    hi = B.t_hi > B.t_lo ? B.t_hi : B.t_lo;
    if (B.xlo <= B.xhi) xc = 0.5f * (B.xlo + B.xhi);
  }
  const int t0 = lo + (int)((int64_t)chunk * (hi - lo) / A.chunks);
  const int t1 = lo + (int)((int64_t)(chunk + 1) * (hi - lo) / A.chunks);
  const int tid = threadIdx.x;
  const float inv_sc = 1.0f / A.sc, inv_h = 1.0f / A.src.g.h;

  float yq[R], q0[R];
  float acc[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t ir = map_row(A.map, A.n, kRows, rb, r * kBwThreads + tid);
    const float2 p = __ldg(A.x + (ir >= 0 ? ir : 0));  // padding rows compute on row 0 and are not written
    yq[r] = p.y;
    q0[r] = A.sc * (p.x - xc);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[r][k] = 0.f;
      sm.ksum[r][k][tid] = 0.f;
      sm.kcomp[r][k][tid] = 0.f;
    }
  }

  // tile t = grow * segs + seg, stepped without a division per tile; each
  // tile's reach is found one tile ahead, with its records
  const int segs = A.src.segs;
  int grow = t0 / segs, seg = t0 - grow * segs;
  TileRun run{0, 0, 0.f};
  float4 P, VG;
  if (t0 < t1) {
    const GridTile T = grid_tile(A, B, grow, seg, inv_sc, inv_h);
    run = tile_run(T);
    train_load_pair(A, T, tid, xc, P, VG);
    sm.sT[0][2 * tid] = P;
    sm.sT[0][2 * tid + 1] = VG;
  }
  __syncthreads();

  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    const bool wrap = seg + 1 == segs;
    grow = wrap ? grow + 1 : grow;
    seg = wrap ? 0 : seg + 1;
    TileRun next{0, 0, 0.f};
    if (t + 1 < t1) {
      const GridTile T = grid_tile(A, B, grow, seg, inv_sc, inv_h);
      next = tile_run(T);
      train_load_pair(A, T, tid, xc, P, VG);
    }
    const float yt = run.yt;
    float dyr[R], ndy2[R];
    float2 S0[R], S1[R], S2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      dyr[r] = yq[r] - yt;
      const float d = A.sc * dyr[r];
      ndy2[r] = -d * d;
      S0[r] = S1[r] = S2[r] = f2(0.f, 0.f);
    }
    // sub-segments of 4 quarters from cs on: all whole but the last
    const int nsg = (run.nq + 3) / 4;
    for (int sg = 0; sg < nsg; ++sg) {
      const int qn = min(4, run.nq - 4 * sg);
      const float ds = A.sc * (grid_x(A.src.g, run.ccs + kBwSeg * sg + kBwSeg / 2) - xc);  // delta_s
      float2 q2[R], ar[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float q = q0[r] - ds;
        const float a = fmaf(-q, q, ndy2[r]);
        q2[r] = f2(q + q, q + q);
        ar[r] = f2(a, a);
      }
      const float4* rec = &sm.sT[buf][2 * sg * (kBwSeg / 2)];
      if (qn == 4) {
        // a whole sub-segment: one block without quarter tests
        train_pairs<R, kBwSeg / 2>(rec, q2, ar, S0, S1, S2);
      } else {
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) {
          if (qq >= qn) break;  // the quarters past the reach: exactly zero
          train_pairs<R, kQuarterPairs>(rec + 4 * qq, q2, ar, S0, S1, S2);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float s0 = S0[r].x + S0[r].y, s1 = S1[r].x + S1[r].y, s2 = S2[r].x + S2[r].y;
      acc[r][0] += s0;
      acc[r][1] += fmaf(q0[r], s0, -s1);
      acc[r][2] = fmaf(dyr[r], s0, acc[r][2]);
      acc[r][3] += fmaf(fmaf(q0[r], q0[r], -ndy2[r]), s0, fmaf(-2.f * q0[r], s1, s2));
    }
    if ((t - t0) % kTrainFold == kTrainFold - 1 || t + 1 == t1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float su = sm.ksum[r][k][tid], co = sm.kcomp[r][k][tid];
          kahan(su, co, acc[r][k]);
          sm.ksum[r][k][tid] = su;
          sm.kcomp[r][k][tid] = co;
          acc[r][k] = 0.f;
        }
      }
    }
    if (t + 1 < t1) {
      sm.sT[buf ^ 1][2 * tid] = P;
      sm.sT[buf ^ 1][2 * tid + 1] = VG;
    }
    run = next;
    __syncthreads();
  }

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = map_row(A.map, A.n, kRows, rb, r * kBwThreads + tid);
    if (i >= 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) A.partial[((int64_t)chunk * 4 + k) * A.n + i] = sm.ksum[r][k][tid] - sm.kcomp[r][k][tid];
    }
  }
}

// Resident CTAs per SM the compiler must leave room for: the training
// forward's row pass ran fastest at 4 (128 registers; 5 and 6 ran slower).
template <bool GRID, bool SELF, bool DV, bool SPLIT>
constexpr int bw_min_blocks() {
  return (GRID && !SELF && !DV && SPLIT) ? 4 : 1;
}

template <bool GRID, bool SELF, bool DV, bool SPLIT = false>
__global__ void __launch_bounds__(kBwThreads, (bw_min_blocks<GRID, SELF, DV, SPLIT>())) bwd_rows_kernel(const __grid_constant__ BwArgs A) {
  __shared__ __align__(16) typename BwCfg<GRID, SELF, DV>::Smem sm;
  const int rb = blockIdx.x / A.chunks;
  if constexpr (GRID && !SELF && !DV && SPLIT) {
    if (train_compact(A, rb)) {
      train_rows_body<BwCfg<GRID, SELF, DV>::R>(A, rb, blockIdx.x - rb * A.chunks, sm);
      return;
    }
  }
  bwd_rows_body<GRID, SELF, DV, SPLIT>(A, rb, blockIdx.x - rb * A.chunks, sm);
}

// Batched form; every problem of one launch has the same kind (grid with or
// without the split exponent and fused d_v, explicit, explicit self-kernel).
template <bool GRID, bool SELF, bool DV, bool SPLIT = false>
__global__ void __launch_bounds__(kBwThreads, (bw_min_blocks<GRID, SELF, DV, SPLIT>()))
    bwd_rows_batched_kernel(const __grid_constant__ Batch<BwArgs> B) {
  __shared__ __align__(16) typename BwCfg<GRID, SELF, DV>::Smem sm;
  const int k = batch_find(B, blockIdx.x);
  const BwArgs& A = B.p[k];
  const int local = blockIdx.x - B.start[k];
  const int rb = local / A.chunks;
  if constexpr (GRID && !SELF && !DV && SPLIT) {
    if (train_compact(A, rb)) {
      train_rows_body<BwCfg<GRID, SELF, DV>::R>(A, rb, local - rb * A.chunks, sm);
      return;
    }
  }
  bwd_rows_body<GRID, SELF, DV, SPLIT>(A, rb, local - rb * A.chunks, sm);
}

// ---------------------------------------------------------------------------
// d_v alone for grid sources: dv_part[rb][j] = sum over the rows i of row
// block rb of k_ij g_i. This is the column half of the backward pass when the
// row sums (A, B, C) come from the training forward (gp_kernel_matvec_train),
// so per pair only the exponent, one exp2 and one accumulation remain:
// 2 FP32 lanes with the split exponent (k = k~ 2^-x'^2, the per-source
// factor applied once per tile), 3 without.
constexpr int kDvR = 8;
constexpr int kDvRows = kBwThreads * kDvR;

struct DvSmem {
  float2 sX[2][kBwPairs];
  float dvred[kBwThreads / 32][kBwTile];
};

// Pair p of tile T's records (see GridTile): columns cs + 2p and cs + 2p + 1.
template <bool SPLIT>
__device__ __forceinline__ void dv_load_pair(const BwArgs& A, const GridTile& T, int p, float2& X) {
  const int c = T.c0 + T.cs;
  const int a = 2 * p, b = 2 * p + 1;
  const float o = grid_x(A.src.g, c + kBwSeg * (a / kBwSeg) + kBwSeg / 2);
  const float xa = (T.cs + a < T.cnt) ? A.sc * (grid_x(A.src.g, c + a) - o) : 0.f;
  const float xb = (T.cs + b < T.cnt) ? A.sc * (grid_x(A.src.g, c + b) - o) : 0.f;
  X = SPLIT ? f2(-2.f * xa, -2.f * xb) : f2(-xa, -xb);
}

// What the d_v sweep of a tile needs (see GridTile and TileRun).
struct DvRun {
  int nq, cs, c0, cnt;
  int64_t j0;
  float yt;
};

__device__ __forceinline__ DvRun dv_run(const BwArgs& A, const GridTile& T) {
  return DvRun{T.clo <= T.chi ? (T.chi - T.cs) / (2 * kQuarterPairs) + 1 : 0, T.cs, T.c0, T.cnt,
               (int64_t)T.grow * A.src.g.W + T.c0, T.yt};
}

// NP consecutive source pairs (records X[0 .. NP)) against the thread's rows:
// kgs[2p], kgs[2p + 1] = sum over the rows of k g for the pair's two sources.
template <bool SPLIT, int NP>
__device__ __forceinline__ void dv_pairs(const float2* __restrict__ X, const float2 (&qa)[kDvR],
                                         const float2 (&qb)[kDvR], const float2 (&gq)[kDvR], float* kgs) {
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) {
    const float2 Xp = X[pp];
    float2 kg = f2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kDvR; ++r) {
      float2 k;
      if (SPLIT) {
        const float2 e = __ffma2_rn(qa[r], Xp, qb[r]);
        k = f2(ex2_approx(e.x), ex2_approx(e.y));
      } else {
        const float2 dx = __fadd2_rn(qa[r], Xp);
        const float2 tt = __ffma2_rn(dx, dx, qb[r]);
        k = f2(ex2_approx(-tt.x), ex2_approx(-tt.y));
      }
      kg = __ffma2_rn(k, gq[r], kg);
    }
    kgs[2 * pp] = kg.x;
    kgs[2 * pp + 1] = kg.y;
  }
}

// All kBwSeg / 2 pairs of a sub-segment in the lane-permuted order that
// warp_reduce_scatter_perm expects: slot pp of lane l takes pair
// pp ^ ((l >> 2) & 7) (eight distinct records of one 64-byte block across
// the warp: no bank conflict).
template <bool SPLIT>
__device__ __forceinline__ void dv_pairs_perm(const float2* __restrict__ X, const float2 (&qa)[kDvR],
                                              const float2 (&qb)[kDvR], const float2 (&gq)[kDvR],
                                              float (&kgs)[kBwSeg], int lane) {
  static_assert(kBwSeg == 16, "the permutation spans the 8 pairs of a 16-column sub-segment");
  const int kp = (lane >> 2) & 7;
#pragma unroll
  for (int pp = 0; pp < kBwSeg / 2; ++pp) dv_pairs<SPLIT, 1>(X + (pp ^ kp), qa, qb, gq, kgs + 2 * pp);
}

template <bool SPLIT>
__device__ __forceinline__ void dv_rows_body(const BwArgs& A, int rb, int chunk, DvSmem& sm) {
  RowBlockInfo B{};
  int lo = 0, hi = A.src.n_tiles;
  if (A.info) {
    B = A.info[rb];
    lo = B.t_lo;
    hi = B.t_hi > B.t_lo ? B.t_hi : B.t_lo;
  }
  const int t0 = lo + (int)((int64_t)chunk * (hi - lo) / A.chunks);
  const int t1 = lo + (int)((int64_t)(chunk + 1) * (hi - lo) / A.chunks);
  const int tid = threadIdx.x;
  const float inv_sc = 1.0f / A.sc, inv_h = 1.0f / A.src.g.h;
  float xq[kDvR], yq[kDvR];
  float2 gq[kDvR];
#pragma unroll
  for (int r = 0; r < kDvR; ++r) {
    const int64_t ir = map_row(A.map, A.n, kDvRows, rb, r * kBwThreads + tid);
    const int64_t i = ir >= 0 ? ir : 0;
    const float2 p = __ldg(A.x + i);
    xq[r] = p.x;
    yq[r] = p.y;
    const float gv = ir >= 0 ? __ldg(A.grow + ir) : 0.f;  // padding rows add nothing
    gq[r] = f2(gv, gv);
  }
  // tile t = grow * segs + seg, stepped without a division per tile; each
  // tile's reach is found one tile ahead, with its records, and its
  // sub-segments are laid from cs on (all whole but the last)
  const int segs = A.src.segs;
  int grow = t0 / segs, seg = t0 - grow * segs;
  DvRun run{0, 0, 0, 0, 0, 0.f};
  float2 X = f2(0.f, 0.f);
  if (t0 < t1) {
    const GridTile T = grid_tile(A, B, grow, seg, inv_sc, inv_h);
    run = dv_run(A, T);
    dv_load_pair<SPLIT>(A, T, tid, X);
    sm.sX[0][tid] = X;
  }
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    const bool wrap = seg + 1 == segs;
    grow = wrap ? grow + 1 : grow;
    seg = wrap ? 0 : seg + 1;
    DvRun next{0, 0, 0, 0, 0, 0.f};
    if (t + 1 < t1) {
      const GridTile T = grid_tile(A, B, grow, seg, inv_sc, inv_h);
      next = dv_run(A, T);
      dv_load_pair<SPLIT>(A, T, tid, X);
    }
    float dy2[kDvR];
#pragma unroll
    for (int r = 0; r < kDvR; ++r) {
      const float d = A.sc * (yq[r] - run.yt);
      dy2[r] = d * d;
    }
    const int nsg = (run.nq + 3) / 4;
    for (int sg = 0; sg < nsg; ++sg) {
      const int qn = min(4, run.nq - 4 * sg);
      const float o = grid_x(A.src.g, run.c0 + run.cs + kBwSeg * sg + kBwSeg / 2);
      // split: (-q, -(q^2 + dy'^2)) against records -2x'; unsplit: (q, dy'^2)
      float2 qa[kDvR], qb[kDvR];
#pragma unroll
      for (int r = 0; r < kDvR; ++r) {
        if (SPLIT) {
          const float nq = A.sc * (o - xq[r]);
          const float a = -fmaf(nq, nq, dy2[r]);
          qa[r] = f2(nq, nq);
          qb[r] = f2(a, a);
        } else {
          const float q = A.sc * (xq[r] - o);
          qa[r] = f2(q, q);
          qb[r] = f2(dy2[r], dy2[r]);
        }
      }
      float kgs[kBwSeg];
      const float2* Xs = &sm.sX[buf][sg * (kBwSeg / 2)];
      if (qn == 4) {
        // a whole sub-segment: one block without quarter tests, in the
        // lane-permuted order
        dv_pairs_perm<SPLIT>(Xs, qa, qb, gq, kgs, tid & 31);
        warp_reduce_scatter_perm(kgs, tid & 31, &sm.dvred[tid >> 5][sg * kBwSeg]);
      } else {
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
          if (qi >= qn) {  // a quarter past the reach: exactly zero
#pragma unroll
            for (int c = 4 * qi; c < 4 * qi + 4; ++c) kgs[c] = 0.f;
            continue;
          }
          dv_pairs<SPLIT, kQuarterPairs>(Xs + 2 * qi, qa, qb, gq, kgs + 4 * qi);
        }
        warp_reduce_scatter(kgs, tid & 31, &sm.dvred[tid >> 5][sg * kBwSeg]);
      }
    }
    __syncthreads();
    // combine the warps in order; row block rb owns these columns of
    // dv_part (exact zeros outside the sub-segments in reach)
    float* dst = A.dv_part + (int64_t)rb * A.src.m + run.j0;
    for (int j = tid; j < run.cnt; j += kBwThreads) {
      const int jj = j - run.cs;
      if (jj < 0 || jj >= nsg * kBwSeg) {
        dst[j] = 0.f;
        continue;
      }
      float sdv = sm.dvred[0][jj];
#pragma unroll
      for (int w = 1; w < kBwThreads / 32; ++w) sdv += sm.dvred[w][jj];
      if (SPLIT) {
        const float2 Xp = sm.sX[buf][jj >> 1];
        const float xj = 0.5f * ((jj & 1) ? Xp.y : Xp.x);  // the record holds -2x'
        sdv *= ex2_approx(-xj * xj);
      }
      dst[j] = sdv;
    }
    if (t + 1 < t1) sm.sX[buf ^ 1][tid] = X;
    run = next;
    __syncthreads();
  }
}

template <bool SPLIT>
__global__ void __launch_bounds__(kBwThreads, 5) dv_rows_kernel(const __grid_constant__ BwArgs A) {
  __shared__ __align__(16) DvSmem sm;
  const int rb = blockIdx.x / A.chunks;
  dv_rows_body<SPLIT>(A, rb, blockIdx.x - rb * A.chunks, sm);
}

template <bool SPLIT>
__global__ void __launch_bounds__(kBwThreads, 5) dv_rows_batched_kernel(const __grid_constant__ Batch<BwArgs> B) {
  __shared__ __align__(16) DvSmem sm;
  const int k = batch_find(B, blockIdx.x);
  const BwArgs& A = B.p[k];
  const int local = blockIdx.x - B.start[k];
  const int rb = local / A.chunks;
  dv_rows_body<SPLIT>(A, rb, local - rb * A.chunks, sm);
}

// Training forward: fixed-order merge of the row-pass chunk partials into the
// per-row moments (A, B_x, B_y, C) and out = var A.
__device__ __forceinline__ void moments_merge_body(const MomMergeP& P, int64_t i) {
  if (i >= P.n) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float s = 0.f, c = 0.f;
    for (int ch = 0; ch < P.chunks; ++ch) kahan(s, c, P.partial[((int64_t)ch * 4 + k) * P.n + i]);
    s -= c;
    P.mom[(int64_t)k * P.n + i] = s;
    if (k == 0) P.out[i] = P.var * s;
  }
}

__global__ void moments_merge_kernel(const __grid_constant__ MomMergeP P) {
  moments_merge_body(P, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void moments_merge_batched_kernel(const __grid_constant__ Batch<MomMergeP> B) {
  const int k = batch_find(B, blockIdx.x);
  moments_merge_body(B.p[k], (int64_t)(blockIdx.x - B.start[k]) * blockDim.x + threadIdx.x);
}

// Per-row merge of chunk partials, the per-row gradients, and per-block FP64
// partials of the two scalar gradients. The per-row products and the warp
// sums (a 32-term pairwise tree) stay in FP32; the warps' sums are added in
// FP64 (FP64 arithmetic runs at a small fraction of the FP32 rate).
__device__ __forceinline__ void bwd_merge_body(const MergeArgs& M, int64_t blk) {
  __shared__ float red[2][kMergeThreads / 32];
  const int64_t i = blk * kMergeThreads + threadIdx.x;
  float sl = 0.f, sv = 0.f;
  if (i < M.n) {
    float s[7], c[7];
    for (int k = 0; k < M.K; ++k) {
      s[k] = 0.f;
      c[k] = 0.f;
      for (int ch = 0; ch < M.chunks; ++ch) kahan(s[k], c[k], M.partial[((int64_t)ch * M.K + k) * M.n + i]);
      s[k] -= c[k];
    }
    const float gi = M.g[i];
    float ddx = gi * s[1] * M.b_scale, ddy = gi * s[2];
    if (M.K == 7) {
      const float vi = M.vrow[i];
      ddx = fmaf(vi, s[5], ddx);
      ddy = fmaf(vi, s[6], ddy);
      if (M.d_v) M.d_v[i] = M.var * s[4];
    }
    // sums were taken over (x_i - y_j); the gradient wants (y_j - x_i)
    if (M.d_x) M.d_x[i] = make_float2(-M.var * M.inv_l2 * ddx, -M.var * M.inv_l2 * ddy);
    sl = __fmul_rn(__fmul_rn(gi, s[3]), M.dl_scale);
    sv = __fmul_rn(gi, s[0]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = sl;
    red[1][w] = sv;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int k = 0; k < kMergeThreads / 32; ++k) t += (double)red[threadIdx.x][k];
    M.scal_part[blk * 2 + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kMergeThreads) bwd_merge_kernel(const __grid_constant__ MergeArgs M) {
  bwd_merge_body(M, blockIdx.x);
}

__global__ void __launch_bounds__(kMergeThreads) bwd_merge_batched_kernel(const __grid_constant__ Batch<MergeArgs> B) {
  const int k = batch_find(B, blockIdx.x);
  bwd_merge_body(B.p[k], blockIdx.x - B.start[k]);
}

// Fixed-order FP64 reduction of the per-block scalar partials: thread t sums
// blocks t, t + 256, ...; warps reduce by xor-shuffle; warp 0 adds the warps
// in order. One CTA of kMergeThreads threads.
__device__ __forceinline__ void scalar_final_body(const double* __restrict__ part, int nblk, double* d_len,
                                                  double* d_var) {
  __shared__ double red[2][kMergeThreads / 32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kMergeThreads) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < kMergeThreads / 32; ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    if (d_len) *d_len = sa;
    if (d_var) *d_var = sb;
  }
}

__global__ void __launch_bounds__(kMergeThreads) bwd_scalar_final_kernel(const double* __restrict__ part, int nblk,
                                                                         double* d_len, double* d_var) {
  scalar_final_body(part, nblk, d_len, d_var);
}

__global__ void __launch_bounds__(kMergeThreads) scalar_batched_kernel(const __grid_constant__ Batch<ScalP> B) {
  const ScalP& P = B.p[blockIdx.x];
  scalar_final_body(P.part, P.nblk, P.d_len, P.d_var);
}

// d_v merge: a CTA of kDvMergeCols x kDvMergeGroups threads takes
// kDvMergeCols consecutive sources of one source grid row (one tile). With
// row-block info a row block wrote this tile only when the tile is in its
// active range (elsewhere its sums are exactly 0 and are not read), so warp 0
// first lists the active row blocks in ascending order in shared memory
// (kDvMergeList at a time). Thread group y then sums list entries y,
// y + kDvMergeGroups, ... (Kahan, four loads in flight), and the groups' sums
// are added in group order: the result is deterministic.
constexpr int kDvMergeCols = 32, kDvMergeGroups = 8, kDvMergeList = 2048;

__device__ __forceinline__ void dv_merge_body(const DvMergeP& P, int64_t blk) {
  __shared__ float part[kDvMergeGroups][kDvMergeCols];
  __shared__ int list[kDvMergeList];
  __shared__ int count_sh;
  const int x = threadIdx.x % kDvMergeCols, y = threadIdx.x / kDvMergeCols;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cw = (P.W + kDvMergeCols - 1) / kDvMergeCols;  // column chunks per grid row
  const int64_t r = blk / cw;
  const int c = (int)(blk - r * cw) * kDvMergeCols + x;
  const bool valid = c < P.W;
  const int64_t j = r * P.W + c;
  const int t = (int)(r * P.segs + ((int64_t)(blk - r * cw) * kDvMergeCols) / kBwTile);
  float s = 0.f, cc = 0.f;
  for (int base = 0; base < P.row_blocks; base += kDvMergeList) {
    const int nb = min(kDvMergeList, P.row_blocks - base);
    if (warp == 0) {
      int count = 0;
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int rb = base + b0 + lane;
        bool act = b0 + lane < nb;
        if (act && P.info) {
          const int2 rr = *reinterpret_cast<const int2*>(&P.info[rb].t_lo);
          act = rr.x <= t && t < rr.y;
        }
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (act) list[count + __popc(m & ((1u << lane) - 1u))] = rb;
        count += __popc(m);
      }
      if (lane == 0) count_sh = count;
    }
    __syncthreads();
    const int count = count_sh;
    if (valid) {
      int i = y;
      for (; i + 3 * kDvMergeGroups < count; i += 4 * kDvMergeGroups) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = P.dv_part[(int64_t)list[i + k * kDvMergeGroups] * P.m + j];
#pragma unroll
        for (int k = 0; k < 4; ++k) kahan(s, cc, v[k]);
      }
      for (; i < count; i += kDvMergeGroups) kahan(s, cc, P.dv_part[(int64_t)list[i] * P.m + j]);
    }
    __syncthreads();  // the list is rewritten for the next window
  }
  part[y][x] = s - cc;
  __syncthreads();
  if (y == 0 && valid) {
    float a = 0.f, ca = 0.f;
#pragma unroll
    for (int k = 0; k < kDvMergeGroups; ++k) kahan(a, ca, part[k][x]);
    P.d_v[j] = P.var * (a - ca);
  }
}

// CTAs of the d_v merge: one per source grid row and kDvMergeCols columns.
inline int64_t dv_merge_blocks(const DvMergeP& P) {
  return P.W > 0 ? P.m / P.W * ((P.W + kDvMergeCols - 1) / kDvMergeCols) : 0;
}

__global__ void __launch_bounds__(kDvMergeCols * kDvMergeGroups) dv_merge_kernel(const __grid_constant__ DvMergeP P) {
  dv_merge_body(P, blockIdx.x);
}

__global__ void __launch_bounds__(kDvMergeCols * kDvMergeGroups)
    dv_merge_batched_kernel(const __grid_constant__ Batch<DvMergeP> B) {
  const int k = batch_find(B, blockIdx.x);
  dv_merge_body(B.p[k], blockIdx.x - B.start[k]);
}

lr_status launch_dv_merge_batched(const DvMergeP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<DvMergeP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += dv_merge_blocks(p[b0 + k]);
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    dv_merge_batched_kernel<<<(unsigned)tot, kDvMergeCols * kDvMergeGroups, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

lr_status launch_bwd_rows_batched(const BwArgs* p, int count, cudaStream_t s) {
  // kinds: 0 grid, 1 explicit, 2 explicit self-kernel, 3 grid + fused d_v,
  // 4 grid split, 5 grid split + fused d_v
  for (int kind = 0; kind < 6; ++kind) {
    Batch<BwArgs> B;
    B.count = 0;
    int64_t tot = 0;
    for (int i = 0; i <= count; ++i) {
      const bool flush = (i == count) || B.count == kMaxBatch;
      if (flush && B.count > 0) {
        B.start[B.count] = (int32_t)tot;
        if (tot > 0) {
          if (kind == 0)
            bwd_rows_batched_kernel<true, false, false><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          else if (kind == 1)
            bwd_rows_batched_kernel<false, false, false><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          else if (kind == 2)
            bwd_rows_batched_kernel<false, true, false><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          else if (kind == 3)
            bwd_rows_batched_kernel<true, false, true><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          else if (kind == 4)
            bwd_rows_batched_kernel<true, false, false, true><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          else
            bwd_rows_batched_kernel<true, false, true, true><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          LR_CHECK_CUDA(cudaGetLastError());
        }
        B.count = 0;
        tot = 0;
      }
      if (i == count) break;
      const bool dvk = p[i].dv_part != nullptr;
      const int pk = p[i].src.xy == nullptr ? (p[i].split ? (dvk ? 5 : 4) : (dvk ? 3 : 0))
                                            : (p[i].gs != nullptr ? 2 : 1);
      if (pk != kind) continue;
      B.p[B.count] = p[i];
      B.start[B.count] = (int32_t)tot;
      tot += row_block_count(p[i].map, p[i].n, p[i].rows_per_cta) * p[i].chunks;
      ++B.count;
    }
  }
  return LR_OK;
}

lr_status launch_bwd_merge_batched(const MergeArgs* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<MergeArgs> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += (p[b0 + k].n + kMergeThreads - 1) / kMergeThreads;
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    bwd_merge_batched_kernel<<<(unsigned)tot, kMergeThreads, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

lr_status launch_scalar_batched(const ScalP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<ScalP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = k;
    }
    B.start[B.count] = B.count;
    scalar_batched_kernel<<<(unsigned)B.count, kMergeThreads, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

lr_status launch_dv_rows_batched(const BwArgs* p, int count, cudaStream_t s) {
  for (int kind = 0; kind < 2; ++kind) {  // 0: unsplit, 1: split exponent
    Batch<BwArgs> B;
    B.count = 0;
    int64_t tot = 0;
    for (int i = 0; i <= count; ++i) {
      const bool flush = (i == count) || B.count == kMaxBatch;
      if (flush && B.count > 0) {
        B.start[B.count] = (int32_t)tot;
        if (tot > 0) {
          if (kind == 1)
            dv_rows_batched_kernel<true><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          else
            dv_rows_batched_kernel<false><<<(unsigned)tot, kBwThreads, 0, s>>>(B);
          LR_CHECK_CUDA(cudaGetLastError());
        }
        B.count = 0;
        tot = 0;
      }
      if (i == count) break;
      if ((p[i].split ? 1 : 0) != kind) continue;
      B.p[B.count] = p[i];
      B.start[B.count] = (int32_t)tot;
      tot += row_block_count(p[i].map, p[i].n, kDvRows) * p[i].chunks;
      ++B.count;
    }
  }
  return LR_OK;
}

lr_status launch_moments_merge_batched(const MomMergeP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<MomMergeP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += (p[b0 + k].n + 255) / 256;
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    moments_merge_batched_kernel<<<(unsigned)tot, 256, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Host side

struct RowPlan {
  int32_t n_tiles, segs, chunks, row_blocks, K, rows_per_cta;
  RowMap map;                                  // row blocks: image tiles of a grid query, else index order
  size_t partial_bytes, scal_bytes, dv_bytes;  // dv_bytes: fused d_v partials (grid sources)
  size_t info_bytes;                           // grid sources: row-block boxes
  int64_t merge_blocks;
};

static lr_status plan_rows(int64_t n, int64_t m, bool grid, const lr_grid* g, bool self, bool fuse_dv,
                           const lr_grid* qgrid, RowPlan* R) {
  RowPlan p{};
  p.K = self ? 7 : 4;
  const bool dv = grid && fuse_dv;
  p.rows_per_cta = dv ? BwCfg<true, false, true>::ROWS : (grid ? BwCfg<true, false, false>::ROWS : kBwRows);
  if (grid) {
    const int W = g->nx * g->ss;
    p.segs = (W + kBwTile - 1) / kBwTile;
    p.n_tiles = (int32_t)((int64_t)p.segs * g->ny * g->ss);
  } else {
    p.n_tiles = (int32_t)((m + kBwTile - 1) / kBwTile);
  }
  p.map = (grid && qgrid) ? make_row_map(qgrid, p.rows_per_cta) : RowMap{};
  p.row_blocks = (int32_t)row_block_count(p.map, n, p.rows_per_cta);
  p.info_bytes = grid ? row_info_bytes(p.map, n, p.rows_per_cta) : 0;
  int dev = 0, n_sm = 1, occ = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  if (self)
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bwd_rows_kernel<false, true, false>, kBwThreads, 0));
  else if (dv) {
    // the split and unsplit variants: plan for the lower occupancy of the two
    int occ2 = 1;
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bwd_rows_kernel<true, false, true>, kBwThreads, 0));
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, bwd_rows_kernel<true, false, true, true>,
                                                                kBwThreads, 0));
    occ = occ < occ2 ? occ : occ2;
  }
  else if (grid) {
    int occ2 = 1;
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bwd_rows_kernel<true, false, false>, kBwThreads, 0));
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, bwd_rows_kernel<true, false, false, true>,
                                                                kBwThreads, 0));
    occ = occ < occ2 ? occ : occ2;
  } else {
    LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bwd_rows_kernel<false, false, false>, kBwThreads, 0));
  }
  const int32_t chunks = plan_chunks(p.row_blocks, p.n_tiles, occ, n_sm, grid ? kSkipWaves : kChunkWaves);
  p.chunks = chunks;
  p.partial_bytes = align256(sizeof(float) * (size_t)p.chunks * p.K * (size_t)n);
  p.merge_blocks = (n + kMergeThreads - 1) / kMergeThreads;
  p.scal_bytes = align256(sizeof(double) * 2 * (size_t)(p.merge_blocks > 0 ? p.merge_blocks : 1));
  p.dv_bytes = grid ? align256(sizeof(float) * (size_t)p.row_blocks * (size_t)m) : 0;
  *R = p;
  return LR_OK;
}

// Merge of non-self row-pass partials [chunks][4][n] (A, B_x, B_y, C) into
// d_x and the FP64 block partials of d_l and d_var.
static MergeArgs row_merge_args(bool grid, float ell, float var, const float* partial, int32_t chunks, int64_t n,
                                const float* g, const float* vrow, float2* dx, double* scal_part) {
  const double c = 1.4426950408889634 / (2.0 * (double)ell * (double)ell);
  MergeArgs mm{};
  mm.partial = partial;
  mm.chunks = chunks;
  mm.K = 4;
  mm.n = n;
  mm.g = g;
  mm.vrow = vrow;
  mm.var = var;
  mm.inv_l2 = (float)(1.0 / ((double)ell * ell));
  // grid path: C = sum k v c d^2 (positive), B in coordinates scaled by sc;
  // explicit path: C = sum k v e with e = -c d^2, B unscaled
  mm.dl_scale = (float)((grid ? 1.0 : -1.0) * (double)var / (c * (double)ell * ell * ell));
  mm.b_scale = grid ? (float)(1.0 / sqrt(c)) : 1.0f;
  mm.d_x = dx;
  mm.d_v = nullptr;
  mm.scal_part = scal_part;
  return mm;
}

// Problem descriptors for the non-self row pass (d_x, d_l, d_var) of explicit
// query points against grid (yg) or explicit (ys) sources, planned as
// gp_kernel_matvec_bwd plans it; ws receives the partials. With ws == NULL
// only *bytes is filled in.
lr_status make_rows_problem(const float2* x, int64_t n, const lr_grid* qgrid, const float2* ys, const lr_grid* yg,
                            int64_t m, const float* v, const float* g, float ell, float var, float2* dx, double* d_len,
                            double* d_var, float* d_v, char* ws, BwArgs* A, MergeArgs* M, ScalP* S, DvMergeP* D,
                            RowInfoP* RI, size_t* bytes) {
  RowPlan R;
  const bool grid = ys == nullptr;
  const bool fuse = grid && d_v != nullptr;
  lr_status st = plan_rows(n, m, grid, yg, false, fuse, qgrid, &R);
  if (st != LR_OK) return st;
  const size_t off_info = R.partial_bytes + R.scal_bytes + (fuse ? R.dv_bytes : 0);
  *bytes = off_info + R.info_bytes;
  if (!ws) return LR_OK;
  BwArgs a{};
  a.x = x;
  a.n = n;
  a.src.xy = ys;
  a.src.g = ys ? GridDev{} : grid_dev(*yg);
  a.src.m = m;
  a.src.segs = R.segs;
  a.src.n_tiles = R.n_tiles;
  a.v = v;
  a.gs = nullptr;
  const double c = 1.4426950408889634 / (2.0 * (double)ell * (double)ell);
  a.neg_c = (float)(-c);
  a.sc = (float)sqrt(c);
  a.split = ys ? 0 : grid_split_ok(a.src.g, a.sc);
  a.chunks = R.chunks;
  a.K = R.K;
  a.rows_per_cta = R.rows_per_cta;
  a.partial = reinterpret_cast<float*>(ws);
  a.grow = fuse ? g : nullptr;
  a.dv_part = fuse ? reinterpret_cast<float*>(ws + R.partial_bytes + R.scal_bytes) : nullptr;
  a.map = R.map;
  a.info = grid ? reinterpret_cast<const RowBlockInfo*>(ws + off_info) : nullptr;
  *A = a;
  if (RI)
    *RI = RowInfoP{x, n, R.map, R.rows_per_cta, R.segs, a.src.g, a.sc,
                   grid ? reinterpret_cast<RowBlockInfo*>(ws + off_info) : nullptr};
  *M = row_merge_args(grid, ell, var, a.partial, R.chunks, n, g, v, dx, reinterpret_cast<double*>(ws + R.partial_bytes));
  S->part = M->scal_part;
  S->nblk = (int32_t)R.merge_blocks;
  S->d_len = d_len;
  S->d_var = d_var;
  if (D) {
    D->dv_part = a.dv_part;
    D->row_blocks = R.row_blocks;
    D->m = m;
    D->var = var;
    D->d_v = fuse ? d_v : nullptr;
    D->info = a.info;
    D->W = grid ? a.src.g.W : 0;
    D->segs = R.segs;
  }
  return LR_OK;
}

static lr_status launch_rows(const float2* x, int64_t n, const lr_grid* qgrid, const float2* ys, const lr_grid* yg,
                             int64_t m, const float* v, const float* gs, const float* g, const float* vrow, float ell,
                             float var, bool self, float2* d_x, float* d_v, double* d_len, double* d_var, char* ws,
                             cudaStream_t s) {
  if (!self) {
    // grid sources fuse d_v into the row pass; explicit sources leave d_v to the caller
    BwArgs A;
    MergeArgs M;
    ScalP S;
    DvMergeP D;
    RowInfoP RI;
    size_t b = 0;
    lr_status st = make_rows_problem(x, n, qgrid, ys, yg, m, v, g, ell, var, d_x, d_len, d_var,
                                     ys == nullptr ? d_v : nullptr, ws, &A, &M, &S, &D, &RI, &b);
    if (st != LR_OK) return st;
    if (RI.info && (st = launch_row_info(RI, s)) != LR_OK) return st;
    const unsigned grid = (unsigned)(row_block_count(A.map, n, A.rows_per_cta) * A.chunks);
    ktimer_begin(LR_KT_BWD_ROWS, s);
    if (ys == nullptr && A.dv_part && A.split)
      bwd_rows_kernel<true, false, true, true><<<grid, kBwThreads, 0, s>>>(A);
    else if (ys == nullptr && A.dv_part)
      bwd_rows_kernel<true, false, true><<<grid, kBwThreads, 0, s>>>(A);
    else if (ys == nullptr && A.split)
      bwd_rows_kernel<true, false, false, true><<<grid, kBwThreads, 0, s>>>(A);
    else if (ys == nullptr)
      bwd_rows_kernel<true, false, false><<<grid, kBwThreads, 0, s>>>(A);
    else
      bwd_rows_kernel<false, false, false><<<grid, kBwThreads, 0, s>>>(A);
    LR_CHECK_CUDA(cudaGetLastError());
    ktimer_end(LR_KT_BWD_ROWS, s);
    bwd_merge_kernel<<<(unsigned)S.nblk, kMergeThreads, 0, s>>>(M);
    LR_CHECK_CUDA(cudaGetLastError());
    if (d_len || d_var) {
      bwd_scalar_final_kernel<<<1, kMergeThreads, 0, s>>>(S.part, S.nblk, d_len, d_var);
      LR_CHECK_CUDA(cudaGetLastError());
    }
    if (A.dv_part) {
      dv_merge_kernel<<<(unsigned)dv_merge_blocks(D), kDvMergeCols * kDvMergeGroups, 0, s>>>(D);
      LR_CHECK_CUDA(cudaGetLastError());
    }
    return LR_OK;
  }
  RowPlan R;
  lr_status st = plan_rows(n, m, false, yg, true, false, nullptr, &R);
  if (st != LR_OK) return st;
  BwArgs A{};
  A.x = x;
  A.n = n;
  A.src.xy = ys;
  A.src.m = m;
  A.src.segs = R.segs;
  A.src.n_tiles = R.n_tiles;
  A.v = v;
  A.gs = gs;
  const double c = 1.4426950408889634 / (2.0 * (double)ell * (double)ell);
  A.neg_c = (float)(-c);
  A.sc = (float)sqrt(c);
  A.split = 0;
  A.chunks = R.chunks;
  A.K = R.K;
  A.rows_per_cta = R.rows_per_cta;
  A.partial = reinterpret_cast<float*>(ws);
  A.grow = nullptr;
  A.dv_part = nullptr;
  const unsigned grid = (unsigned)((int64_t)R.row_blocks * R.chunks);
  ktimer_begin(LR_KT_BWD_ROWS, s);
  bwd_rows_kernel<false, true, false><<<grid, kBwThreads, 0, s>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_BWD_ROWS, s);
  MergeArgs M{};
  M.partial = A.partial;
  M.chunks = R.chunks;
  M.K = R.K;
  M.n = n;
  M.g = g;
  M.vrow = vrow;
  M.var = var;
  M.inv_l2 = (float)(1.0 / ((double)ell * ell));
  // explicit path: C = sum k v e with e = -c d^2; d_len = var/l^3 sum g_i (sum_j k v d^2)
  M.dl_scale = (float)(-(double)var / (c * (double)ell * ell * ell));
  M.b_scale = 1.0f;
  M.d_x = d_x;
  M.d_v = d_v;
  M.scal_part = reinterpret_cast<double*>(ws + R.partial_bytes);
  bwd_merge_kernel<<<(unsigned)R.merge_blocks, kMergeThreads, 0, s>>>(M);
  LR_CHECK_CUDA(cudaGetLastError());
  if (d_len || d_var) {
    bwd_scalar_final_kernel<<<1, kMergeThreads, 0, s>>>(M.scal_part, (int)R.merge_blocks, d_len, d_var);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

// Plan of the d_v-only pass over grid sources (dv_rows_kernel).
static lr_status plan_dv(int64_t n, const lr_grid* g, const lr_grid* qgrid, RowPlan* R) {
  RowPlan p{};
  p.K = 0;
  p.rows_per_cta = kDvRows;
  const int W = g->nx * g->ss;
  p.segs = (W + kBwTile - 1) / kBwTile;
  p.n_tiles = (int32_t)((int64_t)p.segs * g->ny * g->ss);
  p.map = qgrid ? make_row_map(qgrid, kDvRows) : RowMap{};
  p.row_blocks = (int32_t)row_block_count(p.map, n, kDvRows);
  p.info_bytes = row_info_bytes(p.map, n, kDvRows);
  int dev = 0, n_sm = 1, occ = 1, occ2 = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dv_rows_kernel<true>, kBwThreads, 0));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, dv_rows_kernel<false>, kBwThreads, 0));
  p.chunks = plan_chunks(p.row_blocks, p.n_tiles, occ < occ2 ? occ : occ2, n_sm, kSkipWaves);
  const int64_t m = (int64_t)W * g->ny * g->ss;
  p.dv_bytes = align256(sizeof(float) * (size_t)p.row_blocks * (size_t)m);
  *R = p;
  return LR_OK;
}

lr_status make_train_problem(const float2* x, int64_t n, const lr_grid* qgrid, const float2* ys, const lr_grid* yg,
                             int64_t m, const float* v, float ell, float var, float* out, float* mom, char* ws,
                             BwArgs* A, MomMergeP* MM, RowInfoP* RI, size_t* bytes) {
  BwArgs a;
  MergeArgs M;
  ScalP S;
  lr_status st = make_rows_problem(x, n, qgrid, ys, yg, m, v, nullptr, ell, var, nullptr, nullptr, nullptr, nullptr,
                                   ws, ws ? &a : nullptr, ws ? &M : nullptr, ws ? &S : nullptr, nullptr, RI, bytes);
  if (st != LR_OK || !ws) return st;
  *A = a;
  MM->partial = a.partial;
  MM->chunks = a.chunks;
  MM->n = n;
  MM->var = var;
  MM->out = out;
  MM->mom = mom;
  return LR_OK;
}

lr_status make_moment_rows_problem(const float* mom, int64_t n, bool grid, const float* g, const float* v, float ell,
                                   float var, float2* dx, double* d_len, double* d_var, char* ws, MergeArgs* M,
                                   ScalP* S, size_t* bytes) {
  const int64_t nblk = (n + kMergeThreads - 1) / kMergeThreads;
  *bytes = align256(sizeof(double) * 2 * (size_t)(nblk + 1));
  if (!ws) return LR_OK;
  *M = row_merge_args(grid, ell, var, mom, 1, n, g, v, dx, reinterpret_cast<double*>(ws));
  S->part = M->scal_part;
  S->nblk = (int32_t)nblk;
  S->d_len = d_len;
  S->d_var = d_var;
  return LR_OK;
}

lr_status make_dv_problem(const float2* x, int64_t n, const lr_grid* qgrid, const lr_grid* yg, const float* g,
                          float ell, float var, float* d_v, char* ws, BwArgs* A, DvMergeP* D, RowInfoP* RI,
                          size_t* bytes) {
  RowPlan R;
  lr_status st = plan_dv(n, yg, qgrid, &R);
  if (st != LR_OK) return st;
  *bytes = R.dv_bytes + R.info_bytes;
  if (!ws) return LR_OK;
  BwArgs a{};
  a.x = x;
  a.n = n;
  a.src.xy = nullptr;
  a.src.g = grid_dev(*yg);
  a.src.m = (int64_t)a.src.g.W * a.src.g.H;
  a.src.segs = R.segs;
  a.src.n_tiles = R.n_tiles;
  const double c = 1.4426950408889634 / (2.0 * (double)ell * (double)ell);
  a.neg_c = (float)(-c);
  a.sc = (float)sqrt(c);
  a.split = grid_split_ok(a.src.g, a.sc);
  a.chunks = R.chunks;
  a.rows_per_cta = kDvRows;
  a.grow = g;
  a.dv_part = reinterpret_cast<float*>(ws);
  a.map = R.map;
  RowBlockInfo* info = reinterpret_cast<RowBlockInfo*>(ws + R.dv_bytes);
  a.info = info;
  *A = a;
  *D = DvMergeP{a.dv_part, R.row_blocks, a.src.m, var, d_v, info, a.src.g.W, R.segs};
  if (RI) *RI = RowInfoP{x, n, R.map, kDvRows, R.segs, a.src.g, a.sc, info};
  return LR_OK;
}

// d_v of grid sources from the d_v-only pass: dv_part, then the fixed-order
// merge over row blocks. ws: the plan's dv_bytes.
static lr_status launch_dv(const float2* x, int64_t n, const lr_grid* qgrid, const lr_grid* yg, const float* g,
                           float ell, float var, float* d_v, char* ws, cudaStream_t s) {
  BwArgs A;
  DvMergeP D;
  RowInfoP RI;
  size_t b = 0;
  lr_status st = make_dv_problem(x, n, qgrid, yg, g, ell, var, d_v, ws, &A, &D, &RI, &b);
  if (st != LR_OK) return st;
  if ((st = launch_row_info(RI, s)) != LR_OK) return st;
  const unsigned grid = (unsigned)(row_block_count(A.map, n, kDvRows) * A.chunks);
  ktimer_begin(LR_KT_DV_ROWS, s);
  if (A.split)
    dv_rows_kernel<true><<<grid, kBwThreads, 0, s>>>(A);
  else
    dv_rows_kernel<false><<<grid, kBwThreads, 0, s>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_DV_ROWS, s);
  dv_merge_kernel<<<(unsigned)dv_merge_blocks(D), kDvMergeCols * kDvMergeGroups, 0, s>>>(D);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

// Row gradients from the training forward's moments: d_x, d_l, d_var.
// ws: the scalar partials (make_moment_rows_problem's bytes).
static lr_status launch_moment_rows(const float* mom, int64_t n, bool grid, const float* g, const float* v, float ell,
                                    float var, float2* d_x, double* d_len, double* d_var, char* ws, cudaStream_t s) {
  MergeArgs M;
  ScalP S;
  size_t b = 0;
  lr_status st = make_moment_rows_problem(mom, n, grid, g, v, ell, var, d_x, d_len, d_var, ws, &M, &S, &b);
  if (st != LR_OK) return st;
  bwd_merge_kernel<<<(unsigned)S.nblk, kMergeThreads, 0, s>>>(M);
  LR_CHECK_CUDA(cudaGetLastError());
  if (d_len || d_var) {
    bwd_scalar_final_kernel<<<1, kMergeThreads, 0, s>>>(S.part, S.nblk, d_len, d_var);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

static size_t rows_ws(int64_t n, int64_t m, bool grid, const lr_grid* g, bool self, bool fuse_dv,
                      const lr_grid* qgrid, lr_status* st) {
  RowPlan R;
  *st = plan_rows(n, m, grid, g, self, fuse_dv, qgrid, &R);
  return R.partial_bytes + R.scal_bytes + (fuse_dv ? R.dv_bytes : 0) + R.info_bytes;
}

struct BwPlan {
  int64_t n, m;
  int32_t nrhs;
  bool self, q_raytrace, q_grid, s_raytrace, s_grid;
  bool want_lens;       // lens / subhalo gradients of the query's lens
  bool need_dx;         // d_x needed (requested or for the lens gradient)
  bool moments;         // row sums given by the training forward
  bool culled;          // explicit or self sources without moments: culled sweeps
  bool slice;           // the query is rows [row0, row0 + n) of the source set (self-kernel rows)
  bool s_mat;           // grid source written out as points (several right-hand sides)
  int64_t row0;
  CullPlan cp_rows;     // culled: self backward, or the non-self row moments
  CullPlan cp_dy;       // culled, non-self with d_y: row moments with the roles swapped
  size_t off_qbeta, off_sbeta, off_rows, off_dv, off_dx, off_sgrid, off_swap, off_swaprows, off_vjp, off_scal, bytes;
  size_t swap_bytes;    // workspace of the swapped forward (d_v of explicit sources)
};

static lr_status plan_bwd(const lr_points* q, const lr_points* s, int32_t nrhs, const lr_grads* gr, BwPlan* P) {
  lr_status st = validate_points(q, "gp_kernel_matvec_bwd(query)", false);
  if (st != LR_OK) return st;
  if (s) {
    st = validate_points(s, "gp_kernel_matvec_bwd(source)", false);
    if (st != LR_OK) return st;
  }
  LR_REQUIRE(gr != nullptr, "gp_kernel_matvec_bwd: grads is NULL");
  BwPlan p{};
  p.n = q->n;
  p.nrhs = nrhs;
  p.self = s == nullptr;
  p.m = p.self ? q->n : s->n;
  p.q_raytrace = has_lens(q);
  p.q_grid = !p.q_raytrace && q->xy == nullptr;
  p.s_raytrace = !p.self && has_lens(s);
  p.s_grid = !p.self && !p.s_raytrace && s->xy == nullptr;
  LR_REQUIRE(!p.s_raytrace, "gp_kernel_matvec_bwd: a ray-traced source set distinct from the query is not supported");
  LR_REQUIRE(!(gr->d_y && (p.self || p.s_grid)),
             "gp_kernel_matvec_bwd: d_y applies to explicit non-self source points only");
  // several right-hand sides over grid sources: the grid's points are written
  // out and the culled sweeps take them as explicit points
  p.s_mat = p.s_grid && nrhs > 1 && gr->moments_in == nullptr;
  if (p.s_mat) p.s_grid = false;
  p.want_lens = (gr->d_lens || gr->d_sub);
  LR_REQUIRE(!p.want_lens || p.q_raytrace, "gp_kernel_matvec_bwd: lens gradients need a ray-traced query");
  p.need_dx = gr->d_x || p.want_lens;
  LR_REQUIRE(gr->beta_in == nullptr || p.q_raytrace, "gp_kernel_matvec_bwd: beta_in given but the query is not ray-traced");
  LR_REQUIRE(((uintptr_t)gr->beta_in & 7u) == 0, "gp_kernel_matvec_bwd: beta_in must be 8-byte aligned");
  p.moments = gr->moments_in != nullptr;
  const lr_grid* qg = query_layout(q);  // row blocks follow the image tiles
  LR_REQUIRE(!p.moments || !p.self, "gp_kernel_matvec_bwd: moments_in applies to non-self sources only");
  LR_REQUIRE(((uintptr_t)gr->moments_in & 3u) == 0, "gp_kernel_matvec_bwd: moments_in must be 4-byte aligned");
  p.slice = gr->source_rows != 0;
  if (p.slice) {
    LR_REQUIRE(!p.self && !p.s_grid, "gp_kernel_matvec_bwd: source_rows needs explicit source points");
    LR_REQUIRE(!p.moments && gr->d_y == nullptr, "gp_kernel_matvec_bwd: source_rows excludes moments_in and d_y");
    LR_REQUIRE(gr->row0 >= 0 && gr->row0 + p.n <= p.m,
               "gp_kernel_matvec_bwd: rows [%lld, %lld) outside the %lld source points", (long long)gr->row0,
               (long long)(gr->row0 + p.n), (long long)p.m);
  }
  p.culled = !p.s_grid && !p.moments;
  if (p.culled) {
    LR_REQUIRE(nrhs >= 1 && nrhs <= 4, "gp_kernel_matvec_bwd: nrhs = %d; 1..4 right-hand sides", nrhs);
  } else {
    LR_REQUIRE(nrhs == 1, "gp_kernel_matvec_bwd: nrhs = %d; moments_in takes nrhs = 1", nrhs);
  }
  size_t off = 0;
  p.off_qbeta = off;
  if ((p.q_raytrace && !gr->beta_in) || p.q_grid) off += align256(8 * (size_t)p.n);
  p.off_sbeta = off;
  if (p.s_mat) off += align256(8 * (size_t)p.m);
  p.off_rows = off;
  p.off_scal = off;
  if (p.culled) {
    const lr_grid* sg = p.self ? qg : query_layout(s);
    p.row0 = p.slice ? gr->row0 : 0;
    // the self-kernel sweep takes every right-hand side at once; the
    // non-self row moments one at a time
    const bool both = p.self || p.slice;
    st = plan_cull(both ? kCullSelf : kCullMom, both ? nrhs : 1, p.n, qg, p.m, sg, &p.cp_rows);
    if (st != LR_OK) return st;
    off += p.cp_rows.bytes;
    // scalar partials of every right-hand side, summed once at the end
    p.off_scal = off;
    off += align256(sizeof(double) * 2 * (size_t)nrhs * (size_t)(p.cp_rows.scal_blocks > 0 ? p.cp_rows.scal_blocks : 1));
  } else if (p.moments) {
    // scalar partials of the moment merge, then the d_v-only pass of grid sources
    off += align256(sizeof(double) * 2 * (size_t)((p.n + kMergeThreads - 1) / kMergeThreads + 1));
    p.off_dv = off;
    if (p.s_grid && gr->d_v && p.n > 0) {
      RowPlan R;
      st = plan_dv(p.n, &s->grid, qg, &R);
      if (st != LR_OK) return st;
      off += R.dv_bytes + R.info_bytes;
    }
  } else {
    size_t b = rows_ws(p.n, p.m, p.s_grid, p.s_grid ? &s->grid : nullptr, p.self, p.s_grid && gr->d_v != nullptr, qg,
                       &st);
    if (st != LR_OK) return st;
    off += b;
  }
  p.off_dx = off;
  if (p.need_dx && !gr->d_x) off += align256(8 * (size_t)p.n);
  p.off_sgrid = off;
  p.off_swap = off;
  p.off_swaprows = off;
  if (!p.self && !p.slice && gr->d_v && !p.s_grid) {
    // d_v: the forward reduction with the roles swapped (query = the
    // sources, source = the query points)
    lr_points qs = *s, ss = *q;
    qs.lens = nullptr;
    qs.lens_record = nullptr;
    ss.lens = nullptr;
    ss.lens_record = nullptr;
    ss.xy = reinterpret_cast<const float*>(uintptr_t(256));  // planning reads no point
    st = lr_matvec_workspace_size(&qs, &ss, nrhs, &p.swap_bytes);
    if (st != LR_OK) return st;
    off += align256(p.swap_bytes);
  }
  p.off_swaprows = off;
  if (!p.self && gr->d_y) {
    if (p.culled) {
      st = plan_cull(kCullMom, 1, p.m, query_layout(s), p.n, qg, &p.cp_dy);
      if (st != LR_OK) return st;
      off += p.cp_dy.bytes;
    } else {
      size_t b = rows_ws(p.m, p.n, false, nullptr, false, false, nullptr, &st);
      if (st != LR_OK) return st;
      off += b;
    }
  }
  p.off_vjp = off;
  if (p.want_lens) off += raytrace_vjp_ws(p.n, q->n_sub);
  p.bytes = off;
  *P = p;
  return LR_OK;
}

// The culled backward of explicit or self sources: per right-hand side the
// self-kernel sweep (d_v, d_x of both roles, scalar partials) or the row
// moments (d_x, scalar partials); then d_v and d_y of non-self sources with
// the roles swapped; then d_l and d_var from every partial in fixed order.
static lr_status launch_culled_bwd(const BwPlan& P, const lr_points* query, const lr_points* source,
                                   const float2* xq, const float2* ys, const float* v, float ell, float var,
                                   const float* g, const lr_grads& G, float2* dx, char* ws, lr_stream stream) {
  cudaStream_t s = as_cuda(stream);
  const double c = 1.4426950408889634 / (2.0 * (double)ell * (double)ell);
  const float sc = (float)sqrt(c);
  const float dx_scale = (float)((double)var / ((double)ell * ell));
  const float dl_scale = (float)((double)var / ((double)ell * ell * ell));
  const bool want_scal = G.d_lengthscale || G.d_variance;
  double* scal = reinterpret_cast<double*>(ws + P.off_scal);
  const int64_t nblk = P.cp_rows.scal_blocks;
  char* cws = ws + P.off_rows;
  lr_status st;
  // a self-kernel, or rows [row0, row0 + n) of one: both roles of the rows
  const bool both = P.self || P.slice;
  const bool rows_needed = both ? (G.d_v || dx || want_scal) : (dx || want_scal);
  const int sweeps = both ? 1 : P.nrhs;  // the self-kernel sweep takes every column at once
  for (int r = 0; r < sweeps && rows_needed; ++r) {
    st = launch_cull_prep(P.cp_rows, ys, sc, v, both ? g : nullptr, P.nrhs, both ? 0 : r, cws, s);
    if (st != LR_OK) return st;
    CullArgs A{};
    A.x = xq;
    A.n = P.n;
    A.sc = sc;
    A.c = (float)c;
    A.nrhs = 1;
    A.var = var;
    A.dx_scale = dx_scale;
    A.dl_scale = dl_scale;
    // the rows' own g and v: the first n, or rows row0.. of the source set
    A.g = g + (size_t)P.row0 * P.nrhs;
    A.vrow = v + (size_t)P.row0 * P.nrhs;
    A.stride = P.nrhs;
    A.col = both ? 0 : r;
    A.d_x = dx;
    A.dx_accumulate = r > 0;
    A.d_v = both ? G.d_v : nullptr;
    A.scal_part = want_scal ? scal + 2 * (size_t)r * (size_t)nblk : nullptr;
    st = launch_cull_sweep(P.cp_rows, A, cws, LR_KT_BWD_ROWS, s);
    if (st != LR_OK) return st;
  }
  if (want_scal) {
    st = launch_cull_scalar_final(scal, (int64_t)sweeps * nblk, G.d_lengthscale, G.d_variance, s);
    if (st != LR_OK) return st;
  }
  if (!P.self && !P.slice && G.d_v) {
    // d_v_j = var sum_i k_ij g_i: the forward with the roles swapped
    lr_points qs = *source, ss{};
    qs.lens = nullptr;
    qs.lens_record = nullptr;
    ss.xy = reinterpret_cast<const float*>(xq);
    ss.n = P.n;
    const lr_grid* qg = query_layout(query);
    if (qg) ss.grid = *qg;
    st = gp_kernel_matvec(&qs, &ss, g, P.nrhs, ell, var, G.d_v, nullptr, ws + P.off_swap, P.swap_bytes, stream);
    if (st != LR_OK) return st;
  }
  if (!P.self && G.d_y) {
    // d_y_j = var/l^2 v_j sum_i k_ij g_i (x_i - y_j): row moments of g with
    // the roles swapped, rows multiplied by their own v
    char* dws = ws + P.off_swaprows;
    for (int r = 0; r < P.nrhs; ++r) {
      st = launch_cull_prep(P.cp_dy, xq, sc, g, nullptr, P.nrhs, r, dws, s);
      if (st != LR_OK) return st;
      CullArgs A{};
      A.x = ys;
      A.n = P.m;
      A.sc = sc;
      A.c = (float)c;
      A.nrhs = 1;
      A.var = var;
      A.dx_scale = dx_scale;
      A.dl_scale = dl_scale;
      A.g = v;
      A.stride = P.nrhs;
      A.col = r;
      A.d_x = reinterpret_cast<float2*>(G.d_y);
      A.dx_accumulate = r > 0;
      A.scal_part = nullptr;
      st = launch_cull_sweep(P.cp_dy, A, dws, -1, s);
      if (st != LR_OK) return st;
    }
  }
  return LR_OK;
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_matvec_bwd_workspace_size(const lr_points* query, const lr_points* source, int32_t nrhs,
                                                  const lr_grads* grads, size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_matvec_bwd_workspace_size: bytes is NULL");
  BwPlan P;
  lr_status st = plan_bwd(query, source, nrhs, grads, &P);
  if (st != LR_OK) return st;
  *bytes = P.bytes;
  return LR_OK;
}

extern "C" lr_status gp_kernel_matvec_bwd(const lr_points* query, const lr_points* source, const float* v,
                                          int32_t nrhs, float lengthscale, float variance, const float* g_out,
                                          const lr_grads* grads, void* workspace, size_t workspace_bytes,
                                          lr_stream stream) {
  BwPlan P;
  lr_status st = plan_bwd(query, source, nrhs, grads, &P);
  if (st != LR_OK) return st;
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "gp_kernel_matvec_bwd: lengthscale must be > 0");
  LR_REQUIRE(isfinite(variance), "gp_kernel_matvec_bwd: variance is not finite");
  LR_REQUIRE(g_out != nullptr || P.n == 0, "gp_kernel_matvec_bwd: g_out is NULL");
  LR_REQUIRE(v != nullptr || P.m == 0, "gp_kernel_matvec_bwd: v is NULL");
  LR_REQUIRE(workspace_bytes >= P.bytes, "gp_kernel_matvec_bwd: workspace of %zu bytes, %zu needed",
             workspace_bytes, P.bytes);
  LR_REQUIRE(P.bytes == 0 || workspace != nullptr, "gp_kernel_matvec_bwd: workspace is NULL");
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0, "gp_kernel_matvec_bwd: workspace must be 256-byte aligned");
  const lr_grads& G = *grads;
  LR_REQUIRE(((uintptr_t)G.d_x & 7u) == 0 && ((uintptr_t)G.d_y & 7u) == 0 && ((uintptr_t)G.d_lens & 7u) == 0 &&
                 ((uintptr_t)G.d_sub & 7u) == 0 && ((uintptr_t)G.d_lengthscale & 7u) == 0 &&
                 ((uintptr_t)G.d_variance & 7u) == 0,
             "gp_kernel_matvec_bwd: gradient outputs must be 8-byte aligned");
  cudaStream_t s = as_cuda(stream);
  char* ws = static_cast<char*>(workspace);
  if (P.n == 0 || P.m == 0) {
    // every gradient is an empty sum
    const int64_t nv = P.slice ? P.n : P.m;  // d_v covers the query rows in the slice mode
    if (G.d_v && nv) LR_CHECK_CUDA(cudaMemsetAsync(G.d_v, 0, 4 * (size_t)nv * (size_t)P.nrhs, s));
    if (G.d_x && P.n) LR_CHECK_CUDA(cudaMemsetAsync(G.d_x, 0, 8 * (size_t)P.n, s));
    if (G.d_y && P.m) LR_CHECK_CUDA(cudaMemsetAsync(G.d_y, 0, 8 * (size_t)P.m, s));
    if (G.d_lengthscale) LR_CHECK_CUDA(cudaMemsetAsync(G.d_lengthscale, 0, 8, s));
    if (G.d_variance) LR_CHECK_CUDA(cudaMemsetAsync(G.d_variance, 0, 8, s));
    if (G.d_lens) LR_CHECK_CUDA(cudaMemsetAsync(G.d_lens, 0, 56, s));
    if (G.d_sub && query->n_sub) LR_CHECK_CUDA(cudaMemsetAsync(G.d_sub, 0, 32 * (size_t)query->n_sub, s));
    return LR_OK;
  }
  // query points: the forward's ray-traced points when given, else recomputed
  const float2* xq = reinterpret_cast<const float2*>(query->xy);
  if (P.q_raytrace && G.beta_in) {
    xq = reinterpret_cast<const float2*>(G.beta_in);
  } else if (P.q_raytrace || P.q_grid) {
    float2* qb = reinterpret_cast<float2*>(ws + P.off_qbeta);
    st = P.q_raytrace ? launch_raytrace(query, qb, nullptr, s) : launch_grid_points(query->grid, qb, s);
    if (st != LR_OK) return st;
    xq = qb;
  }
  const float2* ys = P.self ? xq : (P.s_grid ? nullptr : reinterpret_cast<const float2*>(source->xy));
  if (P.s_mat) {
    float2* sb = reinterpret_cast<float2*>(ws + P.off_sbeta);
    if ((st = launch_grid_points(source->grid, sb, s)) != LR_OK) return st;
    ys = sb;
  }
  const lr_grid* yg = P.s_grid ? &source->grid : nullptr;
  const lr_grid* qgrid = query_layout(query);
  float2* dx = P.need_dx ? (G.d_x ? reinterpret_cast<float2*>(G.d_x) : reinterpret_cast<float2*>(ws + P.off_dx))
                         : nullptr;
  if (P.moments && P.s_grid) {
    // grid sources with the training forward's moments: the row gradients
    // (then the ray-trace VJP) and d_v from the d_v-only sweep are
    // independent branches; the d_v one runs on a side stream so that the
    // two overlap
    Fork f{};
    const bool side = G.d_v != nullptr;
    if (side && (st = fork_begin(s, &f)) != LR_OK) return st;
    if (side) st = launch_dv(xq, P.n, qgrid, yg, g_out, lengthscale, variance, G.d_v, ws + P.off_dv, f.side);
    if (st == LR_OK)
      st = launch_moment_rows(G.moments_in, P.n, true, g_out, v, lengthscale, variance, dx, G.d_lengthscale,
                              G.d_variance, ws + P.off_rows, s);
    if (st == LR_OK && P.want_lens) st = launch_raytrace_vjp(query, dx, G.d_lens, G.d_sub, ws + P.off_vjp, s);
    const lr_status sj = side ? fork_end(s, &f) : LR_OK;
    return st != LR_OK ? st : sj;
  }
  if (P.culled) {
    // explicit or self sources: the culled sweeps (d_v and d_y included)
    st = launch_culled_bwd(P, query, source, xq, ys, v, lengthscale, variance, g_out, G, dx, ws, stream);
    if (st != LR_OK) return st;
  } else if (P.moments) {
    // row gradients from the training forward's moments
    st = launch_moment_rows(G.moments_in, P.n, P.s_grid, g_out, v, lengthscale, variance, dx, G.d_lengthscale,
                            G.d_variance, ws + P.off_rows, s);
    if (st != LR_OK) return st;
  } else {
    // row pass: d_x (both roles for a self-kernel), self d_v, d_l, d_var
    st = launch_rows(xq, P.n, qgrid, ys, yg, P.m, v, P.self ? g_out : nullptr, g_out, v, lengthscale, variance, P.self,
                     dx,
                     (P.self || P.s_grid) ? G.d_v : nullptr, G.d_lengthscale, G.d_variance, ws + P.off_rows, s);
    if (st != LR_OK) return st;
  }
  // d_v of explicit non-self sources after the training forward: sum_i var
  // k_ij g_i, the forward reduction with the point sets swapped (grid sources
  // have it fused into the row pass)
  if (!P.culled && !P.self && !P.s_grid && G.d_v) {
    lr_points qs = *source, ss{};
    qs.lens = nullptr;
    qs.lens_record = nullptr;
    ss.xy = reinterpret_cast<const float*>(xq);
    ss.n = P.n;
    const lr_grid* qg = query_layout(query);
    if (qg) ss.grid = *qg;
    st = gp_kernel_matvec(&qs, &ss, g_out, 1, lengthscale, variance, G.d_v, nullptr, ws + P.off_swap, P.swap_bytes,
                          stream);
    if (st != LR_OK) return st;
  }
  // d_y of explicit non-self sources after the training forward: the row pass
  // with the point sets swapped
  if (!P.culled && !P.self && G.d_y) {
    st = launch_rows(reinterpret_cast<const float2*>(source->xy), P.m, nullptr, xq, nullptr, P.n, g_out, nullptr, v,
                     g_out,
                     lengthscale, variance, false, reinterpret_cast<float2*>(G.d_y), nullptr, nullptr, nullptr,
                     ws + P.off_swaprows, s);
    if (st != LR_OK) return st;
  }
  // lens and subhalo gradients through the ray-trace
  if (P.want_lens) {
    st = launch_raytrace_vjp(query, dx, G.d_lens, G.d_sub, ws + P.off_vjp, s);
    if (st != LR_OK) return st;
  }
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Training forward: the non-self row pass with the source weights v gives the
// per-row moments (A, B_x, B_y, C); out = var A. One sweep over the pairs
// serves the forward output and the row half of the backward.
namespace lr {

struct TrainPlan {
  int64_t n, m;
  bool q_raytrace, q_grid, s_grid;
  RowPlan R;
  size_t off_qbeta, off_rows, bytes;
};

static lr_status plan_train(const lr_points* q, const lr_points* s, TrainPlan* T) {
  lr_status st = validate_points(q, "gp_kernel_matvec_train(query)", false);
  if (st != LR_OK) return st;
  LR_REQUIRE(s != nullptr, "gp_kernel_matvec_train: a self-kernel (source == NULL) is not supported");
  st = validate_points(s, "gp_kernel_matvec_train(source)", false);
  if (st != LR_OK) return st;
  LR_REQUIRE(!has_lens(s), "gp_kernel_matvec_train: ray-traced sources are not supported");
  TrainPlan p{};
  p.n = q->n;
  p.m = s->n;
  p.q_raytrace = has_lens(q);
  p.q_grid = !p.q_raytrace && q->xy == nullptr;
  p.s_grid = s->xy == nullptr;
  size_t off = 0;
  p.off_qbeta = off;
  if (p.q_raytrace || p.q_grid) off += align256(8 * (size_t)p.n);
  p.off_rows = off;
  if (p.n > 0 && p.m > 0) {
    st = plan_rows(p.n, p.m, p.s_grid, p.s_grid ? &s->grid : nullptr, false, false, query_layout(q), &p.R);
    if (st != LR_OK) return st;
    off += p.R.partial_bytes + p.R.scal_bytes + p.R.info_bytes;
  }
  p.bytes = off;
  *T = p;
  return LR_OK;
}

}  // namespace lr

extern "C" lr_status lr_matvec_train_workspace_size(const lr_points* query, const lr_points* source, int32_t nrhs,
                                                    size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_matvec_train_workspace_size: bytes is NULL");
  LR_REQUIRE(nrhs == 1, "lr_matvec_train_workspace_size: nrhs = %d; this version supports nrhs = 1", nrhs);
  TrainPlan T;
  lr_status st = plan_train(query, source, &T);
  if (st != LR_OK) return st;
  *bytes = T.bytes;
  return LR_OK;
}

extern "C" lr_status gp_kernel_matvec_train(const lr_points* query, const lr_points* source, const float* v,
                                            int32_t nrhs, float lengthscale, float variance, float* out,
                                            float* beta_out, float* moments_out, void* workspace,
                                            size_t workspace_bytes, lr_stream stream) {
  LR_REQUIRE(nrhs == 1, "gp_kernel_matvec_train: nrhs = %d; this version supports nrhs = 1", nrhs);
  TrainPlan T;
  lr_status st = plan_train(query, source, &T);
  if (st != LR_OK) return st;
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "gp_kernel_matvec_train: lengthscale must be > 0");
  LR_REQUIRE(isfinite(variance), "gp_kernel_matvec_train: variance is not finite");
  LR_REQUIRE(T.n == 0 || (out != nullptr && moments_out != nullptr),
             "gp_kernel_matvec_train: out and moments_out are required");
  LR_REQUIRE(v != nullptr || T.m == 0, "gp_kernel_matvec_train: v is NULL");
  LR_REQUIRE(beta_out == nullptr || T.q_raytrace || T.q_grid,
             "gp_kernel_matvec_train: beta_out needs a ray-traced or grid query");
  LR_REQUIRE(((uintptr_t)beta_out & 7u) == 0 && ((uintptr_t)out & 3u) == 0 && ((uintptr_t)moments_out & 3u) == 0,
             "gp_kernel_matvec_train: misaligned output");
  LR_REQUIRE(workspace_bytes >= T.bytes && (T.bytes == 0 || workspace != nullptr),
             "gp_kernel_matvec_train: workspace of %zu bytes, %zu needed", workspace_bytes, T.bytes);
  LR_REQUIRE(((uintptr_t)workspace & 255u) == 0, "gp_kernel_matvec_train: workspace must be 256-byte aligned");
  cudaStream_t s = as_cuda(stream);
  char* ws = static_cast<char*>(workspace);
  if (T.n == 0) return LR_OK;
  const float2* xq = reinterpret_cast<const float2*>(query->xy);
  if (T.q_raytrace || T.q_grid) {
    float2* qb = beta_out ? reinterpret_cast<float2*>(beta_out) : reinterpret_cast<float2*>(ws + T.off_qbeta);
    st = T.q_raytrace ? launch_raytrace(query, qb, nullptr, s) : launch_grid_points(query->grid, qb, s);
    if (st != LR_OK) return st;
    xq = qb;
  }
  if (T.m == 0) {
    LR_CHECK_CUDA(cudaMemsetAsync(out, 0, 4 * (size_t)T.n, s));
    LR_CHECK_CUDA(cudaMemsetAsync(moments_out, 0, 16 * (size_t)T.n, s));
    return LR_OK;
  }
  BwArgs A;
  MomMergeP MM;
  size_t b = 0;
  const float2* ys = T.s_grid ? nullptr : reinterpret_cast<const float2*>(source->xy);
  RowInfoP RI;
  st = make_train_problem(xq, T.n, query_layout(query), ys,
                          T.s_grid ? &source->grid : nullptr, T.m, v, lengthscale, variance, out, moments_out,
                          ws + T.off_rows, &A, &MM, &RI, &b);
  if (st != LR_OK) return st;
  if (RI.info && (st = launch_row_info(RI, s)) != LR_OK) return st;
  const unsigned grid = (unsigned)(row_block_count(A.map, T.n, A.rows_per_cta) * A.chunks);
  ktimer_begin(LR_KT_TRAIN_ROWS, s);
  if (T.s_grid && A.split)
    bwd_rows_kernel<true, false, false, true><<<grid, kBwThreads, 0, s>>>(A);
  else if (T.s_grid)
    bwd_rows_kernel<true, false, false><<<grid, kBwThreads, 0, s>>>(A);
  else
    bwd_rows_kernel<false, false, false><<<grid, kBwThreads, 0, s>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  ktimer_end(LR_KT_TRAIN_ROWS, s);
  moments_merge_kernel<<<(unsigned)((T.n + 255) / 256), 256, 0, s>>>(MM);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
