// Culled Gaussian-kernel reductions over explicit point sets (cull.cuh): the
// forward reduction out_i = var sum_j exp(-|x_i - y_j|^2 / (2 l^2)) v_j with
// up to four right-hand sides (Sec. 3.1 RBF kernel, Sec. 3.3 lazy T y), the
// row moments of the backward, the self-kernel backward (gradient flow
// through the reduction, Sec. 3.3 and 3.6), and the windowed transmission of
// the image-plane layers with its backward (Sec. 3.4, windows of Sec. 3.2).
//
// One CTA per (row block, group range). The CTA keeps its rows in registers
// and lists, in ascending order, the groups and then the chunks within reach
// of its bounding box. The listed chunks' record blocks are copied into
// shared memory by the bulk-copy engine (cp.async.bulk, completed through an
// mbarrier with a bounded wait), two batches in flight: the next batch lands
// while the warps work on the current one. Each warp then tests its own
// bounding box against the chunk's and skips chunks out of its reach.
// Per chunk a thread sums its rows' terms in plain FP32 (packed f32x2 over
// source pairs) and folds the chunk sums into its row totals (Kahan for the
// forward). The order of every sum is fixed by the problem alone.
#include <atomic>

#include "cull.cuh"
#include "host.cuh"

namespace lr {

namespace {

std::atomic<int> g_pair_culling{1};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ float4 box_merge(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

__device__ __forceinline__ float4 warp_box(float4 b) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    float4 t;
    t.x = __shfl_xor_sync(0xffffffffu, b.x, o);
    t.y = __shfl_xor_sync(0xffffffffu, b.y, o);
    t.z = __shfl_xor_sync(0xffffffffu, b.z, o);
    t.w = __shfl_xor_sync(0xffffffffu, b.w, o);
    b = box_merge(b, t);
  }
  return b;
}

constexpr float4 kEmptyBox = {INFINITY, INFINITY, -INFINITY, -INFINITY};

// ---------------------------------------------------------------------------
// Prepare: one warp per chunk (lane = slot) writes the chunk's box and record.
__global__ void __launch_bounds__(256) cull_prep_kernel(const __grid_constant__ CullPrepP P) {
  const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= P.L.n_chunks) return;  // warp-uniform
  const int64_t i = chunk_point(P.L, c, lane);
  const bool valid = i >= 0;
  const float2 pv = valid ? P.pts[i] : f2(0.f, 0.f);
  const float4 box = warp_box(valid ? make_float4(pv.x, pv.y, pv.x, pv.y) : kEmptyBox);
  // an empty slot sits at its chunk's box corner with weight 0
  const float2 p = valid ? pv : f2(box.x, box.y);
  const int RB = rec_bytes(P.nw);
  char* rec = P.rec + (int64_t)c * RB;
  if (lane == 0) P.cbox[c] = box;
  if (!(box.x <= box.z)) {  // an empty chunk: never within reach
    float* w = reinterpret_cast<float*>(rec);
    for (int k = lane; k < RB / 4; k += 32) w[k] = 0.f;
    __syncwarp();
    if (lane == 0) {
      *reinterpret_cast<float4*>(rec) = box;
      if (P.csc) P.csc[c] = INFINITY;
    }
    return;
  }
  const int n_valid = __popc(__ballot_sync(0xffffffffu, valid));
  // kCullWinCols: the points' window constants and the chunk's reach scale
  float wm[4] = {0.f, 0.f, 0.f, 0.f}, reach = INFINITY;
  if (P.kind == kCullWinCols && valid) {
    const float4 wc = P.wcoef[i];
    wm[0] = wc.x;
    wm[1] = wc.y;
    wm[2] = wc.z;
    wm[3] = P.a[i] * wc.w;
    reach = P.wreach[i];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) reach = fminf(reach, __shfl_xor_sync(0xffffffffu, reach, o));
  if (lane == 0) {
    *reinterpret_cast<float4*>(rec) = box;
    *reinterpret_cast<float4*>(rec + 16) = make_float4((float)n_valid, reach, 0.f, 0.f);
    if (P.csc) P.csc[c] = reach;
  }
  // (xa, xb, ya, yb) per source pair: absolute positions, so that the
  // kernels form x_j - x_i directly (correctly rounded: relative error u)
  float* xy = reinterpret_cast<float*>(rec + kRecHead);
  const int pr = lane >> 1, half = lane & 1;
  xy[4 * pr + half] = p.x;
  xy[4 * pr + 2 + half] = p.y;
  float* w = reinterpret_cast<float*>(rec + kRecHead + kRecXY);  // [nw][32], pairs consecutive
  if (P.kind == kCullOut) {
    for (int k = 0; k < P.nw; ++k) w[k * kChunkPts + lane] = valid ? P.a[i * P.stride + k] : 0.f;
  } else if (P.kind == kCullWin || P.kind == kCullWinRows) {
    w[lane] = valid ? P.a[i] : 0.f;
  } else if (P.kind == kCullWinCols) {
    for (int k = 0; k < 4; ++k) w[k * kChunkPts + lane] = wm[k];
  } else if (P.kind == kCullMom) {
    w[lane] = valid ? P.a[i * P.stride + P.col] : 0.f;
  } else {
    // self-kernel: the nrhs columns of a (v), then those of b (g)
    const int nr = P.nw / 2;
    for (int k = 0; k < nr; ++k) {
      w[k * kChunkPts + lane] = valid ? P.a[i * P.stride + k] : 0.f;
      w[(nr + k) * kChunkPts + lane] = valid ? P.b[i * P.stride + k] : 0.f;
    }
  }
}

// Window constants, one thread per point. C = Z + (l^2/2) I and det C are
// formed in FP64 (det cancels by a factor of the condition number); the rest
// is well-conditioned (products, quotients and square roots of positive
// numbers) and runs in FP32 from them: the upper Cholesky factor R of C^-1,
// r11 = sqrt(cyy / det), r12 = -cxy / sqrt(cyy det), r22 = 1 / sqrt(cyy), so
// that d^T C^-1 d = |R d|^2, and lambda_max(C) for the reach.
__global__ void __launch_bounds__(256) window_prep_kernel(const float* __restrict__ z, int64_t n, double half_s,
                                                          float4* __restrict__ wcoef, float* __restrict__ wreach) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double cxx_d = (double)z[3 * i] + half_s, cyy_d = (double)z[3 * i + 2] + half_s;
  const float cxy = z[3 * i + 1];
  const float det = (float)(cxx_d * cyy_d - (double)cxy * (double)cxy);
  const float cxx = (float)cxx_d, cyy = (float)cyy_d;
  const float k = 0.84932180028801904f;  // sqrt(log2(e) / 2)
  const float r11 = sqrtf(cyy / det), r12 = -cxy / sqrtf(cyy * det), r22 = 1.0f / sqrtf(cyy);
  wcoef[i] = make_float4(k * r11, k * r12, k * r22, 0.15915494309189535f / sqrtf(det));  // N = 1/(2 pi sqrt(det))
  const float h = 0.5f * (cxx - cyy);
  const float lmax = 0.5f * (cxx + cyy) + sqrtf(fmaf(h, h, cxy * cxy));
  wreach[i] = sqrtf(0.72134752044448170f / lmax);  // sqrt(log2(e) / (2 lambda_max))
}

// Group boxes (and, with csc, the groups' smallest reach scales): one warp
// per group.
__global__ void __launch_bounds__(256) cull_group_box_kernel(const float4* __restrict__ cbox,
                                                             const float* __restrict__ csc, int n_groups,
                                                             float4* __restrict__ gbox, float* __restrict__ gsc) {
  const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= n_groups) return;
  const int64_t c0 = (int64_t)g * kGroupChunks;
  float4 b = box_merge(cbox[c0 + lane], cbox[c0 + 32 + lane]);
  b = warp_box(b);
  if (lane == 0) gbox[g] = b;
  if (csc) {
    float r = fminf(csc[c0 + lane], csc[c0 + 32 + lane]);
#pragma unroll
    for (int o = 16; o; o >>= 1) r = fminf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) gsc[g] = r;
  }
}

// ---------------------------------------------------------------------------
// The sweep.
template <int KIND, int NW>
struct CullTraits;
template <int NW>
struct CullTraits<kCullOut, NW> {
  static constexpr int K = NW, R = NW <= 2 ? 4 : 2, BATCH = NW == 1 ? 48 : (NW == 2 ? 32 : 16);
};
template <>
struct CullTraits<kCullMom, 1> {
  static constexpr int K = 4, R = 2, BATCH = 32;
};
template <int NW>
struct CullTraits<kCullSelf, NW> {  // NW / 2 right-hand sides
  static constexpr int K = 7 * (NW / 2), R = NW == 2 ? 2 : 1, BATCH = NW == 2 ? 32 : 16;
};
template <>
struct CullTraits<kCullWin, 1> {
  static constexpr int K = 1, R = 4, BATCH = 32;
};
template <>
struct CullTraits<kCullWinRows, 1> {
  static constexpr int K = 6, R = 2, BATCH = 32;
};
template <>
struct CullTraits<kCullWinCols, 4> {
  static constexpr int K = 3, R = 4, BATCH = 16;
};

// Row outputs of one row (totals t[K]) for splits == 1, or of the merge.
// Returns the row's scalar-gradient terms (d_l, d_var) through sl, sv.
template <int KIND, int K>
__device__ __forceinline__ void cull_finalize(const CullArgs& A, int64_t i, const float* t, float& sl, float& sv) {
  sl = 0.f;
  sv = 0.f;
  if constexpr (KIND == kCullOut) {
#pragma unroll
    for (int k = 0; k < K; ++k) A.out[i * A.nrhs + k] = A.var * t[k];
  } else if constexpr (KIND == kCullWin) {
    float o = A.wcoef[i].w * t[0];
    if (A.lik_data) {
      // the likelihood epilogue: the model total and its residual
      if (A.f_in) o = A.f_in[i] + o;
      const float r = o - A.lik_data[i];
      A.lik_g[i] = r * A.lik_isig2;
      sl = 0.5f * (r * r) * A.lik_isig2;
    }
    A.out[i] = o;
  } else if constexpr (KIND == kCullMom) {
    if (A.g == nullptr) {
      A.out[i] = A.var * t[0];
#pragma unroll
      for (int k = 0; k < 4; ++k) A.mom[(int64_t)k * A.n + i] = t[k];
    } else {
      const float gi = A.g[i * A.stride + A.col];
      if (A.d_x) {
        float2 d = f2(A.dx_scale * gi * t[1], A.dx_scale * gi * t[2]);
        if (A.dx_accumulate) {
          const float2 o = A.d_x[i];
          d = f2(o.x + d.x, o.y + d.y);
        }
        A.d_x[i] = d;
      }
      sl = __fmul_rn(__fmul_rn(gi, t[3]), A.dl_scale);
      sv = __fmul_rn(gi, t[0]);
    }
  } else if constexpr (KIND == kCullSelf) {  // K / 7 right-hand sides, 7 sums each
    float dxx = 0.f, dxy = 0.f;
#pragma unroll
    for (int h = 0; h < K / 7; ++h) {
      const float gi = A.g[i * A.stride + h], vi = A.vrow[i * A.stride + h];
      const float* th = t + 7 * h;
      if (A.d_v) A.d_v[i * A.stride + h] = A.var * th[4];
      dxx = fmaf(gi, th[1], fmaf(vi, th[5], dxx));
      dxy = fmaf(gi, th[2], fmaf(vi, th[6], dxy));
      sl = fmaf(__fmul_rn(gi, th[3]), A.dl_scale, sl);
      sv = fmaf(gi, th[0], sv);
    }
    if (A.d_x) {
      float2 d = f2(A.dx_scale * dxx, A.dx_scale * dxy);
      if (A.dx_accumulate) {
        const float2 o = A.d_x[i];
        d = f2(o.x + d.x, o.y + d.y);
      }
      A.d_x[i] = d;
    }
  }
}

// Per-CTA FP64 partials of the two scalar gradients: FP32 per-row terms,
// FP32 warp sums, FP64 across the warps in order.
__device__ __forceinline__ void cta_scalar_partials(float sl, float sv, double* part, int64_t blk, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  if (lane == 0) {
    red[w] = sl;
    red[nw + w] = sv;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += (double)red[threadIdx.x * nw + k];
    part[blk * 2 + threadIdx.x] = t;
  }
}

constexpr int kMaxList = 1024;  // listed chunks per window

// Ordered compaction over the CTA: returns the number of true predicates;
// those threads write `value` to out[base + rank] in thread order.
__device__ __forceinline__ int cta_compact(bool pred, int value, int* out, int base, int* wcnt) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (lane == 0) wcnt[w] = __popc(m);
  __syncthreads();
  int off = base, total = 0;
#pragma unroll
  for (int k = 0; k < kCullThreads / 32; ++k) {
    if (k < w) off += wcnt[k];
    total += wcnt[k];
  }
  if (pred) out[off + __popc(m & ((1u << lane) - 1u))] = value;
  __syncthreads();
  return total;
}

template <int KIND, int NW>
struct CullSmem {
  static constexpr int BATCH = CullTraits<KIND, NW>::BATCH;
  alignas(128) char buf[2][BATCH * rec_bytes(NW)];
  uint64_t bar[2];
  float4 wbox[kCullThreads / 32];
  float wsc[kCullThreads / 32];
  int clist[kMaxList];
  int gsel[kCullThreads];
  int wcnt[kCullThreads / 32];
  float red[2 * kCullThreads / 32];
};

template <int KIND, int NW>
__global__ void __launch_bounds__(kCullThreads) cull_kernel(const __grid_constant__ CullArgs A) {
  using T = CullTraits<KIND, NW>;
  constexpr int R = T::R, K = T::K, BATCH = T::BATCH, RB = rec_bytes(NW);
  constexpr bool WROW = KIND == kCullWin || KIND == kCullWinRows;  // rows carry windows
  constexpr bool WBWD = KIND == kCullWinRows || KIND == kCullWinCols;
  __shared__ CullSmem<KIND, NW> sm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rb = blockIdx.x / A.splits, split = blockIdx.x - rb * A.splits;

  // rows
  float xr[R], yr[R];
  int64_t irow[R];
  float4 mybox = kEmptyBox;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    irow[r] = map_row(A.map, A.n, A.rows_per_cta, rb, tid * R + r);
    const float2 p = irow[r] >= 0 ? A.x[irow[r]] : f2(0.f, 0.f);
    xr[r] = p.x;
    yr[r] = p.y;
    if (irow[r] >= 0) mybox = box_merge(mybox, make_float4(p.x, p.y, p.x, p.y));
  }
  const float4 wb = warp_box(mybox);
  int warp_rows = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) warp_rows += __popc(__ballot_sync(0xffffffffu, irow[r] >= 0));
  float2 NQ[R], NP[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    NQ[r] = f2(-xr[r], -xr[r]);
    NP[r] = f2(-yr[r], -yr[r]);
  }
  const float2 NC = f2(-A.c, -A.c);
  // windowed rows: the scaled Cholesky factor (a, b, c) of C_i^-1 and the
  // reach scales of the skipping test (the smallest over the warp's and the
  // CTA's rows)
  float2 MA[R], MB[R], MC[R];
  float sc_w = A.sc, sc_b = A.sc;
  if constexpr (WROW) {
    float rs = INFINITY;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float a = 0.f, b = 0.f, c = 0.f;
      if (irow[r] >= 0) {
        const float4 wc = A.wcoef[irow[r]];
        a = wc.x;
        b = wc.y;
        c = wc.z;
        rs = fminf(rs, A.wreach[irow[r]]);
      }
      MA[r] = f2(a, a);
      MB[r] = f2(b, b);
      MC[r] = f2(c, c);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) rs = fminf(rs, __shfl_xor_sync(0xffffffffu, rs, o));
    sc_w = rs;
    if (lane == 0) sm.wsc[warp] = rs;
  }
  if (lane == 0) sm.wbox[warp] = wb;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
  }
  __syncthreads();
  float4 cb = sm.wbox[0];
#pragma unroll
  for (int k = 1; k < kCullThreads / 32; ++k) cb = box_merge(cb, sm.wbox[k]);
  if constexpr (WROW) {
    sc_b = sm.wsc[0];
#pragma unroll
    for (int k = 1; k < kCullThreads / 32; ++k) sc_b = fminf(sc_b, sm.wsc[k]);
  }
  const bool cull = A.cull != 0;

  float tot[R][K], comp[R][K];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      tot[r][k] = 0.f;
      comp[r][k] = 0.f;
    }

  uint32_t phases = 0u;  // bit k: parity of buffer k's next completion
  bool failed = false;
  const int g_lo = (int)((int64_t)split * A.n_groups / A.splits);
  const int g_hi = (int)((int64_t)(split + 1) * A.n_groups / A.splits);
  int gpos = g_lo;
  while (gpos < g_hi && !failed) {
    // ---- list the chunks within reach, in ascending order, up to kMaxList
    int count = 0;
    bool full = false;
    while (gpos < g_hi && !full) {
      const int g = gpos + tid;
      const bool gs = g < g_hi && !(cull && boxes_far(cb, A.gbox[g], KIND == kCullWinCols ? A.gsc[g] : sc_b));
      const int ng = cta_compact(gs, g, sm.gsel, 0, sm.wcnt);
      int k = 0;
      for (; k < ng; ++k) {
        if (count + kGroupChunks > kMaxList) break;
        const int gg = sm.gsel[k];
        const int c = gg * kGroupChunks + (tid & (kGroupChunks - 1));
        const bool cs = tid < kGroupChunks &&
                        !(cull ? boxes_far(cb, A.cbox[c], KIND == kCullWinCols ? A.csc[c] : sc_b)
                               : !(A.cbox[c].x <= A.cbox[c].z));
        count += cta_compact(cs, c, sm.clist, count, sm.wcnt);
      }
      if (k < ng) {
        gpos = sm.gsel[k];
        full = true;
      } else {
        gpos = min(gpos + kCullThreads, g_hi);
      }
      __syncthreads();  // gsel is rewritten by the next window
    }
    // ---- stream the listed chunks through shared memory, two batches in flight
    const int nb = (count + BATCH - 1) / BATCH;
    auto issue = [&](int b) {
      const int c0 = b * BATCH, cn = min(BATCH, count - c0);
      char* dst = sm.buf[b & 1];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&sm.bar[b & 1], (uint32_t)(cn * RB));
      for (int k = 0; k < cn; ++k) bulk_g2s(dst + k * RB, A.rec + (int64_t)sm.clist[c0 + k] * RB, RB, &sm.bar[b & 1]);
    };
    if (tid == 0 && nb > 0) issue(0);
    for (int b = 0; b < nb; ++b) {
      if (tid == 0 && b + 1 < nb) issue(b + 1);
      const uint32_t ph = (phases >> (b & 1)) & 1u;
      const bool ok = mbar_wait_bounded(&sm.bar[b & 1], ph, A.fault);
      if (__syncthreads_or(!ok)) {
        failed = true;
        // copies may still be in flight into either buffer: wait for them
        // once more (bounded) before the CTA gives up its shared memory
        if (!ok) mbar_wait_bounded(&sm.bar[b & 1], ph, nullptr);
        if (b + 1 < nb) mbar_wait_bounded(&sm.bar[(b + 1) & 1], (phases >> ((b + 1) & 1)) & 1u, nullptr);
        break;
      }
      phases ^= 1u << (b & 1);
      const int cn = min(BATCH, count - b * BATCH);
      const char* bb = sm.buf[b & 1];
      for (int k = 0; k < cn; ++k) {
        const char* rec = bb + k * RB;
        const float4 box = *reinterpret_cast<const float4*>(rec);
        const float4 head = *reinterpret_cast<const float4*>(rec + 16);  // (valid points, reach scale)
        if (cull && boxes_far(wb, box, KIND == kCullWinCols ? head.y : sc_w)) continue;  // warp-uniform
        if (A.count && lane == 0) {
          const float nv = head.x;
          atomicAdd(A.count, (unsigned long long)(warp_rows * (int)nv));
          atomicAdd(A.count + 1, (unsigned long long)(32 * R * kChunkPts));
        }
        const float4* xy = reinterpret_cast<const float4*>(rec + kRecHead);
        const float2* wt = reinterpret_cast<const float2*>(rec + kRecHead + kRecXY);
        if constexpr (KIND == kCullOut) {
          // k v = 2^(-c |x_j - x_i|^2) v, c = sc^2: 6 FP32 lanes per pair
          float2 acc[R][NW];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int w = 0; w < NW; ++w) acc[r][w] = f2(0.f, 0.f);
#pragma unroll 4
          for (int pp = 0; pp < kChunkPairs; ++pp) {
            const float4 P = xy[pp];
            const float2 X = f2(P.x, P.y), Y = f2(P.z, P.w);
            float2 W[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) W[w] = wt[w * kChunkPairs + pp];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const float2 dx = __fadd2_rn(X, NQ[r]), dy = __fadd2_rn(Y, NP[r]);
              const float2 e = __fmul2_rn(__ffma2_rn(dy, dy, __fmul2_rn(dx, dx)), NC);
              const float2 kk = f2(ex2_approx(e.x), ex2_approx(e.y));
#pragma unroll
              for (int w = 0; w < NW; ++w) acc[r][w] = __ffma2_rn(kk, W[w], acc[r][w]);
            }
          }
          // fold the chunk's sums into the row totals (only nonzero ones, so
          // that a chunk left out and a chunk of exact zeros agree bitwise)
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int w = 0; w < NW; ++w) {
              const float sum = acc[r][w].x + acc[r][w].y;
              if (sum != 0.f) kahan_add(tot[r][w], comp[r][w], sum);
            }
        } else if constexpr (KIND == kCullWin) {
          // G' v = 2^(-|w|^2) v, w = (a d_x + b d_y, c d_y), d = x_j - x_i:
          // 8 FP32 lanes per pair
          float2 acc[R];
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] = f2(0.f, 0.f);
#pragma unroll 2
          for (int pp = 0; pp < kChunkPairs; ++pp) {
            const float4 P = xy[pp];
            const float2 X = f2(P.x, P.y), Y = f2(P.z, P.w);
            const float2 W = wt[pp];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const float2 dx = __fadd2_rn(X, NQ[r]), dy = __fadd2_rn(Y, NP[r]);
              const float2 w1 = __ffma2_rn(MA[r], dx, __fmul2_rn(MB[r], dy)), w2 = __fmul2_rn(MC[r], dy);
              const float2 t = __ffma2_rn(w1, w1, __fmul2_rn(w2, w2));
              const float2 kk = f2(ex2_approx(-t.x), ex2_approx(-t.y));
              acc[r] = __ffma2_rn(kk, W, acc[r]);
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float sum = acc[r].x + acc[r].y;
            if (sum != 0.f) kahan_add(tot[r][0], comp[r][0], sum);
          }
        } else if constexpr (KIND == kCullWinRows) {
          // with w = R_i d (scaled), d = x_j - x_i and u = R_i^T w =
          // k^2 C_i^-1 d (= M'_i (x_i - x_j) with M' = -k^2 C^-1, the merge's
          // form): S += v G', P += v G' u, Q += v G' u u^T
          float2 acc[R][6];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k2 = 0; k2 < 6; ++k2) acc[r][k2] = f2(0.f, 0.f);
#pragma unroll 2
          for (int pp = 0; pp < kChunkPairs; ++pp) {
            const float4 P = xy[pp];
            const float2 X = f2(P.x, P.y), Y = f2(P.z, P.w);
            const float2 W = wt[pp];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const float2 dx = __fadd2_rn(X, NQ[r]), dy = __fadd2_rn(Y, NP[r]);
              const float2 w1 = __ffma2_rn(MA[r], dx, __fmul2_rn(MB[r], dy)), w2 = __fmul2_rn(MC[r], dy);
              const float2 t = __ffma2_rn(w1, w1, __fmul2_rn(w2, w2));
              const float2 ux = __fmul2_rn(MA[r], w1), uy = __ffma2_rn(MB[r], w1, __fmul2_rn(MC[r], w2));
              const float2 kv = __fmul2_rn(f2(ex2_approx(-t.x), ex2_approx(-t.y)), W);
              const float2 kx = __fmul2_rn(kv, ux), ky = __fmul2_rn(kv, uy);
              float2* a = acc[r];
              a[0] = __fadd2_rn(a[0], kv);
              a[1] = __fadd2_rn(a[1], kx);
              a[2] = __fadd2_rn(a[2], ky);
              a[3] = __ffma2_rn(kx, ux, a[3]);
              a[4] = __ffma2_rn(kx, uy, a[4]);
              a[5] = __ffma2_rn(ky, uy, a[5]);
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k2 = 0; k2 < 6; ++k2) tot[r][k2] += acc[r][k2].x + acc[r][k2].y;
        } else if constexpr (KIND == kCullWinCols) {
          // the sources carry the windows: with w = R_j d (scaled),
          // d = x_j - x_i and u = R_j^T w = k^2 C_j^-1 d (= M'_j (x_i - x_j)):
          // T += gN G', U += gN G' u
          float2 acc[R][3];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) acc[r][k2] = f2(0.f, 0.f);
#pragma unroll 2
          for (int pp = 0; pp < kChunkPairs; ++pp) {
            const float4 P = xy[pp];
            const float2 X = f2(P.x, P.y), Y = f2(P.z, P.w);
            const float2 ca = wt[pp], cb = wt[kChunkPairs + pp], cc = wt[2 * kChunkPairs + pp],
                         gn = wt[3 * kChunkPairs + pp];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const float2 dx = __fadd2_rn(X, NQ[r]), dy = __fadd2_rn(Y, NP[r]);
              const float2 w1 = __ffma2_rn(ca, dx, __fmul2_rn(cb, dy)), w2 = __fmul2_rn(cc, dy);
              const float2 t = __ffma2_rn(w1, w1, __fmul2_rn(w2, w2));
              const float2 kg = __fmul2_rn(f2(ex2_approx(-t.x), ex2_approx(-t.y)), gn);
              const float2 ux = __fmul2_rn(ca, w1), uy = __ffma2_rn(cb, w1, __fmul2_rn(cc, w2));
              float2* a = acc[r];
              a[0] = __fadd2_rn(a[0], kg);
              a[1] = __ffma2_rn(kg, ux, a[1]);
              a[2] = __ffma2_rn(kg, uy, a[2]);
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) tot[r][k2] += acc[r][k2].x + acc[r][k2].y;
        } else {
          // row moments from per-pair differences d = x_j - x_i:
          // A += k w, B += k w d, C += k w |d|^2 (and A, B of the second
          // weight for the self-kernel). Differences, not moments about a
          // reference point: a pair at d ~ 0 (the row's own point) adds
          // nothing to B and C instead of two large terms that cancel.
          constexpr int NRH = KIND == kCullSelf ? NW / 2 : 1;  // right-hand sides
          constexpr int NA = KIND == kCullSelf ? 7 * NRH : 4;
          float2 acc[R][NA];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k2 = 0; k2 < NA; ++k2) acc[r][k2] = f2(0.f, 0.f);
#pragma unroll 2
          for (int pp = 0; pp < kChunkPairs; ++pp) {
            const float4 P = xy[pp];
            const float2 X = f2(P.x, P.y), Y = f2(P.z, P.w);
            float2 W[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) W[w] = wt[w * kChunkPairs + pp];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              // the pair's distance and exp2 once, for every right-hand side
              const float2 dx = __fadd2_rn(X, NQ[r]), dy = __fadd2_rn(Y, NP[r]);
              const float2 t = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
              const float2 e = __fmul2_rn(t, NC);
              const float2 kk = f2(ex2_approx(e.x), ex2_approx(e.y));
#pragma unroll
              for (int h = 0; h < NRH; ++h) {
                float2* a = acc[r] + 7 * h;
                const float2 kw = __fmul2_rn(kk, W[h]);
                a[0] = __fadd2_rn(a[0], kw);
                a[1] = __ffma2_rn(kw, dx, a[1]);
                a[2] = __ffma2_rn(kw, dy, a[2]);
                a[3] = __ffma2_rn(kw, t, a[3]);
                if (KIND == kCullSelf) {
                  const float2 kg = __fmul2_rn(kk, W[NRH + h]);
                  a[4] = __fadd2_rn(a[4], kg);
                  a[5] = __ffma2_rn(kg, dx, a[5]);
                  a[6] = __ffma2_rn(kg, dy, a[6]);
                }
              }
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k2 = 0; k2 < NA; ++k2) tot[r][k2] += acc[r][k2].x + acc[r][k2].y;
        }
    
      }
      __syncthreads();  // the buffer is refilled two batches on
    }
  }
  if (failed || A.count) return;

  // ---- outputs
  float sl = 0.f, sv = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (irow[r] < 0) continue;
    float t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = (KIND == kCullOut || KIND == kCullWin) ? tot[r][k] - comp[r][k] : tot[r][k];
    if constexpr (WBWD) {
#pragma unroll
      for (int k = 0; k < K; ++k) A.partial[((int64_t)split * K + k) * A.n + irow[r]] = t[k];
    } else if (A.splits == 1) {
      float a, b;
      cull_finalize<KIND, K>(A, irow[r], t, a, b);
      sl += a;
      sv += b;
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) A.partial[((int64_t)split * K + k) * A.n + irow[r]] = t[k];
    }
  }
  if (A.splits == 1 && A.scal_part) cta_scalar_partials(sl, sv, A.scal_part, blockIdx.x, sm.red);
}

// Fixed-order merge of the group-range partials [splits][K][n], then the
// outputs as the sweep would have written them.
template <int KIND, int K>
__global__ void __launch_bounds__(256) cull_merge_kernel(const __grid_constant__ CullArgs A) {
  __shared__ float red[16];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float sl = 0.f, sv = 0.f;
  if (i < A.n) {
    float t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float s = 0.f, c = 0.f;
      for (int sp = 0; sp < A.splits; ++sp) kahan_add(s, c, A.partial[((int64_t)sp * K + k) * A.n + i]);
      t[k] = s - c;
    }
    cull_finalize<KIND, K>(A, i, t, sl, sv);
  }
  if (A.scal_part) cta_scalar_partials(sl, sv, A.scal_part, blockIdx.x, red);
}

// Fixed-order FP64 sum of scalar partials [nblk][2] into d_len, d_var.
__global__ void __launch_bounds__(256) cull_scalar_final_kernel(const double* __restrict__ part, int64_t nblk,
                                                                double* d_len, double* d_var) {
  __shared__ double red[2][8];
  double a = 0.0, b = 0.0;
  for (int64_t k = threadIdx.x; k < nblk; k += 256) {
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
    for (int w = 0; w < 8; ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    if (d_len) *d_len = sa;
    if (d_var) *d_var = sb;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

int cull_enabled() { return g_pair_culling.load(std::memory_order_relaxed); }

template <int KIND, int NW>
static const void* cull_fn() {
  return reinterpret_cast<const void*>(&cull_kernel<KIND, NW>);
}

static const void* cull_kernel_ptr(int kind, int nw) {
  if (kind == kCullOut) {
    switch (nw) {
      case 1: return cull_fn<kCullOut, 1>();
      case 2: return cull_fn<kCullOut, 2>();
      case 3: return cull_fn<kCullOut, 3>();
      default: return cull_fn<kCullOut, 4>();
    }
  }
  if (kind == kCullMom) return cull_fn<kCullMom, 1>();
  if (kind == kCullWin) return cull_fn<kCullWin, 1>();
  if (kind == kCullWinRows) return cull_fn<kCullWinRows, 1>();
  if (kind == kCullWinCols) return cull_fn<kCullWinCols, 4>();
  switch (nw) {
    case 2: return cull_fn<kCullSelf, 2>();
    case 4: return cull_fn<kCullSelf, 4>();
    case 6: return cull_fn<kCullSelf, 6>();
    default: return cull_fn<kCullSelf, 8>();
  }
}

static int cull_rows_per_thread(int kind, int nw) {
  if (kind == kCullOut) return nw <= 2 ? 4 : 2;
  if (kind == kCullWin || kind == kCullWinCols) return 4;
  return (kind == kCullSelf && nw > 2) ? 1 : 2;
}

lr_status plan_cull(int kind, int nrhs, int64_t n, const lr_grid* qlayout, int64_t m, const lr_grid* slayout,
                    CullPlan* out) {
  CullPlan P{};
  P.kind = kind;
  P.nw = cull_nw(kind, nrhs);
  P.L = make_chunk_layout(slayout, m);
  P.rows_per_cta = kCullThreads * cull_rows_per_thread(kind, P.nw);
  if (qlayout) {
    P.map.W = qlayout->nx * qlayout->ss;
    P.map.H = qlayout->ny * qlayout->ss;
    P.map.tw = kCullTileW;
    P.map.th = P.rows_per_cta / kCullTileW;
    P.map.TW = (P.map.W + P.map.tw - 1) / P.map.tw;
    P.map.TH = (P.map.H + P.map.th - 1) / P.map.th;
  }
  P.row_blocks = row_block_count(P.map, n, P.rows_per_cta);
  int dev = 0, n_sm = 1, occ = 1;
  LR_CHECK_CUDA(cudaGetDevice(&dev));
  LR_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  LR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cull_kernel_ptr(kind, P.nw), kCullThreads, 0));
  // group ranges per row block: only when the row blocks alone leave most of
  // the resident CTA slots empty (small query sets). Windowed points differ
  // in reach by orders of magnitude (pixels next to the lens centre reach
  // arcseconds, half the image), so the work of a row block does too: there
  // many more group ranges spread the heaviest row blocks over the GPU.
  const int64_t slots = (int64_t)(occ > 0 ? occ : 1) * n_sm;
  // (measured on the 400 x 400 image: 48 for the sweeps whose rows carry the
  // windows, 16 for the column sweep, against 2 for the stationary sweeps)
  const int64_t target = (kind == kCullWin || kind == kCullWinRows) ? 48 * slots
                         : kind == kCullWinCols                       ? 16 * slots
                                                                      : 2 * slots;
  int64_t splits = 1;
  if (P.row_blocks > 0 && P.row_blocks < target) splits = (target + P.row_blocks - 1) / P.row_blocks;
  if (splits > P.L.n_groups) splits = P.L.n_groups > 0 ? P.L.n_groups : 1;
  P.splits = (int32_t)splits;
  P.K = cull_k(kind, P.nw);
  const bool wbwd = kind == kCullWinRows || kind == kCullWinCols;
  size_t off = 0;
  P.off_rec = off;
  off += align256((size_t)P.L.n_chunks * rec_bytes(P.nw));
  P.off_cbox = off;
  off += align256(sizeof(float4) * (size_t)P.L.n_chunks);
  P.off_gbox = off;
  off += align256(sizeof(float4) * (size_t)(P.L.n_groups > 0 ? P.L.n_groups : 1));
  P.off_csc = P.off_gsc = off;
  if (kind == kCullWinCols) {
    off += align256(sizeof(float) * (size_t)P.L.n_chunks);
    P.off_gsc = off;
    off += align256(sizeof(float) * (size_t)(P.L.n_groups > 0 ? P.L.n_groups : 1));
  }
  P.off_partial = off;
  if (P.splits > 1 || wbwd) off += align256(sizeof(float) * (size_t)P.splits * P.K * (size_t)n);
  P.scal_blocks = P.splits > 1 ? (n + 255) / 256 : P.row_blocks * P.splits;
  P.off_scal = off;
  off += align256(sizeof(double) * 2 * (size_t)(P.scal_blocks > 0 ? P.scal_blocks : 1));
  P.bytes = off;
  *out = P;
  return LR_OK;
}

lr_status launch_window_prep(const float* z, int64_t n, float lengthscale, float4* wcoef, float* wreach,
                             cudaStream_t s) {
  if (n == 0) return LR_OK;
  const double ell = (double)lengthscale;
  window_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, n, 0.5 * ell * ell, wcoef, wreach);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

lr_status launch_cull_prep(const CullPlan& P, const float2* pts, float sc, const float* a, const float* b,
                           int32_t stride, int32_t col, char* ws, cudaStream_t s, const float4* wcoef,
                           const float* wreach) {
  CullPrepP Q{};
  Q.pts = pts;
  Q.L = P.L;
  Q.sc = sc;
  Q.kind = P.kind;
  Q.nw = P.nw;
  Q.a = a;
  Q.b = b;
  Q.stride = stride;
  Q.col = col;
  Q.rec = ws + P.off_rec;
  Q.cbox = reinterpret_cast<float4*>(ws + P.off_cbox);
  Q.gbox = reinterpret_cast<float4*>(ws + P.off_gbox);
  Q.wcoef = wcoef;
  Q.wreach = wreach;
  if (P.kind == kCullWinCols) {
    Q.csc = reinterpret_cast<float*>(ws + P.off_csc);
    Q.gsc = reinterpret_cast<float*>(ws + P.off_gsc);
  }
  if (P.L.n_chunks == 0) return LR_OK;
  const int64_t warps = P.L.n_chunks;
  cull_prep_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(Q);
  LR_CHECK_CUDA(cudaGetLastError());
  cull_group_box_kernel<<<(unsigned)(((int64_t)P.L.n_groups * 32 + 255) / 256), 256, 0, s>>>(
      Q.cbox, Q.csc, P.L.n_groups, Q.gbox, Q.gsc);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

template <int KIND, int NW>
static lr_status launch_sweep_t(const CullPlan& P, const CullArgs& A, cudaStream_t s) {
  const unsigned grid = (unsigned)(P.row_blocks * P.splits);
  cull_kernel<KIND, NW><<<grid, kCullThreads, 0, s>>>(A);
  LR_CHECK_CUDA(cudaGetLastError());
  // the windowed backward kinds leave their partials to the caller's merge
  if constexpr (KIND != kCullWinRows && KIND != kCullWinCols) {
    if (P.splits > 1 && !A.count) {
      cull_merge_kernel<KIND, CullTraits<KIND, NW>::K><<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A);
      LR_CHECK_CUDA(cudaGetLastError());
    }
  }
  return LR_OK;
}

lr_status launch_cull_sweep(const CullPlan& P, CullArgs A, char* ws, int timer_id, cudaStream_t s) {
  if (P.row_blocks == 0) return LR_OK;
  A.map = P.map;
  A.rows_per_cta = P.rows_per_cta;
  A.cull = cull_enabled();
  A.rec = ws + P.off_rec;
  A.cbox = reinterpret_cast<const float4*>(ws + P.off_cbox);
  A.gbox = reinterpret_cast<const float4*>(ws + P.off_gbox);
  A.n_chunks = P.L.n_chunks;
  A.n_groups = P.L.n_groups;
  A.splits = P.splits;
  A.partial = reinterpret_cast<float*>(ws + P.off_partial);
  if (P.kind == kCullWinCols) {
    A.csc = reinterpret_cast<const float*>(ws + P.off_csc);
    A.gsc = reinterpret_cast<const float*>(ws + P.off_gsc);
  }
  A.fault = fault_ptr();
  LR_REQUIRE(A.fault != nullptr, "could not resolve the device fault word");
  if (timer_id >= 0) ktimer_begin(timer_id, s);
  lr_status st;
  if (P.kind == kCullOut) {
    switch (P.nw) {
      case 1: st = launch_sweep_t<kCullOut, 1>(P, A, s); break;
      case 2: st = launch_sweep_t<kCullOut, 2>(P, A, s); break;
      case 3: st = launch_sweep_t<kCullOut, 3>(P, A, s); break;
      default: st = launch_sweep_t<kCullOut, 4>(P, A, s); break;
    }
  } else if (P.kind == kCullMom) {
    st = launch_sweep_t<kCullMom, 1>(P, A, s);
  } else if (P.kind == kCullWin) {
    st = launch_sweep_t<kCullWin, 1>(P, A, s);
  } else if (P.kind == kCullWinRows) {
    st = launch_sweep_t<kCullWinRows, 1>(P, A, s);
  } else if (P.kind == kCullWinCols) {
    st = launch_sweep_t<kCullWinCols, 4>(P, A, s);
  } else {
    switch (P.nw) {
      case 2: st = launch_sweep_t<kCullSelf, 2>(P, A, s); break;
      case 4: st = launch_sweep_t<kCullSelf, 4>(P, A, s); break;
      case 6: st = launch_sweep_t<kCullSelf, 6>(P, A, s); break;
      default: st = launch_sweep_t<kCullSelf, 8>(P, A, s); break;
    }
  }
  if (timer_id >= 0) ktimer_end(timer_id, s);
  return st;
}

lr_status launch_cull_scalar_final(const double* part, int64_t nblk, double* d_len, double* d_var, cudaStream_t s) {
  if (!d_len && !d_var) return LR_OK;
  cull_scalar_final_kernel<<<1, 256, 0, s>>>(part, nblk, d_len, d_var);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

}  // namespace lr

extern "C" lr_status lr_set_pair_culling(int32_t enable) {
  lr::g_pair_culling.store(enable ? 1 : 0, std::memory_order_relaxed);
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: pairs the culled sweeps evaluate.
using namespace lr;

extern "C" lr_status lr_cull_pairs_evaluated(const lr_points* query, const lr_points* source, float lengthscale,
                                             int32_t sweep, int64_t* pairs, int64_t* slots, lr_stream stream) {
  lr_status st = validate_points(query, "lr_cull_pairs_evaluated(query)", false);
  if (st != LR_OK) return st;
  if (source) {
    st = validate_points(source, "lr_cull_pairs_evaluated(source)", false);
    if (st != LR_OK) return st;
    LR_REQUIRE(source->xy != nullptr || has_lens(source),
               "lr_cull_pairs_evaluated: grid sources take the grid sweeps (lr_grid_pairs_evaluated)");
  }
  LR_REQUIRE(pairs != nullptr, "lr_cull_pairs_evaluated: pairs is NULL");
  LR_REQUIRE(sweep == 0 || sweep == 1, "lr_cull_pairs_evaluated: sweep = %d (0 forward, 1 backward)", sweep);
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "lr_cull_pairs_evaluated: lengthscale must be > 0");
  cudaStream_t s = as_cuda(stream);
  const bool self = source == nullptr;
  const int64_t n = query->n, m = self ? n : source->n;
  *pairs = 0;
  if (slots) *slots = 0;
  if (n == 0 || m == 0) return LR_OK;
  const lr_grid* ql = query_layout(query);
  const lr_grid* sl = self ? ql : query_layout(source);
  const int kind = sweep == 0 ? kCullOut : (self ? kCullSelf : kCullMom);
  CullPlan P;
  st = plan_cull(kind, 1, n, ql, m, sl, &P);
  if (st != LR_OK) return st;
  // temporaries: points, zero weights, workspace, counters
  const size_t b_q = align256(8 * (size_t)n), b_s = align256(8 * (size_t)m), b_w = align256(4 * (size_t)m);
  char* buf = nullptr;
  LR_CHECK_CUDA(cudaMalloc(&buf, b_q + b_s + b_w + P.bytes + 256));
  auto done = [&](lr_status r) {
    cudaFree(buf);
    return r;
  };
  float2* xq = reinterpret_cast<float2*>(buf);
  float2* ys = reinterpret_cast<float2*>(buf + b_q);
  float* w = reinterpret_cast<float*>(buf + b_q + b_s);
  char* ws = buf + b_q + b_s + b_w;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ws + P.bytes);
  if (has_lens(query))
    st = launch_raytrace(query, xq, nullptr, s);
  else if (query->xy == nullptr)
    st = launch_grid_points(query->grid, xq, s);
  else if (cudaMemcpyAsync(xq, query->xy, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    st = cuda_status(cudaGetLastError(), "cudaMemcpyAsync");
  if (st != LR_OK) return done(st);
  const float2* src = xq;
  if (!self) {
    if (has_lens(source))
      st = launch_raytrace(source, ys, nullptr, s);
    else if (cudaMemcpyAsync(ys, source->xy, 8 * (size_t)m, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      st = cuda_status(cudaGetLastError(), "cudaMemcpyAsync");
    if (st != LR_OK) return done(st);
    src = ys;
  }
  if (cudaMemsetAsync(w, 0, 4 * (size_t)m, s) != cudaSuccess || cudaMemsetAsync(cnt, 0, 16, s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "cudaMemsetAsync"));
  const double c = 1.4426950408889634 / (2.0 * (double)lengthscale * (double)lengthscale);
  st = launch_cull_prep(P, src, (float)sqrt(c), w, w, 1, 0, ws, s);
  if (st != LR_OK) return done(st);
  CullArgs A{};
  A.x = xq;
  A.n = n;
  A.sc = (float)sqrt(c);
  A.c = (float)c;
  A.nrhs = 1;
  A.stride = 1;
  A.count = cnt;
  st = launch_cull_sweep(P, A, ws, -1, s);
  if (st != LR_OK) return done(st);
  unsigned long long h[2] = {0, 0};
  if (cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "lr_cull_pairs_evaluated"));
  *pairs = (int64_t)h[0];
  if (slots) *slots = (int64_t)h[1];
  return done(LR_OK);
}
