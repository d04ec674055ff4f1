// Inducing-point density by the k-th nearest neighbour (Sec. 3.4, footnote to
// the factorisation of the covariance) and the transmission weights it sets:
//   rho(q_i) = k / (pi r_k(q_i)^2),  A_i = |2 pi Sigma|^(1/4) / sqrt(rho)
//                                        = pi l sqrt(2 r_k^2 / k)   (Sigma = l^2 I).
// r_k is the distance to the k-th closest OTHER point (excluded by index).
//
// Uniform cell grid over the bounding box (about two points per cell),
// counting sort of the points by cell, then one thread per point (in cell
// order, so a warp works on one neighbourhood) grows square rings of cells
// until k candidates are held and the k-th squared distance is inside the
// ring radius; the k smallest are kept sorted in registers. The result is the
// k-th smallest FP32 squared distance, independent of visiting order.
#include <math.h>

#include "host.cuh"

namespace lr {

constexpr int kKnnMax = 32;
constexpr int kScanBlock = 1024;
constexpr int kBoxBlocks = 256;
constexpr int kMaxCellsPerAxis = 8192;

struct KnnHdr {
  float x0, y0, inv_h, h;
  int32_t gx, gy, pad0, pad1;
};

struct KnnLayout {
  size_t hdr, box, cell, count, cursor, totals, pts, idx, bytes;
  int64_t cmax, nblk;
};

static KnnLayout knn_layout(int64_t m) {
  KnnLayout L{};
  L.cmax = m / 2 + 1;
  L.nblk = (L.cmax + 1 + kScanBlock - 1) / kScanBlock;
  size_t o = 0;
  L.hdr = o;
  o = align256(o + sizeof(KnnHdr));
  L.box = o;
  o = align256(o + sizeof(float4) * kBoxBlocks);
  L.cell = o;
  o = align256(o + 4 * (size_t)m);
  L.count = o;
  o = align256(o + 4 * (size_t)(L.cmax + 1));
  L.cursor = o;
  o = align256(o + 4 * (size_t)L.cmax);
  L.totals = o;
  o = align256(o + 4 * (size_t)L.nblk);
  L.pts = o;
  o = align256(o + 8 * (size_t)m);
  L.idx = o;
  o = align256(o + 4 * (size_t)m);
  L.bytes = o;
  return L;
}

__device__ __forceinline__ float4 box_merge(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

__device__ __forceinline__ float4 box_block_reduce(float4 b) {
  __shared__ float4 part[32];
  for (int o = 16; o; o >>= 1) {
    float4 t;
    t.x = __shfl_xor_sync(0xffffffffu, b.x, o);
    t.y = __shfl_xor_sync(0xffffffffu, b.y, o);
    t.z = __shfl_xor_sync(0xffffffffu, b.z, o);
    t.w = __shfl_xor_sync(0xffffffffu, b.w, o);
    b = box_merge(b, t);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = b;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    b = l < nw ? part[l] : make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
    for (int o = 16; o; o >>= 1) {
      float4 t;
      t.x = __shfl_xor_sync(0xffffffffu, b.x, o);
      t.y = __shfl_xor_sync(0xffffffffu, b.y, o);
      t.z = __shfl_xor_sync(0xffffffffu, b.z, o);
      t.w = __shfl_xor_sync(0xffffffffu, b.w, o);
      b = box_merge(b, t);
    }
  }
  return b;  // valid in thread 0
}

__global__ void knn_box_kernel(const float2* __restrict__ q, int64_t m, float4* __restrict__ box) {
  float4 b = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 p = q[i];
    b = box_merge(b, make_float4(p.x, p.y, p.x, p.y));
  }
  b = box_block_reduce(b);
  if (threadIdx.x == 0) box[blockIdx.x] = b;
}

// Cell side h for about two points per cell, grown until the grid fits the
// workspace (gx * gy <= cmax) and each axis has at most kMaxCellsPerAxis
// cells (which keeps the FP32 cell coordinate error far below a cell).
__global__ void knn_plan_kernel(const float4* __restrict__ box, int nbox, int64_t m, int64_t cmax,
                                KnnHdr* __restrict__ hdr) {
  float4 b = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
  for (int i = threadIdx.x; i < nbox; i += blockDim.x) b = box_merge(b, box[i]);
  b = box_block_reduce(b);
  if (threadIdx.x != 0) return;
  const double ex = (double)b.z - (double)b.x, ey = (double)b.w - (double)b.y;
  const double target = (double)(m / 2 > 0 ? m / 2 : 1);
  double h;
  if (ex > 0.0 && ey > 0.0)
    h = sqrt(ex * ey / target);
  else
    h = fmax(ex, ey) / target;
  int64_t gx = 1, gy = 1;
  if (h > 0.0 && isfinite(h)) {
    for (int it = 0; it < 4096; ++it) {
      gx = (int64_t)floor(ex / h) + 1;
      gy = (int64_t)floor(ey / h) + 1;
      if (gx <= kMaxCellsPerAxis && gy <= kMaxCellsPerAxis && gx * gy <= cmax) break;
      h *= 1.0625;
    }
    if (!(gx <= kMaxCellsPerAxis && gy <= kMaxCellsPerAxis && gx * gy <= cmax)) gx = gy = 1;
  } else {
    h = 1.0;
  }
  KnnHdr H;
  H.x0 = b.x;
  H.y0 = b.y;
  H.h = (float)h;
  H.inv_h = (float)(1.0 / h);
  H.gx = (int32_t)gx;
  H.gy = (int32_t)gy;
  H.pad0 = H.pad1 = 0;
  *hdr = H;
}

__device__ __forceinline__ int cell_coord(float u, int g) {
  int c = (int)u;  // u >= 0 up to rounding; NaN converts to 0
  return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

__global__ void knn_count_kernel(const float2* __restrict__ q, int64_t m, const KnnHdr* __restrict__ hdr,
                                 int32_t* __restrict__ cell, int32_t* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const KnnHdr H = *hdr;
  const float2 p = q[i];
  const int cx = cell_coord((p.x - H.x0) * H.inv_h, H.gx), cy = cell_coord((p.y - H.y0) * H.inv_h, H.gy);
  const int c = cy * H.gx + cx;
  cell[i] = c;
  atomicAdd(count + c, 1);
}

// Exclusive scan of count[0..n) in place, in three passes.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int wsum[32];
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  if (l == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = l < (int)(blockDim.x >> 5) ? wsum[l] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (l >= o) s += y;
    }
    wsum[l] = s;
  }
  __syncthreads();
  const int incl = x + (w > 0 ? wsum[w - 1] : 0);
  *total = wsum[(blockDim.x >> 5) - 1];
  return incl - v;
}

__global__ void __launch_bounds__(kScanBlock) knn_scan_blocks(int32_t* __restrict__ a, int64_t n,
                                                              int32_t* __restrict__ totals) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int v = i < n ? a[i] : 0;
  int tot;
  const int ex = block_exclusive_scan(v, &tot);
  if (i < n) a[i] = ex;
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) knn_scan_totals(int32_t* __restrict__ totals, int64_t nb) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int64_t i = b0 + threadIdx.x;
    const int v = i < nb ? totals[i] : 0;
    int tot;
    const int ex = block_exclusive_scan(v, &tot);
    const int c = carry;
    if (i < nb) totals[i] = ex + c;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanBlock) knn_scan_add(int32_t* __restrict__ a, int64_t n,
                                                           const int32_t* __restrict__ totals) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) a[i] += totals[blockIdx.x];
}

__global__ void knn_scatter_kernel(const float2* __restrict__ q, int64_t m, const int32_t* __restrict__ cell,
                                   const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                                   float2* __restrict__ pts, int32_t* __restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int c = cell[i];
  const int at = start[c] + atomicAdd(cursor + c, 1);
  pts[at] = q[i];
  idx[at] = (int32_t)i;
}

// The k smallest values seen sit at the top of the ascending list best[]:
// best[0 .. kKnnMax-k) hold -inf for good and best[kKnnMax-k .. kKnnMax) the
// k smallest, so the k-th smallest is always best[kKnnMax-1] (a static index,
// which keeps the list in registers). Inserting a value below it by a
// compare-exchange chain drops the old maximum and leaves the -inf padding
// in place.
__device__ __forceinline__ float topk_insert(float (&best)[kKnnMax], float d2) {
#pragma unroll
  for (int j = 0; j < kKnnMax; ++j) {
    const float lo = fminf(best[j], d2), hi = fmaxf(best[j], d2);
    best[j] = lo;
    d2 = hi;
  }
  return best[kKnnMax - 1];
}

__global__ void __launch_bounds__(128) knn_query_kernel(const float2* __restrict__ pts, const int32_t* __restrict__ idx,
                                                        int64_t m, int32_t k, const int32_t* __restrict__ start,
                                                        const KnnHdr* __restrict__ hdr, float a_scale,
                                                        float* __restrict__ r2_out, float* __restrict__ a_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const KnnHdr H = *hdr;
  const float2 p = pts[t];
  const int32_t self = idx[t];
  const int cx = cell_coord((p.x - H.x0) * H.inv_h, H.gx), cy = cell_coord((p.y - H.y0) * H.inv_h, H.gy);
  float best[kKnnMax];
#pragma unroll
  for (int j = 0; j < kKnnMax; ++j) best[j] = j < kKnnMax - k ? -INFINITY : INFINITY;
  float kth = INFINITY;
  int have = 0;
  const int rmax = max(H.gx, H.gy);
  for (int r = 0; r <= rmax; ++r) {
    const int y0 = max(cy - r, 0), y1 = min(cy + r, H.gy - 1);
    for (int y = y0; y <= y1; ++y) {
      const bool edge_row = (y == cy - r) || (y == cy + r);
      const int step = edge_row ? 1 : 2 * r;
      for (int x = cx - r; x <= cx + r; x += (step > 0 ? step : 1)) {
        if (x < 0 || x >= H.gx) continue;
        const int c = y * H.gx + x;
        const int j1 = start[c + 1];
        for (int j = start[c]; j < j1; ++j) {
          if (idx[j] == self) continue;
          const float2 o = pts[j];
          const float dx = p.x - o.x, dy = p.y - o.y;
          const float d2 = fmaf(dx, dx, dy * dy);
          ++have;
          if (d2 < kth) kth = topk_insert(best, d2);
        }
      }
    }
    // every unvisited point is at least (r - margin) cells away
    const float reach = fmaxf((float)r - 0.01f, 0.f) * H.h;
    if (have >= k && kth <= reach * reach) break;
  }
  if (r2_out) r2_out[self] = kth;
  if (a_out) a_out[self] = a_scale * sqrtf(kth);
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_knn_workspace_size(int64_t m, size_t* bytes) {
  LR_REQUIRE(bytes != nullptr, "lr_knn_workspace_size: bytes is NULL");
  LR_REQUIRE(m >= 0 && m < (int64_t(1) << 31), "lr_knn_workspace_size: m out of range");
  *bytes = knn_layout(m).bytes;
  return LR_OK;
}

extern "C" lr_status gp_knn_density(const float* q, int64_t m, int32_t k, float lengthscale, float* r2_out,
                                    float* a_out, void* workspace, size_t workspace_bytes, lr_stream stream) {
  LR_REQUIRE(k >= 1 && k <= kKnnMax, "gp_knn_density: k = %d outside [1, %d]", k, kKnnMax);
  LR_REQUIRE(m >= (int64_t)k + 1 && m < (int64_t(1) << 31),
             "gp_knn_density: %lld points cannot have a %d-th other neighbour", (long long)m, k);
  LR_REQUIRE(q != nullptr && ((uintptr_t)q & 7u) == 0, "gp_knn_density: q NULL or not 8-byte aligned");
  LR_REQUIRE(r2_out != nullptr || a_out != nullptr, "gp_knn_density: no output requested");
  LR_REQUIRE(a_out == nullptr || (isfinite(lengthscale) && lengthscale > 0.f),
             "gp_knn_density: lengthscale must be > 0 for the weights");
  const KnnLayout L = knn_layout(m);
  LR_REQUIRE(workspace != nullptr && workspace_bytes >= L.bytes && ((uintptr_t)workspace & 255u) == 0,
             "gp_knn_density: workspace of %zu bytes (256-byte aligned) needed, %zu given", L.bytes,
             workspace_bytes);
  cudaStream_t s = as_cuda(stream);
  char* w = static_cast<char*>(workspace);
  KnnHdr* hdr = reinterpret_cast<KnnHdr*>(w + L.hdr);
  float4* box = reinterpret_cast<float4*>(w + L.box);
  int32_t* cell = reinterpret_cast<int32_t*>(w + L.cell);
  int32_t* count = reinterpret_cast<int32_t*>(w + L.count);
  int32_t* cursor = reinterpret_cast<int32_t*>(w + L.cursor);
  int32_t* totals = reinterpret_cast<int32_t*>(w + L.totals);
  float2* pts = reinterpret_cast<float2*>(w + L.pts);
  int32_t* idx = reinterpret_cast<int32_t*>(w + L.idx);
  const float2* q2 = reinterpret_cast<const float2*>(q);
  const unsigned nb = (unsigned)((m + 255) / 256);
  const int64_t nbox_want = (m + 255) / 256;
  const unsigned nbox = (unsigned)(nbox_want < kBoxBlocks ? nbox_want : kBoxBlocks);

  LR_CHECK_CUDA(cudaMemsetAsync(count, 0, 4 * (size_t)(L.cmax + 1), s));
  LR_CHECK_CUDA(cudaMemsetAsync(cursor, 0, 4 * (size_t)L.cmax, s));
  knn_box_kernel<<<nbox, 256, 0, s>>>(q2, m, box);
  knn_plan_kernel<<<1, 256, 0, s>>>(box, (int)nbox, m, L.cmax, hdr);
  knn_count_kernel<<<nb, 256, 0, s>>>(q2, m, hdr, cell, count);
  knn_scan_blocks<<<(unsigned)L.nblk, kScanBlock, 0, s>>>(count, L.cmax + 1, totals);
  knn_scan_totals<<<1, kScanBlock, 0, s>>>(totals, L.nblk);
  knn_scan_add<<<(unsigned)L.nblk, kScanBlock, 0, s>>>(count, L.cmax + 1, totals);
  knn_scatter_kernel<<<nb, 256, 0, s>>>(q2, m, cell, count, cursor, pts, idx);
  // A = pi l sqrt(2 r^2 / k)
  const float a_scale = (float)(3.14159265358979323846 * (double)lengthscale * sqrt(2.0 / (double)k));
  knn_query_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(pts, idx, m, k, count, hdr, a_scale, r2_out, a_out);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}
