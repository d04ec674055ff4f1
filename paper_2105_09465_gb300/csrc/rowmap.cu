// Row-block boxes and active source-tile ranges (see rowmap.cuh), single and
// batched.
#include "host.cuh"
#include "problems.cuh"

namespace lr {

__global__ void __launch_bounds__(kRowPrepThreads) row_info_kernel(const float2* __restrict__ x, int64_t n,
                                                                   RowMap map, int rows_per_cta, GridDev g,
                                                                   int32_t segs, float sc,
                                                                   RowBlockInfo* __restrict__ info) {
  row_block_info_body(x, n, map, rows_per_cta, g, segs, sc, blockIdx.x, info);
}

__global__ void __launch_bounds__(kRowPrepThreads) row_info_batched_kernel(const __grid_constant__ Batch<RowInfoP> B) {
  const int k = batch_find(B, blockIdx.x);
  const RowInfoP& P = B.p[k];
  row_block_info_body(P.x, P.n, P.map, P.rows_per_cta, P.g, P.segs, P.sc, blockIdx.x - B.start[k], P.info);
}

lr_status launch_row_info(const RowInfoP& P, cudaStream_t s) {
  const int64_t nb = row_block_count(P.map, P.n, P.rows_per_cta);
  if (nb == 0) return LR_OK;
  row_info_kernel<<<(unsigned)nb, kRowPrepThreads, 0, s>>>(P.x, P.n, P.map, P.rows_per_cta, P.g, P.segs, P.sc,
                                                            P.info);
  LR_CHECK_CUDA(cudaGetLastError());
  return LR_OK;
}

lr_status launch_row_info_batched(const RowInfoP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<RowInfoP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += row_block_count(p[b0 + k].map, p[b0 + k].n, p[b0 + k].rows_per_cta);
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    row_info_batched_kernel<<<(unsigned)tot, kRowPrepThreads, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

}  // namespace lr

namespace lr {

// Pairs the grid-source kernels evaluate for one row-block layout: per row
// block, its valid rows times, over the active tile range, the source columns
// of the source pairs that meet the reachable columns (the kernels' own
// tests: reach_cols and seg_pair_range per sub-segment).
__global__ void __launch_bounds__(kRowPrepThreads) pair_count_kernel(const float2* __restrict__ x, int64_t n,
                                                                     RowMap map, int rows_per_cta, GridDev g,
                                                                     int32_t segs, int32_t tile,
                                                                     float sc, const RowBlockInfo* __restrict__ info,
                                                                     unsigned long long* __restrict__ count) {
  const int64_t rb = blockIdx.x;
  const RowBlockInfo B = info[rb];
  unsigned long long rows = 0, cols = 0;
  for (int w = threadIdx.x; w < rows_per_cta; w += kRowPrepThreads)
    rows += map_row(map, n, rows_per_cta, rb, w) >= 0 ? 1ull : 0ull;
  for (int t = B.t_lo + (int)threadIdx.x; t < B.t_hi; t += kRowPrepThreads) {
    const int grow = t / segs, c0 = (t - grow * segs) * tile;
    const int cnt = min(tile, g.W - c0);
    const float y = grid_y(g, grow);
    int lo, hi;
    reach_cols(B, g, y, sc, c0, cnt, lo, hi);
    for (int s0 = 0; s0 < cnt; s0 += kSplitSeg) {
      int pl, ph;
      seg_pair_range<kSplitSeg>(lo, hi, s0, pl, ph);
      // the kernels evaluate source pairs pl .. ph - 1, whole quarters of the
      // sub-segment (a pair past the tile's last column is padding and
      // counts nothing)
      if (pl < ph) cols += (unsigned long long)(min(s0 + 2 * ph, cnt) - (s0 + 2 * pl));
    }
  }
  for (int o = 16; o; o >>= 1) {
    rows += __shfl_xor_sync(0xffffffffu, rows, o);
    cols += __shfl_xor_sync(0xffffffffu, cols, o);
  }
  __shared__ unsigned long long r2[kRowPrepThreads / 32], c2[kRowPrepThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    r2[threadIdx.x >> 5] = rows;
    c2[threadIdx.x >> 5] = cols;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long R = 0, C = 0;
    for (int k = 0; k < kRowPrepThreads / 32; ++k) {
      R += r2[k];
      C += c2[k];
    }
    atomicAdd(count, R * C);
  }
}

}  // namespace lr

using namespace lr;

extern "C" lr_status lr_grid_pairs_evaluated(const float* x, int64_t n, const lr_grid* query_grid,
                                             const lr_grid* source_grid, float lengthscale, int32_t rows_per_cta,
                                             int64_t* pairs, lr_stream stream) {
  LR_REQUIRE(pairs && source_grid && (x || n == 0), "lr_grid_pairs_evaluated: NULL argument");
  LR_REQUIRE(rows_per_cta > 0 && rows_per_cta % kRowTileW == 0, "lr_grid_pairs_evaluated: bad rows_per_cta %d",
             rows_per_cta);
  LR_REQUIRE(isfinite(lengthscale) && lengthscale > 0.f, "lr_grid_pairs_evaluated: lengthscale must be > 0");
  *pairs = 0;
  if (n == 0) return LR_OK;
  const RowMap map = query_grid ? make_row_map(query_grid, rows_per_cta) : RowMap{};
  LR_REQUIRE(!query_grid || (int64_t)map.W * map.H == n, "lr_grid_pairs_evaluated: n != query grid points");
  const GridDev g = grid_dev(*source_grid);
  const int32_t segs = (g.W + 255) / 256;
  const float sc = (float)sqrt(1.4426950408889634 / (2.0 * (double)lengthscale * (double)lengthscale));
  const int64_t nb = row_block_count(map, n, rows_per_cta);
  cudaStream_t s = as_cuda(stream);
  void* buf = nullptr;
  LR_CHECK_CUDA(cudaMalloc(&buf, sizeof(RowBlockInfo) * (size_t)nb + 256));
  RowBlockInfo* info = static_cast<RowBlockInfo*>(buf);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + sizeof(RowBlockInfo) * nb);
  lr_status st = LR_OK;
  RowInfoP P{reinterpret_cast<const float2*>(x), n, map, rows_per_cta, segs, g, sc, info};
  if (cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s) != cudaSuccess ||
      (st = launch_row_info(P, s)) != LR_OK) {
    cudaFree(buf);
    return st != LR_OK ? st : cuda_status(cudaGetLastError(), "cudaMemsetAsync");
  }
  pair_count_kernel<<<(unsigned)nb, kRowPrepThreads, 0, s>>>(reinterpret_cast<const float2*>(x), n, map,
                                                              rows_per_cta, g, segs, 256, sc, info, cnt);
  unsigned long long h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_status(e, "lr_grid_pairs_evaluated");
  *pairs = (int64_t)h;
  return LR_OK;
}
