// PageRank (Sec. V, the PR benchmark) on the consolidated row-gather kernels.
//
// Power iteration in pull form over the in-edge CSR:
//   rank_{t+1}(v) = (1-d)/n + d * ( D_t/n + sum over in-edges (u,v) of rank_t(u)/outdeg(u) )
// with D_t the rank held by vertices without out-edges (spread uniformly).
// The per-vertex sum over in-edges is the irregular loop: a vertex with more
// in-edges than the threshold is large work, handed to a child kernel at the
// call's level exactly as an SpMV row is (spmv.cu, kModeRank). This file holds
// the two kernels around it: the initial uniform vector and the per-iteration
// prep (contributions, dangling mass, teleport term).
#include "dpc_internal.h"
#include "dpc_runtime.cuh"
#include "rank_reduce.cuh"

namespace dpc {

namespace {

__global__ void __launch_bounds__(256) rank_init_kernel(float *rank, int n, float r0) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) rank[v] = r0;
}

// Contributions and the dangling rank in the fixed shape of rank_reduce.cuh:
// warps take 1,024-vertex chunks; the last block to finish adds the chunk sums
// with one warp, writes the teleport term and resets the counters the gather
// of this iteration uses (the previous gather and its children have finished,
// in stream order).
__global__ void __launch_bounds__(kRankPrepThreads) rank_prep_kernel(RankPrepParams q) {
  const int chunks = ceil_div(q.n, kRankChunk);
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int W = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < chunks; c += W) {
    const float sc = rank_chunk(q.rank_in, q.outdeg, q.contrib, q.n, c);
    if (lane_id() == 0) q.partials[c] = sc;
  }
  if (last_block_done(&q.hdr->done_blocks) && threadIdx.x < kWarp) {
    const float D = rank_total(q.partials, chunks);
    if (threadIdx.x == 0) {
      *q.beta = teleport_term(q.damping, D, q.n);
      q.hdr->cursor = 0;
      q.hdr->done_blocks2 = 0;
      q.hdr->launches = 0;
      for (int c = 0; c < kUnitCursors; ++c) q.hdr->cursors[c * kCursorStride] = 0;  // the child's unit cursors
      if (q.stats) atomicMax(&q.stats->rounds, (unsigned)q.iteration + 1u);
      __threadfence();
    }
  }
}

}  // namespace

cudaError_t rank_init(float *rank, int n, cudaStream_t s) {
  const int blocks = (n + 255) / 256 < kRankPrepBlocks ? (n + 255) / 256 : kRankPrepBlocks;
  rank_init_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(rank, n, 1.f / (float)n);
  return cudaGetLastError();
}

cudaError_t rank_prep(const RankPrepParams &q, cudaStream_t s) {
  // one warp per 1,024-vertex chunk
  const int need = ceil_div(ceil_div(q.n, kRankChunk), kRankPrepThreads / kWarp);
  const int blocks = need < kRankPrepBlocks ? (need > 0 ? need : 1) : kRankPrepBlocks;
  rank_prep_kernel<<<blocks, kRankPrepThreads, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace dpc
