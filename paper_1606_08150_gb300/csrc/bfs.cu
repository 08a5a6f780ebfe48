// Recursive breadth-first search (Sec. V, BFS-Rec) at the consolidation levels.
//
// The recursion of Fig. 1(c) on a graph: visiting vertex v at depth d relaxes
// every out-edge (v, u) with atomicMin(level[u], d + 1); a neighbour whose
// level dropped, and that has out-edges of its own, is visited recursively at
// depth d + 1. Vertices without out-edges are finished inline. The levels
// settle on the breadth-first hop distances whatever order the visits run in:
// a visit that finds its vertex already lowered by another path is stale and
// returns at once, and the path that lowered it visits it again.
//   basic-DP  one child grid per recursive visit (thread per out-edge).
//   warp/block/grid
//             recursive visits are appended, as (vertex, chunk of out-edges)
//             units, to the buffer of the warp, block or grid; one child per
//             buffer visits them all at depth d + 1. Warp and block buffers
//             recurse independently (a vertex may be reached first by a longer
//             path and visited again later); the grid buffer is level-
//             synchronous: generation d holds exactly the vertices at hop
//             distance d, so every vertex is visited once.
//   flat      host-driven level-synchronous BFS, thread per frontier vertex.
//   queue     the grid level as one cooperative grid: a generation, a grid
//             barrier whose last arriver publishes the next generation's
//             extent, the next generation, ... with no device launch.
// A child grid processes its units in rounds of one unit per warp; each round
// ends with the scope's buffer reservation (one atomic per warp, block or
// warp of the grid level) and, at warp and block level, the scope's launch.
#include "dpc_internal.h"
#include "dpc_runtime.cuh"

namespace dpc {

namespace {

constexpr unsigned kInfLevel = 0xFFFFFFFFu;
constexpr int kEdgesPerLane = kBfsMaxChunk / kWarp;  // one unit: at most 8 out-edges per lane

__device__ __forceinline__ void bfs_fail(const BfsParams &p, unsigned code) {
  set_status(&p.hdr->status, code);
  if (p.stats) atomicCAS(&p.stats->status, 0u, code);
}

__device__ __forceinline__ int units_of(const BfsParams &p, int deg) { return deg > 0 ? ceil_div(deg, p.chunk) : 0; }

// The calling lane's out-edges of unit u (edges a + lane + 32 q, q < 8) at
// depth `depth`: relax them and report, per edge slot, the neighbour to visit
// next (or -1) and its unit count. Returns the lane's total of new units.
__device__ __forceinline__ int relax_unit(const BfsParams &p, int2 u, unsigned depth, int cand[kEdgesPerLane],
                                          int nu[kEdgesPerLane], unsigned long long &scanned) {
  int mine = 0;
#pragma unroll
  for (int q = 0; q < kEdgesPerLane; ++q) {
    cand[q] = -1;
    nu[q] = 0;
  }
  if (u.x < 0) return 0;  // placeholder written after a buffer overflow
  if (__ldcg(p.level + u.x) != depth) return 0;  // stale: a shorter path reached the vertex since
  const int a = __ldg(p.off + u.x) + u.y * p.chunk;
  const int b = min(__ldg(p.off + u.x + 1), a + p.chunk);
  const int lane = lane_id();
  const unsigned nd = depth + 1;
  int w[kEdgesPerLane];
#pragma unroll
  for (int q = 0; q < kEdgesPerLane; ++q) {
    const int e = a + lane + q * kWarp;
    w[q] = -1;
    if (e < b) {
      w[q] = checked_index(__ldg(p.col + e), p.n, &p.hdr->status);
      ++scanned;
    }
  }
  unsigned cur[kEdgesPerLane];
#pragma unroll
  for (int q = 0; q < kEdgesPerLane; ++q) cur[q] = w[q] >= 0 ? __ldcg(p.level + w[q]) : 0u;
#pragma unroll
  for (int q = 0; q < kEdgesPerLane; ++q)
    if (w[q] >= 0 && nd < cur[q] && nd < atomicMin(p.level + w[q], nd)) cand[q] = w[q];
#pragma unroll
  for (int q = 0; q < kEdgesPerLane; ++q)
    if (cand[q] >= 0) {
      nu[q] = units_of(p, __ldg(p.off + cand[q] + 1) - __ldg(p.off + cand[q]));
      if (nu[q] == 0) cand[q] = -1;  // no out-edge: finished inline
      mine += nu[q];
    }
  return mine;
}

// Write the lane's new units at pos, pos+1, ...
__device__ __forceinline__ void write_units(const BfsParams &p, const int cand[kEdgesPerLane],
                                            const int nu[kEdgesPerLane], int pos) {
#pragma unroll
  for (int q = 0; q < kEdgesPerLane; ++q)
    for (int j = 0; j < nu[q]; ++j) p.units[pos++] = make_int2(cand[q], j);
}

__device__ __forceinline__ void count_stats(const BfsParams &p, unsigned long long scanned, unsigned long long buf,
                                            unsigned depth) {
  if (!p.stats) return;
  scanned = warp_sum(scanned);
  buf = warp_sum(buf);
  if (lane_id() == 0) {
    stat_add(p.stats, &dpc_stats::relaxations, scanned);
    stat_add(p.stats, &dpc_stats::buffered_items, buf);
    if (scanned) atomicMax(&p.stats->rounds, depth + 1u);
  }
}

}  // namespace

// ------------------------------------------------------------------ basic-DP

// Visit of one vertex: thread per out-edge; every neighbour whose level
// dropped and that has out-edges gets its own recursive child grid.
__global__ void __launch_bounds__(1024) bfs_visit_vertex(BfsParams p, int v, unsigned depth) {
  if (__ldcg(p.level + v) != depth) return;  // stale
  const int a = __ldg(p.off + v), b = __ldg(p.off + v + 1);
  const unsigned nd = depth + 1;
  unsigned long long launched = 0, failed = 0, scanned = 0;
  for (int e = a + blockIdx.x * blockDim.x + threadIdx.x; e < b; e += gridDim.x * blockDim.x) {
    scanned++;
    const int u = checked_index(__ldg(p.col + e), p.n, &p.hdr->status);
    if (kCheckedBuild && u < 0) continue;
    if (!(nd < __ldcg(p.level + u) && nd < atomicMin(p.level + u, nd))) continue;
    const int deg = __ldg(p.off + u + 1) - __ldg(p.off + u);
    if (deg == 0) continue;
    bool ok = false;
    if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
      __threadfence();
      bfs_visit_vertex<<<ceil_div(deg, p.child_threads), p.child_threads, 0, cudaStreamFireAndForget>>>(p, u, nd);
      ok = cudaGetLastError() == cudaSuccess;
      if (!ok) bfs_fail(p, DPC_ERR_DEVICE);
    } else {
      bfs_fail(p, DPC_ERR_DEVICE);
    }
    if (ok) launched++;
    else failed++;
  }
  if (p.stats) {
    launched = warp_sum(launched);
    failed = warp_sum(failed);
    scanned = warp_sum(scanned);
    if (lane_id() == 0) {
      stat_add(p.stats, &dpc_stats::child_launches, launched);
      stat_add(p.stats, &dpc_stats::buffered_items, launched + failed);
      stat_add(p.stats, &dpc_stats::launch_failures, failed);
      stat_add(p.stats, &dpc_stats::relaxations, scanned);
      if (scanned) atomicMax(&p.stats->rounds, depth + 1u);
    }
  }
}

// ------------------------------------------------------------------ consolidated

// Visit the units [0, nunits) of `units` at depth `depth`, rounds of one unit
// per warp. Neighbours to visit next go to the buffer of the warp, block or
// grid; see the file comment.
template <int LEVEL>
__global__ void __launch_bounds__(1024) bfs_visit(BfsParams p, const int2 *__restrict__ units, int nunits,
                                                 unsigned depth) {
  __shared__ int s_scan[33];
  __shared__ unsigned long long s_base;
  const int lane = lane_id();
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int W = gridDim.x * wpb;
  // a negative count: the root's units, counted on the device by bfs_root
  if (nunits < 0) nunits = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[0]);
  unsigned long long scanned = 0, buf = 0;
  for (int r0 = 0; r0 < nunits; r0 += W) {
    const int ui = r0 + gw;
    int cand[kEdgesPerLane], nu[kEdgesPerLane];
    const int mine = relax_unit(p, ui < nunits ? units[ui] : make_int2(-1, 0), depth, cand, nu, scanned);
    // reserve the scope's slice: one atomic per block (block level) or per warp;
    // the check is made on the 64-bit cursor (revisits make its total data-dependent)
    int excl, total;
    unsigned long long base64 = 0;
    if (LEVEL == DPC_BLOCK) {
      excl = block_exclusive_scan(mine, s_scan, &total);
      if (threadIdx.x == 0) s_base = total ? atomicAdd(&p.hdr->cursor, (unsigned long long)total) : 0ull;
      __syncthreads();
      base64 = s_base;
    } else {
      const int inc = warp_inclusive_scan(mine);
      excl = inc - mine;
      total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
      unsigned long long b0 = 0;
      if (lane == kWarp - 1 && total) b0 = atomicAdd(&p.hdr->cursor, (unsigned long long)total);
      base64 = __shfl_sync(0xffffffffu, b0, kWarp - 1);
    }
    const int base = (int)min(base64, (unsigned long long)p.max_units);
    if (total && base64 + (unsigned long long)total > (unsigned long long)p.max_units) {
      if (lane == 0) bfs_fail(p, DPC_ERR_OVERFLOW);
      total = 0;
    } else if (mine) {
      write_units(p, cand, nu, base + excl);
      buf += (unsigned long long)mine;
    }
    // the scope's barrier and its launch (warp and block level)
    if (LEVEL == DPC_WARP || LEVEL == DPC_BLOCK) {
      __threadfence();
      if (LEVEL == DPC_WARP) __syncwarp();
      else __syncthreads();
      const bool leader = LEVEL == DPC_WARP ? lane == 0 : threadIdx.x == 0;
      if (leader && total) {
        bool ok = false;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          bfs_visit<LEVEL><<<child_grid_for(total, p.child_blocks, p.child_threads), p.child_threads, 0,
                             cudaStreamFireAndForget>>>(p, p.units + base, total, depth + 1);
          ok = cudaGetLastError() == cudaSuccess;
        }
        if (ok) {
          stat_add(p.stats, &dpc_stats::child_launches, 1);
        } else {
          bfs_fail(p, DPC_ERR_DEVICE);
          stat_add(p.stats, &dpc_stats::launch_failures, 1);
        }
      }
    }
  }
  count_stats(p, scanned, buf, depth);
  if (LEVEL == DPC_GRID) {
    // generation depth+1 is exactly the units reserved after this one began
    if (last_block_done(&p.hdr->done_blocks) && threadIdx.x == 0) {
      const long long end = (long long)min(*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                                           (unsigned long long)p.max_units);
      const long long start = (long long)(units - p.units) + nunits;
      if (end > start) {
        const int n = (int)(end - start);
        bool ok = false;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          bfs_visit<DPC_GRID><<<child_grid_for(n, p.child_blocks, p.child_threads), p.child_threads, 0,
                                cudaStreamFireAndForget>>>(p, p.units + start, n, depth + 1);
          ok = cudaGetLastError() == cudaSuccess;
        }
        if (ok) {
          stat_add(p.stats, &dpc_stats::child_launches, 1);
        } else {
          bfs_fail(p, DPC_ERR_DEVICE);
          stat_add(p.stats, &dpc_stats::launch_failures, 1);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ queue level

namespace {

// Multi-use barrier of a cooperative grid. Arrival counts only grow, so the
// k-th barrier of a call is complete once k * gridDim.x blocks have arrived;
// the block arriving last publishes the buffer's end before it releases the
// others. Bounded wait; false (and DPC_ERR_TIMEOUT) when it runs out.
__device__ bool generation_barrier(const BfsParams &p, unsigned k, unsigned long long *snap) {
  __shared__ int s_ok;
  __shared__ unsigned long long s_snap;
  __syncthreads();  // orders the block's writes before its master thread's fence and arrival
  if (threadIdx.x == 0) {
    __threadfence();
    int ok = 1;
    const unsigned target = k * gridDim.x;
    if (atomicAdd(&p.hdr->done_blocks2, 1u) == target - 1) {
      p.hdr->aux[1] = *reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor);
      __threadfence();
      atomicExch(&p.hdr->round, k);
    } else {
      WaitClock clk;
      while (*reinterpret_cast<volatile unsigned *>(&p.hdr->round) < k) {
        __nanosleep(64);
        if (clk.expired()) {
          bfs_fail(p, DPC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_snap = *reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[1]);
    s_ok = ok;
  }
  __syncthreads();
  *snap = s_snap;
  return s_ok != 0;
}

}  // namespace

__global__ void __launch_bounds__(1024) bfs_queue(BfsParams p) {
  const int lane = lane_id();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int W = (gridDim.x * blockDim.x) >> 5;
  long long lo = 0, hi = (long long)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[0]);
  unsigned depth = 0;
  unsigned long long scanned = 0, buf = 0;
  for (unsigned k = 1; lo < hi; ++k, ++depth) {
    for (long long ui = lo + gw; ui < hi; ui += W) {
      int cand[kEdgesPerLane], nu[kEdgesPerLane];
      const int mine = relax_unit(p, p.units[ui], depth, cand, nu, scanned);
      const int inc = warp_inclusive_scan(mine);
      const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
      unsigned long long b0 = 0;
      if (lane == kWarp - 1 && total) b0 = atomicAdd(&p.hdr->cursor, (unsigned long long)total);
      const unsigned long long base64 = __shfl_sync(0xffffffffu, b0, kWarp - 1);
      if (total && base64 + (unsigned long long)total > (unsigned long long)p.max_units) {
        if (lane == 0) bfs_fail(p, DPC_ERR_OVERFLOW);
      } else if (mine) {
        write_units(p, cand, nu, (int)base64 + inc - mine);
        buf += (unsigned long long)mine;
      }
    }
    unsigned long long end = 0;
    if (!generation_barrier(p, k, &end)) return;
    lo = hi;
    hi = (long long)min(end, (unsigned long long)p.max_units);
  }
  count_stats(p, scanned, buf, depth > 0 ? depth - 1 : 0);
}

// ------------------------------------------------------------------ set-up and flat

__global__ void bfs_fill(BfsParams p) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += gridDim.x * blockDim.x)
    p.level[v] = v == p.source ? 0u : kInfLevel;
}

// The source's units at the head of the buffer (consolidated and queue levels).
__global__ void bfs_root(BfsParams p) {
  const int deg = p.off[p.source + 1] - p.off[p.source];
  const int nu = units_of(p, deg);
  for (int j = threadIdx.x; j < nu; j += blockDim.x) p.units[j] = make_int2(p.source, j);
  if (threadIdx.x == 0) {
    p.hdr->cursor = (unsigned long long)nu;
    p.hdr->aux[0] = (unsigned long long)nu;
  }
}

// Flat: one level of a host-driven level-synchronous BFS, thread per frontier
// vertex over all its out-edges; newly reached vertices form the next frontier.
__global__ void __launch_bounds__(1024) bfs_flat_level(BfsParams p, const int *frontier, int nf, int *next,
                                                      unsigned depth) {
  const unsigned nd = depth + 1;
  unsigned long long scanned = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const int v = frontier[i];
    const int a = __ldg(p.off + v), b = __ldg(p.off + v + 1);
    scanned += (unsigned long long)(b - a);
    for (int e = a; e < b; ++e) {
      const int u = checked_index(__ldg(p.col + e), p.n, &p.hdr->status);
      if (kCheckedBuild && u < 0) continue;
      if (nd < __ldcg(p.level + u) && nd < atomicMin(p.level + u, nd)) {
        const unsigned long long pos = atomicAdd(&p.hdr->cursor2, 1ull);
        next[pos] = u;
      }
    }
  }
  if (p.stats) {
    scanned = warp_sum(scanned);
    if (lane_id() == 0) {
      stat_add(p.stats, &dpc_stats::relaxations, scanned);
      if (scanned) atomicMax(&p.stats->rounds, depth + 1u);
    }
  }
}

// ------------------------------------------------------------------ host side

size_t bfs_max_units(int n, int m, int chunk, dpc_level level) {
  // level-synchronous levels visit every vertex once: sum of ceil(deg/chunk) <= m/chunk + n;
  // warp and block recursion may visit a vertex again after a shorter path is found
  const size_t once = (size_t)m / (size_t)chunk + (size_t)n + 1;
  return (level == DPC_WARP || level == DPC_BLOCK) ? 4 * once + 1024 : once;
}

size_t bfs_workspace_bytes(int n, int m, dpc_level level, int chunk) {
  size_t b = kHeaderBytes;
  if (level == DPC_FLAT) return b + 2 * align_up((size_t)n * sizeof(int), 256);
  if (level == DPC_BASIC_DP) return b;
  return b + align_up(bfs_max_units(n, m, chunk, level) * sizeof(int2), 256);
}

cudaError_t bfs_launch(BfsParams &p, dpc_level level, int root_blocks, int queue_blocks, cudaStream_t s) {
  cudaError_t e;
  const int fill_blocks = ceil_div(p.n, 256) < 1024 ? ceil_div(p.n, 256) : 1024;
  bfs_fill<<<fill_blocks, 256, 0, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int T = p.child_threads;
  if (level == DPC_BASIC_DP) {
    // the root's visit strides over its out-edges, whatever its grid size
    bfs_visit_vertex<<<root_blocks, T, 0, s>>>(p, p.source, 0u);
    return cudaGetLastError();
  }
  if (level == DPC_FLAT) {
    int *cur = p.frontier, *nxt = p.next;
    int nf = 1;
    HostScratch &hs = host_scratch();
    hs.value = p.source;
    if ((e = cudaMemcpyAsync(cur, &hs.value, sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    for (unsigned depth = 0; nf > 0; ++depth) {
      if ((e = cudaMemsetAsync(&p.hdr->cursor2, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
      const int blocks = ceil_div(nf, T) < p.child_blocks ? ceil_div(nf, T) : p.child_blocks;
      bfs_flat_level<<<blocks, T, 0, s>>>(p, cur, nf, nxt, depth);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      unsigned long long &cnt = hs.count;
      cnt = 0;
      if ((e = cudaMemcpyAsync(&cnt, &p.hdr->cursor2, sizeof(cnt), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      nf = (int)cnt;
      int *t = cur;
      cur = nxt;
      nxt = t;
    }
    return cudaSuccess;
  }
  bfs_root<<<1, 256, 0, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (level) {
    case DPC_WARP: bfs_visit<DPC_WARP><<<root_blocks, T, 0, s>>>(p, p.units, -1, 0u); break;
    case DPC_BLOCK: bfs_visit<DPC_BLOCK><<<root_blocks, T, 0, s>>>(p, p.units, -1, 0u); break;
    case DPC_GRID: bfs_visit<DPC_GRID><<<root_blocks, T, 0, s>>>(p, p.units, -1, 0u); break;
    case DPC_QUEUE: {
      BfsParams q = p;
      void *args[] = {&q};
      return cudaLaunchCooperativeKernel((const void *)bfs_queue, dim3(queue_blocks), dim3(T), args, 0, s);
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

const void *bfs_kernel(dpc_level level) {
  switch (level) {
    case DPC_BASIC_DP: return (const void *)bfs_visit_vertex;
    case DPC_FLAT: return (const void *)bfs_flat_level;
    case DPC_WARP: return (const void *)bfs_visit<DPC_WARP>;
    case DPC_BLOCK: return (const void *)bfs_visit<DPC_BLOCK>;
    case DPC_GRID: return (const void *)bfs_visit<DPC_GRID>;
    case DPC_QUEUE: return (const void *)bfs_queue;
  }
  return nullptr;
}

}  // namespace dpc
