// Graph colouring (Sec. V, the GC benchmark) at the consolidation levels.
//
// Round-sweep colouring (the independent-set rounds of Jones-Plassmann, the
// colour being the round) with the caller's priorities: in round r every vertex
// still uncoloured when the round began takes colour r unless a neighbour also
// uncoloured at the round's start outranks it (higher priority, ties to the
// larger id). The irregular loop is the neighbour scan of each uncoloured
// vertex; a vertex with more than `threshold` neighbours is large work:
//   flat      the thread scans all neighbours itself (host-driven rounds).
//   basic-DP  the thread launches a child grid over the vertex's neighbours.
//   warp/block/grid
//             the thread appends (vertex, chunk) units to its warp's, block's
//             or grid's buffer and one consolidated child scans them all.
//   queue     the grid level's rounds inside one cooperative grid, three grid
//             barriers per round, no device launch.
// Children only record that an outranking competitor exists (blocked[v] = r);
// the round's commit, tail-launched after the parent and all its children,
// colours the large vertices that were not blocked and tail-launches the next
// round's parent. Short vertices are decided by their parent thread at once:
// a vertex coloured r during round r still counts as a competitor in round r
// (colour == r), so the decisions do not depend on the order they are made in.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "dpc_internal.h"
#include "dpc_runtime.cuh"

namespace cg = cooperative_groups;

namespace dpc {

namespace {

constexpr int kScanBatch = 8;

__device__ __forceinline__ void gc_fail(const GcParams &p, unsigned code) {
  set_status(&p.hdr->status, code);
  if (p.stats) atomicCAS(&p.stats->status, 0u, code);
}

__device__ __forceinline__ const int *active_list(const GcParams &p, int r) { return p.list[r & 1]; }
__device__ __forceinline__ int *next_list(const GcParams &p, int r) { return p.list[(r + 1) & 1]; }

// Does some neighbour among col[a + t], col[a + t + T], ... (below b) still
// compete in round r and outrank v? Eight neighbours per batch: their ids,
// then their colours and priorities, then the test. Stops at the first batch
// that finds one.
__device__ __forceinline__ bool outranked(const GcParams &p, int v, unsigned pv, int a, int b, int r, int t, int T,
                                          unsigned long long *scanned) {
  for (int e0 = a + t; e0 < b; e0 += kScanBatch * T) {
    int u[kScanBatch];
#pragma unroll
    for (int q = 0; q < kScanBatch; ++q) {
      const int e = e0 + q * T;
      u[q] = e < b ? checked_index(__ldg(p.col + e), p.n, &p.hdr->status) : -1;
      if (e < b) ++*scanned;
    }
    int c[kScanBatch];
    unsigned pu[kScanBatch];
#pragma unroll
    for (int q = 0; q < kScanBatch; ++q) {
      c[q] = u[q] >= 0 ? __ldcg(p.color + u[q]) : 1;
      pu[q] = u[q] >= 0 ? __ldg(p.prio + u[q]) : 0u;
    }
    bool hit = false;
#pragma unroll
    for (int q = 0; q < kScanBatch; ++q)
      hit |= u[q] >= 0 && u[q] != v && (c[q] == 0 || c[q] == r) && (pu[q] > pv || (pu[q] == pv && u[q] > v));
    if (hit) return true;
  }
  return false;
}

// Append v to the next round's list (warp-aggregated).
__device__ __forceinline__ void push_next(const GcParams &p, int v, int r) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&p.hdr->cursor2, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  next_list(p, r)[base + g.thread_rank()] = v;
}

__device__ __forceinline__ void push_heavy(const GcParams &p, int v) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&p.hdr->aux[1], (unsigned long long)g.size());
  base = g.shfl(base, 0);
  p.heavy[base + g.thread_rank()] = v;
}

// A short vertex decided by its own thread.
__device__ __forceinline__ void decide_inline(const GcParams &p, int v, int a, int b, int r,
                                              unsigned long long *scanned) {
  if (outranked(p, v, __ldg(p.prio + v), a, b, r, 0, 1, scanned)) push_next(p, v, r);
  else p.color[v] = r;
}

// One unit (vertex, chunk) scanned by a full warp; any lane that finds an
// outranking competitor marks the vertex blocked for this round.
__device__ __forceinline__ void gc_unit(const GcParams &p, int2 u, int r, unsigned long long *scanned) {
  if (u.x < 0) return;  // placeholder written after a buffer overflow
  // another unit already found one (decided once for the whole warp)
  if (__shfl_sync(0xffffffffu, lane_id() == 0 ? __ldcg(p.blocked + u.x) : 0u, 0) == (unsigned)r) return;
  const int a0 = __ldg(p.off + u.x), b0 = __ldg(p.off + u.x + 1);
  const int a = a0 + u.y * p.chunk, b = min(b0, a + p.chunk);
  const bool hit = outranked(p, u.x, __ldg(p.prio + u.x), a, b, r, lane_id(), kWarp, scanned);
  if (__any_sync(0xffffffffu, hit) && lane_id() == 0) p.blocked[u.x] = (unsigned)r;
}

__device__ __forceinline__ void gc_units_by_group(const GcParams &p, const int2 *units, int lo, int hi, int w, int W,
                                                  int r, unsigned long long *scanned) {
  for (int i = lo + w; i < hi; i += W) gc_unit(p, units[i], r, scanned);
}

__device__ __forceinline__ int active_size(const GcParams &p) {
  return (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[0]);
}

__device__ __forceinline__ void gc_stats(const GcParams &p, unsigned long long scanned, unsigned long long inl,
                                         unsigned long long buf, unsigned long long launched,
                                         unsigned long long failed) {
  if (!p.stats) return;
  scanned = warp_sum(scanned);
  inl = warp_sum(inl);
  buf = warp_sum(buf);
  launched = warp_sum(launched);
  failed = warp_sum(failed);
  if (lane_id() == 0) {
    stat_add(p.stats, &dpc_stats::relaxations, scanned);
    stat_add(p.stats, &dpc_stats::inline_items, inl);
    stat_add(p.stats, &dpc_stats::buffered_items, buf);
    stat_add(p.stats, &dpc_stats::child_launches, launched);
    stat_add(p.stats, &dpc_stats::launch_failures, failed);
  }
}

}  // namespace

__global__ void gc_commit(GcParams p, int r);

// ------------------------------------------------------------------ children

// Basic-DP child: thread per neighbour of one large vertex.
__global__ void __launch_bounds__(1024) gc_vertex_child(GcParams p, int v, int r) {
  const int a = __ldg(p.off + v), b = __ldg(p.off + v + 1);
  const int e = a + blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b) return;
  const int u = checked_index(__ldg(p.col + e), p.n, &p.hdr->status);
  if (kCheckedBuild && u < 0) return;
  const unsigned pv = __ldg(p.prio + v), pu = __ldg(p.prio + u);
  const int c = __ldcg(p.color + u);
  if (u != v && (c == 0 || c == r) && (pu > pv || (pu == pv && u > v))) p.blocked[v] = (unsigned)r;
}

// Consolidated child: warps take units round-robin (Sec. IV.C), or four at a
// time from a shared cursor when the child is the only one of its round.
__global__ void __launch_bounds__(1024) gc_child(GcParams p, const int2 *__restrict__ units, int nunits, int r,
                                                unsigned long long *cursor) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0;
  if (cursor) {
    for (;;) {
      unsigned long long i0 = 0;
      if (lane_id() == 0) i0 = atomicAdd(cursor, 4ull);
      i0 = __shfl_sync(0xffffffffu, i0, 0);
      if (i0 >= (unsigned long long)nunits) break;
      const int i1 = (int)min(i0 + 4ull, (unsigned long long)nunits);
      for (int u = (int)i0; u < i1; ++u) gc_unit(p, units[u], r, &scanned);
    }
  } else {
    gc_units_by_group(p, units, 0, nunits, gw, nw, r, &scanned);
  }
  if (p.stats) {
    scanned = warp_sum(scanned);
    if (lane_id() == 0) stat_add(p.stats, &dpc_stats::relaxations, scanned);
  }
}

// ------------------------------------------------------------------ parents

namespace {
__device__ __forceinline__ void round_prologue(const GcParams &p, int r) {
  // the round's commit runs after this grid and every child it launches
  if (p.level != DPC_FLAT && blockIdx.x == 0 && threadIdx.x == 0) {
    gc_commit<<<p.commit_blocks, 256, 0, cudaStreamTailLaunch>>>(p, r);
    if (cudaGetLastError() != cudaSuccess) gc_fail(p, DPC_ERR_DEVICE);
    else stat_add(p.stats, &dpc_stats::aux_launches, 1);
  }
}
}  // namespace

// Flat and basic-DP parent: thread per uncoloured vertex.
template <int LEVEL>
__global__ void __launch_bounds__(1024) gc_parent_simple(GcParams p, int r) {
  round_prologue(p, r);
  const int na = active_size(p);
  const int *act = active_list(p, r);
  unsigned long long scanned = 0, inl = 0, buf = 0, launched = 0, failed = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
    const int v = act[i];
    const int a = __ldg(p.off + v), b = __ldg(p.off + v + 1);
    if (LEVEL == DPC_BASIC_DP && b - a > p.threshold) {
      buf++;
      push_heavy(p, v);
      if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
        gc_vertex_child<<<ceil_div(b - a, p.child_threads), p.child_threads, 0, cudaStreamFireAndForget>>>(p, v, r);
        if (cudaGetLastError() == cudaSuccess) {
          launched++;
          scanned += b - a;
          continue;
        }
      }
      failed++;  // the launch was refused: scan here, the commit still decides
      if (outranked(p, v, __ldg(p.prio + v), a, b, r, 0, 1, &scanned)) p.blocked[v] = (unsigned)r;
      continue;
    }
    inl++;
    decide_inline(p, v, a, b, r, &scanned);
  }
  gc_stats(p, scanned, inl, buf, launched, failed);
}

// Warp-, block- and grid-level parent: count the units of the thread's large
// vertices, reserve the group's slice with one atomic, write the units at
// scanned offsets while short vertices are decided inline, then one launch
// per warp / block / grid (Fig. 4b).
template <int LEVEL>
__global__ void __launch_bounds__(1024) gc_parent(GcParams p, int r) {
  __shared__ int s_scan[33];
  __shared__ int s_base, s_fail;
  round_prologue(p, r);
  const int na = active_size(p);
  const int *act = active_list(p, r);
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int bstart = blockIdx.x * blockDim.x;

  int mine = 0;
  for (int i = bstart + threadIdx.x; i < na; i += G) {
    const int v = act[i];
    const int deg = __ldg(p.off + v + 1) - __ldg(p.off + v);
    if (deg > p.threshold) mine += ceil_div(deg, p.chunk);
  }
  int base, gtotal;
  if (LEVEL == DPC_BLOCK) {
    gtotal = block_sum(mine, s_scan);
    if (threadIdx.x == 0) s_base = gtotal ? (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal) : 0;
    __syncthreads();
    base = s_base;
  } else {
    gtotal = warp_sum(mine);
    int b0 = 0;
    if (lane == 0 && gtotal) b0 = (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal);
    base = __shfl_sync(0xffffffffu, b0, 0);
  }
  if (gtotal && base + gtotal > p.max_units) {  // only reachable with malformed input
    if (lane == 0) gc_fail(p, DPC_ERR_OVERFLOW);
    const int lo = LEVEL == DPC_BLOCK ? threadIdx.x : lane, step = LEVEL == DPC_BLOCK ? blockDim.x : kWarp;
    for (int j = base + lo; j < min(base + gtotal, p.max_units); j += step) p.units[j] = make_int2(-1, 0);
    gtotal = 0;  // the group's large vertices are then decided inline below
  }

  int run = base;
  unsigned long long scanned = 0, inl = 0, buf = 0, launched = 0, failed = 0;
  for (int i0 = bstart; i0 < na; i0 += G) {
    const int i = i0 + threadIdx.x;
    int nu = 0, a = 0, b = 0, v = -1;
    if (i < na) {
      v = act[i];
      a = __ldg(p.off + v);
      b = __ldg(p.off + v + 1);
      if (gtotal && b - a > p.threshold) nu = ceil_div(b - a, p.chunk);
    }
    int excl, step;
    if (LEVEL == DPC_BLOCK) {
      excl = block_exclusive_scan(nu, s_scan, &step);
    } else {
      const int inc = warp_inclusive_scan(nu);
      excl = inc - nu;
      step = __shfl_sync(0xffffffffu, inc, kWarp - 1);
    }
    if (nu) {
      const int pos = run + excl;
      for (int k = 0; k < nu; ++k) p.units[pos + k] = make_int2(v, k);
      push_heavy(p, v);
      buf++;
    } else if (v >= 0) {
      inl++;
      decide_inline(p, v, a, b, r, &scanned);
    }
    run += step;
  }

  if (LEVEL == DPC_WARP) {
    __threadfence();
    __syncwarp();
    if (gtotal) {
      int fl = 0;
      if (lane == 0) {
        fl = 1;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          gc_child<<<child_grid_for(gtotal, p.child_blocks, p.child_threads), p.child_threads, 0,
                     cudaStreamFireAndForget>>>(p, p.units + base, gtotal, r, nullptr);
          fl = cudaGetLastError() != cudaSuccess;
        }
        if (fl) failed++;
        else launched++;
      }
      fl = __shfl_sync(0xffffffffu, fl, 0);
      if (fl) gc_units_by_group(p, p.units, base, base + gtotal, 0, 1, r, &scanned);
    }
  } else if (LEVEL == DPC_BLOCK) {
    __threadfence();
    __syncthreads();
    if (gtotal) {
      if (threadIdx.x == 0) {
        s_fail = 1;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          gc_child<<<child_grid_for(gtotal, p.child_blocks, p.child_threads), p.child_threads, 0,
                     cudaStreamFireAndForget>>>(p, p.units + base, gtotal, r, nullptr);
          s_fail = cudaGetLastError() != cudaSuccess;
        }
        if (s_fail) failed++;
        else launched++;
      }
      __syncthreads();
      if (s_fail) gc_units_by_group(p, p.units, base, base + gtotal, threadIdx.x >> 5, blockDim.x >> 5, r, &scanned);
    }
  } else {  // DPC_GRID
    if (last_block_done(&p.hdr->done_blocks)) {
      if (threadIdx.x == 0) {
        const int total = (int)min(*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                                   (unsigned long long)p.max_units);
        s_base = total;
        s_fail = 0;
        if (total > 0) {
          s_fail = 1;
          if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
            gc_child<<<child_grid_for(total, p.child_blocks, p.child_threads), p.child_threads, 0,
                       cudaStreamFireAndForget>>>(p, p.units, total, r, &p.hdr->aux[2]);
            s_fail = cudaGetLastError() != cudaSuccess;
          }
          if (s_fail) failed++;
          else launched++;
        }
      }
      __syncthreads();
      if (s_fail) gc_units_by_group(p, p.units, 0, s_base, threadIdx.x >> 5, blockDim.x >> 5, r, &scanned);
    }
  }
  gc_stats(p, scanned, inl, buf, launched, failed);
}

// Parent of round r for na uncoloured vertices (device side).
__device__ void launch_gc_parent(const GcParams &p, int r, int na, cudaStream_t s) {
  const int need = ceil_div(na, p.parent_threads);
  const int blocks = need < p.parent_blocks ? (need > 0 ? need : 1) : p.parent_blocks;
  switch (p.level) {
    case DPC_BASIC_DP: gc_parent_simple<DPC_BASIC_DP><<<blocks, p.parent_threads, 0, s>>>(p, r); break;
    case DPC_WARP: gc_parent<DPC_WARP><<<blocks, p.parent_threads, 0, s>>>(p, r); break;
    case DPC_BLOCK: gc_parent<DPC_BLOCK><<<blocks, p.parent_threads, 0, s>>>(p, r); break;
    case DPC_GRID: gc_parent<DPC_GRID><<<blocks, p.parent_threads, 0, s>>>(p, r); break;
    default: break;
  }
}

// After round r: colour the large vertices nobody blocked, queue the others,
// reset the round's counters and continue with round r+1 while vertices remain.
__global__ void __launch_bounds__(256) gc_commit(GcParams p, int r) {
  const int nh = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[1]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += gridDim.x * blockDim.x) {
    const int v = __ldcg(p.heavy + i);
    if (__ldcg(p.blocked + v) == (unsigned)r) push_next(p, v, r);
    else p.color[v] = r;
  }
  if (!last_block_done(&p.hdr->done_blocks2)) return;
  if (threadIdx.x == 0) {
    const int nn = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor2);
    p.hdr->aux[0] = (unsigned long long)nn;
    p.hdr->aux[1] = 0ull;
    p.hdr->aux[2] = 0ull;    // the grid-level child's unit cursor
    p.hdr->cursor2 = 0ull;
    p.hdr->cursor = 0ull;
    p.hdr->launches = 0ull;  // the round's children have all finished: their pool slots are free
    p.hdr->round = (unsigned)r;
    __threadfence();
    if (p.stats) atomicMax(&p.stats->rounds, (unsigned)r);
    if (p.level != DPC_FLAT && nn > 0 && r < p.n && p.hdr->status == 0u) {
      launch_gc_parent(p, r + 1, nn, cudaStreamTailLaunch);
      if (cudaGetLastError() != cudaSuccess) gc_fail(p, DPC_ERR_DEVICE);
      else stat_add(p.stats, &dpc_stats::aux_launches, 1);
    }
  }
}

// ------------------------------------------------------------------ queue level

namespace {

// Multi-use barrier of the cooperative grid (arrivals only grow: the k-th
// barrier is complete at k * gridDim.x arrivals). With `end_round`, the last
// arriver closes the round before releasing the others: it publishes the next
// round's size and resets the round's counters. Bounded wait.
__device__ bool round_barrier(const GcParams &p, unsigned k, bool end_round, int *next_size) {
  __shared__ int s_ok, s_nn;
  __syncthreads();  // orders the block's writes before its master thread's fence and arrival
  if (threadIdx.x == 0) {
    __threadfence();
    int ok = 1;
    if (atomicAdd(&p.hdr->done_blocks2, 1u) == k * gridDim.x - 1) {
      if (end_round) {
        p.hdr->aux[0] = *reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor2);
        p.hdr->cursor2 = 0ull;
        p.hdr->cursor = 0ull;
        p.hdr->aux[1] = 0ull;
      }
      __threadfence();
      atomicExch(&p.hdr->round, k);
    } else {
      WaitClock clk;
      while (*reinterpret_cast<volatile unsigned *>(&p.hdr->round) < k) {
        __nanosleep(64);
        if (clk.expired()) {
          gc_fail(p, DPC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_nn = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[0]);
    s_ok = ok;
  }
  __syncthreads();
  *next_size = s_nn;
  return s_ok != 0;
}

}  // namespace

__global__ void __launch_bounds__(1024) gc_queue(GcParams p) {
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gw = gtid >> 5, W = G >> 5;
  int na = active_size(p);
  unsigned k = 0;
  unsigned long long scanned = 0, inl = 0, buf = 0;
  int r = 1;
  for (; na > 0 && r <= p.n; ++r) {
    const int *act = active_list(p, r);
    // large vertices' units into the buffer (one atomic per warp and pass), short ones decided
    for (int i0 = gtid - lane; i0 < na; i0 += G) {
      const int i = i0 + lane;
      int v = -1, a = 0, b = 0, nu = 0;
      if (i < na) {
        v = act[i];
        a = __ldg(p.off + v);
        b = __ldg(p.off + v + 1);
        if (b - a > p.threshold) nu = ceil_div(b - a, p.chunk);
      }
      const int inc = warp_inclusive_scan(nu);
      const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
      int b0 = 0;
      if (lane == kWarp - 1 && total) b0 = (int)atomicAdd(&p.hdr->cursor, (unsigned long long)total);
      const int base = __shfl_sync(0xffffffffu, b0, kWarp - 1);
      const bool room = base + total <= p.max_units;
      if (!room) {  // only reachable with malformed input: placeholders, and the vertices decided here
        if (lane == 0) gc_fail(p, DPC_ERR_OVERFLOW);
        for (int j = base + lane; j < min(base + total, p.max_units); j += kWarp) p.units[j] = make_int2(-1, 0);
      }
      if (nu && room) {
        for (int q = 0; q < nu; ++q) p.units[base + inc - nu + q] = make_int2(v, q);
        push_heavy(p, v);
        buf++;
      } else if (v >= 0) {
        // short vertex (or no room in the buffer): decided here
        inl++;
        if (nu) {
          if (outranked(p, v, __ldg(p.prio + v), a, b, r, 0, 1, &scanned)) p.blocked[v] = (unsigned)r;
          push_heavy(p, v);
        } else {
          decide_inline(p, v, a, b, r, &scanned);
        }
      }
    }
    int dummy = 0;
    if (!round_barrier(p, ++k, false, &dummy)) return;
    const int total = (int)min(*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                               (unsigned long long)p.max_units);
    gc_units_by_group(p, p.units, 0, total, gw, W, r, &scanned);
    if (!round_barrier(p, ++k, false, &dummy)) return;
    const int nh = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[1]);
    for (int i = gtid; i < nh; i += G) {
      const int v = __ldcg(p.heavy + i);
      if (__ldcg(p.blocked + v) == (unsigned)r) push_next(p, v, r);
      else p.color[v] = r;
    }
    if (!round_barrier(p, ++k, true, &na)) return;
  }
  gc_stats(p, scanned, inl, buf, 0, 0);
  if (p.stats && gtid == 0) atomicMax(&p.stats->rounds, (unsigned)(r - 1));
}

// ------------------------------------------------------------------ set-up and host side

__global__ void gc_init(GcParams p) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += gridDim.x * blockDim.x) {
    p.color[v] = 0;
    p.blocked[v] = 0u;
    p.list[1][v] = v;  // round 1 reads list[1]
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) p.hdr->aux[0] = (unsigned long long)p.n;
}

size_t gc_max_units(int n, int m, int threshold, int chunk) {
  size_t large = (size_t)m / ((size_t)threshold + 1);
  if (large > (size_t)n) large = (size_t)n;
  return (size_t)m / (size_t)chunk + large + 1;
}

size_t gc_workspace_bytes(int n, int m, dpc_level level, const LaunchCfg &c) {
  size_t b = kHeaderBytes;
  b += 3 * align_up((size_t)n * sizeof(int), 256);       // two active lists, the large-vertex list
  b += align_up((size_t)n * sizeof(unsigned), 256);      // blocked stamps
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE)
    b += align_up(gc_max_units(n, m, c.threshold, c.chunk) * sizeof(int2), 256);
  return b;
}

const void *gc_parent_kernel(dpc_level level) {
  switch (level) {
    case DPC_FLAT: return (const void *)gc_parent_simple<DPC_FLAT>;
    case DPC_BASIC_DP: return (const void *)gc_parent_simple<DPC_BASIC_DP>;
    case DPC_WARP: return (const void *)gc_parent<DPC_WARP>;
    case DPC_BLOCK: return (const void *)gc_parent<DPC_BLOCK>;
    case DPC_GRID: return (const void *)gc_parent<DPC_GRID>;
    case DPC_QUEUE: return (const void *)gc_queue;
  }
  return nullptr;
}

const void *gc_child_kernel(dpc_level level) {
  if (level == DPC_QUEUE || level == DPC_FLAT) return nullptr;
  return level == DPC_BASIC_DP ? (const void *)gc_vertex_child : (const void *)gc_child;
}

cudaError_t gc_launch(GcParams &p, dpc_level level, int queue_blocks, cudaStream_t s) {
  const int init_blocks = ceil_div(p.n, 256) < 1024 ? ceil_div(p.n, 256) : 1024;
  gc_init<<<init_blocks > 0 ? init_blocks : 1, 256, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int need = ceil_div(p.n, p.parent_threads);
  const int blocks = need < p.parent_blocks ? (need > 0 ? need : 1) : p.parent_blocks;
  switch (level) {
    case DPC_BASIC_DP: gc_parent_simple<DPC_BASIC_DP><<<blocks, p.parent_threads, 0, s>>>(p, 1); break;
    case DPC_WARP: gc_parent<DPC_WARP><<<blocks, p.parent_threads, 0, s>>>(p, 1); break;
    case DPC_BLOCK: gc_parent<DPC_BLOCK><<<blocks, p.parent_threads, 0, s>>>(p, 1); break;
    case DPC_GRID: gc_parent<DPC_GRID><<<blocks, p.parent_threads, 0, s>>>(p, 1); break;
    case DPC_QUEUE: {
      GcParams q = p;
      void *args[] = {&q};
      return cudaLaunchCooperativeKernel((const void *)gc_queue, dim3(queue_blocks), dim3(p.parent_threads), args, 0,
                                         s);
    }
    case DPC_FLAT: {
      // host-driven rounds (no device launches at all)
      unsigned long long &na = host_scratch().count;
      na = (unsigned long long)p.n;
      for (int r = 1; na > 0 && r <= p.n; ++r) {
        const int nb = ceil_div((int)na, p.parent_threads) < p.parent_blocks ? ceil_div((int)na, p.parent_threads)
                                                                             : p.parent_blocks;
        gc_parent_simple<DPC_FLAT><<<nb, p.parent_threads, 0, s>>>(p, r);
        gc_commit<<<p.commit_blocks, 256, 0, s>>>(p, r);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&na, &p.hdr->aux[0], sizeof(na), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
          return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dpc
