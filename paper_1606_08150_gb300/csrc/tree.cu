// Tree descendants and tree heights: parallel recursion (Fig. 1c, Sec. V).
//
// visit(S) processes the child lists of a set S of internal nodes. Every child
// c gets its leaf work (value 0); a child with children of its own is the
// recursive call of Fig. 1c. Its postwork - combining the values of v's
// children into v - may only run after the whole subtree below S is finished:
// on CDP2 that is a tail launch, which waits for the launching grid and every
// grid launched below it, replacing the cudaDeviceSynchronize of Sec. IV.C.
//   basic-DP   one recursive grid per internal child, each with its own
//              postwork tail launch (two launches per internal node).
//   warp/block/grid
//              the internal children found by a warp, block or the whole grid
//              are appended to that scope's buffer; one recursive grid per
//              buffer (Sec. IV.B) and one postwork tail launch per grid. The
//              grid level thus launches once per tree level.
//   flat       the host runs the levels top-down, one kernel per level, then
//              the postwork levels bottom-up; no device launches.
//   queue      the grid level's level buffers inside one cooperative grid:
//              the levels top-down, then the postwork levels bottom-up, a
//              grid barrier between any two; no launch at all.
// Buffer entries are units (node, chunk of `chunk` children), so a node with
// 50,000 children is spread over many threads. Values are integers combined
// with atomics, so every level yields exactly the same result.
#include <climits>
#include <utility>
#include <vector>

#include "dpc_internal.h"
#include "dpc_runtime.cuh"

namespace dpc {

namespace {

__device__ __forceinline__ void tree_fail(const TreeParams &p, unsigned code) {
  set_status(&p.hdr->status, code);
  if (p.stats) atomicCAS(&p.stats->status, 0u, code);
}

// children [a, b) of unit u
__device__ __forceinline__ void unit_range(const TreeParams &p, int2 u, int *a, int *b) {
  if (u.x < 0) {  // placeholder written after a buffer overflow
    *a = *b = 0;
    return;
  }
  const int a0 = __ldg(p.coff + u.x), b0 = __ldg(p.coff + u.x + 1);
  if (p.chunk == INT_MAX) {
    *a = a0;
    *b = b0;
  } else {
    *a = a0 + u.y * p.chunk;
    *b = min(b0, *a + p.chunk);
  }
}

// Children k0 .. k0+7 (below b) and their own child counts, loads issued as a
// batch: two dependent round trips per eight children instead of two per child.
constexpr int kKidBatch = 8;

__device__ __forceinline__ void load_kids(const TreeParams &p, int k0, int b, int (&c)[kKidBatch],
                                          int (&kc)[kKidBatch]) {
#pragma unroll
  for (int j = 0; j < kKidBatch; ++j)
    c[j] = k0 + j < b ? checked_index(__ldg(p.cidx + k0 + j), p.n, &p.hdr->status) : -1;
  int lo[kKidBatch], hi[kKidBatch];
#pragma unroll
  for (int j = 0; j < kKidBatch; ++j) {
    lo[j] = c[j] >= 0 ? __ldg(p.coff + c[j]) : 0;
    hi[j] = c[j] >= 0 ? __ldg(p.coff + c[j] + 1) : 0;
    checked_range(lo[j], hi[j], p.n - 1, &p.hdr->status);
  }
#pragma unroll
  for (int j = 0; j < kKidBatch; ++j) kc[j] = hi[j] - lo[j];
}

__device__ __forceinline__ int units_for(const TreeParams &p, int k) {
  // a power-of-two chunk (the default 8) divides by a shift: on the narrow
  // levels one warp's chain of dependent instructions is the level's cost
  if (k <= 0) return 0;
  if (p.chunk_shift >= 0) return ((k - 1) >> p.chunk_shift) + 1;
  return p.chunk == INT_MAX ? 1 : ceil_div(k, p.chunk);
}

}  // namespace

template <int OP>
__global__ void tree_post(TreeParams p, const int2 *__restrict__ units, int nunits);
template <int OP>
__global__ void tree_post_node(TreeParams p, int v);

// ------------------------------------------------------------------ postwork

// Thread per unit: combine the unit's children into the unit's node.
template <int OP>
__global__ void __launch_bounds__(1024) tree_post(TreeParams p, const int2 *__restrict__ units, int nunits) {
  const int G = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nunits; i += G) {
    const int2 u = units[i];
    int a, b;
    unit_range(p, u, &a, &b);
    if (u.x < 0) continue;
    unsigned sum = 0;
    int h = 0;
    for (int k0 = a; k0 < b; k0 += kKidBatch) {
      int c[kKidBatch], val[kKidBatch];
#pragma unroll
      for (int j = 0; j < kKidBatch; ++j)
        c[j] = k0 + j < b ? checked_index(__ldg(p.cidx + k0 + j), p.n, &p.hdr->status) : -1;
#pragma unroll
      for (int j = 0; j < kKidBatch; ++j) val[j] = c[j] >= 0 ? __ldcg(p.out + c[j]) : 0;
#pragma unroll
      for (int j = 0; j < kKidBatch; ++j) {
        if (c[j] < 0) continue;
        if (OP == kDescendants) sum += 1u + (unsigned)val[j];
        else h = max(h, 1 + val[j]);
      }
    }
    if (OP == kDescendants) atomicAdd(reinterpret_cast<unsigned *>(p.out) + u.x, sum);
    else atomicMax(p.out + u.x, h);
  }
}

// Basic-DP postwork of one node: one block reduces over all of its children.
template <int OP>
__global__ void __launch_bounds__(1024) tree_post_node(TreeParams p, int v) {
  __shared__ int sm[32];
  const int a = __ldg(p.coff + v), b = __ldg(p.coff + v + 1);
  int acc = 0;
  for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
    const int ci = checked_index(__ldg(p.cidx + k), p.n, &p.hdr->status);
    if (kCheckedBuild && ci < 0) continue;
    const int c = __ldcg(p.out + ci);
    acc = OP == kDescendants ? acc + 1 + c : max(acc, 1 + c);
  }
  if (OP == kDescendants) {
    acc = block_sum(acc, sm);
  } else {
    for (int d = 16; d >= 1; d >>= 1) acc = max(acc, __shfl_xor_sync(0xffffffffu, acc, d));
    __syncthreads();
    if (lane_id() == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    acc = (int)lane_id() < (int)(blockDim.x >> 5) ? sm[lane_id()] : 0;
    for (int d = 16; d >= 1; d >>= 1) acc = max(acc, __shfl_xor_sync(0xffffffffu, acc, d));
  }
  if (threadIdx.x == 0) p.out[v] = acc;
}

// ------------------------------------------------------------------ basic-DP visit

// Fig. 1c: thread per child of v; an internal child gets its own recursive grid.
template <int OP>
__global__ void __launch_bounds__(1024) tree_visit_node(TreeParams p, int v, int depth) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    tree_post_node<OP><<<1, 256, 0, cudaStreamTailLaunch>>>(p, v);
    if (cudaGetLastError() != cudaSuccess) tree_fail(p, DPC_ERR_DEVICE);
    else stat_add(p.stats, &dpc_stats::aux_launches, 1);
    if (p.stats) atomicMax(&p.stats->rounds, (unsigned)depth + 1u);
  }
  const int a = __ldg(p.coff + v), b = __ldg(p.coff + v + 1);
  const int G = gridDim.x * blockDim.x;
  unsigned long long launched = 0, visited = 0;
  for (int k = a + blockIdx.x * blockDim.x + threadIdx.x; k < b; k += G) {
    const int c = checked_index(__ldg(p.cidx + k), p.n, &p.hdr->status);
    if (kCheckedBuild && c < 0) continue;
    p.out[c] = 0;
    visited++;
    const int kc = __ldg(p.coff + c + 1) - __ldg(p.coff + c);
    if (kc > 0) {
      bool ok = false;
      if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
        __threadfence();
        tree_visit_node<OP><<<ceil_div(kc, p.child_threads), p.child_threads, 0, cudaStreamFireAndForget>>>(
            p, c, depth + 1);
        ok = cudaGetLastError() == cudaSuccess;
      }
      if (ok) launched++;
      else tree_fail(p, DPC_ERR_DEVICE);
    }
  }
  if (p.stats) {
    launched = warp_sum(launched);
    visited = warp_sum(visited);
    if (lane_id() == 0) {
      stat_add(p.stats, &dpc_stats::child_launches, launched);
      stat_add(p.stats, &dpc_stats::buffered_items, launched);
      stat_add(p.stats, &dpc_stats::relaxations, visited);
      if (visited) atomicMax(&p.stats->rounds, (unsigned)depth + 2u);
    }
  }
}

// ------------------------------------------------------------------ consolidated visit

// visit(S) for S given as units. Two passes over the units: count the units of
// the internal children each thread finds, scan the thread counts over the
// warp (block) and reserve the slice with one atomic, then write. The grid
// level reserves per warp and the last block launches the whole level.
template <int LEVEL, int OP>
__global__ void __launch_bounds__(1024) tree_visit(TreeParams p, const int2 *__restrict__ units, int nunits,
                                                  int depth) {
  __shared__ int s_scan[33];
  __shared__ int s_base;
  const int lane = lane_id();
  // a negative count: the root's units, counted on the device by tree_init
  if (nunits < 0) nunits = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[0]);
  if (p.stats && blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&p.stats->rounds, (unsigned)depth + 1u);
  if (LEVEL != DPC_FLAT && blockIdx.x == 0 && threadIdx.x == 0) {
    const int pb = ceil_div(nunits, 256) < p.child_blocks ? ceil_div(nunits, 256) : p.child_blocks;
    tree_post<OP><<<pb > 0 ? pb : 1, 256, 0, cudaStreamTailLaunch>>>(p, units, nunits);
    if (cudaGetLastError() != cudaSuccess) tree_fail(p, DPC_ERR_DEVICE);
    else stat_add(p.stats, &dpc_stats::aux_launches, 1);
  }
  const int G = gridDim.x * blockDim.x;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;

  // pass 1
  int mine = 0;
  for (int i = g; i < nunits; i += G) {
    int a, b;
    unit_range(p, units[i], &a, &b);
    for (int k0 = a; k0 < b; k0 += kKidBatch) {
      int c[kKidBatch], kc[kKidBatch];
      load_kids(p, k0, b, c, kc);
#pragma unroll
      for (int j = 0; j < kKidBatch; ++j) mine += units_for(p, kc[j]);
    }
  }
  // the thread's offset inside its group's slice, and the slice itself
  int excl, gtotal, base;
  if (LEVEL == DPC_BLOCK) {
    excl = block_exclusive_scan(mine, s_scan, &gtotal);
    if (threadIdx.x == 0) s_base = gtotal ? (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal) : 0;
    __syncthreads();
    base = s_base;
  } else {
    const int inc = warp_inclusive_scan(mine);
    excl = inc - mine;
    gtotal = __shfl_sync(0xffffffffu, inc, kWarp - 1);
    int b0 = 0;
    if (lane == kWarp - 1 && gtotal) b0 = (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal);
    base = __shfl_sync(0xffffffffu, b0, kWarp - 1);
  }
  if (gtotal && base + gtotal > p.max_units) {  // only reachable when the input is not a tree
    if (lane == 0) tree_fail(p, DPC_ERR_OVERFLOW);
    const int lo = LEVEL == DPC_BLOCK ? threadIdx.x : lane, step = LEVEL == DPC_BLOCK ? blockDim.x : kWarp;
    for (int j = base + lo; j < min(base + gtotal, p.max_units); j += step) p.units[j] = make_int2(-1, 0);
    gtotal = 0;
  }

  // pass 2: leaf work for every child, internal children into the buffer
  int pos = base + excl;
  unsigned long long visited = 0, internal = 0;
  for (int i = g; i < nunits; i += G) {
    int a, b;
    unit_range(p, units[i], &a, &b);
    visited += b - a;
    for (int k0 = a; k0 < b; k0 += kKidBatch) {
      int c[kKidBatch], kc[kKidBatch];
      load_kids(p, k0, b, c, kc);
#pragma unroll
      for (int j = 0; j < kKidBatch; ++j) {
        if (c[j] < 0) continue;
        p.out[c[j]] = 0;
        const int nu = units_for(p, kc[j]);
        if (nu && gtotal) {
          internal++;
          for (int q = 0; q < nu; ++q) p.units[pos + q] = make_int2(c[j], q);
          pos += nu;
        }
      }
    }
  }
  if (p.stats) {
    visited = warp_sum(visited);
    internal = warp_sum(internal);
    if (lane == 0) {
      stat_add(p.stats, &dpc_stats::relaxations, visited);
      stat_add(p.stats, &dpc_stats::buffered_items, internal);
      if (visited) atomicMax(&p.stats->rounds, (unsigned)depth + 2u);  // the children's level exists
    }
  }
  if (LEVEL == DPC_FLAT) return;

  // barrier of the consolidation scope, then one launch per buffer
  int launch_lo = -1, launch_n = 0;
  if (LEVEL == DPC_WARP) {
    __threadfence();
    __syncwarp();
    if (lane == 0 && gtotal) {
      launch_lo = base;
      launch_n = gtotal;
    }
  } else if (LEVEL == DPC_BLOCK) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && gtotal) {
      launch_lo = base;
      launch_n = gtotal;
    }
  } else {
    if (last_block_done(&p.hdr->done_blocks) && threadIdx.x == 0) {
      // this level's units are exactly those reserved after the level began
      const int end = (int)min(*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                               (unsigned long long)p.max_units);
      const int start = (int)(units - p.units) + nunits;
      if (end > start) {
        launch_lo = start;
        launch_n = end - start;
      }
    }
  }
  if (launch_n > 0) {
    bool ok = false;
    if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
      const int cb = ceil_div(launch_n, p.child_threads) < p.child_blocks ? ceil_div(launch_n, p.child_threads)
                                                                           : p.child_blocks;
      tree_visit<LEVEL, OP><<<cb, p.child_threads, 0, cudaStreamFireAndForget>>>(p, p.units + launch_lo, launch_n,
                                                                                  depth + 1);
      ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok) stat_add(p.stats, &dpc_stats::child_launches, 1);
    else tree_fail(p, DPC_ERR_DEVICE);
  }
}

__global__ void tree_init(TreeParams p) {
  // root: value 0, its units at the head of the buffer
  const int k = p.coff[p.root + 1] - p.coff[p.root];
  const int nu = p.units && k > 0 ? (p.chunk == INT_MAX ? 1 : ceil_div(k, p.chunk)) : 0;
  for (int j = threadIdx.x; j < nu; j += blockDim.x) p.units[j] = make_int2(p.root, j);
  if (threadIdx.x == 0) {
    p.out[p.root] = 0;
    p.hdr->cursor = (unsigned long long)nu;
    p.hdr->aux[0] = (unsigned long long)nu;
  }
}

// ------------------------------------------------------------------ queue level

// The grid level's recursion inside one cooperative grid: the levels top-down
// (every child's leaf value, the internal children's units appended after the
// level's own), each closed by a grid barrier whose last arriver records where
// the next level's units end; then the postwork. No launch at all. A unit here
// is (node, first child, end child, first-unit flag): the range travels with
// the unit, so a level costs one dependent load fewer than with (node, chunk
// index) units, and one pass both reserves (per warp and batch of children)
// and writes.
//
// The postwork runs without level barriers. A node's value is its children's
// share: each child adds 1 (descendants) or makes it at least 1 (heights),
// plus, from each internal child c, desc(c) or 1 + height(c). The first part
// is known when the node's units are visited, so the visit adds it. The second
// waits for the internal children, which are counted: pend[v] = 1 + the
// internal children of v, par[c] = the parent of internal c. After the last
// level, one pass takes the extra 1 from every internal node; whichever thread
// brings pend[v] to 0 - that pass, or the last internal child reporting - knows
// v's value is complete, adds it to the parent and reports there, up the
// chain. Exactly one thread finishes each node, no thread waits, and a chain
// is at most the tree's depth long. The values are sums and maxima of
// integers, so the order of the additions does not matter.
namespace {

constexpr int kSmallUnits = 2;  // a child with more units has them written by its whole warp

// Multi-use barrier (arrivals only grow; the k-th barrier is complete at k *
// gridDim.x arrivals); with `end_slot` >= 0 the last arriver stores there where
// the units appended so far end, before it releases the others. Bounded wait.
__device__ bool tree_barrier(const TreeParams &p, unsigned k, int end_slot, int head) {
  __shared__ int s_ok;
  __syncthreads();  // orders the block's writes before its master thread's fence and arrival
  if (threadIdx.x == 0) {
    __threadfence();
    int ok = 1;
    if (atomicAdd(&p.hdr->done_blocks2, 1u) == k * gridDim.x - 1) {
      if (end_slot >= 0)
        p.level_ends[end_slot] =
            (int)min((unsigned long long)head + *reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                     (unsigned long long)p.max_units);
      __threadfence();
      atomicExch(&p.hdr->round, k);
    } else {
      WaitClock clk;
      while (*reinterpret_cast<volatile unsigned *>(&p.hdr->round) < k) {
        __nanosleep(32);
        if (clk.expired()) {
          tree_fail(p, DPC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// unit i of the root, whose units are never read back before the postwork
__device__ __forceinline__ int4 root_unit(const TreeParams &p, int i, int ra, int rb) {
  const int a = ra + i * p.chunk;
  return make_int4(p.root, a, a + min(p.chunk, rb - a), i == 0 ? 1 : 0);
}

// unit q of a node whose children are [first, first + k)
__device__ __forceinline__ int4 child_unit(const TreeParams &p, int c, int first, int k, int q) {
  const int a = first + q * p.chunk;
  return make_int4(c, a, a + min(p.chunk, first + k - a), q == 0 ? 1 : 0);
}

}  // namespace

// One top-down level of the queue level: the units [lo, hi) taken by the
// warps of the calling group (warp-uniform start `wstart`, stride `stride`, a
// multiple of 32): every child's value set to a leaf's, the units of the
// children with children appended after the level.
template <bool CHAIN>
__device__ __forceinline__ void queue_visit_level(const TreeParams &p, int4 *units, int nroot, int lo, int hi,
                                                  int wstart, int stride, bool root_level, int ra, int rb,
                                                  unsigned long long &visited, unsigned long long &internal) {
  const int lane = lane_id();
  for (int i0 = lo + wstart; i0 < hi; i0 += stride) {  // warp-uniform
    const int i = i0 + lane;
    int a = 0, b = 0, node = -1;
    if (i < hi) {
      const int4 u = root_level ? root_unit(p, i, ra, rb) : __ldcg(units + i);
      if (u.x >= 0) {
        node = u.x;
        a = u.y;
        b = u.z;
      }
    }
    visited += b - a;
    int inner = 0;  // internal children among this unit's
    int nb = ceil_div(b - a, kKidBatch);
    for (int d = kWarp / 2; d >= 1; d >>= 1) nb = max(nb, __shfl_xor_sync(0xffffffffu, nb, d));
    for (int j = 0; j < nb; ++j) {
      const int k0 = a + j * kKidBatch;
      int c[kKidBatch], first[kKidBatch], kc[kKidBatch];
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t)
        c[t] = k0 + t < b ? checked_index(__ldg(p.cidx + k0 + t), p.n, &p.hdr->status) : -1;
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t) {
        first[t] = c[t] >= 0 ? __ldg(p.coff + c[t]) : 0;
        kc[t] = c[t] >= 0 ? __ldg(p.coff + c[t] + 1) : 0;
        checked_range(first[t], kc[t], p.n - 1, &p.hdr->status);
      }
      int mine = 0;
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t) {
        kc[t] -= first[t];
        mine += units_for(p, kc[t]);
      }
      const int inc = warp_inclusive_scan(mine);
      int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
      unsigned long long b0 = 0;
      if (lane == kWarp - 1 && total) b0 = atomicAdd(&p.hdr->cursor, (unsigned long long)total);
      const unsigned long long base = (unsigned long long)nroot + __shfl_sync(0xffffffffu, b0, kWarp - 1);
      if (total && base + (unsigned long long)total > (unsigned long long)p.max_units) {
        if (lane == 0) tree_fail(p, DPC_ERR_OVERFLOW);  // only when the input is not a tree
        for (unsigned long long q = base + lane; q < (unsigned long long)p.max_units && q < base + total; q += kWarp)
          units[q] = make_int4(-1, 0, 0, 0);
        total = 0;
      }
      int pos = total ? (int)base + inc - mine : 0;
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t) {
        if (c[t] >= 0) p.out[c[t]] = 0;
        const int nu = total && c[t] >= 0 ? units_for(p, kc[t]) : 0;
        if (nu) {
          internal++;
          inner++;
          if (CHAIN) {
            // one pending report (its own token; its visit adds its internal
            // children); a node with children is at least 1 high
            p.link[c[t]] = 1ull << 32;
            if (p.op != kDescendants) p.out[c[t]] = 1;
            p.par[c[t]] = node;
          }
        }
        if (nu <= kSmallUnits)
          for (int q = 0; q < nu; ++q) units[pos + q] = child_unit(p, c[t], first[t], kc[t], q);
        // the units of larger children: the whole warp writes them, child by child
        unsigned big = __ballot_sync(0xffffffffu, nu > kSmallUnits);
        while (big) {
          const int src = __ffs(big) - 1;
          big &= big - 1;
          const int bc = __shfl_sync(0xffffffffu, c[t], src), bf = __shfl_sync(0xffffffffu, first[t], src);
          const int bk = __shfl_sync(0xffffffffu, kc[t], src), bp = __shfl_sync(0xffffffffu, pos, src);
          const int bn = __shfl_sync(0xffffffffu, nu, src);
          for (int q = lane; q < bn; q += kWarp) units[bp + q] = child_unit(p, bc, bf, bk, q);
        }
        pos += nu;
      }
    }
    // chained postwork: the node's share from its children known now (1 per
    // child for descendants; the internal ones report the rest later) and its
    // internal-children count, in one atomic on its link word; a node's units
    // are consecutive, so runs of one node are combined over the warp first
    // and one atomic per node and warp remains
    if (!CHAIN) continue;
    unsigned kids = (unsigned)(b - a), inn = (unsigned)inner;
    const int prev = __shfl_up_sync(0xffffffffu, node, 1);
    if (!__any_sync(0xffffffffu, lane > 0 && node >= 0 && prev == node)) {  // no node holds two lanes
      const unsigned long long add = ((unsigned long long)inn << 32) + (p.op == kDescendants ? kids : 0u);
      if (node >= 0 && add) atomicAdd(p.link + node, add);
      continue;
    }
    int start = lane == 0 || prev != node ? lane : 0;
    for (int d = 1; d < kWarp; d <<= 1) start = max(start, __shfl_up_sync(0xffffffffu, start, d));
    for (int d = 1; d < kWarp; d <<= 1) {
      const unsigned ok = __shfl_up_sync(0xffffffffu, kids, d), oi = __shfl_up_sync(0xffffffffu, inn, d);
      if (lane - d >= start) {
        kids += ok;
        inn += oi;
      }
    }
    const int next = __shfl_down_sync(0xffffffffu, node, 1);
    if (node >= 0 && (lane == kWarp - 1 || next != node)) {
      const unsigned long long add = ((unsigned long long)inn << 32) + (p.op == kDescendants ? kids : 0u);
      if (add) atomicAdd(p.link + node, add);
    }
  }
}

// A stretch of consecutive narrow levels run by the calling block alone
// (block barriers between them), from the units [lo, hi) of level `depth`;
// stops at the first wide or empty level and publishes where (the depth and
// that level's units) in the header for the other blocks. Kept out of line
// so that its registers do not weigh on the wide levels' loop.
template <bool CHAIN>
__device__ __forceinline__ void narrow_stretch_body(const TreeParams &p, int nroot, int lo, int hi, int depth,
                                                    unsigned long long *counts) {
  __shared__ int s_hi;
  int4 *const units = reinterpret_cast<int4 *>(p.units);
  const int narrow = 2 * blockDim.x;
  const int ra = __ldg(p.coff + p.root), rb = __ldg(p.coff + p.root + 1);
  unsigned long long visited = 0, internal = 0;
  while (lo < hi && hi - lo <= narrow && depth < p.n) {
    queue_visit_level<CHAIN>(p, units, nroot, lo, hi, threadIdx.x - lane_id(), blockDim.x, depth == 0, ra, rb,
                             visited, internal);
    __syncthreads();  // the level's appends and the cursor are visible to the block
    if (threadIdx.x == 0) {
      s_hi = (int)min((unsigned long long)nroot + *reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                      (unsigned long long)p.max_units);
      p.level_ends[depth + 2] = s_hi;
    }
    __syncthreads();
    lo = hi;
    hi = s_hi;
    ++depth;
  }
  if (threadIdx.x == 0) {  // where the stretch stopped, for the other blocks
    p.hdr->aux[1] = (unsigned long long)depth;
    p.hdr->aux[2] = (unsigned long long)lo;
    p.hdr->aux[3] = (unsigned long long)hi;
  }
  counts[0] += visited;
  counts[1] += internal;
}

// The stretch out of line, one function per postwork form (template
// instances of an out-of-line function lost the kernel's register cap).
__device__ __noinline__ void queue_narrow_stretch_chain(const TreeParams &p, int nroot, int lo, int hi, int depth,
                                                        unsigned long long *counts) {
  narrow_stretch_body<true>(p, nroot, lo, hi, depth, counts);
}

__device__ __noinline__ void queue_narrow_stretch_levels(const TreeParams &p, int nroot, int lo, int hi, int depth,
                                                         unsigned long long *counts) {
  narrow_stretch_body<false>(p, nroot, lo, hi, depth, counts);
}

// One postwork level: units [a0, a1) combine their children's values into
// their node's. A node's units are consecutive, so consecutive lanes of one
// node first combine over the warp and one atomic per node and warp remains.
template <int OP>
__device__ __forceinline__ void queue_post_level(const TreeParams &p, const int4 *units, int a0, int a1, int wstart,
                                                 int stride) {
  const int lane = lane_id();
  for (int i0 = a0 + wstart; i0 < a1; i0 += stride) {  // warp-uniform
    const int i = i0 + lane;
    int node = -1, a = 0, b = 0;
    if (i < a1) {
      const int4 u = __ldcg(units + i);
      node = u.x;
      if (node >= 0) {
        a = u.y;
        b = u.z;
      }
    }
    unsigned v = 0;  // descendants: sum; heights: max
    for (int k0 = a; k0 < b; k0 += kKidBatch) {
      int c[kKidBatch], val[kKidBatch];
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t)
        c[t] = k0 + t < b ? checked_index(__ldg(p.cidx + k0 + t), p.n, &p.hdr->status) : -1;
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t) val[t] = c[t] >= 0 ? __ldcg(p.out + c[t]) : 0;
#pragma unroll
      for (int t = 0; t < kKidBatch; ++t) {
        if (c[t] < 0) continue;
        if (OP == kDescendants) v += 1u + (unsigned)val[t];
        else v = max(v, 1u + (unsigned)val[t]);
      }
    }
    // segmented inclusive scan over runs of equal nodes
    const int prev = __shfl_up_sync(0xffffffffu, node, 1);
    int start = lane == 0 || prev != node ? lane : 0;
    for (int d = 1; d < kWarp; d <<= 1) start = max(start, __shfl_up_sync(0xffffffffu, start, d));
    for (int d = 1; d < kWarp; d <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, v, d);
      if (lane - d >= start) v = OP == kDescendants ? v + o : max(v, o);
    }
    const int next = __shfl_down_sync(0xffffffffu, node, 1);
    if (node >= 0 && (lane == kWarp - 1 || next != node)) {
      if (OP == kDescendants) atomicAdd(reinterpret_cast<unsigned *>(p.out) + node, v);
      else atomicMax(p.out + node, (int)v);
    }
  }
}

// A narrow postwork level run by the calling block alone.
template <int OP>
__device__ __forceinline__ void queue_post_level_block(const TreeParams &p, int a0, int a1) {
  queue_post_level<OP>(p, reinterpret_cast<const int4 *>(p.units), a0, a1, threadIdx.x - lane_id(), blockDim.x);
  __syncthreads();  // the next narrow level reads these values
}

// The chained postwork (trees below 2^24 nodes, see the comment at the head
// of the queue level). link[v] holds v's count of pending reports in its high
// 32 bits (1 for v's own token plus its internal children) and, for
// descendants, its partial value in the low 32 bits, so one atomic both
// reports a child's share and returns everything reported before it: the
// report that takes the count to 0 holds the node's final value. Heights keep
// the value in the output (each report raises it with atomicMax, then takes
// its count, fenced; the last one reads it after a fence): a compare-and-swap
// on the packed word contended at nodes with hundreds of internal children.
// Thread t of T takes units [t, t+T, ...) and removes the token at the first
// unit of each internal node; whichever operation completes a node reports to
// its parent, up the chain.
constexpr unsigned long long kOneReport = 0xFFFFFFFF00000000ull;  // added: one count fewer

template <int OP>
__device__ __forceinline__ void queue_postwork_chain(const TreeParams &p, const int4 *units, int total, int t, int T) {
  for (int i = t; i < total; i += T) {
    const int4 u = __ldcg(units + i);
    if (u.x < 0 || u.w == 0) continue;  // a unit after a node's first (or a placeholder)
    int c = u.x;
    unsigned long long old = atomicAdd(p.link + c, kOneReport);
    if (old >> 32 != 1ull) continue;
    unsigned val;
    if (OP == kDescendants) {
      val = (unsigned)old;
    } else {
      __threadfence();
      val = (unsigned)__ldcg(p.out + c);
    }
    for (;;) {  // c is complete with value val
      const int v = __ldcg(p.par + c);
      if (OP == kDescendants) p.out[c] = (int)val;
      if (v < 0) break;  // the root
      if (OP == kDescendants) {
        old = atomicAdd(p.link + v, (unsigned long long)val + kOneReport);
        if (old >> 32 != 1ull) break;
        val += (unsigned)old;
      } else {
        atomicMax(p.out + v, (int)(val + 1u));
        __threadfence();
        old = atomicAdd(p.link + v, kOneReport);
        if (old >> 32 != 1ull) break;
        __threadfence();
        val = (unsigned)__ldcg(p.out + v);
      }
      c = v;
    }
  }
}

// 64 registers: four 256-thread blocks fit per SM, for wide trees whose
// levels hold millions of units; deep narrow trees run fewer blocks (the host
// sizes the grid), since their levels are short.
//
// Narrow levels (at most two units per thread of one block: most levels of a
// deep tree hold a few units) are not worth a grid barrier each: block 0 runs
// a stretch of consecutive narrow levels alone, separated by block barriers,
// while the other blocks wait at one grid barrier; it publishes where it
// stopped (the depth, and the next level's units) before it arrives. The
// postwork of trees below 2^24 nodes is one pass with no barrier
// (queue_postwork_chain); larger trees, whose wide levels make the visit's
// extra atomics cost more than the barriers, run it level by level bottom-up,
// a narrow level in block 0 alone as above.
template <int OP, bool CHAIN>
__global__ void __maxnreg__(64) tree_queue(TreeParams p) {
  int4 *const units = reinterpret_cast<int4 *>(p.units);
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int wbase = gtid - lane;
  const int ra = __ldg(p.coff + p.root), rb = __ldg(p.coff + p.root + 1);
  const int nroot = units_for(p, rb - ra);
  if (gtid == 0) {
    p.out[p.root] = !CHAIN || OP == kDescendants || rb == ra ? 0 : 1;
    if (CHAIN) {
      p.link[p.root] = 1ull << 32;
      p.par[p.root] = -1;
    }
    p.level_ends[0] = 0;
    p.level_ends[1] = nroot;
  }
  for (int q = gtid; q < nroot; q += G) units[q] = root_unit(p, q, ra, rb);

  unsigned k = 0;
  // the root's value and counters before its units add to them: block 0 alone
  // when the root level is narrow, else every block after a grid barrier
  if (nroot > 2 * (int)blockDim.x) {
    if (!tree_barrier(p, ++k, -1, 0)) return;
  } else {
    __syncthreads();
  }
  int depth = 0;  // unit levels processed
  int lo = 0, hi = nroot;
  unsigned long long visited = 0, internal = 0;
  while (lo < hi && depth < p.n) {
    if (hi - lo <= 2 * (int)blockDim.x) {
      if (blockIdx.x == 0) {
        unsigned long long counts[2] = {0, 0};
        if (CHAIN) queue_narrow_stretch_chain(p, nroot, lo, hi, depth, counts);
        else queue_narrow_stretch_levels(p, nroot, lo, hi, depth, counts);
        visited += counts[0];
        internal += counts[1];
      }
      if (!tree_barrier(p, ++k, -1, 0)) return;
      depth = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[1]);
      lo = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[2]);
      hi = (int)*reinterpret_cast<volatile unsigned long long *>(&p.hdr->aux[3]);
      continue;
    }
    queue_visit_level<CHAIN>(p, units, nroot, lo, hi, wbase, G, depth == 0, ra, rb, visited, internal);
    if (!tree_barrier(p, ++k, depth + 2, nroot)) return;
    lo = hi;
    hi = __ldcg(p.level_ends + depth + 2);
    ++depth;
  }

  if (CHAIN) {
    // postwork: every level's units are [0, hi); every level's visit is done
    queue_postwork_chain<OP>(p, units, hi, gtid, G);
  } else {
    const int narrow = 2 * blockDim.x;
    auto level_narrow = [&](int L) { return __ldcg(p.level_ends + L + 1) - __ldcg(p.level_ends + L) <= narrow; };
    for (int L = depth - 1; L >= 0; --L) {
      const int a0 = __ldcg(p.level_ends + L), a1 = __ldcg(p.level_ends + L + 1);
      if (a1 - a0 <= narrow) {
        if (blockIdx.x == 0) queue_post_level_block<OP>(p, a0, a1);
        if (L > 0 && !level_narrow(L - 1) && !tree_barrier(p, ++k, -1, 0)) return;
      } else {
        queue_post_level<OP>(p, units, a0, a1, wbase, G);
        if (!tree_barrier(p, ++k, -1, 0)) return;
      }
    }
  }
  if (p.stats) {
    visited = warp_sum(visited);
    internal = warp_sum(internal);
    if (lane == 0) {
      stat_add(p.stats, &dpc_stats::relaxations, visited);
      stat_add(p.stats, &dpc_stats::buffered_items, internal);
    }
    if (gtid == 0) atomicMax(&p.stats->rounds, (unsigned)depth + 1u);
  }
}

const void *tree_queue_kernel(int op, bool chain) {
  if (chain) return op == kDescendants ? (const void *)tree_queue<kDescendants, true> : (const void *)tree_queue<kHeight, true>;
  return op == kDescendants ? (const void *)tree_queue<kDescendants, false> : (const void *)tree_queue<kHeight, false>;
}

cudaError_t tree_queue_launch(const TreeParams &p, int blocks, int threads, cudaStream_t s) {
  TreeParams q = p;
  void *args[] = {&q};
  return cudaLaunchCooperativeKernel(tree_queue_kernel(p.op, p.chain != 0), dim3(blocks), dim3(threads), args, 0, s);
}

// ------------------------------------------------------------------ host side

size_t tree_max_units(int n, int chunk) {
  // sum over internal nodes of ceil(k/chunk) <= (n-1)/chunk + #internal
  return (size_t)(n > 0 ? n - 1 : 0) / (size_t)chunk + (size_t)n + 1;
}

size_t tree_units_bytes(int n, dpc_level level, int chunk) {
  if (level == DPC_BASIC_DP) return 0;
  // queue units are (node, first child, end child, -), the others (node, chunk index)
  const size_t unit = level == DPC_QUEUE ? sizeof(int4) : sizeof(int2);
  return align_up(tree_max_units(n, level == DPC_FLAT ? INT_MAX : chunk) * unit, 256);
}

size_t tree_workspace_bytes(int n, dpc_level level, const LaunchCfg &c) {
  size_t b = kHeaderBytes + tree_units_bytes(n, level, c.chunk);
  if (level == DPC_QUEUE) {
    b += align_up(((size_t)n + 2) * sizeof(int), 256);  // where each level's units end
    if (tree_chained_postwork(n))                       // parents and link words of internal nodes
      b += align_up((size_t)n * sizeof(int), 256) + align_up((size_t)n * sizeof(unsigned long long), 256);
  }
  return b;
}

const void *tree_visit_kernel(dpc_level level, int op) {
  const bool d = op == kDescendants;
  switch (level) {
    case DPC_BASIC_DP: return d ? (const void *)tree_visit_node<kDescendants> : (const void *)tree_visit_node<kHeight>;
    case DPC_FLAT: return d ? (const void *)tree_visit<DPC_FLAT, kDescendants> : (const void *)tree_visit<DPC_FLAT, kHeight>;
    case DPC_WARP: return d ? (const void *)tree_visit<DPC_WARP, kDescendants> : (const void *)tree_visit<DPC_WARP, kHeight>;
    case DPC_BLOCK:
      return d ? (const void *)tree_visit<DPC_BLOCK, kDescendants> : (const void *)tree_visit<DPC_BLOCK, kHeight>;
    case DPC_GRID: return d ? (const void *)tree_visit<DPC_GRID, kDescendants> : (const void *)tree_visit<DPC_GRID, kHeight>;
  }
  return nullptr;
}

template <int OP>
static cudaError_t tree_launch_op(TreeParams &p, dpc_level level, int root_blocks, cudaStream_t s,
                                  unsigned *levels_out) {
  cudaError_t e;
  const int T = p.child_threads;
  if (level == DPC_BASIC_DP) {
    tree_init<<<1, 32, 0, s>>>(p);  // value of the root
    tree_visit_node<OP><<<root_blocks, T, 0, s>>>(p, p.root, 0);
    return cudaGetLastError();
  }
  tree_init<<<1, 256, 0, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (level) {
    case DPC_WARP: tree_visit<DPC_WARP, OP><<<root_blocks, T, 0, s>>>(p, p.units, -1, 0); return cudaGetLastError();
    case DPC_BLOCK: tree_visit<DPC_BLOCK, OP><<<root_blocks, T, 0, s>>>(p, p.units, -1, 0); return cudaGetLastError();
    case DPC_GRID: tree_visit<DPC_GRID, OP><<<root_blocks, T, 0, s>>>(p, p.units, -1, 0); return cudaGetLastError();
    default: break;
  }
  // flat: levels top-down from the host, then postwork bottom-up
  unsigned long long &cnt = host_scratch().count;
  cnt = 0;
  if ((e = cudaMemcpyAsync(&cnt, &p.hdr->aux[0], sizeof(cnt), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  std::vector<std::pair<int, int>> levels;
  int start = 0, num = (int)cnt;
  while (num > 0) {
    levels.emplace_back(start, num);
    const int blocks = ceil_div(num, T) < p.child_blocks ? ceil_div(num, T) : p.child_blocks;
    tree_visit<DPC_FLAT, OP><<<blocks, T, 0, s>>>(p, p.units + start, num, (int)levels.size() - 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&cnt, &p.hdr->cursor, sizeof(cnt), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    start += num;
    num = (int)cnt - start;
  }
  for (size_t i = levels.size(); i-- > 0;) {
    const int n = levels[i].second;
    const int blocks = ceil_div(n, 256) < p.child_blocks ? ceil_div(n, 256) : p.child_blocks;
    tree_post<OP><<<blocks, 256, 0, s>>>(p, p.units + levels[i].first, n);
  }
  if (levels_out) *levels_out = (unsigned)levels.size() + 1;
  return cudaGetLastError();
}

cudaError_t tree_launch(TreeParams &p, dpc_level level, int root_blocks, cudaStream_t s, unsigned *levels_out) {
  return p.op == kDescendants ? tree_launch_op<kDescendants>(p, level, root_blocks, s, levels_out)
                              : tree_launch_op<kHeight>(p, level, root_blocks, s, levels_out);
}

}  // namespace dpc
