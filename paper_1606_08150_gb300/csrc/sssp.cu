// Single-source shortest paths at the five consolidation levels and the queue level.
//
// The SSSP kernel of Fig. 1b, applied round after round: every vertex of the
// frontier relaxes its out-edges; a vertex whose out-degree exceeds
// `threshold` is large work. The rounds are Jacobi-style: round r relaxes with
// the distances that the frontier vertices had when the round began (kept in
// each frontier entry), so the set of vertices entering the next frontier -
// and with it every launch count - is independent of the order in which the
// relaxations of a round happen.
//
// Optionally the rounds follow the near-far work split of Davidson, Baxter,
// Garland & Owens (IPDPS 2014): a split distance S (a multiple of `delta`)
// keeps vertices that dropped to d >= S out of the next frontier (the far
// pile); when the frontier runs empty, S moves to the bucket above the
// smallest far distance and those far vertices form the next frontier. The
// far pile is kept implicitly: a vertex is relaxed only while its distance is
// below the current split, and the split only grows, so after a round the far
// pile is exactly the set of vertices with a finite distance >= S, which a
// split finds by scanning the distances (two coalesced passes) instead of
// appending every far drop to a list.
// A finer sub-split s (a multiple of `sub_delta`) holds heavy frontier
// vertices (above the threshold) back while their distance is not below s, so
// that a hub is relaxed once its distance has settled instead of on every
// drop. Without a split every vertex that dropped is in the next frontier.
//
// One round on the device (every level but flat and queue):
//   parent(r)   block 0 first tail-launches commit(r); threads relax short
//               frontier vertices inline and hand long ones to a child
//               (basic-DP: one child per vertex; warp/block/grid: units of
//               `chunk` edges appended to a consolidation buffer and one
//               consolidated child per warp/block/grid, Sec. IV.B-C); heavy
//               vertices held back by the sub-split wait for a later round.
//   commit(r)   runs after parent(r) and all its children (CDP2 tail launch,
//               the device-side replacement for the cudaDeviceSynchronize of
//               Sec. IV.C); it writes the next frontier's entries (vertex,
//               distance, edge range), sends far vertices to the far pile, and
//               its last block tail-launches parent(r+1), or - when the
//               frontier is empty and the far pile is not - the split.
//   split       split_min (smallest distance >= S over all vertices, the new
//               S and s), then split_apply (vertices with distance in [old S,
//               new S) become the frontier), whose last block tail-launches
//               parent(r+1).
// The flat level runs the same kernels from a host loop, reading the frontier
// and far-pile sizes back after every step; the queue level runs every phase
// in one cooperative grid, separated by grid barriers.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "dpc_internal.h"
#include "dpc_runtime.cuh"

namespace cg = cooperative_groups;

namespace dpc {

namespace {

constexpr unsigned kInf = 0xFFFFFFFFu;
constexpr unsigned kNoSplit = 0xFFFFFFFFu;  // a split distance above every finite distance

__device__ __forceinline__ void sssp_fail(const SsspParams &p, unsigned code) {
  set_status(&p.hdr->status, code);
  if (p.stats) atomicCAS(&p.stats->status, 0u, code);
}

template <typename T>
__device__ __forceinline__ T ld_volatile(const T *a) {
  return *reinterpret_cast<const volatile T *>(a);
}

// The state of the running phase: read from the workspace header once per
// block (by thread 0, at kernel start or after a grid barrier) and kept in
// shared memory, since every warp reading the same header words from L2 after
// each barrier serialises in one L2 slice.
struct Phase {
  unsigned long long nf;     // frontier entries of the round (aux[0])
  unsigned long long aux1;   // queue level: entries of the round's list, published after the children
  unsigned long long next;   // entries of the round's list so far (cursor2)
  unsigned long long units;  // units in the buffer
  unsigned S;                // split distance: below it a vertex that dropped joins the next frontier
  unsigned s;                // sub-split: a heavy frontier vertex is relaxed below it
  unsigned S_old;            // (split in progress) the split before it
  unsigned done;             // a split found no vertex at or above S
  unsigned append;           // queue level: the round's parent phase may buffer units
};
__shared__ Phase s_ph;

__device__ __forceinline__ void phase_load(const SsspParams &p) {
  const WsHeader *h = p.hdr;
  s_ph.nf = ld_volatile(&h->aux[0]);
  s_ph.aux1 = ld_volatile(&h->aux[1]);
  s_ph.next = ld_volatile(&h->cursor2);
  s_ph.units = ld_volatile(&h->cursor);
  s_ph.S = ld_volatile(&h->nf_split);
  s_ph.s = ld_volatile(&h->nf_sub);
  s_ph.S_old = ld_volatile(&h->nf_split_old);
  s_ph.done = ld_volatile(&h->nf_done);
  s_ph.append = ld_volatile(&h->nf_append);
}

// Every thread of the block; at the start of a device-launched kernel.
__device__ __forceinline__ void phase_sync(const SsspParams &p) {
  if (threadIdx.x == 0) phase_load(p);
  __syncthreads();
}

// v enters the next frontier once per round (stamp dedup); warp-aggregated append.
__device__ __forceinline__ void push_next(const SsspParams &p, int v, unsigned r) {
  if (atomicExch(p.stamp + v, r) == r) return;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&p.hdr->cursor2, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  if (checked(base + g.thread_rank(), p.n, &p.hdr->status)) p.fnext[base + g.thread_rank()] = v;
}

__device__ __forceinline__ void relax(const SsspParams &p, int v, unsigned du, unsigned w, unsigned r, unsigned S) {
  if (!checked(v, p.n, &p.hdr->status)) return;
  const unsigned long long nd = (unsigned long long)du + w;
  if (nd >= kInf) {
    sssp_fail(p, DPC_ERR_OVERFLOW);
    return;
  }
  const unsigned d = (unsigned)nd;
  if (d < __ldcg(p.dist + v)) {
    atomicMin(p.dist + v, d);  // result unused: a reduction, no round trip (see relax_batch)
    if (d < S) push_next(p, v, r);  // at or above the split: the far pile, which needs no record
  }
}

// Edges a+t, a+t+T, a+t+2T, ... below b, relaxed eight at a time: the eight
// edge loads, then the eight distance reads, then the eight atomicMin, then the
// eight stamp exchanges are each issued back to back, so a batch costs four
// dependent memory round trips instead of four per edge. New next-frontier
// vertices of a batch are appended with one warp-aggregated reservation.
constexpr int kRelaxBatch = 8;

// Edge loads. On graphs whose edge arrays exceed half of L2 the stream is read
// with the evict-first hint, so that it does not push the distances and round
// stamps (gathered at random, reused every round) out of L2; smaller graphs
// keep their edges cached for the next rounds.
__device__ __forceinline__ int edge_col(const SsspParams &p, int e) {
  return p.stream_edges ? __ldcs(p.col + e) : __ldg(p.col + e);
}
__device__ __forceinline__ unsigned edge_w(const SsspParams &p, int e) {
  return p.stream_edges ? __ldcs(p.w + e) : __ldg(p.w + e);
}

// One batch of up to kRelaxBatch edges per lane: v[j] targets, d[j] offered
// distances (kInf: none). Returns the mask of entries that entered the next
// frontier (fresh in this round); a target that dropped to S or more only
// has its distance lowered (the far pile is implicit).
//
// An offer below the distance read here drops the target's distance in this
// round whoever's atomicMin lands first (the value read is at most the one
// the round began with), so the target belongs to the next frontier either
// way: the atomicMin needs no result and is issued as a reduction, and the
// round stamp alone keeps the target from entering the list twice.
__device__ __forceinline__ unsigned relax_batch(const SsspParams &p, const int (&v)[kRelaxBatch],
                                                const unsigned (&d)[kRelaxBatch], unsigned r, unsigned S) {
  unsigned cur[kRelaxBatch];
#pragma unroll
  for (int j = 0; j < kRelaxBatch; ++j) cur[j] = (v[j] >= 0 && d[j] != kInf) ? __ldcg(p.dist + v[j]) : 0u;
  unsigned improved = 0;
#pragma unroll
  for (int j = 0; j < kRelaxBatch; ++j)
    if (d[j] < cur[j]) {
      atomicMin(p.dist + v[j], d[j]);
      improved |= 1u << j;
    }
  unsigned fresh = 0;
#pragma unroll
  for (int j = 0; j < kRelaxBatch; ++j)
    if ((improved >> j & 1u) && d[j] < S && atomicExch(p.stamp + v[j], r) != r) fresh |= 1u << j;
  return fresh;
}

// In the full-warp loops adjacent lanes hold adjacent edges. An edge whose
// target is the previous lane's and whose offer is not lower adds nothing
// (the previous lane's offer, or a lower one before it, is relaxed), so it is
// dropped before the atomics. Duplicate edges are adjacent in a CSR sorted by
// target, and an R-MAT hub holds thousands of them: without this their
// atomicMin on one address serialise.
__device__ __forceinline__ void drop_adjacent_duplicates(const int (&v)[kRelaxBatch], unsigned (&d)[kRelaxBatch]) {
  const bool first = lane_id() == 0;
#pragma unroll
  for (int j = 0; j < kRelaxBatch; ++j) {
    const int pv = __shfl_up_sync(0xffffffffu, v[j], 1);
    const unsigned pd = __shfl_up_sync(0xffffffffu, d[j], 1);
    if (!first && pv == v[j] && pd <= d[j]) d[j] = kInf;
  }
}

__device__ __forceinline__ void relax_edges(const SsspParams &p, int a, int b, unsigned du, unsigned r, unsigned S,
                                            int t, int T) {
  for (int e0 = a + t; e0 < b; e0 += kRelaxBatch * T) {
    int v[kRelaxBatch];
    unsigned d[kRelaxBatch];
#pragma unroll
    for (int j = 0; j < kRelaxBatch; ++j) {
      const int e = e0 + j * T;
      v[j] = -1;
      d[j] = kInf;
      if (e < b) {
        const unsigned long long nd = (unsigned long long)du + edge_w(p, e);
        v[j] = checked_index(edge_col(p, e), p.n, &p.hdr->status);
        if (nd >= kInf) sssp_fail(p, DPC_ERR_OVERFLOW);
        else d[j] = (unsigned)nd;
      }
    }
    const unsigned fresh = relax_batch(p, v, d, r, S);
    const int cnt = __popc(fresh);
    cg::coalesced_group g = cg::coalesced_threads();
    const int excl = cg::exclusive_scan(g, cnt);
    const int total = g.shfl(excl + cnt, g.size() - 1);
    unsigned long long base = 0;
    if (g.thread_rank() == 0 && total) base = atomicAdd(&p.hdr->cursor2, (unsigned long long)total);
    base = g.shfl(base, 0) + excl;
#pragma unroll
    for (int j = 0; j < kRelaxBatch; ++j)
      if ((fresh >> j & 1u) && checked(base, p.n, &p.hdr->status)) p.fnext[base++] = v[j];
  }
}

// Per-warp staging of next-frontier vertices in shared memory: a full warp
// relaxing units appends its fresh vertices to its own buffer and reserves
// space in the global list only when the buffer would overflow (and once at
// the end), instead of one atomic on the list's single counter per batch.
constexpr int kStage = 256;
// one batch of the whole warp (32 lanes x kRelaxBatch new vertices at most)
// must fit into an emptied stage: the appends of a batch are not checked again
static_assert(kStage >= kWarp * kRelaxBatch, "a warp's relaxation batch must fit in its stage");
constexpr size_t kHeapHead = 16;  // a device-heap buffer: completion counter, padding, then int4 units

struct WarpStage {
  int *buf;  // kStage entries of this warp
  int *cnt;  // entries held
};

__device__ __forceinline__ void stage_flush(const SsspParams &p, const WarpStage &ws) {
  const int c = *ws.cnt;
  __syncwarp();
  if (c == 0) return;
  unsigned long long base = 0;
  if (lane_id() == 0) base = atomicAdd(&p.hdr->cursor2, (unsigned long long)c);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int i = lane_id(); i < c; i += kWarp)
    if (checked(base + i, p.n, &p.hdr->status)) p.fnext[base + i] = ws.buf[i];
  __syncwarp();
  if (lane_id() == 0) *ws.cnt = 0;
  __syncwarp();
}

// Dynamic shared memory of a child grid of `threads` threads.
__host__ __device__ __forceinline__ size_t stage_bytes(int threads) {
  return (size_t)(threads / kWarp) * (kStage + 1) * sizeof(int);
}

// A full warp stages the fresh vertices of one batch (every lane calls it).
__device__ __forceinline__ void stage_batch(const SsspParams &p, const WarpStage &ws, unsigned fresh,
                                            const int (&v)[kRelaxBatch]) {
  const int cnt = __popc(fresh);
  const int inc = warp_inclusive_scan(cnt);
  const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
  if (total == 0) return;
  if (*ws.cnt + total > kStage) stage_flush(p, ws);
  int pos = *ws.cnt + inc - cnt;
#pragma unroll
  for (int j = 0; j < kRelaxBatch; ++j)
    if ((fresh >> j & 1u) && checked(pos, kStage, &p.hdr->status)) ws.buf[pos++] = v[j];
  __syncwarp();
  if (lane_id() == kWarp - 1) *ws.cnt += total;
  __syncwarp();
}

// relax_edges for a full warp (t = lane, T = 32) with staged appends
__device__ __forceinline__ void relax_edges_staged(const SsspParams &p, int a, int b, unsigned du, unsigned r,
                                                   unsigned S, const WarpStage &ws) {
  const int t = lane_id(), T = kWarp;
  for (int e0 = a + t; e0 - t < b; e0 += kRelaxBatch * T) {
    int v[kRelaxBatch];
    unsigned d[kRelaxBatch];
#pragma unroll
    for (int j = 0; j < kRelaxBatch; ++j) {
      const int e = e0 + j * T;
      v[j] = -1;
      d[j] = kInf;
      if (e < b) {
        const unsigned long long nd = (unsigned long long)du + edge_w(p, e);
        v[j] = checked_index(edge_col(p, e), p.n, &p.hdr->status);
        if (nd >= kInf) sssp_fail(p, DPC_ERR_OVERFLOW);
        else d[j] = (unsigned)nd;
      }
    }
    drop_adjacent_duplicates(v, d);
    stage_batch(p, ws, relax_batch(p, v, d, r, S), v);
  }
}

// Inline work of a full warp over the short vertices of its lanes (edges
// [a, b) of the calling lane when `active`): the lanes' edge lists are
// concatenated and dealt out evenly, eight edges per lane and batch, adjacent
// lanes on adjacent edges, so the warp needs ceil(sum of degrees / 256)
// batches instead of as many as its longest vertex has. An edge's vertex is
// the last lane whose exclusive prefix of degrees is not above the edge's
// position (a five-step search over the warp's prefix sums).
__device__ __forceinline__ void relax_inline_warp(const SsspParams &p, int a, int b, unsigned du, unsigned r,
                                                  unsigned S, bool active, const WarpStage &ws) {
  const int lane = lane_id();
  const int deg = active ? b - a : 0;
  const int incl = warp_inclusive_scan(deg);
  const int total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
  const int excl = incl - deg;
  for (int base = 0; base < total; base += kWarp * kRelaxBatch) {
    int v[kRelaxBatch];
    unsigned d[kRelaxBatch];
#pragma unroll
    for (int j = 0; j < kRelaxBatch; ++j) {
      const int k = base + j * kWarp + lane;
      int owner = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int m = owner + step;
        if (__shfl_sync(0xffffffffu, excl, m) <= k) owner = m;
      }
      const int e = __shfl_sync(0xffffffffu, a, owner) + k - __shfl_sync(0xffffffffu, excl, owner);
      const unsigned dl = __shfl_sync(0xffffffffu, du, owner);
      v[j] = -1;
      d[j] = kInf;
      if (k < total) {
        const unsigned long long nd = (unsigned long long)dl + edge_w(p, e);
        v[j] = checked_index(edge_col(p, e), p.n, &p.hdr->status);
        if (nd >= kInf) sssp_fail(p, DPC_ERR_OVERFLOW);
        else d[j] = (unsigned)nd;
      }
    }
    drop_adjacent_duplicates(v, d);
    stage_batch(p, ws, relax_batch(p, v, d, r, S), v);
  }
}

// All edges of u by one thread, in order (inline work of a parent thread).
__device__ __forceinline__ void relax_all(const SsspParams &p, int a, int b, unsigned du, unsigned r, unsigned S) {
  relax_edges(p, a, b, du, r, S, 0, 1);
}

// A unit: (first edge, end edge, distance of its vertex, vertex); a unit whose
// range is empty is a placeholder written after a buffer overflow.
__device__ __forceinline__ void sssp_units_by_group(const SsspParams &p, const int4 *units, int lo, int hi,
                                                    int warp_in_group, int warps_in_group, unsigned r, unsigned S) {
  for (int u = lo + warp_in_group; u < hi; u += warps_in_group) {
    const int4 un = units[u];
    relax_edges(p, un.x, un.y, (unsigned)un.z, r, S, lane_id(), kWarp);
  }
}



// The split state every thread of a phase reads once (it changes only between phases).
struct Split {
  unsigned S;      // near: distance below S
  unsigned s;      // a heavy near vertex is relaxed when its distance is below s
  unsigned S_old;  // (split in progress) the split before it
};

__device__ __forceinline__ Split read_split() {
  Split q;
  q.S = s_ph.S;
  q.s = s_ph.s;
  q.S_old = s_ph.S_old;
  return q;
}

// Does the next round relax this frontier entry? Light vertices always; a
// heavy one only below the sub-split.
__device__ __forceinline__ bool relaxed_now(const SsspParams &p, const int4 &f, unsigned s) {
  return f.w - f.z <= p.threshold || (unsigned)f.y < s;
}

// What the entries appended by a thread mean for the next round: how many of
// them it relaxes, and the smallest distance of a heavy one that waits. Kept
// in registers and added to the header once per warp at the end of a pass
// (flush_near), instead of two more same-address atomics per warp step.
struct NearAcc {
  unsigned long long elig = 0;
  unsigned hmin = kInf;
  unsigned long long pre_edges = 0, pre_items = 0;  // heavy entries buffered ahead (prebuffer)
};

// Queue level (p.prebuffer): a heavy entry that the next round relaxes for
// sure (below the sub-split, which never moves down) goes straight into the
// unit buffer as its units, instead of into the frontier for the next round's
// parent phase to buffer. The next round then needs no grid barrier between
// its parent phase and its consolidated loop, unless the sub-split has to
// advance first (then heavy frontier entries become eligible only in that
// round: nf_append). Returns the entries it could not buffer (only when the
// buffer overflows, which valid input cannot make happen).
template <int N>
__device__ __forceinline__ unsigned buffer_ahead(const SsspParams &p, unsigned pre, const int (&v)[N],
                                                 const unsigned (&dv)[N], const int (&a)[N], const int (&b)[N],
                                                 NearAcc &acc) {
  int nu[N], mine = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    nu[j] = pre >> j & 1u ? ceil_div(b[j] - a[j], p.chunk) : 0;
    mine += nu[j];
  }
  const int inc = warp_inclusive_scan(mine);
  const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
  if (total == 0) return 0u;
  unsigned long long base = 0;
  if (lane_id() == kWarp - 1) base = atomicAdd(&p.hdr->cursor, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, kWarp - 1);
  if (base + (unsigned long long)total > (unsigned long long)p.max_units) {
    if (lane_id() == 0) sssp_fail(p, DPC_ERR_OVERFLOW);
    return pre;
  }
  int pos = (int)base + inc - mine;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    for (int q = 0; q < nu[j]; ++q) {
      const int ua = a[j] + q * p.chunk;
      p.units[pos + q] = make_int4(ua, min(b[j], ua + p.chunk), (int)dv[j], v[j]);
    }
    pos += nu[j];
    if (nu[j]) {
      acc.elig++;
      acc.pre_items++;
      acc.pre_edges += (unsigned long long)(b[j] - a[j]);
    }
  }
  return 0u;
}

// A full warp appends up to N entries per lane (entry j when bit j of `near`
// is set) to the next frontier: (v, d, first edge, end edge) at consecutive
// slots of one reservation per warp step.
template <int N>
__device__ __forceinline__ void append_near(const SsspParams &p, unsigned near, const int (&v)[N],
                                            const unsigned (&dv)[N], const int (&a)[N], const int (&b)[N], unsigned s,
                                            NearAcc &acc) {
  if (p.prebuffer) {
    unsigned pre = 0;
#pragma unroll
    for (int j = 0; j < N; ++j)
      if ((near >> j & 1u) && b[j] - a[j] > p.threshold && dv[j] < s) pre |= 1u << j;
    if (__any_sync(0xffffffffu, pre != 0)) near = (near & ~pre) | buffer_ahead<N>(p, pre, v, dv, a, b, acc);
  }
  const int cnt = __popc(near);
  const int inc = warp_inclusive_scan(cnt);
  const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane_id() == kWarp - 1) base = atomicAdd(&p.hdr->nf_near, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, kWarp - 1) + (unsigned long long)(inc - cnt);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (!(near >> j & 1u)) continue;
    const int4 f = make_int4(v[j], (int)dv[j], a[j], b[j]);
    if (checked(base, p.n, &p.hdr->status)) p.fcur[base++] = f;
    if (relaxed_now(p, f, s)) acc.elig++;
    else if (dv[j] < acc.hmin) acc.hmin = dv[j];
  }
}

__device__ __forceinline__ void flush_near(const SsspParams &p, const NearAcc &acc) {
  const unsigned long long e = warp_sum(acc.elig);
  const unsigned h = __reduce_min_sync(0xffffffffu, acc.hmin);
  if (lane_id() == 0) {
    if (e) atomicAdd(&p.hdr->nf_elig, e);
    if (h != kInf) atomicMin(&p.hdr->nf_hmin, h);
  }
}

// Commit of one entry of the round's list (called by full warps; `valid`
// false for lanes past the end): every listed vertex is below the split (a
// vertex that dropped to the split or above stayed in the far pile), so it
// becomes a next-frontier entry with the distance and edge range it has now.
__device__ __forceinline__ void commit_vertex(const SsspParams &p, bool valid, int v, const Split &q,
                                              NearAcc &acc) {
  int vv[1] = {v}, a[1] = {0}, b[1] = {0};
  unsigned dv[1] = {kInf};
  if (valid) {
    dv[0] = __ldcg(p.dist + v);
    a[0] = __ldg(p.off + v);
    b[0] = __ldg(p.off + v + 1);
    checked_range(a[0], b[0], p.m, &p.hdr->status);
  }
  append_near<1>(p, valid ? 1u : 0u, vv, dv, a, b, q.s, acc);
}

// The split's passes read every distance, four per 16-byte load when the
// array allows (the caller's array may start anywhere; then one at a time).
// Thread t of T takes vertices 4t..4t+3, then 4(t+T).., so a warp reads 512
// consecutive bytes per step.

// Split, first pass, over every vertex: the smallest finite distance at or
// above S (the far pile: those vertices dropped to S or more and have not
// been relaxed since). Called by every thread of a grid of T threads (thread
// t); one reduction per warp at the end.
__device__ __forceinline__ void split_min_pass(const SsspParams &p, const Split &q, int t, int T) {
  unsigned m = kInf;
  auto take = [&](unsigned dv) {
    if (dv >= q.S && dv < m) m = dv;  // kInf (unreached) never lowers m
  };
  if ((reinterpret_cast<uintptr_t>(p.dist) & 15u) == 0) {
    const uint4 *d4 = reinterpret_cast<const uint4 *>(p.dist);
    const int n4 = p.n >> 2;
    for (int i = t; i < n4; i += T) {
      const uint4 v = __ldcg(d4 + i);
      take(v.x);
      take(v.y);
      take(v.z);
      take(v.w);
    }
    for (int v = (n4 << 2) + t; v < p.n; v += T) take(__ldcg(p.dist + v));
  } else {
    for (int v = t; v < p.n; v += T) take(__ldcg(p.dist + v));
  }
  m = __reduce_min_sync(0xffffffffu, m);
  if (lane_id() == 0 && m != kInf) atomicMin(&p.hdr->nf_dmin, m);
}

// Split, second pass, over every vertex (S and s are the new ones): the far
// vertices below the new S (distance in [old S, new S)) form the next
// frontier. Called by every thread of a grid of T threads (T a multiple of 32).
// Out of line: it runs once per split, and inlined its registers weighed on
// the queue kernel's round loop (more spills under the kernel's cap).
__device__ __noinline__ void split_apply_pass(const SsspParams &p, const Split &q, int t, int T, NearAcc &acc) {
  auto in_bucket = [&](unsigned dv) { return dv >= q.S_old && dv < q.S; };
  const int base = t - (int)lane_id();  // warp-uniform loops: the appends need the whole warp
  const bool vec = (reinterpret_cast<uintptr_t>(p.dist) & 15u) == 0;
  const int n4 = vec ? p.n >> 2 : 0;
  const uint4 *d4 = reinterpret_cast<const uint4 *>(p.dist);
  for (int i0 = base; i0 < n4; i0 += T) {
    const int i = i0 + (int)lane_id();
    unsigned dv[4] = {kInf, kInf, kInf, kInf};
    if (i < n4) {
      const uint4 x = __ldcg(d4 + i);
      dv[0] = x.x;
      dv[1] = x.y;
      dv[2] = x.z;
      dv[3] = x.w;
    }
    unsigned near = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (in_bucket(dv[j])) near |= 1u << j;
    if (!__any_sync(0xffffffffu, near != 0)) continue;
    int v[4], a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = 4 * i + j;
      a[j] = b[j] = 0;
      if (near >> j & 1u) {
        a[j] = __ldg(p.off + v[j]);
        b[j] = __ldg(p.off + v[j] + 1);
        checked_range(a[j], b[j], p.m, &p.hdr->status);
      }
    }
    append_near<4>(p, near, v, dv, a, b, q.s, acc);
  }
  for (int v0 = 4 * n4 + base; v0 < p.n; v0 += T) {  // the rest one at a time
    int v[1] = {v0 + (int)lane_id()}, a[1] = {0}, b[1] = {0};
    unsigned dv[1] = {v[0] < p.n ? __ldcg(p.dist + v[0]) : kInf};
    const unsigned near = in_bucket(dv[0]) ? 1u : 0u;
    if (near) {
      a[0] = __ldg(p.off + v[0]);
      b[0] = __ldg(p.off + v[0] + 1);
      checked_range(a[0], b[0], p.m, &p.hdr->status);
    }
    append_near<1>(p, near, v, dv, a, b, q.s, acc);
  }
  flush_near(p, acc);
}

// The top of the width-w bucket of distance d, at most all ones.
__device__ __forceinline__ unsigned bucket_top(unsigned d, unsigned w) {
  const unsigned long long t = ((unsigned long long)d / w + 1) * (unsigned long long)w;
  return t < kNoSplit ? (unsigned)t : kNoSplit;
}

// Make the near set written by a commit or a split the next round's frontier
// (single thread, after every block has finished the phase). When none of its
// entries would be relaxed (only heavy vertices at or above the sub-split),
// the sub-split first moves to the top of the smallest one's sub-bucket.
__device__ __forceinline__ void publish_frontier(const SsspParams &p) {
  WsHeader *h = p.hdr;
  const unsigned long long nn = ld_volatile(&h->nf_near);
  const bool advance = nn > 0 && ld_volatile(&h->nf_elig) == 0 && p.sub_delta;
  if (advance) h->nf_sub = bucket_top(ld_volatile(&h->nf_hmin), p.sub_delta);
  h->aux[0] = nn;
  h->nf_near = 0ull;
  h->nf_elig = 0ull;
  h->nf_hmin = kInf;
  h->cursor2 = 0ull;
  // queue level: the unit buffer holds the next round's units buffered ahead
  // (it was emptied after the children); only a sub-split advance leaves
  // heavy frontier entries for the parent phase to buffer
  if (p.prebuffer) h->nf_append = advance ? 1u : 0u;
  else h->cursor = 0ull;
  h->aux[2] = 0ull;    // the grid-level child's unit cursor
  h->launches = 0ull;  // the round's children have all finished: their pool slots are free
}

// The split's new S and s from the smallest far distance (single thread).
// Returns false, and marks the run done, when no vertex is at or above S.
__device__ __forceinline__ bool advance_split(const SsspParams &p) {
  WsHeader *h = p.hdr;
  const unsigned dmin = ld_volatile(&h->nf_dmin);
  h->nf_dmin = kInf;
  if (dmin == kInf) {
    h->nf_done = 1u;
    return false;
  }
  h->nf_split_old = ld_volatile(&h->nf_split);
  h->nf_split = bucket_top(dmin, p.delta);
  if (p.sub_delta) h->nf_sub = bucket_top(dmin, p.sub_delta);
  return true;
}

// After split_apply: the far vertices it took are the next frontier.
__device__ __forceinline__ void finish_split(const SsspParams &p) { publish_frontier(p); }

}  // namespace

__global__ void sssp_commit(SsspParams p, unsigned r);

// ------------------------------------------------------------------ kernels

__global__ void __launch_bounds__(1024) sssp_init(SsspParams p) {
  const int G = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += G) {
    p.dist[v] = v == p.source ? 0u : kInf;
    p.stamp[v] = kInf;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int a = __ldg(p.off + p.source), b = __ldg(p.off + p.source + 1);
    checked_range(a, b, p.m, &p.hdr->status);
    p.fcur[0] = make_int4(p.source, 0, a, b);
    WsHeader *h = p.hdr;
    h->aux[0] = 1ull;
    h->nf_split = p.delta ? p.delta : kNoSplit;
    h->nf_sub = p.sub_delta ? p.sub_delta : kNoSplit;
    h->nf_split_old = 0u;
    h->nf_dmin = kInf;
    h->nf_hmin = kInf;
    h->nf_append = 1u;  // the source's units (if it is heavy) are buffered by round 0's parent phase
  }
}

// Consolidated child: warps take units round-robin, or - when the child is the
// only one of its round (grid level) - one to four at a time from a shared
// cursor, so that no warp is left with a long tail of work. New frontier
// vertices are staged per warp (see relax_edges_staged).
__global__ void __launch_bounds__(1024) sssp_child(SsspParams p, const int4 *__restrict__ units, int nunits,
                                                  unsigned r, unsigned long long *cursor, unsigned *heap_block) {
  extern __shared__ int s_stage[];  // per warp: kStage entries, then the count (stage_bytes)
  const int wib = threadIdx.x >> 5;
  WarpStage ws{s_stage + wib * (kStage + 1), s_stage + wib * (kStage + 1) + kStage};
  if (lane_id() == 0) *ws.cnt = 0;
  phase_sync(p);
  const unsigned S = s_ph.S;
  auto unit = [&](int4 u) { relax_edges_staged(p, u.x, u.y, (unsigned)u.z, r, S, ws); };
  if (cursor) {
    // every warp's first unit is its own (no atomic while units are fewer than
    // warps); the rest come from the shared cursor
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (gw < nunits) unit(units[gw]);
    if (nunits > nw) {
      const unsigned long long grab = units_per_grab(nunits - nw, nw);
      for (;;) {
        unsigned long long i0 = 0;
        if (lane_id() == 0) i0 = atomicAdd(cursor, grab) + (unsigned long long)nw;
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        if (i0 >= (unsigned long long)nunits) break;
        const int i1 = (int)min(i0 + grab, (unsigned long long)nunits);
        for (int u = (int)i0; u < i1; ++u) unit(units[u]);
      }
    }
  } else {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = gw; u < nunits; u += nw) unit(units[u]);
  }
  stage_flush(p, ws);
  // a buffer from the device heap: the grid's last block to finish returns it
  if (heap_block && last_block_done(heap_block) && threadIdx.x == 0) free(heap_block);
}

// Basic-DP child (Fig. 1b's process_neighbors): thread per edge of one vertex.
__global__ void __launch_bounds__(1024) sssp_vertex_child(SsspParams p, int a, int b, unsigned du, unsigned r) {
  phase_sync(p);
  const int e = a + blockIdx.x * blockDim.x + threadIdx.x;
  if (e < b) relax(p, edge_col(p, e), du, edge_w(p, e), r, s_ph.S);
}

__device__ __forceinline__ void round_prologue(const SsspParams &p, unsigned r) {
  // the round's commit waits for this grid and every child it launches
  if (p.level != DPC_FLAT && blockIdx.x == 0 && threadIdx.x == 0) {
    sssp_commit<<<p.commit_blocks, 256, 0, cudaStreamTailLaunch>>>(p, r);
    if (cudaGetLastError() != cudaSuccess) sssp_fail(p, DPC_ERR_DEVICE);
    else stat_add(p.stats, &dpc_stats::aux_launches, 1);
  }
}

__device__ __forceinline__ void round_stats(const SsspParams &p, unsigned long long relaxed,
                                            unsigned long long inl, unsigned long long buf,
                                            unsigned long long launched, unsigned long long failed) {
  if (!p.stats) return;
  relaxed = warp_sum(relaxed);
  inl = warp_sum(inl);
  buf = warp_sum(buf);
  launched = warp_sum(launched);
  failed = warp_sum(failed);
  if (lane_id() == 0) {
    stat_add(p.stats, &dpc_stats::relaxations, relaxed);
    stat_add(p.stats, &dpc_stats::inline_items, inl);
    stat_add(p.stats, &dpc_stats::buffered_items, buf);
    stat_add(p.stats, &dpc_stats::child_launches, launched);
    stat_add(p.stats, &dpc_stats::launch_failures, failed);
  }
}

// Flat and basic-DP parent: thread per frontier vertex.
template <int LEVEL>
__global__ void __launch_bounds__(1024) sssp_parent_simple(SsspParams p, unsigned r) {
  round_prologue(p, r);
  phase_sync(p);
  const int nf = (int)s_ph.nf;
  const unsigned s = s_ph.s;
  const unsigned S = s_ph.S;
  const int G = gridDim.x * blockDim.x;
  unsigned long long relaxed = 0, inl = 0, buf = 0, launched = 0, failed = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += G) {
    const int4 f = p.fcur[i];
    if (!relaxed_now(p, f, s)) {  // a heavy vertex above the sub-split waits for a later round
      push_next(p, f.x, r);
      continue;
    }
    const int a = f.z, b = f.w;
    relaxed += b - a;
    if (LEVEL == DPC_BASIC_DP && b - a > p.threshold) {
      buf++;
      if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
        sssp_vertex_child<<<ceil_div(b - a, p.child_threads), p.child_threads, 0, cudaStreamFireAndForget>>>(
            p, a, b, (unsigned)f.y, r);
        if (cudaGetLastError() == cudaSuccess) {
          launched++;
          continue;
        }
      }
      failed++;
    } else {
      inl++;
    }
    relax_all(p, a, b, (unsigned)f.y, r, S);
  }
  round_stats(p, relaxed, inl, buf, launched, failed);
}

// Warp-, block- and grid-level parent: the two-pass buffer insertion of the
// SpMV parent (count, reserve the group's slice with one atomic, write at
// scanned offsets), then one launch per warp / block / grid (Fig. 4b).
template <int LEVEL>
__global__ void __launch_bounds__(1024) sssp_parent(SsspParams p, unsigned r) {
  __shared__ int s_scan[33];
  __shared__ int s_base, s_fail;
  __shared__ unsigned *s_heap;
  extern __shared__ int s_stage[];  // per warp: kStage entries, then the count (stage_bytes)
  const WarpStage ws{s_stage + (threadIdx.x >> 5) * (kStage + 1), s_stage + (threadIdx.x >> 5) * (kStage + 1) + kStage};
  if (lane_id() == 0) *ws.cnt = 0;
  __syncwarp();
  round_prologue(p, r);
  phase_sync(p);
  const int nf = (int)s_ph.nf;
  const unsigned sub = s_ph.s;
  const unsigned S = s_ph.S;
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int bstart = blockIdx.x * blockDim.x;

  int mine = 0;
  for (int i = bstart + threadIdx.x; i < nf; i += G) {
    const int4 f = p.fcur[i];
    const int deg = f.w - f.z;
    if (deg > p.threshold && relaxed_now(p, f, sub)) mine += ceil_div(deg, p.chunk);
  }
  // The group's buffer: a slice of the workspace pool, or (p.heap, warp and
  // block levels) a block of its own from the device heap, the paper's
  // default allocator (Sec. IV.E): a completion counter, then the units.
  const bool heap = (LEVEL == DPC_WARP || LEVEL == DPC_BLOCK) && p.heap;
  int base, gtotal;
  int4 *ubuf = p.units;
  unsigned *hblk = nullptr;
  unsigned long long failed = 0;
  if (LEVEL == DPC_BLOCK) {
    gtotal = block_sum(mine, s_scan);
    if (threadIdx.x == 0) {
      s_base = 0;
      s_heap = nullptr;
      if (gtotal && heap) {
        s_heap = static_cast<unsigned *>(malloc(kHeapHead + (size_t)gtotal * sizeof(int4)));
        if (s_heap) *s_heap = 0u;
        else failed++;  // no buffer: the block relaxes these vertices itself
      } else if (gtotal) {
        s_base = (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal);
      }
    }
    __syncthreads();
    base = s_base;
    hblk = s_heap;
    if (heap && !hblk) gtotal = 0;
    if (!heap && base + gtotal > p.max_units) {  // only reachable with malformed input
      if (threadIdx.x == 0) sssp_fail(p, DPC_ERR_OVERFLOW);
      for (int j = base + threadIdx.x; j < min(base + gtotal, p.max_units); j += blockDim.x)
        p.units[j] = make_int4(0, 0, 0, -1);
      gtotal = 0;
    }
  } else {
    gtotal = warp_sum(mine);
    unsigned long long b0 = 0;  // the slice's start, or the heap block's address
    if (lane == 0 && gtotal) {
      if (heap) {
        void *h = malloc(kHeapHead + (size_t)gtotal * sizeof(int4));
        if (h) *static_cast<unsigned *>(h) = 0u;
        else failed++;  // no buffer: the warp relaxes these vertices itself
        b0 = reinterpret_cast<unsigned long long>(h);
      } else {
        b0 = atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal);
      }
    }
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    base = heap ? 0 : (int)b0;
    if (heap) {
      hblk = reinterpret_cast<unsigned *>(b0);
      if (!hblk) gtotal = 0;
    } else if (base + gtotal > p.max_units) {  // only reachable with malformed input
      if (lane == 0) sssp_fail(p, DPC_ERR_OVERFLOW);
      for (int j = base + lane; j < min(base + gtotal, p.max_units); j += kWarp) p.units[j] = make_int4(0, 0, 0, -1);
      gtotal = 0;
    }
  }
  if (hblk) ubuf = reinterpret_cast<int4 *>(reinterpret_cast<char *>(hblk) + kHeapHead);

  int run = base;
  unsigned long long relaxed = 0, inl = 0, buf = 0, launched = 0;
  for (int i0 = bstart; i0 < nf; i0 += G) {
    const int i = i0 + threadIdx.x;
    int nu = 0, a = 0, b = 0;
    int4 f = make_int4(0, 0, 0, 0);
    bool work = false;
    if (i < nf) {
      f = p.fcur[i];
      if (relaxed_now(p, f, sub)) {
        work = true;
        a = f.z;
        b = f.w;
        relaxed += b - a;
        if (gtotal && b - a > p.threshold) nu = ceil_div(b - a, p.chunk);
      } else {
        push_next(p, f.x, r);  // a heavy vertex above the sub-split waits for a later round
      }
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
      for (int k = 0; k < nu; ++k) {
        const int ua = a + k * p.chunk;
        ubuf[pos + k] = make_int4(ua, min(b, ua + p.chunk), f.y, f.x);
      }
      buf++;
    } else if (work) {
      inl++;
    }
    relax_inline_warp(p, a, b, (unsigned)f.y, r, S, work && nu == 0, ws);
    run += step;
  }
  stage_flush(p, ws);

  if (LEVEL == DPC_WARP) {
    __threadfence();
    __syncwarp();
    if (gtotal) {
      int fl = 0;
      if (lane == 0) {
        fl = 1;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          sssp_child<<<child_grid_for(gtotal, p.child_blocks, p.child_threads), p.child_threads,
                       stage_bytes(p.child_threads),
                       cudaStreamFireAndForget>>>(p, ubuf + base, gtotal, r, nullptr, hblk);
          fl = cudaGetLastError() != cudaSuccess;
        }
        if (fl) failed++;
        else launched++;
      }
      fl = __shfl_sync(0xffffffffu, fl, 0);
      if (fl) {
        sssp_units_by_group(p, ubuf, base, base + gtotal, 0, 1, r, S);
        __syncwarp();
        if (lane == 0 && hblk) free(hblk);
      }
    }
  } else if (LEVEL == DPC_BLOCK) {
    __threadfence();
    __syncthreads();
    if (gtotal) {
      if (threadIdx.x == 0) {
        s_fail = 1;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          sssp_child<<<child_grid_for(gtotal, p.child_blocks, p.child_threads), p.child_threads,
                       stage_bytes(p.child_threads),
                       cudaStreamFireAndForget>>>(p, ubuf + base, gtotal, r, nullptr, hblk);
          s_fail = cudaGetLastError() != cudaSuccess;
        }
        if (s_fail) failed++;
        else launched++;
      }
      __syncthreads();
      if (s_fail) {
        sssp_units_by_group(p, ubuf, base, base + gtotal, threadIdx.x >> 5, blockDim.x >> 5, r, S);
        __syncthreads();
        if (threadIdx.x == 0 && hblk) free(hblk);
      }
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
            sssp_child<<<child_grid_for(total, p.child_blocks, p.child_threads), p.child_threads,
                         stage_bytes(p.child_threads),
                         cudaStreamFireAndForget>>>(p, p.units, total, r, &p.hdr->aux[2], nullptr);
            s_fail = cudaGetLastError() != cudaSuccess;
          }
          if (s_fail) failed++;
          else launched++;
        }
      }
      __syncthreads();
      if (s_fail) sssp_units_by_group(p, p.units, 0, s_base, threadIdx.x >> 5, blockDim.x >> 5, r, S);
    }
  }
  round_stats(p, relaxed, inl, buf, launched, failed);
}

// Launch the parent of round r for a frontier of nf vertices (device side).
__device__ void launch_parent(const SsspParams &p, unsigned r, int nf, cudaStream_t s) {
  const int need = ceil_div(nf, p.parent_threads);
  const int blocks = need < p.parent_blocks ? (need > 0 ? need : 1) : p.parent_blocks;
  switch (p.level) {
    case DPC_BASIC_DP: sssp_parent_simple<DPC_BASIC_DP><<<blocks, p.parent_threads, 0, s>>>(p, r); break;
    case DPC_WARP: sssp_parent<DPC_WARP><<<blocks, p.parent_threads, stage_bytes(p.parent_threads), s>>>(p, r); break;
    case DPC_BLOCK: sssp_parent<DPC_BLOCK><<<blocks, p.parent_threads, stage_bytes(p.parent_threads), s>>>(p, r); break;
    case DPC_GRID: sssp_parent<DPC_GRID><<<blocks, p.parent_threads, stage_bytes(p.parent_threads), s>>>(p, r); break;
    default: break;
  }
}

__global__ void sssp_split_min(SsspParams p, unsigned r);
__global__ void sssp_split_apply(SsspParams p, unsigned r);

// What follows round r (or a split before round r+1), decided by one thread
// once the frontier for the next round is published: its parent, the split,
// or the end of the call. Device-launched levels only.
__device__ void continue_after(const SsspParams &p, unsigned next_round) {
  WsHeader *h = p.hdr;
  const unsigned long long nn = ld_volatile(&h->aux[0]);
  h->round = next_round;
  __threadfence();
  const bool ok = ld_volatile(&h->status) == 0u;
  if (ok && nn > 0 && next_round < p.max_rounds) {
    launch_parent(p, next_round, (int)nn, cudaStreamTailLaunch);
  } else if (ok && nn == 0 && p.delta && !ld_volatile(&h->nf_done)) {
    sssp_split_min<<<p.commit_blocks, 256, 0, cudaStreamTailLaunch>>>(p, next_round);
  } else {
    if (ok && nn > 0) sssp_fail(p, DPC_ERR_OVERFLOW);  // the round cap was reached with work left
    if (p.stats) p.stats->rounds = next_round;
    return;
  }
  if (cudaGetLastError() != cudaSuccess) sssp_fail(p, DPC_ERR_DEVICE);
  else stat_add(p.stats, &dpc_stats::aux_launches, 1);
}

// After round r: the vertices that dropped (and heavy ones that wait) become
// the next frontier or go to the far pile.
__global__ void __launch_bounds__(256) sssp_commit(SsspParams p, unsigned r) {
  phase_sync(p);
  const int nn = (int)s_ph.next;
  const Split q = read_split();
  const int G = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  NearAcc acc;
  for (int i0 = gtid - (int)lane_id(); i0 < nn; i0 += G) {
    const int i = i0 + (int)lane_id();
    commit_vertex(p, i < nn, i < nn ? __ldcg(p.fnext + i) : 0, q, acc);
  }
  flush_near(p, acc);
  if (!last_block_done(&p.hdr->done_blocks2)) return;
  if (threadIdx.x == 0) {
    publish_frontier(p);
    if (p.level != DPC_FLAT) continue_after(p, r + 1);
  }
}

// The split, first pass (grid-stride over the current far list).
__global__ void __launch_bounds__(256) sssp_split_min(SsspParams p, unsigned r) {
  phase_sync(p);
  split_min_pass(p, read_split(), blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  if (!last_block_done(&p.hdr->done_blocks2)) return;
  if (threadIdx.x == 0) {
    const bool live = advance_split(p);
    if (p.level == DPC_FLAT) return;
    if (!live) {
      if (p.stats) p.stats->rounds = r;
      return;
    }
    sssp_split_apply<<<gridDim.x, 256, 0, cudaStreamTailLaunch>>>(p, r);
    if (cudaGetLastError() != cudaSuccess) sssp_fail(p, DPC_ERR_DEVICE);
    else stat_add(p.stats, &dpc_stats::aux_launches, 1);
  }
}

// The split, second pass.
__global__ void __launch_bounds__(256) sssp_split_apply(SsspParams p, unsigned r) {
  phase_sync(p);
  if (s_ph.done) return;  // (flat level) the split found no vertex at or above S
  NearAcc acc;
  split_apply_pass(p, read_split(), blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, acc);
  if (!last_block_done(&p.hdr->done_blocks2)) return;
  if (threadIdx.x == 0) {
    finish_split(p);
    if (p.level != DPC_FLAT) continue_after(p, r);
  }
}

// ------------------------------------------------------------------ queue level

// The grid level's rounds inside one cooperative grid: per round a parent
// phase (large frontier vertices' units into the buffer, short ones relaxed
// inline), the consolidated child's loop over the buffer, and the commit, each
// separated by a grid barrier instead of a device launch; a split is two more
// phases. The rounds keep the Jacobi semantics of the other levels (the commit
// snapshots distances after every relaxation of the round), so frontiers,
// rounds and relaxation counts are those of the grid level.
namespace {

enum : int { kBarPlain = 0, kBarChildren = 1, kBarRound = 2, kBarSplitMin = 3, kBarSplitApply = 4 };

// Multi-use barrier (arrivals only grow; the k-th barrier is complete at k *
// gridDim.x arrivals). The last block to arrive acts before it releases the
// others: after the children it publishes the list of vertices that dropped;
// after the commit it publishes the next frontier; after a split's passes it
// sets the new split or makes the far vertices below it the frontier.
// Bounded wait; false (with DPC_ERR_TIMEOUT) when it runs out.
__device__ bool queue_barrier(const SsspParams &p, unsigned k, int kind) {
  __shared__ int s_ok;
  __syncthreads();  // orders the block's writes before its master thread's fence and arrival
  if (threadIdx.x == 0) {
    __threadfence();
    int ok = 1;
    if (atomicAdd(&p.hdr->done_blocks2, 1u) == k * gridDim.x - 1) {
      if (kind == kBarChildren) {
        p.hdr->aux[1] = ld_volatile(&p.hdr->cursor2);
        p.hdr->cursor = 0ull;  // every unit of the round is done: the commit buffers the next round's
      } else if (kind == kBarRound) {
        publish_frontier(p);
      } else if (kind == kBarSplitMin) {
        advance_split(p);
      } else if (kind == kBarSplitApply) {
        finish_split(p);
      }
      __threadfence();
      atomicExch(&p.hdr->round, k);
    } else {
      WaitClock clk;
      while (*reinterpret_cast<volatile unsigned *>(&p.hdr->round) < k) {
        __nanosleep(32);
        if (clk.expired()) {
          sssp_fail(p, DPC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (ok) phase_load(p);  // the next phase's state, once per block
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace

// At most 1,024 threads; with 256-thread blocks six fit on an SM (40
// registers), which large graphs use to keep more loads in flight.
__global__ void __maxnreg__(40) sssp_queue(SsspParams p) {
  extern __shared__ int s_stage[];  // per warp: kStage entries, then the count (stage_bytes)
  const WarpStage ws{s_stage + (threadIdx.x >> 5) * (kStage + 1), s_stage + (threadIdx.x >> 5) * (kStage + 1) + kStage};
  if (lane_id() == 0) *ws.cnt = 0;
  phase_sync(p);
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long relaxed = 0, inl = 0, buf = 0;
  unsigned k = 0, r = 0;
  for (;;) {
    const int nf = (int)s_ph.nf;
    if (nf == 0 && s_ph.units == 0) {
      // the split: the far pile's smallest live distance, then the new frontier from it
      if (!p.delta) break;  // no split: an empty frontier ends the run
      split_min_pass(p, read_split(), gtid, G);
      if (!queue_barrier(p, ++k, kBarSplitMin)) return;
      if (s_ph.done) break;  // no vertex at or above the split: every distance is final
      NearAcc sacc;
      split_apply_pass(p, read_split(), gtid, G, sacc);
      relaxed += sacc.pre_edges;
      buf += sacc.pre_items;
      if (!queue_barrier(p, ++k, kBarSplitApply)) return;
      continue;
    }
    if (r >= p.max_rounds) {
      if (gtid == 0) sssp_fail(p, DPC_ERR_OVERFLOW);  // the round cap was reached with work left
      break;
    }
    const unsigned sub = s_ph.s;
    const unsigned S = s_ph.S;
    // parent phase: units of the large frontier vertices (one reservation per warp), short ones inline
    for (int i0 = gtid - lane; i0 < nf; i0 += G) {
      const int i = i0 + lane;
      int nu = 0, a = 0, b = 0;
      int4 f = make_int4(0, 0, 0, 0);
      bool work = false;
      if (i < nf) {
        f = __ldcg(p.fcur + i);
        if (relaxed_now(p, f, sub)) {
          work = true;
          a = f.z;
          b = f.w;
          relaxed += b - a;
          if (b - a > p.threshold) nu = ceil_div(b - a, p.chunk);
        } else {
          push_next(p, f.x, r);  // a heavy vertex above the sub-split waits for a later round
        }
      }
      const int inc = warp_inclusive_scan(nu);
      const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
      unsigned long long b0 = 0;
      if (lane == kWarp - 1 && total) b0 = atomicAdd(&p.hdr->cursor, (unsigned long long)total);
      const unsigned long long base = __shfl_sync(0xffffffffu, b0, kWarp - 1);
      if (total && base + (unsigned long long)total > (unsigned long long)p.max_units) {
        if (lane == 0) sssp_fail(p, DPC_ERR_OVERFLOW);  // only with malformed input: relax inline instead
        nu = 0;
      }
      if (nu) {
        const int pos = (int)base + inc - nu;
        for (int q = 0; q < nu; ++q) {
          const int ua = a + q * p.chunk;
          p.units[pos + q] = make_int4(ua, min(b, ua + p.chunk), f.y, f.x);
        }
        buf++;
      } else if (work) {
        inl++;
      }
      relax_inline_warp(p, a, b, (unsigned)f.y, r, S, work && nu == 0, ws);
    }
    // the units buffered ahead by the commit are in place since the round's
    // barrier; a barrier is needed only when this phase may have added some
    if (s_ph.append && !queue_barrier(p, ++k, kBarPlain)) return;
    // the consolidated child's loop: every warp's first unit is its own (no
    // atomic while units are fewer than warps), the rest come from a shared cursor
    const int total = (int)min(s_ph.units, (unsigned long long)p.max_units);
    const int nw = G >> 5;
    if ((gtid >> 5) < total) {
      const int4 un = __ldcg(p.units + (gtid >> 5));
      relax_edges_staged(p, un.x, un.y, (unsigned)un.z, r, S, ws);
    }
    if (total > nw) {
      const unsigned long long grab = units_per_grab(total - nw, nw);
      for (;;) {
        unsigned long long i0 = 0;
        if (lane == 0) i0 = atomicAdd(&p.hdr->aux[2], grab) + (unsigned long long)nw;
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        if (i0 >= (unsigned long long)total) break;
        const int i1 = (int)min(i0 + grab, (unsigned long long)total);
        for (int u = (int)i0; u < i1; ++u) {
          const int4 un = __ldcg(p.units + u);
          relax_edges_staged(p, un.x, un.y, (unsigned)un.z, r, S, ws);
        }
      }
    }
    stage_flush(p, ws);
    if (!queue_barrier(p, ++k, kBarChildren)) return;
    // commit: the next frontier's entries and the far pile
    const int nn = (int)s_ph.aux1;
    const Split q = read_split();
    NearAcc acc;
    for (int i0 = gtid - lane; i0 < nn; i0 += G)
      commit_vertex(p, i0 + lane < nn, i0 + lane < nn ? __ldcg(p.fnext + i0 + lane) : 0, q, acc);
    flush_near(p, acc);
    relaxed += acc.pre_edges;
    buf += acc.pre_items;
    ++r;
    if (!queue_barrier(p, ++k, kBarRound)) return;
  }
  round_stats(p, relaxed, inl, buf, 0, 0);
  if (p.stats && gtid == 0) atomicMax(&p.stats->rounds, r);
}

const void *sssp_queue_kernel() { return (const void *)sssp_queue; }

size_t sssp_queue_smem(int threads) { return stage_bytes(threads); }

cudaError_t sssp_queue_launch(const SsspParams &p, int blocks, cudaStream_t s) {
  const int init_blocks = ceil_div(p.n, 256) < 1024 ? ceil_div(p.n, 256) : 1024;
  sssp_init<<<init_blocks > 0 ? init_blocks : 1, 256, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SsspParams q = p;
  void *args[] = {&q};
  return cudaLaunchCooperativeKernel((const void *)sssp_queue, dim3(blocks), dim3(p.parent_threads), args,
                                     stage_bytes(p.parent_threads), s);
}

// ------------------------------------------------------------------ host side

size_t sssp_max_units(int n, int m, int threshold, int chunk) {
  size_t long_vertices = (size_t)m / ((size_t)threshold + 1);
  if (long_vertices > (size_t)n) long_vertices = (size_t)n;
  return (size_t)m / (size_t)chunk + long_vertices + 1;
}

size_t sssp_workspace_bytes(int n, int m, dpc_level level, const LaunchCfg &c) {
  size_t b = kHeaderBytes;
  b += align_up((size_t)n * sizeof(int4), 256);      // fcur
  b += align_up((size_t)n * sizeof(int), 256);       // fnext
  b += align_up((size_t)n * sizeof(unsigned), 256);  // stamp
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE)
    b += align_up(sssp_max_units(n, m, c.threshold, c.chunk) * sizeof(int4), 256);
  return b;
}

void sssp_carve(SsspParams &p, void *workspace, int n, int m, dpc_level level, const LaunchCfg &c) {
  char *b = static_cast<char *>(workspace);
  p.hdr = reinterpret_cast<WsHeader *>(b);
  b += kHeaderBytes;
  p.fcur = reinterpret_cast<int4 *>(b);
  b += align_up((size_t)n * sizeof(int4), 256);
  p.fnext = reinterpret_cast<int *>(b);
  b += align_up((size_t)n * sizeof(int), 256);
  p.stamp = reinterpret_cast<unsigned *>(b);
  b += align_up((size_t)n * sizeof(unsigned), 256);
  p.units = nullptr;
  p.max_units = 0;
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE) {
    const size_t mu = sssp_max_units(n, m, c.threshold, c.chunk);
    p.units = reinterpret_cast<int4 *>(b);
    p.max_units = (int)(mu > (size_t)0x7FFFFFFF ? 0x7FFFFFFF : mu);
  }
}

const void *sssp_parent_kernel(dpc_level level) {
  switch (level) {
    case DPC_FLAT: return (const void *)sssp_parent_simple<DPC_FLAT>;
    case DPC_BASIC_DP: return (const void *)sssp_parent_simple<DPC_BASIC_DP>;
    case DPC_WARP: return (const void *)sssp_parent<DPC_WARP>;
    case DPC_BLOCK: return (const void *)sssp_parent<DPC_BLOCK>;
    case DPC_GRID: return (const void *)sssp_parent<DPC_GRID>;
    case DPC_QUEUE: return (const void *)sssp_queue;
  }
  return nullptr;
}

const void *sssp_child_kernel(dpc_level level) {
  return level == DPC_BASIC_DP ? (const void *)sssp_vertex_child : (const void *)sssp_child;
}

cudaError_t sssp_launch(SsspParams &p, dpc_level level, cudaStream_t s, unsigned *rounds_out) {
  const int init_blocks = ceil_div(p.n, 256) < p.parent_blocks * 4 ? ceil_div(p.n, 256) : p.parent_blocks * 4;
  sssp_init<<<init_blocks > 0 ? init_blocks : 1, 256, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (level != DPC_FLAT) {
    // round 0 has a single frontier vertex; later rounds are launched on the device
    switch (level) {
      case DPC_BASIC_DP: sssp_parent_simple<DPC_BASIC_DP><<<1, p.parent_threads, 0, s>>>(p, 0u); break;
      case DPC_WARP: sssp_parent<DPC_WARP><<<1, p.parent_threads, stage_bytes(p.parent_threads), s>>>(p, 0u); break;
      case DPC_BLOCK: sssp_parent<DPC_BLOCK><<<1, p.parent_threads, stage_bytes(p.parent_threads), s>>>(p, 0u); break;
      case DPC_GRID: sssp_parent<DPC_GRID><<<1, p.parent_threads, stage_bytes(p.parent_threads), s>>>(p, 0u); break;
      default: break;
    }
    return cudaGetLastError();
  }
  // flat: host-driven rounds and splits (no device launches at all); after
  // every step the frontier size (and whether a split found nothing) comes back
  HostScratch &hs = host_scratch();
  unsigned r = 0;
  unsigned long long nf = 1;
  bool split = false;
  for (;;) {
    if (nf > 0) {
      if (r >= p.max_rounds) break;
      const int need = ceil_div((int)nf, p.parent_threads);
      const int blocks = need < p.parent_blocks ? need : p.parent_blocks;
      sssp_parent_simple<DPC_FLAT><<<blocks, p.parent_threads, 0, s>>>(p, r);
      sssp_commit<<<p.commit_blocks, 256, 0, s>>>(p, r);
      ++r;
      split = false;
    } else {
      if (!p.delta || split) break;  // no split, or a split that found no vertex at or above S
      sssp_split_min<<<p.commit_blocks, 256, 0, s>>>(p, r);
      sssp_split_apply<<<p.commit_blocks, 256, 0, s>>>(p, r);
      split = true;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hs.sizes, &p.hdr->aux[0], sizeof(unsigned long long), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    nf = hs.sizes[0];
  }
  if (rounds_out) *rounds_out = r;
  return cudaSuccess;
}

}  // namespace dpc
