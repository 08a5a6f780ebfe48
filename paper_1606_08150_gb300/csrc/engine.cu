// Persistent batched engine: many SSSP / tree problems in one resident kernel.
//
// The consolidated kernels of spmv.cu / sssp.cu / tree.cu hand large work to
// device-launched child grids. For batches of small, uneven problems the
// launches themselves dominate (a device launch or tail link costs 10-20 µs on
// GB300). Here the child launches are replaced by a device work queue, the
// persistent-threads alternative the paper's related work names (Sec. VI):
// one cooperative grid stays resident and every warp repeatedly takes a task
// from the queue. A task is one of
//   INIT    reset distances / stamps of an SSSP problem (1024 vertices)
//   RELAX   up to 32 frontier vertices, one per lane; a vertex above the
//           threshold is not relaxed inline but split into EDGES tasks: the
//           consolidation buffer of the paper, at queue granularity
//   EDGES   one chunk of edges of one vertex (512 by default, 16 per lane)
//   COMMIT  freeze (vertex, distance) of up to 256 next-frontier vertices
//   VISIT   up to 32 tree units (node, chunk of children), one per lane
//   POST    postwork of up to 32 tree units (every unit of the tree at once,
//           in one wave: see the tree pieces below)
// Tasks made while a wave runs go to the next wave's list; waves are separated
// by a grid barrier (bounded spin, so a fault cannot hang the GPU). Each
// problem counts its outstanding tasks; the warp that finishes the last task
// of a phase starts the next phase (commit after a round, next round after a
// commit, next tree level, postwork bottom-up), so problems at different
// phases share every wave.
//
// The engine is resumable: a step admits new problems into free slots, runs
// at most max_waves waves and returns with its queue intact, so a host loop
// can fold arrivals into the running work between steps (continuous batching).
// All per-step arguments live in device memory, so a step can be captured in
// a CUDA graph and replayed.
//
// Resident form (dpc_engine_serve): the kernel stays on the GPU and takes new
// problems from a mailbox in host memory while it runs. The host posts a job
// (descriptor and slot) and publishes it by a release store of the posted
// count; at every wave barrier the last arriving block reads that count, and
// during the next wave one warp per new job admits it into the list of the
// wave after. Finished slots are reported in host memory, so the host sees
// each result the moment it is complete, with no kernel boundary between an
// arrival and its first wave. Every wait is bounded: an idle engine polls the
// mailbox for at most kIdlePollNs per barrier, and the kernel returns once
// it has been idle past its lifetime (or, busy or not, past four lifetimes),
// with its queue intact.
#include <climits>
#include <cstring>
#include <mutex>

#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "dpc_internal.h"
#include "dpc_runtime.cuh"

namespace cg = cooperative_groups;

namespace dpc {
namespace {

constexpr unsigned kInfU = 0xFFFFFFFFu;
constexpr int kInitItems = 1024;   // vertices per INIT task
constexpr int kRelaxItems = 32;    // frontier vertices per RELAX task (one per lane)
constexpr int kCommitItems = 256;  // entries per COMMIT task
constexpr int kTreeItems = 32;     // units per VISIT / POST task (one per lane)
constexpr int kEngTreeChunk = 8;   // children per tree unit: one batch of loads per lane
constexpr int kEdgeBatch = 8;      // edges per lane per EDGES batch
constexpr int kGrab = 8;           // tasks taken per cursor atomic while the list is long

enum TaskKind : int { T_INIT = 1, T_RELAX = 2, T_EDGES = 3, T_COMMIT = 4, T_VISIT = 5, T_POST = 6 };
enum Phase : int { P_FREE = 0, P_INIT = 1, P_RELAX = 2, P_COMMIT = 3, P_VISIT = 4, P_POST = 5, P_DONE = 6 };

struct EngineHeader {
  unsigned long long count[3];   // tasks in each of the three rotating lists
  unsigned long long cursor[3];  // next task to hand out in each list
  unsigned bar_count, bar_gen;   // grid barrier
  unsigned status;               // dpc_status of the device side
  int active;                    // problems admitted and not finished
  unsigned long long snap_count; // taken by the barrier's last arriver: tasks of the next wave,
  int snap_active;               // problems still active,
  unsigned snap_status;          // and the status, so every block takes the same decision
  long long wave;                // waves run since init
  int slots, max_n, max_m, threshold, chunk, tree_chunk;
  // resident form: the range [snap_lo, snap_hi) of mailbox jobs admitted
  // during the coming wave, the exit decision and the start time
  unsigned long long snap_lo, snap_hi;
  int snap_exit;
  unsigned long long t_start;
  unsigned long long mb_seen;  // the mailbox's taken count (read at the launch's first barrier)
  unsigned long long task_cap;   // capacity of one task list
  unsigned long long slot_bytes; // scratch bytes per slot
};
static_assert(sizeof(EngineHeader) <= 256, "engine header too large");

struct Slot {
  dpc_job job;
  int phase;
  int pending;        // outstanding tasks of the current phase
  int round;          // SSSP round / tree level being visited
  int nf;             // SSSP: current frontier size
  unsigned long long next_count;  // SSSP: next frontier size; trees: units handed out
  int post_level;     // trees: level whose postwork runs
  int pre_edges;      // SSSP: EDGES tasks the commit emitted for the next round's heavy vertices
  int pad[2];
};

struct Engine {
  EngineHeader *hdr;
  Slot *slots;
  int4 *tasks[3];
  unsigned char *scratch;
  int *slot_state;   // caller's array: 1 running, 2 finished
  dpc_stats *stats;
  dpc_mailbox *mb;   // resident form: the host's mailbox (else null)
  unsigned long long limit_ns;  // resident form: the kernel's lifetime when idle
};

// Resident form: the longest an idle engine polls the mailbox at one barrier
// (the other blocks wait at that barrier meanwhile, far below its own limit).
constexpr unsigned long long kIdlePollNs = 20000;

// A report to a tree node's link word: one count fewer (high 32 bits).
constexpr unsigned long long kOneReport = 0xFFFFFFFF00000000ull;

// Finished: results complete, then the state the caller polls. The state may
// live in host memory (resident form), hence the system-scope fence.
__device__ __forceinline__ void report_done(const Engine &e, int s) {
  __threadfence_system();
  *reinterpret_cast<volatile int *>(e.slot_state + s) = 2;
}

__device__ __forceinline__ void eng_fail(const Engine &e, unsigned code) {
  atomicCAS(&e.hdr->status, 0u, code);
  if (e.stats) atomicCAS(&e.stats->status, 0u, code);
}

// Per-slot scratch views.
struct SsspView {
  int2 *fcur;
  int *fnext;
  unsigned *stamp;
};
struct TreeView {
  int2 *units;
  int *levels;
  int *par;                  // parent of each internal node (root: -1)
  unsigned long long *link;  // pending reports (high 32 bits), descendants' partial value (low)
  int max_units;
};

__device__ __forceinline__ unsigned char *slot_scratch(const Engine &e, int s) {
  return e.scratch + (size_t)s * e.hdr->slot_bytes;
}

__device__ __forceinline__ SsspView sssp_view(const Engine &e, int s) {
  unsigned char *b = slot_scratch(e, s);
  const size_t n = (size_t)e.hdr->max_n;
  SsspView v;
  v.fcur = reinterpret_cast<int2 *>(b);
  v.fnext = reinterpret_cast<int *>(b + align_up(n * sizeof(int2), 256));
  v.stamp = reinterpret_cast<unsigned *>(b + align_up(n * sizeof(int2), 256) + align_up(n * sizeof(int), 256));
  return v;
}

__device__ __forceinline__ TreeView tree_view(const Engine &e, int s) {
  unsigned char *b = slot_scratch(e, s);
  const size_t n = (size_t)e.hdr->max_n;
  const size_t mu = (n > 0 ? n - 1 : 0) / (size_t)e.hdr->tree_chunk + n + 1;
  TreeView v;
  v.units = reinterpret_cast<int2 *>(b);
  b += align_up(mu * sizeof(int2), 256);
  v.levels = reinterpret_cast<int *>(b);
  b += align_up((n + 2) * sizeof(int), 256);
  v.par = reinterpret_cast<int *>(b);
  b += align_up(n * sizeof(int), 256);
  v.link = reinterpret_cast<unsigned long long *>(b);
  v.max_units = (int)mu;
  return v;
}

__device__ __forceinline__ int4 make_task(int kind, int slot, int a, int b, int c) {
  return make_int4((kind << 24) | slot, a, b, c);
}

// Append `n` tasks of the calling lane to list l (all lanes of the coalesced
// group take part; one atomic per group). Returns the first index, or -1 when
// the list is full (the device status then says DPC_ERR_OVERFLOW).
__device__ __forceinline__ long long reserve_tasks(const Engine &e, int l, int n) {
  cg::coalesced_group g = cg::coalesced_threads();
  const int excl = cg::exclusive_scan(g, n);
  const int total = g.shfl(excl + n, g.size() - 1);
  unsigned long long base = 0;
  if (g.thread_rank() == 0 && total) base = atomicAdd(&e.hdr->count[l], (unsigned long long)total);
  base = g.shfl(base, 0);
  if (base + excl + n > e.hdr->task_cap) {
    eng_fail(e, DPC_ERR_OVERFLOW);
    return -1;
  }
  return (long long)(base + excl);
}

// Warp-cooperative emission of `ntasks` tasks into list l with a single
// reservation: lane 0 reserves the whole slice, then the lanes write task t =
// make(t) strided. A phase transition can emit tens of thousands of tasks; one
// atomic round trip per 32 of them kept the rest of the grid waiting at the
// wave barrier for milliseconds on a 4M-vertex frontier.
template <class F>
__device__ __forceinline__ void emit_tasks(const Engine &e, int l, int ntasks, F make) {
  if (ntasks <= 0) return;
  unsigned long long base = 0;
  if (lane_id() == 0) base = atomicAdd(&e.hdr->count[l], (unsigned long long)ntasks);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (base + (unsigned long long)ntasks > e.hdr->task_cap) {
    if (lane_id() == 0) eng_fail(e, DPC_ERR_OVERFLOW);
    return;
  }
  int4 *dst = e.tasks[l] + base;
  for (int t = lane_id(); t < ntasks; t += kWarp) dst[t] = make(t);
}

// ceil(len/per) range tasks [i, i+per) over [lo, lo+len), argument c in .w.
__device__ __forceinline__ int emit_ranges(const Engine &e, int l, int kind, int slot, int lo, int len, int per,
                                           int c) {
  const int ntasks = ceil_div(len, per);
  emit_tasks(e, l, ntasks, [&](int t) {
    return make_task(kind, slot, lo + t * per, lo + min(len, (t + 1) * per), c);
  });
  return ntasks;
}

// ------------------------------------------------------------------ SSSP pieces

// Edges are read once per relaxation and the resident problems' graphs
// together outgrow L2, so they stream with the evict-first hint: the slots'
// distances and stamps, gathered at random every round, stay in L2.

// Per-warp staging of an EDGES task's new frontier vertices in shared memory
// (kEngStage entries of one slot): the slot's list counter is reserved once
// per flush instead of once per batch, and the buffer is flushed before the
// warp reports the slot's tasks finished (the transition reads the count).
constexpr int kEngStage = 256;
static_assert(kEngStage >= kWarp * kEdgeBatch, "a warp's EDGES batch must fit in its stage");

struct EngStage {
  int *buf;
  int *cnt;
};

__device__ __forceinline__ void eng_flush(const Engine &e, int s, const EngStage &st) {
  const int c = *st.cnt;
  __syncwarp();
  if (c == 0) return;
  unsigned long long base = 0;
  if (lane_id() == 0) base = atomicAdd(&e.slots[s].next_count, (unsigned long long)c);
  base = __shfl_sync(0xffffffffu, base, 0);
  int *fnext = sssp_view(e, s).fnext;
  for (int i = lane_id(); i < c; i += kWarp) fnext[base + i] = st.buf[i];
  __syncwarp();
  if (lane_id() == 0) *st.cnt = 0;
  __syncwarp();
}

// The EDGES form of sssp_relax_edges: a full warp over [a, b), staged appends.
// One batch of up to kEdgeBatch candidate edges per lane (vertex vv, new
// distance d; vv < 0: none): the distance gathers, atomicMin where the
// candidate is smaller, the round's stamp for a vertex that dropped, and the
// warp's new frontier vertices staged in shared memory (flushed to the slot's
// list when the stage would overflow; the caller flushes the rest).
__device__ __forceinline__ void relax_stage_batch(const Engine &e, int s, const SsspView &v, const int (&vv)[kEdgeBatch],
                                                  const unsigned (&d)[kEdgeBatch], unsigned r, const EngStage &st) {
  unsigned *dist = static_cast<unsigned *>(e.slots[s].job.out);
  unsigned cur[kEdgeBatch];
#pragma unroll
  for (int q = 0; q < kEdgeBatch; ++q) cur[q] = (vv[q] >= 0 && d[q] != kInfU) ? __ldcg(dist + vv[q]) : 0u;
  unsigned improved = 0;
#pragma unroll
  for (int q = 0; q < kEdgeBatch; ++q)
    if (d[q] < cur[q] && d[q] < atomicMin(dist + vv[q], d[q])) improved |= 1u << q;
  unsigned fresh = 0;
#pragma unroll
  for (int q = 0; q < kEdgeBatch; ++q)
    if ((improved >> q & 1u) && atomicExch(v.stamp + vv[q], r) != r) fresh |= 1u << q;
  const int cnt = __popc(fresh);
  const int inc = warp_inclusive_scan(cnt);
  const int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
  if (total == 0) return;
  if (*st.cnt + total > kEngStage) eng_flush(e, s, st);
  int pos = *st.cnt + inc - cnt;
#pragma unroll
  for (int q = 0; q < kEdgeBatch; ++q)
    if (fresh >> q & 1u) st.buf[pos++] = vv[q];
  __syncwarp();
  if (lane_id() == kWarp - 1) *st.cnt += total;
  __syncwarp();
}

// The EDGES form: a full warp over [a, b) of one vertex, lane-strided.
__device__ __forceinline__ void sssp_relax_edges_staged(const Engine &e, int s, const SsspView &v, int a, int b,
                                                        unsigned du, unsigned r, const EngStage &st) {
  const int *__restrict__ col = e.slots[s].job.col;
  const unsigned *__restrict__ w = e.slots[s].job.w;
  const int t = lane_id(), T = kWarp;
  for (int base0 = a; base0 < b; base0 += kEdgeBatch * T) {
    int vv[kEdgeBatch];
    unsigned d[kEdgeBatch];
#pragma unroll
    for (int q = 0; q < kEdgeBatch; ++q) {
      const int ed = base0 + t + q * T;
      vv[q] = -1;
      d[q] = kInfU;
      if (ed < b) {
        const unsigned long long nd = (unsigned long long)du + __ldcs(w + ed);
        vv[q] = checked_index(__ldcs(col + ed), e.slots[s].job.n, &e.hdr->status);
        if (nd >= kInfU) eng_fail(e, DPC_ERR_OVERFLOW);
        else d[q] = (unsigned)nd;
      }
    }
    relax_stage_batch(e, s, v, vv, d, r, st);
  }
}

// The RELAX form: the lanes' own light vertices ([a, b), distance du; lanes
// with `active` false have none) relaxed by the whole warp together - the
// edges of the 32 vertices in one sequence, edge k of it taken by lane k mod
// 32 (a search over the lanes' scanned degrees finds its vertex) - instead of
// each lane walking its own vertex while the warp waits for the longest.
__device__ __forceinline__ void sssp_relax_inline_warp(const Engine &e, int s, const SsspView &v, int a, int b,
                                                       unsigned du, unsigned r, bool active, const EngStage &st) {
  const int *__restrict__ col = e.slots[s].job.col;
  const unsigned *__restrict__ w = e.slots[s].job.w;
  const int lane = lane_id();
  const int deg = active ? b - a : 0;
  const int incl = warp_inclusive_scan(deg);
  const int total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
  const int excl = incl - deg;
  for (int base = 0; base < total; base += kWarp * kEdgeBatch) {  // warp-uniform
    int vv[kEdgeBatch];
    unsigned d[kEdgeBatch];
#pragma unroll
    for (int q = 0; q < kEdgeBatch; ++q) {
      const int k = base + q * kWarp + lane;
      int owner = 0;
#pragma unroll
      for (int step = kWarp / 2; step >= 1; step >>= 1) {
        const int m = owner + step;
        if (__shfl_sync(0xffffffffu, excl, m & (kWarp - 1)) <= k && m < kWarp) owner = m;
      }
      const int ed = __shfl_sync(0xffffffffu, a, owner) + k - __shfl_sync(0xffffffffu, excl, owner);
      const unsigned dl = __shfl_sync(0xffffffffu, du, owner);
      vv[q] = -1;
      d[q] = kInfU;
      if (k < total) {
        const unsigned long long nd = (unsigned long long)dl + __ldcs(w + ed);
        vv[q] = checked_index(__ldcs(col + ed), e.slots[s].job.n, &e.hdr->status);
        if (nd >= kInfU) eng_fail(e, DPC_ERR_OVERFLOW);
        else d[q] = (unsigned)nd;
      }
    }
    relax_stage_batch(e, s, v, vv, d, r, st);
  }
}

// ------------------------------------------------------------------ phase transitions

// Called by one full warp after the last task of slot s's current phase
// finished; emits the next phase's tasks into list `nl`.
__device__ void transition(const Engine &e, int s, int nl) {
  Slot &sl = e.slots[s];
  const int lane = lane_id();
  __threadfence();
  const int kind = sl.job.kind;
  int ntasks = 0;
  bool done = false;
  if (kind == DPC_JOB_SSSP) {
    const SsspView v = sssp_view(e, s);
    if (sl.phase == P_INIT) {
      if (lane == 0) {
        v.fcur[0] = make_int2(sl.job.source, 0);
        sl.nf = 1;
        sl.round = 0;
        sl.next_count = 0;
        sl.phase = P_RELAX;
        sl.pending = 1;
        const long long pos = reserve_tasks(e, nl, 1);
        if (pos >= 0) e.tasks[nl][pos] = make_task(T_RELAX, s, 0, 1, 0);
      }
      __syncwarp();
      return;
    }
    if (sl.phase == P_RELAX) {
      const int nn = (int)*reinterpret_cast<volatile unsigned long long *>(&sl.next_count);
      if (nn == 0 || sl.round + 1 > sl.job.n) {
        done = true;
      } else {
        if (lane == 0) {
          sl.phase = P_COMMIT;
          sl.pending = ceil_div(nn, kCommitItems);
        }
        __syncwarp();
        ntasks = emit_ranges(e, nl, T_COMMIT, s, 0, nn, kCommitItems, 0);
      }
    } else if (sl.phase == P_COMMIT) {
      const int nn = (int)*reinterpret_cast<volatile unsigned long long *>(&sl.next_count);
      if (lane == 0) {
        sl.nf = nn;
        sl.next_count = 0;
        sl.round += 1;
        sl.phase = P_RELAX;
        // the commit already queued the heavy vertices' EDGES tasks: they are part of this phase
        sl.pending = ceil_div(nn, kRelaxItems) + *reinterpret_cast<volatile int *>(&sl.pre_edges);
        sl.pre_edges = 0;
      }
      __syncwarp();
      ntasks = emit_ranges(e, nl, T_RELAX, s, 0, nn, kRelaxItems, 0);
    }
    if (lane == 0 && e.stats && done) atomicMax(&e.stats->rounds, (unsigned)sl.round + 1u);
  } else {
    const TreeView v = tree_view(e, s);
    if (sl.phase == P_VISIT) {
      const int L = sl.round;
      const int start = v.levels[L + 1];
      const int end = (int)min(*reinterpret_cast<volatile unsigned long long *>(&sl.next_count),
                               (unsigned long long)v.max_units);
      if (L + 2 > sl.job.n + 1) {
        if (lane == 0) eng_fail(e, DPC_ERR_DEPTH);
        done = true;
      } else if (end > start) {
        if (lane == 0) {
          v.levels[L + 2] = end;
          sl.round = L + 1;
          sl.pending = ceil_div(end - start, kTreeItems);
        }
        __syncwarp();
        // VISIT ranges are absolute unit indices
        ntasks = emit_ranges(e, nl, T_VISIT, s, start, end - start, kTreeItems, L + 1);
      } else {
        // deepest level reached: the postwork of every unit at once (chained, one wave)
        const int hi = v.levels[L + 1];
        if (lane == 0) {
          sl.phase = P_POST;
          sl.post_level = 0;
          sl.pending = ceil_div(hi, kTreeItems);
        }
        __syncwarp();
        ntasks = emit_ranges(e, nl, T_POST, s, 0, hi, kTreeItems, 0);
        if (ntasks == 0) done = true;
      }
      if (lane == 0 && e.stats) atomicMax(&e.stats->rounds, (unsigned)L + 2u);
    } else if (sl.phase == P_POST) {
      done = true;  // every node has reported
    }
  }
  if (ntasks == 0 && !done && sl.phase != P_DONE && lane == 0) {
    // a phase with nothing to do cannot happen for valid input; end the problem rather than stall
    eng_fail(e, DPC_ERR_DEVICE);
    done = true;
  }
  if (done && lane == 0) {
    sl.phase = P_DONE;
    report_done(e, s);
    atomicSub(&e.hdr->active, 1);
  }
  __syncwarp();
}

// The calling warp finished tasks of slot s whose net effect on the slot's
// outstanding count is `delta` (tasks it added minus tasks it finished): one
// atomic for the whole run of same-slot tasks of a grab. The warp that brings
// the count to zero moves the problem to its next phase. Added tasks are
// counted in the same update as the finished ones, so the count cannot touch
// zero while any of the phase's work is still queued.
__device__ __forceinline__ void tasks_done(const Engine &e, int s, int delta, int nl) {
  int last = 0;
  if (lane_id() == 0) {
    __threadfence();
    last = atomicAdd(&e.slots[s].pending, delta) + delta == 0;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) transition(e, s, nl);
}

// ------------------------------------------------------------------ task bodies

// Runs one task; returns the number of tasks it added to its slot's phase (.x,
// the same in every lane) and the edges the calling lane relaxed or visited (.y).
// EDGES tasks stage their new frontier vertices in `st` (flushed by the caller).
__device__ int2 run_task(const Engine &e, int4 t, int nl, const EngStage &st) {
  const int kind = t.x >> 24, s = t.x & 0xFFFFFF;
  const int lane = lane_id();
  // a register copy: the loops below store to global memory, which would
  // otherwise force the descriptor to be re-read after every store
  const dpc_job job = e.slots[s].job;
  int extra = 0, work = 0;
  switch (kind) {
    case T_INIT: {
      const SsspView v = sssp_view(e, s);
      unsigned *dist = static_cast<unsigned *>(job.out);
      for (int i = t.y + lane; i < t.z; i += kWarp) {
        dist[i] = i == job.source ? 0u : kInfU;
        v.stamp[i] = kInfU;
      }
      break;
    }
    case T_RELAX: {
      const SsspView v = sssp_view(e, s);
      const unsigned r = (unsigned)e.slots[s].round;
      const int i = t.y + lane;
      int nu = 0, a = 0, b = 0;
      int2 f = make_int2(0, 0);
      if (i < t.z) {
        f = v.fcur[i];
        a = __ldg(job.off + f.x);
        b = __ldg(job.off + f.x + 1);
        if (b - a > e.hdr->threshold) nu = ceil_div(b - a, e.hdr->chunk);
      }
      // large vertices: one EDGES task per chunk into the next wave - in round 0
      // only (the source); from round 1 on the commit queued them already
      const int emit = r == 0 ? nu : 0;
      const long long pos = reserve_tasks(e, nl, emit);
      if (emit && pos >= 0)
        for (int k = 0; k < emit; ++k) e.tasks[nl][pos + k] = make_task(T_EDGES, s, f.x, k, f.y);
      extra = __reduce_add_sync(0xffffffffu, (unsigned)emit);
      const bool inl = i < t.z && nu == 0;
      sssp_relax_inline_warp(e, s, v, a, b, (unsigned)f.y, r, inl, st);
      if (inl) work = b - a;
      break;
    }
    case T_EDGES: {
      const SsspView v = sssp_view(e, s);
      const unsigned r = (unsigned)e.slots[s].round;
      const int u = t.y, k = t.z;
      const int a0 = __ldg(job.off + u), b0 = __ldg(job.off + u + 1);
      const int a = a0 + k * e.hdr->chunk, b = min(b0, a + e.hdr->chunk);
      sssp_relax_edges_staged(e, s, v, a, b, (unsigned)t.w, r, st);
      work = lane == 0 ? b - a : 0;
      break;
    }
    case T_COMMIT: {
      // the next frontier's (vertex, distance) entries; a heavy vertex's EDGES
      // tasks go straight into the next wave, beside the next round's RELAX
      // tasks, so a round takes two waves instead of three
      const SsspView v = sssp_view(e, s);
      const unsigned *dist = static_cast<const unsigned *>(job.out);
      int emitted = 0;
      for (int i0 = t.y; i0 < t.z; i0 += kWarp) {  // warp-uniform
        const int i = i0 + lane;
        int nu = 0, vtx = 0;
        unsigned d = 0;
        if (i < t.z) {
          vtx = __ldcg(v.fnext + i);
          d = __ldcg(dist + vtx);
          v.fcur[i] = make_int2(vtx, (int)d);
          const int a = __ldg(job.off + vtx), b = __ldg(job.off + vtx + 1);
          if (b - a > e.hdr->threshold) nu = ceil_div(b - a, e.hdr->chunk);
        }
        const long long pos = reserve_tasks(e, nl, nu);
        if (nu && pos >= 0)
          for (int k = 0; k < nu; ++k) e.tasks[nl][pos + k] = make_task(T_EDGES, s, vtx, k, (int)d);
        emitted += (int)__reduce_add_sync(0xffffffffu, (unsigned)nu);
      }
      if (lane == 0 && emitted) atomicAdd(&e.slots[s].pre_edges, emitted);
      break;
    }
    case T_VISIT: {
      // lane per unit; a unit has at most kEngTreeChunk children, loaded as one batch
      const TreeView v = tree_view(e, s);
      const int tc = e.hdr->tree_chunk;
      int *out = static_cast<int *>(job.out);
      const int i = t.y + lane;
      int a = 0, b = 0;
      if (i < t.z) {
        const int2 u = __ldcg(v.units + i);
        if (u.x >= 0) {
          a = __ldg(job.off + u.x) + u.y * tc;
          b = min(__ldg(job.off + u.x + 1), a + tc);
        }
      }
      int c[kEngTreeChunk], first[kEngTreeChunk], kc[kEngTreeChunk];
#pragma unroll
      for (int j = 0; j < kEngTreeChunk; ++j)
        c[j] = a + j < b ? checked_index(__ldg(job.col + a + j), job.n, &e.hdr->status) : -1;
#pragma unroll
      for (int j = 0; j < kEngTreeChunk; ++j) {
        first[j] = c[j] >= 0 ? __ldg(job.off + c[j]) : 0;
        kc[j] = c[j] >= 0 ? __ldg(job.off + c[j] + 1) : 0;
      }
      // count the units of internal children, reserve them for the warp, then write
      int mine = 0;
#pragma unroll
      for (int j = 0; j < kEngTreeChunk; ++j) {
        kc[j] -= first[j];
        mine += kc[j] > 0 ? ceil_div(kc[j], tc) : 0;
      }
      const int inc = warp_inclusive_scan(mine);
      int total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
      unsigned long long b0 = 0;
      if (lane == kWarp - 1 && total) b0 = atomicAdd(&e.slots[s].next_count, (unsigned long long)total);
      const unsigned long long base = __shfl_sync(0xffffffffu, b0, kWarp - 1);
      if (total && base + (unsigned long long)total > (unsigned long long)v.max_units) {
        if (lane == 0) eng_fail(e, DPC_ERR_OVERFLOW);  // only when the input is not a tree
        for (unsigned long long q = base + lane; q < (unsigned long long)v.max_units && q < base + total; q += kWarp)
          v.units[q] = make_int2(-1, 0);
        total = 0;
      }
      int pos = total ? (int)base + inc - mine : 0;
      const bool desc = job.kind == DPC_JOB_TREE_DESCENDANTS;
      int node = -1;
      if (i < t.z) node = __ldcg(v.units + i).x;
      unsigned inner = 0;
#pragma unroll
      for (int j = 0; j < kEngTreeChunk; ++j) {
        if (c[j] >= 0) out[c[j]] = 0;
        const int nu = total && kc[j] > 0 ? ceil_div(kc[j], tc) : 0;
        if (nu) {
          // one pending report (its own token); a node with children is at least 1 high
          inner++;
          v.link[c[j]] = 1ull << 32;
          if (!desc) out[c[j]] = 1;
          v.par[c[j]] = node;
        }
        if (nu <= 2)
          for (int q = 0; q < nu; ++q) v.units[pos + q] = make_int2(c[j], q);
        // a larger child's units are written by the whole warp
        unsigned big = __ballot_sync(0xffffffffu, nu > 2);
        while (big) {
          const int src = __ffs(big) - 1;
          big &= big - 1;
          const int bc = __shfl_sync(0xffffffffu, c[j], src), bp = __shfl_sync(0xffffffffu, pos, src);
          const int bn = __shfl_sync(0xffffffffu, nu, src);
          for (int q = lane; q < bn; q += kWarp) v.units[bp + q] = make_int2(bc, q);
        }
        pos += nu;
      }
      // the node's share known now (1 per child for descendants; its internal
      // children report the rest) and its internal-children count, one atomic
      // per run of one node's units in the warp
      unsigned kids = (unsigned)(b - a);
      const int prev = __shfl_up_sync(0xffffffffu, node, 1);
      int start = lane == 0 || prev != node ? lane : 0;
      for (int d = 1; d < kWarp; d <<= 1) start = max(start, __shfl_up_sync(0xffffffffu, start, d));
      for (int d = 1; d < kWarp; d <<= 1) {
        const unsigned ok = __shfl_up_sync(0xffffffffu, kids, d), oi = __shfl_up_sync(0xffffffffu, inner, d);
        if (lane - d >= start) {
          kids += ok;
          inner += oi;
        }
      }
      const int next = __shfl_down_sync(0xffffffffu, node, 1);
      if (node >= 0 && (lane == kWarp - 1 || next != node)) {
        const unsigned long long add = ((unsigned long long)inner << 32) + (desc ? kids : 0u);
        if (add) atomicAdd(v.link + node, add);
      }
      work = b - a;
      break;
    }
    case T_POST: {
      // lane per unit: at a node's first unit (chunk index 0) remove the
      // node's own token; whichever report completes a node carries its value
      // to the parent, up the chain (the tree queue level's chained postwork)
      const TreeView v = tree_view(e, s);
      int *out = static_cast<int *>(job.out);
      const bool desc = job.kind == DPC_JOB_TREE_DESCENDANTS;
      const int i = t.y + lane;
      int c = -1;
      if (i < t.z) {
        const int2 u = __ldcg(v.units + i);
        if (u.x >= 0 && u.y == 0) c = u.x;
      }
      if (c >= 0) {
        unsigned long long old = atomicAdd(v.link + c, kOneReport);
        if (old >> 32 == 1ull) {
          unsigned val;
          if (desc) {
            val = (unsigned)old;
          } else {
            __threadfence();
            val = (unsigned)__ldcg(out + c);
          }
          for (;;) {  // c is complete with value val
            const int p = __ldcg(v.par + c);
            if (desc) out[c] = (int)val;
            if (p < 0) break;  // the root
            if (desc) {
              old = atomicAdd(v.link + p, (unsigned long long)val + kOneReport);
              if (old >> 32 != 1ull) break;
              val += (unsigned)old;
            } else {
              atomicMax(out + p, (int)(val + 1u));
              __threadfence();
              old = atomicAdd(v.link + p, kOneReport);
              if (old >> 32 != 1ull) break;
              __threadfence();
              val = (unsigned)__ldcg(out + p);
            }
            c = p;
          }
        }
      }
      break;
    }
    default:
      eng_fail(e, DPC_ERR_DEVICE);
      break;
  }
  __syncwarp();
  return make_int2(extra, work);
}

// Start problem `job` in slot s (one warp): first tasks go to list l. A
// descriptor that cannot be valid (bad kind, size beyond the slot, missing
// array, source out of range, slot out of range) is not run: the slot is
// reported finished and the status says DPC_ERR_INVALID_ARG.
__device__ void admit(const Engine &e, const dpc_job &job, int s, int l) {
  const int lane = lane_id();
  const bool tree = job.kind == DPC_JOB_TREE_DESCENDANTS || job.kind == DPC_JOB_TREE_HEIGHT;
  const bool ok = (job.kind == DPC_JOB_SSSP || tree) && job.n >= 1 && job.n <= e.hdr->max_n && job.off &&
                  job.out && job.source >= 0 && job.source < job.n &&
                  (tree ? (job.n == 1 || job.col) : (job.m >= 0 && job.m <= e.hdr->max_m && (job.m == 0 || (job.col && job.w))));
  if (s < 0 || s >= e.hdr->slots) {
    if (lane == 0) eng_fail(e, DPC_ERR_INVALID_ARG);
    return;
  }
  if (!ok) {
    if (lane == 0) {
      eng_fail(e, DPC_ERR_INVALID_ARG);
      e.slots[s].phase = P_DONE;
      report_done(e, s);
    }
    __syncwarp();
    return;
  }
  Slot &sl = e.slots[s];
  if (lane == 0) {
    sl.job = job;
    sl.pending = 0;
    sl.round = 0;
    sl.nf = 0;
    sl.next_count = 0;
    sl.post_level = 0;
    sl.pre_edges = 0;
    *reinterpret_cast<volatile int *>(e.slot_state + s) = 1;
    atomicAdd(&e.hdr->active, 1);
  }
  __syncwarp();
  if (job.kind == DPC_JOB_SSSP) {
    if (lane == 0) {
      sl.phase = P_INIT;
      sl.pending = ceil_div(job.n, kInitItems);
    }
    __syncwarp();
    emit_ranges(e, l, T_INIT, s, 0, job.n, kInitItems, 0);
  } else {
    const TreeView v = tree_view(e, s);
    const int tc = e.hdr->tree_chunk;
    const int k = __ldg(job.off + job.source + 1) - __ldg(job.off + job.source);
    const int nu = k > 0 ? ceil_div(k, tc) : 0;
    for (int q = lane; q < nu; q += kWarp) v.units[q] = make_int2(job.source, q);
    if (lane == 0) {
      // the root: its own token, no parent, at least 1 high when it has children
      static_cast<int *>(job.out)[job.source] = job.kind == DPC_JOB_TREE_HEIGHT && nu > 0 ? 1 : 0;
      v.link[job.source] = 1ull << 32;
      v.par[job.source] = -1;
      v.levels[0] = 0;
      v.levels[1] = nu;
      sl.next_count = (unsigned long long)nu;
      sl.phase = P_VISIT;
      sl.pending = ceil_div(nu, kTreeItems);
    }
    __syncwarp();
    if (nu == 0) {
      if (lane == 0) {
        sl.phase = P_DONE;
        report_done(e, s);
        atomicSub(&e.hdr->active, 1);
      }
      __syncwarp();
      return;
    }
    emit_ranges(e, l, T_VISIT, s, 0, nu, kTreeItems, 0);
  }
}

// Grid-wide barrier for a co-resident (cooperative) grid; bounded spin. False
// when the wait ran out (the status word then says DPC_ERR_TIMEOUT). The last
// block to arrive snapshots the next wave's task count, the active count and
// the status before it releases the others: they cannot change until every
// block has read them (no block can reach the next release before all arrive).
// The mailbox's posted count. When it has moved past `seen`, the read is
// followed by a system-scope fence (acquire: the host's release store of the
// count orders its job descriptors before it); an unchanged count needs none,
// which keeps the fence off the barriers of a busy engine with nothing new.
__device__ __forceinline__ unsigned long long mailbox_posted(const dpc_mailbox *mb, unsigned long long seen) {
  const unsigned long long v = *reinterpret_cast<const volatile unsigned long long *>(&mb->posted);
  if (v != seen) __threadfence_system();
  return v;
}

// Resident form, by the barrier's last arriver: which mailbox jobs the coming
// wave admits (at most one per warp of the grid) and whether the kernel ends.
// An engine with nothing queued, active or posted polls the mailbox for up to
// kIdlePollNs; it ends on the host's stop request, or once its lifetime has
// passed. A busy engine ends after four lifetimes (its queue stays intact).
__device__ void serve_decision(const Engine &e, unsigned long long next_tasks, int active, unsigned status) {
  EngineHeader &h = *e.hdr;
  const unsigned long long now = global_ns();
  if (h.t_start == 0) {
    h.t_start = now;
    // the mailbox keeps its own count of admitted jobs; only this kernel
    // writes it, so a copy read once per launch stays current
    h.mb_seen = *reinterpret_cast<const volatile unsigned long long *>(&e.mb->taken);
  }
  const unsigned long long age = now - h.t_start;
  const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x / kWarp);
  const unsigned long long cap = DPC_MAILBOX_CAP < warps ? DPC_MAILBOX_CAP : warps;
  unsigned long long lo = h.mb_seen;
  unsigned long long posted = mailbox_posted(e.mb, lo);
  int exit_now = status != 0u || age > 4 * e.limit_ns;
  if (!exit_now && next_tasks == 0 && active != 0) {
    // an admitted problem with no task queued can never finish (a bug or malformed input)
    eng_fail(e, DPC_ERR_DEVICE);
    exit_now = 1;
  }
  if (!exit_now && next_tasks == 0 && active == 0 && posted == lo) {  // idle
    const unsigned stop = *reinterpret_cast<const volatile unsigned *>(&e.mb->stop);
    if (stop || age > e.limit_ns) {
      exit_now = 1;
    } else {
      const unsigned long long t0 = global_ns();
      while (posted == lo && global_ns() - t0 < kIdlePollNs) {
        __nanosleep(256);
        posted = mailbox_posted(e.mb, lo);
      }
    }
  }
  const unsigned long long hi = exit_now ? lo : (posted - lo > cap ? lo + cap : posted);
  h.snap_lo = lo;
  h.snap_hi = hi;
  if (hi != lo) {
    h.mb_seen = hi;
    *reinterpret_cast<volatile unsigned long long *>(&e.mb->taken) = hi;
  }
  h.snap_exit = exit_now;
}

// What every thread of a block needs after a barrier, read once per block by
// its master thread (every thread reading the same header words after every
// barrier put tens of thousands of requests on one L2 line per wave).
struct WaveState {
  unsigned long long n;     // tasks in the coming wave's list
  unsigned long long next;  // snapshot: tasks queued for the wave after a finished one
  int active;
  unsigned status;
  unsigned long long lo, hi;  // resident form: mailbox jobs the coming wave admits
  int exit;                   // resident form: the kernel ends
};
__shared__ WaveState s_wave;

// `wave_list`: the list the coming wave takes its tasks from.
__device__ bool grid_barrier(const Engine &e, int next_list, int wave_list) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *gen = &e.hdr->bar_gen;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(&e.hdr->bar_count, 1u) == gridDim.x - 1) {
      __threadfence();
      e.hdr->snap_count = next_list >= 0 ? *reinterpret_cast<volatile unsigned long long *>(&e.hdr->count[next_list]) : 0;
      e.hdr->snap_active = *reinterpret_cast<volatile int *>(&e.hdr->active);
      e.hdr->snap_status = *reinterpret_cast<volatile unsigned *>(&e.hdr->status);
      if (e.mb) serve_decision(e, e.hdr->snap_count, e.hdr->snap_active, e.hdr->snap_status);
      e.hdr->bar_count = 0;
      __threadfence();
      atomicAdd(&e.hdr->bar_gen, 1u);
    } else {
      WaitClock clk;
      while (*gen == g0) {
        __nanosleep(100);
        if (clk.expired()) {
          eng_fail(e, DPC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (ok) {
      const EngineHeader *h = e.hdr;
      s_wave.n = *reinterpret_cast<const volatile unsigned long long *>(&h->count[wave_list]);
      s_wave.next = *reinterpret_cast<const volatile unsigned long long *>(&h->snap_count);
      s_wave.active = *reinterpret_cast<const volatile int *>(&h->snap_active);
      s_wave.status = *reinterpret_cast<const volatile unsigned *>(&h->snap_status);
      s_wave.lo = *reinterpret_cast<const volatile unsigned long long *>(&h->snap_lo);
      s_wave.hi = *reinterpret_cast<const volatile unsigned long long *>(&h->snap_hi);
      s_wave.exit = *reinterpret_cast<const volatile int *>(&h->snap_exit);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace

__global__ void __launch_bounds__(256) engine_kernel(Engine e, const dpc_job *__restrict__ new_jobs,
                                                     const int *__restrict__ new_slots,
                                                     const int *__restrict__ new_count, int max_waves) {
  __shared__ int s_stage[256 / kWarp][kEngStage + 1];
  const int lane = lane_id();
  // resident form: this launch's lifetime starts at its first barrier
  if (e.mb && blockIdx.x == 0 && threadIdx.x == 0) e.hdr->t_start = 0;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const EngStage st{s_stage[threadIdx.x >> 5], &s_stage[threadIdx.x >> 5][kEngStage]};
  if (lane == 0) *st.cnt = 0;
  __syncwarp();
  long long wave = e.hdr->wave;
  // admissions go into the current wave's list
  {
    const int l = (int)(wave % 3);
    const int na = new_count ? *new_count : 0;
    for (int i = gw; i < na; i += nw) admit(e, new_jobs[i], new_slots[i], l);
  }
  // (resident form: the barrier's last arriver also takes the first mailbox posts)
  if (!grid_barrier(e, e.mb ? (int)(wave % 3) : -1, (int)(wave % 3))) return;
  unsigned long long relaxed = 0;
  for (int w = 0; w < max_waves; ++w, ++wave) {
    const int l = (int)(wave % 3), nl = (int)((wave + 1) % 3), ol = (int)((wave + 2) % 3);
    // the list consumed two waves ago is free: block 0 resets it for the next wave's producers
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      e.hdr->count[ol] = 0;
      e.hdr->cursor[ol] = 0;
    }
    if (e.mb) {
      // resident form: the jobs posted before the barrier, one warp each, into the next wave's list
      const unsigned long long lo = s_wave.lo, hi = s_wave.hi;
      if ((unsigned long long)gw < hi - lo) {
        const unsigned long long q = (lo + (unsigned long long)gw) % DPC_MAILBOX_CAP;
        dpc_job job;
        const int4 *src = reinterpret_cast<const int4 *>(&e.mb->jobs[q]);
        int4 *dst = reinterpret_cast<int4 *>(&job);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(dpc_job) / sizeof(int4)); ++k) dst[k] = __ldcv(src + k);
        admit(e, job, __ldcv(&e.mb->slots[q]), nl);
      }
    }
    const unsigned long long n = s_wave.n;
    // tasks are handed out kGrab at a time while many remain, one at a time near
    // the end of the wave: one shared cursor, far fewer atomics on it
    for (;;) {
      unsigned long long i = 0;
      int take = 1;
      if (lane == 0) {
        const unsigned long long c = *reinterpret_cast<volatile unsigned long long *>(&e.hdr->cursor[l]);
        take = (c + (unsigned long long)kGrab * 4 * (unsigned long long)nw < n) ? kGrab : 1;
        i = atomicAdd(&e.hdr->cursor[l], (unsigned long long)take);
      }
      i = __shfl_sync(0xffffffffu, i, 0);
      take = __shfl_sync(0xffffffffu, take, 0);
      if (i >= n) break;
      const unsigned long long end = i + take < n ? i + take : n;
      int cur = -1, delta = 0;
      for (unsigned long long k = i; k < end; ++k) {
        const int4 t = e.tasks[l][k];
        const int s = t.x & 0xFFFFFF;
        if (s != cur && cur >= 0) {
          eng_flush(e, cur, st);
          tasks_done(e, cur, delta, nl);
          delta = 0;
        }
        cur = s;
        const int2 rw = run_task(e, t, nl, st);
        delta += rw.x - 1;
        relaxed += (unsigned long long)rw.y;
      }
      if (cur >= 0) {
        eng_flush(e, cur, st);
        tasks_done(e, cur, delta, nl);
      }
    }
    if (!grid_barrier(e, nl, nl)) return;
    const unsigned long long nn = s_wave.next;
    const int active = s_wave.active;
    const unsigned status = s_wave.status;
    if (e.mb) {
      // resident form: idle waves go on (the barrier polled the mailbox) until the exit decision
      if (s_wave.exit) {
        ++wave;
        break;
      }
      continue;
    }
    if (nn == 0 || status != 0u) {
      // no task for the next wave: either every problem is finished, or one can
      // never finish (a bug or malformed input) - stop rather than spin on empty waves
      if (nn == 0 && active != 0 && blockIdx.x == 0 && threadIdx.x == 0) eng_fail(e, DPC_ERR_DEVICE);
      ++wave;
      break;
    }
  }
  if (e.stats) {
    relaxed = warp_sum(relaxed);
    if (lane == 0) stat_add(e.stats, &dpc_stats::relaxations, relaxed);
  }
  // wave count: every block computed the same value
  if (blockIdx.x == 0 && threadIdx.x == 0) e.hdr->wave = wave;
}

__global__ void engine_reset(EngineHeader *h, Slot *slots, int nslots, int *slot_state, int threshold, int chunk,
                             int tree_chunk, int max_n, int max_m, unsigned long long task_cap,
                             unsigned long long slot_bytes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nslots) {
    slots[i].phase = P_FREE;
    slot_state[i] = 0;
  }
  if (i == 0) {
    for (int l = 0; l < 3; ++l) {
      h->count[l] = 0;
      h->cursor[l] = 0;
    }
    h->bar_count = 0;
    h->bar_gen = 0;
    h->status = 0;
    h->active = 0;
    h->wave = 0;
    h->snap_lo = h->snap_hi = 0;
    h->snap_exit = 0;
    h->t_start = 0;
    h->slots = nslots;
    h->max_n = max_n;
    h->max_m = max_m;
    h->threshold = threshold;
    h->chunk = chunk;
    h->tree_chunk = tree_chunk;
    h->task_cap = task_cap;
    h->slot_bytes = slot_bytes;
  }
}

// ------------------------------------------------------------------ host side

namespace {

size_t slot_bytes_for(int max_n, int tree_chunk) {
  const size_t n = (size_t)max_n;
  const size_t sssp = align_up(n * sizeof(int2), 256) + align_up(n * sizeof(int), 256) +
                      align_up(n * sizeof(unsigned), 256);
  const size_t mu = (n > 0 ? n - 1 : 0) / (size_t)tree_chunk + n + 1;
  const size_t tree = align_up(mu * sizeof(int2), 256) + align_up((n + 2) * sizeof(int), 256) +
                      align_up(n * sizeof(int), 256) + align_up(n * sizeof(unsigned long long), 256);
  return align_up(sssp > tree ? sssp : tree, 256);
}

unsigned long long task_cap_for(int slots, int max_n, int max_m, int threshold, int chunk, int tree_chunk) {
  // per problem and wave: frontier/commit/init ranges, one EDGES task per chunk
  // of every large vertex, tree units / kTreeItems
  const unsigned long long n = (unsigned long long)max_n, m = (unsigned long long)max_m;
  unsigned long long large = m / ((unsigned long long)threshold + 1);
  if (large > n) large = n;
  const unsigned long long sssp = n / kRelaxItems + n / kCommitItems + n / kInitItems + m / chunk + large + 8;
  const unsigned long long tree = (n / tree_chunk + n + 1) / kTreeItems + 8;
  return (unsigned long long)slots * (sssp > tree ? sssp : tree) + 64;
}

struct Layout {
  size_t hdr, slots, tasks, scratch, total;
  unsigned long long task_cap;
  size_t slot_bytes;
};

Layout layout_for(int slots, int max_n, int max_m, int threshold, int chunk, int tree_chunk) {
  Layout L;
  L.task_cap = task_cap_for(slots, max_n, max_m, threshold, chunk, tree_chunk);
  L.slot_bytes = slot_bytes_for(max_n, tree_chunk);
  L.hdr = 0;
  L.slots = kHeaderBytes;
  L.tasks = L.slots + align_up((size_t)slots * sizeof(Slot), 256);
  L.scratch = L.tasks + 3 * align_up(L.task_cap * sizeof(int4), 256);
  L.total = L.scratch + (size_t)slots * L.slot_bytes;
  return L;
}

struct EngineCfg {
  int threshold, chunk, tree_chunk, threads;
};

dpc_status engine_cfg(const dpc_tuning *t, EngineCfg *c) {
  dpc_tuning z;
  std::memset(&z, 0, sizeof(z));
  if (!t) t = &z;
  c->threshold = t->threshold > 0 ? t->threshold : (t->threshold < 0 ? 0 : 32);
  c->chunk = t->chunk > 0 ? t->chunk : 512;  // 512 edges per EDGES task: the autotuner's pick on the served mix
  c->tree_chunk = kEngTreeChunk;
  c->threads = 256;
  if (t->chunk < 0 || c->chunk > (1 << 24)) return DPC_ERR_INVALID_ARG;
  return DPC_OK;
}

std::mutex g_eng_mu;
int g_eng_blocks[64];

int engine_grid(int dev) {
  std::lock_guard<std::mutex> lk(g_eng_mu);
  if (dev < 0 || dev >= 64) return 0;
  if (g_eng_blocks[dev] == 0) {
    int sms = 0, bps = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)engine_kernel, 256, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    g_eng_blocks[dev] = (bps > 0 ? bps : 1) * sms;
  }
  return g_eng_blocks[dev];
}

// slot_state may be device memory or pinned host memory (the resident form's
// host polls it); a pinned host array is used through its device address.
int32_t *state_for_device(int32_t *slot_state) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, slot_state) != cudaSuccess) {
    cudaGetLastError();
    return slot_state;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<int32_t *>(a.devicePointer);
  return slot_state;
}

Engine engine_view(void *ws, int slots, const Layout &L, int *slot_state, dpc_stats *stats) {
  Engine e;
  char *b = static_cast<char *>(ws);
  e.hdr = reinterpret_cast<EngineHeader *>(b + L.hdr);
  e.slots = reinterpret_cast<Slot *>(b + L.slots);
  for (int l = 0; l < 3; ++l)
    e.tasks[l] = reinterpret_cast<int4 *>(b + L.tasks + (size_t)l * align_up(L.task_cap * sizeof(int4), 256));
  e.scratch = reinterpret_cast<unsigned char *>(b + L.scratch);
  e.slot_state = slot_state;
  e.stats = stats;
  e.mb = nullptr;
  e.limit_ns = 0;
  (void)slots;
  return e;
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" {

dpc_status dpc_engine_workspace_size(int32_t slots, int32_t max_n, int32_t max_m, const dpc_tuning *tuning,
                                     size_t *bytes) {
  if (!bytes || slots < 1 || slots > (1 << 20) || max_n < 1 || max_m < 0) return DPC_ERR_INVALID_ARG;
  EngineCfg c;
  dpc_status st = engine_cfg(tuning, &c);
  if (st != DPC_OK) return st;
  *bytes = layout_for(slots, max_n, max_m, c.threshold, c.chunk, c.tree_chunk).total;
  return DPC_OK;
}

dpc_status dpc_engine_init(void *workspace, size_t workspace_bytes, int32_t slots, int32_t max_n, int32_t max_m,
                           const dpc_tuning *tuning, int32_t *slot_state, dpc_stream_t stream) {
  if (slots < 1 || slots > (1 << 20) || max_n < 1 || max_m < 0 || !slot_state) return DPC_ERR_INVALID_ARG;
  EngineCfg c;
  dpc_status st = engine_cfg(tuning, &c);
  if (st != DPC_OK) return st;
  const Layout L = layout_for(slots, max_n, max_m, c.threshold, c.chunk, c.tree_chunk);
  if (!workspace || workspace_bytes < L.total) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  slot_state = state_for_device(slot_state);
  Engine e = engine_view(workspace, slots, L, slot_state, nullptr);
  engine_reset<<<ceil_div(slots, 256), 256, 0, s>>>(e.hdr, e.slots, slots, slot_state, c.threshold, c.chunk,
                                                  c.tree_chunk, max_n, max_m, L.task_cap, L.slot_bytes);
  return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}

dpc_status dpc_engine_step(void *workspace, size_t workspace_bytes, int32_t slots, int32_t max_n, int32_t max_m,
                           const dpc_tuning *tuning, const dpc_job *new_jobs, const int32_t *new_slots,
                           const int32_t *new_count, int32_t max_waves, int32_t *slot_state, dpc_stats *stats,
                           dpc_stream_t stream) {
  if (slots < 1 || max_n < 1 || max_m < 0 || max_waves < 1 || !slot_state) return DPC_ERR_INVALID_ARG;
  if (new_count && (!new_jobs || !new_slots)) return DPC_ERR_INVALID_ARG;
  EngineCfg c;
  dpc_status st = engine_cfg(tuning, &c);
  if (st != DPC_OK) return st;
  const Layout L = layout_for(slots, max_n, max_m, c.threshold, c.chunk, c.tree_chunk);
  if (!workspace || workspace_bytes < L.total) return DPC_ERR_WORKSPACE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPC_ERR_CUDA;
  const int full = engine_grid(dev);
  if (full <= 0) return DPC_ERR_CUDA;
  // every block must be resident (cooperative launch): at most all of them, fewer on request
  const int blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks
                                                                                          : full;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (stats && cudaMemsetAsync(stats, 0, sizeof(dpc_stats), s) != cudaSuccess) return DPC_ERR_CUDA;
  Engine e = engine_view(workspace, slots, L, state_for_device(slot_state), stats);
  void *args[] = {&e, (void *)&new_jobs, (void *)&new_slots, (void *)&new_count, &max_waves};
  // cooperative launch: every block is resident, so the grid barrier cannot deadlock
  if (cudaLaunchCooperativeKernel((const void *)engine_kernel, dim3(blocks), dim3(256), args, 0, s) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return DPC_OK;
}

dpc_status dpc_mailbox_init(dpc_mailbox *mailbox) {
  if (!mailbox) return DPC_ERR_INVALID_ARG;
  std::memset(static_cast<void *>(mailbox), 0, sizeof(dpc_mailbox));
  return DPC_OK;
}

dpc_status dpc_mailbox_post(dpc_mailbox *mailbox, const dpc_job *job, int32_t slot) {
  if (!mailbox || !job || slot < 0) return DPC_ERR_INVALID_ARG;
  const uint64_t p = __atomic_load_n(&mailbox->posted, __ATOMIC_RELAXED);  // the only writer
  const uint64_t t = __atomic_load_n(&mailbox->taken, __ATOMIC_ACQUIRE);
  if (p - t >= (uint64_t)DPC_MAILBOX_CAP) return DPC_ERR_OVERFLOW;
  mailbox->jobs[p % DPC_MAILBOX_CAP] = *job;
  mailbox->slots[p % DPC_MAILBOX_CAP] = slot;
  // the descriptor (and every earlier store of this thread, such as the
  // slot's state set back to 0) before the count that publishes it
  __atomic_store_n(&mailbox->posted, p + 1, __ATOMIC_RELEASE);
  return DPC_OK;
}

dpc_status dpc_mailbox_stop(dpc_mailbox *mailbox) {
  if (!mailbox) return DPC_ERR_INVALID_ARG;
  __atomic_store_n(&mailbox->stop, 1u, __ATOMIC_RELEASE);
  return DPC_OK;
}

dpc_status dpc_mailbox_taken(const dpc_mailbox *mailbox, uint64_t *taken) {
  if (!mailbox || !taken) return DPC_ERR_INVALID_ARG;
  *taken = __atomic_load_n(&mailbox->taken, __ATOMIC_ACQUIRE);
  return DPC_OK;
}

dpc_status dpc_engine_serve(void *workspace, size_t workspace_bytes, int32_t slots, int32_t max_n, int32_t max_m,
                            const dpc_tuning *tuning, dpc_mailbox *mailbox, uint32_t limit_us, int32_t *slot_state,
                            dpc_stats *stats, dpc_stream_t stream) {
  if (slots < 1 || max_n < 1 || max_m < 0 || !mailbox || !slot_state || limit_us < 1 || limit_us > 10000000u)
    return DPC_ERR_INVALID_ARG;
  EngineCfg c;
  dpc_status st = engine_cfg(tuning, &c);
  if (st != DPC_OK) return st;
  const Layout L = layout_for(slots, max_n, max_m, c.threshold, c.chunk, c.tree_chunk);
  if (!workspace || workspace_bytes < L.total) return DPC_ERR_WORKSPACE;
  // the mailbox and the slot states must be pinned host memory the device can address
  void *d_mb = nullptr, *d_state = nullptr;
  if (cudaHostGetDevicePointer(&d_mb, mailbox, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(&d_state, slot_state, 0) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPC_ERR_CUDA;
  const int full = engine_grid(dev);
  if (full <= 0) return DPC_ERR_CUDA;
  const int blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks
                                                                                          : full;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (stats && cudaMemsetAsync(stats, 0, sizeof(dpc_stats), s) != cudaSuccess) return DPC_ERR_CUDA;
  Engine e = engine_view(workspace, slots, L, static_cast<int *>(d_state), stats);
  e.mb = static_cast<dpc_mailbox *>(d_mb);
  e.limit_ns = (unsigned long long)limit_us * 1000ull;
  const dpc_job *no_jobs = nullptr;
  const int32_t *no_slots = nullptr, *no_count = nullptr;
  int max_waves = INT_MAX;
  void *args[] = {&e, (void *)&no_jobs, (void *)&no_slots, (void *)&no_count, &max_waves};
  // cooperative launch: every block is resident, so the grid barrier cannot deadlock
  if (cudaLaunchCooperativeKernel((const void *)engine_kernel, dim3(blocks), dim3(256), args, 0, s) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return DPC_OK;
}

}  // extern "C"
