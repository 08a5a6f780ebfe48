// CSR sparse matrix-vector product y = A x at the five consolidation levels.
//
// The irregular loop of Sec. II.B: each parent thread owns a row; rows with
// more than `threshold` non-zeros are "large work" (the condition of Fig. 1a).
//   flat      the thread computes its whole row, however long (the no-dp code).
//   basic-DP  the thread launches a one-block child for its long row (Fig. 1a).
//   warp/block/grid
//             the thread appends its long row to the buffer of its warp, block
//             or grid (Sec. IV.B) and one consolidated child per buffer handles
//             every buffered row (Sec. IV.C, child transform "multi-block,
//             multi-thread": the child loops over buffered items and many
//             threads cooperate on each).
//   queue     the grid-level buffer without the child launch: the parent is a
//             cooperative grid that, once every block has buffered its long
//             rows, crosses a grid barrier and runs the child's loop over the
//             buffer itself - parent-waits-on-child as a persistent grid
//             instead of a launch, which saves the child's launch latency and
//             the wait for its completion.
//
// Buffer entries are work units rather than rows: a long row is cut into units
// of `chunk` non-zeros, each processed by one warp of the child, so a 200,000
// non-zero row is spread over the whole child grid instead of one block. A row
// split into several units is finished by whichever warp completes its last
// unit, which adds the unit partial sums in unit order: every level sums each
// row in a fixed order, so results are bitwise reproducible run to run. A unit
// carries its own range of non-zeros, (row, first non-zero, end of the row,
// first unit of the row), so processing it needs no row-offset lookup.
//
// The same kernels serve PageRank's pull step (rank.cu) in a second mode: a
// row is a vertex, its entries are the vertex's in-edges, every term is the
// gathered contribution x[src] with no stored value, and the row's result is
// written as alpha * sum + *beta (damping and teleport term).
#include "dpc_internal.h"
#include "dpc_runtime.cuh"
#include "rank_reduce.cuh"

namespace dpc {

namespace {

enum : int { kFull = 0 };

// MODE: kModeSpmv (terms val[k] * x[col[k]], y = sum) or kModeRank (terms
// x[col[k]], y = alpha * sum + *beta), see the file comment.
template <int MODE>
__device__ __forceinline__ float row_result(const SpmvParams &p, float s) {
  if (MODE == kModeRank) return fmaf(p.alpha, s, __ldcg(p.beta));
  return s;
}

__device__ __forceinline__ void spmv_fail(const SpmvParams &p, unsigned code) {
  set_status(&p.hdr->status, code);
  if (p.stats) atomicCAS(&p.stats->status, 0u, code);
}

// One thread, whole range, in order: the inline work of a parent thread. The
// loads of eight terms are issued before their products are accumulated, so a
// short row costs two dependent memory round trips per eight terms instead of
// two per term; the sum is still taken strictly left to right.
template <int MODE>
__device__ __forceinline__ float seq_dot(const SpmvParams &p, int a, int b) {
  checked_range(a, b, p.nnz, &p.hdr->status);
  float s = 0.f;
  int k = a;
  for (; k + 8 <= b; k += 8) {
    int c[8];
    float v[8], xv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = checked_index(__ldg(p.col + k + j), p.ncols, &p.hdr->status);
      v[j] = MODE == kModeSpmv ? __ldg(p.val + k + j) : 1.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      xv[j] = kCheckedBuild && c[j] < 0 ? 0.f : (MODE == kModeSpmv ? __ldg(p.x + c[j]) : __ldcg(p.x + c[j]));
#pragma unroll
    for (int j = 0; j < 8; ++j) s = MODE == kModeSpmv ? fmaf(v[j], xv[j], s) : s + xv[j];
  }
  if (k < b) {
    int c[8];
    float v[8], xv[8];
    const int r = b - k;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = j < r ? checked_index(__ldg(p.col + k + j), p.ncols, &p.hdr->status) : 0;
      v[j] = MODE == kModeSpmv ? (j < r ? __ldg(p.val + k + j) : 0.f) : 1.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      xv[j] = j < r && !(kCheckedBuild && c[j] < 0) ? (MODE == kModeSpmv ? __ldg(p.x + c[j]) : __ldcg(p.x + c[j]))
                                                      : 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < r) s = MODE == kModeSpmv ? fmaf(v[j], xv[j], s) : s + xv[j];
  }
  return s;
}

// Partial dot product of member t of a group of T threads over [a, b). Member
// t takes elements a+t, a+t+T, a+t+2T, ... sixteen at a time: sixteen coalesced
// col/val loads (adjacent members read adjacent elements), then sixteen
// independent x gathers, then the sums in element order. Adjacent members
// gather adjacent non-zeros of the row, so in long, dense rows neighbouring
// lanes often hit the same x sector and one request serves them. The gathers
// bypass L1 (.cg): with x far larger than L1 they would only evict each other.
constexpr int kDotBatch = 16;

template <int MODE>
__device__ __forceinline__ float group_dot(const SpmvParams &p, int a, int b, int t, int T) {
  checked_range(a, b, p.nnz, &p.hdr->status);
  float acc = 0.f;
  for (int i0 = a + t; i0 < b; i0 += kDotBatch * T) {
    int c[kDotBatch];
    float v[kDotBatch], xv[kDotBatch];
#pragma unroll
    for (int j = 0; j < kDotBatch; ++j) {
      const int i = i0 + j * T;
      c[j] = i < b ? checked_index(__ldcs(p.col + i), p.ncols, &p.hdr->status) : -1;
      v[j] = MODE == kModeSpmv ? (i < b ? __ldcs(p.val + i) : 0.f) : 1.f;
    }
#pragma unroll
    for (int j = 0; j < kDotBatch; ++j) xv[j] = c[j] >= 0 ? __ldcg(p.x + c[j]) : 0.f;
#pragma unroll
    for (int j = 0; j < kDotBatch; ++j)
      if (c[j] >= 0) acc = MODE == kModeSpmv ? fmaf(v[j], xv[j], acc) : acc + xv[j];
  }
  return acc;
}

// The end of unit u's sum s (already reduced over the warp): the row's result
// when the unit is the row's only one, else its partial sum, and the row's
// result from the warp that completes the row's last unit. Unit u of the
// buffer, e = (row, a, row_end, first), holds the non-zeros [a, b), b =
// min(a + chunk, row_end); the row's units are first, first + 1, ..., the last
// one reaching row_end, so the row has (u - first) + ceil((row_end - a) /
// chunk) of them.
template <int MODE>
__device__ __forceinline__ void unit_finish(const SpmvParams &p, int u, int4 e, int b, float s) {
  const int lane = lane_id();
  const int row = e.x, a = e.y, row_end = e.z, first = e.w;
  if (u == first && b == row_end) {  // the row's only unit
    if (lane == 0) p.y[row] = row_result<MODE>(p, s);
    return;
  }
  const int nun = (u - first) + ceil_div(row_end - a, p.chunk);
  unsigned last = 0;
  if (lane == 0) {
    p.partial[u] = s;
    __threadfence();
    last = (atomicAdd(p.ucount + first, 1u) == (unsigned)(nun - 1)) ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    float t = 0.f;
    for (int j = lane; j < nun; j += kWarp) t += __ldcg(p.partial + first + j);
    t = warp_sum(t);
    if (lane == 0) {
      p.y[row] = row_result<MODE>(p, t);
      // PageRank's persistent grid reuses the units every iteration
      if (MODE == kModeRank) p.ucount[first] = 0u;
    }
  }
}

// Unit u processed by a full warp.
template <int MODE>
__device__ __forceinline__ void spmv_unit(const SpmvParams &p, int u, int4 e) {
  if (e.x < 0) return;  // placeholder written after a buffer overflow
  const int b = min(e.z, e.y + p.chunk);
  unit_finish<MODE>(p, u, e, b, warp_sum(group_dot<MODE>(p, e.y, b, lane_id(), kWarp)));
}

// Units [lo, hi) processed by the warps of the calling group, warp-strided.
template <int MODE>
__device__ __forceinline__ void spmv_units_by_group(const SpmvParams &p, const int4 *units, int lo, int hi,
                                                    int warp_in_group, int warps_in_group) {
  for (int u = lo + warp_in_group; u < hi; u += warps_in_group) spmv_unit<MODE>(p, u, __ldcg(units + u));
}

// Units [0, n) handed to the calling warp from shared cursors (zero before
// the first warp starts). Row lengths vary, so a fixed warp-strided split ends
// with most of the grid waiting on its slowest warps; on the 1M-row s = 1.5
// matrix the cursor cut the unit phase by about 12 %. SpMV takes
// units_per_grab units at a time (one while units are few per warp: the
// mean-16 matrix 0.114 -> 0.107 ms); PageRank keeps kRankGrab, which measured
// 3-8 % faster than one at a time for its 512-edge units.
constexpr unsigned long long kRankGrab = 4;

// The units are split into kUnitCursors equal partitions, each with its own
// cursor on its own cache line (WsHeader::cursors): every atomic on one
// address serialises in one L2 slice at about 2 ns, and with small units (the
// mean-16 matrix: 35 K units of one row each) a single cursor made the unit
// loop wait on its atomics. A warp starts on the partition of its index and,
// once that one is exhausted, moves on to the next; every grab that lands
// inside the partition is processed by the warp that made it.
//
// The device-launched child (grid level) grabs when it needs a unit. The
// queue level, whose warps all start together, keeps its next grab in flight
// and loads the next unit while it processes the current one, so that
// neither round trip sits between two units. (In the child, whose blocks
// start while the parent still holds the GPU, grabbing ahead let the first
// warps reserve units that later ones would have taken: the grid level lost
// 2-5 %.)
template <int MODE>
__device__ __forceinline__ void spmv_units_on_demand(const SpmvParams &p, const int4 *units, int n,
                                                     unsigned long long *cursors) {
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned long long grab = MODE == kModeSpmv ? units_per_grab(n, nw) : kRankGrab;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int t = 0; t < kUnitCursors; ++t) {
    const int part = (w + t) % kUnitCursors;
    const int lo = (int)((long long)n * part / kUnitCursors), hi = (int)((long long)n * (part + 1) / kUnitCursors);
    for (;;) {
      unsigned long long i0 = 0;
      if (lane_id() == 0) i0 = atomicAdd(cursors + part * kCursorStride, grab);
      i0 = __shfl_sync(0xffffffffu, i0, 0) + (unsigned long long)lo;
      if (i0 >= (unsigned long long)hi) break;
      const int i1 = (int)min(i0 + grab, (unsigned long long)hi);
      for (int u = (int)i0; u < i1; ++u) spmv_unit<MODE>(p, u, __ldcg(units + u));
    }
  }
}

template <int MODE>
__device__ __forceinline__ void spmv_units_dynamic(const SpmvParams &p, const int4 *units, int n,
                                                   unsigned long long *cursors) {
  const int lane = lane_id();
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned long long grab = MODE == kModeSpmv ? units_per_grab(n, nw) : kRankGrab;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int t = 0; t < kUnitCursors; ++t) {
    const int part = (w + t) % kUnitCursors;
    const int lo = (int)((long long)n * part / kUnitCursors), hi = (int)((long long)n * (part + 1) / kUnitCursors);
    unsigned long long *cur = cursors + part * kCursorStride;
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(cur, grab);
    g = __shfl_sync(0xffffffffu, g, 0) + (unsigned long long)lo;
    if (g >= (unsigned long long)hi) continue;
    int u = (int)g, uend = (int)min(g + grab, (unsigned long long)hi);
    int4 e = __ldcg(units + u);
    unsigned long long gn = 0;  // the next grab (lane 0), in flight
    if (lane == 0) gn = atomicAdd(cur, grab);
    for (;;) {
      int un = u + 1, unend = uend;
      if (un >= uend) {
        const unsigned long long g2 = __shfl_sync(0xffffffffu, gn, 0) + (unsigned long long)lo;
        if (g2 < (unsigned long long)hi) {
          un = (int)g2;
          unend = (int)min(g2 + grab, (unsigned long long)hi);
          if (lane == 0) gn = atomicAdd(cur, grab);
        } else {
          un = -1;
        }
      }
      const int4 en = un >= 0 ? __ldcg(units + un) : make_int4(-1, 0, 0, 0);
      spmv_unit<MODE>(p, u, e);
      if (un < 0) break;
      u = un;
      uend = unend;
      e = en;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ kernels

// Consolidated child (moldable): every warp takes units of the buffer
// [lo, lo + n) until they are exhausted, whatever the grid size (Sec. IV.C) -
// from shared cursors when the child is the only one of its call (grid level,
// lo = 0), else round-robin. Unit indices are slots of the whole buffer
// (p.units), the numbering the units' first-unit fields use.
template <int MODE>
__global__ void __launch_bounds__(1024) spmv_child(SpmvParams p, int lo, int n, unsigned long long *cursor) {
  if (cursor) {
    spmv_units_on_demand<MODE>(p, p.units, n, cursor);
    return;
  }
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  spmv_units_by_group<MODE>(p, p.units, lo, lo + n, gw, nw);
}

// Launch the consolidated child for units [lo, lo + n) of the buffer from the device.
template <int MODE>
__device__ __forceinline__ cudaError_t launch_consolidated_child(const SpmvParams &p, int lo, int n,
                                                                 unsigned long long *cursor = nullptr) {
  spmv_child<MODE><<<child_grid_for(n, p.child_blocks, p.child_threads), p.child_threads, 0, cudaStreamFireAndForget>>>(
      p, lo, n, cursor);
  return cudaGetLastError();
}

// Flat: thread per row, the whole row in order. A plain loop: over rows of up
// to 200,000 terms the compiler's own pipelining beats the batched form.
template <int MODE>
__global__ void __launch_bounds__(1024) spmv_flat(SpmvParams p) {
  const int G = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p.nrows; r += G) {
    int a = __ldg(p.off + r), b = __ldg(p.off + r + 1);
    checked_range(a, b, p.nnz, &p.hdr->status);
    float s = 0.f;
    for (int k = a; k < b; ++k) {
      const int c = checked_index(__ldg(p.col + k), p.ncols, &p.hdr->status);
      if (kCheckedBuild && c < 0) continue;
      const float xv = MODE == kModeSpmv ? __ldg(p.x + c) : __ldcg(p.x + c);
      s = MODE == kModeSpmv ? fmaf(__ldg(p.val + k), xv, s) : s + xv;
    }
    p.y[r] = row_result<MODE>(p, s);
  }
}

// Basic-DP child: one block cooperates on one row (solo block, Sec. IV.C).
template <int MODE>
__global__ void __launch_bounds__(1024) spmv_row_child(SpmvParams p, int row) {
  __shared__ float sm[32];
  const int a = __ldg(p.off + row), b = __ldg(p.off + row + 1);
  float s = group_dot<MODE>(p, a, b, threadIdx.x, blockDim.x);
  s = block_sum(s, sm);
  if (threadIdx.x == 0) p.y[row] = row_result<MODE>(p, s);
}

// Basic-DP parent (Fig. 1a): a thread with a long row launches its own child.
template <int MODE>
__global__ void __launch_bounds__(1024) spmv_basic_parent(SpmvParams p) {
  const int G = gridDim.x * blockDim.x;
  unsigned long long launched = 0, inl = 0, failed = 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p.nrows; r += G) {
    const int a = __ldg(p.off + r), b = __ldg(p.off + r + 1);
    if (b - a > p.threshold) {
      if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
        spmv_row_child<MODE><<<1, p.child_threads, 0, cudaStreamFireAndForget>>>(p, r);
        if (cudaGetLastError() == cudaSuccess) {
          launched++;
          continue;
        }
      }
      failed++;
    } else {
      inl++;
    }
    p.y[r] = row_result<MODE>(p, seq_dot<MODE>(p, a, b));
  }
  if (p.stats) {
    launched = warp_sum(launched);
    inl = warp_sum(inl);
    failed = warp_sum(failed);
    if (lane_id() == 0) {
      stat_add(p.stats, &dpc_stats::child_launches, launched);
      stat_add(p.stats, &dpc_stats::buffered_items, launched + failed);
      stat_add(p.stats, &dpc_stats::inline_items, inl);
      stat_add(p.stats, &dpc_stats::launch_failures, failed);
    }
  }
}

// Rows a parent thread keeps in registers between its passes: rows t, t + G,
// ..., up to kRowRegs of them (t the thread's index in the grid, G the grid's
// thread count), as (first non-zero, length). With more rows per thread the
// passes load the offsets again.
constexpr int kRowRegs = 8;

// The long row at (start a, length len) of row r into the buffer from unit
// slot pos on: its ceil(len / chunk) units. Returns the slot after them.
template <int MODE>
__device__ __forceinline__ int write_row_units(const SpmvParams &p, int r, int a, int len, int pos) {
  const int nu = ceil_div(len, p.chunk);
  for (int k = 0; k < nu; ++k) p.units[pos + k] = make_int4(r, a + k * p.chunk, a + len, pos);
  p.ucount[pos] = 0u;
  return pos + nu;
}

// The short rows of this thread computed inline (rows handed to the buffer
// skipped while the group's buffer holds them, `buffered`): from the
// registers of pass 1 (regs), else with the offsets loaded again. (Summing
// four rows side by side in steps of two terms, to keep more loads in flight,
// was slower: a warp's loop then runs until the longest of 128 rows is done.)
template <int MODE>
__device__ __forceinline__ unsigned long long spmv_short_rows(const SpmvParams &p, bool regs, const int *ra,
                                                               const int *rl, int t0, int G, bool buffered) {
  unsigned long long inl = 0;
  if (regs) {
#pragma unroll
    for (int j = 0; j < kRowRegs; ++j) {
      if (rl[j] < 0 || (buffered && rl[j] > p.threshold)) continue;
      p.y[t0 + j * G] = row_result<MODE>(p, seq_dot<MODE>(p, ra[j], ra[j] + rl[j]));
      inl++;
    }
  } else {
    for (int r = t0; r < p.nrows; r += G) {
      const int a = __ldg(p.off + r), b = __ldg(p.off + r + 1);
      if (buffered && b - a > p.threshold) continue;  // handed to the child
      p.y[r] = row_result<MODE>(p, seq_dot<MODE>(p, a, b));
      inl++;
    }
  }
  return inl;
}

// Warp-, block-, grid- and queue-level consolidated parent (Fig. 4b). The first pass
// loads the thread's row offsets and counts the units of its long rows, so
// that the warp (block) reserves its whole buffer with one atomic - the exact
// per-buffer size that the paper's perBufferSize rule estimates (Sec. IV.E);
// each thread then writes its long rows' units into its own stretch of the
// reserved slice, at the offset given by a warp (block) scan; then the
// scope's barrier and the launch; the third pass computes the short rows
// inline while the child already runs (the paper's postwork position, Fig.
// 4b, holds no work here). The queue level arrives at its grid barrier, does
// its short rows and only then waits, so the barrier's latency and the
// blocks' uneven arrival hide behind that work.
template <int LEVEL, int MODE>
__global__ void __launch_bounds__(1024) spmv_parent(SpmvParams p) {
  __shared__ int s_scan[33];
  __shared__ int s_base, s_fail;
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool regs = (long long)p.nrows <= (long long)kRowRegs * G;

  // pass 1: the thread's rows and the units of its long ones
  int ra[kRowRegs], rl[kRowRegs];
  int mine = 0;
  if (regs) {
#pragma unroll
    for (int j = 0; j < kRowRegs; ++j) {
      ra[j] = 0;
      rl[j] = -1;
      const long long r = (long long)t0 + (long long)j * G;
      if (r < p.nrows) {
        int a = __ldg(p.off + r), b = __ldg(p.off + r + 1);
        checked_range(a, b, p.nnz, &p.hdr->status);
        ra[j] = a;
        rl[j] = b - a;
      }
    }
#pragma unroll
    for (int j = 0; j < kRowRegs; ++j)
      if (rl[j] > p.threshold) mine += ceil_div(rl[j], p.chunk);
  } else {
    for (int r = t0; r < p.nrows; r += G) {
      const int len = __ldg(p.off + r + 1) - __ldg(p.off + r);
      if (len > p.threshold) mine += ceil_div(len, p.chunk);
    }
  }
  // reserve the group's slice of the unit list; the thread's stretch starts at pos
  int base, gtotal, pos;
  if (LEVEL == DPC_BLOCK || LEVEL == DPC_QUEUE) {
    const int excl = block_exclusive_scan(mine, s_scan, &gtotal);
    if (threadIdx.x == 0) s_base = gtotal ? (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal) : 0;
    __syncthreads();
    base = s_base;
    pos = base + excl;
    if (base + gtotal > p.max_units) {  // only reachable with malformed offsets
      if (threadIdx.x == 0) spmv_fail(p, DPC_ERR_OVERFLOW);
      for (int j = base + threadIdx.x; j < min(base + gtotal, p.max_units); j += blockDim.x)
        p.units[j] = make_int4(-1, 0, 1, 0);
      gtotal = 0;
    }
  } else {
    const int inc = warp_inclusive_scan(mine);
    gtotal = __shfl_sync(0xffffffffu, inc, kWarp - 1);
    int b0 = 0;
    if (lane == 0 && gtotal) b0 = (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal);
    base = __shfl_sync(0xffffffffu, b0, 0);
    pos = base + inc - mine;
    if (base + gtotal > p.max_units) {  // only reachable with malformed offsets
      if (lane == 0) spmv_fail(p, DPC_ERR_OVERFLOW);
      for (int j = base + lane; j < min(base + gtotal, p.max_units); j += kWarp) p.units[j] = make_int4(-1, 0, 1, 0);
      gtotal = 0;
    }
  }

  // pass 2: long rows into the buffer
  unsigned long long buf = 0;
  if (gtotal) {
    if (regs) {
#pragma unroll
      for (int j = 0; j < kRowRegs; ++j) {
        if (rl[j] <= p.threshold) continue;
        pos = write_row_units<MODE>(p, t0 + j * G, ra[j], rl[j], pos);
        buf++;
      }
    } else {
      for (int r = t0; r < p.nrows; r += G) {
        int a = __ldg(p.off + r), b = __ldg(p.off + r + 1);
        checked_range(a, b, p.nnz, &p.hdr->status);
        if (b - a <= p.threshold) continue;
        pos = write_row_units<MODE>(p, r, a, b - a, pos);
        buf++;
      }
    }
  }

  // barrier of the consolidation scope, then one selected thread launches
  unsigned long long inl = 0;
  if (LEVEL == DPC_WARP) {
    __threadfence();
    __syncwarp();
    if (gtotal) {
      int failed = 0;
      if (lane == 0) {
        failed = 1;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          failed = launch_consolidated_child<MODE>(p, base, gtotal) != cudaSuccess;
        }
        stat_add(p.stats, failed ? &dpc_stats::launch_failures : &dpc_stats::child_launches, 1);
      }
      failed = __shfl_sync(0xffffffffu, failed, 0);
      if (failed) spmv_units_by_group<MODE>(p, p.units, base, base + gtotal, 0, 1);
    }
  } else if (LEVEL == DPC_BLOCK) {
    __threadfence();
    __syncthreads();
    if (gtotal) {
      if (threadIdx.x == 0) {
        s_fail = 1;
        if (take_launch_slot(&p.hdr->launches, p.launch_budget)) {
          s_fail = launch_consolidated_child<MODE>(p, base, gtotal) != cudaSuccess;
        }
        stat_add(p.stats, s_fail ? &dpc_stats::launch_failures : &dpc_stats::child_launches, 1);
      }
      __syncthreads();
      if (s_fail) spmv_units_by_group<MODE>(p, p.units, base, base + gtotal, threadIdx.x >> 5, blockDim.x >> 5);
    }
  } else if (LEVEL == DPC_QUEUE) {
    // every block has buffered its long rows once all have arrived; then the
    // whole grid runs the consolidated child's loop over the buffer
    grid_arrive(&p.hdr->done_blocks2);
    inl = spmv_short_rows<MODE>(p, regs, ra, rl, t0, G, gtotal != 0);
    if (grid_wait_all(&p.hdr->done_blocks2)) {
      const int total = (int)min(*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                                 (unsigned long long)p.max_units);
      spmv_units_dynamic<MODE>(p, p.units, total, p.hdr->cursors);
    } else if (threadIdx.x == 0) {
      spmv_fail(p, DPC_ERR_TIMEOUT);
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
            s_fail = launch_consolidated_child<MODE>(p, 0, total, p.hdr->cursors) != cudaSuccess;
          }
          stat_add(p.stats, s_fail ? &dpc_stats::launch_failures : &dpc_stats::child_launches, 1);
        }
      }
      __syncthreads();
      if (s_fail) spmv_units_by_group<MODE>(p, p.units, 0, s_base, threadIdx.x >> 5, blockDim.x >> 5);
    }
  }

  // pass 3: short rows inline. This comes after the launch so that the
  // consolidated child runs while the parent threads finish their own rows
  // (the queue level did them between the halves of its barrier). The offsets
  // are loaded again: kept in registers across the device launch, they spilled.
  if (LEVEL != DPC_QUEUE) inl = spmv_short_rows<MODE>(p, false, ra, rl, t0, G, gtotal != 0);
  if (p.stats) {
    inl = warp_sum(inl);
    buf = warp_sum(buf);
    if (lane == 0) {
      stat_add(p.stats, &dpc_stats::inline_items, inl);
      stat_add(p.stats, &dpc_stats::buffered_items, buf);
    }
  }
}

// ------------------------------------------------------------------ PageRank, persistent form

// The queue level of PageRank: every iteration in one cooperative grid. The
// in-edge structure does not change between iterations, so the long rows are
// buffered once; then per iteration: contributions and the dangling sum, a
// grid barrier, the teleport term (every block adds the chunk sums in the
// same fixed order, so all get the same bits), the consolidated loop over the
// buffer and the short rows, a grid barrier. The dangling sum has the fixed
// shape of rank_reduce.cuh, so this level agrees with the others to the bit.
// Data written during the kernel
// (ranks, contributions, partial sums, units) is read through L2 (.cg), never
// through the non-coherent caches.
__global__ void __launch_bounds__(1024) rank_queue_kernel(RankQueueArgs a) {
  __shared__ int s_scan[33];
  __shared__ int s_base;
  SpmvParams p = a.p;
  const int lane = lane_id();
  const int G = gridDim.x * blockDim.x;
  const int bstart = blockIdx.x * blockDim.x;
  const int gw = (bstart + threadIdx.x) >> 5, W = G >> 5;
  float *bufs[2] = {a.rank, a.tmp};
  // rank_t lives in the caller's array when iterations - t is even
  auto buf = [&](int t) { return bufs[((a.iterations - t) & 1) ? 1 : 0]; };
  const float r0 = 1.f / (float)p.nrows;
  for (int v = bstart + threadIdx.x; v < p.nrows; v += G) buf(0)[v] = r0;

  // the long rows' units, once (block-scope reservation, as at the queue level of SpMV)
  int mine = 0;
  for (int r = bstart + threadIdx.x; r < p.nrows; r += G) {
    const int len = __ldg(p.off + r + 1) - __ldg(p.off + r);
    if (len > p.threshold) mine += ceil_div(len, p.chunk);
  }
  int gtotal = block_sum(mine, s_scan);
  if (threadIdx.x == 0) s_base = gtotal ? (int)atomicAdd(&p.hdr->cursor, (unsigned long long)gtotal) : 0;
  __syncthreads();
  const int base = s_base;
  if (base + gtotal > p.max_units) {  // only reachable with malformed offsets
    if (threadIdx.x == 0) spmv_fail(p, DPC_ERR_OVERFLOW);
    for (int j = base + threadIdx.x; j < min(base + gtotal, p.max_units); j += blockDim.x)
      p.units[j] = make_int4(-1, 0, 1, 0);
    gtotal = 0;
  }
  int run = base;
  unsigned long long buffered = 0, inl = 0;
  for (int r0i = bstart; r0i < p.nrows; r0i += G) {
    const int r = r0i + threadIdx.x;
    int nu = 0, ra = 0, len = 0;
    if (r < p.nrows && gtotal) {
      int rb = __ldg(p.off + r + 1);
      ra = __ldg(p.off + r);
      checked_range(ra, rb, p.nnz, &p.hdr->status);
      len = rb - ra;
      if (len > p.threshold) nu = ceil_div(len, p.chunk);
    }
    int step;
    const int excl = block_exclusive_scan(nu, s_scan, &step);
    if (nu) {
      write_row_units<kModeRank>(p, r, ra, len, run + excl);
      buffered++;
    } else if (r < p.nrows) {
      inl++;
    }
    run += step;
  }
  unsigned k = 0;
  if (!grid_barrier_seq(&p.hdr->done_blocks2, ++k)) {
    if (threadIdx.x == 0) spmv_fail(p, DPC_ERR_TIMEOUT);
    return;
  }
  const int total = (int)min(*reinterpret_cast<volatile unsigned long long *>(&p.hdr->cursor),
                             (unsigned long long)p.max_units);
  const unsigned long long grab = kRankGrab;
  float *beta = a.betas + blockIdx.x;
  p.beta = beta;
  p.x = a.contrib;
  const int chunks = ceil_div(p.nrows, kRankChunk);
  for (int t = 0; t < a.iterations; ++t) {
    const float *rin = buf(t);
    p.y = buf(t + 1);
    // contributions and the dangling rank, chunk by chunk (the prep kernel's shape)
    if (bstart + threadIdx.x == 0) p.hdr->aux[2] = 0ull;  // the unit cursor of this iteration
    for (int c = gw; c < chunks; c += W) {
      const float sc = rank_chunk(rin, a.outdeg, a.contrib, p.nrows, c);
      if (lane == 0) a.partials[c] = sc;
    }
    if (!grid_barrier_seq(&p.hdr->done_blocks2, ++k)) {
      if (threadIdx.x == 0) spmv_fail(p, DPC_ERR_TIMEOUT);
      return;
    }
    // every block adds the chunk sums the same way: the same teleport term everywhere
    if (threadIdx.x < kWarp) {
      const float D = rank_total(a.partials, chunks);
      if (threadIdx.x == 0) *beta = teleport_term(a.damping, D, p.nrows);
    }
    __syncthreads();
    // units written by this kernel: read through L2
    for (;;) {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&p.hdr->aux[2], grab);
      i0 = __shfl_sync(0xffffffffu, i0, 0);
      if (i0 >= (unsigned long long)total) break;
      const int i1 = (int)min(i0 + grab, (unsigned long long)total);
      for (int u = (int)i0; u < i1; ++u) spmv_unit<kModeRank>(p, u, __ldcg(p.units + u));
    }
    for (int r = bstart + threadIdx.x; r < p.nrows; r += G) {
      const int aa = __ldg(p.off + r), bb = __ldg(p.off + r + 1);
      if (gtotal && bb - aa > p.threshold) continue;  // in the buffer
      p.y[r] = row_result<kModeRank>(p, seq_dot<kModeRank>(p, aa, bb));
    }
    if (!grid_barrier_seq(&p.hdr->done_blocks2, ++k)) {
      if (threadIdx.x == 0) spmv_fail(p, DPC_ERR_TIMEOUT);
      return;
    }
  }
  if (p.stats) {
    buffered = warp_sum(buffered) * (unsigned long long)a.iterations;
    inl = warp_sum(inl) * (unsigned long long)a.iterations;
    if (lane == 0) {
      stat_add(p.stats, &dpc_stats::buffered_items, buffered);
      stat_add(p.stats, &dpc_stats::inline_items, inl);
      if (bstart + threadIdx.x == 0) atomicMax(&p.stats->rounds, (unsigned)a.iterations);
    }
  }
}

const void *rank_queue_kernel_ptr() { return (const void *)rank_queue_kernel; }

cudaError_t rank_queue_launch(const RankQueueArgs &a, int blocks, int threads, cudaStream_t s) {
  RankQueueArgs q = a;
  void *args[] = {&q};
  return cudaLaunchCooperativeKernel((const void *)rank_queue_kernel, dim3(blocks), dim3(threads), args, 0, s);
}

// ------------------------------------------------------------------ host side

size_t spmv_max_units(int nrows, int nnz, int threshold, int chunk) {
  // a long row of L non-zeros yields ceil(L/chunk) <= L/chunk + 1 units, and
  // there are at most min(nrows, nnz/(threshold+1)) long rows
  size_t long_rows = (size_t)nnz / ((size_t)threshold + 1);
  if (long_rows > (size_t)nrows) long_rows = (size_t)nrows;
  return (size_t)nnz / (size_t)chunk + long_rows + 1;
}

size_t spmv_workspace_bytes(int nrows, int nnz, dpc_level level, const LaunchCfg &c) {
  size_t bytes = kHeaderBytes;
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE) {
    const size_t mu = spmv_max_units(nrows, nnz, c.threshold, c.chunk);
    bytes += align_up(mu * sizeof(int4), 256);
    bytes += align_up(mu * sizeof(float), 256);
    bytes += align_up(mu * sizeof(unsigned), 256);
  }
  return bytes;
}

template <int MODE>
const void *parent_kernel_of(dpc_level level) {
  switch (level) {
    case DPC_FLAT: return (const void *)spmv_flat<MODE>;
    case DPC_BASIC_DP: return (const void *)spmv_basic_parent<MODE>;
    case DPC_WARP: return (const void *)spmv_parent<DPC_WARP, MODE>;
    case DPC_BLOCK: return (const void *)spmv_parent<DPC_BLOCK, MODE>;
    case DPC_GRID: return (const void *)spmv_parent<DPC_GRID, MODE>;
    case DPC_QUEUE: return (const void *)spmv_parent<DPC_QUEUE, MODE>;
  }
  return nullptr;
}

const void *spmv_parent_kernel(dpc_level level, int mode) {
  return mode == kModeRank ? parent_kernel_of<kModeRank>(level) : parent_kernel_of<kModeSpmv>(level);
}

const void *spmv_child_kernel(dpc_level level, int mode) {
  if (level == DPC_QUEUE) return nullptr;
  if (mode == kModeRank)
    return level == DPC_BASIC_DP ? (const void *)spmv_row_child<kModeRank> : (const void *)spmv_child<kModeRank>;
  return level == DPC_BASIC_DP ? (const void *)spmv_row_child<kModeSpmv> : (const void *)spmv_child<kModeSpmv>;
}

template <int MODE>
cudaError_t launch_mode(const SpmvParams &p, dpc_level level, const LaunchCfg &c, cudaStream_t s) {
  const dim3 grid(c.parent_blocks), block(c.parent_threads);
  switch (level) {
    case DPC_FLAT: spmv_flat<MODE><<<grid, block, 0, s>>>(p); break;
    case DPC_BASIC_DP: spmv_basic_parent<MODE><<<grid, block, 0, s>>>(p); break;
    case DPC_WARP: spmv_parent<DPC_WARP, MODE><<<grid, block, 0, s>>>(p); break;
    case DPC_BLOCK: spmv_parent<DPC_BLOCK, MODE><<<grid, block, 0, s>>>(p); break;
    case DPC_GRID: spmv_parent<DPC_GRID, MODE><<<grid, block, 0, s>>>(p); break;
    case DPC_QUEUE: {
      // cooperative: every block resident, so the grid barrier cannot deadlock
      SpmvParams q = p;
      void *args[] = {&q};
      return cudaLaunchCooperativeKernel((const void *)spmv_parent<DPC_QUEUE, MODE>, grid, block, args, 0, s);
    }
  }
  return cudaGetLastError();
}

cudaError_t spmv_launch(const SpmvParams &p, dpc_level level, const LaunchCfg &c, cudaStream_t s, int mode) {
  return mode == kModeRank ? launch_mode<kModeRank>(p, level, c, s) : launch_mode<kModeSpmv>(p, level, c, s);
}

}  // namespace dpc
