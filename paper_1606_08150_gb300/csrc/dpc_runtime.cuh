// Consolidation runtime: device primitives shared by the application kernels.
//
// Sec. IV.B of the paper defines three consolidation granularities. A parent
// thread whose work item is too large (or recursive) appends the item to a
// buffer owned by its warp, its block or the whole grid; after a barrier of the
// same scope one selected thread launches a single child kernel for the buffer
// (Fig. 4b). This header provides the pieces that make that cheap on sm_103a:
//   - warp and block scans used to give every buffered item its slot in one
//     pass, so a warp or block reserves its whole buffer with one atomic;
//   - the grid-wide "last block done" ticket (the global barrier counter of
//     Sec. IV.E), which lets the last block launch the grid's child without any
//     block waiting for another (so no co-residency deadlock);
//   - device-side statistics and the status word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dpc.h"

namespace dpc {

constexpr int kWarp = 32;

// Device-side error codes share the numbering of dpc_status.
__device__ __forceinline__ void set_status(unsigned *status, unsigned code) {
  if (status) atomicCAS(status, 0u, code);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & (kWarp - 1); }

// The bounds-checked build (compiled with -DDPC_CHECKED; the library's second
// build, a stand-in for a memory checker): every index read from the caller's
// arrays and every append into a bounded buffer goes through checked(), which
// records DPC_ERR_OVERFLOW in the status word and tells the caller to skip the
// access when the index is out of range. In the regular build checked() is
// the constant true and the compiler removes it.
#ifdef DPC_CHECKED
constexpr bool kCheckedBuild = true;
#else
constexpr bool kCheckedBuild = false;
#endif

__device__ __forceinline__ bool checked(long long i, long long bound, unsigned *status) {
  if (!kCheckedBuild) return true;
  if (i >= 0 && i < bound) return true;
  set_status(status, DPC_ERR_OVERFLOW);
  return false;
}

// An index loaded from a caller's array (a column, a child id): itself, or -1
// (the kernels' "no entry") when the checked build finds it out of range.
__device__ __forceinline__ int checked_index(int v, int bound, unsigned *status) {
  return checked(v, bound, status) ? v : -1;
}

// An edge range [a, b) read from a caller's offsets: itself, or empty when
// the checked build finds it outside [0, m].
__device__ __forceinline__ void checked_range(int &a, int &b, long long m, unsigned *status) {
  if (!kCheckedBuild) return;
  if (a >= 0 && a <= b && b <= m) return;
  set_status(status, DPC_ERR_OVERFLOW);
  a = b = 0;
}

// Bounded waits. Every spin on a word that another block writes gives up once
// kWaitLimitNs of %globaltimer time have passed, or after kWaitPollCap polls
// should the clock not advance; the caller then reports DPC_ERR_TIMEOUT. A
// block that never arrives thus costs the others about two seconds instead of
// a hung GPU. The clock is first read at the 64th poll and then every 64
// polls, so the usual short wait never reads it.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
constexpr long long kWaitPollCap = 1ll << 26;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct WaitClock {
  unsigned long long t0;
  unsigned long long limit;
  long long polls;
  __device__ explicit WaitClock(unsigned long long limit_ns = kWaitLimitNs) : t0(0), limit(limit_ns), polls(0) {}
  // Called once per poll: true once the wait has run out.
  __device__ bool expired() {
    ++polls;
    if (polls > kWaitPollCap) return true;
    if ((polls & 63) != 0) return false;
    const unsigned long long now = global_ns();
    if (polls == 64) t0 = now;
    return now - t0 > limit;
  }
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Units a warp takes per atomic on a consolidated loop's shared unit cursor.
// With few units per warp one at a time spreads them evenly; with many, up to
// four at a time keeps the cursor's atomics (all on one address) from
// serialising. Measured on SSSP rounds: R-MAT 12 / 18 (2-8 units per warp)
// 0.31 -> 0.24 ms and 0.86 -> 0.73 ms with one instead of four; R-MAT 22
// (~36 per warp) 7.65 ms with one, 5.57 with four.
__device__ __forceinline__ unsigned long long units_per_grab(long long units, long long warps) {
  const long long g = units / (8 * (warps > 0 ? warps : 1));
  return g < 1 ? 1ull : (g > 4 ? 4ull : (unsigned long long)g);
}

// Inclusive scan over the 32 lanes of a full warp.
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
  for (int d = 1; d < kWarp; d <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, d);
    if ((int)lane_id() >= d) v += n;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Exclusive scan over a whole block (blockDim.x a multiple of 32, at most 1024).
// `smem` must hold 33 elements. Returns the thread's exclusive prefix and writes
// the block total to *total (identical in every thread). Contains three barriers
// (the first protects `smem` from a previous call still being read).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *smem, T *total) {
  const int lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive_scan(v);
  __syncthreads();
  if (lane == kWarp - 1) smem[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? smem[lane] : T(0);
    T si = warp_inclusive_scan(s);
    if (lane < nw) smem[lane] = si - s;
    if (lane == kWarp - 1) smem[32] = si;
  }
  __syncthreads();
  T r = smem[wid] + inc - v;
  *total = smem[32];
  return r;
}

// Block-wide sum in a fixed order (warp trees, then a tree over warp sums).
// `smem` must hold 32 elements. Every thread returns a sum of the same terms;
// use one fixed thread's value where bitwise reproducibility matters (the
// butterfly associates differently in different lanes). Two barriers.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *smem) {
  const int lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem[wid] = v;
  __syncthreads();
  T s = lane < nw ? smem[lane] : T(0);
  return warp_sum(s);
}

// Grid-level barrier of Sec. IV.E, in its non-blocking form: each block takes a
// ticket after making its writes visible; the block that draws the last ticket
// knows that every other block has finished its buffer insertions. The counter
// is reset by that block so the same workspace can serve the next grid.
// Must be called by all threads of the block; returns true in the last block.
__device__ __forceinline__ bool last_block_done(unsigned *counter) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
    if (s_last) {
      __threadfence();
      *counter = 0u;
    }
  }
  __syncthreads();
  return s_last != 0u;
}

// One-shot grid-wide barrier for a cooperative launch (every block resident),
// used once per call: `counter` must be zero when the grid starts. Each block
// arrives after making its writes visible (grid_arrive) and waits until all
// have arrived (grid_wait_all); work that needs nothing from the other blocks
// may run between the two halves. The wait is bounded (WaitClock); when it
// runs out grid_wait_all returns false in that block and the caller reports
// DPC_ERR_TIMEOUT instead of hanging. Both halves must be called by all
// threads of a block.
__device__ __forceinline__ void grid_arrive(unsigned *counter) {
  __syncthreads();  // orders the block's writes before its master thread's fence and arrival
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
  }
}

__device__ __forceinline__ bool grid_wait_all(unsigned *counter) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    WaitClock clk;
    while (*reinterpret_cast<volatile unsigned *>(counter) < gridDim.x) {
      __nanosleep(64);
      if (clk.expired()) {
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Multi-use blocking barrier of a cooperative grid: arrival counts only grow,
// so the k-th barrier of a call (k = 1, 2, ...) is complete once k * gridDim.x
// blocks have arrived; `counter` must be zero when the grid starts. Bounded
// wait (false when it runs out; the caller reports DPC_ERR_TIMEOUT).
__device__ __forceinline__ bool grid_barrier_seq(unsigned *counter, unsigned k) {
  __shared__ int s_ok2;
  __syncthreads();  // orders the block's writes before its master thread's fence and arrival
  if (threadIdx.x == 0) {
    __threadfence();
    int ok = 1;
    const unsigned target = k * gridDim.x;
    atomicAdd(counter, 1u);
    WaitClock clk;
    while (*reinterpret_cast<volatile unsigned *>(counter) < target) {
      __nanosleep(32);
      if (clk.expired()) {
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok2 = ok;
  }
  __syncthreads();
  return s_ok2 != 0;
}

// The device runtime's pending-launch pool must never overflow: on sm_103a a
// grid whose launches exceed it stalls instead of failing. Every optional
// device launch (one with an inline fallback) first takes a slot from the
// call's budget, which the host sizes below the pool; a refused slot means the
// work is done inline.
__device__ __forceinline__ bool take_launch_slot(unsigned long long *counter, long long budget) {
  return (long long)atomicAdd(counter, 1ull) < budget;
}

// Statistics (only when the caller passed a stats struct).
__device__ __forceinline__ void stat_add(dpc_stats *st, uint64_t dpc_stats::*field, unsigned long long v) {
  if (st && v) atomicAdd(reinterpret_cast<unsigned long long *>(&(st->*field)), v);
}

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Grid size for a consolidated child of `units` warp-sized work units: the KC_X
// configuration (resident blocks / X) of Sec. IV.E, never more blocks than there
// are units to hand out.
__device__ __forceinline__ int child_grid_for(int units, int kc_blocks, int child_threads) {
  int wpb = child_threads / kWarp;
  int need = (units + wpb - 1) / wpb;
  return need < kc_blocks ? (need > 0 ? need : 1) : kc_blocks;
}

}  // namespace dpc
