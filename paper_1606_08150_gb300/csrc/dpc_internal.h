// Internal interface between the C-ABI layer (api.cu) and the application
// kernels (spmv.cu, sssp.cu, tree.cu). Not installed; not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dpc.h"

namespace dpc {

// Launch shape resolved on the host from dpc_tuning and the device.
struct LaunchCfg {
  int threshold;
  int parent_blocks, parent_threads;
  int child_blocks;  // KC_X blocks for a consolidated child (upper bound per launch)
  int child_threads;
  int chunk;
  unsigned flags;
  unsigned delta;      // SSSP near-far split width (0: none)
  unsigned sub_delta;  // SSSP sub-split width for heavy vertices (0: none)
};

// Unit cursors of a consolidated loop: the units are split into kUnitCursors
// partitions, each with a cursor on its own 128-byte line (kCursorStride words).
constexpr int kUnitCursors = 8;
constexpr int kCursorStride = 16;

// Workspace header: counters that every call zeroes before its first kernel.
// Counters that many warps update in the same phase, and the word that the
// blocks of a grid barrier poll, sit on cache lines of their own: atomics on
// one line serialise in one L2 slice, and polls of a line slow its atomics.
struct WsHeader {
  // line 0: arrivals at the grid barriers (last-block tickets, multi-use barriers)
  unsigned done_blocks;
  unsigned done_blocks2;
  // line 1: the release word the waiting blocks poll, the status, the launch counter
  alignas(128) unsigned round;   // SSSP round / tree level reached; release word of the queue barriers
  unsigned status;               // device status (dpc_status numbering)
  unsigned long long launches;   // optional device launches attempted (checked against the budget)
  // line 2: units reserved in the current buffer
  alignas(128) unsigned long long cursor;
  // line 3: second list (SSSP next frontier, tree next level)
  alignas(128) unsigned long long cursor2;
  // line 4: per-application words (frontier size, snapshots, the child's unit cursor)
  alignas(128) unsigned long long aux[4];
  // line 5: SSSP commit counters (near-far split)
  alignas(128) unsigned long long nf_near;  // entries of the next frontier (the near set) written so far
  unsigned long long nf_elig;               // of those, the ones the next round relaxes
  unsigned nf_hmin;                         // smallest distance of a heavy near vertex that waits
  // line 6: the split (read by every phase, written between phases)
  alignas(128) unsigned nf_split;  // split distance S (all ones: no split; finite distances are below it)
  unsigned nf_sub;                 // sub-split distance s for heavy vertices (all ones: none)
  unsigned nf_split_old;           // S before the split in progress
  unsigned nf_dmin;                // smallest distance at or above S (split in progress)
  unsigned nf_done;                // 1: a split found no vertex at or above S (the run is over)
  unsigned nf_append;              // queue level: 1 when the coming round's parent phase may buffer units
  // lines 8-15: the unit cursors of a consolidated loop (SpMV), one partition each
  alignas(128) unsigned long long cursors[kUnitCursors * kCursorStride];
};
constexpr size_t kHeaderBytes = 2048;
static_assert(sizeof(WsHeader) <= kHeaderBytes, "workspace header too large");

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Host memory for the few small copies a host-driven level makes during a
// call (frontier sizes read back, a source index or a round count written).
// It outlives the call: a profiler that records a call's copies and replays
// them later then writes and reads live memory, never a returned stack frame.
struct HostScratch {
  unsigned long long count;
  unsigned long long sizes[3];
  int value;
  unsigned rounds;
};
inline HostScratch &host_scratch() {
  static thread_local HostScratch h;
  return h;
}

// ---------------------------------------------------------------- SpMV
struct SpmvParams {
  const int *off;
  const int *col;
  const float *val;
  const float *x;
  float *y;
  int nrows;
  int ncols;          // entries of x (column indices are below it)
  int nnz;            // entries of col (and val): row ranges lie in [0, nnz]
  int threshold;
  int chunk;
  int max_units;
  int child_blocks;
  int child_threads;
  float alpha;        // kModeRank: y = alpha * sum + *beta (PageRank's damping)
  const float *beta;  // kModeRank: device scalar written before the gather (teleport term)
  long long launch_budget;  // optional device launches allowed in this call
  int4 *units;      // (row, chunk index, units of the row, first unit of the row)
  float *partial;   // per-unit partial sums of rows split over several units
  unsigned *ucount; // per-row completion counters (indexed by the row's first unit)
  WsHeader *hdr;
  dpc_stats *stats;
};

// Row-gather modes of the SpMV kernels: y = A x, or PageRank's pull step
// (terms x[col] without stored values, y = alpha * sum + *beta).
enum : int { kModeSpmv = 0, kModeRank = 1 };

size_t spmv_max_units(int nrows, int nnz, int threshold, int chunk);
size_t spmv_workspace_bytes(int nrows, int nnz, dpc_level level, const LaunchCfg &c);
cudaError_t spmv_launch(const SpmvParams &p, dpc_level level, const LaunchCfg &c, cudaStream_t s,
                        int mode = kModeSpmv);
// Kernel handles for occupancy queries.
const void *spmv_parent_kernel(dpc_level level, int mode = kModeSpmv);
const void *spmv_child_kernel(dpc_level level, int mode = kModeSpmv);

// ---------------------------------------------------------------- PageRank
// One power iteration is a prep kernel (rank.cu) followed by the SpMV kernels
// in kModeRank over the in-edge CSR. The prep kernel turns rank_t into the
// contributions rank_t(u) / outdeg(u), sums the rank of dangling vertices in a
// fixed order, writes the teleport term *beta = (1-d)/n + d * dangling / n and
// resets the gather's workspace counters.
struct RankPrepParams {
  const float *rank_in;
  const int *outdeg;
  int n;
  float damping;
  int iteration;
  float *contrib;   // n
  float *partials;  // one dangling-rank sum per 1,024-vertex chunk
  float *beta;      // device scalar read by the gather
  WsHeader *hdr;    // the gather's workspace header
  dpc_stats *stats;
};
constexpr int kRankPrepBlocks = 1024;
constexpr int kRankPrepThreads = 256;

cudaError_t rank_init(float *rank, int n, cudaStream_t s);
cudaError_t rank_prep(const RankPrepParams &q, cudaStream_t s);

// The queue level: all iterations in one cooperative grid (spmv.cu).
struct RankQueueArgs {
  SpmvParams p;      // kModeRank gather over the in-edge CSR (y, x, beta set by the kernel)
  const int *outdeg;
  float *rank;       // caller's array
  float *tmp;        // second rank buffer
  float *contrib;    // n
  float *partials;   // one dangling-rank sum per 1,024-vertex chunk
  float *betas;      // one teleport term per block (every block computes the same)
  float damping;
  int iterations;
};
const void *rank_queue_kernel_ptr();
cudaError_t rank_queue_launch(const RankQueueArgs &a, int blocks, int threads, cudaStream_t s);

// ---------------------------------------------------------------- recursive BFS
constexpr int kBfsMaxChunk = 256;  // out-edges per unit: one batch of 8 per lane of a warp

struct BfsParams {
  const int *off;
  const int *col;
  unsigned *level;   // output: hop distance, 0xFFFFFFFF unreachable
  int n;
  int source;
  int chunk;         // out-edges per unit, 1..kBfsMaxChunk
  int child_blocks;  // KC_X blocks of a consolidated child
  int child_threads;
  int max_units;
  long long launch_budget;
  int2 *units;       // (vertex, chunk index): visits to run
  int *frontier;     // flat level: current and next frontier
  int *next;
  WsHeader *hdr;     // cursor: units reserved; aux[0]: the source's units; queue level:
                     // done_blocks2 / round / aux[1] are its barrier's arrivals, release and snapshot
  dpc_stats *stats;
};

// ---------------------------------------------------------------- graph colouring
struct GcParams {
  const int *off;
  const int *col;
  const unsigned *prio;  // caller's vertex priorities (ties: the larger id outranks)
  int *color;            // output: colour (round) of every vertex, 0 while uncoloured
  int n;
  int threshold;
  int chunk;
  int level;
  int parent_blocks;     // largest parent grid
  int parent_threads;
  int commit_blocks;
  int child_blocks;
  int child_threads;
  int max_units;
  long long launch_budget;
  int *list[2];          // uncoloured vertices: round r reads list[r & 1], fills list[(r + 1) & 1]
  int *heavy;            // the round's large vertices, decided by the commit
  unsigned *blocked;     // blocked[v] == r: an outranking competitor was found in round r
  int2 *units;           // (vertex, chunk index)
  WsHeader *hdr;         // aux[0]: uncoloured count of the round; aux[1]: large count;
                         // cursor: units; cursor2: next list; queue level: done_blocks2 / round barrier
  dpc_stats *stats;
};

size_t gc_max_units(int n, int m, int threshold, int chunk);
size_t gc_workspace_bytes(int n, int m, dpc_level level, const LaunchCfg &c);
cudaError_t gc_launch(GcParams &p, dpc_level level, int queue_blocks, cudaStream_t s);
const void *gc_parent_kernel(dpc_level level);
const void *gc_child_kernel(dpc_level level);

size_t bfs_max_units(int n, int m, int chunk, dpc_level level);
size_t bfs_workspace_bytes(int n, int m, dpc_level level, int chunk);
cudaError_t bfs_launch(BfsParams &p, dpc_level level, int root_blocks, int queue_blocks, cudaStream_t s);
const void *bfs_kernel(dpc_level level);

}  // namespace dpc

namespace dpc {

// ---------------------------------------------------------------- SSSP
struct SsspParams {
  const int *off;
  const int *col;
  const unsigned *w;
  unsigned *dist;
  int n;
  int m;
  int source;
  int threshold;
  int chunk;
  int level;
  int parent_blocks;  // largest parent grid (persistent size)
  int parent_threads;
  int commit_blocks;
  int child_blocks;
  int child_threads;
  int max_units;
  int heap;           // 1: warp and block buffers come from the device heap (DPC_FLAG_DEVICE_MALLOC)
  int stream_edges;   // 1: col/w larger than half of L2, read with the evict-first hint
  unsigned delta;     // near-far split width (0: no split)
  unsigned sub_delta; // sub-split width for vertices above the threshold (0: none)
  unsigned max_rounds;
  int prebuffer;      // queue level: the commit buffers the units of the next round's heavy vertices
  long long launch_budget;
  int4 *fcur;         // frontier of the current round: (vertex, distance when the round began,
                      // first edge, end edge)
  int *fnext;         // vertices whose distance dropped in the round, and heavy ones that wait
  unsigned *stamp;    // last round in which a vertex entered fnext
  int4 *units;        // (first edge, end edge, distance of the vertex, vertex)
  WsHeader *hdr;      // cursor: units; cursor2: |fnext|; aux[0]: |fcur|; nf_*: the split
  dpc_stats *stats;
};

size_t sssp_workspace_bytes(int n, int m, dpc_level level, const LaunchCfg &c);
// Points the frontier, stamp, far-pile and unit arrays of p (and p.hdr) into the workspace.
void sssp_carve(SsspParams &p, void *workspace, int n, int m, dpc_level level, const LaunchCfg &c);
size_t sssp_max_units(int n, int m, int threshold, int chunk);
// Launches the whole call on `s`; the flat level drives its rounds from the host.
cudaError_t sssp_launch(SsspParams &p, dpc_level level, cudaStream_t s, unsigned *rounds_out);
const void *sssp_parent_kernel(dpc_level level);
const void *sssp_child_kernel(dpc_level level);
// The queue level: every round in one cooperative grid.
const void *sssp_queue_kernel();
size_t sssp_queue_smem(int threads);
cudaError_t sssp_queue_launch(const SsspParams &p, int blocks, cudaStream_t s);

}  // namespace dpc

namespace dpc {

// ---------------------------------------------------------------- trees
enum TreeOp : int { kDescendants = 0, kHeight = 1 };

struct TreeParams {
  const int *coff;
  const int *cidx;
  int *out;           // desc (as uint32 bits) or height
  int n;
  int root;
  int op;             // TreeOp
  int level;
  int chunk;          // children per unit
  int chunk_shift;    // log2(chunk) when chunk is a power of two, else -1
  int child_blocks;   // KC_X grid for a recursive consolidated launch
  int child_threads;
  int max_units;
  long long launch_budget;
  int2 *units;        // (node, chunk index): every level's buffers, carved from one cursor;
                      // the queue level stores int4 units (node, first child, end child, -) there
  int *level_ends;    // queue level: level L's units are [level_ends[L], level_ends[L+1])
  int chain;          // queue level: chained postwork (trees below 2^24 nodes)
  int *par;           // chained postwork: parent of each internal node (root: -1)
  unsigned long long *link;  // chained postwork: pending reports (high 32 bits) and partial value (low)
  WsHeader *hdr;      // cursor: units handed out; queue level: done_blocks2 / round are its barrier
  dpc_stats *stats;
};

size_t tree_max_units(int n, int chunk);
size_t tree_workspace_bytes(int n, dpc_level level, const LaunchCfg &c);
cudaError_t tree_launch(TreeParams &p, dpc_level level, int root_blocks, cudaStream_t s, unsigned *levels_out);
const void *tree_visit_kernel(dpc_level level, int op);
// The queue level: every tree level, then every postwork level, in one cooperative grid.
constexpr int kTreeQueueMaxThreads = 512;  // block size bound of the queue kernel (registers)
const void *tree_queue_kernel(int op, bool chain);
size_t tree_units_bytes(int n, dpc_level level, int chunk);
// The queue level's postwork for trees of n nodes: chained (no level barriers) below 2^24 nodes.
inline bool tree_chained_postwork(int n) { return n < (1 << 24); }
cudaError_t tree_queue_launch(const TreeParams &p, int blocks, int threads, cudaStream_t s);

}  // namespace dpc

