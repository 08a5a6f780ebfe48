/*
 * dpc.h — consolidated dynamic-parallelism kernels for NVIDIA GB300 (sm_103a).
 *
 * C ABI of libdpc.so. The library implements the hot path of workload
 * consolidation for dynamic parallelism (Wu, Li & Becchi, "Compiler-Assisted
 * Workload Consolidation for Efficient Dynamic Parallelism on GPU", arXiv
 * 1606.08150): a parent thread that would launch its own child kernel for a
 * large or recursive piece of work instead appends the work to a warp-, block-
 * or grid-level buffer, and one consolidated child kernel per warp, block or
 * grid processes the whole buffer (Sec. IV.A-B). Seven applications of the
 * paper's evaluation are exported (Sec. V): single-source shortest paths, CSR
 * sparse matrix-vector product, tree descendants, tree heights, PageRank,
 * recursive BFS and graph colouring, each at the five levels of the paper
 * (basic-DP, flat, warp, block, grid) plus a persistent queue level; a batched
 * engine runs many SSSP and tree problems in one resident kernel.
 *
 * Conventions shared by every entry point
 *  - All array pointers are DEVICE pointers owned by the caller. The library
 *    allocates no device memory during a call: scratch space comes from the
 *    caller's workspace (the paper's pre-allocated pool, Sec. IV.E), sized by the
 *    matching *_workspace_size query. Workspace contents need no initialisation
 *    and are meaningless after the call.
 *  - Calls are asynchronous on the given stream (0 = legacy default stream),
 *    except the DPC_FLAT variants of dpc_sssp and of the tree calls, which read a
 *    round/level count back to the host once per round/level and therefore block
 *    the calling thread until the stream has finished the call. Inputs must stay
 *    unchanged and outputs untouched by others until the stream has completed the
 *    call; outputs are fully overwritten.
 *  - Errors the host can see (null pointers, negative sizes, out-of-range
 *    source/root, a too-small workspace, an unsupported level) are returned
 *    immediately and nothing is launched. Errors raised on the device (a child
 *    launch that failed after its inline fallback also failed, a tail launch that
 *    failed, a distance that does not fit below 0xFFFFFFFF) are recorded in the
 *    device status word: copied to stats->status when stats is given, and
 *    checked by a stream synchronisation before returning when the tuning flag
 *    DPC_FLAG_SYNC_CHECK is set.
 *  - Every call enqueues work only on `stream`; concurrent calls on different
 *    streams must use different workspaces.
 */
#ifndef DPC_H
#define DPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without pulling in the CUDA headers */
typedef struct CUstream_st *dpc_stream_t;

/* Consolidation granularity (Sec. IV.B) plus the two baselines of Sec. V. */
typedef enum dpc_level {
  DPC_BASIC_DP = 0, /* one child kernel per parent thread with large work (Fig. 1) */
  DPC_FLAT = 1,     /* no device launches: each thread does all of its own work */
  DPC_WARP = 2,     /* one consolidated child per warp with buffered work */
  DPC_BLOCK = 3,    /* one consolidated child per block with buffered work */
  DPC_GRID = 4,     /* one consolidated child per parent grid */
  DPC_QUEUE = 5     /* one resident (cooperative) grid and no device launches: the grid level's
                       phases (buffering, the consolidated child's loop, commits; for trees the
                       levels top-down, then the postwork levels bottom-up) separated by grid
                       barriers */
} dpc_level;

typedef enum dpc_status {
  DPC_OK = 0,
  DPC_ERR_INVALID_ARG = 1, /* null pointer, negative size, index out of range */
  DPC_ERR_WORKSPACE = 2,   /* workspace missing or smaller than the size query returned */
  DPC_ERR_CUDA = 3,        /* a host-side CUDA call failed (launch configuration, memset, copy) */
  DPC_ERR_DEVICE = 4,      /* a device-side launch failed and the work could not be completed */
  DPC_ERR_TIMEOUT = 5,     /* a bounded device-side wait (a grid barrier of the queue level or of the
                              engine) gave up after about two seconds; see dpc_wait_selftest */
  DPC_ERR_OVERFLOW = 6,    /* a shortest-path distance reached 0xFFFFFFFF */
  DPC_ERR_UNSUPPORTED = 7, /* level or configuration not supported by this call */
  DPC_ERR_DEPTH = 8        /* recursion deeper than the device's nesting limit */
} dpc_status;

/* tuning flags */
#define DPC_FLAG_SYNC_CHECK 0x1u /* synchronise the stream at the end and return the device status */
/* dpc_sssp at the warp and block levels: every consolidation buffer comes from
 * device-side malloc() (the device heap, cudaLimitMallocHeapSize) instead of the
 * workspace pool, the "default" allocator of Sec. IV.E that Fig. 5 compares with
 * the pre-allocated pool; the child grid's last block frees it. A malloc that
 * fails counts as a launch failure and the parent relaxes that group's vertices
 * itself. Other calls and levels ignore the flag. For the allocator study only:
 * the pool is faster. */
#define DPC_FLAG_DEVICE_MALLOC 0x2u

/*
 * Launch configuration and consolidation knobs; the clauses of the paper's
 * directive (Table I: threads, blocks, buffer) and its KC_X rule (Sec. IV.E)
 * become fields. A NULL tuning pointer or a zero field selects the default.
 */
typedef struct dpc_tuning {
  int32_t threshold;      /* items with more work than this go to a child (SSSP edges, SpMV nnz); default 32 */
  int32_t parent_blocks;  /* parent grid size; default: resident blocks per SM x SM count (persistent grid) */
  int32_t parent_threads; /* parent block size; default 256 */
  int32_t child_blocks;   /* consolidated child grid size; default: KC_X rule, capped by the buffered work */
  int32_t child_threads;  /* consolidated child block size; default 256 */
  int32_t chunk;          /* work per child unit: SpMV nnz (2048), PageRank in-edges (512), SSSP and colouring edges (256), BFS edges (256, at most), tree children (32; grid 16, queue 8) */
  int32_t kc;             /* X of KC_X; default 1 (grid), 16 (block), 32 (warp) */
  uint32_t flags;         /* DPC_FLAG_* */
  int32_t delta;          /* dpc_sssp: near-far split width (0: no split; see dpc_sssp) */
  int32_t sub_delta;      /* dpc_sssp: sub-split width for vertices above the threshold (0: none) */
} dpc_tuning;

/*
 * Device-resident call statistics (optional; pass NULL to skip counting). The
 * struct is zeroed at the start of each call and filled on the device; read it
 * after the stream has completed the call.
 */
typedef struct dpc_stats {
  uint64_t child_launches;  /* consolidated (or per-item) child grids launched from the device */
  uint64_t aux_launches;    /* device-side continuation grids (postwork, next round) */
  uint64_t buffered_items;  /* parent work items handed to a child */
  uint64_t inline_items;    /* parent work items processed by the parent thread itself */
  uint64_t relaxations;     /* SSSP: edges examined; trees: child edges visited */
  uint64_t launch_failures; /* device launches that failed (their work was done inline) */
  uint32_t rounds;          /* SSSP rounds, tree levels */
  uint32_t status;          /* dpc_status of the device side */
} dpc_stats;

/* Human-readable name of a status code (static string). */
const char *dpc_status_string(dpc_status s);

/*
 * Diagnostic of the bounded device-side waits (no counterpart in the paper).
 * Every grid barrier of the queue levels and of the batched engine spins on a
 * word that other blocks write, gives up after about two seconds and reports
 * DPC_ERR_TIMEOUT instead of hanging the GPU. This call runs the same wait, on
 * a word that nothing ever writes, for `limit_us` microseconds (1 to
 * 10,000,000) in one block on `stream`. It then writes status[0] =
 * DPC_ERR_TIMEOUT and status[1] = the microseconds actually waited.
 * `status` points to two uint32 in device memory. Returns
 * DPC_ERR_INVALID_ARG for a null status or a limit out of range.
 */
dpc_status dpc_wait_selftest(uint32_t limit_us, uint32_t *status, dpc_stream_t stream);

/*
 * Diagnostic (no counterpart in the paper): the rate of random 4-byte gathers
 * from an array held in L2, which bounds the SpMV kernels' gathers of x (one
 * 32-byte L2 sector per 4 useful bytes when the columns are uniform). A grid
 * of every resident block runs; each thread issues `batches` batches of 16
 * independent loads x[i] at pseudo-random i in [0, n) through L2 and adds them
 * into out[0] (so no load is dropped). n is a power of two from 32 to 2^26;
 * x and out are device pointers. *gathers (host) receives the loads issued.
 * Asynchronous on `stream`: time it with events there. Returns
 * DPC_ERR_INVALID_ARG for bad sizes or null pointers.
 */
dpc_status dpc_gather_rate(const float *x, int32_t n, int32_t batches, float *out, int64_t *gathers,
                           dpc_stream_t stream);

/* Version of this ABI (bumped on incompatible change). */
int32_t dpc_abi_version(void);

/*
 * Prepare `device` for device-side launches: makes it current and sets the
 * device runtime's pending-launch pool (cudaLimitDevRuntimePendingLaunchCount;
 * the fixed-size pool of Sec. III.B) to `pending_launch_limit` (0 selects the
 * library default of 1<<14). Call before the first dpc_* compute call on that
 * device; CUDA only accepts the limit before the device runtime first runs.
 * Every call keeps its optional device launches within the pool (refused
 * launches are done inline, or reported for the recursive applications), so
 * the pool size trades basic-DP's launches per call against launch latency,
 * which grows with the pool on GB300 (about 14 us per tail link at 2,048
 * entries, 21 us at 32,768, 31 us at 131,072 and 81-126 us at 262,144).
 * Returns DPC_ERR_CUDA if CUDA rejects the request.
 */
dpc_status dpc_device_init(int device, size_t pending_launch_limit);

/*
 * Whether the current device can read and write memory at `p`: device or
 * managed memory, or pinned host memory (cudaHostAlloc / cudaHostRegister)
 * mapped into the device's address space at the same address, as it is
 * under unified addressing. Writes 1 or 0 to *accessible (0 for a null
 * pointer and for host memory the CUDA runtime does not know). Reads only
 * the runtime's record of the allocation; nothing runs on the device.
 * Returns DPC_ERR_INVALID_ARG for a null `accessible`, DPC_ERR_CUDA if the
 * runtime cannot be queried.
 */
dpc_status dpc_memory_device_accessible(const void *p, int32_t *accessible);

/*
 * Single-source shortest paths (Sec. III.A, Fig. 1b; Sec. V). CSR graph with
 * n vertices and m directed edges: off[n+1] (int32, off[0]=0, off[n]=m),
 * col[m] (int32 in [0,n)), w[m] (uint32 weights). dist[n] receives the
 * shortest-path distance from `source` (uint32; unreachable = 0xFFFFFFFF).
 * Frontier rounds of relaxation: each frontier vertex with out-degree above
 * tuning.threshold hands its edge list to a child kernel at the given level.
 * Duplicate edges and self-loops are allowed.
 *
 * With tuning.delta > 0 the rounds use the near-far split of Davidson et al.
 * (IPDPS 2014): a vertex whose distance dropped joins the next frontier only
 * below the split distance S (a multiple of delta), else a far pile; when the
 * frontier is empty, S moves to the delta-bucket above the smallest far
 * distance still pending and the far vertices below it form the frontier.
 * With tuning.sub_delta > 0 a frontier vertex above the threshold is relaxed
 * only when its distance is below a sub-split s (a multiple of sub_delta,
 * advanced the same way); until then it waits in the frontier. Both cut the
 * edges relaxed more than once; distances are the same either way.
 * stats->rounds counts relaxation rounds; a run that would exceed 2^32 - 16
 * rounds (n + 1 without a split) ends with DPC_ERR_OVERFLOW.
 */
dpc_status dpc_sssp_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning, size_t *bytes);
dpc_status dpc_sssp(const int32_t *off, const int32_t *col, const uint32_t *w, int32_t n, int32_t m, int32_t source,
                    uint32_t *dist, dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                    dpc_stats *stats, dpc_stream_t stream);

/*
 * CSR sparse matrix-vector product y = A x in fp32 with fp32 accumulation
 * (Sec. V, SpMV; irregular loop of Sec. II.B). off[nrows+1], col[nnz] (int32 in
 * [0,ncols)), val[nnz] (float), x[ncols], y[nrows]. Rows with more than
 * tuning.threshold non-zeros go to a child kernel at the given level. Every
 * level sums each row in a fixed order, so results are bitwise reproducible.
 * x, y and the workspace are device memory. The matrix arrays (off, col,
 * val) may instead be pinned host memory that the device reads in place
 * (dpc_memory_device_accessible says 1): the kernels then read col and val
 * once per call over the host link, so a host-resident matrix needs no device
 * copy (nor device memory); y is bitwise the same. The host link bounds that
 * call, as it bounds copying the matrix over first.
 */
dpc_status dpc_spmv_csr_workspace_size(int32_t nrows, int32_t nnz, dpc_level level, const dpc_tuning *tuning,
                                       size_t *bytes);
dpc_status dpc_spmv_csr(const int32_t *off, const int32_t *col, const float *val, int32_t nrows, int32_t ncols,
                        int32_t nnz, const float *x, float *y, dpc_level level, const dpc_tuning *tuning,
                        void *workspace, size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream);

/*
 * y = A x with the kernels and units of dpc_spmv_csr, for callers that may not
 * allocate device memory: code whose device heap belongs to another memory
 * manager (a framework's caching allocator, an inference server's arena), a
 * service with a fixed memory budget that forbids allocation after start-up,
 * or a latency-critical path on which cudaMalloc/cudaFree would synchronise
 * the device. The paper has no counterpart; this entry point is an addition of
 * the library.
 *
 * Levels DPC_BASIC_DP to DPC_GRID are offered; DPC_QUEUE (a cooperative
 * launch) is not and returns DPC_ERR_INVALID_ARG. At the warp, block and grid
 * levels, and at flat, y is bitwise the y of dpc_spmv_csr. basic-DP computes
 * the long rows that its launch budget refuses inline, in another summation
 * order; the budget comes from the pending-launch pool in force, which this
 * call never sets, so call dpc_device_init first to get the pool (and the
 * bitwise agreement) of dpc_spmv_csr; otherwise y agrees within the SpMV
 * tolerance.
 *
 * Instead of a caller workspace it uses one scratch array of
 * DPC_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits. The caller still passes
 * all inputs and outputs (device pointers, as for dpc_spmv_csr). A problem
 * whose workspace (dpc_spmv_csr_workspace_size) exceeds the array is rejected
 * with DPC_ERR_WORKSPACE before anything is launched. The call allocates
 * nothing and never resizes the device runtime's launch pool.
 *
 * The first call on a device looks up the array's device address with that
 * device current and caches it; make that first call before any stream
 * capture. All calls share the one array and it keeps the previous call's
 * contents (each call clears what must start at zero): calls whose kernels
 * overlap on the GPU, for example on two streams, race and must be avoided.
 */
#define DPC_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
dpc_status dpc_spmv_csr_noalloc(const int32_t *off, const int32_t *col, const float *val, int32_t nrows,
                                int32_t ncols, int32_t nnz, const float *x, float *y, dpc_level level,
                                const dpc_tuning *tuning, dpc_stats *stats, dpc_stream_t stream);

/*
 * PageRank (Sec. V, the PR benchmark): `iterations` power iterations from the
 * uniform vector, in fp32, pulled over the in-edges of an n-vertex graph with
 * m edges given as in_off[n+1] (int32, in_off[0]=0, in_off[n]=m) and
 * in_src[m] (int32 sources in [0,n) of each vertex's in-edges), plus
 * outdeg[n] (int32 out-degree of every vertex, duplicates and self-loops
 * counted; it must match in_src). Each iteration computes
 *   rank'(v) = (1-d)/n + d * ( D/n + sum over in-edges (u,v) of rank(u)/outdeg(u) )
 * with d = damping in [0,1] and D the rank of the vertices whose out-degree is
 * 0 (spread uniformly, so the ranks keep summing to 1). rank[n] receives the
 * result. A vertex with more than tuning.threshold in-edges is large work for a
 * child kernel at the given level, one parent grid per iteration, as for SpMV
 * rows; stats->rounds = iterations. Every level sums each vertex in a fixed
 * order: results are bitwise reproducible, and the warp, block, grid and queue
 * levels agree bit for bit.
 */
dpc_status dpc_pagerank_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning,
                                       size_t *bytes);
dpc_status dpc_pagerank(const int32_t *in_off, const int32_t *in_src, const int32_t *outdeg, int32_t n, int32_t m,
                        float damping, int32_t iterations, float *rank, dpc_level level, const dpc_tuning *tuning,
                        void *workspace, size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream);

/*
 * Recursive breadth-first search (Sec. V, BFS-Rec): bfs_level[v] = fewest
 * edges on a path from `source` to v (uint32; unreachable = 0xFFFFFFFF) over
 * the CSR graph off[n+1], col[m] (int32; duplicates and self-loops allowed).
 * The traversal is the parallel recursion of Fig. 1(c) on a graph: a visit of
 * v at depth d relaxes v's out-edges with atomicMin and visits recursively
 * every neighbour whose level dropped and that has out-edges; at the warp,
 * block and grid levels those visits are consolidated into one child per
 * buffer (tuning.chunk out-edges per unit, at most 256, default 256;
 * tuning.threshold is not used: every vertex with out-edges is recursive
 * work). The flat level is host-driven level-synchronous BFS; the queue level
 * runs the grid level's generations in one cooperative grid. Returns
 * DPC_ERR_INVALID_ARG for a chunk above 256. A recursive level whose launches
 * exceed the call's launch budget, or whose unit buffer overflows, reports
 * DPC_ERR_DEVICE or DPC_ERR_OVERFLOW in the device status.
 */
dpc_status dpc_bfs_rec_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning,
                                      size_t *bytes);
dpc_status dpc_bfs_rec(const int32_t *off, const int32_t *col, int32_t n, int32_t m, int32_t source,
                       uint32_t *bfs_level, dpc_level level, const dpc_tuning *tuning, void *workspace,
                       size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream);

/*
 * Graph colouring (Sec. V, the GC benchmark) by round sweep (the independent-set
 * rounds of Jones-Plassmann, the colour being the round) over an
 * undirected graph given as a symmetric CSR, off[n+1] and col[m] (int32; both
 * directions of every edge present; self-loops ignored, duplicates allowed),
 * with the caller's vertex priorities priority[n] (uint32; the random draws of
 * the method, passed in; equal priorities are ordered by vertex id, the larger
 * id first). In round r = 1, 2, ... every vertex still uncoloured when the
 * round began takes colour r unless a neighbour also uncoloured at the round's
 * start has a higher (priority, id). color[n] receives colours 1..rounds
 * (int32); stats->rounds = the number of colours. A vertex with more than
 * tuning.threshold neighbours hands its neighbour scan to a child kernel at the
 * given level (units of tuning.chunk neighbours, default 256); the round's
 * commit colours those vertices after the children (a CDP2 tail launch).
 * The result does not depend on the level or on scheduling.
 */
dpc_status dpc_graph_coloring_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning,
                                             size_t *bytes);
dpc_status dpc_graph_coloring(const int32_t *off, const int32_t *col, int32_t n, int32_t m, const uint32_t *priority,
                              int32_t *color, dpc_level level, const dpc_tuning *tuning, void *workspace,
                              size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream);

/*
 * Tree descendants and tree heights (Sec. III.A, Fig. 1c; Sec. V): parallel
 * recursion over a rooted tree given as child lists, coff[n+1] (int32,
 * coff[0]=0, coff[n]=n-1) and cidx[n-1] (int32 child ids). The child lists must
 * describe a tree rooted at `root` that contains all n nodes.
 *   dpc_tree_descendants: desc[v] = number of proper descendants (uint32).
 *   dpc_tree_height:      height[v] = 0 for a leaf, else 1 + max child height (int32).
 * A node whose children are not all leaves has its non-leaf children handed to
 * a recursive child kernel at the given level; the postwork that combines the
 * children's values runs after the recursive work (a CDP2 tail launch). The
 * device's nesting limit bounds the tree depth for the recursive levels; deeper
 * trees end with DPC_ERR_DEPTH in the device status. The flat level (host-
 * driven level passes) and the queue level (the levels top-down, then the
 * postwork levels bottom-up, in one cooperative grid) have no depth limit.
 * Child lists are split into units of tuning.chunk children (default 32 at the
 * warp and block levels, 16 at the grid level, 8 at the queue level).
 */
dpc_status dpc_tree_workspace_size(int32_t n, dpc_level level, const dpc_tuning *tuning, size_t *bytes);
dpc_status dpc_tree_descendants(const int32_t *coff, const int32_t *cidx, int32_t n, int32_t root, uint32_t *desc,
                                dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                                dpc_stats *stats, dpc_stream_t stream);
dpc_status dpc_tree_height(const int32_t *coff, const int32_t *cidx, int32_t n, int32_t root, int32_t *height,
                           dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                           dpc_stats *stats, dpc_stream_t stream);

/*
 * Persistent batched engine (the next step after consolidation: batching many
 * problems). Many SSSP and tree problems of uneven sizes run in one resident
 * cooperative kernel whose device work queue replaces child launches: a large
 * frontier vertex becomes queue tasks instead of a child grid, and a problem's
 * next phase (commit, next round, next tree level, postwork) is queued by the
 * warp that finishes the current phase's last task. Waves of tasks are
 * separated by a bounded grid barrier. The paper names persistent threads as
 * related work (Sec. VI); it has no such engine itself.
 *
 * Problems occupy slots; every slot has scratch for a problem of up to max_n
 * vertices / nodes and max_m edges. All pointers in dpc_job are device pointers
 * owned by the caller and must stay valid until the problem's slot reports 2.
 */
typedef enum dpc_job_kind {
  DPC_JOB_SSSP = 0,             /* dist (uint32) from source; off/col/w CSR */
  DPC_JOB_TREE_DESCENDANTS = 1, /* desc (uint32) of every node; off/col = child lists, source = root */
  DPC_JOB_TREE_HEIGHT = 2       /* height (int32) of every node */
} dpc_job_kind;

typedef struct dpc_job {
  int32_t kind;        /* dpc_job_kind */
  int32_t n;           /* vertices / nodes */
  int32_t m;           /* edges (SSSP); n-1 for trees */
  int32_t source;      /* SSSP source / tree root */
  const int32_t *off;  /* n+1 offsets */
  const int32_t *col;  /* m targets / child ids */
  const uint32_t *w;   /* m weights (SSSP only) */
  void *out;           /* n results */
} dpc_job;

/* Workspace for an engine of `slots` slots of up to max_n vertices and max_m edges each. */
dpc_status dpc_engine_workspace_size(int32_t slots, int32_t max_n, int32_t max_m, const dpc_tuning *tuning,
                                     size_t *bytes);

/*
 * Reset an engine: every slot free. slot_state (`slots` int32, device memory or
 * pinned host memory, which the engine uses through its device address) receives
 * 1 when a problem is admitted into a slot and 2 when its results are complete;
 * the engine never writes 0 after the reset, so the caller keeps the slot
 * bookkeeping (a slot whose state is 2 may be reused).
 */
dpc_status dpc_engine_init(void *workspace, size_t workspace_bytes, int32_t slots, int32_t max_n, int32_t max_m,
                           const dpc_tuning *tuning, int32_t *slot_state, dpc_stream_t stream);

/*
 * One engine step: admit *new_count problems (device int32; new_jobs and
 * new_slots are device arrays of at least that many entries; slots must be
 * free) and run at most max_waves waves of tasks, then return with the queue
 * intact; the next step continues where this one stopped. With new_count NULL
 * nothing is admitted. All arguments are fixed device pointers or scalars, so a
 * step can be captured in a CUDA graph and replayed after new admissions are
 * copied into the same arrays. The engine grid is every block that can be
 * resident (a cooperative launch), or tuning->parent_blocks when that is
 * smaller; tuning->threshold (default 32) and tuning->chunk (default 512
 * edges) set the SSSP split of large frontier vertices into EDGES tasks.
 * Problems must fit the slot size (n <= max_n,
 * m <= max_m). The engine checks every admitted descriptor on the device: one
 * that cannot be valid (unknown kind, a size beyond the slot, a missing array,
 * a source or root out of range, a slot out of range) is not run, its slot
 * reports 2 and the status says DPC_ERR_INVALID_ARG; the contents of the
 * arrays (offsets, indices) are not checked. Device-side errors (a task list
 * overflow, a barrier that timed out) go to stats->status.
 */
dpc_status dpc_engine_step(void *workspace, size_t workspace_bytes, int32_t slots, int32_t max_n, int32_t max_m,
                           const dpc_tuning *tuning, const dpc_job *new_jobs, const int32_t *new_slots,
                           const int32_t *new_count, int32_t max_waves, int32_t *slot_state, dpc_stats *stats,
                           dpc_stream_t stream);

/*
 * Resident form of the engine: the kernel stays on the GPU and admits new
 * problems while it runs, from a mailbox in the caller's pinned host memory,
 * so an arrival joins the running waves with no kernel boundary in between
 * (serving with continuous batching, arrivals folded into the running
 * kernel). Like the engine itself, this has no counterpart in the paper.
 *
 * The mailbox is a ring of DPC_MAILBOX_CAP job descriptors with their slots.
 * One host thread posts jobs (dpc_mailbox_post: the descriptor, then a
 * release store of the posted count); the kernel reads the count at each
 * wave barrier and admits the new jobs during the next wave (at most one per
 * warp of its grid per wave), advancing `taken`; the mailbox holds both
 * counts, so a kernel continues from whatever its mailbox says was taken. A
 * slot may be posted to only while it is free: never used since
 * dpc_engine_init, or reported 2 and set back to 0 by the host before the post.
 */
#define DPC_MAILBOX_CAP 1024

typedef struct dpc_mailbox {
  uint64_t posted;                  /* host: jobs posted so far */
  uint32_t stop;                    /* host: 1 = return once idle */
  uint32_t reserved0;
  uint64_t taken;                   /* kernel: jobs admitted so far */
  uint64_t reserved1[5];
  dpc_job jobs[DPC_MAILBOX_CAP];    /* job i in jobs[i % DPC_MAILBOX_CAP] */
  int32_t slots[DPC_MAILBOX_CAP];   /* and its slot */
} dpc_mailbox;

/* Empty mailbox (host memory; no GPU work). */
dpc_status dpc_mailbox_init(dpc_mailbox *mailbox);

/* Post one job into `slot` (host): DPC_ERR_OVERFLOW when DPC_MAILBOX_CAP jobs
 * are posted and not yet taken. Single producer: one host thread posts. */
dpc_status dpc_mailbox_post(dpc_mailbox *mailbox, const dpc_job *job, int32_t slot);

/* Ask a resident kernel to return once it is idle (host). */
dpc_status dpc_mailbox_stop(dpc_mailbox *mailbox);

/* Jobs the kernel has admitted so far (host, acquire load). */
dpc_status dpc_mailbox_taken(const dpc_mailbox *mailbox, uint64_t *taken);

/*
 * Launch the engine in resident form on `stream` (returns at once). mailbox
 * and slot_state (`slots` int32) must be pinned host memory that the device
 * can address (cudaHostAlloc, or pinned memory under unified addressing;
 * anything else is DPC_ERR_INVALID_ARG); slot_state receives 1 when a posted
 * job is admitted and 2, after a system-scope fence, when its results are
 * complete, so the host can poll it while the kernel runs. Results are in
 * device memory: read them on another stream (the kernel's stream is busy
 * until it returns). The kernel returns when it is idle (nothing queued,
 * active or posted) and either the mailbox's stop flag is set or `limit_us`
 * have passed since its start; or after 4 x limit_us even when busy; or on a
 * device error (stats->status). It returns with its queue intact:
 * dpc_engine_serve (or dpc_engine_step) continues the work. limit_us in
 * [1, 10,000,000]. Workspace, slots, sizes and tuning as for dpc_engine_step,
 * after dpc_engine_init with the same slot_state array.
 */
dpc_status dpc_engine_serve(void *workspace, size_t workspace_bytes, int32_t slots, int32_t max_n, int32_t max_m,
                            const dpc_tuning *tuning, dpc_mailbox *mailbox, uint32_t limit_us, int32_t *slot_state,
                            dpc_stats *stats, dpc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DPC_H */
