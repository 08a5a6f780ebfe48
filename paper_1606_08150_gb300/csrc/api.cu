// C-ABI layer of libdpc.so: argument validation, workspace sizing, launch
// configuration (the KC_X rule of Sec. IV.E) and dispatch to the kernels.
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "dpc_internal.h"

namespace dpc {
namespace {

constexpr int kMaxDevices = 64;
// Pending-launch pool set on first use. CDP2 launch latency grows with the
// pool (a tail link between trivial grids: 14 us at 2,048 entries, 21 us at
// 32,768, 31 us at 131,072, 81-126 us at 262,144 on GB300), so the default is
// the smallest pool that still holds the consolidated levels' launches (a
// warp-level round of a 1,024-thread-block parent grid launches at most one
// child per warp); basic-DP callers that want one launch per large item ask
// for a larger pool through dpc_device_init.
constexpr size_t kDefaultPendingLaunches = size_t(1) << 14;
constexpr int kMaxIndex = INT_MAX - (1 << 16);  // headroom for index arithmetic in the kernels
constexpr int kSsspChunk = 256;                 // edges per SSSP child unit (8 per lane of a warp)

struct OccEntry {
  const void *fn;
  int threads;
  int blocks_per_sm;
};

struct DeviceInfo {
  bool ready = false;
  int sms = 0;
  size_t l2 = 0;       // L2 cache bytes
  size_t pool = 2048;  // device runtime pending-launch pool in force
  std::vector<OccEntry> occ;
};

std::mutex g_mu;
DeviceInfo g_dev[kMaxDevices];

dpc_status init_locked(int device, size_t pending) {
  if (device < 0 || device >= kMaxDevices) return DPC_ERR_INVALID_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return DPC_ERR_CUDA;
  if (device != prev && cudaSetDevice(device) != cudaSuccess) return DPC_ERR_CUDA;
  DeviceInfo &d = g_dev[device];
  dpc_status st = DPC_OK;
  if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) st = DPC_ERR_CUDA;
  int l2 = 0;
  if (st == DPC_OK && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess) st = DPC_ERR_CUDA;
  d.l2 = l2 > 0 ? (size_t)l2 : 0;
  if (st == DPC_OK) {
    size_t cur = 0;
    cudaDeviceGetLimit(&cur, cudaLimitDevRuntimePendingLaunchCount);
    if (cur != pending && cudaDeviceSetLimit(cudaLimitDevRuntimePendingLaunchCount, pending) != cudaSuccess) {
      cudaGetLastError();
      st = DPC_ERR_CUDA;
    }
    // the runtime may clamp the request: remember what is really in force
    if (cudaDeviceGetLimit(&cur, cudaLimitDevRuntimePendingLaunchCount) == cudaSuccess) d.pool = cur;
  }
  if (st == DPC_OK) d.ready = true;
  if (device != prev) cudaSetDevice(prev);
  return st;
}

// Device of the calling thread, initialised on first use.
dpc_status current_device(int *dev) {
  if (cudaGetDevice(dev) != cudaSuccess) return DPC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (*dev < 0 || *dev >= kMaxDevices) return DPC_ERR_CUDA;
  if (!g_dev[*dev].ready) {
    dpc_status st = init_locked(*dev, kDefaultPendingLaunches);
    if (st != DPC_OK) {
      // the pool limit could not be changed (device runtime already running):
      // keep going with whatever limit is in force
      if (cudaDeviceGetAttribute(&g_dev[*dev].sms, cudaDevAttrMultiProcessorCount, *dev) != cudaSuccess)
        return DPC_ERR_CUDA;
      int l2 = 0;
      if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, *dev) != cudaSuccess) return DPC_ERR_CUDA;
      g_dev[*dev].l2 = l2 > 0 ? (size_t)l2 : 0;
      size_t cur = 0;
      if (cudaDeviceGetLimit(&cur, cudaLimitDevRuntimePendingLaunchCount) == cudaSuccess) g_dev[*dev].pool = cur;
      g_dev[*dev].ready = true;
    }
  }
  return DPC_OK;
}

size_t l2_bytes(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_dev[dev].l2;
}

int blocks_per_sm(int dev, const void *fn, int threads) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceInfo &d = g_dev[dev];
  for (const OccEntry &e : d.occ)
    if (e.fn == fn && e.threads == threads) return e.blocks_per_sm;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  if (nb < 1) nb = 1;
  d.occ.push_back({fn, threads, nb});
  return nb;
}

// Optional device launches one call may issue: the pending-launch pool less a
// reserve for the mandatory continuation (tail) launches.
long long launch_budget(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  long long pool = (long long)g_dev[dev].pool;
  long long reserve = pool / 8 > 1024 ? pool / 8 : 1024;
  return pool > reserve ? pool - reserve : 0;
}

int sm_count(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_dev[dev].sms > 0 ? g_dev[dev].sms : 1;
}

bool valid_level(dpc_level l) { return l >= DPC_BASIC_DP && l <= DPC_QUEUE; }

bool valid_threads(int t) { return t >= 32 && t <= 1024 && t % 32 == 0; }

int default_kc(dpc_level l) {
  switch (l) {
    case DPC_GRID: return 1;
    case DPC_BLOCK: return 16;
    case DPC_WARP: return 32;
    default: return 1;
  }
}

// Resolve the tuning fields that do not need the device.
dpc_status resolve_static(const dpc_tuning *t, int def_chunk, LaunchCfg *c) {
  dpc_tuning z;
  std::memset(&z, 0, sizeof(z));
  if (!t) t = &z;
  c->threshold = t->threshold > 0 ? t->threshold : (t->threshold < 0 ? 0 : 32);
  c->parent_threads = t->parent_threads ? t->parent_threads : 256;
  c->child_threads = t->child_threads ? t->child_threads : 256;
  c->chunk = t->chunk ? t->chunk : def_chunk;
  c->flags = t->flags;
  c->parent_blocks = t->parent_blocks;
  c->child_blocks = t->child_blocks;
  if (!valid_threads(c->parent_threads) || !valid_threads(c->child_threads)) return DPC_ERR_INVALID_ARG;
  if (c->chunk < 1 || c->chunk > (1 << 24) || t->parent_blocks < 0 || t->child_blocks < 0 || t->kc < 0)
    return DPC_ERR_INVALID_ARG;
  if (t->delta < 0 || t->sub_delta < 0) return DPC_ERR_INVALID_ARG;
  c->delta = (unsigned)t->delta;
  c->sub_delta = (unsigned)t->sub_delta;
  return DPC_OK;
}

// Grid sizes: parent = resident blocks (persistent grid) capped by the items;
// consolidated child = KC_X: resident blocks / X (Sec. IV.E).
void resolve_device(int dev, const dpc_tuning *t, dpc_level level, const void *parent_fn, const void *child_fn,
                    long long items, LaunchCfg *c) {
  const int sms = sm_count(dev);
  if (c->parent_blocks <= 0) {
    long long full = (long long)blocks_per_sm(dev, parent_fn, c->parent_threads) * sms;
    long long need = (items + c->parent_threads - 1) / c->parent_threads;
    if (need < 1) need = 1;
    c->parent_blocks = (int)(need < full ? need : full);
  }
  if (c->child_blocks <= 0 && child_fn) {
    const int kc = (t && t->kc > 0) ? t->kc : default_kc(level);
    long long full = (long long)blocks_per_sm(dev, child_fn, c->child_threads) * sms;
    long long b = full / kc;
    c->child_blocks = (int)(b > 0 ? b : 1);
  }
  if (c->child_blocks <= 0) c->child_blocks = 1;
}

dpc_status finish_call(cudaStream_t s, const LaunchCfg &c, WsHeader *hdr) {
  if (cudaGetLastError() != cudaSuccess) return DPC_ERR_CUDA;
  if (c.flags & DPC_FLAG_SYNC_CHECK) {
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    unsigned st = 0;
    if (cudaMemcpy(&st, &hdr->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return DPC_ERR_CUDA;
    return (dpc_status)st;
  }
  return DPC_OK;
}

dpc_status begin_call(void *ws, dpc_stats *stats, cudaStream_t s) {
  if (cudaMemsetAsync(ws, 0, kHeaderBytes, s) != cudaSuccess) return DPC_ERR_CUDA;
  if (stats && cudaMemsetAsync(stats, 0, sizeof(dpc_stats), s) != cudaSuccess) return DPC_ERR_CUDA;
  return DPC_OK;
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" {

const char *dpc_status_string(dpc_status s) {
  switch (s) {
    case DPC_OK: return "DPC_OK";
    case DPC_ERR_INVALID_ARG: return "DPC_ERR_INVALID_ARG: invalid argument";
    case DPC_ERR_WORKSPACE: return "DPC_ERR_WORKSPACE: workspace missing or too small";
    case DPC_ERR_CUDA: return "DPC_ERR_CUDA: a host-side CUDA call failed";
    case DPC_ERR_DEVICE: return "DPC_ERR_DEVICE: a device-side launch failed";
    case DPC_ERR_TIMEOUT: return "DPC_ERR_TIMEOUT: a bounded device-side wait ran out";
    case DPC_ERR_OVERFLOW: return "DPC_ERR_OVERFLOW: value or buffer overflow";
    case DPC_ERR_UNSUPPORTED: return "DPC_ERR_UNSUPPORTED: unsupported level or configuration";
    case DPC_ERR_DEPTH: return "DPC_ERR_DEPTH: recursion deeper than the device nesting limit";
  }
  return "unknown dpc_status";
}

int32_t dpc_abi_version(void) { return 2; }

dpc_status dpc_device_init(int device, size_t pending_launch_limit) {
  std::lock_guard<std::mutex> lk(g_mu);
  return init_locked(device, pending_launch_limit ? pending_launch_limit : kDefaultPendingLaunches);
}

dpc_status dpc_memory_device_accessible(const void *p, int32_t *accessible) {
  if (!accessible) return DPC_ERR_INVALID_ARG;
  *accessible = 0;
  if (!p) return DPC_OK;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
    *accessible = 1;
  else if (a.type == cudaMemoryTypeHost)  // pinned: mapped at the same address under unified addressing
    *accessible = a.devicePointer == p ? 1 : 0;
  return DPC_OK;
}

// ------------------------------------------------------------------ SpMV

dpc_status dpc_spmv_csr_workspace_size(int32_t nrows, int32_t nnz, dpc_level level, const dpc_tuning *tuning,
                                       size_t *bytes) {
  if (!bytes || nrows < 0 || nnz < 0 || nnz > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, 2048, &c);
  if (st != DPC_OK) return st;
  *bytes = spmv_workspace_bytes(nrows, nnz, level, c);
  return DPC_OK;
}

dpc_status dpc_spmv_csr(const int32_t *off, const int32_t *col, const float *val, int32_t nrows, int32_t ncols,
                        int32_t nnz, const float *x, float *y, dpc_level level, const dpc_tuning *tuning,
                        void *workspace, size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  if (nrows > 0 && (!off || !y)) return DPC_ERR_INVALID_ARG;
  if (nnz > 0 && (!col || !val || !x || ncols == 0)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, 2048, &c);
  if (st != DPC_OK) return st;
  // the queue level's grid also runs the child's loop: 512-thread blocks measured best
  if (level == DPC_QUEUE && !(tuning && tuning->parent_threads)) c.parent_threads = 512;
  if (!workspace || workspace_bytes < spmv_workspace_bytes(nrows, nnz, level, c)) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = current_device(&dev)) != DPC_OK) return st;
  if ((st = begin_call(workspace, stats, s)) != DPC_OK) return st;
  if (nrows == 0) return finish_call(s, c, reinterpret_cast<WsHeader *>(workspace));
  resolve_device(dev, tuning, level, spmv_parent_kernel(level), spmv_child_kernel(level), nrows, &c);
  if (level == DPC_QUEUE) {
    // a cooperative grid must be co-resident: at most the resident blocks; by
    // default all of them, since the whole grid works through the buffer
    const int full = blocks_per_sm(dev, spmv_parent_kernel(level), c.parent_threads) * sm_count(dev);
    c.parent_blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks
                                                                                              : full;
  }

  SpmvParams p;
  std::memset(&p, 0, sizeof(p));
  p.off = off;
  p.col = col;
  p.val = val;
  p.x = x;
  p.y = y;
  p.nrows = nrows;
  p.ncols = ncols;
  p.nnz = nnz;
  p.threshold = c.threshold;
  p.chunk = c.chunk;
  p.child_blocks = c.child_blocks;
  p.child_threads = c.child_threads;
  p.hdr = reinterpret_cast<WsHeader *>(workspace);
  p.stats = stats;
  p.launch_budget = launch_budget(dev);
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE) {
    const size_t mu = spmv_max_units(nrows, nnz, c.threshold, c.chunk);
    char *b = static_cast<char *>(workspace) + kHeaderBytes;
    p.units = reinterpret_cast<int4 *>(b);
    b += align_up(mu * sizeof(int4), 256);
    p.partial = reinterpret_cast<float *>(b);
    b += align_up(mu * sizeof(float), 256);
    p.ucount = reinterpret_cast<unsigned *>(b);
    p.max_units = (int)(mu > (size_t)INT_MAX ? INT_MAX : mu);
  }
  if (spmv_launch(p, level, c, s) != cudaSuccess) return DPC_ERR_CUDA;
  return finish_call(s, c, p.hdr);
}

// ------------------------------------------------------------------ PageRank

namespace {
// Workspace: the gather's (SpMV layout over n rows and m entries), then the
// contributions, the second rank buffer, the prep partials and the teleport term.
struct RankLayout {
  size_t gather, contrib, tmp, partials, beta, total;
};

dpc_status rank_layout(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning, LaunchCfg *c,
                       RankLayout *L) {
  // in-degrees are mostly moderate: 512-entry units balance better than SpMV's 2048
  dpc_status st = resolve_static(tuning, 512, c);
  if (st != DPC_OK) return st;
  L->gather = 0;
  L->contrib = align_up(spmv_workspace_bytes(n, m, level, *c), 256);
  L->tmp = L->contrib + align_up((size_t)n * sizeof(float), 256);
  L->partials = L->tmp + align_up((size_t)n * sizeof(float), 256);
  L->beta = L->partials + align_up(((size_t)n + 1023) / 1024 * sizeof(float), 256);  // chunk sums
  L->total = L->beta + align_up(kRankPrepBlocks * sizeof(float), 256);  // one teleport term per queue block
  return DPC_OK;
}
}  // namespace

dpc_status dpc_pagerank_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning,
                                       size_t *bytes) {
  if (!bytes || n < 1 || n > kMaxIndex || m < 0 || m > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  RankLayout L;
  dpc_status st = rank_layout(n, m, level, tuning, &c, &L);
  if (st != DPC_OK) return st;
  *bytes = L.total;
  return DPC_OK;
}

dpc_status dpc_pagerank(const int32_t *in_off, const int32_t *in_src, const int32_t *outdeg, int32_t n, int32_t m,
                        float damping, int32_t iterations, float *rank, dpc_level level, const dpc_tuning *tuning,
                        void *workspace, size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream) {
  if (n < 1 || n > kMaxIndex || m < 0 || m > kMaxIndex || iterations < 0 || !valid_level(level))
    return DPC_ERR_INVALID_ARG;
  if (!(damping >= 0.f && damping <= 1.f)) return DPC_ERR_INVALID_ARG;  // also rejects NaN
  if (!in_off || !outdeg || !rank || (m > 0 && !in_src)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  RankLayout L;
  dpc_status st = rank_layout(n, m, level, tuning, &c, &L);
  if (st != DPC_OK) return st;
  if (!workspace || workspace_bytes < L.total) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = current_device(&dev)) != DPC_OK) return st;
  if ((st = begin_call(workspace, stats, s)) != DPC_OK) return st;
  resolve_device(dev, tuning, level, spmv_parent_kernel(level, kModeRank), spmv_child_kernel(level, kModeRank), n,
                 &c);
  if (level == DPC_QUEUE) {
    // one cooperative grid for every iteration: co-resident, and at most one partial sum slot per block
    int full = blocks_per_sm(dev, rank_queue_kernel_ptr(), c.parent_threads) * sm_count(dev);
    if (full > kRankPrepBlocks) full = kRankPrepBlocks;
    c.parent_blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks
                                                                                              : full;
  }
  char *ws = static_cast<char *>(workspace);
  SpmvParams p;
  std::memset(&p, 0, sizeof(p));
  p.off = in_off;
  p.col = in_src;
  p.val = nullptr;
  p.x = reinterpret_cast<float *>(ws + L.contrib);
  p.nrows = n;
  p.ncols = n;
  p.nnz = m;
  p.threshold = c.threshold;
  p.chunk = c.chunk;
  p.child_blocks = c.child_blocks;
  p.child_threads = c.child_threads;
  p.alpha = damping;
  p.beta = reinterpret_cast<float *>(ws + L.beta);
  p.hdr = reinterpret_cast<WsHeader *>(ws + L.gather);
  p.stats = stats;
  p.launch_budget = launch_budget(dev);
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE) {
    const size_t mu = spmv_max_units(n, m, c.threshold, c.chunk);
    char *b = ws + L.gather + kHeaderBytes;
    p.units = reinterpret_cast<int4 *>(b);
    b += align_up(mu * sizeof(int4), 256);
    p.partial = reinterpret_cast<float *>(b);
    b += align_up(mu * sizeof(float), 256);
    p.ucount = reinterpret_cast<unsigned *>(b);
    p.max_units = (int)(mu > (size_t)INT_MAX ? INT_MAX : mu);
  }
  float *tmp = reinterpret_cast<float *>(ws + L.tmp);
  if (level == DPC_QUEUE) {
    RankQueueArgs a;
    a.p = p;
    a.outdeg = outdeg;
    a.rank = rank;
    a.tmp = tmp;
    a.contrib = reinterpret_cast<float *>(ws + L.contrib);
    a.partials = reinterpret_cast<float *>(ws + L.partials);
    a.betas = reinterpret_cast<float *>(ws + L.beta);
    a.damping = damping;
    a.iterations = iterations;
    if (rank_queue_launch(a, c.parent_blocks, c.parent_threads, s) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    return finish_call(s, c, p.hdr);
  }
  // rank_t lives in the caller's array when iterations - t is even, so that
  // the last iteration writes it
  auto buf = [&](int t) { return ((iterations - t) % 2 == 0) ? rank : tmp; };
  if (rank_init(buf(0), n, s) != cudaSuccess) return DPC_ERR_CUDA;
  RankPrepParams q;
  q.outdeg = outdeg;
  q.n = n;
  q.damping = damping;
  q.contrib = reinterpret_cast<float *>(ws + L.contrib);
  q.partials = reinterpret_cast<float *>(ws + L.partials);
  q.beta = reinterpret_cast<float *>(ws + L.beta);
  q.hdr = p.hdr;
  q.stats = stats;
  for (int t = 0; t < iterations; ++t) {
    q.rank_in = buf(t);
    q.iteration = t;
    if (rank_prep(q, s) != cudaSuccess) return DPC_ERR_CUDA;
    p.y = buf(t + 1);
    if (spmv_launch(p, level, c, s, kModeRank) != cudaSuccess) return DPC_ERR_CUDA;
  }
  return finish_call(s, c, p.hdr);
}

// ------------------------------------------------------------------ graph colouring

dpc_status dpc_graph_coloring_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning,
                                             size_t *bytes) {
  if (!bytes || n < 1 || m < 0 || m > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, kSsspChunk, &c);
  if (st != DPC_OK) return st;
  *bytes = gc_workspace_bytes(n, m, level, c);
  return DPC_OK;
}

dpc_status dpc_graph_coloring(const int32_t *off, const int32_t *col, int32_t n, int32_t m, const uint32_t *priority,
                              int32_t *color, dpc_level level, const dpc_tuning *tuning, void *workspace,
                              size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream) {
  if (n < 1 || m < 0 || m > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  if (!off || !priority || !color || (m > 0 && !col)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, kSsspChunk, &c);
  if (st != DPC_OK) return st;
  if (!workspace || workspace_bytes < gc_workspace_bytes(n, m, level, c)) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = current_device(&dev)) != DPC_OK) return st;
  if ((st = begin_call(workspace, stats, s)) != DPC_OK) return st;
  resolve_device(dev, tuning, level, gc_parent_kernel(level), gc_child_kernel(level), n, &c);
  int queue_blocks = 0;
  if (level == DPC_QUEUE) {
    const int full = blocks_per_sm(dev, gc_parent_kernel(level), c.parent_threads) * sm_count(dev);
    queue_blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks : full;
  }
  GcParams p;
  std::memset(&p, 0, sizeof(p));
  p.off = off;
  p.col = col;
  p.prio = priority;
  p.color = color;
  p.n = n;
  p.threshold = c.threshold;
  p.chunk = c.chunk;
  p.level = level;
  p.parent_blocks = c.parent_blocks;
  p.parent_threads = c.parent_threads;
  p.commit_blocks = c.parent_blocks;
  p.child_blocks = c.child_blocks;
  p.child_threads = c.child_threads;
  p.launch_budget = launch_budget(dev);
  char *b = static_cast<char *>(workspace);
  p.hdr = reinterpret_cast<WsHeader *>(b);
  b += kHeaderBytes;
  const size_t nb = align_up((size_t)n * sizeof(int), 256);
  p.list[0] = reinterpret_cast<int *>(b);
  p.list[1] = reinterpret_cast<int *>(b + nb);
  p.heavy = reinterpret_cast<int *>(b + 2 * nb);
  p.blocked = reinterpret_cast<unsigned *>(b + 3 * nb);
  b += 3 * nb + align_up((size_t)n * sizeof(unsigned), 256);
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID || level == DPC_QUEUE) {
    const size_t mu = gc_max_units(n, m, c.threshold, c.chunk);
    p.units = reinterpret_cast<int2 *>(b);
    p.max_units = (int)(mu > (size_t)INT_MAX ? INT_MAX : mu);
  }
  p.stats = stats;
  if (gc_launch(p, level, queue_blocks, s) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return finish_call(s, c, p.hdr);
}

// ------------------------------------------------------------------ recursive BFS

namespace {
dpc_status bfs_cfg(const dpc_tuning *tuning, LaunchCfg *c) {
  dpc_status st = resolve_static(tuning, kBfsMaxChunk, c);
  if (st != DPC_OK) return st;
  return c->chunk <= kBfsMaxChunk ? DPC_OK : DPC_ERR_INVALID_ARG;
}
}  // namespace

dpc_status dpc_bfs_rec_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning,
                                      size_t *bytes) {
  if (!bytes || n < 1 || m < 0 || m > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = bfs_cfg(tuning, &c);
  if (st != DPC_OK) return st;
  *bytes = bfs_workspace_bytes(n, m, level, c.chunk);
  return DPC_OK;
}

dpc_status dpc_bfs_rec(const int32_t *off, const int32_t *col, int32_t n, int32_t m, int32_t source,
                       uint32_t *bfs_level, dpc_level level, const dpc_tuning *tuning, void *workspace,
                       size_t workspace_bytes, dpc_stats *stats, dpc_stream_t stream) {
  if (n < 1 || m < 0 || m > kMaxIndex || source < 0 || source >= n || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  if (!off || !bfs_level || (m > 0 && !col)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = bfs_cfg(tuning, &c);
  if (st != DPC_OK) return st;
  if (!workspace || workspace_bytes < bfs_workspace_bytes(n, m, level, c.chunk)) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = current_device(&dev)) != DPC_OK) return st;
  if ((st = begin_call(workspace, stats, s)) != DPC_OK) return st;
  // the root grid and every child run child_threads threads; children are KC_X sized
  const void *fn = bfs_kernel(level);
  resolve_device(dev, tuning, level, fn, fn, n, &c);
  const int full = blocks_per_sm(dev, fn, c.child_threads) * sm_count(dev);
  int root_blocks = (tuning && tuning->parent_blocks > 0) ? tuning->parent_blocks : full;
  const int queue_blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full)
                               ? tuning->parent_blocks : full;
  BfsParams p;
  std::memset(&p, 0, sizeof(p));
  p.off = off;
  p.col = col;
  p.level = bfs_level;
  p.n = n;
  p.source = source;
  p.chunk = c.chunk;
  p.child_blocks = c.child_blocks;
  p.child_threads = c.child_threads;
  p.launch_budget = launch_budget(dev);
  char *b = static_cast<char *>(workspace);
  p.hdr = reinterpret_cast<WsHeader *>(b);
  b += kHeaderBytes;
  if (level == DPC_FLAT) {
    p.frontier = reinterpret_cast<int *>(b);
    p.next = reinterpret_cast<int *>(b + align_up((size_t)n * sizeof(int), 256));
  } else if (level != DPC_BASIC_DP) {
    const size_t mu = bfs_max_units(n, m, c.chunk, level);
    p.units = reinterpret_cast<int2 *>(b);
    p.max_units = (int)(mu > (size_t)INT_MAX ? INT_MAX : mu);
  }
  p.stats = stats;
  if (bfs_launch(p, level, root_blocks, queue_blocks, s) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return finish_call(s, c, p.hdr);
}

// ------------------------------------------------------------------ SSSP

dpc_status dpc_sssp_workspace_size(int32_t n, int32_t m, dpc_level level, const dpc_tuning *tuning, size_t *bytes) {
  if (!bytes || n < 1 || m < 0 || m > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, kSsspChunk, &c);
  if (st != DPC_OK) return st;
  *bytes = sssp_workspace_bytes(n, m, level, c);
  return *bytes ? DPC_OK : DPC_ERR_INVALID_ARG;
}

dpc_status dpc_sssp(const int32_t *off, const int32_t *col, const uint32_t *w, int32_t n, int32_t m, int32_t source,
                    uint32_t *dist, dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                    dpc_stats *stats, dpc_stream_t stream) {
  if (n < 1 || m < 0 || m > kMaxIndex || source < 0 || source >= n || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  if (!off || !dist || (m > 0 && (!col || !w))) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, kSsspChunk, &c);
  if (st != DPC_OK) return st;
  if (!workspace || workspace_bytes < sssp_workspace_bytes(n, m, level, c)) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = current_device(&dev)) != DPC_OK) return st;
  if ((st = begin_call(workspace, stats, s)) != DPC_OK) return st;
  resolve_device(dev, tuning, level, sssp_parent_kernel(level), sssp_child_kernel(level), n, &c);

  SsspParams p;
  std::memset(&p, 0, sizeof(p));
  p.off = off;
  p.col = col;
  p.w = w;
  p.dist = dist;
  p.n = n;
  p.m = m;
  p.source = source;
  p.threshold = c.threshold;
  p.chunk = c.chunk;
  p.level = level;
  p.parent_blocks = c.parent_blocks;
  p.parent_threads = c.parent_threads;
  p.commit_blocks = c.parent_blocks;
  p.child_blocks = c.child_blocks;
  p.child_threads = c.child_threads;
  p.heap = (c.flags & DPC_FLAG_DEVICE_MALLOC) && (level == DPC_WARP || level == DPC_BLOCK) ? 1 : 0;
  p.stream_edges = (size_t)m * (sizeof(int) + sizeof(unsigned)) > l2_bytes(dev) / 2 ? 1 : 0;
  p.delta = c.delta;
  p.sub_delta = c.sub_delta;
  // Without a split the frontier of round n is empty (Bellman-Ford's bound);
  // with one, the cap only keeps the round stamps below their sentinel.
  p.max_rounds = (c.delta || c.sub_delta) ? 0xFFFFFFF0u : (unsigned)n + 1u;
  p.prebuffer = level == DPC_QUEUE ? 1 : 0;
  p.launch_budget = launch_budget(dev);
  sssp_carve(p, workspace, n, m, level, c);
  p.stats = stats;
  if (level == DPC_QUEUE) {
    // one cooperative grid: every block co-resident (occupancy with the staging buffers)
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sssp_queue_kernel(), c.parent_threads,
                                                      sssp_queue_smem(c.parent_threads)) != cudaSuccess ||
        nb < 1) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    const int full = nb * sm_count(dev);
    // Every round crosses three grid barriers, whose cost grows with the
    // blocks, while the relaxations want warps in flight to hide load
    // latency: about one block per 4,096 edges, at least 64 and at most four
    // per SM, below 2^24 edges; all that fit above. Measured best: R-MAT 12 at
    // 38-76 blocks, 14 at 76-152, 16 at 256-304, 18 at 304-912, 22 at six
    // per SM.
    const int sms = sm_count(dev);
    int sized = full;
    // With a near-far split the rounds are many and small, so their barriers
    // weigh more: three blocks per SM measured best on R-MAT 22 (3.8 ms
    // against 4.6 ms with every resident block at split width 200, sub-split 8).
    if (c.delta && m >= (1 << 24) && 3 * sms < full) sized = 3 * sms;
    if (m < (1 << 24)) {
      sized = m >> 12;
      if (sized < 64) sized = 64;
      if (sized > 4 * sms) sized = 4 * sms;
      if (sized > full) sized = full;
    }
    const int blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks
                                                                                              : sized;
    if (sssp_queue_launch(p, blocks, s) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    return finish_call(s, c, p.hdr);
  }
  unsigned rounds = 0;
  if (sssp_launch(p, level, s, &rounds) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  host_scratch().rounds = rounds;
  if (level == DPC_FLAT && stats &&
      cudaMemcpyAsync(&stats->rounds, &host_scratch().rounds, sizeof(rounds), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return DPC_ERR_CUDA;
  if (level == DPC_FLAT && cudaStreamSynchronize(s) != cudaSuccess) return DPC_ERR_CUDA;
  return finish_call(s, c, p.hdr);
}

// ------------------------------------------------------------------ trees

// Children per unit. A unit's children are walked by one thread, so a level
// lasts as long as its longest unit; the levels without launch latency gain
// most from short units (2M-node tree: queue 0.62 ms at 32, 0.20 ms at 8; grid
// 0.83 ms at 32, 0.70 ms at 16), the warp and block levels lose from the
// extra units.
static int tree_default_chunk(dpc_level level) {
  return level == DPC_QUEUE ? 8 : level == DPC_GRID ? 16 : 32;
}

dpc_status dpc_tree_workspace_size(int32_t n, dpc_level level, const dpc_tuning *tuning, size_t *bytes) {
  if (!bytes || n < 1 || n > kMaxIndex || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, tree_default_chunk(level), &c);
  if (st != DPC_OK) return st;
  *bytes = tree_workspace_bytes(n, level, c);
  return *bytes ? DPC_OK : DPC_ERR_INVALID_ARG;
}

static dpc_status tree_call(int op, const int32_t *coff, const int32_t *cidx, int32_t n, int32_t root, int32_t *out,
                            dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                            dpc_stats *stats, dpc_stream_t stream) {
  if (n < 1 || n > kMaxIndex || root < 0 || root >= n || !valid_level(level)) return DPC_ERR_INVALID_ARG;
  if (!coff || !out || (n > 1 && !cidx)) return DPC_ERR_INVALID_ARG;
  LaunchCfg c;
  dpc_status st = resolve_static(tuning, tree_default_chunk(level), &c);
  if (st != DPC_OK) return st;
  if (!workspace || workspace_bytes < tree_workspace_bytes(n, level, c)) return DPC_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = current_device(&dev)) != DPC_OK) return st;
  if ((st = begin_call(workspace, stats, s)) != DPC_OK) return st;
  const void *visit = level == DPC_QUEUE ? tree_queue_kernel(op, tree_chained_postwork(n)) : tree_visit_kernel(level, op);
  resolve_device(dev, tuning, level, visit, visit, n, &c);

  TreeParams p;
  p.chain = 0;  // the queue level sets its postwork form below
  p.par = nullptr;
  p.link = nullptr;
  std::memset(&p, 0, sizeof(p));
  p.coff = coff;
  p.cidx = cidx;
  p.out = out;
  p.n = n;
  p.root = root;
  p.op = op;
  p.level = level;
  p.chunk = level == DPC_FLAT ? INT_MAX : c.chunk;
  p.chunk_shift = level != DPC_FLAT && (c.chunk & (c.chunk - 1)) == 0 ? __builtin_ctz((unsigned)c.chunk) : -1;
  p.child_blocks = c.child_blocks;
  p.child_threads = c.child_threads;
  // every recursive grid keeps a postwork tail launch pending until its subtree
  // is done, so a call may hold twice its optional launches in the pool
  p.launch_budget = launch_budget(dev) / 2;
  p.hdr = reinterpret_cast<WsHeader *>(workspace);
  if (level != DPC_BASIC_DP) {
    const size_t mu = tree_max_units(n, p.chunk);
    p.units = reinterpret_cast<int2 *>(static_cast<char *>(workspace) + kHeaderBytes);
    p.max_units = (int)(mu > (size_t)INT_MAX ? INT_MAX : mu);
    if (level == DPC_QUEUE) {
      char *b = static_cast<char *>(workspace) + kHeaderBytes + tree_units_bytes(n, level, p.chunk);
      p.level_ends = reinterpret_cast<int *>(b);
      b += align_up(((size_t)n + 2) * sizeof(int), 256);
      p.chain = tree_chained_postwork(n) ? 1 : 0;
      if (p.chain) {
        p.par = reinterpret_cast<int *>(b);
        b += align_up((size_t)n * sizeof(int), 256);
        p.link = reinterpret_cast<unsigned long long *>(b);
      }
    }
  }
  p.stats = stats;
  if (level == DPC_QUEUE) {
    // one cooperative grid (every block co-resident), child_threads threads per block (at most 512)
    const int threads = c.child_threads < kTreeQueueMaxThreads ? c.child_threads : kTreeQueueMaxThreads;
    const int nb = blocks_per_sm(dev, visit, threads);
    const int full = nb * sm_count(dev);
    // Trees of 2^24 nodes or more get every resident block, to keep loads in
    // flight over their long levels (depth-5 trees of 32 M and 157 M nodes: 2
    // and 8 % faster with four blocks per SM than with three). Smaller ones
    // get two per SM, since every level ends in a grid barrier (2M-node tree:
    // 0.20 ms with one or two per SM, 0.22-0.23 with three or four).
    const int sized = n >= (1 << 24) ? full : (nb < 2 ? nb : 2) * sm_count(dev);
    const int blocks = (tuning && tuning->parent_blocks > 0 && tuning->parent_blocks < full) ? tuning->parent_blocks
                                                                                              : sized;
    if (tree_queue_launch(p, blocks, threads, s) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    return finish_call(s, c, p.hdr);
  }
  unsigned levels = 0;
  if (tree_launch(p, level, c.parent_blocks, s, &levels) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  host_scratch().rounds = levels;
  if (level == DPC_FLAT && stats &&
      cudaMemcpyAsync(&stats->rounds, &host_scratch().rounds, sizeof(levels), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return DPC_ERR_CUDA;
  if (level == DPC_FLAT && cudaStreamSynchronize(s) != cudaSuccess) return DPC_ERR_CUDA;
  return finish_call(s, c, p.hdr);
}

dpc_status dpc_tree_descendants(const int32_t *coff, const int32_t *cidx, int32_t n, int32_t root, uint32_t *desc,
                                dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                                dpc_stats *stats, dpc_stream_t stream) {
  return tree_call(kDescendants, coff, cidx, n, root, reinterpret_cast<int32_t *>(desc), level, tuning, workspace,
                   workspace_bytes, stats, stream);
}

dpc_status dpc_tree_height(const int32_t *coff, const int32_t *cidx, int32_t n, int32_t root, int32_t *height,
                           dpc_level level, const dpc_tuning *tuning, void *workspace, size_t workspace_bytes,
                           dpc_stats *stats, dpc_stream_t stream) {
  return tree_call(kHeight, coff, cidx, n, root, height, level, tuning, workspace, workspace_bytes, stats, stream);
}

}  // extern "C"
