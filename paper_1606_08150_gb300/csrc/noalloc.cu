// dpc_spmv_csr_noalloc: the SpMV entry point for callers that may not
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need y = A x:
// code running under a memory manager that owns the whole device heap (a
// framework's caching allocator or an inference server's arena, where a
// second allocator would fragment or over-commit the budget), services with a
// fixed memory budget that forbid any allocation after start-up, and code on a
// latency-critical path where cudaMalloc/cudaFree would synchronise the device
// and stall every other stream. For them this entry point takes its scratch
// space from a fixed array compiled into the library instead of a caller
// workspace. It runs exactly the kernels of dpc_spmv_csr.
//
// The scratch array is a file-scope __device__ variable, so every GPU that
// loads the library holds DPC_NOALLOC_SCRATCH_BYTES of it until the process
// exits. Host code may not use the array's name as a device address: the host
// symbol is only a stand-in for it. The first call on each device therefore
// asks the runtime for the array's device address (cudaGetSymbolAddress, with
// that device current) and caches it; make that first call before any stream
// capture. All calls share the one array: the call clears the counters that
// must start at zero, and two calls whose kernels overlap on the GPU (for
// example on two streams) race on it.
#include <climits>
#include <cstring>
#include <mutex>

#include "dpc_internal.h"

namespace dpc {
namespace {

constexpr size_t kScratchBytes = DPC_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocDevices = 64;
constexpr int kMaxIndexNoAlloc = INT_MAX - (1 << 16);

__device__ __align__(256) unsigned char g_spmv_scratch[kScratchBytes];

struct NoAllocDevice {
  void *scratch = nullptr;  // device address of g_spmv_scratch on this device
  int sms = 0;
  int parent_bps[5][33] = {};  // resident blocks per SM, by level and threads/32
  int child_bps[5][33] = {};
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[kNoAllocDevices];

// Once per device, with that device current.
dpc_status noalloc_setup(int dev, NoAllocDevice **out) {
  if (dev < 0 || dev >= kNoAllocDevices) return DPC_ERR_CUDA;
  NoAllocDevice &d = g_noalloc[dev];
  if (!d.scratch) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_spmv_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DPC_ERR_CUDA;
    d.scratch = ptr;
  }
  *out = &d;
  return DPC_OK;
}

int noalloc_bps(int cache[5][33], int level, const void *fn, int threads) {
  int &slot = cache[level][threads / 32];
  if (slot == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess) {
      cudaGetLastError();
      nb = 1;
    }
    slot = nb > 0 ? nb : 1;
  }
  return slot;
}

// The end of a call: a launch error first, then, with DPC_FLAG_SYNC_CHECK, a
// stream synchronisation and the device status word.
dpc_status noalloc_finish(cudaStream_t s, unsigned flags, const WsHeader *hdr) {
  if (cudaGetLastError() != cudaSuccess) return DPC_ERR_CUDA;
  if (flags & DPC_FLAG_SYNC_CHECK) {
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    unsigned dst = 0;
    if (cudaMemcpy(&dst, &hdr->status, sizeof(dst), cudaMemcpyDeviceToHost) != cudaSuccess) return DPC_ERR_CUDA;
    return (dpc_status)dst;
  }
  return DPC_OK;
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" dpc_status dpc_spmv_csr_noalloc(const int32_t *off, const int32_t *col, const float *val, int32_t nrows,
                                           int32_t ncols, int32_t nnz, const float *x, float *y, dpc_level level,
                                           const dpc_tuning *tuning, dpc_stats *stats, dpc_stream_t stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > kMaxIndexNoAlloc || level < DPC_BASIC_DP || level > DPC_GRID)
    return DPC_ERR_INVALID_ARG;
  if (nrows > 0 && (!off || !y)) return DPC_ERR_INVALID_ARG;
  if (nnz > 0 && (!col || !val || !x || ncols == 0)) return DPC_ERR_INVALID_ARG;
  dpc_tuning z;
  std::memset(&z, 0, sizeof(z));
  const dpc_tuning *t = tuning ? tuning : &z;
  LaunchCfg c;
  c.threshold = t->threshold > 0 ? t->threshold : (t->threshold < 0 ? 0 : 32);
  c.parent_threads = t->parent_threads ? t->parent_threads : 256;
  c.child_threads = t->child_threads ? t->child_threads : 256;
  c.chunk = t->chunk ? t->chunk : 2048;
  c.flags = t->flags;
  c.parent_blocks = t->parent_blocks;
  c.child_blocks = t->child_blocks;
  c.delta = 0;
  c.sub_delta = 0;
  for (int th : {c.parent_threads, c.child_threads})
    if (th < 32 || th > 1024 || th % 32) return DPC_ERR_INVALID_ARG;
  if (c.chunk < 1 || c.chunk > (1 << 24) || t->parent_blocks < 0 || t->child_blocks < 0 || t->kc < 0)
    return DPC_ERR_INVALID_ARG;
  // the fixed array must hold everything this call's workspace would
  if (spmv_workspace_bytes(nrows, nnz, level, c) > kScratchBytes) return DPC_ERR_WORKSPACE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice *d = nullptr;
  dpc_status st = noalloc_setup(dev, &d);
  if (st != DPC_OK) return st;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(d->scratch);
  if (cudaMemsetAsync(hdr, 0, kHeaderBytes, s) != cudaSuccess) return DPC_ERR_CUDA;
  if (stats && cudaMemsetAsync(stats, 0, sizeof(dpc_stats), s) != cudaSuccess) return DPC_ERR_CUDA;
  if (nrows == 0) return noalloc_finish(s, c.flags, hdr);

  if (c.parent_blocks <= 0) {
    const long long full =
        (long long)noalloc_bps(d->parent_bps, level, spmv_parent_kernel(level), c.parent_threads) * d->sms;
    const long long need = (nrows + (long long)c.parent_threads - 1) / c.parent_threads;
    c.parent_blocks = (int)(need < full ? need : full);
  }
  if (c.child_blocks <= 0) {
    const int kc = t->kc > 0 ? t->kc : (level == DPC_BLOCK ? 16 : level == DPC_WARP ? 32 : 1);
    const long long full =
        (long long)noalloc_bps(d->child_bps, level, spmv_child_kernel(level), c.child_threads) * d->sms;
    c.child_blocks = (int)(full / kc > 0 ? full / kc : 1);
  }
  // stay below the device runtime's pending-launch pool as it stands (never resized here)
  size_t pool = 2048;
  cudaDeviceGetLimit(&pool, cudaLimitDevRuntimePendingLaunchCount);
  const long long reserve = (long long)pool / 8 > 1024 ? (long long)pool / 8 : 1024;

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
  p.launch_budget = (long long)pool > reserve ? (long long)pool - reserve : 0;
  p.hdr = hdr;
  p.stats = stats;
  if (level == DPC_WARP || level == DPC_BLOCK || level == DPC_GRID) {
    const size_t mu = spmv_max_units(nrows, nnz, c.threshold, c.chunk);
    char *b = static_cast<char *>(d->scratch) + kHeaderBytes;
    p.units = reinterpret_cast<int4 *>(b);
    b += align_up(mu * sizeof(int4), 256);
    p.partial = reinterpret_cast<float *>(b);
    b += align_up(mu * sizeof(float), 256);
    p.ucount = reinterpret_cast<unsigned *>(b);
    p.max_units = (int)mu;
  }
  if (spmv_launch(p, level, c, s) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return noalloc_finish(s, c.flags, hdr);
}
