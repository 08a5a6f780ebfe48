// Diagnostics (no counterpart in the paper).
//
// dpc_wait_selftest: the bounded waits that every grid barrier of the queue
// levels and of the batched engine relies on (WaitClock in dpc_runtime.cuh):
// one block waits for a word that nothing ever sets, gives up when the limit
// has passed and reports DPC_ERR_TIMEOUT, leaving the context usable. This is
// how a run whose blocks stopped arriving at a barrier ends.
//
// dpc_gather_rate: the rate of random 4-byte gathers from an array held in
// L2, the ceiling of the SpMV kernels' x gathers (uniform columns over 2^20
// entries: one 32-byte L2 sector per 4 useful bytes).
#include "dpc_internal.h"
#include "dpc_runtime.cuh"

namespace dpc {
namespace {

__device__ unsigned g_never_set;  // zero-initialised; no code writes it

__global__ void wait_selftest_kernel(unsigned long long limit_ns, unsigned *status) {
  if (threadIdx.x != 0) return;
  const unsigned long long t0 = global_ns();
  WaitClock clk(limit_ns);
  unsigned code = 0;
  while (*reinterpret_cast<volatile unsigned *>(&g_never_set) == 0u) {
    __nanosleep(64);
    if (clk.expired()) {
      code = DPC_ERR_TIMEOUT;
      break;
    }
  }
  const unsigned long long waited = global_ns() - t0;
  status[0] = code;
  status[1] = (unsigned)(waited / 1000ull);  // microseconds waited
}

// Every thread: `batches` batches of kGatherBatch independent loads at
// pseudo-random positions (a linear congruential sequence per thread, bits 7
// and up), issued back to back like the SpMV gathers, then added up.
constexpr int kGatherBatch = 16;

__global__ void __launch_bounds__(256) gather_rate_kernel(const float *__restrict__ x, unsigned mask, int batches,
                                                          float *out) {
  unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  float acc = 0.f;
  for (int b = 0; b < batches; ++b) {
    unsigned idx[kGatherBatch];
#pragma unroll
    for (int j = 0; j < kGatherBatch; ++j) {
      h = h * 1664525u + 1013904223u;
      idx[j] = (h >> 7) & mask;
    }
    float v[kGatherBatch];
#pragma unroll
    for (int j = 0; j < kGatherBatch; ++j) v[j] = __ldcg(x + idx[j]);
#pragma unroll
    for (int j = 0; j < kGatherBatch; ++j) acc += v[j];
  }
  acc = warp_sum(acc);
  if (lane_id() == 0) atomicAdd(out, acc);
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" dpc_status dpc_gather_rate(const float *x, int32_t n, int32_t batches, float *out, int64_t *gathers,
                                      dpc_stream_t stream) {
  if (!x || !out || !gathers || n < 32 || n > (1 << 26) || (n & (n - 1)) || batches < 1) return DPC_ERR_INVALID_ARG;
  int dev = 0, sms = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)gather_rate_kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  const int blocks = (bps > 0 ? bps : 1) * sms;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  gather_rate_kernel<<<blocks, 256, 0, s>>>(x, (unsigned)n - 1u, batches, out);
  *gathers = (int64_t)blocks * 256 * batches * kGatherBatch;
  return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}

extern "C" dpc_status dpc_wait_selftest(uint32_t limit_us, uint32_t *status, dpc_stream_t stream) {
  if (!status || limit_us == 0 || limit_us > 10000000u) return DPC_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)limit_us * 1000ull, status);
  return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}
