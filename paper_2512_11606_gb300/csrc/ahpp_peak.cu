// Row-access peaks of the GPU, for roofline reporting.
//
// The batched kernel moves its data as random 128-byte rows (the 32 queries'
// FP32 values of one node): gathers from the residue / t_V / t_A tables and
// float4 reductions into the next round's t_A.  On this access pattern the
// L2 -> SM path, not HBM, sets the ceiling once a table fits in L2.  This
// file measures that ceiling on the running GPU: the rate of random row
// gathers from, or row reductions into, a table of a given size, with
// enough warps and loads in flight to saturate the memory system.
#include <cuda_runtime.h>

#include <algorithm>

#include "ahpp_host.h"
#include "../../include/ahpp_measure.h"

namespace ahpp {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakDepth = 8;          // row gathers in flight per 8-lane group
constexpr uint64_t kPeakRows = 32ull << 20;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
  return x;
}

// Every 8-lane group reads kPeakDepth random rows at a time, one float4 per
// lane; row indices are mix32(i ^ seed) % rows, so every access is in range.
__global__ void __launch_bounds__(kPeakThreads) k_peak_gather(const float4* __restrict__ t, uint32_t rows,
                                                              uint64_t n, uint32_t seed, float* sink) {
  const uint32_t l8 = threadIdx.x & 7u;
  const uint64_t g0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 3;
  const uint64_t ng = ((uint64_t)gridDim.x * blockDim.x) >> 3;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint64_t i = g0 * kPeakDepth; i < n; i += ng * kPeakDepth) {
    float4 v[kPeakDepth];
#pragma unroll
    for (int d = 0; d < kPeakDepth; ++d) {
      const uint64_t e = i + d;
      const uint32_t r = mix32((uint32_t)e ^ seed) % rows;
      v[d] = e < n ? __ldg(t + (uint64_t)r * 8 + l8) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int d = 0; d < kPeakDepth; ++d) {
      acc.x += v[d].x; acc.y += v[d].y; acc.z += v[d].z; acc.w += v[d].w;
    }
  }
  if (acc.x + acc.y + acc.z + acc.w == 1.0f) sink[0] = 1.f;   // keeps the loads live
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_reduce(float4* t, uint32_t rows, uint64_t n,
                                                              uint32_t seed) {
  const uint32_t l8 = threadIdx.x & 7u;
  const uint64_t g0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 3;
  const uint64_t ng = ((uint64_t)gridDim.x * blockDim.x) >> 3;
  for (uint64_t i = g0; i < n; i += ng) {
    const uint32_t r = mix32((uint32_t)i ^ seed) % rows;
    atomicAdd(t + (uint64_t)r * 8 + l8, make_float4(0.f, 0.f, 0.f, 0.f));
  }
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace ahpp

using namespace ahpp;

extern "C" int ahpp_row_access_peak(int device, uint64_t table_bytes, int op, double* rows_per_s) {
  if (!rows_per_s || (op != 0 && op != 1) || table_bytes < 128 || table_bytes > (8ull << 30) ||
      device < 0) {
    set_error("ahpp_row_access_peak: need device >= 0, op 0 (gather) or 1 (reduce), "
              "128 <= table_bytes <= 8 GiB and an output pointer");
    return AHPP_EINVAL;
  }
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device >= n_dev) {
    set_error("ahpp_row_access_peak: no such CUDA device");
    return AHPP_ECUDA;
  }
  DevGuard guard(device);
  int sms = 0, per_sm = 0;
  AHPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const void* fn = op == 0 ? (const void*)k_peak_gather : (const void*)k_peak_reduce;
  AHPP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0));
  const int grid = std::max(1, sms * std::max(1, per_sm));
  const uint32_t rows = (uint32_t)(table_bytes / 128);

  float4* t = nullptr;
  float* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = AHPP_OK;
  float best = 0.f;
  auto fail = [&](cudaError_t e, const char* where) {
    if (rc == AHPP_OK) rc = cuda_fail(e, where);
  };
  cudaError_t e = cudaMalloc(&t, (size_t)rows * 128);
  if (e != cudaSuccess) {
    set_error("ahpp_row_access_peak: cannot allocate the table");
    rc = AHPP_ENOMEM;
  }
  if (rc == AHPP_OK && (e = cudaMalloc(&sink, 16)) != cudaSuccess) fail(e, "cudaMalloc");
  if (rc == AHPP_OK && (e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
    fail(e, "cudaStreamCreate");
  if (rc == AHPP_OK && (e = cudaEventCreate(&a)) != cudaSuccess) fail(e, "cudaEventCreate");
  if (rc == AHPP_OK && (e = cudaEventCreate(&b)) != cudaSuccess) fail(e, "cudaEventCreate");
  if (rc == AHPP_OK && (e = cudaMemsetAsync(t, 0, (size_t)rows * 128, st)) != cudaSuccess)
    fail(e, "cudaMemsetAsync");
  for (int it = 0; rc == AHPP_OK && it < 6; ++it) {      // one warm-up, best of five
    if ((e = cudaEventRecord(a, st)) != cudaSuccess) { fail(e, "cudaEventRecord"); break; }
    if (op == 0)
      k_peak_gather<<<grid, kPeakThreads, 0, st>>>(t, rows, kPeakRows, 0x9e3779b9u * (it + 1), sink);
    else
      k_peak_reduce<<<grid, kPeakThreads, 0, st>>>(t, rows, kPeakRows, 0x9e3779b9u * (it + 1));
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "row access kernel launch"); break; }
    if ((e = cudaEventRecord(b, st)) != cudaSuccess) { fail(e, "cudaEventRecord"); break; }
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) { fail(e, "row access kernel"); break; }
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) { fail(e, "cudaEventElapsedTime"); break; }
    if (it > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  if (t) cudaFree(t);
  if (rc != AHPP_OK) return rc;
  *rows_per_s = (double)kPeakRows / (best * 1e-3);
  return AHPP_OK;
}
