// Self-test of the device-side failure detection: every wait in the
// persistent kernels is a grid barrier (grid_sync) whose spin is bounded;
// when it gives up it raises the barrier's error flag and returns false, the
// kernel unwinds, and the host reports AHPP_ETIMEOUT.  This runs that same
// barrier with one more participant than the grid has blocks, so the
// barrier can never fill: the wait must give up within its limit, report it,
// and leave the context usable for the next launch.
#include <cuda_runtime.h>

#include "ahpp_host.h"

namespace ahpp {
namespace {

__global__ void k_wait_selftest(GridBarrier* bar, unsigned int participants, unsigned int* gave_up) {
  const bool ok = grid_sync(bar, participants);
  if (threadIdx.x == 0 && !ok) atomicAdd(gave_up, 1u);
}

__global__ void k_after(unsigned int* x) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *x = 42u;
}

}  // namespace
}  // namespace ahpp

using namespace ahpp;

extern "C" int ahpp_selftest_wait_timeout(int device, int* blocks_gave_up, int* context_ok) {
  if (!blocks_gave_up || !context_ok || device < 0) {
    set_error("ahpp_selftest_wait_timeout: need device >= 0 and two output pointers");
    return AHPP_EINVAL;
  }
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device >= n_dev) {
    cudaGetLastError();
    set_error("ahpp_selftest_wait_timeout: no such CUDA device");
    return AHPP_ECUDA;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  AHPP_CUDA(cudaSetDevice(device));
  GridBarrier* bar = nullptr;
  unsigned int* d = nullptr;
  unsigned int h[2] = {0, 0};
  int rc = AHPP_OK;
  cudaError_t e = cudaMalloc(&bar, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMalloc(&d, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(bar, 0, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) {
    // two blocks, three participants: neither block can ever be the last to arrive
    k_wait_selftest<<<2, 64>>>(bar, 3u, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    k_after<<<1, 32>>>(d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = cuda_fail(e, "wait self-test");
  if (d) cudaFree(d);
  if (bar) cudaFree(bar);
  if (prev >= 0) cudaSetDevice(prev);
  if (rc != AHPP_OK) return rc;
  *blocks_gave_up = (int)h[0];
  *context_ok = h[1] == 42u;
  return AHPP_OK;
}

// Arms the graph's wait trap: the next persistent launch on g (single query,
// batch, no-allocation query, power iteration or a serving step) starts with
// a grid barrier that can never fill, so its first wait, before any round,
// runs out; the call that made the launch must report AHPP_ETIMEOUT.
extern "C" int ahpp_selftest_arm_wait_timeout(ahpp_graph* g) {
  if (!g) { set_error("ahpp_selftest_arm_wait_timeout: null graph"); return AHPP_EINVAL; }
  g->wait_trap.store(1);
  return AHPP_OK;
}
