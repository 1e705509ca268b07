// Single-query push with no device allocation: the per-query working state
// (residues, reserves, frontier lists, round accumulators, grid barrier)
// lives in one file-scope device array instead of memory allocated by the
// graph or by the call.
//
// Why: some callers cannot call cudaMalloc / cudaFree at query time - a
// serving framework that has reserved the whole device memory pool for its
// own allocator, a latency-critical thread that must not take the implicit
// device synchronisation those calls can cause, or code that runs where the
// allocator is off limits.  This entry point lets them run a query with only
// the buffers they pass in.
//
// Limits and sharing:
//   - the array holds kNoAllocBytes (32 MiB) on every device that loads the
//     library, for the life of the process;
//   - graphs whose single-query state does not fit are rejected (AHPP_EINVAL);
//   - every call uses the same array and leaves its contents behind; the
//     kernel clears everything that must start at zero.  Calls that overlap
//     on the GPU would race on the array: this entry point serialises its own
//     calls (process-wide lock, and it waits for its stream before returning).
//   - the first call on a device resolves the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture.
#include <cstring>
#include <mutex>

#include "ahpp_host.h"

namespace ahpp {
namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

__global__ void k_scatter_out(const float* __restrict__ pi, const uint32_t* __restrict__ n2o,
                              uint32_t n, float* __restrict__ out) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
    out[n2o[u]] = pi[u];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve the single-query state out of base; returns the bytes needed.
size_t carve(const ahpp_graph* g, char* base, Q1State* s) {
  const size_t nu = g->n_u, nv = std::max<uint64_t>(g->n_v, 1), na = std::max<uint64_t>(g->n_a, 1);
  const size_t ns = std::max<uint32_t>(g->n_split1, 1);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  s->r_u = (float*)take(4 * nu);
  s->pi = (float*)take(4 * nu);
  s->pic = (float*)take(4 * nu);
  s->t_v = (float*)take(4 * nv);
  s->t_a = (float*)take(4 * na);
  s->t_a2 = (float*)take(4 * na);
  s->list_u = (uint32_t*)take(4 * nu);
  s->split_acc = (float*)take(4 * ns);
  s->split_cnt = (uint32_t*)take(4 * ns);
  s->ctl = (QCtl*)take(sizeof(QCtl));
  s->racc = (RAcc*)take(3 * sizeof(RAcc));
  s->bar = (GridBarrier*)take(sizeof(GridBarrier));
  s->final_maxr_bits = (unsigned int*)take(2 * sizeof(unsigned int));
  s->trace_frontier = nullptr;
  s->trace_maxr = nullptr;
  return off;
}

}  // namespace

// Parameters of a single query (shared with the allocating entry points).
Q1Params noalloc_params(const ahpp_graph* g, uint32_t q_new, double eps);

}  // namespace ahpp

using namespace ahpp;

extern "C" int ahpp_query_dense_noalloc(ahpp_graph* g, uint32_t q, double eps, float* d_out_pi,
                                        void* stream) {
  if (!g || !d_out_pi) { set_error("ahpp_query_dense_noalloc: null argument"); return AHPP_EINVAL; }
  if (q >= g->n_u) { set_error("ahpp_query_dense_noalloc: q is not a node of U"); return AHPP_EINVAL; }
  if (!(eps > 0.0) || !std::isfinite(eps)) {
    set_error("ahpp_query_dense_noalloc: eps must be > 0 and finite");
    return AHPP_EINVAL;
  }
  Q1State s;
  const size_t need = carve(g, nullptr, &s);
  if (need > kNoAllocBytes) {
    set_error("ahpp_query_dense_noalloc: the graph needs " + std::to_string(need) +
              " bytes of query state; the static scratch holds " + std::to_string(kNoAllocBytes) +
              " (use ahpp_query_dense)");
    return AHPP_EINVAL;
  }
  if (g->device < 0 || g->device >= kMaxDevices) { set_error("device ordinal out of range"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  if (!g_noalloc_ptr[g->device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "ahpp_query_dense_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[g->device] = ptr;
  }
  carve(g, (char*)g_noalloc_ptr[g->device], &s);
  cudaStream_t st = stream ? (cudaStream_t)stream : g->stream;
  Q1Params p = noalloc_params(g, g->h_u_old2new[q], eps);
  p.trace_cap = 0;
  if (int rc = reset_barrier(g, s.bar, st)) return rc;
  const int e = launch_query1(g->dg, s, p, g->bf16, g->q1_grid, st);
  if (e) return cuda_fail((cudaError_t)e, "ahpp_query_dense_noalloc: launch");
  k_scatter_out<<<std::max(1, g->sm_count * 4), 256, 0, st>>>(s.pi, g->d_u_new2old, (uint32_t)g->n_u,
                                                              d_out_pi);
  AHPP_CUDA(cudaGetLastError());
  QCtl ctl;
  AHPP_CUDA(cudaMemcpyAsync(&ctl, s.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
  int bst = kStatusOk;
  if (int rc = barrier_status(s.bar, st, &bst)) return rc;     // also waits for the stream
  if (ctl.status == kStatusWait || bst == kStatusWait) {
    set_error("ahpp_query_dense_noalloc: a device wait gave up");
    return AHPP_ETIMEOUT;
  }
  if (ctl.status == kStatusCap) return AHPP_ENOTCONVERGED;
  return AHPP_OK;
}
