// Host-side definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ahpp.h"
#include "ahpp_internal.cuh"
#include "ahpp_query1.cuh"
#include "ahpp_batch.cuh"

namespace ahpp {

// NVTX range over a host call (visible in a profiler's timeline; the calls
// do nothing unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

#define AHPP_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::ahpp::cuda_fail(e_, #call); \
  } while (0)

// Host copy of one adjacency direction before upload.
struct HostAdj {
  std::vector<uint32_t> off, idx;
  std::vector<float> w;        // raw weights
  std::vector<float> c;        // direction coefficient (structure only)
};

struct HostItems {
  std::vector<uint4> items;
  std::vector<uint32_t> split_nchunks;
  uint32_t n_long = 0;
};

// Work-item shapes.
struct ItemShape {
  uint32_t short_max;   // rows with at most this many neighbours are "short"
  uint32_t group_rows;  // short rows per item (single query: one per lane)
  uint32_t group_nnz;   // max neighbours per short item (batched)
  uint32_t chunk;       // neighbours per chunk of a long row
};

HostItems build_items(const std::vector<uint32_t>& deg, const ItemShape& shape);
// Batched row units: rows longer than `chunk` (a prefix, rows being sorted by
// degree) become split chunks; every other row is one unit.
HostItems build_units(const std::vector<uint32_t>& deg, uint32_t chunk);

// Device allocation tracked by the graph.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace ahpp

struct ahpp_graph {
  ahpp_config cfg{};
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;

  uint64_t n_u = 0, n_v = 0, n_a = 0, n_e = 0, n_ea = 0;
  double lambda = 1.0;
  uint32_t lambda_T = 0;
  bool bf16 = true;

  ahpp::DevGraph dg{};
  std::vector<ahpp::DevBuf> bufs;   // everything allocated for the graph
  size_t n_graph_bufs = 0;          // bufs[0, n_graph_bufs): the graph's own arrays (what a cache saves)
  uint64_t graph_bytes = 0;

  // internal <-> caller id maps of U
  std::vector<uint32_t> h_u_old2new, h_u_new2old;
  uint32_t* d_u_new2old = nullptr;
  uint32_t* d_u_old2new = nullptr;

  // single-query state
  ahpp::Q1State q1{};
  int q1_grid = 0;
  // single-query kernel's shared-memory plan (see Q1Params)
  uint32_t q1_smem = 0;
  int q1_attr_push = 0, q1_ta_smem = 0;
  uint32_t q1_dense_div = 32;     // pull rounds once the frontier covers > 1/dense_div of the edges
  uint32_t q1_vw_max = ahpp::kQ1VecWidthDefault;   // lanes per short row in the pull phases (at most)
  std::string tune_log;           // the last autotune's measurements (JSON object)
  uint32_t n_split1 = 0;
  uint64_t q1_bytes = 0;

  // batched state (allocated on first use, grown on demand)
  ahpp::BatchState bt{};
  uint32_t batch_tile = 32, batch_groups = 1;
  int bt_grid = 0;
  uint64_t tile_bytes = 0;

  // top-k scratch
  void* topk_scratch = nullptr;
  size_t topk_scratch_bytes = 0;

  // failure-detection self-test: the next launch's grid barriers start with
  // a counter that can never reach the block count (see reset_barrier)
  std::atomic<int> wait_trap{0};

  void* alloc(size_t bytes);          // cudaMalloc + track (nullptr on failure)
  void release_all();
};

namespace ahpp {
// Clear a grid barrier before a persistent launch on `stream`.  When the
// graph's self-test trap is armed (ahpp_selftest_arm_wait_timeout) the
// counter is set far above any grid size instead, so the launch's first
// barrier never fills and every block's bounded spin runs out; the trap is
// consumed by the first launch that sees it.
int reset_barrier(ahpp_graph* g, GridBarrier* bar, cudaStream_t stream, bool keep_trap = false);
// Zero if the barrier's error word is clear; kStatusWait if a wait gave up.
// Synchronous (reads one word from the device on `stream`).
int barrier_status(GridBarrier* bar, cudaStream_t stream, int* status);
int build_graph(const ahpp_graph_desc* desc, ahpp_graph* g);
// The kernels' algorithm id of an AHPP_* constant (-1 if none).
int kernel_algo(int algo);
// Shared-memory plan of the single-query kernel (the grid does not depend on
// it: one block per SM).
void plan_query1_smem(ahpp_graph* g);
// Index into kChunkSizes of a configured chunk size (0: the default), -1 if
// it is not one of them.
int chunk_choice(uint32_t chunk);
// Make chunk choice `choice` (index into kChunkSizes) the active unit lists.
void select_chunk(DevGraph& G, uint32_t choice);
int alloc_query_state(ahpp_graph* g);
int run_lambda(ahpp_graph* g);
int run_query1(ahpp_graph* g, uint32_t q_new, double eps, uint32_t lambda_T_mode,
               cudaStream_t stream, QCtl* h_ctl);
int topk_single(ahpp_graph* g, const float* d_score, uint32_t k, uint32_t* d_nodes,
                float* d_scores, uint32_t* d_n, cudaStream_t stream);
// The batched kernel's grid (computed once per graph).
int batch_plan(ahpp_graph* g, BatchParams& p);
int run_single_device(ahpp_graph* g, uint32_t q, double eps, uint32_t k, uint32_t* d_out_nodes,
                      float* d_out_scores, uint32_t* d_out_n, ahpp_stats* d_stats, cudaStream_t s);
}  // namespace ahpp
