// Top-k of one reserve vector: radix select over distinct 64-bit keys
// (score bits << 32 | ~caller id), so that the k largest keys are exactly the
// k best nodes ordered by score descending, then caller id ascending.  Up to
// six passes of 11/11/10 bits narrow down the k-th key (usually the three
// score passes suffice); the k winners are then gathered and sorted in one
// block (bitonic, k <= AHPP_MAX_K).
#include "ahpp_host.h"

namespace ahpp {

namespace {

constexpr int kPasses = 6;
constexpr int kBinsMax = 2048;
__device__ __constant__ int c_bits[kPasses] = {11, 11, 10, 11, 11, 10};

__device__ __forceinline__ unsigned long long key_of(const float* score, const uint32_t* n2o,
                                                     uint32_t u) {
  return ((unsigned long long)__float_as_uint(fmaxf(score[u], 0.f)) << 32) |
         (unsigned long long)(0xffffffffu - n2o[u]);
}

struct TopkScratch {
  unsigned int* hist;          // [kPasses][kBinsMax]
  unsigned long long* cand;    // [AHPP_MAX_K]
  uint32_t* cand_cnt;
  GridBarrier* bar;
};

__global__ void __launch_bounds__(kThreads)
k_topk1(const float* __restrict__ score, const uint32_t* __restrict__ n2o, uint32_t n, uint32_t k,
        TopkScratch sc, uint32_t* out_nodes, float* out_scores, uint32_t* out_n) {
  __shared__ unsigned int sh[kBinsMax];
  __shared__ unsigned long long sk[AHPP_MAX_K];
  const uint32_t gt = blockIdx.x * kThreads + threadIdx.x, nt = gridDim.x * kThreads;
  const unsigned int nb = gridDim.x;
  for (uint32_t i = gt; i < kPasses * kBinsMax; i += nt) sc.hist[i] = 0;
  if (gt == 0) *sc.cand_cnt = 0;
  if (!grid_sync(sc.bar, nb)) return;
  unsigned long long prefix = 0;
  unsigned long long thresh = 0;   // smallest winning key, once known
  uint32_t krem = k;
  int done_bits = 0;
  // Every block reads the same global histograms, so all blocks stop after
  // the same pass: as soon as the bucket holding the k-th key contains
  // exactly the keys still needed, all of that bucket wins.
  for (int pass = 0; pass < kPasses; ++pass) {
    const int bits = c_bits[pass];
    const int bins = 1 << bits;
    const int shift = 64 - done_bits - bits;
    for (int i = threadIdx.x; i < bins; i += kThreads) sh[i] = 0;
    __syncthreads();
    for (uint32_t u = gt; u < n; u += nt) {
      const unsigned long long key = key_of(score, n2o, u);
      if (done_bits == 0 || (key >> (64 - done_bits)) == prefix)
        atomicAdd(&sh[(key >> shift) & (bins - 1)], 1u);
    }
    __syncthreads();
    unsigned int* gh = sc.hist + pass * kBinsMax;
    for (int i = threadIdx.x; i < bins; i += kThreads)
      if (sh[i]) atomicAdd(&gh[i], sh[i]);
    if (!grid_sync(sc.bar, nb)) return;
    // the merged histogram into shared memory, then a warp-parallel pick
    for (int i = threadIdx.x; i < bins; i += kThreads) sh[i] = __ldcg(&gh[i]);
    __syncthreads();
    int d;
    uint32_t cum, h;
    radix_pick(sh, bins, krem, &d, &cum, &h);
    __syncthreads();
    krem -= cum;
    prefix = (prefix << bits) | (unsigned long long)d;
    done_bits += bits;
    if (h == krem || done_bits == 64) {
      thresh = prefix << (64 - done_bits);
      break;
    }
  }
  // exactly k keys are >= thresh (keys are distinct)
  for (uint32_t u = gt; u < n; u += nt) {
    const unsigned long long key = key_of(score, n2o, u);
    if (key >= thresh) {
      const uint32_t pos = atomicAdd(sc.cand_cnt, 1u);
      if (pos < AHPP_MAX_K) sc.cand[pos] = key;
    }
  }
  if (!grid_sync(sc.bar, nb)) return;
  if (blockIdx.x != 0) return;
  uint32_t m = 1;
  while (m < k) m <<= 1;
  for (uint32_t i = threadIdx.x; i < m; i += kThreads) sk[i] = i < k ? __ldcg(&sc.cand[i]) : 0ull;
  __syncthreads();
  for (uint32_t size = 2; size <= m; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < m; i += kThreads) {
        const uint32_t j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const unsigned long long a = sk[i], b = sk[j];
          if (desc ? (a < b) : (a > b)) { sk[i] = b; sk[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < k; i += kThreads) {
    out_nodes[i] = 0xffffffffu - (uint32_t)(sk[i] & 0xffffffffu);
    out_scores[i] = __uint_as_float((uint32_t)(sk[i] >> 32));
  }
  if (threadIdx.x == 0) *out_n = k;
}

}  // namespace

int topk_single(ahpp_graph* g, const float* d_score, uint32_t k, uint32_t* d_nodes,
                float* d_scores, uint32_t* d_n, cudaStream_t stream) {
  const uint32_t n = (uint32_t)g->n_u;
  if (k > n) k = n;
  if (k == 0) return cudaMemsetAsync(d_n, 0, 4, stream) == cudaSuccess ? AHPP_OK : AHPP_ECUDA;
  const size_t need = kPasses * kBinsMax * 4 + AHPP_MAX_K * 8 + 16 + sizeof(GridBarrier);
  if (!g->topk_scratch) {
    g->topk_scratch = g->alloc(need);
    if (!g->topk_scratch) { set_error("top-k scratch allocation failed"); return AHPP_ENOMEM; }
    g->topk_scratch_bytes = need;
    AHPP_CUDA(cudaMemset(g->topk_scratch, 0, need));
  }
  char* base = (char*)g->topk_scratch;
  TopkScratch sc;
  sc.hist = (unsigned int*)base;
  sc.cand = (unsigned long long*)(base + kPasses * kBinsMax * 4);
  sc.cand_cnt = (uint32_t*)(base + kPasses * kBinsMax * 4 + AHPP_MAX_K * 8);
  sc.bar = (GridBarrier*)(base + kPasses * kBinsMax * 4 + AHPP_MAX_K * 8 + 16);
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_topk1, kThreads, 0) !=
            cudaSuccess || per_sm <= 0) {
      per_sm = 0;
      set_error("top-k occupancy query failed");
      return AHPP_ECUDA;
    }
  }
  int grid = std::min<int>(per_sm * g->sm_count, (int)((n + kThreads - 1) / kThreads));
  grid = std::max(grid, 1);
  const uint32_t* n2o = g->d_u_new2old;
  void* args[] = {(void*)&d_score, (void*)&n2o, (void*)&n, (void*)&k, (void*)&sc,
                  (void*)&d_nodes, (void*)&d_scores, (void*)&d_n};
  AHPP_CUDA(cudaLaunchCooperativeKernel((const void*)k_topk1, dim3(grid), dim3(kThreads), args, 0,
                                        stream));
  return AHPP_OK;
}

}  // namespace ahpp
