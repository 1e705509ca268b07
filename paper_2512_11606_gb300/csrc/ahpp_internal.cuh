// Internal device structures and helpers of the AHPP push library (sm_103a).
//
// Graph layout in HBM (all ids relabeled internally: U, V and A are each
// sorted by degree, largest first, so that hub rows sit together and rows
// of similar length share a warp):
//   CSR_UV  rows u: off[n_u+1], idx v, w(u,v) raw (pull V->U), c_uv (push U->V)
//   CSR_VU  rows v: off[n_v+1], idx u, c_uv (pull U->V), w(u,v) raw (push V->U)
//   CSR_UA  rows u: off[n_u+1], idx a, w(u,a) raw (bf16 or f32)
//   CSC_AU  rows a: off[n_a+1], idx u, w(u,a) raw (bf16 or f32)
//   c_uv(u,v) = (1-alpha)(1-beta) w(u,v) / (d(u) d(v))       (Eq. 1's two factors)
//   rnorm_u[u] = 1 / sum_a w(u,a),  cnorm_a[a] = 1 / sum_u w(u,a)   (Eq. 2)
// One round of Algorithm 3 maps the pushed residues p (marked U nodes) to
//   t_V[v] = sum_u c_uv(u,v) p_u                           = r(v) / d(v)
//   t_A[a] = (1-alpha) beta cnorm_a[a] sum_u w(u,a) rnorm_u[u] p_u = r(a) / W_col(a)
//   r_U'[j] = kept_j + sum_v w(j,v) t_V[v] + sum_a w(j,a) t_A[a]
// either as a pull (gather over the opposite direction, no atomics) or as a
// push (scatter with atomics from the frontier).
//
// Residue encoding: r_u[u] >= 0 is a residue; r_u[u] < 0 marks u as selected
// for the next U-push with residue -r_u[u].  The reserve update
// pi += alpha * p happens when the push is executed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ahpp {

constexpr int kThreads = 256;          // threads per block of every persistent kernel
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kItemLong = 0x40000000u;   // item = one whole long row (warp-cooperative)
constexpr uint32_t kItemSplit = 0x80000000u;  // item = one chunk of a split row (| slot)
constexpr uint32_t kItemMask = 0x3fffffffu;
// Entries per chunk of a long row in the batched pull phases: the unit lists
// of every choice are built at load, ahpp_autotune picks one (default 256).
constexpr int kChunkChoices = 3;
constexpr uint32_t kChunkSizes[kChunkChoices] = {128, 256, 512};
constexpr int kChunkDefault = 1;

// Work items of a pull sweep over one row space.
//   x = first row; y = number of rows (short group, one row per lane) or a flag;
//   z, w = local neighbour range [z, w) for long / split rows.
struct ItemList {
  const uint4* items = nullptr;
  uint32_t n_items = 0;
  uint32_t n_split = 0;                 // split rows
  const uint32_t* split_nchunks = nullptr;
  uint32_t n_long = 0;                  // batched lists: rows [0, n_long) are chunked
};

struct DevGraph {
  uint32_t n_u = 0, n_v = 0, n_a = 0;
  uint32_t n_e = 0, n_ea = 0;
  const uint32_t *uv_off = nullptr, *uv_idx = nullptr;
  const float *uv_w = nullptr, *uv_c = nullptr;
  const uint32_t *vu_off = nullptr, *vu_idx = nullptr;
  const float *vu_c = nullptr, *vu_w = nullptr;
  const uint32_t *ua_off = nullptr, *ua_idx = nullptr;
  const void* ua_w = nullptr;
  const uint32_t *au_off = nullptr, *au_idx = nullptr;
  const void* au_w = nullptr;
  const float* au_c = nullptr;          // A->U pull coefficient w(u,a) / sum_a' w(u,a') (FP32)
  const float* ua_pc = nullptr;         // U->A push coefficient (1-alpha) beta w(u,a) / (sum_a' w(u,a') sum_u' w(u',a))
  const float* rnorm_u = nullptr;
  const float* cnorm_a = nullptr;
  float alpha = 0.f;
  float k_attr = 0.f;                   // (1 - alpha) * beta
  // single-query (one row per lane / warp-cooperative) work items
  ItemList s1_v, s1_a, s1_u;
  // batched row-group units (the active chunk size) and those of every chunk
  // choice (kChunkSizes); b_split_max = the most split slots of any choice
  ItemList b_v, b_a, b_u;
  ItemList b_alt[kChunkChoices][3];
  uint32_t b_chunk = kChunkDefault;
  uint32_t b_split_max = 0;
};

template <typename WA>
__device__ __forceinline__ float wload(const void* p, uint32_t i) {
  return static_cast<float>(static_cast<const WA*>(p)[i]);
}
template <>
__device__ __forceinline__ float wload<__nv_bfloat16>(const void* p, uint32_t i) {
  return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

// ---------------------------------------------------------------- control

enum : int { kPhaseAsync = 0, kPhaseSync = 1, kPhaseDone = 2 };
enum : int { kStatusOk = 0, kStatusCap = 1, kStatusWait = 2, kStatusBadArg = 3 };
// kAlgoAPPS: APP(S), APP's per-node thresholds with ASRP's synchronous switch
// (the ablation arm of Exp-2).
enum : int { kAlgoAPP = 1, kAlgoASRP = 2, kAlgoAPPS = 3 };

// Per-node thresholds r_max (|N(u)| + |A(u)|) in this phase (APP, and APP(S)
// before its switch), else one threshold for every node.
__device__ __forceinline__ bool per_node_threshold(int algo, int phase) {
  return algo == kAlgoAPP || (algo == kAlgoAPPS && phase != kPhaseSync);
}

// Per-query control block (global memory; written by one leader thread,
// mirrored in registers by every thread of a persistent kernel).
struct QCtl {
  double eps;
  double eps_f;        // ASRP: eps / lambda;  APP: r_max = eps / (|E| + |E_A|)
  double lambda;
  uint64_t n_p;        // Algorithm 4's counter
  uint64_t pushes;     // sum of frontier sizes
  uint32_t rounds;
  uint32_t switch_round;
  uint32_t dense_rounds;
  int phase;           // kPhaseAsync / kPhaseSync / kPhaseDone
  int status;          // kStatus*
  int dense;           // next round runs as a pull sweep
  uint32_t q;          // internal id of the source
  uint32_t pad;
  double resid_sum, reserve_sum, max_resid;   // final reductions
};

// Per-round accumulators of one query (triple-buffered by round index).
struct RAcc {
  unsigned int max_r_bits;   // max_u r_U after the round (float bits, values >= 0)
  uint32_t marked;           // nodes marked for the next U-push
  unsigned long long marked_deg;   // sum of |N(u)| + |A(u)| over marked nodes
  unsigned long long np_flush;     // sum of |N(v)| (r(v) > 0) + |A^-1(a)| (r(a) > 0)
  double sum_r;              // sum_u r_U after the round (pull rounds)
  uint32_t n_list_u;               // push rounds: marked list length
  uint32_t pad;
  // APP(S): max_u r(u) / (|N(u)| + |A(u)|) after the round (float bits) and
  // the nodes whose residue exceeds APP's threshold r_max (|N(u)| + |A(u)|)
  unsigned int max_rel_bits;
  uint32_t above;
};

// Software grid barrier for persistent cooperative launches.  Every spin is
// bounded; on expiry the barrier records an error and returns false, and the
// kernel unwinds instead of hanging.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  unsigned int err;
  unsigned int pad;
};

constexpr unsigned int kSpinLimit = 1u << 22;   // x ~256 ns sleep, about one second

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over the blocks [0, nblocks) that share `b`.
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned int nblocks) {
  __shared__ unsigned int s_ok;
  // data written with ordinary stores before the barrier may be read by TMA
  // (the async proxy) after it
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int ok = 1;
    unsigned int g = ld_acquire_u32(&b->gen);
    __threadfence();
    unsigned int arrived = atomicAdd(&b->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      unsigned int spins = 0;
      while (ld_acquire_u32(&b->gen) == g) {
        if (++spins > kSpinLimit) { atomicOr(&b->err, 1u); ok = 0; break; }
        if ((spins & 255u) == 0 && ld_acquire_u32(&b->err)) { ok = 0; break; }
        __nanosleep(256);
      }
    }
    __threadfence();
    if (ld_acquire_u32(&b->err)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return s_ok != 0;
}

// ------------------------------------------------------------ reductions

// Radix-select step on a histogram in shared memory (bins a power of two >= 32):
// the largest digit d such that the keys in buckets above d plus hist[d]
// reach krem.  Warp-collective: lane L sums bins [L*bins/32, (L+1)*bins/32),
// a suffix sum over the lanes and a ballot find the lane holding the
// crossing, and that lane walks its own bins.  Every lane receives d, cum
// (keys in the buckets above d) and h = hist[d].
__device__ __forceinline__ void radix_pick(const unsigned int* hist, int bins, uint32_t krem, int* d_out,
                                           uint32_t* cum_out, uint32_t* h_out) {
  const int lane = threadIdx.x & 31;
  const int per = bins >> 5;
  const unsigned int* mine = hist + lane * per;
  uint32_t sum = 0;
  for (int j = 0; j < per; ++j) sum += mine[(j + lane) & (per - 1)];   // rotated: fewer bank conflicts
  uint32_t suf = sum;                                   // keys in lanes >= lane
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_down_sync(0xffffffffu, suf, o);
    if (lane + o < 32) suf += t;
  }
  const unsigned int ball = __ballot_sync(0xffffffffu, suf >= krem);
  const int L = ball ? 31 - __clz(ball) : 0;
  int d = 0;
  uint32_t cum = 0, h = 0;
  if (lane == L) {
    cum = suf - sum;                                    // keys in the lanes above L
    int j = per - 1;
    for (; j >= 0; --j) {
      h = mine[j];
      if (cum + h >= krem || j == 0) break;
      cum += h;
    }
    d = L * per + j;
  }
  *d_out = __shfl_sync(0xffffffffu, d, L);
  *cum_out = __shfl_sync(0xffffffffu, cum, L);
  *h_out = __shfl_sync(0xffffffffu, h, L);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Thread-local partials of one query, reduced per block then atomically.
struct Partials {
  float max_r = 0.f;
  uint32_t marked = 0;
  unsigned long long marked_deg = 0;
  unsigned long long np_flush = 0;
  double sum_r = 0.0;
  float max_rel = 0.f;       // APP(S) statistics (see RAcc)
  uint32_t above = 0;
};

// Block reduction of Partials into acc (one atomic per field per block);
// NW = warps per block; APPS: also APP(S)'s max_rel and above.
template <int NW, bool APPS = false>
__device__ __forceinline__ void flush_partials(Partials& p, RAcc* acc) {
  __shared__ float s_max[NW];
  __shared__ uint32_t s_marked[NW];
  __shared__ unsigned long long s_deg[NW], s_np[NW];
  __shared__ double s_sum[NW];
  __shared__ float s_rel[NW];
  __shared__ uint32_t s_above[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float m = warp_max(p.max_r);
  uint32_t mk = warp_sum_u32(p.marked);
  unsigned long long dg = warp_sum_u64(p.marked_deg);
  unsigned long long np = warp_sum_u64(p.np_flush);
  double sm = warp_sum_d(p.sum_r);
  float rel = APPS ? warp_max(p.max_rel) : 0.f;
  uint32_t ab = APPS ? warp_sum_u32(p.above) : 0u;
  if (lane == 0) {
    s_max[warp] = m; s_marked[warp] = mk; s_deg[warp] = dg; s_np[warp] = np; s_sum[warp] = sm;
    s_rel[warp] = rel; s_above[warp] = ab;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NW; ++w) {
      m = fmaxf(m, s_max[w]); mk += s_marked[w]; dg += s_deg[w]; np += s_np[w]; sm += s_sum[w];
      if (APPS) { rel = fmaxf(rel, s_rel[w]); ab += s_above[w]; }
    }
    if (APPS && rel > 0.f) atomicMax(&acc->max_rel_bits, __float_as_uint(rel));
    if (APPS && ab) atomicAdd(&acc->above, ab);
    if (m > 0.f) atomicMax(&acc->max_r_bits, __float_as_uint(m));
    if (mk) atomicAdd(&acc->marked, mk);
    if (dg) atomicAdd(&acc->marked_deg, dg);
    if (np) atomicAdd(&acc->np_flush, np);
    if (sm != 0.0) atomicAdd(&acc->sum_r, sm);
  }
  __syncthreads();
  p = Partials();
}

// Kahan-compensated accumulation s += v with compensation c (FP32).
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  float y = v - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

}  // namespace ahpp
