// Single-query persistent push kernel: state and launch parameters.
#pragma once
#include "ahpp_internal.cuh"

namespace ahpp {

// Device state of one query (all arrays indexed by internal ids).
// Block size of the single-query kernel: kQ1Blocks blocks of kQ1Threads per
// SM (64 registers a thread).  Measured on the medium graph: one block of
// 1024 a little faster (34.5 ms a query) than two of 512 (36.1 ms).
constexpr int kQ1Threads = 1024;
constexpr int kQ1Warps = kQ1Threads / 32;
constexpr int kQ1Blocks = 1;
// Default lanes per short row (the fastest on the medium graph: 33.7 ms a
// query against 39.7 / 40.0 / 70.4 for 1 / 8 / 32 lanes, autotuner timings).
constexpr uint32_t kQ1VecWidthDefault = 2;

struct Q1State {
  float *r_u = nullptr, *pi = nullptr, *pic = nullptr;   // residues (sign = marked), reserves, Kahan
  float *t_v = nullptr, *t_a = nullptr;                  // r(v)/d(v), r(a)/W_col(a)
  float* t_a2 = nullptr;                                 // the other t_A buffer (attribute push)
  uint32_t* list_u = nullptr;                            // push rounds: the marked list
  float* split_acc = nullptr;                            // partial sums of split rows
  uint32_t* split_cnt = nullptr;                         // finished chunks of split rows
  QCtl* ctl = nullptr;
  RAcc* racc = nullptr;                                  // [3]
  GridBarrier* bar = nullptr;
  unsigned int* final_maxr_bits = nullptr;               // [2]: max |r_U|, max pi
  uint32_t* trace_frontier = nullptr;                    // [trace_cap] frontier size per round
  float* trace_maxr = nullptr;                           // [trace_cap] max r_U after each round
};

struct Q1Params {
  uint32_t q = 0;              // internal id of the source
  int algo = kAlgoASRP;
  int kahan = 1;
  int switch_rule = 0;
  double eps_f = 0.0;          // ASRP: eps / lambda;  APP: r_max = eps / (|E| + |E_A|)
  double lambda = 1.0;
  double log_inv = 0.0;        // ln(1 / (1 - alpha))
  uint32_t e_tot = 0;          // |E| + |E_A|
  uint32_t max_rounds = 0;
  uint32_t dense_div = 32;     // pull rounds once the frontier covers > 1/dense_div of the edges
  uint32_t n_split = 0;        // split-row slots (phase 1 V + A, phase 2 U)
  uint32_t trace_cap = 0;
  // Pull rounds and shared memory (dynamic, smem_bytes per block):
  //   attr_push: the attribute hop of round t+1 is pushed during round t's
  //     phase 2 into a block-local accumulator over A (shared memory), then
  //     added to the next t_A; otherwise it is pulled in phase 1 over A->U;
  //   ta_smem: phase 2 reads t_A from a shared-memory copy.
  uint32_t smem_bytes = 0;
  int attr_push = 0;
  int ta_smem = 0;
  // short rows of the pull phases: at most vw_max lanes per row (a power of
  // two, 1..32; 1 = one row per lane)
  uint32_t vw_max = 32;
  // Theorem 3 mode: start from r = 1 on every U node, run exactly max_rounds
  // synchronous rounds; the reserves are then pi_T and final_maxr_bits[1]
  // holds max_u pi_T(u).
  int lambda_mode = 0;
  // Algorithm 1 mode: start from r = e_q in the synchronous phase (every
  // positive residue pushed each round) and run exactly max_rounds rounds;
  // the output is then reserves + residues, Algorithm 1's iterate.
  int pi_mode = 0;
};

int launch_query1(const DevGraph& g, const Q1State& s, const Q1Params& p, bool bf16, int grid,
                  cudaStream_t stream);
// Persistent grid of the single-query kernel with smem_bytes of dynamic
// shared memory per block (-1 if it cannot be made resident).
int query1_max_grid(bool bf16, int sm_count, uint32_t smem_bytes);
// Largest dynamic shared memory a block of the single-query kernel may use.
uint32_t query1_max_smem(int device);

}  // namespace ahpp
