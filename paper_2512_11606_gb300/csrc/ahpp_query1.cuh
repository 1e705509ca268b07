// Single-query persistent push kernel: state and launch parameters.
#pragma once
#include "ahpp_internal.cuh"

namespace ahpp {

// Device state of one query (all arrays indexed by internal ids).
struct Q1State {
  float *r_u = nullptr, *pi = nullptr, *pic = nullptr;   // residues (sign = marked), reserves, Kahan
  float *t_v = nullptr, *t_a = nullptr;                  // r(v)/d(v), r(a)/W_col(a)
  uint32_t *list_u = nullptr, *list_v = nullptr, *list_a = nullptr;   // push-round lists
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
int query1_max_grid(bool bf16, int sm_count);

}  // namespace ahpp
