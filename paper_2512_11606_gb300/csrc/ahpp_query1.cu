// Single-query push on the whole GPU: one persistent cooperative launch runs
// every round of APP (Algorithm 3) or ASRP (Algorithm 4) for one source.
//
// A round is either
//   * a push round (small frontier): U-push of the marked list with atomic
//     scatter into t_V / t_A (the U-push of Algorithm 3), then the flush of
//     every touched V node and attribute (its V and attribute steps) into
//     r_U, then the selection of the next frontier (warp-ballot compaction);
//   * a pull round (large frontier, the synchronous sweep of Algorithm 4):
//     phase 1 gathers t_V / t_A from the marked residues over V->U and A->U
//     adjacency, phase 2 gathers r_U' over U->V and U->A adjacency, applies
//     the reserve update of the pushed nodes and marks the next frontier.
// Both forms compute the same linear map of one round.  Rounds switch from
// push to pull when the frontier covers more than 1/dense_div of the edges.
// All control (termination, the ASRP switch test, the push/pull choice) is
// decided on the device from FP64/uint64 round accumulators.
#include "ahpp_internal.cuh"
#include "ahpp_query1.cuh"

namespace ahpp {

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Warp-aggregated append of `val` for the lanes where `pred` holds.
__device__ __forceinline__ void warp_append(bool pred, uint32_t val, uint32_t* list,
                                            uint32_t* counter) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  uint32_t lane = lane_id();
  uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

struct Ctx {
  const DevGraph& g;   // references into the kernel's __grid_constant__ parameters
  const Q1State& s;
  const Q1Params& p;
  uint32_t gw, nw;     // global warp id / count
  uint32_t gt, nt;     // global thread id / count
};

__device__ __forceinline__ float pushed(const float* r_u, uint32_t u) {
  return fmaxf(-r_u[u], 0.f);
}

// ---------------------------------------------------------------- phase 1
// t_V[v] = sum_u c_uv p_u ;  t_A[a] = k_attr cnorm_a[a] sum_u w(u,a) rnorm_u[u] p_u

__device__ __forceinline__ void p1_epilogue(const Ctx& c, bool is_a, uint32_t row, float s,
                                            Partials& part) {
  if (!is_a) {
    c.s.t_v[row] = s;
    if (s > 0.f) part.np_flush += c.g.vu_off[row + 1] - c.g.vu_off[row];
  } else {
    float t = c.g.k_attr * c.g.cnorm_a[row] * s;
    c.s.t_a[row] = t;
    if (t > 0.f) part.np_flush += c.g.au_off[row + 1] - c.g.au_off[row];
  }
}

template <typename WA>
__device__ void phase1(const Ctx& c, Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  const uint32_t nv = g.s1_v.n_items, total = nv + g.s1_a.n_items;
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const bool is_a = it >= nv;
    const uint4 item = is_a ? g.s1_a.items[it - nv] : g.s1_v.items[it];
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    const uint32_t* idx = is_a ? g.au_idx : g.vu_idx;
    if (item.y & (kItemLong | kItemSplit)) {
      const uint32_t row = item.x, base = off[row];
      float s = 0.f;
      if (!is_a) {
        for (uint32_t k = item.z + lane; k < item.w; k += 32) {
          uint32_t u = idx[base + k];
          s = fmaf(g.vu_c[base + k], pushed(c.s.r_u, u), s);
        }
      } else {
        for (uint32_t k = item.z + lane; k < item.w; k += 32) {
          uint32_t u = idx[base + k];
          s = fmaf(wload<WA>(g.au_w, base + k) * g.rnorm_u[u], pushed(c.s.r_u, u), s);
        }
      }
      s = warp_sum(s);
      if (lane == 0) {
        if (item.y & kItemSplit) {
          const uint32_t slot = (item.y & kItemMask) + (is_a ? g.s1_v.n_split : 0);
          const uint32_t nch = is_a ? g.s1_a.split_nchunks[item.y & kItemMask]
                                    : g.s1_v.split_nchunks[item.y & kItemMask];
          atomicAdd(&c.s.split_acc[slot], s);
          __threadfence();
          if (atomicAdd(&c.s.split_cnt[slot], 1u) == nch - 1) {
            float tot = atomicExch(&c.s.split_acc[slot], 0.f);
            c.s.split_cnt[slot] = 0;
            p1_epilogue(c, is_a, row, tot, part);
          }
        } else {
          p1_epilogue(c, is_a, row, s, part);
        }
      }
    } else if (lane < item.y) {
      const uint32_t row = item.x + lane;
      const uint32_t b = off[row], e = off[row + 1];
      float s = 0.f;
      if (!is_a) {
        for (uint32_t k = b; k < e; ++k) s = fmaf(g.vu_c[k], pushed(c.s.r_u, idx[k]), s);
      } else {
        for (uint32_t k = b; k < e; ++k) {
          uint32_t u = idx[k];
          s = fmaf(wload<WA>(g.au_w, k) * g.rnorm_u[u], pushed(c.s.r_u, u), s);
        }
      }
      p1_epilogue(c, is_a, row, s, part);
    }
  }
}

// ---------------------------------------------------------------- phase 2
// r_U'[u] = kept_u + sum_v w(u,v) t_V[v] + sum_a w(u,a) t_A[a]; reserve update of
// the nodes pushed this round; marking of the next frontier with threshold th.

__device__ __forceinline__ void p2_epilogue(const Ctx& c, uint32_t u, float s, uint32_t cnt,
                                            double theta, bool per_node, Partials& part) {
  float r_old = c.s.r_u[u];
  float kept = r_old;
  if (r_old < 0.f) {
    const float add = c.g.alpha * (-r_old);
    if (c.p.kahan) {
      float pv = c.s.pi[u], pc = c.s.pic[u];
      kahan_add(pv, pc, add);
      c.s.pi[u] = pv; c.s.pic[u] = pc;
    } else {
      c.s.pi[u] += add;
    }
    kept = 0.f;
  }
  const float r_new = kept + s;
  part.max_r = fmaxf(part.max_r, r_new);
  part.sum_r += (double)r_new;
  const double th = per_node ? theta * (double)cnt : theta;
  if ((double)r_new > th) {
    c.s.r_u[u] = -r_new;
    part.marked += 1;
    part.marked_deg += cnt;
  } else {
    c.s.r_u[u] = r_new;
  }
}

template <typename WA>
__device__ void phase2(const Ctx& c, double theta, bool per_node, Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  const uint32_t total = g.s1_u.n_items;
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const uint4 item = g.s1_u.items[it];
    if (item.y & (kItemLong | kItemSplit)) {
      const uint32_t u = item.x;
      const uint32_t b1 = g.uv_off[u], dv = g.uv_off[u + 1] - b1;
      const uint32_t b2 = g.ua_off[u], da = g.ua_off[u + 1] - b2;
      float s = 0.f;
      for (uint32_t k = item.z + lane; k < item.w; k += 32) {
        if (k < dv) {
          s = fmaf(g.uv_w[b1 + k], c.s.t_v[g.uv_idx[b1 + k]], s);
        } else {
          uint32_t j = b2 + (k - dv);
          s = fmaf(wload<WA>(g.ua_w, j), c.s.t_a[g.ua_idx[j]], s);
        }
      }
      s = warp_sum(s);
      if (lane == 0) {
        if (item.y & kItemSplit) {
          const uint32_t slot = (item.y & kItemMask) + g.s1_v.n_split + g.s1_a.n_split;
          const uint32_t nch = g.s1_u.split_nchunks[item.y & kItemMask];
          atomicAdd(&c.s.split_acc[slot], s);
          __threadfence();
          if (atomicAdd(&c.s.split_cnt[slot], 1u) == nch - 1) {
            float tot = atomicExch(&c.s.split_acc[slot], 0.f);
            c.s.split_cnt[slot] = 0;
            p2_epilogue(c, u, tot, dv + da, theta, per_node, part);
          }
        } else {
          p2_epilogue(c, u, s, dv + da, theta, per_node, part);
        }
      }
    } else if (lane < item.y) {
      const uint32_t u = item.x + lane;
      const uint32_t b1 = g.uv_off[u], e1 = g.uv_off[u + 1];
      const uint32_t b2 = g.ua_off[u], e2 = g.ua_off[u + 1];
      float s = 0.f;
      for (uint32_t k = b1; k < e1; ++k) s = fmaf(g.uv_w[k], c.s.t_v[g.uv_idx[k]], s);
      for (uint32_t k = b2; k < e2; ++k) s = fmaf(wload<WA>(g.ua_w, k), c.s.t_a[g.ua_idx[k]], s);
      p2_epilogue(c, u, s, (e1 - b1) + (e2 - b2), theta, per_node, part);
    }
  }
}

// --------------------------------------------------------- push (sparse)

template <typename WA>
__device__ void push_u(const Ctx& c, uint32_t n_list, RAcc* acc) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  for (uint32_t i = c.gw; i < n_list; i += c.nw) {
    const uint32_t u = c.s.list_u[i];
    float r = 0.f;
    if (lane == 0) r = c.s.r_u[u];
    r = __shfl_sync(0xffffffffu, r, 0);
    const float p = fmaxf(-r, 0.f);
    if (lane == 0) {
      c.s.r_u[u] = 0.f;
      const float add = c.g.alpha * p;
      if (c.p.kahan) {
        float pv = c.s.pi[u], pc = c.s.pic[u];
        kahan_add(pv, pc, add);
        c.s.pi[u] = pv; c.s.pic[u] = pc;
      } else {
        c.s.pi[u] += add;
      }
    }
    const uint32_t b1 = g.uv_off[u], e1 = g.uv_off[u + 1];
    for (uint32_t k0 = b1; k0 < e1; k0 += 32) {
      const uint32_t k = k0 + lane;
      const bool ok = k < e1;
      uint32_t v = 0;
      bool first = false;
      if (ok) {
        v = g.uv_idx[k];
        first = atomicAdd(&c.s.t_v[v], g.uv_c[k] * p) == 0.f;
      }
      warp_append(first, v, c.s.list_v, &acc->n_list_v);
    }
    const float ka = g.k_attr * g.rnorm_u[u] * p;
    const uint32_t b2 = g.ua_off[u], e2 = g.ua_off[u + 1];
    for (uint32_t k0 = b2; k0 < e2; k0 += 32) {
      const uint32_t k = k0 + lane;
      const bool ok = k < e2;
      uint32_t a = 0;
      bool first = false;
      if (ok) {
        a = g.ua_idx[k];
        first = atomicAdd(&c.s.t_a[a], wload<WA>(g.ua_w, k) * ka * g.cnorm_a[a]) == 0.f;
      }
      warp_append(first, a, c.s.list_a, &acc->n_list_a);
    }
  }
}

template <typename WA>
__device__ void flush_va(const Ctx& c, uint32_t nv, uint32_t na, Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  for (uint32_t i = c.gw; i < nv + na; i += c.nw) {
    const bool is_a = i >= nv;
    const uint32_t x = is_a ? c.s.list_a[i - nv] : c.s.list_v[i];
    float* t = is_a ? c.s.t_a : c.s.t_v;
    float val = 0.f;
    if (lane == 0) val = t[x];
    val = __shfl_sync(0xffffffffu, val, 0);
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    const uint32_t* idx = is_a ? g.au_idx : g.vu_idx;
    const uint32_t b = off[x], e = off[x + 1];
    if (lane == 0) {
      t[x] = 0.f;
      part.np_flush += e - b;
    }
    for (uint32_t k = b + lane; k < e; k += 32) {
      const float w = is_a ? wload<WA>(g.au_w, k) : g.vu_w[k];
      const float add = w * val;
      const float old = atomicAdd(&c.s.r_u[idx[k]], add);
      part.max_r = fmaxf(part.max_r, old + add);
    }
  }
}

// Marking of the next frontier in a push round: r_U > th (per_node: th * cnt(u)).
__device__ void select_frontier(const Ctx& c, double theta, bool per_node, RAcc* acc,
                                Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t n = g.n_u;
  // every warp iterates the same number of times so the ballot is warp-uniform
  const uint32_t span = (n + 31) / 32 * 32;
  for (uint32_t u0 = c.gw * 32; u0 < span; u0 += c.nw * 32) {
    const uint32_t u = u0 + lane_id();
    bool m = false;
    uint32_t cnt = 0;
    float r = 0.f;
    if (u < n) {
      r = c.s.r_u[u];
      if (per_node) {
        cnt = (g.uv_off[u + 1] - g.uv_off[u]) + (g.ua_off[u + 1] - g.ua_off[u]);
        m = (double)r > theta * (double)cnt;
      } else {
        m = (double)r > theta;
        if (m) cnt = (g.uv_off[u + 1] - g.uv_off[u]) + (g.ua_off[u + 1] - g.ua_off[u]);
      }
      if (m) {
        c.s.r_u[u] = -r;
        part.marked += 1;
        part.marked_deg += cnt;
      }
    }
    warp_append(m, u, c.s.list_u, &acc->n_list_u);
  }
}

// At the ASRP switch the speculative marks of a pull round used eps_f; the
// first synchronous round pushes every positive residue, so mark the rest.
__device__ void mark_remaining(const Ctx& c, Partials& part) {
  const DevGraph& g = c.g;
  for (uint32_t u = c.gt; u < g.n_u; u += c.nt) {
    const float r = c.s.r_u[u];
    if (r > 0.f) {
      c.s.r_u[u] = -r;
      part.marked += 1;
      part.marked_deg += (g.uv_off[u + 1] - g.uv_off[u]) + (g.ua_off[u + 1] - g.ua_off[u]);
    }
  }
}

__device__ __forceinline__ double budget_of(const Q1Params& p, double M) {
  const double EE = (double)p.e_tot;
  if (p.switch_rule == 2) return INFINITY;
  if (p.switch_rule == 1) return 2.0 * EE * (log(1.0 / (p.lambda * M)) / p.log_inv);
  return 2.0 * EE * fmax(0.0, log(M / p.eps_f) / p.log_inv);
}

}  // namespace

template <typename WA>
__global__ void __launch_bounds__(kThreads)
k_query1(const __grid_constant__ DevGraph g, const __grid_constant__ Q1State s,
         const __grid_constant__ Q1Params p) {
  Ctx c{g, s, p, (blockIdx.x * kThreads + threadIdx.x) >> 5, (gridDim.x * kThreads) >> 5,
        blockIdx.x * kThreads + threadIdx.x, gridDim.x * kThreads};
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const unsigned int nb = gridDim.x;
  const bool app = p.algo == kAlgoAPP;

  // ---- init: zero the state, mark the source (the initial state of Algorithm 3)
  const float r0 = p.lambda_mode ? -1.f : 0.f;
  for (uint32_t u = c.gt; u < g.n_u; u += c.nt) { s.r_u[u] = r0; s.pi[u] = 0.f; s.pic[u] = 0.f; }
  for (uint32_t v = c.gt; v < g.n_v; v += c.nt) s.t_v[v] = 0.f;
  for (uint32_t a = c.gt; a < g.n_a; a += c.nt) s.t_a[a] = 0.f;
  for (uint32_t i = c.gt; i < p.n_split; i += c.nt) { s.split_acc[i] = 0.f; s.split_cnt[i] = 0; }
  if (c.gt < 3) s.racc[c.gt] = RAcc{};
  if (leader) {
    s.ctl->reserve_sum = 0.0;
    s.ctl->resid_sum = 0.0;
    s.final_maxr_bits[0] = 0u;
    s.final_maxr_bits[1] = 0u;
  }
  // a barrier that gives up here skips the rounds; the leader still reports
  // the status below, so the host never reads a previous call's control block
  bool init_ok = grid_sync(s.bar, nb);
  if (!init_ok) {
  } else if (leader && p.lambda_mode) {
    RAcc* a0 = &s.racc[2];
    a0->marked = g.n_u;
    a0->marked_deg = p.e_tot;
  } else if (leader) {
    const uint32_t cnt = (g.uv_off[p.q + 1] - g.uv_off[p.q]) + (g.ua_off[p.q + 1] - g.ua_off[p.q]);
    const double th = app ? p.eps_f * (double)cnt : p.eps_f;
    RAcc* a0 = &s.racc[2];
    if (1.0 > th) {
      s.r_u[p.q] = -1.f;
      a0->marked = 1;
      a0->marked_deg = cnt;
      a0->n_list_u = 1;
      s.list_u[0] = p.q;
    } else {
      s.r_u[p.q] = 1.f;
    }
  }
  if (init_ok) init_ok = grid_sync(s.bar, nb);

  int phase = (p.lambda_mode || p.pi_mode) ? kPhaseSync : kPhaseAsync;
  int status = init_ok ? kStatusOk : kStatusWait;
  int dense = p.lambda_mode ? 1 : 0;
  uint32_t rounds = 0, switch_round = 0, dense_rounds = 0;
  unsigned long long n_p = 0, pushes = 0;
  Partials part;

  for (; status == kStatusOk;) {
    RAcc* A = &s.racc[rounds % 3];
    const RAcc* P = &s.racc[(rounds + 2) % 3];
    const uint32_t marked = __ldcg(&P->marked);
    const unsigned long long marked_deg = __ldcg(&P->marked_deg);
    if (phase == kPhaseDone || marked == 0) { phase = kPhaseDone; break; }
    if (rounds >= p.max_rounds) { status = kStatusCap; break; }
    if (leader) s.racc[(rounds + 1) % 3] = RAcc{};
    if (!dense && marked_deg * (unsigned long long)p.dense_div > (unsigned long long)p.e_tot) dense = 1;
    if (p.trace_cap && leader && rounds < p.trace_cap) s.trace_frontier[rounds] = marked;
    pushes += marked;
    const double theta = app ? p.eps_f : (phase == kPhaseSync ? 0.0 : p.eps_f);

    if (!dense) {
      push_u<WA>(c, marked, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      const uint32_t nv = __ldcg(&A->n_list_v), na = __ldcg(&A->n_list_a);
      flush_va<WA>(c, nv, na, part);
      flush_partials(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
    } else {
      phase1<WA>(c, part);
      flush_partials(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      phase2<WA>(c, theta, app, part);
      flush_partials(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      ++dense_rounds;
    }
    ++rounds;

    // ---- decision (every thread computes the same result)
    const float M = __uint_as_float(__ldcg(&A->max_r_bits));
    n_p += marked_deg + __ldcg(&A->np_flush);
    if (p.trace_cap && leader && rounds - 1 < p.trace_cap) s.trace_maxr[rounds - 1] = M;
    bool switched = false;
    if (!app) {
      if ((double)M <= p.eps_f) {
        phase = kPhaseDone;
      } else if (phase == kPhaseAsync && (double)n_p >= budget_of(p, (double)M)) {
        phase = kPhaseSync;
        switch_round = rounds + 1;
        switched = true;
      }
    }
    if (phase == kPhaseDone) break;
    if (!dense) {
      const double th_next = app ? p.eps_f : (phase == kPhaseSync ? 0.0 : p.eps_f);
      select_frontier(c, th_next, app, A, part);
      flush_partials(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
    } else if (switched) {
      mark_remaining(c, part);
      flush_partials(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
    }
  }

  // ---- final: reserves pi - compensation, FP64 sums of reserves and residues
  if (status != kStatusWait) {
    double sp = 0.0, sr = 0.0;
    float mr = 0.f, mp = 0.f;
    for (uint32_t u = c.gt; u < g.n_u; u += c.nt) {
      const float v = fmaxf(s.pi[u] - s.pic[u], 0.f);
      const float r = fabsf(s.r_u[u]);
      s.pi[u] = p.pi_mode ? v + r : v;
      s.pic[u] = 0.f;
      sp += v; sr += r; mr = fmaxf(mr, r); mp = fmaxf(mp, v);
    }
    sp = warp_sum_d(sp); sr = warp_sum_d(sr); mr = warp_max(mr); mp = warp_max(mp);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&s.ctl->reserve_sum, sp);
      atomicAdd(&s.ctl->resid_sum, sr);
      atomicMax(&s.final_maxr_bits[0], __float_as_uint(mr));
      atomicMax(&s.final_maxr_bits[1], __float_as_uint(mp));
    }
  }
  if (leader) {
    s.ctl->n_p = n_p;
    s.ctl->pushes = pushes;
    s.ctl->rounds = rounds;
    s.ctl->switch_round = switch_round;
    s.ctl->dense_rounds = dense_rounds;
    s.ctl->phase = phase;
    s.ctl->status = (status == kStatusOk && phase != kPhaseDone) ? kStatusCap : status;
  }
}

template __global__ void k_query1<float>(const __grid_constant__ DevGraph,
                                         const __grid_constant__ Q1State,
                                         const __grid_constant__ Q1Params);
template __global__ void k_query1<__nv_bfloat16>(const __grid_constant__ DevGraph,
                                                 const __grid_constant__ Q1State,
                                                 const __grid_constant__ Q1Params);

// Launch helper: persistent cooperative grid sized to full residency.
int launch_query1(const DevGraph& g, const Q1State& s, const Q1Params& p, bool bf16,
                  int grid, cudaStream_t stream) {
  void* args[] = {(void*)&g, (void*)&s, (void*)&p};
  cudaError_t e;
  if (bf16)
    e = cudaLaunchCooperativeKernel((const void*)k_query1<__nv_bfloat16>, dim3(grid),
                                    dim3(kThreads), args, 0, stream);
  else
    e = cudaLaunchCooperativeKernel((const void*)k_query1<float>, dim3(grid), dim3(kThreads),
                                    args, 0, stream);
  return e == cudaSuccess ? 0 : (int)e;
}

int query1_max_grid(bool bf16, int sm_count) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, bf16 ? (const void*)k_query1<__nv_bfloat16> : (const void*)k_query1<float>,
      kThreads, 0);
  if (e != cudaSuccess || per_sm <= 0) return -1;
  return per_sm * sm_count;
}

}  // namespace ahpp
