// Batched multi-source APP / ASRP: one persistent cooperative launch runs n
// queries packed into tiles of kTile (one query per lane).  Every round of a
// tile is a pull sweep over the whole graph (the synchronous form of
// Algorithm 3's three loops): phase 1 gathers t_V / t_A for all 32 queries
// from the marked residues, phase 2 gathers the new residues, applies the
// reserve update of the pushed nodes and marks the next frontier of each
// query with its own threshold.  Per-query control (termination, the ASRP
// switch test of Algorithm 4) is kept per lane; a query that finishes is
// frozen while the rest of its tile continues, so its result does not depend
// on the other queries of the tile.  Top-k per query is a per-lane radix
// select over (score, caller id) keys.
#include "ahpp_batch.cuh"

namespace ahpp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct BCtx {
  const DevGraph& g;
  const TileBuf& t;
  const BatchParams& p;
  uint32_t gw, nw;     // warp id / count within the group
  uint32_t gt, nt;     // thread id / count within the group
  uint32_t lane;
};

// Per-lane block reduction of Partials into acc[lane].
__device__ __forceinline__ void flush_lane_partials(Partials& p, RAcc* acc) {
  __shared__ float s_max[kWarps][32];
  __shared__ uint32_t s_mk[kWarps][32];
  __shared__ unsigned long long s_dg[kWarps][32], s_np[kWarps][32];
  __shared__ double s_sum[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_max[warp][lane] = p.max_r; s_mk[warp][lane] = p.marked; s_dg[warp][lane] = p.marked_deg;
  s_np[warp][lane] = p.np_flush; s_sum[warp][lane] = p.sum_r;
  __syncthreads();
  if (warp == 0) {
    float m = s_max[0][lane];
    uint32_t mk = s_mk[0][lane];
    unsigned long long dg = s_dg[0][lane], np = s_np[0][lane];
    double sm = s_sum[0][lane];
    for (int w = 1; w < kWarps; ++w) {
      m = fmaxf(m, s_max[w][lane]); mk += s_mk[w][lane]; dg += s_dg[w][lane];
      np += s_np[w][lane]; sm += s_sum[w][lane];
    }
    RAcc* a = &acc[lane];
    if (m > 0.f) atomicMax(&a->max_r_bits, __float_as_uint(m));
    if (mk) atomicAdd(&a->marked, mk);
    if (dg) atomicAdd(&a->marked_deg, dg);
    if (np) atomicAdd(&a->np_flush, np);
    if (sm != 0.0) atomicAdd(&a->sum_r, sm);
  }
  __syncthreads();
  p = Partials();
}

// sum_k coef[k] * max(-x[idx[k]][lane], 0) over [b, e): marked residues.
__device__ __forceinline__ float dot_pushed(const uint32_t* __restrict__ idx,
                                            const float* __restrict__ coef, uint32_t b, uint32_t e,
                                            const float* __restrict__ x, uint32_t lane) {
  float s = 0.f;
  for (uint32_t k0 = b; k0 < e; k0 += 32) {
    const uint32_t n = min(32u, e - k0);
    uint32_t mi = 0;
    float mc = 0.f;
    if (lane < n) { mi = idx[k0 + lane]; mc = coef[k0 + lane]; }
#pragma unroll 8
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t u = __shfl_sync(kFull, mi, j);
      const float cc = __shfl_sync(kFull, mc, j);
      s = fmaf(cc, fmaxf(-x[(size_t)u * kTile + lane], 0.f), s);
    }
  }
  return s;
}

// Same for attribute rows: coefficient w(u,a) * rnorm_u[u].
template <typename WA>
__device__ __forceinline__ float dot_pushed_attr(const DevGraph& g, uint32_t b, uint32_t e,
                                                 const float* __restrict__ x, uint32_t lane) {
  float s = 0.f;
  for (uint32_t k0 = b; k0 < e; k0 += 32) {
    const uint32_t n = min(32u, e - k0);
    uint32_t mi = 0;
    float mc = 0.f;
    if (lane < n) {
      mi = g.au_idx[k0 + lane];
      mc = wload<WA>(g.au_w, k0 + lane) * g.rnorm_u[mi];
    }
#pragma unroll 8
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t u = __shfl_sync(kFull, mi, j);
      const float cc = __shfl_sync(kFull, mc, j);
      s = fmaf(cc, fmaxf(-x[(size_t)u * kTile + lane], 0.f), s);
    }
  }
  return s;
}

// sum_k w[k] * x[idx[k]][lane] over [b, e).
template <typename W>
__device__ __forceinline__ float dot_plain(const uint32_t* __restrict__ idx, const void* w,
                                           uint32_t b, uint32_t e, const float* __restrict__ x,
                                           uint32_t lane) {
  float s = 0.f;
  for (uint32_t k0 = b; k0 < e; k0 += 32) {
    const uint32_t n = min(32u, e - k0);
    uint32_t mi = 0;
    float mc = 0.f;
    if (lane < n) { mi = idx[k0 + lane]; mc = wload<W>(w, k0 + lane); }
#pragma unroll 8
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t v = __shfl_sync(kFull, mi, j);
      const float cc = __shfl_sync(kFull, mc, j);
      s = fmaf(cc, x[(size_t)v * kTile + lane], s);
    }
  }
  return s;
}

// Split-row combine: returns true (warp-uniform) for the chunk that finishes
// the row, with the row total in *tot.
__device__ __forceinline__ bool split_combine(const TileBuf& t, uint32_t slot, uint32_t nch,
                                              float s, uint32_t lane, float* tot) {
  atomicAdd(&t.split_acc[(size_t)slot * kTile + lane], s);
  __threadfence();
  __syncwarp();
  uint32_t last = 0;
  if (lane == 0) last = atomicAdd(&t.split_cnt[slot], 1u) == nch - 1;
  last = __shfl_sync(kFull, last, 0);
  if (last) {
    __threadfence();
    *tot = atomicExch(&t.split_acc[(size_t)slot * kTile + lane], 0.f);
    if (lane == 0) t.split_cnt[slot] = 0;
  }
  return last != 0;
}

// Phase 1: t_V and t_A for the 32 queries of the tile.
template <typename WA>
__device__ __forceinline__ void bphase1(const BCtx& c, Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane;
  const uint32_t nv = g.b_v.n_items, total = nv + g.b_a.n_items;
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const bool is_a = it >= nv;
    const uint4 item = is_a ? g.b_a.items[it - nv] : g.b_v.items[it];
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    uint32_t r0, r1;
    if (item.y & (kItemLong | kItemSplit)) { r0 = item.x; r1 = item.x + 1; }
    else { r0 = item.x; r1 = item.x + item.y; }
    for (uint32_t row = r0; row < r1; ++row) {
      uint32_t b = off[row], e = off[row + 1];
      if (item.y & (kItemLong | kItemSplit)) { e = b + item.w; b = b + item.z; }
      float s = is_a ? dot_pushed_attr<WA>(g, b, e, c.t.r_u, lane)
                     : dot_pushed(g.vu_idx, g.vu_c, b, e, c.t.r_u, lane);
      if (item.y & kItemSplit) {
        const uint32_t sl = item.y & kItemMask;
        const uint32_t slot = sl + (is_a ? g.b_v.n_split : 0);
        const uint32_t nch = is_a ? g.b_a.split_nchunks[sl] : g.b_v.split_nchunks[sl];
        float tot;
        if (!split_combine(c.t, slot, nch, s, lane, &tot)) continue;
        s = tot;
      }
      if (!is_a) {
        c.t.t_v[(size_t)row * kTile + lane] = s;
        if (s > 0.f) part.np_flush += g.vu_off[row + 1] - g.vu_off[row];
      } else {
        const float tv = g.k_attr * g.cnorm_a[row] * s;
        c.t.t_a[(size_t)row * kTile + lane] = tv;
        if (tv > 0.f) part.np_flush += g.au_off[row + 1] - g.au_off[row];
      }
    }
  }
}

struct LaneCtl {
  double eps_f;
  unsigned long long n_p, pushes;
  uint32_t rounds, switch_round;
  int phase, status, active;
};

__device__ __forceinline__ void bepilogue2(const BCtx& c, const LaneCtl& L, uint32_t u, float s,
                                           uint32_t cnt, Partials& part) {
  if (!L.active) return;
  const size_t i = (size_t)u * kTile + c.lane;
  const float r_old = c.t.r_u[i];
  float kept = r_old;
  if (r_old < 0.f) {
    const float add = c.g.alpha * (-r_old);
    if (c.p.kahan) {
      float pv = c.t.pi[i], pc = c.t.pic[i];
      kahan_add(pv, pc, add);
      c.t.pi[i] = pv; c.t.pic[i] = pc;
    } else {
      c.t.pi[i] += add;
    }
    kept = 0.f;
  }
  const float r_new = kept + s;
  part.max_r = fmaxf(part.max_r, r_new);
  part.sum_r += (double)r_new;
  double th;
  if (c.p.algo == kAlgoAPP) th = L.eps_f * (double)cnt;
  else th = (L.phase == kPhaseSync) ? 0.0 : L.eps_f;
  if ((double)r_new > th) {
    c.t.r_u[i] = -r_new;
    part.marked += 1;
    part.marked_deg += cnt;
  } else {
    c.t.r_u[i] = r_new;
  }
}

// Phase 2: new residues of every U node for the 32 queries.
template <typename WA>
__device__ __forceinline__ void bphase2(const BCtx& c, const LaneCtl& L, Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane;
  for (uint32_t it = c.gw; it < g.b_u.n_items; it += c.nw) {
    const uint4 item = g.b_u.items[it];
    if (item.y & (kItemLong | kItemSplit)) {
      const uint32_t u = item.x;
      const uint32_t b1 = g.uv_off[u], dv = g.uv_off[u + 1] - b1;
      const uint32_t b2 = g.ua_off[u], da = g.ua_off[u + 1] - b2;
      // chunk [z, w) of the combined list (V neighbours, then attributes)
      float s = 0.f;
      const uint32_t z = item.z, w = item.w;
      if (z < dv) s += dot_plain<float>(g.uv_idx, g.uv_w, b1 + z, b1 + min(w, dv), c.t.t_v, lane);
      if (w > dv)
        s += dot_plain<WA>(g.ua_idx, g.ua_w, b2 + (z > dv ? z - dv : 0), b2 + (w - dv), c.t.t_a, lane);
      if (item.y & kItemSplit) {
        const uint32_t sl = item.y & kItemMask;
        const uint32_t slot = sl + g.b_v.n_split + g.b_a.n_split;
        float tot;
        if (!split_combine(c.t, slot, g.b_u.split_nchunks[sl], s, lane, &tot)) continue;
        s = tot;
      }
      bepilogue2(c, L, u, s, dv + da, part);
    } else {
      for (uint32_t u = item.x; u < item.x + item.y; ++u) {
        const uint32_t b1 = g.uv_off[u], e1 = g.uv_off[u + 1];
        const uint32_t b2 = g.ua_off[u], e2 = g.ua_off[u + 1];
        float s = dot_plain<float>(g.uv_idx, g.uv_w, b1, e1, c.t.t_v, lane);
        s += dot_plain<WA>(g.ua_idx, g.ua_w, b2, e2, c.t.t_a, lane);
        bepilogue2(c, L, u, s, (e1 - b1) + (e2 - b2), part);
      }
    }
  }
}

__device__ __forceinline__ double bbudget(const BatchParams& p, double eps_f, double M) {
  const double EE = (double)p.e_tot;
  if (p.switch_rule == 2) return INFINITY;
  if (p.switch_rule == 1) return 2.0 * EE * (log(1.0 / (p.lambda * M)) / p.log_inv);
  return 2.0 * EE * fmax(0.0, log(M / eps_f) / p.log_inv);
}

__device__ __forceinline__ unsigned long long score_key(float score, uint32_t caller_id) {
  return ((unsigned long long)__float_as_uint(fmaxf(score, 0.f)) << 32) |
         (unsigned long long)(0xffffffffu - caller_id);
}

}  // namespace

template <typename WA>
__global__ void __launch_bounds__(kThreads, 3)
k_batch(const __grid_constant__ DevGraph g, const __grid_constant__ BatchState st,
        const __grid_constant__ BatchParams p) {
  extern __shared__ unsigned char smem[];
  const uint32_t groups = p.groups;
  const uint32_t nbg = gridDim.x / groups;              // blocks per group
  const uint32_t grp = blockIdx.x / nbg;
  if (grp >= groups) return;                            // leftover blocks
  const uint32_t bid = blockIdx.x - grp * nbg;          // block id within the group
  const TileBuf& tb = st.tb[grp];
  BCtx c{g, tb, p, (bid * kThreads + threadIdx.x) >> 5, (nbg * kThreads) >> 5,
         bid * kThreads + threadIdx.x, nbg * kThreads, threadIdx.x & 31u};
  const uint32_t lane = c.lane;
  const bool app = p.algo == kAlgoAPP;
  const uint32_t n_tiles = (p.n + kTile - 1) / kTile;
  const uint32_t n_split = g.b_v.n_split + g.b_a.n_split + g.b_u.n_split;
  const size_t nu32 = (size_t)g.n_u * kTile;

  for (uint32_t tile = grp; tile < n_tiles; tile += groups) {
    // ---- init the tile (Algorithm 3 lines 1-2 for every lane)
    for (size_t i = c.gt; i < nu32; i += c.nt) { tb.r_u[i] = 0.f; tb.pi[i] = 0.f; tb.pic[i] = 0.f; }
    for (size_t i = c.gt; i < (size_t)g.n_v * kTile; i += c.nt) tb.t_v[i] = 0.f;
    for (size_t i = c.gt; i < (size_t)g.n_a * kTile; i += c.nt) tb.t_a[i] = 0.f;
    for (size_t i = c.gt; i < (size_t)n_split * kTile; i += c.nt) tb.split_acc[i] = 0.f;
    for (size_t i = c.gt; i < n_split; i += c.nt) tb.split_cnt[i] = 0;
    for (size_t i = c.gt; i < (size_t)kRadixPasses * kTile * kRadixBins; i += c.nt) tb.hist[i] = 0;
    if (c.gt < 5 * kTile) tb.racc[c.gt] = RAcc{};
    if (c.gt < kTile) tb.cand_cnt[c.gt] = 0;
    if (!grid_sync(tb.bar, nbg)) return;

    const uint32_t qi = tile * kTile + lane;
    const bool in_range = qi < p.n;
    // ids and eps come from device memory: an invalid one disables its lane
    const bool bad = in_range && (p.q[qi] >= g.n_u || !(p.eps[qi] > 0.0));
    const bool valid = in_range && !bad;
    uint32_t q_new = 0;
    LaneCtl L{0.0, 0, 0, 0, 0, kPhaseAsync, bad ? kStatusBadArg : kStatusOk, 0};
    if (valid) {
      q_new = p.u_old2new[p.q[qi]];
      const double eps = p.eps[qi];
      L.eps_f = app ? eps / (double)p.e_tot : eps / p.lambda;
      L.active = 1;
    }
    if (bid == 0 && threadIdx.x < 32 && valid) {
      const uint32_t cnt = (g.uv_off[q_new + 1] - g.uv_off[q_new]) + (g.ua_off[q_new + 1] - g.ua_off[q_new]);
      const double th = app ? L.eps_f * (double)cnt : L.eps_f;
      RAcc* a0 = &tb.racc[2 * kTile + lane];
      if (1.0 > th) {
        tb.r_u[(size_t)q_new * kTile + lane] = -1.f;
        a0->marked = 1;
        a0->marked_deg = cnt;
      } else {
        tb.r_u[(size_t)q_new * kTile + lane] = 1.f;
      }
    }
    if (!grid_sync(tb.bar, nbg)) return;

    Partials part;
    uint32_t tround = 0;
    bool wait_fail = false;
    for (;;) {
      RAcc* A = &tb.racc[(tround % 3) * kTile];
      const RAcc* P = &tb.racc[((tround + 2) % 3) * kTile];
      const uint32_t marked = __ldcg(&P[lane].marked);
      const unsigned long long marked_deg = __ldcg(&P[lane].marked_deg);
      if (L.active && (L.phase == kPhaseDone || marked == 0)) { L.phase = kPhaseDone; L.active = 0; }
      if (L.active && L.rounds >= p.max_rounds) { L.status = kStatusCap; L.active = 0; }
      if (!__any_sync(kFull, L.active)) break;
      if (bid == 0 && threadIdx.x < kTile) tb.racc[((tround + 1) % 3) * kTile + threadIdx.x] = RAcc{};
      if (L.active) L.pushes += marked;

      bphase1<WA>(c, part);
      flush_lane_partials(part, A);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      bphase2<WA>(c, L, part);
      flush_lane_partials(part, A);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      ++tround;

      bool switched = false;
      if (L.active) {
        ++L.rounds;
        const float M = __uint_as_float(__ldcg(&A[lane].max_r_bits));
        L.n_p += marked_deg + __ldcg(&A[lane].np_flush);
        if (!app) {
          if ((double)M <= L.eps_f) {
            L.phase = kPhaseDone;
            L.active = 0;
          } else if (L.phase == kPhaseAsync && (double)L.n_p >= bbudget(p, L.eps_f, (double)M)) {
            L.phase = kPhaseSync;
            L.switch_round = L.rounds + 1;
            switched = true;
          }
        }
      }
      if (__any_sync(kFull, switched)) {
        // first synchronous round pushes every positive residue of that query
        for (size_t u = c.gw; u < g.n_u; u += c.nw) {
          const size_t i = u * kTile + lane;
          const float r = tb.r_u[i];
          if (switched && r > 0.f) {
            tb.r_u[i] = -r;
            part.marked += 1;
            part.marked_deg += (g.uv_off[u + 1] - g.uv_off[u]) + (g.ua_off[u + 1] - g.ua_off[u]);
          }
        }
        flush_lane_partials(part, A);
        if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      }
    }
    if (wait_fail) L.status = kStatusWait;

    // ---- reserves = pi - compensation; per-query sums; dense output
    {
      Partials pr, pp;
      for (size_t u = c.gw; u < g.n_u; u += c.nw) {
        const size_t i = u * kTile + lane;
        const float v = fmaxf(tb.pi[i] - tb.pic[i], 0.f);
        tb.pi[i] = v;
        const float r = fabsf(tb.r_u[i]);
        pr.sum_r += (double)r;
        pr.max_r = fmaxf(pr.max_r, r);
        pp.sum_r += (double)v;
        if (valid && p.out_dense) p.out_dense[(size_t)qi * g.n_u + p.u_new2old[u]] = v;
      }
      flush_lane_partials(pr, &tb.racc[3 * kTile]);   // residues: sum and max
      flush_lane_partials(pp, &tb.racc[4 * kTile]);   // reserves: sum
    }
    if (!grid_sync(tb.bar, nbg)) return;

    const uint32_t kq = (valid && p.kmax) ? min(min(p.k[qi], p.kmax), g.n_u) : 0u;
    if (bid == 0 && threadIdx.x < kTile && in_range && p.out_stats) {
      ahpp_stats S;
      S.rounds = L.rounds;
      S.switch_round = L.switch_round;
      S.dense_rounds = L.rounds;
      S.status = (uint32_t)((L.status == kStatusOk && L.phase != kPhaseDone && valid) ? kStatusCap
                                                                                   : L.status);
      S.pushes = L.pushes;
      S.n_p = L.n_p;
      S.reserve_sum = __ldcg(&tb.racc[4 * kTile + lane].sum_r);
      S.resid_sum = __ldcg(&tb.racc[3 * kTile + lane].sum_r);
      S.mass_err = fabs(S.reserve_sum + S.resid_sum - 1.0);
      S.max_resid = (double)__uint_as_float(__ldcg(&tb.racc[3 * kTile + lane].max_r_bits));
      S.lambda = p.lambda;
      S.eps_f = L.eps_f;
      p.out_stats[qi] = S;
    }

    // ---- top-k per lane: radix select over 64-bit (score, ~caller id) keys
    if (p.kmax) {
      unsigned int* sh = reinterpret_cast<unsigned int*>(smem);    // [kTile][kRadixBins]
      unsigned long long prefix = 0;
      uint32_t krem = kq;
      for (int pass = 0; pass < kRadixPasses; ++pass) {
        const int shift = 64 - kRadixBits * (pass + 1);
        for (int i = threadIdx.x; i < kTile * kRadixBins; i += kThreads) sh[i] = 0;
        __syncthreads();
        if (krem) {
          for (size_t u = c.gw; u < g.n_u; u += c.nw) {
            const unsigned long long key = score_key(tb.pi[u * kTile + lane], p.u_new2old[u]);
            if (pass == 0 || (key >> (shift + kRadixBits)) == prefix)
              atomicAdd(&sh[lane * kRadixBins + ((key >> shift) & (kRadixBins - 1))], 1u);
          }
        }
        __syncthreads();
        unsigned int* gh = tb.hist + (size_t)pass * kTile * kRadixBins;
        for (int i = threadIdx.x; i < kTile * kRadixBins; i += kThreads)
          if (sh[i]) atomicAdd(&gh[i], sh[i]);
        if (!grid_sync(tb.bar, nbg)) return;
        if (krem) {
          uint32_t cum = 0;
          int d = kRadixBins - 1;
          for (; d > 0; --d) {
            const uint32_t h = __ldcg(&gh[lane * kRadixBins + d]);
            if (cum + h >= krem) break;
            cum += h;
          }
          krem -= cum;
          prefix = (prefix << kRadixBits) | (unsigned long long)d;
        }
      }
      // prefix is the exact key of the kq-th largest; keys are distinct
      if (kq) {
        for (size_t u = c.gw; u < g.n_u; u += c.nw) {
          const unsigned long long key = score_key(tb.pi[u * kTile + lane], p.u_new2old[u]);
          if (key >= prefix) {
            const uint32_t pos = atomicAdd(&tb.cand_cnt[lane], 1u);
            if (pos < p.kmax) tb.cand[(size_t)lane * p.kmax + pos] = key;
          }
        }
      }
      if (!grid_sync(tb.bar, nbg)) return;
      // sort each lane's keys descending (bitonic in shared memory), one block per lane
      unsigned long long* sk = reinterpret_cast<unsigned long long*>(smem);
      for (uint32_t l = bid; l < kTile; l += nbg) {
        const uint32_t ql = tile * kTile + l;
        if (ql >= p.n) continue;
        const bool okl = p.q[ql] < g.n_u && p.eps[ql] > 0.0;
        const uint32_t kl = okl ? min(min(p.k[ql], p.kmax), g.n_u) : 0u;
        uint32_t m = 1;
        while (m < kl) m <<= 1;
        for (uint32_t i = threadIdx.x; i < m; i += kThreads)
          sk[i] = i < kl ? tb.cand[(size_t)l * p.kmax + i] : 0ull;
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
        for (uint32_t i = threadIdx.x; i < kl; i += kThreads) {
          const unsigned long long key = sk[i];
          p.out_nodes[(size_t)ql * p.kmax + i] = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
          p.out_scores[(size_t)ql * p.kmax + i] = __uint_as_float((uint32_t)(key >> 32));
        }
        if (threadIdx.x == 0) p.out_n[ql] = kl;
        __syncthreads();
      }
    } else if (bid == 0 && threadIdx.x < kTile && valid && p.out_n) {
      p.out_n[qi] = 0;
    }
    if (!grid_sync(tb.bar, nbg)) return;
  }
}

template __global__ void k_batch<float>(const __grid_constant__ DevGraph,
                                        const __grid_constant__ BatchState,
                                        const __grid_constant__ BatchParams);
template __global__ void k_batch<__nv_bfloat16>(const __grid_constant__ DevGraph,
                                                const __grid_constant__ BatchState,
                                                const __grid_constant__ BatchParams);

constexpr size_t kBatchSmem = 32 * 1024;   // radix histograms / sort buffer (4096 keys)

int launch_batch(const DevGraph& g, const BatchState& s, const BatchParams& p, bool bf16,
                 int grid, cudaStream_t stream) {
  void* args[] = {(void*)&g, (void*)&s, (void*)&p};
  cudaError_t e;
  if (bf16)
    e = cudaLaunchCooperativeKernel((const void*)k_batch<__nv_bfloat16>, dim3(grid),
                                    dim3(kThreads), args, kBatchSmem, stream);
  else
    e = cudaLaunchCooperativeKernel((const void*)k_batch<float>, dim3(grid), dim3(kThreads),
                                    args, kBatchSmem, stream);
  return e == cudaSuccess ? 0 : (int)e;
}

int batch_max_grid(bool bf16, int sm_count) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, bf16 ? (const void*)k_batch<__nv_bfloat16> : (const void*)k_batch<float>,
      kThreads, kBatchSmem);
  if (e != cudaSuccess || per_sm <= 0) return -1;
  return per_sm * sm_count;
}

}  // namespace ahpp
