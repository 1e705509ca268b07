// Single-query push on the whole GPU: one persistent cooperative launch runs
// every round of APP (Algorithm 3) or ASRP (Algorithm 4) for one source.
//
// A round is either
//   * a push round (small frontier): U-push of the marked list with atomic
//     scatter into t_V / t_A (the U-push of Algorithm 3), then the flush of
//     every V node and attribute with a positive t value (its V and attribute
//     steps) into r_U, in the work items of the pull phase 1 (long rows split
//     into chunks over warps, so a hub's flush is spread over the grid), then
//     the selection of the next frontier (warp-ballot compaction) and the
//     clearing of t_V / t_A;
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

// ---------------------------------------------------------------- phase 1
// t_V[v] = sum_u c_uv p_u ;  t_A[a] = k_attr cnorm_a[a] sum_u (w(u,a) rnorm_u[u]) p_u
// (the A->U pull coefficient w(u,a) rnorm_u[u] is precomputed per entry).

__device__ __forceinline__ void p1_epilogue(const Ctx& c, bool is_a, uint32_t row, float s, float* ta_out,
                                            Partials& part) {
  if (!is_a) {
    c.s.t_v[row] = s;
    if (s > 0.f) part.np_flush += c.g.vu_off[row + 1] - c.g.vu_off[row];
  } else {
    float t = c.g.k_attr * c.g.cnorm_a[row] * s;
    ta_out[row] = t;
    if (t > 0.f) part.np_flush += c.g.au_off[row + 1] - c.g.au_off[row];
  }
}

// sum over k = k0, k0 + st, k0 + 2 st, ... < e of coef(k) x(idx[k]), in that
// order, four entries per step, software-pipelined: the next step's indices
// and coefficients load while this step's gathers are in flight, so a step
// waits for one load latency instead of two (index, then gather).
template <typename CoefF, typename XF>
__device__ __forceinline__ float strided_dot(uint32_t k0, uint32_t e, uint32_t st, const uint32_t* __restrict__ idx,
                                             CoefF coef, XF x, float s) {
  uint32_t i0 = 0, i1 = 0, i2 = 0, i3 = 0;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  auto load = [&](uint32_t k, uint32_t& j0, uint32_t& j1, uint32_t& j2, uint32_t& j3, float& d0, float& d1,
                  float& d2, float& d3) {
    if (k < e) { j0 = idx[k]; d0 = coef(k); }
    if (k + st < e) { j1 = idx[k + st]; d1 = coef(k + st); }
    if (k + 2 * st < e) { j2 = idx[k + 2 * st]; d2 = coef(k + 2 * st); }
    if (k + 3 * st < e) { j3 = idx[k + 3 * st]; d3 = coef(k + 3 * st); }
  };
  load(k0, i0, i1, i2, i3, c0, c1, c2, c3);
  for (uint32_t k = k0; k < e; k += 4 * st) {
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
    load(k + 4 * st, n0, n1, n2, n3, d0, d1, d2, d3);
    const float x0 = x(i0);
    const float x1 = k + st < e ? x(i1) : 0.f;
    const float x2 = k + 2 * st < e ? x(i2) : 0.f;
    const float x3 = k + 3 * st < e ? x(i3) : 0.f;
    s = fmaf(c0, x0, s);
    if (k + st < e) s = fmaf(c1, x1, s);
    if (k + 2 * st < e) s = fmaf(c2, x2, s);
    if (k + 3 * st < e) s = fmaf(c3, x3, s);
    i0 = n0; i1 = n1; i2 = n2; i3 = n3;
    c0 = d0; c1 = d1; c2 = d2; c3 = d3;
  }
  return s;
}

// The first index >= e of the sequence k0, k0 + st, ... (k0 itself if >= e).
__device__ __forceinline__ uint32_t strided_end(uint32_t k0, uint32_t e, uint32_t st) {
  return k0 < e ? k0 + (e - k0 + st - 1) / st * st : k0;
}

// A warp's share of a long row: lane l takes entries z + l, z + l + 32, ...
template <typename CoefF, typename XF>
__device__ __forceinline__ float lane_dot(uint32_t z, uint32_t w, uint32_t lane, const uint32_t* __restrict__ idx,
                                          CoefF coef, XF x, float s) {
  return strided_dot(z + lane, w, 32u, idx, coef, x, s);
}

// Lanes per row for an item of nr short rows holding nnz entries: the mean
// row length rounded up to a power of two, at most vw_max (a power of two
// <= 32).  Rows are sorted by degree, so an item's rows have about that
// length; vw lanes then walk each row together and one load of the warp
// reads contiguous entries.
__device__ __forceinline__ uint32_t vec_width(uint32_t nnz, uint32_t nr, uint32_t vw_max) {
  const uint32_t mean = (nnz + nr - 1) / max(nr, 1u);
  return mean <= 1 ? 1u : min(vw_max, 1u << (32 - __clz(mean - 1)));
}

// Sum over the vw lanes of a row's segment (every lane of the warp calls it).
__device__ __forceinline__ float seg_sum(float s, uint32_t vw) {
  for (uint32_t o = vw >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Rows 0..nr-1 (nr <= 32) of an item, vw lanes per row: part(r, sub) is lane
// sub's share of row r; returns row `lane`'s total in lane `lane` (0 for
// lanes >= nr).  Passes of 32 / vw rows; after pass p the sums of its rows
// sit in lanes 0, vw, 2 vw, ... and move to lanes p (32 / vw) + 0, 1, ...
template <typename PartF>
__device__ __forceinline__ float rows_to_lanes(uint32_t nr, uint32_t vw, uint32_t lane, PartF part) {
  const uint32_t sub = lane & (vw - 1), rpp = 32 / vw, npass = (nr + rpp - 1) / rpp;
  float mine = 0.f;
  for (uint32_t pass = 0; pass < npass; ++pass) {        // warp-uniform
    const uint32_t r = pass * rpp + lane / vw;
    float s = r < nr ? part(r, sub) : 0.f;
    s = seg_sum(s, vw);
    const float t = __shfl_sync(0xffffffffu, s, (lane % rpp) * vw);
    if (lane / rpp == pass) mine = t;
  }
  return mine;
}

template <typename WA>
__device__ void phase1(const Ctx& c, Partials& part, bool do_a, float* ta_out, const float* ta_scan,
                       float* ta_zero) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  if (ta_scan || ta_zero) {
    // t_A of this round was pushed by the previous phase 2: count its active
    // attributes (Algorithm 4's push counter) and clear the next round's buffer
    for (uint32_t a = c.gt; a < g.n_a; a += c.nt) {
      if (ta_scan && ta_scan[a] > 0.f) part.np_flush += g.au_off[a + 1] - g.au_off[a];
      if (ta_zero) ta_zero[a] = 0.f;
    }
  }
  const float* __restrict__ r_u = c.s.r_u;
  auto P = [&](uint32_t u) { return fmaxf(-r_u[u], 0.f); };
  auto cv = [&](uint32_t k) { return g.vu_c[k]; };
  auto ca = [&](uint32_t k) { return g.au_c[k]; };
  const uint32_t nv = g.s1_v.n_items, total = nv + (do_a ? g.s1_a.n_items : 0u);
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const bool is_a = it >= nv;
    const uint4 item = is_a ? g.s1_a.items[it - nv] : g.s1_v.items[it];
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    const uint32_t* idx = is_a ? g.au_idx : g.vu_idx;
    if (item.y & (kItemLong | kItemSplit)) {
      const uint32_t row = item.x, base = off[row];
      float s = is_a ? lane_dot(base + item.z, base + item.w, lane, idx, ca, P, 0.f)
                     : lane_dot(base + item.z, base + item.w, lane, idx, cv, P, 0.f);
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
            p1_epilogue(c, is_a, row, tot, ta_out, part);
          }
        } else {
          p1_epilogue(c, is_a, row, s, ta_out, part);
        }
      }
    } else {
      // up to 32 short rows: vw lanes walk each row (coalesced loads), then
      // lane r holds row r's sum and the epilogues run one row per lane
      const uint32_t r0 = item.x, nr = item.y;
      const uint32_t vw = vec_width(off[r0 + nr] - off[r0], nr, c.p.vw_max);
      const float mine = rows_to_lanes(nr, vw, lane, [&](uint32_t r, uint32_t sub) {
        const uint32_t k = off[r0 + r] + sub, e = off[r0 + r + 1];
        return is_a ? strided_dot(k, e, vw, idx, ca, P, 0.f) : strided_dot(k, e, vw, idx, cv, P, 0.f);
      });
      if (lane < nr) p1_epilogue(c, is_a, r0 + lane, mine, ta_out, part);
    }
  }
}

// ---------------------------------------------------------------- phase 2
// r_U'[u] = kept_u + sum_v w(u,v) t_V[v] + sum_a w(u,a) t_A[a]; reserve update of
// the nodes pushed this round; marking of the next frontier with threshold th;
// with the attribute push, the marked node's attribute share of the next
// round: acc[a] += w(u,a) rnorm_u[u] p_u (block-local, shared memory), added
// to t_A' scaled by k_attr cnorm_a[a] at the end of the phase.

// APP(S)'s round statistics of a residue r of a node with cnt = |N(u)| + |A(u)|:
// the largest r / cnt, and whether r exceeds APP's threshold r_max cnt.
__device__ __forceinline__ void app_stats(const Ctx& c, float r, uint32_t cnt, Partials& part) {
  if (cnt) part.max_rel = fmaxf(part.max_rel, r / (float)cnt);
  if ((double)r > c.p.eps_f * (double)cnt) part.above += 1;
}

// Returns the residue marked for the next push (0 if u is not marked).
template <bool APPS>
__device__ __forceinline__ float p2_epilogue(const Ctx& c, uint32_t u, float s, uint32_t cnt,
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
  if (APPS) app_stats(c, r_new, cnt, part);
  const double th = per_node ? theta * (double)cnt : theta;
  if ((double)r_new > th) {
    c.s.r_u[u] = -r_new;
    part.marked += 1;
    part.marked_deg += cnt;
    return r_new;
  }
  c.s.r_u[u] = r_new;
  return 0.f;
}

template <typename WA>
__device__ __forceinline__ void push_attr_smem(const DevGraph& g, uint32_t u, float p, float* acc) {
  const uint32_t b = g.ua_off[u], e = g.ua_off[u + 1];
  const float f = g.rnorm_u[u] * p;
  for (uint32_t k = b; k < e; ++k) atomicAdd(&acc[g.ua_idx[k]], wload<WA>(g.ua_w, k) * f);
}

template <typename WA, bool APPS>
__device__ void phase2(const Ctx& c, double theta, bool per_node, Partials& part, const float* ta_cur,
                       float* ta_next, float* smem) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  const uint32_t na = g.n_a;
  // shared memory (ta_smem): a copy of t_A and, with the push, its accumulator
  float* s_ta = smem;
  float* s_acc = smem + na;
  if (c.p.ta_smem) {
    for (uint32_t a = threadIdx.x; a < na; a += blockDim.x) {
      s_ta[a] = ta_cur[a];
      if (ta_next) s_acc[a] = 0.f;
    }
    __syncthreads();
  }
  const float* __restrict__ t_v = c.s.t_v;
  auto TV = [&](uint32_t v) { return t_v[v]; };
  auto TA = [&](uint32_t a) { return c.p.ta_smem ? s_ta[a] : ta_cur[a]; };
  auto wv = [&](uint32_t k) { return g.uv_w[k]; };
  auto wa = [&](uint32_t k) { return wload<WA>(g.ua_w, k); };
  const uint32_t total = g.s1_u.n_items;
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const uint4 item = g.s1_u.items[it];
    if (item.y & (kItemLong | kItemSplit)) {
      const uint32_t u = item.x;
      const uint32_t b1 = g.uv_off[u], dv = g.uv_off[u + 1] - b1;
      const uint32_t b2 = g.ua_off[u], da = g.ua_off[u + 1] - b2;
      // chunk [z, w) of the combined list: V neighbours first, then attributes
      float s = 0.f;
      if (item.z < dv) s = lane_dot(b1 + item.z, b1 + min(item.w, dv), lane, g.uv_idx, wv, TV, s);
      if (item.w > dv) s = lane_dot(b2 + (item.z > dv ? item.z - dv : 0), b2 + (item.w - dv), lane, g.ua_idx, wa,
                                    TA, s);
      s = warp_sum(s);
      float pm = 0.f;
      if (lane == 0) {
        if (item.y & kItemSplit) {
          const uint32_t slot = (item.y & kItemMask) + g.s1_v.n_split + g.s1_a.n_split;
          const uint32_t nch = g.s1_u.split_nchunks[item.y & kItemMask];
          atomicAdd(&c.s.split_acc[slot], s);
          __threadfence();
          if (atomicAdd(&c.s.split_cnt[slot], 1u) == nch - 1) {
            float tot = atomicExch(&c.s.split_acc[slot], 0.f);
            c.s.split_cnt[slot] = 0;
            pm = p2_epilogue<APPS>(c, u, tot, dv + da, theta, per_node, part);
          }
        } else {
          pm = p2_epilogue<APPS>(c, u, s, dv + da, theta, per_node, part);
        }
        if (ta_next && pm > 0.f) push_attr_smem<WA>(g, u, pm, s_acc);
      }
    } else {
      // up to 32 short rows (V neighbours, then attributes): vw lanes walk each
      // row, then the epilogues and attribute pushes run one row per lane
      const uint32_t u0 = item.x, nr = item.y;
      const uint32_t nnz = (g.uv_off[u0 + nr] - g.uv_off[u0]) + (g.ua_off[u0 + nr] - g.ua_off[u0]);
      const uint32_t vw = vec_width(nnz, nr, c.p.vw_max);
      const float mine = rows_to_lanes(nr, vw, lane, [&](uint32_t r, uint32_t sub) {
        // lane sub takes entries sub, sub + vw, ... of the combined list:
        // the V neighbours [0, dv), then the attributes [dv, dv + da)
        const uint32_t u = u0 + r;
        const uint32_t b1 = g.uv_off[u], dv = g.uv_off[u + 1] - b1;
        const uint32_t b2 = g.ua_off[u], da = g.ua_off[u + 1] - b2;
        const float s = strided_dot(b1 + sub, b1 + dv, vw, g.uv_idx, wv, TV, 0.f);
        // the same lane's first attribute entry
        const uint32_t ka = strided_end(b1 + sub, b1 + dv, vw) - b1 - dv + b2;
        return strided_dot(ka, b2 + da, vw, g.ua_idx, wa, TA, s);
      });
      if (lane < nr) {
        const uint32_t u = u0 + lane;
        const uint32_t cnt = (g.uv_off[u + 1] - g.uv_off[u]) + (g.ua_off[u + 1] - g.ua_off[u]);
        const float pm = p2_epilogue<APPS>(c, u, mine, cnt, theta, per_node, part);
        if (ta_next && pm > 0.f) push_attr_smem<WA>(g, u, pm, s_acc);
      }
    }
  }
  if (ta_next) {
    __syncthreads();
    for (uint32_t a = threadIdx.x; a < na; a += blockDim.x) {
      const float v = s_acc[a];
      if (v != 0.f) atomicAdd(&ta_next[a], g.k_attr * g.cnorm_a[a] * v);
    }
  }
}

// --------------------------------------------------------- push (sparse)

template <typename WA>
__device__ void push_u(const Ctx& c, uint32_t n_list) {
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
    // non-returning reductions: the flush finds the rows it must move by
    // their value, so no first-touch list is kept
    const uint32_t b1 = g.uv_off[u], e1 = g.uv_off[u + 1];
    for (uint32_t k = b1 + lane; k < e1; k += 32) atomicAdd(&c.s.t_v[g.uv_idx[k]], g.uv_c[k] * p);
    const float ka = g.k_attr * g.rnorm_u[u] * p;
    const uint32_t b2 = g.ua_off[u], e2 = g.ua_off[u + 1];
    for (uint32_t k = b2 + lane; k < e2; k += 32) {
      const uint32_t a = g.ua_idx[k];
      atomicAdd(&c.s.t_a[a], wload<WA>(g.ua_w, k) * ka * g.cnorm_a[a]);
    }
  }
}

// One V (or attribute) row's flush over entries [b, e): r_U[j] += w t for its
// U neighbours j (returning atomics: the new residues feed max r_U).
template <typename WA, bool APPS>
__device__ __forceinline__ void flush_row(const Ctx& c, bool is_a, uint32_t b, uint32_t e, float t,
                                          Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t* idx = is_a ? g.au_idx : g.vu_idx;
  for (uint32_t k = b + lane_id(); k < e; k += 32) {
    const float w = is_a ? wload<WA>(g.au_w, k) : g.vu_w[k];
    const float add = w * t;
    const uint32_t j = idx[k];
    const float old = atomicAdd(&c.s.r_u[j], add);
    part.max_r = fmaxf(part.max_r, old + add);
    // APP(S): a node's last update sees its new residue (counts of nodes
    // above threshold may repeat a node; only zero is tested)
    if (APPS)
      app_stats(c, old + add, (g.uv_off[j + 1] - g.uv_off[j]) + (g.ua_off[j + 1] - g.ua_off[j]), part);
  }
}

// The V and attribute flush of a push round, over the work items of phase 1:
// a short-row item's rows with t > 0 are flushed one after another by the
// warp; a long row's chunk by the warp that owns the chunk.  t_V / t_A are
// only read here (select_frontier clears them after the barrier).
template <typename WA, bool APPS>
__device__ void flush_va(const Ctx& c, Partials& part) {
  const DevGraph& g = c.g;
  const uint32_t lane = lane_id();
  const uint32_t nv = g.s1_v.n_items, total = nv + g.s1_a.n_items;
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const bool is_a = it >= nv;
    const uint4 item = is_a ? g.s1_a.items[it - nv] : g.s1_v.items[it];
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    const float* t = is_a ? c.s.t_a : c.s.t_v;
    if (item.y & (kItemLong | kItemSplit)) {
      const uint32_t row = item.x;
      const float tv = t[row];
      if (!(tv > 0.f)) continue;
      const uint32_t b = off[row];
      if (item.z == 0 && lane == 0) part.np_flush += off[row + 1] - b;
      flush_row<WA, APPS>(c, is_a, b + item.z, b + item.w, tv, part);
    } else {
      const uint32_t r0 = item.x, nr = item.y;
      const float mine = lane < nr ? t[r0 + lane] : 0.f;
      for (unsigned m = __ballot_sync(0xffffffffu, mine > 0.f); m; m &= m - 1) {
        const uint32_t r = __ffs(m) - 1;
        const float tv = __shfl_sync(0xffffffffu, mine, r);
        const uint32_t b = off[r0 + r], e = off[r0 + r + 1];
        if (lane == 0) part.np_flush += e - b;
        flush_row<WA, APPS>(c, is_a, b, e, tv, part);
      }
    }
  }
}

// Marking of the next frontier in a push round: r_U > th (per_node: th * cnt(u)),
// and the clearing of t_V / t_A for the next round's U-push.
__device__ void select_frontier(const Ctx& c, double theta, bool per_node, RAcc* acc,
                                Partials& part) {
  const DevGraph& g = c.g;
  for (uint32_t v = c.gt; v < g.n_v; v += c.nt) c.s.t_v[v] = 0.f;
  for (uint32_t a = c.gt; a < g.n_a; a += c.nt) c.s.t_a[a] = 0.f;
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

template <typename WA, bool APPS>
__global__ void __launch_bounds__(kQ1Threads, kQ1Blocks)
k_query1(const __grid_constant__ DevGraph g, const __grid_constant__ Q1State s,
         const __grid_constant__ Q1Params p) {
  extern __shared__ __align__(16) float q1_smem[];
  Ctx c{g, s, p, (blockIdx.x * kQ1Threads + threadIdx.x) >> 5, (gridDim.x * kQ1Threads) >> 5,
        blockIdx.x * kQ1Threads + threadIdx.x, gridDim.x * kQ1Threads};
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const unsigned int nb = gridDim.x;
  const bool app = p.algo != kAlgoASRP;    // APP's per-node threshold for the source

  // ---- init: zero the state, mark the source (the initial state of Algorithm 3)
  const float r0 = p.lambda_mode ? -1.f : 0.f;
  for (uint32_t u = c.gt; u < g.n_u; u += c.nt) { s.r_u[u] = r0; s.pi[u] = 0.f; s.pic[u] = 0.f; }
  for (uint32_t v = c.gt; v < g.n_v; v += c.nt) s.t_v[v] = 0.f;
  for (uint32_t a = c.gt; a < g.n_a; a += c.nt) { s.t_a[a] = 0.f; s.t_a2[a] = 0.f; }
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
  // attribute push: t_A of a pull round lives in ta_buf[ta_sel] and phase 2
  // pushes the next round's into the other buffer; the first pull round, and
  // the round after the ASRP switch marks more nodes, pull t_A instead
  float* const ta_buf[2] = {s.t_a, s.t_a2};
  int ta_sel = 0;
  bool pull_a = true;

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
    const bool per_node = per_node_threshold(p.algo, phase);
    const double theta = (phase == kPhaseSync && !per_node) ? 0.0 : p.eps_f;

    if (!dense) {
      push_u<WA>(c, marked);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      flush_va<WA, APPS>(c, part);
      flush_partials<kQ1Warps, APPS>(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
    } else {
      float* ta_cur = ta_buf[ta_sel];
      float* ta_next = p.attr_push ? ta_buf[ta_sel ^ 1] : nullptr;
      const bool do_a = !p.attr_push || pull_a;
      phase1<WA>(c, part, do_a, ta_cur, do_a ? nullptr : ta_cur, ta_next);
      flush_partials<kQ1Warps, APPS>(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      phase2<WA, APPS>(c, theta, per_node, part, ta_cur, ta_next, q1_smem);
      flush_partials<kQ1Warps, APPS>(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      if (p.attr_push) ta_sel ^= 1;
      pull_a = false;
      ++dense_rounds;
    }
    ++rounds;

    // ---- decision (every thread computes the same result)
    const float M = __uint_as_float(__ldcg(&A->max_r_bits));
    n_p += marked_deg + __ldcg(&A->np_flush);
    if (p.trace_cap && leader && rounds - 1 < p.trace_cap) s.trace_maxr[rounds - 1] = M;
    bool switched = false;
    if (p.algo == kAlgoASRP) {
      if ((double)M <= p.eps_f) {
        phase = kPhaseDone;
      } else if (phase == kPhaseAsync && (double)n_p >= budget_of(p, (double)M)) {
        phase = kPhaseSync;
        switch_round = rounds + 1;
        switched = true;
      }
    } else if (APPS) {
      // APP's stopping test; the switch budget in units of APP's thresholds
      const float Mrel = __uint_as_float(__ldcg(&A->max_rel_bits));
      if (__ldcg(&A->above) == 0) {
        phase = kPhaseDone;
      } else if (phase == kPhaseAsync && (double)n_p >= budget_of(p, (double)Mrel)) {
        phase = kPhaseSync;
        switch_round = rounds + 1;
        switched = true;
      }
    }
    if (phase == kPhaseDone) break;
    if (!dense) {
      const bool pn_next = per_node_threshold(p.algo, phase);
      const double th_next = (phase == kPhaseSync && !pn_next) ? 0.0 : p.eps_f;
      select_frontier(c, th_next, pn_next, A, part);
      flush_partials<kQ1Warps, APPS>(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
    } else if (switched) {
      mark_remaining(c, part);
      flush_partials<kQ1Warps, APPS>(part, A);
      if (!grid_sync(s.bar, nb)) { status = kStatusWait; break; }
      pull_a = true;       // the new marks did not push their attribute share
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

#define AHPP_Q1_INSTANCE(WA, APPS)                                                   \
  template __global__ void k_query1<WA, APPS>(const __grid_constant__ DevGraph,      \
                                              const __grid_constant__ Q1State,       \
                                              const __grid_constant__ Q1Params);
AHPP_Q1_INSTANCE(float, false)
AHPP_Q1_INSTANCE(__nv_bfloat16, false)
AHPP_Q1_INSTANCE(float, true)
AHPP_Q1_INSTANCE(__nv_bfloat16, true)
#undef AHPP_Q1_INSTANCE

// Launch helper: persistent cooperative grid (one block per SM).
namespace {
// The instance of a launch: APP(S)'s round statistics are compiled only into
// the APP(S) instances.
const void* q1_fn(bool bf16, bool apps = false) {
  if (apps) return bf16 ? (const void*)k_query1<__nv_bfloat16, true> : (const void*)k_query1<float, true>;
  return bf16 ? (const void*)k_query1<__nv_bfloat16, false> : (const void*)k_query1<float, false>;
}
}  // namespace

// Carve out of the SM's unified memory just the shared memory kQ1Blocks
// blocks need (each with 1 KB reserved by the system); the rest stays L1,
// which holds the lines of the rows the lanes are walking.  Sets the dynamic
// shared memory limit of the instance too.
int prepare(const void* fn, uint32_t smem_bytes) {
  int dev = 0, per_sm = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, fn) != cudaSuccess || per_sm <= 0)
    return (int)cudaGetLastError();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return (int)e;
  const uint64_t need = (uint64_t)kQ1Blocks * (smem_bytes + fa.sharedSizeBytes + 1024);
  const int pct = (int)std::min<uint64_t>(100, (100 * need + per_sm - 1) / per_sm);
  return (int)cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

uint32_t query1_max_smem(int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  size_t stat = 0;
  for (int apps = 0; apps < 2; ++apps) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, q1_fn(true, apps)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    stat = std::max(stat, fa.sharedSizeBytes);
  }
  const long room = (long)optin - (long)stat - 1024;   // static shared memory + margin
  return room > 0 ? (uint32_t)(room / 16 * 16) : 0u;
}

int launch_query1(const DevGraph& g, const Q1State& s, const Q1Params& p, bool bf16,
                  int grid, cudaStream_t stream) {
  void* args[] = {(void*)&g, (void*)&s, (void*)&p};
  const void* fn = q1_fn(bf16, p.algo == kAlgoAPPS);
  cudaError_t e = (cudaError_t)prepare(fn, p.smem_bytes);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kQ1Threads), args, p.smem_bytes, stream);
  return e == cudaSuccess ? 0 : (int)e;
}

// Co-resident grid of both instances (a plan serves every algorithm).
int query1_max_grid(bool bf16, int sm_count, uint32_t smem_bytes) {
  int best = -1;
  for (int apps = 0; apps < 2; ++apps) {
    const void* fn = q1_fn(bf16, apps);
    int per_sm = 0;
    cudaError_t e = (cudaError_t)prepare(fn, smem_bytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kQ1Threads, smem_bytes);
    if (e != cudaSuccess || per_sm <= 0) {
      cudaGetLastError();
      return -1;
    }
    best = best < 0 ? per_sm : std::min(best, per_sm);
  }
  return best * sm_count;
}

}  // namespace ahpp
