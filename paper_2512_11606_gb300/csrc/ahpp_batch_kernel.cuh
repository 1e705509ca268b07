// Batched multi-source APP / ASRP: one persistent cooperative launch runs n
// queries packed into tiles of kTile (one query per lane).  Every round of a
// tile is a pull sweep over the whole graph (the synchronous form of
// Algorithm 3's three loops): phase 1 gathers t_V / t_A for all the tile's
// queries from the marked residues, phase 2 gathers the new residues, applies the
// reserve update of the pushed nodes and marks the next frontier of each
// query with its own threshold.  Per-query control (termination, the ASRP
// switch test of Algorithm 4) is kept per lane; a query that finishes is
// frozen while the rest of its tile continues, so its result does not depend
// on the other queries of the tile.  Top-k per query is a per-lane radix
// select over (score, caller id) keys.
// This file is the kernel body of ahpp_batch.cu, which includes it once per
// tile width: AHPP_BT (queries per tile) and AHPP_BT_NS (the namespace of
// that instance) are defined by the includer.  No include guard.
#include "ahpp_batch.cuh"

namespace ahpp {
namespace AHPP_BT_NS {

constexpr int kTile = AHPP_BT;     // queries per tile of this instance


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
  __shared__ float s_max[kBWarps][32];
  __shared__ uint32_t s_mk[kBWarps][32];
  __shared__ unsigned long long s_dg[kBWarps][32], s_np[kBWarps][32];
  __shared__ double s_sum[kBWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_max[warp][lane] = p.max_r; s_mk[warp][lane] = p.marked; s_dg[warp][lane] = p.marked_deg;
  s_np[warp][lane] = p.np_flush; s_sum[warp][lane] = p.sum_r;
  __syncthreads();
  if (warp == 0) {
    float m = s_max[0][lane];
    uint32_t mk = s_mk[0][lane];
    unsigned long long dg = s_dg[0][lane], np = s_np[0][lane];
    double sm = s_sum[0][lane];
    for (int w = 1; w < kBWarps; ++w) {
      m = fmaxf(m, s_max[w][lane]); mk += s_mk[w][lane]; dg += s_dg[w][lane];
      np += s_np[w][lane]; sm += s_sum[w][lane];
    }
    RAcc* a = &acc[lane];
    if (lane < kTile) {
      if (m > 0.f) atomicMax(&a->max_r_bits, __float_as_uint(m));
      if (mk) atomicAdd(&a->marked, mk);
      if (dg) atomicAdd(&a->marked_deg, dg);
      if (np) atomicAdd(&a->np_flush, np);
      if (sm != 0.0) atomicAdd(&a->sum_r, sm);
    }
  }
  __syncthreads();
  p = Partials();
}

// ------------------------------------------------------------------------
// Pull phases with row groups: a warp is 4 groups of 8 lanes; a group owns
// one row (or one chunk of a long row) and each of its lanes owns 4 of the
// tile's 32 queries (lane l of the group: queries 4l .. 4l+3).  One gather
// is a float4 load per lane, so the group reads the 32 queries' values of a
// neighbour as one 128-byte line and one warp instruction moves 4 lines.
// Entries go in waves of 8 (one per lane of the group, coalesced): the 8
// line gathers of a wave are in flight together, and the number of waves is
// the warp's longest row, so short rows (most rows of a power-law graph)
// issue no idle gather slots beyond their last wave.
constexpr int kQL = 4;                 // queries per lane
constexpr int kGL = kTile / kQL;       // lanes per row group (one 128- or 64-byte line)
constexpr int kGPW = 32 / kGL;         // row groups per warp
static_assert(kTile == 16 || kTile == 32, "tile of 16 or 32 queries");

// Smallest float f with (r > th) <=> (r >= f) for every float r: the mark
// test r > th of Algorithm 4 taken exactly against the FP64 threshold.
__device__ __forceinline__ float threshold_up(double th) {
  float f = (float)th;
  if ((double)f <= th) f = nextafterf(f, INFINITY);
  return f;
}

// Graph arrays, reserves and compensations are read once per round:
// streamed with the evict-first policy so that they do not push the
// gathered state rows out of L2.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// out[0..3] += v as a reduction that returns nothing: an atomicAdd on a
// float4 whose result is unused is still issued as a returning atomic, and
// the returned line then takes L2 -> SM bandwidth that the gathers need.
__device__ __forceinline__ void red_add4(float* out, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(out), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

__device__ __forceinline__ float4 f4_fma(float c, float4 x, float4 a) {
  return make_float4(fmaf(c, x.x, a.x), fmaf(c, x.y, a.y), fmaf(c, x.z, a.z), fmaf(c, x.w, a.w));
}

// Sum over the entries [b, e) of this group's row of coef(k) * gather(idx(k)),
// in waves of kGL entries: lane t of the group loads entry t of a wave
// (coalesced), the entry's index and coefficient are broadcast within the
// group, and the wave's kGL row gathers are in flight together.  The next
// wave's index and coefficient loads are issued before the current wave's
// gathers.  Called by the whole warp: `waves` is warp-uniform (the warp's
// longest range, in waves); a group with b == e adds nothing.
template <typename LoadF, typename GatherF>
__device__ __forceinline__ float4 group_accum(uint32_t b, uint32_t e, uint32_t waves, uint32_t gl,
                                              LoadF load, GatherF gather) {
  float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
  uint32_t k = b + gl;
  uint32_t mi = 0;
  float mc = 0.f;
  if (k < e) load(k, mi, mc);
  for (uint32_t w = 0; w < waves; ++w) {
    const uint32_t k0 = b + w * kGL;
    const uint32_t n = k0 < e ? min((uint32_t)kGL, e - k0) : 0u;
    const uint32_t kn = k + kGL;
    uint32_t ni = 0;
    float nc = 0.f;
    if (kn < e) load(kn, ni, nc);
    float4 x[kGL];
#pragma unroll
    for (int t = 0; t < kGL; ++t) {
      const uint32_t id = __shfl_sync(kFull, mi, t, kGL);
      x[t] = (uint32_t)t < n ? gather(id) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kGL; ++t) {
      const float c = __shfl_sync(kFull, mc, t, kGL);
      const float2 cc = make_float2(c, c);
      a01 = __ffma2_rn(cc, make_float2(x[t].x, x[t].y), a01);
      a23 = __ffma2_rn(cc, make_float2(x[t].z, x[t].w), a23);
    }
    mi = ni;
    mc = nc;
    k = kn;
  }
  return make_float4(a01.x, a01.y, a23.x, a23.y);
}

__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Per-query partials of one thread (its 4 queries) summed over the warp's 4
// groups and the block's warps, then added to acc[q] (one atomic per query
// and field per block).
struct Q4Partials {
  float max_r[kQL] = {0.f, 0.f, 0.f, 0.f};
  uint32_t marked[kQL] = {0, 0, 0, 0};
  uint32_t mdeg[kQL] = {0, 0, 0, 0};
  uint32_t np[kQL] = {0, 0, 0, 0};
  float max_rel[kQL] = {0.f, 0.f, 0.f, 0.f};   // APP(S) statistics (see RAcc)
  uint32_t above[kQL] = {0, 0, 0, 0};
};

template <bool APPS>
__device__ __forceinline__ void flush_q4(Q4Partials& p, RAcc* acc) {
  __shared__ float s_max[kBWarps][32];
  __shared__ uint32_t s_mk[kBWarps][32], s_dg[kBWarps][32], s_np[kBWarps][32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kQL; ++j) {
#pragma unroll
    for (int o = kGL; o < 32; o <<= 1) {
      p.max_r[j] = fmaxf(p.max_r[j], __shfl_xor_sync(kFull, p.max_r[j], o));
      p.marked[j] += __shfl_xor_sync(kFull, p.marked[j], o);
      p.mdeg[j] += __shfl_xor_sync(kFull, p.mdeg[j], o);
      p.np[j] += __shfl_xor_sync(kFull, p.np[j], o);
      if (APPS) {
        p.max_rel[j] = fmaxf(p.max_rel[j], __shfl_xor_sync(kFull, p.max_rel[j], o));
        p.above[j] += __shfl_xor_sync(kFull, p.above[j], o);
      }
    }
  }
  if (lane < kGL) {
#pragma unroll
    for (int j = 0; j < kQL; ++j) {
      const uint32_t q = lane * kQL + j;
      s_max[warp][q] = p.max_r[j]; s_mk[warp][q] = p.marked[j];
      s_dg[warp][q] = p.mdeg[j]; s_np[warp][q] = p.np[j];
    }
  }
  __syncthreads();
  if (warp == 0 && lane < kTile) {
    float m = 0.f;
    uint32_t mk = 0;
    unsigned long long dg = 0, np = 0;
    for (int w = 0; w < kBWarps; ++w) {
      m = fmaxf(m, s_max[w][lane]); mk += s_mk[w][lane];
      dg += s_dg[w][lane]; np += s_np[w][lane];
    }
    RAcc* a = &acc[lane];
    if (m > 0.f) atomicMax(&a->max_r_bits, __float_as_uint(m));
    if (mk) atomicAdd(&a->marked, mk);
    if (dg) atomicAdd(&a->marked_deg, dg);
    if (np) atomicAdd(&a->np_flush, np);
  }
  if (APPS) {
    // the APP(S) statistics through the same buffers (max_r / marked reused)
    __syncthreads();
    if (lane < kGL) {
#pragma unroll
      for (int j = 0; j < kQL; ++j) {
        const uint32_t q = lane * kQL + j;
        s_max[warp][q] = p.max_rel[j];
        s_mk[warp][q] = p.above[j];
      }
    }
    __syncthreads();
    if (warp == 0 && lane < kTile) {
      float m = 0.f;
      uint32_t ab = 0;
      for (int w = 0; w < kBWarps; ++w) { m = fmaxf(m, s_max[w][lane]); ab += s_mk[w][lane]; }
      if (m > 0.f) atomicMax(&acc[lane].max_rel_bits, __float_as_uint(m));
      if (ab) atomicAdd(&acc[lane].above, ab);
    }
  }
  __syncthreads();
  p = Q4Partials();
}

// Combine a chunk of a split row (group-collective): returns true in every
// lane of the group whose chunk finishes the row, with the row total.
__device__ __forceinline__ bool split_combine4(const TileBuf& t, uint32_t slot, uint32_t nch,
                                               float4 s, uint32_t gl, unsigned gmask, float4* tot) {
  float* a = &t.split_acc[(size_t)slot * kTile + kQL * gl];
  red_add4(a, s);
  __threadfence();
  __syncwarp(gmask);
  uint32_t last = 0;
  if (gl == 0) last = atomicAdd(&t.split_cnt[slot], 1u) == nch - 1;
  last = __shfl_sync(gmask, last, 0, kGL);
  if (last) {
    __threadfence();
    *tot = __ldcg(reinterpret_cast<const float4*>(a));
    __stcg(reinterpret_cast<float4*>(a), make_float4(0.f, 0.f, 0.f, 0.f));
    __syncwarp(gmask);
    if (gl == 0) t.split_cnt[slot] = 0;
  }
  return last != 0;
}

// Unit u of a row space: units [0, n_items) are chunks of the long rows
// (items[u] = {row, kItemSplit | slot, z, w}); units n_items.. are the short
// rows n_long.. one each.
struct Unit {
  uint32_t row, b, e;     // row and local entry range
  uint32_t slot;          // split slot or ~0
};

__device__ __forceinline__ Unit unit_of(const ItemList& L, uint32_t u, const uint32_t* off) {
  Unit x;
  if (u < L.n_items) {
    const uint4 it = L.items[u];
    x.row = it.x; x.b = it.z; x.e = it.w; x.slot = it.y & kItemMask;
  } else {
    x.row = L.n_long + (u - L.n_items);
    x.b = 0; x.e = off[x.row + 1] - off[x.row]; x.slot = 0xffffffffu;
  }
  return x;
}

// Phase 1: t_V (and, when do_a, t_A into ta_out) of the tile's 32 queries.
//   t_V[v] = sum_u c_uv(u,v) p_u;   t_A[a] = k_attr cnorm_a[a] sum_u w(u,a) rnorm_u[u] p_u
// In a normal round t_A was already pushed by the previous phase 2 into
// ta_scan: phase 1 then only counts its active attributes (Algorithm 4's n_p)
// and clears ta_zero, the buffer the coming phase 2 pushes into.
template <typename WA>
__device__ __forceinline__ void gphase1(const BCtx& c, RAcc* A, bool do_v, bool do_a, float* ta_out,
                                        const float* ta_scan, float* ta_zero, bool count) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane, gl = lane & (kGL - 1), gi = lane / kGL;
  const unsigned gmask = ((1u << kGL) - 1u) << (gi * kGL);
  const float* __restrict__ r_u = c.t.r_u;
  auto gp = [&](uint32_t u) {
    const float4 x = ld4(r_u + (size_t)u * kTile + kQL * gl);
    return make_float4(fmaxf(-x.x, 0.f), fmaxf(-x.y, 0.f), fmaxf(-x.z, 0.f), fmaxf(-x.w, 0.f));
  };
  Q4Partials part;
  if (ta_scan || ta_zero) {
    for (uint32_t a = c.gw * kGPW + gi; a < g.n_a; a += c.nw * kGPW) {
      const size_t i = (size_t)a * kTile + kQL * gl;
      if (ta_scan) {
        const float4 t = *reinterpret_cast<const float4*>(ta_scan + i);
        const uint32_t d = g.au_off[a + 1] - g.au_off[a];
        part.np[0] += t.x > 0.f ? d : 0; part.np[1] += t.y > 0.f ? d : 0;
        part.np[2] += t.z > 0.f ? d : 0; part.np[3] += t.w > 0.f ? d : 0;
      }
      if (ta_zero) *reinterpret_cast<float4*>(ta_zero + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  const uint32_t nuv = do_v ? g.b_v.n_items + (g.n_v - g.b_v.n_long) : 0u;
  const uint32_t nua = do_a ? g.b_a.n_items + (g.n_a - g.b_a.n_long) : 0u;
  const uint32_t total = nuv + nua;
  for (uint32_t base = c.gw * kGPW; base < total; base += c.nw * kGPW) {
    const uint32_t uix = base + gi;
    const bool ok = uix < total;
    const bool is_a = ok && uix >= nuv;
    Unit un{0, 0, 0, 0xffffffffu};
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    if (ok) un = is_a ? unit_of(g.b_a, uix - nuv, g.au_off) : unit_of(g.b_v, uix, g.vu_off);
    const uint32_t b = ok ? off[un.row] + un.b : 0, e = ok ? off[un.row] + un.e : 0;
    const uint32_t waves = warp_max_u32(is_a ? 0u : (e - b + kGL - 1) / kGL);
    // V rows and attribute rows in one warp: both gathers run, each group
    // keeps the one of its own kind (ranges are empty for the other)
    const float4 sv = group_accum(is_a ? 0u : b, is_a ? 0u : e, waves, gl,
        [&](uint32_t k, uint32_t& i, float& w) { i = ld_stream(g.vu_idx + k); w = ld_stream(g.vu_c + k); }, gp);
    const uint32_t waves_a = warp_max_u32(is_a ? (e - b + kGL - 1) / kGL : 0u);
    const float4 sa = group_accum(is_a ? b : 0u, is_a ? e : 0u, waves_a, gl,
        [&](uint32_t k, uint32_t& i, float& w) { i = ld_stream(g.au_idx + k); w = ld_stream(g.au_c + k); }, gp);
    if (!ok) continue;
    float4 s = is_a ? sa : sv;
    if (un.slot != 0xffffffffu) {
      const uint32_t slot = un.slot + (is_a ? g.b_v.n_split : 0);
      const uint32_t nch = is_a ? g.b_a.split_nchunks[un.slot] : g.b_v.split_nchunks[un.slot];
      float4 tot;
      if (!split_combine4(c.t, slot, nch, s, gl, gmask, &tot)) continue;
      s = tot;
    }
    const uint32_t R = un.row;
    if (!is_a) {
      *reinterpret_cast<float4*>(c.t.t_v + (size_t)R * kTile + kQL * gl) = s;
      const uint32_t d = g.vu_off[R + 1] - g.vu_off[R];
      part.np[0] += s.x > 0.f ? d : 0; part.np[1] += s.y > 0.f ? d : 0;
      part.np[2] += s.z > 0.f ? d : 0; part.np[3] += s.w > 0.f ? d : 0;
    } else {
      const float f = g.k_attr * g.cnorm_a[R];
      const float4 tv = make_float4(f * s.x, f * s.y, f * s.z, f * s.w);
      *reinterpret_cast<float4*>(ta_out + (size_t)R * kTile + kQL * gl) = tv;
      const uint32_t d = g.au_off[R + 1] - g.au_off[R];
      part.np[0] += tv.x > 0.f ? d : 0; part.np[1] += tv.y > 0.f ? d : 0;
      part.np[2] += tv.z > 0.f ? d : 0; part.np[3] += tv.w > 0.f ? d : 0;
    }
  }
  if (count) flush_q4<false>(part, A);
}

// Residue update of row u for this lane's 4 queries: reserve update of the
// queries that pushed u this round, then the mark for the next round.
// APPLIKE: APP or APP(S) (per-node thresholds possible, r_max read per query);
// APPS: APP(S)'s round statistics too.  ASRP launches compile neither.
template <bool APPLIKE, bool APPS>
__device__ __forceinline__ float4 gepilogue2(const BCtx& c, uint32_t u, float4 s, uint32_t cnt,
                                             const float* th, const int* act, const int* pn,
                                             const LaneCtl* ctl, Q4Partials& part) {
  float4 pushed = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!(act[0] | act[1] | act[2] | act[3])) return pushed;
  float* pp4 = &pushed.x;
  const uint32_t gl = c.lane & (kGL - 1);
  const size_t i = (size_t)u * kTile + kQL * gl;
  float4* rp = reinterpret_cast<float4*>(c.t.r_u + i);
  float4* pp = reinterpret_cast<float4*>(c.t.pi + i);
  float4* cp = reinterpret_cast<float4*>(c.t.pic + i);
  float4 r = *rp;
  float4 pv = ld_stream(pp), pc = ld_stream(cp);
  float* rr = &r.x;
  float* pvv = &pv.x;
  float* pcc = &pc.x;
  const float* ss = &s.x;
  bool pushed_any = false;
#pragma unroll
  for (int j = 0; j < kQL; ++j) {
    if (!act[j]) continue;
    float kept = rr[j];
    if (kept < 0.f) {
      const float add = c.g.alpha * (-kept);
      if (c.p.kahan) kahan_add(pvv[j], pcc[j], add);
      else pvv[j] += add;
      kept = 0.f;
      pushed_any = true;
    }
    const float r_new = kept + ss[j];
    part.max_r[j] = fmaxf(part.max_r[j], r_new);
    bool mark;
    if (APPLIKE) {
      const double rmx = ctl[kQL * gl + j].eps_f;         // APP's r_max for per-node thresholds
      if (APPS) {
        if (cnt) part.max_rel[j] = fmaxf(part.max_rel[j], r_new / (float)cnt);
        if ((double)r_new > rmx * (double)cnt) part.above[j] += 1;
      }
      mark = pn[j] ? (double)r_new > rmx * (double)cnt : r_new >= th[j];
    } else {
      mark = r_new >= th[j];
    }
    if (mark) {
      rr[j] = -r_new;
      pp4[j] = r_new;
      part.marked[j] += 1;
      part.mdeg[j] += cnt;
    } else {
      rr[j] = r_new;
    }
  }
  *rp = r;
  if (pushed_any) { __stcs(pp, pv); __stcs(cp, pc); }
  return pushed;
}

// Attribute hop of the coming round, pushed as soon as u is marked: for every
// a in A(u), t_A'[a] += k_attr cnorm_a[a] w(u,a) rnorm_u[u] p_u (Eq. 2's two
// factors and Algorithm 3's U-push share, precomputed per entry as ua_pc), one
// float4 reduction per lane and attribute; t_A' is small enough to stay in L2.
template <typename WA>
__device__ __forceinline__ void push_attr(const DevGraph& g, uint32_t u, float4 p, float* ta_push,
                                          uint32_t gl, unsigned gmask) {
  const bool mine = p.x > 0.f || p.y > 0.f || p.z > 0.f || p.w > 0.f;
  if (!__any_sync(gmask, mine)) return;               // group-uniform
  const uint32_t b = g.ua_off[u], e = g.ua_off[u + 1];
  // waves of kGL entries (one per lane of the group, coalesced); every lane
  // then issues one float4 reduction per entry for its 4 queries
  for (uint32_t k0 = b; k0 < e; k0 += kGL) {
    const uint32_t n = min((uint32_t)kGL, e - k0);
    uint32_t mi = 0;
    float mc = 0.f;
    if (gl < n) {
      mi = g.ua_idx[k0 + gl];
      mc = ld_stream(g.ua_pc + k0 + gl);
    }
#pragma unroll
    for (int t = 0; t < kGL; ++t) {
      const uint32_t a = __shfl_sync(gmask, mi, t, kGL);
      const float cf = __shfl_sync(gmask, mc, t, kGL);
      if ((uint32_t)t < n && mine)
        red_add4(ta_push + (size_t)a * kTile + kQL * gl, make_float4(cf * p.x, cf * p.y, cf * p.z, cf * p.w));
    }
  }
}

// Phase 2: new residues of every U node for the tile's 32 queries.
template <typename WA, bool APPLIKE, bool APPS>
__device__ __forceinline__ void gphase2(const BCtx& c, const LaneCtl* ctl, RAcc* A,
                                        const float* ta_in, float* ta_push) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane, gl = lane & (kGL - 1), gi = lane / kGL;
  const unsigned gmask = ((1u << kGL) - 1u) << (gi * kGL);
  // mark thresholds and activity of this lane's 4 queries: APP's per-node
  // thresholds (pn), or one threshold (eps_f, or 0 once synchronous)
  float th[kQL];
  int act[kQL], pn[kQL];
#pragma unroll
  for (int j = 0; j < kQL; ++j) {
    const LaneCtl& q = ctl[kQL * gl + j];
    act[j] = q.active;
    pn[j] = APPLIKE ? per_node_threshold(c.p.algo, q.phase) : 0;
    th[j] = pn[j] ? 0.f : threshold_up(q.phase == kPhaseSync ? 0.0 : q.eps_f);
  }
  const float* __restrict__ t_v = c.t.t_v;
  const float* __restrict__ t_a = ta_in;
  auto gv = [&](uint32_t v) { return ld4(t_v + (size_t)v * kTile + kQL * gl); };
  auto ga = [&](uint32_t a) { return ld4(t_a + (size_t)a * kTile + kQL * gl); };
  Q4Partials part;
  const uint32_t total = g.b_u.n_items + (g.n_u - g.b_u.n_long);
  for (uint32_t base = c.gw * kGPW; base < total; base += c.nw * kGPW) {
    const uint32_t uix = base + gi;
    const bool ok = uix < total;
    uint32_t u = 0, z = 0, w = 0, slot = 0xffffffffu, b1 = 0, dv = 0, b2 = 0, da = 0;
    if (ok) {
      if (uix < g.b_u.n_items) {
        const uint4 it = g.b_u.items[uix];
        u = it.x; z = it.z; w = it.w; slot = it.y & kItemMask;
      } else {
        u = g.b_u.n_long + (uix - g.b_u.n_items);
      }
      b1 = g.uv_off[u]; dv = g.uv_off[u + 1] - b1;
      b2 = g.ua_off[u]; da = g.ua_off[u + 1] - b2;
      if (slot == 0xffffffffu) { z = 0; w = dv + da; }
    }
    // chunk [z, w) of the combined list: V neighbours first, then attributes
    const uint32_t vb = b1 + min(z, dv), ve = b1 + min(w, dv);
    const uint32_t ab = b2 + (z > dv ? z - dv : 0), ae = b2 + (w > dv ? w - dv : 0);
    const uint32_t sv = warp_max_u32((ve - vb + kGL - 1) / kGL), sa = warp_max_u32((ae - ab + kGL - 1) / kGL);
    float4 s = group_accum(vb, ve, sv, gl,
        [&](uint32_t k, uint32_t& i, float& wt) { i = ld_stream(g.uv_idx + k); wt = ld_stream(g.uv_w + k); }, gv);
    const float4 s2 = group_accum(ab, ae, sa, gl,
        [&](uint32_t k, uint32_t& i, float& wt) { i = ld_stream(g.ua_idx + k); wt = wload<WA>(g.ua_w, k); }, ga);
    if (!ok) continue;
    s = make_float4(s.x + s2.x, s.y + s2.y, s.z + s2.z, s.w + s2.w);
    if (slot != 0xffffffffu) {
      const uint32_t sl = slot + g.b_v.n_split + g.b_a.n_split;
      float4 tot;
      if (!split_combine4(c.t, sl, g.b_u.split_nchunks[slot], s, gl, gmask, &tot)) continue;
      s = tot;
    }
    const float4 pushed = gepilogue2<APPLIKE, APPS>(c, u, s, dv + da, th, act, pn, ctl, part);
    if (ta_push) push_attr<WA>(g, u, pushed, ta_push, gl, gmask);
  }
  flush_q4<APPS>(part, A);
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

// One persistent cooperative kernel for both batched queries (SERVE = false:
// n queries packed into tiles, each tile run to completion) and serving steps
// (SERVE = true: every lane of a tile is a slot; NEW slots are admitted into
// tiles already in flight, each live tile advances rounds_per_step rounds,
// slots that finish are finalised and their top-k extracted).
template <typename WA, bool SERVE>
__global__ void __launch_bounds__(kBThreads, kBMinBlocks)
k_tiles(const __grid_constant__ DevGraph g, const __grid_constant__ BatchState st,
        const __grid_constant__ BatchParams p, const __grid_constant__ ServeParams sv) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // Per-query control of the current tile, one entry per lane / query.  Warp 0
  // of every block makes the decisions (all blocks read the same round
  // accumulators after a barrier, so they agree); the phases read it here.
  __shared__ LaneCtl s_ctl[kTile];
  __shared__ unsigned long long s_mdeg[kTile];
  __shared__ int s_switch[kTile];
  __shared__ int s_new[kTile];       // serving: slot admitted at this step
  __shared__ int s_fin[kTile];       // lane finished: finalise and select top-k
  __shared__ uint32_t s_k[kTile];    // top-k size of the lane
  __shared__ int s_pick_d[kTile];    // top-k: digit, keys above it and its count, per lane
  __shared__ uint32_t s_pick_cum[kTile], s_pick_h[kTile];
  __shared__ int s_flag;
  __shared__ TileBuf s_tb;
  const uint32_t groups = SERVE ? 1u : p.groups;
  const uint32_t nbg = gridDim.x / groups;              // blocks per group
  const uint32_t grp = blockIdx.x / nbg;
  if (grp >= groups) return;                            // leftover blocks
  const uint32_t bid = blockIdx.x - grp * nbg;          // block id within the group
  const TileBuf& tb = s_tb;
  BCtx c{g, tb, p, (bid * kBThreads + threadIdx.x) >> 5, (nbg * kBThreads) >> 5,
         bid * kBThreads + threadIdx.x, nbg * kBThreads, threadIdx.x & 31u};
  const uint32_t lane = c.lane;
  const bool lq = lane < (uint32_t)kTile;               // this lane stands for a query
  const bool warp0 = threadIdx.x < 32;
  const bool app = p.algo != kAlgoASRP;   // APP's r_max as eps_f, per-node threshold for the source
  const uint32_t n_work = SERVE ? sv.n_live : (p.n + kTile - 1) / kTile;
  const uint32_t n_split = g.b_v.n_split + g.b_a.n_split + g.b_u.n_split;
  const size_t nu32 = (size_t)g.n_u * kTile;
  const uint32_t kmax = p.kmax;

  for (uint32_t w = grp; w < n_work; w += groups) {
    const uint32_t tile = SERVE ? sv.live[w] : w;
    const TileBuf* tg = SERVE ? &sv.tbufs[tile] : &st.tb[grp];
    if (threadIdx.x == 0) s_tb = *tg;
    __syncthreads();
    const uint32_t qi = tile * kTile + lane;            // query (batch) or slot (serve) index
    uint32_t tround = SERVE ? sv.tile_round[tile] : 0u;

    // ---- admission: the initial state of Algorithm 3 (unit residue at the source) for every new lane
    if (!SERVE) {
      for (size_t i = c.gt; i < nu32; i += c.nt) { tb.r_u[i] = 0.f; tb.pi[i] = 0.f; tb.pic[i] = 0.f; }
      for (size_t i = c.gt; i < (size_t)g.n_v * kTile; i += c.nt) tb.t_v[i] = 0.f;
      for (size_t i = c.gt; i < (size_t)g.n_a * kTile; i += c.nt) { tb.t_a[i] = 0.f; tb.t_a2[i] = 0.f; }
      for (size_t i = c.gt; i < (size_t)n_split * kTile; i += c.nt) tb.split_acc[i] = 0.f;
      for (size_t i = c.gt; i < n_split; i += c.nt) tb.split_cnt[i] = 0;
      if (c.gt < 5 * kTile) tb.racc[c.gt] = RAcc{};
    }
    if (warp0) {
      LaneCtl L{0.0, 0, 0, 0, 0, kPhaseAsync, kStatusOk, 0, 0};
      int is_new = 0;
      uint32_t kk = 0;
      if (!SERVE) {
        const bool in_range = lq && qi < p.n;
        const bool bad = in_range && (p.q[qi] >= g.n_u || !(p.eps[qi] > 0.0));
        if (bad) L.status = kStatusBadArg;
        if (in_range && !bad) {
          L.eps_f = app ? p.eps[qi] / (double)p.e_tot : p.eps[qi] / p.lambda;
          L.active = 1;
          L.valid = 1;
          is_new = 1;
          kk = kmax ? min(min(p.k[qi], kmax), g.n_u) : 0u;
        }
      } else if (lq) {
        const SlotState& S = sv.slots[qi];
        kk = S.k;
        if (S.state == kSlotNew) {
          L.eps_f = S.eps_f;
          L.active = 1;
          L.valid = 1;
          is_new = 1;
        } else if (S.state == kSlotRunning) {
          L = S.ctl;
        }
      }
      if (lq) { s_ctl[lane] = L; s_new[lane] = is_new; s_k[lane] = kk; s_fin[lane] = 0; }
      const int any = __any_sync(kFull, is_new);
      if (lane == 0) s_flag = any;
    }
    __syncthreads();
    if (SERVE && s_flag) {
      // clear the new lanes' columns (the other lanes keep running)
      const bool nw = lq && s_new[lane];
      for (size_t u = c.gw; nw && u < g.n_u; u += c.nw) {
        const size_t i = u * kTile + lane;
        tb.r_u[i] = 0.f; tb.pi[i] = 0.f; tb.pic[i] = 0.f;
      }
      for (size_t a = c.gw; nw && a < g.n_a; a += c.nw) {
        tb.t_a[a * kTile + lane] = 0.f;
        tb.t_a2[a * kTile + lane] = 0.f;
      }
      if (bid == 0 && nw) {
        for (int r = 0; r < 5; ++r) tb.racc[r * kTile + lane] = RAcc{};
      }
    }
    if (!grid_sync(tb.bar, nbg)) return;
    if (bid == 0 && warp0 && lq && s_new[lane]) {
      const uint32_t q_new = SERVE ? sv.slots[qi].q_new : p.u_old2new[p.q[qi]];
      const uint32_t cnt = (g.uv_off[q_new + 1] - g.uv_off[q_new]) + (g.ua_off[q_new + 1] - g.ua_off[q_new]);
      const double th = app ? s_ctl[lane].eps_f * (double)cnt : s_ctl[lane].eps_f;
      RAcc* a0 = &tb.racc[((tround + 2) % 3) * kTile + lane];
      *a0 = RAcc{};
      if (1.0 > th) {
        tb.r_u[(size_t)q_new * kTile + lane] = -1.f;
        a0->marked = 1;
        a0->marked_deg = cnt;
        // the source's attribute push of the first round (see push_attr)
        float* ta_cur = (tround & 1) ? tb.t_a2 : tb.t_a;
        for (uint32_t k = g.ua_off[q_new]; k < g.ua_off[q_new + 1]; ++k)
          ta_cur[(size_t)g.ua_idx[k] * kTile + lane] += g.ua_pc[k];
      } else {
        tb.r_u[(size_t)q_new * kTile + lane] = 1.f;
      }
    }
    if (!grid_sync(tb.bar, nbg)) return;

    // ---- rounds (Algorithm 3 / 4) for the active lanes
    Partials part;
    bool wait_fail = false;
    const uint32_t max_r = SERVE ? sv.rounds_per_step : 0xffffffffu;
    for (uint32_t done_r = 0;; ++done_r) {
      RAcc* A = &tb.racc[(tround % 3) * kTile];
      const RAcc* P = &tb.racc[((tround + 2) % 3) * kTile];
      if (warp0) {
        LaneCtl L{};
        if (lq) {
          L = s_ctl[lane];
          const uint32_t marked = __ldcg(&P[lane].marked);
          s_mdeg[lane] = __ldcg(&P[lane].marked_deg);
          if (L.active && (L.phase == kPhaseDone || marked == 0)) { L.phase = kPhaseDone; L.active = 0; s_fin[lane] = 1; }
          if (L.active && L.rounds >= p.max_rounds) { L.status = kStatusCap; L.active = 0; s_fin[lane] = 1; }
          if (L.active && done_r < max_r) L.pushes += marked;
          s_ctl[lane] = L;
        }
        const int any = __any_sync(kFull, L.active);
        if (lane == 0) s_flag = any && done_r < max_r;
      }
      __syncthreads();
      if (!s_flag) break;
      if (bid == 0 && threadIdx.x < kTile) tb.racc[((tround + 1) % 3) * kTile + threadIdx.x] = RAcc{};

      float* ta_cur = (tround & 1) ? tb.t_a2 : tb.t_a;     // t_A of this round
      float* ta_next = (tround & 1) ? tb.t_a : tb.t_a2;    // t_A of the next round
      gphase1<WA>(c, A, true, false, nullptr, ta_cur, ta_next, true);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      if (p.algo == kAlgoASRP) gphase2<WA, false, false>(c, s_ctl, A, ta_cur, ta_next);
      else if (p.algo == kAlgoAPP) gphase2<WA, true, false>(c, s_ctl, A, ta_cur, ta_next);
      else gphase2<WA, true, true>(c, s_ctl, A, ta_cur, ta_next);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      ++tround;

      if (warp0) {
        LaneCtl L{};
        if (lq) L = s_ctl[lane];
        int switched = 0;
        if (L.active) {
          ++L.rounds;
          const float M = __uint_as_float(__ldcg(&A[lane].max_r_bits));
          L.n_p += s_mdeg[lane] + __ldcg(&A[lane].np_flush);
          if (p.algo == kAlgoASRP) {
            if ((double)M <= L.eps_f) {
              L.phase = kPhaseDone;
              L.active = 0;
              s_fin[lane] = 1;
            } else if (L.phase == kPhaseAsync && (double)L.n_p >= bbudget(p, L.eps_f, (double)M)) {
              L.phase = kPhaseSync;
              L.switch_round = L.rounds + 1;
              switched = 1;
            }
          } else if (p.algo == kAlgoAPPS) {
            // APP's stopping test; the switch budget in units of APP's thresholds
            const float Mrel = __uint_as_float(__ldcg(&A[lane].max_rel_bits));
            if (__ldcg(&A[lane].above) == 0) {
              L.phase = kPhaseDone;
              L.active = 0;
              s_fin[lane] = 1;
            } else if (L.phase == kPhaseAsync && (double)L.n_p >= bbudget(p, L.eps_f, (double)Mrel)) {
              L.phase = kPhaseSync;
              L.switch_round = L.rounds + 1;
              switched = 1;
            }
          }
        }
        if (lq) {
          s_ctl[lane] = L;
          s_switch[lane] = switched;
        }
        const int any = __any_sync(kFull, switched);
        if (lane == 0) s_flag = any;
      }
      __syncthreads();
      if (s_flag) {
        // first synchronous round pushes every positive residue of that query
        const bool sw = lq && s_switch[lane] != 0;
        for (size_t u = c.gw; u < g.n_u; u += c.nw) {
          const size_t i = u * kTile + (lq ? lane : 0);
          const float r = sw ? tb.r_u[i] : 0.f;
          if (sw && r > 0.f) {
            tb.r_u[i] = -r;
            part.marked += 1;
            part.marked_deg += (g.uv_off[u + 1] - g.uv_off[u]) + (g.ua_off[u + 1] - g.ua_off[u]);
          }
        }
        flush_lane_partials(part, A);
        if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
        // the new marks also push into the next round's t_A: recompute it by
        // the pull form from the complete marks (once per switch)
        gphase1<WA>(c, A, false, true, (tround & 1) ? tb.t_a2 : tb.t_a, nullptr, nullptr, false);
        if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      }
    }
    if (wait_fail && warp0 && lq && s_ctl[lane].valid) {
      s_ctl[lane].status = kStatusWait;
      s_ctl[lane].active = 0;
      s_fin[lane] = 1;
    }
    __syncthreads();
    const bool fin = lq && s_fin[lane] && s_ctl[lane].valid;
    const uint32_t kq = fin ? s_k[lane] : 0u;
    int any_fin = 0;
    for (int l = 0; l < kTile; ++l) any_fin |= s_fin[l];

    if (any_fin) {
      // ---- reserves = pi - compensation; per-query sums; dense output
      {
        Partials pr, pp;
        for (size_t u = c.gw; fin && u < g.n_u; u += c.nw) {
          const size_t i = u * kTile + lane;
          const float v = fmaxf(tb.pi[i] - tb.pic[i], 0.f);
          tb.pi[i] = v;
          const float r = fabsf(tb.r_u[i]);
          pr.sum_r += (double)r;
          pr.max_r = fmaxf(pr.max_r, r);
          pp.sum_r += (double)v;
          if (!SERVE && p.out_dense) p.out_dense[(size_t)qi * g.n_u + p.u_new2old[u]] = v;
        }
        flush_lane_partials(pr, &tb.racc[3 * kTile]);   // residues: sum and max
        flush_lane_partials(pp, &tb.racc[4 * kTile]);   // reserves: sum
        for (size_t i = c.gt; i < (size_t)kRadixPasses * kTile * kRadixBins; i += c.nt) tb.hist[i] = 0;
        if (c.gt < kTile) tb.cand_cnt[c.gt] = 0;
      }
      if (!grid_sync(tb.bar, nbg)) return;

      if (bid == 0 && fin) {
        const LaneCtl L = s_ctl[lane];
        ahpp_stats S;
        S.rounds = L.rounds;
        S.switch_round = L.switch_round;
        S.dense_rounds = L.rounds;
        S.status = (uint32_t)((L.status == kStatusOk && L.phase != kPhaseDone) ? kStatusCap : L.status);
        S.pushes = L.pushes;
        S.n_p = L.n_p;
        S.reserve_sum = __ldcg(&tb.racc[4 * kTile + lane].sum_r);
        S.resid_sum = __ldcg(&tb.racc[3 * kTile + lane].sum_r);
        S.mass_err = fabs(S.reserve_sum + S.resid_sum - 1.0);
        S.max_resid = (double)__uint_as_float(__ldcg(&tb.racc[3 * kTile + lane].max_r_bits));
        S.lambda = p.lambda;
        S.eps_f = L.eps_f;
        S.served_ms = 0.0;
        if (p.out_stats) p.out_stats[qi] = S;
      }

      // ---- top-k per lane: radix select over 64-bit (score, ~caller id) keys.
      // A lane stops as soon as the bucket holding its k-th key contains
      // exactly the keys it still needs (then every key of that bucket is a
      // winner); with distinct scores that happens once the score bits are
      // resolved, so the caller-id passes are skipped.
      if (kmax) {
        unsigned int* sh = reinterpret_cast<unsigned int*>(smem);    // [kTile][kRadixBins]
        unsigned long long prefix = 0;
        unsigned long long thresh = 0;        // smallest winning key, once known
        uint32_t krem = kq;
        bool known = kq == 0;
        for (int pass = 0; pass < kRadixPasses; ++pass) {
          // every block holds the same per-lane state (read from the same
          // global histograms), so all blocks leave the loop together
          if (!__syncthreads_or(!known)) break;
          const int shift = 64 - kRadixBits * (pass + 1);
          for (int i = threadIdx.x; i < kTile * kRadixBins; i += kBThreads) sh[i] = 0;
          __syncthreads();
          if (!known) {
            for (size_t u = c.gw; u < g.n_u; u += c.nw) {
              const unsigned long long key = score_key(tb.pi[u * kTile + lane], p.u_new2old[u]);
              if (pass == 0 || (key >> (shift + kRadixBits)) == prefix)
                atomicAdd(&sh[lane * kRadixBins + ((key >> shift) & (kRadixBins - 1))], 1u);
            }
          }
          __syncthreads();
          unsigned int* gh = tb.hist + (size_t)pass * kTile * kRadixBins;
          for (int i = threadIdx.x; i < kTile * kRadixBins; i += kBThreads)
            if (sh[i]) atomicAdd(&gh[i], sh[i]);
          if (!grid_sync(tb.bar, nbg)) return;
          // the merged histograms into shared memory; warp w picks the digit
          // of queries w, w + 8, ... (warp-parallel), lane l reads query l's
          for (int i = threadIdx.x; i < kTile * kRadixBins; i += kBThreads) sh[i] = __ldcg(&gh[i]);
          __syncthreads();
          for (int l = threadIdx.x >> 5; l < kTile; l += kBWarps) {
            const uint32_t kr = __shfl_sync(kFull, krem, l);
            if (__shfl_sync(kFull, (int)known, l)) continue;
            int dd;
            uint32_t cc, hh;
            radix_pick(sh + l * kRadixBins, kRadixBins, kr, &dd, &cc, &hh);
            if ((threadIdx.x & 31) == 0) { s_pick_d[l] = dd; s_pick_cum[l] = cc; s_pick_h[l] = hh; }
          }
          __syncthreads();
          if (!known) {
            const int d = s_pick_d[lane];
            const uint32_t cum = s_pick_cum[lane], h = s_pick_h[lane];
            krem -= cum;
            prefix = (prefix << kRadixBits) | (unsigned long long)d;
            if (h == krem || shift == 0) {
              known = true;
              thresh = prefix << shift;
            }
          }
        }
        // the lane's winners are exactly its keys >= thresh (keys are distinct)
        if (kq) {
          for (size_t u = c.gw; u < g.n_u; u += c.nw) {
            const unsigned long long key = score_key(tb.pi[u * kTile + lane], p.u_new2old[u]);
            if (key >= thresh) {
              const uint32_t pos = atomicAdd(&tb.cand_cnt[lane], 1u);
              if (pos < kmax) tb.cand[(size_t)lane * kmax + pos] = key;
            }
          }
        }
        if (!grid_sync(tb.bar, nbg)) return;
        // sort each lane's keys descending (bitonic in shared memory), one block per lane
        unsigned long long* sk = reinterpret_cast<unsigned long long*>(smem);
        for (uint32_t l = bid; l < kTile; l += nbg) {
          if (!s_fin[l] || !s_ctl[l].valid) continue;
          const uint32_t ql = tile * kTile + l;
          const uint32_t kl = s_k[l];
          uint32_t m = 1;
          while (m < kl) m <<= 1;
          for (uint32_t i = threadIdx.x; i < m; i += kBThreads)
            sk[i] = i < kl ? tb.cand[(size_t)l * kmax + i] : 0ull;
          __syncthreads();
          for (uint32_t size = 2; size <= m; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
              for (uint32_t i = threadIdx.x; i < m; i += kBThreads) {
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
          for (uint32_t i = threadIdx.x; i < kl; i += kBThreads) {
            const unsigned long long key = sk[i];
            p.out_nodes[(size_t)ql * kmax + i] = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
            p.out_scores[(size_t)ql * kmax + i] = __uint_as_float((uint32_t)(key >> 32));
          }
          if (threadIdx.x == 0) p.out_n[ql] = kl;
          __syncthreads();
        }
      } else if (bid == 0 && fin && p.out_n) {
        p.out_n[qi] = 0;
      }
    }
    // ---- bad arguments (batch): report and produce no result
    if (!SERVE && bid == 0 && lq && qi < p.n && s_ctl[lane].status == kStatusBadArg) {
      if (p.out_stats) {
        ahpp_stats S{};
        S.status = kStatusBadArg;
        p.out_stats[qi] = S;
      }
      if (p.out_n) p.out_n[qi] = 0;
    }
    // ---- serving: persist the slots' control and the tile's round counter
    if (SERVE && bid == 0 && warp0) {
      if (lq) {
        SlotState& S = sv.slots[qi];
        if (S.state == kSlotNew || S.state == kSlotRunning) {
          S.ctl = s_ctl[lane];
          S.state = s_fin[lane] ? kSlotFinished : kSlotRunning;
        }
      }
      if (lane == 0) sv.tile_round[tile] = tround;
    }
    if (!grid_sync(tb.bar, nbg)) return;
  }
}

template __global__ void k_tiles<float, false>(const __grid_constant__ DevGraph,
                                               const __grid_constant__ BatchState,
                                               const __grid_constant__ BatchParams,
                                               const __grid_constant__ ServeParams);
template __global__ void k_tiles<__nv_bfloat16, false>(const __grid_constant__ DevGraph,
                                                       const __grid_constant__ BatchState,
                                                       const __grid_constant__ BatchParams,
                                                       const __grid_constant__ ServeParams);
#if AHPP_BT == 32   // serving runs tiles of 32 only
template __global__ void k_tiles<float, true>(const __grid_constant__ DevGraph,
                                              const __grid_constant__ BatchState,
                                              const __grid_constant__ BatchParams,
                                              const __grid_constant__ ServeParams);
template __global__ void k_tiles<__nv_bfloat16, true>(const __grid_constant__ DevGraph,
                                                      const __grid_constant__ BatchState,
                                                      const __grid_constant__ BatchParams,
                                                      const __grid_constant__ ServeParams);
#endif


namespace {
const void* tiles_fn(bool bf16, bool serve) {
  static bool attr_set = false;
  if (!attr_set) {
    attr_set = true;
    for (const void* f : {(const void*)k_tiles<__nv_bfloat16, false>, (const void*)k_tiles<float, false>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
#if AHPP_BT == 32
    for (const void* f : {(const void*)k_tiles<__nv_bfloat16, true>, (const void*)k_tiles<float, true>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
#endif
  }
#if AHPP_BT == 32
  if (serve) return bf16 ? (const void*)k_tiles<__nv_bfloat16, true> : (const void*)k_tiles<float, true>;
#else
  (void)serve;
#endif
  return bf16 ? (const void*)k_tiles<__nv_bfloat16, false> : (const void*)k_tiles<float, false>;
}
}  // namespace

int launch_batch(const DevGraph& g, const BatchState& s, const BatchParams& p, bool bf16,
                 int grid, cudaStream_t stream) {
  ServeParams sv{};
  void* args[] = {(void*)&g, (void*)&s, (void*)&p, (void*)&sv};
  cudaError_t e = cudaLaunchCooperativeKernel(tiles_fn(bf16, false), dim3(grid), dim3(kBThreads), args,
                                              kBatchSmem, stream);
  return e == cudaSuccess ? 0 : (int)e;
}

#if AHPP_BT == 32
int launch_serve_step(const DevGraph& g, const BatchParams& p, const ServeParams& sv, bool bf16,
                      int grid, cudaStream_t stream) {
  BatchState s{};
  void* args[] = {(void*)&g, (void*)&s, (void*)&p, (void*)&sv};
  cudaError_t e = cudaLaunchCooperativeKernel(tiles_fn(bf16, true), dim3(grid), dim3(kBThreads), args,
                                              kBatchSmem, stream);
  return e == cudaSuccess ? 0 : (int)e;
}
#endif

int batch_max_grid(bool bf16, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tiles_fn(bf16, false), kBThreads, kBatchSmem) !=
          cudaSuccess || per_sm <= 0)
    return -1;
#if AHPP_BT == 32
  int per_sm2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, tiles_fn(bf16, true), kBThreads, kBatchSmem) !=
          cudaSuccess || per_sm2 <= 0)
    return -1;
  per_sm = std::min(per_sm, per_sm2);
#endif
  return per_sm * sm_count;
}

}  // namespace AHPP_BT_NS
}  // namespace ahpp
