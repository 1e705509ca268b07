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
#include "ahpp_tma.cuh"

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
#ifndef AHPP_ATTR_PUSH
#define AHPP_ATTR_PUSH 1          // attribute hop pushed from phase 2 (1) or pulled in phase 1 (0); 1 measured faster
#endif
#ifndef AHPP_TMA
#define AHPP_TMA 0                // 1: pull phases gather rows with TMA tile::gather4 (correct, measured 2.6x slower)
#endif
#ifndef AHPP_P1_PASSES
#define AHPP_P1_PASSES 1          // 2: phase 1 gathers the two halves of U in separate passes (measured slower)
#endif
#ifndef AHPP_BATCH_MINB
#define AHPP_BATCH_MINB (AHPP_TMA ? 2 : (AHPP_ATTR_PUSH ? 3 : 4))   // resident blocks per SM the register budget targets (measured best)
#endif

// Smallest float f with (r > th) <=> (r >= f) for every float r: the mark
// test r > th of Algorithm 4 taken exactly against the FP64 threshold.
__device__ __forceinline__ float threshold_up(double th) {
  float f = (float)th;
  if ((double)f <= th) f = nextafterf(f, INFINITY);
  return f;
}

// Gathered state (r_U rows in phase 1, t_V / t_A rows in phase 2) is loaded
// with the L2 evict-last policy so that the streamed graph arrays (loaded
// evict-first) do not push it out of L2 during a phase.
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
#ifndef AHPP_GATHER_HINT
#define AHPP_GATHER_HINT 0        // gathers load with the L2 evict-last policy (measured slower)
#endif
#ifndef AHPP_STREAM_HINT
#define AHPP_STREAM_HINT 1        // graph arrays and reserves are streamed with evict-first loads
#endif
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
#if AHPP_STREAM_HINT
  return __ldcs(p);
#else
  return *p;
#endif
}
#ifndef AHPP_STORE_HINT
#define AHPP_STORE_HINT 0         // rows that the next phase gathers are stored evict-last
#endif
__device__ __forceinline__ float4 ld_keep4(const float* p, uint64_t pol) {
#if AHPP_GATHER_HINT
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
#else
  return *reinterpret_cast<const float4*>(p);
#endif
}
__device__ __forceinline__ void st_keep4(float* p, float4 v) {
#if AHPP_STORE_HINT
  const uint64_t pol = policy_keep();
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
               :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
#else
  *reinterpret_cast<float4*>(p) = v;
#endif
}

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
};

__device__ __forceinline__ void flush_q4(Q4Partials& p, RAcc* acc) {
  __shared__ float s_max[kWarps][32];
  __shared__ uint32_t s_mk[kWarps][32], s_dg[kWarps][32], s_np[kWarps][32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kQL; ++j) {
#pragma unroll
    for (int o = kGL; o < 32; o <<= 1) {
      p.max_r[j] = fmaxf(p.max_r[j], __shfl_xor_sync(kFull, p.max_r[j], o));
      p.marked[j] += __shfl_xor_sync(kFull, p.marked[j], o);
      p.mdeg[j] += __shfl_xor_sync(kFull, p.mdeg[j], o);
      p.np[j] += __shfl_xor_sync(kFull, p.np[j], o);
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
    for (int w = 0; w < kWarps; ++w) {
      m = fmaxf(m, s_max[w][lane]); mk += s_mk[w][lane];
      dg += s_dg[w][lane]; np += s_np[w][lane];
    }
    RAcc* a = &acc[lane];
    if (m > 0.f) atomicMax(&a->max_r_bits, __float_as_uint(m));
    if (mk) atomicAdd(&a->marked, mk);
    if (dg) atomicAdd(&a->marked_deg, dg);
    if (np) atomicAdd(&a->np_flush, np);
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
                                        const float* ta_scan, float* ta_zero, bool count,
                                        int pass = 0, int npass = 1) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane, gl = lane & (kGL - 1), gi = lane / kGL;
  const unsigned gmask = ((1u << kGL) - 1u) << (gi * kGL);
  const float* __restrict__ r_u = c.t.r_u;
  const uint64_t pol = policy_keep();
  auto gp = [&](uint32_t u) {
    const float4 x = ld_keep4(r_u + (size_t)u * kTile + kQL * gl, pol);
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
    uint32_t b = ok ? off[un.row] + un.b : 0, e = ok ? off[un.row] + un.e : 0;
    if (ok && npass == 2) {
      // pass 0 gathers sources u < u_half, pass 1 the rest (entries sorted by u)
      const uint32_t mid = is_a ? g.au_mid[un.row] : g.vu_mid[un.row];
      if (pass == 0) e = max(b, min(e, mid));
      else b = min(e, max(b, mid));
    }
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
    float* out = is_a ? ta_out + (size_t)R * kTile + kQL * gl : c.t.t_v + (size_t)R * kTile + kQL * gl;
    if (npass == 2 && pass == 0) {             // partial sum of the first half
      *reinterpret_cast<float4*>(out) = s;
      continue;
    }
    if (npass == 2) {
      const float4 h = *reinterpret_cast<const float4*>(out);
      s = make_float4(s.x + h.x, s.y + h.y, s.z + h.z, s.w + h.w);
    }
    if (!is_a) {
      st_keep4(c.t.t_v + (size_t)R * kTile + kQL * gl, s);
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
  if (count) flush_q4(part, A);
}

// Residue update of row u for this lane's 4 queries: reserve update of the
// queries that pushed u this round, then the mark for the next round.
__device__ __forceinline__ float4 gepilogue2(const BCtx& c, uint32_t u, float4 s, uint32_t cnt,
                                             const float* th, const int* act, const LaneCtl* app_ctl,
                                             Q4Partials& part) {
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
    const bool mark = app_ctl ? (double)r_new > app_ctl[kQL * gl + j].eps_f * (double)cnt
                              : r_new >= th[j];
    if (mark) {
      rr[j] = -r_new;
      pp4[j] = r_new;
      part.marked[j] += 1;
      part.mdeg[j] += cnt;
    } else {
      rr[j] = r_new;
    }
  }
  st_keep4(c.t.r_u + i, r);
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
template <typename WA>
__device__ __forceinline__ void gphase2(const BCtx& c, const LaneCtl* ctl, RAcc* A,
                                        const float* ta_in, float* ta_push) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane, gl = lane & (kGL - 1), gi = lane / kGL;
  const unsigned gmask = ((1u << kGL) - 1u) << (gi * kGL);
  const bool app = c.p.algo == kAlgoAPP;
  // mark thresholds and activity of this lane's 4 queries
  float th[kQL];
  int act[kQL];
#pragma unroll
  for (int j = 0; j < kQL; ++j) {
    const LaneCtl& q = ctl[kQL * gl + j];
    act[j] = q.active;
    th[j] = app ? 0.f : threshold_up(q.phase == kPhaseSync ? 0.0 : q.eps_f);
  }
  const float* __restrict__ t_v = c.t.t_v;
  const float* __restrict__ t_a = ta_in;
  const uint64_t pol = policy_keep();
  auto gv = [&](uint32_t v) { return ld_keep4(t_v + (size_t)v * kTile + kQL * gl, pol); };
  auto ga = [&](uint32_t a) { return ld_keep4(t_a + (size_t)a * kTile + kQL * gl, pol); };
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
    const float4 pushed = gepilogue2(c, u, s, dv + da, th, act, app ? ctl : nullptr, part);
    if (ta_push) push_attr<WA>(g, u, pushed, ta_push, gl, gmask);
  }
  flush_q4(part, A);
}

// ------------------------------------------------------------------------
// TMA form of the pull phases (one query per lane; kTile == 32).  A warp
// owns an item (up to 32 consecutive rows, or one chunk of a long row) and
// walks its neighbour entries in stages of 32 through a two-buffer gather
// pipeline; row sums go to sp[row][lane] in shared memory.
#if AHPP_TMA
static_assert(kTile == 32, "the TMA phases map one query per lane");

template <bool ADD, typename LoadF, typename XF>
__device__ __forceinline__ void tma_rows(GatherPipe& gp, const CUtensorMap* map, uint32_t nrows,
                                         uint32_t my_end, uint32_t kb, uint32_t ke, uint32_t lane,
                                         LoadF load, XF xform, float* sp, unsigned int* err) {
  if (!ADD)
    for (uint32_t r = 0; r < nrows; ++r) sp[r * 32 + lane] = 0.f;
  const uint32_t nst = (ke - kb + kStage - 1) / kStage;
  uint32_t row = 0;
  uint32_t row_end = __shfl_sync(kFull, my_end, 0);
  float acc = 0.f;
  if (nst == 0) return;
  uint32_t idx = 0;
  float coef = 0.f, coef_next = 0.f;
  {
    const uint32_t n0 = min((uint32_t)kStage, ke - kb);
    if (lane < n0) load(kb + lane, idx, coef);
    pipe_issue(gp, 0, map, lane < n0 ? idx : 0u, n0, lane);
  }
  for (uint32_t st = 0; st < nst; ++st) {
    const int b = st & 1;
    const uint32_t k0 = kb + st * kStage;
    const uint32_t n = min((uint32_t)kStage, ke - k0);
    if (st + 1 < nst) {
      const uint32_t k1 = k0 + kStage;
      const uint32_t n1 = min((uint32_t)kStage, ke - k1);
      uint32_t i1 = 0;
      coef_next = 0.f;
      if (lane < n1) load(k1 + lane, i1, coef_next);
      pipe_issue(gp, b ^ 1, map, lane < n1 ? i1 : 0u, n1, lane);
    }
    pipe_wait(gp, b, err);
    const float* x = gp.buf + b * kStage * 32;
    for (uint32_t j = 0; j < n; ++j) {
      const float cj = __shfl_sync(kFull, coef, j);
      while (k0 + j >= row_end) {
        sp[row * 32 + lane] += acc;
        acc = 0.f;
        ++row;
        row_end = __shfl_sync(kFull, my_end, row & 31u);
      }
      acc = fmaf(cj, xform(x[j * 32 + lane]), acc);
    }
    __syncwarp();
    coef = coef_next;
  }
  if (row < nrows) sp[row * 32 + lane] += acc;
}

// Lane-scalar split-row combine (warp-collective): true for the chunk that
// finishes the row, with the row total in *tot.
__device__ __forceinline__ bool split_combine1(const TileBuf& t, uint32_t slot, uint32_t nch, float s,
                                               uint32_t lane, float* tot) {
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

// Item i of a TMA item list: rows [r0, r0 + nrows) whole, or one chunk.
struct TItem {
  uint32_t r0, nrows, z, w, slot;   // slot ~0: not split
  bool chunk;
};
__device__ __forceinline__ TItem titem(const ItemList& L, uint32_t i) {
  const uint4 it = L.items[i];
  TItem t;
  t.r0 = it.x;
  t.chunk = (it.y & (kItemLong | kItemSplit)) != 0;
  t.nrows = t.chunk ? 1u : it.y;
  t.z = it.z; t.w = it.w;
  t.slot = (it.y & kItemSplit) ? (it.y & kItemMask) : 0xffffffffu;
  return t;
}

template <typename WA>
__device__ __forceinline__ void tphase1(const BCtx& c, const TileBuf* tg, GatherPipe& gp, float* sp,
                                        RAcc* A, unsigned int* err) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane;
  Partials part;
  const uint32_t nv = g.m_v.n_items, total = nv + g.m_a.n_items;
  auto neg = [](float x) { return fmaxf(-x, 0.f); };
  for (uint32_t it = c.gw; it < total; it += c.nw) {
    const bool is_a = it >= nv;
    const TItem t = titem(is_a ? g.m_a : g.m_v, is_a ? it - nv : it);
    const uint32_t* off = is_a ? g.au_off : g.vu_off;
    uint32_t kb, ke, my_end;
    if (t.chunk) {
      kb = off[t.r0] + t.z; ke = off[t.r0] + t.w; my_end = ke;
    } else {
      kb = off[t.r0];
      my_end = lane < t.nrows ? off[t.r0 + lane + 1] : 0xffffffffu;
      ke = __shfl_sync(kFull, my_end, t.nrows - 1);
    }
    if (!is_a)
      tma_rows<false>(gp, &tg->map_ru, t.nrows, my_end, kb, ke, lane,
                      [&](uint32_t k, uint32_t& i, float& w) { i = ld_stream(g.vu_idx + k); w = ld_stream(g.vu_c + k); },
                      neg, sp, err);
    else
      tma_rows<false>(gp, &tg->map_ru, t.nrows, my_end, kb, ke, lane,
                      [&](uint32_t k, uint32_t& i, float& w) {
                        i = ld_stream(g.au_idx + k);
                        w = g.au_c[k];
                      },
                      neg, sp, err);
    for (uint32_t row = 0; row < t.nrows; ++row) {
      const uint32_t R = t.r0 + row;
      float s = sp[row * 32 + lane];
      if (t.slot != 0xffffffffu) {
        const uint32_t slot = t.slot + (is_a ? g.m_v.n_split : 0);
        const uint32_t nch = is_a ? g.m_a.split_nchunks[t.slot] : g.m_v.split_nchunks[t.slot];
        float tot;
        if (!split_combine1(c.t, slot, nch, s, lane, &tot)) continue;
        s = tot;
      }
      if (!is_a) {
        c.t.t_v[(size_t)R * kTile + lane] = s;
        if (s > 0.f) part.np_flush += g.vu_off[R + 1] - g.vu_off[R];
      } else {
        const float tv = g.k_attr * g.cnorm_a[R] * s;
        c.t.t_a[(size_t)R * kTile + lane] = tv;
        if (tv > 0.f) part.np_flush += g.au_off[R + 1] - g.au_off[R];
      }
    }
  }
  flush_lane_partials(part, A);
}

// Residue update of row u for this lane's query (see gepilogue2).
__device__ __forceinline__ void lepilogue2(const BCtx& c, uint32_t u, float s, uint32_t cnt, float th,
                                           bool act, const LaneCtl* app_ctl, Partials& part) {
  if (!act) return;
  const size_t i = (size_t)u * kTile + c.lane;
  const float r_old = c.t.r_u[i];
  float kept = r_old;
  if (r_old < 0.f) {
    const float add = c.g.alpha * (-r_old);
    if (c.p.kahan) {
      float pv = ld_stream(c.t.pi + i), pc = ld_stream(c.t.pic + i);
      kahan_add(pv, pc, add);
      __stcs(c.t.pi + i, pv);
      __stcs(c.t.pic + i, pc);
    } else {
      c.t.pi[i] += add;
    }
    kept = 0.f;
  }
  const float r_new = kept + s;
  part.max_r = fmaxf(part.max_r, r_new);
  const bool mark = app_ctl ? (double)r_new > app_ctl[c.lane].eps_f * (double)cnt : r_new >= th;
  if (mark) {
    c.t.r_u[i] = -r_new;
    part.marked += 1;
    part.marked_deg += cnt;
  } else {
    c.t.r_u[i] = r_new;
  }
}

template <typename WA>
__device__ __forceinline__ void tphase2(const BCtx& c, const TileBuf* tg, const LaneCtl* ctl,
                                        GatherPipe& gp, float* sp, RAcc* A, unsigned int* err) {
  const DevGraph& g = c.g;
  const uint32_t lane = c.lane;
  const bool app = c.p.algo == kAlgoAPP;
  const LaneCtl& me = ctl[lane];
  const bool act = me.active != 0;
  const float th = app ? 0.f : threshold_up(me.phase == kPhaseSync ? 0.0 : me.eps_f);
  auto id = [](float x) { return x; };
  auto lv = [&](uint32_t k, uint32_t& i, float& w) { i = ld_stream(g.uv_idx + k); w = ld_stream(g.uv_w + k); };
  auto la = [&](uint32_t k, uint32_t& i, float& w) { i = ld_stream(g.ua_idx + k); w = wload<WA>(g.ua_w, k); };
  Partials part;
  for (uint32_t it = c.gw; it < g.m_u.n_items; it += c.nw) {
    const TItem t = titem(g.m_u, it);
    if (t.chunk) {
      const uint32_t u = t.r0;
      const uint32_t b1 = g.uv_off[u], dv = g.uv_off[u + 1] - b1;
      const uint32_t b2 = g.ua_off[u], da = g.ua_off[u + 1] - b2;
      const uint32_t vb = b1 + min(t.z, dv), ve = b1 + min(t.w, dv);
      const uint32_t ab = b2 + (t.z > dv ? t.z - dv : 0), ae = b2 + (t.w > dv ? t.w - dv : 0);
      tma_rows<false>(gp, &tg->map_tv, 1, ve, vb, ve, lane, lv, id, sp, err);
      tma_rows<true>(gp, &tg->map_ta, 1, ae, ab, ae, lane, la, id, sp, err);
      float s = sp[lane];
      if (t.slot != 0xffffffffu) {
        const uint32_t sl = t.slot + g.m_v.n_split + g.m_a.n_split;
        float tot;
        if (!split_combine1(c.t, sl, g.m_u.split_nchunks[t.slot], s, lane, &tot)) continue;
        s = tot;
      }
      lepilogue2(c, u, s, dv + da, th, act, app ? ctl : nullptr, part);
    } else {
      const uint32_t r0 = t.r0, nrows = t.nrows;
      const uint32_t end_v = lane < nrows ? g.uv_off[r0 + lane + 1] : 0xffffffffu;
      const uint32_t end_a = lane < nrows ? g.ua_off[r0 + lane + 1] : 0xffffffffu;
      const uint32_t kv0 = g.uv_off[r0], ka0 = g.ua_off[r0];
      const uint32_t kv1 = __shfl_sync(kFull, end_v, nrows - 1);
      const uint32_t ka1 = __shfl_sync(kFull, end_a, nrows - 1);
      tma_rows<false>(gp, &tg->map_tv, nrows, end_v, kv0, kv1, lane, lv, id, sp, err);
      tma_rows<true>(gp, &tg->map_ta, nrows, end_a, ka0, ka1, lane, la, id, sp, err);
      const uint32_t beg_v = __shfl_up_sync(kFull, end_v, 1), beg_a = __shfl_up_sync(kFull, end_a, 1);
      const uint32_t my_cnt = lane < nrows ? (end_v - (lane ? beg_v : kv0)) + (end_a - (lane ? beg_a : ka0)) : 0u;
      for (uint32_t row = 0; row < nrows; ++row) {
        const uint32_t cnt = __shfl_sync(kFull, my_cnt, row);
        lepilogue2(c, r0 + row, sp[row * 32 + lane], cnt, th, act, app ? ctl : nullptr, part);
      }
    }
  }
  flush_lane_partials(part, A);
}
#endif  // AHPP_TMA

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
__global__ void __launch_bounds__(kThreads, AHPP_BATCH_MINB)
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
#if AHPP_TMA
  __shared__ __align__(8) uint64_t s_mbar[kWarps][2];
  GatherPipe gp;
  {
    const uint32_t w = threadIdx.x >> 5;
    gp.buf = reinterpret_cast<float*>(smem) + (size_t)w * (2 * kStage * 32 + 32 * 32);
    gp.bar[0] = smem_u32(&s_mbar[w][0]);
    gp.bar[1] = smem_u32(&s_mbar[w][1]);
    gp.phase = 0;
    if ((threadIdx.x & 31) == 0) {
      mbar_init(gp.bar[0]);
      mbar_init(gp.bar[1]);
      mbar_fence_init();
    }
    __syncwarp();
  }
  float* const sp_tma = reinterpret_cast<float*>(smem) + (size_t)(threadIdx.x >> 5) * (2 * kStage * 32 + 32 * 32) +
                        2 * kStage * 32;
#endif
  const uint32_t groups = SERVE ? 1u : p.groups;
  const uint32_t nbg = gridDim.x / groups;              // blocks per group
  const uint32_t grp = blockIdx.x / nbg;
  if (grp >= groups) return;                            // leftover blocks
  const uint32_t bid = blockIdx.x - grp * nbg;          // block id within the group
  const TileBuf& tb = s_tb;
  BCtx c{g, tb, p, (bid * kThreads + threadIdx.x) >> 5, (nbg * kThreads) >> 5,
         bid * kThreads + threadIdx.x, nbg * kThreads, threadIdx.x & 31u};
  const uint32_t lane = c.lane;
  const bool lq = lane < (uint32_t)kTile;               // this lane stands for a query
  const bool warp0 = threadIdx.x < 32;
  const bool app = p.algo == kAlgoAPP;
  const uint32_t n_work = SERVE ? sv.n_live : (p.n + kTile - 1) / kTile;
  const uint32_t n_split = max(g.b_v.n_split + g.b_a.n_split + g.b_u.n_split,
                               g.m_v.n_split + g.m_a.n_split + g.m_u.n_split);
  const size_t nu32 = (size_t)g.n_u * kTile;
  const uint32_t kmax = p.kmax;

  for (uint32_t w = grp; w < n_work; w += groups) {
    const uint32_t tile = SERVE ? sv.live[w] : w;
    const TileBuf* tg = SERVE ? &sv.tbufs[tile] : &st.tb[grp];   // tensor maps live here
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
        for (uint32_t k = g.ua_off[q_new]; AHPP_ATTR_PUSH && k < g.ua_off[q_new + 1]; ++k)
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
#if AHPP_TMA
      tphase1<WA>(c, tg, gp, sp_tma, A, &tb.bar->err);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      tphase2<WA>(c, tg, s_ctl, gp, sp_tma, A, &tb.bar->err);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      ++tround;
#else
      if (AHPP_P1_PASSES == 2) {
        gphase1<WA>(c, A, true, !AHPP_ATTR_PUSH, ta_cur, nullptr, nullptr, false, 0, 2);
        if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      }
      if (AHPP_ATTR_PUSH)
        gphase1<WA>(c, A, true, false, nullptr, ta_cur, ta_next, true, AHPP_P1_PASSES - 1, AHPP_P1_PASSES);
      else
        gphase1<WA>(c, A, true, true, ta_cur, nullptr, nullptr, true, AHPP_P1_PASSES - 1, AHPP_P1_PASSES);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      gphase2<WA>(c, s_ctl, A, ta_cur, AHPP_ATTR_PUSH ? ta_next : nullptr);
      if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
      ++tround;
#endif

      if (warp0) {
        LaneCtl L{};
        if (lq) L = s_ctl[lane];
        int switched = 0;
        if (L.active) {
          ++L.rounds;
          const float M = __uint_as_float(__ldcg(&A[lane].max_r_bits));
          L.n_p += s_mdeg[lane] + __ldcg(&A[lane].np_flush);
          if (!app) {
            if ((double)M <= L.eps_f) {
              L.phase = kPhaseDone;
              L.active = 0;
              s_fin[lane] = 1;
            } else if (L.phase == kPhaseAsync && (double)L.n_p >= bbudget(p, L.eps_f, (double)M)) {
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
        if (AHPP_ATTR_PUSH) {
          gphase1<WA>(c, A, false, true, (tround & 1) ? tb.t_a2 : tb.t_a, nullptr, nullptr, false);
          if (!grid_sync(tb.bar, nbg)) { wait_fail = true; break; }
        }
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
          for (int i = threadIdx.x; i < kTile * kRadixBins; i += kThreads) sh[i] = 0;
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
          for (int i = threadIdx.x; i < kTile * kRadixBins; i += kThreads)
            if (sh[i]) atomicAdd(&gh[i], sh[i]);
          if (!grid_sync(tb.bar, nbg)) return;
          // the merged histograms into shared memory; warp w picks the digit
          // of queries w, w + 8, ... (warp-parallel), lane l reads query l's
          for (int i = threadIdx.x; i < kTile * kRadixBins; i += kThreads) sh[i] = __ldcg(&gh[i]);
          __syncthreads();
          for (int l = threadIdx.x >> 5; l < kTile; l += kWarps) {
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
          for (uint32_t i = threadIdx.x; i < m; i += kThreads)
            sk[i] = i < kl ? tb.cand[(size_t)l * kmax + i] : 0ull;
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
template __global__ void k_tiles<float, true>(const __grid_constant__ DevGraph,
                                              const __grid_constant__ BatchState,
                                              const __grid_constant__ BatchParams,
                                              const __grid_constant__ ServeParams);
template __global__ void k_tiles<__nv_bfloat16, true>(const __grid_constant__ DevGraph,
                                                      const __grid_constant__ BatchState,
                                                      const __grid_constant__ BatchParams,
                                                      const __grid_constant__ ServeParams);

// radix histograms / sort buffer (4096 keys); with TMA also the per-warp
// gather stages (2 x 32 rows) and row sums (32 rows) of every warp
constexpr size_t kBatchSmem = AHPP_TMA ? std::max<size_t>(32 * 1024, kWarps * (2 * kStage * 32 + 32 * 32) * 4)
                                       : 32 * 1024;

namespace {
const void* tiles_fn(bool bf16, bool serve) {
  static bool attr_set = false;
  if (!attr_set) {
    attr_set = true;
    const void* fns[4] = {(const void*)k_tiles<__nv_bfloat16, true>, (const void*)k_tiles<float, true>,
                          (const void*)k_tiles<__nv_bfloat16, false>, (const void*)k_tiles<float, false>};
    for (const void* f : fns)
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
  }
  if (serve) return bf16 ? (const void*)k_tiles<__nv_bfloat16, true> : (const void*)k_tiles<float, true>;
  return bf16 ? (const void*)k_tiles<__nv_bfloat16, false> : (const void*)k_tiles<float, false>;
}
}  // namespace

// Tensor maps of a tile buffer for the TMA row gathers: r_U ([n_u][kTile]),
// t_V ([n_v][kTile]) and t_A ([n_a][kTile]); box kTile x 1.  Only the TMA
// phases read them, so a build without them encodes nothing.
int encode_tile_maps(TileBuf& t, uint32_t n_u, uint32_t n_v, uint32_t n_a) {
  if (!AHPP_TMA) return 0;
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                               CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                               CUtensorMapFloatOOBfill);
  static EncodeFn enc = nullptr;
  if (!enc) {
    void* fp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fp)
      return -1;
    enc = (EncodeFn)fp;
  }
  auto one = [&](CUtensorMap* m, float* base, uint32_t rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)kTile, (cuuint64_t)(rows ? rows : 1)};
    const cuuint64_t strides[1] = {(cuuint64_t)kTile * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTile, 1};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!one(&t.map_ru, t.r_u, n_u) || !one(&t.map_tv, t.t_v, n_v) || !one(&t.map_ta, t.t_a, n_a)) return -2;
  return 0;
}

int launch_batch(const DevGraph& g, const BatchState& s, const BatchParams& p, bool bf16,
                 int grid, cudaStream_t stream) {
  ServeParams sv{};
  void* args[] = {(void*)&g, (void*)&s, (void*)&p, (void*)&sv};
  cudaError_t e = cudaLaunchCooperativeKernel(tiles_fn(bf16, false), dim3(grid), dim3(kThreads), args,
                                              kBatchSmem, stream);
  return e == cudaSuccess ? 0 : (int)e;
}

int launch_serve_step(const DevGraph& g, const BatchParams& p, const ServeParams& sv, bool bf16,
                      int grid, cudaStream_t stream) {
  BatchState s{};
  void* args[] = {(void*)&g, (void*)&s, (void*)&p, (void*)&sv};
  cudaError_t e = cudaLaunchCooperativeKernel(tiles_fn(bf16, true), dim3(grid), dim3(kThreads), args,
                                              kBatchSmem, stream);
  return e == cudaSuccess ? 0 : (int)e;
}

int batch_max_grid(bool bf16, int sm_count) {
  int per_sm = 0, per_sm2 = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tiles_fn(bf16, false),
                                                                kThreads, kBatchSmem);
  cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, tiles_fn(bf16, true),
                                                                 kThreads, kBatchSmem);
  if (e != cudaSuccess || e2 != cudaSuccess || per_sm <= 0 || per_sm2 <= 0) return -1;
  return std::min(per_sm, per_sm2) * sm_count;
}

}  // namespace ahpp
