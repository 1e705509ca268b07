// Graph construction (host C++), upload, and the lambda estimate of Theorem 3.
//
// Input: COO edges (u, v, w(u,v)) and node-attribute tuples (u, a, w(u,a))
// (Section 2.1).  Duplicate pairs are merged by summing weights.  Nodes of
// U, V and A are relabeled by degree (largest first, ties by caller id) so
// that hub rows are contiguous and rows of similar length share a warp; the
// caller's ids are restored at the ABI.  Attribute weights are quantised to
// bfloat16 before any normaliser is computed, so the stored P_A is exactly
// the P_A of the quantised weights (Eq. 2); normalisers are computed in FP64
// and stored as FP32.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "ahpp_host.h"

namespace ahpp {

namespace {

unsigned worker_count() {
  unsigned n = std::thread::hardware_concurrency();
  return std::max(1u, std::min(n ? n : 1u, 32u));
}

// Run fn(begin, end) over [0, n) split across worker threads.
template <typename F>
void parallel_for(size_t n, F fn) {
  unsigned nt = worker_count();
  if (n < 65536 || nt == 1) { fn(size_t(0), n); return; }
  std::vector<std::thread> th;
  size_t step = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    size_t b = t * step, e = std::min(n, b + step);
    if (b >= e) break;
    th.emplace_back([=] { fn(b, e); });
  }
  for (auto& x : th) x.join();
}

// Rows of (row, col, w) triples: bucketed by row, sorted by col, duplicates
// merged (weights summed in FP64).  w == nullptr means unit weights.
void merge_rows(uint32_t n_rows, uint64_t n, const uint32_t* rows, const uint32_t* cols,
                const float* w, std::vector<uint32_t>& off, std::vector<uint32_t>& col,
                std::vector<double>& wout) {
  std::vector<uint64_t> cnt(n_rows + 1, 0);
  for (uint64_t e = 0; e < n; ++e) cnt[rows[e] + 1]++;
  for (uint32_t i = 0; i < n_rows; ++i) cnt[i + 1] += cnt[i];
  std::vector<std::pair<uint32_t, double>> tmp(n);
  {
    std::vector<uint64_t> pos(cnt.begin(), cnt.end() - 1);
    for (uint64_t e = 0; e < n; ++e) tmp[pos[rows[e]]++] = {cols[e], w ? (double)w[e] : 1.0};
  }
  std::vector<uint32_t> rowlen(n_rows, 0);
  parallel_for(n_rows, [&](size_t b, size_t e) {
    for (size_t i = b; i < e; ++i) {
      auto* s = tmp.data() + cnt[i];
      auto* t = tmp.data() + cnt[i + 1];
      std::sort(s, t, [](const auto& x, const auto& y) { return x.first < y.first; });
      uint64_t out = 0;
      for (auto* p = s; p < t; ++p) {
        if (out && s[out - 1].first == p->first) s[out - 1].second += p->second;
        else s[out++] = *p;
      }
      rowlen[i] = (uint32_t)out;
    }
  });
  off.assign(n_rows + 1, 0);
  for (uint32_t i = 0; i < n_rows; ++i) off[i + 1] = off[i] + rowlen[i];
  col.resize(off[n_rows]);
  wout.resize(off[n_rows]);
  parallel_for(n_rows, [&](size_t b, size_t e) {
    for (size_t i = b; i < e; ++i)
      for (uint32_t k = 0; k < rowlen[i]; ++k) {
        col[off[i] + k] = tmp[cnt[i] + k].first;
        wout[off[i] + k] = tmp[cnt[i] + k].second;
      }
  });
}

// Order of nodes by degree descending, ties by id ascending: new2old.
std::vector<uint32_t> degree_order(const std::vector<uint32_t>& deg) {
  std::vector<uint32_t> ord(deg.size());
  std::iota(ord.begin(), ord.end(), 0u);
  std::stable_sort(ord.begin(), ord.end(),
                   [&](uint32_t a, uint32_t b) { return deg[a] > deg[b]; });
  return ord;
}

// Relabel an adjacency (rows old ids -> new ids, cols old -> new), sorting
// each row by new column id.
void relabel_rows(const std::vector<uint32_t>& off, const std::vector<uint32_t>& col,
                  const std::vector<double>& w, const std::vector<uint32_t>& row_new2old,
                  const std::vector<uint32_t>& col_old2new, std::vector<uint32_t>& noff,
                  std::vector<uint32_t>& ncol, std::vector<double>& nw) {
  const uint32_t n = (uint32_t)row_new2old.size();
  noff.assign(n + 1, 0);
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t o = row_new2old[i];
    noff[i + 1] = noff[i] + (off[o + 1] - off[o]);
  }
  ncol.resize(col.size());
  nw.resize(w.size());
  parallel_for(n, [&](size_t b, size_t e) {
    std::vector<std::pair<uint32_t, double>> row;
    for (size_t i = b; i < e; ++i) {
      uint32_t o = row_new2old[i];
      row.clear();
      for (uint32_t k = off[o]; k < off[o + 1]; ++k) row.push_back({col_old2new[col[k]], w[k]});
      std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (size_t k = 0; k < row.size(); ++k) {
        ncol[noff[i] + k] = row[k].first;
        nw[noff[i] + k] = row[k].second;
      }
    }
  });
}

// Transpose: rows become columns (weights carried along); rows of the result
// are sorted by column id because the source is scanned in row order.
void transpose(uint32_t n_rows, uint32_t n_cols, const std::vector<uint32_t>& off,
               const std::vector<uint32_t>& col, const std::vector<double>& w,
               std::vector<uint32_t>& toff, std::vector<uint32_t>& tcol, std::vector<double>& tw) {
  toff.assign(n_cols + 1, 0);
  for (uint32_t c : col) toff[c + 1]++;
  for (uint32_t i = 0; i < n_cols; ++i) toff[i + 1] += toff[i];
  tcol.resize(col.size());
  tw.resize(w.size());
  std::vector<uint32_t> pos(toff.begin(), toff.end() - 1);
  for (uint32_t r = 0; r < n_rows; ++r)
    for (uint32_t k = off[r]; k < off[r + 1]; ++k) {
      uint32_t p = pos[col[k]]++;
      tcol[p] = r;
      tw[p] = w[k];
    }
}

float bf16_round(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  uint32_t lsb = (b >> 16) & 1u;
  b = (b + 0x7fffu + lsb) & 0xffff0000u;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

}  // namespace

HostItems build_items(const std::vector<uint32_t>& deg, const ItemShape& sh) {
  HostItems h;
  const uint32_t n = (uint32_t)deg.size();
  uint32_t r = 0;
  while (r < n) {
    const uint32_t d = deg[r];
    if (d > sh.short_max) {
      const uint32_t nch = (d + sh.chunk - 1) / sh.chunk;
      if (nch <= 1) {
        h.items.push_back(make_uint4(r, kItemLong, 0, d));
      } else {
        const uint32_t slot = (uint32_t)h.split_nchunks.size();
        h.split_nchunks.push_back(nch);
        for (uint32_t c = 0; c < nch; ++c)
          h.items.push_back(make_uint4(r, kItemSplit | slot, c * sh.chunk,
                                       std::min(d, (c + 1) * sh.chunk)));
      }
      ++r;
    } else {
      uint32_t cnt = 0, nnz = 0;
      while (r + cnt < n && cnt < sh.group_rows && deg[r + cnt] <= sh.short_max &&
             (cnt == 0 || nnz + deg[r + cnt] <= sh.group_nnz)) {
        nnz += deg[r + cnt];
        ++cnt;
      }
      h.items.push_back(make_uint4(r, cnt, 0, 0));
      r += cnt;
    }
  }
  return h;
}

HostItems build_units(const std::vector<uint32_t>& deg, uint32_t chunk) {
  HostItems h;
  const uint32_t n = (uint32_t)deg.size();
  uint32_t r = 0;
  while (r < n && deg[r] > chunk) {
    const uint32_t d = deg[r];
    const uint32_t nch = (d + chunk - 1) / chunk;
    const uint32_t slot = (uint32_t)h.split_nchunks.size();
    h.split_nchunks.push_back(nch);
    for (uint32_t c = 0; c < nch; ++c)
      h.items.push_back(make_uint4(r, kItemSplit | slot, c * chunk, std::min(d, (c + 1) * chunk)));
    ++r;
  }
  h.n_long = r;
  return h;
}

int chunk_choice(uint32_t chunk) {
  if (chunk == 0) return kChunkDefault;
  for (int c = 0; c < kChunkChoices; ++c)
    if (kChunkSizes[c] == chunk) return c;
  return -1;
}

void select_chunk(DevGraph& G, uint32_t choice) {
  G.b_chunk = choice;
  G.b_v = G.b_alt[choice][0];
  G.b_a = G.b_alt[choice][1];
  G.b_u = G.b_alt[choice][2];
}

int build_graph(const ahpp_graph_desc* d, ahpp_graph* g) {
  const ahpp_config& cfg = g->cfg;
  const uint64_t lim = (1ull << 31) - 1;
  if (d->n_u == 0 || d->n_u > lim || d->n_v > lim || d->n_a > lim || d->n_e > lim ||
      d->n_ea > lim) {
    set_error("ahpp_load_graph: counts must satisfy 0 < n_u and all counts < 2^31");
    return AHPP_EINVAL;
  }
  if ((d->n_e && (!d->e_u || !d->e_v)) || (d->n_ea && (!d->ea_u || !d->ea_a))) {
    set_error("ahpp_load_graph: missing edge or attribute arrays");
    return AHPP_EINVAL;
  }
  for (uint64_t e = 0; e < d->n_e; ++e) {
    if (d->e_u[e] >= d->n_u || d->e_v[e] >= d->n_v ||
        (d->e_w && !(d->e_w[e] > 0.f && std::isfinite(d->e_w[e])))) {
      set_error("ahpp_load_graph: edge " + std::to_string(e) + " has an id out of range or w <= 0");
      return AHPP_EINVAL;
    }
  }
  for (uint64_t e = 0; e < d->n_ea; ++e) {
    if (d->ea_u[e] >= d->n_u || d->ea_a[e] >= d->n_a ||
        (d->ea_w && !(d->ea_w[e] > 0.f && std::isfinite(d->ea_w[e])))) {
      set_error("ahpp_load_graph: attribute tuple " + std::to_string(e) +
                " has an id out of range or w <= 0");
      return AHPP_EINVAL;
    }
  }
  const uint32_t nU = (uint32_t)d->n_u, nV = (uint32_t)d->n_v, nA = (uint32_t)d->n_a;
  const double alpha = cfg.alpha, beta = cfg.beta;
  g->bf16 = cfg.attr_bf16 != 0;

  // 1. merge duplicates in caller ids
  std::vector<uint32_t> uv_off0, uv_col0, ua_off0, ua_col0;
  std::vector<double> uv_w0, ua_w0;
  merge_rows(nU, d->n_e, d->e_u, d->e_v, d->e_w, uv_off0, uv_col0, uv_w0);
  merge_rows(nU, d->n_ea, d->ea_u, d->ea_a, d->ea_w, ua_off0, ua_col0, ua_w0);
  if (g->bf16)
    for (auto& x : ua_w0) x = (double)bf16_round((float)x);
  else
    for (auto& x : ua_w0) x = (double)(float)x;
  g->n_u = nU; g->n_v = nV; g->n_a = nA;
  g->n_e = uv_col0.size();
  g->n_ea = ua_col0.size();
  if (g->n_e + g->n_ea > 0xffffffffull) {
    set_error("ahpp_load_graph: |E| + |E_A| must stay below 2^32");
    return AHPP_EINVAL;
  }

  // 2. degrees and relabeling
  std::vector<uint32_t> deg_u(nU), deg_v(nV, 0), deg_a(nA, 0);
  for (uint32_t u = 0; u < nU; ++u)
    deg_u[u] = (uv_off0[u + 1] - uv_off0[u]) + (ua_off0[u + 1] - ua_off0[u]);
  for (uint32_t c : uv_col0) deg_v[c]++;
  for (uint32_t c : ua_col0) deg_a[c]++;
  std::vector<uint32_t> u_n2o = degree_order(deg_u), v_n2o = degree_order(deg_v),
                        a_n2o = degree_order(deg_a);
  std::vector<uint32_t> u_o2n(nU), v_o2n(nV), a_o2n(nA);
  for (uint32_t i = 0; i < nU; ++i) u_o2n[u_n2o[i]] = i;
  for (uint32_t i = 0; i < nV; ++i) v_o2n[v_n2o[i]] = i;
  for (uint32_t i = 0; i < nA; ++i) a_o2n[a_n2o[i]] = i;

  // 3. the four directions in internal ids
  std::vector<uint32_t> uv_off, uv_idx, vu_off, vu_idx, ua_off, ua_idx, au_off, au_idx;
  std::vector<double> uv_w, vu_w, ua_w, au_w;
  relabel_rows(uv_off0, uv_col0, uv_w0, u_n2o, v_o2n, uv_off, uv_idx, uv_w);
  relabel_rows(ua_off0, ua_col0, ua_w0, u_n2o, a_o2n, ua_off, ua_idx, ua_w);
  { std::vector<uint32_t>().swap(uv_off0); std::vector<uint32_t>().swap(uv_col0);
    std::vector<double>().swap(uv_w0); std::vector<uint32_t>().swap(ua_off0);
    std::vector<uint32_t>().swap(ua_col0); std::vector<double>().swap(ua_w0); }
  transpose(nU, nV, uv_off, uv_idx, uv_w, vu_off, vu_idx, vu_w);
  transpose(nU, nA, ua_off, ua_idx, ua_w, au_off, au_idx, au_w);

  // 4. normalisers (FP64) and direction coefficients
  std::vector<double> du(nU, 0.0), dv(nV, 0.0), wr(nU, 0.0), wc(nA, 0.0);
  for (uint32_t u = 0; u < nU; ++u) {
    for (uint32_t k = uv_off[u]; k < uv_off[u + 1]; ++k) { du[u] += uv_w[k]; dv[uv_idx[k]] += uv_w[k]; }
    for (uint32_t k = ua_off[u]; k < ua_off[u + 1]; ++k) { wr[u] += ua_w[k]; wc[ua_idx[k]] += ua_w[k]; }
  }
  const double ks = (1.0 - alpha) * (1.0 - beta);
  std::vector<float> f_uv_w(uv_w.size()), f_uv_c(uv_w.size()), f_vu_w(vu_w.size()),
      f_vu_c(vu_w.size());
  parallel_for(nU, [&](size_t b, size_t e) {
    for (size_t u = b; u < e; ++u)
      for (uint32_t k = uv_off[u]; k < uv_off[u + 1]; ++k) {
        f_uv_w[k] = (float)uv_w[k];
        f_uv_c[k] = (float)(ks * uv_w[k] / (du[u] * dv[uv_idx[k]]));
      }
  });
  parallel_for(nV, [&](size_t b, size_t e) {
    for (size_t v = b; v < e; ++v)
      for (uint32_t k = vu_off[v]; k < vu_off[v + 1]; ++k) {
        f_vu_w[k] = (float)vu_w[k];
        f_vu_c[k] = (float)(ks * vu_w[k] / (du[vu_idx[k]] * dv[v]));
      }
  });
  std::vector<float> rnorm(nU), cnorm(nA);
  for (uint32_t u = 0; u < nU; ++u) rnorm[u] = wr[u] > 0 ? (float)(1.0 / wr[u]) : 0.f;
  for (uint32_t a = 0; a < nA; ++a) cnorm[a] = wc[a] > 0 ? (float)(1.0 / wc[a]) : 0.f;
  // push coefficient of the U->A direction (both factors of Eq. 2 and the
  // (1 - alpha) beta share of the U-push), rounded once to FP32
  std::vector<float> f_ua_pc(ua_w.size());
  const double ka = (1.0 - alpha) * beta;
  parallel_for(nU, [&](size_t b, size_t e) {
    for (size_t u = b; u < e; ++u)
      for (uint32_t k = ua_off[u]; k < ua_off[u + 1]; ++k) {
        const uint32_t a = ua_idx[k];
        f_ua_pc[k] = (wr[u] > 0 && wc[a] > 0) ? (float)(ka * ua_w[k] / (wr[u] * wc[a])) : 0.f;
      }
  });
  // pull coefficient of the A->U direction (the U-side factor of Eq. 2), from
  // the quantised weight and the FP64 row sum, rounded once to FP32
  std::vector<float> f_au_c(au_w.size());
  parallel_for(nA, [&](size_t b, size_t e) {
    for (size_t a = b; a < e; ++a)
      for (uint32_t k = au_off[a]; k < au_off[a + 1]; ++k) {
        const uint32_t u = au_idx[k];
        f_au_c[k] = wr[u] > 0 ? (float)(au_w[k] / wr[u]) : 0.f;
      }
  });

  // 5. work items (rows are sorted by degree, longest first)
  std::vector<uint32_t> dg_u(nU), dg_v(nV), dg_a(nA);
  for (uint32_t u = 0; u < nU; ++u) dg_u[u] = (uv_off[u + 1] - uv_off[u]) + (ua_off[u + 1] - ua_off[u]);
  for (uint32_t v = 0; v < nV; ++v) dg_v[v] = vu_off[v + 1] - vu_off[v];
  for (uint32_t a = 0; a < nA; ++a) dg_a[a] = au_off[a + 1] - au_off[a];
  const ItemShape s1{64, 32, 0xffffffffu, 2048};
  HostItems i1v = build_items(dg_v, s1), i1a = build_items(dg_a, s1), i1u = build_items(dg_u, s1);
  std::vector<HostItems> ib;
  for (int c = 0; c < kChunkChoices; ++c) {
    ib.push_back(build_units(dg_v, kChunkSizes[c]));
    ib.push_back(build_units(dg_a, kChunkSizes[c]));
    ib.push_back(build_units(dg_u, kChunkSizes[c]));
  }

  // 6. upload
  auto up = [&](const void* src, size_t bytes) -> void* {
    void* p = g->alloc(bytes ? bytes : 4);
    if (p && bytes && cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return p;
  };
  DevGraph& G = g->dg;
  G.n_u = nU; G.n_v = nV; G.n_a = nA;
  G.n_e = (uint32_t)g->n_e; G.n_ea = (uint32_t)g->n_ea;
  G.alpha = (float)alpha;
  G.k_attr = (float)((1.0 - alpha) * beta);
  G.uv_off = (const uint32_t*)up(uv_off.data(), uv_off.size() * 4);
  G.uv_idx = (const uint32_t*)up(uv_idx.data(), uv_idx.size() * 4);
  G.uv_w = (const float*)up(f_uv_w.data(), f_uv_w.size() * 4);
  G.uv_c = (const float*)up(f_uv_c.data(), f_uv_c.size() * 4);
  G.vu_off = (const uint32_t*)up(vu_off.data(), vu_off.size() * 4);
  G.vu_idx = (const uint32_t*)up(vu_idx.data(), vu_idx.size() * 4);
  G.vu_c = (const float*)up(f_vu_c.data(), f_vu_c.size() * 4);
  G.vu_w = (const float*)up(f_vu_w.data(), f_vu_w.size() * 4);
  G.ua_off = (const uint32_t*)up(ua_off.data(), ua_off.size() * 4);
  G.ua_idx = (const uint32_t*)up(ua_idx.data(), ua_idx.size() * 4);
  G.au_off = (const uint32_t*)up(au_off.data(), au_off.size() * 4);
  G.au_idx = (const uint32_t*)up(au_idx.data(), au_idx.size() * 4);
  if (g->bf16) {
    std::vector<__nv_bfloat16> a(ua_w.size()), b(au_w.size());
    for (size_t k = 0; k < a.size(); ++k) a[k] = __float2bfloat16_rn((float)ua_w[k]);
    for (size_t k = 0; k < b.size(); ++k) b[k] = __float2bfloat16_rn((float)au_w[k]);
    G.ua_w = up(a.data(), a.size() * 2);
    G.au_w = up(b.data(), b.size() * 2);
  } else {
    std::vector<float> a(ua_w.begin(), ua_w.end()), b(au_w.begin(), au_w.end());
    G.ua_w = up(a.data(), a.size() * 4);
    G.au_w = up(b.data(), b.size() * 4);
  }
  G.au_c = (const float*)up(f_au_c.data(), f_au_c.size() * 4);
  G.ua_pc = (const float*)up(f_ua_pc.data(), f_ua_pc.size() * 4);
  G.rnorm_u = (const float*)up(rnorm.data(), rnorm.size() * 4);
  G.cnorm_a = (const float*)up(cnorm.data(), cnorm.size() * 4);
  auto up_items = [&](const HostItems& h, ItemList& L) {
    L.items = (const uint4*)up(h.items.data(), h.items.size() * sizeof(uint4));
    L.n_items = (uint32_t)h.items.size();
    L.n_split = (uint32_t)h.split_nchunks.size();
    L.split_nchunks = (const uint32_t*)up(h.split_nchunks.data(), h.split_nchunks.size() * 4);
    L.n_long = h.n_long;
  };
  up_items(i1v, G.s1_v); up_items(i1a, G.s1_a); up_items(i1u, G.s1_u);
  G.b_split_max = 0;
  for (int c = 0; c < kChunkChoices; ++c) {
    for (int d = 0; d < 3; ++d) up_items(ib[3 * c + d], G.b_alt[c][d]);
    G.b_split_max = std::max(G.b_split_max,
                             G.b_alt[c][0].n_split + G.b_alt[c][1].n_split + G.b_alt[c][2].n_split);
  }
  select_chunk(G, kChunkDefault);

  g->h_u_old2new = u_o2n;
  g->h_u_new2old = u_n2o;
  g->d_u_new2old = (uint32_t*)up(u_n2o.data(), u_n2o.size() * 4);
  g->d_u_old2new = (uint32_t*)up(u_o2n.data(), u_o2n.size() * 4);
  for (auto& b : g->bufs)
    if (!b.p) { set_error("ahpp_load_graph: device allocation failed"); return AHPP_ENOMEM; }
  if (cudaGetLastError() != cudaSuccess) { set_error("ahpp_load_graph: upload failed"); return AHPP_ECUDA; }

  g->n_graph_bufs = g->bufs.size();
  g->graph_bytes = 0;
  for (auto& b : g->bufs) g->graph_bytes += b.bytes;
  return alloc_query_state(g);
}

// Shared-memory plan of the single-query kernel's pull rounds: phase 2
// holds t_A and, with the attribute push, its accumulator over A when both
// fit in kQ1AttrSmem.  Shared memory not planned here stays L1.
void plan_query1_smem(ahpp_graph* g) {
  constexpr uint64_t kQ1AttrSmem = 96 * 1024;
  const DevGraph& G = g->dg;
  const uint32_t smax = query1_max_smem(g->device);
  const uint64_t na4 = 4ull * G.n_a;
  g->q1_attr_push = 2 * na4 <= std::min<uint64_t>(kQ1AttrSmem, smax);
  g->q1_ta_smem = g->q1_attr_push;
  g->q1_smem = g->q1_attr_push ? (uint32_t)((2 * na4 + 15) / 16 * 16) : 0u;
}

// Single-query state of a loaded graph (working vectors, lists, accumulators,
// barrier, trace) and the launch grid of the single-query kernel.
int alloc_query_state(ahpp_graph* g) {
  const ahpp_config& cfg = g->cfg;
  const DevGraph& G = g->dg;
  const uint32_t nU = G.n_u, nV = G.n_v, nA = G.n_a;
  g->n_split1 = G.s1_v.n_split + G.s1_a.n_split + G.s1_u.n_split;
  const size_t before = g->bufs.size();
  Q1State& s = g->q1;
  s.r_u = (float*)g->alloc(4ull * nU);
  s.pi = (float*)g->alloc(4ull * nU);
  s.pic = (float*)g->alloc(4ull * nU);
  s.t_v = (float*)g->alloc(4ull * std::max(nV, 1u));
  s.t_a = (float*)g->alloc(4ull * std::max(nA, 1u));
  s.t_a2 = (float*)g->alloc(4ull * std::max(nA, 1u));
  s.list_u = (uint32_t*)g->alloc(4ull * nU);
  s.split_acc = (float*)g->alloc(4ull * std::max(g->n_split1, 1u));
  s.split_cnt = (uint32_t*)g->alloc(4ull * std::max(g->n_split1, 1u));
  s.ctl = (QCtl*)g->alloc(sizeof(QCtl));
  s.racc = (RAcc*)g->alloc(3 * sizeof(RAcc));
  s.bar = (GridBarrier*)g->alloc(sizeof(GridBarrier));
  s.final_maxr_bits = (unsigned int*)g->alloc(2 * sizeof(unsigned int));
  const uint32_t trace_cap = 4096;
  s.trace_frontier = (uint32_t*)g->alloc(4ull * trace_cap);
  s.trace_maxr = (float*)g->alloc(4ull * trace_cap);
  g->q1_bytes = 0;
  for (size_t i = before; i < g->bufs.size(); ++i) {
    if (!g->bufs[i].p) { set_error("ahpp_load_graph: device allocation failed"); return AHPP_ENOMEM; }
    g->q1_bytes += g->bufs[i].bytes;
  }
  AHPP_CUDA(cudaMemset(s.bar, 0, sizeof(GridBarrier)));
  AHPP_CUDA(cudaMemset(s.split_acc, 0, 4ull * std::max(g->n_split1, 1u)));
  AHPP_CUDA(cudaMemset(s.split_cnt, 0, 4ull * std::max(g->n_split1, 1u)));
  plan_query1_smem(g);
  g->q1_grid = query1_max_grid(g->bf16, g->sm_count, g->q1_smem);
  if (g->q1_grid <= 0) { set_error("ahpp_load_graph: occupancy query failed"); return AHPP_ECUDA; }
  BatchParams plan;
  if (int rc = batch_plan(g, plan)) return rc;
  if (cfg.hbm_budget_bytes && g->graph_bytes + g->q1_bytes > cfg.hbm_budget_bytes) {
    set_error("ahpp_load_graph: graph and query state exceed hbm_budget_bytes");
    return AHPP_ENOMEM;
  }
  return AHPP_OK;
}

}  // namespace ahpp
