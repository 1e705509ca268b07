// Graph cache: save a loaded graph (its device arrays after duplicate merging,
// relabelling, the four adjacency directions, normalisers, coefficients, work
// items and the lambda estimate) to a file, and load it back without redoing
// the host-side build or the lambda run.
//
// File layout (native byte order; written and read by the same library
// build, which the header checks):
//   magic "AHPPGRF1", u32 format version, u32 sizeof(DevGraph)
//   u64 n_u, n_v, n_a, n_e, n_ea; f64 alpha, beta, lambda; u32 lambda_T;
//   u32 attr_bf16; u32 algo (for the lambda it was computed with); u64 buffers
//   DevGraph bytes (pointer fields meaningless), then for every pointer field
//   of the graph, in a fixed order, the i64 index of its buffer (-1: null)
//   for every buffer: u64 bytes, then the bytes
//   u64 checksum of every byte above (Checksum below), then the end of file
// The loader checks the header, the buffer table, the file length and the
// checksum; it does not re-derive the arrays' contents, so it accepts only
// files this library wrote (a checksum guards against accidental damage,
// not against a file crafted to pass it).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ahpp_host.h"

namespace ahpp {
namespace {

constexpr char kMagic[8] = {'A', 'H', 'P', 'P', 'G', 'R', 'F', '1'};
constexpr uint32_t kVersion = 5;

struct CacheHeader {
  char magic[8];
  uint32_t version, devgraph_bytes;
  uint64_t n_u, n_v, n_a, n_e, n_ea;
  double alpha, beta, lambda;
  uint32_t lambda_T, attr_bf16, algo, pad;
  uint64_t n_buffers;
};

// Every device pointer a loaded graph holds besides its query state, in a
// fixed order.
template <typename F>
void visit_graph_ptrs(ahpp_graph* g, F f) {
  DevGraph& G = g->dg;
  f((const void**)&G.uv_off); f((const void**)&G.uv_idx); f((const void**)&G.uv_w); f((const void**)&G.uv_c);
  f((const void**)&G.vu_off); f((const void**)&G.vu_idx); f((const void**)&G.vu_c); f((const void**)&G.vu_w);
  f((const void**)&G.ua_off); f((const void**)&G.ua_idx); f((const void**)&G.ua_w);
  f((const void**)&G.au_off); f((const void**)&G.au_idx); f((const void**)&G.au_w); f((const void**)&G.au_c);
  f((const void**)&G.ua_pc);
  f((const void**)&G.rnorm_u); f((const void**)&G.cnorm_a);
  ItemList* lists[] = {&G.s1_v, &G.s1_a, &G.s1_u, &G.b_v, &G.b_a, &G.b_u};
  for (ItemList* L : lists) {
    f((const void**)&L->items);
    f((const void**)&L->split_nchunks);
  }
  for (int c = 0; c < kChunkChoices; ++c)
    for (int d = 0; d < 3; ++d) {
      f((const void**)&G.b_alt[c][d].items);
      f((const void**)&G.b_alt[c][d].split_nchunks);
    }
  f((const void**)&g->d_u_new2old);
  f((const void**)&g->d_u_old2new);
}

struct File {
  FILE* f = nullptr;
  explicit File(FILE* x) : f(x) {}
  ~File() { if (f) fclose(f); }
};

// Word-wise multiply-rotate checksum: each 8-byte word (then each tail byte)
// is XORed in, rotated and multiplied by an odd constant.  Every step is a
// bijection of the state, so a file that differs in one word or byte always
// gives a different sum.  Save and load feed it the same sequence of chunks.
struct Checksum {
  uint64_t h = 0x243F6A8885A308D3ull;
  void step(uint64_t w) {
    h ^= w;
    h = (h << 31) | (h >> 33);
    h *= 0x9E3779B97F4A7C15ull;
  }
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
      uint64_t w;
      std::memcpy(&w, b + i, 8);
      step(w);
    }
    for (; i < n; ++i) step(b[i]);
  }
};

bool wr(FILE* f, const void* p, size_t n, Checksum& cs) {
  cs.add(p, n);
  return n == 0 || fwrite(p, 1, n, f) == n;
}
bool rd(FILE* f, void* p, size_t n, Checksum& cs) {
  if (n != 0 && fread(p, 1, n, f) != n) return false;
  cs.add(p, n);
  return true;
}

}  // namespace
}  // namespace ahpp

using namespace ahpp;

extern "C" int ahpp_save_graph(ahpp_graph* g, const char* path) {
  if (!g || !path) { set_error("ahpp_save_graph: null argument"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  // map every graph pointer to its buffer
  std::vector<int64_t> index;
  bool ok = true;
  visit_graph_ptrs(g, [&](const void** pp) {
    int64_t idx = -1;
    if (*pp) {
      for (size_t i = 0; i < g->n_graph_bufs; ++i)
        if (g->bufs[i].p == *pp) { idx = (int64_t)i; break; }
      if (idx < 0) ok = false;
    }
    index.push_back(idx);
  });
  if (!ok) { set_error("ahpp_save_graph: a graph array is not one of the graph's buffers"); return AHPP_ESTATE; }
  File out(fopen(path, "wb"));
  if (!out.f) { set_error(std::string("ahpp_save_graph: cannot open ") + path); return AHPP_EINVAL; }
  CacheHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.devgraph_bytes = sizeof(DevGraph);
  h.n_u = g->n_u; h.n_v = g->n_v; h.n_a = g->n_a; h.n_e = g->n_e; h.n_ea = g->n_ea;
  h.alpha = g->cfg.alpha; h.beta = g->cfg.beta; h.lambda = g->lambda;
  h.lambda_T = g->lambda_T; h.attr_bf16 = g->bf16 ? 1u : 0u; h.algo = (uint32_t)g->cfg.algo;
  h.n_buffers = g->n_graph_bufs;
  Checksum cs;
  bool w = wr(out.f, &h, sizeof(h), cs) && wr(out.f, &g->dg, sizeof(DevGraph), cs) &&
           wr(out.f, index.data(), index.size() * sizeof(int64_t), cs);
  std::vector<unsigned char> host;
  for (size_t i = 0; w && i < g->n_graph_bufs; ++i) {
    const uint64_t n = g->bufs[i].bytes;
    host.resize(n);
    if (n) AHPP_CUDA(cudaMemcpy(host.data(), g->bufs[i].p, n, cudaMemcpyDeviceToHost));
    w = wr(out.f, &n, sizeof(n), cs) && wr(out.f, host.data(), n, cs);
  }
  const uint64_t sum = cs.h;
  w = w && fwrite(&sum, 1, sizeof(sum), out.f) == sizeof(sum);
  if (!w || fflush(out.f) != 0) { set_error(std::string("ahpp_save_graph: write failed: ") + path); return AHPP_EINVAL; }
  return AHPP_OK;
}

extern "C" int ahpp_load_graph_file(const char* path, const ahpp_config* cfg, ahpp_graph** out) {
  ahpp::NvtxRange nvtx_range_("ahpp_load_graph_file");
  if (!path || !out) { set_error("ahpp_load_graph_file: null argument"); return AHPP_EINVAL; }
  *out = nullptr;
  ahpp_config c;
  if (cfg) c = *cfg; else ahpp_config_default(&c);
  File in(fopen(path, "rb"));
  if (!in.f) { set_error(std::string("ahpp_load_graph_file: cannot open ") + path); return AHPP_EINVAL; }
  uint64_t file_bytes = 0;
  if (fseek(in.f, 0, SEEK_END) == 0) {
    const long e = ftell(in.f);
    file_bytes = e > 0 ? (uint64_t)e : 0;
  }
  if (fseek(in.f, 0, SEEK_SET) != 0) { set_error("ahpp_load_graph_file: cannot read the file"); return AHPP_EINVAL; }
  CacheHeader h{};
  Checksum cs;
  if (!rd(in.f, &h, sizeof(h), cs) || std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion) {
    set_error("ahpp_load_graph_file: not a graph cache of this library version");
    return AHPP_EINVAL;
  }
  const uint64_t lim = (1ull << 31) - 1;
  if (h.n_u == 0 || h.n_u > lim || h.n_v > lim || h.n_a > lim || h.n_e > lim || h.n_ea > lim ||
      h.n_buffers > (1u << 20)) {
    set_error("ahpp_load_graph_file: corrupt header");
    return AHPP_EINVAL;
  }
  if (h.devgraph_bytes != sizeof(DevGraph)) {
    set_error("ahpp_load_graph_file: written by a different build of the library");
    return AHPP_EINVAL;
  }
  // the normalisers, coefficients and bf16 weights depend on these
  if (c.alpha != h.alpha || c.beta != h.beta || (uint32_t)(c.attr_bf16 != 0) != h.attr_bf16) {
    set_error("ahpp_load_graph_file: alpha, beta and attr_bf16 must equal the cached graph's");
    return AHPP_EINVAL;
  }
  if (kernel_algo(c.algo) < 0 || c.switch_rule < 0 || c.switch_rule > 2 ||
      (c.algo == AHPP_APP_S && c.switch_rule == 1) ||
      (c.batch_tile != 0 && c.batch_tile != 16 && c.batch_tile != 32) || c.batch_groups > (uint32_t)kMaxGroups ||
      chunk_choice(c.batch_chunk) < 0 || c.single_vec_width > 32 ||
      (c.single_vec_width & (c.single_vec_width - 1))) {
    set_error("ahpp_load_graph_file: bad algo, switch_rule, batch_tile, batch_groups or batch_chunk");
    return AHPP_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    set_error("ahpp_load_graph_file: no CUDA device available (the library has no CPU path)");
    return AHPP_ECUDA;
  }
  if (c.device < 0 || c.device >= ndev) { set_error("ahpp_load_graph_file: bad device ordinal"); return AHPP_EINVAL; }
  AHPP_CUDA(cudaSetDevice(c.device));

  ahpp_graph* g = new ahpp_graph();
  g->cfg = c;
  g->device = c.device;
  g->batch_tile = c.batch_tile ? c.batch_tile : (uint32_t)kTile;
  g->batch_groups = c.batch_groups ? c.batch_groups : 1;
  g->q1_vw_max = c.single_vec_width ? c.single_vec_width : ahpp::kQ1VecWidthDefault;
  g->n_u = h.n_u; g->n_v = h.n_v; g->n_a = h.n_a; g->n_e = h.n_e; g->n_ea = h.n_ea;
  g->bf16 = h.attr_bf16 != 0;
  int rc = AHPP_OK;
  auto fail = [&](int code, const std::string& msg) {
    if (rc == AHPP_OK) { set_error(msg); rc = code; }
  };
  if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    fail(AHPP_ECUDA, "ahpp_load_graph_file: device setup failed");
  }
  std::vector<int64_t> index;
  visit_graph_ptrs(g, [&](const void**) { index.push_back(0); });
  if (rc == AHPP_OK && (!rd(in.f, &g->dg, sizeof(DevGraph), cs) ||
                        !rd(in.f, index.data(), index.size() * sizeof(int64_t), cs)))
    fail(AHPP_EINVAL, "ahpp_load_graph_file: truncated file");
  std::vector<unsigned char> host;
  for (uint64_t i = 0; rc == AHPP_OK && i < h.n_buffers; ++i) {
    uint64_t n = 0;
    const long at = ftell(in.f);
    if (!rd(in.f, &n, sizeof(n), cs) || at < 0 || n > file_bytes - (uint64_t)at) {   // never past the file's end
      fail(AHPP_EINVAL, "ahpp_load_graph_file: truncated file");
      break;
    }
    host.resize(n);
    if (!rd(in.f, host.data(), n, cs)) { fail(AHPP_EINVAL, "ahpp_load_graph_file: truncated file"); break; }
    void* p = g->alloc(n ? n : 4);
    if (!p) { fail(AHPP_ENOMEM, "ahpp_load_graph_file: device allocation failed"); break; }
    if (n && cudaMemcpy(p, host.data(), n, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      fail(AHPP_ECUDA, "ahpp_load_graph_file: upload failed");
    }
  }
  if (rc == AHPP_OK) {
    uint64_t sum = 0;
    const bool got = fread(&sum, 1, sizeof(sum), in.f) == sizeof(sum);
    const long end = ftell(in.f);
    if (!got || end < 0 || (uint64_t)end != file_bytes)
      fail(AHPP_EINVAL, "ahpp_load_graph_file: truncated file or trailing bytes");
    else if (sum != cs.h)
      fail(AHPP_EINVAL, "ahpp_load_graph_file: checksum mismatch (damaged file)");
  }
  if (rc == AHPP_OK) {
    size_t k = 0;
    visit_graph_ptrs(g, [&](const void** pp) {
      const int64_t idx = index[k++];
      if (idx < 0) { *pp = nullptr; return; }
      if ((uint64_t)idx >= h.n_buffers) { fail(AHPP_EINVAL, "ahpp_load_graph_file: corrupt buffer table"); return; }
      *pp = g->bufs[(size_t)idx].p;
    });
  }
  if (rc == AHPP_OK) {
    // the id maps must hold n_u entries each
    for (const void* p : {(const void*)g->d_u_old2new, (const void*)g->d_u_new2old}) {
      bool sized = false;
      for (auto& b : g->bufs)
        if (b.p == p && b.bytes >= 4 * g->n_u) sized = true;
      if (!sized) fail(AHPP_EINVAL, "ahpp_load_graph_file: corrupt id maps");
    }
  }
  if (rc == AHPP_OK) {
    g->n_graph_bufs = g->bufs.size();
    g->graph_bytes = 0;
    for (auto& b : g->bufs) g->graph_bytes += b.bytes;
    g->h_u_old2new.resize(g->n_u);
    g->h_u_new2old.resize(g->n_u);
    if (cudaMemcpy(g->h_u_old2new.data(), g->d_u_old2new, 4 * g->n_u, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(g->h_u_new2old.data(), g->d_u_new2old, 4 * g->n_u, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      fail(AHPP_ECUDA, "ahpp_load_graph_file: id maps");
    }
  }
  if (rc == AHPP_OK) select_chunk(g->dg, (uint32_t)chunk_choice(c.batch_chunk));
  if (rc == AHPP_OK) rc = alloc_query_state(g);
  if (rc == AHPP_OK) {
    // lambda: the configured value, else the cached estimate when it was
    // taken with the same T, else a new estimate on the device
    const uint32_t T_default =
        (uint32_t)std::ceil(std::log(100.0 * (double)g->n_u) / std::log(1.0 / (1.0 - c.alpha)));
    const uint32_t T_want = c.lambda_T > 0 ? (uint32_t)c.lambda_T : T_default;
    if (c.lambda > 0.0) {
      g->lambda = c.lambda;
    } else if (c.algo == AHPP_ASRP) {
      if (h.algo == (uint32_t)AHPP_ASRP && h.lambda_T == T_want && h.lambda > 0.0) {
        g->lambda = h.lambda;
        g->lambda_T = h.lambda_T;
      } else {
        rc = run_lambda(g);
      }
    } else {
      g->lambda = 1.0;
    }
  }
  if (rc != AHPP_OK) {
    const std::string keep = ahpp_last_error();
    ahpp_free_graph(g);
    set_error(keep);
    return rc;
  }
  *out = g;
  return AHPP_OK;
}
