// C ABI entry points: graph load / free / info, single and batched queries.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ahpp_host.h"

namespace ahpp {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }

int cuda_fail(cudaError_t e, const char* where) {
  t_err = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return AHPP_ECUDA;
}

namespace {

constexpr uint32_t kMaxPowerIterations = 100000;

__global__ void k_scatter_dense(const float* __restrict__ pi, const uint32_t* __restrict__ n2o,
                                uint32_t n, float* __restrict__ out) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
    out[n2o[u]] = pi[u];
}

__global__ void k_ctl_to_stats(const QCtl* ctl, const unsigned int* maxr, const GridBarrier* bar,
                               double lambda, double eps_f, ahpp_stats* st) {
  ahpp_stats S;
  S.rounds = ctl->rounds;
  S.switch_round = ctl->switch_round;
  S.dense_rounds = ctl->dense_rounds;
  S.status = bar->err ? (uint32_t)kStatusWait : (uint32_t)ctl->status;
  S.pushes = ctl->pushes;
  S.n_p = ctl->n_p;
  S.resid_sum = ctl->resid_sum;
  S.reserve_sum = ctl->reserve_sum;
  S.mass_err = fabs(ctl->reserve_sum + ctl->resid_sum - 1.0);
  S.max_resid = (double)__uint_as_float(maxr[0]);
  S.lambda = lambda;
  S.eps_f = eps_f;
  S.served_ms = 0.0;
  *st = S;
}

struct WaitBars {
  const GridBarrier* bar[kMaxGroups];
  uint32_t n_bars;
};

__global__ void k_batch_wait_status(const WaitBars wb, uint32_t n, ahpp_stats* st, uint32_t* out_n) {
  unsigned int err = 0;
  for (uint32_t i = 0; i < wb.n_bars; ++i) err |= wb.bar[i]->err;
  if (!err) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (st) st[i].status = kStatusWait;
    if (out_n) out_n[i] = 0;
  }
}

}  // namespace

int kernel_algo(int algo) {
  return algo == AHPP_APP ? kAlgoAPP : algo == AHPP_ASRP ? kAlgoASRP : algo == AHPP_APP_S ? kAlgoAPPS : -1;
}

namespace {

int status_code(int status) {
  if (status == kStatusBadArg) { set_error("a query had q outside U or eps <= 0"); return AHPP_EINVAL; }
  if (status == kStatusCap) return AHPP_ENOTCONVERGED;
  if (status == kStatusWait) { set_error("a device wait gave up (grid barrier timeout)"); return AHPP_ETIMEOUT; }
  return AHPP_OK;
}

uint32_t auto_rounds(double eps_f, double alpha) {
  const double li = std::log(1.0 / (1.0 - alpha));
  const double t = std::ceil(std::log(1.0 / std::max(eps_f, 1e-300)) / li);
  return (uint32_t)std::min(1e6, 64.0 + 20.0 * std::max(t, 1.0));
}

double eps_f_of(const ahpp_graph* g, double eps) {
  return g->cfg.algo == AHPP_ASRP ? eps / g->lambda : eps / (double)(g->n_e + g->n_ea);
}

Q1Params q1_params(const ahpp_graph* g, uint32_t q_new, double eps) {
  Q1Params p;
  p.q = q_new;
  p.algo = kernel_algo(g->cfg.algo);
  p.kahan = g->cfg.kahan;
  p.switch_rule = g->cfg.switch_rule;
  p.eps_f = eps_f_of(g, eps);
  p.lambda = g->lambda;
  p.log_inv = std::log(1.0 / (1.0 - g->cfg.alpha));
  p.e_tot = (uint32_t)(g->n_e + g->n_ea);
  p.max_rounds = g->cfg.max_rounds ? g->cfg.max_rounds : auto_rounds(p.eps_f, g->cfg.alpha);
  p.dense_div = g->q1_dense_div;
  p.n_split = g->n_split1;
  p.trace_cap = 4096;
  p.smem_bytes = g->q1_smem;
  p.attr_push = g->q1_attr_push;
  p.ta_smem = g->q1_ta_smem;
  p.vw_max = g->q1_vw_max;
  return p;
}

// device scratch for the host entry points (grow-only)
struct IoBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

int ensure(ahpp_graph* g, IoBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return AHPP_OK;
  b.p = g->alloc(bytes);
  if (!b.p) { set_error("device allocation failed"); return AHPP_ENOMEM; }
  b.bytes = bytes;
  return AHPP_OK;
}

}  // namespace

Q1Params noalloc_params(const ahpp_graph* g, uint32_t q_new, double eps) {
  return q1_params(g, q_new, eps);
}

int reset_barrier(ahpp_graph* g, GridBarrier* bar, cudaStream_t stream, bool keep_trap) {
  AHPP_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), stream));
  if (g && g->wait_trap.load()) {
    // 0x40404040 arrivals: the block count is never reached
    AHPP_CUDA(cudaMemsetAsync(&bar->count, 0x40, sizeof(bar->count), stream));
    if (!keep_trap) g->wait_trap.store(0);
  }
  return AHPP_OK;
}

int barrier_status(GridBarrier* bar, cudaStream_t stream, int* status) {
  unsigned int err = 0;
  AHPP_CUDA(cudaMemcpyAsync(&err, &bar->err, sizeof(err), cudaMemcpyDeviceToHost, stream));
  AHPP_CUDA(cudaStreamSynchronize(stream));
  *status = err ? kStatusWait : kStatusOk;
  return AHPP_OK;
}

int run_query1_launch(ahpp_graph* g, uint32_t q_new, double eps, cudaStream_t stream) {
  Q1Params p = q1_params(g, q_new, eps);
  if (int rc = reset_barrier(g, g->q1.bar, stream)) return rc;
  int e = launch_query1(g->dg, g->q1, p, g->bf16, g->q1_grid, stream);
  if (e) return cuda_fail((cudaError_t)e, "k_query1 launch");
  return AHPP_OK;
}

int run_lambda(ahpp_graph* g) {
  const double alpha = g->cfg.alpha;
  uint32_t T = g->cfg.lambda_T > 0
                   ? (uint32_t)g->cfg.lambda_T
                   : (uint32_t)std::ceil(std::log(100.0 * (double)g->n_u) / std::log(1.0 / (1.0 - alpha)));
  g->lambda_T = T;
  Q1Params p = q1_params(g, 0, 1.0);
  p.lambda_mode = 1;
  p.algo = kAlgoASRP;
  p.eps_f = 0.0;
  p.kahan = 1;
  p.max_rounds = T;
  p.trace_cap = 0;
  if (int rc = reset_barrier(nullptr, g->q1.bar, g->stream)) return rc;
  int e = launch_query1(g->dg, g->q1, p, g->bf16, g->q1_grid, g->stream);
  if (e) return cuda_fail((cudaError_t)e, "lambda launch");
  unsigned int bits[2] = {0, 0};
  QCtl ctl;
  AHPP_CUDA(cudaMemcpyAsync(bits, g->q1.final_maxr_bits, sizeof(bits), cudaMemcpyDeviceToHost, g->stream));
  AHPP_CUDA(cudaMemcpyAsync(&ctl, g->q1.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, g->stream));
  int bst = kStatusOk;
  if (int rc = barrier_status(g->q1.bar, g->stream, &bst)) return rc;
  if (ctl.status == kStatusWait || bst == kStatusWait) {
    set_error("lambda estimate: device wait gave up");
    return AHPP_ETIMEOUT;
  }
  float maxpi;
  std::memcpy(&maxpi, &bits[1], 4);
  // FP32 rounding of pi_T is covered by a 1e-4 relative margin; the tail
  // term |U| (1-alpha)^T is added exactly as in Theorem 3.
  g->lambda = (double)maxpi * (1.0 + 1e-4) + (double)g->n_u * std::pow(1.0 - alpha, (double)T);
  return AHPP_OK;
}

int batch_plan(ahpp_graph* g, BatchParams& p) {
  if (g->bt_grid <= 0) {
    g->bt_grid = batch_max_grid(g->bf16, g->sm_count);
    if (g->bt_grid <= 0) { set_error("batched occupancy query failed"); return AHPP_ECUDA; }
  }
  (void)p;
  return AHPP_OK;
}

int ensure_batch(ahpp_graph* g, uint32_t groups, uint32_t kmax) {
  BatchState& s = g->bt;
  kmax = std::max<uint32_t>(kmax, 1);
  if (s.n_groups >= groups && s.kmax_cap >= kmax) return AHPP_OK;
  const DevGraph& G = g->dg;
  const size_t n_split = G.b_split_max;        // any chunk choice fits
  const uint32_t kcap = std::max(kmax, s.kmax_cap);
  const uint32_t ng = std::max(groups, s.n_groups);
  uint64_t bytes = 0;
  for (uint32_t i = 0; i < ng; ++i) {
    TileBuf& t = s.tb[i];
    const bool fresh = i >= s.n_groups;
    auto A = [&](size_t b) { bytes += b; return g->alloc(b); };
    if (fresh) {
      t.r_u = (float*)A((size_t)G.n_u * kTile * 4);
      t.pi = (float*)A((size_t)G.n_u * kTile * 4);
      t.pic = (float*)A((size_t)G.n_u * kTile * 4);
      t.t_v = (float*)A((size_t)std::max(G.n_v, 1u) * kTile * 4);
      t.t_a = (float*)A((size_t)std::max(G.n_a, 1u) * kTile * 4);
      t.t_a2 = (float*)A((size_t)std::max(G.n_a, 1u) * kTile * 4);
      t.split_acc = (float*)A(std::max<size_t>(n_split, 1) * kTile * 4);
      t.split_cnt = (uint32_t*)A(std::max<size_t>(n_split, 1) * 4);
      t.racc = (RAcc*)A(5 * kTile * sizeof(RAcc));
      t.bar = (GridBarrier*)A(sizeof(GridBarrier));
      t.hist = (unsigned int*)A((size_t)kRadixPasses * kTile * kRadixBins * 4);
      t.cand_cnt = (uint32_t*)A(kTile * 4);
      if (!t.r_u || !t.pi || !t.pic || !t.t_v || !t.t_a || !t.t_a2 || !t.split_acc || !t.split_cnt ||
          !t.racc || !t.bar || !t.hist || !t.cand_cnt) {
        set_error("batched state allocation failed");
        return AHPP_ENOMEM;
      }
      AHPP_CUDA(cudaMemset(t.bar, 0, sizeof(GridBarrier)));
    }
    if (fresh || kcap > s.kmax_cap) {
      t.cand = (unsigned long long*)A((size_t)kTile * kcap * 8);
      if (!t.cand) { set_error("batched state allocation failed"); return AHPP_ENOMEM; }
    }
  }
  if (s.n_groups == 0) g->tile_bytes = bytes / ng;
  s.n_groups = ng;
  s.kmax_cap = kcap;
  return AHPP_OK;
}

int run_batch_launch(ahpp_graph* g, uint32_t n, const uint32_t* d_q, const double* d_eps,
                     const uint32_t* d_k, uint32_t kmax, uint32_t* d_nodes, float* d_scores,
                     uint32_t* d_n, ahpp_stats* d_stats, float* d_dense, cudaStream_t stream) {
  const uint32_t groups = std::max<uint32_t>(1, std::min<uint32_t>(g->batch_groups, kMaxGroups));
  int rc = ensure_batch(g, groups, kmax);
  if (rc) return rc;
  BatchParams p;
  if ((rc = batch_plan(g, p))) return rc;
  const int grid = g->bt_grid / (int)groups * (int)groups;
  if (grid < (int)groups) { set_error("grid too small for the group count"); return AHPP_EINVAL; }
  p.n = n;
  p.q = d_q;
  p.eps = d_eps;
  p.k = d_k;
  p.kmax = kmax;
  p.out_nodes = d_nodes;
  p.out_scores = d_scores;
  p.out_n = d_n;
  p.out_stats = d_stats;
  p.out_dense = d_dense;
  p.u_old2new = g->d_u_old2new;
  p.u_new2old = g->d_u_new2old;
  p.algo = kernel_algo(g->cfg.algo);
  p.kahan = g->cfg.kahan;
  p.switch_rule = g->cfg.switch_rule;
  p.lambda = g->lambda;
  p.log_inv = std::log(1.0 / (1.0 - g->cfg.alpha));
  p.e_tot = (uint32_t)(g->n_e + g->n_ea);
  // one cap for the whole launch: generous enough for eps down to 1e-14 / lambda
  p.max_rounds = g->cfg.max_rounds ? g->cfg.max_rounds
                                   : auto_rounds(1e-14 / std::max(g->lambda, 1.0), g->cfg.alpha);
  p.groups = groups;
  p.tile = g->batch_tile;
  for (uint32_t i = 0; i < groups; ++i)
    if (int rc = reset_barrier(g, g->bt.tb[i].bar, stream, i + 1 < groups)) return rc;
  int e = launch_batch(g->dg, g->bt, p, g->bf16, grid, stream);
  if (e) return cuda_fail((cudaError_t)e, "k_batch launch");
  // a group whose barrier gave up may have left some of its tiles without
  // results: report every query of the launch as a device wait that gave up
  WaitBars wb{};
  for (uint32_t i = 0; i < groups; ++i) wb.bar[i] = g->bt.tb[i].bar;
  wb.n_bars = groups;
  k_batch_wait_status<<<std::max<uint32_t>(1, std::min<uint32_t>((n + 255) / 256, 1024)), 256, 0, stream>>>(
      wb, n, d_stats, d_n);
  AHPP_CUDA(cudaGetLastError());
  return AHPP_OK;
}

// The plain path into device buffers, on `s`; the caller holds g->mu and has
// validated the arguments.
int run_single_device(ahpp_graph* g, uint32_t q, double eps, uint32_t k, uint32_t* d_out_nodes,
                      float* d_out_scores, uint32_t* d_out_n, ahpp_stats* d_stats, cudaStream_t s) {
  int rc = run_query1_launch(g, g->h_u_old2new[q], eps, s);
  if (rc) return rc;
  if (k) {
    rc = topk_single(g, g->q1.pi, k, d_out_nodes, d_out_scores, d_out_n, s);
    if (rc) return rc;
  } else if (d_out_n) {
    AHPP_CUDA(cudaMemsetAsync(d_out_n, 0, 4, s));
  }
  if (d_stats) {
    k_ctl_to_stats<<<1, 1, 0, s>>>(g->q1.ctl, g->q1.final_maxr_bits, g->q1.bar, g->lambda,
                                   eps_f_of(g, eps), d_stats);
    AHPP_CUDA(cudaGetLastError());
  }
  return AHPP_OK;
}

}  // namespace ahpp

using namespace ahpp;

void* ahpp_graph::alloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    bufs.push_back({nullptr, bytes});
    return nullptr;
  }
  bufs.push_back({p, bytes});
  return p;
}

void ahpp_graph::release_all() {
  for (auto& b : bufs)
    if (b.p) cudaFree(b.p);
  bufs.clear();
}

namespace {
struct GraphIo {
  IoBuf q, eps, k, nodes, scores, n, stats, dense;
};
std::mutex g_io_mu;
std::vector<std::pair<const ahpp_graph*, GraphIo*>> g_io;
GraphIo* io_of(const ahpp_graph* g) {
  std::lock_guard<std::mutex> l(g_io_mu);
  for (auto& x : g_io)
    if (x.first == g) return x.second;
  g_io.push_back({g, new GraphIo()});
  return g_io.back().second;
}
void io_drop(const ahpp_graph* g) {
  std::lock_guard<std::mutex> l(g_io_mu);
  for (size_t i = 0; i < g_io.size(); ++i)
    if (g_io[i].first == g) {
      delete g_io[i].second;
      g_io.erase(g_io.begin() + i);
      return;
    }
}

int check_eps(double eps) {
  if (!(eps > 0.0) || !std::isfinite(eps)) { set_error("eps must be > 0 and finite"); return AHPP_EINVAL; }
  return AHPP_OK;
}
}  // namespace

extern "C" {

void ahpp_config_default(ahpp_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->alpha = 0.15;
  c->beta = 0.35;
  c->algo = AHPP_ASRP;
  c->lambda = 0.0;
  c->lambda_T = 0;
  c->attr_bf16 = 1;
  c->kahan = 1;
  c->switch_rule = 0;
  c->hbm_budget_bytes = 0;
  c->device = 0;
  c->max_rounds = 0;
  c->batch_tile = 0;
  c->batch_groups = 0;
}

const char* ahpp_last_error(void) { return t_err.c_str(); }

int ahpp_load_graph(const ahpp_graph_desc* desc, const ahpp_config* cfg, ahpp_graph** out) {
  ahpp::NvtxRange nvtx_range_("ahpp_load_graph");
  if (!desc || !out) { set_error("ahpp_load_graph: null argument"); return AHPP_EINVAL; }
  *out = nullptr;
  ahpp_config c;
  if (cfg) c = *cfg; else ahpp_config_default(&c);
  if (!(c.alpha > 0.0 && c.alpha < 1.0) || !(c.beta >= 0.0 && c.beta <= 1.0) ||
      kernel_algo(c.algo) < 0 || c.switch_rule < 0 || c.switch_rule > 2 ||
      (c.algo == AHPP_APP_S && c.switch_rule == 1)) {
    set_error("ahpp_load_graph: alpha must be in (0,1), beta in [0,1], algo APP, ASRP or APP_S "
              "(switch_rule 1, the printed formula, is ASRP's only)");
    return AHPP_EINVAL;
  }
  if (c.batch_tile != 0 && c.batch_tile != 16 && c.batch_tile != 32) {
    set_error("ahpp_load_graph: batch_tile must be 0, 16 or 32");
    return AHPP_EINVAL;
  }
  if (c.batch_groups > (uint32_t)kMaxGroups) {
    set_error("ahpp_load_graph: batch_groups must be at most 8");
    return AHPP_EINVAL;
  }
  if (chunk_choice(c.batch_chunk) < 0) {
    set_error("ahpp_load_graph: batch_chunk must be 0, 128, 256 or 512");
    return AHPP_EINVAL;
  }
  if (c.single_vec_width > 32 || (c.single_vec_width & (c.single_vec_width - 1))) {
    set_error("ahpp_load_graph: single_vec_width must be 0 or a power of two up to 32");
    return AHPP_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    set_error("ahpp_load_graph: no CUDA device available (the library has no CPU path)");
    return AHPP_ECUDA;
  }
  if (c.device < 0 || c.device >= ndev) { set_error("ahpp_load_graph: bad device ordinal"); return AHPP_EINVAL; }
  AHPP_CUDA(cudaSetDevice(c.device));
  ahpp_graph* g = new ahpp_graph();
  g->cfg = c;
  g->device = c.device;
  g->batch_tile = c.batch_tile ? c.batch_tile : (uint32_t)ahpp::kTile;
  g->batch_groups = c.batch_groups ? c.batch_groups : 1;
  g->q1_vw_max = c.single_vec_width ? c.single_vec_width : ahpp::kQ1VecWidthDefault;
  int rc = AHPP_OK;
  if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "ahpp_load_graph: device setup");
  }
  if (rc == AHPP_OK) rc = build_graph(desc, g);
  if (rc == AHPP_OK) select_chunk(g->dg, (uint32_t)chunk_choice(c.batch_chunk));
  if (rc == AHPP_OK) {
    if (c.algo == AHPP_ASRP && !(c.lambda > 0.0)) rc = run_lambda(g);
    else g->lambda = c.lambda > 0.0 ? c.lambda : 1.0;
  }
  if (rc != AHPP_OK) {
    std::string keep = t_err;
    ahpp_free_graph(g);
    t_err = keep;
    return rc;
  }
  *out = g;
  return AHPP_OK;
}

void ahpp_free_graph(ahpp_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  g->release_all();
  if (g->stream) cudaStreamDestroy(g->stream);
  io_drop(g);
  delete g;
}

int ahpp_get_graph_info(const ahpp_graph* g, ahpp_graph_info* info) {
  if (!g || !info) { set_error("null argument"); return AHPP_EINVAL; }
  info->n_u = g->n_u; info->n_v = g->n_v; info->n_a = g->n_a;
  info->n_e = g->n_e; info->n_ea = g->n_ea;
  info->lambda = g->lambda;
  info->lambda_T = g->lambda_T;
  info->graph_bytes = g->graph_bytes;
  info->query_state_bytes = g->q1_bytes;
  info->tile_state_bytes = g->tile_bytes;
  info->device = g->device;
  info->sm_count = g->sm_count;
  info->batch_tile = g->batch_tile;
  info->batch_groups = g->batch_groups;
  info->batch_chunk = kChunkSizes[g->dg.b_chunk];
  info->single_dense_div = g->q1_dense_div;
  info->single_attr_push = (uint32_t)g->q1_attr_push;
  info->single_vec_width = g->q1_vw_max;
  info->single_smem_bytes = g->q1_smem;
  return AHPP_OK;
}


int ahpp_query_device(ahpp_graph* g, uint32_t q, double eps, uint32_t k, uint32_t* d_out_nodes,
                      float* d_out_scores, uint32_t* d_out_n, ahpp_stats* d_stats, void* stream) {
  ahpp::NvtxRange nvtx_range_("ahpp_query_device");
  if (!g) { set_error("null graph"); return AHPP_EINVAL; }
  if (q >= g->n_u) { set_error("q is not a node of U"); return AHPP_EINVAL; }
  if (int rc = check_eps(eps)) return rc;
  if (k > AHPP_MAX_K) { set_error("k exceeds AHPP_MAX_K"); return AHPP_EINVAL; }
  if (k && (!d_out_nodes || !d_out_scores || !d_out_n)) { set_error("null output"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  return ahpp::run_single_device(g, q, eps, k, d_out_nodes, d_out_scores, d_out_n, d_stats, s);
}

static int finish_single(ahpp_graph* g, double eps, ahpp_stats* st) {
  QCtl ctl;
  unsigned int bits[2];
  AHPP_CUDA(cudaMemcpyAsync(&ctl, g->q1.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, g->stream));
  AHPP_CUDA(cudaMemcpyAsync(bits, g->q1.final_maxr_bits, sizeof(bits), cudaMemcpyDeviceToHost, g->stream));
  int bst = kStatusOk;
  if (int rc = barrier_status(g->q1.bar, g->stream, &bst)) return rc;
  if (bst == kStatusWait) ctl.status = kStatusWait;
  if (st) {
    st->rounds = ctl.rounds;
    st->switch_round = ctl.switch_round;
    st->dense_rounds = ctl.dense_rounds;
    st->status = (uint32_t)ctl.status;
    st->pushes = ctl.pushes;
    st->n_p = ctl.n_p;
    st->resid_sum = ctl.resid_sum;
    st->reserve_sum = ctl.reserve_sum;
    st->mass_err = std::fabs(ctl.reserve_sum + ctl.resid_sum - 1.0);
    float m;
    std::memcpy(&m, &bits[0], 4);
    st->max_resid = m;
    st->lambda = g->lambda;
    st->eps_f = eps_f_of(g, eps);
    st->served_ms = 0.0;
  }
  return status_code(ctl.status);
}

int ahpp_power_iteration(ahpp_graph* g, uint32_t q, uint32_t T, float* out_pi, ahpp_stats* st) {
  ahpp::NvtxRange nvtx_range_("ahpp_power_iteration");
  if (!g || !out_pi) { set_error("null argument"); return AHPP_EINVAL; }
  if (q >= g->n_u) { set_error("q is not a node of U"); return AHPP_EINVAL; }
  if (T == 0 || T > kMaxPowerIterations) {
    set_error("T must be in [1, " + std::to_string(kMaxPowerIterations) + "]");
    return AHPP_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  GraphIo* io = io_of(g);
  Q1Params p = q1_params(g, g->h_u_old2new[q], 1.0);
  p.pi_mode = 1;
  p.algo = kAlgoASRP;
  p.eps_f = 0.0;
  p.max_rounds = T;
  p.trace_cap = 0;
  if (int rc = reset_barrier(g, g->q1.bar, g->stream)) return rc;
  int e = launch_query1(g->dg, g->q1, p, g->bf16, g->q1_grid, g->stream);
  if (e) return cuda_fail((cudaError_t)e, "power iteration launch");
  int rc;
  if ((rc = ensure(g, io->dense, 4ull * g->n_u))) return rc;
  k_scatter_dense<<<std::max<int>(1, g->sm_count * 4), 256, 0, g->stream>>>(
      g->q1.pi, g->d_u_new2old, (uint32_t)g->n_u, (float*)io->dense.p);
  AHPP_CUDA(cudaGetLastError());
  AHPP_CUDA(cudaMemcpyAsync(out_pi, io->dense.p, 4ull * g->n_u, cudaMemcpyDeviceToHost, g->stream));
  rc = finish_single(g, 1.0, st);
  // T rounds are the stopping rule here, not a cap that was hit
  if (rc == AHPP_ENOTCONVERGED) rc = AHPP_OK;
  if (st && rc == AHPP_OK) { st->status = 0; st->eps_f = 0.0; }
  return rc;
}

int ahpp_query(ahpp_graph* g, uint32_t q, double eps, uint32_t k, uint32_t* out_nodes,
               float* out_scores, uint32_t* out_n, ahpp_stats* st) {
  ahpp::NvtxRange nvtx_range_("ahpp_query");
  if (!g) { set_error("null graph"); return AHPP_EINVAL; }
  if (q >= g->n_u) { set_error("q is not a node of U"); return AHPP_EINVAL; }
  if (int rc = check_eps(eps)) return rc;
  if (k > AHPP_MAX_K) { set_error("k exceeds AHPP_MAX_K"); return AHPP_EINVAL; }
  if (k && (!out_nodes || !out_scores || !out_n)) { set_error("null output"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  GraphIo* io = io_of(g);
  int rc = run_query1_launch(g, g->h_u_old2new[q], eps, g->stream);
  if (rc) return rc;
  const uint32_t kk = (uint32_t)std::min<uint64_t>(k, g->n_u);
  if (kk) {
    if ((rc = ensure(g, io->nodes, 4ull * AHPP_MAX_K)) || (rc = ensure(g, io->scores, 4ull * AHPP_MAX_K)) ||
        (rc = ensure(g, io->n, 16)))
      return rc;
    rc = topk_single(g, g->q1.pi, kk, (uint32_t*)io->nodes.p, (float*)io->scores.p,
                     (uint32_t*)io->n.p, g->stream);
    if (rc) return rc;
    AHPP_CUDA(cudaMemcpyAsync(out_nodes, io->nodes.p, 4ull * kk, cudaMemcpyDeviceToHost, g->stream));
    AHPP_CUDA(cudaMemcpyAsync(out_scores, io->scores.p, 4ull * kk, cudaMemcpyDeviceToHost, g->stream));
  }
  if (out_n) *out_n = kk;
  return finish_single(g, eps, st);
}

int ahpp_query_dense(ahpp_graph* g, uint32_t q, double eps, float* out_pi, ahpp_stats* st) {
  ahpp::NvtxRange nvtx_range_("ahpp_query_dense");
  if (!g || !out_pi) { set_error("null argument"); return AHPP_EINVAL; }
  if (q >= g->n_u) { set_error("q is not a node of U"); return AHPP_EINVAL; }
  if (int rc = check_eps(eps)) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  GraphIo* io = io_of(g);
  int rc = run_query1_launch(g, g->h_u_old2new[q], eps, g->stream);
  if (rc) return rc;
  if ((rc = ensure(g, io->dense, 4ull * g->n_u))) return rc;
  k_scatter_dense<<<std::max<int>(1, g->sm_count * 4), 256, 0, g->stream>>>(
      g->q1.pi, g->d_u_new2old, (uint32_t)g->n_u, (float*)io->dense.p);
  AHPP_CUDA(cudaGetLastError());
  AHPP_CUDA(cudaMemcpyAsync(out_pi, io->dense.p, 4ull * g->n_u, cudaMemcpyDeviceToHost, g->stream));
  return finish_single(g, eps, st);
}

int ahpp_query_batch_device(ahpp_graph* g, uint32_t n, const uint32_t* d_q, const double* d_eps,
                            const uint32_t* d_k, uint32_t kmax, uint32_t* d_out_nodes,
                            float* d_out_scores, uint32_t* d_out_n, ahpp_stats* d_stats,
                            void* stream) {
  ahpp::NvtxRange nvtx_range_("ahpp_query_batch_device");
  if (!g) { set_error("null graph"); return AHPP_EINVAL; }
  if (n == 0) return AHPP_OK;
  if (!d_q || !d_eps) { set_error("null input"); return AHPP_EINVAL; }
  if (kmax > AHPP_MAX_K) { set_error("kmax exceeds AHPP_MAX_K"); return AHPP_EINVAL; }
  if (kmax && (!d_k || !d_out_nodes || !d_out_scores || !d_out_n)) { set_error("null output"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  return run_batch_launch(g, n, d_q, d_eps, d_k, kmax, d_out_nodes, d_out_scores, d_out_n, d_stats,
                          nullptr, s);
}

static int batch_host(ahpp_graph* g, uint32_t n, const uint32_t* q, const double* eps,
                      const uint32_t* k, uint32_t* out_nodes, float* out_scores, uint32_t* out_n,
                      ahpp_stats* st, float* out_dense) {
  if (!g || (n && (!q || !eps))) { set_error("null argument"); return AHPP_EINVAL; }
  if (n == 0) return AHPP_OK;
  uint32_t kmax = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (q[i] >= g->n_u) { set_error("q[" + std::to_string(i) + "] is not a node of U"); return AHPP_EINVAL; }
    if (int rc = check_eps(eps[i])) return rc;
    if (k) {
      if (k[i] > AHPP_MAX_K) { set_error("k exceeds AHPP_MAX_K"); return AHPP_EINVAL; }
      kmax = std::max(kmax, (uint32_t)std::min<uint64_t>(k[i], g->n_u));
    }
  }
  if (kmax && (!out_nodes || !out_scores || !out_n)) { set_error("null output"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  GraphIo* io = io_of(g);
  int rc;
  if ((rc = ensure(g, io->q, 4ull * n)) || (rc = ensure(g, io->eps, 8ull * n)) ||
      (rc = ensure(g, io->k, 4ull * n)) || (rc = ensure(g, io->stats, sizeof(ahpp_stats) * n)) ||
      (rc = ensure(g, io->n, 4ull * n)))
    return rc;
  if (kmax && ((rc = ensure(g, io->nodes, 4ull * n * kmax)) || (rc = ensure(g, io->scores, 4ull * n * kmax))))
    return rc;
  if (out_dense && (rc = ensure(g, io->dense, 4ull * n * g->n_u))) return rc;
  AHPP_CUDA(cudaMemcpyAsync(io->q.p, q, 4ull * n, cudaMemcpyHostToDevice, g->stream));
  AHPP_CUDA(cudaMemcpyAsync(io->eps.p, eps, 8ull * n, cudaMemcpyHostToDevice, g->stream));
  if (k) AHPP_CUDA(cudaMemcpyAsync(io->k.p, k, 4ull * n, cudaMemcpyHostToDevice, g->stream));
  rc = run_batch_launch(g, n, (const uint32_t*)io->q.p, (const double*)io->eps.p,
                        (const uint32_t*)io->k.p, kmax, (uint32_t*)io->nodes.p, (float*)io->scores.p,
                        (uint32_t*)io->n.p, (ahpp_stats*)io->stats.p,
                        out_dense ? (float*)io->dense.p : nullptr, g->stream);
  if (rc) return rc;
  std::vector<ahpp_stats> hs(n);
  AHPP_CUDA(cudaMemcpyAsync(hs.data(), io->stats.p, sizeof(ahpp_stats) * n, cudaMemcpyDeviceToHost, g->stream));
  std::vector<uint32_t> hn(n, 0), hnodes;
  std::vector<float> hscores;
  if (kmax) {
    hnodes.resize((size_t)n * kmax);
    hscores.resize((size_t)n * kmax);
    AHPP_CUDA(cudaMemcpyAsync(hn.data(), io->n.p, 4ull * n, cudaMemcpyDeviceToHost, g->stream));
    AHPP_CUDA(cudaMemcpyAsync(hnodes.data(), io->nodes.p, 4ull * n * kmax, cudaMemcpyDeviceToHost, g->stream));
    AHPP_CUDA(cudaMemcpyAsync(hscores.data(), io->scores.p, 4ull * n * kmax, cudaMemcpyDeviceToHost, g->stream));
  }
  if (out_dense)
    AHPP_CUDA(cudaMemcpyAsync(out_dense, io->dense.p, 4ull * n * g->n_u, cudaMemcpyDeviceToHost, g->stream));
  AHPP_CUDA(cudaStreamSynchronize(g->stream));
  if (kmax) {
    size_t off = 0;
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t c = hn[i];
      std::memcpy(out_nodes + off, hnodes.data() + (size_t)i * kmax, 4ull * c);
      std::memcpy(out_scores + off, hscores.data() + (size_t)i * kmax, 4ull * c);
      out_n[i] = c;
      off += c;
    }
  } else if (out_n) {
    for (uint32_t i = 0; i < n; ++i) out_n[i] = 0;
  }
  int worst = AHPP_OK;
  for (uint32_t i = 0; i < n; ++i) {
    if (st) st[i] = hs[i];
    int c = status_code((int)hs[i].status);
    if (c == AHPP_ETIMEOUT) worst = c;
    else if (c && worst == AHPP_OK) worst = c;
  }
  return worst;
}

int ahpp_query_batch(ahpp_graph* g, uint32_t n, const uint32_t* q, const double* eps,
                     const uint32_t* k, uint32_t* out_nodes, float* out_scores, uint32_t* out_n,
                     ahpp_stats* st) {
  ahpp::NvtxRange nvtx_range_("ahpp_query_batch");
  return batch_host(g, n, q, eps, k, out_nodes, out_scores, out_n, st, nullptr);
}

int ahpp_query_batch_dense(ahpp_graph* g, uint32_t n, const uint32_t* q, const double* eps,
                           float* out_pi, ahpp_stats* st) {
  ahpp::NvtxRange nvtx_range_("ahpp_query_batch_dense");
  if (!out_pi) { set_error("null output"); return AHPP_EINVAL; }
  return batch_host(g, n, q, eps, nullptr, nullptr, nullptr, nullptr, st, out_pi);
}

}  // extern "C"

namespace {

// Device time (ms, CUDA events on the graph's stream) of one batched launch
// of the n queries already in io->q / io->eps, with the graph's current
// launch shape; no outputs besides the stats.
int time_batch(ahpp_graph* g, GraphIo* io, uint32_t n, float* ms) {
  cudaEvent_t a, b;
  AHPP_CUDA(cudaEventCreate(&a));
  AHPP_CUDA(cudaEventCreate(&b));
  int rc = AHPP_OK;
  if (cudaEventRecord(a, g->stream) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "autotune event");
  if (rc == AHPP_OK)
    rc = run_batch_launch(g, n, (const uint32_t*)io->q.p, (const double*)io->eps.p, nullptr, 0, nullptr,
                          nullptr, nullptr, (ahpp_stats*)io->stats.p, nullptr, g->stream);
  if (rc == AHPP_OK && (cudaEventRecord(b, g->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                        cudaEventElapsedTime(ms, a, b) != cudaSuccess))
    rc = cuda_fail(cudaGetLastError(), "autotune timing");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// Device time of single queries (k_query1 + nothing else) over the sample.
int time_single(ahpp_graph* g, const std::vector<uint32_t>& qs, double eps, float* ms) {
  cudaEvent_t a, b;
  AHPP_CUDA(cudaEventCreate(&a));
  AHPP_CUDA(cudaEventCreate(&b));
  int rc = AHPP_OK;
  if (cudaEventRecord(a, g->stream) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "autotune event");
  for (size_t i = 0; rc == AHPP_OK && i < qs.size(); ++i)
    rc = run_query1_launch(g, g->h_u_old2new[qs[i]], eps, g->stream);
  if (rc == AHPP_OK && (cudaEventRecord(b, g->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                        cudaEventElapsedTime(ms, a, b) != cudaSuccess))
    rc = cuda_fail(cudaGetLastError(), "autotune timing");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

}  // namespace

extern "C" int ahpp_autotune(ahpp_graph* g, uint32_t n_sample, const uint32_t* q_sample, double eps) {
  ahpp::NvtxRange nvtx_range_("ahpp_autotune");
  if (!g || (n_sample && !q_sample)) { ahpp::set_error("null argument"); return AHPP_EINVAL; }
  if (n_sample == 0) return AHPP_OK;
  if (int rc = check_eps(eps)) return rc;
  for (uint32_t i = 0; i < n_sample; ++i)
    if (q_sample[i] >= g->n_u) { ahpp::set_error("q_sample holds a node outside U"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(g->mu);
  AHPP_CUDA(cudaSetDevice(g->device));
  GraphIo* io = io_of(g);
  int rc;
  std::string log = "{";
  auto note = [&](const char* knob, uint32_t v, float t) {
    if (log.size() > 1) log += ", ";
    log += "\"" + std::string(knob) + "=" + std::to_string(v) + "\": " + std::to_string(t);
  };
  // ---- batched launch shape, one knob at a time (hub rows in shared memory,
  // entries per chunk of a long row, concurrent tile groups), every candidate
  // on the same queries: the sample replicated to fill four tiles; one
  // warm-up launch first
  const uint32_t n = std::max<uint32_t>(n_sample, 4 * (uint32_t)kTile);
  std::vector<uint32_t> qv(n);
  for (uint32_t i = 0; i < n; ++i) qv[i] = q_sample[i % n_sample];
  std::vector<double> ev(n, eps);
  if ((rc = ensure(g, io->q, 4ull * n)) || (rc = ensure(g, io->eps, 8ull * n)) ||
      (rc = ensure(g, io->stats, sizeof(ahpp_stats) * n)))
    return rc;
  AHPP_CUDA(cudaMemcpyAsync(io->q.p, qv.data(), 4ull * n, cudaMemcpyHostToDevice, g->stream));
  AHPP_CUDA(cudaMemcpyAsync(io->eps.p, ev.data(), 8ull * n, cudaMemcpyHostToDevice, g->stream));
  float ms = 0.f;
  if ((rc = time_batch(g, io, n, &ms)) != AHPP_OK) return rc;
  // try each value of one knob with the others fixed; keep the fastest
  auto tune_batch = [&](const char* knob, auto set, const std::vector<uint32_t>& values) -> int {
    float best = -1.f;
    uint32_t best_v = values[0];
    for (uint32_t v : values) {
      set(v);
      float t = 0.f;
      if (int r = time_batch(g, io, n, &t)) return r;
      note(knob, v, t / (float)n);
      if (best < 0.f || t < best) { best = t; best_v = v; }
    }
    set(best_v);
    return AHPP_OK;
  };
  const uint32_t saved_groups = g->batch_groups, saved_chunk = g->dg.b_chunk, saved_tile = g->batch_tile;
  rc = tune_batch("batch_tile", [&](uint32_t v) { g->batch_tile = v; }, {(uint32_t)kTile, (uint32_t)kTileNarrow});
  if (rc == AHPP_OK)
    rc = tune_batch("batch_chunk_choice", [&](uint32_t v) { select_chunk(g->dg, v); }, {1u, 0u, 2u});
  if (rc == AHPP_OK) rc = tune_batch("batch_groups", [&](uint32_t v) { g->batch_groups = v; }, {1u, 2u, 4u});
  if (rc != AHPP_OK) {
    g->batch_groups = saved_groups;
    select_chunk(g->dg, saved_chunk);
    g->batch_tile = saved_tile;
    return rc;
  }
  // ---- single-query path (up to four sample queries, one warm-up pass):
  // the frontier fraction 1/dense_div at which rounds switch from push to pull
  std::vector<uint32_t> q1(q_sample, q_sample + std::min<uint32_t>(n_sample, 4));
  if ((rc = time_single(g, q1, eps, &ms)) != AHPP_OK) return rc;
  auto tune_single = [&](const char* knob, auto set, const std::vector<uint32_t>& values) -> int {
    float best = -1.f;
    uint32_t best_v = values[0];
    for (uint32_t v : values) {
      set(v);
      float t = 0.f;
      if (int r = time_single(g, q1, eps, &t)) return r;
      note(knob, v, t / (float)q1.size());
      if (best < 0.f || t < best) { best = t; best_v = v; }
    }
    set(best_v);
    return AHPP_OK;
  };
  const uint32_t saved_div = g->q1_dense_div, saved_vw = g->q1_vw_max;
  rc = tune_single("single_vec_width", [&](uint32_t v) { g->q1_vw_max = v; }, {32u, 8u, 2u, 1u});
  if (rc == AHPP_OK)
    rc = tune_single("single_dense_div", [&](uint32_t v) { g->q1_dense_div = v; }, {32u, 8u, 16u, 64u, 128u});
  if (rc != AHPP_OK) {
    g->q1_dense_div = saved_div;
    g->q1_vw_max = saved_vw;
    return rc;
  }
  g->tune_log = log + "}";
  return AHPP_OK;
}

extern "C" int ahpp_autotune_report(const ahpp_graph* g, char* buf, size_t cap, size_t* len) {
  if (!g) { ahpp::set_error("null graph"); return AHPP_EINVAL; }
  const std::string& s = g->tune_log;
  if (len) *len = s.size();
  if (buf && cap) {
    const size_t n = std::min(cap - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return AHPP_OK;
}
