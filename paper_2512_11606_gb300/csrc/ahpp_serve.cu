// Serving loop: continuous batching of AHPP queries on one GPU.
//
// The server owns n_tiles tiles of kTile slots (one query per lane, the same
// query-minor layout as the batched path).  A host thread repeats one step:
//   1. admit queued requests into free slots (any tile, also tiles whose other
//      slots are in flight) - the slot table is the admission state;
//   2. launch the step kernel, which clears the admitted lanes, advances every
//      live tile by rounds_per_step rounds, and finalises the lanes that finish
//      (reserves, statistics, top-k);
//   3. read the slot table back, hand finished results to their tickets and
//      free those slots.
// Requests that arrive while a step runs are admitted at the next step, into
// whatever slots have freed up; their rounds then overlap on the device with
// the queries already in flight.  Each query's lane computes exactly what it
// would compute alone (no decision depends on the other lanes).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ahpp_host.h"

using namespace ahpp;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  uint32_t q;        // caller id
  double eps;
  uint32_t k;
  Clock::time_point t_submit;
};

struct Result {
  int rc = AHPP_OK;
  std::vector<uint32_t> nodes;
  std::vector<float> scores;
  ahpp_stats st{};
};

}  // namespace

struct ahpp_server {
  ahpp_graph* g = nullptr;
  uint32_t n_tiles = 0, n_slots = 0, kmax = AHPP_MAX_K, queue_cap = 65536, rounds_per_step = 4;
  int32_t single_max = 3;
  int grid = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  std::vector<TileBuf> h_tbufs;
  TileBuf* d_tbufs = nullptr;
  SlotState* d_slots = nullptr;
  uint32_t* d_tile_round = nullptr;
  uint32_t* d_live = nullptr;
  uint32_t* d_nodes = nullptr;
  float* d_scores = nullptr;
  uint32_t* d_n = nullptr;
  ahpp_stats* d_stats = nullptr;
  GridBarrier* d_bar = nullptr;
  BatchParams plan;                      // the batched kernel's shared-memory plan (hub rows)
  SlotState* h_slots = nullptr;          // pinned mirror of the slot table
  std::vector<uint64_t> slot_ticket;
  std::vector<Clock::time_point> slot_submit;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_set<uint64_t> pending;
  std::unordered_set<uint64_t> cancel_req;   // in-flight tickets to drop at the next step
  std::unordered_map<uint64_t, Result> done;
  uint64_t next_ticket = 1, submitted = 0, completed = 0, rejected = 0, steps = 0;
  uint32_t in_flight = 0;
  bool stop = false;
  int fatal = AHPP_OK;
  std::thread th;

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    allocs.push_back(p);
    return p;
  }
  void release() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (h_slots) cudaFreeHost(h_slots);
    h_slots = nullptr;
    if (stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

namespace {

// Light load: one request on the single-query path (the whole GPU on one
// query), its results through slot 0's output buffers (no tile lane runs).
int single_step(ahpp_server* s, const Request& r) {
  ahpp_graph* g = s->g;
  Result res;
  const uint32_t kk = (uint32_t)std::min<uint64_t>(r.k, g->n_u);
  res.nodes.resize(kk);
  res.scores.resize(kk);
  {
    std::lock_guard<std::mutex> glock(g->mu);
    int rc = run_single_device(g, r.q, r.eps, kk, s->d_nodes, s->d_scores, s->d_n, s->d_stats, s->stream);
    if (rc) return rc;
    if (kk) {
      AHPP_CUDA(cudaMemcpyAsync(res.nodes.data(), s->d_nodes, 4ull * kk, cudaMemcpyDeviceToHost, s->stream));
      AHPP_CUDA(cudaMemcpyAsync(res.scores.data(), s->d_scores, 4ull * kk, cudaMemcpyDeviceToHost, s->stream));
    }
    AHPP_CUDA(cudaMemcpyAsync(&res.st, s->d_stats, sizeof(ahpp_stats), cudaMemcpyDeviceToHost, s->stream));
    AHPP_CUDA(cudaStreamSynchronize(s->stream));
  }
  const Clock::time_point now = Clock::now();
  res.st.served_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
  res.rc = res.st.status == kStatusCap ? AHPP_ENOTCONVERGED : res.st.status == kStatusWait ? AHPP_ETIMEOUT : AHPP_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->done[r.ticket] = std::move(res);
    --s->in_flight;
    ++s->completed;
    ++s->steps;
  }
  s->cv_done.notify_all();
  return AHPP_OK;
}

// Cancelled in-flight requests give up their slots (under s->mu, between
// steps: the device holds no step of this server at this point).
void apply_cancellations(ahpp_server* s) {
  if (s->cancel_req.empty()) return;
  bool any = false;
  for (uint32_t slot = 0; slot < s->n_slots; ++slot) {
    SlotState& S = s->h_slots[slot];
    if (S.state != kSlotNew && S.state != kSlotRunning) continue;
    const uint64_t t = s->slot_ticket[slot];
    if (!s->cancel_req.count(t)) continue;
    S.state = kSlotFree;
    Result r;
    r.rc = AHPP_ECANCELED;
    s->done[t] = std::move(r);
    s->cancel_req.erase(t);
    --s->in_flight;
    any = true;
  }
  s->cancel_req.clear();      // the rest finished before the cancellation took effect
  if (any) s->cv_done.notify_all();
}

int server_step(ahpp_server* s) {
  NvtxRange nvtx_range_("ahpp_server_step");
  ahpp_graph* g = s->g;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    apply_cancellations(s);
  }
  // 0. light load: nothing in the tiles and a short queue
  {
    Request r{};
    bool single = false;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->single_max > 0 && s->in_flight == 0 && !s->queue.empty() &&
          s->queue.size() <= (size_t)s->single_max) {
        r = s->queue.front();
        s->queue.pop_front();
        ++s->in_flight;
        single = true;
      }
    }
    if (single) return single_step(s, r);
  }
  // 1. admission (under the lock)
  std::vector<uint32_t> live;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint32_t slot = 0; slot < s->n_slots && !s->queue.empty(); ++slot) {
      if (s->h_slots[slot].state != kSlotFree) continue;
      const Request r = s->queue.front();
      s->queue.pop_front();
      SlotState& S = s->h_slots[slot];
      std::memset(&S, 0, sizeof(S));
      S.eps_f = g->cfg.algo == AHPP_ASRP ? r.eps / g->lambda : r.eps / (double)(g->n_e + g->n_ea);
      S.q_new = g->h_u_old2new[r.q];
      S.k = (uint32_t)std::min<uint64_t>(r.k, g->n_u);
      S.state = kSlotNew;
      s->slot_ticket[slot] = r.ticket;
      s->slot_submit[slot] = r.t_submit;
      ++s->in_flight;
    }
    for (uint32_t t = 0; t < s->n_tiles; ++t)
      for (int l = 0; l < kTile; ++l) {
        const uint32_t st = s->h_slots[t * kTile + l].state;
        if (st == kSlotNew || st == kSlotRunning) { live.push_back(t); break; }
      }
  }
  if (live.empty()) return AHPP_OK;
  // 2. one step on the device
  AHPP_CUDA(cudaMemcpyAsync(s->d_slots, s->h_slots, sizeof(SlotState) * s->n_slots,
                            cudaMemcpyHostToDevice, s->stream));
  AHPP_CUDA(cudaMemcpyAsync(s->d_live, live.data(), 4 * live.size(), cudaMemcpyHostToDevice, s->stream));
  if (int rc = reset_barrier(g, s->d_bar, s->stream)) return rc;
  BatchParams p;
  p.kmax = s->kmax;
  p.out_nodes = s->d_nodes;
  p.out_scores = s->d_scores;
  p.out_n = s->d_n;
  p.out_stats = s->d_stats;
  p.u_old2new = g->d_u_old2new;
  p.u_new2old = g->d_u_new2old;
  p.algo = kernel_algo(g->cfg.algo);
  p.kahan = g->cfg.kahan;
  p.switch_rule = g->cfg.switch_rule;
  p.lambda = g->lambda;
  p.log_inv = std::log(1.0 / (1.0 - g->cfg.alpha));
  p.e_tot = (uint32_t)(g->n_e + g->n_ea);
  p.max_rounds = g->cfg.max_rounds ? g->cfg.max_rounds : 100000u;
  p.groups = 1;
  ServeParams sv;
  sv.slots = s->d_slots;
  sv.tbufs = s->d_tbufs;
  sv.tile_round = s->d_tile_round;
  sv.live = s->d_live;
  sv.n_live = (uint32_t)live.size();
  sv.rounds_per_step = s->rounds_per_step;
  const int e = launch_serve_step(g->dg, p, sv, g->bf16, s->grid, s->stream);
  if (e) return cuda_fail((cudaError_t)e, "serving step launch");
  AHPP_CUDA(cudaMemcpyAsync(s->h_slots, s->d_slots, sizeof(SlotState) * s->n_slots,
                            cudaMemcpyDeviceToHost, s->stream));
  int bst = kStatusOk;
  if (int rc = barrier_status(s->d_bar, s->stream, &bst)) return rc;   // also waits for the step
  if (bst == kStatusWait) {
    // a device wait gave up: the step may have stopped part-way through its
    // tiles, so no slot's state can be trusted; the loop fails every request
    set_error("serving step: a device wait gave up (grid barrier timeout)");
    return AHPP_ETIMEOUT;
  }
  // 3. hand out finished results
  std::vector<uint32_t> fin;
  for (uint32_t slot = 0; slot < s->n_slots; ++slot)
    if (s->h_slots[slot].state == kSlotFinished) fin.push_back(slot);
  std::vector<Result> res(fin.size());
  for (size_t i = 0; i < fin.size(); ++i) {
    const uint32_t slot = fin[i];
    const uint32_t kk = s->h_slots[slot].k;
    res[i].nodes.resize(kk);
    res[i].scores.resize(kk);
    if (kk) {
      AHPP_CUDA(cudaMemcpyAsync(res[i].nodes.data(), s->d_nodes + (size_t)slot * s->kmax, 4ull * kk,
                                cudaMemcpyDeviceToHost, s->stream));
      AHPP_CUDA(cudaMemcpyAsync(res[i].scores.data(), s->d_scores + (size_t)slot * s->kmax, 4ull * kk,
                                cudaMemcpyDeviceToHost, s->stream));
    }
    AHPP_CUDA(cudaMemcpyAsync(&res[i].st, s->d_stats + slot, sizeof(ahpp_stats),
                              cudaMemcpyDeviceToHost, s->stream));
  }
  AHPP_CUDA(cudaStreamSynchronize(s->stream));
  const Clock::time_point now = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t i = 0; i < fin.size(); ++i) {
      const uint32_t slot = fin[i];
      Result& r = res[i];
      r.st.served_ms = std::chrono::duration<double, std::milli>(now - s->slot_submit[slot]).count();
      r.rc = r.st.status == kStatusCap ? AHPP_ENOTCONVERGED
             : r.st.status == kStatusWait ? AHPP_ETIMEOUT : AHPP_OK;
      const uint64_t t = s->slot_ticket[slot];
      s->done[t] = std::move(r);
      s->h_slots[slot].state = kSlotFree;
      --s->in_flight;
      ++s->completed;
    }
    ++s->steps;
  }
  if (!fin.empty()) s->cv_done.notify_all();
  return AHPP_OK;
}

void server_loop(ahpp_server* s) {
  cudaSetDevice(s->g->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty() || s->in_flight > 0; });
      if (s->stop) break;
    }
    const int rc = server_step(s);
    if (rc != AHPP_OK) {
      std::lock_guard<std::mutex> lock(s->mu);
      s->fatal = rc;
      s->stop = true;
      s->cv_done.notify_all();
      break;
    }
  }
}

}  // namespace

extern "C" {

int ahpp_server_start(ahpp_graph* g, const ahpp_server_opts* opts, ahpp_server** out) {
  if (!g || !out) { set_error("ahpp_server_start: null argument"); return AHPP_EINVAL; }
  *out = nullptr;
  ahpp_server_opts o{};
  if (opts) o = *opts;
  if (o.tile != 0 && o.tile != (uint32_t)kTile) {
    set_error("ahpp_server_start: tile must be 0 or " + std::to_string(kTile));
    return AHPP_EINVAL;
  }
  AHPP_CUDA(cudaSetDevice(g->device));
  ahpp_server* s = new ahpp_server();
  s->g = g;
  if (o.queue_capacity) s->queue_cap = o.queue_capacity;
  if (o.rounds_per_step) s->rounds_per_step = o.rounds_per_step;
  if (o.single_max) s->single_max = o.single_max;
  // slots: requested, else what the HBM budget leaves after the graph, else 8 tiles
  const DevGraph& G = g->dg;
  const size_t n_split = G.b_split_max;        // any chunk choice fits
  const size_t tile_bytes = (size_t)G.n_u * kTile * 12 + (size_t)std::max(G.n_v, 1u) * kTile * 4 +
                            (size_t)std::max(G.n_a, 1u) * kTile * 4 + std::max<size_t>(n_split, 1) * (kTile + 1) * 4 +
                            (size_t)kRadixPasses * kTile * kRadixBins * 4 + (size_t)kTile * s->kmax * 8 + 4096;
  uint32_t tiles;
  if (o.max_slots) {
    tiles = (o.max_slots + kTile - 1) / kTile;
  } else if (g->cfg.hbm_budget_bytes) {
    const uint64_t used = g->graph_bytes + g->q1_bytes + g->tile_bytes * g->bt.n_groups;
    if (g->cfg.hbm_budget_bytes <= used + tile_bytes) {
      delete s;
      set_error("ahpp_server_start: hbm_budget_bytes leaves no room for one tile of slots");
      return AHPP_ENOMEM;
    }
    tiles = (uint32_t)std::min<uint64_t>(4096, (g->cfg.hbm_budget_bytes - used) / tile_bytes);
  } else {
    tiles = 8;
  }
  s->n_tiles = tiles;
  s->n_slots = tiles * kTile;
  int rc = AHPP_OK;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_slots, sizeof(SlotState) * s->n_slots) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "ahpp_server_start: stream / pinned table");
  }
  if (rc == AHPP_OK) {
    std::memset(s->h_slots, 0, sizeof(SlotState) * s->n_slots);
    s->slot_ticket.assign(s->n_slots, 0);
    s->slot_submit.assign(s->n_slots, Clock::time_point{});
    s->d_bar = (GridBarrier*)s->dalloc(sizeof(GridBarrier));
    s->d_slots = (SlotState*)s->dalloc(sizeof(SlotState) * s->n_slots);
    s->d_tile_round = (uint32_t*)s->dalloc(4ull * tiles);
    s->d_live = (uint32_t*)s->dalloc(4ull * tiles);
    s->d_nodes = (uint32_t*)s->dalloc(4ull * s->n_slots * s->kmax);
    s->d_scores = (float*)s->dalloc(4ull * s->n_slots * s->kmax);
    s->d_n = (uint32_t*)s->dalloc(4ull * s->n_slots);
    s->d_stats = (ahpp_stats*)s->dalloc(sizeof(ahpp_stats) * s->n_slots);
    s->d_tbufs = (TileBuf*)s->dalloc(sizeof(TileBuf) * tiles);
    bool ok = s->d_bar && s->d_slots && s->d_tile_round && s->d_live && s->d_nodes && s->d_scores &&
              s->d_n && s->d_stats && s->d_tbufs;
    s->h_tbufs.resize(tiles);
    for (uint32_t t = 0; ok && t < tiles; ++t) {
      TileBuf& b = s->h_tbufs[t];
      b.r_u = (float*)s->dalloc((size_t)G.n_u * kTile * 4);
      b.pi = (float*)s->dalloc((size_t)G.n_u * kTile * 4);
      b.pic = (float*)s->dalloc((size_t)G.n_u * kTile * 4);
      b.t_v = (float*)s->dalloc((size_t)std::max(G.n_v, 1u) * kTile * 4);
      b.t_a = (float*)s->dalloc((size_t)std::max(G.n_a, 1u) * kTile * 4);
      b.t_a2 = (float*)s->dalloc((size_t)std::max(G.n_a, 1u) * kTile * 4);
      b.split_acc = (float*)s->dalloc(std::max<size_t>(n_split, 1) * kTile * 4);
      b.split_cnt = (uint32_t*)s->dalloc(std::max<size_t>(n_split, 1) * 4);
      b.racc = (RAcc*)s->dalloc(5 * kTile * sizeof(RAcc));
      b.bar = s->d_bar;
      b.hist = (unsigned int*)s->dalloc((size_t)kRadixPasses * kTile * kRadixBins * 4);
      b.cand = (unsigned long long*)s->dalloc((size_t)kTile * s->kmax * 8);
      b.cand_cnt = (uint32_t*)s->dalloc(kTile * 4);
      ok = b.r_u && b.pi && b.pic && b.t_v && b.t_a && b.t_a2 && b.split_acc && b.split_cnt && b.racc &&
           b.hist && b.cand && b.cand_cnt;
      if (ok) {
        // the split accumulators and counters must start at zero (kept zero by the kernel)
        ok = cudaMemset(b.split_acc, 0, std::max<size_t>(n_split, 1) * kTile * 4) == cudaSuccess &&
             cudaMemset(b.split_cnt, 0, std::max<size_t>(n_split, 1) * 4) == cudaSuccess &&
             cudaMemset(b.racc, 0, 5 * kTile * sizeof(RAcc)) == cudaSuccess;
      }
    }
    if (!ok) {
      set_error("ahpp_server_start: device allocation failed for " + std::to_string(tiles) + " tiles");
      rc = AHPP_ENOMEM;
    }
  }
  if (rc == AHPP_OK) {
    if (cudaMemcpy(s->d_tbufs, s->h_tbufs.data(), sizeof(TileBuf) * tiles, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(s->d_tile_round, 0, 4ull * tiles) != cudaSuccess ||
        cudaMemset(s->d_slots, 0, sizeof(SlotState) * s->n_slots) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "ahpp_server_start: table upload");
    if (rc == AHPP_OK) {
      std::lock_guard<std::mutex> glock(g->mu);
      rc = batch_plan(g, s->plan);
      s->grid = g->bt_grid;
    }
  }
  if (rc != AHPP_OK) {
    s->release();
    delete s;
    return rc;
  }
  s->th = std::thread(server_loop, s);
  *out = s;
  return AHPP_OK;
}

int ahpp_submit(ahpp_server* s, uint32_t q, double eps, uint32_t k, uint64_t* ticket) {
  if (!s || !ticket) { set_error("ahpp_submit: null argument"); return AHPP_EINVAL; }
  if (q >= s->g->n_u) { set_error("ahpp_submit: q is not a node of U"); return AHPP_EINVAL; }
  if (!(eps > 0.0) || !std::isfinite(eps)) { set_error("ahpp_submit: eps must be > 0"); return AHPP_EINVAL; }
  if (k > AHPP_MAX_K) { set_error("ahpp_submit: k exceeds AHPP_MAX_K"); return AHPP_EINVAL; }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) { set_error(s->fatal ? "ahpp_submit: server failed" : "ahpp_submit: server stopped"); return AHPP_ESTATE; }
    if (s->queue.size() >= s->queue_cap) {
      ++s->rejected;
      set_error("ahpp_submit: queue full");
      return AHPP_EBUSY;
    }
    const uint64_t t = s->next_ticket++;
    s->queue.push_back(Request{t, q, eps, k, Clock::now()});
    s->pending.insert(t);
    ++s->submitted;
    *ticket = t;
  }
  s->cv_work.notify_one();
  return AHPP_OK;
}

int ahpp_wait(ahpp_server* s, uint64_t ticket, int timeout_ms, uint32_t* nodes, float* scores,
              uint32_t* n, ahpp_stats* st) {
  if (!s) { set_error("ahpp_wait: null server"); return AHPP_EINVAL; }
  std::unique_lock<std::mutex> lock(s->mu);
  if (!s->pending.count(ticket)) { set_error("ahpp_wait: unknown or already delivered ticket"); return AHPP_EINVAL; }
  auto ready = [&] { return s->done.count(ticket) > 0 || s->stop; };
  if (timeout_ms < 0) s->cv_done.wait(lock, ready);
  else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) return AHPP_ETIMEOUT;
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    set_error(s->fatal ? "ahpp_wait: the serving loop failed" : "ahpp_wait: server stopped");
    return s->fatal ? s->fatal : AHPP_ESTATE;
  }
  Result r = std::move(it->second);
  s->done.erase(it);
  s->pending.erase(ticket);
  lock.unlock();
  if (nodes && !r.nodes.empty()) std::memcpy(nodes, r.nodes.data(), 4 * r.nodes.size());
  if (scores && !r.scores.empty()) std::memcpy(scores, r.scores.data(), 4 * r.scores.size());
  if (n) *n = (uint32_t)r.nodes.size();
  if (st) *st = r.st;
  return r.rc;
}

int ahpp_cancel(ahpp_server* s, uint64_t ticket) {
  if (!s) { set_error("ahpp_cancel: null server"); return AHPP_EINVAL; }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->pending.count(ticket)) {
      set_error("ahpp_cancel: unknown or already delivered ticket");
      return AHPP_EINVAL;
    }
    if (s->done.count(ticket)) return AHPP_OK;      // finished: its result is delivered as usual
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
      if (it->ticket != ticket) continue;
      s->queue.erase(it);
      Result r;
      r.rc = AHPP_ECANCELED;
      s->done[ticket] = std::move(r);
      s->cv_done.notify_all();
      return AHPP_OK;
    }
    s->cancel_req.insert(ticket);      // on the device: dropped at the next step
  }
  s->cv_work.notify_one();
  return AHPP_OK;
}

int ahpp_server_info_get(ahpp_server* s, ahpp_server_info* info) {
  if (!s || !info) { set_error("ahpp_server_info_get: null argument"); return AHPP_EINVAL; }
  std::lock_guard<std::mutex> lock(s->mu);
  info->submitted = s->submitted;
  info->completed = s->completed;
  info->rejected = s->rejected;
  info->steps = s->steps;
  info->in_flight = s->in_flight;
  info->queued = (uint32_t)s->queue.size();
  info->slots = s->n_slots;
  return s->fatal;
}

int ahpp_server_stop(ahpp_server* s) {
  if (!s) return AHPP_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->g->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  const int rc = s->fatal;
  s->release();
  delete s;
  return rc;
}

}  // extern "C"
