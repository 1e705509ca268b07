// Batched multi-source push: state and launch parameters.
//
// A tile holds 32 (or 16) queries; every per-node state array of a tile is
// laid out [node][tile] (query-minor), so a warp that visits one neighbour
// reads or writes the tile's values of that neighbour as one 128-byte (or
// 64-byte) line.  Buffers are sized for the widest tile (kTile); the kernel
// instance of a launch's width indexes them with its own width.
// The graph is streamed once per round per tile, shared by all its queries.
// `groups` tiles run concurrently, each on its own slice of the persistent
// grid with its own barrier; a group walks its tiles one after another.
#pragma once
#include "../../include/ahpp.h"
#include "ahpp_internal.cuh"

namespace ahpp {

constexpr int kTile = 32;          // widest tile (queries per tile); serving uses this width
constexpr int kTileNarrow = 16;    // the other width of the batched kernel
constexpr int kRadixBits = 8;      // top-k digit width (per-lane histograms of 256 bins)
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kRadixPasses = 64 / kRadixBits;
// Block size of the batched kernel (three resident blocks per SM: measured
// best for this register budget).
constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kBMinBlocks = 3;
// Dynamic shared memory per block: the top-k radix histograms and sort
// buffer (4096 keys).
constexpr size_t kBatchSmem = 32 * 1024;

// Buffers of one concurrent group (one tile in flight).
struct alignas(64) TileBuf {
  float *r_u = nullptr, *pi = nullptr, *pic = nullptr;   // [n_u][kTile]
  float *t_v = nullptr, *t_a = nullptr;                  // [n_v][kTile], [n_a][kTile]
  float* t_a2 = nullptr;                                 // second t_A buffer (pushed for the next round)
  float* split_acc = nullptr;                            // [n_split][kTile]
  uint32_t* split_cnt = nullptr;                         // [n_split]
  RAcc* racc = nullptr;                                  // [5][kTile]: 3 rounds + 2 final sums
  GridBarrier* bar = nullptr;
  unsigned int* hist = nullptr;                          // [kRadixPasses][kTile][kRadixBins]
  unsigned long long* cand = nullptr;                    // [kTile][kmax] selected keys
  uint32_t* cand_cnt = nullptr;                          // [kTile]
};

constexpr int kMaxGroups = 8;

struct BatchState {
  TileBuf tb[kMaxGroups];
  uint32_t n_groups = 0;       // buffers allocated
  uint32_t kmax_cap = 0;       // candidate capacity per lane
};

struct BatchParams {
  uint32_t n = 0;                          // queries
  const uint32_t* q = nullptr;             // caller ids (device)
  const double* eps = nullptr;             // (device)
  const uint32_t* k = nullptr;             // (device), may be null when kmax == 0
  uint32_t kmax = 0;                       // output stride per query
  uint32_t* out_nodes = nullptr;           // [n][kmax] caller ids
  float* out_scores = nullptr;             // [n][kmax]
  uint32_t* out_n = nullptr;               // [n]
  ahpp_stats* out_stats = nullptr;         // [n], nullable
  float* out_dense = nullptr;              // [n][n_u] caller order, nullable
  const uint32_t* u_old2new = nullptr;
  const uint32_t* u_new2old = nullptr;
  int algo = 2;
  int kahan = 1;
  int switch_rule = 0;
  double lambda = 1.0;
  double log_inv = 0.0;
  uint32_t e_tot = 0;
  uint32_t max_rounds = 0;
  uint32_t groups = 1;
  uint32_t dense_div = 32;
  uint32_t tile = kTile;                   // queries per tile of this launch (kTile or kTileNarrow)
};

// Per-query control of one batched lane (kept in shared memory while a tile
// runs, in the slot table between serving steps).
struct LaneCtl {
  double eps_f;
  unsigned long long n_p, pushes;
  uint32_t rounds, switch_round;
  int phase, status, active, valid;
};

enum : uint32_t { kSlotFree = 0, kSlotNew = 1, kSlotRunning = 2, kSlotFinished = 3 };

// One serving slot (lane qi % kTile of tile qi / kTile).  The host writes
// eps_f, q_new, k and state = kSlotNew; the step kernel moves it to Running
// and Finished; the host frees Finished slots after reading the results.
struct SlotState {
  LaneCtl ctl;
  double eps_f;
  uint32_t q_new;          // internal id of the source
  uint32_t k;              // top-k size (already clamped)
  uint32_t state;
  uint32_t pad;
};

struct ServeParams {
  SlotState* slots = nullptr;        // [n_tiles * kTile]
  const TileBuf* tbufs = nullptr;    // [n_tiles], device array
  uint32_t* tile_round = nullptr;    // [n_tiles] rounds run by each tile (accumulator rotation)
  const uint32_t* live = nullptr;    // [n_live] tiles to advance this step
  uint32_t n_live = 0;
  uint32_t rounds_per_step = 1;
};

int launch_batch(const DevGraph& g, const BatchState& s, const BatchParams& p, bool bf16,
                 int grid, cudaStream_t stream);
int launch_serve_step(const DevGraph& g, const BatchParams& p, const ServeParams& sv, bool bf16,
                      int grid, cudaStream_t stream);
int batch_max_grid(bool bf16, int sm_count);

}  // namespace ahpp
