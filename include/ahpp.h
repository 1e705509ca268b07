/*
 * ahpp.h - C ABI of the GB300 (sm_103a) library for approximate single-source
 * AHPP queries on attributed bipartite graphs.
 *
 * The operation (Section 2.3, "Our Problem"): given an attributed bipartite
 * graph G = (U, V, E, A, E_A) (Section 2.1), a restart probability alpha, an
 * attribute jumping probability beta, a source node u in U and an error
 * threshold eps, return pi_hat(u, u_i) for every u_i in U with
 * |pi(u, u_i) - pi_hat(u, u_i)| <= eps, where pi is AHPP (Def. 2, Eq. 3):
 *     pi(u_i, u_j) = sum_l alpha (1 - alpha)^l P^l[u_i, u_j],
 *     P = (1 - beta) P_S + beta P_A,  P_S of Eq. 1,  P_A of Eq. 2.
 * Two push algorithms compute it: APP (Algorithm 3) and ASRP (Algorithm 4,
 * with the lambda of Theorem 3).  This library adds top-k selection,
 * batching of many sources, and a serving loop.
 *
 * Conventions for every entry point:
 *   - Return value: AHPP_OK (0) or a negative AHPP_E* code; nothing throws
 *     across the ABI.  ahpp_last_error() returns a message for the last
 *     failure on the calling thread.
 *   - Pointers named h_* or documented as "host" are caller-owned host
 *     memory; the library copies what it needs before returning.  Pointers
 *     named d_* are caller-owned device memory of the graph's device.
 *   - Node ids are 0-based: U ids in [0, n_u), V in [0, n_v), A in [0, n_a).
 *   - Top-k results are sorted by score descending, then node id ascending;
 *     k is clamped to n_u and may be at most AHPP_MAX_K.
 *   - A graph handle may be used from one host thread at a time (the
 *     serving loop serialises its own access).
 */
#ifndef AHPP_H_
#define AHPP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AHPP_OK 0
#define AHPP_EINVAL (-1)          /* bad argument: q not in U, eps <= 0, alpha not in (0,1), ... */
#define AHPP_ENOMEM (-2)          /* device or host allocation failed, or HBM budget exceeded */
#define AHPP_ECUDA (-3)           /* a CUDA call failed (message in ahpp_last_error) */
#define AHPP_ENOTCONVERGED (-4)   /* round cap reached; partial results were written */
#define AHPP_EBUSY (-5)           /* serving: no free slot / admission queue full */
#define AHPP_ETIMEOUT (-6)        /* serving: wait timed out, or a device wait gave up */
#define AHPP_ESTATE (-7)          /* handle used in the wrong state (e.g. server stopped) */
#define AHPP_ECANCELED (-8)       /* serving: the request was cancelled (ahpp_cancel) */

#define AHPP_APP 1                /* Algorithm 3 */
#define AHPP_ASRP 2               /* Algorithm 4 */
#define AHPP_APP_S 3              /* APP(S) of Exp-2 (Section 5): APP's per-node thresholds
                                     r_max (|N(u)| + |A(u)|), switching to Algorithm 4's
                                     synchronous pushes when the push count reaches
                                     2 (|E| + |E_A|) log_{1/(1-alpha)}(M' / r_max), M' the
                                     largest r(u) / (|N(u)| + |A(u)|); stops on APP's test */

#define AHPP_MAX_K 4096u          /* largest k accepted by the top-k entry points */

typedef struct ahpp_graph ahpp_graph;   /* opaque; owns all device memory of a graph */
typedef struct ahpp_server ahpp_server; /* opaque; a serving loop over one graph */

/* Graph input (Section 2.1), caller-owned host arrays, copied during load.
 * Edges (u, v, w(u,v)) with w > 0; duplicate (u, v) pairs are merged by
 * summing weights.  Node-attribute tuples (u, a, w(u,a)) with w > 0, merged
 * the same way.  e_w == NULL means unit weights.  Counts below 2^31. */
typedef struct {
    uint64_t n_u, n_v, n_a;
    uint64_t n_e;
    const uint32_t *e_u, *e_v;
    const float *e_w;
    uint64_t n_ea;
    const uint32_t *ea_u, *ea_a;
    const float *ea_w;
} ahpp_graph_desc;

/* Per-graph configuration.  alpha and beta live here because lambda
 * (Theorem 3) depends on them. */
typedef struct {
    double alpha;              /* restart probability, (0, 1); default 0.15 */
    double beta;               /* attribute jumping probability, [0, 1]; default 0.35 */
    int algo;                  /* AHPP_ASRP (default), AHPP_APP or AHPP_APP_S */
    double lambda;             /* ASRP's lambda; <= 0: Theorem 3 estimate at load (default) */
    int lambda_T;              /* iterations of the Theorem 3 estimate; 0: ceil(ln(100|U|)/ln(1/(1-alpha))) */
    int attr_bf16;             /* store attribute weights as bfloat16 (default 1) */
    int kahan;                 /* Kahan-compensated FP32 reserves (default 1) */
    int switch_rule;           /* switch test: 0 corrected (default), 1 as printed (ASRP only), 2 never */
    uint64_t hbm_budget_bytes; /* cap on device memory of graph + query state; 0 = no cap */
    int device;                /* CUDA device ordinal (default 0) */
    uint32_t max_rounds;       /* round cap per query; 0: automatic */
    uint32_t batch_tile;       /* queries per batched tile: 16 or 32; 0: 32 (ahpp_autotune picks one);
                                  serving always uses tiles of 32 */
    uint32_t batch_groups;     /* tiles processed concurrently, 1..8; 0: 1 (ahpp_autotune picks 1, 2 or 4) */
    uint32_t batch_chunk;      /* entries per chunk of a long row in the batched kernel: 128, 256 or
                                  512; 0: 256 (ahpp_autotune picks one) */
    uint32_t single_vec_width; /* single-query kernel: at most this many lanes walk one short row
                                  (1, 2, 4, 8, 16 or 32); 0: 2 (ahpp_autotune picks one) */
} ahpp_config;

/* Per-query statistics. */
typedef struct {
    uint32_t rounds;           /* push rounds executed */
    uint32_t switch_round;     /* ASRP: first synchronous round (0 = never switched) */
    uint32_t dense_rounds;     /* rounds run as full-graph pull sweeps */
    uint32_t status;           /* 0 converged, 1 round cap, 2 device wait gave up, 3 bad q or eps */
    uint64_t pushes;           /* U-node pushes (sum of frontier sizes) */
    uint64_t n_p;              /* Algorithm 4's push counter at exit */
    double resid_sum;          /* sum_u r(u) at exit (FP64 reduction) */
    double reserve_sum;        /* sum_u pi_hat(u) at exit (FP64 reduction) */
    double mass_err;           /* |reserve_sum + resid_sum - 1| (dangling rows leak mass) */
    double max_resid;          /* max_u r(u) at exit */
    double lambda;             /* lambda used (ASRP) */
    double eps_f;              /* eps / lambda (ASRP) or r_max (APP) */
    double served_ms;          /* serving: submit-to-completion time in ms (0 otherwise) */
} ahpp_stats;

typedef struct {
    uint64_t n_u, n_v, n_a, n_e, n_ea;   /* after merging duplicates */
    double lambda;                       /* Theorem 3 estimate (or the configured value) */
    uint32_t lambda_T;
    uint64_t graph_bytes;                /* device bytes held by the graph */
    uint64_t query_state_bytes;          /* device bytes per single-query state */
    uint64_t tile_state_bytes;           /* device bytes per batched tile */
    int device;
    int sm_count;
    uint32_t batch_tile, batch_groups;   /* batched launch shape in use */
    uint32_t batch_chunk;                /* batched: entries per chunk of a long row */
    /* single-query kernel (the plain path): pull rounds once the frontier's
     * degree sum exceeds 1/single_dense_div of |E| + |E_A|; the attribute hop
     * of pull rounds pushed from phase 2 through shared memory (1) or pulled
     * over A->U (0); rows of up to 64 entries walked by at most
     * single_vec_width lanes each (1 = one row per lane); single_smem_bytes
     * of shared memory per block. */
    uint32_t single_dense_div, single_attr_push, single_vec_width, single_smem_bytes;
} ahpp_graph_info;

/* Serving options. */
typedef struct {
    uint32_t max_slots;        /* concurrent queries on the device (rounded up to whole tiles);
                                  0: what hbm_budget_bytes leaves after the graph, else 256 */
    uint32_t queue_capacity;   /* pending requests before AHPP_EBUSY; 0: 65536 */
    uint32_t tile;             /* queries per tile; 0 or the library's tile width */
    uint32_t rounds_per_step;  /* push rounds per device step between admissions; 0: 4 */
    int32_t single_max;        /* light load: while no tile lane runs and at most this many
                                  requests wait, answer the oldest on the single-query path
                                  (lower latency than a tile round for one query);
                                  0: 3, < 0: never */
} ahpp_server_opts;

/* Fill *cfg with the defaults listed above. */
void ahpp_config_default(ahpp_config *cfg);

/* Message of the last failure on this thread ("" if none).  Valid until the
 * next call on the same thread. */
const char *ahpp_last_error(void);

/* Load G onto cfg->device: merges duplicates, relabels nodes by degree
 * internally (ids at the ABI stay the caller's), builds the four
 * adjacency directions (U->V, V->U, U->A, A->U) with their normalisers
 * (Eq. 1, Eq. 2), and, for ASRP with cfg->lambda <= 0, runs the lambda
 * estimate of Theorem 3 on the device.  desc and cfg are caller-owned and
 * copied.  Errors: AHPP_EINVAL (id out of range, w <= 0, bad alpha/beta/algo,
 * counts >= 2^31), AHPP_ENOMEM (budget or allocation), AHPP_ECUDA. */
int ahpp_load_graph(const ahpp_graph_desc *desc, const ahpp_config *cfg, ahpp_graph **out);

/* Graph cache.  ahpp_save_graph writes a loaded graph to `path`: its device
 * arrays after duplicate merging, relabelling and the adjacency build, the
 * normalisers and coefficients (Eq. 1, Eq. 2), the work items, and the lambda
 * estimate (Theorem 3).  ahpp_load_graph_file reads such a file onto
 * cfg->device without redoing that work; cfg's alpha, beta and attr_bf16
 * must equal the cached graph's (the coefficients depend on them), the other
 * fields apply as in ahpp_load_graph.  lambda: cfg->lambda if > 0, else the
 * cached estimate if it was taken with the same lambda_T, else a new one.
 * The file is in native byte order for the same build of this library and
 * ends with a checksum of its contents; the loader checks the header, the
 * buffer table, the length and the checksum but does not re-derive the
 * arrays, so load only files that ahpp_save_graph wrote.
 * Errors: AHPP_EINVAL (null argument, unreadable, truncated, damaged or
 * foreign file, mismatched alpha / beta / attr_bf16), AHPP_ENOMEM,
 * AHPP_ECUDA. */
int ahpp_save_graph(ahpp_graph *g, const char *path);
int ahpp_load_graph_file(const char *path, const ahpp_config *cfg, ahpp_graph **out);

/* Release every device and host resource of g (NULL is ignored). */
void ahpp_free_graph(ahpp_graph *g);

/* Sizes, lambda and launch shape of a loaded graph. */
int ahpp_get_graph_info(const ahpp_graph *g, ahpp_graph_info *info);

/* One eps-approximate single-source query (Section 2.3) from q, pushed on the
 * whole GPU by one persistent launch (the plain one-query-at-a-time path),
 * then top-k.  Host outputs: out_nodes[k], out_scores[k], *out_n = number
 * written (min(k, n_u)).  st may be NULL.  Errors: AHPP_EINVAL,
 * AHPP_ENOTCONVERGED (results written from the partial reserves),
 * AHPP_ECUDA. */
int ahpp_query(ahpp_graph *g, uint32_t q, double eps, uint32_t k,
               uint32_t *out_nodes, float *out_scores, uint32_t *out_n, ahpp_stats *st);

/* As ahpp_query, but returns the whole reserve vector: out_pi[n_u] (host),
 * indexed by the caller's U ids. */
int ahpp_query_dense(ahpp_graph *g, uint32_t q, double eps, float *out_pi, ahpp_stats *st);

/* Power Iteration (Algorithm 1) from q for T iterations, on the GPU:
 * out_pi[n_u] (host, caller's U ids) receives Algorithm 1's iterate
 * pi_T = alpha sum_{l<T} (1-alpha)^l e_q P^l + (1-alpha)^T e_q P^T, whose
 * distance to the exact AHPP vector (Eq. 3) is at most (1-alpha)^T in every
 * entry (FP32 arithmetic, Kahan-compensated sums).  It runs T synchronous
 * push rounds from e_q (every positive residue pushed each round) and adds
 * the final residues to the reserves.  A reference for graphs too large for
 * a CPU solve.  st (nullable): rounds = T, mass sums of the push.
 * AHPP_EINVAL for q outside U, T == 0 or T > 100000, NULL g or out_pi. */
int ahpp_power_iteration(ahpp_graph *g, uint32_t q, uint32_t T, float *out_pi, ahpp_stats *st);

/* n independent queries (q[i], eps[i], k[i]) pushed together: queries are
 * packed into tiles of 32 that share every read of the graph, and one
 * persistent launch runs all tiles.  Host inputs q[n], eps[n], k[n].  Host
 * outputs, concatenated in query order with offsets = exclusive prefix sum of
 * min(k[i], n_u): out_nodes, out_scores; out_n[i] = count for query i.  st
 * (n entries) may be NULL.  Each result equals, within the tolerance of the
 * arithmetic, the result of the same query alone. */
int ahpp_query_batch(ahpp_graph *g, uint32_t n, const uint32_t *q, const double *eps,
                     const uint32_t *k, uint32_t *out_nodes, float *out_scores,
                     uint32_t *out_n, ahpp_stats *st);

/* Batched queries with the whole reserve vectors: out_pi is host [n][n_u]. */
int ahpp_query_batch_dense(ahpp_graph *g, uint32_t n, const uint32_t *q, const double *eps,
                           float *out_pi, ahpp_stats *st);

/* Device-resident variant of ahpp_query_batch for callers that keep inputs
 * and outputs in device memory: d_q[n], d_eps[n], d_k[n] on the graph's
 * device; d_out_nodes / d_out_scores sized n * kmax (query i writes at
 * i * kmax), d_out_n[n]; d_stats (n entries, device) may be NULL.  kmax is
 * the largest k in d_k (at most AHPP_MAX_K).  stream is a cudaStream_t (NULL
 * = the graph's own stream); the call is asynchronous with respect to the
 * host except for internal bookkeeping. */
int ahpp_query_batch_device(ahpp_graph *g, uint32_t n, const uint32_t *d_q, const double *d_eps,
                            const uint32_t *d_k, uint32_t kmax, uint32_t *d_out_nodes,
                            float *d_out_scores, uint32_t *d_out_n, ahpp_stats *d_stats,
                            void *stream);

/* ahpp_query_dense without any device allocation, for callers that cannot
 * allocate at query time (a framework that owns the whole device memory pool,
 * or a thread that must not take the device synchronisation cudaMalloc /
 * cudaFree may cause).  The paper has no counterpart: this is a deployment
 * variant of the single-query push.  The query's working state lives in one
 * static device array of 32 MiB per device, held until the process exits;
 * graphs whose single-query state exceeds it are rejected with AHPP_EINVAL.
 * Outputs: d_out_pi[n_u] (device, caller ids).  stream: cudaStream_t (NULL =
 * the graph's).  The call waits for its stream before returning; calls are
 * serialised because they share the array (overlapping use would race).  The
 * first call on a device resolves the array's address with that device
 * current: make it before any stream capture.  Returns AHPP_OK,
 * AHPP_ENOTCONVERGED, AHPP_EINVAL, AHPP_ETIMEOUT (a device wait gave up) or
 * AHPP_ECUDA. */
int ahpp_query_dense_noalloc(ahpp_graph *g, uint32_t q, double eps, float *d_out_pi, void *stream);

/* Device-resident single query (the plain path) on stream (NULL = graph's):
 * d_out_nodes[k], d_out_scores[k], d_out_n[1], d_stats (nullable). */
int ahpp_query_device(ahpp_graph *g, uint32_t q, double eps, uint32_t k,
                      uint32_t *d_out_nodes, float *d_out_scores, uint32_t *d_out_n,
                      ahpp_stats *d_stats, void *stream);

/* Autotune the launch shapes on a sample of the caller's queries, timing
 * every candidate on the device (CUDA events on the graph's stream), one
 * knob at a time with the others fixed.  Batched kernel, on the sample
 * replicated to fill four tiles of 32: queries per tile (32, 16), entries per
 * chunk of a long row (128, 256, 512), then tiles processed concurrently
 * (1, 2, 4).  Single-query kernel, on
 * up to four sample queries: lanes per short row (32, 8, 2, 1: at most that
 * many lanes walk one row), then the frontier fraction 1/dense_div (8, 16,
 * 32, 64, 128) past which rounds run as pull sweeps.  Every candidate gives the same results
 * within FP32 rounding (only the order of sums changes).  The choice is
 * stored in the graph and reported by ahpp_get_graph_info; the measured
 * times by ahpp_autotune_report.  Do not run it while a server on g is
 * running.  q_sample: host array of n_sample query ids (n_sample == 0
 * changes nothing).  AHPP_EINVAL for a NULL g or q_sample, an id outside U
 * or a bad eps. */
int ahpp_autotune(ahpp_graph *g, uint32_t n_sample, const uint32_t *q_sample, double eps);

/* The last ahpp_autotune's measurements as a JSON object text, one entry
 * "knob=value": milliseconds of device time per query (the batched launch's
 * time over its queries; a single query's time), in the order measured.
 * Copies at most cap - 1 bytes and a terminating zero into buf (host) when
 * buf and cap are given; *len (nullable) receives the full length.  "" if
 * the graph was never tuned.  AHPP_EINVAL for a NULL g. */
int ahpp_autotune_report(const ahpp_graph *g, char *buf, size_t cap, size_t *len);

/* Serving (continuous batching).  A server owns a pool of device slots
 * (one query each, in tiles of 32) sized by opts->max_slots or the HBM
 * budget; submitted requests wait in a queue and are admitted into slots as
 * slots free up, while queries already on the device keep advancing
 * rounds_per_step rounds per device step.  Each request may have its own eps
 * and k.  opts may be NULL (defaults).  AHPP_ENOMEM if not even one tile fits
 * the budget. */
int ahpp_server_start(ahpp_graph *g, const ahpp_server_opts *opts, ahpp_server **out);

/* Queue one request; *ticket identifies it.  AHPP_EBUSY if the queue is
 * full, AHPP_EINVAL for bad arguments, AHPP_ESTATE after stop. */
int ahpp_submit(ahpp_server *s, uint32_t q, double eps, uint32_t k, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a ticket's result; host outputs
 * nodes[k], scores[k], *n; st nullable.  Returns the query's own status
 * (AHPP_OK / AHPP_ENOTCONVERGED), AHPP_ETIMEOUT if not done in time (the
 * ticket stays valid), AHPP_EINVAL for an unknown ticket.  A result is
 * delivered once. */
int ahpp_wait(ahpp_server *s, uint64_t ticket, int timeout_ms, uint32_t *nodes, float *scores,
              uint32_t *n, ahpp_stats *st);

/* Cancel a submitted request that has not been delivered.  A queued request
 * is dropped; a request already on the device gives up its slot at the next
 * step boundary.  Its ahpp_wait then returns AHPP_ECANCELED, unless the
 * query finished before the cancellation took effect, in which case the
 * result is delivered as usual.  AHPP_EINVAL for an unknown or already
 * delivered ticket. */
int ahpp_cancel(ahpp_server *s, uint64_t ticket);

/* Server counters: completed, in flight, queued, rejected, device steps. */
typedef struct {
    uint64_t submitted, completed, rejected, steps;
    uint32_t in_flight, queued, slots;
} ahpp_server_info;
int ahpp_server_info_get(ahpp_server *s, ahpp_server_info *info);

/* Stop the loop, drop queued requests, release the slots and the server.
 * Safe on NULL.  No other call on s may run concurrently or follow. */
int ahpp_server_stop(ahpp_server *s);

/* Self-test of the device-side failure detection (no graph needed).  Every
 * wait inside the persistent kernels is a grid barrier whose spin is bounded
 * (about a second); when it gives up it raises an error flag, the kernel
 * unwinds and the query reports AHPP_ETIMEOUT.  This runs that barrier with
 * more participants than blocks, so it can never fill: *blocks_gave_up
 * receives how many blocks reported giving up (2 expected) and *context_ok
 * whether a kernel launched afterwards ran (1 expected).  Takes a few
 * seconds.  AHPP_EINVAL for bad arguments, AHPP_ECUDA if a CUDA call fails. */
int ahpp_selftest_wait_timeout(int device, int *blocks_gave_up, int *context_ok);

/* Self-test of the same detection inside the query kernels (no fault, no
 * hang: every wait is bounded).  Arms a one-shot trap on g: the next
 * persistent launch made through g (ahpp_query / ahpp_query_dense /
 * ahpp_query_device, the batched entry points, ahpp_query_dense_noalloc,
 * ahpp_power_iteration, or a serving step) clears its grid barrier with a
 * counter that can never reach the block count, so the launch's first wait,
 * before any push round, gives up after about a second.  That call must then
 * report AHPP_ETIMEOUT (batched: stats status 2 for every query; serving:
 * the server fails every request with AHPP_ETIMEOUT and stops), and the
 * graph stays usable for the next call.  AHPP_EINVAL for a NULL g. */
int ahpp_selftest_arm_wait_timeout(ahpp_graph *g);

#ifdef __cplusplus
}
#endif
#endif /* AHPP_H_ */
