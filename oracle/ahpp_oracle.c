/*
 * CPU oracle for approximate single-source AHPP (plain C, FP64, one thread).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use this code.  It shares nothing with the
 * CUDA path: it has its own graph builder, its own loops and its own
 * constants, and it is written for obviousness, not speed.
 *
 * What it computes (notation of Section 2):
 *   - the graph G = (U, V, E, A, E_A) with d(u) = sum_v w(u,v),
 *     d(v) = sum_u w(u,v), W_row(u) = sum_a w(u,a), W_col(a) = sum_u w(u,a)
 *     (Section 2.1; duplicate pairs are merged by summing their weights);
 *   - x -> xP with P = (1-beta) P_S + beta P_A, P_S of Eq. 1 and P_A of
 *     Eq. 2, applied in its two-hop form (U->V->U and U->A->U) without ever
 *     forming P;
 *   - Power Iteration, Algorithm 1;
 *   - the lambda estimate of Theorem 3 (PI from the all-ones vector);
 *   - Forward Push, Algorithm 2 (FIFO order of selected nodes);
 *   - APP, Algorithm 3, and ASRP, Algorithm 4, round by round in the
 *     paper's order: the U-push over every node above its threshold
 *     (evaluated at the start of the round, ascending id), then the flush of
 *     every positive V residue, then of every positive attribute residue.
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes):
 *   - APP's r_max is eps / (|E| + |E_A|) (Section 3.3 writes |E| + |A|; only
 *     the tuple count makes the error argument of Lemma 2 go through).
 *   - ASRP's switch test (Algorithm 4) is read as
 *       n_p >= 2 (|E| + |E_A|) * max(0, log_{1/(1-alpha)}(M / eps_f)),
 *     M = max_u r(u) after the round, following the round count t of the
 *     proof of Theorem 1.  The printed form log(1 / (lambda M)) is kept as
 *     an option (switch_rule = 1).
 *   - A U node without V neighbours (or without attributes) drops the
 *     (1-beta) (or beta) share of its pushed mass; the dropped mass is
 *     reported as "leak".  Eq. 1 and Eq. 2 give such rows no entries.
 *   - APP(S) of Exp-2 (APP with ASRP's synchronous push operations) is
 *     APP's per-node thresholds r_max (|N(u)| + |A(u)|) in an asynchronous
 *     phase, after each of its rounds the switch test above with M / eps_f
 *     replaced by M' / r_max, M' = max over nodes u with |N(u)| + |A(u)| > 0
 *     of r(u) / (|N(u)| + |A(u)|) (the largest residue in units of its own
 *     threshold), then a synchronous phase pushing every positive residue;
 *     it stops on APP's own test (every residue at or below its threshold).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_OK 0
#define OG_ENOTCONVERGED 1
#define OG_EINVAL (-1)
#define OG_ENOMEM (-2)

#define OG_FP 0
#define OG_APP 1
#define OG_ASRP 2
#define OG_APPS 3     /* APP(S): APP with the synchronous switch */

typedef struct {
    uint64_t n_row, nnz;
    uint64_t *off;   /* n_row + 1 */
    uint32_t *col;   /* nnz, ascending within a row */
    double *w;       /* nnz */
} og_adj;

typedef struct {
    uint32_t n_u, n_v, n_a;
    og_adj uv, vu, ua, au;        /* U->V, V->U, U->A, A->U adjacency */
    double *d_u, *d_v;            /* weighted degrees */
    double *wrow_u, *wcol_a;      /* attribute weight sums per node / per attribute */
} og_graph;

/* ---------------------------------------------------------------- graph */

typedef struct { uint32_t c; double w; } og_pair;

static int og_pair_cmp(const void *a, const void *b) {
    uint32_t x = ((const og_pair *)a)->c, y = ((const og_pair *)b)->c;
    return (x > y) - (x < y);
}

static void og_adj_free(og_adj *a) {
    free(a->off); free(a->col); free(a->w);
    memset(a, 0, sizeof(*a));
}

/* Adjacency of (row, col, w) triples: rows bucketed, columns sorted,
 * duplicate (row, col) pairs merged by summing their weights. */
static int og_adj_build(og_adj *a, uint64_t n_row, uint64_t n, const uint32_t *row,
                        const uint32_t *col, const double *w) {
    memset(a, 0, sizeof(*a));
    a->n_row = n_row;
    uint64_t *cnt = calloc(n_row + 1, sizeof(uint64_t));
    og_pair *tmp = malloc((n ? n : 1) * sizeof(og_pair));
    if (!cnt || !tmp) { free(cnt); free(tmp); return OG_ENOMEM; }
    for (uint64_t e = 0; e < n; e++) cnt[row[e] + 1]++;
    for (uint64_t i = 0; i < n_row; i++) cnt[i + 1] += cnt[i];
    uint64_t *pos = malloc((n_row + 1) * sizeof(uint64_t));
    if (!pos) { free(cnt); free(tmp); return OG_ENOMEM; }
    memcpy(pos, cnt, (n_row + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < n; e++) {
        og_pair p = { col[e], w[e] };
        tmp[pos[row[e]]++] = p;
    }
    free(pos);
    /* sort each row, merge duplicates, count the merged size */
    uint64_t out = 0;
    a->off = malloc((n_row + 1) * sizeof(uint64_t));
    if (!a->off) { free(cnt); free(tmp); return OG_ENOMEM; }
    for (uint64_t i = 0; i < n_row; i++) {
        uint64_t b = cnt[i], e = cnt[i + 1];
        qsort(tmp + b, e - b, sizeof(og_pair), og_pair_cmp);
        a->off[i] = out;
        for (uint64_t k = b; k < e; k++) {
            if (out > a->off[i] && tmp[out - 1].c == tmp[k].c) tmp[out - 1].w += tmp[k].w;
            else tmp[out++] = tmp[k];
        }
    }
    a->off[n_row] = out;
    a->nnz = out;
    a->col = malloc((out ? out : 1) * sizeof(uint32_t));
    a->w = malloc((out ? out : 1) * sizeof(double));
    if (!a->col || !a->w) { free(cnt); free(tmp); og_adj_free(a); return OG_ENOMEM; }
    for (uint64_t k = 0; k < out; k++) { a->col[k] = tmp[k].c; a->w[k] = tmp[k].w; }
    free(cnt); free(tmp);
    return OG_OK;
}

/* Transpose of an adjacency (same weights). */
static int og_adj_transpose(og_adj *t, const og_adj *a, uint64_t n_col) {
    uint64_t n = a->nnz;
    uint32_t *r = malloc((n ? n : 1) * sizeof(uint32_t));
    if (!r) return OG_ENOMEM;
    for (uint64_t i = 0; i < a->n_row; i++)
        for (uint64_t k = a->off[i]; k < a->off[i + 1]; k++) r[k] = (uint32_t)i;
    int rc = og_adj_build(t, n_col, n, a->col, r, a->w);
    free(r);
    return rc;
}

void og_free(og_graph *g) {
    if (!g) return;
    og_adj_free(&g->uv); og_adj_free(&g->vu); og_adj_free(&g->ua); og_adj_free(&g->au);
    free(g->d_u); free(g->d_v); free(g->wrow_u); free(g->wcol_a);
    free(g);
}

/* Build the oracle's graph from COO arrays; returns NULL on invalid input. */
og_graph *og_build(uint32_t n_u, uint32_t n_v, uint32_t n_a,
                   uint64_t n_e, const uint32_t *e_u, const uint32_t *e_v, const double *e_w,
                   uint64_t n_ea, const uint32_t *ea_u, const uint32_t *ea_a, const double *ea_w) {
    for (uint64_t e = 0; e < n_e; e++)
        if (e_u[e] >= n_u || e_v[e] >= n_v || !(e_w[e] > 0.0)) return NULL;
    for (uint64_t e = 0; e < n_ea; e++)
        if (ea_u[e] >= n_u || ea_a[e] >= n_a || !(ea_w[e] > 0.0)) return NULL;
    og_graph *g = calloc(1, sizeof(og_graph));
    if (!g) return NULL;
    g->n_u = n_u; g->n_v = n_v; g->n_a = n_a;
    if (og_adj_build(&g->uv, n_u, n_e, e_u, e_v, e_w) ||
        og_adj_transpose(&g->vu, &g->uv, n_v) ||
        og_adj_build(&g->ua, n_u, n_ea, ea_u, ea_a, ea_w) ||
        og_adj_transpose(&g->au, &g->ua, n_a)) { og_free(g); return NULL; }
    g->d_u = calloc(n_u ? n_u : 1, sizeof(double));
    g->d_v = calloc(n_v ? n_v : 1, sizeof(double));
    g->wrow_u = calloc(n_u ? n_u : 1, sizeof(double));
    g->wcol_a = calloc(n_a ? n_a : 1, sizeof(double));
    if (!g->d_u || !g->d_v || !g->wrow_u || !g->wcol_a) { og_free(g); return NULL; }
    for (uint32_t u = 0; u < n_u; u++) {
        for (uint64_t k = g->uv.off[u]; k < g->uv.off[u + 1]; k++) {
            g->d_u[u] += g->uv.w[k];
            g->d_v[g->uv.col[k]] += g->uv.w[k];
        }
        for (uint64_t k = g->ua.off[u]; k < g->ua.off[u + 1]; k++) {
            g->wrow_u[u] += g->ua.w[k];
            g->wcol_a[g->ua.col[k]] += g->ua.w[k];
        }
    }
    return g;
}

uint64_t og_num_edges(const og_graph *g) { return g->uv.nnz; }
uint64_t og_num_attr_edges(const og_graph *g) { return g->ua.nnz; }

/* Copy out the merged structure (for tests): degrees, counts, sums. */
void og_node_stats(const og_graph *g, double *d_u, double *d_v, double *wrow_u, double *wcol_a,
                   uint32_t *cnt_u /* |N(u)| + |A(u)| */) {
    for (uint32_t u = 0; u < g->n_u; u++) {
        if (d_u) d_u[u] = g->d_u[u];
        if (wrow_u) wrow_u[u] = g->wrow_u[u];
        if (cnt_u) cnt_u[u] = (uint32_t)((g->uv.off[u + 1] - g->uv.off[u]) +
                                         (g->ua.off[u + 1] - g->ua.off[u]));
    }
    if (d_v) for (uint32_t v = 0; v < g->n_v; v++) d_v[v] = g->d_v[v];
    if (wcol_a) for (uint32_t a = 0; a < g->n_a; a++) wcol_a[a] = g->wcol_a[a];
}

/* y = x P (row vector times P), P = (1-beta) P_S + beta P_A, via the hops of
 * Eq. 1 (U->V->U) and Eq. 2 (U->A->U).  tv, ta are scratch of |V|, |A|. */
static void og_apply_P(const og_graph *g, double beta, const double *x, double *y,
                       double *tv, double *ta) {
    memset(tv, 0, g->n_v * sizeof(double));
    memset(ta, 0, g->n_a * sizeof(double));
    memset(y, 0, g->n_u * sizeof(double));
    for (uint32_t u = 0; u < g->n_u; u++) {
        if (x[u] == 0.0) continue;
        for (uint64_t k = g->uv.off[u]; k < g->uv.off[u + 1]; k++)
            tv[g->uv.col[k]] += (1.0 - beta) * x[u] * g->uv.w[k] / g->d_u[u];
        for (uint64_t k = g->ua.off[u]; k < g->ua.off[u + 1]; k++)
            ta[g->ua.col[k]] += beta * x[u] * g->ua.w[k] / g->wrow_u[u];
    }
    for (uint32_t v = 0; v < g->n_v; v++) {
        if (tv[v] == 0.0) continue;
        for (uint64_t k = g->vu.off[v]; k < g->vu.off[v + 1]; k++)
            y[g->vu.col[k]] += tv[v] * g->vu.w[k] / g->d_v[v];
    }
    for (uint32_t a = 0; a < g->n_a; a++) {
        if (ta[a] == 0.0) continue;
        for (uint64_t k = g->au.off[a]; k < g->au.off[a + 1]; k++)
            y[g->au.col[k]] += ta[a] * g->au.w[k] / g->wcol_a[a];
    }
}

/* Algorithm 1 (Power Iteration): pi <- e_q, then T times
 * pi <- (1-alpha) pi P + alpha e_q.  The error is at most (1-alpha)^T. */
int og_power_iteration(const og_graph *g, double alpha, double beta, uint32_t q,
                       uint32_t T, double *pi) {
    if (q >= g->n_u || !(alpha > 0.0 && alpha < 1.0) || !(beta >= 0.0 && beta <= 1.0))
        return OG_EINVAL;
    double *y = malloc((g->n_u ? g->n_u : 1) * sizeof(double));
    double *tv = malloc((g->n_v ? g->n_v : 1) * sizeof(double));
    double *ta = malloc((g->n_a ? g->n_a : 1) * sizeof(double));
    if (!y || !tv || !ta) { free(y); free(tv); free(ta); return OG_ENOMEM; }
    memset(pi, 0, g->n_u * sizeof(double));
    pi[q] = 1.0;
    for (uint32_t it = 0; it < T; it++) {
        og_apply_P(g, beta, pi, y, tv, ta);
        for (uint32_t u = 0; u < g->n_u; u++) pi[u] = (1.0 - alpha) * y[u];
        pi[q] += alpha;
    }
    free(y); free(tv); free(ta);
    return OG_OK;
}

/* Theorem 3: pi_T = 1 sum_{l<T} alpha (1-alpha)^l P^l (PI from the all-ones
 * vector), lambda = max_u pi_T(u) + |U| (1-alpha)^T. */
int og_lambda(const og_graph *g, double alpha, double beta, uint32_t T,
              double *lambda, double *pi_T /* nullable, |U| */) {
    if (!(alpha > 0.0 && alpha < 1.0) || !(beta >= 0.0 && beta <= 1.0)) return OG_EINVAL;
    uint32_t n = g->n_u;
    double *x = malloc((n ? n : 1) * sizeof(double));
    double *acc = calloc(n ? n : 1, sizeof(double));
    double *y = malloc((n ? n : 1) * sizeof(double));
    double *tv = malloc((g->n_v ? g->n_v : 1) * sizeof(double));
    double *ta = malloc((g->n_a ? g->n_a : 1) * sizeof(double));
    if (!x || !acc || !y || !tv || !ta) {
        free(x); free(acc); free(y); free(tv); free(ta); return OG_ENOMEM;
    }
    for (uint32_t u = 0; u < n; u++) x[u] = 1.0;
    for (uint32_t l = 0; l < T; l++) {
        for (uint32_t u = 0; u < n; u++) acc[u] += alpha * x[u];
        og_apply_P(g, beta, x, y, tv, ta);
        for (uint32_t u = 0; u < n; u++) x[u] = (1.0 - alpha) * y[u];
    }
    double m = 0.0;
    for (uint32_t u = 0; u < n; u++) if (acc[u] > m) m = acc[u];
    *lambda = m + (double)n * pow(1.0 - alpha, (double)T);
    if (pi_T) memcpy(pi_T, acc, n * sizeof(double));
    free(x); free(acc); free(y); free(tv); free(ta);
    return OG_OK;
}

/* ------------------------------------------------------------ push loops */

typedef struct {
    uint32_t rounds;          /* rounds executed (APP/ASRP) or pushes (FP) */
    uint32_t switch_round;    /* ASRP: first sync round (0 = never switched) */
    uint64_t n_p;             /* Algorithm 4's push counter at the end */
    uint64_t pushes;          /* total U-node pushes */
    double resid_sum;         /* sum_u r(u) at the end */
    double reserve_sum;       /* sum_u pi_hat(u) at the end */
    double leak;              /* mass dropped at dangling rows */
    double max_resid;         /* max_u r(u) at the end */
} og_stats;

typedef struct {              /* per-round record, arrays of length cap */
    uint32_t cap;
    uint64_t *frontier;       /* |F_U| of the round */
    uint64_t *n_p;            /* n_p after the round */
    double *max_r;            /* max_u r(u) after the round */
    double *sum_r;            /* sum_u r(u) after the round */
    double *sum_pi;           /* sum_u pi_hat(u) after the round */
    uint8_t *phase;           /* 0 async / 1 sync */
} og_trace;

/* One round of Algorithm 3 (U-push, then the V and attribute flushes).  The selected set is fixed at the
 * start of the round: node u is pushed iff r_u[u] > th_scale * th_u[u]
 * (th_u == NULL: iff r_u[u] > th_scale).  Returns |F_U|. */
static uint64_t og_round(const og_graph *g, double alpha, double beta,
                         const uint32_t *th_u, double th_scale,
                         double *r_u, double *r_v, double *r_a, double *pi,
                         uint32_t *sel, uint64_t *n_p, double *leak) {
    uint64_t nf = 0;
    for (uint32_t u = 0; u < g->n_u; u++) {
        double th = th_u ? th_scale * (double)th_u[u] : th_scale;
        if (r_u[u] > th) sel[nf++] = u;
    }
    for (uint64_t i = 0; i < nf; i++) {          /* push each selected U node */
        uint32_t u = sel[i];
        double r = r_u[u];
        pi[u] += alpha * r;
        double rho = (1.0 - alpha) * r;
        uint64_t nv = g->uv.off[u + 1] - g->uv.off[u];
        uint64_t na = g->ua.off[u + 1] - g->ua.off[u];
        for (uint64_t k = g->uv.off[u]; k < g->uv.off[u + 1]; k++)
            r_v[g->uv.col[k]] += (1.0 - beta) * g->uv.w[k] / g->d_u[u] * rho;
        for (uint64_t k = g->ua.off[u]; k < g->ua.off[u + 1]; k++)
            r_a[g->ua.col[k]] += beta * g->ua.w[k] / g->wrow_u[u] * rho;
        if (nv == 0) *leak += (1.0 - beta) * rho;
        if (na == 0) *leak += beta * rho;
        r_u[u] = 0.0;
        *n_p += nv + na;
    }
    for (uint32_t v = 0; v < g->n_v; v++) {      /* flush every V residue to U */
        if (!(r_v[v] > 0.0)) continue;
        for (uint64_t k = g->vu.off[v]; k < g->vu.off[v + 1]; k++)
            r_u[g->vu.col[k]] += g->vu.w[k] / g->d_v[v] * r_v[v];
        *n_p += g->vu.off[v + 1] - g->vu.off[v];
        r_v[v] = 0.0;
    }
    for (uint32_t a = 0; a < g->n_a; a++) {      /* flush every attribute residue to U */
        if (!(r_a[a] > 0.0)) continue;
        for (uint64_t k = g->au.off[a]; k < g->au.off[a + 1]; k++)
            r_u[g->au.col[k]] += g->au.w[k] / g->wcol_a[a] * r_a[a];
        *n_p += g->au.off[a + 1] - g->au.off[a];
        r_a[a] = 0.0;
    }
    return nf;
}

static void og_sums(const og_graph *g, const double *r_u, const double *pi,
                    double *max_r, double *sum_r, double *sum_pi) {
    double m = 0.0, s = 0.0, p = 0.0;
    for (uint32_t u = 0; u < g->n_u; u++) {
        if (r_u[u] > m) m = r_u[u];
        s += r_u[u];
        p += pi[u];
    }
    *max_r = m; *sum_r = s; *sum_pi = p;
}

/* Where a push run stands between two rounds: everything besides the
 * residues and reserves that the next round depends on. */
typedef struct {
    uint32_t round;           /* rounds run so far */
    uint32_t sync;            /* ASRP / APP(S): the synchronous phase has begun */
    uint32_t switch_round;    /* first synchronous round (0 = not switched) */
    uint32_t pad;
    uint64_t n_p;             /* Algorithm 4's push counter so far */
    uint64_t pushes;          /* U-node pushes so far */
    double leak;              /* mass dropped at dangling rows so far */
} og_push_state;

static int og_push_args_ok(const og_graph *g, int algo, double alpha, double beta, double eps,
                           double lambda) {
    return (alpha > 0.0 && alpha < 1.0) && (beta >= 0.0 && beta <= 1.0) && (eps > 0.0) &&
           (algo == OG_APP || algo == OG_ASRP || algo == OG_APPS) &&
           !(algo == OG_ASRP && !(lambda > 0.0)) && g != NULL;
}

/* Rounds of APP / ASRP / APP(S) from the state (pi, r_u, *ps) until the loop
 * test of Algorithms 3 and 4 fails (OG_OK) or ps->round reaches round_cap
 * (OG_ENOTCONVERGED).  pi and r_u are updated in place; the trace, if given,
 * records the rounds by their index. */
static int og_push_run(const og_graph *g, int algo, double alpha, double beta, double eps,
                       double lambda, int switch_rule, uint32_t round_cap, double *pi, double *r_u,
                       og_push_state *ps, og_trace *tr) {
    int app_thr = algo == OG_APP || algo == OG_APPS;    /* APP's per-node thresholds */
    uint32_t n = g->n_u;
    double *r_v = calloc(g->n_v ? g->n_v : 1, sizeof(double));
    double *r_a = calloc(g->n_a ? g->n_a : 1, sizeof(double));
    uint32_t *sel = malloc((n ? n : 1) * sizeof(uint32_t));
    uint32_t *cnt = malloc((n ? n : 1) * sizeof(uint32_t));
    if (!r_v || !r_a || !sel || !cnt) {
        free(r_v); free(r_a); free(sel); free(cnt); return OG_ENOMEM;
    }
    for (uint32_t u = 0; u < n; u++)
        cnt[u] = (uint32_t)((g->uv.off[u + 1] - g->uv.off[u]) + (g->ua.off[u + 1] - g->ua.off[u]));
    double EE = (double)(g->uv.nnz + g->ua.nnz);
    double r_max = eps / EE;                        /* APP threshold scale */
    double eps_f = (algo == OG_ASRP) ? eps / lambda : 0.0;
    double lg = log(1.0 / (1.0 - alpha));
    int rc = OG_OK;
    for (;;) {
        /* loop test of Algorithms 3 and 4: some U residue above its threshold */
        int any = 0;
        for (uint32_t u = 0; u < n && !any; u++) {
            double th = app_thr ? r_max * (double)cnt[u] : eps_f;
            if (r_u[u] > th) any = 1;
        }
        if (!any) break;
        if (ps->round >= round_cap) { rc = OG_ENOTCONVERGED; break; }
        uint64_t nf;
        if (algo == OG_APP || (algo == OG_APPS && !ps->sync))
            nf = og_round(g, alpha, beta, cnt, r_max, r_u, r_v, r_a, pi, sel, &ps->n_p, &ps->leak);
        else if (algo == OG_APPS)
            nf = og_round(g, alpha, beta, NULL, 0.0, r_u, r_v, r_a, pi, sel, &ps->n_p, &ps->leak);
        else
            nf = og_round(g, alpha, beta, NULL, ps->sync ? 0.0 : eps_f, r_u, r_v, r_a, pi, sel,
                          &ps->n_p, &ps->leak);
        ps->round++;
        ps->pushes += nf;
        double m, s, p;
        og_sums(g, r_u, pi, &m, &s, &p);
        if (tr && ps->round <= tr->cap) {
            tr->frontier[ps->round - 1] = nf;
            tr->n_p[ps->round - 1] = ps->n_p;
            tr->max_r[ps->round - 1] = m;
            tr->sum_r[ps->round - 1] = s;
            tr->sum_pi[ps->round - 1] = p;
            tr->phase[ps->round - 1] = (uint8_t)ps->sync;
        }
        if (algo == OG_ASRP && !ps->sync) {         /* ASRP's switch test */
            double budget;
            if (switch_rule == 1)
                budget = 2.0 * EE * (log(1.0 / (lambda * m)) / lg);
            else if (switch_rule == 2)
                budget = INFINITY;
            else
                budget = 2.0 * EE * fmax(0.0, log(m / eps_f) / lg);
            if ((double)ps->n_p >= budget) { ps->sync = 1; ps->switch_round = ps->round + 1; }
        }
        if (algo == OG_APPS && !ps->sync) {         /* APP(S): the same test in APP's units */
            double mrel = 0.0;
            for (uint32_t u = 0; u < n; u++)
                if (cnt[u] > 0 && r_u[u] / (double)cnt[u] > mrel) mrel = r_u[u] / (double)cnt[u];
            double budget = 2.0 * EE * fmax(0.0, log(mrel / r_max) / lg);
            if ((double)ps->n_p >= budget) { ps->sync = 1; ps->switch_round = ps->round + 1; }
        }
    }
    free(r_v); free(r_a); free(sel); free(cnt);
    return rc;
}

static void og_push_stats(const og_graph *g, const og_push_state *ps, const double *r_u,
                          const double *pi, og_stats *st) {
    memset(st, 0, sizeof(*st));
    st->rounds = ps->round;
    st->switch_round = ps->switch_round;
    st->n_p = ps->n_p;
    st->pushes = ps->pushes;
    st->leak = ps->leak;
    og_sums(g, r_u, pi, &st->max_resid, &st->resid_sum, &st->reserve_sum);
}

/*
 * APP (Algorithm 3), ASRP (Algorithm 4) or APP(S) (Exp-2) from source q.
 *   eps: error threshold; lambda: ASRP's parameter (eps_f = eps / lambda);
 *   switch_rule: 0 = corrected budget (default), 1 = printed formula,
 *                2 = never switch (asynchronous pushes with eps_f only).
 *   max_rounds: round cap (returns OG_ENOTCONVERGED when hit).
 * Outputs pi (|U|), optionally r_u_out (|U|), stats and a trace.
 */
int og_push(const og_graph *g, int algo, double alpha, double beta, uint32_t q,
            double eps, double lambda, int switch_rule, uint32_t max_rounds,
            double *pi, double *r_u_out, og_stats *st, og_trace *tr) {
    if (!og_push_args_ok(g, algo, alpha, beta, eps, lambda) || q >= g->n_u) return OG_EINVAL;
    uint32_t n = g->n_u;
    double *r_u = calloc(n ? n : 1, sizeof(double));
    if (!r_u) return OG_ENOMEM;
    memset(pi, 0, n * sizeof(double));
    r_u[q] = 1.0;                                   /* unit residue at the source */
    og_push_state ps;
    memset(&ps, 0, sizeof(ps));
    int rc = og_push_run(g, algo, alpha, beta, eps, lambda, switch_rule, max_rounds, pi, r_u, &ps, tr);
    if (rc < 0) { free(r_u); return rc; }
    og_push_stats(g, &ps, r_u, pi, st);
    if (r_u_out) memcpy(r_u_out, r_u, n * sizeof(double));
    free(r_u);
    return rc;
}

/*
 * The same rounds resumed: from the reserves pi, residues r_u and state *ps
 * a previous og_push_start / og_push_resume left (pi and r_u are updated in
 * place), at most more_rounds further rounds.  OG_OK once the loop test
 * fails, OG_ENOTCONVERGED when the rounds ran out first.  A run split into
 * resumed pieces performs exactly the rounds of one uninterrupted og_push.
 */
int og_push_start(const og_graph *g, uint32_t q, double *pi, double *r_u, og_push_state *ps) {
    if (!g || q >= g->n_u) return OG_EINVAL;
    memset(pi, 0, g->n_u * sizeof(double));
    memset(r_u, 0, g->n_u * sizeof(double));
    r_u[q] = 1.0;                                   /* unit residue at the source */
    memset(ps, 0, sizeof(*ps));
    return OG_OK;
}

int og_push_resume(const og_graph *g, int algo, double alpha, double beta, double eps,
                   double lambda, int switch_rule, uint32_t more_rounds, double *pi, double *r_u,
                   og_push_state *ps, og_stats *st) {
    if (!og_push_args_ok(g, algo, alpha, beta, eps, lambda) || !ps) return OG_EINVAL;
    uint32_t cap = ps->round + more_rounds < ps->round ? UINT32_MAX : ps->round + more_rounds;
    int rc = og_push_run(g, algo, alpha, beta, eps, lambda, switch_rule, cap, pi, r_u, ps, NULL);
    if (rc < 0) return rc;
    if (st) og_push_stats(g, ps, r_u, pi, st);
    return rc;
}

/*
 * Forward Push, Algorithm 2: a node whose residue exceeds
 * r_max (|N(u)| + |A(u)|) pushes straight to its two-hop U neighbours
 * (through V with share 1-beta, through A with share beta).  Selected nodes
 * are processed in FIFO order; r_max = eps / (|E| + |E_A|).
 */
int og_forward_push(const og_graph *g, double alpha, double beta, uint32_t q, double eps,
                    uint64_t max_pushes, double *pi, double *r_u_out, og_stats *st) {
    if (q >= g->n_u || !(alpha > 0.0 && alpha < 1.0) || !(beta >= 0.0 && beta <= 1.0) ||
        !(eps > 0.0))
        return OG_EINVAL;
    uint32_t n = g->n_u;
    double *r = calloc(n ? n : 1, sizeof(double));
    uint32_t *queue = malloc(((uint64_t)n + 1) * sizeof(uint32_t));
    uint8_t *inq = calloc(n ? n : 1, 1);
    uint32_t *cnt = malloc((n ? n : 1) * sizeof(uint32_t));
    if (!r || !queue || !inq || !cnt) { free(r); free(queue); free(inq); free(cnt); return OG_ENOMEM; }
    memset(pi, 0, n * sizeof(double));
    memset(st, 0, sizeof(*st));
    for (uint32_t u = 0; u < n; u++)
        cnt[u] = (uint32_t)((g->uv.off[u + 1] - g->uv.off[u]) + (g->ua.off[u + 1] - g->ua.off[u]));
    double r_max = eps / (double)(g->uv.nnz + g->ua.nnz);
    uint64_t head = 0, tail = 0, cap = (uint64_t)n + 1;
    r[q] = 1.0;
    if (r[q] > r_max * cnt[q]) { queue[tail++ % cap] = q; inq[q] = 1; }
    int rc = OG_OK;
    double leak = 0.0;
    while (head != tail) {
        uint32_t u = queue[head++ % cap];
        inq[u] = 0;
        if (!(r[u] > r_max * cnt[u])) continue;
        if (st->pushes >= max_pushes) { rc = OG_ENOTCONVERGED; break; }
        st->pushes++;
        double ru = r[u];
        pi[u] += alpha * ru;                         /* reserve */
        double rho = (1.0 - alpha) * ru;            /* mass to spread */
        r[u] = 0.0;                                  /* residue consumed */
        if (g->uv.off[u + 1] == g->uv.off[u]) leak += (1.0 - beta) * rho;
        if (g->ua.off[u + 1] == g->ua.off[u]) leak += beta * rho;
        for (uint64_t k = g->uv.off[u]; k < g->uv.off[u + 1]; k++) {   /* via V: (1-beta) share */
            uint32_t v = g->uv.col[k];
            double c = (1.0 - beta) * g->uv.w[k] / g->d_u[u] / g->d_v[v] * rho;
            for (uint64_t j = g->vu.off[v]; j < g->vu.off[v + 1]; j++) {
                uint32_t x = g->vu.col[j];
                r[x] += c * g->vu.w[j];
                if (!inq[x] && r[x] > r_max * cnt[x]) { queue[tail++ % cap] = x; inq[x] = 1; }
            }
        }
        for (uint64_t k = g->ua.off[u]; k < g->ua.off[u + 1]; k++) {   /* via A: beta share */
            uint32_t a = g->ua.col[k];
            double c = beta * g->ua.w[k] / g->wrow_u[u] / g->wcol_a[a] * rho;
            for (uint64_t j = g->au.off[a]; j < g->au.off[a + 1]; j++) {
                uint32_t x = g->au.col[j];
                r[x] += c * g->au.w[j];
                if (!inq[x] && r[x] > r_max * cnt[x]) { queue[tail++ % cap] = x; inq[x] = 1; }
            }
        }
    }
    st->leak = leak;
    double m = 0.0, s = 0.0, p = 0.0;
    for (uint32_t u = 0; u < n; u++) { if (r[u] > m) m = r[u]; s += r[u]; p += pi[u]; }
    st->max_resid = m; st->resid_sum = s; st->reserve_sum = p;
    if (r_u_out) memcpy(r_u_out, r, n * sizeof(double));
    free(r); free(queue); free(inq); free(cnt);
    return rc;
}

/* Top-k of a score vector: k largest scores, score descending, then node id
 * ascending.  Selection by repeated scans (k passes): slow and obvious. */
int og_topk(const double *score, uint32_t n, uint32_t k, uint32_t *nodes, double *vals) {
    if (k > n) k = n;
    uint8_t *taken = calloc(n ? n : 1, 1);
    if (!taken) return OG_ENOMEM;
    for (uint32_t i = 0; i < k; i++) {
        int64_t best = -1;
        for (uint32_t u = 0; u < n; u++) {
            if (taken[u]) continue;
            if (best < 0 || score[u] > score[best]) best = u;
        }
        taken[best] = 1;
        nodes[i] = (uint32_t)best;
        vals[i] = score[best];
    }
    free(taken);
    return (int)k;
}
