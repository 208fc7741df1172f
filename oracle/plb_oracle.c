/*
 * CPU ORACLE for canonical 2-hop distance labeling -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  The GPU library shares no code with it.
 *
 * Plain, sequential, obviously-correct restatements of the paper
 * ("Pruned Landmark Labeling Meets Vertex Centric Computation", Jin et al.):
 *
 *   oracle_pll      Alg. 1 (PLL, Sec. 2.1.1): one pruned BFS per root in rank
 *                   order, with the "small revision" (a root is only pushed to
 *                   neighbours it outranks).  The pruning test uses an array
 *                   map of L(u) (Sec. 3.3, cost discussion).
 *   oracle_vcpll    Alg. 3 (VC-PLL, Sec. 3.1): all vertices spread at once,
 *                   one scatter/gather round per distance; unique messages;
 *                   distance check against the labels of the previous round.
 *   oracle_chhl_row Def. 2 (canonical hierarchical hub labeling) for one
 *                   vertex: h is a hub of v iff h has the highest rank in
 *                   P_hv, the set of vertices on all shortest h-v paths.
 *                   One BFS from v; m(x) = best rank over P_vx is carried
 *                   along the BFS DAG.
 *   oracle_query    2-hop query (Sec. 2.1): min over common hubs of
 *                   d(u,h) + d(h,v), by a merge of two hub-sorted lists;
 *                   -1 when no hub is common (different components).
 *   oracle_bfs      textbook BFS distances (-1 unreachable).
 *   oracle_pll_directed
 *                   the directed form (Sec. 5.1): per root u in rank order,
 *                   a forward pruned BFS over out-arcs fills L_in (hub u,
 *                   d(u->v)) and a backward one over in-arcs fills L_out
 *                   (hub u, d(v->u)); a candidate is pruned by a hub w with
 *                   d(u->w) + d(w->v) (resp. d(v->w) + d(w->u)) <= its
 *                   distance, read from L_out(u) and L_in(v) (resp. L_out(v)
 *                   and L_in(u)).  Def. 2 for directed graphs is
 *                   oracle_chhl_row over the in-arcs (L_in) or the out-arcs
 *                   (L_out); the directed query is oracle_query2.
 *   oracle_pll_weighted
 *                   weighted graphs (Sec. 5.1, Sec. 6.4): Alg. 1 with each
 *                   pruned BFS replaced by a pruned Dijkstra search (uint8
 *                   arc weights >= 1, symmetric).
 *   oracle_chhl_row_weighted, oracle_chhl_weighted
 *                   Def. 2 for weighted graphs: one Dijkstra from v, best
 *                   rank carried along the shortest-path DAG in settle order.
 *   oracle_dijkstra textbook Dijkstra distances (-1 unreachable).
 *
 * Conventions: vertices are original ids 0..n-1; the order is given as
 * order[r] = id of rank r (rank 0 = highest); label entries store the hub as
 * its RANK (uint32) and the distance (uint8); each label row is sorted by hub
 * rank ascending.  Readings where the paper is silent: unreachable -> -1;
 * a tie in the distance check prunes (the paper's test is strict "<").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef struct {
    uint32_t* hub;
    uint8_t* dist;
    int64_t len, cap;
} row_t;

typedef struct {
    int64_t n;
    row_t* rows;
    int64_t total;
    int32_t max_dist;
    int32_t rounds;          /* VC-PLL only */
    int64_t stats[4 * 256];  /* VC-PLL per round: messages, unique, accepted, checks */
    int64_t* cost;           /* per vertex: positive distance-check cost (Sec. 4.3), PLL and VC-PLL */
    int64_t checks;          /* PLL: vertices reached (popped) over all searches; BVC-PLL: messages sent */
} labels_t;

static int row_push(row_t* r, uint32_t h, uint8_t d) {
    if (r->len == r->cap) {
        int64_t nc = r->cap ? 2 * r->cap : 4;
        uint32_t* nh = (uint32_t*)realloc(r->hub, sizeof(uint32_t) * (size_t)nc);
        if (!nh) return -1;
        r->hub = nh;
        uint8_t* nd = (uint8_t*)realloc(r->dist, (size_t)nc);
        if (!nd) return -1;
        r->dist = nd;
        r->cap = nc;
    }
    r->hub[r->len] = h;
    r->dist[r->len] = d;
    r->len++;
    return 0;
}

static labels_t* labels_new(int64_t n) {
    labels_t* L = (labels_t*)calloc(1, sizeof(labels_t));
    L->n = n;
    L->rows = (row_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(row_t));
    L->cost = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    return L;
}

void oracle_labels_free(void* h) {
    labels_t* L = (labels_t*)h;
    if (!L) return;
    for (int64_t v = 0; v < L->n; ++v) {
        free(L->rows[v].hub);
        free(L->rows[v].dist);
    }
    free(L->rows);
    free(L->cost);
    free(L);
}

int64_t oracle_labels_total(void* h) { return ((labels_t*)h)->total; }
int64_t oracle_labels_checks(void* h) { return ((labels_t*)h)->checks; }
int32_t oracle_labels_max_dist(void* h) { return ((labels_t*)h)->max_dist; }
int32_t oracle_labels_rounds(void* h) { return ((labels_t*)h)->rounds; }
const int64_t* oracle_labels_stats(void* h) { return ((labels_t*)h)->stats; }

/* Positive distance-check cost per vertex (Sec. 4.3, the positive-check
 * theorem): over the labels (u, d) accepted at v, u != v, the number of v's
 * other labels (v's own (v, 0) left out) that the check of (u, d) reads.
 * PLL (Alg. 1) reads every label accepted before (roots arrive one by one);
 * VC-PLL (Alg. 3) reads the labels of the earlier rounds only. */
void oracle_labels_cost(void* h, int64_t* out) {
    labels_t* L = (labels_t*)h;
    memcpy(out, L->cost, sizeof(int64_t) * (size_t)L->n);
}

/* CSR export: off[n+1], hub[total], dist[total], rows by original id. */
void oracle_labels_export(void* h, int64_t* off, uint32_t* hub, uint8_t* dist) {
    labels_t* L = (labels_t*)h;
    int64_t k = 0;
    off[0] = 0;
    for (int64_t v = 0; v < L->n; ++v) {
        const row_t* r = &L->rows[v];
        if (r->len) {
            memcpy(hub + k, r->hub, sizeof(uint32_t) * (size_t)r->len);
            memcpy(dist + k, r->dist, (size_t)r->len);
        }
        k += r->len;
        off[v + 1] = k;
    }
}

static void finish_totals(labels_t* L) {
    L->total = 0;
    L->max_dist = 0;
    for (int64_t v = 0; v < L->n; ++v) {
        L->total += L->rows[v].len;
        for (int64_t i = 0; i < L->rows[v].len; ++i)
            if (L->rows[v].dist[i] > L->max_dist) L->max_dist = L->rows[v].dist[i];
    }
}

#define INF_D 0x7fffffff

/* ----------------------------------------------------------------- Alg. 1 */
static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Returns NULL on allocation failure or when a label distance exceeds 254.
 * With budget_s > 0 the roots loop stops after the first root that ends past
 * the budget (a bounded sample for timing); *roots_done receives the number
 * of roots processed. */
static void* pll_impl(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order,
                      double budget_s, int64_t* roots_done) {
    const double t_start = now_s();
    labels_t* L = labels_new(n);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));  /* hub rank -> d(u,hub) */
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));  /* BFS distance, -1 unvisited */
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int fail = 0;
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t i = 0; i < n; ++i) {
        T[i] = INF_D;
        D[i] = -1;
    }
    int64_t r = 0;
    for (r = 0; r < n && !fail; ++r) {                   /* roots from high to low rank */
        if (budget_s > 0 && r > 0 && now_s() - t_start > budget_s) break;
        const int32_t u = order[r];
        const row_t* Lu = &L->rows[u];
        const int64_t lu_len = Lu->len;                  /* L(u) before this root */
        for (int64_t i = 0; i < lu_len; ++i) T[Lu->hub[i]] = Lu->dist[i];
        int64_t head = 0, tail = 0;
        Q[tail++] = u;
        D[u] = 0;
        while (head < tail) {
            const int32_t v = Q[head++];
            const int32_t delta = D[v];
            ++L->checks;                                 /* one distance check per reached vertex */
            /* prune iff some common hub w gives T[w] + d(w,v) <= delta */
            int pruned = 0;
            const row_t* Lv = &L->rows[v];
            for (int64_t i = 0; i < Lv->len; ++i) {
                const int32_t tw = T[Lv->hub[i]];
                if (tw != INF_D && tw + (int32_t)Lv->dist[i] <= delta) {
                    pruned = 1;
                    break;
                }
            }
            if (pruned) continue;
            if (delta > 254) {
                fail = 1;
                break;
            }
            if (v != u) L->cost[v] += L->rows[v].len;    /* L(v) holds no (v, 0) yet: v ranks below u */
            if (row_push(&L->rows[v], (uint32_t)r, (uint8_t)delta)) {
                fail = 1;
                break;
            }
            for (int64_t j = off[v]; j < off[v + 1]; ++j) {
                const int32_t w = col[j];
                if (rank[w] > r && D[w] < 0) {           /* small revision */
                    D[w] = delta + 1;
                    Q[tail++] = w;
                }
            }
        }
        for (int64_t i = 0; i < tail; ++i) D[Q[i]] = -1;
        for (int64_t i = 0; i < lu_len; ++i) T[L->rows[u].hub[i]] = INF_D;
    }
    free(rank);
    free(T);
    free(D);
    free(Q);
    if (roots_done) *roots_done = r;
    if (fail) {
        oracle_labels_free(L);
        return NULL;
    }
    finish_totals(L);
    return L;
}

void* oracle_pll(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order) {
    return pll_impl(n, off, col, order, 0.0, NULL);
}

/* Alg. 1 stopped after budget_s seconds (between roots); labels so far. */
void* oracle_pll_budget(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order,
                        double budget_s, int64_t* roots_done) {
    return pll_impl(n, off, col, order, budget_s, roots_done);
}

/* ------------------------------------------------------- directed Alg. 1 */
/* One pruned BFS from root u (rank r) over the arcs (off, col): v at distance
 * delta is pruned when a hub w has Tu[w] + d(w, v) <= delta with d(w, v)
 * read from Lcheck(v); else (r, delta) goes to Ladd(v).  Tu holds the root's
 * side of the test (d(u->w) or d(w->u)). */
static int directed_bfs(const int64_t* off, const int32_t* col, const int32_t* rank, int32_t u, int64_t r,
                        const int32_t* Tu, labels_t* Lcheck, labels_t* Ladd, int32_t* D, int32_t* Q) {
    int64_t head = 0, tail = 0;
    int fail = 0;
    Q[tail++] = u;
    D[u] = 0;
    while (head < tail && !fail) {
        const int32_t v = Q[head++];
        const int32_t delta = D[v];
        int pruned = 0;
        const row_t* Lv = &Lcheck->rows[v];
        for (int64_t i = 0; i < Lv->len; ++i) {
            const int32_t tw = Tu[Lv->hub[i]];
            if (tw != INF_D && tw + (int32_t)Lv->dist[i] <= delta) {
                pruned = 1;
                break;
            }
        }
        if (pruned) continue;
        if (delta > 254 || row_push(&Ladd->rows[v], (uint32_t)r, (uint8_t)delta)) {
            fail = 1;
            break;
        }
        for (int64_t j = off[v]; j < off[v + 1]; ++j) {
            const int32_t w = col[j];
            if (rank[w] > r && D[w] < 0) {               /* small revision */
                D[w] = delta + 1;
                Q[tail++] = w;
            }
        }
    }
    for (int64_t i = 0; i < tail; ++i) D[Q[i]] = -1;
    return fail;
}

/* Directed PLL; returns the L_in set and writes the L_out set to *out_lout
 * (both NULL on failure: allocation or a distance above 254). */
void* oracle_pll_directed(int64_t n, const int64_t* off_out, const int32_t* col_out, const int64_t* off_in,
                          const int32_t* col_in, const int32_t* order, void** out_lout) {
    labels_t* Lin = labels_new(n);
    labels_t* Lout = labels_new(n);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* Tout = (int32_t*)malloc(sizeof(int32_t) * nn);  /* hub rank -> d(u->hub) */
    int32_t* Tin = (int32_t*)malloc(sizeof(int32_t) * nn);   /* hub rank -> d(hub->u) */
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * nn);
    int fail = 0;
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t i = 0; i < n; ++i) {
        Tout[i] = Tin[i] = INF_D;
        D[i] = -1;
    }
    for (int64_t r = 0; r < n && !fail; ++r) {
        const int32_t u = order[r];
        const row_t* Lo = &Lout->rows[u];
        const row_t* Li = &Lin->rows[u];
        const int64_t lo_len = Lo->len, li_len = Li->len;
        for (int64_t i = 0; i < lo_len; ++i) Tout[Lo->hub[i]] = Lo->dist[i];
        for (int64_t i = 0; i < li_len; ++i) Tin[Li->hub[i]] = Li->dist[i];
        /* forward: d(u->w) from L_out(u), d(w->v) from L_in(v); adds to L_in */
        fail = directed_bfs(off_out, col_out, rank, u, r, Tout, Lin, Lin, D, Q);
        /* backward: d(w->u) from L_in(u), d(v->w) from L_out(v); adds to L_out */
        if (!fail) fail = directed_bfs(off_in, col_in, rank, u, r, Tin, Lout, Lout, D, Q);
        for (int64_t i = 0; i < lo_len; ++i) Tout[Lout->rows[u].hub[i]] = INF_D;
        for (int64_t i = 0; i < li_len; ++i) Tin[Lin->rows[u].hub[i]] = INF_D;
    }
    free(rank); free(Tout); free(Tin); free(D); free(Q);
    if (fail) {
        oracle_labels_free(Lin);
        oracle_labels_free(Lout);
        *out_lout = NULL;
        return NULL;
    }
    finish_totals(Lin);
    finish_totals(Lout);
    *out_lout = Lout;
    return Lin;
}

/* ----------------------------------------------------------------- Alg. 3 */
/* Round d: each v gathers (u, d) from every neighbour a with u in dL(a),
 * rank(u) < rank(v) and u not in L(v); unique messages are checked against
 * the labels as they stood after round d-1; the accepted ones form dL(v) and
 * are added to L(v) after all vertices have been gathered. */
void* oracle_vcpll(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order) {
    labels_t* L = labels_new(n);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    row_t* dL = (row_t*)calloc(nn, sizeof(row_t));      /* new labels of the previous round (hub ranks) */
    row_t* ndL = (row_t*)calloc(nn, sizeof(row_t));     /* new labels of this round */
    int32_t* Tv = (int32_t*)malloc(sizeof(int32_t) * nn);  /* hub rank -> d(v,hub), L(v) as an array */
    int32_t* seen = (int32_t*)malloc(sizeof(int32_t) * nn); /* message dedup stamp per hub rank */
    int32_t* msgs = (int32_t*)malloc(sizeof(int32_t) * nn);
    int fail = 0;
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t i = 0; i < n; ++i) {
        Tv[i] = INF_D;
        seen[i] = -1;
    }
    /* Init: dL(v) = L(v) = {(v, 0)} */
    for (int64_t v = 0; v < n; ++v) {
        row_push(&L->rows[v], (uint32_t)rank[v], 0);
        row_push(&dL[v], (uint32_t)rank[v], 0);
    }
    int32_t d = 0;
    int64_t active = n;
    while (active > 0 && !fail) {
        ++d;
        int64_t st_msgs = 0, st_unique = 0, st_acc = 0, st_checks = 0;
        active = 0;
        for (int64_t v = 0; v < n; ++v) {                 /* gather at v */
            const row_t* Lv = &L->rows[v];
            for (int64_t i = 0; i < Lv->len; ++i) Tv[Lv->hub[i]] = Lv->dist[i];
            int64_t nm = 0;
            for (int64_t j = off[v]; j < off[v + 1]; ++j) {
                const row_t* da = &dL[col[j]];
                for (int64_t i = 0; i < da->len; ++i) {
                    const uint32_t u = da->hub[i];       /* rank of u */
                    if ((int64_t)u < (int64_t)rank[v] && Tv[u] == INF_D) {
                        ++st_msgs;
                        if (seen[u] != (int32_t)v) {
                            seen[u] = (int32_t)v;
                            msgs[nm++] = (int32_t)u;
                        }
                    }
                }
            }
            st_unique += nm;
            ndL[v].len = 0;
            for (int64_t k = 0; k < nm; ++k) {
                const uint32_t u = (uint32_t)msgs[k];
                const row_t* Lu = &L->rows[order[u]];
                int pruned = 0;
                for (int64_t i = 0; i < Lu->len; ++i) {
                    ++st_checks;
                    const int32_t tv = Tv[Lu->hub[i]];
                    if (tv != INF_D && tv + (int32_t)Lu->dist[i] <= d) {
                        pruned = 1;
                        break;
                    }
                }
                if (!pruned) {
                    row_push(&ndL[v], u, (uint8_t)(d > 255 ? 255 : d));
                    L->cost[v] += Lv->len - 1;                /* the labels of rounds < d, (v, 0) left out */
                }
            }
            for (int64_t i = 0; i < Lv->len; ++i) Tv[Lv->hub[i]] = INF_D;
            for (int64_t k = 0; k < nm; ++k) seen[msgs[k]] = -1;
        }
        for (int64_t v = 0; v < n; ++v) {                 /* L(v) <- L(v) U dL(v) */
            row_t* nv = &ndL[v];
            if (nv->len == 0) {
                dL[v].len = 0;
                continue;
            }
            if (d > 254) {
                fail = 1;
                break;
            }
            ++active;
            st_acc += nv->len;
            /* keep rows sorted by hub rank: insertion merge */
            row_t* Lv = &L->rows[v];
            for (int64_t k = 0; k < nv->len; ++k) {
                if (row_push(Lv, nv->hub[k], (uint8_t)d)) fail = 1;
                int64_t p = Lv->len - 1;
                while (p > 0 && Lv->hub[p - 1] > Lv->hub[p]) {
                    uint32_t th = Lv->hub[p]; Lv->hub[p] = Lv->hub[p - 1]; Lv->hub[p - 1] = th;
                    uint8_t td = Lv->dist[p]; Lv->dist[p] = Lv->dist[p - 1]; Lv->dist[p - 1] = td;
                    --p;
                }
            }
            row_t t = dL[v];
            dL[v] = *nv;
            *nv = t;
            nv->len = 0;
        }
        if (d < 256) {
            L->stats[4 * d + 0] = st_msgs;
            L->stats[4 * d + 1] = st_unique;
            L->stats[4 * d + 2] = st_acc;
            L->stats[4 * d + 3] = st_checks;
        }
    }
    L->rounds = d;
    for (int64_t v = 0; v < n; ++v) {
        free(dL[v].hub); free(dL[v].dist);
        free(ndL[v].hub); free(ndL[v].dist);
    }
    free(dL); free(ndL); free(rank); free(Tv); free(seen); free(msgs);
    if (fail) {
        oracle_labels_free(L);
        return NULL;
    }
    finish_totals(L);
    return L;
}

/* ----------------------------------------------------------------- Def. 2 */
/* Canonical label of ONE vertex v: BFS from v; best[x] = smallest rank over
 * all vertices on all shortest v-x paths (both ends included).  x is a hub of
 * v iff best[x] == rank(x).  Writes (hub rank, distance) sorted by rank and
 * returns the count (at most cap; -1 if cap is too small).  Scratch: dist and
 * best must hold n entries and start as -1 / anything; dist is restored. */
static int64_t chhl_row_impl(int64_t n, const int64_t* off, const int32_t* col, const int32_t* rank,
                             int32_t v, int32_t* dist, int32_t* best, int32_t* Q,
                             uint32_t* out_hub, uint8_t* out_dist, int64_t cap) {
    (void)n;
    int64_t head = 0, tail = 0;
    Q[tail++] = v;
    dist[v] = 0;
    best[v] = rank[v];
    while (head < tail) {
        const int32_t p = Q[head++];
        for (int64_t j = off[p]; j < off[p + 1]; ++j) {
            const int32_t x = col[j];
            if (dist[x] < 0) {
                dist[x] = dist[p] + 1;
                best[x] = rank[x] < best[p] ? rank[x] : best[p];
                Q[tail++] = x;
            } else if (dist[x] == dist[p] + 1 && best[p] < best[x]) {
                best[x] = best[p];                       /* another shortest path into x */
            }
        }
    }
    int64_t k = 0;
    for (int64_t i = 0; i < tail; ++i) {
        const int32_t x = Q[i];
        if (best[x] == rank[x]) {
            if (k < cap) {
                out_hub[k] = (uint32_t)rank[x];
                out_dist[k] = (uint8_t)(dist[x] > 255 ? 255 : dist[x]);
            }
            ++k;
        }
    }
    for (int64_t i = 0; i < tail; ++i) dist[Q[i]] = -1;
    if (k > cap) return -1;
    /* sort by hub rank (insertion sort; rows are short) */
    for (int64_t i = 1; i < k; ++i) {
        uint32_t h = out_hub[i];
        uint8_t dd = out_dist[i];
        int64_t p = i;
        while (p > 0 && out_hub[p - 1] > h) {
            out_hub[p] = out_hub[p - 1];
            out_dist[p] = out_dist[p - 1];
            --p;
        }
        out_hub[p] = h;
        out_dist[p] = dd;
    }
    return k;
}

int64_t oracle_chhl_row(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order,
                        int32_t v, uint32_t* out_hub, uint8_t* out_dist, int64_t cap) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * nn);
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    int64_t k = chhl_row_impl(n, off, col, rank, v, dist, best, Q, out_hub, out_dist, cap);
    free(rank); free(dist); free(best); free(Q);
    return k;
}

/* Def. 2 for every vertex (n BFS runs; small graphs only). */
void* oracle_chhl(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order) {
    labels_t* L = labels_new(n);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * nn);
    uint32_t* hh = (uint32_t*)malloc(sizeof(uint32_t) * nn);
    uint8_t* dd = (uint8_t*)malloc(nn);
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    for (int64_t v = 0; v < n; ++v) {
        int64_t k = chhl_row_impl(n, off, col, rank, (int32_t)v, dist, best, Q, hh, dd, n);
        for (int64_t i = 0; i < k; ++i) row_push(&L->rows[v], hh[i], dd[i]);
    }
    free(rank); free(dist); free(best); free(Q); free(hh); free(dd);
    finish_totals(L);
    return L;
}

/* ------------------------------------------------------------ 2-hop query */
/* labels as CSR (off, hub sorted per row, dist); pairs[2q]; out[q]. */
void oracle_query(int64_t q, const int64_t* off, const uint32_t* hub, const uint8_t* dist,
                  const int32_t* pairs, int32_t* out) {
    for (int64_t k = 0; k < q; ++k) {
        const int32_t s = pairs[2 * k], t = pairs[2 * k + 1];
        int64_t i = off[s], ie = off[s + 1], j = off[t], je = off[t + 1];
        int32_t best = -1;
        while (i < ie && j < je) {
            if (hub[i] < hub[j]) {
                ++i;
            } else if (hub[i] > hub[j]) {
                ++j;
            } else {
                const int32_t c = (int32_t)dist[i] + (int32_t)dist[j];
                if (best < 0 || c < best) best = c;
                ++i;
                ++j;
            }
        }
        out[k] = best;
    }
}

/* Directed 2-hop query: d(s->t) = min over hubs w of L_out(s) and L_in(t) of
 * d(s->w) + d(w->t); -1 when none is common. */
void oracle_query2(int64_t q, const int64_t* off_s, const uint32_t* hub_s, const uint8_t* dist_s,
                   const int64_t* off_t, const uint32_t* hub_t, const uint8_t* dist_t, const int32_t* pairs,
                   int32_t* out) {
    for (int64_t k = 0; k < q; ++k) {
        const int32_t s = pairs[2 * k], t = pairs[2 * k + 1];
        int64_t i = off_s[s], ie = off_s[s + 1], j = off_t[t], je = off_t[t + 1];
        int32_t best = -1;
        while (i < ie && j < je) {
            if (hub_s[i] < hub_t[j]) {
                ++i;
            } else if (hub_s[i] > hub_t[j]) {
                ++j;
            } else {
                const int32_t c = (int32_t)dist_s[i] + (int32_t)dist_t[j];
                if (best < 0 || c < best) best = c;
                ++i;
                ++j;
            }
        }
        out[k] = best;
    }
}

/* -------------------------------------------------------------------- BFS */
void oracle_bfs(int64_t n, const int64_t* off, const int32_t* col, int32_t src, int32_t* dist) {
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    int64_t head = 0, tail = 0;
    Q[tail++] = src;
    dist[src] = 0;
    while (head < tail) {
        const int32_t p = Q[head++];
        for (int64_t j = off[p]; j < off[p + 1]; ++j)
            if (dist[col[j]] < 0) {
                dist[col[j]] = dist[p] + 1;
                Q[tail++] = col[j];
            }
    }
    free(Q);
}

/* ============================================================ weighted graphs
 * Sec. 5.1 (weighted graphs) and Sec. 6.4: the sequential baseline there is
 * PLL with its BFS replaced by Dijkstra's algorithm.  Arc weights are uint8,
 * per arc (wt[j] belongs to col[j]), positive, the same in both directions. */

/* Binary min-heap of keys dist << 32 | vertex (lazy deletion: an entry whose
 * distance is above the vertex's current tentative distance is skipped). */
typedef struct {
    int64_t* key;
    int64_t len;
} heap_t;

static void heap_push(heap_t* h, int64_t k) {
    int64_t i = h->len++;
    while (i > 0) {
        const int64_t p = (i - 1) / 2;
        if (h->key[p] <= k) break;
        h->key[i] = h->key[p];
        i = p;
    }
    h->key[i] = k;
}

static int64_t heap_pop(heap_t* h) {
    const int64_t top = h->key[0];
    const int64_t last = h->key[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= h->len) break;
        if (c + 1 < h->len && h->key[c + 1] < h->key[c]) ++c;
        if (h->key[c] >= last) break;
        h->key[i] = h->key[c];
        i = c;
    }
    if (h->len > 0) h->key[i] = last;
    return top;
}

#define HKEY(d, v) (((int64_t)(d) << 32) | (int64_t)(uint32_t)(v))
#define HDIST(k) ((int32_t)((k) >> 32))
#define HVERT(k) ((int32_t)((k) & 0xffffffff))

/* PLL with pruned Dijkstra searches (Alg. 1 with Dijkstra in place of BFS):
 * roots in rank order; a settled vertex v at distance delta is pruned when a
 * hub w of L(v) has d(u,w) + d(w,v) <= delta (read from L(u), L(v)); else
 * (u, delta) is appended to L(v) and v relaxes its arcs to vertices u
 * outranks.  NULL on allocation failure or a distance above 254. */
static void* pll_weighted_impl(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt,
                               const int32_t* order, double budget_s, int64_t* roots_done) {
    const double t_start = now_s();
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const int64_t nnz = off[n];
    labels_t* L = labels_new(n);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * nn);   /* tentative distance, -1 untouched */
    int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * nn);
    heap_t hp = {(int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz + 2)), 0};
    int fail = 0;
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t i = 0; i < n; ++i) {
        T[i] = INF_D;
        D[i] = -1;
    }
    int64_t r = 0;
    for (r = 0; r < n && !fail; ++r) {
        if (budget_s > 0 && r > 0 && now_s() - t_start > budget_s) break;
        const int32_t u = order[r];
        const row_t* Lu = &L->rows[u];
        const int64_t lu_len = Lu->len;
        for (int64_t i = 0; i < lu_len; ++i) T[Lu->hub[i]] = Lu->dist[i];
        int64_t nt = 0;
        hp.len = 0;
        D[u] = 0;
        touched[nt++] = u;
        heap_push(&hp, HKEY(0, u));
        while (hp.len > 0) {
            const int64_t k = heap_pop(&hp);
            const int32_t v = HVERT(k), delta = HDIST(k);
            if (delta != D[v]) continue;                 /* stale entry */
            int pruned = 0;
            const row_t* Lv = &L->rows[v];
            for (int64_t i = 0; i < Lv->len; ++i) {
                const int32_t tw = T[Lv->hub[i]];
                if (tw != INF_D && tw + (int32_t)Lv->dist[i] <= delta) {
                    pruned = 1;
                    break;
                }
            }
            if (pruned) continue;
            if (delta > 254) {
                fail = 1;
                break;
            }
            if (row_push(&L->rows[v], (uint32_t)r, (uint8_t)delta)) {
                fail = 1;
                break;
            }
            for (int64_t j = off[v]; j < off[v + 1]; ++j) {
                const int32_t x = col[j];
                if (rank[x] <= r) continue;                /* small revision */
                const int32_t nd = delta + (int32_t)wt[j];
                if (D[x] < 0 || nd < D[x]) {
                    if (D[x] < 0) touched[nt++] = x;
                    D[x] = nd;
                    heap_push(&hp, HKEY(nd, x));
                }
            }
        }
        for (int64_t i = 0; i < nt; ++i) D[touched[i]] = -1;
        for (int64_t i = 0; i < lu_len; ++i) T[L->rows[u].hub[i]] = INF_D;
    }
    free(rank);
    free(T);
    free(D);
    free(touched);
    free(hp.key);
    if (roots_done) *roots_done = r;
    if (fail) {
        oracle_labels_free(L);
        return NULL;
    }
    finish_totals(L);
    return L;
}

void* oracle_pll_weighted(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt,
                          const int32_t* order) {
    return pll_weighted_impl(n, off, col, wt, order, 0.0, NULL);
}

void* oracle_pll_weighted_budget(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt,
                                 const int32_t* order, double budget_s, int64_t* roots_done) {
    return pll_weighted_impl(n, off, col, wt, order, budget_s, roots_done);
}

/* Dijkstra from src over every vertex: dist (-1 unreachable) and the settle
 * order (non-decreasing distance); returns the number settled. */
static int64_t dijkstra_impl(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt, int32_t src,
                             int32_t* dist, char* done, int32_t* settled, heap_t* hp) {
    for (int64_t i = 0; i < n; ++i) {
        dist[i] = -1;
        done[i] = 0;
    }
    int64_t ns = 0;
    hp->len = 0;
    dist[src] = 0;
    heap_push(hp, HKEY(0, src));
    while (hp->len > 0) {
        const int64_t k = heap_pop(hp);
        const int32_t v = HVERT(k), dv = HDIST(k);
        if (done[v] || dv != dist[v]) continue;
        done[v] = 1;
        settled[ns++] = v;
        for (int64_t j = off[v]; j < off[v + 1]; ++j) {
            const int32_t x = col[j];
            const int32_t nd = dv + (int32_t)wt[j];
            if (!done[x] && (dist[x] < 0 || nd < dist[x])) {
                dist[x] = nd;
                heap_push(hp, HKEY(nd, x));
            }
        }
    }
    return ns;
}

void oracle_dijkstra(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt, int32_t src,
                     int32_t* dist) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    char* done = (char*)malloc(nn);
    int32_t* settled = (int32_t*)malloc(sizeof(int32_t) * nn);
    heap_t hp = {(int64_t*)malloc(sizeof(int64_t) * (size_t)(off[n] + 2)), 0};
    dijkstra_impl(n, off, col, wt, src, dist, done, settled, &hp);
    free(done);
    free(settled);
    free(hp.key);
}

/* Def. 2 for one vertex v of a weighted graph: after Dijkstra from v, the
 * vertices are taken in settle order and best[x] = min(rank(x), best[p] over
 * the predecessors p of x on shortest paths, d(v,p) + w(p,x) = d(v,x)); with
 * positive weights every such p settles before x, so best[x] is the highest
 * rank on all shortest v-x paths and x is a hub of v iff best[x] = rank(x). */
static int64_t chhl_row_weighted_impl(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt,
                                      const int32_t* rank, int32_t v, int32_t* dist, int32_t* best, char* done,
                                      int32_t* settled, heap_t* hp, uint32_t* out_hub, uint8_t* out_dist,
                                      int64_t cap) {
    const int64_t ns = dijkstra_impl(n, off, col, wt, v, dist, done, settled, hp);
    int64_t k = 0;
    for (int64_t i = 0; i < ns; ++i) {
        const int32_t x = settled[i];
        int32_t b = rank[x];
        for (int64_t j = off[x]; j < off[x + 1]; ++j) {
            const int32_t p = col[j];
            if (dist[p] >= 0 && dist[p] + (int32_t)wt[j] == dist[x] && best[p] < b) b = best[p];
        }
        best[x] = b;
        if (b == rank[x]) {
            if (k < cap) {
                out_hub[k] = (uint32_t)rank[x];
                out_dist[k] = (uint8_t)(dist[x] > 255 ? 255 : dist[x]);
            }
            ++k;
        }
    }
    if (k > cap) return -1;
    for (int64_t i = 1; i < k; ++i) {                    /* sort by hub rank */
        uint32_t h = out_hub[i];
        uint8_t dd = out_dist[i];
        int64_t p = i;
        while (p > 0 && out_hub[p - 1] > h) {
            out_hub[p] = out_hub[p - 1];
            out_dist[p] = out_dist[p - 1];
            --p;
        }
        out_hub[p] = h;
        out_dist[p] = dd;
    }
    return k;
}

int64_t oracle_chhl_row_weighted(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt,
                                 const int32_t* order, int32_t v, uint32_t* out_hub, uint8_t* out_dist,
                                 int64_t cap) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* settled = (int32_t*)malloc(sizeof(int32_t) * nn);
    char* done = (char*)malloc(nn);
    heap_t hp = {(int64_t*)malloc(sizeof(int64_t) * (size_t)(off[n] + 2)), 0};
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    const int64_t k = chhl_row_weighted_impl(n, off, col, wt, rank, v, dist, best, done, settled, &hp, out_hub,
                                             out_dist, cap);
    free(rank); free(dist); free(best); free(settled); free(done); free(hp.key);
    return k;
}

/* Def. 2 for every vertex of a weighted graph (n Dijkstra runs). */
void* oracle_chhl_weighted(int64_t n, const int64_t* off, const int32_t* col, const uint8_t* wt,
                           const int32_t* order) {
    labels_t* L = labels_new(n);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* settled = (int32_t*)malloc(sizeof(int32_t) * nn);
    char* done = (char*)malloc(nn);
    uint32_t* hh = (uint32_t*)malloc(sizeof(uint32_t) * nn);
    uint8_t* dd = (uint8_t*)malloc(nn);
    heap_t hp = {(int64_t*)malloc(sizeof(int64_t) * (size_t)(off[n] + 2)), 0};
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t k = chhl_row_weighted_impl(n, off, col, wt, rank, (int32_t)v, dist, best, done, settled, &hp,
                                                 hh, dd, n);
        for (int64_t i = 0; i < k; ++i) row_push(&L->rows[v], hh[i], dd[i]);
    }
    free(rank); free(dist); free(best); free(settled); free(done); free(hh); free(dd); free(hp.key);
    finish_totals(L);
    return L;
}

/* ----------------------------------------------------------------- Alg. 4 */
/* BVC-PLL: hubs in batches of B consecutive ranks.  Per batch: the batch's
 * vertices start with dL(u) = {(u, 0)} added to L(u); then vertex-centric
 * rounds: every active a sends each (u, d) of dL(a) to each neighbour v with
 * rank(u) < rank(v) whose candidate bit-vector C(v) does not hold u yet (the
 * bit is set: u reaches v at most once per batch); each v that received
 * messages accepts (u, d) iff d < min over common hubs h of L(u) and L(v) of
 * d(u,h) + d(h,v), with the labels as they stood after the previous round;
 * the accepted ones form dL(v), are added to L(v) and make v active.  C is
 * cleared after the batch.  checks = messages sent.  NULL on a distance
 * above 254 or allocation failure. */
static int32_t row_find(const row_t* r, uint32_t hub) {   /* distance of hub in a rank-sorted row, or -1 */
    int64_t lo = 0, hi = r->len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (r->hub[mid] < hub) lo = mid + 1; else hi = mid;
    }
    return lo < r->len && r->hub[lo] == hub ? (int32_t)r->dist[lo] : -1;
}

static int row_insert_sorted(row_t* r, uint32_t hub, uint8_t d) {
    if (row_push(r, hub, d)) return -1;
    int64_t p = r->len - 1;
    while (p > 0 && r->hub[p - 1] > r->hub[p]) {
        uint32_t th = r->hub[p]; r->hub[p] = r->hub[p - 1]; r->hub[p - 1] = th;
        uint8_t td = r->dist[p]; r->dist[p] = r->dist[p - 1]; r->dist[p - 1] = td;
        --p;
    }
    return 0;
}

void* oracle_bvcpll(int64_t n, const int64_t* off, const int32_t* col, const int32_t* order, int64_t B) {
    labels_t* L = labels_new(n);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    if (B < 1) B = 1;
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * nn);
    row_t* dL = (row_t*)calloc(nn, sizeof(row_t));       /* dL(a): (hub rank, distance) of the last round */
    row_t* msg = (row_t*)calloc(nn, sizeof(row_t));      /* v.messages */
    row_t* ndL = (row_t*)calloc(nn, sizeof(row_t));
    unsigned char* C = (unsigned char*)calloc(nn * (size_t)(B < n ? B : (n > 0 ? n : 1)), 1);  /* C(v), B bits as bytes */
    int32_t* active = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* recv = (int32_t*)malloc(sizeof(int32_t) * nn);
    const int64_t Bw = B < n ? B : (n > 0 ? n : 1);
    int fail = 0;
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int32_t)r;
    for (int64_t lo = 0; lo < n && !fail; lo += B) {
        const int64_t hi = lo + B < n ? lo + B : n;
        int64_t na = 0;
        for (int64_t r = lo; r < hi; ++r) {                /* the batch's vertices: dL(u) = {(u, 0)} */
            const int32_t u = order[r];
            dL[u].len = 0;
            if (row_push(&dL[u], (uint32_t)r, 0) || row_insert_sorted(&L->rows[u], (uint32_t)r, 0)) fail = 1;
            active[na++] = u;
        }
        int32_t d = 0;
        while (na > 0 && !fail) {
            ++d;
            int64_t nr = 0;
            for (int64_t i = 0; i < na; ++i) {             /* scatter */
                const int32_t a = active[i];
                for (int64_t j = off[a]; j < off[a + 1]; ++j) {
                    const int32_t v = col[j];
                    for (int64_t k = 0; k < dL[a].len; ++k) {
                        const uint32_t u = dL[a].hub[k];
                        unsigned char* bit = &C[(size_t)v * (size_t)Bw + (size_t)((int64_t)u - lo)];
                        if ((int64_t)u < (int64_t)rank[v] && !*bit) {
                            *bit = 1;
                            if (msg[v].len == 0) recv[nr++] = v;
                            if (row_push(&msg[v], u, (uint8_t)(dL[a].dist[k] + 1 > 255 ? 255 : dL[a].dist[k] + 1)))
                                fail = 1;
                            ++L->checks;
                        }
                    }
                }
            }
            for (int64_t i = 0; i < na; ++i) dL[active[i]].len = 0;
            for (int64_t i = 0; i < nr; ++i) {             /* gather (labels of the previous rounds) */
                const int32_t v = recv[i];
                const row_t* Lv = &L->rows[v];
                ndL[v].len = 0;
                for (int64_t k = 0; k < msg[v].len; ++k) {
                    const uint32_t u = msg[v].hub[k];
                    const int32_t duv = msg[v].dist[k];
                    const row_t* Lu = &L->rows[order[u]];
                    int pruned = 0;
                    for (int64_t e = 0; e < Lv->len && !pruned; ++e) {
                        const int32_t du = row_find(Lu, Lv->hub[e]);
                        if (du >= 0 && du + (int32_t)Lv->dist[e] <= duv) pruned = 1;
                    }
                    if (!pruned) {
                        if (duv > 254) fail = 1;
                        else if (row_push(&ndL[v], u, (uint8_t)duv)) fail = 1;
                    }
                }
                msg[v].len = 0;
            }
            int64_t nn2 = 0;
            for (int64_t i = 0; i < nr; ++i) {             /* L(v) <- L(v) U dL(v); v becomes active */
                const int32_t v = recv[i];
                if (ndL[v].len == 0) continue;
                for (int64_t k = 0; k < ndL[v].len; ++k)
                    if (row_insert_sorted(&L->rows[v], ndL[v].hub[k], ndL[v].dist[k])) fail = 1;
                row_t t = dL[v];
                dL[v] = ndL[v];
                ndL[v] = t;
                ndL[v].len = 0;
                next[nn2++] = v;
            }
            for (int64_t i = 0; i < nn2; ++i) active[i] = next[i];
            na = nn2;
        }
        for (int64_t i = 0; i < na; ++i) dL[active[i]].len = 0;
        memset(C, 0, nn * (size_t)Bw);                     /* C(v) <- empty after the batch */
    }
    for (int64_t v = 0; v < n; ++v) {
        free(dL[v].hub); free(dL[v].dist);
        free(msg[v].hub); free(msg[v].dist);
        free(ndL[v].hub); free(ndL[v].dist);
    }
    free(dL); free(msg); free(ndL); free(C); free(active); free(next); free(recv); free(rank);
    if (fail) {
        oracle_labels_free(L);
        return NULL;
    }
    finish_totals(L);
    return L;
}
