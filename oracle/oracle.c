/*
 * oracle.c -- CPU oracle for k-core maintenance.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package smoke check and the CPU-baseline leg of
 * the benchmark load this code.  The CUDA library never calls it and shares
 * no code, header, table or helper with it.  Everything here is plain,
 * sequential and unoptimised on purpose, so that it can be checked against
 * the paper by eye.
 *
 * Paper: N. Wang, D. Yu, H. Jin, C. Qian, X. Xie, Q.-S. Hua, "Parallel
 * Algorithms for Core Maintenance in Dynamic Graphs" (arXiv 1612.09368).
 *
 *   O1  or_bz      Batagelj-Zaversnik O(m) peeling, the static decomposition
 *                  the paper cites as [O(m)] in Section I.  Computes core
 *                  numbers by their definition (Section III, Defs. 1-2).
 *   O2  or_brute   core(v) = max over vertex sets S containing v of the
 *                  minimum degree of G[S] (Section III, Defs. 1-2, with
 *                  connectivity dropped -- it does not change core numbers).
 *   O3  mode 0     the sequential single-edge traversal: every edge of a
 *                  batch on its own, through K-SuperiorInsert / InsertRemove
 *                  (Section V, Algorithms 3-4) or K-SuperiorDelete /
 *                  DeleteRemove (Section VI, Algorithms 6-7) with |E_k| = 1.
 *   O4  mode 1     the batched method: SuperiorEdgeInsert (Algorithm 1) and
 *                  SuperiorEdgeDelete (Algorithm 5), each iteration selecting
 *                  a superior edge set (Section IV Definition 6 and the union that
 *                  follows it; Algorithm 2), running Algorithm 3/6 once per
 *                  core level on the cores of the iteration's start, then
 *                  moving every found vertex by one.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  R1 Selection (Algorithm 2) is made well defined by a fixed priority: an
 *     edge's priority is fmix64 of its canonical key (lo << 32 | hi), the
 *     MurmurHash3 64-bit finaliser (A. Appleby, public domain), which is a
 *     bijection, so priorities are distinct.  Each iteration takes, in
 *     increasing priority, every remaining edge none of whose constrained
 *     endpoints (endpoints whose core equals the edge's core number,
 *     Section IV) is already taken.  The result satisfies Definition 6 (ii) at
 *     every level and is maximal.  Two variants (or_set_selection): the
 *     canonical key itself as the priority (lexicographic order), and the
 *     selection run as claim rounds capped at R per iteration -- in a round
 *     every eligible edge bids at its constrained endpoints and an edge
 *     holding the least bid at all of them is selected; run to the end, the
 *     rounds give the same set as the greedy pass, capped they give a
 *     superior edge set that may not be maximal.
 *  R2 The level set C of Algorithm 1 is recomputed from the remaining edges
 *     at the start of every iteration, as Algorithm 5 does explicitly.
 *  R3 Algorithm 3's "if cd[r] >= 0 then cd[r] <- CSD else cd[r] += CSD" is
 *     taken as cd[r] += CSD on first visit (an unvisited cd is 0 or has
 *     only been decremented, so both branches agree).
 *  R4 SD and CSD are measured on the graph after the whole iteration's
 *     superior edge set has been applied, with the cores of the iteration's
 *     start.
 *  R5 Deletion drops a vertex when its count falls strictly below k, as
 *     Algorithms 6-7 test (Lemma 9 is stated with "<=", which would also
 *     drop a vertex that still has exactly k superior neighbours).
 *  R6 Vertex insertion adds the vertex with core 0 and then its edges;
 *     vertex deletion deletes its edges and then the vertex (Section I).
 *     New ids are appended; a deleted vertex keeps its id and reports -1.
 *  R7 A batch is canonicalised to (lo, hi), self-loops dropped, duplicates
 *     collapsed to their first occurrence; inserting a present edge or
 *     deleting an absent one is skipped (the graph is simple, Section III).
 *
 * Planted mistakes: compiling with -DPLANT=n (n > 0) introduces one known
 * bug, so that the test suite can show its pins catch it.  The default
 * build (PLANT undefined) contains none of them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef PLANT
#define PLANT 0
#endif

#define OR_OK 0
#define OR_ERR_INVALID (-1)
#define OR_ERR_OOM (-2)

/* ------------------------------------------------------------------ */
/* MurmurHash3 fmix64 (bijective 64-bit finaliser).                    */
uint64_t or_fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* ------------------------------------------------------------------ */
/* O1: Batagelj-Zaversnik peeling on a simple graph given as an edge
 * list.  Returns OR_OK, or OR_ERR_INVALID for an id out of range, a
 * self-loop or a repeated edge (the oracle only accepts simple graphs). */
static int build_csr(int32_t n, int64_t m, const int32_t* e, int64_t** off_o, int32_t** adj_o) {
    int64_t* off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* adj = (int32_t*)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!off || !adj || !fill) { free(off); free(adj); free(fill); return OR_ERR_OOM; }
    for (int64_t i = 0; i < m; i++) {
        int32_t u = e[2 * i], v = e[2 * i + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) { free(off); free(adj); free(fill); return OR_ERR_INVALID; }
        off[u + 1]++; off[v + 1]++;
    }
    for (int32_t v = 0; v < n; v++) off[v + 1] += off[v];
    for (int64_t i = 0; i < m; i++) {
        int32_t u = e[2 * i], v = e[2 * i + 1];
        adj[off[u] + fill[u]++] = v;
        adj[off[v] + fill[v]++] = u;
    }
    free(fill);
    *off_o = off; *adj_o = adj;
    return OR_OK;
}

static int bz_on_csr(int32_t n, const int64_t* off, const int32_t* adj, int32_t* core) {
    int32_t md = 0;
    int32_t* deg = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t* pos = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t* vert = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!deg || !pos || !vert) { free(deg); free(pos); free(vert); return OR_ERR_OOM; }
    for (int32_t v = 0; v < n; v++) { deg[v] = (int32_t)(off[v + 1] - off[v]); if (deg[v] > md) md = deg[v]; }
    int32_t* bin = (int32_t*)calloc((size_t)md + 2, sizeof(int32_t));
    if (!bin) { free(deg); free(pos); free(vert); return OR_ERR_OOM; }
    /* bin-sort the vertices by degree */
    for (int32_t v = 0; v < n; v++) bin[deg[v]]++;
    int32_t start = 0;
    for (int32_t d = 0; d <= md; d++) { int32_t c = bin[d]; bin[d] = start; start += c; }
    for (int32_t v = 0; v < n; v++) { pos[v] = bin[deg[v]]; vert[pos[v]] = v; bin[deg[v]]++; }
    for (int32_t d = md; d >= 1; d--) bin[d] = bin[d - 1];
    bin[0] = 0;
    /* take vertices in order of current degree; a vertex's core is its
     * degree when taken; each later neighbour loses one degree and moves
     * one bin down */
    for (int32_t i = 0; i < n; i++) {
        int32_t v = vert[i];
        core[v] = deg[v];
        for (int64_t j = off[v]; j < off[v + 1]; j++) {
            int32_t u = adj[j];
#if PLANT == 1
            if (deg[u] >= deg[v] && pos[u] > i) {
#else
            if (deg[u] > deg[v]) {
#endif
                int32_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    free(deg); free(pos); free(vert); free(bin);
    return OR_OK;
}

int or_bz(int32_t n, int64_t m, const int32_t* edges, int32_t* core) {
    if (n < 0 || m < 0) return OR_ERR_INVALID;
    int64_t* off; int32_t* adj;
    int rc = build_csr(n, m, edges, &off, &adj);
    if (rc) return rc;
    /* reject repeated edges: sort each list and look for equal neighbours */
    for (int32_t v = 0; v < n; v++) {
        for (int64_t a = off[v] + 1; a < off[v + 1]; a++) {       /* insertion sort, lists are small in tests */
            int32_t x = adj[a]; int64_t b = a - 1;
            while (b >= off[v] && adj[b] > x) { adj[b + 1] = adj[b]; b--; }
            adj[b + 1] = x;
        }
        for (int64_t a = off[v] + 1; a < off[v + 1]; a++)
            if (adj[a] == adj[a - 1]) { free(off); free(adj); return OR_ERR_INVALID; }
    }
    rc = bz_on_csr(n, off, adj, core);
    free(off); free(adj);
    return rc;
}

/* Same as or_bz but trusts the input to be simple (no sort): for large
 * graphs whose edge lists come from the generators, which dedupe. */
int or_bz_trusted(int32_t n, int64_t m, const int32_t* edges, int32_t* core) {
    if (n < 0 || m < 0) return OR_ERR_INVALID;
    int64_t* off; int32_t* adj;
    int rc = build_csr(n, m, edges, &off, &adj);
    if (rc) return rc;
    rc = bz_on_csr(n, off, adj, core);
    free(off); free(adj);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O2: brute force over all vertex subsets, n <= 20. */
int or_brute(int32_t n, int64_t m, const int32_t* edges, int32_t* core) {
    if (n < 0 || n > 20) return OR_ERR_INVALID;
    uint32_t nb[20];
    memset(nb, 0, sizeof(nb));
    for (int64_t i = 0; i < m; i++) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return OR_ERR_INVALID;
        nb[u] |= 1u << v; nb[v] |= 1u << u;
    }
    for (int32_t v = 0; v < n; v++) core[v] = 0;
    for (uint32_t S = 1; S < (1u << n); S++) {
        int32_t mind = 1 << 30;
        for (int32_t x = 0; x < n; x++)
            if (S >> x & 1) { int32_t d = __builtin_popcount(nb[x] & S); if (d < mind) mind = d; }
        for (int32_t x = 0; x < n; x++)
            if ((S >> x & 1) && core[x] < mind) core[x] = mind;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Dynamic graph state for O3 / O4. */
typedef struct {
    int32_t n, ncap;
    int32_t* core;                 /* -1 for a deleted vertex */
    int32_t* deg; int32_t* cap; int32_t** adj;
    int64_t m;
    /* traversal scratch, reset through the touched list */
    int32_t* cd; uint8_t* visited; uint8_t* removed; uint8_t* touched;
    int32_t* sdv; uint8_t* sdok;
    int32_t* tl; int64_t ntl;
    int32_t* st1; int32_t* st2;
    /* batch bookkeeping */
    uint32_t* taken; uint32_t stamp;
    int64_t nrem, remcap; int32_t* rem; uint64_t* remprio; int32_t bop;
    int32_t sel_order, sel_rounds;    /* R1 variants: 1 = key order; R > 0 = claim rounds capped at R */
    int64_t iters, logcap, nlog; int64_t* log;
} or_graph;

static int g_vgrow(or_graph* g, int32_t need) {
    if (need <= g->ncap) return 0;
    int32_t nc = g->ncap ? g->ncap : 16;
    while (nc < need) nc = nc + nc / 2 + 16;
#define RE(p, T) do { void* q = realloc(g->p, (size_t)nc * sizeof(T)); if (!q) return OR_ERR_OOM; g->p = (T*)q; } while (0)
    RE(core, int32_t); RE(deg, int32_t); RE(cap, int32_t); RE(adj, int32_t*);
    RE(cd, int32_t); RE(visited, uint8_t); RE(removed, uint8_t); RE(touched, uint8_t);
    RE(sdv, int32_t); RE(sdok, uint8_t); RE(tl, int32_t); RE(st1, int32_t); RE(st2, int32_t); RE(taken, uint32_t);
#undef RE
    for (int32_t i = g->ncap; i < nc; i++) {
        g->core[i] = -1; g->deg[i] = 0; g->cap[i] = 0; g->adj[i] = NULL;
        g->cd[i] = 0; g->visited[i] = 0; g->removed[i] = 0; g->touched[i] = 0; g->sdv[i] = 0; g->sdok[i] = 0; g->taken[i] = 0;
    }
    g->ncap = nc;
    return 0;
}

static int has_edge(const or_graph* g, int32_t u, int32_t v) {
    int32_t a = g->deg[u] <= g->deg[v] ? u : v, b = a == u ? v : u;
    for (int32_t i = 0; i < g->deg[a]; i++) if (g->adj[a][i] == b) return 1;
    return 0;
}
static int push_nbr(or_graph* g, int32_t u, int32_t v) {
    if (g->deg[u] == g->cap[u]) {
        int32_t nc = g->cap[u] ? g->cap[u] * 2 : 4;
        int32_t* q = (int32_t*)realloc(g->adj[u], (size_t)nc * sizeof(int32_t));
        if (!q) return OR_ERR_OOM;
        g->adj[u] = q; g->cap[u] = nc;
    }
    g->adj[u][g->deg[u]++] = v;
    return 0;
}
static void drop_nbr(or_graph* g, int32_t u, int32_t v) {
    for (int32_t i = 0; i < g->deg[u]; i++)
        if (g->adj[u][i] == v) { g->adj[u][i] = g->adj[u][--g->deg[u]]; return; }
}
static void add_edge(or_graph* g, int32_t u, int32_t v) { push_nbr(g, u, v); push_nbr(g, v, u); g->m++; }
static void del_edge(or_graph* g, int32_t u, int32_t v) { drop_nbr(g, u, v); drop_nbr(g, v, u); g->m--; }

or_graph* or_create(int32_t n, int64_t m, const int32_t* edges, const int32_t* cores) {
    if (n < 0 || m < 0) return NULL;
    or_graph* g = (or_graph*)calloc(1, sizeof(or_graph));
    if (!g) return NULL;
    if (g_vgrow(g, n > 0 ? n : 1)) { free(g); return NULL; }
    g->n = n;
    for (int32_t v = 0; v < n; v++) g->core[v] = 0;
    for (int64_t i = 0; i < m; i++) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || has_edge(g, u, v)) continue;
        add_edge(g, u, v);
    }
    if (cores) {
        for (int32_t v = 0; v < n; v++) g->core[v] = cores[v];
    } else {
        int32_t* e = (int32_t*)malloc((size_t)(2 * g->m + 1) * sizeof(int32_t));
        int64_t k = 0;
        for (int32_t u = 0; u < n; u++)
            for (int32_t i = 0; i < g->deg[u]; i++)
                if (g->adj[u][i] > u) { e[2 * k] = u; e[2 * k + 1] = g->adj[u][i]; k++; }
        or_bz_trusted(n, k, e, g->core);
        free(e);
    }
    g->stamp = 1;
    return g;
}

void or_free(or_graph* g);

/* The graph or_create builds, for an edge list already known to be simple
 * (ids in range, no self-loop, no pair twice in either orientation), without
 * or_create's per-edge membership test, which costs up to a hub's degree per
 * edge on skewed graphs.  The precondition is NOT checked: a repeated pair
 * would be stored twice.  Cores as in or_create (NULL: O1 on the graph). */
or_graph* or_create_simple(int32_t n, int64_t m, const int32_t* edges, const int32_t* cores) {
    if (n < 0 || m < 0) return NULL;
    or_graph* g = (or_graph*)calloc(1, sizeof(or_graph));
    if (!g) return NULL;
    if (g_vgrow(g, n > 0 ? n : 1)) { free(g); return NULL; }
    g->n = n;
    for (int64_t i = 0; i < 2 * m; i++) {
        if (edges[i] < 0 || edges[i] >= n) { or_free(g); return NULL; }
        g->cap[edges[i]]++;
    }
    for (int32_t v = 0; v < n; v++) {
        g->core[v] = 0;
        if (g->cap[v] && !(g->adj[v] = (int32_t*)malloc((size_t)g->cap[v] * sizeof(int32_t)))) { or_free(g); return NULL; }
    }
    for (int64_t i = 0; i < m; i++) add_edge(g, edges[2 * i], edges[2 * i + 1]);
    if (cores) {
        for (int32_t v = 0; v < n; v++) g->core[v] = cores[v];
    } else if (or_bz_trusted(n, m, edges, g->core) != OR_OK) {
        or_free(g);
        return NULL;
    }
    g->stamp = 1;
    return g;
}

/* Checkpoint restore (no core maintenance): op 0 adds, op 1 removes the k
 * pairs (each must be absent, resp. present, not checked) to the structure
 * only; or_set_cores then overwrites every core number.  Used to put a graph
 * back into a state saved before an update, whose core numbers are known. */
void or_apply_structure(or_graph* g, int32_t op, const int32_t* e, int64_t k) {
    for (int64_t i = 0; i < k; i++) {
        if (op == 0) add_edge(g, e[2 * i], e[2 * i + 1]);
        else del_edge(g, e[2 * i], e[2 * i + 1]);
    }
}
void or_set_cores(or_graph* g, const int32_t* cores) { memcpy(g->core, cores, (size_t)g->n * sizeof(int32_t)); }

void or_free(or_graph* g) {
    if (!g) return;
    for (int32_t i = 0; i < g->ncap; i++) free(g->adj[i]);
    free(g->core); free(g->deg); free(g->cap); free(g->adj); free(g->cd); free(g->visited); free(g->removed);
    free(g->touched); free(g->sdv); free(g->sdok); free(g->tl); free(g->st1); free(g->st2); free(g->taken);
    free(g->rem); free(g->remprio); free(g->log); free(g);
}
int32_t or_n(const or_graph* g) { return g->n; }
int64_t or_m(const or_graph* g) { return g->m; }
void or_get_cores(const or_graph* g, int32_t* out) { memcpy(out, g->core, (size_t)g->n * sizeof(int32_t)); }
int64_t or_edges(const or_graph* g, int32_t* out) {
    int64_t k = 0;
    for (int32_t u = 0; u < g->n; u++)
        for (int32_t i = 0; i < g->deg[u]; i++)
            if (g->adj[u][i] > u) { out[2 * k] = u; out[2 * k + 1] = g->adj[u][i]; k++; }
    return k;
}
int64_t or_last_iterations(const or_graph* g) { return g->iters; }
int64_t or_last_log(const or_graph* g, int64_t* out, int64_t cap) {
    int64_t k = g->nlog < cap ? g->nlog : cap;
    memcpy(out, g->log, (size_t)(2 * k) * sizeof(int64_t));
    return g->nlog;
}

/* ---- scratch handling ---- */
static inline void touch(or_graph* g, int32_t v) { if (!g->touched[v]) { g->touched[v] = 1; g->tl[g->ntl++] = v; } }
static void reset_scratch(or_graph* g) {
    for (int64_t i = 0; i < g->ntl; i++) {
        int32_t v = g->tl[i];
        g->cd[v] = 0; g->visited[v] = 0; g->removed[v] = 0; g->touched[v] = 0; g->sdok[v] = 0;
    }
    g->ntl = 0;
}

/* SD(u), Definition 7 (superior degree): the number of neighbours w with core(w) >= core(u). */
static int32_t SD(or_graph* g, int32_t u) {
    if (g->sdok[u]) return g->sdv[u];
    int32_t c = 0;
    for (int32_t i = 0; i < g->deg[u]; i++) if (g->core[g->adj[u][i]] >= g->core[u]) c++;
    touch(g, u);
    g->sdv[u] = c; g->sdok[u] = 1;
    return c;
}
/* CSD(u), Definition 8 (constraint superior degree): neighbours w with core(w) > core(u), or core(w) = core(u)
 * and SD(w) > core(u). */
static int32_t CSD(or_graph* g, int32_t u) {
    int32_t c = 0, k = g->core[u];
    for (int32_t i = 0; i < g->deg[u]; i++) {
        int32_t w = g->adj[u][i];
#if PLANT == 2
        if (g->core[w] > k || (g->core[w] == k && SD(g, w) >= k)) c++;
#else
        if (g->core[w] > k || (g->core[w] == k && SD(g, w) > k)) c++;
#endif
    }
    return c;
}

/* InsertRemove (Algorithm 4): negative DFS from r at level k. */
static void insert_remove(or_graph* g, int32_t r, int32_t k) {
    int64_t sp = 0;
    g->st2[sp++] = r; touch(g, r); g->removed[r] = 1;
    while (sp) {
        int32_t v = g->st2[--sp];
        for (int32_t i = 0; i < g->deg[v]; i++) {
            int32_t w = g->adj[v][i];
            if (g->core[w] == k) {
                touch(g, w);
                g->cd[w]--;
                if (g->cd[w] == k && !g->removed[w]) { g->st2[sp++] = w; g->removed[w] = 1; }
            }
        }
    }
}

/* K-SuperiorInsert (Algorithm 3) for the k-superior edge set given as
 * pairs; appends the vertices whose core rises to out (V_k). */
static int64_t k_superior_insert(or_graph* g, const int32_t* ek, int64_t ne, int32_t k, int32_t* out) {
    for (int64_t i = 0; i < ne; i++) {
        int32_t u = ek[2 * i], v = ek[2 * i + 1];
        int32_t r = g->core[u] >= g->core[v] ? v : u;     /* the endpoint with core k */
        if (g->visited[r] || g->removed[r]) continue;
        touch(g, r);
        g->cd[r] += CSD(g, r);                              /* reading R3 */
        int64_t sp = 0;
        g->st1[sp++] = r; g->visited[r] = 1;
        while (sp) {
            int32_t x = g->st1[--sp];
            if (g->cd[x] > k) {                              /* positive DFS: expand */
                for (int32_t j = 0; j < g->deg[x]; j++) {
                    int32_t w = g->adj[x][j];
                    if (g->core[w] == k && SD(g, w) > k && !g->visited[w]) {
                        touch(g, w);
                        g->st1[sp++] = w; g->visited[w] = 1;
                        g->cd[w] += CSD(g, w);
                    }
                }
            } else if (!g->removed[x]) {
                insert_remove(g, x, k);                      /* negative DFS */
            }
        }
    }
    int64_t c = 0;
    for (int64_t i = 0; i < g->ntl; i++) {
        int32_t v = g->tl[i];
#if PLANT == 3
        if (g->visited[v]) out[c++] = v;
#else
        if (g->visited[v] && !g->removed[v]) out[c++] = v;
#endif
    }
    return c;
}

/* DeleteRemove (Algorithm 7): negative DFS from r at level k. */
static void delete_remove(or_graph* g, int32_t r, int32_t k) {
    int64_t sp = 0;
    g->st2[sp++] = r; touch(g, r); g->removed[r] = 1;
    while (sp) {
        int32_t v = g->st2[--sp];
        for (int32_t i = 0; i < g->deg[v]; i++) {
            int32_t w = g->adj[v][i];
            if (g->core[w] == k) {
                touch(g, w);
                if (!g->visited[w]) { g->visited[w] = 1; g->cd[w] += SD(g, w); }
                g->cd[w]--;
#if PLANT == 4
                if (g->cd[w] <= k && !g->removed[w]) { g->st2[sp++] = w; g->removed[w] = 1; }
#else
                if (g->cd[w] < k && !g->removed[w]) { g->st2[sp++] = w; g->removed[w] = 1; }   /* reading R5 */
#endif
            }
        }
    }
}

static void del_root(or_graph* g, int32_t x, int32_t k) {
    touch(g, x);
    if (!g->visited[x]) { g->visited[x] = 1; g->cd[x] = SD(g, x); }
    if (!g->removed[x] && g->cd[x] < k) delete_remove(g, x, k);
}

/* K-SuperiorDelete (Algorithm 6); appends V_c (vertices whose core drops). */
static int64_t k_superior_delete(or_graph* g, const int32_t* ek, int64_t ne, int32_t k, int32_t* out) {
    for (int64_t i = 0; i < ne; i++) {
        int32_t u = ek[2 * i], v = ek[2 * i + 1];
        int32_t r = g->core[u] >= g->core[v] ? v : u;
        if (g->core[u] != g->core[v]) {
            del_root(g, r, k);
        } else {
            del_root(g, u, k);
#if PLANT != 5
            del_root(g, v, k);
#endif
        }
    }
    int64_t c = 0;
    for (int64_t i = 0; i < g->ntl; i++) {
        int32_t v = g->tl[i];
        if (g->removed[v] && g->visited[v]) out[c++] = v;
    }
    return c;
}

/* ---- batch ingest (reading R7) ---- */
static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : x > y;
}
/* Validate ids, canonicalise, drop self-loops and repeats (first kept),
 * drop present (op 0) or absent (op 1) edges.  Writes kept pairs to keep
 * (in input order) and returns their number, or OR_ERR_INVALID. */
static int64_t ingest(or_graph* g, int32_t op, const int32_t* e, int64_t k, int32_t* keep) {
    for (int64_t i = 0; i < 2 * k; i++)
        if (e[i] < 0 || e[i] >= g->n || g->core[e[i]] < 0) return OR_ERR_INVALID;
    /* repeats: sort (key, position) and keep the smallest position per key */
    uint64_t* kp = (uint64_t*)malloc((size_t)(2 * k + 2) * sizeof(uint64_t));
    uint8_t* first = (uint8_t*)calloc((size_t)k + 1, 1);
    if (!kp || !first) { free(kp); free(first); return OR_ERR_OOM; }
    int64_t nk = 0;
    for (int64_t i = 0; i < k; i++) {
        int32_t u = e[2 * i], v = e[2 * i + 1];
        if (u == v) continue;
        uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
        kp[2 * nk] = ((uint64_t)lo << 32) | hi; kp[2 * nk + 1] = (uint64_t)i; nk++;
    }
    /* sort pairs (key, pos) lexicographically: pack into a struct-sort */
    typedef struct { uint64_t key, pos; } kp_t;
    kp_t* arr = (kp_t*)kp;
    qsort(arr, (size_t)nk, sizeof(kp_t), cmp_u64);   /* key only; fix positions below */
    for (int64_t a = 0; a < nk;) {
        int64_t b = a; uint64_t mn = arr[a].pos;
        while (b < nk && arr[b].key == arr[a].key) { if (arr[b].pos < mn) mn = arr[b].pos; b++; }
        first[mn] = 1;
        a = b;
    }
    int64_t c = 0;
    for (int64_t i = 0; i < k; i++) {
        if (!first[i]) continue;
        int32_t u = e[2 * i], v = e[2 * i + 1];
        int present = has_edge(g, u, v);
        if ((op == 0 && present) || (op == 1 && !present)) continue;
        keep[2 * c] = u; keep[2 * c + 1] = v; c++;
    }
    free(kp); free(first);
    return c;
}

/* ---- O3: sequential single-edge processing ---- */
static int64_t seq_edges(or_graph* g, int32_t op, const int32_t* e, int64_t k) {
    int32_t* keep = (int32_t*)malloc((size_t)(2 * k + 2) * sizeof(int32_t));
    int32_t* out = (int32_t*)malloc((size_t)(g->n + 1) * sizeof(int32_t));
    if (!keep || !out) { free(keep); free(out); return OR_ERR_OOM; }
    int64_t c = ingest(g, op, e, k, keep);
    if (c < 0) { free(keep); free(out); return c; }
    for (int64_t i = 0; i < c; i++) {
        int32_t u = keep[2 * i], v = keep[2 * i + 1];
        int32_t lvl = g->core[u] < g->core[v] ? g->core[u] : g->core[v];
        int64_t nc;
        if (op == 0) { add_edge(g, u, v); nc = k_superior_insert(g, keep + 2 * i, 1, lvl, out); }
        else { del_edge(g, u, v); nc = k_superior_delete(g, keep + 2 * i, 1, lvl, out); }
        reset_scratch(g);
        for (int64_t j = 0; j < nc; j++) g->core[out[j]] += op == 0 ? 1 : -1;
    }
    g->iters = c;
    free(keep); free(out);
    return c;
}

/* ---- O4: superior edge sets (Algorithms 1, 2, 5) ---- */
typedef struct { uint64_t prio; int64_t idx; } pr_t;
static int cmp_pr(const void* a, const void* b) {
    uint64_t x = ((const pr_t*)a)->prio, y = ((const pr_t*)b)->prio;
    return x < y ? -1 : x > y;
}

int64_t or_batch_begin(or_graph* g, int32_t op, const int32_t* e, int64_t k) {
    int32_t* keep = (int32_t*)malloc((size_t)(2 * k + 2) * sizeof(int32_t));
    if (!keep) return OR_ERR_OOM;
    int64_t c = ingest(g, op, e, k, keep);
    if (c < 0) { free(keep); return c; }
    pr_t* pr = (pr_t*)malloc((size_t)(c + 1) * sizeof(pr_t));
    for (int64_t i = 0; i < c; i++) {
        int32_t u = keep[2 * i], v = keep[2 * i + 1];
        uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
        const uint64_t key = ((uint64_t)lo << 32) | hi;
        pr[i].prio = g->sel_order == 1 ? key : or_fmix64(key); pr[i].idx = i;
    }
    qsort(pr, (size_t)c, sizeof(pr_t), cmp_pr);        /* priorities are distinct (bijection) */
    free(g->rem); free(g->remprio);
    g->rem = (int32_t*)malloc((size_t)(2 * c + 2) * sizeof(int32_t));
    g->remprio = (uint64_t*)malloc((size_t)(c + 1) * sizeof(uint64_t));
    for (int64_t i = 0; i < c; i++) {
        g->rem[2 * i] = keep[2 * pr[i].idx]; g->rem[2 * i + 1] = keep[2 * pr[i].idx + 1];
        g->remprio[i] = pr[i].prio;
    }
    g->nrem = c; g->bop = op; g->iters = 0; g->nlog = 0;
    free(keep); free(pr);
    return c;
}

/* Selection as claim rounds (reading R1, capped variant).  Round after
 * round, every remaining edge that is not selected and none of whose
 * constrained endpoints is taken bids its priority at its constrained
 * endpoints; each edge whose bid is the least at every one of them is
 * selected and takes them.  Stops when a round had no losing bid, or after
 * g->sel_rounds rounds.  Writes the selected edges and their levels and
 * keeps the rest, in priority order, as the remaining edges. */
static void claim_rounds(or_graph* g, int32_t* sel, int32_t* lvl, int64_t* ns_out) {
    const int64_t nrem = g->nrem;
    uint64_t* best = (uint64_t*)malloc((size_t)(g->n + 1) * sizeof(uint64_t));
    uint8_t* chosen = (uint8_t*)calloc((size_t)nrem + 1, 1);
    uint8_t* bids = (uint8_t*)calloc((size_t)nrem + 1, 1);
    for (int32_t round = 0; round < g->sel_rounds; round++) {
        for (int64_t i = 0; i < nrem; i++) { best[g->rem[2 * i]] = UINT64_MAX; best[g->rem[2 * i + 1]] = UINT64_MAX; }
        int64_t nbid = 0, nwin = 0;
        for (int64_t i = 0; i < nrem; i++) {
            int32_t u = g->rem[2 * i], v = g->rem[2 * i + 1];
            int32_t k = g->core[u] < g->core[v] ? g->core[u] : g->core[v];
            int cu = g->core[u] == k, cv = g->core[v] == k;
            bids[i] = !chosen[i] && !(cu && g->taken[u] == g->stamp) && !(cv && g->taken[v] == g->stamp);
            if (!bids[i]) continue;
            nbid++;
            if (cu && g->remprio[i] < best[u]) best[u] = g->remprio[i];
            if (cv && g->remprio[i] < best[v]) best[v] = g->remprio[i];
        }
        for (int64_t i = 0; i < nrem; i++) {
            if (!bids[i]) continue;
            int32_t u = g->rem[2 * i], v = g->rem[2 * i + 1];
            int32_t k = g->core[u] < g->core[v] ? g->core[u] : g->core[v];
            int cu = g->core[u] == k, cv = g->core[v] == k;
            if ((!cu || best[u] == g->remprio[i]) && (!cv || best[v] == g->remprio[i])) { chosen[i] = 1; nwin++; }
        }
        for (int64_t i = 0; i < nrem; i++) {       /* winners take their constrained endpoints */
            if (!bids[i] || !chosen[i]) continue;
            int32_t u = g->rem[2 * i], v = g->rem[2 * i + 1];
            int32_t k = g->core[u] < g->core[v] ? g->core[u] : g->core[v];
            if (g->core[u] == k) g->taken[u] = g->stamp;
            if (g->core[v] == k) g->taken[v] = g->stamp;
        }
        if (nwin == nbid) break;                    /* no bid lost: the set is maximal */
    }
    int64_t ns = 0, nr = 0;
    for (int64_t i = 0; i < nrem; i++) {
        int32_t u = g->rem[2 * i], v = g->rem[2 * i + 1];
        if (chosen[i]) {
            int32_t k = g->core[u] < g->core[v] ? g->core[u] : g->core[v];
            sel[2 * ns] = u; sel[2 * ns + 1] = v; lvl[ns] = k; ns++;
        } else {
            g->rem[2 * nr] = u; g->rem[2 * nr + 1] = v; g->remprio[nr] = g->remprio[i]; nr++;
        }
    }
    g->nrem = nr;
    *ns_out = ns;
    free(best); free(chosen); free(bids);
}

/* Selection variants of reading R1: order 1 ranks edges by their canonical
 * key instead of its fmix64; rounds > 0 caps the claim rounds per
 * iteration.  Takes effect at the next batch. */
void or_set_selection(or_graph* g, int32_t order, int32_t rounds) {
    g->sel_order = order == 1 ? 1 : 0;
    g->sel_rounds = rounds > 0 ? rounds : 0;
}

/* One iteration of Algorithm 1 (op 0) or Algorithm 5 (op 1).  Optionally
 * reports the selected edges and the changed vertices.  Returns 1 if an
 * iteration ran, 0 if no edges remained. */
int32_t or_batch_step(or_graph* g, int32_t* sel_out, int64_t* nsel_out, int32_t* chg_out, int64_t* nchg_out) {
    if (g->nrem == 0) return 0;
    int32_t op = g->bop;
    g->stamp++;
    if (g->stamp == 0) { memset(g->taken, 0, (size_t)g->ncap * sizeof(uint32_t)); g->stamp = 1; }
    /* Algorithm 2 per level, with reading R1: greedy in priority order */
    int32_t* sel = (int32_t*)malloc((size_t)(2 * g->nrem + 2) * sizeof(int32_t));
    int32_t* lvl = (int32_t*)malloc((size_t)(g->nrem + 1) * sizeof(int32_t));
    int64_t ns = 0, nr = 0;
    if (g->sel_rounds > 0) {
        claim_rounds(g, sel, lvl, &ns);
    } else {
        for (int64_t i = 0; i < g->nrem; i++) {
            int32_t u = g->rem[2 * i], v = g->rem[2 * i + 1];
            int32_t k = g->core[u] < g->core[v] ? g->core[u] : g->core[v];
            int cu = g->core[u] == k, cv = g->core[v] == k;      /* constrained endpoints */
#if PLANT == 6
            cv = 0;
#endif
            if ((cu && g->taken[u] == g->stamp) || (cv && g->taken[v] == g->stamp)) {
                g->rem[2 * nr] = u; g->rem[2 * nr + 1] = v; g->remprio[nr] = g->remprio[i]; nr++;
                continue;
            }
            if (cu) g->taken[u] = g->stamp;
            if (cv) g->taken[v] = g->stamp;
            sel[2 * ns] = u; sel[2 * ns + 1] = v; lvl[ns] = k; ns++;
        }
        g->nrem = nr;
    }
    /* insert / delete the union of the E_k (Algorithms 1 and 5) */
    for (int64_t i = 0; i < ns; i++) {
        if (op == 0) add_edge(g, sel[2 * i], sel[2 * i + 1]);
        else del_edge(g, sel[2 * i], sel[2 * i + 1]);
    }
    /* Algorithm 3 / 6 once per level, on the cores of the iteration's start */
    int32_t* chg = (int32_t*)malloc((size_t)(g->n + 1) * sizeof(int32_t));
    int32_t* ek = (int32_t*)malloc((size_t)(2 * ns + 2) * sizeof(int32_t));
    uint8_t* done = (uint8_t*)calloc((size_t)ns + 1, 1);
    int64_t nc = 0;
    for (int64_t i = 0; i < ns; i++) {
        if (done[i]) continue;
        int32_t k = lvl[i];
        int64_t ne = 0;
        for (int64_t j = i; j < ns; j++)
            if (!done[j] && lvl[j] == k) { ek[2 * ne] = sel[2 * j]; ek[2 * ne + 1] = sel[2 * j + 1]; ne++; done[j] = 1; }
        nc += op == 0 ? k_superior_insert(g, ek, ne, k, chg + nc) : k_superior_delete(g, ek, ne, k, chg + nc);
        reset_scratch(g);
    }
    /* the last step of Algorithms 1 and 5: every vertex found moves by one */
    for (int64_t j = 0; j < nc; j++) g->core[chg[j]] += op == 0 ? 1 : -1;
    if (g->nlog == g->logcap) {
        g->logcap = g->logcap ? 2 * g->logcap : 64;
        g->log = (int64_t*)realloc(g->log, (size_t)(2 * g->logcap) * sizeof(int64_t));
    }
    g->log[2 * g->nlog] = ns; g->log[2 * g->nlog + 1] = nc; g->nlog++;
    g->iters++;
    if (sel_out) memcpy(sel_out, sel, (size_t)(2 * ns) * sizeof(int32_t));
    if (nsel_out) *nsel_out = ns;
    if (chg_out) memcpy(chg_out, chg, (size_t)nc * sizeof(int32_t));
    if (nchg_out) *nchg_out = nc;
    free(sel); free(lvl); free(chg); free(ek); free(done);
    return 1;
}

static int64_t batch_edges(or_graph* g, int32_t op, const int32_t* e, int64_t k) {
    int64_t c = or_batch_begin(g, op, e, k);
    if (c < 0) return c;
    while (or_batch_step(g, NULL, NULL, NULL, NULL)) {}
    return c;
}

/* Insert (op 0) or delete (op 1) a batch of edges; mode 0 = O3 sequential,
 * mode 1 = O4 superior edge sets.  Returns the number of edges applied, or
 * a negative error with the graph unchanged. */
int64_t or_update_edges(or_graph* g, int32_t op, const int32_t* e, int64_t k, int32_t mode) {
    if (k < 0 || (op != 0 && op != 1)) return OR_ERR_INVALID;
    return mode == 0 ? seq_edges(g, op, e, k) : batch_edges(g, op, e, k);
}

/* Vertex insertion (reading R6): `count` new vertices with ids n..n+count-1
 * and core 0; vertex i's neighbours are nbrs[off[i] .. off[i+1]).  Then one
 * insert batch of all their edges, in that flattened order.  Returns the
 * first new id or a negative error (graph unchanged). */
int64_t or_insert_vertices(or_graph* g, int32_t count, const int64_t* off, const int32_t* nbrs, int32_t mode) {
    if (count < 0) return OR_ERR_INVALID;
    int32_t base = g->n;
    int64_t tot = off[count];
    for (int64_t j = 0; j < tot; j++) {
        int32_t w = nbrs[j];
        if (w < 0 || w >= base + count || (w < base && g->core[w] < 0)) return OR_ERR_INVALID;
    }
    for (int32_t i = 0; i < count; i++)
        for (int64_t j = off[i]; j < off[i + 1]; j++) if (nbrs[j] == base + i) return OR_ERR_INVALID;
    if (g_vgrow(g, base + count)) return OR_ERR_OOM;
    for (int32_t i = 0; i < count; i++) { g->core[base + i] = 0; g->deg[base + i] = 0; }
    g->n = base + count;
    int32_t* e = (int32_t*)malloc((size_t)(2 * tot + 2) * sizeof(int32_t));
    for (int32_t i = 0; i < count; i++)
        for (int64_t j = off[i]; j < off[i + 1]; j++) { e[2 * j] = base + i; e[2 * j + 1] = nbrs[j]; }
    int64_t rc = or_update_edges(g, 0, e, tot, mode);
    free(e);
    return rc < 0 ? rc : base;
}

/* Vertex deletion (reading R6): one delete batch of all edges incident to
 * the given vertices, then the vertices are marked dead.  Returns the
 * number of edges deleted or a negative error (graph unchanged). */
int64_t or_delete_vertices(or_graph* g, int32_t count, const int32_t* ids, int32_t mode) {
    for (int32_t i = 0; i < count; i++)
        if (ids[i] < 0 || ids[i] >= g->n || g->core[ids[i]] < 0) return OR_ERR_INVALID;
    int64_t tot = 0;
    for (int32_t i = 0; i < count; i++) tot += g->deg[ids[i]];
    int32_t* e = (int32_t*)malloc((size_t)(2 * tot + 2) * sizeof(int32_t));
    int64_t c = 0;
    for (int32_t i = 0; i < count; i++)
        for (int32_t j = 0; j < g->deg[ids[i]]; j++) { e[2 * c] = ids[i]; e[2 * c + 1] = g->adj[ids[i]][j]; c++; }
    int64_t rc = or_update_edges(g, 1, e, c, mode);
    free(e);
    if (rc < 0) return rc;
    for (int32_t i = 0; i < count; i++) g->core[ids[i]] = -1;
    return rc;
}
