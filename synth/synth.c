/*
 * synth.c -- seeded synthetic graphs and update streams.
 *
 * This module only produces inputs: edge lists, update batches, vertex ids.
 * It computes no core numbers and holds none of the maintenance method's
 * arithmetic, so the CPU oracle and the CUDA library can both consume what
 * it writes without sharing any of the method's code.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: draw i of stream s is mix(s + (i + 1) * golden_gamma).
 *
 * Graph families follow the synthetic families of the paper's experiments
 * (Section VII, "Datasets": Erdos-Renyi, Barabasi-Albert, R-MAT) plus a
 * 4-neighbour grid with random shortcuts for the serving workload.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t draw(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GOLDEN); }
static inline uint64_t below(uint64_t x, uint64_t n) { return (uint64_t)(((__uint128_t)x * n) >> 64); }
static inline double unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

typedef struct { uint64_t seed, ctr; } rng_t;
static inline uint64_t rnext(rng_t* r) { return draw(r->seed, r->ctr++); }

/* Stream seed for a tuple of labels (config, graph, round, purpose). */
uint64_t sy_stream(uint64_t base, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    uint64_t s = mix64(base + GOLDEN);
    s = mix64(s ^ (a + 1) * GOLDEN);
    s = mix64(s ^ (b + 2) * GOLDEN);
    s = mix64(s ^ (c + 3) * GOLDEN);
    s = mix64(s ^ (d + 4) * GOLDEN);
    return s;
}
uint64_t sy_draw(uint64_t seed, uint64_t i) { return draw(seed, i); }

static inline uint64_t ekey(int32_t u, int32_t v) {
    uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
    return ((uint64_t)lo << 32) | hi;
}

/* ---------------- open-addressing hash map u64 -> i64 ---------------- */
#define HEMPTY 0xFFFFFFFFFFFFFFFFULL
typedef struct { uint64_t* k; int64_t* v; uint64_t mask; int64_t used; } hmap;

static int hm_init(hmap* h, int64_t expect) {
    uint64_t sz = 16;
    while (sz < (uint64_t)(expect * 2 + 16)) sz <<= 1;
    h->k = (uint64_t*)malloc(sz * sizeof(uint64_t));
    h->v = (int64_t*)malloc(sz * sizeof(int64_t));
    if (!h->k || !h->v) return -1;
    memset(h->k, 0xFF, sz * sizeof(uint64_t));
    h->mask = sz - 1; h->used = 0;
    return 0;
}
static void hm_free(hmap* h) { free(h->k); free(h->v); h->k = 0; h->v = 0; }
static inline uint64_t hm_slot(const hmap* h, uint64_t key) {
    uint64_t b = mix64(key ^ 0x5851F42D4C957F2DULL) & h->mask;
    while (h->k[b] != HEMPTY && h->k[b] != key) b = (b + 1) & h->mask;
    return b;
}
static int64_t* hm_find(hmap* h, uint64_t key) {
    uint64_t b = hm_slot(h, key);
    return h->k[b] == key ? &h->v[b] : NULL;
}
static int hm_grow(hmap* h);
/* returns 1 if inserted, 0 if present */
static int hm_put(hmap* h, uint64_t key, int64_t val) {
    if ((uint64_t)(h->used + 1) * 2 > h->mask + 1) hm_grow(h);
    uint64_t b = hm_slot(h, key);
    if (h->k[b] == key) return 0;
    h->k[b] = key; h->v[b] = val; h->used++;
    return 1;
}
static int hm_grow(hmap* h) {
    hmap n2;
    uint64_t sz = (h->mask + 1) * 2;
    n2.k = (uint64_t*)malloc(sz * sizeof(uint64_t));
    n2.v = (int64_t*)malloc(sz * sizeof(int64_t));
    if (!n2.k || !n2.v) return -1;
    memset(n2.k, 0xFF, sz * sizeof(uint64_t));
    n2.mask = sz - 1; n2.used = 0;
    for (uint64_t i = 0; i <= h->mask; i++)
        if (h->k[i] != HEMPTY) { uint64_t b = hm_slot(&n2, h->k[i]); n2.k[b] = h->k[i]; n2.v[b] = h->v[i]; n2.used++; }
    hm_free(h); *h = n2;
    return 0;
}
/* Deletion with backward-shift (linear probing), keeps probe chains intact. */
static void hm_del(hmap* h, uint64_t key) {
    uint64_t b = hm_slot(h, key);
    if (h->k[b] != key) return;
    uint64_t i = b;
    for (;;) {
        h->k[i] = HEMPTY;
        uint64_t j = i;
        for (;;) {
            j = (j + 1) & h->mask;
            if (h->k[j] == HEMPTY) { h->used--; return; }
            uint64_t home = mix64(h->k[j] ^ 0x5851F42D4C957F2DULL) & h->mask;
            /* can k[j] move to i?  yes unless home lies cyclically in (i, j] */
            int inside = (i <= j) ? (home > i && home <= j) : (home > i || home <= j);
            if (!inside) { h->k[i] = h->k[j]; h->v[i] = h->v[j]; i = j; break; }
        }
    }
}

/* ---------------- radix sort of u64 keys (LSD, 16-bit digits) ---------------- */
static int radix_sort_u64(uint64_t* a, int64_t n) {
    uint64_t* tmp = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    if (!tmp) return -1;
    int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
    uint64_t *src = a, *dst = tmp;
    for (int pass = 0; pass < 4; pass++) {
        int sh = pass * 16;
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < n; i++) cnt[(src[i] >> sh) & 0xFFFF]++;
        int single = 0;
        for (int d = 0; d < 65536; d++) if (cnt[d] == n) { single = 1; break; }
        if (single) continue;
        int64_t s = 0;
        for (int d = 0; d < 65536; d++) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < n; i++) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
    free(tmp); free(cnt);
    return 0;
}

/* ---------------- static graph families ---------------- */

/* Erdos-Renyi G(n, m): m distinct uniform pairs u != v, in draw order. */
int64_t sy_er(int32_t n, int64_t m, uint64_t seed, int32_t* out) {
    if (n < 2 || m < 0 || (double)m > (double)n * (n - 1) / 2) return -1;
    hmap h; if (hm_init(&h, m)) return -2;
    rng_t r = {seed, 0};
    int64_t got = 0;
    while (got < m) {
        int32_t u = (int32_t)below(rnext(&r), (uint64_t)n);
        int32_t v = (int32_t)below(rnext(&r), (uint64_t)n);
        if (u == v) continue;
        if (hm_put(&h, ekey(u, v), got)) { out[2 * got] = u; out[2 * got + 1] = v; got++; }
    }
    hm_free(&h);
    return got;
}

/* R-MAT (Chakrabarti, Zhan & Faloutsos 2004) with quadrant probabilities
 * a, b, c, d = 1-a-b-c, 2^scale vertices, nsamples sampled edges.  The
 * samples are symmetrised (undirected), self-loops and duplicates dropped,
 * and vertex ids relabelled by a seeded random permutation when permute != 0.
 * Output: canonical (lo < hi) pairs in increasing key order; returns m. */
int64_t sy_rmat(int32_t scale, int64_t nsamples, double a, double b, double c,
                uint64_t seed, int32_t permute, int32_t* out) {
    if (scale < 1 || scale > 30 || nsamples < 0) return -1;
    int64_t nv = (int64_t)1 << scale;
    int32_t* perm = (int32_t*)malloc((size_t)nv * sizeof(int32_t));
    uint64_t* keys = (uint64_t*)malloc((size_t)(nsamples > 0 ? nsamples : 1) * sizeof(uint64_t));
    if (!perm || !keys) { free(perm); free(keys); return -2; }
    for (int64_t i = 0; i < nv; i++) perm[i] = (int32_t)i;
    if (permute) {
        rng_t pr = {mix64(seed ^ 0xA0761D6478BD642FULL), 0};
        for (int64_t i = nv - 1; i > 0; i--) {
            int64_t j = (int64_t)below(rnext(&pr), (uint64_t)(i + 1));
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    }
    double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nsamples; i++) {
        uint64_t u = 0, v = 0;
        for (int l = 0; l < scale; l++) {
            double r = unit(draw(seed, (uint64_t)i * (uint64_t)scale + (uint64_t)l));
            int bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | (uint64_t)bu; v = (v << 1) | (uint64_t)bv;
        }
        int32_t pu = perm[u], pv = perm[v];
        keys[i] = (pu == pv) ? HEMPTY : ekey(pu, pv);
    }
    free(perm);
    if (radix_sort_u64(keys, nsamples)) { free(keys); return -2; }
    int64_t m = 0;
    for (int64_t i = 0; i < nsamples; i++) {
        if (keys[i] == HEMPTY) break;
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        out[2 * m] = (int32_t)(keys[i] >> 32); out[2 * m + 1] = (int32_t)(keys[i] & 0xFFFFFFFFu);
        m++;
    }
    free(keys);
    return m;
}

/* Barabasi-Albert: a seed clique on vertices 0..m, then each new vertex
 * v = m+1..n-1 attaches to m distinct earlier vertices chosen with
 * probability proportional to degree (uniform pick from the list of all
 * edge endpoints so far).  Output edge count m(m+1)/2 + (n-m-1)m. */
int64_t sy_ba(int32_t n, int32_t m, uint64_t seed, int32_t* out) {
    if (m < 1 || n < m + 1) return -1;
    int64_t E = (int64_t)m * (m + 1) / 2 + (int64_t)(n - m - 1) * m;
    int32_t* ends = (int32_t*)malloc((size_t)(2 * E) * sizeof(int32_t));
    if (!ends) return -2;
    int64_t ne = 0, nend = 0;
    for (int32_t i = 0; i <= m; i++)
        for (int32_t j = i + 1; j <= m; j++) {
            out[2 * ne] = i; out[2 * ne + 1] = j; ne++;
            ends[nend++] = i; ends[nend++] = j;
        }
    rng_t r = {seed, 0};
    int32_t tg[64];
    for (int32_t v = m + 1; v < n; v++) {
        int32_t k = 0;
        int64_t lim = nend;
        while (k < m) {
            int32_t t = ends[below(rnext(&r), (uint64_t)lim)];
            int dup = 0;
            for (int32_t q = 0; q < k; q++) if (tg[q] == t) { dup = 1; break; }
            if (!dup) tg[k++] = t;
        }
        for (int32_t q = 0; q < m; q++) {
            out[2 * ne] = tg[q]; out[2 * ne + 1] = v; ne++;
            ends[nend++] = tg[q]; ends[nend++] = v;
        }
    }
    free(ends);
    return ne;
}

/* side x side 4-neighbour grid (vertex r*side+c) plus nshort distinct
 * uniform random non-grid pairs. */
int64_t sy_grid(int32_t side, int64_t nshort, uint64_t seed, int32_t* out) {
    if (side < 2) return -1;
    int64_t n = (int64_t)side * side, ne = 0;
    hmap h; if (hm_init(&h, 2 * n + nshort)) return -2;
    for (int32_t r0 = 0; r0 < side; r0++)
        for (int32_t c0 = 0; c0 < side; c0++) {
            int32_t v = r0 * side + c0;
            if (c0 + 1 < side) { out[2 * ne] = v; out[2 * ne + 1] = v + 1; hm_put(&h, ekey(v, v + 1), ne); ne++; }
            if (r0 + 1 < side) { out[2 * ne] = v; out[2 * ne + 1] = v + side; hm_put(&h, ekey(v, v + side), ne); ne++; }
        }
    rng_t r = {seed, 0};
    int64_t got = 0;
    while (got < nshort) {
        int32_t u = (int32_t)below(rnext(&r), (uint64_t)n), v = (int32_t)below(rnext(&r), (uint64_t)n);
        if (u == v) continue;
        if (hm_put(&h, ekey(u, v), ne)) { out[2 * ne] = u; out[2 * ne + 1] = v; ne++; got++; }
    }
    hm_free(&h);
    return ne;
}

/* ---------------- dynamic edge-set model for update streams ----------------
 * Tracks the evolving vertex and edge sets so that batches of "new" edges
 * (not present) and "existing" edges (present) can be drawn, and so that
 * vertex insertions get the ids a dense append-only numbering assigns. */
typedef struct { int32_t w; int32_t e; } slot_t;   /* neighbour, edge index */
typedef struct {
    int32_t n, ncap;
    int8_t* alive;
    int32_t* deg; int32_t* cap; slot_t** adj;
    int32_t* live; int32_t* live_pos; int32_t nlive;
    uint64_t* ek; int32_t* epl; int32_t* eph; int64_t ne, ecap;  /* key, slot in adj[lo], slot in adj[hi] */
    hmap h;                                               /* key -> edge index */
} sy_dyn;

static int dyn_vgrow(sy_dyn* d, int32_t need) {
    if (need <= d->ncap) return 0;
    int32_t nc = d->ncap ? d->ncap : 16;
    while (nc < need) nc = nc + nc / 2 + 16;
    d->alive = (int8_t*)realloc(d->alive, (size_t)nc);
    d->deg = (int32_t*)realloc(d->deg, (size_t)nc * 4);
    d->cap = (int32_t*)realloc(d->cap, (size_t)nc * 4);
    d->adj = (slot_t**)realloc(d->adj, (size_t)nc * sizeof(slot_t*));
    d->live = (int32_t*)realloc(d->live, (size_t)nc * 4);
    d->live_pos = (int32_t*)realloc(d->live_pos, (size_t)nc * 4);
    if (!d->alive || !d->deg || !d->cap || !d->adj || !d->live || !d->live_pos) return -1;
    for (int32_t i = d->ncap; i < nc; i++) { d->alive[i] = 0; d->deg[i] = 0; d->cap[i] = 0; d->adj[i] = NULL; d->live_pos[i] = -1; }
    d->ncap = nc;
    return 0;
}
static void dyn_add_vertex(sy_dyn* d) {
    int32_t v = d->n++;
    dyn_vgrow(d, d->n);
    d->alive[v] = 1; d->live_pos[v] = d->nlive; d->live[d->nlive++] = v;
}
static void adj_push(sy_dyn* d, int32_t u, int32_t w, int32_t e, int32_t* pos) {
    if (d->deg[u] == d->cap[u]) {
        int32_t nc = d->cap[u] ? d->cap[u] * 2 : 4;
        d->adj[u] = (slot_t*)realloc(d->adj[u], (size_t)nc * sizeof(slot_t));
        d->cap[u] = nc;
    }
    *pos = d->deg[u];
    d->adj[u][d->deg[u]].w = w; d->adj[u][d->deg[u]].e = e; d->deg[u]++;
}
static inline void fix_slot(sy_dyn* d, int32_t u, int32_t p) {
    slot_t s = d->adj[u][p];
    if ((int32_t)(d->ek[s.e] >> 32) == u) d->epl[s.e] = p; else d->eph[s.e] = p;
}
static int dyn_insert(sy_dyn* d, int32_t u, int32_t v) {
    if (u == v || u < 0 || v < 0 || u >= d->n || v >= d->n || !d->alive[u] || !d->alive[v]) return 0;
    uint64_t k = ekey(u, v);
    if (hm_find(&d->h, k)) return 0;
    if (d->ne == d->ecap) {
        d->ecap = d->ecap ? d->ecap * 2 : 1024;
        d->ek = (uint64_t*)realloc(d->ek, (size_t)d->ecap * 8);
        d->epl = (int32_t*)realloc(d->epl, (size_t)d->ecap * 4);
        d->eph = (int32_t*)realloc(d->eph, (size_t)d->ecap * 4);
    }
    int64_t e = d->ne++;
    d->ek[e] = k;
    int32_t lo = (int32_t)(k >> 32), hi = (int32_t)(k & 0xFFFFFFFFu), p;
    adj_push(d, lo, hi, (int32_t)e, &p); d->epl[e] = p;
    adj_push(d, hi, lo, (int32_t)e, &p); d->eph[e] = p;
    hm_put(&d->h, k, e);
    return 1;
}
static void adj_remove(sy_dyn* d, int32_t u, int32_t p) {
    int32_t last = --d->deg[u];
    if (p != last) { d->adj[u][p] = d->adj[u][last]; fix_slot(d, u, p); }
}
static int dyn_delete(sy_dyn* d, int32_t u, int32_t v) {
    if (u == v || u < 0 || v < 0 || u >= d->n || v >= d->n) return 0;
    uint64_t k = ekey(u, v);
    int64_t* pe = hm_find(&d->h, k);
    if (!pe) return 0;
    int64_t e = *pe;
    int32_t lo = (int32_t)(k >> 32), hi = (int32_t)(k & 0xFFFFFFFFu);
    adj_remove(d, lo, d->epl[e]);
    adj_remove(d, hi, d->eph[e]);
    hm_del(&d->h, k);
    int64_t last = --d->ne;
    if (e != last) {
        d->ek[e] = d->ek[last]; d->epl[e] = d->epl[last]; d->eph[e] = d->eph[last];
        int32_t l2 = (int32_t)(d->ek[e] >> 32), h2 = (int32_t)(d->ek[e] & 0xFFFFFFFFu);
        d->adj[l2][d->epl[e]].e = (int32_t)e;
        d->adj[h2][d->eph[e]].e = (int32_t)e;
        *hm_find(&d->h, d->ek[e]) = e;
    }
    return 1;
}

sy_dyn* sy_dyn_create(int32_t n, int64_t m, const int32_t* edges) {
    sy_dyn* d = (sy_dyn*)calloc(1, sizeof(sy_dyn));
    if (!d) return NULL;
    if (hm_init(&d->h, m + 1024)) { free(d); return NULL; }
    dyn_vgrow(d, n > 0 ? n : 1);
    for (int32_t i = 0; i < n; i++) dyn_add_vertex(d);
    for (int64_t i = 0; i < m; i++) dyn_insert(d, edges[2 * i], edges[2 * i + 1]);
    return d;
}
void sy_dyn_free(sy_dyn* d) {
    if (!d) return;
    for (int32_t i = 0; i < d->ncap; i++) free(d->adj[i]);
    free(d->alive); free(d->deg); free(d->cap); free(d->adj); free(d->live); free(d->live_pos);
    free(d->ek); free(d->epl); free(d->eph); hm_free(&d->h); free(d);
}
int32_t sy_dyn_n(const sy_dyn* d) { return d->n; }
int64_t sy_dyn_m(const sy_dyn* d) { return d->ne; }
int32_t sy_dyn_nlive(const sy_dyn* d) { return d->nlive; }
int32_t sy_dyn_degree(const sy_dyn* d, int32_t v) { return (v >= 0 && v < d->n) ? d->deg[v] : -1; }

/* Current edge list (canonical lo<hi), in internal order; returns count. */
int64_t sy_dyn_edges(const sy_dyn* d, int32_t* out) {
    for (int64_t e = 0; e < d->ne; e++) { out[2 * e] = (int32_t)(d->ek[e] >> 32); out[2 * e + 1] = (int32_t)(d->ek[e] & 0xFFFFFFFFu); }
    return d->ne;
}
void sy_dyn_alive(const sy_dyn* d, int8_t* out) { memcpy(out, d->alive, (size_t)d->n); }

static int32_t pick_live(sy_dyn* d, rng_t* r) { return d->live[below(rnext(r), (uint64_t)d->nlive)]; }
static int32_t pick_pref(sy_dyn* d, rng_t* r) {      /* endpoint of a uniform edge: P(v) ~ deg(v) */
    uint64_t x = rnext(r);
    int64_t e = (int64_t)below(x, (uint64_t)d->ne);
    return (x & 1) ? (int32_t)(d->ek[e] >> 32) : (int32_t)(d->ek[e] & 0xFFFFFFFFu);
}

/* Draw `count` distinct new edges (absent from the graph, both endpoints
 * live, u != v).  mode 0: both endpoints uniform over live vertices;
 * mode 1: both endpoints degree-proportional.  Does not apply them.
 * Returns the number written (fewer only if the graph is nearly complete). */
int64_t sy_dyn_sample_insert(sy_dyn* d, int64_t count, int32_t mode, uint64_t seed, int32_t* out) {
    hmap b; if (hm_init(&b, count)) return -2;
    rng_t r = {seed, 0};
    int64_t got = 0, tries = 0, lim = 64 * count + 1024;
    while (got < count && tries < lim) {
        tries++;
        int32_t u, v;
        if (mode == 1 && d->ne > 0) { u = pick_pref(d, &r); v = pick_pref(d, &r); }
        else { if (d->nlive < 2) break; u = pick_live(d, &r); v = pick_live(d, &r); }
        if (u == v) continue;
        uint64_t k = ekey(u, v);
        if (hm_find(&d->h, k)) continue;
        if (hm_put(&b, k, got)) { out[2 * got] = u; out[2 * got + 1] = v; got++; }
    }
    hm_free(&b);
    return got;
}

/* Draw `count` distinct existing edges.  mode 0: a uniform live vertex with
 * degree > 0, then a uniform neighbour of it; mode 1: a uniform random edge
 * (both endpoints degree-proportional).  Does not apply them. */
int64_t sy_dyn_sample_delete(sy_dyn* d, int64_t count, int32_t mode, uint64_t seed, int32_t* out) {
    if (count > d->ne) count = d->ne;
    hmap b; if (hm_init(&b, count)) return -2;
    rng_t r = {seed, 0};
    int64_t got = 0, tries = 0, lim = 64 * count + 1024;
    while (got < count && tries < lim) {
        tries++;
        uint64_t k;
        int32_t u, v;
        if (mode == 1) {
            int64_t e = (int64_t)below(rnext(&r), (uint64_t)d->ne);
            k = d->ek[e]; u = (int32_t)(k >> 32); v = (int32_t)(k & 0xFFFFFFFFu);
            if (rnext(&r) & 1) { int32_t t = u; u = v; v = t; }
        } else {
            u = pick_live(d, &r);
            if (d->deg[u] == 0) continue;
            v = d->adj[u][below(rnext(&r), (uint64_t)d->deg[u])].w;
            k = ekey(u, v);
        }
        if (hm_put(&b, k, got)) { out[2 * got] = u; out[2 * got + 1] = v; got++; }
    }
    hm_free(&b);
    return got;
}

/* Apply a batch to the model: op 0 inserts (skipping present edges,
 * self-loops, dead or unknown ids), op 1 deletes (skipping absent edges).
 * Returns the number applied. */
int64_t sy_dyn_apply(sy_dyn* d, int32_t op, const int32_t* edges, int64_t k) {
    int64_t a = 0;
    for (int64_t i = 0; i < k; i++)
        a += op == 0 ? dyn_insert(d, edges[2 * i], edges[2 * i + 1]) : dyn_delete(d, edges[2 * i], edges[2 * i + 1]);
    return a;
}

/* Append `count` new vertices (ids n, n+1, ...), each joined to `degree`
 * distinct uniform live vertices that existed before this call; applies
 * them and writes the neighbour lists (count x degree) to out_nbrs. */
int64_t sy_dyn_add_vertices(sy_dyn* d, int32_t count, int32_t degree, uint64_t seed, int32_t* out_nbrs) {
    int32_t base = d->n, pool = d->nlive;
    if (pool < degree) return -1;
    int32_t* snapshot = (int32_t*)malloc((size_t)(pool > 0 ? pool : 1) * 4);
    memcpy(snapshot, d->live, (size_t)pool * 4);
    rng_t r = {seed, 0};
    for (int32_t i = 0; i < count; i++) dyn_add_vertex(d);
    for (int32_t i = 0; i < count; i++) {
        int32_t* nb = out_nbrs + (int64_t)i * degree;
        int32_t k = 0;
        while (k < degree) {
            int32_t w = snapshot[below(rnext(&r), (uint64_t)pool)];
            int dup = 0;
            for (int32_t q = 0; q < k; q++) if (nb[q] == w) { dup = 1; break; }
            if (!dup) nb[k++] = w;
        }
        for (int32_t q = 0; q < degree; q++) dyn_insert(d, base + i, nb[q]);
    }
    free(snapshot);
    return (int64_t)count * degree;
}

/* Choose `count` distinct uniform live vertices, delete their incident
 * edges and mark them dead (ids are not reused).  Writes the ids. */
int64_t sy_dyn_delete_vertices(sy_dyn* d, int32_t count, uint64_t seed, int32_t* out_ids) {
    rng_t r = {seed, 0};
    int32_t got = 0;
    while (got < count && d->nlive > 0) {
        int32_t v = pick_live(d, &r);
        while (d->deg[v] > 0) { int32_t w = d->adj[v][d->deg[v] - 1].w; dyn_delete(d, v, w); }
        d->alive[v] = 0;
        int32_t p = d->live_pos[v], lastv = d->live[--d->nlive];
        d->live[p] = lastv; d->live_pos[lastv] = p; d->live_pos[v] = -1;
        out_ids[got++] = v;
    }
    return got;
}

/* Incident edges of v (as pairs v, w) -- for callers that expand a vertex
 * deletion into edge deletions themselves. */
int64_t sy_dyn_incident(const sy_dyn* d, int32_t v, int32_t* out) {
    if (v < 0 || v >= d->n) return -1;
    for (int32_t i = 0; i < d->deg[v]; i++) { out[2 * i] = v; out[2 * i + 1] = d->adj[v][i].w; }
    return d->deg[v];
}

/* ---------------- batch samplers for a large static graph ----------------
 * For graphs too large for the dynamic model: `keys` are the graph's
 * canonical edge keys (lo << 32 | hi) sorted increasingly (sy_rmat's output
 * order), `edges` the same edges as pairs. */
static int key_present(const uint64_t* keys, int64_t m, uint64_t k) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo < m && keys[lo] == k;
}

/* New edges (absent from the graph, distinct, u != v).  law 0: endpoints
 * uniform in [0, n); law 1: endpoints degree-proportional (an endpoint of a
 * uniform edge). */
int64_t sy_static_sample_insert(const int32_t* edges, int64_t m, int32_t n, int64_t count, int32_t law,
                                uint64_t seed, int32_t* out) {
    uint64_t* keys = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!keys) return -2;
    for (int64_t i = 0; i < m; i++) keys[i] = ekey(edges[2 * i], edges[2 * i + 1]);
    int sorted = 1;
    for (int64_t i = 1; i < m && sorted; i++) if (keys[i] <= keys[i - 1]) sorted = 0;
    if (!sorted && radix_sort_u64(keys, m)) { free(keys); return -2; }
    hmap b; if (hm_init(&b, count)) { free(keys); return -2; }
    rng_t r = {seed, 0};
    int64_t got = 0, tries = 0, lim = 64 * count + 1024;
    while (got < count && tries < lim) {
        tries++;
        int32_t u, v;
        if (law == 1 && m > 0) {
            uint64_t x = rnext(&r), y = rnext(&r);
            int64_t e1 = (int64_t)below(x, (uint64_t)m), e2 = (int64_t)below(y, (uint64_t)m);
            u = (x & 1) ? edges[2 * e1] : edges[2 * e1 + 1];
            v = (y & 1) ? edges[2 * e2] : edges[2 * e2 + 1];
        } else {
            u = (int32_t)below(rnext(&r), (uint64_t)n);
            v = (int32_t)below(rnext(&r), (uint64_t)n);
        }
        if (u == v) continue;
        uint64_t k = ekey(u, v);
        if (key_present(keys, m, k)) continue;
        if (hm_put(&b, k, got)) { out[2 * got] = u; out[2 * got + 1] = v; got++; }
    }
    hm_free(&b);
    free(keys);
    return got;
}

/* Existing edges (distinct).  law 1: a uniform random edge (endpoints
 * degree-proportional); law 0: a uniform vertex with degree > 0, then a
 * uniform neighbour of it (needs the CSR row_off/adj of the graph). */
int64_t sy_static_sample_delete(const int32_t* edges, int64_t m, int32_t n, const int64_t* row_off,
                                const int32_t* adj, int64_t count, int32_t law, uint64_t seed, int32_t* out) {
    if (count > m) count = m;
    hmap b; if (hm_init(&b, count)) return -2;
    rng_t r = {seed, 0};
    int64_t got = 0, tries = 0, lim = 64 * count + 1024;
    while (got < count && tries < lim) {
        tries++;
        int32_t u, v;
        if (law == 1 || !row_off) {
            int64_t e = (int64_t)below(rnext(&r), (uint64_t)m);
            u = edges[2 * e]; v = edges[2 * e + 1];
        } else {
            u = (int32_t)below(rnext(&r), (uint64_t)n);
            int64_t d = row_off[u + 1] - row_off[u];
            if (d == 0) continue;
            v = adj[row_off[u] + (int64_t)below(rnext(&r), (uint64_t)d)];
        }
        uint64_t k = ekey(u, v);
        if (hm_put(&b, k, got)) { out[2 * got] = u; out[2 * got + 1] = v; got++; }
    }
    hm_free(&b);
    return got;
}

/* CSR (both directions) of an edge list: row_off has n+1 entries, adj 2m. */
int sy_csr(int32_t n, int64_t m, const int32_t* edges, int64_t* row_off, int32_t* adj) {
    memset(row_off, 0, (size_t)(n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < m; i++) { row_off[edges[2 * i] + 1]++; row_off[edges[2 * i + 1] + 1]++; }
    for (int32_t v = 0; v < n; v++) row_off[v + 1] += row_off[v];
    int64_t* fill = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!fill) return -2;
    memcpy(fill, row_off, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < m; i++) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        adj[fill[u]++] = v;
        adj[fill[v]++] = u;
    }
    free(fill);
    return 0;
}

/* ---------------- many Barabasi-Albert graphs with per-graph batches ----------------
 * Graph i (n = ns[i], attachment m = ms[i], seed gseeds[i]) is written at
 * edges + 2*eoff[i].  For round r and graph i (slot j = r*ng + i, so each
 * round's batches are contiguous in graph order) kins[j] distinct uniform
 * pairs absent from the generated graph go to ins + 2*ioff[j] and kdel[j]
 * distinct uniform edges of it to del + 2*doff[j] (seed bseeds[j]).  Every
 * round is drawn against the graph as generated.  Graphs run in parallel.
 * Returns 0, or -1 (bad arguments), -2 (memory), -3 (a batch could not be
 * filled). */
int sy_ba_many(int32_t ng, const int32_t* ns, const int32_t* ms, const uint64_t* gseeds, const int64_t* eoff,
               int32_t* edges, int32_t rounds, const int64_t* kins, const int64_t* kdel, const uint64_t* bseeds,
               const int64_t* ioff, const int64_t* doff, int32_t* ins, int32_t* del) {
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < ng; i++) {
        int32_t* e = edges + 2 * eoff[i];
        int64_t m = sy_ba(ns[i], ms[i], gseeds[i], e);
        if (m != eoff[i + 1] - eoff[i]) {
#pragma omp atomic write
            status = -1;
            continue;
        }
        uint64_t* keys = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
        if (!keys) {
#pragma omp atomic write
            status = -2;
            continue;
        }
        for (int64_t q = 0; q < m; q++) keys[q] = ekey(e[2 * q], e[2 * q + 1]);
        if (radix_sort_u64(keys, m)) {
            free(keys);
#pragma omp atomic write
            status = -2;
            continue;
        }
        for (int32_t r = 0; r < rounds; r++) {
            const int64_t j = (int64_t)r * ng + i;
            rng_t g = {bseeds[j], 0};
            hmap b;
            if (hm_init(&b, kins[j] + kdel[j])) {
#pragma omp atomic write
                status = -2;
                break;
            }
            int32_t* oi = ins + 2 * ioff[j];
            int64_t got = 0, tries = 0, lim = 64 * kins[j] + 1024;
            while (got < kins[j] && tries++ < lim) {
                int32_t u = (int32_t)below(rnext(&g), (uint64_t)ns[i]);
                int32_t v = (int32_t)below(rnext(&g), (uint64_t)ns[i]);
                if (u == v) continue;
                uint64_t k = ekey(u, v);
                if (key_present(keys, m, k)) continue;
                if (hm_put(&b, k, got)) { oi[2 * got] = u; oi[2 * got + 1] = v; got++; }
            }
            int32_t* od = del + 2 * doff[j];
            int64_t gd = 0;
            tries = 0;
            lim = 64 * kdel[j] + 1024;
            while (gd < kdel[j] && m > 0 && tries++ < lim) {
                int64_t q = (int64_t)below(rnext(&g), (uint64_t)m);
                if (hm_put(&b, ~ekey(e[2 * q], e[2 * q + 1]), gd)) {   /* own key space: never an insert key */
                    od[2 * gd] = e[2 * q];
                    od[2 * gd + 1] = e[2 * q + 1];
                    gd++;
                }
            }
            hm_free(&b);
            if (got < kins[j] || gd < kdel[j]) {
#pragma omp atomic write
                status = -3;
            }
        }
        free(keys);
    }
    return status;
}
