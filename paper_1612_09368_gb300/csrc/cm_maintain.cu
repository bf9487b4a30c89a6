// cm_maintain.cu -- batch ingest and the persistent maintenance kernel.
//
// One launch of maintain_kernel runs every iteration of SuperiorEdgeInsert
// (Algorithm 1) or SuperiorEdgeDelete (Algorithm 5) for one batch.  Each
// iteration:
//   SELECT   a maximal superior edge set (Section IV, Definition 6 and the
//            union after it; Algorithm 2 made deterministic): an edge's
//            constrained endpoints are those whose core equals the edge's
//            core number min(core(u), core(v)); in claim rounds every
//            eligible edge writes its priority fmix64(key) into its
//            constrained endpoints with atomicMin, and wins when it holds
//            all of them.  Winners take their endpoints; edges touching a
//            taken endpoint are blocked until the next iteration.  The result
//            is the greedy (lexicographically first) maximal set in priority
//            order.
//   APPLY    insert / delete the selected edges in the slack CSR and move
//            SD (the superior degree, Definition 7) of constrained endpoints.
//   insert:  DISCOVER the candidate sets of all levels at once (the exKPT of
//            Definition 10, traversed breadth-first instead of depth-first):
//            from the constrained endpoints, through vertices w with
//            core(w) = k and SD(w) > k, expanding only from vertices whose
//            CSD (Definition 8) exceeds k.  Each vertex's support starts at
//            CSD.  EVICT in waves: a vertex whose support is <= k can not
//            rise (Lemma 8); it takes one support from every core-k visited
//            neighbour, which is evicted when its support falls to k
//            (InsertRemove, Algorithm 4).  Survivors rise by one (Algorithm 1
//            line 7, Lemma 7).
//   delete:  EVICT in waves from the constrained endpoints whose SD fell
//            below k (Algorithm 6); an evicted vertex takes one from the
//            support (initially SD) of every core-k neighbour, which is
//            evicted when its support falls below k (DeleteRemove,
//            Algorithm 7).  Evicted vertices drop by one (Algorithm 5 line 7).
//   COMMIT   move the cores, recompute SD of moved vertices and adjust SD of
//            their unmoved neighbours whose core equals the moved vertex's
//            new core (insert) or old core (delete).
// All levels run together on the cores of the iteration's start: a vertex
// only ever meets neighbours of its own level in discovery and eviction.
#include <cstdio>

#include "cm_common.cuh"
#include "cm_launch.h"

namespace cm {

// ------------------------------------------------------------------ ingest
__global__ void ingest_a_kernel(const int32_t* __restrict__ E, long long k, DevGraph g, BSet* bs,
                                unsigned long long bmask, Ctl* c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    int32_t u = E[2 * i], v = E[2 * i + 1];
    if (u < 0 || v < 0 || u >= g.n || v >= g.n || g.hs[u].x < 0 || g.hs[v].x < 0) {
        atomicMin(&c->bad_index, i);
        atomicCAS(&c->error, 0, E_INVALID);
        return;
    }
    if (u == v) return;
    unsigned long long key = ekey(u, v);
    unsigned long long b = fmix64(key) & bmask;
    for (unsigned long long p = 0; p <= bmask; p++) {
        unsigned long long kk = bs[b].key;
        if (kk == KEY_EMPTY) {
            unsigned long long old = atomicCAS(&bs[b].key, KEY_EMPTY, key);
            if (old == KEY_EMPTY || old == key) { atomicMin(&bs[b].pos, (uint32_t)i); return; }
        } else if (kk == key) {
            atomicMin(&bs[b].pos, (uint32_t)i);
            return;
        }
        b = (b + 1) & bmask;
    }
}

__global__ void ingest_b_kernel(const int32_t* __restrict__ E, long long k, int op, DevGraph g,
                                const BSet* __restrict__ bs, unsigned long long bmask, REdge* R0, int32_t* ovl,
                                Ctl* c) {
    if (vload32(&c->error)) return;   // uniform: the flag is final before this kernel starts
    long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; base < k; base += stride) {
        long long i = base + lane_id();
        bool keep = false;
        REdge r = {0, 0, 0, 0};
        bool ov_lo = false, ov_hi = false;
        if (i < k) {
            int32_t u = E[2 * i], v = E[2 * i + 1];
            if (u != v) {
                unsigned long long key = ekey(u, v);
                unsigned long long b = fmix64(key) & bmask;
                unsigned long long probe = 0;
                while (bs[b].key != key && probe <= bmask) {   // present: ingest_a put it there
                    b = (b + 1) & bmask;
                    probe++;
                }
                if (probe <= bmask && bs[b].pos == (uint32_t)i) {
                    int32_t lo = min(u, v), hi = max(u, v);
                    if (op == 0) {
                        bool existed = false;
                        long long bk = idx_insert(g.idx, g.idx_mask, key, &existed);
                        if (bk < 0) {
                            atomicCAS(&c->error, 0, E_INDEX_FULL);
                        } else if (!existed) {
                            g.idx[bk].slo = -2;
                            g.idx[bk].shi = -2;
                            keep = true;
                            r.lo = lo; r.hi = hi; r.bkt = (uint32_t)bk; r.flags = 0;
                            int a = atomicAdd(&g.need[lo], 1);
                            int el = g.end[lo], cl = g.cap[lo];
                            ov_lo = (el + a + 1 > cl) && (el + a <= cl);
                            int bb = atomicAdd(&g.need[hi], 1);
                            int eh = g.end[hi], ch = g.cap[hi];
                            ov_hi = (eh + bb + 1 > ch) && (eh + bb <= ch);
                        }
                    } else {
                        long long bk = idx_find(g.idx, g.idx_mask, key);
                        if (bk >= 0) {
                            keep = true;
                            r.lo = lo; r.hi = hi; r.bkt = (uint32_t)bk; r.flags = 0;
                        }
                    }
                }
            }
        }
        warp_push_edge(&c->nrem, R0, keep, r);
        warp_push(&c->noverflow, ovl, ~0ull, ov_lo, r.lo);
        warp_push(&c->noverflow, ovl, ~0ull, ov_hi, r.hi);
    }
}

cudaError_t ingest_a(const int32_t* E, long long k, DevGraph g, BSet* bs, unsigned long long bmask, Ctl* c,
                     cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    int t = 256;
    long long b = (k + t - 1) / t;
    ingest_a_kernel<<<(unsigned)b, t, 0, s>>>(E, k, g, bs, bmask, c);
    return cudaGetLastError();
}

cudaError_t ingest_b(const int32_t* E, long long k, int op, DevGraph g, const BSet* bs, unsigned long long bmask,
                     REdge* R0, int32_t* ovl, Ctl* c, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    int t = 256;
    long long b = (k + t - 1) / t;
    if (b > 4096) b = 4096;
    ingest_b_kernel<<<(unsigned)b, t, 0, s>>>(E, k, op, g, bs, bmask, R0, ovl, c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ relocation
// Vertices whose capacity a batch would exceed move to fresh space at the
// end of the adjacency pool, compacting their holes; the index learns the
// new slots.  Space is left as garbage at the old place.
__global__ void reloc_size_kernel(const int32_t* ovl, long long novl, DevGraph g, Ctl* c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= novl) return;
    int x = ovl[i];
    int nc = cap_for((long long)g.deg[x] + g.need[x], g.slack_pct, g.min_cap);
    atomicAdd(&c->reloc_need, (unsigned long long)nc);
}

__global__ void relocate_kernel(const int32_t* ovl, long long novl, DevGraph g, Ctl* c) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < novl; w += nw) {
        int x = ovl[w];
        int nc = cap_for((long long)g.deg[x] + g.need[x], g.slack_pct, g.min_cap);
        unsigned long long nb = 0;
        if (lane == 0) nb = atomicAdd(&c->adj_top, (unsigned long long)nc);
        nb = __shfl_sync(0xffffffffu, nb, 0);
        if ((long long)nb + nc > g.adj_cap) {       // host sized the pool; never expected
            if (lane == 0) atomicCAS(&c->error, 0, E_CAPACITY);
            continue;
        }
        long long o = g.off[x];
        int len = g.end[x];
        int outp = 0;
        for (int j0 = 0; j0 < len; j0 += 32) {
            int j = j0 + lane;
            int y = j < len ? g.adj[o + j] : HOLE;
            bool live = y >= 0;
            unsigned int b = __ballot_sync(0xffffffffu, live);
            int p = outp + __popc(b & ((1u << lane) - 1));
            if (live) {
                g.adj[nb + p] = y;
                long long bk = idx_find(g.idx, g.idx_mask, ekey(x, y));
                if (bk >= 0) {
                    if (x < y) g.idx[bk].slo = p; else g.idx[bk].shi = p;
                }
            }
            outp += __popc(b);
        }
        if (lane == 0) {
            g.off[x] = (int64_t)nb;
            g.end[x] = outp;
            g.cap[x] = nc;
        }
    }
}

__global__ void clear_need_kernel(const REdge* R, long long n, DevGraph g) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    g.need[R[i].lo] = 0;
    g.need[R[i].hi] = 0;
}

cudaError_t reloc_size(const int32_t* ovl, long long novl, DevGraph g, Ctl* c, cudaStream_t s) {
    if (novl <= 0) return cudaSuccess;
    reloc_size_kernel<<<(unsigned)((novl + 255) / 256), 256, 0, s>>>(ovl, novl, g, c);
    return cudaGetLastError();
}
cudaError_t relocate(const int32_t* ovl, long long novl, DevGraph g, Ctl* c, cudaStream_t s) {
    if (novl <= 0) return cudaSuccess;
    long long blocks = (novl * 32 + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    relocate_kernel<<<(unsigned)blocks, 256, 0, s>>>(ovl, novl, g, c);
    return cudaGetLastError();
}
cudaError_t clear_need(const REdge* R, long long n, DevGraph g, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    clear_need_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, n, g);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ structure-only apply
// Applies every kept edge of a batch to the CSR at once, without touching
// core numbers or SD: the first half of the full re-peel comparator.
__global__ void apply_structure_kernel(const REdge* __restrict__ R, long long n, int op, DevGraph g, Ctl* c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    REdge E = R[i];
    if (op == 0) {
        int pu = atomicAdd(&g.end[E.lo], 1), pv = atomicAdd(&g.end[E.hi], 1);
        if (pu < g.cap[E.lo] && pv < g.cap[E.hi]) {
            g.adj[g.off[E.lo] + pu] = E.hi;
            g.adj[g.off[E.hi] + pv] = E.lo;
            g.idx[E.bkt].slo = pu;
            g.idx[E.bkt].shi = pv;
        } else {
            atomicCAS(&c->error, 0, E_CAPACITY);
        }
        atomicAdd(&g.deg[E.lo], 1);
        atomicAdd(&g.deg[E.hi], 1);
    } else {
        Bucket b = g.idx[E.bkt];
        if (b.slo >= 0 && b.slo < g.end[E.lo] && b.shi >= 0 && b.shi < g.end[E.hi]) {
            g.adj[g.off[E.lo] + b.slo] = HOLE;
            g.adj[g.off[E.hi] + b.shi] = HOLE;
        } else {
            atomicCAS(&c->error, 0, E_CAPACITY);
        }
        g.idx[E.bkt].key = KEY_TOMB;
        atomicSub(&g.deg[E.lo], 1);
        atomicSub(&g.deg[E.hi], 1);
    }
}

cudaError_t apply_structure(const REdge* R, long long n, int op, DevGraph g, Ctl* c, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    apply_structure_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, n, op, g, c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ maintenance kernel
struct LocalStats {
    long long vis = 0, visl = 0, ev = 0, evl = 0, ch = 0, chl = 0, sel = 0;
};

__device__ __forceinline__ void edge_level(const DevGraph& g, const REdge& E, int& k, bool& clo, bool& chi) {
    int a = g.hs[E.lo].x, b = g.hs[E.hi].x;
    k = min(a, b);
    clo = a == k;
    chi = b == k;
}

// Selection, claim phase of round r.
__device__ __forceinline__ void claim_edge(const DevGraph& g, REdge* R, long long i, int r, uint32_t e) {
    REdge E = R[i];
    int k; bool clo, chi;
    edge_level(g, E, k, clo, chi);
    uint32_t f = E.flags;
    if ((f >> 2) == (uint32_t)r && r > 0) {   // claimed in round r-1: clear that buffer
        unsigned long long* cb = ((r - 1) & 1) ? g.claim1 : g.claim0;
        if (clo) cb[E.lo] = CLAIM_FREE;
        if (chi) cb[E.hi] = CLAIM_FREE;
    }
    if (f & (F_SEL | F_BLK)) return;
    if ((clo && g.taken[E.lo] == e) || (chi && g.taken[E.hi] == e)) {
        R[i].flags = f | F_BLK;
        return;
    }
    unsigned long long prio = fmix64(ekey(E.lo, E.hi));
    unsigned long long* cb = (r & 1) ? g.claim1 : g.claim0;
    if (clo) atomicMin(&cb[E.lo], prio);
    if (chi) atomicMin(&cb[E.hi], prio);
    R[i].flags = (f & 3u) | ((uint32_t)(r + 1) << 2);
}

// Selection, check phase of round r.  Returns 1 if the edge claimed and lost.
__device__ __forceinline__ int check_edge(const DevGraph& g, REdge* R, long long i, int r, uint32_t e,
                                          long long& nsel) {
    REdge E = R[i];
    if ((E.flags >> 2) != (uint32_t)(r + 1)) return 0;
    int k; bool clo, chi;
    edge_level(g, E, k, clo, chi);
    unsigned long long prio = fmix64(ekey(E.lo, E.hi));
    const unsigned long long* cb = (r & 1) ? g.claim1 : g.claim0;
    bool win = (!clo || cb[E.lo] == prio) && (!chi || cb[E.hi] == prio);
    if (!win) return 1;
    R[i].flags = E.flags | F_SEL;
    if (clo) g.taken[E.lo] = e;
    if (chi) g.taken[E.hi] = e;
    nsel++;
    return 0;
}

__global__ void __launch_bounds__(512) maintain_kernel(MaintainParams P) {
    Ctl* C = P.ctl;
    const DevGraph g = P.g;
    const int lane = lane_id();
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long qm = P.qmask;
    LocalStats ls;
    REdge* Rc = P.R0;
    REdge* Rn = P.R1;
    unsigned long long nrem = P.nrem0;
    uint32_t e = P.epoch0;
    unsigned long long vq_t = 0, eq_t = 0, cq_t = 0;
    long long iters = 0, rounds = 0, waves = 0, remsum = 0;
    bool ok = true;

    while (nrem > 0) {
        if (iters >= P.max_iters) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&C->error, 0, E_ITER_LIMIT);
            break;
        }
        remsum += (long long)nrem;
        // ------------------------------------------------ SELECT
        int r = 0;
        for (;;) {
            for (long long base = gwarp * 32; base < (long long)nrem; base += nwarps * 32) {
                long long i = base + lane;
                if (i < (long long)nrem) claim_edge(g, Rc, i, r, e);
            }
            if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
            int lost = 0;
            for (long long base = gwarp * 32; base < (long long)nrem; base += nwarps * 32) {
                long long i = base + lane;
                if (i < (long long)nrem) lost += check_edge(g, Rc, i, r, e, ls.sel);
            }
            lost = warp_sum(lost);
            if (lane == 0 && lost) atomicAdd(&C->pc[0], (unsigned long long)lost);
            if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
            r++;
            if (vload64(&C->spc[0]) == 0) break;
        }
        if (!ok) break;
        rounds += r;
        // ------------------------------------------------ APPLY
        const unsigned long long vq0 = vq_t, eq0 = eq_t, cq0 = cq_t;
        for (long long base = gwarp * 32; base < (long long)nrem; base += nwarps * 32) {
            long long i = base + lane;
            bool valid = i < (long long)nrem;
            REdge E = {0, 0, 0, 0};
            bool sel = false, s_lo = false, s_hi = false;
            if (valid) {
                E = Rc[i];
                int k; bool clo, chi;
                edge_level(g, E, k, clo, chi);
                if ((E.flags >> 2) == (uint32_t)r) {     // claimed in the final round
                    unsigned long long* cb = ((r - 1) & 1) ? g.claim1 : g.claim0;
                    if (clo) cb[E.lo] = CLAIM_FREE;
                    if (chi) cb[E.hi] = CLAIM_FREE;
                }
                sel = (E.flags & F_SEL) != 0;
                if (sel) {
                    if (P.op == 0) {
                        int pu = atomicAdd(&g.end[E.lo], 1), pv = atomicAdd(&g.end[E.hi], 1);
                        if (pu < g.cap[E.lo] && pv < g.cap[E.hi]) {
                            g.adj[g.off[E.lo] + pu] = E.hi;
                            g.adj[g.off[E.hi] + pv] = E.lo;
                            g.idx[E.bkt].slo = pu;
                            g.idx[E.bkt].shi = pv;
                        } else {
                            atomicCAS(&C->error, 0, E_CAPACITY);
                        }
                        atomicAdd(&g.deg[E.lo], 1);
                        atomicAdd(&g.deg[E.hi], 1);
                        if (clo) {
                            int m = atomicAdd(&g.hs[E.lo].y, 1) + 1;
                            s_lo = m > k && atomicExch((unsigned int*)&g.hs[E.lo].z, e) != e;
                        }
                        if (chi) {
                            int m = atomicAdd(&g.hs[E.hi].y, 1) + 1;
                            s_hi = m > k && atomicExch((unsigned int*)&g.hs[E.hi].z, e) != e;
                        }
                    } else {
                        Bucket b = g.idx[E.bkt];
                        if (b.slo >= 0 && b.slo < g.end[E.lo] && b.shi >= 0 && b.shi < g.end[E.hi]) {
                            g.adj[g.off[E.lo] + b.slo] = HOLE;
                            g.adj[g.off[E.hi] + b.shi] = HOLE;
                        } else {
                            atomicCAS(&C->error, 0, E_CAPACITY);
                        }
                        g.idx[E.bkt].key = KEY_TOMB;
                        atomicSub(&g.deg[E.lo], 1);
                        atomicSub(&g.deg[E.hi], 1);
                        if (clo) {
                            int m = atomicSub(&g.hs[E.lo].y, 1) - 1;
                            if (m < k) { s_lo = true; g.chg[E.lo] = e; }
                        }
                        if (chi) {
                            int m = atomicSub(&g.hs[E.hi].y, 1) - 1;
                            if (m < k) { s_hi = true; g.chg[E.hi] = e; }
                        }
                    }
                }
                E.flags = 0;
            }
            warp_push_edge(&C->pc[1], Rn, valid && !sel, E);
            unsigned long long* qt = P.op == 0 ? &C->tail[0] : &C->tail[1];
            int32_t* q = P.op == 0 ? P.VQ : P.EQ;
            warp_push(qt, q, qm, s_lo, E.lo);
            warp_push(qt, q, qm, s_hi, E.hi);
        }
        if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
        const unsigned long long nrem_next = vload64(&C->spc[1]);
        vq_t = vload64(&C->stail[0]);
        eq_t = vload64(&C->stail[1]);

        if (P.op == 0) {
            // -------------------------------------------- DISCOVER (insert)
            unsigned long long lo = vq0, hi = vq_t;
            while (hi > lo) {
                waves++;
                const unsigned long long cnt = hi - lo;
                for (;;) {
                    unsigned long long j = 0;
                    if (lane == 0) j = atomicAdd(&C->pc[2], 1ull);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (j >= cnt) break;
                    const int v = P.VQ[(lo + j) & qm];
                    const int k = g.hs[v].x;
                    const long long o = g.off[v];
                    const int len = g.end[v];
                    int pcd = 0;
                    for (int t = lane; t < len; t += 32) {
                        int w = g.adj[o + t];
                        if (w >= 0) {
                            int4 hw = g.hs[w];
                            pcd += (hw.x > k) || (hw.x == k && hw.y > k);
                        }
                    }
                    pcd = warp_sum(pcd);
                    if (lane == 0) {
                        g.hs[v].w = pcd;
                        ls.vis++;
                        ls.visl += len;
                    }
                    if (pcd > k) {
                        for (int t0 = 0; t0 < len; t0 += 32) {
                            int t = t0 + lane;
                            int w = t < len ? g.adj[o + t] : HOLE;
                            bool p = false;
                            if (w >= 0) {
                                int4 hw = g.hs[w];
                                if (hw.x == k && hw.y > k && (uint32_t)hw.z != e)
                                    p = atomicExch((unsigned int*)&g.hs[w].z, e) != e;
                            }
                            warp_push(&C->tail[0], P.VQ, qm, p, w);
                        }
                    } else {
                        warp_push(&C->tail[1], P.EQ, qm, lane == 0, v);
                    }
                }
                if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
                lo = hi;
                hi = vload64(&C->stail[0]);
            }
            if (!ok) break;
            vq_t = hi;
            // -------------------------------------------- EVICT (insert)
            lo = eq0;
            hi = vload64(&C->stail[1]);
            while (hi > lo) {
                waves++;
                const unsigned long long cnt = hi - lo;
                for (;;) {
                    unsigned long long j = 0;
                    if (lane == 0) j = atomicAdd(&C->pc[2], 1ull);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (j >= cnt) break;
                    const int v = P.EQ[(lo + j) & qm];
                    const int k = g.hs[v].x;
                    const long long o = g.off[v];
                    const int len = g.end[v];
                    for (int t0 = 0; t0 < len; t0 += 32) {
                        int t = t0 + lane;
                        int w = t < len ? g.adj[o + t] : HOLE;
                        bool p = false;
                        if (w >= 0) {
                            int4 hw = g.hs[w];
                            if (hw.x == k && (uint32_t)hw.z == e && hw.w > k) p = atomicSub(&g.hs[w].w, 1) == k + 1;
                        }
                        warp_push(&C->tail[1], P.EQ, qm, p, w);
                    }
                    if (lane == 0) {
                        ls.ev++;
                        ls.evl += len;
                    }
                }
                if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
                lo = hi;
                hi = vload64(&C->stail[1]);
            }
            if (!ok) break;
            eq_t = hi;
            // -------------------------------------------- COMMIT A (insert): survivors rise
            for (long long base = gwarp * 32; base < (long long)(vq_t - vq0); base += nwarps * 32) {
                long long i = base + lane;
                bool up = false;
                int v = 0;
                if (i < (long long)(vq_t - vq0)) {
                    v = P.VQ[(vq0 + i) & qm];
                    int4 h = g.hs[v];
                    if (h.w > h.x) {
                        g.hs[v].x = h.x + 1;
                        g.chg[v] = e;
                        up = true;
                    }
                }
                warp_push(&C->tail[2], P.CQ, qm, up, v);
            }
            if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
            cq_t = vload64(&C->stail[2]);
            // -------------------------------------------- COMMIT B (insert): SD fix-up
            {
                const unsigned long long cnt = cq_t - cq0;
                for (;;) {
                    unsigned long long j = 0;
                    if (lane == 0) j = atomicAdd(&C->pc[2], 1ull);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (j >= cnt) break;
                    const int v = P.CQ[(cq0 + j) & qm];
                    const int kn = g.hs[v].x;
                    const long long o = g.off[v];
                    const int len = g.end[v];
                    int sd = 0;
                    for (int t = lane; t < len; t += 32) {
                        int w = g.adj[o + t];
                        if (w >= 0) {
                            int cw = g.hs[w].x;
                            sd += cw >= kn;
                            if (cw == kn && g.chg[w] != e) atomicAdd(&g.hs[w].y, 1);
                        }
                    }
                    sd = warp_sum(sd);
                    if (lane == 0) {
                        g.hs[v].y = sd;
                        ls.ch++;
                        ls.chl += len;
                    }
                }
            }
            if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
        } else {
            // -------------------------------------------- EVICT (delete)
            unsigned long long lo = eq0, hi = eq_t;
            while (hi > lo) {
                waves++;
                const unsigned long long cnt = hi - lo;
                for (;;) {
                    unsigned long long j = 0;
                    if (lane == 0) j = atomicAdd(&C->pc[2], 1ull);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (j >= cnt) break;
                    const int v = P.EQ[(lo + j) & qm];
                    const int k = g.hs[v].x;
                    const long long o = g.off[v];
                    const int len = g.end[v];
                    for (int t0 = 0; t0 < len; t0 += 32) {
                        int t = t0 + lane;
                        int w = t < len ? g.adj[o + t] : HOLE;
                        bool p = false;
                        if (w >= 0) {
                            int4 hw = g.hs[w];
                            // live support of w is SD(w) - (evicted neighbours so far); w leaves
                            // when it first drops below k, i.e. when the count reaches SD-k+1.
                            const int thr = hw.y - k + 1;
                            bool done = thr <= 0 || ((uint32_t)hw.z == e && hw.w >= thr);
                            if (hw.x == k && !done) {
                                unsigned long long* pw = (unsigned long long*)&g.hs[w].z;
                                unsigned long long old = vload64(pw);
                                uint32_t cntw = 0;
                                for (int tries = 0; tries < (1 << 22); tries++) {
                                    uint32_t oe = (uint32_t)old, oc = (uint32_t)(old >> 32);
                                    cntw = (oe == e) ? oc + 1 : 1;
                                    unsigned long long nw = ((unsigned long long)cntw << 32) | e;
                                    unsigned long long prev = atomicCAS(pw, old, nw);
                                    if (prev == old) break;
                                    old = prev;
                                    cntw = 0;
                                }
                                if (cntw == 0) atomicCAS(&C->error, 0, E_ITER_LIMIT);
                                p = (int)cntw == thr;
                                if (p) g.chg[w] = e;
                            }
                        }
                        warp_push(&C->tail[1], P.EQ, qm, p, w);
                    }
                    if (lane == 0) {
                        ls.ev++;
                        ls.evl += len;
                    }
                }
                if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
                lo = hi;
                hi = vload64(&C->stail[1]);
            }
            if (!ok) break;
            eq_t = hi;
            // -------------------------------------------- COMMIT A (delete): evicted drop
            for (long long i = gwarp * 32 + lane; i < (long long)(eq_t - eq0); i += nwarps * 32) {
                int v = P.EQ[(eq0 + i) & qm];
                g.hs[v].x -= 1;
            }
            if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
            // -------------------------------------------- COMMIT B (delete): SD fix-up
            {
                const unsigned long long cnt = eq_t - eq0;
                for (;;) {
                    unsigned long long j = 0;
                    if (lane == 0) j = atomicAdd(&C->pc[2], 1ull);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (j >= cnt) break;
                    const int v = P.EQ[(eq0 + j) & qm];
                    const int kn = g.hs[v].x;
                    const long long o = g.off[v];
                    const int len = g.end[v];
                    int sd = 0;
                    for (int t = lane; t < len; t += 32) {
                        int w = g.adj[o + t];
                        if (w >= 0) {
                            int cw = g.hs[w].x;
                            sd += cw >= kn;
                            if (cw == kn + 1 && g.chg[w] != e) atomicSub(&g.hs[w].y, 1);
                        }
                    }
                    sd = warp_sum(sd);
                    if (lane == 0) {
                        g.hs[v].y = sd;
                        ls.ch++;
                        ls.chl += len;
                    }
                }
            }
            if (!(ok = grid_sync(C, P.expect, P.limit_ns))) break;
        }
        REdge* t = Rc;
        Rc = Rn;
        Rn = t;
        nrem = nrem_next;
        e++;
        iters++;
    }
    (void)cq_t;
    // flush statistics: one atomic per warp
    if (lane == 0) {
        if (ls.vis) atomicAdd(&C->st[ST_VISITED], (unsigned long long)ls.vis);
        if (ls.visl) atomicAdd(&C->st[ST_VISSLOTS], (unsigned long long)ls.visl);
        if (ls.ev) atomicAdd(&C->st[ST_EVICTED], (unsigned long long)ls.ev);
        if (ls.evl) atomicAdd(&C->st[ST_EVSLOTS], (unsigned long long)ls.evl);
        if (ls.ch) atomicAdd(&C->st[ST_CHANGED], (unsigned long long)ls.ch);
        if (ls.chl) atomicAdd(&C->st[ST_CHSLOTS], (unsigned long long)ls.chl);
    }
    long long sel = ls.sel;
    for (int o = 16; o > 0; o >>= 1) sel += __shfl_xor_sync(0xffffffffu, sel, o);
    if (lane == 0 && sel) atomicAdd(&C->st[ST_SELECTED], (unsigned long long)sel);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        C->st[ST_ITERS] = (unsigned long long)iters;
        C->st[ST_ROUNDS] = (unsigned long long)rounds;
        C->st[ST_WAVES] = (unsigned long long)waves;
        C->st[ST_REMSUM] = (unsigned long long)remsum;
        C->wc = e;
    }
}

int maintain_blocks_per_sm(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, maintain_kernel, threads, 0) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_maintain(const MaintainParams& p, int blocks, int threads, cudaStream_t s) {
    MaintainParams q = p;
    void* args[] = {&q};
    return cudaLaunchCooperativeKernel((const void*)maintain_kernel, dim3(blocks), dim3(threads), args, 0, s);
}

}  // namespace cm
