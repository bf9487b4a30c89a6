// cm_maintain.cu -- batch ingest (validate, canonicalise, dedupe against the
// batch and the edge index), relocation of vertices whose slack a batch
// exceeds, and the structure-only apply used by the re-peel comparator.
// The superior-edge-set iterations themselves are in cm_iterate.cu.
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

}  // namespace cm
