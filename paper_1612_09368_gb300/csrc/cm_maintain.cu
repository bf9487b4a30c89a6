// cm_maintain.cu -- batch ingest (validate, canonicalise, dedupe against the
// batch and the edge index), relocation of vertices whose slack a batch
// exceeds, and the structure-only apply used by the re-peel comparator.
// The superior-edge-set iterations themselves are in cm_iterate.cu.
#include <cstddef>
#include <cstdio>

#include "cm_common.cuh"
#include "cm_launch.h"

namespace cm {

// Kernels of the update path take their item count either from the host
// (k) or, inside a captured update step, from device memory (kp != NULL,
// k then being the capacity the grid was sized for), and a captured step
// skips its remaining kernels once Ctl::defer is set.
__device__ __forceinline__ long long item_count(long long k, const unsigned long long* kp) {
    return kp ? (long long)vload64(kp) : k;
}

// ------------------------------------------------------------------ control block
// One launch instead of a row of small memsets and copies before a call's
// kernels: the host-exchange words ingest fills (error, kept and overflow
// counts, smallest bad position), and, before the maintenance launches, the
// barrier words, ring tails, counters and timers, plus the resume record
// the first launch reads.  take_nrem: the remaining-edge count is the one
// ingest left in the control block (the host did not read it back).
__global__ void ctl_reset_ingest_kernel(Ctl* c) {
    c->error = 0;
    c->err_info = 0;
    c->nrem = 0;
    c->noverflow = 0;
    c->reloc_need = 0;
    c->bad_index = 0x7F7F7F7F7F7F7F7FLL;   // larger than any position
    c->gather_n = 0;
    c->defer = 0;
}

__global__ void ctl_begin_maintain_kernel(Ctl* c, Resume rs, int take_nrem) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(c);
    constexpr int head = (int)(offsetof(Ctl, error) / 8);
    constexpr int z0 = (int)(offsetof(Ctl, tail) / 8), z1 = (int)(offsetof(Ctl, nrem) / 8);
    static_assert(offsetof(Ctl, error) % 8 == 0 && offsetof(Ctl, tail) % 8 == 0 && offsetof(Ctl, nrem) % 8 == 0,
                  "zeroed ranges are whole 8-byte words");
    for (int i = threadIdx.x; i < head; i += blockDim.x) w[i] = 0;
    for (int i = z0 + threadIdx.x; i < z1; i += blockDim.x) w[i] = 0;
    if (threadIdx.x == 0) {
        if (take_nrem) rs.nrem = c->nrem;
        c->rs = rs;
    }
}

cudaError_t ctl_reset_ingest(Ctl* c, cudaStream_t s) {
    ctl_reset_ingest_kernel<<<1, 1, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t ctl_begin_maintain(Ctl* c, const Resume& rs, int take_nrem, cudaStream_t s) {
    ctl_begin_maintain_kernel<<<1, 256, 0, s>>>(c, rs, take_nrem);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ ingest
__global__ void ingest_a_kernel(const int32_t* __restrict__ E, long long k, const unsigned long long* kp, DevGraph g,
                                BSet* bs, unsigned long long bmask, Ctl* c) {
    if (vload32(&c->defer)) return;
    k = item_count(k, kp);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        int32_t u = E[2 * i], v = E[2 * i + 1];
        if (u < 0 || v < 0 || u >= g.n || v >= g.n || g.hc[u].x < 0 || g.hc[v].x < 0) {
            atomicMin(&c->bad_index, i);
            atomicCAS(&c->error, 0, E_INVALID);
            continue;
        }
        if (u == v) continue;
        unsigned long long key = ekey(u, v);
        unsigned long long b = fmix64(key) & bmask;
        for (unsigned long long p = 0; p <= bmask; p++) {
            unsigned long long kk = bs[b].key;
            if (kk == KEY_EMPTY) {
                unsigned long long old = atomicCAS(&bs[b].key, KEY_EMPTY, key);
                if (old == KEY_EMPTY || old == key) { atomicMin(&bs[b].pos, (uint32_t)i); break; }
            } else if (kk == key) {
                atomicMin(&bs[b].pos, (uint32_t)i);
                break;
            }
            b = (b + 1) & bmask;
        }
    }
}

// Keeps the first occurrence of every edge of the batch that is absent
// (insert) or present (delete) in the graph.  Inserted keys enter the edge
// index later (index_new_edges), after the step has committed to running;
// the batch holds each key once, so no two threads look for the same one.
__global__ void ingest_b_kernel(const int32_t* __restrict__ E, long long k, const unsigned long long* kp, int op,
                                DevGraph g, const BSet* __restrict__ bs, unsigned long long bmask, REdge* R0,
                                int32_t* ovl, Ctl* c) {
    if (vload32(&c->error) || vload32(&c->defer)) return;   // uniform: final before this kernel starts
    k = item_count(k, kp);
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
                    long long bk = idx_find(g.idx, g.idx_mask, key);
                    if (op == 0 && bk < 0) {
                        keep = true;
                        r.lo = lo; r.hi = hi; r.bkt = 0u; r.flags = 0;
                        int a = atomicAdd(&g.need[lo], 1);
                        int el = g.end[lo], cl = g.cap[lo];
                        ov_lo = (el + a + 1 > cl) && (el + a <= cl);
                        int bb = atomicAdd(&g.need[hi], 1);
                        int eh = g.end[hi], ch = g.cap[hi];
                        ov_hi = (eh + bb + 1 > ch) && (eh + bb <= ch);
                    } else if (op == 1 && bk >= 0) {
                        keep = true;
                        r.lo = lo; r.hi = hi; r.bkt = (uint32_t)bk; r.flags = 0;
                    }
                }
            }
        }
        warp_push_edge(&c->nrem, R0, keep, r);
        warp_push(&c->noverflow, ovl, ~0ull, ov_lo, r.lo);
        warp_push(&c->noverflow, ovl, ~0ull, ov_hi, r.hi);
    }
}

// Inserts the kept edges' keys into the edge index (slots unknown until the
// maintenance kernel places the edge).
__global__ void index_new_edges_kernel(REdge* R, long long n, const unsigned long long* np, DevGraph g, Ctl* c) {
    if (vload32(&c->error) || vload32(&c->defer)) return;
    n = item_count(n, np);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        bool existed = false;
        long long bk = idx_insert(g.idx, g.idx_mask, ekey(R[i].lo, R[i].hi), &existed);
        if (bk < 0 || existed) {
            atomicCAS(&c->error, 0, E_INDEX_FULL);
            continue;
        }
        g.idx[bk].slo = -2;
        g.idx[bk].shi = -2;
        R[i].bkt = (uint32_t)bk;
    }
}

static unsigned grid_of(long long k, int t, long long cap) {
    long long b = (k + t - 1) / t;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t ingest_a(const int32_t* E, long long k, const unsigned long long* kp, DevGraph g, BSet* bs,
                     unsigned long long bmask, Ctl* c, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    ingest_a_kernel<<<grid_of(k, 256, 8192), 256, 0, s>>>(E, k, kp, g, bs, bmask, c);
    return cudaGetLastError();
}

cudaError_t ingest_b(const int32_t* E, long long k, const unsigned long long* kp, int op, DevGraph g,
                     const BSet* bs, unsigned long long bmask, REdge* R0, int32_t* ovl, Ctl* c, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    ingest_b_kernel<<<grid_of(k, 256, 4096), 256, 0, s>>>(E, k, kp, op, g, bs, bmask, R0, ovl, c);
    return cudaGetLastError();
}

cudaError_t index_new_edges(REdge* R, long long n, const unsigned long long* np, DevGraph g, Ctl* c,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    index_new_edges_kernel<<<grid_of(n, 256, 8192), 256, 0, s>>>(R, n, np, g, c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ relocation
// Vertices whose capacity a batch would exceed move to fresh space at the
// end of the adjacency pool, compacting their holes; the index learns the
// new slots.  Space is left as garbage at the old place.
__global__ void reloc_size_kernel(const int32_t* ovl, long long novl, const unsigned long long* np, DevGraph g,
                                  Ctl* c) {
    if (vload32(&c->defer)) return;
    novl = item_count(novl, np);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < novl; i += stride) {
        int x = ovl[i];
        int nc = cap_for((long long)g.deg[x] + g.need[x], g.slack_pct, g.min_cap);
        atomicAdd(&c->reloc_need, (unsigned long long)nc);
    }
}

// Captured step: stop before anything changes if the pool cannot take the
// relocations (the host grows it and redoes the step's remaining phases).
__global__ void reloc_gate_kernel(DevGraph g, Ctl* c, StepLog* log, int phase) {
    if (vload32(&c->defer)) return;
    if (vload32(&c->error)) {
        c->defer = 2;
        log->defer = phase + 1;
        return;
    }
    if ((long long)(vload64(&c->adj_top) + vload64(&c->reloc_need)) > g.adj_cap) {
        c->defer = 1;
        log->defer = phase + 1;
    }
}

__global__ void relocate_kernel(const int32_t* ovl, long long novl, const unsigned long long* np, DevGraph g,
                                Ctl* c) {
    if (vload32(&c->defer)) return;
    novl = item_count(novl, np);
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < novl; w += nw) {
        int x = ovl[w];
        int nc = cap_for((long long)g.deg[x] + g.need[x], g.slack_pct, g.min_cap);
        unsigned long long nb = 0;
        if (lane == 0) nb = atomicAdd(&c->adj_top, (unsigned long long)nc);
        nb = __shfl_sync(0xffffffffu, nb, 0);
        if ((long long)nb + nc > g.adj_cap) {       // the host or the gate sized the pool; never expected
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

__global__ void clear_need_kernel(const REdge* R, long long n, const unsigned long long* np, DevGraph g) {
    n = item_count(n, np);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        g.need[R[i].lo] = 0;
        g.need[R[i].hi] = 0;
    }
}

cudaError_t reloc_size(const int32_t* ovl, long long novl, const unsigned long long* np, DevGraph g, Ctl* c,
                       cudaStream_t s) {
    if (novl <= 0) return cudaSuccess;
    reloc_size_kernel<<<grid_of(novl, 256, 4096), 256, 0, s>>>(ovl, novl, np, g, c);
    return cudaGetLastError();
}
cudaError_t reloc_gate(DevGraph g, Ctl* c, StepLog* log, int phase, cudaStream_t s) {
    reloc_gate_kernel<<<1, 1, 0, s>>>(g, c, log, phase);
    return cudaGetLastError();
}
cudaError_t relocate(const int32_t* ovl, long long novl, const unsigned long long* np, DevGraph g, Ctl* c,
                     cudaStream_t s) {
    if (novl <= 0) return cudaSuccess;
    relocate_kernel<<<grid_of(novl * 32, 256, 8192), 256, 0, s>>>(ovl, novl, np, g, c);
    return cudaGetLastError();
}
cudaError_t clear_need(const REdge* R, long long n, const unsigned long long* np, DevGraph g, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    clear_need_kernel<<<grid_of(n, 256, 8192), 256, 0, s>>>(R, n, np, g);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ captured-step bookkeeping
// Step start: clear the exchange words and the log.
__global__ void step_begin_kernel(Ctl* c, StepLog* log) {
    c->error = 0;
    c->err_info = 0;
    c->defer = 0;
    c->nrem = 0;
    c->noverflow = 0;
    c->reloc_need = 0;
    c->bad_index = 0x7FFFFFFFFFFFFFFFll;
    c->gather_n = 0;
    unsigned char* p = reinterpret_cast<unsigned char*>(log);
    for (unsigned i = 0; i < sizeof(StepLog); i++) p[i] = 0;
}

// Phase start: an error so far (invalid ids) stops the step; otherwise the
// ingest counters restart.
__global__ void phase_begin_kernel(Ctl* c, StepLog* log, int phase) {
    if (c->defer) return;
    if (c->error) {
        c->defer = 2;
        log->defer = phase + 1;
        log->error[phase] = c->error;
        return;
    }
    c->nrem = 0;
    c->noverflow = 0;
    c->reloc_need = 0;
}

// Before the maintenance loop of a phase: reset the launch zone (barrier,
// tails, counters, statistics) and the resume state from the ingest count;
// the iteration stamp carries over from the previous call.
__global__ void phase_maintain_kernel(Ctl* c, StepLog* log, int phase) {
    const int stop = c->defer != 0 || c->error != 0;
    if (c->error && !c->defer) {
        c->defer = 2;
        log->defer = phase + 1;
    }
    c->arrive = 0;
    c->release = 0;
    for (int i = 0; i < kTails; i++) c->tail[i] = c->pc[i] = c->stail[i] = c->spc[i] = 0;
    for (int i = 0; i < ST_COUNT; i++) c->st[i] = 0;
    for (int i = 0; i < PH_COUNT; i++) c->ph[i] = 0;
    c->passes = 0;
    log->kept[phase] = stop ? 0 : c->nrem;
    c->rs.nrem = stop ? 0 : c->nrem;
    c->rs.rsel = 0;
    c->rs.done = stop || c->nrem == 0;
    c->rs.want = 0;
    c->rs.iters = 0;
    c->rs.mid = 0;
}

// After the loop: copy the phase's counters to the log; an error stops the step.
__global__ void phase_end_kernel(Ctl* c, StepLog* log, int phase) {
    for (int i = 0; i < ST_COUNT; i++) log->st[phase][i] = c->st[i];
    for (int i = 0; i < PH_COUNT; i++) log->ph[phase][i] = c->ph[i];
    log->passes[phase] = c->passes;
    log->iters_end[phase] = c->rs.iters;
    log->epoch_end = c->rs.epoch;
    if (c->error) {
        log->error[phase] = c->error;
        if (!c->defer) {
            c->defer = 2;
            log->defer = phase + 1;
        }
    }
}

cudaError_t step_begin(Ctl* c, StepLog* log, cudaStream_t s) {
    step_begin_kernel<<<1, 1, 0, s>>>(c, log);
    return cudaGetLastError();
}
cudaError_t phase_begin(Ctl* c, StepLog* log, int phase, cudaStream_t s) {
    phase_begin_kernel<<<1, 1, 0, s>>>(c, log, phase);
    return cudaGetLastError();
}
cudaError_t phase_maintain(Ctl* c, StepLog* log, int phase, cudaStream_t s) {
    phase_maintain_kernel<<<1, 1, 0, s>>>(c, log, phase);
    return cudaGetLastError();
}
cudaError_t phase_end(Ctl* c, StepLog* log, int phase, cudaStream_t s) {
    phase_end_kernel<<<1, 1, 0, s>>>(c, log, phase);
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
