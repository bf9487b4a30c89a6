// cm_iterate.cu -- the superior-edge-set iterations of one update batch.
//
// maintain_kernel<MODE> runs the iterations of SuperiorEdgeInsert
// (Algorithm 1) or SuperiorEdgeDelete (Algorithm 5) on the remaining edges
// of a batch.  MODE 0 is a cooperative launch filling the GPU, with grid-wide
// barriers; MODE 1 is one block of 512 threads with __syncthreads barriers,
// for the long tail of iterations that carry little work (a barrier there
// costs ~0.1 us instead of a few us).  Either kernel stops at an iteration
// boundary when the other mode suits the work better and records where to
// resume (Ctl::rs); the host queues a grid launch and a block launch back to
// back, so the handover needs no host round trip.
//
// Each iteration:
//   SELECT   a maximal superior edge set (Section IV, Definition 6 and the
//            union after it; Algorithm 2 made deterministic).  An edge's
//            constrained endpoints are those whose core equals the edge's
//            core number min(core(u), core(v)).  In claim rounds every
//            eligible edge writes its priority fmix64(key) into its
//            constrained endpoints with atomicMin and wins when it holds all
//            of them; winners take their endpoints and edges touching a taken
//            endpoint wait for the next iteration.  The result is the greedy
//            (lexicographically first) maximal set in priority order.
//   APPLY    insert / delete the selected edges in the slack CSR and move
//            SD (superior degree, Definition 7) of constrained endpoints.
//   insert:  positive and negative search of Algorithms 3-4, run as
//            breadth-first waves in which both progress together (single-
//            block mode) or as a task queue without level barriers (grid
//            mode, below async_search: the order of processing does not
//            change the result).  The
//            constrained endpoints are the first frontier.  Processing a
//            frontier vertex v adds CSD(v) (Definition 8) to its support
//            count, which already holds one decrement per evicted neighbour
//            (the paper's pre-decremented cd).  If the count exceeds k, v
//            visits its unvisited core-k neighbours with SD > k (the next
//            frontier); otherwise v is evicted (Lemma 8).  An evicted vertex
//            takes one from the count of every core-k neighbour with SD > k,
//            visited or not; a processed neighbour whose count falls to k is
//            evicted too (InsertRemove, Algorithm 4).  Frontier and evictions
//            of a wave run in the same phase, so evictions prune the search
//            as it grows.  COMMIT: processed vertices still above k rise by
//            one (the last step of Algorithm 1, Lemma 7).
//   delete:  EVICT in waves (or, grid-wide, as queued tasks) from the
//            constrained endpoints whose SD fell below k (Algorithm 6); an
//            evicted vertex drops by one and takes
//            one from the support (initially SD) of every core-k neighbour,
//            which leaves when its support falls below k (DeleteRemove,
//            Algorithm 7; the last step of Algorithm 5).
//   FIX-UP   recompute SD of moved vertices and adjust SD of unmoved
//            neighbours whose core equals the moved vertex's new core
//            (insert) or old core (delete).  It only writes SD, which the
//            next iteration first reads in APPLY, so it runs inside the next
//            iteration's first claim phase and costs no barrier of its own.
// All levels run together on the cores of the iteration's start: searches
// and evictions only ever follow neighbours of the vertex's own level.
//
// The per-vertex bodies and the per-iteration vertex word are in cm_vertex.cuh.
//
// Per-vertex work of a wave is done by one warp per vertex (vertices fetched
// dynamically); a vertex with at least P.block_len adjacency slots (256 in
// single-block mode) is deferred
// and then processed by the whole block of the warp that fetched it.
#include "cm_common.cuh"
#include "cm_launch.h"
#include "cm_vertex.cuh"

namespace cm {

constexpr int kBlockThreads = 512;    // single-block mode
constexpr int kGridThreads = 512;     // grid mode, per block
static_assert(kGridThreads / 32 == kGridWarps, "one kept-task slot per grid-mode warp");
constexpr int kMaxBig = 64;
constexpr int kBlockLenSingle = 256;   // single-block mode: the block scans lists from this size

template <int MODE>
struct Barrier {
    Ctl* c;
    uint32_t expect;
    unsigned long long limit;
    unsigned long long t_last;
    bool timer;
    __device__ bool operator()(int phase) {
        bool ok = MODE == 0 ? grid_sync(c, expect, limit) : block_sync(c);
        if (timer) {
            unsigned long long now = gtimer();
            c->ph[phase] += now - t_last;
            c->st[ST_BARRIERS] += 1;
            t_last = now;
        }
        return ok;
    }
};

// ---------------------------------------------------------------- vertex loop (waves)
// Runs body(v, Group) for every vertex of ring[lo, hi): one warp per vertex.
// Each warp's first vertex is dealt by its warp index; the rest are fetched
// dynamically (counter *ctr, zeroed at every barrier), so a phase with no
// more vertices than warps touches no shared counter, and a larger one does
// not start with every warp of the grid at the same counter.  A vertex
// with at least P.block_len slots (kBlockLenSingle in single-block mode) is
// deferred by the warp that fetched it and then processed by that warp's
// whole block, so a long list does not hold a wave on one warp.  Every
// thread of the launch must call it.
template <int MODE, class Body>
__device__ __forceinline__ void for_each_vertex(const DevGraph& g, const MaintainParams& P, unsigned long long* ctr,
                                                const int32_t* ring, unsigned long long qm, unsigned long long lo,
                                                unsigned long long hi, Body body) {
    constexpr int NT = MODE == 0 ? kGridThreads : kBlockThreads;
    const int lane = lane_id();
    __shared__ int s_big[kMaxBig];
    __shared__ int s_nbig;
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long cnt = hi - lo;
    unsigned long long j = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (;;) {
        if (j >= cnt) break;
        const int v = ring[(lo + j) & qm];
        int defer = 0;
        if (lane == 0 && g.end[v] >= (MODE == 0 ? P.block_len : kBlockLenSingle)) {
            int s = atomicAdd(&s_nbig, 1);
            if (s < kMaxBig) {
                s_big[s] = v;
                defer = 1;
            }
        }
        if (!__shfl_sync(0xffffffffu, defer, 0)) body(v, WarpGroup{});
        if (cnt <= nw) break;   // every vertex was dealt by index
        if (lane == 0) j = nw + atomicAdd(ctr, 1ull);
        j = __shfl_sync(0xffffffffu, j, 0);
    }
    __syncthreads();
    const int nb = min(s_nbig, kMaxBig);
    for (int b = 0; b < nb; b++) {
        body(s_big[b], BlockGroup<NT>{});
        __syncthreads();
    }
}

// Single-block mode: adjacency slots of the vertices of ring ranges
// [lo0, hi0) and [lo1, hi1) (a wave about to run), summed by the block.
__device__ __forceinline__ long long wave_slots(const DevGraph& g, const int32_t* r0, unsigned long long lo0,
                                                unsigned long long hi0, const int32_t* r1, unsigned long long lo1,
                                                unsigned long long hi1, unsigned long long qm) {
    __shared__ long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    long long part = 0;
    for (unsigned long long i = lo0 + threadIdx.x; i < hi0; i += blockDim.x) part += g.end[r0[i & qm]];
    for (unsigned long long i = lo1 + threadIdx.x; i < hi1; i += blockDim.x) part += g.end[r1[i & qm]];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane_id() == 0 && part) atomicAdd((unsigned long long*)&s_sum, (unsigned long long)part);
    __syncthreads();
    const long long total = s_sum;
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------- grid-mode task queue
// In grid mode the search of an iteration (insert: positive search and
// evictions; delete: evictions) runs without level barriers.  Every vertex
// that enters the frontier or is evicted also becomes a task in a queue
// (push_vertex), and warps claim tasks one at a time until the queue is
// quiescent: every task pushed has finished.  The proof of the interleaved
// search does not depend on the order in which vertices are processed, so
// the waves of the single-block mode and this order reach the same cores.
//
// A vertex with at least P.hub_len slots becomes a hub item instead, whose
// list is split into kChunk-slot chunk tasks that any warp may take:
//   HUB_FRONT: each chunk adds its share of CSD to the item; the warp that
//     finishes the last chunk adds the sum to the support word at once
//     (setting the processed flag, as a whole-list scan would) and either
//     queues an expansion item (support > k) or evicts the vertex;
//   HUB_EXPAND: each chunk visits its share of the core-k neighbours;
//   HUB_EVICT_INS / HUB_EVICT_DEL: each chunk evicts its share; the last one
//     lowers the core (delete) and counts the vertex.
// The support word tolerates the delay: decrements from evicted neighbours
// land before or after the CSD sum in any order, and a processed hub whose
// count later falls to k is evicted by the decrement that does it.

// Creates a hub item and its chunk tasks (warp-collective); false if the
// item ring is full (the caller then scans the list itself).
__device__ __forceinline__ bool make_hub(Ctl* C, const MaintainParams& P, int v, int kind, int k, long long off,
                                         int len) {
    const int lane = lane_id();
    const int nch = (len + kChunk - 1) / kChunk;
    unsigned long long idx = 0, tb = 0;
    int ok = 0;
    if (lane == 0) {
        if (vload64(&C->hub_created) - vload64(&C->hub_finished) < kHubRingSafe) {
            idx = atomicAdd(&C->hub_created, 1ull);
            HubItem* it = &P.HQ[idx & (kHubRing - 1)];
            it->off = off;
            it->v = v;
            it->kind = kind;
            it->k = k;
            it->len = len;
            it->nch = nch;
            it->acc = 0;
            it->done = 0u;
            __threadfence();   // the item before its tasks
            tb = atomicAdd(&C->task_tail, (unsigned long long)nch);
            ok = 1;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    idx = __shfl_sync(0xffffffffu, idx, 0);
    tb = __shfl_sync(0xffffffffu, tb, 0);
    if (!task_room(C, P, tb, (unsigned long long)nch)) return true;   // error recorded; the search stops
    const unsigned long long base = ((idx & (kHubRing - 1)) << kTaskChunkBits);
    for (int j = lane; j < nch; j += 32)
        vstore64(&P.TQ[(tb + j) & P.tqmask], mk_task(T_CHUNK, base | (unsigned long long)j));
    return true;
}

__device__ __forceinline__ int vload32i(const int* p) { return *(const volatile int*)p; }

// One chunk task (warp-collective).
__device__ __forceinline__ void run_chunk(const DevGraph& g, Ctl* C, const MaintainParams& P, uint32_t e,
                                          LocalStats& ls, unsigned long long payload) {
    using WG = WarpGroup;
    const int lane = lane_id();
    HubItem* it = &P.HQ[payload >> kTaskChunkBits];
    const int ci = (int)(payload & ((1ull << kTaskChunkBits) - 1));
    // the item was written by another SM: read it from L2
    const int v = vload32i(&it->v), kind = vload32i(&it->kind), k = vload32i(&it->k);
    const int len = vload32i(&it->len), nch = vload32i(&it->nch);
    const long long off = (long long)vload64((const unsigned long long*)&it->off);
    const int s0 = ci * kChunk, s1 = min(s0 + kChunk, len);
    if (kind == HUB_FRONT || kind == HUB_FRONT_SPEC) {
        const int part = WG::sum(kind == HUB_FRONT_SPEC ? csd_expand_range<WG, true>(g, C, P, k, off, s0, s1, e)
                                                        : csd_part<WG>(g, k, off, s0, s1));
        int decide = 0;   // 1 expand, 2 evict
        if (lane == 0) {
            atomicAdd(&it->acc, part);
            __threadfence();
            if (atomicAdd(&it->done, 1u) == (uint32_t)(nch - 1)) {
                __threadfence();
                const int acc = atomicAdd(&it->acc, 0);
                uint32_t of;
                int32_t oc;
                add_word(g, C, v, e, acc, kProcessed, of, oc);
                ls.vis++;
                ls.visl += len;
                decide = oc + acc > k ? 1 : 2;
                atomicAdd(&C->hub_finished, 1ull);
            }
        }
        decide = __shfl_sync(0xffffffffu, decide, 0);
        if (decide == 1 && kind == HUB_FRONT && !make_hub(C, P, v, HUB_EXPAND, k, off, len))
            expand_range<WG, true>(g, C, P, k, off, 0, len, e);
        if (decide == 2) push_vertex<true>(C, P, lane == 0, v, 1, true);
        return;
    }
    if (kind == HUB_EXPAND) expand_range<WG, true>(g, C, P, k, off, s0, s1, e);
    else if (kind == HUB_EVICT_INS) evict_ins_range<WG, true>(g, C, P, k, off, s0, s1, e);
    else evict_del_range<WG, true>(g, C, P, k, off, s0, s1, e);
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&it->done, 1u) == (uint32_t)(nch - 1)) {
            if (kind == HUB_EVICT_DEL) {
                g.hc[v].x = k - 1;
                g.kc[v] = key_of(k - 1, 0);   // the SD fix-up of the next claim phase sets its bit
            }
            if (kind != HUB_EXPAND) {
                ls.ev++;
                ls.evl += len;
            }
            atomicAdd(&C->hub_finished, 1ull);
        }
    }
}

// Search (iteration number) whose queue the block's poller found quiescent.
__shared__ volatile uint32_t s_quiet;

// Drains the task queue (every warp of the grid).  Returns false on error.
// A warp claims up to P.claim_max consecutive slots with one atomic: it
// doubles its claim while its slots are ready at once and drops back to one
// slot after a wait.  One slot at a time balances best when tasks are large
// (a warp holding a run of large tasks leaves others idle); several save
// head-counter traffic when tasks are tiny (the many-graph workload), so the
// limit is a schedule knob.  Finished tasks are reported in batches, always
// before the warp waits on an empty slot (so a waiting warp never holds back
// the quiescence test).  Inlined into the kernel: as a separate function it
// took the graph and the parameters by reference, which put both in local
// memory and made every pointer it used a local load (measured 8-15% slower
// per call, although the inlined kernel spills more registers).
__device__ __forceinline__ bool async_search(const DevGraph& g, Ctl* C, const MaintainParams& P, uint32_t e,
                                          LocalStats& ls) {
    using WG = WarpGroup;
    const int lane = lane_id();
    const unsigned long long t_start = gtimer();
    unsigned long long idx = 0, ndone = 0;
    int left = 0, claim = 1;
    bool waited = false;
    const int cmax = P.claim_max > 1 ? P.claim_max : 1;
    // one warp per block tests quiescence and tells the others through
    // shared memory: a test reads two hot counters, and thousands of
    // waiting warps reading them would slow the claims and pushes that
    // share those counters' L2 slices
    const bool poller = threadIdx.x < 32;
    if (lane == 0) kept_task() = TASK_EMPTY;
    __syncwarp();
    for (;;) {
        unsigned long long t = kept_task();
        int quit = 0;
        const bool own = t != TASK_EMPTY;   // the task this warp kept from its last one
        __syncwarp();
        if (own) {
            if (lane == 0) kept_task() = TASK_EMPTY;
        } else if (lane == 0) {
            if (left == 0) {
                claim = waited ? 1 : min(2 * claim, cmax);
                waited = false;
                idx = atomicAdd(&C->task_head, (unsigned long long)claim);
                left = claim;
            }
            unsigned long long* slot = &P.TQ[idx & P.tqmask];
            unsigned int nap = 32;
            for (unsigned int spins = 0;; spins++) {
                t = vload64(slot);
                if (t != TASK_EMPTY) {
                    vstore64(slot, TASK_EMPTY);   // free for the next search
                    break;
                }
                waited = true;
                if (ndone) {   // report before waiting
                    __threadfence();
                    atomicAdd(&C->task_done, ndone);
                    ndone = 0;
                }
                if (poller) {
                    // quiescent: every task pushed has finished (done read first)
                    const unsigned long long d = ld_acquire64(&C->task_done);   // read before the tail
                    if (d == vload64(&C->task_tail) || vload32(&C->error)) {
                        s_quiet = e;
                        quit = 1;
                        break;
                    }
                } else if (s_quiet == e) {
                    quit = 1;
                    break;
                }
                if ((spins & 3u) == 0 && gtimer() - t_start > P.limit_ns) {
                    atomicCAS(&C->error, 0, E_BARRIER_TIMEOUT);
                    quit = 1;
                    break;
                }
                __nanosleep(nap);
                if (nap < 512) nap <<= 1;
            }
            idx++;
            left--;
        }
        if (__shfl_sync(0xffffffffu, quit, 0)) break;
        t = __shfl_sync(0xffffffffu, t, 0);
        __syncwarp();
        // acquire: the task's vertex data as its producers left it (measured
        // necessary: without it, warps running several claimed tasks in a
        // row reached wrong cores on small delete batches)
        __threadfence();
        const int type = (int)(t >> 62);
        const unsigned long long payload = t & ((1ull << 62) - 1);
        if (type == T_CHUNK) {
            run_chunk(g, C, P, e, ls, payload);
        } else {
            const int v = (int)payload;
            const VInfo vi = load_vinfo(g, v);
            const bool hub = P.hub_len > 0 && vi.len >= P.hub_len;
            if (type == T_FRONT) {
                if (!hub || !make_hub(C, P, v, expand_early(P, vi.h.y, vi.h.x) ? HUB_FRONT_SPEC : HUB_FRONT, vi.h.x,
                                      vi.o, vi.len))
                    process_frontier<WG, true>(g, C, P, v, vi, e, ls);
            } else if (P.op == 0) {
                if (!hub || !make_hub(C, P, v, HUB_EVICT_INS, vi.h.x, vi.o, vi.len))
                    evict_insert_vertex<WG, true>(g, C, P, vi, e, ls);
            } else {
                if (!hub || !make_hub(C, P, v, HUB_EVICT_DEL, vi.h.x, vi.o, vi.len))
                    evict_delete_vertex<WG, true>(g, C, P, v, vi, e, ls);
            }
        }
        __syncwarp();
        // this task's pushes precede the fence of the next report; a kept
        // task was never counted in the tail
        if (lane == 0 && !own) ndone++;
    }
    return vload32(&C->error) == 0;
}

// Queues tasks for log entries [lo, hi) that are already in the log (a
// search resumed from the single-block mode).  Every warp calls it.
__device__ __forceinline__ void seed_tasks(Ctl* C, const MaintainParams& P, const int32_t* log, unsigned long long lo,
                                           unsigned long long hi, int type) {
    const int lane = lane_id();
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long base = lo + (unsigned long long)gwarp * 32; base < hi;
         base += (unsigned long long)nwarps * 32) {
        const unsigned long long cnt = min(32ull, hi - base);
        unsigned long long tb = 0;
        if (lane == 0) tb = atomicAdd(&C->task_tail, cnt);
        tb = __shfl_sync(0xffffffffu, tb, 0);
        if (task_room(C, P, tb, cnt) && (unsigned long long)lane < cnt)
            vstore64(&P.TQ[(tb + lane) & P.tqmask],
                     mk_task(type, (unsigned long long)(uint32_t)log[(base + lane) & P.qmask]));
    }
}

// An edge's core number k = min(core(lo), core(hi)) and its constrained
// endpoints: those whose core is k (Definition 6), except pinned vertices.
// An insertion never has pinned vertices (they exist only while a vertex
// deletion removes their edges), so it reads the cores from the 4-byte keys.
__device__ __forceinline__ void edge_level(const DevGraph& g, const REdge& E, bool ins, int& k, bool& clo,
                                           bool& chi) {
    if (ins) {
        const int a = key_core(g.kc[E.lo]);
        const int b = key_core(g.kc[E.hi]);
        k = min(a, b);
        clo = a == k;
        chi = b == k;
        return;
    }
    const int2 a = g.hc[E.lo];
    const int2 b = g.hc[E.hi];
    k = min(a.x, b.x);
    clo = a.x == k && a.y < PIN_SD;
    chi = b.x == k && b.y < PIN_SD;
}

// An edge's selection priority (smaller wins): fmix64 of its canonical key,
// a bijection, or the key itself (lexicographic order of (lo, hi)).
__device__ __forceinline__ unsigned long long edge_prio(const REdge& E, bool by_key) {
    const unsigned long long key = ekey(E.lo, E.hi);
    return by_key ? key : fmix64(key);
}

// Selection, claim phase of round r.  An edge already selected or blocked
// that did not claim in round r-1 has nothing to do and gathers nothing.
__device__ __forceinline__ void claim_edge(const DevGraph& g, REdge* R, long long i, int r, uint32_t e, bool by_key,
                                           bool ins) {
    REdge E = R[i];
    const uint32_t f = E.flags;
    const bool claimed_last = r > 0 && (f >> 2) == (uint32_t)r;
    if ((f & (F_SEL | F_BLK)) && !claimed_last) return;
    int k; bool clo, chi;
    edge_level(g, E, ins, k, clo, chi);
    if (claimed_last) {   // claimed in round r-1: clear that buffer
        unsigned long long* cb = ((r - 1) & 1) ? g.claim1 : g.claim0;
        if (clo) cb[E.lo] = CLAIM_FREE;
        if (chi) cb[E.hi] = CLAIM_FREE;
    }
    if (f & (F_SEL | F_BLK)) return;
    if ((clo && g.taken[E.lo] == e) || (chi && g.taken[E.hi] == e)) {
        R[i].flags = f | F_BLK;
        return;
    }
    const unsigned long long prio = edge_prio(E, by_key);
    unsigned long long* cb = (r & 1) ? g.claim1 : g.claim0;
    if (clo) atomicMin(&cb[E.lo], prio);
    if (chi) atomicMin(&cb[E.hi], prio);
    R[i].flags = (f & 3u) | ((uint32_t)(r + 1) << 2);
}

// Selection, check phase of round r.  Returns 1 if the edge claimed and lost.
__device__ __forceinline__ int check_edge(const DevGraph& g, REdge* R, long long i, int r, uint32_t e,
                                          uint32_t& nsel, bool by_key, bool ins) {
    REdge E = R[i];
    if ((E.flags >> 2) != (uint32_t)(r + 1)) return 0;
    int k; bool clo, chi;
    edge_level(g, E, ins, k, clo, chi);
    const unsigned long long prio = edge_prio(E, by_key);
    const unsigned long long* cb = (r & 1) ? g.claim1 : g.claim0;
    bool win = (!clo || cb[E.lo] == prio) && (!chi || cb[E.hi] == prio);
    if (!win) return 1;
    R[i].flags = E.flags | F_SEL;
    if (clo) g.taken[E.lo] = e;
    if (chi) g.taken[E.hi] = e;
    nsel++;
    return 0;
}

constexpr unsigned long long kMaxPasses = 256;   // launch pairs per phase of a captured step

// Inside a captured update step the launch pairs (grid kernel, then
// single-block kernel) are the body of a conditional WHILE node: the
// single-block kernel ends every pass by setting the node's condition, so
// the loop runs until the call is done or failed with no host round trip.
__device__ __forceinline__ void loop_control(const MaintainParams& P, Ctl* C) {
    if (!P.use_cond || threadIdx.x != 0) return;
    const unsigned long long n = C->passes + 1;
    C->passes = n;
    int err = vload32(&C->error);
    const int done = *(volatile int*)&C->rs.done;
    if (!err && !done && n >= kMaxPasses) {
        atomicCAS(&C->error, 0, E_ITER_LIMIT);
        err = 1;
    }
    cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, (!err && !done) ? 1u : 0u);
}

template <int MODE>
__global__ void __launch_bounds__(MODE == 0 ? kGridThreads : kBlockThreads, MODE == 0 ? 2 : 1)
    maintain_kernel(MaintainParams P) {
    Ctl* C = P.ctl;
    const DevGraph g = P.g;
    // where to resume (the host or the other mode wrote it before this launch)
    const int done0 = *(volatile int*)&C->rs.done;
    const int want = *(volatile int*)&C->rs.want;
    if (done0 || want != MODE || vload32(&C->error)) {
        if (MODE == 1) loop_control(P, C);
        return;
    }
    if (MODE == 0) {   // shared memory starts undefined: no search is quiescent yet
        if (threadIdx.x == 0) s_quiet = ~0u;
        __syncthreads();
    }
    const int lane = lane_id();
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long qm = P.qmask;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    Barrier<MODE> sync{C, P.expect, P.limit_ns, gtimer(), leader};
    const uint32_t rsel0 = *(volatile uint32_t*)&C->rs.rsel;
    REdge* Rc = rsel0 ? P.R1 : P.R0;
    REdge* Rn = rsel0 ? P.R0 : P.R1;
    unsigned long long nrem = vload64(&C->rs.nrem);
    uint32_t e = *(volatile uint32_t*)&C->rs.epoch;
    const long long iters0 = *(volatile long long*)&C->rs.iters;
    unsigned long long vq_t = vload64(&C->tail[0]), eq_t = vload64(&C->tail[1]), cq_t = vload64(&C->tail[2]);
    // grid mode: the task queue starts empty for every search
    auto reset_tasks = [&]() {
        if (leader) {
            C->task_head = 0;
            C->task_tail = P.phantom_task ? 1 : 0;   // a phantom is never queued: no quiescence
            C->task_done = 0;
            C->hub_created = 0;
            C->hub_finished = 0;
        }
    };
    LocalStats ls;
    int iters = 0, rounds = 0, waves = 0;   // per launch (a call is capped far below 2^31 iterations)
    long long remsum = 0;
    // resume inside the search waves of an iteration the single-block mode began
    bool mid = *(volatile int*)&C->rs.mid != 0;
    bool escalate = false;
    unsigned long long nrem_next = 0, vq0 = 0, eq0 = 0, cq0 = 0, flo = 0, fhi = 0, elo = 0, ehi = 0;
    if (mid) {
        nrem_next = nrem;                  // edges left for the next iteration, in buffer rsel
        REdge* t0 = Rc;
        Rc = Rn;
        Rn = t0;
        vq0 = vload64(&C->rs.vq0);
        eq0 = vload64(&C->rs.eq0);
        cq0 = vload64(&C->rs.cq0);
        flo = vload64(&C->rs.flo);
        fhi = vload64(&C->rs.fhi);
        elo = vload64(&C->rs.elo);
        ehi = vload64(&C->rs.ehi);
    }
    bool ok = true;
    // pending SD fix-up of the previous iteration
    bool fx = false;
    unsigned long long fx_lo = 0, fx_hi = 0;
    uint32_t fx_e = 0;
    // a call whose ingest kept no edge (its count read on the device) is done at once
    int next_want = MODE, finished = (!mid && nrem == 0) ? 1 : 0;
    const int32_t* FXQ = P.op == 0 ? P.CQ : P.EQ;
    auto fixup_body = [&](int v, auto grp) { fixup_vertex<decltype(grp)>(g, v, fx_e, P.op, ls); };

    while (mid || nrem > 0) {
      if (!mid) {
        if (iters0 + iters >= P.max_iters) {
            if (leader) atomicCAS(&C->error, 0, E_ITER_LIMIT);
            ok = false;
            break;
        }
        remsum += (long long)nrem;
        // ------------------------------------------------ SELECT
        int r = 0;
        for (;;) {
            if (r == 0 && fx) {
                for_each_vertex<MODE>(g, P, &C->pc[2], FXQ, qm, fx_lo, fx_hi, fixup_body);
                fx = false;
            }
            if (MODE == 0 && r == 0) reset_tasks();   // nobody pushes tasks before APPLY
            for (long long base = gwarp * 32; base < (long long)nrem; base += nwarps * 32) {
                long long i = base + lane;
                if (i < (long long)nrem) claim_edge(g, Rc, i, r, e, P.sel_key != 0, P.op == 0);
            }
            if (!(ok = sync(PH_CLAIM))) break;
            int lost = 0;
            for (long long base = gwarp * 32; base < (long long)nrem; base += nwarps * 32) {
                long long i = base + lane;
                if (i < (long long)nrem) lost += check_edge(g, Rc, i, r, e, ls.sel, P.sel_key != 0, P.op == 0);
            }
            lost = warp_sum(lost);
            if (lane == 0 && lost) atomicAdd(&C->pc[0], (unsigned long long)lost);
            if (!(ok = sync(PH_CHECK))) break;
            r++;
            if (vload64(&C->spc[0]) == 0) break;           // no edge lost: the set is maximal
            if (P.sel_rounds > 0 && r >= P.sel_rounds) break;   // capped: a superior edge set all the same
        }
        if (!ok) break;
        rounds += r;
        // ------------------------------------------------ APPLY
        vq0 = vq_t;
        eq0 = eq_t;
        cq0 = cq_t;
        for (long long base = gwarp * 32; base < (long long)nrem; base += nwarps * 32) {
            long long i = base + lane;
            bool valid = i < (long long)nrem;
            REdge E = {0, 0, 0, 0};
            bool sel = false, s_lo = false, s_hi = false;
            if (valid) {
                E = Rc[i];
                int k = 0; bool clo = false, chi = false;
                // only a selected edge or one that claimed in the final round needs its level
                if ((E.flags & F_SEL) || (E.flags >> 2) == (uint32_t)r) edge_level(g, E, P.op == 0, k, clo, chi);
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
                        // a constrained endpoint's SD rises; with SD > k it roots the search
                        // (one selected edge per constrained endpoint and level: this is the
                        // only SD change of the endpoint in APPLY, so its key bit follows it)
                        if (clo) {
                            const int sd = atomicAdd(&g.hc[E.lo].y, 1) + 1;
                            if (sd > k) atomicOr(&g.kc[E.lo], 1u);
                            s_lo = sd > k && visit(g, C, E.lo, e);
                        }
                        if (chi) {
                            const int sd = atomicAdd(&g.hc[E.hi].y, 1) + 1;
                            if (sd > k) atomicOr(&g.kc[E.hi], 1u);
                            s_hi = sd > k && visit(g, C, E.hi, e);
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
                            int m = atomicSub(&g.hc[E.lo].y, 1) - 1;
                            if (m <= k) atomicAnd(&g.kc[E.lo], ~1u);
                            if (m < k) { s_lo = true; g.chg[E.lo] = e; }
                        }
                        if (chi) {
                            int m = atomicSub(&g.hc[E.hi].y, 1) - 1;
                            if (m <= k) atomicAnd(&g.kc[E.hi], ~1u);
                            if (m < k) { s_hi = true; g.chg[E.hi] = e; }
                        }
                    }
                }
                E.flags = 0;
            }
            warp_push_edge(&C->pc[1], Rn, valid && !sel, E);
            // roots: frontier (insert) or evicted (delete) constrained endpoints
            push_vertex<MODE == 0>(C, P, s_lo, E.lo, P.op == 0 ? 0 : 1);
            push_vertex<MODE == 0>(C, P, s_hi, E.hi, P.op == 0 ? 0 : 1);
        }
        if (!(ok = sync(PH_APPLY))) break;
        nrem_next = vload64(&C->spc[1]);
        vq_t = vload64(&C->stail[0]);
        eq_t = vload64(&C->stail[1]);
        flo = vq0;
        fhi = vq_t;
        elo = eq0;
        ehi = eq_t;
      }
      const bool resumed = mid;
      mid = false;

        if (P.op == 0) {
            // -------------------------------------------- SEARCH (insert): frontier + evictions
            if (MODE == 0) {
                if (resumed) {   // the single-block mode began this search
                    reset_tasks();
                    if (!(ok = sync(PH_APPLY))) break;
                    seed_tasks(C, P, P.VQ, flo, fhi, T_FRONT);
                    seed_tasks(C, P, P.EQ, elo, ehi, T_EVICT);
                    if (!(ok = sync(PH_APPLY))) break;
                }
                waves++;
                ok = async_search(g, C, P, e, ls);
                if (!(ok = sync(PH_DISCOVER) && ok)) break;
                fhi = vload64(&C->stail[0]);
                ehi = vload64(&C->stail[1]);
            } else {
                while (fhi > flo || ehi > elo) {
                    // a wave too big for one block (by vertices, or by the slots
                    // of its vertices' lists) goes to the grid
                    if ((fhi - flo) + (ehi - elo) > (unsigned long long)P.big_wave ||
                        wave_slots(g, P.VQ, flo, fhi, P.EQ, elo, ehi, qm) > P.big_slots) {
                        escalate = true;
                        break;
                    }
                    waves++;
                    for_each_vertex<MODE>(g, P, &C->pc[2], P.VQ, qm, flo, fhi, [&](int v, auto grp) {
                        process_frontier<decltype(grp), false>(g, C, P, v, load_vinfo(g, v), e, ls);
                    });
                    for_each_vertex<MODE>(g, P, &C->pc[3], P.EQ, qm, elo, ehi, [&](int v, auto grp) {
                        evict_insert_vertex<decltype(grp), false>(g, C, P, load_vinfo(g, v), e, ls);
                    });
                    if (!(ok = sync(PH_DISCOVER))) break;
                    flo = fhi;
                    fhi = vload64(&C->stail[0]);
                    elo = ehi;
                    ehi = vload64(&C->stail[1]);
                }
            }
            if (!ok || escalate) break;
            vq_t = fhi;
            eq_t = ehi;
            // -------------------------------------------- COMMIT (insert): survivors rise
            for (long long base = gwarp * 32; base < (long long)(vq_t - vq0); base += nwarps * 32) {
                long long i = base + lane;
                bool up = false;
                int v = 0;
                if (i < (long long)(vq_t - vq0)) {
                    v = P.VQ[(vq0 + i) & qm];
                    const int core = g.hc[v].x;
                    const int support = ww(g.hw[v]);
                    if (support > core) {
                        g.hc[v].x = core + 1;
                        g.kc[v] = key_of(core + 1, 0);   // bit set by the SD fix-up
                        g.chg[v] = e;
                        up = true;
                    }
                }
                warp_push(&C->tail[2], P.CQ, qm, up, v);
            }
            if (!(ok = sync(PH_COMMIT))) break;
            cq_t = vload64(&C->stail[2]);
            fx = cq_t > cq0;
            fx_lo = cq0;
            fx_hi = cq_t;
        } else {
            // -------------------------------------------- EVICT (delete); evicted vertices drop by one
            if (MODE == 0) {
                if (resumed) {
                    reset_tasks();
                    if (!(ok = sync(PH_APPLY))) break;
                    seed_tasks(C, P, P.EQ, elo, ehi, T_EVICT);
                    if (!(ok = sync(PH_APPLY))) break;
                }
                waves++;
                ok = async_search(g, C, P, e, ls);
                if (!(ok = sync(PH_EVICT) && ok)) break;
                ehi = vload64(&C->stail[1]);
            } else {
                while (ehi > elo) {
                    if (ehi - elo > (unsigned long long)P.big_wave ||
                        wave_slots(g, P.EQ, elo, ehi, P.EQ, 0, 0, qm) > P.big_slots) {
                        escalate = true;
                        break;
                    }
                    waves++;
                    for_each_vertex<MODE>(g, P, &C->pc[2], P.EQ, qm, elo, ehi, [&](int v, auto grp) {
                        evict_delete_vertex<decltype(grp), false>(g, C, P, v, load_vinfo(g, v), e, ls);
                    });
                    if (!(ok = sync(PH_EVICT))) break;
                    elo = ehi;
                    ehi = vload64(&C->stail[1]);
                }
            }
            if (!ok || escalate) break;
            eq_t = ehi;
            fx = eq_t > eq0;
            fx_lo = eq0;
            fx_hi = eq_t;
        }
        fx_e = e;
        // ------------------------------------------------ next iteration, or hand over
        const unsigned long long nsel = nrem - nrem_next;
        const unsigned long long work = (vq_t - vq0) + (eq_t - eq0) + (cq_t - cq0) + nsel;
        REdge* t = Rc;
        Rc = Rn;
        Rn = t;
        nrem = nrem_next;
        e++;
        iters++;
        if (nrem == 0) {
            finished = 1;
            break;
        }
        if (P.yield_each) {   // debug: end the launch here (the fix-up below still runs); resume in this mode
            next_want = MODE;
            break;
        }
        if (MODE == 0 && nrem <= (unsigned long long)P.small_edges && work <= (unsigned long long)P.small_work) {
            next_want = 1;
            break;
        }
        if (MODE == 1 && work > (unsigned long long)P.big_work) {
            next_want = 0;
            break;
        }
    }
    if (ok && fx) {
        for_each_vertex<MODE>(g, P, &C->pc[2], FXQ, qm, fx_lo, fx_hi, fixup_body);
        ok = sync(PH_FIXUP);
    }
    // statistics: one atomic per warp
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
    if (leader) {
        C->st[ST_ITERS] += (unsigned long long)iters;
        if (MODE == 0) C->st[ST_GRID_ITERS] += (unsigned long long)iters;
        C->st[ST_ROUNDS] += (unsigned long long)rounds;
        C->st[ST_WAVES] += (unsigned long long)waves;
        C->st[ST_REMSUM] += (unsigned long long)remsum;
        if (ok && escalate) {
            C->rs.nrem = nrem_next;
            C->rs.rsel = Rn == P.R1 ? 1u : 0u;
            C->rs.epoch = e;
            C->rs.iters = iters0 + iters;
            C->rs.done = 0;
            C->rs.want = 0;
            C->rs.mid = 1;
            C->rs.vq0 = vq0;
            C->rs.eq0 = eq0;
            C->rs.cq0 = cq0;
            C->rs.flo = flo;
            C->rs.fhi = fhi;
            C->rs.elo = elo;
            C->rs.ehi = ehi;
            __threadfence();
        } else if (ok) {
            C->rs.nrem = nrem;
            C->rs.rsel = Rc == P.R1 ? 1u : 0u;
            C->rs.epoch = e;
            C->rs.iters = iters0 + iters;
            C->rs.done = finished;
            C->rs.want = next_want;
            C->rs.mid = 0;
            __threadfence();
        }
    }
    if (MODE == 1) loop_control(P, C);   // thread 0 is the leader: its writes above come first
}

int maintain_blocks_per_sm(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, maintain_kernel<0>, threads, 0) != cudaSuccess) return 0;
    return nb;
}

// Cooperative (co-resident blocks, which the grid barrier needs); the
// attribute form also records into a graph under stream capture.
cudaError_t launch_maintain(const MaintainParams& p, int blocks, int threads, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, maintain_kernel<0>, p);
}

const void* maintain_kernel_symbol(int mode) {
    return mode == 0 ? (const void*)maintain_kernel<0> : (const void*)maintain_kernel<1>;
}

cudaError_t launch_maintain_block(const MaintainParams& p, int threads, cudaStream_t s) {
    (void)threads;
    maintain_kernel<1><<<1, kBlockThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace cm
