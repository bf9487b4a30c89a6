// cm_vertex.cuh -- per-vertex work of the maintenance waves (included by
// cm_iterate.cu only).
//
// Each body scans one vertex's adjacency with a group of threads: one warp,
// or a whole block for a high-degree vertex.  Scans read the list four slots
// per thread with one 16-byte load (lists start 16-byte aligned and their
// capacity is a multiple of 4, so the load never leaves the list's
// allocation) and issue the four neighbour gathers before using any, so a
// warp keeps four independent loads in flight per lane.  Loops are
// warp-uniform, so warp collectives may run inside them.
//
// The per-iteration word of a vertex is hw[v], read and updated as one
// 64-bit value: low half z = stamp (iteration << 2 | flags), high half w = a
// count; a scan step sees it as the z / w fields of an int4 {core, SD, z, w}.  A word
// with an older stamp reads as "no flags, count 0"; the first update in an
// iteration stamps it with one CAS, later updates are single atomicAdd /
// atomicOr operations on the 64-bit word.  Insert flags: 1 visited (in a
// frontier), 2 processed (CSD added); w = support.  Delete: w = evicted
// neighbours.
#pragma once
#include "cm_common.cuh"
#include "cm_launch.h"

namespace cm {

constexpr uint32_t kVisited = 1u, kProcessed = 2u;

// Per-warp counters of one launch, added to the control block's 64-bit
// statistics when the launch ends.  32 bits each (registers are what the
// grid kernel is short of): a warp's share of one launch stays far below
// 2^32 vertices or list slots.
struct LocalStats {
    uint32_t vis = 0, visl = 0, ev = 0, evl = 0, ch = 0, chl = 0, sel = 0;
};

// ---------------------------------------------------------------- per-iteration word
__device__ __forceinline__ bool same_iter(uint32_t z, uint32_t e) { return (z >> 2) == e; }
__device__ __forceinline__ unsigned long long* iter_word(const DevGraph& g, int v) {
    return &g.hw[v];
}
__device__ __forceinline__ uint32_t wz(unsigned long long x) { return (uint32_t)x; }
__device__ __forceinline__ int32_t ww(unsigned long long x) { return (int32_t)(uint32_t)(x >> 32); }

// Stamps v's word with iteration e if it is older (count 0, no flags).
// `seen` is a value of the word the caller already read (from the 16-byte
// vertex gather), which saves a load: a word stamped e stays stamped e for
// the rest of the iteration.  Retries are bounded; past the bound an error
// is recorded.
__device__ __forceinline__ void make_current(const DevGraph& g, Ctl* C, int v, uint32_t e, unsigned long long seen) {
    if (same_iter(wz(seen), e)) return;
    unsigned long long* p = iter_word(g, v);
    unsigned long long old = seen;
    const unsigned long long fresh = (unsigned long long)(e << 2);
    for (int tries = 0; tries < (1 << 20); tries++) {
        if (same_iter(wz(old), e)) return;
        unsigned long long prev = atomicCAS(p, old, fresh);
        if (prev == old) return;
        old = prev;
    }
    atomicCAS(&C->error, 0, E_ITER_LIMIT);
}
__device__ __forceinline__ void make_current(const DevGraph& g, Ctl* C, int v, uint32_t e) {
    make_current(g, C, v, e, vload64(iter_word(g, v)));
}
__device__ __forceinline__ unsigned long long word_of(const int4& h) {
    return ((unsigned long long)(uint32_t)h.w << 32) | (uint32_t)h.z;
}

// Adds delta to v's count and low_add to its flag bits (only bits that are
// clear); returns the previous (flags, count) of iteration e.  A word that
// `seen` shows from an older iteration is restamped and updated by one CAS
// when nobody else touched it since.
__device__ __forceinline__ void add_word(const DevGraph& g, Ctl* C, int v, uint32_t e, int32_t delta,
                                         uint32_t low_add, uint32_t& oflags, int32_t& ocount,
                                         unsigned long long seen) {
    unsigned long long* p = iter_word(g, v);
    if (!same_iter(wz(seen), e)) {
        const unsigned long long want =
            ((unsigned long long)(uint32_t)delta << 32) | (unsigned long long)((e << 2) | low_add);
        const unsigned long long prev = atomicCAS(p, seen, want);
        if (prev == seen) {
            oflags = 0;
            ocount = 0;
            return;
        }
        seen = prev;
    }
    make_current(g, C, v, e, seen);
    unsigned long long old = atomicAdd(p, ((unsigned long long)(uint32_t)delta << 32) + (unsigned long long)low_add);
    oflags = wz(old) & 3u;
    ocount = ww(old);
}
__device__ __forceinline__ void add_word(const DevGraph& g, Ctl* C, int v, uint32_t e, int32_t delta,
                                         uint32_t low_add, uint32_t& oflags, int32_t& ocount) {
    add_word(g, C, v, e, delta, low_add, oflags, ocount, vload64(iter_word(g, v)));
}

// Marks v visited in iteration e; true if this call did it (one CAS when the
// word is still the older one `seen` shows).
__device__ __forceinline__ bool visit(const DevGraph& g, Ctl* C, int v, uint32_t e, unsigned long long seen) {
    unsigned long long* p = iter_word(g, v);
    if (!same_iter(wz(seen), e)) {
        const unsigned long long prev = atomicCAS(p, seen, (unsigned long long)((e << 2) | kVisited));
        if (prev == seen) return true;
        seen = prev;
    }
    make_current(g, C, v, e, seen);
    unsigned long long old = atomicOr(p, (unsigned long long)kVisited);
    return (wz(old) & kVisited) == 0;
}
__device__ __forceinline__ bool visit(const DevGraph& g, Ctl* C, int v, uint32_t e) {
    return visit(g, C, v, e, vload64(iter_word(g, v)));
}

// The same two operations for the four slots of a lane's scan step, with
// the four first atomics issued before any result is used; a slot whose
// word changed since it was gathered takes the slow path of add_word /
// visit.  Slots with want[q] / cand[q] false are left alone.
__device__ __forceinline__ void add_word4(const DevGraph& g, Ctl* C, const int (&v)[4], const bool (&want)[4],
                                          uint32_t e, int32_t delta, const unsigned long long (&seen)[4],
                                          uint32_t (&oflags)[4], int32_t (&ocount)[4]) {
    const unsigned long long inc = (unsigned long long)(uint32_t)delta << 32;
    const unsigned long long fresh = inc | (unsigned long long)(e << 2);
    unsigned long long r[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        r[q] = 0;
        if (want[q]) r[q] = same_iter(wz(seen[q]), e) ? atomicAdd(iter_word(g, v[q]), inc)
                                                       : atomicCAS(iter_word(g, v[q]), seen[q], fresh);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        oflags[q] = 0;
        ocount[q] = 0;
        if (!want[q]) continue;
        if (same_iter(wz(seen[q]), e)) {
            oflags[q] = wz(r[q]) & 3u;
            ocount[q] = ww(r[q]);
        } else if (r[q] != seen[q]) {   // someone touched it first: restamp if needed, then add
            make_current(g, C, v[q], e, r[q]);
            const unsigned long long old = atomicAdd(iter_word(g, v[q]), inc);
            oflags[q] = wz(old) & 3u;
            ocount[q] = ww(old);
        }
    }
}

__device__ __forceinline__ void visit4(const DevGraph& g, Ctl* C, const int (&v)[4], bool (&cand)[4], uint32_t e,
                                       const unsigned long long (&seen)[4]) {
    const unsigned long long fresh = (unsigned long long)((e << 2) | kVisited);
    unsigned long long r[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        r[q] = 0;
        if (cand[q]) r[q] = same_iter(wz(seen[q]), e) ? atomicOr(iter_word(g, v[q]), (unsigned long long)kVisited)
                                                       : atomicCAS(iter_word(g, v[q]), seen[q], fresh);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!cand[q]) continue;
        if (same_iter(wz(seen[q]), e)) cand[q] = (wz(r[q]) & kVisited) == 0;
        else if (r[q] != seen[q]) cand[q] = visit(g, C, v[q], e, r[q]);
    }
}

// ---------------------------------------------------------------- thread groups
// A group of threads sharing one vertex's adjacency: one warp, or the block.
struct WarpGroup {
    static constexpr int G = 32;
    __device__ static int first() { return 0; }                    // first thread of this warp in the group
    __device__ static bool rank0() { return lane_id() == 0; }
    __device__ static bool warp0() { return true; }
    __device__ static int sum(int v) { return warp_sum(v); }
};
template <int NT>
struct BlockGroup {
    static constexpr int G = NT;
    __device__ static int first() { return threadIdx.x & ~31; }
    __device__ static bool rank0() { return threadIdx.x == 0; }
    __device__ static bool warp0() { return threadIdx.x < 32; }
    __device__ static int sum(int v) {
        __shared__ int s_part[NT / 32];
        v = warp_sum(v);
        __syncthreads();
        if (lane_id() == 0) s_part[threadIdx.x >> 5] = v;
        __syncthreads();
        int t = 0;
        for (int i = 0; i < NT / 32; i++) t += s_part[i];
        return t;
    }
};

// ---------------------------------------------------------------- queue pushes
// A vertex that enters the frontier (insert) or is evicted goes to the
// visited log VQ / evicted log EQ of the iteration.  In the grid-wide mode
// (ASYNC) it also becomes a task of the iteration's task queue, which warps
// drain without level barriers (cm_iterate.cu).  All 32 lanes call these.
constexpr unsigned long long TASK_EMPTY = ~0ull;
enum { T_FRONT = 0, T_EVICT = 1, T_CHUNK = 2 };
constexpr int kTaskChunkBits = 22;          // chunk index within a hub item
constexpr unsigned long long kTaskMargin = 1ull << 16;   // slots kept free for claims past the tail

__device__ __forceinline__ unsigned long long mk_task(int type, unsigned long long payload) {
    return ((unsigned long long)type << 62) | payload;
}

// Appends tasks [tb, tb + n) (already reserved); false if the queue is full.
__device__ __forceinline__ bool task_room(Ctl* C, const MaintainParams& P, unsigned long long tb, unsigned long long n) {
    if (tb + n + kTaskMargin > P.tqmask + 1) {
        atomicCAS(&C->error, 0, E_TASKS);
        return false;
    }
    return true;
}

// The task a warp keeps for itself (grid mode).  Of the vertices a warp
// produces in the last scan step of its current task, the first is not
// queued: the warp runs it next, which saves the hand-off through the queue
// (the slot write, another warp's poll and its back-off) on every level of a
// dependency chain, such as a frontier vertex that fails and evicts itself or
// an eviction that evicts a neighbour.  The kept task is not counted in the
// queue's tail and is not reported done; the task that produced it is
// reported only after the warp has run it, so quiescence still waits for it.
constexpr int kGridWarps = 16;   // warps per grid-mode block
__shared__ unsigned long long s_keep[kGridWarps];
__device__ __forceinline__ unsigned long long& kept_task() { return s_keep[threadIdx.x >> 5]; }

// Pushes the vertices of the lanes with pred set (warp-collective).  keep:
// this is the task's last scan step, so the warp may keep one of them.
template <bool ASYNC>
__device__ __forceinline__ void push_vertex(Ctl* C, const MaintainParams& P, bool pred, int32_t v, int which,
                                            bool keep = false) {
    // which 0: frontier (VQ, T_FRONT), 1: eviction (EQ, T_EVICT)
    const unsigned int b = __ballot_sync(0xffffffffu, pred);
    if (!b) return;
    const int lane = lane_id();
    const int leader = __ffs(b) - 1;
    const unsigned long long cnt = (unsigned long long)__popc(b);
    if (ASYNC) keep = keep && kept_task() == TASK_EMPTY;   // the same value in every lane
    const unsigned long long nq = cnt - (ASYNC && keep ? 1 : 0);
    unsigned long long lb = 0, tb = 0;
    if (lane == leader) {
        lb = atomicAdd(&C->tail[which], cnt);
        if (ASYNC && nq) tb = atomicAdd(&C->task_tail, nq);
    }
    lb = __shfl_sync(0xffffffffu, lb, leader);
    const unsigned int rank = __popc(b & ((1u << lane) - 1));
    int32_t* log = which == 0 ? P.VQ : P.EQ;
    if (pred) log[(lb + rank) & P.qmask] = v;
    if (ASYNC) {
        tb = __shfl_sync(0xffffffffu, tb, leader);
        const unsigned long long task = mk_task(which == 0 ? T_FRONT : T_EVICT, (unsigned long long)v);
        const bool room = nq == 0 || task_room(C, P, tb, nq);
        if (pred && keep && rank == 0) kept_task() = task;
        else if (pred && room) vstore64(&P.TQ[(tb + rank - (keep ? 1 : 0)) & P.tqmask], task);
        __syncwarp();
    }
}

// The same for up to four vertices per lane (one scan step), with one
// atomic per queue for the whole warp.
template <bool ASYNC>
__device__ __forceinline__ void push_vertex4(Ctl* C, const MaintainParams& P, const bool pred[4], const int32_t v[4],
                                             int which, bool keep = false) {
    const int lane = lane_id();
    const int mine = (int)pred[0] + (int)pred[1] + (int)pred[2] + (int)pred[3];
    if (!__any_sync(0xffffffffu, mine != 0)) return;
    int incl = mine;   // inclusive prefix over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned long long total = (unsigned long long)__shfl_sync(0xffffffffu, incl, 31);
    if (ASYNC) keep = keep && kept_task() == TASK_EMPTY;
    const unsigned long long nq = total - (ASYNC && keep ? 1 : 0);
    unsigned long long lb = 0, tb = 0;
    if (lane == 31) {
        lb = atomicAdd(&C->tail[which], total);
        if (ASYNC && nq) tb = atomicAdd(&C->task_tail, nq);
    }
    lb = __shfl_sync(0xffffffffu, lb, 31);
    unsigned long long at = (unsigned long long)(incl - mine);
    int32_t* log = which == 0 ? P.VQ : P.EQ;
    bool room = true;
    if (ASYNC) {
        tb = __shfl_sync(0xffffffffu, tb, 31);
        room = nq == 0 || task_room(C, P, tb, nq);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!pred[q]) continue;
        log[(lb + at) & P.qmask] = v[q];
        if (ASYNC) {
            const unsigned long long task = mk_task(which == 0 ? T_FRONT : T_EVICT, (unsigned long long)v[q]);
            if (keep && at == 0) kept_task() = task;
            else if (room) vstore64(&P.TQ[(tb + at - (keep ? 1 : 0)) & P.tqmask], task);
        }
        at++;
    }
    if (ASYNC) __syncwarp();
}

// The words of a scan step's four neighbours as {core, SD, z, w}.  First
// the 4-byte key of every slot (core and whether SD > core), then, in a
// second round of loads, only for the slots that can be candidates at level
// k: the per-iteration word (insert: core k and SD > k) or the exact SD and
// the per-iteration word (delete, whose threshold is SD - k + 1: core k).
// The others get SD = core + the key bit and z = w = 0, which no body reads
// for a non-candidate.
__device__ __forceinline__ void gather4(const DevGraph& g, const int (&w)[4], int k, bool del, int4 (&h)[4]) {
    uint32_t key[4];
#pragma unroll
    for (int q = 0; q < 4; q++) key[q] = w[q] >= 0 ? g.kc[w[q]] : KEY_DEAD;
    int2 c[4];
    unsigned long long s[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int core = key_core(key[q]);
        c[q] = make_int2(core, core + (int)(key[q] & 1u));
        const bool need = core == k && (del || (key[q] & 1u));
        s[q] = need ? g.hw[w[q]] : 0ull;
        if (del && need) c[q].y = g.hc[w[q]].y;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) h[q] = make_int4(c[q].x, c[q].y, (int)(uint32_t)s[q], (int)(uint32_t)(s[q] >> 32));
}

// Four neighbour ids of this lane for the step starting at `base` (HOLE for
// slots at or past len).
__device__ __forceinline__ void load4(const DevGraph& g, long long o, int len, int t0, int w[4]) {
    int4 a = make_int4(HOLE, HOLE, HOLE, HOLE);
    if (t0 < len) a = __ldcs(reinterpret_cast<const int4*>(g.adj + o + t0));   // streamed: keep L2 for the keys
    w[0] = a.x;
    w[1] = t0 + 1 < len ? a.y : HOLE;
    w[2] = t0 + 2 < len ? a.z : HOLE;
    w[3] = t0 + 3 < len ? a.w : HOLE;
}

// Slots [s0, s1) of a list (s0 a multiple of 4), four per thread per step.
#define SCAN4_RANGE(Grp, s0, s1)                                                      \
    for (int base_ = (s0) + Grp::first() * 4; base_ < (s1); base_ += Grp::G * 4) {     \
        const int t0_ = base_ + lane_id() * 4;
#define SCAN4_BEGIN(Grp, len) SCAN4_RANGE(Grp, 0, len)
#define SCAN4_END }

// The same walk with the list read two steps ahead: each lane loads the
// 16-byte words of two consecutive steps before the first step's gathers,
// so a step's neighbour gathers do not wait behind its own list read.  List
// reads are streamed (evict-first) so that L2 keeps the per-vertex keys.
// Inside, `int w[4]` holds the step's four neighbour ids (HOLE past s1)
// and `last_` is set in the group's last step.
#define SCANP_RANGE(Grp, o, s0, s1)                                                              \
    for (int blk_ = (s0) + Grp::first() * 4; blk_ < (s1); blk_ += Grp::G * 8) {                  \
        int4 A_[2];                                                                               \
        _Pragma("unroll") for (int j_ = 0; j_ < 2; j_++) {                                         \
            const int t_ = blk_ + j_ * Grp::G * 4 + lane_id() * 4;                                \
            A_[j_] = t_ < (s1) ? __ldcs(reinterpret_cast<const int4*>(g.adj + (o) + t_))                 \
                               : make_int4(HOLE, HOLE, HOLE, HOLE);                               \
        }                                                                                         \
        _Pragma("unroll") for (int j_ = 0; j_ < 2; j_++) {                                         \
            if (blk_ + j_ * Grp::G * 4 >= (s1)) break;                                            \
            const int t0_ = blk_ + j_ * Grp::G * 4 + lane_id() * 4;                               \
            const bool last_ = blk_ + (j_ + 1) * Grp::G * 4 >= (s1);                              \
            int w[4];                                                                             \
            w[0] = A_[j_].x;                                                                      \
            w[1] = t0_ + 1 < (s1) ? A_[j_].y : HOLE;                                              \
            w[2] = t0_ + 2 < (s1) ? A_[j_].z : HOLE;                                              \
            w[3] = t0_ + 3 < (s1) ? A_[j_].w : HOLE;
#define SCANP_END \
        }         \
    }

// ---------------------------------------------------------------- range scans
// Each scan covers slots [s0, s1) of the list at offset o of a vertex at
// level k, so a vertex can be scanned whole by one group or in chunks by
// many blocks.

// This thread's part of CSD over the range (Definition 8 with the SD of
// Definition 7: neighbours above k, and core-k neighbours with SD > k).
template <class Grp>
__device__ __forceinline__ int csd_part(const DevGraph& g, int k, long long o, int s0, int s1) {
    int pcd = 0;
    SCANP_RANGE(Grp, o, s0, s1)
        uint32_t key[4];
#pragma unroll
        for (int q = 0; q < 4; q++) key[q] = w[q] >= 0 ? g.kc[w[q]] : KEY_DEAD;
#pragma unroll
        for (int q = 0; q < 4; q++) pcd += key_core(key[q]) > k || (key_core(key[q]) == k && (key[q] & 1u));
    SCANP_END
    return pcd;
}

// Visits the unvisited core-k neighbours with SD > k in the range and
// appends them to the next frontier.
template <class Grp, bool ASYNC>
__device__ __forceinline__ void expand_range(const DevGraph& g, Ctl* C, const MaintainParams& P, int k, long long o,
                                             int s0, int s1, uint32_t e) {
    SCANP_RANGE(Grp, o, s0, s1)
        int4 h[4];
        gather4(g, w, k, false, h);
        bool p[4];
        unsigned long long sw[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const bool seen = same_iter((uint32_t)h[q].z, e) && ((uint32_t)h[q].z & kVisited);
            p[q] = h[q].x == k && h[q].y > k && !seen;
            sw[q] = word_of(h[q]);
        }
        visit4(g, C, w, p, e, sw);
        push_vertex4<ASYNC>(C, P, p, w, 0, last_);
    SCANP_END
}

// CSD over the range (this thread's part, as csd_part) while visiting the
// range's unvisited core-k neighbours with SD > k in the same pass: the
// expansion of Algorithm 3 done before the vertex's support is known
// (speculative expansion, see process_frontier).
template <class Grp, bool ASYNC>
__device__ __forceinline__ int csd_expand_range(const DevGraph& g, Ctl* C, const MaintainParams& P, int k,
                                                long long o, int s0, int s1, uint32_t e) {
    int pcd = 0;
    SCANP_RANGE(Grp, o, s0, s1)
        int4 h[4];
        gather4(g, w, k, false, h);
        bool p[4];
        unsigned long long sw[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            pcd += (h[q].x > k) || (h[q].x == k && h[q].y > k);
            const bool seen = same_iter((uint32_t)h[q].z, e) && ((uint32_t)h[q].z & kVisited);
            p[q] = h[q].x == k && h[q].y > k && !seen;
            sw[q] = word_of(h[q]);
        }
        visit4(g, C, w, p, e, sw);
        push_vertex4<ASYNC>(C, P, p, w, 0, last_);
    SCANP_END
    return pcd;
}

// Whether a frontier vertex expands early: it visits its candidates in the
// same pass that sums its CSD, before its support is known to exceed k,
// which saves the second pass over its list (and, for a hub, a whole round
// of chunk tasks).  A vertex that then stays at or below k has visited
// vertices the paper's search (expand only once the support exceeds k,
// Algorithm 3) would not have; they are processed like any other and the
// cores are the same (see the design notes).  On R-MAT sweeps the visited
// vertices grow by about 1.5% and the inserts get up to 20% faster, so it
// is the default; expand_early = -1 restores the paper's order.
__device__ __forceinline__ bool expand_early(const MaintainParams& P, int sd, int k) {
    (void)sd;
    (void)k;
    return P.expand_early >= 0;
}

// InsertRemove over the range (Algorithm 4): every core-k neighbour with
// SD > k (visited or not) loses one support; a processed one whose support
// falls to k leaves too.
template <class Grp, bool ASYNC>
__device__ __forceinline__ void evict_ins_range(const DevGraph& g, Ctl* C, const MaintainParams& P, int k,
                                                long long o, int s0, int s1, uint32_t e) {
    SCANP_RANGE(Grp, o, s0, s1)
        int4 h[4];
        gather4(g, w, k, false, h);
        bool cand[4], p[4];
        unsigned long long sw[4];
        uint32_t of[4];
        int32_t oc[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const bool gone = same_iter((uint32_t)h[q].z, e) && ((uint32_t)h[q].z & kProcessed) && h[q].w <= k;
            cand[q] = h[q].x == k && h[q].y > k && !gone;
            sw[q] = word_of(h[q]);
        }
        add_word4(g, C, w, cand, e, -1, sw, of, oc);
#pragma unroll
        for (int q = 0; q < 4; q++) p[q] = cand[q] && (of[q] & kProcessed) && oc[q] == k + 1;
        push_vertex4<ASYNC>(C, P, p, w, 1, last_);
    SCANP_END
}

// DeleteRemove over the range (Algorithm 7): each core-k neighbour w loses
// one support (initially SD(w)) and leaves when it falls below k, i.e. when
// its count of evicted neighbours reaches SD(w) - k + 1.
template <class Grp, bool ASYNC>
__device__ __forceinline__ void evict_del_range(const DevGraph& g, Ctl* C, const MaintainParams& P, int k,
                                                long long o, int s0, int s1, uint32_t e) {
    SCANP_RANGE(Grp, o, s0, s1)
        int4 h[4];
        gather4(g, w, k, true, h);
        uint32_t c[4];
#pragma unroll
        for (int q = 0; q < 4; q++) c[q] = h[q].x == k ? g.chg[w[q]] : 0u;   // only core-k slots can be candidates
        bool cand[4], p[4];
        unsigned long long sw[4];
        uint32_t of[4];
        int32_t oc[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int thr = h[q].y - k + 1;
            const bool gone = thr <= 0 || (same_iter((uint32_t)h[q].z, e) && h[q].w >= thr);
            // evicted vertices (chg == e) are skipped: their cores already
            // dropped, so one that fell from k+1 would pass for level k
            cand[q] = h[q].x == k && !gone && c[q] != e;
            sw[q] = word_of(h[q]);
        }
        add_word4(g, C, w, cand, e, 1, sw, of, oc);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            p[q] = cand[q] && oc[q] + 1 == h[q].y - k + 1;
            if (p[q]) g.chg[w[q]] = e;
        }
        push_vertex4<ASYNC>(C, P, p, w, 1, last_);
    SCANP_END
}

// ---------------------------------------------------------------- per-vertex phase bodies
// A task's vertex: {core, SD}, its per-iteration word, list offset and
// length, loaded together (independent loads) before anything uses them.
struct VInfo {
    int4 h;
    long long o;
    int len;
};
__device__ __forceinline__ VInfo load_vinfo(const DevGraph& g, int v) {
    VInfo r;
    const int2 c = g.hc[v];
    const unsigned long long x = g.hw[v];
    r.h = make_int4(c.x, c.y, (int)(uint32_t)x, (int)(uint32_t)(x >> 32));
    r.o = g.off[v];
    r.len = g.end[v];
    return r;
}

// Positive search step (Algorithm 3) for a frontier vertex v at level k:
// support += CSD(v); above k -> visit the unvisited core-k neighbours with
// SD > k, else v is evicted.
template <class Grp, bool ASYNC>
__device__ __forceinline__ void process_frontier(const DevGraph& g, Ctl* C, const MaintainParams& P, int v,
                                                 const VInfo& vi, uint32_t e, LocalStats& ls) {
    const int lane = lane_id();
    const int k = vi.h.x;
    const long long o = vi.o;
    const int len = vi.len;
    if constexpr (Grp::G == 32) {
        if (len <= 128) {   // one scan step: CSD and expansion from the same gathers
            int w[4];
            load4(g, o, len, lane * 4, w);
            int4 h[4];
            gather4(g, w, k, false, h);
            int part = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) part += (h[q].x > k) || (h[q].x == k && h[q].y > k);
            const int pcd = warp_sum(part);
            int32_t sup = 0;
            if (lane == 0) {
                uint32_t of;
                int32_t oc;
                add_word(g, C, v, e, pcd, kProcessed, of, oc, word_of(vi.h));
                sup = oc + pcd;
                ls.vis++;
                ls.visl += len;
            }
            sup = __shfl_sync(0xffffffffu, sup, 0);
            if (sup > k) {
                bool p[4];
                unsigned long long sw[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const bool seen = same_iter((uint32_t)h[q].z, e) && ((uint32_t)h[q].z & kVisited);
                    p[q] = h[q].x == k && h[q].y > k && !seen;
                    sw[q] = word_of(h[q]);
                }
                visit4(g, C, w, p, e, sw);
                push_vertex4<ASYNC>(C, P, p, w, 0, true);
            } else {
                push_vertex<ASYNC>(C, P, lane == 0, v, 1, true);
            }
            return;
        }
    }
    const bool early = expand_early(P, vi.h.y, k);
    const int pcd = Grp::sum(early ? csd_expand_range<Grp, ASYNC>(g, C, P, k, o, 0, len, e)
                                   : csd_part<Grp>(g, k, o, 0, len));
    int32_t sup = 0;
    if (Grp::rank0()) {
        uint32_t of;
        int32_t oc;
        add_word(g, C, v, e, pcd, kProcessed, of, oc, word_of(vi.h));
        sup = oc + pcd;
        ls.vis++;
        ls.visl += len;
    }
    if constexpr (Grp::G == 32) {
        sup = __shfl_sync(0xffffffffu, sup, 0);
    } else {
        sup = Grp::sum(Grp::rank0() ? sup : 0);
    }
    if (sup > k) {
        if (!early) expand_range<Grp, ASYNC>(g, C, P, k, o, 0, len, e);
    } else if (Grp::warp0()) {
        push_vertex<ASYNC>(C, P, lane == 0, v, 1, Grp::G == 32);
    }
}

// InsertRemove step (Algorithm 4) for an evicted vertex v.
template <class Grp, bool ASYNC>
__device__ __forceinline__ void evict_insert_vertex(const DevGraph& g, Ctl* C, const MaintainParams& P,
                                                    const VInfo& vi, uint32_t e, LocalStats& ls) {
    const int len = vi.len;
    evict_ins_range<Grp, ASYNC>(g, C, P, vi.h.x, vi.o, 0, len, e);
    if (Grp::rank0()) {
        ls.ev++;
        ls.evl += len;
    }
}

// DeleteRemove step (Algorithm 7) for an evicted vertex v, which drops to k-1.
template <class Grp, bool ASYNC>
__device__ __forceinline__ void evict_delete_vertex(const DevGraph& g, Ctl* C, const MaintainParams& P, int v,
                                                    const VInfo& vi, uint32_t e, LocalStats& ls) {
    const int k = vi.h.x;
    const int len = vi.len;
    evict_del_range<Grp, ASYNC>(g, C, P, k, vi.o, 0, len, e);
    if constexpr (Grp::G > 32) __syncthreads();   // every warp has read k before it changes
    if (Grp::rank0()) {
        g.hc[v].x = k - 1;
        g.kc[v] = key_of(k - 1, 0);   // bit set by the SD fix-up
        ls.ev++;
        ls.evl += len;
    }
}

// SD fix-up of a vertex whose core moved in iteration e (op 0 rose, op 1 dropped).
template <class Grp>
__device__ __forceinline__ void fixup_vertex(const DevGraph& g, int v, uint32_t e, int op, LocalStats& ls) {
    const int kn = g.hc[v].x;
    const long long o = g.off[v];
    const int len = g.end[v];
    const int adj_core = op == 0 ? kn : kn + 1;   // neighbours whose SD counts v differently now
    int sd = 0;
    SCANP_RANGE(Grp, o, 0, len)
        int cw[4];   // cores from the keys (a core change rewrites the key with it)
#pragma unroll
        for (int q = 0; q < 4; q++) cw[q] = w[q] >= 0 ? key_core(g.kc[w[q]]) : -1;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (w[q] < 0) continue;
            sd += cw[q] >= kn;
            if (cw[q] == adj_core && g.chg[w[q]] != e) {
                // the key bit of w (SD > its core adj_core) moves with its SD:
                // all of this phase's changes to w go the same way, so only
                // the update that crosses the core sets (insert) or clears it
                if (op == 0) {
                    if (atomicAdd(&g.hc[w[q]].y, 1) == adj_core) atomicOr(&g.kc[w[q]], 1u);
                } else {
                    if (atomicSub(&g.hc[w[q]].y, 1) == adj_core + 1) atomicAnd(&g.kc[w[q]], ~1u);
                }
            }
        }
    SCANP_END
    sd = Grp::sum(sd);
    if (Grp::rank0()) {
        g.hc[v].y = sd;
        g.kc[v] = key_of(kn, sd);
        ls.ch++;
        ls.chl += len;
    }
}

}  // namespace cm
