// cm_common.cuh -- device-side layout and primitives shared by the kernels.
//
// Device layout of one graph (all arrays indexed by vertex id unless noted):
//   hc[v]   int2  {core, SD}: core is the core number (-1 dead); SD is the
//           superior degree (Section IV, Definition 7: neighbours with core
//           >= core(v)).  Scans read it only where the exact SD matters
//           (a core-k neighbour in a deletion scan, an edge level during a
//           deletion); everything else reads the key kc below.
//   hw[v]   u64   the per-iteration word: low 32 bits a stamp (iteration << 2
//           | flags), high 32 bits a count (insert: visited / processed
//           flags and support; delete: evicted-neighbour count).  Scans load
//           it only for the neighbours that can be candidates at their level.
//   kc[v]   u32   core(v) << 1 | (SD(v) > core(v)): all an insert scan needs
//           to know of a neighbour besides its per-iteration word (CSD,
//           Definition 8, counts neighbours above k and core-k neighbours
//           with SD > k; the candidates are the latter).  4 bytes per vertex:
//           at 2^24 vertices the array (67 MB) fits in L2.  Every write of a
//           core or an SD updates it (see key_of and its callers).
//   off[v]  int64 first adjacency slot; end[v] used slots (live + holes);
//   cap[v]  allocated slots (multiple of 4, so lists start 16-byte aligned);
//   deg[v]  live degree.  adj[] holds neighbour ids, HOLE (-1) for a deleted
//           entry.  Slack CSR: cap ~ (1 + slack) * degree.
//   chg[v]  epoch in which v's core last changed; taken[v] selection stamp;
//   claim0/claim1[v] 64-bit claim words (two buffers alternate per round).
//   need[v] pending insertions of the current call (capacity check).
//   idx[]   open-addressing edge index: canonical key (lo<<32|hi) -> the
//           slot of hi in adj(lo) and of lo in adj(hi).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cm {

constexpr int32_t HOLE = -1;
// SD value of a vertex being deleted (a pinned vertex): during the call its
// core stays fixed, it constrains no edge, it never becomes a root and its
// support never runs out (see cm_delete_vertices)
constexpr int32_t PIN_SD = 1 << 30;
constexpr unsigned long long KEY_EMPTY = 0xFFFFFFFFFFFFFFFFull;
constexpr unsigned long long KEY_TOMB = 0xFFFFFFFFFFFFFFFEull;
constexpr unsigned long long CLAIM_FREE = 0xFFFFFFFFFFFFFFFFull;

// device error codes (Ctl::error)
constexpr int E_BARRIER_TIMEOUT = 1;
constexpr int E_ITER_LIMIT = 2;
constexpr int E_CAPACITY = 3;
constexpr int E_INVALID = 4;
constexpr int E_INDEX_FULL = 5;
constexpr int E_TASKS = 6;              // the grid-mode task queue ran out of slots

struct __align__(16) Bucket {
    unsigned long long key;
    int32_t slo;   // slot of hi in adj(lo); -2 while pending
    int32_t shi;   // slot of lo in adj(hi)
};

// A remaining edge of the current batch (16 bytes).
struct __align__(16) REdge {
    int32_t lo, hi;
    uint32_t bkt;    // index bucket
    uint32_t flags;  // bit0 selected, bit1 blocked, bits 2.. last claim round + 1
};
constexpr uint32_t F_SEL = 1u, F_BLK = 2u;

// Stats slots (Ctl::st)
enum {
    ST_ITERS = 0, ST_ROUNDS, ST_SELECTED, ST_REMSUM, ST_VISITED, ST_VISSLOTS, ST_EVICTED, ST_EVSLOTS,
    ST_CHANGED, ST_CHSLOTS, ST_WAVES, ST_LEVELS, ST_BARRIERS, ST_GRID_ITERS, ST_COUNT
};
// Phase ids of the per-phase timers (Ctl::ph)
enum { PH_CLAIM = 0, PH_CHECK, PH_APPLY, PH_DISCOVER, PH_EVICT, PH_COMMIT, PH_FIXUP, PH_COUNT };

// Where a maintenance launch resumes: written by the host before the first
// launch of a call and by a kernel that hands the call over to the other
// execution mode (grid-wide or single-block) at an iteration boundary.
struct Resume {
    unsigned long long nrem;   // remaining edges (mid: those left for the next iteration)
    uint32_t rsel;             // which remaining-edge buffer holds them
    uint32_t epoch;            // next iteration's stamp (mid: the current one)
    int done;                  // every edge applied
    int want;                  // 0: grid mode next, 1: single-block mode next
    long long iters;           // completed iterations (for the cap)
    int mid;                   // 1: resume inside the search waves of iteration `epoch`
    int pad;
    // mid-search state: ring positions at the iteration's start and the
    // pending frontier / eviction ranges of the next wave
    unsigned long long vq0, eq0, cq0, flo, fhi, elo, ehi;
};

constexpr int kTails = 4;

// A vertex whose adjacency is scanned by all warps of a grid-mode launch,
// in chunk tasks of kChunk slots (32 bytes; a ring of kHubRing per handle).
// kind: HUB_FRONT (insert frontier: chunks sum CSD, the last one decides),
// HUB_EVICT_INS / HUB_EVICT_DEL (eviction scans), HUB_EXPAND (visit the
// frontier neighbours of a hub whose support stayed above k).
// HUB_FRONT_SPEC: as HUB_FRONT, but each chunk also visits its candidates
// at once (speculative expansion, see process_frontier), so no HUB_EXPAND
// round follows.
enum { HUB_FRONT = 0, HUB_EVICT_INS = 1, HUB_EVICT_DEL = 2, HUB_EXPAND = 3, HUB_FRONT_SPEC = 4 };
struct __align__(16) HubItem {
    long long off;                 // adjacency offset
    int32_t v, kind, k, len;
    int32_t nch;                   // chunks
    int32_t acc;                   // partial-sum accumulator (HUB_FRONT)
    uint32_t done;                 // chunks finished
    int32_t pad;
};
constexpr int kChunk = 512;                 // slots per chunk: four 4-wide passes of one warp
constexpr unsigned long long kHubRing = 1ull << 20;
constexpr unsigned long long kHubRingSafe = kHubRing - 4096;   // items in flight stay below this

// Device control block, one per handle.  The barrier words and counters are
// 64-bit and monotone within a launch where noted.
struct __align__(128) Ctl {
    unsigned long long arrive;     // grid barrier: arrivals (monotone in a launch)
    unsigned long long release;    // grid barrier: released generation
    int error;                     // first device error (E_*)
    int err_info;
    // ring tails (monotone in a call): 0 VQ, 1 EQ, 2 CQ, 3 spare.  Counters
    // that every warp updates during a search sit on lines of their own
    // (128 bytes apart), so their atomics do not queue behind one another.
    alignas(128) unsigned long long tail[kTails];
    alignas(128) unsigned long long pc[kTails];     // phase counters, copied to spc and zeroed at every barrier
    alignas(128) unsigned long long stail[kTails];  // snapshot of tail at the last barrier
    unsigned long long spc[kTails];    // snapshot of pc at the last barrier
    unsigned long long st[ST_COUNT];
    unsigned long long ph[PH_COUNT];   // nanoseconds per phase (block 0's view)
    // ingest / host exchange
    unsigned long long nrem;       // edges kept by ingest
    unsigned long long noverflow;  // vertices whose capacity the batch exceeds
    unsigned long long reloc_need; // slots needed to relocate them
    unsigned long long adj_top;    // bump pointer of the adjacency pool
    long long bad_index;           // smallest invalid input position
    unsigned long long gather_n;   // gathered incident edges (vertex deletion)
    int min_deg;                   // peel: smallest remaining degree
    int defer;                     // captured step: skip its remaining kernels (1 pool short, 2 error)
    unsigned long long passes;     // captured step: launch pairs of the current phase
    // grid-mode task queue of the current search (reset before each search)
    alignas(128) unsigned long long task_head;  // next slot a warp claims
    alignas(128) unsigned long long task_tail;  // slots reserved by producers
    alignas(128) unsigned long long task_done;  // tasks finished
    alignas(128) unsigned long long hub_created;    // hub items of the current search
    unsigned long long hub_finished;
    alignas(128) Resume rs;
};

// What a captured update step records per phase (0 insert, 1 delete) for
// the host to read after the replay.
struct StepLog {
    unsigned long long st[2][ST_COUNT];
    unsigned long long ph[2][PH_COUNT];
    unsigned long long kept[2];    // edges kept by ingest
    unsigned long long passes[2];
    long long iters_end[2];
    int error[2];
    int defer;                     // phase at which the step stopped (+1), 0 if it ran to the end
    uint32_t epoch_end;
};

// Plain-old-data view of a graph passed to kernels by value.
struct DevGraph {
    int32_t n;             // vertex count (ids < n)
    int32_t slack_pct;
    int32_t min_cap;
    int32_t pad;
    int2* hc;
    unsigned long long* hw;
    uint32_t* kc;
    int64_t* off;
    int32_t* end;
    int32_t* cap;
    int32_t* deg;
    int32_t* adj;
    uint32_t* chg;
    uint32_t* taken;
    unsigned long long* claim0;
    unsigned long long* claim1;
    int32_t* need;
    Bucket* idx;
    unsigned long long idx_mask;
    int64_t adj_cap;
};

// The insert-scan key of a vertex with core `core` and superior degree sd;
// a dead vertex (core -1) reads back as core -1.
__device__ __forceinline__ uint32_t key_of(int core, int sd) {
    return ((uint32_t)core << 1) | (sd > core ? 1u : 0u);
}
__device__ __forceinline__ int key_core(uint32_t key) { return (int32_t)key >> 1; }
constexpr uint32_t KEY_DEAD = 0xFFFFFFFFu;

// ---------------------------------------------------------------- hashing
// MurmurHash3 64-bit finaliser (Appleby, public domain): a bijection, used
// both to place keys in the index and as the selection priority of an edge.
__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}
__device__ __forceinline__ unsigned long long ekey(int32_t a, int32_t b) {
    uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    return ((unsigned long long)lo << 32) | hi;
}

// Find a key in the index; returns the bucket or -1.
__device__ __forceinline__ long long idx_find(const Bucket* idx, unsigned long long mask, unsigned long long key) {
    unsigned long long b = fmix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; probe++) {
        unsigned long long k = idx[b].key;
        if (k == key) return (long long)b;
        if (k == KEY_EMPTY) return -1;
        b = (b + 1) & mask;
    }
    return -1;
}
// Insert a key if absent.  Returns bucket, with *existed set; -1 if full.
__device__ __forceinline__ long long idx_insert(Bucket* idx, unsigned long long mask, unsigned long long key, bool* existed) {
    unsigned long long b = fmix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; probe++) {
        unsigned long long k = idx[b].key;
        if (k == key) { *existed = true; return (long long)b; }
        if (k == KEY_EMPTY) {
            unsigned long long old = atomicCAS(&idx[b].key, KEY_EMPTY, key);
            if (old == KEY_EMPTY) { *existed = false; return (long long)b; }
            if (old == key) { *existed = true; return (long long)b; }
        }
        b = (b + 1) & mask;
    }
    return -1;
}

// ---------------------------------------------------------------- timing / sync
__device__ __forceinline__ void vstore64(unsigned long long* p, unsigned long long v) {
    *(volatile unsigned long long*)p = v;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A load with acquire semantics at device scope (later loads of this
// thread see at least what the writer released before the loaded value).
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long vload64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ int vload32(const int* p) { return *(const volatile int*)p; }

// Grid-wide barrier for a cooperative (co-resident) launch.  Every wait is
// bounded by limit_ns: past it the block records E_BARRIER_TIMEOUT and
// returns.  The last block to arrive copies the live tails and phase
// counters into their snapshots and zeroes the phase counters before it
// releases the others, so after the barrier every block reads the same
// snapshot.  `expect` is the number of blocks the barrier waits for
// (gridDim.x in production).  Returns false once an error is recorded.
__device__ __forceinline__ bool grid_sync(Ctl* c, unsigned int expect, unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long t = atomicAdd(&c->arrive, 1ull);
        unsigned long long gen = t / expect;
        if (t % expect == expect - 1) {
            for (int i = 0; i < kTails; i++) {
                c->stail[i] = vload64(&c->tail[i]);
                c->spc[i] = vload64(&c->pc[i]);
                c->pc[i] = 0;
            }
            __threadfence();
            atomicExch(&c->release, gen + 1);
        } else {
            unsigned long long t0 = gtimer();
            unsigned int spins = 0;
            while (vload64(&c->release) < gen + 1) {
                if (vload32(&c->error)) break;
                if ((++spins & 63u) == 0 && gtimer() - t0 > limit_ns) {
                    atomicCAS(&c->error, 0, E_BARRIER_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = vload32(&c->error) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// The same contract for a launch of one block: __syncthreads is the
// barrier and thread 0 takes the snapshots.
__device__ __forceinline__ bool block_sync(Ctl* c) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTails; i++) {
            c->stail[i] = vload64(&c->tail[i]);
            c->spc[i] = vload64(&c->pc[i]);
            c->pc[i] = 0;
        }
        s_ok = vload32(&c->error) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Warp-aggregated append of `val` (where pred) to a ring buffer; all 32
// lanes of the warp must call it together.
__device__ __forceinline__ void warp_push(unsigned long long* tail, int32_t* ring, unsigned long long mask,
                                          bool pred, int32_t val) {
    unsigned int b = __ballot_sync(0xffffffffu, pred);
    if (!b) return;
    unsigned long long base = 0;
    int lane = lane_id();
    int leader = __ffs(b) - 1;
    if (lane == leader) base = atomicAdd(tail, (unsigned long long)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) ring[(base + __popc(b & ((1u << lane) - 1))) & mask] = val;
}

// Warp-aggregated append of a 16-byte edge to an array.
__device__ __forceinline__ void warp_push_edge(unsigned long long* tail, REdge* arr, bool pred, REdge e) {
    unsigned int b = __ballot_sync(0xffffffffu, pred);
    if (!b) return;
    unsigned long long base = 0;
    int lane = lane_id();
    int leader = __ffs(b) - 1;
    if (lane == leader) base = atomicAdd(tail, (unsigned long long)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) arr[base + __popc(b & ((1u << lane) - 1))] = e;
}

__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int round4(long long x) { return (int)((x + 3) & ~3ll); }

// Adjacency capacity for an expected degree d.
__device__ __forceinline__ int cap_for(long long d, int slack_pct, int min_cap) {
    long long c = (d * (100 + slack_pct) + 99) / 100;
    if (c < min_cap) c = min_cap;
    return round4(c);
}

}  // namespace cm
