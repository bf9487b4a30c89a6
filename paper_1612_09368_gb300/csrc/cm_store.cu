// cm_store.cu -- device graph store: construction, full decomposition by
// bucket peeling, superior degrees, vertex insertion/deletion helpers and
// export.
#include "cm_common.cuh"
#include "cm_launch.h"

namespace cm {

constexpr uint32_t BKT_DROP = 0xFFFFFFFFu;
constexpr int UNPEELED = -2;

static inline unsigned grid_for(long long n, int t, long long cap = 1 << 20) {
    long long b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// ------------------------------------------------------------------ construction
// Validate ids, drop self-loops and repeats (first index insertion wins),
// record each kept edge's bucket.
__global__ void build_index_kernel(const int32_t* __restrict__ E, long long m, DevGraph g, uint32_t* ebkt, Ctl* c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int32_t u = E[2 * i], v = E[2 * i + 1];
    ebkt[i] = BKT_DROP;
    if (u < 0 || v < 0 || u >= g.n || v >= g.n) {
        atomicMin(&c->bad_index, i);
        atomicCAS(&c->error, 0, E_INVALID);
        return;
    }
    if (u == v) return;
    bool existed = false;
    long long b = idx_insert(g.idx, g.idx_mask, ekey(u, v), &existed);
    if (b < 0) { atomicCAS(&c->error, 0, E_INDEX_FULL); return; }
    if (existed) return;
    g.idx[b].slo = -2;
    g.idx[b].shi = -2;
    ebkt[i] = (uint32_t)b;
}

__global__ void count_degrees_kernel(const int32_t* __restrict__ E, const uint32_t* __restrict__ ebkt, long long m,
                                     DevGraph g) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || ebkt[i] == BKT_DROP) return;
    atomicAdd(&g.deg[E[2 * i]], 1);
    atomicAdd(&g.deg[E[2 * i + 1]], 1);
}

// Sum of capacities (into c->reloc_need) when sum_only, else assign each
// vertex of [v0, v1) a slot range by a warp-level scan and one pool
// allocation per warp.
__global__ void offsets_kernel(DevGraph g, int32_t v0, int32_t v1, Ctl* c, int sum_only) {
    long long base = (long long)v0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll);
    long long stride = (long long)gridDim.x * blockDim.x;
    int lane = lane_id();
    for (; base < v1; base += stride) {
        long long v = base + lane;
        int cp = 0;
        if (v < v1) cp = cap_for(g.deg[v], g.slack_pct, g.min_cap);
        int incl = cp;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long wb = 0;
        if (lane == 31) wb = atomicAdd(sum_only ? &c->reloc_need : &c->adj_top, (unsigned long long)tot);
        wb = __shfl_sync(0xffffffffu, wb, 31);
        if (!sum_only && v < v1) {
            g.off[v] = (int64_t)(wb + incl - cp);
            g.cap[v] = cp;
            g.end[v] = 0;
        }
    }
}

__global__ void scatter_kernel(const int32_t* __restrict__ E, const uint32_t* __restrict__ ebkt, long long m,
                               DevGraph g) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint32_t b = ebkt[i];
    if (b == BKT_DROP) return;
    int32_t lo = min(E[2 * i], E[2 * i + 1]), hi = max(E[2 * i], E[2 * i + 1]);
    int pu = atomicAdd(&g.end[lo], 1), pv = atomicAdd(&g.end[hi], 1);
    g.adj[g.off[lo] + pu] = hi;
    g.adj[g.off[hi] + pv] = lo;
    g.idx[b].slo = pu;
    g.idx[b].shi = pv;
}

// Given cores (a checkpoint): core -1 marks a deleted vertex, which gets the
// dead key; a live vertex's key bit is set by the SD pass that follows.
__global__ void set_cores_kernel(const int32_t* __restrict__ cores, DevGraph g) {
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    const int c = cores[v];
    g.hc[v].x = c;
    g.kc[v] = c < 0 ? KEY_DEAD : key_of(c, 0);
}

// SD(v), Definition 7: neighbours with core >= core(v).  Warp per vertex;
// four slots per lane per step with one 16-byte list load (lists start
// 16-byte aligned and their capacity is a multiple of 4) and the four
// neighbour gathers issued before any is used.  The cores are read from a
// compact copy (4 bytes per vertex, which stays in L2 at the sizes here)
// instead of the 8-byte {core, SD} words.
__global__ void copy_cores_kernel(DevGraph g, int32_t* core) {
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    core[v] = g.hc[v].x;
}

__global__ void init_mcd_kernel(DevGraph g, int32_t v0, int32_t v1, const int32_t* __restrict__ core) {
    long long w = v0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < v1; w += nw) {
        int k = core[w];
        if (k < 0) continue;
        long long o = g.off[w];
        int len = g.end[w], sd = 0;
        for (int t0 = lane * 4; t0 < len; t0 += 128) {
            const int4 a = __ldcs(reinterpret_cast<const int4*>(g.adj + o + t0));
            const int x[4] = {a.x, t0 + 1 < len ? a.y : HOLE, t0 + 2 < len ? a.z : HOLE, t0 + 3 < len ? a.w : HOLE};
            int c[4];
#pragma unroll
            for (int q = 0; q < 4; q++) c[q] = x[q] >= 0 ? core[x[q]] : -1;
#pragma unroll
            for (int q = 0; q < 4; q++) sd += c[q] >= k;
        }
        sd = warp_sum(sd);
        if (lane == 0) {
            g.hc[w].y = sd;
            g.kc[w] = key_of(k, sd);
        }
    }
}

cudaError_t build_index(const int32_t* E, long long m, DevGraph g, uint32_t* ebkt, Ctl* c, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    build_index_kernel<<<grid_for(m, 256, 1ll << 31), 256, 0, s>>>(E, m, g, ebkt, c);
    return cudaGetLastError();
}
cudaError_t count_degrees(const int32_t* E, const uint32_t* ebkt, long long m, DevGraph g, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    count_degrees_kernel<<<grid_for(m, 256, 1ll << 31), 256, 0, s>>>(E, ebkt, m, g);
    return cudaGetLastError();
}
cudaError_t assign_offsets(DevGraph g, int32_t v0, int32_t v1, Ctl* c, cudaStream_t s) {
    if (v1 <= v0) return cudaSuccess;
    offsets_kernel<<<grid_for(v1 - v0, 256, 65536), 256, 0, s>>>(g, v0, v1, c, 0);
    return cudaGetLastError();
}
cudaError_t scatter_edges(const int32_t* E, const uint32_t* ebkt, long long m, DevGraph g, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    scatter_kernel<<<grid_for(m, 256, 1ll << 31), 256, 0, s>>>(E, ebkt, m, g);
    return cudaGetLastError();
}
cudaError_t set_cores(const int32_t* cores, DevGraph g, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    set_cores_kernel<<<grid_for(g.n, 256, 1ll << 31), 256, 0, s>>>(cores, g);
    return cudaGetLastError();
}
cudaError_t init_mcd(DevGraph g, int32_t v0, int32_t v1, int32_t* core_scratch, cudaStream_t s) {
    if (v1 <= v0) return cudaSuccess;
    copy_cores_kernel<<<grid_for(g.n, 256, 1ll << 31), 256, 0, s>>>(g, core_scratch);
    init_mcd_kernel<<<grid_for((long long)(v1 - v0) * 32, 256, 65536), 256, 0, s>>>(g, v0, v1, core_scratch);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ peeling
// Level-synchronous bucket peeling (the static O(m) decomposition the paper
// cites, run level by level): at level k every remaining vertex whose
// degree is <= k gets core k and leaves; each departure takes one degree
// from every remaining neighbour, and neighbours that reach k leave at the
// same level.  Empty levels are skipped to the smallest remaining degree.
//
// Working degrees only fall, one at a time, and a vertex leaves at level k
// exactly when its degree reaches k (the decrement from k + 1 to k, or the
// level's scan finding it at k).  So at the scan of level k every remaining
// vertex has degree >= k and every vertex that left has degree < k: the
// scan reads the working degree alone (never the vertex's {core, SD} word)
// to tell the three cases apart.
//
// A frontier vertex with at least kPeelBig slots is not scanned by the warp
// that takes it: its list is cut into kPeelChunk-slot chunk tasks that every
// warp takes after a barrier, so one high-degree vertex does not hold a whole
// sub-wave on a single warp.
//
// No counter is shared by the whole grid per vertex: the level scan
// compacts a tile of kScanTile entries per block in shared memory and
// appends it with one atomic per list; frontier vertices and chunk tasks
// are dealt to warps by index, not claimed; and the vertices a sub-wave
// peels collect in a per-warp shared buffer that reaches the frontier ring
// with one atomic per flush.  (With one atomic per warp per step on a few
// counters, the serialised atomics at those counters were most of the
// peel's time.)
constexpr int kPeelThreads = 512;
constexpr int kPeelWarps = kPeelThreads / 32;
constexpr int kPeelBig = 2048;
constexpr int kPeelChunk = 512;
constexpr unsigned long long kPeelNoTask = ~0ull;
constexpr int kScanTile = 4 * kPeelThreads;   // list entries per block and scan step
constexpr int kPushBuf = 256;                 // per-warp buffer of peeled vertices
constexpr int kPushFlush = kPushBuf - 128;    // a scan step adds at most 128

struct PeelShared {
    int32_t keep[kScanTile];            // level scan: survivors of the tile
    int32_t peel[kScanTile];            // level scan: vertices of degree k
    int32_t buf[kPeelWarps][kPushBuf];  // sub-waves: peeled vertices per warp
    int wcnt[kPeelWarps];
    int nkeep, npeel, mx;
    unsigned long long kbase, pbase, wbase;
};

// Appends the warp's buffered vertices to the frontier ring (one atomic).
__device__ __forceinline__ void flush_peeled(Ctl* C, const PeelParams& P, int32_t* buf, int& cnt) {
    if (cnt == 0) return;
    unsigned long long b = 0;
    if (lane_id() == 0) b = atomicAdd(&C->tail[0], (unsigned long long)cnt);
    b = __shfl_sync(0xffffffffu, b, 0);
    for (int i = lane_id(); i < cnt; i += 32) P.F[b + i] = buf[i];
    __syncwarp();
    cnt = 0;
}

// End of a sub-wave: the block's warps append their buffers to the frontier
// ring together, with one atomic.  Every thread of the block calls it.
__device__ __forceinline__ void block_flush_peeled(Ctl* C, const PeelParams& P, PeelShared& S, int& cnt) {
    const int wib = threadIdx.x >> 5;
    if (lane_id() == 0) S.wcnt[wib] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int i = 0; i < kPeelWarps; i++) tot += S.wcnt[i];
        S.wbase = tot ? atomicAdd(&C->tail[0], (unsigned long long)tot) : 0;
    }
    __syncthreads();
    int pre = 0;
    for (int i = 0; i < wib; i++) pre += S.wcnt[i];
    for (int i = lane_id(); i < cnt; i += 32) P.F[S.wbase + pre + i] = S.buf[wib][i];
    cnt = 0;
}

// Slots [s0, s1) of the list at offset o (s0 a multiple of 4) at level k:
// one degree off every neighbour; a neighbour that reaches k leaves now and
// goes to the warp's buffer.  Four slots per lane per step with one 16-byte
// load (lists start 16-byte aligned, capacities are multiples of 4).
// Warp-collective.
__device__ __forceinline__ void peel_range(const DevGraph& g, const PeelParams& P, Ctl* C, long long o, int s0,
                                           int s1, int k, int32_t* buf, int& cnt) {
    const int lane = lane_id();
    for (int base = s0; base < s1; base += 128) {
        const int t0 = base + lane * 4;
        int4 a = make_int4(HOLE, HOLE, HOLE, HOLE);
        if (t0 < s1) a = __ldcs(reinterpret_cast<const int4*>(g.adj + o + t0));
        const int w[4] = {a.x, t0 + 1 < s1 ? a.y : HOLE, t0 + 2 < s1 ? a.z : HOLE, t0 + 3 < s1 ? a.w : HOLE};
        int r[4];
#pragma unroll
        for (int q = 0; q < 4; q++) r[q] = w[q] >= 0 ? atomicSub(&P.dcur[w[q]], 1) : 0;
        int mine = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) mine += w[q] >= 0 && r[q] == k + 1;
        if (!__any_sync(0xffffffffu, mine != 0)) continue;
        int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        int at = cnt + incl - mine;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (w[q] >= 0 && r[q] == k + 1) {
                g.hc[w[q]].x = k;
                buf[at++] = w[q];
            }
        }
        cnt += __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        if (cnt > kPushFlush) flush_peeled(C, P, buf, cnt);
    }
}

// The peel's grid barrier.  The contract of grid_sync (the last block to
// arrive copies the live tails and phase counters into their snapshots and
// zeroes the counters before it releases the others; false once an error
// is recorded), with the ordering carried by the operations themselves: the
// arrival is an acquire-release add, the release a release store that also
// carries the error state, each waiter's poll an acquire load.  The peel
// runs ~5 barrier-separated phases per level, so the barrier's critical
// path (last arrival, snapshot, release, the waiters' next poll) is a large
// part of its time.  The release word is (generation << 1) | error; the
// launch zone is zeroed before every peel launch.
__device__ __forceinline__ bool peel_sync(Ctl* c, unsigned int expect, unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], 1;" : "=l"(t) : "l"(&c->arrive) : "memory");
        const unsigned long long gen = t / expect;
        int ok = 1;
        if (t % expect == expect - 1) {
            for (int i = 0; i < kTails; i++) {
                c->stail[i] = vload64(&c->tail[i]);
                c->spc[i] = vload64(&c->pc[i]);
                c->pc[i] = 0;
            }
            ok = vload32(&c->error) == 0;
            const unsigned long long rel = ((gen + 1) << 1) | (ok ? 0ull : 1ull);
            asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(&c->release), "l"(rel) : "memory");
        } else {
            const unsigned long long t0 = gtimer();
            unsigned int spins = 0;
            for (;;) {
                const unsigned long long rel = ld_acquire64(&c->release);
                if ((rel >> 1) >= gen + 1) {
                    ok = (rel & 1ull) == 0;
                    break;
                }
                if (vload32(&c->error)) {
                    ok = 0;
                    break;
                }
                if ((++spins & 63u) == 0 && gtimer() - t0 > limit_ns) {
                    atomicCAS(&c->error, 0, E_BARRIER_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Phases of the peel timed at its barriers (block 0's view, into Ctl::ph):
// the level scans, the sub-waves and the chunk phases.
enum { PP_SCAN = 0, PP_WAVE = 1, PP_CHUNK = 2 };
struct PeelClock {
    Ctl* c;
    unsigned long long t;
    bool on;
    __device__ bool sync(const PeelParams& P, int phase) {
        const bool ok = peel_sync(c, P.expect, P.limit_ns);
        if (on) {
            const unsigned long long now = gtimer();
            c->ph[phase] += now - t;
            c->st[ST_BARRIERS] += 1;
            t = now;
        }
        return ok;
    }
};

__global__ void __launch_bounds__(kPeelThreads) peel_kernel(PeelParams P) {
    Ctl* C = P.ctl;
    const DevGraph g = P.g;
    __shared__ PeelShared S;
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long gwarp = gtid >> 5, nwarps = nthr >> 5;
    int32_t* buf = S.buf[wib];
    int cnt = 0;
    PeelClock clk{C, gtimer(), blockIdx.x == 0 && threadIdx.x == 0};
    // live vertices start unpeeled with their live degree (compacted into
    // the remaining list a tile at a time, like the level scans below)
    for (long long t0 = (long long)blockIdx.x * kScanTile; t0 < g.n; t0 += (long long)gridDim.x * kScanTile) {
        if (threadIdx.x == 0) S.nkeep = 0;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const long long v = t0 + q * kPeelThreads + threadIdx.x;
            bool live = false;
            if (v < g.n) {
                live = g.hc[v].x != -1;
                if (live) {
                    P.dcur[v] = g.deg[v];
                    g.hc[v].x = UNPEELED;
                }
            }
            const unsigned lb = __ballot_sync(0xffffffffu, live);
            int kp = 0;
            if (lane == 0 && lb) kp = atomicAdd(&S.nkeep, __popc(lb));
            kp = __shfl_sync(0xffffffffu, kp, 0);
            if (live) S.keep[kp + __popc(lb & ((1u << lane) - 1))] = (int32_t)v;
        }
        __syncthreads();
        if (threadIdx.x == 0) S.kbase = S.nkeep ? atomicAdd(&C->pc[1], (unsigned long long)S.nkeep) : 0;
        __syncthreads();
        for (int j = threadIdx.x; j < S.nkeep; j += kPeelThreads) P.L0[S.kbase + j] = S.keep[j];
        __syncthreads();
    }
    if (!clk.sync(P, PP_SCAN)) return;
    unsigned long long nl = vload64(&C->spc[1]);
    int32_t* Lc = P.L0;
    int32_t* Ln = P.L1;
    int k = 0;
    unsigned long long ft = 0;
    long long levels = 0;
    long long slots = 0;   // adjacency slots this warp scanned (algorithmic-byte counters)
    while (nl > 0) {
        // scan the remaining list, one tile per block at a time: degree k
        // leaves now, above k stays, below k left at an earlier level
        if (blockIdx.x == 0 && threadIdx.x == 0) C->st[ST_VISITED] += nl;
        const unsigned long long f0 = ft;
        for (long long t0 = (long long)blockIdx.x * kScanTile; t0 < (long long)nl;
             t0 += (long long)gridDim.x * kScanTile) {
            if (threadIdx.x == 0) {
                S.nkeep = 0;
                S.npeel = 0;
                S.mx = 0;
            }
            __syncthreads();
            int mx = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const long long i = t0 + q * kPeelThreads + threadIdx.x;
                bool peel = false, keep = false;
                int v = 0;
                if (i < (long long)nl) {
                    v = Lc[i];
                    const int d = P.dcur[v];
                    if (d == k) {
                        g.hc[v].x = k;
                        peel = true;
                    } else if (d > k) {
                        keep = true;
                        mx = max(mx, 0x7FFFFFFF - d);
                    }
                }
                const unsigned kb = __ballot_sync(0xffffffffu, keep), pb = __ballot_sync(0xffffffffu, peel);
                int kp = 0, pp = 0;
                if (lane == 0) {
                    if (kb) kp = atomicAdd(&S.nkeep, __popc(kb));
                    if (pb) pp = atomicAdd(&S.npeel, __popc(pb));
                }
                kp = __shfl_sync(0xffffffffu, kp, 0);
                pp = __shfl_sync(0xffffffffu, pp, 0);
                const unsigned below = (1u << lane) - 1;
                if (keep) S.keep[kp + __popc(kb & below)] = v;
                if (peel) S.peel[pp + __popc(pb & below)] = v;
            }
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0 && mx) atomicMax(&S.mx, mx);
            __syncthreads();
            if (threadIdx.x == 0) {
                S.kbase = S.nkeep ? atomicAdd(&C->pc[1], (unsigned long long)S.nkeep) : 0;
                S.pbase = S.npeel ? atomicAdd(&C->tail[0], (unsigned long long)S.npeel) : 0;
                if (S.mx) atomicMax(&C->pc[3], (unsigned long long)S.mx);
            }
            __syncthreads();
            for (int j = threadIdx.x; j < S.nkeep; j += kPeelThreads) Ln[S.kbase + j] = S.keep[j];
            for (int j = threadIdx.x; j < S.npeel; j += kPeelThreads) P.F[S.pbase + j] = S.peel[j];
            __syncthreads();
        }
        if (!clk.sync(P, PP_SCAN)) return;
        unsigned long long fhi = vload64(&C->stail[0]);
        unsigned long long nln = vload64(&C->spc[1]);
        unsigned long long smx = vload64(&C->spc[3]);
        int32_t* t = Lc;
        Lc = Ln;
        Ln = t;
        nl = nln;
        if (fhi == f0) {
            if (nl == 0) break;
            k = 0x7FFFFFFF - (int)smx;   // jump to the smallest remaining degree
            continue;
        }
        // sub-waves at level k.  A peeled neighbour needs no test: its
        // working degree is at most k when it leaves and only falls after,
        // so a decrement can bring exactly k + 1 down to k only for a
        // vertex still in the graph.
        unsigned long long lo = f0, hi = fhi;
        while (hi > lo) {
            const unsigned long long cnt_f = hi - lo;
            for (unsigned long long j = (unsigned long long)gwarp; j < cnt_f; j += (unsigned long long)nwarps) {
                const int v = P.F[lo + j];
                const long long o = g.off[v];
                const int len = g.end[v];
                slots += len;
                if (len >= kPeelBig) {
                    // chunk tasks (vertex, chunk), run by every warp after the barrier
                    const int nch = (len + kPeelChunk - 1) / kPeelChunk;
                    unsigned long long tb = 0;
                    if (lane == 0) tb = atomicAdd(&C->pc[3], (unsigned long long)nch);
                    tb = __shfl_sync(0xffffffffu, tb, 0);
                    const bool fits = tb + nch <= P.chunk_cap;
                    for (int c = lane; c < nch; c += 32) {
                        if (tb + c >= P.chunk_cap) break;
                        P.chunks[tb + c] = fits ? (((unsigned long long)(uint32_t)v << 32) | (uint32_t)c)
                                                : kPeelNoTask;
                    }
                    if (fits) continue;
                }
                peel_range(g, P, C, o, 0, len, k, buf, cnt);
            }
            block_flush_peeled(C, P, S, cnt);
            if (!clk.sync(P, PP_WAVE)) return;
            const unsigned long long nchunks = min(vload64(&C->spc[3]), P.chunk_cap);
            if (nchunks > 0) {
                for (unsigned long long c = (unsigned long long)gwarp; c < nchunks; c += (unsigned long long)nwarps) {
                    const unsigned long long task = P.chunks[c];
                    if (task == kPeelNoTask) continue;
                    const int v = (int)(task >> 32);
                    const int s0 = (int)(task & 0xFFFFFFFFu) * kPeelChunk;
                    peel_range(g, P, C, g.off[v], s0, min(g.end[v], s0 + kPeelChunk), k, buf, cnt);
                }
                block_flush_peeled(C, P, S, cnt);
                if (!clk.sync(P, PP_CHUNK)) return;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) C->st[ST_WAVES]++;
            lo = hi;
            hi = vload64(&C->stail[0]);
        }
        ft = hi;
        k++;
        levels++;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) C->st[ST_LEVELS] = (unsigned long long)levels;
    if (lane == 0 && slots) atomicAdd(&C->st[ST_VISSLOTS], (unsigned long long)slots);
}

// The peel always runs kPeelThreads-thread blocks (its tiles and per-warp
// buffers are laid out for them); `threads` is ignored.
int peel_blocks_per_sm(int threads) {
    (void)threads;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, peel_kernel, kPeelThreads, 0) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_peel(const PeelParams& p, int blocks, int threads, cudaStream_t s) {
    (void)threads;
    PeelParams q = p;
    void* args[] = {&q};
    return cudaLaunchCooperativeKernel((const void*)peel_kernel, dim3(blocks), dim3(kPeelThreads), args, 0, s);
}

// ------------------------------------------------------------------ index rehash
__global__ void rehash_kernel(const Bucket* __restrict__ old_idx, unsigned long long old_size, DevGraph g, Ctl* c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)old_size) return;
    Bucket b = old_idx[i];
    if (b.key == KEY_EMPTY || b.key == KEY_TOMB) return;
    bool existed = false;
    long long nb = idx_insert(g.idx, g.idx_mask, b.key, &existed);
    if (nb < 0) { atomicCAS(&c->error, 0, E_INDEX_FULL); return; }
    g.idx[nb].slo = b.slo;
    g.idx[nb].shi = b.shi;
}

cudaError_t rehash(const Bucket* old_idx, unsigned long long old_size, DevGraph g, Ctl* c, cudaStream_t s) {
    if (old_size == 0) return cudaSuccess;
    rehash_kernel<<<grid_for((long long)old_size, 256, 1ll << 31), 256, 0, s>>>(old_idx, old_size, g, c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ vertex insertion
// Neighbour lists of `count` new vertices (ids base..base+count-1): every
// neighbour is live or new, and not the vertex itself.  Warp per vertex.
__global__ void validate_vertices_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ nb, int32_t count,
                                         int32_t base, DevGraph g, Ctl* c) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < count; w += nw) {
        long long a = off[w], b = off[w + 1];
        if (a < 0 || b < a) {
            if (lane == 0) atomicCAS(&c->error, 0, E_INVALID);
            continue;
        }
        for (long long j = a + lane; j < b; j += 32) {
            int32_t x = nb[j];
            bool bad = x < 0 || x >= base + count || x == base + w || (x < base && g.hc[x].x < 0);
            if (bad) {
                atomicMin(&c->bad_index, j);
                atomicCAS(&c->error, 0, E_INVALID);
            }
        }
    }
}

__global__ void init_vertices_kernel(const int64_t* __restrict__ off, int32_t count, int32_t base, DevGraph g, Ctl* c) {
    long long b0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
    long long stride = (long long)gridDim.x * blockDim.x;
    int lane = lane_id();
    for (; b0 < count; b0 += stride) {
        long long i = b0 + lane;
        int cp = 0;
        if (i < count) cp = cap_for(off[i + 1] - off[i], g.slack_pct, g.min_cap);
        int incl = cp;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long wb = 0;
        if (lane == 31) wb = atomicAdd(&c->adj_top, (unsigned long long)tot);
        wb = __shfl_sync(0xffffffffu, wb, 31);
        if (i < count) {
            long long v = base + i;
            g.off[v] = (int64_t)(wb + incl - cp);
            g.cap[v] = cp;
            g.end[v] = 0;
            g.deg[v] = 0;
            g.hc[v] = make_int2(0, 0);
            g.kc[v] = key_of(0, 0);
            g.hw[v] = 0ull;
            g.chg[v] = 0;
            g.taken[v] = 0;
            g.claim0[v] = CLAIM_FREE;
            g.claim1[v] = CLAIM_FREE;
            g.need[v] = 0;
        }
    }
}

__global__ void expand_vertex_edges_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ nb,
                                           int32_t count, int32_t base, int32_t* E) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < count; w += nw) {
        for (long long j = off[w] + lane; j < off[w + 1]; j += 32) {
            E[2 * j] = base + (int32_t)w;
            E[2 * j + 1] = nb[j];
        }
    }
}

cudaError_t validate_vertices(const int64_t* nbr_off, const int32_t* nbrs, int32_t count, int32_t base, DevGraph g,
                              Ctl* c, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    validate_vertices_kernel<<<grid_for((long long)count * 32, 256, 65536), 256, 0, s>>>(nbr_off, nbrs, count, base, g, c);
    return cudaGetLastError();
}
cudaError_t init_vertices(const int64_t* nbr_off, int32_t count, int32_t base, DevGraph g, Ctl* c, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    init_vertices_kernel<<<grid_for(count, 256, 65536), 256, 0, s>>>(nbr_off, count, base, g, c);
    return cudaGetLastError();
}
cudaError_t expand_vertex_edges(const int64_t* nbr_off, const int32_t* nbrs, int32_t count, int32_t base, int32_t* E,
                                cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    expand_vertex_edges_kernel<<<grid_for((long long)count * 32, 256, 65536), 256, 0, s>>>(nbr_off, nbrs, count, base, E);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ vertex deletion
__global__ void validate_ids_kernel(const int32_t* __restrict__ ids, int32_t count, DevGraph g, Ctl* c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int32_t v = ids[i];
    if (v < 0 || v >= g.n || g.hc[v].x < 0) {
        atomicMin(&c->bad_index, i);
        atomicCAS(&c->error, 0, E_INVALID);
        return;
    }
    atomicAdd(&c->reloc_need, (unsigned long long)g.end[v]);   // upper bound on incident edges
}

__global__ void gather_incident_kernel(const int32_t* __restrict__ ids, int32_t count, DevGraph g, int2* E,
                                       long long cap, Ctl* c) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < count; w += nw) {
        int v = ids[w];
        long long o = g.off[v];
        int len = g.end[v];
        for (int t0 = 0; t0 < len; t0 += 32) {
            int t = t0 + lane;
            int x = t < len ? g.adj[o + t] : HOLE;
            bool live = x >= 0;
            unsigned int b = __ballot_sync(0xffffffffu, live);
            unsigned long long base = 0;
            if (lane == 0 && b) base = atomicAdd(&c->gather_n, (unsigned long long)__popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            long long p = (long long)base + __popc(b & ((1u << lane) - 1));
            if (live && p < cap) E[p] = make_int2(v, x);
        }
    }
}

__global__ void mark_dead_kernel(const int32_t* __restrict__ ids, int32_t count, DevGraph g) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int32_t v = ids[i];
    g.hc[v] = make_int2(-1, 0);
    g.kc[v] = KEY_DEAD;
    g.hw[v] = 0ull;
    g.end[v] = 0;
    g.deg[v] = 0;
}

// Vertices being deleted keep their core for the rest of the call and count
// as fixed support for their neighbours while their edges go (PIN_SD).
__global__ void pin_vertices_kernel(const int32_t* __restrict__ ids, int32_t count, DevGraph g) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    g.hc[ids[i]].y = PIN_SD;
    atomicOr(&g.kc[ids[i]], 1u);
}

cudaError_t pin_vertices(const int32_t* ids, int32_t count, DevGraph g, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    pin_vertices_kernel<<<grid_for(count, 256), 256, 0, s>>>(ids, count, g);
    return cudaGetLastError();
}

cudaError_t validate_ids(const int32_t* ids, int32_t count, DevGraph g, Ctl* c, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    validate_ids_kernel<<<grid_for(count, 256), 256, 0, s>>>(ids, count, g, c);
    return cudaGetLastError();
}
cudaError_t gather_incident(const int32_t* ids, int32_t count, DevGraph g, int32_t* E, long long cap, Ctl* c,
                            cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    gather_incident_kernel<<<grid_for((long long)count * 32, 256, 65536), 256, 0, s>>>(ids, count, g, (int2*)E, cap, c);
    return cudaGetLastError();
}
cudaError_t mark_dead(const int32_t* ids, int32_t count, DevGraph g, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    mark_dead_kernel<<<grid_for(count, 256), 256, 0, s>>>(ids, count, g);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ export
__global__ void export_cores_kernel(DevGraph g, int32_t* out) {
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    out[v] = g.hc[v].x;
}

// SD (Definition 7) of every vertex; -1 for a deleted vertex.
__global__ void export_sd_kernel(DevGraph g, int32_t* out) {
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    const int2 h = g.hc[v];
    out[v] = h.x < 0 ? -1 : h.y;
}

__global__ void export_edges_kernel(DevGraph g, int2* out, Ctl* c) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int lane = lane_id();
    for (; w < g.n; w += nw) {
        long long o = g.off[w];
        int len = g.end[w];
        for (int t0 = 0; t0 < len; t0 += 32) {
            int t = t0 + lane;
            int x = t < len ? g.adj[o + t] : HOLE;
            bool p = x > (int)w;
            unsigned int b = __ballot_sync(0xffffffffu, p);
            unsigned long long base = 0;
            if (lane == 0 && b) base = atomicAdd(&c->gather_n, (unsigned long long)__popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (p) out[base + __popc(b & ((1u << lane) - 1))] = make_int2((int)w, x);
        }
    }
}

// Consistency of the store with its own definitions (a debug check, run on
// request).  Per live vertex v, from its list: SD (Definition 7) recounted
// from the neighbours' cores against hc[v].y; the scan key against core and
// the stored SD; the live degree against the list's non-hole slots; every
// slot a hole or a live vertex id; and the k-core condition (at least
// core(v) neighbours of core >= core(v)).  A pinned vertex (vertex deletion
// in progress) keeps its pinned SD and is not compared on SD, key or the
// k-core condition.  A dead vertex must carry the dead key.  Warp per
// vertex; out[0..4] count the mismatches of the five checks, out[5] the
// vertices checked, out[6] the smallest vertex that failed a check.
__global__ void check_store_kernel(DevGraph g, unsigned long long* out) {
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int lane = lane_id();
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        const int2 h = g.hc[v];
        const uint32_t key = g.kc[v];
        if (h.x < 0) {
            if (lane == 0) {
                atomicAdd(&out[5], 1ull);
                if (key != KEY_DEAD) {
                    atomicAdd(&out[1], 1ull);
                    atomicMin(&out[6], (unsigned long long)v);
                }
            }
            continue;
        }
        const long long o = g.off[v];
        const int len = g.end[v];
        int sd = 0, live = 0, bad = 0;
        for (int t = lane; t < len; t += 32) {
            const int w = g.adj[o + t];
            if (w == HOLE) continue;
            if (w < 0 || w >= g.n) {
                bad++;
                continue;
            }
            const int cw = g.hc[w].x;
            if (cw < 0) {
                bad++;
                continue;
            }
            live++;
            sd += cw >= h.x;
        }
        sd = warp_sum(sd);
        live = warp_sum(live);
        bad = warp_sum(bad);
        if (lane == 0) {
            const bool pinned = h.y == PIN_SD;
            bool fail = false;
            if (!pinned && sd != h.y) {
                atomicAdd(&out[0], 1ull);
                fail = true;
            }
            if (!pinned && key != key_of(h.x, h.y)) {
                atomicAdd(&out[1], 1ull);
                fail = true;
            }
            if (live != g.deg[v]) {
                atomicAdd(&out[2], 1ull);
                fail = true;
            }
            if (bad) {
                atomicAdd(&out[3], (unsigned long long)bad);
                fail = true;
            }
            if (!pinned && sd < h.x) {
                atomicAdd(&out[4], 1ull);
                fail = true;
            }
            atomicAdd(&out[5], 1ull);
            if (fail) atomicMin(&out[6], (unsigned long long)v);
        }
    }
}

cudaError_t check_store(DevGraph g, unsigned long long* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(out + 6, 0xFF, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (g.n <= 0) return cudaSuccess;
    check_store_kernel<<<grid_for((long long)g.n * 32, 256, 65536), 256, 0, s>>>(g, out);
    return cudaGetLastError();
}

cudaError_t export_cores(DevGraph g, int32_t* out, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    export_cores_kernel<<<grid_for(g.n, 256, 1ll << 31), 256, 0, s>>>(g, out);
    return cudaGetLastError();
}
cudaError_t export_sd(DevGraph g, int32_t* out, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    export_sd_kernel<<<grid_for(g.n, 256, 1ll << 31), 256, 0, s>>>(g, out);
    return cudaGetLastError();
}
cudaError_t export_edges(DevGraph g, int32_t* out, Ctl* c, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    export_edges_kernel<<<grid_for((long long)g.n * 32, 256, 65536), 256, 0, s>>>(g, (int2*)out, c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ multi-graph helpers
// Local ids of a concatenated per-graph batch -> global ids.  prefix[i] is
// the first batch entry of graph i (ng+1 entries).
__global__ void localize_multi_kernel(int32_t* E, long long k, const unsigned long long* kp,
                                      const long long* __restrict__ prefix, const int32_t* __restrict__ bases,
                                      int32_t ng) {
    if (kp) k = (long long)vload64(kp);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        int lo = 0, hi = ng - 1;
        while (lo < hi) {                 // last graph whose prefix <= i
            int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= i) lo = mid; else hi = mid - 1;
        }
        int b = bases[lo];
        int nv = bases[lo + 1] - b;       // bases has ng+1 entries
        int32_t u = E[2 * i], v = E[2 * i + 1];
        // an id outside its graph stays invalid (negative) so ingest rejects it
        E[2 * i] = (u >= 0 && u < nv) ? u + b : -1;
        E[2 * i + 1] = (v >= 0 && v < nv) ? v + b : -1;
    }
}

__global__ void count_multi_kernel(const REdge* __restrict__ R, long long n, const unsigned long long* np,
                                   const int32_t* __restrict__ bases, int32_t ng, unsigned long long* per_graph) {
    if (np) n = (long long)vload64(np);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int x = R[i].lo;
        int lo = 0, hi = ng - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (bases[mid] <= x) lo = mid; else hi = mid - 1;
        }
        atomicAdd(&per_graph[lo], 1ull);
    }
}

// Captured step: every id of a batch names a live vertex (checked for both
// batches before anything changes).  bad_index gets (phase << 40) | i.
__global__ void validate_pairs_kernel(const int32_t* __restrict__ E, long long k, const unsigned long long* kp,
                                      int phase, DevGraph g, Ctl* c) {
    if (kp) k = (long long)vload64(kp);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        int32_t u = E[2 * i], v = E[2 * i + 1];
        if (u < 0 || v < 0 || u >= g.n || v >= g.n || g.hc[u].x < 0 || g.hc[v].x < 0) {
            atomicMin(&c->bad_index, ((long long)phase << 40) | i);
            atomicCAS(&c->error, 0, E_INVALID);
        }
    }
}

cudaError_t localize_multi(int32_t* E, long long k, const unsigned long long* kp, const long long* prefix,
                           const int32_t* bases, int32_t ng, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    localize_multi_kernel<<<grid_for(k, 256, 8192), 256, 0, s>>>(E, k, kp, prefix, bases, ng);
    return cudaGetLastError();
}
cudaError_t count_multi(const REdge* R, long long n, const unsigned long long* np, const int32_t* bases, int32_t ng,
                        unsigned long long* per_graph, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_multi_kernel<<<grid_for(n, 256, 8192), 256, 0, s>>>(R, n, np, bases, ng, per_graph);
    return cudaGetLastError();
}
cudaError_t validate_pairs(const int32_t* E, long long k, const unsigned long long* kp, int phase, DevGraph g, Ctl* c,
                           cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    validate_pairs_kernel<<<grid_for(k, 256, 8192), 256, 0, s>>>(E, k, kp, phase, g, c);
    return cudaGetLastError();
}

// capacity totals for a vertex range: sum_only pass of offsets_kernel
cudaError_t sum_caps(DevGraph g, int32_t v0, int32_t v1, Ctl* c, cudaStream_t s) {
    if (v1 <= v0) return cudaSuccess;
    offsets_kernel<<<grid_for(v1 - v0, 256, 65536), 256, 0, s>>>(g, v0, v1, c, 1);
    return cudaGetLastError();
}

}  // namespace cm
