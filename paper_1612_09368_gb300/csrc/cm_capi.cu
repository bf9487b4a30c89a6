// cm_capi.cu -- host implementation of the C ABI in include/coremaint.h.
//
// A handle owns one graph (or a disjoint union of many) in device memory
// and runs every call on its stream.  An update call is:
//   copy batch in -> ingest (validate, canonicalise, dedupe, filter against
//   the edge index) -> read back counts -> relocate vertices whose slack the
//   batch exceeds -> one cooperative launch of the maintenance kernel, which
//   runs all superior-edge-set iterations -> read back status and counters.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/coremaint.h"
#include "cm_common.cuh"
#include "cm_launch.h"

using namespace cm;

static thread_local std::string g_create_err = "no error";
constexpr int kGridThreadsHost = 512;   // threads per block of both maintenance kernels

struct cm_graph {
    cm_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int32_t n = 0, ncap = 0;
    int64_t m = 0;
    unsigned long long idx_size = 0;
    int64_t idx_live = 0, idx_tomb = 0;
    uint32_t epoch = 1;
    bool poisoned = false, cores_stale = false;
    std::string err = "no error";
    DevGraph g{};
    Ctl* ctl = nullptr;
    Ctl* hctl = nullptr;   // pinned mirror
    // batch buffers
    int32_t* dbatch = nullptr;
    long long batch_cap = 0;  // pairs
    BSet* bset = nullptr;
    unsigned long long bset_size = 0;
    REdge* R0 = nullptr;
    REdge* R1 = nullptr;
    long long rcap = 0;
    // per-vertex scratch rings (also the peel's scratch)
    int32_t* VQ = nullptr;
    int32_t* EQ = nullptr;
    int32_t* CQ = nullptr;
    int32_t* OVL = nullptr;
    unsigned long long qmask = 0;
    // multi-graph (small arrays, plain cudaMalloc)
    int32_t ngraphs = 1;
    std::vector<int32_t> bases;
    int32_t* dbases = nullptr;
    long long* dprefix = nullptr;
    unsigned long long* dpergraph = nullptr;
    unsigned long long* dchk = nullptr;   // counters of the consistency check (allocated on first use)
    // timing and counters
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cm_stats last{};
    long long launches = 0;
    // execution-mode thresholds of the maintenance kernel (see cm_iterate.cu)
    long long small_edges = 16384, small_work = 1024, big_work = 8192;
    // grid-wide chunked scans of high-degree vertices (cm_iterate.cu)
    HubItem* HQ = nullptr;
    unsigned long long* TQ = nullptr;   // grid-mode task queue (TASK_EMPTY = all ones when free)
    unsigned long long tq_size = 0;
    int32_t hub_len = 1024;
    int32_t block_len = 4096, block_len_del = 1024;
    int32_t claim_max = 1;
    int32_t sel_key = 0, sel_rounds = 0;   // selection order and claim-round cap (options)
};

// ------------------------------------------------------------------ helpers
static int set_err(cm_graph* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_err = buf;
    return code;
}

static int fail_cuda(cm_graph* h, cudaError_t e, const char* what) {
    if (h) h->poisoned = true;
    return set_err(h, CM_ERR_CUDA, "CUDA error in %s: %s", what, cudaGetErrorString(e));
}

#define CK(h, x)                                            \
    do {                                                    \
        cudaError_t _e = (x);                               \
        if (_e != cudaSuccess) return fail_cuda(h, _e, #x); \
    } while (0)

#define LAUNCH(h, x)     \
    do {                 \
        (h)->launches++; \
        CK(h, x);        \
    } while (0)

static void* dalloc(cm_graph* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (h->opt.alloc) return h->opt.alloc(bytes, (void*)h->stream, h->opt.alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
static void dfree(cm_graph* h, void* p, size_t bytes) {
    if (!p) return;
    if (h->opt.free) h->opt.free(p, bytes ? bytes : 16, (void*)h->stream, h->opt.alloc_ctx);
    else cudaFree(p);
}

template <class T>
static bool realloc_dev(cm_graph* h, T*& p, size_t old_elems, size_t new_elems, size_t keep_elems) {
    T* q = (T*)dalloc(h, new_elems * sizeof(T));
    if (!q) return false;
    if (p && keep_elems) {
        if (cudaMemcpyAsync(q, p, keep_elems * sizeof(T), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) {
            dfree(h, q, new_elems * sizeof(T));
            return false;
        }
    }
    if (p) {
        cudaStreamSynchronize(h->stream);
        dfree(h, p, old_elems * sizeof(T));
    }
    p = q;
    return true;
}

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static unsigned long long pow2_at_least(unsigned long long x) {
    unsigned long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

static int rd_ctl(cm_graph* h) {
    CK(h, cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return CM_OK;
}

// Reset the fields a persistent launch uses (barrier, tails, counters,
// stats).  The error word stays: an error of the ingest kernels (which the
// host does not read back on every path) stops the maintenance kernel.
static int reset_launch_zone(cm_graph* h) {
    CK(h, cudaMemsetAsync(h->ctl, 0, offsetof(Ctl, error), h->stream));
    CK(h, cudaMemsetAsync(&h->ctl->tail[0], 0, offsetof(Ctl, nrem) - offsetof(Ctl, tail), h->stream));
    return CM_OK;
}

// Reset the host-exchange words; adj_top stays (it is device-owned).
static int reset_ingest_zone(cm_graph* h) {
    CK(h, cudaMemsetAsync(&h->ctl->error, 0, sizeof(int) * 2, h->stream));
    CK(h, cudaMemsetAsync(&h->ctl->nrem, 0, sizeof(unsigned long long) * 3, h->stream));
    CK(h, cudaMemsetAsync(&h->ctl->bad_index, 0x7F, sizeof(long long), h->stream));   // large positive
    CK(h, cudaMemsetAsync(&h->ctl->gather_n, 0, sizeof(unsigned long long), h->stream));
    CK(h, cudaMemsetAsync(&h->ctl->defer, 0, sizeof(int), h->stream));
    return CM_OK;
}

// ------------------------------------------------------------------ capacity management
static int grow_vertices(cm_graph* h, int32_t need) {
    if (need <= h->ncap) return CM_OK;
    long long nc = (long long)need + need / 4 + 1024;
    if (nc > INT32_MAX) nc = INT32_MAX;
    int32_t keep = h->n;
    DevGraph& g = h->g;
    size_t oc = (size_t)h->ncap;
    bool ok = realloc_dev(h, g.hc, oc, nc, keep) && realloc_dev(h, g.hw, oc, nc, keep) &&
              realloc_dev(h, g.kc, oc, nc, keep) &&
              realloc_dev(h, g.off, oc, nc, keep) &&
              realloc_dev(h, g.end, oc, nc, keep) && realloc_dev(h, g.cap, oc, nc, keep) &&
              realloc_dev(h, g.deg, oc, nc, keep) && realloc_dev(h, g.chg, oc, nc, keep) &&
              realloc_dev(h, g.taken, oc, nc, keep) && realloc_dev(h, g.claim0, oc, nc, keep) &&
              realloc_dev(h, g.claim1, oc, nc, keep) && realloc_dev(h, g.need, oc, nc, keep);
    if (!ok) return set_err(h, CM_ERR_OOM, "out of device memory growing vertex arrays to %lld", nc);
    size_t tail = (size_t)(nc - keep);
    CK(h, cudaMemsetAsync(g.hc + keep, 0, tail * sizeof(int2), h->stream));
    CK(h, cudaMemsetAsync(g.hw + keep, 0, tail * sizeof(unsigned long long), h->stream));
    CK(h, cudaMemsetAsync(g.kc + keep, 0, tail * sizeof(uint32_t), h->stream));
    CK(h, cudaMemsetAsync(g.end + keep, 0, tail * sizeof(int32_t), h->stream));
    CK(h, cudaMemsetAsync(g.cap + keep, 0, tail * sizeof(int32_t), h->stream));
    CK(h, cudaMemsetAsync(g.deg + keep, 0, tail * sizeof(int32_t), h->stream));
    CK(h, cudaMemsetAsync(g.off + keep, 0, tail * sizeof(int64_t), h->stream));
    CK(h, cudaMemsetAsync(g.chg + keep, 0, tail * sizeof(uint32_t), h->stream));
    CK(h, cudaMemsetAsync(g.taken + keep, 0, tail * sizeof(uint32_t), h->stream));
    CK(h, cudaMemsetAsync(g.claim0 + keep, 0xFF, tail * sizeof(unsigned long long), h->stream));
    CK(h, cudaMemsetAsync(g.claim1 + keep, 0xFF, tail * sizeof(unsigned long long), h->stream));
    CK(h, cudaMemsetAsync(g.need + keep, 0, tail * sizeof(int32_t), h->stream));
    unsigned long long qn = pow2_at_least((unsigned long long)nc);
    size_t oq = h->qmask ? (size_t)(h->qmask + 1) : 0;
    if (qn != oq) {
        ok = realloc_dev(h, h->VQ, oq, qn, 0) && realloc_dev(h, h->EQ, oq, qn, 0) &&
             realloc_dev(h, h->CQ, oq, qn, 0) && realloc_dev(h, h->OVL, oq, qn, 0);
        if (!ok) return set_err(h, CM_ERR_OOM, "out of device memory for queues");
        h->qmask = qn - 1;
    }
    h->ncap = (int32_t)nc;
    return CM_OK;
}

// Make room for need_slots more adjacency slots after the pool top.
static int grow_pool(cm_graph* h, long long need_slots) {
    unsigned long long top = 0;
    CK(h, cudaMemcpyAsync(&h->hctl->adj_top, &h->ctl->adj_top, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    top = h->hctl->adj_top;
    if ((long long)top + need_slots <= h->g.adj_cap) return CM_OK;
    long long nc = (long long)top + need_slots;
    nc = nc + nc / 4 + 4096;
    if (!realloc_dev(h, h->g.adj, (size_t)h->g.adj_cap, (size_t)nc, (size_t)top))
        return set_err(h, CM_ERR_OOM, "out of device memory growing the adjacency pool to %lld slots", nc);
    h->g.adj_cap = nc;
    return CM_OK;
}

static int alloc_index(cm_graph* h, unsigned long long size) {
    Bucket* p = (Bucket*)dalloc(h, size * sizeof(Bucket));
    if (!p) return set_err(h, CM_ERR_OOM, "out of device memory for an edge index of %llu buckets", size);
    CK(h, cudaMemsetAsync(p, 0xFF, size * sizeof(Bucket), h->stream));
    h->g.idx = p;
    h->g.idx_mask = size - 1;
    h->idx_size = size;
    return CM_OK;
}

// Grow or clean the index so that `adding` more keys keep its load <= 1/2.
static int ensure_index(cm_graph* h, long long adding) {
    long long used = h->idx_live + h->idx_tomb + adding;
    if ((unsigned long long)used * 2 <= h->idx_size) return CM_OK;
    long long want = (h->idx_live + adding) * 5 / 2 + 1024;
    unsigned long long ns = pow2_at_least((unsigned long long)want);
    if (ns < h->idx_size) ns = h->idx_size;
    Bucket* old = h->g.idx;
    unsigned long long old_size = h->idx_size;
    int rc = alloc_index(h, ns);
    if (rc) {
        h->g.idx = old;
        h->g.idx_mask = old_size - 1;
        h->idx_size = old_size;
        return rc;
    }
    LAUNCH(h, rehash(old, old_size, h->g, h->ctl, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    dfree(h, old, old_size * sizeof(Bucket));
    h->idx_tomb = 0;
    return CM_OK;
}

// Task queue of the grid-mode search: room for every vertex entering the
// frontier and being evicted once per iteration, plus the chunk tasks of
// high-degree lists (three passes per list, at least 128 slots per hub) and
// the claims warps make past the tail.
static int ensure_tasks(cm_graph* h) {
    const unsigned long long need =
        pow2_at_least(2ull * (unsigned long long)h->ncap + (unsigned long long)h->g.adj_cap / 32 + (1ull << 18));
    if (need <= h->tq_size) return CM_OK;
    unsigned long long* q = (unsigned long long*)dalloc(h, need * 8);
    if (!q) return set_err(h, CM_ERR_OOM, "out of device memory for a task queue of %llu slots", need);
    CK(h, cudaMemsetAsync(q, 0xFF, need * 8, h->stream));
    if (h->TQ) {
        CK(h, cudaStreamSynchronize(h->stream));
        dfree(h, h->TQ, h->tq_size * 8);
    }
    h->TQ = q;
    h->tq_size = need;
    return CM_OK;
}

// Batch buffers for k edges: staging copy, dedupe set, remaining lists.
static int ensure_batch(cm_graph* h, long long k) {
    if (k > h->batch_cap) {
        long long nc = k + k / 2 + 1024;
        int32_t* q = (int32_t*)dalloc(h, (size_t)nc * 2 * sizeof(int32_t));
        if (!q) return set_err(h, CM_ERR_OOM, "out of device memory for a batch of %lld edges", k);
        dfree(h, h->dbatch, (size_t)h->batch_cap * 2 * sizeof(int32_t));
        h->dbatch = q;
        h->batch_cap = nc;
    }
    unsigned long long bs = pow2_at_least((unsigned long long)(2 * k + 16));
    if (bs > h->bset_size) {
        BSet* q = (BSet*)dalloc(h, bs * sizeof(BSet));
        if (!q) return set_err(h, CM_ERR_OOM, "out of device memory for a batch set");
        dfree(h, h->bset, h->bset_size * sizeof(BSet));
        h->bset = q;
        h->bset_size = bs;
    }
    if (k > h->rcap) {
        long long nc = k + k / 2 + 1024;
        REdge* a = (REdge*)dalloc(h, (size_t)nc * sizeof(REdge));
        REdge* b = (REdge*)dalloc(h, (size_t)nc * sizeof(REdge));
        if (!a || !b) {
            dfree(h, a, (size_t)nc * sizeof(REdge));
            dfree(h, b, (size_t)nc * sizeof(REdge));
            return set_err(h, CM_ERR_OOM, "out of device memory for remaining-edge lists");
        }
        dfree(h, h->R0, (size_t)h->rcap * sizeof(REdge));
        dfree(h, h->R1, (size_t)h->rcap * sizeof(REdge));
        h->R0 = a;
        h->R1 = b;
        h->rcap = nc;
    }
    return CM_OK;
}

// ------------------------------------------------------------------ launch geometry
// Persistent kernels fill max_sms SMs (all by default) with as many blocks
// as stay resident.  A small batch gets fewer blocks: grid barriers then
// cost less, and there is not enough work for the whole GPU anyway.
static void persistent_geometry(cm_graph* h, int kind, long long work, int* blocks, int* threads) {
    const int t = 512;   // both persistent kernels run 512-thread blocks
    int occ = kind == 0 ? maintain_blocks_per_sm(t) : peel_blocks_per_sm(t);
    if (occ < 1) occ = 1;
    int bps = h->opt.blocks_per_sm > 0 ? (h->opt.blocks_per_sm < occ ? h->opt.blocks_per_sm : occ) : occ;
    int sms = h->opt.max_sms > 0 && h->opt.max_sms < h->num_sms ? h->opt.max_sms : h->num_sms;
    long long b = (long long)sms * bps;
    if (kind == 0 && h->opt.blocks_per_sm <= 0) {
        long long want = (work * 64 + t - 1) / t;
        if (want < sms) want = sms;
        if (want < b) b = want;
    }
    if (b < 1) b = 1;
    *blocks = (int)b;
    *threads = t;
}

// ------------------------------------------------------------------ create / destroy
extern "C" void cm_default_options(cm_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->slack_pct = 25;
    o->min_cap = 4;
    o->block_threads = 512;
    o->spin_limit_ns = 4000000000ll;
    o->block_mode_edges = 16384;
    o->block_mode_enter = 1024;
    o->block_mode_leave = 8192;
    o->hub_slots = 1024;
    o->block_slots = 4096;
    o->block_slots_delete = 1024;
    o->task_claim = 1;
}

static void free_all(cm_graph* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaDeviceSynchronize();
    DevGraph& g = h->g;
    size_t nc = (size_t)h->ncap;
    dfree(h, g.hc, nc * sizeof(int2));
    dfree(h, g.hw, nc * sizeof(unsigned long long));
    dfree(h, g.kc, nc * sizeof(uint32_t));
    dfree(h, g.off, nc * 8);
    dfree(h, g.end, nc * 4);
    dfree(h, g.cap, nc * 4);
    dfree(h, g.deg, nc * 4);
    dfree(h, g.chg, nc * 4);
    dfree(h, g.taken, nc * 4);
    dfree(h, g.claim0, nc * 8);
    dfree(h, g.claim1, nc * 8);
    dfree(h, g.need, nc * 4);
    dfree(h, g.adj, (size_t)g.adj_cap * 4);
    dfree(h, g.idx, h->idx_size * sizeof(Bucket));
    size_t qn = h->qmask ? (size_t)(h->qmask + 1) : 0;
    dfree(h, h->VQ, qn * 4);
    dfree(h, h->EQ, qn * 4);
    dfree(h, h->CQ, qn * 4);
    dfree(h, h->OVL, qn * 4);
    dfree(h, h->HQ, kHubRing * sizeof(HubItem));
    dfree(h, h->TQ, h->tq_size * 8);
    dfree(h, h->dbatch, (size_t)h->batch_cap * 8);
    dfree(h, h->bset, h->bset_size * sizeof(BSet));
    dfree(h, h->R0, (size_t)h->rcap * sizeof(REdge));
    dfree(h, h->R1, (size_t)h->rcap * sizeof(REdge));
    if (h->dbases) cudaFree(h->dbases);
    if (h->dprefix) cudaFree(h->dprefix);
    if (h->dpergraph) cudaFree(h->dpergraph);
    if (h->dchk) cudaFree(h->dchk);
    if (h->ctl) cudaFree(h->ctl);
    if (h->hctl) cudaFreeHost(h->hctl);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

static int peel_all(cm_graph* h);
static int run_check(cm_graph* h, cm_check_report* r);
static bool check_clean(const cm_check_report& r);

// Builds the store from a device edge list (global ids).
static int build_store(cm_graph* h, const int32_t* dE, long long m, const int32_t* dcores) {
    DevGraph& g = h->g;
    uint32_t* ebkt = (uint32_t*)dalloc(h, (size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    if (!ebkt) return set_err(h, CM_ERR_OOM, "out of device memory (create)");
    int rc = CM_OK;
    do {
        if ((rc = reset_ingest_zone(h))) break;
        h->launches += 3;
        cudaError_t e = build_index(dE, m, g, ebkt, h->ctl, h->stream);
        if (e == cudaSuccess) e = count_degrees(dE, ebkt, m, g, h->stream);
        if (e == cudaSuccess) e = sum_caps(g, 0, g.n, h->ctl, h->stream);
        if (e != cudaSuccess) { rc = fail_cuda(h, e, "build"); break; }
        if ((rc = rd_ctl(h))) break;
        if (h->hctl->error == E_INVALID) {
            rc = set_err(h, CM_ERR_INVALID, "edge %lld has an id outside [0, %d)", h->hctl->bad_index, g.n);
            break;
        }
        if (h->hctl->error) {
            rc = set_err(h, CM_ERR_CUDA, "device error %d while building the index", h->hctl->error);
            break;
        }
        long long total = (long long)h->hctl->reloc_need;
        long long pool = total + total / 4 + 4096;
        g.adj = (int32_t*)dalloc(h, (size_t)pool * sizeof(int32_t));
        if (!g.adj) { rc = set_err(h, CM_ERR_OOM, "out of device memory for %lld adjacency slots", pool); break; }
        g.adj_cap = pool;
        if ((e = cudaMemsetAsync(&h->ctl->adj_top, 0, 8, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "memset"); break; }
        h->launches += 2;
        e = assign_offsets(g, 0, g.n, h->ctl, h->stream);
        if (e == cudaSuccess) e = scatter_edges(dE, ebkt, m, g, h->stream);
        if (e != cudaSuccess) { rc = fail_cuda(h, e, "scatter"); break; }
        if (dcores) {
            h->launches++;
            if ((e = set_cores(dcores, g, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "set_cores"); break; }
        } else {
            if ((rc = peel_all(h))) break;
        }
        h->launches += 2;
        if ((e = init_mcd(g, 0, g.n, h->CQ, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "init_mcd"); break; }
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "create"); break; }
    } while (0);
    cudaStreamSynchronize(h->stream);
    dfree(h, ebkt, (size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    return rc;
}

static int count_live_edges(cm_graph* h, long long* m) {
    std::vector<int32_t> deg((size_t)h->n);
    if (h->n) CK(h, cudaMemcpy(deg.data(), h->g.deg, (size_t)h->n * 4, cudaMemcpyDeviceToHost));
    long long s = 0;
    for (int32_t d : deg) s += d;
    *m = s / 2;
    return CM_OK;
}

// Creates a handle around n vertices and a DEVICE-or-host edge list.
static int create_common(int32_t n, const int32_t* edges, long long m, const int32_t* cores, const cm_options* opt,
                         void* stream, cm_graph** hout) {
    cm_graph* h = new (std::nothrow) cm_graph();
    if (!h) return set_err(nullptr, CM_ERR_OOM, "out of host memory");
    *hout = h;
    if (opt) h->opt = *opt; else cm_default_options(&h->opt);
    if (h->opt.slack_pct < 0) h->opt.slack_pct = 0;
    if (h->opt.min_cap < 4) h->opt.min_cap = 4;
    if (h->opt.spin_limit_ns <= 0) h->opt.spin_limit_ns = 4000000000ll;
    if (h->opt.block_threads <= 0 || h->opt.block_threads > 512 || h->opt.block_threads % 32)
        h->opt.block_threads = 512;
    h->stream = (cudaStream_t)stream;
    h->small_edges = h->opt.block_mode_edges > 0 ? h->opt.block_mode_edges : h->opt.block_mode_edges < 0 ? 0 : 16384;
    h->small_work = h->opt.block_mode_enter > 0 ? h->opt.block_mode_enter : 1024;
    h->big_work = h->opt.block_mode_leave > 0 ? h->opt.block_mode_leave : 8192;
    h->hub_len = h->opt.hub_slots > 0 ? (h->opt.hub_slots < 128 ? 128 : h->opt.hub_slots)
                                      : h->opt.hub_slots < 0 ? 0 : 1024;
    h->block_len = h->opt.block_slots >= 32 ? h->opt.block_slots : 4096;
    h->block_len_del = h->opt.block_slots_delete >= 32 ? h->opt.block_slots_delete : 1024;
    h->claim_max = h->opt.task_claim >= 1 && h->opt.task_claim <= 8 ? h->opt.task_claim : 1;
    h->sel_key = h->opt.select_order == CM_SELECT_KEY ? 1 : 0;
    h->sel_rounds = h->opt.select_rounds > 0 ? h->opt.select_rounds : 0;
    CK(h, cudaGetDevice(&h->device));
    CK(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    int coop = 0;
    CK(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    if (!coop) return set_err(h, CM_ERR_CUDA, "device does not support cooperative launches");
    for (auto& e : h->ev) CK(h, cudaEventCreate(&e));
    CK(h, cudaMalloc(&h->ctl, sizeof(Ctl)));
    CK(h, cudaMemset(h->ctl, 0, sizeof(Ctl)));
    h->HQ = (HubItem*)dalloc(h, kHubRing * sizeof(HubItem));
    if (!h->HQ) return set_err(h, CM_ERR_OOM, "out of device memory for the hub items");
    CK(h, cudaMallocHost(&h->hctl, sizeof(Ctl)));
    memset(h->hctl, 0, sizeof(Ctl));
    h->g.slack_pct = h->opt.slack_pct;
    h->g.min_cap = h->opt.min_cap;
    h->n = 0;                                  // grow_vertices keeps (and does not clear) [0, n)
    int rc = grow_vertices(h, n > 0 ? n : 1);
    if (rc) return rc;
    h->n = n;
    h->g.n = n;
    if ((rc = alloc_index(h, pow2_at_least((unsigned long long)(2 * m + m / 2 + 1024))))) return rc;
    const int32_t* dE = edges;
    int32_t* tmp = nullptr;
    if (m > 0 && !is_device_ptr(edges)) {
        tmp = (int32_t*)dalloc(h, (size_t)m * 2 * sizeof(int32_t));
        if (!tmp) return set_err(h, CM_ERR_OOM, "out of device memory for %lld input edges", m);
        CK(h, cudaMemcpyAsync(tmp, edges, (size_t)m * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
        dE = tmp;
    }
    const int32_t* dC = cores;
    int32_t* tmpc = nullptr;
    if (cores && !is_device_ptr(cores)) {
        tmpc = (int32_t*)dalloc(h, (size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        if (!tmpc) {
            dfree(h, tmp, (size_t)m * 8);
            return set_err(h, CM_ERR_OOM, "out of device memory for cores");
        }
        CK(h, cudaMemcpyAsync(tmpc, cores, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
        dC = tmpc;
    }
    rc = build_store(h, dE, m, dC);
    cudaStreamSynchronize(h->stream);
    dfree(h, tmp, (size_t)m * 8);
    dfree(h, tmpc, (size_t)(n > 0 ? n : 1) * 4);
    if (rc) return rc;
    long long live = 0;
    if ((rc = count_live_edges(h, &live))) return rc;
    h->m = live;
    h->idx_live = live;
    h->bases = {0, n};
    return CM_OK;
}

extern "C" int cm_create(cm_graph** out, int32_t n, const int32_t* edges, int64_t m, const int32_t* cores,
                         const cm_options* opt, void* stream) {
    if (!out) return set_err(nullptr, CM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n < 0 || m < 0 || (m > 0 && !edges)) return set_err(nullptr, CM_ERR_INVALID, "bad sizes or NULL edges");
    cm_graph* h = nullptr;
    int rc = create_common(n, edges, m, cores, opt, stream, &h);
    if (rc) {
        if (h) {
            g_create_err = h->err;
            free_all(h);
        }
        return rc;
    }
    *out = h;
    return CM_OK;
}

extern "C" void cm_destroy(cm_graph* h) { free_all(h); }

// ------------------------------------------------------------------ peel
static int peel_all(cm_graph* h) {
    CK(h, cudaMemsetAsync(&h->ctl->error, 0, sizeof(int) * 2, h->stream));
    int rc = reset_launch_zone(h);
    if (rc) return rc;
    PeelParams p{};
    p.g = h->g;
    p.g.n = h->n;
    p.ctl = h->ctl;
    p.dcur = h->CQ;
    p.L0 = h->VQ;
    p.L1 = h->EQ;
    p.F = h->OVL;
    p.qmask = h->qmask;
    // the hub-item ring is scratch outside a maintenance search
    p.chunks = reinterpret_cast<unsigned long long*>(h->HQ);
    p.chunk_cap = kHubRing * sizeof(HubItem) / sizeof(unsigned long long);
    p.limit_ns = (unsigned long long)h->opt.spin_limit_ns;
    int blocks, threads;
    persistent_geometry(h, 1, h->n, &blocks, &threads);
    p.expect = (uint32_t)blocks;
    LAUNCH(h, launch_peel(p, blocks, threads, h->stream));
    if ((rc = rd_ctl(h))) return rc;
    if (h->hctl->error) {
        h->poisoned = true;
        return set_err(h, CM_ERR_LIMIT, "peeling stopped with device error %d", h->hctl->error);
    }
    h->last.peel_levels = (int64_t)h->hctl->st[ST_LEVELS];
    h->last.waves = (int64_t)h->hctl->st[ST_WAVES];   // sub-waves of the peel
    h->last.barriers = (int64_t)h->hctl->st[ST_BARRIERS];
    // phase times of the peel: level scans, sub-waves, chunk phases
    for (int i = 0; i < 3; i++) h->last.phase_ns[i] = (int64_t)h->hctl->ph[i];
    // Algorithmic bytes of the peel: 16 B per vertex to start it (degree
    // read, working degree, core and list writes); 12 B per remaining-list
    // entry scanned at a level (id, working degree, list write); 12 B per
    // adjacency slot of a peeled vertex (neighbour id, the working-degree
    // atomic, 4 B of its word when it leaves).
    h->last.alg_bytes += 16 * (int64_t)h->n + 12 * (int64_t)h->hctl->st[ST_VISITED] +
                         12 * (int64_t)h->hctl->st[ST_VISSLOTS];
    return CM_OK;
}

static int begin_call(cm_graph* h) {
    if (!h) return CM_ERR_INVALID;
    if (h->poisoned) return set_err(h, CM_ERR_STATE, "handle poisoned by an earlier failure: %s", h->err.c_str());
    h->launches = 0;
    memset(&h->last, 0, sizeof(h->last));
    CK(h, cudaEventRecord(h->ev[0], h->stream));
    return CM_OK;
}

static int end_call(cm_graph* h, int rc) {
    if (rc == CM_OK) {
        cudaEventRecord(h->ev[1], h->stream);
        cudaEventSynchronize(h->ev[1]);
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
        h->last.call_ms = ms;
    }
    h->last.launches = h->launches;
    return rc;
}

extern "C" int cm_recompute_cores(cm_graph* h) {
    int rc = begin_call(h);
    if (rc) return rc;
    CK(h, cudaEventRecord(h->ev[2], h->stream));
    if ((rc = peel_all(h))) return end_call(h, rc);
    DevGraph g = h->g;
    g.n = h->n;
    h->launches++;   // init_mcd launches two kernels
    LAUNCH(h, init_mcd(g, 0, h->n, h->CQ, h->stream));   // CQ holds >= n entries
    CK(h, cudaEventRecord(h->ev[3], h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]);
    h->last.maintain_ms = ms;
    // the superior degrees after the peel: 16 B per vertex (offset, length,
    // SD write) and 8 B per adjacency entry (neighbour id and core)
    h->last.alg_bytes += 16 * (int64_t)h->n + 16 * (int64_t)h->m;
    h->cores_stale = false;
    return end_call(h, CM_OK);
}

// ------------------------------------------------------------------ updates
// Adds one maintenance call's device counters (Ctl::st / ph layout) to s.
// Algorithmic bytes: per iteration 16 B per remaining edge (pair + both
// cores) and 16 B per selected edge (claims, CSR writes); 16 B per visited
// vertex (its row) plus 12 B per slot (neighbour id, core, SD); 12 B per
// slot of an evicted vertex (id, core, support update); 8 B per changed
// vertex plus 8 B per slot (id, core) for the SD fix-up.
static void add_maintain_counters(cm_stats& s, const unsigned long long* st, const unsigned long long* ph) {
    s.iterations += (int64_t)st[ST_ITERS];
    s.select_rounds += (int64_t)st[ST_ROUNDS];
    s.selected += (int64_t)st[ST_SELECTED];
    s.remaining_sum += (int64_t)st[ST_REMSUM];
    s.visited += (int64_t)st[ST_VISITED];
    s.visited_slots += (int64_t)st[ST_VISSLOTS];
    s.evicted += (int64_t)st[ST_EVICTED];
    s.evicted_slots += (int64_t)st[ST_EVSLOTS];
    s.changed += (int64_t)st[ST_CHANGED];
    s.changed_slots += (int64_t)st[ST_CHSLOTS];
    s.waves += (int64_t)st[ST_WAVES];
    s.barriers += (int64_t)st[ST_BARRIERS];
    s.grid_iterations += (int64_t)st[ST_GRID_ITERS];
    for (int i = 0; i < PH_COUNT && i < 7; i++) s.phase_ns[i] += (int64_t)ph[i];
    s.alg_bytes += 16 * (int64_t)st[ST_REMSUM] + 16 * (int64_t)st[ST_SELECTED] + 16 * (int64_t)st[ST_VISITED] +
                   12 * (int64_t)st[ST_VISSLOTS] + 12 * (int64_t)st[ST_EVSLOTS] + 8 * (int64_t)st[ST_CHANGED] +
                   8 * (int64_t)st[ST_CHSLOTS];
}

// Parameters of a maintenance launch pair from the handle: its buffers and
// the schedule its options set (a captured step overrides the schedule).
// The task queue must be allocated first (ensure_tasks).
static MaintainParams handle_params(const cm_graph* h, int op) {
    MaintainParams p{};
    p.g = h->g;
    p.g.n = h->n;
    p.ctl = h->ctl;
    p.R0 = h->R0;
    p.R1 = h->R1;
    p.VQ = h->VQ;
    p.EQ = h->EQ;
    p.CQ = h->CQ;
    p.qmask = h->qmask;
    p.op = op;
    p.limit_ns = (unsigned long long)h->opt.spin_limit_ns;
    p.small_edges = h->small_edges;
    p.small_work = h->small_work;
    p.big_work = h->big_work;
    p.big_wave = h->big_work / 8 > 64 ? h->big_work / 8 : 64;
    p.big_slots = 4 * p.big_work;
    p.HQ = h->HQ;
    p.TQ = h->TQ;
    p.tqmask = h->tq_size - 1;
    p.hub_len = h->hub_len;
    p.block_len = op == CM_OP_INSERT ? h->block_len : h->block_len_del;
    p.claim_max = h->claim_max;
    p.sel_key = h->sel_key;
    p.sel_rounds = h->sel_rounds;
    p.expand_early = h->opt.expand_early;
    return p;
}

// mode 0: maintain cores; mode 1: structure only (cores become stale).
// per_graph (host, nullable): per-graph kept counts of a multi-graph batch.
static int update_device(cm_graph* h, int op, const int32_t* dE, long long k, int64_t* n_applied, int mode,
                         int64_t* per_graph) {
    DevGraph& g = h->g;
    g.n = h->n;
    int rc;
    if (op == CM_OP_INSERT && (rc = ensure_index(h, k))) return rc;
    // A plain delete needs nothing from ingest on the host before the
    // maintenance launches (no relocation, no index growth): the kept count
    // stays on the device, the first launch takes it from there, and an
    // invalid id stops every kernel after ingest (they test the error word
    // first) before anything changed.  The host reads the control block
    // once, at the end.
    const bool device_count = op == CM_OP_DELETE && mode == 0 && !per_graph;
    if (device_count && (rc = ensure_tasks(h))) return rc;
    CK(h, cudaMemsetAsync(h->bset, 0xFF, h->bset_size * sizeof(BSet), h->stream));
    LAUNCH(h, ctl_reset_ingest(h->ctl, h->stream));
    LAUNCH(h, ingest_a(dE, k, nullptr, g, h->bset, h->bset_size - 1, h->ctl, h->stream));
    LAUNCH(h, ingest_b(dE, k, nullptr, op, g, h->bset, h->bset_size - 1, h->R0, h->OVL, h->ctl, h->stream));
    Ctl& c = *h->hctl;
    long long nrem0 = k;   // an upper bound until the count is read
    if (!device_count) {
        if ((rc = rd_ctl(h))) return rc;
        if (c.error == E_INVALID)
            return set_err(h, CM_ERR_INVALID, "edge %lld of the batch names a vertex out of range or deleted",
                           c.bad_index);
        if (c.error) {
            h->poisoned = true;
            return set_err(h, CM_ERR_CUDA, "device error %d during ingest", c.error);
        }
        nrem0 = (long long)c.nrem;
    }
    if (per_graph && h->dpergraph) {
        CK(h, cudaMemsetAsync(h->dpergraph, 0, (size_t)h->ngraphs * 8, h->stream));
        LAUNCH(h, count_multi(h->R0, nrem0, nullptr, h->dbases, h->ngraphs, h->dpergraph, h->stream));
        CK(h, cudaMemcpyAsync(per_graph, h->dpergraph, (size_t)h->ngraphs * 8, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    if (op == CM_OP_INSERT) {
        // Device memory the call may still need comes first: up to here
        // ingest only counted pending insertions (need[]), so a failed
        // allocation clears them and leaves the graph as it was.
        auto undo_need = [&](int why) {
            if (clear_need(h->R0, nrem0, nullptr, h->g, h->stream) != cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess) {
                cudaGetLastError();
                h->poisoned = true;
            }
            return why;
        };
        const long long novl = (long long)c.noverflow;
        if (novl > 0) {
            LAUNCH(h, reloc_size(h->OVL, novl, nullptr, g, h->ctl, h->stream));
            if ((rc = rd_ctl(h))) return rc;
            if ((rc = grow_pool(h, (long long)h->hctl->reloc_need))) return undo_need(rc);
        }
        // relocation moves lists without changing the graph
        if (mode == 0 && nrem0 > 0 && (rc = ensure_tasks(h))) return undo_need(rc);
        if (novl > 0) LAUNCH(h, relocate(h->OVL, novl, nullptr, h->g, h->ctl, h->stream));
        h->idx_live += nrem0;
        LAUNCH(h, index_new_edges(h->R0, nrem0, nullptr, h->g, h->ctl, h->stream));
        LAUNCH(h, clear_need(h->R0, nrem0, nullptr, h->g, h->stream));
    } else if (mode == 0 && nrem0 > 0 && (rc = ensure_tasks(h))) {
        return rc;   // nothing changed yet
    }
    if (nrem0 > 0 && mode == 1) {
        LAUNCH(h, apply_structure(h->R0, nrem0, op, h->g, h->ctl, h->stream));
        if ((rc = rd_ctl(h))) return rc;
        if (c.error) {
            h->poisoned = true;
            return set_err(h, CM_ERR_LIMIT, "structure update failed with device error %d", c.error);
        }
    } else if (nrem0 > 0) {
        if (h->epoch > 0x3F000000u) {   // 30-bit stamps about to wrap: clear them
            CK(h, cudaMemsetAsync(g.chg, 0, (size_t)h->n * 4, h->stream));
            CK(h, cudaMemsetAsync(g.taken, 0, (size_t)h->n * 4, h->stream));
            CK(h, cudaMemsetAsync(g.hw, 0, (size_t)h->n * sizeof(unsigned long long), h->stream));
            h->epoch = 1;
        }
        MaintainParams p = handle_params(h, op);
        p.max_iters = nrem0 + 1;
        int blocks, threads;
        persistent_geometry(h, 0, nrem0, &blocks, &threads);
        p.expect = (uint32_t)blocks;
        bool debug_hang = (h->opt.debug_flags & CM_DEBUG_BARRIER_NEVER_RELEASES) != 0;
        if (debug_hang) {
            p.expect = (uint32_t)blocks + 1;   // test hook: no grid barrier can complete
            p.small_edges = -1;                // and the grid mode must run
            h->opt.debug_flags &= ~CM_DEBUG_BARRIER_NEVER_RELEASES;
        }
        if (h->opt.debug_flags & CM_DEBUG_ITER_CAP) {   // test hook: one iteration at most
            p.max_iters = 1;
            h->opt.debug_flags &= ~CM_DEBUG_ITER_CAP;
        }
        if (h->opt.debug_flags & CM_DEBUG_TASK_WAIT_NEVER_ENDS) {   // test hook: the search never quiesces
            p.phantom_task = 1;
            p.small_edges = -1;
            h->opt.debug_flags &= ~CM_DEBUG_TASK_WAIT_NEVER_ENDS;
        }
        // debug mode: one iteration per launch pair, the store checked after each
        const bool check_each = (h->opt.debug_flags & CM_DEBUG_CHECK_ITERATIONS) != 0;
        p.yield_each = check_each ? 1 : 0;
        // where the call starts: all kept edges remain, in R0
        Resume rs{};
        rs.nrem = (unsigned long long)nrem0;   // replaced on the device by ingest's count (device_count)
        rs.rsel = 0;
        rs.epoch = h->epoch;
        rs.done = 0;
        // every call starts grid-wide: even one edge can start a search over a
        // whole dense shell; the kernel hands down after a small iteration
        rs.want = 0;
        rs.iters = 0;
        LAUNCH(h, ctl_begin_maintain(h->ctl, rs, device_count ? 1 : 0, h->stream));
        CK(h, cudaEventRecord(h->ev[2], h->stream));
        // grid launch then block launch: whichever the resume state names runs,
        // the other returns at once; a handover inside the pair needs no host.
        bool want_grid = rs.want == 0;
        for (int pass = 0;; pass++) {
            if (pass >= (check_each ? (1 << 24) : 256)) {
                h->poisoned = true;
                return set_err(h, CM_ERR_LIMIT, "maintenance did not finish within %d launch pairs", pass);
            }
            if (want_grid) LAUNCH(h, launch_maintain(p, blocks, threads, h->stream));
            LAUNCH(h, launch_maintain_block(p, 1024, h->stream));
            if ((rc = rd_ctl(h))) return rc;
            if (check_each && !c.error) {
                cm_check_report r{};
                if ((rc = run_check(h, &r))) return rc;
                if (!check_clean(r)) {
                    h->poisoned = true;
                    return set_err(h, CM_ERR_LIMIT,
                                   "consistency check failed after iteration %d: %lld SD, %lld key, %lld degree, "
                                   "%lld neighbour-id, %lld k-core mismatches (first vertex %lld)",
                                   pass + 1, (long long)r.sd_mismatches, (long long)r.key_mismatches,
                                   (long long)r.degree_mismatches, (long long)r.bad_neighbour_ids,
                                   (long long)r.kcore_violations, (long long)r.first_bad_vertex);
                }
            }
            if (c.error || c.rs.done) break;
            want_grid = c.rs.want == 0;
        }
        CK(h, cudaEventRecord(h->ev[3], h->stream));
        if (device_count) {   // what ingest found, read with the maintenance counters
            if (c.error == E_INVALID)
                return set_err(h, CM_ERR_INVALID, "edge %lld of the batch names a vertex out of range or deleted",
                               c.bad_index);
            nrem0 = (long long)c.nrem;
        }
        if (c.error) {
            h->poisoned = true;
            const char* why = c.error == E_BARRIER_TIMEOUT ? "a grid barrier or task-queue wait ran out"
                              : c.error == E_ITER_LIMIT   ? "an iteration or retry limit ran out"
                              : c.error == E_CAPACITY     ? "an adjacency list overflowed"
                              : c.error == E_TASKS        ? "the search task queue ran out of slots"
                                                          : "device error";
            return set_err(h, CM_ERR_LIMIT, "maintenance stopped: %s (code %d)", why, c.error);
        }
        CK(h, cudaEventSynchronize(h->ev[3]));
        h->epoch = c.rs.epoch;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]);
        h->last.maintain_ms += ms;
        add_maintain_counters(h->last, c.st, c.ph);
    }
    if (op == CM_OP_DELETE) {
        h->idx_live -= nrem0;
        h->idx_tomb += nrem0;
        h->m -= nrem0;
    } else {
        h->m += nrem0;
    }
    h->last.applied += nrem0;
    if (n_applied) *n_applied = nrem0;
    return CM_OK;
}

static int stage_edges(cm_graph* h, const int32_t* edges, long long k, const int32_t** dE) {
    int rc = ensure_batch(h, k);
    if (rc) return rc;
    if (is_device_ptr(edges)) {
        *dE = edges;
    } else {
        CK(h, cudaMemcpyAsync(h->dbatch, edges, (size_t)k * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
        *dE = h->dbatch;
    }
    return CM_OK;
}

static int update_edges(cm_graph* h, int op, const int32_t* edges, long long k, int64_t* n_applied, int mode) {
    int rc = begin_call(h);
    if (rc) return rc;
    if (k < 0 || (k > 0 && !edges)) return end_call(h, set_err(h, CM_ERR_INVALID, "bad batch size or NULL edges"));
    if (mode == 0 && h->cores_stale)
        return end_call(h, set_err(h, CM_ERR_STATE, "cores are stale: call cm_recompute_cores"));
    if (k == 0) {
        if (n_applied) *n_applied = 0;
        return end_call(h, CM_OK);
    }
    const int32_t* dE = nullptr;
    if ((rc = stage_edges(h, edges, k, &dE))) return end_call(h, rc);
    return end_call(h, update_device(h, op, dE, k, n_applied, mode, nullptr));
}

extern "C" int cm_insert_edges(cm_graph* h, const int32_t* edges, int64_t k, int64_t* n_applied) {
    return update_edges(h, CM_OP_INSERT, edges, k, n_applied, 0);
}
extern "C" int cm_delete_edges(cm_graph* h, const int32_t* edges, int64_t k, int64_t* n_applied) {
    return update_edges(h, CM_OP_DELETE, edges, k, n_applied, 0);
}
extern "C" int cm_apply_edges(cm_graph* h, int32_t op, const int32_t* edges, int64_t k, int64_t* n_applied) {
    if (op != CM_OP_INSERT && op != CM_OP_DELETE) return h ? set_err(h, CM_ERR_INVALID, "bad op") : CM_ERR_INVALID;
    int rc = update_edges(h, op, edges, k, n_applied, 1);
    if (rc == CM_OK) h->cores_stale = true;
    return rc;
}

// ------------------------------------------------------------------ vertex operations
extern "C" int cm_insert_vertices(cm_graph* h, int32_t count, const int64_t* nbr_off, const int32_t* nbrs,
                                  int32_t* first_id, int64_t* n_applied) {
    int rc = begin_call(h);
    if (rc) return rc;
    if (count < 0 || (count > 0 && !nbr_off))
        return end_call(h, set_err(h, CM_ERR_INVALID, "bad vertex count or NULL offsets"));
    if (h->cores_stale) return end_call(h, set_err(h, CM_ERR_STATE, "cores are stale"));
    if ((long long)h->n + count > INT32_MAX) return end_call(h, set_err(h, CM_ERR_CAPACITY, "vertex ids would exceed int32"));
    if (count == 0) {
        if (first_id) *first_id = h->n;
        if (n_applied) *n_applied = 0;
        return end_call(h, CM_OK);
    }
    std::vector<int64_t> hoff((size_t)count + 1);
    if (is_device_ptr(nbr_off)) CK(h, cudaMemcpy(hoff.data(), nbr_off, hoff.size() * 8, cudaMemcpyDeviceToHost));
    else memcpy(hoff.data(), nbr_off, hoff.size() * 8);
    if (hoff[0] != 0) return end_call(h, set_err(h, CM_ERR_INVALID, "nbr_off[0] must be 0"));
    long long slots = 0;
    for (int32_t i = 0; i < count; i++) {
        long long d = hoff[i + 1] - hoff[i];
        if (d < 0) return end_call(h, set_err(h, CM_ERR_INVALID, "nbr_off must be non-decreasing"));
        long long c = (d * (100 + h->opt.slack_pct) + 99) / 100;
        if (c < h->opt.min_cap) c = h->opt.min_cap;
        slots += (c + 3) & ~3ll;
    }
    const long long tot = hoff[count];
    if (tot > 0 && !nbrs) return end_call(h, set_err(h, CM_ERR_INVALID, "NULL neighbour list"));
    // staging in the batch buffer: [edges 2*tot int32][offsets count+1 int64][neighbours tot int32]
    long long ints = 2 * tot + 2 * ((long long)count + 1) + tot + 8;
    if ((rc = ensure_batch(h, (ints + 1) / 2 > tot ? (ints + 1) / 2 : tot))) return end_call(h, rc);
    int64_t* doff = (int64_t*)(h->dbatch + 2 * tot);
    int32_t* dnb = (int32_t*)(doff + count + 1);
    CK(h, cudaMemcpyAsync(doff, hoff.data(), hoff.size() * 8, cudaMemcpyHostToDevice, h->stream));
    const int32_t* nbsrc = nbrs;
    if (tot > 0 && !is_device_ptr(nbrs)) {
        CK(h, cudaMemcpyAsync(dnb, nbrs, (size_t)tot * 4, cudaMemcpyHostToDevice, h->stream));
        nbsrc = dnb;
    }
    if ((rc = reset_ingest_zone(h))) return end_call(h, rc);
    DevGraph g = h->g;
    g.n = h->n;
    LAUNCH(h, validate_vertices(doff, nbsrc, count, h->n, g, h->ctl, h->stream));
    if ((rc = rd_ctl(h))) return end_call(h, rc);
    if (h->hctl->error)
        return end_call(h, set_err(h, CM_ERR_INVALID, "neighbour %lld is out of range, deleted or the vertex itself",
                                   h->hctl->bad_index));
    if ((rc = grow_vertices(h, h->n + count))) return end_call(h, rc);
    if ((rc = grow_pool(h, slots))) return end_call(h, rc);
    const int32_t base = h->n;
    LAUNCH(h, init_vertices(doff, count, base, h->g, h->ctl, h->stream));
    LAUNCH(h, expand_vertex_edges(doff, nbsrc, count, base, h->dbatch, h->stream));
    h->n += count;
    h->g.n = h->n;
    if (first_id) *first_id = base;
    int64_t applied = 0;
    rc = tot > 0 ? update_device(h, CM_OP_INSERT, h->dbatch, tot, &applied, 0, nullptr) : CM_OK;
    if (rc == CM_OK) {
        if (n_applied) *n_applied = applied;
    } else if (rc == CM_ERR_OOM && !h->poisoned) {
        // no edge of the new vertices went in: take the vertices back
        // (their list space stays allocated in the pool, unused)
        h->n = base;
        h->g.n = base;
    } else {
        h->poisoned = true;   // the vertices exist but their edges failed
    }
    return end_call(h, rc);
}

extern "C" int cm_insert_vertex(cm_graph* h, const int32_t* nbrs, int32_t d, int32_t* new_id) {
    if (!h) return CM_ERR_INVALID;
    if (d < 0) return set_err(h, CM_ERR_INVALID, "negative degree");
    int64_t off[2] = {0, d};
    return cm_insert_vertices(h, 1, off, nbrs, new_id, nullptr);
}

extern "C" int cm_delete_vertices(cm_graph* h, int32_t count, const int32_t* ids, int64_t* n_applied) {
    int rc = begin_call(h);
    if (rc) return rc;
    if (count < 0 || (count > 0 && !ids)) return end_call(h, set_err(h, CM_ERR_INVALID, "bad count or NULL ids"));
    if (h->cores_stale) return end_call(h, set_err(h, CM_ERR_STATE, "cores are stale"));
    if (count == 0) {
        if (n_applied) *n_applied = 0;
        return end_call(h, CM_OK);
    }
    int32_t* dids = (int32_t*)dalloc(h, (size_t)count * 4);
    if (!dids) return end_call(h, set_err(h, CM_ERR_OOM, "out of device memory"));
    do {
        cudaError_t e = cudaMemcpyAsync(dids, ids, (size_t)count * 4,
                                        is_device_ptr(ids) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) { rc = fail_cuda(h, e, "copy ids"); break; }
        if ((rc = reset_ingest_zone(h))) break;
        DevGraph g = h->g;
        g.n = h->n;
        h->launches++;
        if ((e = validate_ids(dids, count, g, h->ctl, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "validate_ids"); break; }
        if ((rc = rd_ctl(h))) break;
        if (h->hctl->error) {
            rc = set_err(h, CM_ERR_INVALID, "vertex at position %lld is out of range or already deleted", h->hctl->bad_index);
            break;
        }
        long long bound = (long long)h->hctl->reloc_need;
        if ((rc = ensure_batch(h, bound + 8))) break;
        if ((rc = reset_ingest_zone(h))) break;
        h->launches++;
        if ((e = gather_incident(dids, count, g, h->dbatch, bound, h->ctl, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "gather"); break; }
        if ((rc = rd_ctl(h))) break;
        long long k = (long long)h->hctl->gather_n;
        int64_t applied = 0;
        // The deleted vertices are pinned: their cores stay fixed until they
        // are marked dead, so they never constrain an edge and never drop.
        // Each remaining vertex still loses at most one edge per iteration
        // at its level (Definition 6 for the other endpoints), and once the
        // last edge of a pinned vertex is gone it supports nobody, so the
        // other vertices end with the cores of the graph without them;
        // a hub's edges then go in one iteration instead of one per
        // iteration.
        // the call's last allocation before the graph changes: pinning and
        // the deletions below allocate nothing
        if ((rc = ensure_tasks(h))) break;
        h->launches++;
        if ((e = pin_vertices(dids, count, g, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "pin"); break; }
        if (k > 0 && (rc = update_device(h, CM_OP_DELETE, h->dbatch, k, &applied, 0, nullptr))) break;
        h->launches++;
        if ((e = mark_dead(dids, count, h->g, h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "mark_dead"); break; }
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { rc = fail_cuda(h, e, "sync"); break; }
        if (n_applied) *n_applied = applied;
    } while (0);
    cudaStreamSynchronize(h->stream);
    dfree(h, dids, (size_t)count * 4);
    return end_call(h, rc);
}

extern "C" int cm_delete_vertex(cm_graph* h, int32_t v) {
    int32_t ids[1] = {v};
    return cm_delete_vertices(h, 1, ids, nullptr);
}

// ------------------------------------------------------------------ queries
extern "C" int cm_get_cores(const cm_graph* hc, int32_t* out, int32_t* n_total) {
    cm_graph* h = const_cast<cm_graph*>(hc);
    if (!h) return CM_ERR_INVALID;
    if (h->poisoned) return set_err(h, CM_ERR_STATE, "handle poisoned: %s", h->err.c_str());
    if (n_total) *n_total = h->n;
    if (!out) return CM_OK;
    if (h->cores_stale) return set_err(h, CM_ERR_STATE, "cores are stale: call cm_recompute_cores");
    DevGraph g = h->g;
    g.n = h->n;
    if (is_device_ptr(out)) {
        LAUNCH(h, export_cores(g, out, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return CM_OK;
    }
    LAUNCH(h, export_cores(g, h->CQ, h->stream));   // CQ holds >= n entries
    CK(h, cudaMemcpyAsync(out, h->CQ, (size_t)h->n * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return CM_OK;
}

extern "C" int cm_get_superior_degrees(const cm_graph* hc, int32_t* out, int32_t* n_total) {
    cm_graph* h = const_cast<cm_graph*>(hc);
    if (!h) return CM_ERR_INVALID;
    if (h->poisoned) return set_err(h, CM_ERR_STATE, "handle poisoned: %s", h->err.c_str());
    if (n_total) *n_total = h->n;
    if (!out) return CM_OK;
    if (h->cores_stale) return set_err(h, CM_ERR_STATE, "superior degrees are stale: call cm_recompute_cores");
    DevGraph g = h->g;
    g.n = h->n;
    if (is_device_ptr(out)) {
        LAUNCH(h, export_sd(g, out, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return CM_OK;
    }
    LAUNCH(h, export_sd(g, h->CQ, h->stream));   // CQ holds >= n entries
    CK(h, cudaMemcpyAsync(out, h->CQ, (size_t)h->n * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return CM_OK;
}

// ------------------------------------------------------------------ consistency check
static int run_check(cm_graph* h, cm_check_report* r) {
    if (!h->dchk) {
        if (cudaMalloc(&h->dchk, 8 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            h->dchk = nullptr;
            return set_err(h, CM_ERR_OOM, "out of device memory for the check counters");
        }
    }
    DevGraph g = h->g;
    g.n = h->n;
    LAUNCH(h, check_store(g, h->dchk, h->stream));
    unsigned long long v[7];
    CK(h, cudaMemcpyAsync(v, h->dchk, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    r->sd_mismatches = (int64_t)v[0];
    r->key_mismatches = (int64_t)v[1];
    r->degree_mismatches = (int64_t)v[2];
    r->bad_neighbour_ids = (int64_t)v[3];
    r->kcore_violations = (int64_t)v[4];
    r->vertices_checked = (int64_t)v[5];
    r->first_bad_vertex = v[6] == ~0ull ? -1 : (int64_t)v[6];
    return CM_OK;
}

static bool check_clean(const cm_check_report& r) {
    return r.sd_mismatches == 0 && r.key_mismatches == 0 && r.degree_mismatches == 0 && r.bad_neighbour_ids == 0 &&
           r.kcore_violations == 0;
}

extern "C" int cm_check(cm_graph* h, cm_check_report* out) {
    if (!h || !out) return CM_ERR_INVALID;
    if (h->poisoned) return set_err(h, CM_ERR_STATE, "handle poisoned: %s", h->err.c_str());
    if (h->cores_stale) return set_err(h, CM_ERR_STATE, "cores are stale: call cm_recompute_cores");
    memset(out, 0, sizeof(*out));
    return run_check(h, out);
}

extern "C" int cm_get_edges(const cm_graph* hc, int32_t* out, int64_t cap, int64_t* m) {
    cm_graph* h = const_cast<cm_graph*>(hc);
    if (!h) return CM_ERR_INVALID;
    if (h->poisoned) return set_err(h, CM_ERR_STATE, "handle poisoned: %s", h->err.c_str());
    if (m) *m = h->m;
    if (!out) return CM_OK;
    if (cap < h->m) return set_err(h, CM_ERR_CAPACITY, "capacity %lld < %lld edges", (long long)cap, (long long)h->m);
    int rc = reset_ingest_zone(h);
    if (rc) return rc;
    DevGraph g = h->g;
    g.n = h->n;
    bool dev = is_device_ptr(out);
    int32_t* dst = out;
    size_t bytes = (size_t)(h->m > 0 ? h->m : 1) * 8;
    if (!dev) {
        dst = (int32_t*)dalloc(h, bytes);
        if (!dst) return set_err(h, CM_ERR_OOM, "out of device memory");
    }
    LAUNCH(h, export_edges(g, dst, h->ctl, h->stream));
    if (!dev) CK(h, cudaMemcpyAsync(out, dst, (size_t)h->m * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!dev) dfree(h, dst, bytes);
    return CM_OK;
}

extern "C" int32_t cm_num_vertices(const cm_graph* h) { return h ? h->n : -1; }
extern "C" int64_t cm_num_edges(const cm_graph* h) { return h ? h->m : -1; }

extern "C" int cm_get_stats(const cm_graph* h, cm_stats* out) {
    if (!h || !out) return CM_ERR_INVALID;
    *out = h->last;
    return CM_OK;
}

extern "C" int cm_set_stream(cm_graph* h, void* stream) {
    if (!h) return CM_ERR_INVALID;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->stream = (cudaStream_t)stream;
    return CM_OK;
}

extern "C" const char* cm_last_error(const cm_graph* h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

// ------------------------------------------------------------------ multi-graph
extern "C" int cm_create_multi(cm_graph** out, int32_t ngraphs, const int32_t* ns, const int64_t* ms,
                               const int32_t* edges, const int32_t* cores, const cm_options* opt, void* stream) {
    if (!out || ngraphs <= 0 || !ns || !ms) return set_err(nullptr, CM_ERR_INVALID, "bad multi-graph arguments");
    *out = nullptr;
    std::vector<int32_t> bases((size_t)ngraphs + 1, 0);
    std::vector<long long> eprefix((size_t)ngraphs + 1, 0);
    long long nt = 0;
    for (int32_t i = 0; i < ngraphs; i++) {
        if (ns[i] < 0 || ms[i] < 0) return set_err(nullptr, CM_ERR_INVALID, "negative size for graph %d", i);
        bases[i] = (int32_t)nt;
        nt += ns[i];
        eprefix[i + 1] = eprefix[i] + ms[i];
        if (nt > INT32_MAX) return set_err(nullptr, CM_ERR_CAPACITY, "total vertex count exceeds int32");
    }
    bases[ngraphs] = (int32_t)nt;
    const long long mt = eprefix[ngraphs];
    if (mt > 0 && !edges) return set_err(nullptr, CM_ERR_INVALID, "NULL edges");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* dE = nullptr;
    int32_t* dB = nullptr;
    long long* dP = nullptr;
    unsigned long long* dG = nullptr;
    if (cudaMalloc(&dE, (size_t)(mt > 0 ? mt : 1) * 8) != cudaSuccess || cudaMalloc(&dB, bases.size() * 4) != cudaSuccess ||
        cudaMalloc(&dP, eprefix.size() * 8) != cudaSuccess || cudaMalloc(&dG, bases.size() * 8) != cudaSuccess) {
        cudaGetLastError();
        if (dE) cudaFree(dE);
        if (dB) cudaFree(dB);
        if (dP) cudaFree(dP);
        if (dG) cudaFree(dG);
        return set_err(nullptr, CM_ERR_OOM, "out of device memory");
    }
    bool ok = true;
    if (mt > 0)
        ok = ok && cudaMemcpyAsync(dE, edges, (size_t)mt * 8,
                                   is_device_ptr(edges) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dB, bases.data(), bases.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dP, eprefix.data(), eprefix.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && localize_multi(dE, mt, nullptr, dP, dB, ngraphs, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    int rc = CM_OK;
    cm_graph* h = nullptr;
    if (!ok) {
        rc = set_err(nullptr, CM_ERR_CUDA, "CUDA error while staging a multi-graph");
    } else {
        rc = create_common((int32_t)nt, dE, mt, cores, opt, stream, &h);
        if (rc) {
            if (h) {
                g_create_err = h->err;
                free_all(h);
                h = nullptr;
            }
        }
    }
    cudaFree(dE);
    if (!h) {
        cudaFree(dB);
        cudaFree(dP);
        cudaFree(dG);
        return rc;
    }
    h->ngraphs = ngraphs;
    h->bases = bases;
    h->dbases = dB;
    h->dprefix = dP;
    h->dpergraph = dG;
    *out = h;
    return CM_OK;
}

extern "C" int cm_multi_bases(const cm_graph* h, int32_t* bases, int32_t* ngraphs) {
    if (!h) return CM_ERR_INVALID;
    if (ngraphs) *ngraphs = h->ngraphs;
    if (bases)
        for (int32_t i = 0; i < h->ngraphs; i++) bases[i] = (size_t)i < h->bases.size() ? h->bases[(size_t)i] : 0;
    return CM_OK;
}

extern "C" int cm_update_multi(cm_graph* h, int32_t op, const int64_t* counts, const int32_t* edges,
                               int64_t* n_applied) {
    int rc = begin_call(h);
    if (rc) return rc;
    if ((op != CM_OP_INSERT && op != CM_OP_DELETE) || !counts)
        return end_call(h, set_err(h, CM_ERR_INVALID, "bad arguments"));
    if (h->cores_stale) return end_call(h, set_err(h, CM_ERR_STATE, "cores are stale"));
    if (!h->dprefix) return end_call(h, set_err(h, CM_ERR_STATE, "not a multi-graph handle"));
    const int32_t ng = h->ngraphs;
    std::vector<long long> pre((size_t)ng + 1, 0);
    for (int32_t i = 0; i < ng; i++) {
        if (counts[i] < 0) return end_call(h, set_err(h, CM_ERR_INVALID, "negative count for graph %d", i));
        pre[i + 1] = pre[i] + counts[i];
    }
    const long long k = pre[ng];
    if (k == 0) {
        if (n_applied)
            for (int32_t i = 0; i < ng; i++) n_applied[i] = 0;
        return end_call(h, CM_OK);
    }
    if (!edges) return end_call(h, set_err(h, CM_ERR_INVALID, "NULL edges"));
    if ((rc = ensure_batch(h, k))) return end_call(h, rc);
    CK(h, cudaMemcpyAsync(h->dbatch, edges, (size_t)k * 8,
                          is_device_ptr(edges) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->dprefix, pre.data(), pre.size() * 8, cudaMemcpyHostToDevice, h->stream));
    LAUNCH(h, localize_multi(h->dbatch, k, nullptr, h->dprefix, h->dbases, ng, h->stream));
    int64_t applied = 0;
    std::vector<int64_t> per((size_t)ng, 0);
    rc = update_device(h, op, h->dbatch, k, &applied, 0, per.data());
    if (rc) return end_call(h, rc);
    if (n_applied)
        for (int32_t i = 0; i < ng; i++) n_applied[i] = per[(size_t)i];
    return end_call(h, CM_OK);
}

// ------------------------------------------------------------------ captured update steps
// A step applies one insert batch and then one delete batch to every graph
// of a handle as ONE CUDA graph: localisation and validation of both
// batches, then per phase ingest, relocation behind a device-side capacity
// gate, and the maintenance launch pairs as the body of a conditional WHILE
// node that the single-block kernel drives.  Nothing returns to the host
// between the step's kernels; the host stages inputs before the replay and
// reads one log after it.  The device pointers and kernel parameters are
// baked in at capture, so a change of any of them (growth of a buffer, new
// vertices, another configuration) triggers a re-capture before the replay.

struct StepSig {   // everything a captured step bakes in
    DevGraph g;
    BSet* bset;
    unsigned long long bset_size;
    REdge* R0;
    REdge* R1;
    int32_t* VQ;
    int32_t* EQ;
    int32_t* CQ;
    int32_t* OVL;
    unsigned long long qmask;
    unsigned long long* TQ;
    unsigned long long tq_size;
    cudaStream_t stream;
    cm_step_config cfg;
};

struct cm_step {
    cm_graph* h = nullptr;
    long long max_ins = 0, max_del = 0;
    int32_t ng = 1;
    cm_step_config cfg{};
    cudaStream_t cs = nullptr, cs2 = nullptr;   // capture streams
    int32_t* dE[2] = {nullptr, nullptr};
    long long* dPre = nullptr;                 // 2 x (ng + 1)
    unsigned long long* dK = nullptr;          // 2
    unsigned long long* dPer = nullptr;        // 2 x ng
    StepLog* dLog = nullptr;
    long long* hPre = nullptr;                 // pinned mirrors
    unsigned long long* hK = nullptr;
    unsigned long long* hPer = nullptr;
    StepLog* hLog = nullptr;
    uint32_t* hEpoch = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    StepSig sig{};
    bool captured = false;
    long long captures = 0, replays = 0, fallbacks = 0;
    long long fixed_kernels = 0;                // kernel nodes outside the loop bodies
};

static void step_default_config(const cm_graph* h, cm_step_config* c) {
    memset(c, 0, sizeof(*c));
    c->block_mode_edges = (int32_t)(h->small_edges > 0 ? h->small_edges : -1);
    c->block_mode_enter = (int32_t)h->small_work;
    c->block_mode_leave = (int32_t)h->big_work;
    c->hub_slots = h->hub_len > 0 ? h->hub_len : -1;
    c->blocks_per_sm = 0;
    c->block_slots = h->block_len;
    c->task_claim = h->claim_max;
}

static StepSig step_signature(const cm_step* s) {
    StepSig z;
    memset(&z, 0, sizeof(z));
    const cm_graph* h = s->h;
    z.g = h->g;
    z.g.n = h->n;
    z.bset = h->bset;
    z.bset_size = h->bset_size;
    z.R0 = h->R0;
    z.R1 = h->R1;
    z.VQ = h->VQ;
    z.EQ = h->EQ;
    z.CQ = h->CQ;
    z.OVL = h->OVL;
    z.qmask = h->qmask;
    z.TQ = h->TQ;
    z.tq_size = h->tq_size;
    z.stream = h->stream;
    z.cfg = s->cfg;
    return z;
}

static void step_release_graph(cm_step* s) {
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->exec = nullptr;
    s->graph = nullptr;
    s->captured = false;
}

static MaintainParams step_params(const cm_step* s, int op, int* blocks, int* threads) {
    const cm_graph* h = s->h;
    const cm_step_config& c = s->cfg;
    MaintainParams p = handle_params(h, op);
    p.max_iters = (op == CM_OP_INSERT ? s->max_ins : s->max_del) + 1;
    // the step's own schedule
    p.small_edges = c.block_mode_edges > 0 ? c.block_mode_edges : c.block_mode_edges < 0 ? 0 : 16384;
    p.small_work = c.block_mode_enter > 0 ? c.block_mode_enter : 1024;
    p.big_work = c.block_mode_leave > 0 ? c.block_mode_leave : 8192;
    p.big_wave = p.big_work / 8 > 64 ? p.big_work / 8 : 64;
    p.big_slots = 4 * p.big_work;
    p.hub_len = c.hub_slots > 0 ? (c.hub_slots < 128 ? 128 : c.hub_slots) : c.hub_slots < 0 ? 0 : 1024;
    p.block_len = op == CM_OP_INSERT ? (c.block_slots >= 32 ? c.block_slots : 4096) : h->block_len_del;
    p.claim_max = c.task_claim >= 1 && c.task_claim <= 8 ? c.task_claim : 1;
    int occ = maintain_blocks_per_sm(kGridThreadsHost);
    if (occ < 1) occ = 1;
    int bps = c.blocks_per_sm > 0 && c.blocks_per_sm < occ ? c.blocks_per_sm : occ;
    int sms = h->opt.max_sms > 0 && h->opt.max_sms < h->num_sms ? h->opt.max_sms : h->num_sms;
    *blocks = sms * bps;
    *threads = kGridThreadsHost;
    p.expect = (uint32_t)*blocks;
    return p;
}

// Adds the maintenance loop of one phase to the capture on s->cs: a WHILE
// node whose body is the grid-mode launch and the single-block launch.
static cudaError_t capture_loop(cm_step* s, int op) {
    cudaStreamCaptureStatus st;
    unsigned long long id = 0;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s->cs, &st, &id, &cg, &deps, &edata, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle hc;
    if ((e = cudaGraphConditionalHandleCreate(&hc, cg, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, cg, deps, edata, nd, &cp)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(s->cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s->cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
        return e;
    int blocks = 0, threads = 0;
    MaintainParams p = step_params(s, op, &blocks, &threads);
    p.use_cond = 1;
    p.cond = (unsigned long long)hc;
    cudaError_t e1 = launch_maintain(p, blocks, threads, s->cs2);
    cudaError_t e2 = e1 == cudaSuccess ? launch_maintain_block(p, kGridThreadsHost, s->cs2) : e1;
    cudaGraph_t out = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(s->cs2, &out);
    return e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
}

static cudaError_t capture_phase(cm_step* s, int phase) {
    cm_graph* h = s->h;
    const int op = phase == 0 ? CM_OP_INSERT : CM_OP_DELETE;
    const long long kmax = phase == 0 ? s->max_ins : s->max_del;
    cudaStream_t cs = s->cs;
    DevGraph g = h->g;
    g.n = h->n;
    cudaError_t e;
    unsigned long long* kp = s->dK + phase;
    unsigned long long* np = &h->ctl->nrem;
    s->fixed_kernels += (op == CM_OP_INSERT ? 10 : 5) + (h->dbases ? 1 : 0);
    if ((e = phase_begin(h->ctl, s->dLog, phase, cs)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(h->bset, 0xFF, h->bset_size * sizeof(BSet), cs)) != cudaSuccess) return e;
    if ((e = ingest_a(s->dE[phase], kmax, kp, g, h->bset, h->bset_size - 1, h->ctl, cs)) != cudaSuccess) return e;
    if ((e = ingest_b(s->dE[phase], kmax, kp, op, g, h->bset, h->bset_size - 1, h->R0, h->OVL, h->ctl, cs)) !=
        cudaSuccess)
        return e;
    if (h->dbases) {
        if ((e = cudaMemsetAsync(s->dPer + (size_t)phase * s->ng, 0, (size_t)s->ng * 8, cs)) != cudaSuccess) return e;
        if ((e = count_multi(h->R0, kmax, np, h->dbases, s->ng, s->dPer + (size_t)phase * s->ng, cs)) != cudaSuccess)
            return e;
    }
    if (op == CM_OP_INSERT) {
        if ((e = reloc_size(h->OVL, 2 * kmax, &h->ctl->noverflow, g, h->ctl, cs)) != cudaSuccess) return e;
        if ((e = reloc_gate(g, h->ctl, s->dLog, phase, cs)) != cudaSuccess) return e;
        if ((e = relocate(h->OVL, 2 * kmax, &h->ctl->noverflow, g, h->ctl, cs)) != cudaSuccess) return e;
        // relocation moved rows: the kernels below read offsets from memory, not from g
        if ((e = index_new_edges(h->R0, kmax, np, g, h->ctl, cs)) != cudaSuccess) return e;
        if ((e = clear_need(h->R0, kmax, np, g, cs)) != cudaSuccess) return e;
    }
    if ((e = phase_maintain(h->ctl, s->dLog, phase, cs)) != cudaSuccess) return e;
    if ((e = capture_loop(s, op)) != cudaSuccess) return e;
    return phase_end(h->ctl, s->dLog, phase, cs);
}

static int step_capture(cm_step* s) {
    cm_graph* h = s->h;
    step_release_graph(s);
    DevGraph g = h->g;
    g.n = h->n;
    s->fixed_kernels = 1;
    for (int p = 0; p < 2; p++)
        if ((p == 0 ? s->max_ins : s->max_del) > 0) s->fixed_kernels += h->dbases ? 2 : 1;
    cudaError_t e = cudaStreamBeginCapture(s->cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = step_begin(h->ctl, s->dLog, s->cs);
    for (int p = 0; p < 2 && e == cudaSuccess; p++) {
        const long long kmax = p == 0 ? s->max_ins : s->max_del;
        if (kmax <= 0) continue;
        if (h->dbases)
            e = localize_multi(s->dE[p], kmax, s->dK + p, s->dPre + (size_t)p * (s->ng + 1), h->dbases, s->ng, s->cs);
        if (e == cudaSuccess) e = validate_pairs(s->dE[p], kmax, s->dK + p, p, g, h->ctl, s->cs);
    }
    for (int p = 0; p < 2 && e == cudaSuccess; p++)
        if ((p == 0 ? s->max_ins : s->max_del) > 0) e = capture_phase(s, p);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s->cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec, graph, 0);
    s->graph = graph;
    if (e != cudaSuccess) {
        cudaGetLastError();
        step_release_graph(s);
        return fail_cuda(h, e, "capturing the update step");
    }
    s->sig = step_signature(s);
    s->captured = true;
    s->captures++;
    return CM_OK;
}

extern "C" int cm_step_create(cm_step** out, cm_graph* h, int64_t max_insert, int64_t max_delete,
                              const cm_step_config* cfg) {
    if (!out || !h || max_insert < 0 || max_delete < 0 || max_insert + max_delete == 0)
        return h ? set_err(h, CM_ERR_INVALID, "bad step arguments") : CM_ERR_INVALID;
    *out = nullptr;
    if (h->poisoned) return set_err(h, CM_ERR_STATE, "handle poisoned by an earlier failure: %s", h->err.c_str());
    if (h->stream == nullptr || h->stream == cudaStreamLegacy)
        return set_err(h, CM_ERR_STATE, "a captured step needs a handle on a created (non-default) stream");
    cm_step* s = new (std::nothrow) cm_step();
    if (!s) return set_err(h, CM_ERR_OOM, "out of host memory");
    s->h = h;
    s->max_ins = max_insert;
    s->max_del = max_delete;
    s->ng = h->ngraphs;
    if (cfg) s->cfg = *cfg; else step_default_config(h, &s->cfg);
    const long long kmax = max_insert > max_delete ? max_insert : max_delete;
    int rc = ensure_batch(h, kmax);
    bool ok = rc == CM_OK;
    ok = ok && cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->cs2, cudaStreamNonBlocking) == cudaSuccess;
    for (int p = 0; p < 2 && ok; p++) {
        const long long k = p == 0 ? max_insert : max_delete;
        s->dE[p] = (int32_t*)dalloc(h, (size_t)(k > 0 ? k : 1) * 8);
        ok = s->dE[p] != nullptr;
    }
    ok = ok && cudaMalloc(&s->dPre, (size_t)2 * (s->ng + 1) * 8) == cudaSuccess;
    ok = ok && cudaMalloc(&s->dK, 2 * 8) == cudaSuccess;
    ok = ok && cudaMalloc(&s->dPer, (size_t)2 * s->ng * 8) == cudaSuccess;
    ok = ok && cudaMalloc(&s->dLog, sizeof(StepLog)) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->hPre, (size_t)2 * (s->ng + 1) * 8) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->hK, 2 * 8) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->hPer, (size_t)2 * s->ng * 8) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->hLog, sizeof(StepLog)) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->hEpoch, 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cm_step_destroy(s);
        return rc ? rc : set_err(h, CM_ERR_OOM, "out of memory for an update step");
    }
    *out = s;
    return CM_OK;
}

extern "C" void cm_step_destroy(cm_step* s) {
    if (!s) return;
    if (s->h && s->h->stream) cudaStreamSynchronize(s->h->stream);
    step_release_graph(s);
    if (s->h) {
        for (int p = 0; p < 2; p++) {
            const long long k = p == 0 ? s->max_ins : s->max_del;
            dfree(s->h, s->dE[p], (size_t)(k > 0 ? k : 1) * 8);
        }
    }
    if (s->dPre) cudaFree(s->dPre);
    if (s->dK) cudaFree(s->dK);
    if (s->dPer) cudaFree(s->dPer);
    if (s->dLog) cudaFree(s->dLog);
    if (s->hPre) cudaFreeHost(s->hPre);
    if (s->hK) cudaFreeHost(s->hK);
    if (s->hPer) cudaFreeHost(s->hPer);
    if (s->hLog) cudaFreeHost(s->hLog);
    if (s->hEpoch) cudaFreeHost(s->hEpoch);
    if (s->cs) cudaStreamDestroy(s->cs);
    if (s->cs2) cudaStreamDestroy(s->cs2);
    delete s;
}

extern "C" int cm_step_get_config(const cm_step* s, cm_step_config* cfg) {
    if (!s || !cfg) return CM_ERR_INVALID;
    *cfg = s->cfg;
    return CM_OK;
}

extern "C" int cm_step_set_config(cm_step* s, const cm_step_config* cfg) {
    if (!s || !cfg) return CM_ERR_INVALID;
    s->cfg = *cfg;   // re-captured before the next replay
    return CM_OK;
}

extern "C" int cm_step_counters(const cm_step* s, int64_t* captures, int64_t* replays, int64_t* fallbacks) {
    if (!s) return CM_ERR_INVALID;
    if (captures) *captures = s->captures;
    if (replays) *replays = s->replays;
    if (fallbacks) *fallbacks = s->fallbacks;
    return CM_OK;
}

// Stages one step's batches into the step's buffers (local ids, graph
// order) and its counts; returns the batch sizes.
static int step_stage(cm_step* s, const int64_t* const counts[2], const int32_t* const edges[2], long long k[2]) {
    cm_graph* h = s->h;
    for (int p = 0; p < 2; p++) {
        long long* pre = s->hPre + (size_t)p * (s->ng + 1);
        pre[0] = 0;
        for (int32_t i = 0; i < s->ng; i++) {
            const long long c = counts[p] ? counts[p][i] : 0;
            if (c < 0) return set_err(h, CM_ERR_INVALID, "negative count for graph %d", i);
            pre[i + 1] = pre[i] + c;
        }
        k[p] = pre[s->ng];
        if (k[p] > (p == 0 ? s->max_ins : s->max_del))
            return set_err(h, CM_ERR_CAPACITY, "%s batch of %lld edges exceeds the step's capacity",
                           p == 0 ? "insert" : "delete", k[p]);
        if (k[p] > 0 && !edges[p]) return set_err(h, CM_ERR_INVALID, "NULL edges");
        s->hK[p] = (unsigned long long)k[p];
    }
    for (int p = 0; p < 2; p++) {
        if (k[p] > 0)
            CK(h, cudaMemcpyAsync(s->dE[p], edges[p], (size_t)k[p] * 8,
                                  is_device_ptr(edges[p]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream));
    }
    CK(h, cudaMemcpyAsync(s->dPre, s->hPre, (size_t)2 * (s->ng + 1) * 8, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(s->dK, s->hK, 16, cudaMemcpyHostToDevice, h->stream));
    return CM_OK;
}

// Host-side preconditions of a replay; re-captures when anything baked in changed.
static int step_prepare(cm_step* s, long long kins) {
    cm_graph* h = s->h;
    int rc;
    if ((rc = ensure_index(h, kins))) return rc;
    const long long kmax = s->max_ins > s->max_del ? s->max_ins : s->max_del;
    if ((rc = ensure_batch(h, kmax))) return rc;
    if ((rc = ensure_tasks(h))) return rc;
    if (h->epoch > 0x3F000000u) {   // 30-bit stamps about to wrap: clear them
        DevGraph& g = h->g;
        CK(h, cudaMemsetAsync(g.chg, 0, (size_t)h->n * 4, h->stream));
        CK(h, cudaMemsetAsync(g.taken, 0, (size_t)h->n * 4, h->stream));
        CK(h, cudaMemsetAsync(g.hw, 0, (size_t)h->n * sizeof(unsigned long long), h->stream));
        h->epoch = 1;
    }
    *s->hEpoch = h->epoch;
    CK(h, cudaMemcpyAsync(&h->ctl->rs.epoch, s->hEpoch, 4, cudaMemcpyHostToDevice, h->stream));
    StepSig now = step_signature(s);
    if (!s->captured || memcmp(&now, &s->sig, sizeof(StepSig)) != 0) {
        CK(h, cudaStreamSynchronize(h->stream));
        if ((rc = step_capture(s))) return rc;
    }
    return CM_OK;
}

// Reads the log of a replay and brings the host mirrors up to date.  If the
// pool could not take the insert phase's relocations, the step stopped
// before changing anything and both phases run on the ordinary path.
static int step_finish(cm_step* s, const long long k[2], int64_t* applied[2]) {
    cm_graph* h = s->h;
    CK(h, cudaMemcpyAsync(s->hLog, s->dLog, sizeof(StepLog), cudaMemcpyDeviceToHost, h->stream));
    if (h->dbases)
        CK(h, cudaMemcpyAsync(s->hPer, s->dPer, (size_t)2 * s->ng * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const StepLog& L = *s->hLog;
    const Ctl& c = *h->hctl;
    for (int p = 0; p < 2; p++) {
        if (L.error[p] == E_INVALID || (L.defer == p + 1 && c.error == E_INVALID)) {
            const long long bi = c.bad_index;
            return set_err(h, CM_ERR_INVALID, "edge %lld of the %s batch names a vertex out of range or deleted",
                           bi & ((1ll << 40) - 1), (bi >> 40) ? "delete" : "insert");
        }
    }
    if (c.error == E_INVALID) {
        const long long bi = c.bad_index;
        return set_err(h, CM_ERR_INVALID, "edge %lld of the %s batch names a vertex out of range or deleted",
                       bi & ((1ll << 40) - 1), (bi >> 40) ? "delete" : "insert");
    }
    if (c.error) {
        h->poisoned = true;
        return set_err(h, CM_ERR_LIMIT, "captured step stopped with device error %d", c.error);
    }
    h->epoch = L.epoch_end;
    cm_stats& st = h->last;
    for (int p = 0; p < 2; p++) {
        const bool ran = L.defer == 0 || L.defer > p + 1;
        if (!ran) break;
        const long long kept = (long long)L.kept[p];
        if (p == 0) {
            h->idx_live += kept;
            h->m += kept;
        } else {
            h->idx_live -= kept;
            h->idx_tomb += kept;
            h->m -= kept;
        }
        st.applied += kept;
        add_maintain_counters(st, L.st[p], L.ph[p]);
        if (applied[p]) {
            if (h->dbases) {
                for (int32_t i = 0; i < s->ng; i++) applied[p][i] = (int64_t)s->hPer[(size_t)p * s->ng + i];
            } else {
                applied[p][0] = kept;
            }
        }
    }
    if (L.defer == 1) {   // pool short: ordinary path for both phases (the graph is unchanged)
        s->fallbacks++;
        for (int p = 0; p < 2; p++) {
            if (k[p] == 0) {
                if (applied[p])
                    for (int32_t i = 0; i < s->ng; i++) applied[p][i] = 0;
                continue;
            }
            std::vector<int64_t> per((size_t)s->ng, 0);
            int64_t a = 0;
            int rc = update_device(h, p == 0 ? CM_OP_INSERT : CM_OP_DELETE, s->dE[p], k[p], &a, 0,
                                   h->dbases ? per.data() : nullptr);
            if (rc) return rc;
            if (applied[p]) {
                if (h->dbases) {
                    for (int32_t i = 0; i < s->ng; i++) applied[p][i] = per[(size_t)i];
                } else {
                    applied[p][0] = a;
                }
            }
        }
    }
    return CM_OK;
}

static int step_run_staged(cm_step* s, const long long k[2], int64_t* applied[2]) {
    cm_graph* h = s->h;
    int rc = step_prepare(s, k[0]);
    if (rc) return rc;
    CK(h, cudaEventRecord(h->ev[2], h->stream));
    CK(h, cudaGraphLaunch(s->exec, h->stream));
    CK(h, cudaEventRecord(h->ev[3], h->stream));
    s->replays++;
    rc = step_finish(s, k, applied);
    // kernels the replay ran: the fixed nodes and two per loop pass
    h->launches += s->fixed_kernels + 2 * (long long)(s->hLog->passes[0] + s->hLog->passes[1]);
    if (rc) return rc;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]);
    h->last.maintain_ms += ms;
    return CM_OK;
}

extern "C" int cm_step_run(cm_step* s, const int64_t* ins_counts, const int32_t* ins_edges,
                           const int64_t* del_counts, const int32_t* del_edges, int64_t* ins_applied,
                           int64_t* del_applied) {
    if (!s) return CM_ERR_INVALID;
    cm_graph* h = s->h;
    int rc = begin_call(h);
    if (rc) return rc;
    if (h->cores_stale) return end_call(h, set_err(h, CM_ERR_STATE, "cores are stale: call cm_recompute_cores"));
    const int64_t* counts[2] = {ins_counts, del_counts};
    const int32_t* edges[2] = {ins_edges, del_edges};
    long long k[2];
    if ((rc = step_stage(s, counts, edges, k))) return end_call(h, rc);
    int64_t* applied[2] = {ins_applied, del_applied};
    return end_call(h, step_run_staged(s, k, applied));
}

// ------------------------------------------------------------------ autotuner
// Times candidate configurations of a step on a real batch: the graph's
// state is saved once, and before every trial the state and the raw batch
// are restored, so each trial replays the same work from the same graph.
struct Snapshot {
    size_t nv = 0, adj = 0, idx = 0;
    unsigned char* words = nullptr;   // hc, hw, then kc (20 bytes per vertex)
    int64_t* off = nullptr;
    int32_t* i32 = nullptr;        // end, cap, deg, chg, taken (5 x nv)
    unsigned long long* claims = nullptr;   // claim0, claim1 (2 x nv)
    int32_t* pool = nullptr;
    Bucket* index = nullptr;
    Ctl* ctl = nullptr;
    int64_t m = 0, idx_live = 0, idx_tomb = 0;
    uint32_t epoch = 0;
    int32_t n = 0;
};

static void snap_free(cm_graph* h, Snapshot& z) {
    dfree(h, z.words, z.nv * 20);
    dfree(h, z.off, z.nv * 8);
    dfree(h, z.i32, z.nv * 4 * 5);
    dfree(h, z.claims, z.nv * 8 * 2);
    dfree(h, z.pool, z.adj * 4);
    dfree(h, z.index, z.idx * sizeof(Bucket));
    dfree(h, z.ctl, sizeof(Ctl));
    z = Snapshot{};
}

static int snap_copy(cm_graph* h, Snapshot& z, bool save) {
    DevGraph& g = h->g;
    const cudaMemcpyKind kd = cudaMemcpyDeviceToDevice;
    cudaStream_t st = h->stream;
    auto cp = [&](void* snap, void* live, size_t bytes) {
        return save ? cudaMemcpyAsync(snap, live, bytes, kd, st) : cudaMemcpyAsync(live, snap, bytes, kd, st);
    };
    const size_t nv = z.nv;
    CK(h, cp(z.words, g.hc, nv * 8));
    CK(h, cp(z.words + nv * 8, g.hw, nv * 8));
    CK(h, cp(z.words + nv * 16, g.kc, nv * 4));
    CK(h, cp(z.off, g.off, nv * 8));
    CK(h, cp(z.i32 + 0 * nv, g.end, nv * 4));
    CK(h, cp(z.i32 + 1 * nv, g.cap, nv * 4));
    CK(h, cp(z.i32 + 2 * nv, g.deg, nv * 4));
    CK(h, cp(z.i32 + 3 * nv, g.chg, nv * 4));
    CK(h, cp(z.i32 + 4 * nv, g.taken, nv * 4));
    CK(h, cp(z.claims, g.claim0, nv * 8));
    CK(h, cp(z.claims + nv, g.claim1, nv * 8));
    if (z.adj) CK(h, cp(z.pool, g.adj, z.adj * 4));
    CK(h, cp(z.index, g.idx, z.idx * sizeof(Bucket)));
    CK(h, cp(z.ctl, h->ctl, sizeof(Ctl)));
    if (save) {
        z.m = h->m;
        z.idx_live = h->idx_live;
        z.idx_tomb = h->idx_tomb;
        z.epoch = h->epoch;
        z.n = h->n;
    } else {
        h->m = z.m;
        h->idx_live = z.idx_live;
        h->idx_tomb = z.idx_tomb;
        h->epoch = z.epoch;
        h->n = z.n;
    }
    return CM_OK;
}

static int snap_take(cm_graph* h, Snapshot& z) {
    CK(h, cudaMemcpyAsync(&h->hctl->adj_top, &h->ctl->adj_top, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    z.nv = (size_t)h->n;
    z.adj = (size_t)h->hctl->adj_top;
    z.idx = (size_t)h->idx_size;
    z.words = (unsigned char*)dalloc(h, z.nv * 20);
    z.off = (int64_t*)dalloc(h, z.nv * 8);
    z.i32 = (int32_t*)dalloc(h, z.nv * 4 * 5);
    z.claims = (unsigned long long*)dalloc(h, z.nv * 8 * 2);
    z.pool = (int32_t*)dalloc(h, z.adj * 4);
    z.index = (Bucket*)dalloc(h, z.idx * sizeof(Bucket));
    z.ctl = (Ctl*)dalloc(h, sizeof(Ctl));
    if (!z.words || !z.off || !z.i32 || !z.claims || !z.pool || !z.index || !z.ctl) {
        snap_free(h, z);
        return set_err(h, CM_ERR_OOM, "out of device memory for the tuner's copy of the graph");
    }
    return snap_copy(h, z, true);
}

extern "C" int cm_step_autotune(cm_step* s, const int64_t* ins_counts, const int32_t* ins_edges,
                                const int64_t* del_counts, const int32_t* del_edges, int32_t reps,
                                cm_tune_report* report) {
    if (!s) return CM_ERR_INVALID;
    cm_graph* h = s->h;
    int rc = begin_call(h);
    if (rc) return rc;
    if (h->cores_stale) return end_call(h, set_err(h, CM_ERR_STATE, "cores are stale"));
    if (reps < 1) reps = 1;
    const int64_t* counts[2] = {ins_counts, del_counts};
    const int32_t* edges[2] = {ins_edges, del_edges};
    long long k[2];
    if ((rc = step_stage(s, counts, edges, k))) return end_call(h, rc);
    // every buffer the step uses is in place before the graph is saved, so
    // no trial reallocates and every trial sees the same pointers
    if ((rc = ensure_index(h, k[0]))) return end_call(h, rc);
    // keep the raw batches: the step localises them in place
    int32_t* raw[2] = {nullptr, nullptr};
    for (int p = 0; p < 2; p++) {
        if (k[p] == 0) continue;
        raw[p] = (int32_t*)dalloc(h, (size_t)k[p] * 8);
        if (!raw[p]) {
            dfree(h, raw[0], (size_t)k[0] * 8);
            return end_call(h, set_err(h, CM_ERR_OOM, "out of device memory for the tuner's batch copy"));
        }
        CK(h, cudaMemcpyAsync(raw[p], s->dE[p], (size_t)k[p] * 8, cudaMemcpyDeviceToDevice, h->stream));
    }
    Snapshot z;
    if ((rc = snap_take(h, z))) {
        for (int p = 0; p < 2; p++) dfree(h, raw[p], (size_t)k[p] * 8);
        return end_call(h, rc);
    }
    // coordinate descent over the knobs, in this order: frontier
    // granularity (hub threshold, then block-scan threshold), block shape
    // (resident blocks per SM), execution-mode thresholds; each knob takes
    // the best of its values with the others at the best found so far
    const cm_step_config first = s->cfg;
    double best_ms = 1e30, first_ms = 0;
    cm_step_config best = first;
    int tried = 0;
    int64_t* none[2] = {nullptr, nullptr};
    std::vector<float> t;
    auto time_config = [&](const cm_step_config& c, double* med) -> int {
        s->cfg = c;
        t.clear();
        for (int r = 0; r < reps; r++) {
            int e = snap_copy(h, z, false);
            if (e) return e;
            for (int p = 0; p < 2; p++)
                if (k[p]) CK(h, cudaMemcpyAsync(s->dE[p], raw[p], (size_t)k[p] * 8, cudaMemcpyDeviceToDevice, h->stream));
            CK(h, cudaMemcpyAsync(s->dPre, s->hPre, (size_t)2 * (s->ng + 1) * 8, cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaMemcpyAsync(s->dK, s->hK, 16, cudaMemcpyHostToDevice, h->stream));
            memset(&h->last, 0, sizeof(h->last));
            if ((e = step_run_staged(s, k, none))) return e;
            t.push_back((float)h->last.maintain_ms);
        }
        std::sort(t.begin(), t.end());
        *med = t[t.size() / 2];
        tried++;
        return CM_OK;
    };
    rc = time_config(first, &first_ms);
    best_ms = first_ms;
    const int32_t hubs[] = {512, 1024, 4096, -1};
    const int32_t blocks[] = {256, 1024, 4096};
    const int32_t bps[] = {1, 2};
    const int32_t modes[][3] = {{16384, 1024, 8192}, {65536, 4096, 32768}, {-1, 1024, 8192}};
    const int32_t claims[] = {1, 2, 8};
    for (int knob = 0; knob < 5 && rc == CM_OK; knob++) {
        const int nv = knob == 0 ? 4 : knob == 1 ? 3 : knob == 2 ? 2 : 3;
        cm_step_config base = best;
        for (int v = 0; v < nv && rc == CM_OK; v++) {
            cm_step_config c = base;
            if (knob == 0) c.hub_slots = hubs[v];
            else if (knob == 1) c.block_slots = blocks[v];
            else if (knob == 2) c.blocks_per_sm = bps[v];
            else if (knob == 4) c.task_claim = claims[v];
            else {
                c.block_mode_edges = modes[v][0];
                c.block_mode_enter = modes[v][1];
                c.block_mode_leave = modes[v][2];
            }
            double med = 0;
            if ((rc = time_config(c, &med))) break;
            if (med < best_ms) {
                best_ms = med;
                best = c;
            }
        }
    }
    // leave the graph as it was before tuning and the step on the winner
    int rc2 = snap_copy(h, z, false);
    CK(h, cudaStreamSynchronize(h->stream));
    snap_free(h, z);
    for (int p = 0; p < 2; p++) dfree(h, raw[p], (size_t)k[p] * 8);
    s->cfg = rc == CM_OK ? best : first;
    if (rc == CM_OK) rc = rc2;
    if (rc == CM_OK && report) {
        report->best = best;
        report->best_ms = best_ms;
        report->first_ms = first_ms;
        report->tried = tried;
        report->reps = reps;
    }
    memset(&h->last, 0, sizeof(h->last));
    return end_call(h, rc);
}
