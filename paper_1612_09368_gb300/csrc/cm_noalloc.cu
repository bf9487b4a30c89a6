// cm_noalloc.cu -- core numbers of a caller-provided CSR graph without any
// device allocation (cm_core_numbers_noalloc).
//
// Who needs this: callers that cannot call cudaMalloc -- a process whose
// framework has already reserved the device memory for its own pool, or a
// latency-critical loop that must not wait on the allocator (cudaMalloc and
// cudaFree can synchronise the device).  Every other entry point of this
// library allocates its graph store; this one only reads the caller's CSR
// and writes the caller's output array.
//
// Its scratch lives in one file-scope __device__ array (kScratchBytes, sized
// for kMaxVertices vertices).  Every GPU that loads the library holds it
// until the process exits.  All calls share it: a call clears what must
// start at zero, and two calls whose work overlaps on the GPU (for example
// on two streams) race on it.  The device address of the array is looked
// up once per device, on the first call made with that device current;
// make that first call before any stream capture.  Every call waits for its
// stream (it reads the kernel's error word back) before it returns.
#include <mutex>

#include "../../include/coremaint.h"
#include "cm_common.cuh"

namespace cm {

constexpr int32_t kMaxVertices = 1 << 20;
constexpr size_t kCtlBytes = 4096;
constexpr int kBigDegree = 2048;                  // a vertex this large is scanned in chunk tasks
constexpr int kChunkSlots = 512;                  // slots per chunk task
constexpr unsigned long long kMaxChunks = 1 << 18;   // chunk tasks per sub-wave (more: the warp scans alone)
constexpr unsigned long long kNoChunk = ~0ull;
// Ctl, 4 int32 per vertex, then the chunk tasks of a sub-wave
constexpr size_t kScratchBytes = kCtlBytes + 4ull * sizeof(int32_t) * kMaxVertices + kMaxChunks * 8;
static_assert(sizeof(Ctl) <= kCtlBytes, "control block does not fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kNoallocUnpeeled = -2;

struct PeelCsrParams {
    int32_t n;
    uint32_t expect;
    const int64_t* row_off;
    const int32_t* adj;
    int32_t* cores;
    unsigned char* scratch;
    unsigned long long limit_ns;
};

// Level-synchronous bucket peeling of a static CSR graph (the same procedure
// as the store's full decomposition): at level k every remaining vertex with
// degree <= k gets core k and leaves, taking one degree from each remaining
// neighbour; neighbours that reach k leave at the same level; empty levels
// are skipped to the smallest remaining degree.  A departing vertex of at
// least kBigDegree neighbours is not scanned by the warp that takes it: its
// list becomes kChunkSlots-slot chunk tasks that every warp takes after the
// sub-wave's barrier, so one hub does not hold the whole grid at the next
// barrier.
__global__ void __launch_bounds__(512) peel_csr_kernel(PeelCsrParams P) {
    Ctl* C = reinterpret_cast<Ctl*>(P.scratch);
    int32_t* dcur = reinterpret_cast<int32_t*>(P.scratch + kCtlBytes);
    int32_t* L0 = dcur + kMaxVertices;
    int32_t* L1 = L0 + kMaxVertices;
    int32_t* F = L1 + kMaxVertices;
    unsigned long long* chunks = reinterpret_cast<unsigned long long*>(F + kMaxVertices);
    const int lane = lane_id();
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = gwarp * 32; base < P.n; base += nwarps * 32) {
        long long v = base + lane;
        bool in = v < P.n;
        if (in) {
            dcur[v] = (int32_t)(P.row_off[v + 1] - P.row_off[v]);
            P.cores[v] = kNoallocUnpeeled;
        }
        warp_push(&C->pc[1], L0, ~0ull, in, (int32_t)v);
    }
    if (!grid_sync(C, P.expect, P.limit_ns)) return;
    unsigned long long nl = vload64(&C->spc[1]);
    int32_t* Lc = L0;
    int32_t* Ln = L1;
    int k = 0;
    unsigned long long ft = 0;
    while (nl > 0) {
        const unsigned long long f0 = ft;
        int mx = 0;
        for (long long base = gwarp * 32; base < (long long)nl; base += nwarps * 32) {
            long long i = base + lane;
            bool peel = false, keep = false;
            int v = 0;
            if (i < (long long)nl) {
                v = Lc[i];
                if (P.cores[v] == kNoallocUnpeeled) {
                    int d = dcur[v];
                    if (d <= k) {
                        P.cores[v] = k;
                        peel = true;
                    } else {
                        keep = true;
                        mx = max(mx, 0x7FFFFFFF - d);
                    }
                }
            }
            warp_push(&C->tail[0], F, ~0ull, peel, v);
            warp_push(&C->pc[1], Ln, ~0ull, keep, v);
        }
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx) atomicMax(&C->pc[3], (unsigned long long)mx);
        if (!grid_sync(C, P.expect, P.limit_ns)) return;
        const unsigned long long fhi = vload64(&C->stail[0]);
        const unsigned long long nln = vload64(&C->spc[1]);
        const unsigned long long smx = vload64(&C->spc[3]);
        int32_t* t = Lc;
        Lc = Ln;
        Ln = t;
        nl = nln;
        if (fhi == f0) {
            if (nl == 0) break;
            k = 0x7FFFFFFF - (int)smx;
            continue;
        }
        // one degree off every unpeeled neighbour in list slots [a, b); a
        // neighbour brought to k leaves now and joins the frontier
        auto decrement = [&](long long a, long long b) {
            for (long long t0 = a; t0 < b; t0 += 32) {
                long long tt = t0 + lane;
                int w = tt < b ? P.adj[tt] : -1;
                bool p = false;
                if (w >= 0 && w < P.n && P.cores[w] == kNoallocUnpeeled) {
                    if (atomicSub(&dcur[w], 1) == k + 1) {
                        P.cores[w] = k;
                        p = true;
                    }
                }
                warp_push(&C->tail[0], F, ~0ull, p, w);
            }
        };
        unsigned long long lo = f0, hi = fhi;
        while (hi > lo) {
            const unsigned long long cnt = hi - lo;
            for (;;) {
                unsigned long long j = 0;
                if (lane == 0) j = atomicAdd(&C->pc[2], 1ull);
                j = __shfl_sync(0xffffffffu, j, 0);
                if (j >= cnt) break;
                const int v = F[lo + j];
                const long long a = P.row_off[v], b = P.row_off[v + 1];
                if (b - a >= kBigDegree) {   // chunk tasks (vertex, chunk), counted in pc[0]
                    const unsigned long long nch = (unsigned long long)((b - a + kChunkSlots - 1) / kChunkSlots);
                    unsigned long long tb = 0;
                    if (lane == 0) tb = atomicAdd(&C->pc[0], nch);
                    tb = __shfl_sync(0xffffffffu, tb, 0);
                    const bool fits = tb + nch <= kMaxChunks;
                    for (unsigned long long c = lane; c < nch && tb + c < kMaxChunks; c += 32)
                        chunks[tb + c] = fits ? (((unsigned long long)(uint32_t)v << 32) | (uint32_t)c) : kNoChunk;
                    if (fits) continue;
                }
                decrement(a, b);
            }
            if (!grid_sync(C, P.expect, P.limit_ns)) return;
            const unsigned long long nch = min(vload64(&C->spc[0]), kMaxChunks);
            if (nch > 0) {
                for (unsigned long long c = (unsigned long long)gwarp; c < nch; c += (unsigned long long)nwarps) {
                    const unsigned long long task = chunks[c];
                    if (task == kNoChunk) continue;
                    const int v = (int)(task >> 32);
                    const long long a = P.row_off[v] + (long long)(task & 0xFFFFFFFFu) * kChunkSlots;
                    const long long end = P.row_off[v + 1];
                    decrement(a, a + kChunkSlots < end ? a + (long long)kChunkSlots : end);
                }
                if (!grid_sync(C, P.expect, P.limit_ns)) return;
            }
            lo = hi;
            hi = vload64(&C->stail[0]);
        }
        ft = hi;
        k++;
    }
}

// Per-device address of the scratch array (looked up once per device).
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

static int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CM_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    return CM_OK;
}

static bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A failed runtime call: clear the error it left, so that a later
// cudaGetLastError of the caller (or of a framework) does not report it.
static int cuda_failed() {
    cudaGetLastError();
    return CM_ERR_CUDA;
}

}  // namespace cm

using namespace cm;

extern "C" int cm_core_numbers_noalloc(int32_t n, const int64_t* row_off, const int32_t* adj, int32_t* cores,
                                       void* stream) {
    if (n < 0) return CM_ERR_INVALID;
    if (n > kMaxVertices) return CM_ERR_CAPACITY;
    if (n == 0) return CM_OK;
    if (!row_off || !adj || !cores) return CM_ERR_INVALID;
    if (!on_device(row_off) || !on_device(adj) || !on_device(cores)) return CM_ERR_INVALID;
    unsigned char* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the control block must start at zero; the per-vertex arrays are written before they are read
    if (cudaMemsetAsync(scratch, 0, kCtlBytes, s) != cudaSuccess) return cuda_failed();
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_failed();
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cuda_failed();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, peel_csr_kernel, 512, 0) != cudaSuccess || occ < 1)
        return cuda_failed();
    int blocks = sms * occ;
    long long want = ((long long)n + 511) / 512;
    if (want < blocks) blocks = (int)(want > 0 ? want : 1);
    PeelCsrParams p{};
    p.n = n;
    p.expect = (uint32_t)blocks;
    p.row_off = row_off;
    p.adj = adj;
    p.cores = cores;
    p.scratch = scratch;
    p.limit_ns = 4000000000ull;
    void* args[] = {&p};
    if (cudaLaunchCooperativeKernel((const void*)peel_csr_kernel, dim3(blocks), dim3(512), args, 0, s) != cudaSuccess)
        return cuda_failed();
    int err = 0;
    if (cudaMemcpyAsync(&err, &reinterpret_cast<Ctl*>(scratch)->error, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_failed();
    return err ? CM_ERR_LIMIT : CM_OK;
}
