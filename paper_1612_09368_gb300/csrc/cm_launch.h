// cm_launch.h -- host-side declarations of the kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cm_common.cuh"

namespace cm {

// Batch-dedupe hash set entry: key -> smallest input position.
struct __align__(16) BSet {
    unsigned long long key;
    uint32_t pos;
    uint32_t pad;
};

// Parameters of a maintenance launch; where the call stands (remaining
// edges, epoch, mode) lives in Ctl::rs.
struct MaintainParams {
    DevGraph g;
    Ctl* ctl;
    REdge* R0;
    REdge* R1;
    int32_t* VQ;
    int32_t* EQ;
    int32_t* CQ;
    unsigned long long qmask;
    int32_t op;               // 0 insert, 1 delete
    uint32_t expect;          // blocks a grid barrier waits for
    unsigned long long limit_ns;
    long long max_iters;
    long long small_edges;    // grid -> block mode when at most this many edges remain ...
    long long small_work;     // ... and the last iteration touched at most this many items
    long long big_work;       // block -> grid mode when an iteration touches more
    long long big_wave;       // block -> grid mode, inside an iteration, before a wave this large
    long long big_slots;      // ... or before a wave whose vertices' lists hold this many slots
    HubItem* HQ;              // hub items of the current search (ring of kHubRing)
    unsigned long long* TQ;   // grid-mode task queue (ring, TASK_EMPTY when free)
    unsigned long long tqmask;
    int32_t hub_len;          // grid mode: vertices with at least this many slots are scanned grid-wide
    int32_t block_len;        // vertices with at least this many slots are scanned by a whole block
    int32_t claim_max;        // grid-mode task queue: most slots a warp claims at once
    int32_t sel_key;          // selection order: 0 fmix64 of the canonical key, 1 the key itself
    int32_t sel_rounds;       // claim rounds per iteration (0 = until the set is maximal)
    int32_t use_cond;         // inside a captured step: the single-block kernel drives the loop node
    int32_t phantom_task;     // test hook: every grid search counts one task that is never queued
    int32_t expand_early;     // frontier expansion in the CSD pass: >= 0 yes (default), -1 after it (paper's order)
    int32_t yield_each;       // debug: end the launch after every iteration (its SD fix-up done)
    unsigned long long cond;  // that node's conditional handle
};

struct PeelParams {
    DevGraph g;
    Ctl* ctl;
    int32_t* dcur;    // working degree [n]
    int32_t* L0;      // remaining-vertex lists [n]
    int32_t* L1;
    int32_t* F;       // frontier ring [qmask+1]
    unsigned long long qmask;
    unsigned long long* chunks;     // chunk tasks of high-degree frontier vertices
    unsigned long long chunk_cap;
    uint32_t expect;
    uint32_t pad;
    unsigned long long limit_ns;
};

// ---- maintenance (cm_maintain.cu); kp / np: device item counts of a captured step (else NULL)
cudaError_t ctl_reset_ingest(Ctl* c, cudaStream_t s);
cudaError_t ctl_begin_maintain(Ctl* c, const Resume& rs, int take_nrem, cudaStream_t s);
cudaError_t ingest_a(const int32_t* E, long long k, const unsigned long long* kp, DevGraph g, BSet* bs,
                     unsigned long long bmask, Ctl* c, cudaStream_t s);
cudaError_t ingest_b(const int32_t* E, long long k, const unsigned long long* kp, int op, DevGraph g,
                     const BSet* bs, unsigned long long bmask, REdge* R0, int32_t* ovl, Ctl* c, cudaStream_t s);
cudaError_t index_new_edges(REdge* R, long long n, const unsigned long long* np, DevGraph g, Ctl* c,
                            cudaStream_t s);
cudaError_t reloc_size(const int32_t* ovl, long long novl, const unsigned long long* np, DevGraph g, Ctl* c,
                       cudaStream_t s);
cudaError_t reloc_gate(DevGraph g, Ctl* c, StepLog* log, int phase, cudaStream_t s);
cudaError_t relocate(const int32_t* ovl, long long novl, const unsigned long long* np, DevGraph g, Ctl* c,
                     cudaStream_t s);
cudaError_t clear_need(const REdge* R, long long n, const unsigned long long* np, DevGraph g, cudaStream_t s);
cudaError_t step_begin(Ctl* c, StepLog* log, cudaStream_t s);
cudaError_t phase_begin(Ctl* c, StepLog* log, int phase, cudaStream_t s);
cudaError_t phase_maintain(Ctl* c, StepLog* log, int phase, cudaStream_t s);
cudaError_t phase_end(Ctl* c, StepLog* log, int phase, cudaStream_t s);
cudaError_t apply_structure(const REdge* R, long long n, int op, DevGraph g, Ctl* c, cudaStream_t s);
cudaError_t launch_maintain(const MaintainParams& p, int blocks, int threads, cudaStream_t s);
cudaError_t launch_maintain_block(const MaintainParams& p, int threads, cudaStream_t s);
// kernel symbols of the two execution modes, for graph capture
const void* maintain_kernel_symbol(int mode);
int maintain_blocks_per_sm(int threads);

// ---- store / peel (cm_store.cu)
cudaError_t build_index(const int32_t* E, long long m, DevGraph g, uint32_t* ebkt, Ctl* c, cudaStream_t s);
cudaError_t count_degrees(const int32_t* E, const uint32_t* ebkt, long long m, DevGraph g, cudaStream_t s);
cudaError_t assign_offsets(DevGraph g, int32_t v0, int32_t v1, Ctl* c, cudaStream_t s);
cudaError_t scatter_edges(const int32_t* E, const uint32_t* ebkt, long long m, DevGraph g, cudaStream_t s);
cudaError_t set_cores(const int32_t* cores, DevGraph g, cudaStream_t s);
// core_scratch: n int32 of scratch (receives a compact copy of the cores)
cudaError_t init_mcd(DevGraph g, int32_t v0, int32_t v1, int32_t* core_scratch, cudaStream_t s);
cudaError_t launch_peel(const PeelParams& p, int blocks, int threads, cudaStream_t s);
int peel_blocks_per_sm(int threads);
cudaError_t rehash(const Bucket* old_idx, unsigned long long old_size, DevGraph g, Ctl* c, cudaStream_t s);
cudaError_t validate_vertices(const int64_t* nbr_off, const int32_t* nbrs, int32_t count, int32_t base, DevGraph g,
                              Ctl* c, cudaStream_t s);
cudaError_t init_vertices(const int64_t* nbr_off, int32_t count, int32_t base, DevGraph g, Ctl* c, cudaStream_t s);
cudaError_t expand_vertex_edges(const int64_t* nbr_off, const int32_t* nbrs, int32_t count, int32_t base, int32_t* E,
                                cudaStream_t s);
cudaError_t validate_ids(const int32_t* ids, int32_t count, DevGraph g, Ctl* c, cudaStream_t s);
cudaError_t gather_incident(const int32_t* ids, int32_t count, DevGraph g, int32_t* E, long long cap, Ctl* c,
                            cudaStream_t s);
cudaError_t mark_dead(const int32_t* ids, int32_t count, DevGraph g, cudaStream_t s);
cudaError_t pin_vertices(const int32_t* ids, int32_t count, DevGraph g, cudaStream_t s);
cudaError_t export_cores(DevGraph g, int32_t* out, cudaStream_t s);
cudaError_t export_sd(DevGraph g, int32_t* out, cudaStream_t s);
cudaError_t check_store(DevGraph g, unsigned long long* out, cudaStream_t s);
cudaError_t export_edges(DevGraph g, int32_t* out, Ctl* c, cudaStream_t s);
cudaError_t localize_multi(int32_t* E, long long k, const unsigned long long* kp, const long long* prefix,
                           const int32_t* bases, int32_t ng, cudaStream_t s);
cudaError_t validate_pairs(const int32_t* E, long long k, const unsigned long long* kp, int phase, DevGraph g, Ctl* c,
                           cudaStream_t s);
cudaError_t sum_caps(DevGraph g, int32_t v0, int32_t v1, Ctl* c, cudaStream_t s);
cudaError_t count_multi(const REdge* R, long long n, const unsigned long long* np, const int32_t* bases, int32_t ng,
                        unsigned long long* per_graph, cudaStream_t s);

}  // namespace cm
