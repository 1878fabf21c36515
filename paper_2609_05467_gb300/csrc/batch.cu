// batch.cu -- many parts, one launch: the batched hemispherical cast over a
// ray-work queue spanning all parts, replayed from a CUDA graph, and the
// autotuner that picks its launch knobs on the batch itself.
#include <string.h>

#include <vector>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

rc_status point_order(rc_bvh h, const float* P, int64_t n, int32_t* order, cudaStream_t s);
rc_status launch_batch(const BatchPart* d_parts, int n_parts, long long n_items, int ppi, const float4* tdirs,
                       const rc_params* p, unsigned long long* work, cudaStream_t s);
rc_status prepare_batch_kernel(int n_dirs);
rc_status device_dirs_for_cast(const rc_params* p, const float4** tdirs);
rc_status check_params_public(const rc_params* p);
bool use_wide(const rc_params* p);

struct HostPart {
    rc_bvh h;
    const float* P;
    const float* N;
    int64_t n;
    uint32_t* bits;
    int32_t* count;
    int64_t* counters;
    int32_t* order = nullptr;      // owned, Morton order (computed when first needed)
};

}  // namespace rc

struct rc_batch_s {
    rc_params p;
    int device = 0;
    int64_t budget = 0;            // admission budget in device bytes (0 = none)
    int64_t used = 0;              // device bytes of the parts admitted so far
    std::vector<rc::HostPart> parts;
    std::vector<int64_t> part_bytes;
    cudaEvent_t done = nullptr;    // recorded after the last launch's work
    bool launched = false;
    rc::BatchPart* d_parts = nullptr;
    unsigned long long* d_work = nullptr;
    int cap = 0;
    long long n_items = 0;
    bool dirty = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

using namespace rc;

static void drop_graph(rc_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Upload the part descriptors for the current knobs and capture the launch
// (work-counter reset, per-part counter resets, batched kernel) as a graph.
static rc_status prepare(rc_batch b, cudaStream_t s)
{
    drop_graph(b);
    const int np = (int)b->parts.size();
    if (np == 0) return RC_OK;
    const int ppi = b->p.points_per_item > 0 ? b->p.points_per_item : 1;
    std::vector<BatchPart> hp(np);
    long long first = 0;
    for (int k = 0; k < np; ++k) {
        HostPart& q = b->parts[k];
        if (b->p.point_order == 0 && !q.order && q.n > 1) {
            RC_CUDA(cudaMalloc(&q.order, sizeof(int32_t) * q.n));
            rc_status st = point_order(q.h, q.P, q.n, q.order, s);
            if (st != RC_OK) return st;
        }
        BatchPart& d = hp[k];
        d.nodes = use_wide(&b->p) ? q.h->wnodes : q.h->nodes;
        d.tris = q.h->tris;
        d.P = q.P;
        d.N = q.N;
        d.order = b->p.point_order == 0 ? q.order : nullptr;
        d.bits = q.bits;
        d.count = q.count;
        d.counters = (unsigned long long*)q.counters;
        d.n = q.n;
        d.first_item = first;
        d.max_steps = (int)(2 * (q.h->n_int + q.h->T) + 64);
        d.scene_maxabs = q.h->scene_maxabs;
        first += (q.n + ppi - 1) / ppi;
    }
    b->n_items = first;
    if (np > b->cap) {
        if (b->d_parts) cudaFree(b->d_parts);
        b->d_parts = nullptr;
        RC_CUDA(cudaMalloc(&b->d_parts, sizeof(BatchPart) * np));
        b->cap = np;
    }
    RC_CUDA(cudaMemcpyAsync(b->d_parts, hp.data(), sizeof(BatchPart) * np, cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaStreamSynchronize(s));
    const float4* tdirs = nullptr;
    rc_status st = device_dirs_for_cast(&b->p, &tdirs);
    if (st != RC_OK) return st;
    st = prepare_batch_kernel(b->p.n_dirs);
    if (st != RC_OK) return st;
    // capture on the batch's private stream; nothing runs during capture
    RC_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long), b->cap_stream);
    for (int k = 0; k < np; ++k)
        if (b->parts[k].counters) cudaMemsetAsync(b->parts[k].counters, 0, sizeof(int64_t) * 4, b->cap_stream);
    rc_status lst = launch_batch(b->d_parts, np, b->n_items, ppi, tdirs, &b->p, b->d_work, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (lst != RC_OK) { if (g) cudaGraphDestroy(g); return lst; }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    b->graph = g;
    RC_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->dirty = false;
    return RC_OK;
}

extern "C" {

rc_status rc_batch_create(const rc_params* p, int64_t hbm_budget_bytes, rc_batch* out)
{
    RC_RANGE();
    if (!out) return set_error(RC_E_ARG, "out is NULL");
    *out = nullptr;
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (hbm_budget_bytes < 0) return set_error(RC_E_ARG, "hbm_budget_bytes must be >= 0");
    rc_batch b = new rc_batch_s();
    b->p = *p;
    b->budget = hbm_budget_bytes;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b->d_work, sizeof(unsigned long long)) != cudaSuccess) {
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        if (b->done) cudaEventDestroy(b->done);
        delete b;
        return set_error(RC_E_CUDA, "batch set-up failed");
    }
    *out = b;
    return RC_OK;
}

rc_status rc_batch_add_part(rc_batch b, rc_bvh h, const float* d_P, const float* d_N, int64_t n, uint32_t* d_bits,
                            int32_t* d_count, int64_t* d_counters, int64_t* part_id)
{
    RC_RANGE();
    if (!b || !h) return set_error(RC_E_ARG, "batch or handle is NULL");
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n > 0 && (!d_P || !d_N || !d_bits || !d_count)) return set_error(RC_E_ARG, "array pointer is NULL");
    if (h->device != b->device) return set_error(RC_E_ARG, "handle and batch are on different devices");
    // the part's device bytes: its handle (vertices, faces, trees, face
    // data), its caller-owned points, normals, bits and counts, and the
    // batch's own point order
    const int64_t W = (b->p.n_dirs + 31) / 32;
    const int64_t bytes = 12 * h->nV + 260 * h->T + n * (24 + 4 * W + 4 + 4) + 64;
    if (b->budget > 0 && b->used + bytes > b->budget)
        return set_error(RC_E_OOM, "the part does not fit into the batch's HBM budget");
    HostPart q;
    q.h = h;
    q.P = d_P;
    q.N = d_N;
    q.n = n;
    q.bits = d_bits;
    q.count = d_count;
    q.counters = d_counters;
    b->parts.push_back(q);
    b->part_bytes.push_back(bytes);
    b->used += bytes;
    b->dirty = true;
    if (part_id) *part_id = (int64_t)b->parts.size() - 1;
    return RC_OK;
}

rc_status rc_batch_clear(rc_batch b)
{
    RC_RANGE();
    if (!b) return set_error(RC_E_ARG, "batch is NULL");
    for (HostPart& q : b->parts)
        if (q.order) cudaFree(q.order);
    b->parts.clear();
    b->part_bytes.clear();
    b->used = 0;
    b->launched = false;
    drop_graph(b);
    b->dirty = true;
    return RC_OK;
}

rc_status rc_batch_set_params(rc_batch b, const rc_params* p)
{
    RC_RANGE();
    if (!b) return set_error(RC_E_ARG, "batch is NULL");
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    b->p = *p;
    b->dirty = true;
    return RC_OK;
}

rc_status rc_batch_launch(rc_batch b, void* stream)
{
    RC_RANGE();
    if (!b) return set_error(RC_E_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->dirty) {
        rc_status st = prepare(b, s);
        if (st != RC_OK) return st;
    }
    if (!b->exec) return RC_OK;   // no parts
    RC_CUDA(cudaGraphLaunch(b->exec, s));
    count_launch();
    RC_CUDA(cudaEventRecord(b->done, s));
    b->launched = true;
    return RC_OK;
}

rc_status rc_batch_poll(rc_batch b, int64_t part_id, int32_t* done)
{
    RC_RANGE();
    if (!b || !done) return set_error(RC_E_ARG, "batch or done is NULL");
    if (part_id < 0 || part_id >= (int64_t)b->parts.size()) return set_error(RC_E_ARG, "part_id out of range");
    *done = 0;
    if (!b->launched) return RC_OK;
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaErrorNotReady) return RC_OK;
    if (e != cudaSuccess) return cuda_error(e, "cudaEventQuery");
    *done = 1;
    return RC_OK;
}

rc_status rc_batch_autotune(rc_batch b, void* stream, int32_t repeats, rc_params* best)
{
    RC_RANGE();
    if (!b) return set_error(RC_E_ARG, "batch is NULL");
    if (repeats < 1) repeats = 1;
    cudaStream_t s = (cudaStream_t)stream;
    const rc_params base = b->p;
    rc_params win = base;
    float best_ms = -1.0f;
    cudaEvent_t e0, e1;
    RC_CUDA(cudaEventCreate(&e0));
    RC_CUDA(cudaEventCreate(&e1));
    const int per_sm[] = {4, 6, 8};
    const int ppis[] = {1, 2, 4};
    for (int order = 0; order < 2; ++order)
        for (int tile = 0; tile < 2; ++tile)
            for (int a : per_sm)
                for (int q : ppis) {
                    rc_params c = base;
                    c.point_order = order;
                    c.tile_mode = tile;
                    c.blocks_per_sm = a;
                    c.points_per_item = q;
                    b->p = c;
                    b->dirty = true;
                    rc_status st = rc_batch_launch(b, stream);   // capture + warm-up
                    if (st != RC_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); b->p = base; return st; }
                    RC_CUDA(cudaEventRecord(e0, s));
                    for (int r = 0; r < repeats; ++r) RC_CUDA(cudaGraphLaunch(b->exec, s));
                    RC_CUDA(cudaEventRecord(e1, s));
                    RC_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.0f;
                    RC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (best_ms < 0.0f || ms < best_ms) { best_ms = ms; win = c; }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->p = win;
    b->dirty = true;
    if (best) *best = win;
    return RC_OK;
}

rc_status rc_batch_destroy(rc_batch b)
{
    RC_RANGE();
    if (!b) return RC_OK;
    for (HostPart& q : b->parts)
        if (q.order) cudaFree(q.order);
    drop_graph(b);
    if (b->d_parts) cudaFree(b->d_parts);
    if (b->d_work) cudaFree(b->d_work);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
    return RC_OK;
}

}  // extern "C"
