// batch.cu -- many parts, one launch: the batched hemispherical cast over a
// ray-work queue spanning all parts, replayed from a CUDA graph, and the
// autotuner that picks its launch knobs on the batch itself.  Parts added
// for analysis also get, in the same graph after the cast, the rest of the
// path of Sections 3.1-3.3: the directional reduction, the orthogonal cast
// and the reachability classes with their setup histogram; their part-level
// results come back in one copy (rc_batch_results).
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
rc_status device_dirs_canonical(int32_t N, const float4** canon);
int64_t ortho_scratch_words(int nf, int64_t n);
rc_status launch_orthogonal_frames_into(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                                        const FrameDev* fds, int nf, uint8_t* mask, float* travel,
                                        unsigned long long* counters, const int32_t* order, uint32_t* mbits,
                                        cudaStream_t s);
rc_status launch_classes(rc_bvh h, const uint8_t* mask, const float* travel, const int32_t* face, int64_t n,
                         const rc_params* p, uint8_t* cls, const double* frame_d, const double* fbox_d,
                         uint8_t* fixture, unsigned long long* hist, cudaStream_t s);

// Part-level results of an analysis part, one record per part in one
// device buffer: the reduction's sums (the first kVarWsumOffset + 16 bytes
// of its scratch), the 64 + 4 class histogram, orthogonal and cast counters.
constexpr size_t kRecSums = 0, kRecHist = 128, kRecOrtho = kRecHist + 68 * 8, kRecCast = kRecOrtho + 32;
constexpr size_t kRecBytes = (kRecCast + 32 + 255) / 256 * 256;

struct HostPart {
    rc_bvh h;
    const float* P;
    const float* N;
    int64_t n;
    uint32_t* bits;
    int32_t* count;
    int64_t* counters;
    int32_t* order = nullptr;      // owned, Morton order (computed when first needed)
    // analysis parts only
    const int32_t* face = nullptr; // caller's face ids of the points (null: cast only)
    int rec = -1;                  // index of the part's result record
    char* block = nullptr;         // owned: frame, reduction scratch, masks, travel, classes, fixture flags, scratch
    float4* ftree = nullptr;       // owned: frame-space tree (turned frames)
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
    int n_full = 0;                // analysis parts
    char* records = nullptr;       // owned: n_full result records (kRecBytes each)
    int records_cap = 0;
    // capture branches: the analysis parts' steps after the cast run on
    // kBranches streams forked from the capture stream (parallel graph paths)
    cudaStream_t branch[8] = {nullptr};
    cudaEvent_t fork_ev = nullptr, cast_ev = nullptr, join_ev[8] = {nullptr};
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

// layout of an analysis part's block (offsets rounded to 256 bytes)
struct FullLayout { size_t fd, var, mask, travel, cls, fixture, mbits, total; };
static FullLayout full_layout(int64_t n, int64_t T)
{
    FullLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    L.fd = take(sizeof(FrameDev));
    L.var = take(kVarScratchBytes);
    L.mask = take((size_t)n);
    L.travel = take(sizeof(float) * 6 * (size_t)n);
    L.cls = take((size_t)n);
    L.fixture = take((size_t)T);
    L.mbits = take(sizeof(uint32_t) * (size_t)ortho_scratch_words(1, n));
    L.total = off;
    return L;
}

// the device bytes of a part: its handle (vertices, faces, trees, face
// data), its caller-owned points, normals, bits and counts, and the batch's
// own point order
static int64_t base_bytes(rc_batch b, rc_bvh h, int64_t n)
{
    const int64_t W = (b->p.n_dirs + 31) / 32;
    return 12 * h->nV + 260 * h->T + n * (24 + 4 * W + 4 + 4) + 64;
}

static void release_part(HostPart& q)
{
    if (q.order) cudaFree(q.order);
    if (q.block) cudaFree(q.block);
    if (q.ftree) cudaFree(q.ftree);
    q.order = nullptr;
    q.block = nullptr;
    q.ftree = nullptr;
}

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
    // analysis parts: their buffers, frame trees (turned frames) and records
    if (b->n_full > b->records_cap) {
        if (b->records) cudaFree(b->records);
        b->records = nullptr;
        RC_CUDA(cudaMalloc(&b->records, kRecBytes * (size_t)b->n_full));
        b->records_cap = b->n_full;
    }
    for (int k = 0; k < np; ++k) {
        HostPart& q = b->parts[k];
        if (!q.face) continue;
        if (!q.block) RC_CUDA(cudaMalloc(&q.block, full_layout(q.n, q.h->T).total));
        if (q.ftree) { cudaFree(q.ftree); q.ftree = nullptr; }
        if (use_wide(&b->p) && !is_identity_frame(b->p.frame)) {
            const int64_t nodes = q.h->host_sc.wide_nodes > 0 ? q.h->host_sc.wide_nodes : q.h->n_int;
            RC_CUDA(cudaMalloc(&q.ftree, sizeof(float4) * 8 * nodes));
            rc_status fst = frame_tree(q.h, b->p.frame, q.ftree, s);
            if (fst != RC_OK) return fst;
        }
        // the cast's counters of an analysis part go to its record
        hp[k].counters = (unsigned long long*)(b->records + kRecBytes * q.rec + kRecCast);
    }
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
    const float4* canon = nullptr;
    if (b->n_full > 0 && (st = device_dirs_canonical(b->p.n_dirs, &canon)) != RC_OK) return st;
    RC_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaStream_t cs = b->cap_stream;
    cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long), cs);
    for (int k = 0; k < np; ++k)
        if (!b->parts[k].face && b->parts[k].counters) cudaMemsetAsync(b->parts[k].counters, 0, sizeof(int64_t) * 4, cs);
    if (b->n_full > 0) cudaMemsetAsync(b->records, 0, kRecBytes * (size_t)b->n_full, cs);
    // the rest of the path for the analysis parts: part k on branch k % 8.
    // The orthogonal cast and the classes need only the points, so the
    // branches fork before the cast and take the SMs as its blocks drain;
    // the reduction of each part waits for the cast
    const int nbr = b->n_full > 0 ? (b->n_full < 8 ? b->n_full : 8) : 0;
    rc_status lst = RC_OK;
    if (nbr > 0 && cudaEventRecord(b->fork_ev, cs) != cudaSuccess) lst = set_error(RC_E_CUDA, "fork");
    for (int j = 0; j < nbr && lst == RC_OK; ++j)
        if (cudaStreamWaitEvent(b->branch[j], b->fork_ev, 0) != cudaSuccess) lst = set_error(RC_E_CUDA, "fork");
    if (lst == RC_OK) lst = launch_batch(b->d_parts, np, b->n_items, ppi, tdirs, &b->p, b->d_work, cs);
    if (lst == RC_OK && nbr > 0 && cudaEventRecord(b->cast_ev, cs) != cudaSuccess) lst = set_error(RC_E_CUDA, "cast");
    for (int pass = 0; pass < 2 && lst == RC_OK; ++pass)
    for (int k = 0; k < np && lst == RC_OK; ++k) {
        HostPart& q = b->parts[k];
        if (!q.face || q.n == 0) continue;
        cudaStream_t cs = b->branch[q.rec % nbr];
        const FullLayout L = full_layout(q.n, q.h->T);
        FrameDev* fd = (FrameDev*)(q.block + L.fd);
        char* rec = b->records + kRecBytes * q.rec;
        if (pass == 1) {
            // after every orthogonal cast of this branch: wait for the cast once
            if (q.rec < nbr && cudaStreamWaitEvent(cs, b->cast_ev, 0) != cudaSuccess) {
                lst = set_error(RC_E_CUDA, "cast wait");
                break;
            }
            lst = launch_variability(q.bits, q.N, nullptr, q.n, canon, &b->p, nullptr, nullptr, nullptr, nullptr,
                                     q.block + L.var, cs);
            if (lst != RC_OK) break;
            if (cudaMemcpyAsync(rec + kRecSums, q.block + L.var, kVarWsumOffset + 16, cudaMemcpyDeviceToDevice, cs) !=
                cudaSuccess) { lst = set_error(RC_E_CUDA, "record copy"); break; }
            continue;
        }
        if ((lst = frame_setup(q.h, &b->p, fd, cs, q.ftree)) != RC_OK) break;
        lst = launch_orthogonal_frames_into(q.h, q.P, q.N, q.n, &b->p, fd, 1, (uint8_t*)(q.block + L.mask),
                                            (float*)(q.block + L.travel), (unsigned long long*)(rec + kRecOrtho),
                                            b->p.point_order == 0 ? q.order : nullptr,
                                            (uint32_t*)(q.block + L.mbits), cs);
        if (lst != RC_OK) break;
        lst = launch_classes(q.h, (const uint8_t*)(q.block + L.mask), (const float*)(q.block + L.travel), q.face,
                             q.n, &b->p, (uint8_t*)(q.block + L.cls), fd->frame, fd->fbox,
                             (uint8_t*)(q.block + L.fixture), (unsigned long long*)(rec + kRecHist), cs);
    }
    for (int j = 0; j < nbr && lst == RC_OK; ++j)
        if (cudaEventRecord(b->join_ev[j], b->branch[j]) != cudaSuccess ||
            cudaStreamWaitEvent(cs, b->join_ev[j], 0) != cudaSuccess)
            lst = set_error(RC_E_CUDA, "join");
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
        cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->cast_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b->d_work, sizeof(unsigned long long)) != cudaSuccess) {
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        if (b->done) cudaEventDestroy(b->done);
        if (b->fork_ev) cudaEventDestroy(b->fork_ev);
        if (b->cast_ev) cudaEventDestroy(b->cast_ev);
        delete b;
        return set_error(RC_E_CUDA, "batch set-up failed");
    }
    for (int j = 0; j < 8; ++j)
        if (cudaStreamCreateWithFlags(&b->branch[j], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[j], cudaEventDisableTiming) != cudaSuccess) {
            rc_batch_destroy(b);
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
    const int64_t bytes = base_bytes(b, h, n);
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

rc_status rc_batch_add_analysis(rc_batch b, rc_bvh h, const float* d_P, const float* d_N, const int32_t* d_face,
                                int64_t n, uint32_t* d_bits, int32_t* d_count, int64_t* part_id)
{
    RC_RANGE();
    if (!d_face && n > 0) return set_error(RC_E_ARG, "face ids are NULL");
    if (b && h && n >= 0) {
        // the batch's own buffers of the part count against the budget too
        const int64_t all = base_bytes(b, h, n) + (int64_t)full_layout(n, h->T).total + (int64_t)kRecBytes;
        if (b->budget > 0 && b->used + all > b->budget)
            return set_error(RC_E_OOM, "the part does not fit into the batch's HBM budget");
    }
    int64_t id = -1;
    rc_status st = rc_batch_add_part(b, h, d_P, d_N, n, d_bits, d_count, nullptr, &id);
    if (st != RC_OK) return st;
    HostPart& q = b->parts.back();
    q.face = d_face;
    q.rec = b->n_full++;
    const int64_t extra = (int64_t)full_layout(n, h->T).total + (int64_t)kRecBytes;
    b->part_bytes.back() += extra;
    b->used += extra;
    if (part_id) *part_id = id;
    return RC_OK;
}

rc_status rc_batch_results(rc_batch b, rc_part_result* h_out, int64_t n_out)
{
    RC_RANGE();
    if (!b || (!h_out && n_out > 0)) return set_error(RC_E_ARG, "batch or results is NULL");
    if (n_out < 0 || n_out > (int64_t)b->parts.size()) return set_error(RC_E_ARG, "n_out outside [0, parts]");
    if (!b->launched) return set_error(RC_E_ARG, "the batch has not been launched");
    if (b->dirty) return set_error(RC_E_ARG, "parts or parameters changed since the last launch");
    RC_CUDA(cudaEventSynchronize(b->done));
    std::vector<char> rec(kRecBytes * (size_t)b->n_full);
    if (b->n_full > 0) RC_CUDA(cudaMemcpy(rec.data(), b->records, rec.size(), cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < n_out; ++k) {
        rc_part_result& o = h_out[k];
        memset(&o, 0, sizeof o);
        const HostPart& q = b->parts[k];
        if (!q.face) continue;
        const char* r = rec.data() + kRecBytes * q.rec;
        long long sums[kVarSums];
        double wsum[2];
        memcpy(sums, r + kRecSums, sizeof sums);
        memcpy(wsum, r + kRecSums + kVarWsumOffset, sizeof wsum);
        fill_summary(sums, wsum, q.n, b->p.n_dirs, false, &o.summary);
        rc_status st = rc_classify(&o.summary, &b->p, &o.label);
        if (st != RC_OK) return st;
        unsigned long long hist[68];
        memcpy(hist, r + kRecHist, sizeof hist);
        for (int m = 0; m < 64; ++m) o.setups.mask_hist[m] = (int64_t)hist[m];
        for (int c = 0; c < 4; ++c) o.setups.class_counts[c] = (int64_t)hist[64 + c];
        if ((st = rc_setup_cover(o.setups.mask_hist, &o.setups)) != RC_OK) return st;
        o.setups_ran = 1;
        memcpy(o.ortho_counters, r + kRecOrtho, sizeof o.ortho_counters);
        memcpy(o.cast_counters, r + kRecCast, sizeof o.cast_counters);
    }
    return RC_OK;
}

rc_status rc_batch_clear(rc_batch b)
{
    RC_RANGE();
    if (!b) return set_error(RC_E_ARG, "batch is NULL");
    for (HostPart& q : b->parts) release_part(q);
    b->parts.clear();
    b->n_full = 0;
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
    // the timing events are destroyed, and on a failure the batch's own
    // parameters restored, on every path out
    struct Tune {
        rc_batch b;
        rc_params base;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = false;
        ~Tune()
        {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (!ok) {
                b->p = base;
                b->dirty = true;
            }
        }
    } tune{b, base};
    RC_CUDA(cudaEventCreate(&tune.e0));
    RC_CUDA(cudaEventCreate(&tune.e1));
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
                    if (st != RC_OK) return st;
                    RC_CUDA(cudaEventRecord(tune.e0, s));
                    for (int r = 0; r < repeats; ++r) RC_CUDA(cudaGraphLaunch(b->exec, s));
                    RC_CUDA(cudaEventRecord(tune.e1, s));
                    RC_CUDA(cudaEventSynchronize(tune.e1));
                    float ms = 0.0f;
                    RC_CUDA(cudaEventElapsedTime(&ms, tune.e0, tune.e1));
                    if (best_ms < 0.0f || ms < best_ms) { best_ms = ms; win = c; }
                }
    tune.ok = true;
    b->p = win;
    b->dirty = true;
    if (best) *best = win;
    return RC_OK;
}

rc_status rc_batch_destroy(rc_batch b)
{
    RC_RANGE();
    if (!b) return RC_OK;
    for (HostPart& q : b->parts) release_part(q);
    drop_graph(b);
    if (b->records) cudaFree(b->records);
    if (b->d_parts) cudaFree(b->d_parts);
    if (b->d_work) cudaFree(b->d_work);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->done) cudaEventDestroy(b->done);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->cast_ev) cudaEventDestroy(b->cast_ev);
    for (int j = 0; j < 8; ++j) {
        if (b->branch[j]) cudaStreamDestroy(b->branch[j]);
        if (b->join_ev[j]) cudaEventDestroy(b->join_ev[j]);
    }
    delete b;
    return RC_OK;
}

}  // extern "C"
