// serve.cu -- a persistent request loop for part analyses (the interactive
// use the paper aims at): requests of different sizes arrive at any time,
// are admitted as execution slots and device memory free up, and run
// concurrently on the slots' streams, so their work overlaps on the GPU.
// Each part's BVH, sample points and visibility maps stay resident, keyed by
// the caller's part key; a re-submission with the same triangle list is
// refitted instead of rebuilt, and with cfg.incremental its points stay on
// their faces and only the rays the edit can change are cast again.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

rc_status check_params_public(const rc_params* p);

static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// 64-bit hash of a triangle list, eight bytes at a time (splitmix-style
// finaliser per word); used only to recognise an unchanged topology
static uint64_t hash_faces(const int32_t* a, int64_t n)
{
    uint64_t h = 0x9E3779B97F4A7C15ULL ^ (uint64_t)n;
    const int64_t words = n / 2;
    for (int64_t i = 0; i < words; ++i) {
        uint64_t w;
        memcpy(&w, a + 2 * i, 8);
        w ^= w >> 31;
        w *= 0xBF58476D1CE4E5B9ULL;
        h = (h ^ w) * 0x94D049BB133111EBULL;
        h ^= h >> 29;
    }
    if (n & 1) h = (h ^ (uint64_t)(uint32_t)a[n - 1]) * 0x94D049BB133111EBULL;
    return h;
}

// device bytes a part keeps resident (handle + per-point arrays) and the
// transient scratch of one analysis, from the allocations the calls make
static int64_t resident_bytes(int64_t nV, int64_t T, int64_t n, int32_t N)
{
    return 12 * nV + 260 * T + n * (12 + 12 + 4 + 4 + 1 + 24 + 1) + n * (int64_t)(N / 8) + 64;
}
static int64_t scratch_bytes(int64_t nV, int64_t T, int64_t n)
{
    return 12 * nV + 12 * T + 80 * T + 24 * n + (1 << 20);
}

struct SrvEntry {
    uint64_t key = 0;
    rc_bvh h = nullptr;
    int64_t nV = 0, T = 0, n = 0, cap_n = 0;
    int32_t N = 0;
    uint64_t fhash = 0;
    bool fhash_valid = false;      // false: fhash is computed after the result is delivered
    float* P = nullptr;
    float* Nn = nullptr;
    int32_t* face = nullptr;
    uint32_t* bits = nullptr;
    int32_t* count = nullptr;
    uint8_t* mask = nullptr;
    float* travel = nullptr;
    uint8_t* cls = nullptr;
    int64_t* ctr = nullptr;
    int64_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct SrvRequest {
    int64_t id = 0;
    uint64_t key = 0;
    std::vector<float> V;
    std::vector<int32_t> F;
    int64_t nV = 0, T = 0, n = 0;
    int64_t est = 0;
    int state = 0;   // 0 queued, 1 running, 2 done
    bool large = false;   // in the largest size class (admitted one at a time)
    rc_request_result res;
};

// per-part arrays are stream-ordered allocations; an entry is freed only when
// idle (its stream synchronised), so the legacy stream is a safe order
static void free_entry_arrays(SrvEntry* e)
{
    void* a[] = {e->P, e->Nn, e->face, e->bits, e->count, e->mask, e->travel, e->cls, e->ctr};
    for (void* p : a)
        if (p) cudaFreeAsync(p, 0);
    e->P = e->Nn = e->travel = nullptr;
    e->face = e->count = nullptr;
    e->bits = nullptr;
    e->mask = e->cls = nullptr;
    e->ctr = nullptr;
    e->cap_n = 0;
}

static void free_entry(SrvEntry* e)
{
    free_entry_arrays(e);
    if (e->h) rc_destroy_bvh(e->h);
    delete e;
}

}  // namespace rc

struct rc_server_s {
    rc_params p;
    rc_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<rc::SrvRequest*> queue;
    std::unordered_map<int64_t, rc::SrvRequest*> reqs;
    std::unordered_map<uint64_t, rc::SrvEntry*> cache;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;        // [slot * levels + level], level 0 = highest priority
    int levels = 1;
    int large_running = 0;                    // admitted requests of the largest size class
    int64_t used = 0;              // resident + reserved bytes
    int64_t next_id = 1;
    uint64_t tick = 0;
    bool stop = false;
    rc_server_stats st;
};

using namespace rc;

// Pick the first queued request that can run now (its part is not in use
// and its bytes fit, after evicting idle resident parts if needed).
// Called with the lock held.  Requests that can never fit fail at once.
// stream priority level of a request: 0 (highest) up to small_rays
// hemisphere rays, one level lower per doubling
static int level_of(rc_server s, const SrvRequest* r)
{
    int level = s->levels - 1;
    if (s->cfg.small_rays > 0) {
        level = 0;
        for (double lim = (double)s->cfg.small_rays; (double)r->n * s->p.n_dirs > lim && level < s->levels - 1;
             lim *= 2.0)
            ++level;
    }
    return level;
}

// Requests of the largest size class (the lowest priority level) are
// admitted one at a time, in arrival order: one of them fills the GPU alone,
// and two side by side would only take twice as long each.  Smaller requests
// are admitted beside them and run on higher-priority streams.
static bool is_large(rc_server s, const SrvRequest* r)
{
    return s->levels > 1 && s->cfg.small_rays > 0 && level_of(s, r) == s->levels - 1;
}

static SrvRequest* admit(rc_server s)
{
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        SrvRequest* r = *it;
        auto ce = s->cache.find(r->key);
        if (ce != s->cache.end() && ce->second->busy) continue;
        if (s->large_running > 0 && is_large(s, r)) continue;
        const int64_t have = ce != s->cache.end() ? ce->second->bytes : 0;
        const int64_t need = r->est - have;
        if (r->est > s->cfg.hbm_budget_bytes) {
            r->res.status = RC_E_OOM;
            snprintf(r->res.message, sizeof r->res.message, "request needs %lld bytes, budget is %lld",
                     (long long)r->est, (long long)s->cfg.hbm_budget_bytes);
            r->state = 2;
            r->res.t_end = now_s();
            s->st.rejected++;
            s->queue.erase(it);
            s->cv_done.notify_all();
            return admit(s);
        }
        while (s->used + need > s->cfg.hbm_budget_bytes) {
            SrvEntry* victim = nullptr;
            for (auto& kv : s->cache)
                if (!kv.second->busy && kv.first != r->key && (!victim || kv.second->last_use < victim->last_use))
                    victim = kv.second;
            if (!victim) break;
            s->used -= victim->bytes;
            s->cache.erase(victim->key);
            free_entry(victim);
            s->st.evicted++;
        }
        if (s->used + need > s->cfg.hbm_budget_bytes) continue;   // wait for memory
        SrvEntry* e;
        if (ce == s->cache.end()) {
            e = new SrvEntry();
            e->key = r->key;
            s->cache[r->key] = e;
        } else {
            e = ce->second;
        }
        e->busy = true;
        s->used += need;
        e->bytes = r->est;
        r->large = is_large(s, r);
        if (r->large) s->large_running++;
        r->state = 1;
        r->res.t_admit = now_s();
        s->queue.erase(it);
        return r;
    }
    return nullptr;
}

#define SRV_TRY(call)                                   \
    do {                                                \
        rc_status _r = (call);                          \
        if (_r != RC_OK) return _r;                     \
    } while (0)
#define SRV_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return cuda_error(_e, #call);            \
    } while (0)

static rc_status run_request(rc_server s, SrvRequest* r, SrvEntry* e, cudaStream_t st)
{
    rc_params p = s->p;
    if (s->cfg.cast_blocks_per_sm > 0) p.blocks_per_sm = s->cfg.cast_blocks_per_sm;
    const int32_t N = p.n_dirs;
    // the triangle-list hash decides refit vs rebuild; it is needed now only
    // when a resident part of the same size exists (otherwise the worker
    // computes it after delivering the result, before the part is released)
    const bool candidate = e->h && e->T == r->T && e->nV == r->nV;
    const uint64_t fh = candidate ? hash_faces(r->F.data(), r->T * 3) : 0;
    // the request's scratch (vertices, faces, changed-face flags) is freed
    // in stream order when this function returns, on every path
    struct Scratch {
        cudaStream_t st;
        void* p[3] = {nullptr, nullptr, nullptr};
        ~Scratch()
        {
            for (void* q : p)
                if (q) cudaFreeAsync(q, st);
        }
    } tmp{st};
    // geometry: refit when the triangle list is unchanged, else (re)build
    float* dV = nullptr;
    int32_t* dF = nullptr;
    SRV_CUDA(cudaMallocAsync(&dV, sizeof(float) * 3 * r->nV, st));
    tmp.p[0] = dV;
    SRV_CUDA(cudaMemcpyAsync(dV, r->V.data(), sizeof(float) * 3 * r->nV, cudaMemcpyHostToDevice, st));
    rc_status rs;
    const bool same_topology = candidate && e->fhash_valid && e->fhash == fh;
    // incremental re-analysis: same triangle list, point count and directions,
    // and the resident results of the previous request on this key
    const bool incremental = s->cfg.incremental && same_topology && e->P && e->n == r->n && e->N == N && r->n > 0;
    uint8_t* changed = nullptr;
    float box[6];
    int64_t n_changed = 0;
    if (incremental) {
        // compare with the resident vertices before the refit replaces them
        SRV_CUDA(cudaMallocAsync(&changed, (size_t)r->T, st));
        tmp.p[2] = changed;
        SRV_TRY(rc_changed_faces(e->h->V, dV, r->nV, e->h->F, r->T, changed, box, &n_changed, st));
    }
    if (same_topology) {
        rs = rc_refit_bvh(e->h, dV, st);
        r->res.rebuilt = 0;
    } else {
        if (e->h) rc_destroy_bvh(e->h);
        e->h = nullptr;
        SRV_CUDA(cudaMallocAsync(&dF, sizeof(int32_t) * 3 * r->T, st));
        tmp.p[1] = dF;
        SRV_CUDA(cudaMemcpyAsync(dF, r->F.data(), sizeof(int32_t) * 3 * r->T, cudaMemcpyHostToDevice, st));
        rs = rc_build_bvh(dV, r->nV, dF, r->T, st, &e->h);
        r->res.rebuilt = 1;
    }
    if (rs != RC_OK) return rs;
    e->T = r->T;
    e->nV = r->nV;
    e->fhash = fh;
    e->fhash_valid = candidate;
    // resident per-point arrays
    const int64_t n = r->n;
    if (n > e->cap_n || N != e->N) {
        free_entry_arrays(e);
        const int64_t c = n > 0 ? n : 1;
        SRV_CUDA(cudaMallocAsync(&e->P, sizeof(float) * 3 * c, st));
        SRV_CUDA(cudaMallocAsync(&e->Nn, sizeof(float) * 3 * c, st));
        SRV_CUDA(cudaMallocAsync(&e->face, sizeof(int32_t) * c, st));
        SRV_CUDA(cudaMallocAsync(&e->bits, sizeof(uint32_t) * ((N + 31) / 32) * c, st));
        SRV_CUDA(cudaMallocAsync(&e->count, sizeof(int32_t) * c, st));
        SRV_CUDA(cudaMallocAsync(&e->mask, c, st));
        SRV_CUDA(cudaMallocAsync(&e->travel, sizeof(float) * 6 * c, st));
        SRV_CUDA(cudaMallocAsync(&e->cls, c, st));
        SRV_CUDA(cudaMallocAsync(&e->ctr, sizeof(int64_t) * 8, st));
        e->cap_n = n;
        e->N = N;
    }
    e->n = n;
    rc_part_result& o = r->res.result;
    if (incremental) {
        rs = rc_sample_points_on_faces(e->h, n, &p, e->face, e->P, e->Nn, st);
        if (rs == RC_OK)
            rs = rc_hemisphere_update(e->h, e->P, e->Nn, e->face, n, changed, box, &p, e->bits, e->count, e->ctr,
                                      st);
        if (rs != RC_OK) return rs;
        r->res.updated = 1;
    } else {
        SRV_TRY(rc_sample_points(e->h, n, &p, e->P, e->Nn, e->face, nullptr, st));
        SRV_TRY(rc_hemisphere_cast(e->h, e->P, e->Nn, n, &p, e->bits, e->count, e->ctr, st));
    }
    SRV_TRY(rc_direction_variability(e->bits, e->Nn, nullptr, n, &p, nullptr, nullptr, nullptr, nullptr, &o.summary,
                                     st));
    SRV_TRY(rc_classify(&o.summary, &p, &o.label));
    SRV_CUDA(cudaMemcpyAsync(o.cast_counters, e->ctr, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, st));
    if (p.always_setups || o.label == 0) {
        SRV_TRY(rc_orthogonal_cast(e->h, e->P, e->Nn, n, &p, e->mask, e->travel, e->ctr + 4, st));
        SRV_CUDA(cudaMemcpyAsync(o.ortho_counters, e->ctr + 4, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, st));
        SRV_TRY(rc_min_setups(e->h, e->mask, e->travel, e->face, n, &p, e->cls, &o.setups, st));
        o.setups_ran = 1;
    }
    SRV_CUDA(cudaStreamSynchronize(st));
    r->res.resident_bytes = resident_bytes(r->nV, r->T, n, N);
    return RC_OK;
}

// The server's device is current for the scope of an API call made from
// the caller's thread, and the caller's device is restored afterwards.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

static void worker(rc_server s, int slot)
{
    cudaSetDevice(s->device);
    for (;;) {
        SrvRequest* r = nullptr;
        SrvEntry* e = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop) return;
                r = admit(s);
                if (r) break;
                s->cv_work.wait(lk);
            }
            e = s->cache[r->key];
            s->st.running++;
        }
        r->res.t_start = now_s();
        r->res.slot = slot;
        // smaller requests get higher stream priority
        const int level = level_of(s, r);
        cudaStream_t st = s->streams[slot * s->levels + level];
        r->res.priority_level = level;
        const rc_status rs = run_request(s, r, e, st);
        const double t_end = now_s();
        // a new part's triangle-list hash is computed after its result is
        // delivered; the part stays busy (not re-used or evicted) until then
        const bool hash_later = rs == RC_OK && !e->fhash_valid;
        std::vector<int32_t> faces;
        if (hash_later) faces = std::move(r->F);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            r->res.status = rs;
            if (rs != RC_OK) {
                snprintf(r->res.message, sizeof r->res.message, "%s", rc_last_error());
                s->st.failed++;
                // drop the part: its device state is unknown
                s->used -= e->bytes;
                s->cache.erase(e->key);
                for (int l = 0; l < s->levels; ++l) cudaStreamSynchronize(s->streams[slot * s->levels + l]);
                free_entry(e);
            } else {
                const int64_t actual = r->res.resident_bytes;
                s->used += actual - e->bytes;
                e->bytes = actual;
                if (!hash_later) {
                    e->busy = false;
                    e->last_use = ++s->tick;
                }
                s->st.completed++;
            }
            r->res.t_end = t_end;
            r->state = 2;
            if (r->large) s->large_running--;
            s->st.running--;
            s->cv_done.notify_all();
            s->cv_work.notify_all();
        }
        if (hash_later) {
            const uint64_t fh = hash_faces(faces.data(), (int64_t)faces.size());
            std::lock_guard<std::mutex> lk(s->mu);
            e->fhash = fh;
            e->fhash_valid = true;
            e->busy = false;
            e->last_use = ++s->tick;
            s->cv_work.notify_all();
            s->cv_done.notify_all();
        }
    }
}

extern "C" {

rc_status rc_server_create(const rc_params* p, const rc_server_config* cfg, rc_server* out)
{
    RC_RANGE();
    if (!out || !cfg) return set_error(RC_E_ARG, "NULL argument");
    *out = nullptr;
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (cfg->slots < 1 || cfg->slots > 64) return set_error(RC_E_ARG, "slots must be in [1, 64]");
    if (cfg->hbm_budget_bytes <= 0) return set_error(RC_E_ARG, "hbm_budget_bytes must be positive");
    if (cfg->incremental != 0 && cfg->incremental != 1) return set_error(RC_E_ARG, "incremental must be 0 or 1");
    rc_server s = new rc_server_s();
    s->p = *p;
    s->cfg = *cfg;
    memset(&s->st, 0, sizeof s->st);
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return set_error(RC_E_CUDA, "no CUDA device"); }
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    s->levels = prio_lo - prio_hi + 1;   // e.g. priorities 0 (lowest) .. -5 (highest)
    if (s->levels < 1) s->levels = 1;
    for (int k = 0; k < cfg->slots; ++k)
        for (int l = 0; l < s->levels; ++l) {
            cudaStream_t q = nullptr;
            if (cudaStreamCreateWithPriority(&q, cudaStreamNonBlocking, prio_hi + l) != cudaSuccess) {
                for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
                delete s;
                return set_error(RC_E_CUDA, "stream creation failed");
            }
            s->streams.push_back(q);
        }
    for (int k = 0; k < cfg->slots; ++k) s->workers.emplace_back(worker, s, k);
    *out = s;
    return RC_OK;
}

rc_status rc_server_submit(rc_server s, uint64_t part_key, const float* h_V, int64_t nV, const int32_t* h_F,
                           int64_t T, int64_t n, int64_t* req_id)
{
    RC_RANGE();
    if (!s || !h_V || !h_F || !req_id) return set_error(RC_E_ARG, "NULL argument");
    if (nV < 3 || T < 1 || n < 0) return set_error(RC_E_ARG, "empty mesh or negative n");
    if (s->p.sample_mode == RC_SAMPLE_FACE_CENTROID && n != T)
        return set_error(RC_E_ARG, "centroid sampling needs n == T");
    SrvRequest* r = new SrvRequest();
    r->key = part_key;
    r->V.assign(h_V, h_V + 3 * nV);
    r->F.assign(h_F, h_F + 3 * T);
    r->nV = nV;
    r->T = T;
    r->n = n;
    r->est = resident_bytes(nV, T, n, s->p.n_dirs) + scratch_bytes(nV, T, n);
    memset(&r->res, 0, sizeof r->res);
    r->res.t_submit = now_s();
    r->res.part_key = part_key;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->res.request_id = r->id;
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        s->st.submitted++;
    }
    s->cv_work.notify_all();
    *req_id = r->id;
    return RC_OK;
}

rc_status rc_server_wait(rc_server s, int64_t req_id, double timeout_s, rc_request_result* out)
{
    RC_RANGE();
    if (!s || !out) return set_error(RC_E_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return set_error(RC_E_ARG, "unknown request id");
    SrvRequest* r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->state != 2) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2)
            return set_error(RC_E_TIMEOUT, "request not finished within the timeout");
    }
    *out = r->res;
    s->reqs.erase(it);
    delete r;
    return RC_OK;
}

rc_status rc_server_read_bits(rc_server s, uint64_t part_key, uint32_t* h_bits, int64_t bits_words,
                              int32_t* h_count, int64_t n)
{
    RC_RANGE();
    if (!s) return set_error(RC_E_ARG, "server is NULL");
    if (n < 0 || bits_words < 0) return set_error(RC_E_ARG, "n and bits_words must be >= 0");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->cache.find(part_key);
    if (it == s->cache.end()) return set_error(RC_E_ARG, "part is not resident");
    // a part in use (being analysed, or finishing its bookkeeping) is read
    // once it is idle again; the wait is bounded
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(60);
    while (it->second->busy) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second->busy)
            return set_error(RC_E_TIMEOUT, "part stayed busy for 60 s");
        it = s->cache.find(part_key);
        if (it == s->cache.end()) return set_error(RC_E_ARG, "part is not resident");
    }
    SrvEntry* e = it->second;
    if (n != e->n) return set_error(RC_E_ARG, "n differs from the resident part's point count");
    const int64_t words = (int64_t)((e->N + 31) / 32) * n;
    if (h_bits && bits_words < words)
        return set_error(RC_E_ARG, "h_bits holds fewer than n * ceil(n_dirs / 32) words");
    // copy with the lock released; the part stays busy meanwhile, so it is
    // neither re-analysed nor evicted
    e->busy = true;
    lk.unlock();
    cudaError_t ce = cudaSuccess;
    {
        DeviceScope ds(s->device);
        if (h_bits && n) ce = cudaMemcpy(h_bits, e->bits, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess && h_count && n) ce = cudaMemcpy(h_count, e->count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    }
    lk.lock();
    e->busy = false;
    e->last_use = ++s->tick;
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (ce != cudaSuccess) return cuda_error(ce, "cudaMemcpy (resident bits)");
    return RC_OK;
}

rc_status rc_server_get_stats(rc_server s, rc_server_stats* out)
{
    RC_RANGE();
    if (!s || !out) return set_error(RC_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->queued = (int64_t)s->queue.size();
    out->resident_parts = (int64_t)s->cache.size();
    out->used_bytes = s->used;
    return RC_OK;
}

rc_status rc_server_destroy(rc_server s)
{
    RC_RANGE();
    if (!s) return RC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread& t : s->workers) t.join();
    DeviceScope ds(s->device);
    for (cudaStream_t q : s->streams) cudaStreamSynchronize(q);
    for (auto& kv : s->cache) free_entry(kv.second);
    for (auto& kv : s->reqs) delete kv.second;
    for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
    delete s;
    return RC_OK;
}

}  // extern "C"
