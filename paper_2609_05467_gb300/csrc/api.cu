// api.cu -- the C ABI of include/rc.h: argument validation, handle
// management, the host-side direction table, classification and the setup
// cover.  Every per-face, per-point and per-ray step runs in the kernels of
// build.cu, cast.cu and reduce.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

rc_status build_bvh(rc_bvh h, cudaStream_t s);
rc_status refit_bvh(rc_bvh h, cudaStream_t s);
rc_status sample_points(rc_bvh h, int64_t n, const rc_params* p, float* P, float* N, int32_t* face,
                        double* weight, cudaStream_t s);
rc_status launch_hemisphere(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                            uint32_t* bits, int32_t* count, unsigned long long* counters, bool stats,
                            cudaStream_t s, long long* relist = nullptr, long long relist_cap = 0);
rc_status launch_orthogonal(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                            uint8_t* mask, float* travel, unsigned long long* counters, cudaStream_t s);
rc_status launch_classes(rc_bvh h, const uint8_t* mask, const float* travel, const int32_t* face, int64_t n,
                         const rc_params* p, uint8_t* cls, const double* frame_d, const double* fbox_d,
                         uint8_t* fixture, unsigned long long* hist, cudaStream_t s);

// ---------------------------------------------------------------------------
// errors and counters
// ---------------------------------------------------------------------------
static thread_local std::string t_err;
static std::atomic<long long> g_launches{0};

rc_status set_error(rc_status st, const std::string& msg)
{
    t_err = msg;
    return st;
}

rc_status cuda_error(cudaError_t e, const char* what)
{
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RC_E_OOM : RC_E_CUDA;
}

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// direction table (Section 3.1, Fig. 1): Fibonacci hemisphere in FP64 on the
// host, rounded to fp32; cached on each device per N.
// ---------------------------------------------------------------------------
static void fibonacci_hemisphere(int32_t N, float* out /*N x 3*/)
{
    const double golden_angle = M_PI * (3.0 - sqrt(5.0));
    for (int32_t j = 0; j < N; ++j) {
        const double z = 1.0 - ((double)j + 0.5) / (double)N;
        const double rad = sqrt(1.0 - z * z);
        const double phi = (double)j * golden_angle;
        out[3 * j + 0] = (float)(rad * cos(phi));
        out[3 * j + 1] = (float)(rad * sin(phi));
        out[3 * j + 2] = (float)z;
    }
}

// Tile order for the cast.  The direction set's z is uniform in its index,
// so runs of consecutive indices are elevation bands.  Each band holds a
// whole number m of tiles of 32 directions sorted by azimuth, so that every
// tile is an azimuth sector of one band.  A band of 32 m directions at polar
// angle theta spans dz = 32 m / N, that is d(theta) = dz / sin(theta) of
// elevation, and each of its sectors an arc of 2 pi sin(theta) / m;
// m = sin(theta) sqrt(2 pi N / (32 kTileAspect)) makes the arc kTileAspect
// times the elevation span.  Walk lengths change fastest with elevation (the
// grazing rays near the horizon walk longest), so tiles narrow in elevation
// keep a tile's walks alike.  Consecutive bands sweep the azimuth in
// alternate directions, so consecutive tiles are neighbours; the last
// N mod 32 directions form the partial tile.  Returns the canonical index
// per slot.
static std::vector<int32_t> tile_order(int32_t N, const float* h)
{
    constexpr double kTileAspect = 3.0;
    std::vector<int32_t> ord;
    ord.reserve(N);
    std::vector<std::pair<double, int32_t>> key;
    const int32_t ntiles = N / 32;
    int32_t j = 0, t = 0, band = 0;
    while (t < ntiles) {
        const double z = 1.0 - ((double)j + 0.5) / (double)N;
        const double s = sqrt(std::max(0.0, 1.0 - z * z));
        int32_t m = (int32_t)llround(s * sqrt(2.0 * M_PI * (double)N / (32.0 * kTileAspect)));
        m = std::max(1, std::min(m, ntiles - t));
        key.clear();
        for (int32_t k = j; k < j + 32 * m; ++k) {
            const double phi = atan2((double)h[3 * k + 1], (double)h[3 * k]);
            key.push_back({(band & 1) ? -phi : phi, k});
        }
        std::sort(key.begin(), key.end());
        for (const auto& e : key) ord.push_back(e.second);
        j += 32 * m;
        t += m;
        ++band;
    }
    for (int32_t k = j; k < N; ++k) ord.push_back(k);
    return ord;
}

struct DirTables { float4* canon; float4* tiled; };
static std::mutex g_dir_mu;
static std::map<std::pair<int, int>, DirTables> g_dirs;

static rc_status device_dirs(int32_t N, const float4** canon, const float4** tiled = nullptr)
{
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dir_mu);
    auto it = g_dirs.find({dev, N});
    if (it == g_dirs.end()) {
        // both tables hold 32 * ceil(N / 32) entries; the entries past N
        // pad the last tile: canonical index -1 and the direction of entry
        // 0 (a real direction, so a cast may trace them and discard them)
        const int32_t N32 = (N + 31) / 32 * 32;
        std::vector<float> h(3 * (size_t)N);
        fibonacci_hemisphere(N, h.data());
        const std::vector<int32_t> ord = tile_order(N, h.data());
        float pad_w;
        const int32_t minus1 = -1;
        memcpy(&pad_w, &minus1, sizeof pad_w);
        std::vector<float4> h4(2 * (size_t)N32, make_float4(h[0], h[1], h[2], pad_w));
        for (int32_t j = 0; j < N; ++j) {
            float w;
            memcpy(&w, &j, sizeof w);
            h4[j] = make_float4(h[3 * j], h[3 * j + 1], h[3 * j + 2], w);
        }
        for (int32_t k = 0; k < N; ++k) {
            const int32_t j = ord[k];
            float w;
            memcpy(&w, &j, sizeof w);
            h4[N32 + k] = make_float4(h[3 * j], h[3 * j + 1], h[3 * j + 2], w);
        }
        float4* d = nullptr;
        RC_CUDA(cudaMalloc(&d, sizeof(float4) * 2 * N32));
        RC_CUDA(cudaMemcpy(d, h4.data(), sizeof(float4) * 2 * N32, cudaMemcpyHostToDevice));
        it = g_dirs.emplace(std::make_pair(dev, N), DirTables{d, d + N32}).first;
    }
    *canon = it->second.canon;
    if (tiled) *tiled = it->second.tiled;
    return RC_OK;
}

// The classification thresholds (Section 3.3): any value but NaN, which no
// comparison would decide.
static rc_status check_thresholds(const rc_params* p)
{
    if (std::isnan(p->t_acc) || std::isnan(p->t_share) || std::isnan(p->t_conc))
        return set_error(RC_E_ARG, "t_acc, t_share and t_conc must not be NaN");
    return RC_OK;
}

static rc_status check_params(const rc_params* p)
{
    if (!p) return set_error(RC_E_ARG, "params is NULL");
    if (p->n_dirs < 1 || p->n_dirs > kMaxDirs) return set_error(RC_E_ARG, "n_dirs must be in [1, 65536]");
    if (!(p->origin_offset >= 0.0) || !isfinite(p->origin_offset))
        return set_error(RC_E_ARG, "origin_offset must be finite and >= 0");
    if (p->sample_mode != RC_SAMPLE_AREA_RANDOM && p->sample_mode != RC_SAMPLE_FACE_CENTROID)
        return set_error(RC_E_ARG, "unknown sample_mode");
    if (p->conc_mode != 0 && p->conc_mode != 1) return set_error(RC_E_ARG, "conc_mode must be 0 or 1");
    for (int k = 0; k < 9; ++k)
        if (!isfinite(p->frame[k])) return set_error(RC_E_ARG, "frame must be finite");
    for (int c = 0; c < 3; ++c)
        if (p->frame[c] == 0.0f && p->frame[3 + c] == 0.0f && p->frame[6 + c] == 0.0f)
            return set_error(RC_E_ARG, "frame columns (the machining axes) must be non-zero");
    if (p->block_threads != 0 && p->block_threads != 128)
        return set_error(RC_E_UNSUPPORTED, "block_threads must be 0 (default) or 128");
    if (p->point_order != 0 && p->point_order != 1) return set_error(RC_E_ARG, "point_order must be 0 or 1");
    if (p->tile_mode != 0 && p->tile_mode != 1) return set_error(RC_E_ARG, "tile_mode must be 0 or 1");
    if (p->points_per_item < 0 || p->points_per_item > 64)
        return set_error(RC_E_ARG, "points_per_item must be in [0, 64]");
    if (p->launch_mode != 0 && p->launch_mode != 1) return set_error(RC_E_ARG, "launch_mode must be 0 or 1");
    if (p->fetch_mode != 0) return set_error(RC_E_ARG, "fetch_mode must be 0 (reserved)");
    if (p->tree_width != 0 && p->tree_width != 2 && p->tree_width != 4)
        return set_error(RC_E_ARG, "tree_width must be 0 (default), 2 or 4");
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 64) return set_error(RC_E_ARG, "blocks_per_sm out of range");
    if (p->collect_stats != 0 && p->collect_stats != 1) return set_error(RC_E_ARG, "collect_stats must be 0 or 1");
    if (!(p->parallel_tol >= 0.0 && p->parallel_tol <= 0.5))
        return set_error(RC_E_ARG, "parallel_tol must be in [0, 0.5]");
    if (p->always_setups != 0 && p->always_setups != 1) return set_error(RC_E_ARG, "always_setups must be 0 or 1");
    if (!(p->tool_length >= 0.0f)) return set_error(RC_E_ARG, "tool_length must be >= 0 (+inf: no limit)");
    return check_thresholds(p);
}

rc_status check_params_public(const rc_params* p) { return check_params(p); }

// Direction table a cast uses: tile order (default) or canonical order.
rc_status device_dirs_canonical(int32_t N, const float4** canon) { return device_dirs(N, canon); }

rc_status device_dirs_for_cast(const rc_params* p, const float4** tdirs)
{
    const float4 *canon = nullptr, *tiled = nullptr;
    rc_status st = device_dirs(p->n_dirs, &canon, &tiled);
    if (st != RC_OK) return st;
    *tdirs = p->tile_mode == 1 ? canon : tiled;
    return RC_OK;
}

// Scene bounds = the union of the binary root's two child boxes (every
// referenced vertex); read after every build and refit.
static rc_status scene_box(rc_bvh h)
{
    float4 root[3];
    if (cudaMemcpy(root, h->nodes, sizeof root, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(RC_E_CUDA, "reading the root node failed");
    h->lo[0] = fminf(root[0].x, root[1].x); h->hi[0] = fmaxf(root[0].y, root[1].y);
    h->lo[1] = fminf(root[0].z, root[1].z); h->hi[1] = fmaxf(root[0].w, root[1].w);
    h->lo[2] = fminf(root[2].x, root[2].z); h->hi[2] = fmaxf(root[2].y, root[2].w);
    return RC_OK;
}

// device scratch freed in stream order when the scope ends, on every path
struct ApiScratch {
    cudaStream_t s;
    void* p[3] = {nullptr, nullptr, nullptr};
    ~ApiScratch()
    {
        for (void* q : p)
            if (q) cudaFreeAsync(q, s);
    }
};

static rc_status use_device_of(rc_bvh h)
{
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) RC_CUDA(cudaSetDevice(h->device));
    return RC_OK;
}

// Handle memory comes from the stream-ordered pool: it is returned with
// cudaFreeAsync on the legacy default stream, which does not stall other
// streams' work (cudaFree would synchronise the whole device).
static void free_handle(rc_bvh h)
{
    if (!h) return;
    void* ptrs[] = {h->V, h->F, h->tris, h->nodes, h->wnodes, h->parent, h->child, h->range, h->order, h->nbox,
                    h->visits, h->fnorm, h->farea, h->cdf, h->sc};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, 0);
    delete h;
}

// Keep freed pool memory for reuse instead of returning it to the driver at
// every synchronisation (once per device; a process-local setting).
void keep_pool_memory()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}

}  // namespace rc

using namespace rc;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

rc_status rc_params_default(rc_params* p)
{
    if (!p) return set_error(RC_E_ARG, "params is NULL");
    memset(p, 0, sizeof *p);
    p->n_dirs = 256;
    p->sample_mode = RC_SAMPLE_AREA_RANDOM;
    p->origin_offset = 1e-4;
    p->seed = 0;
    for (int k = 0; k < 9; ++k) p->frame[k] = (k % 4 == 0) ? 1.0f : 0.0f;
    p->tool_length = 100.0f;
    p->conc_mode = 0;
    p->t_acc = 0.60;
    p->t_share = 0.45;
    p->t_conc = 0.41;
    p->parallel_tol = 1e-4;
    return RC_OK;
}

const char* rc_last_error(void) { return t_err.c_str(); }

int64_t rc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

rc_status rc_stream_status(void* stream)
{
    RC_RANGE();
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "work queued on the stream");
    return RC_OK;
}

rc_status rc_build_bvh(const float* d_V, int64_t nV, const int32_t* d_F, int64_t T, void* stream, rc_bvh* out)
{
    RC_RANGE();
    return rc_build_bvh_ex(d_V, nV, d_F, T, RC_BUILDER_KARRAS, stream, out);
}

rc_status rc_build_bvh_ex(const float* d_V, int64_t nV, const int32_t* d_F, int64_t T, int32_t builder, void* stream,
                          rc_bvh* out)
{
    RC_RANGE();
    if (!out) return set_error(RC_E_ARG, "out is NULL");
    if (builder != RC_BUILDER_KARRAS && builder != RC_BUILDER_PLOC)
        return set_error(RC_E_ARG, "builder must be RC_BUILDER_KARRAS or RC_BUILDER_PLOC");
    *out = nullptr;
    if (!d_V || !d_F) return set_error(RC_E_ARG, "vertex or face pointer is NULL");
    if (nV < 3) return set_error(RC_E_ARG, "need at least 3 vertices");
    if (T < 1) return set_error(RC_E_ARG, "need at least one triangle");
    if (T > (1LL << 28) || nV > (1LL << 31) - 1) return set_error(RC_E_ARG, "mesh too large");
    cudaStream_t s = (cudaStream_t)stream;
    rc_bvh h = new rc_bvh_s();
    auto fail = [&](rc_status st) { std::string m = t_err; cudaStreamSynchronize(s); free_handle(h); t_err = m; return st; };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(set_error(RC_E_CUDA, "no CUDA device"));
    keep_pool_memory();
    h->nV = nV;
    h->T = T;
    h->builder = builder;
#define RC_TRY(call) do { cudaError_t _e = (call); if (_e != cudaSuccess) return fail(cuda_error(_e, #call)); } while (0)
    RC_TRY(cudaMallocAsync(&h->V, sizeof(float) * 3 * nV, s));
    RC_TRY(cudaMallocAsync(&h->F, sizeof(int32_t) * 3 * T, s));
    RC_TRY(cudaMallocAsync(&h->fnorm, sizeof(float) * 3 * T, s));
    RC_TRY(cudaMallocAsync(&h->farea, sizeof(double) * T, s));
    RC_TRY(cudaMallocAsync(&h->cdf, sizeof(long long) * T, s));
    RC_TRY(cudaMallocAsync(&h->sc, sizeof(DevScalars), s));
    RC_TRY(cudaMemcpyAsync(h->V, d_V, sizeof(float) * 3 * nV, cudaMemcpyDeviceToDevice, s));
    RC_TRY(cudaMemcpyAsync(h->F, d_F, sizeof(int32_t) * 3 * T, cudaMemcpyDeviceToDevice, s));
#undef RC_TRY
    rc_status st = build_bvh(h, s);
    if (st != RC_OK) return fail(st);
    if ((st = scene_box(h)) != RC_OK) return fail(st);
    *out = h;
    return RC_OK;
}

rc_status rc_refit_bvh(rc_bvh h, const float* d_V, void* stream)
{
    RC_RANGE();
    if (!h || !d_V) return set_error(RC_E_ARG, "handle or vertex pointer is NULL");
    rc_status st = use_device_of(h);
    if (st != RC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RC_CUDA(cudaMemcpyAsync(h->V, d_V, sizeof(float) * 3 * h->nV, cudaMemcpyDeviceToDevice, s));
    st = refit_bvh(h, s);
    if (st != RC_OK) return st;
    return scene_box(h);
}

rc_status rc_destroy_bvh(rc_bvh h)
{
    RC_RANGE();
    if (!h) return RC_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(h->device);
    free_handle(h);
    cudaSetDevice(dev);
    return RC_OK;
}

rc_status rc_bvh_get_info(rc_bvh h, rc_bvh_info* out)
{
    RC_RANGE();
    if (!h || !out) return set_error(RC_E_ARG, "handle or out is NULL");
    out->n_tris = h->T;
    out->n_nodes = h->n_int;
    out->node_bytes = h->n_int * 64;
    out->tri_bytes = h->T * 48;
    out->max_depth = h->max_depth;
    out->leaf_size = kLeafMax;
    for (int k = 0; k < 3; ++k) { out->scene_lo[k] = h->lo[k]; out->scene_hi[k] = h->hi[k]; }
    return RC_OK;
}

rc_status rc_sample_points(rc_bvh h, int64_t n, const rc_params* p, float* d_P, float* d_N, int32_t* d_face,
                           double* d_weight, void* stream)
{
    RC_RANGE();
    if (!h) return set_error(RC_E_ARG, "handle is NULL");
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (p->sample_mode == RC_SAMPLE_FACE_CENTROID && n != h->T)
        return set_error(RC_E_ARG, "centroid sampling needs n == T");
    if (n == 0) return RC_OK;
    if (!d_P || !d_N || !d_face) return set_error(RC_E_ARG, "output pointer is NULL");
    if (p->sample_mode == RC_SAMPLE_AREA_RANDOM && h->host_sc.amax_bits == 0)
        return set_error(RC_E_DEGENERATE, "part has no positive-area face");
    if ((st = use_device_of(h)) != RC_OK) return st;
    return sample_points(h, n, p, d_P, d_N, d_face, d_weight, (cudaStream_t)stream);
}

rc_status rc_direction_table(int32_t n_dirs, float* h_dirs)
{
    RC_RANGE();
    if (!h_dirs) return set_error(RC_E_ARG, "output is NULL");
    if (n_dirs < 1 || n_dirs > kMaxDirs) return set_error(RC_E_ARG, "n_dirs out of range");
    fibonacci_hemisphere(n_dirs, h_dirs);
    return RC_OK;
}

rc_status rc_hemisphere_cast(rc_bvh h, const float* d_P, const float* d_N, int64_t n, const rc_params* p,
                             uint32_t* d_bits, int32_t* d_count, int64_t* d_counters, void* stream)
{
    RC_RANGE();
    if (!h) return set_error(RC_E_ARG, "handle is NULL");
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = use_device_of(h)) != RC_OK) return st;
    const bool stats = p->collect_stats != 0;
    if (stats && !d_counters) return set_error(RC_E_ARG, "collect_stats needs the counters array");
    if (d_counters) RC_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * (stats ? 8 : 4), s));
    if (n == 0) return RC_OK;
    if (!d_P || !d_N || !d_bits || !d_count) return set_error(RC_E_ARG, "array pointer is NULL");
    const float4 *dirs = nullptr, *tdirs = nullptr;
    if ((st = device_dirs(p->n_dirs, &dirs, &tdirs)) != RC_OK) return st;
    h->dirs = dirs;
    h->tdirs = p->tile_mode == 1 ? dirs : tdirs;
    h->dirs_n = p->n_dirs;
    return launch_hemisphere(h, d_P, d_N, n, p, d_bits, d_count, (unsigned long long*)d_counters, stats, s);
}

rc_status rc_hemisphere_cast_retests(rc_bvh h, const float* d_P, const float* d_N, int64_t n, const rc_params* p,
                                     uint32_t* d_bits, int32_t* d_count, int64_t* d_counters, int64_t* d_list,
                                     int64_t cap, void* stream)
{
    RC_RANGE();
    if (!h) return set_error(RC_E_ARG, "handle is NULL");
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (!d_counters) return set_error(RC_E_ARG, "the counters array is NULL");
    if (cap < 0 || (cap > 0 && !d_list)) return set_error(RC_E_ARG, "list is NULL or cap < 0");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = use_device_of(h)) != RC_OK) return st;
    RC_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * 8, s));
    if (n == 0) return RC_OK;
    if (!d_P || !d_N || !d_bits || !d_count) return set_error(RC_E_ARG, "array pointer is NULL");
    const float4 *dirs = nullptr, *tdirs = nullptr;
    if ((st = device_dirs(p->n_dirs, &dirs, &tdirs)) != RC_OK) return st;
    h->dirs = dirs;
    h->tdirs = p->tile_mode == 1 ? dirs : tdirs;
    h->dirs_n = p->n_dirs;
    return launch_hemisphere(h, d_P, d_N, n, p, d_bits, d_count, (unsigned long long*)d_counters, true, s,
                             (long long*)d_list, cap);
}

rc_status rc_direction_variability(const uint32_t* d_bits, const float* d_N, const double* d_weight, int64_t n,
                                   const rc_params* p, float* d_acc, int8_t* d_dom, float* d_conc,
                                   double* d_dir_area, rc_summary* h_summary, void* stream)
{
    RC_RANGE();
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n > 0 && (!d_bits || !d_N)) return set_error(RC_E_ARG, "bits or normals pointer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const float4* dirs = nullptr;
    if ((st = device_dirs(p->n_dirs, &dirs)) != RC_OK) return st;
    void* scratch = nullptr;
    unsigned char back[kVarPartOffset];
    {
        ApiScratch sf{s};
        RC_CUDA(cudaMallocAsync(&scratch, kVarScratchBytes, s));
        sf.p[0] = scratch;
        st = launch_variability(d_bits, d_N, d_weight, n, dirs, p, d_acc, d_dom, d_conc, d_dir_area, scratch, s);
        if (st != RC_OK) return st;
        if (h_summary) RC_CUDA(cudaMemcpyAsync(back, scratch, sizeof back, cudaMemcpyDeviceToHost, s));
    }
    if (!h_summary) return RC_OK;
    RC_CUDA(cudaStreamSynchronize(s));
    fill_summary((const long long*)back, (const double*)(back + kVarWsumOffset), n, p->n_dirs, d_weight != nullptr,
                 h_summary);
    return RC_OK;
}

rc_status rc_classify(const rc_summary* s, const rc_params* p, int32_t* label)
{
    RC_RANGE();
    if (!s || !p || !label) return set_error(RC_E_ARG, "NULL argument");
    rc_status st = check_thresholds(p);
    if (st != RC_OK) return st;
    const double mx = std::max(s->axis_share[0], std::max(s->axis_share[1], s->axis_share[2]));
    *label = (s->overall_access < p->t_acc || mx < p->t_share || s->mean_conc > p->t_conc) ? 1 : 0;
    return RC_OK;
}

rc_status rc_orthogonal_cast(rc_bvh h, const float* d_P, const float* d_N, int64_t n, const rc_params* p,
                             uint8_t* d_mask, float* d_travel, int64_t* d_counters, void* stream)
{
    RC_RANGE();
    if (!h) return set_error(RC_E_ARG, "handle is NULL");
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = use_device_of(h)) != RC_OK) return st;
    const bool stats = p->collect_stats != 0;
    if (stats && !d_counters) return set_error(RC_E_ARG, "collect_stats needs the counters array");
    if (d_counters) RC_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * (stats ? 8 : 4), s));
    if (n == 0) return RC_OK;
    if (!d_P || !d_N || !d_mask || !d_travel) return set_error(RC_E_ARG, "array pointer is NULL");
    return launch_orthogonal(h, d_P, d_N, n, p, d_mask, d_travel, (unsigned long long*)d_counters, s);
}

rc_status rc_min_setups(rc_bvh h, const uint8_t* d_mask, const float* d_travel, const int32_t* d_face, int64_t n,
                        const rc_params* p, uint8_t* d_class, rc_setups* h_out, void* stream)
{
    RC_RANGE();
    if (!h || !h_out) return set_error(RC_E_ARG, "handle or output is NULL");
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n > 0 && (!d_mask || !d_travel || !d_face)) return set_error(RC_E_ARG, "array pointer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = use_device_of(h)) != RC_OK) return st;
    // scratch: frame, fixture flags, 68 counters
    FrameDev* fd = nullptr;
    uint8_t* fixture = nullptr;
    unsigned long long* hist = nullptr;
    unsigned long long hh[68];
    {
        ApiScratch sf{s};
        RC_CUDA(cudaMallocAsync(&fd, sizeof(FrameDev), s));
        sf.p[0] = fd;
        RC_CUDA(cudaMallocAsync(&fixture, h->T, s));
        sf.p[1] = fixture;
        RC_CUDA(cudaMallocAsync(&hist, sizeof(unsigned long long) * 68, s));
        sf.p[2] = hist;
        RC_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 68, s));
        if ((st = frame_setup(h, p, fd, s)) != RC_OK) return st;
        st = launch_classes(h, d_mask, d_travel, d_face, n, p, d_class, fd->frame, fd->fbox, fixture, hist, s);
        if (st != RC_OK) return st;
        RC_CUDA(cudaMemcpyAsync(hh, hist, sizeof hh, cudaMemcpyDeviceToHost, s));
    }
    RC_CUDA(cudaStreamSynchronize(s));
    memset(h_out, 0, sizeof *h_out);
    for (int k = 0; k < 64; ++k) h_out->mask_hist[k] = (int64_t)hh[k];
    for (int k = 0; k < 4; ++k) h_out->class_counts[k] = (int64_t)hh[64 + k];
    return rc_setup_cover(h_out->mask_hist, h_out);
}

// Two non-blocking side streams (the orthogonal cast; the copy of the bits
// back to the host) and their events per host thread and device, created on
// first use and kept for the life of the thread.
struct SideStream {
    cudaStream_t s = nullptr, copy = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, cast_done = nullptr;
};

static rc_status side_stream(SideStream** out)
{
    static thread_local std::map<int, SideStream> per_device;
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    SideStream& ss = per_device[dev];
    if (!ss.s) {
        RC_CUDA(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
        RC_CUDA(cudaStreamCreateWithFlags(&ss.copy, cudaStreamNonBlocking));
        RC_CUDA(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
        RC_CUDA(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming));
        RC_CUDA(cudaEventCreateWithFlags(&ss.cast_done, cudaEventDisableTiming));
    }
    *out = &ss;
    return RC_OK;
}

rc_status rc_analyze_part(const float* h_V, int64_t nV, const int32_t* h_F, int64_t T, int64_t n,
                          const rc_params* p, uint32_t* h_bits, int32_t* h_count, uint8_t* h_mask,
                          uint8_t* h_class, rc_part_result* h_out, void* stream)
{
    RC_RANGE();
    if (!h_V || !h_F || !h_out) return set_error(RC_E_ARG, "NULL argument");
    rc_status st = check_params(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (p->sample_mode == RC_SAMPLE_FACE_CENTROID && n != T)
        return set_error(RC_E_ARG, "centroid sampling needs n == T");
    if (nV < 3 || T < 1) return set_error(RC_E_ARG, "empty mesh");
    cudaStream_t s = (cudaStream_t)stream;
    memset(h_out, 0, sizeof *h_out);
    const int W = (p->n_dirs + 31) / 32;
    const bool centroid = p->sample_mode == RC_SAMPLE_FACE_CENTROID;
    // one device block for everything, carved into aligned pieces
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t oV = take(sizeof(float) * 3 * nV), oF = take(sizeof(int32_t) * 3 * T);
    const size_t oP = take(sizeof(float) * 3 * n), oN = take(sizeof(float) * 3 * n);
    const size_t oface = take(sizeof(int32_t) * n), ow = take(centroid ? sizeof(double) * n : 0);
    const size_t obits = take(sizeof(uint32_t) * W * n), ocnt = take(sizeof(int32_t) * n);
    const size_t octr = take(sizeof(int64_t) * 8), omask = take(n), otrav = take(sizeof(float) * 6 * n);
    const size_t ocls = take(n);
    char* base = nullptr;
    RC_CUDA(cudaMallocAsync((void**)&base, off ? off : 256, s));
    float* dV = (float*)(base + oV);
    int32_t* dF = (int32_t*)(base + oF);
    float* dP = (float*)(base + oP);
    float* dN = (float*)(base + oN);
    int32_t* dface = (int32_t*)(base + oface);
    double* dw = centroid ? (double*)(base + ow) : nullptr;
    uint32_t* dbits = (uint32_t*)(base + obits);
    int32_t* dcnt = (int32_t*)(base + ocnt);
    int64_t* dctr = (int64_t*)(base + octr);
    uint8_t* dmask = (uint8_t*)(base + omask);
    float* dtrav = (float*)(base + otrav);
    uint8_t* dcls = (uint8_t*)(base + ocls);
    rc_bvh h = nullptr;
    // with always_setups the orthogonal cast (it needs only the points) runs
    // on a side stream beside the hemispherical cast and the reduction on
    // `s`; the side stream joins `s` before the setups
    SideStream* side = nullptr;
    bool forked = false, copying = false;
    auto done = [&](rc_status r) {
        std::string m = t_err;
        if (forked) cudaStreamSynchronize(side->s);
        if (copying) cudaStreamSynchronize(side->copy);
        cudaFreeAsync(base, s);
        cudaStreamSynchronize(s);
        if (h) rc_destroy_bvh(h);
        t_err = m;
        return r;
    };
#define RC_STEP(call) do { rc_status _r = (call); if (_r != RC_OK) return done(_r); } while (0)
#define RC_CSTEP(call) do { cudaError_t _e = (call); if (_e != cudaSuccess) return done(cuda_error(_e, #call)); } while (0)
    RC_CSTEP(cudaMemcpyAsync(dV, h_V, sizeof(float) * 3 * nV, cudaMemcpyHostToDevice, s));
    RC_CSTEP(cudaMemcpyAsync(dF, h_F, sizeof(int32_t) * 3 * T, cudaMemcpyHostToDevice, s));
    RC_STEP(rc_build_bvh(dV, nV, dF, T, stream, &h));
    RC_STEP(rc_sample_points(h, n, p, dP, dN, dface, dw, stream));
    const bool copy_bits = n > 0 && (h_bits || h_count);
    if ((p->always_setups || copy_bits) && n > 0) RC_STEP(side_stream(&side));
    if (p->always_setups && n > 0) RC_CSTEP(cudaEventRecord(side->fork, s));
    RC_STEP(rc_hemisphere_cast(h, dP, dN, n, p, dbits, dcnt, dctr, stream));
    if (copy_bits) {
        // the bits and counts go back to the host beside the reduction
        RC_CSTEP(cudaEventRecord(side->cast_done, s));
        RC_CSTEP(cudaStreamWaitEvent(side->copy, side->cast_done, 0));
        copying = true;
        if (h_bits)
            RC_CSTEP(cudaMemcpyAsync(h_bits, dbits, sizeof(uint32_t) * W * n, cudaMemcpyDeviceToHost, side->copy));
        if (h_count)
            RC_CSTEP(cudaMemcpyAsync(h_count, dcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, side->copy));
    }
    if (p->always_setups && n > 0) {
        // issued after the hemispherical cast, whose persistent kernel then
        // holds the SMs first; the orthogonal cast fills them as it drains
        RC_CSTEP(cudaStreamWaitEvent(side->s, side->fork, 0));
        forked = true;
        RC_STEP(rc_orthogonal_cast(h, dP, dN, n, p, dmask, dtrav, dctr + 4, side->s));
        RC_CSTEP(cudaEventRecord(side->join, side->s));
    }
    RC_CSTEP(cudaMemcpyAsync(h_out->cast_counters, dctr, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, s));
    RC_STEP(rc_direction_variability(dbits, dN, dw, n, p, nullptr, nullptr, nullptr, nullptr, &h_out->summary, stream));
    RC_STEP(rc_classify(&h_out->summary, p, &h_out->label));
    if (p->always_setups || h_out->label == 0) {
        if (forked) RC_CSTEP(cudaStreamWaitEvent(s, side->join, 0));
        else RC_STEP(rc_orthogonal_cast(h, dP, dN, n, p, dmask, dtrav, dctr + 4, stream));
        RC_CSTEP(cudaMemcpyAsync(h_out->ortho_counters, dctr + 4, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, s));
        RC_STEP(rc_min_setups(h, dmask, dtrav, dface, n, p, dcls, &h_out->setups, stream));
        h_out->setups_ran = 1;
        if (h_mask && n) RC_CSTEP(cudaMemcpyAsync(h_mask, dmask, n, cudaMemcpyDeviceToHost, s));
        if (h_class && n) RC_CSTEP(cudaMemcpyAsync(h_class, dcls, n, cudaMemcpyDeviceToHost, s));
    }
#undef RC_STEP
#undef RC_CSTEP
    return done(RC_OK);
}

rc_status rc_setup_cover(const int64_t* h_mask_hist, rc_setups* out)
{
    RC_RANGE();
    if (!h_mask_hist || !out) return set_error(RC_E_ARG, "NULL argument");
    int64_t hh[64];
    for (int m = 0; m < 64; ++m) {
        if (h_mask_hist[m] < 0) return set_error(RC_E_ARG, "negative histogram count");
        hh[m] = m ? h_mask_hist[m] : 0;
    }
    // exact cover: smallest |S|, ties to the smallest bitmask
    out->setups_exact = 0;
    out->chosen_exact = 0;
    bool any = false;
    for (int m = 1; m < 64; ++m) any |= hh[m] != 0;
    if (any) {
        bool done = false;
        for (int size = 1; size <= 6 && !done; ++size)
            for (int S = 1; S < 64 && !done; ++S) {
                if (__builtin_popcount(S) != size) continue;
                bool ok = true;
                for (int m = 1; m < 64 && ok; ++m) ok = hh[m] == 0 || (m & S);
                if (ok) { out->setups_exact = size; out->chosen_exact = (uint8_t)S; done = true; }
            }
    }
    // greedy cover: the axis covering most uncovered viable points, ties to the lower axis
    int S = 0;
    int64_t left[64];
    for (int m = 0; m < 64; ++m) left[m] = hh[m];
    for (;;) {
        bool rem = false;
        for (int m = 1; m < 64; ++m) rem |= left[m] != 0;
        if (!rem) break;
        int best = -1;
        int64_t bc = 0;
        for (int a = 0; a < 6; ++a) {
            if ((S >> a) & 1) continue;
            int64_t c = 0;
            for (int m = 1; m < 64; ++m)
                if ((m >> a) & 1) c += left[m];
            if (best < 0 || c > bc) { best = a; bc = c; }
        }
        S |= 1 << best;
        for (int m = 1; m < 64; ++m)
            if ((m >> best) & 1) left[m] = 0;
    }
    out->setups_greedy = __builtin_popcount(S);
    out->chosen_greedy = (uint8_t)S;
    return RC_OK;
}

}  // extern "C"
