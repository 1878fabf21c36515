// noalloc.cu -- rc_direction_variability_noalloc: the directional-variability
// reduction with its scratch in a fixed static device array instead of
// stream-ordered allocations.
//
// Some callers cannot let a library allocate device memory: a process that
// reserves its whole HBM budget for its own arena at start-up and routes every
// allocation through it, or one that runs at its device-memory limit, where a
// cudaMalloc/cudaMallocAsync inside a library call would fail or break the
// caller's accounting.  This entry point performs no device (or host heap)
// allocation; it uses the static array below, which every GPU that loads the
// library holds until the process exits.
#include <string.h>

#include <mutex>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

rc_status launch_variability(const uint32_t* bits, const float* N, const double* weight, int64_t n,
                             const float4* dirs, const rc_params* p, float* acc, int8_t* dom, float* conc,
                             double* dir_area, unsigned long long* scratch, cudaStream_t s);
rc_status set_error(rc_status st, const std::string& msg);

// Layout: [ 9 + kNoAllocMaxDirs uint64 accumulators | kNoAllocMaxDirs float4 directions ]
constexpr int kNoAllocMaxDirs = 8192;
constexpr size_t kNoAllocAccBytes = ((9 + (size_t)kNoAllocMaxDirs) * 8 + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocAccBytes + (size_t)kNoAllocMaxDirs * 16;   // 196,864 bytes

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;

struct NoAllocDevice {
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
    int32_t dirs_n = 0;              // direction count currently stored in the table
};

static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
static float g_noalloc_h3[3 * kNoAllocMaxDirs];        // host staging, no heap use
static float4 g_noalloc_h4[kNoAllocMaxDirs];

}  // namespace rc

using namespace rc;

extern "C" rc_status rc_direction_variability_noalloc(const uint32_t* d_bits, const float* d_N,
                                                      const double* d_weight, int64_t n, const rc_params* p,
                                                      float* d_acc, int8_t* d_dom, float* d_conc,
                                                      double* d_dir_area, rc_summary* h_summary, void* stream)
{
    RC_RANGE();
    if (!p) return set_error(RC_E_ARG, "params is NULL");
    if (p->n_dirs < 1) return set_error(RC_E_ARG, "n_dirs must be >= 1");
    if (p->n_dirs > kNoAllocMaxDirs)
        return set_error(RC_E_UNSUPPORTED, "rc_direction_variability_noalloc supports at most 8192 directions "
                                           "(its static scratch is 196,864 bytes per device)");
    if (p->conc_mode != 0 && p->conc_mode != 1) return set_error(RC_E_ARG, "conc_mode must be 0 or 1");
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n > 0 && (!d_bits || !d_N)) return set_error(RC_E_ARG, "bits or normals pointer is NULL");
    if (d_weight && n > (1LL << 21))
        return set_error(RC_E_UNSUPPORTED, "weighted summaries support at most 2^21 points");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(RC_E_UNSUPPORTED, "device index out of range");

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.base) {
        // once per device, with that device current: the host-side name of
        // the array is only a stand-in, the kernels need its device address
        void* ptr = nullptr;
        RC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        d.base = (unsigned char*)ptr;
    }
    unsigned long long* acc = (unsigned long long*)d.base;
    float4* dirs = (float4*)(d.base + kNoAllocAccBytes);
    if (d.dirs_n != p->n_dirs) {
        rc_status st = rc_direction_table(p->n_dirs, g_noalloc_h3);
        if (st != RC_OK) return st;
        for (int32_t j = 0; j < p->n_dirs; ++j)
            g_noalloc_h4[j] = make_float4(g_noalloc_h3[3 * j], g_noalloc_h3[3 * j + 1], g_noalloc_h3[3 * j + 2], 0.0f);
        RC_CUDA(cudaMemcpyAsync(dirs, g_noalloc_h4, sizeof(float4) * p->n_dirs, cudaMemcpyHostToDevice, s));
        d.dirs_n = p->n_dirs;
    }
    // the sums, the max weight and the per-direction counters start at zero
    RC_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (9 + (size_t)p->n_dirs), s));
    rc_status st = launch_variability(d_bits, d_N, d_weight, n, dirs, p, d_acc, d_dom, d_conc, d_dir_area, acc, s);
    if (st != RC_OK) return st;
    if (!h_summary) return RC_OK;
    long long sums[8];
    RC_CUDA(cudaMemcpyAsync(sums, acc, sizeof sums, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    rc_summary& o = *h_summary;
    memset(&o, 0, sizeof o);
    const long long counted = sums[0];
    o.n_points = n;
    o.n_counted = counted;
    o.n_zero_visible = n - counted;
    for (int k = 0; k < 3; ++k) {
        o.dom_count[k] = sums[1 + k];
        o.axis_share[k] = counted ? (double)sums[1 + k] / (double)counted : 0.0;
    }
    o.count_sum = sums[4];
    o.weighted_count_q = sums[5];
    o.weight_sum_q = sums[6];
    o.conc_sum_q = sums[7];
    const long long den = sums[6] * (long long)p->n_dirs;
    o.overall_access = den ? (double)sums[5] / (double)den : 0.0;
    o.overall_access_unweighted = n ? (double)sums[4] / ((double)n * (double)p->n_dirs) : 0.0;
    o.mean_conc = counted ? (double)sums[7] / (1099511627776.0 * (double)counted) : 0.0;
    return RC_OK;
}
