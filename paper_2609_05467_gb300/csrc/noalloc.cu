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

rc_status check_params_public(const rc_params* p);

// Layout: [ the reduction's scratch (kVarScratchBytes, rounded up to 256) |
//           32 * ceil(kNoAllocMaxDirs / 32) float4 directions ]
constexpr int kNoAllocMaxDirs = 8192;
constexpr size_t kNoAllocAccBytes = (kVarScratchBytes + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocAccBytes + (size_t)kNoAllocMaxDirs * 16;   // 164,096 bytes
static_assert(kNoAllocBytes == 164096, "size stated in rc.h");

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
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (p->n_dirs > kNoAllocMaxDirs)
        return set_error(RC_E_UNSUPPORTED, "rc_direction_variability_noalloc supports at most 8192 directions "
                                           "(its static scratch is 164,096 bytes per device)");
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n > 0 && (!d_bits || !d_N)) return set_error(RC_E_ARG, "bits or normals pointer is NULL");
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
    void* acc = d.base;
    float4* dirs = (float4*)(d.base + kNoAllocAccBytes);
    if (d.dirs_n != p->n_dirs) {
        // the table is rewritten from host memory; a stream that is being
        // captured would record that copy instead of running it now
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        RC_CUDA(cudaStreamIsCapturing(s, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return set_error(RC_E_UNSUPPORTED, "rc_direction_variability_noalloc: the direction table for this "
                                               "n_dirs is uploaded by a call outside stream capture");
        st = rc_direction_table(p->n_dirs, g_noalloc_h3);
        if (st != RC_OK) return st;
        // as the allocating call's table: entry j carries index j in w, and
        // the last tile is padded with entry 0's direction and index -1
        const int32_t N = p->n_dirs, N32 = (N + 31) / 32 * 32;
        float pad_w;
        const int32_t minus1 = -1;
        memcpy(&pad_w, &minus1, sizeof pad_w);
        for (int32_t j = 0; j < N32; ++j) {
            const int32_t k = j < N ? j : 0;
            float w = pad_w;
            if (j < N) memcpy(&w, &j, sizeof w);
            g_noalloc_h4[j] = make_float4(g_noalloc_h3[3 * k], g_noalloc_h3[3 * k + 1], g_noalloc_h3[3 * k + 2], w);
        }
        RC_CUDA(cudaMemcpyAsync(dirs, g_noalloc_h4, sizeof(float4) * N32, cudaMemcpyHostToDevice, s));
        d.dirs_n = N;
    }
    // launch_variability clears the sums it accumulates into on `stream`
    st = launch_variability(d_bits, d_N, d_weight, n, dirs, p, d_acc, d_dom, d_conc, d_dir_area, acc, s);
    if (st != RC_OK) return st;
    if (!h_summary) return RC_OK;
    unsigned char back[kVarPartOffset];
    RC_CUDA(cudaMemcpyAsync(back, acc, sizeof back, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    fill_summary((const long long*)back, (const double*)(back + kVarWsumOffset), n, p->n_dirs, d_weight != nullptr,
                 h_summary);
    return RC_OK;
}
