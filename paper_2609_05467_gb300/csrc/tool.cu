// tool.cu -- tool-aware accessibility along the six machining axes: the
// orthogonal cast of Section 3.2 with the thin ray replaced by a sampled
// ball-end tool of radius r (centre ray plus a ring of parallel rays); the
// kernel is k_tool_cast_axis in cast.cu.
#include <math.h>

#include <vector>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {
rc_status launch_tool_cast(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p, double radius,
                           const double2* ring, int K, uint8_t* mask, unsigned long long* counters, cudaStream_t s);
rc_status check_params_public(const rc_params* p);
}  // namespace rc

using namespace rc;

extern "C" rc_status rc_tool_cast(rc_bvh h, const float* d_P, const float* d_N, int64_t n, const rc_params* p,
                                  double tool_radius, int32_t ring_rays, uint8_t* d_mask, int64_t* d_counters,
                                  void* stream)
{
    RC_RANGE();
    if (!h) return set_error(RC_E_ARG, "handle is NULL");
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (!(tool_radius >= 0.0 && tool_radius <= 1e4)) return set_error(RC_E_ARG, "tool_radius must be in [0, 1e4] mm");
    if (ring_rays < 0 || ring_rays > 64) return set_error(RC_E_ARG, "ring_rays must be in [0, 64]");
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) RC_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (d_counters) RC_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * 4, s));
    if (n == 0) return RC_OK;
    if (!d_P || !d_N || !d_mask) return set_error(RC_E_ARG, "array pointer is NULL");
    // ring directions t_k = (2 pi k) / K, host libm
    std::vector<double2> ring(ring_rays > 0 ? ring_rays : 1);
    for (int k = 0; k < ring_rays; ++k) {
        const double t = 2.0 * M_PI * (double)k / (double)ring_rays;
        ring[k] = make_double2(cos(t), sin(t));
    }
    double2* d_ring = nullptr;
    RC_CUDA(cudaMallocAsync(&d_ring, sizeof(double2) * ring.size(), s));
    // a copy from pageable memory has read the host vector when it returns
    const cudaError_t e = cudaMemcpyAsync(d_ring, ring.data(), sizeof(double2) * ring.size(),
                                          cudaMemcpyHostToDevice, s);
    st = e == cudaSuccess ? launch_tool_cast(h, d_P, d_N, n, p, tool_radius, d_ring, ring_rays, d_mask,
                                             (unsigned long long*)d_counters, s)
                          : cuda_error(e, "ring table upload");
    // stream-ordered: released after the kernel that reads it
    cudaFreeAsync(d_ring, s);
    return st;
}
