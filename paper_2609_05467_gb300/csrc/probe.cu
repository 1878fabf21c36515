// probe.cu -- ceilings a BVH traversal meets when its tree stays in L2:
// random record reads from an L2-resident buffer (node- or triangle-sized
// records, as the traversal fetches them) and FP32 issue (the slab and
// triangle tests).  Reported beside the HBM roofline; not part of the
// paper's method.
#include "rc_internal.cuh"

namespace rc {

constexpr int kProbeThreads = 256;

// each thread walks a pseudo-random sequence of records (index = splitmix64
// of a counter, masked to the buffer) and xors what it reads; a record is
// `vecs` consecutive float4 (1 = 16 B, 8 = 128 B, the size of a 4-wide node)
__global__ void __launch_bounds__(kProbeThreads)
k_probe_l2(const float4* __restrict__ buf, unsigned long long mask, int reads, int vecs, unsigned* sink)
{
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned acc = 0;
    for (int k = 0; k < reads; ++k) {
        const unsigned long long rec = splitmix64(t * 0x100000001B3ULL + (unsigned long long)k) & mask;
        for (int v = 0; v < vecs; ++v) {
            const float4 x = __ldg(&buf[rec * vecs + v]);
            acc ^= __float_as_uint(x.x) ^ __float_as_uint(x.w);
        }
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;    // keeps the loads alive
}

// eight independent FMA chains per thread
__global__ void __launch_bounds__(kProbeThreads) k_probe_fp32(int iters, float seed, float* sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + (float)(threadIdx.x + k);
    const float m = 0.999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.678f) sink[0] = s;
}

}  // namespace rc

using namespace rc;

extern "C" {

rc_status rc_probe_l2(int64_t buffer_bytes, int32_t record_bytes, int32_t reads_per_thread, double* h_gbs,
                      void* stream)
{
    if (!h_gbs) return set_error(RC_E_ARG, "output is NULL");
    if (record_bytes != 16 && record_bytes != 32 && record_bytes != 64 && record_bytes != 128)
        return set_error(RC_E_ARG, "record_bytes must be 16, 32, 64 or 128");
    if (buffer_bytes < (1 << 20) || buffer_bytes > (1LL << 30) || (buffer_bytes & (buffer_bytes - 1)))
        return set_error(RC_E_ARG, "buffer_bytes must be a power of two in [1 MiB, 1 GiB]");
    if (reads_per_thread < 1 || reads_per_thread > 4096) return set_error(RC_E_ARG, "reads_per_thread out of range");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    RC_CUDA(cudaGetDevice(&dev));
    RC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float4* buf = nullptr;
    unsigned* sink = nullptr;
    RC_CUDA(cudaMallocAsync(&buf, (size_t)buffer_bytes, s));
    RC_CUDA(cudaMallocAsync(&sink, sizeof(unsigned), s));
    RC_CUDA(cudaMemsetAsync(buf, 0x3C, (size_t)buffer_bytes, s));   // also brings it into L2
    const int vecs = record_bytes / 16;
    const unsigned long long mask = (unsigned long long)(buffer_bytes / record_bytes) - 1;
    const unsigned blocks = (unsigned)sms * 8;
    cudaEvent_t e0, e1;
    RC_CUDA(cudaEventCreate(&e0));
    RC_CUDA(cudaEventCreate(&e1));
    k_probe_l2<<<blocks, kProbeThreads, 0, s>>>(buf, mask, reads_per_thread, vecs, sink);   // warm-up
    RC_LAUNCHED();
    RC_CUDA(cudaEventRecord(e0, s));
    k_probe_l2<<<blocks, kProbeThreads, 0, s>>>(buf, mask, reads_per_thread, vecs, sink);
    RC_LAUNCHED();
    RC_CUDA(cudaEventRecord(e1, s));
    RC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    RC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    cudaFreeAsync(sink, s);
    *h_gbs = (double)blocks * kProbeThreads * reads_per_thread * record_bytes / (ms * 1e-3) / 1e9;
    return RC_OK;
}

rc_status rc_probe_fp32(int32_t iters, double* h_tflops, void* stream)
{
    if (!h_tflops) return set_error(RC_E_ARG, "output is NULL");
    if (iters < 1 || iters > (1 << 20)) return set_error(RC_E_ARG, "iters out of range");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    RC_CUDA(cudaGetDevice(&dev));
    RC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    RC_CUDA(cudaMallocAsync(&sink, sizeof(float), s));
    const unsigned blocks = (unsigned)sms * 8;
    cudaEvent_t e0, e1;
    RC_CUDA(cudaEventCreate(&e0));
    RC_CUDA(cudaEventCreate(&e1));
    k_probe_fp32<<<blocks, kProbeThreads, 0, s>>>(iters, 1.0f, sink);
    RC_LAUNCHED();
    RC_CUDA(cudaEventRecord(e0, s));
    k_probe_fp32<<<blocks, kProbeThreads, 0, s>>>(iters, 1.0f, sink);
    RC_LAUNCHED();
    RC_CUDA(cudaEventRecord(e1, s));
    RC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    RC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    *h_tflops = (double)blocks * kProbeThreads * iters * 8 * 2.0 / (ms * 1e-3) / 1e12;
    return RC_OK;
}

}  // extern "C"
