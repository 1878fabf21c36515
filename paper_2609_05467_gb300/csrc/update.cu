// update.cu -- re-analysis of an edited part whose triangle list is
// unchanged (a feature moved, the mesh topology kept).  The paper aims at
// interactive use while a part is designed (Sections 1 and 5); after an edit
// only rays that can reach the edited region need to be cast again.
//
// Reading: every sample point stays on its face.  In area mode point i keeps
// its face and its own counter-based u1, u2 (its barycentric position) on the
// moved triangle; in centroid mode it is the moved centroid.  The result is
// then exactly the full analysis of the edited part at those points.
#include <float.h>
#include <math.h>
#include <string.h>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

rc_status launch_hemisphere_update(rc_bvh h, const float* P, const float* N, int64_t n, const int32_t* face,
                                   const uint8_t* changed, const float box[6], const float4* tdirs,
                                   const rc_params* p, uint32_t* bits, int32_t* count, unsigned long long* counters,
                                   cudaStream_t s);
rc_status device_dirs_for_cast(const rc_params* p, const float4** tdirs);
rc_status check_params_public(const rc_params* p);

__device__ __forceinline__ double uniform01_u(unsigned long long seed, long long i, int k)
{
    const unsigned long long ctr = (unsigned long long)(3 * i + k) * 0x9E3779B97F4A7C15ULL;
    const unsigned long long r = splitmix64(seed ^ ctr);
    return __dmul_rn(__ull2double_rn(r >> 11), 1.0 / 9007199254740992.0);
}

// point i on face[i]: area mode at (1 - s) A + s (1 - u2) B + s u2 C with
// s = sqrt(u1) (the sampler's formula and numbers), centroid mode at the
// face centroid; bad[0] receives the first point whose face is out of range
__global__ void k_sample_on_faces(const float* __restrict__ V, const int32_t* __restrict__ F, int64_t T,
                                  const float* __restrict__ fnorm, int64_t n,
                                  unsigned long long seed, int centroid, const int32_t* __restrict__ face,
                                  float* P, float* Nout, unsigned long long* bad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t f = face[i];
    if (f < 0 || f >= T) {
        atomicMin(bad, (unsigned long long)i);
        return;
    }
    if (centroid) {
        for (int k = 0; k < 3; ++k) {
            P[3 * i + k] = face_centroid(V, F, f, k);
            Nout[3 * i + k] = fnorm[3 * f + k];
        }
        return;
    }
    const double u1 = uniform01_u(seed, i, 1), u2 = uniform01_u(seed, i, 2);
    const double sq = __dsqrt_rn(u1);
    const double wa = __dsub_rn(1.0, sq), wb = __dmul_rn(sq, __dsub_rn(1.0, u2)), wc = __dmul_rn(sq, u2);
    for (int k = 0; k < 3; ++k) {
        const double A = V[3 * (int64_t)F[3 * f + 0] + k];
        const double B = V[3 * (int64_t)F[3 * f + 1] + k];
        const double C = V[3 * (int64_t)F[3 * f + 2] + k];
        double q = __dadd_rn(__dmul_rn(wa, A), __dmul_rn(wb, B));
        q = __dadd_rn(q, __dmul_rn(wc, C));
        P[3 * i + k] = __double2float_rn(q);
        Nout[3 * i + k] = fnorm[3 * f + k];
    }
}

// faces with a moved vertex (bit-for-bit comparison), their count and the box
// of their old and new triangles (order-preserving integer min / max, reduced
// over the warp before the atomics)
__global__ void k_changed_faces(const float* __restrict__ V0, const float* __restrict__ V1, int64_t nV,
                                const int32_t* __restrict__ F, int64_t T, uint8_t* __restrict__ changed,
                                int* box /*lo xyz, hi xyz*/, unsigned long long* n_changed,
                                unsigned long long* bad)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool moved = false;
    if (f < T) {
        int64_t v[3];
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
            v[c] = F[3 * f + c];
            if (v[c] < 0 || v[c] >= nV) ok = false;
        }
        if (!ok) {
            atomicMin(bad, (unsigned long long)f);
            changed[f] = 0;
        } else {
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k)
                    moved |= __float_as_uint(V0[3 * v[c] + k]) != __float_as_uint(V1[3 * v[c] + k]);
            changed[f] = moved ? 1 : 0;
            if (moved)
                for (int k = 0; k < 3; ++k)
                    for (int c = 0; c < 3; ++c) {
                        lo[k] = fminf(lo[k], fminf(V0[3 * v[c] + k], V1[3 * v[c] + k]));
                        hi[k] = fmaxf(hi[k], fmaxf(V0[3 * v[c] + k], V1[3 * v[c] + k]));
                    }
        }
    }
    const unsigned FULL = 0xFFFFFFFFu;
    const unsigned m = __ballot_sync(FULL, moved);
    if (m == 0u) return;
    for (int off = 16; off; off >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(FULL, lo[k], off));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(FULL, hi[k], off));
        }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(n_changed, (unsigned long long)__popc(m));
        for (int k = 0; k < 3; ++k) {
            atomicMin(&box[k], float_to_ordered(lo[k]));
            atomicMax(&box[3 + k], float_to_ordered(hi[k]));
        }
    }
}

__global__ void k_changed_init(int* box, unsigned long long* n_changed, unsigned long long* bad)
{
    if (threadIdx.x < 3) box[threadIdx.x] = 0x7FFFFFFF;
    else if (threadIdx.x < 6) box[threadIdx.x] = (int)0x80000000;
    if (threadIdx.x == 0) {
        *n_changed = 0;
        *bad = ~0ULL;
    }
}

// one device scratch buffer, freed in stream order when the scope ends
struct ScratchOne {
    cudaStream_t s;
    void* p = nullptr;
    ~ScratchOne()
    {
        if (p) cudaFreeAsync(p, s);
    }
};

static rc_status on_device(rc_bvh h)
{
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) RC_CUDA(cudaSetDevice(h->device));
    return RC_OK;
}

}  // namespace rc

using namespace rc;

extern "C" {

rc_status rc_sample_points_on_faces(rc_bvh h, int64_t n, const rc_params* p, const int32_t* d_face, float* d_P,
                                    float* d_N, void* stream)
{
    RC_RANGE();
    if (!h) return set_error(RC_E_ARG, "handle is NULL");
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n == 0) return RC_OK;
    if (!d_face || !d_P || !d_N) return set_error(RC_E_ARG, "array pointer is NULL");
    if ((st = on_device(h)) != RC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* bad = nullptr;
    ScratchOne sf{s};
    RC_CUDA(cudaMallocAsync(&bad, sizeof(unsigned long long), s));
    sf.p = bad;
    RC_CUDA(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), s));
    k_sample_on_faces<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->V, h->F, h->T, h->fnorm, n, p->seed,
                                                                  p->sample_mode == RC_SAMPLE_FACE_CENTROID, d_face,
                                                                  d_P, d_N, bad);
    RC_LAUNCHED();
    unsigned long long hb = 0;
    RC_CUDA(cudaMemcpyAsync(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    if (hb != ~0ULL) return set_error(RC_E_ARG, "face of point " + std::to_string(hb) + " is outside [0, T)");
    return RC_OK;
}

rc_status rc_changed_faces(const float* d_V_old, const float* d_V_new, int64_t nV, const int32_t* d_F, int64_t T,
                           uint8_t* d_changed, float* h_box, int64_t* h_n_changed, void* stream)
{
    RC_RANGE();
    if (!h_box || !h_n_changed) return set_error(RC_E_ARG, "output is NULL");
    if (nV < 0 || T < 0) return set_error(RC_E_ARG, "sizes must be >= 0");
    if (T > 0 && (!d_V_old || !d_V_new || !d_F || !d_changed)) return set_error(RC_E_ARG, "array pointer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    struct Scratch { int box[6]; int pad[2]; unsigned long long n, bad; };
    Scratch* d = nullptr;
    ScratchOne sf{s};
    RC_CUDA(cudaMallocAsync(&d, sizeof(Scratch), s));
    sf.p = d;
    k_changed_init<<<1, 32, 0, s>>>(d->box, &d->n, &d->bad);
    RC_LAUNCHED();
    if (T > 0) {
        k_changed_faces<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(d_V_old, d_V_new, nV, d_F, T, d_changed, d->box,
                                                                     &d->n, &d->bad);
        RC_LAUNCHED();
    }
    Scratch hs;
    RC_CUDA(cudaMemcpyAsync(&hs, d, sizeof hs, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    if (hs.bad != ~0ULL) return set_error(RC_E_ARG, "face " + std::to_string(hs.bad) + " has a vertex index outside [0, nV)");
    *h_n_changed = (int64_t)hs.n;
    for (int k = 0; k < 6; ++k)     // no changed face: an empty box (lo > hi) that no ray enters
        h_box[k] = hs.n ? ordered_to_float(hs.box[k]) : (k < 3 ? FLT_MAX : -FLT_MAX);
    return RC_OK;
}

rc_status rc_hemisphere_update(rc_bvh h, const float* d_P, const float* d_N, const int32_t* d_face, int64_t n,
                               const uint8_t* d_changed, const float* h_box, const rc_params* p, uint32_t* d_bits,
                               int32_t* d_count, int64_t* d_counters, void* stream)
{
    RC_RANGE();
    if (!h || !h_box) return set_error(RC_E_ARG, "handle or box is NULL");
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    for (int k = 0; k < 6; ++k)
        if (!isfinite(h_box[k])) return set_error(RC_E_ARG, "box must be finite");
    if ((st = on_device(h)) != RC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_counters) RC_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * 4, s));
    if (n == 0) return RC_OK;
    if (!d_P || !d_N || !d_face || !d_changed || !d_bits || !d_count)
        return set_error(RC_E_ARG, "array pointer is NULL");
    const float4* tdirs = nullptr;
    if ((st = device_dirs_for_cast(p, &tdirs)) != RC_OK) return st;
    return launch_hemisphere_update(h, d_P, d_N, n, d_face, d_changed, h_box, tdirs, p, d_bits, d_count,
                                    (unsigned long long*)d_counters, s);
}

}  // extern "C"
