// reduce.cu -- Section 3.3 reductions: directional variability of the
// visible directions (dominant axis, axis concentration, part sums), the
// per-direction visible-area histogram, fixture faces and face classes with
// the 64-bin histogram of reachable-axis masks for the setup cover.
//
// The counts, shares and concentrations are int64 sums of fixed-point
// values, and the area-weighted sums are FP64 sums in a fixed order (per
// warp, per block, then over the blocks by one warp), so the summary does
// not depend on the order in which blocks finish.
#include <math.h>
#include <string.h>

#include "rc_internal.cuh"

namespace rc {

enum { S_COUNTED = 0, S_DOM = 1, S_COUNT = 4, S_CONC = 5, S_N = 6 };
static_assert(S_N <= kVarSums, "integer sums of the variability scratch");

// round(x * 2^40) to nearest, ties to even, for an fp32 x with |x| < 8, in
// fp32 arithmetic: x * 2^40 = hi * 2^22 + lo with hi = rint(x * 2^18) and
// lo = rint((x * 2^18 - hi) * 2^22).  x * 2^18 and its remainder are exact;
// each rint adds 1.5 * 2^23, whose ulp is 1, and reads the integer from the
// bits.  hi * 2^22 is even, so rounding the remainder alone makes the same
// tie decisions as rounding the whole (equal to llrint((double)x * 2^40)).
__device__ __forceinline__ void fixed40_split(float x, int& hi, int& lo)
{
    const float C = 12582912.0f;
    const float t = __fmul_rn(x, 262144.0f);
    const float a = __fadd_rn(t, C);
    hi = __float_as_int(a) - __float_as_int(C);
    const float r = __fsub_rn(t, __fsub_rn(a, C));
    lo = __float_as_int(__fmaf_rn(r, 4194304.0f, C)) - __float_as_int(C);
}

// One warp per point: recompute each visible direction, sum llrint(d*2^40)
// per axis, count visible rays per largest-|component| axis.  The point's
// bit row is read 32 words at a time by the whole warp (one coalesced load)
// and each word is handed to the lanes by a shuffle, so the loop over the
// words waits on memory once per 32 words instead of once per word.
__global__ void __launch_bounds__(256)
k_variability(const uint32_t* __restrict__ bits, const float* __restrict__ Nrm,
              const double* __restrict__ weight, int64_t n,
              const float4* __restrict__ dirs, int n_dirs, int conc_mode, float* acc, int8_t* dom,
              float* conc, unsigned long long* sums, double* wpart)
{
    __shared__ long long blk[S_N];
    __shared__ double wsh[2][8];
    if (threadIdx.x < S_N) blk[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int W = (n_dirs + 31) >> 5;
    long long loc[S_N] = {0, 0, 0, 0, 0, 0};
    double lwc = 0.0, lw = 0.0;   // lane 0: sum w_i count_i and sum w_i of the warp's points, in order
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const float nx = Nrm[3 * i], ny = Nrm[3 * i + 1], nz = Nrm[3 * i + 2];
        const Onb b = make_onb(nx, ny, nz);
        long long M0 = 0, M1 = 0, M2 = 0;
        int a0 = 0, a1 = 0, a2 = 0, cnt = 0;
        for (int w0 = 0; w0 < W; w0 += 32) {
            const int wn = min(32, W - w0);
            const uint32_t mine = lane < wn ? __ldg(&bits[i * W + w0 + lane]) : 0u;
            // per 32 words a lane adds at most 32 terms: |sum hi| < 2^24,
            // |sum lo| < 2^27, so int32 partial sums are exact
            int h0 = 0, h1 = 0, h2 = 0, l0 = 0, l1 = 0, l2 = 0;
            for (int dw = 0; dw < wn; ++dw) {
                const int w = w0 + dw;
                const uint32_t word = __shfl_sync(0xFFFFFFFFu, mine, dw);
                if (!((word >> lane) & 1u)) continue;
                const float4 h = __ldg(&dirs[32 * w + lane]);
                float dx, dy, dz;
                local_to_world(b, nx, ny, nz, h.x, h.y, h.z, dx, dy, dz);
                int qh, ql;
                fixed40_split(dx, qh, ql);
                h0 += qh;
                l0 += ql;
                fixed40_split(dy, qh, ql);
                h1 += qh;
                l1 += ql;
                fixed40_split(dz, qh, ql);
                h2 += qh;
                l2 += ql;
                int best = 0;
                float bv = fabsf(dx);
                if (fabsf(dy) > bv) { best = 1; bv = fabsf(dy); }
                if (fabsf(dz) > bv) best = 2;
                a0 += best == 0;
                a1 += best == 1;
                a2 += best == 2;
                ++cnt;
            }
            M0 += (long long)h0 * 4194304LL + l0;
            M1 += (long long)h1 * 4194304LL + l1;
            M2 += (long long)h2 * 4194304LL + l2;
        }
        for (int off = 16; off; off >>= 1) {
            M0 += __shfl_xor_sync(0xFFFFFFFFu, M0, off);
            M1 += __shfl_xor_sync(0xFFFFFFFFu, M1, off);
            M2 += __shfl_xor_sync(0xFFFFFFFFu, M2, off);
            a0 += __shfl_xor_sync(0xFFFFFFFFu, a0, off);
            a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, off);
            a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, off);
            cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
        }
        if (lane == 0) {
            const long long Ma[3] = {M0 < 0 ? -M0 : M0, M1 < 0 ? -M1 : M1, M2 < 0 ? -M2 : M2};
            const int ac[3] = {a0, a1, a2};
            int dm = -1;
            double cc = 0.0;
            if (cnt > 0) {
                dm = 0;
                if (Ma[1] > Ma[dm]) dm = 1;
                if (Ma[2] > Ma[dm]) dm = 2;
                if (conc_mode == 0)
                    cc = __ddiv_rn((double)ac[dm], (double)cnt);
                else
                    cc = __ddiv_rn(__ll2double_rn(Ma[dm]), __dmul_rn(1099511627776.0, (double)cnt));
                loc[S_COUNTED] += 1;
                loc[S_DOM + dm] += 1;
                loc[S_CONC] += llrint(__dmul_rn(cc, 1099511627776.0));
            }
            loc[S_COUNT] += cnt;
            if (weight) {
                const double wi = weight[i];
                lwc = __dadd_rn(lwc, __dmul_rn(wi, (double)cnt));
                lw = __dadd_rn(lw, wi);
            }
            if (acc) acc[i] = __double2float_rn(__ddiv_rn((double)cnt, (double)n_dirs));
            if (dom) dom[i] = (int8_t)dm;
            if (conc) conc[i] = __double2float_rn(cc);
        }
    }
    if (lane == 0)
        for (int k = 0; k < S_N; ++k)
            if (loc[k]) atomicAdd((unsigned long long*)&blk[k], (unsigned long long)loc[k]);
    if (weight && lane == 0) {
        wsh[0][threadIdx.x >> 5] = lwc;
        wsh[1][threadIdx.x >> 5] = lw;
    }
    __syncthreads();
    if (threadIdx.x < S_N && blk[threadIdx.x])
        atomicAdd(&sums[threadIdx.x], (unsigned long long)blk[threadIdx.x]);
    if (weight && threadIdx.x == 0) {
        // the block's weighted sums, its warps in order; every block writes
        // its slot (zero when it had no point)
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a = __dadd_rn(a, wsh[0][k]);
            b = __dadd_rn(b, wsh[1][k]);
        }
        wpart[blockIdx.x] = a;
        wpart[kVarMaxBlocks + blockIdx.x] = b;
    }
}

// Sum of the blocks' weighted partials in a fixed order: lane l adds blocks
// l, l + 32, ... in turn, then a fixed butterfly over the lanes.  One warp.
__global__ void k_wsum_finish(const double* __restrict__ wpart, int nblocks, double* out /*[2]*/)
{
    const int lane = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int k = lane; k < nblocks; k += 32) {
        a = __dadd_rn(a, wpart[k]);
        b = __dadd_rn(b, wpart[kVarMaxBlocks + k]);
    }
    for (int off = 16; off; off >>= 1) {
        a = __dadd_rn(a, __shfl_xor_sync(0xFFFFFFFFu, a, off));
        b = __dadd_rn(b, __shfl_xor_sync(0xFFFFFFFFu, b, off));
    }
    if (lane == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// Per-direction visible weight: sum over points where direction j is
// visible of w_i (1 for unit weights).  One warp per (word, chunk of
// points), lane = bit; each warp adds its FP64 chunk sum atomically.  With
// unit weights every sum is an integer below 2^53, so the result is exact
// in any order; with real weights the order of the additions is not fixed
// (relative differences of order 1e-16 between runs).
constexpr int kDirChunk = 512;

__global__ void k_dir_hist(const uint32_t* __restrict__ bits, int64_t n, int W, int n_dirs,
                           const double* __restrict__ weight, double* dir_area)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nchunks = (n + kDirChunk - 1) / kDirChunk;
    if (wid >= nchunks * W) return;
    const int w = (int)(wid % W);
    const int64_t c = wid / W;
    double s = 0.0;
    const int64_t e = min64(n, (c + 1) * kDirChunk);
    for (int64_t i = c * kDirChunk; i < e; ++i) {
        const uint32_t word = __ldg(&bits[i * W + w]);
        if ((word >> lane) & 1u) s = __dadd_rn(s, weight ? weight[i] : 1.0);
    }
    const int j = 32 * w + lane;
    if (s != 0.0 && j < n_dirs) atomicAdd(&dir_area[j], s);
}

// Fixture faces: all three vertices within tol of one frame bounding-box
// plane and the normal pointing out through it to within 1e-6.
__global__ void k_fixture(const float* __restrict__ V, const int32_t* __restrict__ F,
                          const float* __restrict__ fnorm, int64_t T, const double* __restrict__ frame,
                          const double* __restrict__ fbox, uint8_t* fixture)
{
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    const double d0 = __dsub_rn(fbox[3], fbox[0]), d1 = __dsub_rn(fbox[4], fbox[1]), d2 = __dsub_rn(fbox[5], fbox[2]);
    const double diag = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
    const double tol = __dmul_rn(1e-6, diag);
    const double lim = 1.0 - 1e-6;
    // fp32 pre-check.  The frame entries are fp32 values, so the fp32 frame
    // coordinate q of a vertex (three rounded operations) is within 3 u s of
    // the exact one, s = sum |V_i f_i|, and the fp32 plane within u |plane|
    // of the FP64 one; a vertex farther than tol + 4 u (s + |plane|) from a
    // plane in fp32 is farther than tol in FP64 (whose own error is far
    // smaller), and the FP64 test of that plane is skipped
    const float u4 = 4.0f * 5.9604644775390625e-8f;
    const float tolf = (float)tol;
    bool fx = false;
    for (int k = 0; k < 3; ++k) {
        const float f0 = (float)frame[k], f1 = (float)frame[3 + k], f2 = (float)frame[6 + k];
        const float blo = (float)fbox[k], bhi = (float)fbox[3 + k];
        bool near_lo = true, near_hi = true;
        for (int a = 0; a < 3; ++a) {
            const int64_t v = F[3 * f + a];
            const float x = V[3 * v], y = V[3 * v + 1], z = V[3 * v + 2];
            const float q = fmaf(x, f0, fmaf(y, f1, z * f2));
            const float sv = (fabsf(x * f0) + fabsf(y * f1) + fabsf(z * f2)) * 1.01f;
            near_lo &= fabsf(q - blo) <= tolf + u4 * (sv + fabsf(blo));
            near_hi &= fabsf(q - bhi) <= tolf + u4 * (sv + fabsf(bhi));
        }
        if (!near_lo && !near_hi) continue;
        bool hi_all = true, lo_all = true;
        for (int a = 0; a < 3; ++a) {
            const int64_t v = F[3 * f + a];
            double q = __dadd_rn(__dmul_rn((double)V[3 * v], frame[k]), __dmul_rn((double)V[3 * v + 1], frame[3 + k]));
            q = __dadd_rn(q, __dmul_rn((double)V[3 * v + 2], frame[6 + k]));
            hi_all &= fabs(__dsub_rn(q, fbox[3 + k])) <= tol;
            lo_all &= fabs(__dsub_rn(q, fbox[k])) <= tol;
        }
        double nq = __dadd_rn(__dmul_rn((double)fnorm[3 * f], frame[k]), __dmul_rn((double)fnorm[3 * f + 1], frame[3 + k]));
        nq = __dadd_rn(nq, __dmul_rn((double)fnorm[3 * f + 2], frame[6 + k]));
        fx |= (hi_all && nq >= lim) || (lo_all && nq <= -lim);
    }
    fixture[f] = fx ? 1 : 0;
}

// Face classes and the 64-bin histogram of viable reachable masks.
__global__ void k_classes(const uint8_t* __restrict__ mask, const float* __restrict__ travel,
                          const int32_t* __restrict__ face, const uint8_t* __restrict__ fixture, int64_t T, int64_t n,
                          float tool_length, uint8_t* cls_out, unsigned long long* hist /*64 + 4*/)
{
    __shared__ unsigned int h[68];
    for (int k = threadIdx.x; k < 68; k += blockDim.x) h[k] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned m = mask[i];
        unsigned reach = 0;
        for (int a = 0; a < 6; ++a)
            if (((m >> a) & 1u) && travel[6 * i + a] <= tool_length) reach |= 1u << a;
        unsigned c = reach ? 0u : (m ? 1u : 2u);
        const int32_t fi = face[i];
        if (fi >= 0 && fi < T && fixture[fi]) c = 3u;
        if (cls_out) cls_out[i] = (uint8_t)c;
        atomicAdd(&h[64 + c], 1u);
        if (c == 0u) atomicAdd(&h[reach], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 68; k += blockDim.x)
        if (h[k]) atomicAdd(&hist[k], (unsigned long long)h[k]);
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
rc_status launch_variability(const uint32_t* bits, const float* N, const double* weight, int64_t n,
                             const float4* dirs, const rc_params* p, float* acc, int8_t* dom, float* conc,
                             double* dir_area, void* scratch, cudaStream_t s)
{
    const int nd = p->n_dirs;
    unsigned long long* sums = (unsigned long long*)scratch;
    double* wsum = (double*)((char*)scratch + kVarWsumOffset);
    double* wpart = (double*)((char*)scratch + kVarPartOffset);
    RC_CUDA(cudaMemsetAsync(scratch, 0, kVarWsumOffset + 2 * sizeof(double), s));
    if (n > 0) {
        int sm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        int64_t blocks = (n + 7) / 8;
        if (blocks > (int64_t)sm * 8) blocks = (int64_t)sm * 8;
        if (blocks > kVarMaxBlocks) blocks = kVarMaxBlocks;
        k_variability<<<(unsigned)blocks, 256, 0, s>>>(bits, N, weight, n, dirs, nd, p->conc_mode, acc, dom, conc,
                                                       sums, wpart);
        RC_LAUNCHED();
        if (weight) {
            k_wsum_finish<<<1, 32, 0, s>>>(wpart, (int)blocks, wsum);
            RC_LAUNCHED();
        }
    }
    if (dir_area) {
        RC_CUDA(cudaMemsetAsync(dir_area, 0, sizeof(double) * (size_t)nd, s));
        const int W = (nd + 31) / 32;
        const int64_t warps = ((n + kDirChunk - 1) / kDirChunk) * W;
        if (warps > 0) {
            k_dir_hist<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(bits, n, W, nd, weight, dir_area);
            RC_LAUNCHED();
        }
    }
    return RC_OK;
}

void fill_summary(const long long* sums, const double* wsum, int64_t n, int32_t n_dirs, bool weighted,
                  rc_summary* out)
{
    rc_summary& o = *out;
    memset(&o, 0, sizeof o);
    const long long counted = sums[S_COUNTED];
    o.n_points = n;
    o.n_counted = counted;
    o.n_zero_visible = n - counted;
    for (int k = 0; k < 3; ++k) {
        o.dom_count[k] = sums[S_DOM + k];
        o.axis_share[k] = counted ? (double)sums[S_DOM + k] / (double)counted : 0.0;
    }
    o.count_sum = sums[S_COUNT];
    o.conc_sum_q = sums[S_CONC];
    if (weighted) {
        o.weighted_count = wsum[0];
        o.weight_sum = wsum[1];
    } else {
        o.weighted_count = (double)sums[S_COUNT];
        o.weight_sum = (double)n;
    }
    const double den = o.weight_sum * (double)n_dirs;
    o.overall_access = den > 0.0 ? o.weighted_count / den : 0.0;
    o.overall_access_unweighted = n ? (double)sums[S_COUNT] / ((double)n * (double)n_dirs) : 0.0;
    o.mean_conc = counted ? (double)sums[S_CONC] / (1099511627776.0 * (double)counted) : 0.0;
}

rc_status launch_classes(rc_bvh h, const uint8_t* mask, const float* travel, const int32_t* face, int64_t n,
                         const rc_params* p, uint8_t* cls, const double* frame_d, const double* fbox_d,
                         uint8_t* fixture, unsigned long long* hist, cudaStream_t s)
{
    k_fixture<<<(unsigned)((h->T + 255) / 256), 256, 0, s>>>(h->V, h->F, h->fnorm, h->T, frame_d, fbox_d, fixture);
    RC_LAUNCHED();
    if (n > 0) {
        int64_t blocks = (n + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        k_classes<<<(unsigned)blocks, 256, 0, s>>>(mask, travel, face, fixture, h->T, n, p->tool_length, cls, hist);
        RC_LAUNCHED();
    }
    return RC_OK;
}

}  // namespace rc
