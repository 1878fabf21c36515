// build.cu -- device construction of the part's acceleration structure and
// the per-face data of Section 3.1 (normal, area, centroid), plus sampling.
//
// Pipeline (one stream):
//   face_prep   : FP64 normal / area / centroid per face, fp32 face boxes,
//                 mesh validation, scene bounds (atomics)
//   morton      : 48-bit Morton code of each face-box centre (16 bits per axis)
//   radix sort  : 6 passes of 8-bit LSD (histogram / scan / stable scatter)
//   karras      : binary radix tree over the sorted codes (Karras, HPG 2012)
//   refit       : bottom-up boxes with arrival counters
//   pack        : BVH2 nodes holding both child boxes (64 B), leaves of up
//                 to kLeafMax consecutive triangles, triangle records 48 B
//   wide        : top-down collapse into 4-wide nodes (128 B): the top
//                 levels one launch each, the subtrees below depth-first
//   area cdf    : 2^32-quantised face areas, inclusive int64 prefix
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rc_internal.cuh"

namespace rc {

// device scratch of a build step, freed in stream order when the scope ends
// (on every path, error returns included)
struct BuildScratch {
    cudaStream_t s;
    void* p[3] = {nullptr, nullptr, nullptr};
    ~BuildScratch()
    {
        for (void* q : p)
            if (q) cudaFreeAsync(q, s);
    }
};


// ---------------------------------------------------------------------------
// face preparation and validation
// ---------------------------------------------------------------------------
__global__ void k_face_prep(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ F,
                            int64_t T, float* fnorm, double* farea, float* tbox, DevScalars* sc)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // contributions to the scene bounds, reduced over the warp before the
    // atomics (one set per warp instead of per face); neutral when absent
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    float mabs = 0.0f;
    double amax = 0.0;
    if (f < T) {
        int32_t id[3];
        bool bad = false;
        for (int k = 0; k < 3; ++k) {
            id[k] = F[3 * f + k];
            if (id[k] < 0 || id[k] >= nV) bad = true;
        }
        if (bad) {
            atomicMin(&sc->err_index, (int)f);
            for (int k = 0; k < 6; ++k) tbox[6 * f + k] = 0.0f;
        } else {
            float v[3][3];
            for (int a = 0; a < 3; ++a) {
                for (int k = 0; k < 3; ++k) {
                    v[a][k] = V[3 * (int64_t)id[a] + k];
                    if (!isfinite(v[a][k])) {
                        atomicMin(&sc->err_vertex, id[a]);
                        v[a][k] = 0.0f;
                    }
                    mabs = fmaxf(mabs, fabsf(v[a][k]));
                }
            }
            // c = (B - A) x (C - A) in FP64, each operation rounded separately
            double e1[3], e2[3];
            for (int k = 0; k < 3; ++k) {
                e1[k] = __dsub_rn((double)v[1][k], (double)v[0][k]);
                e2[k] = __dsub_rn((double)v[2][k], (double)v[0][k]);
            }
            const double c0 = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
            const double c1 = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
            const double c2 = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
            const double len =
                __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(c0, c0), __dmul_rn(c1, c1)), __dmul_rn(c2, c2)));
            farea[f] = 0.5 * len;
            amax = 0.5 * len;
            float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
            if (len > 0.0) {
                n0 = __double2float_rn(__ddiv_rn(c0, len));
                n1 = __double2float_rn(__ddiv_rn(c1, len));
                n2 = __double2float_rn(__ddiv_rn(c2, len));
            }
            fnorm[3 * f + 0] = n0;
            fnorm[3 * f + 1] = n1;
            fnorm[3 * f + 2] = n2;
            for (int k = 0; k < 3; ++k) {
                const float lo = fminf(v[0][k], fminf(v[1][k], v[2][k]));
                const float hi = fmaxf(v[0][k], fmaxf(v[1][k], v[2][k]));
                tbox[6 * f + k] = lo;
                tbox[6 * f + 3 + k] = hi;
                const float c = 0.5f * (lo + hi);
                cmin[k] = c;
                cmax[k] = c;
            }
        }
    }
    const unsigned FULL = 0xFFFFFFFFu;
    for (int off = 16; off; off >>= 1) {
        for (int k = 0; k < 3; ++k) {
            cmin[k] = fminf(cmin[k], __shfl_xor_sync(FULL, cmin[k], off));
            cmax[k] = fmaxf(cmax[k], __shfl_xor_sync(FULL, cmax[k], off));
        }
        mabs = fmaxf(mabs, __shfl_xor_sync(FULL, mabs, off));
        amax = fmax(amax, __shfl_xor_sync(FULL, amax, off));
    }
    if ((threadIdx.x & 31) == 0 && cmin[0] <= cmax[0]) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&sc->cmin[k], float_to_ordered(cmin[k]));
            atomicMax(&sc->cmax[k], float_to_ordered(cmax[k]));
        }
        atomicMax(&sc->vmaxabs, float_to_ordered(mabs));
        atomicMax(&sc->amax_bits, (unsigned long long)__double_as_longlong(amax));
    }
}

// ---------------------------------------------------------------------------
// Morton codes
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long spread21(unsigned long long x)
{
    x &= 0x1FFFFFULL;
    x = (x | (x << 32)) & 0x1F00000000FFFFULL;
    x = (x | (x << 16)) & 0x1F0000FF0000FFULL;
    x = (x | (x << 8)) & 0x100F00F00F00F00FULL;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

// Morton code of each face-box centre, kMortonBits per axis (interleaved
// x, y, z from the top); the radix sort then needs kMortonPasses byte passes
#ifndef RC_MORTON_BITS
#define RC_MORTON_BITS 16
#endif
constexpr int kMortonBits = RC_MORTON_BITS;
constexpr int kMortonPasses = (3 * kMortonBits + 7) / 8;
static_assert(kMortonBits >= 8 && kMortonBits <= 21, "Morton bits per axis out of range");
static_assert(kMortonPasses % 2 == 0, "an even number of sort passes leaves the result in place");

__global__ void k_morton(const float* __restrict__ tbox, int64_t T, const DevScalars* sc,
                         unsigned long long* keys, int32_t* vals)
{
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    unsigned long long code = 0;
    for (int k = 0; k < 3; ++k) {
        float lo = ordered_to_float(sc->cmin[k]);
        float hi = ordered_to_float(sc->cmax[k]);
        float c = 0.5f * (tbox[6 * f + k] + tbox[6 * f + 3 + k]);
        float ext = hi - lo;
        float u = ext > 0.0f ? (c - lo) / ext : 0.0f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        const float cells = (float)(1 << kMortonBits);
        unsigned long long q = (unsigned long long)fminf(u * cells, cells - 1.0f);
        code |= spread21(q) << (2 - k);
    }
    keys[f] = code;
    vals[f] = (int32_t)f;
}

// ---------------------------------------------------------------------------
// LSD radix sort of (uint64 key, int32 value), 8-bit digits, stable
// ---------------------------------------------------------------------------
constexpr int kMaxWalk = 4096;   // bound on leaf-to-root walks
constexpr int kSortThreads = 256;
constexpr int kSortTile = 4096;   // most keys per block

__global__ void k_sort_hist(const unsigned long long* __restrict__ keys, int64_t T, int shift, int tile,
                            int nblk, unsigned int* __restrict__ counts)
{
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * tile;
    int64_t end = min64(T, base + tile);
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) counts[(int64_t)i * nblk + blockIdx.x] = h[i];
}

__device__ __forceinline__ unsigned int warp_incl_scan(unsigned int v, int lane)
{
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned int u = __shfl_up_sync(0xFFFFFFFFu, v, off);
        if (lane >= off) v += u;
    }
    return v;
}

// per digit, the exclusive prefix of its counts over the blocks (in place,
// digit-major layout counts[d * nblk + b]) and the digit's total; one warp
// per digit, 32 counts per step
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned int* __restrict__ counts, int nblk,
                                                    unsigned int* __restrict__ totals)
{
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (d >= 256) return;
    unsigned int* c = counts + (int64_t)d * nblk;
    unsigned int carry = 0;
    for (int b = 0; b < nblk; b += 32) {
        const int i = b + lane;
        const unsigned int v = i < nblk ? c[i] : 0u;
        const unsigned int inc = warp_incl_scan(v, lane);
        if (i < nblk) c[i] = carry + inc - v;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    if (lane == 0) totals[d] = carry;
}

__global__ void k_sort_scatter(const unsigned long long* __restrict__ kin, const int32_t* __restrict__ vin,
                               int64_t T, int shift, int tile, int nblk, const unsigned int* __restrict__ offs,
                               const unsigned int* __restrict__ totals, unsigned long long* __restrict__ kout,
                               int32_t* __restrict__ vout, unsigned int* err)
{
    constexpr int W = kSortThreads / 32;
    static_assert(kSortThreads == 256, "one thread per digit");
    __shared__ unsigned int base[256];
    __shared__ unsigned int wcnt[W][256];
    __shared__ unsigned int wsum[W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the digit's start = the totals of the smaller digits (a block scan of
    // the 256 totals) + this digit's count in the blocks before this one
    {
        const unsigned int t = totals[threadIdx.x];
        const unsigned int inc = warp_incl_scan(t, lane);
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        unsigned int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        base[threadIdx.x] = before + inc - t + offs[(int64_t)threadIdx.x * nblk + blockIdx.x];
    }
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * tile;
    const int64_t e0 = min64(T, b0 + tile);
    for (int64_t c0 = b0; c0 < e0; c0 += kSortThreads) {
        for (int i = threadIdx.x; i < W * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = c0 + threadIdx.x;
        const bool ok = i < e0;
        unsigned long long key = ok ? kin[i] : 0ULL;
        int32_t val = ok ? vin[i] : 0;
        const unsigned int dig = ok ? (unsigned int)((key >> shift) & 255) : 256u + lane;
        const unsigned int peers = __match_any_sync(0xFFFFFFFFu, dig);
        const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        if (ok) {
            unsigned int pos = base[dig] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][dig];
            if (pos < (unsigned long long)T) {
                kout[pos] = key;
                vout[pos] = val;
            } else {
                atomicAdd(err, 1u);
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) {
            unsigned int s = 0;
            for (int w = 0; w < W; ++w) s += wcnt[w][d];
            base[d] += s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Karras binary radix tree
// ---------------------------------------------------------------------------
__device__ __forceinline__ int kdelta(const unsigned long long* keys, int64_t T, int64_t i, int64_t j)
{
    if (j < 0 || j >= T) return -1;
    unsigned long long a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((unsigned int)(i ^ j));
    return __clzll(a ^ b);
}

__global__ void k_karras(const unsigned long long* __restrict__ keys, int64_t T, int32_t* child,
                         int32_t* range, int32_t* parent)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n_int = T - 1;
    if (i >= n_int) return;
    const int d = (kdelta(keys, T, i, i + 1) - kdelta(keys, T, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = kdelta(keys, T, i, i - d);
    int64_t lmax = 2;
    while (kdelta(keys, T, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (kdelta(keys, T, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = kdelta(keys, T, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(keys, T, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    const int32_t left = (int32_t)(lo == gamma ? n_int + gamma : gamma);
    const int32_t right = (int32_t)(hi == gamma + 1 ? n_int + gamma + 1 : gamma + 1);
    child[2 * i] = left;
    child[2 * i + 1] = right;
    range[2 * i] = (int32_t)lo;
    range[2 * i + 1] = (int32_t)hi;
    parent[left] = (int32_t)i;
    parent[right] = (int32_t)i;
    if (i == 0) parent[0] = -1;
}

// ---------------------------------------------------------------------------
// PLOC (Meister and Bittner, "Parallel Locally-Ordered Clustering for
// Bounding Volume Hierarchy Construction", IEEE TVCG 2018): clusters start as
// the Morton-ordered leaves; each round every cluster finds, within kPlocR
// positions, the cluster whose merged box has the smallest surface area;
// mutual nearest neighbours merge into a new interior node (at the lower
// position) and the array is compacted in order.  Raw interior ids come from
// an atomic counter; the tree is then renumbered in depth-first order (root
// 0, each subtree's leaves contiguous) so that packing, the 4-wide collapse
// and refit work on it as on the Karras tree.
// ---------------------------------------------------------------------------
constexpr int kPlocR = 16;
constexpr int kPlocThreads = 256;

__device__ __forceinline__ float merged_area(const float* a, const float* b)
{
    const float dx = fmaxf(a[3], b[3]) - fminf(a[0], b[0]);
    const float dy = fmaxf(a[4], b[4]) - fminf(a[1], b[1]);
    const float dz = fmaxf(a[5], b[5]) - fminf(a[2], b[2]);
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_ploc_init(const float* __restrict__ tbox, const int32_t* __restrict__ order, int64_t T,
                            int64_t n_int, int32_t* cl, float* cb, int* n_ptr)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k == 0) *n_ptr = (int)T;
    if (k >= T) return;
    cl[k] = (int32_t)(n_int + k);
    const int32_t f = order[k];
    for (int c = 0; c < 6; ++c) cb[6 * k + c] = tbox[6 * (int64_t)f + c];
}

__global__ void __launch_bounds__(kPlocThreads)
k_ploc_nn(const int* __restrict__ n_ptr, const float* __restrict__ cb, int32_t* __restrict__ nn)
{
    __shared__ float sb[kPlocThreads + 2 * kPlocR][6];
    const int n = *n_ptr;
    const int base = blockIdx.x * kPlocThreads;
    if (base >= n) return;
    for (int t = threadIdx.x; t < kPlocThreads + 2 * kPlocR; t += blockDim.x) {
        const int j = base - kPlocR + t;
        if (j >= 0 && j < n)
            for (int c = 0; c < 6; ++c) sb[t][c] = cb[6 * (int64_t)j + c];
    }
    __syncthreads();
    const int i = base + threadIdx.x;
    if (i >= n) return;
    const float* bi = sb[threadIdx.x + kPlocR];
    int best = -1;
    float ba = INFINITY;
    const int j0 = max(0, i - kPlocR), j1 = min(n - 1, i + kPlocR);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        const float a = merged_area(bi, sb[j - base + kPlocR]);
        if (a < ba) { ba = a; best = j; }          // ascending j: ties go to the lower position
    }
    nn[i] = best;
}

__global__ void k_ploc_merge(const int* __restrict__ n_ptr, const int32_t* __restrict__ nn,
                             const int32_t* __restrict__ cl, const float* __restrict__ cb, int32_t* cl_tmp,
                             float* cb_tmp, int* keep, int32_t* child_raw, int32_t* parent_raw, int* counter,
                             int64_t n_int)
{
    const int n = *n_ptr;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = nn[i];
    if (j >= 0 && nn[j] == i) {
        if (i > j) { keep[i] = 0; return; }        // merged into its partner
        const int id = atomicAdd(counter, 1);
        if (id >= n_int) { keep[i] = 0; return; }  // cannot happen for a valid cluster array
        const int32_t a = cl[i], b = cl[j];
        child_raw[2 * id] = a;
        child_raw[2 * id + 1] = b;
        parent_raw[a] = id;
        parent_raw[b] = id;
        for (int c = 0; c < 3; ++c) {
            cb_tmp[6 * (int64_t)i + c] = fminf(cb[6 * (int64_t)i + c], cb[6 * (int64_t)j + c]);
            cb_tmp[6 * (int64_t)i + 3 + c] = fmaxf(cb[6 * (int64_t)i + 3 + c], cb[6 * (int64_t)j + 3 + c]);
        }
        cl_tmp[i] = id;
    } else {
        cl_tmp[i] = cl[i];
        for (int c = 0; c < 6; ++c) cb_tmp[6 * (int64_t)i + c] = cb[6 * (int64_t)i + c];
    }
    keep[i] = 1;
}

// order-preserving compaction of the kept clusters: per-block counts, one
// block scanning them (it also writes the new count), then the scatter
constexpr int kCompact = 1024;

__global__ void k_ploc_count(const int* __restrict__ n_ptr, const int* __restrict__ keep, int* bsum)
{
    __shared__ int warp_tot[kCompact / 32];
    const int n = *n_ptr;
    const int i = blockIdx.x * kCompact + threadIdx.x;
    const int v = i < n ? keep[i] : 0;
    const int c = __popc(__ballot_sync(0xFFFFFFFFu, v));
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kCompact / 32; ++w) t += warp_tot[w];
        bsum[blockIdx.x] = t;
    }
}

__global__ void k_ploc_scan(int* bsum, int nb, const int* __restrict__ n_ptr, int* n_next)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = *n_ptr;
    const int used = (n + kCompact - 1) / kCompact;
    int run = 0;
    for (int b = 0; b < nb && b < used; ++b) {
        const int v = bsum[b];
        bsum[b] = run;
        run += v;
    }
    *n_next = run;
}

__global__ void k_ploc_scatter(const int* __restrict__ n_ptr, const int* __restrict__ keep,
                               const int* __restrict__ bsum, const int32_t* __restrict__ cl_tmp,
                               const float* __restrict__ cb_tmp, int32_t* cl_out, float* cb_out)
{
    __shared__ int warp_pre[kCompact / 32];
    const int n = *n_ptr;
    const int i = blockIdx.x * kCompact + threadIdx.x;
    const int v = i < n ? keep[i] : 0;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_pre[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < kCompact / 32; ++k) {
            const int c = warp_pre[k];
            warp_pre[k] = run;
            run += c;
        }
    }
    __syncthreads();
    if (!v) return;
    const int pos = bsum[blockIdx.x] + warp_pre[w] + __popc(bal & ((1u << lane) - 1u));
    cl_out[pos] = cl_tmp[i];
    for (int c = 0; c < 6; ++c) cb_out[6 * (int64_t)pos + c] = cb_tmp[6 * (int64_t)i + c];
}

// subtree sizes (leaves, interior nodes) bottom-up with arrival counters;
// sizes of raw interior id p at sz_leaf[p], sz_int[p]
__global__ void k_ploc_sizes(int64_t T, int64_t n_int, const int32_t* __restrict__ parent_raw,
                             const int32_t* __restrict__ child_raw, int32_t* sz_leaf, int32_t* sz_int, int32_t* visits,
                             int* err)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    int32_t p = parent_raw[n_int + k];
    for (int steps = 0; p >= 0; ++steps) {
        if (steps > kMaxWalk) { atomicExch(err, 1); return; }
        __threadfence();
        if (atomicAdd(&visits[p], 1) == 0) return;
        const int32_t a = child_raw[2 * p], b = child_raw[2 * p + 1];
        const int la = a >= n_int ? 1 : __ldcg(&sz_leaf[a]), lb = b >= n_int ? 1 : __ldcg(&sz_leaf[b]);
        const int ia = a >= n_int ? 0 : __ldcg(&sz_int[a]), ib = b >= n_int ? 0 : __ldcg(&sz_int[b]);
        __stcg(&sz_leaf[p], la + lb);
        __stcg(&sz_int[p], ia + ib + 1);
        p = parent_raw[p];
    }
}

// depth-first numbering: every node walks to the root adding, for each
// ancestor whose right subtree it is in, the sizes of the left sibling
// subtree.  Interior raw id p -> preorder index newid[p]; leaf k -> leaf
// position pos[k] (a subtree's leaves are contiguous in that order).
__global__ void k_ploc_number(int64_t T, int64_t n_int, const int32_t* __restrict__ parent_raw,
                              const int32_t* __restrict__ child_raw, const int32_t* __restrict__ sz_leaf,
                              const int32_t* __restrict__ sz_int, int32_t* newid, int32_t* leafstart,
                              int32_t* pos, int* err)
{
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= n_int + T) return;
    int pre = x < n_int ? 0 : 0, lstart = 0;
    int32_t cur = (int32_t)x;
    int steps = 0;
    for (int32_t p = parent_raw[cur]; p >= 0; cur = p, p = parent_raw[p]) {
        if (++steps > kMaxWalk) { atomicExch(err, 1); return; }
        const int32_t left = child_raw[2 * p];
        pre += 1;                                   // the parent comes first
        if (cur != left) {
            pre += left >= n_int ? 0 : sz_int[left];
            lstart += left >= n_int ? 1 : sz_leaf[left];
        }
    }
    if (x < n_int) {
        newid[x] = pre;
        leafstart[x] = lstart;
    } else {
        pos[x - n_int] = lstart;
    }
}

// the renumbered tree: child / parent in combined indexing (interior
// preorder ids, leaf n_int + position), ranges, and the leaf order
__global__ void k_ploc_emit(int64_t T, int64_t n_int, const int32_t* __restrict__ parent_raw,
                            const int32_t* __restrict__ child_raw, const int32_t* __restrict__ newid,
                            const int32_t* __restrict__ leafstart, const int32_t* __restrict__ sz_leaf,
                            const int32_t* __restrict__ pos, const int32_t* __restrict__ order_in, int32_t* child,
                            int32_t* range, int32_t* parent, int32_t* order_out)
{
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= n_int + T) return;
    auto map = [&](int32_t c) -> int32_t { return c >= n_int ? (int32_t)(n_int + pos[c - n_int]) : newid[c]; };
    const int32_t p = parent_raw[x];
    const int32_t me = map((int32_t)x);
    parent[me] = p >= 0 ? newid[p] : -1;
    if (x < n_int) {
        child[2 * me] = map(child_raw[2 * x]);
        child[2 * me + 1] = map(child_raw[2 * x + 1]);
        range[2 * me] = leafstart[x];
        range[2 * me + 1] = leafstart[x] + sz_leaf[x] - 1;
    } else {
        order_out[pos[x - n_int]] = order_in[x - n_int];
    }
}

// ---------------------------------------------------------------------------
// bottom-up refit
// ---------------------------------------------------------------------------
__global__ void k_leaf_boxes(const float* __restrict__ tbox, const int32_t* __restrict__ order,
                             int64_t T, int64_t n_int, float* nbox)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    const int32_t f = order[k];
    for (int c = 0; c < 6; ++c) nbox[6 * (n_int + k) + c] = f >= 0 && f < T ? tbox[6 * (int64_t)f + c] : 0.0f;
}

__global__ void k_refit(int64_t T, int64_t n_int, const int32_t* __restrict__ parent,
                        const int32_t* __restrict__ child, float* nbox, int32_t* visits, DevScalars* sc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t cur = (int32_t)(n_int + k);
    // every chain ends at the root; the caps only guard against a malformed
    // tree (the build then reports an error instead of looping)
    int depth = 0;
    if (k < T)
        for (int32_t p = parent[cur]; p >= 0 && depth <= kMaxWalk; p = parent[p]) ++depth;
    int wmax = depth;                               // one atomic per warp
    for (int off = 16; off; off >>= 1) wmax = max(wmax, __shfl_xor_sync(0xFFFFFFFFu, wmax, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&sc->max_depth, wmax);
    if (k >= T || depth > kMaxWalk) return;
    int32_t p = parent[cur];
    for (int steps = 0; p >= 0 && steps <= kMaxWalk; ++steps) {
        __threadfence();
        if (atomicAdd(&visits[p], 1) == 0) return;   // first arrival stops
        const int32_t a = child[2 * p], b = child[2 * p + 1];
        float box[6];
        for (int c = 0; c < 3; ++c) {
            box[c] = fminf(__ldcg(&nbox[6 * (int64_t)a + c]), __ldcg(&nbox[6 * (int64_t)b + c]));
            box[3 + c] = fmaxf(__ldcg(&nbox[6 * (int64_t)a + 3 + c]), __ldcg(&nbox[6 * (int64_t)b + 3 + c]));
        }
        for (int c = 0; c < 6; ++c) __stcg(&nbox[6 * (int64_t)p + c], box[c]);
        p = parent[p];
    }
}

// ---------------------------------------------------------------------------
// packing into the traversal layout
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t encode_child(int32_t c, int64_t n_int, const int32_t* range)
{
    if (c >= n_int) {
        const int32_t first = (int32_t)(c - n_int);
        return -1 - (first * 8 + 0);
    }
    const int32_t lo = range[2 * c], hi = range[2 * c + 1];
    const int32_t cnt = hi - lo + 1;
    if (cnt <= kLeafMax) return -1 - (lo * 8 + (cnt - 1));
    return c;
}

__global__ void k_pack(int64_t n_int, const int32_t* __restrict__ child, const int32_t* __restrict__ range,
                       const float* __restrict__ nbox, float4* nodes)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const int32_t a = child[2 * i], b = child[2 * i + 1];
    const float* A = nbox + 6 * (int64_t)a;
    const float* B = nbox + 6 * (int64_t)b;
    nodes[4 * i + 0] = make_float4(A[0], A[3], A[1], A[4]);
    nodes[4 * i + 1] = make_float4(B[0], B[3], B[1], B[4]);
    nodes[4 * i + 2] = make_float4(A[2], A[5], B[2], B[5]);
    nodes[4 * i + 3] = make_float4(__int_as_float(encode_child(a, n_int, range)),
                                   __int_as_float(encode_child(b, n_int, range)), 0.0f, 0.0f);
}

// ---------------------------------------------------------------------------
// 4-wide tree: top-down collapse of the binary tree, one level per launch.
// A wide node starts from a binary interior node's two children and keeps
// replacing its interior child of largest box surface area by that child's
// two children until it has four children or only leaves.  Wide node layout
// (8 float4, 128 B): lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the four
// children, then the four child indices (>= 0 wide node, < 0 leaf as in the
// binary layout), then padding.  Empty slots have an empty box.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool bin_is_leaf(int32_t c, int64_t n_int, const int32_t* range)
{
    return c >= n_int || range[2 * c + 1] - range[2 * c] + 1 <= kLeafMax;
}

__device__ __forceinline__ float half_area(const float* b)
{
    const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return dx * dy + dy * dz + dz * dx;
}

// the children of the wide node made from binary interior node b: start
// from b's two children and keep replacing the interior child of largest box
// surface area by its two children until there are four or only leaves
__device__ __forceinline__ int wide_children(int32_t b, int64_t n_int, const int32_t* __restrict__ child,
                                             const int32_t* __restrict__ range, const float* __restrict__ nbox,
                                             int32_t ch[4])
{
    int nch = 2;
    ch[0] = child[2 * b];
    ch[1] = child[2 * b + 1];
    while (nch < 4) {
        int best = -1;
        float ba = -1.0f;
        for (int k = 0; k < nch; ++k) {
            if (bin_is_leaf(ch[k], n_int, range)) continue;
            const float a = half_area(nbox + 6 * (int64_t)ch[k]);
            if (a > ba) { ba = a; best = k; }
        }
        if (best < 0) break;
        const int32_t c = ch[best];
        ch[best] = child[2 * c];
        ch[nch++] = child[2 * c + 1];
    }
    return nch;
}

// write wide node w: the boxes of its nch children and their indices idx
// (wide node >= 0, leaf < 0); empty slots get an empty box and index -1
__device__ __forceinline__ void wide_write(float4* wnodes, int32_t w, const float* __restrict__ nbox,
                                           const int32_t ch[4], const int32_t idx[4], int nch)
{
    float lo[3][4], hi[3][4];
    int32_t ix[4];
    for (int k = 0; k < 4; ++k) {
        if (k < nch) {
            const float* bb = nbox + 6 * (int64_t)ch[k];
            for (int a = 0; a < 3; ++a) { lo[a][k] = bb[a]; hi[a][k] = bb[3 + a]; }
            ix[k] = idx[k];
        } else {
            for (int a = 0; a < 3; ++a) { lo[a][k] = INFINITY; hi[a][k] = -INFINITY; }
            ix[k] = -1;
        }
    }
    float4* nd = wnodes + 8 * (int64_t)w;
    nd[0] = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
    nd[1] = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
    nd[2] = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
    nd[3] = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
    nd[4] = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
    nd[5] = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
    nd[6] = make_float4(__int_as_float(ix[0]), __int_as_float(ix[1]), __int_as_float(ix[2]), __int_as_float(ix[3]));
    // the binary nodes the children were made from (-1: empty slot), for
    // the boxes of the same tree in another coordinate frame
    nd[7] = make_float4(__int_as_float(nch > 0 ? ch[0] : -1), __int_as_float(nch > 1 ? ch[1] : -1),
                        __int_as_float(nch > 2 ? ch[2] : -1), __int_as_float(nch > 3 ? ch[3] : -1));
}

// one level of the top of the tree: each queued binary node becomes a wide
// node; its interior children go to the next level's queue
__global__ void k_wide_level(int64_t n_int, const int32_t* __restrict__ child, const int32_t* __restrict__ range,
                             const float* __restrict__ nbox, const int32_t* __restrict__ qin_bin,
                             const int32_t* __restrict__ qin_wide, const int* __restrict__ qin_count,
                             int32_t* qout_bin, int32_t* qout_wide, int* qout_count, int* wide_count,
                             float4* wnodes, DevScalars* sc, int level)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *qin_count) return;
    const int32_t b = qin_bin[t], w = qin_wide[t];
    int32_t ch[4], idx[4];
    const int nch = wide_children(b, n_int, child, range, nbox, ch);
    for (int k = 0; k < nch; ++k) {
        if (bin_is_leaf(ch[k], n_int, range)) {
            idx[k] = encode_child(ch[k], n_int, range);
        } else {
            const int nw = atomicAdd(wide_count, 1);
            const int q = atomicAdd(qout_count, 1);
            qout_bin[q] = ch[k];
            qout_wide[q] = nw;
            idx[k] = nw;
        }
    }
    wide_write(wnodes, w, nbox, ch, idx, nch);
    atomicMax(&sc->wide_depth, level + 1);
}

// the rest of the tree: each thread finishes the subtree below one queued
// binary node depth-first, so a subtree's wide nodes are made by one thread
// (numbered with the siblings of a node consecutive).  A subtree deeper than
// the stack reports a wide depth that the host rejects.
constexpr int kWideDfs = 96;
#ifndef RC_WIDE_SUBTREE
#define RC_WIDE_SUBTREE 4.0      // binary nodes per subtree thread (0: one launch per level throughout)
#endif

__global__ void k_wide_subtrees(int64_t n_int, const int32_t* __restrict__ child, const int32_t* __restrict__ range,
                                const float* __restrict__ nbox, const int32_t* __restrict__ qin_bin,
                                const int32_t* __restrict__ qin_wide, const int* __restrict__ qin_count,
                                int* wide_count, float4* wnodes, DevScalars* sc, int level)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *qin_count) return;
    int32_t sb[kWideDfs], sw[kWideDfs];
    uint8_t sd[kWideDfs];
    sb[0] = qin_bin[t];
    sw[0] = qin_wide[t];
    sd[0] = 0;
    int sp = 1, maxd = 0;
    while (sp > 0) {
        --sp;
        const int32_t b = sb[sp], w = sw[sp];
        const int d = sd[sp];
        int32_t ch[4], idx[4];
        const int nch = wide_children(b, n_int, child, range, nbox, ch);
        int ni = 0;
        for (int k = 0; k < nch; ++k) ni += bin_is_leaf(ch[k], n_int, range) ? 0 : 1;
        if (sp + ni > kWideDfs || d + 1 > 250) {
            atomicMax(&sc->wide_depth, kStack4);
            return;
        }
        int nw = ni ? atomicAdd(wide_count, ni) : 0;
        for (int k = 0; k < nch; ++k) idx[k] = bin_is_leaf(ch[k], n_int, range) ? encode_child(ch[k], n_int, range)
                                                                                 : nw++;
        wide_write(wnodes, w, nbox, ch, idx, nch);
        maxd = max(maxd, d + 1);
        for (int k = nch - 1; k >= 0; --k) {     // the first child is taken next
            if (idx[k] < 0) continue;
            sb[sp] = ch[k];
            sw[sp] = idx[k];
            sd[sp] = (uint8_t)(d + 1);
            ++sp;
        }
    }
    atomicMax(&sc->wide_depth, level + maxd);
}

// wide root for parts with at most kLeafMax triangles: one leaf child
__global__ void k_wide_small(int64_t T, const float* __restrict__ tbox, float4* wnodes, DevScalars* sc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t f = 0; f < T; ++f)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], tbox[6 * f + c]);
            hi[c] = fmaxf(hi[c], tbox[6 * f + 3 + c]);
        }
    const float I = INFINITY;
    wnodes[0] = make_float4(lo[0], I, I, I);
    wnodes[1] = make_float4(hi[0], -I, -I, -I);
    wnodes[2] = make_float4(lo[1], I, I, I);
    wnodes[3] = make_float4(hi[1], -I, -I, -I);
    wnodes[4] = make_float4(lo[2], I, I, I);
    wnodes[5] = make_float4(hi[2], -I, -I, -I);
    wnodes[6] = make_float4(__int_as_float(-1 - (int)(T - 1)), __int_as_float(-1), __int_as_float(-1),
                            __int_as_float(-1));
    wnodes[7] = make_float4(__int_as_float(kAllTris), __int_as_float(-1), __int_as_float(-1), __int_as_float(-1));
    sc->wide_depth = 1;
    sc->wide_nodes = 1;
}

__global__ void k_wide_init(int32_t* q_bin, int32_t* q_wide, int* counts)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        q_bin[0] = 0;
        q_wide[0] = 0;
        counts[0] = 1;   // queue A size
        counts[1] = 0;   // queue B size
        counts[2] = 1;   // wide nodes allocated
    }
}

// single-leaf root for parts with at most kLeafMax triangles
__global__ void k_pack_small(int64_t T, const float* __restrict__ tbox, float4* nodes)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t f = 0; f < T; ++f)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], tbox[6 * f + c]);
            hi[c] = fmaxf(hi[c], tbox[6 * f + 3 + c]);
        }
    nodes[0] = make_float4(lo[0], hi[0], lo[1], hi[1]);
    nodes[1] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    nodes[2] = make_float4(lo[2], hi[2], INFINITY, -INFINITY);
    nodes[3] = make_float4(__int_as_float(-1 - (0 * 8 + (int)(T - 1))), __int_as_float(-1), 0.0f, 0.0f);
}

__global__ void k_tri_records(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ F,
                              const int32_t* __restrict__ order, int64_t T, float4* tris)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    const int32_t f = order[k];
    float v[3][3] = {};
    // a bad mesh (reported by the build) must not be gathered out of range
    if (f >= 0 && f < T) {
        for (int a = 0; a < 3; ++a) {
            const int64_t vi = F[3 * (int64_t)f + a];
            if (vi >= 0 && vi < nV)
                for (int c = 0; c < 3; ++c) v[a][c] = V[3 * vi + c];
        }
    }
    float le = 0.0f;
    for (int c = 0; c < 3; ++c) {
        le = fmaxf(le, fabsf(v[1][c] - v[0][c]));
        le = fmaxf(le, fabsf(v[2][c] - v[1][c]));
        le = fmaxf(le, fabsf(v[0][c] - v[2][c]));
    }
    tris[3 * k + 0] = make_float4(v[0][0], v[0][1], v[0][2], le);
    tris[3 * k + 1] = make_float4(v[1][0], v[1][1], v[1][2], __int_as_float(f));
    tris[3 * k + 2] = make_float4(v[2][0], v[2][1], v[2][2], 0.0f);
}

// ---------------------------------------------------------------------------
// area CDF (2^32-quantised areas, inclusive prefix in int64)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;

__global__ void k_quant_area(const double* __restrict__ farea, int64_t T, const DevScalars* sc,
                             long long* q)
{
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    const double amax = __longlong_as_double((long long)sc->amax_bits);
    q[f] = amax > 0.0 ? llround(__dmul_rn(__ddiv_rn(farea[f], amax), 4294967296.0)) : 0LL;
}

// block-wise inclusive scan, writing per-block totals
__global__ void k_scan_block(long long* x, int64_t n, long long* bsum)
{
    __shared__ long long s[kScanBlock];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    s[threadIdx.x] = i < n ? x[i] : 0;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        long long v = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < n) x[i] = s[threadIdx.x];
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(long long* x, int64_t n, const long long* bsum_incl)
{
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i >= n || blockIdx.x == 0) return;
    x[i] += bsum_incl[blockIdx.x - 1];
}

__global__ void k_store_total(const long long* cdf, int64_t T, DevScalars* sc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->total = T > 0 ? cdf[T - 1] : 0;
}

static rc_status scan_inclusive(long long* x, int64_t n, cudaStream_t s)
{
    if (n <= 0) return RC_OK;
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    long long* bs = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&bs, sizeof(long long) * nb, s));
    g.p[0] = bs;
    k_scan_block<<<(unsigned)nb, kScanBlock, 0, s>>>(x, n, bs);
    RC_LAUNCHED();
    if (nb > 1) {
        rc_status st = scan_inclusive(bs, nb, s);
        if (st != RC_OK) return st;
        k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(x, n, bs);
        RC_LAUNCHED();
    }
    return RC_OK;
}

// ---------------------------------------------------------------------------
// sampling (Section 3.1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double uniform01(unsigned long long seed, long long i, int k)
{
    const unsigned long long ctr = (unsigned long long)(3 * i + k) * 0x9E3779B97F4A7C15ULL;
    const unsigned long long r = splitmix64(seed ^ ctr);
    return __dmul_rn(__ull2double_rn(r >> 11), 1.0 / 9007199254740992.0);
}

__global__ void k_sample_area(const float* __restrict__ V, const int32_t* __restrict__ F, int64_t T,
                              const long long* __restrict__ cdf, const DevScalars* sc,
                              const float* __restrict__ fnorm, int64_t n, unsigned long long seed,
                              float* P, float* Nout, int32_t* face, double* weight)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double u0 = uniform01(seed, i, 0), u1 = uniform01(seed, i, 1), u2 = uniform01(seed, i, 2);
    const long long total = sc->total;
    const long long target = (long long)floor(__dmul_rn(u0, __ll2double_rn(total)));
    int64_t lo = 0, hi = T - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    const int64_t f = lo;
    const double s = __dsqrt_rn(u1);
    const double wa = __dsub_rn(1.0, s);
    const double wb = __dmul_rn(s, __dsub_rn(1.0, u2));
    const double wc = __dmul_rn(s, u2);
    for (int k = 0; k < 3; ++k) {
        const double A = V[3 * (int64_t)F[3 * f + 0] + k];
        const double B = V[3 * (int64_t)F[3 * f + 1] + k];
        const double C = V[3 * (int64_t)F[3 * f + 2] + k];
        double p = __dadd_rn(__dmul_rn(wa, A), __dmul_rn(wb, B));
        p = __dadd_rn(p, __dmul_rn(wc, C));
        P[3 * i + k] = __double2float_rn(p);
        Nout[3 * i + k] = fnorm[3 * f + k];
    }
    face[i] = (int32_t)f;
    if (weight) weight[i] = 1.0;
}

__global__ void k_sample_centroid(const float* __restrict__ V, const int32_t* __restrict__ F,
                                  const float* __restrict__ fnorm,
                                  const double* __restrict__ farea, int64_t T, float* P, float* Nout,
                                  int32_t* face, double* weight)
{
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    for (int k = 0; k < 3; ++k) {
        P[3 * f + k] = face_centroid(V, F, f, k);
        Nout[3 * f + k] = fnorm[3 * f + k];
    }
    face[f] = (int32_t)f;
    if (weight) weight[f] = farea[f];
}

// Morton code (10 bits per axis) of each point inside the box [lo, hi]
__global__ void k_point_morton(const float* __restrict__ P, int64_t n, float lx, float ly, float lz, float sx,
                               float sy, float sz, unsigned long long* keys, int32_t* vals)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float lo[3] = {lx, ly, lz}, sc[3] = {sx, sy, sz};
    unsigned long long code = 0;
    for (int k = 0; k < 3; ++k) {
        float u = (P[3 * i + k] - lo[k]) * sc[k];
        u = fminf(fmaxf(u, 0.0f), 1023.0f);
        unsigned long long q = (unsigned long long)u;
        q = (q | (q << 16)) & 0x030000FFULL;
        q = (q | (q << 8)) & 0x0300F00FULL;
        q = (q | (q << 4)) & 0x030C30C3ULL;
        q = (q | (q << 2)) & 0x09249249ULL;
        code |= q << (2 - k);
    }
    keys[i] = code;
    vals[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
static inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Stable LSD sort of (key, value) pairs by the low `passes` bytes of the key;
// the result is back in (keys, vals) when `passes` is even.
static rc_status sort_pairs(unsigned long long* keys, int32_t* vals, int64_t n, int passes, unsigned int* err,
                            cudaStream_t s)
{
    if (n <= 1) return RC_OK;
    unsigned long long* k1 = nullptr;
    int32_t* v1 = nullptr;
    unsigned int* counts = nullptr;
    // about two tiles per SM (a multiple of the block size, 512 to 4096 keys):
    // small sorts spread over the GPU, large ones keep the count table short
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    int64_t tile = (n + 2 * sms - 1) / (2 * sms);
    tile = std::min<int64_t>(kSortTile, std::max<int64_t>(512, (tile + kSortThreads - 1) / kSortThreads * kSortThreads));
    const int nblk = (int)((n + tile - 1) / tile);
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&k1, sizeof(unsigned long long) * n, s));
    g.p[0] = k1;
    RC_CUDA(cudaMallocAsync(&v1, sizeof(int32_t) * n, s));
    g.p[1] = v1;
    RC_CUDA(cudaMallocAsync(&counts, sizeof(unsigned int) * (256 * (size_t)nblk + 256), s));   // counts, then digit totals
    g.p[2] = counts;
    unsigned long long *kin = keys, *kout = k1;
    int32_t *vin = vals, *vout = v1;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_sort_hist<<<nblk, kSortThreads, 0, s>>>(kin, n, shift, (int)tile, nblk, counts);
        RC_LAUNCHED();
        k_sort_scan<<<8, 1024, 0, s>>>(counts, nblk, counts + (int64_t)256 * nblk);
        RC_LAUNCHED();
        k_sort_scatter<<<nblk, kSortThreads, 0, s>>>(kin, vin, n, shift, (int)tile, nblk, counts,
                                                     counts + (int64_t)256 * nblk, kout, vout, err);
        RC_LAUNCHED();
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return RC_OK;
}

// Processing order of sample points: indices sorted by the Morton code of
// the point within the part's bounding box (written to `order`).
rc_status point_order(rc_bvh h, const float* P, int64_t n, int32_t* order, cudaStream_t s)
{
    unsigned long long* keys = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&keys, sizeof(unsigned long long) * n, s));
    g.p[0] = keys;
    float sc[3];
    for (int k = 0; k < 3; ++k) {
        const float ext = h->hi[k] - h->lo[k];
        sc[k] = ext > 0.0f ? 1024.0f / ext : 0.0f;
    }
    k_point_morton<<<nblocks(n, 256), 256, 0, s>>>(P, n, h->lo[0], h->lo[1], h->lo[2], sc[0], sc[1], sc[2], keys,
                                                   order);
    RC_LAUNCHED();
    return sort_pairs(keys, order, n, 4, (unsigned int*)&h->sc->pad, s);
}

__global__ void k_init_scalars(DevScalars* sc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    sc->amax_bits = 0;
    sc->total = 0;
    for (int k = 0; k < 3; ++k) { sc->cmin[k] = 0x7FFFFFFF; sc->cmax[k] = (int)0x80000000; }
    sc->vmaxabs = 0;
    sc->err_index = 0x7FFFFFFF;
    sc->err_vertex = 0x7FFFFFFF;
    sc->max_depth = 0;
    sc->pad = 0;
    sc->wide_depth = 0;
    sc->wide_nodes = 0;
}

static rc_status init_scalars(DevScalars* sc, cudaStream_t s)
{
    k_init_scalars<<<1, 32, 0, s>>>(sc);
    RC_LAUNCHED();
    return RC_OK;
}

static rc_status face_data(rc_bvh h, float* tbox, cudaStream_t s)
{
    rc_status st = init_scalars(h->sc, s);
    if (st != RC_OK) return st;
    k_face_prep<<<nblocks(h->T, 256), 256, 0, s>>>(h->V, h->nV, h->F, h->T, h->fnorm, h->farea, tbox, h->sc);
    RC_LAUNCHED();
    k_quant_area<<<nblocks(h->T, 256), 256, 0, s>>>(h->farea, h->T, h->sc, h->cdf);
    RC_LAUNCHED();
    st = scan_inclusive(h->cdf, h->T, s);
    if (st != RC_OK) return st;
    k_store_total<<<1, 1, 0, s>>>(h->cdf, h->T, h->sc);
    RC_LAUNCHED();
    return RC_OK;
}

// mesh validity and scene bounds from the scalars already read back
static rc_status checked_scalars(rc_bvh h)
{
    const DevScalars& d = h->host_sc;
    if (d.err_index != 0x7FFFFFFF)
        return set_error(RC_E_ARG, "face " + std::to_string(d.err_index) + " has a vertex index outside [0, nV)");
    if (d.err_vertex != 0x7FFFFFFF)
        return set_error(RC_E_ARG, "vertex " + std::to_string(d.err_vertex) + " is not finite");
    h->scene_maxabs = std::max(1.0f, ordered_to_float(d.vmaxabs));
    // the tree depth is set by the build once the tree exists (a refit keeps
    // the topology and hence the depth)
    return RC_OK;
}

static rc_status check_scalars(rc_bvh h, cudaStream_t s)
{
    RC_CUDA(cudaMemcpyAsync(&h->host_sc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    return checked_scalars(h);
}

// PLOC build of the binary tree over the Morton-sorted leaves (h->order);
// writes h->child, h->range, h->parent in the Karras layout and replaces
// h->order by the depth-first leaf order.
static rc_status build_ploc(rc_bvh h, const float* tbox, cudaStream_t s)
{
    const int64_t T = h->T, n_int = h->n_int;
    if (T > 0x7FFFFFFF / 2) return set_error(RC_E_UNSUPPORTED, "too many triangles for the PLOC build");
    const int64_t nb_max = (T + kCompact - 1) / kCompact;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t o_cla = take(4 * T), o_clt = take(4 * T), o_cba = take(24 * T), o_cbt = take(24 * T);
    const size_t o_nn = take(4 * T), o_keep = take(4 * T), o_bsum = take(4 * nb_max), o_n = take(16);
    const size_t o_craw = take(8 * n_int), o_praw = take(4 * (n_int + T)), o_szl = take(4 * n_int);
    const size_t o_szi = take(4 * n_int), o_nid = take(4 * n_int), o_ls = take(4 * n_int), o_pos = take(4 * T);
    const size_t o_ord = take(4 * T);
    char* base = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync((void**)&base, off, s));
    g.p[0] = base;
    int32_t* cl_a = (int32_t*)(base + o_cla);
    int32_t* cl_t = (int32_t*)(base + o_clt);
    float* cb_a = (float*)(base + o_cba);
    float* cb_t = (float*)(base + o_cbt);
    int32_t* nn = (int32_t*)(base + o_nn);
    int* keep = (int*)(base + o_keep);
    int* bsum = (int*)(base + o_bsum);
    int* dn = (int*)(base + o_n);          // [0], [1]: cluster counts (ping-pong), [2]: node counter, [3]: error
    int32_t* child_raw = (int32_t*)(base + o_craw);
    int32_t* parent_raw = (int32_t*)(base + o_praw);
    int32_t* sz_leaf = (int32_t*)(base + o_szl);
    int32_t* sz_int = (int32_t*)(base + o_szi);
    int32_t* newid = (int32_t*)(base + o_nid);
    int32_t* lstart = (int32_t*)(base + o_ls);
    int32_t* pos = (int32_t*)(base + o_pos);
    int32_t* order_out = (int32_t*)(base + o_ord);
    RC_CUDA(cudaMemsetAsync(dn, 0, 16, s));
    RC_CUDA(cudaMemsetAsync(parent_raw, 0xFF, 4 * (n_int + T), s));
    k_ploc_init<<<nblocks(T, 256), 256, 0, s>>>(tbox, h->order, T, n_int, cl_a, cb_a, dn);
    RC_LAUNCHED();
    int cur = 0;
    int64_t n_host = T;
    const int kRoundsPerCheck = 8;
    int rounds = 0;
    while (n_host > 1) {
        if (rounds > 64 + 8 * 64) return set_error(RC_E_DEVICE, "PLOC build did not converge");
        const unsigned g_nn = (unsigned)((n_host + kPlocThreads - 1) / kPlocThreads);
        const unsigned g_c = (unsigned)((n_host + kCompact - 1) / kCompact);
        for (int r = 0; r < kRoundsPerCheck; ++r, ++rounds) {
            k_ploc_nn<<<g_nn, kPlocThreads, 0, s>>>(dn + cur, cb_a, nn);
            RC_LAUNCHED();
            k_ploc_merge<<<g_nn, kPlocThreads, 0, s>>>(dn + cur, nn, cl_a, cb_a, cl_t, cb_t, keep, child_raw,
                                                       parent_raw, dn + 2, n_int);
            RC_LAUNCHED();
            k_ploc_count<<<g_c, kCompact, 0, s>>>(dn + cur, keep, bsum);
            RC_LAUNCHED();
            k_ploc_scan<<<1, 32, 0, s>>>(bsum, (int)g_c, dn + cur, dn + 1 - cur);
            RC_LAUNCHED();
            k_ploc_scatter<<<g_c, kCompact, 0, s>>>(dn + cur, keep, bsum, cl_t, cb_t, cl_a, cb_a);
            RC_LAUNCHED();
            cur = 1 - cur;
        }
        int hn[3];
        RC_CUDA(cudaMemcpyAsync(hn, dn, sizeof hn, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        n_host = hn[cur];
        if (n_host == 1 && hn[2] != n_int)
            return set_error(RC_E_DEVICE, "PLOC build made a wrong number of interior nodes");
    }
    // depth-first renumbering into the Karras layout
    RC_CUDA(cudaMemsetAsync(h->visits, 0, sizeof(int32_t) * n_int, s));
    k_ploc_sizes<<<nblocks(T, 256), 256, 0, s>>>(T, n_int, parent_raw, child_raw, sz_leaf, sz_int, h->visits,
                                                 dn + 3);
    RC_LAUNCHED();
    k_ploc_number<<<nblocks(n_int + T, 256), 256, 0, s>>>(T, n_int, parent_raw, child_raw, sz_leaf, sz_int, newid,
                                                          lstart, pos, dn + 3);
    RC_LAUNCHED();
    k_ploc_emit<<<nblocks(n_int + T, 256), 256, 0, s>>>(T, n_int, parent_raw, child_raw, newid, lstart, sz_leaf, pos,
                                                        h->order, h->child, h->range, h->parent, order_out);
    RC_LAUNCHED();
    RC_CUDA(cudaMemcpyAsync(h->order, order_out, sizeof(int32_t) * T, cudaMemcpyDeviceToDevice, s));
    int herr = 0;
    RC_CUDA(cudaMemcpyAsync(&herr, dn + 3, sizeof herr, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    if (herr) return set_error(RC_E_DEVICE, "PLOC tree walk exceeded its bound");
    return RC_OK;
}

// Collapse the binary tree into the 4-wide layout (wnodes), or make the
// one-leaf wide root for tiny parts.  Needs the binary tree and its boxes.
static rc_status build_wide(rc_bvh h, const float* tbox, cudaStream_t s)
{
    const int64_t T = h->T;
    if (!h->wnodes) RC_CUDA(cudaMallocAsync(&h->wnodes, sizeof(float4) * 8 * h->n_int, s));
    if (T <= kLeafMax) {
        k_wide_small<<<1, 32, 0, s>>>(T, tbox, h->wnodes, h->sc);
        RC_LAUNCHED();
        return RC_OK;
    }
    const int64_t n_int = h->n_int;
    int32_t* q = nullptr;
    int* counts = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&q, sizeof(int32_t) * 4 * n_int, s));
    g.p[0] = q;
    RC_CUDA(cudaMallocAsync(&counts, sizeof(int) * 4, s));
    g.p[1] = counts;
    int32_t *qa_bin = q, *qa_wide = q + n_int, *qb_bin = q + 2 * n_int, *qb_wide = q + 3 * n_int;
    int *ca = counts, *cb = counts + 1;
    k_wide_init<<<1, 32, 0, s>>>(qa_bin, qa_wide, counts);
    RC_LAUNCHED();
    // The top `split` levels take one launch each (a level's queue is at most
    // 4^level long); then one launch finishes every queued subtree, a thread
    // each, once the queue holds about n_int / RC_WIDE_SUBTREE nodes.  Levels
    // past the bottom of a shallow tree find an empty queue.
    int split = 0;
    while (split < 30 && std::pow(4.0, (double)split) * RC_WIDE_SUBTREE < (double)n_int) ++split;
    if (RC_WIDE_SUBTREE <= 0) split = kStack;      // a deeper tree is rejected anyway
    int level = 0;
    for (; level < split; ++level) {
        const double cap = std::min((double)n_int, std::pow(4.0, (double)std::min(level, 30)));
        const unsigned grid = (unsigned)std::max(1.0, std::ceil(cap / 256.0));
        RC_CUDA(cudaMemsetAsync(cb, 0, sizeof(int), s));
        k_wide_level<<<grid, 256, 0, s>>>(n_int, h->child, h->range, h->nbox, qa_bin, qa_wide, ca, qb_bin, qb_wide,
                                          cb, counts + 2, h->wnodes, h->sc, level);
        RC_LAUNCHED();
        std::swap(qa_bin, qb_bin);
        std::swap(qa_wide, qb_wide);
        std::swap(ca, cb);
    }
    {
        const double cap = std::min((double)n_int, std::pow(4.0, (double)std::min(level, 30)));
        const unsigned grid = (unsigned)std::max(1.0, std::ceil(cap / 256.0));
        k_wide_subtrees<<<grid, 256, 0, s>>>(n_int, h->child, h->range, h->nbox, qa_bin, qa_wide, ca, counts + 2,
                                             h->wnodes, h->sc, level);
        RC_LAUNCHED();
    }
    RC_CUDA(cudaMemcpyAsync(&h->sc->wide_nodes, counts + 2, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return RC_OK;
}

// ---------------------------------------------------------------------------
// The 4-wide tree with its child boxes in the coordinates of a machining
// frame (rows of M = the frame's columns): the same nodes, codes and
// triangles; each box is the bounding box of the frame coordinates of its
// triangles' vertices, evaluated in FP64 and rounded outward to fp32.  The
// axis walk of the orthogonal cast tests these boxes (its rays run along a
// frame axis) and still tests triangles in world coordinates.
// ---------------------------------------------------------------------------
__global__ void k_frame_leaf_boxes(const float* __restrict__ V, const int32_t* __restrict__ F,
                                   const int32_t* __restrict__ order, int64_t T, int64_t nV, int64_t n_int,
                                   FrameArgs fa, float* __restrict__ nbox_f)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    const int32_t f = order[k];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (f >= 0 && f < T)
        for (int a = 0; a < 3; ++a) {
            const int64_t v = F[3 * (int64_t)f + a];
            if (v < 0 || v >= nV) continue;
            const double x = V[3 * v], y = V[3 * v + 1], z = V[3 * v + 2];
            for (int j = 0; j < 3; ++j) {
                // frame coordinate j: column j of the row-major frame
                const double q = __dadd_rn(__dadd_rn(__dmul_rn(x, (double)fa.f[j]), __dmul_rn(y, (double)fa.f[3 + j])),
                                           __dmul_rn(z, (double)fa.f[6 + j]));
                lo[j] = fmin(lo[j], q);
                hi[j] = fmax(hi[j], q);
            }
        }
    float* b = nbox_f + 6 * (n_int + k);
    for (int j = 0; j < 3; ++j) {
        b[j] = __double2float_rd(lo[j]);
        b[3 + j] = __double2float_ru(hi[j]);
    }
}

__global__ void k_frame_pack(const float4* __restrict__ wnodes, int64_t n_int, int64_t T,
                             const DevScalars* __restrict__ sc, const float* __restrict__ nbox_f,
                             const float* __restrict__ all_box, float4* __restrict__ ftree)
{
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= sc->wide_nodes || w >= n_int) return;
    const float4* nd = wnodes + 8 * w;
    const float4 idv = nd[7];
    const int32_t ids[4] = {__float_as_int(idv.x), __float_as_int(idv.y), __float_as_int(idv.z), __float_as_int(idv.w)};
    float lo[3][4], hi[3][4];
    for (int k = 0; k < 4; ++k) {
        const float* b = nullptr;
        if (ids[k] == kAllTris) b = all_box;
        else if (ids[k] >= 0 && ids[k] < n_int + T) b = nbox_f + 6 * (int64_t)ids[k];
        for (int a = 0; a < 3; ++a) {
            lo[a][k] = b ? b[a] : INFINITY;
            hi[a][k] = b ? b[3 + a] : -INFINITY;
        }
    }
    float4* o = ftree + 8 * w;
    for (int a = 0; a < 3; ++a) {
        o[2 * a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
        o[2 * a + 1] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
    }
    o[6] = nd[6];
    o[7] = idv;
}

// box of all leaf slots [0, T) of nbox_f (tiny parts: the one-leaf root)
__global__ void k_frame_all_box(const float* __restrict__ nbox_f, int64_t n_int, int64_t T, float* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = 0; k < T; ++k)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], nbox_f[6 * (n_int + k) + a]);
            hi[a] = fmaxf(hi[a], nbox_f[6 * (n_int + k) + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) { out[a] = lo[a]; out[3 + a] = hi[a]; }
}

rc_status frame_tree(rc_bvh h, const float f9[9], float4* ftree, cudaStream_t s)
{
    const int64_t T = h->T, n_int = h->n_int;
    FrameArgs fa;
    for (int k = 0; k < 9; ++k) fa.f[k] = f9[k];
    float* nbox_f = nullptr;
    int32_t* visits = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&nbox_f, sizeof(float) * 6 * (n_int + T + 1), s));
    g.p[0] = nbox_f;
    float* all_box = nbox_f + 6 * (n_int + T);
    k_frame_leaf_boxes<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(h->V, h->F, h->order, T, h->nV, n_int, fa, nbox_f);
    RC_LAUNCHED();
    if (T > kLeafMax) {
        RC_CUDA(cudaMallocAsync(&visits, sizeof(int32_t) * n_int, s));
        g.p[1] = visits;
        RC_CUDA(cudaMemsetAsync(visits, 0, sizeof(int32_t) * n_int, s));
        k_refit<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(T, n_int, h->parent, h->child, nbox_f, visits, h->sc);
        RC_LAUNCHED();
    } else {
        k_frame_all_box<<<1, 32, 0, s>>>(nbox_f, n_int, T, all_box);
        RC_LAUNCHED();
    }
    k_frame_pack<<<(unsigned)((n_int + 255) / 256), 256, 0, s>>>(h->wnodes, n_int, T, h->sc, nbox_f, all_box, ftree);
    RC_LAUNCHED();
    return RC_OK;
}

rc_status build_bvh(rc_bvh h, cudaStream_t s)
{
    const int64_t T = h->T;
    float* tbox = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&tbox, sizeof(float) * 6 * T, s));
    g.p[0] = tbox;
    // No host synchronisation until the end: a bad mesh is reported from the
    // one final readback (every kernel in between guards its gathers).
    rc_status st = face_data(h, tbox, s);
    if (st != RC_OK) return st;

    h->n_int = T > kLeafMax ? T - 1 : 1;
    RC_CUDA(cudaMallocAsync(&h->nodes, sizeof(float4) * 4 * h->n_int, s));
    RC_CUDA(cudaMallocAsync(&h->tris, sizeof(float4) * 3 * T, s));
    RC_CUDA(cudaMallocAsync(&h->order, sizeof(int32_t) * T, s));

    if (T <= kLeafMax) {
        int32_t ord[kLeafMax];
        for (int i = 0; i < kLeafMax; ++i) ord[i] = i;
        RC_CUDA(cudaMemcpyAsync(h->order, ord, sizeof(int32_t) * T, cudaMemcpyHostToDevice, s));
        k_pack_small<<<1, 32, 0, s>>>(T, tbox, h->nodes);
        RC_LAUNCHED();
        h->max_depth = 1;
    } else {
        unsigned long long* k0 = nullptr;
        RC_CUDA(cudaMallocAsync(&k0, sizeof(unsigned long long) * T, s));
        g.p[1] = k0;
        k_morton<<<nblocks(T, 256), 256, 0, s>>>(tbox, T, h->sc, k0, h->order);
        RC_LAUNCHED();
        rc_status sst = sort_pairs(k0, h->order, T, kMortonPasses, (unsigned int*)&h->sc->pad, s);
        if (sst != RC_OK) return sst;
        // after an even number of passes the sorted data is back in (k0, h->order)
        const int64_t n_int = h->n_int;
        RC_CUDA(cudaMallocAsync(&h->parent, sizeof(int32_t) * (n_int + T), s));
        RC_CUDA(cudaMallocAsync(&h->child, sizeof(int32_t) * 2 * n_int, s));
        RC_CUDA(cudaMallocAsync(&h->range, sizeof(int32_t) * 2 * n_int, s));
        RC_CUDA(cudaMallocAsync(&h->nbox, sizeof(float) * 6 * (n_int + T), s));
        RC_CUDA(cudaMallocAsync(&h->visits, sizeof(int32_t) * n_int, s));
        if (h->builder == RC_BUILDER_PLOC) {
            rc_status pst = build_ploc(h, tbox, s);
            if (pst != RC_OK) return pst;
        } else {
            k_karras<<<nblocks(n_int, 256), 256, 0, s>>>(k0, T, h->child, h->range, h->parent);
            RC_LAUNCHED();
        }
        RC_CUDA(cudaMemsetAsync(h->visits, 0, sizeof(int32_t) * n_int, s));
        k_leaf_boxes<<<nblocks(T, 256), 256, 0, s>>>(tbox, h->order, T, n_int, h->nbox);
        RC_LAUNCHED();
        k_refit<<<nblocks(T, 256), 256, 0, s>>>(T, n_int, h->parent, h->child, h->nbox, h->visits, h->sc);
        RC_LAUNCHED();
        k_pack<<<nblocks(n_int, 256), 256, 0, s>>>(n_int, h->child, h->range, h->nbox, h->nodes);
        RC_LAUNCHED();
    }
    st = build_wide(h, tbox, s);
    if (st != RC_OK) return st;
    k_tri_records<<<nblocks(T, 256), 256, 0, s>>>(h->V, h->nV, h->F, h->order, T, h->tris);
    RC_LAUNCHED();
    RC_CUDA(cudaMemcpyAsync(&h->host_sc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    if ((st = checked_scalars(h)) != RC_OK) return st;
    if (h->host_sc.pad != 0) return set_error(RC_E_DEVICE, "radix sort produced an out-of-range position");
    if (T > kLeafMax) h->max_depth = h->host_sc.max_depth;
    h->wide_depth = h->host_sc.wide_depth;
    for (int k = 0; k < 3; ++k) { h->lo[k] = 0; h->hi[k] = 0; }
    if (h->max_depth >= kStack)
        return set_error(RC_E_UNSUPPORTED, "BVH depth " + std::to_string(h->max_depth) +
                                               " exceeds the traversal stack");
    if (3 * h->wide_depth + 1 >= kStack4)
        return set_error(RC_E_UNSUPPORTED, "4-wide BVH depth " + std::to_string(h->wide_depth) +
                                               " exceeds the traversal stack");
    return RC_OK;
}

rc_status refit_bvh(rc_bvh h, cudaStream_t s)
{
    const int64_t T = h->T;
    float* tbox = nullptr;
    BuildScratch g{s};
    RC_CUDA(cudaMallocAsync(&tbox, sizeof(float) * 6 * T, s));
    g.p[0] = tbox;
    rc_status st = face_data(h, tbox, s);
    if (st != RC_OK) return st;
    st = check_scalars(h, s);
    if (st != RC_OK) return st;
    if (T <= kLeafMax) {
        k_pack_small<<<1, 32, 0, s>>>(T, tbox, h->nodes);
        RC_LAUNCHED();
    } else {
        const int64_t n_int = h->n_int;
        RC_CUDA(cudaMemsetAsync(h->visits, 0, sizeof(int32_t) * n_int, s));
        k_leaf_boxes<<<nblocks(T, 256), 256, 0, s>>>(tbox, h->order, T, n_int, h->nbox);
        RC_LAUNCHED();
        k_refit<<<nblocks(T, 256), 256, 0, s>>>(T, n_int, h->parent, h->child, h->nbox, h->visits, h->sc);
        RC_LAUNCHED();
        k_pack<<<nblocks(n_int, 256), 256, 0, s>>>(n_int, h->child, h->range, h->nbox, h->nodes);
        RC_LAUNCHED();
    }
    st = build_wide(h, tbox, s);
    if (st != RC_OK) return st;
    k_tri_records<<<nblocks(T, 256), 256, 0, s>>>(h->V, h->nV, h->F, h->order, T, h->tris);
    RC_LAUNCHED();
    RC_CUDA(cudaMemcpyAsync(&h->host_sc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    h->wide_depth = h->host_sc.wide_depth;
    if (3 * h->wide_depth + 1 >= kStack4)
        return set_error(RC_E_UNSUPPORTED, "4-wide BVH depth exceeds the traversal stack after refit");
    return RC_OK;
}

rc_status sample_points(rc_bvh h, int64_t n, const rc_params* p, float* P, float* N, int32_t* face,
                        double* weight, cudaStream_t s)
{
    if (p->sample_mode == RC_SAMPLE_FACE_CENTROID) {
        k_sample_centroid<<<nblocks(h->T, 256), 256, 0, s>>>(h->V, h->F, h->fnorm, h->farea, h->T, P, N, face,
                                                             weight);
        RC_LAUNCHED();
        return RC_OK;
    }
    k_sample_area<<<nblocks(n, 256), 256, 0, s>>>(h->V, h->F, h->T, h->cdf, h->sc, h->fnorm, n, p->seed,
                                                  P, N, face, weight);
    RC_LAUNCHED();
    return RC_OK;
}

}  // namespace rc
