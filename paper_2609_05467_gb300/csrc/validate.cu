// validate.cu -- index checks of a built tree, the device-side bounds
// checking that stands in for a memory checker: every index the casts
// dereference is checked against the array it points into, and the 4-wide
// nodes must number children above their parent (so every descent strictly
// increases the node index and no walk can cycle).  Violations are counted,
// never trapped.
#include <algorithm>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

struct CheckCounts {
    unsigned long long wide_child;     // interior child out of range or not above its parent
    unsigned long long wide_leaf;      // leaf triangle range outside [0, T)
    unsigned long long wide_box;       // a used slot with lo > hi or a non-finite bound
    unsigned long long binary_child;   // packed binary node child outside its range
    unsigned long long tri_face;       // triangle record whose face id is outside [0, T)
    unsigned long long nodes_seen;     // wide nodes reached from the root
};

__device__ __forceinline__ bool leaf_ok(int32_t c, int64_t T)
{
    const int32_t v = -1 - c;
    const int64_t first = v >> 3, cnt = (v & 7) + 1;
    return first >= 0 && first + cnt <= T;
}

// one level of the 4-wide tree: check each queued node's four slots and
// queue its interior children
__global__ void k_check_wide_level(const float4* __restrict__ wnodes, int64_t n_int, int64_t T,
                                   const int32_t* __restrict__ qin, const int* __restrict__ qin_count,
                                   int32_t* qout, int* qout_count, int cap, CheckCounts* cc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= min(*qin_count, cap)) return;
    const int32_t w = qin[t];
    atomicAdd(&cc->nodes_seen, 1ULL);
    const float4* nd = wnodes + 8 * (int64_t)w;
    const float4 ci = nd[6];
    const int32_t c[4] = {__float_as_int(ci.x), __float_as_int(ci.y), __float_as_int(ci.z), __float_as_int(ci.w)};
    const float4 lx = nd[0], hx = nd[1], ly = nd[2], hy = nd[3], lz = nd[4], hz = nd[5];
    const float lo[3][4] = {{lx.x, lx.y, lx.z, lx.w}, {ly.x, ly.y, ly.z, ly.w}, {lz.x, lz.y, lz.z, lz.w}};
    const float hi[3][4] = {{hx.x, hx.y, hx.z, hx.w}, {hy.x, hy.y, hy.z, hy.w}, {hz.x, hz.y, hz.z, hz.w}};
    for (int k = 0; k < 4; ++k) {
        if (c[k] == -1 && lo[0][k] == INFINITY) continue;      // empty slot
        bool box_ok = true;
        for (int a = 0; a < 3; ++a) box_ok &= isfinite(lo[a][k]) && isfinite(hi[a][k]) && lo[a][k] <= hi[a][k];
        if (!box_ok) atomicAdd(&cc->wide_box, 1ULL);
        if (c[k] >= 0) {
            if (c[k] <= w || c[k] >= n_int) {
                atomicAdd(&cc->wide_child, 1ULL);
            } else {
                const int slot = atomicAdd(qout_count, 1);
                if (slot < cap) qout[slot] = c[k];
                else atomicAdd(&cc->wide_child, 1ULL);     // more nodes on a level than the tree can hold
            }
        } else if (!leaf_ok(c[k], T)) {
            atomicAdd(&cc->wide_leaf, 1ULL);
        }
    }
}

// packed binary nodes: child indices within their ranges
__global__ void k_check_binary(const float4* __restrict__ nodes, int64_t n_int, int64_t T, CheckCounts* cc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const float4 n3 = nodes[4 * i + 3];
    const int32_t c[2] = {__float_as_int(n3.x), __float_as_int(n3.y)};
    for (int k = 0; k < 2; ++k) {
        const bool ok = c[k] >= 0 ? (int64_t)c[k] < n_int : leaf_ok(c[k], T);
        if (!ok) atomicAdd(&cc->binary_child, 1ULL);
    }
}

// triangle records: the face id in the second record's w lane
__global__ void k_check_tris(const float4* __restrict__ tris, int64_t T, CheckCounts* cc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    const int32_t f = __float_as_int(tris[3 * k + 1].w);
    if (f < 0 || (int64_t)f >= T) atomicAdd(&cc->tri_face, 1ULL);
}

}  // namespace rc

using namespace rc;

extern "C" rc_status rc_bvh_validate(rc_bvh h, int64_t* h_counts, void* stream)
{
    RC_RANGE();
    if (!h || !h_counts) return set_error(RC_E_ARG, "handle or output is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_int = h->n_int, T = h->T;
    const int64_t cap = std::max<int64_t>(n_int, 1);      // wide nodes never outnumber binary interior nodes
    if (cap > 0x7FFFFFFF) return set_error(RC_E_UNSUPPORTED, "tree too large to check");
    CheckCounts* cc = nullptr;
    int32_t* q = nullptr;
    int* counts = nullptr;
    RC_CUDA(cudaMallocAsync(&cc, sizeof(CheckCounts), s));
    RC_CUDA(cudaMallocAsync(&q, sizeof(int32_t) * 2 * cap, s));
    RC_CUDA(cudaMallocAsync(&counts, sizeof(int) * 2, s));
    RC_CUDA(cudaMemsetAsync(cc, 0, sizeof(CheckCounts), s));
    // the root is node 0; a level's queue holds at most n_int nodes
    const int root_and_count[2] = {0, 1};
    int32_t* qa = q;
    int32_t* qb = q + cap;
    RC_CUDA(cudaMemcpyAsync(qa, &root_and_count[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaMemcpyAsync(counts, &root_and_count[1], sizeof(int), cudaMemcpyHostToDevice, s));
    int* ca = counts;
    int* cb = counts + 1;
    int level_count = 1;
    // children number above their parent, so no walk is longer than n_int
    // levels; a valid tree ends after its depth
    for (int64_t level = 0; level_count > 0 && level <= n_int; ++level) {
        RC_CUDA(cudaMemsetAsync(cb, 0, sizeof(int), s));
        k_check_wide_level<<<(unsigned)((level_count + 255) / 256), 256, 0, s>>>(h->wnodes, n_int, T, qa, ca, qb, cb,
                                                                                 (int)cap, cc);
        RC_LAUNCHED();
        RC_CUDA(cudaMemcpyAsync(&level_count, cb, sizeof(int), cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        level_count = (int)std::min<int64_t>(level_count, cap);
        std::swap(qa, qb);
        std::swap(ca, cb);
    }
    if (T > kLeafMax) {
        k_check_binary<<<(unsigned)((n_int + 255) / 256), 256, 0, s>>>(h->nodes, n_int, T, cc);
        RC_LAUNCHED();
    }
    k_check_tris<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(h->tris, T, cc);
    RC_LAUNCHED();
    CheckCounts hc;
    RC_CUDA(cudaMemcpyAsync(&hc, cc, sizeof hc, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaFreeAsync(cc, s));
    RC_CUDA(cudaFreeAsync(q, s));
    RC_CUDA(cudaFreeAsync(counts, s));
    RC_CUDA(cudaStreamSynchronize(s));
    h_counts[0] = (int64_t)hc.wide_child;
    h_counts[1] = (int64_t)hc.wide_leaf;
    h_counts[2] = (int64_t)hc.wide_box;
    h_counts[3] = (int64_t)hc.binary_child;
    h_counts[4] = (int64_t)hc.tri_face;
    h_counts[5] = (int64_t)hc.nodes_seen;
    return RC_OK;
}
