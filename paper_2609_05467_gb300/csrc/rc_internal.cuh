// rc_internal.cuh -- device-side helpers and the handle layout of the
// sm_103a ray-casting library.  Included by the library's .cu files only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/rc.h"

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
namespace rc {

rc_status set_error(rc_status st, const std::string& msg);
rc_status cuda_error(cudaError_t e, const char* what);
void count_launch(int k = 1);

#define RC_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::rc::cuda_error(_e, #call);        \
    } while (0)

#define RC_LAUNCHED()                                                     \
    do {                                                                  \
        ::rc::count_launch();                                             \
        cudaError_t _e = cudaGetLastError();                              \
        if (_e != cudaSuccess) return ::rc::cuda_error(_e, "kernel launch"); \
    } while (0)

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
#ifndef RC_LEAF_MAX
#define RC_LEAF_MAX 2
#endif
constexpr int kLeafMax = RC_LEAF_MAX;   // triangles per packed leaf (1..8)
constexpr int kStack = 64;         // binary traversal stack entries (>= max tree depth)
constexpr int kStack4 = 96;        // 4-wide traversal stack entries (>= 3 * wide depth + 1)
constexpr double kTau = 1e-9;      // relative ambiguity band of the occlusion test
constexpr int kMaxDirs = 65536;

// scratch of the variability reduction: kVarSums int64 sums, then the two
// FP64 weighted sums, then the per-block FP64 partials (two rows of
// kVarMaxBlocks); no per-direction scratch
constexpr int kVarSums = 8;
constexpr int kVarMaxBlocks = 2048;
constexpr size_t kVarWsumOffset = 8 * kVarSums;
constexpr size_t kVarPartOffset = kVarWsumOffset + 64;
constexpr size_t kVarScratchBytes = kVarPartOffset + 2 * sizeof(double) * kVarMaxBlocks;   // 32,896 bytes

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct DevScalars {
    unsigned long long amax_bits;  // max face area (FP64 bits, >= 0)
    long long total;               // total quantised area
    int cmin[3], cmax[3];          // box-centre bounds (orderable float ints)
    int vmaxabs;                   // max |coordinate| (orderable float int)
    int err_index;                 // first bad face (index out of range), else -1
    int err_vertex;                // first bad vertex (non-finite), else -1
    int max_depth;
    int pad;
    int wide_depth;
    int wide_nodes;                // 4-wide nodes allocated
};

constexpr int kAllTris = -2;       // wide-node child made of all triangles (parts with <= kLeafMax of them)

// machining frame on the device (Section 3.2)
struct FrameArgs { float f[9]; const float4* tree; double sc_c[3]; double sc_r; };
struct FrameDev {
    float axes[18];     // +X', -X', +Y', -Y', +Z', -Z' (fp32)
    float pad[2];
    double frame[9];    // row-major frame, FP64
    double fbox[6];     // frame-coordinate bounding box of the vertices (lo xyz, hi xyz)
    long long box[6];   // ordered-integer accumulators for fbox
    const float4* tree; // 4-wide tree with child boxes in frame coordinates (the world tree for the identity)
    double gram[9];     // G = F^T F of the fp32 frame F (FP64): how far the axes are from orthonormal
    double sc_c[3];     // centre of the part's bounding box (world)
    double sc_r;        // half its diagonal
};

// one part of a batched cast (device descriptor)
struct BatchPart {
    const float4* nodes;
    const float4* tris;
    const float* P;
    const float* N;
    const int32_t* order;          // processing order of the part's points, or null
    uint32_t* bits;
    int32_t* count;
    unsigned long long* counters;  // [4] per part, or null
    long long n;                   // points
    long long first_item;          // first global work item of the part
    int max_steps;
    float scene_maxabs;
};

// machining frames on the device (cast.cu, build.cu): the frame's axes,
// FP64 matrix, vertex box and Gram matrix, and the tree its axis rays walk
// (nullptr: the world tree)
rc_status frame_setup(rc_bvh h, const rc_params* p, FrameDev* d, cudaStream_t s, const float4* tree = nullptr);
rc_status frame_setup_f(rc_bvh h, const float* f9, FrameDev* d, cudaStream_t s, const float4* tree = nullptr);
// the 4-wide tree of h with its child boxes in the coordinates of frame f9
// (ftree: as many nodes as h's 4-wide tree)
rc_status frame_tree(rc_bvh h, const float f9[9], float4* ftree, cudaStream_t s);
// *ftree = a new frame tree for f9, or nullptr when the axis rays walk the
// world tree (identity frame, binary tree); release with cudaFreeAsync
rc_status make_frame_tree(rc_bvh h, const float f9[9], const rc_params* p, float4** ftree, cudaStream_t s);
bool is_identity_frame(const float f9[9]);

// variability reduction (reduce.cu): queues the kernels on s; `scratch` is
// kVarScratchBytes of device memory (cleared here)
rc_status launch_variability(const uint32_t* bits, const float* N, const double* weight, int64_t n,
                             const float4* dirs, const rc_params* p, float* acc, int8_t* dom, float* conc,
                             double* dir_area, void* scratch, cudaStream_t s);
// the part-level summary from the scratch's sums read back to the host
// (sums: kVarSums int64; wsum: the two weighted FP64 sums)
void fill_summary(const long long* sums, const double* wsum, int64_t n, int32_t n_dirs, bool weighted,
                  rc_summary* out);

}  // namespace rc

struct rc_bvh_s {
    int device = 0;
    int builder = 0;               // RC_BUILDER_KARRAS or RC_BUILDER_PLOC
    int64_t nV = 0, T = 0;
    float* V = nullptr;            // [nV][3] copy of the vertices
    int32_t* F = nullptr;          // [T][3] copy of the faces
    float4* tris = nullptr;        // [T][3] triangle records in Morton order
    float4* nodes = nullptr;       // [n_int][4] packed BVH2 nodes
    float4* wnodes = nullptr;      // [<= n_int][8] packed 4-wide nodes
    int wide_depth = 0;
    int64_t n_int = 0;             // internal nodes (>= 1)
    int32_t* parent = nullptr;     // [n_int + T]: parent of internal i at i, of leaf k at n_int+k
    int32_t* child = nullptr;      // [n_int][2] combined indices (leaf k -> n_int+k)
    int32_t* range = nullptr;      // [n_int][2] first,last sorted leaf
    int32_t* order = nullptr;      // [T] original face id of sorted slot
    float* nbox = nullptr;         // [n_int + T][6] boxes (lo xyz, hi xyz)
    int32_t* visits = nullptr;     // [n_int] refit arrival counters
    float* fnorm = nullptr;        // [T][3] fp32 unit normals
    double* farea = nullptr;       // [T] FP64 areas
    long long* cdf = nullptr;      // [T] inclusive quantised-area prefix
    rc::DevScalars* sc = nullptr;  // device scalars
    rc::DevScalars host_sc;        // copy after build
    float scene_maxabs = 1.0f;     // max(1, max |vertex coordinate|)
    int max_depth = 0;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    // direction tables of the last cast (device, cached per device and N):
    // canonical order (x, y, z, 0) and tile order (x, y, z, canonical index)
    int32_t dirs_n = 0;
    const float4* dirs = nullptr;
    const float4* tdirs = nullptr;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
namespace rc {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ int float_to_ordered(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ __forceinline__ float ordered_to_float(int i)
{
#ifdef __CUDA_ARCH__
    return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
#else
    union { int i; float f; } u;
    u.i = i >= 0 ? i : i ^ 0x7FFFFFFF;
    return u.f;
#endif
}
__device__ __forceinline__ long long double_to_ordered(double d)
{
    long long i = __double_as_longlong(d);
    return i >= 0 ? i : i ^ 0x7FFFFFFFFFFFFFFFLL;
}
__host__ __device__ __forceinline__ double ordered_to_double(long long i)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(i >= 0 ? i : i ^ 0x7FFFFFFFFFFFFFFFLL);
#else
    union { long long i; double d; } u;
    u.i = i >= 0 ? i : i ^ 0x7FFFFFFFFFFFFFFFLL;
    return u.d;
#endif
}

// splitmix64 (Steele, Lea, Flood 2014): mix(x + golden)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Orthonormal basis (t1, t2) of unit normal n: the branchless construction
// of Duff et al., JCGT 6(1), 2017, evaluated in fp32 with every operation
// rounded separately (no contraction), left to right.
struct Onb { float t1x, t1y, t1z, t2x, t2y, t2z; };

__device__ __forceinline__ Onb make_onb(float nx, float ny, float nz)
{
    Onb b;
    const float sgn = copysignf(1.0f, nz);
    const float a = __fdiv_rn(-1.0f, __fadd_rn(sgn, nz));
    const float bb = __fmul_rn(__fmul_rn(nx, ny), a);
    b.t1x = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sgn, nx), nx), a));
    b.t1y = __fmul_rn(sgn, bb);
    b.t1z = __fmul_rn(-sgn, nx);
    b.t2x = bb;
    b.t2y = __fadd_rn(sgn, __fmul_rn(__fmul_rn(ny, ny), a));
    b.t2z = -ny;
    return b;
}

// World direction of local hemisphere sample h: (t1*hx + t2*hy) + n*hz per
// component, fp32, in that order.
__device__ __forceinline__ void local_to_world(const Onb& b, float nx, float ny, float nz, float hx,
                                               float hy, float hz, float& dx, float& dy, float& dz)
{
    dx = __fadd_rn(__fadd_rn(__fmul_rn(b.t1x, hx), __fmul_rn(b.t2x, hy)), __fmul_rn(nx, hz));
    dy = __fadd_rn(__fadd_rn(__fmul_rn(b.t1y, hx), __fmul_rn(b.t2y, hy)), __fmul_rn(ny, hz));
    dz = __fadd_rn(__fadd_rn(__fmul_rn(b.t1z, hx), __fmul_rn(b.t2z, hy)), __fmul_rn(nz, hz));
}

// Coordinate k of the centroid of face f (Section 3.1):
// fl32((A_k + B_k + C_k) / 3), summed left to right in FP64.
__device__ __forceinline__ float face_centroid(const float* __restrict__ V, const int32_t* __restrict__ F,
                                               int64_t f, int k)
{
    const double a = V[3 * (int64_t)F[3 * f] + k], b = V[3 * (int64_t)F[3 * f + 1] + k];
    const double s = __dadd_rn(__dadd_rn(a, b), (double)V[3 * (int64_t)F[3 * f + 2] + k]);
    return __double2float_rn(__ddiv_rn(s, 3.0));
}

// Offset origin fl32(p + eps*n), evaluated in FP64 without contraction.
__device__ __forceinline__ float offset_coord(float p, float n, double eps)
{
    return __double2float_rn(__dadd_rn((double)p, __dmul_rn(eps, (double)n)));
}

}  // namespace rc
