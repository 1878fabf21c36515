// frames.cu -- automatic machining frame.  Section 3.2 places the part in a
// canonical frame whose axes are the machine axes and Section 3.3 counts the
// setups in it; the paper does not say how the frame is found.  This file
// proposes candidates (the given frame, the surface's principal axes, its
// dominant face normals, and the box-minimising rotation of each) and picks
// the one with the fewest setups, evaluating all candidates in one
// orthogonal-cast launch.
//
// Device: FP64 surface moments (fixed-order block reduction), the
// cube-map histogram of face-normal lines, the exact FP64 bounding boxes of
// 384 rotations per base frame (with an fp32 pre-pass).  Host: 3x3 eigen-decomposition (cyclic Jacobi),
// snapping and Gram-Schmidt, the choice.  Host code is compiled without
// floating-point contraction, so every FP64 expression is rounded operation
// by operation, left to right.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rc_internal.cuh"
#include "nvtx_range.h"

namespace rc {

rc_status launch_orthogonal_frames(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                                   const FrameDev* fds, int nf, uint8_t* mask, float* travel,
                                   unsigned long long* counters, cudaStream_t s);
rc_status launch_classes(rc_bvh h, const uint8_t* mask, const float* travel, const int32_t* face, int64_t n,
                         const rc_params* p, uint8_t* cls, const double* frame_d, const double* fbox_d,
                         uint8_t* fixture, unsigned long long* hist, cudaStream_t s);
rc_status check_params_public(const rc_params* p);

constexpr int kCells = 32;                       // cube-map cells per side
constexpr int kNumCells = 3 * kCells * kCells;   // three axes (lines, not directions)
constexpr double kSnap = 1048576.0;              // 2^20
constexpr double kGap = 1e-3;                    // relative eigenvalue gap for principal axes
constexpr double kOrtho = 0.2;                   // |cos| to Z' of the second normal cell's centre
constexpr int kMomentBlocks = 256;
constexpr int kMomentThreads = 256;

// ---------------------------------------------------------------------------
// device: area moments of the surface relative to r.  Per face, FP64:
//   S0 += A, S1 += A s / 3, S2 += A / 12 (a a^T + b b^T + c c^T + s s^T),
// s = a + b + c (the exact integral of x x^T over a triangle).  Ten sums
// (S0, S1 xyz, S2 xx xy xz yy yz zz) per block, tree-reduced in a fixed
// order; k_moments_final adds the block partials in block order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMomentThreads)
k_moments(const float* __restrict__ V, const int32_t* __restrict__ F, const double* __restrict__ farea, int64_t T,
          double rx, double ry, double rz, double* __restrict__ partial /*[blocks][10]*/)
{
    __shared__ double sh[10][kMomentThreads];
    double acc[10];
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    const double r[3] = {rx, ry, rz};
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < T; f += (int64_t)gridDim.x * blockDim.x) {
        double v[3][3];
        for (int c = 0; c < 3; ++c) {
            const int64_t vi = F[3 * f + c];
            for (int k = 0; k < 3; ++k) v[c][k] = __dsub_rn((double)V[3 * vi + k], r[k]);
        }
        double sv[3];
        for (int k = 0; k < 3; ++k) sv[k] = __dadd_rn(__dadd_rn(v[0][k], v[1][k]), v[2][k]);
        const double A = farea[f];
        const double w = __ddiv_rn(A, 12.0);
        acc[0] = __dadd_rn(acc[0], A);
        for (int k = 0; k < 3; ++k) acc[1 + k] = __dadd_rn(acc[1 + k], __ddiv_rn(__dmul_rn(A, sv[k]), 3.0));
        int q = 4;
        for (int k = 0; k < 3; ++k)
            for (int l = k; l < 3; ++l) {
                double m = __dmul_rn(v[0][k], v[0][l]);
                m = __dadd_rn(m, __dmul_rn(v[1][k], v[1][l]));
                m = __dadd_rn(m, __dmul_rn(v[2][k], v[2][l]));
                m = __dadd_rn(m, __dmul_rn(sv[k], sv[l]));
                acc[q] = __dadd_rn(acc[q], __dmul_rn(w, m));
                ++q;
            }
    }
    for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int off = kMomentThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] = __dadd_rn(sh[k][threadIdx.x], sh[k][threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x < 10) partial[10 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_moments_final(const double* __restrict__ partial, int blocks, double* __restrict__ out)
{
    if (threadIdx.x >= 10) return;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s = __dadd_rn(s, partial[10 * b + threadIdx.x]);
    out[threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// device: cube-map cell of each face normal taken as a line.  Major axis k
// (lowest on ties); the normal is flipped so n_k > 0; the other components
// in (k+1, k+2) order are divided by n_k and binned into 32 cells per side.
// H[cell] += quantised area; rep[cell] = max of (qa << 31 | (2^31-1 - face)),
// i.e. the largest face, lowest id on ties.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_index(double u)
{
    int i = (int)floor(__dmul_rn(__dadd_rn(u, 1.0), (double)(kCells / 2)));
    return i < 0 ? 0 : (i > kCells - 1 ? kCells - 1 : i);
}

__global__ void k_normal_cells(const float* __restrict__ fnorm, const long long* __restrict__ cdf, int64_t T,
                               unsigned long long* __restrict__ H, unsigned long long* __restrict__ rep)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    const long long qa = cdf[f] - (f ? cdf[f - 1] : 0LL);
    if (qa <= 0) return;
    const double n[3] = {(double)fnorm[3 * f], (double)fnorm[3 * f + 1], (double)fnorm[3 * f + 2]};
    int k = 0;
    if (fabs(n[1]) > fabs(n[k])) k = 1;
    if (fabs(n[2]) > fabs(n[k])) k = 2;
    const double sg = n[k] < 0.0 ? -1.0 : 1.0;
    const double m = fabs(n[k]);
    const double u = __ddiv_rn(__dmul_rn(n[(k + 1) % 3], sg), m);
    const double v = __ddiv_rn(__dmul_rn(n[(k + 2) % 3], sg), m);
    const int cell = (k * kCells + cell_index(u)) * kCells + cell_index(v);
    atomicAdd(&H[cell], (unsigned long long)qa);
    atomicMax(&rep[cell], ((unsigned long long)qa << 31) | (unsigned long long)(0x7FFFFFFFLL - f));
}

// ---------------------------------------------------------------------------
// device: bounding boxes of the vertices in many FP64 frames G (columns).
// The defined coordinate is Q64 = fl64((x G0k + y G1k) + z G2k), its min and
// max over the vertices exact.  FP64 is slow on this part, so two passes:
//   A (fp32): Q32 with the fp32-rounded frame, per column its min and max
//     and the largest S32 = |x||g0k| + |y||g1k| + |z||g2k|;
//   B: vertices whose Q32 lies within W = 2^-19 max S32 of an fp32 extreme
//     get Q64, and only those enter the FP64 min / max.
// |Q32 - Q64| <= e = 4.1 * 2^-24 * S32 (rounding of the frame to fp32, two
// three-term dot products), so the vertex holding the FP64 extreme has Q32
// within 2 max e of the fp32 extreme; W = 2^-19 max S32 covers that twice,
// including the rounding of the threshold itself.  The result is exactly the
// one-pass FP64 result.  Block (x, g) handles a chunk of vertices for frame g;
// per block and column one atomic on order-preserving integers.
// ---------------------------------------------------------------------------
constexpr int kBoxThreads = 256;
constexpr int kBoxChunk = 8192;

__global__ void k_box_init(long long* box, int* box32, int nf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf * 6) box[i] = (i % 6) < 3 ? 0x7FFFFFFFFFFFFFFFLL : (long long)0x8000000000000000ULL;
    if (i < nf * 9) {
        const int c = i % 9;   // lo xyz, hi xyz, max S xyz
        box32[i] = c < 3 ? 0x7FFFFFFF : (c < 6 ? (int)0x80000000 : 0);
    }
}

__device__ __forceinline__ float dot32(float x, float y, float z, float g0, float g1, float g2)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(x, g0), __fmul_rn(y, g1)), __fmul_rn(z, g2));
}

__global__ void __launch_bounds__(kBoxThreads)
k_box_pass32(const float* __restrict__ V, int64_t nV, const double* __restrict__ G /*[nf][9]*/,
             int* __restrict__ box32 /*[nf][9]*/)
{
    const int g = blockIdx.y;
    float gm[9];
    for (int k = 0; k < 9; ++k) gm[k] = __double2float_rn(G[9 * g + k]);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, sm[3] = {0, 0, 0};
    const int64_t v0 = (int64_t)blockIdx.x * kBoxChunk;
    const int64_t v1 = min64(v0 + kBoxChunk, nV);
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const float x = V[3 * v], y = V[3 * v + 1], z = V[3 * v + 2];
        for (int k = 0; k < 3; ++k) {
            const float q = dot32(x, y, z, gm[k], gm[3 + k], gm[6 + k]);
            lo[k] = fminf(lo[k], q);
            hi[k] = fmaxf(hi[k], q);
            sm[k] = fmaxf(sm[k], dot32(fabsf(x), fabsf(y), fabsf(z), fabsf(gm[k]), fabsf(gm[3 + k]),
                                       fabsf(gm[6 + k])));
        }
    }
    for (int off = 16; off; off >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], off));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], off));
            sm[k] = fmaxf(sm[k], __shfl_xor_sync(0xFFFFFFFFu, sm[k], off));
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k)
            if (lo[k] <= hi[k]) {
                atomicMin(&box32[9 * g + k], float_to_ordered(lo[k]));
                atomicMax(&box32[9 * g + 3 + k], float_to_ordered(hi[k]));
                atomicMax(&box32[9 * g + 6 + k], float_to_ordered(sm[k]));
            }
}

__global__ void __launch_bounds__(kBoxThreads)
k_box_pass64(const float* __restrict__ V, int64_t nV, const double* __restrict__ G /*[nf][9]*/,
             const int* __restrict__ box32 /*[nf][9]*/, long long* __restrict__ box /*[nf][6]*/)
{
    const int g = blockIdx.y;
    double gd[9];
    float gm[9];
    for (int k = 0; k < 9; ++k) {
        gd[k] = G[9 * g + k];
        gm[k] = __double2float_rn(gd[k]);
    }
    float tlo[3], thi[3];
    for (int k = 0; k < 3; ++k) {
        const float w = ordered_to_float(box32[9 * g + 6 + k]) * 1.9073486328125e-06f;   // 2^-19
        tlo[k] = __fadd_rn(ordered_to_float(box32[9 * g + k]), w);
        thi[k] = __fsub_rn(ordered_to_float(box32[9 * g + 3 + k]), w);
    }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int64_t v0 = (int64_t)blockIdx.x * kBoxChunk;
    const int64_t v1 = min64(v0 + kBoxChunk, nV);
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const float x = V[3 * v], y = V[3 * v + 1], z = V[3 * v + 2];
        for (int k = 0; k < 3; ++k) {
            const float q32 = dot32(x, y, z, gm[k], gm[3 + k], gm[6 + k]);
            if (q32 <= tlo[k] || q32 >= thi[k]) {
                double q = __dadd_rn(__dmul_rn((double)x, gd[k]), __dmul_rn((double)y, gd[3 + k]));
                q = __dadd_rn(q, __dmul_rn((double)z, gd[6 + k]));
                lo[k] = fmin(lo[k], q);
                hi[k] = fmax(hi[k], q);
            }
        }
    }
    for (int off = 16; off; off >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], off));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], off));
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            if (lo[k] <= hi[k]) atomicMin(&box[6 * g + k], double_to_ordered(lo[k]));
            if (lo[k] <= hi[k]) atomicMax(&box[6 * g + 3 + k], double_to_ordered(hi[k]));
        }
}

// ---------------------------------------------------------------------------
// host: small FP64 linear algebra (one rounding per operation)
// ---------------------------------------------------------------------------
struct V3 { double x[3]; };

static double dot3(const V3& a, const V3& b) { return (a.x[0] * b.x[0] + a.x[1] * b.x[1]) + a.x[2] * b.x[2]; }

static V3 unit3(const V3& a)
{
    const double n = sqrt((a.x[0] * a.x[0] + a.x[1] * a.x[1]) + a.x[2] * a.x[2]);
    return V3{{a.x[0] / n, a.x[1] / n, a.x[2] / n}};
}

static V3 cross3(const V3& a, const V3& b)
{
    return V3{{a.x[1] * b.x[2] - a.x[2] * b.x[1], a.x[2] * b.x[0] - a.x[0] * b.x[2],
               a.x[0] * b.x[1] - a.x[1] * b.x[0]}};
}

// components to multiples of 2^-20 (nearest, halves to even; -0 becomes +0),
// sign so the largest-magnitude component (lowest index on ties) is positive
static V3 snap3(const V3& u)
{
    V3 w;
    for (int k = 0; k < 3; ++k) w.x[k] = nearbyint(u.x[k] * kSnap) / kSnap + 0.0;
    int m = 0;
    for (int k = 1; k < 3; ++k)
        if (fabs(w.x[k]) > fabs(w.x[m])) m = k;
    if (w.x[m] < 0.0)
        for (int k = 0; k < 3; ++k) w.x[k] = -w.x[k];
    return w;
}

// right-handed orthonormal frame with column ca along snap(u) and column cb
// along snap(v) made orthogonal to it; row-major FP64
static void frame_from(int ca, const V3& u, int cb, const V3& v, double R[9])
{
    const V3 ea = unit3(snap3(u));
    const V3 w = snap3(v);
    const double d = dot3(w, ea);
    const V3 eb = unit3(V3{{w.x[0] - d * ea.x[0], w.x[1] - d * ea.x[1], w.x[2] - d * ea.x[2]}});
    const int cc = 3 - ca - cb;
    const V3 ec = (ca + 1) % 3 == cb ? cross3(ea, eb) : cross3(eb, ea);
    for (int r = 0; r < 3; ++r) {
        R[3 * r + ca] = ea.x[r];
        R[3 * r + cb] = eb.x[r];
        R[3 * r + cc] = ec.x[r];
    }
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (Golub and Van Loan, Matrix Computations, Sec. 8.5): eigenvalues w
// descending, unit eigenvectors in the columns of U (row-major).
static void jacobi3(const double Min[9], double w[3], double U[9])
{
    double A[3][3];
    double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = Min[3 * i + j];
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {           // A <- A J
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {           // A <- J^T A
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {           // Q <- Q J
                    const double qkp = Q[k][p], qkq = Q[k][q];
                    Q[k][p] = c * qkp - s * qkq;
                    Q[k][q] = s * qkp + c * qkq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    std::stable_sort(idx, idx + 3, [&](int a, int b) { return A[a][a] > A[b][b]; });
    for (int c = 0; c < 3; ++c) {
        w[c] = A[idx[c]][idx[c]];
        for (int r = 0; r < 3; ++r) U[3 * r + c] = Q[r][idx[c]];
    }
}

// the RC_BOX_STEPS rotations about each column of base frame B (fp32, row
// major), in (column, j) order: column a held, b' = cos b + sin c,
// c' = cos c - sin b, tan(theta/2) = j / RC_BOX_STEPS
static void box_rotations(const float B32[9], std::vector<double>& G)
{
    double B[9];
    for (int k = 0; k < 9; ++k) B[k] = (double)B32[k];
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int j = 0; j < RC_BOX_STEPS; ++j) {
            const double t = (double)j / (double)RC_BOX_STEPS;
            const double t2 = t * t;
            const double den = 1.0 + t2;
            const double cs = (1.0 - t2) / den;
            const double sn = (2.0 * t) / den;
            double g[9];
            for (int k = 0; k < 9; ++k) g[k] = B[k];
            for (int r = 0; r < 3; ++r) {
                g[3 * r + b] = cs * B[3 * r + b] + sn * B[3 * r + c];
                g[3 * r + c] = cs * B[3 * r + c] - sn * B[3 * r + b];
            }
            G.insert(G.end(), g, g + 9);
        }
    }
}

static double box_volume(const long long* box6)
{
    double e[3];
    for (int k = 0; k < 3; ++k) e[k] = ordered_to_double(box6[3 + k]) - ordered_to_double(box6[k]);
    return (e[0] * e[1]) * e[2];
}

// device scratch freed in stream order when the scope ends, on every path
struct FrameScratch {
    cudaStream_t s;
    void* p[3] = {nullptr, nullptr, nullptr};
    ~FrameScratch()
    {
        for (void* q : p)
            if (q) cudaFreeAsync(q, s);
    }
};

static rc_status on_device(rc_bvh h)
{
    int dev = 0;
    RC_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) RC_CUDA(cudaSetDevice(h->device));
    return RC_OK;
}

// principal axes (F1): surface moments on the device, Jacobi on the host
static rc_status principal_frame(rc_bvh h, cudaStream_t s, double w[3], bool* ok, double R[9])
{
    *ok = false;
    w[0] = w[1] = w[2] = 0.0;
    double* part = nullptr;
    FrameScratch sf{s};
    RC_CUDA(cudaMallocAsync(&part, sizeof(double) * 10 * (kMomentBlocks + 1), s));
    sf.p[0] = part;
    const double r[3] = {0.5 * ((double)h->lo[0] + (double)h->hi[0]), 0.5 * ((double)h->lo[1] + (double)h->hi[1]),
                         0.5 * ((double)h->lo[2] + (double)h->hi[2])};
    k_moments<<<kMomentBlocks, kMomentThreads, 0, s>>>(h->V, h->F, h->farea, h->T, r[0], r[1], r[2], part);
    RC_LAUNCHED();
    k_moments_final<<<1, 32, 0, s>>>(part, kMomentBlocks, part + 10 * kMomentBlocks);
    RC_LAUNCHED();
    double m[10];
    RC_CUDA(cudaMemcpyAsync(m, part + 10 * kMomentBlocks, sizeof m, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    const double S0 = m[0];
    if (!(S0 > 0.0)) return RC_OK;
    const double c[3] = {m[1] / S0, m[2] / S0, m[3] / S0};
    double M[9];
    int q = 4;
    for (int k = 0; k < 3; ++k)
        for (int l = k; l < 3; ++l) {
            M[3 * k + l] = m[q] - S0 * (c[k] * c[l]);
            M[3 * l + k] = M[3 * k + l];
            ++q;
        }
    double U[9];
    jacobi3(M, w, U);
    if (!(w[0] > 0.0) || (w[0] - w[1]) <= kGap * w[0] || (w[1] - w[2]) <= kGap * w[0]) return RC_OK;
    frame_from(0, V3{{U[0], U[3], U[6]}}, 1, V3{{U[1], U[4], U[7]}}, R);
    *ok = true;
    return RC_OK;
}

// dominant normals (F2)
static rc_status normals_frame(rc_bvh h, cudaStream_t s, bool* ok, double R[9])
{
    *ok = false;
    unsigned long long* d = nullptr;
    RC_CUDA(cudaMallocAsync(&d, sizeof(unsigned long long) * 2 * kNumCells, s));
    RC_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * 2 * kNumCells, s));
    if (h->T > 0) {
        k_normal_cells<<<(unsigned)((h->T + 255) / 256), 256, 0, s>>>(h->fnorm, h->cdf, h->T, d, d + kNumCells);
        RC_LAUNCHED();
    }
    std::vector<unsigned long long> hr(2 * kNumCells);
    RC_CUDA(cudaMemcpyAsync(hr.data(), d, sizeof(unsigned long long) * 2 * kNumCells, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaFreeAsync(d, s));
    RC_CUDA(cudaStreamSynchronize(s));
    const unsigned long long* H = hr.data();
    const unsigned long long* rep = hr.data() + kNumCells;
    int c1 = -1;
    for (int c = 0; c < kNumCells; ++c)
        if (H[c] > 0 && (c1 < 0 || H[c] > H[c1])) c1 = c;
    if (c1 < 0) return RC_OK;
    auto face_normal = [&](int cell, V3* u) -> rc_status {
        const int64_t f = 0x7FFFFFFFLL - (int64_t)(rep[cell] & 0x7FFFFFFFULL);
        float nf[3];
        RC_CUDA(cudaMemcpy(nf, h->fnorm + 3 * f, sizeof nf, cudaMemcpyDeviceToHost));
        int k = 0;
        if (fabs((double)nf[1]) > fabs((double)nf[k])) k = 1;
        if (fabs((double)nf[2]) > fabs((double)nf[k])) k = 2;
        const double sg = nf[k] < 0.0f ? -1.0 : 1.0;
        for (int i = 0; i < 3; ++i) u->x[i] = (double)nf[i] * sg;
        return RC_OK;
    };
    V3 u1, u2;
    rc_status st = face_normal(c1, &u1);
    if (st != RC_OK) return st;
    const V3 e1 = unit3(snap3(u1));
    int c2 = -1;
    for (int c = 0; c < kNumCells; ++c) {
        if (H[c] == 0) continue;
        const int k = c / (kCells * kCells), i = (c / kCells) % kCells, j = c % kCells;
        V3 wv;
        wv.x[k] = 1.0;
        wv.x[(k + 1) % 3] = ((double)i + 0.5) / (double)(kCells / 2) - 1.0;
        wv.x[(k + 2) % 3] = ((double)j + 0.5) / (double)(kCells / 2) - 1.0;
        const double nw = sqrt((wv.x[0] * wv.x[0] + wv.x[1] * wv.x[1]) + wv.x[2] * wv.x[2]);
        if (fabs(dot3(wv, e1)) <= kOrtho * nw && (c2 < 0 || H[c] > H[c2])) c2 = c;
    }
    if (c2 < 0) return RC_OK;
    if ((st = face_normal(c2, &u2)) != RC_OK) return st;
    frame_from(2, u1, 0, u2, R);
    *ok = true;
    return RC_OK;
}

}  // namespace rc

using namespace rc;

extern "C" {

rc_status rc_frame_candidates(rc_bvh h, const rc_params* p, rc_frames* out, void* stream)
{
    RC_RANGE();
    if (!h || !out) return set_error(RC_E_ARG, "handle or output is NULL");
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if ((st = on_device(h)) != RC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    memset(out, 0, sizeof *out);
    out->best = -1;
    // base frames: given, principal axes, dominant normals (fp32)
    float bases[3][9];
    int bsrc[3], nb = 0;
    for (int k = 0; k < 9; ++k) bases[0][k] = p->frame[k];
    bsrc[nb++] = RC_FRAME_GIVEN;
    double R[9];
    bool ok = false;
    if ((st = principal_frame(h, s, out->principal, &ok, R)) != RC_OK) return st;
    if (ok) {
        for (int k = 0; k < 9; ++k) bases[nb][k] = (float)R[k];
        bsrc[nb++] = RC_FRAME_PRINCIPAL;
    }
    if ((st = normals_frame(h, s, &ok, R)) != RC_OK) return st;
    if (ok) {
        for (int k = 0; k < 9; ++k) bases[nb][k] = (float)R[k];
        bsrc[nb++] = RC_FRAME_NORMALS;
    }
    // box search: 3 x RC_BOX_STEPS rotations per base, all on the device
    std::vector<double> G;
    for (int b = 0; b < nb; ++b) box_rotations(bases[b], G);
    const int nf = (int)(G.size() / 9);
    const int64_t chunks = std::max<int64_t>(1, (h->nV + kBoxChunk - 1) / kBoxChunk);
    if (chunks > 0x7FFFFFFF) return set_error(RC_E_UNSUPPORTED, "too many vertices");
    double* dG = nullptr;
    long long* dbox = nullptr;
    int* dbox32 = nullptr;
    FrameScratch sf{s};
    RC_CUDA(cudaMallocAsync(&dG, sizeof(double) * G.size(), s));
    sf.p[0] = dG;
    RC_CUDA(cudaMallocAsync(&dbox, sizeof(long long) * 6 * nf, s));
    sf.p[1] = dbox;
    RC_CUDA(cudaMallocAsync(&dbox32, sizeof(int) * 9 * nf, s));
    sf.p[2] = dbox32;
    RC_CUDA(cudaMemcpyAsync(dG, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, s));
    k_box_init<<<(9 * nf + 255) / 256, 256, 0, s>>>(dbox, dbox32, nf);
    RC_LAUNCHED();
    k_box_pass32<<<dim3((unsigned)chunks, (unsigned)nf), kBoxThreads, 0, s>>>(h->V, h->nV, dG, dbox32);
    RC_LAUNCHED();
    k_box_pass64<<<dim3((unsigned)chunks, (unsigned)nf), kBoxThreads, 0, s>>>(h->V, h->nV, dG, dbox32, dbox);
    RC_LAUNCHED();
    std::vector<long long> box(6 * (size_t)nf);
    RC_CUDA(cudaMemcpyAsync(box.data(), dbox, sizeof(long long) * 6 * nf, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    // candidates: each base, then its best rotation, negative zeros made
    // positive; a frame whose axes are (up to sign and order) those of an
    // earlier candidate has the same six directions and is dropped
    auto same_axes = [](const float* A, const float* B) {
        for (int k = 0; k < 3; ++k) {
            bool found = false;
            for (int j = 0; j < 3 && !found; ++j) {
                bool eq = true, neg = true;
                for (int r = 0; r < 3; ++r) {
                    eq &= A[3 * r + k] == B[3 * r + j];
                    neg &= A[3 * r + k] == -B[3 * r + j];
                }
                found = eq || neg;
            }
            if (!found) return false;
        }
        return true;
    };
    auto add = [&](int src, const float f0[9], int a, int j) {
        float f[9];
        for (int k = 0; k < 9; ++k) f[k] = f0[k] + 0.0f;
        for (int c = 0; c < out->k; ++c)
            if (same_axes(f, out->frame[c])) return;
        const int c = out->k++;
        out->source[c] = src;
        out->box_axis[c] = a;
        out->box_step[c] = j;
        memcpy(out->frame[c], f, sizeof(float) * 9);
    };
    const int per = 3 * RC_BOX_STEPS;
    for (int b = 0; b < nb; ++b) {
        int best = 0;
        double bv = box_volume(&box[6 * (size_t)(b * per)]);
        for (int g = 1; g < per; ++g) {
            const double v = box_volume(&box[6 * (size_t)(b * per + g)]);
            if (v < bv) { bv = v; best = g; }
        }
        float fb[9];
        for (int k = 0; k < 9; ++k) fb[k] = (float)G[9 * (size_t)(b * per + best) + k];
        add(bsrc[b], bases[b], -1, -1);
        add(RC_FRAME_BOX + bsrc[b], fb, best / RC_BOX_STEPS, best % RC_BOX_STEPS);
    }
    // volumes of the fp32 candidate frames (as the casts use them)
    FrameDev* fds = nullptr;
    RC_CUDA(cudaMallocAsync(&fds, sizeof(FrameDev) * out->k, s));
    for (int c = 0; c < out->k && st == RC_OK; ++c) st = frame_setup_f(h, out->frame[c], fds + c, s);
    std::vector<FrameDev> hf(out->k);
    if (st == RC_OK)
        st = cudaMemcpyAsync(hf.data(), fds, sizeof(FrameDev) * out->k, cudaMemcpyDeviceToHost, s) == cudaSuccess
                 ? RC_OK : set_error(RC_E_CUDA, "frame copy failed");
    cudaFreeAsync(fds, s);
    if (st != RC_OK) return st;
    RC_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < out->k; ++c) out->volume[c] = box_volume(hf[c].box);
    return RC_OK;
}

rc_status rc_frame_select(rc_bvh h, const float* d_P, const float* d_N, const int32_t* d_face, int64_t n,
                          const rc_params* p, rc_frames* io, int64_t* d_counters, void* stream)
{
    RC_RANGE();
    if (!h || !io) return set_error(RC_E_ARG, "handle or frames is NULL");
    rc_status st = check_params_public(p);
    if (st != RC_OK) return st;
    if (io->k < 1 || io->k > RC_MAX_FRAMES) return set_error(RC_E_ARG, "frames.k must be in [1, RC_MAX_FRAMES]");
    for (int c = 0; c < io->k; ++c) {
        for (int k = 0; k < 9; ++k)
            if (!isfinite(io->frame[c][k])) return set_error(RC_E_ARG, "frame must be finite");
        for (int a = 0; a < 3; ++a)
            if (io->frame[c][a] == 0.0f && io->frame[c][3 + a] == 0.0f && io->frame[c][6 + a] == 0.0f)
                return set_error(RC_E_ARG, "frame columns (the machining axes) must be non-zero");
    }
    if (n < 0) return set_error(RC_E_ARG, "n must be >= 0");
    if (n > 0 && (!d_P || !d_N || !d_face)) return set_error(RC_E_ARG, "array pointer is NULL");
    if (p->collect_stats && !d_counters) return set_error(RC_E_ARG, "collect_stats needs the counters array");
    if ((st = on_device(h)) != RC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = io->k;
    // one stream-ordered block: frames, masks, travel, fixture flags, histograms
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t ofd = take(sizeof(FrameDev) * K), omask = take((size_t)K * n), otrav = take(sizeof(float) * 6 * K * n);
    const size_t ofix = take((size_t)h->T), ohist = take(sizeof(unsigned long long) * 68 * K);
    char* base = nullptr;
    RC_CUDA(cudaMallocAsync((void**)&base, off, s));
    FrameDev* fds = (FrameDev*)(base + ofd);
    uint8_t* mask = (uint8_t*)(base + omask);
    float* trav = (float*)(base + otrav);
    uint8_t* fixture = (uint8_t*)(base + ofix);
    unsigned long long* hist = (unsigned long long*)(base + ohist);
    std::vector<unsigned long long> hh(68 * (size_t)K);
    std::vector<FrameDev> hf(K);
    std::vector<float4*> ftrees(K, nullptr);
    do {
        if (cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 68 * K, s) != cudaSuccess) {
            st = set_error(RC_E_CUDA, "memset failed");
            break;
        }
        if (d_counters && cudaMemsetAsync(d_counters, 0, sizeof(int64_t) * (p->collect_stats ? 8 : 4), s) !=
                              cudaSuccess) {
            st = set_error(RC_E_CUDA, "memset failed");
            break;
        }
        for (int c = 0; c < K && st == RC_OK; ++c) {
            // each turned frame's axis rays walk the tree with boxes in its coordinates
            if (n > 0) st = make_frame_tree(h, io->frame[c], p, &ftrees[c], s);
            if (st == RC_OK) st = frame_setup_f(h, io->frame[c], fds + c, s, ftrees[c]);
        }
        if (st != RC_OK) break;
        if (n > 0) {
            st = launch_orthogonal_frames(h, d_P, d_N, n, p, fds, K, mask, trav, (unsigned long long*)d_counters, s);
            if (st != RC_OK) break;
        }
        // fixture faces and classes frame by frame (one fixture buffer, stream order)
        for (int c = 0; c < K && st == RC_OK; ++c)
            st = launch_classes(h, mask + (size_t)c * n, trav + (size_t)6 * c * n, d_face, n, p, nullptr,
                                fds[c].frame, fds[c].fbox, fixture, hist + 68 * c, s);
        if (st != RC_OK) break;
        if (cudaMemcpyAsync(hh.data(), hist, sizeof(unsigned long long) * 68 * K, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(hf.data(), fds, sizeof(FrameDev) * K, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = set_error(RC_E_CUDA, "result copy failed");
    } while (0);
    for (float4* t : ftrees)
        if (t) cudaFreeAsync(t, s);
    cudaFreeAsync(base, s);
    if (st != RC_OK) return st;
    RC_CUDA(cudaStreamSynchronize(s));
    io->best = -1;
    for (int c = 0; c < K; ++c) {
        rc_setups& su = io->setups[c];
        memset(&su, 0, sizeof su);
        for (int m = 0; m < 64; ++m) su.mask_hist[m] = (int64_t)hh[68 * c + m];
        for (int k = 0; k < 4; ++k) su.class_counts[k] = (int64_t)hh[68 * c + 64 + k];
        if ((st = rc_setup_cover(su.mask_hist, &su)) != RC_OK) return st;
        io->volume[c] = box_volume(hf[c].box);
    }
    // fewest setups, then fewest over-threshold + inaccessible, then the
    // smallest box, then the lowest index
    for (int c = 0; c < K; ++c) {
        if (io->best < 0) { io->best = c; continue; }
        const rc_setups& a = io->setups[c];
        const rc_setups& b = io->setups[io->best];
        const int64_t la = a.class_counts[1] + a.class_counts[2], lb = b.class_counts[1] + b.class_counts[2];
        if (a.setups_exact != b.setups_exact ? a.setups_exact < b.setups_exact
            : la != lb ? la < lb
            : io->volume[c] < io->volume[io->best])
            io->best = c;
    }
    return RC_OK;
}

}  // extern "C"
