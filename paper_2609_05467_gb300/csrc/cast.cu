// cast.cu -- any-hit occlusion traversal (Section 3.1 hemispherical cast,
// Section 3.2 orthogonal cast).
//
// Each ray/triangle pair is first decided in FP32 with the watertight test
// of Woop, Benthin and Wald (JCGT 2013) together with a forward error bound
// on its edge functions U, V, W, on det = U+V+W and on the unscaled
// plane-crossing value T' = U*az + V*bz + W*cz (see tri_test32).  The FP32
// outcome is accepted only when it is certain -- a clear hit outside the
// 1e-9 relative ambiguity band, or certainly no hit -- otherwise the pair is
// re-decided in FP64 (retest64), which evaluates the occlusion predicate
// directly (signed volumes against each edge, plane crossing N.a / N.d) and
// reports whether the pair lies inside the ambiguity band.  Box tests are
// conservative, so no triangle that can be hit at t > 0 is skipped: the
// 4-wide walk computes each slab distance with one FMA and widens it by a
// proven absolute margin (make_slab_ray), the binary walk scales the far
// distance by 1 + 2*gamma_3 (Ize, JCGT 2013).
//
// Kernels: k_hemisphere (the default cast: persistent warps, one point per
// warp in tiles of 32 directions, the last points in parts),
// k_hemisphere_update (re-cast after an edit), k_batch (many parts in one
// launch), k_orthogonal_axis (one frame axis for 32 points per work item),
// k_tool_cast_axis (the sampled ball-end tool), and the frame set-up
// kernels (k_frame_init, k_frame_box).
#include <math.h>

#include <algorithm>

#include "rc_internal.cuh"

namespace rc {

enum { kMiss = 0, kHit = 1, kUnsure = 2 };

struct Ray {
    float ox, oy, oz;
    float dx, dy, dz;
    float ix, iy, iz;   // 1/d (IEEE, +-inf for zero components)
    float Sx, Sy;       // watertight shear
    int kx, ky, kz;     // watertight permutation
    float rs;           // bound on max(1, |o|inf, |vertex|inf)
    float dkz;          // d[kz]
    float ef;           // sheared-coordinate error per unit of max |translated coordinate|
};

__device__ __forceinline__ float sel3(float a, float b, float c, int k)
{
    return k == 0 ? a : (k == 1 ? b : c);
}

__device__ __forceinline__ void setup_ray(Ray& r, float ox, float oy, float oz, float dx, float dy,
                                          float dz, float scene_maxabs)
{
    r.ox = ox; r.oy = oy; r.oz = oz;
    r.dx = dx; r.dy = dy; r.dz = dz;
    // reciprocals; a zero (or tiny) component gets +-2^100 instead of
    // +-inf, so slab products stay finite (no inf * 0 = NaN) and, 2^100
    // being a power of two, exact: such a slab is decided by the sign of
    // b - o alone
    r.ix = __frcp_rn(dx);
    r.iy = __frcp_rn(dy);
    r.iz = __frcp_rn(dz);
    if (!(fabsf(r.ix) <= 0x1p100f)) r.ix = copysignf(0x1p100f, dx);
    if (!(fabsf(r.iy) <= 0x1p100f)) r.iy = copysignf(0x1p100f, dy);
    if (!(fabsf(r.iz) <= 0x1p100f)) r.iz = copysignf(0x1p100f, dz);
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    int kz = ax >= ay ? (ax >= az ? 0 : 2) : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dk = sel3(dx, dy, dz, kz);
    if (dk < 0.0f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.dkz = dk;
    const float rk = __frcp_rn(dk);
    r.Sx = __fmul_rn(sel3(dx, dy, dz, kx), rk);
    r.Sy = __fmul_rn(sel3(dx, dy, dz, ky), rk);
    // translation rounds once (u|a|); a non-zero shear adds the rounding of
    // S (2u|S||a_z|: reciprocal and product), of a_z (u|S||a_z|) and of the
    // fused subtraction (u|A|); a zero shear leaves the subtraction exact
    const float sm = fmaxf(fabsf(r.Sx), fabsf(r.Sy));
    const float u = 5.9604644775390625e-8f;
    r.ef = sm == 0.0f ? 1.01f * u : (2.0f + 4.0f * sm) * 1.01f * u;
    r.rs = fmaxf(fmaxf(1.0f, scene_maxabs), fmaxf(fabsf(ox), fmaxf(fabsf(oy), fabsf(oz))));
}

// FP32 watertight test with a forward error bound.  Returns kHit only when
// the pair is certainly a clear hit (both outside the ambiguity band and
// certain in sign), kMiss only when it is certainly not a hit, else kUnsure.
//
// Error model (u = 2^-24, all translated coordinates |.| <= M, all sheared
// coordinates |.| <= P, S = max(|Sx|,|Sy|) <= 1 because kz is the largest |d|):
//   sheared coordinate error        E  <= (2 + 4 S) u M, and u M when S = 0
//                                        (the fused subtraction is then exact)
//   edge function error             eU <= 4 P E + 6 E^2 + 3 u P^2
//   det error                       eD <= 3 eU + 2.01 u S        (S = sum |U|)
//   plane-crossing error            eT <= eU Zs + 4.01 u S Zm    (Zs = sum |z|, Zm = max |z|)
// each scaled by 1.0625 for the rounding of the bound itself.
__device__ __forceinline__ int tri_test32(const Ray& r, const float4 v0, const float4 v1,
                                          const float4 v2)
{
    const float u = 5.9604644775390625e-8f;
    const float a0 = v0.x - r.ox, a1 = v0.y - r.oy, a2 = v0.z - r.oz;
    const float b0 = v1.x - r.ox, b1 = v1.y - r.oy, b2 = v1.z - r.oz;
    const float c0 = v2.x - r.ox, c1 = v2.y - r.oy, c2 = v2.z - r.oz;
    const float ax = sel3(a0, a1, a2, r.kx), ay = sel3(a0, a1, a2, r.ky), az = sel3(a0, a1, a2, r.kz);
    const float bx = sel3(b0, b1, b2, r.kx), by = sel3(b0, b1, b2, r.ky), bz = sel3(b0, b1, b2, r.kz);
    const float cx = sel3(c0, c1, c2, r.kx), cy = sel3(c0, c1, c2, r.ky), cz = sel3(c0, c1, c2, r.kz);
    const float Ax = fmaf(-r.Sx, az, ax), Ay = fmaf(-r.Sy, az, ay);
    const float Bx = fmaf(-r.Sx, bz, bx), By = fmaf(-r.Sy, bz, by);
    const float Cx = fmaf(-r.Sx, cz, cx), Cy = fmaf(-r.Sy, cz, cy);
    const float U = fmaf(Cx, By, -(Cy * Bx));
    const float V = fmaf(Ax, Cy, -(Ay * Cx));
    const float W = fmaf(Bx, Ay, -(By * Ax));

    const float M = fmaxf(fmaxf(fmaxf(fabsf(a0), fabsf(a1)), fmaxf(fabsf(a2), fabsf(b0))),
                          fmaxf(fmaxf(fabsf(b1), fabsf(b2)), fmaxf(fmaxf(fabsf(c0), fabsf(c1)), fabsf(c2))));
    const float P = fmaxf(fmaxf(fmaxf(fabsf(Ax), fabsf(Ay)), fmaxf(fabsf(Bx), fabsf(By))),
                          fmaxf(fabsf(Cx), fabsf(Cy)));
    const float E = r.ef * M;
    const float eU = (4.0f * E * P + 6.0f * E * E + 3.0f * u * P * P) * 1.0625f;
    const bool uc = fabsf(U) > eU, vc = fabsf(V) > eU, wc = fabsf(W) > eU;
    const bool pos = (uc && U > 0.0f) || (vc && V > 0.0f) || (wc && W > 0.0f);
    const bool neg = (uc && U < 0.0f) || (vc && V < 0.0f) || (wc && W < 0.0f);
    if (pos && neg) return kMiss;

    const float S = fabsf(U) + fabsf(V) + fabsf(W);
    const float det = U + V + W;
    const float Tp = fmaf(U, az, fmaf(V, bz, W * cz));
    const float Zs = fabsf(az) + fabsf(bz) + fabsf(cz);
    const float Zm = fmaxf(fabsf(az), fmaxf(fabsf(bz), fabsf(cz)));
    const float eD = (3.0f * eU + 2.01f * u * S) * 1.0625f;
    const float eT = (eU * Zs + 4.01f * u * S * Zm) * 1.0625f;
    const bool det_ok = fabsf(det) > eD;
    const bool tp_ok = fabsf(Tp) > eT;
    // sign of t = sign(T') * sign(det) * sign(d[kz])
    const bool ahead = ((Tp > 0.0f) == (det > 0.0f)) == (r.dkz > 0.0f);
    if (det_ok && tp_ok && !ahead) return kMiss;   // plane crossed behind the origin

    // clear hit: every edge function beyond its error and the tau band, and
    // the crossing ahead and beyond tau*R along the ray
    const float tau_edge = 3.0f * 1e-9f * r.rs * v0.w * 1.01f;
    const float thr = eU + tau_edge;
    if (fabsf(U) > thr && fabsf(V) > thr && fabsf(W) > thr && tp_ok && ahead) {
        const float need = eT + 1e-9f * r.rs * (fabsf(det) + eD) * 1.01f;
        if (fabsf(Tp) > need) return kHit;
    }
    return kUnsure;
}

// FP64 decision of one pair, written from the definition: the ray's line
// meets the closed triangle iff the signed volumes of the ray direction with
// each edge (relative to the origin) do not take both signs; the plane is
// crossed at t = (N.a)/(N.d).  `state` is kMiss / kHit / kUnsure (= the
// pair lies in the 1e-9 relative ambiguity band); `hit64` is the plain FP64
// sign decision (used for rays that only ambiguous pairs decide).
struct Pair64 { int state; bool hit64; };

__device__ __noinline__ Pair64 retest64(const Ray& r, const float4 v0, const float4 v1, const float4 v2)
{
    const double o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
    const double A[3] = {v0.x, v0.y, v0.z}, B[3] = {v1.x, v1.y, v1.z}, C[3] = {v2.x, v2.y, v2.z};
    double a[3], b[3], c[3], eab[3], ebc[3], eca[3];
    double R = 1.0;
    for (int k = 0; k < 3; ++k) {
        a[k] = A[k] - o[k];
        b[k] = B[k] - o[k];
        c[k] = C[k] - o[k];
        eab[k] = B[k] - A[k];
        ebc[k] = C[k] - B[k];
        eca[k] = A[k] - C[k];
        R = fmax(R, fmax(fabs(o[k]), fmax(fabs(A[k]), fmax(fabs(B[k]), fabs(C[k])))));
    }
    const double band = kTau * R;
    // signed volume of (p, e, d) and |e x d| for the three edges
    const double* P3[3] = {b, c, a};
    const double* E3[3] = {ebc, eca, eab};
    double Ev[3], Lv[3];
    for (int k = 0; k < 3; ++k) {
        const double* p = P3[k];
        const double* e = E3[k];
        const double w0 = p[1] * e[2] - p[2] * e[1];
        const double w1 = p[2] * e[0] - p[0] * e[2];
        const double w2 = p[0] * e[1] - p[1] * e[0];
        Ev[k] = w0 * d[0] + w1 * d[1] + w2 * d[2];
        const double x0 = e[1] * d[2] - e[2] * d[1];
        const double x1 = e[2] * d[0] - e[0] * d[2];
        const double x2 = e[0] * d[1] - e[1] * d[0];
        Lv[k] = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
    }
    Pair64 res;
    const bool spos = Ev[0] > 0.0 || Ev[1] > 0.0 || Ev[2] > 0.0;
    const bool sneg = Ev[0] < 0.0 || Ev[1] < 0.0 || Ev[2] < 0.0;
    // N = (B-A) x (C-A) = eab x (-eca)
    const double N0 = -(eab[1] * eca[2] - eab[2] * eca[1]);
    const double N1 = -(eab[2] * eca[0] - eab[0] * eca[2]);
    const double N2 = -(eab[0] * eca[1] - eab[1] * eca[0]);
    const double nd = N0 * d[0] + N1 * d[1] + N2 * d[2];
    const double na = N0 * a[0] + N1 * a[1] + N2 * a[2];
    res.hit64 = !(spos && sneg) && nd != 0.0 && na != 0.0 && ((na > 0.0) == (nd > 0.0));

    bool pos = false, neg = false, small = false;
    for (int k = 0; k < 3; ++k) {
        if (fabs(Ev[k]) <= band * Lv[k]) { small = true; continue; }
        if (Ev[k] > 0.0) pos = true; else neg = true;
    }
    if (pos && neg) { res.state = kMiss; return res; }
    if (nd == 0.0) { res.state = small ? kUnsure : kMiss; return res; }
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (fabs(na) * dn <= band * fabs(nd)) { res.state = kUnsure; return res; }
    if ((na > 0.0) != (nd > 0.0)) { res.state = kMiss; return res; }
    res.state = small ? kUnsure : kHit;
    return res;
}

// Conservative slab test of both children of a packed node.
__device__ __forceinline__ void box2(const Ray& r, const float4 n0, const float4 n1, const float4 n2,
                                     bool& h0, bool& h1, float& t0, float& t1)
{
    const float rob = 1.0f + 2.0f * 1.7881394e-7f;   // 1 + 2*gamma_3, gamma_3 = 3u/(1-3u)
    const bool sx = signbit(r.ix), sy = signbit(r.iy), sz = signbit(r.iz);
    // child 0: (n0.x lo_x, n0.y hi_x, n0.z lo_y, n0.w hi_y, n2.x lo_z, n2.y hi_z)
    float nx = ((sx ? n0.y : n0.x) - r.ox) * r.ix, fx = ((sx ? n0.x : n0.y) - r.ox) * r.ix;
    float ny = ((sy ? n0.w : n0.z) - r.oy) * r.iy, fy = ((sy ? n0.z : n0.w) - r.oy) * r.iy;
    float nz = ((sz ? n2.y : n2.x) - r.oz) * r.iz, fz = ((sz ? n2.x : n2.y) - r.oz) * r.iz;
    float tn = fmaxf(fmaxf(nx, ny), fmaxf(nz, 0.0f));
    float tf = fminf(fminf(fx, fy), fz) * rob;
    h0 = tn <= tf;
    t0 = tn;
    // child 1: (n1.x lo_x, n1.y hi_x, n1.z lo_y, n1.w hi_y, n2.z lo_z, n2.w hi_z)
    nx = ((sx ? n1.y : n1.x) - r.ox) * r.ix; fx = ((sx ? n1.x : n1.y) - r.ox) * r.ix;
    ny = ((sy ? n1.w : n1.z) - r.oy) * r.iy; fy = ((sy ? n1.z : n1.w) - r.oy) * r.iy;
    nz = ((sz ? n2.w : n2.z) - r.oz) * r.iz; fz = ((sz ? n2.z : n2.w) - r.oz) * r.iz;
    tn = fmaxf(fmaxf(nx, ny), fmaxf(nz, 0.0f));
    tf = fminf(fminf(fx, fy), fz) * rob;
    h1 = tn <= tf;
    t1 = tn;
}

// Per-warp-lane counters of a cast.
struct CastAccFwd {
    int amb = 0, retests = 0, overflow = 0;
    long long rays = 0, nvis = 0, ntri = 0;
};

// Result bits of trace(): bit 0 blocked, bit 1 decided by ambiguous pairs.
// With kStats the walk also counts interior-node fetches and triangle tests
// (the instrumented build used to measure algorithmic bytes per ray).
struct TraceOut { int flags; int retests; int overflow; int nodes; int tris; };

template <bool kStats>
__device__ __forceinline__ TraceOut trace(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                          const Ray& r, int max_steps)
{
    TraceOut out = {0, 0, 0, 0, 0};
    int stack[kStack];
    int sp = 0;
    int cur = 0;
    bool amb = false, ambhit = false;
    // a well-formed tree visits each node at most once, so max_steps (the
    // node count) is never reached; the cap only bounds a malformed tree
    for (int steps = 0;; ++steps) {
        if (steps > max_steps) { out.overflow = 1; out.flags = 1; return out; }
        if (cur >= 0) {
            if (kStats) ++out.nodes;
            const float4 n0 = __ldg(&nodes[4 * cur + 0]);
            const float4 n1 = __ldg(&nodes[4 * cur + 1]);
            const float4 n2 = __ldg(&nodes[4 * cur + 2]);
            const float4 n3 = __ldg(&nodes[4 * cur + 3]);
            bool h0, h1;
            float t0, t1;
            box2(r, n0, n1, n2, h0, h1, t0, t1);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                if (sp >= kStack) { out.overflow = 1; out.flags = 1; return out; }
                stack[sp++] = first0 ? c1 : c0;
                cur = first0 ? c0 : c1;
                continue;
            }
            if (h0) { cur = c0; continue; }
            if (h1) { cur = c1; continue; }
        } else {
            const int v = -1 - cur;
            const int first = v >> 3, cnt = (v & 7) + 1;
            for (int k = 0; k < cnt; ++k) {
                const float4* t = tris + 3 * (first + k);
                const float4 v0 = __ldg(t), v1 = __ldg(t + 1), v2 = __ldg(t + 2);
                if (kStats) ++out.tris;
                const int s = tri_test32(r, v0, v1, v2);
                if (s == kHit) { out.flags = 1; return out; }
                if (s == kUnsure) {
                    ++out.retests;
                    const Pair64 p = retest64(r, v0, v1, v2);
                    if (p.state == kHit) { out.flags = 1; return out; }
                    if (p.state == kUnsure) { amb = true; ambhit |= p.hit64; }
                }
            }
        }
        if (sp == 0) break;
        cur = stack[--sp];
    }
    out.flags = (ambhit ? 1 : 0) | (amb ? 2 : 0);
    return out;
}

// Any-hit walk of the 4-wide tree: the same ray, box and triangle decisions
// as trace(); per node the four child boxes are tested together, the
// nearest hit child is visited next and the others are pushed (the default
// walk orders them only partly, the while-while walk fully, far-to-near).
// Per-ray constants of the 4-wide slab test.  A slab distance is one FMA,
// t = b * i - o * i, with the near / far bound of each axis picked by the
// load address (the node stores lo and hi of an axis in adjacent float4s).
// Conservative: with u = 2^-24, i = fl(1/d), M >= |every box coordinate|,
// the computed b*i - fl(o*i) differs from (b - o)/d by at most
// 2u|t| + 2u|o i| (+ lower-order terms) <= 4.01 u (M + |o|) |i|; every near
// distance is lowered and every far distance raised by E = 5 u (M + |o|) |i|
// (folded into the subtracted constant, its rounding included), so a box
// the exact ray enters is never rejected.  An axis with i = +-2^100 (the
// direction has no component along it) needs no margin: see setup_ray.
struct SlabRay {
    float ix, iy, iz;
    float nox, noy, noz;    // o * i + E  (subtracted for near distances)
    float fox, foy, foz;    // o * i - E  (subtracted for far distances)
    int offx, offy, offz;   // 1 when the axis runs backwards: near = hi
};

__device__ __forceinline__ SlabRay make_slab_ray(const Ray& r, float M)
{
    const float u = 5.9604644775390625e-8f;
    SlabRay s;
    s.ix = r.ix; s.iy = r.iy; s.iz = r.iz;
    // a +-2^100 reciprocal (axis parallel to the slab) makes b*i and o*i
    // exact, so only the sign-preserving final rounding remains: no margin
    const float ex = fabsf(r.ix) == 0x1p100f ? 0.0f : 5.0f * u * ((M + fabsf(r.ox)) * fabsf(r.ix));
    const float ey = fabsf(r.iy) == 0x1p100f ? 0.0f : 5.0f * u * ((M + fabsf(r.oy)) * fabsf(r.iy));
    const float ez = fabsf(r.iz) == 0x1p100f ? 0.0f : 5.0f * u * ((M + fabsf(r.oz)) * fabsf(r.iz));
    const float oix = r.ox * r.ix, oiy = r.oy * r.iy, oiz = r.oz * r.iz;
    s.nox = oix + ex; s.noy = oiy + ey; s.noz = oiz + ez;
    s.fox = oix - ex; s.foy = oiy - ey; s.foz = oiz - ez;
    s.offx = signbit(r.ix) ? 1 : 0;
    s.offy = signbit(r.iy) ? 1 : 0;
    s.offz = signbit(r.iz) ? 1 : 0;
    return s;
}

// Slab test of the four children of wide node nd: d[k] = entry distance of a
// hit child (else +inf), c[k] = child index; returns the number of hits.
// kShared: nd is a frontier group in shared memory (the same layout).
template <bool kShared = false>
__device__ __forceinline__ float4 node_ld(const float4* p)
{
    if (kShared) return *p;
    return __ldg(p);
}

template <bool kShared = false>
__device__ __forceinline__ int slab4(const float4* __restrict__ nd, const SlabRay& s, float d[4], int c[4])
{
    const float4 nxv = node_ld<kShared>(nd + 0 + s.offx), fxv = node_ld<kShared>(nd + 1 - s.offx);
    const float4 nyv = node_ld<kShared>(nd + 2 + s.offy), fyv = node_ld<kShared>(nd + 3 - s.offy);
    const float4 nzv = node_ld<kShared>(nd + 4 + s.offz), fzv = node_ld<kShared>(nd + 5 - s.offz);
    const float4 ci = node_ld<kShared>(nd + 6);
    const float nx[4] = {nxv.x, nxv.y, nxv.z, nxv.w}, fx[4] = {fxv.x, fxv.y, fxv.z, fxv.w};
    const float ny[4] = {nyv.x, nyv.y, nyv.z, nyv.w}, fy[4] = {fyv.x, fyv.y, fyv.z, fyv.w};
    const float nz[4] = {nzv.x, nzv.y, nzv.z, nzv.w}, fz[4] = {fzv.x, fzv.y, fzv.z, fzv.w};
    const int cc[4] = {__float_as_int(ci.x), __float_as_int(ci.y), __float_as_int(ci.z), __float_as_int(ci.w)};
    int nh = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float tn = fmaxf(fmaxf(fmaf(nx[k], s.ix, -s.nox), fmaf(ny[k], s.iy, -s.noy)),
                               fmaxf(fmaf(nz[k], s.iz, -s.noz), 0.0f));
        const float tf = fminf(fminf(fmaf(fx[k], s.ix, -s.fox), fmaf(fy[k], s.iy, -s.foy)),
                               fmaf(fz[k], s.iz, -s.foz));
        const bool hit = tn <= tf;
        d[k] = hit ? tn : INFINITY;
        c[k] = cc[k];
        nh += hit;
    }
    return nh;
}

// ---------------------------------------------------------------------------
// Per-point frontier of the 4-wide walk.  All hemisphere rays of a point
// start at the same origin o, and a box that contains o is entered by every
// one of them: its near slab distances are <= 0 and its far ones >= 0, and
// the conservative margin only lowers the near and raises the far ones.  So
// every ray's walk from the root visits the same nodes whose boxes contain o
// (the origin set: the root and every child box containing o below it).
// The warp finds that set once per point and keeps in shared memory what
// each ray must still decide for itself: the triangles of the leaves whose
// boxes contain o (local triangles), and the children of origin-set nodes
// whose boxes do not contain o (the frontier, in the wide node's layout,
// four entries per group).  A ray tests the local triangles, tests every
// frontier box with its own slab test and walks the subtrees it enters:
// exactly the triangles its walk from the root would test, so the same
// decisions.  A local triangle wholly below the point's tangent plane is
// dropped, because a hemisphere ray leaves that plane (d.n > 0 for every
// direction of the set, N <= 65536, when n is of unit length to within the
// rounding of an fp32 normal) and meets no point of it at t > 0; that
// exact FP64 test runs once per point.  For the same reason a frontier box
// wholly below the plane is dropped, and so is a frontier leaf whose
// triangles all lie below it (conservative fp32 tests).  A point whose frontier or local
// triangles do not fit walks from the root instead.
// ---------------------------------------------------------------------------
constexpr int kFrontGroups = 16;   // frontier entries, four per group
constexpr int kFrontTris = 12;     // local triangles kept per point
constexpr int kStackF = kStack4 + 4 * kFrontGroups;

struct Frontier {
    float4 grp[kFrontGroups * 7];  // per group: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of 4 entries, their codes
    float4 tri[kFrontTris * 3];    // local triangle records
    int ngroups, ntris, ok, nvis;
};

// n . (v - o) < 0 for the three vertices, in FP64: the differences of fp32
// values are exact there and the products and sums round far below the
// margin taken (4e-15 of the sum of the terms' magnitudes)
__device__ __forceinline__ bool below_tangent(float4 v, float ox, float oy, float oz, float nx, float ny, float nz)
{
    const double a = (double)v.x - ox, b = (double)v.y - oy, c = (double)v.z - oz;
    const double s = __dadd_rn(__dadd_rn(__dmul_rn((double)nx, a), __dmul_rn((double)ny, b)), __dmul_rn((double)nz, c));
    const double m = fabs((double)nx * a) + fabs((double)ny * b) + fabs((double)nz * c);
    return s < -4e-15 * m;
}

// Shortcuts that skip what lies below a point's tangent plane need every
// direction of the set above it.  With |n|^2 = 1 + delta the basis tilts by
// about |delta|, so d.n >= z_min - 3 |delta| - 1e-6 with z_min = 1/(2N) >=
// 1/(64 W) (W = ceil(N/32)); a normal further from unit length takes none.
__device__ __forceinline__ bool tangent_shortcuts_ok(float nx, float ny, float nz, int W)
{
    const double nn = (double)nx * nx + (double)ny * ny + (double)nz * nz;
    return fabs(nn - 1.0) <= 0.25 * (1.0 / (64.0 * W) - 2e-6);
}

// A box wholly below the tangent plane through o: the largest n.(x - o) over
// its corners, sum over the axes of max(n_k (lo_k - o_k), n_k (hi_k - o_k)),
// is negative beyond the rounding of its fp32 evaluation (each difference,
// product and sum rounds once: under 4u of the sum of the terms' magnitudes,
// 8u taken).  Every triangle inside such a box is wholly below the plane too.
__device__ __forceinline__ bool box_below_tangent(float lx, float hx, float ly, float hy, float lz, float hz,
                                                  float ox, float oy, float oz, float nx, float ny, float nz)
{
    const float mx = fmaxf(nx * (lx - ox), nx * (hx - ox));
    const float my = fmaxf(ny * (ly - oy), ny * (hy - oy));
    const float mz = fmaxf(nz * (lz - oz), nz * (hz - oz));
    const float u = 5.9604644775390625e-8f;
    return (mx + my) + mz < -8.0f * u * (fabsf(mx) + fabsf(my) + fabsf(mz));
}

// Lane 0 of the warp: the origin set of o (a walk over the boxes that
// contain o), its frontier and local triangles into *f.
__device__ __noinline__ void build_frontier(const float4* __restrict__ wnodes, const float4* __restrict__ tris,
                                            int max_steps, float ox, float oy, float oz, float nx, float ny,
                                            float nz, bool drop, Frontier* f)
{
    int qs[kStack4];
    int qsp = 0;
    qs[qsp++] = 0;
    int ne = 0, nt = 0, nvis = 0;
    bool ok = true;
    float* g = (float*)f->grp;
    while (qsp > 0 && ok) {
        if (++nvis > max_steps) { ok = false; break; }
        const int cur = qs[--qsp];
        const float4* nd = wnodes + 8 * (int64_t)cur;
        const float4 lxv = __ldg(nd), hxv = __ldg(nd + 1), lyv = __ldg(nd + 2), hyv = __ldg(nd + 3);
        const float4 lzv = __ldg(nd + 4), hzv = __ldg(nd + 5), civ = __ldg(nd + 6);
        const float LX[4] = {lxv.x, lxv.y, lxv.z, lxv.w}, HX[4] = {hxv.x, hxv.y, hxv.z, hxv.w};
        const float LY[4] = {lyv.x, lyv.y, lyv.z, lyv.w}, HY[4] = {hyv.x, hyv.y, hyv.z, hyv.w};
        const float LZ[4] = {lzv.x, lzv.y, lzv.z, lzv.w}, HZ[4] = {hzv.x, hzv.y, hzv.z, hzv.w};
        const int CI[4] = {__float_as_int(civ.x), __float_as_int(civ.y), __float_as_int(civ.z), __float_as_int(civ.w)};
        for (int k = 0; k < 4 && ok; ++k) {
            if (!(LX[k] <= HX[k])) continue;   // empty slot (its code -1 is also a leaf's)
            const bool inside = LX[k] <= ox && ox <= HX[k] && LY[k] <= oy && oy <= HY[k] && LZ[k] <= oz &&
                                oz <= HZ[k];
            if (inside && CI[k] >= 0) {
                if (qsp >= kStack4) { ok = false; break; }
                qs[qsp++] = CI[k];
            } else if (inside) {
                const int v = -1 - CI[k], first = v >> 3, cnt = (v & 7) + 1;
                for (int t = 0; t < cnt; ++t) {
                    const float4* tp = tris + 3 * (int64_t)(first + t);
                    const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
                    if (drop && below_tangent(v0, ox, oy, oz, nx, ny, nz) &&
                        below_tangent(v1, ox, oy, oz, nx, ny, nz) && below_tangent(v2, ox, oy, oz, nx, ny, nz))
                        continue;
                    if (nt >= kFrontTris) { ok = false; break; }
                    f->tri[3 * nt] = v0;
                    f->tri[3 * nt + 1] = v1;
                    f->tri[3 * nt + 2] = v2;
                    ++nt;
                }
            } else {
                // a box below the tangent plane holds no hit of any ray of the
                // point, and neither does a leaf whose triangles all lie below it
                if (drop && box_below_tangent(LX[k], HX[k], LY[k], HY[k], LZ[k], HZ[k], ox, oy, oz, nx, ny, nz))
                    continue;
                if (drop && CI[k] < 0) {
                    const int v = -1 - CI[k], first = v >> 3, cnt = (v & 7) + 1;
                    bool below = true;
                    for (int t = 0; t < cnt && below; ++t) {
                        const float4* tp = tris + 3 * (int64_t)(first + t);
                        for (int q = 0; q < 3 && below; ++q) {
                            const float4 w = __ldg(tp + q);
                            below = box_below_tangent(w.x, w.x, w.y, w.y, w.z, w.z, ox, oy, oz, nx, ny, nz);
                        }
                    }
                    if (below) continue;
                }
                if (ne >= 4 * kFrontGroups) { ok = false; break; }
                float* gp = g + 28 * (ne >> 2) + (ne & 3);
                gp[0] = LX[k]; gp[4] = HX[k]; gp[8] = LY[k]; gp[12] = HY[k]; gp[16] = LZ[k]; gp[20] = HZ[k];
                gp[24] = __int_as_float(CI[k]);
                ++ne;
            }
        }
    }
    // the last group's unused slots: empty boxes, which no slab test enters
    for (int e = ne; e < ((ne + 3) & ~3); ++e) {
        float* gp = g + 28 * (e >> 2) + (e & 3);
        gp[0] = INFINITY; gp[4] = -INFINITY; gp[8] = INFINITY; gp[12] = -INFINITY; gp[16] = INFINITY;
        gp[20] = -INFINITY;
        gp[24] = __int_as_float(-1);
    }
    f->ngroups = (ne + 3) >> 2;
    f->ntris = nt;
    f->ok = ok ? 1 : 0;
    f->nvis = nvis;
}

template <bool kStats>
__device__ __forceinline__ TraceOut trace4(const float4* __restrict__ wnodes, const float4* __restrict__ tris,
                                           const Ray& r, int max_steps, const Frontier* front = nullptr)
{
    TraceOut out = {0, 0, 0, 0, 0};
    int stack[kStackF];
    int sp = 0;
    int cur = 0;
    bool amb = false, ambhit = false;
    const SlabRay sr = make_slab_ray(r, r.rs);
    if (front) {
        // the point's local triangles, then its frontier boxes: the entered
        // ones go on the stack, the deepest (nearest the origin) on top
        for (int t = 0; t < front->ntris; ++t) {
            const float4 v0 = front->tri[3 * t], v1 = front->tri[3 * t + 1], v2 = front->tri[3 * t + 2];
            if (kStats) ++out.tris;
            const int st = tri_test32(r, v0, v1, v2);
            if (st == kHit) { out.flags = 1; return out; }
            if (st == kUnsure) {
                ++out.retests;
                const Pair64 p = retest64(r, v0, v1, v2);
                if (p.state == kHit) { out.flags = 1; return out; }
                if (p.state == kUnsure) { amb = true; ambhit |= p.hit64; }
            }
        }
        for (int gi = 0; gi < front->ngroups; ++gi) {
            if (kStats) ++out.nodes;
            float d[4];
            int c[4];
            slab4<true>(front->grp + 7 * gi, sr, d, c);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (d[k] != INFINITY) stack[sp++] = c[k];
        }
        if (sp == 0) {
            out.flags = (ambhit ? 1 : 0) | (amb ? 2 : 0);
            return out;
        }
        cur = stack[--sp];
    }
    for (int steps = 0;; ++steps) {
        if (steps > max_steps) { out.overflow = 1; out.flags = 1; return out; }
        if (cur >= 0) {
            if (kStats) ++out.nodes;
            float d[4];
            int c[4];
            const int nh = slab4(wnodes + 8 * cur, sr, d, c);
            if (nh == 0) {
                if (sp == 0) break;
                cur = stack[--sp];
                continue;
            }
#define RC_CSWAP(a, b)                                              \
    if (d[b] < d[a]) {                                              \
        const float td = d[a]; d[a] = d[b]; d[b] = td;              \
        const int tc = c[a]; c[a] = c[b]; c[b] = tc;                \
    }
            // three of the five exchanges of the sorting network: the nearest
            // child reaches slot 0 and the others stay partly ordered (faster
            // than the full network, and no more nodes visited)
            RC_CSWAP(0, 1) RC_CSWAP(2, 3) RC_CSWAP(0, 2)
#undef RC_CSWAP
            if (sp + nh - 1 > kStackF) { out.overflow = 1; out.flags = 1; return out; }
            if (d[3] != INFINITY) stack[sp++] = c[3];
            if (d[2] != INFINITY) stack[sp++] = c[2];
            if (d[1] != INFINITY) stack[sp++] = c[1];
            cur = c[0];
            continue;
        } else {
            const int v = -1 - cur;
            const int first = v >> 3, cnt = (v & 7) + 1;
            for (int k = 0; k < cnt; ++k) {
                const float4* t = tris + 3 * (first + k);
                const float4 v0 = __ldg(t), v1 = __ldg(t + 1), v2 = __ldg(t + 2);
                if (kStats) ++out.tris;
                const int s = tri_test32(r, v0, v1, v2);
                if (s == kHit) { out.flags = 1; return out; }
                if (s == kUnsure) {
                    ++out.retests;
                    const Pair64 p = retest64(r, v0, v1, v2);
                    if (p.state == kHit) { out.flags = 1; return out; }
                    if (p.state == kUnsure) { amb = true; ambhit |= p.hit64; }
                }
            }
        }
        if (sp == 0) break;
        cur = stack[--sp];
    }
    out.flags = (ambhit ? 1 : 0) | (amb ? 2 : 0);
    return out;
}

template <bool kStats, bool kWide>
__device__ __forceinline__ TraceOut trace_any(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                              const Ray& r, int max_steps, const Frontier* front = nullptr)
{
    if (kWide) return trace4<kStats>(nodes, tris, r, max_steps, front);
    return trace<kStats>(nodes, tris, r, max_steps);
}

// ---------------------------------------------------------------------------
// Axis rays (Section 3.2: rays along the six principal directions of the
// machining frame).  Their walk tests the child boxes of the frame's own tree
// (the same nodes with boxes in frame coordinates, FrameDev::tree) and the
// triangles in world coordinates, exactly as the hemispherical walk does.
// A ray o + t d, d = +-column k of the fp32 frame F, has frame coordinates
// q(o) + t F^T d = q(o) +- t G[:, k] (G = F^T F): along k they grow (shrink)
// with t, and across k they drift by at most t |G[j][k]|, a few ulps times
// t for an fp32 frame.  Every hit lies in the part's box, so t is at most
// (|o - c| + r) / |d| (c, r: the box's centre and half diagonal).  The ray
// can therefore only meet triangles whose frame boxes overlap the band
// [q_j(o) - tol_j, q_j(o) + tol_j] across k and lie on its side of q_k(o)
// along k, where tol_j covers that drift, the 1e-9 R ambiguity band and the
// FP64 rounding of q and of the boxes; the band is rounded outward to fp32.
// For the identity frame the drift is zero and the tree is the world tree.
// A ray along a wall 1e-4 mm above it, which the world boxes of a turned
// part's wall triangles all admit, lies outside their frame boxes.
// ---------------------------------------------------------------------------
struct AxisRay {
    float lo[3], hi[3];   // frame-coordinate band the ray can reach (+-inf on its far side along k)
    int k;                // frame axis of the ray
    int pos;              // 1: along +column k, 0: along -column k
};

__device__ __forceinline__ AxisRay make_axis_ray(const FrameDev& fd, int a, float ox, float oy, float oz, float rs)
{
    AxisRay ar;
    const int k = a >> 1;
    const bool pos = (a & 1) == 0;
    const double x = ox, y = oy, z = oz;
    double q[3], qs[3];
    for (int j = 0; j < 3; ++j) {
        q[j] = __dadd_rn(__dadd_rn(__dmul_rn(x, fd.frame[j]), __dmul_rn(y, fd.frame[3 + j])), __dmul_rn(z, fd.frame[6 + j]));
        qs[j] = fabs(x * fd.frame[j]) + fabs(y * fd.frame[3 + j]) + fabs(z * fd.frame[6 + j]);
    }
    const double ex = x - fd.sc_c[0], ey = y - fd.sc_c[1], ez = z - fd.sc_c[2];
    const double reach = 1.01 * (sqrt(ex * ex + ey * ey + ez * ez) + fd.sc_r) / sqrt(fd.gram[4 * k]) + 1e-6;
    for (int j = 0; j < 3; ++j) {
        double tol = 1e-9 * (double)rs + 1e-15 * (qs[j] + 4.0 * (double)rs + 1.0);
        if (j != k) tol += reach * (fabs(fd.gram[3 * j + k]) + 1e-15);
        double l = q[j] - tol, h = q[j] + tol;
        if (j == k) {
            if (pos) h = INFINITY;
            else l = -INFINITY;
        }
        ar.lo[j] = __double2float_rd(l);
        ar.hi[j] = __double2float_ru(h);
    }
    ar.k = k;
    ar.pos = pos ? 1 : 0;
    return ar;
}

template <bool kStats>
__device__ __forceinline__ TraceOut trace_axis(const float4* __restrict__ ftree, const float4* __restrict__ tris,
                                               const Ray& r, const AxisRay& ar, int max_steps)
{
    TraceOut out = {0, 0, 0, 0, 0};
    int stack[kStack4];
    int sp = 0;
    int cur = 0;
    bool amb = false, ambhit = false;
    // near face of a child along the ray: lo of axis k going +, hi going -
    const int near_off = 2 * ar.k + (ar.pos ? 0 : 1);
    for (int steps = 0;; ++steps) {
        if (steps > max_steps) { out.overflow = 1; out.flags = 1; return out; }
        if (cur >= 0) {
            if (kStats) ++out.nodes;
            const float4* nd = ftree + 8 * (int64_t)cur;
            const float4 lxv = __ldg(nd), hxv = __ldg(nd + 1), lyv = __ldg(nd + 2), hyv = __ldg(nd + 3);
            const float4 lzv = __ldg(nd + 4), hzv = __ldg(nd + 5), ci = __ldg(nd + 6), ev = __ldg(nd + near_off);
            const float LX[4] = {lxv.x, lxv.y, lxv.z, lxv.w}, HX[4] = {hxv.x, hxv.y, hxv.z, hxv.w};
            const float LY[4] = {lyv.x, lyv.y, lyv.z, lyv.w}, HY[4] = {hyv.x, hyv.y, hyv.z, hyv.w};
            const float LZ[4] = {lzv.x, lzv.y, lzv.z, lzv.w}, HZ[4] = {hzv.x, hzv.y, hzv.z, hzv.w};
            const float E[4] = {ev.x, ev.y, ev.z, ev.w};
            const int cc[4] = {__float_as_int(ci.x), __float_as_int(ci.y), __float_as_int(ci.z), __float_as_int(ci.w)};
            float d[4];
            int c[4];
            int nh = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool hit = LX[q] <= ar.hi[0] && HX[q] >= ar.lo[0] && LY[q] <= ar.hi[1] && HY[q] >= ar.lo[1] &&
                                 LZ[q] <= ar.hi[2] && HZ[q] >= ar.lo[2];
                d[q] = hit ? (ar.pos ? E[q] : -E[q]) : INFINITY;
                c[q] = cc[q];
                nh += hit;
            }
            if (nh == 0) {
                if (sp == 0) break;
                cur = stack[--sp];
                continue;
            }
#define RC_CSWAP(a, b)                                              \
    if (d[b] < d[a]) {                                              \
        const float td = d[a]; d[a] = d[b]; d[b] = td;              \
        const int tc = c[a]; c[a] = c[b]; c[b] = tc;                \
    }
            RC_CSWAP(0, 1) RC_CSWAP(2, 3) RC_CSWAP(0, 2)
#undef RC_CSWAP
            if (sp + nh - 1 > kStack4) { out.overflow = 1; out.flags = 1; return out; }
            if (d[3] != INFINITY) stack[sp++] = c[3];
            if (d[2] != INFINITY) stack[sp++] = c[2];
            if (d[1] != INFINITY) stack[sp++] = c[1];
            cur = c[0];
            continue;
        } else {
            const int v = -1 - cur;
            const int first = v >> 3, cnt = (v & 7) + 1;
            for (int k = 0; k < cnt; ++k) {
                const float4* t = tris + 3 * (first + k);
                const float4 v0 = __ldg(t), v1 = __ldg(t + 1), v2 = __ldg(t + 2);
                if (kStats) ++out.tris;
                const int st = tri_test32(r, v0, v1, v2);
                if (st == kHit) { out.flags = 1; return out; }
                if (st == kUnsure) {
                    ++out.retests;
                    const Pair64 p = retest64(r, v0, v1, v2);
                    if (p.state == kHit) { out.flags = 1; return out; }
                    if (p.state == kUnsure) { amb = true; ambhit |= p.hit64; }
                }
            }
        }
        if (sp == 0) break;
        cur = stack[--sp];
    }
    out.flags = (ambhit ? 1 : 0) | (amb ? 2 : 0);
    return out;
}

__device__ __forceinline__ void warp_add_counters(unsigned long long* counters, long long rays,
                                                  int amb, int retests, int overflow, long long nvis = 0,
                                                  long long ntri = 0)
{
    const unsigned full = 0xFFFFFFFFu;
    for (int off = 16; off; off >>= 1) {
        rays += __shfl_xor_sync(full, rays, off);
        amb += __shfl_xor_sync(full, amb, off);
        retests += __shfl_xor_sync(full, retests, off);
        overflow += __shfl_xor_sync(full, overflow, off);
        nvis += __shfl_xor_sync(full, nvis, off);
        ntri += __shfl_xor_sync(full, ntri, off);
    }
    if ((threadIdx.x & 31) == 0 && counters) {
        if (rays) atomicAdd(&counters[0], (unsigned long long)rays);
        if (amb) atomicAdd(&counters[1], (unsigned long long)amb);
        if (retests) atomicAdd(&counters[2], (unsigned long long)retests);
        if (overflow) atomicAdd(&counters[3], (unsigned long long)overflow);
        if (nvis) atomicAdd(&counters[4], (unsigned long long)nvis);
        if (ntri) atomicAdd(&counters[5], (unsigned long long)ntri);
    }
}

// ---------------------------------------------------------------------------
// Section 3.1: hemispherical cast.  One warp per point (dynamic work
// counter).  The warp casts the point's N directions in N/32 tiles of 32
// spatially close directions (the table is stored in tile order, each entry
// carrying its canonical index j), so that the lanes of a warp walk nearly
// the same part of the tree.  Each visible direction sets bit j & 31 of word
// j >> 5 in the warp's shared-memory row, which is written out in canonical
// order once the point is done; the count is the sum of the tile ballots.
// ---------------------------------------------------------------------------
#ifndef RC_HEMI_MIN_BLOCKS
#define RC_HEMI_MIN_BLOCKS 7
#endif
#ifndef RC_TAIL_SPLITS
#define RC_TAIL_SPLITS 4
#endif
#ifndef RC_TAIL_POINTS
#define RC_TAIL_POINTS 2        // points cast in parts, per resident warp
#endif

using CastAcc = CastAccFwd;

// The hemispherical cast of one point by one warp (see above).  `tdirs` is
// the tile-ordered table, `row` the warp's shared-memory row of W words.
// Tiles [t0, t1) are cast; a whole point (0, W) writes its bit row and count,
// a part of a point ORs its bits into the (zeroed) row in memory and adds
// its count.
template <bool kStats, bool kWide>
__device__ __forceinline__ void cast_point(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                           int max_steps, float scene_maxabs, const float* __restrict__ P,
                                           const float* __restrict__ Nrm, int64_t i,
                                           const float4* __restrict__ tdirs, int W, double eps, uint32_t* row,
                                           uint32_t* __restrict__ bits, int32_t* __restrict__ count, CastAcc& acc,
                                           int t0 = 0, int t1 = -1, long long* relist = nullptr,
                                           long long relist_cap = 0, unsigned long long* relist_ctr = nullptr,
                                           Frontier* front = nullptr)
{
    const int lane = threadIdx.x & 31;
    const bool whole = t1 < 0;
    if (whole) t1 = W;
    for (int w = lane; w < W; w += 32) row[w] = 0u;
    const float px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
    const float nx = Nrm[3 * i], ny = Nrm[3 * i + 1], nz = Nrm[3 * i + 2];
    const float ox = offset_coord(px, nx, eps), oy = offset_coord(py, ny, eps), oz = offset_coord(pz, nz, eps);
    if (kWide && front && lane == 0)
        build_frontier(nodes, tris, max_steps, ox, oy, oz, nx, ny, nz, tangent_shortcuts_ok(nx, ny, nz, W), front);
    __syncwarp();
    const Frontier* fr = kWide && front && front->ok ? front : nullptr;
    if (kStats && front && lane == 0) acc.nvis += front->nvis;
    const Onb b = make_onb(nx, ny, nz);
    int cnt = 0;
    for (int t = t0; t < t1; ++t) {
        // canonical index j; when 32 does not divide N the last tile is
        // padded with entries j = -1 that carry a real direction: they are
        // cast like the others (no branch in the loop) and then discarded
        const float4 h = __ldg(&tdirs[32 * t + lane]);
        const int j = __float_as_int(h.w);
        float dx, dy, dz;
        local_to_world(b, nx, ny, nz, h.x, h.y, h.z, dx, dy, dz);
        Ray r;
        setup_ray(r, ox, oy, oz, dx, dy, dz, scene_maxabs);
        const TraceOut tr = trace_any<kStats, kWide>(nodes, tris, r, max_steps, fr);
        acc.retests += tr.retests;
        acc.overflow += tr.overflow;
        acc.amb += (j >= 0) & ((tr.flags >> 1) & 1);
        if (kStats) {
            acc.nvis += tr.nodes;
            acc.ntri += tr.tris;
            // the instrumented cast can list the rays an FP64 re-test took part in
            if (relist && tr.retests > 0 && j >= 0) {
                const unsigned long long k = atomicAdd(relist_ctr, 1ULL);
                if (k < (unsigned long long)relist_cap) relist[k] = (long long)i * 65536 + j;
            }
        }
        const bool visible = (tr.flags & 1) == 0 && j >= 0;
        if (visible) atomicOr(&row[j >> 5], 1u << (j & 31));
        cnt += __popc(__ballot_sync(0xFFFFFFFFu, visible));
    }
    __syncwarp();
    if (whole) {
        for (int w = lane; w < W; w += 32) bits[i * W + w] = row[w];
        if (lane == 0) count[i] = cnt;
    } else {
        for (int w = lane; w < W; w += 32)
            if (row[w]) atomicOr(&bits[i * W + w], row[w]);
        if (lane == 0) atomicAdd(&count[i], cnt);
    }
    __syncwarp();
    // rays per lane: the tiles cast, less the pad of the last tile if this
    // lane has one
    acc.rays += (t1 - t0) - (t1 == W && __float_as_int(__ldg(&tdirs[32 * (W - 1) + lane]).w) < 0 ? 1 : 0);
}

// Dynamic shared memory of the point casts: each warp's bit row of W words,
// then (4-wide tree) each warp's frontier, 16-byte aligned.
__host__ __device__ __forceinline__ size_t rows_bytes(int warps, int W)
{
    return ((size_t)warps * W * sizeof(uint32_t) + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t cast_smem(int warps, int W, bool wide)
{
    return rows_bytes(warps, W) + (wide ? (size_t)warps * sizeof(Frontier) : 0);
}

template <bool kStats, bool kWide>
__global__ void __launch_bounds__(128, RC_HEMI_MIN_BLOCKS)
k_hemisphere(const float4* __restrict__ nodes, const float4* __restrict__ tris, int max_steps, float scene_maxabs,
             const float* __restrict__ P, const float* __restrict__ Nrm, int64_t n,
             const int32_t* __restrict__ order, const float4* __restrict__ tdirs, int n_dirs, double eps,
             uint32_t* __restrict__ bits, int32_t* __restrict__ count, unsigned long long* counters,
             unsigned long long* work, int64_t n_whole, int splits, long long* relist, long long relist_cap)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const int lane = threadIdx.x & 31;
    const int W = (n_dirs + 31) >> 5;
    uint32_t* row = (uint32_t*)s_dyn + (threadIdx.x >> 5) * W;
    Frontier* front = kWide ? (Frontier*)(s_dyn + rows_bytes(blockDim.x >> 5, W)) + (threadIdx.x >> 5) : nullptr;
    CastAcc acc;
    // With a work counter the warps take work until none is left: the first
    // n_whole points of the processing order whole, then the last n - n_whole
    // points in `splits` parts each, so that the launch ends on short items
    // instead of whole points.  Without a counter (grid sized to the work)
    // each warp casts exactly its own point, so blocks are short-lived and
    // kernels of concurrent requests interleave.
    const unsigned long long own = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned long long items = (unsigned long long)n_whole + (unsigned long long)(n - n_whole) * splits;
    const int tw = (W + splits - 1) / splits;
    for (bool first = true;; first = false) {
        unsigned long long k = items;
        if (work) {
            if (lane == 0) k = atomicAdd(work, 1ULL);
            k = __shfl_sync(0xFFFFFFFFu, k, 0);
        } else if (first) {
            k = own;
        }
        if (k >= items) break;
        // item k: a whole point (tiles 0..W, t1 = -1) or a part of one
        int64_t r = (int64_t)k;
        int t0 = 0, t1 = -1;
        if (k >= (unsigned long long)n_whole) {
            const unsigned long long q = k - (unsigned long long)n_whole;
            r = n_whole + (int64_t)(q / splits);
            t0 = (int)(q % splits) * tw;
            t1 = min(W, t0 + tw);
            if (t0 >= t1) continue;
        }
        const int64_t i = order ? (int64_t)__ldg(&order[r]) : r;
        cast_point<kStats, kWide>(nodes, tris, max_steps, scene_maxabs, P, Nrm, i, tdirs, W, eps, row, bits, count,
                                  acc, t0, t1, relist, relist_cap, counters ? counters + 6 : nullptr, front);
    }
    warp_add_counters(counters, acc.rays, acc.amb, acc.retests, acc.overflow, acc.nvis, acc.ntri);
}

// zero the bit rows and counts of the points cast in parts (positions
// [n_whole, n) of the processing order)
__global__ void k_zero_split(const int32_t* __restrict__ order, int64_t n_whole, int64_t n, int W,
                             uint32_t* __restrict__ bits, int32_t* __restrict__ count)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = n_whole + t / W;
    if (r >= n) return;
    const int64_t i = order ? (int64_t)order[r] : r;
    const int w = (int)(t % W);
    bits[i * W + w] = 0u;
    if (w == 0) count[i] = 0;
}

// ---------------------------------------------------------------------------
// Re-analysis after an edit that keeps the triangle list (reading: every
// sample point stays on its face).  The result of a ray depends only on the
// triangles it can meet; the edited triangles lie in the box [blo, bhi] in
// both the old and the new part, so a ray from an unmoved point that cannot
// enter that box (the conservative slab test of the traversal, monotone in
// the box) keeps its old bit.  Points on moved faces are cast in full; an
// unmoved point whose tangent plane has the whole box behind it (every
// hemisphere direction has d.n > 0 when its normal is of unit length, see
// tangent_shortcuts_ok) is skipped outright.  Rays whose old
// and new decisions are both made only by FP64-ambiguous pairs may differ
// from a full re-cast; they are counted as ambiguous like any other.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ray_enters_box(const Ray& r, const float4 lo, const float4 hi)
{
    const float rob = 1.0f + 2.0f * 1.7881394e-7f;
    const bool sx = signbit(r.ix), sy = signbit(r.iy), sz = signbit(r.iz);
    const float nx = ((sx ? hi.x : lo.x) - r.ox) * r.ix, fx = ((sx ? lo.x : hi.x) - r.ox) * r.ix;
    const float ny = ((sy ? hi.y : lo.y) - r.oy) * r.iy, fy = ((sy ? lo.y : hi.y) - r.oy) * r.iy;
    const float nz = ((sz ? hi.z : lo.z) - r.oz) * r.iz, fz = ((sz ? lo.z : hi.z) - r.oz) * r.iz;
    const float tn = fmaxf(fmaxf(nx, ny), fmaxf(nz, 0.0f));
    const float tf = fminf(fminf(fx, fy), fz) * rob;
    return tn <= tf;
}

// max over the box corners of (c - o).n in FP64, with its rounding bound
__device__ __forceinline__ bool box_in_front(const float4 lo, const float4 hi, float ox, float oy, float oz, float nx,
                                             float ny, float nz)
{
    double best = -INFINITY, mag = 0.0;
    for (int c = 0; c < 8; ++c) {
        const double x = __dsub_rn((double)((c & 1) ? hi.x : lo.x), (double)ox);
        const double y = __dsub_rn((double)((c & 2) ? hi.y : lo.y), (double)oy);
        const double z = __dsub_rn((double)((c & 4) ? hi.z : lo.z), (double)oz);
        const double a = __dmul_rn(x, (double)nx), b = __dmul_rn(y, (double)ny), e = __dmul_rn(z, (double)nz);
        best = fmax(best, __dadd_rn(__dadd_rn(a, b), e));
        mag = fmax(mag, __dadd_rn(__dadd_rn(fabs(a), fabs(b)), fabs(e)));
    }
    return best > -1e-12 * mag;
}

template <bool kWide>
__global__ void __launch_bounds__(128, RC_HEMI_MIN_BLOCKS)
k_hemisphere_update(const float4* __restrict__ nodes, const float4* __restrict__ tris, int max_steps,
                    float scene_maxabs, const float* __restrict__ P, const float* __restrict__ Nrm, int64_t n,
                    const int32_t* __restrict__ order, const int32_t* __restrict__ face,
                    const uint8_t* __restrict__ changed, float4 blo, float4 bhi, const float4* __restrict__ tdirs,
                    int n_dirs, double eps, uint32_t* __restrict__ bits, int32_t* __restrict__ count,
                    unsigned long long* counters, unsigned long long* work)
{
    extern __shared__ uint32_t s_rows[];
    const int lane = threadIdx.x & 31;
    const int W = (n_dirs + 31) >> 5;
    uint32_t* row = s_rows + (threadIdx.x >> 5) * W;
    CastAcc acc;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(work, 1ULL);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= (unsigned long long)n) break;
        const int64_t i = order ? (int64_t)__ldg(&order[k]) : (int64_t)k;
        const bool moved = changed[face[i]] != 0;
        const float px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
        const float nx = Nrm[3 * i], ny = Nrm[3 * i + 1], nz = Nrm[3 * i + 2];
        const float ox = offset_coord(px, nx, eps), oy = offset_coord(py, ny, eps), oz = offset_coord(pz, nz, eps);
        if (!moved && tangent_shortcuts_ok(nx, ny, nz, W) && !box_in_front(blo, bhi, ox, oy, oz, nx, ny, nz))
            continue;   // nothing can change
        for (int w = lane; w < W; w += 32) row[w] = moved ? 0u : bits[i * W + w];
        __syncwarp();
        const Onb b = make_onb(nx, ny, nz);
        for (int t = 0; t < W; ++t) {
            const float4 h = __ldg(&tdirs[32 * t + lane]);
            const int j = __float_as_int(h.w);
            if (j < 0) continue;
            float dx, dy, dz;
            local_to_world(b, nx, ny, nz, h.x, h.y, h.z, dx, dy, dz);
            Ray r;
            setup_ray(r, ox, oy, oz, dx, dy, dz, scene_maxabs);
            if (!moved && !ray_enters_box(r, blo, bhi)) continue;              // keeps its old bit
            const TraceOut tr = trace_any<false, kWide>(nodes, tris, r, max_steps);
            acc.retests += tr.retests;
            acc.overflow += tr.overflow;
            acc.amb += (tr.flags >> 1) & 1;
            acc.rays += 1;
            if ((tr.flags & 1) == 0) atomicOr(&row[j >> 5], 1u << (j & 31));
            else atomicAnd(&row[j >> 5], ~(1u << (j & 31)));
        }
        __syncwarp();
        int cnt = 0;
        for (int w = lane; w < W; w += 32) {
            bits[i * W + w] = row[w];
            cnt += __popc(row[w]);
        }
        for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
        if (lane == 0) count[i] = cnt;
        __syncwarp();
    }
    warp_add_counters(counters, acc.rays, acc.amb, acc.retests, acc.overflow);
}

// ---------------------------------------------------------------------------
// Batched hemispherical cast: one persistent launch over the points of many
// parts.  Work items are runs of `ppi` consecutive points (in each part's
// processing order) of one part; a warp takes items from one global counter,
// finds the part by binary search over the parts' first item, and casts the
// points as k_hemisphere does.  Counters are kept per part.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void flush_part_counters(unsigned long long* c, CastAcc& a)
{
    warp_add_counters(c, a.rays, a.amb, a.retests, a.overflow);
    a = CastAcc();
}

#ifndef RC_BATCH_MIN_BLOCKS
#define RC_BATCH_MIN_BLOCKS 6
#endif

template <bool kStats, bool kWide>
__global__ void __launch_bounds__(128, RC_BATCH_MIN_BLOCKS)
k_batch(const BatchPart* __restrict__ parts, int n_parts, long long n_items, int ppi,
        const float4* __restrict__ tdirs, int n_dirs, double eps, unsigned long long* work)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const int lane = threadIdx.x & 31;
    const int W = (n_dirs + 31) >> 5;
    uint32_t* row = (uint32_t*)s_dyn + (threadIdx.x >> 5) * W;
    Frontier* front = kWide ? (Frontier*)(s_dyn + rows_bytes(blockDim.x >> 5, W)) + (threadIdx.x >> 5) : nullptr;
    CastAcc acc;
    int cur = -1;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(work, 1ULL);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= (unsigned long long)n_items) break;
        int lo = 0, hi = n_parts - 1;            // last part with first_item <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)parts[mid].first_item <= k) lo = mid; else hi = mid - 1;
        }
        const BatchPart& bp = parts[lo];
        if (lo != cur) {
            if (cur >= 0) flush_part_counters(parts[cur].counters, acc);
            cur = lo;
        }
        const long long q0 = ((long long)k - bp.first_item) * ppi;
        const long long q1 = q0 + ppi < bp.n ? q0 + ppi : bp.n;
        for (long long q = q0; q < q1; ++q) {
            const int64_t i = bp.order ? (int64_t)__ldg(&bp.order[q]) : (int64_t)q;
            cast_point<kStats, kWide>(bp.nodes, bp.tris, bp.max_steps, bp.scene_maxabs, bp.P, bp.N, i, tdirs, W,
                                      eps, row, bp.bits, bp.count, acc, 0, -1, nullptr, 0, nullptr, front);
        }
    }
    if (cur >= 0) flush_part_counters(parts[cur].counters, acc);
}

// ---------------------------------------------------------------------------
// Section 3.2: orthogonal cast along the six frame axes (+X', -X', +Y', -Y',
// +Z', -Z').  A work item (frame f, axis a, group g) is 32 consecutive points
// of the Morton processing order cast along one axis, one ray per lane --
// parallel rays from neighbouring origins.  Warps take items one at a time
// from a counter, because a few rays that graze a surface parallel to an axis
// (along a fillet or a bore) take far longer than the rest.  Travel to the
// frame bounding box is FP64.  Frame f writes travel[f n + i][6]; reachable
// bits gather in mbits[f n + i] (zeroed by the caller) and are packed into
// mask[f n + i] afterwards.
// ---------------------------------------------------------------------------
template <bool kStats, bool kWide>
__global__ void __launch_bounds__(128, RC_BATCH_MIN_BLOCKS)
k_orthogonal_axis(const float4* __restrict__ nodes, const float4* __restrict__ tris, int max_steps,
                  float scene_maxabs, const float* __restrict__ P, const float* __restrict__ Nrm, int64_t n,
                  const int32_t* __restrict__ order, const FrameDev* __restrict__ fds, int nf, double eps,
                  double par_tol, uint32_t* __restrict__ mbits, float* __restrict__ travel,
                  unsigned long long* counters, unsigned long long* work)
{
    const int lane = threadIdx.x & 31;
    int amb = 0, retests = 0, overflow = 0;
    long long rays = 0, nvis = 0, ntri = 0;
    const int64_t G = (n + 31) >> 5;
    const int64_t items = (int64_t)nf * 6 * G;
    // without a work counter (grid sized to the work) each warp casts only
    // its own item, so blocks stay short and concurrent requests interleave
    const unsigned long long own = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (bool first = true;; first = false) {
        unsigned long long w = (unsigned long long)items;
        if (work) {
            if (lane == 0) w = atomicAdd(work, 1ULL);
            w = __shfl_sync(0xFFFFFFFFu, w, 0);
        } else if (first) {
            w = own;
        }
        const int64_t it = (int64_t)w;
        if (it >= items) break;
        const int fa = (int)(it / G);
        const int64_t g = it - (int64_t)fa * G;
        const int f = fa / 6, a = fa - 6 * f;
        const int64_t k = g * 32 + lane;
        if (k >= n) continue;
        const int64_t i = order ? (int64_t)__ldg(&order[k]) : k;
        const float px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
        const float nx = Nrm[3 * i], ny = Nrm[3 * i + 1], nz = Nrm[3 * i + 2];
        const float* axes = fds[f].axes;
        const double* frame = fds[f].frame;
        const double* fbox = fds[f].fbox;
        const int64_t row = (int64_t)f * n + i;
        const float dx = axes[3 * a], dy = axes[3 * a + 1], dz = axes[3 * a + 2];
        const int kk = a >> 1;
        double q = __dadd_rn(__dmul_rn((double)px, frame[kk]), __dmul_rn((double)py, frame[3 + kk]));
        q = __dadd_rn(q, __dmul_rn((double)pz, frame[6 + kk]));
        const double tv = (a & 1) ? __dsub_rn(q, fbox[kk]) : __dsub_rn(fbox[3 + kk], q);
        travel[6 * row + a] = __double2float_rn(tv);
        // eligibility n.a >= -parallel_tol (FP64, x, y, z order)
        double nd = __dadd_rn(__dmul_rn((double)nx, (double)dx), __dmul_rn((double)ny, (double)dy));
        nd = __dadd_rn(nd, __dmul_rn((double)nz, (double)dz));
        if (nd >= -par_tol) {
            Ray r;
            const float ox = offset_coord(px, nx, eps), oy = offset_coord(py, ny, eps), oz = offset_coord(pz, nz, eps);
            setup_ray(r, ox, oy, oz, dx, dy, dz, scene_maxabs);
            TraceOut t;
            if (kWide) {
                const AxisRay ar = make_axis_ray(fds[f], a, ox, oy, oz, r.rs);
                t = trace_axis<kStats>(fds[f].tree, tris, r, ar, max_steps);
            } else {
                t = trace_any<kStats, kWide>(nodes, tris, r, max_steps);
            }
            retests += t.retests;
            overflow += t.overflow;
            amb += (t.flags >> 1) & 1;
            if ((t.flags & 1) == 0) atomicOr(&mbits[row], 1u << a);
            rays += 1;
            if (kStats) { nvis += t.nodes; ntri += t.tris; }
        }
    }
    warp_add_counters(counters, rays, amb, retests, overflow, nvis, ntri);
}

__global__ void k_mask_pack(const uint32_t* __restrict__ mbits, int64_t m, uint8_t* __restrict__ mask)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < m) mask[r] = (uint8_t)mbits[r];
}

// ---------------------------------------------------------------------------
// Tool-aware accessibility (a reading of the accessibility cones of the prior
// art the paper cites; the paper itself casts thin rays).  A ball-end tool of
// radius r touches the point: centre c = p + (r + eps) n (FP64).  Along axis
// a its shank is sampled by the ray from c and K rays from the ring
// c + r (cos t_k u + sin t_k v), (u, v) the branchless orthonormal basis of
// a (Duff et al. 2017) in FP64; origins are rounded to fp32, every ray goes
// along a.  The axis is tool-accessible iff it is eligible (n.a >=
// -parallel_tol) and none of the 1 + K rays is obstructed.  Work items are
// (axis, 32 consecutive points) as in the orthogonal cast; accessible bits
// gather in mbits[i] (zeroed by the caller).
// ---------------------------------------------------------------------------
template <bool kWide>
__global__ void __launch_bounds__(128, RC_BATCH_MIN_BLOCKS)
k_tool_cast_axis(const float4* __restrict__ nodes, const float4* __restrict__ tris, int max_steps,
                 float scene_maxabs, const float* __restrict__ P, const float* __restrict__ Nrm, int64_t n,
                 const int32_t* __restrict__ order, const FrameDev* __restrict__ fd, double eps, double par_tol,
                 double radius, const double2* __restrict__ ring /*cos, sin*/, int K, uint32_t* __restrict__ mbits,
                 unsigned long long* counters, unsigned long long* work)
{
    const int lane = threadIdx.x & 31;
    int amb = 0, retests = 0, overflow = 0;
    long long rays = 0;
    const int64_t G = (n + 31) >> 5;
    const int64_t items = 6 * G;
    for (;;) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(work, 1ULL);
        const int64_t it = (int64_t)__shfl_sync(0xFFFFFFFFu, w, 0);
        if (it >= items) break;
        const int a = (int)(it / G);
        const int64_t k = (it - (int64_t)a * G) * 32 + lane;
        if (k >= n) continue;
        const int64_t i = order ? (int64_t)__ldg(&order[k]) : k;
        const double px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
        const double nx = Nrm[3 * i], ny = Nrm[3 * i + 1], nz = Nrm[3 * i + 2];
        const float dx = fd->axes[3 * a], dy = fd->axes[3 * a + 1], dz = fd->axes[3 * a + 2];
        double nd = __dadd_rn(__dmul_rn(nx, (double)dx), __dmul_rn(ny, (double)dy));
        nd = __dadd_rn(nd, __dmul_rn(nz, (double)dz));
        if (!(nd >= -par_tol)) continue;
        const double h = __dadd_rn(radius, eps);
        const double cx = __dadd_rn(px, __dmul_rn(h, nx)), cy = __dadd_rn(py, __dmul_rn(h, ny)),
                     cz = __dadd_rn(pz, __dmul_rn(h, nz));
        // orthonormal basis (u, v) of the axis, FP64
        const double ax = dx, ay = dy, az = dz;
        const double sg = az >= 0.0 ? 1.0 : -1.0;
        const double q = __ddiv_rn(-1.0, __dadd_rn(sg, az));
        const double bb = __dmul_rn(__dmul_rn(ax, ay), q);
        const double ux = __dadd_rn(1.0, __dmul_rn(__dmul_rn(__dmul_rn(sg, ax), ax), q));
        const double uy = __dmul_rn(sg, bb), uz = __dmul_rn(-sg, ax);
        const double vx = bb, vy = __dadd_rn(sg, __dmul_rn(__dmul_rn(ay, ay), q)), vz = -ay;
        bool open = true;
        for (int r = -1; r < K && open; ++r) {
            float ox, oy, oz;
            if (r < 0) {
                ox = __double2float_rn(cx);
                oy = __double2float_rn(cy);
                oz = __double2float_rn(cz);
            } else {
                const double rc = __dmul_rn(radius, ring[r].x), rs = __dmul_rn(radius, ring[r].y);
                ox = __double2float_rn(__dadd_rn(__dadd_rn(cx, __dmul_rn(rc, ux)), __dmul_rn(rs, vx)));
                oy = __double2float_rn(__dadd_rn(__dadd_rn(cy, __dmul_rn(rc, uy)), __dmul_rn(rs, vy)));
                oz = __double2float_rn(__dadd_rn(__dadd_rn(cz, __dmul_rn(rc, uz)), __dmul_rn(rs, vz)));
            }
            Ray ray;
            setup_ray(ray, ox, oy, oz, dx, dy, dz, scene_maxabs);
            TraceOut t;
            if (kWide) {
                const AxisRay ar = make_axis_ray(*fd, a, ox, oy, oz, ray.rs);
                t = trace_axis<false>(fd->tree, tris, ray, ar, max_steps);
            } else {
                t = trace_any<false, kWide>(nodes, tris, ray, max_steps);
            }
            retests += t.retests;
            overflow += t.overflow;
            amb += (t.flags >> 1) & 1;
            rays += 1;
            open = (t.flags & 1) == 0;
        }
        if (open) atomicOr(&mbits[i], 1u << a);
    }
    warp_add_counters(counters, rays, amb, retests, overflow);
}

// FP64 bounding box of the vertices in frame coordinates: per-thread
// min/max over a grid-stride range, warp reduction, one atomic per warp.
__global__ void k_frame_box(const float* __restrict__ V, int64_t nV, const double* __restrict__ frame,
                            long long* box /*lo3 hi3 ordered*/)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nV; v += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            double q = __dadd_rn(__dmul_rn((double)V[3 * v], frame[k]), __dmul_rn((double)V[3 * v + 1], frame[3 + k]));
            q = __dadd_rn(q, __dmul_rn((double)V[3 * v + 2], frame[6 + k]));
            lo[k] = fmin(lo[k], q);
            hi[k] = fmax(hi[k], q);
        }
    }
    for (int off = 16; off; off >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], off));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], off));
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            if (lo[k] <= hi[k]) {
                atomicMin(&box[k], double_to_ordered(lo[k]));
                atomicMax(&box[3 + k], double_to_ordered(hi[k]));
            }
        }
}

__global__ void k_frame_box_finish(long long* box, double* fbox)
{
    if (threadIdx.x < 6) fbox[threadIdx.x] = ordered_to_double(box[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
static int max_steps(rc_bvh h) { return (int)(2 * (h->n_int + h->T) + 64); }

// the 4-wide tree is the default; tree_width 2 selects the binary tree
bool use_wide(const rc_params* p) { return p->tree_width != 2; }

static int g_sm_count = 0;

static int sm_count()
{
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

rc_status point_order(rc_bvh h, const float* P, int64_t n, int32_t* order, cudaStream_t s);

// device scratch of a launch, freed in stream order when the scope ends
struct LaunchScratch {
    cudaStream_t s;
    void* p[3] = {nullptr, nullptr, nullptr};
    ~LaunchScratch()
    {
        for (void* q : p)
            if (q) cudaFreeAsync(q, s);
    }
};

rc_status launch_hemisphere(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                            uint32_t* bits, int32_t* count, unsigned long long* counters, bool stats,
                            cudaStream_t s, long long* relist, long long relist_cap)
{
    LaunchScratch ls{s};
    unsigned long long* work = nullptr;
    if (p->launch_mode == 0) {
        RC_CUDA(cudaMallocAsync(&work, sizeof(unsigned long long), s));
        ls.p[0] = work;
        RC_CUDA(cudaMemsetAsync(work, 0, sizeof(unsigned long long), s));
    }
    int32_t* order = nullptr;
    if (p->point_order == 0 && n > 1) {
        RC_CUDA(cudaMallocAsync(&order, sizeof(int32_t) * n, s));
        ls.p[1] = order;
        rc_status st = point_order(h, P, n, order, s);
        if (st != RC_OK) return st;
    }
    const int threads = 128;
    const int per_sm = p->blocks_per_sm > 0 ? p->blocks_per_sm : RC_HEMI_MIN_BLOCKS;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (n * 32 + threads - 1) / threads;
    if (blocks > need || p->launch_mode == 1) blocks = need;
    if (blocks < 1) blocks = 1;
    if (blocks > 0x7FFFFFFF) return set_error(RC_E_UNSUPPORTED, "too many points for one launch");
    if (p->launch_mode == 1) work = nullptr;
    const bool wide = use_wide(p);
    const size_t smem = cast_smem(threads / 32, (p->n_dirs + 31) / 32, wide);
    if (smem > 48 * 1024) {
        RC_CUDA(cudaFuncSetAttribute(k_hemisphere<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RC_CUDA(cudaFuncSetAttribute(k_hemisphere<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RC_CUDA(cudaFuncSetAttribute(k_hemisphere<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RC_CUDA(cudaFuncSetAttribute(k_hemisphere<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const float4* tree = wide ? h->wnodes : h->nodes;
    {
        // the last points (RC_TAIL_POINTS per resident warp) are cast in parts;
        // with a grid sized to the work (one item per warp) the parts are the
        // highest blocks, which the block scheduler starts last
        const int W = (p->n_dirs + 31) / 32;
        const int64_t resident_warps = (int64_t)sm_count() * per_sm * (threads / 32);
        int splits = std::min(RC_TAIL_SPLITS, W);
        int64_t n_split = splits > 1 ? std::min<int64_t>(n, RC_TAIL_POINTS * resident_warps) : 0;
        if (n_split == 0) splits = 1;
        if (!work) {
            const int64_t items = (n - n_split) + n_split * splits;
            blocks = std::max<int64_t>(1, (items * 32 + threads - 1) / threads);
            if (blocks > 0x7FFFFFFF) return set_error(RC_E_UNSUPPORTED, "too many points for one launch");
        }
        if (n_split > 0) {
            k_zero_split<<<(unsigned)((n_split * W + 255) / 256), 256, 0, s>>>(order, n - n_split, n, W, bits, count);
            RC_LAUNCHED();
        }
#define RC_HEMI(ST, WD)                                                                                    \
    k_hemisphere<ST, WD><<<(unsigned)blocks, threads, smem, s>>>(tree, h->tris, max_steps(h), h->scene_maxabs, \
                                                                 P, N, n, order, h->tdirs, p->n_dirs,         \
                                                                 p->origin_offset, bits, count, counters, work, \
                                                                 n - n_split, splits, relist, relist_cap)
        if (stats && wide) RC_HEMI(true, true);
        else if (stats) RC_HEMI(true, false);
        else if (wide) RC_HEMI(false, true);
        else RC_HEMI(false, false);
#undef RC_HEMI
    }
    RC_LAUNCHED();
    return RC_OK;
}

// Re-analysis of the points after an edit (see k_hemisphere_update); bits
// and count hold the old results on entry.
rc_status launch_hemisphere_update(rc_bvh h, const float* P, const float* N, int64_t n, const int32_t* face,
                                   const uint8_t* changed, const float box[6], const float4* tdirs,
                                   const rc_params* p, uint32_t* bits, int32_t* count, unsigned long long* counters,
                                   cudaStream_t s)
{
    LaunchScratch ls{s};
    unsigned long long* work = nullptr;
    RC_CUDA(cudaMallocAsync(&work, sizeof(unsigned long long), s));
    ls.p[0] = work;
    RC_CUDA(cudaMemsetAsync(work, 0, sizeof(unsigned long long), s));
    int32_t* order = nullptr;
    if (p->point_order == 0 && n > 1) {
        RC_CUDA(cudaMallocAsync(&order, sizeof(int32_t) * n, s));
        ls.p[1] = order;
        rc_status st = point_order(h, P, n, order, s);
        if (st != RC_OK) return st;
    }
    const int threads = 128;
    const int per_sm = p->blocks_per_sm > 0 ? p->blocks_per_sm : RC_HEMI_MIN_BLOCKS;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (n * 32 + threads - 1) / threads;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    const size_t smem = (size_t)(threads / 32) * ((p->n_dirs + 31) / 32) * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        RC_CUDA(cudaFuncSetAttribute(k_hemisphere_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RC_CUDA(cudaFuncSetAttribute(k_hemisphere_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const float4 lo = make_float4(box[0], box[1], box[2], 0.0f), hi = make_float4(box[3], box[4], box[5], 0.0f);
    if (use_wide(p))
        k_hemisphere_update<true><<<(unsigned)blocks, threads, smem, s>>>(h->wnodes, h->tris, max_steps(h),
                                                                         h->scene_maxabs, P, N, n, order, face,
                                                                         changed, lo, hi, tdirs, p->n_dirs,
                                                                         p->origin_offset, bits, count, counters,
                                                                         work);
    else
        k_hemisphere_update<false><<<(unsigned)blocks, threads, smem, s>>>(h->nodes, h->tris, max_steps(h),
                                                                          h->scene_maxabs, P, N, n, order, face,
                                                                          changed, lo, hi, tdirs, p->n_dirs,
                                                                          p->origin_offset, bits, count, counters,
                                                                          work);
    RC_LAUNCHED();
    return RC_OK;
}

__global__ void k_frame_init(FrameArgs a, FrameDev* d)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int k = 0; k < 9; ++k) d->frame[k] = (double)a.f[k];
    d->tree = a.tree;
    for (int j = 0; j < 3; ++j) {
        d->sc_c[j] = a.sc_c[j];
        for (int k = 0; k < 3; ++k)
            d->gram[3 * j + k] = __dadd_rn(__dadd_rn(__dmul_rn((double)a.f[j], (double)a.f[k]),
                                                     __dmul_rn((double)a.f[3 + j], (double)a.f[3 + k])),
                                           __dmul_rn((double)a.f[6 + j], (double)a.f[6 + k]));
    }
    d->sc_r = a.sc_r;
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) {
            d->axes[3 * (2 * k) + c] = a.f[3 * c + k];
            d->axes[3 * (2 * k + 1) + c] = -a.f[3 * c + k];
        }
    for (int k = 0; k < 3; ++k) {
        d->box[k] = 0x7FFFFFFFFFFFFFFFLL;
        d->box[3 + k] = (long long)0x8000000000000000ULL;
    }
}

// Frame axes, frame matrix (FP64) and the vertices' frame bounding box, all
// on the device; the frame travels as a kernel argument (no host copy).
rc_status frame_setup_f(rc_bvh h, const float* f9, FrameDev* d, cudaStream_t s, const float4* tree)
{
    FrameArgs a;
    for (int k = 0; k < 9; ++k) a.f[k] = f9[k];
    a.tree = tree ? tree : h->wnodes;
    double r2 = 0.0;
    for (int j = 0; j < 3; ++j) {
        a.sc_c[j] = 0.5 * ((double)h->lo[j] + (double)h->hi[j]);
        r2 += ((double)h->hi[j] - (double)h->lo[j]) * ((double)h->hi[j] - (double)h->lo[j]);
    }
    a.sc_r = 0.5 * sqrt(r2);
    k_frame_init<<<1, 32, 0, s>>>(a, d);
    RC_LAUNCHED();
    const int64_t fb = std::min<int64_t>((h->nV + 255) / 256, (int64_t)sm_count() * 4);
    k_frame_box<<<(unsigned)std::max<int64_t>(fb, 1), 256, 0, s>>>(h->V, h->nV, d->frame, d->box);
    RC_LAUNCHED();
    k_frame_box_finish<<<1, 32, 0, s>>>(d->box, d->fbox);
    RC_LAUNCHED();
    return RC_OK;
}

rc_status frame_setup(rc_bvh h, const rc_params* p, FrameDev* d, cudaStream_t s, const float4* tree)
{
    return frame_setup_f(h, p->frame, d, s, tree);
}

bool is_identity_frame(const float f9[9])
{
    for (int k = 0; k < 9; ++k)
        if (f9[k] != ((k % 4) == 0 ? 1.0f : 0.0f)) return false;
    return true;
}

rc_status make_frame_tree(rc_bvh h, const float f9[9], const rc_params* p, float4** ftree, cudaStream_t s)
{
    *ftree = nullptr;
    if (!use_wide(p) || is_identity_frame(f9)) return RC_OK;
    const int64_t nodes = h->host_sc.wide_nodes > 0 ? h->host_sc.wide_nodes : h->n_int;
    RC_CUDA(cudaMallocAsync(ftree, sizeof(float4) * 8 * nodes, s));
    const rc_status st = frame_tree(h, f9, *ftree, s);
    if (st != RC_OK) {
        cudaFreeAsync(*ftree, s);
        *ftree = nullptr;
    }
    return st;
}

// Orthogonal cast of n points in nf frames (fds: device array of nf set-up
// frames); mask [nf][n], travel [nf][n][6].
// Orthogonal cast into caller-provided scratch: order (n points in their
// processing order, or null for index order; filled by the caller) and
// mbits (ortho_scratch_words(nf, n) words, cleared here).  Allocates nothing,
// so it can be captured in a graph.
int64_t ortho_scratch_words(int nf, int64_t n) { return ((((int64_t)nf * n) + 1) & ~(int64_t)1) + 2; }

rc_status launch_orthogonal_frames_into(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                                        const FrameDev* fds, int nf, uint8_t* mask, float* travel,
                                        unsigned long long* counters, const int32_t* order, uint32_t* mbits,
                                        cudaStream_t s)
{
    if (n == 0) return RC_OK;
    const int64_t m = (int64_t)nf * n;
    const int64_t mw = (m + 1) & ~(int64_t)1;   // m words, then the item counter
    RC_CUDA(cudaMemsetAsync(mbits, 0, sizeof(uint32_t) * (mw + 2), s));
    unsigned long long* work = (unsigned long long*)(mbits + mw);
    const int64_t items = (int64_t)nf * 6 * ((n + 31) / 32);
    const int64_t cap = (int64_t)sm_count() * RC_BATCH_MIN_BLOCKS;
    int64_t blocks = (items + 3) / 4;
    if (blocks > cap && p->launch_mode == 0) blocks = cap;
    if (p->launch_mode == 1) work = nullptr;
    const float4* tree = use_wide(p) ? h->wnodes : h->nodes;
#define RC_ORTHO(ST, WD)                                                                                      \
    k_orthogonal_axis<ST, WD><<<(unsigned)blocks, 128, 0, s>>>(tree, h->tris, max_steps(h), h->scene_maxabs, \
                                                               P, N, n, order, fds, nf, p->origin_offset,    \
                                                               p->parallel_tol, mbits, travel, counters, work)
    const bool stats = p->collect_stats != 0;
    if (stats && use_wide(p)) RC_ORTHO(true, true);
    else if (stats) RC_ORTHO(true, false);
    else if (use_wide(p)) RC_ORTHO(false, true);
    else RC_ORTHO(false, false);
#undef RC_ORTHO
    RC_LAUNCHED();
    k_mask_pack<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(mbits, m, mask);
    RC_LAUNCHED();
    return RC_OK;
}

rc_status launch_orthogonal_frames(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                                   const FrameDev* fds, int nf, uint8_t* mask, float* travel,
                                   unsigned long long* counters, cudaStream_t s)
{
    if (n == 0) return RC_OK;
    LaunchScratch ls{s};
    int32_t* order = nullptr;
    if (p->point_order == 0 && n > 1) {
        RC_CUDA(cudaMallocAsync(&order, sizeof(int32_t) * n, s));
        ls.p[0] = order;
        rc_status pst = point_order(h, P, n, order, s);
        if (pst != RC_OK) return pst;
    }
    uint32_t* mbits = nullptr;
    RC_CUDA(cudaMallocAsync(&mbits, sizeof(uint32_t) * ortho_scratch_words(nf, n), s));
    ls.p[1] = mbits;
    return launch_orthogonal_frames_into(h, P, N, n, p, fds, nf, mask, travel, counters, order, mbits, s);
}

rc_status launch_orthogonal(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p,
                            uint8_t* mask, float* travel, unsigned long long* counters, cudaStream_t s)
{
    FrameDev* fd = nullptr;
    float4* ftree = nullptr;
    RC_CUDA(cudaMallocAsync(&fd, sizeof(FrameDev), s));
    rc_status st = n > 0 ? make_frame_tree(h, p->frame, p, &ftree, s) : RC_OK;
    if (st == RC_OK) st = frame_setup(h, p, fd, s, ftree);
    if (st == RC_OK) st = launch_orthogonal_frames(h, P, N, n, p, fd, 1, mask, travel, counters, s);
    if (ftree) cudaFreeAsync(ftree, s);
    cudaFreeAsync(fd, s);
    return st;
}

// RC_LAUNCHED without the early return
static rc_status launch_status()
{
    count_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : cuda_error(e, "kernel launch");
}

rc_status launch_tool_cast(rc_bvh h, const float* P, const float* N, int64_t n, const rc_params* p, double radius,
                          const double2* ring, int K, uint8_t* mask, unsigned long long* counters, cudaStream_t s)
{
    if (n == 0) return RC_OK;
    FrameDev* fd = nullptr;
    int32_t* order = nullptr;
    uint32_t* mbits = nullptr;                     // n words, then the item counter
    const int64_t mw = (n + 1) & ~(int64_t)1;
    cudaError_t e = cudaMallocAsync(&fd, sizeof(FrameDev), s);
    if (e == cudaSuccess && p->point_order == 0 && n > 1) e = cudaMallocAsync(&order, sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&mbits, sizeof(uint32_t) * (mw + 2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mbits, 0, sizeof(uint32_t) * (mw + 2), s);
    rc_status st = e == cudaSuccess ? RC_OK : cuda_error(e, "tool cast scratch");
    float4* ftree = nullptr;
    if (st == RC_OK) st = make_frame_tree(h, p->frame, p, &ftree, s);
    if (st == RC_OK) st = frame_setup(h, p, fd, s, ftree);
    if (st == RC_OK && order) st = point_order(h, P, n, order, s);
    if (st == RC_OK) {
        int64_t blocks = (6 * ((n + 31) / 32) + 3) / 4;
        const int64_t cap = (int64_t)sm_count() * RC_BATCH_MIN_BLOCKS;
        if (blocks > cap) blocks = cap;
        unsigned long long* work = (unsigned long long*)(mbits + mw);
        if (use_wide(p))
            k_tool_cast_axis<true><<<(unsigned)blocks, 128, 0, s>>>(h->wnodes, h->tris, max_steps(h), h->scene_maxabs,
                                                                   P, N, n, order, fd, p->origin_offset,
                                                                   p->parallel_tol, radius, ring, K, mbits, counters,
                                                                   work);
        else
            k_tool_cast_axis<false><<<(unsigned)blocks, 128, 0, s>>>(h->nodes, h->tris, max_steps(h), h->scene_maxabs,
                                                                    P, N, n, order, fd, p->origin_offset,
                                                                    p->parallel_tol, radius, ring, K, mbits, counters,
                                                                    work);
        st = launch_status();
    }
    if (st == RC_OK) {
        k_mask_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mbits, n, mask);
        st = launch_status();
    }
    if (mbits) cudaFreeAsync(mbits, s);
    if (order) cudaFreeAsync(order, s);
    if (ftree) cudaFreeAsync(ftree, s);
    if (fd) cudaFreeAsync(fd, s);
    return st;
}

rc_status launch_batch(const BatchPart* d_parts, int n_parts, long long n_items, int ppi, const float4* tdirs,
                       const rc_params* p, unsigned long long* work, cudaStream_t s)
{
    const int threads = 128;
    const size_t smem = cast_smem(threads / 32, (p->n_dirs + 31) / 32, use_wide(p));
    const int per_sm = p->blocks_per_sm > 0 ? p->blocks_per_sm : RC_BATCH_MIN_BLOCKS;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (n_items * 32 + threads - 1) / threads;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (use_wide(p))
        k_batch<false, true><<<(unsigned)blocks, threads, smem, s>>>(d_parts, n_parts, n_items, ppi, tdirs,
                                                                    p->n_dirs, p->origin_offset, work);
    else
        k_batch<false, false><<<(unsigned)blocks, threads, smem, s>>>(d_parts, n_parts, n_items, ppi, tdirs,
                                                                     p->n_dirs, p->origin_offset, work);
    RC_LAUNCHED();
    return RC_OK;
}

rc_status prepare_batch_kernel(int n_dirs)
{
    const size_t smem = cast_smem(4, (n_dirs + 31) / 32, true);
    if (smem > 48 * 1024) {
        RC_CUDA(cudaFuncSetAttribute(k_batch<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RC_CUDA(cudaFuncSetAttribute(k_batch<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    return RC_OK;
}

}  // namespace rc
