/*
 * oracle.c -- plain, slow, FP64 CPU oracle for hemispherical ray-casting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call this code;
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no source with the CUDA library.
 *
 * What it computes, and from which passage of the paper:
 *   - face normal / area / centroid ............. Section 3.1
 *   - sample points (face centroids, or seeded area-weighted random points)
 *                                                  Section 3.1
 *   - uniform hemisphere direction set ........... Section 3.1, Fig. 1
 *   - rotation of the set to each normal and the offset origin
 *                                                  Section 3.1
 *   - any-hit ray/triangle occlusion ............. Section 3.1, Fig. 2
 *   - per-point unobstructed count and ratio ..... Section 3.1
 *   - dominant axis and axis concentration ....... Section 3.3
 *   - orthogonal (six-axis) cast and tool travel . Sections 3.2, 3.3
 *
 * Arithmetic is FP64 except where a value is defined as an fp32 quantity
 * (the stored normal, the sample point, the ray origin and direction): those
 * are rounded exactly as the readings below state, so that the CUDA side,
 * implementing the same definitions separately, produces the same bits.
 * Build with -ffp-contract=off: no operation may be fused.
 *
 * Readings where the paper is silent:
 *   R1 normal orientation: right-hand rule on the stored winding.
 *   R2 direction set: Fibonacci hemisphere z_j = 1-(j+1/2)/N,
 *      phi_j = j*pi*(3-sqrt5), r_j = sqrt(1-z_j^2), in FP64, rounded to fp32.
 *   R3 local frame: branchless orthonormal basis of Duff et al. (2017) in
 *      fp32 arithmetic; d = (t1*hx + t2*hy) + n*hz per component, fp32, in
 *      that order, no fused multiply-add.
 *   R4 origin: o = fl32(p + eps*n) evaluated in FP64.
 *   R5 occlusion: a ray is obstructed iff some triangle (any, including the
 *      sample's own; both sides) meets o + t d at t > 0.
 *   R6 ambiguity band (tau = 1e-9, R = max(1, |o|inf, |A|inf, |B|inf, |C|inf)):
 *      a ray/triangle pair is AMBIGUOUS when the ray's line passes within
 *      tau*R of an edge line of the triangle while no other edge puts it
 *      clearly outside, or when the plane crossing lies within tau*R of the
 *      origin along the ray.  A ray is HIT if some pair is a clear hit,
 *      otherwise AMBIGUOUS if some pair is ambiguous, otherwise MISS.
 *   R7 area sampling: splitmix64 counter stream; triangle chosen by an
 *      integer (2^32-quantised) area CDF; point by Osada et al. (2002).
 *   R9 re-analysis of an edited part (same triangle list, moved vertices):
 *      every sample point stays on its face -- in area mode at the position
 *      its own u1, u2 give on the moved triangle, in centroid mode at the
 *      moved centroid -- and the result is the full analysis of the edited
 *      part at those points.
 *   R8 orthogonal eligibility: axis a is eligible for a point with normal n
 *      when n.a >= -parallel_tol (FP64, x, y, z order); a face parallel to
 *      the axis is side-milled, and the tolerance absorbs the tilt that fp32
 *      vertex rounding gives the normals of such faces.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_TAU 1e-9

/* ------------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the published mixer.     */
/* ------------------------------------------------------------------------ */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* k-th uniform double in [0,1) of sample i: 53 high bits of
 * splitmix64(seed XOR golden*(3i+k)). */
static double or_uniform(uint64_t seed, int64_t i, int k)
{
    uint64_t ctr = (uint64_t)(3 * i + k) * 0x9E3779B97F4A7C15ULL;
    uint64_t r = or_splitmix64(seed ^ ctr);
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Face preparation (Section 3.1: "for each triangular face, the centroid,  */
/* surface normal and area are computed").                                  */
/* ------------------------------------------------------------------------ */
static void cross3(const double* u, const double* v, double* w)
{
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

static double dot3(const double* u, const double* v)
{
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

static void load_vert(const float* V, int32_t idx, double* out)
{
    out[0] = V[3 * (int64_t)idx + 0];
    out[1] = V[3 * (int64_t)idx + 1];
    out[2] = V[3 * (int64_t)idx + 2];
}

/* c = (B-A) x (C-A) in FP64; area = |c|/2; n = fl32(c/|c|) (zero for a
 * zero-area triangle); centroid = fl32((A+B+C)/3). */
void or_face_prep(const float* V, const int32_t* F, int64_t T, float* nrm, double* area,
                  float* centroid)
{
    for (int64_t f = 0; f < T; ++f) {
        double A[3], B[3], C[3], e1[3], e2[3], c[3];
        load_vert(V, F[3 * f + 0], A);
        load_vert(V, F[3 * f + 1], B);
        load_vert(V, F[3 * f + 2], C);
        for (int k = 0; k < 3; ++k) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; }
        cross3(e1, e2, c);
        double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (area) area[f] = 0.5 * len;
        if (nrm) {
            for (int k = 0; k < 3; ++k) nrm[3 * f + k] = len > 0.0 ? (float)(c[k] / len) : 0.0f;
        }
        if (centroid) {
            for (int k = 0; k < 3; ++k) centroid[3 * f + k] = (float)((A[k] + B[k] + C[k]) / 3.0);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sample points (Section 3.1 uses face centroids; the area-weighted random */
/* mode is reading R7).                                                     */
/* ------------------------------------------------------------------------ */
/* Points kept on given faces (re-analysis of an edited part whose triangle  */
/* list is unchanged, reading R9): point i lies on face[i] at the barycentric */
/* position its own u1, u2 give in area mode; in centroid mode at the face   */
/* centroid.  Returns the first out-of-range face position, or -1.          */
/* ------------------------------------------------------------------------ */
int64_t or_sample_on_faces(const float* V, const int32_t* F, int64_t T, int64_t n, uint64_t seed,
                           int centroid, const int32_t* face, float* P, float* Nout)
{
    float* nrm = (float*)malloc(sizeof(float) * 3 * (size_t)(T > 0 ? T : 1));
    float* cen = (float*)malloc(sizeof(float) * 3 * (size_t)(T > 0 ? T : 1));
    double* area = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    or_face_prep(V, F, T, nrm, area, cen);
    int64_t bad = -1;
    for (int64_t i = 0; i < n && bad < 0; ++i) {
        const int64_t f = face[i];
        if (f < 0 || f >= T) { bad = i; break; }
        if (centroid) {
            for (int k = 0; k < 3; ++k) { P[3 * i + k] = cen[3 * f + k]; Nout[3 * i + k] = nrm[3 * f + k]; }
            continue;
        }
        double u1 = or_uniform(seed, i, 1), u2 = or_uniform(seed, i, 2);
        double A[3], B[3], C[3];
        load_vert(V, F[3 * f + 0], A);
        load_vert(V, F[3 * f + 1], B);
        load_vert(V, F[3 * f + 2], C);
        double s = sqrt(u1);
        double wa = 1.0 - s, wb = s * (1.0 - u2), wc = s * u2;
        for (int k = 0; k < 3; ++k) {
            double p = wa * A[k] + wb * B[k];
            p = p + wc * C[k];
            P[3 * i + k] = (float)p;
            Nout[3 * i + k] = nrm[3 * f + k];
        }
    }
    free(nrm); free(cen); free(area);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Area mode.  Returns 0 on success, -1 when the part has no positive area. */
int or_sample_area(const float* V, const int32_t* F, int64_t T, int64_t n, uint64_t seed,
                   float* P, float* Nout, int32_t* face)
{
    double* area = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    float* nrm = (float*)malloc(sizeof(float) * 3 * (size_t)(T > 0 ? T : 1));
    int64_t* cdf = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
    or_face_prep(V, F, T, nrm, area, NULL);
    double amax = 0.0;
    for (int64_t f = 0; f < T; ++f) if (area[f] > amax) amax = area[f];
    if (!(amax > 0.0)) { free(area); free(nrm); free(cdf); return -1; }
    /* quantised areas a_f = llround(area_f / amax * 2^32); inclusive prefix */
    int64_t run = 0;
    for (int64_t f = 0; f < T; ++f) {
        run += (int64_t)llround(area[f] / amax * 4294967296.0);
        cdf[f] = run;
    }
    int64_t total = run;
    for (int64_t i = 0; i < n; ++i) {
        double u0 = or_uniform(seed, i, 0), u1 = or_uniform(seed, i, 1), u2 = or_uniform(seed, i, 2);
        int64_t target = (int64_t)floor(u0 * (double)total);
        /* first f with cdf[f] > target */
        int64_t lo = 0, hi = T - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > target) hi = mid; else lo = mid + 1;
        }
        int64_t f = lo;
        double A[3], B[3], C[3];
        load_vert(V, F[3 * f + 0], A);
        load_vert(V, F[3 * f + 1], B);
        load_vert(V, F[3 * f + 2], C);
        /* Osada et al. 2002: p = (1-s)A + s(1-u2)B + s*u2*C, s = sqrt(u1) */
        double s = sqrt(u1);
        double wa = 1.0 - s, wb = s * (1.0 - u2), wc = s * u2;
        for (int k = 0; k < 3; ++k) {
            double p = wa * A[k] + wb * B[k];
            p = p + wc * C[k];
            P[3 * i + k] = (float)p;
            Nout[3 * i + k] = nrm[3 * f + k];
        }
        face[i] = (int32_t)f;
    }
    free(area); free(nrm); free(cdf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Hemisphere direction set (Section 3.1, Fig. 1; reading R2).              */
/* ------------------------------------------------------------------------ */
void or_direction_table(int32_t N, double* h64, float* h32)
{
    const double ga = M_PI * (3.0 - sqrt(5.0));
    for (int32_t j = 0; j < N; ++j) {
        double z = 1.0 - ((double)j + 0.5) / (double)N;
        double r = sqrt(1.0 - z * z);
        double phi = (double)j * ga;
        double h[3] = {r * cos(phi), r * sin(phi), z};
        for (int k = 0; k < 3; ++k) {
            if (h64) h64[3 * j + k] = h[k];
            if (h32) h32[3 * j + k] = (float)h[k];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Ray construction (Section 3.1: samples rotated to the face normal, cast  */
/* from an offset point; readings R3, R4).                                  */
/* ------------------------------------------------------------------------ */
static void onb_f32(const float* n, float* t1, float* t2)
{
    float sgn = copysignf(1.0f, n[2]);
    float a = -1.0f / (sgn + n[2]);
    float b = n[0] * n[1] * a;
    t1[0] = 1.0f + sgn * n[0] * n[0] * a;
    t1[1] = sgn * b;
    t1[2] = -sgn * n[0];
    t2[0] = b;
    t2[1] = sgn + n[1] * n[1] * a;
    t2[2] = -n[1];
}

void or_ray_dir(const float* n, const float* h, float* d)
{
    float t1[3], t2[3];
    onb_f32(n, t1, t2);
    for (int k = 0; k < 3; ++k) {
        float x = t1[k] * h[0];
        float y = t2[k] * h[1];
        float s = x + y;
        float z = n[k] * h[2];
        d[k] = s + z;
    }
}

void or_ray_origin(const float* p, const float* n, double eps, float* o)
{
    for (int k = 0; k < 3; ++k) {
        double off = eps * (double)n[k];
        o[k] = (float)((double)p[k] + off);
    }
}

/* Directions of point normal n for the whole table (exported for tests). */
void or_ray_dirs(const float* n, const float* h32, int32_t N, float* D)
{
    for (int32_t j = 0; j < N; ++j) or_ray_dir(n, h32 + 3 * j, D + 3 * j);
}

/* ------------------------------------------------------------------------ */
/* Ray / triangle predicate (Section 3.1, Fig. 2; readings R5, R6).          */
/* ------------------------------------------------------------------------ */
enum { OR_MISS = 0, OR_HIT = 1, OR_AMB = 2 };

static double maxabs3(const double* v)
{
    double m = fabs(v[0]);
    if (fabs(v[1]) > m) m = fabs(v[1]);
    if (fabs(v[2]) > m) m = fabs(v[2]);
    return m;
}

static double norm2(const double* v) { return sqrt(dot3(v, v)); }

/* Classify the pair (ray o + t d, triangle ABC).
 *
 * With a = A-o, b = B-o, c = C-o, the signed volumes
 *   U = det(b, C-B, d)   (edge BC),  V = det(c, A-C, d)  (edge CA),
 *   W = det(a, B-A, d)   (edge AB)
 * are each |e x d| times the signed distance between the ray's line and
 * that edge's line; the line meets the closed triangle iff U, V, W are all
 * >= 0 or all <= 0.  The plane crossing is t = (N.a)/(N.d) with
 * N = (B-A) x (C-A). */
int or_pair(const double* o, const double* d, const double* A, const double* B,
            const double* C)
{
    double a[3], b[3], c[3], eab[3], ebc[3], eca[3], eac[3], w[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = A[k] - o[k];
        b[k] = B[k] - o[k];
        c[k] = C[k] - o[k];
        eab[k] = B[k] - A[k];
        ebc[k] = C[k] - B[k];
        eca[k] = A[k] - C[k];
        eac[k] = C[k] - A[k];
    }
    double R = 1.0, m;
    if ((m = maxabs3(o)) > R) R = m;
    if ((m = maxabs3(A)) > R) R = m;
    if ((m = maxabs3(B)) > R) R = m;
    if ((m = maxabs3(C)) > R) R = m;
    const double band = OR_TAU * R;

    double E[3], L[3];
    cross3(b, ebc, w); E[0] = dot3(w, d);
    cross3(c, eca, w); E[1] = dot3(w, d);
    cross3(a, eab, w); E[2] = dot3(w, d);
    cross3(ebc, d, w); L[0] = norm2(w);
    cross3(eca, d, w); L[1] = norm2(w);
    cross3(eab, d, w); L[2] = norm2(w);

    int pos = 0, neg = 0, small = 0;
    for (int k = 0; k < 3; ++k) {
        if (fabs(E[k]) <= band * L[k]) { small = 1; continue; }
        if (E[k] > 0.0) pos = 1; else neg = 1;
    }
    if (pos && neg) return OR_MISS;          /* clearly outside an edge */

    double N[3];
    cross3(eab, eac, N);
    double nd = dot3(N, d);
    double na = dot3(N, a);
    if (nd == 0.0) return small ? OR_AMB : OR_MISS;
    /* crossing within tau*R of the origin along the ray */
    if (fabs(na) * norm2(d) <= band * fabs(nd)) return OR_AMB;
    int ahead = (na > 0.0) == (nd > 0.0);
    if (!ahead) return OR_MISS;
    return small ? OR_AMB : OR_HIT;
}

/* Exported wrapper taking fp32 ray and triangle (promoted exactly). */
int or_pair_f32(const float* o, const float* d, const float* A, const float* B, const float* C)
{
    double o64[3], d64[3], A64[3], B64[3], C64[3];
    for (int k = 0; k < 3; ++k) {
        o64[k] = o[k]; d64[k] = d[k]; A64[k] = A[k]; B64[k] = B[k]; C64[k] = C[k];
    }
    return or_pair(o64, d64, A64, B64, C64);
}

/* ------------------------------------------------------------------------ */
/* Acceleration: brute force, or a plain top-down median-split BVH in FP64. */
/* Boxes are widened by 4*tau*R and the slab test admits t >= -2*tau*R/|d|, */
/* so the BVH never skips a pair the brute force would call HIT or AMB.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
    int64_t left, right;   /* children, or -1 */
    int64_t first, count;  /* leaf range in the permuted triangle list */
} or_node;

typedef struct {
    const float* V;
    const int32_t* F;
    int64_t T;
    or_node* nodes;
    int64_t n_nodes;
    int64_t* perm;
    double* tri;          /* 9 doubles per permuted triangle */
    double pad;           /* box widening */
} or_bvh;

static void tri_bounds(const double* t, double* lo, double* hi)
{
    for (int k = 0; k < 3; ++k) {
        double a = t[k], b = t[3 + k], c = t[6 + k];
        lo[k] = fmin(a, fmin(b, c));
        hi[k] = fmax(a, fmax(b, c));
    }
}

typedef struct { double* cen; int64_t* idx; } or_sel_ctx;

/* quickselect: put the k-th smallest key (by cen[idx*3+axis]) at position k */
static void or_select(int64_t* idx, const double* cen, int axis, int64_t lo, int64_t hi, int64_t k)
{
    while (hi > lo) {
        double pivot = cen[3 * idx[(lo + hi) / 2] + axis];
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (cen[3 * idx[i] + axis] < pivot) ++i;
            while (cen[3 * idx[j] + axis] > pivot) --j;
            if (i <= j) { int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t; ++i; --j; }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return;
    }
}

static int64_t or_build_rec(or_bvh* b, const double* cen, const double* tb, int64_t lo, int64_t hi)
{
    int64_t id = b->n_nodes++;
    or_node* nd = &b->nodes[id];
    for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = lo; i < hi; ++i) {
        int64_t t = b->perm[i];
        for (int k = 0; k < 3; ++k) {
            nd->lo[k] = fmin(nd->lo[k], tb[6 * t + k]);
            nd->hi[k] = fmax(nd->hi[k], tb[6 * t + 3 + k]);
            clo[k] = fmin(clo[k], cen[3 * t + k]);
            chi[k] = fmax(chi[k], cen[3 * t + k]);
        }
    }
    for (int k = 0; k < 3; ++k) { nd->lo[k] -= b->pad; nd->hi[k] += b->pad; }
    nd->left = nd->right = -1;
    nd->first = lo;
    nd->count = hi - lo;
    if (hi - lo <= 4) return id;
    int axis = 0;
    double ext = chi[0] - clo[0];
    if (chi[1] - clo[1] > ext) { axis = 1; ext = chi[1] - clo[1]; }
    if (chi[2] - clo[2] > ext) { axis = 2; }
    int64_t mid = lo + (hi - lo) / 2;
    or_select(b->perm, cen, axis, lo, hi - 1, mid);
    int64_t l = or_build_rec(b, cen, tb, lo, mid);
    int64_t r = or_build_rec(b, cen, tb, mid, hi);
    nd = &b->nodes[id];
    nd->left = l;
    nd->right = r;
    nd->count = 0;
    return id;
}

void* or_bvh_build(const float* V, int64_t nV, const int32_t* F, int64_t T)
{
    or_bvh* b = (or_bvh*)calloc(1, sizeof(or_bvh));
    b->V = V; b->F = F; b->T = T;
    double R = 1.0;
    for (int64_t i = 0; i < 3 * nV; ++i) if (fabs((double)V[i]) > R) R = fabs((double)V[i]);
    /* origins sit within a few offsets of the surface; +1 covers them */
    b->pad = 4.0 * OR_TAU * (R + 1.0);
    b->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
    b->nodes = (or_node*)malloc(sizeof(or_node) * (size_t)(2 * T + 1));
    double* cen = (double*)malloc(sizeof(double) * 3 * (size_t)(T > 0 ? T : 1));
    double* tb = (double*)malloc(sizeof(double) * 6 * (size_t)(T > 0 ? T : 1));
    double* raw = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    for (int64_t t = 0; t < T; ++t) {
        load_vert(V, F[3 * t + 0], raw + 9 * t);
        load_vert(V, F[3 * t + 1], raw + 9 * t + 3);
        load_vert(V, F[3 * t + 2], raw + 9 * t + 6);
        tri_bounds(raw + 9 * t, tb + 6 * t, tb + 6 * t + 3);
        for (int k = 0; k < 3; ++k) cen[3 * t + k] = 0.5 * (tb[6 * t + k] + tb[6 * t + 3 + k]);
        b->perm[t] = t;
    }
    b->n_nodes = 0;
    if (T > 0) or_build_rec(b, cen, tb, 0, T);
    b->tri = (double*)malloc(sizeof(double) * 9 * (size_t)(T > 0 ? T : 1));
    for (int64_t i = 0; i < T; ++i) memcpy(b->tri + 9 * i, raw + 9 * b->perm[i], sizeof(double) * 9);
    free(cen); free(tb); free(raw);
    return b;
}

void or_bvh_free(void* p)
{
    or_bvh* b = (or_bvh*)p;
    if (!b) return;
    free(b->perm); free(b->nodes); free(b->tri); free(b);
}

int64_t or_bvh_nodes(void* p) { return ((or_bvh*)p)->n_nodes; }

static int box_hit(const or_node* nd, const double* o, const double* d, double tlo)
{
    double t0 = tlo, t1 = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < nd->lo[k] || o[k] > nd->hi[k]) return 0;
            continue;
        }
        double inv = 1.0 / d[k];
        double a = (nd->lo[k] - o[k]) * inv, b = (nd->hi[k] - o[k]) * inv;
        if (a > b) { double t = a; a = b; b = t; }
        a -= 1e-12 * (fabs(a) + 1.0);
        b += 1e-12 * (fabs(b) + 1.0);
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* One ray against the BVH (or all triangles when b is the brute-force flag). */
static int or_ray_bvh(const or_bvh* b, const double* o, const double* d)
{
    if (b->T == 0) return OR_MISS;
    double tlo = -2.0 * b->pad / norm2(d);
    int64_t stack[256];
    int sp = 0, amb = 0;
    stack[sp++] = 0;
    while (sp) {
        const or_node* nd = &b->nodes[stack[--sp]];
        if (!box_hit(nd, o, d, tlo)) continue;
        if (nd->left < 0) {
            for (int64_t i = nd->first; i < nd->first + nd->count; ++i) {
                const double* t = b->tri + 9 * i;
                int r = or_pair(o, d, t, t + 3, t + 6);
                if (r == OR_HIT) return OR_HIT;
                if (r == OR_AMB) amb = 1;
            }
        } else {
            stack[sp++] = nd->right;
            stack[sp++] = nd->left;
        }
    }
    return amb ? OR_AMB : OR_MISS;
}

static int or_ray_brute(const float* V, const int32_t* F, int64_t T, const double* o, const double* d)
{
    int amb = 0;
    for (int64_t t = 0; t < T; ++t) {
        double A[3], B[3], C[3];
        load_vert(V, F[3 * t + 0], A);
        load_vert(V, F[3 * t + 1], B);
        load_vert(V, F[3 * t + 2], C);
        int r = or_pair(o, d, A, B, C);
        if (r == OR_HIT) return OR_HIT;
        if (r == OR_AMB) amb = 1;
    }
    return amb ? OR_AMB : OR_MISS;
}

/* ------------------------------------------------------------------------ */
/* Threaded drivers                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* geometry */
    const or_bvh* bvh;   /* NULL -> brute force */
    const float* V;
    const int32_t* F;
    int64_t T;
    /* work */
    int kind;            /* 0 rays, 1 hemisphere, 2 orthogonal */
    double par_tol;      /* orthogonal eligibility tolerance (R8) */
    int64_t n;           /* work items */
    int64_t next;        /* shared cursor (atomic) */
    /* rays */
    const float* O;
    const float* D;
    int8_t* state;
    /* hemisphere / orthogonal */
    const float* P;
    const float* Nrm;
    double eps;
    int32_t N;
    const float* h32;
    uint32_t* bits;
    uint32_t* amb;
    int32_t* count;
    const float* axes;   /* 6 x 3 fp32 directions */
    uint8_t* mask;
    uint8_t* amask;
} or_job;

static int or_trace(const or_job* J, const float* o32, const float* d32)
{
    double o[3] = {o32[0], o32[1], o32[2]}, d[3] = {d32[0], d32[1], d32[2]};
    return J->bvh ? or_ray_bvh(J->bvh, o, d) : or_ray_brute(J->V, J->F, J->T, o, d);
}

static void* or_worker(void* arg)
{
    or_job* J = (or_job*)arg;
    const int64_t chunk = J->kind == 0 ? 256 : 1;
    for (;;) {
        int64_t i0 = __atomic_fetch_add(&J->next, chunk, __ATOMIC_RELAXED);
        if (i0 >= J->n) break;
        int64_t i1 = i0 + chunk < J->n ? i0 + chunk : J->n;
        for (int64_t i = i0; i < i1; ++i) {
            if (J->kind == 0) {
                J->state[i] = (int8_t)or_trace(J, J->O + 3 * i, J->D + 3 * i);
            } else if (J->kind == 1) {
                float o[3], d[3];
                or_ray_origin(J->P + 3 * i, J->Nrm + 3 * i, J->eps, o);
                int32_t W = (J->N + 31) / 32, cnt = 0;
                uint32_t* brow = J->bits + (int64_t)W * i;
                uint32_t* arow = J->amb ? J->amb + (int64_t)W * i : NULL;
                for (int32_t w = 0; w < W; ++w) { brow[w] = 0; if (arow) arow[w] = 0; }
                for (int32_t j = 0; j < J->N; ++j) {
                    or_ray_dir(J->Nrm + 3 * i, J->h32 + 3 * j, d);
                    int r = or_trace(J, o, d);
                    if (r == OR_MISS) { brow[j >> 5] |= 1u << (j & 31); ++cnt; }
                    if (r == OR_AMB && arow) arow[j >> 5] |= 1u << (j & 31);
                }
                J->count[i] = cnt;
            } else {
                float o[3];
                or_ray_origin(J->P + 3 * i, J->Nrm + 3 * i, J->eps, o);
                uint8_t m = 0, am = 0;
                for (int a = 0; a < 6; ++a) {
                    const float* ax = J->axes + 3 * a;
                    const float* n = J->Nrm + 3 * i;
                    /* eligibility (R8): n . a >= -parallel_tol in FP64 (x, y, z order) */
                    double nd = (double)n[0] * ax[0] + (double)n[1] * ax[1];
                    nd = nd + (double)n[2] * ax[2];
                    if (!(nd >= -J->par_tol)) continue;
                    int r = or_trace(J, o, ax);
                    if (r == OR_MISS) m |= (uint8_t)(1u << a);
                    if (r == OR_AMB) am |= (uint8_t)(1u << a);
                }
                J->mask[i] = m;
                if (J->amask) J->amask[i] = am;
            }
        }
    }
    return NULL;
}

static void or_run(or_job* J, int nthreads)
{
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    J->next = 0;
    pthread_t th[512];
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, or_worker, J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

int or_num_cores(void) { return (int)sysconf(_SC_NPROCESSORS_ONLN); }

/* Per-ray state (0 MISS, 1 HIT, 2 AMBIGUOUS) for explicit fp32 rays. */
void or_cast_rays(void* bvh, const float* V, const int32_t* F, int64_t T, const float* O,
                  const float* D, int64_t nrays, int8_t* state, int nthreads)
{
    or_job J;
    memset(&J, 0, sizeof J);
    J.bvh = (const or_bvh*)bvh; J.V = V; J.F = F; J.T = T;
    J.kind = 0; J.n = nrays; J.O = O; J.D = D; J.state = state;
    or_run(&J, nthreads);
}

/* Hemisphere cast (Section 3.1): bit j of row i = 1 iff ray j of point i is
 * MISS (unobstructed); amb bit = 1 iff AMBIGUOUS; count = popcount(bits). */
void or_hemisphere(void* bvh, const float* V, const int32_t* F, int64_t T, const float* P,
                   const float* Nrm, int64_t n, int32_t N, double eps, uint32_t* bits,
                   uint32_t* amb, int32_t* count, int nthreads)
{
    float* h32 = (float*)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    or_direction_table(N, NULL, h32);
    or_job J;
    memset(&J, 0, sizeof J);
    J.bvh = (const or_bvh*)bvh; J.V = V; J.F = F; J.T = T;
    J.kind = 1; J.n = n; J.P = P; J.Nrm = Nrm; J.eps = eps; J.N = N; J.h32 = h32;
    J.bits = bits; J.amb = amb; J.count = count;
    or_run(&J, nthreads);
    free(h32);
}

/* Orthogonal cast (Section 3.2): axes are six fp32 directions
 * (+X', -X', +Y', -Y', +Z', -Z' of the machining frame). */
void or_orthogonal(void* bvh, const float* V, const int32_t* F, int64_t T, const float* P,
                   const float* Nrm, int64_t n, const float* axes, double eps, double par_tol,
                   uint8_t* mask, uint8_t* amask, int nthreads)
{
    or_job J;
    memset(&J, 0, sizeof J);
    J.bvh = (const or_bvh*)bvh; J.V = V; J.F = F; J.T = T;
    J.kind = 2; J.n = n; J.P = P; J.Nrm = Nrm; J.eps = eps; J.axes = axes; J.par_tol = par_tol;
    J.mask = mask; J.amask = amask;
    or_run(&J, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Directional variability (Section 3.3): per point, the fixed-point sum of  */
/* visible world directions M_k = sum llrint(d_k * 2^40), the dominant axis  */
/* argmax_k |M_k| (ties to the lower axis), and the per-axis counts of      */
/* visible rays whose largest |component| is axis k (ties to the lower k).  */
/* ------------------------------------------------------------------------ */
void or_variability(const uint32_t* bits, const float* Nrm, int64_t n, int32_t N,
                    int64_t* Msum /*n x 3*/, int32_t* axis_cnt /*n x 3*/, int8_t* dom)
{
    float* h32 = (float*)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    or_direction_table(N, NULL, h32);
    const int32_t W = (N + 31) / 32;
    for (int64_t i = 0; i < n; ++i) {
        int64_t M[3] = {0, 0, 0};
        int32_t ac[3] = {0, 0, 0};
        int32_t cnt = 0;
        for (int32_t j = 0; j < N; ++j) {
            if (!((bits[(int64_t)W * i + (j >> 5)] >> (j & 31)) & 1u)) continue;
            float d[3];
            or_ray_dir(Nrm + 3 * i, h32 + 3 * j, d);
            for (int k = 0; k < 3; ++k) M[k] += (int64_t)llrint((double)d[k] * 1099511627776.0);
            int best = 0;
            if (fabsf(d[1]) > fabsf(d[best])) best = 1;
            if (fabsf(d[2]) > fabsf(d[best])) best = 2;
            ac[best]++;
            cnt++;
        }
        int8_t dm = -1;
        if (cnt > 0) {
            dm = 0;
            for (int k = 1; k < 3; ++k) {
                int64_t mk = M[k] < 0 ? -M[k] : M[k];
                int64_t md = M[dm] < 0 ? -M[dm] : M[dm];
                if (mk > md) dm = (int8_t)k;
            }
        }
        for (int k = 0; k < 3; ++k) { Msum[3 * i + k] = M[k]; axis_cnt[3 * i + k] = ac[k]; }
        dom[i] = dm;
    }
    free(h32);
}
