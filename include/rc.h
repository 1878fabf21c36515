/*
 * rc.h -- C ABI of the GB300 (sm_103a) hemispherical ray-casting library.
 *
 * The library implements the hot path of the milling-accessibility method of
 * Baltadouros, Lauwers and Duflou, "Hemispherical Ray-Casting Analysis for
 * Milling Configuration Classification and Machinability Assessment":
 * every surface sample point of a triangulated part casts N hemisphere
 * directions about its normal as any-hit occlusion rays against the part's
 * own triangles (Section 3.1), the visible directions are reduced to
 * directional indicators (Section 3.3), the part is classified as 3-axis or
 * multi-axis (Section 3.3), and 3-axis parts get a six-axis orthogonal cast
 * (Section 3.2) and a minimum-setup search (Section 3.3).
 *
 * Conventions (apply to every call):
 *  - Status: every call returns rc_status.  RC_OK is 0.  A failing call
 *    stores a message retrievable with rc_last_error() (thread-local).
 *    Errors in pointers, sizes and parameters are detected on the host and
 *    returned before any kernel is launched (a cast may already have queued
 *    the zeroing of its d_counters array).  The contents of device arrays
 *    (vertex indices, vertex coordinates, face ids) are checked on the
 *    device by the calls that say so (rc_build_bvh, rc_refit_bvh,
 *    rc_sample_points_on_faces, rc_changed_faces): they synchronise
 *    `stream`, free their scratch and return RC_E_ARG.
 *  - Memory: arrays named d_* are DEVICE pointers owned by the caller
 *    (e.g. torch CUDA tensors); arrays named h_* are host pointers owned by
 *    the caller.  The library owns only the opaque handles it returns and
 *    internal scratch, which it allocates and frees itself.  No call keeps
 *    a caller pointer after it returns, except where stated (batches).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is queued asynchronously on it unless the call
 *    says it synchronises.  A call that forks work onto streams of its own
 *    (rc_analyze_part, the batch's graph branches, the server's slots) joins
 *    them before it returns or orders them before later work on `stream`.
 *  - Devices: a call that takes a BVH handle runs on the device the handle
 *    was built on; it makes that device current on the calling thread and
 *    leaves it current (rc_destroy_bvh and the server calls restore the
 *    caller's device), so `stream` must belong to that device.
 *  - Layouts: points, normals and vertices are row-major float32 xyz
 *    ([n][3]); faces are int32 vertex indices ([T][3]), wound
 *    counter-clockwise seen from outside (the normal is the right-hand rule
 *    on the stored winding).  Visibility bits: row i has W = ceil(n_dirs/32)
 *    uint32 words; bit (j & 31) of word (j >> 5) is 1 iff hemisphere
 *    direction j of point i is unobstructed; bits j >= n_dirs are 0.
 *  - Precision: traversal and intersection run in FP32 with a forward error
 *    bound per ray/triangle test; tests whose FP32 outcome is not certain
 *    are re-decided in FP64 (Section 3.1's intersection test made exact
 *    outside a 1e-9 relative ambiguity band).
 *  - Every kernel is hand-written CUDA for sm_103a.  There is no CPU
 *    fallback: without a usable GB300 the calls fail with RC_E_CUDA.
 */
#ifndef RC_H
#define RC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RC_OK = 0,
    RC_E_ARG = 1,          /* invalid argument (null pointer, bad size, bad mesh) */
    RC_E_CUDA = 2,         /* a CUDA runtime call failed */
    RC_E_OOM = 3,          /* device allocation failed or budget exceeded */
    RC_E_TIMEOUT = 4,      /* a bounded device wait ran out */
    RC_E_DEGENERATE = 5,   /* the part has no positive-area face to sample */
    RC_E_UNSUPPORTED = 6,  /* a limit of this implementation was exceeded */
    RC_E_DEVICE = 7        /* a kernel reported an internal error (see counters) */
} rc_status;

typedef struct rc_bvh_s* rc_bvh;

/* Sampling modes (Section 3.1 samples one point per face at its centroid;
 * the area-weighted random mode draws points in proportion to area). */
enum { RC_SAMPLE_AREA_RANDOM = 0, RC_SAMPLE_FACE_CENTROID = 1 };

/* Analysis parameters.  Fill with rc_params_default() and override. */
typedef struct {
    int32_t n_dirs;          /* N: hemisphere directions per point, 1..65536 (the paper uses 150) */
    int32_t sample_mode;     /* RC_SAMPLE_* */
    double origin_offset;    /* mm; rays start at fl32(p + origin_offset * n) (Section 3.1) */
    uint64_t seed;           /* area-random sampling seed */
    float frame[9];          /* row-major 3x3 machining frame; its columns are X', Y', Z' (Section 3.2); finite,
                                no zero column (RC_E_ARG) */
    float tool_length;       /* mm; reachability threshold (Section 3.3); >= 0, +inf = no limit (RC_E_ARG otherwise) */
    int32_t conc_mode;       /* 0: share of visible rays along the dominant axis; 1: |mean direction| along it */
    double t_acc;            /* multi-axis if overall accessibility < t_acc (Section 3.3) */
    double t_share;          /* ... or the largest dominant-axis share < t_share */
    double t_conc;           /* ... or the mean axis concentration > t_conc (none of the three NaN: RC_E_ARG) */
    int32_t block_threads;   /* traversal kernel: threads per block (0 = default; only 128 is supported) */
    int32_t blocks_per_sm;   /* traversal kernel: resident blocks per SM (0 = tuned default) */
    int32_t collect_stats;   /* 1: casts run the instrumented traversal (counters[4..5]) */
    int32_t always_setups;   /* rc_analyze_part: 1 = orthogonal cast and setups for every part, 0 = 3-axis parts only
                                (0 or 1: RC_E_ARG otherwise) */
    int32_t point_order;     /* hemispherical cast: 0 = cast points in Morton order (default), 1 = in index order */
    int32_t tile_mode;       /* hemispherical cast: 0 = directions in coherent tiles of 32 (default), 1 = index order */
    int32_t points_per_item; /* batched cast: points per work item (0 = 1) */
    int32_t launch_mode;     /* casts: 0 = persistent grid (default), 1 = one warp per point, grid sized to the work
                                (short blocks, so concurrent casts on other streams interleave) */
    int32_t fetch_mode;      /* reserved, must be 0 (the lanes of a warp cast one tile of 32 rays together) */
    int32_t tree_width;      /* casts: 0 or 4 = 4-wide tree (default), 2 = binary tree */
    double parallel_tol;     /* orthogonal cast: axis a is eligible when n.a >= -parallel_tol (FP64); a face
                                parallel to the axis is side-milled, and the tolerance absorbs the tilt that
                                fp32 vertex rounding gives such faces' normals; 0 .. 0.5, default 1e-4 */
} rc_params;

/* Part-level indicators (Sections 3.1 and 3.3). */
typedef struct {
    double overall_access;            /* sum w_i count_i / (N sum w_i) (Section 3.1's area-weighted score) */
    double overall_access_unweighted; /* sum count_i / (N n) */
    double axis_share[3];             /* fraction of counted points whose dominant axis is x, y, z */
    double mean_conc;                 /* mean axis concentration over counted points */
    int64_t n_points;                 /* n */
    int64_t n_counted;                /* points with at least one visible direction */
    int64_t n_zero_visible;           /* n - n_counted */
    int64_t dom_count[3];             /* counted points per dominant axis */
    int64_t count_sum;                /* sum of unobstructed counts */
    double weighted_count;            /* sum w_i count_i, FP64 in a fixed order (= count_sum for unit weights) */
    double weight_sum;                /* sum w_i, FP64 in a fixed order (= n for unit weights) */
    int64_t conc_sum_q;               /* sum llrint(conc_i * 2^40) over counted points */
} rc_summary;

/* Minimum-setup result (Section 3.3). */
typedef struct {
    int32_t setups_exact;    /* smallest number of axes covering every viable point (Section 5: theoretical minimum) */
    int32_t setups_greedy;   /* greedy set cover, ties to the lower axis (Section 3.3) */
    uint8_t chosen_exact;    /* bit a = axis a in (+X', -X', +Y', -Y', +Z', -Z') */
    uint8_t chosen_greedy;
    uint8_t pad[6];
    int64_t class_counts[4]; /* viable, over-threshold, inaccessible, fixture */
    int64_t mask_hist[64];   /* viable points per reachable-axis mask */
} rc_setups;

/* Geometry summary of a built BVH. */
typedef struct {
    int64_t n_tris;
    int64_t n_nodes;         /* packed internal nodes */
    int64_t node_bytes;
    int64_t tri_bytes;
    int32_t max_depth;       /* deepest leaf (root = 0) */
    int32_t leaf_size;       /* largest triangles per leaf */
    float scene_lo[3];
    float scene_hi[3];
} rc_bvh_info;

/* ---------------------------------------------------------------------- */
/* Library                                                                */
/* ---------------------------------------------------------------------- */

/* Fills *p with the defaults: n_dirs 256, area-random sampling, seed 0,
 * origin_offset 1e-4 mm, identity frame, tool_length 100 mm, conc_mode 0,
 * thresholds 0.60 / 0.45 / 0.41, parallel_tol 1e-4.  Returns RC_E_ARG if p is NULL. */
rc_status rc_params_default(rc_params* p);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* rc_last_error(void);

/* Number of kernels this library has launched in this process (all threads).
 * Used by benchmarks to report launch counts; never fails. */
int64_t rc_launch_count(void);

/* Waits for the work queued on `stream` (NULL = the legacy default stream)
 * and reports an error that asynchronous work raised there: RC_OK, or
 * RC_E_CUDA with the CUDA error text in rc_last_error().  The library's own
 * device-side failures (a traversal bound exceeded) are reported through
 * the counters of each call instead. */
rc_status rc_stream_status(void* stream);

/* ---------------------------------------------------------------------- */
/* Geometry and acceleration structure                                    */
/* ---------------------------------------------------------------------- */

/* Build the part's device acceleration structure (Section 3.1: "for each
 * triangular face, the centroid, surface normal and area are computed";
 * the BVH itself is not in the paper).  Steps, all on `stream`: FP64 face
 * normal/area/centroid, 48-bit Morton codes of triangle-box centres (16
 * bits per axis), LSD radix sort, Karras binary radix tree, bottom-up AABB
 * refit, packing into the traversal layout, collapse into the 4-wide tree
 * the default walk uses, integer area CDF for sampling.
 *   d_V [nV][3] float32, d_F [T][3] int32 (device, caller-owned; read
 *   during the call only -- the handle keeps its own copies).
 * Synchronises `stream` before returning (validation result).
 * Errors: RC_E_ARG for NULL pointers, nV < 3, T < 1, T > 2^28, an index
 * outside [0, nV) or a non-finite vertex; RC_E_UNSUPPORTED if a tree is
 * deeper than its traversal stack holds (binary depth 64 or more, or a
 * 4-wide depth d with 3d + 1 >= 96); RC_E_OOM; RC_E_CUDA. */
rc_status rc_build_bvh(const float* d_V, int64_t nV, const int32_t* d_F, int64_t T, void* stream,
                       rc_bvh* out);

/* Binary-tree builders for rc_build_bvh_ex. */
enum { RC_BUILDER_KARRAS = 0, RC_BUILDER_PLOC = 1 };

/* rc_build_bvh with a choice of the binary tree under the 4-wide tree:
 * RC_BUILDER_KARRAS (rc_build_bvh's: the binary radix tree of the sorted
 * Morton codes, Karras 2012) or RC_BUILDER_PLOC (parallel locally-ordered
 * clustering, Meister and Bittner 2018: mutual nearest neighbours by merged
 * surface area within 16 positions of the Morton order, merged round by
 * round; fewer node visits per ray, a slower build).  Both give the same
 * casts' results (up to rays decided by FP64-ambiguous pairs).  Errors: as
 * rc_build_bvh, and RC_E_ARG for an unknown builder. */
rc_status rc_build_bvh_ex(const float* d_V, int64_t nV, const int32_t* d_F, int64_t T, int32_t builder,
                          void* stream, rc_bvh* out);

/* Refit an existing handle to moved vertices of the same triangle list
 * (same F, same nV): recomputes face data, leaf and node boxes bottom-up
 * and the area CDF; the tree topology is kept.  Synchronises `stream`.
 * Errors as rc_build_bvh (non-finite vertices -> RC_E_ARG).  After a failed
 * refit the handle keeps its topology and index arrays, so later calls stay
 * within its buffers, but its geometry is undefined until a refit with
 * valid vertices succeeds; destroy or refit it. */
rc_status rc_refit_bvh(rc_bvh h, const float* d_V, void* stream);

/* Release a handle and its device memory.  NULL is accepted.  The memory
 * comes from CUDA's stream-ordered pool and is returned asynchronously, in
 * order on the legacy default stream, so destroying a handle never stalls
 * other streams; do not destroy a handle while work that uses it may still
 * run on another (non-blocking) stream. */
rc_status rc_destroy_bvh(rc_bvh h);

/* Sizes, depth and scene bounds of a built handle (host struct). */
rc_status rc_bvh_get_info(rc_bvh h, rc_bvh_info* out);

/* Index checks of a built tree (the device-side bounds checking that stands
 * in for a memory checker): every interior child of a 4-wide node must be a
 * node above its parent's number and below n_int (so no walk can cycle),
 * every leaf's triangle range inside [0, T), every used child box finite
 * with lo <= hi, every packed binary child inside its range, and every
 * triangle record's face id inside [0, T).  h_counts[6] receives the
 * violations of each kind in that order and, last, the number of 4-wide
 * nodes reached from the root.  Synchronises `stream`.
 * Errors: RC_E_ARG (NULL), RC_E_CUDA. */
rc_status rc_bvh_validate(rc_bvh h, int64_t* h_counts, void* stream);

/* ---------------------------------------------------------------------- */
/* Section 3.1: sampling, directions, hemispherical cast                  */
/* ---------------------------------------------------------------------- */

/* Sample points on the part (Section 3.1).
 * RC_SAMPLE_FACE_CENTROID: n must equal T; point f = fl32((A+B+C)/3),
 *   normal = face normal, face = f, weight = FP64 face area.
 * RC_SAMPLE_AREA_RANDOM: point i draws u0,u1,u2 from splitmix64 counters
 *   (seed XOR golden*(3i+k)); the face is the first f whose inclusive
 *   2^32-quantised area prefix exceeds floor(u0*total); the point is Osada
 *   et al.'s (1-s)A + s(1-u2)B + s*u2*C with s = sqrt(u1), in FP64; weight 1.
 *   d_P, d_N [n][3] float32; d_face [n] int32; d_weight [n] double (may be NULL).
 * n == 0 is a no-op.  Errors: RC_E_ARG (NULL, n < 0, centroid n != T),
 * RC_E_DEGENERATE (no positive-area face), RC_E_CUDA. */
rc_status rc_sample_points(rc_bvh h, int64_t n, const rc_params* p, float* d_P, float* d_N,
                           int32_t* d_face, double* d_weight, void* stream);

/* The canonical hemisphere direction set (Section 3.1, Fig. 1: a uniformly
 * sampled hemisphere; here the Fibonacci set z_j = 1-(j+1/2)/N,
 * phi_j = j*pi*(3-sqrt5), computed in FP64 on the host and rounded to
 * float32).  h_dirs [n_dirs][3] float32, host.  Errors: RC_E_ARG. */
rc_status rc_direction_table(int32_t n_dirs, float* h_dirs);

/* Hemispherical cast (Section 3.1: hemisphere samples rotated to each
 * normal, rays cast from an offset point, "GPU-accelerated ray-triangle
 * intersection tests determine whether rays are obstructed").
 * For point i and direction j the ray is o_i = fl32(p_i + eps*n_i) (FP64),
 * d_ij = (t1*hx + t2*hy) + n*hz in float32 with (t1, t2) the orthonormal
 * basis of Duff et al. (2017); it is obstructed iff some triangle meets it
 * at t > 0.  Normals are taken as given: unit normals (such as
 * rc_sample_points writes) let the walk skip what lies below a point's
 * tangent plane, and a normal whose squared length is further than
 * (1/(64 ceil(n_dirs/32)) - 2e-6) / 4 from 1 is cast without that shortcut,
 * with the same result for the rays as defined.
 *   d_P, d_N [n][3]; d_bits [n][W] uint32, W = ceil(n_dirs/32), (written); d_count [n]
 *   int32 unobstructed counts (written); d_counters int64[4] (written, may be
 *   NULL): rays cast, rays decided by an ambiguous pair, ray/triangle pairs
 *   re-tested in FP64, internal errors (must be 0).  With p->collect_stats
 *   the counters array must hold 8 entries and [4] receives the interior
 *   nodes fetched (112 B each on the 4-wide tree, 64 B on the binary tree)
 *   and [5] the triangles tested (48 B each) over all rays, from an
 *   instrumented copy of the same traversal.
 * n == 0 is a no-op.  Asynchronous.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_hemisphere_cast(rc_bvh h, const float* d_P, const float* d_N, int64_t n,
                             const rc_params* p, uint32_t* d_bits, int32_t* d_count,
                             int64_t* d_counters, void* stream);

/* The instrumented cast of rc_hemisphere_cast (as with p->collect_stats: the
 * same rays and decisions, counters int64[8] with the node and triangle
 * counts in [4] and [5]) that also lists the rays whose walk re-tested a
 * pair in FP64 (Section 3.1's intersection test made exact; see the
 * precision note above): d_list[k] = i * 65536 + j for point i and
 * direction j, in no particular order, for the first min(cap, total) such
 * rays; counters[6] receives the total.  For tests and measurement.
 *   d_list int64[cap] (device, may be NULL when cap == 0).
 * Asynchronous.  Errors: RC_E_ARG (NULL counters, cap < 0), RC_E_CUDA. */
rc_status rc_hemisphere_cast_retests(rc_bvh h, const float* d_P, const float* d_N, int64_t n,
                                     const rc_params* p, uint32_t* d_bits, int32_t* d_count,
                                     int64_t* d_counters, int64_t* d_list, int64_t cap, void* stream);

/* ---------------------------------------------------------------------- */
/* Section 3.3: directional variability and classification                */
/* ---------------------------------------------------------------------- */

/* Per-point and part-level directional indicators from the visibility
 * bits (Section 3.3: "directional biases in unobstructed rays are analyzed
 * to identify dominant axis alignment and directional concentration").
 * Per point: acc = count/N; M_k = sum over visible j of llrint(d_ij,k*2^40);
 * dom = argmax_k |M_k| (ties to the lower axis; -1 if nothing is visible);
 * conc (conc_mode 0) = share of visible rays whose largest |component| is
 * axis dom, (conc_mode 1) = |M_dom| / (2^40 count).
 *   d_bits [n][W], d_N [n][3] unit normals (the world directions d_ij are
 *   rebuilt from them as in rc_hemisphere_cast; the fixed-point sums are
 *   exact for |d_ij,k| < 16, which unit normals keep far inside);
 *   d_weight [n] (NULL = unit weights);
 *   outputs (each may be NULL): d_acc [n] float32, d_dom [n] int8,
 *   d_conc [n] float32, d_dir_area [N] double (sum over points of weight
 *   times visibility of direction j: exact for unit weights; with real
 *   weights FP64 sums whose order of addition is not fixed); h_summary
 *   (host, may be NULL).  The part-level weighted sums are FP64 sums in a
 *   fixed order (per point, per warp, per block, then over the blocks), so
 *   the summary is the same on every run; it differs from the exact
 *   weighted mean by a relative error of order 1e-15.
 * Synchronises `stream` when h_summary is not NULL.  Errors: RC_E_ARG,
 * RC_E_CUDA. */
rc_status rc_direction_variability(const uint32_t* d_bits, const float* d_N,
                                   const double* d_weight, int64_t n, const rc_params* p,
                                   float* d_acc, int8_t* d_dom, float* d_conc, double* d_dir_area,
                                   rc_summary* h_summary, void* stream);

/* Same computation and outputs as rc_direction_variability, but without
 * any allocation.  The paper has no counterpart: this exists for callers
 * that cannot let a library allocate device memory -- for example a process
 * that reserves its whole HBM budget for its own arena at start-up and
 * routes every allocation through it, or one that runs at its memory limit,
 * where a cudaMalloc/cudaMallocAsync inside the call would fail or break
 * the caller's accounting.  The call performs no device or host heap
 * allocation (no cudaMalloc, cudaFree or allocating library routine).
 * Its scratch -- the part-level sums, the per-block weighted partials and
 * the direction table -- lives in one static device array of 164,096
 * bytes, which every GPU that loads the library holds until the process
 * exits; hence p->n_dirs is limited to 8192 (larger values up to 65536
 * return RC_E_UNSUPPORTED).  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current)
 * and uploads the direction table, so make that first call before any
 * stream capture.  The array holds one direction table: a call whose
 * n_dirs differs from the last upload's on that device uploads its own
 * table from host memory on `stream` (refused with RC_E_UNSUPPORTED while
 * `stream` is being captured), and work already queued reads whichever
 * table the array holds when it runs.  The sums are cleared on `stream` at
 * every call.  All calls on a device share the array and it keeps the last
 * call's contents, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race with each other; serialise them.  Arguments,
 * outputs, synchronisation and errors are otherwise as for
 * rc_direction_variability. */
rc_status rc_direction_variability_noalloc(const uint32_t* d_bits, const float* d_N,
                                           const double* d_weight, int64_t n, const rc_params* p,
                                           float* d_acc, int8_t* d_dom, float* d_conc,
                                           double* d_dir_area, rc_summary* h_summary, void* stream);

/* Threshold classification (Section 3.3: "if any threshold is exceeded, the
 * part is classified as requiring multi-axis machining").  *label = 1
 * (multi-axis) iff overall_access < t_acc, or max axis_share < t_share, or
 * mean_conc > t_conc; else 0 (3-axis).  Host only.  Errors: RC_E_ARG for a
 * NULL argument or a NaN threshold. */
rc_status rc_classify(const rc_summary* s, const rc_params* p, int32_t* label);

/* ---------------------------------------------------------------------- */
/* Section 3.2 / 3.3: orthogonal cast, reachability, setups                */
/* ---------------------------------------------------------------------- */

/* Orthogonal (directional) cast (Section 3.2: rays along the six principal
 * directions of the canonical frame from the offset point, with the same
 * intersection kernel).  Axis a in (+X', -X', +Y', -Y', +Z', -Z') is
 * eligible iff n.a >= -parallel_tol (FP64) and accessible iff also
 * unobstructed.
 * Travel (Section 3.3, tool travel distance) = distance from p to the
 * part's bounding box (in frame coordinates) along a.
 *   d_mask [n] uint8 (bit a = accessible), d_travel [n][6] float32,
 *   d_counters int64[4] as for rc_hemisphere_cast (may be NULL; 8 entries
 *   with node and triangle counts when p->collect_stats is set).
 * Asynchronous.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_orthogonal_cast(rc_bvh h, const float* d_P, const float* d_N, int64_t n,
                             const rc_params* p, uint8_t* d_mask, float* d_travel,
                             int64_t* d_counters, void* stream);

/* Tool-aware accessibility along the six axes of the frame (a variant the
 * paper does not run: its rays are thin; the accessibility cones of the
 * prior art it cites account for the tool).  A ball-end tool of radius r
 * touches point p: centre c = p + (r + origin_offset) n.  Along axis a its
 * shank is sampled by the ray from c and ring_rays parallel rays from
 * c + r (cos t_k u + sin t_k v), t_k = 2 pi k / ring_rays, (u, v) the
 * branchless orthonormal basis of a (Duff et al. 2017), all in FP64 with
 * origins rounded to fp32.  Bit a of d_mask[i] is set iff a is eligible
 * (n.a >= -parallel_tol) and none of those rays is obstructed.  With r = 0
 * and ring_rays = 0 this is the mask of rc_orthogonal_cast.
 *   d_P, d_N [n][3]; d_mask [n] uint8 (written); d_counters int64[4] as
 *   for rc_orthogonal_cast (may be NULL).  Asynchronous.
 * Errors: RC_E_ARG (tool_radius outside [0, 1e4] mm, ring_rays outside
 * [0, 64]), RC_E_CUDA. */
rc_status rc_tool_cast(rc_bvh h, const float* d_P, const float* d_N, int64_t n, const rc_params* p,
                       double tool_radius, int32_t ring_rays, uint8_t* d_mask, int64_t* d_counters, void* stream);

/* Reachability, fixture exclusion, face classes and setup count (Section
 * 3.3: directions whose travel exceeds the tool length are discarded,
 * bounding-box faces are excluded as fixture surfaces, faces are viable /
 * over-threshold / fully inaccessible, and a set cover picks the setups).
 * A face is a fixture face when its three vertices lie within 1e-6*diag of
 * one bounding-box plane of the frame and its normal points out through
 * that plane to within 1e-6.
 *   d_mask [n], d_travel [n][6], d_face [n]: from the calls above;
 *   d_class [n] uint8 written (0 viable, 1 over-threshold, 2 inaccessible,
 *   3 fixture; may be NULL); h_out (host) receives counts, the 64-bin
 *   histogram of viable reachable masks and both covers.
 * Synchronises `stream`.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_min_setups(rc_bvh h, const uint8_t* d_mask, const float* d_travel,
                        const int32_t* d_face, int64_t n, const rc_params* p, uint8_t* d_class,
                        rc_setups* h_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Batches: many parts in one persistent launch                           */
/* ---------------------------------------------------------------------- */

/* Result of rc_analyze_part and of a batch's analysis part (host struct). */
typedef struct {
    rc_summary summary;          /* Section 3.3 indicators */
    rc_setups setups;            /* zero unless the setup stage ran */
    int32_t label;               /* 0 = 3-axis, 1 = multi-axis */
    int32_t setups_ran;          /* 1 if the orthogonal cast and setup search ran */
    int64_t cast_counters[4];    /* hemispherical cast: rays, ambiguous rays, FP64 re-tests, errors */
    int64_t ortho_counters[4];   /* orthogonal cast: same */
} rc_part_result;

typedef struct rc_batch_s* rc_batch;

/* Create an empty batch for the hemispherical cast of many parts with the
 * parameters *p (copied).  The paper casts one part at a time; a batch puts
 * the points of all its parts on one ray-work queue and casts them in one
 * persistent launch, replayed from a CUDA graph.  hbm_budget_bytes (0 = no
 * limit) bounds the device bytes of the parts the batch admits (see
 * rc_batch_add_part).  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_batch_create(const rc_params* p, int64_t hbm_budget_bytes, rc_batch* out);

/* Add a part: its handle and the device arrays of rc_hemisphere_cast
 * (points, normals, n, bits, counts, counters int64[4] or NULL).  The batch
 * keeps these pointers until rc_batch_clear/rc_batch_destroy: they must stay
 * valid.  *part_id (may be NULL) receives the part's index.  The part's
 * device bytes -- 12 nV + 260 T for its handle plus n (32 + 4 W) for its
 * points, normals, bits, counts and the batch's point order, W =
 * ceil(n_dirs / 32) -- count against the batch's budget.  Errors: RC_E_ARG,
 * RC_E_OOM (the part would exceed the budget; it is not added). */
rc_status rc_batch_add_part(rc_batch b, rc_bvh h, const float* d_P, const float* d_N, int64_t n,
                            uint32_t* d_bits, int32_t* d_count, int64_t* d_counters, int64_t* part_id);

/* Add a part for the whole path of Sections 3.1-3.3 (an analysis part): the
 * arrays of rc_batch_add_part plus the points' face ids d_face [n] (as from
 * rc_sample_points; kept until clear/destroy like the other pointers).  Its
 * launch casts the part's rays with the others, then -- in the same graph --
 * reduces its bits to the indicators of rc_direction_variability (unit
 * weights), casts the six axes of p->frame (rc_orthogonal_cast) and counts
 * its face classes and reachable-axis masks (rc_min_setups); the batch owns
 * the masks, travel, classes and per-part scratch (6 + 30 n + T + ~33 KB
 * bytes), which count against its budget with the part's other bytes.
 * Errors: as rc_batch_add_part, RC_E_ARG (NULL face ids). */
rc_status rc_batch_add_analysis(rc_batch b, rc_bvh h, const float* d_P, const float* d_N, const int32_t* d_face,
                                int64_t n, uint32_t* d_bits, int32_t* d_count, int64_t* part_id);

/* Part-level results of the most recent launch for parts [0, n_out): for an
 * analysis part the summary, label, setups (both covers, class counts,
 * mask histogram; setups_ran = 1 for every part, whatever its label) and the
 * cast's and the orthogonal cast's counters, as rc_analyze_part reports
 * them for the same points; a part added with rc_batch_add_part gets zeros
 * (its bits, counts and counters are in its own arrays).  Waits for the
 * launch; reads every analysis part's record in one copy.  Errors: RC_E_ARG
 * (no launch yet, parts or parameters changed since the last launch, n_out
 * outside [0, parts]), RC_E_CUDA. */
rc_status rc_batch_results(rc_batch b, rc_part_result* h_out, int64_t n_out);

/* Remove every part (the batch can then be refilled). */
rc_status rc_batch_clear(rc_batch b);

/* Replace the batch's parameters (the next launch re-captures its graph). */
rc_status rc_batch_set_params(rc_batch b, const rc_params* p);

/* Cast every part of the batch on `stream`: the first launch after a change
 * uploads the part descriptors, computes the parts' point orders and
 * captures [reset counters, batched kernel] as a CUDA graph (on a private
 * stream); every launch replays that graph on `stream`.  Outputs per part are
 * exactly those of rc_hemisphere_cast.  Asynchronous after the first
 * launch.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_batch_launch(rc_batch b, void* stream);

/* *done = 1 once the work of the most recent rc_batch_launch (every part of
 * the batch, part_id included) has completed on the device, 0 while it is
 * still running or before the first launch.  Never blocks.  Errors:
 * RC_E_ARG (part_id outside the batch), RC_E_CUDA (the launch failed). */
rc_status rc_batch_poll(rc_batch b, int64_t part_id, int32_t* done);

/* Autotuner: time the batch under every combination of point order (Morton
 * / index), direction order (tiles / index), resident blocks per SM (4, 6,
 * 8) and points per work item (1, 2, 4), `repeats` graph launches each, on
 * `stream`, and keep the fastest; *best (may be NULL) receives it.  The
 * batch's outputs hold the last timed run.  Synchronises `stream`. */
rc_status rc_batch_autotune(rc_batch b, void* stream, int32_t repeats, rc_params* best);

/* Release a batch (not its parts' handles or arrays). */
rc_status rc_batch_destroy(rc_batch b);

/* The whole pipeline of Sections 3.1-3.3 on HOST arrays, in one call: copy
 * the mesh to the device, build the BVH, sample n points (centroid mode
 * needs n == T), cast n*N hemisphere rays, reduce them to the indicators,
 * classify, and -- for 3-axis parts, or for every part if
 * p->always_setups -- cast the six axes and search the setups; then copy
 * the requested per-point results back.
 *   h_V [nV][3], h_F [T][3] (host; pinned memory makes the copies
 *   asynchronous); outputs h_bits [n][W], h_count [n], h_mask [n],
 *   h_class [n] are host arrays and may each be NULL; h_out receives the
 *   part-level result.
 * Device memory is allocated on `stream` and released before returning.
 * Requested bits and counts are copied back on a second stream of the
 * calling thread while the reduction and the setups run; with
 * p->always_setups the orthogonal cast runs on a third beside the
 * hemispherical cast.  Both join before the call returns.
 * Synchronises `stream`.  Errors: as the individual calls. */
rc_status rc_analyze_part(const float* h_V, int64_t nV, const int32_t* h_F, int64_t T, int64_t n,
                          const rc_params* p, uint32_t* h_bits, int32_t* h_count, uint8_t* h_mask,
                          uint8_t* h_class, rc_part_result* h_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Serving: a persistent request loop for part analyses                   */
/* ---------------------------------------------------------------------- */
/* The paper aims at interactive use inside CAD (Sections 1 and 5).  A
 * server keeps worker slots (one host thread and one CUDA stream each)
 * that take requests as they arrive: a queued request is admitted as soon
 * as a slot is free and its device bytes fit into the budget (idle resident
 * parts are evicted, least recently used first), so requests that arrive
 * while others are on the GPU run concurrently with them.  Each part's BVH,
 * sample points and visibility maps stay resident under the caller's part
 * key; a re-submission with the same triangle list is refitted, otherwise
 * rebuilt.  Each request runs the pipeline of rc_analyze_part.  Every slot has
 * one stream per device priority level and a request runs on the level its
 * size gives it (smaller = higher, see cfg->small_rays), so the blocks of
 * small requests are scheduled ahead of a large request's; with
 * p->launch_mode = 1 the casts use short-lived blocks and concurrent
 * requests interleave on the SMs. */

typedef struct rc_server_s* rc_server;

typedef struct {
    int32_t slots;              /* concurrent requests (1..64) */
    int32_t cast_blocks_per_sm; /* blocks per SM of each request's cast (0 = the params' value) */
    int64_t hbm_budget_bytes;   /* admission budget for resident parts plus running requests */
    int64_t small_rays;         /* requests with at most this many hemisphere rays run at the highest
                                   stream priority, each doubling one level lower (0 = all at the lowest) */
    int32_t incremental;        /* 1: a re-submission with the same triangle list and point count keeps the
                                   part's sample points on their faces (rc_sample_points_on_faces) and casts
                                   again only what the edit can change (rc_changed_faces +
                                   rc_hemisphere_update); its result is the analysis of the edited part at
                                   those points.  0: every request samples afresh */
    int32_t pad;
} rc_server_config;

typedef struct {
    int64_t request_id;
    uint64_t part_key;
    rc_status status;           /* RC_OK, RC_E_OOM (never fits the budget), or the failing call's status */
    int32_t slot;               /* worker slot that ran it */
    int32_t rebuilt;            /* 1 = BVH built, 0 = refitted */
    int32_t priority_level;     /* stream priority level it ran at (0 = highest) */
    int32_t updated;            /* 1 = incremental re-analysis (cfg.incremental), 0 = full analysis */
    int32_t pad;
    double t_submit, t_admit, t_start, t_end;   /* steady-clock seconds */
    int64_t resident_bytes;     /* device bytes the part keeps resident */
    rc_part_result result;
    char message[128];          /* error text when status != RC_OK */
} rc_request_result;

typedef struct {
    int64_t submitted, completed, failed, rejected, evicted;
    int64_t running, queued, resident_parts, used_bytes;
} rc_server_stats;

/* Start a server with parameters *p (copied; p->always_setups applies) on
 * the current device.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_server_create(const rc_params* p, const rc_server_config* cfg, rc_server* out);

/* Queue an analysis of the host mesh (h_V [nV][3], h_F [T][3], copied before
 * returning) with n sample points, under part_key.  Returns at once with
 * *req_id.  Errors: RC_E_ARG. */
rc_status rc_server_submit(rc_server s, uint64_t part_key, const float* h_V, int64_t nV, const int32_t* h_F,
                           int64_t T, int64_t n, int64_t* req_id);

/* Wait up to timeout_s seconds for a request; on completion copy its result
 * to *out and forget the request.  Errors: RC_E_TIMEOUT (still running or
 * queued; the request stays known), RC_E_ARG (unknown id). */
rc_status rc_server_wait(rc_server s, int64_t req_id, double timeout_s, rc_request_result* out);

/* Copy a resident part's visibility bits [n][W], W = ceil(n_dirs / 32),
 * and counts [n] to host arrays (either may be NULL).  bits_words is the
 * capacity of h_bits in uint32 words and must be at least n * W.  A part
 * in use is read once it is idle again (waiting at most 60 s).
 * Errors: RC_E_ARG (not resident, n differs, h_bits too small),
 * RC_E_TIMEOUT, RC_E_CUDA (the copy failed). */
rc_status rc_server_read_bits(rc_server s, uint64_t part_key, uint32_t* h_bits, int64_t bits_words,
                              int32_t* h_count, int64_t n);

/* Counters of the server (host struct). */
rc_status rc_server_get_stats(rc_server s, rc_server_stats* out);

/* Stop the workers after their current requests and free everything. */
rc_status rc_server_destroy(rc_server s);

/* The two setup covers of Section 3.3 from a 64-bin histogram of viable
 * points per reachable-axis mask (bin 0 is ignored): the exact minimum
 * (smallest |S|, ties to the smallest bitmask) and the greedy cover (most
 * uncovered points first, ties to the lower axis).  Fills setups_* and
 * chosen_* of *out; other fields are left unchanged.  Host only, no GPU.
 * Errors: RC_E_ARG (NULL, negative count). */
rc_status rc_setup_cover(const int64_t* h_mask_hist, rc_setups* out);

/* ---------------------------------------------------------------------- */
/* Re-analysis after an edit that keeps the triangle list                 */
/* (interactive design, Sections 1 and 5; not a step of the paper)        */
/* ---------------------------------------------------------------------- */

/* Sample points kept on given faces: point i lies on d_face[i] of the
 * part in h (typically edited since the points were drawn).  Area mode:
 * at (1 - s) A + s (1 - u2) B + s u2 C, s = sqrt(u1), with point i's own
 * counter-based u1, u2 (p->seed) -- on an unedited part exactly the point
 * rc_sample_points drew; centroid mode: at the face centroid.  d_N gets
 * the face normals.  Synchronises `stream`.  Errors: RC_E_ARG (a face id
 * outside [0, T)), RC_E_CUDA. */
rc_status rc_sample_points_on_faces(rc_bvh h, int64_t n, const rc_params* p, const int32_t* d_face, float* d_P,
                                    float* d_N, void* stream);

/* Faces whose vertices moved between d_V_old and d_V_new (bit-for-bit
 * comparison, same triangle list d_F [T][3]): d_changed [T] = 1 / 0,
 * *h_n_changed their number, h_box [6] (lo xyz, hi xyz) the bounding box
 * of their old and new triangles (an empty box, lo > hi, when none moved).
 * Synchronises `stream`.  Errors: RC_E_ARG (a vertex index outside
 * [0, nV)), RC_E_CUDA. */
rc_status rc_changed_faces(const float* d_V_old, const float* d_V_new, int64_t nV, const int32_t* d_F, int64_t T,
                           uint8_t* d_changed, float* h_box, int64_t* h_n_changed, void* stream);

/* Hemispherical cast of the edited part h, re-using the results of the
 * unedited part: d_bits / d_count hold the old results of the same points
 * (rc_sample_points_on_faces) on entry and the new ones on return.  Points
 * on changed faces are cast in full; for the others only rays that can
 * enter h_box (the conservative slab test of the traversal) are cast again,
 * and a point whose tangent plane has the whole box behind it is skipped.
 * The result equals rc_hemisphere_cast of the edited part at these points
 * (rays decided by FP64-ambiguous pairs may differ, as between any two
 * trees).  d_counters int64[4]: rays cast again, ambiguous, FP64
 * re-tests, errors (may be NULL).  Asynchronous.  Errors: RC_E_ARG,
 * RC_E_CUDA. */
rc_status rc_hemisphere_update(rc_bvh h, const float* d_P, const float* d_N, const int32_t* d_face, int64_t n,
                               const uint8_t* d_changed, const float* h_box, const rc_params* p, uint32_t* d_bits,
                               int32_t* d_count, int64_t* d_counters, void* stream);

/* ---------------------------------------------------------------------- */
/* STL import and the paper's face-level analysis                         */
/* ---------------------------------------------------------------------- */

/* Read an STL file (binary, or ASCII "solid ... endsolid") into the mesh
 * layout of rc_build_bvh.  A file is binary when its size is 84 + 50 *
 * (facet count at byte 80); otherwise it must be ASCII.  Facet vertices are
 * taken in stored order (counter-clockwise seen from outside); the stored
 * normal is ignored.  Vertices with identical coordinates (bit for bit, -0
 * read as +0) are merged in order of first appearance.
 *   Size query: h_V = h_F = NULL fills *nV, *T only.
 *   Otherwise h_V [cap_V][3] float32 and h_F [cap_F][3] int32 (host,
 *   caller-owned) receive the mesh if cap_V >= *nV and cap_F >= *T.
 * Host only.  Errors: RC_E_ARG (cannot open, malformed or truncated file,
 * non-finite vertex, arrays too small -- *nV and *T are still set). */
rc_status rc_stl_read(const char* path, float* h_V, int64_t cap_V, int32_t* h_F, int64_t cap_F, int64_t* nV,
                      int64_t* T);

/* The paper's per-part analysis of an STL file (Section 3.1 casts from
 * every face centroid; Sections 3.2-3.3 give the summary of Tables 1-2):
 * rc_stl_read, then rc_analyze_part.  With p->sample_mode ==
 * RC_SAMPLE_FACE_CENTROID the points are the face centroids (n is ignored
 * and set to T) and the overall accessibility is area-weighted; with area
 * sampling n points are drawn.  p->n_dirs may be any value in 1..65536 (the
 * paper uses 150).  Per-point outputs are not returned.  Synchronises
 * `stream`.  Errors: those of rc_stl_read and rc_analyze_part. */
rc_status rc_analyze_stl(const char* path, int64_t n, const rc_params* p, rc_part_result* h_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Automatic machining frame (Section 3.2 assumes the part sits in a      */
/* canonical frame whose axes are the machine axes; how that frame is     */
/* found is not stated -- the definitions below are this library's)       */
/* ---------------------------------------------------------------------- */

#define RC_MAX_FRAMES 6
#define RC_BOX_STEPS 128

/* Candidate sources.  A box-minimising rotation of base b has source
 * RC_FRAME_BOX + b. */
enum { RC_FRAME_GIVEN = 0, RC_FRAME_PRINCIPAL = 1, RC_FRAME_NORMALS = 2, RC_FRAME_BOX = 3 };

/* Candidate frames and, after rc_frame_select, their setups. */
typedef struct {
    int32_t k;                          /* candidates in frame[0 .. k) */
    int32_t best;                       /* rc_frame_select: the chosen candidate; -1 before */
    int32_t source[RC_MAX_FRAMES];      /* RC_FRAME_* */
    int32_t box_axis[RC_MAX_FRAMES];    /* box rotations: the base column held (0..2), else -1 */
    int32_t box_step[RC_MAX_FRAMES];    /* box rotations: j with tan(theta/2) = j / RC_BOX_STEPS, else -1 */
    float frame[RC_MAX_FRAMES][9];      /* row-major 3x3, columns X', Y', Z' (the rc_params.frame layout) */
    double volume[RC_MAX_FRAMES];       /* volume of the vertices' bounding box in the frame (mm^3, FP64) */
    double principal[3];                /* eigenvalues of the surface second moment (mm^4), descending */
    rc_setups setups[RC_MAX_FRAMES];    /* rc_frame_select: per candidate, as rc_min_setups */
} rc_frames;

/* Candidate machining frames of the part, in this order (a candidate whose
 * axes are, up to sign and order, those of an earlier one has the same six
 * machining directions and is dropped):
 *   1. p->frame (RC_FRAME_GIVEN);
 *   2. principal axes (RC_FRAME_PRINCIPAL): eigenvectors of the surface's
 *      area second moment about its area centroid, sum over faces of the
 *      exact triangle integral A/12 (a a^T + b b^T + c c^T + s s^T),
 *      s = a + b + c; X' = largest eigenvalue, Y' = second, Z' = X' x Y';
 *      absent when two adjacent eigenvalues (descending) differ by at most
 *      1e-3 times the largest;
 *   3. dominant normals (RC_FRAME_NORMALS): face normals binned as lines on
 *      a 3 x 32 x 32 cube map, weighted by llround(A / A_max * 2^32); Z' =
 *      normal of the largest face of the heaviest cell, X' = that of the
 *      heaviest cell whose centre w has |w . Z'| <= 0.2 |w|, orthogonalised;
 *   4. after each base frame, its box-minimising rotation (RC_FRAME_BOX +
 *      base): one column held, the other two turned by theta with
 *      tan(theta/2) = j/128, j = 0..127; smallest vertex bounding-box
 *      volume, ties to the lower column, then the lower j.
 * Axes of 2 and 3 are rounded to multiples of 2^-20 per component, signed
 * so the largest component is positive, orthonormalised in FP64 and
 * rounded to fp32; no candidate holds a negative zero.  Fills k, source, box_axis, box_step, frame, volume,
 * principal; best = -1.  Synchronises `stream`.
 * Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_frame_candidates(rc_bvh h, const rc_params* p, rc_frames* out, void* stream);

/* Evaluate io->frame[0 .. io->k) on the part's sample points: orthogonal
 * cast, reachability, fixture faces, classes and both setup covers per
 * frame (the steps of rc_orthogonal_cast and rc_min_setups, all frames in
 * one cast launch), then choose: fewest setups (exact cover), then fewest
 * over-threshold plus inaccessible points, then the smallest bounding-box
 * volume, then the lowest index.  Fills io->setups, io->volume, io->best.
 *   d_P, d_N [n][3], d_face [n] (device, as from rc_sample_points);
 *   d_counters int64[4] (rays, ambiguous, FP64 re-tests, overflow; may be
 *   NULL; 8 entries with node and triangle counts when p->collect_stats is
 *   set).  The frames may come from rc_frame_candidates or the caller.
 * Synchronises `stream`.  Errors: RC_E_ARG (k outside 1..RC_MAX_FRAMES,
 * non-finite frame), RC_E_CUDA. */
rc_status rc_frame_select(rc_bvh h, const float* d_P, const float* d_N, const int32_t* d_face, int64_t n,
                          const rc_params* p, rc_frames* io, int64_t* d_counters, void* stream);

/* ---------------------------------------------------------------------- */
/* Measurement probes (no counterpart in the paper): the ceilings of a    */
/* traversal whose tree stays in L2                                       */
/* ---------------------------------------------------------------------- */

/* Random reads of record_bytes (16, 32, 64 or 128: 128 is the size of a
 * 4-wide node) from an L2-resident buffer of buffer_bytes (a power of two
 * in [1 MiB, 1 GiB]; records picked by splitmix64 of a counter),
 * reads_per_thread records per thread over 8 blocks of 256 threads per SM:
 * *h_gbs receives the read bandwidth in GB/s (one timed launch after a
 * warm-up).  Synchronises `stream`.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_probe_l2(int64_t buffer_bytes, int32_t record_bytes, int32_t reads_per_thread, double* h_gbs,
                      void* stream);

/* FP32 fused multiply-add throughput: eight independent chains of iters
 * FMAs per thread over 8 blocks of 256 threads per SM; *h_tflops receives
 * TFLOP/s (2 per FMA).  Synchronises `stream`.  Errors: RC_E_ARG, RC_E_CUDA. */
rc_status rc_probe_fp32(int32_t iters, double* h_tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RC_H */
