/*
 * hd.h -- C ABI of the GB300 (sm_103a) branch-and-bound for the one-sided
 * Pompeiu-Hausdorff distance between triangle soups,
 *
 *     h(A, B) = max_{p in A} min_{q in B} |p - q|          (Section 3, Eq. hausdorff_distance)
 *
 * after Sacht & Jacobson, "Cascading upper bounds for triangle soup
 * Pompeiu-Hausdorff distance" (SGP 2024).  A call returns l <= h(A,B) <= u with
 * u - l <= eps (Section 3, Eq. output_bounds; the stopping rule of Section 3.1).
 *
 * Conventions for every entry point:
 *   - Meshes are triangle soups: V is row-major nV x 3 (float32 or float64),
 *     F is row-major nF x 3 int32 vertex indices (Section 3, first paragraph).
 *   - Pointers are host or device memory as each argument says; the caller owns
 *     them.  Host arrays are copied before the call returns.  Device arrays must
 *     stay valid until the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Entry points that return results to the host synchronise that stream.
 *   - Every entry point returns an HD_* status code; hd_status_str() names it.
 *     On HD_ERR_INVALID nothing was launched.  On HD_ERR_CUDA the CUDA error
 *     string is available from hd_last_error().
 */
#ifndef HD_H_
#define HD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
  HD_OK = 0,            /* done; the bracket is within tolerance                        */
  HD_ERR_INVALID = 1,   /* bad argument: empty mesh, index out of range, non-finite
                           coordinate, tol <= 0, unknown option                          */
  HD_ERR_CAPACITY = 2,  /* face cap m * n_A (Section 4) or the frontier memory limit was
                           reached; [lower, upper] is still a valid bracket of h           */
  HD_ERR_NUMERIC = 3,   /* every sub-triangle was discarded while u > l: only rounding can
                           do this (Section 5.3, mesh 441717); FP64 mode only              */
  HD_ERR_TIMEOUT = 4,   /* max_rounds reached; [lower, upper] is a valid bracket           */
  HD_ERR_CUDA = 5       /* a CUDA call failed; see hd_last_error()                         */
};

/* vertex element types */
enum { HD_F32 = 0, HD_F64 = 1 };
/* tolerance modes: eps = tol, or eps = tol * (bbox diagonal of A's referenced vertices) */
enum { HD_TOL_ABS = 0, HD_TOL_REL = 1 };
/* arithmetic of the bound and distance computations */
enum {
  HD_FP64 = 0,  /* IEEE double, round-to-nearest, as in the paper (Section 4)              */
  HD_MIXED = 1  /* FP32 with certified (outward-rounded) bounds; FP64 only for sliver
                   triangles of B whose FP32 result cannot be certified tightly            */
};

typedef struct {
  const void* V;     /* nV x 3 vertices, element type vtype                               */
  int64_t nV;
  const int32_t* F;  /* nF x 3 vertex indices                                             */
  int64_t nF;
  int32_t vtype;     /* HD_F32 or HD_F64                                                  */
  int32_t on_device; /* 1: V and F are device pointers on the current device; 0: host    */
} hd_mesh;

typedef struct {
  int32_t tol_mode;        /* HD_TOL_ABS or HD_TOL_REL                                    */
  int32_t precision;       /* HD_FP64 or HD_MIXED                                         */
  double max_face_factor;  /* m of Section 4: at most m * n_A faces are processed
                              (n_A + 4 per split); default 1e7                           */
  int64_t frontier_chunk;  /* most sub-triangles split in one round (0 = automatic)       */
  int32_t leaf_size;       /* triangles per BVH leaf, 1..16 (default 1)                   */
  int32_t block_size;      /* threads per block of the round kernels, a multiple of 32
                              (default 64); above what the kernels' register use allows
                              (a few hundred) hd_hausdorff returns HD_ERR_INVALID       */
  uint8_t bound_order[4];  /* cascade order, values 1..4 = u1..u4 (default 1,2,3,4)        */
  int32_t n_bounds;        /* how many entries of bound_order are used, 1..4 (default 4)  */
  int64_t max_rounds;      /* frontier rounds before HD_ERR_TIMEOUT (default 1e6)         */
  int64_t max_frontier_bytes; /* device memory for frontier + vertex pool (0 = automatic) */
  int32_t flags;           /* HD_FLAG_* bits (default 0)                                  */
  int32_t reserved;        /* must be 0                                                   */
} hd_options;

/* hd_options.flags.  By default the UpperBound of a child sub-triangle is clamped to its
 * parent's: h(child, B) <= h(parent, B) <= U(parent) since the child lies inside the parent.
 * The paper's cascade (Section 4) has no such clamp; HD_FLAG_NO_PARENT_CLAMP turns it off. */
enum {
  HD_FLAG_NO_PARENT_CLAMP = 1,
  HD_FLAG_ASYNC_BUILD = 2,
  HD_FLAG_SHARE_MIDPOINTS = 4,
  HD_FLAG_WELD_B = 8,
  HD_FLAG_NO_SMALL_ROUNDS = 16,
  HD_FLAG_BATCH_STREAMS = 32,
  HD_FLAG_EXACT_QUERIES = 64
};
/* HD_FLAG_EXACT_QUERIES: every vertex query runs until its nearest triangle of B is certain,
 * as in the paper (Section 4).  By default (when u1 is in bound_order) a query stops as soon
 * as it has found a triangle of B within l - e of the vertex, l the running lower bound and e
 * the longest edge of A: u1 then discards every sub-triangle at that vertex whatever its exact
 * distance, so the vertex keeps the triangle found, with a lower bound of 0.  The sub-triangles
 * discarded, the splits, the rounds and the bracket are the same either way (up to the FP32
 * certification width of MIXED distances, which can only make a face survive that exact
 * queries would discard); only the traversal work differs. */
/* HD_FLAG_BATCH_STREAMS (read by hd_hausdorff_batched): run the pairs as independent single
 * runs on host threads with one stream each, instead of the default batched run in which every
 * kernel launch works on the items of all pairs. */
/* HD_FLAG_NO_SMALL_ROUNDS: every frontier round runs as a sequence of grid-wide kernels.  By
 * default, rounds over a frontier of at most 64 items (the last rounds of most runs) run
 * inside one single-block kernel that loops over them without the host; the results are the
 * same either way. */
/* HD_FLAG_WELD_B (read by hd_build_B, for the mesh it builds a BVH of; for
 * hd_hausdorff_sym give it when building A's BVH too): vertices at exactly the same
 * position get one id before the adjacency
 * test of u3 (Section 3.2, Kang's case 1: two triangles of B sharing an edge), so a soup
 * (every triangle with its own three vertices) is treated like the indexed mesh it came
 * from.  Positions are compared exactly (-0 equals +0); the coordinates and the distances
 * are unchanged. */
/* HD_FLAG_SHARE_MIDPOINTS: an edge split by two sub-triangles in the same round gets one
 * midpoint vertex (and one nearest query) instead of two, through a per-round hash table of
 * split edges.  Results are the same up to the order of floating-point maxima; it pays where
 * neighbouring sub-triangles split together (deep refinement), and costs a little where
 * splits are sparse.  The table also caps the splits per round at about the faces of A. */
/* HD_FLAG_ASYNC_BUILD (read by hd_build_B): return as soon as the build is queued on the
 * stream, without waiting for it.  B's validity (indices in range, finite coordinates) is
 * then known only on the device: hd_hausdorff and its variants check it with their first
 * read-back and return HD_ERR_INVALID for an invalid B; hd_nearest, hd_nearest_noalloc and
 * hd_upper_bounds give undefined values (but stay in bounds) on such a BVH. */

typedef struct {
  int64_t rounds;            /* frontier rounds after round 0                              */
  int64_t splits;            /* sub-triangles split 1->4 (Section 4's B&B iterations)      */
  int64_t queries;           /* nearest-triangle queries (vertices of A and midpoints)     */
  int64_t pointtri_evals;    /* point-triangle distance evaluations (leaf tests + u3)      */
  int64_t leaf_tests;        /* ... of which in the BVH traversal (leaf triangles tested)  */
  int64_t box_tests;         /* BVH child-box distance evaluations (one per non-empty child
                                of each node visited, so up to 4 per node)                 */
  int64_t discards[6];       /* sub-triangles discarded, by the deciding bound: exact, u1,
                                u2, u3, u4; [5] = discarded later because l grew past U    */
  int64_t retired;           /* sub-triangles kept but never split again: l <= U <= l + eps */
  int64_t fp64_escalations;  /* MIXED: point-triangle tests redone in FP64 (slivers whose
                                FP32 certificate was loose)                                 */
  int64_t peak_frontier;     /* largest live frontier                                       */
  int64_t pool_vertices;     /* vertices of A + midpoints made (an edge split by two
                                sub-triangles in one round gets one midpoint)             */
  double eps_abs;            /* absolute tolerance used                                     */
  double dA;                 /* bbox diagonal of A's referenced vertices                    */
  int64_t long_queries;      /* queries whose traversal a whole warp finished (part of
                                queries: those with many BVH boxes within their distance)  */
  int64_t kernel_launches;   /* GPU kernels the call launched                               */
  int64_t d2h_bytes;         /* bytes the call read back from the device (run-state
                                snapshots of its rounds)                                    */
  int64_t promoted;          /* MIXED: sub-triangles whose gap U - l fell within the FP32 error
                                width of their vertex distances, so they were finished in the
                                FP64 certification phase (Section 5.3's rounding limit)    */
  int64_t node_visits;       /* BVH nodes (128 bytes each) fetched by the traversals        */
  int64_t long_node_visits;  /* ... of which by the warp-cooperative traversal of long queries */
  int64_t long_leaf_tests;   /* leaf tests of the warp-cooperative traversal (part of
                                leaf_tests)                                                  */
  int64_t queries_cut;       /* queries stopped before the nearest triangle was certain,
                                once the triangle found was close enough that bound u1
                                (Eq. u1) discards every face at the vertex (part of queries;
                                0 with HD_FLAG_EXACT_QUERIES)                               */
} hd_stats;

typedef struct {
  double lower, upper; /* l <= h(A,B) <= u (valid on HD_OK, HD_ERR_CAPACITY, HD_ERR_TIMEOUT) */
  int32_t status;
  hd_stats stats;
} hd_result;

/* Opaque: B, its bounding-volume hierarchy and per-triangle data, on one device. */
typedef struct hd_bvh hd_bvh;

/* Fill *opt with the defaults listed above. */
void hd_options_default(hd_options* opt);

/* Build the BVH of B (Section 4: an AABB hierarchy over B, built once and used for the
 * distances D, nearest triangles I and closest points C of points of A).  GPU build:
 * Morton codes of the triangle centroids, radix sort, binary radix tree (Karras 2012),
 * bottom-up boxes rounded outward, leaves of up to opt->leaf_size triangles.
 * B may have at most 2^27 - 1 triangles.  On HD_OK *out owns device memory until
 * hd_free_B(*out).  opt may be NULL. */
int hd_build_B(const hd_mesh* B, const hd_options* opt, void* stream, hd_bvh** out);

/* Release everything hd_build_B allocated.  NULL is allowed.  The device memory goes
 * back to the device's stream-ordered pool in stream order on the legacy default stream,
 * so it follows earlier work on blocking streams; work that reads the BVH on a stream
 * created non-blocking (hd_nearest, hd_nearest_noalloc, hd_upper_bounds are asynchronous)
 * must be synchronized before this call.  hd_hausdorff returns after its work is done. */
void hd_free_B(hd_bvh* bvh);

/* Triangle count of B and whether its vertices were given as float64. */
int64_t hd_bvh_num_faces(const hd_bvh* bvh);

/* One-sided h(A, B) to tolerance tol (Sections 3.1 and 4): returns [lower, upper] in
 * *out.  A is read according to A->on_device.  The frontier-parallel rounds run on the
 * GPU (nearest queries through the BVH, atomic lower bound, the exact case and the
 * u1..u4 cascade, compaction and 1->4 split); only the final bracket and statistics
 * come back to the host.  opt may be NULL (defaults).  Host arrays of A (on_device = 0) are
 * copied on an upload stream of the library's own that does not wait for work queued earlier
 * on `stream` (so the copy overlaps, say, B's asynchronous build); `stream` waits for the
 * copy.  They must therefore hold their values when the call is made. */
int hd_hausdorff(const hd_bvh* B, const hd_mesh* A, double tol, const hd_options* opt, void* stream,
                 hd_result* out);

/* hd_hausdorff with l starting at l0 >= 0, a lower bound already known for the quantity
 * being bracketed (Section 3.1 starts l at the largest vertex distance; a larger known value
 * lets sub-triangles bounded below it go at once).  *out then brackets max(l0, h(A, B)),
 * which is h(A, B) whenever l0 <= h(A, B).  Used for the two-sided distance and for A's
 * faces split over several GPUs, whose ranks share the largest vertex distance. */
int hd_hausdorff_from(const hd_bvh* B, const hd_mesh* A, double tol, double l0, const hd_options* opt,
                      void* stream, hd_result* out);

/* Two-sided H(A, B) = max(h(A, B), h(B, A)) (Section 6, conclusion and future work):
 * h(A, B) as hd_hausdorff (bvhB is B's BVH), then h(B, A) through A's BVH (bvhA) at the
 * same absolute tolerance, with l starting from h(A, B)'s final lower bound, as the paper
 * suggests: sub-triangles of B bounded below that value are discarded at once.  *out gets
 * the bracket of H (lower = max of the lowers, upper = max of the uppers) and the summed
 * statistics; ab and ba (either may be NULL) get the two runs.  ba brackets
 * max(l_AB, h(B, A)), which is all H needs; it is not h(B, A) itself when h(B, A) is the
 * smaller side.  tol follows opt->tol_mode for the first run (HD_TOL_REL: tol times A's
 * bbox diagonal).  Returns the first error of the two runs. */
int hd_hausdorff_sym(const hd_bvh* bvhB, const hd_mesh* A, const hd_bvh* bvhA, const hd_mesh* B, double tol,
                     const hd_options* opt, void* stream, hd_result* out, hd_result* ab, hd_result* ba);

/* npairs independent problems h(As[i], Bs[i]) with one tolerance and one option set;
 * outs[i] receives each result (Sections 3.1 and 4 for every pair).  By default the pairs run
 * together on `stream` in one batched branch and bound: every kernel launch of a round (the
 * nearest queries, the bounds, the selection and split) takes its work from a device-side
 * queue holding the items of all pairs, each pair keeps its own l, u, tolerance and status on
 * the device and retires on its own gap, and the host reads one small snapshot per round for
 * the whole batch.  Each pair's bracket has the meaning of its single run's; kernel_launches and
 * d2h_bytes of every result are the batch's totals.  All pairs' frontiers and sub-triangle
 * vertices share buffers sized from the batch (up to half the free device memory unless
 * opt->max_frontier_bytes is set); pairs still running when those run out are finished
 * afterwards as single runs, as with HD_FLAG_BATCH_STREAMS.  With HD_FLAG_BATCH_STREAMS (or
 * HD_FLAG_SHARE_MIDPOINTS, which the batched run does not implement), host threads (two per
 * host core, 8 to 64), each with its own non-blocking stream, take the pairs in turn as single
 * runs; they start after the work already queued on `stream`.  Every pair is complete when the
 * call returns.  All Bs[i] must live on the current device.  Returns HD_ERR_INVALID when the
 * arguments are invalid (checked before anything is launched) or a pair's mesh is found
 * invalid on the device, HD_ERR_CUDA on a CUDA failure, else HD_OK; per-pair
 * CAPACITY/TIMEOUT/NUMERIC are reported in outs[i].status. */
int hd_hausdorff_batched(const hd_bvh* const* Bs, const hd_mesh* As, int64_t npairs, double tol,
                         const hd_options* opt, void* stream, hd_result* outs);

/* Batched nearest-triangle queries (the D, I, C of Section 4) for n points:
 * P (device, n x 3, element type ptype) -> dist (device, n doubles), idx (device, n
 * int32: row of F_B), foot (device, n x 3 doubles: the closest point).  precision
 * HD_FP64 computes in double; HD_MIXED returns a certified bracket instead:
 * dist = an upper bound of d(p, B) realised by triangle idx, foot its closest point,
 * and, if dist_lo is not NULL, dist_lo (device, n doubles) a lower bound of d(p, B).
 * Asynchronous on `stream`. */
int hd_nearest(const hd_bvh* B, const void* P, int32_t ptype, int64_t n, int32_t precision, void* stream,
               double* dist, int32_t* idx, double* foot, double* dist_lo);

/* Largest n accepted by hd_nearest_noalloc. */
#define HD_NOALLOC_MAX_POINTS 65536

/* The same queries as hd_nearest (same arguments, same results), for callers that cannot
 * let a library allocate device memory during the call: programs whose device memory is all
 * handed to their own allocator, services held to a fixed device-memory budget, loops that
 * must not wait in the driver for an allocation.  The paper has no counterpart; this is an
 * interface variant.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch is a fixed
 * array of 4 MiB + 512 B in the library's device image, which every GPU that loads the
 * library keeps until the process exits.  n may be at most HD_NOALLOC_MAX_POINTS (65,536);
 * larger n returns HD_ERR_INVALID without launching anything.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current, so
 * make the first call on a device before any stream capture.  The address is kept until the
 * process exits: do not call this entry point on a device after a cudaDeviceReset of it (the
 * reset destroys the array the address points to).  All calls share the array:
 * calls that overlap on the GPU (different streams or threads without ordering) race and
 * must be serialised by the caller.  Asynchronous on `stream`. */
int hd_nearest_noalloc(const hd_bvh* B, const void* P, int32_t ptype, int64_t n, int32_t precision, void* stream,
                       double* dist, int32_t* idx, double* foot, double* dist_lo);

/* UpperBound(T, l) of Section 4 for n triangles given by their vertices and the
 * vertices' nearest-triangle data (as returned by hd_nearest in HD_FP64):
 * T (device, n x 9 doubles: v1, v2, v3), Td (n x 3), TI (n x 3 int32), Tq (n x 9),
 * all device memory.  Writes U (n doubles) and code (n int32: 0 exact case,
 * 1..4 the bound that discarded T (U < l), 5 kept: U = min of the computed bounds).
 * opt->precision HD_FP64 (the default): FP64 arithmetic.  HD_MIXED: the certified FP32
 * arithmetic of the rounds (each vertex as a float pair, its distance rounded up, its closest
 * point as a float offset with the offset's rounding as error radius; u4 evaluated in place),
 * so U bounds h(T, B) from above whenever Td and Tq are exact.  Asynchronous on `stream`. */
int hd_upper_bounds(const hd_bvh* B, const double* T, const double* Td, const int32_t* TI, const double* Tq,
                    int64_t n, double l, const hd_options* opt, void* stream, double* U, int32_t* code);

/* Kernel timing trace.  While enabled (process-wide), the library records a CUDA event
 * pair on the launching stream around each of its kernels and accumulates, per kind,
 * the number of launches and their total device time in milliseconds.  Each pair costs a
 * few microseconds of host time.  Kinds: the whole BVH build of one hd_build_B call
 * (counted as one launch), the nearest-triangle lane traversal (k_query), UpperBound of
 * faces and children, select/split/compaction, validation/pool set-up, the single-block
 * kernel that runs whole rounds over small frontiers, and the warp-cooperative traversal of
 * long queries (k_query_long). */
enum { HD_K_BUILD = 0, HD_K_QUERY = 1, HD_K_BOUND = 2, HD_K_SELECT = 3, HD_K_PREP = 4, HD_K_SMALL = 5, HD_K_LONG = 6,
       HD_K_KINDS = 7 };
typedef struct {
  int64_t launches[8];
  double ms[8];
} hd_trace;

/* Turn the trace on (1) or off (0). */
void hd_trace_enable(int on);

/* Copy the accumulated trace into *out (waits for the recorded events); reset != 0
 * clears it afterwards. */
int hd_trace_read(hd_trace* out, int reset);

/* Name of a status code (static string). */
const char* hd_status_str(int status);

/* Text of the last HD_ERR_CUDA on this thread (static buffer, "" if none). */
const char* hd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HD_H_ */
