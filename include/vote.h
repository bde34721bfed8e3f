/*
 * vote.h -- C ABI of the GB300 general-voting library (libvote.so).
 *
 * General voting (Aiger, Lynen, Hosang, Zeisl, arXiv 2107.11810) finds a point of
 * approximately maximal depth among n k-surfaces in R^d: the point that lies
 * within eps (per dependent coordinate, vertical distance) of the most surfaces.
 * Each surface has the parametric form of Sec. 3, Eq. 1:
 *     x_j = F_j(x_1..x_k; t) + f_j,   j = k+1..d,
 * with t the essential and f the free additive parameters.  The search is
 * Algorithm 2 (SurfaceConsensus) with canonization (Sec. 3.2) and bound-based
 * pruning (Sec. 3.3): level by level, the surfaces reaching a cell are rounded to
 * a grid tied to the cell size, identical rounded surfaces are merged, every
 * child cell is tested against every surface for proximity within eps plus the
 * cell radius (the "subset of the conditions" surface-box test of Sec. 3.2),
 * cells whose upper bound is below the best lower bound are dropped, and the
 * rest split 2^d ways.  Leaves are cells no wider than eps in any coordinate.
 *
 * Conventions for every entry point:
 *   - Return value: VOTE_OK or an error code; vote_last_error() gives a message
 *     (thread-local).  No exception crosses the ABI and no kernel traps.  On
 *     error the outputs are unspecified and the context stays usable.
 *   - Ownership: the caller owns every input/output buffer.  The context owns
 *     its device working memory (grown on demand, reused, freed by
 *     vote_destroy).
 *   - Threads: one context per host thread; calls on one context are serial.
 *   - Work runs on the context's CUDA stream (vote_set_stream; default: the
 *     legacy default stream).  Entry points that return host results
 *     synchronise that stream before returning.
 *   - Results are fully determined by the inputs (not by scheduling or GPU
 *     work order): counts, depth, leaf and mask are bit-identical to the FP64
 *     definition for both precision modes.
 */
#ifndef GV_VOTE_H
#define GV_VOTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vote_ctx vote_ctx;

typedef enum {
    VOTE_OK = 0,
    VOTE_EINVAL = 1,       /* bad argument, non-finite input, value out of range    */
    VOTE_ENOMEM = 2,       /* device or host allocation failed                       */
    VOTE_ECUDA = 3,        /* a CUDA runtime call failed                             */
    VOTE_ECAPACITY = 4,    /* a fixed-size buffer (trace) or key width was exceeded  */
    VOTE_ETIMEOUT = 5,     /* a bounded device-side wait ran out                     */
    VOTE_EUNSUPPORTED = 6, /* family / size combination not supported                */
    VOTE_EINTERNAL = 7     /* a self-check failed (e.g. popcount(mask) != depth)     */
} vote_status;

/* Surface families.  Coordinates are ordered free first, then dependent.
 *   VOTE_LINE2D      d=2 k=1: coords (m, b); input rows (x, y) of image points;
 *                    surface b = y - x m (point-line duality, Sec. 3, Eq. 2).
 *   VOTE_PLANE3D_SPH d=3 k=2: coords (theta, phi, d); input rows (qx, qy, qz);
 *                    surface d = q . (sin th cos ph, sin th sin ph, cos th)
 *                    (hyperplane fitting of Sec. 4.1 in spherical form).
 *   VOTE_POSE3DOF    d=3 k=1: coords (yaw, x, y); input rows (w1, w2, a, b);
 *                    surfaces x = w1 - (a cos yaw - b sin yaw),
 *                    y = w2 - (a sin yaw + b cos yaw) (camera posing with known
 *                    gravity, focal length and height; the 3DoF reduction of
 *                    the Sec. 4.2.1 formulation).
 *   VOTE_POSE6DOF    d=6 k=4: coords (phi1, phi2, phi3, z, x, y), phi the
 *                    axis-angle vector of the rotation and (x, y, z) the
 *                    translation of the camera frame X = R(phi) w + (x, y, z);
 *                    input rows (w1, w2, w3, xi, eta) of a match between world
 *                    point w and normalized image point (xi, eta); surfaces
 *                    x = xi (r3 . w + z) - r1 . w, y = eta (r3 . w + z) - r2 . w
 *                    (calibrated camera, Sec. 4.2.3: Sec. 4.2.2 with f = 1).
 *                    The tolerance of x and y is a constant vertical distance;
 *                    cells split into 64 children.
 *   VOTE_RAYS3D      d=3 k=1: coords (x, y, z); input rows (a, b, c, d) of the
 *                    ray y = a x + b, z = c x + d (intersection of rays in
 *                    3-space, Sec. 4.3).
 *   VOTE_POINTSET2D  d=4 k=2: coords (c, d, a, b); input rows (px, py, qx, qy) of a
 *                    hypothetical correspondence p -> q under q_x = a p_x + b p_y
 *                    + c, q_y = -b p_x + a p_y + d (point-set similarity
 *                    alignment, Sec. 4.4); surfaces a = (p . (q - (c, d)))/|p|^2,
 *                    b = (p_y (q_x - c) - p_x (q_y - d))/|p|^2; 16 children.
 *   VOTE_AFFINE4D    d=4 k=3: coords (a1, a2, a3, b); input rows (x1, x2, x3, x4)
 *                    of points of 4-space; surface b = x4 - (a1 x1 + a2 x2 + a3 x3)
 *                    (hyperplane fitting in the affine form, Sec. 4.1);
 *                    16 children.
 *   VOTE_RADIAL5DOF  d=5 k=4: coords (phi1, phi2, phi3, y, x) of the radial camera
 *                    with rows (r1, -y) and (r2, x) (unknown focal length,
 *                    Sec. 4.2.4); input rows (w1, w2, w3, xi, eta) as for 6DoF
 *                    (xi != 0); surface x = eta (r1 . w - y) / xi - r2 . w; the
 *                    tolerance of x is a constant distance; 32 children. */
typedef enum {
    VOTE_LINE2D = 1,
    VOTE_PLANE3D_SPH = 2,
    VOTE_POSE3DOF = 3,
    VOTE_POSE6DOF = 4,
    VOTE_RAYS3D = 5,
    VOTE_POINTSET2D = 6,
    VOTE_AFFINE4D = 7,
    VOTE_RADIAL5DOF = 8
} vote_family;

/* Options for vote_set_option. */
typedef enum {
    VOTE_OPT_PRECISION = 1,   /* 0 = plain FP64 predicate; 1 = FP32 screen with FP64
                                 recheck of the borderline band (default 1)          */
    VOTE_OPT_PRUNE = 2,       /* 1 = prune cells with UB < best LB (default); 0 = off */
    VOTE_OPT_CHUNK_RECORDS = 3, /* records processed per expansion step; default 2^27
                                 for planes (their pruning hardly depends on the
                                 step size, so larger steps only save per-step
                                 overhead), 2^25 for the other families with d = 2
                                 or 3 (finer depth-first steps keep their pruning
                                 effective), 2^23 for d = 4 or 5 and 2^21 for d = 6
                                 (a step's children can hold 2^d times its records) */
    VOTE_OPT_TRACE_CAP = 4,   /* >0: record (level, coords, UB, LB) of every tested
                                 child, up to this many entries (debug; default 0)   */
    VOTE_OPT_GROUP = 5,       /* merging of identical canonical surfaces:
                                 0 = off, 1 = on (default 0; results do not depend
                                 on it)                                             */
    VOTE_OPT_FAULT_ALLOC_AT = 6, /* test hook: fail the k-th device allocation with
                                 VOTE_ENOMEM (0 = off)                               */
    VOTE_OPT_INITIAL_LB = 7,  /* a known lower bound on the best depth (warm start of
                                 the B&B bound, e.g. from a previous frame); must not
                                 exceed the true maximum depth; default 0            */
    VOTE_OPT_KERNEL_TIMING = 8, /* 1 = time each kernel class with CUDA events on the
                                 context's stream (see vote_get_kernel_times)        */
    VOTE_OPT_BATCH_WORKERS = 10, /* host workers (streams) of vote_solve_batched, 1..32,
                                 default 4                                           */
    VOTE_OPT_DIVE = 11,       /* 1: before the sweep, expand one root-to-leaf path
                                 that always takes the child with the largest UB, so
                                 pruning starts from a leaf's count; 0: off; 2
                                 (default): on for n >= 131072 surfaces.  Results do
                                 not depend on it (Sec. 3.3: any valid bound may
                                 prune)                                              */
    VOTE_OPT_SPIN_LIMIT = 12, /* polls of a bounded device-side wait (the proximity
                                 passes' wait for their bulk copies) before the kernel
                                 gives up and the solve returns VOTE_ETIMEOUT;
                                 default 4194304; 0 gives up at once (test hook)     */
} vote_option;

/* Kernel classes reported by vote_get_kernel_times. */
enum {
    VOTE_K_LIFT = 0, VOTE_K_CELL_GEO = 1, VOTE_K_TEST_COUNT = 2, VOTE_K_TEST_EMIT = 3,
    VOTE_K_CHILDREN = 4, VOTE_K_REPLAY = 5, VOTE_K_GROUP = 6, VOTE_K_CLASSES = 8
};

/* Per-solve counters (vote_get_stats). */
typedef struct {
    int64_t levels;          /* L                                                 */
    int64_t cells;           /* cells expanded (canonized and tested)            */
    int64_t records;         /* (cell, canonical surface) records tested          */
    int64_t tests;           /* (child cell, canonical surface) predicate calls   */
    int64_t rechecks;        /* tests re-evaluated in FP64 because the FP32 screen
                                could not decide them (whole records: every child
                                of a record with one uncertain test), plus child
                                snaps taken in FP64                               */
    int64_t chunks;          /* expansion steps                                   */
    int64_t leaves;          /* leaves evaluated                                  */
    int64_t peak_records;    /* largest record count held at one level            */
    int64_t launches;        /* kernels launched                                  */
    double  seconds;         /* wall time of the last solve                       */
} vote_stats;

/* Create a context for one surface family.
 *   eps[d]      > 0: per-coordinate eps; for dependent coordinates it is the
 *               inlier tolerance (Sec. 3.2 uses a different eps per coordinate),
 *               for every coordinate the leaf width.
 *   bounds[2d]  lo0, hi0, lo1, hi1, ...: the voting domain (Sec. 3 scales it to
 *               the unit cube; here each coordinate keeps its own range).
 * d and k must match the family (LINE2D 2/1, PLANE3D_SPH 3/2, POSE3DOF 3/1). */
vote_status vote_create(int family, int d, int k, const double *eps, const double *bounds,
                        vote_ctx **out);

/* Set an option (see vote_option).  Returns VOTE_EINVAL for unknown keys or
 * out-of-range values. */
vote_status vote_set_option(vote_ctx *ctx, int key, double value);

/* Use this CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all work of the context. */
vote_status vote_set_stream(vote_ctx *ctx, void *cuda_stream);

/* Solve one problem whose surfaces are already on the device.
 *   surfaces     device pointer, FP64, structure of arrays [P][n] (P = 2, 3, 4
 *                rows for LINE2D, PLANE3D_SPH, POSE3DOF); not modified.
 *   n            number of surfaces, >= 0.
 *   best_point   host [d]: centre of the best leaf (Algorithm 2 returns B_c).
 *   best_leaf    host [d] or NULL: integer coordinates of the best leaf.
 *   depth        host: number of surfaces reaching the best leaf (its upper bound).
 *   inlier_mask  device [(n+31)/32] uint32 or NULL: bit i set iff surface i
 *                reaches the best leaf (merges are tracked, Sec. 3.2); the
 *                popcount equals depth.
 * Ties between leaves of equal depth go to the lexicographically smallest leaf
 * coordinates.  n = 0 gives depth 0 and leaf (0, .., 0). */
vote_status vote_solve(vote_ctx *ctx, const double *surfaces, int64_t n, double *best_point,
                       int64_t *best_leaf, int64_t *depth, uint32_t *inlier_mask);

/* Same as vote_solve with HOST buffers: surfaces host [P][n], inlier_mask host
 * [(n+31)/32] or NULL.  Copies in and out through the context's stream. */
vote_status vote_solve_host(vote_ctx *ctx, const double *surfaces, int64_t n, double *best_point,
                            int64_t *best_leaf, int64_t *depth, uint32_t *inlier_mask);

/* Solve B independent problems of this context's family, eps and bounds.
 *   surfaces    device: problem b's surfaces are the FP64 structure-of-arrays
 *               block [P][n_b] starting at element P * offsets[b];
 *   offsets     host [B+1], offsets[0] = 0, n_b = offsets[b+1] - offsets[b];
 *   best_points host [B*d];  best_leaves host [B*d] or NULL;  depths host [B];
 *   masks       device or NULL: problem b's mask words start at word
 *               sum_{b'<b} ceil(n_b'/32);
 *   latency_ms  host [B] or NULL: completion time of each problem, in ms from
 *               the start of the call.
 * Problems are taken from a shared queue by VOTE_OPT_BATCH_WORKERS host workers,
 * each with its own stream and working memory, so small problems overlap on the
 * GPU.  Each problem's results equal those of vote_solve on it alone. */
vote_status vote_solve_batched(vote_ctx *ctx, const double *surfaces, const int64_t *offsets, int B,
                               double *best_points, int64_t *best_leaves, int64_t *depths, uint32_t *masks,
                               double *latency_ms);

/* Upper and lower bound of one cell, by replaying every surface from the root
 * along the path to the cell (the counts Algorithm 2 assigns to that cell,
 * independent of pruning).
 *   surfaces  device [P][n];  level in [0, L];  coords host [d], coordinate j in
 *             [0, 2^min(level, L_j));  ub, lb host;  reach device
 *             [(n+31)/32] or NULL (bit set per surface reaching the cell). */
vote_status vote_cell_counts(vote_ctx *ctx, const double *surfaces, int64_t n, int level,
                             const int64_t *coords, int64_t *ub, int64_t *lb, uint32_t *reach);

/* Soft inlier score used to refine the voting result (not part of the paper's
 * voting itself; Sec. 4.2 hands the approximate pose to "a more accurate
 * method"):
 *     S(p) = sum_i w_i exp(-u_i^2 / 2),   u_i^2 = sum_j (r_ij / tol_j)^2,
 * r_ij the vertical residual of surface i at point p in dependent coordinate j
 * (Eq. 1, global form), w_i = bit i of mask (NULL: all ones).
 *   surfaces  device [P][n];  mask device [(n+31)/32] or NULL;  point device [d];
 *   tol       host [d-k] or NULL (= eps of the dependent coordinates);
 *   score     device [1] (forward).
 * Backward: grad_score device [1] (upstream gradient); grad_point device [d] or
 * NULL receives grad_score * dS/dp; grad_surfaces device [P][n] or NULL receives
 * grad_score * dS/d(surface parameters).  Residuals are recomputed, not stored.
 * Reductions are deterministic (fixed grid, ordered final sum). */
vote_status vote_softscore_fwd(vote_ctx *ctx, const double *surfaces, int64_t n, const uint32_t *mask,
                               const double *point, const double *tol, double *score);
vote_status vote_softscore_bwd(vote_ctx *ctx, const double *surfaces, int64_t n, const uint32_t *mask,
                               const double *point, const double *tol, const double *grad_score,
                               double *grad_point, double *grad_surfaces);

/* Projected gradient ascent of S inside the box [cell_lo, cell_hi] (host [d]),
 * preconditioned by the squared box widths, with Armijo backtracking, at most
 * iters steps.  point_inout host [d] (start, clamped into the box; result);
 * score_out host or NULL: S at the result.  mask/tol as for vote_softscore_fwd. */
vote_status vote_refine(vote_ctx *ctx, const double *surfaces, int64_t n, const uint32_t *mask,
                        const double *cell_lo, const double *cell_hi, const double *tol, int iters,
                        double *point_inout, double *score_out);

/* Bounds of a leaf cell: lo[j] = lo_j + leaf[j] * w_j, hi[j] = lo[j] + w_j with w_j the
 * leaf width in coordinate j (W_j 2^-L_j).  leaf host [d] (integer leaf coordinates, as
 * vote_solve returns them), lo and hi host [d].  VOTE_EINVAL if a coordinate is out of
 * range. */
vote_status vote_leaf_box(vote_ctx *ctx, const int64_t *leaf, double *lo, double *hi);

/* Number of levels L and per-coordinate split counts L_j (host [d]). */
vote_status vote_levels(vote_ctx *ctx, int *L, int *Lj);

/* The level structure of a problem, without a context or a device (host code only):
 * the canonization's snap steps and accumulated error bound (Sec. 3.2,
 * "Canonization" and the eps update).  family, d, k, eps[d], bounds[2d] as for
 * vote_create.  Out (host; any of Lj, s_f, s_t, A may be NULL): *L levels; Lj [d]
 * splits per coordinate; s_f [d-k] snap step of the dependent residuals; s_t
 * [L * le] snap step of essential parameter m at level l (index l * le + m, le the
 * family's essential-parameter count); A [L * (d-k)] accumulated canonization error
 * bound after the snap at level l (A_{l+1}; index l * (d-k) + j).  L is at most 31,
 * so arrays of 31 levels always suffice.  VOTE_EINVAL / VOTE_EUNSUPPORTED as for
 * vote_create. */
vote_status vote_level_constants(int family, int d, int k, const double *eps, const double *bounds, int *L,
                                 int *Lj, double *s_f, double *s_t, double *A);

/* Debug trace of the last solve (needs VOTE_OPT_TRACE_CAP > 0): host arrays of
 * capacity cap; level[i], coords[i*d + j], ub[i], lb[i]; *count = entries
 * written.  Returns VOTE_ECAPACITY if the trace overflowed. */
vote_status vote_get_trace(vote_ctx *ctx, int64_t cap, int32_t *level, int64_t *coords,
                           int64_t *ub, int64_t *lb, int64_t *count);

/* Counters of the last solve; after vote_solve_batched, totals over the whole
 * batch (levels and peak_records: the largest over its problems). */
vote_status vote_get_stats(vote_ctx *ctx, vote_stats *out);

/* Per kernel class (VOTE_K_*): summed device milliseconds, launches and
 * algorithmic bytes (records read/written, as defined per class) of the last
 * solve, measured with CUDA events when VOTE_OPT_KERNEL_TIMING is 1.  Arrays of
 * VOTE_K_CLASSES entries (host). */
vote_status vote_get_kernel_times(vote_ctx *ctx, double *ms, int64_t *launches, double *bytes);

/* Per-level work of the last solve, for l in [0, L) (host arrays of at least L
 * entries, each may be NULL): cells[l] expanded and record slots[l] tested at
 * level l; with VOTE_OPT_GROUP on, grouped_in[l] records entered the grouping of
 * level l (the canonization's merge of equal canonical surfaces, Sec. 3.2) and
 * grouped_out[l] canonical records left it (both 0 with grouping off), so
 * 1 - grouped_out/grouped_in is the level's merge fraction. */
vote_status vote_get_level_stats(vote_ctx *ctx, int64_t *cells, int64_t *records, int64_t *grouped_in,
                                 int64_t *grouped_out);

/* UB and LB of one cell, like vote_cell_counts, for callers that cannot allocate
 * device memory: code running where cudaMalloc is not allowed or not wanted (a
 * host that pre-plans all GPU memory, a real-time loop with a fixed memory
 * budget, a plugin inside another framework's allocator).  There is no
 * counterpart in the paper; it exists for such callers.
 *
 * It needs no context and allocates nothing: its scratch (level constants, the
 * root-to-cell path geometry and two counters, VOTE_NOALLOC_SCRATCH_BYTES in all)
 * is one file-scope __device__ array of the library, which every GPU that loads
 * the library holds until the process exits.  The caller passes the inputs and
 * outputs exactly as for vote_cell_counts, plus the CUDA stream to use (NULL:
 * legacy default stream).
 *   family, d, k, eps[d], bounds[2d]   as for vote_create;
 *   surfaces, n, level, coords, ub, lb, reach   as for vote_cell_counts.
 * Problems with more levels than the array holds (L > 31) return
 * VOTE_EUNSUPPORTED.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress).  Every call copies between host and device
 * memory and synchronises the stream, so no call may be made while the stream is
 * being captured into a CUDA graph.  All calls share the array and it keeps the last call's contents (the counters
 * are cleared at the start of each call): calls that may overlap on the GPU (on
 * different streams or host threads) race and must be serialised by the caller.
 * The call synchronises the stream before returning. */
#define VOTE_NOALLOC_SCRATCH_BYTES 65536
vote_status vote_cell_counts_noalloc(int family, int d, int k, const double *eps, const double *bounds,
                                     const double *surfaces, int64_t n, int level, const int64_t *coords,
                                     int64_t *ub, int64_t *lb, uint32_t *reach, void *cuda_stream);

/* Message for the last error on this host thread (static storage). */
const char *vote_last_error(void);

/* Free the context and all device memory it owns.  NULL is ignored. */
void vote_destroy(vote_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GV_VOTE_H */
