/*
 * fmm.h -- C ABI of the B300 (sm_103a) black-box FMM library libfmm_b300.so.
 *
 * The library evaluates, for N charged particles x_i with charges q_i, the
 * pairwise sums of the paper's eq. 1 with the Laplace kernels of eq. 2
 * (Agullo et al., "Pipelining the Fast Multipole Method over a Runtime
 * System", 2012, Sec. 2 and Sec. 2.1):
 *
 *     phi_i = sum_{j != i} q_j / |x_i - x_j|
 *     F_i   = sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3      (= -grad phi_i)
 *
 * by the black-box FMM of Sec. 2.1: an octree of `height` levels (0 .. h-1,
 * leaf level h-1), Chebyshev interpolation with `order` roots per axis
 * (eq. 3-5; the paper's l, so a cell carries order^3 coefficients), P2M,
 * M2M, M2L (the up to 189 far cells of Sec. 2.1.2), L2L, L2P, and P2P over
 * the up to 27 near leaves.  Pairs at distance zero (a particle with itself,
 * coincident particles) contribute nothing.  F is the field per unit target
 * charge; the force on particle i is q_i F_i.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an fmm_status; no exception or signal crosses the
 *    ABI.  On failure the handle's message is available from fmm_last_error.
 *  - Pointers to particle data may be device pointers (cudaMalloc, PyTorch
 *    CUDA tensors, managed memory) or host pointers (pageable or pinned); the
 *    library tells them apart with cudaPointerGetAttributes.  With host
 *    pointers the call copies through the device and returns only when the
 *    copy is complete.  Arrays are dense, row-major, FP64.
 *  - Work is enqueued on the handle's stream (fmm_set_stream).
 *  - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef FMM_B300_H
#define FMM_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx* fmm_handle;

#define FMM_P2P_VARIANTS 16 /* shapes of the mixed-precision P2P kernel (fmm_autotune) */
#define FMM_SCHED_CANDIDATES 8 /* evaluation schedules timed by fmm_autotune (fmm_get_schedule) */

typedef enum {
  FMM_OK = 0,
  FMM_ERR_ARG = -1,     /* invalid argument (range, null pointer, non-finite input) */
  FMM_ERR_OOM = -2,     /* device allocation failed */
  FMM_ERR_CUDA = -3,    /* a CUDA runtime call or a kernel launch failed */
  FMM_ERR_STATE = -4,   /* call out of order (e.g. evaluate before set_particles) */
  FMM_ERR_TIMEOUT = -5  /* a bounded device-side wait ran out (kernel returned early) */
} fmm_status;

typedef enum {
  FMM_FP64 = 0,   /* every stage in FP64 on the GPU */
  FMM_MIXED = 1   /* FP32 P2P and expansions; M2L on the tensor cores for order <= 7 as three
                     products of FP16 hi/lo operand pairs (TF32 hi/lo pairs when the environment
                     sets FMM_M2L_MATH=tf32 at fmm_create), FP32 accumulate; M2L on the CUDA cores
                     in FP32 for order >= 8 */
} fmm_precision;

typedef enum {
  FMM_M2L_FULL = 0,  /* the 316 full-rank operators K_t (l^3 x l^3 each) */
  FMM_M2L_SVD = 1    /* the paper's compressed operators (default), see fmm_set_m2l */
} fmm_m2l_method;

/* Creates a handle for trees of `height` levels (1..11) and interpolation
 * order `order` (2..10 roots per axis; Sec. 2.1.1, the paper's l).  Allocates
 * the translation operators of Sec. 2.1.1-2.1.2 on the current CUDA device
 * and computes them there in FP64 (the 316 M2L operators for unit cell
 * half-width, scaled per level by homogeneity).  *out receives the handle
 * (NULL on failure).  Errors: FMM_ERR_ARG (range, out == NULL),
 * FMM_ERR_CUDA (no device), FMM_ERR_OOM. */
fmm_status fmm_create(int height, int order, fmm_handle* out);

/* Releases every device buffer, stream and graph the handle owns.  NULL is
 * accepted.  Synchronises the handle's stream first. */
fmm_status fmm_destroy(fmm_handle h);

/* Sets the CUDA stream (a cudaStream_t, NULL = legacy default stream) on
 * which later calls enqueue their work.  The caller keeps the stream alive. */
fmm_status fmm_set_stream(fmm_handle h, void* cuda_stream);

/* Chooses the arithmetic of later evaluations (default FMM_MIXED). */
fmm_status fmm_set_precision(fmm_handle h, int precision);

/* Chooses the M2L operators of later evaluations (Sec. 2.1.2).
 *   FMM_M2L_SVD (default): the "improved M2L operator" of Sec. 2.1.2.  The
 *     316 operators are images of 16 canonical ones (transfer vectors with
 *     0 <= t1 <= t2 <= t3) under the cube's symmetries, which permute the
 *     interpolation nodes; each canonical operator is compressed by its own
 *     SVD, keeping the singular values s_i >= eps * s_0, and M2L applies
 *     y = V^T (permuted M), L += (1/a) (permuted U Sigma y).  eps <= 0 selects
 *     10^-order, the pairing (l, eps) = (Acc, 10^-Acc) of Table 1.  The SVDs
 *     run once per handle and eps, on the device in FP64 (one-sided Jacobi),
 *     inside the first evaluation (or fmm_get_svd_ranks).
 *   FMM_M2L_FULL: the full-rank K_t, so that the order alone sets the
 *     approximation.
 * Errors: FMM_ERR_ARG (unknown method, eps >= 1 or NaN). */
fmm_status fmm_set_m2l(fmm_handle h, int method, double eps);

/* Chooses the kernel of later evaluations from the family
 * P(x, y) = (|x - y|^2 + c^2)^(-s/2), -2 <= s <= 4, s != 0, c >= 0 (default
 * s = 1, c = 0, the Laplace kernel of eq. 2; c = 0: |x - y|^-s; c > 0 the
 * multiquadrics: s = -1 multiquadric, s = 1 inverse multiquadric, s = 2
 * inverse quadric).  phi_i = sum_j q_j P(x_i, x_j) and F_i = -grad phi_i =
 * s sum_j q_j (x_i - x_j) (|x_i - x_j|^2 + c^2)^(-(s+2)/2); pairs at distance 0
 * are skipped (also for c > 0: a caller wanting the diagonal adds q_i P(0)).
 * The black-box method (Sec. 2.2) needs nothing but kernel values: the M2L
 * operators become K_t[m][n] = P_(c/a)(2t + xbar_n - xbar_m) scaled by a^-s
 * at half-width a.  c = 0 is homogeneous: one set serves every level, and the
 * compressed operators (fmm_set_m2l) are recomputed for it.  c > 0 is not:
 * one full-rank set per level 2..h-1 (c/a of that level), rebuilt when the
 * root width changes; the compression and batches (fmm_set_batch) need c = 0
 * (with c > 0 the full-rank operators are used whatever fmm_set_m2l chose,
 * and evaluating a batch fails with FMM_ERR_STATE).  The near field
 * evaluates the kernel (other than 1/r in one kernel shape; see
 * fmm_autotune).  Drops the handle's M2L operators (rebuilt by the next
 * evaluation); synchronises the stream.  Errors: FMM_ERR_ARG (s or c out of
 * range, or not finite). */
fmm_status fmm_set_kernel(fmm_handle h, double s, double c);

/* Stokes kernel (Sec. 2.2 names it with Laplace among the kernels of the
 * black-box method): velocities u_i = sum_k [f_k / r + d (d . f_k) / r^3],
 * d = x_i - x_k, r = |d| (the Stokeslet with unit viscosity factor: multiply
 * by 1/(8 pi mu) for a fluid of viscosity mu), at the handle's particles
 * (fmm_set_particles; their charges are not used) for forces f [n][3]
 * (caller order, host or device); u [n][3] (host or device).  Computed from
 * four 1/r passes on the handle's tree, with the charges f_x, f_y, f_z and
 * (y - o) . f (o = the root cube's centre):
 *     u_i = phi^i + sum_j (x_i - o)_j F^j_i - F^3_i,
 * since d (d . f) / r^3 = -grad_x(1/r) ((x - o) . f - (y - o) . f); the
 * handle's precision, M2L form and P2P variant apply to each pass.  The
 * handle's charges are restored afterwards.  Pairs at distance 0 are
 * skipped.  Synchronises the stream for host output.  Errors: FMM_ERR_STATE
 * (no particles, a batch, or a kernel other than 1/r), FMM_ERR_ARG. */
fmm_status fmm_evaluate_stokes(fmm_handle h, const double* f, double* u);

/* Ranks of the 16 compressed canonical operators, in lexicographic order of
 * their transfer vectors ((0,0,2), (0,0,3), (0,1,2), ..., (3,3,3)), for the
 * handle's order and the eps of fmm_set_m2l; computes the SVDs if they are
 * not there yet (synchronises the stream).  ranks: 16 int32, host.
 * Errors: FMM_ERR_STATE (height < 3: no M2L), FMM_ERR_CUDA (an SVD did not
 * converge). */
fmm_status fmm_get_svd_ranks(fmm_handle h, int32_t* ranks);

/* Loads n particles and builds the tree (Sec. 3.2 subdivision, Sec. 4.2
 * Morton order): root cube = per-axis minimum corner and largest extent
 * (side 1 if all points coincide), leaf-level Morton keys
 * floor(((x - lo) / W) * 2^(h-1)) clamped to the cube with x the most
 * significant bit of each triple, a stable radix sort (ties keep input
 * order), leaf ranges and the non-empty cells of every level.
 *   xyz: [n][3] FP64, q: [n] FP64 (device or host).  The data are copied;
 *   the caller may release both after the call returns (the call
 *   synchronises the stream: the per-level cell counts come back to the host).
 *   n = 0 is valid.  n <= 2^30.
 * Errors: FMM_ERR_ARG (n out of range, NULL with n > 0, a non-finite
 * coordinate or charge -- detected on the device), FMM_ERR_OOM, FMM_ERR_CUDA. */
fmm_status fmm_set_particles(fmm_handle h, int64_t n, const double* xyz, const double* q);

/* Loads a batch of nprob independent problems (1 .. 4096) and builds one
 * tree over all of them, so that every later fmm_evaluate runs each stage of
 * the method for the whole batch in one launch.  Problem k has counts[k]
 * particles (0 allowed) and its own tree of heights[k] levels (1..10), and is
 * solved exactly as fmm_set_particles + fmm_evaluate would solve it alone on
 * a handle of that height and the handle's order: its own root cube,
 * Morton keys and cells (Sec. 3.2, Sec. 4.2), no interaction with any other
 * problem.
 *   xyz: [sum counts][3] FP64 and q: [sum counts] FP64 (device or host), the
 *   problems' particles one after another in problem order.
 * Layout: problem k occupies an aligned slot of the batch tree -- one cell of
 * level Lf - (heights[k] - 1), where Lf is the batch tree's leaf level -- and
 * its particles are mapped into that cell (coordinates scaled by
 * lambda_k = slot width / W_k); cells of different problems are never
 * neighbours; fmm_evaluate rescales phi by lambda_k and F by lambda_k^2, so the
 * outputs are in each problem's own units, in the concatenated input order.
 * The slots' leaf cells, sum over problems of 8^(heights[k]-1), must fit in
 * 8^9.  The handle's own height is not used (fmm_set_particles restores it);
 * the introspection calls (fmm_get_order, fmm_get_level_*, fmm_get_box,
 * fmm_get_work, fmm_get_expansion) describe the batch tree.  Synchronises the
 * stream.
 * Errors: FMM_ERR_ARG (nprob, a count or a height out of range, too many
 * leaf cells, NULL with particles, a non-finite input), FMM_ERR_OOM,
 * FMM_ERR_CUDA. */
fmm_status fmm_set_batch(fmm_handle h, int32_t nprob, const int64_t* counts, const int32_t* heights,
                         const double* xyz, const double* q);

/* The slot layout fmm_set_batch uses, computed on the host only (no device
 * needed): problems with particles, sorted by decreasing height (ties in
 * input order), take consecutive ranges of 8^(height-1) leaf keys of the
 * batch tree, so every range starts at a multiple of its size and is one
 * cell of level *leaf_level - (height - 1); *leaf_level is the smallest
 * level that holds every range and every problem's own leaf level.
 * slot_key[k] = first leaf key of problem k's slot, slot_level[k] = the
 * slot cell's level (both -1 for a problem without particles); host arrays
 * of nprob.  Errors (message from fmm_last_error(NULL)): FMM_ERR_ARG (ranges
 * as in fmm_set_batch, or more than 8^9 leaf keys in all). */
fmm_status fmm_batch_plan(int32_t nprob, const int64_t* counts, const int32_t* heights, int64_t* slot_key,
                          int64_t* slot_level, int32_t* leaf_level);

/* Problem k of the last fmm_set_batch:
 *   info[0] = Morton rank of its first particle in the batch tree (its
 *             particles hold ranks info[0] .. info[0] + info[1] - 1, in the
 *             problem's own Morton order),
 *   info[1] = particle count, info[2] = level of its slot cell in the batch
 *   tree (-1 if it has no particles), info[3] = first leaf key of the slot
 *   (the problem's own leaf key of a particle is its batch leaf key minus
 *   info[3]), info[4] = leaf level of the batch tree, info[5] = the problem's
 *   height, info[6] = index of its first particle in the input, info[7] = 0;
 *   box[0..3] = the problem's root cube (lower corner, side), as
 *   fmm_get_box would report it for the problem alone.
 * Either pointer may be NULL.  Host memory.  Errors: FMM_ERR_STATE (no batch
 * loaded), FMM_ERR_ARG (k out of range). */
fmm_status fmm_get_batch_info(fmm_handle h, int32_t k, int64_t* info, double* box);

/* Runs one FMM pass over the particles of the last fmm_set_particles (or
 * fmm_set_batch): P2M, M2M, M2L, L2L, L2P on one branch and P2P on another
 * (Sec. 3.2), and writes phi [n] and F [n][3] (FP64) in the caller's input
 * order.
 * Device outputs: the call returns after enqueueing (stream-ordered).
 * Host outputs: the call returns after the results are in host memory.
 * Errors: FMM_ERR_STATE (no particles loaded), FMM_ERR_ARG (NULL with
 * n > 0), FMM_ERR_CUDA, FMM_ERR_TIMEOUT (a bounded wait inside the previous
 * evaluation's tensor-core M2L ran out: that evaluation's results are
 * invalid; the flag travels with the stream, so it is reported by the next
 * call on the handle). */
fmm_status fmm_evaluate(fmm_handle h, double* phi, double* F);

/* Picks the shape of the mixed-precision P2P kernel (the near field of
 * Sec. 2.1, the largest kernel on surface distributions and batches) for the
 * current tree by timing each variant three times on the handle's stream
 * with CUDA events, and keeps the fastest for later evaluations (the
 * evaluation graph is rebuilt).  Variants 0..5: two sources per
 * instruction (packed FP32 pairs), (warps per block, sources staged per
 * chunk, unroll of the pair loop) = (8,128,4) -- the default --, (4,128,4),
 * (4,256,2), (4,128,2), (8,128,2), (8,256,2); variants 6..11: one source per
 * instruction, (warps, chunk) = (4,256), (2,128), (2,256), (4,128), (8,128),
 * (8,256); variants 12, 13: packed, leaf-cooperative (a block of 8 warps
 * takes up to 8 work items of one leaf and stages each chunk of their common
 * sources once), chunks of 512 and 1024 sources; variants 14, 15: packed,
 * persistent (blocks of 4 warps, as many as fit on the GPU at once; every
 * warp takes the next work item from a counter until none is left), (chunk,
 * unroll) = (128, 4), (256, 2).  They give the same sums up to the grouping
 * of FP32 partial sums.
 * The work items are binned by leaf occupancy -- leaves of at most 64
 * particles ("small") and larger ones -- and each bin is timed alone in
 * every shape (the cooperative shapes on large leaves only) and keeps its
 * fastest; later evaluations run the bins as two launches with their own
 * shapes (one launch when the shapes agree), unless one launch of a single
 * shape over every item -- the item shape with the least time over both
 * bins, timed as one launch -- is faster; fmm_get_p2p_bins reports the
 * result.
 * Last, in mixed precision with a far field (height >= 3), the evaluation
 * schedule: whole evaluations (two passes over the candidates, each
 * building the candidate's graph afresh and timing three runs; the slower
 * pass counts) in each schedule of fmm_set_schedule (2 and 3 only with the
 * compressed tensor-core M2L on FP16 operands), each with the chosen shapes
 * and -- when those include a persistent shape (14, 15), whose blocks hold
 * their SMs until the last work item is taken -- with the fastest
 * non-persistent shapes per bin; the fastest candidate's schedule and
 * shapes are kept (fmm_get_schedule).  The paper's schedulers decide where near- and
 * far-field tasks run from measured costs (Sec. 4 and 5); this is the same
 * decision for one GPU's fixed launch order.
 * choice (may be NULL): the small leaves' shape (the large leaves' if there
 * are no small ones): [0] index, [1] warps per block, [2] sources per
 * chunk, [3] sources per instruction, [4] unroll; times_ms (may be NULL):
 * FMM_P2P_VARIANTS mean times of each shape run over both bins (a
 * cooperative shape with shape 14 on the small leaves).  With a kernel other than 1/r
 * (fmm_set_kernel) the near field has one shape (8 warps, 128-source chunks,
 * two sources per instruction): choice = {-1, 8, 128, 2, 4} and every time is
 * that shape's.  Synchronises the
 * stream.  Errors: FMM_ERR_STATE (no particles loaded). */
fmm_status fmm_autotune(fmm_handle h, int32_t* choice, float* times_ms);

/* Time limit of each bounded wait inside the tensor-core M2L kernels (the
 * pipeline waits of Sec. 2.1.2's M2L between the copies, the MMAs and the
 * epilogue; default 2 s, far beyond any real stage): a wait that runs out
 * makes the kernel raise its error word, wait for the copies and MMAs it has
 * already issued (always with the 2 s limit), free its tensor memory and
 * return, and the next call on the handle reports FMM_ERR_TIMEOUT.  The
 * paper has no counterpart; this is failure detection without a fault.
 * 0 < seconds <= 60.  The evaluation graph is rebuilt.  Errors: FMM_ERR_ARG. */
fmm_status fmm_set_wait_limit(fmm_handle h, double seconds);

/* Sets the P2P variant directly (0 .. FMM_P2P_VARIANTS-1; 0 is the default),
 * e.g. to reuse a choice fmm_autotune made on another handle, for every
 * leaf (a cooperative shape, 12 or 13, takes the large leaves and shape 14
 * the small ones). */
fmm_status fmm_set_p2p_variant(fmm_handle h, int variant);

/* The near field's occupancy bins on the current tree (mixed precision,
 * 1/r): out[0] = shape of the small leaves' work items (leaves of at most 64
 * particles), out[1] = shape of the large leaves' items, out[2] / out[3] =
 * work items (32 targets of one leaf each) in each bin; times_ms (may be
 * NULL): [2][FMM_P2P_VARIANTS] per-bin times of the last fmm_autotune (-1:
 * not timed).  The paper has no counterpart; it stands in for the
 * calibration of Sec. 5 that lets its scheduler pick a worker per task.
 * out: 4 int64, host.  Errors: FMM_ERR_STATE (no particles loaded). */
fmm_status fmm_get_p2p_bins(fmm_handle h, int64_t* out, float* times_ms);

/* 1 if this library is the debug build (compiled with FMM_DEBUG: bounds
 * checks at the index computations of the tree build, the near field's
 * staging and the compressed M2L's setup and projection, each recording its
 * first failure and skipping the access it guards), 0 otherwise.  The paper
 * has no counterpart; this is race- and bounds-checking without a
 * sanitizer. */
int fmm_debug_build(void);

/* The first bounds check that failed since the previous call, as (site << 32
 * | index), 0 if none (always 0 in the normal build); the record is cleared.
 * Sites: 1 a particle's sorted index (tree gather), 2 a cell index (tree
 * levels), 3 a staged near-field source outside its neighbour leaf, 4 a
 * neighbour key outside a level's grid (M2L tile setup), 5 a
 * destination-map index, 6 a projection's destination row (compressed M2L).
 * Synchronises the device.  first_failure: host.  Errors: FMM_ERR_ARG
 * (NULL), FMM_ERR_CUDA. */
fmm_status fmm_debug_check(uint64_t* first_failure);

/* Where the near-field branch (P2P, Sec. 2.1) starts in the evaluation
 * graph, its blocks at the low launch priority: 0 (the default) with the
 * compressed M2L's expansion kernel, after the projection; 1 at the start
 * of the evaluation, beside the upward pass, filling the SMs that the
 * upward pass and the M2L bookkeeping kernels leave idle; 2 with the
 * projection, which then runs three pipeline stages instead of four so that
 * P2P blocks fit beside its CTA on every SM; 3 as 2, and the expansion
 * with two stages (room for P2P blocks beside it too).  With another M2L
 * form, 2 and 3 act as 0.  The arithmetic is the same in every schedule:
 * the results are bit-identical.  fmm_autotune sets it from measured
 * evaluations.  The evaluation graph is rebuilt.  Errors: FMM_ERR_ARG
 * (sched outside 0..3). */
fmm_status fmm_set_schedule(fmm_handle h, int sched);

/* The current schedule (*sched, host int32) and, in times_ms (may be NULL;
 * FMM_SCHED_CANDIDATES floats, host), the evaluation time of each candidate
 * of the last fmm_autotune (the larger of two passes' means of three runs,
 * each pass with the candidate's graph built afresh; the smallest is kept,
 * the first on a tie): [k] schedule k with the chosen
 * near-field shapes, [4 + k] schedule k with the fastest non-persistent
 * shapes (k = 0..3); -1 where not timed. */
fmm_status fmm_get_schedule(fmm_handle h, int32_t* sched, float* times_ms);

/* Releases every device buffer that belongs to the current tree (particles,
 * cells, expansions, M2L work tables and projections, staging) and keeps the
 * translation operators and the compressed factors, so that a later
 * fmm_set_particles / fmm_set_batch rebuilds without recomputing them.  Until
 * then evaluate and the tree getters report FMM_ERR_STATE.  Synchronises the
 * handle's streams.  (A long-lived process -- the solve server below -- uses
 * it to keep idle handles small.) */
fmm_status fmm_trim(fmm_handle h);

/* Morton permutation of the last fmm_set_particles: perm[r] = input index of
 * the particle with Morton rank r.  perm: [n] int64, device or host. */
fmm_status fmm_get_order(fmm_handle h, int64_t* perm);

/* Root cube of the last fmm_set_particles: out[0..2] = lower corner,
 * out[3] = side.  out: 4 doubles, host. */
fmm_status fmm_get_box(fmm_handle h, double* out);

/* Number of non-empty cells at `level` (0 .. height-1) of the current tree,
 * host int64. */
fmm_status fmm_get_level_size(fmm_handle h, int level, int64_t* out);

/* Sorted Morton keys (at that level's resolution) of the non-empty cells of
 * `level`; keys: [level_size] uint64, device or host. */
fmm_status fmm_get_level_keys(fmm_handle h, int level, uint64_t* keys);

/* Leaf level: first particle (Morton rank) and particle count per leaf;
 * other levels: first child index (at level+1) and child count per cell.
 * first, count: [level_size] int64, device or host. */
fmm_status fmm_get_level_ranges(fmm_handle h, int level, int64_t* first, int64_t* count);

/* Multipole (which = 0) or local (which = 1) expansion of every non-empty
 * cell of `level` after the last fmm_evaluate, widened to FP64:
 * out [level_size][order^3], coefficient index (mx * p + my) * p + mz.
 * Levels below 2 carry none (FMM_ERR_ARG).  Synchronises the stream. */
fmm_status fmm_get_expansion(fmm_handle h, int level, int which, double* out);

/* Counters of the handle: out[0] = kernel launches enqueued by the last
 * fmm_set_particles, out[1] = kernels launched by one fmm_evaluate
 * (nodes of its CUDA graph + the output launch), out[2] = 1 if evaluations
 * replay a CUDA graph, out[3] = bytes of device memory the handle holds,
 * out[4] = M2L kernels of the current precision and method (full-rank
 * operators: 0 = FP64 CUDA cores, 1 = FP32 CUDA cores on split operands,
 * 2 = tcgen05 tensor cores; compressed operators: 3 = FP64 CUDA cores,
 * 4 = FP32 CUDA cores, 5 = tcgen05 tensor cores), out[5] = 1 if the
 * tensor-core M2L (out[4] = 2 or 5) takes FP16 hi/lo operands (the default;
 * 0: TF32 hi/lo, chosen at fmm_create by the environment variable
 * FMM_M2L_MATH=tf32, or a CUDA-core M2L),
 * out[6] = evaluations that ran their launches without a CUDA graph because
 * the stream capture of the graph failed with a capture error (the same
 * kernels, launched one by one; the capture's message stays available from
 * fmm_last_error; any other CUDA error fails the evaluation), out[7] = 0
 * (reserved).  out: 8 int64, host. */
fmm_status fmm_get_stats(fmm_handle h, int64_t* out);

/* Algorithmic work of one evaluation on the current tree (Sec. 4.3 counts
 * work the same way): out[0] = directed P2P particle pairs (each target with
 * every particle of its up to 27 near leaves, itself excluded), out[1 + l] =
 * M2L (target, source) cell pairs at level l for l = 0 .. 10 (zero outside
 * 2 .. height-1), out[12] = (M2L tile, transfer vector) pairs with at least
 * one source (each is one 128-row block of M2L products), out[13] = sum
 * over the M2L pairs of the rank of their compressed operator (0 until the
 * compressed operators exist; one pair costs 4 * order^3 * rank flop),
 * out[14] / out[15] = sum over the (M2L tile, transfer vector) blocks of the
 * compressed projection / expansion of the Y columns per cell (the rank,
 * rounded up to 16 on the mixed path -- to 8 with the FP16 tensor-core
 * operands, whose expansion runs each tile over its child class's
 * concatenated ranks: out[15] = tiles x that K; 0 until the compressed
 * operators exist): the projection multiplies 128 x order^3 by order^3 x
 * out[14] columns, the expansion 128 x out[15] by out[15] x order^3 (summed
 * over blocks).
 * Synchronises the stream.  out: 16 int64, host. */
fmm_status fmm_get_work(fmm_handle h, int64_t* out);

/* Per-stage device times of the last fmm_evaluate in milliseconds (CUDA
 * events recorded inside the evaluation when timing is on), in this order:
 * [0] upward pass (P2M + M2M), [1] M2L (all levels), [2] the main M2L
 * kernel (CUDA-core kernels: the leaf level; tensor-core kernel: every
 * level), [3] the rest of M2L (coarser levels; or the FP64 reduction of the
 * tensor-core partial sums), [4] L2L (all levels), [5] P2P, [6] L2P +
 * output, [7] whole evaluation.
 * fmm_set_timing(h, mode) turns the events on (the evaluation graph is
 * rebuilt): mode 1 keeps the normal schedule, where P2P overlaps M2L and its
 * time [5] is that of the overlapped branch; mode 2 runs P2P alone before
 * M2L so that every stage is timed in isolation; mode 0 turns the events
 * off (FMM_ERR_ARG outside 0..2).  fmm_get_stage_times synchronises the
 * stream.  out: 8 floats, host. */
fmm_status fmm_set_timing(fmm_handle h, int mode);
fmm_status fmm_get_stage_times(fmm_handle h, float* out);

/* Device times in milliseconds of the tensor-core M2L kernels of the last
 * timed fmm_evaluate (Sec. 2.1.2's M2L; CUDA events recorded around each
 * launch inside the evaluation graph while fmm_set_timing is on):
 * out[0] = the compressed projection y = V^T M (k_svd_proj_tc; 0 on the
 * full-rank path), out[1] = the compressed expansion L += U y
 * (k_svd_expand_tc) or the full-rank product (k_m2l_tc).  Synchronises the
 * stream.  Errors: FMM_ERR_STATE (timing off, no timed evaluation, or an M2L
 * path that does not run on the tensor cores).  out: 2 floats, host. */
fmm_status fmm_get_m2l_kernel_times(fmm_handle h, float* out);

/* FP32 arithmetic rate of the current device, measured (the paper has no
 * counterpart: it gives the roofline that the near field, Sec. 2.1's P2P, is
 * judged against).  A throughput kernel runs independent FMA chains on 8
 * blocks of 256 threads per SM for about 10 ms per launch (one warm-up launch,
 * then the best of three): out[0] = scalar fma.rn.f32 rate in flop/s (2 flop
 * per FMA and lane), out[1] = packed fma.rn.f32x2 rate in flop/s (4 flop per
 * instruction and lane), out[2] = the SM count the kernel ran on
 * (cudaDevAttrMultiProcessorCount), out[3] = 0.  Uses its own stream and
 * synchronises it; no handle needed.  out: 4 doubles, host.
 * Errors: FMM_ERR_ARG (out NULL), FMM_ERR_CUDA. */
fmm_status fmm_measure_fp32_rate(double* out);

/* Allocation-free Morton ordering (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they
 * run -- processes whose HBM is owned by a pool reserved at start-up, such as
 * a serving loop that must never stall in the driver's allocator, and
 * plug-ins that only receive buffers from their host application).
 * It computes the first steps of fmm_set_particles for a tree of `height`
 * levels (1..11) -- root cube, leaf-level Morton keys, stable sort -- and
 * writes, for Morton rank r, keys[r] = leaf key and perm[r] = input index:
 * the same permutation fmm_get_order returns and the keys of
 * fmm_get_level_keys(height-1) repeated over each leaf's particles.
 *   xyz: [n][3] FP64 device; keys: [n] uint64 device; perm: [n] int64 device;
 *   stream: a cudaStream_t (NULL = legacy default stream).
 *   n <= 262144 (2^18); larger n -> FMM_ERR_ARG with a message.
 * It allocates nothing: every intermediate lives in one fixed array of about
 * 4.3 MB compiled into the library, which each GPU that loads the library
 * holds until the process exits.  All calls on a GPU share that array, so
 * calls whose work overlaps on the GPU race and must be serialised by the
 * caller.  Every call looks the array's address up on the current device (a
 * host-side query, so a device reset between calls is harmless) and
 * synchronises `stream` before it returns (it reads back the input check into
 * host memory): it cannot be called while the calling thread captures a
 * stream into a CUDA graph.  Errors (message from fmm_last_error(NULL)):
 * FMM_ERR_ARG (range, NULL, non-finite coordinate), FMM_ERR_CUDA. */
fmm_status fmm_morton_order_noalloc(int64_t n, const double* xyz, int height, uint64_t* keys, int64_t* perm,
                                    void* stream);

/* ---- Solve server: continuous batching of independent requests ------------
 *
 * A server owns `lanes` worker threads on the current device, each with its
 * own CUDA stream and one resident FMM handle per interpolation order (trees,
 * expansions and operators stay on the device between batches).  A free lane
 * takes the oldest queued request (or, while that one has waited less than
 * 50 ms, the oldest request of the order the lane ran last, whose tree it
 * holds) and every later queued request of the same
 * order that still fits -- at most max_batch_particles particles and
 * max_batch_requests requests per batch, the batch tree's leaf cells within
 * fmm_set_batch's limit, and the device-memory estimate of all batches in
 * flight within hbm_budget_bytes -- and solves them as one fmm_set_batch +
 * fmm_evaluate.  Requests that arrive while lanes are busy wait in the queue
 * and are admitted as lanes and memory free up; batches on different lanes
 * overlap on the device.  Each request is solved exactly as it would be alone
 * (fmm_set_batch's guarantee); only the rounding of the tensor-core partial
 * sums may differ.  The paper has no counterpart (its runtime schedules the
 * tasks of one FMM). */
typedef struct fmm_server* fmm_server_handle;

typedef struct {
  int32_t lanes;               /* concurrent batches (1..16) */
  int32_t precision;           /* FMM_MIXED or FMM_FP64 */
  int64_t hbm_budget_bytes;    /* device-memory estimate of all batches in flight at most */
  int64_t max_batch_particles; /* particles per batch at most (a larger single request runs alone) */
  int32_t max_batch_requests;  /* requests per batch at most (1..4096) */
  int32_t reserved;
} fmm_server_config;

/* Device memory a request is charged for admission: 256 bytes per particle
 * plus, per cell (1.15 x min(n, 8^(height-1)) cells), its expansions
 * (28 bytes x order^3 rounded up to 32) and its share of the compressed M2L's
 * projections (4 bytes x 189 x 16 at order <= 5, x 32 above) and tables
 * (1 KB).  A request above hbm_budget_bytes is refused. */
int64_t fmm_server_request_bytes(int64_t n, int height, int order);

/* Creates a server (threads start at once, idle).  Errors: FMM_ERR_ARG (a
 * config field out of range), FMM_ERR_CUDA (no device, stream creation). */
fmm_status fmm_server_create(const fmm_server_config* cfg, fmm_server_handle* out);

/* Creates every lane's handle for `order` and its compressed M2L operators
 * (the FP64 SVDs, seconds at order 7) before traffic; blocks until done. */
fmm_status fmm_server_warmup(fmm_server_handle s, int order);

/* Queues one request: n particles (xyz [n][3], q [n], FP64) for a tree of
 * `height` levels (1..10) and interpolation order `order` (2..10); results
 * phi [n] and F [n][3] (FP64, input order) are written by the lane.  All four
 * pointers may be host (pageable or pinned) or device memory and must stay
 * valid until fmm_server_wait returns for the ticket.  Returns at once;
 * *ticket identifies the request.  Errors: FMM_ERR_ARG (range, NULL),
 * FMM_ERR_OOM (the request alone exceeds the budget), FMM_ERR_STATE (server
 * stopping). */
fmm_status fmm_server_submit(fmm_server_handle s, int64_t n, int height, int order, const double* xyz,
                             const double* q, double* phi, double* F, int64_t* ticket);

/* Waits up to timeout_s seconds (< 0: forever) for a request.  On completion
 * the ticket is released and the request's own status is returned (FMM_OK or
 * the failing call's status, message in fmm_server_last_error); times (may be
 * NULL) receives, in ms of the host's steady clock: [0] submit -> batch start
 * (queueing), [1] batch start -> results in the caller's memory (service),
 * [2] submit -> results (latency), [3] requests in the request's batch.
 * Errors: FMM_ERR_ARG (unknown ticket), FMM_ERR_TIMEOUT (still pending; the
 * ticket stays valid). */
fmm_status fmm_server_wait(fmm_server_handle s, int64_t ticket, double timeout_s, double* times);

/* Counters: out[0] requests completed, [1] batches run, [2] particles
 * completed, [3] peak memory charge at an admission (bytes), [4] peak number
 * of batches running at once, [5] largest batch (requests), [6] requests
 * queued now, [7] device bytes held by the lanes (handles and staging),
 * [8] [9] [10] lane time summed over batches, in microseconds: copying the
 * inputs, fmm_set_batch, fmm_evaluate + copying the results, [11] trims of
 * idle handles, [12] evaluations on the lanes' handles that ran without a
 * CUDA graph because capturing it failed (fmm_get_stats out[6], summed; 0
 * expected).  out: 13 int64, host. */
fmm_status fmm_server_stats(fmm_server_handle s, int64_t* out);

/* Stops the lanes after their current batch, fails the requests still
 * queued, joins the threads and releases the server and its device memory.
 * No other call on the server may be in progress or follow.  NULL accepted. */
fmm_status fmm_server_destroy(fmm_server_handle s);

/* Message of the last failure of a server call or of a request it ran. */
const char* fmm_server_last_error(fmm_server_handle s);

/* Message of the last failed call on this handle ("" if none).  With
 * h == NULL: the message of the last failed fmm_create in this thread. */
const char* fmm_last_error(fmm_handle h);

#ifdef __cplusplus
}
#endif
#endif /* FMM_B300_H */
