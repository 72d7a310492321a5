/*
 * oracle.h -- plain FP64 CPU oracle for the black-box FMM (Laplace 1/r,
 * potentials and forces) of Agullo, Bramas, Coulaud, Darve, Messner and
 * Takahashi, "Pipelining the Fast Multipole Method over a Runtime System"
 * (INRIA RR-7981, 2012).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no source, header, table or
 * helper with the CUDA path.
 *
 * Conventions (the readings the product follows as well):
 *   height h: levels 0 .. h-1, leaf level h-1, up to 8^(h-1) leaves.
 *   order p: number of Chebyshev roots per dimension (the paper's l), so a
 *     cell carries p^3 expansion coefficients, flattened with z fastest:
 *     m = (mx * p + my) * p + mz.
 *   root cube: corner lo = per-axis minimum, side W = largest extent
 *     (W = 1 if every particle sits at one point, or n = 0).
 *   Morton key at level l: the cell's integer coordinates interleaved, x the
 *     most significant bit of each triple.
 *   F_i = sum_j q_j (x_i - x_j) / |x_i - x_j|^3  (= -grad phi; eq. 2 gives the
 *     formula and the sign is taken from it); pairs with r = 0 are skipped.
 * Arrays are row-major; xyz is [n][3].  All functions are thread-safe on
 * distinct contexts and use OpenMP internally.
 */
#ifndef FMM_ORACLE_H
#define FMM_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ofmm ofmm;

/* Chebyshev roots xbar_k = cos((2k+1) pi / (2p)), k = 0..p-1 (Sec. 2.1.1). */
void ofmm_cheb_nodes(int order, double* xbar);
/* S(xbar, xi) of eq. 5 and its derivative in xi. */
double ofmm_cheb_S(int order, double xbar, double xi);
double ofmm_cheb_dS(int order, double xbar, double xi);

/* Root cube (corner lo[3], side *width) of n points. */
void ofmm_bounding_cube(int64_t n, const double* xyz, double* lo, double* width);
/* Leaf-level Morton keys of n points for a tree whose leaf level is `leaf`. */
void ofmm_keys(int64_t n, const double* xyz, const double* lo, double width,
               int leaf, uint64_t* keys);

/* Builds box, keys, stable sort and the cell levels; NULL on bad arguments
 * (height 1..12, order 2..12, n >= 0, finite inputs). */
ofmm* ofmm_create(int64_t n, const double* xyz, const double* q, int height, int order);
void ofmm_destroy(ofmm* c);
/* Kernel P(x, y) = (|x - y|^2 + kc^2)^(-s/2), -2 <= s <= 4, s != 0, kc >= 0
 * (the default s = 1, kc = 0 is the Laplace kernel of eq. 2; F = -grad phi;
 * kc > 0: multiquadric s = -1, inverse multiquadric s = 1).  Rebuilds the M2L
 * operators and drops a compressed set.  kc = 0 is homogeneous of degree -s:
 * one set of unit half-width scaled by a^-s; kc > 0 is not: one set per
 * level, the kernel at the level's own node positions, and no compression.
 * 0 on success, -1 for arguments out of range. */
int ofmm_set_kernel(ofmm* c, double s, double kc);

void ofmm_box(const ofmm* c, double* lo, double* width);
int64_t ofmm_level_size(const ofmm* c, int level);
/* Sorted keys of the non-empty cells at `level`. */
void ofmm_level_keys(const ofmm* c, int level, uint64_t* keys);
/* Leaf level: first particle rank and particle count per leaf.  Other levels:
 * first child index (at level+1) and child count per cell. */
void ofmm_level_ranges(const ofmm* c, int level, int64_t* first, int64_t* count);
/* Morton rank -> input index. */
void ofmm_perm(const ofmm* c, int64_t* perm);

/* The operators, in the order the paper's two traversals apply them (Sec. 3.2). */
void ofmm_p2m(ofmm* c);
void ofmm_m2m(ofmm* c);
void ofmm_m2l(ofmm* c);
void ofmm_l2l(ofmm* c);
/* Far-field (L2P) and near-field (P2P) parts per particle, Morton order:
 * phi [n], F [n][3]. */
void ofmm_l2p(const ofmm* c, double* phi, double* F);
void ofmm_p2p(const ofmm* c, double* phi, double* F);
/* M (which = 0) or L (which = 1) at a level, [level_size][p^3]. */
void ofmm_expansion(const ofmm* c, int level, int which, double* out);

/* Whole pass; phi [n], F [n][3] in input order. */
void ofmm_evaluate(ofmm* c, double* phi, double* F);
/* FMM result for the input indices idx[0..ns-1] only (upward pass in full,
 * downward pass along the sampled leaves' ancestors). */
void ofmm_evaluate_sampled(ofmm* c, int64_t ns, const int64_t* idx, double* phi, double* F);

/* SVD-compressed M2L (Sec. 2.1.2, "Improved M2L operator").
 * Cube symmetry taking the canonical vector that (|t| sorted ascending) to t:
 * t_d = sign[d] * that[axis[d]]. */
void ofmm_transfer_symmetry(const int* t, int* that, int* axis, int* sign);
/* Index 0..15 of a canonical vector in lexicographic order, else -1. */
int ofmm_canonical_index(const int* that);
/* sm[m] = the node index the symmetry (axis, sign) maps node m to. */
void ofmm_node_permutation(int order, const int* axis, const int* sign, int32_t* sm);
/* A = U diag(s) V^T, n x n row-major, s descending (one-sided Jacobi).
 * Returns the number of sweeps, -1 if it did not converge. */
int ofmm_jacobi_svd(int n, const double* A, double* U, double* s, double* V);
/* Switches the context's M2L to the 16 compressed operators truncated at
 * s_i >= eps * s_0 (0 on success; needs height >= 3). */
int ofmm_set_m2l_svd(ofmm* c, double eps);
/* Copies the compressed operators of src (same order) into dst; 0 on success. */
int ofmm_copy_m2l_svd(ofmm* dst, const ofmm* src);
/* Rank of canonical operator k (0..15), -1 if the compression is off. */
int ofmm_svd_rank(const ofmm* c, int k);
/* out[C] += (operator of transfer vector t at unit half-width) M[C]
 * (homogeneous kernels; with kc > 0 out is left unchanged). */
void ofmm_m2l_apply(const ofmm* c, const int* t, const double* M, double* out);

/* Number of ordered (target, source) cell pairs M2L visits at `level`. */
int64_t ofmm_m2l_pair_count(const ofmm* c, int level);
/* For every ordered pair of leaves (T, S): how many times the near field
 * (P2P) and the far field (M2L at any level, through ancestors) cover it.
 * counts is [nleaf][nleaf]. */
void ofmm_coverage(const ofmm* c, int32_t* counts);

/* Direct O(N^2) sums of eq. 1 with the kernels of eq. 2. */
void ofmm_direct(int64_t n, const double* xyz, const double* q, double* phi, double* F);
/* The same sums with the kernel (r^2 + kc^2)^(-s/2): phi_i = sum q_j
 * (r^2 + kc^2)^(-s/2), F_i = s sum q_j (x_i - x_j) (r^2 + kc^2)^(-(s+2)/2);
 * pairs at distance 0 are skipped. */
void ofmm_direct_kernel(int64_t n, const double* xyz, const double* q, double s, double kc, double* phi,
                        double* F);
void ofmm_direct_sampled_kernel(int64_t n, const double* xyz, const double* q, double s, double kc, int64_t ns,
                                const int64_t* idx, double* phi, double* F);
/* Stokeslet sums u_i = sum_{k != i} [ f_k / r + d (d . f_k) / r^3 ], d = x_i - x_k
 * (pairs at distance 0 skipped); f, u [n][3]. */
void ofmm_stokes_direct(int64_t n, const double* xyz, const double* f, double* u);
void ofmm_direct_sampled(int64_t n, const double* xyz, const double* q, int64_t ns,
                         const int64_t* idx, double* phi, double* F);

#ifdef __cplusplus
}
#endif
#endif
