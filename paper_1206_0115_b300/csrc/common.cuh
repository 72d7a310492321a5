// common.cuh -- internal declarations of libfmm_b300 (not part of the ABI).
//
// Data layout in HBM (one handle):
//   particles, Morton order: pos64 [n] double4 (x, y, z, q), pos32 [n] float4
//     ((x - c_leaf) / w_leaf, ..., q) -- coordinates in leaf widths relative to
//     the leaf centre, so P2P offsets between neighbouring leaves are exact
//     integers and xi = 2 * pos32 for P2M / L2P; pos32lo [n] float4 holds the
//     FP32 rounding residual of each coordinate (used for close pairs).
//   cells per level l: key (uint32 Morton key at level resolution), first and
//     count (leaf: particle range; other levels: child range at l+1), parent,
//     a dense grid[8^l] key -> cell index (-1 = empty) for neighbour lookups,
//     and the level's cells grouped by child class (key & 7) for M2L.
//   expansions: one buffer per kind, rows of `cpad` coefficients
//     (order^3 rounded up to 32, pad columns zero), level l occupying rows
//     row_off[l] .. row_off[l] + ncell[l], the last row of each level all zero
//     (the source row of a missing M2L neighbour).
//   M2L operators: 316 transfer vectors t (|t|_inf in {2,3}) in lexicographic
//     order; K_t[m][n] = 1 / |2t + xbar_n - xbar_m| for unit half-width.
//   batched problems (fmm_set_batch): one octree over a unit "forest" cube in
//     which problem k owns an aligned slot, the cell of level S_k = Lf - L_k
//     (L_k its own leaf level) whose leaf keys are [slot_k, slot_k + 8^L_k);
//     its particles are mapped into the slot by x' = o_k + (x - lo_k) 2^-S_k / W_k,
//     cells carry the problem of their slot (slot[l][cell], -1 above the
//     slots), and cells of different problems are never neighbours, so every
//     stage runs over all problems in one launch; results are rescaled by
//     lambda_k = 2^-S_k / W_k (phi * lambda, F * lambda^2) on output.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fmm.h"

#define FMM_MAX_LEVELS 11
#define FMM_MAX_ORDER 10
#define FMM_NT 316       // transfer vectors
#define FMM_NT_CLASS 189 // transfer vectors of one child class
#define FMM_TILE 128     // M2L target rows per tile
#define CNT_P2P 126      // counters[] slot of the persistent P2P kernels' work counter (zeroed per launch)
#define CNT_P2P2 124     // the same for the small leaves' launch when the two bins run side by side
#define CNT_PUNITS 125   // counters[] slot of the compressed M2L projection's unit count (per evaluation)
#define P2P_BIG 64       // a leaf with more particles is "large" for the near field's bins

namespace fmm {

struct Tile {
  int level;  // tree level (2 .. leaf)
  int cls;    // child class of every target (key & 7)
  int first;  // offset into the level's class-grouped cell list
  int count;  // targets in the tile (<= FMM_TILE)
};

// Per-level device pointers handed to kernels by value.
struct LevelPtrs {
  uint32_t* key[FMM_MAX_LEVELS];
  int32_t* first[FMM_MAX_LEVELS];
  int32_t* count[FMM_MAX_LEVELS];
  int32_t* parent[FMM_MAX_LEVELS];
  int32_t* grid[FMM_MAX_LEVELS];
  int32_t* cls[FMM_MAX_LEVELS];
  int32_t* slot[FMM_MAX_LEVELS];  // batched trees: problem of each cell (-1: none); nullptr for one problem
  int64_t row_off[FMM_MAX_LEVELS];
  int32_t ncell[FMM_MAX_LEVELS];  // host-known sizes (valid after the readback)
};

// The kernel family P(x, y) = (|x - y|^2 + c^2)^(-s/2) (s = 1, c = 0: the
// Laplace kernel of eq. 2; fmm_set_kernel).  P(a rho) = a^-s (|rho|^2 +
// (c/a)^2)^(-s/2): with cell half-width a the M2L operators are a^-s K_t,
// K_t[m][n] = P_(c/a)(2t + xbar_n - xbar_m), one set for every level when
// c = 0 (homogeneous), one set per level (c2 = (c/a)^2) when c > 0.  s = 1,
// c = 0 keeps the reciprocal square root exactly as before.
__host__ __device__ inline double kernel_r2(double r2, double s, double c2 = 0.0) {
  return (s == 1.0 && c2 == 0.0) ? 1.0 / sqrt(r2) : pow(r2 + c2, -0.5 * s);
}
__host__ __device__ inline double kernel_scale(double inv_a, double s) { return s == 1.0 ? inv_a : pow(inv_a, s); }

// Batched trees: whether cell g at level l may interact with a cell whose
// problem is `mine` (the problem of the asking cell; -1 above the slots).
__host__ __device__ inline bool same_problem(const LevelPtrs& lv, int l, int mine, int g) {
  return !lv.slot[l] || (mine >= 0 && lv.slot[l][g] == mine);
}
__host__ __device__ inline int problem_of(const LevelPtrs& lv, int l, int cell) {
  return lv.slot[l] ? lv.slot[l][cell] : 0;
}

// One problem of a batch (device copy, input order).
struct BatchProb {
  uint32_t slot_key;  // first forest leaf key of the problem's slot
  int32_t L;          // the problem's own leaf level (height - 1)
  int32_t S;          // level of its slot cell in the forest (Lf - L)
  int32_t thr;        // offset of its leaf-level cell thresholds in the batch's table
};

#define FMM_MAX_FOREST_LEAF 9  // leaf level of a batched tree at most (dense grid 8^9 x 4 bytes)
#define FMM_MAX_BATCH 4096     // problems per batch at most

}  // namespace fmm

// The handle of include/fmm.h.
struct fmm_ctx {
  using Tile = fmm::Tile;
  using LevelPtrs = fmm::LevelPtrs;
  int height = 0, order = 0, leaf = 0, ncoef = 0, cpad = 0;
  int precision = FMM_MIXED;
  double kernel_s = 1.0;  // P(x, y) = (|x - y|^2 + kernel_c^2)^(-kernel_s / 2)
  double kernel_c = 0.0;
  int dev = 0;
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t side = nullptr;    // P2P branch
  cudaStream_t side2 = nullptr;   // the small leaves' P2P bin beside the large leaves' one
  cudaEvent_t ev_bin0 = nullptr, ev_bin1 = nullptr;  // its fork and join
  cudaStream_t cap = nullptr;     // graph capture
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_p2p = nullptr;  // where the P2P branch starts (after the compressed M2L projection)
  cudaStream_t side3 = nullptr;   // the compressed M2L's tree-only bookkeeping beside the upward pass
  cudaEvent_t ev_start = nullptr, ev_prep = nullptr;  // its fork (the evaluation's start) and join
  bool m2l_prep_done = false;     // that bookkeeping was launched on side3 (ev_prep marks its end)
  cudaStream_t side4 = nullptr;   // the leaf level's FP16 class-order multipoles beside the M2M levels
  cudaEvent_t ev_p2m = nullptr, ev_gleaf = nullptr;  // its fork (P2M done) and join
  bool leaf_gather_done = false;  // that gather was launched on side4 (ev_gleaf marks its end)
  bool p2p_after_proj = false;   // ev_p2p was recorded by the M2L launch (the P2P branch starts there)
  char err[512] = {0};
  cudaError_t last_cuda = cudaSuccess;  // the CUDA error behind the last FMM_ERR_CUDA / FMM_ERR_OOM

  // particles
  int64_t n = 0, ncap = 0;
  bool loaded = false;
  uint32_t *key_a = nullptr, *key_b = nullptr, *idx_a = nullptr, *idx_b = nullptr;
  uint32_t* skey = nullptr;  // sorted keys (points at key_a or key_b)
  int32_t* perm = nullptr;
  int32_t* pleaf = nullptr;  // leaf of every particle (Morton order)
  double4* pos64 = nullptr;
  float4* pos32 = nullptr;
  float4* pos32lo = nullptr;  // rounding residuals of pos32's coordinates (x = hi + lo to ~2^-48)
  float4* near32 = nullptr;
  int32_t* p2p_items = nullptr;  // per leaf: first P2P work item (batches of 32 targets)
  int64_t p2p_items_cap = 0;
  int32_t* p2p_leaf = nullptr;   // per work item: its leaf
  int64_t p2p_leaf_cap = 0;
  int32_t* p2p_units = nullptr;  // cooperative P2P units: first item of each (up to 8 items of a leaf)
  int64_t p2p_units_cap = 0;
  int p2p_nunits = 0;
  int p2p_nitems = 0;
  // bins by leaf occupancy (P2P_BIG): the items of each bin
  int32_t* p2p_small = nullptr;
  int32_t* p2p_large = nullptr;
  int p2p_nsmall = 0, p2p_nlarge = 0;
  int p2p_variant = 0;           // shape of the mixed P2P kernel (kP2PVariants): small leaves (or all)
  int p2p_big_variant = -1;      // shape for the large leaves' items (-1: p2p_variant)
  float p2p_bin_ms[2][FMM_P2P_VARIANTS] = {{0.f}};  // the last fmm_autotune's per-bin times
  // where the near-field branch starts in the evaluation graph: 0 with the
  // compressed M2L's expansion kernel, 1 at the start, beside the upward
  // pass, 2 with the projection (three projection stages), 3 as 2 with two
  // expansion stages (fmm_set_schedule)
  int p2p_sched = 0;
  float sched_ms[FMM_SCHED_CANDIDATES] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f};  // the last fmm_autotune's evaluation times
  double4* near64 = nullptr;
  double *stage_in = nullptr, *stage_out = nullptr;  // host-pointer staging
  int64_t stage_in_cap = 0, stage_out_cap = 0;
  double* stokes_buf = nullptr;  // fmm_evaluate_stokes: 4 passes' outputs, saved charges, forces, result
  int64_t stokes_cap = 0;
  bool skip_p2p = false;         // evaluations without the near field (the Stokes far-field passes)

  // scratch
  uint32_t* scratch = nullptr;
  int64_t scratch_cap = 0;  // in uint32 words
  double* box = nullptr;    // lo[3], W
  int32_t* counters = nullptr;   // device: [0..L) ncell, [16 + 8 l + c] class counts, [127] bad input
  void* pinned = nullptr;         // the handle's 1 KB slot of pinned host memory (below)
  int32_t* counters_h = nullptr; // pinned host mirror
  double* box_h = nullptr;       // pinned

  // tree
  LevelPtrs lv;
  int64_t lcap[FMM_MAX_LEVELS] = {0};  // capacity (cells) of the per-level arrays
  int32_t* slot_buf[FMM_MAX_LEVELS] = {nullptr};  // storage of lv.slot (set only for batched trees)
  int prev_leaf = -1;                  // leaf level of the previous tree (its grid entries get cleared)
  int32_t cls_off[FMM_MAX_LEVELS][9] = {{0}};
  int prev_ncell[FMM_MAX_LEVELS] = {0};
  bool have_prev = false;
  double box_host[4] = {0, 0, 0, 1};

  // batched problems (fmm_set_batch)
  bool forest = false;             // the current tree holds a batch
  int nprob = 0, fb_cap = 0, fb_bcap = 0;
  std::vector<int64_t> fb_start_h;   // [nprob + 1] input offsets
  std::vector<fmm::BatchProb> fb_prob_h;
  std::vector<int64_t> fb_first_h;   // [nprob] first Morton rank of each problem
  std::vector<double> fb_box_h;      // [nprob][4] after the build
  int64_t* fb_pstart = nullptr;      // [nprob + 1]
  fmm::BatchProb* fb_prob = nullptr; // [nprob]
  double* fb_box = nullptr;          // [nprob][4]: lo, W
  double* fb_scale = nullptr;        // [nprob]: lambda_k (output scale)
  double* fb_frame = nullptr;        // [nprob][4]: 2^-e, FP32 pair 2^L / (W 2^-e), 1 / W (W = m 2^e)
  int64_t* fb_thr = nullptr;         // cell thresholds, 3 << L per problem (BatchProb::thr)
  int64_t fb_thr_cap = 0;
  uint32_t* fb_sstart = nullptr;     // [nslot]: slot start keys, ascending
  int32_t* fb_sprob = nullptr;       // [nslot]: problem of each slot
  int32_t* fb_bstart = nullptr;      // [nprob + 1]: bounding-box blocks per problem (prefix)
  int fb_nslot = 0;
  int fb_nblocks = 0;                // bounding-box blocks of the batch

  // expansions
  int64_t rows = 0, rows_cap32 = 0, rows_cap64 = 0;  // buffers of one precision exist once it is used
  float *Mhi = nullptr, *Mlo = nullptr, *L32 = nullptr;
  double *M64 = nullptr, *L64 = nullptr;

  // M2L work
  Tile* tiles = nullptr;
  int ntiles = 0, tiles_cap = 0;
  int32_t* tile_src = nullptr;  // [tile][189][128]
  int16_t* tile_act = nullptr;  // [tile][189]
  int32_t* tile_nact = nullptr; // [tile]
  int16_t* src_act = nullptr;   // [tile][189]: indices into src_t of the tile's cells as sources with a target
  int32_t* src_nact = nullptr;  // [tile]
  uint32_t* tile_mask = nullptr; // [2][tile][6]: the setup's transfer-vector bit masks (targets, sources)
  int leaf_tiles = 0;           // tiles [0, leaf_tiles) belong to the leaf level
  int leaf_tile_end() const { return leaf_tiles; }

  // operators
  double* nodes64 = nullptr;   // [p]
  double* cheb64 = nullptr;    // [p][p]: T_n(xbar_m)
  float* cheb32 = nullptr;
  double* m2m64 = nullptr;     // [2][p][p]: S(xbar_m, (s + xbar_m')/2), s = -1, +1
  float* m2m32 = nullptr;
  int8_t* tvec = nullptr;      // [316][3]
  int16_t* cls_t = nullptr;    // [8][189] -> transfer vector index
  int16_t* src_t = nullptr;    // [8][189]: transfer vectors with which a source of the class serves a target
  double* K64 = nullptr;       // [banks][316][C][C]
  float *Khi = nullptr, *Klo = nullptr;  // [banks][316][cpad][cpad], TF32 split
  bool ops64 = false, ops32 = false;
  bool ops32_f16 = false;   // the mixed banks hold FP16 hi/lo pairs (tensor-core FP16 form), scaled by ops_kscale
  float ops_kscale = 1.f;
  uint32_t* tc_mmax = nullptr;  // full-rank FP16 form: max |M| per (problem + 1, level)
  // banks: 1 (homogeneous kernel), or one per level 2..leaf (c > 0), built for
  // root width ops*_W (c > 0 only)
  int ops64_nb = 0, ops32_nb = 0;
  double ops64_W = 0.0, ops32_W = 0.0;

  // evaluation schedule
  std::vector<int64_t> graph_sig;  // what the captured graph depends on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_fallbacks = 0;  // evaluations run without a graph after a failed capture
  bool graph_ok = false;
  int graph_precision = -1;
  bool use_graph = true;
  bool p2p_priority = true;  // P2P graph nodes at the low launch priority (the rest high)
  int timing = 0;  // 0 off, 1 events in the overlapped schedule, 2 events with P2P run alone
  cudaEvent_t tev[14] = {nullptr};  // [9..12]: around the tensor-core M2L kernels
  bool tev_recorded = false;

  // tensor-core M2L
  bool use_tc = true;
  float* tc_partial = nullptr;
  int64_t tc_partial_cap = 0;
  int32_t* tc_err = nullptr;      // device error word of the tensor-core kernel
  int32_t* tc_err_h = nullptr;    // pinned mirror, copied after every evaluation
  uint64_t wait_ns = 2000000000ull;  // limit of each pipeline wait of the tensor-core kernels (fmm_set_wait_limit)
  alignas(64) unsigned char tm_khi[128], tm_klo[128];  // CUtensorMap of the operator bank
  int64_t tm_rows = -1;
  alignas(64) unsigned char tm_vthi[128], tm_vtlo[128], tm_uhi[128], tm_ulo[128];  // compressed banks
  const void* tm_svd_ptr = nullptr;
  int svd_tc_nst = 0;
  float* svd_Mcls = nullptr;       // multipoles in class order, interleaved hi/lo slabs
  int svd_mcbase[FMM_MAX_LEVELS][8] = {{0}};  // first row of each (level, class) segment
  int64_t svd_mcls_rows = 0;
  void* svd_recs = nullptr;      // projection work units (records of k_svd_groups)
  int16_t* svd_eslot = nullptr;  // expansion tables (k_svd_exp_setup)
  int8_t* svd_ekch = nullptr;
  int64_t* svd_yidx = nullptr;
  int64_t svd_ecap = 0;
  int64_t svd_gcap = 0;
  const void* tm_khi_ptr = nullptr;
  int tm_khi_nb = 0;
  bool tm_khi_f16 = false;
  int tc_nst = 0, num_sms = 0;

  // SVD-compressed M2L (m2l_svd.cu)
  int m2l_method = FMM_M2L_SVD;
  double svd_eps = 0.0;       // <= 0: 10^-order
  bool svd_ready = false, svd64 = false, svd32 = false;
  double svd_eps_used = 0.0;
  int64_t svd_gen = 0;
  int svd_rank[16] = {0};
  int t_rank_h[FMM_NT] = {0};
  int svd_rmax = 0, svd_rp = 0;
  double *svd_W = nullptr, *svd_Z = nullptr, *svd_vals = nullptr, *svd_colmean = nullptr;
  int32_t *svd_ord = nullptr, *svd_rank_d = nullptr, *svd_sweeps_d = nullptr;
  int16_t* svd_sm = nullptr;
  int8_t *svd_canon = nullptr, *svd_tcanon = nullptr;
  double *svd_V64 = nullptr, *svd_U64 = nullptr;  // [316][C][rmax]
  size_t svd_bank64_bytes = 0;
  float* svd_VThi = nullptr;  // mixed projection factors, interleaved hi/lo slabs per class (m2l_svd.cu)
  float* svd_Uhi = nullptr;   // mixed expansion factors, interleaved hi/lo slabs, mean-split
  size_t svd_vt_bytes = 0, svd_u_bytes = 0;
  // compressed tensor-core M2L with FP16 hi/lo operands (m2l_f16): the mixed
  // banks' format, their scales, and per-level max |M| and |Y| (device words)
  bool m2l_f16 = false, svd_bank_f16 = false;
  float svd_vscale = 1.f, svd_uscale = 1.f;
  uint32_t* svd_umax = nullptr;  // max |Y| per (problem + 1, level): [FMM_MAX_BATCH + 1][FMM_MAX_LEVELS]
  float* svd_mscale = nullptr;   // scale of each class-ordered multipole row (FP16 operands)
  // FP16 tensor-core form (svd_wants_f16): ranks padded to 8; the projection
  // writes y straight into the expansion's operand layout Yx ([tile][kc][128
  // rows], interleaved FP16 hi/lo 64-byte rows), through the destination map
  // dst[src-list index][expansion row] = tile * 128 + row (-1: no target);
  // the expansion's factor bank Uc is U per target class along the class's
  // concatenated ranks (kap8: start of t's ranks / 8 per target class, kt8:
  // the class's total / 8, kct: 32-value chunks per tile row).
  void* svd_Yx = nullptr;
  size_t svd_Yx_cap = 0;
  int32_t* svd_dst = nullptr;
  size_t svd_dst_cap = 0;
  int16_t* svd_kap8 = nullptr;    // [8][316], -1 if t is not in the class's list
  int16_t* svd_srcidx = nullptr;  // [8][316]: index of t in the source class's list, -1 if none
  int svd_kt8 = 0, svd_kct = 0;
  uint32_t* svd_Uc = nullptr;
  size_t svd_uc_bytes = 0;
  int svd_x_groups = 0;           // K groups of the last expansion launch (partial slices per tile)
  std::vector<int32_t> svd_yoff_h;
  int32_t *svd_ry = nullptr, *svd_trank = nullptr, *svd_yoff = nullptr;  // [316], [316], [8][316]
  int64_t svd_YS = 0;            // Y values per cell row
  void* svd_Y = nullptr;         // Y[row][YS]: the projections of each cell's M, row = the expansion row
  size_t svd_Y_cap = 0;
  std::vector<int64_t> svd_ysig;
  std::vector<Tile> tiles_h;     // host copy of the M2L tiles
  std::vector<int16_t> cls_t_h;  // host copy of cls_t
  std::vector<int16_t> src_t_h;  // host copy of src_t
  int64_t tree_gen = 0;          // bumped by every tree build

  // stats
  int64_t launches_set = 0, launches_eval = 0, bytes = 0;
};

namespace fmm {

using Ctx = ::fmm_ctx;

// ---- error plumbing --------------------------------------------------------
fmm_status set_err(Ctx* c, fmm_status s, const char* fmt, ...);
fmm_status cuda_err(Ctx* c, cudaError_t e, const char* what);
#define FMM_CUDA(c, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_err((c), e_, #call); \
  } while (0)
#define FMM_TRY(expr)               \
  do {                              \
    fmm_status s_ = (expr);         \
    if (s_ != FMM_OK) return s_;    \
  } while (0)

fmm_status dalloc(Ctx* c, void** p, size_t bytes);
// a block of the library's device pool, ready for any stream when it returns
cudaError_t pool_alloc(int dev, cudaStream_t s, void** p, size_t bytes);
fmm_status raise_smem_limit(Ctx* c, const void* func, int bytes);
void dfree(Ctx* c, void* p, size_t bytes);

// ---- stages (host launchers) -------------------------------------------------
fmm_status tree_build(Ctx* c, int64_t n, const double* xyz, const double* q);
// expansion buffers of one precision for the current tree's rows (new buffers start at zero)
fmm_status ensure_expansions(Ctx* c, int precision);
// releases every buffer that depends on the tree (the operators stay)
void release_tree(Ctx* c);
// slot of every problem of a batch (host only): first leaf key, slot level, batch leaf level; -1 if too big
int batch_plan(int nprob, const int64_t* counts, const int32_t* heights, int64_t* slot, int64_t* level, int* leaf);
// slots of a batch (sets c->forest, c->leaf and the device tables); *n_total = sum of counts
fmm_status batch_layout(Ctx* c, int nprob, const int64_t* counts, const int32_t* heights, int64_t* n_total);
fmm_status operators_init(Ctx* c);
fmm_status operators_m2l(Ctx* c, int precision);
fmm_status launch_p2p(Ctx* c, cudaStream_t s);
// one occupancy bin of the mixed near field (0: leaves of at most P2P_BIG particles, 1: larger) in shape v
fmm_status launch_p2p_bin(Ctx* c, cudaStream_t s, int bin, int v);
bool is_p2p_kernel(const void* func);
void p2p_carveout();
extern const int kP2PVariants[FMM_P2P_VARIANTS][4];
fmm_status launch_upward(Ctx* c, cudaStream_t s, cudaEvent_t after_p2m = nullptr);  // P2M + M2M
fmm_status launch_m2l_simt(Ctx* c, cudaStream_t s, int first_tile, int ntiles);
fmm_status svd_prepare(Ctx* c);        // SVD of the canonical operators (ranks to the host)
fmm_status m2l_svd_prepare(Ctx* c);    // + factor banks and the Y layout of the current tree
fmm_status launch_m2l_svd_simt(Ctx* c, cudaStream_t s, int first_tile, int ntiles);
bool m2l_tc_supported(const Ctx* c);
fmm_status m2l_tc_prepare(Ctx* c);
fmm_status launch_m2l_tc(Ctx* c, cudaStream_t s, cudaEvent_t mid);
fmm_status launch_m2l_tc_reduce(Ctx* c, cudaStream_t s, const float* partial, int gt);
bool m2l_svd_tc_supported(const Ctx* c);
fmm_status m2l_svd_tc_prepare(Ctx* c);
fmm_status launch_m2l_svd_tc(Ctx* c, cudaStream_t s, cudaEvent_t mid);
// M2L of every level; `mid` separates the main kernel from the rest (see fmm_get_stage_times)
fmm_status launch_m2l(Ctx* c, cudaStream_t s, cudaEvent_t mid);
fmm_status launch_m2l_prep(Ctx* c, cudaStream_t s);
bool m2l_has_prep(const Ctx* c);
bool svd_leaf_gather_apart(const Ctx* c);                  // the leaf-level gather may run beside M2M
fmm_status launch_svd_leaf_gather(Ctx* c, cudaStream_t s);  // it, on s (records ev_gleaf)
fmm_status svd_tree_setup(Ctx* c, cudaStream_t s);
bool svd_has_tree_setup(const Ctx* c);
fmm_status launch_l2l(Ctx* c, cudaStream_t s);
fmm_status launch_l2p_out(Ctx* c, cudaStream_t s, double* phi, double* F);
fmm_status expansion_to_f64(Ctx* c, int level, int which, double* out);
int64_t count_launches_eval(const Ctx* c);
fmm_status work_counts(Ctx* c, int64_t* out);
// 0 FP64 SIMT, 1 FP32 SIMT, 2 tcgen05 (full-rank operators); 3 FP64 SIMT, 4 FP32 SIMT,
// 5 tcgen05 (SVD-compressed)
int m2l_kind(const Ctx* c);
// Stokes from four 1/r passes (stokes.cu)
fmm_status launch_stokes_save(Ctx* c, double* q0);
fmm_status launch_stokes_charges(Ctx* c, const double* f, const double* q0, int j);
fmm_status launch_stokes_combine(Ctx* c, const double* phi4, const double* F4, const float4* unear, double* u);
fmm_status launch_stokes_forces(Ctx* c, const double* f, float4* f32);
fmm_status launch_p2p_stokes(Ctx* c, cudaStream_t s, const float4* f32, float4* out);
// The compressed operators need one operator set for every level: c = 0.
inline bool uses_svd(const Ctx* c) { return c->m2l_method == FMM_M2L_SVD && c->kernel_c == 0.0; }
// The compressed tensor-core M2L takes FP16 hi/lo operands (m2l_f16), scaled
// per multipole row and per (problem, level), for single problems and
// batches alike.
inline bool m2l_uses_f16(const Ctx* c) { return c->m2l_f16; }
// The mixed compressed factor banks are FP16 hi/lo pairs (the tensor-core
// kernels' FP16 form) or TF32 hi/lo pairs.
bool svd_wants_f16(const Ctx* c);
// Full-rank operator banks: one, or one per level 2..leaf when c > 0.
inline int op_banks(const Ctx* c) { return c->kernel_c > 0.0 && c->leaf > 2 ? c->leaf - 1 : 1; }

// ---- device helpers ----------------------------------------------------------
// Spreads the low 10 bits of v so that bit b lands at bit 3b.
__host__ __device__ inline uint32_t spread3(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ inline uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030C30C3u;
  v = (v | (v >> 4)) & 0x0300F00Fu;
  v = (v | (v >> 8)) & 0x030000FFu;
  v = (v | (v >> 16)) & 0x000003FFu;
  return v;
}
// Morton key with x the most significant bit of each (x, y, z) triple.
__host__ __device__ inline uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}
__host__ __device__ inline void demorton3(uint32_t k, int& x, int& y, int& z) {
  x = (int)compact3(k >> 2);
  y = (int)compact3(k >> 1);
  z = (int)compact3(k);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Bounds checks of the debug build (FMM_DEBUG; fmm_debug_check).  FMM_GUARD(
// cond, site, idx) is `cond`: in the debug build a false condition also
// records (site << 32 | idx) in this file's first-failure word, and callers
// skip the access it guards; in the normal build it is `true` and costs
// nothing.  The words are per compilation unit (no relocatable device code),
// each read and cleared by its file's fmm_debug_take_<file>().
#ifdef FMM_DEBUG
static __device__ unsigned long long g_fmm_first_failure;
__device__ __forceinline__ bool fmm_guard(bool cond, unsigned site, unsigned idx) {
  if (!cond) atomicCAS(&g_fmm_first_failure, 0ull, ((unsigned long long)site << 32) | idx);
  return cond;
}
#define FMM_GUARD(cond, site, idx) fmm_guard((cond), (site), (unsigned)(idx))
#define FMM_DEBUG_TAKE_FN(name)                                                                      \
  unsigned long long name() {                                                                       \
    unsigned long long v = 0, z = 0;                                                                \
    if (cudaMemcpyFromSymbol(&v, g_fmm_first_failure, sizeof(v)) != cudaSuccess ||                \
        cudaMemcpyToSymbol(g_fmm_first_failure, &z, sizeof(z)) != cudaSuccess) {                   \
      cudaGetLastError();                                                                           \
      return ~0ull;                                                                                 \
    }                                                                                               \
    return v;                                                                                       \
  }
#else
#define FMM_GUARD(cond, site, idx) true
#define FMM_DEBUG_TAKE_FN(name) \
  unsigned long long name() { return 0ull; }
#endif
// check sites (the high word of a recorded failure)
enum : unsigned {
  CHK_GATHER_INDEX = 1,      // k_gather: the sorted index of a particle outside [0, n)
  CHK_LEVEL_CELL = 2,        // k_lv_write: a cell index below 0
  CHK_P2P_SOURCE = 3,        // near field: a staged source outside its neighbour leaf's range
  CHK_SETUP_KEY = 4,         // M2L tile setup: a neighbour key outside the level's grid
  CHK_SCATTER_DST = 5,       // compressed M2L setup: a destination-map index outside the map
  CHK_PROJ_DST = 6,          // compressed M2L projection: a destination row outside the expansion operand
};
unsigned long long fmm_debug_take_tree();
unsigned long long fmm_debug_take_nearfield();
unsigned long long fmm_debug_take_m2l_svd_tc();

// An NVTX range over a scope ("fmm:<stage>"): the API calls and the stages
// of an evaluation show up by name in a profiler's timeline (NVTX v3 is
// header-only; without a tool attached a range costs a branch).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace fmm
