// m2l_svd_tc.cu -- the SVD-compressed M2L (Sec. 2.1.2, "Improved M2L
// operator"; the factors are those of m2l_svd.cu) on the sm_103a tensor
// cores, mixed precision: three products hi*hi + hi*lo + lo*hi of split
// operands, FP16 hi/lo pairs (the default, kind::f16) or TF32 hi/lo pairs
// (FMM_M2L_MATH=tf32, kind::tf32).
//
// k_svd_proj_tc -- projection from the sources.  Work unit = (tile of 128
//   cells of one level and class, group of consecutive active source
//   transfer vectors whose padded ranks add up to at most SP_ACC columns).
//   A = the tile's multipoles (K = the cpad coefficients) from a
//   class-ordered, pre-swizzled copy of M; B = the group's V_t factors
//   stacked (VT bank rows, pre-swizzled); every slab arrives by one linear
//   bulk copy, and one MMA of N = the group's columns computes every product
//   of the group.  Each t owns a column range of the TMEM accumulator (two
//   buffers of SP_ACC columns alternate between units).  The epilogue:
//     FP16 form: each y_(S,t) goes straight into the expansion's operand
//       layout Yx -- the target T = S - t's tile row, at t's place in T's
//       class's concatenated ranks -- scaled by the power of two of the
//       (problem, level) bound ||M||_2 and split into FP16 hi/lo; the
//       destination comes from a map built per evaluation
//       (k_svd_scatter_setup), which also zeroes the rows of targets
//       without a source for t;
//     TF32 form: the cells' FP32 Y rows.
// k_svd_expand16_tc -- FP16 expansion at the targets: work unit = (K group,
//   target tile, column half); A = the tile's Yx slab, B = the class's factor
//   bank Uc along the same concatenated K, one bulk copy each per 32 values
//   of K.
// k_svd_expand_tc -- TF32 expansion: work unit = (target tile, column half,
//   group of EX_GT active transfer vectors); A gathered from the sources' Y
//   rows and split into TF32 hi/lo on the way into tensor memory, B = U_t.
// Both expansions: the tensor cores' FP32 accumulation does not round to
// nearest, so an accumulator takes a chain of about order^3 values of K (the
// chain of one full-rank operator) before the epilogue adds it into FP32
// running sums in shared memory; k_m2l_tc_reduce adds a tile's group slices
// and scales by 1/a.
// Roles per CTA (one CTA per SM, persistent): producers (one bulk-copy
// thread; the TF32 expansion: warps in sets of four, one thread per row),
// four epilogue warps (one per TMEM lane quarter), one MMA warp (one elected
// thread issues).  Every mbarrier wait is bounded in time (fmm_set_wait_limit);
// on expiry the CTA raises the error word, drains what it has in flight
// (bounded), frees TMEM and returns.
#include "tc_ptx.cuh"

namespace fmm {

using namespace tc;

namespace {

constexpr int KC = 16;          // K elements per pipeline stage (64-byte rows)
constexpr int MAXST = 4;        // pipeline stages at most

// ---- projection -------------------------------------------------------------
constexpr int SP_PROD = 0;                    // TMA producer warp (one thread issues)
constexpr int SP_MMA = 1;                     // the MMA warp
constexpr int SP_EPI = 2;                     // first of the eight epilogue warps (two per TMEM lane quarter)
constexpr int SP_NEPI = 8;
constexpr int SP_THREADS = 32 * (SP_EPI + SP_NEPI);
constexpr int SP_ACC = 256;                   // accumulator columns per buffer (two buffers: all of TMEM)
constexpr int SP_MAXG = SP_ACC / 16;          // transfer vectors per group at most (ranks >= 16)
constexpr int SP_A_BYTES = FMM_TILE * KC * 4; // one half (hi or lo) of a stage's A: 8 KB
constexpr int SP_B_BYTES = SP_ACC * KC * 4;   // one half of a stage's B: 16 KB

// One projection unit: a tile and a group of its active source transfer
// vectors (consecutive, sum of ranks <= SP_ACC columns), written by
// k_svd_groups so that the kernel's roles read one 64-byte record per unit
// instead of chains of dependent index loads.
struct __align__(16) ProjRec {
  int32_t crow;            // row_off[level]: cell rows are crow + cls[level][first + r]
  int32_t first;           // the tile's first position in the level's class list
  int32_t arow;            // the tile's first row in the class-ordered multipole copy
  int16_t count;           // cells in the tile
  int8_t cls, level, n;    // child class, level, transfer vectors in the group (0: no unit)
  uint8_t cols8;           // sum of the padded ranks / 8 (the MMA's N is this x 8 rounded up to 16)
  int16_t yo8[SP_MAXG];    // their Y offsets in the class's rows / 8 (= their factor rows)
  uint8_t ry8[SP_MAXG];    // their padded ranks / 8
  uint8_t kidx[SP_MAXG];   // their index in the source class's list (src_t)
  int16_t kap8[SP_MAXG];   // FP16 form: start of their ranks in the target class's concatenated K, / 8
  uint8_t pad[14];
};
static_assert(sizeof(ProjRec) == 128, "one record = 128 bytes");

// Where each (level, class) segment of the class-ordered multipole copy
// starts (multiples of 128 rows, so that every tile starts a swizzle block).
struct McBase {
  int base[FMM_MAX_LEVELS][8];
  int clsoff[FMM_MAX_LEVELS][8];
};

struct ProjArgs {
  const ProjRec* recs;   // the units, compact, a tile's groups one after another (CTAs running at
                         // the same time share a tile's multipoles in L2)
  const int32_t* nunits; // their number
  float* Y;              // TF32 form: the sources' Y rows
  // FP16 form: y goes to the expansion's operand layout Yx through the
  // destination map dst[src-list index][expansion row] (tile * 128 + row of
  // the target, -1: none), scaled by pow2_scale of the bound ||M||_2 of its
  // (problem, level) (ybound)
  uint32_t* Yx;
  const int32_t* dst;
  int64_t drows;
  int kct;
  const uint32_t* ybound;
  int32_t* err;
  int64_t YS;
  int64_t mrows;         // rows of the class-ordered multipole copy per chunk of coefficients
  const float *Mc, *VT;  // interleaved hi/lo slabs (il_idx)
  int ntiles, ngroups, kchunks, nst;
  // FP16 operands: each class-ordered multipole row's scale (pow2_scale of
  // the cell's max |M|) and the VT bank's scale, undone in the epilogue
  const float* mscale;
  float vscale;
  uint64_t wait_ns;      // limit of a pipeline wait (fmm_set_wait_limit)
};

// Slot of a per-(problem, level) value (the FP16 form's bound of |y|):
// problem -1 (cells above a batch's problem slots) first.
__host__ __device__ inline int ymax_index(int prob, int level) { return (prob + 1) * FMM_MAX_LEVELS + level; }

// Greedy grouping of each tile's active source transfer vectors into units
// (every record of the tile is written, n = 0 past the last group).  One
// block per tile: the threads fetch the ranks and offsets, one thread draws
// the group boundaries, the threads write the records.
__global__ void __launch_bounds__(256)
k_svd_groups(int ntiles, int ngroups, const Tile* __restrict__ tiles, LevelPtrs lv, McBase mb,
             const int16_t* __restrict__ src_act, const int32_t* __restrict__ src_nact,
             const int16_t* __restrict__ src_t, const int32_t* __restrict__ t_ry,
             const int32_t* __restrict__ yoff, const int8_t* __restrict__ tvec, const int16_t* __restrict__ kap8,
             ProjRec* __restrict__ recs, int32_t* __restrict__ nunits, int32_t* __restrict__ err) {
  __shared__ int16_t s_kap8[FMM_NT_CLASS];
  __shared__ int16_t s_yo8[FMM_NT_CLASS];
  __shared__ uint8_t s_ry8[FMM_NT_CLASS];
  __shared__ uint8_t s_kidx[FMM_NT_CLASS];
  __shared__ int16_t s_gs[FMM_NT_CLASS + 2];
  __shared__ int s_ng, s_base;
  const int tile = blockIdx.x;
  const Tile tl = tiles[tile];
  const int nact = src_nact[tile];
  for (int a = threadIdx.x; a < nact; a += blockDim.x) {
    const int k = src_act[(int64_t)tile * FMM_NT_CLASS + a];
    const int slot = src_t[tl.cls * FMM_NT_CLASS + k];
    s_kidx[a] = (uint8_t)k;
    s_ry8[a] = (uint8_t)(t_ry[slot] / 8);
    s_yo8[a] = (int16_t)(yoff[tl.cls * FMM_NT + slot] / 8);
    // the targets' class: the source's with the parities of t flipped
    const int ct = tl.cls ^ (((tvec[3 * slot] & 1) << 2) | ((tvec[3 * slot + 1] & 1) << 1) | (tvec[3 * slot + 2] & 1));
    s_kap8[a] = kap8 ? kap8[ct * FMM_NT + slot] : (int16_t)-1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0, cols = 0, members = 0;
    for (int a = 0; a < nact; ++a) {
      const int ry = 8 * s_ry8[a];
      if (a == 0 || cols + ry > SP_ACC || members == SP_MAXG) {
        s_gs[n++] = (int16_t)a;
        cols = 0;
        members = 0;
      }
      cols += ry;
      ++members;
    }
    s_gs[n] = (int16_t)nact;
    if (n > ngroups) atomicOr(err, 2);  // more groups than the bound (cannot happen by construction)
    n = min(n, ngroups);
    s_ng = n;
    // the tile's units go to consecutive records of the compact list
    s_base = n > 0 ? atomicAdd(nunits, n) : 0;
  }
  __syncthreads();
  const int ng = s_ng;
  for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
    ProjRec r;
    r.crow = (int32_t)lv.row_off[tl.level];
    r.first = tl.first;
    r.arow = mb.base[tl.level][tl.cls] + (tl.first - mb.clsoff[tl.level][tl.cls]);
    r.count = (int16_t)tl.count;
    r.cls = (int8_t)tl.cls;
    r.level = (int8_t)tl.level;
    int n = 0, cols = 0;
    if (gi < ng) {
      const int a0 = s_gs[gi], a1 = s_gs[gi + 1];
      for (int a = a0; a < a1; ++a, ++n) {
        r.ry8[n] = s_ry8[a];
        r.yo8[n] = s_yo8[a];
        r.kidx[n] = s_kidx[a];
        r.kap8[n] = s_kap8[a];
        cols += 8 * s_ry8[a];
      }
    }
    r.n = (int8_t)n;
    r.cols8 = (uint8_t)(cols / 8);
    recs[s_base + gi] = r;
  }
}

// The multipoles of each level in class order (the order of lv.cls), each
// (level, class) segment starting at a multiple of 128 rows, so that the 128
// cells of a tile are 128 consecutive rows of a swizzle-aligned slab:
// Mc row (kc * rows + base[l][c] + j - clsoff[l][c]) = coefficients 16 kc ..
// 16 kc + 15 of M[row_off + cls[j]], hi and lo interleaved (il_idx).  One
// block per cell.
__global__ void k_gather_cls(int l, LevelPtrs lv, McBase mb, int cpad, int64_t rows, const float* __restrict__ Mhi,
                             const float* __restrict__ Mlo, float* __restrict__ Mc) {
  const int j = blockIdx.x;
  const int cell = lv.cls[l][j];
  const int c = lv.key[l][cell] & 7;
  const int64_t row = mb.base[l][c] + (j - mb.clsoff[l][c]), src = (lv.row_off[l] + cell) * cpad;
  for (int k = threadIdx.x; k < cpad; k += blockDim.x) {
    const int64_t G = (int64_t)(k >> 4) * rows + row;
    Mc[il_idx(G, 0, k & 15)] = Mhi[src + k];
    Mc[il_idx(G, 1, k & 15)] = Mlo[src + k];
  }
}

// k_gather_cls with FP16 operands: the same rows, 32 coefficients per row
// (chunk kc = k / 32), two per 32-bit word, scaled by pow2_scale of the
// cell's own max |M| (recorded per row for the projection's epilogue).  A
// warp per cell (four per block), a lane per pair of coefficients k, k + 1
// (k = 2 lane + 64 i), each read once into registers.
// ybound (FP16 form, may be NULL): the largest ||M_S||_2 of every (problem,
// level), by atomic max.  A projection y = V^T M_S has |y_i| <= ||M_S||_2
// (V has orthonormal columns), so a power of two taken from this bound keeps
// every projection of the (problem, level) inside the FP16 range before the
// projection runs.
constexpr int GC_PAIRS = 8;  // pairs per lane: cpad <= 512

__global__ void __launch_bounds__(128)
k_gather_cls16(int l, int ncell, LevelPtrs lv, McBase mb, int cpad, int64_t rows, const float* __restrict__ Mhi,
               const float* __restrict__ Mlo, uint32_t* __restrict__ Mc, float* __restrict__ mscale,
               uint32_t* __restrict__ ybound) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (j >= ncell) return;
  const int cell = lv.cls[l][j];
  const int c = lv.key[l][cell] & 7;
  const int64_t row = mb.base[l][c] + (j - mb.clsoff[l][c]), src = (lv.row_off[l] + cell) * cpad;
  float2 v[GC_PAIRS];
  float m = 0.f, sq = 0.f;
#pragma unroll
  for (int i = 0; i < GC_PAIRS; ++i) {
    const int k = 2 * lane + 64 * i;
    v[i] = make_float2(0.f, 0.f);
    if (k < cpad) {
      const float2 h = *(const float2*)&Mhi[src + k], o = *(const float2*)&Mlo[src + k];
      v[i] = make_float2(h.x + o.x, h.y + o.y);
      m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
      sq = fmaf(v[i].x, v[i].x, fmaf(v[i].y, v[i].y, sq));
    }
  }
  const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));  // non-negative floats order like bits
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  const float sc = pow2_scale(__uint_as_float(wm));
  if (lane == 0) mscale[row] = sc;
  if (lane == 0 && ybound) {
    // the norm rounded up a little (FP32 sums of 343 squares): a bound, not an estimate
    const float nrm = sqrtf(sq) * 1.001f;
    atomicMax(ybound + ymax_index(problem_of(lv, l, cell), l), __float_as_uint(nrm));
  }
#pragma unroll
  for (int i = 0; i < GC_PAIRS; ++i) {
    const int k = 2 * lane + 64 * i;
    if (k < cpad) {
      const int64_t G = (int64_t)(k >> 5) * rows + row;
      uint32_t hi, lo;
      split_h2(v[i].x * sc, v[i].y * sc, hi, lo);
      const int w = (k & 31) >> 1;
      Mc[il_idx(G, 0, w)] = hi;
      Mc[il_idx(G, 1, w)] = lo;
    }
  }
}

__device__ inline ProjRec load_rec(const ProjRec* p) {
  ProjRec r;
  const int4* s = (const int4*)p;
  int4* d = (int4*)&r;
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = s[i];
  return r;
}

__device__ inline void st_cs_v4(float* p, float a, float b, float c, float d) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
// 32 / 16 bytes, streaming (the projection's Yx rows are read once, by the
// expansion); the address must be 32 / 16-byte aligned.
__device__ inline void st_cs_u8(uint32_t* p, const uint32_t* v) {
  asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(v[0]), "r"(v[1]),
               "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ inline void st_cs_u4(uint32_t* p, const uint32_t* v) {
  asm volatile("st.global.cs.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

// F16: operands are FP16 hi/lo pairs (32 coefficients per 64-byte row, one
// MMA of K = 16 per half row, at twice the TF32 rate; M scaled per level, VT
// by vscale, both undone exactly in the epilogue); otherwise TF32 hi/lo.
template <bool F16>
__global__ void __launch_bounds__(SP_THREADS, 1)
k_svd_proj_tc(ProjArgs a, LevelPtrs lv) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  // stage s: A (128 rows, hi/lo interleaved) | B (stacked factor rows, hi/lo interleaved)
  const uint32_t stage_bytes = 2u * SP_A_BYTES + 2u * SP_B_BYTES;
  const uint32_t bars = base + (uint32_t)a.nst * stage_bytes;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (MAXST + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * MAXST + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * MAXST + 2 + b); };
  const uint32_t mma_done = bars + 8u * (2 * MAXST + 4);
  unsigned char* gbase = smem_raw + (base - raw);
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(gbase + (bars - base) + 8u * (2 * MAXST + 6));
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const uint32_t tmem_cols = 2u * SP_ACC;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // FP16 form: per epilogue warp, each lane's destinations for the unit's t [q][lane]
  int32_t* epi_dst = (int32_t*)(gbase + (bars - base) + 256) + (warp - SP_EPI) * (SP_MAXG * 32);
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXST; ++s) {
      mbar_init(full(s), 1);  // the producer's expect_tx
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), 32 * SP_NEPI);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == SP_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nunits = *a.nunits;  // the compact list's length (k_svd_groups)

  if (warp == SP_PROD) {
    // ---------------------------------------------------------- copy producer
    // per stage: the tile's slab of 16 coefficients (128 rows, one copy) and
    // the group's factor rows (one copy per run of transfer vectors that are
    // consecutive in the class's rows), issued by lanes after lane 0 has
    // posted the stage's byte count
    uint32_t it = 0, last = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      const ProjRec g = load_rec(a.recs + unit);
      if (g.n == 0) continue;
      // lane q < n: the run of transfer vectors starting at q (if one starts there)
      int off = 0, run = 0;
      bool starts = false;
      if (lane < g.n) {
        for (int q = 0; q < lane; ++q) off += 8 * g.ry8[q];
        starts = lane == 0 || g.yo8[lane] != g.yo8[lane - 1] + g.ry8[lane - 1];
        if (starts) {
          int q = lane;
          do {
            run += 8 * g.ry8[q];
            ++q;
          } while (q < g.n && g.yo8[q] == g.yo8[q - 1] + g.ry8[q - 1]);
        }
      }
      for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
        const int s = (int)(it % a.nst);
        const uint32_t ph = (it / a.nst) & 1u;
        if (!warp_wait(empty(s), ph ^ 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        const uint32_t st = base + (uint32_t)s * stage_bytes;
        const uint32_t sb = st + 2u * SP_A_BYTES;
        if (lane == 0) mbar_expect_tx(full(s), 2u * SP_A_BYTES + (uint32_t)g.cols8 * 8u * 128u);
        __syncwarp();
        if (lane == SP_MAXG) {
          bulk_g2s(st, a.Mc + ((int64_t)kc * a.mrows + g.arow) * 32, 2u * SP_A_BYTES, full(s));
        } else if (starts) {
          const int64_t G = ((int64_t)g.cls * a.kchunks + kc) * a.YS + 8 * g.yo8[lane];
          bulk_g2s(sb + (uint32_t)off * 128u, a.VT + G * 32, (uint32_t)run * 128u, full(s));
        }
        last = it + 1;
      }
    }
    if (!ok) {
      if (lane == 0) {
        *abort_flag = 1;
        atomicOr(a.err, 1);
        // let the copies already issued land before the CTA leaves (bounded)
        for (uint32_t j = last > (uint32_t)a.nst ? last - a.nst : 0; j < last; ++j)
          mbar_wait(full((int)(j % a.nst)), (j / a.nst) & 1u);
      }
    }
    __syncwarp();
  } else if (warp == SP_MMA) {
    // ---------------------------------------------------------- MMA issuer
    uint32_t it = 0, uu = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      // N: the group's columns rounded up to the MMA granule of 16 (the rows past
      // the group's in the stage are stale; their columns are never read)
      const int n = a.recs[unit].n, cols = (8 * a.recs[unit].cols8 + 15) / 16 * 16;
      if (n == 0) continue;
      const int b = (int)(uu & 1u);
      if (!warp_wait(acc_empty(b), ((uu >> 1) & 1u) ^ 1u, abort_flag, a.wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d0 = tmem + (uint32_t)(b * SP_ACC);
      // the group's factors are stacked in the stage, so one MMA of
      // N = sum of the ranks covers every transfer vector of the group
      const uint32_t idesc = F16 ? idesc_f16(FMM_TILE, cols) : idesc_tf32(FMM_TILE, cols);
      for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
        const int s = (int)(it % a.nst);
        const uint32_t ph = (it / a.nst) & 1u;
        if (!warp_wait(full(s), ph, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t st = base + (uint32_t)s * stage_bytes;
          const uint32_t sb = st + 2u * SP_A_BYTES;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ahi = sdesc_sw64s(st + ks * 32u, 1024), alo = sdesc_sw64s(st + 512u + ks * 32u, 1024);
            const uint64_t bhi = sdesc_sw64s(sb + ks * 32u, 1024), blo = sdesc_sw64s(sb + 512u + ks * 32u, 1024);
            if (F16) {
              mma_f16(d0, ahi, bhi, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
              mma_f16(d0, ahi, blo, idesc, 1u);
              mma_f16(d0, alo, bhi, idesc, 1u);
            } else {
              mma_tf32(d0, ahi, bhi, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
              mma_tf32(d0, ahi, blo, idesc, 1u);
              mma_tf32(d0, alo, bhi, idesc, 1u);
            }
          }
          mma_commit(empty(s));
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(acc_full(b));
      __syncwarp();
      ++uu;
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
    if (lane == 0) {
      mma_commit(mma_done);
      mbar_wait(mma_done, 0);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    // TMEM lane quarter = warp % 4; row = the cell's position in the tile; the
    // two warps of a quarter take the group's transfer vectors in turn (half)
    const int qd = warp & 3, row = qd * 32 + lane, half = (warp - SP_EPI) >> 2;
    uint32_t uu = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      const ProjRec g = load_rec(a.recs + unit);
      if (g.n == 0) continue;
      const bool valid = row < g.count;
      const int cell = valid ? lv.cls[g.level][g.first + row] : 0;
      const int64_t cellrow = (int64_t)g.crow + cell;
      float f = 0.f;
      if (F16) {
        // read while the unit's MMAs run: the destinations of this row's
        // projections (the target's tile row per t) and the factor that takes
        // y back from the operand scales into the scale of the (problem,
        // level) bound (powers of two: exact)
        for (int q = half; q < g.n; q += 2)
          epi_dst[q * 32 + lane] = valid ? a.dst[(int64_t)g.kidx[q] * a.drows + cellrow] : -1;
        if (valid)
          f = pow2_scale(__uint_as_float(a.ybound[ymax_index(problem_of(lv, g.level, cell), g.level)])) /
              (a.mscale[g.arow + row] * a.vscale);
      }
      const int b = (int)(uu & 1u);
      if (!warp_wait(acc_full(b), (uu >> 1) & 1u, abort_flag, a.wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * SP_ACC);
      __syncwarp();
      int off = 0;  // the group's columns before t
      for (int q = 0; q < g.n; ++q) {
        const int c0 = off, c1 = off + 8 * g.ry8[q];
        off = c1;
        if ((q & 1) != half) continue;
        if (F16) {
          // y of t goes to the target's row of the expansion operand Yx, at
          // t's place in the target class's concatenated ranks, split into
          // FP16 hi/lo; 8 values (one 16-byte group) at a time
          // Two groups of 8 that fill the same 32-byte sector of a Yx row (an
          // even and the next odd group of 8 in the row; the 64-byte swizzle
          // keeps such a pair together) leave in one 32-byte store.
          int d = epi_dst[q * 32 + lane];
          if (d >= 0 && !FMM_GUARD(d < a.ntiles * FMM_TILE, CHK_PROJ_DST, d)) d = -1;
          const int k8 = g.kap8[q];
          for (int c = c0 & ~15; c < c1; c += 16) {
            float v[16];
            tmem_ld16(tb + (uint32_t)c, v);
            uint32_t h8[8], l8[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) split_h2(v[2 * i] * f, v[2 * i + 1] * f, h8[i], l8[i]);
            if (d < 0) continue;
            // the 16 columns hold groups j0 = (c - c0) / 8 (may be -1) and j0 + 1
            const int j0 = (c - c0) >> 3;
            const int a0 = k8 + j0;  // K group of the first half
            const bool has0 = c >= c0, has1 = c + 8 < c1;
            if (has0 && has1 && !(a0 & 1)) {
              // the pair's 16-byte chunks sit at p0 = (a0 & 3) ^ sw and p0 ^ 1 of
              // the swizzled row: one aligned 32-byte sector, the second group
              // first when p0 is odd
              const int64_t G = (((int64_t)(d >> 7) * a.kct + (a0 >> 2)) << 7) + (d & 127);
              const int sw = (int)((G >> 1) & 3), p0 = (a0 & 3) ^ sw;
              const int64_t off = 4 * (p0 & ~1) - 4 * sw;  // from il_idx(G, lo, 0)
              if (p0 & 1) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const uint32_t th = h8[i], tl = l8[i];
                  h8[i] = h8[i + 4];
                  l8[i] = l8[i + 4];
                  h8[i + 4] = th;
                  l8[i + 4] = tl;
                }
              }
              st_cs_u8(a.Yx + il_idx(G, 0, 0) + off, h8);
              st_cs_u8(a.Yx + il_idx(G, 1, 0) + off, l8);
            } else {
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                if (hh == 0 ? !has0 : !has1) continue;
                const int a8 = a0 + hh;
                const int64_t G = (((int64_t)(d >> 7) * a.kct + (a8 >> 2)) << 7) + (d & 127);
                st_cs_u4(a.Yx + il_idx(G, 0, 4 * (a8 & 3)), h8 + 4 * hh);
                st_cs_u4(a.Yx + il_idx(G, 1, 4 * (a8 & 3)), l8 + 4 * hh);
              }
            }
          }
        } else {
          // TF32 form: the ranks are multiples of 16, so are the offsets
          float* y = a.Y + cellrow * a.YS + 8 * g.yo8[q];
          for (int c = c0; c < c1; c += 16) {
            float v[16];
            tmem_ld16(tb + (uint32_t)c, v);
            if (valid) {
              st_cs_v4(y + (c - c0), v[0], v[1], v[2], v[3]);
              st_cs_v4(y + (c - c0) + 4, v[4], v[5], v[6], v[7]);
              st_cs_v4(y + (c - c0) + 8, v[8], v[9], v[10], v[11]);
              st_cs_v4(y + (c - c0) + 12, v[12], v[13], v[14], v[15]);
            }
          }
        }
      }
      __syncwarp();
      tc_fence_before();
      mbar_arrive(acc_empty(b));
      ++uu;
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == SP_MMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---- expansion ----------------------------------------------------------------
constexpr int EX_SETS = 3;
constexpr int EX_EPI = 4 * EX_SETS;
constexpr int EX_MMA = EX_EPI + 4;
constexpr int EX_THREADS = 32 * (EX_MMA + 1);
constexpr int EX_GT = 64;    // transfer vectors per work unit
constexpr int EX_GROUPS = (FMM_NT_CLASS + EX_GT - 1) / EX_GT;
// transfer vectors per accumulator before it is drained (ExpArgs::tpa): as
// many as keep the accumulation chain within one full-rank operator's
// (order^3 products), at least 4, at most 16

struct ExpArgs {
  const int32_t* tile_nact;
  const int16_t* eslot;   // [tile][189] operator slot of active transfer vector ai
  const int8_t* ekch;     // [tile][189] its padded rank / 16 (TF32: its pipeline stages)
  const int64_t* yidx;    // [tile][189][128] first Y value of the row's source, -1 if none
  const float* Y;
  const float* U;  // interleaved hi/lo slabs (il_idx)
  float* partial;  // [group][tile][128][cpad]
  int32_t* err;
  int64_t YS;
  int ntiles, cpad, nh, nhalf, nst, tpa;
  uint32_t acol, tmem_cols;
  uint64_t wait_ns;  // limit of a pipeline wait (fmm_set_wait_limit)
};

constexpr int EXS_CHUNK = 8;  // active transfer vectors per setup block

// Per (tile, active transfer vector): the operator slot, its pipeline stages
// (rank / 16), and per target row the first Y value of its source for t (-1:
// no source), so that the expansion's roles read flat tables.  One block per
// (tile, chunk of EXS_CHUNK transfer vectors), one thread per row.
__global__ void __launch_bounds__(FMM_TILE)
k_svd_exp_setup(const Tile* __restrict__ tiles, const int32_t* __restrict__ tile_src,
                const int16_t* __restrict__ tile_act, const int32_t* __restrict__ tile_nact, LevelPtrs lv,
                const int16_t* __restrict__ cls_t, const int32_t* __restrict__ t_ry, const int32_t* __restrict__ yoff,
                int64_t YS, int16_t* __restrict__ eslot, int8_t* __restrict__ ekch, int64_t* __restrict__ yidx) {
  const int tile = blockIdx.x, r = threadIdx.x;
  const Tile tl = tiles[tile];
  const int l = tl.level, zero = lv.ncell[l], nact = tile_nact[tile];
  const int64_t rbase = lv.row_off[l];
  const int a_end = min(nact, (int)(blockIdx.y + 1) * EXS_CHUNK);
  for (int ai = blockIdx.y * EXS_CHUNK; ai < a_end; ++ai) {
    const int k = tile_act[(int64_t)tile * FMM_NT_CLASS + ai];
    const int slot = cls_t[tl.cls * FMM_NT_CLASS + k];
    if (r == 0) {
      eslot[(int64_t)tile * FMM_NT_CLASS + ai] = (int16_t)slot;
      ekch[(int64_t)tile * FMM_NT_CLASS + ai] = (int8_t)(t_ry[slot] / KC);
    }
    const int src = tile_src[((int64_t)tile * FMM_NT_CLASS + k) * FMM_TILE + r];
    yidx[((int64_t)tile * FMM_NT_CLASS + ai) * FMM_TILE + r] =
        src == zero ? -1 : (rbase + src) * YS + yoff[(lv.key[l][src] & 7) * FMM_NT + slot];
  }
}

// FP16 form, per evaluation: for every (target tile, transfer vector of the
// tile's class, row) either the destination of the source's projection --
// dst[the source class's list index of t][the source's expansion row] =
// tile * 128 + row -- or, where the target has no source for t, zeros in the
// target's Yx row over t's ranks; the tail of each Yx row past the class's
// concatenated ranks is zeroed too (the factor bank is zero there, and the
// products must be finite).  Rows past the tile's count are left alone:
// their outputs are never read.  One block per (tile, chunk of EXS_CHUNK
// transfer vectors), one thread per row.
__global__ void __launch_bounds__(FMM_TILE)
k_svd_scatter_setup(const Tile* __restrict__ tiles, const int32_t* __restrict__ tile_src, LevelPtrs lv,
                    const int16_t* __restrict__ cls_t, const int32_t* __restrict__ t_ry,
                    const int16_t* __restrict__ kap8, const int16_t* __restrict__ srcidx, int kct, int64_t drows,
                    int32_t* __restrict__ dst, uint32_t* __restrict__ Yx) {
  const int tile = blockIdx.x, r = threadIdx.x;
  const Tile tl = tiles[tile];
  if (r >= tl.count) return;
  const int l = tl.level, zero = lv.ncell[l];
  const int64_t rbase = lv.row_off[l];
  const uint32_t z[4] = {0u, 0u, 0u, 0u};
  const int k0 = blockIdx.y * EXS_CHUNK, k_end = min(FMM_NT_CLASS, k0 + EXS_CHUNK);
  // the chunk's sources, then their classes, each as independent loads in flight together
  int srcs[EXS_CHUNK], cls[EXS_CHUNK];
#pragma unroll
  for (int j = 0; j < EXS_CHUNK; ++j)
    srcs[j] = k0 + j < k_end ? tile_src[((int64_t)tile * FMM_NT_CLASS + k0 + j) * FMM_TILE + r] : zero;
#pragma unroll
  for (int j = 0; j < EXS_CHUNK; ++j) cls[j] = srcs[j] != zero ? (int)(lv.key[l][srcs[j]] & 7) : 0;
#pragma unroll
  for (int j = 0; j < EXS_CHUNK; ++j) {
    const int k = k0 + j;
    if (k >= k_end) break;
    const int slot = cls_t[tl.cls * FMM_NT_CLASS + k];
    const int src = srcs[j];
    if (src != zero) {
      const int64_t di = (int64_t)srcidx[cls[j] * FMM_NT + slot] * drows + rbase + src;
      if (FMM_GUARD(di >= 0 && di < (int64_t)FMM_NT_CLASS * drows, CHK_SCATTER_DST, k)) dst[di] = tile * FMM_TILE + r;
    } else {
      const int k8 = kap8[tl.cls * FMM_NT + slot], n8 = t_ry[slot] / 8;
      for (int j = 0; j < n8; ++j) {
        const int a8 = k8 + j;
        const int64_t G = (((int64_t)tile * kct + (a8 >> 2)) << 7) + r;
        *(uint4*)(Yx + il_idx(G, 0, 4 * (a8 & 3))) = *(const uint4*)z;
        *(uint4*)(Yx + il_idx(G, 1, 4 * (a8 & 3))) = *(const uint4*)z;
      }
    }
  }
  if (blockIdx.y == 0) {
    // the tail past the class's ranks (kap8 of the class's last t + its ranks)
    const int last = cls_t[tl.cls * FMM_NT_CLASS + FMM_NT_CLASS - 1];
    for (int a8 = kap8[tl.cls * FMM_NT + last] + t_ry[last] / 8; a8 < 4 * kct; ++a8) {
      const int64_t G = (((int64_t)tile * kct + (a8 >> 2)) << 7) + r;
      *(uint4*)(Yx + il_idx(G, 0, 4 * (a8 & 3))) = *(const uint4*)z;
      *(uint4*)(Yx + il_idx(G, 1, 4 * (a8 & 3))) = *(const uint4*)z;
    }
  }
}

// ---- expansion, FP16 form ---------------------------------------------------
// L_T += U y over all of a target's sources at once: A = the tile's Yx rows
// (written by the projection, K = the target class's transfer vectors with
// their ranks concatenated), B = the class's factor bank Uc along the same K
// (one column half); both arrive by one linear bulk copy per 32-value chunk,
// so no role gathers or converts anything.  Work unit = (K group, tile,
// column half).  The tensor cores' FP32 accumulation does not round to
// nearest: an accumulator takes `chain` chunks (about order^3 values of K,
// the chain of one full-rank operator) before the epilogue adds it into FP32
// running sums in shared memory; the two accumulators alternate.
constexpr int X_PROD = 0, X_MMA = 1, X_EPI = 2;
constexpr int X_THREADS = 32 * (X_EPI + 4);
constexpr int X_A_BYTES = FMM_TILE * 128;  // 128 rows x (32 FP16 hi + 32 FP16 lo)

struct Exp16Args {
  const uint32_t* Yx;    // [tile][kct][128 rows] interleaved FP16 hi/lo rows (il_idx)
  const uint32_t* Uc;    // [class][kct][cpad rows] interleaved FP16 hi/lo rows
  float* partial;        // [group][tile][128][cpad]
  int32_t* err;
  const Tile* tiles;
  const uint32_t* ybound;  // the rows' scales (the projection's)
  int ntiles, kct, ngroups, cpg, nh, nhalf, cpad, nst, chain;
  float uscale;
  uint64_t wait_ns;
};

__device__ inline void x_unit(const Exp16Args& a, int u, int& g, int& tile, int& h, int& k0, int& k1) {
  const int per_g = a.ntiles * a.nh;
  g = u / per_g;
  const int rem = u - g * per_g;
  tile = rem / a.nh;
  h = rem - tile * a.nh;
  k0 = g * a.cpg;
  k1 = min(a.kct, k0 + a.cpg);
}

__global__ void __launch_bounds__(X_THREADS, 1)
k_svd_expand16_tc(Exp16Args a, LevelPtrs lv) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t b_bytes = (uint32_t)a.nhalf * 128u;
  const uint32_t stage_bytes = X_A_BYTES + b_bytes;
  const uint32_t sum_off = (uint32_t)a.nst * stage_bytes;
  const uint32_t bars = base + sum_off + (uint32_t)a.nhalf * FMM_TILE * 4u;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (MAXST + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * MAXST + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * MAXST + 2 + b); };
  const uint32_t mma_done = bars + 8u * (2 * MAXST + 4);
  unsigned char* gbase = smem_raw + (base - raw);
  float* S = (float*)(gbase + sum_off);
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(gbase + (bars - base) + 8u * (2 * MAXST + 6));
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  uint32_t tmem_cols = 32;
  while ((int)tmem_cols < 2 * a.nhalf) tmem_cols <<= 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXST; ++s) {
      mbar_init(full(s), 1);  // the producer's expect_tx
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), 128);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == X_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nunits = a.ngroups * a.ntiles * a.nh;

  if (warp == X_PROD) {
    // ---------------------------------------------------------- copy producer
    uint32_t it = 0, last = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, tile, h, k0, k1;
      x_unit(a, unit, g, tile, h, k0, k1);
      const int cls = a.tiles[tile].cls;
      for (int kc = k0; kc < k1; ++kc, ++it) {
        const int s = (int)(it % a.nst);
        const uint32_t ph = (it / a.nst) & 1u;
        if (!warp_wait(empty(s), ph ^ 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          const uint32_t st = base + (uint32_t)s * stage_bytes;
          mbar_expect_tx(full(s), X_A_BYTES + b_bytes);
          bulk_g2s(st, a.Yx + (((int64_t)tile * a.kct + kc) << 7) * 32, X_A_BYTES, full(s));
          bulk_g2s(st + X_A_BYTES, a.Uc + (((int64_t)cls * a.kct + kc) * a.cpad + (int64_t)h * a.nhalf) * 32,
                   b_bytes, full(s));
        }
        __syncwarp();
        last = it + 1;
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
      // let the copies already issued land before the CTA leaves (bounded)
      for (uint32_t j = last > (uint32_t)a.nst ? last - a.nst : 0; j < last; ++j)
        mbar_wait(full((int)(j % a.nst)), (j / a.nst) & 1u);
    }
    __syncwarp();
  } else if (warp == X_MMA) {
    // ---------------------------------------------------------- MMA issuer
    uint32_t it = 0, tt = 0;
    bool ok = true;
    const uint32_t idesc = idesc_f16(FMM_TILE, a.nhalf);
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, tile, h, k0, k1;
      x_unit(a, unit, g, tile, h, k0, k1);
      for (int kc0 = k0; kc0 < k1 && ok; kc0 += a.chain, ++tt) {
        const int kc1 = min(k1, kc0 + a.chain);
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_empty(b), ((tt >> 1) & 1u) ^ 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * a.nhalf);
        for (int kc = kc0; kc < kc1; ++kc, ++it) {
          const int s = (int)(it % a.nst);
          const uint32_t ph = (it / a.nst) & 1u;
          if (!warp_wait(full(s), ph, abort_flag, a.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t st = base + (uint32_t)s * stage_bytes;
            const uint32_t sb = st + X_A_BYTES;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint64_t ahi = sdesc_sw64s(st + ks * 32u, 1024), alo = sdesc_sw64s(st + 512u + ks * 32u, 1024);
              const uint64_t bhi = sdesc_sw64s(sb + ks * 32u, 1024), blo = sdesc_sw64s(sb + 512u + ks * 32u, 1024);
              mma_f16(d, ahi, bhi, idesc, (kc > kc0 || ks > 0) ? 1u : 0u);
              mma_f16(d, ahi, blo, idesc, 1u);
              mma_f16(d, alo, bhi, idesc, 1u);
            }
            mma_commit(empty(s));
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) mma_commit(acc_full(b));
        __syncwarp();
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
    // every MMA issued so far has finished before TMEM is freed (bounded)
    if (lane == 0) {
      mma_commit(mma_done);
      mbar_wait(mma_done, 0);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    // TMEM lane quarter = warp % 4; row = the target's position in the tile
    const int q = warp & 3, row = q * 32 + lane;
    uint32_t tt = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, tile, h, k0, k1;
      x_unit(a, unit, g, tile, h, k0, k1);
      for (int kc0 = k0; kc0 < k1; kc0 += a.chain, ++tt) {
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_full(b), (tt >> 1) & 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * a.nhalf);
        const bool first = kc0 == k0;
        int cb = 0;
        for (; cb + 32 <= a.nhalf; cb += 32) {
          float v[32];
          tmem_ld32(tbase + (uint32_t)cb, v);
          float* sp = S + cb * FMM_TILE + row;
#pragma unroll
          for (int i = 0; i < 32; ++i) sp[i * FMM_TILE] = first ? v[i] : sp[i * FMM_TILE] + v[i];
        }
        if (cb < a.nhalf) {  // nhalf is a multiple of 16
          float v[16];
          tmem_ld16(tbase + (uint32_t)cb, v);
          float* sp = S + cb * FMM_TILE + row;
#pragma unroll
          for (int i = 0; i < 16; ++i) sp[i * FMM_TILE] = first ? v[i] : sp[i * FMM_TILE] + v[i];
        }
        tc_fence_before();
        mbar_arrive(acc_empty(b));
      }
      if (!ok) break;
      const Tile tl = a.tiles[tile];
      if (k0 < k1 && row < tl.count) {
        float* out = a.partial + (((int64_t)g * a.ntiles + tile) * FMM_TILE + row) * a.cpad + h * a.nhalf;
        // back from the operands' scales (powers of two: exact)
        const int prob = problem_of(lv, tl.level, lv.cls[tl.level][tl.first + row]);
        const float inv =
            1.f / (pow2_scale(__uint_as_float(a.ybound[ymax_index(prob, tl.level)])) * a.uscale);
        for (int c = 0; c < a.nhalf; c += 4)
          *(float4*)(out + c) = make_float4(S[c * FMM_TILE + row] * inv, S[(c + 1) * FMM_TILE + row] * inv,
                                            S[(c + 2) * FMM_TILE + row] * inv, S[(c + 3) * FMM_TILE + row] * inv);
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == X_MMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Unit u -> (group g, tile, column half h), the halves of a tile adjacent so
// that CTAs running at the same time gather the same Y rows (L2 reuse).
__device__ inline void exp_unit(const ExpArgs& a, int u, int& g, int& h, int& tile) {
  const int per_g = a.ntiles * a.nh;
  g = u / per_g;
  const int rem = u - g * per_g;
  tile = rem / a.nh;
  h = rem - tile * a.nh;
}

// TF32 hi/lo operands (FMM_M2L_MATH=tf32); the FP16 form is k_svd_expand16_tc.
__global__ void __launch_bounds__(EX_THREADS, 1)
k_svd_expand_tc(ExpArgs a, LevelPtrs lv) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t b_bytes = (uint32_t)a.nhalf * KC * 4;
  const uint32_t stage_bytes = 2u * b_bytes;
  const uint32_t sum_off = (uint32_t)a.nst * stage_bytes;
  const uint32_t bars = base + sum_off + (uint32_t)a.nhalf * FMM_TILE * 4u;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (MAXST + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * MAXST + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * MAXST + 2 + b); };
  const uint32_t mma_done = bars + 8u * (2 * MAXST + 4);
  unsigned char* gbase = smem_raw + (base - raw);
  float* S = (float*)(gbase + sum_off);
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(gbase + (bars - base) + 8u * (2 * MAXST + 6));
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXST; ++s) {
      mbar_init(full(s), FMM_TILE + 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), 128);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == EX_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nunits = a.ntiles * a.nh * EX_GROUPS;

  if (warp < EX_EPI) {
    // ---------------------------------------------------------- producers
    // thread r loads 16 Y values of its target's source for the stage, splits
    // them into TF32 hi/lo and writes them into its TMEM lane; one
    // thread issues the B slab (U_t rows of this column half x the stage's
    // rank columns).
    const int set = warp >> 2;
    const int r = threadIdx.x & (FMM_TILE - 1);
    uint32_t it = 0, last = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, h, tile;
      exp_unit(a, unit, g, h, tile);
      const int nact = a.tile_nact[tile];
      const int a0 = g * EX_GT, a1 = min(nact, a0 + EX_GT);
      if (a0 >= a1) continue;
      const int64_t tb = (int64_t)tile * FMM_NT_CLASS;
      // the next transfer vector's slot, stages and source offset are loaded
      // while the current one is being copied
      int nslot = a.eslot[tb + a0], nkch = a.ekch[tb + a0];
      int64_t nyi = a.yidx[(tb + a0) * FMM_TILE + r];
      for (int ai = a0; ai < a1 && ok; ++ai) {
        const int slot = nslot, kch = nkch;
        const int64_t yi = nyi;
        if (ai + 1 < a1) {
          nslot = a.eslot[tb + ai + 1];
          nkch = a.ekch[tb + ai + 1];
          nyi = a.yidx[(tb + ai + 1) * FMM_TILE + r];
        }
        const int kc0 = (set - (int)(it % EX_SETS) + EX_SETS) % EX_SETS;
        if (kc0 < kch) {
          const float* yr = yi < 0 ? nullptr : a.Y + yi;
          for (int kc = kc0; kc < kch; kc += EX_SETS) {
            const uint32_t j = it + (uint32_t)kc;
            uint32_t vh[16], vl[16];
            if (yr) {
              ld_v8(yr + kc * KC, vh);
              ld_v8(yr + kc * KC + 8, vh + 8);
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float y = __uint_as_float(vh[i]);
                const float hi = tf32_rna(y);
                vh[i] = __float_as_uint(hi);
                vl[i] = __float_as_uint(tf32_rna(y - hi));
              }
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) vh[i] = vl[i] = 0u;
            }
            const int s = (int)(j % a.nst);
            const uint32_t ph = (j / a.nst) & 1u;
            if (!warp_wait(empty(s), ph ^ 1u, abort_flag, a.wait_ns)) {
              ok = false;
              break;
            }
            const uint32_t st = base + (uint32_t)s * stage_bytes;
            if (r == 0) {
              mbar_expect_tx(full(s), 2u * b_bytes);
              const int64_t G = ((int64_t)kc * FMM_NT + slot) * a.cpad + h * a.nhalf;
              bulk_g2s(st, a.U + G * 32, 2u * b_bytes, full(s));
            }
            const uint32_t ta = tmem + ((uint32_t)(r & ~31) << 16) + a.acol + (uint32_t)s * 32u;
            tmem_st16(ta, vh);
            tmem_st16(ta + 16u, vl);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(full(s));
            last = j + 1;
          }
        }
        it += (uint32_t)kch;
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
    if (!ok && r == 0) {
      for (uint32_t j = last > (uint32_t)a.nst ? last - a.nst : 0; j < last; ++j)
        if ((int)(j % EX_SETS) == set) mbar_wait(full((int)(j % a.nst)), (j / a.nst) & 1u);
    }
    __syncwarp();
  } else if (warp == EX_MMA) {
    // ---------------------------------------------------------- MMA issuer
    uint32_t it = 0, tt = 0;
    bool ok = true;
    const uint32_t idesc = idesc_tf32(FMM_TILE, a.nhalf);
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, h, tile;
      exp_unit(a, unit, g, h, tile);
      const int nact = a.tile_nact[tile];
      const int a0 = g * EX_GT, a1 = min(nact, a0 + EX_GT);
      if (a0 >= a1) continue;
      // stages of the unit's transfer vectors, two per lane (EX_GT = 64)
      const int64_t tb = (int64_t)tile * FMM_NT_CLASS;
      const int kA = a0 + lane < a1 ? a.ekch[tb + a0 + lane] : 0;
      const int kB = a0 + 32 + lane < a1 ? a.ekch[tb + a0 + 32 + lane] : 0;
      for (int ag = a0; ag < a1 && ok; ag += a.tpa, ++tt) {
        const int ae = min(a1, ag + a.tpa);
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_empty(b), ((tt >> 1) & 1u) ^ 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * a.nhalf);
        bool first = true;
        for (int ai = ag; ai < ae && ok; ++ai) {
          const int u = ai - a0;
          const int kch = __shfl_sync(0xffffffffu, u < 32 ? kA : kB, u & 31);
          for (int kc = 0; kc < kch; ++kc, ++it) {
            const int s = (int)(it % a.nst);
            const uint32_t ph = (it / a.nst) & 1u;
            if (!warp_wait(full(s), ph, abort_flag, a.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            if (lane == 0) {
              const uint32_t st = base + (uint32_t)s * stage_bytes;
              const uint32_t ahi0 = tmem + a.acol + (uint32_t)s * 32u;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint32_t ahi = ahi0 + ks * 8u, alo = ahi0 + 16u + ks * 8u;
                const uint64_t bhi = sdesc_sw64s(st + ks * 32u, 1024);
                const uint64_t blo = sdesc_sw64s(st + 512u + ks * 32u, 1024);
                mma_tf32_ta(d, ahi, bhi, idesc, (first && ks == 0) ? 0u : 1u);
                mma_tf32_ta(d, ahi, blo, idesc, 1u);
                mma_tf32_ta(d, alo, bhi, idesc, 1u);
              }
              mma_commit(empty(s));
            }
            __syncwarp();
            first = false;
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit(acc_full(b));
        __syncwarp();
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
    if (lane == 0) {
      mma_commit(mma_done);
      mbar_wait(mma_done, 0);
    }
    __syncwarp();
  } else if (warp < EX_MMA) {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3, row = q * 32 + lane;
    uint32_t tt = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, h, tile;
      exp_unit(a, unit, g, h, tile);
      const int nact = a.tile_nact[tile];
      const int a0 = g * EX_GT, a1 = min(nact, a0 + EX_GT);
      if (a0 >= a1) continue;
      for (int ag = a0; ag < a1; ag += a.tpa, ++tt) {
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_full(b), (tt >> 1) & 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * a.nhalf);
        const bool first = ag == a0;
        int cb = 0;
        for (; cb + 32 <= a.nhalf; cb += 32) {
          float v[32];
          tmem_ld32(tbase + (uint32_t)cb, v);
          float* sp = S + cb * FMM_TILE + row;
#pragma unroll
          for (int i = 0; i < 32; ++i) sp[i * FMM_TILE] = first ? v[i] : sp[i * FMM_TILE] + v[i];
        }
        if (cb < a.nhalf) {
          float v[16];
          tmem_ld16(tbase + (uint32_t)cb, v);
          float* sp = S + cb * FMM_TILE + row;
#pragma unroll
          for (int i = 0; i < 16; ++i) sp[i * FMM_TILE] = first ? v[i] : sp[i * FMM_TILE] + v[i];
        }
        tc_fence_before();
        mbar_arrive(acc_empty(b));
      }
      if (!ok) break;
      float* out = a.partial + (((int64_t)g * a.ntiles + tile) * FMM_TILE + row) * a.cpad + h * a.nhalf;
      for (int c = 0; c < a.nhalf; c += 4)
        *(float4*)(out + c) =
            make_float4(S[c * FMM_TILE + row], S[(c + 1) * FMM_TILE + row], S[(c + 2) * FMM_TILE + row],
                        S[(c + 3) * FMM_TILE + row]);
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == EX_MMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// groups per tile at most: every group but the last holds SP_MAXG transfer
// vectors or more than SP_ACC - Rp columns
int sp_ngroups(int Rp) {
  return std::min(FMM_NT_CLASS, (FMM_NT_CLASS * Rp + (SP_ACC - Rp)) / (SP_ACC - Rp + 1) +
                                    (FMM_NT_CLASS + SP_MAXG - 1) / SP_MAXG + 1);
}
int sp_stage_bytes() { return 2 * SP_A_BYTES + 2 * SP_B_BYTES; }
int sp_nst() { return std::min(MAXST, (227 * 1024 - 1024 - 256 - SP_NEPI * SP_MAXG * 32 * 4) / sp_stage_bytes()); }
int sp_smem(int nst) { return nst * sp_stage_bytes() + 1024 + 256 + SP_NEPI * SP_MAXG * 32 * 4; }
// Columns per half: cp, or cp / 2 when one accumulator of cp columns is
// wider than an MMA or the two accumulators would leave TMEM room for fewer A
// stages than there are producer sets (parity waits need every set to run at
// most one phase ahead of the MMA; p = 6, cp = 224, would leave two stages).
int ex_nhalf(int cp) { return (cp > 256 || 2 * cp + 32 * EX_SETS > 512) ? cp / 2 : cp; }
int ex_stage_bytes(int cp) { return 2 * ex_nhalf(cp) * KC * 4; }
int ex_smem(int cp, int nst) { return nst * ex_stage_bytes(cp) + ex_nhalf(cp) * FMM_TILE * 4 + 1024 + 256; }

// FP16 expansion: stages of one Yx slab and one factor slab, the running sums
int x_stage_bytes(int cp) { return X_A_BYTES + ex_nhalf(cp) * 128; }
int x_fixed_bytes(int cp) { return ex_nhalf(cp) * FMM_TILE * 4 + 1024 + 256; }
int x_nst(int cp) { return std::min(MAXST, (227 * 1024 - x_fixed_bytes(cp)) / x_stage_bytes(cp)); }
// chunks of 32 K per accumulator: a chain of about order^3 products
int x_chain(const Ctx* c) { return std::max(1, (c->ncoef + 31) / 32); }
// K groups per tile: about 12 units per SM over all tiles and column halves,
// each group a whole number of chains, no group empty
void x_groups(const Ctx* c, int* ngroups, int* cpg) {
  const int kct = c->svd_kct, chain = x_chain(c), nh = c->cpad / ex_nhalf(c->cpad);
  const int sms = c->num_sms > 0 ? c->num_sms : 148;
  int ng = (int)std::lround(12.0 * sms / std::max(1, c->ntiles * nh));
  const int chains = (kct + chain - 1) / chain;
  ng = std::max(1, std::min(ng, std::min(chains, 8)));
  int per = (chains + ng - 1) / ng * chain;  // chunks per group
  *cpg = per;
  *ngroups = (kct + per - 1) / per;
}

}  // namespace

// Mixed precision with the rank padding of 16 (always) and output columns
// that fit two TMEM accumulators beside the A stages: order <= 7.
bool m2l_svd_tc_supported(const Ctx* c) {
  const int nhalf = ex_nhalf(c->cpad);
  return c->cpad % 32 == 0 && nhalf <= 256 && nhalf % 16 == 0 && 2 * nhalf + 32 * EX_SETS <= 512 && c->svd_rp <= SP_ACC;
}

// Tensor maps of the compressed factor banks, the partial-sum buffer and the
// kernels' shared-memory limits (before an evaluation is captured).
fmm_status m2l_svd_tc_prepare(Ctx* c) {
  if (c->ntiles == 0) return FMM_OK;
  const int cp = c->cpad, Rp = c->svd_rp, nhalf = ex_nhalf(cp);
  const bool f16 = m2l_uses_f16(c);
  if (c->num_sms == 0) FMM_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
  int xng = EX_GROUPS, xcpg = 0;
  if (f16) x_groups(c, &xng, &xcpg);
  const int64_t need = (int64_t)c->ntiles * xng * FMM_TILE * cp;
  if (need > c->tc_partial_cap) {
    dfree(c, c->tc_partial, 4 * (size_t)c->tc_partial_cap);
    c->tc_partial = nullptr;
    c->tc_partial_cap = 0;
    void* p;
    FMM_TRY(dalloc(c, &p, 4 * (size_t)need));
    c->tc_partial = (float*)p;
    c->tc_partial_cap = need;
  }
  if (!c->tc_err) {
    void* p;
    FMM_TRY(dalloc(c, &p, 64));
    c->tc_err = (int32_t*)p;
    FMM_CUDA(c, cudaMemsetAsync(c->tc_err, 0, 64, c->stream));
  }
  if (!c->tc_err_h) return set_err(c, FMM_ERR_STATE, "internal: no host error word");
  const int64_t gneed = (int64_t)c->ntiles * sp_ngroups(Rp);
  if (gneed > c->svd_gcap) {
    dfree(c, c->svd_recs, sizeof(ProjRec) * (size_t)c->svd_gcap);
    c->svd_recs = nullptr;
    c->svd_gcap = 0;
    void* p;
    FMM_TRY(dalloc(c, &p, sizeof(ProjRec) * (size_t)gneed));
    c->svd_recs = p;
    c->svd_gcap = gneed;
  }
  if (f16) {
    // the expansion operand Yx and the projection's destination map
    const size_t yx = (size_t)c->ntiles * c->svd_kct * FMM_TILE * 128;
    if (yx > c->svd_Yx_cap) {
      dfree(c, c->svd_Yx, c->svd_Yx_cap);
      c->svd_Yx = nullptr;
      c->svd_Yx_cap = 0;
      const size_t cap = yx + yx / 8;
      void* p;
      FMM_TRY(dalloc(c, &p, cap));
      c->svd_Yx = p;
      c->svd_Yx_cap = cap;
    }
    const size_t db = sizeof(int32_t) * FMM_NT_CLASS * (size_t)c->rows;
    if (db > c->svd_dst_cap) {
      dfree(c, c->svd_dst, c->svd_dst_cap);
      c->svd_dst = nullptr;
      c->svd_dst_cap = 0;
      const size_t cap = db + db / 8;
      void* p;
      FMM_TRY(dalloc(c, &p, cap));
      c->svd_dst = (int32_t*)p;
      c->svd_dst_cap = cap;
    }
  }
  // class-ordered copy of the multipoles (rows as M) and its tensor maps
  if (!f16 && c->ntiles > c->svd_ecap) {
    dfree(c, c->svd_eslot, sizeof(int16_t) * (size_t)c->svd_ecap * FMM_NT_CLASS);
    dfree(c, c->svd_ekch, sizeof(int8_t) * (size_t)c->svd_ecap * FMM_NT_CLASS);
    dfree(c, c->svd_yidx, sizeof(int64_t) * (size_t)c->svd_ecap * FMM_NT_CLASS * FMM_TILE);
    c->svd_eslot = nullptr;
    c->svd_ekch = nullptr;
    c->svd_yidx = nullptr;
    c->svd_ecap = 0;
    const int64_t cap = c->tiles_cap;
    void* p;
    FMM_TRY(dalloc(c, &p, sizeof(int16_t) * (size_t)cap * FMM_NT_CLASS));
    c->svd_eslot = (int16_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int8_t) * (size_t)cap * FMM_NT_CLASS));
    c->svd_ekch = (int8_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int64_t) * (size_t)cap * FMM_NT_CLASS * FMM_TILE));
    c->svd_yidx = (int64_t*)p;
    c->svd_ecap = cap;
  }
  // class-ordered multipole copy: (level, class) segments rounded up to 128 rows
  int64_t mrows = 0;
  for (int l = 2; l <= c->leaf; ++l)
    for (int k = 0; k < 8; ++k) {
      c->svd_mcbase[l][k] = (int)mrows;
      mrows += (c->cls_off[l][k + 1] - c->cls_off[l][k] + FMM_TILE - 1) / FMM_TILE * FMM_TILE;
    }
  mrows += FMM_TILE;
  if (mrows > c->svd_mcls_rows) {
    dfree(c, c->svd_Mcls, 8 * (size_t)c->svd_mcls_rows * cp);
    dfree(c, c->svd_mscale, 4 * (size_t)c->svd_mcls_rows);
    c->svd_Mcls = nullptr;
    c->svd_mscale = nullptr;
    c->svd_mcls_rows = 0;
    const int64_t cap = (mrows + mrows / 8 + FMM_TILE - 1) / FMM_TILE * FMM_TILE;  // chunks start on 8-row groups
    void* p;
    FMM_TRY(dalloc(c, &p, 8 * (size_t)cap * cp));
    FMM_CUDA(c, cudaMemsetAsync(p, 0, 8 * (size_t)cap * cp, c->stream));
    c->svd_Mcls = (float*)p;
    FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));  // FP16 operands: each row's scale
    c->svd_mscale = (float*)p;
    c->svd_mcls_rows = cap;
  }
  // stages: shared memory and the TMEM columns beside the accumulators
  int nst = (227 * 1024 - ex_smem(cp, 0)) / ex_stage_bytes(cp);
  nst = std::min(nst, (512 - 2 * nhalf) / 32);
  nst = std::min(nst, MAXST);
  const int nst_p = sp_nst();
  if (nst < EX_SETS || nst_p < 2)
    return set_err(c, FMM_ERR_ARG, "compressed M2L tensor path: fewer stages than producer sets");
  c->svd_tc_nst = nst;
  if (m2l_uses_f16(c)) {
    FMM_TRY(raise_smem_limit(c, (const void*)k_svd_proj_tc<true>, sp_smem(nst_p)));
    if (x_nst(cp) < 2) return set_err(c, FMM_ERR_ARG, "compressed M2L tensor path: fewer than two expansion stages");
    FMM_TRY(raise_smem_limit(c, (const void*)k_svd_expand16_tc, x_nst(cp) * x_stage_bytes(cp) + x_fixed_bytes(cp)));
    if (!c->svd_umax) {  // max |Y| per (problem + 1, level): every batch size
      void* p;
      FMM_TRY(dalloc(c, &p, sizeof(uint32_t) * (FMM_MAX_BATCH + 1) * FMM_MAX_LEVELS));
      c->svd_umax = (uint32_t*)p;
    }
  } else {
    FMM_TRY(raise_smem_limit(c, (const void*)k_svd_proj_tc<false>, sp_smem(nst_p)));
    FMM_TRY(raise_smem_limit(c, (const void*)k_svd_expand_tc, ex_smem(cp, nst)));
  }
  return FMM_OK;
}

// Projection of every tile, then the expansion and (after `mid`) the FP64
// reduction of its partial sums.
bool svd_wants_f16(const Ctx* c) { return m2l_uses_f16(c) && c->use_tc && m2l_svd_tc_supported(c); }

// Whether svd_tree_setup's work depends on the tree alone: the FP16 form
// (the TF32 form's records are the same, but it has no destination map and
// keeps them beside its other setup).
bool svd_has_tree_setup(const Ctx* c) { return m2l_uses_f16(c); }

// The projection's work records (k_svd_groups: per tile, groups of active
// source transfer vectors; the unit count) and, in the FP16 form, its
// destination map (k_svd_scatter_setup: per (source cell, t), the row of
// the target tile's operand slab; zeros where a target has no source):
// functions of the tree and the operators' ranks, not of the multipoles.
fmm_status svd_tree_setup(Ctx* c, cudaStream_t s) {
  const bool f16 = m2l_uses_f16(c);
  McBase mb;
  for (int l = 0; l < FMM_MAX_LEVELS; ++l)
    for (int k = 0; k < 8; ++k) {
      mb.base[l][k] = l >= 2 && l <= c->leaf ? c->svd_mcbase[l][k] : 0;
      mb.clsoff[l][k] = c->cls_off[l][k];
    }
  int32_t* nunits = c->counters + CNT_PUNITS;
  FMM_CUDA(c, cudaMemsetAsync(nunits, 0, sizeof(int32_t), s));
  k_svd_groups<<<c->ntiles, 256, 0, s>>>(c->ntiles, sp_ngroups(c->svd_rp), c->tiles, c->lv, mb, c->src_act,
                                         c->src_nact, c->src_t, c->svd_ry, c->svd_yoff, c->tvec,
                                         f16 ? c->svd_kap8 : nullptr, (ProjRec*)c->svd_recs, nunits, c->tc_err);
  if (f16) {
    // destinations of the projections (and zeros where a target has no source)
    FMM_CUDA(c, cudaMemsetAsync(c->svd_dst, 0xFF, sizeof(int32_t) * FMM_NT_CLASS * (size_t)c->rows, s));
    k_svd_scatter_setup<<<dim3(c->ntiles, (FMM_NT_CLASS + EXS_CHUNK - 1) / EXS_CHUNK), FMM_TILE, 0, s>>>(
        c->tiles, c->tile_src, c->lv, c->cls_t, c->svd_ry, c->svd_kap8, c->svd_srcidx, c->svd_kct, c->rows,
        c->svd_dst, (uint32_t*)c->svd_Yx);
  }
  return cuda_err(c, cudaGetLastError(), "compressed M2L setup");
}

// Where each class of each level starts in the class-ordered multipoles.
static McBase mc_base(const Ctx* c) {
  McBase mb;
  for (int l = 0; l < FMM_MAX_LEVELS; ++l)
    for (int k = 0; k < 8; ++k) {
      mb.base[l][k] = l >= 2 && l <= c->leaf ? c->svd_mcbase[l][k] : 0;
      mb.clsoff[l][k] = c->cls_off[l][k];
    }
  return mb;
}

// FP16 class-order copies of levels l0..l1 (k_gather_cls16), after zeroing
// the bounds ||M||_2 per (problem, level) that the gathers record afresh
// when zero_bounds (the first gather launch of an evaluation).
static fmm_status svd_gather16(Ctx* c, cudaStream_t s, int l0, int l1, bool zero_bounds) {
  const int cp = c->cpad;
  if (cp > 64 * GC_PAIRS) return set_err(c, FMM_ERR_STATE, "internal: %d coefficients per row exceed the gather's", cp);
  const McBase mb = mc_base(c);
  if (zero_bounds) {
    const int nslots = (c->forest ? c->nprob : 1) + 1;
    FMM_CUDA(c, cudaMemsetAsync(c->svd_umax, 0, sizeof(uint32_t) * nslots * FMM_MAX_LEVELS, s));
  }
  for (int l = l0; l <= l1; ++l)
    if (c->lv.ncell[l] > 0)
      k_gather_cls16<<<ceil_div(c->lv.ncell[l], 4), 128, 0, s>>>(l, c->lv.ncell[l], c->lv, mb, cp, c->svd_mcls_rows,
                                                                 c->Mhi, c->Mlo, (uint32_t*)c->svd_Mcls,
                                                                 c->svd_mscale, c->svd_umax);
  return cuda_err(c, cudaGetLastError(), "compressed M2L gather");
}

// The leaf level's gather reads the leaf multipoles alone, final once P2M
// has run, so it may run on a branch of its own beside the M2M levels.
bool svd_leaf_gather_apart(const Ctx* c) {
  return c->ntiles > 0 && c->n > 0 && c->leaf >= 2 && c->precision == FMM_MIXED && m2l_kind(c) == 5 &&
         m2l_uses_f16(c) && c->svd_bank_f16 && c->lv.ncell[c->leaf] > 0;
}

fmm_status launch_svd_leaf_gather(Ctx* c, cudaStream_t s) {
  c->leaf_gather_done = false;
  if (!svd_leaf_gather_apart(c)) return FMM_OK;
  FMM_TRY(svd_gather16(c, s, c->leaf, c->leaf, true));
  FMM_CUDA(c, cudaEventRecord(c->ev_gleaf, s));
  c->leaf_gather_done = true;
  return FMM_OK;
}

fmm_status launch_m2l_svd_tc(Ctx* c, cudaStream_t s, cudaEvent_t mid) {
  if (c->ntiles == 0) return FMM_OK;
  const int cp = c->cpad, Rp = c->svd_rp;
  const bool f16 = m2l_uses_f16(c);
  if (f16 != c->svd_bank_f16) return set_err(c, FMM_ERR_STATE, "internal: compressed M2L banks in the other format");
  // multipoles in class order, every level with far field
  const int64_t mrows = c->svd_mcls_rows;
  const McBase mb = mc_base(c);
  if (f16) {
    if (c->leaf_gather_done) {
      // the leaf level ran beside the M2M levels, after zeroing the bounds
      c->leaf_gather_done = false;
      FMM_CUDA(c, cudaStreamWaitEvent(s, c->ev_gleaf, 0));
      FMM_TRY(svd_gather16(c, s, 2, c->leaf - 1, false));
    } else {
      FMM_TRY(svd_gather16(c, s, 2, c->leaf, true));
    }
  } else {
    for (int l = 2; l <= c->leaf; ++l)
      if (c->lv.ncell[l] > 0)
        k_gather_cls<<<c->lv.ncell[l], 128, 0, s>>>(l, c->lv, mb, cp, mrows, c->Mhi, c->Mlo, c->svd_Mcls);
  }
  ProjArgs p;
  p.Y = (float*)c->svd_Y;
  p.Yx = (uint32_t*)c->svd_Yx;
  p.dst = c->svd_dst;
  p.drows = c->rows;
  p.kct = c->svd_kct;
  p.ybound = c->svd_umax;
  p.err = c->tc_err;
  p.YS = c->svd_YS;
  p.ntiles = c->ntiles;
  p.ngroups = sp_ngroups(Rp);
  p.recs = (const ProjRec*)c->svd_recs;
  p.kchunks = cp / (f16 ? 32 : KC);
  p.mrows = mrows;
  p.Mc = c->svd_Mcls;
  p.VT = c->svd_VThi;
  p.nst = sp_nst();
  p.mscale = c->svd_mscale;
  p.vscale = c->svd_vscale;
  p.wait_ns = c->wait_ns;
  int32_t* nunits = c->counters + CNT_PUNITS;
  p.nunits = nunits;
  if (c->m2l_prep_done) FMM_CUDA(c, cudaStreamWaitEvent(s, c->ev_prep, 0));  // svd_tree_setup ran beside
  else FMM_TRY(svd_tree_setup(c, s));
  const int up = p.ntiles * p.ngroups;
  // schedules 2 and 3 start the near field with the projection: three
  // pipeline stages instead of four leave shared memory for P2P blocks on
  // every SM beside the projection's CTA
  const bool near_with_proj = c->timing != 2 && c->p2p_priority && c->p2p_sched >= 2;
  if (near_with_proj) {
    p.nst = std::min(p.nst, 3);
    FMM_CUDA(c, cudaEventRecord(c->ev_p2p, s));
    c->p2p_after_proj = true;
  }
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[9], s, cudaEventRecordExternal));
  if (f16)
    k_svd_proj_tc<true><<<std::min(up, c->num_sms), SP_THREADS, sp_smem(p.nst), s>>>(p, c->lv);
  else
    k_svd_proj_tc<false><<<std::min(up, c->num_sms), SP_THREADS, sp_smem(p.nst), s>>>(p, c->lv);
  FMM_CUDA(c, cudaGetLastError());
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[10], s, cudaEventRecordExternal));
  if (f16) {
    Exp16Args e;
    e.Yx = (const uint32_t*)c->svd_Yx;
    e.Uc = c->svd_Uc;
    e.partial = c->tc_partial;
    e.err = c->tc_err;
    e.tiles = c->tiles;
    e.ybound = c->svd_umax;
    e.ntiles = c->ntiles;
    e.kct = c->svd_kct;
    x_groups(c, &e.ngroups, &e.cpg);
    e.nhalf = ex_nhalf(cp);
    e.nh = cp / e.nhalf;
    e.cpad = cp;
    e.nst = x_nst(cp);
    if (near_with_proj && c->p2p_sched == 3) e.nst = 2;  // room for P2P blocks beside the expansion too
    e.chain = x_chain(c);
    e.uscale = c->svd_uscale;
    e.wait_ns = c->wait_ns;
    if ((int64_t)e.ngroups * c->ntiles * FMM_TILE * cp > c->tc_partial_cap)
      return set_err(c, FMM_ERR_STATE, "internal: M2L partial sums smaller than the expansion's groups");
    c->svd_x_groups = e.ngroups;
    const int ue = e.ngroups * c->ntiles * e.nh;
    if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[11], s, cudaEventRecordExternal));
    if (c->timing != 2 && c->p2p_priority && !near_with_proj) {
      FMM_CUDA(c, cudaEventRecord(c->ev_p2p, s));
      c->p2p_after_proj = true;
    }
    k_svd_expand16_tc<<<std::min(ue, c->num_sms), X_THREADS, e.nst * x_stage_bytes(cp) + x_fixed_bytes(cp), s>>>(
        e, c->lv);
    FMM_CUDA(c, cudaGetLastError());
    if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[12], s, cudaEventRecordExternal));
    if (mid) FMM_CUDA(c, cudaEventRecordWithFlags(mid, s, cudaEventRecordExternal));
    return launch_m2l_tc_reduce(c, s, c->tc_partial, -e.ngroups);
  }
  k_svd_exp_setup<<<dim3(c->ntiles, (FMM_NT_CLASS + EXS_CHUNK - 1) / EXS_CHUNK), FMM_TILE, 0, s>>>(c->tiles, c->tile_src, c->tile_act, c->tile_nact, c->lv, c->cls_t,
                                                 c->svd_ry, c->svd_yoff, c->svd_YS, c->svd_eslot, c->svd_ekch,
                                                 c->svd_yidx);
  ExpArgs e;
  e.tile_nact = c->tile_nact;
  e.eslot = c->svd_eslot;
  e.ekch = c->svd_ekch;
  e.yidx = c->svd_yidx;
  e.Y = (const float*)c->svd_Y;
  e.U = c->svd_Uhi;
  e.partial = c->tc_partial;
  e.err = c->tc_err;
  e.YS = c->svd_YS;
  e.ntiles = c->ntiles;
  e.cpad = cp;
  e.nhalf = ex_nhalf(cp);
  e.nh = cp / e.nhalf;
  e.nst = c->svd_tc_nst;
  e.tpa = std::max(4, std::min(16, c->ncoef / std::max(16, Rp)));
  e.acol = (uint32_t)(2 * e.nhalf);
  e.wait_ns = c->wait_ns;
  e.tmem_cols = 32;
  while ((int)e.tmem_cols < 2 * e.nhalf + 32 * e.nst) e.tmem_cols <<= 1;
  const int ue = c->ntiles * e.nh * EX_GROUPS;
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[11], s, cudaEventRecordExternal));
  // the P2P branch is released here: its blocks and the expansion's CTAs
  // become ready together and the expansion's (higher launch priority) are
  // placed first, one per SM, with P2P blocks in the room beside them
  if (c->timing != 2 && c->p2p_priority && !near_with_proj) {
    FMM_CUDA(c, cudaEventRecord(c->ev_p2p, s));
    c->p2p_after_proj = true;
  }
  k_svd_expand_tc<<<std::min(ue, c->num_sms), EX_THREADS, ex_smem(cp, e.nst), s>>>(e, c->lv);
  FMM_CUDA(c, cudaGetLastError());
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[12], s, cudaEventRecordExternal));
  if (mid) FMM_CUDA(c, cudaEventRecordWithFlags(mid, s, cudaEventRecordExternal));
  return launch_m2l_tc_reduce(c, s, c->tc_partial, EX_GT);
}

FMM_DEBUG_TAKE_FN(fmm_debug_take_m2l_svd_tc)

}  // namespace fmm
