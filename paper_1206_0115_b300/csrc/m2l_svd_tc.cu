// m2l_svd_tc.cu -- the SVD-compressed M2L (Sec. 2.1.2, "Improved M2L
// operator"; the factors and the Y layout are those of m2l_svd.cu) on the
// sm_103a tensor cores, mixed precision, 3xTF32 (hi*hi + hi*lo + lo*hi).
//
// k_svd_proj_tc -- projection from the sources.  Work unit = (tile of 128
//   cells of one level and class, group of up to G active source transfer
//   vectors).  The A operand is the tile's multipoles (one row per cell),
//   K = the cpad coefficients; B is the group's V_t factors side by side
//   (VT bank rows, N = ry_t each), so each A chunk is loaded once for the G
//   products.  Each t accumulates into its own columns of a TMEM accumulator
//   (two buffers of SP_ACC columns alternate between units) and the epilogue
//   writes them to the cells' Y rows.
// k_svd_expand_tc -- expansion at the targets, the layout of k_m2l_tc
//   (m2l_tc.cu): work unit = (target tile, half of the output columns, group
//   of EX_GT active transfer vectors); the A operand is gathered from the
//   sources' Y rows (ry_t values per t, split into TF32 hi/lo on the way into
//   tensor memory; an absent source gives zeros), B = U_t (mean-split rows)
//   by TMA, ry_t / 16 pipeline stages per t.  The tensor cores' FP32
//   accumulation does not round to nearest, so an accumulator takes at most
//   EX_TPA transfer vectors (a chain no longer than that of one full-rank
//   operator) before the epilogue adds it into FP32 running sums in shared
//   memory; k_m2l_tc_reduce adds a tile's group slices in FP64 and scales by
//   1/a.
// Roles per CTA (one CTA per SM, persistent): producer warps in sets of four
// (one thread per row), four epilogue warps (one per TMEM lane quarter), one
// MMA warp (one elected thread issues).  Every mbarrier wait is bounded in
// time; on expiry the CTA raises the error word, drains what it has in
// flight (bounded), frees TMEM and returns.
#include "tc_ptx.cuh"

namespace fmm {

using namespace tc;

namespace {

constexpr int KC = 16;          // K elements per pipeline stage (64-byte rows)
constexpr int MAXST = 4;        // pipeline stages at most

// ---- projection -------------------------------------------------------------
constexpr int SP_SETS = 2;                    // producer sets of four warps
constexpr int SP_EPI = 4 * SP_SETS;           // first epilogue warp
constexpr int SP_MMA = SP_EPI + 4;            // the MMA warp
constexpr int SP_THREADS = 32 * (SP_MMA + 1);
constexpr int SP_ACC = 192;                   // accumulator columns per buffer (two buffers)
constexpr int SP_MAXG = 12;                   // transfer vectors per unit at most

struct ProjArgs {
  const Tile* tiles;
  const int16_t* src_act;
  const int32_t* src_nact;
  const int16_t* src_t;
  const int32_t* t_ry;
  const int32_t* yoff;
  float* Y;
  int32_t* err;
  int64_t YS;
  int ntiles, G, ngroups, cpad, kchunks, nst, Rp;
};

struct Group {
  int n, cols;
  int slot[SP_MAXG], ry[SP_MAXG], off[SP_MAXG];
};

__device__ inline void proj_group(const ProjArgs& a, int cls, int tile, int a0, int a1, Group& g) {
  g.n = a1 - a0;
  int o = 0;
  for (int j = 0; j < SP_MAXG; ++j) {
    if (j < g.n) {
      const int k = a.src_act[(int64_t)tile * FMM_NT_CLASS + a0 + j];
      const int slot = a.src_t[cls * FMM_NT_CLASS + k];
      g.slot[j] = slot;
      g.ry[j] = a.t_ry[slot];
      g.off[j] = o;
      o += g.ry[j];
    }
  }
  g.cols = o;
}

__global__ void __launch_bounds__(SP_THREADS, 1)
k_svd_proj_tc(const __grid_constant__ CUtensorMap tm_vhi, const __grid_constant__ CUtensorMap tm_vlo, ProjArgs a,
              LevelPtrs lv, const float* __restrict__ Mhi, const float* __restrict__ Mlo) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t half_bytes = (uint32_t)SP_ACC * KC * 4;  // one half (hi or lo) of a stage's B
  const uint32_t stage_bytes = 2u * half_bytes;
  const uint32_t bars = base + (uint32_t)a.nst * stage_bytes;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (MAXST + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * MAXST + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * MAXST + 2 + b); };
  const uint32_t mma_done = bars + 8u * (2 * MAXST + 4);
  unsigned char* gbase = smem_raw + (base - raw);
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(gbase + (bars - base) + 8u * (2 * MAXST + 6));
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const uint32_t acol = 2u * SP_ACC, tmem_cols = 512;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXST; ++s) {
      mbar_init(full(s), FMM_TILE + 1);  // 128 A-row producers + the B copies' expect_tx
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
  const int nunits = a.ntiles * a.ngroups;

  if (warp < SP_EPI) {
    // ---------------------------------------------------------- producers
    const int set = warp >> 2;
    const int r = threadIdx.x & (FMM_TILE - 1);
    uint32_t it = 0, last = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      const int gi = unit / a.ntiles, tile = unit - gi * a.ntiles;
      const int nact = a.src_nact[tile];
      const int a0 = gi * a.G, a1 = min(nact, a0 + a.G);
      if (a0 >= a1) continue;
      const Tile tl = a.tiles[tile];
      Group g;
      if (r == 0) proj_group(a, tl.cls, tile, a0, a1, g);
      const int l = tl.level;
      const int64_t cellrow = lv.row_off[l] + (r < tl.count ? lv.cls[l][tl.first + r] : lv.ncell[l]);
      const float* ghi = Mhi + cellrow * a.cpad;
      const float* glo = Mlo + cellrow * a.cpad;
      const int kc0 = (set - (int)(it % SP_SETS) + SP_SETS) % SP_SETS;
      for (int kc = kc0; kc < a.kchunks; kc += SP_SETS) {
        const uint32_t j = it + (uint32_t)kc;
        uint32_t vh[16], vl[16];
        ld_v8(ghi + kc * KC, vh);
        ld_v8(ghi + kc * KC + 8, vh + 8);
        ld_v8(glo + kc * KC, vl);
        ld_v8(glo + kc * KC + 8, vl + 8);
        const int s = (int)(j % a.nst);
        const uint32_t ph = (j / a.nst) & 1u;
        if (!warp_wait(empty(s), ph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        const uint32_t st = base + (uint32_t)s * stage_bytes;
        if (r == 0) {
          mbar_expect_tx(full(s), 2u * (uint32_t)g.cols * KC * 4u);
          for (int q = 0; q < g.n; ++q)
            for (int b16 = 0; b16 < g.ry[q]; b16 += 16) {
              const uint32_t dst = st + (uint32_t)(g.off[q] + b16) * (KC * 4);
              const int y = g.slot[q] * a.Rp + b16;
              tma_2d(dst, &tm_vhi, kc * KC, y, full(s));
              tma_2d(dst + half_bytes, &tm_vlo, kc * KC, y, full(s));
            }
        }
        const uint32_t ta = tmem + ((uint32_t)(r & ~31) << 16) + acol + (uint32_t)s * 32u;
        tmem_st16(ta, vh);
        tmem_st16(ta + 16u, vl);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        mbar_arrive(full(s));
        last = j + 1;
      }
      it += (uint32_t)a.kchunks;
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
    if (!ok && r == 0) {
      for (uint32_t j = last > (uint32_t)a.nst ? last - a.nst : 0; j < last; ++j)
        if ((int)(j % SP_SETS) == set) mbar_wait(full((int)(j % a.nst)), (j / a.nst) & 1u);
    }
    __syncwarp();
  } else if (warp == SP_MMA) {
    // ---------------------------------------------------------- MMA issuer
    uint32_t it = 0, uu = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      const int gi = unit / a.ntiles, tile = unit - gi * a.ntiles;
      const int nact = a.src_nact[tile];
      const int a0 = gi * a.G, a1 = min(nact, a0 + a.G);
      if (a0 >= a1) continue;
      const Tile tl = a.tiles[tile];
      Group g;
      proj_group(a, tl.cls, tile, a0, a1, g);
      const int b = (int)(uu & 1u);
      if (!warp_wait(acc_empty(b), ((uu >> 1) & 1u) ^ 1u, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d0 = tmem + (uint32_t)(b * SP_ACC);
      for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
        const int s = (int)(it % a.nst);
        const uint32_t ph = (it / a.nst) & 1u;
        if (!warp_wait(full(s), ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t st = base + (uint32_t)s * stage_bytes;
          const uint32_t a_hi = tmem + acol + (uint32_t)s * 32u;
          for (int q = 0; q < g.n; ++q) {
            const uint32_t idesc = idesc_tf32(FMM_TILE, g.ry[q]);
            const uint32_t d = d0 + (uint32_t)g.off[q];
            const uint32_t bq = st + (uint32_t)g.off[q] * (KC * 4);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t ahi = a_hi + ks * 8u, alo = a_hi + 16u + ks * 8u;
              const uint64_t bhi = sdesc_sw64(bq + ks * 32u);
              const uint64_t blo = sdesc_sw64(bq + half_bytes + ks * 32u);
              mma_tf32_ta(d, ahi, bhi, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
              mma_tf32_ta(d, ahi, blo, idesc, 1u);
              mma_tf32_ta(d, alo, bhi, idesc, 1u);
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
  } else if (warp < SP_MMA) {
    // ---------------------------------------------------------- epilogue
    const int qd = warp & 3, row = qd * 32 + lane;
    uint32_t uu = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      const int gi = unit / a.ntiles, tile = unit - gi * a.ntiles;
      const int nact = a.src_nact[tile];
      const int a0 = gi * a.G, a1 = min(nact, a0 + a.G);
      if (a0 >= a1) continue;
      const Tile tl = a.tiles[tile];
      Group g;
      proj_group(a, tl.cls, tile, a0, a1, g);
      const int b = (int)(uu & 1u);
      if (!warp_wait(acc_full(b), (uu >> 1) & 1u, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int l = tl.level;
      const bool valid = row < tl.count;
      const int64_t cellrow = lv.row_off[l] + (valid ? lv.cls[l][tl.first + row] : lv.ncell[l]);
      const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * SP_ACC);
      for (int q = 0; q < g.n; ++q) {
        float* y = a.Y + cellrow * a.YS + a.yoff[tl.cls * FMM_NT + g.slot[q]];
        for (int c16 = 0; c16 < g.ry[q]; c16 += 16) {
          float v[16];
          tmem_ld16(tb + (uint32_t)(g.off[q] + c16), v);
          if (valid) {
            float4* o = (float4*)(y + c16);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
            o[2] = make_float4(v[8], v[9], v[10], v[11]);
            o[3] = make_float4(v[12], v[13], v[14], v[15]);
          }
        }
      }
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
constexpr int EX_TPA = 4;    // transfer vectors per accumulator before it is drained

struct ExpArgs {
  const Tile* tiles;
  const int32_t* tile_src;
  const int16_t* tile_act;
  const int32_t* tile_nact;
  const int16_t* cls_t;
  const int32_t* t_ry;
  const int32_t* yoff;
  const float* Y;
  float* partial;  // [group][tile][128][cpad]
  int32_t* err;
  int64_t YS;
  int ntiles, cpad, nh, nhalf, nst;
  uint32_t acol, tmem_cols;
};

__device__ inline void exp_unit(const ExpArgs& a, int u, int& g, int& h, int& tile) {
  const int per_g = a.ntiles * a.nh;
  g = u / per_g;
  const int rem = u - g * per_g;
  h = rem / a.ntiles;
  tile = rem - h * a.ntiles;
}

__global__ void __launch_bounds__(EX_THREADS, 1)
k_svd_expand_tc(const __grid_constant__ CUtensorMap tm_uhi, const __grid_constant__ CUtensorMap tm_ulo, ExpArgs a,
                LevelPtrs lv) {
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
    // them into TF32 hi/lo and writes them into its TMEM lane; one thread
    // issues the B slab (U_t rows of this column half x 16 rank columns).
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
      const Tile tl = a.tiles[tile];
      const int l = tl.level, zero = lv.ncell[l];
      const int64_t rbase = lv.row_off[l];
      for (int ai = a0; ai < a1 && ok; ++ai) {
        const int k = a.tile_act[(int64_t)tile * FMM_NT_CLASS + ai];
        const int slot = a.cls_t[tl.cls * FMM_NT_CLASS + k];
        const int kch = a.t_ry[slot] / KC;
        const int kc0 = (set - (int)(it % EX_SETS) + EX_SETS) % EX_SETS;
        if (kc0 < kch) {
          const int src = a.tile_src[((int64_t)tile * FMM_NT_CLASS + k) * FMM_TILE + r];
          const float* yr =
              src == zero ? nullptr : a.Y + (rbase + src) * a.YS + a.yoff[(lv.key[l][src] & 7) * FMM_NT + slot];
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
            if (!warp_wait(empty(s), ph ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t st = base + (uint32_t)s * stage_bytes;
            if (r == 0) {
              mbar_expect_tx(full(s), 2u * b_bytes);
              const int y = slot * a.cpad + h * a.nhalf;
              tma_2d(st, &tm_uhi, kc * KC, y, full(s));
              tma_2d(st + b_bytes, &tm_ulo, kc * KC, y, full(s));
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
      const Tile tl = a.tiles[tile];
      for (int ag = a0; ag < a1 && ok; ag += EX_TPA, ++tt) {
        const int ae = min(a1, ag + EX_TPA);
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_empty(b), ((tt >> 1) & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * a.nhalf);
        bool first = true;
        for (int ai = ag; ai < ae && ok; ++ai) {
          const int k = a.tile_act[(int64_t)tile * FMM_NT_CLASS + ai];
          const int kch = a.t_ry[a.cls_t[tl.cls * FMM_NT_CLASS + k]] / KC;
          for (int kc = 0; kc < kch; ++kc, ++it) {
            const int s = (int)(it % a.nst);
            const uint32_t ph = (it / a.nst) & 1u;
            if (!warp_wait(full(s), ph, abort_flag)) {
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
                const uint64_t bhi = sdesc_sw64(st + ks * 32u);
                const uint64_t blo = sdesc_sw64(st + b_bytes + ks * 32u);
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
      for (int ag = a0; ag < a1; ag += EX_TPA, ++tt) {
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_full(b), (tt >> 1) & 1u, abort_flag)) {
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
        *(float4*)(out + c) = make_float4(S[c * FMM_TILE + row], S[(c + 1) * FMM_TILE + row],
                                          S[(c + 2) * FMM_TILE + row], S[(c + 3) * FMM_TILE + row]);
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

int sp_group(int Rp) { return std::max(1, std::min(SP_MAXG, SP_ACC / Rp)); }
int sp_stage_bytes() { return 2 * SP_ACC * KC * 4; }
int sp_smem(int nst) { return nst * sp_stage_bytes() + 1024 + 256; }
int ex_nhalf(int cp) { return cp > 256 ? cp / 2 : cp; }
int ex_stage_bytes(int cp) { return 2 * ex_nhalf(cp) * KC * 4; }
int ex_smem(int cp, int nst) { return nst * ex_stage_bytes(cp) + ex_nhalf(cp) * FMM_TILE * 4 + 1024 + 256; }

}  // namespace

// Mixed precision with the rank padding of 16 (always) and output columns
// that fit two TMEM accumulators beside the A stages: order <= 7.
bool m2l_svd_tc_supported(const Ctx* c) {
  const int nhalf = ex_nhalf(c->cpad);
  return c->cpad % 32 == 0 && nhalf <= 256 && nhalf % 16 == 0 && 2 * nhalf + 32 * 2 <= 512 && c->svd_rp <= SP_ACC;
}

// Tensor maps of the compressed factor banks, the partial-sum buffer and the
// kernels' shared-memory limits (before an evaluation is captured).
fmm_status m2l_svd_tc_prepare(Ctx* c) {
  if (c->ntiles == 0) return FMM_OK;
  const int cp = c->cpad, Rp = c->svd_rp, nhalf = ex_nhalf(cp);
  const int64_t need = (int64_t)c->ntiles * EX_GROUPS * FMM_TILE * cp;
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
    FMM_CUDA(c, cudaMemset(c->tc_err, 0, 64));
  }
  if (!c->tc_err_h) return set_err(c, FMM_ERR_STATE, "internal: no host error word");
  if (c->tm_svd_ptr != c->svd_VThi) {
    bool ok = encode_2d((CUtensorMap*)c->tm_vthi, c->svd_VThi, cp, (uint64_t)FMM_NT * Rp, KC, 16) &&
              encode_2d((CUtensorMap*)c->tm_vtlo, c->svd_VTlo, cp, (uint64_t)FMM_NT * Rp, KC, 16) &&
              encode_2d((CUtensorMap*)c->tm_uhi, c->svd_Uhi, Rp, (uint64_t)FMM_NT * cp, KC, nhalf) &&
              encode_2d((CUtensorMap*)c->tm_ulo, c->svd_Ulo, Rp, (uint64_t)FMM_NT * cp, KC, nhalf);
    if (!ok) return set_err(c, FMM_ERR_CUDA, "compressed M2L tensor path: cuTensorMapEncodeTiled failed");
    c->tm_svd_ptr = c->svd_VThi;
  }
  // stages: shared memory and the TMEM columns beside the accumulators
  int nst = (227 * 1024 - ex_smem(cp, 0)) / ex_stage_bytes(cp);
  nst = std::min(nst, (512 - 2 * nhalf) / 32);
  nst = std::min(nst, MAXST);
  const int nst_p = std::min(MAXST, (512 - 2 * SP_ACC) / 32);
  if (nst < 2 || nst_p < 2) return set_err(c, FMM_ERR_ARG, "compressed M2L tensor path: no room for 2 stages");
  c->svd_tc_nst = nst;
  if (sp_smem(nst_p) > c->svd_tc_smem_set[0]) {
    FMM_CUDA(c, cudaFuncSetAttribute(k_svd_proj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sp_smem(nst_p)));
    c->svd_tc_smem_set[0] = sp_smem(nst_p);
  }
  if (ex_smem(cp, nst) > c->svd_tc_smem_set[1]) {
    FMM_CUDA(c, cudaFuncSetAttribute(k_svd_expand_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     ex_smem(cp, nst)));
    c->svd_tc_smem_set[1] = ex_smem(cp, nst);
  }
  if (c->num_sms == 0) FMM_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
  return FMM_OK;
}

// Projection of every tile, then the expansion and (after `mid`) the FP64
// reduction of its partial sums.
fmm_status launch_m2l_svd_tc(Ctx* c, cudaStream_t s, cudaEvent_t mid) {
  if (c->ntiles == 0) return FMM_OK;
  const int cp = c->cpad, Rp = c->svd_rp;
  ProjArgs p;
  p.tiles = c->tiles;
  p.src_act = c->src_act;
  p.src_nact = c->src_nact;
  p.src_t = c->src_t;
  p.t_ry = c->svd_ry;
  p.yoff = c->svd_yoff;
  p.Y = (float*)c->svd_Y;
  p.err = c->tc_err;
  p.YS = c->svd_YS;
  p.ntiles = c->ntiles;
  p.G = sp_group(Rp);
  p.ngroups = (FMM_NT_CLASS + p.G - 1) / p.G;
  p.cpad = cp;
  p.kchunks = cp / KC;
  p.nst = std::min(MAXST, (512 - 2 * SP_ACC) / 32);
  p.Rp = Rp;
  const int up = p.ntiles * p.ngroups;
  k_svd_proj_tc<<<std::min(up, c->num_sms), SP_THREADS, sp_smem(p.nst), s>>>(
      *(const CUtensorMap*)c->tm_vthi, *(const CUtensorMap*)c->tm_vtlo, p, c->lv, c->Mhi, c->Mlo);
  FMM_CUDA(c, cudaGetLastError());
  ExpArgs e;
  e.tiles = c->tiles;
  e.tile_src = c->tile_src;
  e.tile_act = c->tile_act;
  e.tile_nact = c->tile_nact;
  e.cls_t = c->cls_t;
  e.t_ry = c->svd_ry;
  e.yoff = c->svd_yoff;
  e.Y = (const float*)c->svd_Y;
  e.partial = c->tc_partial;
  e.err = c->tc_err;
  e.YS = c->svd_YS;
  e.ntiles = c->ntiles;
  e.cpad = cp;
  e.nhalf = ex_nhalf(cp);
  e.nh = cp / e.nhalf;
  e.nst = c->svd_tc_nst;
  e.acol = (uint32_t)(2 * e.nhalf);
  e.tmem_cols = 32;
  while ((int)e.tmem_cols < 2 * e.nhalf + 32 * e.nst) e.tmem_cols <<= 1;
  const int ue = c->ntiles * e.nh * EX_GROUPS;
  k_svd_expand_tc<<<std::min(ue, c->num_sms), EX_THREADS, ex_smem(cp, e.nst), s>>>(
      *(const CUtensorMap*)c->tm_uhi, *(const CUtensorMap*)c->tm_ulo, e, c->lv);
  FMM_CUDA(c, cudaGetLastError());
  if (mid) FMM_CUDA(c, cudaEventRecordWithFlags(mid, s, cudaEventRecordExternal));
  return launch_m2l_tc_reduce(c, s, c->tc_partial, EX_GT);
}

}  // namespace fmm
