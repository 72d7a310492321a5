// m2l_tc.cu -- M2L (Sec. 2.1.2) on the sm_103a tensor cores.
//
// For one level and one child class every target cell T needs
//     L_T = (1/a) sum_{t in the class's 189 transfer vectors} K_t M_{T+t},
// a GEMM whose rows are target cells (128 per tile), whose columns are the
// output coefficients (the mean-split bank: deviations + cell mean, padded to
// cpad), and whose K dimension runs over (t, source coefficient).  The A
// operand is gathered: row r of a tile holds M of the source cell T_r + t
// (the level's zero row when absent).
//
// Work unit = (tile, half of the output columns, group of TC_GT consecutive
// active transfer vectors).  The tensor cores' FP32 accumulation rounds
// toward zero, so its error grows linearly with the accumulation chain
// (measured: x11 longer chain, x13 larger error).  Each transfer vector
// therefore gets a fresh TMEM accumulator (one of two, alternating), which the
// epilogue adds into a running sum in shared memory with ordinary FP32
// round-to-nearest additions while the next transfer vector accumulates; a
// unit's sum goes to its own partial slice and k_m2l_tc_reduce adds the
// slices of a tile in FP64.
//
// Precision: 3xTF32 -- multipoles and operators are TF32 hi/lo pairs and each
// K-step issues hi*hi + hi*lo + lo*hi into the same FP32 accumulator.
//
// Roles (one CTA per SM, 544 threads, persistent over the units):
//   warps 0-11 producers in three sets of four warps taking turns per stage
//              (16 source coefficients of one t): thread r loads its target
//              row's 16 multipole coefficients (hi and lo, two 32-byte loads
//              each) and writes them into its own TMEM lane r (tcgen05.st), so
//              the gathered operand A never passes through shared memory; one
//              thread also issues the B slab K_t[0..cpad)[k0..k0+16) as 2-D
//              tiled TMA loads into shared memory (64-byte swizzle).  The MMA
//              reads A from TMEM and B from shared memory;
//   warps 12-15 epilogue (one per TMEM lane quarter): tcgen05.ld of each
//              accumulator into the running sums, the sums to the unit's slice;
//   warp 16    TMEM allocation and the tcgen05.mma issuer (one thread).
// Every mbarrier wait is bounded in time; on expiry the CTA raises the error
// word, drains what it has in flight (again bounded), frees TMEM and returns.
#include "tc_ptx.cuh"

namespace fmm {

using namespace tc;

namespace {

constexpr int TC_SETS = 3;                      // producer sets of 4 warps, one stage each in turn
constexpr int TC_EPI_WARP = 4 * TC_SETS;         // first of the 4 epilogue warps
constexpr int TC_MMA_WARP = TC_EPI_WARP + 4;     // the MMA issuer
constexpr int TC_THREADS = 32 * (TC_MMA_WARP + 1);
constexpr int TC_KC = 16;      // K elements per stage (64-byte rows)
constexpr int TC_MAXST = 4;    // pipeline stages at most
constexpr int TC_A_BYTES = FMM_TILE * TC_KC * 4;   // one half (hi or lo) of A: 8 KB
struct TcArgs {
  const Tile* tiles;
  const int32_t* tile_src;
  const int16_t* tile_act;
  const int32_t* tile_nact;
  const int16_t* cls_t;
  float* partial;  // [group][tile][128][cpad]
  int32_t* err;    // nonzero after a timed-out wait
  int ntiles, groups, gt, cpad, nh, nhalf, kchunks, nst;
  int lev_ops;         // one operator bank per level 2.. (kernels with c > 0)
  // FP16 operands: max |M| per (problem + 1, level) (float bits; a target
  // row's gathered multipoles, all of its own problem, are scaled by
  // pow2_scale of it) and the operator banks' scale, undone per row
  const uint32_t* mmax;
  float kscale;
  uint32_t acol;       // first TMEM column of the A stages (after the two accumulators)
  uint32_t tmem_cols;  // power of two >= 2 * nhalf + 32 * nst
  uint64_t wait_ns;    // limit of a pipeline wait (fmm_set_wait_limit)
};

// Work unit u -> (group g, column half h, tile): groups outermost so that the
// CTAs running at the same time share transfer vectors (operator slabs stay
// in L2).
__device__ inline void unit_coords(const TcArgs& a, int u, int& g, int& h, int& tile) {
  const int per_g = a.ntiles * a.nh;
  g = u / per_g;
  const int rem = u - g * per_g;
  h = rem / a.ntiles;
  tile = rem - h * a.ntiles;
}

// pow2_scale of the max |M| of the problem of target row r of a tile.
__device__ inline float row_mscale(const TcArgs& a, const LevelPtrs& lv, const Tile& tl, int r) {
  if (r >= tl.count) return 1.f;
  const int prob = problem_of(lv, tl.level, lv.cls[tl.level][tl.first + r]);
  return pow2_scale(__uint_as_float(a.mmax[(prob + 1) * FMM_MAX_LEVELS + tl.level]));
}

// FP16 form: the max |M| of each (problem, level 2..), over the multipole
// rows of the levels (one warp per row; a level's zero row is skipped).
__global__ void __launch_bounds__(256)
k_m_absmax(LevelPtrs lv, int lmin, int lmax, int cpad, const float* __restrict__ Mhi, const float* __restrict__ Mlo,
           uint32_t* __restrict__ mmax) {
  const int64_t r0 = lv.row_off[lmin], r1 = lv.row_off[lmax] + lv.ncell[lmax] + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t r = r0 + (int64_t)blockIdx.x * 8 + warp; r < r1; r += (int64_t)gridDim.x * 8) {
    int l = lmin;
    while (l < lmax && r >= lv.row_off[l + 1]) ++l;
    const int64_t cell = r - lv.row_off[l];
    if (cell >= lv.ncell[l]) continue;  // the level's zero row (warp-uniform)
    float m = 0.f;
    for (int k = lane; k < cpad; k += 32) m = fmaxf(m, fabsf(Mhi[r * cpad + k] + Mlo[r * cpad + k]));
    const uint32_t mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));  // non-negative floats order like bits
    const int prob = problem_of(lv, l, (int)cell);
    if (lane == 0 && mb) atomicMax(mmax + (prob + 1) * FMM_MAX_LEVELS + l, mb);
  }
}

// F16: operands FP16 hi/lo pairs (32 coefficients per stage, two MMAs of
// K = 16, at twice the TF32 rate; operator banks as rows of packed FP16
// pairs, copied by the same float32 tensor maps as 32-bit words); otherwise
// TF32 hi/lo pairs.
template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_m2l_tc(const __grid_constant__ CUtensorMap tm_khi, const __grid_constant__ CUtensorMap tm_klo, TcArgs a,
         LevelPtrs lv, const float* __restrict__ Mhi, const float* __restrict__ Mlo) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
  const uint32_t b_bytes = (uint32_t)a.nhalf * TC_KC * 4;      // one half (hi or lo) of B
  const uint32_t stage_bytes = 2u * b_bytes;
  const uint32_t sum_off = (uint32_t)a.nst * stage_bytes;     // running sums S[col][row], FP32
  const uint32_t bars = base + sum_off + (uint32_t)a.nhalf * FMM_TILE * 4u;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (TC_MAXST + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * TC_MAXST + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * TC_MAXST + 2 + b); };
  const uint32_t mma_done = bars + 8u * (2 * TC_MAXST + 4);
  unsigned char* gbase = smem_raw + (base - raw);
  float* S = (float*)(gbase + sum_off);
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(gbase + (bars - base) + 8u * (2 * TC_MAXST + 6));
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_MAXST; ++s) {
      mbar_init(full(s), FMM_TILE + 1);  // 128 A-row producers + the B copy's expect_tx
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
  if (warp == TC_MMA_WARP) {
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
  const int nunits = a.ntiles * a.nh * a.groups;

  if (warp < TC_EPI_WARP) {
    // ------------------------------------------------------------ producers
    // Set k (warps 4k .. 4k+3) fills the stages j with j % TC_SETS == k, so
    // three stages' worth of gathered loads are in flight at once.  Thread r
    // of a set gathers A row r (the source multipole of target r for the
    // current t) with plain 16-byte loads and stores it in the 64-byte swizzle
    // pattern: chunk c of row r goes to chunk c ^ ((r >> 1) & 3).
    const int set = warp >> 2;
    const int r = threadIdx.x & (FMM_TILE - 1);
    const uint32_t rsw = (uint32_t)((r >> 1) & 3);
    uint32_t it = 0, last = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, h, tile;
      unit_coords(a, unit, g, h, tile);
      const int nact = a.tile_nact[tile];
      const int a0 = g * a.gt, a1 = min(nact, a0 + a.gt);
      if (a0 >= a1) continue;
      const Tile tl = a.tiles[tile];
      const int64_t rbase = lv.row_off[tl.level];
      const float msc = F16 ? row_mscale(a, lv, tl, r) : 1.f;
      for (int ai = a0; ai < a1 && ok; ++ai) {
        // stages of this transfer vector owned by the set
        const uint32_t kc0 = (uint32_t)((set - (int)(it % TC_SETS) + TC_SETS) % TC_SETS);
        if ((int)kc0 >= a.kchunks) {
          it += a.kchunks;
          continue;
        }
        const int k = a.tile_act[(int64_t)tile * FMM_NT_CLASS + ai];
        const int slot = a.cls_t[tl.cls * FMM_NT_CLASS + k] + (a.lev_ops ? (tl.level - 2) * FMM_NT : 0);
        const int64_t src = rbase + a.tile_src[((int64_t)tile * FMM_NT_CLASS + k) * FMM_TILE + r];
        const float* ghi = Mhi + src * a.cpad;
        const float* glo = Mlo + src * a.cpad;
        for (int kc = (int)kc0; kc < a.kchunks; kc += TC_SETS) {
          const uint32_t j = it + (uint32_t)kc;
          uint32_t vh[16], vl[16];
          if (F16) {
            // 32 coefficients: M = hi + lo, scaled, split into FP16 pairs
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t wh[8], wl[8];
              ld_v8((const float*)ghi + kc * 32 + 8 * q, wh);
              ld_v8((const float*)glo + kc * 32 + 8 * q, wl);
#pragma unroll
              for (int i = 0; i < 4; ++i)
                split_h2((__uint_as_float(wh[2 * i]) + __uint_as_float(wl[2 * i])) * msc,
                         (__uint_as_float(wh[2 * i + 1]) + __uint_as_float(wl[2 * i + 1])) * msc, vh[4 * q + i],
                         vl[4 * q + i]);
            }
          } else {
            ld_v8((const float*)ghi + kc * TC_KC, vh);
            ld_v8((const float*)ghi + kc * TC_KC + 8, vh + 8);
            ld_v8((const float*)glo + kc * TC_KC, vl);
            ld_v8((const float*)glo + kc * TC_KC + 8, vl + 8);
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
            const int y = slot * a.cpad + h * a.nhalf;
            // x in 32-bit words: 16 per stage (TF32: 16 values; FP16: 32 values)
            tma_2d(st, &tm_khi, kc * 16, y, full(s));
            tma_2d(st + b_bytes, &tm_klo, kc * 16, y, full(s));
          }
          // A row r -> TMEM lane r: hi in columns [0, 16), lo in [16, 32) of the stage's slot
          const uint32_t ta = tmem + ((uint32_t)(r & ~31) << 16) + a.acol + (uint32_t)s * 32u;
          tmem_st16(ta, vh);
          tmem_st16(ta + 16u, vl);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          mbar_arrive(full(s));
          last = j + 1;
        }
        it += a.kchunks;
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
    // let the operator copies this set issued land before the CTA leaves (bounded)
    if (!ok && r == 0) {
      for (uint32_t j = last > (uint32_t)a.nst ? last - a.nst : 0; j < last; ++j)
        if ((int)(j % TC_SETS) == set) mbar_wait(full((int)(j % a.nst)), (j / a.nst) & 1u);
    }
    __syncwarp();
  } else if (warp == TC_MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    // one accumulator per transfer vector, alternating between two TMEM
    // buffers so that the epilogue drains t while t+1 accumulates
    uint32_t it = 0, tt = 0;
    bool ok = true;
    const uint32_t idesc = F16 ? idesc_f16(FMM_TILE, a.nhalf) : idesc_tf32(FMM_TILE, a.nhalf);
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, h, tile;
      unit_coords(a, unit, g, h, tile);
      const int nact = a.tile_nact[tile];
      const int a0 = g * a.gt, a1 = min(nact, a0 + a.gt);
      if (a0 >= a1) continue;
      for (int ai = a0; ai < a1 && ok; ++ai, ++tt) {
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_empty(b), ((tt >> 1) & 1u) ^ 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * a.nhalf);
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
            const uint32_t ahi0 = tmem + a.acol + (uint32_t)s * 32u;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t ahi = ahi0 + ks * 8u, alo = ahi0 + 16u + ks * 8u;
              const uint64_t bhi = sdesc_sw64(st + ks * 32u);
              const uint64_t blo = sdesc_sw64(st + b_bytes + ks * 32u);
              if (F16) {
                mma_f16_ta(d, ahi, bhi, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                mma_f16_ta(d, ahi, blo, idesc, 1u);
                mma_f16_ta(d, alo, bhi, idesc, 1u);
              } else {
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
  } else if (warp < TC_MMA_WARP) {
    // ------------------------------------------------------------ epilogue (warps 12-15)
    // S[col][row] += accumulator of each transfer vector (FP32, round to
    // nearest); at the end of the unit S goes to the unit's partial slice.
    const int q = warp & 3, row = q * 32 + lane;
    uint32_t tt = 0;
    bool ok = true;
    for (int unit = blockIdx.x; unit < nunits && ok; unit += gridDim.x) {
      int g, h, tile;
      unit_coords(a, unit, g, h, tile);
      const int nact = a.tile_nact[tile];
      const int a0 = g * a.gt, a1 = min(nact, a0 + a.gt);
      if (a0 >= a1) continue;
      for (int ai = a0; ai < a1; ++ai, ++tt) {
        const int b = (int)(tt & 1u);
        if (!warp_wait(acc_full(b), (tt >> 1) & 1u, abort_flag, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * a.nhalf);
        const bool first = ai == a0;
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
      float* out = a.partial + (((int64_t)g * a.ntiles + tile) * FMM_TILE + row) * a.cpad + h * a.nhalf;
      // F16: back from the operands' scales (powers of two: exact)
      const float inv = F16 ? 1.f / (row_mscale(a, lv, a.tiles[tile], row) * a.kscale) : 1.f;
      for (int c = 0; c < a.nhalf; c += 4)
        *(float4*)(out + c) = make_float4(S[c * FMM_TILE + row] * inv, S[(c + 1) * FMM_TILE + row] * inv,
                                          S[(c + 2) * FMM_TILE + row] * inv, S[(c + 3) * FMM_TILE + row] * inv);
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == TC_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// L_T[m] = (1/a) * sum over the tile's groups of the partial sums: at most
// three FP32 slices, added in FP32.  Block (tile, slice): rows 16*slice ..
// 16*slice+15 of the tile, four coefficients per thread.
constexpr int RED_BATCH = 8;  // partial slices loaded at once by the reduction

__global__ void __launch_bounds__(256)
k_m2l_tc_reduce(const Tile* __restrict__ tiles, const int32_t* __restrict__ tile_nact, LevelPtrs lv, int ntiles,
                int gt, int cpad, int ncol, const float* __restrict__ partial, float* __restrict__ L,
                const double* __restrict__ box, double ks) {
  const int tile = blockIdx.x, r0 = blockIdx.y * 16;
  const Tile tl = tiles[tile];
  if (r0 >= tl.count) return;
  const int nrow = min(16, tl.count - r0);
  // gt > 0: slices of gt transfer vectors each (only as many as the tile has);
  // gt <= 0: -gt slices for every tile
  const int ng = gt > 0 ? (tile_nact[tile] + gt - 1) / gt : -gt;
  const float inv_a = (float)kernel_scale(ldexp(1.0, tl.level + 1) / box[3], ks);
  const int64_t rbase = lv.row_off[tl.level];
  const int nq = (ncol + 3) / 4;  // float4 columns (cpad is a multiple of 32)
  for (int idx = threadIdx.x; idx < nrow * nq; idx += blockDim.x) {
    const int row = r0 + idx / nq, c4 = 4 * (idx % nq);
    // the slices' loads issued together (up to RED_BATCH in flight), then
    // added in slice order
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int g0 = 0; g0 < ng; g0 += RED_BATCH) {
      float4 v[RED_BATCH];
#pragma unroll
      for (int k = 0; k < RED_BATCH; ++k)
        if (g0 + k < ng)
          v[k] = *(const float4*)&partial[(((int64_t)(g0 + k) * ntiles + tile) * FMM_TILE + row) * cpad + c4];
#pragma unroll
      for (int k = 0; k < RED_BATCH; ++k)
        if (g0 + k < ng) {
          s.x += v[k].x;
          s.y += v[k].y;
          s.z += v[k].z;
          s.w += v[k].w;
        }
    }
    const int cell = lv.cls[tl.level][tl.first + row];
    *(float4*)&L[(rbase + cell) * cpad + c4] = make_float4(s.x * inv_a, s.y * inv_a, s.z * inv_a, s.w * inv_a);
  }
}

}  // namespace

// The tensor-core path serves the mixed precision when the accumulator
// (cpad FP32 columns) fits the 512 TMEM columns: order <= 7.
bool m2l_tc_supported(const Ctx* c) { return c->cpad <= 512 && c->cpad % 32 == 0; }

namespace {
constexpr int TC_GT = 64;  // transfer vectors per work unit
constexpr int TC_GROUPS = (FMM_NT_CLASS + TC_GT - 1) / TC_GT;
// Column halves per tile: two when one accumulator of cp columns is wider
// than an MMA (256) or when the two accumulators would leave TMEM room for
// fewer A stages than there are producer sets.  A set waits on its stage's
// barrier by phase parity, which is only unambiguous while it runs at most
// one phase ahead of the MMA; with fewer stages than sets it could run two
// ahead (p = 6: cp = 224 leaves room for two stages).
int tc_nh(int cp) { return (cp > 256 || 2 * cp + 32 * TC_SETS > 512) ? 2 : 1; }
int tc_stage_bytes(int cp) { return 2 * (cp / tc_nh(cp)) * TC_KC * 4; }
int tc_fixed_bytes(int cp) { return (cp / tc_nh(cp)) * FMM_TILE * 4 + 1024 + 256; }  // sums, alignment, barriers
}  // namespace

// Buffers, tensor maps and kernel attributes of the tensor-core M2L for the
// current tree: called before an evaluation is captured or launched (it may
// allocate, which a stream capture forbids).
fmm_status m2l_tc_prepare(Ctx* c) {
  if (c->ntiles == 0) return FMM_OK;
  const int cp = c->cpad;
  const int nh = tc_nh(cp), nhalf = cp / nh;
  if (nhalf % 16 != 0 || nhalf > 256) return set_err(c, FMM_ERR_ARG, "M2L tensor path: unsupported cpad %d", cp);
  const int64_t need = (int64_t)c->ntiles * TC_GROUPS * FMM_TILE * cp;
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
  const int nb = op_banks(c);
  const bool f16 = c->ops32_f16;
  if (c->tm_khi_ptr != c->Khi || c->tm_khi_nb != nb || c->tm_khi_f16 != f16) {
    // rows of cpad values: TF32 (cpad words) or packed FP16 pairs (cpad / 2 words), 16 words per box row
    const uint64_t rows = (uint64_t)FMM_NT * cp * nb, words = f16 ? cp / 2 : cp;
    bool ok = encode_2d((CUtensorMap*)c->tm_khi, c->Khi, words, rows, 16, nhalf) &&
              encode_2d((CUtensorMap*)c->tm_klo, c->Klo, words, rows, 16, nhalf);
    if (!ok) return set_err(c, FMM_ERR_CUDA, "M2L tensor path: cuTensorMapEncodeTiled failed");
    c->tm_khi_ptr = c->Khi;
    c->tm_khi_nb = nb;
    c->tm_khi_f16 = f16;
  }
  if (f16 && !c->tc_mmax) {  // max |M| per (problem + 1, level): every batch size
    void* p;
    FMM_TRY(dalloc(c, &p, sizeof(uint32_t) * (FMM_MAX_BATCH + 1) * FMM_MAX_LEVELS));
    c->tc_mmax = (uint32_t*)p;
  }
  int nst = (227 * 1024 - tc_fixed_bytes(cp)) / tc_stage_bytes(cp);
  const int tmem_stages = (512 - 2 * (cp / tc_nh(cp))) / 32;  // A stages beside the two accumulators
  if (nst > tmem_stages) nst = tmem_stages;
  if (nst > TC_MAXST) nst = TC_MAXST;
  if (nst < TC_SETS) return set_err(c, FMM_ERR_ARG, "M2L tensor path: fewer stages than producer sets for cpad %d", cp);
  c->tc_nst = nst;
  const int smem = nst * tc_stage_bytes(cp) + tc_fixed_bytes(cp);
  FMM_TRY(raise_smem_limit(c, f16 ? (const void*)k_m2l_tc<true> : (const void*)k_m2l_tc<false>, smem));
  if (c->num_sms == 0) FMM_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
  return FMM_OK;
}

// L_T = (1/a) * (sum of the partial slices) for every tile (see k_m2l_tc_reduce).
fmm_status launch_m2l_tc_reduce(Ctx* c, cudaStream_t s, const float* partial, int gt) {
  k_m2l_tc_reduce<<<dim3(c->ntiles, FMM_TILE / 16), 256, 0, s>>>(c->tiles, c->tile_nact, c->lv, c->ntiles, gt,
                                                                  c->cpad, c->ncoef + 1, partial, c->L32, c->box, c->kernel_s);
  return cuda_err(c, cudaGetLastError(), "M2L reduction launch");
}

// Launches the tensor-core M2L over every tile of every level and the
// reduction of its partial sums; `mid` (optional) is recorded between them.
fmm_status launch_m2l_tc(Ctx* c, cudaStream_t s, cudaEvent_t mid) {
  if (c->ntiles == 0) return FMM_OK;
  const int cp = c->cpad;
  const int nh = tc_nh(cp), nhalf = cp / nh;
  TcArgs a;
  a.tiles = c->tiles;
  a.tile_src = c->tile_src;
  a.tile_act = c->tile_act;
  a.tile_nact = c->tile_nact;
  a.cls_t = c->cls_t;
  a.partial = c->tc_partial;
  a.err = c->tc_err;
  a.wait_ns = c->wait_ns;
  a.ntiles = c->ntiles;
  a.groups = TC_GROUPS;
  a.gt = TC_GT;
  a.cpad = cp;
  a.nh = nh;
  a.nhalf = nhalf;
  const bool f16 = c->ops32_f16;
  a.kchunks = cp / (f16 ? 32 : TC_KC);
  a.nst = c->tc_nst;
  a.lev_ops = op_banks(c) > 1;
  a.mmax = c->tc_mmax;
  a.kscale = c->ops_kscale;
  a.acol = (uint32_t)(2 * nhalf);
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < 2 * nhalf + 32 * c->tc_nst) a.tmem_cols <<= 1;
  const int smem = c->tc_nst * tc_stage_bytes(cp) + tc_fixed_bytes(cp);
  const int nunits = c->ntiles * nh * TC_GROUPS;
  const int grid = nunits < c->num_sms ? nunits : c->num_sms;
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[11], s, cudaEventRecordExternal));
  if (f16) {
    // the largest |M| per (problem, level) sets each target row's scale
    FMM_CUDA(c, cudaMemsetAsync(c->tc_mmax, 0,
                                sizeof(uint32_t) * ((c->forest ? c->nprob : 1) + 1) * FMM_MAX_LEVELS, s));
    const int64_t mrows = c->lv.row_off[c->leaf] + c->lv.ncell[c->leaf] + 1 - c->lv.row_off[2];
    k_m_absmax<<<(int)std::min<int64_t>(ceil_div(mrows, 8), 8 * 1184), 256, 0, s>>>(c->lv, 2, c->leaf, cp, c->Mhi,
                                                                                     c->Mlo, c->tc_mmax);
  }
  // the P2P branch is released here: its blocks and this kernel's CTAs become
  // ready together and the CTAs (higher launch priority) are placed first,
  // one per SM; released earlier, P2P blocks would hold the registers a CTA
  // needs and delay the CTA's statically assigned units
  if (c->timing != 2 && c->p2p_priority) {
    FMM_CUDA(c, cudaEventRecord(c->ev_p2p, s));
    c->p2p_after_proj = true;
  }
  if (f16) {
    k_m2l_tc<true><<<grid, TC_THREADS, smem, s>>>(*(const CUtensorMap*)c->tm_khi, *(const CUtensorMap*)c->tm_klo, a,
                                                  c->lv, c->Mhi, c->Mlo);
  } else {
    k_m2l_tc<false><<<grid, TC_THREADS, smem, s>>>(*(const CUtensorMap*)c->tm_khi, *(const CUtensorMap*)c->tm_klo, a,
                                                   c->lv, c->Mhi, c->Mlo);
  }
  FMM_CUDA(c, cudaGetLastError());
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[12], s, cudaEventRecordExternal));
  if (mid) FMM_CUDA(c, cudaEventRecordWithFlags(mid, s, cudaEventRecordExternal));
  k_m2l_tc_reduce<<<dim3(c->ntiles, FMM_TILE / 16), 256, 0, s>>>(c->tiles, c->tile_nact, c->lv, c->ntiles, TC_GT, cp, c->ncoef + 1,
                                            c->tc_partial, c->L32, c->box, c->kernel_s);
  return cuda_err(c, cudaGetLastError(), "M2L tensor-core launch");
}

}  // namespace fmm
