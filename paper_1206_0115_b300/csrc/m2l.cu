// m2l.cu -- M2L dispatch (Sec. 2.1.2): the FP64 path runs the CUDA-core
// kernels in FP64; the mixed path runs the tcgen05 kernels -- three products
// of FP16 hi/lo operand pairs by default, of TF32 hi/lo pairs with
// FMM_M2L_MATH=tf32 -- when the order allows it (p <= 7: the padded rows,
// order^3 + 1 rounded up to 32, fit the tensor-core kernels' accumulators)
// and otherwise (p >= 8) the CUDA-core kernels on FP32 sums of the
// split pairs.
#include "common.cuh"

namespace fmm {

int m2l_kind(const Ctx* c) {
  if (uses_svd(c)) {
    if (c->precision == FMM_FP64) return 3;
    return (c->use_tc && m2l_svd_tc_supported(c)) ? 5 : 4;
  }
  if (c->precision == FMM_FP64) return 0;
  return (c->use_tc && m2l_tc_supported(c)) ? 2 : 1;
}

fmm_status launch_m2l(Ctx* c, cudaStream_t s, cudaEvent_t mid) {
  if (c->ntiles <= 0 || c->n == 0) {
    if (mid) FMM_CUDA(c, cudaEventRecordWithFlags(mid, s, cudaEventRecordExternal));
    return FMM_OK;
  }
  const int kind = m2l_kind(c);
  if (kind == 2) return launch_m2l_tc(c, s, mid);
  if (kind == 5) return launch_m2l_svd_tc(c, s, mid);
  auto run = kind >= 3 ? launch_m2l_svd_simt : launch_m2l_simt;
  // CUDA cores: leaf level, then the coarser levels
  FMM_TRY(run(c, s, 0, c->leaf_tiles));
  if (mid) FMM_CUDA(c, cudaEventRecordWithFlags(mid, s, cudaEventRecordExternal));
  return run(c, s, c->leaf_tiles, c->ntiles - c->leaf_tiles);
}

// The part of the M2L bookkeeping that depends on the tree alone (not on
// the multipoles), launched on its own branch so that it runs beside the
// upward pass; launch_m2l then waits for it (c->ev_prep) instead of
// launching it.  Only the compressed tensor-core form with FP16 operands has
// such a part (its projection records and destination map).
bool m2l_has_prep(const Ctx* c) {
  return c->ntiles > 0 && c->n > 0 && m2l_kind(c) == 5 && svd_has_tree_setup(c);
}

fmm_status launch_m2l_prep(Ctx* c, cudaStream_t s) {
  c->m2l_prep_done = false;
  if (!m2l_has_prep(c)) return FMM_OK;
  FMM_TRY(svd_tree_setup(c, s));
  FMM_CUDA(c, cudaEventRecord(c->ev_prep, s));
  c->m2l_prep_done = true;
  return FMM_OK;
}

namespace {

__global__ void __launch_bounds__(FMM_TILE)
k_count_m2l_pairs(const Tile* __restrict__ tiles, const int32_t* __restrict__ tile_src,
                  const int16_t* __restrict__ tile_act, const int32_t* __restrict__ tile_nact, LevelPtrs lv,
                  const int16_t* __restrict__ cls_t, const int32_t* __restrict__ trank,
                  const int16_t* __restrict__ src_act, const int32_t* __restrict__ src_nact,
                  const int16_t* __restrict__ src_t, const int32_t* __restrict__ t_ry, int64_t xk,
                  unsigned long long* __restrict__ out) {
  const Tile tl = tiles[blockIdx.x];
  const int row = threadIdx.x, zero = lv.ncell[tl.level];
  const int nact = tile_nact[blockIdx.x];
  unsigned long long cnt = 0, rsum = 0;
  for (int a = 0; a < nact; ++a) {
    const int k = tile_act[(int64_t)blockIdx.x * FMM_NT_CLASS + a];
    const int s = tile_src[((int64_t)blockIdx.x * FMM_NT_CLASS + k) * FMM_TILE + row];
    const bool pair = row < tl.count && s != zero;
    cnt += pair;
    if (trank && pair) rsum += trank[cls_t[tl.cls * FMM_NT_CLASS + k]];
  }
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
  }
  if ((row & 31) == 0) {
    atomicAdd(&out[1 + tl.level], cnt);
    atomicAdd(&out[13], rsum);
  }
  if (row == 0) atomicAdd(&out[12], (unsigned long long)nact);
  if (row == 0 && t_ry) {
    // 128-row blocks of the compressed M2L, in Y columns: projection (the
    // tile's cells as sources) and expansion (as targets)
    unsigned long long yp = 0, ye = 0;
    const int ns = src_nact[blockIdx.x];
    for (int a = 0; a < ns; ++a)
      yp += t_ry[src_t[tl.cls * FMM_NT_CLASS + src_act[(int64_t)blockIdx.x * FMM_NT_CLASS + a]]];
    for (int a = 0; a < nact; ++a)
      ye += t_ry[cls_t[tl.cls * FMM_NT_CLASS + tile_act[(int64_t)blockIdx.x * FMM_NT_CLASS + a]]];
    // FP16 tensor-core form: the expansion runs every tile over its class's
    // whole concatenated K (xk values)
    if (xk > 0) ye = (unsigned long long)xk;
    atomicAdd(&out[14], yp);
    atomicAdd(&out[15], ye);
  }
}

__global__ void k_count_p2p_pairs(LevelPtrs lv, int leaf, int nleaf, unsigned long long* __restrict__ out) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= nleaf) return;
  int ix, iy, iz;
  demorton3(lv.key[leaf][T], ix, iy, iz);
  const int top = (1 << leaf) - 1;
  unsigned long long src = 0;
  for (int k = 0; k < 27; ++k) {
    const int sx = ix + k / 9 - 1, sy = iy + (k / 3) % 3 - 1, sz = iz + k % 3 - 1;
    if (sx < 0 || sy < 0 || sz < 0 || sx > top || sy > top || sz > top) continue;
    const int g = lv.grid[leaf][morton3(sx, sy, sz)];
    if (g >= 0 && same_problem(lv, leaf, problem_of(lv, leaf, T), g)) src += lv.count[leaf][g];
  }
  const unsigned long long nt = lv.count[leaf][T];
  atomicAdd(&out[0], nt * src - nt);
}

}  // namespace

fmm_status work_counts(Ctx* c, int64_t* out) {
  for (int k = 0; k < 16; ++k) out[k] = 0;
  if (c->n == 0) return FMM_OK;
  unsigned long long* d = (unsigned long long*)c->scratch;
  FMM_CUDA(c, cudaMemsetAsync(d, 0, 16 * sizeof(unsigned long long), c->stream));
  const int nleaf = c->lv.ncell[c->leaf];
  k_count_p2p_pairs<<<ceil_div(nleaf, 128), 128, 0, c->stream>>>(c->lv, c->leaf, nleaf, d);
  if (c->ntiles > 0)
    k_count_m2l_pairs<<<c->ntiles, FMM_TILE, 0, c->stream>>>(c->tiles, c->tile_src, c->tile_act, c->tile_nact,
                                                             c->lv, c->cls_t, c->svd_ready ? c->svd_trank : nullptr,
                                                             c->src_act, c->src_nact, c->src_t,
                                                             c->svd_ready ? c->svd_ry : nullptr,
                                                             m2l_kind(c) == 5 && svd_wants_f16(c) && c->svd_kct > 0
                                                                 ? 32 * (int64_t)c->svd_kct
                                                                 : 0,
                                                             d);
  FMM_CUDA(c, cudaGetLastError());
  FMM_CUDA(c, cudaMemcpyAsync(out, d, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  return FMM_OK;
}

int64_t count_launches_eval(const Ctx* c) {
  const int Lf = c->leaf;
  int64_t k = 2;  // P2P, L2P/output
  if (Lf >= 2 && c->n > 0) {
    k += 1 + (Lf - 2);                                      // P2M, M2M
    const int kind = m2l_kind(c), per = kind >= 3 ? 2 : 1;
    k += kind == 2 ? (2 + (c->ops32_f16 ? 1 : 0)) * (c->ntiles > 0)
                   : kind == 5 ? (5 + (Lf - 1)) * (c->ntiles > 0)
                               : per * ((c->leaf_tiles > 0) + (c->ntiles > c->leaf_tiles));
    k += (Lf - 2);                                          // L2L
  }
  return k;
}

}  // namespace fmm
