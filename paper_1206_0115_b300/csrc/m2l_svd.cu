// m2l_svd.cu -- the SVD-compressed M2L of Sec. 2.1.2 ("Improved M2L operator").
//
// The 316 operators K_t are images of 16 canonical ones under the symmetries
// of the cube.  With t = sigma(that), sigma permuting the axes and flipping
// signs ((sigma v)_d = sign_d v_{axis_d}, that = |t| sorted ascending),
//     K_t[sigma.m][sigma.n] = K_that[m][n],
// where sigma.m is the node index sigma maps node m to (the Chebyshev roots
// are symmetric, xbar_{p-1-j} = -xbar_j, so sigma maps nodes onto nodes and
// distances are unchanged).  Each K_that is compressed by its own SVD,
// truncated at s_i >= eps s_0 (eps = 10^-p unless the caller sets it: the
// pairing (l, eps) = (Acc, 10^-Acc) of Table 1).  Per (target T, source S,
// transfer vector t) the M2L becomes
//     y = V_t^T M_S,           V_t[sigma.n][i] = V_that[n][i]      (r_t values)
//     L_T += (1/a) U_t y,      U_t[sigma.m][i] = s_i U_that[m][i],
// the paper's "16 matrix-matrix products coupled with permutations", with
// the permutations folded into 316 permuted copies of the 16 factor pairs.
//
// Precompute (once per handle and eps; FP64 on the GPU):
//   k_canon_ops64   the 16 canonical K_that (the formula of operators.cu);
//   k_svd_jacobi    a one-sided Jacobi SVD per operator: one block, the
//                   column pairs in round-robin order so that the warps of a
//                   block rotate disjoint pairs at once, sweeps until no pair
//                   needs a rotation (|a_i . a_j| <= 1e-15 |a_i| |a_j|), at
//                   most 60 (a bounded loop; a non-converged operator is an
//                   error the host reports);
//   k_svd_order     singular values (column norms), their descending order,
//                   the rank and, for the mixed banks, the mean of every
//                   column of U Sigma;
//   k_svd_banks64 / k_svd_banks32   the permuted factors of all 316 t.
// Evaluation, per M2L tile (128 cells of one level and child class):
//   k_m2l_proj    from the sources: Y[S][t] = V_t^T M_S for each cell S of the
//                 tile and each t with which S serves a target (src_t, src_act),
//                 so that every M row is read once per (tile, t) without a gather
//   k_m2l_expand  at the targets: L_T = (1/a) sum_t U_t Y[T + t][t] (the short
//                 Y rows are gathered, not the multipoles)
// The mixed path stores U in the mean-split form of the local expansions
// (row C = the mean over m of U_t[m][.], rows m < C the deviations), its
// factors as TF32 hi/lo pairs (FP16 hi/lo pairs for the tensor cores' FP16
// form, whose expansion bank Uc runs along each child class's concatenated
// ranks), and pads every rank with zero factors to a multiple of 16 (8 in the
// FP16 form: one 16-byte group of FP16 values) -- the result is that of
// rank r_t.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "tc_ptx.cuh"

namespace fmm {

namespace {

constexpr int SVD_THREADS = 1024;
constexpr int SVD_MAX_SWEEPS = 60;

using tc::tf32_rna;

// K_that[m][n] = |2 that + xbar_n - xbar_m|^-s for the 16 canonical vectors.
__global__ void k_canon_ops64(int p, int C, const double* __restrict__ nodes, const int8_t* __restrict__ canon,
                              double ks, double* __restrict__ K) {
  const int64_t total = (int64_t)16 * C * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / ((int64_t)C * C));
    const int rem = (int)(e - (int64_t)k * C * C);
    const int m = rem / C, nn = rem - m * C;
    const int mi[3] = {m / (p * p), (m / p) % p, m % p};
    const int ni[3] = {nn / (p * p), (nn / p) % p, nn % p};
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double r = 2.0 * canon[3 * k + d] + nodes[ni[d]] - nodes[mi[d]];
      r2 += r * r;
    }
    K[e] = kernel_r2(r2, ks);
  }
}

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-sided Jacobi SVD of the 16 operators (block k = operator k).  W[k][j]
// starts as column j of K and Z[k][j] as column j of the identity; rotating
// the pair (i, j) by the angle that makes columns i and j of W orthogonal
// and applying the same rotation to Z keeps K Z = W.  At convergence the
// columns of W are s_j u_j and those of Z are v_j.
__global__ void __launch_bounds__(SVD_THREADS)
k_svd_jacobi(int C, const double* __restrict__ K, double* __restrict__ W, double* __restrict__ Z,
             int32_t* __restrict__ sweeps_out) {
  const int k = blockIdx.x;
  const double* A = K + (size_t)k * C * C;
  double* Wk = W + (size_t)k * C * C;
  double* Zk = Z + (size_t)k * C * C;
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const int j = e / C, i = e - j * C;
    Wk[e] = A[(size_t)i * C + j];
    Zk[e] = i == j ? 1.0 : 0.0;
  }
  __shared__ int rotated;
  const int n2 = C + (C & 1);  // an odd C gets a dummy column, paired with nobody
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int done = -1;
  __syncthreads();
  for (int sweep = 1; sweep <= SVD_MAX_SWEEPS && done < 0; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < n2 - 1; ++r) {
      // round r of the circle method: every column in exactly one pair
      for (int q = warp; q < n2 / 2; q += nw) {
        int i = q == 0 ? n2 - 1 : (r + q) % (n2 - 1);
        int j = q == 0 ? r : (r - q + n2 - 1) % (n2 - 1);
        if (i >= C || j >= C) continue;
        if (i > j) {
          const int x = i;
          i = j;
          j = x;
        }
        double* wi = Wk + (size_t)i * C;
        double* wj = Wk + (size_t)j * C;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int e = lane; e < C; e += 32) {
          const double x = wi[e], y = wj[e];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        // butterfly sums: every lane holds the same totals, so the branch is warp-uniform
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        if (lane == 0) rotated = 1;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        double* zi = Zk + (size_t)i * C;
        double* zj = Zk + (size_t)j * C;
        for (int e = lane; e < C; e += 32) {
          double x = wi[e], y = wj[e];
          wi[e] = cs * x - sn * y;
          wj[e] = sn * x + cs * y;
          x = zi[e];
          y = zj[e];
          zi[e] = cs * x - sn * y;
          zj[e] = sn * x + cs * y;
        }
      }
      __syncthreads();
    }
    if (rotated == 0) done = sweep;
    __syncthreads();
  }
  if (threadIdx.x == 0) sweeps_out[k] = done;
}

// Singular values s_j = |W[k][j]|, the descending order ord (ties by index),
// the rank #{s >= eps s_max}, and the column means of U Sigma (mixed banks).
__global__ void __launch_bounds__(SVD_THREADS)
k_svd_order(int C, double eps, const double* __restrict__ W, double* __restrict__ svals,
            int32_t* __restrict__ ord, int32_t* __restrict__ rank, double* __restrict__ colmean) {
  __shared__ double sv[FMM_MAX_ORDER * FMM_MAX_ORDER * FMM_MAX_ORDER];
  const int k = blockIdx.x;
  const double* Wk = W + (size_t)k * C * C;
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    double s = 0.0;
    for (int e = 0; e < C; ++e) s += Wk[(size_t)j * C + e] * Wk[(size_t)j * C + e];
    sv[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < C; ++i) r += (sv[i] > sv[j]) || (sv[i] == sv[j] && i < j);
    ord[k * C + r] = j;
    svals[k * C + r] = sv[j];
  }
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int j = 0; j < C; ++j) smax = fmax(smax, sv[j]);
    int r = 0;
    for (int j = 0; j < C; ++j) r += sv[j] >= eps * smax;
    rank[k] = r;
  }
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    double s = 0.0;
    for (int e = 0; e < C; ++e) s += Wk[(size_t)j * C + e];
    colmean[k * C + j] = s / C;
  }
}

// FP64 banks [316][C][R]: V_t[sigma.n][i] = Z[k][ord_i][n], U_t[sigma.n][i] =
// W[k][ord_i][n] for i < rank, 0 beyond.  One thread per (t, n).
__global__ void k_svd_banks64(int C, int R, const int8_t* __restrict__ t_canon, const int16_t* __restrict__ sm,
                              const int32_t* __restrict__ ord, const int32_t* __restrict__ rank,
                              const double* __restrict__ W, const double* __restrict__ Z, double* __restrict__ V64,
                              double* __restrict__ U64) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)FMM_NT * C) return;
  const int t = (int)(e / C), n = (int)(e - (int64_t)t * C);
  const int k = t_canon[t], r = rank[k];
  const int np = sm[e];
  for (int i = 0; i < R; ++i) {
    const int j = i < r ? ord[k * C + i] : 0;
    V64[((int64_t)t * C + np) * R + i] = i < r ? Z[((size_t)k * C + j) * C + n] : 0.0;
    U64[((int64_t)t * C + np) * R + i] = i < r ? W[((size_t)k * C + j) * C + n] : 0.0;
  }
}

// Mixed banks (TF32 hi/lo, zero-initialised by the caller), in interleaved
// hi/lo slabs of 64-byte rows (il_idx) along chunks of 16 of the contracted
// index, so that a tensor-core operand slab is one contiguous block:
//   VT (projection B, K = n): per source class, the class's transfer
//     vectors stacked in the order of its Y rows: row G = (cls * (cpad / 16)
//     + n / 16) * YS + yoff[cls][t] + i holds V_t[sigma.n][i];
//   U (expansion B, K = i): row G = ((i / 16) * 316 + t) * cpad + sigma.m
//     holds U_t - mean_m U_t (rows m < C) and the mean (row C).
__global__ void k_svd_banks32(int C, int cpad, int64_t YS, const int8_t* __restrict__ t_canon,
                              const int16_t* __restrict__ sm, const int32_t* __restrict__ ord,
                              const int32_t* __restrict__ rank, const double* __restrict__ W,
                              const double* __restrict__ Z, const double* __restrict__ colmean,
                              const int32_t* __restrict__ yoff, float* __restrict__ VT, float* __restrict__ U) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)FMM_NT * C) return;
  const int t = (int)(e / C), n = (int)(e - (int64_t)t * C);
  const int k = t_canon[t], r = rank[k];
  const int np = sm[e];
  const int kch = cpad / 16;
  for (int i = 0; i < r; ++i) {
    const int j = ord[k * C + i];
    const double v = Z[((size_t)k * C + j) * C + n];
    const double u = W[((size_t)k * C + j) * C + n] - colmean[k * C + j];
    const float vh = tf32_rna((float)v), vl = tf32_rna((float)(v - (double)vh));
    for (int cls = 0; cls < 8; ++cls) {
      const int yo = yoff[cls * FMM_NT + t];
      if (yo < 0) continue;
      const int64_t G = ((int64_t)cls * kch + (np >> 4)) * YS + yo + i;
      VT[tc::il_idx(G, 0, np & 15)] = vh;
      VT[tc::il_idx(G, 1, np & 15)] = vl;
    }
    const int64_t Gu = ((int64_t)(i >> 4) * FMM_NT + t) * cpad + np;
    float h = tf32_rna((float)u);
    U[tc::il_idx(Gu, 0, i & 15)] = h;
    U[tc::il_idx(Gu, 1, i & 15)] = tf32_rna((float)(u - (double)h));
    if (n == 0) {  // the mean row
      const double mu = colmean[k * C + j];
      const int64_t Gm = ((int64_t)(i >> 4) * FMM_NT + t) * cpad + C;
      h = tf32_rna((float)mu);
      U[tc::il_idx(Gm, 0, i & 15)] = h;
      U[tc::il_idx(Gm, 1, i & 15)] = tf32_rna((float)(mu - (double)h));
    }
  }
}

// The same banks with FP16 hi/lo operands for the tensor-core kernels' FP16
// form: 32 values of the contracted index per 64-byte row (two per 32-bit
// word, the even one in the low half), V scaled by vscale and U by uscale
// (powers of two that keep them below 2^13):
//   VT row G = (cls * (cpad / 32) + n / 32) * YS + yoff[cls][t] + i,
//   U row  G = ((i / 32) * 316 + t) * cpad + sigma.m (mean row C).
// Halves are stored one by one (threads of different n share a word).
__device__ inline void put_h(uint16_t* b, int64_t G, int e, double x) {
  const __half h = __float2half_rn((float)x);
  const __half l = __float2half_rn((float)(x - (double)__half2float(h)));
  b[2 * tc::il_idx(G, 0, e >> 1) + (e & 1)] = __half_as_ushort(h);
  b[2 * tc::il_idx(G, 1, e >> 1) + (e & 1)] = __half_as_ushort(l);
}

__global__ void k_svd_banks16(int C, int cpad, int64_t YS, const int8_t* __restrict__ t_canon,
                              const int16_t* __restrict__ sm, const int32_t* __restrict__ ord,
                              const int32_t* __restrict__ rank, const double* __restrict__ W,
                              const double* __restrict__ Z, const double* __restrict__ colmean,
                              const int32_t* __restrict__ yoff, double vscale, double uscale,
                              uint16_t* __restrict__ VT, uint16_t* __restrict__ U) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)FMM_NT * C) return;
  const int t = (int)(e / C), n = (int)(e - (int64_t)t * C);
  const int k = t_canon[t], r = rank[k];
  const int np = sm[e];
  const int kch = cpad / 32;
  for (int i = 0; i < r; ++i) {
    const int j = ord[k * C + i];
    const double v = Z[((size_t)k * C + j) * C + n] * vscale;
    const double u = (W[((size_t)k * C + j) * C + n] - colmean[k * C + j]) * uscale;
    for (int cls = 0; cls < 8; ++cls) {
      const int yo = yoff[cls * FMM_NT + t];
      if (yo < 0) continue;
      put_h(VT, ((int64_t)cls * kch + (np >> 5)) * YS + yo + i, np & 31, v);
    }
    if (!U) continue;
    put_h(U, ((int64_t)(i >> 5) * FMM_NT + t) * cpad + np, i & 31, u);
    if (n == 0) put_h(U, ((int64_t)(i >> 5) * FMM_NT + t) * cpad + C, i & 31, colmean[k * C + j] * uscale);
  }
}

// The expansion's factor bank of the FP16 tensor-core form, by target class:
// the class's transfer vectors in the order of its list (cls_t), each taking
// its rank rounded up to 8 of the contracted index (kap8 = where its ranks
// start, / 8), so that one slab of 32 contracted values covers consecutive
// transfer vectors and the expansion's K runs over all of a target's
// sources at once.  Row G = (cls * kct + k / 32) * cpad + sigma.m (mean row C),
// FP16 hi/lo scaled by uscale, element k % 32; padding stays zero.
__global__ void k_svd_bank_uc16(int C, int cpad, int kct, const int8_t* __restrict__ t_canon,
                                const int16_t* __restrict__ sm, const int32_t* __restrict__ ord,
                                const int32_t* __restrict__ rank, const double* __restrict__ W,
                                const double* __restrict__ colmean, const int16_t* __restrict__ kap8, double uscale,
                                uint16_t* __restrict__ Uc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)FMM_NT * C) return;
  const int t = (int)(e / C), n = (int)(e - (int64_t)t * C);
  const int k = t_canon[t], r = rank[k];
  const int np = sm[e];
  for (int i = 0; i < r; ++i) {
    const int j = ord[k * C + i];
    const double u = (W[((size_t)k * C + j) * C + n] - colmean[k * C + j]) * uscale;
    for (int cls = 0; cls < 8; ++cls) {
      const int kp = kap8[cls * FMM_NT + t];
      if (kp < 0) continue;
      const int kk = 8 * kp + i;
      const int64_t G = ((int64_t)cls * kct + (kk >> 5)) * cpad;
      put_h(Uc, G + np, kk & 31, u);
      if (n == 0) put_h(Uc, G + C, kk & 31, colmean[k * C + j] * uscale);
    }
  }
}

// ---------------------------------------------------------------- evaluation

struct SvdArgs {
  const Tile* tiles;
  const int32_t* tile_src;
  const int16_t* tile_act;
  const int32_t* tile_nact;
  const int16_t* src_act;
  const int32_t* src_nact;
  const int16_t* cls_t;
  const int16_t* src_t;
  const int32_t* t_ry;   // [316] Y values per (cell, t): the rank (mixed: rounded up to 16)
  const int32_t* yoff;   // [8][316] offset of t's values in a cell's Y row (class of the cell), -1 if none
  int64_t YS;            // Y row length
};

// Projection, from the sources: one block per (tile, active source transfer
// vector), one thread per cell S of the tile: Y[S][t] = V_t^T M_S (ry values),
// V staged in shared memory in chunks of 32 n x 16 i.  FP64 bank
// [316][C][R]; mixed bank VT hi/lo [316][Rp][cpad], used as the FP32 sum.
template <typename T, bool MIXED>
__global__ void __launch_bounds__(FMM_TILE)
k_m2l_proj(SvdArgs a, LevelPtrs lv, int C, int cpad, int R, const T* __restrict__ Vb, const T* __restrict__ Vlo,
           const T* __restrict__ Mhi, const T* __restrict__ Mlo, T* __restrict__ Y) {
  __shared__ T sV[32][16];
  const int tile = blockIdx.x, ai = blockIdx.y, row = threadIdx.x;
  if (ai >= a.src_nact[tile]) return;
  const Tile tl = a.tiles[tile];
  const int l = tl.level;
  const int k = a.src_act[(int64_t)tile * FMM_NT_CLASS + ai];
  const int slot = a.src_t[tl.cls * FMM_NT_CLASS + k];
  const int ry = a.t_ry[slot];
  const bool valid = row < tl.count;
  const int64_t cellrow = lv.row_off[l] + (valid ? lv.cls[l][tl.first + row] : lv.ncell[l]);
  const int64_t mrow = cellrow * cpad;
  T* yout = Y + cellrow * a.YS + a.yoff[tl.cls * FMM_NT + slot];
  for (int i0 = 0; i0 < ry; i0 += 16) {
    T acc[16];
#pragma unroll
    for (int ii = 0; ii < 16; ++ii) acc[ii] = T(0);
    for (int n0 = 0; n0 < C; n0 += 32) {
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * 16; e += FMM_TILE) {
        const int nn = e >> 4, ii = e & 15, n = n0 + nn, i = i0 + ii;
        T v = T(0);
        if (n < C && i < R) {
          if (MIXED) {
            const int64_t G = ((int64_t)tl.cls * (cpad / 16) + (n >> 4)) * a.YS + a.yoff[tl.cls * FMM_NT + slot] + i;
            v = Vb[tc::il_idx(G, 0, n & 15)] + Vb[tc::il_idx(G, 1, n & 15)];
          } else {
            v = Vb[((int64_t)slot * C + n) * R + i];
          }
        }
        sV[nn][ii] = v;
      }
      __syncthreads();
      const int nmax = min(32, C - n0);
      for (int nn = 0; nn < nmax; ++nn) {
        T m = Mhi[mrow + n0 + nn];
        if (MIXED) m += Mlo[mrow + n0 + nn];
#pragma unroll
        for (int ii = 0; ii < 16; ++ii) acc[ii] += sV[nn][ii] * m;
      }
    }
    if (valid) {
#pragma unroll
      for (int ii = 0; ii < 16; ++ii)
        if (i0 + ii < ry) yout[i0 + ii] = acc[ii];
    }
  }
}

// Expansion, at the targets: one CTA computes 64 target rows x 64
// coefficients, a GEMM whose K dimension runs over (active transfer vector t,
// i < ry_t): A = the sources' Y values for t (gathered; the level's zero row,
// an absent source, gives zeros), B = U_t.  Per transfer vector the products
// are summed in T and added into a Kahan-compensated total.  FP64 bank
// [316][C][R]; mixed bank U hi/lo [316][cpad][Rp] with the mean row C.
template <typename T, bool MIXED>
__global__ void __launch_bounds__(256)
k_m2l_expand(SvdArgs a, LevelPtrs lv, int C, int cpad, int R, const T* __restrict__ Ub, const T* __restrict__ Ulo,
             const T* __restrict__ Y, T* __restrict__ Lout, const double* __restrict__ box, double ks) {
  __shared__ T As[16][64];
  __shared__ T Bs[16][64 + 1];
  __shared__ int64_t sy[64];
  const int tile = blockIdx.x, half = blockIdx.y, col0 = blockIdx.z * 64;
  const int ncol = MIXED ? C + 1 : C;
  if (col0 >= ncol) return;
  const Tile tl = a.tiles[tile];
  if (half * 64 >= tl.count) return;
  const int l = tl.level;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nact = a.tile_nact[tile];
  const int64_t rbase = lv.row_off[l];
  const int zero = lv.ncell[l];
  T acc[4][4], tot[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) tot[i][j] = cmp[i][j] = T(0);
  for (int ai = 0; ai < nact; ++ai) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int k = a.tile_act[(int64_t)tile * FMM_NT_CLASS + ai];
    const int slot = a.cls_t[tl.cls * FMM_NT_CLASS + k];
    const int ry = a.t_ry[slot];
    __syncthreads();
    if (tid < 64) {
      const int s = a.tile_src[((int64_t)tile * FMM_NT_CLASS + k) * FMM_TILE + half * 64 + tid];
      sy[tid] = s == zero ? -1 : (rbase + s) * a.YS + a.yoff[(lv.key[l][s] & 7) * FMM_NT + slot];
    }
    for (int i0 = 0; i0 < ry; i0 += 16) {
      __syncthreads();
      for (int e = tid; e < 64 * 16; e += 256) {
        const int r = e >> 4, kk = e & 15;
        As[kk][r] = (i0 + kk < ry && sy[r] >= 0) ? Y[sy[r] + i0 + kk] : T(0);
      }
      for (int e = tid; e < 64 * 16; e += 256) {
        const int cc = e >> 4, kk = e & 15;
        const int m = col0 + cc, i = i0 + kk;
        T v = T(0);
        if (m < ncol && i < ry && i < R) {
          if (MIXED) {
            const int64_t G = ((int64_t)(i >> 4) * FMM_NT + slot) * cpad + m;
            v = Ub[tc::il_idx(G, 0, i & 15)] + Ub[tc::il_idx(G, 1, i & 15)];
          } else {
            v = Ub[((int64_t)slot * C + m) * R + i];
          }
        }
        Bs[kk][cc] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        T av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const T y = acc[i][j] - cmp[i][j];
        const T s = tot[i][j] + y;
        cmp[i][j] = (s - tot[i][j]) - y;
        tot[i][j] = s;
      }
  }
  const double inv_a = kernel_scale(ldexp(1.0, l + 1) / box[3], ks);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = half * 64 + ty + 16 * i;
    if (r >= tl.count) continue;
    const int64_t row = rbase + lv.cls[l][tl.first + r];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = col0 + tx + 16 * j;
      if (m < ncol) Lout[row * cpad + m] = (T)((double)tot[i][j] * inv_a);
    }
  }
}

// Host symmetry tables: canonical index of every transfer vector (in the
// lexicographic slot order of operators.cu) and its node map sigma.
void symmetry_tables(int p, std::vector<int8_t>& canon, std::vector<int8_t>& t_canon, std::vector<int16_t>& sm) {
  std::vector<std::array<int, 3>> cv;
  for (int a = 0; a <= 3; ++a)
    for (int b = a; b <= 3; ++b)
      for (int c = b; c <= 3; ++c)
        if (c >= 2) cv.push_back({a, b, c});
  canon.clear();
  for (auto& v : cv)
    for (int d = 0; d < 3; ++d) canon.push_back((int8_t)v[d]);
  const int C = p * p * p;
  t_canon.assign(FMM_NT, 0);
  sm.assign((size_t)FMM_NT * C, 0);
  int slot = 0;
  for (int x = -3; x <= 3; ++x)
    for (int y = -3; y <= 3; ++y)
      for (int z = -3; z <= 3; ++z) {
        if (std::abs(x) < 2 && std::abs(y) < 2 && std::abs(z) < 2) continue;
        const int t[3] = {x, y, z};
        int av[3] = {std::abs(x), std::abs(y), std::abs(z)};
        std::array<int, 3> th = {av[0], av[1], av[2]};
        std::sort(th.begin(), th.end());
        int axis[3], sign[3];
        bool used[3] = {false, false, false};
        for (int d = 0; d < 3; ++d) {
          sign[d] = t[d] < 0 ? -1 : 1;
          for (int j = 0; j < 3; ++j)
            if (!used[j] && th[j] == av[d]) {
              axis[d] = j;
              used[j] = true;
              break;
            }
        }
        int k = 0;
        while (cv[k] != th) ++k;
        t_canon[slot] = (int8_t)k;
        for (int m = 0; m < C; ++m) {
          const int mi[3] = {m / (p * p), (m / p) % p, m % p};
          int r[3];
          for (int d = 0; d < 3; ++d) r[d] = sign[d] > 0 ? mi[axis[d]] : p - 1 - mi[axis[d]];
          sm[(size_t)slot * C + m] = (int16_t)((r[0] * p + r[1]) * p + r[2]);
        }
        ++slot;
      }
}

}  // namespace

double svd_eps_of(const Ctx* c) { return c->svd_eps > 0.0 ? c->svd_eps : std::pow(10.0, -c->order); }

// SVD of the 16 canonical operators for the handle's order and eps; ranks
// read back to the host.  Synchronous (once per handle and eps).
fmm_status svd_prepare(Ctx* c) {
  const double eps = svd_eps_of(c);
  if (c->svd_ready && c->svd_eps_used == eps) return FMM_OK;
  const int p = c->order, C = c->ncoef;
  cudaStream_t s = c->stream;
  std::vector<int8_t> canon, t_canon;
  std::vector<int16_t> sm;
  symmetry_tables(p, canon, t_canon, sm);
  // work buffers: K, W, Z [16][C][C], singular values, order, colmean, ranks, sweeps
  const size_t mat = (size_t)16 * C * C;
  void* ptr;
  if (!c->svd_W) {
    FMM_TRY(dalloc(c, &ptr, sizeof(double) * mat * 2));
    c->svd_W = (double*)ptr;
    c->svd_Z = c->svd_W + mat;
    FMM_TRY(dalloc(c, &ptr, sizeof(double) * 16 * C * 2 + sizeof(int32_t) * (16 * C + 64)));
    c->svd_vals = (double*)ptr;
    c->svd_colmean = c->svd_vals + 16 * C;
    c->svd_ord = (int32_t*)(c->svd_colmean + 16 * C);
    c->svd_rank_d = c->svd_ord + 16 * C;
    c->svd_sweeps_d = c->svd_rank_d + 16;
    FMM_TRY(dalloc(c, &ptr, (size_t)FMM_NT * C * sizeof(int16_t) + 64 + FMM_NT));
    c->svd_sm = (int16_t*)ptr;
    c->svd_canon = (int8_t*)(c->svd_sm + (size_t)FMM_NT * C);
    c->svd_tcanon = c->svd_canon + 48;
    FMM_CUDA(c, cudaMemcpyAsync(c->svd_sm, sm.data(), sm.size() * sizeof(int16_t), cudaMemcpyHostToDevice, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->svd_canon, canon.data(), canon.size(), cudaMemcpyHostToDevice, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->svd_tcanon, t_canon.data(), t_canon.size(), cudaMemcpyHostToDevice, c->stream));
    FMM_CUDA(c, cudaStreamSynchronize(c->stream));  // host tables go out of scope
  }
  double* K;
  FMM_TRY(dalloc(c, &ptr, sizeof(double) * mat));
  K = (double*)ptr;
  k_canon_ops64<<<ceil_div(mat, 256), 256, 0, s>>>(p, C, c->nodes64, c->svd_canon, c->kernel_s, K);
  k_svd_jacobi<<<16, SVD_THREADS, 0, s>>>(C, K, c->svd_W, c->svd_Z, c->svd_sweeps_d);
  k_svd_order<<<16, SVD_THREADS, 0, s>>>(C, eps, c->svd_W, c->svd_vals, c->svd_ord, c->svd_rank_d, c->svd_colmean);
  FMM_CUDA(c, cudaGetLastError());
  int32_t hr[32];
  FMM_CUDA(c, cudaMemcpyAsync(hr, c->svd_rank_d, sizeof(int32_t) * 32, cudaMemcpyDeviceToHost, s));
  FMM_CUDA(c, cudaStreamSynchronize(s));
  dfree(c, K, sizeof(double) * mat);
  for (int k = 0; k < 16; ++k)
    if (hr[16 + k] < 0) return set_err(c, FMM_ERR_CUDA, "SVD of canonical M2L operator %d did not converge", k);
  int rmax = 0;
  for (int k = 0; k < 16; ++k) {
    c->svd_rank[k] = hr[k];
    rmax = std::max(rmax, hr[k]);
  }
  for (int t = 0; t < FMM_NT; ++t) c->t_rank_h[t] = c->svd_rank[t_canon[t]];
  c->svd_rmax = rmax;
  c->svd_rp = (rmax + 15) / 16 * 16;
  c->svd_ready = true;
  c->svd_eps_used = eps;
  c->svd_gen++;
  c->svd64 = c->svd32 = false;
  return FMM_OK;
}

// Factor banks for the current precision (after svd_prepare).
fmm_status svd_banks(Ctx* c) {
  const int C = c->ncoef, cp = c->cpad;
  cudaStream_t s = c->stream;
  void* ptr;
  const int grid = ceil_div((int64_t)FMM_NT * C, 128);
  if (c->precision == FMM_FP64 && !c->svd64) {
    const int R = c->svd_rmax;
    const size_t bytes = sizeof(double) * (size_t)FMM_NT * C * R;
    dfree(c, c->svd_V64, c->svd_bank64_bytes);
    dfree(c, c->svd_U64, c->svd_bank64_bytes);
    c->svd_V64 = c->svd_U64 = nullptr;
    FMM_TRY(dalloc(c, &ptr, bytes));
    c->svd_V64 = (double*)ptr;
    FMM_TRY(dalloc(c, &ptr, bytes));
    c->svd_U64 = (double*)ptr;
    c->svd_bank64_bytes = bytes;
    k_svd_banks64<<<grid, 128, 0, s>>>(C, R, c->svd_tcanon, c->svd_sm, c->svd_ord, c->svd_rank_d, c->svd_W, c->svd_Z,
                                       c->svd_V64, c->svd_U64);
    FMM_CUDA(c, cudaGetLastError());
    FMM_CUDA(c, cudaStreamSynchronize(s));
    c->svd64 = true;
  }
  const bool f16 = c->precision == FMM_MIXED && svd_wants_f16(c);
  if (c->precision == FMM_MIXED && (!c->svd32 || c->svd_bank_f16 != f16)) {
    // TF32: VT 8 classes x cpad/16 chunks x YS rows, U Rp/16 chunks x 316 x cpad rows, 2 halves x 16 floats
    // per row; FP16: chunks of 32 (cpad/32, ceil(Rp/32)), 2 halves x 32 FP16 per row (the same 128 bytes)
    const int Rp = c->svd_rp;
    const int kw = f16 ? 32 : 16;
    const size_t vbytes = sizeof(float) * 32 * (size_t)8 * (cp / kw) * c->svd_YS;
    // FP16: the expansion takes the class-ordered bank Uc instead (below)
    const size_t ubytes = f16 ? 128 : sizeof(float) * 32 * (size_t)((Rp + kw - 1) / kw) * FMM_NT * cp;
    dfree(c, c->svd_VThi, c->svd_vt_bytes);
    dfree(c, c->svd_Uhi, c->svd_u_bytes);
    c->svd_VThi = c->svd_Uhi = nullptr;
    FMM_TRY(dalloc(c, &ptr, vbytes));
    c->svd_VThi = (float*)ptr;
    FMM_CUDA(c, cudaMemsetAsync(ptr, 0, vbytes, s));
    FMM_TRY(dalloc(c, &ptr, ubytes));
    c->svd_Uhi = (float*)ptr;
    FMM_CUDA(c, cudaMemsetAsync(ptr, 0, ubytes, s));
    c->svd_vt_bytes = vbytes;
    c->svd_u_bytes = ubytes;
    if (f16) {
      // |U entries| <= 2 s_max (columns of U Sigma and their means), |V entries| <= 1
      std::vector<double> sv((size_t)16 * C);
      FMM_CUDA(c, cudaMemcpyAsync(sv.data(), c->svd_vals, sizeof(double) * sv.size(), cudaMemcpyDeviceToHost, c->stream));
      FMM_CUDA(c, cudaStreamSynchronize(c->stream));
      double smax = 0.0;
      for (double v : sv) smax = std::max(smax, std::fabs(v));
      c->svd_vscale = tc::pow2_scale(1.0f);
      c->svd_uscale = tc::pow2_scale((float)(2.0 * smax));
      k_svd_banks16<<<grid, 128, 0, s>>>(C, cp, c->svd_YS, c->svd_tcanon, c->svd_sm, c->svd_ord, c->svd_rank_d,
                                         c->svd_W, c->svd_Z, c->svd_colmean, c->svd_yoff, (double)c->svd_vscale,
                                         (double)c->svd_uscale, (uint16_t*)c->svd_VThi, nullptr);
      // the expansion's bank by target class, along the class's concatenated ranks
      const size_t ucb = (size_t)128 * 8 * c->svd_kct * cp;
      dfree(c, c->svd_Uc, c->svd_uc_bytes);
      c->svd_Uc = nullptr;
      c->svd_uc_bytes = 0;
      FMM_TRY(dalloc(c, &ptr, ucb));
      c->svd_Uc = (uint32_t*)ptr;
      c->svd_uc_bytes = ucb;
      FMM_CUDA(c, cudaMemsetAsync(ptr, 0, ucb, s));
      k_svd_bank_uc16<<<grid, 128, 0, s>>>(C, cp, c->svd_kct, c->svd_tcanon, c->svd_sm, c->svd_ord, c->svd_rank_d,
                                           c->svd_W, c->svd_colmean, c->svd_kap8, (double)c->svd_uscale,
                                           (uint16_t*)c->svd_Uc);
    } else {
      k_svd_banks32<<<grid, 128, 0, s>>>(C, cp, c->svd_YS, c->svd_tcanon, c->svd_sm, c->svd_ord, c->svd_rank_d,
                                         c->svd_W, c->svd_Z, c->svd_colmean, c->svd_yoff, c->svd_VThi, c->svd_Uhi);
    }
    FMM_CUDA(c, cudaGetLastError());
    FMM_CUDA(c, cudaStreamSynchronize(s));
    c->svd32 = true;
    c->svd_bank_f16 = f16;
  }
  return FMM_OK;
}

// Y layout for the current precision and ranks (row length per transfer
// vector, offsets within a cell's row by the cell's class), and the Y buffer
// for the current tree (one row per expansion row).  Called before an
// evaluation is captured.
fmm_status m2l_svd_prepare(Ctx* c) {
  FMM_TRY(svd_prepare(c));
  const bool mixed = c->precision == FMM_MIXED;
  // FP16 tensor-core form: ranks padded to 8 (the projection's columns and
  // the expansion's concatenated K); TF32 forms and the CUDA-core kernels: 16
  const bool xf16 = mixed && svd_wants_f16(c);
  const std::vector<int64_t> sig = {c->precision, c->svd_gen, xf16};
  void* ptr;
  if (sig != c->svd_ysig) {
    c->svd32 = false;  // the mixed banks follow the Y layout
    const int pad = xf16 ? 8 : 16;
    std::vector<int32_t> ry(FMM_NT), rank(FMM_NT), yoff(8 * FMM_NT, -1);
    for (int t = 0; t < FMM_NT; ++t) {
      rank[t] = c->t_rank_h[t];
      ry[t] = mixed ? (rank[t] + pad - 1) / pad * pad : rank[t];
    }
    int64_t ys = 0;
    for (int cls = 0; cls < 8; ++cls) {
      int64_t o = 0;
      for (int k = 0; k < FMM_NT_CLASS; ++k) {
        const int slot = c->src_t_h[cls * FMM_NT_CLASS + k];
        yoff[cls * FMM_NT + slot] = (int32_t)o;
        o += ry[slot];
      }
      ys = std::max(ys, o);
    }
    c->svd_YS = (ys + 15) / 16 * 16;  // 64-byte aligned rows (FP32)
    if (!c->svd_ry) {
      FMM_TRY(dalloc(c, &ptr, sizeof(int32_t) * (2 * FMM_NT + 8 * FMM_NT)));
      c->svd_ry = (int32_t*)ptr;
      c->svd_trank = c->svd_ry + FMM_NT;
      c->svd_yoff = c->svd_trank + FMM_NT;
    }
    FMM_CUDA(c, cudaMemcpyAsync(c->svd_ry, ry.data(), sizeof(int32_t) * FMM_NT, cudaMemcpyHostToDevice, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->svd_trank, rank.data(), sizeof(int32_t) * FMM_NT, cudaMemcpyHostToDevice, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->svd_yoff, yoff.data(), sizeof(int32_t) * yoff.size(), cudaMemcpyHostToDevice, c->stream));
    if (xf16) {
      // per target class: where each t's ranks start in the concatenated K (/ 8);
      // per source class: the index of each t in the class's source list
      std::vector<int16_t> tab(2 * 8 * FMM_NT, -1);
      int kt8 = 0;
      for (int ct = 0; ct < 8; ++ct) {
        int o = 0;
        for (int k = 0; k < FMM_NT_CLASS; ++k) {
          const int slot = c->cls_t_h[ct * FMM_NT_CLASS + k];
          tab[ct * FMM_NT + slot] = (int16_t)(o / 8);
          o += ry[slot];
        }
        kt8 = std::max(kt8, o / 8);
      }
      for (int cs = 0; cs < 8; ++cs)
        for (int k = 0; k < FMM_NT_CLASS; ++k) tab[8 * FMM_NT + cs * FMM_NT + c->src_t_h[cs * FMM_NT_CLASS + k]] = (int16_t)k;
      if (!c->svd_kap8) {
        FMM_TRY(dalloc(c, &ptr, sizeof(int16_t) * tab.size()));
        c->svd_kap8 = (int16_t*)ptr;
        c->svd_srcidx = c->svd_kap8 + 8 * FMM_NT;
      }
      FMM_CUDA(c, cudaMemcpyAsync(c->svd_kap8, tab.data(), sizeof(int16_t) * tab.size(), cudaMemcpyHostToDevice,
                                  c->stream));
      c->svd_kt8 = kt8;
      c->svd_kct = (8 * kt8 + 31) / 32;
    }
    FMM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->svd_ysig = sig;
    c->svd_yoff_h = yoff;
  }
  FMM_TRY(svd_banks(c));  // the mixed factor bank is laid out by the Y offsets
  if (xf16) return FMM_OK;  // the FP16 tensor-core form keeps no Y rows (m2l_svd_tc_prepare: Yx)
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  const size_t ybytes = (size_t)(c->rows > 0 ? c->rows : 1) * c->svd_YS * esz;
  if (ybytes > c->svd_Y_cap) {
    dfree(c, c->svd_Y, c->svd_Y_cap);
    c->svd_Y = nullptr;
    c->svd_Y_cap = 0;
    const size_t cap = ybytes + ybytes / 8;
    FMM_TRY(dalloc(c, &ptr, cap));
    c->svd_Y = ptr;
    c->svd_Y_cap = cap;
  }
  return FMM_OK;
}

fmm_status launch_m2l_svd_simt(Ctx* c, cudaStream_t s, int first_tile, int ntiles) {
  if (ntiles <= 0) return FMM_OK;
  SvdArgs a;
  a.tiles = c->tiles + first_tile;
  a.tile_src = c->tile_src + (int64_t)first_tile * FMM_NT_CLASS * FMM_TILE;
  a.tile_act = c->tile_act + (int64_t)first_tile * FMM_NT_CLASS;
  a.tile_nact = c->tile_nact + first_tile;
  a.src_act = c->src_act + (int64_t)first_tile * FMM_NT_CLASS;
  a.src_nact = c->src_nact + first_tile;
  a.cls_t = c->cls_t;
  a.src_t = c->src_t;
  a.t_ry = c->svd_ry;
  a.yoff = c->svd_yoff;
  a.YS = c->svd_YS;
  const int C = c->ncoef, cp = c->cpad;
  dim3 gp(ntiles, FMM_NT_CLASS);
  if (c->precision == FMM_MIXED) {
    dim3 ge(ntiles, 2, ceil_div(C + 1, 64));
    float* Y = (float*)c->svd_Y;
    k_m2l_proj<float, true><<<gp, FMM_TILE, 0, s>>>(a, c->lv, C, cp, c->svd_rp, c->svd_VThi, nullptr, c->Mhi,
                                                     c->Mlo, Y);
    k_m2l_expand<float, true><<<ge, 256, 0, s>>>(a, c->lv, C, cp, c->svd_rp, c->svd_Uhi, nullptr, Y, c->L32,
                                                 c->box, c->kernel_s);
  } else {
    dim3 ge(ntiles, 2, ceil_div(C, 64));
    double* Y = (double*)c->svd_Y;
    k_m2l_proj<double, false><<<gp, FMM_TILE, 0, s>>>(a, c->lv, C, cp, c->svd_rmax, c->svd_V64, nullptr, c->M64,
                                                       nullptr, Y);
    k_m2l_expand<double, false><<<ge, 256, 0, s>>>(a, c->lv, C, cp, c->svd_rmax, c->svd_U64, nullptr, Y, c->L64,
                                                   c->box, c->kernel_s);
  }
  return cuda_err(c, cudaGetLastError(), "compressed M2L launch");
}

}  // namespace fmm
