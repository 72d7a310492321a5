// farfield.cu -- P2M, M2M, L2L, L2P (+ final sum and scatter) and the SIMT
// M2L of the black-box FMM (Sec. 2.1, eq. 3-5; Sec. 3.2 traversal order).
//
// Interpolation: S(xbar_m, xi) = 1/p + 2/p sum_{n=1}^{p-1} T_n(xbar_m) T_n(xi)
// (eq. 5) with T_n(xbar_m) from a table and T_n(xi) by the recurrence;
// S_m(x) is the tensor product of eq. 4 (multi-index z fastest).
//   P2M (leaf)  M_m = sum_j q_j S_m((y_j - c)/a)
//   M2M         M_P = sum_children (A_sx (x) A_sy (x) A_sz) M_C, applied as three
//               1-D contractions (the tensor-product reformulation of Sec. 2.1.1)
//   M2L         L_T = (1/a) sum_{far S} K_t M_S            (Sec. 2.1.2)
//   L2L         L_C += (A_sx (x) A_sy (x) A_sz)^T L_P
//   L2P         phi = sum_m S_m(xi) L_m, F = -(1/a) sum_m grad_xi S_m(xi) L_m
// Mixed precision keeps multipoles as a TF32 hi/lo pair (hi + lo = M to FP32
// rounding) for the tensor-core M2L, and a local expansion as its cell mean
// (slot C of the row) plus FP32 deviations from it: with like-signed charges
// the far potential is large and smooth, and node values stored whole in FP32
// would lose the gradient (the force) to rounding by a factor that doubles
// per level.  FP64 keeps both whole in FP64.
#include "common.cuh"

namespace fmm {

namespace {

__device__ inline float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// S(xbar_m, xi) for m < P, and optionally dS/dxi.
template <int P, typename T, bool DERIV>
__device__ inline void interp_weights(const T* __restrict__ sC, T xi, T* S, T* dS) {
  T Tn[P], dTn[P];
  Tn[0] = T(1);
  if (P > 1) Tn[1] = xi;
#pragma unroll
  for (int n = 2; n < P; ++n) Tn[n] = T(2) * xi * Tn[n - 1] - Tn[n - 2];
  if (DERIV) {
    // dT_n/dxi = n U_{n-1}(xi)
    T U0 = T(1), U1 = T(2) * xi;
    dTn[0] = T(0);
    if (P > 1) dTn[1] = T(1);
#pragma unroll
    for (int n = 2; n < P; ++n) {
      dTn[n] = T(n) * U1;
      T U2 = T(2) * xi * U1 - U0;
      U0 = U1;
      U1 = U2;
    }
  }
#pragma unroll
  for (int m = 0; m < P; ++m) {
    T s = T(0), ds = T(0);
#pragma unroll
    for (int n = 1; n < P; ++n) {
      s += sC[m * P + n] * Tn[n];
      if (DERIV) ds += sC[m * P + n] * dTn[n];
    }
    S[m] = T(1) / T(P) + T(2) / T(P) * s;
    if (DERIV) dS[m] = T(2) / T(P) * ds;
  }
}

__device__ inline void cell_centre(const double* box, int level, uint32_t key, double* c, double& a) {
  int ix, iy, iz;
  demorton3(key, ix, iy, iz);
  double w = ldexp(box[3], -level);
  c[0] = box[0] + ((double)ix + 0.5) * w;
  c[1] = box[1] + ((double)iy + 0.5) * w;
  c[2] = box[2] + ((double)iz + 0.5) * w;
  a = 0.5 * w;
}

// ---------------------------------------------------------------- P2M

// One block per leaf (leaves of many particles).  The multipole is a sum of
// tensor products, M[mx][my][mz] = sum_j q_j Sx_j[mx] Sy_j[my] Sz_j[mz]: the
// weights of 32 particles at a time are staged in shared memory, thread
// (my, mz) forms w = q Sy Sz once per particle and adds w Sx[mx] for every mx
// (one staged load per multiply, the Sx row a broadcast), and 128 / P^2
// particle subsets run side by side and are added at the end.
template <int P, typename T, bool MIXED>
__global__ void __launch_bounds__(128)
k_p2m(LevelPtrs lv, int leaf, const double* __restrict__ box, const T* __restrict__ cheb, int cpad,
      const double4* __restrict__ pos64, const float4* __restrict__ pos32, T* __restrict__ Mout,
      T* __restrict__ Mlo) {
  constexpr int C = P * P * P, NB = 32, PP = P * P;
  constexpr int PARTS = PP <= 128 ? 128 / PP : 1;  // particle subsets summed side by side
  static_assert(PP <= 128, "one thread per (my, mz) pair");
  __shared__ T sS[NB][3][P];
  __shared__ T sq[NB];
  __shared__ T sC[P * P];
  __shared__ T red[PARTS > 1 ? PARTS - 1 : 1][C];
  const int cell = blockIdx.x, tid = threadIdx.x;
  const int pair = tid % PP, part = tid / PP, my = pair / P, mz = pair % P;
  const bool active = part < PARTS;
  for (int i = tid; i < P * P; i += 128) sC[i] = cheb[i];
  const int first = lv.first[leaf][cell], cnt = lv.count[leaf][cell];
  double ctr[3], a = 1.0;
  if (!MIXED) cell_centre(box, leaf, lv.key[leaf][cell], ctr, a);
  T acc[P];
#pragma unroll
  for (int k = 0; k < P; ++k) acc[k] = T(0);
  __syncthreads();
  for (int b0 = 0; b0 < cnt; b0 += NB) {
    const int nb = min(NB, cnt - b0);
    if (tid < 3 * nb) {
      const int j = tid / 3, d = tid - 3 * j;
      T xi, qq;
      if (MIXED) {
        float4 pp = pos32[first + b0 + j];
        xi = T(2) * (d == 0 ? pp.x : d == 1 ? pp.y : pp.z);
        qq = pp.w;
      } else {
        double4 pp = pos64[first + b0 + j];
        double v = d == 0 ? pp.x : d == 1 ? pp.y : pp.z;
        xi = (T)((v - ctr[d]) / a);
        qq = (T)pp.w;
      }
      T S[P];
      interp_weights<P, T, false>(sC, xi, S, nullptr);
#pragma unroll
      for (int m = 0; m < P; ++m) sS[j][d][m] = S[m];
      if (d == 0) sq[j] = qq;
    }
    __syncthreads();
    if (active)
      for (int j = part; j < nb; j += PARTS) {
        const T w = sq[j] * sS[j][1][my] * sS[j][2][mz];
#pragma unroll
        for (int mx = 0; mx < P; ++mx) acc[mx] += w * sS[j][0][mx];
      }
    __syncthreads();
  }
  if (active && part > 0)
#pragma unroll
    for (int mx = 0; mx < P; ++mx) red[part - 1][mx * PP + pair] = acc[mx];
  __syncthreads();
  if (part == 0) {
    const int64_t row = lv.row_off[leaf] + cell;
#pragma unroll
    for (int mx = 0; mx < P; ++mx) {
      T v = acc[mx];
      for (int q = 0; q + 1 < PARTS; ++q) v += red[q][mx * PP + pair];
      const int m = mx * PP + pair;  // (mx * P + my) * P + mz
      if (MIXED) {
        const float hi = tf32_rna((float)v);
        Mout[row * cpad + m] = hi;
        Mlo[row * cpad + m] = tf32_rna((float)v - hi);
      } else {
        Mout[row * cpad + m] = v;
      }
    }
  }
}

// Four leaves per block, a warp each (trees whose leaves hold a few
// particles, where a block per leaf would be mostly idle): the lanes compute
// the interpolation weights of up to 32 particles at a time, then each lane
// accumulates the coefficients m = lane, lane + 32, ...
template <int P, typename T, bool MIXED>
__global__ void __launch_bounds__(128)
k_p2m_warp(LevelPtrs lv, int leaf, int nleaf, const double* __restrict__ box, const T* __restrict__ cheb, int cpad,
           const double4* __restrict__ pos64, const float4* __restrict__ pos32, T* __restrict__ Mout,
           T* __restrict__ Mlo) {
  constexpr int C = P * P * P, NPER = (C + 31) / 32;
  __shared__ T sS[4][32][3][P];
  __shared__ T sq[4][32];
  __shared__ T sC[P * P];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < P * P; i += 128) sC[i] = cheb[i];
  __syncthreads();
  const int cell = blockIdx.x * 4 + warp;
  if (cell >= nleaf) return;
  const int first = lv.first[leaf][cell], cnt = lv.count[leaf][cell];
  double ctr[3], a = 1.0;
  if (!MIXED) cell_centre(box, leaf, lv.key[leaf][cell], ctr, a);
  T acc[NPER];
#pragma unroll
  for (int k = 0; k < NPER; ++k) acc[k] = T(0);
  for (int b0 = 0; b0 < cnt; b0 += 32) {
    const int nb = min(32, cnt - b0);
    if (lane < nb) {
      T xi[3], qq;
      if (MIXED) {
        const float4 pp = pos32[first + b0 + lane];
        xi[0] = T(2) * pp.x;
        xi[1] = T(2) * pp.y;
        xi[2] = T(2) * pp.z;
        qq = pp.w;
      } else {
        const double4 pp = pos64[first + b0 + lane];
        xi[0] = (T)((pp.x - ctr[0]) / a);
        xi[1] = (T)((pp.y - ctr[1]) / a);
        xi[2] = (T)((pp.z - ctr[2]) / a);
        qq = (T)pp.w;
      }
      for (int d = 0; d < 3; ++d) {
        T S[P];
        interp_weights<P, T, false>(sC, xi[d], S, nullptr);
#pragma unroll
        for (int m = 0; m < P; ++m) sS[warp][lane][d][m] = S[m];
      }
      sq[warp][lane] = qq;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NPER; ++k) {
      const int m = lane + 32 * k;
      if (m < C) {
        const int mx = m / (P * P), my = (m / P) % P, mz = m % P;
        T s = acc[k];
        for (int j = 0; j < nb; ++j)
          s += sq[warp][j] * sS[warp][j][0][mx] * sS[warp][j][1][my] * sS[warp][j][2][mz];
        acc[k] = s;
      }
    }
    __syncwarp();
  }
  const int64_t row = lv.row_off[leaf] + cell;
#pragma unroll
  for (int k = 0; k < NPER; ++k) {
    const int m = lane + 32 * k;
    if (m < C) {
      if (MIXED) {
        const float hi = tf32_rna((float)acc[k]);
        Mout[row * cpad + m] = hi;
        Mlo[row * cpad + m] = tf32_rna((float)acc[k] - hi);
      } else {
        Mout[row * cpad + m] = acc[k];
      }
    }
  }
}

// Mixed precision, a warp per leaf (4 per block), any leaf size: lanes
// compute the interpolation weights of up to 32 particles at a time (the
// charge folded into the x weights) into the warp's shared rows; then lane
// L owns the (my, mz) pairs L, L + 32, ... and, per particle, adds
// Sy[my] Sz[mz] q Sx[mx] into its P accumulators per pair -- the multipole
// as a sum of outer products, M[mx][(my, mz)] = sum_j (q_j Sx_j[mx])
// (Sy_j[my] Sz_j[mz]), with the particle's x row read once per particle and
// shared by the lane's pairs.  The results are written per mx row, lanes on
// consecutive coefficients.
template <int P>
__global__ void __launch_bounds__(128)
k_p2m_pairs(LevelPtrs lv, int leaf, int nleaf, const float* __restrict__ cheb, int cpad,
            const float4* __restrict__ pos32, float* __restrict__ Mhi, float* __restrict__ Mlo) {
  constexpr int PP = P * P, NPAIR = (PP + 31) / 32, PX = (P + 3) / 4 * 4;
  __shared__ __align__(16) float sX[4][32][PX];
  __shared__ float sY[4][32][P], sZ[4][32][P];
  __shared__ float sC[P * P];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < P * P; i += 128) sC[i] = cheb[i];
  __syncthreads();
  const int cell = blockIdx.x * 4 + warp;
  if (cell >= nleaf) return;
  const int first = lv.first[leaf][cell], cnt = lv.count[leaf][cell];
  int my[NPAIR], mz[NPAIR];
  bool own[NPAIR];
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const int pr = lane + 32 * k;
    own[k] = pr < PP;
    my[k] = own[k] ? pr / P : 0;
    mz[k] = own[k] ? pr % P : 0;
  }
  float acc[NPAIR][P];
#pragma unroll
  for (int k = 0; k < NPAIR; ++k)
#pragma unroll
    for (int mx = 0; mx < P; ++mx) acc[k][mx] = 0.f;
  for (int b0 = 0; b0 < cnt; b0 += 32) {
    const int nb = min(32, cnt - b0);
    if (lane < nb) {
      const float4 pp = pos32[first + b0 + lane];
      float S[P];
      interp_weights<P, float, false>(sC, 2.f * pp.x, S, nullptr);
#pragma unroll
      for (int m = 0; m < PX; ++m) sX[warp][lane][m] = m < P ? pp.w * S[m] : 0.f;
      interp_weights<P, float, false>(sC, 2.f * pp.y, S, nullptr);
#pragma unroll
      for (int m = 0; m < P; ++m) sY[warp][lane][m] = S[m];
      interp_weights<P, float, false>(sC, 2.f * pp.z, S, nullptr);
#pragma unroll
      for (int m = 0; m < P; ++m) sZ[warp][lane][m] = S[m];
    }
    __syncwarp();
    for (int j = 0; j < nb; ++j) {
      float x[PX];
#pragma unroll
      for (int m = 0; m < PX; m += 4) *(float4*)&x[m] = *(const float4*)&sX[warp][j][m];
#pragma unroll
      for (int k = 0; k < NPAIR; ++k) {
        const float w = sY[warp][j][my[k]] * sZ[warp][j][mz[k]];
#pragma unroll
        for (int mx = 0; mx < P; ++mx) acc[k][mx] = fmaf(w, x[mx], acc[k][mx]);
      }
    }
    __syncwarp();
  }
  const int64_t row = lv.row_off[leaf] + cell;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    if (!own[k]) continue;
#pragma unroll
    for (int mx = 0; mx < P; ++mx) {
      const int m = mx * PP + lane + 32 * k;
      const float hi = tf32_rna(acc[k][mx]);
      Mhi[row * cpad + m] = hi;
      Mlo[row * cpad + m] = tf32_rna(acc[k][mx] - hi);
    }
  }
}

// ---------------------------------------------------------------- M2M

// Children rows staged together (up to 8, within 16 KB of shared memory, so
// that every order stays inside the 48 KB of static shared memory): one
// global-load round trip per batch of children instead of one per child.
template <int C, typename T>
constexpr int child_batch() {
  return (16384 / (C * (int)sizeof(T))) >= 8 ? 8 : ((16384 / (C * (int)sizeof(T))) < 1 ? 1 : 16384 / (C * (int)sizeof(T)));
}

template <int P, typename T, bool MIXED>
__global__ void __launch_bounds__(256)
k_m2m(LevelPtrs lv, int l, const T* __restrict__ A, int cpad, const T* __restrict__ Mhi,
      const T* __restrict__ Mlo, T* __restrict__ Mout_hi, T* __restrict__ Mout_lo) {
  constexpr int C = P * P * P, NPER = (C + 255) / 256, CB = child_batch<C, T>();
  __shared__ T sA[2 * P * P];
  __shared__ T sin_[CB][C];
  __shared__ T su[C], sv[C];
  const int cell = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < 2 * P * P; i += 256) sA[i] = A[i];
  T acc[NPER];
#pragma unroll
  for (int k = 0; k < NPER; ++k) acc[k] = T(0);
  const int c0 = lv.first[l][cell], nc = lv.count[l][cell];
  for (int cb = c0; cb < c0 + nc; cb += CB) {
    const int nb = min(CB, c0 + nc - cb);
    __syncthreads();
    for (int e = tid; e < nb * C; e += 256) {
      const int k = e / C, m = e - k * C;
      const int64_t row = lv.row_off[l + 1] + cb + k;
      T v = Mhi[row * cpad + m];
      if (MIXED) v += Mlo[row * cpad + m];
      sin_[k][m] = v;
    }
    for (int k = 0; k < nb; ++k) {
      const uint32_t b = lv.key[l + 1][cb + k] & 7u;
      const T* Ax = sA + ((b >> 2) & 1) * P * P;
      const T* Ay = sA + ((b >> 1) & 1) * P * P;
      const T* Az = sA + (b & 1) * P * P;
      const T* in = sin_[k];
      __syncthreads();
      // z: u[x][y][mz] = sum_k Az[mz][k] in[x][y][k]
      for (int m = tid; m < C; m += 256) {
        const int xy = m / P, mz = m % P;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) s += Az[mz * P + q] * in[xy * P + q];
        su[m] = s;
      }
      __syncthreads();
      // y: v[x][my][z] = sum_k Ay[my][k] u[x][k][z]
      for (int m = tid; m < C; m += 256) {
        const int x = m / (P * P), my = (m / P) % P, z = m % P;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) s += Ay[my * P + q] * su[(x * P + q) * P + z];
        sv[m] = s;
      }
      __syncthreads();
      // x: acc[mx][y][z] += sum_k Ax[mx][k] v[k][y][z]
#pragma unroll
      for (int kk = 0; kk < NPER; ++kk) {
        const int m = tid + 256 * kk;
        if (m < C) {
          const int mx = m / (P * P), yz = m % (P * P);
          T s = T(0);
#pragma unroll
          for (int q = 0; q < P; ++q) s += Ax[mx * P + q] * sv[q * P * P + yz];
          acc[kk] += s;
        }
      }
    }
  }
  const int64_t row = lv.row_off[l] + cell;
#pragma unroll
  for (int k = 0; k < NPER; ++k) {
    const int m = tid + 256 * k;
    if (m < C) {
      if (MIXED) {
        float hi = tf32_rna((float)acc[k]);
        Mout_hi[row * cpad + m] = hi;
        Mout_lo[row * cpad + m] = tf32_rna((float)acc[k] - hi);
      } else {
        Mout_hi[row * cpad + m] = acc[k];
      }
    }
  }
}

// Mixed precision, one block per parent, every child at once: the three
// one-dimensional passes of the tensor-product M2M operator run over all
// children together, and children that differ only in the bit of the axis
// just transformed are added right after that pass (the operators of the
// remaining axes do not depend on it): 8 staged children -> z pass, pairs
// added -> 4 partial sums -> y pass -> 2 -> x pass -> the parent.  Three
// block barriers per parent instead of three per child; 14 C one-dimensional
// sums per parent instead of 24 C.
template <int P>
constexpr bool m2m_fused_fits() {
  return (14 * P * P * P + 2 * P * P) * 4 <= 46 * 1024;
}

template <int P>
__global__ void __launch_bounds__(256)
k_m2m_fused(LevelPtrs lv, int l, const float* __restrict__ A, int cpad, float* __restrict__ Mhi,
            float* __restrict__ Mlo) {
  constexpr int C = P * P * P, PP = P * P;
  __shared__ float sA[2 * PP];
  __shared__ float sin_[8][C];
  __shared__ float su[4][C];
  __shared__ float sv[2][C];
  const int cell = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < 2 * PP; i += 256) sA[i] = A[i];
  const int c0 = lv.first[l][cell], nc = lv.count[l][cell];
  __shared__ int slot_of[8];
  if (tid < 8) slot_of[tid] = -1;
  __syncthreads();
  if (tid < nc) slot_of[lv.key[l + 1][c0 + tid] & 7u] = c0 + tid;
  __syncthreads();
  for (int e = tid; e < 8 * C; e += 256) {
    const int b = e / C, m = e - b * C;
    const int ch = slot_of[b];
    float v = 0.f;
    if (ch >= 0) {
      const int64_t row = lv.row_off[l + 1] + ch;
      v = Mhi[row * cpad + m] + Mlo[row * cpad + m];
    }
    sin_[b][m] = v;
  }
  __syncthreads();
  // z: u[g][x][y][mz] = sum over bit0 and q of Az_bit0[mz][q] in[2 g + bit0][x][y][q]
  for (int e = tid; e < 4 * C; e += 256) {
    const int g = e / C, m = e - g * C, xy = m / P, mz = m % P;
    float s = 0.f;
#pragma unroll
    for (int b0 = 0; b0 < 2; ++b0) {
      const float* Az = sA + b0 * PP + mz * P;
      const float* in = sin_[2 * g + b0] + xy * P;
#pragma unroll
      for (int q = 0; q < P; ++q) s += Az[q] * in[q];
    }
    su[g][m] = s;
  }
  __syncthreads();
  // y: v[g][x][my][z] = sum over bit1 and q of Ay_bit1[my][q] u[2 g + bit1][x][q][z]
  for (int e = tid; e < 2 * C; e += 256) {
    const int g = e / C, m = e - g * C, x = m / PP, my = (m / P) % P, z = m % P;
    float s = 0.f;
#pragma unroll
    for (int b1 = 0; b1 < 2; ++b1) {
      const float* Ay = sA + b1 * PP + my * P;
      const float* u = su[2 * g + b1] + x * PP + z;
#pragma unroll
      for (int q = 0; q < P; ++q) s += Ay[q] * u[q * P];
    }
    sv[g][m] = s;
  }
  __syncthreads();
  // x: parent[mx][y][z] = sum over bit2 and q of Ax_bit2[mx][q] v[bit2][q][y][z]
  const int64_t prow = lv.row_off[l] + cell;
  for (int m = tid; m < C; m += 256) {
    const int mx = m / PP, yz = m % PP;
    float s = 0.f;
#pragma unroll
    for (int b2 = 0; b2 < 2; ++b2) {
      const float* Ax = sA + b2 * PP + mx * P;
      const float* v = sv[b2] + yz;
#pragma unroll
      for (int q = 0; q < P; ++q) s += Ax[q] * v[q * PP];
    }
    const float hi = tf32_rna(s);
    Mhi[prow * cpad + m] = hi;
    Mlo[prow * cpad + m] = tf32_rna(s - hi);
  }
}

// Mixed precision L2L, one block per parent, every child at once (the
// mirror of k_m2m_fused): the parent's deviations through the z pass for
// both values of a child's z bit (2 arrays), the y pass for both y bits (4),
// then the x pass straight into each child's row (its own M2L part added);
// the parent's mean passes to every child unchanged.
template <int P>
__global__ void __launch_bounds__(256)
k_l2l_fused(LevelPtrs lv, int l, const float* __restrict__ A, int cpad, float* __restrict__ Lbuf) {
  constexpr int C = P * P * P, PP = P * P;
  __shared__ float sA[2 * PP];
  __shared__ float sin_[C];
  __shared__ float su[2][C];
  __shared__ float sv[4][C];
  __shared__ int bits[8];
  const int cell = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < 2 * PP; i += 256) sA[i] = A[i];
  const int64_t prow = lv.row_off[l] + cell;
  for (int m = tid; m < C; m += 256) sin_[m] = Lbuf[prow * cpad + m];
  const float mean = Lbuf[prow * cpad + C];
  const int c0 = lv.first[l][cell], nc = lv.count[l][cell];
  if (tid < nc) bits[tid] = (int)(lv.key[l + 1][c0 + tid] & 7u);
  __syncthreads();
  // z: u[b0][mx][my][z'] = sum_q Az_b0[q][z'] in[mx][my][q]
  for (int e = tid; e < 2 * C; e += 256) {
    const int b0 = e / C, m = e - b0 * C, xy = m / P, zp = m % P;
    const float* Az = sA + b0 * PP + zp;
    const float* in = sin_ + xy * P;
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < P; ++q) s += Az[q * P] * in[q];
    su[b0][m] = s;
  }
  __syncthreads();
  // y: v[2 b1 + b0][mx][y'][z'] = sum_q Ay_b1[q][y'] u[b0][mx][q][z']
  for (int e = tid; e < 4 * C; e += 256) {
    const int g = e / C, m = e - g * C, x = m / PP, yp = (m / P) % P, z = m % P;
    const float* Ay = sA + (g >> 1) * PP + yp;
    const float* u = su[g & 1] + x * PP + z;
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < P; ++q) s += Ay[q * P] * u[q * P];
    sv[g][m] = s;
  }
  __syncthreads();
  // x: L_child[x'][y'][z'] += sum_q Ax_b2[q][x'] v[child's (b1, b0)][q][y'][z']; thread (g, y'z')
  // holds v[g][.][y'z'] in registers and serves the children of group g = (b1, b0)
  for (int e = tid; e < 4 * PP; e += 256) {
    const int g = e / PP, yz = e - g * PP;
    float vr[P];
#pragma unroll
    for (int q = 0; q < P; ++q) vr[q] = sv[g][q * PP + yz];
    for (int k = 0; k < nc; ++k) {
      const int b = bits[k];
      if ((b & 3) != g) continue;
      const float* Ax = sA + ((b >> 2) & 1) * PP;
      float* out = Lbuf + (lv.row_off[l + 1] + c0 + k) * cpad + yz;
#pragma unroll
      for (int xp = 0; xp < P; ++xp) {
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < P; ++q) s += Ax[q * P + xp] * vr[q];
        out[xp * PP] += s;
      }
    }
  }
  if (tid < nc) Lbuf[(lv.row_off[l + 1] + c0 + tid) * cpad + C] += mean;
}

// ---------------------------------------------------------------- L2L

template <int P, typename T, bool MEAN>
__global__ void __launch_bounds__(256)
k_l2l(LevelPtrs lv, int l, const T* __restrict__ A, int cpad, T* __restrict__ Lbuf) {
  constexpr int C = P * P * P, CB = child_batch<C + 1, T>();
  __shared__ T sA[2 * P * P];
  __shared__ T sin_[C], su[C], sv[C];
  __shared__ T sch[CB][C + 1];  // the children's own rows (from M2L), staged per batch
  const int cell = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < 2 * P * P; i += 256) sA[i] = A[i];
  const int64_t prow = lv.row_off[l] + cell;
  for (int m = tid; m < C; m += 256) sin_[m] = Lbuf[prow * cpad + m];
  // interpolation reproduces constants, so the parent's mean passes to each
  // child unchanged and only the deviations go through the L2L matrices
  const T mean = MEAN ? Lbuf[prow * cpad + C] : T(0);
  const int c0 = lv.first[l][cell], nc = lv.count[l][cell];
  for (int cb = c0; cb < c0 + nc; cb += CB) {
    const int nb = min(CB, c0 + nc - cb);
    __syncthreads();
    for (int e = tid; e < nb * (C + 1); e += 256) {
      const int k = e / (C + 1), m = e - k * (C + 1);
      sch[k][m] = (MEAN || m < C) ? Lbuf[(lv.row_off[l + 1] + cb + k) * cpad + m] : T(0);
    }
    for (int k = 0; k < nb; ++k) {
      const int ch = cb + k;
      const uint32_t b = lv.key[l + 1][ch] & 7u;
      const T* Ax = sA + ((b >> 2) & 1) * P * P;
      const T* Ay = sA + ((b >> 1) & 1) * P * P;
      const T* Az = sA + (b & 1) * P * P;
      __syncthreads();
      // z: u[mx][my][z'] = sum_k Az[k][z'] in[mx][my][k]
      for (int m = tid; m < C; m += 256) {
        const int xy = m / P, zp = m % P;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) s += Az[q * P + zp] * sin_[xy * P + q];
        su[m] = s;
      }
      __syncthreads();
      // y: v[mx][y'][z'] = sum_k Ay[k][y'] u[mx][k][z']
      for (int m = tid; m < C; m += 256) {
        const int x = m / (P * P), yp = (m / P) % P, z = m % P;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) s += Ay[q * P + yp] * su[(x * P + q) * P + z];
        sv[m] = s;
      }
      __syncthreads();
      // x: L_C[x'][y'][z'] += sum_k Ax[k][x'] v[k][y'][z']
      const int64_t crow = lv.row_off[l + 1] + ch;
      for (int m = tid; m < C; m += 256) {
        const int xp = m / (P * P), yz = m % (P * P);
        T s = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) s += Ax[q * P + xp] * sv[q * P * P + yz];
        Lbuf[crow * cpad + m] = sch[k][m] + s;
      }
      if (MEAN && tid == 0) Lbuf[crow * cpad + C] = sch[k][C] + mean;
    }
  }
}

// ---------------------------------------------------------------- L2P + output

// Far-field potential of one particle from its leaf's local expansion Lr (C
// values; the mixed path's cell mean in Lr[C]) at xi, the particle's position
// in the leaf's frame, and the potential's derivatives with respect to xi
// (the field is -1/a times them, a = the leaf's half-width).
template <int P, typename T, bool MIXED>
__device__ __forceinline__ void l2p_eval(const T* __restrict__ Lrow, const T* __restrict__ sC, const T xi[3],
                                         T& pf, T& ax, T& ay, T& az) {
  constexpr int C = P * P * P;
  T Sx[P], Sy[P], Sz[P], dSx[P], dSy[P], dSz[P];
  interp_weights<P, T, true>(sC, xi[0], Sx, dSx);
  interp_weights<P, T, true>(sC, xi[1], Sy, dSy);
  interp_weights<P, T, true>(sC, xi[2], Sz, dSz);
  T f = T(0);
  ax = ay = az = T(0);
  // the x loop stays rolled: unrolling all P^3 terms needs more registers
  // than occupancy allows
#pragma unroll 1
  for (int mx = 0; mx < P; ++mx) {
#pragma unroll
    for (int my = 0; my < P; ++my) {
      const T* Lr = Lrow + (mx * P + my) * P;
      T sz = T(0), dz = T(0);
#pragma unroll
      for (int mz = 0; mz < P; ++mz) {
        sz += Lr[mz] * Sz[mz];
        dz += Lr[mz] * dSz[mz];
      }
      const T sxy = Sx[mx] * Sy[my];
      f += sxy * sz;
      ax += dSx[mx] * Sy[my] * sz;
      ay += Sx[mx] * dSy[my] * sz;
      az += sxy * dz;
    }
  }
  pf = MIXED ? f + Lrow[C] : f;  // mixed: cell mean + deviations
}

// xi of particle r in its leaf's frame
template <typename T, bool MIXED>
__device__ __forceinline__ void leaf_xi(int64_t r, const double4* __restrict__ pos64, const float4* __restrict__ pos32,
                                        const double* ctr, double a, T* xi) {
  if (MIXED) {
    const float4 pp = pos32[r];
    xi[0] = T(2) * pp.x;
    xi[1] = T(2) * pp.y;
    xi[2] = T(2) * pp.z;
  } else {
    const double4 pp = pos64[r];
    xi[0] = (T)((pp.x - ctr[0]) / a);
    xi[1] = (T)((pp.y - ctr[1]) / a);
    xi[2] = (T)((pp.z - ctr[2]) / a);
  }
}

// far + near, scaled to the problem's units (scaled: a batched tree, lam and
// lam2 the factors of phi and F), scattered to the caller's order.  Mixed:
// the far field (FP32, field = -ia times the xi derivatives, ia = 1 / a) and
// the FP32 near field are added in FP32 and widened to FP64 for the output;
// FP64: everything in FP64.
template <typename T, bool MIXED>
__device__ __forceinline__ void l2p_store(int64_t r, T pf, T ax, T ay, T az, double a, float ia, bool scaled,
                                          double lam, double lam2, const float4* __restrict__ near32,
                                          const double4* __restrict__ near64, const int32_t* __restrict__ perm,
                                          double* __restrict__ phi, double* __restrict__ F) {
  const int64_t i = perm[r];
  double v[4];
  if (MIXED) {
    const float4 nr = near32[r];
    v[0] = (double)((float)pf + nr.x);
    v[1] = (double)fmaf(-(float)ax, ia, nr.y);
    v[2] = (double)fmaf(-(float)ay, ia, nr.z);
    v[3] = (double)fmaf(-(float)az, ia, nr.w);
  } else {
    const double4 nr = near64[r];
    v[0] = (double)pf + nr.x;
    v[1] = -(double)ax / a + nr.y;
    v[2] = -(double)ay / a + nr.z;
    v[3] = -(double)az / a + nr.w;
  }
  if (scaled) {
    v[0] *= lam;
    v[1] *= lam2;
    v[2] *= lam2;
    v[3] *= lam2;
  }
  phi[i] = v[0];
  F[3 * i] = v[1];
  F[3 * i + 1] = v[2];
  F[3 * i + 2] = v[3];
}

// One warp per leaf: the leaf's local expansion is staged in shared memory
// and the lanes take its particles (leaves with many particles).
template <int P, typename T, bool MIXED>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 2)
k_l2p_out(LevelPtrs lv, int leaf, int nleaf, const double* __restrict__ box, const T* __restrict__ cheb,
          int cpad, const T* __restrict__ L, int has_far, const double4* __restrict__ pos64,
          const float4* __restrict__ pos32, const float4* __restrict__ near32,
          const double4* __restrict__ near64, const int32_t* __restrict__ perm, double* __restrict__ phi,
          double* __restrict__ F, const double* __restrict__ fscale, double ks) {
  constexpr int C = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sL = (T*)smem_raw;
  __shared__ T sC[P * P];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < P * P; i += 128) sC[i] = cheb[i];
  __syncthreads();
  const int cell = blockIdx.x * 4 + warp;
  if (cell >= nleaf) return;
  T* myL = sL + warp * cpad;
  if (has_far) {
    const int64_t row = lv.row_off[leaf] + cell;
    for (int m = lane; m <= C; m += 32) myL[m] = (MIXED || m < C) ? L[row * cpad + m] : T(0);
  }
  __syncwarp();
  const int first = lv.first[leaf][cell], cnt = lv.count[leaf][cell];
  double ctr[3] = {0.0, 0.0, 0.0}, a = 1.0;
  if (!MIXED) cell_centre(box, leaf, lv.key[leaf][cell], ctr, a);
  const float ia = MIXED ? __double2float_rn(box[6]) : 1.f;
  // batched trees: back from the forest cube to the problem's own units
  // (distances there are lambda times the problem's: phi scales by lambda^s,
  // F by lambda^(s+1))
  const int prob = fscale ? lv.slot[leaf][cell] : -1;
  const double lam = prob >= 0 ? kernel_scale(fscale[prob], ks) : 1.0;
  const double lam2 = prob >= 0 ? lam * fscale[prob] : 1.0;
  for (int r = first + lane; r < first + cnt; r += 32) {
    T pf = T(0), ax = T(0), ay = T(0), az = T(0);
    if (has_far) {
      T xi[3];
      leaf_xi<T, MIXED>(r, pos64, pos32, ctr, a, xi);
      l2p_eval<P, T, MIXED>(myL, sC, xi, pf, ax, ay, az);
    }
    l2p_store<T, MIXED>(r, pf, ax, ay, az, a, ia, prob >= 0, lam, lam2, near32, near64, perm, phi, F);
  }
}

// Mixed precision, a warp per leaf, the lanes on the leaf's particles (the
// arithmetic of l2p_eval): the leaf's local expansion is staged in shared
// memory as P^2 rows of the mz coefficients padded to a multiple of four,
// and the Chebyshev table likewise, so that each row arrives by 16-byte
// shared loads (two per row at P = 7, against seven 4-byte loads).
template <int P>
__device__ __forceinline__ void interp_weights_pad(const float* __restrict__ sCp, float xi, float* S, float* dS) {
  constexpr int PX = (P + 3) / 4 * 4;
  float Tn[PX], dTn[PX];
  Tn[0] = 1.f;
  if (P > 1) Tn[1] = xi;
#pragma unroll
  for (int n = 2; n < PX; ++n) Tn[n] = n < P ? 2.f * xi * Tn[n - 1] - Tn[n - 2] : 0.f;
  float U0 = 1.f, U1 = 2.f * xi;
  dTn[0] = 0.f;
  if (P > 1) dTn[1] = 1.f;
#pragma unroll
  for (int n = 2; n < PX; ++n) {
    dTn[n] = n < P ? (float)n * U1 : 0.f;
    const float U2 = 2.f * xi * U1 - U0;
    U0 = U1;
    U1 = U2;
  }
#pragma unroll
  for (int m = 0; m < P; ++m) {
    float row[PX];
#pragma unroll
    for (int n = 0; n < PX; n += 4) *(float4*)&row[n] = *(const float4*)&sCp[m * PX + n];
    float s = 0.f, ds = 0.f;
#pragma unroll
    for (int n = 1; n < P; ++n) {
      s += row[n] * Tn[n];
      ds += row[n] * dTn[n];
    }
    S[m] = 1.f / (float)P + 2.f / (float)P * s;
    dS[m] = 2.f / (float)P * ds;
  }
}

template <int P>
__global__ void __launch_bounds__(128, 8)
k_l2p_mixed(LevelPtrs lv, int leaf, int nleaf, const double* __restrict__ box, const float* __restrict__ cheb,
            int cpad, const float* __restrict__ L, int has_far, const float4* __restrict__ pos32,
            const float4* __restrict__ near32, const int32_t* __restrict__ perm, double* __restrict__ phi,
            double* __restrict__ F, const double* __restrict__ fscale, double ks) {
  constexpr int C = P * P * P, PP = P * P, PX = (P + 3) / 4 * 4;
  __shared__ __align__(16) float sCp[P * PX];
  __shared__ __align__(16) float sL[4][PP * PX];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < P * PX; i += 128) sCp[i] = (i % PX) < P ? cheb[(i / PX) * P + i % PX] : 0.f;
  __syncthreads();
  const int cell = blockIdx.x * 4 + warp;
  if (cell >= nleaf) return;
  float* myL = sL[warp];
  float mean = 0.f;
  if (has_far) {
    const int64_t row = lv.row_off[leaf] + cell;
    for (int e = lane; e < PP * PX; e += 32) {
      const int r = e / PX, z = e - r * PX;
      myL[e] = z < P ? L[row * cpad + r * P + z] : 0.f;
    }
    mean = L[row * cpad + C];
  }
  __syncwarp();
  const int first = lv.first[leaf][cell], cnt = lv.count[leaf][cell];
  const float ia = __double2float_rn(box[6]);
  const int prob = fscale ? lv.slot[leaf][cell] : -1;
  const double lam = prob >= 0 ? kernel_scale(fscale[prob], ks) : 1.0;
  const double lam2 = prob >= 0 ? lam * fscale[prob] : 1.0;
  for (int r = first + lane; r < first + cnt; r += 32) {
    float pf = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    if (has_far) {
      const float4 pp = pos32[r];
      float Sx[P], Sy[P], Sz[P], dSx[P], dSy[P], dSz[P];
      interp_weights_pad<P>(sCp, 2.f * pp.x, Sx, dSx);
      interp_weights_pad<P>(sCp, 2.f * pp.y, Sy, dSy);
      interp_weights_pad<P>(sCp, 2.f * pp.z, Sz, dSz);
      // per mx: the z contraction of its P rows, then the y contraction
      // (Ty = sum Sy sz, dTy = sum dSy sz, Tz = sum Sy dz), then x
      float f = 0.f;
#pragma unroll 1
      for (int mx = 0; mx < P; ++mx) {
        float Ty = 0.f, dTy = 0.f, Tz = 0.f;
#pragma unroll
        for (int my = 0; my < P; ++my) {
          float Lr[PX];
#pragma unroll
          for (int n = 0; n < PX; n += 4) *(float4*)&Lr[n] = *(const float4*)&myL[(mx * P + my) * PX + n];
          float sz = 0.f, dz = 0.f;
#pragma unroll
          for (int mz = 0; mz < P; ++mz) {
            sz += Lr[mz] * Sz[mz];
            dz += Lr[mz] * dSz[mz];
          }
          Ty += Sy[my] * sz;
          dTy += dSy[my] * sz;
          Tz += Sy[my] * dz;
        }
        f += Sx[mx] * Ty;
        ax += dSx[mx] * Ty;
        ay += Sx[mx] * dTy;
        az += Sx[mx] * Tz;
      }
      pf = f + mean;
    }
    l2p_store<float, true>(r, pf, ax, ay, az, 1.0, ia, prob >= 0, lam, lam2, near32, nullptr, perm, phi, F);
  }
}

// One thread per particle (leaves with few particles, where a warp per leaf
// would leave most lanes idle): the particle's leaf comes from the per-
// particle leaf index and its local expansion is read through the L1 cache
// (neighbouring threads share leaves, so the loads are mostly broadcasts).
template <int P, typename T, bool MIXED>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 2)
k_l2p_pp(LevelPtrs lv, int leaf, int64_t n, const int32_t* __restrict__ pleaf, const double* __restrict__ box,
         const T* __restrict__ cheb, int cpad, const T* __restrict__ L, int has_far,
         const double4* __restrict__ pos64, const float4* __restrict__ pos32, const float4* __restrict__ near32,
         const double4* __restrict__ near64, const int32_t* __restrict__ perm, double* __restrict__ phi,
         double* __restrict__ F, const double* __restrict__ fscale, double ks) {
  __shared__ T sC[P * P];
  for (int i = threadIdx.x; i < P * P; i += 128) sC[i] = cheb[i];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (r >= n) return;
  const int cell = pleaf[r];
  double ctr[3] = {0.0, 0.0, 0.0}, a = 1.0;
  if (!MIXED) cell_centre(box, leaf, lv.key[leaf][cell], ctr, a);
  const float ia = MIXED ? __double2float_rn(box[6]) : 1.f;
  const int prob = fscale ? lv.slot[leaf][cell] : -1;
  const double lam = prob >= 0 ? kernel_scale(fscale[prob], ks) : 1.0;
  const double lam2 = prob >= 0 ? lam * fscale[prob] : 1.0;
  T pf = T(0), ax = T(0), ay = T(0), az = T(0);
  if (has_far) {
    T xi[3];
    leaf_xi<T, MIXED>(r, pos64, pos32, ctr, a, xi);
    l2p_eval<P, T, MIXED>(L + (lv.row_off[leaf] + cell) * (int64_t)cpad, sC, xi, pf, ax, ay, az);
  }
  l2p_store<T, MIXED>(r, pf, ax, ay, az, a, ia, prob >= 0, lam, lam2, near32, near64, perm, phi, F);
}

// ---------------------------------------------------------------- M2L (SIMT)
// One CTA computes 64 target rows x 64 coefficients of a tile's local
// expansions: a GEMM whose K dimension runs over (active transfer vector t,
// source coefficient n), the A operand gathered from the source cells'
// multipoles and B = K_t^T.  SPLIT: operands are TF32 hi/lo pairs (used as
// FP32 sums), the operator bank has row stride cpad.

template <typename T, bool SPLIT>
__global__ void __launch_bounds__(256)
k_m2l_simt(const Tile* __restrict__ tiles, const int32_t* __restrict__ tile_src,
           const int16_t* __restrict__ tile_act, const int32_t* __restrict__ tile_nact, LevelPtrs lv,
           const int16_t* __restrict__ cls_t, const T* __restrict__ Khi, const T* __restrict__ Klo,
           int kstride, int C, int cpad, const T* __restrict__ Mhi, const T* __restrict__ Mlo,
           T* __restrict__ Lout, const double* __restrict__ box, double ks, int lev_ops) {
  __shared__ T As[16][64];
  __shared__ T Bs[16][64 + 1];
  __shared__ int srow[64];
  const int tile = blockIdx.x, half = blockIdx.y, col0 = blockIdx.z * 64;
  const int ncol = SPLIT ? C + 1 : C;  // mixed: deviations + the cell mean (row C of the bank)
  if (col0 >= ncol) return;
  const Tile tl = tiles[tile];
  if (half * 64 >= tl.count) return;
  const int l = tl.level;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nact = tile_nact[tile];
  const int64_t rbase = lv.row_off[l];
  // Per transfer vector the products are summed in T; the running total over
  // transfer vectors is compensated (Kahan) so that the long sum, whose terms
  // largely cancel in the deviation columns, keeps FP32 precision.
  T acc[4][4], tot[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) tot[i][j] = cmp[i][j] = T(0);
  for (int a = 0; a < nact; ++a) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int k = tile_act[(int64_t)tile * FMM_NT_CLASS + a];
    // lev_ops: one operator bank per level 2.. (kernels with c > 0)
    const int slot = cls_t[tl.cls * FMM_NT_CLASS + k] + (lev_ops ? (l - 2) * FMM_NT : 0);
    __syncthreads();
    if (tid < 64) srow[tid] = tile_src[((int64_t)tile * FMM_NT_CLASS + k) * FMM_TILE + half * 64 + tid];
    const T* Kh = Khi + (int64_t)slot * kstride * kstride;
    const T* Kl = SPLIT ? Klo + (int64_t)slot * kstride * kstride : nullptr;
    for (int n0 = 0; n0 < C; n0 += 16) {
      __syncthreads();
      // A: 64 rows x 16 coefficients (16 consecutive threads read one row segment)
#pragma unroll
      for (int e = tid; e < 64 * 16; e += 256) {
        const int r = e >> 4, kk = e & 15;
        const int64_t off = (rbase + srow[r]) * cpad + n0 + kk;
        T v = Mhi[off];
        if (SPLIT) v += Mlo[off];
        As[kk][r] = v;
      }
      // B: Bs[kk][c] = K_t[col0 + c][n0 + kk]
#pragma unroll
      for (int e = tid; e < 64 * 16; e += 256) {
        const int cc = e >> 4, kk = e & 15;
        const int m = col0 + cc, nn = n0 + kk;
        T v = T(0);
        if (m < ncol && nn < C) {
          v = Kh[(int64_t)m * kstride + nn];
          if (SPLIT) v += Kl[(int64_t)m * kstride + nn];
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
    const int cell = lv.cls[l][tl.first + r];
    const int64_t row = rbase + cell;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = col0 + tx + 16 * j;
      if (m < ncol) Lout[row * cpad + m] = (T)((double)tot[i][j] * inv_a);
    }
  }
}

// ---------------------------------------------------------------- readout

// b: second half of a split pair; add_mean: add the row's mean slot (column C)
template <typename T>
__global__ void k_rows_to_f64(int64_t nrows, int64_t row0, int C, int cpad, const T* __restrict__ a,
                              const T* __restrict__ b, int add_mean, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * C) return;
  int64_t r = i / C;
  int m = (int)(i - r * C);
  double v = (double)a[(row0 + r) * cpad + m];
  if (b) v += (double)b[(row0 + r) * cpad + m];
  if (add_mean) v += (double)a[(row0 + r) * cpad + C];
  out[i] = v;
}

// ---------------------------------------------------------------- launchers

template <int P>
fmm_status upward_p(Ctx* c, cudaStream_t s, cudaEvent_t after_p2m) {
  const int Lf = c->leaf;
  // leaves of a few particles (the same lane-utilisation rule as L2P): a warp per leaf
  const int nleaf = c->lv.ncell[Lf];
  const bool small = 10 * c->n < 6 * 32 * (int64_t)c->p2p_nitems;
  if (c->precision == FMM_MIXED) {
    k_p2m_pairs<P><<<ceil_div(nleaf, 4), 128, 0, s>>>(c->lv, Lf, nleaf, c->cheb32, c->cpad, c->pos32, c->Mhi,
                                                      c->Mlo);
    if (after_p2m) FMM_CUDA(c, cudaEventRecord(after_p2m, s));  // the leaf level's multipoles are final
    for (int l = Lf - 1; l >= 2; --l) {
      if constexpr (m2m_fused_fits<P>())
        k_m2m_fused<P><<<c->lv.ncell[l], 256, 0, s>>>(c->lv, l, c->m2m32, c->cpad, c->Mhi, c->Mlo);
      else
        k_m2m<P, float, true><<<c->lv.ncell[l], 256, 0, s>>>(c->lv, l, c->m2m32, c->cpad, c->Mhi, c->Mlo, c->Mhi,
                                                             c->Mlo);
    }
  } else {
    if (small)
      k_p2m_warp<P, double, false><<<ceil_div(nleaf, 4), 128, 0, s>>>(c->lv, Lf, nleaf, c->box, c->cheb64, c->cpad,
                                                                      c->pos64, c->pos32, c->M64, nullptr);
    else
      k_p2m<P, double, false><<<nleaf, 128, 0, s>>>(c->lv, Lf, c->box, c->cheb64, c->cpad, c->pos64, c->pos32,
                                                    c->M64, nullptr);
    for (int l = Lf - 1; l >= 2; --l)
      k_m2m<P, double, false><<<c->lv.ncell[l], 256, 0, s>>>(c->lv, l, c->m2m64, c->cpad, c->M64, nullptr,
                                                             c->M64, nullptr);
  }
  return cuda_err(c, cudaGetLastError(), "upward pass launch");
}

template <int P>
fmm_status l2l_p(Ctx* c, cudaStream_t s) {
  for (int l = 2; l <= c->leaf - 1; ++l) {
    if (c->precision == FMM_MIXED) {
      if constexpr (m2m_fused_fits<P>())
        k_l2l_fused<P><<<c->lv.ncell[l], 256, 0, s>>>(c->lv, l, c->m2m32, c->cpad, c->L32);
      else
        k_l2l<P, float, true><<<c->lv.ncell[l], 256, 0, s>>>(c->lv, l, c->m2m32, c->cpad, c->L32);
    } else
      k_l2l<P, double, false><<<c->lv.ncell[l], 256, 0, s>>>(c->lv, l, c->m2m64, c->cpad, c->L64);
  }
  return cuda_err(c, cudaGetLastError(), "L2L launch");
}

template <int P>
fmm_status l2p_p(Ctx* c, cudaStream_t s, double* phi, double* F) {
  const int Lf = c->leaf, nleaf = c->lv.ncell[Lf];
  const int has_far = Lf >= 2;
  if (nleaf == 0) return FMM_OK;
  const double* fs = c->forest ? c->fb_scale : nullptr;
  // a warp per leaf keeps n / (32 x warps) of its lanes busy (one warp per
  // 32-particle batch of a leaf, as the P2P work items count them); below 60 %
  // one thread per particle wins
  const bool pp = c->pleaf && 10 * c->n < 6 * 32 * (int64_t)c->p2p_nitems;
  if (c->precision == FMM_MIXED) {
    if (pp)
      k_l2p_pp<P, float, true><<<ceil_div(c->n, 128), 128, 0, s>>>(
          c->lv, Lf, c->n, c->pleaf, c->box, c->cheb32, c->cpad, c->L32, has_far, c->pos64, c->pos32, c->near32,
          c->near64, c->perm, phi, F, fs, c->kernel_s);
    else
      k_l2p_mixed<P><<<ceil_div(nleaf, 4), 128, 0, s>>>(c->lv, Lf, nleaf, c->box, c->cheb32, c->cpad, c->L32,
                                                        has_far, c->pos32, c->near32, c->perm, phi, F, fs,
                                                        c->kernel_s);
  } else {
    if (pp)
      k_l2p_pp<P, double, false><<<ceil_div(c->n, 128), 128, 0, s>>>(
          c->lv, Lf, c->n, c->pleaf, c->box, c->cheb64, c->cpad, c->L64, has_far, c->pos64, c->pos32, c->near32,
          c->near64, c->perm, phi, F, fs, c->kernel_s);
    else
      k_l2p_out<P, double, false><<<ceil_div(nleaf, 4), 128, 4 * c->cpad * sizeof(double), s>>>(
          c->lv, Lf, nleaf, c->box, c->cheb64, c->cpad, c->L64, has_far, c->pos64, c->pos32, c->near32, c->near64,
          c->perm, phi, F, fs, c->kernel_s);
  }
  return cuda_err(c, cudaGetLastError(), "L2P launch");
}

}  // namespace

fmm_status launch_upward(Ctx* c, cudaStream_t s, cudaEvent_t after_p2m) {
  if (c->leaf < 2 || c->n == 0) return FMM_OK;
#define CALL(P) upward_p<P>(c, s, after_p2m)
  switch (c->order) {
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 5: return CALL(5);
    case 6: return CALL(6);
    case 7: return CALL(7);
    case 8: return CALL(8);
    case 9: return CALL(9);
    case 10: return CALL(10);
  }
#undef CALL
  return FMM_ERR_ARG;
}

fmm_status launch_l2l(Ctx* c, cudaStream_t s) {
  if (c->leaf < 3 || c->n == 0) return FMM_OK;
#define CALL(P) l2l_p<P>(c, s)
  switch (c->order) {
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 5: return CALL(5);
    case 6: return CALL(6);
    case 7: return CALL(7);
    case 8: return CALL(8);
    case 9: return CALL(9);
    case 10: return CALL(10);
  }
#undef CALL
  return FMM_ERR_ARG;
}

fmm_status launch_l2p_out(Ctx* c, cudaStream_t s, double* phi, double* F) {
  if (c->n == 0) return FMM_OK;
#define CALL(P) l2p_p<P>(c, s, phi, F)
  switch (c->order) {
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 5: return CALL(5);
    case 6: return CALL(6);
    case 7: return CALL(7);
    case 8: return CALL(8);
    case 9: return CALL(9);
    case 10: return CALL(10);
  }
#undef CALL
  return FMM_ERR_ARG;
}

fmm_status launch_m2l_simt(Ctx* c, cudaStream_t s, int first_tile, int ntiles) {
  if (ntiles <= 0) return FMM_OK;
  dim3 grid(ntiles, 2, ceil_div(c->ncoef + 1, 64));
  const Tile* tiles = c->tiles + first_tile;
  const int32_t* src = c->tile_src + (int64_t)first_tile * FMM_NT_CLASS * FMM_TILE;
  const int16_t* act = c->tile_act + (int64_t)first_tile * FMM_NT_CLASS;
  const int32_t* nact = c->tile_nact + first_tile;
  if (c->precision == FMM_MIXED)
    k_m2l_simt<float, true><<<grid, 256, 0, s>>>(tiles, src, act, nact, c->lv, c->cls_t, c->Khi, c->Klo, c->cpad,
                                                 c->ncoef, c->cpad, c->Mhi, c->Mlo, c->L32, c->box, c->kernel_s,
                                                 op_banks(c) > 1);
  else
    k_m2l_simt<double, false><<<grid, 256, 0, s>>>(tiles, src, act, nact, c->lv, c->cls_t, c->K64, nullptr,
                                                   c->ncoef, c->ncoef, c->cpad, c->M64, nullptr, c->L64,
                                                   c->box, c->kernel_s, op_banks(c) > 1);
  return cuda_err(c, cudaGetLastError(), "M2L launch");
}

fmm_status expansion_to_f64(Ctx* c, int level, int which, double* out) {
  const int64_t nrows = c->lv.ncell[level];
  if (nrows == 0) return FMM_OK;
  if (c->precision == FMM_MIXED ? !c->Mhi : !c->M64)
    return set_err(c, FMM_ERR_STATE, "fmm_get_expansion: no evaluation in the current precision on this tree");
  const int64_t row0 = c->lv.row_off[level];
  const int64_t total = nrows * c->ncoef;
  const int grid = ceil_div(total, 256);
  if (c->precision == FMM_MIXED) {
    if (which == 0)
      k_rows_to_f64<float><<<grid, 256, 0, c->stream>>>(nrows, row0, c->ncoef, c->cpad, c->Mhi, c->Mlo, 0, out);
    else
      k_rows_to_f64<float><<<grid, 256, 0, c->stream>>>(nrows, row0, c->ncoef, c->cpad, c->L32, nullptr, 1, out);
  } else {
    k_rows_to_f64<double><<<grid, 256, 0, c->stream>>>(nrows, row0, c->ncoef, c->cpad,
                                                       which == 0 ? c->M64 : c->L64, nullptr, 0, out);
  }
  return cuda_err(c, cudaGetLastError(), "expansion readout");
}

}  // namespace fmm
