// stokes.cu -- the Stokes kernel of the black-box method (Sec. 2.2 names it
// with Laplace) from four 1/r passes on one tree.
//
// The Stokeslet sums u_i = sum_k [f_k / r + d (d . f_k) / r^3], d = x_i - x_k,
// split as d (d . f) / r^3 = -grad_x(1/r) ((x . f) - (y . f)).  With phi^j,
// F^j = -grad phi^j the 1/r potentials and fields of the charges f_j
// (j = 0, 1, 2) and phi^3, F^3 those of the charges y . f:
//
//     u_i = phi^i + sum_j x_j F^j_i - F^3_i.
//
// The identity holds for any origin; positions are taken relative to the
// root cube's centre, so the products x_j F^j and the charges y . f stay of
// the size of the cube.  The host entry point (fmm_evaluate_stokes, api.cu)
// swaps the handle's charges, runs the four evaluations and restores them.
// Near pairs cancel badly in the identity (its terms are |x - o| / r times
// the result): the mixed path runs the four passes without their near field
// and adds the Stokeslet summed directly over the 27 near leaves
// (k_p2p_stokes32, nearfield.cu).
#include "common.cuh"

namespace fmm {

namespace {

constexpr int ST_THREADS = 256;

// j = 0..2: charges f_j; j = 3: (y - centre) . f; j = -1: the saved charges q0.
__global__ void __launch_bounds__(ST_THREADS)
k_stokes_charges(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ f,
                 const double* __restrict__ q0, int j, const double* __restrict__ box, double4* __restrict__ pos64,
                 float4* __restrict__ pos32) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t i = perm[r];
  double qq;
  if (j < 0) {
    qq = q0[r];
  } else if (j < 3) {
    qq = f[3 * i + j];
  } else {
    const double h = 0.5 * box[3];
    const double4 p = pos64[r];
    qq = (p.x - (box[0] + h)) * f[3 * i] + (p.y - (box[1] + h)) * f[3 * i + 1] + (p.z - (box[2] + h)) * f[3 * i + 2];
  }
  pos64[r].w = qq;
  pos32[r].w = (float)qq;
}

__global__ void __launch_bounds__(ST_THREADS)
k_stokes_save(int64_t n, const double4* __restrict__ pos64, double* __restrict__ q0) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) q0[r] = pos64[r].w;
}

// Forces in Morton order as float4 (f, 0) for the Stokeslet near field.
__global__ void __launch_bounds__(ST_THREADS)
k_stokes_forces(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ f,
                float4* __restrict__ f32) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t i = perm[r];
  f32[r] = make_float4((float)f[3 * i], (float)f[3 * i + 1], (float)f[3 * i + 2], 0.f);
}

// phi4 [4][n], F4 [4][n][3] in the caller's order; unear (may be null) the
// near field in Morton order; u [n][3].
__global__ void __launch_bounds__(ST_THREADS)
k_stokes_combine(int64_t n, const int32_t* __restrict__ perm, const double4* __restrict__ pos64,
                 const double* __restrict__ box, const double* __restrict__ phi4, const double* __restrict__ F4,
                 const float4* __restrict__ unear, double* __restrict__ u) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t i = perm[r];
  const double h = 0.5 * box[3];
  const double4 p = pos64[r];
  const double x[3] = {p.x - (box[0] + h), p.y - (box[1] + h), p.z - (box[2] + h)};
  double v[3];
  for (int c = 0; c < 3; ++c) {
    v[c] = phi4[c * n + i] - F4[(3 * n + i) * 3 + c];
    for (int j = 0; j < 3; ++j) v[c] += x[j] * F4[(j * n + i) * 3 + c];
  }
  if (unear) {
    const float4 un = unear[r];
    v[0] += un.x;
    v[1] += un.y;
    v[2] += un.z;
  }
  for (int c = 0; c < 3; ++c) u[3 * i + c] = v[c];
}

}  // namespace

fmm_status launch_stokes_save(Ctx* c, double* q0) {
  k_stokes_save<<<ceil_div(c->n, ST_THREADS), ST_THREADS, 0, c->stream>>>(c->n, c->pos64, q0);
  return cuda_err(c, cudaGetLastError(), "Stokes charge save");
}

fmm_status launch_stokes_charges(Ctx* c, const double* f, const double* q0, int j) {
  k_stokes_charges<<<ceil_div(c->n, ST_THREADS), ST_THREADS, 0, c->stream>>>(c->n, c->perm, f, q0, j, c->box,
                                                                            c->pos64, c->pos32);
  return cuda_err(c, cudaGetLastError(), "Stokes charges");
}

fmm_status launch_stokes_forces(Ctx* c, const double* f, float4* f32) {
  k_stokes_forces<<<ceil_div(c->n, ST_THREADS), ST_THREADS, 0, c->stream>>>(c->n, c->perm, f, f32);
  return cuda_err(c, cudaGetLastError(), "Stokes forces");
}

fmm_status launch_stokes_combine(Ctx* c, const double* phi4, const double* F4, const float4* unear, double* u) {
  k_stokes_combine<<<ceil_div(c->n, ST_THREADS), ST_THREADS, 0, c->stream>>>(c->n, c->perm, c->pos64, c->box, phi4,
                                                                            F4, unear, u);
  return cuda_err(c, cudaGetLastError(), "Stokes combine");
}

}  // namespace fmm
