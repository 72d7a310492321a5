// nearfield.cu -- P2P: the direct part of eq. 1 with the kernels of eq. 2 over
// the up to 27 near leaves of every leaf (Sec. 2.1.2 near field; Sec. 5's GPU
// P2P kernel does the same work per group of cells).
//
// One warp per target leaf.  The 27 neighbour ranges are looked up in the
// leaf grid by lanes 0..26 and prefix-summed with shuffles; the warp then
// streams the concatenated source list through shared memory in chunks
// (coalesced float4 / double4 loads), each lane holding one target.  A leaf
// with fewer than 16 targets gives each target g = 2, 4, ... lanes that split
// the sources and are combined with shuffles at the end, so lanes stay busy
// on sparse leaves.
//
// Mixed precision: positions are FP32 offsets from the target leaf's centre in
// leaf widths (integer shifts between neighbouring leaves), 1/r by rsqrtf,
// chunk sums in FP32 added into FP64 accumulators; results are scaled by 1/w
// (phi) and 1/w^2 (F) at the end.  Rounding a position to FP32 costs up to
// 2^-25 leaf widths, which is a large relative error for a pair much closer
// than a leaf width, and such pairs dominate the forces of their particles.
// Pairs closer than w/32 therefore take a slow path that rebuilds the
// difference exactly from the FP32 value and its FP32 rounding residual (a
// TwoSum makes the hi - hi difference exact, and the integer leaf shift then
// cancels exactly), so its error is relative to the distance itself.  The
// slow path is rare (about 5e-6 of the pairs of a uniform cloud).  A pair at
// distance 0 (the particle itself or a coincident one) contributes nothing.
#include "common.cuh"

namespace fmm {

namespace {

constexpr int P2P_WARPS = 4;
constexpr int P2P_CH = 256;
constexpr float P2P_CLOSE2 = 1.0f / 1024.0f;  // (w/32)^2 in leaf units

// a - b exactly as hi + lo (Knuth's TwoSum on a + (-b)).
__device__ inline void two_diff(float a, float b, float& hi, float& lo) {
  hi = __fsub_rn(a, b);
  const float bb = __fsub_rn(hi, a);
  lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(-b, bb));
}

// Exact-ish difference (target - source) along one axis for a close pair:
// target th + tl, source sh + sl + off (off the integer leaf shift).
__device__ inline float close_diff(float th, float tl, float sh, float sl, float off) {
  float a, e;
  two_diff(th, sh, a, e);
  return __fadd_rn(__fsub_rn(a, off), __fadd_rn(e, __fsub_rn(tl, sl)));
}

template <bool MIXED>
__global__ void __launch_bounds__(P2P_WARPS * 32)
k_p2p(LevelPtrs lv, int leaf, int nleaf, const float4* __restrict__ pos32, const float4* __restrict__ pos32lo,
      const double4* __restrict__ pos64, const double* __restrict__ box, float4* __restrict__ out32,
      double4* __restrict__ out64) {
  using V = typename std::conditional<MIXED, float4, double4>::type;
  __shared__ V src[P2P_WARPS][P2P_CH];
  __shared__ int sidx[P2P_WARPS][MIXED ? P2P_CH : 1];
  __shared__ int nb_first[P2P_WARPS][27];
  __shared__ int nb_pre[P2P_WARPS][28];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = blockIdx.x * P2P_WARPS + warp;
  if (T >= nleaf) return;
  const int tf = lv.first[leaf][T], tc = lv.count[leaf][T];
  int ix, iy, iz;
  demorton3(lv.key[leaf][T], ix, iy, iz);
  const int top = (1 << leaf) - 1;
  int nf = 0, ncnt = 0;
  if (lane < 27) {
    const int sx = ix + lane / 9 - 1, sy = iy + (lane / 3) % 3 - 1, sz = iz + lane % 3 - 1;
    if (sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top) {
      const int g = lv.grid[leaf][morton3(sx, sy, sz)];
      if (g >= 0) {
        nf = lv.first[leaf][g];
        ncnt = lv.count[leaf][g];
      }
    }
  }
  int incl = ncnt;
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane < 27) {
    nb_first[warp][lane] = nf;
    nb_pre[warp][lane] = incl - ncnt;
  }
  if (lane == 0) nb_pre[warp][27] = total;
  __syncwarp();

  for (int tb = 0; tb < tc; tb += 32) {
    const int nt = min(32, tc - tb);
    int lg = 0;
    while ((nt << (lg + 1)) <= 32) ++lg;
    const int g = 1 << lg, ti = lane >> lg, sub = lane & (g - 1);
    const bool tvalid = ti < nt;
    V xt;
    float4 tlo = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MIXED) {
      xt = tvalid ? ((const V*)pos32)[tf + tb + ti] : V{};
      if (tvalid) tlo = pos32lo[tf + tb + ti];
    } else {
      xt = tvalid ? ((const V*)pos64)[tf + tb + ti] : V{};
    }
    double aphi = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    for (int c0 = 0; c0 < total; c0 += P2P_CH) {
      const int cn = min(P2P_CH, total - c0);
      __syncwarp();
      for (int k = lane; k < cn; k += 32) {
        const int s = c0 + k;
        int lo = 0, hi = 26;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (nb_pre[warp][mid] <= s) lo = mid;
          else hi = mid - 1;
        }
        const int j = nb_first[warp][lo] + (s - nb_pre[warp][lo]);
        if (MIXED) {
          float4 pp = pos32[j];
          pp.x += (float)(lo / 9 - 1);
          pp.y += (float)((lo / 3) % 3 - 1);
          pp.z += (float)(lo % 3 - 1);
          ((float4*)&src[warp][0])[k] = pp;
          sidx[warp][MIXED ? k : 0] = j;
        } else {
          ((double4*)&src[warp][0])[k] = pos64[j];
        }
      }
      __syncwarp();
      if (MIXED) {
        float fphi = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        const float4* S = (const float4*)&src[warp][0];
        const float4 t = *(const float4*)&xt;
#pragma unroll 4
        for (int k = sub; k < cn; k += g) {
          const float4 pp = S[k];
          float dx = t.x - pp.x, dy = t.y - pp.y, dz = t.z - pp.z;
          float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (r2 < P2P_CLOSE2 && r2 > 0.f) {
            const int j = sidx[warp][MIXED ? k : 0];
            const float4 sh = pos32[j], sl = pos32lo[j];
            dx = close_diff(t.x, tlo.x, sh.x, sl.x, rintf(pp.x - sh.x));
            dy = close_diff(t.y, tlo.y, sh.y, sl.y, rintf(pp.y - sh.y));
            dz = close_diff(t.z, tlo.z, sh.z, sl.z, rintf(pp.z - sh.z));
            r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          }
          const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
          const float qi = pp.w * inv;
          const float qi3 = qi * inv * inv;
          fphi += qi;
          fx = fmaf(qi3, dx, fx);
          fy = fmaf(qi3, dy, fy);
          fz = fmaf(qi3, dz, fz);
        }
        aphi += fphi;
        ax += fx;
        ay += fy;
        az += fz;
      } else {
        const double4* S = (const double4*)&src[warp][0];
        const double4 t = *(const double4*)&xt;
        for (int k = sub; k < cn; k += g) {
          const double4 pp = S[k];
          const double dx = t.x - pp.x, dy = t.y - pp.y, dz = t.z - pp.z;
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 > 0.0) {
            const double rr = sqrt(r2);
            aphi += pp.w / rr;
            const double q3 = pp.w / (rr * r2);
            ax += q3 * dx;
            ay += q3 * dy;
            az += q3 * dz;
          }
        }
      }
    }
    for (int o = g >> 1; o > 0; o >>= 1) {
      aphi += __shfl_xor_sync(0xffffffffu, aphi, o);
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (tvalid && sub == 0) {
      if (MIXED) {
        const double s1 = 1.0 / ldexp(box[3], -leaf), s2 = s1 * s1;
        out32[tf + tb + ti] = make_float4((float)(aphi * s1), (float)(ax * s2), (float)(ay * s2), (float)(az * s2));
      } else {
        out64[tf + tb + ti] = make_double4(aphi, ax, ay, az);
      }
    }
  }
}

}  // namespace

fmm_status launch_p2p(Ctx* c, cudaStream_t s) {
  const int Lf = c->leaf, nleaf = c->lv.ncell[Lf];
  if (nleaf == 0) return FMM_OK;
  if (c->precision == FMM_MIXED)
    k_p2p<true><<<ceil_div(nleaf, P2P_WARPS), P2P_WARPS * 32, 0, s>>>(c->lv, Lf, nleaf, c->pos32, c->pos32lo,
                                                                     c->pos64, c->box, c->near32, c->near64);
  else
    k_p2p<false><<<ceil_div(nleaf, P2P_WARPS), P2P_WARPS * 32, 0, s>>>(c->lv, Lf, nleaf, c->pos32, c->pos32lo,
                                                                      c->pos64, c->box, c->near32, c->near64);
  return cuda_err(c, cudaGetLastError(), "P2P launch");
}

}  // namespace fmm
