// nearfield.cu -- P2P: the direct part of eq. 1 with the kernels of eq. 2 over
// the up to 27 near leaves of every leaf (Sec. 2.1.2 near field; Sec. 5's GPU
// P2P kernel does the same work per group of cells).
//
// One warp per work item = one batch of up to 32 targets of a leaf (leaves on
// a surface differ in occupancy by orders of magnitude, and the per-leaf work
// grows like its square, so whole leaves per warp leave a long tail of heavy
// leaves; batches keep the items within a factor of ~27 of each other and
// let the block scheduler balance them).  The 27 neighbour ranges are looked up in the
// leaf grid by lanes 0..26 and prefix-summed with shuffles; the warp then
// streams the concatenated source list through shared memory in chunks
// (coalesced loads), each lane holding one target.  A leaf with fewer than
// 16 targets gives each target g = 2, 4, ... lanes that split the sources and
// are combined with shuffles at the end, so lanes stay busy on sparse leaves.
//
// Mixed precision: positions are offsets from the particle's own leaf centre
// in leaf widths, held as FP32 hi (a multiple of 2^-23, |hi| <= 1/2) + FP32
// lo (the remainder), so a position is known to ~2^-48 leaf widths.  Every
// pair takes
//     d = (x_t,hi - x_s,hi) + (x_t,lo - x_s,lo),
// the shift of a neighbouring leaf (an integer in -1..1) being added to
// x_s,hi when the source is staged.  On the 2^-23 grid that sum and the hi
// difference (|.| <= 2) are exact, so the distance keeps full FP32 relative
// accuracy however small it is, also across leaf faces (a plain FP32
// position would carry up to 2^-25 leaf widths of error, which dominates the
// force of a particle with a very close neighbour).
// 1/r by the MUFU rsqrt approximation; per-chunk FP32 sums are added into FP32 totals with Kahan
// compensation; results are scaled by 1/w (phi) and 1/w^2 (F) at the end.
// Sources are staged with the target's own leaf first: only those can hold
// the particle itself (or a coincident one), so only they need the r > 0
// test; a pair at distance 0 contributes nothing.

#include <mutex>

#include "common.cuh"

namespace fmm {

namespace {

// FP64 kernel shape; the mixed kernel's shape (warps per block, sources per
// staged chunk) is one of the variants below, chosen per handle (fmm_autotune)
constexpr int P2P_WARPS = 4;
constexpr int P2P_CH = 256;

// 1/sqrt(x) by the MUFU approximation with denormal inputs flushed: every
// r^2 that reaches it is 0 (a pair of the target's own leaf, masked after)
// or far above FP32's normal range (positions are accurate to ~2^-46 leaf
// widths: distinct particles are at least ~2^-47 apart, r^2 >= 2^-94), so this is what rsqrtf
// computes without its range-scaling instructions for denormal inputs.
__device__ __forceinline__ float rsqrt_nf(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// rsqrt_nf of both halves of a packed pair, the results formed as a pair in
// one piece of PTX (so that they can land in the register pair the packed
// products read).
__device__ __forceinline__ unsigned long long rsqrt_nf2(unsigned long long x) {
  unsigned long long y;
  asm("{\n\t.reg .f32 a, b, c, d;\n\tmov.b64 {a, b}, %1;\n\trsqrt.approx.ftz.f32 c, a;\n\t"
      "rsqrt.approx.ftz.f32 d, b;\n\tmov.b64 %0, {c, d};\n\t}"
      : "=l"(y)
      : "l"(x));
  return y;
}

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Sums the pairs of one target with the staged sources k = k0, k0 + G, ...
// < k1 (G lanes share the target; a compile-time stride keeps the shared-
// memory addressing in immediate offsets).  SELF: the range may hold the
// target itself (r = 0 pairs are skipped).
template <int G, bool SELF>
__device__ __forceinline__ void p2p_span(const float4* __restrict__ shi, const float4* __restrict__ slo, int k0,
                                         int k1, float4 th, float4 tl, float& fphi, float& fx, float& fy,
                                         float& fz) {
#pragma unroll 4
  for (int k = k0; k < k1; k += G) {
    const float4 sh = shi[k], sl = slo[k];
    const float dx = (th.x - sh.x) + (tl.x - sl.x);
    const float dy = (th.y - sh.y) + (tl.y - sl.y);
    const float dz = (th.z - sh.z) + (tl.z - sl.z);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrt_nf(r2);
    if (SELF) inv = r2 > 0.f ? inv : 0.f;
    const float qi = sh.w * inv;
    const float qi3 = qi * inv * inv;
    fphi += qi;
    fx = fmaf(qi3, dx, fx);
    fy = fmaf(qi3, dy, fy);
    fz = fmaf(qi3, dz, fz);
  }
}

template <int G>
__device__ __forceinline__ void p2p_chunk(const float4* shi, const float4* slo, int sub, int kown, int cn,
                                          float4 th, float4 tl, float& fphi, float& fx, float& fy, float& fz) {
  p2p_span<G, true>(shi, slo, sub, kown, th, tl, fphi, fx, fy, fz);
  const int k0 = kown + ((sub - kown) % G + G) % G;
  p2p_span<G, false>(shi, slo, k0, cn, th, tl, fphi, fx, fy, fz);
}

template <int W, int CH>
__global__ void __launch_bounds__(W * 32)
k_p2p32(LevelPtrs lv, int leaf, int nleaf, const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of,
        int nitems,
        const float4* __restrict__ pos32, const float4* __restrict__ pos32lo, const double* __restrict__ box,
        float4* __restrict__ out, const int32_t* __restrict__ ilist) {
  __shared__ float4 shi[W][CH];
  __shared__ float4 slo[W][CH];
  __shared__ int nb_first[W][27];
  __shared__ int nb_pre[W][28];
  __shared__ int8_t nb_off[W][27][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * W + warp;
  if (idx >= nitems) return;
  const int item = ilist ? ilist[idx] : idx;  // ilist: the items of one bin
  const int T = leaf_of[item];  // the leaf holding this item
  const int tf = lv.first[leaf][T], tc = lv.count[leaf][T];
  const int tb = (item - items[T]) * 32;
  int ix, iy, iz;
  demorton3(lv.key[leaf][T], ix, iy, iz);
  const int top = (1 << leaf) - 1;
  const int mine = problem_of(lv, leaf, T);
  // neighbour j of lane j: lane 0 is the target leaf itself, lanes 1..26 the others
  int nf = 0, ncnt = 0, ox = 0, oy = 0, oz = 0;
  if (lane < 27) {
    const int k = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);
    ox = k / 9 - 1;
    oy = (k / 3) % 3 - 1;
    oz = k % 3 - 1;
    const int sx = ix + ox, sy = iy + oy, sz = iz + oz;
    if (sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top) {
      const int g = lv.grid[leaf][morton3(sx, sy, sz)];
      if (g >= 0 && same_problem(lv, leaf, mine, g)) {
        nf = lv.first[leaf][g];
        ncnt = lv.count[leaf][g];
      }
    }
  }
  int incl = ncnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane < 27) {
    nb_first[warp][lane] = nf;
    nb_pre[warp][lane] = incl - ncnt;
    nb_off[warp][lane][0] = (int8_t)ox;
    nb_off[warp][lane][1] = (int8_t)oy;
    nb_off[warp][lane][2] = (int8_t)oz;
  }
  if (lane == 0) nb_pre[warp][27] = total;
  __syncwarp();
  const int own = tc;  // sources [0, own) are the target leaf's particles

  {
    const int nt = min(32, tc - tb);
    int lg = 0;
    while ((nt << (lg + 1)) <= 32) ++lg;
    const int g = 1 << lg, ti = lane >> lg, sub = lane & (g - 1);
    const bool tvalid = ti < nt;
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
    if (tvalid) {
      th = pos32[tf + tb + ti];
      tl = pos32lo[tf + tb + ti];
    }
    Kahan kp, kx, ky, kz;
    for (int c0 = 0; c0 < total; c0 += CH) {
      const int cn = min(CH, total - c0);
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
        float4 ph = pos32[j];
        ph.x += (float)nb_off[warp][lo][0];
        ph.y += (float)nb_off[warp][lo][1];
        ph.z += (float)nb_off[warp][lo][2];
        shi[warp][k] = ph;
        slo[warp][k] = pos32lo[j];
      }
      __syncwarp();
      float fphi = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
      // sources [0, kown) of this chunk are the target leaf's own particles
      const int kown = min(cn, max(0, own - c0));
      const float4* sh = &shi[warp][0];
      const float4* sl = &slo[warp][0];
      switch (g) {
        case 1: p2p_chunk<1>(sh, sl, sub, kown, cn, th, tl, fphi, fx, fy, fz); break;
        case 2: p2p_chunk<2>(sh, sl, sub, kown, cn, th, tl, fphi, fx, fy, fz); break;
        case 4: p2p_chunk<4>(sh, sl, sub, kown, cn, th, tl, fphi, fx, fy, fz); break;
        case 8: p2p_chunk<8>(sh, sl, sub, kown, cn, th, tl, fphi, fx, fy, fz); break;
        case 16: p2p_chunk<16>(sh, sl, sub, kown, cn, th, tl, fphi, fx, fy, fz); break;
        default: p2p_chunk<32>(sh, sl, sub, kown, cn, th, tl, fphi, fx, fy, fz); break;
      }
      kp.add(fphi);
      kx.add(fx);
      ky.add(fy);
      kz.add(fz);
    }
    float aphi = kp.s, ax = kx.s, ay = ky.s, az = kz.s;
    for (int o = g >> 1; o > 0; o >>= 1) {
      aphi += __shfl_xor_sync(0xffffffffu, aphi, o);
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (tvalid && sub == 0) {
      const float s1 = (float)(1.0 / ldexp(box[3], -leaf)), s2 = s1 * s1;
      out[tf + tb + ti] = make_float4(aphi * s1, ax * s2, ay * s2, az * s2);
    }
  }
}

// ---- packed-pair variant --------------------------------------------------
// The same sums with two sources per instruction: sm_100-class SMs execute
// FP32 add / mul / fma on register pairs (add/sub/mul/fma.rn.f32x2), one
// issue slot for two operations.  The near-field loop is issue-bound (one
// interaction is 19 FP32 operations, a reciprocal square root and shared
// loads), so halving its FP32 issue count lets the FP32 pipe, not the issue
// port, set the pace.  Sources are staged as pairs in a structure-of-pairs
// layout: for pair j (sources 2j, 2j+1) the words (x0,x1 | y0,y1),
// (z0,z1 | q0,q1), (xl0,xl1 | yl0,yl1), (zl0,zl1), so every operand is a
// register pair loaded by one 128- or 64-bit shared load.  An odd chunk is
// padded with a zero charge 64 leaf widths away.  The arithmetic of each
// pair is that of p2p_span: d = (hi_t - hi_s) + (lo_t - lo_s) per component.

typedef unsigned long long f2_t;  // two FP32 values (low word = first)

__device__ __forceinline__ f2_t f2pack(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 f2unpack(f2_t r) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
  return make_float2(a, b);
}
__device__ __forceinline__ f2_t f2add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct PairAcc {
  f2_t phi, fx, fy, fz;
};

// General kernels (GEN, fmm_set_kernel): e = r^2 + c^2 in leaf widths,
// phi += q e^(-s/2) = q 2^(-s/2 log2 e), F += s q d / e (three MUFU
// operations per source, the rest in pairs).
struct GenK {
  float hs;         // s / 2
  f2_t sk, cw2;     // (s, s), (c^2, c^2) in leaf widths
};

template <int G, bool SELF, int U, bool GEN>
__device__ __forceinline__ void p2p_pairs(const ulonglong2* __restrict__ sA, const ulonglong2* __restrict__ sB,
                                          const ulonglong2* __restrict__ sC, const f2_t* __restrict__ sD, int j0,
                                          int j1, f2_t TX, f2_t TY, f2_t TZ, f2_t LX, f2_t LY, f2_t LZ,
                                          const GenK& gk, PairAcc& acc) {
#pragma unroll U
  for (int j = j0; j < j1; j += G) {
    const ulonglong2 a = sA[j], b = sB[j], c = sC[j];
    const f2_t dlz = sD[j];
    const f2_t dx = f2add(f2sub(TX, a.x), f2sub(LX, c.x));
    const f2_t dy = f2add(f2sub(TY, a.y), f2sub(LY, c.y));
    const f2_t dz = f2add(f2sub(TZ, b.x), f2sub(LZ, dlz));
    const f2_t r2 = f2fma(dx, dx, f2fma(dy, dy, f2mul(dz, dz)));
    const float2 rr = f2unpack(r2);
    f2_t qi, qi3;
    if (GEN) {
      const float2 ee = f2unpack(f2add(r2, gk.cw2));
      float p0 = exp2f(-gk.hs * __log2f(ee.x)), p1 = exp2f(-gk.hs * __log2f(ee.y));
      float e0 = __fdividef(1.f, ee.x), e1 = __fdividef(1.f, ee.y);
      if (SELF) {  // pairs at distance 0 contribute nothing, also when c > 0
        p0 = rr.x > 0.f ? p0 : 0.f;
        p1 = rr.y > 0.f ? p1 : 0.f;
        e0 = rr.x > 0.f ? e0 : 0.f;
        e1 = rr.y > 0.f ? e1 : 0.f;
      }
      qi = f2mul(b.y, f2pack(p0, p1));
      qi3 = f2mul(f2mul(qi, gk.sk), f2pack(e0, e1));
    } else {
      f2_t inv;
      if (SELF) {
        float i0 = rsqrt_nf(rr.x), i1 = rsqrt_nf(rr.y);
        i0 = rr.x > 0.f ? i0 : 0.f;
        i1 = rr.y > 0.f ? i1 : 0.f;
        inv = f2pack(i0, i1);
      } else {
        inv = rsqrt_nf2(r2);
      }
      qi = f2mul(b.y, inv);
      qi3 = f2mul(f2mul(qi, inv), inv);
    }
    acc.phi = f2add(acc.phi, qi);
    acc.fx = f2fma(qi3, dx, acc.fx);
    acc.fy = f2fma(qi3, dy, acc.fy);
    acc.fz = f2fma(qi3, dz, acc.fz);
  }
}

template <int G, int U, bool GEN = false>
__device__ __forceinline__ void p2p_pair_chunk(const ulonglong2* sA, const ulonglong2* sB, const ulonglong2* sC,
                                               const f2_t* sD, int sub, int jown, int np, f2_t TX, f2_t TY, f2_t TZ,
                                               f2_t LX, f2_t LY, f2_t LZ, PairAcc& acc, const GenK& gk = GenK{}) {
  p2p_pairs<G, true, 1, GEN>(sA, sB, sC, sD, sub, jown, TX, TY, TZ, LX, LY, LZ, gk, acc);
  const int j0 = jown + ((sub - jown) % G + G) % G;
  p2p_pairs<G, false, U, GEN>(sA, sB, sC, sD, j0, np, TX, TY, TZ, LX, LY, LZ, gk, acc);
}

// One work item (32 targets of one leaf against its up to 27 near leaves) of
// the packed-pair near field, by one warp, with the warp's own staging
// arrays (sA..sD of CH / 2 pairs, the neighbour tables).  GEN: the kernels of
// fmm_set_kernel other than 1/r (ks, kc); outputs scaled by w^-s and
// w^-(s+1).
template <int CH, int U, bool GEN>
__device__ __forceinline__ void p2p32x2_item(int item, const LevelPtrs& lv, int leaf,
                                             const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of,
                                             const float4* __restrict__ pos32, const float4* __restrict__ pos32lo,
                                             const double* __restrict__ box, float4* __restrict__ out, double ks,
                                             double kc, ulonglong2* sA, ulonglong2* sB, ulonglong2* sC, f2_t* sD,
                                             int* nb_first, int* nb_pre, int8_t (*nb_off)[3]) {
  const int lane = threadIdx.x & 31;
  const int T = leaf_of[item];  // the leaf holding this item
  const int tf = lv.first[leaf][T], tc = lv.count[leaf][T];
  const int tb = (item - items[T]) * 32;
  int ix, iy, iz;
  demorton3(lv.key[leaf][T], ix, iy, iz);
  const int top = (1 << leaf) - 1;
  const int mine = problem_of(lv, leaf, T);
  int nf = 0, ncnt = 0, ox = 0, oy = 0, oz = 0;
  if (lane < 27) {
    const int k = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);
    ox = k / 9 - 1;
    oy = (k / 3) % 3 - 1;
    oz = k % 3 - 1;
    const int sx = ix + ox, sy = iy + oy, sz = iz + oz;
    if (sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top) {
      const int g = lv.grid[leaf][morton3(sx, sy, sz)];
      if (g >= 0 && same_problem(lv, leaf, mine, g)) {
        nf = lv.first[leaf][g];
        ncnt = lv.count[leaf][g];
      }
    }
  }
  int incl = ncnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();  // the previous item's readers are done with the tables
  if (lane < 27) {
    nb_first[lane] = nf;
    nb_pre[lane] = incl - ncnt;
    nb_off[lane][0] = (int8_t)ox;
    nb_off[lane][1] = (int8_t)oy;
    nb_off[lane][2] = (int8_t)oz;
  }
  if (lane == 0) nb_pre[27] = total;
  __syncwarp();
  const int own = tc;  // sources [0, own) are the target leaf's particles

  const int nt = min(32, tc - tb);
  int lg = 0;
  while ((nt << (lg + 1)) <= 32) ++lg;
  const int g = 1 << lg, ti = lane >> lg, sub = lane & (g - 1);
  const bool tvalid = ti < nt;
  float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
  if (tvalid) {
    th = pos32[tf + tb + ti];
    tl = pos32lo[tf + tb + ti];
  }
  const f2_t TX = f2pack(th.x, th.x), TY = f2pack(th.y, th.y), TZ = f2pack(th.z, th.z);
  const f2_t LX = f2pack(tl.x, tl.x), LY = f2pack(tl.y, tl.y), LZ = f2pack(tl.z, tl.z);
  GenK gk{};
  if (GEN) {
    const double ckw = kc / ldexp(box[3], -leaf);  // c in leaf widths
    gk.hs = (float)(0.5 * ks);
    gk.sk = f2pack((float)ks, (float)ks);
    gk.cw2 = f2pack((float)(ckw * ckw), (float)(ckw * ckw));
  }
  Kahan kp, kx, ky, kz;
  // staged source s of the chunk starting at c0: position (hi with the
  // neighbour shift, lo) and charge
  // the neighbour leaf holding staged source s: the last lo with nb_pre[lo] <= s;
  // a thread's s only grows (its pairs within a chunk, then later chunks), so
  // its cursor moves forward from the previous answer
  int lo = 0;
  auto fetch = [&](int s, float4& ph, float4& pl) {
    while (lo < 26 && nb_pre[lo + 1] <= s) ++lo;
    if (!FMM_GUARD(s >= nb_pre[lo] && s < nb_pre[lo + 1], CHK_P2P_SOURCE, s)) {
      ph = make_float4(64.f, 64.f, 64.f, 0.f);  // skipped: no charge, far from every target
      pl = make_float4(0.f, 0.f, 0.f, 0.f);
      return;
    }
    const int j = nb_first[lo] + (s - nb_pre[lo]);
    ph = pos32[j];
    ph.x += (float)nb_off[lo][0];
    ph.y += (float)nb_off[lo][1];
    ph.z += (float)nb_off[lo][2];
    pl = pos32lo[j];
  };
  for (int c0 = 0; c0 < total; c0 += CH) {
    const int cn = min(CH, total - c0);
    const int np = (cn + 1) >> 1;
    __syncwarp();
    for (int m = lane; m < np; m += 32) {
      float4 h0, l0, h1, l1;
      fetch(c0 + 2 * m, h0, l0);
      if (2 * m + 1 < cn) {
        fetch(c0 + 2 * m + 1, h1, l1);
      } else {  // padding: no charge, far from every target
        h1 = make_float4(64.f, 64.f, 64.f, 0.f);
        l1 = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      sA[m] = make_ulonglong2(f2pack(h0.x, h1.x), f2pack(h0.y, h1.y));
      sB[m] = make_ulonglong2(f2pack(h0.z, h1.z), f2pack(h0.w, h1.w));
      sC[m] = make_ulonglong2(f2pack(l0.x, l1.x), f2pack(l0.y, l1.y));
      sD[m] = f2pack(l0.z, l1.z);
    }
    __syncwarp();
    PairAcc acc{0ull, 0ull, 0ull, 0ull};
    // pairs [0, jown) may hold the target's own leaf (r = 0 pairs skipped)
    const int kown = min(cn, max(0, own - c0));
    const int jown = (kown + 1) >> 1;
    switch (g) {
      case 1: p2p_pair_chunk<1, U, GEN>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc, gk); break;
      case 2: p2p_pair_chunk<2, U, GEN>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc, gk); break;
      case 4: p2p_pair_chunk<4, U, GEN>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc, gk); break;
      case 8: p2p_pair_chunk<8, U, GEN>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc, gk); break;
      case 16: p2p_pair_chunk<16, U, GEN>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc, gk); break;
      default: p2p_pair_chunk<32, U, GEN>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc, gk); break;
    }
    const float2 ph = f2unpack(acc.phi), px = f2unpack(acc.fx), py = f2unpack(acc.fy), pz = f2unpack(acc.fz);
    kp.add(ph.x + ph.y);
    kx.add(px.x + px.y);
    ky.add(py.x + py.y);
    kz.add(pz.x + pz.y);
  }
  float aphi = kp.s, ax = kx.s, ay = ky.s, az = kz.s;
  for (int o = g >> 1; o > 0; o >>= 1) {
    aphi += __shfl_xor_sync(0xffffffffu, aphi, o);
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
  if (tvalid && sub == 0) {
    const double iw = 1.0 / ldexp(box[3], -leaf);
    const float s1 = GEN ? (float)pow(iw, ks) : (float)iw;
    const float s2 = GEN ? (float)(pow(iw, ks) * iw) : s1 * s1;
    out[tf + tb + ti] = make_float4(aphi * s1, ax * s2, ay * s2, az * s2);
  }
}

// One warp per work item, W warps per block.
template <int W, int CH, int U, bool GEN = false>
__global__ void __launch_bounds__(W * 32)
k_p2p32x2(LevelPtrs lv, int leaf, int nleaf, const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of,
          int nitems,
          const float4* __restrict__ pos32, const float4* __restrict__ pos32lo, const double* __restrict__ box,
          float4* __restrict__ out, const int32_t* __restrict__ ilist = nullptr, double ks = 1.0, double kc = 0.0) {
  constexpr int NP = CH / 2;
  __shared__ ulonglong2 sA[W][NP];
  __shared__ ulonglong2 sB[W][NP];
  __shared__ ulonglong2 sC[W][NP];
  __shared__ f2_t sD[W][NP];
  __shared__ int nb_first[W][27];
  __shared__ int nb_pre[W][28];
  __shared__ int8_t nb_off[W][27][3];
  const int warp = threadIdx.x >> 5;
  const int idx = blockIdx.x * W + warp;
  if (idx >= nitems) return;
  const int item = ilist ? ilist[idx] : idx;  // ilist: the items of one bin
  p2p32x2_item<CH, U, GEN>(item, lv, leaf, items, leaf_of, pos32, pos32lo, box, out, ks, kc, sA[warp], sB[warp],
                           sC[warp], sD[warp], nb_first[warp], nb_pre[warp], nb_off[warp]);
}

// Persistent warps: every warp takes the next work item (of ilist, if
// given) from a counter (items in leaf order, so warps running at the same
// time read neighbouring leaves) until none is left, so no warp slot waits for the slowest warp of
// its block and no wave of blocks leaves SMs idle at the end.  *counter is
// zero at launch.
template <int W, int CH, int U>
__global__ void __launch_bounds__(W * 32)
k_p2p32x2p(LevelPtrs lv, int leaf, const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of, int nitems,
           const float4* __restrict__ pos32, const float4* __restrict__ pos32lo, const double* __restrict__ box,
           float4* __restrict__ out, int32_t* __restrict__ counter, const int32_t* __restrict__ ilist) {
  constexpr int NP = CH / 2;
  __shared__ ulonglong2 sA[W][NP];
  __shared__ ulonglong2 sB[W][NP];
  __shared__ ulonglong2 sC[W][NP];
  __shared__ f2_t sD[W][NP];
  __shared__ int nb_first[W][27];
  __shared__ int nb_pre[W][28];
  __shared__ int8_t nb_off[W][27][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(counter, 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= nitems) return;
    const int item = ilist ? ilist[idx] : idx;  // ilist: the items of one bin
    p2p32x2_item<CH, U, false>(item, lv, leaf, items, leaf_of, pos32, pos32lo, box, out, 1.0, 0.0, sA[warp],
                               sB[warp], sC[warp], sD[warp], nb_first[warp], nb_pre[warp], nb_off[warp]);
  }
}

// Leaf-cooperative packed kernel, for leaves of many particles: a block of
// 8 warps takes a unit of up to 8 consecutive work items of one leaf (their
// targets share the 27-leaf source list), stages each chunk of sources once
// for all of them, and every warp sums its own 32 targets against it.  A
// leaf's sources are staged once per unit instead of once per item.
constexpr int CW = 8;  // warps per block = items per unit

// Double-buffered: chunk c + 1 is staged (into the other buffer, in dynamic
// shared memory: 2 x CH / 2 pairs x 56 bytes) while chunk c is summed, with
// one block barrier per chunk.
template <int CH>
constexpr int coop_smem_bytes() {
  return 2 * (CH / 2) * (3 * (int)sizeof(ulonglong2) + (int)sizeof(f2_t));
}

template <int CH, int U>
__global__ void __launch_bounds__(CW * 32)
k_p2p32x2c(LevelPtrs lv, int leaf, const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of,
           const int32_t* __restrict__ units, int nunits, const float4* __restrict__ pos32,
           const float4* __restrict__ pos32lo, const double* __restrict__ box, float4* __restrict__ out) {
  constexpr int NP = CH / 2;
  extern __shared__ __align__(16) unsigned char coop_smem[];
  ulonglong2* const bA = (ulonglong2*)coop_smem;  // [2][NP] each
  ulonglong2* const bB = bA + 2 * NP;
  ulonglong2* const bC = bB + 2 * NP;
  f2_t* const bD = (f2_t*)(bC + 2 * NP);
  __shared__ int nb_first[27];
  __shared__ int nb_pre[28];
  __shared__ int8_t nb_off[27][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  if ((int)blockIdx.x >= nunits) return;
  const int item0 = units[blockIdx.x];
  const int T = leaf_of[item0];
  const int tf = lv.first[leaf][T], tc = lv.count[leaf][T];
  const int nit = (tc + 31) >> 5;                        // the leaf's items
  const int item = item0 + warp;
  const bool active = item - items[T] < nit;             // this warp has an item
  const int tb = (item - items[T]) * 32;
  if (warp == 0) {
    int ix, iy, iz;
    demorton3(lv.key[leaf][T], ix, iy, iz);
    const int top = (1 << leaf) - 1;
    const int mine = problem_of(lv, leaf, T);
    int nf = 0, ncnt = 0, ox = 0, oy = 0, oz = 0;
    if (lane < 27) {
      const int k = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);
      ox = k / 9 - 1;
      oy = (k / 3) % 3 - 1;
      oz = k % 3 - 1;
      const int sx = ix + ox, sy = iy + oy, sz = iz + oz;
      if (sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top) {
        const int g = lv.grid[leaf][morton3(sx, sy, sz)];
        if (g >= 0 && same_problem(lv, leaf, mine, g)) {
          nf = lv.first[leaf][g];
          ncnt = lv.count[leaf][g];
        }
      }
    }
    int incl = ncnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane < 27) {
      nb_first[lane] = nf;
      nb_pre[lane] = incl - ncnt;
      nb_off[lane][0] = (int8_t)ox;
      nb_off[lane][1] = (int8_t)oy;
      nb_off[lane][2] = (int8_t)oz;
    }
    if (lane == 31) nb_pre[27] = incl;
  }
  __syncthreads();
  const int total = nb_pre[27];
  const int own = tc;
  const int nt = active ? min(32, tc - tb) : 1;
  int lg = 0;
  while ((nt << (lg + 1)) <= 32) ++lg;
  const int g = 1 << lg, ti = lane >> lg, sub = lane & (g - 1);
  const bool tvalid = active && ti < nt;
  float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
  if (tvalid) {
    th = pos32[tf + tb + ti];
    tl = pos32lo[tf + tb + ti];
  }
  const f2_t TX = f2pack(th.x, th.x), TY = f2pack(th.y, th.y), TZ = f2pack(th.z, th.z);
  const f2_t LX = f2pack(tl.x, tl.x), LY = f2pack(tl.y, tl.y), LZ = f2pack(tl.z, tl.z);
  Kahan kp, kx, ky, kz;
  // the neighbour leaf holding staged source s: the last lo with nb_pre[lo] <= s;
  // a thread's s only grows (its pairs within a chunk, then later chunks), so
  // its cursor moves forward from the previous answer
  int lo = 0;
  auto fetch = [&](int s, float4& ph, float4& pl) {
    while (lo < 26 && nb_pre[lo + 1] <= s) ++lo;
    if (!FMM_GUARD(s >= nb_pre[lo] && s < nb_pre[lo + 1], CHK_P2P_SOURCE, s)) {
      ph = make_float4(64.f, 64.f, 64.f, 0.f);  // skipped: no charge, far from every target
      pl = make_float4(0.f, 0.f, 0.f, 0.f);
      return;
    }
    const int j = nb_first[lo] + (s - nb_pre[lo]);
    ph = pos32[j];
    ph.x += (float)nb_off[lo][0];
    ph.y += (float)nb_off[lo][1];
    ph.z += (float)nb_off[lo][2];
    pl = pos32lo[j];
  };
  // stage the chunk starting at c0 into buffer b
  auto stage = [&](int c0, int b) {
    const int cn = min(CH, total - c0);
    const int np = (cn + 1) >> 1;
    ulonglong2 *sA = bA + b * NP, *sB = bB + b * NP, *sC = bC + b * NP;
    f2_t* sD = bD + b * NP;
    for (int m = tid; m < np; m += CW * 32) {
      float4 h0, l0, h1, l1;
      fetch(c0 + 2 * m, h0, l0);
      if (2 * m + 1 < cn) {
        fetch(c0 + 2 * m + 1, h1, l1);
      } else {  // padding: no charge, far from every target
        h1 = make_float4(64.f, 64.f, 64.f, 0.f);
        l1 = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      sA[m] = make_ulonglong2(f2pack(h0.x, h1.x), f2pack(h0.y, h1.y));
      sB[m] = make_ulonglong2(f2pack(h0.z, h1.z), f2pack(h0.w, h1.w));
      sC[m] = make_ulonglong2(f2pack(l0.x, l1.x), f2pack(l0.y, l1.y));
      sD[m] = f2pack(l0.z, l1.z);
    }
  };
  if (total > 0) stage(0, 0);
  __syncthreads();
  for (int c0 = 0, b = 0; c0 < total; c0 += CH, b ^= 1) {
    const int cn = min(CH, total - c0);
    const int np = (cn + 1) >> 1;
    // the other buffer's last readers passed the barrier that ended the previous chunk
    if (c0 + CH < total) stage(c0 + CH, b ^ 1);
    const ulonglong2 *sA = bA + b * NP, *sB = bB + b * NP, *sC = bC + b * NP;
    const f2_t* sD = bD + b * NP;
    if (active) {
      PairAcc acc{0ull, 0ull, 0ull, 0ull};
      const int kown = min(cn, max(0, own - c0));
      const int jown = (kown + 1) >> 1;
      switch (g) {
        case 1: p2p_pair_chunk<1, U>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc); break;
        case 2: p2p_pair_chunk<2, U>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc); break;
        case 4: p2p_pair_chunk<4, U>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc); break;
        case 8: p2p_pair_chunk<8, U>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc); break;
        case 16: p2p_pair_chunk<16, U>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc); break;
        default: p2p_pair_chunk<32, U>(sA, sB, sC, sD, sub, jown, np, TX, TY, TZ, LX, LY, LZ, acc); break;
      }
      const float2 ph = f2unpack(acc.phi), px = f2unpack(acc.fx), py = f2unpack(acc.fy), pz = f2unpack(acc.fz);
      kp.add(ph.x + ph.y);
      kx.add(px.x + px.y);
      ky.add(py.x + py.y);
      kz.add(pz.x + pz.y);
    }
    __syncthreads();  // the next chunk is staged; this one is no longer read
  }
  if (!active) return;
  float aphi = kp.s, ax = kx.s, ay = ky.s, az = kz.s;
  for (int o = g >> 1; o > 0; o >>= 1) {
    aphi += __shfl_xor_sync(0xffffffffu, aphi, o);
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
  if (tvalid && sub == 0) {
    const float s1 = (float)(1.0 / ldexp(box[3], -leaf)), s2 = s1 * s1;
    out[tf + tb + ti] = make_float4(aphi * s1, ax * s2, ay * s2, az * s2);
  }
}

// ---- the Stokeslet near field (fmm_evaluate_stokes, mixed precision) ------
// Work items, staging and exact hi/lo differences of k_p2p32, with each
// source's force staged beside its position: per pair u += f / r +
// d (d . f) / r^3 directly, in leaf widths (u scales by 1/w).  The four 1/r
// passes that give the far field would give the near field only as a
// difference of terms |x - o| / r times larger than it, which FP32 cannot
// carry for close pairs.
template <int G, bool SELF>
__device__ __forceinline__ void p2p_span_stokes(const float4* __restrict__ shi, const float4* __restrict__ slo,
                                                const float4* __restrict__ sfo, int k0, int k1, float4 th, float4 tl,
                                                float& ux, float& uy, float& uz) {
#pragma unroll 4
  for (int k = k0; k < k1; k += G) {
    const float4 sh = shi[k], sl = slo[k], sf = sfo[k];
    const float dx = (th.x - sh.x) + (tl.x - sl.x);
    const float dy = (th.y - sh.y) + (tl.y - sl.y);
    const float dz = (th.z - sh.z) + (tl.z - sl.z);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrt_nf(r2);
    if (SELF) inv = r2 > 0.f ? inv : 0.f;
    const float t = fmaf(dx, sf.x, fmaf(dy, sf.y, dz * sf.z)) * (inv * inv * inv);
    ux = fmaf(sf.x, inv, fmaf(dx, t, ux));
    uy = fmaf(sf.y, inv, fmaf(dy, t, uy));
    uz = fmaf(sf.z, inv, fmaf(dz, t, uz));
  }
}

template <int W, int CH>
__global__ void __launch_bounds__(W * 32)
k_p2p_stokes32(LevelPtrs lv, int leaf, const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of,
               int nitems, const float4* __restrict__ pos32, const float4* __restrict__ pos32lo,
               const float4* __restrict__ f32, const double* __restrict__ box, float4* __restrict__ out) {
  __shared__ float4 shi[W][CH];
  __shared__ float4 slo[W][CH];
  __shared__ float4 sfo[W][CH];
  __shared__ int nb_first[W][27];
  __shared__ int nb_pre[W][28];
  __shared__ int8_t nb_off[W][27][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * W + warp;
  if (item >= nitems) return;
  const int T = leaf_of[item];
  const int tf = lv.first[leaf][T], tc = lv.count[leaf][T];
  const int tb = (item - items[T]) * 32;
  int ix, iy, iz;
  demorton3(lv.key[leaf][T], ix, iy, iz);
  const int top = (1 << leaf) - 1;
  const int mine = problem_of(lv, leaf, T);
  int nf = 0, ncnt = 0, ox = 0, oy = 0, oz = 0;
  if (lane < 27) {
    const int k = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);
    ox = k / 9 - 1;
    oy = (k / 3) % 3 - 1;
    oz = k % 3 - 1;
    const int sx = ix + ox, sy = iy + oy, sz = iz + oz;
    if (sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top) {
      const int g = lv.grid[leaf][morton3(sx, sy, sz)];
      if (g >= 0 && same_problem(lv, leaf, mine, g)) {
        nf = lv.first[leaf][g];
        ncnt = lv.count[leaf][g];
      }
    }
  }
  int incl = ncnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane < 27) {
    nb_first[warp][lane] = nf;
    nb_pre[warp][lane] = incl - ncnt;
    nb_off[warp][lane][0] = (int8_t)ox;
    nb_off[warp][lane][1] = (int8_t)oy;
    nb_off[warp][lane][2] = (int8_t)oz;
  }
  if (lane == 0) nb_pre[warp][27] = total;
  __syncwarp();
  const int own = tc;
  const int nt = min(32, tc - tb);
  int lg = 0;
  while ((nt << (lg + 1)) <= 32) ++lg;
  const int g = 1 << lg, ti = lane >> lg, sub = lane & (g - 1);
  const bool tvalid = ti < nt;
  float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
  if (tvalid) {
    th = pos32[tf + tb + ti];
    tl = pos32lo[tf + tb + ti];
  }
  Kahan kx, ky, kz;
  for (int c0 = 0; c0 < total; c0 += CH) {
    const int cn = min(CH, total - c0);
    __syncwarp();
    for (int k = lane; k < cn; k += 32) {
      const int sidx = c0 + k;
      int lo = 0, hi = 26;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nb_pre[warp][mid] <= sidx) lo = mid;
        else hi = mid - 1;
      }
      const int j = nb_first[warp][lo] + (sidx - nb_pre[warp][lo]);
      float4 ph = pos32[j];
      ph.x += (float)nb_off[warp][lo][0];
      ph.y += (float)nb_off[warp][lo][1];
      ph.z += (float)nb_off[warp][lo][2];
      shi[warp][k] = ph;
      slo[warp][k] = pos32lo[j];
      sfo[warp][k] = f32[j];
    }
    __syncwarp();
    float ux = 0.f, uy = 0.f, uz = 0.f;
    const int kown = min(cn, max(0, own - c0));
    const float4* sh = &shi[warp][0];
    const float4* sl = &slo[warp][0];
    const float4* sf = &sfo[warp][0];
    switch (g) {
#define SPAN_ST(G)                                                                                \
  case G: {                                                                                       \
    p2p_span_stokes<G, true>(sh, sl, sf, sub, kown, th, tl, ux, uy, uz);                          \
    const int k0 = kown + ((sub - kown) % G + G) % G;                                             \
    p2p_span_stokes<G, false>(sh, sl, sf, k0, cn, th, tl, ux, uy, uz);                            \
  } break;
      SPAN_ST(1) SPAN_ST(2) SPAN_ST(4) SPAN_ST(8) SPAN_ST(16) SPAN_ST(32)
#undef SPAN_ST
    }
    kx.add(ux);
    ky.add(uy);
    kz.add(uz);
  }
  float ax = kx.s, ay = ky.s, az = kz.s;
  for (int o = g >> 1; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
  if (tvalid && sub == 0) {
    const float iw = (float)(1.0 / ldexp(box[3], -leaf));
    out[tf + tb + ti] = make_float4(ax * iw, ay * iw, az * iw, 0.f);
  }
}

// FP64: positions as given, exact skip of r = 0.
__global__ void __launch_bounds__(P2P_WARPS * 32)
k_p2p64(LevelPtrs lv, int leaf, int nleaf, const int32_t* __restrict__ items, const int32_t* __restrict__ leaf_of,
        int nitems,
        const double4* __restrict__ pos64, double ks, double kc2, double4* __restrict__ out) {
  __shared__ double4 src[P2P_WARPS][P2P_CH];
  __shared__ int nb_first[P2P_WARPS][27];
  __shared__ int nb_pre[P2P_WARPS][28];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * P2P_WARPS + warp;
  if (item >= nitems) return;
  const int T = leaf_of[item];  // the leaf holding this item
  const int tf = lv.first[leaf][T], tc = lv.count[leaf][T];
  const int tb = (item - items[T]) * 32;
  int ix, iy, iz;
  demorton3(lv.key[leaf][T], ix, iy, iz);
  const int top = (1 << leaf) - 1;
  const int mine = problem_of(lv, leaf, T);
  int nf = 0, ncnt = 0;
  if (lane < 27) {
    const int sx = ix + lane / 9 - 1, sy = iy + (lane / 3) % 3 - 1, sz = iz + lane % 3 - 1;
    if (sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top) {
      const int g = lv.grid[leaf][morton3(sx, sy, sz)];
      if (g >= 0 && same_problem(lv, leaf, mine, g)) {
        nf = lv.first[leaf][g];
        ncnt = lv.count[leaf][g];
      }
    }
  }
  int incl = ncnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane < 27) {
    nb_first[warp][lane] = nf;
    nb_pre[warp][lane] = incl - ncnt;
  }
  if (lane == 0) nb_pre[warp][27] = total;
  __syncwarp();
  {
    const int nt = min(32, tc - tb);
    int lg = 0;
    while ((nt << (lg + 1)) <= 32) ++lg;
    const int g = 1 << lg, ti = lane >> lg, sub = lane & (g - 1);
    const bool tvalid = ti < nt;
    const double4 t = tvalid ? pos64[tf + tb + ti] : make_double4(0, 0, 0, 0);
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
        src[warp][k] = pos64[nb_first[warp][lo] + (s - nb_pre[warp][lo])];
      }
      __syncwarp();
      for (int k = sub; k < cn; k += g) {
        const double4 pp = src[warp][k];
        const double dx = t.x - pp.x, dy = t.y - pp.y, dz = t.z - pp.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > 0.0) {
          double q1, q3;
          if (ks == 1.0 && kc2 == 0.0) {
            const double rr = sqrt(r2);
            q1 = pp.w / rr;
            q3 = pp.w / (rr * r2);
          } else {  // e = r^2 + c^2: phi += q e^(-s/2), F += s q d e^(-(s+2)/2)
            const double e = r2 + kc2;
            q1 = pp.w * pow(e, -0.5 * ks);
            q3 = ks * q1 / e;
          }
          aphi += q1;
          ax += q3 * dx;
          ay += q3 * dy;
          az += q3 * dz;
        }
      }
    }
    for (int o = g >> 1; o > 0; o >>= 1) {
      aphi += __shfl_xor_sync(0xffffffffu, aphi, o);
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (tvalid && sub == 0) out[tf + tb + ti] = make_double4(aphi, ax, ay, az);
  }
}

}  // namespace

// (warps per block, sources per staged chunk) of the mixed P2P variants, in
// the order of fmm_autotune's index
// variants 6.. are the packed-pair kernel (k_p2p32x2) in the same shapes
// (warps, chunk, sources per instruction, unroll of the pair loop); index 0
// is the default (the packed kernel, fastest on every workload measured)
// 12, 13: the leaf-cooperative packed kernel (8 warps share each staged chunk)
const int kP2PVariants[FMM_P2P_VARIANTS][4] = {{8, 128, 2, 4}, {4, 128, 2, 4}, {4, 256, 2, 2}, {4, 128, 2, 2},
                                               {8, 128, 2, 2}, {8, 256, 2, 2}, {4, 256, 1, 4}, {2, 128, 1, 4},
                                               {2, 256, 1, 4}, {4, 128, 1, 4}, {8, 128, 1, 4}, {8, 256, 1, 4},
                                               {8, 512, 2, 4}, {8, 1024, 2, 4}, {4, 128, 2, 4}, {4, 256, 2, 2}};

// Whether a kernel is one of the P2P kernels (graph nodes of the near field
// get the low launch priority, see build_graph).
bool is_p2p_kernel(const void* f) {
  const void* ks[] = {(const void*)k_p2p32<4, 256>,      (const void*)k_p2p32<2, 128>,
                      (const void*)k_p2p32<2, 256>,      (const void*)k_p2p32<4, 128>,
                      (const void*)k_p2p32<8, 128>,      (const void*)k_p2p32<8, 256>,
                      (const void*)k_p2p32x2<8, 128, 4>, (const void*)k_p2p32x2<4, 128, 4>,
                      (const void*)k_p2p32x2<4, 256, 2>, (const void*)k_p2p32x2<4, 128, 2>,
                      (const void*)k_p2p32x2<8, 128, 2>, (const void*)k_p2p32x2<8, 256, 2>,
                      (const void*)k_p2p32x2c<512, 4>,   (const void*)k_p2p32x2c<1024, 4>,
                      (const void*)k_p2p32x2p<4, 128, 4>, (const void*)k_p2p32x2p<4, 256, 2>,
                      (const void*)k_p2p32x2<8, 128, 4, true>, (const void*)k_p2p_stokes32<4, 128>,
                      (const void*)k_p2p64};
  for (const void* k : ks)
    if (k == f) return true;
  return false;
}

// The P2P kernels prefer the largest shared-memory carveout, so that their
// blocks can join an SM configured for a persistent tensor-core M2L CTA.
void p2p_carveout() {
  static std::once_flag once;
  std::call_once(once, [] {
    const void* ks[] = {(const void*)k_p2p32<4, 256>,      (const void*)k_p2p32<2, 128>,
                        (const void*)k_p2p32<2, 256>,      (const void*)k_p2p32<4, 128>,
                        (const void*)k_p2p32<8, 128>,      (const void*)k_p2p32<8, 256>,
                        (const void*)k_p2p32x2<8, 128, 4>, (const void*)k_p2p32x2<4, 128, 4>,
                        (const void*)k_p2p32x2<4, 256, 2>, (const void*)k_p2p32x2<4, 128, 2>,
                        (const void*)k_p2p32x2<8, 128, 2>, (const void*)k_p2p32x2<8, 256, 2>,
                        (const void*)k_p2p32x2c<512, 4>,   (const void*)k_p2p32x2c<1024, 4>,
                        (const void*)k_p2p32x2p<4, 128, 4>, (const void*)k_p2p32x2p<4, 256, 2>,
                        (const void*)k_p2p32x2<8, 128, 4, true>};
    for (const void* k : ks) cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaGetLastError();
  });
}

namespace {

bool is_coop_variant(int v) { return v == 12 || v == 13; }

// One mixed-precision 1/r near-field launch of shape v over the work items of
// ilist (n of them; NULL: items 0 .. n-1) or, for the cooperative shapes,
// over the large leaves' units.
fmm_status launch_p2p_shape(Ctx* c, cudaStream_t s, int v, const int32_t* ilist, int n, int ctr_slot = CNT_P2P) {
  const int Lf = c->leaf, nleaf = c->lv.ncell[Lf];
  if (n <= 0) return FMM_OK;
#define P2P_LAUNCH(W, CH)                                                                              \
  k_p2p32<W, CH><<<ceil_div(n, W), W * 32, 0, s>>>(c->lv, Lf, nleaf, c->p2p_items, c->p2p_leaf, n, c->pos32,  \
                                                  c->pos32lo, c->box, c->near32, ilist)
#define P2P_LAUNCH2(W, CH, U)                                                                          \
  k_p2p32x2<W, CH, U><<<ceil_div(n, W), W * 32, 0, s>>>(c->lv, Lf, nleaf, c->p2p_items, c->p2p_leaf, n,     \
                                                       c->pos32, c->pos32lo, c->box, c->near32, ilist)
  switch (v) {
    case 1: P2P_LAUNCH2(4, 128, 4); break;
    case 2: P2P_LAUNCH2(4, 256, 2); break;
    case 3: P2P_LAUNCH2(4, 128, 2); break;
    case 4: P2P_LAUNCH2(8, 128, 2); break;
    case 5: P2P_LAUNCH2(8, 256, 2); break;
    case 6: P2P_LAUNCH(4, 256); break;
    case 7: P2P_LAUNCH(2, 128); break;
    case 8: P2P_LAUNCH(2, 256); break;
    case 9: P2P_LAUNCH(4, 128); break;
    case 10: P2P_LAUNCH(8, 128); break;
    case 11: P2P_LAUNCH(8, 256); break;
    case 12:
      if (c->p2p_nunits > 0)
        k_p2p32x2c<512, 4><<<c->p2p_nunits, CW * 32, coop_smem_bytes<512>(), s>>>(c->lv, Lf, c->p2p_items, c->p2p_leaf, c->p2p_units,
                                                            c->p2p_nunits, c->pos32, c->pos32lo, c->box, c->near32);
      break;
    case 13:
      // double-buffered chunks of 1024 sources need more than the default 48 KB of shared memory
      FMM_TRY(raise_smem_limit(c, (const void*)k_p2p32x2c<1024, 4>, coop_smem_bytes<1024>()));
      if (c->p2p_nunits > 0)
        k_p2p32x2c<1024, 4><<<c->p2p_nunits, CW * 32, coop_smem_bytes<1024>(), s>>>(c->lv, Lf, c->p2p_items, c->p2p_leaf, c->p2p_units,
                                                             c->p2p_nunits, c->pos32, c->pos32lo, c->box, c->near32);
      break;
    case 14:
    case 15: {
      // persistent warps: as many blocks as fit on every SM at once, a zeroed work counter
      static int occ[2] = {0, 0};
      int& o = occ[v - 14];
      if (o == 0) {
        if (v == 14)
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_p2p32x2p<4, 128, 4>, 128, 0);
        else
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_p2p32x2p<4, 256, 2>, 128, 0);
        cudaGetLastError();
        if (o <= 0) o = 4;
      }
      if (c->num_sms == 0) FMM_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
      int32_t* ctr = c->counters + ctr_slot;
      FMM_CUDA(c, cudaMemsetAsync(ctr, 0, sizeof(int32_t), s));
      const int grid = std::min(ceil_div(n, 4), o * c->num_sms);
      if (v == 14)
        k_p2p32x2p<4, 128, 4><<<grid, 128, 0, s>>>(c->lv, Lf, c->p2p_items, c->p2p_leaf, n, c->pos32, c->pos32lo,
                                                   c->box, c->near32, ctr, ilist);
      else
        k_p2p32x2p<4, 256, 2><<<grid, 128, 0, s>>>(c->lv, Lf, c->p2p_items, c->p2p_leaf, n, c->pos32, c->pos32lo,
                                                   c->box, c->near32, ctr, ilist);
      break;
    }
    default: P2P_LAUNCH2(8, 128, 4); break;
  }
#undef P2P_LAUNCH
#undef P2P_LAUNCH2
  return cuda_err(c, cudaGetLastError(), "P2P launch");
}

}  // namespace

// The near field.  Mixed precision, 1/r: the work items of small leaves
// (at most P2P_BIG particles) run shape p2p_variant, those of large leaves
// shape p2p_big_variant (-1: the same); one launch over all items when the
// two agree.  The cooperative shapes take large leaves only (their blocks of
// 8 warps share a leaf's sources); small leaves then take the persistent
// shape 14.
fmm_status launch_p2p(Ctx* c, cudaStream_t s) {
  const int Lf = c->leaf, nleaf = c->lv.ncell[Lf];
  if (nleaf == 0 || c->p2p_nitems == 0) return FMM_OK;
  if (c->skip_p2p) {  // far field only (fmm_evaluate_stokes): no near part
    void* nb = c->precision == FMM_MIXED ? (void*)c->near32 : (void*)c->near64;
    const size_t bytes = (c->precision == FMM_MIXED ? sizeof(float4) : sizeof(double4)) * (size_t)c->n;
    return cuda_err(c, cudaMemsetAsync(nb, 0, bytes, s), "P2P skip");
  }
  if (c->precision == FMM_MIXED && (c->kernel_s != 1.0 || c->kernel_c != 0.0)) {
    k_p2p32x2<8, 128, 4, true><<<ceil_div(c->p2p_nitems, 8), 256, 0, s>>>(c->lv, Lf, nleaf, c->p2p_items, c->p2p_leaf,
                                                                           c->p2p_nitems, c->pos32, c->pos32lo, c->box,
                                                                           c->near32, nullptr, c->kernel_s,
                                                                           c->kernel_c);
    return cuda_err(c, cudaGetLastError(), "P2P launch");
  }
  if (c->precision != FMM_MIXED) {
    k_p2p64<<<ceil_div(c->p2p_nitems, P2P_WARPS), P2P_WARPS * 32, 0, s>>>(c->lv, Lf, nleaf, c->p2p_items, c->p2p_leaf,
                                                                          c->p2p_nitems, c->pos64, c->kernel_s,
                                                                          c->kernel_c * c->kernel_c, c->near64);
    return cuda_err(c, cudaGetLastError(), "P2P launch");
  }
  int vs = c->p2p_variant;
  const int vl = c->p2p_big_variant >= 0 ? c->p2p_big_variant : c->p2p_variant;
  if (is_coop_variant(vs)) vs = 14;
  if (vs == vl && !is_coop_variant(vl)) return launch_p2p_shape(c, s, vs, nullptr, c->p2p_nitems);
  if (c->p2p_nsmall == 0) return launch_p2p_shape(c, s, vl, c->p2p_large, c->p2p_nlarge);
  if (c->p2p_nlarge == 0) return launch_p2p_shape(c, s, vs, c->p2p_small, c->p2p_nsmall);
  // the two bins run side by side: the small leaves' launch on a second
  // stream, forked from and joined back into s (in a captured graph: two
  // parallel nodes); the persistent shapes keep separate work counters
  FMM_CUDA(c, cudaEventRecord(c->ev_bin0, s));
  FMM_CUDA(c, cudaStreamWaitEvent(c->side2, c->ev_bin0, 0));
  FMM_TRY(launch_p2p_shape(c, c->side2, vs, c->p2p_small, c->p2p_nsmall, CNT_P2P2));
  FMM_TRY(launch_p2p_shape(c, s, vl, c->p2p_large, c->p2p_nlarge));
  FMM_CUDA(c, cudaEventRecord(c->ev_bin1, c->side2));
  FMM_CUDA(c, cudaStreamWaitEvent(s, c->ev_bin1, 0));
  return FMM_OK;
}

// One bin of the near field alone (fmm_autotune): bin 0 small leaves, 1 large.
fmm_status launch_p2p_bin(Ctx* c, cudaStream_t s, int bin, int v) {
  if (bin == 0) return is_coop_variant(v) ? FMM_OK : launch_p2p_shape(c, s, v, c->p2p_small, c->p2p_nsmall);
  return launch_p2p_shape(c, s, v, c->p2p_large, c->p2p_nlarge);
}

// Stokeslet near field of the loaded tree for forces f32 (Morton order,
// float4 (f, 0)); out [n] float4 (u, 0) in Morton order.
fmm_status launch_p2p_stokes(Ctx* c, cudaStream_t s, const float4* f32, float4* out) {
  const int Lf = c->leaf;
  if (c->lv.ncell[Lf] == 0 || c->p2p_nitems == 0) return FMM_OK;
  k_p2p_stokes32<4, 128><<<ceil_div(c->p2p_nitems, 4), 128, 0, s>>>(c->lv, Lf, c->p2p_items, c->p2p_leaf,
                                                                    c->p2p_nitems, c->pos32, c->pos32lo, f32, c->box,
                                                                    out);
  return cuda_err(c, cudaGetLastError(), "Stokes P2P launch");
}

FMM_DEBUG_TAKE_FN(fmm_debug_take_nearfield)

}  // namespace fmm
