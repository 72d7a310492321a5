// operators.cu -- translation operators of the black-box FMM (Sec. 2.1.1-2.1.2).
//
//  * Chebyshev roots xbar_k = cos((2k+1) pi / (2p)) (eq. 5's interpolation
//    points), the table T_n(xbar_m) used by every interpolation kernel, and
//    the 1-D child <-> parent matrices A_s[m][m'] = S(xbar_m, (s + xbar_m')/2),
//    s = -1 / +1, from which M2M and L2L are built by the tensor-product
//    ansatz (eq. 4).  These are small; the host computes them in FP64.
//  * The 316 M2L operators for unit half-width (Sec. 2.1.2: 1/r is
//    homogeneous, so one set serves every level after a 1/a scale):
//    K_t[m][n] = 1 / |2t + xbar_n - xbar_m| (3-vectors, multi-index z
//    fastest), computed on the GPU in FP64 and kept as FP64 and, for the
//    mixed path, in mean-split form (see k_m2l_ops_split) as TF32 hi/lo pairs
//    (hi = tf32(v), lo = tf32(v - hi)).  Other kernels (fmm_set_kernel): the
//    same formula with P = (r^2 + c2)^(-s/2), scaled by a^-s; with c > 0 one
//    bank per level, c2 = (c / a_l)^2 for that level's half-width a_l.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fmm {

namespace {

__device__ inline float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// FP64 bank: K_t[m][n] for m, n < C.
__global__ void k_m2l_ops64(int p, int C, const double* __restrict__ nodes, const int8_t* __restrict__ tvec,
                            double ks, double c2, double* __restrict__ K64) {
  const int64_t total = (int64_t)FMM_NT * C * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / ((int64_t)C * C));
    const int rem = (int)(i - (int64_t)t * C * C);
    const int m = rem / C, nn = rem - m * C;
    const int mi[3] = {m / (p * p), (m / p) % p, m % p};
    const int ni[3] = {nn / (p * p), (nn / p) % p, nn % p};
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double r = 2.0 * tvec[3 * t + d] + nodes[ni[d]] - nodes[mi[d]];
      r2 += r * r;
    }
    K64[i] = kernel_r2(r2, ks, c2);
  }
}

// Mixed bank, mean-split: row C holds Kbar_t[n] = (1/C) sum_m K_t[m][n] and
// rows m < C hold D_t[m][n] = K_t[m][n] - Kbar_t[n], so that M2L yields the
// cell mean of the local expansion (row C) and the deviations from it
// (rows < C) as separate FP32 numbers; every value is split into TF32 hi/lo.
// One thread per (t, n).
__global__ void k_m2l_ops_split(int p, int C, int cpad, const double* __restrict__ nodes,
                                const int8_t* __restrict__ tvec, double ks, double c2, float* __restrict__ Khi,
                                float* __restrict__ Klo) {
  const int64_t total = (int64_t)FMM_NT * cpad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / cpad), nn = (int)(i - (int64_t)t * cpad);
    float* hi = Khi + (int64_t)t * cpad * cpad;
    float* lo = Klo + (int64_t)t * cpad * cpad;
    if (nn >= C) {
      for (int m = 0; m < cpad; ++m) hi[(int64_t)m * cpad + nn] = lo[(int64_t)m * cpad + nn] = 0.f;
      continue;
    }
    const int ni[3] = {nn / (p * p), (nn / p) % p, nn % p};
    double y[3];
    for (int d = 0; d < 3; ++d) y[d] = 2.0 * tvec[3 * t + d] + nodes[ni[d]];
    auto K = [&](int m) {
      double r2 = 0.0;
      const int mi[3] = {m / (p * p), (m / p) % p, m % p};
      for (int d = 0; d < 3; ++d) {
        const double r = y[d] - nodes[mi[d]];
        r2 += r * r;
      }
      return kernel_r2(r2, ks, c2);
    };
    double mean = 0.0;
    for (int m = 0; m < C; ++m) mean += K(m);
    mean /= C;
    for (int m = 0; m < cpad; ++m) {
      const double v = m < C ? K(m) - mean : (m == C ? mean : 0.0);
      const float h = tf32_rna((float)v);
      hi[(int64_t)m * cpad + nn] = h;
      lo[(int64_t)m * cpad + nn] = tf32_rna((float)(v - (double)h));
    }
  }
}

// The same mean-split values as FP16 hi/lo pairs for the tensor-core
// kernel's FP16 form (rows of cpad halves; the kernel's tensor maps copy them
// as 32-bit words), scaled by `scale`.  mode 0: only the largest magnitude
// (float bits, atomic max into *vmax); mode 1: the banks.  One thread per
// (t, n).
__global__ void k_m2l_ops_split16(int p, int C, int cpad, const double* __restrict__ nodes,
                                  const int8_t* __restrict__ tvec, double ks, double c2, int mode, float scale,
                                  uint32_t* __restrict__ vmax, __half* __restrict__ Khi, __half* __restrict__ Klo) {
  const int64_t total = (int64_t)FMM_NT * cpad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / cpad), nn = (int)(i - (int64_t)t * cpad);
    __half* hi = Khi + (int64_t)t * cpad * cpad;
    __half* lo = Klo + (int64_t)t * cpad * cpad;
    if (nn >= C) {
      if (mode == 1)
        for (int m = 0; m < cpad; ++m) hi[(int64_t)m * cpad + nn] = lo[(int64_t)m * cpad + nn] = __float2half(0.f);
      continue;
    }
    const int ni[3] = {nn / (p * p), (nn / p) % p, nn % p};
    double y[3];
    for (int d = 0; d < 3; ++d) y[d] = 2.0 * tvec[3 * t + d] + nodes[ni[d]];
    auto K = [&](int m) {
      double r2 = 0.0;
      const int mi[3] = {m / (p * p), (m / p) % p, m % p};
      for (int d = 0; d < 3; ++d) {
        const double r = y[d] - nodes[mi[d]];
        r2 += r * r;
      }
      return kernel_r2(r2, ks, c2);
    };
    double mean = 0.0;
    for (int m = 0; m < C; ++m) mean += K(m);
    mean /= C;
    float mx = 0.f;
    for (int m = 0; m < cpad; ++m) {
      const double v = m < C ? K(m) - mean : (m == C ? mean : 0.0);
      if (mode == 0) {
        mx = fmaxf(mx, (float)fabs(v));
      } else {
        const double x = v * scale;
        const __half h = __float2half_rn((float)x);
        hi[(int64_t)m * cpad + nn] = h;
        lo[(int64_t)m * cpad + nn] = __float2half_rn((float)(x - (double)__half2float(h)));
      }
    }
    if (mode == 0) atomicMax(vmax, __float_as_uint(mx));
  }
}

double cheb_S_host(int p, const double* Tb, double xi) {
  double T0 = 1.0, T1 = xi, s = 0.0;
  for (int n = 1; n < p; ++n) {
    s += Tb[n] * T1;
    double T2 = 2.0 * xi * T1 - T0;
    T0 = T1;
    T1 = T2;
  }
  return 1.0 / p + 2.0 / p * s;
}

}  // namespace

fmm_status operators_init(Ctx* c) {
  const int p = c->order;
  std::vector<double> nodes(p, 0.0), cheb(p * p), A(2 * p * p);
  for (int k = 0; 2 * k + 1 < p; ++k) {
    nodes[k] = std::cos((2.0 * k + 1.0) * M_PI / (2.0 * p));
    nodes[p - 1 - k] = -nodes[k];
  }
  for (int m = 0; m < p; ++m) {
    double T0 = 1.0, T1 = nodes[m];
    cheb[m * p] = 1.0;
    for (int n = 1; n < p; ++n) {
      cheb[m * p + n] = T1;
      double T2 = 2.0 * nodes[m] * T1 - T0;
      T0 = T1;
      T1 = T2;
    }
  }
  for (int s = 0; s < 2; ++s)
    for (int m = 0; m < p; ++m)
      for (int mm = 0; mm < p; ++mm)
        A[(s * p + m) * p + mm] = cheb_S_host(p, &cheb[m * p], ((s ? 1.0 : -1.0) + nodes[mm]) / 2.0);

  // transfer vectors and the 189 of each child class
  std::vector<int8_t> tv;
  int slot_of[7][7][7];
  for (int x = -3; x <= 3; ++x)
    for (int y = -3; y <= 3; ++y)
      for (int z = -3; z <= 3; ++z) {
        slot_of[x + 3][y + 3][z + 3] = -1;
        if (std::abs(x) >= 2 || std::abs(y) >= 2 || std::abs(z) >= 2) {
          slot_of[x + 3][y + 3][z + 3] = (int)tv.size() / 3;
          tv.push_back((int8_t)x);
          tv.push_back((int8_t)y);
          tv.push_back((int8_t)z);
        }
      }
  std::vector<int16_t> ct;
  for (int cls = 0; cls < 8; ++cls) {
    int b[3] = {(cls >> 2) & 1, (cls >> 1) & 1, cls & 1};
    int lo[3];
    for (int d = 0; d < 3; ++d) lo[d] = b[d] ? -3 : -2;  // parent offset (b + t) >> 1 in {-1, 0, 1}
    for (int x = lo[0]; x < lo[0] + 6; ++x)
      for (int y = lo[1]; y < lo[1] + 6; ++y)
        for (int z = lo[2]; z < lo[2] + 6; ++z) {
          int sl = slot_of[x + 3][y + 3][z + 3];
          if (sl >= 0) ct.push_back((int16_t)sl);
        }
  }
  if ((int)tv.size() != 3 * FMM_NT || (int)ct.size() != 8 * FMM_NT_CLASS)
    return set_err(c, FMM_ERR_CUDA, "internal: transfer-vector tables have the wrong size");
  c->cls_t_h = ct;
  // the same pairs seen from the source: for a source of class cs, the t with
  // which it is a far-field source of some target T = S - t (T's class is cs
  // with the parities of t flipped, and t must be in T's class list)
  std::vector<int16_t> st;
  for (int cs = 0; cs < 8; ++cs)
    for (int sl = 0; sl < FMM_NT; ++sl) {
      const int ctg = cs ^ (((tv[3 * sl] & 1) << 2) | ((tv[3 * sl + 1] & 1) << 1) | (tv[3 * sl + 2] & 1));
      bool in = false;
      for (int k = 0; k < FMM_NT_CLASS; ++k) in = in || ct[ctg * FMM_NT_CLASS + k] == sl;
      if (in) st.push_back((int16_t)sl);
    }
  if ((int)st.size() != 8 * FMM_NT_CLASS)
    return set_err(c, FMM_ERR_CUDA, "internal: source-side transfer-vector tables have the wrong size");
  c->src_t_h = st;

  std::vector<float> cheb32(cheb.begin(), cheb.end()), A32(A.begin(), A.end());
  void* ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(double) * p));
  c->nodes64 = (double*)ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(double) * p * p));
  c->cheb64 = (double*)ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(float) * p * p));
  c->cheb32 = (float*)ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(double) * 2 * p * p));
  c->m2m64 = (double*)ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(float) * 2 * p * p));
  c->m2m32 = (float*)ptr;
  FMM_TRY(dalloc(c, &ptr, tv.size()));
  c->tvec = (int8_t*)ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(int16_t) * ct.size()));
  c->cls_t = (int16_t*)ptr;
  FMM_TRY(dalloc(c, &ptr, sizeof(int16_t) * st.size()));
  c->src_t = (int16_t*)ptr;
  FMM_CUDA(c, cudaMemcpyAsync(c->nodes64, nodes.data(), sizeof(double) * p, cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->cheb64, cheb.data(), sizeof(double) * p * p, cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->cheb32, cheb32.data(), sizeof(float) * p * p, cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->m2m64, A.data(), sizeof(double) * 2 * p * p, cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->m2m32, A32.data(), sizeof(float) * 2 * p * p, cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->tvec, tv.data(), tv.size(), cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->cls_t, ct.data(), sizeof(int16_t) * ct.size(), cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->src_t, st.data(), sizeof(int16_t) * st.size(), cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
  return FMM_OK;
}

// M2L operator banks for one precision, built on first use.  With c > 0 the
// banks depend on the root width: they are regenerated in place (same
// buffers, so captured graphs stay valid) when the width changes, and
// reallocated when the number of levels does.
fmm_status operators_m2l(Ctx* c, int precision) {
  const int p = c->order, C = c->ncoef, cp = c->cpad;
  if (c->leaf < 2) return FMM_OK;
  const int nb = op_banks(c);
  const double W = c->kernel_c > 0.0 ? c->box_host[3] : 0.0;
  const bool mixed = precision == FMM_MIXED;
  // the tensor-core kernel's FP16 form takes FP16 banks; the CUDA-core kernel TF32 ones
  const bool f16 = mixed && m2l_uses_f16(c) && m2l_kind(c) == 2;
  bool& built = mixed ? c->ops32 : c->ops64;
  int& bnb = mixed ? c->ops32_nb : c->ops64_nb;
  double& bW = mixed ? c->ops32_W : c->ops64_W;
  if (mixed && built && c->ops32_f16 != f16) built = false;
  if (built && bnb == nb && bW == W) return FMM_OK;
  const size_t bank64 = (size_t)FMM_NT * C * C, bank32 = (size_t)FMM_NT * cp * cp;
  void* ptr;
  if (built && bnb != nb) {  // a tree with another number of levels
    if (mixed) {
      dfree(c, c->Khi, sizeof(float) * bank32 * bnb);
      dfree(c, c->Klo, sizeof(float) * bank32 * bnb);
      c->Khi = c->Klo = nullptr;
    } else {
      dfree(c, c->K64, sizeof(double) * bank64 * bnb);
      c->K64 = nullptr;
    }
    built = false;
    c->graph_ok = false;
  }
  if (mixed && !c->Khi) {
    FMM_TRY(dalloc(c, &ptr, sizeof(float) * bank32 * nb));
    c->Khi = (float*)ptr;
    FMM_TRY(dalloc(c, &ptr, sizeof(float) * bank32 * nb));
    c->Klo = (float*)ptr;
  }
  if (!mixed && !c->K64) {
    FMM_TRY(dalloc(c, &ptr, sizeof(double) * bank64 * nb));
    c->K64 = (double*)ptr;
  }
  if (f16) {
    // one scale for every bank: the largest magnitude first
    uint32_t* vmax = (uint32_t*)c->scratch;
    FMM_CUDA(c, cudaMemsetAsync(vmax, 0, sizeof(uint32_t), c->stream));
    for (int b = 0; b < nb; ++b) {
      const double ca = c->kernel_c > 0.0 ? c->kernel_c * std::ldexp(1.0, 2 + b + 1) / W : 0.0;
      k_m2l_ops_split16<<<ceil_div((int64_t)FMM_NT * cp, 128), 128, 0, c->stream>>>(
          p, C, cp, c->nodes64, c->tvec, c->kernel_s, ca * ca, 0, 1.f, vmax, nullptr, nullptr);
    }
    uint32_t vb = 0;
    FMM_CUDA(c, cudaMemcpyAsync(&vb, vmax, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    FMM_CUDA(c, cudaStreamSynchronize(c->stream));
    float vf;
    std::memcpy(&vf, &vb, sizeof(vf));
    c->ops_kscale = tc::pow2_scale(vf);
  }
  for (int b = 0; b < nb; ++b) {
    // bank b serves level 2 + b (c > 0): c / a_l = c 2^(l+1) / W
    const double ca = c->kernel_c > 0.0 ? c->kernel_c * std::ldexp(1.0, 2 + b + 1) / W : 0.0;
    if (f16)
      k_m2l_ops_split16<<<ceil_div((int64_t)FMM_NT * cp, 128), 128, 0, c->stream>>>(
          p, C, cp, c->nodes64, c->tvec, c->kernel_s, ca * ca, 1, c->ops_kscale, nullptr,
          (__half*)c->Khi + bank32 * b, (__half*)c->Klo + bank32 * b);
    else if (mixed)
      k_m2l_ops_split<<<ceil_div((int64_t)FMM_NT * cp, 128), 128, 0, c->stream>>>(
          p, C, cp, c->nodes64, c->tvec, c->kernel_s, ca * ca, c->Khi + bank32 * b, c->Klo + bank32 * b);
    else
      k_m2l_ops64<<<1184, 256, 0, c->stream>>>(p, C, c->nodes64, c->tvec, c->kernel_s, ca * ca, c->K64 + bank64 * b);
  }
  FMM_CUDA(c, cudaGetLastError());
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  built = true;
  bnb = nb;
  bW = W;
  if (mixed) {
    c->ops32_f16 = f16;
    c->graph_ok = false;  // the tensor maps and the kernel's form follow the banks' format
  }
  return FMM_OK;
}

}  // namespace fmm
