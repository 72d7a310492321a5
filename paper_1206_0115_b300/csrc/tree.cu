// tree.cu -- octree construction on the device (Sec. 3.2 hierarchical
// subdivision into cells; Sec. 4.2 Morton ordering of cells).
//
// Steps: bounding cube (exact FP64 min/max) -> leaf-level Morton keys
// (IEEE FP64 quantisation, no contraction) -> stable LSD radix sort of
// (key, input index) -> gather into Morton order -> per level, the unique
// cell keys with particle / child ranges -> dense key -> cell grids ->
// cells grouped by child class -> M2L tiles and their source lists.
// Every step is integer or exact, so the tree is bit-identical to any other
// implementation of the same rules.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace fmm {

namespace {

constexpr int BB_THREADS = 256;
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int CNT_BAD = 127;  // counters[] slot of the non-finite-input flag
constexpr int CNT_CLS = 16;   // counters[16 + 8 l + c] = cells of class c at level l
constexpr int CNT_ITEMS = 120;  // counters[120] = P2P work items (leaf, 32-target batch)
constexpr int CNT_UNITS = 121;  // counters[121] = cooperative P2P units (up to 8 items of one leaf)
constexpr int CNT_BINS = 122;   // counters[122], [123] (one 64-bit word) = P2P items of small / large leaves
// the work-list totals are 64-bit words: (items, units) and (small, large)
static_assert(CNT_UNITS == CNT_ITEMS + 1 && CNT_ITEMS % 2 == 0 && CNT_BINS % 2 == 0, "64-bit counter words");

__device__ inline double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Order key of a double: an int64 that orders as the double does (-0 just
// below +0), so min / max / comparisons run on the integer pipes (FP64
// arithmetic runs at 1/64 of the FP32 rate on this part).
__device__ inline int64_t dkey(double x) {
  const int64_t b = __double_as_longlong(x);
  return b ^ ((b >> 63) & INT64_MAX);
}
__device__ inline double dkey_inv(int64_t k) { return __longlong_as_double(k ^ ((k >> 63) & INT64_MAX)); }
__device__ inline int bits_nonfinite(int64_t b) { return ((b >> 52) & 0x7ff) == 0x7ff; }
constexpr int64_t KEY_PINF = 0x7ff0000000000000LL;             // dkey(+inf)
constexpr int64_t KEY_NINF = (int64_t)0x800fffffffffffffULL;   // dkey(-inf)
__device__ inline int64_t warp_min64(int64_t v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, o));
  return v;
}
__device__ inline int64_t warp_max64(int64_t v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, o));
  return v;
}

// Per-block min/max of each coordinate (on order keys: exact, the same
// values as FP64 min/max); raises the flag on non-finite input.
__global__ void __launch_bounds__(BB_THREADS)
k_bbox_partial(int64_t n, const double* __restrict__ xyz, const double* __restrict__ q,
               double* __restrict__ part, int32_t* __restrict__ counters) {
  int64_t mn[3] = {KEY_PINF, KEY_PINF, KEY_PINF}, mx[3] = {KEY_NINF, KEY_NINF, KEY_NINF};
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      const int64_t b = __double_as_longlong(xyz[3 * i + d]);
      bad |= bits_nonfinite(b);
      const int64_t k = b ^ ((b >> 63) & INT64_MAX);
      mn[d] = min(mn[d], k);
      mx[d] = max(mx[d], k);
    }
    bad |= bits_nonfinite(__double_as_longlong(q[i]));
  }
  __shared__ int64_t s[2][3][BB_THREADS / 32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = 0; d < 3; ++d) {
    int64_t a = warp_min64(mn[d]), b = warp_max64(mx[d]);
    if (lane == 0) {
      s[0][d][w] = a;
      s[1][d][w] = b;
    }
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; ++d) {
      int64_t a = s[0][d][0], b = s[1][d][0];
      for (int k = 1; k < BB_THREADS / 32; ++k) {
        a = min(a, s[0][d][k]);
        b = max(b, s[1][d][k]);
      }
      part[6 * blockIdx.x + d] = dkey_inv(a);
      part[6 * blockIdx.x + 3 + d] = dkey_inv(b);
    }
    if (bad) atomicOr(&counters[CNT_BAD], 1);
  }
}

// Leaf cell of coordinate x along one axis: floor(((x - lo) / W) * 2^leaf)
// clamped to the cube.  Multiplying by 2^leaf is exact; the subtraction and
// the division are the IEEE round-to-nearest operations, written out so
// nothing is contracted.  Each step rounds monotonically, so the cell is a
// nondecreasing function of x.
__device__ inline int cell_of(double x, double lo, double W, int leaf) {
  const double t = __ddiv_rn(__dsub_rn(x, lo), W);
  const double u = floor(__dmul_rn(t, (double)(1u << leaf)));
  const int top = (1 << leaf) - 1;
  return (u >= 0.0) ? (u <= (double)top ? (int)u : top) : 0;
}

// Order key of the smallest double x with cell_of(x) >= k (1 <= k <= top):
// bracketed around lo + k W 2^-leaf, then bisected over order keys.  The
// bracket holds cell_of(a) < k <= cell_of(b); cell_of(lo) = 0 and
// cell_of(DBL_MAX) = top bound it, and every key in [dkey(lo), dkey(DBL_MAX)]
// is a finite double.
__device__ int64_t cell_threshold(double lo, double W, int leaf, int k) {
  const int64_t kmin = dkey(lo), kmax = dkey(DBL_MAX);
  int64_t m = dkey(lo + W * ((double)k / (double)(1 << leaf)));
  m = min(max(m, kmin), kmax);
  int64_t a = m, b = m;
  uint64_t step = 16;
  while (a > kmin && cell_of(dkey_inv(a), lo, W, leaf) >= k) {
    a = ((uint64_t)a - (uint64_t)kmin > step) ? (int64_t)((uint64_t)a - step) : kmin;
    step = min(step << 1, (uint64_t)1 << 62);  // every pass moves; at most ~64 passes
  }
  step = 16;
  while (b < kmax && cell_of(dkey_inv(b), lo, W, leaf) < k) {
    b = ((uint64_t)kmax - (uint64_t)b > step) ? (int64_t)((uint64_t)b + step) : kmax;
    step = min(step << 1, (uint64_t)1 << 62);
  }
  while ((uint64_t)b - (uint64_t)a > 1) {
    const int64_t mid = (int64_t)((uint64_t)a + (((uint64_t)b - (uint64_t)a) >> 1));
    if (cell_of(dkey_inv(mid), lo, W, leaf) >= k) b = mid;
    else a = mid;
  }
  return b;
}

// Root cube: corner = minimum per axis, side = largest extent (1 if zero).
// Every block reduces the per-block partials (min and max are exact in any
// order); block 0 writes box[0..3], the leaf frame of k_gather, box[4] =
// 2^-e (W = m 2^e, 1 <= m < 2) and box[5] holding the FP32 pair
// Rh + Rl = 2^leaf / m, and box[6] = 2^(leaf + 1) / W, the reciprocal of a
// leaf's half-width.  With thr given, the blocks then fill the cell
// thresholds of the leaf level, thr[d 2^leaf + k] = cell_threshold(k) for
// k = 1 .. 2^leaf - 1 (the cell of x along axis d is the number of them <= x).
__global__ void __launch_bounds__(256) k_bbox_final(int nblocks, const double* __restrict__ part,
                                                    double* __restrict__ box, int leaf, int64_t* __restrict__ thr) {
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      mn[d] = fmin(mn[d], part[6 * b + d]);
      mx[d] = fmax(mx[d], part[6 * b + 3 + d]);
    }
  __shared__ double s[2][3][8];
  __shared__ double cube[4];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = 0; d < 3; ++d) {
    const double a = warp_min(mn[d]), b = warp_max(mx[d]);
    if (lane == 0) {
      s[0][d][w] = a;
      s[1][d][w] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double w3 = 0.0;
    for (int d = 0; d < 3; ++d) {
      double a = s[0][d][0], b = s[1][d][0];
      for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
        a = fmin(a, s[0][d][k]);
        b = fmax(b, s[1][d][k]);
      }
      cube[d] = a;
      w3 = fmax(w3, __dsub_rn(b, a));
    }
    cube[3] = (w3 > 0.0) ? w3 : 1.0;
    if (blockIdx.x == 0) {
      for (int d = 0; d < 4; ++d) box[d] = cube[d];
      int e = 0;
      frexp(cube[3], &e);  // W = m 2^(e - 1), 1 <= m < 2
      e = min(max(e - 1, -1021), 1021);
      const double scl = ldexp(1.0, -e);
      const double R = __ddiv_rn((double)(1u << leaf), __dmul_rn(cube[3], scl));
      const float Rh = __double2float_rn(R);
      box[4] = scl;
      box[6] = __ddiv_rn((double)(2u << leaf), cube[3]);  // 1 / (half-width of a leaf)
      float* f = (float*)(box + 5);
      f[0] = Rh;
      f[1] = __double2float_rn(__dsub_rn(R, (double)Rh));
      if (thr)
        for (int d = 0; d < 3; ++d) thr[d << leaf] = INT64_MIN;  // never read by the search
    }
  }
  if (!thr) return;
  __syncthreads();
  const int top = (1 << leaf) - 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * top; t += gridDim.x * blockDim.x) {
    const int d = t / top, k = t - d * top + 1;
    thr[(d << leaf) + k] = cell_threshold(cube[d], cube[3], leaf, k);
  }
}

// Leaf-level key: per axis the number of cell thresholds <= x (the rule of
// cell_of, exactly), found by binary search over the table in shared memory.
__global__ void __launch_bounds__(256) k_morton(int64_t n, const double* __restrict__ xyz,
                                                const int64_t* __restrict__ thr, int leaf,
                                                uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
  extern __shared__ int64_t sthr[];
  for (int t = threadIdx.x; t < (3 << leaf); t += blockDim.x) sthr[t] = thr[t];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[3];
    for (int d = 0; d < 3; ++d) {
      const int64_t kx = dkey(xyz[3 * i + d]);
      const int64_t* T = sthr + (d << leaf);
      int pos = 0;
      for (int step = 1 << leaf >> 1; step > 0; step >>= 1)
        if (T[pos + step] <= kx) pos += step;
      c[d] = (uint32_t)pos;
    }
    key[i] = morton3(c[0], c[1], c[2]);
    idx[i] = (uint32_t)i;
  }
}

// ---- stable LSD radix sort (8-bit digits) -------------------------------------

__global__ void __launch_bounds__(RS_THREADS)
k_radix_hist(int64_t n, const uint32_t* __restrict__ keys, int shift, uint32_t* __restrict__ hist,
             int ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
    int64_t g = base + k;
    if (g < n) atomicAdd(&h[(keys[g] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `count` words in one block; the total goes to *total.
template <typename W>
__global__ void __launch_bounds__(1024) k_scan1(W* __restrict__ data, int64_t count, W* total) {
  __shared__ W part[1024];
  const int t = threadIdx.x;
  int64_t per = (count + 1023) / 1024;
  int64_t b = t * per, e = b + per < count ? b + per : count;
  W s = 0;
  for (int64_t i = b; i < e; ++i) s += data[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    W v = (t >= o) ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  W run = part[t] - s;
  for (int64_t i = b; i < e; ++i) {
    W v = data[i];
    data[i] = run;
    run += v;
  }
  if (t == 1023 && total) *total = part[1023];
}

// Exclusive prefix of v over the NT threads of a block (warp shuffles,
// then warp 0 over the NT / 32 warp totals); total = the block's sum.
// Every thread of the block calls it; ws: NT / 32 words of shared memory.
template <int NT, typename W>
__device__ __forceinline__ W block_excl_scan(W v, W* ws, W& total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  W incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const W t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    W y = lane < NW ? ws[lane] : W(0);
    for (int o = 1; o < 32; o <<= 1) {
      const W t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    if (lane < NW) ws[lane] = y;
  }
  __syncthreads();
  const W before = w > 0 ? ws[w - 1] : W(0);
  total = ws[NW - 1];
  __syncthreads();  // ws is free for the next call
  return before + incl - v;
}

// Exclusive scan of data[0..count) in place by one block of 1024 threads,
// in chunks of 1024 x SB_ITEMS entries (each thread scans SB_ITEMS
// consecutive ones) with a running carry; the next chunk's loads are issued
// before the current chunk is scanned.  The total goes to *total (if not
// NULL).  For counts up to SB_MAX, where the three-pass scan's launches cost
// more than the work.
constexpr int SB_ITEMS = 8;
constexpr int SB_CHUNK = 1024 * SB_ITEMS;
constexpr int64_t SB_MAX = 16384;

template <typename W>
__global__ void __launch_bounds__(1024) k_scan_block(W* __restrict__ data, int64_t count, W* total) {
  __shared__ W ws[32];
  const int tid = threadIdx.x;
  W cur[SB_ITEMS], nxt[SB_ITEMS];
#pragma unroll
  for (int j = 0; j < SB_ITEMS; ++j) {
    const int64_t i = (int64_t)tid * SB_ITEMS + j;
    cur[j] = i < count ? data[i] : W(0);
  }
  W carry = 0;
  for (int64_t c0 = 0; c0 < count; c0 += SB_CHUNK) {
#pragma unroll
    for (int j = 0; j < SB_ITEMS; ++j) {
      const int64_t i = c0 + SB_CHUNK + (int64_t)tid * SB_ITEMS + j;
      nxt[j] = i < count ? data[i] : W(0);
    }
    W sum = 0;
#pragma unroll
    for (int j = 0; j < SB_ITEMS; ++j) sum += cur[j];
    W tot;
    W run = carry + block_excl_scan<1024>(sum, ws, tot);
#pragma unroll
    for (int j = 0; j < SB_ITEMS; ++j) {
      const int64_t i = c0 + (int64_t)tid * SB_ITEMS + j;
      if (i < count) data[i] = run;
      run += cur[j];
      cur[j] = nxt[j];
    }
    carry += tot;
  }
  if (tid == 0 && total) *total = carry;
}

// Exclusive scan of long arrays in three passes: per-block sums of
// SC_CHUNK-entry chunks (coalesced), k_scan_block over the block sums, and a
// per-block scan of each chunk staged through shared memory (coalesced loads
// and stores; each thread scans SC_ITEMS consecutive entries).
constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_CHUNK = SC_THREADS * SC_ITEMS;

template <typename W>
__global__ void __launch_bounds__(SC_THREADS) k_scan_sums(const W* __restrict__ data, int64_t count,
                                                         W* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
  W v = 0;
  for (int k = threadIdx.x; k < SC_CHUNK; k += SC_THREADS) {
    const int64_t i = base + k;
    if (i < count) v += data[i];
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ W ws[SC_THREADS / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    W t = 0;
    for (int w = 0; w < SC_THREADS / 32; ++w) t += ws[w];
    bsum[blockIdx.x] = t;
  }
}

template <typename W>
__global__ void __launch_bounds__(SC_THREADS) k_scan_chunks(W* __restrict__ data, int64_t count,
                                                           const W* __restrict__ boff) {
  __shared__ W sm[SC_CHUNK];
  __shared__ W ws[SC_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < SC_CHUNK; k += SC_THREADS) {
    const int64_t i = base + k;
    sm[k] = i < count ? data[i] : W(0);
  }
  __syncthreads();
  W loc[SC_ITEMS];
  W sum = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    loc[j] = sm[tid * SC_ITEMS + j];
    sum += loc[j];
  }
  W incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const W v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  W woff = 0;
  for (int w = 0; w < warp; ++w) woff += ws[w];
  W run = boff[blockIdx.x] + woff + incl - sum;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    sm[tid * SC_ITEMS + j] = run;
    run += loc[j];
  }
  __syncthreads();
  for (int k = tid; k < SC_CHUNK; k += SC_THREADS) {
    const int64_t i = base + k;
    if (i < count) data[i] = sm[k];
  }
}

// Exclusive scan of data[0..count) in place; the total goes to *total (if
// not NULL).  work: ceil(count / SC_CHUNK) words of scratch.
template <typename W>
void scan_excl(cudaStream_t s, W* data, int64_t count, W* total, W* work, int64_t* launches) {
  if (count <= SB_MAX) {
    k_scan_block<W><<<1, 1024, 0, s>>>(data, count, total);
    *launches += 1;
    return;
  }
  const int nb = ceil_div(count, SC_CHUNK);
  k_scan_sums<W><<<nb, SC_THREADS, 0, s>>>(data, count, work);
  k_scan_block<W><<<1, 1024, 0, s>>>(work, nb, total);
  k_scan_chunks<W><<<nb, SC_THREADS, 0, s>>>(data, count, work);
  *launches += 3;
}

// Scatter of one digit pass.  The tile is walked in order, 256 keys at a time;
// within a round a key's rank among equal digits is (earlier rounds) +
// (earlier warps of this round) + (lower lanes of its warp), so equal keys
// keep their input order.
__global__ void __launch_bounds__(RS_THREADS)
k_radix_scatter(int64_t n, const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int shift,
                const uint32_t* __restrict__ offs, int ntiles) {
  __shared__ uint32_t base_off[256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[RS_THREADS / 32][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  base_off[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
  run[tid] = 0;
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ITEMS; ++r) {
    for (int i = tid; i < (RS_THREADS / 32) * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    int64_t g = tile0 + (int64_t)r * RS_THREADS + tid;
    bool valid = g < n;
    uint32_t k = valid ? kin[g] : 0u, v = valid ? vin[g] : 0u;
    uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
    __syncthreads();
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int wrank = __popc(peers & lt);
    if (valid && wrank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[tid];
      for (int w = 0; w < RS_THREADS / 32; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      run[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = base_off[d] + wcnt[warp][d] + (uint32_t)wrank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();  // the next round clears wcnt, which this round's scatter still reads
  }
}

// Root cube, leaf frame and cell thresholds (k_bbox_final), then the keys
// (k_morton); part holds the per-block partials of k_bbox_partial.
void launch_cube_keys(cudaStream_t s, int64_t n, const double* xyz, int nbb, const double* part, double* box,
                      int64_t* thr, int leaf, uint32_t* key, uint32_t* idx) {
  const int top = (1 << leaf) - 1;
  k_bbox_final<<<std::max(1, ceil_div(3 * top, 256)), 256, 0, s>>>(nbb, part, box, leaf, thr);
  const int64_t nb = std::min<int64_t>(ceil_div(n, 256), 148 * 8);
  k_morton<<<(int)nb, 256, (size_t)(3 << leaf) * sizeof(int64_t), s>>>(n, xyz, thr, leaf, key, idx);
}

// Leaf-frame coordinate along one axis, v = (x - lo) / w - (i + 1/2) with w
// the leaf width and i the leaf's cell, split as hi + lo: hi on the grid of
// multiples of 2^-23 (|hi| <= 1/2 + 2^-23: hi plus a neighbour shift of +-1
// and the difference of two such values are exact in FP32, which the near
// field relies on) and lo the remainder.  One FP64 subtraction and an exact
// power-of-two scaling give d = (x - lo) 2^-e; d is cut into two FP32 words
// (the upper 24 significand bits and the rounded rest) and multiplied by
// 2^leaf / (W 2^-e), held as two FP32 words, in double-float arithmetic:
// Dekker's product with an FMA for the leading term, Knuth's two-sum for the
// offset from the cell centre.  v carries ~2^-46 relative error of
// (x - lo) / w, i.e. about 2^(leaf - 46) leaf widths.
__device__ inline void leaf_frame(double x, double lo, double scl, float Rh, float Rl, int i, float& hi,
                                  float& rest) {
  const double d = __dmul_rn(__dsub_rn(x, lo), scl);
  const double d1 = __longlong_as_double(__double_as_longlong(d) & ~0x1fffffffLL);
  const float dh = __double2float_rn(d1), dl = __double2float_rn(__dsub_rn(d, d1));
  const float p = __fmul_rn(dh, Rh);
  const float e = __fmaf_rn(dh, Rl, __fmaf_rn(dl, Rh, __fmaf_rn(dh, Rh, -p)));
  const float c = __fadd_rn((float)i, 0.5f);
  const float s = __fsub_rn(p, c);
  const float bv = __fsub_rn(s, p);
  const float t = __fadd_rn(__fadd_rn(__fsub_rn(p, __fsub_rn(s, bv)), __fsub_rn(-c, bv)), e);  // v = s + t
  hi = __fsub_rn(__fadd_rn(__fadd_rn(s, t), 1.5f), 1.5f);
  rest = __fadd_rn(__fsub_rn(s, hi), t);
}

// Morton-ordered particle copies: FP64 (x, y, z, q), FP32 leaf-frame
// coordinates (hi, with q) and their remainders (leaf_frame; the frame
// constants are box[4] and box[5], written by k_bbox_final).
__global__ void k_gather(int64_t n, const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sidx,
                         const double* __restrict__ xyz, const double* __restrict__ q,
                         const double* __restrict__ box, int32_t* __restrict__ perm,
                         double4* __restrict__ pos64, float4* __restrict__ pos32, float4* __restrict__ pos32lo) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  uint32_t i = sidx[r];
  if (!FMM_GUARD((int64_t)i < n, CHK_GATHER_INDEX, r)) return;
  perm[r] = (int32_t)i;
  double x = xyz[3 * (int64_t)i], y = xyz[3 * (int64_t)i + 1], z = xyz[3 * (int64_t)i + 2];
  double qq = q[i];
  pos64[r] = make_double4(x, y, z, qq);
  int ix, iy, iz;
  demorton3(skey[r], ix, iy, iz);
  const double scl = box[4];
  const float2 R = *(const float2*)(box + 5);
  float hx, hy, hz, lx, ly, lz;
  leaf_frame(x, box[0], scl, R.x, R.y, ix, hx, lx);
  leaf_frame(y, box[1], scl, R.x, R.y, iy, hy, ly);
  leaf_frame(z, box[2], scl, R.x, R.y, iz, hz, lz);
  pos32[r] = make_float4(hx, hy, hz, (float)qq);
  pos32lo[r] = make_float4(lx, ly, lz, 0.f);
}

// ---- batched problems (one tree over all problems' slots) ----------------------

constexpr int FB_CHUNK = BB_THREADS * 8;  // particles per bounding-box block

// last k in [0, cnt) with a[k] <= v (a ascending, a[0] <= v)
template <typename A, typename V>
__device__ inline int last_le(const A* __restrict__ a, int cnt, V v) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((V)a[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per-block min/max of one problem's chunk (blocks of a problem are
// consecutive: bstart[k] .. bstart[k+1]; order keys as in k_bbox_partial);
// raises the flag on non-finite input.
__global__ void __launch_bounds__(BB_THREADS)
k_fbox_partial(int nprob, const int32_t* __restrict__ bstart, const int64_t* __restrict__ pstart,
               const double* __restrict__ xyz, const double* __restrict__ q, double* __restrict__ part,
               int32_t* __restrict__ counters) {
  const int k = last_le(bstart, nprob, (int32_t)blockIdx.x);
  const int64_t beg = pstart[k] + (int64_t)(blockIdx.x - bstart[k]) * FB_CHUNK;
  const int64_t end = min(pstart[k + 1], beg + FB_CHUNK);
  int64_t mn[3] = {KEY_PINF, KEY_PINF, KEY_PINF}, mx[3] = {KEY_NINF, KEY_NINF, KEY_NINF};
  int bad = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += BB_THREADS) {
    for (int d = 0; d < 3; ++d) {
      const int64_t b = __double_as_longlong(xyz[3 * i + d]);
      bad |= bits_nonfinite(b);
      const int64_t kk = b ^ ((b >> 63) & INT64_MAX);
      mn[d] = min(mn[d], kk);
      mx[d] = max(mx[d], kk);
    }
    bad |= bits_nonfinite(__double_as_longlong(q[i]));
  }
  __shared__ int64_t sm[2][3][BB_THREADS / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = 0; d < 3; ++d) {
    const int64_t a = warp_min64(mn[d]), b = warp_max64(mx[d]);
    if (lane == 0) {
      sm[0][d][w] = a;
      sm[1][d][w] = b;
    }
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; ++d) {
      int64_t a = sm[0][d][0], b = sm[1][d][0];
      for (int j = 1; j < BB_THREADS / 32; ++j) {
        a = min(a, sm[0][d][j]);
        b = max(b, sm[1][d][j]);
      }
      part[6 * blockIdx.x + d] = dkey_inv(a);
      part[6 * blockIdx.x + 3 + d] = dkey_inv(b);
    }
    if (bad) atomicOr(&counters[CNT_BAD], 1);
  }
}

// Root cube of each problem (one block per problem; the rule of k_bbox_final),
// its output scale lambda_k = 2^-S_k / W_k, its leaf frame (frame[4k]: 2^-e,
// the FP32 pair 2^L / (W 2^-e), 1 / W) and its cell thresholds (thr +
// prob[k].thr, laid out as in k_bbox_final).
__global__ void __launch_bounds__(256)
k_fbox_final(const int32_t* __restrict__ bstart, const double* __restrict__ part,
             const BatchProb* __restrict__ prob, double* __restrict__ fbox, double* __restrict__ fscale,
             double* __restrict__ frame, int64_t* __restrict__ thr) {
  const int k = blockIdx.x;
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = bstart[k] + threadIdx.x; b < bstart[k + 1]; b += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      mn[d] = fmin(mn[d], part[6 * b + d]);
      mx[d] = fmax(mx[d], part[6 * b + 3 + d]);
    }
  __shared__ double sm[2][3][8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = 0; d < 3; ++d) {
    const double a = warp_min(mn[d]), b = warp_max(mx[d]);
    if (lane == 0) {
      sm[0][d][w] = a;
      sm[1][d][w] = b;
    }
  }
  __syncthreads();
  __shared__ double cube[4];
  const BatchProb pb = prob[k];
  if (threadIdx.x == 0) {
    const bool empty = bstart[k + 1] == bstart[k];
    double w3 = 0.0;
    for (int d = 0; d < 3; ++d) {
      double a = sm[0][d][0], b = sm[1][d][0];
      for (int j = 1; j < (int)(blockDim.x >> 5); ++j) {
        a = fmin(a, sm[0][d][j]);
        b = fmax(b, sm[1][d][j]);
      }
      cube[d] = empty ? 0.0 : a;
      w3 = empty ? 0.0 : fmax(w3, __dsub_rn(b, a));
    }
    const double W = (w3 > 0.0) ? w3 : 1.0;
    cube[3] = W;
    for (int d = 0; d < 4; ++d) fbox[4 * k + d] = cube[d];
    fscale[k] = __ddiv_rn(ldexp(1.0, -pb.S), W);
    int e = 0;
    frexp(W, &e);
    e = min(max(e - 1, -1021), 1021);
    const double scl = ldexp(1.0, -e);
    const double R = __ddiv_rn((double)(1u << pb.L), __dmul_rn(W, scl));
    const float Rh = __double2float_rn(R);
    frame[4 * k] = scl;
    float* f = (float*)(frame + 4 * k + 1);
    f[0] = Rh;
    f[1] = __double2float_rn(__dsub_rn(R, (double)Rh));
    frame[4 * k + 2] = 1.0 / W;
    for (int d = 0; d < 3; ++d) thr[pb.thr + (d << pb.L)] = INT64_MIN;  // never read by the search
  }
  __syncthreads();
  const int top = (1 << pb.L) - 1;
  for (int t = threadIdx.x; t < 3 * top; t += blockDim.x) {
    const int d = t / top, kk = t - d * top + 1;
    thr[pb.thr + (d << pb.L) + kk] = cell_threshold(cube[d], cube[3], pb.L, kk);
  }
}

// Forest leaf key of every particle: the slot's first key + the key the
// single-problem rule (cell_of) gives in the problem's own cube, read off the
// problem's cell thresholds by binary search.
__global__ void k_fmorton(int64_t n, int nprob, const int64_t* __restrict__ pstart,
                          const BatchProb* __restrict__ prob, const int64_t* __restrict__ thr,
                          const double* __restrict__ xyz, uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = last_le(pstart, nprob, i);
  const BatchProb pb = prob[k];
  uint32_t c[3];
  for (int d = 0; d < 3; ++d) {
    const int64_t kx = dkey(xyz[3 * i + d]);
    const int64_t* T = thr + pb.thr + (d << pb.L);
    int pos = 0;
    for (int step = 1 << pb.L >> 1; step > 0; step >>= 1)
      if (__ldg(T + pos + step) <= kx) pos += step;
    c[d] = (uint32_t)pos;
  }
  key[i] = pb.slot_key + morton3(c[0], c[1], c[2]);
  idx[i] = (uint32_t)i;
}

// Morton-ordered copies of a batch: FP64 positions mapped into the forest
// cube (x' = o_k + t 2^-S_k, t = (x - lo_k) / W_k with the correctly rounded
// 1 / W_k), FP32 leaf-frame coordinates from the problem's own cube
// (leaf_frame with the problem's frame).
__global__ void k_fgather(int64_t n, int nprob, const int64_t* __restrict__ pstart,
                          const BatchProb* __restrict__ prob, const double* __restrict__ fbox,
                          const double* __restrict__ frame, const uint32_t* __restrict__ skey,
                          const uint32_t* __restrict__ sidx, const double* __restrict__ xyz,
                          const double* __restrict__ q, int32_t* __restrict__ perm, double4* __restrict__ pos64,
                          float4* __restrict__ pos32, float4* __restrict__ pos32lo) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t i = sidx[r];
  if (!FMM_GUARD((int64_t)i < n, CHK_GATHER_INDEX, r)) return;
  perm[r] = (int32_t)i;
  const int k = last_le(pstart, nprob, (int64_t)i);
  const BatchProb pb = prob[k];
  const double* box = fbox + 4 * k;
  const double x = xyz[3 * (int64_t)i], y = xyz[3 * (int64_t)i + 1], z = xyz[3 * (int64_t)i + 2];
  const double qq = q[i];
  int ox, oy, oz;
  demorton3(pb.slot_key >> (3 * pb.L), ox, oy, oz);
  const double ws = ldexp(1.0, -pb.S), iW = frame[4 * k + 2];
  const double tx = (x - box[0]) * iW, ty = (y - box[1]) * iW, tz = (z - box[2]) * iW;
  pos64[r] = make_double4(__dadd_rn((double)ox * ws, __dmul_rn(tx, ws)), __dadd_rn((double)oy * ws, __dmul_rn(ty, ws)),
                          __dadd_rn((double)oz * ws, __dmul_rn(tz, ws)), qq);
  int ix, iy, iz;
  demorton3(skey[r] - pb.slot_key, ix, iy, iz);
  const double scl = frame[4 * k];
  const float2 R = *(const float2*)(frame + 4 * k + 1);
  float hx, hy, hz, lx, ly, lz;
  leaf_frame(x, box[0], scl, R.x, R.y, ix, hx, lx);
  leaf_frame(y, box[1], scl, R.x, R.y, iy, hy, ly);
  leaf_frame(z, box[2], scl, R.x, R.y, iz, hz, lz);
  pos32[r] = make_float4(hx, hy, hz, (float)qq);
  pos32lo[r] = make_float4(lx, ly, lz, 0.f);
}

// Problem of every cell of level l: the slot containing the cell's first
// leaf key, if the cell lies inside it (l >= S_k); -1 for cells above the slots.
__global__ void k_cell_slot(const int32_t* __restrict__ n_ptr, const uint32_t* __restrict__ key, int l, int Lf,
                            int nslot, const uint32_t* __restrict__ sstart, const int32_t* __restrict__ sprob,
                            const BatchProb* __restrict__ prob, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_ptr) return;
  const uint64_t kk = (uint64_t)key[i] << (3 * (Lf - l));
  const int j = last_le(sstart, nslot, kk);
  const int k = sprob[j];
  const BatchProb pb = prob[k];
  const bool inside = (uint64_t)sstart[j] <= kk && l >= pb.S && kk < (uint64_t)pb.slot_key + (1ull << (3 * pb.L));
  out[i] = inside ? k : -1;
}

// ---- tree levels and work lists from the sorted keys -------------------------------


// The dense grids of several levels in one launch: thread i belongs to
// level l with off[l] <= i < off[l + 1]; cell j = i - off[l] < n_l (n_l from
// counts[l] on the device, else nstatic[l]) sets grid_l[key_l[j]] to j, or
// to -1 when clearing the previous tree's entries.
struct GridSetAll {
  const uint32_t* key[FMM_MAX_LEVELS];
  int32_t* grid[FMM_MAX_LEVELS];
  int64_t off[FMM_MAX_LEVELS + 1];
  int64_t nstatic[FMM_MAX_LEVELS];
  const int32_t* counts;  // counters (cells of level l at [l]) or nullptr
  int nlev, clear;
};

__global__ void k_grid_set_all(GridSetAll a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.off[a.nlev]) return;
  int l = 0;
  while (l + 1 < a.nlev && i >= a.off[l + 1]) ++l;
  const int64_t j = i - a.off[l];
  const int64_t n = a.counts ? a.counts[l] : a.nstatic[l];
  if (j < n) a.grid[l][a.key[l][j]] = a.clear ? -1 : (int32_t)j;
}

// Every level of the tree from the sorted particle keys in three passes
// over the particles (in place of one unique pass per level).  Particle i
// opens a cell at level l when its key differs from particle i - 1's in the
// bits above 3 (Lf - l); that holds at every level from lmin(i) = Lf -
// floor(hb / 3) down to the leaves, hb the highest differing bit (lmin = 0
// for i = 0, none when the keys are equal).
//  1. k_lv_count: per block of LV_TILE particles, the cells it opens at
//     each level, level-major: sums[l * nb + b];
//  2. one exclusive scan of sums (per-level offsets are differences);
//  3. k_lv_write: each opening particle's cell index per level, with the
//     cell's key (key >> 3 (Lf - l)), first (the particle at the leaves, the
//     first child's index above), parent (the cell of the level above that
//     holds the particle), every particle's leaf (pleaf) and counters[l].
// k_lv_counts then derives the children (or particle) counts.  The results
// are those of a unique pass per level, the same cells in Morton order.
constexpr int LV_THREADS = 256;
constexpr int LV_ITEMS = 8;
constexpr int LV_TILE = LV_THREADS * LV_ITEMS;
constexpr int LV_WORDS = 3;  // 16-bit fields, 4 levels per word: up to 12 levels
static_assert(FMM_MAX_LEVELS <= 4 * LV_WORDS, "a field per level");

__device__ __forceinline__ int lv_open_level(const uint32_t* __restrict__ key, int64_t i, int Lf) {
  if (i == 0) return 0;
  const uint32_t d = key[i] ^ key[i - 1];
  if (d == 0) return Lf + 1;
  const int hb = 31 - __clz(d);
  const int l = Lf - hb / 3;
  return l < 0 ? 0 : l;
}

__global__ void __launch_bounds__(LV_THREADS)
k_lv_count(int64_t n, const uint32_t* __restrict__ key, int Lf, int32_t* __restrict__ sums) {
  __shared__ int cnt[FMM_MAX_LEVELS];
  if (threadIdx.x < FMM_MAX_LEVELS) cnt[threadIdx.x] = 0;
  __syncthreads();
  int c[FMM_MAX_LEVELS];
  for (int l = 0; l <= Lf; ++l) c[l] = 0;
  const int64_t i0 = (int64_t)blockIdx.x * LV_TILE;
  for (int k = threadIdx.x; k < LV_TILE; k += LV_THREADS) {
    const int64_t i = i0 + k;
    if (i >= n) break;
    const int lo = lv_open_level(key, i, Lf);
    for (int l = lo; l <= Lf; ++l) c[l]++;
  }
  for (int l = 0; l <= Lf; ++l) {
    int v = c[l];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cnt[l], v);
  }
  __syncthreads();
  if (threadIdx.x <= Lf) sums[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// LevelOut: the per-level arrays written by k_lv_write.
struct LevelOut {
  uint32_t* key[FMM_MAX_LEVELS];
  int32_t* first[FMM_MAX_LEVELS];
  int32_t* parent[FMM_MAX_LEVELS];
};

__global__ void __launch_bounds__(LV_THREADS)
k_lv_write(int64_t n, const uint32_t* __restrict__ key, int Lf, const int32_t* __restrict__ sums,
           const int32_t* __restrict__ total, LevelOut out, int32_t* __restrict__ pleaf, int32_t* __restrict__ counters) {
  __shared__ unsigned long long ws[LV_THREADS / 32];
  __shared__ int base[FMM_MAX_LEVELS];
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  if (tid <= Lf) {
    const int s0 = sums[(int64_t)tid * nb];
    base[tid] = sums[(int64_t)tid * nb + b] - s0;
    if (b == 0) counters[tid] = (tid < Lf ? sums[(int64_t)(tid + 1) * nb] : *total) - s0;
  }
  // this thread's particles and the level at which each opens cells
  const int64_t i0 = (int64_t)b * LV_TILE + (int64_t)tid * LV_ITEMS;
  int lo[LV_ITEMS];
  unsigned long long w[LV_WORDS] = {0ull, 0ull, 0ull};
#pragma unroll
  for (int j = 0; j < LV_ITEMS; ++j) {
    const int64_t i = i0 + j;
    lo[j] = i < n ? lv_open_level(key, i, Lf) : Lf + 1;
    for (int l = lo[j]; l <= Lf; ++l) w[l >> 2] += 1ull << (16 * (l & 3));
  }
  unsigned long long pre[LV_WORDS];
#pragma unroll
  for (int q = 0; q < LV_WORDS; ++q) {
    unsigned long long t;
    pre[q] = block_excl_scan<LV_THREADS>(w[q], ws, t);
  }
  // run[l]: cells of level l opened before this particle (a running index)
  int run[FMM_MAX_LEVELS];
  for (int l = 0; l <= Lf; ++l) run[l] = base[l] + (int)((pre[l >> 2] >> (16 * (l & 3))) & 0xffffull);
#pragma unroll
  for (int j = 0; j < LV_ITEMS; ++j) {
    const int64_t i = i0 + j;
    if (i >= n) break;
    const uint32_t k = key[i];
    for (int l = lo[j]; l <= Lf; ++l) ++run[l];  // run[l] - 1: the level-l cell holding i
    for (int l = Lf; l >= lo[j]; --l) {
      const int cell = run[l] - 1;
      if (!FMM_GUARD(cell >= 0, CHK_LEVEL_CELL, i)) continue;
      out.key[l][cell] = k >> (3 * (Lf - l));
      out.first[l][cell] = l == Lf ? (int32_t)i : run[l + 1] - 1;
      if (l >= 1) out.parent[l][cell] = run[l - 1] - 1;
    }
    pleaf[i] = run[Lf] - 1;
  }
}

// Children (particles at the leaves) per cell, every level in one launch:
// thread t belongs to level l with off[l] <= t < off[l + 1].
struct LevelCounts {
  const int32_t* first[FMM_MAX_LEVELS];
  int32_t* count[FMM_MAX_LEVELS];
  int64_t off[FMM_MAX_LEVELS + 1];
  int64_t n;
  int nlev;
};

__global__ void k_lv_counts(LevelCounts a, const int32_t* __restrict__ counters) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.off[a.nlev]) return;
  int l = 0;
  while (l + 1 < a.nlev && t >= a.off[l + 1]) ++l;
  const int64_t c = t - a.off[l];
  const int nc = counters[l];
  if (c >= nc) return;
  const int64_t e = c + 1 < nc ? a.first[l][c + 1] : (l + 1 == a.nlev ? a.n : counters[l + 1]);
  a.count[l][c] = (int32_t)(e - a.first[l][c]);
}

// The near field's work lists of the leaves (in place of k_p2p_items,
// k_item_leaf, k_unit_count, k_unit_write and their three scans, with the
// same results): per leaf T its first work item items[T] (one item per 32
// targets), the leaf of every item, the cooperative units of large leaves
// (more than P2P_BIG particles; up to P2P_UNIT items each) and the two
// bins' item lists.  Two 64-bit sums per leaf -- (items | units << 32) and
// (small items | large items << 32) -- are scanned: k_lw_count sums them per
// block of LW_TILE leaves, two scans of the block sums give the blocks'
// offsets and the totals (the 64-bit words at counters[CNT_ITEMS] and
// [CNT_BINS]), and k_lw_write scans inside each block and writes the lists.
constexpr int P2P_UNIT = 8;  // work items per cooperative unit (the near field's leaf-cooperative shapes)
constexpr int LW_THREADS = 256;
constexpr int LW_ITEMS = 4;
constexpr int LW_TILE = LW_THREADS * LW_ITEMS;

__device__ __forceinline__ void lw_leaf(const int32_t* __restrict__ count, int T, int nleaf, int& ni, bool& big,
                                        unsigned long long& iu, unsigned long long& sl) {
  const int cn = T < nleaf ? count[T] : 0;
  ni = (cn + 31) >> 5;
  big = cn > P2P_BIG;
  const unsigned long long nu = big ? (unsigned long long)((ni + P2P_UNIT - 1) / P2P_UNIT) : 0ull;
  iu = (unsigned long long)ni | (nu << 32);
  sl = big ? (unsigned long long)ni << 32 : (unsigned long long)ni;
}

__global__ void __launch_bounds__(LW_THREADS)
k_lw_count(const int32_t* __restrict__ nleaf_ptr, const int32_t* __restrict__ count,
           unsigned long long* __restrict__ sums) {
  const int nleaf = *nleaf_ptr, nb = gridDim.x;
  unsigned long long iu = 0, sl = 0;
  for (int k = threadIdx.x; k < LW_TILE; k += LW_THREADS) {
    const int T = blockIdx.x * LW_TILE + k;
    int ni;
    bool big;
    unsigned long long a, b;
    lw_leaf(count, T, nleaf, ni, big, a, b);
    iu += a;
    sl += b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    iu += __shfl_xor_sync(0xffffffffu, iu, o);
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
  }
  __shared__ unsigned long long w0[LW_THREADS / 32], w1[LW_THREADS / 32];
  if ((threadIdx.x & 31) == 0) {
    w0[threadIdx.x >> 5] = iu;
    w1[threadIdx.x >> 5] = sl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t0 = 0, t1 = 0;
    for (int q = 0; q < LW_THREADS / 32; ++q) {
      t0 += w0[q];
      t1 += w1[q];
    }
    sums[blockIdx.x] = t0;
    sums[nb + blockIdx.x] = t1;
  }
}

__global__ void __launch_bounds__(LW_THREADS)
k_lw_write(const int32_t* __restrict__ nleaf_ptr, const int32_t* __restrict__ count,
           const unsigned long long* __restrict__ sums, int32_t* __restrict__ items, int32_t* __restrict__ leaf_of,
           int32_t* __restrict__ units, int32_t* __restrict__ small, int32_t* __restrict__ large) {
  __shared__ unsigned long long ws[LW_THREADS / 32];
  const int nleaf = *nleaf_ptr, nb = gridDim.x;
  if (blockIdx.x * LW_TILE >= nleaf) return;  // the whole block (uniform)
  const int t0 = blockIdx.x * LW_TILE + threadIdx.x * LW_ITEMS;
  int ni[LW_ITEMS];
  bool big[LW_ITEMS];
  unsigned long long iu = 0, sl = 0;
#pragma unroll
  for (int j = 0; j < LW_ITEMS; ++j) {
    unsigned long long a, b;
    lw_leaf(count, t0 + j, nleaf, ni[j], big[j], a, b);
    iu += a;
    sl += b;
  }
  unsigned long long tt;
  unsigned long long piu = sums[blockIdx.x] + block_excl_scan<LW_THREADS>(iu, ws, tt);
  unsigned long long psl = sums[nb + blockIdx.x] + block_excl_scan<LW_THREADS>(sl, ws, tt);
#pragma unroll
  for (int j = 0; j < LW_ITEMS; ++j) {
    const int T = t0 + j;
    if (T >= nleaf) break;
    const int it = (int)(piu & 0xffffffffull), uo = (int)(piu >> 32);
    items[T] = it;
    for (int k = 0; k < ni[j]; ++k) leaf_of[it + k] = T;
    if (big[j]) {
      const int nu = (ni[j] + P2P_UNIT - 1) / P2P_UNIT;
      for (int k = 0; k < nu; ++k) units[uo + k] = it + k * P2P_UNIT;
      const int o = (int)(psl >> 32);
      for (int k = 0; k < ni[j]; ++k) large[o + k] = it + k;
      piu += (unsigned long long)ni[j] | ((unsigned long long)nu << 32);
      psl += (unsigned long long)ni[j] << 32;
    } else {
      const int o = (int)(psl & 0xffffffffull);
      for (int k = 0; k < ni[j]; ++k) small[o + k] = it + k;
      piu += (unsigned long long)ni[j];
      psl += (unsigned long long)ni[j];
    }
  }
}

struct ClassArgs {
  uint32_t* key[FMM_MAX_LEVELS];
  int32_t* out[FMM_MAX_LEVELS];
};

// Groups the cells of every level l >= 2 by child class (key & 7), keeping
// Morton order inside each class (the M2L tiles are runs of one class).  The
// cells of each level go in chunks of CP_CHUNK; (1) per chunk the count
// of each class, laid out per level as [class][chunk] behind the previous
// levels; (2) one exclusive scan over all of it; (3) per chunk a stable
// scatter: a cell's position is its level's class offset + the counts of
// its class in earlier chunks + its rank among the chunk's cells of its class.
constexpr int CP_THREADS = 256;
constexpr int CP_ITEMS = 8;
constexpr int CP_CHUNK = CP_THREADS * CP_ITEMS;

struct ClassChunks {
  int lmin, nlev;
  int blk0[FMM_MAX_LEVELS + 1];  // first block of each level (from lmin), and the total
  int seg0[FMM_MAX_LEVELS + 1];  // first count of each level in the scanned array, and its length
};

__device__ inline int cp_level(const ClassChunks& a, int b) {
  int k = 0;
  while (k + 1 < a.nlev && a.blk0[k + 1] <= b) ++k;
  return k;
}

__global__ void __launch_bounds__(CP_THREADS)
k_cls_count(ClassChunks a, const int32_t* __restrict__ counters, ClassArgs ca, int32_t* __restrict__ cnt) {
  const int k = cp_level(a, blockIdx.x), l = a.lmin + k;
  const int nb = a.blk0[k + 1] - a.blk0[k], bl = blockIdx.x - a.blk0[k];
  const int n = counters[l];
  const uint32_t* key = ca.key[l];
  int c8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int j = threadIdx.x; j < CP_CHUNK; j += CP_THREADS) {
    const int i = bl * CP_CHUNK + j;
    if (i < n) c8[key[i] & 7]++;
  }
  __shared__ int ws[8][CP_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < 8; ++c) {
    int v = c8[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[c][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    int t = 0;
    for (int j = 0; j < CP_THREADS / 32; ++j) t += ws[threadIdx.x][j];
    cnt[a.seg0[k] + threadIdx.x * nb + bl] = t;
  }
}

__global__ void __launch_bounds__(CP_THREADS)
k_cls_scatter(ClassChunks a, int32_t* __restrict__ counters, ClassArgs ca, const int32_t* __restrict__ off) {
  const int k = cp_level(a, blockIdx.x), l = a.lmin + k;
  const int nb = a.blk0[k + 1] - a.blk0[k], bl = blockIdx.x - a.blk0[k];
  const int n = counters[l];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  __shared__ uint8_t scls[CP_CHUNK];
  __shared__ int pre[8][CP_THREADS];
  __shared__ int base[8];
  const uint32_t* key = ca.key[l];
  for (int j = tid; j < CP_CHUNK; j += CP_THREADS) {
    const int i = bl * CP_CHUNK + j;
    scls[j] = i < n ? (uint8_t)(key[i] & 7) : (uint8_t)8;
  }
  if (tid < 8) {
    const int level0 = off[a.seg0[k]];  // the scanned array restarts per level at this value
    base[tid] = off[a.seg0[k] + tid * nb + bl] - level0;
    if (bl == 0) {
      const int end = tid < 7 ? off[a.seg0[k] + (tid + 1) * nb] : off[a.seg0[k + 1]];
      counters[CNT_CLS + 8 * l + tid] = end - off[a.seg0[k] + tid * nb];
    }
  }
  __syncthreads();
  int c8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int j = 0; j < CP_ITEMS; ++j) {
    const int c = scls[tid * CP_ITEMS + j];
    if (c < 8) c8[c]++;
  }
  for (int c = 0; c < 8; ++c) pre[c][tid] = c8[c];
  __syncthreads();
  // warp c scans class c over the threads (8 values per lane)
  if (w < 8) {
    int* row = pre[w];
    int v[CP_THREADS / 32], sum = 0;
    for (int j = 0; j < CP_THREADS / 32; ++j) {
      v[j] = row[lane * (CP_THREADS / 32) + j];
      sum += v[j];
    }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    int run = incl - sum;
    for (int j = 0; j < CP_THREADS / 32; ++j) {
      row[lane * (CP_THREADS / 32) + j] = run;
      run += v[j];
    }
  }
  __syncthreads();
  int pos[8];
  for (int c = 0; c < 8; ++c) pos[c] = base[c] + pre[c][tid];
  int32_t* out = ca.out[l];
  for (int j = 0; j < CP_ITEMS; ++j) {
    const int c = scls[tid * CP_ITEMS + j];
    if (c < 8) out[pos[c]++] = bl * CP_CHUNK + tid * CP_ITEMS + j;
  }
}

// The ordered list of the set bits of a 189-bit mask (transfer vectors with
// at least one pair): thread k < 189 writes k at its rank among the set bits.
__device__ inline void mask_to_list(const uint32_t* mask, int k, int16_t* out, int32_t* count) {
  if (k < FMM_NT_CLASS && ((mask[k >> 5] >> (k & 31)) & 1u)) {
    int pos = __popc(mask[k >> 5] & ((1u << (k & 31)) - 1u));
    for (int w = 0; w < (k >> 5); ++w) pos += __popc(mask[w]);
    out[pos] = (int16_t)k;
  }
  if (k == 0) {
    int n = 0;
    for (int w = 0; w < (FMM_NT_CLASS + 31) / 32; ++w) n += __popc(mask[w]);
    *count = n;
  }
}

constexpr int SETUP_BATCH = 7;  // 189 = 27 x 7 independent grid lookups in flight per thread
static_assert(FMM_NT_CLASS % SETUP_BATCH == 0, "setup batches cover the transfer vectors");

// Per M2L tile and each of the class's 189 transfer vectors t: as targets,
// the source cell S = T + t of every target row (the level's zero row when
// the source is absent, outside the cube or in another problem) and whether
// any row has one; as sources, whether any cell S of the tile has a target
// T = S - t in the tree (the class's source list src_t).  Block (tile,
// chunk, side) looks up SETUP_SPLIT_K transfer vectors for the tile's 128
// rows in batches of independent loads, a warp ballot per transfer vector
// sets the block's bits, and the block ORs them into the tile's mask in
// global memory (zero at launch); k_m2l_setup_lists turns the masks into
// the ordered lists of active transfer vectors.
constexpr int SETUP_SPLIT_K = 3 * SETUP_BATCH;
constexpr int SETUP_SPLIT = FMM_NT_CLASS / SETUP_SPLIT_K;
constexpr int SETUP_WORDS = (FMM_NT_CLASS + 31) / 32;
static_assert(FMM_NT_CLASS % SETUP_SPLIT_K == 0, "setup chunks cover the transfer vectors");

__global__ void __launch_bounds__(FMM_TILE)
k_m2l_setup_split(const Tile* __restrict__ tiles, LevelPtrs lv, const int16_t* __restrict__ cls_t,
                  const int16_t* __restrict__ src_t, const int8_t* __restrict__ tvec, int32_t* __restrict__ tile_src,
                  uint32_t* __restrict__ masks) {
  const Tile tl = tiles[blockIdx.x];
  const int side = blockIdx.z, kb = blockIdx.y * SETUP_SPLIT_K;
  const int l = tl.level, row = threadIdx.x, lane = row & 31;
  const bool valid = row < tl.count;
  const int zero_row = lv.ncell[l];
  int ix = 0, iy = 0, iz = 0, mine = 0;
  uint32_t key = 0;
  if (valid) {
    const int cell = lv.cls[l][tl.first + row];
    key = lv.key[l][cell];
    demorton3(key, ix, iy, iz);
    mine = problem_of(lv, l, cell);
  }
  const int top = (1 << l) - 1;
  const int sgn = side == 0 ? 1 : -1;  // targets look at S = T + t, sources at T = S - t
  const int16_t* list = side == 0 ? cls_t : src_t;
  // the chunk's offsets (with the side's sign) and each one's |component|
  // spread to its axis's bits of a Morton key, so that the neighbour's key
  // is the cell's key plus the offset in dilated arithmetic (per axis:
  // ((key | ~mask) + d) & mask upwards, ((key & mask) - d) & mask downwards)
  __shared__ int8_t s_t[SETUP_SPLIT_K][3];
  __shared__ uint32_t s_d[SETUP_SPLIT_K][3];
  __shared__ uint32_t mask[SETUP_WORDS];
  if (row < SETUP_WORDS) mask[row] = 0u;
  if (row < SETUP_SPLIT_K) {
    const int slot = list[tl.cls * FMM_NT_CLASS + kb + row];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int t = sgn * tvec[3 * slot + a];
      s_t[row][a] = (int8_t)t;
      s_d[row][a] = spread3((uint32_t)(t < 0 ? -t : t)) << (2 - a);
    }
  }
  __syncthreads();
  int32_t* out = tile_src + (int64_t)blockIdx.x * FMM_NT_CLASS * FMM_TILE + row;
  constexpr uint32_t MASK[3] = {0x24924924u, 0x12492492u, 0x09249249u};  // x, y, z bits of a key
  for (int k0 = kb; k0 < kb + SETUP_SPLIT_K; k0 += SETUP_BATCH) {
    int g[SETUP_BATCH];
#pragma unroll
    for (int j = 0; j < SETUP_BATCH; ++j) {
      const int k = k0 + j - kb;
      const int tx = s_t[k][0], ty = s_t[k][1], tz = s_t[k][2];
      const int sx = ix + tx, sy = iy + ty, sz = iz + tz;
      uint32_t skey = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int t = a == 0 ? tx : (a == 1 ? ty : tz);
        const uint32_t d = s_d[k][a];
        skey |= t < 0 ? ((key & MASK[a]) - d) & MASK[a] : ((key | ~MASK[a]) + d) & MASK[a];
      }
      const bool inside = valid && sx >= 0 && sy >= 0 && sz >= 0 && sx <= top && sy <= top && sz <= top;
      g[j] = (inside && FMM_GUARD(skey < (1u << (3 * l)), CHK_SETUP_KEY, skey)) ? lv.grid[l][skey] : -1;
    }
#pragma unroll
    for (int j = 0; j < SETUP_BATCH; ++j) {
      const bool has = g[j] >= 0 && same_problem(lv, l, mine, g[j]);
      if (side == 0) out[(int64_t)(k0 + j) * FMM_TILE] = has ? g[j] : zero_row;
      const uint32_t any = __ballot_sync(0xffffffffu, has);
      if (lane == 0 && any) atomicOr(&mask[(k0 + j) >> 5], 1u << ((k0 + j) & 31));
    }
  }
  __syncthreads();
  if (row < SETUP_WORDS && mask[row])
    atomicOr(&masks[((int64_t)side * gridDim.x + blockIdx.x) * SETUP_WORDS + row], mask[row]);
}

__global__ void __launch_bounds__(2 * FMM_TILE)
k_m2l_setup_lists(const uint32_t* __restrict__ masks, int ntiles, int16_t* __restrict__ tile_act,
                  int32_t* __restrict__ tile_nact, int16_t* __restrict__ src_act, int32_t* __restrict__ src_nact) {
  const int side = blockIdx.y;
  __shared__ uint32_t mask[SETUP_WORDS];
  if (threadIdx.x < SETUP_WORDS)
    mask[threadIdx.x] = masks[((int64_t)side * ntiles + blockIdx.x) * SETUP_WORDS + threadIdx.x];
  __syncthreads();
  if (side == 0)
    mask_to_list(mask, threadIdx.x, tile_act + (int64_t)blockIdx.x * FMM_NT_CLASS, tile_nact + blockIdx.x);
  else
    mask_to_list(mask, threadIdx.x, src_act + (int64_t)blockIdx.x * FMM_NT_CLASS, src_nact + blockIdx.x);
}

__global__ void k_zero_rows(int nrows, const int64_t* __restrict__ rows, int cpad, float* a, float* b,
                            float* c, double* d, double* e) {
  int r = blockIdx.x;
  if (r >= nrows) return;
  int64_t o = rows[r] * cpad;
  for (int k = threadIdx.x; k < cpad; k += blockDim.x) {
    if (a) a[o + k] = 0.f;
    if (b) b[o + k] = 0.f;
    if (c) c[o + k] = 0.f;
    if (d) d[o + k] = 0.0;
    if (e) e[o + k] = 0.0;
  }
}

int64_t pow8(int l) { return (int64_t)1 << (3 * l); }

fmm_status ensure_particles(Ctx* c, int64_t n) {
  if (n <= c->ncap) return FMM_OK;
  int64_t cap = n + n / 8 + 1024;
  void* p;
#define REALLOC(field, T, count)                                  \
  dfree(c, c->field, sizeof(T) * (size_t)c->ncap * (count));      \
  c->field = nullptr;                                             \
  FMM_TRY(dalloc(c, &p, sizeof(T) * (size_t)cap * (count)));      \
  c->field = (decltype(c->field))p;
  REALLOC(key_a, uint32_t, 1)
  REALLOC(key_b, uint32_t, 1)
  REALLOC(idx_a, uint32_t, 1)
  REALLOC(idx_b, uint32_t, 1)
  REALLOC(perm, int32_t, 1)
  REALLOC(pleaf, int32_t, 1)
  REALLOC(pos64, double4, 1)
  REALLOC(pos32, float4, 1)
  REALLOC(pos32lo, float4, 1)
  REALLOC(near32, float4, 1)
  REALLOC(near64, double4, 1)
#undef REALLOC
  c->ncap = cap;
  int64_t words = 65536 + cap / 8 + 4096;
  if (words > c->scratch_cap) {
    dfree(c, c->scratch, sizeof(uint32_t) * (size_t)c->scratch_cap);
    c->scratch = nullptr;
    FMM_TRY(dalloc(c, &p, sizeof(uint32_t) * (size_t)words));
    c->scratch = (uint32_t*)p;
    c->scratch_cap = words;
  }
  return FMM_OK;
}

fmm_status ensure_level(Ctx* c, int l, int64_t cells) {
  if (cells <= c->lcap[l]) return FMM_OK;
  int64_t cap = cells + cells / 8 + 64;
  int64_t old = c->lcap[l];
  void* p;
  dfree(c, c->lv.key[l], 4 * (size_t)old);
  dfree(c, c->lv.first[l], 4 * (size_t)old);
  dfree(c, c->lv.count[l], 4 * (size_t)old);
  dfree(c, c->lv.parent[l], 4 * (size_t)old);
  dfree(c, c->lv.cls[l], 4 * (size_t)old);
  dfree(c, c->slot_buf[l], 4 * (size_t)old);
  c->lv.key[l] = nullptr;
  c->lv.first[l] = c->lv.count[l] = c->lv.parent[l] = c->lv.cls[l] = nullptr;
  c->slot_buf[l] = c->lv.slot[l] = nullptr;
  FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
  c->lv.key[l] = (uint32_t*)p;
  FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
  c->lv.first[l] = (int32_t*)p;
  FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
  c->lv.count[l] = (int32_t*)p;
  FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
  c->lv.parent[l] = (int32_t*)p;
  FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
  c->lv.cls[l] = (int32_t*)p;
  FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
  c->slot_buf[l] = (int32_t*)p;
  c->lcap[l] = cap;
  return FMM_OK;
}

// dense key -> cell grids of levels 0 .. Lf (all -1 when allocated)
fmm_status ensure_grids(Ctx* c, int Lf) {
  for (int l = 0; l <= Lf; ++l) {
    if (c->lv.grid[l]) continue;
    void* p;
    const size_t bytes = sizeof(int32_t) * ((size_t)1 << (3 * l));
    FMM_TRY(dalloc(c, &p, bytes));
    c->lv.grid[l] = (int32_t*)p;
    FMM_CUDA(c, cudaMemsetAsync(p, 0xFF, bytes, c->stream));
  }
  return FMM_OK;
}


}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free Morton ordering.
//
// For callers that cannot allocate device memory while they run: processes
// whose HBM is owned by a pool they reserved at start-up (a serving loop that
// must not stall in the driver's allocator, or a framework allocator that
// holds nearly all of the device), and plug-ins that only ever receive
// buffers from their host application.  This entry point computes what the
// front of fmm_set_particles computes -- the root cube, the leaf-level Morton
// keys and the stable sort -- with every intermediate in one fixed array
// compiled into the library, so it never calls cudaMalloc or cudaFree.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 4.3 MB) until the process exits, and every call on
// that GPU reuses it.  Calls whose work overlaps on the same GPU (different
// streams, or host threads) therefore race on it and must be serialised by
// the caller.  Host code cannot use the variable's name as a device address;
// the first call on each device looks the address up (cudaGetSymbolAddress)
// with that device current and caches it, so make that first call before any
// stream capture.
namespace {

constexpr int64_t NOALLOC_MAX_N = (int64_t)1 << 18;
constexpr int64_t NOALLOC_TILES = (NOALLOC_MAX_N + RS_TILE - 1) / RS_TILE;
constexpr int NOALLOC_BBOX_BLOCKS = 128;
// word offsets inside the array
constexpr int64_t NA_KEY_A = 0;
constexpr int64_t NA_KEY_B = NA_KEY_A + NOALLOC_MAX_N;
constexpr int64_t NA_IDX_A = NA_KEY_B + NOALLOC_MAX_N;
constexpr int64_t NA_IDX_B = NA_IDX_A + NOALLOC_MAX_N;
constexpr int64_t NA_HIST = NA_IDX_B + NOALLOC_MAX_N;
constexpr int64_t NA_PART = NA_HIST + 256 * NOALLOC_TILES;          // doubles: 8-byte aligned
constexpr int64_t NA_BOX = NA_PART + 2 * 6 * NOALLOC_BBOX_BLOCKS;   // 8 doubles
constexpr int64_t NA_THR = NA_BOX + 2 * 8;                          // 3 << (FMM_MAX_LEVELS - 1) int64
constexpr int64_t NA_COUNTERS = NA_THR + 2 * (3 << (FMM_MAX_LEVELS - 1));  // 128 int32
constexpr int64_t NA_WORDS = NA_COUNTERS + 128;

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

__global__ void k_noalloc_out(int64_t n, const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sidx,
                              uint64_t* __restrict__ keys, int64_t* __restrict__ perm) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  keys[r] = skey[r];
  perm[r] = sidx[r];
}

}  // namespace
}  // namespace fmm

extern "C" fmm_status fmm_morton_order_noalloc(int64_t n, const double* xyz, int height, uint64_t* keys,
                                               int64_t* perm, void* stream) {
  using namespace fmm;
  if (height < 1 || height > FMM_MAX_LEVELS)
    return set_err(nullptr, FMM_ERR_ARG, "fmm_morton_order_noalloc: height %d outside 1..%d", height,
                   FMM_MAX_LEVELS);
  if (n < 0 || n > NOALLOC_MAX_N)
    return set_err(nullptr, FMM_ERR_ARG,
                   "fmm_morton_order_noalloc: n = %lld outside 0..%lld (the fixed scratch array holds %lld points)",
                   (long long)n, (long long)NOALLOC_MAX_N, (long long)NOALLOC_MAX_N);
  if (n == 0) return FMM_OK;
  if (!xyz || !keys || !perm) return set_err(nullptr, FMM_ERR_ARG, "fmm_morton_order_noalloc: NULL pointer");
  // The array's device address on the current device, looked up on every
  // call (a host-side query, no device work): in host code the symbol is a
  // host-side stand-in, and a cached address would go stale after the
  // caller resets the device.
  uint32_t* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&base, g_noalloc_scratch);
  if (e != cudaSuccess || !base) {
    cudaGetLastError();
    return set_err(nullptr, FMM_ERR_CUDA, "fmm_morton_order_noalloc: cudaGetSymbolAddress: %s",
                   cudaGetErrorString(e));
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *ka = base + NA_KEY_A, *kb = base + NA_KEY_B, *va = base + NA_IDX_A, *vb = base + NA_IDX_B;
  uint32_t* hist = base + NA_HIST;
  double* part = (double*)(base + NA_PART);
  double* box = (double*)(base + NA_BOX);
  int64_t* thr = (int64_t*)(base + NA_THR);
  int32_t* counters = (int32_t*)(base + NA_COUNTERS);
  const int Lf = height - 1;
  // the array keeps the previous call's contents: clear the input-error flag
  e = cudaMemsetAsync(counters, 0, 128 * sizeof(int32_t), s);
  int nbb = ceil_div(n, BB_THREADS * 8);
  if (nbb > NOALLOC_BBOX_BLOCKS) nbb = NOALLOC_BBOX_BLOCKS;
  // positions only: the charge check of the cube kernel re-reads coordinates
  if (e == cudaSuccess) {
    k_bbox_partial<<<nbb, BB_THREADS, 0, s>>>(n, xyz, xyz, part, counters);
    launch_cube_keys(s, n, xyz, nbb, part, box, thr, Lf, ka, va);
    const int ntiles = ceil_div(n, RS_TILE);
    for (int sh = 0; sh < 3 * Lf; sh += 8) {
      k_radix_hist<<<ntiles, RS_THREADS, 0, s>>>(n, ka, sh, hist, ntiles);
      k_scan1<uint32_t><<<1, 1024, 0, s>>>(hist, (int64_t)256 * ntiles, nullptr);
      k_radix_scatter<<<ntiles, RS_THREADS, 0, s>>>(n, ka, va, kb, vb, sh, hist, ntiles);
      uint32_t* tmp = ka;
      ka = kb;
      kb = tmp;
      tmp = va;
      va = vb;
      vb = tmp;
    }
    k_noalloc_out<<<ceil_div(n, 256), 256, 0, s>>>(n, ka, va, keys, perm);
    e = cudaGetLastError();
  }
  int32_t bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, counters + CNT_BAD, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, FMM_ERR_CUDA, "fmm_morton_order_noalloc: %s", cudaGetErrorString(e));
  }
  if (bad) return set_err(nullptr, FMM_ERR_ARG, "fmm_morton_order_noalloc: non-finite coordinate");
  return FMM_OK;
}

namespace fmm {

// Slots of a batch: problems with particles, largest slot first (ties in input
// order), take consecutive ranges of forest leaf keys; a slot of 8^L keys then
// starts at a multiple of 8^L, i.e. it is one cell of level Lf - L.  The forest
// leaf level Lf is the smallest that holds every slot (and at least every
// problem's own leaf level).  Host only; returns -1 if the slots do not fit
// in 8^FMM_MAX_FOREST_LEAF keys.
int batch_plan(int nprob, const int64_t* counts, const int32_t* heights, int64_t* slot, int64_t* level, int* leaf) {
  std::vector<int> order;
  int maxL = 0;
  for (int k = 0; k < nprob; ++k) {
    slot[k] = -1;
    level[k] = -1;
    if (counts[k] > 0) {
      order.push_back(k);
      maxL = std::max(maxL, heights[k] - 1);
    }
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return heights[a] > heights[b]; });
  uint64_t off = 0;
  for (int k : order) {
    slot[k] = (int64_t)off;
    off += (uint64_t)1 << (3 * (heights[k] - 1));
    if (off > ((uint64_t)1 << (3 * FMM_MAX_FOREST_LEAF))) return -1;
  }
  int Lf = maxL;
  while (((uint64_t)1 << (3 * Lf)) < off) ++Lf;
  for (int k : order) level[k] = Lf - (heights[k] - 1);
  *leaf = Lf;
  return 0;
}
fmm_status batch_layout(Ctx* c, int nprob, const int64_t* counts, const int32_t* heights, int64_t* n_total) {
  std::vector<int64_t> start(nprob + 1, 0);
  std::vector<BatchProb> prob(nprob);
  std::vector<int> order;
  for (int k = 0; k < nprob; ++k) {
    start[k + 1] = start[k] + counts[k];
    prob[k] = BatchProb{0u, heights[k] - 1, 0, 0};
  }
  int64_t nthr = 0;  // cell thresholds: 3 << L per problem
  for (int k = 0; k < nprob; ++k) {
    prob[k].thr = (int32_t)nthr;
    nthr += (int64_t)3 << prob[k].L;
  }
  if (nthr > INT32_MAX) return set_err(c, FMM_ERR_ARG, "fmm_set_batch: too many problems in one batch");
  int Lf = 0;
  {
    std::vector<int64_t> slot(nprob), lev(nprob);
    if (batch_plan(nprob, counts, heights, slot.data(), lev.data(), &Lf) != 0)
      return set_err(c, FMM_ERR_ARG,
                     "fmm_set_batch: the problems' leaf cells (sum of 8^(height-1)) exceed 8^%d; split the batch",
                     FMM_MAX_FOREST_LEAF);
    for (int k = 0; k < nprob; ++k)
      if (counts[k] > 0) {
        prob[k].slot_key = (uint32_t)slot[k];
        order.push_back(k);
      }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return prob[a].slot_key < prob[b].slot_key; });
  }
  std::vector<uint32_t> sstart;
  std::vector<int32_t> sprob;
  std::vector<int64_t> first(nprob, 0);
  int64_t rank = 0;
  for (int k : order) {
    prob[k].S = Lf - prob[k].L;
    sstart.push_back(prob[k].slot_key);
    sprob.push_back(k);
    first[k] = rank;
    rank += counts[k];
  }
  for (int k = 0; k < nprob; ++k)
    if (counts[k] == 0) first[k] = rank;
  std::vector<int32_t> bstart(nprob + 1, 0);
  for (int k = 0; k < nprob; ++k)
    bstart[k + 1] = bstart[k] + (int32_t)((counts[k] + FB_CHUNK - 1) / FB_CHUNK);
  if (nprob + 1 > c->fb_cap) {
    dfree(c, c->fb_pstart, 8 * (size_t)c->fb_cap);
    dfree(c, c->fb_prob, sizeof(BatchProb) * (size_t)c->fb_cap);
    dfree(c, c->fb_box, 32 * (size_t)c->fb_cap);
    dfree(c, c->fb_scale, 8 * (size_t)c->fb_cap);
    dfree(c, c->fb_frame, 32 * (size_t)c->fb_cap);
    dfree(c, c->fb_sstart, 4 * (size_t)c->fb_cap);
    dfree(c, c->fb_sprob, 4 * (size_t)c->fb_cap);
    dfree(c, c->fb_bstart, 4 * (size_t)c->fb_cap);
    c->fb_pstart = nullptr;
    c->fb_prob = nullptr;
    c->fb_box = c->fb_scale = c->fb_frame = nullptr;
    c->fb_sstart = nullptr;
    c->fb_sprob = c->fb_bstart = nullptr;
    c->fb_cap = 0;
    const int cap = nprob + 1 + 64;
    void* p;
    FMM_TRY(dalloc(c, &p, 8 * (size_t)cap));
    c->fb_pstart = (int64_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(BatchProb) * (size_t)cap));
    c->fb_prob = (BatchProb*)p;
    FMM_TRY(dalloc(c, &p, 32 * (size_t)cap));
    c->fb_box = (double*)p;
    FMM_TRY(dalloc(c, &p, 8 * (size_t)cap));
    c->fb_scale = (double*)p;
    FMM_TRY(dalloc(c, &p, 32 * (size_t)cap));
    c->fb_frame = (double*)p;
    FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
    c->fb_sstart = (uint32_t*)p;
    FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
    c->fb_sprob = (int32_t*)p;
    FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
    c->fb_bstart = (int32_t*)p;
    c->fb_cap = cap;
  }
  if (nthr > c->fb_thr_cap) {
    dfree(c, c->fb_thr, 8 * (size_t)c->fb_thr_cap);
    c->fb_thr = nullptr;
    c->fb_thr_cap = 0;
    void* p;
    const int64_t cap = nthr + nthr / 4 + 64;
    FMM_TRY(dalloc(c, &p, 8 * (size_t)cap));
    c->fb_thr = (int64_t*)p;
    c->fb_thr_cap = cap;
  }
  // the tables are small; copies on the handle's stream, waited for, keep the
  // host vectors' lifetime simple (no legacy-stream operation)
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->fb_pstart, start.data(), 8 * (size_t)(nprob + 1), cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->fb_prob, prob.data(), sizeof(BatchProb) * (size_t)nprob, cudaMemcpyHostToDevice, c->stream));
  FMM_CUDA(c, cudaMemcpyAsync(c->fb_bstart, bstart.data(), 4 * (size_t)(nprob + 1), cudaMemcpyHostToDevice, c->stream));
  if (!sstart.empty()) {
    FMM_CUDA(c, cudaMemcpyAsync(c->fb_sstart, sstart.data(), 4 * sstart.size(), cudaMemcpyHostToDevice, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->fb_sprob, sprob.data(), 4 * sprob.size(), cudaMemcpyHostToDevice, c->stream));
  }
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->forest = true;
  c->nprob = nprob;
  c->leaf = Lf;
  c->fb_nslot = (int)sstart.size();
  c->fb_nblocks = bstart[nprob];
  c->fb_start_h = start;
  c->fb_prob_h = prob;
  c->fb_first_h = first;
  *n_total = start[nprob];
  return FMM_OK;
}

fmm_status ensure_expansions(Ctx* c, int precision) {
  const int64_t rows = c->rows;
  const size_t cp = (size_t)c->cpad;
  void* p;
  if (precision == FMM_MIXED && rows > c->rows_cap32) {
    dfree(c, c->Mhi, 4 * cp * c->rows_cap32);
    dfree(c, c->Mlo, 4 * cp * c->rows_cap32);
    dfree(c, c->L32, 4 * cp * c->rows_cap32);
    c->Mhi = c->Mlo = c->L32 = nullptr;
    c->rows_cap32 = 0;
    const int64_t cap = rows + rows / 8 + 16;
    FMM_TRY(dalloc(c, &p, 4 * cp * cap));
    c->Mhi = (float*)p;
    FMM_TRY(dalloc(c, &p, 4 * cp * cap));
    c->Mlo = (float*)p;
    FMM_TRY(dalloc(c, &p, 4 * cp * cap));
    c->L32 = (float*)p;
    FMM_CUDA(c, cudaMemsetAsync(c->Mhi, 0, 4 * cp * cap, c->stream));
    FMM_CUDA(c, cudaMemsetAsync(c->Mlo, 0, 4 * cp * cap, c->stream));
    FMM_CUDA(c, cudaMemsetAsync(c->L32, 0, 4 * cp * cap, c->stream));
    c->rows_cap32 = cap;
  }
  if (precision == FMM_FP64 && rows > c->rows_cap64) {
    dfree(c, c->M64, 8 * cp * c->rows_cap64);
    dfree(c, c->L64, 8 * cp * c->rows_cap64);
    c->M64 = c->L64 = nullptr;
    c->rows_cap64 = 0;
    const int64_t cap = rows + rows / 8 + 16;
    FMM_TRY(dalloc(c, &p, 8 * cp * cap));
    c->M64 = (double*)p;
    FMM_TRY(dalloc(c, &p, 8 * cp * cap));
    c->L64 = (double*)p;
    FMM_CUDA(c, cudaMemsetAsync(c->M64, 0, 8 * cp * cap, c->stream));
    FMM_CUDA(c, cudaMemsetAsync(c->L64, 0, 8 * cp * cap, c->stream));
    c->rows_cap64 = cap;
  }
  return FMM_OK;
}

void release_tree(Ctx* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  auto rel = [&](auto*& ptr, size_t bytes) {
    dfree(c, (void*)ptr, bytes);
    ptr = nullptr;
  };
  const size_t nc = (size_t)c->ncap;
  rel(c->key_a, 4 * nc);
  rel(c->key_b, 4 * nc);
  rel(c->idx_a, 4 * nc);
  rel(c->idx_b, 4 * nc);
  rel(c->perm, 4 * nc);
  rel(c->pleaf, 4 * nc);
  rel(c->pos64, 32 * nc);
  rel(c->pos32, 16 * nc);
  rel(c->pos32lo, 16 * nc);
  rel(c->near32, 16 * nc);
  rel(c->near64, 32 * nc);
  c->skey = nullptr;
  c->ncap = 0;
  rel(c->scratch, 4 * (size_t)c->scratch_cap);
  c->scratch_cap = 0;
  rel(c->p2p_items, 4 * (size_t)c->p2p_items_cap);
  c->p2p_items_cap = 0;
  rel(c->p2p_leaf, 4 * (size_t)c->p2p_leaf_cap);
  c->p2p_leaf_cap = 0;
  rel(c->p2p_units, 4 * (size_t)c->p2p_units_cap);
  rel(c->p2p_small, 4 * (size_t)c->p2p_units_cap);
  rel(c->p2p_large, 4 * (size_t)c->p2p_units_cap);
  c->p2p_units_cap = 0;
  c->p2p_nunits = 0;
  c->p2p_nitems = 0;
  c->p2p_nsmall = c->p2p_nlarge = 0;
  rel(c->stage_in, 8 * (size_t)c->stage_in_cap);
  rel(c->stage_out, 8 * (size_t)c->stage_out_cap);
  c->stage_in_cap = c->stage_out_cap = 0;
  rel(c->stokes_buf, 8 * (size_t)c->stokes_cap);
  c->stokes_cap = 0;
  for (int l = 0; l < FMM_MAX_LEVELS; ++l) {
    const size_t lc = 4 * (size_t)c->lcap[l];
    rel(c->lv.key[l], lc);
    rel(c->lv.first[l], lc);
    rel(c->lv.count[l], lc);
    rel(c->lv.parent[l], lc);
    rel(c->lv.cls[l], lc);
    rel(c->slot_buf[l], lc);
    c->lv.slot[l] = nullptr;
    c->lcap[l] = 0;
    rel(c->lv.grid[l], sizeof(int32_t) * ((size_t)1 << (3 * l)));
    c->lv.ncell[l] = 0;
    c->prev_ncell[l] = 0;
  }
  c->have_prev = false;
  c->prev_leaf = -1;
  const size_t cp = (size_t)c->cpad;
  rel(c->Mhi, 4 * cp * c->rows_cap32);
  rel(c->Mlo, 4 * cp * c->rows_cap32);
  rel(c->L32, 4 * cp * c->rows_cap32);
  rel(c->M64, 8 * cp * c->rows_cap64);
  rel(c->L64, 8 * cp * c->rows_cap64);
  c->rows_cap32 = c->rows_cap64 = 0;
  c->rows = 0;
  const size_t tc = (size_t)c->tiles_cap;
  rel(c->tiles, sizeof(Tile) * tc);
  rel(c->tile_src, sizeof(int32_t) * tc * FMM_NT_CLASS * FMM_TILE);
  rel(c->tile_act, sizeof(int16_t) * tc * FMM_NT_CLASS);
  rel(c->tile_nact, sizeof(int32_t) * tc);
  rel(c->src_act, sizeof(int16_t) * tc * FMM_NT_CLASS);
  rel(c->src_nact, sizeof(int32_t) * tc);
  rel(c->tile_mask, sizeof(uint32_t) * 2 * SETUP_WORDS * tc);
  c->tiles_cap = 0;
  c->ntiles = c->leaf_tiles = 0;
  c->tiles_h.clear();
  rel(c->tc_partial, 4 * (size_t)c->tc_partial_cap);
  c->tc_partial_cap = 0;
  dfree(c, c->svd_Y, c->svd_Y_cap);
  c->svd_Y = nullptr;
  c->svd_Y_cap = 0;
  dfree(c, c->svd_Yx, c->svd_Yx_cap);
  c->svd_Yx = nullptr;
  c->svd_Yx_cap = 0;
  dfree(c, c->svd_dst, c->svd_dst_cap);
  c->svd_dst = nullptr;
  c->svd_dst_cap = 0;
  dfree(c, c->svd_recs, 128 * (size_t)c->svd_gcap);
  c->svd_recs = nullptr;
  c->svd_gcap = 0;
  const size_t ec = (size_t)c->svd_ecap;
  rel(c->svd_eslot, sizeof(int16_t) * ec * FMM_NT_CLASS);
  rel(c->svd_ekch, sizeof(int8_t) * ec * FMM_NT_CLASS);
  rel(c->svd_yidx, sizeof(int64_t) * ec * FMM_NT_CLASS * FMM_TILE);
  c->svd_ecap = 0;
  rel(c->svd_Mcls, 8 * (size_t)c->svd_mcls_rows * cp);
  c->svd_mcls_rows = 0;
  c->loaded = false;
  c->forest = false;
  c->n = 0;
  c->tree_gen++;
}

fmm_status tree_build(Ctx* c, int64_t n, const double* xyz, const double* q) {
  cudaStream_t s = c->stream;
  const int Lf = c->leaf;
  c->launches_set = 0;
  c->loaded = false;
  FMM_TRY(ensure_particles(c, n > 0 ? n : 1));

  // forget the previous tree in the dense grids (every level in one launch)
  if (c->have_prev) {
    GridSetAll ga{};
    ga.nlev = c->prev_leaf + 1;
    ga.clear = 1;
    ga.off[0] = 0;
    for (int l = 0; l < ga.nlev; ++l) {
      ga.key[l] = c->lv.key[l];
      ga.grid[l] = c->lv.grid[l];
      ga.nstatic[l] = c->prev_ncell[l];
      ga.off[l + 1] = ga.off[l] + c->prev_ncell[l];
    }
    if (ga.off[ga.nlev] > 0) {
      k_grid_set_all<<<ceil_div(ga.off[ga.nlev], 256), 256, 0, s>>>(ga);
      c->launches_set++;
    }
    c->have_prev = false;
  }
  c->prev_leaf = Lf;
  for (int l = 0; l < FMM_MAX_LEVELS; ++l) c->prev_ncell[l] = 0;
  FMM_TRY(ensure_grids(c, Lf));
  FMM_CUDA(c, cudaMemsetAsync(c->counters, 0, 128 * sizeof(int32_t), s));

  // per-level capacities from upper bounds
  int64_t ub[FMM_MAX_LEVELS];
  for (int l = Lf; l >= 0; --l) {
    int64_t b = (l == Lf) ? n : ub[l + 1];
    ub[l] = b < pow8(l) ? b : pow8(l);
    FMM_TRY(ensure_level(c, l, ub[l] > 0 ? ub[l] : 1));
  }
  if (ub[Lf] + 1 > c->p2p_items_cap) {
    dfree(c, c->p2p_items, 4 * (size_t)c->p2p_items_cap);
    c->p2p_items = nullptr;
    c->p2p_items_cap = 0;
    void* p;
    const int64_t cap = ub[Lf] + ub[Lf] / 8 + 64;
    FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
    c->p2p_items = (int32_t*)p;
    c->p2p_items_cap = cap;
  }
  {
    // items: at most one per leaf plus one per 32 particles
    const int64_t need = ub[Lf] + n / 32 + 2;
    if (need > c->p2p_leaf_cap) {
      dfree(c, c->p2p_leaf, 4 * (size_t)c->p2p_leaf_cap);
      c->p2p_leaf = nullptr;
      c->p2p_leaf_cap = 0;
      void* p;
      const int64_t cap = need + need / 8 + 64;
      FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
      c->p2p_leaf = (int32_t*)p;
      c->p2p_leaf_cap = cap;
    }
    // units: at most one per leaf plus one per 8 items; the bins' item
    // lists: at most all items
    if (need > c->p2p_units_cap) {
      dfree(c, c->p2p_units, 4 * (size_t)c->p2p_units_cap);
      dfree(c, c->p2p_small, 4 * (size_t)c->p2p_units_cap);
      dfree(c, c->p2p_large, 4 * (size_t)c->p2p_units_cap);
      c->p2p_units = c->p2p_small = c->p2p_large = nullptr;
      c->p2p_units_cap = 0;
      void* p;
      const int64_t cap = need + need / 8 + 64;
      FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
      c->p2p_units = (int32_t*)p;
      FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
      c->p2p_small = (int32_t*)p;
      FMM_TRY(dalloc(c, &p, 4 * (size_t)cap));
      c->p2p_large = (int32_t*)p;
      c->p2p_units_cap = cap;
    }
  }

  if (n > 0 && c->forest) {
    // bounding cube of every problem, then forest keys
    const int nbb = c->fb_nblocks;
    double* part = (double*)c->scratch;
    k_fbox_partial<<<nbb, BB_THREADS, 0, s>>>(c->nprob, c->fb_bstart, c->fb_pstart, xyz, q, part, c->counters);
    k_fbox_final<<<c->nprob, 256, 0, s>>>(c->fb_bstart, part, c->fb_prob, c->fb_box, c->fb_scale, c->fb_frame,
                                          c->fb_thr);
    k_fmorton<<<ceil_div(n, 256), 256, 0, s>>>(n, c->nprob, c->fb_pstart, c->fb_prob, c->fb_thr, xyz, c->key_a,
                                               c->idx_a);
    // the forest cube itself is the unit cube at the origin
    // (and its leaf constants as k_bbox_final writes them: 2^-e = 1,
    // 2^Lf / m = 2^Lf exactly, 1 / half-width = 2^(Lf + 1))
    c->box_h[0] = c->box_h[1] = c->box_h[2] = 0.0;
    c->box_h[3] = 1.0;
    c->box_h[4] = 1.0;
    const float R2[2] = {(float)(1u << Lf), 0.f};
    memcpy(c->box_h + 5, R2, sizeof(R2));
    c->box_h[6] = (double)(2u << Lf);
    c->box_h[7] = 0.0;
    FMM_CUDA(c, cudaMemcpyAsync(c->box, c->box_h, 8 * sizeof(double), cudaMemcpyHostToDevice, s));
    c->launches_set += 3;
  } else if (n > 0) {
    // bounding cube
    int nbb = ceil_div(n, BB_THREADS * 8);
    if (nbb > 1184) nbb = 1184;
    double* part = (double*)c->scratch;
    k_bbox_partial<<<nbb, BB_THREADS, 0, s>>>(n, xyz, q, part, c->counters);
    // cube, leaf frame, cell thresholds (scratch words 32768.., past the partials) and keys
    launch_cube_keys(s, n, xyz, nbb, part, c->box, (int64_t*)(c->scratch + 32768), Lf, c->key_a, c->idx_a);
    c->launches_set += 3;
  }
  if (n > 0) {
    // sort
    uint32_t *ka = c->key_a, *kb = c->key_b, *va = c->idx_a, *vb = c->idx_b;
    int bits = 3 * Lf;
    int ntiles = ceil_div(n, RS_TILE);
    uint32_t* hist = c->scratch;
    for (int sh = 0; sh < bits; sh += 8) {
      k_radix_hist<<<ntiles, RS_THREADS, 0, s>>>(n, ka, sh, hist, ntiles);
      scan_excl<uint32_t>(s, hist, (int64_t)256 * ntiles, nullptr, hist + (int64_t)256 * ntiles,
                          &c->launches_set);
      k_radix_scatter<<<ntiles, RS_THREADS, 0, s>>>(n, ka, va, kb, vb, sh, hist, ntiles);
      c->launches_set += 2;
      uint32_t* t = ka;
      ka = kb;
      kb = t;
      t = va;
      va = vb;
      vb = t;
    }
    c->skey = ka;
    if (c->forest)
      k_fgather<<<ceil_div(n, 256), 256, 0, s>>>(n, c->nprob, c->fb_pstart, c->fb_prob, c->fb_box, c->fb_frame, ka,
                                                 va, xyz, q,
                                                 c->perm, c->pos64, c->pos32, c->pos32lo);
    else
      k_gather<<<ceil_div(n, 256), 256, 0, s>>>(n, ka, va, xyz, q, c->box, c->perm, c->pos64, c->pos32,
                                                c->pos32lo);
    c->launches_set++;
    // every level from the sorted keys (k_lv_count, one scan, k_lv_write),
    // then the cells' counts
    {
      const int nb = ceil_div(n, LV_TILE);
      const int64_t ns = (int64_t)(Lf + 1) * nb;
      int32_t* sums = (int32_t*)c->scratch;
      int32_t* tot = sums + ns;
      k_lv_count<<<nb, LV_THREADS, 0, s>>>(n, ka, Lf, sums);
      scan_excl<int32_t>(s, sums, ns, tot, tot + 1, &c->launches_set);
      LevelOut lo{};
      LevelCounts lc{};
      lc.nlev = Lf + 1;
      lc.n = n;
      lc.off[0] = 0;
      for (int k = 0; k <= Lf; ++k) {
        lo.key[k] = c->lv.key[k];
        lo.first[k] = c->lv.first[k];
        lo.parent[k] = c->lv.parent[k];
        lc.first[k] = c->lv.first[k];
        lc.count[k] = c->lv.count[k];
        lc.off[k + 1] = lc.off[k] + ub[k];
      }
      k_lv_write<<<nb, LV_THREADS, 0, s>>>(n, ka, Lf, sums, tot, lo, c->pleaf, c->counters);
      k_lv_counts<<<ceil_div(lc.off[lc.nlev], 256), 256, 0, s>>>(lc, c->counters);
      c->launches_set += 3;
    }
    {
      GridSetAll ga{};
      ga.nlev = Lf + 1;
      ga.clear = 0;
      ga.counts = c->counters;
      ga.off[0] = 0;
      for (int k = 0; k <= Lf; ++k) {
        ga.key[k] = c->lv.key[k];
        ga.grid[k] = c->lv.grid[k];
        ga.off[k + 1] = ga.off[k] + ub[k];
      }
      k_grid_set_all<<<ceil_div(ga.off[ga.nlev], 256), 256, 0, s>>>(ga);
      c->launches_set++;
    }
    if (c->forest)
      for (int l = 0; l <= Lf; ++l) {
        k_cell_slot<<<ceil_div(ub[l], 256), 256, 0, s>>>(c->counters + l, c->lv.key[l], l, Lf, c->fb_nslot,
                                                         c->fb_sstart, c->fb_sprob, c->fb_prob, c->slot_buf[l]);
        c->launches_set++;
      }
    // P2P work lists: per leaf its first item; totals at counters[CNT_ITEMS]
    // (items | units << 32) and [CNT_BINS] (small | large items << 32)
    {
      const int nbw = ceil_div(ub[Lf], LW_TILE);
      unsigned long long* sums = (unsigned long long*)c->scratch;
      unsigned long long* work = sums + 2 * (int64_t)nbw;
      k_lw_count<<<nbw, LW_THREADS, 0, s>>>(c->counters + Lf, c->lv.count[Lf], sums);
      scan_excl<unsigned long long>(s, sums, nbw, (unsigned long long*)(c->counters + CNT_ITEMS), work,
                                    &c->launches_set);
      scan_excl<unsigned long long>(s, sums + nbw, nbw, (unsigned long long*)(c->counters + CNT_BINS), work,
                                    &c->launches_set);
      k_lw_write<<<nbw, LW_THREADS, 0, s>>>(c->counters + Lf, c->lv.count[Lf], sums, c->p2p_items, c->p2p_leaf,
                                            c->p2p_units, c->p2p_small, c->p2p_large);
      c->launches_set += 2;
    }
    if (Lf >= 2) {
      ClassArgs ca;
      for (int l = 0; l < FMM_MAX_LEVELS; ++l) {
        ca.key[l] = c->lv.key[l];
        ca.out[l] = c->lv.cls[l];
      }
      // chunked partition (levels 2 .. Lf; sized by the cells' upper bounds)
      ClassChunks cc;
      cc.lmin = 2;
      cc.nlev = Lf - 1;
      cc.blk0[0] = 0;
      cc.seg0[0] = 0;
      for (int k = 0; k < cc.nlev; ++k) {
        const int nb = ceil_div(ub[2 + k] > 0 ? ub[2 + k] : 1, CP_CHUNK);
        cc.blk0[k + 1] = cc.blk0[k] + nb;
        cc.seg0[k + 1] = cc.seg0[k] + 8 * nb;
      }
      const int64_t nseg = cc.seg0[cc.nlev];
      // counts + 1 trailing zero (its exclusive prefix is the grand total), then the scan's block sums
      int32_t* cnt = (int32_t*)c->scratch + 64;
      int32_t* work = cnt + nseg + 1;
      FMM_CUDA(c, cudaMemsetAsync(cnt + nseg, 0, sizeof(int32_t), s));
      k_cls_count<<<cc.blk0[cc.nlev], CP_THREADS, 0, s>>>(cc, c->counters, ca, cnt);
      scan_excl<int32_t>(s, cnt, nseg + 1, nullptr, work, &c->launches_set);
      k_cls_scatter<<<cc.blk0[cc.nlev], CP_THREADS, 0, s>>>(cc, c->counters, ca, cnt);
      c->launches_set += 2;
    }
    FMM_CUDA(c, cudaGetLastError());
  }

  FMM_CUDA(c, cudaMemcpyAsync(c->counters_h, c->counters, 128 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(c, cudaMemcpyAsync(c->box_h, c->box, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (c->forest && n > 0) {
    c->fb_box_h.assign(4 * (size_t)c->nprob, 0.0);
    FMM_CUDA(c, cudaMemcpyAsync(c->fb_box_h.data(), c->fb_box, 4 * sizeof(double) * c->nprob,
                                cudaMemcpyDeviceToHost, s));
  }
  FMM_CUDA(c, cudaStreamSynchronize(s));
  for (int l = 0; l < FMM_MAX_LEVELS; ++l) c->lv.slot[l] = (c->forest && l <= Lf) ? c->slot_buf[l] : nullptr;
  if (c->counters_h[CNT_BAD]) {
    for (int l = 0; l <= Lf; ++l) c->prev_ncell[l] = n > 0 ? c->counters_h[l] : 0;
    c->have_prev = n > 0;
    return set_err(c, FMM_ERR_ARG, "fmm_set_particles: non-finite coordinate or charge");
  }
  c->n = n;
  c->p2p_nitems = n > 0 ? c->counters_h[CNT_ITEMS] : 0;
  c->p2p_nunits = n > 0 ? c->counters_h[CNT_UNITS] : 0;
  c->p2p_nsmall = n > 0 ? c->counters_h[CNT_BINS] : 0;
  c->p2p_nlarge = n > 0 ? c->counters_h[CNT_BINS + 1] : 0;
  if (n > 0) {
    for (int d = 0; d < 4; ++d) c->box_host[d] = c->box_h[d];
  } else {
    c->box_host[0] = c->box_host[1] = c->box_host[2] = 0.0;
    c->box_host[3] = 1.0;
  }
  for (int l = 0; l < FMM_MAX_LEVELS; ++l) c->lv.ncell[l] = (l <= Lf && n > 0) ? c->counters_h[l] : 0;
  for (int l = 0; l <= Lf; ++l) c->prev_ncell[l] = c->lv.ncell[l];
  c->have_prev = n > 0;
  for (int l = 0; l <= Lf; ++l) {
    c->cls_off[l][0] = 0;
    for (int k = 0; k < 8; ++k)
      c->cls_off[l][k + 1] = c->cls_off[l][k] + ((l >= 2) ? c->counters_h[CNT_CLS + 8 * l + k] : 0);
  }

  // expansion rows: levels 2..leaf, each followed by one zero row
  int64_t rows = 0;
  for (int l = 0; l < FMM_MAX_LEVELS; ++l) c->lv.row_off[l] = 0;
  for (int l = 2; l <= Lf; ++l) {
    c->lv.row_off[l] = rows;
    rows += c->lv.ncell[l] + 1;
  }
  c->rows = rows;
  FMM_TRY(ensure_expansions(c, c->precision));

  // M2L tiles, leaf level first (largest first for the combined launch)
  std::vector<Tile> tiles;
  c->leaf_tiles = 0;
  for (int l = Lf; l >= 2; --l)
    for (int k = 0; k < 8; ++k) {
      int b = c->cls_off[l][k], e = c->cls_off[l][k + 1];
      for (int f = b; f < e; f += FMM_TILE) tiles.push_back(Tile{l, k, f, (e - f) < FMM_TILE ? e - f : FMM_TILE});
    }
  c->ntiles = (int)tiles.size();
  for (const Tile& tl : tiles) c->leaf_tiles += tl.level == Lf;
  c->tiles_h = tiles;
  c->tree_gen++;
  if (c->ntiles > c->tiles_cap) {
    int cap = c->ntiles + c->ntiles / 8 + 16;
    dfree(c, c->tiles, sizeof(Tile) * (size_t)c->tiles_cap);
    dfree(c, c->tile_src, sizeof(int32_t) * (size_t)c->tiles_cap * FMM_NT_CLASS * FMM_TILE);
    dfree(c, c->tile_act, sizeof(int16_t) * (size_t)c->tiles_cap * FMM_NT_CLASS);
    dfree(c, c->tile_nact, sizeof(int32_t) * (size_t)c->tiles_cap);
    dfree(c, c->src_act, sizeof(int16_t) * (size_t)c->tiles_cap * FMM_NT_CLASS);
    dfree(c, c->src_nact, sizeof(int32_t) * (size_t)c->tiles_cap);
    dfree(c, c->tile_mask, sizeof(uint32_t) * 2 * SETUP_WORDS * (size_t)c->tiles_cap);
    c->tile_mask = nullptr;
    c->src_act = nullptr;
    c->src_nact = nullptr;
    c->tiles = nullptr;
    c->tile_src = nullptr;
    c->tile_act = nullptr;
    c->tile_nact = nullptr;
    c->tiles_cap = 0;
    void* p;
    FMM_TRY(dalloc(c, &p, sizeof(Tile) * (size_t)cap));
    c->tiles = (Tile*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int32_t) * (size_t)cap * FMM_NT_CLASS * FMM_TILE));
    c->tile_src = (int32_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int16_t) * (size_t)cap * FMM_NT_CLASS));
    c->tile_act = (int16_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int32_t) * (size_t)cap));
    c->tile_nact = (int32_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int16_t) * (size_t)cap * FMM_NT_CLASS));
    c->src_act = (int16_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(int32_t) * (size_t)cap));
    c->src_nact = (int32_t*)p;
    FMM_TRY(dalloc(c, &p, sizeof(uint32_t) * 2 * SETUP_WORDS * (size_t)cap));
    c->tile_mask = (uint32_t*)p;
    c->tiles_cap = cap;
  }
  if (c->ntiles > 0) {
    FMM_CUDA(c, cudaMemcpyAsync(c->tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, s));
    uint32_t* masks = c->tile_mask;
    FMM_CUDA(c, cudaMemsetAsync(masks, 0, sizeof(uint32_t) * 2 * SETUP_WORDS * (size_t)c->ntiles, s));
    k_m2l_setup_split<<<dim3(c->ntiles, SETUP_SPLIT, 2), FMM_TILE, 0, s>>>(c->tiles, c->lv, c->cls_t, c->src_t,
                                                                           c->tvec, c->tile_src, masks);
    k_m2l_setup_lists<<<dim3(c->ntiles, 2), 2 * FMM_TILE, 0, s>>>(masks, c->ntiles, c->tile_act, c->tile_nact,
                                                                   c->src_act, c->src_nact);
    c->launches_set += 2;
  }
  if (rows > 0) {
    std::vector<int64_t> zr;
    for (int l = 2; l <= Lf; ++l) zr.push_back(c->lv.row_off[l] + c->lv.ncell[l]);
    int64_t* dz = (int64_t*)c->scratch;
    FMM_CUDA(c, cudaMemcpyAsync(dz, zr.data(), sizeof(int64_t) * zr.size(), cudaMemcpyHostToDevice, s));
    k_zero_rows<<<(int)zr.size(), 128, 0, s>>>((int)zr.size(), dz, c->cpad, c->Mhi, c->Mlo, c->L32, c->M64, c->L64);
    c->launches_set++;
  }
  // (host->device copies from pageable vectors are staged before returning)
  FMM_CUDA(c, cudaGetLastError());
  c->loaded = true;
  return FMM_OK;
}

FMM_DEBUG_TAKE_FN(fmm_debug_take_tree)

}  // namespace fmm
