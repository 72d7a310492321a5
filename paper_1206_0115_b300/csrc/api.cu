// api.cu -- the C ABI of include/fmm.h.
//
// Evaluation schedule (Sec. 3.2's two traversals plus the independent P2P):
// one CUDA graph per tree shape and precision, captured on an internal stream
// and replayed on the caller's stream:
//
//     P2M --> M2M (leaf-1 .. 2) --> fork --> M2L (all levels) --> L2L (2 .. leaf-1) --> join
//                                      \--> P2P -------------------------------------'
//
// followed by one plain launch of L2P, which adds the near field and scatters
// phi and F to the caller's order (its arguments are the caller's output
// pointers, which change from call to call).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace fmm {

static thread_local char g_create_err[512] = "";

fmm_status set_err(Ctx* c, fmm_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c ? c->err : g_create_err, 512, fmt, ap);
  va_end(ap);
  return s;
}

fmm_status cuda_err(Ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FMM_OK;
  if (c) c->last_cuda = e;
  if (e == cudaErrorMemoryAllocation) return set_err(c, FMM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_err(c, FMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device memory of every handle comes from one stream-ordered pool per device
// that keeps freed blocks cached (release threshold: never): buffers that
// grow, shrink (fmm_trim) or move between handles are recycled without
// cudaMalloc / cudaFree, whose device-wide synchronisation would serialise
// handles that run on different streams.  The pool reuses a block freed on
// another stream only once that free has completed (no implicit cross-stream
// dependencies).
cudaMemPool_t device_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = UINT64_MAX;
  int no = 0;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  pools[dev] = pool;
  return pool;
}

cudaError_t pool_alloc(int dev, cudaStream_t s, void** p, size_t bytes) {
  cudaMemPool_t pool = device_pool(dev);
  if (!pool) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Allocates on the handle's stream and waits for that stream, so that the
// block is ready for any stream (a block reused from a free on the same
// stream is only free in that stream's order).
fmm_status dalloc(Ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = pool_alloc(c->dev, c->stream, p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(c, e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA,
                   "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  c->bytes += (int64_t)bytes;
  return FMM_OK;
}

// Returns a block to the pool in the handle's stream order (after the work
// already enqueued there, which includes the joined P2P branch).
void dfree(Ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (cudaFreeAsync(p, c->stream) != cudaSuccess) cudaGetLastError();
  c->bytes -= (int64_t)(bytes ? bytes : 16);
}

// A kernel's dynamic shared-memory limit belongs to the function in the
// device's context, not to a handle: handles of different orders need
// different sizes, so the limit is only ever raised (one record per device
// and function, under a lock shared by every thread).
fmm_status raise_smem_limit(Ctx* c, const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> set;
  std::lock_guard<std::mutex> lk(mu);
  int& cur = set[{c->dev, func}];
  if (bytes <= cur) return FMM_OK;
  FMM_CUDA(c, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur = bytes;
  return FMM_OK;
}

// Small pinned host words of the handles (the readback of cell counts, the
// root cube and the tensor-core error word), 1 KB per handle, carved from
// pinned slabs that the process keeps: cudaFreeHost synchronises the device,
// which a handle destroyed on one thread must not do to work (or a graph
// capture) running on another thread's stream.
constexpr size_t PINNED_SLOT = 1024, PINNED_SLAB_SLOTS = 256;

struct PinnedSlots {
  std::mutex mu;
  std::vector<void*> free_slots;
};
PinnedSlots& pinned_slots() {
  static PinnedSlots* p = new PinnedSlots();  // outlives every handle (never destroyed)
  return *p;
}

void* pinned_slot() {
  PinnedSlots& ps = pinned_slots();
  std::lock_guard<std::mutex> lk(ps.mu);
  if (ps.free_slots.empty()) {
    void* slab = nullptr;
    if (cudaMallocHost(&slab, PINNED_SLOT * PINNED_SLAB_SLOTS) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (size_t k = 0; k < PINNED_SLAB_SLOTS; ++k) ps.free_slots.push_back((char*)slab + k * PINNED_SLOT);
  }
  void* p = ps.free_slots.back();
  ps.free_slots.pop_back();
  return p;
}

void pinned_release(void* p) {
  if (!p) return;
  PinnedSlots& ps = pinned_slots();
  std::lock_guard<std::mutex> lk(ps.mu);
  ps.free_slots.push_back(p);
}

namespace {

// Errors that a stream capture raises when the capture itself cannot
// proceed (the launches it records would run fine one by one).
bool is_capture_error(cudaError_t e) {
  switch (e) {
    case cudaErrorStreamCaptureUnsupported:
    case cudaErrorStreamCaptureInvalidated:
    case cudaErrorStreamCaptureMerge:
    case cudaErrorStreamCaptureUnmatched:
    case cudaErrorStreamCaptureUnjoined:
    case cudaErrorStreamCaptureIsolation:
    case cudaErrorStreamCaptureImplicit:
    case cudaErrorCapturedEvent:
    case cudaErrorStreamCaptureWrongThread:
      return true;
    default:
      return false;
  }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

fmm_status ensure_stage(Ctx* c, double** buf, int64_t* cap, int64_t count) {
  if (count <= *cap) return FMM_OK;
  dfree(c, *buf, sizeof(double) * (size_t)*cap);
  *buf = nullptr;
  *cap = 0;
  void* p;
  int64_t nc = count + count / 8 + 64;
  FMM_TRY(dalloc(c, &p, sizeof(double) * (size_t)nc));
  *buf = (double*)p;
  *cap = nc;
  return FMM_OK;
}

__global__ void k_widen_i32(int64_t n, const int32_t* __restrict__ a, int64_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i];
}
__global__ void k_widen_u32(int64_t n, const uint32_t* __restrict__ a, uint64_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i];
}

// copies n 8-byte values from a device temp to the caller (device or host)
fmm_status deliver(Ctx* c, void* dst, const void* devsrc, int64_t n) {
  if (n == 0) return FMM_OK;
  FMM_CUDA(c, cudaMemcpyAsync(dst, devsrc, 8 * (size_t)n, cudaMemcpyDefault, c->stream));
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  return FMM_OK;
}

fmm_status enqueue_eval(Ctx* c, cudaStream_t s) {
  // The near field (P2P) runs on a side branch beside the far field.  Where
  // it starts is the handle's schedule (p2p_sched, picked by fmm_autotune):
  // 0, with the compressed M2L's expansion kernel (the branch waits for the
  // projection); 1, at the start of the evaluation, so that its blocks fill
  // the SMs that the upward pass and the M2L bookkeeping kernels leave idle
  // (at the low launch priority, build_graph: the persistent M2L kernels
  // take each SM as the P2P blocks on it finish); 2 and 3, with the
  // projection, whose CTAs then leave shared memory for P2P blocks beside
  // them (and, in 3, the expansion's too; launch_m2l_svd_tc).
  // timing mode 2 runs P2P alone first (no overlap) so that every stage is timed in isolation
  cudaStream_t ps = c->timing == 2 ? s : c->side;
  const bool early = c->timing != 2 && c->p2p_sched == 1;
  auto near_branch = [&](cudaEvent_t start) -> fmm_status {
    FMM_CUDA(c, cudaStreamWaitEvent(c->side, start, 0));
    if (c->timing == 1) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[5], ps, cudaEventRecordExternal));
    {
      NvtxRange r("fmm:p2p");
      FMM_TRY(launch_p2p(c, ps));
    }
    if (c->timing == 1) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[6], ps, cudaEventRecordExternal));
    FMM_CUDA(c, cudaEventRecord(c->ev_join, c->side));
    return FMM_OK;
  };
  if (c->timing == 2) {
    FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[5], s, cudaEventRecordExternal));
    FMM_TRY(launch_p2p(c, s));
    FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[6], s, cudaEventRecordExternal));
  }
  // the compressed M2L's tree-only bookkeeping on a third branch, beside
  // the upward pass (launch_m2l joins it before the projection)
  c->m2l_prep_done = false;
  const bool prep = c->timing != 2 && m2l_has_prep(c);
  if (early || prep) FMM_CUDA(c, cudaEventRecord(c->ev_start, s));
  if (prep) {
    FMM_CUDA(c, cudaStreamWaitEvent(c->side3, c->ev_start, 0));
    FMM_TRY(launch_m2l_prep(c, c->side3));
  }
  if (early) FMM_TRY(near_branch(c->ev_start));
  // the leaf level's FP16 class-order multipoles (compressed M2L) need P2M
  // alone: a fourth branch runs that gather beside the M2M levels
  // (launch_m2l joins it before the coarser levels' gathers)
  c->leaf_gather_done = false;
  const bool gather_apart = c->timing != 2 && svd_leaf_gather_apart(c);
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[0], s, cudaEventRecordExternal));
  {
    NvtxRange r("fmm:upward");
    FMM_TRY(launch_upward(c, s, gather_apart ? c->ev_p2m : nullptr));
  }
  if (gather_apart) {
    FMM_CUDA(c, cudaStreamWaitEvent(c->side4, c->ev_p2m, 0));
    FMM_TRY(launch_svd_leaf_gather(c, c->side4));
  }
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[1], s, cudaEventRecordExternal));
  if (!early) FMM_CUDA(c, cudaEventRecord(c->ev_fork, s));
  c->p2p_after_proj = false;
  {
    NvtxRange r("fmm:m2l");
    FMM_TRY(launch_m2l(c, s, c->timing ? c->tev[2] : nullptr));
  }
  // schedule 0: the P2P branch starts with the persistent expansion kernel,
  // so that its blocks fill the room beside the expansion's CTAs instead of
  // holding the SMs the persistent kernels need (see launch_m2l_svd_tc)
  if (!early && c->timing == 2) {  // P2P ran alone above: an empty branch
    FMM_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    FMM_CUDA(c, cudaEventRecord(c->ev_join, c->side));
  } else if (!early) {
    FMM_TRY(near_branch(c->p2p_after_proj ? c->ev_p2p : c->ev_fork));
  }
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[3], s, cudaEventRecordExternal));
  {
    NvtxRange r("fmm:l2l");
    FMM_TRY(launch_l2l(c, s));
  }
  if (c->timing) FMM_CUDA(c, cudaEventRecordWithFlags(c->tev[4], s, cudaEventRecordExternal));
  FMM_CUDA(c, cudaStreamWaitEvent(s, c->ev_join, 0));
  return FMM_OK;
}

// Everything the captured evaluation graph bakes into its kernel arguments.
std::vector<int64_t> graph_signature(const Ctx* c) {
  std::vector<int64_t> s = {c->precision, c->timing, c->ntiles, c->leaf_tiles, c->n, m2l_kind(c), c->tc_nst,
                            c->p2p_nitems, (int64_t)(uintptr_t)c->p2p_items, c->leaf, c->forest,
                            (int64_t)(uintptr_t)c->fb_scale, c->p2p_variant, (int64_t)(uintptr_t)c->p2p_leaf,
                            c->p2p_big_variant, c->p2p_nsmall, c->p2p_nlarge, (int64_t)(uintptr_t)c->p2p_small,
                            (int64_t)(uintptr_t)c->p2p_large,
                            (int64_t)(uintptr_t)c->p2p_units, c->p2p_nunits,
                            (int64_t)(c->kernel_s * 1e6), (int64_t)(c->kernel_c * 1e9), c->skip_p2p,
                            c->m2l_f16, (int64_t)c->wait_ns, c->p2p_sched};
  for (int l = 0; l <= c->leaf; ++l) {
    s.push_back(c->lv.ncell[l]);
    s.push_back(c->lv.row_off[l]);
    for (int k = 0; k < 9; ++k) s.push_back(c->cls_off[l][k]);  // baked into the compressed M2L's launches
    for (const void* p : {(const void*)c->lv.key[l], (const void*)c->lv.first[l], (const void*)c->lv.count[l],
                          (const void*)c->lv.parent[l], (const void*)c->lv.grid[l], (const void*)c->lv.cls[l],
                          (const void*)c->lv.slot[l]})
      s.push_back((int64_t)(uintptr_t)p);
  }
  for (const void* p : {(const void*)c->pos32, (const void*)c->pos32lo, (const void*)c->pos64, (const void*)c->near32,
                        (const void*)c->near64, (const void*)c->Mhi, (const void*)c->Mlo, (const void*)c->L32,
                        (const void*)c->M64, (const void*)c->L64, (const void*)c->tiles, (const void*)c->tile_src,
                        (const void*)c->tile_act, (const void*)c->tile_nact, (const void*)c->K64,
                        (const void*)c->Khi, (const void*)c->Klo, (const void*)c->perm,
                        (const void*)c->tc_partial, (const void*)c->tc_err, (const void*)c->svd_Y,
                        (const void*)c->src_act, (const void*)c->svd_ry, (const void*)c->svd_V64,
                        (const void*)c->svd_recs, (const void*)c->svd_Mcls, (const void*)c->svd_yidx,
                        (const void*)c->svd_U64, (const void*)c->svd_VThi, (const void*)c->svd_Uhi})
    s.push_back((int64_t)(uintptr_t)p);
  s.push_back(c->svd_rmax);
  s.push_back(c->svd_rp);
  s.push_back(c->svd_YS);
  return s;
}

void drop_graph(Ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->graph_ok = false;
}

// A tensor-core M2L wait that ran out is reported by the next call (the flag
// comes back with the previous evaluation's stream work).
fmm_status check_device_error(Ctx* c) {
  if (c->tc_err_h && *(volatile int32_t*)c->tc_err_h) {
    const int32_t e = *(volatile int32_t*)c->tc_err_h;
    *(volatile int32_t*)c->tc_err_h = 0;
    if (c->tc_err) cudaMemsetAsync(c->tc_err, 0, sizeof(int32_t), c->stream);
    if (e & 1)
      return set_err(c, FMM_ERR_TIMEOUT, "M2L tensor-core kernel: a pipeline wait ran out and the kernel returned "
                                         "early; the previous evaluation's results are invalid");
    return set_err(c, FMM_ERR_CUDA, "M2L tensor-core path: internal work-table overflow (error word %d); the "
                                    "previous evaluation's results are invalid", e);
  }
  return FMM_OK;
}

fmm_status build_graph(Ctx* c) {
  drop_graph(c);
  c->last_cuda = cudaSuccess;
  cudaStream_t cap = c->cap;
  FMM_CUDA(c, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  fmm_status st = enqueue_eval(c, cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  if (st != FMM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  FMM_CUDA(c, e);
  c->graph = g;
  size_t nn = 0;
  FMM_CUDA(c, cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  FMM_CUDA(c, cudaGraphGetNodes(g, nodes.data(), &nn));
  // Launch priorities: the near field (P2P, FP32 pipe) gets the lowest, every
  // other kernel the highest, so that the persistent tensor-core M2L kernels
  // take their one CTA per SM as soon as the P2P branch (started first)
  // frees room, and P2P blocks then run in the room left beside them.
  int prio_low = 0, prio_high = 0;
  FMM_CUDA(c, cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  int64_t kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    ++kernels;
    cudaKernelNodeParams kp;
    if (c->p2p_priority && cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess) {
      cudaKernelNodeAttrValue v;
      memset(&v, 0, sizeof(v));
      v.priority = is_p2p_kernel(kp.func) ? prio_low : prio_high;
      FMM_CUDA(c, cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v));
    }
  }
  cudaGetLastError();
  FMM_CUDA(c, cudaGraphInstantiate(&c->gexec, g, 0));
  c->launches_eval = kernels + 1;  // + the L2P/output launch
  c->graph_sig = graph_signature(c);
  c->graph_ok = true;
  c->graph_precision = c->precision;
  return FMM_OK;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" {

fmm_status fmm_create(int height, int order, fmm_handle* out) {
  if (!out) return set_err(nullptr, FMM_ERR_ARG, "fmm_create: out is NULL");
  *out = nullptr;
  if (height < 1 || height > FMM_MAX_LEVELS)
    return set_err(nullptr, FMM_ERR_ARG, "fmm_create: height %d outside 1..%d", height, FMM_MAX_LEVELS);
  if (order < 2 || order > FMM_MAX_ORDER)
    return set_err(nullptr, FMM_ERR_ARG, "fmm_create: order %d outside 2..%d", order, FMM_MAX_ORDER);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaFree(nullptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, FMM_ERR_CUDA, "fmm_create: no usable CUDA device (%s)", cudaGetErrorString(e));
  }
  Ctx* c = new Ctx();
  c->dev = dev;
  c->height = height;
  c->order = order;
  c->leaf = height - 1;
  c->ncoef = order * order * order;
  c->cpad = (c->ncoef + 1 + 31) / 32 * 32;  // + the mean slot of mixed local expansions
  {
    const char* e = getenv("FMM_M2L_KERNEL");  // "simt": CUDA-core M2L in mixed precision too
    c->use_tc = !(e && strcmp(e, "simt") == 0);
    // compressed tensor-core M2L operands: FP16 hi/lo pairs (default, twice the
    // TF32 MMA rate) or "tf32": TF32 hi/lo pairs
    const char* mm = getenv("FMM_M2L_MATH");
    c->m2l_f16 = !(mm && strcmp(mm, "tf32") == 0);
    const char* pr = getenv("FMM_P2P_PRIORITY");  // "0": every graph node at the default priority
    c->p2p_priority = !(pr && strcmp(pr, "0") == 0);
    if (c->p2p_priority) p2p_carveout();
  }
  fmm_status st = FMM_OK;
  auto fail = [&](fmm_status s) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", c->err);
    fmm_destroy(c);
    return s;
  };
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side3, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side4, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_p2m, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_gleaf, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_prep, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_bin0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_bin1, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_p2p, cudaEventDisableTiming) != cudaSuccess) {
    cuda_err(c, cudaGetLastError(), "fmm_create: stream/event creation");
    return fail(FMM_ERR_CUDA);
  }
  for (int k = 0; k < 14; ++k)
    if (cudaEventCreate(&c->tev[k]) != cudaSuccess) {
      cuda_err(c, cudaGetLastError(), "fmm_create: event creation");
      return fail(FMM_ERR_CUDA);
    }
  // Creation is ordered on the handle's own non-blocking side stream (the
  // caller's stream is not known yet): no legacy-stream operation and no
  // device-wide synchronisation, so that handles created on one thread leave
  // graph captures running on other threads' streams undisturbed.
  c->stream = c->side;
  void* p;
  // corner, side, and the leaf frame of the FP32 coordinates (tree.cu, k_bbox_final)
  if ((st = dalloc(c, &p, 8 * sizeof(double))) != FMM_OK) return fail(st);
  c->box = (double*)p;
  if ((st = dalloc(c, &p, 128 * sizeof(int32_t))) != FMM_OK) return fail(st);
  c->counters = (int32_t*)p;
  c->pinned = pinned_slot();
  if (!c->pinned) {
    set_err(c, FMM_ERR_OOM, "fmm_create: pinned host memory");
    return fail(FMM_ERR_OOM);
  }
  // 512 B of counters, 64 B of cube, the error word
  c->counters_h = (int32_t*)c->pinned;
  c->box_h = (double*)((char*)c->pinned + 512);
  c->tc_err_h = (int32_t*)((char*)c->pinned + 576);
  *c->tc_err_h = 0;
  for (int l = 0; l <= c->leaf; ++l) {
    size_t bytes = sizeof(int32_t) * ((size_t)1 << (3 * l));
    if ((st = dalloc(c, &p, bytes)) != FMM_OK) return fail(st);
    c->lv.grid[l] = (int32_t*)p;
    if (cudaMemsetAsync(p, 0xFF, bytes, c->side) != cudaSuccess) {
      cuda_err(c, cudaGetLastError(), "fmm_create: grid memset");
      return fail(FMM_ERR_CUDA);
    }
  }
  if ((st = operators_init(c)) != FMM_OK) return fail(st);
  if (cudaStreamSynchronize(c->side) != cudaSuccess) {
    cuda_err(c, cudaGetLastError(), "fmm_create");
    return fail(FMM_ERR_CUDA);
  }
  c->stream = nullptr;  // the default until fmm_set_stream: the legacy stream
  *out = c;
  return FMM_OK;
}

fmm_status fmm_destroy(fmm_handle h) {
  Ctx* c = h;
  if (!c) return FMM_OK;
  // the handle's stream (NULL: the legacy stream) may still copy into its pinned slot
  if (c->side) cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  drop_graph(c);
  void* bufs[] = {c->key_a, c->key_b, c->idx_a, c->idx_b, c->perm, c->pleaf, c->pos64, c->pos32, c->pos32lo,
                  c->p2p_items, c->p2p_small, c->p2p_large,
                  c->p2p_leaf, c->p2p_units,
                  c->near32,
                  c->near64,
                  c->stage_in, c->stage_out, c->stokes_buf, c->scratch, c->box, c->counters, c->Mhi, c->Mlo, c->L32, c->M64,
                  c->L64, c->tiles, c->tile_src, c->tile_act, c->tile_nact, c->nodes64, c->cheb64, c->cheb32,
                  c->m2m64, c->m2m32, c->tvec, c->cls_t, c->K64, c->Khi, c->Klo, c->tc_partial, c->tc_err,
                  c->svd_W, c->svd_vals, c->svd_sm, c->svd_V64, c->svd_U64, c->svd_VThi,
                  c->svd_Uhi, c->svd_ry, c->svd_Y, c->src_t, c->src_act, c->src_nact, c->tile_mask,
                  c->svd_recs, c->svd_Mcls, c->svd_eslot, c->svd_ekch, c->svd_yidx, c->svd_umax, c->svd_mscale, c->tc_mmax,
                  c->fb_pstart, c->fb_prob, c->fb_box, c->fb_scale, c->fb_frame, c->fb_thr, c->fb_sstart, c->fb_sprob,
                  c->fb_bstart, c->svd_Yx, c->svd_dst, c->svd_kap8, c->svd_Uc};
  // back to the pool on the handle's own side stream (both streams are idle)
  for (void* b : bufs)
    if (b) cudaFreeAsync(b, c->side);
  for (int l = 0; l < FMM_MAX_LEVELS; ++l) {
    void* lb[] = {c->lv.key[l], c->lv.first[l], c->lv.count[l], c->lv.parent[l], c->lv.grid[l], c->lv.cls[l],
                  c->slot_buf[l]};
    for (void* b : lb)
      if (b) cudaFreeAsync(b, c->side);
  }
  if (c->side) cudaStreamSynchronize(c->side);
  cudaGetLastError();
  pinned_release(c->pinned);
  if (c->side2) {
    cudaStreamSynchronize(c->side2);
    cudaStreamDestroy(c->side2);
  }
  if (c->side3) {
    cudaStreamSynchronize(c->side3);
    cudaStreamDestroy(c->side3);
  }
  if (c->side4) {
    cudaStreamSynchronize(c->side4);
    cudaStreamDestroy(c->side4);
  }
  if (c->ev_p2m) cudaEventDestroy(c->ev_p2m);
  if (c->ev_gleaf) cudaEventDestroy(c->ev_gleaf);
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  if (c->ev_prep) cudaEventDestroy(c->ev_prep);
  if (c->ev_bin0) cudaEventDestroy(c->ev_bin0);
  if (c->ev_bin1) cudaEventDestroy(c->ev_bin1);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_p2p) cudaEventDestroy(c->ev_p2p);
  for (int k = 0; k < 14; ++k)
    if (c->tev[k]) cudaEventDestroy(c->tev[k]);
  delete c;
  return FMM_OK;
}

fmm_status fmm_set_stream(fmm_handle h, void* stream) {
  if (!h) return FMM_ERR_ARG;
  // buffers are freed in the handle's stream order: finish the old stream first
  if (h->stream != (cudaStream_t)stream) FMM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->stream = (cudaStream_t)stream;
  return FMM_OK;
}

fmm_status fmm_set_precision(fmm_handle h, int precision) {
  if (!h) return FMM_ERR_ARG;
  if (precision != FMM_FP64 && precision != FMM_MIXED)
    return set_err(h, FMM_ERR_ARG, "fmm_set_precision: unknown precision %d", precision);
  if (precision != h->precision) {
    h->precision = precision;
    h->graph_ok = false;
  }
  return FMM_OK;
}

fmm_status fmm_set_kernel(fmm_handle h, double s, double kc) {
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  if (!(s >= -2.0 && s <= 4.0 && s != 0.0))
    return set_err(c, FMM_ERR_ARG, "fmm_set_kernel: exponent %g outside [-2, 4] or 0", s);
  if (!(kc >= 0.0 && std::isfinite(kc))) return set_err(c, FMM_ERR_ARG, "fmm_set_kernel: offset %g", kc);
  if (s == c->kernel_s && kc == c->kernel_c) return FMM_OK;
  FMM_CUDA(c, cudaSetDevice(c->dev));
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->kernel_s = s;
  c->kernel_c = kc;
  // the M2L operators are values of the kernel: dropped here, rebuilt by the next evaluation
  const size_t C = (size_t)c->ncoef, cp = (size_t)c->cpad;
  dfree(c, c->K64, sizeof(double) * FMM_NT * C * C * c->ops64_nb);
  dfree(c, c->Khi, sizeof(float) * FMM_NT * cp * cp * c->ops32_nb);
  dfree(c, c->Klo, sizeof(float) * FMM_NT * cp * cp * c->ops32_nb);
  c->K64 = nullptr;
  c->Khi = c->Klo = nullptr;
  c->ops64 = c->ops32 = false;
  c->ops64_nb = c->ops32_nb = 0;
  c->svd_ready = false;
  c->graph_ok = false;
  return FMM_OK;
}

fmm_status fmm_set_m2l(fmm_handle h, int method, double eps) {
  if (!h) return FMM_ERR_ARG;
  if (method != FMM_M2L_FULL && method != FMM_M2L_SVD)
    return set_err(h, FMM_ERR_ARG, "fmm_set_m2l: unknown method %d", method);
  if (!(eps < 1.0) || eps != eps) return set_err(h, FMM_ERR_ARG, "fmm_set_m2l: eps must be < 1");
  if (method != h->m2l_method || eps != h->svd_eps) {
    h->m2l_method = method;
    h->svd_eps = eps;
    h->graph_ok = false;
  }
  return FMM_OK;
}

fmm_status fmm_get_svd_ranks(fmm_handle h, int32_t* ranks) {
  if (!h || !ranks) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  if (c->leaf < 2) return set_err(c, FMM_ERR_STATE, "fmm_get_svd_ranks: height < 3 has no M2L");
  if (c->kernel_c > 0.0) return set_err(c, FMM_ERR_STATE, "fmm_get_svd_ranks: no compression with c > 0");
  FMM_CUDA(c, cudaSetDevice(c->dev));
  FMM_TRY(svd_prepare(c));
  for (int k = 0; k < 16; ++k) ranks[k] = c->svd_rank[k];
  return FMM_OK;
}

fmm_status fmm_set_particles(fmm_handle h, int64_t n, const double* xyz, const double* q) {
  NvtxRange nvtx_range("fmm:set_particles");
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  if (n < 0 || n > ((int64_t)1 << 30))
    return set_err(c, FMM_ERR_ARG, "fmm_set_particles: n = %lld outside 0..2^30", (long long)n);
  if (n > 0 && (!xyz || !q)) return set_err(c, FMM_ERR_ARG, "fmm_set_particles: NULL input with n > 0");
  FMM_CUDA(c, cudaSetDevice(c->dev));
  const double* dxyz = xyz;
  const double* dq = q;
  if (n > 0 && !(is_device_ptr(xyz) && is_device_ptr(q))) {
    FMM_TRY(ensure_stage(c, &c->stage_in, &c->stage_in_cap, 4 * n));
    FMM_CUDA(c, cudaMemcpyAsync(c->stage_in, xyz, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->stage_in + 3 * n, q, sizeof(double) * n, cudaMemcpyDefault, c->stream));
    dxyz = c->stage_in;
    dq = c->stage_in + 3 * n;
  }
  c->forest = false;
  c->nprob = 0;
  c->leaf = c->height - 1;
  FMM_TRY(tree_build(c, n, dxyz, dq));
  return FMM_OK;
}

fmm_status fmm_set_batch(fmm_handle h, int32_t nprob, const int64_t* counts, const int32_t* heights,
                         const double* xyz, const double* q) {
  NvtxRange nvtx_range("fmm:set_batch");
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  c->loaded = false;
  if (nprob < 1 || nprob > FMM_MAX_BATCH)
    return set_err(c, FMM_ERR_ARG, "fmm_set_batch: nprob = %d outside 1..%d", nprob, FMM_MAX_BATCH);
  if (!counts || !heights) return set_err(c, FMM_ERR_ARG, "fmm_set_batch: NULL counts or heights");
  int64_t n = 0;
  for (int k = 0; k < nprob; ++k) {
    if (counts[k] < 0 || counts[k] > ((int64_t)1 << 30))
      return set_err(c, FMM_ERR_ARG, "fmm_set_batch: count[%d] = %lld outside 0..2^30", k, (long long)counts[k]);
    if (heights[k] < 1 || heights[k] > FMM_MAX_FOREST_LEAF + 1)
      return set_err(c, FMM_ERR_ARG, "fmm_set_batch: height[%d] = %d outside 1..%d", k, heights[k],
                     FMM_MAX_FOREST_LEAF + 1);
    n += counts[k];
  }
  if (n > ((int64_t)1 << 30)) return set_err(c, FMM_ERR_ARG, "fmm_set_batch: %lld particles > 2^30", (long long)n);
  if (n > 0 && (!xyz || !q)) return set_err(c, FMM_ERR_ARG, "fmm_set_batch: NULL input with particles");
  FMM_CUDA(c, cudaSetDevice(c->dev));
  const double* dxyz = xyz;
  const double* dq = q;
  if (n > 0 && !(is_device_ptr(xyz) && is_device_ptr(q))) {
    FMM_TRY(ensure_stage(c, &c->stage_in, &c->stage_in_cap, 4 * n));
    FMM_CUDA(c, cudaMemcpyAsync(c->stage_in, xyz, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(c->stage_in + 3 * n, q, sizeof(double) * n, cudaMemcpyDefault, c->stream));
    dxyz = c->stage_in;
    dq = c->stage_in + 3 * n;
  }
  int64_t total = 0;
  FMM_TRY(batch_layout(c, nprob, counts, heights, &total));
  FMM_TRY(tree_build(c, total, dxyz, dq));
  return FMM_OK;
}

fmm_status fmm_batch_plan(int32_t nprob, const int64_t* counts, const int32_t* heights, int64_t* slot_key,
                          int64_t* slot_level, int32_t* leaf_level) {
  if (nprob < 1 || nprob > FMM_MAX_BATCH || !counts || !heights || !slot_key || !slot_level || !leaf_level)
    return set_err(nullptr, FMM_ERR_ARG, "fmm_batch_plan: bad arguments");
  for (int k = 0; k < nprob; ++k)
    if (counts[k] < 0 || heights[k] < 1 || heights[k] > FMM_MAX_FOREST_LEAF + 1)
      return set_err(nullptr, FMM_ERR_ARG, "fmm_batch_plan: count or height of problem %d out of range", k);
  int Lf = 0;
  if (batch_plan(nprob, counts, heights, slot_key, slot_level, &Lf) != 0)
    return set_err(nullptr, FMM_ERR_ARG, "fmm_batch_plan: the leaf cells exceed 8^%d", FMM_MAX_FOREST_LEAF);
  *leaf_level = Lf;
  return FMM_OK;
}

fmm_status fmm_get_batch_info(fmm_handle h, int32_t k, int64_t* info, double* box) {
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  if (!c->loaded || !c->forest) return set_err(c, FMM_ERR_STATE, "fmm_get_batch_info: no batch loaded");
  if (k < 0 || k >= c->nprob) return set_err(c, FMM_ERR_ARG, "fmm_get_batch_info: problem %d outside 0..%d", k,
                                             c->nprob - 1);
  const int64_t cnt = c->fb_start_h[k + 1] - c->fb_start_h[k];
  if (info) {
    info[0] = c->fb_first_h[k];
    info[1] = cnt;
    info[2] = cnt > 0 ? c->fb_prob_h[k].S : -1;
    info[3] = cnt > 0 ? (int64_t)c->fb_prob_h[k].slot_key : -1;
    info[4] = c->leaf;
    info[5] = c->fb_prob_h[k].L + 1;
    info[6] = c->fb_start_h[k];
    info[7] = 0;
  }
  if (box) {
    const bool has = cnt > 0 && c->fb_box_h.size() >= 4 * (size_t)(k + 1);
    for (int d = 0; d < 4; ++d) box[d] = has ? c->fb_box_h[4 * k + d] : (d == 3 ? 1.0 : 0.0);
  }
  return FMM_OK;
}

fmm_status fmm_evaluate(fmm_handle h, double* phi, double* F) {
  NvtxRange nvtx_range("fmm:evaluate");
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  if (!c->loaded) return set_err(c, FMM_ERR_STATE, "fmm_evaluate: no particles loaded");
  const int64_t n = c->n;
  if (n == 0) return FMM_OK;
  if (!phi || !F) return set_err(c, FMM_ERR_ARG, "fmm_evaluate: NULL output");
  FMM_CUDA(c, cudaSetDevice(c->dev));
  FMM_TRY(check_device_error(c));
  FMM_TRY(ensure_expansions(c, c->precision));
  if (c->forest && c->kernel_c > 0.0)
    return set_err(c, FMM_ERR_STATE, "fmm_evaluate: batches need a homogeneous kernel (c = 0)");
  if (uses_svd(c)) {
    if (c->leaf >= 2) FMM_TRY(m2l_svd_prepare(c));
    if (c->leaf >= 2 && m2l_kind(c) == 5) FMM_TRY(m2l_svd_tc_prepare(c));
  } else {
    FMM_TRY(operators_m2l(c, c->precision));
    if (m2l_kind(c) == 2) FMM_TRY(m2l_tc_prepare(c));
  }
  const bool dev_out = is_device_ptr(phi) && is_device_ptr(F);
  double *dphi = phi, *dF = F;
  if (!dev_out) {
    FMM_TRY(ensure_stage(c, &c->stage_out, &c->stage_out_cap, 4 * n));
    dphi = c->stage_out;
    dF = c->stage_out + n;
  }
  bool eager = !c->use_graph;
  if (c->use_graph && (!c->graph_ok || c->graph_sig != graph_signature(c))) {
    const fmm_status gs = build_graph(c);
    if (gs != FMM_OK) {
      // Only a failed capture falls back (a capture error is not sticky):
      // the same launches run without a graph, counted in fmm_get_stats
      // out[6], and the capture's message stays in fmm_last_error.  Any
      // other failure -- instantiation, a launch error, a device fault -- is
      // returned.
      if (gs != FMM_ERR_CUDA || !is_capture_error(c->last_cuda)) return gs;
      cudaGetLastError();
      drop_graph(c);
      c->graph_fallbacks++;
      eager = true;
    }
  }
  if (eager) FMM_TRY(enqueue_eval(c, c->stream));
  else FMM_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
  if (c->timing) FMM_CUDA(c, cudaEventRecord(c->tev[7], c->stream));
  FMM_TRY(launch_l2p_out(c, c->stream, dphi, dF));
  if (c->timing) FMM_CUDA(c, cudaEventRecord(c->tev[8], c->stream));
  c->tev_recorded = c->timing;
  if (c->tc_err && (m2l_kind(c) == 2 || m2l_kind(c) == 5))
    FMM_CUDA(c, cudaMemcpyAsync(c->tc_err_h, c->tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  if (!dev_out) {
    FMM_CUDA(c, cudaMemcpyAsync(phi, dphi, sizeof(double) * n, cudaMemcpyDefault, c->stream));
    FMM_CUDA(c, cudaMemcpyAsync(F, dF, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
    FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return FMM_OK;
}

fmm_status fmm_evaluate_stokes(fmm_handle h, const double* f, double* u) {
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  if (!c->loaded) return set_err(c, FMM_ERR_STATE, "fmm_evaluate_stokes: no particles loaded");
  if (c->forest) return set_err(c, FMM_ERR_STATE, "fmm_evaluate_stokes: single problems only");
  if (c->kernel_s != 1.0 || c->kernel_c != 0.0)
    return set_err(c, FMM_ERR_STATE, "fmm_evaluate_stokes: needs the 1/r kernel");
  const int64_t n = c->n;
  if (n == 0) return FMM_OK;
  if (!f || !u) return set_err(c, FMM_ERR_ARG, "fmm_evaluate_stokes: NULL argument");
  FMM_CUDA(c, cudaSetDevice(c->dev));
  FMM_TRY(ensure_stage(c, &c->stokes_buf, &c->stokes_cap, 27 * n));
  float4* f32 = (float4*)c->stokes_buf;    // [n] forces, Morton order (mixed)
  float4* unear = f32 + n;                 // [n] Stokeslet near field, Morton order (mixed)
  double* phi4 = c->stokes_buf + 4 * n;    // [4][n]
  double* F4 = phi4 + 4 * n;               // [4][n][3]
  double* q0 = F4 + 12 * n;                // [n] the loaded charges, Morton order
  double* df = q0 + n;                     // [n][3] forces on the device
  double* du = df + 3 * n;                 // [n][3] result on the device
  const double* fd = f;
  if (!is_device_ptr(f)) {
    FMM_CUDA(c, cudaMemcpyAsync(df, f, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
    fd = df;
  }
  const bool dev_out = is_device_ptr(u);
  // Mixed precision: the four 1/r passes give the far field only and the
  // near field is the Stokeslet summed directly (the identity's terms are
  // |x - o| / r times the result there, too much for FP32 on close pairs);
  // FP64 takes all of u from the four passes.
  const bool mixed = c->precision == FMM_MIXED;
  FMM_TRY(launch_stokes_save(c, q0));
  fmm_status st = FMM_OK;
  c->skip_p2p = mixed;
  for (int j = 0; j < 4 && st == FMM_OK; ++j) {
    st = launch_stokes_charges(c, fd, q0, j);
    if (st == FMM_OK) st = fmm_evaluate(h, phi4 + j * n, F4 + 3 * j * n);
  }
  c->skip_p2p = false;
  if (st == FMM_OK && mixed) st = launch_stokes_forces(c, fd, f32);
  if (st == FMM_OK && mixed) st = launch_p2p_stokes(c, c->stream, f32, unear);
  if (st == FMM_OK) st = launch_stokes_combine(c, phi4, F4, mixed ? unear : nullptr, dev_out ? u : du);
  // the handle's own charges come back whatever happened above
  const fmm_status rs = launch_stokes_charges(c, nullptr, q0, -1);
  if (st != FMM_OK) return st;
  if (rs != FMM_OK) return rs;
  if (!dev_out) {
    FMM_CUDA(c, cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
    FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return FMM_OK;
}

fmm_status fmm_set_wait_limit(fmm_handle h, double seconds) {
  if (!h) return FMM_ERR_ARG;
  if (!(seconds > 0.0 && seconds <= 60.0))
    return set_err(h, FMM_ERR_ARG, "fmm_set_wait_limit: %g s outside (0, 60]", seconds);
  const double ns = std::ceil(seconds * 1e9);
  h->wait_ns = (uint64_t)ns;
  h->graph_ok = false;  // the limit is a kernel argument baked into the graph
  return FMM_OK;
}

fmm_status fmm_set_p2p_variant(fmm_handle h, int variant) {
  if (!h) return FMM_ERR_ARG;
  if (variant < 0 || variant >= FMM_P2P_VARIANTS)
    return set_err(h, FMM_ERR_ARG, "fmm_set_p2p_variant: %d outside 0..%d", variant, FMM_P2P_VARIANTS - 1);
  if (variant != h->p2p_variant || h->p2p_big_variant != -1) {
    h->p2p_variant = variant;
    h->p2p_big_variant = -1;  // one shape for every leaf
    h->graph_ok = false;
  }
  return FMM_OK;
}

}  // extern "C"

namespace fmm {
namespace {

bool persistent_shape(int v) { return v == 14 || v == 15; }
bool is_coop_shape(int v) { return v == 12 || v == 13; }

// The evaluation schedule (fmm_autotune's last stage): whole evaluations in
// up to eight candidates -- the near-field branch starting with the
// compressed M2L's expansion (schedule 0), at the start (1), or with the
// projection (2; 3 with two expansion stages), each with the shapes chosen
// so far and with the fastest shapes per bin that hold no SM for the whole
// launch (not the persistent 14, 15: their blocks stay until the last work
// item is taken, so a persistent M2L kernel cannot start beside them) --
// each run once to build its graph, then timed three times with CUDA events
// on the handle's stream; the fastest is kept.
fmm_status autotune_schedule(Ctx* c) {
  for (int k = 0; k < FMM_SCHED_CANDIDATES; ++k) c->sched_ms[k] = -1.f;
  if (c->leaf < 2 || c->n == 0 || !c->use_graph) return FMM_OK;  // no far field to order against
  const int keep_timing = c->timing;
  if (c->timing == 2) c->timing = 0;  // mode 2 runs P2P alone: no schedule to time
  const int nb[2] = {(int)c->p2p_nsmall, (int)c->p2p_nlarge};
  // the non-persistent alternative, per bin, from the bins' own times
  int alt[2] = {-1, -1};
  for (int b = 0; b < 2; ++b) {
    float bt = -1.f;
    for (int v = 0; v < FMM_P2P_VARIANTS; ++v) {
      const float ms = c->p2p_bin_ms[b][v];
      if (ms < 0.f || nb[b] == 0 || persistent_shape(v) || (b == 0 && is_coop_shape(v))) continue;
      if (bt < 0.f || ms < bt) {
        bt = ms;
        alt[b] = v;
      }
    }
  }
  const int chosen_var = c->p2p_variant, chosen_big = c->p2p_big_variant;
  int alt_var = nb[0] > 0 ? alt[0] : (alt[1] >= 0 && !is_coop_shape(alt[1]) ? alt[1] : 0);
  int alt_big = nb[1] > 0 ? alt[1] : -1;
  if (alt_big == alt_var) alt_big = -1;
  const int eff_small = is_coop_shape(chosen_var) ? 14 : chosen_var;
  const int eff_large = chosen_big >= 0 ? chosen_big : chosen_var;
  const bool uses_persistent = (nb[0] > 0 && persistent_shape(eff_small)) || (nb[1] > 0 && persistent_shape(eff_large));
  const bool have_alt = uses_persistent && (nb[0] == 0 || alt[0] >= 0) && (nb[1] == 0 || alt[1] >= 0);

  fmm_status st = ensure_stage(c, &c->stage_out, &c->stage_out_cap, 4 * c->n);
  double* phi = c->stage_out;
  double* F = c->stage_out + c->n;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == FMM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = cuda_err(c, cudaGetLastError(), "fmm_autotune: events");
  // Two passes over the candidates, each building every candidate's graph
  // afresh; a candidate counts with the slower of its two times, so that a
  // lead seen in one pass only (the order in which the block scheduler
  // places the near field's blocks beside the M2L CTAs can differ between
  // runs of the same graph) does not decide.
  for (int pass = 0; pass < 2 && st == FMM_OK; ++pass)
    for (int k = 0; k < FMM_SCHED_CANDIDATES && st == FMM_OK; ++k) {
      const bool use_alt = k >= 4;
      if (use_alt && !have_alt) continue;
      if ((k & 3) >= 2 && !(m2l_kind(c) == 5 && svd_wants_f16(c))) continue;  // the compressed FP16 M2L's stages
      c->p2p_sched = k & 3;
      c->p2p_variant = use_alt ? alt_var : chosen_var;
      c->p2p_big_variant = use_alt ? alt_big : chosen_big;
      c->graph_ok = false;
      st = fmm_evaluate(c, phi, F);  // builds this candidate's graph
      if (st == FMM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess)
        st = cuda_err(c, cudaGetLastError(), "event");
      for (int r = 0; r < 3 && st == FMM_OK; ++r) st = fmm_evaluate(c, phi, F);
      float ms = 0.f;
      if (st == FMM_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = cuda_err(c, cudaGetLastError(), "fmm_autotune: timing");
      if (st != FMM_OK) break;
      c->sched_ms[k] = pass == 0 ? ms / 3.f : std::max(c->sched_ms[k], ms / 3.f);
    }
  int best = -1;
  float best_ms = -1.f;
  for (int k = 0; k < FMM_SCHED_CANDIDATES && st == FMM_OK; ++k)
    if (c->sched_ms[k] >= 0.f && (best < 0 || c->sched_ms[k] < best_ms)) {
      best = k;
      best_ms = c->sched_ms[k];
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->timing = keep_timing;
  const int pick = best >= 0 ? best : 0;
  c->p2p_sched = st == FMM_OK ? (pick & 3) : 0;
  c->p2p_variant = (st == FMM_OK && pick >= 4) ? alt_var : chosen_var;
  c->p2p_big_variant = (st == FMM_OK && pick >= 4) ? alt_big : chosen_big;
  c->graph_ok = false;
  return st;
}

}  // namespace
}  // namespace fmm

extern "C" {

fmm_status fmm_autotune(fmm_handle h, int32_t* choice, float* times_ms) {
  NvtxRange nvtx_range("fmm:autotune");
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  if (!c->loaded) return set_err(c, FMM_ERR_STATE, "fmm_autotune: no particles loaded");
  FMM_CUDA(c, cudaSetDevice(c->dev));
  if (c->kernel_s != 1.0 || c->kernel_c != 0.0) {
    // one shape of the general-kernel P2P: report its time only
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = -1.f;
    const int keep = c->precision;
    c->precision = FMM_MIXED;
    fmm_status st = FMM_OK;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
      st = launch_p2p(c, c->stream);
      if (st == FMM_OK && cudaEventRecord(e0, c->stream) == cudaSuccess) {
        for (int k = 0; k < 3 && st == FMM_OK; ++k) st = launch_p2p(c, c->stream);
        if (st == FMM_OK && cudaEventRecord(e1, c->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
          cudaEventElapsedTime(&ms, e0, e1);
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    c->precision = keep;
    if (st != FMM_OK) return st;
    if (choice) {
      const int32_t v[5] = {-1, 8, 128, 2, 4};
      for (int k = 0; k < 5; ++k) choice[k] = v[k];
    }
    if (times_ms)
      for (int k = 0; k < FMM_P2P_VARIANTS; ++k) times_ms[k] = ms / 3.f;
    return FMM_OK;
  }
  // Each occupancy bin (small leaves, large leaves) is timed alone in every
  // shape (the cooperative shapes only on large leaves) and keeps its fastest.
  const int keep_prec = c->precision, keep_var = c->p2p_variant, keep_big = c->p2p_big_variant;
  c->precision = FMM_MIXED;  // the variants are shapes of the mixed kernel
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fmm_status st = FMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = cuda_err(c, cudaGetLastError(), "fmm_autotune: events");
  const int nb[2] = {c->p2p_nsmall, c->p2p_nlarge};
  int best[2] = {keep_var, keep_big};
  for (int b = 0; b < 2; ++b) {
    float bt = -1.f;
    for (int v = 0; v < FMM_P2P_VARIANTS; ++v) {
      c->p2p_bin_ms[b][v] = -1.f;
      if (st != FMM_OK || nb[b] == 0 || (b == 0 && (v == 12 || v == 13))) continue;
      float ms = 0.f;
      st = launch_p2p_bin(c, c->stream, b, v);  // warm-up
      if (st == FMM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = cuda_err(c, cudaGetLastError(), "event");
      for (int k = 0; k < 3 && st == FMM_OK; ++k) st = launch_p2p_bin(c, c->stream, b, v);
      if (st == FMM_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = cuda_err(c, cudaGetLastError(), "fmm_autotune: timing");
      ms /= 3.f;
      c->p2p_bin_ms[b][v] = ms;
      if (st == FMM_OK && (bt < 0.f || ms < bt)) {
        bt = ms;
        best[b] = v;
      }
    }
  }
  // The bins against one launch over every item: the item shape with the
  // least time over both bins, timed as one launch; kept if it beats the
  // bins' two launches (a small bin whose leaves border large ones costs
  // about as much per item as the large bin, and one launch balances better).
  int one = -1;
  float one_ms = -1.f, binned_ms = 0.f;
  if (st == FMM_OK && nb[0] > 0 && nb[1] > 0) {
    binned_ms = c->p2p_bin_ms[0][best[0]] + c->p2p_bin_ms[1][best[1]];
    float est = -1.f;
    for (int v = 0; v < FMM_P2P_VARIANTS; ++v) {
      if (v == 12 || v == 13 || c->p2p_bin_ms[0][v] < 0.f || c->p2p_bin_ms[1][v] < 0.f) continue;
      const float t = c->p2p_bin_ms[0][v] + c->p2p_bin_ms[1][v];
      if (est < 0.f || t < est) {
        est = t;
        one = v;
      }
    }
    if (one >= 0) {
      c->p2p_variant = one;
      c->p2p_big_variant = -1;
      float ms = 0.f;
      st = launch_p2p(c, c->stream);  // warm-up
      if (st == FMM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = cuda_err(c, cudaGetLastError(), "event");
      for (int k = 0; k < 3 && st == FMM_OK; ++k) st = launch_p2p(c, c->stream);
      if (st == FMM_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = cuda_err(c, cudaGetLastError(), "fmm_autotune: timing");
      one_ms = ms / 3.f;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->precision = keep_prec;
  if (st == FMM_OK && one >= 0 && one_ms < binned_ms) {
    c->p2p_variant = one;  // one launch over every item
    c->p2p_big_variant = -1;
  } else if (st == FMM_OK) {
    // small leaves' shape (the large leaves' if there are no small ones), the large leaves' own
    c->p2p_variant = nb[0] > 0 ? best[0] : (nb[1] > 0 && !(best[1] == 12 || best[1] == 13) ? best[1] : keep_var);
    c->p2p_big_variant = nb[1] > 0 ? best[1] : -1;
  } else {
    c->p2p_variant = keep_var;
    c->p2p_big_variant = keep_big;
  }
  c->graph_ok = false;
  if (st != FMM_OK) return st;
  if (c->precision == FMM_MIXED) FMM_TRY(autotune_schedule(c));
  if (times_ms)  // each shape used for every item, as fmm_set_p2p_variant would
    for (int v = 0; v < FMM_P2P_VARIANTS; ++v) {
      const float a = nb[0] > 0 ? c->p2p_bin_ms[0][(v == 12 || v == 13) ? 14 : v] : 0.f;
      const float b = nb[1] > 0 ? c->p2p_bin_ms[1][v] : 0.f;
      times_ms[v] = a + b;
    }
  if (choice) {
    choice[0] = c->p2p_variant;
    for (int k = 0; k < 4; ++k) choice[1 + k] = kP2PVariants[c->p2p_variant][k];
  }
  return FMM_OK;
}

int fmm_debug_build(void) {
#ifdef FMM_DEBUG
  return 1;
#else
  return 0;
#endif
}

fmm_status fmm_debug_check(uint64_t* first_failure) {
  if (!first_failure) return set_err(nullptr, FMM_ERR_ARG, "fmm_debug_check: first_failure is NULL");
  unsigned long long v = 0;
  for (unsigned long long (*take)() : {fmm_debug_take_tree, fmm_debug_take_nearfield, fmm_debug_take_m2l_svd_tc}) {
    const unsigned long long x = take();
    if (x == ~0ull) return set_err(nullptr, FMM_ERR_CUDA, "fmm_debug_check: the check words could not be read");
    if (!v) v = x;
  }
  *first_failure = v;
  return FMM_OK;
}

fmm_status fmm_set_schedule(fmm_handle h, int sched) {
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  if (sched < 0 || sched > 3) return set_err(c, FMM_ERR_ARG, "fmm_set_schedule: %d outside 0..3", sched);
  if (sched != c->p2p_sched) {
    c->p2p_sched = sched;
    c->graph_ok = false;
  }
  return FMM_OK;
}

fmm_status fmm_get_schedule(fmm_handle h, int32_t* sched, float* times_ms) {
  if (!h || !sched) return FMM_ERR_ARG;
  Ctx* c = h;
  *sched = c->p2p_sched;
  if (times_ms)
    for (int k = 0; k < FMM_SCHED_CANDIDATES; ++k) times_ms[k] = c->sched_ms[k];
  return FMM_OK;
}

fmm_status fmm_get_p2p_bins(fmm_handle h, int64_t* out, float* times_ms) {
  if (!h || !out) return FMM_ERR_ARG;
  Ctx* c = h;
  if (!c->loaded) return set_err(c, FMM_ERR_STATE, "fmm_get_p2p_bins: no particles loaded");
  const bool coop = c->p2p_variant == 12 || c->p2p_variant == 13;
  out[0] = coop ? 14 : c->p2p_variant;
  out[1] = c->p2p_big_variant >= 0 ? c->p2p_big_variant : c->p2p_variant;
  out[2] = c->p2p_nsmall;
  out[3] = c->p2p_nlarge;
  if (times_ms)
    for (int b = 0; b < 2; ++b)
      for (int v = 0; v < FMM_P2P_VARIANTS; ++v) times_ms[b * FMM_P2P_VARIANTS + v] = c->p2p_bin_ms[b][v];
  return FMM_OK;
}

fmm_status fmm_trim(fmm_handle h) {
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  c->err[0] = 0;
  FMM_CUDA(c, cudaSetDevice(c->dev));
  drop_graph(c);
  release_tree(c);
  return FMM_OK;
}

fmm_status fmm_get_order(fmm_handle h, int64_t* perm) {
  if (!h) return FMM_ERR_ARG;
  Ctx* c = h;
  if (!c->loaded) return set_err(c, FMM_ERR_STATE, "fmm_get_order: no particles loaded");
  if (c->n == 0) return FMM_OK;
  if (!perm) return set_err(c, FMM_ERR_ARG, "fmm_get_order: NULL output");
  FMM_TRY(ensure_stage(c, &c->stage_out, &c->stage_out_cap, c->n));
  k_widen_i32<<<ceil_div(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, (int64_t*)c->stage_out);
  FMM_CUDA(c, cudaGetLastError());
  return deliver(c, perm, c->stage_out, c->n);
}

fmm_status fmm_get_box(fmm_handle h, double* out) {
  if (!h || !out) return FMM_ERR_ARG;
  if (!h->loaded) return set_err(h, FMM_ERR_STATE, "fmm_get_box: no particles loaded");
  for (int d = 0; d < 4; ++d) out[d] = h->box_host[d];
  return FMM_OK;
}

fmm_status fmm_get_level_size(fmm_handle h, int level, int64_t* out) {
  if (!h || !out) return FMM_ERR_ARG;
  if (!h->loaded) return set_err(h, FMM_ERR_STATE, "fmm_get_level_size: no particles loaded");
  if (level < 0 || level > h->leaf) return set_err(h, FMM_ERR_ARG, "level %d outside 0..%d", level, h->leaf);
  *out = h->lv.ncell[level];
  return FMM_OK;
}

fmm_status fmm_get_level_keys(fmm_handle h, int level, uint64_t* keys) {
  int64_t nc;
  FMM_TRY(fmm_get_level_size(h, level, &nc));
  Ctx* c = h;
  if (nc == 0) return FMM_OK;
  if (!keys) return set_err(c, FMM_ERR_ARG, "NULL output");
  FMM_TRY(ensure_stage(c, &c->stage_out, &c->stage_out_cap, nc));
  k_widen_u32<<<ceil_div(nc, 256), 256, 0, c->stream>>>(nc, c->lv.key[level], (uint64_t*)c->stage_out);
  FMM_CUDA(c, cudaGetLastError());
  return deliver(c, keys, c->stage_out, nc);
}

fmm_status fmm_get_level_ranges(fmm_handle h, int level, int64_t* first, int64_t* count) {
  int64_t nc;
  FMM_TRY(fmm_get_level_size(h, level, &nc));
  Ctx* c = h;
  if (nc == 0) return FMM_OK;
  if (!first || !count) return set_err(c, FMM_ERR_ARG, "NULL output");
  FMM_TRY(ensure_stage(c, &c->stage_out, &c->stage_out_cap, nc));
  k_widen_i32<<<ceil_div(nc, 256), 256, 0, c->stream>>>(nc, c->lv.first[level], (int64_t*)c->stage_out);
  FMM_CUDA(c, cudaGetLastError());
  FMM_TRY(deliver(c, first, c->stage_out, nc));
  k_widen_i32<<<ceil_div(nc, 256), 256, 0, c->stream>>>(nc, c->lv.count[level], (int64_t*)c->stage_out);
  FMM_CUDA(c, cudaGetLastError());
  return deliver(c, count, c->stage_out, nc);
}

fmm_status fmm_get_expansion(fmm_handle h, int level, int which, double* out) {
  int64_t nc;
  FMM_TRY(fmm_get_level_size(h, level, &nc));
  Ctx* c = h;
  if (level < 2 || (which != 0 && which != 1))
    return set_err(c, FMM_ERR_ARG, "fmm_get_expansion: level %d / which %d invalid", level, which);
  if (nc == 0) return FMM_OK;
  if (!out) return set_err(c, FMM_ERR_ARG, "NULL output");
  const int64_t total = nc * c->ncoef;
  FMM_TRY(ensure_stage(c, &c->stage_out, &c->stage_out_cap, total));
  FMM_TRY(expansion_to_f64(c, level, which, c->stage_out));
  return deliver(c, out, c->stage_out, total);
}

fmm_status fmm_get_stats(fmm_handle h, int64_t* out) {
  if (!h || !out) return FMM_ERR_ARG;
  out[0] = h->launches_set;
  out[1] = h->graph_ok ? h->launches_eval : count_launches_eval(h);
  out[2] = h->use_graph ? 1 : 0;
  out[3] = h->bytes;
  out[4] = m2l_kind(h);
  out[5] = (m2l_uses_f16(h) && (out[4] == 2 || out[4] == 5)) ? 1 : 0;  // the tensor-core kernels' operand form
  out[6] = h->graph_fallbacks;  // evaluations run without a graph after a failed capture
  out[7] = 0;
  return FMM_OK;
}

fmm_status fmm_get_work(fmm_handle h, int64_t* out) {
  if (!h || !out) return FMM_ERR_ARG;
  if (!h->loaded) return set_err(h, FMM_ERR_STATE, "fmm_get_work: no particles loaded");
  return work_counts(h, out);
}

fmm_status fmm_set_timing(fmm_handle h, int mode) {
  if (!h) return FMM_ERR_ARG;
  if (mode < 0 || mode > 2) return set_err(h, FMM_ERR_ARG, "fmm_set_timing: mode %d outside 0..2", mode);
  if (mode != h->timing) {
    h->timing = mode;
    h->graph_ok = false;
  }
  return FMM_OK;
}

fmm_status fmm_get_stage_times(fmm_handle h, float* out) {
  if (!h || !out) return FMM_ERR_ARG;
  Ctx* c = h;
  if (!c->tev_recorded) return set_err(c, FMM_ERR_STATE, "fmm_get_stage_times: no timed evaluation");
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  auto el = [&](int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->tev[a], c->tev[b]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.f;
    }
    return ms;
  };
  out[0] = el(0, 1);  // P2M + M2M
  out[1] = el(1, 3);  // M2L, all levels
  out[2] = el(1, 2);  // main M2L kernel
  out[3] = el(2, 3);  // rest of M2L
  out[4] = el(3, 4);  // L2L
  out[5] = el(5, 6);  // P2P
  out[6] = el(7, 8);  // L2P + output
  out[7] = el(0, 8);  // whole evaluation (from the branch start)
  return FMM_OK;
}

fmm_status fmm_get_m2l_kernel_times(fmm_handle h, float* out) {
  if (!h || !out) return FMM_ERR_ARG;
  Ctx* c = h;
  const int kind = m2l_kind(c);
  if (!c->tev_recorded || (kind != 2 && kind != 5) || c->ntiles == 0)
    return set_err(c, FMM_ERR_STATE, "fmm_get_m2l_kernel_times: no timed evaluation on the tensor-core M2L path");
  FMM_CUDA(c, cudaStreamSynchronize(c->stream));
  auto el = [&](int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->tev[a], c->tev[b]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.f;
    }
    return ms;
  };
  out[0] = kind == 5 ? el(9, 10) : 0.f;
  out[1] = el(11, 12);
  return FMM_OK;
}

const char* fmm_last_error(fmm_handle h) { return h ? h->err : g_create_err; }

}  // extern "C"
