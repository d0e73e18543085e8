// C-ABI entry points of libmmba (declared in include/ba.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ba.h"
#include "checked.cuh"
#include "mmba_internal.cuh"
#include "mmba_kernels.h"

using namespace mmba;

namespace {

thread_local std::string g_create_error;

struct DevAlloc {
  void* ptr;
  size_t bytes;
};

}  // namespace

struct ba_handle {
  ba_config cfg;
  cudaStream_t stream = nullptr;
  std::string err;
  ba_batch* batch = nullptr;  // batch this handle is in, if any
  int64_t launches = 0;
  bool loaded = false;
  std::vector<DevAlloc> keep;  // problem buffers
  std::vector<DevAlloc> temp;  // freed at the end of a load
  DevLayout L{};
  bool mixed = false;
  LoadInput in_keep{};   // device copies of the inputs (mixed precision re-anchors from them)
  LayoutBuffers lb{};
  MixedBuffers mb{};
  DevMixed X{};
  DevState* d_state = nullptr;
  double* poses2 = nullptr;
  double* planes2 = nullptr;
  double* gH = nullptr;
  double* pred_part = nullptr;
  double* cost_part = nullptr;
  int64_t n_cost = 0;
  double* d_shard = nullptr;  // voxel-sharded solve: this handle's summed trial cost
  // copy stream and events of a load that overlaps the clusters' copy with the set-up
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> copy_events;
  // per-kernel event timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks;  // (kind, index of the start event)
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

ba_status fail(ba_handle* h, ba_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return s;
}

ba_status cuda_fail(ba_handle* h, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(h, BA_ERR_OOM, "%s: out of device memory", what);
  return fail(h, BA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call, what)                          \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

// Library-owned stream-ordered memory pool per device.  Its release threshold
// is unlimited, so memory freed by one problem is reused by the next without
// being unmapped and mapped again (the default pool returns it at every
// synchronisation); ba_release_cached_memory() trims it.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaMemPool_t lib_pool(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep_all = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

void* dev_alloc(ba_handle* h, std::vector<DevAlloc>& list, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h->cfg.alloc) {
    p = h->cfg.alloc(bytes, (void*)h->stream, h->cfg.alloc_ctx);
  } else {
    cudaMemPool_t pool = lib_pool(h->cfg.device);
    const cudaError_t e =
        pool ? cudaMallocFromPoolAsync(&p, bytes, pool, h->stream) : cudaMallocAsync(&p, bytes, h->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) list.push_back({p, bytes});
  return p;
}

void free_list(ba_handle* h, std::vector<DevAlloc>& list) {
  for (auto& a : list) {
    if (h->cfg.free)
      h->cfg.free(a.ptr, a.bytes, (void*)h->stream, h->cfg.alloc_ctx);
    else
      cudaFreeAsync(a.ptr, h->stream);
  }
  list.clear();
}

void* keep_fn(void* self, size_t bytes) {
  ba_handle* h = (ba_handle*)self;
  return dev_alloc(h, h->keep, bytes);
}
void* temp_fn(void* self, size_t bytes) {
  ba_handle* h = (ba_handle*)self;
  return dev_alloc(h, h->temp, bytes);
}

void release_problem(ba_handle* h) {
  free_list(h, h->temp);
  free_list(h, h->keep);
  h->loaded = false;
  h->L = DevLayout{};
  h->lb = LayoutBuffers{};
  h->mb = MixedBuffers{};
  h->X = DevMixed{};
  h->in_keep = LoadInput{};
  h->d_state = nullptr;
  h->poses2 = h->planes2 = h->gH = h->pred_part = h->cost_part = nullptr;
  h->d_shard = nullptr;
}

// small state-control kernel: flags for the solve loop and cost bookkeeping
__global__ void control_kernel(DevState* st, int honor_stop, int reset_stop) {
  st->honor_stop = honor_stop;
  if (reset_stop) st->stop = 0;
}

__global__ void set_state_kernel(DevState* st, double mu, double nu) {
  st->cur = 0;
  if (mu > 0.0) st->mu = mu;
  if (nu > 0.0) st->nu = nu;
  st->consec_reject = 0;
  st->converged = 0;
  st->stop = 0;
  st->scan_pending = 0;
  st->solve_fail_flag = 0;
}

__global__ void copy_current_poses_kernel(const DevState* st, const double* poses2, int64_t n, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = poses2[(int64_t)st->cur * n + i];
}

__global__ void expand_gh_kernel(const double* gH, int32_t n_scans, double* g, double* H) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_scans) return;
  const double* a = gH + (int64_t)j * kGH;
  if (g)
    for (int k = 0; k < 6; ++k) g[6 * (int64_t)j + k] = a[k];
  if (H) {
    int idx = 6;
    for (int r = 0; r < 6; ++r)
      for (int c = r; c < 6; ++c) {
        H[36 * (int64_t)j + 6 * r + c] = a[idx];
        H[36 * (int64_t)j + 6 * c + r] = a[idx];
        ++idx;
      }
  }
}

ba_status read_state(ba_handle* h, DevState* out) {
  CK(h, cudaMemcpyAsync(out, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream), "read state");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (out->wait_timeout == kErrIndex)
    return fail(h, BA_ERR_STATE, "a kernel read an index out of range (checked build)");
  if (out->wait_timeout)
    return fail(h, BA_ERR_TIMEOUT, "a bounded device-side wait gave up (staged copies of the scan pass did not land)");
  return BA_OK;
}

void fill_stats(const DevState& s, double cost_before, int32_t iters_call, ba_stats* out) {
  out->cost = s.cost;
  out->cost_before = cost_before;
  out->mu = s.mu;
  out->nu = s.nu;
  out->last_rho = s.last_rho;
  out->last_pred = s.last_pred;
  out->last_trial_cost = s.last_trial_cost;
  out->iters = s.iters;
  out->accepted = s.accepted;
  out->consec_reject = s.consec_reject;
  out->last_accepted = s.last_accepted;
  out->converged = s.converged;
  out->solve_failed = s.solve_failed;
  out->iters_this_call = iters_call;
  out->reserved = 0;
}

// Voxel pass with the decision folded into its last block (decide_mode as
// for launch_voxel_pass_*).
cudaError_t voxel_pass(ba_handle* h, double* full, int use_trial, int decide_mode) {
  if (h->mixed)
    return launch_voxel_pass_mixed(h->L, h->X, full, h->cost_part, h->pred_part, h->d_state, use_trial, decide_mode,
                                   h->stream);
  return launch_voxel_pass_f64(h->L, h->poses2, h->planes2, full, h->cost_part, h->pred_part, h->d_state, use_trial,
                               decide_mode, h->stream);
}

cudaError_t scan_pass(ba_handle* h, int force) {
  if (h->mixed) return launch_scan_pass_mixed(h->L, h->X, h->poses2, h->gH, h->d_state, force, h->stream);
  return launch_scan_pass_f64(h->L, h->poses2, h->planes2, h->gH, h->d_state, force, h->stream);
}

ba_status evaluate_current(ba_handle* h) {
  // planes, and the summed cost installed as the current cost (last block)
  CK(h, voxel_pass(h, nullptr, 0, 1), "voxel pass");
  CK(h, scan_pass(h, 1), "scan pass");
  h->launches += 2;
  return BA_OK;
}

// Event pair around one launch when profiling (start recorded here, stop by
// the returned index + 1 after the launch).
cudaError_t prof_begin(ba_handle* h, int kind, size_t* idx) {
  if (!h->profiling) return cudaSuccess;
  while (h->ev_pool.size() < h->ev_used + 2) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    h->ev_pool.push_back(e);
  }
  *idx = h->ev_used;
  h->ev_used += 2;
  h->ev_marks.push_back({kind, *idx});
  return cudaEventRecord(h->ev_pool[*idx], h->stream);
}

cudaError_t prof_end(ba_handle* h, size_t idx) {
  if (!h->profiling) return cudaSuccess;
  return cudaEventRecord(h->ev_pool[idx + 1], h->stream);
}

ba_status launch_iteration(ba_handle* h) {
  size_t ev = 0;
  CK(h, prof_begin(h, BA_KERNEL_SOLVE, &ev), "event");
  CK(h, launch_solve_f64(h->L, h->poses2, h->gH, h->pred_part, h->d_state, h->mixed ? h->mb.sref : nullptr,
                         h->mixed ? h->mb.stab2 : nullptr, h->stream),
     "solve");
  CK(h, prof_end(h, ev), "event");
  CK(h, prof_begin(h, BA_KERNEL_VOXEL_PASS, &ev), "event");
  // the trial cost and the LM decision (in the pass's last block)
  CK(h, voxel_pass(h, nullptr, 1, 0), "trial voxel pass");
  CK(h, prof_end(h, ev), "event");
  CK(h, prof_begin(h, BA_KERNEL_SCAN_PASS, &ev), "event");
  CK(h, scan_pass(h, 0), "scan pass");
  CK(h, prof_end(h, ev), "event");
  h->launches += 3;
  return BA_OK;
}

ba_status check_loaded(ba_handle* h) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!h->loaded) return fail(h, BA_ERR_STATE, "no problem loaded");
  return BA_OK;
}

// Copy n bytes of host or device memory into a temporary device buffer
// (device pointers are used in place).
// With own = true the input is always copied into the handle's kept buffers
// (from host or device memory), else host inputs go to temporaries and device
// inputs are read in place.
template <typename T>
const T* stage(ba_handle* h, const T* src, size_t count, int mem_kind, bool own, cudaError_t* err) {
  *err = cudaSuccess;
  if (mem_kind == BA_MEM_DEVICE && !own) return src;
  T* d = (T*)dev_alloc(h, own ? h->keep : h->temp, sizeof(T) * (count ? count : 1));
  if (!d) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  if (count)
    *err = cudaMemcpyAsync(d, src, sizeof(T) * count,
                           mem_kind == BA_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  return d;
}

ba_status check_validation(ba_handle* h, const ValidateResult& res, int32_t n_scans) {
  if (res.first_bad_offset != LLONG_MAX)
    return fail(h, BA_ERR_INVALID_ARG,
                "voxel_offsets must start at 0, increase and end at n_obs (first violation at index %lld)",
                res.first_bad_offset);
  if (res.first_empty_voxel != LLONG_MAX)
    return fail(h, BA_ERR_INVALID_ARG, "voxel %lld has no observation", res.first_empty_voxel);
  if (res.first_bad_scan != LLONG_MAX)
    return fail(h, BA_ERR_INVALID_ARG, "obs_scan[%lld] out of range [0, %d)", res.first_bad_scan, n_scans);
  if (res.first_nonfinite_agg != LLONG_MAX)
    return fail(h, BA_ERR_INVALID_ARG, "cluster %lld has a non-finite value", res.first_nonfinite_agg);
  if (res.first_bad_count != LLONG_MAX)
    return fail(h, BA_ERR_INVALID_ARG, "cluster %lld has a point count below 1", res.first_bad_count);
  if (res.first_bad_pose != LLONG_MAX)
    return fail(h, BA_ERR_INVALID_ARG, "pose %lld is not a finite proper rotation (orthonormal to 1e-6)",
                res.first_bad_pose);
  if (res.max_len >= (1ll << 24))
    return fail(h, BA_ERR_CAPACITY, "a voxel has %lld observations (limit 2^24)", res.max_len);
  return BA_OK;
}

// Waits for the copy stream when a load leaves early while its copies may
// still be writing into buffers that the next load or destroy would free.
struct CopyDrain {
  cudaStream_t s = nullptr;
  ~CopyDrain() {
    if (s) cudaStreamSynchronize(s);
  }
};


ba_status load_impl(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs, const int64_t* voxel_off,
                    const int32_t* obs_scan, const double* agg, int32_t agg_form, const double* poses, int32_t mem_kind,
                    int32_t agg_mem_kind) {
  cudaError_t e;
  LoadInput in{};
  in.n_scans = n_scans;
  in.n_voxels = n_voxels;
  in.n_obs = n_obs;
  in.agg_form = agg_form;
  // mixed precision keeps device copies of the inputs: the FP32 copies are
  // rebuilt from them when the reference poses change (ba_set_state)
  const bool own = h->mixed;
  // A mixed load of host inputs copies the clusters in chunks of input
  // voxels on a copy stream, and sets up each chunk's voxels (frames,
  // anchors, slots staged voxel by voxel in the sorted voxel order) while the
  // next chunk is on its way.
  const bool pipelined = h->mixed && mem_kind == BA_MEM_HOST && agg_mem_kind == BA_MEM_HOST && n_voxels > kWindow;
  in.voxel_off = stage(h, voxel_off, (size_t)n_voxels + 1, mem_kind, own, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage voxel offsets");
  in.obs_scan = stage(h, obs_scan, (size_t)n_obs, mem_kind, own, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage obs_scan");
  if (pipelined) {
    double* d = (double*)dev_alloc(h, h->keep, sizeof(double) * 10 * (size_t)n_obs);
    if (!d) return fail(h, BA_ERR_OOM, "clusters: out of device memory");
    in.agg = d;
  } else {
    in.agg = stage(h, agg, (size_t)n_obs * 10, agg_mem_kind, own, &e);
    if (e != cudaSuccess) return cuda_fail(h, e, "stage clusters");
  }
  in.poses = stage(h, poses, (size_t)n_scans * 12, mem_kind, false, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage poses");

  // The clusters' copy, chunk by chunk, behind the allocation on the handle's
  // stream, started before validation (the copy of a load that fails is
  // drained before the load returns).  The chunk boundaries come from the
  // host offsets, so they are checked here first: every copy stays inside the
  // caller's array and the device buffer, whatever the rest of the offsets hold.
  CopyDrain drain;
  int64_t chunk_v[kMaxCopyChunks + 1] = {0};
  int n_chunks = 0;
  if (pipelined) {
    const int64_t windows = (n_voxels + kWindow - 1) / kWindow;
    // Chunk sizes in windows, halving towards the end (..., 4, 2, 1), the
    // first chunk taking the rest: a chunk's set-up takes less time than the
    // copy of the next chunk, half its size, so the set-ups keep pace and
    // only the last, one-window chunk's is left when the copy ends.
    n_chunks = 1;
    while (n_chunks < kMaxCopyChunks && ((int64_t)1 << n_chunks) - 1 < windows) ++n_chunks;
    int64_t size[kMaxCopyChunks];
    for (int k = 1; k < n_chunks; ++k) size[k] = (int64_t)1 << (n_chunks - 1 - k);
    size[0] = windows - (((int64_t)1 << (n_chunks - 1)) - 1);
    bool bounds_ok = voxel_off[0] == 0 && voxel_off[n_voxels] == n_obs;
    int64_t w_end = 0;
    for (int k = 0; k < n_chunks && bounds_ok; ++k) {
      w_end += size[k];
      chunk_v[k + 1] = std::min(n_voxels, w_end * kWindow);
      const int64_t o0 = voxel_off[chunk_v[k]], o1 = voxel_off[chunk_v[k + 1]];
      bounds_ok = 0 <= o0 && o0 <= o1 && o1 <= n_obs;
    }
    // offsets that fail here fail the device validation below, which names the
    // first violation; no copy is started for them
    if (!bounds_ok) n_chunks = 0;
  }
  if (n_chunks > 0) {
    if (!h->copy_stream) CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream");
    while (h->copy_events.size() < kMaxCopyChunks + 1) {
      cudaEvent_t ev;
      CK(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "copy event");
      h->copy_events.push_back(ev);
    }
    CK(h, cudaEventRecord(h->copy_events[kMaxCopyChunks], h->stream), "copy order");
    CK(h, cudaStreamWaitEvent(h->copy_stream, h->copy_events[kMaxCopyChunks], 0), "copy order");
    drain.s = h->copy_stream;
    for (int k = 0; k < n_chunks; ++k) {
      const int64_t o0 = voxel_off[chunk_v[k]], o1 = voxel_off[chunk_v[k + 1]];
      CK(h, cudaMemcpyAsync(const_cast<double*>(in.agg) + 10 * o0, agg + 10 * o0, sizeof(double) * 10 * (o1 - o0),
                            cudaMemcpyHostToDevice, h->copy_stream),
         "copy clusters");
      CK(h, cudaEventRecord(h->copy_events[k], h->copy_stream), "copy event");
    }
  }

  // validation (the clusters of a pipelined load are checked chunk by chunk)
  ValidateResult init;
  init.first_bad_offset = init.first_empty_voxel = init.first_bad_scan = init.first_bad_count =
      init.first_nonfinite_agg = init.first_bad_pose = LLONG_MAX;
  init.n_obs_seen = 0;
  init.max_len = 0;
  ValidateResult* d_val = (ValidateResult*)dev_alloc(h, h->temp, sizeof(ValidateResult));
  if (!d_val) return fail(h, BA_ERR_OOM, "validation buffer: out of device memory");
  CK(h, cudaMemcpyAsync(d_val, &init, sizeof init, cudaMemcpyHostToDevice, h->stream), "validation init");
  CK(h, launch_validate(in, d_val, !pipelined, h->stream, &h->launches), "validate");
  ValidateResult res;
  CK(h, cudaMemcpyAsync(&res, d_val, sizeof res, cudaMemcpyDeviceToHost, h->stream), "validation result");
  CK(h, cudaStreamSynchronize(h->stream), "validation sync");
  ba_status vs = check_validation(h, res, n_scans);
  if (vs != BA_OK) return vs;
  if (pipelined && n_chunks == 0) return fail(h, BA_ERR_CUDA, "internal: cluster copy not started");

  // layout
  LayoutBuffers& lb = h->lb;
  lb = LayoutBuffers{};
  Allocator keep{keep_fn, h}, temp{temp_fn, h};
  {
    cudaError_t be =
        build_layout(in, (int)res.max_len, !h->mixed, pipelined, keep, temp, &lb, h->stream, &h->launches);
    if (be != cudaSuccess) return cuda_fail(h, be, "layout build");
  }
  DevLayout& L = h->L;
  L.n_scans = n_scans;
  L.fixed_scan = h->cfg.fixed_scan;
  L.n_voxels = n_voxels;
  L.n_obs = n_obs;
  L.n_elems = lb.n_elems;
  L.n_slices = lb.n_slices;
  L.slice_off = lb.slice_off;
  L.vlen = lb.vlen;
  L.vperm = lb.vperm;
  L.ve = lb.ve;
  L.ve_scan = lb.ve_scan;
  L.scan_off = lb.scan_off;
  L.se = lb.se;
  L.se_vox = lb.se_vox;
  {
    // scan-pass block order: scans by decreasing observation count (ties by
    // index), so the longest start first
    std::vector<int64_t> so((size_t)n_scans + 1);
    CK(h, cudaMemcpyAsync(so.data(), lb.scan_off, sizeof(int64_t) * so.size(), cudaMemcpyDeviceToHost, h->stream),
       "scan order");
    CK(h, cudaStreamSynchronize(h->stream), "scan order");
    std::vector<int32_t> ord((size_t)n_scans);
    for (int32_t j = 0; j < n_scans; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int32_t a, int32_t b) { return so[a + 1] - so[a] > so[b + 1] - so[b]; });
    int32_t* d_ord = (int32_t*)dev_alloc(h, h->keep, sizeof(int32_t) * (size_t)n_scans);
    if (!d_ord) return fail(h, BA_ERR_OOM, "scan order: out of device memory");
    CK(h, cudaMemcpyAsync(d_ord, ord.data(), sizeof(int32_t) * ord.size(), cudaMemcpyHostToDevice, h->stream),
       "scan order");
    L.scan_order = d_ord;
  }

  // iteration buffers
  h->n_cost = voxel_pass_blocks(n_voxels);
  h->poses2 = (double*)dev_alloc(h, h->keep, sizeof(double) * 24 * (size_t)n_scans);
  h->planes2 = (double*)dev_alloc(h, h->keep, sizeof(double) * 2 * kPlaneStride * (size_t)n_voxels);
  h->gH = (double*)dev_alloc(h, h->keep, sizeof(double) * kGH * (size_t)n_scans);
  h->pred_part = (double*)dev_alloc(h, h->keep, sizeof(double) * (size_t)n_scans);
  h->cost_part = (double*)dev_alloc(h, h->keep, sizeof(double) * (size_t)h->n_cost);
  h->d_state = (DevState*)dev_alloc(h, h->keep, sizeof(DevState));
  if (!h->poses2 || !h->planes2 || !h->gH || !h->pred_part || !h->cost_part || !h->d_state)
    return fail(h, BA_ERR_OOM, "iteration buffers: out of device memory");
  CK(h, cudaMemcpyAsync(h->poses2, in.poses, sizeof(double) * 12 * (size_t)n_scans, cudaMemcpyDeviceToDevice,
                        h->stream),
     "initial poses");
  if (h->mixed) {
    MixedBuffers& mb = h->mb;
    mb.ve32 = (float4*)dev_alloc(h, h->keep, sizeof(float4) * kVe32 * (size_t)lb.n_elems);
    mb.vstate = (float4*)dev_alloc(h, h->keep, sizeof(float4) * 2 * (size_t)n_voxels);
    // + 16 bytes: the staged scan pass copies the float2 array from even indices to even ends
    mb.se32 = (float*)dev_alloc(h, h->keep, sizeof(float) * 10 * (size_t)n_obs + 16);
    mb.vanchor = (float4*)dev_alloc(h, h->keep, sizeof(float4) * (size_t)n_voxels);
    // FP64 reference poses, their FP32 copy (see scan_ref_kernel), then the FP64
    // quaternions of dR of both pose buffers (sq2_of)
    mb.sref = (double*)dev_alloc(h, h->keep, (18 + 8) * sizeof(double) * (size_t)n_scans);
    mb.stab2 = (float*)dev_alloc(h, h->keep, sizeof(float) * 2 * kTab * (size_t)n_scans);
    mb.planes32_2 = (float4*)dev_alloc(h, h->keep, sizeof(float4) * 2 * 2 * (size_t)n_voxels);
    if (!mb.ve32 || !mb.vstate || !mb.se32 || !mb.vanchor || !mb.sref || !mb.stab2 || !mb.planes32_2)
      return fail(h, BA_ERR_OOM, "mixed-precision copies: out of device memory");
    h->in_keep = in;
    h->in_keep.poses = nullptr;
    if (pipelined) {
      CK(h, build_mixed_begin(in, h->poses2, mb, h->stream, &h->launches), "mixed-precision copies");
      // slots staged in the sorted voxel order and their scan-major entries
      // filled while the chunks arrive, the slots placed in their slices
      // (spatial windows draw voxels from every chunk) at the end
      float4* staging = (float4*)dev_alloc(h, h->temp, sizeof(float4) * 3 * (size_t)n_obs);
      uint32_t* chunk_q = (uint32_t*)dev_alloc(h, h->temp, sizeof(uint32_t) * (size_t)n_obs);
      if (!staging || !chunk_q) return fail(h, BA_ERR_OOM, "slot staging: out of device memory");
      {
        // each chunk's scan-major positions, listed while the first chunk is copied
        ChunkBounds cb{};
        cb.n = n_chunks;
        for (int k = 0; k <= n_chunks; ++k) cb.o[k] = voxel_off[chunk_v[k]];
        CK(h, group_by_chunk(lb.scan_order, n_obs, cb, chunk_q, temp, h->stream, &h->launches), "chunk order");
      }
      for (int k = 0; k < n_chunks; ++k) {
        const int64_t v0 = chunk_v[k], v1 = chunk_v[k + 1];
        CK(h, cudaStreamWaitEvent(h->stream, h->copy_events[k], 0), "wait for clusters");
        CK(h, launch_validate_agg(in, voxel_off[v0], voxel_off[v1], d_val, h->stream, &h->launches), "validate");
        CK(h, launch_vscale(in, v0, v1, lb.vscale, h->stream, &h->launches), "voxel scales");
        CK(h, build_mixed_voxels(in, lb, h->poses2, mb, v0, v1, voxel_off[v0], voxel_off[v1], staging, chunk_q,
                                 h->stream, &h->launches),
           "mixed-precision copies");
      }
      CK(h, build_mixed_place(in, lb, mb, staging, h->stream, &h->launches), "mixed-precision copies");
      CK(h, build_mixed_end(in, lb, h->poses2, mb, h->stream, &h->launches, true), "mixed-precision copies");
      CK(h, cudaMemcpyAsync(&res, d_val, sizeof res, cudaMemcpyDeviceToHost, h->stream), "validation result");
      CK(h, cudaStreamSynchronize(h->stream), "validation sync");
      if ((vs = check_validation(h, res, n_scans)) != BA_OK) return vs;
    } else {
      CK(h, build_mixed(in, lb, h->poses2, mb, h->stream, &h->launches), "mixed-precision copies");
    }
    h->X.ve32 = mb.ve32;
    h->X.vstate = mb.vstate;
    h->X.se32 = mb.se32;
    h->X.vanchor = mb.vanchor;
    h->X.sref = mb.sref;
    h->X.stab2 = mb.stab2;
    h->X.planes32_2 = mb.planes32_2;
  }
  DevState s0{};
  s0.mu = h->cfg.mu0;
  s0.nu = 2.0;
  s0.last_rho = NAN;
  s0.last_pred = NAN;
  s0.last_trial_cost = NAN;
  s0.rel_tol = h->cfg.rel_tol;
  s0.abs_tol = h->cfg.abs_tol;
  s0.max_iters = h->cfg.max_iters;
  s0.max_consec_reject = h->cfg.max_consec_reject;
  s0.hess_mode = h->cfg.hessian_mode;
  CK(h, cudaMemcpyAsync(h->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, h->stream), "state init");
  ba_status st = evaluate_current(h);
  if (st != BA_OK) return st;
  DevState s;
  st = read_state(h, &s);  // also drains the stream before temporaries are freed
  if (st != BA_OK) return st;
  free_list(h, h->temp);
  h->loaded = true;
  if (!std::isfinite(s.cost)) return fail(h, BA_ERR_NUMERIC, "cost at the initial poses is not finite");
  return BA_OK;
}

ba_status check_sizes(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs, int32_t mem_kind) {
  if (n_scans < 1) return fail(h, BA_ERR_INVALID_ARG, "n_scans must be >= 1");
  if (n_scans >= (1 << kPermShift)) return fail(h, BA_ERR_CAPACITY, "n_scans must be below 2^29");
  if (n_voxels < 1) return fail(h, BA_ERR_INVALID_ARG, "n_voxels must be >= 1");
  if (n_obs < n_voxels) return fail(h, BA_ERR_INVALID_ARG, "n_obs must be >= n_voxels (one observation per voxel)");
  if (n_obs >= (1ll << 31) || n_voxels >= (1ll << 31))
    return fail(h, BA_ERR_CAPACITY, "n_obs and n_voxels must be below 2^31");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  return BA_OK;
}

}  // namespace

namespace mmba {
cudaMemPool_t library_pool(int device) { return lib_pool(device); }
}  // namespace mmba

extern "C" {

void ba_config_default(ba_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->precision = BA_FP64;
  cfg->max_iters = 200;
  cfg->rel_tol = 1e-8;
  cfg->abs_tol = 0.0;
  cfg->mu0 = 1e-4;
  cfg->fixed_scan = 0;
  cfg->hessian_mode = BA_HESS_EXACT;
  cfg->max_consec_reject = 10;
  cfg->device = 0;
}

ba_status ba_create(const ba_config* cfg, ba_handle** out) {
  if (!out) return fail(nullptr, BA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ba_config c;
  if (cfg)
    c = *cfg;
  else
    ba_config_default(&c);
  if (c.precision != BA_FP64 && c.precision != BA_MIXED)
    return fail(nullptr, BA_ERR_INVALID_ARG, "precision must be BA_FP64 or BA_MIXED");
  if (c.hessian_mode != BA_HESS_EXACT && c.hessian_mode != BA_HESS_GAUSS_NEWTON)
    return fail(nullptr, BA_ERR_INVALID_ARG, "bad hessian_mode");
  if (!(c.mu0 > 0.0) || !(c.rel_tol >= 0.0) || !(c.abs_tol >= 0.0) || c.max_iters < 0 || c.max_consec_reject < 1)
    return fail(nullptr, BA_ERR_INVALID_ARG, "bad tolerances or limits");
  if ((c.alloc == nullptr) != (c.free == nullptr))
    return fail(nullptr, BA_ERR_INVALID_ARG, "alloc and free must be given together");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail(nullptr, BA_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  if (c.device < 0 || c.device >= ndev) return fail(nullptr, BA_ERR_INVALID_ARG, "device %d out of range", c.device);
  ba_handle* h = new ba_handle();
  h->cfg = c;
  h->stream = (cudaStream_t)c.cuda_stream;
  h->mixed = c.precision == BA_MIXED;
  *out = h;
  return BA_OK;
}

ba_status ba_load_observations(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs,
                               const int64_t* voxel_offsets, const int32_t* obs_scan, const double* agg,
                               int32_t agg_form, const double* poses, int32_t mem_kind) {
  if (!h) return BA_ERR_INVALID_ARG;
  DeviceGuard g(h->cfg.device);
  if (!g.ok) return fail(h, BA_ERR_CUDA, "cudaSetDevice failed");
  ba_status s = check_sizes(h, n_scans, n_voxels, n_obs, mem_kind);
  if (s != BA_OK) return s;
  if (!voxel_offsets || !obs_scan || !agg || !poses) return fail(h, BA_ERR_INVALID_ARG, "NULL input pointer");
  if (agg_form != BA_AGG_RAW_SUMS && agg_form != BA_AGG_CENTRED) return fail(h, BA_ERR_INVALID_ARG, "bad agg_form");
  if (h->cfg.fixed_scan >= n_scans) return fail(h, BA_ERR_INVALID_ARG, "fixed_scan out of range");
  if (h->batch) return fail(h, BA_ERR_STATE, "the handle is in a batch: remove it before loading");
  release_problem(h);
  s = load_impl(h, n_scans, n_voxels, n_obs, voxel_offsets, obs_scan, agg, agg_form, poses, mem_kind, mem_kind);
  if (s != BA_OK) {
    cudaStreamSynchronize(h->stream);
    release_problem(h);
  }
  return s;
}

ba_status ba_load_points(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs, const int64_t* voxel_offsets,
                         const int32_t* obs_scan, const int64_t* point_offsets, const double* points,
                         const double* poses, int32_t mem_kind) {
  if (!h) return BA_ERR_INVALID_ARG;
  DeviceGuard g(h->cfg.device);
  if (!g.ok) return fail(h, BA_ERR_CUDA, "cudaSetDevice failed");
  ba_status s = check_sizes(h, n_scans, n_voxels, n_obs, mem_kind);
  if (s != BA_OK) return s;
  if (!voxel_offsets || !obs_scan || !point_offsets || !points || !poses)
    return fail(h, BA_ERR_INVALID_ARG, "NULL input pointer");
  if (h->cfg.fixed_scan >= n_scans) return fail(h, BA_ERR_INVALID_ARG, "fixed_scan out of range");
  if (h->batch) return fail(h, BA_ERR_STATE, "the handle is in a batch: remove it before loading");
  release_problem(h);
  // point offsets: need the point count to stage the points
  std::vector<int64_t> hoff;
  const int64_t* off_host = point_offsets;
  if (mem_kind == BA_MEM_DEVICE) {
    hoff.resize((size_t)n_obs + 1);
    cudaError_t e = cudaMemcpyAsync(hoff.data(), point_offsets, sizeof(int64_t) * (n_obs + 1), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "read point offsets");
    off_host = hoff.data();
  }
  if (off_host[0] != 0) return fail(h, BA_ERR_INVALID_ARG, "point_offsets[0] must be 0");
  for (int64_t o = 0; o < n_obs; ++o)
    if (off_host[o + 1] <= off_host[o])
      return fail(h, BA_ERR_INVALID_ARG, "observation %lld has no point", (long long)o);
  const int64_t n_points = off_host[n_obs];
  cudaError_t e;
  const int64_t* d_off = stage(h, point_offsets, (size_t)n_obs + 1, mem_kind, false, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage point offsets");
  const double* d_pts = stage(h, points, (size_t)n_points * 3, mem_kind, false, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage points");
  double* d_agg = (double*)dev_alloc(h, h->temp, sizeof(double) * 10 * (size_t)n_obs);
  if (!d_agg) return fail(h, BA_ERR_OOM, "cluster buffer: out of device memory");
  e = launch_aggregate_points(n_obs, d_off, d_pts, d_agg, h->stream);
  ++h->launches;
  if (e != cudaSuccess) return cuda_fail(h, e, "aggregate points");
  s = load_impl(h, n_scans, n_voxels, n_obs, voxel_offsets, obs_scan, d_agg, BA_AGG_CENTRED, poses, mem_kind,
                BA_MEM_DEVICE);
  if (s != BA_OK) {
    cudaStreamSynchronize(h->stream);
    release_problem(h);
  }
  return s;
}

ba_status ba_iterate(ba_handle* h, int32_t n_iters, ba_stats* out) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (n_iters < 0) return fail(h, BA_ERR_INVALID_ARG, "n_iters must be >= 0");
  DeviceGuard g(h->cfg.device);
  double cost_before = NAN;
  if (out) {
    DevState st;
    if ((s = read_state(h, &st)) != BA_OK) return s;
    cost_before = st.cost;
  }
  control_kernel<<<1, 1, 0, h->stream>>>(h->d_state, 0, 1);
  ++h->launches;
  CK(h, cudaGetLastError(), "control");
  for (int32_t k = 0; k < n_iters; ++k)
    if ((s = launch_iteration(h)) != BA_OK) return s;
  if (out) {
    DevState st;
    if ((s = read_state(h, &st)) != BA_OK) return s;
    fill_stats(st, cost_before, n_iters, out);
    if (!std::isfinite(st.cost)) return fail(h, BA_ERR_NUMERIC, "cost is not finite");
  }
  return BA_OK;
}

ba_status ba_solve(ba_handle* h, ba_stats* out) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  DeviceGuard g(h->cfg.device);
  DevState st;
  if ((s = read_state(h, &st)) != BA_OK) return s;
  const double cost_before = st.cost;
  const int32_t iters0 = st.iters;
  control_kernel<<<1, 1, 0, h->stream>>>(h->d_state, 1, 1);
  ++h->launches;
  CK(h, cudaGetLastError(), "control");
  const int chunk = 8;
  for (;;) {
    if (st.iters >= h->cfg.max_iters) break;
    int32_t todo = h->cfg.max_iters - st.iters;
    if (todo > chunk) todo = chunk;
    for (int32_t k = 0; k < todo; ++k)
      if ((s = launch_iteration(h)) != BA_OK) return s;
    if ((s = read_state(h, &st)) != BA_OK) return s;
    if (st.stop) break;
  }
  control_kernel<<<1, 1, 0, h->stream>>>(h->d_state, 0, 0);
  ++h->launches;
  CK(h, cudaGetLastError(), "control");
  if ((s = read_state(h, &st)) != BA_OK) return s;
  if (out) fill_stats(st, cost_before, st.iters - iters0, out);
  if (!std::isfinite(st.cost)) return fail(h, BA_ERR_NUMERIC, "cost is not finite");
  return BA_OK;
}

ba_status ba_poses(ba_handle* h, double* out, int32_t mem_kind) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!out) return fail(h, BA_ERR_INVALID_ARG, "out is NULL");
  DeviceGuard g(h->cfg.device);
  const int64_t n = 12 * (int64_t)h->L.n_scans;
  if (mem_kind == BA_MEM_DEVICE) {
    copy_current_poses_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d_state, h->poses2, n, out);
    ++h->launches;
    CK(h, cudaGetLastError(), "copy poses");
    return BA_OK;
  }
  if (mem_kind != BA_MEM_HOST) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  DevState st;
  if ((s = read_state(h, &st)) != BA_OK) return s;
  CK(h, cudaMemcpyAsync(out, h->poses2 + (int64_t)st.cur * n, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream),
     "read poses");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return BA_OK;
}

ba_status ba_cost(ba_handle* h, double* out) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!out) return fail(h, BA_ERR_INVALID_ARG, "out is NULL");
  DeviceGuard g(h->cfg.device);
  DevState st;
  if ((s = read_state(h, &st)) != BA_OK) return s;
  *out = st.cost;
  return BA_OK;
}

ba_status ba_get_stats(ba_handle* h, ba_stats* out) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!out) return fail(h, BA_ERR_INVALID_ARG, "out is NULL");
  DeviceGuard g(h->cfg.device);
  DevState st;
  if ((s = read_state(h, &st)) != BA_OK) return s;
  fill_stats(st, st.cost, 0, out);
  return BA_OK;
}

ba_status ba_set_state(ba_handle* h, const double* poses, double mu, double nu, int32_t mem_kind) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!poses) return fail(h, BA_ERR_INVALID_ARG, "poses is NULL");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  DeviceGuard g(h->cfg.device);
  const int64_t n = 12 * (int64_t)h->L.n_scans;
  if (mem_kind == BA_MEM_HOST)
    for (int64_t i = 0; i < n; ++i)
      if (!std::isfinite(poses[i])) return fail(h, BA_ERR_INVALID_ARG, "pose value %lld is not finite", (long long)i);
  set_state_kernel<<<1, 1, 0, h->stream>>>(h->d_state, mu, nu);
  ++h->launches;
  CK(h, cudaGetLastError(), "set state");
  CK(h, cudaMemcpyAsync(h->poses2, poses, sizeof(double) * n,
                        mem_kind == BA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream),
     "copy poses");
  // mixed precision: the new poses become the reference poses (re-anchoring)
  if (h->mixed) CK(h, build_mixed(h->in_keep, h->lb, h->poses2, h->mb, h->stream, &h->launches), "re-anchor");
  if ((s = evaluate_current(h)) != BA_OK) return s;
  DevState st;
  if ((s = read_state(h, &st)) != BA_OK) return s;
  if (!std::isfinite(st.cost)) return fail(h, BA_ERR_NUMERIC, "cost is not finite");
  return BA_OK;
}

ba_status ba_planes(ba_handle* h, double* out, int32_t mem_kind) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!out) return fail(h, BA_ERR_INVALID_ARG, "out is NULL");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  DeviceGuard g(h->cfg.device);
  const size_t bytes = sizeof(double) * 9 * (size_t)h->L.n_voxels;
  double* full = mem_kind == BA_MEM_DEVICE ? out : (double*)dev_alloc(h, h->temp, bytes);
  if (!full) return fail(h, BA_ERR_OOM, "plane buffer: out of device memory");
  CK(h, voxel_pass(h, full, 0, -1), "voxel pass");
  ++h->launches;
  if (mem_kind == BA_MEM_HOST) {
    CK(h, cudaMemcpyAsync(out, full, bytes, cudaMemcpyDeviceToHost, h->stream), "read planes");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    free_list(h, h->temp);
  }
  return BA_OK;
}

ba_status ba_gradient(ba_handle* h, double* g, double* H, int32_t mem_kind) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  DeviceGuard guard(h->cfg.device);
  const int32_t ns = h->L.n_scans;
  double *dg = g, *dH = H;
  if (mem_kind == BA_MEM_HOST) {
    dg = g ? (double*)dev_alloc(h, h->temp, sizeof(double) * 6 * (size_t)ns) : nullptr;
    dH = H ? (double*)dev_alloc(h, h->temp, sizeof(double) * 36 * (size_t)ns) : nullptr;
    if ((g && !dg) || (H && !dH)) return fail(h, BA_ERR_OOM, "gradient buffer: out of device memory");
  }
  expand_gh_kernel<<<(ns + 127) / 128, 128, 0, h->stream>>>(h->gH, ns, dg, dH);
  ++h->launches;
  CK(h, cudaGetLastError(), "expand gradient");
  if (mem_kind == BA_MEM_HOST) {
    if (g) CK(h, cudaMemcpyAsync(g, dg, sizeof(double) * 6 * ns, cudaMemcpyDeviceToHost, h->stream), "read g");
    if (H) CK(h, cudaMemcpyAsync(H, dH, sizeof(double) * 36 * ns, cudaMemcpyDeviceToHost, h->stream), "read H");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    free_list(h, h->temp);
  }
  return BA_OK;
}

int64_t ba_kernel_launches(const ba_handle* h) { return h ? h->launches : 0; }

ba_status ba_shard_partials(ba_handle* h, double* gH, double* cost, int32_t mem_kind) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  DeviceGuard g(h->cfg.device);
  const cudaMemcpyKind kind = mem_kind == BA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (gH)
    CK(h, cudaMemcpyAsync(gH, h->gH, sizeof(double) * kGH * (size_t)h->L.n_scans, kind, h->stream), "read g, H");
  if (cost) CK(h, cudaMemcpyAsync(cost, &h->d_state->cost, sizeof(double), kind, h->stream), "read cost");
  if (mem_kind == BA_MEM_HOST) CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return BA_OK;
}

ba_status ba_shard_set_totals(ba_handle* h, const double* gH_total, double cost_total, int32_t mem_kind) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!gH_total) return fail(h, BA_ERR_INVALID_ARG, "gH_total is NULL");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  if (!std::isfinite(cost_total) || cost_total < 0.0) return fail(h, BA_ERR_INVALID_ARG, "cost_total must be finite, >= 0");
  DeviceGuard g(h->cfg.device);
  const cudaMemcpyKind kind = mem_kind == BA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(h, cudaMemcpyAsync(h->gH, gH_total, sizeof(double) * kGH * (size_t)h->L.n_scans, kind, h->stream), "g, H");
  // the host values are consumed before the call returns
  DevState* st = h->d_state;
  const int32_t one = 1;
  CK(h, cudaMemcpyAsync(&st->cost, &cost_total, sizeof(double), cudaMemcpyHostToDevice, h->stream), "cost");
  CK(h, cudaMemcpyAsync(&st->shard, &one, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream), "shard flag");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return BA_OK;
}

ba_status ba_shard_trial(ba_handle* h, double* trial_cost) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  if (!trial_cost) return fail(h, BA_ERR_INVALID_ARG, "trial_cost is NULL");
  DeviceGuard g(h->cfg.device);
  if (!h->d_shard && !(h->d_shard = (double*)dev_alloc(h, h->keep, sizeof(double))))
    return fail(h, BA_ERR_OOM, "out of device memory");
  control_kernel<<<1, 1, 0, h->stream>>>(h->d_state, 0, 1);
  CK(h, cudaGetLastError(), "control");
  CK(h, launch_solve_f64(h->L, h->poses2, h->gH, h->pred_part, h->d_state, h->mixed ? h->mb.sref : nullptr,
                         h->mixed ? h->mb.stab2 : nullptr, h->stream),
     "solve");
  CK(h, voxel_pass(h, nullptr, 1, -1), "trial voxel pass");
  CK(h, launch_shard_cost(h->L, h->cost_part, h->d_shard, h->stream), "trial cost");
  h->launches += 4;
  CK(h, cudaMemcpyAsync(trial_cost, h->d_shard, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read cost");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return BA_OK;
}

ba_status ba_shard_decide(ba_handle* h, double trial_cost_total, int32_t* accepted) {
  ba_status s = check_loaded(h);
  if (s != BA_OK) return s;
  DeviceGuard g(h->cfg.device);
  CK(h, launch_shard_decide(h->L, h->pred_part, h->d_state, trial_cost_total, h->stream), "decide");
  CK(h, scan_pass(h, 0), "scan pass");
  h->launches += 2;
  DevState st;
  if ((s = read_state(h, &st)) != BA_OK) return s;
  if (accepted) *accepted = st.last_accepted;
  if (!std::isfinite(st.cost)) return fail(h, BA_ERR_NUMERIC, "cost is not finite");
  return BA_OK;
}

ba_status ba_release_cached_memory(int32_t device) {
  if (device < 0 || device >= 64) return BA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[device]) return BA_OK;
  DeviceGuard g(device);
  if (!g.ok) return BA_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(g_pools[device], 0) != cudaSuccess) {
    cudaGetLastError();
    return BA_ERR_CUDA;
  }
  return BA_OK;
}

ba_status ba_check_bounded_wait(int32_t device, int32_t polls) {
  if (polls < 1 || polls > 1000000) return BA_ERR_INVALID_ARG;
  DeviceGuard g(device);
  if (!g.ok) return BA_ERR_CUDA;
  int32_t* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int32_t)) != cudaSuccess) return BA_ERR_CUDA;
  int32_t res[2] = {0, 0};
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int32_t));
  if (e == cudaSuccess) e = launch_wait_probe(polls, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(res, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
  // the context must still take work
  if (e == cudaSuccess) e = cudaMemset(d + 1, 0xff, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(res + 1, d + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess || res[1] != -1) return BA_ERR_CUDA;
  return res[0] == 1 ? BA_OK : BA_ERR_TIMEOUT;
}

int64_t ba_device_bytes(const ba_handle* h) {
  if (!h) return 0;
  int64_t b = 0;
  for (auto& a : h->keep) b += (int64_t)a.bytes;
  return b;
}

int64_t ba_estimate_bytes(int32_t precision, int32_t n_scans, int64_t n_voxels, int64_t n_obs, int64_t* peak_extra) {
  // slots of the slice layout exceed n_obs by the padding of each slice (at
  // most the longest voxel's length per 32 voxels); take 1/8 extra plus 64
  const int64_t slots = n_obs + n_obs / 8 + 64;
  int64_t per_obs, per_slot;
  if (precision == BA_MIXED) {
    per_obs = 80 + 4 + 40 + 4 + 4 + 4;  // kept FP64 input, obs_scan, scan-major FP32, se_vox, order, obs_vox
    per_slot = 16 * kVe32;
  } else {
    per_obs = 80 + 4;  // scan-major FP64 copy + se_vox
    per_slot = 80 + 4;
  }
  // (+ 8: the mixed layout's spatial-order observation offsets)
  const int64_t per_voxel = 8 + 4 + 4 + 4 + 8 + 2 * 32 + 16 + 32 + 8 + 2 * 32 + 16 + (precision == BA_MIXED ? 8 : 0);
  const int64_t per_scan = 8 + 24 * 8 + 27 * 8 + 8 + 26 * 8 + 2 * kTab * 4;
  const int64_t keep = per_obs * n_obs + per_slot * slots + per_voxel * n_voxels + per_scan * (int64_t)n_scans +
                       (1 << 16);
  // load: staged inputs (host inputs), sort keys/values and scratch, the
  // spatial order's per-voxel means and prefixes, and (mixed loads of host
  // inputs) the staged slots, the scan-major positions grouped by chunk and
  // that grouping's sort keys, buffers and scratch
  const int64_t nsort = n_obs > n_voxels ? n_obs : n_voxels;
  if (peak_extra)
    *peak_extra = (80 + 4 + 8 + (precision == BA_MIXED ? 16 * kVe32 + 4 + 12 + 2 : 0)) * n_obs + 16 * nsort +
                  24 * nsort / 16 + (8 + 16 + 8 + 8) * (int64_t)n_voxels;
  return keep;
}

ba_status ba_profile_enable(ba_handle* h, int32_t enable) {
  if (!h) return BA_ERR_INVALID_ARG;
  DeviceGuard g(h->cfg.device);
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  h->profiling = enable != 0;
  h->ev_used = 0;
  h->ev_marks.clear();
  return BA_OK;
}

ba_status ba_profile_read(ba_handle* h, int32_t kind, double* total_ms, int64_t* launches) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!total_ms || !launches) return fail(h, BA_ERR_INVALID_ARG, "NULL output");
  DeviceGuard g(h->cfg.device);
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  double tot = 0.0;
  int64_t n = 0;
  for (auto& m : h->ev_marks) {
    if (m.first != kind) continue;
    float ms = 0.0f;
    CK(h, cudaEventElapsedTime(&ms, h->ev_pool[m.second], h->ev_pool[m.second + 1]), "event time");
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *launches = n;
  return BA_OK;
}

void ba_destroy(ba_handle* h) {
  if (!h) return;
  if (h->batch) ba_batch_remove(h->batch, h);
  DeviceGuard g(h->cfg.device);
  cudaStreamSynchronize(h->stream);
  if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
  release_problem(h);
  cudaStreamSynchronize(h->stream);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (auto e : h->copy_events) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
}

const char* ba_last_error(const ba_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

const char* ba_status_string(ba_status s) {
  switch (s) {
    case BA_OK: return "BA_OK";
    case BA_ERR_INVALID_ARG: return "BA_ERR_INVALID_ARG";
    case BA_ERR_OOM: return "BA_ERR_OOM";
    case BA_ERR_CUDA: return "BA_ERR_CUDA";
    case BA_ERR_STATE: return "BA_ERR_STATE";
    case BA_ERR_NUMERIC: return "BA_ERR_NUMERIC";
    case BA_ERR_TIMEOUT: return "BA_ERR_TIMEOUT";
    case BA_ERR_CAPACITY: return "BA_ERR_CAPACITY";
  }
  return "unknown";
}

ba_status ba_aggregate_points(int64_t n_obs, const int64_t* point_offsets, const double* points, double* agg_out,
                              void* stream) {
  if (n_obs < 0) return fail(nullptr, BA_ERR_INVALID_ARG, "n_obs must be >= 0");
  if (n_obs == 0) return BA_OK;
  if (!point_offsets || !points || !agg_out) return fail(nullptr, BA_ERR_INVALID_ARG, "NULL pointer");
  cudaError_t e = launch_aggregate_points(n_obs, point_offsets, points, agg_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, BA_ERR_CUDA, "aggregate points: %s", cudaGetErrorString(e));
  return BA_OK;
}

}  // extern "C"

// ============================================================================
// Batched execution
// ============================================================================

struct ba_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = -1;
  bool mixed = false;
  std::vector<ba_handle*> jobs;
  std::string err;
  int64_t launches = 0;
  // device job table
  JobView* d_jobs = nullptr;
  int64_t* d_prefix = nullptr;  // vblk | sblk | oblk, (n + 1) each
  int32_t* d_done = nullptr;    // per job stop flag, then the active count
  size_t cap = 0;
  int64_t n_vblk = 0, n_sblk = 0, n_oblk = 0;
  // the iteration kernels' job groups (kernel parameters), with each group's
  // voxel-pass, scan-pass and solve block counts
  std::vector<JobGroup> groups;
  std::vector<int64_t> group_blocks;  // 3 per group
  // branch streams and events of the captured graph (group g >= 1 runs on
  // branch g - 1; the groups' jobs are independent)
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> branch_ev;  // fork, then one join per branch
  bool dirty = true;
  // captured iterations
  cudaGraphExec_t graph = nullptr;
  int graph_iters = -1;
  // tuned launch settings of the mixed voxel pass (results do not depend on them)
  int vp_min_blocks = 6;
  int vp_prefetch = 2;
  // per-kernel timing: while on, iterations are launched directly (no graph)
  // with an event pair around each kernel launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks;  // (kernel kind, first event)
};

namespace {

ba_status bfail(ba_batch* b, ba_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  b->err = buf;
  return s;
}

#define BCK(b, call, what)                                                                        \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return bfail(b, BA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

JobView job_view(const ba_handle* h) {
  JobView v{};
  v.L = h->L;
  v.X = h->X;
  v.st = h->d_state;
  v.poses2 = h->poses2;
  v.planes2 = h->planes2;
  v.gH = h->gH;
  v.pred_part = h->pred_part;
  v.cost_part = h->cost_part;
  v.n_cost = h->n_cost;
  return v;
}

JobTable table_of(const ba_batch* b) {
  const size_t n = b->jobs.size();
  JobTable T{};
  T.jobs = b->d_jobs;
  T.vblk = b->d_prefix;
  T.sblk = b->d_prefix + (n + 1);
  T.oblk = b->d_prefix + 2 * (n + 1);
  T.n_jobs = (int32_t)n;
  return T;
}

void drop_graph(ba_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_iters = -1;
}

// (re)upload the job table after a membership change
ba_status refresh(ba_batch* b) {
  if (!b->dirty) return BA_OK;
  const size_t n = b->jobs.size();
  if (n > b->cap) {
    cudaFree(b->d_jobs);
    cudaFree(b->d_prefix);
    cudaFree(b->d_done);
    b->d_jobs = nullptr;
    b->d_prefix = nullptr;
    b->d_done = nullptr;
    size_t cap = n < 16 ? 16 : 2 * n;
    BCK(b, cudaMalloc(&b->d_jobs, sizeof(JobView) * cap), "batch table");
    BCK(b, cudaMalloc(&b->d_prefix, sizeof(int64_t) * 3 * (cap + 1)), "batch table");
    BCK(b, cudaMalloc(&b->d_done, sizeof(int32_t) * (cap + 2)), "batch table");
    b->cap = cap;
  }
  std::vector<JobView> views(n);
  std::vector<int64_t> pre(3 * (n + 1), 0);
  for (size_t k = 0; k < n; ++k) {
    const ba_handle* h = b->jobs[k];
    views[k] = job_view(h);
    pre[k + 1] = pre[k] + voxel_pass_blocks(h->L.n_voxels);
    pre[(n + 1) + k + 1] = pre[(n + 1) + k] + h->L.n_scans;
    pre[2 * (n + 1) + k + 1] = pre[2 * (n + 1) + k] + solve_blocks(h->L.n_scans);
  }
  b->n_vblk = pre[n];
  b->n_sblk = pre[(n + 1) + n];
  b->n_oblk = pre[2 * (n + 1) + n];
  const size_t ng = (n + kGroupJobs - 1) / kGroupJobs;
  b->groups.assign(ng, JobGroup{});
  b->group_blocks.assign(3 * ng, 0);
  for (size_t g = 0; g < ng; ++g) {
    JobGroup& G = b->groups[g];
    const size_t k0 = g * kGroupJobs, k1 = std::min(n, k0 + kGroupJobs);
    G.n_jobs = (int32_t)(k1 - k0);
    int64_t v = 0, sc = 0, o = 0;
    for (size_t k = k0; k < k1; ++k) {
      const int i = (int)(k - k0);
      G.jobs[i] = views[k];
      G.vblk[i] = (int32_t)v;
      G.sblk[i] = (int32_t)sc;
      G.oblk[i] = (int32_t)o;
      v += pre[k + 1] - pre[k];
      sc += pre[(n + 1) + k + 1] - pre[(n + 1) + k];
      o += pre[2 * (n + 1) + k + 1] - pre[2 * (n + 1) + k];
    }
    if (v > INT32_MAX || sc > INT32_MAX || o > INT32_MAX)
      return bfail(b, BA_ERR_CAPACITY, "a group of %d jobs needs more than 2^31 - 1 blocks per launch", G.n_jobs);
    G.vblk[G.n_jobs] = (int32_t)v;
    G.sblk[G.n_jobs] = (int32_t)sc;
    G.oblk[G.n_jobs] = (int32_t)o;
    b->group_blocks[3 * g] = v;
    b->group_blocks[3 * g + 1] = sc;
    b->group_blocks[3 * g + 2] = o;
  }
  if (n) {
    BCK(b, cudaMemcpyAsync(b->d_jobs, views.data(), sizeof(JobView) * n, cudaMemcpyHostToDevice, b->stream),
        "batch table upload");
    BCK(b, cudaMemcpyAsync(b->d_prefix, pre.data(), sizeof(int64_t) * pre.size(), cudaMemcpyHostToDevice, b->stream),
        "batch table upload");
    BCK(b, cudaStreamSynchronize(b->stream), "batch table upload");
  }
  drop_graph(b);
  b->dirty = false;
  return BA_OK;
}

__global__ void batch_control_kernel(JobTable T, int honor_stop, int reset_stop) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_jobs) return;
  DevState* st = T.jobs[k].st;
  st->honor_stop = honor_stop;
  if (reset_stop) st->stop = 0;
}

// done[k] = stop flag of job k; done[n] = jobs still running; done[n + 1] =
// jobs whose bounded device-side waits gave up
__global__ void batch_status_kernel(JobTable T, int32_t* done) {
  __shared__ int32_t active, timeouts;
  if (threadIdx.x == 0) active = timeouts = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < T.n_jobs; k += blockDim.x) {
    const int32_t s = T.jobs[k].st->stop;
    done[k] = s;
    if (!s) atomicAdd(&active, 1);
    if (T.jobs[k].st->wait_timeout) atomicAdd(&timeouts, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    done[T.n_jobs] = active;
    done[T.n_jobs + 1] = timeouts;
  }
}

// event pair around one launch when profiling (start recorded here, stop at
// the returned index + 1 after the launch)
cudaError_t bprof_begin(ba_batch* b, int kind, cudaStream_t stream, size_t* idx) {
  if (!b->profiling) return cudaSuccess;
  while (b->ev_pool.size() < b->ev_used + 2) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    b->ev_pool.push_back(e);
  }
  *idx = b->ev_used;
  b->ev_used += 2;
  b->ev_marks.push_back({kind, *idx});
  return cudaEventRecord(b->ev_pool[*idx], stream);
}

cudaError_t bprof_end(ba_batch* b, cudaStream_t stream, size_t idx) {
  if (!b->profiling) return cudaSuccess;
  return cudaEventRecord(b->ev_pool[idx + 1], stream);
}

// one iteration of the jobs of group g, on stream
ba_status launch_group_iteration(ba_batch* b, size_t g, cudaStream_t stream) {
  const JobGroup& G = b->groups[g];
  const int64_t* nb = &b->group_blocks[3 * g];
  size_t ev = 0;
  BCK(b, bprof_begin(b, BA_KERNEL_SOLVE, stream, &ev), "event");
  BCK(b, launch_batch_solve(G, nb[2], stream), "batch solve");
  BCK(b, bprof_end(b, stream, ev), "event");
  BCK(b, bprof_begin(b, BA_KERNEL_VOXEL_PASS, stream, &ev), "event");
  BCK(b, b->mixed ? launch_batch_voxel_pass_mixed(G, nb[0], 1, stream, b->vp_min_blocks, b->vp_prefetch)
                  : launch_batch_voxel_pass_f64(G, nb[0], 1, stream),
      "batch voxel pass");
  BCK(b, bprof_end(b, stream, ev), "event");
  BCK(b, bprof_begin(b, BA_KERNEL_SCAN_PASS, stream, &ev), "event");
  BCK(b, b->mixed ? launch_batch_scan_pass_mixed(G, nb[1], stream) : launch_batch_scan_pass_f64(G, nb[1], stream),
      "batch scan pass");
  BCK(b, bprof_end(b, stream, ev), "event");
  return BA_OK;
}

// work a member queued on its own stream must finish before the batch's
ba_status sync_members(ba_batch* b) {
  std::vector<cudaStream_t> seen;
  for (auto* h : b->jobs) {
    bool dup = false;
    for (auto s : seen) dup = dup || s == h->stream;
    if (dup) continue;
    seen.push_back(h->stream);
    BCK(b, cudaStreamSynchronize(h->stream), "synchronize member stream");
  }
  return BA_OK;
}

// n iterations as one CUDA graph (captured on first use for this count)
ba_status prepare_graph(ba_batch* b, int n) {
  if (b->graph_iters != n) {
    drop_graph(b);
    const size_t ng = b->groups.size();
    while (b->branch.size() + 1 < ng) {
      cudaStream_t st = nullptr;
      BCK(b, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "branch stream");
      b->branch.push_back(st);
    }
    while (b->branch_ev.size() < ng) {
      cudaEvent_t ev = nullptr;
      BCK(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "branch event");
      b->branch_ev.push_back(ev);
    }
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    // group 0 on the batch's stream, every other group on a branch forked
    // from it and joined back at the end
    ba_status s = BA_OK;
    cudaError_t e = cudaSuccess;
    if (ng > 1) {
      e = cudaEventRecord(b->branch_ev[0], b->stream);
      for (size_t k = 1; k < ng && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->branch[k - 1], b->branch_ev[0], 0);
    }
    if (e != cudaSuccess) s = bfail(b, BA_ERR_CUDA, "graph fork: %s", cudaGetErrorString(e));
    for (size_t grp = 0; grp < ng && s == BA_OK; ++grp) {
      cudaStream_t st = grp == 0 ? b->stream : b->branch[grp - 1];
      for (int k = 0; k < n && s == BA_OK; ++k) s = launch_group_iteration(b, grp, st);
    }
    for (size_t k = 1; k < ng; ++k) {
      cudaError_t ej = cudaEventRecord(b->branch_ev[k], b->branch[k - 1]);
      if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->stream, b->branch_ev[k], 0);
      if (ej != cudaSuccess && s == BA_OK) s = bfail(b, BA_ERR_CUDA, "graph join: %s", cudaGetErrorString(ej));
    }
    e = cudaStreamEndCapture(b->stream, &g);
    if (s != BA_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    BCK(b, e, "graph capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    BCK(b, e, "graph instantiate");
    b->graph_iters = n;
  }
  return BA_OK;
}

ba_status run_iterations(ba_batch* b, int n) {
  if (b->profiling) {  // direct launches, groups one after another on the batch's stream
    for (int k = 0; k < n; ++k)
      for (size_t grp = 0; grp < b->groups.size(); ++grp) {
        ba_status s = launch_group_iteration(b, grp, b->stream);
        if (s != BA_OK) return s;
      }
    b->launches += 3 * (int64_t)n * (int64_t)b->groups.size();
    return BA_OK;
  }
  ba_status s = prepare_graph(b, n);
  if (s != BA_OK) return s;
  BCK(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
  b->launches += 3 * (int64_t)n * (int64_t)b->groups.size();
  return BA_OK;
}

// jobs still running (after the work queued so far)
ba_status active_jobs(ba_batch* b, int32_t* active) {
  const JobTable T = table_of(b);
  batch_status_kernel<<<1, 256, 0, b->stream>>>(T, b->d_done);
  ++b->launches;
  BCK(b, cudaGetLastError(), "batch status");
  int32_t counts[2] = {0, 0};
  BCK(b, cudaMemcpyAsync(counts, b->d_done + T.n_jobs, sizeof(counts), cudaMemcpyDeviceToHost, b->stream), "status");
  BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
  if (counts[1]) return bfail(b, BA_ERR_TIMEOUT, "%d job(s): a bounded device-side wait gave up", counts[1]);
  *active = counts[0];
  return BA_OK;
}

}  // namespace

extern "C" {

ba_status ba_batch_create(void* stream, ba_batch** out) {
  if (!out) return BA_ERR_INVALID_ARG;
  *out = nullptr;
  ba_batch* b = new ba_batch();
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    // graphs cannot be captured on the legacy default stream: use a private one
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(nullptr, BA_ERR_CUDA, "batch stream creation failed");
    }
    b->own_stream = true;
  }
  *out = b;
  return BA_OK;
}

ba_status ba_batch_add(ba_batch* b, ba_handle* h) {
  if (!b || !h) return BA_ERR_INVALID_ARG;
  if (!h->loaded) return bfail(b, BA_ERR_STATE, "the handle has no problem loaded");
  if (h->batch) return bfail(b, BA_ERR_INVALID_ARG, "the handle is already in a batch");
  if (!b->jobs.empty()) {
    if (h->cfg.device != b->device) return bfail(b, BA_ERR_INVALID_ARG, "device differs from the batch's");
    if (h->mixed != b->mixed) return bfail(b, BA_ERR_INVALID_ARG, "precision differs from the batch's");
  } else {
    b->device = h->cfg.device;
    b->mixed = h->mixed;
  }
  DeviceGuard g(h->cfg.device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bfail(b, BA_ERR_CUDA, "synchronize job: %s", cudaGetErrorString(e));
  b->jobs.push_back(h);
  h->batch = b;
  b->dirty = true;
  return BA_OK;
}

ba_status ba_batch_remove(ba_batch* b, ba_handle* h) {
  if (!b || !h) return BA_ERR_INVALID_ARG;
  for (size_t k = 0; k < b->jobs.size(); ++k)
    if (b->jobs[k] == h) {
      DeviceGuard g(b->device);
      cudaStreamSynchronize(b->stream);
      b->jobs.erase(b->jobs.begin() + (long)k);
      h->batch = nullptr;
      b->dirty = true;
      return BA_OK;
    }
  return bfail(b, BA_ERR_INVALID_ARG, "the handle is not in this batch");
}

int32_t ba_batch_size(const ba_batch* b) { return b ? (int32_t)b->jobs.size() : 0; }

int64_t ba_batch_kernel_launches(const ba_batch* b) { return b ? b->launches : 0; }

ba_status ba_batch_iterate(ba_batch* b, int32_t n_iters) {
  if (!b) return BA_ERR_INVALID_ARG;
  if (n_iters < 0) return bfail(b, BA_ERR_INVALID_ARG, "n_iters must be >= 0");
  if (b->jobs.empty() || n_iters == 0) return BA_OK;
  DeviceGuard g(b->device);
  ba_status s = refresh(b);
  if (s != BA_OK) return s;
  if ((s = sync_members(b)) != BA_OK) return s;
  const JobTable T = table_of(b);
  batch_control_kernel<<<(T.n_jobs + 127) / 128, 128, 0, b->stream>>>(T, 0, 1);
  ++b->launches;
  BCK(b, cudaGetLastError(), "batch control");
  if ((s = run_iterations(b, n_iters)) != BA_OK) return s;
  batch_status_kernel<<<1, 256, 0, b->stream>>>(T, b->d_done);
  ++b->launches;
  BCK(b, cudaGetLastError(), "batch status");
  int32_t timeouts = 0;
  BCK(b, cudaMemcpyAsync(&timeouts, b->d_done + T.n_jobs + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream),
      "status");
  BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
  if (timeouts) return bfail(b, BA_ERR_TIMEOUT, "%d job(s): a bounded device-side wait gave up", timeouts);
  return BA_OK;
}

ba_status ba_batch_solve(ba_batch* b, int32_t chunk, int32_t max_rounds, int32_t* n_active_out) {
  if (!b) return BA_ERR_INVALID_ARG;
  if (chunk < 1) return bfail(b, BA_ERR_INVALID_ARG, "chunk must be >= 1");
  if (n_active_out) *n_active_out = 0;
  if (b->jobs.empty()) return BA_OK;
  DeviceGuard g(b->device);
  ba_status s = refresh(b);
  if (s != BA_OK) return s;
  if ((s = sync_members(b)) != BA_OK) return s;
  const JobTable T = table_of(b);
  const int n = T.n_jobs;
  batch_control_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(T, 1, 0);
  ++b->launches;
  BCK(b, cudaGetLastError(), "batch control");
  int32_t active = n;
  for (int round = 0; max_rounds <= 0 || round < max_rounds; ++round) {
    if ((s = run_iterations(b, chunk)) != BA_OK) return s;
    batch_status_kernel<<<1, 256, 0, b->stream>>>(T, b->d_done);
    ++b->launches;
    BCK(b, cudaGetLastError(), "batch status");
    int32_t counts[2] = {0, 0};
    BCK(b, cudaMemcpyAsync(counts, b->d_done + n, sizeof(counts), cudaMemcpyDeviceToHost, b->stream), "status");
    BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
    active = counts[0];
    if (counts[1]) return bfail(b, BA_ERR_TIMEOUT, "%d job(s): a bounded device-side wait gave up", counts[1]);
    if (active == 0) break;
  }
  if (n_active_out) *n_active_out = active;
  return BA_OK;
}

ba_status ba_batch_done(ba_batch* b, int32_t* done_out) {
  if (!b || !done_out) return BA_ERR_INVALID_ARG;
  if (b->jobs.empty()) return BA_OK;
  DeviceGuard g(b->device);
  ba_status s = refresh(b);
  if (s != BA_OK) return s;
  const JobTable T = table_of(b);
  batch_status_kernel<<<1, 256, 0, b->stream>>>(T, b->d_done);
  ++b->launches;
  BCK(b, cudaGetLastError(), "batch status");
  BCK(b, cudaMemcpyAsync(done_out, b->d_done, sizeof(int32_t) * T.n_jobs, cudaMemcpyDeviceToHost, b->stream),
      "status");
  BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
  return BA_OK;
}

ba_status ba_batch_autotune(ba_batch* b, int32_t iters_per_trial, int32_t passes, ba_tune_report* out) {
  if (!b || !out) return BA_ERR_INVALID_ARG;
  if (iters_per_trial < 1 || passes < 1) return bfail(b, BA_ERR_INVALID_ARG, "iters_per_trial and passes must be >= 1");
  *out = ba_tune_report{};
  out->chosen = -1;
  if (b->jobs.empty() || !b->mixed) return BA_OK;  // the FP64 voxel pass has no such knobs
  DeviceGuard g(b->device);
  ba_status s = refresh(b);
  if (s != BA_OK) return s;
  if ((s = sync_members(b)) != BA_OK) return s;
  const JobTable T = table_of(b);
  batch_control_kernel<<<(T.n_jobs + 127) / 128, 128, 0, b->stream>>>(T, 1, 0);  // these are solve iterations
  ++b->launches;
  BCK(b, cudaGetLastError(), "batch control");
  const int mb[3] = {4, 6, 8}, pf[3] = {0, 2, 4};
  int n = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j, ++n) {
      out->min_blocks[n] = mb[i];
      out->prefetch[n] = pf[j];
    }
  out->n_candidates = n;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(b, cudaEventCreate(&e0), "tuner events");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfail(b, BA_ERR_CUDA, "tuner events");
  }
  struct Events {
    cudaEvent_t a, b;
    ~Events() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  const int keep_mb = b->vp_min_blocks, keep_pf = b->vp_prefetch;
  std::vector<double> sum(n, 0.0);
  int full_passes = 0;
  // candidates interleaved pass by pass, so that jobs stopping along the way
  // (less work per iteration) affect every candidate alike; only complete
  // passes with every job still running count
  for (int pass = 0; pass < passes; ++pass) {
    std::vector<double> ms(n, 0.0);
    for (int c = 0; c < n; ++c) {
      if (b->vp_min_blocks != out->min_blocks[c] || b->vp_prefetch != out->prefetch[c]) {
        b->vp_min_blocks = out->min_blocks[c];
        b->vp_prefetch = out->prefetch[c];
        drop_graph(b);
      }
      if ((s = prepare_graph(b, iters_per_trial)) != BA_OK) return s;
      BCK(b, cudaEventRecord(e0, b->stream), "tuner events");
      BCK(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
      b->launches += 3 * (int64_t)iters_per_trial * (int64_t)b->groups.size();
      BCK(b, cudaEventRecord(e1, b->stream), "tuner events");
      BCK(b, cudaEventSynchronize(e1), "tuner events");
      float t = 0.f;
      BCK(b, cudaEventElapsedTime(&t, e0, e1), "tuner events");
      ms[c] = t / iters_per_trial;
    }
    int32_t active = 0;
    if ((s = active_jobs(b, &active)) != BA_OK) return s;
    if (active < T.n_jobs) break;  // a job stopped during this pass: the pass is not comparable
    for (int c = 0; c < n; ++c) sum[c] += ms[c];
    ++full_passes;
  }
  out->passes = full_passes;
  if (full_passes == 0) {
    b->vp_min_blocks = keep_mb;
    b->vp_prefetch = keep_pf;
  } else {
    int best = 0;
    for (int c = 0; c < n; ++c) {
      out->ms_per_iter[c] = sum[c] / full_passes;
      if (sum[c] < sum[best]) best = c;
    }
    out->chosen = best;
    b->vp_min_blocks = out->min_blocks[best];
    b->vp_prefetch = out->prefetch[best];
  }
  drop_graph(b);
  return BA_OK;
}

ba_status ba_batch_profile_enable(ba_batch* b, int32_t enable) {
  if (!b) return BA_ERR_INVALID_ARG;
  if (b->device >= 0) {
    DeviceGuard g(b->device);
    BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
  }
  b->profiling = enable != 0;
  b->ev_used = 0;
  b->ev_marks.clear();
  return BA_OK;
}

ba_status ba_batch_profile_read(ba_batch* b, int32_t kind, double* total_ms, int64_t* launches) {
  if (!b) return BA_ERR_INVALID_ARG;
  if (!total_ms || !launches) return bfail(b, BA_ERR_INVALID_ARG, "NULL output");
  double tot = 0.0;
  int64_t n = 0;
  if (!b->ev_marks.empty()) {
    DeviceGuard g(b->device);
    BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
    for (auto& m : b->ev_marks) {
      if (m.first != kind) continue;
      float ms = 0.0f;
      BCK(b, cudaEventElapsedTime(&ms, b->ev_pool[m.second], b->ev_pool[m.second + 1]), "event time");
      tot += ms;
      ++n;
    }
  }
  *total_ms = tot;
  *launches = n;
  return BA_OK;
}

ba_status ba_batch_set_launch(ba_batch* b, int32_t min_blocks, int32_t prefetch) {
  if (!b) return BA_ERR_INVALID_ARG;
  if ((min_blocks != 4 && min_blocks != 6 && min_blocks != 8) || prefetch < 0 || prefetch > 16)
    return bfail(b, BA_ERR_INVALID_ARG, "min_blocks must be 4, 6 or 8 and prefetch in [0, 16]");
  if (b->vp_min_blocks != min_blocks || b->vp_prefetch != prefetch) {
    b->vp_min_blocks = min_blocks;
    b->vp_prefetch = prefetch;
    drop_graph(b);
  }
  return BA_OK;
}

void ba_batch_destroy(ba_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device >= 0 ? b->device : 0);
  cudaStreamSynchronize(b->stream);
  for (auto* h : b->jobs) h->batch = nullptr;
  drop_graph(b);
  cudaFree(b->d_jobs);
  cudaFree(b->d_prefix);
  cudaFree(b->d_done);
  for (auto st : b->branch) cudaStreamDestroy(st);
  for (auto ev : b->branch_ev) cudaEventDestroy(ev);
  for (auto ev : b->ev_pool) cudaEventDestroy(ev);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* ba_batch_last_error(const ba_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
