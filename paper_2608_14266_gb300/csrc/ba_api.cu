// C-ABI entry points of libmmba (declared in include/ba.h).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ba.h"
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
  int64_t launches = 0;
  bool loaded = false;
  std::vector<DevAlloc> keep;  // problem buffers
  std::vector<DevAlloc> temp;  // freed at the end of a load
  DevLayout L{};
  DevState* d_state = nullptr;
  double* poses2 = nullptr;
  double* planes2 = nullptr;
  double* gH = nullptr;
  double* pred_part = nullptr;
  double* cost_part = nullptr;
  int64_t n_cost = 0;
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

void* dev_alloc(ba_handle* h, std::vector<DevAlloc>& list, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h->cfg.alloc) {
    p = h->cfg.alloc(bytes, (void*)h->stream, h->cfg.alloc_ctx);
  } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
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
  h->d_state = nullptr;
  h->poses2 = h->planes2 = h->gH = h->pred_part = h->cost_part = nullptr;
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

// Evaluate planes, cost, gradient and Hessian at the current poses.
ba_status evaluate_current(ba_handle* h) {
  CK(h, launch_voxel_pass_f64(h->L, h->poses2, h->planes2, nullptr, h->cost_part, h->d_state, 0, h->stream),
     "voxel pass");
  CK(h, launch_decide(h->cost_part, h->n_cost, h->pred_part, h->L.n_scans, h->d_state, 1, h->stream), "cost sum");
  CK(h, launch_scan_pass_f64(h->L, h->poses2, h->planes2, h->gH, h->d_state, 1, h->stream), "scan pass");
  h->launches += 3;
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
  CK(h, launch_solve_f64(h->L, h->poses2, h->gH, h->pred_part, h->d_state, h->stream), "solve");
  CK(h, prof_end(h, ev), "event");
  CK(h, prof_begin(h, BA_KERNEL_VOXEL_PASS, &ev), "event");
  CK(h, launch_voxel_pass_f64(h->L, h->poses2, h->planes2, nullptr, h->cost_part, h->d_state, 1, h->stream),
     "trial voxel pass");
  CK(h, prof_end(h, ev), "event");
  CK(h, prof_begin(h, BA_KERNEL_DECIDE, &ev), "event");
  CK(h, launch_decide(h->cost_part, h->n_cost, h->pred_part, h->L.n_scans, h->d_state, 0, h->stream), "decide");
  CK(h, prof_end(h, ev), "event");
  CK(h, prof_begin(h, BA_KERNEL_SCAN_PASS, &ev), "event");
  CK(h, launch_scan_pass_f64(h->L, h->poses2, h->planes2, h->gH, h->d_state, 0, h->stream), "scan pass");
  CK(h, prof_end(h, ev), "event");
  h->launches += 4;
  return BA_OK;
}

ba_status check_loaded(ba_handle* h) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!h->loaded) return fail(h, BA_ERR_STATE, "no problem loaded");
  return BA_OK;
}

// Copy n bytes of host or device memory into a temporary device buffer
// (device pointers are used in place).
template <typename T>
const T* stage(ba_handle* h, const T* src, size_t count, int mem_kind, cudaError_t* err) {
  *err = cudaSuccess;
  if (mem_kind == BA_MEM_DEVICE) return src;
  T* d = (T*)dev_alloc(h, h->temp, sizeof(T) * (count ? count : 1));
  if (!d) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  if (count) *err = cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, h->stream);
  return d;
}

ba_status load_impl(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs, const int64_t* voxel_off,
                    const int32_t* obs_scan, const double* agg, int32_t agg_form, const double* poses, int32_t mem_kind,
                    int32_t agg_mem_kind) {
  cudaError_t e;
  LoadInput in{};
  in.n_scans = n_scans;
  in.n_voxels = n_voxels;
  in.n_obs = n_obs;
  in.agg_form = agg_form;
  in.voxel_off = stage(h, voxel_off, (size_t)n_voxels + 1, mem_kind, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage voxel offsets");
  in.obs_scan = stage(h, obs_scan, (size_t)n_obs, mem_kind, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage obs_scan");
  in.agg = stage(h, agg, (size_t)n_obs * 10, agg_mem_kind, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage clusters");
  in.poses = stage(h, poses, (size_t)n_scans * 12, mem_kind, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage poses");

  // validation
  ValidateResult init;
  init.first_bad_offset = init.first_empty_voxel = init.first_bad_scan = init.first_bad_count =
      init.first_nonfinite_agg = init.first_bad_pose = LLONG_MAX;
  init.n_obs_seen = 0;
  init.max_len = 0;
  ValidateResult* d_val = (ValidateResult*)dev_alloc(h, h->temp, sizeof(ValidateResult));
  if (!d_val) return fail(h, BA_ERR_OOM, "validation buffer: out of device memory");
  CK(h, cudaMemcpyAsync(d_val, &init, sizeof init, cudaMemcpyHostToDevice, h->stream), "validation init");
  CK(h, launch_validate(in, d_val, h->stream, &h->launches), "validate");
  ValidateResult res;
  CK(h, cudaMemcpyAsync(&res, d_val, sizeof res, cudaMemcpyDeviceToHost, h->stream), "validation result");
  CK(h, cudaStreamSynchronize(h->stream), "validation sync");
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

  // layout
  LayoutBuffers lb{};
  Allocator keep{keep_fn, h}, temp{temp_fn, h};
  {
    cudaError_t be = build_layout(in, (int)res.max_len, keep, temp, &lb, h->stream, &h->launches);
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
  if (n_voxels < 1) return fail(h, BA_ERR_INVALID_ARG, "n_voxels must be >= 1");
  if (n_obs < n_voxels) return fail(h, BA_ERR_INVALID_ARG, "n_obs must be >= n_voxels (one observation per voxel)");
  if (n_obs >= (1ll << 31) || n_voxels >= (1ll << 31))
    return fail(h, BA_ERR_CAPACITY, "n_obs and n_voxels must be below 2^31");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return fail(h, BA_ERR_INVALID_ARG, "bad mem_kind");
  return BA_OK;
}

}  // namespace

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
  if (c.precision == BA_MIXED)
    return fail(nullptr, BA_ERR_INVALID_ARG, "BA_MIXED is not available in this build");
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
  const int64_t* d_off = stage(h, point_offsets, (size_t)n_obs + 1, mem_kind, &e);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage point offsets");
  const double* d_pts = stage(h, points, (size_t)n_points * 3, mem_kind, &e);
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
  CK(h, launch_voxel_pass_f64(h->L, h->poses2, h->planes2, full, h->cost_part, h->d_state, 0, h->stream),
     "voxel pass");
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
  DeviceGuard g(h->cfg.device);
  cudaStreamSynchronize(h->stream);
  release_problem(h);
  cudaStreamSynchronize(h->stream);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
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
