// Preprocessing on the device (Sec. IV-B, Algorithm 1): L1 voxelisation of
// raw scans (Eq. 4), bottom-up voxel levels (Eq. 5, BottomUpVoxelization),
// selection by planarity (Selection), and the voxel-major observation list
// that ba_load_observations takes.
//
// Order of the output (shared with the CPU reference of the tests): voxels by
// level, then by integer index (x, y, z); the observations of a voxel by scan.
// The arithmetic that decides indices and forms clusters uses explicitly
// rounded operations (no contraction), so indices and clusters do not depend
// on the compiler's choices.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/ba.h"
#include "mmba_internal.cuh"
#include "mmba_kernels.h"

using namespace mmba;

namespace {

constexpr long long kKeyRange = 1ll << 20;  // indices in [-2^20, 2^20) per axis
constexpr int kKeyBits = 63;                // 21 bits per axis

__device__ __forceinline__ uint64_t pack_key(long long ix, long long iy, long long iz) {
  return ((uint64_t)(ix + kKeyRange) << 42) | ((uint64_t)(iy + kKeyRange) << 21) | (uint64_t)(iz + kKeyRange);
}

__device__ __forceinline__ void unpack_key(uint64_t k, long long* i) {
  i[0] = (long long)((k >> 42) & 0x1fffffull) - kKeyRange;
  i[1] = (long long)((k >> 21) & 0x1fffffull) - kKeyRange;
  i[2] = (long long)(k & 0x1fffffull) - kKeyRange;
}

__device__ __forceinline__ long long half_floor(long long i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

// scan offsets: start at 0, never decrease, end at n (first violation, or
// LLONG_MAX); poses finite
__global__ void check_inputs_kernel(int32_t n_scans, const int64_t* spo, int64_t n, const double* poses,
                                    long long* bad_off, long long* bad_pose) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n_scans) return;
  if (j == 0 && spo[0] != 0) atomicMin(bad_off, 0ll);
  if (j == n_scans) {
    if (spo[j] != n) atomicMin(bad_off, (long long)j);
    return;
  }
  if (spo[j + 1] < spo[j]) atomicMin(bad_off, (long long)(j + 1));
  bool fin = true;
  for (int k = 0; k < 12; ++k) fin = fin && isfinite(poses[12 * (int64_t)j + k]);
  if (!fin) atomicMin(bad_pose, (long long)j);
}

// L1 (Eq. 4): world point w = R p + t, index floor(w / d), 64-bit key
__global__ void l1_keys_kernel(int32_t n_scans, const int64_t* spo, const double* pts, const double* poses, double d,
                               int64_t n, uint64_t* keys, uint32_t* vals, int32_t* pscan, long long* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_scans;  // the scan of point i: the last j with spo[j] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (spo[mid] <= i)
      lo = mid;
    else
      hi = mid;
  }
  const double* T = poses + 12 * (int64_t)lo;
  const double* p = pts + 3 * i;
  long long ix[3];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double w = fma(T[3 * a], p[0], fma(T[3 * a + 1], p[1], fma(T[3 * a + 2], p[2], T[9 + a])));
    const double f = floor(__ddiv_rn(w, d));
    ok = ok && f >= -(double)kKeyRange && f < (double)kKeyRange;
    ix[a] = ok ? (long long)f : 0;
  }
  if (!ok) atomicMin(bad, (long long)i);
  keys[i] = pack_key(ix[0], ix[1], ix[2]);
  vals[i] = (uint32_t)i;
  pscan[i] = lo;
}

// 1 where a new (key, scan) group starts in sorted order
__device__ __forceinline__ bool group_head(int64_t i, const uint64_t* keys, const uint32_t* vals, const int32_t* scan) {
  return i == 0 || keys[i] != keys[i - 1] || scan[vals[i]] != scan[vals[i - 1]];
}

__global__ void heads_kernel(int64_t n, const uint64_t* keys, const uint32_t* vals, const int32_t* scan,
                             int64_t* pos) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pos[i] = group_head(i, keys, vals, scan) ? 1 : 0;
}

// after the exclusive scan: start of every group, and the end sentinel
__global__ void starts_kernel(int64_t n, const uint64_t* keys, const uint32_t* vals, const int32_t* scan,
                              const int64_t* pos, int64_t* start, int64_t n_groups) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && group_head(i, keys, vals, scan)) start[pos[i]] = i;
  if (i == 0) start[n_groups] = n;
}

// L1 clusters (Eq. 2, centred): mean, then scatter about it, over the group's
// points in point order
__global__ void l1_clusters_kernel(int64_t n1, const int64_t* start, const uint32_t* vals, const uint64_t* keys,
                                   const int32_t* pscan, const double* pts, double* c, uint64_t* ckey,
                                   int32_t* cscan) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n1) return;
  const int64_t a = start[g], b = start[g + 1];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t k = a; k < b; ++k) {
    const double* p = pts + 3 * (int64_t)vals[k];
    s0 = __dadd_rn(s0, p[0]);
    s1 = __dadd_rn(s1, p[1]);
    s2 = __dadd_rn(s2, p[2]);
  }
  const double n = (double)(b - a);
  const double m0 = __ddiv_rn(s0, n), m1 = __ddiv_rn(s1, n), m2 = __ddiv_rn(s2, n);
  double S[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = a; k < b; ++k) {
    const double* p = pts + 3 * (int64_t)vals[k];
    const double x = __dsub_rn(p[0], m0), y = __dsub_rn(p[1], m1), z = __dsub_rn(p[2], m2);
    S[0] = __dadd_rn(S[0], __dmul_rn(x, x));
    S[1] = __dadd_rn(S[1], __dmul_rn(x, y));
    S[2] = __dadd_rn(S[2], __dmul_rn(x, z));
    S[3] = __dadd_rn(S[3], __dmul_rn(y, y));
    S[4] = __dadd_rn(S[4], __dmul_rn(y, z));
    S[5] = __dadd_rn(S[5], __dmul_rn(z, z));
  }
  double* o = c + 10 * g;
  for (int q = 0; q < 6; ++q) o[q] = S[q];
  o[6] = m0;
  o[7] = m1;
  o[8] = m2;
  o[9] = n;
  ckey[g] = keys[a];
  cscan[g] = pscan[vals[a]];
}

// Eq. 5: parent key of every cluster; sort keys (scan first, then parent)
__global__ void parent_keys_kernel(int64_t nc, const uint64_t* ckey, const int32_t* cscan, uint64_t* pkey,
                                   uint32_t* skey, uint32_t* vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  long long ix[3];
  unpack_key(ckey[i], ix);
  pkey[i] = pack_key(half_floor(ix[0]), half_floor(ix[1]), half_floor(ix[2]));
  skey[i] = (uint32_t)cscan[i];
  vals[i] = (uint32_t)i;
}

__global__ void gather_keys_kernel(int64_t n, const uint64_t* src, const uint32_t* vals, uint64_t* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[vals[i]];
}

// merge of two centred clusters, the operations in a fixed order:
// N = Na + Nb, d = mb - ma, S = Sa + Sb + (Na Nb / N) d d^T, m = ma + (Nb / N) d
__device__ __forceinline__ void merge_into(double* acc, const double* b) {
  const double na = acc[9], nb = b[9], n = __dadd_rn(na, nb);
  const double d[3] = {__dsub_rn(b[6], acc[6]), __dsub_rn(b[7], acc[7]), __dsub_rn(b[8], acc[8])};
  const double f = __ddiv_rn(__dmul_rn(na, nb), n);
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      acc[idx] = __dadd_rn(__dadd_rn(acc[idx], b[idx]), __dmul_rn(__dmul_rn(f, d[i]), d[j]));
      ++idx;
    }
  const double w = __ddiv_rn(nb, n);
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[6 + i] = __dadd_rn(acc[6 + i], __dmul_rn(w, d[i]));
  acc[9] = n;
}

// level-k clusters: the children of each (parent, scan) group merged in order
__global__ void merge_kernel(int64_t np, const int64_t* start, const uint32_t* vals, const double* child,
                             const uint64_t* pkeys_sorted, const int32_t* cscan, double* c, uint64_t* ckey,
                             int32_t* oscan) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= np) return;
  const int64_t a = start[g], b = start[g + 1];
  double acc[10];
  for (int q = 0; q < 10; ++q) acc[q] = child[10 * (int64_t)vals[a] + q];
  for (int64_t k = a + 1; k < b; ++k) merge_into(acc, child + 10 * (int64_t)vals[k]);
  for (int q = 0; q < 10; ++q) c[10 * g + q] = acc[q];
  ckey[g] = pkeys_sorted[a];
  oscan[g] = cscan[vals[a]];
}

// voxels of a level: runs of equal key among its clusters (sorted by key, scan)
__global__ void voxel_heads_kernel(int64_t nc, const uint64_t* ckey, int64_t* pos) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc) pos[i] = (i == 0 || ckey[i] != ckey[i - 1]) ? 1 : 0;
}

__global__ void voxel_starts_kernel(int64_t nc, const uint64_t* ckey, const int64_t* pos, int64_t* vstart,
                                    int64_t nv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc && (i == 0 || ckey[i] != ckey[i - 1])) vstart[pos[i]] = i;
  if (i == 0) vstart[nv] = nc;
}

// Selection (Algorithm 1): voxel covariance at the poses (Eq. 1-2, centred),
// kept if it has min_obs observations and lambda0 < tau lambda1 (tau > 0).
// keep[v] = observations kept (0 or the voxel's count); the partial sums use
// the CPU reference's order of operations.
__global__ void select_kernel(int64_t nv, const int64_t* vstart, const double* c, const int32_t* cscan,
                              const double* poses, double tau, int32_t min_obs, int64_t* keep_obs,
                              int64_t* keep_vox) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int64_t a = vstart[v], b = vstart[v + 1];
  bool keep = (b - a) >= (int64_t)min_obs;
  if (keep && tau > 0.0) {
    double n = 0.0, m[3] = {0, 0, 0};
    for (int64_t t = a; t < b; ++t) {
      const double* cl = c + 10 * t;
      const double* T = poses + 12 * (int64_t)cscan[t];
      for (int q = 0; q < 3; ++q) {
        const double w = fma(T[3 * q], cl[6], fma(T[3 * q + 1], cl[7], fma(T[3 * q + 2], cl[8], T[9 + q])));
        m[q] = __dadd_rn(m[q], __dmul_rn(cl[9], w));
      }
      n = __dadd_rn(n, cl[9]);
    }
    for (int q = 0; q < 3; ++q) m[q] = __ddiv_rn(m[q], n);
    double A[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t t = a; t < b; ++t) {
      const double* cl = c + 10 * t;
      const double* R = poses + 12 * (int64_t)cscan[t];
      double dd[3];
      for (int q = 0; q < 3; ++q) {
        const double w = fma(R[3 * q], cl[6], fma(R[3 * q + 1], cl[7], fma(R[3 * q + 2], cl[8], R[9 + q])));
        dd[q] = __dsub_rn(w, m[q]);
      }
      const double Sm[3][3] = {{cl[0], cl[1], cl[2]}, {cl[1], cl[3], cl[4]}, {cl[2], cl[4], cl[5]}};
      double RS[3][3];
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
          RS[x][y] = __dadd_rn(__dadd_rn(__dmul_rn(R[3 * x], Sm[0][y]), __dmul_rn(R[3 * x + 1], Sm[1][y])),
                               __dmul_rn(R[3 * x + 2], Sm[2][y]));
      int idx = 0;
      for (int x = 0; x < 3; ++x)
        for (int y = x; y < 3; ++y) {
          const double rsr = __dadd_rn(__dadd_rn(__dmul_rn(RS[x][0], R[3 * y]), __dmul_rn(RS[x][1], R[3 * y + 1])),
                                       __dmul_rn(RS[x][2], R[3 * y + 2]));
          A[idx] = __dadd_rn(A[idx], __dadd_rn(rsr, __dmul_rn(__dmul_rn(cl[9], dd[x]), dd[y])));
          ++idx;
        }
    }
    for (int q = 0; q < 6; ++q) A[q] = __ddiv_rn(A[q], n);
    double lam[3], V[9];
    eig3_sym(A, lam, V);
    keep = lam[0] < tau * lam[1];
  }
  keep_obs[v] = keep ? (b - a) : 0;
  keep_vox[v] = keep ? 1 : 0;
}

// kept voxels of a level written at their places in the output
__global__ void emit_kernel(int64_t nv, const int64_t* vstart, const uint64_t* ckey, const int32_t* cscan,
                            const double* c, const int64_t* obs_pos, const int64_t* vox_pos, const int64_t* keep_vox,
                            int32_t level, int64_t v_base, int64_t o_base, int64_t* voxel_off, int32_t* obs_scan,
                            double* agg, int32_t* lev, int32_t* index) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv || !keep_vox[v]) return;
  const int64_t a = vstart[v], b = vstart[v + 1];
  const int64_t ov = v_base + vox_pos[v], oo = o_base + obs_pos[v];
  voxel_off[ov + 1] = oo + (b - a);
  lev[ov] = level;
  long long ix[3];
  unpack_key(ckey[a], ix);
  for (int q = 0; q < 3; ++q) index[3 * ov + q] = (int32_t)ix[q];
  for (int64_t t = a; t < b; ++t) {
    obs_scan[oo + (t - a)] = cscan[t];
    for (int q = 0; q < 10; ++q) agg[10 * (oo + (t - a)) + q] = c[10 * t + q];
  }
}

// ---- host helpers ------------------------------------------------------------

thread_local std::string g_vox_error;

struct Buf {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit Buf(cudaStream_t st) : s(st) {}
  ~Buf() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  T* get(int64_t n) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, sizeof(T) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
};

unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

int bit_width_u(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

ba_status vfail(ba_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_vox_error = buf;
  return s;
}

#define VCK(call, what)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return e_ == cudaErrorMemoryAllocation ? vfail(BA_ERR_OOM, "%s: out of device memory", what) \
                                             : vfail(BA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

// group starts of a sorted (key, scan) sequence; returns the group count
ba_status group_starts(int64_t n, const uint64_t* keys, const uint32_t* vals, const int32_t* scan, Buf& tmp,
                       int64_t** start_out, int64_t* n_groups, cudaStream_t st, int64_t* launches) {
  int64_t* pos = tmp.get<int64_t>(n + 1);
  int64_t* scr = tmp.get<int64_t>(scan_scratch_count(n + 1));
  if (!pos || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  heads_kernel<<<blocks_for(n), 256, 0, st>>>(n, keys, vals, scan, pos);
  VCK(cudaGetLastError(), "voxelize");
  VCK(cudaMemsetAsync(pos + n, 0, sizeof(int64_t), st), "voxelize");
  VCK(exclusive_scan_i64(pos, n + 1, scr, st, launches), "voxelize");
  int64_t ng = 0;
  VCK(cudaMemcpyAsync(&ng, pos + n, sizeof ng, cudaMemcpyDeviceToHost, st), "voxelize");
  VCK(cudaStreamSynchronize(st), "voxelize");
  int64_t* start = tmp.get<int64_t>(ng + 1);
  if (!start) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  starts_kernel<<<blocks_for(n), 256, 0, st>>>(n, keys, vals, scan, pos, start, ng);
  VCK(cudaGetLastError(), "voxelize");
  *launches += 2;
  *start_out = start;
  *n_groups = ng;
  return BA_OK;
}

}  // namespace

struct ba_voxels {
  int device = 0;
  int64_t n_voxels = 0, n_obs = 0;
  int64_t* voxel_off = nullptr;
  int32_t* obs_scan = nullptr;
  double* agg = nullptr;
  int32_t* level = nullptr;
  int32_t* index = nullptr;
  int64_t launches = 0;
};

extern "C" {

void ba_voxelize_config_default(ba_voxelize_config* cfg) {
  if (!cfg) return;
  cfg->voxel_size = 1.0;
  cfg->levels = 1;
  cfg->tau = 0.0;
  cfg->min_obs = 1;
  cfg->device = 0;
  cfg->cuda_stream = nullptr;
}

const char* ba_voxelize_last_error(void) { return g_vox_error.c_str(); }

ba_status ba_voxelize(const ba_voxelize_config* cfg, int32_t n_scans, const int64_t* scan_point_off,
                      const double* points, const double* poses, int32_t mem_kind, ba_voxels** out) {
  if (!cfg || !out || !scan_point_off || !poses) return vfail(BA_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n_scans < 1) return vfail(BA_ERR_INVALID_ARG, "n_scans must be >= 1");
  if (!(cfg->voxel_size > 0.0) || !std::isfinite(cfg->voxel_size))
    return vfail(BA_ERR_INVALID_ARG, "voxel_size must be positive and finite");
  if (cfg->levels < 1 || cfg->levels > 20) return vfail(BA_ERR_INVALID_ARG, "levels must be in 1..20");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return vfail(BA_ERR_INVALID_ARG, "bad mem_kind");
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(cfg->device) != cudaSuccess) return vfail(BA_ERR_CUDA, "cannot use device %d", cfg->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};
  cudaStream_t st = (cudaStream_t)cfg->cuda_stream;
  Buf tmp(st);
  int64_t launches = 0;

  // stage the inputs
  int64_t n = 0;
  const int64_t* spo = scan_point_off;
  const double *pts = points, *T = poses;
  if (mem_kind == BA_MEM_HOST) {
    n = scan_point_off[n_scans];
    if (n < 0) return vfail(BA_ERR_INVALID_ARG, "scan_point_off must end at the point count");
    int64_t* d_spo = tmp.get<int64_t>(n_scans + 1);
    double* d_pts = tmp.get<double>(3 * n);
    double* d_T = tmp.get<double>(12 * (int64_t)n_scans);
    if (!d_spo || !d_pts || !d_T) return vfail(BA_ERR_OOM, "voxelize inputs: out of device memory");
    VCK(cudaMemcpyAsync(d_spo, spo, sizeof(int64_t) * (n_scans + 1), cudaMemcpyHostToDevice, st), "stage");
    if (n) VCK(cudaMemcpyAsync(d_pts, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st), "stage");
    VCK(cudaMemcpyAsync(d_T, T, sizeof(double) * 12 * n_scans, cudaMemcpyHostToDevice, st), "stage");
    spo = d_spo;
    pts = d_pts;
    T = d_T;
  } else {
    VCK(cudaMemcpyAsync(&n, scan_point_off + n_scans, sizeof n, cudaMemcpyDeviceToHost, st), "read point count");
    VCK(cudaStreamSynchronize(st), "read point count");
    if (n < 0) return vfail(BA_ERR_INVALID_ARG, "scan_point_off must end at the point count");
  }
  if (n >= (1ll << 32)) return vfail(BA_ERR_CAPACITY, "at most 2^32 - 1 points per call");
  if (n > 0 && !points) return vfail(BA_ERR_INVALID_ARG, "NULL points");

  // validation of the offsets and poses, then the L1 keys
  long long* bad = tmp.get<long long>(3);
  if (!bad) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  const long long init[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
  VCK(cudaMemcpyAsync(bad, init, sizeof init, cudaMemcpyHostToDevice, st), "voxelize");
  check_inputs_kernel<<<blocks_for(n_scans + 1), 256, 0, st>>>(n_scans, spo, n, T, bad, bad + 1);
  ++launches;
  VCK(cudaGetLastError(), "voxelize");
  long long res[3];
  VCK(cudaMemcpyAsync(res, bad, sizeof res, cudaMemcpyDeviceToHost, st), "voxelize");
  VCK(cudaStreamSynchronize(st), "voxelize");
  if (res[0] != LLONG_MAX)
    return vfail(BA_ERR_INVALID_ARG, "scan_point_off must start at 0, not decrease and end at %lld (index %lld)",
                 (long long)n, res[0]);
  if (res[1] != LLONG_MAX) return vfail(BA_ERR_INVALID_ARG, "pose %lld is not finite", res[1]);

  std::vector<int64_t*> lv_start;  // per level: voxel starts (device), counts
  struct Level {
    int64_t nc = 0, nv = 0;
    double* c = nullptr;
    uint64_t* key = nullptr;
    int32_t* scan = nullptr;
    int64_t* vstart = nullptr;
  };
  std::vector<Level> lv(cfg->levels);
  if (n > 0) {
    uint64_t* keys = tmp.get<uint64_t>(n);
    uint64_t* tkeys = tmp.get<uint64_t>(n);
    uint32_t* vals = tmp.get<uint32_t>(n);
    uint32_t* tvals = tmp.get<uint32_t>(n);
    int32_t* pscan = tmp.get<int32_t>(n);
    int64_t* scr = tmp.get<int64_t>(radix_scratch_count(n));
    if (!keys || !tkeys || !vals || !tvals || !pscan || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    l1_keys_kernel<<<blocks_for(n), 256, 0, st>>>(n_scans, spo, pts, T, cfg->voxel_size, n, keys, vals, pscan,
                                                  bad + 2);
    ++launches;
    VCK(cudaGetLastError(), "voxelize keys");
    VCK(cudaMemcpyAsync(res + 2, bad + 2, sizeof(long long), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaStreamSynchronize(st), "voxelize");
    if (res[2] != LLONG_MAX)
      return vfail(BA_ERR_CAPACITY, "point %lld lies outside the voxel index range [-2^20, 2^20) at this voxel size",
                   res[2]);
    // stable by key over points in scan order: groups ordered by (key, scan, point)
    VCK(radix_sort_pairs64(keys, vals, tkeys, tvals, n, kKeyBits, scr, st, &launches), "voxelize sort");
    int64_t* start = nullptr;
    int64_t n1 = 0;
    ba_status s = group_starts(n, keys, vals, pscan, tmp, &start, &n1, st, &launches);
    if (s != BA_OK) return s;
    Level& L1 = lv[0];
    L1.nc = n1;
    L1.c = tmp.get<double>(10 * n1);
    L1.key = tmp.get<uint64_t>(n1);
    L1.scan = tmp.get<int32_t>(n1);
    if (!L1.c || !L1.key || !L1.scan) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    l1_clusters_kernel<<<blocks_for(n1), 256, 0, st>>>(n1, start, vals, keys, pscan, pts, L1.c, L1.key, L1.scan);
    ++launches;
    VCK(cudaGetLastError(), "voxelize clusters");
    // levels 2..L (Eq. 5)
    for (int k = 1; k < cfg->levels; ++k) {
      const Level& ch = lv[k - 1];
      const int64_t nc = ch.nc;
      uint64_t* pkey = tmp.get<uint64_t>(nc);
      uint64_t* k64 = tmp.get<uint64_t>(nc);
      uint64_t* t64 = tmp.get<uint64_t>(nc);
      uint32_t* skey = tmp.get<uint32_t>(nc);
      uint32_t* tsk = tmp.get<uint32_t>(nc);
      uint32_t* cv = tmp.get<uint32_t>(nc);
      uint32_t* tcv = tmp.get<uint32_t>(nc);
      int64_t* scr2 = tmp.get<int64_t>(radix_scratch_count(nc));
      if (!pkey || !k64 || !t64 || !skey || !tsk || !cv || !tcv || !scr2)
        return vfail(BA_ERR_OOM, "voxelize: out of device memory");
      parent_keys_kernel<<<blocks_for(nc), 256, 0, st>>>(nc, ch.key, ch.scan, pkey, skey, cv);
      ++launches;
      VCK(cudaGetLastError(), "voxelize levels");
      // by scan (stable), then by parent key (stable): order (parent, scan, child)
      VCK(radix_sort_pairs(skey, cv, tsk, tcv, nc, bit_width_u((uint64_t)(n_scans - 1)), scr2, st, &launches),
          "voxelize sort");
      gather_keys_kernel<<<blocks_for(nc), 256, 0, st>>>(nc, pkey, cv, k64);
      ++launches;
      VCK(cudaGetLastError(), "voxelize levels");
      VCK(radix_sort_pairs64(k64, cv, t64, tcv, nc, kKeyBits, scr2, st, &launches), "voxelize sort");
      int64_t* pst = nullptr;
      int64_t np = 0;
      if ((s = group_starts(nc, k64, cv, ch.scan, tmp, &pst, &np, st, &launches)) != BA_OK) return s;
      Level& P = lv[k];
      P.nc = np;
      P.c = tmp.get<double>(10 * np);
      P.key = tmp.get<uint64_t>(np);
      P.scan = tmp.get<int32_t>(np);
      if (!P.c || !P.key || !P.scan) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
      merge_kernel<<<blocks_for(np), 256, 0, st>>>(np, pst, cv, ch.c, k64, ch.scan, P.c, P.key, P.scan);
      ++launches;
      VCK(cudaGetLastError(), "voxelize merge");
    }
  }

  // voxels of every level, selection, and the output
  ba_voxels* v = new ba_voxels();
  v->device = cfg->device;
  struct Guard {
    ba_voxels** pv;
    ~Guard() {
      if (*pv) ba_voxels_destroy(*pv);
    }
  } guard{&v};
  std::vector<int64_t*> keep_obs(cfg->levels), keep_vox(cfg->levels), obs_pos(cfg->levels), vox_pos(cfg->levels);
  std::vector<int64_t> lv_nv(cfg->levels, 0), lv_no(cfg->levels, 0);
  int64_t total_v = 0, total_o = 0;
  for (int k = 0; k < cfg->levels; ++k) {
    Level& L = lv[k];
    if (L.nc == 0) continue;
    int64_t* pos = tmp.get<int64_t>(L.nc + 1);
    int64_t* scr = tmp.get<int64_t>(scan_scratch_count(L.nc + 1));
    if (!pos || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    voxel_heads_kernel<<<blocks_for(L.nc), 256, 0, st>>>(L.nc, L.key, pos);
    VCK(cudaGetLastError(), "voxelize");
    VCK(cudaMemsetAsync(pos + L.nc, 0, sizeof(int64_t), st), "voxelize");
    VCK(exclusive_scan_i64(pos, L.nc + 1, scr, st, &launches), "voxelize");
    VCK(cudaMemcpyAsync(&L.nv, pos + L.nc, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaStreamSynchronize(st), "voxelize");
    L.vstart = tmp.get<int64_t>(L.nv + 1);
    keep_obs[k] = tmp.get<int64_t>(L.nv + 1);
    keep_vox[k] = tmp.get<int64_t>(L.nv + 1);
    obs_pos[k] = tmp.get<int64_t>(L.nv + 1);
    vox_pos[k] = tmp.get<int64_t>(L.nv + 1);
    int64_t* scr3 = tmp.get<int64_t>(scan_scratch_count(L.nv + 1));
    if (!L.vstart || !keep_obs[k] || !keep_vox[k] || !obs_pos[k] || !vox_pos[k] || !scr3)
      return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    voxel_starts_kernel<<<blocks_for(L.nc), 256, 0, st>>>(L.nc, L.key, pos, L.vstart, L.nv);
    select_kernel<<<blocks_for(L.nv), 256, 0, st>>>(L.nv, L.vstart, L.c, L.scan, T, cfg->tau, cfg->min_obs,
                                                   keep_obs[k], keep_vox[k]);
    launches += 3;
    VCK(cudaGetLastError(), "voxelize select");
    VCK(cudaMemsetAsync(keep_obs[k] + L.nv, 0, sizeof(int64_t), st), "voxelize");
    VCK(cudaMemsetAsync(keep_vox[k] + L.nv, 0, sizeof(int64_t), st), "voxelize");
    VCK(cudaMemcpyAsync(obs_pos[k], keep_obs[k], sizeof(int64_t) * (L.nv + 1), cudaMemcpyDeviceToDevice, st),
        "voxelize");
    VCK(cudaMemcpyAsync(vox_pos[k], keep_vox[k], sizeof(int64_t) * (L.nv + 1), cudaMemcpyDeviceToDevice, st),
        "voxelize");
    VCK(exclusive_scan_i64(obs_pos[k], L.nv + 1, scr3, st, &launches), "voxelize");
    VCK(exclusive_scan_i64(vox_pos[k], L.nv + 1, scr3, st, &launches), "voxelize");
    VCK(cudaMemcpyAsync(&lv_no[k], obs_pos[k] + L.nv, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaMemcpyAsync(&lv_nv[k], vox_pos[k] + L.nv, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaStreamSynchronize(st), "voxelize");
    total_v += lv_nv[k];
    total_o += lv_no[k];
  }
  v->n_voxels = total_v;
  v->n_obs = total_o;
  if (cudaMalloc(&v->voxel_off, sizeof(int64_t) * (total_v + 1)) != cudaSuccess ||
      cudaMalloc(&v->obs_scan, sizeof(int32_t) * (total_o > 0 ? total_o : 1)) != cudaSuccess ||
      cudaMalloc(&v->agg, sizeof(double) * 10 * (total_o > 0 ? total_o : 1)) != cudaSuccess ||
      cudaMalloc(&v->level, sizeof(int32_t) * (total_v > 0 ? total_v : 1)) != cudaSuccess ||
      cudaMalloc(&v->index, sizeof(int32_t) * 3 * (total_v > 0 ? total_v : 1)) != cudaSuccess) {
    cudaGetLastError();
    return vfail(BA_ERR_OOM, "voxelize output: out of device memory");
  }
  VCK(cudaMemsetAsync(v->voxel_off, 0, sizeof(int64_t), st), "voxelize");
  int64_t vb = 0, ob = 0;
  for (int k = 0; k < cfg->levels; ++k) {
    const Level& L = lv[k];
    if (L.nv == 0) continue;
    emit_kernel<<<blocks_for(L.nv), 256, 0, st>>>(L.nv, L.vstart, L.key, L.scan, L.c, obs_pos[k], vox_pos[k],
                                                 keep_vox[k], k + 1, vb, ob, v->voxel_off, v->obs_scan, v->agg,
                                                 v->level, v->index);
    ++launches;
    VCK(cudaGetLastError(), "voxelize emit");
    vb += lv_nv[k];
    ob += lv_no[k];
  }
  VCK(cudaStreamSynchronize(st), "voxelize");
  v->launches = launches;
  *out = v;
  v = nullptr;  // handed out
  return BA_OK;
}

ba_status ba_voxels_size(const ba_voxels* v, int64_t* n_voxels, int64_t* n_obs) {
  if (!v) return BA_ERR_INVALID_ARG;
  if (n_voxels) *n_voxels = v->n_voxels;
  if (n_obs) *n_obs = v->n_obs;
  return BA_OK;
}

ba_status ba_voxels_read(const ba_voxels* v, int64_t* voxel_off, int32_t* obs_scan, double* agg, int32_t* level,
                         int32_t* index, int32_t mem_kind) {
  if (!v) return BA_ERR_INVALID_ARG;
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return vfail(BA_ERR_INVALID_ARG, "bad mem_kind");
  const cudaMemcpyKind kind = mem_kind == BA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(v->device) != cudaSuccess) return vfail(BA_ERR_CUDA, "cannot use device %d", v->device);
  cudaError_t e = cudaSuccess;
  if (voxel_off) e = cudaMemcpy(voxel_off, v->voxel_off, sizeof(int64_t) * (v->n_voxels + 1), kind);
  if (e == cudaSuccess && obs_scan && v->n_obs) e = cudaMemcpy(obs_scan, v->obs_scan, sizeof(int32_t) * v->n_obs, kind);
  if (e == cudaSuccess && agg && v->n_obs) e = cudaMemcpy(agg, v->agg, sizeof(double) * 10 * v->n_obs, kind);
  if (e == cudaSuccess && level && v->n_voxels) e = cudaMemcpy(level, v->level, sizeof(int32_t) * v->n_voxels, kind);
  if (e == cudaSuccess && index && v->n_voxels)
    e = cudaMemcpy(index, v->index, sizeof(int32_t) * 3 * v->n_voxels, kind);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return vfail(BA_ERR_CUDA, "read voxels: %s", cudaGetErrorString(e));
  return BA_OK;
}

int64_t ba_voxels_kernel_launches(const ba_voxels* v) { return v ? v->launches : 0; }

void ba_voxels_destroy(ba_voxels* v) {
  if (!v) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(v->device);
  cudaFree(v->voxel_off);
  cudaFree(v->obs_scan);
  cudaFree(v->agg);
  cudaFree(v->level);
  cudaFree(v->index);
  if (prev >= 0) cudaSetDevice(prev);
  delete v;
}

}  // extern "C"
