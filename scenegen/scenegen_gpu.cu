// CUDA counterpart of the scene generator (input synthesis only, no
// bundle-adjustment arithmetic).  The same counter-based streams as
// scenegen.c:
//  - sgd_points: one thread per point, FP64, so a scene's points match the
//    host generator's up to the last bits of log, cos and sqrt;
//  - sgd_job: a whole scene without a view radius built on the device from its
//    parameters and voxel offsets (ground-truth and initial poses, planar
//    patches, the observing scans of every voxel), equal to the host's scene
//    (integers exactly, poses and patches to the last bits of the math
//    library), so thousands of jobs can be generated where they are solved;
//  - sgd_points_fast: the points of such a scene drawn from the same
//    per-observation counters but in FP32 (uniform variates from the top 23
//    bits, Box-Muller with the fast intrinsics), written as float64.  These points differ from the host's by the FP32
//    rounding of the draws and of the scan-frame coordinates (a few
//    micrometres at 100 m), far below the 1-2 cm noise of the workloads; the
//    GPU's FP64 pipe, narrow on this part, stays out of the per-point work.
#include <cuda_runtime.h>

#include <cstdint>

#include "scenegen.h"

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;
// stream identifiers of scenegen.c
constexpr uint64_t kStPoseGt = 1, kStPosePerturb = 2, kStPlane = 3, kStObsPick = 5, kStPoints = 6;
constexpr int kMaxPick = 64;  // largest obs_max sgd_job handles

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Rng {
  uint64_t key, ctr;
  __device__ Rng(uint64_t seed, uint64_t stream, uint64_t index)
      : key(mix64(mix64(seed ^ (stream * kStreamMul)) + index * kGolden)), ctr(0) {}
  __device__ uint64_t next() { return mix64(key + (++ctr) * kGolden); }
  __device__ double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  __device__ double unit_open0() { return ((double)(next() >> 11) + 1.0) * (1.0 / 9007199254740992.0); }
  __device__ double uniform(double lo, double hi) { return lo + (hi - lo) * unit(); }
  __device__ double normal() {
    const double u1 = unit_open0();
    const double u2 = unit();
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
  }
  __device__ int64_t integer(int64_t lo, int64_t hi) {
    const uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int64_t)(next() % span);
  }
};

__device__ __forceinline__ double unit64(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
__device__ __forceinline__ double unit64_open0(uint64_t x) {
  return ((double)(x >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

__device__ void quat_to_mat(const double q[4], double R[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

__device__ void normalize3(double v[3]) {
  const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n;
  v[1] /= n;
  v[2] /= n;
}

__device__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__global__ void points_kernel(uint64_t seed, int32_t npo, double sigma, const double* __restrict__ plane,
                              const double* __restrict__ extent, const double* __restrict__ pose_gt,
                              const int32_t* __restrict__ obs_scan, const int32_t* __restrict__ obs_voxel,
                              int64_t obs_begin, int64_t n_points, double* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_points) return;
  const int64_t o = obs_begin + g / npo;
  const int64_t k = g % npo;
  const int32_t v = obs_voxel[o];
  const double* P = plane + 12 * (int64_t)v;
  const double* G = pose_gt + 12 * (int64_t)obs_scan[o];
  const double s1 = extent[2 * v], s2 = extent[2 * v + 1];
  const uint64_t key = mix64(mix64(seed ^ (kStPoints * kStreamMul)) + (uint64_t)o * kGolden);
  const int draws = sigma > 0.0 ? 4 : 2;
  uint64_t ctr = (uint64_t)k * draws;
  const double a = -0.5 * s1 + s1 * unit64(mix64(key + (++ctr) * kGolden));
  const double b = -0.5 * s2 + s2 * unit64(mix64(key + (++ctr) * kGolden));
  double eps = 0.0;
  if (sigma > 0.0) {
    const double u1 = unit64_open0(mix64(key + (++ctr) * kGolden));
    const double u2 = unit64(mix64(key + (++ctr) * kGolden));
    eps = sigma * (sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2));
  }
  double w[3];
  for (int d = 0; d < 3; ++d) w[d] = P[d] + a * P[6 + d] + b * P[9 + d] + eps * P[3 + d] - G[9 + d];
  double* dst = out + 3 * g;
  for (int d = 0; d < 3; ++d) dst[d] = G[d] * w[0] + G[3 + d] * w[1] + G[6 + d] * w[2];
}

// ground-truth and initial pose of every scan (gen_poses of scenegen.c)
__global__ void job_poses_kernel(sg_params p, double* __restrict__ pose_gt, double* __restrict__ pose_init) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.n_scans) return;
  Rng r(p.seed, kStPoseGt, (uint64_t)j);
  double q[4];
  for (int k = 0; k < 4; ++k) q[k] = r.normal();
  const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] /= qn;
  double G[12];
  quat_to_mat(q, G);
  G[9] = r.uniform(0.0, p.box[0]);
  G[10] = r.uniform(0.0, p.box[1]);
  G[11] = r.uniform(0.0, p.box[2]);
  double I[12];
  for (int k = 0; k < 12; ++k) I[k] = G[k];
  if (j != 0 || p.perturb_scan0) {
    Rng rp(p.seed, kStPosePerturb, (uint64_t)j);
    const double sr = p.rot_sigma_deg * (3.14159265358979323846 / 180.0);
    double phi[3];
    for (int k = 0; k < 3; ++k) phi[k] = sr * rp.normal();
    const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    double dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (th > 0.0) {
      const double sh = sin(0.5 * th) / th;
      dq[0] = cos(0.5 * th);
      dq[1] = sh * phi[0];
      dq[2] = sh * phi[1];
      dq[3] = sh * phi[2];
    }
    double dR[9];
    quat_to_mat(dq, dR);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) I[3 * a + b] = dR[3 * a] * G[b] + dR[3 * a + 1] * G[3 + b] + dR[3 * a + 2] * G[6 + b];
    I[9] = G[9] + p.trans_sigma * rp.normal();
    I[10] = G[10] + p.trans_sigma * rp.normal();
    I[11] = G[11] + p.trans_sigma * rp.normal();
  }
  for (int k = 0; k < 12; ++k) {
    pose_gt[12 * (int64_t)j + k] = G[k];
    pose_init[12 * (int64_t)j + k] = I[k];
  }
}

// planar patch of every voxel (gen_planes of scenegen.c)
__global__ void job_planes_kernel(sg_params p, double* __restrict__ plane, double* __restrict__ extent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n_voxels) return;
  Rng r(p.seed, kStPlane, (uint64_t)i);
  double* P = plane + 12 * i;
  double c[3];
  for (int d = 0; d < 3; ++d) c[d] = r.uniform(0.0, p.box[d]);
  double n[3], a[3];
  for (int d = 0; d < 3; ++d) n[d] = r.normal();
  normalize3(n);
  for (int d = 0; d < 3; ++d) a[d] = r.normal();
  double e1[3], e2[3];
  cross3(n, a, e1);
  normalize3(e1);
  cross3(n, e1, e2);
  for (int d = 0; d < 3; ++d) {
    P[d] = c[d];
    P[3 + d] = n[d];
    P[6 + d] = e1[d];
    P[9 + d] = e2[d];
  }
  const double side = p.side_max > p.side_min ? exp(r.uniform(log(p.side_min), log(p.side_max))) : p.side_min;
  double w2 = side;
  if (r.unit() < p.degenerate_frac) {
    const double ratio = r.uniform(2.0, 10.0);
    const double sig = p.noise_sigma > 0.0 ? p.noise_sigma : 0.01;
    w2 = sqrt(12.0 * ratio) * sig;
  }
  extent[2 * i] = side;
  extent[2 * i + 1] = w2;
}

// observing scans of every voxel (pick_scans of scenegen.c: Floyd's sampling
// of k distinct scans, then ascending order); the count k comes from the
// offsets, which the host derives from the count stream
__global__ void job_picks_kernel(sg_params p, const int64_t* __restrict__ voxel_off, int32_t* __restrict__ obs_scan,
                                 int32_t* __restrict__ obs_voxel, int32_t* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n_voxels) return;
  const int64_t o0 = voxel_off[i];
  const int32_t k = (int32_t)(voxel_off[i + 1] - o0);
  if (k < 0 || k > kMaxPick || k > p.n_scans) {
    atomicExch(bad, 1);
    return;
  }
  Rng rp(p.seed, kStObsPick, (uint64_t)i);
  int32_t out[kMaxPick];
  int32_t n = 0;
  const int32_t pool = p.n_scans;
  for (int32_t t = pool - k; t < pool; ++t) {
    const int32_t r = (int32_t)rp.integer(0, t);
    bool taken = false;
    for (int32_t q = 0; q < n; ++q) taken = taken || out[q] == r;
    out[n++] = taken ? t : r;
  }
  for (int32_t a = 1; a < k; ++a) {  // insertion sort (k is small)
    const int32_t x = out[a];
    int32_t b = a - 1;
    while (b >= 0 && out[b] > x) {
      out[b + 1] = out[b];
      --b;
    }
    out[b + 1] = x;
  }
  for (int32_t q = 0; q < k; ++q) {
    obs_scan[o0 + q] = out[q];
    obs_voxel[o0 + q] = (int32_t)i;
  }
}

// binary64 of a binary32 by its bits (normal numbers and zero; the
// coordinates here are never subnormal)
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0) return 0.0;
  const uint64_t d = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + (1023 - 127)) << 52) | ((uint64_t)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// [0, 1) from the top 23 bits of a draw, in FP32
__device__ __forceinline__ float unit32(uint64_t x) {
  return __uint_as_float(0x3f800000u | (uint32_t)(x >> 41)) - 1.0f;
}

// Per warp 32 observations: first every lane takes one observation's frame
// terms (FP64, then rounded once: the patch origin in the scan frame
// R^T (c - t) and its axes R^T e1, R^T e2, R^T n) and its stream key into
// shared memory -- a GB300 FP64 warp instruction costs the same with one
// active lane as with 32, so the terms of 32 observations cost what one
// would -- then the warp draws the observations' points one observation at a
// time, lane k taking points k, k + 32, ... in FP32.
constexpr int kFastWarps = 8;
struct FastObs {
  float t[14];  // origin (3), e1 (3), e2 (3), n (3) in the scan frame; side lengths s1, s2
  uint32_t key_lo, key_hi;
};

__global__ void __launch_bounds__(32 * kFastWarps) points_fast_kernel(
    uint64_t seed, int32_t npo, double sigma, const double* __restrict__ plane, const double* __restrict__ extent,
    const double* __restrict__ pose_gt, const int32_t* __restrict__ obs_scan, const int32_t* __restrict__ obs_voxel,
    int64_t obs_begin, int64_t n_obs, double* __restrict__ out) {
  __shared__ FastObs sh[kFastWarps][32];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * kFastWarps + wib) * 32;  // first observation (relative) of the warp
  if (w0 >= n_obs) return;  // the whole warp
  const int64_t mine = w0 + lane;
  if (mine < n_obs) {
    const int64_t o = obs_begin + mine;
    const int32_t v = obs_voxel[o];
    const double* P = plane + 12 * (int64_t)v;
    const double* G = pose_gt + 12 * (int64_t)obs_scan[o];
    const double dc[3] = {P[0] - G[9], P[1] - G[10], P[2] - G[11]};
    FastObs& f = sh[wib][lane];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      f.t[d] = (float)(G[d] * dc[0] + G[3 + d] * dc[1] + G[6 + d] * dc[2]);
      f.t[3 + d] = (float)(G[d] * P[6] + G[3 + d] * P[7] + G[6 + d] * P[8]);
      f.t[6 + d] = (float)(G[d] * P[9] + G[3 + d] * P[10] + G[6 + d] * P[11]);
      f.t[9 + d] = (float)(G[d] * P[3] + G[3 + d] * P[4] + G[6 + d] * P[5]);
    }
    f.t[12] = (float)extent[2 * v];
    f.t[13] = (float)extent[2 * v + 1];
    const uint64_t key = mix64(mix64(seed ^ (kStPoints * kStreamMul)) + (uint64_t)o * kGolden);
    f.key_lo = (uint32_t)key;
    f.key_hi = (uint32_t)(key >> 32);
  }
  __syncwarp();
  const float sg = (float)sigma;
  const int draws = sigma > 0.0 ? 4 : 2;
  const int nq = (int)min((int64_t)32, n_obs - w0);
  for (int q = 0; q < nq; ++q) {
    const FastObs& f = sh[wib][q];
    const uint64_t key = ((uint64_t)f.key_hi << 32) | f.key_lo;
    double* dst = out + 3 * ((w0 + q) * (int64_t)npo);
    for (int k = lane; k < npo; k += 32) {
      uint64_t ctr = (uint64_t)k * draws;
      const float a = f.t[12] * (unit32(mix64(key + (++ctr) * kGolden)) - 0.5f);
      const float b = f.t[13] * (unit32(mix64(key + (++ctr) * kGolden)) - 0.5f);
      float eps = 0.f;
      if (sigma > 0.0) {
        // (0, 1] like the host's ((x >> 11) + 1) 2^-53, from the top 32 bits
        // (relative precision kept for small values, where the log is steep)
        const float u1 = fmaf(__uint2float_rn((uint32_t)(mix64(key + (++ctr) * kGolden) >> 32)),
                              2.3283064365386963e-10f, 1.1641532182693481e-10f);
        const float u2 = unit32(mix64(key + (++ctr) * kGolden));
        // cos(2 pi u2) = -cos(2 pi u2 - pi), the fast cosine's argument kept in [-pi, pi)
        eps = sg * (sqrtf(-2.0f * logf(u1)) * -__cosf(6.28318530717958647692f * u2 - 3.14159265358979323846f));
      }
#pragma unroll
      for (int d = 0; d < 3; ++d)
        dst[3 * k + d] = f32_to_f64_bits(fmaf(a, f.t[3 + d], fmaf(b, f.t[6 + d], fmaf(eps, f.t[9 + d], f.t[d]))));
    }
  }
}

}  // namespace

// Points of observations [obs_begin, obs_end), pts_per_obs each, xyz triples
// into out.  Every pointer is device memory; obs_voxel[o] is the voxel of
// observation o.  Returns 0, or the CUDA error code of the launch.
extern "C" int sgd_points(uint64_t seed, int32_t pts_per_obs, double noise_sigma, const double* plane,
                          const double* extent, const double* pose_gt, const int32_t* obs_scan,
                          const int32_t* obs_voxel, int64_t obs_begin, int64_t obs_end, double* out, void* stream) {
  const int64_t n = (obs_end - obs_begin) * (int64_t)pts_per_obs;
  if (n <= 0) return 0;
  points_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      seed, pts_per_obs, noise_sigma, plane, extent, pose_gt, obs_scan, obs_voxel, obs_begin, n, out);
  return (int)cudaGetLastError();
}

// The scene *p (no view radius, obs_max <= 64) on the device: pose_gt and
// pose_init (n_scans x 12), plane (n_voxels x 12), extent (n_voxels x 2),
// obs_scan and obs_voxel (n_obs), from voxel_off (n_voxels + 1, device, as
// sg_voxel_offsets gives it).  bad: one device int, set to 1 if an offset
// range is out of bounds (the voxel is then skipped).  All launches on
// `stream`; returns -1 for parameters it does not handle, else the CUDA error
// code of the launches.
extern "C" int sgd_job(const sg_params* p, const int64_t* voxel_off, double* pose_gt, double* pose_init,
                       double* plane, double* extent, int32_t* obs_scan, int32_t* obs_voxel, int32_t* bad,
                       void* stream) {
  if (!p || p->n_scans < 1 || p->n_voxels < 0 || p->obs_min < 1 || p->obs_max < p->obs_min ||
      p->obs_max > kMaxPick || p->view_radius > 0.0)
    return -1;
  cudaStream_t s = (cudaStream_t)stream;
  job_poses_kernel<<<(unsigned)((p->n_scans + 127) / 128), 128, 0, s>>>(*p, pose_gt, pose_init);
  if (p->n_voxels > 0) {
    const unsigned nb = (unsigned)((p->n_voxels + 127) / 128);
    job_planes_kernel<<<nb, 128, 0, s>>>(*p, plane, extent);
    job_picks_kernel<<<nb, 128, 0, s>>>(*p, voxel_off, obs_scan, obs_voxel, bad);
  }
  return (int)cudaGetLastError();
}

// Fast points (FP32 draws, see the top of this file) of observations
// [obs_begin, obs_end) into out (device, (obs_end - obs_begin) x pts_per_obs
// x 3 doubles).  Returns 0, or the CUDA error code of the launch.
extern "C" int sgd_points_fast(uint64_t seed, int32_t pts_per_obs, double noise_sigma, const double* plane,
                               const double* extent, const double* pose_gt, const int32_t* obs_scan,
                               const int32_t* obs_voxel, int64_t obs_begin, int64_t obs_end, double* out,
                               void* stream) {
  const int64_t n = obs_end - obs_begin;
  if (n <= 0 || pts_per_obs < 1) return 0;
  const int64_t per_block = 32 * kFastWarps;  // observations per block
  points_fast_kernel<<<(unsigned)((n + per_block - 1) / per_block), 32 * kFastWarps, 0, (cudaStream_t)stream>>>(
      seed, pts_per_obs, noise_sigma, plane, extent, pose_gt, obs_scan, obs_voxel, obs_begin, n, out);
  return (int)cudaGetLastError();
}
