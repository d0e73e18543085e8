// CUDA counterpart of sg_points (input synthesis only, no bundle-adjustment
// arithmetic): the same counter-based streams as scenegen.c, one thread per
// point, so a scene's points match the host generator's up to the last bits
// of log, cos and sqrt.  Used to synthesise large many-job workloads quickly;
// the CPU oracle always takes host-generated points.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamPoints = 6;  // ST_POINTS in scenegen.c

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
__device__ __forceinline__ double unit_open0(uint64_t x) {
  return ((double)(x >> 11) + 1.0) * (1.0 / 9007199254740992.0);
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
  const uint64_t key = mix64(mix64(seed ^ (kStreamPoints * 0xD1B54A32D192ED03ull)) + (uint64_t)o * kGolden);
  const int draws = sigma > 0.0 ? 4 : 2;
  uint64_t ctr = (uint64_t)k * draws;
  const double a = -0.5 * s1 + s1 * unit(mix64(key + (++ctr) * kGolden));
  const double b = -0.5 * s2 + s2 * unit(mix64(key + (++ctr) * kGolden));
  double eps = 0.0;
  if (sigma > 0.0) {
    const double u1 = unit_open0(mix64(key + (++ctr) * kGolden));
    const double u2 = unit(mix64(key + (++ctr) * kGolden));
    eps = sigma * (sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2));
  }
  double w[3];
  for (int d = 0; d < 3; ++d) w[d] = P[d] + a * P[6 + d] + b * P[9 + d] + eps * P[3 + d] - G[9 + d];
  double* dst = out + 3 * g;
  for (int d = 0; d < 3; ++d) dst[d] = G[d] * w[0] + G[3 + d] * w[1] + G[6 + d] * w[2];
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
