// Allocation-free cost evaluation (ba_eval_cost_noalloc, see include/ba.h).
//
// Some callers cannot allocate device memory at the point where they need a
// cost: a mapping loop running on a vehicle under a fixed memory budget
// (cudaMalloc/cudaFree may synchronise the device and stall the loop), or a
// host application whose own allocator has already reserved the GPU memory.
// This entry point therefore takes only caller-owned inputs and outputs; its
// scratch (the per-block partial sums of the cost and an error word) is a
// file-scope __device__ array that every GPU loading the library holds until
// the process exits.  Host code may not use the array's name as a device
// address, so the address is fetched once per device with
// cudaGetSymbolAddress and passed to the kernels.  The cached address belongs
// to the device's context of that moment: after cudaDeviceReset (or anything
// else that tears down and recreates the primary context) the library's
// module is loaded anew and the cache is stale, so the entry point must not
// be used across a device reset.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/ba.h"
#include "mmba_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int64_t kMaxBlocks = BA_NOALLOC_MAX_VOXELS / kThreads;
static_assert(BA_NOALLOC_MAX_VOXELS % kThreads == 0, "capacity must be a whole number of blocks");

// scratch shared by every call on a device: block partials, then the error word
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 32];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_ready[kMaxDevices];
double* g_ptr[kMaxDevices];

// One thread per voxel over the caller's voxel-major CSR: posed cluster means
// q = R m + t, anchored sums about the voxel's first q, covariance, smallest
// eigenvalue (the voxel's cost, Eq. 1).  Invalid offsets or scan indices set
// the error word and leave the voxel out.
__global__ void __launch_bounds__(kThreads) noalloc_cost_kernel(int64_t n_voxels, int64_t n_obs,
                                                                const int64_t* __restrict__ off,
                                                                const int32_t* __restrict__ obs_scan,
                                                                const double* __restrict__ agg,
                                                                const double* __restrict__ poses, int32_t n_scans,
                                                                double* __restrict__ lam0_out, double* scratch) {
  __shared__ double red[kThreads / 32];
  unsigned long long* err = reinterpret_cast<unsigned long long*>(scratch + kMaxBlocks);
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double lam0 = 0.0;
  if (i < n_voxels) {
    const int64_t a = off[i], b = off[i + 1];
    bool ok = a >= 0 && b > a && b <= n_obs;
    double n = 0.0, ax = 0.0, ay = 0.0, az = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    double m00 = 0.0, m01 = 0.0, m02 = 0.0, m11 = 0.0, m12 = 0.0, m22 = 0.0;
    for (int64_t o = a; ok && o < b; ++o) {
      const int32_t j = obs_scan[o];
      if (j < 0 || j >= n_scans) {
        ok = false;
        break;
      }
      const double* P = poses + 12 * (int64_t)j;
      const double* c = agg + 10 * o;
      const double qx = fma(P[0], c[6], fma(P[1], c[7], fma(P[2], c[8], P[9])));
      const double qy = fma(P[3], c[6], fma(P[4], c[7], fma(P[5], c[8], P[10])));
      const double qz = fma(P[6], c[6], fma(P[7], c[7], fma(P[8], c[8], P[11])));
      if (o == a) {
        ax = qx;
        ay = qy;
        az = qz;
      }
      const double dx = qx - ax, dy = qy - ay, dz = qz - az, N = c[9];
      // R S R^T from the packed scatter (xx, xy, xz, yy, yz, zz)
      double RS[3][3];
      const double S[3][3] = {{c[0], c[1], c[2]}, {c[1], c[3], c[4]}, {c[2], c[4], c[5]}};
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) RS[r][k] = fma(P[3 * r], S[0][k], fma(P[3 * r + 1], S[1][k], P[3 * r + 2] * S[2][k]));
      auto rsr = [&](int r, int k) { return fma(RS[r][0], P[3 * k], fma(RS[r][1], P[3 * k + 1], RS[r][2] * P[3 * k + 2])); };
      m00 += rsr(0, 0) + N * dx * dx;
      m01 += rsr(0, 1) + N * dx * dy;
      m02 += rsr(0, 2) + N * dx * dz;
      m11 += rsr(1, 1) + N * dy * dy;
      m12 += rsr(1, 2) + N * dy * dz;
      m22 += rsr(2, 2) + N * dz * dz;
      sx += N * dx;
      sy += N * dy;
      sz += N * dz;
      n += N;
    }
    if (ok && n > 0.0) {
      const double inv = 1.0 / n;
      const double cx = sx * inv, cy = sy * inv, cz = sz * inv;
      double A[6] = {fma(-cx, cx, m00 * inv), fma(-cx, cy, m01 * inv), fma(-cx, cz, m02 * inv),
                     fma(-cy, cy, m11 * inv), fma(-cy, cz, m12 * inv), fma(-cz, cz, m22 * inv)};
      double lam[3], V[9];
      mmba::eig3_sym(A, lam, V);
      lam0 = lam[0];
    } else {
      atomicMin(err, (unsigned long long)i);
    }
    if (lam0_out) lam0_out[i] = ok ? lam0 : __longlong_as_double(0x7ff8000000000000ll);
  }
  const double tot = mmba::block_sum<kThreads>(lam0, red);
  if (threadIdx.x == 0) scratch[blockIdx.x] = tot;
}

__global__ void noalloc_reset_kernel(double* scratch) {
  *reinterpret_cast<unsigned long long*>(scratch + kMaxBlocks) = ~0ull;
}

// Sums the block partials in a fixed order; a recorded error makes the cost NaN.
__global__ void __launch_bounds__(256) noalloc_sum_kernel(int64_t n_blocks, const double* scratch, double* cost_out) {
  __shared__ double red[256 / 32];
  double v = 0.0;
  for (int64_t k = threadIdx.x; k < n_blocks; k += 256) v += scratch[k];
  const double tot = mmba::block_sum<256>(v, red);
  if (threadIdx.x == 0) {
    const unsigned long long e = *reinterpret_cast<const unsigned long long*>(scratch + kMaxBlocks);
    *cost_out = e == ~0ull ? tot : __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace

extern "C" ba_status ba_eval_cost_noalloc(int32_t n_scans, int64_t n_voxels, int64_t n_obs,
                                          const int64_t* voxel_offsets, const int32_t* obs_scan,
                                          const double* agg_centred, const double* poses, double* cost_out,
                                          double* lambda0_out, void* stream) {
  if (n_scans < 1 || n_voxels < 1 || n_obs < n_voxels) return BA_ERR_INVALID_ARG;
  if (n_voxels > BA_NOALLOC_MAX_VOXELS) return BA_ERR_CAPACITY;
  if (!voxel_offsets || !obs_scan || !agg_centred || !poses || !cost_out) return BA_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BA_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ready[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return BA_ERR_CUDA;
      }
      g_ptr[dev] = static_cast<double*>(p);
      g_ready[dev] = true;
    }
    scratch = g_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t blocks = (n_voxels + kThreads - 1) / kThreads;
  // an error left pending by earlier, unrelated work on this thread is not
  // this call's to report: clear it, then check each launch on its own
  (void)cudaGetLastError();
  noalloc_reset_kernel<<<1, 1, 0, s>>>(scratch);
  if (cudaGetLastError() != cudaSuccess) return BA_ERR_CUDA;
  noalloc_cost_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(n_voxels, n_obs, voxel_offsets, obs_scan, agg_centred,
                                                            poses, n_scans, lambda0_out, scratch);
  if (cudaGetLastError() != cudaSuccess) return BA_ERR_CUDA;
  noalloc_sum_kernel<<<1, 256, 0, s>>>(blocks, scratch, cost_out);
  return cudaGetLastError() == cudaSuccess ? BA_OK : BA_ERR_CUDA;
}
