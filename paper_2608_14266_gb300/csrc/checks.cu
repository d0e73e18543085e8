// Device-side self-checks of helpers whose results must match a hardware
// reference bit for bit (run by the tests on the GPU).
#include <cuda_runtime.h>

#include "../../include/ba.h"
#include "mmba_internal.cuh"

namespace {

__device__ inline unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Bit patterns: random doubles over the whole binary32 range and beyond,
// values next to rounding ties, and special values; each is converted both
// ways by the integer helpers and by the hardware.
__global__ void conversion_check_kernel(long long n, unsigned long long seed, unsigned long long* bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long r = mix64(seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1));
  double x;
  switch (i % 4) {
    case 0:  // any exponent around the binary32 range (incl. subnormal and overflow results)
      x = __longlong_as_double((long long)((r & 0x800fffffffffffffull) |
                                           ((unsigned long long)(1023 - 160 + (int)((r >> 52) % 330)) << 52)));
      break;
    case 1: {  // near and exactly at ties: low 29 fraction bits around 0x10000000
      const unsigned long long low = 0x10000000ull + (long long)((r >> 40) % 5) - 2;
      x = __longlong_as_double((long long)(((r & 0x800fffffe0000000ull) | low) |
                                           ((unsigned long long)(1023 + (int)((r >> 52) % 60) - 30) << 52)));
      break;
    }
    case 2:  // values of the sizes the set-up converts (metres, squared metres)
      x = (double)(long long)(r >> 11) * 0x1.0p-53 * 4000.0 - 2000.0;
      break;
    default: {  // special values and the extremes
      const double sp[8] = {0.0, -0.0, 1.0 / 0.0, -1.0 / 0.0, 3.4028234663852886e38, 3.4028235677973366e38,
                            1.1754943508222875e-38, 1.401298464324817e-45};
      x = sp[(r >> 7) % 8];
      break;
    }
  }
  const float a = mmba::f64_to_f32(x), b = (float)x;
  if (__float_as_uint(a) != __float_as_uint(b) && !(isnan(a) && isnan(b))) atomicAdd(bad, 1ull);
  const double c = mmba::f32_to_f64(b), d = (double)b;
  if (__double_as_longlong(c) != __double_as_longlong(d) && !(isnan(c) && isnan(d))) atomicAdd(bad + 1, 1ull);
}

}  // namespace

extern "C" ba_status ba_check_conversions(int32_t device, int64_t n, uint64_t seed, uint64_t* mismatches) {
  if (n < 1 || !mismatches) return BA_ERR_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return BA_ERR_CUDA;
  unsigned long long* d = nullptr;
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMalloc(&d, sizeof h);
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof h);
  if (e == cudaSuccess) {
    conversion_check_kernel<<<(unsigned)((n + 255) / 256), 256>>>((long long)n, (unsigned long long)seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return BA_ERR_CUDA;
  mismatches[0] = h[0];
  mismatches[1] = h[1];
  return BA_OK;
}
