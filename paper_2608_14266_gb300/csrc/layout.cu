// Device-side layout build (the index mappers of Algorithm 1) and the
// primitives it uses: a stable LSD radix sort of (key, value) pairs, an
// exclusive scan, input validation and point-cluster formation (Eq. 2).
// Everything here runs once per load; none of it is on the per-iteration path.
#include <cfloat>

#include "mmba_internal.cuh"
#include "mmba_kernels.h"

namespace mmba {

#define RETURN_IF(err)                   \
  do {                                   \
    cudaError_t e_ = (err);              \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

// ============================================================================
// Exclusive scan of int64 (three-phase: per-tile scan + tile sums, recursive
// scan of the tile sums, add back).
// ============================================================================
constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanBlock * kScanItems;

__global__ void __launch_bounds__(kScanBlock) scan_tiles_kernel(int64_t* data, int64_t n, int64_t* tile_sums) {
  __shared__ int64_t warp_tot[kScanBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t x = (base + k < n) ? data[base + k] : 0;
    v[k] = run;
    run += x;
  }
  // exclusive scan of per-thread totals across the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
    int64_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kScanBlock / 32) warp_tot[lane] = ti - t;  // exclusive warp prefix
    if (lane == kScanBlock / 32 - 1 && tile_sums) tile_sums[blockIdx.x] = ti;
  }
  __syncthreads();
  const int64_t pre = warp_tot[w] + incl - run;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) data[base + k] = v[k] + pre;
}

__global__ void scan_add_kernel(int64_t* data, int64_t n, const int64_t* tile_pre) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) data[i] += tile_pre[i / kScanTile];
}

int64_t scan_scratch_count(int64_t n) {
  int64_t total = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    total += n + 1;
  }
  return total + 1;
}

cudaError_t exclusive_scan_i64(int64_t* data, int64_t n, int64_t* scratch, cudaStream_t stream, int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    scan_tiles_kernel<<<1, kScanBlock, 0, stream>>>(data, n, nullptr);
    ++*launches;
    return cudaGetLastError();
  }
  int64_t* sums = scratch;
  scan_tiles_kernel<<<(unsigned)tiles, kScanBlock, 0, stream>>>(data, n, sums);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  RETURN_IF(exclusive_scan_i64(sums, tiles, scratch + tiles + 1, stream, launches));
  scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(data, n, sums);
  ++*launches;
  return cudaGetLastError();
}

// ============================================================================
// Stable LSD radix sort, 8-bit digits.
//  pass: (1) per-tile digit histograms -> hist[digit * n_tiles + tile];
//        (2) exclusive scan of hist (digit-major) -> global start of each
//            (digit, tile) group;
//        (3) each tile loads its elements (all loads issued up front); each
//            warp ranks its 512 consecutive elements in order with match
//            masks and warp-private digit counters (stable, deterministic,
//            no block barrier); per-digit prefix sums over the warps and the
//            digits place the tile digit-sorted in shared memory, and every
//            digit's run goes to its global place with consecutive threads on
//            consecutive addresses (full-sector writes).
// ============================================================================
constexpr int kRadixBlock = 256;
constexpr int kRadixItems = 16;  // chunks per tile
constexpr int64_t kRadixTile = (int64_t)kRadixBlock * kRadixItems;
constexpr int kRadixWarps = kRadixBlock / 32;

template <typename K>
__global__ void __launch_bounds__(kRadixBlock) radix_hist_kernel(const K* keys, int64_t n, int shift,
                                                                 int64_t* hist, int64_t n_tiles) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  // every key of the thread loaded before the first count (the loads are then
  // all in flight at once instead of one per shared-memory atomic)
  unsigned dig[kRadixItems];
#pragma unroll
  for (int c = 0; c < kRadixItems; ++c) {
    const int64_t i = base + (int64_t)c * kRadixBlock + threadIdx.x;
    dig[c] = i < n ? (unsigned)(keys[i] >> shift) & 255u : 256u;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kRadixItems; ++c)
    if (dig[c] < 256u) atomicAdd(&cnt[dig[c]], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

template <typename K>
constexpr size_t radix_scatter_smem() {
  return (size_t)kRadixTile * (sizeof(K) + sizeof(uint32_t));
}

template <typename K>
__global__ void __launch_bounds__(kRadixBlock) radix_scatter_kernel(const K* keys_in, const uint32_t* vals_in,
                                                                    K* keys_out, uint32_t* vals_out, int64_t n,
                                                                    int shift, const int64_t* hist, int64_t n_tiles) {
  extern __shared__ __align__(16) unsigned char radix_smem[];
  K* skey = reinterpret_cast<K*>(radix_smem);
  uint32_t* sval = reinterpret_cast<uint32_t*>(radix_smem + sizeof(K) * kRadixTile);
  __shared__ int64_t gstart[256];          // global start of this tile's run of each digit
  __shared__ int lstart[256];              // tile-local start of each digit
  __shared__ int wc[kRadixWarps][256];     // per warp: count, then start, of each digit
  __shared__ int wsum[kRadixWarps];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  const int tile_n = (int)(n - base < kRadixTile ? n - base : kRadixTile);
  gstart[tid] = hist[(int64_t)tid * n_tiles + blockIdx.x];
#pragma unroll
  for (int k = 0; k < kRadixWarps; ++k) wc[k][tid] = 0;
  // warp w owns the tile's elements [w * 512, (w + 1) * 512), 32 per round
  K key[kRadixItems];
  uint32_t val[kRadixItems];
  unsigned dig[kRadixItems];
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const int li = w * (32 * kRadixItems) + j * 32 + lane;
    dig[j] = 256u;  // sentinel for lanes past the end
    if (li < tile_n) {
      key[j] = keys_in[base + li];
      val[j] = vals_in[base + li];
      dig[j] = (unsigned)(key[j] >> shift) & 255u;
    }
  }
  __syncthreads();
  // rank within the warp, in element order (rounds, then lanes)
  int rk[kRadixItems];
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const unsigned d = dig[j];
    const unsigned same = __match_any_sync(0xffffffffu, d);
    const int before = d < 256u ? wc[w][d] : 0;
    rk[j] = before + __popc(same & ((1u << lane) - 1u));
    __syncwarp();
    if (d < 256u && lane == __ffs(same) - 1) wc[w][d] = before + __popc(same);
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread tid = digit): warps' starts within the digit, tile total
  int run = 0;
#pragma unroll
  for (int k = 0; k < kRadixWarps; ++k) {
    const int x = wc[k][tid];
    wc[k][tid] = run;
    run += x;
  }
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int wpre = 0;
  for (int k = 0; k < w; ++k) wpre += wsum[k];
  lstart[tid] = wpre + incl - run;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const unsigned d = dig[j];
    if (d < 256u) {
      const int p = lstart[d] + wc[w][d] + rk[j];
      skey[p] = key[j];
      sval[p] = val[j];
    }
  }
  __syncthreads();
  for (int p = tid; p < tile_n; p += kRadixBlock) {
    const K k = skey[p];
    const unsigned d = (unsigned)(k >> shift) & 255u;
    const int64_t dst = gstart[d] + (p - lstart[d]);
    keys_out[dst] = k;
    vals_out[dst] = sval[p];
  }
}

int64_t radix_scratch_count(int64_t n) {
  const int64_t tiles = (n + kRadixTile - 1) / kRadixTile;
  const int64_t h = 256 * (tiles > 0 ? tiles : 1);
  return h + scan_scratch_count(h);
}

template <typename K>
static cudaError_t radix_sort_pairs_t(K* keys, uint32_t* vals, K* tmp_keys, uint32_t* tmp_vals, int64_t n, int bits,
                                      int64_t* scratch, cudaStream_t stream, int64_t* launches) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t tiles = (n + kRadixTile - 1) / kRadixTile;
  int64_t* hist = scratch;
  int64_t* scan_scratch = scratch + 256 * tiles;
  K *ki = keys, *ko = tmp_keys;
  uint32_t *vi = vals, *vo = tmp_vals;
  const int passes = (bits + 7) / 8;
  RETURN_IF(cudaFuncSetAttribute(radix_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)radix_scatter_smem<K>()));
  for (int p = 0; p < passes; ++p) {
    radix_hist_kernel<K><<<(unsigned)tiles, kRadixBlock, 0, stream>>>(ki, n, 8 * p, hist, tiles);
    ++*launches;
    RETURN_IF(cudaGetLastError());
    RETURN_IF(exclusive_scan_i64(hist, 256 * tiles, scan_scratch, stream, launches));
    radix_scatter_kernel<K><<<(unsigned)tiles, kRadixBlock, radix_scatter_smem<K>(), stream>>>(ki, vi, ko, vo, n,
                                                                                              8 * p, hist, tiles);
    ++*launches;
    RETURN_IF(cudaGetLastError());
    K* t = ki;
    ki = ko;
    ko = t;
    uint32_t* u = vi;
    vi = vo;
    vo = u;
  }
  if (ki != keys) {
    RETURN_IF(cudaMemcpyAsync(keys, ki, sizeof(K) * n, cudaMemcpyDeviceToDevice, stream));
    RETURN_IF(cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, stream));
  }
  return cudaSuccess;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tmp_keys, uint32_t* tmp_vals, int64_t n,
                             int bits, int64_t* scratch, cudaStream_t stream, int64_t* launches) {
  return radix_sort_pairs_t<uint32_t>(keys, vals, tmp_keys, tmp_vals, n, bits, scratch, stream, launches);
}

cudaError_t radix_sort_pairs64(uint64_t* keys, uint32_t* vals, uint64_t* tmp_keys, uint32_t* tmp_vals, int64_t n,
                               int bits, int64_t* scratch, cudaStream_t stream, int64_t* launches) {
  return radix_sort_pairs_t<uint64_t>(keys, vals, tmp_keys, tmp_vals, n, bits, scratch, stream, launches);
}

// ============================================================================
// Validation: the first violating index of each check (atomicMin, so the
// result does not depend on scheduling).
// ============================================================================
__device__ inline void amin(long long* p, long long v) { atomicMin(p, v); }

// every thread of a block reaches the warp reduction (whole warps: the block
// size is a multiple of 32)
__global__ void validate_voxels_kernel(LoadInput in, ValidateResult* r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int len = 0;  // the voxel's observation count (capped at 2^31 - 1), 0 if none or invalid
  if (i <= in.n_voxels) {
    const int64_t a = in.voxel_off[i];
    if (i == 0 && a != 0) amin(&r->first_bad_offset, 0);
    if (i == in.n_voxels) {
      if (a != in.n_obs) amin(&r->first_bad_offset, i);
    } else {
      const int64_t b = in.voxel_off[i + 1];
      if (b < a || a < 0 || b > in.n_obs) amin(&r->first_bad_offset, i);
      else if (b == a) amin(&r->first_empty_voxel, i);
      else len = (int)(b - a > 0x7fffffff ? 0x7fffffff : b - a);
    }
  }
  // one atomic per warp (one per voxel serialises on the single word)
  const int wmax = __reduce_max_sync(0xffffffffu, len);
  if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(&r->max_len, (long long)wmax);
}

__global__ void validate_scan_ids_kernel(LoadInput in, ValidateResult* r) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= in.n_obs) return;
  const int32_t j = in.obs_scan[o];
  if (j < 0 || j >= in.n_scans) amin(&r->first_bad_scan, o);
}

// clusters of observations [o0, o1): finite, and at least one point
__global__ void validate_agg_kernel(LoadInput in, int64_t o0, int64_t o1, ValidateResult* r) {
  const int64_t o = o0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= o1) return;
  const double* a = in.agg + 10 * o;
  bool fin = true;
#pragma unroll
  for (int k = 0; k < 10; ++k) fin = fin && isfinite(a[k]);
  if (!fin) amin(&r->first_nonfinite_agg, o);
  if (!(a[9] >= 1.0)) amin(&r->first_bad_count, o);
}

__global__ void validate_poses_kernel(LoadInput in, ValidateResult* r) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= in.n_scans) return;
  const double* P = in.poses + 12 * (int64_t)j;
  bool ok = true;
  for (int k = 0; k < 12; ++k) ok = ok && isfinite(P[k]);
  for (int a = 0; a < 3 && ok; ++a)
    for (int b = 0; b < 3; ++b) {
      const double d = P[3 * a] * P[3 * b] + P[3 * a + 1] * P[3 * b + 1] + P[3 * a + 2] * P[3 * b + 2];
      if (fabs(d - (a == b ? 1.0 : 0.0)) > 1e-6) ok = false;
    }
  if (ok) {  // proper rotation: det = +1
    const double det = P[0] * (P[4] * P[8] - P[5] * P[7]) - P[1] * (P[3] * P[8] - P[5] * P[6]) +
                       P[2] * (P[3] * P[7] - P[4] * P[6]);
    if (det < 0.0) ok = false;
  }
  if (!ok) amin(&r->first_bad_pose, j);
}

cudaError_t launch_validate(const LoadInput& in, ValidateResult* d_res, bool with_agg, cudaStream_t stream,
                            int64_t* launches) {
  validate_voxels_kernel<<<(unsigned)((in.n_voxels + 1 + 255) / 256), 256, 0, stream>>>(in, d_res);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  if (in.n_obs > 0) {
    validate_scan_ids_kernel<<<(unsigned)((in.n_obs + 255) / 256), 256, 0, stream>>>(in, d_res);
    ++*launches;
    RETURN_IF(cudaGetLastError());
    if (with_agg) RETURN_IF(launch_validate_agg(in, 0, in.n_obs, d_res, stream, launches));
  }
  validate_poses_kernel<<<(unsigned)((in.n_scans + 127) / 128), 128, 0, stream>>>(in, d_res);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_validate_agg(const LoadInput& in, int64_t o0, int64_t o1, ValidateResult* d_res,
                                cudaStream_t stream, int64_t* launches) {
  if (o1 <= o0) return cudaSuccess;
  validate_agg_kernel<<<(unsigned)((o1 - o0 + 255) / 256), 256, 0, stream>>>(in, o0, o1, d_res);
  ++*launches;
  return cudaGetLastError();
}

// ============================================================================
// Layout build
// ============================================================================

// Input cluster -> centred (S, m, N).  Raw sums: m = v / N and
// S_ab = fma(-v_a, m_b, P_ab).
__device__ inline void to_centred(const double* a, int form, double out[10]) {
  if (form == 1) {
#pragma unroll
    for (int k = 0; k < 10; ++k) out[k] = a[k];
    return;
  }
  const double n = a[9];
  const double mx = a[6] / n, my = a[7] / n, mz = a[8] / n;
  out[0] = fma(-a[6], mx, a[0]);
  out[1] = fma(-a[6], my, a[1]);
  out[2] = fma(-a[6], mz, a[2]);
  out[3] = fma(-a[7], my, a[3]);
  out[4] = fma(-a[7], mz, a[4]);
  out[5] = fma(-a[8], mz, a[5]);
  out[6] = mx;
  out[7] = my;
  out[8] = mz;
  out[9] = n;
}

// ---- spatial order of the voxels ----
// Mean translation of the scans observing each voxel (FP32, summed in the
// voxel's observation order), and the bounding box of those means as
// order-preserving unsigned encodings of the floats (min and max are exact,
// so the box does not depend on the order of the atomics).
__device__ __forceinline__ uint32_t float_order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float float_from_order_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void observer_mean_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ obs_scan,
                                     const double* __restrict__ poses, int64_t n_voxels, float4* __restrict__ mean,
                                     uint32_t* __restrict__ box) {
  __shared__ uint32_t sbox[6];
  if (threadIdx.x < 6) sbox[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
  __syncthreads();
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n_voxels) {
    const int64_t a0 = off[v], a1 = off[v + 1];
    float x = 0.f, y = 0.f, z = 0.f;
    for (int64_t o = a0; o < a1; ++o) {
      const double* t = poses + 12 * (int64_t)obs_scan[o] + 9;
      x += f64_to_f32(t[0]);
      y += f64_to_f32(t[1]);
      z += f64_to_f32(t[2]);
    }
    const float inv = 1.0f / (float)(a1 - a0);
    const float m[3] = {x * inv, y * inv, z * inv};
    mean[v] = make_float4(m[0], m[1], m[2], 0.f);
    for (int c = 0; c < 3; ++c) {
      atomicMin(&sbox[c], float_order_key(m[c]));
      atomicMax(&sbox[3 + c], float_order_key(m[c]));
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) atomicMin(&box[threadIdx.x], sbox[threadIdx.x]);
  else if (threadIdx.x < 6) atomicMax(&box[threadIdx.x], sbox[threadIdx.x]);
}

// 10 bits of each coordinate spread to every third bit
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void morton_keys_kernel(const float4* __restrict__ mean, int64_t n_voxels, const uint32_t* __restrict__ box,
                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_voxels) return;
  const float4 m = mean[v];
  const float mc[3] = {m.x, m.y, m.z};
  uint32_t code = 0;
  for (int c = 0; c < 3; ++c) {
    const float lo = float_from_order_key(box[c]), hi = float_from_order_key(box[3 + c]);
    uint32_t q = 0;
    if (hi > lo) {
      const float t = (mc[c] - lo) / (hi - lo) * 1023.0f;
      q = t <= 0.f ? 0u : t >= 1023.f ? 1023u : (uint32_t)t;
    }
    code |= spread3(q) << c;
  }
  keys[v] = code;
  vals[v] = (uint32_t)v;
}

// after the spatial sort (vals[r] = voxel of spatial rank r): window of the
// rank, then length descending
__global__ void window_keys_kernel(const int64_t* __restrict__ off, const uint32_t* __restrict__ vals,
                                   int64_t n_voxels, int max_len, int len_bits, uint32_t* __restrict__ keys) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_voxels) return;
  const uint32_t v = vals[r];
  const int64_t len = off[v + 1] - off[v];
  keys[r] = ((uint32_t)(r / kWindow) << len_bits) | (uint32_t)(max_len - len);
}

__global__ void slice_len_kernel(const int64_t* off, const uint32_t* vperm, int64_t n_voxels, int64_t n_slices,
                                 int64_t* slice_off, int32_t* vlen, int32_t* vperm_out, int32_t* vrank) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_voxels) {
    const uint32_t v = vperm[p];
    const int32_t len = (int32_t)(off[v + 1] - off[v]);
    vlen[p] = len;
    vperm_out[p] = (int32_t)v;
    vrank[v] = (int32_t)p;
    if ((p & 31) == 0) slice_off[p >> 5] = (int64_t)kSlice * len;  // first voxel is the longest of its slice
  }
  if (p == 0) slice_off[n_slices] = 0;
}

__global__ void fill_sell_kernel(LoadInput in, const int32_t* vperm, const int32_t* vlen, const int64_t* slice_off,
                                 int64_t n_voxels, double* ve, int32_t* ve_scan, int64_t n_elems) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = p >> 5;
  if (s * kSlice >= n_voxels) return;
  const int lane = (int)(p & 31);
  const int64_t base = slice_off[s] + lane;
  const int64_t rows = (slice_off[s + 1] - slice_off[s]) / kSlice;
  const bool real = p < n_voxels;
  const int32_t len = real ? vlen[p] : 0;
  const int64_t o0 = real ? in.voxel_off[vperm[p]] : 0;
  for (int64_t k = 0; k < rows; ++k) {
    const int64_t e = base + k * kSlice;
    double c[10], f[10];
    uint32_t scan = 0;
    if (k < len) {
      to_centred(in.agg + 10 * (o0 + k), in.agg_form, c);
      // the scatter as its pivoted LDL^T, the mean permuted alike
      const uint32_t code = ldlt3_pivoted(c, f);
      int p0, p1, p2;
      perm_decode(code, p0, p1, p2);
      f[6] = c[6 + p0];
      f[7] = c[6 + p1];
      f[8] = c[6 + p2];
      f[9] = c[9];
      scan = (uint32_t)in.obs_scan[o0 + k] | (code << kPermShift);
    } else {
#pragma unroll
      for (int q = 0; q < 10; ++q) f[q] = 0.0;
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) ve[q * n_elems + e] = f[q];
    ve_scan[e] = (int32_t)scan;
  }
}

// voxel of every observation, and (unless vscale is null) each voxel's 2 / N_i
__global__ void obs_voxel_kernel(LoadInput in, int32_t* obs_vox, double* vscale) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= in.n_voxels) return;
  double n = 0.0;
  for (int64_t o = in.voxel_off[v]; o < in.voxel_off[v + 1]; ++o) {
    obs_vox[o] = (int32_t)v;
    if (vscale) n += in.agg[10 * o + 9];
  }
  if (vscale) vscale[v] = 2.0 / n;
}

// 2 / N_i of voxels [v0, v1)
__global__ void vscale_kernel(LoadInput in, int64_t v0, int64_t v1, double* vscale) {
  const int64_t v = v0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= v1) return;
  double n = 0.0;
  for (int64_t o = in.voxel_off[v]; o < in.voxel_off[v + 1]; ++o) n += in.agg[10 * o + 9];
  vscale[v] = 2.0 / n;
}

// observations listed by sorted voxel position (pbase[p] = observations of
// the voxels before position p), keyed by scan for the stable sort that makes
// the scan-major copy: inside a scan, observations follow the voxel order, so
// the scan pass gathers the plane records of nearby voxels
__global__ void scan_keys_kernel(LoadInput in, const int32_t* obs_vox, const int32_t* vrank, const int64_t* pbase,
                                 uint32_t* keys, uint32_t* vals) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= in.n_obs) return;
  const int32_t v = obs_vox[o];
  const int64_t q = pbase[vrank[v]] + (o - in.voxel_off[v]);
  keys[q] = (uint32_t)in.obs_scan[o];
  vals[q] = (uint32_t)o;
}

// scan_off[j] = the first scan-major position of scan j (n at the end), from
// the scan ids sorted ascending: position q starts every scan after its
// predecessor's id up to its own (scans with no observation included), so
// each entry is written once
__global__ void scan_off_kernel(const uint32_t* keys, int64_t n, int32_t n_scans, int64_t* scan_off) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q > n) return;
  const int64_t lo = q == 0 ? 0 : (int64_t)keys[q - 1] + 1;
  const int64_t hi = q == n ? (int64_t)n_scans : (int64_t)keys[q];
  for (int64_t j = lo; j <= hi; ++j) scan_off[j] = q;
}

__global__ void vlen_i64_kernel(const int32_t* vlen, int64_t n_voxels, int64_t* out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_voxels) out[p] = vlen[p];
  if (p == 0) out[n_voxels] = 0;
}

__global__ void fill_scan_major_kernel(LoadInput in, const uint32_t* order, const int32_t* obs_vox,
                                       const double* vscale, const int32_t* vrank, double* se, int32_t* se_vox) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= in.n_obs) return;
  const int64_t o = order[q];
  const int32_t v = obs_vox[o];
  se_vox[q] = vrank[v];
  if (!se) return;
  double c[10];
  to_centred(in.agg + 10 * o, in.agg_form, c);
  const double k = vscale[v];
#pragma unroll
  for (int a = 0; a < 6; ++a) c[a] *= k;
  c[9] *= k;
  const int64_t n = in.n_obs;
#pragma unroll
  for (int a = 0; a < 10; ++a) se[a * n + q] = c[a];
}

// chunk index of each scan-major position's observation (its place among
// the chunk bounds), keyed for a stable one-digit partition
__global__ void chunk_keys_kernel(const uint32_t* order, int64_t n, ChunkBounds cb, uint32_t* keys, uint32_t* vals) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int64_t o = order[q];
  uint32_t c = 0;
  for (int k = 1; k < cb.n; ++k) c += o >= cb.o[k] ? 1u : 0u;
  keys[q] = c;
  vals[q] = (uint32_t)q;
}

static int bit_width(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

cudaError_t launch_vscale(const LoadInput& in, int64_t v0, int64_t v1, double* vscale, cudaStream_t stream,
                          int64_t* launches) {
  if (v1 <= v0) return cudaSuccess;
  vscale_kernel<<<(unsigned)((v1 - v0 + 255) / 256), 256, 0, stream>>>(in, v0, v1, vscale);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t group_by_chunk(const uint32_t* order, int64_t n_obs, const ChunkBounds& cb, uint32_t* out_q,
                           Allocator temp, cudaStream_t stream, int64_t* launches) {
  if (n_obs <= 0) return cudaSuccess;
  if (cb.n < 1 || cb.n > kMaxCopyChunks) return cudaErrorInvalidValue;
  uint32_t* keys = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * n_obs);
  uint32_t* tk = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * n_obs);
  uint32_t* tv = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * n_obs);
  int64_t* scratch = (int64_t*)temp.fn(temp.self, sizeof(int64_t) * radix_scratch_count(n_obs));
  if (!keys || !tk || !tv || !scratch) return cudaErrorMemoryAllocation;
  chunk_keys_kernel<<<(unsigned)((n_obs + 255) / 256), 256, 0, stream>>>(order, n_obs, cb, keys, out_q);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  return radix_sort_pairs(keys, out_q, tk, tv, n_obs, bit_width((uint64_t)(cb.n - 1)), scratch, stream, launches);
}

cudaError_t build_layout(const LoadInput& in, int max_len, bool fill_f64, bool defer_scale, Allocator keep,
                         Allocator temp, LayoutBuffers* out, cudaStream_t stream, int64_t* launches) {
  const int64_t nv = in.n_voxels, no = in.n_obs;
  const int64_t n_slices = (nv + kSlice - 1) / kSlice;
  const int64_t nsort = nv > no ? nv : no;
  // temporaries (the maps are kept when the FP32 copies will be rebuilt later)
  Allocator maps = fill_f64 ? temp : keep;
  uint32_t* keys = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * nsort);
  uint32_t* vals = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * nsort);
  uint32_t* tk = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * nsort);
  uint32_t* tv = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * nsort);
  int64_t* scratch = (int64_t*)temp.fn(temp.self, sizeof(int64_t) * (radix_scratch_count(nsort) +
                                                                      scan_scratch_count(n_slices + no + 2)));
  int32_t* vrank = (int32_t*)maps.fn(maps.self, sizeof(int32_t) * nv);
  int32_t* obs_vox = (int32_t*)maps.fn(maps.self, sizeof(int32_t) * no);
  double* vscale = (double*)maps.fn(maps.self, sizeof(double) * nv);
  uint32_t* order = fill_f64 ? nullptr : (uint32_t*)keep.fn(keep.self, sizeof(uint32_t) * no);
  // persistent
  out->slice_off = (int64_t*)keep.fn(keep.self, sizeof(int64_t) * (n_slices + 1));
  out->vlen = (int32_t*)keep.fn(keep.self, sizeof(int32_t) * nv);
  out->vperm = (int32_t*)keep.fn(keep.self, sizeof(int32_t) * nv);
  out->scan_off = (int64_t*)keep.fn(keep.self, sizeof(int64_t) * (in.n_scans + 1));
  out->se = fill_f64 ? (double*)keep.fn(keep.self, sizeof(double) * 10 * no) : nullptr;
  // + 4 entries: the staged mixed scan pass copies whole 16-byte groups
  out->se_vox = (int32_t*)keep.fn(keep.self, sizeof(int32_t) * (no + 4));
  if (!keys || !vals || !tk || !tv || !scratch || !vrank || !obs_vox || !vscale || !out->slice_off || !out->vlen ||
      !out->vperm || !out->scan_off || (fill_f64 && !out->se) || (!fill_f64 && !order) || !out->se_vox)
    return cudaErrorMemoryAllocation;
  out->vrank = vrank;
  out->obs_vox = obs_vox;
  out->vscale = vscale;
  out->scan_order = order;

  // ---- voxel order: spatial windows, length-descending inside each ----
  const int len_bits = bit_width((uint64_t)max_len);
  const int win_bits = bit_width((uint64_t)((nv - 1) / kWindow));
  if (len_bits + win_bits > 32) return cudaErrorInvalidValue;
  {
    float4* mean = (float4*)temp.fn(temp.self, sizeof(float4) * nv);
    uint32_t* box = (uint32_t*)temp.fn(temp.self, sizeof(uint32_t) * 8);
    if (!mean || !box) return cudaErrorMemoryAllocation;
    RETURN_IF(cudaMemsetAsync(box, 0xff, sizeof(uint32_t) * 3, stream));  // minima
    RETURN_IF(cudaMemsetAsync(box + 3, 0, sizeof(uint32_t) * 3, stream));  // maxima
    const unsigned nb = (unsigned)((nv + 255) / 256);
    observer_mean_kernel<<<nb, 256, 0, stream>>>(in.voxel_off, in.obs_scan, in.poses, nv, mean, box);
    morton_keys_kernel<<<nb, 256, 0, stream>>>(mean, nv, box, keys, vals);
    *launches += 2;
    RETURN_IF(cudaGetLastError());
    RETURN_IF(radix_sort_pairs(keys, vals, tk, tv, nv, 30, scratch, stream, launches));
    window_keys_kernel<<<nb, 256, 0, stream>>>(in.voxel_off, vals, nv, max_len, len_bits, keys);
    ++*launches;
    RETURN_IF(cudaGetLastError());
  }
  RETURN_IF(radix_sort_pairs(keys, vals, tk, tv, nv, len_bits + win_bits, scratch, stream, launches));
  slice_len_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, stream>>>(in.voxel_off, vals, nv, n_slices,
                                                                     out->slice_off, out->vlen, out->vperm, vrank);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  RETURN_IF(exclusive_scan_i64(out->slice_off, n_slices + 1, scratch, stream, launches));
  int64_t n_elems = 0;
  RETURN_IF(cudaMemcpyAsync(&n_elems, out->slice_off + n_slices, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  RETURN_IF(cudaStreamSynchronize(stream));
  out->n_elems = n_elems;
  out->n_slices = n_slices;
  out->max_len = max_len;
  // the FP64 slice copy (the mixed path builds its own FP32 slots)
  if (fill_f64) {
    out->ve = (double*)keep.fn(keep.self, sizeof(double) * 10 * n_elems);
    out->ve_scan = (int32_t*)keep.fn(keep.self, sizeof(int32_t) * n_elems);
    if (!out->ve || !out->ve_scan) return cudaErrorMemoryAllocation;
    fill_sell_kernel<<<(unsigned)((n_slices * kSlice + 255) / 256), 256, 0, stream>>>(
        in, out->vperm, out->vlen, out->slice_off, nv, out->ve, out->ve_scan, n_elems);
    ++*launches;
    RETURN_IF(cudaGetLastError());
  }

  // ---- scan-major copy ----
  obs_voxel_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, stream>>>(in, obs_vox, defer_scale ? nullptr : vscale);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  {
    // kept by a load that stages its slots (they are staged in this order)
    Allocator pb_alloc = defer_scale ? keep : temp;
    int64_t* pbase = (int64_t*)pb_alloc.fn(pb_alloc.self, sizeof(int64_t) * (nv + 1));
    int64_t* pscratch = (int64_t*)temp.fn(temp.self, sizeof(int64_t) * scan_scratch_count(nv + 1));
    if (!pbase || !pscratch) return cudaErrorMemoryAllocation;
    vlen_i64_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, stream>>>(out->vlen, nv, pbase);
    ++*launches;
    RETURN_IF(cudaGetLastError());
    RETURN_IF(exclusive_scan_i64(pbase, nv + 1, pscratch, stream, launches));
    out->vstart = defer_scale ? pbase : nullptr;
    scan_keys_kernel<<<(unsigned)((no + 255) / 256), 256, 0, stream>>>(in, obs_vox, vrank, pbase, keys, vals);
    ++*launches;
    RETURN_IF(cudaGetLastError());
  }
  RETURN_IF(radix_sort_pairs(keys, vals, tk, tv, no, bit_width((uint64_t)(in.n_scans - 1)), scratch, stream,
                             launches));
  scan_off_kernel<<<(unsigned)((no + 1 + 255) / 256), 256, 0, stream>>>(keys, no, in.n_scans, out->scan_off);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  fill_scan_major_kernel<<<(unsigned)((no + 255) / 256), 256, 0, stream>>>(in, vals, obs_vox, vscale, vrank, out->se,
                                                                           out->se_vox);
  ++*launches;
  RETURN_IF(cudaGetLastError());
  if (order) RETURN_IF(cudaMemcpyAsync(order, vals, sizeof(uint32_t) * no, cudaMemcpyDeviceToDevice, stream));
  return cudaSuccess;
}

// ============================================================================
// Point clusters (Eq. 2) in centred form: two lanes per observation (sixteen
// observations per warp; the pair reads neighbouring points, so a sector's
// three coordinates come from one fetch), one pass over the points as sums
// shifted by the observation's first point p0: with d = p - p0,
//   m = p0 + (sum d) / N,   S = sum d d^T - (sum d)(sum d)^T / N,
// algebraically the mean and the scatter about it (Eq. 2 fixes the sums, not
// their order).
//
// The sums are exact integer sums in fixed point.  An observation's scale is
// 2^-F with F = 1076 - E0, E0 the largest biased binary exponent of p0's
// coordinates: p0's largest coordinate then has its last bit at 2^-F, every
// coordinate of that size or larger (up to 2^9 times) is an exact integer
// multiple of 2^-F, and smaller ones are rounded to it (an error below half
// the last bit of p0's largest coordinate, the resolution of FP64 arithmetic
// on these points).  d, sum d and sum d d^T are then 64- and 128-bit integer
// sums with no rounding at all, on the integer pipe; GB300's FP64 pipe (1/64
// of FP32) only converts the nine sums and forms m and S once per
// observation.  An observation whose points do not fit (a coordinate over 2^9
// times p0's largest, a spread over 2^56 steps, more than 2^14 points, a
// first point at the origin, or a scale outside 2^-500 .. 2^500) takes the
// same shifted sums in FP64.
// ============================================================================
constexpr int kAggLanes = 2;

// 2^-F as an FP64 value, for F in [-1022, 1022]
__device__ __forceinline__ double pow2_neg(int F) { return __hiloint2double((1023 - F) << 20, 0); }

// round(p 2^F) to the nearest integer (halves away from zero); ok is cleared
// when the result would reach 2^62
__device__ __forceinline__ long long fix_round(double p, int F, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(p);
  const int E = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1075 + F;
  unsigned long long v = 0;
  if (E != 0) {  // zero and subnormal values are below the resolution
    if (sh >= 0) {
      ok = ok && sh <= 9;
      v = m << (sh & 15);
    } else if (sh > -63) {
      const int r = -sh;
      v = (m + (1ull << (r - 1))) >> r;
    }
  }
  return (b >> 63) ? -(long long)v : (long long)v;
}

// the nearest FP64 values to the magnitude's two 64-bit halves, combined by
// one FMA (an error of about one unit in the last place); the sign is set in
// the bits
__device__ __forceinline__ double i128_to_double(__int128 v) {
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const double r = fma((double)(unsigned long long)(u >> 64), 0x1p64, (double)(unsigned long long)u);
  return __longlong_as_double(__double_as_longlong(r) | ((long long)neg << 63));
}

__device__ __forceinline__ __int128 shfl_xor_i128(unsigned mask, __int128 v, int lane) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
  const unsigned long long lo2 = __shfl_xor_sync(mask, lo, lane), hi2 = __shfl_xor_sync(mask, hi, lane);
  return (__int128)(((unsigned __int128)hi2 << 64) | lo2);
}

// the shifted sums in FP64 (observations the fixed point does not fit)
__device__ void aggregate_f64(int64_t a, int64_t b, int sub, unsigned mask, const double* __restrict__ pts,
                              double* __restrict__ r) {
  const double p0x = pts[3 * a], p0y = pts[3 * a + 1], p0z = pts[3 * a + 2];
  double sx = 0.0, sy = 0.0, sz = 0.0;
  double c00 = 0.0, c01 = 0.0, c02 = 0.0, c11 = 0.0, c12 = 0.0, c22 = 0.0;
  for (int64_t k = a + sub; k < b; k += kAggLanes) {
    const double x = pts[3 * k] - p0x, y = pts[3 * k + 1] - p0y, z = pts[3 * k + 2] - p0z;
    sx += x;
    sy += y;
    sz += z;
    c00 = fma(x, x, c00);
    c01 = fma(x, y, c01);
    c02 = fma(x, z, c02);
    c11 = fma(y, y, c11);
    c12 = fma(y, z, c12);
    c22 = fma(z, z, c22);
  }
  sx += __shfl_xor_sync(mask, sx, 1);
  sy += __shfl_xor_sync(mask, sy, 1);
  sz += __shfl_xor_sync(mask, sz, 1);
  c00 += __shfl_xor_sync(mask, c00, 1);
  c01 += __shfl_xor_sync(mask, c01, 1);
  c02 += __shfl_xor_sync(mask, c02, 1);
  c11 += __shfl_xor_sync(mask, c11, 1);
  c12 += __shfl_xor_sync(mask, c12, 1);
  c22 += __shfl_xor_sync(mask, c22, 1);
  const double n = (double)(b - a);
  const double rn = 1.0 / n;
  const double dx = sx * rn, dy = sy * rn, dz = sz * rn;
  if (sub == 0) {
    r[0] = fma(-sx, dx, c00);
    r[1] = fma(-sx, dy, c01);
    r[2] = fma(-sx, dz, c02);
    r[3] = fma(-sy, dy, c11);
    r[4] = fma(-sy, dz, c12);
  } else {
    r[5] = fma(-sz, dz, c22);
    r[6] = p0x + dx;
    r[7] = p0y + dy;
    r[8] = p0z + dz;
    r[9] = n;
  }
}

__global__ void aggregate_points_kernel(int64_t n_obs, const int64_t* __restrict__ off,
                                        const double* __restrict__ pts, double* __restrict__ out) {
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kAggLanes;
  const int sub = threadIdx.x & (kAggLanes - 1);
  const unsigned mask = 0x3u << (threadIdx.x & 30);  // the two lanes of this observation
  if (o >= n_obs) return;  // both lanes of a pair leave together
  const int64_t a = off[o], b = off[o + 1];
  double* r = out + 10 * o;
  if (b <= a) {
    for (int k = sub; k < 10; k += kAggLanes) r[k] = 0.0;
    return;
  }
  const double p0x = pts[3 * a], p0y = pts[3 * a + 1], p0z = pts[3 * a + 2];
  int E0 = (__double2hiint(p0x) >> 20) & 0x7ff;
  E0 = max(E0, (__double2hiint(p0y) >> 20) & 0x7ff);
  E0 = max(E0, (__double2hiint(p0z) >> 20) & 0x7ff);
  const int F = 1076 - E0;
  bool ok = E0 != 0 && F >= -500 && F <= 500 && b - a <= (1 << 14);
  const long long X0x = fix_round(p0x, F, ok), X0y = fix_round(p0y, F, ok), X0z = fix_round(p0z, F, ok);
  __int128 s1x = 0, s1y = 0, s1z = 0, s00 = 0, s01 = 0, s02 = 0, s11 = 0, s12 = 0, s22 = 0;
  constexpr long long kMaxD = 1ll << 56;
  for (int64_t k = a + sub; k < b && ok; k += kAggLanes) {
    const long long dx = fix_round(pts[3 * k], F, ok) - X0x;
    const long long dy = fix_round(pts[3 * k + 1], F, ok) - X0y;
    const long long dz = fix_round(pts[3 * k + 2], F, ok) - X0z;
    ok = ok && dx > -kMaxD && dx < kMaxD && dy > -kMaxD && dy < kMaxD && dz > -kMaxD && dz < kMaxD;
    s1x += dx;
    s1y += dy;
    s1z += dz;
    s00 += (__int128)dx * dx;
    s01 += (__int128)dx * dy;
    s02 += (__int128)dx * dz;
    s11 += (__int128)dy * dy;
    s12 += (__int128)dy * dz;
    s22 += (__int128)dz * dz;
  }
  // both lanes take the shuffle (a short-circuit would skip it on one of them)
  const int partner_ok = __shfl_xor_sync(mask, (int)ok, 1);
  ok = ok && partner_ok != 0;
  if (!ok) {
    aggregate_f64(a, b, sub, mask, pts, r);
    return;
  }
  s1x += shfl_xor_i128(mask, s1x, 1);
  s1y += shfl_xor_i128(mask, s1y, 1);
  s1z += shfl_xor_i128(mask, s1z, 1);
  s00 += shfl_xor_i128(mask, s00, 1);
  s01 += shfl_xor_i128(mask, s01, 1);
  s02 += shfl_xor_i128(mask, s02, 1);
  s11 += shfl_xor_i128(mask, s11, 1);
  s12 += shfl_xor_i128(mask, s12, 1);
  s22 += shfl_xor_i128(mask, s22, 1);
  // Both lanes hold the exact sums.  Each converts five of them and writes
  // half of the record through one instruction sequence whose operands are
  // chosen per lane (lane 0: S xx, xy, xz, yy, yz = C - s_a d_b; lane 1: S zz,
  // then m = p0 + d and N), since GB300 issues an FP64 warp instruction at the
  // same cost whatever the number of lanes on each side of a branch.
  const double sc = pow2_neg(F);  // F is in [-500, 500]
  const double sc2 = sc * sc;
  const double n = (double)(b - a);
  const double rn = 1.0 / n;
  const double sx = i128_to_double(s1x) * sc, sy = i128_to_double(s1y) * sc, sz = i128_to_double(s1z) * sc;
  const double dx = sx * rn, dy = sy * rn, dz = sz * rn;
  const bool l0 = sub == 0;
  const __int128 v[5] = {l0 ? s00 : s22, l0 ? s01 : (__int128)X0x, l0 ? s02 : (__int128)X0y,
                         l0 ? s11 : (__int128)X0z, l0 ? s12 : (__int128)0};
  const double A[5] = {l0 ? -sx : -sz, l0 ? -sx : 1.0, l0 ? -sx : 1.0, l0 ? -sy : 1.0, l0 ? -sy : n};
  const double B[5] = {l0 ? dx : dz, l0 ? dy : dx, l0 ? dz : dy, l0 ? dy : dz, l0 ? dz : 1.0};
  const double S[5] = {sc2, l0 ? sc2 : sc, l0 ? sc2 : sc, l0 ? sc2 : sc, sc2};
  double* w = r + 5 * sub;
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = fma(A[k], B[k], i128_to_double(v[k]) * S[k]);
}

cudaError_t launch_aggregate_points(int64_t n_obs, const int64_t* point_off, const double* points, double* agg_out,
                                    cudaStream_t stream) {
  if (n_obs <= 0) return cudaSuccess;
  const int64_t threads = n_obs * kAggLanes;
  aggregate_points_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(n_obs, point_off, points, agg_out);
  return cudaGetLastError();
}

}  // namespace mmba
