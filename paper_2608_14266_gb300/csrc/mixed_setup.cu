// Set-up of the mixed-precision copies (once per load and at ba_set_state):
// per-scan reference poses, per-voxel anchors and starting frames at those
// poses, and the FP32 re-centred clusters in the slice layout (offset to the
// anchor plus each observation's scatter as eigenvalues and the quaternion of
// its eigenvectors) and in the scan-major layout (reference axes, scaled by
// 2 / N_i).  FP64 is used where digits would otherwise be lost (offsets of
// scene-sized positions from the anchor, the scatter in the basis of its FP32
// eigenvectors); the rest is FP32 (GB300's FP64 rate is 1/64 of FP32).
#include <algorithm>

#include "mmba_internal.cuh"
#include "mmba_kernels.h"

namespace mmba {

namespace {

constexpr int kFillRows = 4;  // slice rows per thread of the slot fill

__device__ inline void centred_cluster(const double* a, int form, double out[10]) {
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

// reference pose of each scan: R_ref = R, t_ref = t rounded to FP32; the
// sref buffer holds n_scans x 12 doubles followed by the same 12 values of
// every scan in FP32 (sref32), so per-observation set-up needs no FP64 -> FP32
// conversions of the rotation
__global__ void scan_ref_kernel(int32_t n_scans, const double* poses, double* sref) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_scans) return;
  const double* P = poses + 12 * (int64_t)j;
  double* o = sref + 12 * (int64_t)j;
  float* f = reinterpret_cast<float*>(sref + 12 * (int64_t)n_scans) + 12 * (int64_t)j;
  for (int k = 0; k < 9; ++k) {
    o[k] = P[k];
    f[k] = (float)P[k];
  }
  for (int k = 9; k < 12; ++k) {
    o[k] = (double)(float)P[k];
    f[k] = (float)P[k];
  }
}

__device__ __forceinline__ const float* sref32_of(const double* sref, int32_t n_scans, int32_t j) {
  return reinterpret_cast<const float*>(sref + 12 * (int64_t)n_scans) + 12 * (int64_t)j;
}

// packed symmetric R S R^T in FP32 (R row-major, S packed xx xy xz yy yz zz)
__device__ inline void rot_sym_f(const float* Rf, const float* Sf, float* out) {
  float M[3][3];
  M[0][0] = Sf[0];
  M[0][1] = M[1][0] = Sf[1];
  M[0][2] = M[2][0] = Sf[2];
  M[1][1] = Sf[3];
  M[1][2] = M[2][1] = Sf[4];
  M[2][2] = Sf[5];
  float T[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) T[r][c] = fmaf(Rf[3 * r], M[0][c], fmaf(Rf[3 * r + 1], M[1][c], Rf[3 * r + 2] * M[2][c]));
  int idx = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c)
      out[idx++] = fmaf(T[r][0], Rf[3 * c], fmaf(T[r][1], Rf[3 * c + 1], T[r][2] * Rf[3 * c + 2]));
}


// Double-float (hi + lo, two binary32 values) arithmetic from the classical
// error-free transformations: Knuth's two-sum and the FMA form of Dekker's
// two-product (the rounding error of a * b is fma(a, b, -a * b) exactly).
// It carries ~46 significant bits on the FP32 pipe, where GB300 issues 64
// times the FP64 rate.  The transformations use the _rn intrinsics, which
// the compiler never contracts into FMAs (a contraction would break their
// exactness).
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// acc + x * (y_hi + y_lo) for a binary32 x
__device__ __forceinline__ DF df_fma(DF acc, float x, DF y) {
  const float p = __fmul_rn(x, y.hi);
  const float e = fmaf(x, y.hi, -p);  // exact error of the product
  const DF s = df_two_sum(acc.hi, p);
  return DF{s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, fmaf(x, y.lo, e)))};
}

// FP32 copies of a cluster's scatter, mean and count (integer-arithmetic
// conversions: GB300 converts on its narrow FP64 pipe)
__device__ __forceinline__ void cluster_f32(const double* c, float* Sf, float* mf, float& N) {
#pragma unroll
  for (int k = 0; k < 6; ++k) Sf[k] = f64_to_f32(c[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) mf[k] = f64_to_f32(c[6 + k]);
  N = f64_to_f32(c[9]);
}

// posed mean R m + t_ref in FP32 (from the FP32 reference table: R, t_ref)
__device__ __forceinline__ void posed_f32(const float* ref32, const float* m, float* q) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    q[a] = fmaf(ref32[3 * a], m[0], fmaf(ref32[3 * a + 1], m[1], fmaf(ref32[3 * a + 2], m[2], ref32[9 + a])));
}

// anchor (FP32-rounded centroid) and starting frame (eigenvectors, normal
// last, proper rotation) of each voxel at the reference poses, kFrameLanes
// threads per voxel taking its observations in turn (lane l the l-th, then
// every kFrameLanes-th) in one pass: sums of N d and N d d^T + R S R^T with d
// the posed mean's offset from the voxel's first posed mean, combined by a
// butterfly so that every lane holds the same totals, then moved to the
// centroid (A = M - s s^T / n); the group's first lane solves the 3x3
// eigenproblem.  Both results only seed the iteration (the voxel pass moves
// the frame and the centroid every pass, and the anchor only has to be an FP32
// value near the centroid), so the sums are FP32: errors of the order of an
// FP32 ulp of the scene coordinates (~1e-4 m at 2 km) and of the voxel's
// spread move nothing but the seed.
constexpr int kFrameLanes = 8;

// x summed over the group of kFrameLanes lanes (the same value in every lane:
// each step adds the same two values in either order)
__device__ __forceinline__ float group_sum(unsigned mask, float x) {
#pragma unroll
  for (int k = 1; k < kFrameLanes; k <<= 1) x += __shfl_xor_sync(mask, x, k);
  return x;
}

__global__ void __launch_bounds__(128) voxel_frames_kernel(LoadInput in, int64_t v0, int64_t v1, const double* sref,
                                                           const int32_t* vrank, float4* vstate, float4* vanchor,
                                                           float4* planes2) {
  static_assert(32 % kFrameLanes == 0 && 128 % kFrameLanes == 0, "groups must not straddle warps");
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = v0 + t / kFrameLanes;
  const int sub = (int)(t % kFrameLanes);
  if (v >= v1) return;  // whole groups leave together
  const unsigned mask = ((1u << kFrameLanes) - 1u) << ((threadIdx.x & 31) & ~(kFrameLanes - 1));
  const int64_t a0 = in.voxel_off[v], a1 = in.voxel_off[v + 1];
  float p0[3];
  {
    float Sf[6], mf[3], N;
    double c[10];
    centred_cluster(in.agg + 10 * a0, in.agg_form, c);
    cluster_f32(c, Sf, mf, N);
    posed_f32(sref32_of(sref, in.n_scans, in.obs_scan[a0]), mf, p0);
  }
  float n = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
  float M[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t o = a0 + sub; o < a1; o += kFrameLanes) {
    double c[10];
    centred_cluster(in.agg + 10 * o, in.agg_form, c);
    float Sf[6], mf[3], N, q[3], rs[6];
    cluster_f32(c, Sf, mf, N);
    const float* Rf = sref32_of(sref, in.n_scans, in.obs_scan[o]);
    posed_f32(Rf, mf, q);
    rot_sym_f(Rf, Sf, rs);
    const float dx = q[0] - p0[0], dy = q[1] - p0[1], dz = q[2] - p0[2];
    sx = fmaf(N, dx, sx);
    sy = fmaf(N, dy, sy);
    sz = fmaf(N, dz, sz);
    n += N;
    M[0] += fmaf(N * dx, dx, rs[0]);
    M[1] += fmaf(N * dx, dy, rs[1]);
    M[2] += fmaf(N * dx, dz, rs[2]);
    M[3] += fmaf(N * dy, dy, rs[3]);
    M[4] += fmaf(N * dy, dz, rs[4]);
    M[5] += fmaf(N * dz, dz, rs[5]);
  }
  n = group_sum(mask, n);
  sx = group_sum(mask, sx);
  sy = group_sum(mask, sy);
  sz = group_sum(mask, sz);
#pragma unroll
  for (int k = 0; k < 6; ++k) M[k] = group_sum(mask, M[k]);
  const float cx = sx / n, cy = sy / n, cz = sz / n;  // centroid - p0
  const float A[6] = {fmaf(-sx, cx, M[0]), fmaf(-sx, cy, M[1]), fmaf(-sx, cz, M[2]),
                      fmaf(-sy, cy, M[3]), fmaf(-sy, cz, M[4]), fmaf(-sz, cz, M[5])};
  if (sub != 0) return;
  float lam[3], V[9];
  eig3_sym_f(A, lam, V);
  // rows: e1 (largest), e2, n (smallest)
  float U[9] = {V[6], V[7], V[8], V[3], V[4], V[5], V[0], V[1], V[2]};
  const float det = U[0] * (U[4] * U[8] - U[5] * U[7]) - U[1] * (U[3] * U[8] - U[5] * U[6]) +
                    U[2] * (U[3] * U[7] - U[4] * U[6]);
  if (det < 0.f)
    for (int k = 0; k < 3; ++k) U[k] = -U[k];
  float q[4];
  mat_to_quat<float>(U, q);
  // anchor: the centroid rounded to FP32; the running centroid starts at the
  // remainder (FP32 arithmetic, exact for the rounding step of a sum)
  const float ax = p0[0] + cx, ay = p0[1] + cy, az = p0[2] + cz;
  const int64_t p = vrank[v];
  vanchor[p] = make_float4(ax, ay, az, 0.0f);
  // the anchor also sits beside the plane in both buffers of plane records
  planes2[2 * p + 1] = make_float4(ax, ay, az, 0.0f);
  planes2[2 * (in.n_voxels + p) + 1] = make_float4(ax, ay, az, 0.0f);
  vstate[2 * p] = make_float4(q[0], q[1], q[2], q[3]);
  vstate[2 * p + 1] = make_float4((p0[0] - ax) + cx, (p0[1] - ay) + cy, (p0[2] - az) + cz, 0.0f);
}

// b = R_ref m + t_ref - a (world axes), for an observation of a voxel whose
// anchor is an
__device__ inline void offset_b(const double* c, const double* ref, float4 an, double b[3]) {
  b[0] = ref[0] * c[6] + ref[1] * c[7] + ref[2] * c[8] + (ref[9] - f32_to_f64(an.x));
  b[1] = ref[3] * c[6] + ref[4] * c[7] + ref[5] * c[8] + (ref[10] - f32_to_f64(an.y));
  b[2] = ref[6] * c[6] + ref[7] * c[7] + ref[8] * c[8] + (ref[11] - f32_to_f64(an.z));
}

// the slot of observation o of a voxel with anchor an: offset to the anchor
// and count, eigenvalues of the scatter and scan id, eigenvector quaternion
__device__ void mixed_slot(const LoadInput& in, int64_t o, const double* sref, float4 an, float4& s0, float4& s1,
                           float4& s2) {
  double c[10], b[3];
  centred_cluster(in.agg + 10 * o, in.agg_form, c);
  const double* ref = sref + 12 * (int64_t)in.obs_scan[o];
  offset_b(c, ref, an, b);
  // eigen-decomposition of the scatter in the scan frame: an FP32 Jacobi
  // gives V0; W = V0^T S V0 is diagonal up to FP32 rounding, and its FP32
  // Jacobi gives the variances to FP32 relative precision (the normal one
  // included); V = V0 W_vec.  A direction error d of the stored vectors
  // changes a variance only by (spread) d^2.
  float sf[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) sf[q] = f64_to_f32(c[q]);
  float lam0[3], v0[9];
  eig3_sym_f(sf, lam0, v0);  // eigenvectors as rows of v0 (vector c at v0[3c..3c+2])
  // W = V0^T S V0.  The entries of the two smallest directions (W_00,
  // W_01, W_11) are small next to S's largest entries and lose digits to
  // cancellation in FP32, so they are formed in double-float arithmetic (~46
  // bits, from S's FP64 entries; the FP32 eigenvectors are exact): W_00 is the normal
  // variance of a planar cluster, and for a rod-like cluster (two small,
  // nearly equal variances) the voxel normal can be any direction of that
  // pair.  The entries with the largest direction only need absolute
  // precision (off-diagonals of order 1e-7 of the spread turn V0 by ~1e-7
  // rad, a second-order change of the variances).
  float wf[6];
  {
    // S as double-floats: hi the binary32 rounding of each entry, lo the
    // exact remainder rounded once (one FP64 subtraction per entry)
    DF Sd[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) Sd[q] = DF{sf[q], f64_to_f32(c[q] - f32_to_f64(sf[q]))};
    const DF S[3][3] = {{Sd[0], Sd[1], Sd[2]}, {Sd[1], Sd[3], Sd[4]}, {Sd[2], Sd[4], Sd[5]}};
    DF Sv[2][3];  // S v_k, k = 0, 1 (v_k binary32, exact)
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        DF acc{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 3; ++q) acc = df_fma(acc, v0[3 * k + q], S[r][q]);
        Sv[k][r] = acc;
      }
    auto dot = [&](int i, int k) {
      DF acc{0.f, 0.f};
#pragma unroll
      for (int r = 0; r < 3; ++r) acc = df_fma(acc, v0[3 * i + r], Sv[k][r]);
      return __fadd_rn(acc.hi, acc.lo);
    };
    wf[0] = dot(0, 0);
    wf[1] = dot(0, 1);
    wf[3] = dot(1, 1);
    const float M[3][3] = {{sf[0], sf[1], sf[2]}, {sf[1], sf[3], sf[4]}, {sf[2], sf[4], sf[5]}};
    float T[3];  // S v_2 (FP32)
    for (int r = 0; r < 3; ++r) T[r] = fmaf(M[r][0], v0[6], fmaf(M[r][1], v0[7], M[r][2] * v0[8]));
    // packed (00, 01, 02, 11, 12, 22)
    wf[2] = fmaf(v0[0], T[0], fmaf(v0[1], T[1], v0[2] * T[2]));
    wf[4] = fmaf(v0[3], T[0], fmaf(v0[4], T[1], v0[5] * T[2]));
    wf[5] = fmaf(v0[6], T[0], fmaf(v0[7], T[1], v0[8] * T[2]));
  }
  float sg[3], wv[9];
  eig3_sym_f(wf, sg, wv);
  // world-axis eigenvectors as columns: V = R_ref V0^T-rows ... = R_ref [v0 rows]^T W
  const float* Rf = sref32_of(sref, in.n_scans, in.obs_scan[o]);
  float V[9];
  for (int cc = 0; cc < 3; ++cc) {
    float u[3];  // scan-frame vector cc = sum_k v0_k W[k][cc]
    for (int r = 0; r < 3; ++r)
      u[r] = fmaf(v0[r], wv[3 * cc], fmaf(v0[3 + r], wv[3 * cc + 1], v0[6 + r] * wv[3 * cc + 2]));
    for (int r = 0; r < 3; ++r) V[3 * r + cc] = fmaf(Rf[3 * r], u[0], fmaf(Rf[3 * r + 1], u[1], Rf[3 * r + 2] * u[2]));
  }
  const float det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                    V[2] * (V[3] * V[7] - V[4] * V[6]);
  if (det < 0.f) {
    V[0] = -V[0];
    V[3] = -V[3];
    V[6] = -V[6];
  }
  float qf[4];
  mat_to_quat<float>(V, qf);
  s0 = make_float4(f64_to_f32(b[0]), f64_to_f32(b[1]), f64_to_f32(b[2]), f64_to_f32(c[9]));
  s1 = make_float4(sg[0], sg[1], sg[2], __int_as_float(in.obs_scan[o]));
  s2 = make_float4(qf[0], qf[1], qf[2], qf[3]);
}

// slots of the slices that start at sorted positions [p0, p1) (p0 a multiple
// of kSlice): thread (p, blockIdx.y) fills rows kFillRows * blockIdx.y ..
// + kFillRows - 1 of voxel p, then the same rows gridDim.y * kFillRows on
// (eight resident blocks of 128 per SM: 64 registers, measured faster than
// five blocks at the registers the compiler takes unbounded)
__global__ void __launch_bounds__(128, 8)
    fill_sell_mixed_kernel(LoadInput in, const int32_t* vperm, const int32_t* vlen, const int64_t* slice_off,
                           int64_t n_voxels, int64_t p0, int64_t p1, const double* sref, const float4* vanchor,
                           float4* ve32) {
  const int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = p >> 5;
  if (s * kSlice >= n_voxels || s * kSlice >= p1) return;
  const int lane = (int)(p & 31);
  const int64_t base = slice_off[s] + lane;
  const int64_t rows = (slice_off[s + 1] - slice_off[s]) / kSlice;
  const bool real = p < n_voxels;
  const int32_t len = real ? vlen[p] : 0;
  const int64_t o0 = real ? in.voxel_off[vperm[p]] : 0;
  const float4 an = real ? vanchor[p] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t k0 = (int64_t)blockIdx.y * kFillRows; k0 < rows; k0 += (int64_t)gridDim.y * kFillRows) {
    for (int64_t k = k0; k < k0 + kFillRows && k < rows; ++k) {
      const int64_t e = base + k * kSlice;
      float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
      if (k < len) mixed_slot(in, o0 + k, sref, an, s0, s1, s2);
      ve32[kVe32 * e] = s0;
      ve32[kVe32 * e + 1] = s1;
      ve32[kVe32 * e + 2] = s2;
    }
  }
}

// The same slots staged voxel by voxel in the sorted voxel order (slot of
// row k of the voxel at sorted position p at staging[3 (vstart[p] + k)]): a
// pipelined load computes each arriving chunk's slots there (each voxel's
// rows one contiguous run), then places them all in their slices once every
// chunk is done, each slice reading one contiguous stretch.
__global__ void fill_staging_kernel(LoadInput in, int64_t o0, int64_t o1, const int32_t* obs_vox,
                                    const int32_t* vrank, const int64_t* vstart, const double* sref,
                                    const float4* vanchor, float4* staging) {
  const int64_t o = o0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= o1) return;
  const int32_t v = obs_vox[o];
  const int64_t p = vrank[v];
  float4 s0, s1, s2;
  mixed_slot(in, o, sref, vanchor[p], s0, s1, s2);
  float4* dst = staging + 3 * (vstart[p] + (o - in.voxel_off[v]));
  dst[0] = s0;
  dst[1] = s1;
  dst[2] = s2;
}

// staged slots to their slices, padding rows zero; thread (p, blockIdx.y)
// as in fill_sell_mixed_kernel (coalesced writes)
__global__ void place_slots_kernel(const int64_t* vstart, const int32_t* vlen, const int64_t* slice_off,
                                   int64_t n_voxels, int64_t n_slices, const float4* staging, float4* ve32) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = p >> 5;
  if (s >= n_slices) return;
  const int64_t base = slice_off[s] + (p & 31);
  const int64_t rows = (slice_off[s + 1] - slice_off[s]) / kSlice;
  const bool real = p < n_voxels;
  const int32_t len = real ? vlen[p] : 0;
  const int64_t o0 = real ? vstart[p] : 0;
  for (int64_t k0 = (int64_t)blockIdx.y * kFillRows; k0 < rows; k0 += (int64_t)gridDim.y * kFillRows) {
    for (int64_t k = k0; k < k0 + kFillRows && k < rows; ++k) {
      const int64_t e = base + k * kSlice;
      float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
      if (k < len) {
        const float4* src = staging + 3 * (o0 + k);
        s0 = src[0];
        s1 = src[1];
        s2 = src[2];
      }
      ve32[kVe32 * e] = s0;
      ve32[kVe32 * e + 1] = s1;
      ve32[kVe32 * e + 2] = s2;
    }
  }
}

// Scan-major FP32 copy from the slots: the offset and count as they are, the
// scatter in reference axes rebuilt from its eigenvalues and eigenvector
// quaternion (R_ref S R_ref^T = V diag(sigma) V^T), each scaled by 2 / N_i.
// Observation o's slot is at sorted voxel position p, row k:
// slice_off[p / 32] + 32 k + p % 32, or, with staging non-null, at
// staging[3 (vstart[p] + k)].
__device__ __forceinline__ void fill_scan_one(int64_t q, int64_t o, int64_t n_obs, const int32_t* obs_vox,
                                              const double* vscale, const int32_t* vrank, const int64_t* voxel_off,
                                              const int64_t* slice_off, const float4* ve32, const int64_t* vstart,
                                              const float4* staging, float* se32) {
  const int32_t v = obs_vox[o];
  const int64_t p = vrank[v];
  const int64_t k = o - voxel_off[v];
  const float4* src =
      staging ? staging + 3 * (vstart[p] + k) : ve32 + kVe32 * (slice_off[p >> 5] + k * kSlice + (p & 31));
  const float4 s0 = src[0], s1 = src[1], s2 = src[2];
  float V[9];
  quat_to_mat_f(s2.x, s2.y, s2.z, s2.w, V);
  const float sg[3] = {s1.x, s1.y, s1.z};
  float sw[6];
  int idx = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c)
      sw[idx++] = fmaf(V[3 * r] * sg[0], V[3 * c], fmaf(V[3 * r + 1] * sg[1], V[3 * c + 1], V[3 * r + 2] * sg[2] * V[3 * c + 2]));
  const float ks = f64_to_f32(vscale[v]);
  float4* bN = reinterpret_cast<float4*>(se32);
  float4* S4 = bN + n_obs;
  float2* S2 = reinterpret_cast<float2*>(S4 + n_obs);
  bN[q] = make_float4(s0.x, s0.y, s0.z, ks * s0.w);
  S4[q] = make_float4(ks * sw[0], ks * sw[1], ks * sw[2], ks * sw[3]);
  S2[q] = make_float2(ks * sw[4], ks * sw[5]);
}

// thread per scan-major position q = qlist[i] (q = i without a list), i in
// [i0, i1); order[q] = its observation (a pipelined load fills each chunk's
// entries as the chunk is set up)
__global__ void fill_scan_mixed_kernel(int64_t n_obs, const uint32_t* qlist, int64_t i0, int64_t i1,
                                       const uint32_t* order, const int32_t* obs_vox, const double* vscale,
                                       const int32_t* vrank, const int64_t* voxel_off, const int64_t* slice_off,
                                       const float4* ve32, const int64_t* vstart, const float4* staging,
                                       float* se32) {
  const int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= i1) return;
  const int64_t q = qlist ? (int64_t)qlist[i] : i;
  fill_scan_one(q, order[q], n_obs, obs_vox, vscale, vrank, voxel_off, slice_off, ve32, vstart, staging, se32);
}

// blocks of 128 threads for kFrameLanes threads per voxel of n voxels
unsigned frame_blocks(int64_t n) { return (unsigned)((n * kFrameLanes + 127) / 128); }

}  // namespace

cudaError_t build_mixed_begin(const LoadInput& in, const double* poses2, MixedBuffers& mb, cudaStream_t stream,
                              int64_t* launches) {
  scan_ref_kernel<<<(in.n_scans + 127) / 128, 128, 0, stream>>>(in.n_scans, poses2, mb.sref);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t build_mixed_voxels(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                               int64_t v0, int64_t v1, int64_t o0, int64_t o1, float4* staging,
                               const uint32_t* chunk_q, cudaStream_t stream, int64_t* launches) {
  if (v1 <= v0) return cudaSuccess;
  LoadInput cur = in;
  cur.poses = poses2;  // buffer 0
  voxel_frames_kernel<<<frame_blocks(v1 - v0), 128, 0, stream>>>(cur, v0, v1, mb.sref, lb.vrank, mb.vstate,
                                                                 mb.vanchor, mb.planes32_2);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || o1 <= o0) return e;
  fill_staging_kernel<<<(unsigned)((o1 - o0 + 127) / 128), 128, 0, stream>>>(cur, o0, o1, lb.obs_vox, lb.vrank,
                                                                            lb.vstart, mb.sref, mb.vanchor, staging);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the chunk's scan-major entries (scattered over the whole copy)
  return build_mixed_scan_major(in, lb, mb, staging, chunk_q, o0, o1, stream, launches);
}

cudaError_t build_mixed_place(const LoadInput& in, const LayoutBuffers& lb, MixedBuffers& mb, const float4* staging,
                              cudaStream_t stream, int64_t* launches) {
  const int64_t n = lb.n_slices * kSlice;
  if (n == 0) return cudaSuccess;
  const unsigned row_blocks =
      (unsigned)std::min<int64_t>(std::max<int64_t>((lb.max_len + kFillRows - 1) / kFillRows, 1), 65535);
  place_slots_kernel<<<dim3((unsigned)((n + 127) / 128), row_blocks), 128, 0, stream>>>(
      lb.vstart, lb.vlen, lb.slice_off, in.n_voxels, lb.n_slices, staging, mb.ve32);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t build_mixed_scan_major(const LoadInput& in, const LayoutBuffers& lb, MixedBuffers& mb,
                                   const float4* staging, const uint32_t* qlist, int64_t i0, int64_t i1,
                                   cudaStream_t stream, int64_t* launches) {
  if (i1 <= i0) return cudaSuccess;
  fill_scan_mixed_kernel<<<(unsigned)((i1 - i0 + 255) / 256), 256, 0, stream>>>(
      in.n_obs, qlist, i0, i1, lb.scan_order, lb.obs_vox, lb.vscale, lb.vrank, in.voxel_off, lb.slice_off, mb.ve32,
      lb.vstart, staging, mb.se32);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t build_mixed_end(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                            cudaStream_t stream, int64_t* launches, bool scan_filled) {
  if (!scan_filled) {
    cudaError_t e = build_mixed_scan_major(in, lb, mb, nullptr, nullptr, 0, in.n_obs, stream, launches);
    if (e != cudaSuccess) return e;
  }
  ++*launches;
  return launch_scan_table(in.n_scans, poses2, mb.sref, mb.stab2, 0, stream);
}

cudaError_t build_mixed(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                        cudaStream_t stream, int64_t* launches) {
  cudaError_t e = build_mixed_begin(in, poses2, mb, stream, launches);
  if (e != cudaSuccess) return e;
  LoadInput cur = in;
  cur.poses = poses2;  // buffer 0
  const int64_t nv = in.n_voxels;
  if (nv > 0) {
    voxel_frames_kernel<<<frame_blocks(nv), 128, 0, stream>>>(cur, 0, nv, mb.sref, lb.vrank, mb.vstate, mb.vanchor,
                                                               mb.planes32_2);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // every slot, padding included, by sorted position (coalesced writes)
    const int64_t p1 = ((nv + kSlice - 1) / kSlice) * kSlice;
    const unsigned row_blocks =
        (unsigned)std::min<int64_t>(std::max<int64_t>((lb.max_len + kFillRows - 1) / kFillRows, 1), 65535);
    fill_sell_mixed_kernel<<<dim3((unsigned)((p1 + 127) / 128), row_blocks), 128, 0, stream>>>(
        cur, lb.vperm, lb.vlen, lb.slice_off, nv, 0, p1, mb.sref, mb.vanchor, mb.ve32);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return build_mixed_end(in, lb, poses2, mb, stream, launches);
}

}  // namespace mmba
