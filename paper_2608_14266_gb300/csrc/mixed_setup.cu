// Set-up of the mixed-precision copies (once per load and at ba_set_state):
// per-scan reference poses, per-voxel anchors and starting frames at those
// poses, and the FP32 re-centred clusters in the slice layout (offset to the
// anchor plus each observation's scatter as eigenvalues and the quaternion of
// its eigenvectors) and in the scan-major layout (reference axes, scaled by
// 2 / N_i).  All arithmetic here is FP64; only the stored results are rounded
// to FP32.
#include "mmba_internal.cuh"
#include "mmba_kernels.h"

namespace mmba {

namespace {

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

// R S R^T (S packed xx xy xz yy yz zz), packed result
__device__ inline void rot_sym(const double* R, const double* S, double* out) {
  const double M[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  double T[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) T[r][c] = R[3 * r] * M[0][c] + R[3 * r + 1] * M[1][c] + R[3 * r + 2] * M[2][c];
  int idx = 0;
  for (int r = 0; r < 3; ++r)
    for (int c = r; c < 3; ++c) out[idx++] = T[r][0] * R[3 * c] + T[r][1] * R[3 * c + 1] + T[r][2] * R[3 * c + 2];
}

__device__ inline double det3(const double* M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// reference pose of each scan: R_ref = R, t_ref = t rounded to FP32
__global__ void scan_ref_kernel(int32_t n_scans, const double* poses, double* sref) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_scans) return;
  const double* P = poses + 12 * (int64_t)j;
  double* o = sref + 12 * (int64_t)j;
  for (int k = 0; k < 9; ++k) o[k] = P[k];
  for (int k = 9; k < 12; ++k) o[k] = (double)(float)P[k];
}

// anchor (FP32-rounded centroid) and starting frame (eigenvectors, normal
// last, proper rotation) of each voxel at the reference poses
__global__ void voxel_frames_kernel(LoadInput in, const double* sref, const int32_t* vrank, float4* vstate,
                                    float4* vanchor, float4* planes2) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= in.n_voxels) return;
  const int64_t a0 = in.voxel_off[v], a1 = in.voxel_off[v + 1];
  double n = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
  for (int64_t o = a0; o < a1; ++o) {
    double c[10];
    centred_cluster(in.agg + 10 * o, in.agg_form, c);
    const double* R = sref + 12 * (int64_t)in.obs_scan[o];
    const double* P = in.poses + 12 * (int64_t)in.obs_scan[o];
    cx += c[9] * (R[0] * c[6] + R[1] * c[7] + R[2] * c[8] + P[9]);
    cy += c[9] * (R[3] * c[6] + R[4] * c[7] + R[5] * c[8] + P[10]);
    cz += c[9] * (R[6] * c[6] + R[7] * c[7] + R[8] * c[8] + P[11]);
    n += c[9];
  }
  cx /= n;
  cy /= n;
  cz /= n;
  double A[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t o = a0; o < a1; ++o) {
    double c[10], rs[6];
    centred_cluster(in.agg + 10 * o, in.agg_form, c);
    const double* R = sref + 12 * (int64_t)in.obs_scan[o];
    const double* P = in.poses + 12 * (int64_t)in.obs_scan[o];
    const double dx = R[0] * c[6] + R[1] * c[7] + R[2] * c[8] + P[9] - cx;
    const double dy = R[3] * c[6] + R[4] * c[7] + R[5] * c[8] + P[10] - cy;
    const double dz = R[6] * c[6] + R[7] * c[7] + R[8] * c[8] + P[11] - cz;
    rot_sym(R, c, rs);
    A[0] += rs[0] + c[9] * dx * dx;
    A[1] += rs[1] + c[9] * dx * dy;
    A[2] += rs[2] + c[9] * dx * dz;
    A[3] += rs[3] + c[9] * dy * dy;
    A[4] += rs[4] + c[9] * dy * dz;
    A[5] += rs[5] + c[9] * dz * dz;
  }
  double lam[3], V[9];
  eig3_sym(A, lam, V);
  // rows: e1 (largest), e2, n (smallest)
  double U[9] = {V[6], V[7], V[8], V[3], V[4], V[5], V[0], V[1], V[2]};
  if (det3(U) < 0.0)
    for (int k = 0; k < 3; ++k) U[k] = -U[k];
  double q[4];
  mat_to_quat<double>(U, q);
  const int64_t p = vrank[v];
  const float ax = (float)cx, ay = (float)cy, az = (float)cz;
  vanchor[p] = make_float4(ax, ay, az, 0.0f);
  // the anchor also sits beside the plane in both buffers of plane records
  planes2[2 * p + 1] = make_float4(ax, ay, az, 0.0f);
  planes2[2 * (in.n_voxels + p) + 1] = make_float4(ax, ay, az, 0.0f);
  vstate[2 * p] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
  // the running centroid starts where the anchor's rounding left it
  vstate[2 * p + 1] = make_float4((float)(cx - (double)ax), (float)(cy - (double)ay), (float)(cz - (double)az), 0.0f);
}

// b = R_ref m + t_ref - a (world axes), for an observation of a voxel whose
// anchor is an
__device__ inline void offset_b(const double* c, const double* ref, float4 an, double b[3]) {
  b[0] = ref[0] * c[6] + ref[1] * c[7] + ref[2] * c[8] + (ref[9] - (double)an.x);
  b[1] = ref[3] * c[6] + ref[4] * c[7] + ref[5] * c[8] + (ref[10] - (double)an.y);
  b[2] = ref[6] * c[6] + ref[7] * c[7] + ref[8] * c[8] + (ref[11] - (double)an.z);
}

__global__ void fill_sell_mixed_kernel(LoadInput in, const int32_t* vperm, const int32_t* vlen,
                                       const int64_t* slice_off, int64_t n_voxels, const double* sref,
                                       const float4* vanchor, float4* ve32) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = p >> 5;
  if (s * kSlice >= n_voxels) return;
  const int lane = (int)(p & 31);
  const int64_t base = slice_off[s] + lane;
  const int64_t rows = (slice_off[s + 1] - slice_off[s]) / kSlice;
  const bool real = p < n_voxels;
  const int32_t len = real ? vlen[p] : 0;
  const int64_t o0 = real ? in.voxel_off[vperm[p]] : 0;
  const float4 an = real ? vanchor[p] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t k = 0; k < rows; ++k) {
    const int64_t e = base + k * kSlice;
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
    if (k < len) {
      const int64_t o = o0 + k;
      double c[10], b[3], sw[6], lam[3], vec[9];
      centred_cluster(in.agg + 10 * o, in.agg_form, c);
      const double* ref = sref + 12 * (int64_t)in.obs_scan[o];
      offset_b(c, ref, an, b);
      rot_sym(ref, c, sw);
      // eigenvectors: an FP32 Jacobi gives V0, the FP64 Jacobi then finishes on
      // V0^T S V0, which is diagonal up to FP32 rounding (one or two sweeps
      // instead of the four to six a full FP64 solve takes; FP64 is 1/64 rate)
      float swf[6] = {(float)sw[0], (float)sw[1], (float)sw[2], (float)sw[3], (float)sw[4], (float)sw[5]};
      float lamf[3], vecf[9];
      eig3_sym_f(swf, lamf, vecf);
      double V0[9];  // row-major, eigenvectors as columns
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) V0[3 * r + cc] = (double)vecf[3 * cc + r];
      double V0t[9];
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) V0t[3 * r + cc] = V0[3 * cc + r];
      double sp[6];
      rot_sym(V0t, sw, sp);  // V0^T S V0
      eig3_sym(sp, lam, vec);
      // V = V0 W (W: eigenvectors of V0^T S V0 as columns), made a proper rotation
      double V[9];
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc)
          V[3 * r + cc] = V0[3 * r] * vec[3 * cc] + V0[3 * r + 1] * vec[3 * cc + 1] + V0[3 * r + 2] * vec[3 * cc + 2];
      if (det3(V) < 0.0) {
        V[0] = -V[0];
        V[3] = -V[3];
        V[6] = -V[6];
      }
      double q[4];
      mat_to_quat<double>(V, q);
      const float qf[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
      // sigma as Rayleigh quotients along the columns of the rotation the
      // kernel will rebuild from the FP32 quaternion, so that the stored
      // normal variance belongs to exactly that direction
      const double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
      const double nq = 1.0 / (w * w + x * x + y * y + z * z);
      const double Vf[9] = {1 - 2 * (y * y + z * z) * nq, 2 * (x * y - w * z) * nq, 2 * (x * z + w * y) * nq,
                            2 * (x * y + w * z) * nq, 1 - 2 * (x * x + z * z) * nq, 2 * (y * z - w * x) * nq,
                            2 * (x * z - w * y) * nq, 2 * (y * z + w * x) * nq, 1 - 2 * (x * x + y * y) * nq};
      const double M[3][3] = {{sw[0], sw[1], sw[2]}, {sw[1], sw[3], sw[4]}, {sw[2], sw[4], sw[5]}};
      float sg[3];
      for (int cc = 0; cc < 3; ++cc) {
        double acc = 0.0;
        for (int r = 0; r < 3; ++r)
          for (int t = 0; t < 3; ++t) acc += Vf[3 * r + cc] * M[r][t] * Vf[3 * t + cc];
        sg[cc] = (float)acc;
      }
      s0 = make_float4((float)b[0], (float)b[1], (float)b[2], (float)c[9]);
      s1 = make_float4(sg[0], sg[1], sg[2], __int_as_float(in.obs_scan[o]));
      s2 = make_float4(qf[0], qf[1], qf[2], qf[3]);
    }
    ve32[kVe32 * e] = s0;
    ve32[kVe32 * e + 1] = s1;
    ve32[kVe32 * e + 2] = s2;
  }
}

__global__ void fill_scan_mixed_kernel(LoadInput in, const uint32_t* order, const int32_t* obs_vox,
                                       const double* vscale, const int32_t* vrank, const double* sref,
                                       const float4* vanchor, float* se32) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= in.n_obs) return;
  const int64_t o = order[q];
  const int32_t v = obs_vox[o];
  const float4 an = vanchor[vrank[v]];
  double c[10], b[3], sw[6];
  centred_cluster(in.agg + 10 * o, in.agg_form, c);
  const double* ref = sref + 12 * (int64_t)in.obs_scan[o];
  offset_b(c, ref, an, b);
  rot_sym(ref, c, sw);
  const double k = vscale[v];
  const int64_t n = in.n_obs;
  for (int a = 0; a < 3; ++a) se32[a * n + q] = (float)b[a];
  for (int a = 0; a < 6; ++a) se32[(3 + a) * n + q] = (float)(k * sw[a]);
  se32[9 * n + q] = (float)(k * c[9]);
}

}  // namespace

cudaError_t build_mixed(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                        cudaStream_t stream, int64_t* launches) {
  const int64_t nv = in.n_voxels, no = in.n_obs;
  LoadInput cur = in;
  cur.poses = poses2;  // buffer 0
  scan_ref_kernel<<<(in.n_scans + 127) / 128, 128, 0, stream>>>(in.n_scans, poses2, mb.sref);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  voxel_frames_kernel<<<(unsigned)((nv + 127) / 128), 128, 0, stream>>>(cur, mb.sref, lb.vrank, mb.vstate,
                                                                        mb.vanchor, mb.planes32_2);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fill_sell_mixed_kernel<<<(unsigned)((lb.n_slices * kSlice + 127) / 128), 128, 0, stream>>>(
      cur, lb.vperm, lb.vlen, lb.slice_off, nv, mb.sref, mb.vanchor, mb.ve32);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fill_scan_mixed_kernel<<<(unsigned)((no + 255) / 256), 256, 0, stream>>>(cur, lb.scan_order, lb.obs_vox, lb.vscale,
                                                                           lb.vrank, mb.sref, mb.vanchor, mb.se32);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ++*launches;
  return launch_scan_table(in.n_scans, poses2, mb.sref, mb.stab2, 0, stream);
}

}  // namespace mmba
