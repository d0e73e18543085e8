// Internal definitions shared by the library's CUDA translation units.
//
// Device layout of a loaded problem (all in the handle's device memory):
//
//  * Voxel-sorted slices (SELL-32): voxels are sorted by observation count
//    (descending) inside windows of kWindow consecutive input voxels, and
//    grouped 32 to a slice; one thread owns one voxel.  Row k of slice s holds
//    the k-th observation of each of its 32 voxels at
//    slice_off[s] + 32 * k + lane, so a warp reading row k touches 32
//    consecutive elements.  Rows past a voxel's own length are padding
//    (never read: vlen bounds the loop).  Cluster values are stored as
//    structure-of-arrays, component c of element e at ve[c * n_elems + e]:
//    S (xx, xy, xz, yy, yz, zz), m (x, y, z), N.
//  * Scan-major copy (the M_s mapper of Algorithm 1): observations sorted
//    (stably) by scan, scan j owning scan_off[j] .. scan_off[j+1]-1, with
//    the sorted voxel position of each (se_vox, the M_v mapper) and the
//    cluster scaled by 2 / N_i (S and N scaled, m unchanged), which is the
//    factor every derivative term of voxel i carries.
//  * Two pose buffers and two plane buffers (current / trial), selected by
//    DevState::cur on the device, so that accept/reject never needs the host.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mmba {

constexpr int kSlice = 32;          // voxels per slice (one warp)
constexpr int64_t kWindow = 8192;   // length sort window (multiple of kSlice)
constexpr int kPlaneStride = 4;     // plane record used by the scan pass: u (3), d
constexpr int kGH = 27;             // per-scan g (6) then upper triangle of H (21)

struct DevLayout {
  int32_t n_scans;
  int32_t fixed_scan;
  int64_t n_voxels;
  int64_t n_obs;
  int64_t n_elems;
  int64_t n_slices;
  const int64_t* slice_off;  // n_slices + 1
  const int32_t* vlen;       // n_voxels (sorted position)
  const int32_t* vperm;      // sorted position -> input voxel
  const double* ve;          // 10 x n_elems
  const int32_t* ve_scan;    // n_elems
  const int64_t* scan_off;   // n_scans + 1
  const double* se;          // 10 x n_obs
  const int32_t* se_vox;     // n_obs
};

struct DevState {
  double cost;
  double mu;
  double nu;
  double last_rho;
  double last_pred;
  double last_trial_cost;
  double rel_tol;
  double abs_tol;
  int32_t cur;
  int32_t iters;
  int32_t accepted;
  int32_t consec_reject;
  int32_t last_accepted;
  int32_t converged;
  int32_t solve_failed;
  int32_t solve_fail_flag;  // set by the solve kernel, consumed by the decision
  int32_t stop;             // solve loop finished (only honoured when honor_stop)
  int32_t honor_stop;
  int32_t max_iters;
  int32_t max_consec_reject;
  int32_t hess_mode;
  int32_t scan_pending;     // an accepted step needs g, H at the new poses
};

// ---- small FP64 device math ------------------------------------------------

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, Matrix Computations, Sec. 8.5).  a = (xx, xy, xz, yy, yz, zz) is
// overwritten; on return lam[] ascending and vec[3*c + r] = component r of the
// unit eigenvector of lam[c].  Stops when every off-diagonal entry is below
// 1e-18 of the geometric mean of its diagonal pair, or after 24 sweeps.
__device__ __forceinline__ void jacobi_rotate(double& app, double& aqq, double& apq, double& arp, double& arq,
                                              double* vp, double* vq) {
  double theta = (aqq - app) / (2.0 * apq);
  double t = fabs(theta) > 1e150 ? 0.5 / theta
                                 : copysign(1.0, theta) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
  double c = rsqrt(fma(t, t, 1.0));
  double s = t * c;
  app = fma(-t, apq, app);
  aqq = fma(t, apq, aqq);
  apq = 0.0;
  double rp = arp, rq = arq;
  arp = c * rp - s * rq;
  arq = s * rp + c * rq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double x = vp[k], y = vq[k];
    vp[k] = c * x - s * y;
    vq[k] = s * x + c * y;
  }
}

__device__ __forceinline__ bool jacobi_small(double apq, double app, double aqq) {
  return apq == 0.0 || fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq));
}

__device__ inline void eig3_sym(const double* a_in, double lam[3], double vec[9]) {
  double a00 = a_in[0], a01 = a_in[1], a02 = a_in[2], a11 = a_in[3], a12 = a_in[4], a22 = a_in[5];
  double v0[3] = {1.0, 0.0, 0.0}, v1[3] = {0.0, 1.0, 0.0}, v2[3] = {0.0, 0.0, 1.0};
  for (int sweep = 0; sweep < 24; ++sweep) {
    bool done = true;
    if (!jacobi_small(a01, a00, a11)) {  // (p, q, r) = (0, 1, 2)
      jacobi_rotate(a00, a11, a01, a02, a12, v0, v1);
      done = false;
    }
    if (!jacobi_small(a02, a00, a22)) {  // (0, 2, 1)
      jacobi_rotate(a00, a22, a02, a01, a12, v0, v2);
      done = false;
    }
    if (!jacobi_small(a12, a11, a22)) {  // (1, 2, 0)
      jacobi_rotate(a11, a22, a12, a01, a02, v1, v2);
      done = false;
    }
    if (done) break;
  }
  // sort ascending (stable on ties)
  double d[3] = {a00, a11, a22};
  int i0 = 0, i1 = 1, i2 = 2, t;
  if (d[i1] < d[i0]) { t = i0; i0 = i1; i1 = t; }
  if (d[i2] < d[i1]) { t = i1; i1 = i2; i2 = t; }
  if (d[i1] < d[i0]) { t = i0; i0 = i1; i1 = t; }
  const double* vs[3] = {v0, v1, v2};
  int order[3] = {i0, i1, i2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    lam[c] = d[order[c]];
#pragma unroll
    for (int r = 0; r < 3; ++r) vec[3 * c + r] = vs[order[c]][r];
  }
}

// LDL^T of the symmetric 6x6 A (full, row-major) without pivoting, then
// solve A x = b.  Returns false if a pivot is not positive and finite.
__device__ inline bool ldlt6_solve(const double* A, const double* b, double* x) {
  double L[6][6], D[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double dj = A[6 * j + j];
#pragma unroll
    for (int k = 0; k < j; ++k) dj -= L[j][k] * L[j][k] * D[k];
    if (!(dj > 0.0) || !isfinite(dj)) return false;
    D[j] = dj;
    double inv = 1.0 / dj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      double v = A[6 * i + j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k] * D[k];
      L[i][j] = v * inv;
    }
  }
  double y[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double v = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] /= D[i];
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    double v = y[i];
#pragma unroll
    for (int k = i + 1; k < 6; ++k) v -= L[k][i] * x[k];
    x[i] = v;
  }
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 6; ++i) ok = ok && isfinite(x[i]);
  return ok;
}

// Exp map of so(3) (Rodrigues' formula), R row-major.  Below |phi| = 1e-6 the
// second-order series I + [phi]x + [phi]x^2 / 2 is used; otherwise
// R = I + (sin th / th) K + (2 sin^2(th/2) / th^2) K^2.
__device__ inline void so3_exp(const double* phi, double* R) {
  double x = phi[0], y = phi[1], z = phi[2];
  double th2 = x * x + y * y + z * z;
  double th = sqrt(th2);
  double a, b;
  if (th < 1e-6) {
    a = 1.0;
    b = 0.5;
  } else {
    double sh = sin(0.5 * th);
    a = sin(th) / th;
    b = 2.0 * sh * sh / th2;
  }
  // K^2 = phi phi^T - th2 I
  R[0] = 1.0 + b * (x * x - th2);
  R[1] = -a * z + b * x * y;
  R[2] = a * y + b * x * z;
  R[3] = a * z + b * x * y;
  R[4] = 1.0 + b * (y * y - th2);
  R[5] = -a * x + b * y * z;
  R[6] = -a * y + b * x * z;
  R[7] = a * x + b * y * z;
  R[8] = 1.0 + b * (z * z - th2);
}

// Deterministic block-wide sum (fixed shape for a given blockDim).
template <int kThreads>
__device__ inline double block_sum(double v, double* smem /* kThreads / 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) smem[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) r += smem[k];
  }
  __syncthreads();
  return r;  // valid in thread 0
}

}  // namespace mmba
