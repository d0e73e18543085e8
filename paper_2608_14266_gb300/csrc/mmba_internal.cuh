// Internal definitions shared by the library's CUDA translation units.
//
// Device layout of a loaded problem (all in the handle's device memory):
//
//  * Voxel-sorted slices (SELL-32): voxels are put in a spatial order (the
//    Morton code of the mean position of the scans observing each voxel, at
//    the input poses), cut into windows of kWindow voxels consecutive in that
//    order, sorted by observation count (descending) inside each window, and
//    grouped 32 to a slice; one thread owns one voxel.  Voxels seen by the
//    same scans share slices, so a slice row reads few distinct per-scan
//    entries, and a scan's observations gather plane records that lie close.  Row k of slice s holds
//    the k-th observation of each of its 32 voxels at
//    slice_off[s] + 32 * k + lane, so a warp reading row k touches 32
//    consecutive elements.  Rows past a voxel's own length are padding
//    (never read: vlen bounds the loop).  Cluster values are stored as
//    structure-of-arrays, component c of element e at ve[c * n_elems + e]:
//    the pivoted LDL^T of S (l10, l20, l21, D0, D1, D2), the permuted mean
//    P m (3), N; the permutation's code sits in the top bits of ve_scan.
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
constexpr int64_t kWindow = 8192;   // length sort window, in spatial order (multiple of kSlice)
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
  // scans by decreasing observation count: scan-pass block b works on scan
  // scan_order[b], so the longest scans start first and the tail is short
  // (NULL = block b, scan b)
  const int32_t* scan_order;
};

__device__ __forceinline__ int scan_of_block(const DevLayout& L, int64_t b) {
  return L.scan_order ? L.scan_order[b] : (int)b;
}

// Mixed-precision copies (FP32 per observation, re-centred).  For every
// voxel i an anchor a_i (the FP32-representable rounding of its centroid at
// the reference poses) and an orthonormal frame B_i (rows e1, e2, n: the
// eigenvectors of its covariance there, normal last); for every scan j a
// reference pose (R_ref,j, t_ref,j) with t_ref FP32-representable.  With
// dR_j = R_j R_ref,j^T = I + E_j and dt_j = t_j - t_ref,j, an observation's
// posed mean relative to its anchor is
//   q_o - a_i = b_o + E_j l_o + dt_j,   l_o = b_o + (a_i - t_ref,j),
// where b_o = R_ref m_o + t_ref - a_i is stored; every quantity is
// plane-sized except the lever l_o, which only meets the small E_j.  E_j is
// carried as a rotation vector phi and the coefficients of
// E = a [phi]x + b [phi]x^2 (Rodrigues).
//
// The voxel pass stores each observation's scatter through its own
// eigen-decomposition R_ref S R_ref^T = V diag(sigma) V^T (sigma and the
// quaternion of V): one scan's view of a patch is planar, so its normal
// variance sigma_3 keeps full FP32 relative precision.  The sums run in a
// per-voxel frame B that follows the voxel's latest eigenvectors, so the
// normal direction of the sums stays small; G = B dR V is the only rotation
// applied per observation.
struct DevMixed {
  // SELL slots, 3 float4 each (48 B, one slot after another):
  //   (b0, b1, b2, N), (sigma0, sigma1, sigma2, scan index as int bits), quaternion of V (w, x, y, z)
  const float4* ve32;
  float4* vstate;        // per sorted voxel, 2 x float4: quaternion of B; (centroid - anchor) world (3), 0
  // scan-major, three vector arrays one after another (k = 2/N_i):
  //   float4 (b (3), k N) x n_obs | float4 k S (xx, xy, xz, yy) x n_obs | float2 k S (yz, zz) x n_obs
  // with S = R_ref S_o R_ref^T
  const float* se32;
  const float4* vanchor; // per sorted voxel: a (3), 0
  const double* sref;    // per scan: R_ref (9), t_ref (3)
  float* stab2;          // 2 buffers x n_scans x kTab: q of dR (w, v), dt (3), t_ref (3), 0, 0
  float4* planes32_2;    // 2 buffers x n_voxels x 2 float4: (u (3), u . (c - a)), (a (3), 0)
};
constexpr int kTab = 12;
constexpr int kScanChunk = 64;        // observations per staged chunk of the mixed scan pass
constexpr int kWaitLimit = 1 << 22;   // polls of an mbarrier before a wait gives up
constexpr int kVe32 = 3;  // float4 per slot of the voxel-pass copy

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_mat_f(float w, float x, float y, float z, float* R) {
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
              wz = w * z;
  R[0] = 1.f - 2.f * (yy + zz);
  R[1] = 2.f * (xy - wz);
  R[2] = 2.f * (xz + wy);
  R[3] = 2.f * (xy + wz);
  R[4] = 1.f - 2.f * (xx + zz);
  R[5] = 2.f * (yz - wx);
  R[6] = 2.f * (xz - wy);
  R[7] = 2.f * (yz + wx);
  R[8] = 1.f - 2.f * (xx + yy);
}

// ---- conversions between binary64 and binary32 in integer arithmetic ----
// GB300 runs FP64 <-> FP32 conversions on its narrow FP64 pipe; set-up code
// that converts tens of values per observation uses these instead.  Both
// follow IEEE 754: binary64 -> binary32 rounds to nearest, ties to even;
// binary32 -> binary64 is exact.  Values outside the normal ranges (zero,
// subnormal, overflow, infinity, NaN) take the hardware conversion.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32);
  const int ef = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;  // binary32 biased exponent
  if (ef <= 0 || ef >= 255) return (float)x;
  const unsigned int mf = (unsigned int)((b >> 29) & 0x7fffffu);  // top 23 of 52 fraction bits
  const unsigned int rest = (unsigned int)(b & 0x1fffffffu);     // the 29 bits dropped
  unsigned int r = ((unsigned int)ef << 23) | mf;
  // nearest, ties to even; a carry out of the fraction moves to the next binade
  // (and to infinity past the largest finite value), as rounding requires
  if (rest > 0x10000000u || (rest == 0x10000000u && (mf & 1u))) r += 1u;
  return __uint_as_float(r | (hi & 0x80000000u));
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)f;
  const unsigned long long r = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e - 127u + 1023u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)r);
}

// Unit quaternion (w, x, y, z) of a rotation matrix (row-major), from the
// largest of 1 + tr, 1 + 2 R_kk - tr (Shepperd's method, J. Guidance and
// Control 1, 1978), normalised.
template <typename T>
__device__ __forceinline__ void mat_to_quat(const T* R, T q[4]) {
  const T tr = R[0] + R[4] + R[8];
  T w, x, y, z;
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    const T s = sqrt(T(1) + tr) * T(2);
    w = T(0.25) * s;
    x = (R[7] - R[5]) / s;
    y = (R[2] - R[6]) / s;
    z = (R[3] - R[1]) / s;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const T s = sqrt(T(1) + R[0] - R[4] - R[8]) * T(2);
    w = (R[7] - R[5]) / s;
    x = T(0.25) * s;
    y = (R[1] + R[3]) / s;
    z = (R[2] + R[6]) / s;
  } else if (R[4] >= R[8]) {
    const T s = sqrt(T(1) + R[4] - R[0] - R[8]) * T(2);
    w = (R[2] - R[6]) / s;
    x = (R[1] + R[3]) / s;
    y = T(0.25) * s;
    z = (R[5] + R[7]) / s;
  } else {
    const T s = sqrt(T(1) + R[8] - R[0] - R[4]) * T(2);
    w = (R[3] - R[1]) / s;
    x = (R[2] + R[6]) / s;
    y = (R[5] + R[7]) / s;
    z = T(0.25) * s;
  }
  const T inv = T(1) / sqrt(w * w + x * x + y * y + z * z);
  q[0] = w * inv;
  q[1] = x * inv;
  q[2] = y * inv;
  q[3] = z * inv;
}

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
  int32_t wait_timeout;     // a bounded device-side wait gave up (sticky)
  uint32_t blocks_done;     // voxel-pass blocks finished in the current launch (decision in the last)
  int32_t shard;            // g, H and cost are totals over several handles' voxels (voxel-sharded solve)
  int32_t pad_;
};

// One job of a batch: everything its kernels touch.  A batch launches each
// kernel kind once per iteration over all its jobs; block b of a launch
// belongs to the job whose prefix range holds b, and runs exactly the block
// that the job's own launch would run, so a job's results do not depend on
// the batch it is in.
struct JobView {
  DevLayout L;
  DevMixed X;
  DevState* st;
  double* poses2;
  double* planes2;
  double* gH;
  double* pred_part;
  double* cost_part;
  int64_t n_cost;
};

struct JobTable {
  const JobView* jobs;
  const int64_t* vblk;   // n_jobs + 1: prefix of voxel-pass blocks
  const int64_t* sblk;   // n_jobs + 1: prefix of scan-pass blocks (one per scan)
  const int64_t* oblk;   // n_jobs + 1: prefix of solve blocks
  int32_t n_jobs;
};

// The iteration kernels of a batch take their jobs by value, as a kernel
// parameter: a group of up to kGroupJobs job views with block prefixes
// relative to the group.  The views then sit in the constant bank like the
// arguments of a single job's launch, so the per-job bases the observation
// loops use cost no registers (read from a table in global memory they are
// held in registers across the loops, and the passes spill).  A batch of more
// jobs launches one group per kernel kind and group, each group's chain of
// launches on its own branch of the captured graph.
constexpr int kGroupJobs = 128;
struct JobGroup {
  JobView jobs[kGroupJobs];
  int32_t vblk[kGroupJobs + 1];  // prefix of voxel-pass blocks
  int32_t sblk[kGroupJobs + 1];  // prefix of scan-pass blocks (one per scan)
  int32_t oblk[kGroupJobs + 1];  // prefix of solve blocks
  int32_t n_jobs;
};
static_assert(sizeof(JobGroup) <= 32000, "a job group must fit the kernel parameter space");

// job owning block b: the largest i with prefix[i] <= b
template <typename P>
__device__ __forceinline__ int find_job(const P* prefix, int n_jobs, int64_t b) {
  int lo = 0, hi = n_jobs;  // prefix[lo] <= b < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// ---- small FP64 device math ------------------------------------------------

// Cyclic Jacobi for symmetric 3x3 matrices (Golub & Van Loan, Matrix
// Computations, Sec. 8.5).
//
// One rotation in the (p, q) plane sets apq to zero and rotates the third
// row/column entries (arp, arq) and the eigenvector estimates vp, vq with it.
// The tangent of the rotation angle is t = 2e / (1 + sqrt(1 + 4e^2)) with
// e = apq / (aqq - app).  For |e| < 1e-4 (the usual case once the matrix is
// nearly diagonal) t is taken from its series e - e^3 + 2e^5 - ... (the
// Catalan numbers) cut after e^3, relative error below 2e^4 < 2e-16, and
// c = 1 / sqrt(1 + t^2) from 1 - t^2/2 + 3t^4/8 (error below 5t^6/16, so
// c^2 + s^2 = 1 to rounding): one division and no square root.
__device__ __forceinline__ void jacobi_rotate(double& app, double& aqq, double& apq, double& arp, double& arq,
                                              double* vp, double* vq) {
  const double d = aqq - app;
  double t, c;
  if (fabs(apq) < 1e-4 * fabs(d)) {
    const double e = apq / d;
    t = fma(-e * e, e, e);
    const double t2 = t * t;
    c = fma(t2, fma(0.375, t2, -0.5), 1.0);
  } else {
    const double theta = d / (2.0 * apq);
    t = fabs(theta) > 1e150 ? 0.5 / theta : copysign(1.0, theta) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
    c = rsqrt(fma(t, t, 1.0));
  }
  const double s = t * c;
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

// apq is negligible against its diagonal pair: |apq| <= u sqrt(|app aqq|)
// with u = 2^-53, compared in squares (eig3_sym scales its matrix so that the
// largest entry lies in [1, 2), so the squares neither overflow nor lose the
// entries that matter)
__device__ __forceinline__ bool jacobi_small(double apq, double app, double aqq) {
  return apq == 0.0 || apq * apq <= 0x1p-106 * fabs(app * aqq);
}

// FP32 counterpart of eig3_sym for matrices expressed in a frame where they
// are close to diagonal (small off-diagonal entries keep the smallest
// eigenvalue relatively accurate); at most 8 sweeps.  The rotation takes the
// small-angle form of jacobi_rotate when |apq| < 0.01 |aqq - app| (then
// t = e - e^3 is within 2e^4 < 2e-8 of the exact tangent and
// c = 1 - t^2/2 + 3t^4/8 within 5t^6/16 < 1e-12 of 1 / sqrt(1 + t^2): an
// orthogonal rotation to binary32 rounding, from one approximate division);
// the stopping test compares squares.
__device__ __forceinline__ void jacobi_rotate_f(float& app, float& aqq, float& apq, float& arp, float& arq, float* vp,
                                                float* vq) {
  const float d = aqq - app;
  float t, c;
  if (fabsf(apq) < 1e-2f * fabsf(d)) {
    const float e = __fdividef(apq, d);
    t = fmaf(-e * e, e, e);
    const float t2 = t * t;
    c = fmaf(t2, fmaf(0.375f, t2, -0.5f), 1.0f);
  } else {
    const float theta = d / (2.0f * apq);
    t = fabsf(theta) > 1e18f ? 0.5f / theta : copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
    c = rsqrtf(fmaf(t, t, 1.0f));
  }
  const float s = t * c;
  app = fmaf(-t, apq, app);
  aqq = fmaf(t, apq, aqq);
  apq = 0.0f;
  float rp = arp, rq = arq;
  arp = c * rp - s * rq;
  arq = s * rp + c * rq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float x = vp[k], y = vq[k];
    vp[k] = c * x - s * y;
    vq[k] = s * x + c * y;
  }
}

// |apq| <= 1e-9 sqrt|app aqq|, in squares
__device__ __forceinline__ bool jacobi_small_f(float apq, float app, float aqq) {
  return apq == 0.0f || apq * apq <= 1e-18f * fabsf(app * aqq);
}

__device__ inline void eig3_sym_f(const float* a_in, float lam[3], float vec[9]) {
  float a00 = a_in[0], a01 = a_in[1], a02 = a_in[2], a11 = a_in[3], a12 = a_in[4], a22 = a_in[5];
  float v0[3] = {1.f, 0.f, 0.f}, v1[3] = {0.f, 1.f, 0.f}, v2[3] = {0.f, 0.f, 1.f};
  for (int sweep = 0; sweep < 8; ++sweep) {
    bool done = true;
    if (!jacobi_small_f(a01, a00, a11)) {
      jacobi_rotate_f(a00, a11, a01, a02, a12, v0, v1);
      done = false;
    }
    if (!jacobi_small_f(a02, a00, a22)) {
      jacobi_rotate_f(a00, a22, a02, a01, a12, v0, v2);
      done = false;
    }
    if (!jacobi_small_f(a12, a11, a22)) {
      jacobi_rotate_f(a11, a22, a12, a01, a02, v1, v2);
      done = false;
    }
    if (done) break;
  }
  // ascending, stable on ties; swaps of values keep everything in registers
  float d0 = a00, d1 = a11, d2 = a22;
  auto cswap = [](float& da, float& db, float* va, float* vb) {
    if (db < da) {
      const float t = da;
      da = db;
      db = t;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float u = va[r];
        va[r] = vb[r];
        vb[r] = u;
      }
    }
  };
  cswap(d0, d1, v0, v1);
  cswap(d1, d2, v1, v2);
  cswap(d0, d1, v0, v1);
  lam[0] = d0;
  lam[1] = d1;
  lam[2] = d2;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    vec[r] = v0[r];
    vec[3 + r] = v1[r];
    vec[6 + r] = v2[r];
  }
}

// Cyclic Jacobi in binary32 from the identity, unsorted: on return F
// (row-major) is the product of the rotations applied, a proper rotation
// whose columns approximate the eigenvectors of a.  Stops at binary32
// resolution (|apq| <= 1e-7 sqrt|app aqq|) or after 6 sweeps.
__device__ __forceinline__ void jacobi3_frame_f(const float* a_in, float* F) {
  float a00 = a_in[0], a01 = a_in[1], a02 = a_in[2], a11 = a_in[3], a12 = a_in[4], a22 = a_in[5];
  float v0[3] = {1.f, 0.f, 0.f}, v1[3] = {0.f, 1.f, 0.f}, v2[3] = {0.f, 0.f, 1.f};
  auto small = [](float apq, float app, float aqq) { return apq == 0.0f || apq * apq <= 1e-14f * fabsf(app * aqq); };
  for (int sweep = 0; sweep < 6; ++sweep) {
    bool done = true;
    if (!small(a01, a00, a11)) {
      jacobi_rotate_f(a00, a11, a01, a02, a12, v0, v1);
      done = false;
    }
    if (!small(a02, a00, a22)) {
      jacobi_rotate_f(a00, a22, a02, a01, a12, v0, v2);
      done = false;
    }
    if (!small(a12, a11, a22)) {
      jacobi_rotate_f(a11, a22, a12, a01, a02, v1, v2);
      done = false;
    }
    if (done) break;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    F[3 * r] = v0[r];
    F[3 * r + 1] = v1[r];
    F[3 * r + 2] = v2[r];
  }
}

// Symmetric 3x3 eigen-decomposition in FP64.  a = (xx, xy, xz, yy, yz, zz);
// on return lam[] ascending and vec[3*c + r] = component r of the unit
// eigenvector of lam[c].
//
// The matrix is scaled by a power of two (exact) so that its largest entry
// lies in [1, 2).  Cyclic Jacobi in binary32 on its rounding gives a rotation
// close to the eigenvectors; its quaternion q, turned into a rotation matrix
// Q with the exact normalisation 2 / |q|^2, is orthogonal to FP64 rounding,
// and Q^T A Q is nearly diagonal (off-diagonal entries of the order of the
// binary32 rounding of A, against the eigenvalue gaps).  FP64 Jacobi sweeps
// finish from there, with rotations of the small-angle form, in one to three
// sweeps instead of four to six from the identity (GB300 runs FP64 at 1/64 of
// its FP32 rate, so the binary32 sweeps cost little).  Stops when every
// off-diagonal entry is negligible (jacobi_small) or after 24 sweeps; if the
// binary32 frame is not usable (non-finite), the sweeps start from the
// identity.
__device__ inline void eig3_sym(const double* a_in, double lam[3], double vec[9]) {
  int emax = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int ek = (__double2hiint(a_in[k]) >> 20) & 0x7ff;
    emax = ek > emax ? ek : emax;
  }
  int es = 2046 - emax;  // biased exponent of the scale that takes the largest entry to [1, 2)
  es = es < 1 ? 1 : (es > 2045 ? 2045 : es);
  const double sc = __hiloint2double(es << 20, 0);
  const double isc = __hiloint2double((2046 - es) << 20, 0);  // 1 / sc
  const double A[6] = {a_in[0] * sc, a_in[1] * sc, a_in[2] * sc, a_in[3] * sc, a_in[4] * sc, a_in[5] * sc};
  float af[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) af[k] = f64_to_f32(A[k]);
  float F[9], qf[4];
  jacobi3_frame_f(af, F);
  mat_to_quat<float>(F, qf);
  const float nf = qf[0] * qf[0] + qf[1] * qf[1] + qf[2] * qf[2] + qf[3] * qf[3];
  if (!(nf > 0.999f && nf < 1.001f)) {
    qf[0] = 1.0f;
    qf[1] = qf[2] = qf[3] = 0.0f;
  }
  const double w = f32_to_f64(qf[0]), x = f32_to_f64(qf[1]), y = f32_to_f64(qf[2]), z = f32_to_f64(qf[3]);
  const double n2 = fma(w, w, fma(x, x, fma(y, y, z * z)));
  // 2 / n2: n2 is within 1e-6 of 1, so r0 = 2 - n2 approximates 1 / n2 to
  // (n2 - 1)^2, and one Newton step for the reciprocal, r0 + r0 (1 - n2 r0),
  // leaves an error of the order of (n2 - 1)^4, below the FP64 rounding
  const double r0 = 2.0 - n2;
  const double s2 = 2.0 * fma(r0, fma(-n2, r0, 1.0), r0);
  // products of binary32 values are exact in FP64
  const double xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
               wz = w * z;
  const double Q[9] = {fma(-s2, yy + zz, 1.0), s2 * (xy - wz),          s2 * (xz + wy),
                       s2 * (xy + wz),          fma(-s2, xx + zz, 1.0), s2 * (yz - wx),
                       s2 * (xz - wy),          s2 * (yz + wx),          fma(-s2, xx + yy, 1.0)};
  // B = Q^T A Q (upper triangle), through T = A Q
  double T[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T[c] = fma(A[0], Q[c], fma(A[1], Q[3 + c], A[2] * Q[6 + c]));
    T[3 + c] = fma(A[1], Q[c], fma(A[3], Q[3 + c], A[4] * Q[6 + c]));
    T[6 + c] = fma(A[2], Q[c], fma(A[4], Q[3 + c], A[5] * Q[6 + c]));
  }
  double b00 = fma(Q[0], T[0], fma(Q[3], T[3], Q[6] * T[6]));
  double b01 = fma(Q[0], T[1], fma(Q[3], T[4], Q[6] * T[7]));
  double b02 = fma(Q[0], T[2], fma(Q[3], T[5], Q[6] * T[8]));
  double b11 = fma(Q[1], T[1], fma(Q[4], T[4], Q[7] * T[7]));
  double b12 = fma(Q[1], T[2], fma(Q[4], T[5], Q[7] * T[8]));
  double b22 = fma(Q[2], T[2], fma(Q[5], T[5], Q[8] * T[8]));
  double v0[3] = {1.0, 0.0, 0.0}, v1[3] = {0.0, 1.0, 0.0}, v2[3] = {0.0, 0.0, 1.0};
  for (int sweep = 0; sweep < 24; ++sweep) {
    bool done = true;
    if (!jacobi_small(b01, b00, b11)) {  // (p, q, r) = (0, 1, 2)
      jacobi_rotate(b00, b11, b01, b02, b12, v0, v1);
      done = false;
    }
    if (!jacobi_small(b02, b00, b22)) {  // (0, 2, 1)
      jacobi_rotate(b00, b22, b02, b01, b12, v0, v2);
      done = false;
    }
    if (!jacobi_small(b12, b11, b22)) {  // (1, 2, 0)
      jacobi_rotate(b11, b22, b12, b01, b02, v1, v2);
      done = false;
    }
    if (done) break;
  }
  // ascending, stable on ties; swaps of values keep everything in registers
  double d0 = b00, d1 = b11, d2 = b22;
  auto cswap = [](double& da, double& db, double* va, double* vb) {
    if (db < da) {
      const double t = da;
      da = db;
      db = t;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double u = va[r];
        va[r] = vb[r];
        vb[r] = u;
      }
    }
  };
  cswap(d0, d1, v0, v1);
  cswap(d1, d2, v1, v2);
  cswap(d0, d1, v0, v1);
  lam[0] = d0 * isc;
  lam[1] = d1 * isc;
  lam[2] = d2 * isc;
  // eigenvectors back in the input axes: Q v
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    vec[r] = fma(Q[3 * r], v0[0], fma(Q[3 * r + 1], v0[1], Q[3 * r + 2] * v0[2]));
    vec[3 + r] = fma(Q[3 * r], v1[0], fma(Q[3 * r + 1], v1[1], Q[3 * r + 2] * v1[2]));
    vec[6 + r] = fma(Q[3 * r], v2[0], fma(Q[3 * r + 1], v2[1], Q[3 * r + 2] * v2[2]));
  }
}

// ---- FP64 slots: pivoted LDL^T of each observation's scatter ----
//
// The FP64 voxel pass stores an observation's scatter S (symmetric positive
// semidefinite) as P S P^T = L D L^T, with P the permutation of complete
// (diagonal) pivoting, largest remaining diagonal first, and L unit lower
// triangular (|l| <= 1 for a semidefinite S; Higham, Accuracy and Stability
// of Numerical Algorithms, Sec. 10.3).  For a scan rotation R, with W the
// columns of R P^T L,
//   R S R^T = D0 W0 W0^T + D1 W1 W1^T + D2 W2 W2^T,
// W0 = R_pi0 + l10 R_pi1 + l20 R_pi2, W1 = R_pi1 + l21 R_pi2, W2 = R_pi2
// (R_k the k-th column of R): 9 FMAs instead of the 27 of R S, and no square
// root (a D entry a rounding below zero is kept as it is).  The mean is
// stored permuted too (P m), so that R m = sum_a R_pia (P m)_a.  The
// permutation's code (0..5) sits in the top bits of the slot's scan index.
constexpr int kPermShift = 29;                      // scan index bits below, code above
constexpr uint32_t kScanMask = (1u << kPermShift) - 1u;
// 4 bits per code: pi0 | pi1 << 2 (pi2 = 3 - pi0 - pi1); codes 0..5 are the
// permutations (0 1 2), (0 2 1), (1 0 2), (1 2 0), (2 0 1), (2 1 0)
constexpr uint32_t kPermTable = 0x629184u;

__device__ __forceinline__ void perm_decode(uint32_t code, int& p0, int& p1, int& p2) {
  const uint32_t f = (kPermTable >> (4u * code)) & 15u;
  p0 = (int)(f & 3u);
  p1 = (int)(f >> 2);
  p2 = 3 - p0 - p1;
}

// S = (xx, xy, xz, yy, yz, zz) -> out = (l10, l20, l21, D0, D1, D2); returns
// the permutation's code.  A zero pivot leaves its column of L zero.  For a
// semidefinite S every |l| <= 1; where rounding breaks that (a pivot and the
// entries it divides are all at the rounding level of S, as in the Schur
// complement of a rank-one scatter) the multiplier is clamped to [-1, 1],
// which changes the factored matrix only at that level and keeps the terms
// D_a W_a W_a^T from growing past |S|.
__device__ __forceinline__ double ldlt_mult(double x, double d) {
  return d > 0.0 ? fmin(fmax(x / d, -1.0), 1.0) : 0.0;
}

__device__ inline uint32_t ldlt3_pivoted(const double* S, double* out) {
  const double Sm[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  int p0 = 0;
  if (Sm[1][1] > Sm[p0][p0]) p0 = 1;
  if (Sm[2][2] > Sm[p0][p0]) p0 = 2;
  const int ra = p0 == 0 ? 1 : 0, rb = p0 == 2 ? 1 : 2;  // the two others, ascending
  const double D0 = Sm[p0][p0];
  const double la = ldlt_mult(Sm[ra][p0], D0), lb = ldlt_mult(Sm[rb][p0], D0);
  // Schur complement of the pivot on the remaining pair
  const double saa = fma(-la * D0, la, Sm[ra][ra]), sbb = fma(-lb * D0, lb, Sm[rb][rb]);
  const double sab = fma(-la * D0, lb, Sm[ra][rb]);
  const bool a_first = !(sbb > saa);
  const int p1 = a_first ? ra : rb, p2 = a_first ? rb : ra;
  const double D1 = a_first ? saa : sbb, s22 = a_first ? sbb : saa;
  const double l10 = a_first ? la : lb, l20 = a_first ? lb : la;
  const double l21 = ldlt_mult(sab, D1);
  out[0] = l10;
  out[1] = l20;
  out[2] = l21;
  out[3] = D0;
  out[4] = D1;
  out[5] = fma(-l21 * D1, l21, s22);
  (void)p2;
  // code of (p0, p1)
  return p0 == 0 ? (p1 == 1 ? 0u : 1u) : p0 == 1 ? (p1 == 0 ? 2u : 3u) : (p1 == 0 ? 4u : 5u);
}

// Per-scan FP32 table entry for the mixed path from an FP64 pose P and its
// reference (R_ref, t_ref): the unit quaternion q = (w, v) of
// dR = R R_ref^T (w >= 0), dt = t - t_ref and t_ref, as
//   (w, vx, vy, vz), (dt0, dt1, dt2, t_ref0), (t_ref1, t_ref2, 0, 0).
// For a unit q, dR x = x + E x with E x = 2w (v x x) + 2 v x (v x x).
// The entry from the FP64 quaternion q of dR and the pose's translation.
__device__ inline void scan_table_from_quat(const double* q, const double* P, const double* ref, float* out) {
  const double sg = q[0] < 0.0 ? -1.0 : 1.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) out[k] = f64_to_f32(sg * q[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out[4 + k] = f64_to_f32(P[9 + k] - ref[9 + k]);
    out[7 + k] = f64_to_f32(ref[9 + k]);
  }
  out[10] = 0.0f;
  out[11] = 0.0f;
}

// The entry from the pose matrix (at set-up); the FP64 quaternion of dR,
// kept to compose later steps onto, is written to qout.
__device__ inline void scan_table_entry(const double* P, const double* ref, float* out, double* qout) {
  double D[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) D[3 * r + c] = P[3 * r] * ref[3 * c] + P[3 * r + 1] * ref[3 * c + 1] + P[3 * r + 2] * ref[3 * c + 2];
  mat_to_quat<double>(D, qout);
  scan_table_from_quat(qout, P, ref, out);
}

// The FP64 quaternions of dR of both pose buffers, after the FP64 and FP32
// reference poses in the sref allocation: 2 x n_scans x 4 doubles.
__device__ __forceinline__ double* sq2_of(const double* sref, int64_t n_scans) {
  return const_cast<double*>(sref) + 18 * n_scans;  // 12 doubles + 12 floats per scan before it
}

// Hamilton product p q of FP64 quaternions (w, x, y, z)
__device__ __forceinline__ void quat_mul_d(const double* p, const double* q, double* r) {
  r[0] = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
  r[1] = p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2];
  r[2] = p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1];
  r[3] = p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0];
}

// Unit quaternion of Exp(phi): (cos(th/2), sin(th/2) phi / th), th = |phi|;
// below th = 0.1 from the Taylor series of both functions (terms to th^8;
// the first dropped term is below 1e-19).
__device__ inline void so3_exp_quat(const double* phi, double* q) {
  const double x = phi[0], y = phi[1], z = phi[2];
  const double t2 = x * x + y * y + z * z;
  double c, s;  // cos(th/2), sin(th/2) / th
  if (t2 < 0.01) {
    c = 1.0 + t2 * (-1.0 / 8 + t2 * (1.0 / 384 + t2 * (-1.0 / 46080 + t2 * (1.0 / 10321920))));
    s = 0.5 + t2 * (-1.0 / 48 + t2 * (1.0 / 3840 + t2 * (-1.0 / 645120 + t2 * (1.0 / 185794560))));
  } else {
    const double th = sqrt(t2);
    double sh;
    sincos(0.5 * th, &sh, &c);
    s = sh / th;
  }
  q[0] = c;
  q[1] = s * x;
  q[2] = s * y;
  q[3] = s * z;
}

// Hamilton product p q of quaternions held as float4 (w, x, y, z) in the
// fields (x, y, z, w): rot(p q) = rot(p) rot(q)
__device__ __forceinline__ float4 quat_mul_f(float4 p, float4 q) {
  return make_float4(fmaf(p.x, q.x, -fmaf(p.y, q.y, fmaf(p.z, q.z, p.w * q.w))),
                     fmaf(p.x, q.y, fmaf(p.y, q.x, fmaf(p.z, q.w, -p.w * q.z))),
                     fmaf(p.x, q.z, fmaf(-p.y, q.w, fmaf(p.z, q.x, p.w * q.y))),
                     fmaf(p.x, q.w, fmaf(p.y, q.z, fmaf(-p.z, q.y, p.w * q.x))));
}

// LDL^T of the symmetric 6x6 A (full, row-major) without pivoting, then
// solve A x = b.  Returns false if a pivot is not positive and finite.
__device__ inline bool ldlt6_solve(const double* A, const double* b, double* x) {
  // LD[i][k] = L[i][k] D[k], kept as the numerator it is (before the scaling
  // by 1 / D[k]), so every update is one FMA; the pivots' reciprocals serve
  // the factorisation and the diagonal solve alike (an FP64 division is a
  // long instruction sequence on this part)
  double L[6][6], LD[6][6], Di[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double dj = A[6 * j + j];
#pragma unroll
    for (int k = 0; k < j; ++k) dj = fma(-L[j][k], LD[j][k], dj);
    if (!(dj > 0.0) || !isfinite(dj)) return false;
    const double inv = 1.0 / dj;
    Di[j] = inv;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      double v = A[6 * i + j];
#pragma unroll
      for (int k = 0; k < j; ++k) v = fma(-L[i][k], LD[j][k], v);
      LD[i][j] = v;
      L[i][j] = v * inv;
    }
  }
  double y[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double v = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v = fma(-L[i][k], y[k], v);
    y[i] = v;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] *= Di[i];
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
// Between 1e-6 and 0.1 rad the coefficients come from their Taylor series
// sin(th)/th = sum (-1)^k th^2k / (2k+1)!, (1 - cos th)/th^2 = sum
// (-1)^k th^2k / (2k+2)! to th^8 (truncation below 1e-17 there), which saves
// the FP64 sin/cos.
__device__ inline void so3_exp(const double* phi, double* R) {
  double x = phi[0], y = phi[1], z = phi[2];
  double th2 = x * x + y * y + z * z;
  double a, b;
  if (th2 < 1e-12) {
    a = 1.0;
    b = 0.5;
  } else if (th2 < 0.01) {  // theta < 0.1: the series, no square root
    a = 1.0 + th2 * (-1.0 / 6 + th2 * (1.0 / 120 + th2 * (-1.0 / 5040 + th2 * (1.0 / 362880))));
    b = 0.5 + th2 * (-1.0 / 24 + th2 * (1.0 / 720 + th2 * (-1.0 / 40320 + th2 * (1.0 / 3628800))));
  } else {
    const double th = sqrt(th2);
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

// This thread's share of sum(p[0..n)) with a fixed assignment of indices:
// four independent load streams so the loads are in flight together.
template <int kThreads>
__device__ inline double strided_sum(const double* __restrict__ p, int64_t n) {
  // eight loads in flight per round
  double c[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int64_t k = threadIdx.x;
  for (; k + 7 * kThreads < n; k += 8 * kThreads) {
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] += __ldcg(p + k + u * kThreads);
  }
  for (; k < n; k += kThreads) c[0] += __ldcg(p + k);
  return ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
}

// Warp reduce-scatter of 32 values per lane: afterwards a[0] of lane l holds
// the warp's total of value l (fixed tree; 31 shuffles instead of 5 per value).
// At the level with offset o, the lanes with bit o set keep the upper half of
// their remaining values and receive it from the partner lane, the others
// keep and receive the lower half.
__device__ __forceinline__ void warp_reduce_scatter32(float (&a)[32]) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const bool up = (l & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = up ? a[k] : a[k + o];
      const float keep = up ? a[k + o] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// ---- bulk asynchronous copies (TMA engine) into shared memory ----
// A copy needs 16-byte aligned source and destination and a size that is a
// multiple of 16; it completes on an mbarrier as transaction bytes.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :
               : "r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// true once the barrier's phase with this parity has completed; false if it
// did not within the iteration limit
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit = kWaitLimit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(bar), "r"(bytes) : "memory");
}

// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory"); }

// order this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy writes (re-filling a buffer that was just read)
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" : : : "memory"); }

// Deterministic block-wide sum (fixed shape for a given blockDim).
template <int kThreads, typename T = double>
__device__ inline T block_sum(T v, T* smem /* kThreads / 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) smem[w] = v;
  __syncthreads();
  T r = T(0);
  if (w == 0) {
    // the warp sums reduced by warp 0 (fixed tree)
    r = l < kThreads / 32 ? smem[l] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      if (o < kThreads / 32) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// LM decision (one block): sums the trial cost and the predicted reduction
// in a fixed order, accepts iff every solve succeeded, the prediction is
// positive and the cost decreased, and updates the damping (Nielsen's rule:
// mu *= max(1/3, 1 - (2 rho - 1)^3), nu = 2 on acceptance; mu *= nu, nu *= 2
// otherwise).  Acceptance flips the current pose/plane buffers.
// With mode = 1 it only installs the summed cost as the current cost.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decide_apply(DevState* st, double csum, double psum);

template <int kThreads>
__device__ __forceinline__ void decide_body(const double* __restrict__ cost_part, int64_t n_cost,
                                            const double* __restrict__ pred_part, int64_t n_pred, DevState* st,
                                            int mode, double* red) {
  if (mode == 0 && st->honor_stop && st->stop) {
    if (threadIdx.x == 0) st->scan_pending = 0;
    return;
  }
  const double csum = block_sum<kThreads>(strided_sum<kThreads>(cost_part, n_cost), red);
  const double psum =
      block_sum<kThreads>(mode == 0 ? strided_sum<kThreads>(pred_part, n_pred) : 0.0, red);
  if (threadIdx.x != 0) return;
  if (mode == 1) {
    st->cost = csum;
    return;
  }
  decide_apply(st, csum, psum);
}

// The decision itself (thread 0), from the summed trial cost and predicted
// reduction.
__device__ __forceinline__ void decide_apply(DevState* st, double csum, double psum) {
  // work on a register copy: one load and one store of the state instead of a
  // chain of dependent global accesses
  DevState s = *st;
  const int fail = s.solve_fail_flag;
  const bool accept = !fail && psum > 0.0 && csum < s.cost;
  s.iters += 1;
  s.last_pred = psum;
  s.last_trial_cost = csum;
  s.solve_failed = fail;
  s.solve_fail_flag = 0;
  if (accept) {
    const double rho = (s.cost - csum) / psum;
    const double x = 2.0 * rho - 1.0;
    const double f = 1.0 - x * x * x;
    s.mu *= f > (1.0 / 3.0) ? f : (1.0 / 3.0);
    s.nu = 2.0;
    s.last_rho = rho;
    s.converged = (s.cost - csum) <= s.rel_tol * s.cost + s.abs_tol;
    s.cost = csum;
    s.cur = 1 - s.cur;
    s.accepted += 1;
    s.consec_reject = 0;
  } else {
    s.mu *= s.nu;
    s.nu *= 2.0;
    s.last_rho = (!fail && psum > 0.0) ? (s.cost - csum) / psum : __longlong_as_double(0x7ff8000000000000ll);
    s.consec_reject += 1;
  }
  s.last_accepted = accept;
  s.scan_pending = accept;
  if (s.honor_stop && (s.converged || s.iters >= s.max_iters || s.consec_reject >= s.max_consec_reject)) s.stop = 1;
  *st = s;
}


// Epilogue of a voxel pass that decides in its last block: every block adds
// one to the state's counter after its cost partial is visible device-wide;
// the block that brings the counter to n_cost sums all partials (in the same
// fixed order as a separate decision launch, so results do not depend on which
// block finishes last), decides, and re-arms the counter.  mode as for
// decide_body; with mode < 0 nothing is decided.
template <int kThreads>
__device__ __forceinline__ void voxel_pass_decide(const double* cost_part, int64_t n_cost, const double* pred_part,
                                                  int64_t n_pred, DevState* st, int mode, double* red,
                                                  int* is_last) {
  if (mode < 0) return;
  __syncthreads();  // thread 0 has written this block's partial
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&st->blocks_done, 1u);
    *is_last = prev == (unsigned)(n_cost - 1);
  }
  __syncthreads();
  if (!*is_last) return;
  __threadfence();
  decide_body<kThreads>(cost_part, n_cost, pred_part, n_pred, st, mode, red);
  if (threadIdx.x == 0) st->blocks_done = 0u;
}

}  // namespace mmba
