// FP64 iteration kernels: voxel pass (CalRes), scan pass (CalJH), per-scan
// damped solve + retraction (Solver) and the device-side LM decision
// (Algorithm 2 and Sec. IV-C of the paper).
#include "checked.cuh"
#include "mmba_internal.cuh"
#include "mmba_kernels.h"

namespace mmba {

// ---------------------------------------------------------------------------
// Voxel pass: one thread per voxel over the SELL-32 slices.
//
// For voxel i with observations o = (i, j): q_o = R_j m_o + t_j is the posed
// cluster mean; with an anchor a (the first q_o of the voxel) the thread sums
//   n = sum N_o,  s = sum N_o (q_o - a),  M = sum [R_j S_o R_j^T + N_o (q_o - a)(q_o - a)^T]
// so that the centroid is c = a + s / n and the world-point covariance of
// Eq. 1 is A = M / n - (c - a)(c - a)^T.  The anchor keeps the subtraction
// small (plane-sized instead of scene-sized).  R_j S_o R_j^T comes from the
// slot's pivoted LDL^T of S_o (ldlt3_pivoted): 61 FP64 operations per
// observation instead of 76 with S itself.  Then lambda_min(A) and its
// eigenvector give the plane (u, d = u^T c); the voxel's cost is lambda_min.
// ---------------------------------------------------------------------------
template <bool kFull>
__device__ __forceinline__ void voxel_pass_f64_body(const DevLayout& L, const double* __restrict__ poses2,
                                                    double* __restrict__ planes2, double* __restrict__ full_out,
                                                    double* __restrict__ cost_part,
                                                    const double* __restrict__ pred_part, DevState* __restrict__ st,
                                                    int use_trial, int decide_mode, int64_t blk, double* red,
                                                    int* is_last) {
  if (st->honor_stop && st->stop) {
    // a stopped solve takes no step, so no gradient is pending either
    if (decide_mode == 0 && blk == 0 && threadIdx.x == 0) st->scan_pending = 0;
    return;
  }
  const int buf = use_trial ? 1 - st->cur : st->cur;
  const double* __restrict__ poses = poses2 + (int64_t)buf * L.n_scans * 12;
  double* __restrict__ planes = planes2 + (int64_t)buf * L.n_voxels * kPlaneStride;
  const int64_t p = blk * kVoxelThreads + threadIdx.x;
  double lam0 = 0.0;
  if (p < L.n_voxels) {
    const int64_t s = p >> 5;
    const int lane = (int)(p & 31);
    const int len = L.vlen[p];
    const int64_t base = L.slice_off[s] + lane;
    const int64_t ne = L.n_elems;
    double n = 0.0, ax = 0.0, ay = 0.0, az = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    double m00 = 0.0, m01 = 0.0, m02 = 0.0, m11 = 0.0, m12 = 0.0, m22 = 0.0;
    for (int k = 0; k < len; ++k) {
      const int64_t e = base + (int64_t)k * kSlice;
      const uint32_t sv = (uint32_t)__ldg(L.ve_scan + e);
      int p0, p1, p2;
      perm_decode(sv >> kPermShift, p0, p1, p2);
      const double* __restrict__ P = poses + 12 * (int64_t)MMBA_IDX((int32_t)(sv & kScanMask), L.n_scans, st);
      const double l10 = __ldg(L.ve + e), l20 = __ldg(L.ve + ne + e), l21 = __ldg(L.ve + 2 * ne + e);
      const double D0 = __ldg(L.ve + 3 * ne + e), D1 = __ldg(L.ve + 4 * ne + e), D2 = __ldg(L.ve + 5 * ne + e);
      const double m0 = __ldg(L.ve + 6 * ne + e), m1 = __ldg(L.ve + 7 * ne + e), m2 = __ldg(L.ve + 8 * ne + e);
      const double N = __ldg(L.ve + 9 * ne + e);
      // columns pi0, pi1, pi2 of R
      const double a0 = P[p0], a1 = P[3 + p0], a2 = P[6 + p0];
      const double b0 = P[p1], b1 = P[3 + p1], b2 = P[6 + p1];
      const double c0 = P[p2], c1 = P[3 + p2], c2 = P[6 + p2];
      const double qx = fma(a0, m0, fma(b0, m1, fma(c0, m2, P[9])));
      const double qy = fma(a1, m0, fma(b1, m1, fma(c1, m2, P[10])));
      const double qz = fma(a2, m0, fma(b2, m1, fma(c2, m2, P[11])));
      if (k == 0) {
        ax = qx;
        ay = qy;
        az = qz;
      }
      const double dx = qx - ax, dy = qy - ay, dz = qz - az;
      // R S R^T = sum_a D_a W_a W_a^T with W = R P^T L
      const double w00 = fma(l10, b0, fma(l20, c0, a0)), w01 = fma(l10, b1, fma(l20, c1, a1)),
                   w02 = fma(l10, b2, fma(l20, c2, a2));
      const double w10 = fma(l21, c0, b0), w11 = fma(l21, c1, b1), w12 = fma(l21, c2, b2);
      const double u00 = D0 * w00, u01 = D0 * w01, u02 = D0 * w02;
      const double u10 = D1 * w10, u11 = D1 * w11, u12 = D1 * w12;
      const double u20 = D2 * c0, u21 = D2 * c1, u22 = D2 * c2;
      const double Nx = N * dx, Ny = N * dy, Nz = N * dz;
      m00 = fma(u00, w00, fma(u10, w10, fma(u20, c0, fma(Nx, dx, m00))));
      m01 = fma(u00, w01, fma(u10, w11, fma(u20, c1, fma(Nx, dy, m01))));
      m02 = fma(u00, w02, fma(u10, w12, fma(u20, c2, fma(Nx, dz, m02))));
      m11 = fma(u01, w01, fma(u11, w11, fma(u21, c1, fma(Ny, dy, m11))));
      m12 = fma(u01, w02, fma(u11, w12, fma(u21, c2, fma(Ny, dz, m12))));
      m22 = fma(u02, w02, fma(u12, w12, fma(u22, c2, fma(Nz, dz, m22))));
      sx += Nx;
      sy += Ny;
      sz += Nz;
      n += N;
    }
    const double inv = 1.0 / n;
    const double cx = sx * inv, cy = sy * inv, cz = sz * inv;  // centroid - anchor
    double A[6] = {fma(-cx, cx, m00 * inv), fma(-cx, cy, m01 * inv), fma(-cx, cz, m02 * inv),
                   fma(-cy, cy, m11 * inv), fma(-cy, cz, m12 * inv), fma(-cz, cz, m22 * inv)};
    double lam[3], V[9];
    eig3_sym(A, lam, V);
    const double ux = V[0], uy = V[1], uz = V[2];
    const double Cx = ax + cx, Cy = ay + cy, Cz = az + cz;
    double* pl = planes + p * kPlaneStride;
    pl[0] = ux;
    pl[1] = uy;
    pl[2] = uz;
    pl[3] = fma(ux, Cx, fma(uy, Cy, uz * Cz));
    if (kFull) {
      double* f = full_out + 9 * (int64_t)L.vperm[p];
      f[0] = lam[0];
      f[1] = lam[1];
      f[2] = lam[2];
      f[3] = ux;
      f[4] = uy;
      f[5] = uz;
      f[6] = Cx;
      f[7] = Cy;
      f[8] = Cz;
    }
    lam0 = lam[0];
  }
  const double tot = block_sum<kVoxelThreads>(lam0, red);
  if (threadIdx.x == 0) cost_part[blk] = tot;
  voxel_pass_decide<kVoxelThreads>(cost_part, voxel_pass_blocks(L.n_voxels), pred_part, solve_blocks(L.n_scans), st,
                                   decide_mode, red, is_last);
}

template <bool kFull>
__global__ void __launch_bounds__(kVoxelThreads) voxel_pass_f64_kernel(DevLayout L, const double* __restrict__ poses2,
                                                                      double* __restrict__ planes2,
                                                                      double* __restrict__ full_out,
                                                                      double* __restrict__ cost_part,
                                                                      const double* __restrict__ pred_part,
                                                                      DevState* __restrict__ st, int use_trial,
                                                                      int decide_mode) {
  __shared__ double red[kVoxelThreads / 32];
  __shared__ int is_last;
  voxel_pass_f64_body<kFull>(L, poses2, planes2, full_out, cost_part, pred_part, st, use_trial, decide_mode,
                             blockIdx.x, red, &is_last);
}

__global__ void __launch_bounds__(kVoxelThreads) voxel_pass_f64_batch_kernel(const __grid_constant__ JobGroup G,
                                                                             int use_trial) {
  __shared__ double red[kVoxelThreads / 32];
  __shared__ int is_last;
  const int job = find_job(G.vblk, G.n_jobs, blockIdx.x);
  const JobView& J = G.jobs[job];
  voxel_pass_f64_body<false>(J.L, J.poses2, J.planes2, nullptr, J.cost_part, J.pred_part, J.st, use_trial,
                             use_trial ? 0 : 1, (int64_t)blockIdx.x - G.vblk[job], red, &is_last);
}

// ---------------------------------------------------------------------------
// Scan pass: one block per scan over the scan-major copy.
//
// Per observation (voxel i, scan j) the surrogate's gradient and Hessian are
// accumulated in scan coordinates and rotated to the world frame once per
// scan.  With w = R^T u (normal in scan coordinates), r = w^T m + u^T t - d
// (residual of the cluster mean) and m' = S w + N r m:
//   g_rot = m' x w,               g_trans = N r w,
//   H_rr  = [w]x (S + N m m^T) [w]x^T + (w m'^T + m' w^T)/2 - (w^T m') I,
//   H_rt  = N (m x w) w^T,        H_tt = N w w^T,
// all carrying the factor 2 / N_i, which the scan-major copy has folded into
// S and N.  The world-frame blocks are R (.) R^T.  Gauss-Newton mode drops
// the (w m'^T + m' w^T)/2 - (w^T m') I term.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scan_pass_f64_body(const DevLayout& L, const double* __restrict__ poses2,
                                                   const double* __restrict__ planes2, double* __restrict__ gH,
                                                   const DevState* __restrict__ st, int force, int j,
                                                   double (*red)[kGH]) {
  // a rejected step (or an iteration after the solve stopped) leaves g, H unchanged
  if (!force && !st->scan_pending) return;
  const int buf = st->cur;
  const double* __restrict__ P = poses2 + ((int64_t)buf * L.n_scans + j) * 12;
  const double* __restrict__ planes = planes2 + (int64_t)buf * L.n_voxels * kPlaneStride;
  const bool gn = st->hess_mode != 0;
  const double r00 = P[0], r01 = P[1], r02 = P[2], r10 = P[3], r11 = P[4], r12 = P[5], r20 = P[6], r21 = P[7],
               r22 = P[8];
  const double tx = P[9], ty = P[10], tz = P[11];
  double acc[kGH];
#pragma unroll
  for (int k = 0; k < kGH; ++k) acc[k] = 0.0;
  double dg0 = 0.0, dg1 = 0.0, dg2 = 0.0;  // sums of w_a m'_a (exact Hessian's diagonal)
  const int64_t lo = L.scan_off[j], hi = L.scan_off[j + 1];
  const int64_t no = L.n_obs;
  for (int64_t o = lo + threadIdx.x; o < hi; o += kScanThreads) {
    const double4_32a pl =
        *reinterpret_cast<const double4_32a*>(planes + (int64_t)MMBA_IDX(__ldg(L.se_vox + o), L.n_voxels, st) * kPlaneStride);
    const double S00 = __ldg(L.se + o), S01 = __ldg(L.se + no + o), S02 = __ldg(L.se + 2 * no + o);
    const double S11 = __ldg(L.se + 3 * no + o), S12 = __ldg(L.se + 4 * no + o), S22 = __ldg(L.se + 5 * no + o);
    const double mx = __ldg(L.se + 6 * no + o), my = __ldg(L.se + 7 * no + o), mz = __ldg(L.se + 8 * no + o);
    const double N = __ldg(L.se + 9 * no + o);
    // w = R^T u
    const double wx = fma(r00, pl.x, fma(r10, pl.y, r20 * pl.z));
    const double wy = fma(r01, pl.x, fma(r11, pl.y, r21 * pl.z));
    const double wz = fma(r02, pl.x, fma(r12, pl.y, r22 * pl.z));
    const double e = fma(pl.x, tx, fma(pl.y, ty, fma(pl.z, tz, -pl.w)));
    const double r = fma(wx, mx, fma(wy, my, fma(wz, mz, e)));
    const double Nr = N * r;
    // S w and m' = S w + N r m
    const double swx = fma(S00, wx, fma(S01, wy, S02 * wz));
    const double swy = fma(S01, wx, fma(S11, wy, S12 * wz));
    const double swz = fma(S02, wx, fma(S12, wy, S22 * wz));
    const double mpx = fma(Nr, mx, swx), mpy = fma(Nr, my, swy), mpz = fma(Nr, mz, swz);
    // gradient (FMA chains into the sums)
    acc[0] = fma(mpy, wz, fma(-mpz, wy, acc[0]));
    acc[1] = fma(mpz, wx, fma(-mpx, wz, acc[1]));
    acc[2] = fma(mpx, wy, fma(-mpy, wx, acc[2]));
    acc[3] = fma(Nr, wx, acc[3]);
    acc[4] = fma(Nr, wy, acc[4]);
    acc[5] = fma(Nr, wz, acc[5]);
    // P = S + N m m^T
    const double Nmx = N * mx, Nmy = N * my, Nmz = N * mz;
    const double p00 = fma(Nmx, mx, S00), p01 = fma(Nmx, my, S01), p02 = fma(Nmx, mz, S02);
    const double p11 = fma(Nmy, my, S11), p12 = fma(Nmy, mz, S12), p22 = fma(Nmz, mz, S22);
    // B = [w]x P  (rows: b_r = (w x P_col)...), computed as columns c of P: w x P[:, c]
    const double b00 = wy * p02 - wz * p01, b10 = wz * p00 - wx * p02, b20 = wx * p01 - wy * p00;
    const double b01 = wy * p12 - wz * p11, b11 = wz * p01 - wx * p12, b21 = wx * p11 - wy * p01;
    const double b02 = wy * p22 - wz * p12, b12 = wz * p02 - wx * p22;
    // B [w]x^T into the rotation block; [w]x rows: (0,-wz,wy), (wz,0,-wx), (-wy,wx,0)
    acc[6] = fma(wy, b02, fma(-wz, b01, acc[6]));
    acc[7] = fma(wz, b00, fma(-wx, b02, acc[7]));
    acc[8] = fma(wx, b01, fma(-wy, b00, acc[8]));
    acc[12] = fma(wz, b10, fma(-wx, b12, acc[12]));
    acc[13] = fma(wx, b11, fma(-wy, b10, acc[13]));
    acc[17] = fma(wx, b21, fma(-wy, b20, acc[17]));
    if (!gn) {
      // exact term sym(w m'^T) - (w . m') I: the off-diagonal halves go into
      // the sums here, the diagonal products into dg (the trace is taken off
      // once per thread after the loop, as the term is linear)
      const double hx = 0.5 * mpx, hy = 0.5 * mpy, hz = 0.5 * mpz;
      acc[7] = fma(wx, hy, fma(hx, wy, acc[7]));
      acc[8] = fma(wx, hz, fma(hx, wz, acc[8]));
      acc[13] = fma(wy, hz, fma(hy, wz, acc[13]));
      dg0 = fma(wx, mpx, dg0);
      dg1 = fma(wy, mpy, dg1);
      dg2 = fma(wz, mpz, dg2);
    }
    // rotation-translation block: N (m x w) w^T
    const double cx = Nmy * wz - Nmz * wy, cy = Nmz * wx - Nmx * wz, cz = Nmx * wy - Nmy * wx;
    acc[9] += cx * wx;
    acc[10] += cx * wy;
    acc[11] += cx * wz;
    acc[14] += cy * wx;
    acc[15] += cy * wy;
    acc[16] += cy * wz;
    acc[18] += cz * wx;
    acc[19] += cz * wy;
    acc[20] += cz * wz;
    // translation block: N w w^T
    const double Nwx = N * wx, Nwy = N * wy;
    acc[21] += Nwx * wx;
    acc[22] += Nwx * wy;
    acc[23] += Nwx * wz;
    acc[24] += Nwy * wy;
    acc[25] += Nwy * wz;
    acc[26] += N * wz * wz;
  }
  if (!gn) {
    const double tr = dg0 + dg1 + dg2;
    acc[6] += dg0 - tr;
    acc[12] += dg1 - tr;
    acc[17] += dg2 - tr;
  }
  // deterministic block reduction
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kGH; ++k) {
    double v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (l == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[kGH];
#pragma unroll
    for (int k = 0; k < kGH; ++k) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < kScanThreads / 32; ++q) v += red[q][k];
      a[k] = v;
    }
    // scan-frame 6x6 (upper triangle layout of acc[6..26], row-major over the 6x6)
    double Hs[6][6];
    int idx = 6;
    for (int r = 0; r < 6; ++r)
      for (int c = r; c < 6; ++c) {
        Hs[r][c] = a[idx];
        Hs[c][r] = a[idx];
        ++idx;
      }
    const double R[3][3] = {{r00, r01, r02}, {r10, r11, r12}, {r20, r21, r22}};
    double* out = gH + (int64_t)j * kGH;
    for (int r = 0; r < 3; ++r) {
      out[r] = R[r][0] * a[0] + R[r][1] * a[1] + R[r][2] * a[2];
      out[3 + r] = R[r][0] * a[3] + R[r][1] * a[4] + R[r][2] * a[5];
    }
    // world blocks: R B R^T for each 3x3 block of Hs
    double Hw[6][6];
    for (int br = 0; br < 2; ++br)
      for (int bc = 0; bc < 2; ++bc) {
        double T[3][3];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c)
            T[r][c] = R[r][0] * Hs[3 * br + 0][3 * bc + c] + R[r][1] * Hs[3 * br + 1][3 * bc + c] +
                      R[r][2] * Hs[3 * br + 2][3 * bc + c];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c)
            Hw[3 * br + r][3 * bc + c] = T[r][0] * R[c][0] + T[r][1] * R[c][1] + T[r][2] * R[c][2];
      }
    idx = 6;
    for (int r = 0; r < 6; ++r)
      for (int c = r; c < 6; ++c) out[idx++] = 0.5 * (Hw[r][c] + Hw[c][r]);
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_pass_f64_kernel(DevLayout L, const double* __restrict__ poses2,
                                                                    const double* __restrict__ planes2,
                                                                    double* __restrict__ gH,
                                                                    const DevState* __restrict__ st, int force) {
  __shared__ double red[kScanThreads / 32][kGH];
  scan_pass_f64_body(L, poses2, planes2, gH, st, force, MMBA_IDX(scan_of_block(L, blockIdx.x), L.n_scans, st), red);
}

__global__ void __launch_bounds__(kScanThreads) scan_pass_f64_batch_kernel(const __grid_constant__ JobGroup G) {
  __shared__ double red[kScanThreads / 32][kGH];
  const int job = find_job(G.sblk, G.n_jobs, blockIdx.x);
  const JobView& J = G.jobs[job];
  scan_pass_f64_body(J.L, J.poses2, J.planes2, J.gH, J.st, 0,
                     MMBA_IDX(scan_of_block(J.L, (int64_t)blockIdx.x - G.sblk[job]), J.L.n_scans, J.st), red);
}

// ---------------------------------------------------------------------------
// Solver: one thread per scan.  A = H + mu diag(H), A delta = -g by LDL^T,
// trial pose R' = Exp(dphi) R, t' = t + dt, and the scan's share of the
// predicted reduction -(g^T delta + delta^T H delta / 2).  The fixed scan and
// scans without observations keep their pose.
// ---------------------------------------------------------------------------
// *stepped = false: the pose is kept (fixed scan, no observation, failed
// factorisation); otherwise dlt holds the increment.
__device__ inline double solve_scan(const DevLayout& L, int j, const double* __restrict__ P, double* __restrict__ Pt,
                                    const double* __restrict__ gH, DevState* st, double* dlt, bool* stepped) {
  *stepped = false;
  const double* a = gH + (int64_t)j * kGH;
  // a scan nobody observes keeps its pose: no observation in this handle's
  // layout, or, for a voxel-sharded solve (g, H totals over all shards), an
  // all-zero total Hessian diagonal (an observation always makes it nonzero)
  const bool unseen = st->shard ? (a[6] == 0.0 && a[12] == 0.0 && a[17] == 0.0 && a[21] == 0.0 && a[24] == 0.0 &&
                                   a[26] == 0.0)
                                : L.scan_off[j + 1] == L.scan_off[j];
  if (j == L.fixed_scan || unseen) {
    for (int k = 0; k < 12; ++k) Pt[k] = P[k];
    return 0.0;
  }
  double g[6], H[36], A[36], b[6];
  for (int k = 0; k < 6; ++k) g[k] = a[k];
  int idx = 6;
  for (int r = 0; r < 6; ++r)
    for (int c = r; c < 6; ++c) {
      H[6 * r + c] = a[idx];
      H[6 * c + r] = a[idx];
      ++idx;
    }
  const double mu = st->mu;
  for (int k = 0; k < 36; ++k) A[k] = H[k];
  for (int k = 0; k < 6; ++k) {
    A[7 * k] = fma(mu, H[7 * k], H[7 * k]);
    b[k] = -g[k];
  }
  if (!ldlt6_solve(A, b, dlt)) {
    atomicOr(&st->solve_fail_flag, 1);
    for (int k = 0; k < 12; ++k) Pt[k] = P[k];
    return 0.0;
  }
  // L = -(g^T D + D^T H D / 2); the quadratic form from H's upper triangle
  double gd = 0.0, half = 0.0;
  for (int r = 0; r < 6; ++r) {
    gd = fma(g[r], dlt[r], gd);
    double hr = 0.5 * H[7 * r] * dlt[r];
    for (int c = r + 1; c < 6; ++c) hr = fma(H[6 * r + c], dlt[c], hr);
    half = fma(dlt[r], hr, half);
  }
  const double pred = -(gd + half);
  double E[9];
  so3_exp(dlt, E);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Pt[3 * r + c] = E[3 * r] * P[c] + E[3 * r + 1] * P[3 + c] + E[3 * r + 2] * P[6 + c];
  Pt[9] = P[9] + dlt[3];
  Pt[10] = P[10] + dlt[4];
  Pt[11] = P[11] + dlt[5];
  *stepped = true;
  return pred;
}

// With stab2 given (mixed precision) the trial scan's FP32 table entry is
// written too, from the trial pose and the scan's reference pose.  Block blk
// (scans blk * kSolveThreads ..) writes the sum of its scans' predicted
// reductions to pred_part[blk], in a fixed order.
__device__ __forceinline__ void solve_f64_body(const DevLayout& L, double* __restrict__ poses2,
                                               const double* __restrict__ gH, double* __restrict__ pred_part,
                                               DevState* st, const double* __restrict__ sref,
                                               float* __restrict__ stab2, int64_t blk, double* red) {
  if (st->honor_stop && st->stop) return;  // uniform over the block
  const int64_t j = blk * kSolveThreads + threadIdx.x;
  double pred = 0.0;
  if (j < L.n_scans) {
    const int cur = st->cur;
    const double* P = poses2 + ((int64_t)cur * L.n_scans + j) * 12;
    double* Pt = poses2 + ((int64_t)(1 - cur) * L.n_scans + j) * 12;
    double dlt[6];
    bool stepped;
    pred = solve_scan(L, (int)j, P, Pt, gH, st, dlt, &stepped);
    if (stab2) {
      // FP64 quaternion of the trial dR: the step's Exp composed onto the
      // current one (no matrix-to-quaternion conversion per step)
      double* sq2 = sq2_of(sref, L.n_scans);
      const double* qc = sq2 + ((int64_t)cur * L.n_scans + j) * 4;
      double* qt = sq2 + ((int64_t)(1 - cur) * L.n_scans + j) * 4;
      double qn[4];
      if (stepped) {
        double qe[4];
        so3_exp_quat(dlt, qe);
        quat_mul_d(qe, qc, qn);
      } else {
        for (int k = 0; k < 4; ++k) qn[k] = qc[k];
      }
      for (int k = 0; k < 4; ++k) qt[k] = qn[k];
      scan_table_from_quat(qn, Pt, sref + 12 * (int64_t)j, stab2 + ((int64_t)(1 - cur) * L.n_scans + j) * kTab);
    }
  }
  const double tot = block_sum<kSolveThreads>(pred, red);
  if (threadIdx.x == 0) pred_part[blk] = tot;
}

__global__ void __launch_bounds__(kSolveThreads) solve_f64_kernel(DevLayout L, double* __restrict__ poses2,
                                                                 const double* __restrict__ gH,
                                                                 double* __restrict__ pred_part, DevState* st,
                                                                 const double* __restrict__ sref,
                                                                 float* __restrict__ stab2) {
  __shared__ double red[kSolveThreads / 32];
  solve_f64_body(L, poses2, gH, pred_part, st, sref, stab2, blockIdx.x, red);
}

__global__ void __launch_bounds__(kSolveThreads) solve_f64_batch_kernel(const __grid_constant__ JobGroup G) {
  __shared__ double red[kSolveThreads / 32];
  const int job = find_job(G.oblk, G.n_jobs, blockIdx.x);
  const JobView& J = G.jobs[job];
  solve_f64_body(J.L, J.poses2, J.gH, J.pred_part, J.st, J.X.sref, J.X.stab2, (int64_t)blockIdx.x - G.oblk[job], red);
}

__global__ void __launch_bounds__(kDecideThreads) decide_kernel(const double* __restrict__ cost_part, int64_t n_cost,
                                                               const double* __restrict__ pred_part, int64_t n_pred,
                                                               DevState* st, int mode) {
  __shared__ double red[kDecideThreads / 32];
  decide_body<kDecideThreads>(cost_part, n_cost, pred_part, n_pred, st, mode, red);
}

// Voxel-sharded solve: this handle's part of the trial cost (its cost
// partials summed in the decision's fixed order) ...
__global__ void __launch_bounds__(kDecideThreads) shard_cost_kernel(const double* __restrict__ cost_part, int64_t n_cost,
                                                                   double* __restrict__ out) {
  __shared__ double red[kDecideThreads / 32];
  const double csum = block_sum<kDecideThreads>(strided_sum<kDecideThreads>(cost_part, n_cost), red);
  if (threadIdx.x == 0) *out = csum;
}

// ... and the decision from the trial cost summed over every shard (the
// predicted reduction comes from the total g, H, so every shard has it whole)
__global__ void __launch_bounds__(kDecideThreads) shard_decide_kernel(const double* __restrict__ pred_part,
                                                                     int64_t n_pred, DevState* st, double trial_total) {
  __shared__ double red[kDecideThreads / 32];
  const double psum = block_sum<kDecideThreads>(strided_sum<kDecideThreads>(pred_part, n_pred), red);
  if (threadIdx.x == 0) decide_apply(st, trial_total, psum);
}

// ---- launchers ---------------------------------------------------------------

cudaError_t launch_voxel_pass_f64(const DevLayout& L, const double* poses2, double* planes2, double* full_out,
                                  double* cost_part, const double* pred_part, DevState* st, int use_trial,
                                  int decide_mode, cudaStream_t stream) {
  const int64_t nb = voxel_pass_blocks(L.n_voxels);
  if (full_out)
    voxel_pass_f64_kernel<true><<<(unsigned)nb, kVoxelThreads, 0, stream>>>(L, poses2, planes2, full_out, cost_part,
                                                                            pred_part, st, use_trial, decide_mode);
  else
    voxel_pass_f64_kernel<false><<<(unsigned)nb, kVoxelThreads, 0, stream>>>(L, poses2, planes2, nullptr, cost_part,
                                                                             pred_part, st, use_trial, decide_mode);
  return cudaGetLastError();
}

cudaError_t launch_scan_pass_f64(const DevLayout& L, const double* poses2, const double* planes2, double* gH,
                                 const DevState* st, int force, cudaStream_t stream) {
  if (L.n_scans == 0) return cudaSuccess;
  scan_pass_f64_kernel<<<(unsigned)L.n_scans, kScanThreads, 0, stream>>>(L, poses2, planes2, gH, st, force);
  return cudaGetLastError();
}

cudaError_t launch_shard_cost(const DevLayout& L, const double* cost_part, double* out, cudaStream_t stream) {
  shard_cost_kernel<<<1, kDecideThreads, 0, stream>>>(cost_part, voxel_pass_blocks(L.n_voxels), out);
  return cudaGetLastError();
}

cudaError_t launch_shard_decide(const DevLayout& L, const double* pred_part, DevState* st, double trial_total,
                                cudaStream_t stream) {
  shard_decide_kernel<<<1, kDecideThreads, 0, stream>>>(pred_part, solve_blocks(L.n_scans), st, trial_total);
  return cudaGetLastError();
}

cudaError_t launch_solve_f64(const DevLayout& L, double* poses2, const double* gH, double* pred_part, DevState* st,
                             const double* sref, float* stab2, cudaStream_t stream) {
  solve_f64_kernel<<<(unsigned)solve_blocks(L.n_scans), kSolveThreads, 0, stream>>>(L, poses2, gH, pred_part, st, sref,
                                                                                    stab2);
  return cudaGetLastError();
}

cudaError_t launch_decide(const double* cost_part, int64_t n_cost, const double* pred_part, int64_t n_pred,
                          DevState* st, int mode, cudaStream_t stream) {
  decide_kernel<<<1, kDecideThreads, 0, stream>>>(cost_part, n_cost, pred_part, n_pred, st, mode);
  return cudaGetLastError();
}

cudaError_t launch_batch_solve(const JobGroup& T, int64_t n_blocks, cudaStream_t stream) {
  solve_f64_batch_kernel<<<(unsigned)n_blocks, kSolveThreads, 0, stream>>>(T);
  return cudaGetLastError();
}

cudaError_t launch_batch_voxel_pass_f64(const JobGroup& T, int64_t n_blocks, int use_trial, cudaStream_t stream) {
  voxel_pass_f64_batch_kernel<<<(unsigned)n_blocks, kVoxelThreads, 0, stream>>>(T, use_trial);
  return cudaGetLastError();
}

cudaError_t launch_batch_scan_pass_f64(const JobGroup& T, int64_t n_blocks, cudaStream_t stream) {
  scan_pass_f64_batch_kernel<<<(unsigned)n_blocks, kScanThreads, 0, stream>>>(T);
  return cudaGetLastError();
}

}  // namespace mmba
