// Mixed-precision iteration kernels: FP32 per observation on re-centred
// clusters (anchors and reference poses fixed at load or at ba_set_state),
// FP64 only per scan (6x6 solve, pose composition), in the sum over voxel
// blocks and in the set-up that builds the FP32 copies.
#include "checked.cuh"
#include "mmba_internal.cuh"
#include "mmba_kernels.h"

namespace mmba {

// rows of the voxel-pass slots fetched into L2 ahead of the current one (the
// batch executor's tuner may pick another distance; results do not depend on it)
constexpr int kVoxPrefetch = 2;

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }


// E x for E = a [phi]x + b [phi]x^2:  a (phi x x) + b (phi x (phi x x))
__device__ __forceinline__ void apply_E(const float* ph, float a, float b, float x0, float x1, float x2, float& y0,
                                        float& y1, float& y2) {
  const float c0 = ph[1] * x2 - ph[2] * x1, c1 = ph[2] * x0 - ph[0] * x2, c2 = ph[0] * x1 - ph[1] * x0;
  const float d0 = ph[1] * c2 - ph[2] * c1, d1 = ph[2] * c0 - ph[0] * c2, d2 = ph[0] * c1 - ph[1] * c0;
  y0 = fmaf(a, c0, b * d0);
  y1 = fmaf(a, c1, b * d1);
  y2 = fmaf(a, c2, b * d2);
}

// ---------------------------------------------------------------------------
// Voxel pass (mixed): one thread per voxel over SELL-32 FP32 slices.
// Per observation, in the voxel's current frame B (rows e1, e2, n) and about
// its latest centroid delta (world axes, relative to the anchor):
//   x   = B (b + E l + dt - delta)                (posed mean - centroid)
//   M_o = G diag(sigma) G^T,   G = B dR V,  dR = I + E
// (G from the product of the quaternions of B, dR and V)
// where V, sigma are the observation's stored eigen-decomposition.  The sums
// of N x, M_o + N x x^T and N have a small normal direction in B, so FP32
// keeps lambda_min relatively accurate; an FP32 Jacobi in B gives the plane,
// and B and delta then move to the new eigenvectors and centroid.
// ---------------------------------------------------------------------------
template <bool kFull>
__device__ __forceinline__ void voxel_pass_mixed_body(const DevLayout& L, const DevMixed& X,
                                                      double* __restrict__ full_out, double* __restrict__ cost_part,
                                                      const double* __restrict__ pred_part, DevState* __restrict__ st,
                                                      int use_trial, int decide_mode, int64_t blk, float* red,
                                                      double* dred, int* is_last, int pf) {
  if (st->honor_stop && st->stop) {
    // a stopped solve takes no step, so no gradient is pending either
    if (decide_mode == 0 && blk == 0 && threadIdx.x == 0) st->scan_pending = 0;
    return;
  }
  const int buf = use_trial ? 1 - st->cur : st->cur;
  const float* __restrict__ stab = X.stab2 + (int64_t)buf * L.n_scans * kTab;
  float4* __restrict__ planes = X.planes32_2 + (int64_t)buf * L.n_voxels * 2;
  const int64_t p = blk * kVoxelThreads + threadIdx.x;
  float lam0 = 0.f;
  if (p < L.n_voxels) {
    const int64_t sl = p >> 5;
    const int lane = (int)(p & 31);
    const int len = L.vlen[p];
    const int64_t base = L.slice_off[sl] + lane;
    const float4 an = X.vanchor[p];
    const float4 qb = X.vstate[2 * p];
    const float4 dw = X.vstate[2 * p + 1];
    float B[9];
    quat_to_mat_f(qb.x, qb.y, qb.z, qb.w, B);
    float n = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float m00 = 0.f, m01 = 0.f, m02 = 0.f, m11 = 0.f, m12 = 0.f, m22 = 0.f;
    // the slot of observation k + 1 (three 128-bit loads) is fetched while k is processed
    const float4* __restrict__ slot = X.ve32 + kVe32 * base;
    float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0, n2 = n0;
    if (len > 0) {
      n0 = __ldg(slot);
      n1 = __ldg(slot + 1);
      n2 = __ldg(slot + 2);
    }
    for (int k = 0; k < len; ++k) {
      const float4 f0 = n0, f1 = n1, f2 = n2;
      // rows further ahead go to L2 without holding registers (the lanes'
      // 48-byte slots tile the row, so the warp covers all of its lines)
      if (pf > 0 && k + pf < len) prefetch_l2(slot + pf * kVe32 * kSlice);
      if (k + 1 < len) {
        slot += kVe32 * kSlice;
        n0 = __ldg(slot);
        n1 = __ldg(slot + 1);
        n2 = __ldg(slot + 2);
      }
      const int j = MMBA_IDX(__float_as_int(f1.w), L.n_scans, st);
      const float4* T4 = reinterpret_cast<const float4*>(stab + (int64_t)j * kTab);
      const float4 qd = __ldg(T4), t1 = __ldg(T4 + 1), t2 = __ldg(T4 + 2);
      const float ph[3] = {qd.y, qd.z, qd.w};
      const float b0 = f0.x, b1 = f0.y, b2 = f0.z, N = f0.w;
      // posed mean about the latest centroid (world axes), then voxel frame:
      // x = B (b + E l + dt - delta), lever l = b + a - t_ref
      const float l0 = b0 + (an.x - t1.w), l1 = b1 + (an.y - t2.x), l2 = b2 + (an.z - t2.y);
      float el0, el1, el2;
      apply_E(ph, 2.f * qd.x, 2.f, l0, l1, l2, el0, el1, el2);
      const float xw0 = (b0 - dw.x) + el0 + t1.x, xw1 = (b1 - dw.y) + el1 + t1.y, xw2 = (b2 - dw.z) + el2 + t1.z;
      const float x0 = fmaf(B[0], xw0, fmaf(B[1], xw1, B[2] * xw2));
      const float x1 = fmaf(B[3], xw0, fmaf(B[4], xw1, B[5] * xw2));
      const float x2 = fmaf(B[6], xw0, fmaf(B[7], xw1, B[8] * xw2));
      // G = B dR V as one quaternion product
      float G[9];
      const float4 qg = quat_mul_f(quat_mul_f(qb, qd), f2);
      quat_to_mat_f(qg.x, qg.y, qg.z, qg.w, G);
      const float sg0 = f1.x, sg1 = f1.y, sg2 = f1.z;
      // G diag(sigma) G^T + N x x^T, upper triangle
      const float g00 = G[0] * sg0, g01 = G[1] * sg1, g02 = G[2] * sg2;
      const float g10 = G[3] * sg0, g11 = G[4] * sg1, g12 = G[5] * sg2;
      const float g20 = G[6] * sg0, g21 = G[7] * sg1, g22 = G[8] * sg2;
      const float Nx0 = N * x0, Nx1 = N * x1, Nx2 = N * x2;
      m00 += fmaf(g00, G[0], fmaf(g01, G[1], fmaf(g02, G[2], Nx0 * x0)));
      m01 += fmaf(g00, G[3], fmaf(g01, G[4], fmaf(g02, G[5], Nx0 * x1)));
      m02 += fmaf(g00, G[6], fmaf(g01, G[7], fmaf(g02, G[8], Nx0 * x2)));
      m11 += fmaf(g10, G[3], fmaf(g11, G[4], fmaf(g12, G[5], Nx1 * x1)));
      m12 += fmaf(g10, G[6], fmaf(g11, G[7], fmaf(g12, G[8], Nx1 * x2)));
      m22 += fmaf(g20, G[6], fmaf(g21, G[7], fmaf(g22, G[8], Nx2 * x2)));
      s0 += Nx0;
      s1 += Nx1;
      s2 += Nx2;
      n += N;
    }
    const float inv = 1.0f / n;
    const float d0 = s0 * inv, d1 = s1 * inv, d2 = s2 * inv;  // centroid - delta, frame axes
    float A[6] = {fmaf(-d0, d0, m00 * inv), fmaf(-d0, d1, m01 * inv), fmaf(-d0, d2, m02 * inv),
                  fmaf(-d1, d1, m11 * inv), fmaf(-d1, d2, m12 * inv), fmaf(-d2, d2, m22 * inv)};
    float lam[3], W[9];
    eig3_sym_f(A, lam, W);
    // centroid - anchor and normal, world axes (B^T times frame vectors)
    const float cw0 = dw.x + fmaf(B[0], d0, fmaf(B[3], d1, B[6] * d2));
    const float cw1 = dw.y + fmaf(B[1], d0, fmaf(B[4], d1, B[7] * d2));
    const float cw2 = dw.z + fmaf(B[2], d0, fmaf(B[5], d1, B[8] * d2));
    float U[9];  // rows: new e1 (largest), e2, n (smallest), world axes
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = 2 - k;
      U[3 * k] = fmaf(B[0], W[3 * c], fmaf(B[3], W[3 * c + 1], B[6] * W[3 * c + 2]));
      U[3 * k + 1] = fmaf(B[1], W[3 * c], fmaf(B[4], W[3 * c + 1], B[7] * W[3 * c + 2]));
      U[3 * k + 2] = fmaf(B[2], W[3 * c], fmaf(B[5], W[3 * c + 1], B[8] * W[3 * c + 2]));
    }
    const float u0 = U[6], u1 = U[7], u2 = U[8];
    const float dp = fmaf(u0, cw0, fmaf(u1, cw1, u2 * cw2));  // u . (c - a)
    planes[2 * p] = make_float4(u0, u1, u2, dp);
    if (!kFull) {
      // the frame follows the eigenvectors (made right-handed), delta the centroid
      const float det = U[0] * (U[4] * U[8] - U[5] * U[7]) - U[1] * (U[3] * U[8] - U[5] * U[6]) +
                        U[2] * (U[3] * U[7] - U[4] * U[6]);
      if (det < 0.f) {
        U[0] = -U[0];
        U[1] = -U[1];
        U[2] = -U[2];
      }
      float qn[4];
      mat_to_quat<float>(U, qn);
      X.vstate[2 * p] = make_float4(qn[0], qn[1], qn[2], qn[3]);
      X.vstate[2 * p + 1] = make_float4(cw0, cw1, cw2, 0.f);
    } else {
      double* f = full_out + 9 * (int64_t)L.vperm[p];
      f[0] = lam[0];
      f[1] = lam[1];
      f[2] = lam[2];
      f[3] = u0;
      f[4] = u1;
      f[5] = u2;
      f[6] = (double)an.x + (double)cw0;
      f[7] = (double)an.y + (double)cw1;
      f[8] = (double)an.z + (double)cw2;
    }
    lam0 = lam[0];
  }
  // FP32 block sum of lambda_min (relative rounding ~1e-7 of a block's cost);
  // the sum over blocks is FP64
  const float tot = block_sum<kVoxelThreads, float>(lam0, red);
  if (threadIdx.x == 0) cost_part[blk] = (double)tot;
  voxel_pass_decide<kVoxelThreads>(cost_part, voxel_pass_blocks(L.n_voxels), pred_part, solve_blocks(L.n_scans), st,
                                   decide_mode, dred, is_last);
}

template <bool kFull>
__global__ void __launch_bounds__(kVoxelThreads, 6) voxel_pass_mixed_kernel(DevLayout L, DevMixed X,
                                                                        double* __restrict__ full_out,
                                                                        double* __restrict__ cost_part,
                                                                        const double* __restrict__ pred_part,
                                                                        DevState* __restrict__ st, int use_trial,
                                                                        int decide_mode) {
  __shared__ float red[kVoxelThreads / 32];
  __shared__ double dred[kVoxelThreads / 32];
  __shared__ int is_last;
  voxel_pass_mixed_body<kFull>(L, X, full_out, cost_part, pred_part, st, use_trial, decide_mode, blockIdx.x, red,
                               dred, &is_last, kVoxPrefetch);
}

// kMinBlocks (resident blocks per SM the registers are capped for) and pf are
// the batch tuner's knobs: neither changes any arithmetic
template <int kMinBlocks>
__global__ void __launch_bounds__(kVoxelThreads, kMinBlocks)
    voxel_pass_mixed_batch_kernel(const __grid_constant__ JobGroup G, int use_trial, int pf) {
  __shared__ float red[kVoxelThreads / 32];
  __shared__ double dred[kVoxelThreads / 32];
  __shared__ int is_last;
  const int job = find_job(G.vblk, G.n_jobs, blockIdx.x);
  const JobView& J = G.jobs[job];
  voxel_pass_mixed_body<false>(J.L, J.X, nullptr, J.cost_part, J.pred_part, J.st, use_trial, use_trial ? 0 : 1,
                               (int64_t)blockIdx.x - G.vblk[job], red, dred, &is_last, pf);
}

// ---------------------------------------------------------------------------
// Scan pass (mixed): one warp per scan.  The residual of an observation's
// mean is r = u . (q - c) = u . x - u . (c - a) with x = b + E l + dt as in
// the voxel pass (world axes).  The derivative terms are those of the FP64
// scan pass written in the scan's reference axes (lever l, scatter S_ref and
// w = dR^T u = u + E^T u), accumulated in FP32 per lane, reduced in FP32 per
// warp and rotated by dR once per scan.
//
// The scan's observations are contiguous in the scan-major copy, so they are
// staged into shared memory by bulk asynchronous copies (the TMA engine) in
// chunks of kScanChunk observations, double-buffered and completed on an
// mbarrier: one chunk is in flight while the previous one is processed, with
// no registers held for it.  Every wait is bounded; a wait that gives up sets
// the state's wait_timeout flag and the warp leaves after its copies land.
// ---------------------------------------------------------------------------

// one observation's terms added to the 27 sums (scan reference axes); E is
// dR - I of the scan, row-major
__device__ __forceinline__ void scan_obs_terms(float (&acc)[32], float4 bN, float4 S4, float2 S2, float4 pl, float4 an,
                                               const float (&E)[9], float dt0, float dt1, float dt2, float tr0,
                                               float tr1, float tr2, bool gn) {
  const float b0 = bN.x, b1 = bN.y, b2 = bN.z, N = bN.w;
  const float S00 = S4.x, S01 = S4.y, S02 = S4.z, S11 = S4.w, S12 = S2.x, S22 = S2.y;
  const float l0 = b0 + (an.x - tr0), l1 = b1 + (an.y - tr1), l2 = b2 + (an.z - tr2);
  const float el0 = fmaf(E[0], l0, fmaf(E[1], l1, E[2] * l2));
  const float el1 = fmaf(E[3], l0, fmaf(E[4], l1, E[5] * l2));
  const float el2 = fmaf(E[6], l0, fmaf(E[7], l1, E[8] * l2));
  const float x0 = b0 + el0 + dt0, x1 = b1 + el1 + dt1, x2 = b2 + el2 + dt2;
  const float r = fmaf(pl.x, x0, fmaf(pl.y, x1, fmaf(pl.z, x2, -pl.w)));
  // w = dR^T u = u + E^T u
  const float wx = fmaf(E[0], pl.x, fmaf(E[3], pl.y, fmaf(E[6], pl.z, pl.x)));
  const float wy = fmaf(E[1], pl.x, fmaf(E[4], pl.y, fmaf(E[7], pl.z, pl.y)));
  const float wz = fmaf(E[2], pl.x, fmaf(E[5], pl.y, fmaf(E[8], pl.z, pl.z)));
  const float Nr = N * r;
  const float swx = fmaf(S00, wx, fmaf(S01, wy, S02 * wz));
  const float swy = fmaf(S01, wx, fmaf(S11, wy, S12 * wz));
  const float swz = fmaf(S02, wx, fmaf(S12, wy, S22 * wz));
  const float mpx = fmaf(Nr, l0, swx), mpy = fmaf(Nr, l1, swy), mpz = fmaf(Nr, l2, swz);
  acc[0] = fmaf(mpy, wz, fmaf(-mpz, wy, acc[0]));
  acc[1] = fmaf(mpz, wx, fmaf(-mpx, wz, acc[1]));
  acc[2] = fmaf(mpx, wy, fmaf(-mpy, wx, acc[2]));
  acc[3] = fmaf(Nr, wx, acc[3]);
  acc[4] = fmaf(Nr, wy, acc[4]);
  acc[5] = fmaf(Nr, wz, acc[5]);
  const float Nlx = N * l0, Nly = N * l1, Nlz = N * l2;
  const float p00 = fmaf(Nlx, l0, S00), p01 = fmaf(Nlx, l1, S01), p02 = fmaf(Nlx, l2, S02);
  const float p11 = fmaf(Nly, l1, S11), p12 = fmaf(Nly, l2, S12), p22 = fmaf(Nlz, l2, S22);
  const float b00 = wy * p02 - wz * p01, b10 = wz * p00 - wx * p02, b20 = wx * p01 - wy * p00;
  const float b01 = wy * p12 - wz * p11, b11 = wz * p01 - wx * p12, b21 = wx * p11 - wy * p01;
  const float b02 = wy * p22 - wz * p12, b12 = wz * p02 - wx * p22;
  acc[6] = fmaf(wy, b02, fmaf(-wz, b01, acc[6]));
  acc[7] = fmaf(-wx, b02, fmaf(wz, b00, acc[7]));
  acc[8] = fmaf(wx, b01, fmaf(-wy, b00, acc[8]));
  acc[12] = fmaf(-wx, b12, fmaf(wz, b10, acc[12]));
  acc[13] = fmaf(wx, b11, fmaf(-wy, b10, acc[13]));
  acc[17] = fmaf(wx, b21, fmaf(-wy, b20, acc[17]));
  if (!gn) {
    const float wm = fmaf(wx, mpx, fmaf(wy, mpy, wz * mpz));
    acc[6] = fmaf(wx, mpx, acc[6] - wm);
    acc[12] = fmaf(wy, mpy, acc[12] - wm);
    acc[17] = fmaf(wz, mpz, acc[17] - wm);
    acc[7] = fmaf(0.5f, fmaf(wx, mpy, mpx * wy), acc[7]);
    acc[8] = fmaf(0.5f, fmaf(wx, mpz, mpx * wz), acc[8]);
    acc[13] = fmaf(0.5f, fmaf(wy, mpz, mpy * wz), acc[13]);
  }
  const float cx = Nly * wz - Nlz * wy, cy = Nlz * wx - Nlx * wz, cz = Nlx * wy - Nly * wx;
  acc[9] = fmaf(cx, wx, acc[9]);
  acc[10] = fmaf(cx, wy, acc[10]);
  acc[11] = fmaf(cx, wz, acc[11]);
  acc[14] = fmaf(cy, wx, acc[14]);
  acc[15] = fmaf(cy, wy, acc[15]);
  acc[16] = fmaf(cy, wz, acc[16]);
  acc[18] = fmaf(cz, wx, acc[18]);
  acc[19] = fmaf(cz, wy, acc[19]);
  acc[20] = fmaf(cz, wz, acc[20]);
  const float Nwx = N * wx, Nwy = N * wy, Nwz = N * wz;
  acc[21] = fmaf(Nwx, wx, acc[21]);
  acc[22] = fmaf(Nwx, wy, acc[22]);
  acc[23] = fmaf(Nwx, wz, acc[23]);
  acc[24] = fmaf(Nwy, wy, acc[24]);
  acc[25] = fmaf(Nwy, wz, acc[25]);
  acc[26] = fmaf(Nwz, wz, acc[26]);
}

// Shared-memory image of one chunk of a scan's observations.  Every array
// starts and ends on a 16-byte boundary (bulk copies need both); the float2
// and int32 arrays are copied from the 16-byte boundary at or below the
// chunk's first observation, hence the slack.
struct ScanChunk {
  float4 bN[kScanChunk];
  float4 S4[kScanChunk];
  float2 S2[kScanChunk + 2];
  int32_t vox[kScanChunk + 8];
};

// lane 0: copies of observations [o0, o1) of the scan-major arrays into S,
// completing on the barrier
__device__ __forceinline__ void issue_scan_chunk(ScanChunk& S, uint32_t bar, const float4* sbN, const float4* sS4,
                                                 const float2* sS2, const int32_t* svox, int64_t o0, int64_t o1) {
  const int64_t n = o1 - o0;
  const int64_t s2 = o0 & ~1ll, e2 = (o1 + 1) & ~1ll;
  const int64_t s4 = o0 & ~3ll, e4 = (o1 + 3) & ~3ll;
  const uint32_t bytes = (uint32_t)(32 * n + 8 * (e2 - s2) + 4 * (e4 - s4));
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(bar), "r"(bytes) : "memory");
  bulk_g2s(smem_u32(S.bN), sbN + o0, (uint32_t)(16 * n), bar);
  bulk_g2s(smem_u32(S.S4), sS4 + o0, (uint32_t)(16 * n), bar);
  bulk_g2s(smem_u32(S.S2), sS2 + s2, (uint32_t)(8 * (e2 - s2)), bar);
  bulk_g2s(smem_u32(S.vox), svox + s4, (uint32_t)(4 * (e4 - s4)), bar);
}

__device__ __forceinline__ void scan_pass_mixed_body(const DevLayout& L, const DevMixed& X,
                                                     double* __restrict__ gH, DevState* __restrict__ st,
                                                     int force, int j, float (*red)[kGH], float* tot, float* dR,
                                                     ScanChunk* chunks, uint64_t* bars) {
  if (!force && !st->scan_pending) return;
  const int lane = threadIdx.x & 31;
  const int buf = st->cur;
  const float* tb = X.stab2 + ((int64_t)buf * L.n_scans + j) * kTab;
  // dR = I + E, E x = ca (v x x) + cb v x (v x x) for the unit quaternion (w, v) of dR
  const float ph[3] = {tb[1], tb[2], tb[3]};
  const float ca = 2.f * tb[0], cb = 2.f;
  // E = dR - I = ca [phi]x + cb [phi]x^2 (row-major), once per scan
  float E[9];
  {
    const float vx = ph[0], vy = ph[1], vz = ph[2];
    E[0] = -cb * (vy * vy + vz * vz);
    E[4] = -cb * (vx * vx + vz * vz);
    E[8] = -cb * (vx * vx + vy * vy);
    E[1] = fmaf(cb * vx, vy, -ca * vz);
    E[3] = fmaf(cb * vx, vy, ca * vz);
    E[2] = fmaf(cb * vx, vz, ca * vy);
    E[6] = fmaf(cb * vx, vz, -ca * vy);
    E[5] = fmaf(cb * vy, vz, -ca * vx);
    E[7] = fmaf(cb * vy, vz, ca * vx);
  }
  const float dt0 = tb[4], dt1 = tb[5], dt2 = tb[6], tr0 = tb[7], tr1 = tb[8], tr2 = tb[9];
  const float4* __restrict__ prec = X.planes32_2 + (int64_t)buf * L.n_voxels * 2;
  const bool gn = st->hess_mode != 0;
  float acc[32];  // kGH sums, padded to a warp for the reduce-scatter
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.f;
  const int64_t lo = L.scan_off[j], hi = L.scan_off[j + 1];
  const int64_t no = L.n_obs;
  const float4* sbN = reinterpret_cast<const float4*>(X.se32);
  const float4* sS4 = sbN + no;
  const float2* sS2 = reinterpret_cast<const float2*>(sS4 + no);
  const int64_t nch = (hi - lo + kScanChunk - 1) / kScanChunk;
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
    if (nch > 0) issue_scan_chunk(chunks[0], bar0, sbN, sS4, sS2, L.se_vox, lo, min(hi, lo + kScanChunk));
    if (nch > 1)
      issue_scan_chunk(chunks[1], bar1, sbN, sS4, sS2, L.se_vox, lo + kScanChunk, min(hi, lo + 2 * kScanChunk));
  }
  __syncwarp();
  int64_t k = 0;
  bool ok = true;
  for (; k < nch; ++k) {
    const int b = (int)(k & 1);
    const bool landed = mbar_wait_bounded(b ? bar1 : bar0, (uint32_t)((k >> 1) & 1));
    if (__any_sync(0xffffffffu, !landed)) {
      ok = false;
      break;
    }
    const ScanChunk& S = chunks[b];
    const int64_t c0 = lo + k * kScanChunk;
    const int n = (int)min((int64_t)kScanChunk, hi - c0);
    const int off2 = (int)(c0 & 1), off4 = (int)(c0 & 3);
    // the planes of the lane's observations of the chunk first (L2 gathers in flight together)
    float4 pl[kScanChunk / 32], an[kScanChunk / 32];
#pragma unroll
    for (int q = 0; q < kScanChunk / 32; ++q) {
      const int i = lane + 32 * q;
      if (i < n) {
        const int64_t pv = MMBA_IDX((int64_t)S.vox[i + off4], L.n_voxels, st);
        pl[q] = __ldg(prec + 2 * pv);
        an[q] = __ldg(prec + 2 * pv + 1);
      }
    }
#pragma unroll
    for (int q = 0; q < kScanChunk / 32; ++q) {
      const int i = lane + 32 * q;
      if (i < n)
        scan_obs_terms(acc, S.bN[i], S.S4[i], S.S2[i + off2], pl[q], an[q], E, dt0, dt1, dt2, tr0, tr1, tr2, gn);
    }
    __syncwarp();
    if (lane == 0 && k + 2 < nch) {
      // the buffer's previous contents were read through the generic proxy
      asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
      issue_scan_chunk(chunks[b], b ? bar1 : bar0, sbN, sS4, sS2, L.se_vox, c0 + 2 * kScanChunk,
                       min(hi, c0 + 3 * kScanChunk));
    }
  }
  if (!ok) {
    // flag the failure, let the copies already issued land (bounded again), and leave
    if (lane == 0) {
      atomicExch(&st->wait_timeout, kErrTimeout);
      for (int64_t q = k; q < nch && q < k + 2; ++q) mbar_wait_bounded((q & 1) ? bar1 : bar0, (uint32_t)((q >> 1) & 1));
    }
    __syncwarp();
    return;
  }
  // FP32 warp reduction: the per-scan sums only need FP32 (their rounding is
  // far below what moves a pose by 1e-9 rad given H's size), and GB300's FP64
  // pipe is 1/64 of FP32, so FP64 is kept out of the reduction.
  static_assert(kScanMixedThreads == 32, "the staged scan pass runs one warp per scan");
  (void)red;
  warp_reduce_scatter32(acc);
  if (lane < kGH) tot[lane] = acc[0];
  if (threadIdx.x < 9) {
    // dR = I + a [phi]x + b [phi]x^2, entry (r, c)
    const int r = threadIdx.x / 3, c = threadIdx.x % 3;
    const float K[3][3] = {{0.f, -ph[2], ph[1]}, {ph[2], 0.f, -ph[0]}, {-ph[1], ph[0], 0.f}};
    const float k2 = ph[r] * ph[c] - (r == c ? ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2] : 0.f);
    dR[threadIdx.x] = (r == c ? 1.f : 0.f) + ca * K[r][c] + cb * k2;
  }
  __syncthreads();
  // world frame: g = blockdiag(dR, dR) g', H = blockdiag(dR, dR) H' blockdiag(dR, dR)^T,
  // one output entry per thread (6 of g, 21 of H's upper triangle)
  if (threadIdx.x < kGH) {
    const int t = threadIdx.x;
    double* out = gH + (int64_t)j * kGH;
    if (t < 6) {
      const int b = t / 3, r = t % 3;
      out[t] = f32_to_f64(dR[3 * r] * tot[3 * b] + dR[3 * r + 1] * tot[3 * b + 1] + dR[3 * r + 2] * tot[3 * b + 2]);
    } else {
      int r = 0, rem = t - 6;
      while (rem >= 6 - r) {
        rem -= 6 - r;
        ++r;
      }
      const int c = r + rem;
      const int br = r / 3, bc = c / 3, rr = r % 3, cc = c % 3;
      float v = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          int i = 3 * br + a, k = 3 * bc + b;
          if (i > k) {
            const int tmp = i;
            i = k;
            k = tmp;
          }
          const float h = tot[6 + 6 * i - i * (i - 1) / 2 + (k - i)];
          v = fmaf(dR[3 * rr + a] * h, dR[3 * cc + b], v);
        }
      out[t] = f32_to_f64(v);
    }
  }
}

__global__ void __launch_bounds__(kScanMixedThreads, 24) scan_pass_mixed_kernel(DevLayout L, DevMixed X,
                                                                                  double* __restrict__ gH,
                                                                                  DevState* __restrict__ st, int force) {
  __shared__ float red[1][kGH];
  __shared__ float tot[kGH];
  __shared__ float dR[9];
  __shared__ ScanChunk chunks[2];
  __shared__ uint64_t bars[2];
  scan_pass_mixed_body(L, X, gH, st, force, MMBA_IDX(scan_of_block(L, blockIdx.x), L.n_scans, st), red, tot, dR,
                       chunks, bars);
}

__global__ void __launch_bounds__(kScanMixedThreads, 24)
    scan_pass_mixed_batch_kernel(const __grid_constant__ JobGroup G) {
  __shared__ float red[1][kGH];
  __shared__ float tot[kGH];
  __shared__ float dR[9];
  __shared__ ScanChunk chunks[2];
  __shared__ uint64_t bars[2];
  const int job = find_job(G.sblk, G.n_jobs, blockIdx.x);
  const JobView& J = G.jobs[job];
  scan_pass_mixed_body(J.L, J.X, J.gH, J.st, 0,
                       MMBA_IDX(scan_of_block(J.L, (int64_t)blockIdx.x - G.sblk[job]), J.L.n_scans, J.st), red, tot,
                       dR, chunks, bars);
}

// Check of the bounded wait itself: an mbarrier that nothing arrives on, so
// the wait must give up after `limit` polls.  out[0] = 1 if it gave up.
__global__ void wait_probe_kernel(int limit, int32_t* out) {
  __shared__ uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
  }
  __syncwarp();
  const bool landed = mbar_wait_bounded(b, 0u, limit);
  if (threadIdx.x == 0) out[0] = landed ? 0 : 1;
}

// Per-scan FP32 table of buffer `buf` from the FP64 poses of that buffer.
__global__ void scan_table_kernel(int32_t n_scans, const double* poses2, const double* sref, float* stab2, int buf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_scans) return;
  scan_table_entry(poses2 + ((int64_t)buf * n_scans + j) * 12, sref + 12 * (int64_t)j,
                   stab2 + ((int64_t)buf * n_scans + j) * kTab, sq2_of(sref, n_scans) + ((int64_t)buf * n_scans + j) * 4);
}

// ---- launchers ---------------------------------------------------------------

cudaError_t launch_voxel_pass_mixed(const DevLayout& L, const DevMixed& X, double* full_out, double* cost_part,
                                    const double* pred_part, DevState* st, int use_trial, int decide_mode,
                                    cudaStream_t stream) {
  const int64_t nb = voxel_pass_blocks(L.n_voxels);
  if (full_out)
    voxel_pass_mixed_kernel<true><<<(unsigned)nb, kVoxelThreads, 0, stream>>>(L, X, full_out, cost_part, pred_part,
                                                                              st, use_trial, decide_mode);
  else
    voxel_pass_mixed_kernel<false><<<(unsigned)nb, kVoxelThreads, 0, stream>>>(L, X, nullptr, cost_part, pred_part,
                                                                               st, use_trial, decide_mode);
  return cudaGetLastError();
}

cudaError_t launch_scan_pass_mixed(const DevLayout& L, const DevMixed& X, const double* poses2, double* gH,
                                   DevState* st, int force, cudaStream_t stream) {
  if (L.n_scans == 0) return cudaSuccess;
  (void)poses2;
  scan_pass_mixed_kernel<<<(unsigned)L.n_scans, kScanMixedThreads, 0, stream>>>(L, X, gH, st, force);
  return cudaGetLastError();
}

cudaError_t launch_batch_voxel_pass_mixed(const JobGroup& T, int64_t n_blocks, int use_trial, cudaStream_t stream,
                                          int min_blocks, int pf) {
  switch (min_blocks) {
    case 4:
      voxel_pass_mixed_batch_kernel<4><<<(unsigned)n_blocks, kVoxelThreads, 0, stream>>>(T, use_trial, pf);
      break;
    case 8:
      voxel_pass_mixed_batch_kernel<8><<<(unsigned)n_blocks, kVoxelThreads, 0, stream>>>(T, use_trial, pf);
      break;
    default:
      voxel_pass_mixed_batch_kernel<6><<<(unsigned)n_blocks, kVoxelThreads, 0, stream>>>(T, use_trial, pf);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_scan_pass_mixed(const JobGroup& T, int64_t n_blocks, cudaStream_t stream) {
  scan_pass_mixed_batch_kernel<<<(unsigned)n_blocks, kScanMixedThreads, 0, stream>>>(T);
  return cudaGetLastError();
}

cudaError_t launch_wait_probe(int limit, int32_t* out, cudaStream_t stream) {
  wait_probe_kernel<<<1, 32, 0, stream>>>(limit, out);
  return cudaGetLastError();
}

cudaError_t launch_scan_table(int32_t n_scans, const double* poses2, const double* sref, float* stab2, int buf,
                              cudaStream_t stream) {
  scan_table_kernel<<<(n_scans + 127) / 128, 128, 0, stream>>>(n_scans, poses2, sref, stab2, buf);
  return cudaGetLastError();
}

}  // namespace mmba
