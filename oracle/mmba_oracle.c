/*
 * CPU oracle for the MM LiDAR bundle-adjustment iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain sequential FP64 code that follows the
 * paper's formulation step by step; only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it.  It shares no code with the CUDA
 * library.  Sums run in CSR order, one observation after another.
 *
 * What each function follows:
 *  - point clusters: Eq. 2 (Sec. III);
 *  - cost: Eq. 1, the sum over voxels of the smallest eigenvalue of the
 *    voxel's world-point covariance;
 *  - surrogate: Eq. 3 (BALM3's majorizer, Sec. III);
 *  - residual evaluation / Jacobian-Hessian / solver: Algorithm 2 (CalRes,
 *    CalJH, Solver) and Sec. IV-C;
 *  - LM control: Sec. IV-C-1 and Fig. 1 (damping adjusted on the host side).
 * The paper defers the surrogate's derivatives to BALM3; the gradient and
 * Hessian below are derived from Eq. 3 for the left perturbation
 * R' = Exp(dphi) R, t' = t + dt (tests pin them by finite differences).
 */
#include "mmba_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- small dense helpers ------------------------------------------------ */

static void sym_unpack(const double* a, double M[3][3]) {
  M[0][0] = a[0];
  M[0][1] = M[1][0] = a[1];
  M[0][2] = M[2][0] = a[2];
  M[1][1] = a[3];
  M[1][2] = M[2][1] = a[4];
  M[2][2] = a[5];
}

static void pose_R(const double* pose, double R[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[r][c] = pose[3 * r + c];
}

static void mat_mul(const double A[3][3], const double B[3][3], double C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

static void mat_mul_bt(const double A[3][3], const double B[3][3], double C[3][3]) /* A B^T */ {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[j][k];
      C[i][j] = s;
    }
}

static void mat_vec(const double A[3][3], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i) y[i] = A[i][0] * x[0] + A[i][1] * x[1] + A[i][2] * x[2];
}

static void mat_t_vec(const double A[3][3], const double x[3], double y[3]) /* A^T x */ {
  for (int i = 0; i < 3; ++i) y[i] = A[0][i] * x[0] + A[1][i] * x[1] + A[2][i] * x[2];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static void skew(const double u[3], double K[3][3]) /* K x = u x x */ {
  K[0][0] = 0.0;
  K[0][1] = -u[2];
  K[0][2] = u[1];
  K[1][0] = u[2];
  K[1][1] = 0.0;
  K[1][2] = -u[0];
  K[2][0] = -u[1];
  K[2][1] = u[0];
  K[2][2] = 0.0;
}

/* R S R^T for symmetric S */
static void rotate_sym(const double R[3][3], const double S[3][3], double out[3][3]) {
  double T[3][3];
  mat_mul(R, S, T);
  mat_mul_bt(T, R, out);
}

/* ---- a0: points -> point clusters (Eq. 2) ------------------------------- */

void orc_points_to_raw(int64_t n_obs, const int64_t* point_off, const double* pts, double* raw) {
  for (int64_t o = 0; o < n_obs; ++o) {
    double* a = raw + 10 * o;
    memset(a, 0, 10 * sizeof(double));
    for (int64_t k = point_off[o]; k < point_off[o + 1]; ++k) {
      const double* p = pts + 3 * k;
      a[0] += p[0] * p[0];
      a[1] += p[0] * p[1];
      a[2] += p[0] * p[2];
      a[3] += p[1] * p[1];
      a[4] += p[1] * p[2];
      a[5] += p[2] * p[2];
      a[6] += p[0];
      a[7] += p[1];
      a[8] += p[2];
    }
    a[9] = (double)(point_off[o + 1] - point_off[o]);
  }
}

void orc_points_to_centred(int64_t n_obs, const int64_t* point_off, const double* pts, double* centred) {
  for (int64_t o = 0; o < n_obs; ++o) {
    double* a = centred + 10 * o;
    memset(a, 0, 10 * sizeof(double));
    int64_t n = point_off[o + 1] - point_off[o];
    a[9] = (double)n;
    if (n == 0) continue;
    double m[3] = {0.0, 0.0, 0.0};
    for (int64_t k = point_off[o]; k < point_off[o + 1]; ++k)
      for (int d = 0; d < 3; ++d) m[d] += pts[3 * k + d];
    for (int d = 0; d < 3; ++d) m[d] /= (double)n;
    for (int64_t k = point_off[o]; k < point_off[o + 1]; ++k) {
      double x = pts[3 * k] - m[0], y = pts[3 * k + 1] - m[1], z = pts[3 * k + 2] - m[2];
      a[0] += x * x;
      a[1] += x * y;
      a[2] += x * z;
      a[3] += y * y;
      a[4] += y * z;
      a[5] += z * z;
    }
    a[6] = m[0];
    a[7] = m[1];
    a[8] = m[2];
  }
}

/* Raw sums -> centred form: m = v / N, S_ab = P_ab - v_a m_b, every entry by
 * one fused multiply-add so the conversion is bit-reproducible. */
void orc_raw_to_centred(int64_t n_obs, const double* raw, double* centred) {
  static const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int64_t o = 0; o < n_obs; ++o) {
    const double* r = raw + 10 * o;
    double* c = centred + 10 * o;
    double n = r[9];
    double m[3] = {r[6] / n, r[7] / n, r[8] / n};
    for (int e = 0; e < 6; ++e) c[e] = fma(-r[6 + ia[e]], m[ib[e]], r[e]);
    c[6] = m[0];
    c[7] = m[1];
    c[8] = m[2];
    c[9] = n;
  }
}

/* ---- 3x3 symmetric eigen-solve: cyclic Jacobi --------------------------- */
/* Golub & Van Loan, Matrix Computations, Sec. 8.5 (symmetric Schur 2x2 and
 * the cyclic-by-row sweep), run until every off-diagonal entry is negligible
 * relative to its diagonal pair. */
int orc_eig3(const double* A, double* lam, double* V) {
  double a[3][3], v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  sym_unpack(A, a);
  static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
  int sweep;
  for (sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < 3; ++r) {
      int p = P[r], q = Q[r];
      double apq = a[p][q];
      if (apq == 0.0) continue;
      if (fabs(apq) <= 1e-18 * sqrt(fabs(a[p][p] * a[q][q]))) continue;
      rotated = 1;
      double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
      double t;
      if (fabs(tau) > 1e150)
        t = 0.5 / tau;
      else
        t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      for (int k = 0; k < 3; ++k) { /* A <- A J */
        double akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) { /* A <- J^T A */
        double apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
      a[p][q] = a[q][p] = 0.0;
      for (int k = 0; k < 3; ++k) { /* V <- V J */
        double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
    if (!rotated) break;
  }
  int idx[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i) /* ascending order, stable */
    for (int j = i + 1; j < 3; ++j)
      if (a[idx[j]][idx[j]] < a[idx[i]][idx[i]]) {
        int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  for (int c = 0; c < 3; ++c) {
    lam[c] = a[idx[c]][idx[c]];
    for (int r = 0; r < 3; ++r) V[3 * r + c] = v[r][idx[c]];
  }
  return sweep;
}

static double eig_min(const double C[3][3], double u[3], double lam3[3]) {
  double packed[6] = {C[0][0], C[0][1], C[0][2], C[1][1], C[1][2], C[2][2]};
  double lam[3], V[9];
  orc_eig3(packed, lam, V);
  if (u) {
    u[0] = V[0];
    u[1] = V[3];
    u[2] = V[6];
  }
  if (lam3) memcpy(lam3, lam, sizeof lam);
  return lam[0];
}

/* ---- cost, Eq. 1 -------------------------------------------------------- */

double orc_cost_points(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan,
                       const int64_t* point_off, const double* pts, const double* poses, double* lam0) {
  double cost = 0.0;
  for (int64_t i = 0; i < n_voxels; ++i) {
    double n = 0.0, c[3] = {0, 0, 0};
    for (int64_t o = voxel_off[i]; o < voxel_off[i + 1]; ++o) {
      double R[3][3], q[3];
      const double* t = poses + 12 * (int64_t)obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)obs_scan[o], R);
      for (int64_t k = point_off[o]; k < point_off[o + 1]; ++k) {
        mat_vec(R, pts + 3 * k, q);
        for (int d = 0; d < 3; ++d) c[d] += q[d] + t[d];
        n += 1.0;
      }
    }
    if (n == 0.0) {
      if (lam0) lam0[i] = 0.0;
      continue;
    }
    for (int d = 0; d < 3; ++d) c[d] /= n;
    double C[3][3] = {{0}};
    for (int64_t o = voxel_off[i]; o < voxel_off[i + 1]; ++o) {
      double R[3][3], q[3];
      const double* t = poses + 12 * (int64_t)obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)obs_scan[o], R);
      for (int64_t k = point_off[o]; k < point_off[o + 1]; ++k) {
        mat_vec(R, pts + 3 * k, q);
        double x[3] = {q[0] + t[0] - c[0], q[1] + t[1] - c[1], q[2] + t[2] - c[2]};
        for (int r = 0; r < 3; ++r)
          for (int s = 0; s < 3; ++s) C[r][s] += x[r] * x[s];
      }
    }
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) C[r][s] /= n;
    double l = eig_min(C, NULL, NULL);
    if (lam0) lam0[i] = l;
    cost += l;
  }
  return cost;
}

double orc_cost_eq1(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan, const double* raw,
                    const double* poses, double* lam0) {
  double cost = 0.0;
  for (int64_t i = 0; i < n_voxels; ++i) {
    double P[3][3] = {{0}}, v[3] = {0, 0, 0}, n = 0.0;
    for (int64_t o = voxel_off[i]; o < voxel_off[i + 1]; ++o) {
      const double* a = raw + 10 * o;
      double R[3][3], Pf[3][3], RPR[3][3], Rv[3];
      const double* t = poses + 12 * (int64_t)obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)obs_scan[o], R);
      sym_unpack(a, Pf);
      rotate_sym(R, Pf, RPR);
      mat_vec(R, a + 6, Rv);
      double N = a[9];
      /* Eq. 2: P_ij = R P_f R^T + R v_f t^T + t v_f^T R^T + N t t^T */
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) P[r][s] += RPR[r][s] + Rv[r] * t[s] + t[r] * Rv[s] + N * t[r] * t[s];
      for (int r = 0; r < 3; ++r) v[r] += Rv[r] + N * t[r]; /* v_ij = R v_f + N t */
      n += N;
    }
    if (n == 0.0) {
      if (lam0) lam0[i] = 0.0;
      continue;
    }
    double C[3][3];
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) C[r][s] = P[r][s] / n - v[r] * v[s] / (n * n);
    double l = eig_min(C, NULL, NULL);
    if (lam0) lam0[i] = l;
    cost += l;
  }
  return cost;
}

double orc_voxel_pass(const orc_problem* p, const double* poses, double* planes) {
  double cost = 0.0;
  for (int64_t i = 0; i < p->n_voxels; ++i) {
    double n = 0.0, c[3] = {0, 0, 0};
    for (int64_t o = p->voxel_off[i]; o < p->voxel_off[i + 1]; ++o) {
      const double* a = p->agg + 10 * o;
      double R[3][3], q[3];
      const double* t = poses + 12 * (int64_t)p->obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)p->obs_scan[o], R);
      mat_vec(R, a + 6, q);
      for (int d = 0; d < 3; ++d) c[d] += a[9] * (q[d] + t[d]);
      n += a[9];
    }
    double* pl = planes + 9 * i;
    if (n == 0.0) {
      memset(pl, 0, 9 * sizeof(double));
      continue;
    }
    for (int d = 0; d < 3; ++d) c[d] /= n;
    double A[3][3] = {{0}};
    for (int64_t o = p->voxel_off[i]; o < p->voxel_off[i + 1]; ++o) {
      const double* a = p->agg + 10 * o;
      double R[3][3], S[3][3], RSR[3][3], q[3];
      const double* t = poses + 12 * (int64_t)p->obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)p->obs_scan[o], R);
      sym_unpack(a, S);
      rotate_sym(R, S, RSR);
      mat_vec(R, a + 6, q);
      double x[3] = {q[0] + t[0] - c[0], q[1] + t[1] - c[1], q[2] + t[2] - c[2]};
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) A[r][s] += RSR[r][s] + a[9] * x[r] * x[s];
    }
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) A[r][s] /= n;
    double u[3], lam[3];
    eig_min(A, u, lam);
    pl[0] = lam[0];
    pl[1] = lam[1];
    pl[2] = lam[2];
    pl[3] = u[0];
    pl[4] = u[1];
    pl[5] = u[2];
    pl[6] = c[0];
    pl[7] = c[1];
    pl[8] = c[2];
    cost += lam[0];
  }
  return cost;
}

/* ---- MM surrogate, Eq. 3 ------------------------------------------------ */

double orc_surrogate_eq3(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan, const double* raw,
                         const double* poses, const double* planes_l, const double* poses_l) {
  double total = 0.0;
  for (int64_t i = 0; i < n_voxels; ++i) {
    const double* u = planes_l + 9 * i + 3;
    double n = 0.0, z = 0.0;
    /* z = 1/2 sum_j u^T v_ij evaluated at T^(l) */
    for (int64_t o = voxel_off[i]; o < voxel_off[i + 1]; ++o) {
      const double* a = raw + 10 * o;
      double R[3][3], Rv[3];
      const double* t = poses_l + 12 * (int64_t)obs_scan[o] + 9;
      pose_R(poses_l + 12 * (int64_t)obs_scan[o], R);
      mat_vec(R, a + 6, Rv);
      double vij[3] = {Rv[0] + a[9] * t[0], Rv[1] + a[9] * t[1], Rv[2] + a[9] * t[2]};
      z += 0.5 * dot3(u, vij);
      n += a[9];
    }
    if (n == 0.0) continue;
    double sum = 0.0;
    for (int64_t o = voxel_off[i]; o < voxel_off[i + 1]; ++o) {
      const double* a = raw + 10 * o;
      double R[3][3], Pf[3][3], RPR[3][3], Rv[3], Pij[3][3], vij[3], Pu[3];
      const double* t = poses + 12 * (int64_t)obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)obs_scan[o], R);
      sym_unpack(a, Pf);
      rotate_sym(R, Pf, RPR);
      mat_vec(R, a + 6, Rv);
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) Pij[r][s] = RPR[r][s] + Rv[r] * t[s] + t[r] * Rv[s] + a[9] * t[r] * t[s];
      for (int r = 0; r < 3; ++r) vij[r] = Rv[r] + a[9] * t[r];
      mat_vec(Pij, u, Pu);
      sum += dot3(u, Pu) / n - 4.0 * z * dot3(u, vij) / (n * n);
    }
    total += sum + 4.0 * z * z / (n * n);
  }
  return total;
}

double orc_surrogate_points(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan,
                            const int64_t* point_off, const double* pts, const double* poses,
                            const double* planes_l) {
  double total = 0.0;
  for (int64_t i = 0; i < n_voxels; ++i) {
    const double* u = planes_l + 9 * i + 3;
    double d = dot3(u, planes_l + 9 * i + 6);
    double n = 0.0, sum = 0.0;
    for (int64_t o = voxel_off[i]; o < voxel_off[i + 1]; ++o) {
      double R[3][3], q[3];
      const double* t = poses + 12 * (int64_t)obs_scan[o] + 9;
      pose_R(poses + 12 * (int64_t)obs_scan[o], R);
      for (int64_t k = point_off[o]; k < point_off[o + 1]; ++k) {
        mat_vec(R, pts + 3 * k, q);
        double r = u[0] * (q[0] + t[0]) + u[1] * (q[1] + t[1]) + u[2] * (q[2] + t[2]) - d;
        sum += r * r;
        n += 1.0;
      }
    }
    if (n > 0.0) total += sum / n;
  }
  return total;
}

/* ---- surrogate gradient and Hessian ------------------------------------- */
/* Per observation o = (voxel i, scan j), with w = R^T u, e = u^T t - d,
 * s = w^T v_f + N e, m = R (P_f w + e v_f), K = [u]x:
 *   g_o = (2/N_i) [ m x u ; s u ]
 *   H_o = (2/N_i) [[ K (R P_f R^T) K^T + (u m^T + m u^T)/2 - (u^T m) I , ((R v_f) x u) u^T ],
 *                  [ u ((R v_f) x u)^T                                  , N u u^T          ]]
 * (the (u m^T + m u^T)/2 - (u^T m) I term is the second-order rotation term;
 * Gauss-Newton drops it).  Summed per scan in CSR order. */
void orc_grad_hess(const orc_problem* p, const double* poses, const double* planes, int gauss_newton, double* g,
                   double* H) {
  memset(g, 0, sizeof(double) * 6 * (size_t)p->n_scans);
  memset(H, 0, sizeof(double) * 36 * (size_t)p->n_scans);
  for (int64_t i = 0; i < p->n_voxels; ++i) {
    const double* u = planes + 9 * i + 3;
    double d = dot3(u, planes + 9 * i + 6);
    double n = 0.0;
    for (int64_t o = p->voxel_off[i]; o < p->voxel_off[i + 1]; ++o) n += p->agg[10 * o + 9];
    if (n == 0.0) continue;
    double K[3][3];
    skew(u, K);
    for (int64_t o = p->voxel_off[i]; o < p->voxel_off[i + 1]; ++o) {
      const double* a = p->agg + 10 * o;
      int32_t j = p->obs_scan[o];
      double R[3][3];
      const double* t = poses + 12 * (int64_t)j + 9;
      pose_R(poses + 12 * (int64_t)j, R);
      double N = a[9];
      /* raw cluster from the centred one: P_f = S + N m m^T, v_f = N m */
      double Pf[3][3], vf[3];
      sym_unpack(a, Pf);
      for (int r = 0; r < 3; ++r) {
        vf[r] = N * a[6 + r];
        for (int s = 0; s < 3; ++s) Pf[r][s] += N * a[6 + r] * a[6 + s];
      }
      double w[3], Pw[3], tmp[3], m[3];
      mat_t_vec(R, u, w);
      double e = dot3(u, t) - d;
      double sres = dot3(w, vf) + N * e;
      mat_vec(Pf, w, Pw);
      for (int r = 0; r < 3; ++r) tmp[r] = Pw[r] + e * vf[r];
      mat_vec(R, tmp, m);
      double mxu[3];
      cross3(m, u, mxu);
      double sc = 2.0 / n;
      double* gj = g + 6 * (int64_t)j;
      for (int r = 0; r < 3; ++r) {
        gj[r] += sc * mxu[r];
        gj[3 + r] += sc * sres * u[r];
      }
      double RPR[3][3], KM[3][3], KMKt[3][3], Rv[3], Rvxu[3];
      rotate_sym(R, Pf, RPR);
      mat_mul(K, RPR, KM);
      mat_mul_bt(KM, K, KMKt);
      mat_vec(R, vf, Rv);
      cross3(Rv, u, Rvxu);
      double um = dot3(u, m);
      double* Hj = H + 36 * (int64_t)j;
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
          double hrr = KMKt[r][s];
          if (!gauss_newton) hrr += 0.5 * (u[r] * m[s] + m[r] * u[s]) - (r == s ? um : 0.0);
          Hj[6 * r + s] += sc * hrr;
          Hj[6 * r + 3 + s] += sc * Rvxu[r] * u[s];
          Hj[6 * (3 + r) + s] += sc * u[r] * Rvxu[s];
          Hj[6 * (3 + r) + 3 + s] += sc * N * u[r] * u[s];
        }
    }
  }
}

/* ---- solve and retraction ----------------------------------------------- */

int orc_ldlt6(const double* A, const double* b, double* x) {
  double L[6][6] = {{0}}, D[6], y[6];
  for (int j = 0; j < 6; ++j) {
    double dj = A[6 * j + j];
    for (int k = 0; k < j; ++k) dj -= L[j][k] * L[j][k] * D[k];
    if (!(dj > 0.0) || !isfinite(dj)) return -1;
    D[j] = dj;
    L[j][j] = 1.0;
    for (int i = j + 1; i < 6; ++i) {
      double v = A[6 * i + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k] * D[k];
      L[i][j] = v / dj;
    }
  }
  for (int i = 0; i < 6; ++i) { /* L y = b */
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v;
  }
  for (int i = 0; i < 6; ++i) y[i] /= D[i];
  for (int i = 5; i >= 0; --i) { /* L^T x = y */
    double v = y[i];
    for (int k = i + 1; k < 6; ++k) v -= L[k][i] * x[k];
    x[i] = v;
  }
  for (int i = 0; i < 6; ++i)
    if (!isfinite(x[i])) return -1;
  return 0;
}

/* Rodrigues: Exp(phi) = I + (sin th / th) K + ((1 - cos th) / th^2) K^2 with
 * K = [phi]x; 1 - cos th is formed as 2 sin^2(th/2); below th = 1e-6 the
 * second-order series I + K + K^2/2 is used. */
void orc_exp_so3(const double* phi, double* R) {
  double th = sqrt(dot3(phi, phi));
  double K[3][3], K2[3][3];
  skew(phi, K);
  mat_mul(K, K, K2);
  double a, b;
  if (th < 1e-6) {
    a = 1.0;
    b = 0.5;
  } else {
    double sh = sin(0.5 * th);
    a = sin(th) / th;
    b = 2.0 * sh * sh / (th * th);
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[3 * r + c] = (r == c ? 1.0 : 0.0) + a * K[r][c] + b * K2[r][c];
}

void orc_retract(const double* pose, const double* delta, double* out) {
  double E[9], Ee[3][3], R[3][3], Rn[3][3];
  orc_exp_so3(delta, E);
  pose_R(E, Ee);
  pose_R(pose, R);
  mat_mul(Ee, R, Rn);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) out[3 * r + c] = Rn[r][c];
  for (int d = 0; d < 3; ++d) out[9 + d] = pose[9 + d] + delta[3 + d];
}

/* ---- Levenberg-Marquardt ------------------------------------------------ */
/* Damping: A = H + mu diag(H) per scan (Algorithm 2, Solver).  Gain ratio
 * rho = (c(T) - c(T')) / L with L = sum_j -(g_j^T D_j + D_j^T H_j D_j / 2).
 * A step is accepted iff every per-scan solve succeeded, L > 0 and
 * c(T') < c(T).  Damping update (Nielsen's rule, Madsen, Nielsen & Tingleff,
 * "Methods for Non-Linear Least Squares Problems", 2004): on acceptance
 * mu *= max(1/3, 1 - (2 rho - 1)^3), nu = 2; on rejection mu *= nu, nu *= 2. */

void orc_lm_init(const orc_problem* p, const orc_lm_config* cfg, const double* poses, double* planes, double* g,
                 double* H, orc_lm_state* st) {
  memset(st, 0, sizeof *st);
  st->cost = orc_voxel_pass(p, poses, planes);
  orc_grad_hess(p, poses, planes, cfg->gauss_newton, g, H);
  st->mu = cfg->mu0;
  st->nu = 2.0;
  st->last_rho = NAN;
  st->last_pred = NAN;
  st->last_trial_cost = NAN;
}

int orc_lm_step(const orc_problem* p, const orc_lm_config* cfg, double* poses, double* planes, double* g, double* H,
                orc_lm_state* st) {
  int32_t ns = p->n_scans;
  int64_t* nobs = (int64_t*)calloc((size_t)ns, sizeof(int64_t));
  for (int64_t o = 0; o < p->n_obs; ++o) nobs[p->obs_scan[o]]++;
  double* delta = (double*)calloc((size_t)ns * 6, sizeof(double));
  double* trial = (double*)malloc(sizeof(double) * 12 * (size_t)ns);
  double* tplanes = (double*)malloc(sizeof(double) * 9 * (size_t)(p->n_voxels > 0 ? p->n_voxels : 1));
  int ok = 1;
  double pred = 0.0;
  for (int32_t j = 0; j < ns; ++j) {
    double* D = delta + 6 * (int64_t)j;
    if (j == cfg->fixed_scan || nobs[j] == 0) continue;
    const double* Hj = H + 36 * (int64_t)j;
    const double* gj = g + 6 * (int64_t)j;
    double A[36], b[6];
    memcpy(A, Hj, sizeof A);
    for (int k = 0; k < 6; ++k) {
      A[7 * k] += st->mu * Hj[7 * k];
      b[k] = -gj[k];
    }
    if (orc_ldlt6(A, b, D) != 0) {
      ok = 0;
      memset(D, 0, 6 * sizeof(double));
      continue;
    }
    double gD = 0.0, DHD = 0.0;
    for (int r = 0; r < 6; ++r) {
      gD += gj[r] * D[r];
      for (int c = 0; c < 6; ++c) DHD += D[r] * Hj[6 * r + c] * D[c];
    }
    pred += -(gD + 0.5 * DHD);
  }
  double trial_cost = NAN;
  if (ok) {
    for (int32_t j = 0; j < ns; ++j) orc_retract(poses + 12 * (int64_t)j, delta + 6 * (int64_t)j, trial + 12 * (int64_t)j);
    trial_cost = orc_voxel_pass(p, trial, tplanes);
  }
  st->iters += 1;
  st->last_pred = pred;
  st->last_trial_cost = trial_cost;
  st->solve_failed = !ok;
  int accept = ok && pred > 0.0 && trial_cost < st->cost;
  if (accept) {
    double rho = (st->cost - trial_cost) / pred;
    double f = 1.0 - pow(2.0 * rho - 1.0, 3.0);
    st->mu *= (f > 1.0 / 3.0 ? f : 1.0 / 3.0);
    st->nu = 2.0;
    st->last_rho = rho;
    double dc = st->cost - trial_cost;
    st->converged = dc <= cfg->rel_tol * st->cost + cfg->abs_tol;
    st->cost = trial_cost;
    memcpy(poses, trial, sizeof(double) * 12 * (size_t)ns);
    memcpy(planes, tplanes, sizeof(double) * 9 * (size_t)p->n_voxels);
    orc_grad_hess(p, poses, planes, cfg->gauss_newton, g, H);
    st->accepted += 1;
    st->consec_reject = 0;
  } else {
    st->mu *= st->nu;
    st->nu *= 2.0;
    st->last_rho = pred > 0.0 && ok ? (st->cost - trial_cost) / pred : NAN;
    st->consec_reject += 1;
  }
  st->last_accepted = accept;
  free(nobs);
  free(delta);
  free(trial);
  free(tplanes);
  return accept;
}

int orc_lm_solve(const orc_problem* p, const orc_lm_config* cfg, double* poses, double* planes, double* g, double* H,
                 orc_lm_state* st) {
  int n = 0;
  while (st->iters < cfg->max_iters && !st->converged && st->consec_reject < cfg->max_consec_reject) {
    orc_lm_step(p, cfg, poses, planes, g, H, st);
    ++n;
  }
  return n;
}
