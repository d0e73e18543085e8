/*
 * CPU oracle for the majorization-minimization (MM) LiDAR bundle-adjustment
 * iteration.  TEST INFRASTRUCTURE ONLY: plain, slow, sequential FP64 code
 * written from the paper's formulation; it is used by the tests, by the smoke
 * check and by the benchmark's CPU-baseline leg, never by the library.
 *
 * Conventions
 *  - Pose (12 doubles): R row-major (scan -> world), then t; q = R p + t.
 *  - Raw point cluster (10 doubles, Eq. 2): P_f = sum p p^T as
 *    (xx, xy, xz, yy, yz, zz), v_f = sum p (x, y, z), N.
 *  - Centred cluster (10 doubles): S = sum (p-m)(p-m)^T as (xx..zz),
 *    m = v_f / N (x, y, z), N.
 *  - Voxel-major CSR: observations of voxel i are voxel_off[i] ..
 *    voxel_off[i+1]-1; obs_scan[o] is the scan of observation o.
 *  - Plane record (9 doubles per voxel): lambda0 <= lambda1 <= lambda2,
 *    u (unit eigenvector of lambda0), c (voxel centroid); d = u^T c.
 *  - Increment (6 doubles): rotation part dphi first, then dt; the update is
 *    R' = Exp(dphi) R, t' = t + dt.
 *  - Per-scan gradient g: 6 doubles; Hessian H: 36 doubles row-major.
 */
#ifndef MMBA_ORACLE_H
#define MMBA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_scans;
  int32_t pad;
  int64_t n_voxels;
  int64_t n_obs;
  const int64_t* voxel_off;
  const int32_t* obs_scan;
  const double* agg; /* centred clusters, n_obs x 10 */
} orc_problem;

/* ---- a0: points -> point clusters (Eq. 2) ------------------------------- */
void orc_points_to_raw(int64_t n_obs, const int64_t* point_off, const double* pts, double* raw);
void orc_points_to_centred(int64_t n_obs, const int64_t* point_off, const double* pts, double* centred);
void orc_raw_to_centred(int64_t n_obs, const double* raw, double* centred);

/* ---- 3x3 symmetric eigen-solve (cyclic Jacobi) -------------------------- */
/* A packed (xx, xy, xz, yy, yz, zz).  lam ascending; V columns are the
 * eigenvectors (V[3*r + c] = component r of eigenvector c).  Returns sweeps. */
int orc_eig3(const double* A, double* lam, double* V);

/* ---- cost, Eq. 1 --------------------------------------------------------- */
/* Brute force from raw points: covariance of each voxel's world points. */
double orc_cost_points(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan,
                       const int64_t* point_off, const double* pts, const double* poses, double* lam0);
/* Eq. 1 with Eq. 2, literally: P_i = sum_j P_ij, v_i = sum_j v_ij from raw
 * clusters, cov = P_i/N_i - v_i v_i^T / N_i^2. */
double orc_cost_eq1(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan, const double* raw,
                    const double* poses, double* lam0);
/* Voxel pass (residual evaluation of Algorithm 2) on centred clusters:
 * returns c(T) and writes the plane record of every voxel. */
double orc_voxel_pass(const orc_problem* p, const double* poses, double* planes);

/* ---- MM surrogate, Eq. 3 ------------------------------------------------- */
/* Eq. 3 as printed, from raw clusters: u is the plane normal of planes_l
 * (the voxel pass at T^(l)) and z = 1/2 sum_j u^T v_ij is evaluated at
 * poses_l. */
double orc_surrogate_eq3(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan, const double* raw,
                         const double* poses, const double* planes_l, const double* poses_l);
/* Fixed-plane form (1/N_i) sum_jk (u^T(R_j p + t_j) - d)^2 from raw points. */
double orc_surrogate_points(int64_t n_voxels, const int64_t* voxel_off, const int32_t* obs_scan,
                            const int64_t* point_off, const double* pts, const double* poses,
                            const double* planes_l);

/* ---- surrogate gradient / Hessian per scan ------------------------------ */
/* gauss_newton != 0 drops the second-order rotation term. */
void orc_grad_hess(const orc_problem* p, const double* poses, const double* planes, int gauss_newton, double* g,
                   double* H);

/* ---- solve and retraction ----------------------------------------------- */
/* LDL^T of a symmetric 6x6 without pivoting; returns 0, or -1 if a pivot is
 * not positive and finite. */
int orc_ldlt6(const double* A, const double* b, double* x);
void orc_exp_so3(const double* phi, double* R);
void orc_retract(const double* pose, const double* delta, double* out);

/* ---- Levenberg-Marquardt on the surrogate ------------------------------- */
typedef struct {
  double mu0;
  double rel_tol;
  double abs_tol;
  int32_t fixed_scan;        /* -1: none */
  int32_t gauss_newton;      /* 0: exact surrogate Hessian */
  int32_t max_iters;
  int32_t max_consec_reject; /* stop after this many rejected steps in a row */
} orc_lm_config;

typedef struct {
  double cost;
  double mu;
  double nu;
  double last_rho;
  double last_pred;
  double last_trial_cost;
  int32_t iters;
  int32_t accepted;
  int32_t consec_reject;
  int32_t last_accepted;
  int32_t converged;
  int32_t solve_failed;
} orc_lm_state;

/* Evaluate planes, cost, g and H at poses and reset mu, nu. */
void orc_lm_init(const orc_problem* p, const orc_lm_config* cfg, const double* poses, double* planes, double* g,
                 double* H, orc_lm_state* st);
/* One LM iteration: per-scan damped solve, retraction, trial voxel pass,
 * accept/reject, damping update; on acceptance poses, planes, g and H move to
 * the new point.  Returns 1 if accepted. */
int orc_lm_step(const orc_problem* p, const orc_lm_config* cfg, double* poses, double* planes, double* g, double* H,
                orc_lm_state* st);
/* Iterate until converged, max_iters or max_consec_reject; returns iterations run. */
int orc_lm_solve(const orc_problem* p, const orc_lm_config* cfg, double* poses, double* planes, double* g, double* H,
                 orc_lm_state* st);

#ifdef __cplusplus
}
#endif
#endif
