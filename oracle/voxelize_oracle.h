/*
 * CPU oracle of the paper's preprocessing (Sec. IV-B, Algorithm 1): L1
 * voxelisation of raw scans, bottom-up voxel levels (Eq. 5), and voxel
 * selection by the planarity threshold.  TEST INFRASTRUCTURE ONLY: plain,
 * sequential FP64 code used by the tests and the benchmark's baseline, never
 * by the library.
 *
 * Conventions (as in mmba_oracle.h): pose = R row-major then t (scan ->
 * world); clusters are centred (S xx..zz, m, N) in scan coordinates.
 *
 * Output order: voxels by level (1 first), then by integer index (x, then y,
 * then z); the observations of a voxel by scan.  A level-k voxel with index
 * (ix, iy, iz) covers [i d_k, (i + 1) d_k) per axis, d_k = 2^(k-1) d.
 */
#ifndef VOXELIZE_ORACLE_H
#define VOXELIZE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n_voxels;
  int64_t n_obs;
  int64_t* voxel_off; /* n_voxels + 1 */
  int32_t* obs_scan;  /* n_obs */
  double* agg;        /* n_obs x 10, centred, scan coordinates */
  int32_t* level;     /* n_voxels, 1 .. levels */
  int32_t* index;     /* n_voxels x 3 */
} orc_voxels;

/* World point of a scan point: w_a = fma(R_a0, p0, fma(R_a1, p1, fma(R_a2, p2, t_a))). */
void orc_world_point(const double* pose, const double* p, double* w);

/* Points of scan j are scan_point_off[j] .. scan_point_off[j+1]-1 of pts
 * (n x 3).  levels >= 1; tau > 0 keeps voxels with lambda0 < tau * lambda1 of
 * their world covariance at `poses` (tau <= 0 keeps every voxel); voxels with
 * fewer than min_obs observations are dropped.  Returns 0, or -1 if an index
 * leaves [-2^20, 2^20) or memory runs out. */
int orc_voxelize(int32_t n_scans, const int64_t* scan_point_off, const double* pts, const double* poses, double d,
                 int32_t levels, double tau, int32_t min_obs, orc_voxels* out);
void orc_voxels_free(orc_voxels* v);

/* Merge of two centred clusters (the reduction by voxel index of Eq. 4-5):
 * N = Na + Nb, m = ma + (Nb / N)(mb - ma), S = Sa + Sb + (Na Nb / N) dd^T. */
void orc_merge_clusters(const double* a, const double* b, double* out);

#ifdef __cplusplus
}
#endif
#endif
