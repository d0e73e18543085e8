/*
 * Seeded synthetic planar scenes for LiDAR bundle adjustment (input synthesis
 * only; no bundle-adjustment arithmetic lives here).
 *
 * Scene model (the recipe the synthetic workloads follow):
 *  - ground-truth scan poses: Haar-uniform rotation (normalised Gaussian
 *    quaternion), translation uniform in the box [0,box0]x[0,box1]x[0,box2];
 *  - planar patches (voxels): centre uniform in the box, unit normal uniform
 *    on the sphere, random in-plane basis, side length fixed or log-uniform in
 *    [side_min, side_max]; a fraction degenerate_frac are strips whose second
 *    in-plane width w2 gives variance w2^2/12 = ratio*sigma^2, ratio~U(2,10);
 *  - each voxel is observed by k ~ U{obs_min..obs_max} distinct scans, chosen
 *    uniformly among all scans or, if view_radius > 0, among scans within that
 *    horizontal (xy) distance of the patch centre;
 *  - each observation holds pts_per_obs points uniform on the patch plus
 *    N(0, noise_sigma^2) offsets along the normal, expressed in the scan frame
 *    p = R_gt^T (w - t_gt);
 *  - initial poses: R0 = Exp(phi) R_gt with phi ~ N(0, rot_sigma^2 I) (world-
 *    frame perturbation), t0 = t_gt + N(0, trans_sigma^2 I); scan 0 is left at
 *    ground truth unless perturb_scan0 is set.
 * Poses are 12 doubles: R (row-major, scan -> world) then t.
 */
#ifndef SCENEGEN_H
#define SCENEGEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint64_t seed;
  int32_t n_scans;
  int32_t pts_per_obs;
  int64_t n_voxels;
  int32_t obs_min;
  int32_t obs_max;
  double box[3];
  double side_min;
  double side_max;
  double noise_sigma;
  double rot_sigma_deg;
  double trans_sigma;
  double degenerate_frac;
  double view_radius;
  int32_t perturb_scan0;
  int32_t reserved;
} sg_params;

typedef struct sg_scene sg_scene;

sg_scene* sg_create(const sg_params* params);
void sg_destroy(sg_scene* s);
int64_t sg_n_obs(const sg_scene* s);
int64_t sg_n_points(const sg_scene* s);
/* Any output pointer may be NULL.  plane: n_voxels x 12 (centre, normal, e1,
 * e2); extent: n_voxels x 2. */
void sg_copy(const sg_scene* s, double* pose_gt, double* pose_init, double* plane, double* extent, int64_t* voxel_off,
             int32_t* obs_scan);
/* Raw scan-frame points of observations [obs_begin, obs_end), pts_per_obs
 * each, written as xyz triples to out.  Returns 0, or -1 on a bad range. */
int sg_points(const sg_scene* s, int64_t obs_begin, int64_t obs_end, double* out, int nthreads);

/* Voxel-major observation offsets (n_voxels + 1) of the scene p describes,
 * from the observation-count stream alone, without building the scene.  Only
 * for scenes without a view radius, where a voxel's count does not depend on
 * the scans near it.  Returns n_obs, or -1 for bad parameters or a scene with
 * a view radius. */
int64_t sg_voxel_offsets(const sg_params* p, int64_t* voxel_off);

#ifdef __cplusplus
}
#endif
#endif
