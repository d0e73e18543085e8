/*
 * Seeded synthetic planar scenes for LiDAR bundle adjustment.
 *
 * This module only synthesises inputs: ground-truth scan poses, planar
 * patches, which scans observe which patch, raw scan-frame points and the
 * perturbed initial poses.  It contains none of the bundle-adjustment
 * arithmetic (no point-cluster sums, no covariance, no eigen-solve, no
 * derivative); both the CPU oracle and the CUDA library consume what it
 * produces.
 *
 * Randomness is counter based, so any range of observations can be generated
 * independently (and by several threads) with bit-identical results:
 *   value(stream, counter) = mix64(key(stream) + counter * GOLDEN)
 * where mix64 is the SplitMix64 output function (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014).
 */
#include "scenegen.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Stream identifiers: each kind of draw has its own stream so that changing,
 * e.g., the number of points per observation does not move the poses. */
enum {
  ST_POSE_GT = 1,
  ST_POSE_PERTURB = 2,
  ST_PLANE = 3,
  ST_OBS_COUNT = 4,
  ST_OBS_PICK = 5,
  ST_POINTS = 6,
};

typedef struct {
  uint64_t key;
  uint64_t ctr;
} rng_t;

static rng_t rng_make(uint64_t seed, uint64_t stream, uint64_t index) {
  rng_t r;
  r.key = mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + index * GOLDEN);
  r.ctr = 0;
  return r;
}

static uint64_t rng_next(rng_t* r) {
  r->ctr += 1;
  return mix64(r->key + r->ctr * GOLDEN);
}

/* uniform in [0, 1) with 53 random bits */
static double rng_unit(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform in (0, 1] */
static double rng_unit_open0(rng_t* r) { return ((double)(rng_next(r) >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

static double rng_uniform(rng_t* r, double lo, double hi) { return lo + (hi - lo) * rng_unit(r); }

/* standard normal by the Box-Muller transform (one value per call) */
static double rng_normal(rng_t* r) {
  double u1 = rng_unit_open0(r);
  double u2 = rng_unit(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

static int64_t rng_int(rng_t* r, int64_t lo, int64_t hi) /* inclusive */ {
  uint64_t span = (uint64_t)(hi - lo + 1);
  return lo + (int64_t)(rng_next(r) % span);
}

/* ---- small rotation helpers (scene synthesis only) ---------------------- */

/* rotation matrix (row-major) of the unit quaternion (w, x, y, z) */
static void quat_to_mat(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

static void matmul3(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

static void normalize3(double v[3]) {
  double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n;
  v[1] /= n;
  v[2] /= n;
}

static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---- scene -------------------------------------------------------------- */

struct sg_scene {
  sg_params p;
  int64_t n_obs;
  double* pose_gt;   /* n_scans x 12: R row-major, then t (scan -> world) */
  double* pose_init; /* n_scans x 12 */
  double* plane;     /* n_voxels x 12: centre(3) normal(3) e1(3) e2(3) */
  double* extent;    /* n_voxels x 2: in-plane side lengths along e1, e2 */
  int64_t* voxel_off;
  int32_t* obs_scan;
};

static void gen_poses(sg_scene* s) {
  const sg_params* p = &s->p;
  for (int32_t j = 0; j < p->n_scans; ++j) {
    rng_t r = rng_make(p->seed, ST_POSE_GT, (uint64_t)j);
    double q[4] = {rng_normal(&r), rng_normal(&r), rng_normal(&r), rng_normal(&r)};
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) q[k] /= qn; /* Haar-uniform rotation */
    double* G = s->pose_gt + 12 * (int64_t)j;
    quat_to_mat(q, G);
    G[9] = rng_uniform(&r, 0.0, p->box[0]);
    G[10] = rng_uniform(&r, 0.0, p->box[1]);
    G[11] = rng_uniform(&r, 0.0, p->box[2]);

    double* I = s->pose_init + 12 * (int64_t)j;
    memcpy(I, G, 12 * sizeof(double));
    if (j == 0 && !p->perturb_scan0) continue;
    rng_t rp = rng_make(p->seed, ST_POSE_PERTURB, (uint64_t)j);
    double sr = p->rot_sigma_deg * (3.14159265358979323846 / 180.0);
    double phi[3] = {sr * rng_normal(&rp), sr * rng_normal(&rp), sr * rng_normal(&rp)};
    double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    double dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (th > 0.0) {
      double sh = sin(0.5 * th) / th;
      dq[0] = cos(0.5 * th);
      dq[1] = sh * phi[0];
      dq[2] = sh * phi[1];
      dq[3] = sh * phi[2];
    }
    double dR[9];
    quat_to_mat(dq, dR);
    matmul3(dR, G, I); /* initial rotation = (world-frame perturbation) * ground truth */
    I[9] = G[9] + p->trans_sigma * rng_normal(&rp);
    I[10] = G[10] + p->trans_sigma * rng_normal(&rp);
    I[11] = G[11] + p->trans_sigma * rng_normal(&rp);
  }
}

static void gen_planes(sg_scene* s) {
  const sg_params* p = &s->p;
  for (int64_t i = 0; i < p->n_voxels; ++i) {
    rng_t r = rng_make(p->seed, ST_PLANE, (uint64_t)i);
    double* P = s->plane + 12 * i;
    P[0] = rng_uniform(&r, 0.0, p->box[0]);
    P[1] = rng_uniform(&r, 0.0, p->box[1]);
    P[2] = rng_uniform(&r, 0.0, p->box[2]);
    double n[3] = {rng_normal(&r), rng_normal(&r), rng_normal(&r)};
    normalize3(n);
    double a[3] = {rng_normal(&r), rng_normal(&r), rng_normal(&r)};
    double e1[3], e2[3];
    cross3(n, a, e1);
    normalize3(e1);
    cross3(n, e1, e2);
    memcpy(P + 3, n, sizeof n);
    memcpy(P + 6, e1, sizeof e1);
    memcpy(P + 9, e2, sizeof e2);
    double side;
    if (p->side_max > p->side_min)
      side = exp(rng_uniform(&r, log(p->side_min), log(p->side_max)));
    else
      side = p->side_min;
    double w2 = side;
    double u = rng_unit(&r);
    if (u < p->degenerate_frac) {
      /* a strip: its second in-plane variance is ratio * sigma^2, ratio ~ U(2, 10) */
      double ratio = rng_uniform(&r, 2.0, 10.0);
      double sig = p->noise_sigma > 0.0 ? p->noise_sigma : 0.01;
      w2 = sqrt(12.0 * ratio) * sig;
    }
    s->extent[2 * i] = side;
    s->extent[2 * i + 1] = w2;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Pick the observing scans of voxel i (sorted ascending, distinct) and return
 * their count.  cand/ncand: candidate scans (NULL = all scans).  k distinct
 * pool positions are drawn with Floyd's algorithm (R. W. Floyd, "A sample of
 * brilliance", CACM 1987): for t = pool-k .. pool-1 draw r in [0, t] and take
 * r, or t if r was taken already. */
static int32_t pick_scans(const sg_params* p, int64_t i, const int32_t* cand, int32_t ncand, int32_t* out,
                          int32_t* work) {
  (void)work;
  rng_t rc = rng_make(p->seed, ST_OBS_COUNT, (uint64_t)i);
  int32_t k = (int32_t)rng_int(&rc, p->obs_min, p->obs_max);
  int32_t pool = cand ? ncand : p->n_scans;
  if (k > pool) k = pool;
  rng_t rp = rng_make(p->seed, ST_OBS_PICK, (uint64_t)i);
  int32_t n = 0;
  for (int32_t t = pool - k; t < pool; ++t) {
    int32_t r = (int32_t)rng_int(&rp, 0, t);
    int taken = 0;
    for (int32_t q = 0; q < n; ++q)
      if (out[q] == r) {
        taken = 1;
        break;
      }
    out[n++] = taken ? t : r;
  }
  for (int32_t q = 0; q < n; ++q) out[q] = cand ? cand[out[q]] : out[q];
  qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
  return k;
}

sg_scene* sg_create(const sg_params* params) {
  sg_scene* s = (sg_scene*)calloc(1, sizeof(sg_scene));
  if (!s) return NULL;
  s->p = *params;
  const sg_params* p = &s->p;
  if (p->n_scans < 1 || p->n_voxels < 0 || p->obs_min < 1 || p->obs_max < p->obs_min) {
    free(s);
    return NULL;
  }
  s->pose_gt = (double*)malloc(sizeof(double) * 12 * (size_t)p->n_scans);
  s->pose_init = (double*)malloc(sizeof(double) * 12 * (size_t)p->n_scans);
  s->plane = (double*)malloc(sizeof(double) * 12 * (size_t)(p->n_voxels + 1));
  s->extent = (double*)malloc(sizeof(double) * 2 * (size_t)(p->n_voxels + 1));
  s->voxel_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(p->n_voxels + 1));
  gen_poses(s);
  gen_planes(s);

  /* candidate scans: all scans, or those within view_radius (xy distance) */
  int32_t* work = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->n_scans);
  int32_t* cand = NULL;
  int32_t* pick = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->n_scans);
  /* grid over xy for radius queries */
  int32_t gx = 1, gy = 1;
  int32_t *cell_off = NULL, *cell_scan = NULL;
  if (p->view_radius > 0.0) {
    cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->n_scans);
    gx = (int32_t)ceil(p->box[0] / p->view_radius);
    gy = (int32_t)ceil(p->box[1] / p->view_radius);
    if (gx < 1) gx = 1;
    if (gy < 1) gy = 1;
    cell_off = (int32_t*)calloc((size_t)gx * gy + 1, sizeof(int32_t));
    cell_scan = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->n_scans);
    int32_t* fill = (int32_t*)calloc((size_t)gx * gy, sizeof(int32_t));
    for (int32_t j = 0; j < p->n_scans; ++j) {
      const double* t = s->pose_gt + 12 * (int64_t)j + 9;
      int32_t cx = (int32_t)(t[0] / p->view_radius), cy = (int32_t)(t[1] / p->view_radius);
      cx = cx < 0 ? 0 : (cx >= gx ? gx - 1 : cx);
      cy = cy < 0 ? 0 : (cy >= gy ? gy - 1 : cy);
      cell_off[cy * gx + cx + 1]++;
    }
    for (int32_t c = 0; c < gx * gy; ++c) cell_off[c + 1] += cell_off[c];
    for (int32_t j = 0; j < p->n_scans; ++j) {
      const double* t = s->pose_gt + 12 * (int64_t)j + 9;
      int32_t cx = (int32_t)(t[0] / p->view_radius), cy = (int32_t)(t[1] / p->view_radius);
      cx = cx < 0 ? 0 : (cx >= gx ? gx - 1 : cx);
      cy = cy < 0 ? 0 : (cy >= gy ? gy - 1 : cy);
      int32_t c = cy * gx + cx;
      cell_scan[cell_off[c] + fill[c]++] = j; /* scans in ascending order per cell */
    }
    free(fill);
  }

  /* two passes: count, then fill */
  int64_t cap = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int64_t n = 0;
    s->voxel_off[0] = 0;
    for (int64_t i = 0; i < p->n_voxels; ++i) {
      const int32_t* cptr = NULL;
      int32_t nc = 0;
      if (cand) {
        const double* c = s->plane + 12 * i;
        int32_t cx = (int32_t)(c[0] / p->view_radius), cy = (int32_t)(c[1] / p->view_radius);
        for (int32_t yy = cy - 1; yy <= cy + 1; ++yy)
          for (int32_t xx = cx - 1; xx <= cx + 1; ++xx) {
            if (xx < 0 || yy < 0 || xx >= gx || yy >= gy) continue;
            int32_t cc = yy * gx + xx;
            for (int32_t q = cell_off[cc]; q < cell_off[cc + 1]; ++q) {
              int32_t j = cell_scan[q];
              const double* t = s->pose_gt + 12 * (int64_t)j + 9;
              double dx = t[0] - c[0], dy = t[1] - c[1];
              if (dx * dx + dy * dy <= p->view_radius * p->view_radius) cand[nc++] = j;
            }
          }
        cptr = cand;
        if (nc == 0) { /* no scan in range: fall back to scan nearest the centre */
          double best = 1e300;
          int32_t bj = 0;
          for (int32_t j = 0; j < p->n_scans; ++j) {
            const double* t = s->pose_gt + 12 * (int64_t)j + 9;
            double dx = t[0] - c[0], dy = t[1] - c[1];
            if (dx * dx + dy * dy < best) best = dx * dx + dy * dy, bj = j;
          }
          cand[0] = bj;
          nc = 1;
        }
      }
      int32_t k = pick_scans(p, i, cptr, nc, pick, work);
      if (pass == 1)
        for (int32_t t = 0; t < k; ++t) s->obs_scan[n + t] = pick[t];
      n += k;
      s->voxel_off[i + 1] = n;
    }
    if (pass == 0) {
      cap = n;
      s->obs_scan = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    }
  }
  s->n_obs = cap;
  free(work);
  free(pick);
  free(cand);
  free(cell_off);
  free(cell_scan);
  return s;
}

int64_t sg_voxel_offsets(const sg_params* p, int64_t* voxel_off) {
  if (!p || !voxel_off || p->n_scans < 1 || p->n_voxels < 0 || p->obs_min < 1 || p->obs_max < p->obs_min ||
      p->view_radius > 0.0)
    return -1;
  int64_t n = 0;
  voxel_off[0] = 0;
  for (int64_t i = 0; i < p->n_voxels; ++i) {
    rng_t rc = rng_make(p->seed, ST_OBS_COUNT, (uint64_t)i);
    int64_t k = rng_int(&rc, p->obs_min, p->obs_max);
    if (k > p->n_scans) k = p->n_scans;
    n += k;
    voxel_off[i + 1] = n;
  }
  return n;
}

void sg_destroy(sg_scene* s) {
  if (!s) return;
  free(s->pose_gt);
  free(s->pose_init);
  free(s->plane);
  free(s->extent);
  free(s->voxel_off);
  free(s->obs_scan);
  free(s);
}

int64_t sg_n_obs(const sg_scene* s) { return s->n_obs; }

int64_t sg_n_points(const sg_scene* s) { return s->n_obs * (int64_t)s->p.pts_per_obs; }

void sg_copy(const sg_scene* s, double* pose_gt, double* pose_init, double* plane, double* extent, int64_t* voxel_off,
             int32_t* obs_scan) {
  const sg_params* p = &s->p;
  if (pose_gt) memcpy(pose_gt, s->pose_gt, sizeof(double) * 12 * (size_t)p->n_scans);
  if (pose_init) memcpy(pose_init, s->pose_init, sizeof(double) * 12 * (size_t)p->n_scans);
  if (plane) memcpy(plane, s->plane, sizeof(double) * 12 * (size_t)p->n_voxels);
  if (extent) memcpy(extent, s->extent, sizeof(double) * 2 * (size_t)p->n_voxels);
  if (voxel_off) memcpy(voxel_off, s->voxel_off, sizeof(int64_t) * (size_t)(p->n_voxels + 1));
  if (obs_scan) memcpy(obs_scan, s->obs_scan, sizeof(int32_t) * (size_t)s->n_obs);
}

/* voxel of each observation, by bisection on voxel_off */
static int64_t voxel_of(const sg_scene* s, int64_t o) {
  int64_t lo = 0, hi = s->p.n_voxels; /* voxel_off[lo] <= o < voxel_off[hi] */
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) / 2;
    if (s->voxel_off[mid] <= o)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

static void gen_points_range(const sg_scene* s, int64_t o0, int64_t o1, double* out /* points of obs o0.. */) {
  const sg_params* p = &s->p;
  int64_t npo = p->pts_per_obs;
  int64_t v = o0 < o1 ? voxel_of(s, o0) : 0;
  for (int64_t o = o0; o < o1; ++o) {
    while (s->voxel_off[v + 1] <= o) ++v;
    const double* P = s->plane + 12 * v;
    const double* c = P;
    const double* n = P + 3;
    const double* e1 = P + 6;
    const double* e2 = P + 9;
    double s1 = s->extent[2 * v], s2 = s->extent[2 * v + 1];
    const double* G = s->pose_gt + 12 * (int64_t)s->obs_scan[o];
    rng_t r = rng_make(p->seed, ST_POINTS, (uint64_t)o);
    double* dst = out + 3 * (o - o0) * npo;
    for (int64_t k = 0; k < npo; ++k) {
      double a = rng_uniform(&r, -0.5 * s1, 0.5 * s1);
      double b = rng_uniform(&r, -0.5 * s2, 0.5 * s2);
      double eps = p->noise_sigma > 0.0 ? p->noise_sigma * rng_normal(&r) : 0.0;
      double w[3];
      for (int d = 0; d < 3; ++d) w[d] = c[d] + a * e1[d] + b * e2[d] + eps * n[d] - G[9 + d];
      /* scan frame: R^T (w - t) */
      for (int d = 0; d < 3; ++d) dst[3 * k + d] = G[d] * w[0] + G[3 + d] * w[1] + G[6 + d] * w[2];
    }
  }
}

typedef struct {
  const sg_scene* s;
  int64_t o0, o1, base;
  double* out;
} job_t;

static void* job_run(void* arg) {
  job_t* j = (job_t*)arg;
  gen_points_range(j->s, j->o0, j->o1, j->out + 3 * (j->o0 - j->base) * j->s->p.pts_per_obs);
  return NULL;
}

int sg_points(const sg_scene* s, int64_t obs_begin, int64_t obs_end, double* out, int nthreads) {
  if (obs_begin < 0 || obs_end > s->n_obs || obs_begin > obs_end) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  int64_t n = obs_end - obs_begin;
  if (nthreads == 1 || n < 4096) {
    gen_points_range(s, obs_begin, obs_end, out);
    return 0;
  }
  pthread_t th[256];
  job_t jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].s = s;
    jobs[t].o0 = obs_begin + n * t / nthreads;
    jobs[t].o1 = obs_begin + n * (t + 1) / nthreads;
    jobs[t].base = obs_begin;
    jobs[t].out = out;
    pthread_create(&th[t], NULL, job_run, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}
