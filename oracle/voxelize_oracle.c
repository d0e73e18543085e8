/*
 * CPU oracle of the paper's preprocessing (Sec. IV-B, Algorithm 1).
 * TEST INFRASTRUCTURE ONLY (see voxelize_oracle.h).
 *
 *   L1 voxelisation (Sec. IV-B-1, Eq. 4): every point to world coordinates,
 *     integer index floor(w / d) per axis, one centred cluster per
 *     (voxel, scan) from that scan's points in the voxel (Eq. 2).
 *   Bottom-up levels (Sec. IV-B-2, Eq. 5, Algorithm 1 BottomUpVoxelization):
 *     the level-k index of a level-(k-1) cluster is floor(index / 2); the
 *     clusters with the same (level-k index, scan) are merged.
 *   Selection (Sec. IV-B-3, Algorithm 1 Selection): the clusters of a voxel
 *     are taken to world coordinates at the given poses (Eq. 2) and combined;
 *     the voxel is kept if lambda0 < tau * lambda1 of its covariance.
 */
#include "voxelize_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "mmba_oracle.h"

void orc_world_point(const double* T, const double* p, double* w) {
  for (int a = 0; a < 3; ++a) w[a] = fma(T[3 * a], p[0], fma(T[3 * a + 1], p[1], fma(T[3 * a + 2], p[2], T[9 + a])));
}

void orc_merge_clusters(const double* a, const double* b, double* out) {
  const double na = a[9], nb = b[9], n = na + nb;
  const double d[3] = {b[6] - a[6], b[7] - a[7], b[8] - a[8]};
  const double f = na * nb / n;
  double r[10];
  int idx = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      r[idx] = a[idx] + b[idx] + f * d[i] * d[j];
      ++idx;
    }
  for (int i = 0; i < 3; ++i) r[6 + i] = a[6 + i] + (nb / n) * d[i];
  r[9] = n;
  memcpy(out, r, sizeof r);
}

/* floor(i / 2) for signed integers */
static int64_t half_floor(int64_t i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

typedef struct {
  int64_t ix, iy, iz;
  int32_t scan;
  int64_t item; /* point index (level 1) or child cluster index (higher levels) */
} rec;

static int rec_cmp(const void* pa, const void* pb) {
  const rec* a = (const rec*)pa;
  const rec* b = (const rec*)pb;
  if (a->ix != b->ix) return a->ix < b->ix ? -1 : 1;
  if (a->iy != b->iy) return a->iy < b->iy ? -1 : 1;
  if (a->iz != b->iz) return a->iz < b->iz ? -1 : 1;
  if (a->scan != b->scan) return a->scan < b->scan ? -1 : 1;
  if (a->item != b->item) return a->item < b->item ? -1 : 1;
  return 0;
}

static int same_key(const rec* a, const rec* b) {
  return a->ix == b->ix && a->iy == b->iy && a->iz == b->iz && a->scan == b->scan;
}

typedef struct {
  int64_t n;
  int64_t* ix; /* n x 3 */
  int32_t* scan;
  double* c; /* n x 10 */
} level_set;

static void level_free(level_set* s) {
  free(s->ix);
  free(s->scan);
  free(s->c);
  memset(s, 0, sizeof *s);
}

static int level_alloc(level_set* s, int64_t n) {
  s->n = n;
  s->ix = (int64_t*)malloc(sizeof(int64_t) * 3 * (n ? n : 1));
  s->scan = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
  s->c = (double*)malloc(sizeof(double) * 10 * (n ? n : 1));
  return s->ix && s->scan && s->c ? 0 : -1;
}

static const int64_t kRange = (int64_t)1 << 20;

int orc_voxelize(int32_t n_scans, const int64_t* scan_point_off, const double* pts, const double* poses, double d,
                 int32_t levels, double tau, int32_t min_obs, orc_voxels* out) {
  memset(out, 0, sizeof *out);
  if (levels < 1 || !(d > 0.0)) return -1;
  const int64_t n_pts = scan_point_off[n_scans];
  level_set* lv = (level_set*)calloc((size_t)levels, sizeof(level_set));
  rec* r = (rec*)malloc(sizeof(rec) * (n_pts ? n_pts : 1));
  if (!lv || !r) return -1;
  int status = 0;

  /* ---- level 1: points -> (voxel, scan) clusters ---- */
  for (int32_t j = 0; j < n_scans && !status; ++j)
    for (int64_t k = scan_point_off[j]; k < scan_point_off[j + 1]; ++k) {
      double w[3];
      orc_world_point(poses + 12 * (int64_t)j, pts + 3 * k, w);
      const double fx = floor(w[0] / d), fy = floor(w[1] / d), fz = floor(w[2] / d);
      const double lo = -(double)kRange, hi = (double)kRange;
      if (!(fx >= lo && fx < hi && fy >= lo && fy < hi && fz >= lo && fz < hi)) {
        status = -1;
        break;
      }
      r[k].ix = (int64_t)fx;
      r[k].iy = (int64_t)fy;
      r[k].iz = (int64_t)fz;
      r[k].scan = j;
      r[k].item = k;
    }
  if (!status) qsort(r, (size_t)n_pts, sizeof(rec), rec_cmp);
  int64_t n1 = 0;
  for (int64_t k = 0; k < n_pts && !status; ++k)
    if (k == 0 || !same_key(&r[k], &r[k - 1])) ++n1;
  if (!status && level_alloc(&lv[0], n1)) status = -1;
  for (int64_t k = 0, c = 0; k < n_pts && !status;) {
    int64_t e = k + 1;
    while (e < n_pts && same_key(&r[e], &r[k])) ++e;
    /* centred cluster of the group's points, in point order (Eq. 2) */
    double s[3] = {0, 0, 0};
    for (int64_t q = k; q < e; ++q)
      for (int a = 0; a < 3; ++a) s[a] += pts[3 * r[q].item + a];
    const double n = (double)(e - k);
    const double m[3] = {s[0] / n, s[1] / n, s[2] / n};
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t q = k; q < e; ++q) {
      const double* p = pts + 3 * r[q].item;
      const double x = p[0] - m[0], y = p[1] - m[1], z = p[2] - m[2];
      S[0] += x * x;
      S[1] += x * y;
      S[2] += x * z;
      S[3] += y * y;
      S[4] += y * z;
      S[5] += z * z;
    }
    double* cc = lv[0].c + 10 * c;
    for (int a = 0; a < 6; ++a) cc[a] = S[a];
    for (int a = 0; a < 3; ++a) cc[6 + a] = m[a];
    cc[9] = n;
    lv[0].ix[3 * c] = r[k].ix;
    lv[0].ix[3 * c + 1] = r[k].iy;
    lv[0].ix[3 * c + 2] = r[k].iz;
    lv[0].scan[c] = r[k].scan;
    ++c;
    k = e;
  }
  free(r);

  /* ---- levels 2..L: parent index, then merge by (parent, scan) ---- */
  for (int32_t L = 1; L < levels && !status; ++L) {
    const level_set* ch = &lv[L - 1];
    rec* q = (rec*)malloc(sizeof(rec) * (ch->n ? ch->n : 1));
    if (!q) {
      status = -1;
      break;
    }
    for (int64_t i = 0; i < ch->n; ++i) {
      q[i].ix = half_floor(ch->ix[3 * i]);
      q[i].iy = half_floor(ch->ix[3 * i + 1]);
      q[i].iz = half_floor(ch->ix[3 * i + 2]);
      q[i].scan = ch->scan[i];
      q[i].item = i;
    }
    qsort(q, (size_t)ch->n, sizeof(rec), rec_cmp);
    int64_t np = 0;
    for (int64_t i = 0; i < ch->n; ++i)
      if (i == 0 || !same_key(&q[i], &q[i - 1])) ++np;
    if (level_alloc(&lv[L], np)) {
      free(q);
      status = -1;
      break;
    }
    for (int64_t i = 0, c = 0; i < ch->n;) {
      int64_t e = i + 1;
      while (e < ch->n && same_key(&q[e], &q[i])) ++e;
      double acc[10];
      memcpy(acc, ch->c + 10 * q[i].item, sizeof acc);
      for (int64_t t = i + 1; t < e; ++t) orc_merge_clusters(acc, ch->c + 10 * q[t].item, acc);
      memcpy(lv[L].c + 10 * c, acc, sizeof acc);
      lv[L].ix[3 * c] = q[i].ix;
      lv[L].ix[3 * c + 1] = q[i].iy;
      lv[L].ix[3 * c + 2] = q[i].iz;
      lv[L].scan[c] = q[i].scan;
      ++c;
      i = e;
    }
    free(q);
  }

  /* ---- voxels of all levels (clusters are sorted by index, then scan), selection ---- */
  int64_t nv_all = 0, no_all = 0;
  for (int32_t L = 0; L < levels && !status; ++L) {
    no_all += lv[L].n;
    for (int64_t i = 0; i < lv[L].n; ++i)
      if (i == 0 || memcmp(lv[L].ix + 3 * i, lv[L].ix + 3 * (i - 1), 3 * sizeof(int64_t)) != 0) ++nv_all;
  }
  if (!status) {
    out->voxel_off = (int64_t*)malloc(sizeof(int64_t) * (nv_all + 1));
    out->obs_scan = (int32_t*)malloc(sizeof(int32_t) * (no_all ? no_all : 1));
    out->agg = (double*)malloc(sizeof(double) * 10 * (no_all ? no_all : 1));
    out->level = (int32_t*)malloc(sizeof(int32_t) * (nv_all ? nv_all : 1));
    out->index = (int32_t*)malloc(sizeof(int32_t) * 3 * (nv_all ? nv_all : 1));
    if (!out->voxel_off || !out->obs_scan || !out->agg || !out->level || !out->index) status = -1;
  }
  int64_t nv = 0, no = 0;
  if (!status) out->voxel_off[0] = 0;
  for (int32_t L = 0; L < levels && !status; ++L) {
    const level_set* s = &lv[L];
    for (int64_t i = 0; i < s->n;) {
      int64_t e = i + 1;
      while (e < s->n && memcmp(s->ix + 3 * e, s->ix + 3 * i, 3 * sizeof(int64_t)) == 0) ++e;
      int keep = (e - i) >= (int64_t)min_obs;
      if (keep && tau > 0.0) {
        /* world covariance of the voxel at the poses (Eq. 1-2), centred form */
        double n = 0.0, c[3] = {0, 0, 0};
        for (int64_t t = i; t < e; ++t) {
          const double* cl = s->c + 10 * t;
          double w[3];
          orc_world_point(poses + 12 * (int64_t)s->scan[t], cl + 6, w);
          for (int a = 0; a < 3; ++a) c[a] += cl[9] * w[a];
          n += cl[9];
        }
        for (int a = 0; a < 3; ++a) c[a] /= n;
        double A[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t t = i; t < e; ++t) {
          const double* cl = s->c + 10 * t;
          const double* R = poses + 12 * (int64_t)s->scan[t];
          double w[3];
          orc_world_point(R, cl + 6, w);
          const double dd[3] = {w[0] - c[0], w[1] - c[1], w[2] - c[2]};
          const double Sm[3][3] = {{cl[0], cl[1], cl[2]}, {cl[1], cl[3], cl[4]}, {cl[2], cl[4], cl[5]}};
          double RS[3][3];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) RS[a][b] = R[3 * a] * Sm[0][b] + R[3 * a + 1] * Sm[1][b] + R[3 * a + 2] * Sm[2][b];
          int idx = 0;
          for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) {
              const double rsr = RS[a][0] * R[3 * b] + RS[a][1] * R[3 * b + 1] + RS[a][2] * R[3 * b + 2];
              A[idx++] += rsr + cl[9] * dd[a] * dd[b];
            }
        }
        for (int a = 0; a < 6; ++a) A[a] /= n;
        double lam[3], V[9];
        orc_eig3(A, lam, V);
        keep = lam[0] < tau * lam[1];
      }
      if (keep) {
        for (int64_t t = i; t < e; ++t) {
          out->obs_scan[no] = s->scan[t];
          memcpy(out->agg + 10 * no, s->c + 10 * t, 10 * sizeof(double));
          ++no;
        }
        out->level[nv] = L + 1;
        for (int a = 0; a < 3; ++a) out->index[3 * nv + a] = (int32_t)s->ix[3 * i + a];
        ++nv;
        out->voxel_off[nv] = no;
      }
      i = e;
    }
  }
  for (int32_t L = 0; L < levels; ++L) level_free(&lv[L]);
  free(lv);
  if (status) {
    orc_voxels_free(out);
    return status;
  }
  out->n_voxels = nv;
  out->n_obs = no;
  return 0;
}

void orc_voxels_free(orc_voxels* v) {
  free(v->voxel_off);
  free(v->obs_scan);
  free(v->agg);
  free(v->level);
  free(v->index);
  memset(v, 0, sizeof *v);
}
