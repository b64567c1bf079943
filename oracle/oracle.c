/*
 * FP64 CPU oracle for the ARTEMIS neural-animal rendering path
 * (arXiv 2202.05628, Sec. 3.1).  TEST INFRASTRUCTURE ONLY: it is called by
 * the tests, by __graft_entry__.smoke() and by the CPU-baseline leg of the
 * benchmark, never by the product path.  It shares no code with the CUDA
 * library.
 *
 * Plain, slow, direct evaluation of:
 *   - forward kinematics of the skeleton S = {r, R, T}        (Sec. 3.1, Eq. 4)
 *   - linear blend skinning A_i = sum_k w_ik M^t_j (M^c_j)^-1  (Eq. 4)
 *   - pinhole rays through pixel centres                     (Sec. 3.1, "Dynamic Volume Rendering")
 *   - exact ray / warped-voxel intersection, chord delta_i    (Eq. 6, "distance of the ray travelling through a voxel")
 *   - front-to-back compositing F = sum_i T_i (1 - exp(-sigma_i delta_i)) f_i,
 *     T_i = exp(-sum_{j<i} sigma_j delta_j), A = 1 - T_final,
 *     early stop once T < tau                                  (Eq. 5, Eq. 6, early-stop paragraph)
 *   - direct convolutions of the shading network              (Sec. 3.1, "Neural Shading")
 *   - the depth buffer: entry distance of the first voxel along a ray denser
 *     than a threshold                                          (Sec. 3.1, "Hybrid Rendering")
 *   - view-dependent features: spherical-harmonics coefficients evaluated at
 *     the ray direction in the voxel's canonical frame          (Eq. 2, Sec. 3.1)
 *   - the paper's own per-frame index: warped voxel centres snapped to the
 *     lattice of the canonical leaves, collisions resolved, the query Q of
 *     the voxel regularisation term, and the render of the occupied cells
 *                                                              (Sec. 3.1, "Dynamic Volume Rendering", "Training")
 *   - the learned ray-interval proposal's labels, the composite restricted to
 *     a depth interval with the exact transmittance mass it loses, and the
 *     coarse optical-depth bound per screen tile and depth bin (project
 *     addition; the paper's nearest passage is the early-stop rule)
 *   - the analytic gradient of the composite with respect to features,
 *     densities and the blended transforms, of LBS with respect to the
 *     skinning weights, and of the view-dependent feature map with respect
 *     to the SH coefficients (project addition; the paper trains end to end).
 *
 * Readings where the paper is silent or garbled:
 *   - T_i uses the exclusive sum j < i (Eq. 6 prints j <= i; with j < i the
 *     accumulated alpha equals 1 - T_final, which is how the coarse opacity
 *     map is defined).
 *   - the warped voxel is the parallelepiped A_i * (canonical cube); the ray is
 *     mapped into the canonical frame by A_i^-1 (not renormalised, so the ray
 *     parameter t is preserved) and slab-tested against the cube.
 *   - hits are ordered by (t0, t1, voxel id); the stop test follows each hit.
 *   - the depth buffer's voxel (the nearest along the ray denser than the
 *     threshold) is the first such hit in that order among all of the ray's
 *     hits in [near, far] (the early stop does not cut the search), its depth
 *     the entry distance t0 from the camera centre along the unit ray, +inf
 *     where the ray meets no such voxel.
 *   - Eq. 2's spherical harmonics are the real orthonormal ones (without the
 *     Condon-Shortley phase in the real basis), indexed h = l^2 + l + m; the
 *     paper's 91 bases is not a square (l <= 8 gives 81, l <= 9 gives 100):
 *     the degree is a parameter (<= 9).  The rotation R_i^t that maps a ray
 *     into voxel i's canonical frame is read, for a blend of joint
 *     transforms (not a rotation), as the rotation factor of the polar
 *     decomposition of its linear part.
 *   - a voxel whose blended linear part has det < 1e-3, or any of whose eight
 *     warped corners has camera z <= 1e-6, is not rendered.
 *   - the per-frame index is the lattice of the canonical octree's leaves
 *     (same origin and leaf size, unbounded); a voxel goes to the cell
 *     holding its warped centre; of the voxels that collide in one cell the
 *     smallest id survives (the paper says features are overwritten, not
 *     which); a ray composites the occupied cells it crosses, each an
 *     axis-aligned leaf box with its survivor's feature and density.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_DET_MIN 1e-3
#define ORC_Z_MIN 1e-6

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Small matrix helpers (row-major 3x3 and 3x4).                              */
/* ------------------------------------------------------------------------ */

/* Rodrigues' formula R = I + sin(th) K + (1 - cos(th)) K^2, K = [axis]_x. */
void orc_rodrigues(const double r[3], double R[9]) {
  double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  memset(R, 0, 9 * sizeof(double));
  R[0] = R[4] = R[8] = 1.0;
  if (th == 0.0) return;
  double k[3] = {r[0] / th, r[1] / th, r[2] / th};
  double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int m = 0; m < 3; ++m) s += K[i * 3 + m] * K[m * 3 + j];
      K2[i * 3 + j] = s;
    }
  double s = sin(th), c = 1.0 - cos(th);
  for (int i = 0; i < 9; ++i) R[i] += s * K[i] + c * K2[i];
}

/* C = A * B for 3x4 affine matrices (implicit bottom row 0 0 0 1). */
static void affine_mul(const double A[12], const double B[12], double C[12]) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 4; ++j) {
      double s = (j == 3) ? A[i * 4 + 3] : 0.0;
      for (int m = 0; m < 3; ++m) s += A[i * 4 + m] * B[m * 4 + j];
      C[i * 4 + j] = s;
    }
  }
}

static double det3(const double* A, int ld) {
  /* determinant of the 3x3 block of a matrix with leading dimension ld */
  return A[0] * (A[ld + 1] * A[2 * ld + 2] - A[ld + 2] * A[2 * ld + 1]) -
         A[1] * (A[ld] * A[2 * ld + 2] - A[ld + 2] * A[2 * ld]) +
         A[2] * (A[ld] * A[2 * ld + 1] - A[ld + 1] * A[2 * ld]);
}

/* Inverse of a 3x4 affine matrix via the adjugate of its 3x3 block. */
static int affine_inv(const double A[12], double Ai[12]) {
  double d = det3(A, 4);
  if (d == 0.0) return 0;
  double a = A[0], b = A[1], c = A[2];
  double e = A[4], f = A[5], g = A[6];
  double h = A[8], i = A[9], k = A[10];
  double inv[9] = {(f * k - g * i), -(b * k - c * i), (b * g - c * f),
                   -(e * k - g * h), (a * k - c * h), -(a * g - c * e),
                   (e * i - f * h), -(a * i - b * h), (a * f - b * e)};
  for (int r = 0; r < 3; ++r) {
    for (int s = 0; s < 3; ++s) Ai[r * 4 + s] = inv[r * 3 + s] / d;
    Ai[r * 4 + 3] = -(Ai[r * 4 + 0] * A[3] + Ai[r * 4 + 1] * A[7] + Ai[r * 4 + 2] * A[11]);
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Forward kinematics and LBS (Eq. 4).                                        */
/* ------------------------------------------------------------------------ */

/*
 * Skeleton S = {r, R, T}: joint j has local transform [Rod(r_j) | rest_j -
 * rest_parent] (root: [Rod(r_0) | rest_0], premultiplied by the global
 * [Rod(R) | T]).  M^t_j = M^t_parent * local_j; canonical M^c_j = [I | rest_j]
 * (zero joint rotations).  Output G_j = M^t_j (M^c_j)^-1 as 3x4 row-major.
 * Requires parent[j] < j.  Returns 0 on success, -1 on a bad parent array.
 */
int orc_fk(int J, const int32_t* parent, const double* rest, const double* axis_angle,
           const double Rg[3], const double T[3], double* G) {
  double* M = (double*)malloc(sizeof(double) * 12 * (size_t)J);
  if (!M) return -2;
  double glob[12], Rm[9];
  orc_rodrigues(Rg, Rm);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) glob[i * 4 + j] = Rm[i * 3 + j];
    glob[i * 4 + 3] = T[i];
  }
  for (int j = 0; j < J; ++j) {
    int p = parent[j];
    if (p >= j || (p < 0 && p != -1) || (j > 0 && p < 0) || (j == 0 && p != -1)) {
      free(M);
      return -1;
    }
    double local[12];
    orc_rodrigues(axis_angle + 3 * j, Rm);
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) local[a * 4 + b] = Rm[a * 3 + b];
      local[a * 4 + 3] = rest[3 * j + a] - (p >= 0 ? rest[3 * p + a] : 0.0);
    }
    affine_mul(p >= 0 ? M + 12 * p : glob, local, M + 12 * j);
    /* G_j = M^t_j [I | -rest_j] */
    double Minv_c[12] = {1, 0, 0, -rest[3 * j], 0, 1, 0, -rest[3 * j + 1], 0, 0, 1, -rest[3 * j + 2]};
    affine_mul(M + 12 * j, Minv_c, G + 12 * j);
  }
  free(M);
  return 0;
}

/* A_i = sum_{k<4} w_ik G_{j_ik} (not re-orthonormalised); det of its 3x3 block. */
void orc_lbs(int64_t n, int J, const double* G, const uint8_t* jidx, const double* w, double* A,
             double* det) {
  for (int64_t i = 0; i < n; ++i) {
    double* a = A + 12 * i;
    for (int m = 0; m < 12; ++m) a[m] = 0.0;
    for (int k = 0; k < 4; ++k) {
      int j = jidx[4 * i + k];
      double wk = w[4 * i + k];
      if (j >= J) j = J - 1; /* callers validate; keep the oracle memory-safe */
      for (int m = 0; m < 12; ++m) a[m] += wk * G[12 * j + m];
    }
    if (det) det[i] = det3(a, 4);
  }
}

/* ------------------------------------------------------------------------ */
/* Camera rays and the ray / warped-voxel hit.                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int W, H;
  double fx, fy, cx, cy;
  double w2c[12];
  double near_, far_;
} orc_cam;

/* Ray through the centre of pixel (x, y): origin o = -R^T t (camera centre)
 * and direction d = R^T dc / |R^T dc| with dc = ((x+1/2-cx)/fx, (y+1/2-cy)/fy, 1).
 * d is normalised after the rotation so that it is a unit vector even when R
 * is not exactly orthonormal (e.g. stored in FP32); t is then a distance. */
static void cam_ray(const orc_cam* c, int x, int y, double o[3], double d[3]) {
  double dc[3] = {((double)x + 0.5 - c->cx) / c->fx, ((double)y + 0.5 - c->cy) / c->fy, 1.0};
  for (int a = 0; a < 3; ++a) {
    d[a] = c->w2c[0 * 4 + a] * dc[0] + c->w2c[1 * 4 + a] * dc[1] + c->w2c[2 * 4 + a] * dc[2];
    o[a] = -(c->w2c[0 * 4 + a] * c->w2c[3] + c->w2c[1 * 4 + a] * c->w2c[7] +
             c->w2c[2 * 4 + a] * c->w2c[11]);
  }
  double nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int a = 0; a < 3; ++a) d[a] /= nrm;
}

void orc_pixel_ray(const orc_cam* c, int x, int y, double* o, double* d) { cam_ray(c, x, y, o, d); }

/* Unit directions of every pixel's ray, d [H*W][3] (row-major pixels). */
void orc_ray_dirs(const orc_cam* c, double* d) {
  double o[3];
  for (int y = 0; y < c->H; ++y)
    for (int x = 0; x < c->W; ++x) cam_ray(c, x, y, o, d + 3 * ((size_t)y * c->W + x));
}

/*
 * Slab test of the ray (o, d) against the canonical cube [lo, lo + h]^3 after
 * mapping the ray into the canonical frame with Ainv (world -> canonical).
 * t is the world ray parameter (distance, since |d| = 1).  The interval is
 * clipped to [near, far]; a hit needs t1 > t0.  On a hit, the entry/exit
 * planes are returned as axis*2 + side (side 0 = lo, 1 = hi) or -1 for a
 * near/far clip.
 */
static int hit_voxel(const double Ainv[12], const double lo[3], double h, const double o[3],
                     const double d[3], double tnear, double tfar, double* t0, double* t1,
                     int* p0, int* p1) {
  double a0 = tnear, a1 = tfar;
  int q0 = -1, q1 = -1;
  for (int a = 0; a < 3; ++a) {
    double oa = Ainv[a * 4 + 0] * o[0] + Ainv[a * 4 + 1] * o[1] + Ainv[a * 4 + 2] * o[2] + Ainv[a * 4 + 3];
    double da = Ainv[a * 4 + 0] * d[0] + Ainv[a * 4 + 1] * d[1] + Ainv[a * 4 + 2] * d[2];
    double pl = lo[a], ph = lo[a] + h;
    if (da == 0.0) {
      if (oa < pl || oa > ph) return 0;
      continue;
    }
    double ta = (pl - oa) / da, tb = (ph - oa) / da;
    int sa = 0, sb = 1;
    if (ta > tb) {
      double tt = ta; ta = tb; tb = tt;
      sa = 1; sb = 0;
    }
    if (ta > a0) { a0 = ta; q0 = 2 * a + sa; }
    if (tb < a1) { a1 = tb; q1 = 2 * a + sb; }
  }
  *t0 = a0;
  *t1 = a1;
  if (p0) *p0 = q0;
  if (p1) *p1 = q1;
  return a1 > a0;
}

/* ------------------------------------------------------------------------ */
/* Scene bookkeeping: per-voxel canonical cube, inverse transform, bbox.      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  int C;
  double h;
  double origin[3];
  const uint16_t* ijk;
  const double* A;     /* [n][12] blended transforms */
  const double* feat;  /* [n][C] */
  const double* sigma; /* [n] */
} orc_scene;

typedef struct {
  double Ainv[12];
  double lo[3];
  int ok;                 /* det >= DET_MIN and all corners in front */
  double umin, umax, vmin, vmax;
  double dmin, dmax;      /* distance bounds |c - o| -+ r */
} vox_info;

/* The box A * [lo, lo + h]^3 seen from camera c: inverse transform, validity,
 * projected bounding box and distance bounds. */
static void box_info(const double A[12], const double lo[3], double h, const orc_cam* c, vox_info* v) {
  for (int a = 0; a < 3; ++a) v->lo[a] = lo[a];
  v->ok = det3(A, 4) >= ORC_DET_MIN && affine_inv(A, v->Ainv);
  if (!v->ok) return;
  double o[3];
  for (int a = 0; a < 3; ++a)
    o[a] = -(c->w2c[0 * 4 + a] * c->w2c[3] + c->w2c[1 * 4 + a] * c->w2c[7] + c->w2c[2 * 4 + a] * c->w2c[11]);
  double cw[3], corners[8][3];
  for (int a = 0; a < 3; ++a) {
    double cc[3] = {v->lo[0] + 0.5 * h, v->lo[1] + 0.5 * h, v->lo[2] + 0.5 * h};
    cw[a] = A[a * 4] * cc[0] + A[a * 4 + 1] * cc[1] + A[a * 4 + 2] * cc[2] + A[a * 4 + 3];
  }
  v->umin = v->vmin = INFINITY;
  v->umax = v->vmax = -INFINITY;
  double r = 0.0;
  for (int q = 0; q < 8; ++q) {
    double p[3] = {v->lo[0] + ((q & 1) ? h : 0.0), v->lo[1] + ((q & 2) ? h : 0.0),
                   v->lo[2] + ((q & 4) ? h : 0.0)};
    double dd = 0;
    for (int a = 0; a < 3; ++a) {
      corners[q][a] = A[a * 4] * p[0] + A[a * 4 + 1] * p[1] + A[a * 4 + 2] * p[2] + A[a * 4 + 3];
      dd += (corners[q][a] - cw[a]) * (corners[q][a] - cw[a]);
    }
    if (sqrt(dd) > r) r = sqrt(dd);
    double X = c->w2c[0] * corners[q][0] + c->w2c[1] * corners[q][1] + c->w2c[2] * corners[q][2] + c->w2c[3];
    double Y = c->w2c[4] * corners[q][0] + c->w2c[5] * corners[q][1] + c->w2c[6] * corners[q][2] + c->w2c[7];
    double Z = c->w2c[8] * corners[q][0] + c->w2c[9] * corners[q][1] + c->w2c[10] * corners[q][2] + c->w2c[11];
    if (Z <= ORC_Z_MIN) {
      v->ok = 0;
      return;
    }
    double u = c->fx * X / Z + c->cx, vv = c->fy * Y / Z + c->cy;
    if (u < v->umin) v->umin = u;
    if (u > v->umax) v->umax = u;
    if (vv < v->vmin) v->vmin = vv;
    if (vv > v->vmax) v->vmax = vv;
  }
  double dc = sqrt((cw[0] - o[0]) * (cw[0] - o[0]) + (cw[1] - o[1]) * (cw[1] - o[1]) +
                   (cw[2] - o[2]) * (cw[2] - o[2]));
  v->dmin = dc - r;
  v->dmax = dc + r;
}

static void voxel_info(const orc_scene* s, const orc_cam* c, int64_t i, vox_info* v) {
  double lo[3];
  for (int a = 0; a < 3; ++a) lo[a] = s->origin[a] + (double)s->ijk[3 * i + a] * s->h;
  box_info(s->A + 12 * i, lo, s->h, c, v);
}

/* ------------------------------------------------------------------------ */
/* Per-pixel hit lists and compositing (Eq. 5, Eq. 6).                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  double t0, t1;
  int64_t id;
  int p0, p1;
} hit_t;

static int hit_cmp(const void* a, const void* b) {
  const hit_t* x = (const hit_t*)a;
  const hit_t* y = (const hit_t*)b;
  if (x->t0 != y->t0) return x->t0 < y->t0 ? -1 : 1;
  if (x->t1 != y->t1) return x->t1 < y->t1 ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* Front-to-back compositing of an ordered hit list (Eq. 5, Eq. 6):
 *   T_i = exp(-sum_{j<i} sigma_j delta_j),  F = sum_i T_i (1 - exp(-sigma_i delta_i)) f_i,
 *   stop after the first hit at which exp(-sum_{j<=i} sigma_j delta_j) < tau,
 *   A = 1 - exp(-sum over composited hits).
 * Returns the number of composited hits. */
static int composite(const orc_scene* s, const hit_t* hits, int m, double tau, double* F, double* Aout) {
  for (int c = 0; c < s->C; ++c) F[c] = 0.0;
  double optical = 0.0;
  int used = 0;
  for (int i = 0; i < m; ++i) {
    double sig = s->sigma[hits[i].id];
    double delta = hits[i].t1 - hits[i].t0;
    double Ti = exp(-optical);
    double alpha = 1.0 - exp(-sig * delta);
    const double* f = s->feat + (size_t)hits[i].id * s->C;
    for (int c = 0; c < s->C; ++c) F[c] += Ti * alpha * f[c];
    optical += sig * delta;
    used = i + 1;
    if (exp(-optical) < tau) break;
  }
  *Aout = 1.0 - exp(-optical);
  return used;
}

/* Candidate lists: voxel i is a candidate of every pixel whose centre lies in
 * its projected-corner bounding box grown by one pixel (a superset of the
 * pixels whose ray can hit it; the exact test decides). */
typedef struct {
  int64_t* off; /* [W*H + 1] */
  int64_t* vid;
} cand_t;

static int build_candidates(const orc_scene* s, const orc_cam* c, const vox_info* info, cand_t* out) {
  int64_t npx = (int64_t)c->W * c->H;
  int64_t* cnt = (int64_t*)calloc((size_t)npx + 1, sizeof(int64_t));
  if (!cnt) return -2;
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t i = 0; i < s->n; ++i) {
      const vox_info* v = info + i;
      if (!v->ok) continue;
      int x0 = (int)ceil(v->umin - 0.5) - 1, x1 = (int)floor(v->umax - 0.5) + 1;
      int y0 = (int)ceil(v->vmin - 0.5) - 1, y1 = (int)floor(v->vmax - 0.5) + 1;
      if (x0 < 0) x0 = 0;
      if (y0 < 0) y0 = 0;
      if (x1 > c->W - 1) x1 = c->W - 1;
      if (y1 > c->H - 1) y1 = c->H - 1;
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
          int64_t p = (int64_t)y * c->W + x;
          if (pass == 0)
            cnt[p + 1]++;
          else
            out->vid[cnt[p]++] = i;
        }
    }
    if (pass == 0) {
      for (int64_t p = 0; p < npx; ++p) cnt[p + 1] += cnt[p];
      out->off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)npx + 1));
      out->vid = (int64_t*)malloc(sizeof(int64_t) * ((size_t)cnt[npx] + 1));
      if (!out->off || !out->vid) {
        free(cnt);
        return -2;
      }
      memcpy(out->off, cnt, sizeof(int64_t) * ((size_t)npx + 1));
    }
  }
  free(cnt);
  return 0;
}

static int pixel_hits(const orc_scene* s, const orc_cam* c, const vox_info* info, const int64_t* ids,
                      int64_t nid, int x, int y, hit_t** buf, int* cap) {
  double o[3], d[3];
  cam_ray(c, x, y, o, d);
  int m = 0;
  for (int64_t k = 0; k < nid; ++k) {
    int64_t i = ids ? ids[k] : k;
    const vox_info* v = info + i;
    if (!v->ok) continue;
    double t0, t1;
    int p0, p1;
    if (hit_voxel(v->Ainv, v->lo, s->h, o, d, c->near_, c->far_, &t0, &t1, &p0, &p1)) {
      if (m == *cap) {
        *cap = *cap ? 2 * *cap : 64;
        *buf = (hit_t*)realloc(*buf, sizeof(hit_t) * (size_t)*cap);
      }
      (*buf)[m].t0 = t0;
      (*buf)[m].t1 = t1;
      (*buf)[m].id = i;
      (*buf)[m].p0 = p0;
      (*buf)[m].p1 = p1;
      ++m;
    }
  }
  qsort(*buf, (size_t)m, sizeof(hit_t), hit_cmp);
  return m;
}

static vox_info* all_info(const orc_scene* s, const orc_cam* c) {
  vox_info* info = (vox_info*)malloc(sizeof(vox_info) * (size_t)(s->n > 0 ? s->n : 1));
  if (!info) return NULL;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) voxel_info(s, c, i, info + i);
  return info;
}

/*
 * Render feature map F [H][W][C] and coarse opacity A [H][W].
 * Optional outputs (NULL to skip): nhit [H*W] total hits, nused [H*W]
 * composited hits, and the ordered hit lists as CSR (hit_off [H*W+1],
 * hit_id / hit_t0 / hit_t1 [hit_cap]).  Returns the total hit count, or
 * -(needed) when hit_cap is too small, or < -2^40 on allocation failure.
 */
int64_t orc_render(const orc_scene* s, const orc_cam* c, double tau, double* F, double* Aout,
                   int32_t* nhit, int32_t* nused, int64_t* hit_off, int64_t* hit_id, double* hit_t0,
                   double* hit_t1, int64_t hit_cap) {
  vox_info* info = all_info(s, c);
  if (!info) return -((int64_t)1 << 41);
  cand_t cand = {0, 0};
  if (build_candidates(s, c, info, &cand) != 0) {
    free(info);
    return -((int64_t)1 << 41);
  }
  int64_t npx = (int64_t)c->W * c->H;
  int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)npx);
  int64_t total = 0;
#pragma omp parallel
  {
    hit_t* buf = NULL;
    int cap = 0;
#pragma omp for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t p = 0; p < npx; ++p) {
      int x = (int)(p % c->W), y = (int)(p / c->W);
      int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
      int used = composite(s, buf, m, tau, F + p * s->C, Aout + p);
      if (nhit) nhit[p] = m;
      if (nused) nused[p] = used;
      cnt[p] = m;
      total += m;
    }
    free(buf);
  }
  int64_t ret = total;
  if (hit_off) {
    if (total > hit_cap) {
      ret = -total;
    } else {
      hit_off[0] = 0;
      for (int64_t p = 0; p < npx; ++p) hit_off[p + 1] = hit_off[p] + cnt[p];
#pragma omp parallel
      {
        hit_t* buf = NULL;
        int cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < npx; ++p) {
          int x = (int)(p % c->W), y = (int)(p / c->W);
          int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
          for (int k = 0; k < m; ++k) {
            hit_id[hit_off[p] + k] = buf[k].id;
            hit_t0[hit_off[p] + k] = buf[k].t0;
            hit_t1[hit_off[p] + k] = buf[k].t1;
          }
        }
        free(buf);
      }
    }
  }
  free(cnt);
  free(cand.off);
  free(cand.vid);
  free(info);
  return ret;
}

/*
 * Depth buffer (Sec. 3.1 "Hybrid Rendering": a pixel's depth is how far
 * along its ray the nearest voxel denser than a set threshold lies).
 * Per pixel: the entry distance t0 of the first hit, in the compositing
 * order (t0, t1, voxel id), whose density exceeds sigma_min — over all of the
 * ray's hits inside [near, far], not only those composited before the early
 * stop — and +inf where there is none.  depth, chord: [H*W]; chord (may be
 * NULL) gets t1 - t0 of that hit (+inf where none).  Returns 0, or -1 on
 * allocation failure.
 */
int orc_depth(const orc_scene* s, const orc_cam* c, double sigma_min, double* depth, double* chord) {
  vox_info* info = all_info(s, c);
  if (!info) return -1;
  cand_t cand = {0, 0};
  if (build_candidates(s, c, info, &cand) != 0) {
    free(info);
    return -1;
  }
  int64_t npx = (int64_t)c->W * c->H;
#pragma omp parallel
  {
    hit_t* buf = NULL;
    int cap = 0;
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < npx; ++p) {
      int x = (int)(p % c->W), y = (int)(p / c->W);
      int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
      depth[p] = INFINITY;
      if (chord) chord[p] = INFINITY;
      for (int k = 0; k < m; ++k)
        if (s->sigma[buf[k].id] > sigma_min) {
          depth[p] = buf[k].t0;
          if (chord) chord[p] = buf[k].t1 - buf[k].t0;
          break;
        }
    }
    free(buf);
  }
  free(cand.off);
  free(cand.vid);
  free(info);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's own per-frame index (Sec. 3.1, "Dynamic Volume Rendering",     */
/* and the query operator Q of the voxel regularisation term, "Training").   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t c[3];
  int64_t id;
} snap_t;

static int snap_cmp(const void* a, const void* b) {
  const snap_t* x = (const snap_t*)a;
  const snap_t* y = (const snap_t*)b;
  for (int k = 0; k < 3; ++k)
    if (x->c[k] != y->c[k]) return x->c[k] < y->c[k] ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

/*
 * Places each voxel's warped centre p_i^t = A_i p_i^c (Eq. 4, p_i^c the centre
 * of its canonical cube) in the cell floor((p_i^t - origin) / h) of the
 * lattice of the canonical octree's leaves: the index the paper rebuilds
 * under every pose.  Voxels that land in one cell collide and one survives;
 * Q(p, T^t) returns the survivor of the cell holding p.  Readings: the lattice
 * is the canonical octree's (origin, leaf size h) without bounds; the
 * survivor of a collision is the smallest voxel id; a voxel whose blend has
 * det < 1e-3 (or a centre beyond 2^40 cells) is not placed.
 * cell [n][3]: lattice coordinates (any sign; 0 when not placed);
 * winner [n]: the survivor of voxel i's cell, -1 when i is not placed.
 * Returns the number of occupied cells, or -1 on allocation failure.
 */
int64_t orc_grid_snap(const orc_scene* s, int64_t* cell, int64_t* winner) {
  snap_t* e = (snap_t*)malloc(sizeof(snap_t) * (size_t)(s->n > 0 ? s->n : 1));
  if (!e) return -1;
  int64_t m = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    const double* A = s->A + 12 * i;
    winner[i] = -1;
    cell[3 * i] = cell[3 * i + 1] = cell[3 * i + 2] = 0;
    if (det3(A, 4) < ORC_DET_MIN) continue;
    double pc[3], q[3];
    for (int a = 0; a < 3; ++a) pc[a] = s->origin[a] + ((double)s->ijk[3 * i + a] + 0.5) * s->h;
    int ok = 1;
    for (int a = 0; a < 3; ++a) {
      double p = A[a * 4] * pc[0] + A[a * 4 + 1] * pc[1] + A[a * 4 + 2] * pc[2] + A[a * 4 + 3];
      q[a] = floor((p - s->origin[a]) / s->h);
      if (!(fabs(q[a]) <= 1099511627776.0)) ok = 0;
    }
    if (!ok) continue;
    for (int a = 0; a < 3; ++a) e[m].c[a] = cell[3 * i + a] = (int64_t)q[a];
    e[m].id = i;
    ++m;
  }
  qsort(e, (size_t)m, sizeof(snap_t), snap_cmp);
  int64_t cells = 0;
  for (int64_t k = 0; k < m;) {
    int64_t j = k;
    while (j < m && e[j].c[0] == e[k].c[0] && e[j].c[1] == e[k].c[1] && e[j].c[2] == e[k].c[2]) {
      winner[e[j].id] = e[k].id;
      ++j;
    }
    ++cells;
    k = j;
  }
  free(e);
  return cells;
}

/*
 * Renders the snapped index: each occupied cell is the axis-aligned box
 * origin + h [cell, cell + 1]^3 with its survivor's feature and density, and
 * each pixel's ray composites the cells it crosses front to back as the
 * voxel path does (Eq. 5, Eq. 6, early stop), in the order (t0, t1,
 * survivor id).  A cell with a corner at camera z <= 1e-6 is not rendered.
 * F [H*W][C], Aout [H*W], nhit [H*W] (may be NULL).  Returns the number of
 * occupied cells, or -1 on allocation failure.
 */
int64_t orc_render_grid(const orc_scene* s, const orc_cam* c, double tau, double* F, double* Aout,
                        int32_t* nhit) {
  static const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  const size_t n1 = (size_t)(s->n > 0 ? s->n : 1);
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * 3 * n1);
  int64_t* win = (int64_t*)malloc(sizeof(int64_t) * n1);
  vox_info* info = (vox_info*)malloc(sizeof(vox_info) * n1);
  double* sig = (double*)malloc(sizeof(double) * n1);
  double* feat = (double*)malloc(sizeof(double) * n1 * (size_t)s->C);
  int64_t nc = (cell && win && info && sig && feat) ? orc_grid_snap(s, cell, win) : -1;
  cand_t cand = {0, 0};
  if (nc >= 0) {
    int64_t k = 0;
    for (int64_t i = 0; i < s->n; ++i) {
      if (win[i] != i) continue;
      double lo[3];
      for (int a = 0; a < 3; ++a) lo[a] = s->origin[a] + (double)cell[3 * i + a] * s->h;
      box_info(I, lo, s->h, c, info + k);
      sig[k] = s->sigma[i];
      memcpy(feat + (size_t)k * s->C, s->feat + (size_t)i * s->C, sizeof(double) * (size_t)s->C);
      ++k;
    }
    orc_scene g = {nc, s->C, s->h, {s->origin[0], s->origin[1], s->origin[2]}, NULL, NULL, feat, sig};
    if (build_candidates(&g, c, info, &cand) != 0) {
      nc = -1;
    } else {
      const int64_t npx = (int64_t)c->W * c->H;
#pragma omp parallel
      {
        hit_t* buf = NULL;
        int cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < npx; ++p) {
          int x = (int)(p % c->W), y = (int)(p / c->W);
          int m = pixel_hits(&g, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
          composite(&g, buf, m, tau, F + p * s->C, Aout + p);
          if (nhit) nhit[p] = m;
        }
        free(buf);
      }
    }
  }
  free(cand.off);
  free(cand.vid);
  free(feat);
  free(sig);
  free(info);
  free(win);
  free(cell);
  return nc;
}

/* ------------------------------------------------------------------------ */
/* View-dependent features (Eq. 2): per voxel, spherical-harmonics           */
/* coefficient vectors k_h in R^C evaluated at the ray direction mapped into  */
/* the voxel's canonical frame, d^c = R_i^-1 d (Sec. 3.1, "Dynamic Volume     */
/* Rendering"), S = sum_h k_h Y_h(d^c).                                       */
/* ------------------------------------------------------------------------ */

#define ORC_SH_LMAX 9
#define ORC_PI 3.14159265358979323846

/* Real orthonormal spherical harmonics of degree <= L (L <= ORC_SH_LMAX) at
 * the unit direction d, Y[l*l + l + m] for -l <= m <= l:
 *   Y_{l,0} = K_l^0 P_l^0(z),
 *   Y_{l,m} = sqrt(2) K_l^m P_l^m(z) cos(m phi),  Y_{l,-m} = sqrt(2) K_l^m P_l^m(z) sin(m phi)  (m > 0),
 *   K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
 * P_l^m the associated Legendre functions without the Condon-Shortley
 * phase, z = cos(theta) = d_z, phi = atan2(d_y, d_x).  Returns 0, or -1 for
 * a degree out of range. */
int orc_sh_basis(int L, const double d[3], double* Y) {
  if (L < 0 || L > ORC_SH_LMAX) return -1;
  const int S = ORC_SH_LMAX + 1;
  double P[(ORC_SH_LMAX + 1) * (ORC_SH_LMAX + 1)];
  const double z = d[2], st = hypot(d[0], d[1]), phi = atan2(d[1], d[0]);
  for (int m = 0; m <= L; ++m) {
    double pmm = 1.0;
    for (int k = 1; k <= m; ++k) pmm *= (double)(2 * k - 1) * st;
    P[m * S + m] = pmm;
    if (m + 1 <= L) P[(m + 1) * S + m] = z * (double)(2 * m + 1) * pmm;
    for (int l = m + 2; l <= L; ++l)
      P[l * S + m] = ((double)(2 * l - 1) * z * P[(l - 1) * S + m] - (double)(l + m - 1) * P[(l - 2) * S + m]) /
                     (double)(l - m);
  }
  for (int l = 0; l <= L; ++l)
    for (int m = 0; m <= l; ++m) {
      double ratio = 1.0; /* (l-m)! / (l+m)! */
      for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
      const double K = sqrt((double)(2 * l + 1) / (4.0 * ORC_PI) * ratio);
      if (m == 0) {
        Y[l * l + l] = K * P[l * S];
      } else {
        Y[l * l + l + m] = sqrt(2.0) * K * P[l * S + m] * cos((double)m * phi);
        Y[l * l + l - m] = sqrt(2.0) * K * P[l * S + m] * sin((double)m * phi);
      }
    }
  return 0;
}

/* Rotation factor R of the polar decomposition A_lin = R S (S symmetric
 * positive definite) of the 3x3 block of a 3x4 affine matrix with a positive
 * determinant, by Newton's iteration X <- (X + X^-T) / 2 from X = A_lin
 * (Higham 1986).  R: [9] row-major.  Returns 0, or -1 when det <= 0. */
int orc_polar_rotation(const double A[12], double R[9]) {
  double X[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) X[r * 3 + c] = A[r * 4 + c];
  if (det3(X, 3) <= 0.0) return -1;
  for (int it = 0; it < 100; ++it) {
    const double d = det3(X, 3);
    /* X^-T = cofactor(X) / det */
    const double cof[9] = {X[4] * X[8] - X[5] * X[7], X[5] * X[6] - X[3] * X[8], X[3] * X[7] - X[4] * X[6],
                           X[2] * X[7] - X[1] * X[8], X[0] * X[8] - X[2] * X[6], X[1] * X[6] - X[0] * X[7],
                           X[1] * X[5] - X[2] * X[4], X[2] * X[3] - X[0] * X[5], X[0] * X[4] - X[1] * X[3]};
    double diff = 0.0;
    for (int k = 0; k < 9; ++k) {
      const double xn = 0.5 * (X[k] + cof[k] / d);
      diff = fmax(diff, fabs(xn - X[k]));
      X[k] = xn;
    }
    if (diff < 1e-15) break;
  }
  memcpy(R, X, sizeof(X));
  return 0;
}

/*
 * Feature map and coarse opacity with view-dependent features: as orc_render
 * (Eq. 5, Eq. 6, early stop) but each hit's feature is
 * S = sum_h coef[i][h][:] Y_h(R_i^T d), R_i the rotation factor of voxel i's
 * blended transform, d the unit pixel ray direction, H = (L+1)^2.
 * coef: [n][H][C] (C = the scene's channel count; the scene's own features
 * are not used).  F [H*W][C], A [H*W].  Returns 0, or -1 on allocation
 * failure or a degree out of range.
 */
int orc_render_sh(const orc_scene* s, const orc_cam* c, double tau, int L, const double* coef, double* F,
                  double* Aout) {
  if (L < 0 || L > ORC_SH_LMAX) return -1;
  const int H = (L + 1) * (L + 1), C = s->C;
  vox_info* info = all_info(s, c);
  if (!info) return -1;
  double* rot = (double*)malloc(sizeof(double) * 9 * (size_t)(s->n > 0 ? s->n : 1));
  cand_t cand = {0, 0};
  if (!rot || build_candidates(s, c, info, &cand) != 0) {
    free(rot);
    free(info);
    return -1;
  }
  for (int64_t i = 0; i < s->n; ++i)
    if (!info[i].ok || orc_polar_rotation(s->A + 12 * i, rot + 9 * i) != 0) info[i].ok = 0;
  const int64_t npx = (int64_t)c->W * c->H;
#pragma omp parallel
  {
    hit_t* buf = NULL;
    int cap = 0;
    double Y[(ORC_SH_LMAX + 1) * (ORC_SH_LMAX + 1)];
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < npx; ++p) {
      const int x = (int)(p % c->W), y = (int)(p / c->W);
      int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
      double o[3], d[3];
      cam_ray(c, x, y, o, d);
      double* Fp = F + p * C;
      for (int k = 0; k < C; ++k) Fp[k] = 0.0;
      double optical = 0.0;
      for (int q = 0; q < m; ++q) {
        const int64_t id = buf[q].id;
        const double* R = rot + 9 * id;
        const double dc[3] = {R[0] * d[0] + R[3] * d[1] + R[6] * d[2], R[1] * d[0] + R[4] * d[1] + R[7] * d[2],
                              R[2] * d[0] + R[5] * d[1] + R[8] * d[2]};
        orc_sh_basis(L, dc, Y);
        const double sig = s->sigma[id], delta = buf[q].t1 - buf[q].t0;
        const double w = exp(-optical) * (1.0 - exp(-sig * delta));
        const double* kq = coef + (size_t)id * H * C;
        for (int k = 0; k < C; ++k) {
          double f = 0.0;
          for (int h = 0; h < H; ++h) f += kq[(size_t)h * C + k] * Y[h];
          Fp[k] += w * f;
        }
        optical += sig * delta;
        if (exp(-optical) < tau) break;
      }
      Aout[p] = 1.0 - exp(-optical);
    }
    free(buf);
  }
  free(cand.off);
  free(cand.vid);
  free(rot);
  free(info);
  return 0;
}

/*
 * Gradient of the view-dependent feature map with respect to the SH
 * coefficients: for dL/dF = gF [H*W][C], accumulates
 *   dL/dcoef[i][h][c] = sum over the pixels whose composite uses hit i of
 *                        w_i Y_h(R_i^T d) gF[c],   w_i = T_i (1 - exp(-sigma_i delta_i)),
 * over the hits composited before the early stop (F is linear in the
 * coefficients).  gcoef [n][(L+1)^2][C], zeroed here.  Serial over pixels.
 * Returns 0, or -1 on allocation failure or a degree out of range.
 */
int orc_render_sh_backward(const orc_scene* s, const orc_cam* c, double tau, int L, const double* gF,
                           double* gcoef) {
  if (L < 0 || L > ORC_SH_LMAX) return -1;
  const int H = (L + 1) * (L + 1), C = s->C;
  vox_info* info = all_info(s, c);
  if (!info) return -1;
  double* rot = (double*)malloc(sizeof(double) * 9 * (size_t)(s->n > 0 ? s->n : 1));
  cand_t cand = {0, 0};
  if (!rot || build_candidates(s, c, info, &cand) != 0) {
    free(rot);
    free(info);
    return -1;
  }
  for (int64_t i = 0; i < s->n; ++i)
    if (!info[i].ok || orc_polar_rotation(s->A + 12 * i, rot + 9 * i) != 0) info[i].ok = 0;
  memset(gcoef, 0, sizeof(double) * (size_t)s->n * H * C);
  hit_t* buf = NULL;
  int cap = 0;
  double Y[(ORC_SH_LMAX + 1) * (ORC_SH_LMAX + 1)];
  const int64_t npx = (int64_t)c->W * c->H;
  for (int64_t p = 0; p < npx; ++p) {
    const int x = (int)(p % c->W), y = (int)(p / c->W);
    int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
    double o[3], d[3];
    cam_ray(c, x, y, o, d);
    double optical = 0.0;
    for (int q = 0; q < m; ++q) {
      const int64_t id = buf[q].id;
      const double* R = rot + 9 * id;
      const double dc[3] = {R[0] * d[0] + R[3] * d[1] + R[6] * d[2], R[1] * d[0] + R[4] * d[1] + R[7] * d[2],
                            R[2] * d[0] + R[5] * d[1] + R[8] * d[2]};
      orc_sh_basis(L, dc, Y);
      const double sig = s->sigma[id], delta = buf[q].t1 - buf[q].t0;
      const double w = exp(-optical) * (1.0 - exp(-sig * delta));
      double* gk = gcoef + (size_t)id * H * C;
      for (int h = 0; h < H; ++h)
        for (int k = 0; k < C; ++k) gk[(size_t)h * C + k] += w * Y[h] * gF[p * C + k];
      optical += sig * delta;
      if (exp(-optical) < tau) break;
    }
  }
  free(buf);
  free(cand.off);
  free(cand.vid);
  free(rot);
  free(info);
  return 0;
}

/*
 * One pixel, by brute force over every voxel (no candidate pre-selection).
 * Writes F [C], A, and up to cap ordered hits.  Returns the number of hits.
 */
int orc_pixel_brute(const orc_scene* s, const orc_cam* c, int x, int y, double tau, double* F,
                    double* Aout, int64_t* ids, double* t0, double* t1, int cap, int* used) {
  vox_info* info = all_info(s, c);
  if (!info) return -1;
  hit_t* buf = NULL;
  int bcap = 0;
  int m = pixel_hits(s, c, info, NULL, s->n, x, y, &buf, &bcap);
  int u = composite(s, buf, m, tau, F, Aout);
  if (used) *used = u;
  for (int k = 0; k < m && k < cap; ++k) {
    ids[k] = buf[k].id;
    t0[k] = buf[k].t0;
    t1[k] = buf[k].t1;
  }
  free(buf);
  free(info);
  return m;
}

/*
 * A list of pixels (px, py [np]) rendered one by one, each by brute force over
 * all voxels.  Used to check sampled outputs of full-size frames.
 */
int orc_pixels(const orc_scene* s, const orc_cam* c, int64_t np, const int32_t* px, const int32_t* py,
               double tau, double* F, double* Aout, int32_t* nhit, double tie_eps, double* tie) {
  vox_info* info = all_info(s, c);
  if (!info) return -1;
#pragma omp parallel
  {
    hit_t* buf = NULL;
    int bcap = 0;
#pragma omp for schedule(dynamic, 1)
    for (int64_t k = 0; k < np; ++k) {
      int m = pixel_hits(s, c, info, NULL, s->n, px[k], py[k], &buf, &bcap);
      int used = composite(s, buf, m, tau, F + k * s->C, Aout + k);
      if (nhit) nhit[k] = m;
      if (tie) {
        /* Order-ambiguous pairs: consecutive hits among the composited ones
         * (and the first after the stop) whose entry distances differ by less
         * than tie_eps.  Swapping such a pair i, i+1 changes F by
         * T_i alpha_i alpha_{i+1} (f_i - f_{i+1}); the largest channel change
         * over the pixel's pairs is reported (0 when there is none). */
        double worst = 0.0, optical = 0.0;
        for (int i = 0; i + 1 < m && i <= used; ++i) {
          const double si = s->sigma[buf[i].id], sj = s->sigma[buf[i + 1].id];
          const double ai = 1.0 - exp(-si * (buf[i].t1 - buf[i].t0));
          if (buf[i + 1].t0 - buf[i].t0 < tie_eps) {
            const double aj = 1.0 - exp(-sj * (buf[i + 1].t1 - buf[i + 1].t0));
            const double* fi = s->feat + (size_t)buf[i].id * s->C;
            const double* fj = s->feat + (size_t)buf[i + 1].id * s->C;
            double df = 0.0;
            for (int ch = 0; ch < s->C; ++ch) df = fmax(df, fabs(fi[ch] - fj[ch]));
            const double e = exp(-optical) * ai * aj * df;
            if (e > worst) worst = e;
          }
          optical += si * (buf[i].t1 - buf[i].t0);
        }
        tie[k] = worst;
      }
    }
    free(buf);
  }
  free(info);
  return 0;
}

/*
 * Screen-tile coverage: voxel i covers tile (tx, ty) of size tsx x tsy when its
 * projected-corner bounding box contains at least one pixel centre of the
 * tile.  Voxels that are degenerate, cross the camera plane, or whose
 * distance range [|c-o| - r, |c-o| + r] misses [near, far] cover nothing.
 * Writes (tile id, voxel id) pairs in voxel order; returns the pair count or
 * -(needed) when cap is too small.
 */
int64_t orc_tile_pairs(const orc_scene* s, const orc_cam* c, int tsx, int tsy, int32_t* tile, int64_t* vid,
                       int64_t cap) {
  vox_info* info = all_info(s, c);
  if (!info) return -((int64_t)1 << 41);
  int tw = (c->W + tsx - 1) / tsx;
  int64_t m = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    const vox_info* v = info + i;
    if (!v->ok || v->dmin > c->far_ || v->dmax < c->near_) continue;
    int x0 = (int)ceil(v->umin - 0.5), x1 = (int)floor(v->umax - 0.5);
    int y0 = (int)ceil(v->vmin - 0.5), y1 = (int)floor(v->vmax - 0.5);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > c->W - 1) x1 = c->W - 1;
    if (y1 > c->H - 1) y1 = c->H - 1;
    if (x0 > x1 || y0 > y1) continue;
    for (int ty = y0 / tsy; ty <= y1 / tsy; ++ty)
      for (int tx = x0 / tsx; tx <= x1 / tsx; ++tx) {
        if (m < cap) {
          tile[m] = ty * tw + tx;
          vid[m] = i;
        }
        ++m;
      }
  }
  free(info);
  return m <= cap ? m : -m;
}

/* Per-voxel distance bounds and projected bounding boxes (for tests). */
void orc_voxel_bounds(const orc_scene* s, const orc_cam* c, double* out /*[n][7]: ok,umin,umax,vmin,vmax,dmin,dmax*/) {
  vox_info* info = all_info(s, c);
  if (!info) return;
  for (int64_t i = 0; i < s->n; ++i) {
    out[7 * i + 0] = info[i].ok;
    out[7 * i + 1] = info[i].umin;
    out[7 * i + 2] = info[i].umax;
    out[7 * i + 3] = info[i].vmin;
    out[7 * i + 4] = info[i].vmax;
    out[7 * i + 5] = info[i].dmin;
    out[7 * i + 6] = info[i].dmax;
  }
  free(info);
}

/* ------------------------------------------------------------------------ */
/* Learned ray-interval proposal (project addition; the nearest passage of  */
/* the paper is the early-stop rule of Sec. 3.1 "Dynamic Volume Rendering"):  */
/* labels from the plain composite, compositing restricted to an interval,  */
/* the exact transmittance mass that the restriction loses, and a coarse    */
/* per-(tile, depth bin) bound of the optical depth.                         */
/* ------------------------------------------------------------------------ */

/* Depth interval of the bin pair (bn, bf) over nb uniform bins of [near, far]:
 * [near + bn D, near + (bf + 1) D], D = (far - near) / nb.  bf < bn is empty. */
static void bin_interval(const orc_cam* c, int nb, int bn, int bf, double* lo, double* hi) {
  double D = (c->far_ - c->near_) / nb;
  *lo = c->near_ + bn * D;
  *hi = c->near_ + (bf + 1) * D;
}

/* One ray, ordered hits [0, m).  Restricted set S = hits with t1 >= lo and
 * t0 <= hi (none when empty); front P = hits with t1 < lo (all hits when
 * empty); back Q = hits with t0 > hi.  S is composited with the stop rule of
 * composite().  missed = (1 - exp(-tau_P)) + T_end (1 - exp(-tau_Q)), T_end the
 * transmittance after S.  *amb is set when a hit lies within eps of the
 * interval's ends (its membership is decided by rounding). */
static void composite_interval(const orc_scene* s, const hit_t* hits, int m, double tau, int empty, double lo,
                               double hi, double eps, double* F, double* Aout, double* missed, int* amb) {
  for (int c = 0; c < s->C; ++c) F[c] = 0.0;
  double opt = 0.0, optP = 0.0, optQ = 0.0;
  int stopped = 0;
  *amb = 0;
  for (int i = 0; i < m; ++i) {
    double sig = s->sigma[hits[i].id];
    double delta = hits[i].t1 - hits[i].t0;
    if (!empty && (fabs(hits[i].t1 - lo) < eps || fabs(hits[i].t0 - hi) < eps)) *amb = 1;
    if (empty || hits[i].t1 < lo) {
      optP += sig * delta;
      continue;
    }
    if (hits[i].t0 > hi) {
      optQ += sig * delta;
      continue;
    }
    if (stopped) continue;
    double Ti = exp(-opt);
    double alpha = 1.0 - exp(-sig * delta);
    const double* f = s->feat + (size_t)hits[i].id * s->C;
    for (int c = 0; c < s->C; ++c) F[c] += Ti * alpha * f[c];
    opt += sig * delta;
    if (exp(-opt) < tau) stopped = 1;
  }
  *Aout = 1.0 - exp(-opt);
  *missed = (1.0 - exp(-optP)) + exp(-opt) * (1.0 - exp(-optQ));
}

/*
 * Per pixel: the label of the plain composite, and the composite restricted
 * to the interval of bins [p][0..1] (NULL: no restriction).
 *   labels [H*W][3] (NULL to skip): (min t1, max t0) over the composited hits
 *     whose weight T_i alpha_i exceeds wmin, and the transmittance just after
 *     the last of them; (+inf, -inf, 1) when there is none.
 *   F [H*W][C], A [H*W]: restricted composite; missed [H*W]: its exact lost
 *     mass; amb [H*W] (int32): a hit within eps of an interval end.
 */
int orc_render_interval(const orc_scene* s, const orc_cam* c, double tau, int nb, const int32_t* bins, double wmin,
                        double eps, double* labels, double* F, double* Aout, double* missed, int32_t* amb) {
  vox_info* info = all_info(s, c);
  if (!info) return -2;
  cand_t cand = {0, 0};
  if (build_candidates(s, c, info, &cand) != 0) {
    free(info);
    return -2;
  }
  int64_t npx = (int64_t)c->W * c->H;
#pragma omp parallel
  {
    hit_t* buf = NULL;
    int cap = 0;
    double* tmpF = (double*)malloc(sizeof(double) * (size_t)s->C);
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < npx; ++p) {
      int x = (int)(p % c->W), y = (int)(p / c->W);
      int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
      if (labels) {
        double lo = INFINITY, hi = -INFINITY, Ts = 1.0, opt = 0.0;
        for (int i = 0; i < m; ++i) {
          double sig = s->sigma[buf[i].id];
          double delta = buf[i].t1 - buf[i].t0;
          double w = exp(-opt) * (1.0 - exp(-sig * delta));
          opt += sig * delta;
          if (w > wmin) {
            if (buf[i].t1 < lo) lo = buf[i].t1;
            if (buf[i].t0 > hi) hi = buf[i].t0;
            Ts = exp(-opt);
          }
          if (exp(-opt) < tau) break;
        }
        labels[3 * p] = lo;
        labels[3 * p + 1] = hi;
        labels[3 * p + 2] = Ts;
      }
      double lo = c->near_, hi = c->far_;
      int empty = 0;
      if (bins) {
        empty = bins[2 * p + 1] < bins[2 * p];
        bin_interval(c, nb, bins[2 * p], bins[2 * p + 1], &lo, &hi);
      }
      int a = 0;
      double ms = 0.0, Ap = 0.0;
      composite_interval(s, buf, m, tau, empty, lo, hi, eps, F ? F + p * s->C : tmpF, &Ap, &ms, &a);
      if (Aout) Aout[p] = Ap;
      if (missed) missed[p] = ms;
      if (amb) amb[p] = a;
    }
    free(tmpF);
    free(buf);
  }
  free(cand.off);
  free(cand.vid);
  free(info);
  return 0;
}

/*
 * Coarse optical-depth bound per (screen tile, depth bin): every voxel that
 * covers a tile (the coverage rule of orc_tile_pairs) adds sigma_i * 2 r_i,
 * an upper bound of sigma_i delta_i for any ray (a chord of the box is at most
 * the diameter of its bounding sphere), to each bin that its distance range
 * [dmin, dmax] = [|c - o| - r, |c - o| + r] overlaps (bins clamped to
 * [0, nb - 1]).  hist [tiles][nb] is overwritten.
 */
int orc_tau_hist(const orc_scene* s, const orc_cam* c, int tsx, int tsy, int nb, double* hist) {
  vox_info* info = all_info(s, c);
  if (!info) return -2;
  int tw = (c->W + tsx - 1) / tsx, th = (c->H + tsy - 1) / tsy;
  memset(hist, 0, sizeof(double) * (size_t)tw * th * nb);
  double D = (c->far_ - c->near_) / nb;
  for (int64_t i = 0; i < s->n; ++i) {
    const vox_info* v = info + i;
    if (!v->ok || v->dmin > c->far_ || v->dmax < c->near_) continue;
    int x0 = (int)ceil(v->umin - 0.5), x1 = (int)floor(v->umax - 0.5);
    int y0 = (int)ceil(v->vmin - 0.5), y1 = (int)floor(v->vmax - 0.5);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > c->W - 1) x1 = c->W - 1;
    if (y1 > c->H - 1) y1 = c->H - 1;
    if (x0 > x1 || y0 > y1) continue;
    double taub = s->sigma[i] * (v->dmax - v->dmin);
    int b0 = (int)floor((v->dmin - c->near_) / D), b1 = (int)floor((v->dmax - c->near_) / D);
    if (b0 < 0) b0 = 0;
    if (b1 > nb - 1) b1 = nb - 1;
    for (int ty = y0 / tsy; ty <= y1 / tsy; ++ty)
      for (int tx = x0 / tsx; tx <= x1 / tsx; ++tx)
        for (int b = b0; b <= b1; ++b) hist[((size_t)ty * tw + tx) * nb + b] += taub;
  }
  free(info);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradients of the composite (project addition; the paper optimises the    */
/* FLUT end to end through Eq. 5-6).                                          */
/* ------------------------------------------------------------------------ */

/*
 * For loss L with dL/dF = gF [H][W][C] and dL/dA = gA [H][W], accumulate
 * dL/df_i into gfeat [n][C], dL/dsigma_i into gsigma [n] and dL/dAinv_i into
 * gAinv [n][12] (Ainv_i maps world -> canonical).  The hit set, the order
 * and the stop index are held fixed.
 *
 * With w_i = T_i a_i, a_i = 1 - exp(-sigma_i delta_i), T_{i+1} = T_i (1-a_i):
 *   dF/df_i      = w_i
 *   dF/dsigma_i  = delta_i (T_{i+1} f_i - sum_{k>i} w_k f_k)
 *   dA/dsigma_i  = delta_i T_final
 *   d/ddelta_i   = the same with sigma_i in place of delta_i
 *   dt/dAinv[a,:] = -[x_hit, 1] / d'_a for the active slab plane of axis a.
 */
int orc_render_backward(const orc_scene* s, const orc_cam* c, double tau, const double* gF, const double* gA,
                        double* gfeat, double* gsigma, double* gAinv) {
  vox_info* info = all_info(s, c);
  if (!info) return -2;
  cand_t cand = {0, 0};
  if (build_candidates(s, c, info, &cand) != 0) {
    free(info);
    return -2;
  }
  int64_t npx = (int64_t)c->W * c->H;
  int C = s->C;
  /* serial over pixels: accumulation order is fixed and the oracle stays simple */
  hit_t* buf = NULL;
  int cap = 0;
  double* suffix = (double*)malloc(sizeof(double) * (size_t)C);
  double* Fp = (double*)malloc(sizeof(double) * (size_t)C);
  for (int64_t p = 0; p < npx; ++p) {
    int x = (int)(p % c->W), y = (int)(p / c->W);
    int zero = gA[p] == 0.0;
    for (int cc = 0; cc < C && zero; ++cc) zero = gF[p * C + cc] == 0.0;
    if (zero) continue; /* a pixel without upstream gradient contributes nothing */
    int m = pixel_hits(s, c, info, cand.vid + cand.off[p], cand.off[p + 1] - cand.off[p], x, y, &buf, &cap);
    if (m == 0) continue;
    double Ap;
    int used = composite(s, buf, m, tau, Fp, &Ap);
    const double* g = gF + p * C;
    double ga = gA[p];
    double o[3], d[3];
    cam_ray(c, x, y, o, d);
    /* T_i before each hit, and T_final */
    double* Tb = (double*)malloc(sizeof(double) * (size_t)(used + 1));
    double optical = 0.0;
    for (int i = 0; i < used; ++i) {
      Tb[i] = exp(-optical);
      optical += s->sigma[buf[i].id] * (buf[i].t1 - buf[i].t0);
    }
    Tb[used] = exp(-optical);
    double Tfinal = Tb[used];
    for (int cc = 0; cc < C; ++cc) suffix[cc] = 0.0;
    for (int i = used - 1; i >= 0; --i) {
      int64_t id = buf[i].id;
      double sig = s->sigma[id];
      double delta = buf[i].t1 - buf[i].t0;
      double a = 1.0 - exp(-sig * delta);
      double wgt = Tb[i] * a;
      const double* f = s->feat + (size_t)id * C;
      double fg = 0.0, sg = 0.0;
      for (int cc = 0; cc < C; ++cc) {
        gfeat[(size_t)id * C + cc] += wgt * g[cc];
        fg += f[cc] * g[cc];
        sg += suffix[cc] * g[cc];
      }
      double core = Tb[i + 1] * fg - sg + Tfinal * ga; /* d L / d(sigma*delta) */
      gsigma[id] += delta * core;
      double gdelta = sig * core;
      /* delta = t1 - t0 */
      const double* Ai = info[id].Ainv;
      for (int side = 0; side < 2; ++side) {
        int plane = side ? buf[i].p1 : buf[i].p0;
        if (plane < 0) continue; /* near/far clip: no geometric dependence */
        double t = side ? buf[i].t1 : buf[i].t0;
        double sgn = side ? 1.0 : -1.0;
        int ax = plane / 2;
        double dp = Ai[ax * 4] * d[0] + Ai[ax * 4 + 1] * d[1] + Ai[ax * 4 + 2] * d[2];
        double xh[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        double gt = sgn * gdelta;
        for (int k = 0; k < 3; ++k) gAinv[12 * id + ax * 4 + k] += gt * (-xh[k] / dp);
        gAinv[12 * id + ax * 4 + 3] += gt * (-1.0 / dp);
      }
      for (int cc = 0; cc < C; ++cc) suffix[cc] += wgt * f[cc];
    }
    free(Tb);
  }
  free(suffix);
  free(Fp);
  free(buf);
  free(cand.off);
  free(cand.vid);
  free(info);
  return 0;
}

/*
 * LBS backward: dL/dA_i from dL/dAinv_i (dN = -N dM N for N = M^-1, with M
 * the 4x4 affine form of A_i), then dL/dw_ik = <dL/dA_i, G_{j_ik}>.
 */
void orc_lbs_backward(int64_t n, int J, const double* G, const uint8_t* jidx, const double* A,
                      const double* gAinv, double* gA_out, double* gw) {
  for (int64_t i = 0; i < n; ++i) {
    double N[16] = {0}, M4[16] = {0}, GN[16] = {0}, GM[16];
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 4; ++k) M4[r * 4 + k] = A[12 * i + r * 4 + k];
    M4[15] = 1.0;
    double Ai[12];
    if (!affine_inv(A + 12 * i, Ai)) {
      for (int k = 0; k < 4; ++k) gw[4 * i + k] = 0.0;
      continue;
    }
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 4; ++k) {
        N[r * 4 + k] = Ai[r * 4 + k];
        GN[r * 4 + k] = gAinv[12 * i + r * 4 + k];
      }
    N[15] = 1.0;
    /* GM = -N^T GN N^T */
    double tmp[16];
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) {
        double acc = 0.0;
        for (int m = 0; m < 4; ++m) acc += N[m * 4 + r] * GN[m * 4 + k];
        tmp[r * 4 + k] = acc;
      }
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) {
        double acc = 0.0;
        for (int m = 0; m < 4; ++m) acc += tmp[r * 4 + m] * N[k * 4 + m];
        GM[r * 4 + k] = -acc;
      }
    (void)M4;
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 4; ++k)
        if (gA_out) gA_out[12 * i + r * 4 + k] = GM[r * 4 + k];
    for (int q = 0; q < 4; ++q) {
      int j = jidx[4 * i + q];
      if (j >= J) j = J - 1;
      double acc = 0.0;
      for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 4; ++k) acc += GM[r * 4 + k] * G[12 * j + r * 4 + k];
      gw[4 * i + q] = acc;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Shading network primitives (Sec. 3.1, "Neural Shading"), NHWC, FP64.      */
/* ------------------------------------------------------------------------ */

/* out[y][x][co] = act(b[co] + sum_{r,s,ci} w[co][r][s][ci] in[y+r-k/2][x+s-k/2][ci]),
 * zero padding outside the image; act 0 = identity, 1 = ReLU, 2 = sigmoid. */
void orc_conv2d(int H, int W, int Cin, int Cout, int k, const double* in, const double* w, const double* b,
                double* out, int act) {
  int pad = k / 2;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      double* o = out + ((size_t)y * W + x) * Cout;
      for (int co = 0; co < Cout; ++co) {
        double acc = b ? b[co] : 0.0;
        for (int r = 0; r < k; ++r) {
          int yy = y + r - pad;
          if (yy < 0 || yy >= H) continue;
          for (int s2 = 0; s2 < k; ++s2) {
            int xx = x + s2 - pad;
            if (xx < 0 || xx >= W) continue;
            const double* ip = in + ((size_t)yy * W + xx) * Cin;
            const double* wp = w + (((size_t)co * k + r) * k + s2) * Cin;
            for (int ci = 0; ci < Cin; ++ci) acc += wp[ci] * ip[ci];
          }
        }
        if (act == 1) acc = acc > 0.0 ? acc : 0.0;
        if (act == 2) acc = 1.0 / (1.0 + exp(-acc));
        o[co] = acc;
      }
    }
  }
}

/* 2x2 max pooling with stride 2 (H, W even). */
void orc_maxpool2(int H, int W, int C, const double* in, double* out) {
  for (int y = 0; y < H / 2; ++y)
    for (int x = 0; x < W / 2; ++x)
      for (int c = 0; c < C; ++c) {
        double m = -INFINITY;
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            double v = in[(((size_t)(2 * y + dy)) * W + (2 * x + dx)) * C + c];
            if (v > m) m = v;
          }
        out[((size_t)y * (W / 2) + x) * C + c] = m;
      }
}

/* Nearest-neighbour x2 upsampling: out[y][x] = in[y/2][x/2]. */
void orc_upsample2(int H, int W, int C, const double* in, double* out) {
  for (int y = 0; y < 2 * H; ++y)
    for (int x = 0; x < 2 * W; ++x)
      for (int c = 0; c < C; ++c)
        out[((size_t)y * 2 * W + x) * C + c] = in[((size_t)(y / 2) * W + (x / 2)) * C + c];
}
