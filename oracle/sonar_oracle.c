/*
 * FP64 CPU oracle for per-ping coherent echo formation in a volumetric 3D sonar
 * ("Towards Realistic 3D Sonar Simulation", Sec. II.A-II.B, Sec. III Eq. 1-3).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke(), and bench.py's
 * cpu_baseline leg and reference arm. The product path never loads it. It is written
 * plainly (no blocking, no fusion, FP64 everywhere, closed forms evaluated directly)
 * so that each step can be checked against the reading of the paper stated beside it.
 *
 * Parity unpinned: Lambertian amplitudes on general meshes, speckle statistics and
 * multi-bounce mesh routes beyond one mirror have no closed form or brute-force check.
 * Curved-ray mesh hits are cross-checked, not pinned: the exact-arc route and the
 * independent Runge-Kutta field route agree to the arcs' chord error. Cross terms,
 * volume scatterers and field rays have their own pins (tests/test_oracle_cross.py,
 * test_oracle_volume.py, test_oracle_field.py).
 */
#include "sonar_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
#define PI 3.14159265358979323846
#define TWO_PI (2.0 * PI)
#define EPS_HIT 1e-7          /* a hit must lie beyond this distance along a segment [m] */
#define ARC_EPS_SAGITTA 1e-4  /* chord sagitta bound for curved rays [m] */
#define ARC_H_MAX 2.0         /* maximum chord arc length [m] */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ small vector math */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* Rotation matrix of the unit quaternion q = (w, x, y, z): sonar frame -> world. */
static void quat_to_matrix(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
static void mat_vec(const double R[9], const double v[3], double r[3]) {
  r[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
  r[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
  r[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}
static void mat_t_vec(const double R[9], const double v[3], double r[3]) {
  r[0] = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
  r[1] = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
  r[2] = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
}

static double sinc(double x) { return fabs(x) < 1e-4 ? 1.0 - x * x / 6.0 : sin(x) / x; }
static double frac(double x) { return x - floor(x); }
static double wrap_pi(double a) { return a - TWO_PI * floor((a + PI) / TWO_PI); }

/* ------------------------------------------------------------------ hash (Sec. II.B speckle) */
/* pcg4d from Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 9(3), 2020. */
void orc_pcg4d(uint32_t v[4]) {
  for (int i = 0; i < 4; ++i) v[i] = v[i] * 1664525u + 1013904223u;
  v[0] += v[1] * v[3]; v[1] += v[2] * v[0]; v[2] += v[0] * v[1]; v[3] += v[1] * v[2];
  for (int i = 0; i < 4; ++i) v[i] ^= v[i] >> 16;
  v[0] += v[1] * v[3]; v[1] += v[2] * v[0]; v[2] += v[0] * v[1]; v[3] += v[1] * v[2];
}
static uint32_t seed32(uint64_t s) { return (uint32_t)(s ^ (s >> 32)); }
static double u24(uint32_t h) { return (double)(h >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------ pulse (Sec. II.B) */
/* Pulse p(t) = w(t) exp(j pi (B/T) t^2), |t| <= T/2, Hann w(t) = (1 + cos(2 pi t/T))/2.
   R(u) = (1/E) int p(v+u) conj(p(v)) dv with E = 3T/8. Writing w as three complex
   exponentials (c0 = 1/2, c+-1 = 1/4) turns the integrand into nine exponentials in v,
   each integrated exactly over the overlap [L, U] of the two pulse supports. */
void orc_pulse_acf(double u, double T, double B, double* re, double* im) {
  if (!(fabs(u) < T)) { *re = 0; *im = 0; return; }
  const double kappa = B / T, Om = TWO_PI / T, E = 3.0 * T / 8.0;
  const double L = fmax(-T / 2, -T / 2 - u), U = fmin(T / 2, T / 2 - u);
  cplx sum = 0;
  for (int a = -1; a <= 1; ++a) {
    for (int b = -1; b <= 1; ++b) {
      double ca = a == 0 ? 0.5 : 0.25, cb = b == 0 ? 0.5 : 0.25;
      double beta = (a + b) * Om + TWO_PI * kappa * u;
      /* int_L^U e^{j beta v} dv = (U-L) sinc(beta (U-L)/2) e^{j beta (U+L)/2} */
      cplx integral = (U - L) * sinc(beta * (U - L) / 2) * cexp(I * beta * (U + L) / 2);
      sum += ca * cb * cexp(I * a * Om * u) * integral;
    }
  }
  cplx r = cexp(I * PI * kappa * u * u) * sum / E;
  *re = creal(r);
  *im = cimag(r);
}

/* The transmitted pulse itself (its raw, uncompressed echo): p(t) = w(t) exp(j pi (B/T)
   t^2) for |t| <= T/2, zero outside, w the Hann window above. */
void orc_pulse(double t, double T, double B, double* re, double* im) {
  if (!(fabs(t) <= T / 2)) { *re = 0; *im = 0; return; }
  const double w = 0.5 * (1.0 + cos(TWO_PI * t / T)), ph = PI * (B / T) * t * t;
  *re = w * cos(ph);
  *im = w * sin(ph);
}

/* ------------------------------------------------------------------ geometry */
static void tri_verts(const orc_scene* sc, int32_t prim, double a[3], double b[3], double c[3]) {
  const int32_t* t = sc->tris + 3 * (int64_t)prim;
  for (int k = 0; k < 3; ++k) {
    a[k] = sc->verts[3 * (int64_t)t[0] + k];
    b[k] = sc->verts[3 * (int64_t)t[1] + k];
    c[k] = sc->verts[3 * (int64_t)t[2] + k];
  }
}

/* Two-sided ray/triangle test (Moller & Trumbore 1997), inclusive edges. */
static int tri_test(const double o[3], const double d[3], const double a[3], const double b[3],
                    const double c[3], double* t, double* margin) {
  double e1[3], e2[3], p[3], s[3], q[3];
  sub3(b, a, e1);
  sub3(c, a, e2);
  cross3(d, e2, p);
  double det = dot3(e1, p);
  if (det == 0.0) return 0;
  sub3(o, a, s);
  double u = dot3(s, p) / det;
  if (!(u >= 0.0 && u <= 1.0)) return 0;
  cross3(s, e1, q);
  double v = dot3(d, q) / det;
  if (!(v >= 0.0 && u + v <= 1.0)) return 0;
  *t = dot3(e2, q) / det;
  double w = 1.0 - u - v;
  *margin = fmin(u, fmin(v, w));
  return 1;
}

static void tri_normal(const orc_scene* sc, int32_t prim, double n[3]) {
  double a[3], b[3], c[3], e1[3], e2[3];
  tri_verts(sc, prim, a, b, c);
  sub3(b, a, e1);
  sub3(c, a, e2);
  cross3(e1, e2, n);
  double l = norm3(n);
  n[0] /= l; n[1] /= l; n[2] /= l;
}

/* Median-split BVH over triangle centroids, FP64 boxes. */
typedef struct { double lo[3], hi[3]; int32_t left, right, first, count; } bnode;
typedef struct { bnode* nodes; int32_t n_nodes; int32_t* order; double* cent; } bvh_t;

static int cmp_axis_g;
static const double* cmp_cent_g;
static int cmp_prims(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  double ca = cmp_cent_g[3 * (int64_t)a + cmp_axis_g], cb = cmp_cent_g[3 * (int64_t)b + cmp_axis_g];
  if (ca < cb) return -1;
  if (ca > cb) return 1;
  return a < b ? -1 : (a > b);
}

static int32_t bvh_build_rec(bvh_t* bv, const orc_scene* sc, int32_t first, int32_t count) {
  int32_t id = bv->n_nodes++;
  bnode* nd = &bv->nodes[id];
  for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
  double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int32_t i = first; i < first + count; ++i) {
    double a[3], b[3], c[3];
    tri_verts(sc, bv->order[i], a, b, c);
    for (int k = 0; k < 3; ++k) {
      nd->lo[k] = fmin(nd->lo[k], fmin(a[k], fmin(b[k], c[k])));
      nd->hi[k] = fmax(nd->hi[k], fmax(a[k], fmax(b[k], c[k])));
      double ce = bv->cent[3 * (int64_t)bv->order[i] + k];
      clo[k] = fmin(clo[k], ce);
      chi[k] = fmax(chi[k], ce);
    }
  }
  if (count <= 4) {
    nd->left = nd->right = -1;
    nd->first = first;
    nd->count = count;
    return id;
  }
  int axis = 0;
  for (int k = 1; k < 3; ++k)
    if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
  cmp_axis_g = axis;
  cmp_cent_g = bv->cent;
  qsort(bv->order + first, (size_t)count, sizeof(int32_t), cmp_prims);
  int32_t half = count / 2;
  int32_t l = bvh_build_rec(bv, sc, first, half);
  int32_t r = bvh_build_rec(bv, sc, first + half, count - half);
  nd = &bv->nodes[id];
  nd->left = l;
  nd->right = r;
  nd->first = -1;
  nd->count = 0;
  return id;
}

static void bvh_build(bvh_t* bv, const orc_scene* sc) {
  int64_t n = sc->n_tris;
  bv->nodes = (bnode*)malloc(sizeof(bnode) * (size_t)(2 * n + 1));
  bv->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  bv->cent = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
  bv->n_nodes = 0;
  for (int64_t i = 0; i < n; ++i) {
    double a[3], b[3], c[3];
    tri_verts(sc, (int32_t)i, a, b, c);
    bv->order[i] = (int32_t)i;
    for (int k = 0; k < 3; ++k) bv->cent[3 * i + k] = (a[k] + b[k] + c[k]) / 3.0;
  }
  if (n > 0) bvh_build_rec(bv, sc, 0, (int32_t)n);
}
static void bvh_free(bvh_t* bv) {
  free(bv->nodes);
  free(bv->order);
  free(bv->cent);
}

/* Conservative slab test; boxes are padded by a relative 1e-9 so that no hit is lost. */
static int box_test(const double lo[3], const double hi[3], const double o[3], const double d[3],
                    double tmin, double tmax) {
  double t0 = tmin, t1 = tmax;
  for (int k = 0; k < 3; ++k) {
    double pad = 1e-9 * (fabs(lo[k]) + fabs(hi[k]) + 1.0);
    double l = lo[k] - pad, h = hi[k] + pad;
    if (d[k] == 0.0) {
      if (o[k] < l || o[k] > h) return 0;
      continue;
    }
    double ta = (l - o[k]) / d[k], tb = (h - o[k]) / d[k];
    if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
    ta -= 1e-12 * (fabs(ta) + 1.0);
    tb += 1e-12 * (fabs(tb) + 1.0);
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
    if (t0 > t1) return 0;
  }
  return 1;
}

typedef struct {
  double t, margin, t2;
  int32_t prim;
} hitq;

static void consider(hitq* hq, int32_t prim, double t, double margin) {
  if (t < hq->t || (t == hq->t && prim < hq->prim)) {
    hq->t2 = hq->t;
    hq->t = t;
    hq->prim = prim;
    hq->margin = margin;
  } else if (t < hq->t2) {
    hq->t2 = t;
  }
}

/* Nearest hit with t in (tmin, tmax], ties to the lowest prim id; also the runner-up
   distance among all other hits in the same interval. */
static hitq closest(const orc_scene* sc, const bvh_t* bv, const double o[3], const double d[3],
                    double tmin, double tmax, int32_t exclude) {
  hitq hq = {INFINITY, 0.0, INFINITY, -1};
  if (bv == NULL) {
    for (int64_t i = 0; i < sc->n_tris; ++i) {
      if ((int32_t)i == exclude) continue;
      double a[3], b[3], c[3], t, m;
      tri_verts(sc, (int32_t)i, a, b, c);
      if (tri_test(o, d, a, b, c, &t, &m) && t > tmin && t <= tmax) consider(&hq, (int32_t)i, t, m);
    }
    return hq;
  }
  if (bv->n_nodes == 0) return hq;
  int32_t stack[256];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const bnode* nd = &bv->nodes[stack[--sp]];
    double lim = fmin(tmax, hq.t2);
    if (!box_test(nd->lo, nd->hi, o, d, tmin, lim)) continue;
    if (nd->count > 0) {
      for (int32_t i = nd->first; i < nd->first + nd->count; ++i) {
        int32_t prim = bv->order[i];
        if (prim == exclude) continue;
        double a[3], b[3], c[3], t, m;
        tri_verts(sc, prim, a, b, c);
        if (tri_test(o, d, a, b, c, &t, &m) && t > tmin && t <= tmax) consider(&hq, prim, t, m);
      }
    } else {
      stack[sp++] = nd->left;
      stack[sp++] = nd->right;
    }
  }
  return hq;
}

int32_t orc_closest_hit(const orc_scene* sc, const double o[3], const double d[3], double tmin,
                        double tmax, int32_t exclude, int use_bvh, double* t, double* margin,
                        double* t_second) {
  bvh_t bv;
  const bvh_t* pb = NULL;
  if (use_bvh) {
    bvh_build(&bv, sc);
    pb = &bv;
  }
  hitq hq = closest(sc, pb, o, d, tmin, tmax, exclude);
  if (use_bvh) bvh_free(&bv);
  *t = hq.t;
  *margin = hq.margin;
  *t_second = hq.t2;
  return hq.prim;
}

/* ------------------------------------------------------------------ sound-speed profile */
/* Sec. II.A: rays bend by Snell's law in a depth-dependent sound speed. Supported
   profiles: isovelocity (n_ssp <= 1) and one linear gradient c(z) = c0 + g (z - z0)
   through two nodes (z up, extended linearly beyond the nodes). */
typedef struct { double z0, c0, g; int curved; } ssp_t;

static int ssp_make(const double* z, const double* c, int32_t n, double c_default, ssp_t* s) {
  s->z0 = 0.0;
  s->g = 0.0;
  s->curved = 0;
  if (n <= 0) {
    s->c0 = c_default;
    return c_default > 0 ? 0 : 1;
  }
  if (n == 1) {
    s->c0 = c[0];
    return c[0] > 0 ? 0 : 1;
  }
  if (n > 2 || z[1] == z[0]) return 2;
  s->z0 = z[0];
  s->c0 = c[0];
  s->g = (c[1] - c[0]) / (z[1] - z[0]);
  s->curved = s->g != 0.0;
  return 0;
}
static double ssp_c(const ssp_t* s, double z) { return s->c0 + s->g * (z - s->z0); }

/* Exact circular-arc advance by arc length ds in a linear profile (curvature -xi g):
   theta' = theta - xi g ds; horizontal and vertical displacements
   ds cos(theta_m) sinc(delta/2) and ds sin(theta_m) sinc(delta/2), theta_m the mean angle;
   one-way time (atanh(sin theta) - atanh(sin theta'))/g written through
   X = (sin theta - sin theta')/(1 - sin theta sin theta') so that g -> 0 stays finite. */
static void arc_advance(const ssp_t* s, double z, double theta, double xi, double ds,
                        double* dh, double* dz, double* theta_new, double* dt) {
  double delta = xi * s->g * ds;
  double thm = theta - delta / 2;
  double sc = sinc(delta / 2);
  *dh = ds * cos(thm) * sc;
  *dz = ds * sin(thm) * sc;
  *theta_new = theta - delta;
  double cm = cos(thm);
  if (fabs(cos(theta)) < 1e-12) {
    /* vertical ray: straight line, time = ln(c1/c0)/(g sin theta) */
    double c0 = ssp_c(s, z), c1 = ssp_c(s, z + *dz);
    *dt = s->g == 0.0 ? ds / c0 : log(c1 / c0) / (s->g * sin(theta));
    return;
  }
  double sh = sin(delta / 2);
  double x_over_g = cm * xi * ds * sc / (sh * sh + cm * cm);
  double x = s->g * x_over_g;
  double ratio = fabs(x) < 1e-6 ? 1.0 + x * x / 3.0 : atanh(x) / x;
  *dt = ratio * x_over_g;
}

static double arc_step(const ssp_t* s, double xi) {
  double k = xi * fabs(s->g);
  if (k <= 0.0) return ARC_H_MAX;
  return fmin(ARC_H_MAX, sqrt(8.0 / k * ARC_EPS_SAGITTA));
}

/* Decompose a unit direction into horizontal unit e and grazing angle theta. */
static void dir_split(const double d[3], double e[2], double* theta) {
  double hz = sqrt(d[0] * d[0] + d[1] * d[1]);
  if (hz > 0) {
    e[0] = d[0] / hz;
    e[1] = d[1] / hz;
  } else {
    e[0] = 1.0;
    e[1] = 0.0;
  }
  *theta = atan2(d[2], hz);
}

void orc_arc_nodes(const double* ssp_z, const double* ssp_cc, int32_t n_ssp, const double o[3],
                   const double d[3], double h, int32_t n_nodes, double* pos, double* times,
                   double* theta_out) {
  ssp_t s;
  ssp_make(ssp_z, ssp_cc, n_ssp, 1500.0, &s);
  double p[3] = {o[0], o[1], o[2]}, e[2], th, T = 0;
  dir_split(d, e, &th);
  double xi = cos(th) / ssp_c(&s, p[2]);
  for (int32_t i = 0; i < n_nodes; ++i) {
    pos[3 * i] = p[0]; pos[3 * i + 1] = p[1]; pos[3 * i + 2] = p[2];
    times[i] = T;
    theta_out[i] = th;
    double dh, dz, thn, dt;
    arc_advance(&s, p[2], th, xi, h, &dh, &dz, &thn, &dt);
    p[0] += dh * e[0];
    p[1] += dh * e[1];
    p[2] += dz;
    th = thn;
    T += dt;
  }
}

/* Eigen-arc between o and x: the circle through both points whose centre lies on the
   height where the linear profile reaches c = 0 (every ray of a linear profile is such
   a circle). */
int orc_eigen_arc(const double* ssp_z, const double* ssp_cc, int32_t n_ssp, const double o[3],
                  const double x[3], double d_out[3], double* t_out, double* s_out) {
  ssp_t s;
  if (ssp_make(ssp_z, ssp_cc, n_ssp, 1500.0, &s) != 0 || !s.curved) return 1;
  double dx = x[0] - o[0], dy = x[1] - o[1];
  double D = sqrt(dx * dx + dy * dy);
  double co = ssp_c(&s, o[2]), cx = ssp_c(&s, x[2]);
  if (D == 0.0) {
    double dz = x[2] - o[2];
    d_out[0] = 0; d_out[1] = 0; d_out[2] = dz > 0 ? 1.0 : -1.0;
    *t_out = log(cx / co) / (s.g * d_out[2]);
    *s_out = fabs(dz);
    return 0;
  }
  double e[2] = {dx / D, dy / D};
  double a = co / s.g, b = cx / s.g; /* heights above the c = 0 line */
  double hc = (D * D + b * b - a * a) / (2 * D);
  double R = sqrt(hc * hc + a * a);
  double sg = s.g > 0 ? 1.0 : -1.0;
  double th0 = atan2(sg * hc, sg * a);
  double th1 = atan2(sg * (hc - D), sg * b);
  d_out[0] = cos(th0) * e[0];
  d_out[1] = cos(th0) * e[1];
  d_out[2] = sin(th0);
  double s0 = sin(th0), s1 = sin(th1);
  double X = (s0 - s1) / (1 - s0 * s1);
  *t_out = atanh(X) / s.g;
  /* arc length: radius times the angle between the radii to o and to x */
  double r0[2] = {-hc, a}, r1[2] = {D - hc, b};
  double ang = atan2(fabs(r0[0] * r1[1] - r0[1] * r1[0]), r0[0] * r1[0] + r0[1] * r1[1]);
  *s_out = R * ang;
  return 0;
}

/* ------------------------------------------------------------------ hit list */
typedef struct {
  int32_t ray, sub, seg, prim;
  double tau, len, amp, psi, phi, u[3], margin, gap;
  double kinc, gam;  /* incidence cosine at a mesh facet, one-way reflection product */
} ohit;
typedef struct { ohit* v; int64_t n, cap; } hbuf;
static void hb_push(hbuf* b, const ohit* h) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 16;
    b->v = (ohit*)realloc(b->v, sizeof(ohit) * (size_t)b->cap);
  }
  b->v[b->n++] = *h;
}

typedef struct {
  const orc_scene* sc;
  const orc_params* p;
  const bvh_t* bv;
  ssp_t ssp;
  double c_ref, T_stop, R[9], t[3];
  uint32_t s32;
  int has_surface;
} tctx;

/* Sec. II.B per-hit backscatter: Lambertian intensity mu cos^2(k) over the footprint
   L^2 dOmega / cos(k) gives amplitude Gamma^2 sqrt(mu cos(k) dOmega)/L, two-way
   attenuation exp(-2 alpha L); speckle phase psi uniform from the hash; carrier phase
   set by the two-way delay: c = a exp(j (psi - 2 pi frac(f0 tau))). */
static void emit_mesh_hit(const tctx* c, hbuf* hb, int32_t ray, int32_t sub, int32_t seg,
                          int32_t prim, double T_oneway, double L, double gam, double kinc,
                          double dOmega, const double us[3], double margin, double gap) {
  ohit h = {0};
  h.ray = ray; h.sub = sub; h.seg = seg; h.prim = prim;
  h.tau = 2.0 * T_oneway;
  h.len = L;
  double mu = c->sc->mu[prim];
  h.amp = gam * gam * sqrt(mu * kinc * dOmega) / L * exp(-2.0 * c->p->alpha * L);
  h.kinc = kinc;
  h.gam = gam;
  uint32_t v[4] = {(uint32_t)ray, (uint32_t)sub, (uint32_t)(1 + seg), c->s32};
  orc_pcg4d(v);
  h.psi = TWO_PI * u24(v[0]);
  h.phi = wrap_pi(h.psi - TWO_PI * frac(c->p->f0 * h.tau));
  h.u[0] = us[0]; h.u[1] = us[1]; h.u[2] = us[2];
  h.margin = margin;
  h.gap = gap;
  hb_push(hb, &h);
}

static void reflect(double d[3], const double n[3]) {
  double k = 2.0 * dot3(d, n);
  d[0] -= k * n[0]; d[1] -= k * n[1]; d[2] -= k * n[2];
}

/* Cross-term multipath of a mesh hit reached after one or more reflections (Sec. II.B
   multi-bounce paths, extended to routes whose outgoing and returning legs differ):
   out along the route and back on the straight line to the array, and the reciprocal
   path (out straight, back along the route). The route's ray tube samples the surface
   with footprint L^2 dOmega / cos(k_route); bistatic Lambertian scattering
   mu cos(k_in) cos(k_out) over it, spread over L^2 on the route and L_d^2 on the straight
   leg, leaves the amplitude Gamma sqrt(mu cos(k_d) dOmega) / L_d exp(-alpha (L + L_d))
   for either path, with Gamma the route's one-way reflection product and delay
   (L + L_d) / c. The straight leg must reach the facet from the side the route arrives
   on and pass no other triangle closer than L_d - CROSS_CLEAR. Both paths share one
   speckle phase (reciprocity), keyed apart from the route's own. seg carries the
   bounce count plus 16 (returns straight, arrives from the hit's direction) or 32
   (returns along the route, arrives along the launch direction). */
#define CROSS_CLEAR 1e-4
static void cross_mesh(const tctx* c, hbuf* hb, int32_t ray, int32_t sub, int32_t seg, int32_t prim,
                       const double x[3], double L, double gam, const double dir[3], const double n[3],
                       double dOmega, const double us[3], double margin, double gap) {
  const orc_params* p = c->p;
  double v[3];
  sub3(x, c->t, v);
  double Ld = norm3(v);
  if (!(Ld > CROSS_CLEAR)) return;
  double tau = (L + Ld) / c->ssp.c0;
  if (!(tau <= 2.0 * c->T_stop)) return;
  double vn = dot3(v, n);
  if (!(dot3(dir, n) * vn > 0)) return;
  double ud[3] = {v[0] / Ld, v[1] / Ld, v[2] / Ld};
  hitq sh = closest(c->sc, c->bv, c->t, ud, EPS_HIT, Ld - CROSS_CLEAR, prim);
  if (sh.prim >= 0) return;
  ohit h = {0};
  h.ray = ray; h.sub = sub; h.prim = prim;
  h.tau = tau;
  h.len = 0.5 * (L + Ld);
  h.amp = gam * sqrt(c->sc->mu[prim] * (fabs(vn) / Ld) * dOmega) / Ld * exp(-p->alpha * (L + Ld));
  uint32_t k[4] = {(uint32_t)ray, (uint32_t)sub, (uint32_t)(9 + seg), c->s32};
  orc_pcg4d(k);
  h.psi = TWO_PI * u24(k[0]);
  h.phi = wrap_pi(h.psi - TWO_PI * frac(p->f0 * h.tau));
  h.margin = margin;
  h.gap = gap;
  h.seg = seg | 16;
  mat_t_vec(c->R, ud, h.u);
  hb_push(hb, &h);
  h.seg = seg | 32;
  h.u[0] = us[0]; h.u[1] = us[1]; h.u[2] = us[2];
  hb_push(hb, &h);
}

/* Isovelocity route (Sec. II.A ray casting, Sec. II.B limited secondary reflections):
   straight segments; a triangle hit scatters and, when the triangle is a specular
   mirror and bounces remain, the ray reflects about the geometric normal; the sea
   surface only reflects. Stops at the one-way time T_stop. */
static void route_straight(const tctx* c, const double o[3], const double d0[3], const double us[3],
                           int32_t ray, int32_t sub, double dOmega, hbuf* hb) {
  const orc_params* p = c->p;
  double cw = c->ssp.c0;
  double L_stop = c->T_stop * cw;
  double pos[3] = {o[0], o[1], o[2]}, dir[3] = {d0[0], d0[1], d0[2]};
  double L = 0.0, gam = 1.0;
  int32_t bounce = 0, prev = -1;
  for (;;) {
    double tlim = L_stop - L;
    if (!(tlim > 0)) break;
    hitq hq = closest(c->sc, c->bv, pos, dir, EPS_HIT, tlim, prev);
    double ts = INFINITY;
    if (c->has_surface && prev != -2 && dir[2] != 0.0) {
      double t = (p->surface_z - pos[2]) / dir[2];
      if (t > EPS_HIT && t <= tlim) ts = t;
    }
    if (hq.prim < 0 && ts == INFINITY) break;
    if (ts < hq.t) {
      if (bounce >= p->max_bounces) break;
      for (int k = 0; k < 3; ++k) pos[k] += ts * dir[k];
      L += ts;
      dir[2] = -dir[2];
      gam *= p->r_surface;
      bounce++;
      prev = -2;
      continue;
    }
    double n[3];
    tri_normal(c->sc, hq.prim, n);
    for (int k = 0; k < 3; ++k) pos[k] += hq.t * dir[k];
    L += hq.t;
    double kinc = fabs(dot3(dir, n));
    emit_mesh_hit(c, hb, ray, sub, bounce, hq.prim, L / cw, L, gam, kinc, dOmega, us, hq.margin,
                  hq.t2 - hq.t);
    if (p->cross && bounce > 0)
      cross_mesh(c, hb, ray, sub, bounce, hq.prim, pos, L, gam, dir, n, dOmega, us, hq.margin, hq.t2 - hq.t);
    if ((c->sc->flags[hq.prim] & 1) && bounce < p->max_bounces) {
      reflect(dir, n);
      gam *= p->r_seabed;
      bounce++;
      prev = hq.prim;
      continue;
    }
    break;
  }
}

/* Refracting route in a linear profile: the ray is an exact circular arc, intersected
   as chords between arc nodes spaced h = min(h_max, sqrt(8 R eps)) (sagitta <= eps);
   the hit time interpolates the node times linearly in the chord fraction. A specular
   reflection reflects the arc tangent at the hit; the Snell invariant is recomputed. */
static void route_curved(const tctx* c, const double o[3], const double d0[3], const double us[3],
                         int32_t ray, int32_t sub, double dOmega, hbuf* hb) {
  const orc_params* p = c->p;
  const ssp_t* s = &c->ssp;
  double pos[3] = {o[0], o[1], o[2]}, e[2], th;
  dir_split(d0, e, &th);
  double xi = cos(th) / ssp_c(s, pos[2]);
  double T = 0.0, sarc = 0.0, gam = 1.0;
  int32_t bounce = 0, prev = -1;
  for (int iter = 0; iter < 1000000; ++iter) {
    if (!(T < c->T_stop)) break;
    double h = arc_step(s, xi);
    double dh, dz, thn, dt;
    arc_advance(s, pos[2], th, xi, h, &dh, &dz, &thn, &dt);
    double nxt[3] = {pos[0] + dh * e[0], pos[1] + dh * e[1], pos[2] + dz};
    double ch[3];
    sub3(nxt, pos, ch);
    double len = norm3(ch);
    double dc[3] = {ch[0] / len, ch[1] / len, ch[2] / len};
    hitq hq = closest(c->sc, c->bv, pos, dc, EPS_HIT, len, prev >= 0 ? prev : -1);
    double ts = INFINITY;
    if (c->has_surface && prev != -2 && dc[2] != 0.0) {
      double t = (p->surface_z - pos[2]) / dc[2];
      if (t > EPS_HIT && t <= len) ts = t;
    }
    if (hq.prim < 0 && ts == INFINITY) {
      pos[0] = nxt[0]; pos[1] = nxt[1]; pos[2] = nxt[2];
      th = thn;
      T += dt;
      sarc += h;
      prev = -1;
      continue;
    }
    int surf = ts < hq.t;
    double thit = surf ? ts : hq.t;
    double f = thit / len;
    double T_hit = T + f * dt, s_hit = sarc + f * h;
    if (!(T_hit <= c->T_stop)) break;
    double hp[3] = {pos[0] + thit * dc[0], pos[1] + thit * dc[1], pos[2] + thit * dc[2]};
    double n[3];
    if (surf) {
      if (bounce >= p->max_bounces) break;
      n[0] = 0; n[1] = 0; n[2] = 1;
      gam *= p->r_surface;
    } else {
      tri_normal(c->sc, hq.prim, n);
      double kinc = fabs(dot3(dc, n));
      emit_mesh_hit(c, hb, ray, sub, bounce, hq.prim, T_hit, s_hit, gam, kinc, dOmega, us,
                    hq.margin, hq.t2 - hq.t);
      if (!((c->sc->flags[hq.prim] & 1) && bounce < p->max_bounces)) break;
      gam *= p->r_seabed;
    }
    /* reflect the arc tangent at the hit point */
    double thh = th - xi * s->g * (f * h);
    double tg[3] = {cos(thh) * e[0], cos(thh) * e[1], sin(thh)};
    reflect(tg, n);
    dir_split(tg, e, &th);
    pos[0] = hp[0]; pos[1] = hp[1]; pos[2] = hp[2];
    xi = cos(th) / ssp_c(s, pos[2]);
    T = T_hit;
    sarc = s_hit;
    bounce++;
    prev = surf ? -2 : hq.prim;
  }
}

/* Shadow test of the straight leg a -> b against the mesh (endpoints excluded). */
static int leg_clear(const tctx* c, const double a[3], const double b[3]) {
  double d[3];
  sub3(b, a, d);
  double len = norm3(d);
  if (len <= 2e-6) return 1;
  d[0] /= len; d[1] /= len; d[2] /= len;
  hitq hq = closest(c->sc, c->bv, a, d, 1e-6, len - 1e-6, -1);
  return hq.prim < 0;
}

static void mirror_point(const double pl[4], const double x[3], double r[3]) {
  double k = 2.0 * (pl[0] * x[0] + pl[1] * x[1] + pl[2] * x[2] - pl[3]);
  r[0] = x[0] - k * pl[0]; r[1] = x[1] - k * pl[1]; r[2] = x[2] - k * pl[2];
}

/* ------------------------------------------------------------------ 2-D sound-speed field */
/* Sec. II.A rays bent by a range- and depth-dependent sound speed (Snell's law in its
   continuous form). c(x, z) comes from a regular grid, bilinear in each cell; positions
   outside the grid are clamped to it, so c is constant outward and the gradient
   component across a clamped axis is zero. Returns c and (dc/dx, dc/dz). */
static void field_eval(const orc_params* p, double x, double z, double* c, double* cx, double* cz) {
  const int32_t nx = p->fld_nx, nz = p->fld_nz;
  double fx = (x - p->fld_x0) / p->fld_dx, fz = (z - p->fld_z0) / p->fld_dz;
  int inx = 1, inz = 1;
  if (fx < 0.0) { fx = 0.0; inx = 0; } else if (fx > nx - 1) { fx = nx - 1; inx = 0; }
  if (fz < 0.0) { fz = 0.0; inz = 0; } else if (fz > nz - 1) { fz = nz - 1; inz = 0; }
  int32_t i = (int32_t)floor(fx), j = (int32_t)floor(fz);
  if (i > nx - 2) i = nx - 2;
  if (j > nz - 2) j = nz - 2;
  const double u = fx - i, v = fz - j;
  const double* C = p->fld_c;
  const double c00 = C[j * nx + i], c10 = C[j * nx + i + 1];
  const double c01 = C[(j + 1) * nx + i], c11 = C[(j + 1) * nx + i + 1];
  *c = (1.0 - u) * (1.0 - v) * c00 + u * (1.0 - v) * c10 + (1.0 - u) * v * c01 + u * v * c11;
  *cx = inx ? ((1.0 - v) * (c10 - c00) + v * (c11 - c01)) / p->fld_dx : 0.0;
  *cz = inz ? ((1.0 - u) * (c01 - c00) + u * (c11 - c10)) / p->fld_dz : 0.0;
}

/* Ray equations in arc length s for the state (r, t, T), t the unit tangent:
   dr/ds = t, dt/ds = ((grad c . t) t - grad c) / c, dT/ds = 1 / c. */
static void field_deriv(const orc_params* p, const double y[7], double f[7]) {
  double c, cx, cz;
  field_eval(p, y[0], y[2], &c, &cx, &cz);
  const double gt = cx * y[3] + cz * y[5];
  f[0] = y[3];
  f[1] = y[4];
  f[2] = y[5];
  f[3] = (gt * y[3] - cx) / c;
  f[4] = gt * y[4] / c;
  f[5] = (gt * y[5] - cz) / c;
  f[6] = 1.0 / c;
}

/* One classical Runge-Kutta step of length h, the tangent renormalised after it. */
static void rk4_step(const orc_params* p, const double y[7], double h, double out[7]) {
  double k1[7], k2[7], k3[7], k4[7], tmp[7];
  field_deriv(p, y, k1);
  for (int i = 0; i < 7; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
  field_deriv(p, tmp, k2);
  for (int i = 0; i < 7; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
  field_deriv(p, tmp, k3);
  for (int i = 0; i < 7; ++i) tmp[i] = y[i] + h * k3[i];
  field_deriv(p, tmp, k4);
  for (int i = 0; i < 7; ++i) out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  const double n = sqrt(out[3] * out[3] + out[4] * out[4] + out[5] * out[5]);
  out[3] /= n;
  out[4] /= n;
  out[5] /= n;
}

int orc_field_ray(const orc_params* p, const double o[3], const double d[3], double h, int32_t n, double out[7]) {
  if (p->fld_nx < 2 || p->fld_nz < 2 || !(p->fld_dx > 0) || !(p->fld_dz > 0) || !p->fld_c || n < 0) return 5;
  double y[7] = {o[0], o[1], o[2], d[0], d[1], d[2], 0.0};
  for (int32_t k = 0; k < n; ++k) {
    double yn[7];
    rk4_step(p, y, h, yn);
    for (int i = 0; i < 7; ++i) y[i] = yn[i];
  }
  for (int i = 0; i < 7; ++i) out[i] = y[i];
  return 0;
}

/* Route in a 2-D field: RK4 steps of fld_h; the chord of each step is intersected with
   the scene and the sea surface like the chords of a circular arc. A hit's time and arc
   length interpolate the step's end values linearly in the chord fraction f; at a
   reflection the tangent is (1 - f) t_i + f t_i+1, normalised, reflected about the
   normal. */
static void route_field(const tctx* c, const double o[3], const double d0[3], const double us[3],
                        int32_t ray, int32_t sub, double dOmega, hbuf* hb) {
  const orc_params* p = c->p;
  double y[7] = {o[0], o[1], o[2], d0[0], d0[1], d0[2], 0.0};
  double sarc = 0.0, gam = 1.0;
  int32_t bounce = 0, prev = -1;
  for (int iter = 0; iter < 1000000; ++iter) {
    if (!(y[6] < c->T_stop)) break;
    double yn[7];
    rk4_step(p, y, p->fld_h, yn);
    double ch[3] = {yn[0] - y[0], yn[1] - y[1], yn[2] - y[2]};
    const double len = norm3(ch);
    if (!(len > 0)) break;
    const double dc[3] = {ch[0] / len, ch[1] / len, ch[2] / len};
    hitq hq = closest(c->sc, c->bv, y, dc, EPS_HIT, len, prev >= 0 ? prev : -1);
    double ts = INFINITY;
    if (c->has_surface && prev != -2 && dc[2] != 0.0) {
      const double t = (p->surface_z - y[2]) / dc[2];
      if (t > EPS_HIT && t <= len) ts = t;
    }
    if (hq.prim < 0 && ts == INFINITY) {
      for (int i = 0; i < 7; ++i) y[i] = yn[i];
      sarc += p->fld_h;
      prev = -1;
      continue;
    }
    const int surf = ts < hq.t;
    const double thit = surf ? ts : hq.t;
    const double f = thit / len;
    const double T_hit = y[6] + f * (yn[6] - y[6]), s_hit = sarc + f * p->fld_h;
    if (!(T_hit <= c->T_stop)) break;
    const double hp[3] = {y[0] + thit * dc[0], y[1] + thit * dc[1], y[2] + thit * dc[2]};
    double n[3];
    if (surf) {
      if (bounce >= p->max_bounces) break;
      n[0] = 0; n[1] = 0; n[2] = 1;
      gam *= p->r_surface;
    } else {
      tri_normal(c->sc, hq.prim, n);
      const double kinc = fabs(dot3(dc, n));
      emit_mesh_hit(c, hb, ray, sub, bounce, hq.prim, T_hit, s_hit, gam, kinc, dOmega, us, hq.margin,
                    hq.t2 - hq.t);
      if (!((c->sc->flags[hq.prim] & 1) && bounce < p->max_bounces)) break;
      gam *= p->r_seabed;
    }
    double tg[3];
    for (int k = 0; k < 3; ++k) tg[k] = (1.0 - f) * y[3 + k] + f * yn[3 + k];
    const double tn = norm3(tg);
    for (int k = 0; k < 3; ++k) tg[k] /= tn;
    reflect(tg, n);
    for (int k = 0; k < 3; ++k) {
      y[k] = hp[k];
      y[3 + k] = tg[k];
    }
    y[6] = T_hit;
    sarc = s_hit;
    bounce++;
    prev = surf ? -2 : hq.prim;
  }
}

/* Point scatterers: monostatic image-source eigen-routes (Sec. II.B limited secondary
   reflections). Mirror planes: the sea surface (reflection r_surface) then the scene's
   planes (reflection r_seabed). Routes are plane sequences without immediate repeats,
   enumerated by length then lexicographically; each leg is shadow-tested. Amplitude
   sigma Gamma^2 / L^2, no speckle. With cross terms every ordered pair (i, j) of distinct
   valid routes adds the path out along i and back along j: delay (L_i + L_j) / c,
   amplitude sigma Gamma_i Gamma_j / (L_i L_j) exp(-alpha (L_i + L_j)), arriving along
   route j; sub = 0x10000 | i << 8 | j (route indices), seg = the total reflections. */
static void point_routes(const tctx* c, hbuf* hb) {
  const orc_scene* sc = c->sc;
  const orc_params* p = c->p;
  int np = (c->has_surface ? 1 : 0) + (int)sc->n_planes;
  double planes[64][4], gams[64];
  if (np > 64) np = 64;
  int q = 0;
  if (c->has_surface) {
    planes[q][0] = 0; planes[q][1] = 0; planes[q][2] = 1; planes[q][3] = p->surface_z;
    gams[q++] = p->r_surface;
  }
  for (int64_t i = 0; i < sc->n_planes && q < np; ++i, ++q) {
    for (int k = 0; k < 4; ++k) planes[q][k] = sc->planes[4 * i + k];
    gams[q] = p->r_seabed;
  }
  int maxb = p->max_bounces > 3 ? 3 : p->max_bounces;
  for (int64_t ip = 0; ip < sc->n_points; ++ip) {
    double x[3] = {sc->points[3 * ip], sc->points[3 * ip + 1], sc->points[3 * ip + 2]};
    double sigma = sc->sigma[ip];
    if (c->ssp.curved) {
      /* linear profile: direct eigen-arc only */
      double dw[3], T, sarc;
      double zz[2] = {c->ssp.z0, c->ssp.z0 + 1.0}, cc[2] = {c->ssp.c0, c->ssp.c0 + c->ssp.g};
      if (orc_eigen_arc(zz, cc, 2, c->t, x, dw, &T, &sarc) != 0) continue;
      if (!(T <= c->T_stop)) continue;
      /* shadow test along chords of the arc */
      double pos[3] = {c->t[0], c->t[1], c->t[2]}, e[2], th;
      dir_split(dw, e, &th);
      double xi = cos(th) / ssp_c(&c->ssp, pos[2]);
      double left = sarc;
      int clear = 1;
      while (left > 0 && clear) {
        double h = fmin(arc_step(&c->ssp, xi), left);
        double dh, dz, thn, dt;
        arc_advance(&c->ssp, pos[2], th, xi, h, &dh, &dz, &thn, &dt);
        double nxt[3] = {pos[0] + dh * e[0], pos[1] + dh * e[1], pos[2] + dz};
        if (left - h <= 0) { nxt[0] = x[0]; nxt[1] = x[1]; nxt[2] = x[2]; }
        clear = leg_clear(c, pos, nxt);
        pos[0] = nxt[0]; pos[1] = nxt[1]; pos[2] = nxt[2];
        th = thn;
        left -= h;
      }
      if (!clear) continue;
      ohit h = {0};
      h.ray = (int32_t)ip; h.sub = 0; h.seg = 0; h.prim = -1;
      h.tau = 2.0 * T;
      h.len = sarc;
      h.amp = sigma / (sarc * sarc) * exp(-2.0 * p->alpha * sarc);
      h.psi = 0.0;
      h.phi = wrap_pi(-TWO_PI * frac(p->f0 * h.tau));
      mat_t_vec(c->R, dw, h.u);
      h.margin = INFINITY;
      h.gap = INFINITY;
      hb_push(hb, &h);
      continue;
    }
    int32_t route = 0;
    struct { int32_t idx, len; double L, gam, u[3]; } pr[256];
    int npr = 0;
    for (int len = 0; len <= maxb; ++len) {
      int64_t count = len == 0 ? 1 : np;
      for (int k = 1; k < len; ++k) count *= (np - 1);
      if (len > 0 && np == 0) count = 0;
      for (int64_t r = 0; r < count; ++r, ++route) {
        int seq[4];
        int64_t rem = r, div = 1;
        for (int k = 1; k < len; ++k) div *= (np - 1);
        for (int k = 0; k < len; ++k) {
          int64_t digit = rem / div;
          rem %= div;
          if (k + 1 < len) div /= (np - 1);
          if (k == 0) seq[k] = (int)digit;
          else seq[k] = (int)digit < seq[k - 1] ? (int)digit : (int)digit + 1;
        }
        double img[3] = {x[0], x[1], x[2]};
        double gam = 1.0;
        for (int k = len - 1; k >= 0; --k) {
          mirror_point(planes[seq[k]], img, img);
          gam *= gams[seq[k]];
        }
        double dv[3];
        sub3(img, c->t, dv);
        double L = norm3(dv);
        if (!(L > 0) || !(L / c->ssp.c0 <= c->T_stop)) continue;
        /* walk the unfolded route: reflection points in order */
        double a[3] = {c->t[0], c->t[1], c->t[2]}, tgt[3] = {img[0], img[1], img[2]};
        int ok = 1;
        for (int k = 0; k < len && ok; ++k) {
          const double* pl = planes[seq[k]];
          double da = pl[0] * a[0] + pl[1] * a[1] + pl[2] * a[2] - pl[3];
          double dt_ = pl[0] * tgt[0] + pl[1] * tgt[1] + pl[2] * tgt[2] - pl[3];
          if (!(da * dt_ < 0)) { ok = 0; break; }
          double f = da / (da - dt_);
          double sp[3] = {a[0] + f * (tgt[0] - a[0]), a[1] + f * (tgt[1] - a[1]), a[2] + f * (tgt[2] - a[2])};
          if (!leg_clear(c, a, sp)) { ok = 0; break; }
          mirror_point(pl, tgt, tgt);
          a[0] = sp[0]; a[1] = sp[1]; a[2] = sp[2];
        }
        if (!ok || !leg_clear(c, a, x)) continue;
        ohit h = {0};
        h.ray = (int32_t)ip; h.sub = route; h.seg = len; h.prim = -1;
        h.tau = 2.0 * L / c->ssp.c0;
        h.len = L;
        h.amp = sigma * gam * gam / (L * L) * exp(-2.0 * p->alpha * L);
        h.psi = 0.0;
        h.phi = wrap_pi(-TWO_PI * frac(p->f0 * h.tau));
        double dw[3] = {dv[0] / L, dv[1] / L, dv[2] / L};
        mat_t_vec(c->R, dw, h.u);
        h.margin = INFINITY;
        h.gap = INFINITY;
        hb_push(hb, &h);
        if (p->cross && npr < 256) {
          pr[npr].idx = route; pr[npr].len = len; pr[npr].L = L; pr[npr].gam = gam;
          for (int k = 0; k < 3; ++k) pr[npr].u[k] = h.u[k];
          ++npr;
        }
      }
    }
    for (int i = 0; i < npr; ++i)
      for (int j = 0; j < npr; ++j) {
        if (i == j) continue;
        ohit h = {0};
        h.ray = (int32_t)ip; h.sub = 0x10000 | (pr[i].idx << 8) | pr[j].idx;
        h.seg = pr[i].len + pr[j].len; h.prim = -1;
        double Ls = pr[i].L + pr[j].L;
        h.tau = Ls / c->ssp.c0;
        h.len = 0.5 * Ls;
        h.amp = sigma * pr[i].gam * pr[j].gam / (pr[i].L * pr[j].L) * exp(-p->alpha * Ls);
        h.psi = 0.0;
        h.phi = wrap_pi(-TWO_PI * frac(p->f0 * h.tau));
        for (int k = 0; k < 3; ++k) h.u[k] = pr[j].u[k];
        h.margin = INFINITY;
        h.gap = INFINITY;
        hb_push(hb, &h);
      }
  }
}

/* Water-column (volume) reverberation (Sec. II.B volumetric backscatter paths, Sec. V
   clutter): vol_n point scatterers frozen in the world frame, uniform in the box
   [vol_lo, vol_hi]; the i-th sits at lo + (hi - lo) u, u the first three 24-bit
   fractions of pcg4d(i mod 2^32, i div 2^32, 0x564F4C, seed). Each has the amplitude
   coefficient sigma = sqrt(s_v V / n), V the box volume, so that the backscattering
   cross-section per unit volume is s_v, and echoes on its direct route when the leg is
   clear: amplitude sigma / L^2 exp(-2 alpha L), delay 2 L / c, no speckle phase (the
   random positions make the speckle). ray = i, sub = 0x20000. */
static void volume_scatter(const tctx* c, int64_t i0, int64_t i1, hbuf* hb) {
  const orc_params* p = c->p;
  double V = 1.0;
  for (int k = 0; k < 3; ++k) V *= p->vol_hi[k] - p->vol_lo[k];
  const double sigma = sqrt(p->vol_sv * V / (double)p->vol_n);
  const double L_stop = c->T_stop * c->ssp.c0;
  for (int64_t i = i0; i < i1; ++i) {
    uint32_t v[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0x564F4Cu, c->s32};
    orc_pcg4d(v);
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = p->vol_lo[k] + (p->vol_hi[k] - p->vol_lo[k]) * u24(v[k]);
    double dv[3];
    sub3(x, c->t, dv);
    double L = norm3(dv);
    if (!(L > 0) || !(L <= L_stop)) continue;
    if (!leg_clear(c, c->t, x)) continue;
    ohit h = {0};
    h.ray = (int32_t)i; h.sub = 0x20000; h.seg = 0; h.prim = -1;
    h.tau = 2.0 * L / c->ssp.c0;
    h.len = L;
    h.amp = sigma / (L * L) * exp(-2.0 * p->alpha * L);
    h.psi = 0.0;
    h.phi = wrap_pi(-TWO_PI * frac(p->f0 * h.tau));
    double dw[3] = {dv[0] / L, dv[1] / L, dv[2] / L};
    mat_t_vec(c->R, dw, h.u);
    h.margin = INFINITY;
    h.gap = INFINITY;
    hb_push(hb, &h);
  }
}

int orc_trace(const orc_scene* sc, const orc_params* p, const double pose_t[3], const double pose_q[4],
              const double* ssp_z, const double* ssp_cc, int32_t n_ssp, int use_bvh, orc_hits* out) {
  tctx c;
  memset(&c, 0, sizeof(c));
  c.sc = sc;
  c.p = p;
  if (p->n_sub != 1 && p->n_sub != 4) return 3;
  if (ssp_make(ssp_z, ssp_cc, n_ssp, p->c_ref, &c.ssp) != 0) return 2;
  const int field = p->fld_nx > 0;
  if (field) {
    if (p->fld_nx < 2 || p->fld_nz < 2 || !(p->fld_dx > 0) || !(p->fld_dz > 0) || !(p->fld_h > 0) || !p->fld_c)
      return 5;
    for (int64_t k = 0; k < (int64_t)p->fld_nx * p->fld_nz; ++k)
      if (!(p->fld_c[k] > 0)) return 5;
    if (p->cross || p->vol_n > 0) return 4; /* field routes carry no cross terms or volume */
  }
  if (p->cross && c.ssp.curved) return 4; /* cross terms are formed for isovelocity routes only */
  if (p->vol_n < 0 || p->vol_n > (1LL << 28)) return 5;
  if (p->vol_n > 0) {
    if (c.ssp.curved) return 4; /* volume scatterers: isovelocity direct routes only */
    for (int k = 0; k < 3; ++k)
      if (!(p->vol_hi[k] > p->vol_lo[k]) || !(p->vol_sv >= 0)) return 5;
  }
  c.c_ref = p->c_ref > 0 ? p->c_ref : ssp_c(&c.ssp, pose_t[2]);
  if (field && !(p->c_ref > 0)) {
    double gx, gz;
    field_eval(p, pose_t[0], pose_t[2], &c.c_ref, &gx, &gz);
  }
  /* one-way time after which no echo reaches the last range sample */
  c.T_stop = p->r_max / c.c_ref + p->pulse / 2.0;
  double qn = sqrt(pose_q[0] * pose_q[0] + pose_q[1] * pose_q[1] + pose_q[2] * pose_q[2] + pose_q[3] * pose_q[3]);
  double q[4] = {pose_q[0] / qn, pose_q[1] / qn, pose_q[2] / qn, pose_q[3] / qn};
  quat_to_matrix(q, c.R);
  c.t[0] = pose_t[0]; c.t[1] = pose_t[1]; c.t[2] = pose_t[2];
  c.s32 = seed32(p->seed);
  c.has_surface = !isnan(p->surface_z);
  bvh_t bv;
  if (use_bvh) {
    bvh_build(&bv, sc);
    c.bv = &bv;
  }
  out->c_ref = c.c_ref;

  /* Sec. III Eq. 2-3 sampling grid, cell-centred: n_ray_az x n_ray_el cells over the
     fields of view; n_sub = 4 splits a cell into 2x2 quarters, each sampled at a
     hash-jittered point. */
  const int32_t nra = p->n_ray_az, nre = p->n_ray_el;
  const double daz = p->hfov / nra, del = p->vfov / nre;
  /* rows: one per elevation row of rays, the point scatterers, then the volume
     scatterers in chunks (kept in index order) */
  const int32_t nvc = p->vol_n > 0 ? 64 : 0;
  const int32_t nrows = nre + 1 + nvc;
  hbuf* rows = (hbuf*)calloc((size_t)nrows, sizeof(hbuf));
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < nre; ++j) {
    double el_lo = -p->vfov / 2 + j * del, el_hi = el_lo + del;
    double dOmega = daz * (sin(el_hi) - sin(el_lo)) / p->n_sub;
    for (int32_t i = 0; i < nra; ++i) {
      int32_t ray = j * nra + i;
      for (int32_t s = 0; s < p->n_sub; ++s) {
        double ox = 0.0, oy = 0.0;
        if (p->n_sub == 4) {
          uint32_t v[4] = {(uint32_t)ray, (uint32_t)s, 0u, c.s32};
          orc_pcg4d(v);
          ox = ((s & 1) + u24(v[0])) / 2.0 - 0.5;
          oy = ((s >> 1) + u24(v[1])) / 2.0 - 0.5;
        }
        double az = -p->hfov / 2 + (i + 0.5 + ox) * daz;
        double el = -p->vfov / 2 + (j + 0.5 + oy) * del;
        double us[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
        double dw[3];
        mat_vec(c.R, us, dw);
        if (p->fld_nx > 0) route_field(&c, c.t, dw, us, ray, s, dOmega, &rows[j]);
        else if (c.ssp.curved) route_curved(&c, c.t, dw, us, ray, s, dOmega, &rows[j]);
        else route_straight(&c, c.t, dw, us, ray, s, dOmega, &rows[j]);
      }
    }
  }
  if (!field) point_routes(&c, &rows[nre]); /* no eigen-ray search in a 2-D field */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t q = 0; q < nvc; ++q)
    volume_scatter(&c, p->vol_n * q / nvc, p->vol_n * (q + 1) / nvc, &rows[nre + 1 + q]);
  if (use_bvh) bvh_free(&bv);

  int64_t total = 0;
  for (int32_t j = 0; j < nrows; ++j) total += rows[j].n;
  out->n = total;
  int rc = 0;
  if (total > out->cap) {
    rc = (int)(-total > -2147483647 ? -total : -2147483647);
  } else {
    int64_t w = 0;
    for (int32_t j = 0; j < nrows; ++j) {
      for (int64_t k = 0; k < rows[j].n; ++k, ++w) {
        const ohit* h = &rows[j].v[k];
        out->ray[w] = h->ray; out->sub[w] = h->sub; out->seg[w] = h->seg; out->prim[w] = h->prim;
        out->tau[w] = h->tau; out->len[w] = h->len; out->amp[w] = h->amp;
        out->psi[w] = h->psi; out->phi[w] = h->phi;
        out->ux[w] = h->u[0]; out->uy[w] = h->u[1]; out->uz[w] = h->u[2];
        out->cr[w] = h->amp * cos(h->phi); out->ci[w] = h->amp * sin(h->phi);
        out->margin[w] = h->margin; out->gap[w] = h->gap;
        out->kinc[w] = h->kinc; out->gam[w] = h->gam;
      }
    }
  }
  for (int32_t j = 0; j < nrows; ++j) free(rows[j].v);
  free(rows);
  return rc;
}

/* ------------------------------------------------------------------ element echoes */
/* Sec. II.B complex baseband accumulated along rays, already pulse-compressed:
   s_m[n] = sum_k c_k R(t_n - tau_k) exp(j k_a u_k . p_m), k_a = 2 pi f0 / c_ref,
   t_n = 2 (r_min + (n + 1/2) dr) / c_ref, elements p_m = (0, y_m, z_m) on a centred
   nx x ny grid of the given pitch, m = my * nx + mx. */
/* raw != 0: the raw (uncompressed) element series instead, r_m(t) = sum_k c_k p(t - tau_k)
   exp(j k_a u_k . p_m), sampled at t_n + shift. */
static void synth_core(const orc_params* p, const orc_hits* h, const int32_t* ns, int64_t n_ns, int raw,
                       double shift, double* s_out) {
  const int32_t nx = p->nx, ny = p->ny, M = nx * ny;
  const double c_ref = h->c_ref, dr = (p->r_max - p->r_min) / p->n_range;
  const double ka = TWO_PI * p->f0 / c_ref;
  const double support = raw ? p->pulse / 2 : p->pulse;  /* |u| inside: p on [-T/2, T/2], R on (-T, T) */
  memset(s_out, 0, sizeof(double) * 2 * (size_t)M * (size_t)n_ns);
  /* per hit, the requested samples inside its pulse window and c_k R(t_n - tau_k) */
  int64_t* cnt = (int64_t*)calloc((size_t)h->n + 1, sizeof(int64_t));
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < h->n; ++k) {
    int64_t c = 0;
    for (int64_t i = 0; i < n_ns; ++i) {
      double tn = 2.0 * (p->r_min + (ns[i] + 0.5) * dr) / c_ref + shift;
      if (raw ? fabs(tn - h->tau[k]) <= support : fabs(tn - h->tau[k]) < support) ++c;
    }
    cnt[k + 1] = c;
  }
  for (int64_t k = 0; k < h->n; ++k) cnt[k + 1] += cnt[k];
  int64_t npairs = cnt[h->n];
  int64_t* pi = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npairs + 1));
  cplx* pg = (cplx*)malloc(sizeof(cplx) * (size_t)(npairs + 1));
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < h->n; ++k) {
    int64_t w = cnt[k];
    cplx ck = h->cr[k] + I * h->ci[k];
    for (int64_t i = 0; i < n_ns; ++i) {
      double tn = 2.0 * (p->r_min + (ns[i] + 0.5) * dr) / c_ref + shift;
      double u = tn - h->tau[k];
      if (raw ? fabs(u) <= support : fabs(u) < support) {
        double re, im;
        if (raw)
          orc_pulse(u, p->pulse, p->bw, &re, &im);
        else
          orc_pulse_acf(u, p->pulse, p->bw, &re, &im);
        pi[w] = i;
        pg[w] = ck * (re + I * im);
        ++w;
      }
    }
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int32_t m = 0; m < M; ++m) {
    int32_t mx = m % nx, my = m / nx;
    double ym = (mx - (nx - 1) / 2.0) * p->pitch, zm = (my - (ny - 1) / 2.0) * p->pitch;
    for (int64_t k = 0; k < h->n; ++k) {
      if (cnt[k + 1] == cnt[k]) continue;
      cplx ph = cexp(I * ka * (h->uy[k] * ym + h->uz[k] * zm));
      for (int64_t w = cnt[k]; w < cnt[k + 1]; ++w) {
        cplx v = pg[w] * ph;
        s_out[2 * ((size_t)pi[w] * M + m)] += creal(v);
        s_out[2 * ((size_t)pi[w] * M + m) + 1] += cimag(v);
      }
    }
  }
  free(cnt);
  free(pi);
  free(pg);
}

void orc_synth(const orc_params* p, const orc_hits* h, const int32_t* ns, int64_t n_ns, double* s_out) {
  synth_core(p, h, ns, n_ns, 0, 0.0, s_out);
}

/* Raw element series (the uncompressed echo before a matched filter): r_m at
   t_n + s dt / U, dt = 2 dr / c_ref, for the requested samples n. */
void orc_raw(const orc_params* p, const orc_hits* h, int32_t U, int32_t s, const int32_t* ns, int64_t n_ns,
             double* s_out) {
  const double dt = 2.0 * (p->r_max - p->r_min) / p->n_range / h->c_ref;
  synth_core(p, h, ns, n_ns, 1, s * dt / U, s_out);
}

/* Wideband element echoes: the plane-wave delay across the aperture kept in the envelope
   as well as in the phase. An element at p_m hears a hit arriving from u_k earlier by
   u_k . p_m / c, so s_m(t) = sum_k c_k R(t - tau_k + u_k . p_m / c) exp(j k_a u_k . p_m),
   evaluated at t = t_n + shift for the requested samples n. */
void orc_synth_wb(const orc_params* p, const orc_hits* h, double shift, const int32_t* ns, int64_t n_ns,
                  double* s_out) {
  const int32_t nx = p->nx, ny = p->ny, M = nx * ny;
  const double c_ref = h->c_ref, dr = (p->r_max - p->r_min) / p->n_range;
  const double ka = TWO_PI * p->f0 / c_ref;
  memset(s_out, 0, sizeof(double) * 2 * (size_t)M * (size_t)n_ns);
#pragma omp parallel for schedule(dynamic, 4)
  for (int32_t m = 0; m < M; ++m) {
    int32_t mx = m % nx, my = m / nx;
    double ym = (mx - (nx - 1) / 2.0) * p->pitch, zm = (my - (ny - 1) / 2.0) * p->pitch;
    for (int64_t k = 0; k < h->n; ++k) {
      double up = h->uy[k] * ym + h->uz[k] * zm;  /* u_k . p_m (the array lies in the y-z plane) */
      cplx ck = (h->cr[k] + I * h->ci[k]) * cexp(I * ka * up);
      for (int64_t i = 0; i < n_ns; ++i) {
        double u = 2.0 * (p->r_min + (ns[i] + 0.5) * dr) / c_ref + shift - h->tau[k] + up / c_ref;
        if (!(fabs(u) < p->pulse)) continue;
        double re, im;
        orc_pulse_acf(u, p->pulse, p->bw, &re, &im);
        cplx v = ck * (re + I * im);
        s_out[2 * ((size_t)i * M + m)] += creal(v);
        s_out[2 * ((size_t)i * M + m) + 1] += cimag(v);
      }
    }
  }
}

/* Beam directions (Sec. III Eq. 2-3, cell-centred): az_i = -HFOV/2 + (i+1/2) HFOV/N_az,
   el_j likewise, b = j N_az + i, u_b = (cos el cos az, cos el sin az, sin el). */
static void beam_dir(const orc_params* p, int32_t b, double u[3]) {
  int32_t i = b % p->n_beam_az, j = b / p->n_beam_az;
  double az = -p->hfov / 2 + (i + 0.5) * p->hfov / p->n_beam_az;
  double el = -p->vfov / 2 + (j + 0.5) * p->vfov / p->n_beam_el;
  u[0] = cos(el) * cos(az);
  u[1] = cos(el) * sin(az);
  u[2] = sin(el);
}

/* Sec. II.B coherent summation into beams: phase-shift beamforming
   B[b][n] = sum_m w_m exp(-j k_a u_b . p_m) s_m[n] / sum_m w_m. */
void orc_beamform(const orc_params* p, double c_ref, const float* taper, const double* s, int64_t n_ns,
                  const int32_t* beams, int64_t n_beams, double* b_out) {
  const int32_t nx = p->nx, ny = p->ny, M = nx * ny;
  const double ka = TWO_PI * p->f0 / c_ref;
  double wsum = 0;
  for (int32_t m = 0; m < M; ++m) wsum += taper ? taper[m] : 1.0;
  cplx* W = (cplx*)malloc(sizeof(cplx) * (size_t)n_beams * M);
#pragma omp parallel for schedule(static)
  for (int64_t bi = 0; bi < n_beams; ++bi) {
    double u[3];
    beam_dir(p, beams[bi], u);
    for (int32_t m = 0; m < M; ++m) {
      int32_t mx = m % nx, my = m / nx;
      double ym = (mx - (nx - 1) / 2.0) * p->pitch, zm = (my - (ny - 1) / 2.0) * p->pitch;
      double w = taper ? taper[m] : 1.0;
      W[bi * M + m] = w * cexp(-I * ka * (u[1] * ym + u[2] * zm)) / wsum;
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n_ns; ++i) {
    const double* si = s + 2 * (size_t)i * M;
    for (int64_t bi = 0; bi < n_beams; ++bi) {
      cplx acc = 0;
      for (int32_t m = 0; m < M; ++m) acc += W[bi * M + m] * (si[2 * m] + I * si[2 * m + 1]);
      b_out[2 * ((size_t)bi * n_ns + i)] = creal(acc);
      b_out[2 * ((size_t)bi * n_ns + i) + 1] = cimag(acc);
    }
  }
  free(W);
}

/* True-time-delay beamforming of the wideband echoes, exact in time: each element is
   read at its steering delay, B[b][n] = sum_m w_m exp(-j k_a u_b . p_m)
   s_m(t_n - u_b . p_m / c) / sum_m w_m, evaluated from the hits as
   sum_k c_k sum_m w_m exp(j k_a (u_k - u_b) . p_m) R(t_n - tau_k + (u_k - u_b) . p_m / c)
   / sum_m w_m. */
void orc_ttd(const orc_params* p, const orc_hits* h, const float* taper, const int32_t* ns, int64_t n_ns,
             const int32_t* beams, int64_t n_beams, double* b_out) {
  const int32_t nx = p->nx, ny = p->ny, M = nx * ny;
  const double c_ref = h->c_ref, dr = (p->r_max - p->r_min) / p->n_range;
  const double ka = TWO_PI * p->f0 / c_ref;
  double wsum = 0;
  for (int32_t m = 0; m < M; ++m) wsum += taper ? taper[m] : 1.0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t bi = 0; bi < n_beams; ++bi) {
    double ub[3];
    beam_dir(p, beams[bi], ub);
    for (int64_t i = 0; i < n_ns; ++i) {
      const double tn = 2.0 * (p->r_min + (ns[i] + 0.5) * dr) / c_ref;
      cplx acc = 0;
      for (int64_t k = 0; k < h->n; ++k) {
        /* the delays across the array are below the aperture over c: skip hits whose
           pulse cannot reach t_n from any element */
        if (!(fabs(tn - h->tau[k]) < p->pulse + 2.0 * (nx + ny) * p->pitch / c_ref)) continue;
        const cplx ck = h->cr[k] + I * h->ci[k];
        const double dy = h->uy[k] - ub[1], dz = h->uz[k] - ub[2];
        for (int32_t m = 0; m < M; ++m) {
          int32_t mx = m % nx, my = m / nx;
          double ym = (mx - (nx - 1) / 2.0) * p->pitch, zm = (my - (ny - 1) / 2.0) * p->pitch;
          double dp = dy * ym + dz * zm;
          double u = tn - h->tau[k] + dp / c_ref;
          if (!(fabs(u) < p->pulse)) continue;
          double re, im;
          orc_pulse_acf(u, p->pulse, p->bw, &re, &im);
          acc += (taper ? taper[m] : 1.0) * ck * cexp(I * ka * dp) * (re + I * im);
        }
      }
      acc /= wsum;
      b_out[2 * ((size_t)bi * n_ns + i)] = creal(acc);
      b_out[2 * ((size_t)bi * n_ns + i) + 1] = cimag(acc);
    }
  }
}

/* Envelope with time-varied gain TVG(r) = r exp(2 alpha r), r_n at bin centres. */
void orc_envelope(const orc_params* p, const double* b, const int32_t* ns, int64_t n_ns, int64_t n_beams,
                  double* e_out) {
  const double dr = (p->r_max - p->r_min) / p->n_range;
  for (int64_t bi = 0; bi < n_beams; ++bi) {
    for (int64_t i = 0; i < n_ns; ++i) {
      double r = p->r_min + (ns[i] + 0.5) * dr;
      double re = b[2 * ((size_t)bi * n_ns + i)], im = b[2 * ((size_t)bi * n_ns + i) + 1];
      e_out[(size_t)bi * n_ns + i] = hypot(re, im) * r * exp(2.0 * p->alpha * r);
    }
  }
}

/* Sec. II.A volumetric output as a point cloud: per beam the strongest bin at or beyond
   r_blank (first on ties), kept when it reaches the threshold (absolute, or relative to
   the ping maximum over the same bins); position R(q) (r_n u_b) + t. */
int64_t orc_peaks(const orc_params* p, const double pose_t[3], const double pose_q[4], const double* e,
                  double* pts, int32_t* pbeam, int32_t* pbin) {
  const int32_t Nb = p->n_beam_az * p->n_beam_el, Nr = p->n_range;
  const double dr = (p->r_max - p->r_min) / Nr;
  int32_t nb0 = 0;
  while (nb0 < Nr && p->r_min + (nb0 + 0.5) * dr < p->r_blank) ++nb0;
  double vmax = 0;
  for (int32_t b = 0; b < Nb; ++b)
    for (int32_t n = nb0; n < Nr; ++n) vmax = fmax(vmax, e[(size_t)b * Nr + n]);
  double thr = p->thr_mode == 1 ? p->thr * vmax : p->thr;
  double qn = sqrt(pose_q[0] * pose_q[0] + pose_q[1] * pose_q[1] + pose_q[2] * pose_q[2] + pose_q[3] * pose_q[3]);
  double q[4] = {pose_q[0] / qn, pose_q[1] / qn, pose_q[2] / qn, pose_q[3] / qn}, R[9];
  quat_to_matrix(q, R);
  int64_t cnt = 0;
  for (int32_t b = 0; b < Nb; ++b) {
    int32_t best = -1;
    double bv = -1;
    for (int32_t n = nb0; n < Nr; ++n) {
      double v = e[(size_t)b * Nr + n];
      if (v > bv) { bv = v; best = n; }
    }
    if (best < 0 || !(bv >= thr)) continue;
    double u[3], w[3];
    beam_dir(p, b, u);
    double r = p->r_min + (best + 0.5) * dr;
    double v[3] = {r * u[0], r * u[1], r * u[2]};
    mat_vec(R, v, w);
    pts[4 * cnt] = w[0] + pose_t[0];
    pts[4 * cnt + 1] = w[1] + pose_t[1];
    pts[4 * cnt + 2] = w[2] + pose_t[2];
    pts[4 * cnt + 3] = bv;
    pbeam[cnt] = b;
    pbin[cnt] = best;
    ++cnt;
  }
  return cnt;
}
