/*
 * oracle.c -- plain, slow FP64 CPU reference for direct volume ray casting of
 * trivariate LR-splines (Fuchs, Barrowclough, Hjelmervik, Dahl: "Direct
 * interactive visualization of locally refined spline volumes for scalar and
 * vector fields").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code
 * with the CUDA path.
 *
 * What it computes, each function following its passage of the paper:
 *   orc_bspline      univariate B-spline by the Cox-de Boor recursion on a
 *                    local knot vector (Sec. 3.1, Eq. 1 factors)
 *   orc_find_element the element holding a point, by scanning every element
 *                    box in turn (the O(N) search Sec. 3.2 sets against the
 *                    acceleration structures)
 *   orc_eval         f(x) = sum_i c_i gamma_i N_i(x)  (Eq. 2), the sum running
 *                    over the B-splines whose support contains the element of
 *                    x, found by scanning all B-splines
 *   orc_render       per pixel: ray setup, sampling at a fixed step, at the
 *                    adaptive distance of Eq. 4, or at Eq. 4 scaled by a given
 *                    per-element multiplier (the learned step), transfer
 *                    function, optional gradient shading (Sec. 4.1) and
 *                    trimming interval, and front-to-back compositing (Alg. 2)
 *   orc_bspline_d1, orc_eval_grad
 *                    derivative of each Eq. 1 factor, gradient of Eq. 2
 *   orc_labels       training labels of the learned step (Eq. 4 visits judged
 *                    against fine-step Alg. 2 composites)
 *   orc_trim         per-pixel first front / last back face of a closed mesh
 *                    (the z-prepass of Sec. 4.1), watertight FP32 hits
 *   orc_streamlines  streamlines by explicit Runge-Kutta methods (Sec. 5,
 *                    Eq. 5), FP64 outer loop, fixed / Eq. 4 / adaptive steps
 *   orc_tubes        streamline tubes as capsules (Sec. 5.3)
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *   - intervals are half open, [lo, hi); the upper domain face x = 1 belongs
 *     to the last non-empty interval / the element with hi = 1;
 *   - element and step decisions depend on the sample position, so sample
 *     positions, ray parameters and the loop bounds are computed in FP32 with
 *     the operation order stated below (the precision the kernels use); the
 *     field, the transfer function and the compositing are FP64;
 *   - Eq. 4 uses d = max(p1,p2,p3) and the element's sides in parameter units;
 *     the step is rounded once to FP32;
 *   - the segment of Alg. 2 belonging to sample k is the forward segment to
 *     the next sample, the last one clipped at the exit parameter;
 *   - the TF is linear interpolation over 256 entries spanning [vmin, vmax],
 *     colour not premultiplied (Alg. 2 multiplies by (1-T)(1-alpha_dst));
 *   - early termination when alpha_dst >= alpha_stop; background transparent.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXP 4
#define ORC_NONE 0xFFFFFFFFu

typedef struct {
  int p[3];
  int nc;
  int64_t n_elem;
  double *box; /* n_elem x 6: lo xyz, hi xyz */
  int64_t n_basis;
  int kw;          /* knots per B-spline: p0+p1+p2+6 */
  double *knots;   /* n_basis x kw, x then y then z */
  double *coef;    /* n_basis x nc */
  double *weight;  /* n_basis: gamma */
} orc_vol;

/* ------------------------------------------------------------------------ */
/* Eq. 1 factor: one univariate B-spline of degree p on knots xi[0..p+1].    */
/* ------------------------------------------------------------------------ */
double orc_bspline(const double *xi, int p, double x) {
  double N[ORC_MAXP + 2];
  if (x < xi[0] || x > xi[p + 1]) return 0.0;
  for (int j = 0; j <= p; ++j) N[j] = (xi[j] <= x && x < xi[j + 1]) ? 1.0 : 0.0;
  if (x == xi[p + 1] && x == 1.0) {
    /* upper domain face: belongs to the last non-empty interval */
    for (int j = p; j >= 0; --j)
      if (xi[j] < xi[j + 1]) {
        N[j] = 1.0;
        break;
      }
  }
  for (int r = 1; r <= p; ++r) {
    for (int j = 0; j + r <= p; ++j) {
      double left = 0.0, right = 0.0;
      if (xi[j + r] != xi[j]) left = (x - xi[j]) / (xi[j + r] - xi[j]) * N[j];
      if (xi[j + r + 1] != xi[j + 1]) right = (xi[j + r + 1] - x) / (xi[j + r + 1] - xi[j + 1]) * N[j + 1];
      N[j] = left + right;
    }
  }
  return N[0];
}

/* Derivative of the B-spline above: the textbook recurrence
 * B'_p = p (B_{p-1}[xi_0..xi_p] / (xi_p - xi_0) - B_{p-1}[xi_1..xi_{p+1}] / (xi_{p+1} - xi_1)),
 * a term with a zero denominator dropped.  At a knot it is the derivative
 * of the piece on the right (half-open intervals, as for the value). */
double orc_bspline_d1(const double *xi, int p, double x) {
  if (p == 0) return 0.0;
  double d = 0.0;
  if (xi[p] != xi[0]) d += orc_bspline(xi, p - 1, x) / (xi[p] - xi[0]);
  if (xi[p + 1] != xi[1]) d -= orc_bspline(xi + 1, p - 1, x) / (xi[p + 1] - xi[1]);
  return (double)p * d;
}

orc_vol *orc_create(const int *deg, int nc, int64_t n_elem, const double *box, int64_t n_basis,
                    const double *knots, const double *coef, const double *weight) {
  for (int a = 0; a < 3; ++a)
    if (deg[a] < 0 || deg[a] > ORC_MAXP) return NULL;
  if (nc < 1 || nc > 3 || n_elem < 1 || n_basis < 1) return NULL;
  orc_vol *v = (orc_vol *)calloc(1, sizeof(orc_vol));
  for (int a = 0; a < 3; ++a) v->p[a] = deg[a];
  v->nc = nc;
  v->n_elem = n_elem;
  v->n_basis = n_basis;
  v->kw = deg[0] + deg[1] + deg[2] + 6;
  v->box = (double *)malloc(sizeof(double) * 6 * n_elem);
  v->knots = (double *)malloc(sizeof(double) * v->kw * n_basis);
  v->coef = (double *)malloc(sizeof(double) * nc * n_basis);
  v->weight = (double *)malloc(sizeof(double) * n_basis);
  memcpy(v->box, box, sizeof(double) * 6 * n_elem);
  memcpy(v->knots, knots, sizeof(double) * v->kw * n_basis);
  memcpy(v->coef, coef, sizeof(double) * nc * n_basis);
  memcpy(v->weight, weight, sizeof(double) * n_basis);
  return v;
}

void orc_destroy(orc_vol *v) {
  if (!v) return;
  free(v->box);
  free(v->knots);
  free(v->coef);
  free(v->weight);
  free(v);
}

static const double *knots_of(const orc_vol *v, int64_t i, int a) {
  const double *k = v->knots + i * v->kw;
  if (a >= 1) k += v->p[0] + 2;
  if (a >= 2) k += v->p[1] + 2;
  return k;
}

/* x in element e: lo <= x < hi per axis, with x == hi allowed when hi == 1. */
static int in_element(const orc_vol *v, int64_t e, const double *x) {
  const double *b = v->box + 6 * e;
  for (int a = 0; a < 3; ++a) {
    double lo = b[a], hi = b[3 + a];
    if (!(lo <= x[a] && (x[a] < hi || (x[a] == hi && hi == 1.0)))) return 0;
  }
  return 1;
}

/* The element holding x, by linear search over all elements; ORC_NONE outside [0,1]^3. */
uint32_t orc_find_element(const orc_vol *v, const double *x) {
  for (int a = 0; a < 3; ++a)
    if (!(x[a] >= 0.0 && x[a] <= 1.0)) return ORC_NONE;
  for (int64_t e = 0; e < v->n_elem; ++e)
    if (in_element(v, e, x)) return (uint32_t)e;
  return ORC_NONE;
}

/* B-splines whose support contains element e, by scanning all B-splines.
 * out must hold n_basis entries; returns the count. */
int64_t orc_incidence(const orc_vol *v, int64_t e, int64_t *out) {
  const double *b = v->box + 6 * e;
  int64_t n = 0;
  for (int64_t i = 0; i < v->n_basis; ++i) {
    int ok = 1;
    for (int a = 0; a < 3 && ok; ++a) {
      const double *k = knots_of(v, i, a);
      ok = (k[0] <= b[a]) && (b[3 + a] <= k[v->p[a] + 1]);
    }
    if (ok) out[n++] = i;
  }
  return n;
}

/* Eq. 2 at x, given the incidence list of the element holding x. */
static void eval_with(const orc_vol *v, const int64_t *inc, int64_t ninc, const double *x, double *out) {
  for (int c = 0; c < v->nc; ++c) out[c] = 0.0;
  for (int64_t q = 0; q < ninc; ++q) {
    int64_t i = inc[q];
    double N = v->weight[i];
    for (int a = 0; a < 3; ++a) N *= orc_bspline(knots_of(v, i, a), v->p[a], x[a]);
    for (int c = 0; c < v->nc; ++c) out[c] += v->coef[i * v->nc + c] * N;
  }
}

/* Eq. 2 and its gradient at x: grad[3*c + a] = d f_c / d x_a, each factor
 * differentiated by orc_bspline_d1 (product rule over the three axes). */
static void eval_grad_with(const orc_vol *v, const int64_t *inc, int64_t ninc, const double *x, double *val,
                           double *grad) {
  for (int c = 0; c < v->nc; ++c) {
    val[c] = 0.0;
    grad[3 * c] = grad[3 * c + 1] = grad[3 * c + 2] = 0.0;
  }
  for (int64_t q = 0; q < ninc; ++q) {
    int64_t i = inc[q];
    double B[3], D[3];
    for (int a = 0; a < 3; ++a) {
      B[a] = orc_bspline(knots_of(v, i, a), v->p[a], x[a]);
      D[a] = orc_bspline_d1(knots_of(v, i, a), v->p[a], x[a]);
    }
    const double g = v->weight[i];
    const double N = g * B[0] * B[1] * B[2];
    const double dN[3] = {g * D[0] * B[1] * B[2], g * B[0] * D[1] * B[2], g * B[0] * B[1] * D[2]};
    for (int c = 0; c < v->nc; ++c) {
      const double cc = v->coef[i * v->nc + c];
      val[c] += cc * N;
      for (int a = 0; a < 3; ++a) grad[3 * c + a] += cc * dN[a];
    }
  }
}

/* f(x) and its gradient (grad: 3 x nc, component-major).  Returns the element id. */
uint32_t orc_eval_grad(const orc_vol *v, const double *x, double *val, double *grad) {
  uint32_t e = orc_find_element(v, x);
  if (e == ORC_NONE) {
    for (int c = 0; c < v->nc; ++c) val[c] = grad[3 * c] = grad[3 * c + 1] = grad[3 * c + 2] = 0.0;
    return e;
  }
  int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * v->n_basis);
  int64_t n = orc_incidence(v, e, inc);
  eval_grad_with(v, inc, n, x, val, grad);
  free(inc);
  return e;
}

/* f(x) (Eq. 2).  Returns the element id, ORC_NONE (and zeros) outside the domain. */
uint32_t orc_eval(const orc_vol *v, const double *x, double *out) {
  uint32_t e = orc_find_element(v, x);
  if (e == ORC_NONE) {
    for (int c = 0; c < v->nc; ++c) out[c] = 0.0;
    return e;
  }
  int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * v->n_basis);
  int64_t n = orc_incidence(v, e, inc);
  eval_with(v, inc, n, x, out);
  free(inc);
  return e;
}

/* ------------------------------------------------------------------------ */
/* threaded batches                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_vol *v;
  const float *pts_f;
  const double *pts_d;
  int64_t n;
  int tid, nth;
  uint32_t *elem;
  double *val;
  double *grad; /* with val: n x 3 x nc gradients */
} batch_job;

static void *batch_worker(void *arg) {
  batch_job *j = (batch_job *)arg;
  const orc_vol *v = j->v;
  int64_t *inc = j->val ? (int64_t *)malloc(sizeof(int64_t) * v->n_basis) : NULL;
  uint32_t cur = ORC_NONE;
  int64_t ninc = 0;
  for (int64_t q = j->tid; q < j->n; q += j->nth) {
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = j->pts_f ? (double)j->pts_f[3 * q + a] : j->pts_d[3 * q + a];
    uint32_t e = orc_find_element(v, x);
    if (j->elem) j->elem[q] = e;
    if (j->val) {
      if (e == ORC_NONE) {
        for (int c = 0; c < v->nc; ++c) j->val[q * v->nc + c] = 0.0;
        if (j->grad)
          for (int c = 0; c < 3 * v->nc; ++c) j->grad[q * 3 * v->nc + c] = 0.0;
        continue;
      }
      if (e != cur) {
        ninc = orc_incidence(v, e, inc);
        cur = e;
      }
      if (j->grad)
        eval_grad_with(v, inc, ninc, x, j->val + q * v->nc, j->grad + q * 3 * v->nc);
      else
        eval_with(v, inc, ninc, x, j->val + q * v->nc);
    }
  }
  free(inc);
  return NULL;
}

static void run_batch(batch_job *proto, int nth) {
  if (nth < 1) nth = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nth);
  batch_job *jobs = (batch_job *)malloc(sizeof(batch_job) * nth);
  for (int t = 0; t < nth; ++t) {
    jobs[t] = *proto;
    jobs[t].tid = t;
    jobs[t].nth = nth;
    pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
  }
  for (int t = 0; t < nth; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* Element ids of n FP32 points (n x 3). */
void orc_lookup_batch(const orc_vol *v, const float *pts, int64_t n, uint32_t *elem, int nth) {
  batch_job j = {v, pts, NULL, n, 0, 1, elem, NULL, NULL};
  run_batch(&j, nth);
}

/* f at n FP32 points (val: n x nc) and their element ids (may be NULL). */
void orc_eval_batch_f32(const orc_vol *v, const float *pts, int64_t n, double *val, uint32_t *elem, int nth) {
  batch_job j = {v, pts, NULL, n, 0, 1, elem, val, NULL};
  run_batch(&j, nth);
}

/* f and its gradient at n FP32 points (val: n x nc, grad: n x nc x 3). */
void orc_eval_grad_batch_f32(const orc_vol *v, const float *pts, int64_t n, double *val, double *grad, int nth) {
  batch_job j = {v, pts, NULL, n, 0, 1, NULL, val, grad};
  run_batch(&j, nth);
}

/* f and its gradient at n FP64 points. */
void orc_eval_grad_batch_f64(const orc_vol *v, const double *pts, int64_t n, double *val, double *grad, int nth) {
  batch_job j = {v, NULL, pts, n, 0, 1, NULL, val, grad};
  run_batch(&j, nth);
}

/* f at n FP64 points. */
void orc_eval_batch_f64(const orc_vol *v, const double *pts, int64_t n, double *val, uint32_t *elem, int nth) {
  batch_job j = {v, NULL, pts, n, 0, 1, elem, val, NULL};
  run_batch(&j, nth);
}

/* ------------------------------------------------------------------------ */
/* rendering (Sec. 4)                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t projection; /* 0 ortho, 1 persp */
  int32_t width, height;
  double eye[3], target[3], up[3];
  double fovy;   /* persp: full vertical field of view (radians) */
  double extent; /* ortho: full height of the view window */
} orc_camera;

typedef struct {
  const double *table; /* 256 x 4 RGBA */
  double vmin, vmax;
} orc_tf;

typedef struct {
  int32_t mode;  /* 0 fixed, 1 heuristic (Eq. 4), 2 learned: Eq. 4 times a per-element multiplier */
  int32_t field; /* 0 scalar, 1 magnitude, 2 component */
  int32_t component;
  double h, xi, alpha_stop;
  const float *mult; /* mode 2: per-element step multipliers (FP32) */
  int32_t shading;   /* 1: gradient shading of C_src (Sec. 4.1) */
  double light[3];   /* towards the light; all zero: towards the eye along the ray */
  const float *trim; /* NULL, or per pixel (t_front, t_back) of a trimming mesh (orc_trim) */
} orc_step;

typedef struct {
  /* FP32 ray-generation constants, from FP64 camera algebra rounded once */
  float E[3], F[3], R[3], U[3];
  float sxs, sxo, sys, syo;
  int persp;
} ray_consts;

static void camera_consts(const orc_camera *c, ray_consts *k) {
  double F[3], R[3], U[3], n;
  for (int a = 0; a < 3; ++a) F[a] = c->target[a] - c->eye[a];
  n = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  for (int a = 0; a < 3; ++a) F[a] = F[a] / n;
  R[0] = F[1] * c->up[2] - F[2] * c->up[1];
  R[1] = F[2] * c->up[0] - F[0] * c->up[2];
  R[2] = F[0] * c->up[1] - F[1] * c->up[0];
  n = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  for (int a = 0; a < 3; ++a) R[a] = R[a] / n;
  U[0] = R[1] * F[2] - R[2] * F[1];
  U[1] = R[2] * F[0] - R[0] * F[2];
  U[2] = R[0] * F[1] - R[1] * F[0];
  double ty = c->projection == 1 ? tan(0.5 * c->fovy) : 0.5 * c->extent;
  double tx = ty * (double)c->width / (double)c->height;
  for (int a = 0; a < 3; ++a) {
    k->E[a] = (float)c->eye[a];
    k->F[a] = (float)F[a];
    k->R[a] = (float)R[a];
    k->U[a] = (float)U[a];
  }
  k->sxs = (float)(2.0 * tx / (double)c->width);
  k->sxo = (float)(-tx);
  k->sys = (float)(-2.0 * ty / (double)c->height);
  k->syo = (float)ty;
  k->persp = c->projection == 1;
}

/* FP32 ray of pixel (i, j) (j = 0 is the top row) and its parameter interval
 * in the unit cube.  Returns 0 when the ray misses the cube. */
static int ray_setup(const ray_consts *k, int i, int j, float o[3], float d[3], float *tin, float *tout) {
  float a = fmaf((float)i + 0.5f, k->sxs, k->sxo);
  float b = fmaf((float)j + 0.5f, k->sys, k->syo);
  if (k->persp) {
    for (int c = 0; c < 3; ++c) {
      d[c] = fmaf(a, k->R[c], fmaf(b, k->U[c], k->F[c]));
      o[c] = k->E[c];
    }
    float n2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
    float n = sqrtf(n2);
    for (int c = 0; c < 3; ++c) d[c] = d[c] / n;
  } else {
    for (int c = 0; c < 3; ++c) {
      o[c] = fmaf(a, k->R[c], fmaf(b, k->U[c], k->E[c]));
      d[c] = k->F[c];
    }
  }
  float t0 = 0.0f, t1 = INFINITY;
  for (int c = 0; c < 3; ++c) {
    if (d[c] == 0.0f) {
      if (o[c] < 0.0f || o[c] > 1.0f) return 0;
      continue;
    }
    float inv = 1.0f / d[c];
    float ta = (0.0f - o[c]) * inv;
    float tb = (1.0f - o[c]) * inv;
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  }
  *tin = t0;
  *tout = t1;
  return t0 < t1;
}

/* ------------------------------------------------------------------------ */
/* Trimming (Sec. 4.1): the ray interval is cut to the first front face and  */
/* the last back face of a closed triangle mesh, the two depth buffers of a  */
/* z-prepass.  Hits use the watertight ray/triangle test of Woop, Benthin    */
/* and Wald (JCGT 2013) in FP32 with the kernel's order of operations (hits  */
/* are decisions), falling back to FP64 for an edge function that is        */
/* exactly 0.  Front faces are those wound counter-clockwise seen from the   */
/* ray's origin side (det > 0).                                              */
/* ------------------------------------------------------------------------ */
static int tri_hit(const float o[3], const float d[3], const float *v, float *t, int *front) {
  int kz = 0;
  if (fabsf(d[1]) > fabsf(d[kz])) kz = 1;
  if (fabsf(d[2]) > fabsf(d[kz])) kz = 2;
  int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
  if (d[kz] < 0.0f) {
    int w = kx;
    kx = ky;
    ky = w;
  }
  const float Sx = d[kx] / d[kz], Sy = d[ky] / d[kz], Sz = 1.0f / d[kz];
  float A[3], B[3], C[3];
  for (int c = 0; c < 3; ++c) {
    A[c] = v[c] - o[c];
    B[c] = v[3 + c] - o[c];
    C[c] = v[6 + c] - o[c];
  }
  const float Ax = A[kx] - Sx * A[kz], Ay = A[ky] - Sy * A[kz];
  const float Bx = B[kx] - Sx * B[kz], By = B[ky] - Sy * B[kz];
  const float Cx = C[kx] - Sx * C[kz], Cy = C[ky] - Sy * C[kz];
  float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;
  const float det = U + V + W;
  if (det == 0.0f) return 0;
  const float Az = Sz * A[kz], Bz = Sz * B[kz], Cz = Sz * C[kz];
  const float T = U * Az + V * Bz + W * Cz;
  if (det > 0.0f ? !(T > 0.0f) : !(T < 0.0f)) return 0; /* hits at t <= 0 do not count */
  *t = T / det;
  *front = det > 0.0f;
  return 1;
}

typedef struct {
  const orc_camera *cam;
  const float *tri;
  int64_t n_tri;
  float *out;
  int tid, nth;
} trim_job;

static void *trim_worker(void *arg) {
  trim_job *J = (trim_job *)arg;
  ray_consts K;
  camera_consts(J->cam, &K);
  const int64_t npix = (int64_t)J->cam->width * J->cam->height;
  for (int64_t q = J->tid; q < npix; q += J->nth) {
    const int i = (int)(q % J->cam->width), j = (int)(q / J->cam->width);
    float o[3], d[3], tin, tout;
    ray_setup(&K, i, j, o, d, &tin, &tout);
    float tf = INFINITY, tb = 0.0f;
    for (int64_t k = 0; k < J->n_tri; ++k) {
      float t;
      int front;
      if (!tri_hit(o, d, J->tri + 9 * k, &t, &front)) continue;
      if (front) {
        if (t < tf) tf = t;
      } else if (t > tb) {
        tb = t;
      }
    }
    J->out[2 * q] = tf;
    J->out[2 * q + 1] = tb;
  }
  return NULL;
}

/* Per pixel (t_front, t_back): the nearest front-face hit (+inf if none) and
 * the farthest back-face hit (0 if none) of n_tri triangles (n x 9 floats). */
void orc_trim(const orc_camera *cam, const float *tri, int64_t n_tri, float *out, int nth) {
  if (nth < 1) nth = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nth);
  trim_job *jobs = (trim_job *)malloc(sizeof(trim_job) * nth);
  for (int t = 0; t < nth; ++t) {
    trim_job J = {cam, tri, n_tri, out, t, nth};
    jobs[t] = J;
    pthread_create(&th[t], NULL, trim_worker, &jobs[t]);
  }
  for (int t = 0; t < nth; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* The ray interval [tin, tout] cut by a pixel's trimming interval: no hit
 * hides the pixel; only back faces (the eye inside the mesh) keep [tin,
 * t_back]; only front faces (an open mesh) keep [t_front, tout]. */
static int trim_interval(const float *tr, float *tin, float *tout) {
  const float tf = tr[0], tb = tr[1];
  if (tf == INFINITY && tb == 0.0f) return 0;
  if (tf != INFINITY && tf > *tin) *tin = tf;
  if (tb != 0.0f && tb < *tout) *tout = tb;
  return *tin < *tout;
}

/* Eq. 4: 2^-d times the shortest side of element e, d = max degree, rounded once to FP32. */
float orc_heuristic_step(const orc_vol *v, uint32_t e) {
  const double *b = v->box + 6 * (int64_t)e;
  int d = v->p[0];
  if (v->p[1] > d) d = v->p[1];
  if (v->p[2] > d) d = v->p[2];
  double m = b[3] - b[0];
  if (b[4] - b[1] < m) m = b[4] - b[1];
  if (b[5] - b[2] < m) m = b[5] - b[2];
  return (float)ldexp(m, -d);
}

/* Transfer function: linear interpolation over 256 entries spanning [vmin, vmax]. */
static void tf_lookup(const orc_tf *tf, double v, double rgba[4]) {
  double x = (v - tf->vmin) / (tf->vmax - tf->vmin);
  if (!(x > 0.0)) x = 0.0;
  if (x > 1.0) x = 1.0;
  x *= 255.0;
  int i0 = (int)floor(x);
  if (i0 > 254) i0 = 254;
  double f = x - (double)i0;
  for (int c = 0; c < 4; ++c) rgba[c] = (1.0 - f) * tf->table[4 * i0 + c] + f * tf->table[4 * (i0 + 1) + c];
}

typedef struct {
  int64_t samples;
  int64_t lookups;
  int64_t rays_hit;
} orc_stats;

typedef struct {
  const orc_vol *v;
  const orc_camera *cam;
  const orc_tf *tf;
  const orc_step *st;
  const int32_t *pix; /* npix x 2 (i, j) or NULL for the full image */
  int64_t npix;
  double *rgba; /* npix x 4 */
  int tid, nth;
  orc_stats stats;
  int32_t max_trace; /* records kept per pixel (trace only) */
  double *trace;     /* NULL, or npix x max_trace x 4: t, element id, value, segment */
  int32_t *count;    /* NULL, or npix: samples composited */
} render_job;

static void *render_worker(void *arg) {
  render_job *J = (render_job *)arg;
  const orc_vol *v = J->v;
  ray_consts K;
  camera_consts(J->cam, &K);
  int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * v->n_basis);
  double val[3];
  for (int64_t q = J->tid; q < J->npix; q += J->nth) {
    int i = J->pix ? J->pix[2 * q] : (int)(q % J->cam->width);
    int j = J->pix ? J->pix[2 * q + 1] : (int)(q / J->cam->width);
    double *out = J->rgba + 4 * q;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    float o[3], d[3], tin, tout;
    if (!ray_setup(&K, i, j, o, d, &tin, &tout)) continue;
    if (J->st->trim && !trim_interval(J->st->trim + 2 * ((int64_t)j * J->cam->width + i), &tin, &tout)) continue;
    J->stats.rays_hit++;
    double C[3] = {0, 0, 0}, A = 0.0;
    uint32_t cur = ORC_NONE;
    int64_t ninc = 0;
    float t = tin;
    int64_t k = 0;
    while (t < tout) {
      float pf[3];
      double x[3];
      for (int c = 0; c < 3; ++c) {
        pf[c] = fminf(fmaxf(fmaf(t, d[c], o[c]), 0.0f), 1.0f);
        x[c] = (double)pf[c];
      }
      if (cur == ORC_NONE || !in_element(v, cur, x)) {
        cur = orc_find_element(v, x);
        ninc = orc_incidence(v, cur, inc);
        J->stats.lookups++;
      }
      float tn;
      if (J->st->mode == 1) {
        tn = t + orc_heuristic_step(v, cur);
      } else if (J->st->mode == 2) {
        /* learned step: the Eq. 4 step scaled by the element's multiplier, one FP32 product */
        tn = t + orc_heuristic_step(v, cur) * J->st->mult[cur];
      } else {
        tn = fmaf((float)(k + 1), (float)J->st->h, tin);
      }
      if (!(tn > t)) tn = nextafterf(t, INFINITY);
      double seg = (double)fminf(tn, tout) - (double)t;
      double shade = 1.0;
      if (J->st->shading) {
        /* I = max(0.4, |l . n|), l the unit vector towards the light */
        double g[9];
        eval_grad_with(v, inc, ninc, x, val, g);
        double l[3], ll = 0.0, gl = 0.0, gg = 0.0;
        for (int c = 0; c < 3; ++c) {
          l[c] = J->st->light[c];
          ll += l[c] * l[c];
        }
        if (ll == 0.0)
          for (int c = 0; c < 3; ++c) {
            l[c] = -(double)d[c];
            ll += l[c] * l[c];
          }
        for (int c = 0; c < 3; ++c) {
          gl += l[c] * g[c];
          gg += g[c] * g[c];
        }
        /* |grad f| below eps = 1e-3 (vmax - vmin) counts as no gradient, continuously:
           n = grad f / max(|grad f|, eps) */
        const double eps = 1e-3 * (J->tf->vmax - J->tf->vmin);
        double gn = sqrt(gg);
        if (gn < eps) gn = eps;
        shade = fabs(gl) / (gn * sqrt(ll));
        if (shade < 0.4) shade = 0.4;
      } else {
        eval_with(v, inc, ninc, x, val);
      }
      double s;
      if (J->st->field == 1)
        s = sqrt(val[0] * val[0] + val[1] * val[1] + val[2] * val[2]);
      else if (J->st->field == 2)
        s = val[J->st->component];
      else
        s = val[0];
      if (J->trace && k < J->max_trace) {
        double *rec = J->trace + 4 * ((int64_t)q * J->max_trace + k);
        rec[0] = (double)t;
        rec[1] = (double)cur;
        rec[2] = s;
        rec[3] = seg;
      }
      double src[4];
      tf_lookup(J->tf, s, src);
      /* Alg. 2 */
      double T = pow(1.0 - src[3], seg / J->st->xi);
      double w = (1.0 - T) * (1.0 - A);
      for (int c = 0; c < 3; ++c) C[c] += w * shade * src[c];
      A += w;
      J->stats.samples++;
      ++k;
      t = tn;
      if (A >= J->st->alpha_stop) break;
    }
    out[0] = C[0];
    out[1] = C[1];
    out[2] = C[2];
    out[3] = A;
    if (J->count) J->count[q] = (int32_t)k;
  }
  free(inc);
  return NULL;
}

static void render_common(const orc_vol *v, const orc_camera *cam, const orc_tf *tf, const orc_step *st,
                          const int32_t *pix, int64_t npix, double *rgba, int nth, orc_stats *stats,
                          int32_t max_trace, double *trace, int32_t *count) {
  if (nth < 1) nth = 1;
  if (!pix) npix = (int64_t)cam->width * cam->height;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nth);
  render_job *jobs = (render_job *)calloc(nth, sizeof(render_job));
  for (int t = 0; t < nth; ++t) {
    render_job J = {v, cam, tf, st, pix, npix, rgba, t, nth, {0, 0, 0}, max_trace, trace, count};
    jobs[t] = J;
    pthread_create(&th[t], NULL, render_worker, &jobs[t]);
  }
  orc_stats s = {0, 0, 0};
  for (int t = 0; t < nth; ++t) {
    pthread_join(th[t], NULL);
    s.samples += jobs[t].stats.samples;
    s.lookups += jobs[t].stats.lookups;
    s.rays_hit += jobs[t].stats.rays_hit;
  }
  if (stats) *stats = s;
  free(th);
  free(jobs);
}

/* Render npix pixels (pix = NULL: the whole width x height image, row major). */
void orc_render(const orc_vol *v, const orc_camera *cam, const orc_tf *tf, const orc_step *st,
                const int32_t *pix, int64_t npix, double *rgba, int nth, orc_stats *stats) {
  render_common(v, cam, tf, st, pix, npix, rgba, nth, stats, 0, NULL, NULL);
}

/* The same march, also keeping each pixel's samples in order: for sample k <
   max_trace of pixel q, trace[q][k] = (t_k, element id, value before the
   transfer function, segment min(t_{k+1}, t_out) - t_k), and count[q] = the
   samples composited (Sec. 4, Alg. 1, Eq. 4, Alg. 2). */
void orc_render_trace(const orc_vol *v, const orc_camera *cam, const orc_tf *tf, const orc_step *st,
                      const int32_t *pix, int64_t npix, int32_t max_trace, double *trace, int32_t *count,
                      double *rgba, int nth, orc_stats *stats) {
  render_common(v, cam, tf, st, pix, npix, rgba, nth, stats, max_trace, trace, count);
}

/* The FP32 ray of one pixel (for tests of the ray setup). */
int orc_ray(const orc_camera *cam, int i, int j, float *o, float *d, float *tin, float *tout) {
  ray_consts K;
  camera_consts(cam, &K);
  return ray_setup(&K, i, j, o, d, tin, tout);
}

/* ------------------------------------------------------------------------ */
/* Training labels of the learned step (the definition in lrvol.h, FP64      */
/* compositing).  Per ray: the Eq. 4 march defines visits [t_a, t_b) and the */
/* reference transmittance T_front in front of each.  Candidate i marches    */
/* from t_a with cand[i] times the element's Eq. 4 step until its first      */
/* sample outside the element, t_i; over [t_a, t_i) Alg. 2 runs from         */
/* transparent with that step and with the fine step (reference), every      */
/* sample evaluated in the element that holds it, so the error includes     */
/* what the long last step skips of the next elements.  Candidate i is       */
/* acceptable when T_front * max(|dC|, |d alpha|) <= tau; the label of the  */
/* element is the smallest, over its visits, largest prefix of acceptable    */
/* candidates.                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t cur;
  int64_t ninc;
  int64_t *inc;
} seg_cache;

static void seg_eval_at(const orc_vol *v, seg_cache *sc, const float pf[3], double val[3]) {
  double x[3] = {(double)pf[0], (double)pf[1], (double)pf[2]};
  if (sc->cur == ORC_NONE || !in_element(v, sc->cur, x)) {
    sc->cur = orc_find_element(v, x);
    sc->ninc = orc_incidence(v, sc->cur, sc->inc);
  }
  eval_with(v, sc->inc, sc->ninc, x, val);
}

/* Alg. 2 from transparent over [ta, tb) with samples fmaf(k, h, ta). */
static void seg_composite(const orc_vol *v, const orc_tf *tf, const orc_step *st, const float o[3], const float d[3],
                          float ta, float tb, float h, seg_cache *sc, double C[3], double *A) {
  C[0] = C[1] = C[2] = 0.0;
  *A = 0.0;
  for (int64_t k = 0;; ++k) {
    float t = fmaf((float)k, h, ta);
    if (!(t < tb)) break;
    float pf[3];
    for (int c = 0; c < 3; ++c) pf[c] = fminf(fmaxf(fmaf(t, d[c], o[c]), 0.0f), 1.0f);
    double val[3];
    seg_eval_at(v, sc, pf, val);
    float tn = fmaf((float)(k + 1), h, ta);
    double seg = (double)fminf(tn, tb) - (double)t;
    double src[4];
    tf_lookup(tf, val[0], src);
    double T = pow(1.0 - src[3], seg / st->xi);
    double w = (1.0 - T) * (1.0 - *A);
    for (int c = 0; c < 3; ++c) C[c] += w * src[c];
    *A += w;
  }
}

typedef struct {
  const orc_vol *v;
  const orc_camera *cam;
  const orc_tf *tf;
  const orc_step *st;
  double h_fine, tau;
  const float *cand;
  int n_cand;
  int32_t *label;
  int tid, nth;
} label_job;

static void *label_worker(void *arg) {
  label_job *J = (label_job *)arg;
  const orc_vol *v = J->v;
  ray_consts K;
  camera_consts(J->cam, &K);
  seg_cache sc = {ORC_NONE, 0, (int64_t *)malloc(sizeof(int64_t) * v->n_basis)};
  int64_t npix = (int64_t)J->cam->width * J->cam->height;
  for (int64_t q = J->tid; q < npix; q += J->nth) {
    int i = (int)(q % J->cam->width), j = (int)(q / J->cam->width);
    float o[3], d[3], tin, tout;
    if (!ray_setup(&K, i, j, o, d, &tin, &tout)) continue;
    double Tfront = 1.0;
    float t = tin;
    while (t < tout && Tfront > 1.0 - J->st->alpha_stop) {
      float pf[3];
      double x[3];
      for (int c = 0; c < 3; ++c) {
        pf[c] = fminf(fmaxf(fmaf(t, d[c], o[c]), 0.0f), 1.0f);
        x[c] = (double)pf[c];
      }
      uint32_t e = orc_find_element(v, x);
      float ds = orc_heuristic_step(v, e);
      float tb = t;
      for (;;) {
        tb = tb + ds;
        if (!(tb < tout)) break;
        for (int c = 0; c < 3; ++c) x[c] = (double)fminf(fmaxf(fmaf(tb, d[c], o[c]), 0.0f), 1.0f);
        if (!in_element(v, e, x)) break;
      }
      tb = fminf(tb, tout);
      double R[3], RA, Cc[3], CA, F[3], FA;
      seg_composite(v, J->tf, J->st, o, d, t, tb, (float)J->h_fine, &sc, R, &RA);
      int best = 0;
      for (int c = 1; c < J->n_cand; ++c) {
        /* the candidate's first sample outside e (or the ray's exit) */
        float s = ds * J->cand[c], tc = t;
        for (int64_t k = 1;; ++k) {
          tc = fmaf((float)k, s, t);
          if (!(tc < tout)) break;
          for (int ch = 0; ch < 3; ++ch) x[ch] = (double)fminf(fmaxf(fmaf(tc, d[ch], o[ch]), 0.0f), 1.0f);
          if (!in_element(v, e, x)) break;
        }
        tc = fminf(tc, tout);
        seg_composite(v, J->tf, J->st, o, d, t, tc, (float)J->h_fine, &sc, F, &FA);
        seg_composite(v, J->tf, J->st, o, d, t, tc, s, &sc, Cc, &CA);
        double err = fabs(CA - FA);
        for (int ch = 0; ch < 3; ++ch)
          if (fabs(Cc[ch] - F[ch]) > err) err = fabs(Cc[ch] - F[ch]);
        if (!(Tfront * err <= J->tau)) break;
        best = c;
      }
      if (best < J->label[e]) J->label[e] = best;
      Tfront *= 1.0 - RA;
      t = tb;
    }
  }
  free(sc.inc);
  return NULL;
}

/* label: n_elem int32, in/out (min over visits); thread-private copies merged by min. */
void orc_labels(const orc_vol *v, const orc_camera *cam, const orc_tf *tf, const orc_step *st, double h_fine,
                double tau, const float *cand, int n_cand, int32_t *label, int nth) {
  if (nth < 1) nth = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nth);
  label_job *jobs = (label_job *)malloc(sizeof(label_job) * nth);
  for (int t = 0; t < nth; ++t) {
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * v->n_elem);
    memcpy(own, label, sizeof(int32_t) * v->n_elem);
    label_job J = {v, cam, tf, st, h_fine, tau, cand, n_cand, own, t, nth};
    jobs[t] = J;
    pthread_create(&th[t], NULL, label_worker, &jobs[t]);
  }
  for (int t = 0; t < nth; ++t) {
    pthread_join(th[t], NULL);
    for (int64_t e = 0; e < v->n_elem; ++e)
      if (jobs[t].label[e] < label[e]) label[e] = jobs[t].label[e];
    free(jobs[t].label);
  }
  free(th);
  free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Streamlines (Sec. 5): dx/dt = f(x) by explicit Runge-Kutta methods (Eq. 5) */
/* in FP64, f evaluated by Eq. 2.  Butcher tableaus of the published         */
/* methods; the step is fixed, the Eq. 4 step of the element holding x_n     */
/* times a base factor (Sec. 5.2), or chosen by the embedded error estimate. */
/* Element decisions (the Eq. 4 step, leaving the domain) are taken on the   */
/* FP32 rounding of the point, as for ray samples.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t method;    /* 0 RK1 .. 8 RKF45 (order of the list in lrvol.h) */
  int32_t step_rule; /* 0 fixed, 1 Eq. 4 times h, 2 adaptive (embedded methods) */
  double h, t_end, tol;
  int32_t max_samples;
} orc_sl_params;

typedef struct {
  int s;            /* stages */
  double c[6], a[6][6], b[6], bh[6];
  int embedded, q_low; /* bh: the other solution of an embedded pair, q_low its order */
} orc_tableau;

static void tableau_of(int m, orc_tableau *T) {
  memset(T, 0, sizeof(*T));
  switch (m) {
    case 0: /* explicit Euler */
      T->s = 1; T->b[0] = 1.0;
      break;
    case 1: /* explicit midpoint */
      T->s = 2; T->c[1] = 0.5; T->a[1][0] = 0.5; T->b[1] = 1.0;
      break;
    case 2: /* Kutta's third-order method */
      T->s = 3; T->c[1] = 0.5; T->c[2] = 1.0;
      T->a[1][0] = 0.5; T->a[2][0] = -1.0; T->a[2][1] = 2.0;
      T->b[0] = 1.0 / 6; T->b[1] = 2.0 / 3; T->b[2] = 1.0 / 6;
      break;
    case 3: /* classic fourth order */
      T->s = 4; T->c[1] = 0.5; T->c[2] = 0.5; T->c[3] = 1.0;
      T->a[1][0] = 0.5; T->a[2][1] = 0.5; T->a[3][2] = 1.0;
      T->b[0] = 1.0 / 6; T->b[1] = 1.0 / 3; T->b[2] = 1.0 / 3; T->b[3] = 1.0 / 6;
      break;
    case 4: /* 3/8 rule */
      T->s = 4; T->c[1] = 1.0 / 3; T->c[2] = 2.0 / 3; T->c[3] = 1.0;
      T->a[1][0] = 1.0 / 3; T->a[2][0] = -1.0 / 3; T->a[2][1] = 1.0;
      T->a[3][0] = 1.0; T->a[3][1] = -1.0; T->a[3][2] = 1.0;
      T->b[0] = 1.0 / 8; T->b[1] = 3.0 / 8; T->b[2] = 3.0 / 8; T->b[3] = 1.0 / 8;
      break;
    case 5: /* Fehlberg, fifth-order solution */
    case 8: /* Fehlberg 4(5), fifth order propagated, fourth order for the estimate */
      T->s = 6;
      T->c[1] = 0.25; T->c[2] = 3.0 / 8; T->c[3] = 12.0 / 13; T->c[4] = 1.0; T->c[5] = 0.5;
      T->a[1][0] = 0.25;
      T->a[2][0] = 3.0 / 32; T->a[2][1] = 9.0 / 32;
      T->a[3][0] = 1932.0 / 2197; T->a[3][1] = -7200.0 / 2197; T->a[3][2] = 7296.0 / 2197;
      T->a[4][0] = 439.0 / 216; T->a[4][1] = -8.0; T->a[4][2] = 3680.0 / 513; T->a[4][3] = -845.0 / 4104;
      T->a[5][0] = -8.0 / 27; T->a[5][1] = 2.0; T->a[5][2] = -3544.0 / 2565; T->a[5][3] = 1859.0 / 4104;
      T->a[5][4] = -11.0 / 40;
      T->b[0] = 16.0 / 135; T->b[2] = 6656.0 / 12825; T->b[3] = 28561.0 / 56430; T->b[4] = -9.0 / 50;
      T->b[5] = 2.0 / 55;
      T->bh[0] = 25.0 / 216; T->bh[2] = 1408.0 / 2565; T->bh[3] = 2197.0 / 4104; T->bh[4] = -1.0 / 5;
      T->embedded = m == 8; T->q_low = 4;
      break;
    case 6: /* Heun-Euler 2(1) */
      T->s = 2; T->c[1] = 1.0; T->a[1][0] = 1.0;
      T->b[0] = 0.5; T->b[1] = 0.5;
      T->bh[0] = 1.0;
      T->embedded = 1; T->q_low = 1;
      break;
    case 7: /* Bogacki-Shampine 3(2) */
      T->s = 4; T->c[1] = 0.5; T->c[2] = 0.75; T->c[3] = 1.0;
      T->a[1][0] = 0.5; T->a[2][1] = 0.75;
      T->a[3][0] = 2.0 / 9; T->a[3][1] = 1.0 / 3; T->a[3][2] = 4.0 / 9;
      T->b[0] = 2.0 / 9; T->b[1] = 1.0 / 3; T->b[2] = 4.0 / 9;
      T->bh[0] = 7.0 / 24; T->bh[1] = 0.25; T->bh[2] = 1.0 / 3; T->bh[3] = 0.125;
      T->embedded = 1; T->q_low = 2;
      break;
  }
}

/* inside [0,1]^3 as an FP32 point; its element through e (cached) */
static int sl_point(const orc_vol *v, const double *x, uint32_t *e, double xf[3]) {
  for (int a = 0; a < 3; ++a) {
    xf[a] = (double)(float)x[a];
    if (!(xf[a] >= 0.0 && xf[a] <= 1.0)) return 0;
  }
  if (*e == ORC_NONE || !in_element(v, *e, xf)) *e = orc_find_element(v, xf);
  return *e != ORC_NONE;
}

typedef struct {
  const orc_vol *v;
  const orc_sl_params *P;
  const double *seeds;
  int64_t n;
  double *out;
  int32_t *count, *status;
  int tid, nth;
} sl_job;

static void *sl_worker(void *arg) {
  sl_job *J = (sl_job *)arg;
  const orc_vol *v = J->v;
  const orc_sl_params *P = J->P;
  orc_tableau T;
  tableau_of(P->method, &T);
  int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * v->n_basis);
  for (int64_t q = J->tid; q < J->n; q += J->nth) {
    double x[3] = {J->seeds[3 * q], J->seeds[3 * q + 1], J->seeds[3 * q + 2]};
    double *o = J->out + q * (int64_t)P->max_samples * 4;
    double t = 0.0, xf[3];
    uint32_t e = ORC_NONE, ei = ORC_NONE;
    int64_t ninc = 0;
    int n = 0, st = 0;
    if (!sl_point(v, x, &e, xf)) {
      J->count[q] = 0;
      J->status[q] = 1;
      continue;
    }
    o[0] = x[0]; o[1] = x[1]; o[2] = x[2]; o[3] = 0.0;
    n = 1;
    double h = P->step_rule == 0 ? P->h : (P->step_rule == 1 ? P->h * (double)orc_heuristic_step(v, e)
                                                             : (P->h > 0 ? P->h : (double)orc_heuristic_step(v, e)));
    for (;;) {
      if (!(t < P->t_end)) { st = 0; break; }
      if (n >= P->max_samples) { st = 2; break; }
      if (P->step_rule == 1) h = P->h * (double)orc_heuristic_step(v, e);
      if (P->step_rule == 0) h = P->h;
      int tries = 0, taken = 0, out = 0;
      double xn[3];
      while (!taken) {
        double hs = h, last = 0;
        if (t + hs > P->t_end) { hs = P->t_end - t; last = 1; }
        double k[6][3];
        for (int i = 0; i < T.s && !out; ++i) {
          double y[3];
          for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (int j = 0; j < i; ++j) acc += T.a[i][j] * k[j][a];
            y[a] = x[a] + hs * acc;
          }
          uint32_t es = e;
          if (!sl_point(v, y, &es, xf)) { out = 1; break; }
          if (es != ei) { ninc = orc_incidence(v, es, inc); ei = es; }
          /* the field is evaluated at the FP32 point (single-precision spline
             evaluation under a double-precision outer loop, Sec. 5.5) */
          double val[3];
          eval_with(v, inc, ninc, xf, val);
          for (int a = 0; a < 3; ++a) k[i][a] = val[a];
        }
        if (out) break;
        double dx[3], err2 = 0.0;
        for (int a = 0; a < 3; ++a) {
          double acc = 0.0, ea = 0.0;
          for (int i = 0; i < T.s; ++i) {
            acc += T.b[i] * k[i][a];
            ea += (T.b[i] - T.bh[i]) * k[i][a];
          }
          dx[a] = hs * acc;
          err2 += (hs * ea) * (hs * ea);
        }
        if (P->step_rule == 2) {
          double err = sqrt(err2);
          double fac = err > 0.0 ? 0.9 * pow(P->tol / err, 1.0 / (T.q_low + 1)) : 5.0;
          if (fac < 0.2) fac = 0.2;
          if (fac > 5.0) fac = 5.0;
          if (err > P->tol) {
            h = hs * fac;
            if (++tries >= 64) break;
            continue;
          }
          if (!last) h = hs * fac;
        }
        for (int a = 0; a < 3; ++a) xn[a] = x[a] + dx[a];
        uint32_t en = e;
        if (!sl_point(v, xn, &en, xf)) { out = 1; break; }
        e = en;
        t = last ? P->t_end : t + hs;
        taken = 1;
      }
      if (out) { st = 1; break; }
      if (!taken) { st = 3; break; }
      for (int a = 0; a < 3; ++a) x[a] = xn[a];
      double *w = o + 4 * n;
      w[0] = x[0]; w[1] = x[1]; w[2] = x[2]; w[3] = t;
      ++n;
    }
    J->count[q] = n;
    J->status[q] = st;
  }
  free(inc);
  return NULL;
}

/* n streamlines from seeds (n x 3); out n x max_samples x 4 (x, y, z, t),
 * count[n] samples written (the seed first), status[n]: 0 reached t_end,
 * 1 left the domain, 2 max_samples, 3 step control failed. */
void orc_streamlines(const orc_vol *v, const orc_sl_params *P, const double *seeds, int64_t n, double *out,
                     int32_t *count, int32_t *status, int nth) {
  if (nth < 1) nth = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nth);
  sl_job *jobs = (sl_job *)malloc(sizeof(sl_job) * nth);
  for (int t = 0; t < nth; ++t) {
    sl_job J = {v, P, seeds, n, out, count, status, t, nth};
    jobs[t] = J;
    pthread_create(&th[t], NULL, sl_worker, &jobs[t]);
  }
  for (int t = 0; t < nth; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Streamline tubes (Sec. 5.3): every segment of a streamline drawn as a     */
/* capsule of radius r.  Visibility is a decision, taken in FP32 with the    */
/* kernel's order of operations: per pixel the hit with the smallest t       */
/* (ties: the smallest segment index) wins.  The pixel's colour is the       */
/* colour map at the speed |f| of the closest point on the winning segment's */
/* axis, times I = max(0.4, |n . d|) with n the capsule normal at the hit;   */
/* alpha is 1.                                                               */
/* ------------------------------------------------------------------------ */
static float dot3f(const float *x, const float *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; }

static int capsule_hit(const float o[3], const float d[3], const float a[3], const float b[3], float r, float *t) {
  float ba[3], oa[3], ob[3];
  for (int c = 0; c < 3; ++c) {
    ba[c] = b[c] - a[c];
    oa[c] = o[c] - a[c];
    ob[c] = o[c] - b[c];
  }
  const float baba = dot3f(ba, ba), bard = dot3f(ba, d), baoa = dot3f(ba, oa);
  const float rdoa = dot3f(d, oa), oaoa = dot3f(oa, oa), rr = r * r;
  const float A = baba - bard * bard;
  if (A > 0.0f) {
    const float B = baba * rdoa - baoa * bard;
    const float C = baba * oaoa - baoa * baoa - rr * baba;
    const float H = B * B - A * C;
    if (H >= 0.0f) {
      const float tb = (-B - sqrtf(H)) / A;
      const float y = baoa + tb * bard;
      if (y > 0.0f && y < baba) {
        if (tb > 0.0f) {
          *t = tb;
          return 1;
        }
        return 0;
      }
    }
  }
  /* the caps: spheres at a and b, nearer positive hit */
  float best = INFINITY;
  for (int k = 0; k < 2; ++k) {
    const float *oc = k == 0 ? oa : ob;
    const float bb = dot3f(d, oc), cc = dot3f(oc, oc) - rr;
    const float h = bb * bb - cc;
    if (h > 0.0f) {
      const float tc = -bb - sqrtf(h);
      if (tc > 0.0f && tc < best) best = tc;
    }
  }
  if (best < INFINITY) {
    *t = best;
    return 1;
  }
  return 0;
}

typedef struct {
  const orc_vol *v;
  const orc_camera *cam;
  const float *seg; /* n_seg x 6: a, b (FP32) */
  int64_t n_seg;
  float radius;
  const orc_tf *cmap;
  double *out;
  int tid, nth;
} tube_job;

static void *tube_worker(void *arg) {
  tube_job *J = (tube_job *)arg;
  ray_consts K;
  camera_consts(J->cam, &K);
  int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * J->v->n_basis);
  const int64_t npix = (int64_t)J->cam->width * J->cam->height;
  for (int64_t q = J->tid; q < npix; q += J->nth) {
    const int i = (int)(q % J->cam->width), j = (int)(q / J->cam->width);
    float o[3], d[3], tin, tout;
    ray_setup(&K, i, j, o, d, &tin, &tout);
    float tbest = INFINITY;
    int64_t sbest = -1;
    for (int64_t s = 0; s < J->n_seg; ++s) {
      float t;
      if (!capsule_hit(o, d, J->seg + 6 * s, J->seg + 6 * s + 3, J->radius, &t)) continue;
      if (t < tbest) { /* strictly smaller: the first (smallest) index wins ties */
        tbest = t;
        sbest = s;
      }
    }
    double *out = J->out + 4 * q;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (sbest < 0) continue;
    const float *a = J->seg + 6 * sbest, *b = a + 3;
    float p[3], ba[3], pa[3], qa[3];
    for (int c = 0; c < 3; ++c) {
      p[c] = o[c] + tbest * d[c];
      ba[c] = b[c] - a[c];
      pa[c] = p[c] - a[c];
    }
    const float baba = dot3f(ba, ba);
    float hcl = baba > 0.0f ? dot3f(pa, ba) / baba : 0.0f;
    if (hcl < 0.0f) hcl = 0.0f;
    if (hcl > 1.0f) hcl = 1.0f;
    for (int c = 0; c < 3; ++c) qa[c] = a[c] + hcl * ba[c];
    /* speed at the axis point (FP32 position, FP64 field) */
    double x[3] = {qa[0], qa[1], qa[2]}, val[3] = {0.0, 0.0, 0.0};
    const uint32_t e = orc_find_element(J->v, x);
    if (e != ORC_NONE) {
      const int64_t n = orc_incidence(J->v, e, inc);
      eval_with(J->v, inc, n, x, val);
    }
    const double speed = sqrt(val[0] * val[0] + val[1] * val[1] + val[2] * val[2]);
    double rgba[4];
    tf_lookup(J->cmap, speed, rgba);
    double nrm[3], nn = 0.0, nd = 0.0;
    for (int c = 0; c < 3; ++c) {
      nrm[c] = (double)p[c] - (double)qa[c];
      nn += nrm[c] * nrm[c];
      nd += nrm[c] * (double)d[c];
    }
    double I = nn > 0.0 ? fabs(nd) / sqrt(nn) : 1.0;
    if (I < 0.4) I = 0.4;
    out[0] = I * rgba[0];
    out[1] = I * rgba[1];
    out[2] = I * rgba[2];
    out[3] = 1.0;
  }
  free(inc);
  return NULL;
}

/* RGBA (H x W x 4, FP64) of n_seg capsule segments (FP32 a, b per segment). */
void orc_tubes(const orc_vol *v, const orc_camera *cam, const float *seg, int64_t n_seg, float radius,
               const orc_tf *cmap, double *out, int nth) {
  if (nth < 1) nth = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nth);
  tube_job *jobs = (tube_job *)malloc(sizeof(tube_job) * nth);
  for (int t = 0; t < nth; ++t) {
    tube_job J = {v, cam, seg, n_seg, radius, cmap, out, t, nth};
    jobs[t] = J;
    pthread_create(&th[t], NULL, tube_worker, &jobs[t]);
  }
  for (int t = 0; t < nth; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}
