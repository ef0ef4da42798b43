/*
 * hlbm_oracle.c -- plain, slow FP64 CPU oracle of one HLBM time step.
 *
 * TEST INFRASTRUCTURE ONLY (see hlbm_oracle.h).  Straight loops, two lattices,
 * no blocking, no fusion, no reordering beyond the paper's own order of
 * operations, so that every line can be checked against the paper by eye.
 *
 * Build: plain C99, no fast-math, and floating-point contraction switched off
 * (-ffp-contract=off) so that the single FP32 decision below rounds every
 * operation on its own, on x86-64 and on aarch64 alike.  Built a second time
 * with -fopenmp for timing on all host cores: the collision and streaming
 * loops over z slices and the momentum-exchange loop over particles are
 * shared among threads; every cell and every particle is still computed by
 * one thread with the same operations, so both builds give identical
 * results.
 *
 * Citations are to the paper's sections and equations (arXiv:2312.14172):
 *   Sec. 2.2   Newton-Euler equations (Eqs. particlemotiontrans, motionrot)
 *   Sec. 3.1   D3Q19 set, moments, collision (Eq. collide), streaming
 *              (Eq. stream), BGK (Eq. bgk), relaxation time (Eq. relaxation),
 *              equilibrium (Eq. maxbolt), weights and speed of sound
 *   Sec. 3.2   indicator B (Eq. B), velocity difference (Eq. hlbm:du),
 *              exact-difference source (Eq. kupershtokh), momentum exchange
 *              (Eq. hlbm:mea), force and torque sums (Eqs. hydrodynamicforce,
 *              hydrodynamictorque)
 *   Sec. 4.2.5 order of one time step (Algorithm 1)
 *   Sec. 5.1   external force on a particle, weight minus buoyancy
 */
#include "hlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q ORACLE_Q
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: the D3Q19 velocity set, written as listed in the paper: the rest
 * vector, the six axis vectors, then the twelve face diagonals.  Within each
 * group the order is this library's convention (each vector is followed by
 * its opposite). */
static const int C[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
};

/* Sec. 3.1: weights 1/3 (rest), 1/18 (axis), 1/36 (diagonal). */
static double weight_of(int i) {
  int n2 = C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2];
  if (n2 == 0) return 1.0 / 3.0;
  if (n2 == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* the index ibar with c_ibar = -c_i, found by search (Sec. 3.2, below Eq. hlbm:mea) */
static int opposite_of(int i) {
  for (int j = 0; j < Q; ++j)
    if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2]) return j;
  return -1;
}

void oracle_velocity_set(int c[Q][3], double w[Q], int opp[Q]) {
  for (int i = 0; i < Q; ++i) {
    for (int a = 0; a < 3; ++a) c[i][a] = C[i][a];
    w[i] = weight_of(i);
    opp[i] = opposite_of(i);
  }
}

/* Eq. maxbolt with c_s^2 = 1/3 (Sec. 3.1). */
void oracle_equilibrium(double rho, const double u[3], double feq[Q]) {
  const double cs2 = 1.0 / 3.0;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    feq[i] = weight_of(i) * rho *
             (1.0 + cu / cs2 + (cu * cu) / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. B.  The printed middle case misses one closing parenthesis; the reading
 * used is cos^2( (pi/2) (d/eps + 1/2) ), which is continuous at d = +-eps/2
 * and gives B(0) = 1/2. */
double oracle_indicator(double d, double eps) {
  if (d <= -eps / 2.0) return 1.0;
  if (d >= eps / 2.0) return 0.0;
  double c = cos(PI / 2.0 * (d / eps + 0.5));
  return c * c;
}

/* Signed distance d_s (Sec. 3.2: negative inside, positive outside) of a
 * body-frame offset.  The paper's studies use spheres; for the other shapes
 * (the paper allows any shape, Sec. 5.4) these readings are used:
 *   sphere, radius a[0]:        |r| - a
 *   cuboid, half-extents a:     exact box distance
 *   ellipsoid, semi-axes a:     gradient-normalised algebraic distance
 *                               (k - 1) k / |r / a^2| with k = |r / a|, which
 *                               equals |r| - a for a sphere
 *   capsule, radius a[0], half-length a[2] of its axis segment (body z):
 *                               exact distance |r - clamp(r_z, -a[2], a[2]) e_z| - a[0] */
double oracle_sdf_body(int shape, const double a[3], const double r[3]) {
  if (shape == ORACLE_SPHERE) {
    return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) - a[0];
  }
  if (shape == ORACLE_CAPSULE) {
    double c = r[2] < -a[2] ? -a[2] : (r[2] > a[2] ? a[2] : r[2]);
    double t = r[2] - c;
    return sqrt(r[0] * r[0] + r[1] * r[1] + t * t) - a[0];
  }
  if (shape == ORACLE_ELLIPSOID) {
    double k2 = 0.0, g2 = 0.0;
    for (int j = 0; j < 3; ++j) {
      k2 += (r[j] / a[j]) * (r[j] / a[j]);
      g2 += (r[j] / (a[j] * a[j])) * (r[j] / (a[j] * a[j]));
    }
    if (g2 == 0.0) {
      double amin = a[0];
      if (a[1] < amin) amin = a[1];
      if (a[2] < amin) amin = a[2];
      return -amin;
    }
    double k = sqrt(k2);
    return (k - 1.0) * k / sqrt(g2);
  }
  /* cuboid */
  double qv[3], out2 = 0.0, qmax = -1e300;
  for (int j = 0; j < 3; ++j) {
    qv[j] = fabs(r[j]) - a[j];
    if (qv[j] > 0.0) out2 += qv[j] * qv[j];
    if (qv[j] > qmax) qmax = qv[j];
  }
  return sqrt(out2) + (qmax < 0.0 ? qmax : 0.0);
}

/* Rotation (body -> world) of a unit quaternion q = (w, x, y, z); row-major. */
void oracle_rotation(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* A signed-distance grid (shape ORACLE_GRID): FP32 samples of the signed
 * distance on a regular body-frame grid, point (i, j, k) at
 * ((i - (n0 - 1)/2) h, (j - (n1 - 1)/2) h, (k - (n2 - 1)/2) h), x fastest,
 * with what the library derives from it at registration. */
typedef struct {
  int n[3];
  double h;
  float* v;
  double V, I1[3]; /* volume and principal moments per unit density */
  double rc;       /* radius of the cells holding any negative corner */
  double rinf;     /* radius of the cells holding any corner below eps/2 */
} grid_shape;

/* Trilinear interpolation of a distance grid at the body-frame point r, in
 * FP64; +infinity (no coupling) outside the grid's box.  The reading of a
 * voxelised distance (the paper's outlook on arbitrary shapes, Sec. 6): the
 * distance between samples is the trilinear blend of the eight corners of
 * the grid cell that holds the point. */
static double grid_value(const grid_shape* g, const double r[3]) {
  double t[3];
  int i0[3];
  for (int j = 0; j < 3; ++j) {
    double x = r[j] / g->h + 0.5 * (g->n[j] - 1);
    if (!(x >= 0.0 && x <= (double)(g->n[j] - 1))) return INFINITY;
    int i = (int)floor(x);
    if (i > g->n[j] - 2) i = g->n[j] - 2;
    i0[j] = i;
    t[j] = x - i;
  }
  double c[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        c[dz][dy][dx] = g->v[((long)(i0[2] + dz) * g->n[1] + (i0[1] + dy)) * g->n[0] + (i0[0] + dx)];
  double e[2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy) e[dz][dy] = c[dz][dy][0] + t[0] * (c[dz][dy][1] - c[dz][dy][0]);
  double f0 = e[0][0] + t[1] * (e[0][1] - e[0][0]);
  double f1 = e[1][0] + t[1] * (e[1][1] - e[1][0]);
  return f0 + t[2] * (f1 - f0);
}

/* The same blend in FP32, every operation rounded on its own in this order
 * (the inside test of a grid particle; see oracle_inside_fp32):
 *   x_j = b_j * fp32(1/h) + fp32((n_j - 1)/2); outside [0, n_j - 1]: not inside
 *   i_j = min(floor(x_j), n_j - 2), t_j = x_j - i_j
 *   lerp(a, b, t) = a + t * (b - a); along x (four), then y (two), then z */
static float grid_value_fp32(const grid_shape* g, const float b[3]) {
  float t[3];
  int i0[3];
  float ih = (float)(1.0 / g->h);
  for (int j = 0; j < 3; ++j) {
    float half = (float)(0.5 * (g->n[j] - 1));
    float x = b[j] * ih;
    x = x + half;
    if (!(x >= 0.0f && x <= (float)(g->n[j] - 1))) return INFINITY;
    int i = (int)floorf(x);
    if (i > g->n[j] - 2) i = g->n[j] - 2;
    i0[j] = i;
    t[j] = x - (float)i;
  }
  float c[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        c[dz][dy][dx] = g->v[((long)(i0[2] + dz) * g->n[1] + (i0[1] + dy)) * g->n[0] + (i0[0] + dx)];
  float e[2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy) {
      float d = c[dz][dy][1] - c[dz][dy][0];
      d = t[0] * d;
      e[dz][dy] = c[dz][dy][0] + d;
    }
  float d0 = e[0][1] - e[0][0];
  d0 = t[1] * d0;
  float f0 = e[0][0] + d0;
  float d1 = e[1][1] - e[1][0];
  d1 = t[1] * d1;
  float f1 = e[1][0] + d1;
  float d2 = f1 - f0;
  d2 = t[2] * d2;
  return f0 + d2;
}

/* "Cells whose centre is inside the particle" (Sec. 3.2, above Eq.
 * hydrodynamicforce).  Reading: strictly d_s < 0.  This yes/no decision is
 * taken in FP32, in the same precision and operation order as the GPU kernel,
 * so that both sides agree on the set of cells: every operation below is a
 * single rounded FP32 operation (the file is built without contraction).
 *   Xh = fp32(X), Xl = fp32(X - Xh)        position as a float pair
 *   r0 = fp32(cell) - Xh                  exact
 *   periodic axes: r0 -= L if r0 > L/2, r0 += L if r0 < -L/2 (exact)
 *   r  = r0 - Xl
 *   sphere:    (rx*rx + ry*ry) + rz*rz < fp32(a*a)
 *   ellipsoid: b = M^T r with M = fp32(R(q)), e_j = b_j * fp32(1/a_j),
 *              (e0*e0 + e1*e1) + e2*e2 < 1
 *   cuboid:    |b_j| < fp32(a_j) for all j
 *   capsule:   t = b2 - clamp(b2, -fp32(a2), fp32(a2)),
 *              (b0*b0 + b1*b1) + t*t < fp32(a0*a0)                          */
int oracle_inside_fp32(int shape, const double a[3], const double q[4], const double X[3],
                       const int cell[3], const int n[3], int bc_flags) {
  float r[3];
  for (int j = 0; j < 3; ++j) {
    float xh = (float)X[j];
    float xl = (float)(X[j] - (double)xh);
    float r0 = (float)cell[j] - xh;
    if (!(bc_flags & (1 << j))) {
      float L = (float)n[j];
      float half = 0.5f * L;
      if (r0 > half) r0 = r0 - L;
      else if (r0 < -half) r0 = r0 + L;
    }
    r[j] = r0 - xl;
  }
  if (shape == ORACLE_SPHERE) {
    float s = r[0] * r[0];
    s = s + r[1] * r[1];
    s = s + r[2] * r[2];
    return s < (float)(a[0] * a[0]);
  }
  double Rd[9];
  oracle_rotation(q, Rd);
  float M[9];
  for (int k = 0; k < 9; ++k) M[k] = (float)Rd[k];
  float b[3];
  for (int j = 0; j < 3; ++j) {
    /* (M^T r)_j = M[0][j] r0 + M[1][j] r1 + M[2][j] r2 */
    float t = M[0 * 3 + j] * r[0];
    t = t + M[1 * 3 + j] * r[1];
    t = t + M[2 * 3 + j] * r[2];
    b[j] = t;
  }
  if (shape == ORACLE_CAPSULE) {
    float h = (float)a[2];
    float c = b[2] < -h ? -h : (b[2] > h ? h : b[2]);
    float t = b[2] - c;
    float s = b[0] * b[0];
    s = s + b[1] * b[1];
    s = s + t * t;
    return s < (float)(a[0] * a[0]);
  }
  if (shape == ORACLE_ELLIPSOID) {
    float e0 = b[0] * (float)(1.0 / a[0]);
    float e1 = b[1] * (float)(1.0 / a[1]);
    float e2 = b[2] * (float)(1.0 / a[2]);
    float s = e0 * e0;
    s = s + e1 * e1;
    s = s + e2 * e2;
    return s < 1.0f;
  }
  return fabsf(b[0]) < (float)a[0] && fabsf(b[1]) < (float)a[1] && fabsf(b[2]) < (float)a[2];
}

/* The inside test of a grid particle: the FP32 offset r and body-frame
 * offset b = M^T r exactly as in oracle_inside_fp32, then the FP32 blend of
 * grid_value_fp32 strictly below zero. */
static int inside_grid_fp32(const grid_shape* g, const double q[4], const double X[3], const int cell[3],
                            const int n[3], int bc_flags) {
  float r[3];
  for (int j = 0; j < 3; ++j) {
    float xh = (float)X[j];
    float xl = (float)(X[j] - (double)xh);
    float r0 = (float)cell[j] - xh;
    if (!(bc_flags & (1 << j))) {
      float L = (float)n[j];
      float half = 0.5f * L;
      if (r0 > half) r0 = r0 - L;
      else if (r0 < -half) r0 = r0 + L;
    }
    r[j] = r0 - xl;
  }
  double Rd[9];
  oracle_rotation(q, Rd);
  float M[9], b[3];
  for (int k = 0; k < 9; ++k) M[k] = (float)Rd[k];
  for (int j = 0; j < 3; ++j) {
    float t = M[0 * 3 + j] * r[0];
    t = t + M[1 * 3 + j] * r[1];
    t = t + M[2 * 3 + j] * r[2];
    b[j] = t;
  }
  return grid_value_fp32(g, b) < 0.0f;
}

/* ------------------------------------------------------------------------ */
typedef struct {
  int shape;
  double a[3];
  const grid_shape* grid; /* ORACLE_GRID only */
  double X[3], U[3], W[3], q[4];
  double rho, V, m, I[3], rc;
  double F[3], T[3]; /* hydrodynamic force and torque of the last step */
} particle;

struct oracle_sim {
  int n[3];
  int bc;
  double tau, eps, g[3], ff[3];
  long ncell;
  double* f;    /* post-streaming populations f_i(x, t), [i][cell] */
  double* post; /* post-collision populations f*_i(x, t), [i][cell] */
  double* B;    /* indicator field */
  int* pid;     /* particle that owns B at a cell, or -1 */
  int np, cap;
  particle* p;
  long steps;
  double contact_k, contact_zeta; /* contact stiffness and range (0: off) */
  int ngrid;
  grid_shape* grids[ORACLE_MAX_GRIDS];
};

static double influence_radius(const particle* P, double eps);

static long cell_index(const oracle_sim* s, int x, int y, int z) {
  return ((long)z * s->n[1] + y) * s->n[0] + x;
}

static int is_wall(const oracle_sim* s, int axis) { return (s->bc >> axis) & 1; }

/* neighbour coordinate along one axis: wraps on periodic axes; returns -1 when
 * the neighbour lies beyond a wall */
static int neighbour(const oracle_sim* s, int axis, int x, int dx) {
  int y = x + dx;
  int n = s->n[axis];
  if (y >= 0 && y < n) return y;
  if (is_wall(s, axis)) return -1;
  return ((y % n) + n) % n;
}

/* minimum-image offset of the point x from the centre X along one axis */
static double min_image(const oracle_sim* s, int axis, double d) {
  if (is_wall(s, axis)) return d;
  double L = (double)s->n[axis];
  if (d > L / 2.0) return d - L;
  if (d < -L / 2.0) return d + L;
  return d;
}

static void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

oracle_sim* oracle_create(int nx, int ny, int nz, double tau, double eps, int bc_flags,
                          const double gravity[3], const double fluid_force[3]) {
  if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || !(eps > 0.0)) return NULL;
  oracle_sim* s = (oracle_sim*)calloc(1, sizeof(oracle_sim));
  s->n[0] = nx;
  s->n[1] = ny;
  s->n[2] = nz;
  s->bc = bc_flags & 7;
  s->tau = tau;
  s->eps = eps;
  for (int a = 0; a < 3; ++a) {
    s->g[a] = gravity ? gravity[a] : 0.0;
    s->ff[a] = fluid_force ? fluid_force[a] : 0.0;
  }
  s->ncell = (long)nx * ny * nz;
  s->f = (double*)malloc(sizeof(double) * Q * s->ncell);
  s->post = (double*)malloc(sizeof(double) * Q * s->ncell);
  s->B = (double*)malloc(sizeof(double) * s->ncell);
  s->pid = (int*)malloc(sizeof(int) * s->ncell);
  if (!s->f || !s->post || !s->B || !s->pid) {
    oracle_destroy(s);
    return NULL;
  }
  /* initial state: fluid at rest with rho = 1, i.e. f_i = w_i */
  for (int i = 0; i < Q; ++i)
    for (long x = 0; x < s->ncell; ++x) s->f[i * s->ncell + x] = weight_of(i);
  return s;
}

void oracle_destroy(oracle_sim* s) {
  if (!s) return;
  free(s->f);
  free(s->post);
  free(s->B);
  free(s->pid);
  free(s->p);
  for (int g = 0; g < s->ngrid; ++g) {
    free(s->grids[g]->v);
    free(s->grids[g]);
  }
  free(s);
}

long oracle_steps_done(const oracle_sim* s) { return s->steps; }
int oracle_num_particles(const oracle_sim* s) { return s->np; }

/* volume, mass and principal moments of inertia of the analytic shapes and
 * of registered grids */
static void shape_mass_properties(particle* P) {
  const double* a = P->a;
  if (P->shape == ORACLE_GRID) {
    P->V = P->grid->V;
    P->m = P->rho * P->V;
    for (int j = 0; j < 3; ++j) P->I[j] = P->rho * P->grid->I1[j];
    P->rc = P->grid->rc;
  } else if (P->shape == ORACLE_SPHERE) {
    P->V = 4.0 / 3.0 * PI * a[0] * a[0] * a[0];
    P->m = P->rho * P->V;
    for (int j = 0; j < 3; ++j) P->I[j] = 0.4 * P->m * a[0] * a[0];
    P->rc = a[0];
  } else if (P->shape == ORACLE_ELLIPSOID) {
    P->V = 4.0 / 3.0 * PI * a[0] * a[1] * a[2];
    P->m = P->rho * P->V;
    P->I[0] = P->m * (a[1] * a[1] + a[2] * a[2]) / 5.0;
    P->I[1] = P->m * (a[0] * a[0] + a[2] * a[2]) / 5.0;
    P->I[2] = P->m * (a[0] * a[0] + a[1] * a[1]) / 5.0;
    P->rc = a[0];
    if (a[1] > P->rc) P->rc = a[1];
    if (a[2] > P->rc) P->rc = a[2];
  } else if (P->shape == ORACLE_CAPSULE) {
    /* a cylinder of radius r and length 2h with two hemispherical caps; a
     * cap's moment about a diameter of its flat face is 2/5 m r^2, moved to
     * the centre through the cap's centroid (3r/8 from the face) */
    const double r = a[0], h = a[2];
    const double Vc = PI * r * r * 2.0 * h, Vs = 4.0 / 3.0 * PI * r * r * r;
    P->V = Vc + Vs;
    P->m = P->rho * P->V;
    const double mc = P->rho * Vc, ms = P->rho * Vs;
    P->I[0] = P->I[1] = mc * (r * r / 4.0 + h * h / 3.0) + ms * (0.4 * r * r + h * h + 0.75 * h * r);
    P->I[2] = mc * r * r / 2.0 + ms * 0.4 * r * r;
    P->rc = h + r;
  } else {
    P->V = 8.0 * a[0] * a[1] * a[2];
    P->m = P->rho * P->V;
    P->I[0] = P->m * (a[1] * a[1] + a[2] * a[2]) / 3.0;
    P->I[1] = P->m * (a[0] * a[0] + a[2] * a[2]) / 3.0;
    P->I[2] = P->m * (a[0] * a[0] + a[1] * a[1]) / 3.0;
    P->rc = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  }
}

static void wrap_position(const oracle_sim* s, double X[3]) {
  for (int a = 0; a < 3; ++a) {
    if (is_wall(s, a)) continue;
    double L = (double)s->n[a];
    X[a] = X[a] - L * floor(X[a] / L);
    if (X[a] >= L) X[a] -= L;
  }
}

int oracle_add_particles(oracle_sim* s, int n, const int* shape, const double* a,
                         const double* X, const double* U, const double* omega,
                         const double* quat, const double* rho_p) {
  if (n < 0) return -1;
  if (s->steps > 0) return -5;
  if (s->np + n > s->cap) {
    int cap = s->cap ? s->cap : 16;
    while (cap < s->np + n) cap *= 2;
    particle* np_ = (particle*)realloc(s->p, sizeof(particle) * cap);
    if (!np_) return -1;
    s->p = np_;
    s->cap = cap;
  }
  for (int k = 0; k < n; ++k) {
    particle P;
    memset(&P, 0, sizeof(P));
    P.shape = shape[k];
    if (P.shape < 0 || P.shape > 4) return -1;
    if (P.shape == ORACLE_GRID) {
      double id = a[3 * k];
      if (!(id >= 0.0 && id < s->ngrid && id == floor(id))) return -1;
      P.grid = s->grids[(int)id];
    }
    for (int j = 0; j < 3; ++j) {
      P.a[j] = (P.shape == ORACLE_SPHERE || P.shape == ORACLE_GRID || (P.shape == ORACLE_CAPSULE && j == 1))
                   ? a[3 * k] : a[3 * k + j];
      if (!(P.a[j] > 0.0) && P.shape != ORACLE_GRID) return -1;
      P.X[j] = X[3 * k + j];
      P.U[j] = U ? U[3 * k + j] : 0.0;
      P.W[j] = omega ? omega[3 * k + j] : 0.0;
    }
    if (quat) {
      double nq = 0.0;
      for (int j = 0; j < 4; ++j) nq += quat[4 * k + j] * quat[4 * k + j];
      if (!(nq > 0.0)) return -1;
      nq = sqrt(nq);
      for (int j = 0; j < 4; ++j) P.q[j] = quat[4 * k + j] / nq;
    } else {
      P.q[0] = 1.0;
    }
    P.rho = rho_p[k];
    if (!(P.rho > 0.0)) return -1;
    shape_mass_properties(&P);
    for (int j = 0; j < 3; ++j) {
      if (is_wall(s, j)) {
        if (!(P.X[j] > -0.5 && P.X[j] < s->n[j] - 0.5)) return -1;
      } else if (!(2.0 * (influence_radius(&P, s->eps) + 2.0) < s->n[j])) {
        return -1;
      }
    }
    wrap_position(s, P.X);
    s->p[s->np + k] = P;
  }
  s->np += n;
  return 0;
}

int oracle_set_particle_state(oracle_sim* s, const double* X, const double* U,
                              const double* omega, const double* quat) {
  for (int k = 0; k < s->np; ++k) {
    particle* P = &s->p[k];
    for (int j = 0; j < 3; ++j) {
      if (X) P->X[j] = X[3 * k + j];
      if (U) P->U[j] = U[3 * k + j];
      if (omega) P->W[j] = omega[3 * k + j];
    }
    if (quat) {
      double nq = 0.0;
      for (int j = 0; j < 4; ++j) nq += quat[4 * k + j] * quat[4 * k + j];
      if (!(nq > 0.0)) return -1;
      nq = sqrt(nq);
      for (int j = 0; j < 4; ++j) P->q[j] = quat[4 * k + j] / nq;
    }
    wrap_position(s, P->X);
  }
  return 0;
}

void oracle_particle_state(const oracle_sim* s, double* X, double* U, double* omega,
                           double* quat, double* F, double* T) {
  for (int k = 0; k < s->np; ++k) {
    const particle* P = &s->p[k];
    for (int j = 0; j < 3; ++j) {
      if (X) X[3 * k + j] = P->X[j];
      if (U) U[3 * k + j] = P->U[j];
      if (omega) omega[3 * k + j] = P->W[j];
      if (F) F[3 * k + j] = P->F[j];
      if (T) T[3 * k + j] = P->T[j];
    }
    if (quat)
      for (int j = 0; j < 4; ++j) quat[4 * k + j] = P->q[j];
  }
}

void oracle_get_populations(const oracle_sim* s, double* f) {
  memcpy(f, s->f, sizeof(double) * Q * s->ncell);
}

void oracle_set_populations(oracle_sim* s, const double* f) {
  memcpy(s->f, f, sizeof(double) * Q * s->ncell);
}

/* ------------------------------------------------------------------------ */
/* Eq. hlbm:mea as printed, at cell x, on the post-streaming populations:
 *   sum_i (c_i - u_p) f_i(x + c_i) + (c_i + u_p) f_ibar(x).
 * Links whose far end x + c_i lies beyond a wall carry no fluid cell and are
 * left out. */
void oracle_mea_printed_cell(const oracle_sim* s, const int x[3], const double up[3],
                             double Fh[3]) {
  Fh[0] = Fh[1] = Fh[2] = 0.0;
  long cx = cell_index(s, x[0], x[1], x[2]);
  for (int i = 0; i < Q; ++i) {
    int y0 = neighbour(s, 0, x[0], C[i][0]);
    int y1 = neighbour(s, 1, x[1], C[i][1]);
    int y2 = neighbour(s, 2, x[2], C[i][2]);
    if (y0 < 0 || y1 < 0 || y2 < 0) continue;
    long cy = cell_index(s, y0, y1, y2);
    double fi_y = s->f[(long)i * s->ncell + cy];
    double fo_x = s->f[(long)opposite_of(i) * s->ncell + cx];
    for (int a = 0; a < 3; ++a) Fh[a] += (C[i][a] - up[a]) * fi_y + (C[i][a] + up[a]) * fo_x;
  }
}

/* Eqs. hydrodynamicforce and hydrodynamictorque: sums over the cells x_b
 * whose centre is inside particle p, at the particle state before this
 * step's update (Algorithm 1 couples fluid to particles first).
 *
 * Reading of the sign: evaluated on the post-streaming populations, the
 * printed sum of Eq. hlbm:mea is the momentum that cell x hands over to the
 * fluid through its links minus the momentum it receives (outflow minus
 * inflow, each shifted by the Galilean term with u_p).  The force the fluid
 * exerts on the particle is the opposite of that (Newton's third law), so the
 * printed per-cell sum enters here with a minus sign.
 *
 * The torque arm x_b - X_p is the minimum-image offset on periodic axes. */
long oracle_mea(const oracle_sim* s, int p, double F[3], double T[3]) {
  const particle* P = &s->p[p];
  long count = 0;
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)floor(P->X[a] - P->rc) - 1;
    hi[a] = (int)ceil(P->X[a] + P->rc) + 1;
    if (is_wall(s, a)) {
      if (lo[a] < 0) lo[a] = 0;
      if (hi[a] > s->n[a] - 1) hi[a] = s->n[a] - 1;
    }
  }
  F[0] = F[1] = F[2] = 0.0;
  T[0] = T[1] = T[2] = 0.0;
  for (int kz = lo[2]; kz <= hi[2]; ++kz)
    for (int ky = lo[1]; ky <= hi[1]; ++ky)
      for (int kx = lo[0]; kx <= hi[0]; ++kx) {
        int x[3];
        int k[3] = {kx, ky, kz};
        for (int a = 0; a < 3; ++a) x[a] = ((k[a] % s->n[a]) + s->n[a]) % s->n[a];
        if (P->shape == ORACLE_GRID ? !inside_grid_fp32(P->grid, P->q, P->X, x, s->n, s->bc)
                                    : !oracle_inside_fp32(P->shape, P->a, P->q, P->X, x, s->n, s->bc))
          continue;
        double r[3], wr[3], up[3], Fh[3], Fc[3], tc[3];
        for (int a = 0; a < 3; ++a) r[a] = min_image(s, a, (double)x[a] - P->X[a]);
        cross(P->W, r, wr);
        for (int a = 0; a < 3; ++a) up[a] = P->U[a] + wr[a]; /* u_p(x), Sec. 3.2 */
        oracle_mea_printed_cell(s, x, up, Fh);
        for (int a = 0; a < 3; ++a) Fc[a] = -Fh[a];
        cross(r, Fc, tc);
        for (int a = 0; a < 3; ++a) {
          F[a] += Fc[a];
          T[a] += tc[a];
        }
        ++count;
      }
  return count;
}

/* ------------------------------------------------------------------------ */
/* Eq. B over the lattice: B(x) = max over particles of B_p(d_s,p(x)).
 * Reading for overlapping smooth zones (the paper is silent): the largest B
 * wins and ties go to the lowest particle index; that particle also supplies
 * u_p(x).  B_p is evaluated only within the influence sphere |x - X_p| <
 * R_inf, outside of which d_s >= eps/2 and hence B_p = 0 exactly:
 *   sphere, cuboid, capsule (exact     R_inf = r_c + eps/2, r_c the
 *   distances):                        circumscribed radius;
 *   ellipsoid (algebraic distance):    d_s >= (k - 1) a_min and |r| <= k a_max
 *                                      give R_inf = a_max (1 + eps / (2 a_min)). */
static double influence_radius(const particle* P, double eps) {
  if (P->shape == ORACLE_GRID) return P->grid->rinf;
  if (P->shape == ORACLE_ELLIPSOID) {
    double amin = P->a[0], amax = P->a[0];
    for (int j = 1; j < 3; ++j) {
      if (P->a[j] < amin) amin = P->a[j];
      if (P->a[j] > amax) amax = P->a[j];
    }
    return amax * (1.0 + eps / (2.0 * amin));
  }
  return P->rc + eps / 2.0;
}

void oracle_indicator_field(const oracle_sim* s, double* B, int* pid) {
  for (long x = 0; x < s->ncell; ++x) {
    B[x] = 0.0;
    pid[x] = -1;
  }
  for (int p = 0; p < s->np; ++p) {
    const particle* P = &s->p[p];
    double rinf = influence_radius(P, s->eps);
    double R[9];
    oracle_rotation(P->q, R);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = (int)floor(P->X[a] - rinf) - 1;
      hi[a] = (int)ceil(P->X[a] + rinf) + 1;
      if (is_wall(s, a)) {
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > s->n[a] - 1) hi[a] = s->n[a] - 1;
      }
    }
    for (int kz = lo[2]; kz <= hi[2]; ++kz)
      for (int ky = lo[1]; ky <= hi[1]; ++ky)
        for (int kx = lo[0]; kx <= hi[0]; ++kx) {
          int k[3] = {kx, ky, kz}, x[3];
          double r[3], rb[3];
          for (int a = 0; a < 3; ++a) {
            x[a] = ((k[a] % s->n[a]) + s->n[a]) % s->n[a];
            r[a] = min_image(s, a, (double)x[a] - P->X[a]);
          }
          if (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] >= rinf * rinf) continue;
          /* body-frame offset R^T r */
          for (int j = 0; j < 3; ++j) rb[j] = R[0 * 3 + j] * r[0] + R[1 * 3 + j] * r[1] + R[2 * 3 + j] * r[2];
          double d = P->shape == ORACLE_GRID ? grid_value(P->grid, rb) : oracle_sdf_body(P->shape, P->a, rb);
          double b = oracle_indicator(d, s->eps);
          long c = cell_index(s, x[0], x[1], x[2]);
          if (b > B[c]) {
            B[c] = b;
            pid[c] = p;
          }
        }
  }
}

/* ------------------------------------------------------------------------ */
/* Collision of every cell (Eqs. collide, bgk, maxbolt) with the HLBM source
 * (Eqs. hlbm:du, kupershtokh).  rho and u come from the current populations
 * (Sec. 3.1); the velocity difference uses that plain u (reading: no
 * half-force shift inside Delta u).  A uniform body-force density F_f on the
 * fluid (zero unless set; the paper's counter pressure gradient of Sec. 5.1
 * enters this way) adds F_f / rho to the velocity shift of the same source. */
static void collide_into(const oracle_sim* s, const double* B, const int* pid, double* post) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int z = 0; z < s->n[2]; ++z)
    for (int y = 0; y < s->n[1]; ++y)
      for (int xx = 0; xx < s->n[0]; ++xx) {
        long c = cell_index(s, xx, y, z);
        double f[Q], rho = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3], du[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
          f[i] = s->f[(long)i * s->ncell + c];
          rho += f[i];
          for (int a = 0; a < 3; ++a) j[a] += C[i][a] * f[i];
        }
        for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
        if (pid && pid[c] >= 0) {
          const particle* P = &s->p[pid[c]];
          double r[3] = {min_image(s, 0, xx - P->X[0]), min_image(s, 1, y - P->X[1]),
                         min_image(s, 2, z - P->X[2])};
          double wr[3], up[3];
          cross(P->W, r, wr);
          for (int a = 0; a < 3; ++a) up[a] = P->U[a] + wr[a];
          for (int a = 0; a < 3; ++a) du[a] = B[c] * (up[a] - u[a]);
        }
        for (int a = 0; a < 3; ++a) du[a] += s->ff[a] / rho;
        double feq[Q], feq_shift[Q], ushift[3] = {u[0] + du[0], u[1] + du[1], u[2] + du[2]};
        oracle_equilibrium(rho, u, feq);
        oracle_equilibrium(rho, ushift, feq_shift);
        for (int i = 0; i < Q; ++i) {
          double omega_i = -(f[i] - feq[i]) / s->tau; /* Eq. bgk */
          double S_i = feq_shift[i] - feq[i];         /* Eq. kupershtokh */
          post[(long)i * s->ncell + c] = f[i] + omega_i + S_i; /* Eq. collide */
        }
      }
}

void oracle_collide_only(const oracle_sim* s, double* post) {
  double* B = (double*)malloc(sizeof(double) * s->ncell);
  int* pid = (int*)malloc(sizeof(int) * s->ncell);
  oracle_indicator_field(s, B, pid);
  collide_into(s, B, pid, post);
  free(B);
  free(pid);
}

/* Eq. stream, f_i(x + c_i, t + 1) = f*_i(x, t), written for each target cell
 * y as f_i(y) = f*_i(y - c_i).  Periodic axes wrap.  On a wall axis the node
 * beyond the wall is solid and the population returns by half-way bounce-back:
 * f_i(y, t + 1) = f*_ibar(y, t) when y - c_i is beyond the wall. */
void oracle_stream_only(oracle_sim* s, const double* post) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int z = 0; z < s->n[2]; ++z)
    for (int y = 0; y < s->n[1]; ++y)
      for (int x = 0; x < s->n[0]; ++x) {
        long c = cell_index(s, x, y, z);
        for (int i = 0; i < Q; ++i) {
          int s0 = neighbour(s, 0, x, -C[i][0]);
          int s1 = neighbour(s, 1, y, -C[i][1]);
          int s2 = neighbour(s, 2, z, -C[i][2]);
          double v;
          if (s0 < 0 || s1 < 0 || s2 < 0)
            v = post[(long)opposite_of(i) * s->ncell + c];
          else
            v = post[(long)i * s->ncell + cell_index(s, s0, s1, s2)];
          s->f[(long)i * s->ncell + c] = v;
        }
      }
}

/* ------------------------------------------------------------------------ */
/* Newton-Euler update of one particle with total force F and torque T
 * (Eqs. particlemotiontrans, motionrot).  The paper fixes neither the time
 * integrator nor the orientation representation; the reading used here:
 *   U <- U + F / m;  X <- X + U                         (symplectic Euler)
 *   sphere:  omega <- omega + T / I
 *   other:   omega_b = R^T omega, T_b = R^T T,
 *            omega_b <- omega_b + I^-1 (T_b - omega_b x (I omega_b)),
 *            omega <- R omega_b                          (R of the old q)
 *   q <- normalise(q + 1/2 q (x) (0, omega_b))           (omega_b = new body rate)
 *   X wrapped into [0, L) on periodic axes. */
static void integrate_particle(const oracle_sim* s, particle* P, const double F[3],
                               const double T[3]) {
  for (int a = 0; a < 3; ++a) {
    P->U[a] += F[a] / P->m;
    P->X[a] += P->U[a];
  }
  double R[9], wb[3];
  oracle_rotation(P->q, R);
  if (P->shape == ORACLE_SPHERE) {
    for (int a = 0; a < 3; ++a) P->W[a] += T[a] / P->I[a];
    for (int j = 0; j < 3; ++j) wb[j] = R[0 * 3 + j] * P->W[0] + R[1 * 3 + j] * P->W[1] + R[2 * 3 + j] * P->W[2];
  } else {
    double Tb[3], Lb[3], gyro[3];
    for (int j = 0; j < 3; ++j) {
      wb[j] = R[0 * 3 + j] * P->W[0] + R[1 * 3 + j] * P->W[1] + R[2 * 3 + j] * P->W[2];
      Tb[j] = R[0 * 3 + j] * T[0] + R[1 * 3 + j] * T[1] + R[2 * 3 + j] * T[2];
    }
    for (int j = 0; j < 3; ++j) Lb[j] = P->I[j] * wb[j];
    cross(wb, Lb, gyro);
    for (int j = 0; j < 3; ++j) wb[j] += (Tb[j] - gyro[j]) / P->I[j];
    for (int a = 0; a < 3; ++a) P->W[a] = R[a * 3 + 0] * wb[0] + R[a * 3 + 1] * wb[1] + R[a * 3 + 2] * wb[2];
  }
  /* dq/dt = 1/2 q (x) (0, omega_b) */
  double w = P->q[0], x = P->q[1], y = P->q[2], z = P->q[3];
  double dq[4];
  dq[0] = 0.5 * (-x * wb[0] - y * wb[1] - z * wb[2]);
  dq[1] = 0.5 * (w * wb[0] + y * wb[2] - z * wb[1]);
  dq[2] = 0.5 * (w * wb[1] + z * wb[0] - x * wb[2]);
  dq[3] = 0.5 * (w * wb[2] + x * wb[1] - y * wb[0]);
  double nq = 0.0;
  for (int j = 0; j < 4; ++j) {
    P->q[j] += dq[j];
    nq += P->q[j] * P->q[j];
  }
  nq = sqrt(nq);
  for (int j = 0; j < 4; ++j) P->q[j] /= nq;
  wrap_position(s, P->X);
}

void oracle_integrate_only(oracle_sim* s, const double* F, const double* T) {
  for (int p = 0; p < s->np; ++p) integrate_particle(s, &s->p[p], F + 3 * p, T + 3 * p);
}

/* ------------------------------------------------------------------------ */
/* Signed-distance grids (the paper's outlook on shapes beyond spheres, Sec.
 * 6, in the voxelised form).  Registration derives what the Newton-Euler
 * update and the coupling need from the samples alone:
 *   volume and second moments: midpoint rule over every grid cell split
 *     into 4 x 4 x 4 sub-cells, a sub-cell counting when the FP64 blend at
 *     its centre is negative;
 *   rc: the largest |corner| of the grid cells with a negative corner (the
 *     blend lies between the corner values, so the body is inside them);
 *   rinf: the same for corners below eps/2 (B of Eq. B is zero elsewhere). */
int oracle_add_grid(oracle_sim* s, int n0, int n1, int n2, double h, const float* values) {
  if (s->ngrid >= ORACLE_MAX_GRIDS || n0 < 2 || n1 < 2 || n2 < 2 || !(h > 0.0) || !values) return -1;
  const int n[3] = {n0, n1, n2};
  long nv = (long)n0 * n1 * n2;
  int neg = 0;
  for (long k = 0; k < nv; ++k) {
    if (!isfinite(values[k])) return -1;
    if (values[k] < 0.0f) neg = 1;
  }
  if (!neg) return -1;
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        int face = i == 0 || j == 0 || k == 0 || i == n0 - 1 || j == n1 - 1 || k == n2 - 1;
        if (face && !((double)values[((long)k * n1 + j) * n0 + i] >= s->eps / 2.0)) return -1;
      }
  grid_shape* g = (grid_shape*)calloc(1, sizeof(grid_shape));
  g->v = (float*)malloc(sizeof(float) * nv);
  memcpy(g->v, values, sizeof(float) * nv);
  for (int j = 0; j < 3; ++j) g->n[j] = n[j];
  g->h = h;
  /* radii from the cells' corners */
  double rc = 0.0, rinf = 0.0;
  for (int k = 0; k + 1 < n2; ++k)
    for (int j = 0; j + 1 < n1; ++j)
      for (int i = 0; i + 1 < n0; ++i) {
        double vmin = INFINITY, cmax = 0.0;
        for (int c = 0; c < 8; ++c) {
          int ii = i + (c & 1), jj = j + ((c >> 1) & 1), kk = k + (c >> 2);
          double v = values[((long)kk * n1 + jj) * n0 + ii];
          if (v < vmin) vmin = v;
          double x = (ii - 0.5 * (n0 - 1)) * h, y = (jj - 0.5 * (n1 - 1)) * h, z = (kk - 0.5 * (n2 - 1)) * h;
          double d = sqrt(x * x + y * y + z * z);
          if (d > cmax) cmax = d;
        }
        if (vmin < 0.0 && cmax > rc) rc = cmax;
        if (vmin < s->eps / 2.0 && cmax > rinf) rinf = cmax;
      }
  g->rc = rc;
  g->rinf = rinf;
  /* volume, centroid and second moments over 4^3 sub-cells per cell */
  const int sub = 4;
  double V = 0.0, c1[3] = {0.0, 0.0, 0.0}, S[3][3] = {{0.0}};
  const double dv = (h / sub) * (h / sub) * (h / sub);
  for (int k = 0; k + 1 < n2; ++k)
    for (int j = 0; j + 1 < n1; ++j)
      for (int i = 0; i + 1 < n0; ++i)
        for (int mz = 0; mz < sub; ++mz)
          for (int my = 0; my < sub; ++my)
            for (int mx = 0; mx < sub; ++mx) {
              double r[3] = {(i + (mx + 0.5) / sub - 0.5 * (n0 - 1)) * h, (j + (my + 0.5) / sub - 0.5 * (n1 - 1)) * h,
                             (k + (mz + 0.5) / sub - 0.5 * (n2 - 1)) * h};
              if (!(grid_value(g, r) < 0.0)) continue;
              V += dv;
              for (int a = 0; a < 3; ++a) {
                c1[a] += r[a] * dv;
                for (int b = 0; b < 3; ++b) S[a][b] += r[a] * r[b] * dv;
              }
            }
  g->V = V;
  g->I1[0] = S[1][1] + S[2][2];
  g->I1[1] = S[0][0] + S[2][2];
  g->I1[2] = S[0][0] + S[1][1];
  double imax = g->I1[0];
  if (g->I1[1] > imax) imax = g->I1[1];
  if (g->I1[2] > imax) imax = g->I1[2];
  int ok = V > 0.0;
  for (int a = 0; a < 3; ++a) ok = ok && fabs(c1[a] / V) <= h / 100.0;
  ok = ok && fabs(S[0][1]) <= 1e-3 * imax && fabs(S[0][2]) <= 1e-3 * imax && fabs(S[1][2]) <= 1e-3 * imax;
  if (!ok) {
    free(g->v);
    free(g);
    return -2;
  }
  s->grids[s->ngrid] = g;
  return s->ngrid++;
}

double oracle_grid_sdf(const oracle_sim* s, int grid, const double r_body[3]) {
  if (grid < 0 || grid >= s->ngrid) return NAN;
  return grid_value(s->grids[grid], r_body);
}

void oracle_grid_properties(const oracle_sim* s, int grid, double out[6]) {
  const grid_shape* g = s->grids[grid];
  out[0] = g->V;
  for (int j = 0; j < 3; ++j) out[1 + j] = g->I1[j];
  out[4] = g->rc;
  out[5] = g->rinf;
}

int oracle_inside_grid_fp32(const oracle_sim* s, int grid, const double q[4], const double X[3],
                            const int cell[3]) {
  return inside_grid_fp32(s->grids[grid], q, X, cell, s->n, s->bc);
}

/* ------------------------------------------------------------------------ */
/* Contact (an extension).  The paper lists contact treatment among the forces
 * on a particle (Sec. 2.2) and points to a published contact model for convex
 * shapes without stating it; its own runs have none (Sec. 3.2), and it names
 * the missing contact as the cause of the deviations at high solid fraction
 * (Sec. 5.3).  The reading used here is a short-range repulsion of the
 * quadratic-ramp kind used in resolved particle simulations:
 *   - every particle's contact body is a capsule enclosing it: the points
 *     within r_c of the segment X +- h_c e (sphere: r_c = a, h_c = 0;
 *     capsule: itself; ellipsoid: e along its longest semi-axis a_k,
 *     r_c = the larger of the two others, h_c = a_k - r_c; cuboid: e along
 *     its longest half-extent h_k, r_c = |(h_i, h_j)|, h_c = h_k);
 *   - two capsules whose segments come closest at points p_i, p_j (minimum
 *     image), with gap delta = |p_i - p_j| - r_i - r_j < zeta, push each
 *     other apart along n = (p_i - p_j) / |p_i - p_j| with the force
 *     k ((zeta - delta) / zeta)^2, applied at the contact surface, so that
 *     particle i receives the torque (p_i - X_i) x F_i;
 *   - a wall of axis a (at -1/2 or n_a - 1/2) pushes the capsule's nearest
 *     segment end the same way, with delta its distance to the wall minus r_c.
 * The forces of a pair are equal and opposite and act on one line. */
static void contact_capsule(const particle* P, double e[3], double* h, double* r) {
  double R[9];
  oracle_rotation(P->q, R);
  int k = 2;
  if (P->shape == ORACLE_SPHERE || P->shape == ORACLE_GRID) {
    *h = 0.0;
    *r = P->shape == ORACLE_GRID ? P->rc : P->a[0];
  } else if (P->shape == ORACLE_CAPSULE) {
    *h = P->a[2];
    *r = P->a[0];
  } else {
    k = 0;
    if (P->a[1] > P->a[k]) k = 1;
    if (P->a[2] > P->a[k]) k = 2;
    int i = (k + 1) % 3, j = (k + 2) % 3;
    if (P->shape == ORACLE_ELLIPSOID) {
      *r = P->a[i] > P->a[j] ? P->a[i] : P->a[j];
      *h = P->a[k] - *r;
    } else {
      *r = sqrt(P->a[i] * P->a[i] + P->a[j] * P->a[j]);
      *h = P->a[k];
    }
  }
  /* body axis k in world coordinates: column k of the rotation */
  for (int a = 0; a < 3; ++a) e[a] = R[a * 3 + k];
}

static double clamp(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* parameters s, t of the closest points P + s u and Q + t v of two segments,
 * |s| <= hu, |t| <= hv, u and v unit vectors, Qp the second segment's centre
 * (the classic method: the
 * closest points of the two lines, s clamped, t from s and clamped, s again
 * from t and clamped) */
static void segment_closest(const double P[3], const double u[3], double hu, const double Qp[3],
                            const double v[3], double hv, double* s, double* t) {
  double w[3], b = 0.0, d = 0.0, f = 0.0;
  for (int a = 0; a < 3; ++a) {
    w[a] = P[a] - Qp[a];
    b += u[a] * v[a];
    d += u[a] * w[a];
    f += v[a] * w[a];
  }
  double den = 1.0 - b * b;
  double ss = den > 1e-12 ? clamp((b * f - d) / den, -hu, hu) : 0.0;
  double tt = clamp(b * ss + f, -hv, hv);
  ss = clamp(b * tt - d, -hu, hu);
  *s = ss;
  *t = tt;
}

static double ramp_force(double k, double zeta, double gap) {
  double x = (zeta - gap) / zeta;
  return k * x * x;
}

int oracle_set_contact(oracle_sim* s, double k, double zeta) {
  if (!(k >= 0.0) || !(zeta > 0.0)) return -1;
  s->contact_k = k;
  s->contact_zeta = zeta;
  return 0;
}

void oracle_contact_forces(const oracle_sim* s, double* F, double* T) {
  for (int p = 0; p < 3 * s->np; ++p) F[p] = T[p] = 0.0;
  if (s->contact_k <= 0.0) return;
  const double k = s->contact_k, zeta = s->contact_zeta;
  for (int i = 0; i < s->np; ++i) {
    const particle* Pi = &s->p[i];
    double ei[3], hi, ri;
    contact_capsule(Pi, ei, &hi, &ri);
    /* walls */
    for (int a = 0; a < 3; ++a) {
      if (!is_wall(s, a)) continue;
      for (int side = 0; side < 2; ++side) {
        /* the segment end nearest to this wall */
        double dir = side == 0 ? -1.0 : 1.0;
        double t = ei[a] * dir > 0.0 ? hi : (ei[a] * dir < 0.0 ? -hi : 0.0);
        double pt[3];
        for (int c = 0; c < 3; ++c) pt[c] = Pi->X[c] + t * ei[c];
        double gap = (side == 0 ? pt[a] + 0.5 : (s->n[a] - 0.5) - pt[a]) - ri;
        if (gap >= zeta) continue;
        double f[3] = {0.0, 0.0, 0.0}, arm[3], tq[3];
        f[a] = -dir * ramp_force(k, zeta, gap);
        for (int c = 0; c < 3; ++c) arm[c] = pt[c] - Pi->X[c];
        cross(arm, f, tq);
        for (int c = 0; c < 3; ++c) {
          F[3 * i + c] += f[c];
          T[3 * i + c] += tq[c];
        }
      }
    }
    /* pairs i < j */
    for (int j = i + 1; j < s->np; ++j) {
      const particle* Pj = &s->p[j];
      double ej[3], hj, rj, Xj[3];
      contact_capsule(Pj, ej, &hj, &rj);
      for (int a = 0; a < 3; ++a) Xj[a] = Pi->X[a] + min_image(s, a, Pj->X[a] - Pi->X[a]);
      double si, tj;
      segment_closest(Pi->X, ei, hi, Xj, ej, hj, &si, &tj);
      double pi_[3], pj_[3], dv[3], dist = 0.0;
      for (int a = 0; a < 3; ++a) {
        pi_[a] = Pi->X[a] + si * ei[a];
        pj_[a] = Xj[a] + tj * ej[a];
        dv[a] = pi_[a] - pj_[a];
        dist += dv[a] * dv[a];
      }
      dist = sqrt(dist);
      double gap = dist - ri - rj;
      if (gap >= zeta || !(dist > 0.0)) continue;
      double fm = ramp_force(k, zeta, gap), f[3], ai[3], aj[3], ti[3], tj_[3], fn[3];
      for (int a = 0; a < 3; ++a) {
        f[a] = fm * dv[a] / dist;
        fn[a] = -f[a];
        ai[a] = pi_[a] - Pi->X[a];
        aj[a] = pj_[a] - Xj[a];
      }
      cross(ai, f, ti);
      cross(aj, fn, tj_);
      for (int a = 0; a < 3; ++a) {
        F[3 * i + a] += f[a];
        T[3 * i + a] += ti[a];
        F[3 * j + a] += fn[a];
        T[3 * j + a] += tj_[a];
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One time step in the order of Algorithm 1 (its communication rows have no
 * counterpart on one process). */
void oracle_step(oracle_sim* s, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    /* couple fluid to particles (MEA) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < s->np; ++p) oracle_mea(s, p, s->p[p].F, s->p[p].T);
    /* apply external forces: weight minus buoyancy, (rho_p - rho_f) V g
     * (Sec. 5.1 prints (rho_f - rho_p) V g with "accelerated in z"; the
     * reading is that heavier particles move along the gravity vector g),
     * and the contact forces when switched on (an extension, see above),
     * all taken at the state before this update */
    double* Fc = NULL;
    double* Tc = NULL;
    if (s->contact_k > 0.0 && s->np > 0) {
      Fc = (double*)malloc(sizeof(double) * 3 * s->np);
      Tc = (double*)malloc(sizeof(double) * 3 * s->np);
      oracle_contact_forces(s, Fc, Tc);
    }
    for (int p = 0; p < s->np; ++p) {
      particle* P = &s->p[p];
      double Ftot[3], Ttot[3];
      for (int a = 0; a < 3; ++a) {
        Ftot[a] = P->F[a] + (P->rho - 1.0) * P->V * s->g[a];
        Ttot[a] = P->T[a];
        if (Fc) {
          Ftot[a] += Fc[3 * p + a];
          Ttot[a] += Tc[3 * p + a];
        }
      }
      /* solve the equations of motion */
      integrate_particle(s, P, Ftot, Ttot);
    }
    free(Fc);
    free(Tc);
    /* couple particles to fluid (EDM), then collide and stream */
    oracle_indicator_field(s, s->B, s->pid);
    collide_into(s, s->B, s->pid, s->post);
    oracle_stream_only(s, s->post);
    s->steps++;
  }
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
