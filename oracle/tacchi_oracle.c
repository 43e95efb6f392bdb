/*
 * tacchi_oracle.c -- plain, slow FP64 CPU oracle of the Tacchi elastomer
 * simulation and tactile rendering (arXiv 2301.08343).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  It shares no code with the CUDA path.
 *
 * What it follows, step by step:
 *   - initialization, Sec. III-A "Initialization", Eq. 1: F = I, C = 0, v = 0;
 *     particles on a 2x2x2-per-cell lattice, optionally jittered by the
 *     counter-based splitmix64 generator (Steele, Lea & Flood 2014);
 *   - particle-to-grid, Eqs. 2-5 with quadratic B-spline weights;
 *   - grid velocity, Eq. 3 and Eq. 6, then the rigid indenter, the fixed base
 *     (Eq. 10, applied on grid nodes) and the padding band;
 *   - grid-to-particle, Eqs. 7-9, the base override of Eq. 10 and the
 *     advection of Eq. 11; the indenter pose advances by Eq. 11 too;
 *   - height map of the deformed top surface (Sec. III-B, "2D interpolation");
 *   - Phong shading, Eqs. 12-14.
 *
 * Readings where the paper is silent or garbled:
 *   - S_p of Eq. 5 is the fixed-corotated Kirchhoff stress
 *       tau = 2 mu (F - R) F^T + lambda J (J - 1) I,  R = polar factor of F;
 *   - Eq. 4 carries m_p on the affine term: w m_p (v_p + C_p (X_i - x_p));
 *   - Eq. 8 sums grid velocities: C_p = 4/dX^2 sum_i w_ip V_i (X_i - x_p)^T;
 *   - a node with M_i = 0 gets V_i = 0; gravity defaults to 0;
 *   - the indenter acts on grid nodes: a node inside it at the pose of the
 *     start of the substep takes the indenter's rigid velocity (no slip);
 *   - the inside/outside decision is taken in FP32 with a fixed operation
 *     order, the precision of the GPU kernel, so both sides decide alike;
 *   - nodes at or below the base plane, and the two outermost node layers,
 *     get V = 0; a particle whose stencil would touch that band is an error;
 *   - the surface height of a top-layer particle is the rest top plane plus
 *     its vertical displacement; the 2D interpolation is a z-max splat of
 *     radius dX/2 followed by nearest-covered-pixel hole filling.
 *
 * Polar decomposition: cyclic Jacobi eigen-decomposition of F^T F in FP64
 * (a different method from the GPU's Newton iteration), R = F (F^T F)^{-1/2}.
 */
#include "tacchi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct ora_sim {
  ora_params p;
  int G[3];
  long long nodes;
  long long N;
  double origin[3]; /* world position of grid node (0,0,0), m */
  double V0, m, mu, la;
  double z_top; /* world z of the rest top surface, m */
  double *xi;   /* [N][3] position in grid-cell units */
  double *v;    /* [N][3] */
  double *C;    /* [N][9] */
  double *F;    /* [N][9] */
  uint8_t *flags;
  double *rest_z; /* [N] rest z in cells */
  double *gm;     /* [nodes] M_i of the last P2G */
  double *gp;     /* [nodes][3] MG_i of the last P2G */
  double *gv;     /* [nodes][3] V_i after the grid update */
  int ind_kind;
  double ind_params[8];
  int hm_w, hm_h;
  double hm_pixel;
  float *hm;
  double pose[7], vel[6];
  /* indenter represented by particles (Eq. 10, p in I): local positions (m)
   * in the indenter frame and the mass of each; 0 points = grid boundary */
  long long ind_np;
  double *ind_pts;
  double ind_mass;
};

static int g_threads = 1;
void ora_set_threads(int n) { g_threads = n > 0 ? n : 1; }

/* ------------------------------------------------------------------ */
/* splitmix64 in counter form: output k is the mix of seed + (k+1)*gamma. */
uint64_t ora_splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Particle sampling (Sec. III-A, Initialization): 2x2x2 sub-cells per
 * elastomer cell, one particle per sub-cell at (sub + U) * dX/2, U uniform
 * in [0,1) from splitmix64 (or 1/2 without jitter).  Canonical order:
 * cell z, y, x, then sub z, y, x; three draws per particle (x, y, z). */
int ora_lattice(int nx, int ny, int nz, int pad_side, int pad_bottom,
                uint64_t seed, int jitter, float *u, uint8_t *flags) {
  long long N = 8ll * nx * ny * nz;
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx)
        for (int sz = 0; sz < 2; ++sz)
          for (int sy = 0; sy < 2; ++sy)
            for (int sx = 0; sx < 2; ++sx) {
              long long p = (((long long)cz * ny + cy) * nx + cx) * 8 + (sz * 4 + sy * 2 + sx);
              int cell[3] = {cx + pad_side, cy + pad_side, cz + pad_bottom};
              int sub[3] = {sx, sy, sz};
              for (int a = 0; a < 3; ++a) {
                double U = 0.5;
                if (jitter) {
                  uint64_t r = ora_splitmix64_at(seed, (uint64_t)(3 * p + a));
                  U = (double)(r >> 11) * (1.0 / 9007199254740992.0);
                }
                double t = ((double)sub[a] + U) * 0.5;
                double pos = (double)cell[a] + t;
                u[a * N + p] = (float)pos;
              }
              uint8_t f = 0;
              if (cz == 0) f |= 1;                 /* base layer, Eq. 10 set B */
              if (cz == nz - 1 && sz == 1) f |= 2; /* top particle layer */
              flags[p] = f;
            }
  return 0;
}

/* ------------------------------------------------------------------ */
ora_sim *ora_create(const ora_params *p) {
  ora_sim *s = (ora_sim *)calloc(1, sizeof(ora_sim));
  s->p = *p;
  s->G[0] = p->nx + 2 * p->pad_side + 1;
  s->G[1] = p->ny + 2 * p->pad_side + 1;
  s->G[2] = p->nz + p->pad_bottom + p->pad_top + 1;
  s->nodes = (long long)s->G[0] * s->G[1] * s->G[2];
  s->N = 8ll * p->nx * p->ny * p->nz;
  s->origin[0] = -p->pad_side * p->dx;
  s->origin[1] = -p->pad_side * p->dx;
  s->origin[2] = -p->pad_bottom * p->dx;
  s->z_top = p->nz * p->dx;
  s->V0 = p->dx * p->dx * p->dx / 8.0;        /* initial particle volume V_p^0 */
  s->m = p->rho * s->V0;                       /* particle mass m_p */
  s->mu = p->E / (2.0 * (1.0 + p->nu));        /* Lame parameters from E, nu */
  s->la = p->E * p->nu / ((1.0 + p->nu) * (1.0 - 2.0 * p->nu));
  s->xi = (double *)calloc(3 * s->N, sizeof(double));
  s->v = (double *)calloc(3 * s->N, sizeof(double));
  s->C = (double *)calloc(9 * s->N, sizeof(double));
  s->F = (double *)calloc(9 * s->N, sizeof(double));
  s->flags = (uint8_t *)calloc(s->N, 1);
  s->rest_z = (double *)calloc(s->N, sizeof(double));
  s->gm = (double *)calloc(s->nodes, sizeof(double));
  s->gp = (double *)calloc(3 * s->nodes, sizeof(double));
  s->gv = (double *)calloc(3 * s->nodes, sizeof(double));
  for (long long q = 0; q < s->N; ++q) {
    s->F[9 * q + 0] = s->F[9 * q + 4] = s->F[9 * q + 8] = 1.0; /* Eq. 1: F = I */
  }
  s->pose[3] = 1.0;
  return s;
}

void ora_destroy(ora_sim *s) {
  if (!s) return;
  free(s->xi); free(s->v); free(s->C); free(s->F); free(s->flags);
  free(s->rest_z); free(s->gm); free(s->gp); free(s->gv); free(s->hm);
  free(s->ind_pts);
  free(s);
}

long long ora_num_particles(const ora_sim *s) { return s->N; }
void ora_grid_dims(const ora_sim *s, int dims[3]) {
  dims[0] = s->G[0]; dims[1] = s->G[1]; dims[2] = s->G[2];
}

void ora_set_state(ora_sim *s, const float *u, const float *v, const float *C,
                   const float *Fm, const uint8_t *flags) {
  long long N = s->N;
  for (long long q = 0; q < N; ++q) {
    for (int a = 0; a < 3; ++a) {
      s->xi[3 * q + a] = (double)u[a * N + q];
      s->v[3 * q + a] = v ? (double)v[a * N + q] : 0.0;
    }
    for (int e = 0; e < 9; ++e) {
      s->C[9 * q + e] = C ? (double)C[e * N + q] : 0.0;
      double id = (e == 0 || e == 4 || e == 8) ? 1.0 : 0.0;
      s->F[9 * q + e] = id + (Fm ? (double)Fm[e * N + q] : 0.0);
    }
    if (flags) s->flags[q] = flags[q];
  }
}

void ora_set_rest(ora_sim *s, const float *u0) {
  for (long long q = 0; q < s->N; ++q) s->rest_z[q] = (double)u0[2 * s->N + q];
}

void ora_get_state(const ora_sim *s, double *xi, double *v, double *C, double *F) {
  long long N = s->N;
  for (long long q = 0; q < N; ++q) {
    for (int a = 0; a < 3; ++a) {
      if (xi) xi[a * N + q] = s->xi[3 * q + a];
      if (v) v[a * N + q] = s->v[3 * q + a];
    }
    for (int e = 0; e < 9; ++e) {
      if (C) C[e * N + q] = s->C[9 * q + e];
      if (F) F[e * N + q] = s->F[9 * q + e];
    }
  }
}

void ora_get_state_f32(const ora_sim *s, float *u, float *v, float *C, float *Fm) {
  long long N = s->N;
  for (long long q = 0; q < N; ++q) {
    for (int a = 0; a < 3; ++a) {
      if (u) u[a * N + q] = (float)s->xi[3 * q + a];
      if (v) v[a * N + q] = (float)s->v[3 * q + a];
    }
    for (int e = 0; e < 9; ++e) {
      double id = (e == 0 || e == 4 || e == 8) ? 1.0 : 0.0;
      if (C) C[e * N + q] = (float)s->C[9 * q + e];
      if (Fm) Fm[e * N + q] = (float)(s->F[9 * q + e] - id);
    }
  }
}

/* ------------------------------------------------------------------ */
/* Quadratic B-spline weights (Sec. III-A, particle-to-grid; [CJ16]).
 * For each axis the stencil starts at base = floor(xi - 1/2) and the
 * particle sits at fraction f = xi - base in [1/2, 3/2) from it. */
void ora_weights(const double xi[3], int base[3], double w[27]) {
  double wa[3][3];
  for (int a = 0; a < 3; ++a) {
    base[a] = (int)floor(xi[a] - 0.5);
    double f = xi[a] - (double)base[a];
    wa[a][0] = 0.5 * (1.5 - f) * (1.5 - f);
    wa[a][1] = 0.75 - (f - 1.0) * (f - 1.0);
    wa[a][2] = 0.5 * (f - 0.5) * (f - 0.5);
  }
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) w[(k * 3 + j) * 3 + i] = wa[0][i] * wa[1][j] * wa[2][k];
}

/* ------------------------------------------------------------------ */
/* 3x3 helpers, row-major. */
static void mat_mul(const double *A, const double *B, double *Cm) {
  double t[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += A[r * 3 + k] * B[k * 3 + c];
      t[r * 3 + c] = acc;
    }
  memcpy(Cm, t, sizeof(t));
}
static void mat_transpose(const double *A, double *T) {
  double t[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) t[c * 3 + r] = A[r * 3 + c];
  memcpy(T, t, sizeof(t));
}
static double mat_det(const double *A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* Symmetric eigen-decomposition A = Q diag(lam) Q^T by cyclic Jacobi
 * rotations (FP64). */
static void sym_eig3(const double *Ain, double lam[3], double Q[9]) {
  double A[9];
  memcpy(A, Ain, sizeof(A));
  for (int e = 0; e < 9; ++e) Q[e] = (e == 0 || e == 4 || e == 8) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-40 * diag || off == 0.0) break;
    for (int pq = 0; pq < 3; ++pq) {
      int p = pq == 2 ? 1 : 0;
      int q = pq == 0 ? 1 : 2;
      double apq = A[p * 3 + q];
      if (apq == 0.0) continue;
      double app = A[p * 3 + p], aqq = A[q * 3 + q];
      double theta = (aqq - app) / (2.0 * apq);
      double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
      /* A <- J^T A J with J the rotation in the (p,q) plane */
      for (int k = 0; k < 3; ++k) {
        double akp = A[k * 3 + p], akq = A[k * 3 + q];
        A[k * 3 + p] = c * akp - sn * akq;
        A[k * 3 + q] = sn * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        double apk = A[p * 3 + k], aqk = A[q * 3 + k];
        A[p * 3 + k] = c * apk - sn * aqk;
        A[q * 3 + k] = sn * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        double qkp = Q[k * 3 + p], qkq = Q[k * 3 + q];
        Q[k * 3 + p] = c * qkp - sn * qkq;
        Q[k * 3 + q] = sn * qkp + c * qkq;
      }
    }
  }
  lam[0] = A[0]; lam[1] = A[4]; lam[2] = A[8];
}

/* Polar decomposition F = R S: S = (F^T F)^{1/2}, R = F S^{-1}. */
void ora_polar(const double F[9], double R[9]) {
  double Ft[9], FtF[9], lam[3], Q[9], Sinv[9];
  mat_transpose(F, Ft);
  mat_mul(Ft, F, FtF);
  sym_eig3(FtF, lam, Q);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += Q[r * 3 + k] * Q[c * 3 + k] / sqrt(lam[k]);
      Sinv[r * 3 + c] = acc;
    }
  mat_mul(F, Sinv, R);
}

/* Elasticity term S_p of Eq. 5 (reading: fixed-corotated Kirchhoff stress).
 * tau = 2 mu (F - R) F^T + lambda J (J - 1) I. */
void ora_stress(const double F[9], double mu, double la, double tau[9]) {
  double R[9], D[9], Ft[9];
  ora_polar(F, R);
  for (int e = 0; e < 9; ++e) D[e] = F[e] - R[e];
  mat_transpose(F, Ft);
  mat_mul(D, Ft, tau);
  double J = mat_det(F);
  for (int e = 0; e < 9; ++e) tau[e] *= 2.0 * mu;
  for (int a = 0; a < 3; ++a) tau[a * 4] += la * J * (J - 1.0);
}

/* ------------------------------------------------------------------ */
/* Rigid indenter.  Pose = position (m) + unit quaternion (w,x,y,z) mapping
 * the indenter's local frame to the world. */
typedef struct {
  float c[3];  /* centre in cells */
  float r[9];  /* local->world rotation, row-major */
  float s0, s1, s2, s3; /* shape constants in cells */
  float inv_pix, offx, offy; /* height map sampling */
} frame32;

static void quat_to_mat(const double q_in[4], double Rm[9]) {
  double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
  Rm[0] = 1.0 - 2.0 * (y * y + z * z); Rm[1] = 2.0 * (x * y - w * z);       Rm[2] = 2.0 * (x * z + w * y);
  Rm[3] = 2.0 * (x * y + w * z);       Rm[4] = 1.0 - 2.0 * (x * x + z * z); Rm[5] = 2.0 * (y * z - w * x);
  Rm[6] = 2.0 * (x * z - w * y);       Rm[7] = 2.0 * (y * z + w * x);       Rm[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* FP32 constants of the inside test, rounded from the FP64 pose. */
static void make_frame32(const ora_sim *s, frame32 *f) {
  double dx = s->p.dx, Rm[9];
  for (int a = 0; a < 3; ++a) f->c[a] = (float)((s->pose[a] - s->origin[a]) / dx);
  quat_to_mat(s->pose + 3, Rm);
  for (int e = 0; e < 9; ++e) f->r[e] = (float)Rm[e];
  const double *P = s->ind_params;
  f->s0 = f->s1 = f->s2 = f->s3 = 0.f;
  f->inv_pix = f->offx = f->offy = 0.f;
  switch (s->ind_kind) {
    case ORA_IND_SPHERE: /* params: radius */
      f->s0 = (float)((P[0] / dx) * (P[0] / dx));
      break;
    case ORA_IND_CYLINDER: /* params: radius, half length (axis = local x) */
      f->s0 = (float)((P[0] / dx) * (P[0] / dx));
      f->s1 = (float)(P[1] / dx);
      break;
    case ORA_IND_CONE: /* params: half angle (rad), height; apex at origin, axis +z */
      f->s0 = (float)tan(P[0]);
      f->s1 = (float)(P[1] / dx);
      break;
    case ORA_IND_PRISM: /* params: half angle, half length (local y), height */
      f->s0 = (float)tan(P[0]);
      f->s1 = (float)(P[1] / dx);
      f->s2 = (float)(P[2] / dx);
      break;
    case ORA_IND_HEIGHTMAP: /* params: cap thickness above the back plane */
      f->s0 = (float)(P[0] / dx);
      f->inv_pix = (float)(dx / s->hm_pixel);
      f->offx = (float)(s->hm_w * 0.5 - 0.5);
      f->offy = (float)(s->hm_h * 0.5 - 0.5);
      break;
    default:
      break;
  }
}

/* Inside test of node (i,j,k) in FP32 with a fixed operation order (the
 * file is compiled without floating-point contraction). */
static int inside32(const ora_sim *s, const frame32 *f, int i, int j, int k) {
  if (s->ind_kind == ORA_IND_NONE) return 0;
  float d0 = (float)i - f->c[0];
  float d1 = (float)j - f->c[1];
  float d2 = (float)k - f->c[2];
  if (s->ind_kind == ORA_IND_SPHERE) {
    float a = d0 * d0;
    float b = d1 * d1;
    float c = d2 * d2;
    float r2 = (a + b) + c;
    return r2 <= f->s0;
  }
  /* local = R^T (X - c) */
  float l0 = ((f->r[0] * d0) + (f->r[3] * d1)) + (f->r[6] * d2);
  float l1 = ((f->r[1] * d0) + (f->r[4] * d1)) + (f->r[7] * d2);
  float l2 = ((f->r[2] * d0) + (f->r[5] * d1)) + (f->r[8] * d2);
  switch (s->ind_kind) {
    case ORA_IND_CYLINDER: {
      float a = l1 * l1;
      float b = l2 * l2;
      return fabsf(l0) <= f->s1 && (a + b) <= f->s0;
    }
    case ORA_IND_CONE: {
      if (!(l2 >= 0.f && l2 <= f->s1)) return 0;
      float a = l0 * l0;
      float b = l1 * l1;
      float tz = f->s0 * l2;
      return (a + b) <= tz * tz;
    }
    case ORA_IND_PRISM: {
      if (!(fabsf(l1) <= f->s1 && l2 >= 0.f && l2 <= f->s2)) return 0;
      return fabsf(l0) <= f->s0 * l2;
    }
    case ORA_IND_HEIGHTMAP: {
      int w = s->hm_w, h = s->hm_h;
      float fx = (l0 * f->inv_pix) + f->offx;
      float fy = (l1 * f->inv_pix) + f->offy;
      if (fx < -0.5f || fx > (float)w - 0.5f || fy < -0.5f || fy > (float)h - 0.5f) return 0;
      float cx = fx < 0.f ? 0.f : (fx > (float)(w - 1) ? (float)(w - 1) : fx);
      float cy = fy < 0.f ? 0.f : (fy > (float)(h - 1) ? (float)(h - 1) : fy);
      int ix = (int)floorf(cx);
      int iy = (int)floorf(cy);
      if (ix > w - 2) ix = w - 2;
      if (iy > h - 2) iy = h - 2;
      float tx = cx - (float)ix;
      float ty = cy - (float)iy;
      const float *H = s->hm;
      float ux = 1.0f - tx, uy = 1.0f - ty;
      float a0 = H[iy * w + ix] * ux;
      float a1 = H[iy * w + ix + 1] * tx;
      float r0 = a0 + a1;
      float b0 = H[(iy + 1) * w + ix] * ux;
      float b1 = H[(iy + 1) * w + ix + 1] * tx;
      float r1 = b0 + b1;
      float hh = (r0 * uy) + (r1 * ty);
      return l2 >= -hh && l2 <= f->s0;
    }
    default:
      return 0;
  }
}

int ora_set_indenter(ora_sim *s, int kind, const double *params, int hm_w,
                     int hm_h, double hm_pixel_m, const float *hm,
                     const double pose[7], const double vel[6]) {
  if (kind < 0 || kind > ORA_IND_HEIGHTMAP) return -1;
  s->ind_kind = kind;
  for (int e = 0; e < 8; ++e) s->ind_params[e] = params ? params[e] : 0.0;
  free(s->hm);
  s->hm = NULL;
  s->hm_w = s->hm_h = 0;
  if (kind == ORA_IND_HEIGHTMAP) {
    if (hm_w < 2 || hm_h < 2 || !hm || !(hm_pixel_m > 0)) return -1;
    s->hm_w = hm_w; s->hm_h = hm_h; s->hm_pixel = hm_pixel_m;
    s->hm = (float *)malloc(sizeof(float) * hm_w * hm_h);
    for (int e = 0; e < hm_w * hm_h; ++e) s->hm[e] = (float)((double)hm[e] / s->p.dx);
  }
  for (int e = 0; e < 7; ++e) s->pose[e] = pose[e];
  for (int e = 0; e < 6; ++e) s->vel[e] = vel ? vel[e] : 0.0;
  return 0;
}

/* Represent the indenter by n particles at local positions pts (m, [n][3],
 * in the frame the pose maps to the world), each of the given mass: Eq. 10
 * gives them the indenter's velocity, and Sec. III-C initialises them from a
 * point cloud of the object.  n = 0 restores the grid-boundary indenter. */
int ora_set_indenter_particles(ora_sim *s, long long n, const double *pts, double mass) {
  if (n < 0 || (n > 0 && (!pts || !(mass > 0.0)))) return -1;
  free(s->ind_pts);
  s->ind_pts = NULL;
  s->ind_np = 0;
  s->ind_mass = 0.0;
  if (n == 0) return 0;
  s->ind_pts = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  memcpy(s->ind_pts, pts, sizeof(double) * 3 * (size_t)n);
  s->ind_np = n;
  s->ind_mass = mass;
  return 0;
}

void ora_get_pose(const ora_sim *s, double pose[7]) {
  for (int e = 0; e < 7; ++e) pose[e] = s->pose[e];
}

int ora_node_inside(const ora_sim *s, int i, int j, int k) {
  frame32 f;
  make_frame32(s, &f);
  return inside32(s, &f, i, j, k);
}

/* Rigid motion of the indenter over one substep (Eq. 11 applied to the
 * indenter): position += dt v; orientation rotated by the angle |w| dt. */
static void advance_pose(ora_sim *s, double dt) {
  for (int a = 0; a < 3; ++a) s->pose[a] += dt * s->vel[a];
  double wx = s->vel[3], wy = s->vel[4], wz = s->vel[5];
  double wn = sqrt(wx * wx + wy * wy + wz * wz);
  if (wn > 0.0) {
    double half = 0.5 * wn * dt;
    double cw = cos(half), sw = sin(half) / wn;
    double r[4] = {cw, sw * wx, sw * wy, sw * wz};
    double *q = s->pose + 3;
    double nq[4];
    nq[0] = r[0] * q[0] - r[1] * q[1] - r[2] * q[2] - r[3] * q[3];
    nq[1] = r[0] * q[1] + r[1] * q[0] + r[2] * q[3] - r[3] * q[2];
    nq[2] = r[0] * q[2] - r[1] * q[3] + r[2] * q[0] + r[3] * q[1];
    nq[3] = r[0] * q[3] + r[1] * q[2] - r[2] * q[1] + r[3] * q[0];
    double n = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int e = 0; e < 4; ++e) q[e] = nq[e] / n;
  }
}

/* ------------------------------------------------------------------ */
static long long node_index(const ora_sim *s, int i, int j, int k) {
  return ((long long)k * s->G[1] + j) * s->G[0] + i;
}

/* Particle-to-grid, Eqs. 2-5.  M_i = sum_p w_ip m_p;
 * MM_i = sum_p w_ip m_p (v_p + C_p (X_i - x_p));
 * ME_i = -dt sum_p (4/dX^2) w_ip V_p^0 S_p (X_i - x_p);  MG_i = MM_i + ME_i. */
static void p2g_into(ora_sim *s, double dt, double *mass, double *mom) {
  long long nodes = s->nodes, N = s->N;
  double dx = s->p.dx, Dinv = 4.0 / (dx * dx);
  int nt = g_threads;
  double *priv = (double *)calloc((size_t)nt * 4 * nodes, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double *pm = priv + (size_t)t * 4 * nodes;
#pragma omp for schedule(static)
    for (long long q = 0; q < N; ++q) {
      int base[3];
      double w[27], tau[9];
      const double *xi = s->xi + 3 * q;
      ora_weights(xi, base, w);
      ora_stress(s->F + 9 * q, s->mu, s->la, tau);
      const double *vp = s->v + 3 * q, *Cp = s->C + 9 * q;
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j)
          for (int i = 0; i < 3; ++i) {
            int I = base[0] + i, J = base[1] + j, K = base[2] + k;
            if (I < 0 || J < 0 || K < 0 || I >= s->G[0] || J >= s->G[1] || K >= s->G[2]) continue;
            double wip = w[(k * 3 + j) * 3 + i];
            double dpos[3] = {((double)I - xi[0]) * dx, ((double)J - xi[1]) * dx, ((double)K - xi[2]) * dx};
            long long n = node_index(s, I, J, K);
            pm[4 * n + 0] += wip * s->m; /* Eq. 2 */
            for (int a = 0; a < 3; ++a) {
              double Cd = Cp[a * 3 + 0] * dpos[0] + Cp[a * 3 + 1] * dpos[1] + Cp[a * 3 + 2] * dpos[2];
              double Sd = tau[a * 3 + 0] * dpos[0] + tau[a * 3 + 1] * dpos[1] + tau[a * 3 + 2] * dpos[2];
              double MM = wip * s->m * (vp[a] + Cd);      /* Eq. 4 */
              double ME = -dt * Dinv * wip * s->V0 * Sd;  /* Eq. 5 */
              pm[4 * n + 1 + a] += MM + ME;               /* Eq. 3 */
            }
          }
    }
  }
  /* Indenter particles (Eq. 10, p in I), at the pose of the start of the
   * substep: world position x = c + R l, the rigid velocity v = v_c +
   * w x (x - c), whose gradient C = skew(w) is the affine velocity of Eq. 4;
   * they carry no elastic stress (rigid), so Eq. 5 adds nothing for them. */
  if (s->ind_np > 0) {
    double Rm[9];
    quat_to_mat(s->pose + 3, Rm);
    const double *w = s->vel + 3;
    const double Cw[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    double *pm = priv; /* serial: the first thread's private grid */
    for (long long q = 0; q < s->ind_np; ++q) {
      const double *l = s->ind_pts + 3 * q;
      double x[3], r[3], v[3], xi[3];
      for (int a = 0; a < 3; ++a) {
        r[a] = Rm[a * 3 + 0] * l[0] + Rm[a * 3 + 1] * l[1] + Rm[a * 3 + 2] * l[2];
        x[a] = s->pose[a] + r[a];
        xi[a] = (x[a] - s->origin[a]) / dx;
      }
      v[0] = s->vel[0] + (w[1] * r[2] - w[2] * r[1]);
      v[1] = s->vel[1] + (w[2] * r[0] - w[0] * r[2]);
      v[2] = s->vel[2] + (w[0] * r[1] - w[1] * r[0]);
      int base[3];
      double wt[27];
      ora_weights(xi, base, wt);
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j)
          for (int i = 0; i < 3; ++i) {
            int I = base[0] + i, J = base[1] + j, K = base[2] + k;
            if (I < 0 || J < 0 || K < 0 || I >= s->G[0] || J >= s->G[1] || K >= s->G[2]) continue;
            double wip = wt[(k * 3 + j) * 3 + i];
            double dpos[3] = {((double)I - xi[0]) * dx, ((double)J - xi[1]) * dx, ((double)K - xi[2]) * dx};
            long long n = node_index(s, I, J, K);
            pm[4 * n + 0] += wip * s->ind_mass; /* Eq. 2 */
            for (int a = 0; a < 3; ++a) {
              double Cd = Cw[a * 3 + 0] * dpos[0] + Cw[a * 3 + 1] * dpos[1] + Cw[a * 3 + 2] * dpos[2];
              pm[4 * n + 1 + a] += wip * s->ind_mass * (v[a] + Cd); /* Eqs. 3-4 */
            }
          }
    }
  }
  for (long long n = 0; n < nodes; ++n) {
    double acc[4] = {0, 0, 0, 0};
    for (int t = 0; t < nt; ++t)
      for (int c = 0; c < 4; ++c) acc[c] += priv[(size_t)t * 4 * nodes + 4 * n + c];
    mass[n] = acc[0];
    for (int a = 0; a < 3; ++a) mom[a * nodes + n] = acc[1 + a];
  }
  free(priv);
}

void ora_p2g(ora_sim *s, double dt, double *mass, double *mom) { p2g_into(s, dt, mass, mom); }

/* Outward unit normal of the grid-boundary indenter's surface at node
 * (i, j, k), in FP64, for the slip contact mode (the paper's indenter is
 * no-slip, Eq. 10; slip removes only the relative velocity into it).
 * Sphere: radial from the centre.  Cylinder (axis local x): radial from the
 * axis.  Cone (apex at the pose, opening to local +z, half angle a) and prism
 * (edge along local y, faces at x_l = +-tan(a) z_l): the lateral face,
 * (rho_hat, -tan a) / sqrt(1 + tan^2 a).  Height map (surface z_l = -h):
 * (-dh/dx_l, -dh/dy_l, -1) / |.| from the bilinear interpolant.  Undefined
 * cases (a node on an axis or edge) take the local -z direction. */
static void indenter_normal(const ora_sim *s, int i, int j, int k, double n[3]) {
  double Rm[9], d[3], m[3] = {0.0, 0.0, -1.0};
  quat_to_mat(s->pose + 3, Rm);
  double X[3] = {s->origin[0] + i * s->p.dx, s->origin[1] + j * s->p.dx, s->origin[2] + k * s->p.dx};
  for (int a = 0; a < 3; ++a) d[a] = X[a] - s->pose[a];
  if (s->ind_kind == ORA_IND_SPHERE) {
    double q = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (q > 0.0) {
      for (int a = 0; a < 3; ++a) n[a] = d[a] / q;
      return;
    }
  } else {
    double l[3];
    for (int b = 0; b < 3; ++b) l[b] = Rm[0 * 3 + b] * d[0] + Rm[1 * 3 + b] * d[1] + Rm[2 * 3 + b] * d[2];
    const double *P = s->ind_params;
    if (s->ind_kind == ORA_IND_CYLINDER) {
      double q = sqrt(l[1] * l[1] + l[2] * l[2]);
      if (q > 0.0) { m[0] = 0.0; m[1] = l[1] / q; m[2] = l[2] / q; }
    } else if (s->ind_kind == ORA_IND_CONE) {
      double t = tan(P[0]), q = sqrt(l[0] * l[0] + l[1] * l[1]), c = 1.0 / sqrt(1.0 + t * t);
      if (q > 0.0) { m[0] = l[0] / q * c; m[1] = l[1] / q * c; m[2] = -t * c; }
    } else if (s->ind_kind == ORA_IND_PRISM) {
      double t = tan(P[0]), c = 1.0 / sqrt(1.0 + t * t);
      if (l[0] != 0.0) { m[0] = (l[0] > 0.0 ? 1.0 : -1.0) * c; m[1] = 0.0; m[2] = -t * c; }
    } else if (s->ind_kind == ORA_IND_HEIGHTMAP) {
      int w = s->hm_w, h = s->hm_h;
      double fx = l[0] / s->hm_pixel + (w * 0.5 - 0.5), fy = l[1] / s->hm_pixel + (h * 0.5 - 0.5);
      double cx = fx < 0.0 ? 0.0 : (fx > w - 1.0 ? w - 1.0 : fx);
      double cy = fy < 0.0 ? 0.0 : (fy > h - 1.0 ? h - 1.0 : fy);
      int ix = (int)floor(cx), iy = (int)floor(cy);
      if (ix > w - 2) ix = w - 2;
      if (iy > h - 2) iy = h - 2;
      double tx = cx - ix, ty = cy - iy;
      const float *H = s->hm; /* cells */
      double h00 = H[iy * w + ix], h01 = H[iy * w + ix + 1], h10 = H[(iy + 1) * w + ix], h11 = H[(iy + 1) * w + ix + 1];
      /* slope: cells of height per pixel, times dX / pixel */
      double sc = s->p.dx / s->hm_pixel;
      double gx = (fx > 0.0 && fx < w - 1.0) ? ((h01 - h00) * (1.0 - ty) + (h11 - h10) * ty) * sc : 0.0;
      double gy = (fy > 0.0 && fy < h - 1.0) ? ((h10 - h00) * (1.0 - tx) + (h11 - h01) * tx) * sc : 0.0;
      double c = 1.0 / sqrt(1.0 + gx * gx + gy * gy);
      m[0] = -gx * c; m[1] = -gy * c; m[2] = -c;
    }
  }
  for (int a = 0; a < 3; ++a) n[a] = Rm[a * 3 + 0] * m[0] + Rm[a * 3 + 1] * m[1] + Rm[a * 3 + 2] * m[2];
}

/* Grid velocity, Eq. 6, then the boundary conditions (indenter, Eq. 10 on
 * the base nodes, padding band). */
static void grid_update(ora_sim *s, double dt) {
  frame32 f;
  make_frame32(s, &f);
  long long nodes = s->nodes;
  double dx = s->p.dx;
  int base_k = s->p.pad_bottom; /* node layer of the base plane z = 0 */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long long n = 0; n < nodes; ++n) {
    int i = (int)(n % s->G[0]);
    int j = (int)((n / s->G[0]) % s->G[1]);
    int k = (int)(n / ((long long)s->G[0] * s->G[1]));
    double V[3] = {0, 0, 0};
    double M = s->gm[n];
    if (M > 0.0)
      for (int a = 0; a < 3; ++a) V[a] = s->gp[a * nodes + n] / M + dt * s->p.gravity[a];
    if (s->ind_np == 0 && inside32(s, &f, i, j, k)) {
      double X[3] = {s->origin[0] + i * dx, s->origin[1] + j * dx, s->origin[2] + k * dx};
      double r[3] = {X[0] - s->pose[0], X[1] - s->pose[1], X[2] - s->pose[2]};
      const double *w = s->vel + 3;
      double W[3] = {s->vel[0] + (w[1] * r[2] - w[2] * r[1]), s->vel[1] + (w[2] * r[0] - w[0] * r[2]),
                     s->vel[2] + (w[0] * r[1] - w[1] * r[0])};
      if (s->p.slip && M > 0.0) {
        /* slip: remove only the velocity into the indenter, relative to it */
        double nrm[3];
        indenter_normal(s, i, j, k, nrm);
        double q[3] = {V[0] - W[0], V[1] - W[1], V[2] - W[2]};
        double vn = q[0] * nrm[0] + q[1] * nrm[1] + q[2] * nrm[2];
        if (vn < 0.0)
          for (int a = 0; a < 3; ++a) V[a] = W[a] + (q[a] - vn * nrm[a]);
      } else { /* sticky (Eq. 10's rigid indenter), or an empty node */
        for (int a = 0; a < 3; ++a) V[a] = W[a];
      }
    }
    if (s->p.fix_base && k <= base_k) V[0] = V[1] = V[2] = 0.0;
    if (i < 2 || j < 2 || k < 2 || i > s->G[0] - 3 || j > s->G[1] - 3 || k > s->G[2] - 3)
      V[0] = V[1] = V[2] = 0.0;
    for (int a = 0; a < 3; ++a) s->gv[3 * n + a] = V[a];
  }
}

/* Grid-to-particle and advection, Eqs. 7-11. */
static int g2p(ora_sim *s, double dt) {
  long long N = s->N;
  double dx = s->p.dx, Dinv = 4.0 / (dx * dx);
  int err = 0;
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(| : err)
  for (long long q = 0; q < N; ++q) {
    int base[3];
    double w[27];
    double *xi = s->xi + 3 * q;
    ora_weights(xi, base, w);
    double vn[3] = {0, 0, 0}, Cn[9] = {0};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          int I = base[0] + i, J = base[1] + j, K = base[2] + k;
          if (I < 0 || J < 0 || K < 0 || I >= s->G[0] || J >= s->G[1] || K >= s->G[2]) continue;
          double wip = w[(k * 3 + j) * 3 + i];
          double dpos[3] = {((double)I - xi[0]) * dx, ((double)J - xi[1]) * dx, ((double)K - xi[2]) * dx};
          const double *V = s->gv + 3 * node_index(s, I, J, K);
          for (int a = 0; a < 3; ++a) {
            vn[a] += wip * V[a]; /* Eq. 7 */
            for (int b = 0; b < 3; ++b) Cn[a * 3 + b] += Dinv * wip * V[a] * dpos[b]; /* Eq. 8 */
          }
        }
    /* Eq. 9: F <- (I + dt C) F */
    double Fo[9], Mx[9];
    memcpy(Fo, s->F + 9 * q, sizeof(Fo));
    for (int e = 0; e < 9; ++e) Mx[e] = ((e == 0 || e == 4 || e == 8) ? 1.0 : 0.0) + dt * Cn[e];
    mat_mul(Mx, Fo, s->F + 9 * q);
    memcpy(s->C + 9 * q, Cn, sizeof(Cn));
    if (s->p.fix_base && (s->flags[q] & 1)) vn[0] = vn[1] = vn[2] = 0.0; /* Eq. 10 */
    for (int a = 0; a < 3; ++a) {
      s->v[3 * q + a] = vn[a];
      xi[a] += dt * vn[a] / dx; /* Eq. 11, in cell units */
    }
    for (int a = 0; a < 3; ++a) {
      int b = (int)floor(xi[a] - 0.5);
      if (b < 2 || b > s->G[a] - 5) err |= ORA_ERR_OUT_OF_GRID;
      if (!(xi[a] == xi[a])) err |= ORA_ERR_NUMERICAL;
    }
    double J = mat_det(s->F + 9 * q);
    if (!(J > 0.0)) err |= ORA_ERR_NUMERICAL;
  }
  return err;
}

int ora_substep(ora_sim *s, double dt) {
  p2g_into(s, dt, s->gm, s->gp);
  grid_update(s, dt);
  int err = g2p(s, dt);
  advance_pose(s, dt);
  return err;
}

int ora_run(ora_sim *s, int n, double dt) {
  int err = 0;
  for (int k = 0; k < n; ++k) err |= ora_substep(s, dt);
  return err;
}

/* Grid-to-particle step alone (Eqs. 7-11) from a given grid velocity V
 * ([3][nodes], x fastest): the same g2p() that ends ora_substep, without
 * P2G, grid update or the pose advance.  For tests that prescribe V. */
int ora_g2p(ora_sim *s, const double *V, double dt) {
  for (long long n = 0; n < s->nodes; ++n)
    for (int a = 0; a < 3; ++a) s->gv[3 * n + a] = V[a * s->nodes + n];
  return g2p(s, dt);
}

void ora_last_grid(const ora_sim *s, double *mass, double *mom) {
  memcpy(mass, s->gm, sizeof(double) * s->nodes);
  memcpy(mom, s->gp, sizeof(double) * 3 * s->nodes);
}

/* V_i of the last grid update, [3][nodes]. */
void ora_last_grid_velocity(const ora_sim *s, double *V) {
  for (long long n = 0; n < s->nodes; ++n)
    for (int a = 0; a < 3; ++a) V[a * s->nodes + n] = s->gv[3 * n + a];
}

/* ------------------------------------------------------------------ */
/* Height map of the deformed top surface (Sec. III-B).  Each top-layer
 * particle carries the height z_top + dX (z_p - z_p^0); a pixel centre within
 * dX/2 of a particle in the xy plane takes the largest such height; pixels
 * no particle covers copy the nearest covered pixel within fill_radius
 * (ties: lowest row-major index) or the rest top plane. */
void ora_heightmap(const ora_sim *s, const double window[4], int w, int h,
                   int fill_radius, double *H) {
  double dx = s->p.dx;
  double pxc = ((window[2] - window[0]) / (double)w) / dx;
  double pyc = ((window[3] - window[1]) / (double)h) / dx;
  float A0X = (float)((window[0] - s->origin[0]) / dx + 0.5 * pxc);
  float A0Y = (float)((window[1] - s->origin[1]) / dx + 0.5 * pyc);
  float SX = (float)pxc, SY = (float)pyc;
  long long P = (long long)w * h;
  double *cov = (double *)malloc(sizeof(double) * P);
  unsigned char *has = (unsigned char *)calloc(P, 1);
  for (long long e = 0; e < P; ++e) cov[e] = 0.0;
  for (long long q = 0; q < s->N; ++q) {
    if (!(s->flags[q] & 2)) continue;
    float ux = (float)s->xi[3 * q + 0], uy = (float)s->xi[3 * q + 1];
    double hp = s->z_top + dx * (s->xi[3 * q + 2] - s->rest_z[q]);
    /* conservative pixel box around the particle, then the exact test */
    int c0 = (int)floor(((double)ux - 0.5 - (double)A0X) / (double)SX) - 2;
    int c1 = (int)ceil(((double)ux + 0.5 - (double)A0X) / (double)SX) + 2;
    int r0 = (int)floor(((double)uy - 0.5 - (double)A0Y) / (double)SY) - 2;
    int r1 = (int)ceil(((double)uy + 0.5 - (double)A0Y) / (double)SY) + 2;
    if (c0 < 0) c0 = 0;
    if (r0 < 0) r0 = 0;
    if (c1 > w - 1) c1 = w - 1;
    if (r1 > h - 1) r1 = h - 1;
    for (int r = r0; r <= r1; ++r)
      for (int c = c0; c <= c1; ++c) {
        float qx = fmaf((float)c, SX, A0X);
        float qy = fmaf((float)r, SY, A0Y);
        float ex = qx - ux;
        float ey = qy - uy;
        float a = ex * ex;
        float b = ey * ey;
        if ((a + b) <= 0.25f) {
          long long e = (long long)r * w + c;
          if (!has[e] || hp > cov[e]) cov[e] = hp;
          has[e] = 1;
        }
      }
  }
  for (int r = 0; r < h; ++r)
    for (int c = 0; c < w; ++c) {
      long long e = (long long)r * w + c;
      if (has[e]) { H[e] = cov[e]; continue; }
      long long best = -1, bestd = 0;
      for (int rr = r - fill_radius; rr <= r + fill_radius; ++rr)
        for (int cc = c - fill_radius; cc <= c + fill_radius; ++cc) {
          if (rr < 0 || cc < 0 || rr >= h || cc >= w) continue;
          long long f = (long long)rr * w + cc;
          if (!has[f]) continue;
          long long d = (long long)(rr - r) * (rr - r) + (long long)(cc - c) * (cc - c);
          if (best < 0 || d < bestd || (d == bestd && f < best)) { best = f; bestd = d; }
        }
      H[e] = best >= 0 ? cov[best] : s->z_top;
    }
  free(cov);
  free(has);
}

/* Phong shading of the height map, Eqs. 12-14.  D = z_top - H is the
 * indentation depth; N = normalize(dD/dx, dD/dy, -1) by the [-1,0,1]/(2r)
 * stencil with replicated edges; V = (0,0,-1) points at the camera. */
void ora_shade(const double *H, int w, int h, double pixel_x_m, double pixel_y_m,
               double z_top_m, const ora_render_params *rp, double *rgb) {
  for (int r = 0; r < h; ++r)
    for (int c = 0; c < w; ++c) {
      int cl = c > 0 ? c - 1 : 0, cr = c < w - 1 ? c + 1 : w - 1;
      int ru = r > 0 ? r - 1 : 0, rd = r < h - 1 ? r + 1 : h - 1;
      double Dl = z_top_m - H[(long long)r * w + cl], Dr = z_top_m - H[(long long)r * w + cr];
      double Du = z_top_m - H[(long long)ru * w + c], Dd = z_top_m - H[(long long)rd * w + c];
      double gx = (Dr - Dl) / (2.0 * pixel_x_m);
      double gy = (Dd - Du) / (2.0 * pixel_y_m);
      double nn = sqrt(gx * gx + gy * gy + 1.0);
      double N[3] = {gx / nn, gy / nn, -1.0 / nn};
      double Vv[3] = {0.0, 0.0, -1.0};
      double I[3];
      for (int ch = 0; ch < 3; ++ch) I[ch] = rp->ka * rp->ambient[ch];
      for (int m = 0; m < rp->n_lights; ++m) {
        const double *L = rp->dir[m];
        double LN = L[0] * N[0] + L[1] * N[1] + L[2] * N[2];
        double R[3];
        for (int a = 0; a < 3; ++a) R[a] = 2.0 * LN * N[a] - L[a]; /* Eq. 13 */
        double RV = R[0] * Vv[0] + R[1] * Vv[1] + R[2] * Vv[2];
        double dif = LN > 0.0 ? LN : 0.0;
        double spe = RV > 0.0 ? pow(RV, rp->alpha) : 0.0;
        for (int ch = 0; ch < 3; ++ch)
          I[ch] += rp->kd * dif * rp->diffuse[m][ch] + rp->ks * spe * rp->specular[m][ch];
      }
      for (int ch = 0; ch < 3; ++ch) {
        double x = I[ch];
        rgb[((long long)r * w + c) * 3 + ch] = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
      }
    }
}
