/*
 * tacchi_oracle.h -- plain, slow FP64 CPU oracle of the Tacchi elastomer
 * method (arXiv 2301.08343, Sec. III-A and III-B).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and tacchi_oracle.c are used by the
 * tests, by smoke() and by the CPU-baseline leg of bench.py.  The product
 * library never includes, links or calls any of it, and nothing here comes
 * from the product library: no shared headers, kernels, helpers or tables.
 *
 * State convention shared with the product only through plain arrays:
 *   positions  u  : float [3][N], grid-cell units relative to grid node 0
 *                   (x_m = origin_m + u * dx), SoA by axis;
 *   velocities v  : float [3][N], m/s;
 *   affine     C  : float [9][N], 1/s, row-major 3x3 entry (r*3+c) major;
 *   deformation Fm: float [9][N], F - I (row-major entry major);
 *   flags        : uint8 [N], bit0 = base layer (Eq. 10 set B),
 *                  bit1 = top surface layer (height map, Sec. III-B).
 */
#ifndef TACCHI_ORACLE_H
#define TACCHI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;                 /* elastomer block in grid cells */
  int pad_side, pad_bottom, pad_top; /* grid padding around the block, cells */
  double dx;                      /* grid node interval Delta X [m] */
  double E, nu, rho;              /* Young's modulus [Pa], Poisson, density */
  double gravity[3];              /* [m/s^2], 0 unless a test sets it */
  int fix_base;                   /* 1: base set B and base nodes held fixed */
  int slip;                       /* 1: slip contact with the grid-boundary
                                     indenter (else sticky, Eq. 10) */
} ora_params;

typedef struct {
  int n_lights;                   /* <= 8 */
  double dir[8][3];               /* unit vector surface -> light, L_m */
  double diffuse[8][3];           /* i_{m,d} per RGB channel */
  double specular[8][3];          /* i_{m,s} per RGB channel */
  double ambient[3];              /* i_a */
  double ka, kd, ks, alpha;       /* reflectance constants of Eq. 12 */
} ora_render_params;

typedef struct ora_sim ora_sim;

/* error bits returned by ora_substep / ora_run */
#define ORA_ERR_OUT_OF_GRID 1
#define ORA_ERR_NUMERICAL 2

/* indenter kinds */
#define ORA_IND_NONE 0
#define ORA_IND_SPHERE 1
#define ORA_IND_CYLINDER 2
#define ORA_IND_CONE 3
#define ORA_IND_PRISM 4
#define ORA_IND_HEIGHTMAP 5

int ora_lattice(int nx, int ny, int nz, int pad_side, int pad_bottom,
                uint64_t seed, int jitter, float *u, uint8_t *flags);
uint64_t ora_splitmix64_at(uint64_t seed, uint64_t counter);

ora_sim *ora_create(const ora_params *p);
void ora_destroy(ora_sim *s);
long long ora_num_particles(const ora_sim *s);
void ora_grid_dims(const ora_sim *s, int dims[3]);
void ora_set_threads(int n);

void ora_set_state(ora_sim *s, const float *u, const float *v, const float *C,
                   const float *Fm, const uint8_t *flags);
void ora_set_rest(ora_sim *s, const float *u0);
void ora_get_state(const ora_sim *s, double *xi, double *v, double *C, double *F);
void ora_get_state_f32(const ora_sim *s, float *u, float *v, float *C, float *Fm);

int ora_set_indenter(ora_sim *s, int kind, const double *params, int hm_w,
                     int hm_h, double hm_pixel_m, const float *hm,
                     const double pose[7], const double vel[6]);
/* Indenter represented by n particles (Eq. 10, p in I): local positions
 * pts (m, [n][3]) in the indenter frame, each of the given mass; they add
 * mass and momentum to the grid at the rigid velocity, and grid nodes are no
 * longer overridden by the shape.  n = 0 restores the grid boundary.
 * Returns 0, or -1 on bad arguments. */
int ora_set_indenter_particles(ora_sim *s, long long n, const double *pts, double mass);
void ora_get_pose(const ora_sim *s, double pose[7]);
int ora_node_inside(const ora_sim *s, int i, int j, int k);

void ora_p2g(ora_sim *s, double dt, double *mass, double *mom);
int ora_substep(ora_sim *s, double dt);
int ora_run(ora_sim *s, int n, double dt);
/* Eqs. 7-11 alone from the grid velocity V [3][nodes]; returns error bits. */
int ora_g2p(ora_sim *s, const double *V, double dt);
void ora_last_grid(const ora_sim *s, double *mass, double *mom);
void ora_last_grid_velocity(const ora_sim *s, double *V);

void ora_weights(const double xi[3], int base[3], double w[27]);
void ora_polar(const double F[9], double R[9]);
void ora_stress(const double F[9], double mu, double la, double tau[9]);

void ora_heightmap(const ora_sim *s, const double window[4], int w, int h,
                   int fill_radius, double *H);
void ora_shade(const double *H, int w, int h, double pixel_x_m,
               double pixel_y_m, double z_top_m, const ora_render_params *rp,
               double *rgb);

#ifdef __cplusplus
}
#endif
#endif
