/*
 * tacchi.h -- C ABI of the GB300 elastomer simulator and tactile renderer.
 *
 * The library simulates the elastomer of an optical tactile sensor pressed by
 * a rigid indenter with the Material Point Method (Tacchi, arXiv 2301.08343,
 * Sec. III-A) and renders the deformed top surface into a tactile image
 * (Sec. III-B).  Every step of the computation runs in the library's own
 * CUDA kernels for sm_103a on one GPU.
 *
 * Conventions for every call:
 *   - A call returns a tacchi_status; TACCHI_OK is 0, errors are negative.
 *   - Work is queued asynchronously on the stream given at creation.
 *     Errors detected on the device (a particle leaving the grid, NaN,
 *     det F <= 0, a bounded wait running out) are recorded in a device error
 *     word and reported by the next call that synchronises (tacchi_sync,
 *     tacchi_get_state, and heightmap/render calls with host outputs).
 *     Once reported they stay set ("sticky") until tacchi_set_state or
 *     tacchi_clear_error.
 *   - The library copies everything it is given; the caller owns its
 *     buffers.  "dev" pointers must be device memory of the context's device;
 *     "host" pointers are ordinary host memory; a pointer documented as
 *     "host or dev" may be either (the library checks which).
 *   - Positions in state buffers are in grid-cell units measured from grid
 *     node 0: x_world = origin_m + u * dx_m (see tacchi_info).  F is carried
 *     as F - I for precision near the rest state.
 *   - Arrays of per-particle quantities are structure-of-arrays: component c
 *     of particle p is at [c * n_particles + p]; 3x3 matrices are row-major,
 *     entry (r, c) is component r * 3 + c.
 */
#ifndef TACCHI_H
#define TACCHI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tacchi_ctx *tacchi_handle; /* opaque, library-owned */

typedef enum {
  TACCHI_OK = 0,
  TACCHI_ERR_INVALID_ARG = -1, /* a size, pointer or parameter is out of range */
  TACCHI_ERR_OOM = -2,         /* device or host allocation failed */
  TACCHI_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  TACCHI_ERR_NUMERICAL = -4,   /* NaN/Inf or det F <= 0 seen on the device */
  TACCHI_ERR_OUT_OF_GRID = -5, /* a particle's stencil reached the padding band */
  TACCHI_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
  TACCHI_ERR_STATE = -7,       /* call not valid in the current state */
  TACCHI_ERR_CFL = -8          /* a particle moved a cell or more in one substep */
} tacchi_status;

/* Elastomer block and material (Sec. IV-B: block size, Young's modulus and
 * Poisson's ratio; the paper gives no density, so it is a parameter).
 * The block occupies [0, extent_m[0]] x [0, extent_m[1]] x [0, extent_m[2]]
 * in the world frame; its bottom face z = 0 is the sensor base. */
typedef struct {
  double extent_m[3];  /* block size (m); each must be a whole multiple of dx_m */
  double dx_m;         /* grid node interval Delta X (m) */
  double E_pa;         /* Young's modulus (Pa), > 0 */
  double nu;           /* Poisson's ratio, in (-1, 0.5) */
  double density;      /* kg/m^3, > 0 */
  uint64_t seed;       /* seed of the jittered particle lattice */
  int jitter;          /* 1: jitter each particle in its sub-cell; 0: centres */
  int pad_side;        /* grid cells around the block in x and y (0 -> 4; 3..1024) */
  int pad_bottom;      /* grid cells below the base (0 -> 3; 3..1024) */
  int pad_top;         /* grid cells above the top face (0 -> 4; 3..1024) */
  double gravity[3];   /* m/s^2, applied on the grid; the paper uses none */
  int free_base;       /* 0: base held fixed (Eq. 10); 1: no base condition */
  int block[3];        /* particle-sort block in cells (0 -> library default) */
  int threads_per_cell; /* transfer threads sharing a cell: 1 or 3 (0 -> 1); 3
                           needs an 8x8x4 or 4x4x4 block; see tacchi_set_transfer */
  int contact_mode;     /* grid-boundary indenter contact: TACCHI_CONTACT_STICKY
                           (0, the default) or TACCHI_CONTACT_SLIP (1) */
} tacchi_elastomer_desc;

/* Contact of the grid-boundary indenter with the elastomer (Sec. III-A, Eq. 10:
 * the paper's indenter moves the grid nodes it covers with its own velocity,
 * a no-slip contact; it has no friction model, Sec. V).
 * STICKY: a grid node inside the indenter takes the indenter's rigid velocity.
 * SLIP: a node inside the indenter that holds mass keeps its velocity except
 * for the part that moves into the indenter relative to it: with n the
 * outward normal of the indenter's surface at the node (radial for the sphere
 * and the cylinder, the lateral face for the cone and the prism, the surface
 * gradient for a height map) and W the indenter's velocity there,
 * V <- V - min(0, (V - W).n) n; empty nodes take W. */
#define TACCHI_CONTACT_STICKY 0
#define TACCHI_CONTACT_SLIP 1

typedef enum {
  TACCHI_INDENTER_NONE = 0,
  TACCHI_INDENTER_SPHERE = 1,    /* params[0] = radius; pose = centre */
  TACCHI_INDENTER_CYLINDER = 2,  /* params = radius, half length; axis = local x */
  TACCHI_INDENTER_CONE = 3,      /* params = half angle (rad), height; apex at pose, opens to local +z */
  TACCHI_INDENTER_PRISM = 4,     /* params = half angle, half length (local y), height; edge at pose */
  TACCHI_INDENTER_HEIGHTMAP = 5  /* params[0] = thickness above the back plane; see hm */
} tacchi_indenter_kind;

/* Rigid indenter (Sec. III-A, Eq. 10; Sec. III-C).  The indenter acts on the
 * grid: a grid node inside the solid at the pose of the start of a substep
 * takes the indenter's rigid velocity.  For TACCHI_INDENTER_HEIGHTMAP the
 * solid is { |x_l|,|y_l| within the map, -hm(x_l, y_l) <= z_l <= params[0] }
 * in the local frame: hm holds protrusion heights (m, >= 0) below the flat
 * back plane z_l = 0, sampled at pixel centres, row j along local y. */
typedef struct {
  int kind;           /* tacchi_indenter_kind */
  double params[8];   /* shape lengths in metres, angles in radians */
  int hm_w, hm_h;     /* height-map samples (>= 2 each) */
  double hm_pixel_m;  /* height-map sample spacing (m) */
  const float *hm;    /* host, [hm_h][hm_w]; copied by the call */
} tacchi_indenter_desc;

/* Phong lighting (Eqs. 12-14).  dir[m] is the unit vector from the surface
 * towards light m; the camera looks along +z from below (V = (0,0,-1)). */
typedef struct {
  int n_lights;          /* 0..8 */
  float dir[8][3];
  float diffuse[8][3];   /* i_{m,d}, RGB */
  float specular[8][3];  /* i_{m,s}, RGB */
  float ambient[3];      /* i_a, RGB */
  float ka, kd, ks, alpha;
} tacchi_render_params;

typedef struct {
  int64_t n_particles;
  int64_t n_surface;      /* particles of the top layer (height map samples) */
  int grid[3];            /* grid nodes per axis */
  int64_t n_nodes;
  double origin_m[3];     /* world position of grid node 0 */
  double dx_m;
  double z_top_m;         /* rest height of the top face */
  int block[3];           /* particle-sort block in cells */
  int64_t n_blocks;
  size_t device_bytes;    /* device memory held by the context */
  int threads_per_cell;   /* transfer threads sharing a cell (1 or 3) */
  int pipelined;          /* fused transfers run pipelined (tacchi_set_pipeline) */
} tacchi_info_t;

/* Create a simulator on the current CUDA device (Sec. III-A, Initialization;
 * Eq. 1).  Particles: 2x2x2 per grid cell of the block, each in its own
 * sub-cell, jittered with the counter-based splitmix64 generator seeded by
 * desc->seed (draw 3p+a for axis a of particle p); v = 0, C = 0, F = I.
 * Particles of the bottom cell layer form the fixed set B of Eq. 10; the
 * upper particle layer of the top cell layer gives the height-map samples.
 * stream: a cudaStream_t (NULL = the legacy default stream); the library
 * does not take ownership.  *out receives the handle.
 * Errors: INVALID_ARG (bad sizes/material, extents not multiples of dx_m,
 * padding outside 3..1024, more than 2e9 particles or 2^31 - 1 grid nodes),
 * OOM, CUDA. */
tacchi_status tacchi_create(const tacchi_elastomer_desc *desc, void *stream,
                            tacchi_handle *out);

/* Release every resource of the context (waits for its queued work). */
void tacchi_destroy(tacchi_handle h);

/* Sizes and frames of the context; out: host. */
tacchi_status tacchi_info(tacchi_handle h, tacchi_info_t *out);

/* Indenter shape, pose and velocity (Sec. III-C: the main simulator supplies
 * the indenter's position or velocity every step).  Each argument may be
 * NULL to keep the current value.  pose = position (m) and unit quaternion
 * (w, x, y, z) of the local frame; vel = linear (m/s) and angular (rad/s)
 * velocity in the world frame.  Within a tacchi_step the pose advances by
 * dt * vel per substep (Eq. 11 applied to the rigid indenter).
 * Errors: INVALID_ARG (unknown kind, bad height map, non-finite values). */
tacchi_status tacchi_set_indenter(tacchi_handle h, const tacchi_indenter_desc *desc,
                                  const double pose[7], const double vel[6]);

/* Current indenter pose (after the substeps queued so far); out: host. */
tacchi_status tacchi_get_indenter_pose(tacchi_handle h, double pose[7]);

/* Advance n_substeps explicit MLS-MPM substeps of length dt (Sec. III-A:
 * particle-to-grid Eqs. 2-5, grid velocity Eq. 6 with the indenter, the
 * fixed base and the padding band, grid-to-particle Eqs. 7-9, the base
 * override Eq. 10 and advection Eq. 11).  Asynchronous; the substeps run as
 * one CUDA graph.  Errors: INVALID_ARG (n_substeps < 1, dt <= 0), CUDA;
 * device-side errors are reported by the next synchronising call. */
tacchi_status tacchi_step(tacchi_handle h, int n_substeps, double dt);

/* Height map of the deformed top surface (Sec. III-B, "2D interpolation").
 * Each top-layer particle carries the height z_top + dx * (u_z - u_z_rest);
 * a pixel whose centre lies within dx/2 of a particle in the xy plane takes
 * the largest height among such particles; other pixels copy the nearest
 * covered pixel within fill_radius pixels (ties: lowest row-major index), or
 * z_top if none.  window_m = (x0, y0, x1, y1) in the world frame; pixel
 * (r, c) is centred at (x0 + (c + 1/2)(x1-x0)/w, y0 + (r + 1/2)(y1-y0)/hgt).
 * out: host or dev, float [hgt][w], metres (host output synchronises).
 * Errors: INVALID_ARG (w, hgt < 1, empty window, fill_radius outside 0..64). */
tacchi_status tacchi_heightmap(tacchi_handle h, int w, int hgt, const double window_m[4],
                               int fill_radius, float *out);

/* Tactile image (Sec. III-B, Eqs. 12-14): the height map above, converted to
 * the indentation depth D = z_top - H, shaded with Phong's model; normals
 * N = normalize(dD/dx, dD/dy, -1) from the [-1, 0, 1] / (2 r) stencil with
 * replicated edges; each channel clamped to [0, 1].
 * out_rgb: host or dev, float [hgt][w][3]; out_height: optional (NULL) host
 * or dev float [hgt][w].  Errors as tacchi_heightmap, plus INVALID_ARG for
 * n_lights outside 0..8. */
tacchi_status tacchi_render(tacchi_handle h, const tacchi_render_params *rp, int w,
                            int hgt, const double window_m[4], int fill_radius,
                            float *out_rgb, float *out_height);

/* Shading alone (Eqs. 12-14) of a caller-provided height map H_dev (dev,
 * float [hgt][w], metres) with pixel sizes pixel_x_m, pixel_y_m and rest top
 * height z_top_m, into rgb_dev (dev, float [hgt][w][3]), on stream.
 * Needs no context.  Errors: INVALID_ARG, CUDA. */
tacchi_status tacchi_shade(const tacchi_render_params *rp, const float *H_dev, int w,
                           int hgt, double pixel_x_m, double pixel_y_m, double z_top_m,
                           float *rgb_dev, void *stream);

/* Largest height map, in pixels, that tacchi_heightmap_static accepts. */
#define TACCHI_STATIC_HEIGHTMAP_MAX_PIXELS (1 << 20)

/* Height map without any memory allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they run, such as a robot simulator's real-time control thread (where
 * cudaMalloc can block and synchronise the device for an unbounded time) or a
 * plugin whose host application owns the whole device-memory budget.
 * It computes the same height map as tacchi_heightmap, but from particle
 * arrays the caller passes in: u_dev (dev, float [3][n_particles], positions
 * in cells from grid node 0, the layout of tacchi_get_state), surf_dev (dev,
 * uint32 [n_surface], ids of the top-layer particles, flag bit 1), z0_dev
 * (dev, float [n_surface], their rest z in cells), dx_m, origin_m (x and y of
 * grid node 0, m), z_top_m (rest height of the top face).  Every id in
 * surf_dev must be below n_particles: the library cannot check device data
 * from the host without a copy, and a larger id reads past u_dev.
 * window_m, w, hgt, fill_radius and out_dev (dev, float [hgt][w], metres) are
 * as in tacchi_heightmap; the work is queued on stream.
 * Scratch: a static device array of TACCHI_STATIC_HEIGHTMAP_MAX_PIXELS ints
 * (4 MiB) that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address (with the
 * device current).  That first call, like the first launch of any of the
 * library's kernels on a device, may also load the library's GPU code, and
 * loading can allocate device memory (the 4 MiB array included).  So make
 * one warm-up call per device at initialisation, before any stream capture
 * and before the real-time loop; later calls allocate nothing.  Every call
 * clears and reuses the same array, so calls that overlap on the GPU
 * (unordered streams or threads) race and corrupt each other's output.
 * Errors: INVALID_ARG (null pointers, w * hgt above the maximum, bad window),
 * CUDA. */
tacchi_status tacchi_heightmap_static(const float *u_dev, int64_t n_particles,
                                      const uint32_t *surf_dev, const float *z0_dev,
                                      int n_surface, double dx_m, const double origin_m[2],
                                      double z_top_m, int w, int hgt, const double window_m[4],
                                      int fill_radius, float *out_dev, void *stream);

/* Copy the particle state out (synchronises).  Each pointer may be NULL to
 * skip it; all are dev: u float [3][N] (cells), v float [3][N] (m/s),
 * C float [9][N] (1/s), Fm float [9][N] (F - I), flags uint8 [N] (bit 0 =
 * base set of Eq. 10, bit 1 = top-layer surface particle).  Returns the
 * sticky device error, if any, after copying. */
tacchi_status tacchi_get_state(tacchi_handle h, float *u, float *v, float *C, float *Fm,
                               uint8_t *flags);

/* Replace the particle state (dev pointers in the layout of tacchi_get_state;
 * v, C, Fm may be NULL for zero / zero / identity).  Clears the sticky error
 * and re-sorts the particles.  Errors: INVALID_ARG (u NULL), CUDA. */
tacchi_status tacchi_set_state(tacchi_handle h, const float *u, const float *v,
                               const float *C, const float *Fm);

/* Grid mass and momentum of the most recent particle-to-grid transfer
 * (Eqs. 2-5), i.e. of the state at the start of the last substep of the last
 * tacchi_step.  out: dev float [n_nodes][4] = (M_i, MG_i x, y, z), node
 * index (k * grid[1] + j) * grid[0] + i.  Errors: STATE (no step yet). */
tacchi_status tacchi_get_grid(tacchi_handle h, float *out);

/* Device time per kernel kind, accumulated while profiling is on. */
typedef struct {
  double grid_ms;        /* grid updates (Eq. 6 + boundaries) */
  double fused_ms;       /* fused G2P + P2G transfers (Eqs. 2-5, 7-11) */
  double edge_ms;        /* P2G-only and G2P-only transfers opening/closing a step */
  double sort_ms;        /* particle sort (three kernels, timed together) */
  int64_t grid_launches, fused_launches, edge_launches, sort_launches;
  int64_t sort_runs;     /* sorts that did work: some particle had left its block
                            (the others only checked the flag) */
} tacchi_profile_t;

/* Turn kernel timing on (1) or off (0).  While on, every step graph carries
 * CUDA events around its kernels and tacchi_step synchronises after each
 * graph launch to accumulate their durations.  Errors: INVALID_ARG. */
tacchi_status tacchi_set_profiling(tacchi_handle h, int on);

/* Accumulated kernel times since profiling was turned on or last reset;
 * reset != 0 zeroes them after reading.  Synchronises the stream (to read the
 * device count of sorts).  out: host.  Errors: INVALID_ARG, CUDA. */
tacchi_status tacchi_get_profile(tacchi_handle h, tacchi_profile_t *out, int reset);

/* Measured FP32 FMA throughput of the current device, the ALU roof of the
 * fused transfer (which does about 15 FP32 operations per byte it moves; the
 * paper gives no roofline, this is measurement support).  Runs independent
 * FMA chains, scalar and packed two-lane, over four full waves of every SM
 * and writes the best rate in TFLOP/s (2 flop per lane per FMA) to *tflops;
 * *sm_count and *sm_clock_khz (optional) receive the SM count and the
 * device's maximum SM clock attribute (0 when the driver does not report
 * it).  Allocates 4 bytes of device memory and a stream for the duration of
 * the call; synchronises.  Errors: INVALID_ARG (null tflops), CUDA, OOM. */
tacchi_status tacchi_measure_fp32_peak(double *tflops, int *sm_count, int *sm_clock_khz);

/* Wait for the context's queued work and report the sticky device error. */
tacchi_status tacchi_sync(tacchi_handle h);

/* Clear the sticky device error. */
tacchi_status tacchi_clear_error(tacchi_handle h);

/* The particle lattice tacchi_create would make, written to host arrays
 * (no GPU needed): u float [3][N] cells, flags uint8 [N];
 * N = 8 * nx * ny * nz.  Errors: INVALID_ARG. */
tacchi_status tacchi_init_lattice(int nx, int ny, int nz, int pad_side, int pad_bottom,
                                  uint64_t seed, int jitter, float *u, uint8_t *flags);

/* ---- Batches of independent sensors --------------------------------------
 * A batch holds n independent elastomer instances (each with its own size,
 * material, particles, grid and indenter) that advance together: one
 * tacchi_step runs every substep of every instance as one CUDA graph launch,
 * each kernel covering all instances.  A handle made by tacchi_create is a
 * batch of one; the calls above act on instance 0 of any handle.  The paper
 * simulates one sensor at a time; batching is this library's addition. */

/* Create a batch of n instances from descs[0..n-1] (host array), on the
 * current device and the given stream.  Errors: as tacchi_create, and
 * INVALID_ARG for n < 1 or n > 65536. */
tacchi_status tacchi_batch_create(int n, const tacchi_elastomer_desc *descs, void *stream,
                                  tacchi_handle *out);

/* Number of instances of a handle (1 for tacchi_create); out: host. */
tacchi_status tacchi_batch_size(tacchi_handle h, int *out);

/* Per-instance forms of tacchi_info / tacchi_set_indenter /
 * tacchi_get_indenter_pose / tacchi_heightmap / tacchi_render /
 * tacchi_get_state / tacchi_set_state (same arguments, layouts and errors;
 * state arrays hold that instance's n_particles).  INVALID_ARG if i is out
 * of range. */
tacchi_status tacchi_batch_info(tacchi_handle h, int i, tacchi_info_t *out);
tacchi_status tacchi_batch_set_indenter(tacchi_handle h, int i, const tacchi_indenter_desc *desc,
                                        const double pose[7], const double vel[6]);
tacchi_status tacchi_batch_get_indenter_pose(tacchi_handle h, int i, double pose[7]);
tacchi_status tacchi_batch_heightmap(tacchi_handle h, int i, int w, int hgt, const double window_m[4],
                                     int fill_radius, float *out);
tacchi_status tacchi_batch_render(tacchi_handle h, int i, const tacchi_render_params *rp, int w,
                                  int hgt, const double window_m[4], int fill_radius, float *out_rgb,
                                  float *out_height);
tacchi_status tacchi_batch_get_state(tacchi_handle h, int i, float *u, float *v, float *C, float *Fm,
                                     uint8_t *flags);
tacchi_status tacchi_batch_set_state(tacchi_handle h, int i, const float *u, const float *v,
                                     const float *C, const float *Fm);

/* Top-surface displacement of instance i sampled on a w x hgt pixel grid
 * over window_m (world frame): pixel (r, c) takes the displacement (m, x/y/z)
 * of the top-layer particle whose rest sub-cell (the particle lattice at
 * spacing dx/2 over the block's top face, clamped to it) contains the pixel
 * centre.  The surrogate's training target and error reference; the paper
 * has no counterpart.  out_dev: dev float [hgt][w][3].  Asynchronous. */
tacchi_status tacchi_batch_displacement_map(tacchi_handle h, int i, int w, int hgt, const double window_m[4],
                                            float *out_dev);

/* Indenter represented by particles, the paper's own contact model (Eq. 10:
 * the particles of set I share the rigid indenter's velocity; Sec. III-C:
 * they are initialised from a point cloud of the object, and a sparse cloud
 * gives the surface "defects" of Sec. IV-B).  local_m: host float [n][3],
 * positions (m) in the indenter's local frame (the frame its pose maps to
 * the world); mass_kg: the mass of each.  At the pose of the start of every
 * substep each particle adds w m and w m (v + C (X_i - x)) to its grid nodes
 * (Eqs. 2-4), with v the rigid velocity at its position and C = skew of the
 * angular velocity, and no elastic term; grid nodes are then no longer
 * overridden by the shape, which keeps serving the penetration map.  n = 0
 * returns instance i to the grid-boundary indenter.  Synchronises; drops
 * cached step graphs.  Errors: INVALID_ARG (n < 0 or > 2^26, non-finite
 * positions, mass <= 0), OOM, CUDA. */
tacchi_status tacchi_batch_set_indenter_particles(tacchi_handle h, int i, int n, const float *local_m,
                                                  double mass_kg);
tacchi_status tacchi_set_indenter_particles(tacchi_handle h, int n, const float *local_m, double mass_kg);

/* Marker motion (the outlook of Sec. V: markers on the elastomer surface are
 * particles that share the markers' positions, so recording the surface
 * particles' motion gives the markers').  Marker k of instance i at rest at
 * xy_dev[k] = (x, y) (world frame, m, on the top face) follows the top-layer
 * particle whose rest sub-cell (the particle lattice at spacing dx/2 over the
 * top face, clamped to it) contains (x, y): out_dev[k] = its displacement
 * from rest (m, x/y/z).  The same selection as tacchi_batch_displacement_map.
 * xy_dev: dev float [n][2]; out_dev: dev float [n][3].  Asynchronous.
 * Errors: INVALID_ARG (i out of range, n < 1 or > 2^24, null pointers). */
tacchi_status tacchi_batch_markers(tacchi_handle h, int i, int n, const float *xy_dev, float *out_dev);

/* Penetration of instance i's indenter into the rest top face at its current
 * pose: per pixel centre (x, y) of window_m, max(0, z_top - z_b(x, y)) with
 * z_b the lowest point of the indenter over (x, y) (m).  Only rotations
 * about the vertical axis are supported.  The surrogate's input; the paper
 * has no counterpart.  out_dev: dev float [hgt][w].  Errors: INVALID_ARG
 * (a pose tilted out of the horizontal plane). */
tacchi_status tacchi_batch_penetration_map(tacchi_handle h, int i, int w, int hgt, const double window_m[4],
                                           float *out_dev);

/* Comparison renderer: the depth-smoothing simulators Tacchi is compared
 * with in Sec. II build a pseudo elastomer surface by smoothing the
 * indenter's depth map with a Gaussian kernel, with no physics; the image is
 * then shaded like Tacchi's (Eqs. 12-14).  For instance i at its current
 * pose: p = the penetration map of tacchi_batch_penetration_map, extended
 * beyond the window (evaluated from the shape); s = p convolved with the
 * normalised discrete Gaussian of standard deviation sigma_m (m) on the
 * pixel lattice, truncated at R = ceil(3 sigma_m / pitch) pixels per axis
 * (sigma_m = 0: s = p); out_height = z_top - s; out_rgb = its shading with
 * rp (required).  out_rgb [hgt][w][3], out_height [hgt][w] or NULL;
 * each a device or a host pointer (host: the call synchronises).  Only
 * rotations about the vertical axis.  Errors: INVALID_ARG (a tilted pose,
 * sigma_m < 0 or not finite, R > 256 pixels, hgt + 2 R > 65535, a bad
 * window, rp NULL), OOM, CUDA. */
tacchi_status tacchi_batch_render_smoothed(tacchi_handle h, int i, const tacchi_render_params *rp, int w, int hgt,
                                           const double window_m[4], double sigma_m, float *out_rgb,
                                           float *out_height);
tacchi_status tacchi_render_smoothed(tacchi_handle h, const tacchi_render_params *rp, int w, int hgt,
                                     const double window_m[4], double sigma_m, float *out_rgb, float *out_height);

/* Put every instance back to its initial particle lattice (v = 0, C = 0,
 * F = I), clear the device error and re-sort; indenters are kept.  Lets a
 * caller reuse one handle (and its cached step graphs) for new presses.
 * Asynchronous.  Errors: INVALID_ARG, CUDA. */
tacchi_status tacchi_batch_reset(tacchi_handle h);

/* Sort-block shape (cells) used by the transfer kernel for every instance:
 * 4x4x4, 8x8x4, 8x8x8 or 16x8x4, with one thread per cell (the same as
 * tacchi_set_transfer(h, bx, by, bz, 1)).  Re-sorts the particles and drops
 * cached graphs.  Errors: INVALID_ARG for other shapes. */
tacchi_status tacchi_set_block(tacchi_handle h, int bx, int by, int bz);

/* Transfer plan of the fused G2P+P2G kernel (Sec. III-A, Eqs. 2-11): the
 * sort block (bx, by, bz) in cells and how many threads share a cell.
 * threads_per_cell = 1: one thread runs every particle of its cell and holds
 * the cell's 27 node sums; any of the four block shapes.  threads_per_cell =
 * 3: three threads split a cell's particles for G2P and the stress and its
 * node planes for P2G; blocks 8x8x4 or 4x4x4.  The library default is 8x8x4
 * with one thread per cell.  Both
 * compute the same substep up to FP32 rounding order.  Re-sorts the
 * particles and drops cached graphs.  Errors: INVALID_ARG for other plans. */
tacchi_status tacchi_set_transfer(tacchi_handle h, int bx, int by, int bz, int threads_per_cell);

/* Launch form of tacchi_step (Sec. III-A's substep loop; the paper runs it
 * as separate Taichi kernels).  GRAPH (the default): each chunk of up to 512
 * substeps is one CUDA graph of five kernels per substep.  PERSISTENT: each
 * chunk is one cooperative kernel that keeps every CTA resident and runs all
 * phases (grid update, fused transfer, sort when needed) with grid-wide
 * barriers between them; needs the 8x8x4 block with one thread per cell
 * (INVALID_ARG otherwise; a later change of plan falls back to GRAPH).
 * Every barrier wait is bounded (tacchi_set_barrier_wait): a CTA that gives
 * up reports TACCHI_ERR_TIMEOUT at the next synchronising call and every CTA
 * returns.  Synchronises.  Errors: INVALID_ARG, CUDA. */
#define TACCHI_LAUNCH_GRAPH 0
#define TACCHI_LAUNCH_PERSISTENT 1
tacchi_status tacchi_set_launch(tacchi_handle h, int mode);

/* Fused transfers of the graph form by the pipelined kernel (on = 1) or one
 * CTA per sort block (on = 0, the default; tacchi_autotune turns it on when
 * it times the pipelined form faster for the plan it picks).  The pipelined kernel
 * (Sec. III-A, Eqs. 2-11, the same arithmetic) keeps two CTAs per SM resident
 * over the sort's non-empty blocks: while a CTA runs one block's particles,
 * bulk asynchronous copies bring the next block's particle slots, home cells
 * and grid velocities into shared memory.  It exists for the 8x8x4 block with
 * one thread per cell; other plans use the per-block kernel whatever the
 * setting.  Its copy waits are bounded by tacchi_set_barrier_wait's max_polls
 * (TACCHI_ERR_TIMEOUT).  Synchronises.  Errors: INVALID_ARG (on not 0 or 1). */
tacchi_status tacchi_set_pipeline(tacchi_handle h, int on);

/* Bound of the persistent step's grid-barrier waits and of the pipelined
 * transfer's copy waits: a CTA gives up after max_polls polls (about 0.1 us
 * each; default 2^24), and a barrier waits for extra_arrivals arrivals beyond
 * its own (default 0).  A positive extra_arrivals makes every such wait wait
 * for arrivals that never come: it exists to exercise the bounded wait, which
 * then ends the step with TACCHI_ERR_TIMEOUT (a pipelined CTA that gives up
 * supplies the missing arrivals itself and waits for its copies in flight
 * before it leaves).  Errors: INVALID_ARG (max_polls < 1, extra_arrivals < 0
 * or > 65536). */
tacchi_status tacchi_set_barrier_wait(tacchi_handle h, int64_t max_polls, int extra_arrivals);

/* Number of transfer plans the autotuner tries, in this order:
 * 4x4x4/1, 8x8x4/1, 8x8x8/1, 16x8x4/1, 8x8x4/3, 4x4x4/3
 * (block shape / threads per cell). */
#define TACCHI_NUM_TRANSFER_PLANS 6

/* Autotuner: times n_substeps substeps of length dt with each transfer plan
 * on the handle's current state (which it saves and restores, together with
 * the indenter poses), a plan with a pipelined form both ways
 * (tacchi_set_pipeline), keeps the fastest and writes its plan to best[4]
 * (host: bx, by, bz, threads per cell); ms_per_substep (host, optional,
 * TACCHI_NUM_TRANSFER_PLANS entries) receives the time per substep of each
 * plan in the order above (of its faster form, where both were timed).  Synchronises.  Errors: INVALID_ARG, CUDA, and
 * any device error raised while timing. */
tacchi_status tacchi_autotune(tacchi_handle h, int n_substeps, double dt, int best[4],
                              double ms_per_substep[TACCHI_NUM_TRANSFER_PLANS]);

/* ---- Learned surrogate ------------------------------------------------------
 * A U-Net that maps per-pixel inputs (the indenter's penetration map over the
 * top face and the press depth) to per-pixel outputs (the top-surface
 * displacement), trained and run by the library's BF16 tensor-core kernels
 * with FP32 accumulation.  The paper has no surrogate; the MPM above stays
 * the reference and the fallback.
 * Architecture: encoder levels l = 0..levels-1 of width widths[l] with two
 * 3x3 conv+ReLU and 2x2 average pooling between levels; decoder levels with
 * nearest 2x upsampling, concatenation with the encoder output of the same
 * level and two 3x3 conv+ReLU; a 1x1 head.  Loss: mean squared error.
 * Parameters (FP32, host order): for each 3x3 conv in execution order
 * (enc0a, enc0b, ..., enc{L-1}b, dec{L-2}a, dec{L-2}b, ..., dec0b) the
 * weights [3][3][c_in][c_out] then the bias [c_out]; then the head
 * [widths[0]][out_channels] and its bias. */
typedef struct tacchi_nn *tacchi_nn_handle;

/* Create a network for height x width images (multiples of 2^(levels-1)),
 * in_channels <= 32, out_channels in {1, 2, 3, 4, 8, 16}, widths multiples
 * of 32, at most max_batch images per call; weights He-normal from
 * splitmix64(seed).
 * stream: cudaStream_t for all its work.  Errors: INVALID_ARG, OOM, CUDA. */
tacchi_status tacchi_nn_create(int levels, const int *widths, int in_channels, int out_channels, int height,
                               int width, int max_batch, uint64_t seed, void *stream, tacchi_nn_handle *out);
void tacchi_nn_destroy(tacchi_nn_handle n);
tacchi_status tacchi_nn_num_params(tacchi_nn_handle n, int64_t *out);
/* Copy the parameters (which = 0) or the last gradients (which = 1) to host
 * memory (float [num_params]), or set the parameters (resets Adam). */
tacchi_status tacchi_nn_get_params(tacchi_nn_handle n, int which, float *host);
tacchi_status tacchi_nn_set_params(tacchi_nn_handle n, const float *host);
/* y_dev (dev, float [batch][height][width][out_channels]) = network(x_dev),
 * x_dev (dev, float [batch][height][width][in_channels]).  Asynchronous. */
tacchi_status tacchi_nn_forward(tacchi_nn_handle n, int batch, const float *x_dev, float *y_dev);
/* Forward and backward: the gradients of the mean squared error against
 * target_dev (layout of y); loss_host (optional) receives the loss. */
tacchi_status tacchi_nn_gradients(tacchi_nn_handle n, int batch, const float *x_dev, const float *target_dev,
                                  float *loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on
 * that loss.  loss_host (optional) receives the loss before the step. */
tacchi_status tacchi_nn_train_step(tacchi_nn_handle n, int batch, const float *x_dev, const float *target_dev,
                                   float lr, float *loss_host);

/* Short English description of a status. */
const char *tacchi_status_string(tacchi_status s);

/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
int tacchi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TACCHI_H */
