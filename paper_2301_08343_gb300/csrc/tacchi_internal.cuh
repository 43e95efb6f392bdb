// tacchi_internal.cuh -- device-side data layout and small shared helpers of
// the GB300 Tacchi library.  Included only by the library's own .cu files.
//
// Layout in HBM (all instances of a batch concatenated):
//   particles (global index p, total Ntot):
//     ps [Ntot][3] float4  the per-substep state as one 48-byte record:
//                  (u0, u1, u2, H0) (H1, H2, H3, H4) (H5, H6, H7, H8), with
//                  u the position in grid-cell units from the instance's
//                  node 0 and H = F - I row-major; one thread loads or stores
//                  a particle with three 16-byte accesses
//     v  [3][Ntot], C [9][Ntot]  structure of arrays, only written at the
//                  end of a step call and read by the first transfer of the
//                  next call
//     flags [Ntot]  bit0 base set (Eq. 10), bit1 top-layer surface particle
//   sort: idx [Ntot] particle ids grouped by grid block, bstart [Nblk+1],
//     key [Ntot], bcount/cursor [Nblk]
//   grid (global node n, total Nnodes): gmm float4 (M, MGx, MGy, MGz),
//     gv float4 (Vx, Vy, Vz, 0)
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace tacchi {

// NVTX range over a host API call, shown on profiler timelines (a no-op
// unless a tool is attached).  The substep kernels run inside CUDA graphs,
// which profilers already list kernel by kernel.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};


enum : int {
  ERRBIT_OUT_OF_GRID = 1,
  ERRBIT_NUMERICAL = 2,
  ERRBIT_CFL = 4,
  ERRBIT_TIMEOUT = 8,
};

enum : int {
  IND_NONE = 0,
  IND_SPHERE = 1,
  IND_CYLINDER = 2,
  IND_CONE = 3,
  IND_PRISM = 4,
  IND_HEIGHTMAP = 5,
};

// Indenter frame of one substep, rounded to FP32 on the host from the FP64
// pose.  Local coordinates of node X: l = R^T (X - c), in cells.
struct IndenterFrame {
  float c[3];     // centre, cells
  float r[9];     // local -> world rotation, row-major
  float vlin[3];  // m/s
  float w[3];     // rad/s
};

struct IndenterShape {
  int kind;
  float s0, s1, s2, s3;        // shape constants in cells (see set_indenter)
  float inv_pix, offx, offy;   // height-map sampling
  int hm_w, hm_h;
  const float *hm;             // device, heights in cells
};

// One elastomer instance of a batch.
struct Instance {
  int G[3];          // nodes per axis
  int nb[3];         // sort blocks per axis
  int pad_bottom;    // node layer of the base plane
  int fix_base;
  long long node_off, N, part_off, block_off, nblocks;
  float dx, inv_dx;  // m, 1/m
  float m, V0;       // particle mass (kg), rest volume (m^3)
  float mu, la;      // Lame parameters (Pa)
  float gdt[3];      // gravity (m/s^2), multiplied by dt on use
  IndenterShape shape;
  const IndenterFrame *frames;  // [substep] for the running step chunk
  int ind_np;        // indenter particles (Eq. 10, p in I); 0: the grid boundary
  float ind_m;       // mass of each indenter particle (kg)
  int slip;          // contact mode of the grid-boundary indenter: 0 sticky, 1 slip
};

// A non-empty sort block as the pipelined transfer takes it, written by the
// sort in block order: particle range, instance, cell origin B0, and the
// instance's grid extent and first node (so that one 48-byte read places it).
struct BlockRec {
  uint32_t start, n;
  int ii, B0x, B0y, B0z;
  int G0, G1, G2, pad;
  long long node_off;
};
static_assert(sizeof(BlockRec) == 48, "block records are three 16-byte words");

struct Batch {
  const Instance *inst;       // [n_inst]
  const long long *node_offs; // [n_inst] first global node of each instance
  const long long *part_offs; // [n_inst] first global particle of each instance
  const uint32_t *block_inst; // [Nblk] instance of each global block
  int n_inst;
  long long Ntot, Nnodes, Nblk;
  float4 *ps;
  float *v, *C;
  const uint8_t *flags;
  uint32_t *idx, *key, *bstart, *bcount, *cursor;
  // home cell of the particle at each idx slot, within its sort block's cells
  // grown by one on every side ((ez * (BY + 2) + ey) * (BX + 2) + ex), or
  // kNotHome; written by the sort and by every transfer that groups its block,
  // which also leaves the block's idx slots in cell order
  uint16_t *hcell;
  BlockRec *brec;   // [Nblk] non-empty blocks, in block order
  uint32_t *blkq;   // [0] records in brec, [1] next record to hand out, [2] CTAs finished
  float4 *gmm, *gv;
  // indenter particles of all instances: local positions (cells) and the
  // instance of each
  const float *ind_pts;         // [Np][3]
  const uint32_t *ind_inst;     // [Np]
  long long Np;
  int *err;
  int *movers;  // [0] a particle left its block in the last transfer; [1] sorts that did work
};

constexpr uint16_t kNotHome = 0xFFFF;

// Particle records (see the layout above).
__device__ __forceinline__ void load_particle(const float4 *ps, long long p, float u[3], float H[9]) {
  const float4 *r = ps + 3 * p;
  const float4 a = r[0], b = r[1], c = r[2];
  u[0] = a.x; u[1] = a.y; u[2] = a.z;
  H[0] = a.w; H[1] = b.x; H[2] = b.y; H[3] = b.z; H[4] = b.w;
  H[5] = c.x; H[6] = c.y; H[7] = c.z; H[8] = c.w;
}

__device__ __forceinline__ void store_particle(float4 *ps, long long p, const float u[3], const float H[9]) {
  float4 *r = ps + 3 * p;
  r[0] = make_float4(u[0], u[1], u[2], H[0]);
  r[1] = make_float4(H[1], H[2], H[3], H[4]);
  r[2] = make_float4(H[5], H[6], H[7], H[8]);
}

__device__ __forceinline__ float4 load_position(const float4 *ps, long long p) { return ps[3 * p]; }

// Largest i with offs[i] <= x (offs ascending, offs[0] = 0).
__device__ __forceinline__ int find_instance(const long long *offs, int n, long long x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(offs + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Inside test of grid node (i, j, k), FP32, operation order fixed by
// round-to-nearest intrinsics (no contraction), so that any FP32
// implementation of the same sequence decides identically.
__device__ __forceinline__ bool inside_indenter(const IndenterShape &s, const IndenterFrame &f,
                                                int i, int j, int k) {
  if (s.kind == IND_NONE) return false;
  float d0 = __fsub_rn((float)i, f.c[0]);
  float d1 = __fsub_rn((float)j, f.c[1]);
  float d2 = __fsub_rn((float)k, f.c[2]);
  if (s.kind == IND_SPHERE) {
    float r2 = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
    return r2 <= s.s0;
  }
  float l0 = __fadd_rn(__fadd_rn(__fmul_rn(f.r[0], d0), __fmul_rn(f.r[3], d1)), __fmul_rn(f.r[6], d2));
  float l1 = __fadd_rn(__fadd_rn(__fmul_rn(f.r[1], d0), __fmul_rn(f.r[4], d1)), __fmul_rn(f.r[7], d2));
  float l2 = __fadd_rn(__fadd_rn(__fmul_rn(f.r[2], d0), __fmul_rn(f.r[5], d1)), __fmul_rn(f.r[8], d2));
  switch (s.kind) {
    case IND_CYLINDER:
      return fabsf(l0) <= s.s1 && __fadd_rn(__fmul_rn(l1, l1), __fmul_rn(l2, l2)) <= s.s0;
    case IND_CONE: {
      if (!(l2 >= 0.f && l2 <= s.s1)) return false;
      float tz = __fmul_rn(s.s0, l2);
      return __fadd_rn(__fmul_rn(l0, l0), __fmul_rn(l1, l1)) <= __fmul_rn(tz, tz);
    }
    case IND_PRISM:
      if (!(fabsf(l1) <= s.s1 && l2 >= 0.f && l2 <= s.s2)) return false;
      return fabsf(l0) <= __fmul_rn(s.s0, l2);
    case IND_HEIGHTMAP: {
      const int w = s.hm_w, h = s.hm_h;
      float fx = __fadd_rn(__fmul_rn(l0, s.inv_pix), s.offx);
      float fy = __fadd_rn(__fmul_rn(l1, s.inv_pix), s.offy);
      if (fx < -0.5f || fx > __fsub_rn((float)w, 0.5f) || fy < -0.5f || fy > __fsub_rn((float)h, 0.5f))
        return false;
      float cx = fx < 0.f ? 0.f : (fx > (float)(w - 1) ? (float)(w - 1) : fx);
      float cy = fy < 0.f ? 0.f : (fy > (float)(h - 1) ? (float)(h - 1) : fy);
      int ix = (int)floorf(cx), iy = (int)floorf(cy);
      ix = ix > w - 2 ? w - 2 : ix;
      iy = iy > h - 2 ? h - 2 : iy;
      float tx = __fsub_rn(cx, (float)ix), ty = __fsub_rn(cy, (float)iy);
      float ux = __fsub_rn(1.0f, tx), uy = __fsub_rn(1.0f, ty);
      const float *H = s.hm;
      float r0 = __fadd_rn(__fmul_rn(__ldg(H + iy * w + ix), ux), __fmul_rn(__ldg(H + iy * w + ix + 1), tx));
      float r1 = __fadd_rn(__fmul_rn(__ldg(H + (iy + 1) * w + ix), ux),
                           __fmul_rn(__ldg(H + (iy + 1) * w + ix + 1), tx));
      float hh = __fadd_rn(__fmul_rn(r0, uy), __fmul_rn(r1, ty));
      return l2 >= -hh && l2 <= s.s0;
    }
    default:
      return false;
  }
}

// Outward unit normal (world frame) of the indenter's contact surface at a
// grid node inside it, for the slip contact mode (reading of Sec. III-A: the
// paper's indenter is no-slip; slip removes only the relative velocity into
// the indenter).  Sphere: radial from the centre.  Cylinder: radial from the
// axis (local x).  Cone and prism: the lateral face the node lies under,
// (rho_hat, -t) / sqrt(1 + t^2) with t the tangent of the half angle.
// Height map: the protruding surface z_l = -h(x_l, y_l), normal (-h_x, -h_y,
// -1) / |.| from the gradient of the bilinear interpolant.  Where the normal
// is undefined (on an axis or edge) it is the indenter's -z_l direction.
__device__ __forceinline__ void indenter_normal(const IndenterShape &s, const IndenterFrame &f, int i, int j,
                                                int k, float n[3]) {
  const float d0 = (float)i - f.c[0], d1 = (float)j - f.c[1], d2 = (float)k - f.c[2];
  if (s.kind == IND_SPHERE) {
    const float q = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    if (q > 0.f) {
      n[0] = d0 / q; n[1] = d1 / q; n[2] = d2 / q;
    } else {
      n[0] = -f.r[2]; n[1] = -f.r[5]; n[2] = -f.r[8];
    }
    return;
  }
  const float l0 = f.r[0] * d0 + f.r[3] * d1 + f.r[6] * d2;
  const float l1 = f.r[1] * d0 + f.r[4] * d1 + f.r[7] * d2;
  const float l2 = f.r[2] * d0 + f.r[5] * d1 + f.r[8] * d2;
  float m0 = 0.f, m1 = 0.f, m2 = -1.f;  // local normal
  if (s.kind == IND_CYLINDER) {
    const float q = sqrtf(l1 * l1 + l2 * l2);
    if (q > 0.f) { m0 = 0.f; m1 = l1 / q; m2 = l2 / q; }
  } else if (s.kind == IND_CONE) {
    const float q = sqrtf(l0 * l0 + l1 * l1), t = s.s0, c = rsqrtf(1.f + t * t);
    if (q > 0.f) { m0 = l0 / q * c; m1 = l1 / q * c; m2 = -t * c; }
  } else if (s.kind == IND_PRISM) {
    const float t = s.s0, c = rsqrtf(1.f + t * t);
    if (l0 != 0.f) { m0 = (l0 > 0.f ? 1.f : -1.f) * c; m1 = 0.f; m2 = -t * c; }
  } else if (s.kind == IND_HEIGHTMAP) {
    const int w = s.hm_w, h = s.hm_h;
    const float fx = l0 * s.inv_pix + s.offx, fy = l1 * s.inv_pix + s.offy;
    const float cx = fminf(fmaxf(fx, 0.f), (float)(w - 1)), cy = fminf(fmaxf(fy, 0.f), (float)(h - 1));
    const int ix = min((int)floorf(cx), w - 2), iy = min((int)floorf(cy), h - 2);
    const float tx = cx - (float)ix, ty = cy - (float)iy;
    const float *H = s.hm;
    const float h00 = __ldg(H + iy * w + ix), h01 = __ldg(H + iy * w + ix + 1);
    const float h10 = __ldg(H + (iy + 1) * w + ix), h11 = __ldg(H + (iy + 1) * w + ix + 1);
    // gradient in cells per cell (zero where the sample point is clamped)
    const float gx = (fx > 0.f && fx < (float)(w - 1)) ? ((h01 - h00) * (1.f - ty) + (h11 - h10) * ty) * s.inv_pix : 0.f;
    const float gy = (fy > 0.f && fy < (float)(h - 1)) ? ((h10 - h00) * (1.f - tx) + (h11 - h01) * tx) * s.inv_pix : 0.f;
    const float c = rsqrtf(1.f + gx * gx + gy * gy);
    m0 = -gx * c; m1 = -gy * c; m2 = -c;
  }
  n[0] = f.r[0] * m0 + f.r[1] * m1 + f.r[2] * m2;
  n[1] = f.r[3] * m0 + f.r[4] * m1 + f.r[5] * m2;
  n[2] = f.r[6] * m0 + f.r[7] * m1 + f.r[8] * m2;
}

// Launchers implemented in mpm.cu / render.cu (host side).
// Transfer plan: the sort block in cells and the threads that share a cell
// in the transfer kernel (1: k_transfer, mpm.cu; 3: k_transfer3,
// transfer3.cu).
struct SortBlock {
  int x, y, z;
  int t = 1;
};
cudaError_t launch_grid_update(const Batch &b, int substep, float dt, int clear, cudaStream_t st);
cudaError_t launch_transfer(const Batch &b, SortBlock blk, int mode, float dt, cudaStream_t st);
// The pipelined fused transfer (a persistent grid of grid CTAs over the
// sort's block records; see mpm.cu), for the plans pipe_supported accepts.
bool pipe_supported(SortBlock blk);
cudaError_t prepare_pipe(SortBlock blk, int *grid);
cudaError_t launch_transfer_pipe(const Batch &b, SortBlock blk, float dt, int grid, long long max_polls, int extra,
                                 cudaStream_t st);
cudaError_t launch_sort(const Batch &b, SortBlock blk, int force, cudaStream_t st);
cudaError_t prepare_transfer(SortBlock blk);

// Control words of the persistent step (device memory, cleared before each
// launch) and its waiting policy.
struct PersistCtl {
  unsigned *bar;        // [0] arrivals at the current grid barrier, [1] its generation,
                        // [3] the next sort block of the running transfer phase
  int *abort;           // set by a CTA that gave up waiting; every CTA then returns
  long long max_polls;  // polls of a barrier before giving up (ERRBIT_TIMEOUT)
  unsigned extra;       // arrivals a barrier waits for beyond the grid: 0, except to
                        // exercise the bounded wait (they never come)
};
bool persistent_supported(SortBlock blk);
// Opts the persistent kernel into its shared memory and returns the number
// of CTAs that can be co-resident on the device (the cooperative grid).
cudaError_t prepare_persistent(SortBlock blk, int *grid);
cudaError_t launch_persistent(const Batch &b, SortBlock blk, int n, float dt, const PersistCtl &ctl, int grid,
                              cudaStream_t st);
bool transfer3_supported(SortBlock blk);
cudaError_t prepare_transfer3(SortBlock blk);
cudaError_t launch_transfer3(const Batch &b, SortBlock blk, int mode, float dt, cudaStream_t st);
// P2G of the indenter particles of every instance at the frame of `substep`.
cudaError_t launch_indenter_p2g(const Batch &b, int substep, cudaStream_t st);
// Particles [o, o + n) of the records from / to structure-of-arrays u [3][n]
// and Fm [9][n] (F - I); a null Fm packs F = I, a null output is skipped.
cudaError_t launch_pack_state(float4 *ps, long long o, long long n, const float *u, const float *Fm,
                              cudaStream_t st);
cudaError_t launch_unpack_state(const float4 *ps, long long o, long long n, float *u, float *Fm, cudaStream_t st);

enum : int { XFER_P2G = 1, XFER_G2P = 2, XFER_FUSED = 3 };

// Largest hole-fill radius (pixels) of a height map, for every entry point.
constexpr int kMaxFillRadius = 64;

struct HeightmapArgs {
  const float4 *ps;       // particle records [Ntot][3], or null: then
  const float *u;         // particle positions [3][Ntot] (caller's arrays)
  long long Ntot;
  const uint32_t *surf;   // [Ns] global particle ids of top-layer particles
  const float *z0;        // [Ns] rest z (cells)
  int Ns;
  float A0X, A0Y, SX, SY; // pixel (r, c) centre = (c*SX + A0X, r*SY + A0Y) in cells
  float z_top, dx;        // m
  int w, h, fill_radius;
  int *cov;               // [h*w] scratch, ordered-int heights
  float *out;             // [h*w] metres
};
cudaError_t launch_heightmap(const HeightmapArgs &a, cudaStream_t st);

// Top-surface displacement sampled per pixel: the top-layer particle whose
// rest sub-cell contains the pixel centre (lattice index (i, j) -> surface
// index ((j/2) nx + i/2) 4 + (j%2) 2 + i%2).
struct DispMapArgs {
  const float4 *ps;        // particle records [Ntot][3] (positions in cells)
  long long Ntot;
  const uint32_t *surf;    // [Ns] particle ids of the instance's surface list
  const float *rest;       // [3][Ns_tot] rest positions (cells), instance slice
  long long rest_stride;   // Ns_tot
  int nx, ny;              // elastomer cells (the block's corner is world (0, 0))
  float X0, Y0, PW, PH;    // pixel (r, c) centre = (X0 + c PW, Y0 + r PH), metres
  const float *xy;         // or, when set, point e = (xy[2e], xy[2e + 1]) (markers), h = 1
  float dx;
  int w, h;
  float *out;              // [h][w][3] metres
};
cudaError_t launch_dispmap(const DispMapArgs &a, cudaStream_t st);

// Penetration of a yaw-only posed indenter into the rest top face.
struct PenMapArgs {
  int kind;
  float p0, p1, p2;        // shape parameters (metres, radians)
  float cx, cy, cz;        // pose position (metres, world)
  float cosy, siny;        // yaw
  const float *hm;         // heightmap in cells (device), or null
  int hm_w, hm_h;
  float hm_pix, dx;        // metres
  float z_top;
  float X0, Y0, PW, PH;
  int w, h;
  float *out;              // [h][w] metres
};
cudaError_t launch_penmap(const PenMapArgs &a, cudaStream_t st);

// Gaussian-smoothed penetration map (the depth-smoothing renderers of
// Sec. II): rows pass over the window extended by ry rows above and below
// (penetration evaluated from the shape, also beyond the window) into tmp
// [h + 2 ry][w], then the columns pass into H = z_top - s [h][w].
constexpr int kMaxSmoothRadius = 256;
struct SmoothArgs {
  PenMapArgs pen;          // pen.out unused
  int rx, ry;              // kernel half widths (pixels)
  float gx[kMaxSmoothRadius + 1], gy[kMaxSmoothRadius + 1];  // g(0..R), symmetric
  float *tmp;              // [h + 2 ry][w]
  float *H;                // [h][w] metres
};
cudaError_t launch_smoothed(const SmoothArgs &a, cudaStream_t st);

struct ShadeArgs {
  int n_lights;
  float dir[8][3], dif[8][3], spe[8][3], amb[3];
  float ka, kd, ks, alpha;
  float inv2px, inv2py, z_top;
  int w, h;
};
cudaError_t launch_shade(const ShadeArgs &a, const float *H, float *rgb, cudaStream_t st);

}  // namespace tacchi
