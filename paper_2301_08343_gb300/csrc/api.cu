// api.cu -- host implementation of the C ABI declared in include/tacchi.h.
//
// One tacchi_ctx owns one elastomer instance laid out as a batch of one (the
// batched entry points reuse the same kernels over many instances).  A
// tacchi_step of n substeps is queued as one CUDA graph:
//   clear grid -> P2G -> [grid update(k) -> fused G2P+P2G -> sort?] x (n-1)
//   -> grid update(n-1) -> G2P -> sort?
// The indenter's per-substep FP32 frames are computed on the host in FP64
// and uploaded before each graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tacchi.h"
#include "tacchi_internal.cuh"

using namespace tacchi;

namespace {

constexpr int kMaxChunk = 512;      // substeps per captured graph
constexpr int kMaxGraphs = 8;       // cached (n, dt) graphs per context
constexpr int kMaxFillRadius = 64;

bool finite3(const double *a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// splitmix64, counter form: output k mixes seed + (k + 1) * golden gamma
// (Steele, Lea & Flood, OOPSLA 2014).
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
inline double uniform01(uint64_t seed, uint64_t k) {
  const uint64_t r = mix64(seed + (k + 1ull) * 0x9E3779B97F4A7C15ull);
  return (double)(r >> 11) * 0x1.0p-53;
}

// Particle lattice: particle p = cell * 8 + sub, cells ordered z, y, x;
// sub = sz * 4 + sy * 2 + sx; axis a at (cell + (sub_a + U) / 2) cells.
void make_lattice(int nx, int ny, int nz, int pad_side, int pad_bottom, uint64_t seed, int jitter,
                  float *u, uint8_t *flags) {
  const long long N = 8ll * nx * ny * nz;
  for (long long cell = 0; cell < (long long)nx * ny * nz; ++cell) {
    const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((long long)nx * ny));
    const int org[3] = {cx + pad_side, cy + pad_side, cz + pad_bottom};
    for (int sub = 0; sub < 8; ++sub) {
      const long long p = cell * 8 + sub;
      const int sa[3] = {sub & 1, (sub >> 1) & 1, (sub >> 2) & 1};
      for (int a = 0; a < 3; ++a) {
        const double U = jitter ? uniform01(seed, (uint64_t)(3 * p + a)) : 0.5;
        const double off = ((double)sa[a] + U) * 0.5;
        u[a * N + p] = (float)((double)org[a] + off);
      }
      flags[p] = (uint8_t)((cz == 0 ? 1 : 0) | (cz == nz - 1 && sa[2] == 1 ? 2 : 0));
    }
  }
}

// Block shapes the transfer kernel is instantiated for.
bool block_supported(SortBlock b) {
  return (b.x == 8 && b.y == 8 && b.z == 4) || (b.x == 4 && b.y == 4 && b.z == 4) ||
         (b.x == 8 && b.y == 8 && b.z == 8) || (b.x == 16 && b.y == 8 && b.z == 4);
}

tacchi_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TACCHI_OK : TACCHI_ERR_CUDA; }

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

}  // namespace

// Timing events of one kernel (or kernel group) inside a captured graph.
struct TimedSpan {
  int kind;  // 0 grid, 1 fused, 2 edge transfer, 3 sort
  cudaEvent_t a, b;
};

struct GraphEntry {
  int n = 0;
  float dt = 0.f;
  bool profiled = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<TimedSpan> spans;
};

struct tacchi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap = nullptr;

  // geometry (host, FP64)
  int nx = 0, ny = 0, nz = 0, pad_side = 0, pad_bottom = 0, pad_top = 0;
  int G[3] = {0, 0, 0};
  double dx = 0, origin[3] = {0, 0, 0}, z_top = 0;
  long long N = 0, nodes = 0;
  SortBlock blk{8, 8, 4};
  long long nblocks = 0;

  Instance inst{};  // host mirror
  Batch b{};        // device pointers

  // device buffers
  Instance *d_inst = nullptr;
  long long *d_offs = nullptr;  // [2]: node offset, particle offset (one instance)
  uint32_t *d_block_inst = nullptr;
  IndenterFrame *d_frames = nullptr;
  float *d_hm = nullptr;
  uint32_t *d_surf = nullptr;
  float *d_z0 = nullptr;
  int Ns = 0;
  int *d_cov = nullptr;
  size_t cov_cap = 0;
  float *d_hbuf = nullptr;
  size_t hbuf_cap = 0;
  float *d_rgb = nullptr;
  size_t rgb_cap = 0;

  // host staging for the per-step upload (pinned)
  struct Stage {
    Instance inst;
    IndenterFrame frames[kMaxChunk];
  } *h_stage = nullptr;
  cudaEvent_t stage_done = nullptr;
  int *h_err = nullptr;

  // indenter (host, FP64)
  int ind_kind = IND_NONE;
  double ind_params[8] = {0};
  int hm_w = 0, hm_h = 0;
  double hm_pixel = 0;
  double pose[7] = {0, 0, 0, 1, 0, 0, 0};
  double vel[6] = {0, 0, 0, 0, 0, 0};

  std::vector<GraphEntry> graphs;
  bool profiling = false;
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_n[4] = {0, 0, 0, 0};
  bool stepped = false;
  size_t device_bytes = 0;
};

namespace {

template <typename T>
cudaError_t dalloc(tacchi_ctx *c, T **p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e == cudaSuccess) c->device_bytes += bytes;
  return e;
}

// Shape constants of the inside test in cells, FP32 (rounded from FP64).
IndenterShape make_shape(const tacchi_ctx *c) {
  IndenterShape s{};
  s.kind = c->ind_kind;
  const double dx = c->dx;
  const double *P = c->ind_params;
  switch (c->ind_kind) {
    case IND_SPHERE:
      s.s0 = (float)((P[0] / dx) * (P[0] / dx));
      break;
    case IND_CYLINDER:
      s.s0 = (float)((P[0] / dx) * (P[0] / dx));
      s.s1 = (float)(P[1] / dx);
      break;
    case IND_CONE:
      s.s0 = (float)std::tan(P[0]);
      s.s1 = (float)(P[1] / dx);
      break;
    case IND_PRISM:
      s.s0 = (float)std::tan(P[0]);
      s.s1 = (float)(P[1] / dx);
      s.s2 = (float)(P[2] / dx);
      break;
    case IND_HEIGHTMAP:
      s.s0 = (float)(P[0] / dx);
      s.inv_pix = (float)(dx / c->hm_pixel);
      s.offx = (float)(c->hm_w * 0.5 - 0.5);
      s.offy = (float)(c->hm_h * 0.5 - 0.5);
      s.hm_w = c->hm_w;
      s.hm_h = c->hm_h;
      s.hm = c->d_hm;
      break;
    default:
      break;
  }
  return s;
}

// Local-to-world rotation of a (not necessarily unit) quaternion (w,x,y,z).
void rotation_of(const double *q, double R[9]) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
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

IndenterFrame frame_of(const tacchi_ctx *c, const double *pose, const double *vel) {
  IndenterFrame f{};
  for (int a = 0; a < 3; ++a) f.c[a] = (float)((pose[a] - c->origin[a]) / c->dx);
  double R[9];
  rotation_of(pose + 3, R);
  for (int e = 0; e < 9; ++e) f.r[e] = (float)R[e];
  for (int a = 0; a < 3; ++a) {
    f.vlin[a] = (float)vel[a];
    f.w[a] = (float)vel[3 + a];
  }
  return f;
}

// Rigid motion over one substep: position += dt v; orientation turned by the
// angle |w| dt about w (quaternion product on the left), renormalised.
void advance_pose(double *pose, const double *vel, double dt) {
  for (int a = 0; a < 3; ++a) pose[a] += dt * vel[a];
  const double wx = vel[3], wy = vel[4], wz = vel[5];
  const double wn = std::sqrt(wx * wx + wy * wy + wz * wz);
  if (wn > 0.0) {
    const double half = 0.5 * wn * dt;
    const double cw = std::cos(half), sw = std::sin(half) / wn;
    const double r0 = cw, r1 = sw * wx, r2 = sw * wy, r3 = sw * wz;
    double *q = pose + 3;
    const double n0 = r0 * q[0] - r1 * q[1] - r2 * q[2] - r3 * q[3];
    const double n1 = r0 * q[1] + r1 * q[0] + r2 * q[3] - r3 * q[2];
    const double n2 = r0 * q[2] - r1 * q[3] + r2 * q[0] + r3 * q[1];
    const double n3 = r0 * q[3] + r1 * q[2] - r2 * q[1] + r3 * q[0];
    const double nn = std::sqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
    q[0] = n0 / nn;
    q[1] = n1 / nn;
    q[2] = n2 / nn;
    q[3] = n3 / nn;
  }
}

void destroy_entry(GraphEntry &ge) {
  if (ge.exec) cudaGraphExecDestroy(ge.exec);
  for (auto &sp : ge.spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  ge.spans.clear();
  ge.exec = nullptr;
}

// Enqueue one kernel (group) on the capture stream, bracketed by timing
// events when the graph is built for profiling.
template <typename F>
cudaError_t timed(tacchi_ctx *c, GraphEntry *ge, int kind, F &&launch) {
  if (!ge) return launch();
  TimedSpan sp{kind, nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&sp.a);
  if (e == cudaSuccess) e = cudaEventCreate(&sp.b);
  if (e != cudaSuccess) return e;
  ge->spans.push_back(sp);
  // external record nodes: the events are really recorded when the graph runs
  e = cudaEventRecordWithFlags(sp.a, c->cap, cudaEventRecordExternal);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(sp.b, c->cap, cudaEventRecordExternal);
  return e;
}

cudaError_t build_graph(tacchi_ctx *c, int n, float dt, GraphEntry *ge) {
  cudaGraph_t g = nullptr;
  GraphEntry *pe = ge->profiled ? ge : nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const Batch &b = c->b;
  const SortBlock blk = c->blk;
  cudaStream_t s = c->cap;
  cudaError_t le = cudaMemsetAsync(b.gmm, 0, sizeof(float4) * c->nodes, s);
  if (le == cudaSuccess) le = timed(c, pe, 2, [&] { return launch_transfer(b, blk, XFER_P2G, dt, s); });
  for (int k = 0; k + 1 < n && le == cudaSuccess; ++k) {
    le = timed(c, pe, 0, [&] { return launch_grid_update(b, k, dt, 1, s); });
    if (le == cudaSuccess) le = timed(c, pe, 1, [&] { return launch_transfer(b, blk, XFER_FUSED, dt, s); });
    if (le == cudaSuccess) le = timed(c, pe, 3, [&] { return launch_sort(b, blk, 0, s); });
  }
  if (le == cudaSuccess) le = timed(c, pe, 0, [&] { return launch_grid_update(b, n - 1, dt, 0, s); });
  if (le == cudaSuccess) le = timed(c, pe, 2, [&] { return launch_transfer(b, blk, XFER_G2P, dt, s); });
  if (le == cudaSuccess) le = timed(c, pe, 3, [&] { return launch_sort(b, blk, 0, s); });
  e = cudaStreamEndCapture(c->cap, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&ge->exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

cudaError_t graph_for(tacchi_ctx *c, int n, float dt, GraphEntry **out) {
  for (auto &ge : c->graphs)
    if (ge.n == n && ge.dt == dt && ge.profiled == c->profiling) {
      *out = &ge;
      return cudaSuccess;
    }
  if ((int)c->graphs.size() >= kMaxGraphs) {
    destroy_entry(c->graphs.front());
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back(GraphEntry{});
  GraphEntry &ge = c->graphs.back();
  ge.n = n;
  ge.dt = dt;
  ge.profiled = c->profiling;
  cudaError_t e = build_graph(c, n, dt, &ge);
  if (e != cudaSuccess) {
    destroy_entry(ge);
    c->graphs.pop_back();
    return e;
  }
  *out = &ge;
  return cudaSuccess;
}

cudaError_t collect_profile(tacchi_ctx *c, GraphEntry *ge) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  for (auto &sp : ge->spans) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, sp.a, sp.b);
    if (e != cudaSuccess) return e;
    c->prof_ms[sp.kind] += ms;
    c->prof_n[sp.kind] += 1;
  }
  return cudaSuccess;
}

tacchi_status error_from_bits(int bits) {
  if (bits & ERRBIT_NUMERICAL) return TACCHI_ERR_NUMERICAL;
  if (bits & ERRBIT_OUT_OF_GRID) return TACCHI_ERR_OUT_OF_GRID;
  if (bits & ERRBIT_CFL) return TACCHI_ERR_CFL;
  if (bits & ERRBIT_TIMEOUT) return TACCHI_ERR_TIMEOUT;
  return TACCHI_OK;
}

tacchi_status sync_and_check(tacchi_ctx *c) {
  CK(cudaMemcpyAsync(c->h_err, c->b.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return error_from_bits(*c->h_err);
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t ensure(tacchi_ctx *c, T **p, size_t *cap, size_t count) {
  if (*cap >= count) return cudaSuccess;
  if (*p) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    cudaFree(*p);
    c->device_bytes -= *cap * sizeof(T);
    *p = nullptr;
    *cap = 0;
  }
  cudaError_t e = dalloc(c, p, count);
  if (e == cudaSuccess) *cap = count;
  return e;
}

tacchi_status validate_window(int w, int h, const double *win, int fill_radius) {
  if (w < 1 || h < 1 || !win || !finite3(win, 4)) return TACCHI_ERR_INVALID_ARG;
  if (!(win[2] > win[0]) || !(win[3] > win[1])) return TACCHI_ERR_INVALID_ARG;
  if (fill_radius < 0 || fill_radius > kMaxFillRadius) return TACCHI_ERR_INVALID_ARG;
  if ((long long)w * h > (1ll << 28)) return TACCHI_ERR_INVALID_ARG;
  return TACCHI_OK;
}

tacchi_status run_heightmap(tacchi_ctx *c, int w, int h, const double *win, int fill_radius, float *dev_out) {
  CK(ensure(c, &c->d_cov, &c->cov_cap, (size_t)w * h));
  HeightmapArgs a{};
  a.u = c->b.u;
  a.Ntot = c->N;
  a.surf = c->d_surf;
  a.z0 = c->d_z0;
  a.Ns = c->Ns;
  const double pxc = ((win[2] - win[0]) / (double)w) / c->dx;
  const double pyc = ((win[3] - win[1]) / (double)h) / c->dx;
  a.A0X = (float)((win[0] - c->origin[0]) / c->dx + 0.5 * pxc);
  a.A0Y = (float)((win[1] - c->origin[1]) / c->dx + 0.5 * pyc);
  a.SX = (float)pxc;
  a.SY = (float)pyc;
  if (!(a.SX > 0.f) || !(a.SY > 0.f)) return TACCHI_ERR_INVALID_ARG;
  a.z_top = (float)c->z_top;
  a.dx = (float)c->dx;
  a.w = w;
  a.h = h;
  a.fill_radius = fill_radius;
  a.cov = c->d_cov;
  a.out = dev_out;
  CK(launch_heightmap(a, c->stream));
  return TACCHI_OK;
}

tacchi_status fill_shade_args(const tacchi_render_params *rp, int w, int h, double px, double py,
                              double z_top, ShadeArgs *a) {
  if (!rp || rp->n_lights < 0 || rp->n_lights > 8) return TACCHI_ERR_INVALID_ARG;
  if (!(px > 0) || !(py > 0) || !std::isfinite(z_top) || w < 1 || h < 1) return TACCHI_ERR_INVALID_ARG;
  *a = ShadeArgs{};
  a->n_lights = rp->n_lights;
  for (int m = 0; m < 8; ++m)
    for (int k = 0; k < 3; ++k) {
      a->dir[m][k] = rp->dir[m][k];
      a->dif[m][k] = rp->diffuse[m][k];
      a->spe[m][k] = rp->specular[m][k];
    }
  for (int k = 0; k < 3; ++k) a->amb[k] = rp->ambient[k];
  a->ka = rp->ka;
  a->kd = rp->kd;
  a->ks = rp->ks;
  a->alpha = rp->alpha;
  a->inv2px = (float)(1.0 / (2.0 * px));
  a->inv2py = (float)(1.0 / (2.0 * py));
  a->z_top = (float)z_top;
  a->w = w;
  a->h = h;
  return TACCHI_OK;
}

void release(tacchi_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto &g : c->graphs) destroy_entry(g);
  c->graphs.clear();
  void *bufs[] = {c->b.u, c->b.Fm, c->b.v, c->b.C, (void *)c->b.flags, c->b.idx, c->b.key, c->b.bstart,
                  c->b.bcount, c->b.cursor, c->b.gmm, c->b.gv, c->b.err, c->b.movers, c->d_inst, c->d_offs,
                  c->d_block_inst, c->d_frames, c->d_hm, c->d_surf, c->d_z0, c->d_cov, c->d_hbuf, c->d_rgb};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->stage_done) cudaEventDestroy(c->stage_done);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace

// ===========================================================================
extern "C" {

const char *tacchi_status_string(tacchi_status s) {
  switch (s) {
    case TACCHI_OK: return "ok";
    case TACCHI_ERR_INVALID_ARG: return "invalid argument";
    case TACCHI_ERR_OOM: return "out of memory";
    case TACCHI_ERR_CUDA: return "CUDA runtime error";
    case TACCHI_ERR_NUMERICAL: return "numerical failure (NaN/Inf or det F <= 0)";
    case TACCHI_ERR_OUT_OF_GRID: return "a particle reached the grid's padding band";
    case TACCHI_ERR_TIMEOUT: return "a bounded device wait timed out";
    case TACCHI_ERR_STATE: return "call not valid in the current state";
    case TACCHI_ERR_CFL: return "a particle moved a cell or more in one substep";
  }
  return "unknown status";
}

int tacchi_version(void) { return 100; }

tacchi_status tacchi_init_lattice(int nx, int ny, int nz, int pad_side, int pad_bottom, uint64_t seed,
                                  int jitter, float *u, uint8_t *flags) {
  if (nx < 1 || ny < 1 || nz < 1 || pad_side < 0 || pad_bottom < 0 || !u || !flags)
    return TACCHI_ERR_INVALID_ARG;
  if (8.0 * nx * ny * nz > 2.0e9) return TACCHI_ERR_INVALID_ARG;
  make_lattice(nx, ny, nz, pad_side, pad_bottom, seed, jitter, u, flags);
  return TACCHI_OK;
}

tacchi_status tacchi_create(const tacchi_elastomer_desc *d, void *stream, tacchi_handle *out) {
  if (!d || !out) return TACCHI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(d->dx_m > 0) || !std::isfinite(d->dx_m) || !finite3(d->extent_m, 3) || !finite3(d->gravity, 3))
    return TACCHI_ERR_INVALID_ARG;
  if (!(d->E_pa > 0) || !(d->nu > -1.0 && d->nu < 0.5) || !(d->density > 0) || !std::isfinite(d->E_pa) ||
      !std::isfinite(d->density))
    return TACCHI_ERR_INVALID_ARG;
  int n[3];
  for (int a = 0; a < 3; ++a) {
    const double r = d->extent_m[a] / d->dx_m;
    n[a] = (int)std::llround(r);
    if (n[a] < 1 || std::fabs(r - n[a]) > 1e-6 * std::max(1.0, r)) return TACCHI_ERR_INVALID_ARG;
  }
  const int ps = d->pad_side ? d->pad_side : 4;
  const int pb = d->pad_bottom ? d->pad_bottom : 3;
  const int pt = d->pad_top ? d->pad_top : 4;
  if (ps < 3 || pb < 3 || pt < 3) return TACCHI_ERR_INVALID_ARG;
  const double Nd = 8.0 * n[0] * n[1] * n[2];
  if (Nd > 2.0e9) return TACCHI_ERR_INVALID_ARG;
  const bool user_block = d->block[0] != 0 || d->block[1] != 0 || d->block[2] != 0;
  if (user_block && !block_supported(SortBlock{d->block[0], d->block[1], d->block[2]}))
    return TACCHI_ERR_INVALID_ARG;

  tacchi_ctx *c = new (std::nothrow) tacchi_ctx();
  if (!c) return TACCHI_ERR_OOM;
  auto fail = [&](tacchi_status s) {
    release(c);
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(TACCHI_ERR_CUDA);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&c->stream) != cudaSuccess) return fail(TACCHI_ERR_CUDA);
    c->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(TACCHI_ERR_CUDA);
  if (cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming) != cudaSuccess)
    return fail(TACCHI_ERR_CUDA);

  c->nx = n[0];
  c->ny = n[1];
  c->nz = n[2];
  c->pad_side = ps;
  c->pad_bottom = pb;
  c->pad_top = pt;
  c->G[0] = n[0] + 2 * ps + 1;
  c->G[1] = n[1] + 2 * ps + 1;
  c->G[2] = n[2] + pb + pt + 1;
  c->dx = d->dx_m;
  c->origin[0] = -ps * d->dx_m;
  c->origin[1] = -ps * d->dx_m;
  c->origin[2] = -pb * d->dx_m;
  c->z_top = n[2] * d->dx_m;
  c->N = (long long)Nd;
  c->nodes = (long long)c->G[0] * c->G[1] * c->G[2];
  if (user_block) {
    c->blk = SortBlock{d->block[0], d->block[1], d->block[2]};
  } else {
    c->blk = c->N < 2000000 ? SortBlock{4, 4, 4} : SortBlock{8, 8, 4};
  }
  int nb[3] = {(c->G[0] + c->blk.x - 1) / c->blk.x, (c->G[1] + c->blk.y - 1) / c->blk.y,
               (c->G[2] + c->blk.z - 1) / c->blk.z};
  c->nblocks = (long long)nb[0] * nb[1] * nb[2];

  // instance constants
  Instance &I = c->inst;
  for (int a = 0; a < 3; ++a) {
    I.G[a] = c->G[a];
    I.nb[a] = nb[a];
    I.gdt[a] = (float)d->gravity[a];
  }
  I.pad_bottom = pb;
  I.fix_base = d->free_base ? 0 : 1;
  I.node_off = 0;
  I.N = c->N;
  I.part_off = 0;
  I.block_off = 0;
  I.nblocks = c->nblocks;
  const double V0 = d->dx_m * d->dx_m * d->dx_m / 8.0;
  I.dx = (float)d->dx_m;
  I.inv_dx = (float)(1.0 / d->dx_m);
  I.m = (float)(d->density * V0);
  I.V0 = (float)V0;
  I.mu = (float)(d->E_pa / (2.0 * (1.0 + d->nu)));
  I.la = (float)(d->E_pa * d->nu / ((1.0 + d->nu) * (1.0 - 2.0 * d->nu)));
  I.shape = IndenterShape{};

  const long long N = c->N, Nn = c->nodes;
  bool ok = dalloc(c, &c->b.u, 3 * N) == cudaSuccess && dalloc(c, &c->b.Fm, 9 * N) == cudaSuccess &&
            dalloc(c, &c->b.v, 3 * N) == cudaSuccess && dalloc(c, &c->b.C, 9 * N) == cudaSuccess &&
            dalloc(c, (uint8_t **)&c->b.flags, N) == cudaSuccess && dalloc(c, &c->b.idx, N) == cudaSuccess &&
            dalloc(c, &c->b.key, N) == cudaSuccess && dalloc(c, &c->b.bstart, c->nblocks + 1) == cudaSuccess &&
            dalloc(c, &c->b.bcount, c->nblocks) == cudaSuccess &&
            dalloc(c, &c->b.cursor, c->nblocks) == cudaSuccess && dalloc(c, &c->b.gmm, Nn) == cudaSuccess &&
            dalloc(c, &c->b.gv, Nn) == cudaSuccess && dalloc(c, &c->b.err, 1) == cudaSuccess &&
            dalloc(c, &c->b.movers, 1) == cudaSuccess && dalloc(c, &c->d_inst, 1) == cudaSuccess &&
            dalloc(c, &c->d_offs, 2) == cudaSuccess && dalloc(c, &c->d_block_inst, c->nblocks) == cudaSuccess &&
            dalloc(c, &c->d_frames, kMaxChunk) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return fail(TACCHI_ERR_OOM);
  }
  if (cudaMallocHost((void **)&c->h_stage, sizeof(tacchi_ctx::Stage)) != cudaSuccess ||
      cudaMallocHost((void **)&c->h_err, sizeof(int)) != cudaSuccess)
    return fail(TACCHI_ERR_OOM);
  *c->h_err = 0;
  I.frames = c->d_frames;

  // initial particles (Eq. 1): lattice positions, v = 0, C = 0, F = I
  std::vector<float> hu;
  std::vector<uint8_t> hf;
  try {
    hu.resize(3 * N);
    hf.resize(N);
  } catch (...) {
    return fail(TACCHI_ERR_OOM);
  }
  make_lattice(n[0], n[1], n[2], ps, pb, d->seed, d->jitter, hu.data(), hf.data());
  std::vector<uint32_t> surf;
  std::vector<float> z0;
  for (long long p = 0; p < N; ++p)
    if (hf[p] & 2) {
      surf.push_back((uint32_t)p);
      z0.push_back(hu[2 * N + p]);
    }
  c->Ns = (int)surf.size();
  if (dalloc(c, &c->d_surf, surf.size()) != cudaSuccess || dalloc(c, &c->d_z0, z0.size()) != cudaSuccess)
    return fail(TACCHI_ERR_OOM);

  c->b.inst = c->d_inst;
  c->b.node_offs = c->d_offs;
  c->b.part_offs = c->d_offs + 1;
  c->b.block_inst = c->d_block_inst;
  c->b.n_inst = 1;
  c->b.Ntot = N;
  c->b.Nnodes = Nn;
  c->b.Nblk = c->nblocks;

  const long long zero2[2] = {0, 0};
  cudaStream_t st = c->stream;
  bool up = cudaMemcpy(c->b.u, hu.data(), sizeof(float) * 3 * N, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy((void *)c->b.flags, hf.data(), N, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->d_surf, surf.data(), sizeof(uint32_t) * surf.size(), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(c->d_z0, z0.data(), sizeof(float) * z0.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->d_offs, zero2, sizeof(zero2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->d_inst, &c->inst, sizeof(Instance), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemsetAsync(c->b.Fm, 0, sizeof(float) * 9 * N, st) == cudaSuccess &&
            cudaMemsetAsync(c->b.v, 0, sizeof(float) * 3 * N, st) == cudaSuccess &&
            cudaMemsetAsync(c->b.C, 0, sizeof(float) * 9 * N, st) == cudaSuccess &&
            cudaMemsetAsync(c->d_block_inst, 0, sizeof(uint32_t) * c->nblocks, st) == cudaSuccess &&
            cudaMemsetAsync(c->b.bcount, 0, sizeof(uint32_t) * c->nblocks, st) == cudaSuccess &&
            cudaMemsetAsync(c->b.gmm, 0, sizeof(float4) * Nn, st) == cudaSuccess &&
            cudaMemsetAsync(c->b.gv, 0, sizeof(float4) * Nn, st) == cudaSuccess &&
            cudaMemsetAsync(c->b.err, 0, sizeof(int), st) == cudaSuccess &&
            cudaMemsetAsync(c->b.movers, 0, sizeof(int), st) == cudaSuccess &&
            prepare_transfer(c->blk) == cudaSuccess && launch_sort(c->b, c->blk, 1, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess;
  if (!up) {
    cudaGetLastError();
    return fail(TACCHI_ERR_CUDA);
  }
  *out = c;
  return TACCHI_OK;
}

void tacchi_destroy(tacchi_handle h) { release(h); }

tacchi_status tacchi_info(tacchi_handle c, tacchi_info_t *o) {
  if (!c || !o) return TACCHI_ERR_INVALID_ARG;
  o->n_particles = c->N;
  o->n_surface = c->Ns;
  for (int a = 0; a < 3; ++a) {
    o->grid[a] = c->G[a];
    o->origin_m[a] = c->origin[a];
  }
  o->n_nodes = c->nodes;
  o->dx_m = c->dx;
  o->z_top_m = c->z_top;
  o->block[0] = c->blk.x;
  o->block[1] = c->blk.y;
  o->block[2] = c->blk.z;
  o->n_blocks = c->nblocks;
  o->device_bytes = c->device_bytes;
  return TACCHI_OK;
}

tacchi_status tacchi_set_indenter(tacchi_handle c, const tacchi_indenter_desc *d, const double pose[7],
                                  const double vel[6]) {
  if (!c) return TACCHI_ERR_INVALID_ARG;
  if (pose && !finite3(pose, 7)) return TACCHI_ERR_INVALID_ARG;
  if (pose && !(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6] > 0))
    return TACCHI_ERR_INVALID_ARG;
  if (vel && !finite3(vel, 6)) return TACCHI_ERR_INVALID_ARG;
  if (d) {
    if (d->kind < IND_NONE || d->kind > IND_HEIGHTMAP || !finite3(d->params, 8)) return TACCHI_ERR_INVALID_ARG;
    const double *P = d->params;
    switch (d->kind) {
      case IND_SPHERE:
        if (!(P[0] > 0)) return TACCHI_ERR_INVALID_ARG;
        break;
      case IND_CYLINDER:
        if (!(P[0] > 0) || !(P[1] > 0)) return TACCHI_ERR_INVALID_ARG;
        break;
      case IND_CONE:
        if (!(P[0] > 0 && P[0] < 1.5707963267948966) || !(P[1] > 0)) return TACCHI_ERR_INVALID_ARG;
        break;
      case IND_PRISM:
        if (!(P[0] > 0 && P[0] < 1.5707963267948966) || !(P[1] > 0) || !(P[2] > 0)) return TACCHI_ERR_INVALID_ARG;
        break;
      case IND_HEIGHTMAP: {
        if (d->hm_w < 2 || d->hm_h < 2 || !d->hm || !(d->hm_pixel_m > 0) || !(P[0] >= 0))
          return TACCHI_ERR_INVALID_ARG;
        if ((long long)d->hm_w * d->hm_h > (1ll << 26)) return TACCHI_ERR_INVALID_ARG;
        const long long n = (long long)d->hm_w * d->hm_h;
        std::vector<float> cells(n);
        for (long long e = 0; e < n; ++e) {
          if (!std::isfinite(d->hm[e])) return TACCHI_ERR_INVALID_ARG;
          cells[e] = (float)((double)d->hm[e] / c->dx);
        }
        // queued work may still read the old map: free it in stream order
        if (c->d_hm) CK(cudaFreeAsync(c->d_hm, c->stream));
        c->d_hm = nullptr;
        CK(cudaMallocAsync((void **)&c->d_hm, sizeof(float) * n, c->stream));
        CK(cudaMemcpyAsync(c->d_hm, cells.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));  // host vector goes out of scope
        c->hm_w = d->hm_w;
        c->hm_h = d->hm_h;
        c->hm_pixel = d->hm_pixel_m;
        break;
      }
      default:
        break;
    }
    c->ind_kind = d->kind;
    for (int e = 0; e < 8; ++e) c->ind_params[e] = P[e];
  }
  if (pose)
    for (int e = 0; e < 7; ++e) c->pose[e] = pose[e];
  if (vel)
    for (int e = 0; e < 6; ++e) c->vel[e] = vel[e];
  return TACCHI_OK;
}

tacchi_status tacchi_get_indenter_pose(tacchi_handle c, double pose[7]) {
  if (!c || !pose) return TACCHI_ERR_INVALID_ARG;
  for (int e = 0; e < 7; ++e) pose[e] = c->pose[e];
  return TACCHI_OK;
}

tacchi_status tacchi_step(tacchi_handle c, int n_substeps, double dt) {
  if (!c || n_substeps < 1 || !(dt > 0) || !std::isfinite(dt)) return TACCHI_ERR_INVALID_ARG;
  const float fdt = (float)dt;
  int left = n_substeps;
  while (left > 0) {
    const int n = std::min(left, kMaxChunk);
    GraphEntry *ge = nullptr;
    CK(graph_for(c, n, fdt, &ge));
    // the previous upload must have left the pinned staging buffer
    CK(cudaEventSynchronize(c->stage_done));
    tacchi_ctx::Stage *s = c->h_stage;
    s->inst = c->inst;
    s->inst.shape = make_shape(c);
    s->inst.frames = c->d_frames;
    for (int k = 0; k < n; ++k) {
      s->frames[k] = frame_of(c, c->pose, c->vel);
      advance_pose(c->pose, c->vel, dt);
    }
    CK(cudaMemcpyAsync(c->d_inst, &s->inst, sizeof(Instance), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_frames, s->frames, sizeof(IndenterFrame) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecord(c->stage_done, c->stream));
    CK(cudaGraphLaunch(ge->exec, c->stream));
    if (ge->profiled) CK(collect_profile(c, ge));
    left -= n;
  }
  c->stepped = true;
  return TACCHI_OK;
}

tacchi_status tacchi_heightmap(tacchi_handle c, int w, int h, const double window_m[4], int fill_radius,
                               float *out) {
  if (!c || !out) return TACCHI_ERR_INVALID_ARG;
  tacchi_status s = validate_window(w, h, window_m, fill_radius);
  if (s != TACCHI_OK) return s;
  const bool dev = is_device_ptr(out);
  float *dst = out;
  if (!dev) {
    CK(ensure(c, &c->d_hbuf, &c->hbuf_cap, (size_t)w * h));
    dst = c->d_hbuf;
  }
  s = run_heightmap(c, w, h, window_m, fill_radius, dst);
  if (s != TACCHI_OK) return s;
  if (!dev) {
    CK(cudaMemcpyAsync(out, dst, sizeof(float) * w * h, cudaMemcpyDeviceToHost, c->stream));
    return sync_and_check(c);
  }
  return TACCHI_OK;
}

tacchi_status tacchi_render(tacchi_handle c, const tacchi_render_params *rp, int w, int h,
                            const double window_m[4], int fill_radius, float *out_rgb, float *out_height) {
  if (!c || !out_rgb) return TACCHI_ERR_INVALID_ARG;
  tacchi_status s = validate_window(w, h, window_m, fill_radius);
  if (s != TACCHI_OK) return s;
  ShadeArgs sa;
  s = fill_shade_args(rp, w, h, (window_m[2] - window_m[0]) / w, (window_m[3] - window_m[1]) / h, c->z_top, &sa);
  if (s != TACCHI_OK) return s;
  const bool rgb_dev = is_device_ptr(out_rgb);
  const bool h_dev = out_height && is_device_ptr(out_height);
  float *H = h_dev ? out_height : nullptr;
  if (!H) {
    CK(ensure(c, &c->d_hbuf, &c->hbuf_cap, (size_t)w * h));
    H = c->d_hbuf;
  }
  float *rgb = out_rgb;
  if (!rgb_dev) {
    CK(ensure(c, &c->d_rgb, &c->rgb_cap, (size_t)w * h * 3));
    rgb = c->d_rgb;
  }
  s = run_heightmap(c, w, h, window_m, fill_radius, H);
  if (s != TACCHI_OK) return s;
  CK(launch_shade(sa, H, rgb, c->stream));
  bool need_sync = false;
  if (!rgb_dev) {
    CK(cudaMemcpyAsync(out_rgb, rgb, sizeof(float) * 3 * w * h, cudaMemcpyDeviceToHost, c->stream));
    need_sync = true;
  }
  if (out_height && !h_dev) {
    CK(cudaMemcpyAsync(out_height, H, sizeof(float) * w * h, cudaMemcpyDeviceToHost, c->stream));
    need_sync = true;
  }
  return need_sync ? sync_and_check(c) : TACCHI_OK;
}

tacchi_status tacchi_shade(const tacchi_render_params *rp, const float *H_dev, int w, int h, double pixel_x_m,
                           double pixel_y_m, double z_top_m, float *rgb_dev, void *stream) {
  if (!H_dev || !rgb_dev || (long long)w * h > (1ll << 28)) return TACCHI_ERR_INVALID_ARG;
  ShadeArgs sa;
  tacchi_status s = fill_shade_args(rp, w, h, pixel_x_m, pixel_y_m, z_top_m, &sa);
  if (s != TACCHI_OK) return s;
  CK(launch_shade(sa, H_dev, rgb_dev, (cudaStream_t)stream));
  return TACCHI_OK;
}

tacchi_status tacchi_get_state(tacchi_handle c, float *u, float *v, float *C, float *Fm, uint8_t *flags) {
  if (!c) return TACCHI_ERR_INVALID_ARG;
  const long long N = c->N;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (u) CK(cudaMemcpyAsync(u, c->b.u, sizeof(float) * 3 * N, k, c->stream));
  if (v) CK(cudaMemcpyAsync(v, c->b.v, sizeof(float) * 3 * N, k, c->stream));
  if (C) CK(cudaMemcpyAsync(C, c->b.C, sizeof(float) * 9 * N, k, c->stream));
  if (Fm) CK(cudaMemcpyAsync(Fm, c->b.Fm, sizeof(float) * 9 * N, k, c->stream));
  if (flags) CK(cudaMemcpyAsync(flags, c->b.flags, N, k, c->stream));
  return sync_and_check(c);
}

tacchi_status tacchi_set_state(tacchi_handle c, const float *u, const float *v, const float *C, const float *Fm) {
  if (!c || !u) return TACCHI_ERR_INVALID_ARG;
  const long long N = c->N;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  cudaStream_t st = c->stream;
  CK(cudaMemcpyAsync(c->b.u, u, sizeof(float) * 3 * N, k, st));
  if (v) CK(cudaMemcpyAsync(c->b.v, v, sizeof(float) * 3 * N, k, st));
  else CK(cudaMemsetAsync(c->b.v, 0, sizeof(float) * 3 * N, st));
  if (C) CK(cudaMemcpyAsync(c->b.C, C, sizeof(float) * 9 * N, k, st));
  else CK(cudaMemsetAsync(c->b.C, 0, sizeof(float) * 9 * N, st));
  if (Fm) CK(cudaMemcpyAsync(c->b.Fm, Fm, sizeof(float) * 9 * N, k, st));
  else CK(cudaMemsetAsync(c->b.Fm, 0, sizeof(float) * 9 * N, st));
  CK(cudaMemsetAsync(c->b.err, 0, sizeof(int), st));
  CK(launch_sort(c->b, c->blk, 1, st));
  CK(cudaMemsetAsync(c->b.movers, 0, sizeof(int), st));
  c->stepped = false;
  return TACCHI_OK;
}

tacchi_status tacchi_get_grid(tacchi_handle c, float *out) {
  if (!c || !out) return TACCHI_ERR_INVALID_ARG;
  if (!c->stepped) return TACCHI_ERR_STATE;
  CK(cudaMemcpyAsync(out, c->b.gmm, sizeof(float4) * c->nodes, cudaMemcpyDeviceToDevice, c->stream));
  return TACCHI_OK;
}

tacchi_status tacchi_set_profiling(tacchi_handle c, int on) {
  if (!c) return TACCHI_ERR_INVALID_ARG;
  c->profiling = on != 0;
  return TACCHI_OK;
}

tacchi_status tacchi_get_profile(tacchi_handle c, tacchi_profile_t *o, int reset) {
  if (!c || !o) return TACCHI_ERR_INVALID_ARG;
  o->grid_ms = c->prof_ms[0];
  o->fused_ms = c->prof_ms[1];
  o->edge_ms = c->prof_ms[2];
  o->sort_ms = c->prof_ms[3];
  o->grid_launches = c->prof_n[0];
  o->fused_launches = c->prof_n[1];
  o->edge_launches = c->prof_n[2];
  o->sort_launches = c->prof_n[3];
  if (reset)
    for (int k = 0; k < 4; ++k) {
      c->prof_ms[k] = 0;
      c->prof_n[k] = 0;
    }
  return TACCHI_OK;
}

tacchi_status tacchi_sync(tacchi_handle c) {
  if (!c) return TACCHI_ERR_INVALID_ARG;
  return sync_and_check(c);
}

tacchi_status tacchi_clear_error(tacchi_handle c) {
  if (!c) return TACCHI_ERR_INVALID_ARG;
  CK(cudaMemsetAsync(c->b.err, 0, sizeof(int), c->stream));
  return TACCHI_OK;
}

}  // extern "C"
