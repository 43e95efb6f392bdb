// noalloc.cu -- a height-map entry point that allocates no memory.
//
// Some callers cannot allocate device memory while they run.  A robot
// simulator's real-time control thread must not call cudaMalloc, which can
// block and synchronise the device for an unbounded time; a plugin inside a
// host application that owns the whole device-memory budget may not allocate
// at all.  tacchi_heightmap_static serves them: the caller passes the
// particle arrays and the output buffer, and the only scratch the computation
// needs (the per-pixel coverage buffer) lives in a fixed static device array
// declared below.  Every GPU that loads the library holds that array
// (TACCHI_STATIC_HEIGHTMAP_MAX_PIXELS ints, 4 MiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "tacchi.h"
#include "tacchi_internal.cuh"

namespace {

// Coverage scratch shared by every call on a device.  Host code must not
// pass this name to a kernel: on the host it is only a stand-in, and its
// device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) int g_hm_scratch[TACCHI_STATIC_HEIGHTMAP_MAX_PIXELS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
tacchi_status scratch_on_current_device(int **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TACCHI_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TACCHI_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_hm_scratch);
    if (e != cudaSuccess || !p) return TACCHI_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<int *>(p);
  }
  *out = g_scratch_addr[dev];
  return TACCHI_OK;
}

bool finite_all(const double *a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

extern "C" tacchi_status tacchi_heightmap_static(const float *u_dev, int64_t n_particles,
                                                 const uint32_t *surf_dev, const float *z0_dev,
                                                 int n_surface, double dx_m, const double origin_m[2],
                                                 double z_top_m, int w, int hgt, const double window_m[4],
                                                 int fill_radius, float *out_dev, void *stream) {
  if (!u_dev || !out_dev || !origin_m || !window_m || n_particles < 1 || n_surface < 0)
    return TACCHI_ERR_INVALID_ARG;
  if (n_surface > 0 && (!surf_dev || !z0_dev)) return TACCHI_ERR_INVALID_ARG;
  if (!(dx_m > 0) || !std::isfinite(dx_m) || !std::isfinite(z_top_m) || !finite_all(origin_m, 2) ||
      !finite_all(window_m, 4))
    return TACCHI_ERR_INVALID_ARG;
  if (w < 1 || hgt < 1 || (long long)w * hgt > (long long)TACCHI_STATIC_HEIGHTMAP_MAX_PIXELS)
    return TACCHI_ERR_INVALID_ARG;
  if (!(window_m[2] > window_m[0]) || !(window_m[3] > window_m[1]) || fill_radius < 0 ||
      fill_radius > tacchi::kMaxFillRadius)
    return TACCHI_ERR_INVALID_ARG;

  int *scratch = nullptr;
  const tacchi_status s = scratch_on_current_device(&scratch);
  if (s != TACCHI_OK) return s;

  tacchi::HeightmapArgs a{};
  a.u = u_dev;
  a.Ntot = n_particles;
  a.surf = surf_dev;
  a.z0 = z0_dev;
  a.Ns = n_surface;
  const double pxc = ((window_m[2] - window_m[0]) / (double)w) / dx_m;
  const double pyc = ((window_m[3] - window_m[1]) / (double)hgt) / dx_m;
  a.A0X = (float)((window_m[0] - origin_m[0]) / dx_m + 0.5 * pxc);
  a.A0Y = (float)((window_m[1] - origin_m[1]) / dx_m + 0.5 * pyc);
  a.SX = (float)pxc;
  a.SY = (float)pyc;
  if (!(a.SX > 0.f) || !(a.SY > 0.f)) return TACCHI_ERR_INVALID_ARG;
  a.z_top = (float)z_top_m;
  a.dx = (float)dx_m;
  a.w = w;
  a.h = hgt;
  a.fill_radius = fill_radius;
  a.cov = scratch;  // cleared by the first kernel of every call
  a.out = out_dev;
  return tacchi::launch_heightmap(a, (cudaStream_t)stream) == cudaSuccess ? TACCHI_OK : TACCHI_ERR_CUDA;
}
