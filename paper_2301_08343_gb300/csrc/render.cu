// render.cu -- tactile rendering kernels for sm_103a (Tacchi, arXiv
// 2301.08343, Sec. III-B).
//
//   k_hm_clear / k_hm_splat / k_hm_fill  height map of the deformed top
//       surface: z-max splat of the top-layer particles (coverage radius
//       dx/2, decided in FP32 with a fixed operation order), then
//       nearest-covered-pixel hole filling within a bounded radius.
//   k_shade  Phong shading, Eqs. 12-14, one thread per pixel.
#include "tacchi_internal.cuh"

#include <climits>

namespace tacchi {

// Monotone map of floats to ints so that atomicMax orders heights.
__device__ __forceinline__ int ordered_from_float(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float float_from_ordered(int i) {
  return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
}

__global__ void __launch_bounds__(256) k_hm_clear(int *cov, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) cov[e] = INT_MIN;
}

__global__ void __launch_bounds__(256) k_hm_splat(HeightmapArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.Ns) return;
  const uint32_t p = a.surf[s];
  float ux, uy, uz;
  if (a.ps) {
    const float4 q = load_position(a.ps, p);
    ux = q.x; uy = q.y; uz = q.z;
  } else {
    ux = a.u[p]; uy = a.u[a.Ntot + p]; uz = a.u[2 * a.Ntot + p];
  }
  // rest top plane plus the particle's vertical displacement (metres)
  const float h = a.z_top + a.dx * (uz - a.z0[s]);
  if (!(isfinite(ux) && isfinite(uy) && isfinite(h))) return;
  // conservative pixel box of the disc of radius 1/2 cell; the exact test decides.
  // The box edges are clamped just outside the image before they become
  // integers, so a position far outside it cannot overflow them.
  const float bx0 = fminf(fmaxf((ux - 0.5f - a.A0X) / a.SX, -2.f), (float)a.w + 1.f);
  const float bx1 = fminf(fmaxf((ux + 0.5f - a.A0X) / a.SX, -2.f), (float)a.w + 1.f);
  const float by0 = fminf(fmaxf((uy - 0.5f - a.A0Y) / a.SY, -2.f), (float)a.h + 1.f);
  const float by1 = fminf(fmaxf((uy + 0.5f - a.A0Y) / a.SY, -2.f), (float)a.h + 1.f);
  int c0 = (int)floorf(bx0) - 1;
  int c1 = (int)ceilf(bx1) + 1;
  int r0 = (int)floorf(by0) - 1;
  int r1 = (int)ceilf(by1) + 1;
  c0 = max(c0, 0);
  r0 = max(r0, 0);
  c1 = min(c1, a.w - 1);
  r1 = min(r1, a.h - 1);
  const int key = ordered_from_float(h);
  for (int r = r0; r <= r1; ++r) {
    const float qy = __fmaf_rn((float)r, a.SY, a.A0Y);
    const float ey = __fsub_rn(qy, uy);
    const float b2 = __fmul_rn(ey, ey);
    for (int c = c0; c <= c1; ++c) {
      const float qx = __fmaf_rn((float)c, a.SX, a.A0X);
      const float ex = __fsub_rn(qx, ux);
      if (__fadd_rn(__fmul_rn(ex, ex), b2) <= 0.25f) atomicMax(a.cov + (long long)r * a.w + c, key);
    }
  }
}

__global__ void __launch_bounds__(256) k_hm_fill(HeightmapArgs a) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.w * a.h) return;
  const int r = (int)(e / a.w), c = (int)(e % a.w);
  const int key = a.cov[e];
  if (key != INT_MIN) {
    a.out[e] = float_from_ordered(key);
    return;
  }
  const int R = a.fill_radius;
  long long best = -1;
  int bestd = 0;
  for (int rr = max(r - R, 0); rr <= min(r + R, a.h - 1); ++rr)
    for (int cc = max(c - R, 0); cc <= min(c + R, a.w - 1); ++cc) {
      const long long f = (long long)rr * a.w + cc;
      if (a.cov[f] == INT_MIN) continue;
      const int d = (rr - r) * (rr - r) + (cc - c) * (cc - c);
      if (best < 0 || d < bestd) {  // row-major scan: first hit wins ties
        best = f;
        bestd = d;
      }
    }
  a.out[e] = best >= 0 ? float_from_ordered(a.cov[best]) : a.z_top;
}

cudaError_t launch_heightmap(const HeightmapArgs &a, cudaStream_t st) {
  const long long P = (long long)a.w * a.h;
  const unsigned gp = (unsigned)((P + 255) / 256);
  k_hm_clear<<<gp, 256, 0, st>>>(a.cov, P);
  if (a.Ns > 0) k_hm_splat<<<(a.Ns + 255) / 256, 256, 0, st>>>(a);
  k_hm_fill<<<gp, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Eqs. 12-14: D = z_top - H; N = normalize(dD/dx, dD/dy, -1) by central
// differences with replicated edges; V = (0, 0, -1);
// I = ka ia + sum_m kd max(L.N, 0) i_md + ks max(R.V, 0)^alpha i_ms,
// R = 2 (L.N) N - L; clamped to [0, 1].
__global__ void __launch_bounds__(256) k_shade(ShadeArgs a, const float *__restrict__ H, float *__restrict__ rgb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.w * a.h) return;
  const int r = (int)(e / a.w), c = (int)(e % a.w);
  const int cl = c > 0 ? c - 1 : 0, cr = c < a.w - 1 ? c + 1 : a.w - 1;
  const int ru = r > 0 ? r - 1 : 0, rd = r < a.h - 1 ? r + 1 : a.h - 1;
  const float Dl = a.z_top - H[(long long)r * a.w + cl], Dr = a.z_top - H[(long long)r * a.w + cr];
  const float Du = a.z_top - H[(long long)ru * a.w + c], Dd = a.z_top - H[(long long)rd * a.w + c];
  const float gx = (Dr - Dl) * a.inv2px;
  const float gy = (Dd - Du) * a.inv2py;
  const float inn = 1.0f / sqrtf(gx * gx + gy * gy + 1.0f);
  const float N0 = gx * inn, N1 = gy * inn, N2 = -inn;
  float I0 = a.ka * a.amb[0], I1 = a.ka * a.amb[1], I2 = a.ka * a.amb[2];
  for (int m = 0; m < a.n_lights; ++m) {
    const float L0 = a.dir[m][0], L1 = a.dir[m][1], L2 = a.dir[m][2];
    const float LN = L0 * N0 + L1 * N1 + L2 * N2;
    const float R2 = 2.0f * LN * N2 - L2;  // R.V with V = (0, 0, -1) is -R_z
    const float RV = -R2;
    const float dif = a.kd * fmaxf(LN, 0.0f);
    const float spe = RV > 0.0f ? a.ks * powf(RV, a.alpha) : 0.0f;
    I0 += dif * a.dif[m][0] + spe * a.spe[m][0];
    I1 += dif * a.dif[m][1] + spe * a.spe[m][1];
    I2 += dif * a.dif[m][2] + spe * a.spe[m][2];
  }
  rgb[3 * e + 0] = fminf(fmaxf(I0, 0.0f), 1.0f);
  rgb[3 * e + 1] = fminf(fmaxf(I1, 0.0f), 1.0f);
  rgb[3 * e + 2] = fminf(fmaxf(I2, 0.0f), 1.0f);
}

cudaError_t launch_shade(const ShadeArgs &a, const float *H, float *rgb, cudaStream_t st) {
  const long long P = (long long)a.w * a.h;
  k_shade<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a, H, rgb);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dispmap(DispMapArgs a) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.w * a.h) return;
  const int r = (int)(e / a.w), c = (int)(e % a.w);
  // rest lattice of the top particle layer: spacing dx/2 from the block corner
  const float X = a.xy ? a.xy[2 * e] : a.X0 + (float)c * a.PW;
  const float Y = a.xy ? a.xy[2 * e + 1] : a.Y0 + (float)r * a.PH;
  int i = (int)floorf(X / (0.5f * a.dx)), j = (int)floorf(Y / (0.5f * a.dx));
  i = min(max(i, 0), 2 * a.nx - 1);
  j = min(max(j, 0), 2 * a.ny - 1);
  const long long s = ((long long)(j >> 1) * a.nx + (i >> 1)) * 4 + (j & 1) * 2 + (i & 1);
  const uint32_t p = a.surf[s];
  const float4 q = load_position(a.ps, p);
  a.out[3 * e + 0] = a.dx * (q.x - a.rest[s]);
  a.out[3 * e + 1] = a.dx * (q.y - a.rest[a.rest_stride + s]);
  a.out[3 * e + 2] = a.dx * (q.z - a.rest[2 * a.rest_stride + s]);
}

cudaError_t launch_dispmap(const DispMapArgs &a, cudaStream_t st) {
  const long long P = (long long)a.w * a.h;
  k_dispmap<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// Lowest point of the indenter over world (x, y); +inf where it is absent.
__device__ float indenter_bottom(const PenMapArgs &a, float x, float y) {
  const float dxw = x - a.cx, dyw = y - a.cy;
  const float lx = a.cosy * dxw + a.siny * dyw;   // local frame (yaw only)
  const float ly = -a.siny * dxw + a.cosy * dyw;
  const float INF = __int_as_float(0x7f800000);
  switch (a.kind) {
    case IND_SPHERE: {  // p0 = radius, pose = centre
      const float r2 = lx * lx + ly * ly;
      return r2 < a.p0 * a.p0 ? a.cz - sqrtf(a.p0 * a.p0 - r2) : INF;
    }
    case IND_CYLINDER:  // p0 = radius, p1 = half length along local x
      return (fabsf(lx) <= a.p1 && fabsf(ly) < a.p0) ? a.cz - sqrtf(a.p0 * a.p0 - ly * ly) : INF;
    case IND_CONE: {    // p0 = half angle, p1 = height; apex at the pose
      const float r = sqrtf(lx * lx + ly * ly);
      const float t = tanf(a.p0);
      return r <= a.p1 * t ? a.cz + r / t : INF;
    }
    case IND_PRISM: {   // p0 = half angle, p1 = half length (local y), p2 = height
      const float t = tanf(a.p0);
      return (fabsf(ly) <= a.p1 && fabsf(lx) <= a.p2 * t) ? a.cz + fabsf(lx) / t : INF;
    }
    case IND_HEIGHTMAP: {  // protrusions below the back plane at the pose
      const float fx = lx / a.hm_pix + (0.5f * a.hm_w - 0.5f), fy = ly / a.hm_pix + (0.5f * a.hm_h - 0.5f);
      if (fx < -0.5f || fx > a.hm_w - 0.5f || fy < -0.5f || fy > a.hm_h - 0.5f) return INF;
      const float cx = fminf(fmaxf(fx, 0.f), (float)(a.hm_w - 1)), cy = fminf(fmaxf(fy, 0.f), (float)(a.hm_h - 1));
      const int ix = min((int)floorf(cx), a.hm_w - 2), iy = min((int)floorf(cy), a.hm_h - 2);
      const float tx = cx - ix, ty = cy - iy;
      const float *H = a.hm;
      const float h0 = H[iy * a.hm_w + ix] * (1.f - tx) + H[iy * a.hm_w + ix + 1] * tx;
      const float h1 = H[(iy + 1) * a.hm_w + ix] * (1.f - tx) + H[(iy + 1) * a.hm_w + ix + 1] * tx;
      return a.cz - a.dx * (h0 * (1.f - ty) + h1 * ty);
    }
    default:
      return INF;
  }
}

__global__ void __launch_bounds__(256) k_penmap(PenMapArgs a) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.w * a.h) return;
  const int r = (int)(e / a.w), c = (int)(e % a.w);
  const float zb = indenter_bottom(a, a.X0 + (float)c * a.PW, a.Y0 + (float)r * a.PH);
  a.out[e] = fmaxf(a.z_top - zb, 0.f);
}

cudaError_t launch_penmap(const PenMapArgs &a, cudaStream_t st) {
  const long long P = (long long)a.w * a.h;
  k_penmap<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// Rows pass: one CTA per 256 pixels of an (extended) row.  The row's
// penetration over the segment and its rx-pixel margins is evaluated once
// into shared memory, then each thread sums its 2 rx + 1 taps.
constexpr int kSmoothTile = 256;
__global__ void __launch_bounds__(kSmoothTile) k_smooth_rows(SmoothArgs a) {
  __shared__ float sp[kSmoothTile + 2 * kMaxSmoothRadius];
  __shared__ float sg[kMaxSmoothRadius + 1];
  const PenMapArgs &p = a.pen;
  const int t = threadIdx.x, rx = a.rx;
  const int r = (int)blockIdx.y - a.ry;  // window row; outside [0, h) in the margins
  const int c0 = (int)blockIdx.x * kSmoothTile;
  const float y = p.Y0 + (float)r * p.PH;
  for (int e = t; e < kSmoothTile + 2 * rx; e += kSmoothTile) {
    const int c = c0 - rx + e;
    sp[e] = fmaxf(p.z_top - indenter_bottom(p, p.X0 + (float)c * p.PW, y), 0.f);
  }
  for (int e = t; e <= rx; e += kSmoothTile) sg[e] = a.gx[e];
  __syncthreads();
  const int c = c0 + t;
  if (c >= p.w) return;
  const float *q = sp + t + rx;
  float s = sg[0] * q[0];
  for (int k = 1; k <= rx; ++k) s = fmaf(sg[k], q[-k] + q[k], s);
  a.tmp[(size_t)blockIdx.y * p.w + c] = s;
}

// Columns pass: thread per pixel; the 2 ry + 1 taps of a column are
// consecutive rows of tmp, so a warp's loads are coalesced.
__global__ void __launch_bounds__(kSmoothTile) k_smooth_cols(SmoothArgs a) {
  __shared__ float sg[kMaxSmoothRadius + 1];
  const int t = threadIdx.x, ry = a.ry, w = a.pen.w;
  for (int e = t; e <= ry; e += kSmoothTile) sg[e] = a.gy[e];
  __syncthreads();
  const int c = (int)blockIdx.x * kSmoothTile + t;
  if (c >= w) return;
  const int r = (int)blockIdx.y;
  const float *q = a.tmp + (size_t)(r + ry) * w + c;
  float s = sg[0] * q[0];
  for (int l = 1; l <= ry; ++l) s = fmaf(sg[l], q[-(ptrdiff_t)l * w] + q[(ptrdiff_t)l * w], s);
  a.H[(size_t)r * w + c] = a.pen.z_top - s;
}

cudaError_t launch_smoothed(const SmoothArgs &a, cudaStream_t st) {
  const unsigned gx = (unsigned)((a.pen.w + kSmoothTile - 1) / kSmoothTile);
  k_smooth_rows<<<dim3(gx, (unsigned)(a.pen.h + 2 * a.ry)), kSmoothTile, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_smooth_cols<<<dim3(gx, (unsigned)a.pen.h), kSmoothTile, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tacchi
