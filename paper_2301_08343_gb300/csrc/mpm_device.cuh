// mpm_device.cuh -- device helpers shared by the MLS-MPM transfer kernels
// (Tacchi, arXiv 2301.08343, Sec. III-A): 3x3 algebra, the left stretch of
// the polar decomposition and the fixed-corotated stress (Eq. 5's S_p),
// quadratic B-spline weights, block-wide scans of the cell grouping, the
// single-particle scatter to the grid and the asynchronous-copy wrappers.  Included only by the library's .cu files.
#pragma once
#include "tacchi_internal.cuh"

namespace tacchi {

// ---------------------------------------------------------------------------
// 3x3 helpers (row-major).
__device__ __forceinline__ void cofactor3(const float Y[9], float c[9]) {
  c[0] = Y[4] * Y[8] - Y[5] * Y[7];
  c[1] = Y[5] * Y[6] - Y[3] * Y[8];
  c[2] = Y[3] * Y[7] - Y[4] * Y[6];
  c[3] = Y[2] * Y[7] - Y[1] * Y[8];
  c[4] = Y[0] * Y[8] - Y[2] * Y[6];
  c[5] = Y[1] * Y[6] - Y[0] * Y[7];
  c[6] = Y[1] * Y[5] - Y[2] * Y[4];
  c[7] = Y[2] * Y[3] - Y[0] * Y[5];
  c[8] = Y[0] * Y[4] - Y[1] * Y[3];
}

// Symmetric 3x3 matrices are held as their six entries (00, 11, 22, 01, 02, 12).
__device__ __forceinline__ void cofactor_sym(const float Y[6], float c[6]) {
  c[0] = Y[1] * Y[2] - Y[5] * Y[5];
  c[1] = Y[0] * Y[2] - Y[4] * Y[4];
  c[2] = Y[0] * Y[1] - Y[3] * Y[3];
  c[3] = Y[4] * Y[5] - Y[3] * Y[2];
  c[4] = Y[3] * Y[5] - Y[4] * Y[1];
  c[5] = Y[3] * Y[4] - Y[0] * Y[5];
}

// Entries (00, 11, 22, 01, 02, 12) of S + P Z for symmetric P and Z that
// commute (polynomials in one matrix), so that P Z is symmetric too.
__device__ __forceinline__ void sym_mul_add(const float P[6], const float Z[6], const float S[6], float R[6]) {
  R[0] = S[0] + P[0] * Z[0] + P[3] * Z[3] + P[4] * Z[4];
  R[1] = S[1] + P[3] * Z[3] + P[1] * Z[1] + P[5] * Z[5];
  R[2] = S[2] + P[4] * Z[4] + P[5] * Z[5] + P[2] * Z[2];
  R[3] = S[3] + P[0] * Z[3] + P[3] * Z[1] + P[4] * Z[5];
  R[4] = S[4] + P[0] * Z[4] + P[3] * Z[5] + P[4] * Z[2];
  R[5] = S[5] + P[3] * Z[4] + P[1] * Z[5] + P[5] * Z[2];
}

// Left stretch V = (F F^T)^{1/2} of the polar decomposition F = V R, from
// H = F - I, carried as Y = V - I with B = F F^T = I + P so that both keep
// their relative precision near the rest state.  P = H + H^T + H H^T.
// Start: the series I + P/2 - P^2/8 (error about |P|^3 / 16) while |P| is
// small, else Newton's first iterate (I + B) / 2 (positive definite for any
// nonsingular F).  Then Newton's iteration V <- (V + B V^{-1}) / 2 for the
// square root of B (Higham, Functions of Matrices, Sec. 6.3): every iterate
// is a polynomial in B, so the products stay symmetric, and the error in each
// eigenvalue goes as e <- e^2 / (2 v).  With V = I + Y:
// det V = 1 + tr Y + m2(Y) + det Y = 1 + d,  V^{-1} - I = [ -(m2 + det Y) I - Y + cof Y ] / (1 + d) = Z,
// B V^{-1} = I + P + Z + P Z,  hence  Y <- (Y + P + Z + P Z) / 2.
// Output P and Y; the stress needs no rotation.
__device__ __forceinline__ void left_stretch_delta(const float H[9], float P[6], float Y[6]) {
  P[0] = 2.0f * H[0] + (H[0] * H[0] + H[1] * H[1] + H[2] * H[2]);
  P[1] = 2.0f * H[4] + (H[3] * H[3] + H[4] * H[4] + H[5] * H[5]);
  P[2] = 2.0f * H[8] + (H[6] * H[6] + H[7] * H[7] + H[8] * H[8]);
  P[3] = (H[1] + H[3]) + (H[0] * H[3] + H[1] * H[4] + H[2] * H[5]);
  P[4] = (H[2] + H[6]) + (H[0] * H[6] + H[1] * H[7] + H[2] * H[8]);
  P[5] = (H[5] + H[7]) + (H[3] * H[6] + H[4] * H[7] + H[5] * H[8]);
  float pmag = 0.f;
#pragma unroll
  for (int e = 0; e < 6; ++e) pmag = fmaxf(pmag, fabsf(P[e]));
  float PP[6];
  const float zero[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  sym_mul_add(P, P, zero, PP);
  const bool series = pmag < 0.5f;
#pragma unroll
  for (int e = 0; e < 6; ++e) Y[e] = series ? fmaf(-0.125f, PP[e], 0.5f * P[e]) : 0.5f * P[e];
  // Newton converges quadratically: with |Y_{k+1} - Y_k| = e the next error is
  // about e^2 / 2, below 5e-8 of the strain scale |P| once e^2 <= 1e-7 |P|.
  // The series start alone is that close once (3 |P|)^3 / 16 <= 5e-8 |P|.
  const float tol2 = 1e-7f * pmag;
  if (series && pmag * pmag <= 2.9e-8f) return;
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    float c[6];
    cofactor_sym(Y, c);
    const float m2 = c[0] + c[1] + c[2];
    const float dY = Y[0] * c[0] + Y[3] * c[3] + Y[4] * c[4];
    const float d = (Y[0] + Y[1] + Y[2]) + m2 + dY;
    // approximate reciprocal: the iteration corrects its own rounding
    const float inv = __fdividef(1.0f, 1.0f + d);
    const float s = -(m2 + dY);
    float Z[6], BZ[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) Z[e] = ((e < 3 ? s : 0.f) + (c[e] - Y[e])) * inv;
    sym_mul_add(P, Z, Z, BZ);  // B V^{-1} - I - P = Z + P Z
    float diff = 0.f;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const float yn = 0.5f * ((Y[e] + P[e]) + BZ[e]);
      diff = fmaxf(diff, fabsf(yn - Y[e]));
      Y[e] = yn;
    }
    if (!(diff * diff > tol2)) break;
  }
}

// Elasticity term S_p of Eq. 5 as the fixed-corotated Kirchhoff stress
// tau = 2 mu (F - R) F^T + lambda J (J - 1) I, from H = F - I.  With
// F = V R:  (F - R) F^T = F F^T - R R^T V = B - V, so
// tau = 2 mu (P - Y) + lambda J (J - 1) I  (symmetric; no rotation needed).
// Returns J - 1 (computed as tr H + m2(H) + det H).
__device__ __forceinline__ float kirchhoff_stress(const float H[9], float mu, float la, float tau[9]) {
  float P[6], Y[6];
  left_stretch_delta(H, P, Y);
  float c[9];
  cofactor3(H, c);
  const float Jm1 = (H[0] + H[4] + H[8]) + (c[0] + c[4] + c[8]) + (H[0] * c[0] + H[1] * c[1] + H[2] * c[2]);
  const float J = 1.0f + Jm1;
  const float pr = la * J * Jm1;
  const float tm = 2.0f * mu;
  tau[0] = tm * (P[0] - Y[0]) + pr;
  tau[4] = tm * (P[1] - Y[1]) + pr;
  tau[8] = tm * (P[2] - Y[2]) + pr;
  tau[1] = tau[3] = tm * (P[3] - Y[3]);
  tau[2] = tau[6] = tm * (P[4] - Y[4]);
  tau[5] = tau[7] = tm * (P[5] - Y[5]);
  return Jm1;
}

// Quadratic B-spline weights of one axis at fraction f in [1/2, 3/2) from
// the stencil base, and node offsets (i - f) in cells.
__device__ __forceinline__ void bspline3(float f, float w[3], float d[3]) {
  const float a = 1.5f - f, b = f - 1.0f, c = f - 0.5f;
  w[0] = 0.5f * a * a;
  w[1] = 0.75f - b * b;
  w[2] = 0.5f * c * c;
  d[0] = -f;
  d[1] = 1.0f - f;
  d[2] = 2.0f - f;
}

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// Exclusive scan over n (<= THREADS * PER) entries of `a` into `out` (out[n] =
// total); also compacts the indices with a[c] > 0 into `cells`, returning
// their number.  All threads of the CTA call it.
template <int THREADS, int PER>
__device__ __forceinline__ uint32_t block_scan_compact(const uint32_t *a, uint32_t *out, uint16_t *cells,
                                                       int n, uint32_t *warp_buf) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = THREADS / 32;
  uint32_t v[PER], nz[PER];
  uint32_t sum = 0, nzs = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int c = tid * PER + q;
    v[q] = c < n ? a[c] : 0u;
    nz[q] = v[q] > 0 ? 1u : 0u;
    sum += v[q];
    nzs += nz[q];
  }
  // pack both running sums: counts < 2^20 per CTA, non-empty cells < 2^12
  uint32_t x = sum | (nzs << 20);
  const uint32_t mine = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_buf[warp] = x;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += warp_buf[w];
  uint32_t run = x - mine + wpre;
  uint32_t rs = run & 0xFFFFFu, rn = run >> 20;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int c = tid * PER + q;
    if (c < n) {
      out[c] = rs;
      if (nz[q]) cells[rn] = (uint16_t)c;
    }
    rs += v[q];
    rn += nz[q];
  }
  uint32_t tot = 0;
  for (int w = 0; w < NWARP; ++w) tot += warp_buf[w];
  if (tid == 0) out[n] = tot & 0xFFFFFu;
  __syncthreads();
  return tot >> 20;
}

// Stable partition of the n non-empty cells (cells[0..n), index order) into
// four classes by particle count, heaviest first: >= 11, 9-10, 7-8, <= 6.
// The thread-per-cell loop then runs cells of similar count side by side in
// a warp, so that lanes and warps finish together when the particles of a
// strained block have spread unevenly over its cells (at rest every cell
// holds 8).  Within a class the index order (and the locality of
// neighbouring cells in a warp) is kept.  All threads of the CTA call it.
template <int THREADS, int PER>
__device__ __forceinline__ void order_cells_by_load(const uint16_t *cells, const uint32_t *start, int n,
                                                    uint16_t *order, unsigned long long *warp_buf) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = THREADS / 32;
  auto cls = [](uint32_t k) { return k >= 11 ? 0 : (k >= 9 ? 1 : (k >= 7 ? 2 : 3)); };
  int myc[PER];
  unsigned long long cnt = 0;  // four 16-bit class counts of this thread's chunk
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = tid * PER + q;
    myc[q] = -1;
    if (i < n) {
      const uint32_t c = cells[i];
      myc[q] = cls(start[c + 1] - start[c]);
      cnt += 1ull << (16 * myc[q]);
    }
  }
  unsigned long long x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_buf[warp] = x;
  __syncthreads();
  unsigned long long pre = x - cnt, tot = 0;
  for (int w = 0; w < NWARP; ++w) {
    if (w < warp) pre += warp_buf[w];
    tot += warp_buf[w];
  }
  // class base = sum of the totals of the heavier classes
  uint32_t base[4];
  base[0] = 0;
#pragma unroll
  for (int k = 1; k < 4; ++k) base[k] = base[k - 1] + (uint32_t)((tot >> (16 * (k - 1))) & 0xFFFFu);
  uint32_t run[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) run[k] = base[k] + (uint32_t)((pre >> (16 * k)) & 0xFFFFu);
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = tid * PER + q;
    if (i < n) order[run[myc[q]]++] = cells[i];
  }
  __syncthreads();
}

// P2G of one particle straight into the grid (particles that change cell
// during the substep, and the fallback when a block cannot be grouped):
// Eqs. 2-5 at the 27 nodes of the stencil with base (bx, by, bz), one vector
// reduction per node.  Returns false, writing nothing, when the stencil is
// not inside the grid of G0 x G1 x G2 nodes.
__device__ __forceinline__ bool scatter_particle_global(float4 *g, int G0, int G1, int G2, int bx, int by,
                                                        int bz, float m, const float f[3], const float mv[3],
                                                        const float A[9]) {
  // compared against G - 3, not as b + 2 >= G: a position far outside the grid
  // (a run that has already failed its CFL check) saturates floor() at INT_MAX,
  // where b + 2 would wrap negative and pass
  if (bx < 0 || by < 0 || bz < 0 || bx > G0 - 3 || by > G1 - 3 || bz > G2 - 3) return false;
  float wx[3], wy[3], wz[3], dpx[3], dpy[3], dpz[3];
  bspline3(f[0], wx, dpx);
  bspline3(f[1], wy, dpy);
  bspline3(f[2], wz, dpz);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float wjk = wy[j] * wz[k];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float w = wx[i] * wjk;
        float r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
          r[a] = w * (mv[a] + A[a * 3 + 0] * dpx[i] + A[a * 3 + 1] * dpy[j] + A[a * 3 + 2] * dpz[k]);
        atomicAdd(g + ((long long)(bz + k) * G1 + (by + j)) * G0 + (bx + i), make_float4(m * w, r[0], r[1], r[2]));
      }
    }
  return true;
}

// Bulk asynchronous copies global -> shared done by the copy engine, whose
// completion is counted in bytes on an mbarrier (they are not part of the
// cp.async groups above).  Both addresses 16-byte aligned, size a multiple
// of 16.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// orders this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// one arrival that also announces the bytes this thread's copies will bring
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// one arrival without bytes
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of the given parity; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long max_polls) {
  for (long long it = 0; it < max_polls; ++it)
    if (mbar_test(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// 16-byte asynchronous copy global -> shared (L2 only), and its group fences.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace tacchi
