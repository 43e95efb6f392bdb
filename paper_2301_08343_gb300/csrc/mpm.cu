// mpm.cu -- MLS-MPM substep kernels for sm_103a (Tacchi, arXiv 2301.08343,
// Sec. III-A).
//
//   k_grid_update  Eq. 6 (V = MG / M) fused with the rigid indenter, the fixed
//                  base (Eq. 10 on the grid) and the padding band.
//   k_transfer     one CTA per sort block of cells.  G2P of substep k
//                  (Eqs. 7-9, the base override of Eq. 10 and advection,
//                  Eq. 11) fused with P2G of substep k+1 (Eqs. 2-5) into a
//                  shared-memory grid tile, flushed with vector reductions.
//                  P2G-only and G2P-only variants start and end a step.
//   k_sort_*       counting sort of particle ids by grid block, run only when
//                  a particle left its block during the last transfer.
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

// Rotation R of the polar decomposition F = R S by Newton's iteration
// X <- (X + X^{-T}) / 2 (Higham 1986), carried in the form Y = X - I so that
// R - I keeps its relative precision near the rest state.  With
// X = I + Y:  det X = 1 + tr Y + m2(Y) + det Y  and
// cof X = (1 + tr Y) I - Y^T + cof Y, hence
// X^{-T} - I = [ -(m2 + det Y) I - Y^T + cof Y ] / det X.
// Input H = F - I; output Y = R - I.
__device__ __forceinline__ void polar_rotation_delta(const float H[9], float Y[9]) {
  float hmag = 0.f;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    Y[e] = H[e];
    hmag = fmaxf(hmag, fabsf(H[e]));
  }
  const float tol = 1e-7f * hmag;
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    float c[9];
    cofactor3(Y, c);
    const float m2 = c[0] + c[4] + c[8];
    const float dY = Y[0] * c[0] + Y[1] * c[1] + Y[2] * c[2];
    const float d = (Y[0] + Y[4] + Y[8]) + m2 + dY;
    const float inv = 1.0f / (1.0f + d);
    const float s = -(m2 + dY);
    float Yn[9];
    float diff = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float Z = ((r == q ? s : 0.f) - Y[q * 3 + r] + c[r * 3 + q]) * inv;
        Yn[r * 3 + q] = 0.5f * (Y[r * 3 + q] + Z);
        diff = fmaxf(diff, fabsf(Yn[r * 3 + q] - Y[r * 3 + q]));
      }
#pragma unroll
    for (int e = 0; e < 9; ++e) Y[e] = Yn[e];
    if (!(diff > tol)) break;
  }
}

// Elasticity term S_p of Eq. 5 as the fixed-corotated Kirchhoff stress
// tau = 2 mu (F - R) F^T + lambda J (J - 1) I, from H = F - I.
// Returns J - 1 (computed as tr H + m2(H) + det H).
__device__ __forceinline__ float kirchhoff_stress(const float H[9], float mu, float la, float tau[9]) {
  float Y[9];
  polar_rotation_delta(H, Y);
  float c[9];
  cofactor3(H, c);
  const float Jm1 = (H[0] + H[4] + H[8]) + (c[0] + c[4] + c[8]) + (H[0] * c[0] + H[1] * c[1] + H[2] * c[2]);
  const float J = 1.0f + Jm1;
  float D[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) D[e] = H[e] - Y[e];  // F - R
  const float pr = la * J * Jm1;
  const float tm = 2.0f * mu;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      // (D (I + H)^T)_{rq} = D_rq + sum_k D_rk H_qk
      float t = D[r * 3 + q] + D[r * 3 + 0] * H[q * 3 + 0] + D[r * 3 + 1] * H[q * 3 + 1] + D[r * 3 + 2] * H[q * 3 + 2];
      tau[r * 3 + q] = tm * t + (r == q ? pr : 0.f);
    }
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

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_grid_update(Batch b, int substep, float dt, int clear) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n == 0) *b.movers = 0;  // the sort of the previous transfer has consumed it
  if (n >= b.Nnodes) return;
  const int ii = find_instance(b.node_offs, b.n_inst, n);
  const Instance &I = b.inst[ii];
  const long long loc = n - I.node_off;
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
  const int i = (int)(loc % G0);
  const int j = (int)((loc / G0) % G1);
  const int k = (int)(loc / ((long long)G0 * G1));
  const float4 mm = b.gmm[n];
  float V0 = 0.f, V1 = 0.f, V2 = 0.f;
  if (mm.x > 0.f) {  // Eq. 6; empty nodes keep V = 0
    V0 = mm.y / mm.x + I.gdt[0] * dt;
    V1 = mm.z / mm.x + I.gdt[1] * dt;
    V2 = mm.w / mm.x + I.gdt[2] * dt;
  }
  if (I.shape.kind != IND_NONE) {
    const IndenterFrame f = I.frames[substep];
    if (inside_indenter(I.shape, f, i, j, k)) {  // rigid indenter velocity
      const float r0 = ((float)i - f.c[0]) * I.dx;
      const float r1 = ((float)j - f.c[1]) * I.dx;
      const float r2 = ((float)k - f.c[2]) * I.dx;
      V0 = f.vlin[0] + (f.w[1] * r2 - f.w[2] * r1);
      V1 = f.vlin[1] + (f.w[2] * r0 - f.w[0] * r2);
      V2 = f.vlin[2] + (f.w[0] * r1 - f.w[1] * r0);
    }
  }
  if (I.fix_base && k <= I.pad_bottom) V0 = V1 = V2 = 0.f;  // sensor base, Eq. 10
  if (i < 2 || j < 2 || k < 2 || i > G0 - 3 || j > G1 - 3 || k > G2 - 3) V0 = V1 = V2 = 0.f;
  b.gv[n] = make_float4(V0, V1, V2, 0.f);
  if (clear) b.gmm[n] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
template <int BX, int BY, int BZ, int MODE>
__global__ void __launch_bounds__(256) k_transfer(Batch b, float dt) {
  constexpr bool DO_G2P = (MODE & XFER_G2P) != 0;
  constexpr bool DO_P2G = (MODE & XFER_P2G) != 0;
  constexpr int TX = BX + 4, TY = BY + 4, TZ = BZ + 4, TN = TX * TY * TZ;
  extern __shared__ float tile[];  // [4][TN] when DO_P2G
  __shared__ int s_moved;

  const long long gblk = blockIdx.x;
  const uint32_t start = b.bstart[gblk], end = b.bstart[gblk + 1];
  if (start == end) return;
  const int ii = b.block_inst[gblk];
  const Instance &I = b.inst[ii];
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
  const long long lb = gblk - I.block_off;
  const int nb0 = I.nb[0], nb1 = I.nb[1];
  const int cbx = (int)(lb % nb0), cby = (int)((lb / nb0) % nb1), cbz = (int)(lb / ((long long)nb0 * nb1));
  const int T0x = cbx * BX - 1, T0y = cby * BY - 1, T0z = cbz * BZ - 1;
  const long long Ntot = b.Ntot;
  const float inv_dx = I.inv_dx, dx = I.dx, m = I.m;

  if (DO_P2G)
    for (int t = threadIdx.x; t < 4 * TN; t += blockDim.x) tile[t] = 0.f;
  if (threadIdx.x == 0) s_moved = 0;
  __syncthreads();

  for (uint32_t it = start + threadIdx.x; it < end; it += blockDim.x) {
    const uint32_t p = b.idx[it];
    float u[3] = {b.u[p], b.u[Ntot + p], b.u[2 * Ntot + p]};
    float H[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) H[e] = b.Fm[e * Ntot + p];
    float v[3], Bm[9];  // Bm = sum_i w V (i - f)^T (cells); C = 4/dx Bm
    int err = 0;

    if (DO_G2P) {
      int bs[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bs[a] = (int)floorf(u[a] - 0.5f);
        f[a] = u[a] - (float)bs[a];
      }
      if (bs[0] < 0 || bs[1] < 0 || bs[2] < 0 || bs[0] > G0 - 3 || bs[1] > G1 - 3 || bs[2] > G2 - 3) {
        err |= ERRBIT_OUT_OF_GRID;  // keep memory access inside the grid
        bs[0] = clampi(bs[0], 0, G0 - 3);
        bs[1] = clampi(bs[1], 0, G1 - 3);
        bs[2] = clampi(bs[2], 0, G2 - 3);
        f[0] = f[1] = f[2] = 1.0f;
      }
      float wx[3], wy[3], wz[3], dpx[3], dpy[3], dpz[3];
      bspline3(f[0], wx, dpx);
      bspline3(f[1], wy, dpy);
      bspline3(f[2], wz, dpz);
      float wdx[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) wdx[i] = wx[i] * dpx[i];
#pragma unroll
      for (int e = 0; e < 9; ++e) Bm[e] = 0.f;
      v[0] = v[1] = v[2] = 0.f;
      const float4 *gv = b.gv + I.node_off;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float4 *row = gv + ((long long)(bs[2] + k) * G1 + (bs[1] + j)) * G0 + bs[0];
          const float4 V0 = __ldg(row), V1 = __ldg(row + 1), V2 = __ldg(row + 2);
          // row sums over i: s = sum w_i V_i, t = sum w_i (i - f_x) V_i
          const float s0 = wx[0] * V0.x + wx[1] * V1.x + wx[2] * V2.x;
          const float s1 = wx[0] * V0.y + wx[1] * V1.y + wx[2] * V2.y;
          const float s2 = wx[0] * V0.z + wx[1] * V1.z + wx[2] * V2.z;
          const float t0 = wdx[0] * V0.x + wdx[1] * V1.x + wdx[2] * V2.x;
          const float t1 = wdx[0] * V0.y + wdx[1] * V1.y + wdx[2] * V2.y;
          const float t2 = wdx[0] * V0.z + wdx[1] * V1.z + wdx[2] * V2.z;
          const float wjk = wy[j] * wz[k];
          const float wjy = wjk * dpy[j], wjz = wjk * dpz[k];
          v[0] += wjk * s0; v[1] += wjk * s1; v[2] += wjk * s2;               // Eq. 7
          Bm[0] += wjk * t0; Bm[3] += wjk * t1; Bm[6] += wjk * t2;            // Eq. 8
          Bm[1] += wjy * s0; Bm[4] += wjy * s1; Bm[7] += wjy * s2;
          Bm[2] += wjz * s0; Bm[5] += wjz * s1; Bm[8] += wjz * s2;
        }
      // Eq. 9: F <- (I + dt C) F, i.e. H <- H + dt C (I + H), C = 4/dx Bm
      const float c4 = 4.0f * dt * inv_dx;
      float Hn[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float M0 = (q == 0 ? 1.f : 0.f) + H[0 * 3 + q];
          const float M1 = (q == 1 ? 1.f : 0.f) + H[1 * 3 + q];
          const float M2 = (q == 2 ? 1.f : 0.f) + H[2 * 3 + q];
          Hn[r * 3 + q] = H[r * 3 + q] + c4 * (Bm[r * 3 + 0] * M0 + Bm[r * 3 + 1] * M1 + Bm[r * 3 + 2] * M2);
        }
#pragma unroll
      for (int e = 0; e < 9; ++e) H[e] = Hn[e];
      if (I.fix_base && (b.flags[p] & 1)) v[0] = v[1] = v[2] = 0.f;  // Eq. 10
#pragma unroll
      for (int a = 0; a < 3; ++a) u[a] = u[a] + dt * inv_dx * v[a];  // Eq. 11
      // the particle's new stencil must stay clear of the padding band
      int nbs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) nbs[a] = (int)floorf(u[a] - 0.5f);
      if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) err |= ERRBIT_NUMERICAL;
      if (nbs[0] < 2 || nbs[1] < 2 || nbs[2] < 2 || nbs[0] > G0 - 5 || nbs[1] > G1 - 5 || nbs[2] > G2 - 5)
        err |= ERRBIT_OUT_OF_GRID;
      if (nbs[0] < T0x + 1 || nbs[0] > T0x + BX || nbs[1] < T0y + 1 || nbs[1] > T0y + BY ||
          nbs[2] < T0z + 1 || nbs[2] > T0z + BZ)
        s_moved = 1;  // left its sort block: re-sort after this transfer
      b.u[p] = u[0];
      b.u[Ntot + p] = u[1];
      b.u[2 * Ntot + p] = u[2];
#pragma unroll
      for (int e = 0; e < 9; ++e) b.Fm[e * Ntot + p] = H[e];
      if (!DO_P2G) {
#pragma unroll
        for (int a = 0; a < 3; ++a) b.v[a * Ntot + p] = v[a];
#pragma unroll
        for (int e = 0; e < 9; ++e) b.C[e * Ntot + p] = 4.0f * inv_dx * Bm[e];
      }
    } else {
      // first transfer of a step: v and C come from the stored state
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = b.v[a * Ntot + p];
#pragma unroll
      for (int e = 0; e < 9; ++e) Bm[e] = 0.25f * dx * b.C[e * Ntot + p];
    }

    if (DO_P2G) {
      // Eqs. 2-5 with S_p = tau and the affine term of Eq. 4 carrying m_p:
      // MG_i += w (m v + A (X_i - x)),  A (X_i - x) = Abar (i - f),
      // Abar = dx (m C - dt V0 (4/dx^2) tau) = 4 m Bm - (4 dt V0 / dx) tau.
      float tau[9];
      const float Jm1 = kirchhoff_stress(H, I.mu, I.la, tau);
      if (!(1.0f + Jm1 > 0.f)) err |= ERRBIT_NUMERICAL;
      const float ks = 4.0f * dt * I.V0 * inv_dx;
      float A[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) A[e] = 4.0f * m * Bm[e] - ks * tau[e];
      int bs[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bs[a] = (int)floorf(u[a] - 0.5f);
        f[a] = u[a] - (float)bs[a];
      }
      const int lx = bs[0] - T0x, ly = bs[1] - T0y, lz = bs[2] - T0z;
      if (lx < 0 || ly < 0 || lz < 0 || lx > TX - 3 || ly > TY - 3 || lz > TZ - 3 || (err & ERRBIT_NUMERICAL)) {
        err |= ERRBIT_CFL;  // moved a cell or more in one substep: not scattered
      } else {
        float wx[3], wy[3], wz[3], dpx[3], dpy[3], dpz[3];
        bspline3(f[0], wx, dpx);
        bspline3(f[1], wy, dpy);
        bspline3(f[2], wz, dpz);
        float ax[3][3], ay[3][3], az[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            ax[i][a] = A[a * 3 + 0] * dpx[i];
            ay[i][a] = A[a * 3 + 1] * dpy[i];
            az[i][a] = A[a * 3 + 2] * dpz[i];
          }
        const float mv0 = m * v[0], mv1 = m * v[1], mv2 = m * v[2];
        float wxm[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) wxm[i] = wx[i] * m;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float wjk = wy[j] * wz[k];
            const float q0 = mv0 + ay[j][0] + az[k][0];
            const float q1 = mv1 + ay[j][1] + az[k][1];
            const float q2 = mv2 + ay[j][2] + az[k][2];
            float *t = tile + ((lz + k) * TY + (ly + j)) * TX + lx;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const float w = wx[i] * wjk;
              atomicAdd(t + i, wxm[i] * wjk);                       // Eq. 2
              atomicAdd(t + TN + i, w * (q0 + ax[i][0]));           // Eqs. 3-5
              atomicAdd(t + 2 * TN + i, w * (q1 + ax[i][1]));
              atomicAdd(t + 3 * TN + i, w * (q2 + ax[i][2]));
            }
          }
      }
    }
    if (err) atomicOr(b.err, err);
  }
  __syncthreads();
  if (DO_G2P && threadIdx.x == 0 && s_moved) *b.movers = 1;
  if (DO_P2G) {
    float4 *gmm = b.gmm + I.node_off;
    for (int t = threadIdx.x; t < TN; t += blockDim.x) {
      const float mass = tile[t];
      if (mass == 0.f) continue;
      const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
      const int gx = T0x + tx, gy = T0y + ty, gz = T0z + tz;
      if (gx < 0 || gy < 0 || gz < 0 || gx >= G0 || gy >= G1 || gz >= G2) continue;
      atomicAdd(gmm + ((long long)gz * G1 + gy) * G0 + gx,
                make_float4(mass, tile[TN + t], tile[2 * TN + t], tile[3 * TN + t]));
    }
  }
}

// ---------------------------------------------------------------------------
// Block of a particle: its stencil base cell floor(u - 1/2), divided by the
// block size, clamped into the instance's block grid.
__device__ __forceinline__ uint32_t particle_block(const Batch &b, const Instance &I, SortBlock blk,
                                                   long long p) {
  const int bx = clampi((int)floorf(b.u[p] - 0.5f), 0, I.G[0] - 1) / blk.x;
  const int by = clampi((int)floorf(b.u[b.Ntot + p] - 0.5f), 0, I.G[1] - 1) / blk.y;
  const int bz = clampi((int)floorf(b.u[2 * b.Ntot + p] - 0.5f), 0, I.G[2] - 1) / blk.z;
  const int cx = clampi(bx, 0, I.nb[0] - 1), cy = clampi(by, 0, I.nb[1] - 1), cz = clampi(bz, 0, I.nb[2] - 1);
  return (uint32_t)(I.block_off + ((long long)cz * I.nb[1] + cy) * I.nb[0] + cx);
}

__global__ void __launch_bounds__(256) k_sort_keys(Batch b, SortBlock blk, int force) {
  if (!force && *(volatile int *)b.movers == 0) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < b.Ntot;
  uint32_t key = 0xFFFFFFFFu;
  if (valid) {
    const int ii = find_instance(b.part_offs, b.n_inst, p);
    key = particle_block(b, b.inst[ii], blk, p);
    b.key[p] = key;
  }
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
  const int leader = __ffs(peers) - 1;
  if (valid && (int)(threadIdx.x & 31) == leader) atomicAdd(b.bcount + key, (uint32_t)__popc(peers));
}

// Exclusive scan of the block counts by one CTA of 1024 threads; also sets
// the scatter cursors and clears the counts for the next sort.
__global__ void __launch_bounds__(1024) k_sort_scan(Batch b, int force) {
  if (!force && *(volatile int *)b.movers == 0) return;
  __shared__ uint32_t warp_tot[32];
  const long long n = b.Nblk;
  const int T = blockDim.x;
  const long long per = (n + T - 1) / T;
  const long long lo = threadIdx.x * per;
  const long long hi = lo + per < n ? lo + per : n;
  uint32_t local = 0;
  for (long long i = lo; i < hi; ++i) local += b.bcount[i];
  // inclusive scan of the per-thread totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < (T >> 5) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t run = x - local + (wid > 0 ? warp_tot[wid - 1] : 0u);
  for (long long i = lo; i < hi; ++i) {
    const uint32_t c = b.bcount[i];
    b.bstart[i] = run;
    b.cursor[i] = run;
    b.bcount[i] = 0u;
    run += c;
  }
  if (threadIdx.x == T - 1) b.bstart[n] = run;
}

__global__ void __launch_bounds__(256) k_sort_scatter(Batch b, int force) {
  if (!force && *(volatile int *)b.movers == 0) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < b.Ntot;
  const uint32_t key = valid ? b.key[p] : 0xFFFFFFFFu;
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (valid && lane == leader) base = atomicAdd(b.cursor + key, (uint32_t)__popc(peers));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (valid) b.idx[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)p;
}

// ---------------------------------------------------------------------------
cudaError_t launch_grid_update(const Batch &b, int substep, float dt, int clear, cudaStream_t st) {
  const long long nb = (b.Nnodes + 255) / 256;
  k_grid_update<<<(unsigned)nb, 256, 0, st>>>(b, substep, dt, clear);
  return cudaGetLastError();
}

template <int BX, int BY, int BZ>
static cudaError_t launch_transfer_t(const Batch &b, int mode, float dt, cudaStream_t st) {
  constexpr int TN = (BX + 4) * (BY + 4) * (BZ + 4);
  const size_t smem = (mode & XFER_P2G) ? 4 * TN * sizeof(float) : 0;
  const unsigned grid = (unsigned)b.Nblk;
  switch (mode) {
    case XFER_P2G:
      k_transfer<BX, BY, BZ, XFER_P2G><<<grid, 256, smem, st>>>(b, dt);
      break;
    case XFER_G2P:
      k_transfer<BX, BY, BZ, XFER_G2P><<<grid, 256, smem, st>>>(b, dt);
      break;
    case XFER_FUSED:
      k_transfer<BX, BY, BZ, XFER_FUSED><<<grid, 256, smem, st>>>(b, dt);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_transfer(const Batch &b, SortBlock blk, int mode, float dt, cudaStream_t st) {
  if (b.Nblk == 0) return cudaSuccess;
  if (blk.x == 8 && blk.y == 8 && blk.z == 4) return launch_transfer_t<8, 8, 4>(b, mode, dt, st);
  if (blk.x == 4 && blk.y == 4 && blk.z == 4) return launch_transfer_t<4, 4, 4>(b, mode, dt, st);
  if (blk.x == 8 && blk.y == 8 && blk.z == 8) return launch_transfer_t<8, 8, 8>(b, mode, dt, st);
  if (blk.x == 16 && blk.y == 8 && blk.z == 4) return launch_transfer_t<16, 8, 4>(b, mode, dt, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sort(const Batch &b, SortBlock blk, int force, cudaStream_t st) {
  if (b.Ntot == 0) return cudaSuccess;
  const unsigned gp = (unsigned)((b.Ntot + 255) / 256);
  k_sort_keys<<<gp, 256, 0, st>>>(b, blk, force);
  k_sort_scan<<<1, 1024, 0, st>>>(b, force);
  k_sort_scatter<<<gp, 256, 0, st>>>(b, force);
  return cudaGetLastError();
}

}  // namespace tacchi
