// transfer3.cu -- the MLS-MPM transfer kernel with three threads per cell
// (Tacchi, arXiv 2301.08343, Sec. III-A: G2P of substep k, Eqs. 7-11, fused
// with P2G of substep k+1, Eqs. 2-5).
//
// Like k_transfer (mpm.cu), one CTA takes one sort block of cells, groups its
// particles by home cell (the stencil base floor(u - 1/2)) in shared memory
// and accumulates each cell's P2G contributions in registers before adding
// them to the grid.  The difference is how a cell is split over
// threads.  Here three threads of a warp share a cell:
//   * particle work is split by particle: thread r of the triple runs G2P,
//     the F update, advection and the polar stress for particles r, r + 3,
//     r + 6, ... of the cell, so no particle is computed twice;
//   * P2G is split by node plane: thread r owns the nine nodes of plane
//     k = r of the cell's 3 x 3 x 3 stencil and adds every particle of the
//     cell to them, receiving the other two particles of each round (their
//     fractional position, m v and the affine matrix A: 15 floats) by warp
//     shuffles.
// A thread therefore holds 36 accumulators instead of a whole cell's 108,
// which brings it under 128 registers and doubles the warps an SM keeps
// resident.  Lanes 30 and 31 of each warp take no cell.  Each thread adds its
// plane's sums to the grid with vector reductions to global memory.
#include "mpm_device.cuh"

namespace tacchi {

template <int BX, int BY, int BZ, int THREADS_>
struct Xfer3Plan {
  static constexpr int THREADS = THREADS_;
  static constexpr int NT = THREADS / 32 * 10;                      // cell triples per CTA
  static constexpr int EX = BX + 2, EY = BY + 2, EZ = BZ + 2;       // home cells [B0-1, B0+B]
  static constexpr int NE = EX * EY * EZ;
  static constexpr int VX = BX + 4, VY = BY + 4, VZ = BZ + 4;       // V tile, nodes [B0-1, B0+B+3)
  static constexpr int VN = VX * VY * VZ;
  static constexpr int MAXP = 12 * BX * BY * BZ;                    // particles grouped in smem (1.5x nominal)
  static constexpr int PER = (NE + 1 + THREADS - 1) / THREADS;      // scan entries per thread
  static constexpr size_t OFF_KEY = 0;                              // u32 [MAXP] rank and cell per particle
  static constexpr size_t OFF_V = OFF_KEY + 4 * (size_t)MAXP;       // float4 [VN]
  static constexpr size_t OFF_LIST = OFF_V + 16 * (size_t)VN;       // u32 [MAXP] particles by cell
  static constexpr size_t OFF_PID = OFF_LIST + 4 * (size_t)MAXP;    // u32 [MAXP] particle ids in idx order
  static constexpr size_t OFF_CNT = OFF_PID + 4 * (size_t)MAXP;     // u32 [NE] counts
  static constexpr size_t OFF_START = OFF_CNT + 4 * (size_t)NE;     // u32 [NE + 1]
  static constexpr size_t OFF_CELLS = OFF_START + 4 * (size_t)(NE + 1);  // u16 [NE] non-empty cells
  static constexpr size_t OFF_ORDER = OFF_CELLS + 2 * (size_t)NE;   // u16 [NE] cells, heaviest class first
  static constexpr size_t OFF_STAGE = (OFF_ORDER + 2 * (size_t)NE + 15) / 16 * 16;  // float4 [2][3][THREADS]
  static constexpr size_t BYTES = OFF_STAGE + 16 * 2 * 3 * (size_t)THREADS;
  static_assert(THREADS % 32 == 0, "whole warps");
};

// Register budget: THREADS x 128 registers per CTA, so that 65,536 / (THREADS
// x 128) CTAs share an SM.
template <int BX, int BY, int BZ, int THREADS, int MODE>
__global__ void __launch_bounds__(THREADS, 65536 / (THREADS * 128)) k_transfer3(Batch b, float dt) {
  using P = Xfer3Plan<BX, BY, BZ, THREADS>;
  constexpr bool DO_G2P = (MODE & XFER_G2P) != 0;
  constexpr bool DO_P2G = (MODE & XFER_P2G) != 0;
  constexpr int VX = P::VX, VY = P::VY, VZ = P::VZ;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_key = reinterpret_cast<uint32_t *>(smem + P::OFF_KEY);
  float4 *vt = reinterpret_cast<float4 *>(smem + P::OFF_V);
  uint32_t *s_list = reinterpret_cast<uint32_t *>(smem + P::OFF_LIST);
  uint32_t *s_pid = reinterpret_cast<uint32_t *>(smem + P::OFF_PID);
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + P::OFF_CNT);
  uint32_t *s_start = reinterpret_cast<uint32_t *>(smem + P::OFF_START);
  uint16_t *s_cells = reinterpret_cast<uint16_t *>(smem + P::OFF_CELLS);
  uint16_t *s_order = reinterpret_cast<uint16_t *>(smem + P::OFF_ORDER);
  __shared__ uint32_t s_warp[THREADS / 32];
  __shared__ unsigned long long s_warp64[THREADS / 32];
  __shared__ int s_moved, s_overflow;

  const long long gblk = blockIdx.x;
  const uint32_t start = b.bstart[gblk], end = b.bstart[gblk + 1];
  if (start == end) return;
  const uint32_t n = end - start;
  const int ii = b.block_inst[gblk];
  const Instance &I = b.inst[ii];
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
  const long long lb = gblk - I.block_off;
  const int nb0 = I.nb[0], nb1 = I.nb[1];
  const int B0x = (int)(lb % nb0) * BX, B0y = (int)((lb / nb0) % nb1) * BY,
            B0z = (int)(lb / ((long long)nb0 * nb1)) * BZ;
  const long long Ntot = b.Ntot;
  const float inv_dx = I.inv_dx, dx = I.dx, m = I.m, mu = I.mu, la = I.la;
  const bool fix_base = I.fix_base != 0;
  const long long node_off = I.node_off;
  const float c4 = 4.0f * dt * inv_dx;
  const float ks = 4.0f * dt * I.V0 * inv_dx;
  const int tid = threadIdx.x;
  float4 *__restrict__ gps = b.ps;
  const uint8_t *__restrict__ gfl = b.flags;

  // ---- grid velocities of nodes [B0-1, B0+B+3) into the V tile, copied
  // asynchronously while the particles are grouped (zeros outside the grid)
  if (DO_G2P) {
    const float4 *gv = b.gv + node_off;
    for (int t = tid; t < P::VN; t += THREADS) {
      const int x = B0x - 1 + t % VX, y = B0y - 1 + (t / VX) % VY, z = B0z - 1 + t / (VX * VY);
      const bool in = x >= 0 && y >= 0 && z >= 0 && x < G0 && y < G1 && z < G2;
      cp_async16_zfill(vt + t, in ? gv + ((long long)z * G1 + y) * G0 + x : gv, in);
    }
  }
  cp_async_commit();

  // ---- group the block's particles by home cell
  for (int c = tid; c < P::NE; c += THREADS) s_cnt[c] = 0;
  if (tid == 0) {
    s_moved = 0;
    s_overflow = n > (uint32_t)P::MAXP;
  }
  __syncthreads();
  if (n <= (uint32_t)P::MAXP) {
    constexpr int GB = 2048 / THREADS;  // loads in flight per thread
    for (uint32_t l0 = 0; l0 < n; l0 += GB * THREADS) {
      uint32_t pp[GB];
      float4 px[GB];
#pragma unroll
      for (int g = 0; g < GB; ++g) {
        const uint32_t l = l0 + g * THREADS + tid;
        pp[g] = l < n ? b.idx[start + l] : 0u;
      }
#pragma unroll
      for (int g = 0; g < GB; ++g) {
        const uint32_t l = l0 + g * THREADS + tid;
        px[g] = l < n ? load_position(gps, pp[g]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int g = 0; g < GB; ++g) {
        const uint32_t l = l0 + g * THREADS + tid;
        if (l >= n) continue;
        s_pid[l] = pp[g];
        const int ex = (int)floorf(px[g].x - 0.5f) - (B0x - 1);
        const int ey = (int)floorf(px[g].y - 0.5f) - (B0y - 1);
        const int ez = (int)floorf(px[g].z - 0.5f) - (B0z - 1);
        uint32_t key = 0xFFFFFFFFu;
        if (ex >= 0 && ey >= 0 && ez >= 0 && ex < P::EX && ey < P::EY && ez < P::EZ) {
          const uint32_t c = (uint32_t)((ez * P::EY + ey) * P::EX + ex);
          key = (atomicAdd(s_cnt + c, 1u) << 12) | c;  // rank, cell (< 4096)
        } else {
          s_overflow = 1;  // not at home: the sort invariant is broken
        }
        s_key[l] = key;
      }
    }
  }
  __syncthreads();
  const bool grouped = !s_overflow;
  uint32_t ncells = 0;
  if (grouped) {
    ncells = block_scan_compact<THREADS, P::PER>(s_cnt, s_start, s_cells, P::NE, s_warp);
    for (uint32_t l = tid; l < n; l += THREADS) {
      const uint32_t key = s_key[l];
      s_list[s_start[key & 0xFFFu] + (key >> 12)] = s_pid[l];
    }
    order_cells_by_load<THREADS, P::PER>(s_cells, s_start, (int)ncells, s_order, s_warp64);
  }
  __syncthreads();
  cp_async_wait<0>();  // this thread's part of the V tile
  __syncthreads();

  // One particle: G2P against the V tile (Eqs. 7-11) or, for the first
  // transfer of a step, v and C from the stored state; then the stress and
  // the P2G inputs of Eqs. 2-5: A = 4 m Bm - (4 dt V0 / dx) tau (so that the
  // momentum added to node i is w (m v + A (i - f)), Eq. 4 with m_p on the
  // affine term) and f, the position from the new stencil base nbs.
  // Returns error bits; sets `moved` when the particle left its home range.
  auto particle = [&](uint32_t p, uint32_t fl, float u[3], float H[9], float f[3], int nbs[3], float mv[3],
                      float A[9]) -> int {
    int err = 0;
    float v[3], Bm[9];  // Bm = sum_i w V (i - f)^T (cells); C = 4/dx Bm
    if (DO_G2P) {
      int bs[3];
      float fo[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bs[a] = (int)floorf(u[a] - 0.5f);
        fo[a] = u[a] - (float)bs[a];
      }
      float wx[3], wy[3], wz[3], dpx[3], dpy[3], dpz[3];
      bspline3(fo[0], wx, dpx);
      bspline3(fo[1], wy, dpy);
      bspline3(fo[2], wz, dpz);
      float2 wxd[3], wdxd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        wxd[i] = make_float2(wx[i], wx[i]);
        wdxd[i] = make_float2(wx[i] * dpx[i], wx[i] * dpx[i]);
      }
      const float2 z2 = make_float2(0.f, 0.f);
      float2 vxy = z2, b0xy = z2, b1xy = z2, b2xy = z2;  // v (Eq. 7), Bm columns (Eq. 8), rows x, y
      float vz = 0.f, b0z = 0.f, b1z = 0.f, b2z = 0.f;    // row z
      // home cells lie inside the V tile; clamp only as a guard
      const int vx = clampi(bs[0] - (B0x - 1), 0, VX - 3), vy = clampi(bs[1] - (B0y - 1), 0, VY - 3),
                vz0 = clampi(bs[2] - (B0z - 1), 0, VZ - 3);
      if (vx != bs[0] - (B0x - 1) || vy != bs[1] - (B0y - 1) || vz0 != bs[2] - (B0z - 1)) err |= ERRBIT_CFL;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float4 *row = vt + ((vz0 + k) * VY + (vy + j)) * VX + vx;
          const float4 V0 = row[0], V1 = row[1], V2 = row[2];
          float2 sxy = __fmul2_rn(wxd[0], make_float2(V0.x, V0.y));
          float2 txy = __fmul2_rn(wdxd[0], make_float2(V0.x, V0.y));
          sxy = __ffma2_rn(wxd[1], make_float2(V1.x, V1.y), sxy);
          txy = __ffma2_rn(wdxd[1], make_float2(V1.x, V1.y), txy);
          sxy = __ffma2_rn(wxd[2], make_float2(V2.x, V2.y), sxy);
          txy = __ffma2_rn(wdxd[2], make_float2(V2.x, V2.y), txy);
          const float sz = wx[0] * V0.z + wx[1] * V1.z + wx[2] * V2.z;
          const float tz = wdxd[0].x * V0.z + wdxd[1].x * V1.z + wdxd[2].x * V2.z;
          const float wjk = wy[j] * wz[k];
          const float wjy = wjk * dpy[j], wjz = wjk * dpz[k];
          vxy = __ffma2_rn(make_float2(wjk, wjk), sxy, vxy);      // Eq. 7
          b0xy = __ffma2_rn(make_float2(wjk, wjk), txy, b0xy);    // Eq. 8
          b1xy = __ffma2_rn(make_float2(wjy, wjy), sxy, b1xy);
          b2xy = __ffma2_rn(make_float2(wjz, wjz), sxy, b2xy);
          vz += wjk * sz;
          b0z += wjk * tz;
          b1z += wjy * sz;
          b2z += wjz * sz;
        }
      v[0] = vxy.x; v[1] = vxy.y; v[2] = vz;
      Bm[0] = b0xy.x; Bm[1] = b1xy.x; Bm[2] = b2xy.x;
      Bm[3] = b0xy.y; Bm[4] = b1xy.y; Bm[5] = b2xy.y;
      Bm[6] = b0z; Bm[7] = b1z; Bm[8] = b2z;
      // Eq. 9: F <- (I + dt C) F, i.e. H <- H + dt C (I + H), C = 4/dx Bm
      float Hn[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float M0 = (c == 0 ? 1.f : 0.f) + H[0 * 3 + c];
          const float M1 = (c == 1 ? 1.f : 0.f) + H[1 * 3 + c];
          const float M2 = (c == 2 ? 1.f : 0.f) + H[2 * 3 + c];
          Hn[r * 3 + c] = H[r * 3 + c] + c4 * (Bm[r * 3 + 0] * M0 + Bm[r * 3 + 1] * M1 + Bm[r * 3 + 2] * M2);
        }
#pragma unroll
      for (int e = 0; e < 9; ++e) H[e] = Hn[e];
      if (fix_base && (fl & 1u)) v[0] = v[1] = v[2] = 0.f;  // Eq. 10
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float du = dt * inv_dx * v[a];
        if (!(fabsf(du) < 1.0f)) err |= ERRBIT_CFL;  // a cell or more in one substep
        u[a] = u[a] + du;  // Eq. 11
      }
      if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) err |= ERRBIT_NUMERICAL;
      store_particle(gps, p, u, H);
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
    // the particle's (new) stencil must stay clear of the padding band
#pragma unroll
    for (int a = 0; a < 3; ++a) nbs[a] = (int)floorf(u[a] - 0.5f);
    if (nbs[0] < 2 || nbs[1] < 2 || nbs[2] < 2 || nbs[0] > G0 - 5 || nbs[1] > G1 - 5 || nbs[2] > G2 - 5)
      err |= ERRBIT_OUT_OF_GRID;
    if (DO_G2P && (nbs[0] < B0x - 1 || nbs[0] > B0x + BX || nbs[1] < B0y - 1 || nbs[1] > B0y + BY ||
                   nbs[2] < B0z - 1 || nbs[2] > B0z + BZ))
      s_moved = 1;  // left its home cells: re-sort after this transfer
    if (DO_P2G) {
      // Eqs. 2-5 with S_p = tau: Abar = dx (m C - dt V0 (4/dx^2) tau)
      float tau[9];
      const float Jm1 = kirchhoff_stress(H, mu, la, tau);
      if (!(1.0f + Jm1 > 0.f)) err |= ERRBIT_NUMERICAL;
#pragma unroll
      for (int e = 0; e < 9; ++e) A[e] = 4.0f * m * Bm[e] - ks * tau[e];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        mv[a] = m * v[a];
        f[a] = u[a] - (float)nbs[a];
      }
    }
    return err;
  };

  if (grouped) {
    const int lane = tid & 31, warp = tid >> 5;
    if (lane < 30) {
      const int r = lane % 3;              // node plane k = r of the cell's stencil
      const int g = warp * 10 + lane / 3;  // cell triple
      const unsigned tmask = 7u << (lane - r);
      const int src1 = lane - r + (r + 1) % 3, src2 = lane - r + (r + 2) % 3;
      // weight of plane r at fraction f: the r-th of bspline3's three,
      // written as s_r (f - h_r)^2 + o_r
      const float h_r = 1.5f - 0.5f * (float)r;
      const float s_r = r == 1 ? -1.0f : 0.5f;
      const float o_r = r == 1 ? 0.75f : 0.0f;
      const float fr = (float)r;
      // round r0 gives triple g the cell at position r0 + g, mirrored on odd
      // rounds so the triples that took the heaviest cells of one round take
      // the lightest of the next
      auto work_of = [&](uint32_t r0) -> uint32_t {
        return r0 + (((r0 / P::NT) & 1u) ? (uint32_t)(P::NT - 1 - g) : (uint32_t)g);
      };
      // particle r of the triple's cell at round r0, if there is one
      auto first_of = [&](uint32_t r0, uint32_t &pout) -> bool {
        const uint32_t wk = work_of(r0);
        if (wk >= ncells) return false;
        const uint32_t c = s_order[wk];
        const uint32_t qa = s_start[c] + (uint32_t)r;
        if (qa >= s_start[c + 1]) return false;
        pout = s_list[qa];
        return true;
      };
      float4 *stage = reinterpret_cast<float4 *>(smem + P::OFF_STAGE) + tid;
      auto fetch = [&](uint32_t pp, int slot) {
        const float4 *src = gps + 3 * (long long)pp;
#pragma unroll
        for (int j = 0; j < 3; ++j) cp_async16(stage + (slot * 3 + j) * THREADS, src + j);
        cp_async_commit();
      };
      // pn: this thread's next particle; its record is in flight into stage
      // slot `slot` while `have` is set
      int slot = 0;
      uint32_t pn = 0, fln = 0;
      bool have = false;
      // accumulators of plane r: (MG x, MG y) and (MG z, sum of w) per node
      float2 acc01[9], acc2w[9];
      // P2G of one particle onto plane r
      auto accumulate = [&](const float f[3], const float mv[3], const float A[9]) {
        float wx[3], wy[3], dpx[3], dpy[3];
        bspline3(f[0], wx, dpx);
        bspline3(f[1], wy, dpy);
        const float tz = f[2] - h_r;
        const float wz = fmaf(s_r * tz, tz, o_r);
        const float dz = fr - f[2];
        const float2 Axy0 = make_float2(A[0], A[3]), Axy1 = make_float2(A[1], A[4]);
        float2 axy[3], ayxy[3];
        float axz[3], ayz[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          axy[i] = __fmul2_rn(Axy0, make_float2(dpx[i], dpx[i]));
          ayxy[i] = __fmul2_rn(Axy1, make_float2(dpy[i], dpy[i]));
          axz[i] = A[6] * dpx[i];
          ayz[i] = A[7] * dpy[i];
        }
        const float2 mvxy = make_float2(mv[0] + A[2] * dz, mv[1] + A[5] * dz);
        const float mvz = mv[2] + A[8] * dz;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float wjk = wy[j] * wz;
          const float2 wjk2 = make_float2(wjk, wjk);
          const float2 rxy = __fadd2_rn(mvxy, ayxy[j]);
          const float rz = mvz + ayz[j];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const int e = j * 3 + i;
            const float2 w2 = __fmul2_rn(make_float2(wx[i], wx[i]), wjk2);
            acc01[e] = __ffma2_rn(w2, __fadd2_rn(rxy, axy[i]), acc01[e]);          // Eqs. 3-5
            acc2w[e] = __ffma2_rn(w2, make_float2(rz + axz[i], 1.0f), acc2w[e]);  // and Eq. 2 (/ m)
          }
        }
      };
      for (uint32_t r0 = 0; r0 < ncells; r0 += P::NT) {
        const uint32_t wk = work_of(r0);
        if (wk >= ncells) break;  // later rounds give this triple later positions
        const uint32_t c = s_order[wk];
        const uint32_t q0 = s_start[c], q1 = s_start[c + 1];
        const int cx = (int)(c % P::EX), cy = (int)((c / P::EX) % P::EY), cz = (int)(c / (P::EX * P::EY));
        // a thread without a particle in the previous cell has not looked
        // ahead into this one
        if (!have && q0 + (uint32_t)r < q1) {
          pn = s_list[q0 + (uint32_t)r];
          fetch(pn, slot);
          if (DO_G2P) fln = gfl[pn];
          have = true;
        }
        if (DO_P2G) {
#pragma unroll
          for (int e = 0; e < 9; ++e) acc01[e] = acc2w[e] = make_float2(0.f, 0.f);
        }
        for (uint32_t qb = q0; qb < q1; qb += 3) {
          const uint32_t q = qb + (uint32_t)r;
          float pf[3] = {0.f, 0.f, 0.f}, pmv[3] = {0.f, 0.f, 0.f}, pA[9];
#pragma unroll
          for (int e = 0; e < 9; ++e) pA[e] = 0.f;
          int pok = 0;
          if (q < q1) {
            const uint32_t p = pn, fl = fln;
            const int cur = slot;
            bool ahead = false;
            if (q + 3 < q1) {
              pn = s_list[q + 3];
              ahead = true;
            } else {
              ahead = first_of(r0 + P::NT, pn);
            }
            if (ahead) {
              slot ^= 1;
              fetch(pn, slot);
              if (DO_G2P) fln = gfl[pn];
              cp_async_wait<1>();
            } else {
              cp_async_wait<0>();
            }
            have = ahead;
            float u[3], H[9];
            {
              const float4 a = stage[(cur * 3 + 0) * THREADS], bq = stage[(cur * 3 + 1) * THREADS],
                           cq = stage[(cur * 3 + 2) * THREADS];
              u[0] = a.x; u[1] = a.y; u[2] = a.z;
              H[0] = a.w; H[1] = bq.x; H[2] = bq.y; H[3] = bq.z; H[4] = bq.w;
              H[5] = cq.x; H[6] = cq.y; H[7] = cq.z; H[8] = cq.w;
            }
            int nbs[3];
            int err = particle(p, fl, u, H, pf, nbs, pmv, pA);
            if (DO_P2G) {
              const bool same_cell =
                  nbs[0] - (B0x - 1) == cx && nbs[1] - (B0y - 1) == cy && nbs[2] - (B0z - 1) == cz;
              if (err & ERRBIT_NUMERICAL) {
                err |= ERRBIT_CFL;  // not scattered
              } else if (same_cell) {
                pok = 1;
              } else {
                // changed cell during the substep: scatters on its own
                if (!scatter_particle_global(b.gmm + node_off, G0, G1, G2, nbs[0], nbs[1], nbs[2], m, pf, pmv, pA))
                  err |= ERRBIT_OUT_OF_GRID;  // stencil outside the grid: not scattered
              }
            }
            if (err) atomicOr(b.err, err);
          }
          if (DO_P2G) {
            // this thread's particle, then the other two of the round
            if (pok) accumulate(pf, pmv, pA);
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              const int src = o == 0 ? src1 : src2;
              const int ok = __shfl_sync(tmask, pok, src);
              float f2[3], mv2[3], A2[9];
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                f2[a] = __shfl_sync(tmask, pf[a], src);
                mv2[a] = __shfl_sync(tmask, pmv[a], src);
              }
#pragma unroll
              for (int e = 0; e < 9; ++e) A2[e] = __shfl_sync(tmask, pA[e], src);
              if (ok) accumulate(f2, mv2, A2);
            }
          }
        }
        if (DO_P2G) {
          // plane r of the cell's nodes straight to the grid, one vector
          // reduction per node; the cell's base node is B0 - 1 + c
          const int bx = B0x - 1 + cx, by = B0y - 1 + cy, bz = B0z - 1 + cz + r;
          float4 *g0 = b.gmm + node_off;
          const bool inside = bx >= 0 && by >= 0 && bz >= 0 && bx + 2 < G0 && by + 2 < G1 && bz < G2;
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const int e = j * 3 + i;
              if (inside || (bx + i >= 0 && by + j >= 0 && bz >= 0 && bx + i < G0 && by + j < G1 && bz < G2))
                atomicAdd(g0 + ((long long)bz * G1 + (by + j)) * G0 + (bx + i),
                          make_float4(m * acc2w[e].y, acc01[e].x, acc01[e].y, acc2w[e].x));
            }
        }
      }
      cp_async_wait<0>();
    }
  } else {
    // Grouping failed (a particle is not at home, or the block holds more
    // particles than the shared lists): one particle per thread, each
    // scattered on its own.
    for (uint32_t l = tid; l < n; l += THREADS) {
      const uint32_t p = b.idx[start + l];
      const uint32_t fl = DO_G2P ? gfl[p] : 0u;
      float u[3], H[9], f[3], mv[3], A[9];
      int nbs[3];
      load_particle(gps, p, u, H);
      int err = particle(p, fl, u, H, f, nbs, mv, A);
      if (DO_P2G) {
        if (err & ERRBIT_NUMERICAL)
          err |= ERRBIT_CFL;  // not scattered
        else if (!scatter_particle_global(b.gmm + node_off, G0, G1, G2, nbs[0], nbs[1], nbs[2], m, f, mv, A))
          err |= ERRBIT_OUT_OF_GRID;
      }
      if (err) atomicOr(b.err, err);
    }
  }
  __syncthreads();
  if (DO_G2P && tid == 0 && s_moved) *b.movers = 1;
}

template <int BX, int BY, int BZ, int THREADS>
static cudaError_t launch3_t(const Batch &b, int mode, float dt, cudaStream_t st) {
  using P = Xfer3Plan<BX, BY, BZ, THREADS>;
  const unsigned grid = (unsigned)b.Nblk;
  switch (mode) {
    case XFER_P2G:
      k_transfer3<BX, BY, BZ, THREADS, XFER_P2G><<<grid, THREADS, P::BYTES, st>>>(b, dt);
      break;
    case XFER_G2P:
      k_transfer3<BX, BY, BZ, THREADS, XFER_G2P><<<grid, THREADS, P::BYTES, st>>>(b, dt);
      break;
    case XFER_FUSED:
      k_transfer3<BX, BY, BZ, THREADS, XFER_FUSED><<<grid, THREADS, P::BYTES, st>>>(b, dt);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int BX, int BY, int BZ, int THREADS>
static cudaError_t prepare3_t() {
  const int smem = (int)Xfer3Plan<BX, BY, BZ, THREADS>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_transfer3<BX, BY, BZ, THREADS, XFER_P2G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_transfer3<BX, BY, BZ, THREADS, XFER_G2P>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_transfer3<BX, BY, BZ, THREADS, XFER_FUSED>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

bool transfer3_supported(SortBlock blk) {
  return (blk.x == 8 && blk.y == 8 && blk.z == 4) || (blk.x == 4 && blk.y == 4 && blk.z == 4);
}

cudaError_t prepare_transfer3(SortBlock blk) {
  if (blk.x == 8 && blk.y == 8 && blk.z == 4) return prepare3_t<8, 8, 4, 256>();
  if (blk.x == 4 && blk.y == 4 && blk.z == 4) return prepare3_t<4, 4, 4, 128>();
  return cudaErrorInvalidValue;
}

cudaError_t launch_transfer3(const Batch &b, SortBlock blk, int mode, float dt, cudaStream_t st) {
  if (b.Nblk == 0) return cudaSuccess;
  if (blk.x == 8 && blk.y == 8 && blk.z == 4) return launch3_t<8, 8, 4, 256>(b, mode, dt, st);
  if (blk.x == 4 && blk.y == 4 && blk.z == 4) return launch3_t<4, 4, 4, 128>(b, mode, dt, st);
  return cudaErrorInvalidValue;
}

}  // namespace tacchi
