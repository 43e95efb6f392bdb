// mpm.cu -- MLS-MPM substep kernels for sm_103a (Tacchi, arXiv 2301.08343,
// Sec. III-A).
//
//   k_grid_update  Eq. 6 (V = MG / M) fused with the rigid indenter (sticky,
//                  or slip: only the relative velocity into it removed), the
//                  fixed base (Eq. 10 on the grid) and the padding band.
//   k_transfer     one CTA per sort block of cells.  G2P of substep k
//                  (Eqs. 7-9, the base override of Eq. 10 and advection,
//                  Eq. 11) fused with P2G of substep k+1 (Eqs. 2-5), summed
//                  per cell in registers and added to the grid with vector
//                  reductions.
//                  P2G-only and G2P-only variants start and end a step.
//   k_sort_*       counting sort of particle ids by grid block, run only when
//                  a particle left its block during the last transfer.
#include "mpm_device.cuh"

namespace tacchi {

// ---------------------------------------------------------------------------
// Grid update of node n < Nnodes whose (M, MG) is mm.
__device__ __forceinline__ void grid_update_node(const Batch &b, long long n, float4 mm, int substep, float dt,
                                                 int clear) {
  const int ii = find_instance(b.node_offs, b.n_inst, n);
  const Instance &I = b.inst[ii];
  // an instance has fewer than 2^31 nodes: 32-bit index arithmetic
  const unsigned loc = (unsigned)(n - I.node_off);
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
  const unsigned row = loc / (unsigned)G0;
  const int i = (int)(loc - row * (unsigned)G0);
  const int k = (int)(row / (unsigned)G1);
  const int j = (int)(row - (unsigned)k * (unsigned)G1);
  float V0 = 0.f, V1 = 0.f, V2 = 0.f;
  if (mm.x > 0.f) {  // Eq. 6; empty nodes keep V = 0
    V0 = mm.y / mm.x + I.gdt[0] * dt;
    V1 = mm.z / mm.x + I.gdt[1] * dt;
    V2 = mm.w / mm.x + I.gdt[2] * dt;
  }
  if (I.shape.kind != IND_NONE && I.ind_np == 0) {  // grid-boundary indenter
    const IndenterFrame f = I.frames[substep];
    if (inside_indenter(I.shape, f, i, j, k)) {  // rigid indenter velocity
      const float r0 = ((float)i - f.c[0]) * I.dx;
      const float r1 = ((float)j - f.c[1]) * I.dx;
      const float r2 = ((float)k - f.c[2]) * I.dx;
      const float W0 = f.vlin[0] + (f.w[1] * r2 - f.w[2] * r1);
      const float W1 = f.vlin[1] + (f.w[2] * r0 - f.w[0] * r2);
      const float W2 = f.vlin[2] + (f.w[0] * r1 - f.w[1] * r0);
      if (I.slip && mm.x > 0.f) {
        // slip: only the velocity into the indenter, relative to it, is removed
        float nrm[3];
        indenter_normal(I.shape, f, i, j, k, nrm);
        const float q0 = V0 - W0, q1 = V1 - W1, q2 = V2 - W2;
        const float vn = q0 * nrm[0] + q1 * nrm[1] + q2 * nrm[2];
        if (vn < 0.f) {
          V0 = W0 + (q0 - vn * nrm[0]);
          V1 = W1 + (q1 - vn * nrm[1]);
          V2 = W2 + (q2 - vn * nrm[2]);
        }
      } else {  // sticky (the default), or an empty node
        V0 = W0;
        V1 = W1;
        V2 = W2;
      }
    }
  }
  if (I.fix_base && k <= I.pad_bottom) V0 = V1 = V2 = 0.f;  // sensor base, Eq. 10
  if (i < 2 || j < 2 || k < 2 || i > G0 - 3 || j > G1 - 3 || k > G2 - 3) V0 = V1 = V2 = 0.f;
  b.gv[n] = make_float4(V0, V1, V2, 0.f);
  if (clear) b.gmm[n] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Six resident CTAs per SM (40 registers): the pass reads the grid sums the
// transfer just reduced into L2 and is latency bound; at the 55 registers it
// takes unbounded only four CTAs fit (C1: 4.4% of the step against 4.8%).
__global__ void __launch_bounds__(256, 6) k_grid_update(Batch b, int substep, float dt, int clear) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n == 0) *b.movers = 0;  // the sort of the previous transfer has consumed it
  if (n < b.Nnodes) grid_update_node(b, n, b.gmm[n], substep, dt, clear);
}

// The grid update over every node by all threads of a persistent grid, with
// UNR nodes' loads in flight per thread (the persistent grid has far fewer
// threads than nodes, and the pass is bound by HBM latency otherwise; eight
// measured no better than four).
__device__ __forceinline__ void grid_update_all(const Batch &b, int substep, float dt, int clear) {
  constexpr int UNR = 4;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gt == 0) *b.movers = 0;
  for (long long q0 = gt; q0 < b.Nnodes; q0 += UNR * nth) {
    float4 mm[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const long long q = q0 + u * nth;
      mm[u] = q < b.Nnodes ? b.gmm[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const long long q = q0 + u * nth;
      if (q < b.Nnodes) grid_update_node(b, q, mm[u], substep, dt, clear);
    }
  }
}

// ---------------------------------------------------------------------------
// Transfer kernel.  One CTA per sort block of BX x BY x BZ cells with origin
// B0.  A particle belongs to the block while its stencil base ("home cell")
// stays within one cell of it, cells [B0-1, B0+B]; the sort runs only after
// some particle leaves that range.  The CTA groups its particles by home cell
// (counting sort in shared memory) and gives each non-empty cell to one
// thread, which runs G2P for the cell's particles against the shared
// velocity tile and accumulates their P2G contributions to the cell's 27
// nodes in registers; the accumulators reach the grid once per cell, by
// vector reductions to global memory.  A particle whose stencil base changes
// during the substep scatters on its own, also straight to the grid.
template <int BX, int BY, int BZ>
struct XferPlan {
  static constexpr int THREADS = 128;
  static constexpr int EX = BX + 2, EY = BY + 2, EZ = BZ + 2;       // home cells
  static constexpr int NE = EX * EY * EZ;
  static constexpr int VX = BX + 4, VY = BY + 4, VZ = BZ + 4;       // V tile, nodes [B0-1, B0+B+3)
  static constexpr int VN = VX * VY * VZ;
  // particles grouped in shared memory: 1.5x the nominal 8 per cell, 1.25x
  // for blocks of 512 cells or more (a fuller block takes the ungrouped path)
  static constexpr int MAXP = (BX * BY * BZ >= 512 ? 10 : 12) * BX * BY * BZ;
  static constexpr int PER = (NE + 1 + THREADS - 1) / THREADS;      // scan entries per thread
  // per-thread staging of the next particle record: float4 [2 slots][3][THREADS]
  static constexpr size_t STAGE_BYTES = 16 * 2 * 3 * (size_t)THREADS;
  // byte offsets in dynamic shared memory
  static constexpr size_t OFF_KEY = 0;                              // u32 [MAXP] rank and cell per particle
  // u32 [MAXP + 8] particle ids in idx order (8 spare for a 16-byte-aligned copy)
  static constexpr size_t OFF_PID = OFF_KEY + 4 * (size_t)MAXP;
  static constexpr size_t OFF_V = (OFF_PID + 4 * (size_t)(MAXP + 8) + 15) / 16 * 16;  // float4 [VN]
  static constexpr size_t OFF_LIST = OFF_V + 16 * (size_t)VN;       // u32 [MAXP] particles by cell
  static constexpr size_t OFF_CNT = OFF_LIST + 4 * (size_t)MAXP;    // u32 [NE] count, then start
  static constexpr size_t OFF_START = OFF_CNT + 4 * (size_t)NE;     // u32 [NE + 1]
  static constexpr size_t OFF_CELLS = OFF_START + 4 * (size_t)(NE + 1);  // u16 [NE] non-empty cells
  static constexpr size_t OFF_ORDER = OFF_CELLS + 2 * (size_t)NE;   // u16 [NE] cells, heaviest class first
  static constexpr size_t END = (OFF_ORDER + 2 * (size_t)NE + 15) / 16 * 16;
  // the keys and ids are dead once the cell lists are built, before the first
  // record is staged: the staging slots reuse their space when it is large enough
  // (61 KB instead of 75 KB for 8 x 8 x 4, leaving more of the SM's memory as L1)
  static constexpr bool STAGE_IN_KEYS = 8 * (size_t)MAXP >= STAGE_BYTES;
  static constexpr size_t OFF_STAGE = STAGE_IN_KEYS ? OFF_KEY : END;
  static constexpr size_t BYTES = STAGE_IN_KEYS ? END : END + STAGE_BYTES;
};

// Resident transfer CTAs per SM the register allocation is bounded for.
#ifndef TACCHI_XFER_MIN_BLOCKS
#define TACCHI_XFER_MIN_BLOCKS 2
#endif

// Block gblk's place: its particle range, instance and cell origin B0.
struct XBlock {
  uint32_t start, n;
  int ii, B0x, B0y, B0z;
};

template <int BX, int BY, int BZ>
__device__ __forceinline__ XBlock block_of(const Batch &b, long long gblk) {
  XBlock x;
  x.start = b.bstart[gblk];
  x.n = b.bstart[gblk + 1] - x.start;
  x.ii = (int)b.block_inst[gblk];
  const Instance &I = b.inst[x.ii];
  const long long lb = gblk - I.block_off;
  const int nb0 = I.nb[0], nb1 = I.nb[1];
  x.B0x = (int)(lb % nb0) * BX;
  x.B0y = (int)((lb / nb0) % nb1) * BY;
  x.B0z = (int)(lb / ((long long)nb0 * nb1)) * BZ;
  return x;
}

// The particle loop of a grouped block (steps 2-3 of the transfer): cells
// by thread, G2P against the V tile vt, F update, stress and P2G into the
// cell's register accumulators, flushed to the grid per cell.  All threads
// of the CTA call it after the grouping (s_list, s_start, s_order) is built;
// it ends with a barrier.
template <int BX, int BY, int BZ, int MODE>
__device__ __forceinline__ void transfer_cells(const Batch &b, float dt, const XBlock &xb, unsigned char *smem,
                                               const float4 *vt, bool grouped, uint32_t ncells, int *s_moved) {
  using P = XferPlan<BX, BY, BZ>;
  constexpr bool DO_G2P = (MODE & XFER_G2P) != 0;
  constexpr bool DO_P2G = (MODE & XFER_P2G) != 0;
  constexpr int VX = P::VX, VY = P::VY;
  const uint32_t *s_list = reinterpret_cast<const uint32_t *>(smem + P::OFF_LIST);
  const uint32_t *s_start = reinterpret_cast<const uint32_t *>(smem + P::OFF_START);
  const uint16_t *s_order = reinterpret_cast<const uint16_t *>(smem + P::OFF_ORDER);
  const uint32_t start = xb.start, n = xb.n;
  const Instance &I = b.inst[xb.ii];
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
  const int B0x = xb.B0x, B0y = xb.B0y, B0z = xb.B0z;
  const long long Ntot = b.Ntot;
  // the instance record is read once: stores to the particle arrays below
  // could otherwise alias it and force reloads inside the particle loop
  const float inv_dx = I.inv_dx, dx = I.dx, m = I.m, mu = I.mu, la = I.la;
  const bool fix_base = I.fix_base != 0;
  const long long node_off = I.node_off;
  const float c4 = 4.0f * dt * inv_dx;
  const float ks = 4.0f * dt * I.V0 * inv_dx;
  const int tid = threadIdx.x;
  float4 *__restrict__ gps = b.ps;
  const uint8_t *__restrict__ gfl = b.flags;

  // ---- one cell per thread (or, without grouping, one particle per thread)
  const uint32_t nwork = grouped ? ncells : n;
  // round r gives thread t the cell at position r * THREADS + t, mirrored on
  // odd rounds, so the warp that took the heaviest cells of one round takes
  // the lightest of the next
  auto work_of = [&](uint32_t r0) -> uint32_t {
    return r0 + (((r0 / P::THREADS) & 1u) ? (uint32_t)(P::THREADS - 1 - tid) : (uint32_t)tid);
  };
  // first particle of work item wk
  auto first_of = [&](uint32_t wk) -> uint32_t {
    return grouped ? s_list[s_start[s_order[wk]]] : b.idx[start + wk];
  };
  // The record of the next particle -- the next of the cell, or the first of
  // the thread's next cell -- is copied into this thread's other staging
  // slot while the current one computes.
  float4 *stage = reinterpret_cast<float4 *>(smem + P::OFF_STAGE) + tid;
  auto fetch = [&](uint32_t pp, int slot) {
    const float4 *src = gps + 3 * (long long)pp;
#pragma unroll
    for (int j = 0; j < 3; ++j) cp_async16(stage + (slot * 3 + j) * P::THREADS, src + j);
    cp_async_commit();
  };
  int slot = 0;
  uint32_t pn = 0, fln = 0;
  if (work_of(0) < nwork) {
    pn = first_of(work_of(0));
    fetch(pn, 0);
    if (DO_G2P) fln = gfl[pn];
  }
  for (uint32_t r0 = 0; r0 < nwork; r0 += P::THREADS) {
    const uint32_t wk = work_of(r0);
    if (wk >= nwork) continue;
    uint32_t q0, q1;
    int cx, cy, cz;
    if (grouped) {
      const uint32_t c = s_order[wk];
      q0 = s_start[c];
      q1 = s_start[c + 1];
      cx = (int)(c % P::EX);
      cy = (int)((c / P::EX) % P::EY);
      cz = (int)(c / (P::EX * P::EY));
    } else {
      q0 = wk;
      q1 = wk + 1;
      cx = cy = cz = 0;
    }
    // accumulators of the cell's 27 nodes: sum of w (mass / m) and of
    // w (m v + A (X_i - x)) per axis
    float2 acc01[27], acc2w[27];  // (MG x, MG y), (MG z, sum of w)
    if (DO_P2G && grouped) {
#pragma unroll
      for (int e = 0; e < 27; ++e) acc01[e] = acc2w[e] = make_float2(0.f, 0.f);
    }
    for (uint32_t q = q0; q < q1; ++q) {
      const uint32_t p = pn;
      const uint32_t fl = fln;
      const int cur = slot;
      bool ahead = false;
      if (q + 1 < q1) {
        pn = grouped ? s_list[q + 1] : b.idx[start + q + 1];
        ahead = true;
      } else {
        const uint32_t nk = work_of(r0 + P::THREADS);
        if (nk < nwork) {
          pn = first_of(nk);
          ahead = true;
        }
      }
      if (ahead) {
        slot ^= 1;
        fetch(pn, slot);
        if (DO_G2P) fln = gfl[pn];
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      float u[3], H[9];
      {
        const float4 a = stage[(cur * 3 + 0) * P::THREADS], bq = stage[(cur * 3 + 1) * P::THREADS],
                     cq = stage[(cur * 3 + 2) * P::THREADS];
        u[0] = a.x; u[1] = a.y; u[2] = a.z;
        H[0] = a.w; H[1] = bq.x; H[2] = bq.y; H[3] = bq.z; H[4] = bq.w;
        H[5] = cq.x; H[6] = cq.y; H[7] = cq.z; H[8] = cq.w;
      }
      int bs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) bs[a] = (int)floorf(u[a] - 0.5f);
      float v[3], Bm[9];  // Bm = sum_i w V (i - f)^T (cells); C = 4/dx Bm
      int err = 0;
      if (DO_G2P) {
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[a] = u[a] - (float)bs[a];
        float wx[3], wy[3], wz[3], dpx[3], dpy[3], dpz[3];
        bspline3(f[0], wx, dpx);
        bspline3(f[1], wy, dpy);
        bspline3(f[2], wz, dpz);
        // x and y velocity components in packed FP32 pairs (two lanes per
        // instruction), z in scalars
        float2 wxd[3], wdxd[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          wxd[i] = make_float2(wx[i], wx[i]);
          wdxd[i] = make_float2(wx[i] * dpx[i], wx[i] * dpx[i]);
        }
        const float2 z2 = make_float2(0.f, 0.f);
        float2 vxy = z2, b0xy = z2, b1xy = z2, b2xy = z2;  // v (Eq. 7), Bm columns (Eq. 8), rows x, y
        float2 vb0z = z2, b12z = z2;                        // row z: (v, Bm col 0), (Bm cols 1, 2)
        float2 wst[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) wst[i] = make_float2(wx[i], wdxd[i].x);
        // home cells lie inside the V tile; clamp only as a guard
        const int vx = clampi(bs[0] - (B0x - 1), 0, VX - 3), vy = clampi(bs[1] - (B0y - 1), 0, VY - 3),
                  vz0 = clampi(bs[2] - (B0z - 1), 0, P::VZ - 3);
        if (vx != bs[0] - (B0x - 1) || vy != bs[1] - (B0y - 1) || vz0 != bs[2] - (B0z - 1)) err |= ERRBIT_CFL;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float4 *row = vt + ((vz0 + k) * VY + (vy + j)) * VX + vx;
            const float4 V0 = row[0], V1 = row[1], V2 = row[2];
            // row sums over i: s = sum w_i V_i, t = sum w_i (i - f_x) V_i
            float2 sxy = __fmul2_rn(wxd[0], make_float2(V0.x, V0.y));
            float2 txy = __fmul2_rn(wdxd[0], make_float2(V0.x, V0.y));
            sxy = __ffma2_rn(wxd[1], make_float2(V1.x, V1.y), sxy);
            txy = __ffma2_rn(wdxd[1], make_float2(V1.x, V1.y), txy);
            sxy = __ffma2_rn(wxd[2], make_float2(V2.x, V2.y), sxy);
            txy = __ffma2_rn(wdxd[2], make_float2(V2.x, V2.y), txy);
            // z component: (sum w_i V_i.z, sum w_i (i - f_x) V_i.z) as one pair
            float2 st = __fmul2_rn(wst[0], make_float2(V0.z, V0.z));
            st = __ffma2_rn(wst[1], make_float2(V1.z, V1.z), st);
            st = __ffma2_rn(wst[2], make_float2(V2.z, V2.z), st);
            const float wjk = wy[j] * wz[k];
            const float wjy = wjk * dpy[j], wjz = wjk * dpz[k];
            vxy = __ffma2_rn(make_float2(wjk, wjk), sxy, vxy);      // Eq. 7
            b0xy = __ffma2_rn(make_float2(wjk, wjk), txy, b0xy);    // Eq. 8
            b1xy = __ffma2_rn(make_float2(wjy, wjy), sxy, b1xy);
            b2xy = __ffma2_rn(make_float2(wjz, wjz), sxy, b2xy);
            vb0z = __ffma2_rn(make_float2(wjk, wjk), st, vb0z);
            b12z = __ffma2_rn(make_float2(wjy, wjz), make_float2(st.x, st.x), b12z);
          }
        v[0] = vxy.x; v[1] = vxy.y; v[2] = vb0z.x;
        Bm[0] = b0xy.x; Bm[1] = b1xy.x; Bm[2] = b2xy.x;
        Bm[3] = b0xy.y; Bm[4] = b1xy.y; Bm[5] = b2xy.y;
        Bm[6] = vb0z.y; Bm[7] = b12z.x; Bm[8] = b12z.y;
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
      int nbs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) nbs[a] = (int)floorf(u[a] - 0.5f);
      if (nbs[0] < 2 || nbs[1] < 2 || nbs[2] < 2 || nbs[0] > G0 - 5 || nbs[1] > G1 - 5 || nbs[2] > G2 - 5)
        err |= ERRBIT_OUT_OF_GRID;
      const bool home = nbs[0] >= B0x - 1 && nbs[0] <= B0x + BX && nbs[1] >= B0y - 1 && nbs[1] <= B0y + BY &&
                        nbs[2] >= B0z - 1 && nbs[2] <= B0z + BZ;
      if (DO_G2P && !home) *s_moved = 1;  // left its home cells: re-sort after this transfer
      // the next transfer groups the block from these: slot q of the block's
      // idx range (its cell order now, when grouped) and the new home cell
      {
        const uint16_t hc = home ? (uint16_t)(((nbs[2] - (B0z - 1)) * P::EY + (nbs[1] - (B0y - 1))) * P::EX +
                                              (nbs[0] - (B0x - 1)))
                                 : kNotHome;
        if (grouped) b.idx[start + q] = p;
        b.hcell[start + q] = hc;
      }

      if (DO_P2G) {
        // Eqs. 2-5 with S_p = tau and the affine term of Eq. 4 carrying m_p:
        // MG_i += w (m v + A (X_i - x)),  A (X_i - x) = Abar (i - f),
        // Abar = dx (m C - dt V0 (4/dx^2) tau) = 4 m Bm - (4 dt V0 / dx) tau.
        float tau[9];
        const float Jm1 = kirchhoff_stress(H, mu, la, tau);
        if (!(1.0f + Jm1 > 0.f)) err |= ERRBIT_NUMERICAL;
        float A[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) A[e] = 4.0f * m * Bm[e] - ks * tau[e];
        const float mv[3] = {m * v[0], m * v[1], m * v[2]};
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[a] = u[a] - (float)nbs[a];
        const bool same_cell = grouped && nbs[0] - (B0x - 1) == cx && nbs[1] - (B0y - 1) == cy &&
                               nbs[2] - (B0z - 1) == cz;
        if (err & ERRBIT_NUMERICAL) {
          err |= ERRBIT_CFL;  // not scattered
        } else if (same_cell) {
          float wx[3], wy[3], wz[3], dpx[3], dpy[3], dpz[3];
          bspline3(f[0], wx, dpx);
          bspline3(f[1], wy, dpy);
          bspline3(f[2], wz, dpz);
          // packed pairs: (x, y) momentum components, and (z, mass weight)
          // with 1 in the second lane, so one FFMA2 adds w to the mass sum
          const float2 Axy0 = make_float2(A[0], A[3]), Axy1 = make_float2(A[1], A[4]),
                       Axy2 = make_float2(A[2], A[5]);
          float2 axy[3], ayxy[3], azxy[3];
          float axz[3], ayz[3], azz[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            axy[i] = __fmul2_rn(Axy0, make_float2(dpx[i], dpx[i]));
            ayxy[i] = __fmul2_rn(Axy1, make_float2(dpy[i], dpy[i]));
            azxy[i] = __fmul2_rn(Axy2, make_float2(dpz[i], dpz[i]));
            axz[i] = A[6] * dpx[i];
            ayz[i] = A[7] * dpy[i];
            azz[i] = A[8] * dpz[i];
          }
          const float2 mvxy = make_float2(mv[0], mv[1]);
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const float wjk = wy[j] * wz[k];
              const float2 wjk2 = make_float2(wjk, wjk);
              const float2 rxy = __fadd2_rn(__fadd2_rn(mvxy, ayxy[j]), azxy[k]);
              const float rz = mv[2] + ayz[j] + azz[k];
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                const int e = (k * 3 + j) * 3 + i;
                const float2 w2 = __fmul2_rn(make_float2(wx[i], wx[i]), wjk2);
                acc01[e] = __ffma2_rn(w2, __fadd2_rn(rxy, axy[i]), acc01[e]);          // Eqs. 3-5
                acc2w[e] = __ffma2_rn(w2, make_float2(rz + axz[i], 1.0f), acc2w[e]);  // and Eq. 2 (/ m)
              }
            }
        } else {
          // changed cell during the substep (or no grouping): scatters on its own
          const float wm[3] = {mv[0], mv[1], mv[2]};
          if (!scatter_particle_global(b.gmm + node_off, G0, G1, G2, nbs[0], nbs[1], nbs[2], m, f, wm, A))
            err |= ERRBIT_OUT_OF_GRID;  // stencil outside the grid: not scattered
        }
      }
      if (err) atomicOr(b.err, err);
    }
    if (DO_P2G && grouped && q1 > q0) {
      // the cell's 27 node sums go straight to the grid, one vector reduction
      // per node (red.global.add.v4.f32: no return value, so nothing waits on
      // it); the cell's base node is B0 - 1 + c
      const int bx = B0x - 1 + cx, by = B0y - 1 + cy, bz = B0z - 1 + cz;
      float4 *g0 = b.gmm + node_off;
      const bool inside = bx >= 0 && by >= 0 && bz >= 0 && bx + 2 < G0 && by + 2 < G1 && bz + 2 < G2;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const int e = (k * 3 + j) * 3 + i;
            if (inside || (bx + i >= 0 && by + j >= 0 && bz + k >= 0 && bx + i < G0 && by + j < G1 && bz + k < G2))
              atomicAdd(g0 + ((long long)(bz + k) * G1 + (by + j)) * G0 + (bx + i),
                        make_float4(m * acc2w[e].y, acc01[e].x, acc01[e].y, acc2w[e].x));
          }
    }
  }
  __syncthreads();
  if (DO_G2P && tid == 0 && *s_moved) *b.movers = 1;
}

// The transfer of sort block gblk by the calling CTA (all its threads), in
// dynamic shared memory smem of XferPlan::BYTES; the kernel below runs one
// block per CTA, the persistent step one block after another.
template <int BX, int BY, int BZ, int MODE>
__device__ __forceinline__ void transfer_block(const Batch &b, float dt, long long gblk, unsigned char *smem) {
  using P = XferPlan<BX, BY, BZ>;
  constexpr bool DO_G2P = (MODE & XFER_G2P) != 0;
  constexpr int VX = P::VX, VY = P::VY;
  uint32_t *s_key = reinterpret_cast<uint32_t *>(smem + P::OFF_KEY);
  float4 *vt = reinterpret_cast<float4 *>(smem + P::OFF_V);
  uint32_t *s_list = reinterpret_cast<uint32_t *>(smem + P::OFF_LIST);
  uint32_t *s_pid = reinterpret_cast<uint32_t *>(smem + P::OFF_PID);
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + P::OFF_CNT);
  uint32_t *s_start = reinterpret_cast<uint32_t *>(smem + P::OFF_START);
  uint16_t *s_cells = reinterpret_cast<uint16_t *>(smem + P::OFF_CELLS);
  uint16_t *s_order = reinterpret_cast<uint16_t *>(smem + P::OFF_ORDER);
  __shared__ uint32_t s_warp[P::THREADS / 32];
  __shared__ unsigned long long s_warp64[P::THREADS / 32];
  __shared__ int s_moved, s_overflow;

  const XBlock xb = block_of<BX, BY, BZ>(b, gblk);
  if (xb.n == 0) return;
  const uint32_t start = xb.start, n = xb.n;
  const Instance &I = b.inst[xb.ii];
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
  const int B0x = xb.B0x, B0y = xb.B0y, B0z = xb.B0z;
  const long long node_off = I.node_off;
  const int tid = threadIdx.x;

  // ---- grid velocities of nodes [B0-1, B0+B+3) into the V tile, copied
  // asynchronously while the particles are grouped (zeros outside the grid)
  if (DO_G2P) {
    const float4 *gv = b.gv + node_off;
    for (int t = tid; t < P::VN; t += P::THREADS) {
      const int x = B0x - 1 + t % VX, y = B0y - 1 + (t / VX) % VY, z = B0z - 1 + t / (VX * VY);
      const bool in = x >= 0 && y >= 0 && z >= 0 && x < G0 && y < G1 && z < G2;
      cp_async16_zfill(vt + t, in ? gv + ((long long)z * G1 + y) * G0 + x : gv, in);
    }
  }
  cp_async_commit();

  // ---- group the block's particles by home cell
  for (int c = tid; c < P::NE; c += P::THREADS) s_cnt[c] = 0;
  if (tid == 0) {
    s_moved = 0;
    s_overflow = n > (uint32_t)P::MAXP;
  }
  __syncthreads();
  if (n <= (uint32_t)P::MAXP) {
    // GB slots per thread per round, so that their id and home-cell loads are
    // all in flight together (two contiguous reads, no gather of positions)
    constexpr int GB = 16;
    static_assert(P::NE < kNotHome, "home cells must fit below the not-home mark");
    const uint16_t *__restrict__ ghc = b.hcell + start;
    for (uint32_t l0 = 0; l0 < n; l0 += GB * P::THREADS) {
      uint32_t pp[GB], hc[GB];
#pragma unroll
      for (int g = 0; g < GB; ++g) {
        const uint32_t l = l0 + g * P::THREADS + tid;
        pp[g] = l < n ? b.idx[start + l] : 0u;
        hc[g] = l < n ? (uint32_t)ghc[l] : (uint32_t)kNotHome;
      }
#pragma unroll
      for (int g = 0; g < GB; ++g) {
        const uint32_t l = l0 + g * P::THREADS + tid;
        if (l >= n) continue;
        s_pid[l] = pp[g];
        uint32_t key = 0xFFFFFFFFu;
        if (hc[g] < (uint32_t)P::NE) {
          key = (atomicAdd(s_cnt + hc[g], 1u) << 12) | hc[g];  // rank, cell (< 4096)
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
    ncells = block_scan_compact<P::THREADS, P::PER>(s_cnt, s_start, s_cells, P::NE, s_warp);
    for (uint32_t l = tid; l < n; l += P::THREADS) {
      const uint32_t key = s_key[l];
      s_list[s_start[key & 0xFFFu] + (key >> 12)] = s_pid[l];
    }
    order_cells_by_load<P::THREADS, P::PER>(s_cells, s_start, (int)ncells, s_order, s_warp64);
  }
  __syncthreads();
  cp_async_wait<0>();  // this thread's part of the V tile
  __syncthreads();
  transfer_cells<BX, BY, BZ, MODE>(b, dt, xb, smem, vt, grouped, ncells, &s_moved);
}

template <int BX, int BY, int BZ, int MODE>
__global__ void __launch_bounds__(128, TACCHI_XFER_MIN_BLOCKS) k_transfer(Batch b, float dt) {
  extern __shared__ __align__(16) unsigned char smem[];
  transfer_block<BX, BY, BZ, MODE>(b, dt, blockIdx.x, smem);
}

// ---------------------------------------------------------------------------
// Pipelined fused transfer.  A persistent grid (the transfer's resident CTAs,
// two per SM) takes the sort's non-empty block records one after another.
// While a CTA runs the particle loop of one block, the copy engine brings the
// next block's idx slots, home cells and V tile into the other set of buffers
// (bulk copies counted in bytes on one mbarrier), so that between two blocks
// only the shared-memory grouping is left of the per-block prologue.  Records
// are handed out by an atomic counter (brec order is block order, so CTAs
// running at the same time work on neighbouring blocks); the last CTA to
// finish resets the counters for the next launch.
template <int BX, int BY, int BZ>
struct PipePlan {
  using X = XferPlan<BX, BY, BZ>;
  // the XferPlan layout (its PID region holds the copied idx slots) plus a
  // second V tile and the copied home cells
  static constexpr size_t OFF_V2 = (X::BYTES + 15) / 16 * 16;                 // float4 [VN]
  static constexpr size_t OFF_HC = OFF_V2 + 16 * (size_t)X::VN;              // u16 [MAXP + 16]
  static constexpr size_t BYTES = (OFF_HC + 2 * (size_t)(X::MAXP + 16) + 15) / 16 * 16;
};

// Issue the copies of block r into V tile vb and the id / home-cell buffers
// pid and hc (all threads; each arrives once on bar with the bytes of its own
// copies).  The idx and home-cell copies start at the 16-byte boundary at or
// below r.start: slot l of the block is then pid[(r.start & 3) + l] and
// hc[(r.start & 7) + l].  They are skipped for a block too large to group.
template <int BX, int BY, int BZ>
__device__ __forceinline__ void pipe_prefetch(const Batch &b, const BlockRec &r, float4 *vb, uint32_t *pid,
                                              uint16_t *hc, uint64_t *bar) {
  using X = XferPlan<BX, BY, BZ>;
  constexpr int VX = X::VX, VY = X::VY, VZ = X::VZ, T = X::THREADS;
  const int tid = threadIdx.x;
  // earlier generic accesses of these buffers (the last block's grouping and
  // particle loop, behind a barrier) come before the copy engine's writes
  fence_proxy_async_smem();
  const bool groupable = r.n <= (uint32_t)X::MAXP;
  const uint32_t a0 = r.start & ~3u, a1 = (r.start + r.n + 3u) & ~3u;  // idx, u32
  const uint32_t h0 = r.start & ~7u, h1 = (r.start + r.n + 7u) & ~7u;  // hcell, u16
  const float4 *gv = b.gv + r.node_off;
  const int x0 = max(r.B0x - 1, 0), x1 = min(r.B0x - 1 + VX, r.G0);
  uint32_t bytes = 0;
  if (tid == 0 && groupable) bytes += 4u * (a1 - a0);
  if (tid == 1 && groupable) bytes += 2u * (h1 - h0);
  for (int rr = tid; rr < VY * VZ; rr += T) {
    const int y = r.B0y - 1 + rr % VY, z = r.B0z - 1 + rr / VY;
    if (y >= 0 && z >= 0 && y < r.G1 && z < r.G2 && x1 > x0) bytes += 16u * (uint32_t)(x1 - x0);
  }
  mbar_arrive_tx(bar, bytes);
  if (tid == 0 && groupable) bulk_g2s(pid, b.idx + a0, 4u * (a1 - a0), bar);
  if (tid == 1 && groupable) bulk_g2s(hc, b.hcell + h0, 2u * (h1 - h0), bar);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int rr = tid; rr < VY * VZ; rr += T) {
    const int y = r.B0y - 1 + rr % VY, z = r.B0z - 1 + rr / VY;
    float4 *row = vb + rr * VX;
    if (y >= 0 && z >= 0 && y < r.G1 && z < r.G2 && x1 > x0) {
      bulk_g2s(row + (x0 - (r.B0x - 1)), gv + ((long long)z * r.G1 + y) * r.G0 + x0, 16u * (uint32_t)(x1 - x0), bar);
      for (int t = 0; t < x0 - (r.B0x - 1); ++t) row[t] = zero;     // nodes left of the grid
      for (int t = x1 - (r.B0x - 1); t < VX; ++t) row[t] = zero;    // right of it
    } else {
      for (int t = 0; t < VX; ++t) row[t] = zero;                    // row outside the grid
    }
  }
}

template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(128, TACCHI_XFER_MIN_BLOCKS) k_transfer_pipe(Batch b, float dt, long long max_polls,
                                                                               int extra) {
  using X = XferPlan<BX, BY, BZ>;
  using Q = PipePlan<BX, BY, BZ>;
  constexpr int T = X::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_key = reinterpret_cast<uint32_t *>(smem + X::OFF_KEY);
  uint32_t *s_pidbuf = reinterpret_cast<uint32_t *>(smem + X::OFF_PID);
  uint16_t *s_hcbuf = reinterpret_cast<uint16_t *>(smem + Q::OFF_HC);
  uint32_t *s_list = reinterpret_cast<uint32_t *>(smem + X::OFF_LIST);
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + X::OFF_CNT);
  uint32_t *s_start = reinterpret_cast<uint32_t *>(smem + X::OFF_START);
  uint16_t *s_cells = reinterpret_cast<uint16_t *>(smem + X::OFF_CELLS);
  uint16_t *s_order = reinterpret_cast<uint16_t *>(smem + X::OFF_ORDER);
  float4 *vcur = reinterpret_cast<float4 *>(smem + X::OFF_V);
  float4 *vnext = reinterpret_cast<float4 *>(smem + Q::OFF_V2);
  __shared__ __align__(8) uint64_t bar;
  // ring of block records: the current block, the next (its copies in
  // flight) and the one after (its record in flight)
  __shared__ __align__(16) BlockRec s_rec[3];
  __shared__ uint32_t s_warp[T / 32];
  __shared__ unsigned long long s_warp64[T / 32];
  __shared__ int s_moved, s_overflow, s_abort;
  const int tid = threadIdx.x;
  const uint32_t nrec = b.blkq[0];

  if (tid == 0) {
    mbar_init(&bar, T + extra);  // extra > 0: arrivals that never come (tests the bounded wait)
    mbar_init_fence();
    const uint32_t k0 = atomicAdd(b.blkq + 1, 1u), k1 = atomicAdd(b.blkq + 1, 1u);
    BlockRec none{};
    s_rec[0] = k0 < nrec ? b.brec[k0] : none;
    s_rec[1] = k1 < nrec ? b.brec[k1] : none;
    s_abort = 0;
  }
  __syncthreads();
  uint32_t parity = 0;
  if (s_rec[0].n > 0) pipe_prefetch<BX, BY, BZ>(b, s_rec[0], vcur, s_pidbuf, s_hcbuf, &bar);
  for (int cur = 0;; cur = cur == 2 ? 0 : cur + 1) {
    const int nxt = cur == 2 ? 0 : cur + 1, aft = nxt == 2 ? 0 : nxt + 1;
    const BlockRec rc = s_rec[cur];
    if (rc.n == 0) break;  // the records are used up (uniform: read from shared memory)
    // the record after next: its index now, its copy once the grouping is done
    uint32_t kk = 0;
    if (tid == 0) kk = atomicAdd(b.blkq + 1, 1u);
    // this block's copies
    if (!mbar_wait_bounded(&bar, parity, max_polls)) s_abort = 1;
    for (int c = tid; c < X::NE; c += T) s_cnt[c] = 0;
    if (tid == 0) {
      s_moved = 0;
      s_overflow = rc.n > (uint32_t)X::MAXP;
    }
    __syncthreads();
    if (s_abort) break;
    parity ^= 1u;
    // ---- grouping from the copied slots and home cells
    const uint32_t n = rc.n;
    const uint32_t *s_pid = s_pidbuf + (rc.start & 3u);
    const uint16_t *s_hc = s_hcbuf + (rc.start & 7u);
    if (n <= (uint32_t)X::MAXP) {
      for (uint32_t l = tid; l < n; l += T) {
        const uint32_t h = s_hc[l];
        uint32_t key = 0xFFFFFFFFu;
        if (h < (uint32_t)X::NE) {
          key = (atomicAdd(s_cnt + h, 1u) << 12) | h;  // rank, cell (< 4096)
        } else {
          s_overflow = 1;  // not at home: the sort invariant is broken
        }
        s_key[l] = key;
      }
    }
    __syncthreads();
    const bool grouped = !s_overflow;
    uint32_t ncells = 0;
    if (grouped) {
      ncells = block_scan_compact<T, X::PER>(s_cnt, s_start, s_cells, X::NE, s_warp);
      for (uint32_t l = tid; l < n; l += T) {
        const uint32_t key = s_key[l];
        s_list[s_start[key & 0xFFFu] + (key >> 12)] = s_pid[l];
      }
      order_cells_by_load<T, X::PER>(s_cells, s_start, (int)ncells, s_order, s_warp64);
    }
    __syncthreads();
    // ---- the next block's copies, into the buffers this one no longer needs,
    // and the record after it
    const BlockRec rn = s_rec[nxt];
    if (rn.n > 0) pipe_prefetch<BX, BY, BZ>(b, rn, vnext, s_pidbuf, s_hcbuf, &bar);
    if (tid == 0) {
      if (kk < nrec) {
        const float4 *src = reinterpret_cast<const float4 *>(b.brec + kk);
        float4 *dst = reinterpret_cast<float4 *>(&s_rec[aft]);
#pragma unroll
        for (int j = 0; j < 3; ++j) cp_async16(dst + j, src + j);
      } else {
        s_rec[aft].n = 0;
      }
      cp_async_commit();
    }
    // ---- the particle loop (ends with a barrier)
    const XBlock xb{rc.start, rc.n, rc.ii, rc.B0x, rc.B0y, rc.B0z};
    transfer_cells<BX, BY, BZ, XFER_FUSED>(b, dt, xb, smem, vcur, grouped, ncells, &s_moved);
    cp_async_wait<0>();  // the record copy, where thread 0 had no particle to wait on
    __syncthreads();
    float4 *t = vcur;
    vcur = vnext;
    vnext = t;
  }
  // a wait that gave up: before the CTA leaves, give the phase its missing
  // arrivals and wait again for the copies still in flight, with a bound of
  // its own (2^26 polls) rather than the caller's, so that no copy lands in
  // the shared memory of a finished CTA
  if (s_abort) {
    if (tid == 0)
      for (int e = 0; e < extra; ++e) mbar_arrive(&bar);
    mbar_wait_bounded(&bar, parity, 1ll << 26);
  }
  __syncthreads();
  if (tid == 0) {
    if (s_abort) atomicOr(b.err, ERRBIT_TIMEOUT);
    __threadfence();
    if (atomicAdd(b.blkq + 2, 1u) == gridDim.x - 1) {  // last CTA: reset the hand-out
      b.blkq[1] = 0u;
      b.blkq[2] = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// Block of a particle: its stencil base cell floor(u - 1/2), divided by the
// block size, clamped into the instance's block grid.
__device__ __forceinline__ uint32_t particle_block(const Batch &b, const Instance &I, SortBlock blk,
                                                   long long p) {
  const float4 u = load_position(b.ps, p);
  const int bx = clampi((int)floorf(u.x - 0.5f), 0, I.G[0] - 1) / blk.x;
  const int by = clampi((int)floorf(u.y - 0.5f), 0, I.G[1] - 1) / blk.y;
  const int bz = clampi((int)floorf(u.z - 0.5f), 0, I.G[2] - 1) / blk.z;
  const int cx = clampi(bx, 0, I.nb[0] - 1), cy = clampi(by, 0, I.nb[1] - 1), cz = clampi(bz, 0, I.nb[2] - 1);
  return (uint32_t)(I.block_off + ((long long)cz * I.nb[1] + cy) * I.nb[0] + cx);
}

// The sort kernels run on a small grid-stride grid: most substeps no particle
// has left its block and they only read the flag and return, which must cost
// a few microseconds, not a launch of one CTA per 256 particles.
// The three sort passes, each run by CTAs cta, cta + ncta, ... of blockDim.x
// threads (grid-stride over the particles; base is warp-uniform).
__device__ __forceinline__ void sort_keys_pass(const Batch &b, SortBlock blk, long long cta, long long ncta) {
  const long long stride = ncta * blockDim.x;
  for (long long base = cta * blockDim.x; base < b.Ntot; base += stride) {
    const long long p = base + threadIdx.x;  // base is warp-uniform
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
}

__global__ void __launch_bounds__(256) k_sort_keys(Batch b, SortBlock blk, int force) {
  if (!force && *(volatile int *)b.movers == 0) return;
  sort_keys_pass(b, blk, blockIdx.x, gridDim.x);
}

// Exclusive scan of the block counts by one CTA (any size up to 1024
// threads); also sets the scatter cursors and clears the counts for the next
// sort.
__device__ __forceinline__ void sort_scan_cta(const Batch &b, SortBlock blk) {
  __shared__ unsigned long long warp_tot[32];
  const long long n = b.Nblk;
  const int T = blockDim.x;
  const long long per = (n + T - 1) / T;
  const long long lo = threadIdx.x * per;
  const long long hi = lo + per < n ? lo + per : n;
  // particles (low word) and non-empty blocks (high word) of this thread's
  // range, scanned together
  uint32_t local = 0, nz = 0;
  for (long long i = lo; i < hi; ++i) {
    const uint32_t c = b.bcount[i];
    local += c;
    nz += c > 0u;
  }
  const unsigned long long mine = (unsigned long long)local | ((unsigned long long)nz << 32);
  // inclusive scan of the per-thread totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned long long t = lane < (T >> 5) ? warp_tot[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  const unsigned long long pre = x - mine + (wid > 0 ? warp_tot[wid - 1] : 0ull);
  uint32_t run = (uint32_t)pre, arun = (uint32_t)(pre >> 32);
  for (long long i = lo; i < hi; ++i) {
    const uint32_t c = b.bcount[i];
    b.bstart[i] = run;
    b.cursor[i] = run;
    b.bcount[i] = 0u;
    if (c > 0u) {
      BlockRec r;
      r.start = run;
      r.n = c;
      r.ii = (int)b.block_inst[i];
      const Instance &I = b.inst[r.ii];
      const long long lb = i - I.block_off;
      const int nb0 = I.nb[0], nb1 = I.nb[1];
      r.B0x = (int)(lb % nb0) * blk.x;
      r.B0y = (int)((lb / nb0) % nb1) * blk.y;
      r.B0z = (int)(lb / ((long long)nb0 * nb1)) * blk.z;
      r.G0 = I.G[0];
      r.G1 = I.G[1];
      r.G2 = I.G[2];
      r.pad = 0;
      r.node_off = I.node_off;
      b.brec[arun++] = r;
    }
    run += c;
  }
  if (threadIdx.x == T - 1) {
    b.bstart[n] = run;
    b.blkq[0] = arun;
    b.movers[1] += 1;  // sorts that did work, read by the profile
  }
}

__global__ void __launch_bounds__(1024) k_sort_scan(Batch b, SortBlock blk, int force) {
  if (!force && *(volatile int *)b.movers == 0) return;
  sort_scan_cta(b, blk);
}

// Home cell of particle p in sort block key (see Batch::hcell), decided in
// floats so that a position far outside the grid cannot overflow an integer.
__device__ __forceinline__ uint16_t sort_home_cell(const Batch &b, SortBlock blk, uint32_t key, long long p) {
  const Instance &I = b.inst[b.block_inst[key]];
  const long long lb = (long long)key - I.block_off;
  const int nb0 = I.nb[0], nb1 = I.nb[1];
  const float o0 = (float)((int)(lb % nb0) * blk.x - 1), o1 = (float)((int)((lb / nb0) % nb1) * blk.y - 1),
              o2 = (float)((int)(lb / ((long long)nb0 * nb1)) * blk.z - 1);
  const float4 u = load_position(b.ps, p);
  const float ex = floorf(u.x - 0.5f) - o0, ey = floorf(u.y - 0.5f) - o1, ez = floorf(u.z - 0.5f) - o2;
  const int EX = blk.x + 2, EY = blk.y + 2, EZ = blk.z + 2;
  if (!(ex >= 0.f && ey >= 0.f && ez >= 0.f && ex < (float)EX && ey < (float)EY && ez < (float)EZ)) return kNotHome;
  return (uint16_t)(((int)ez * EY + (int)ey) * EX + (int)ex);
}

__device__ __forceinline__ void sort_scatter_pass(const Batch &b, SortBlock blk, long long cta, long long ncta) {
  const long long stride = ncta * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long base = cta * blockDim.x; base < b.Ntot; base += stride) {
    const long long p = base + threadIdx.x;
    const bool valid = p < b.Ntot;
    const uint32_t key = valid ? b.key[p] : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base_slot = 0;
    if (valid && lane == leader) base_slot = atomicAdd(b.cursor + key, (uint32_t)__popc(peers));
    base_slot = __shfl_sync(0xFFFFFFFFu, base_slot, leader);
    if (valid) {
      const uint32_t slot = base_slot + __popc(peers & ((1u << lane) - 1u));
      b.idx[slot] = (uint32_t)p;
      b.hcell[slot] = sort_home_cell(b, blk, key, p);
    }
  }
}

__global__ void __launch_bounds__(256) k_sort_scatter(Batch b, SortBlock blk, int force) {
  if (!force && *(volatile int *)b.movers == 0) return;
  sort_scatter_pass(b, blk, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Indenter represented by particles (Eq. 10, p in I; Sec. III-C: initialised
// from a point cloud of the object): each particle sits at x = c + R l on
// the rigid indenter and moves with it, v = v_c + w x (x - c), so its affine
// velocity (Eq. 4) is C = skew(w); a rigid particle carries no elastic
// stress (Eq. 5 adds nothing).  It adds its mass and momentum to the grid
// nodes of its stencil inside the grid (Eqs. 2-4) with vector reductions.
__device__ __forceinline__ void indenter_p2g_one(const Batch &b, long long q, int substep) {
  if (q >= b.Np) return;
  const Instance &I = b.inst[b.ind_inst[q]];
  const IndenterFrame f = I.frames[substep];
  const float l0 = b.ind_pts[3 * q], l1 = b.ind_pts[3 * q + 1], l2 = b.ind_pts[3 * q + 2];
  float r[3], x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = f.r[a * 3 + 0] * l0 + f.r[a * 3 + 1] * l1 + f.r[a * 3 + 2] * l2;  // cells
    x[a] = f.c[a] + r[a];
  }
  const float dx = I.dx, m = I.ind_m;
  const float v0 = f.vlin[0] + (f.w[1] * r[2] - f.w[2] * r[1]) * dx;
  const float v1 = f.vlin[1] + (f.w[2] * r[0] - f.w[0] * r[2]) * dx;
  const float v2 = f.vlin[2] + (f.w[0] * r[1] - f.w[1] * r[0]) * dx;
  int bs[3];
  float wt[3][3], dp[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bs[a] = (int)floorf(x[a] - 0.5f);
    bspline3(x[a] - (float)bs[a], wt[a], dp[a]);
  }
  float4 *gmm = b.gmm + I.node_off;
  const int G0 = I.G[0], G1 = I.G[1], G2 = I.G[2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int X = bs[0] + i, Y = bs[1] + j, Z = bs[2] + k;
        if (X < 0 || Y < 0 || Z < 0 || X >= G0 || Y >= G1 || Z >= G2) continue;
        const float w = wt[0][i] * wt[1][j] * wt[2][k];
        // node offset from the particle (m) and its rigid velocity w x d
        const float d0 = dp[0][i] * dx, d1 = dp[1][j] * dx, d2 = dp[2][k] * dx;
        const float mw = m * w;
        atomicAdd(gmm + ((long long)Z * G1 + Y) * G0 + X,
                  make_float4(mw, mw * (v0 + (f.w[1] * d2 - f.w[2] * d1)), mw * (v1 + (f.w[2] * d0 - f.w[0] * d2)),
                              mw * (v2 + (f.w[0] * d1 - f.w[1] * d0))));
      }
}

__global__ void __launch_bounds__(256) k_indenter_p2g(Batch b, int substep) {
  indenter_p2g_one(b, (long long)blockIdx.x * blockDim.x + threadIdx.x, substep);
}

cudaError_t launch_indenter_p2g(const Batch &b, int substep, cudaStream_t st) {
  if (b.Np <= 0) return cudaSuccess;
  k_indenter_p2g<<<(unsigned)((b.Np + 255) / 256), 256, 0, st>>>(b, substep);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conversion between the particle records and the structure-of-arrays layout
// of the C ABI.
__global__ void __launch_bounds__(256) k_pack_state(float4 *ps, long long o, long long n, const float *u,
                                                   const float *Fm) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float x[3], H[9];
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = u[a * n + q];
#pragma unroll
  for (int e = 0; e < 9; ++e) H[e] = Fm ? Fm[e * n + q] : 0.f;
  store_particle(ps, o + q, x, H);
}

__global__ void __launch_bounds__(256) k_unpack_state(const float4 *ps, long long o, long long n, float *u,
                                                     float *Fm) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float x[3], H[9];
  load_particle(ps, o + q, x, H);
  if (u)
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a * n + q] = x[a];
  if (Fm)
#pragma unroll
    for (int e = 0; e < 9; ++e) Fm[e * n + q] = H[e];
}

cudaError_t launch_pack_state(float4 *ps, long long o, long long n, const float *u, const float *Fm,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_pack_state<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ps, o, n, u, Fm);
  return cudaGetLastError();
}

cudaError_t launch_unpack_state(const float4 *ps, long long o, long long n, float *u, float *Fm,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_unpack_state<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ps, o, n, u, Fm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
cudaError_t launch_grid_update(const Batch &b, int substep, float dt, int clear, cudaStream_t st) {
  const long long nb = (b.Nnodes + 255) / 256;
  k_grid_update<<<(unsigned)nb, 256, 0, st>>>(b, substep, dt, clear);
  return cudaGetLastError();
}

template <int BX, int BY, int BZ>
static cudaError_t launch_transfer_t(const Batch &b, int mode, float dt, cudaStream_t st) {
  const size_t smem = XferPlan<BX, BY, BZ>::BYTES;
  const unsigned grid = (unsigned)b.Nblk;
  switch (mode) {
    case XFER_P2G:
      k_transfer<BX, BY, BZ, XFER_P2G><<<grid, XferPlan<BX, BY, BZ>::THREADS, smem, st>>>(b, dt);
      break;
    case XFER_G2P:
      k_transfer<BX, BY, BZ, XFER_G2P><<<grid, XferPlan<BX, BY, BZ>::THREADS, smem, st>>>(b, dt);
      break;
    case XFER_FUSED:
      k_transfer<BX, BY, BZ, XFER_FUSED><<<grid, XferPlan<BX, BY, BZ>::THREADS, smem, st>>>(b, dt);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int BX, int BY, int BZ>
static cudaError_t prepare_t() {
  const int smem = (int)XferPlan<BX, BY, BZ>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_transfer<BX, BY, BZ, XFER_P2G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_transfer<BX, BY, BZ, XFER_G2P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_transfer<BX, BY, BZ, XFER_FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  return e;
}

// Opt the transfer kernels of a block shape into their shared-memory size;
// called once per context before any launch or capture.
cudaError_t prepare_transfer(SortBlock blk) {
  if (blk.t == 3) return prepare_transfer3(blk);
  if (blk.t != 1) return cudaErrorInvalidValue;
  if (blk.x == 8 && blk.y == 8 && blk.z == 4) return prepare_t<8, 8, 4>();
  if (blk.x == 4 && blk.y == 4 && blk.z == 4) return prepare_t<4, 4, 4>();
  if (blk.x == 8 && blk.y == 8 && blk.z == 8) return prepare_t<8, 8, 8>();
  if (blk.x == 16 && blk.y == 8 && blk.z == 4) return prepare_t<16, 8, 4>();
  return cudaErrorInvalidValue;
}

cudaError_t launch_transfer(const Batch &b, SortBlock blk, int mode, float dt, cudaStream_t st) {
  if (b.Nblk == 0) return cudaSuccess;
  if (blk.t == 3) return launch_transfer3(b, blk, mode, dt, st);
  if (blk.t != 1) return cudaErrorInvalidValue;
  if (blk.x == 8 && blk.y == 8 && blk.z == 4) return launch_transfer_t<8, 8, 4>(b, mode, dt, st);
  if (blk.x == 4 && blk.y == 4 && blk.z == 4) return launch_transfer_t<4, 4, 4>(b, mode, dt, st);
  if (blk.x == 8 && blk.y == 8 && blk.z == 8) return launch_transfer_t<8, 8, 8>(b, mode, dt, st);
  if (blk.x == 16 && blk.y == 8 && blk.z == 4) return launch_transfer_t<16, 8, 4>(b, mode, dt, st);
  return cudaErrorInvalidValue;
}

template <int BX, int BY, int BZ>
static cudaError_t prepare_pipe_t(int *grid) {
  const int smem = (int)PipePlan<BX, BY, BZ>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_transfer_pipe<BX, BY, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transfer_pipe<BX, BY, BZ>, XferPlan<BX, BY, BZ>::THREADS,
                                                    smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = per_sm * sms;
  return cudaSuccess;
}

bool pipe_supported(SortBlock blk) { return blk.t == 1 && blk.x == 8 && blk.y == 8 && blk.z == 4; }

cudaError_t prepare_pipe(SortBlock blk, int *grid) {
  if (!pipe_supported(blk)) return cudaErrorInvalidValue;
  return prepare_pipe_t<8, 8, 4>(grid);
}

cudaError_t launch_transfer_pipe(const Batch &b, SortBlock blk, float dt, int grid, long long max_polls, int extra,
                                 cudaStream_t st) {
  if (!pipe_supported(blk) || grid < 1) return cudaErrorInvalidValue;
  k_transfer_pipe<8, 8, 4><<<grid, XferPlan<8, 8, 4>::THREADS, PipePlan<8, 8, 4>::BYTES, st>>>(b, dt, max_polls, extra);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent step: one cooperative launch runs a whole chunk of substeps
// (grid clear, the opening P2G, then per substep the grid update, the fused
// transfer or the closing G2P, and the sort when a particle left its block),
// with a grid-wide barrier between phases instead of kernel boundaries.
// Every CTA is co-resident (cooperative launch), so a barrier only waits for
// CTAs that are running; each wait is still bounded: a CTA that polls
// max_polls times gives up, records ERRBIT_TIMEOUT and sets the abort word,
// and every CTA returns at its next barrier.  No asynchronous copy is in
// flight at a barrier (each block's transfer waits for its own copies).
__device__ __forceinline__ bool grid_barrier(const PersistCtl &c, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *gen = c.bar + 1;
    const unsigned g = *gen;
    __threadfence();  // this CTA's writes before its arrival
    if (atomicAdd(c.bar, 1u) == gridDim.x + c.extra - 1u) {
      atomicExch(c.bar, 0u);
      atomicExch(c.bar + 3, 0u);  // the next phase's blocks are taken from 0 again
      __threadfence();
      atomicAdd(c.bar + 1, 1u);  // release the others
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (*(volatile int *)c.abort) {
          ok = 0;
          break;
        }
        if (++polls > c.max_polls) {
          atomicOr(err, ERRBIT_TIMEOUT);
          atomicExch(c.abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Transfer of every sort block by the persistent grid: each CTA takes the
// next untaken block (an atomic counter, reset at every barrier), so that
// blocks of uneven cost spread like the hardware scheduler would spread CTAs
// (taking two at a time starves small grids of parallelism: measured slower).
template <int BX, int BY, int BZ, int MODE>
__device__ __forceinline__ void transfer_all(const Batch &b, float dt, const PersistCtl &c, unsigned char *smem) {
  __shared__ unsigned s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(c.bar + 3, 1u);
    __syncthreads();
    const long long g = s_next;
    __syncthreads();
    if (g >= b.Nblk) break;
    transfer_block<BX, BY, BZ, MODE>(b, dt, g, smem);
  }
}

template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(128, TACCHI_XFER_MIN_BLOCKS)
    k_persistent(Batch b, SortBlock blk, int n, float dt, PersistCtl c) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long q = gt; q < b.Nnodes; q += nth) b.gmm[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!grid_barrier(c, b.err)) return;
  transfer_all<BX, BY, BZ, XFER_P2G>(b, dt, c, smem);
  for (long long q = gt; q < b.Np; q += nth) indenter_p2g_one(b, q, 0);
  if (!grid_barrier(c, b.err)) return;
  for (int k = 0; k < n; ++k) {
    const bool last = k + 1 == n;
    grid_update_all(b, k, dt, last ? 0 : 1);
    if (!grid_barrier(c, b.err)) return;
    if (last) {
      transfer_all<BX, BY, BZ, XFER_G2P>(b, dt, c, smem);
    } else {
      transfer_all<BX, BY, BZ, XFER_FUSED>(b, dt, c, smem);
      for (long long q = gt; q < b.Np; q += nth) indenter_p2g_one(b, q, k + 1);
    }
    if (!grid_barrier(c, b.err)) return;
    // every CTA reads the flag after the barrier and before anyone clears it
    // (the next grid update, past the sort's barriers)
    if (*(volatile int *)b.movers) {
      sort_keys_pass(b, blk, blockIdx.x, gridDim.x);
      if (!grid_barrier(c, b.err)) return;
      if (blockIdx.x == 0) sort_scan_cta(b, SortBlock{BX, BY, BZ, 1});
      if (!grid_barrier(c, b.err)) return;
      sort_scatter_pass(b, SortBlock{BX, BY, BZ, 1}, blockIdx.x, gridDim.x);
      if (!grid_barrier(c, b.err)) return;
    }
  }
}

bool persistent_supported(SortBlock blk) { return blk.x == 8 && blk.y == 8 && blk.z == 4 && blk.t == 1; }

cudaError_t prepare_persistent(SortBlock blk, int *grid) {
  if (!persistent_supported(blk)) return cudaErrorInvalidValue;
  const int smem = (int)XferPlan<8, 8, 4>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_persistent<8, 8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int dev = 0, sms = 0, per = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<8, 8, 4>, 128, smem);
  if (e == cudaSuccess && (per < 1 || sms < 1)) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) *grid = per * sms;
  return e;
}

cudaError_t launch_persistent(const Batch &b, SortBlock blk, int n, float dt, const PersistCtl &ctl, int grid,
                              cudaStream_t st) {
  if (!persistent_supported(blk) || grid < 1 || n < 1) return cudaErrorInvalidValue;
  Batch bb = b;
  SortBlock sb = blk;
  int nn = n;
  float d = dt;
  PersistCtl c = ctl;
  void *args[] = {&bb, &sb, &nn, &d, &c};
  return cudaLaunchCooperativeKernel((const void *)k_persistent<8, 8, 4>, dim3(grid), dim3(128), args,
                                     XferPlan<8, 8, 4>::BYTES, st);
}

cudaError_t launch_sort(const Batch &b, SortBlock blk, int force, cudaStream_t st) {
  if (b.Ntot == 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0)
      sms = 152;
  }
  const long long full = (b.Ntot + 255) / 256;
  const unsigned gp = (unsigned)(full < 8LL * sms ? full : 8LL * sms);  // 8 CTAs of 256 fill an SM
  k_sort_keys<<<gp, 256, 0, st>>>(b, blk, force);
  k_sort_scan<<<1, 1024, 0, st>>>(b, blk, force);
  k_sort_scatter<<<gp, 256, 0, st>>>(b, blk, force);
  return cudaGetLastError();
}

}  // namespace tacchi
