// nn.cu -- the learned surrogate: a U-Net trained and run with hand-written
// BF16 tensor-core kernels (FP32 accumulation) on sm_103a.
//
// The paper has no surrogate; it is this library's addition: a network that
// maps the indenter's penetration map over the top face (and the depth) to
// the top-surface displacement field that the MPM would produce.
//
// Network (NHWC activations in BF16, parameters in FP32 with BF16 copies):
//   encoder levels l = 0..L-1: conv3x3+ReLU, conv3x3+ReLU, 2x2 average pool
//   (not after the last level); decoder levels l = L-2..0: nearest 2x
//   upsampling, concatenation [upsampled, skip], conv3x3+ReLU twice; head:
//   1x1 convolution to the output channels (FP32).  Loss: mean squared error.
//
// Kernels:
//   k_conv3x3_tc   implicit-GEMM 3x3 convolution on the 5th-generation tensor
//                  cores: rows = pixels, columns = output channels, K = 9 x
//                  C_in; TMA tile loads (the image border as zero fill) into
//                  a ring of 64-byte-swizzled stages, one producer thread and
//                  one tcgen05.mma issuer synchronised by full/empty
//                  mbarriers, the FP32 accumulator in tensor memory, and a
//                  bias+ReLU+BF16 epilogue from tcgen05.ld.  The data gradient
//                  runs the same kernel on the output gradient with the
//                  weights flipped and transposed.
//   k_conv3x3_wgrad_tc  weight gradient on the same tensor-core machinery:
//                  rows = (tap, C_in), columns = C_out, K = pixels, both
//                  operands MN-major from TMA boxes, split over pixel chunks
//                  whose partial sums meet in dW through float4 reductions.
//   elementwise kernels for pooling, upsampling, concatenation, the ReLU
//   mask fused with the bias gradients, the 1x1 head, the loss and Adam.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tacchi.h"

namespace {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): operands in shared memory described
// by matrix descriptors, the FP32 accumulator in tensor memory (TMEM).
//
// Shared-memory operand layout (K-major, no swizzle): the tile is a grid of
// "core matrices" of 8 rows x 16 bytes (8 BF16 along K), each stored as 128
// contiguous bytes (row r at +16 r).  With K_CH = BK / 8 core matrices per
// 8-row group along K, core matrix (row group g, K chunk j) sits at byte
// (g * K_CH + j) * 128: the descriptor's leading-dimension offset (between K
// neighbours) is 128 B and its stride-dimension offset (between 8-row groups)
// K_CH * 128 B.
namespace tc {

// K-major operand whose rows are 64 bytes (32 BF16 along K) with the 64-byte
// swizzle the TMA applies (16-byte chunk j of row r stored at chunk
// j ^ ((r >> 1) & 3)): 8-row groups 512 bytes apart (stride-dimension
// offset); the leading-dimension offset is unused while an MMA's K (32
// bytes) stays inside the 64-byte row.  A K step inside the row advances the
// start address; the tile must sit on a 512-byte boundary.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;               // leading-dimension offset (unused): 16 bytes
  d |= (uint64_t)(512 >> 4) << 32;      // stride-dimension offset: 512 bytes
  d |= (uint64_t)1 << 46;               // descriptor version; base offset 0
  d |= (uint64_t)4 << 61;               // 64-byte swizzle
  return d;
}

// 2D / 4D tiled TMA loads completing on an mbarrier (transaction bytes).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 and 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at
// bit 24.
template <int M, int N>
__device__ __forceinline__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count));
}
// Bounded wait for the phase with the given parity; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// D (TMEM) (+)= A (smem) * B (smem)^T, issued by one thread.
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued so far is done.
__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_addr(bar))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Y[m][co] = act(b[co] + sum_k A[m][k] Wk[co][k]) for one 3x3 'same'
// convolution as an implicit GEMM: row m = pixel (n, y, x), K = 9 taps x Cin,
// A[m][k] = X at pixel m shifted by tap(k) = 3 dy + dx in channel ci(k)
// (zero outside the image), k = tap * Cin + ci; Wk is K-major [Cout][9 Cin].
// One CTA computes 128 pixels x N output channels.  The 128 pixels are a box
// of wb x hb x nb (x, y, image) of the NHWC activation, so the A slice of a
// stage -- 32 channels of one tap -- is one 4D TMA load of that box shifted
// by (dx, dy), the image border coming back as the TMA's zero fill; the B
// slice (N x 32 of the weights) is one 2D TMA load.  Both land 64-byte
// swizzled in a ring of STAGES shared-memory stages:
//   thread 0 (producer) waits for a stage's "empty" mbarrier, arms its
//   "full" mbarrier with the bytes to expect and issues the two loads;
//   thread 32 (MMA issuer) waits for "full", issues the stage's two
//   128 x N x 16 tcgen05.mma into tensor memory and commits them to "empty".
// After the last stage the issuer commits to "done"; all four warps then read
// TMEM lane = pixel, add the bias, apply ReLU and store BF16.  Requires Cin %
// 32 == 0, Cout % N == 0.  A wait that gives up sets *err, abandons the tile
// and frees TMEM.
template <int N, int STAGES, int TCOLS>
__global__ void __launch_bounds__(128) k_conv3x3_tc(const __grid_constant__ CUtensorMap tmX,
                                                    const __grid_constant__ CUtensorMap tmW,
                                                    const float *__restrict__ bias, bf16 *__restrict__ Y, int nimg,
                                                    int H, int W, int Cin, int Cout, int relu, int *err) {
  constexpr int BM = 128, BK = 32;
  constexpr int A_BYTES = BM * BK * 2, B_BYTES = N * BK * 2, STAGE = A_BYTES + B_BYTES;
  static_assert(N % 16 == 0 && N >= 32 && N <= 256, "UMMA N for M = 128");
  static_assert(STAGE % 1024 == 0, "stages keep the 512-byte alignment of the swizzled tiles");
  static_assert(TCOLS >= N && (TCOLS & (TCOLS - 1)) == 0 && TCOLS <= 512, "tensor-memory allocation");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  // swizzled tiles need 512-byte alignment: round the dynamic base up
  unsigned char *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = nimg * H * W;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * N;
  const int nk = 9 * Cin / BK;
  // the tile's first pixel: a corner of the wb x hb x nb box
  const int bx0 = m0 % W, by0 = (m0 / W) % H, bn0 = m0 / (W * H);

  if (tid == 0) {
    for (int s2 = 0; s2 < STAGES; ++s2) {
      tc::mbar_init(&full[s2], 1);
      tc::mbar_init(&empty[s2], 1);
    }
    tc::mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (tid == 0) {  // producer
    for (int kk = 0; kk < nk && ok; ++kk) {
      const int buf = kk % STAGES;
      if (kk >= STAGES) ok = tc::mbar_wait(&empty[buf], (uint32_t)(kk / STAGES - 1) & 1u);
      if (!ok) break;
      const int k0 = kk * BK, tap = k0 / Cin, ci0 = k0 - tap * Cin;
      unsigned char *sa = smem + buf * STAGE;
      tc::mbar_expect_tx(&full[buf], (uint32_t)STAGE);
      tc::tma_load_4d(sa, &tmX, ci0, bx0 + tap % 3 - 1, by0 + tap / 3 - 1, bn0, &full[buf]);
      tc::tma_load_2d(sa + A_BYTES, &tmW, k0, n0, &full[buf]);
    }
  } else if (tid == 32) {  // MMA issuer
    constexpr uint32_t IDESC = tc::instr_desc<BM, N>();
    for (int kk = 0; kk < nk && ok; ++kk) {
      const int buf = kk % STAGES;
      ok = tc::mbar_wait(&full[buf], (uint32_t)(kk / STAGES) & 1u);
      if (!ok) break;
      tc::fence_after();
      const uint32_t a0 = smem_addr(smem + buf * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int ks = 0; ks < BK / 16; ++ks)  // K = 16 per MMA: 32 bytes along the 64-byte row
        tc::mma(tmem, tc::smem_desc_sw64(a0 + 32 * ks), tc::smem_desc_sw64(b0 + 32 * ks), IDESC,
                (kk > 0 || ks > 0) ? 1u : 0u);
      tc::commit(&empty[buf]);
    }
    if (ok) tc::commit(&done);
  }
  // everyone waits for the accumulator (bounded), then the epilogue
  if (ok) ok = tc::mbar_wait(&done, 0);
  const bool failed = __syncthreads_or(!ok);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    tc::fence_after();
    // warp w owns TMEM lanes 32 w .. 32 w + 31 = rows (pixels) of the tile
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
        uint32_t packed[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float x0 = v[2 * q] + (bias ? bias[n0 + c0 + 2 * q] : 0.f);
          float x1 = v[2 * q + 1] + (bias ? bias[n0 + c0 + 2 * q + 1] : 0.f);
          if (relu) {
            x0 = fmaxf(x0, 0.f);
            x1 = fmaxf(x1, 0.f);
          }
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
          packed[q] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(Y + (long long)row * Cout + n0 + c0);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// MN-major operand (rows = K, 64 bytes = 32 elements along M or N per row,
// 64-byte swizzled as the TMA writes it): a 64-byte column group of K_ROWS
// rows is one TMA box; column groups lie box_bytes apart (leading-dimension
// offset) and 8-row groups along K 512 bytes apart (stride-dimension offset).
__device__ __forceinline__ uint64_t smem_desc_sw64_mn(uint32_t addr, uint32_t box_bytes) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((box_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Weight gradient on the tensor cores: dW[k][co] += sum over pixels p of
// X(p shifted by tap(k))[ci(k)] * G[p][co], k = tap * Cin + ci.  A CTA owns
// 128 rows k (four 32-row groups, each one tap and 32 channels) x NC output
// channels and a chunk of pixels; per stage of 64 pixels (a box of whole
// image rows) the producer issues four 4D TMA loads of X (one per row group,
// shifted by its tap, zero outside the image) and NC / 32 2D loads of G,
// 64-byte swizzled; both operands are MN-major (K = pixels runs along the
// rows of the boxes).  The issuer runs four 128 x NC x 16 MMAs per stage
// into tensor memory; the epilogue adds the partial sums to dW with float4
// reductions (rows k >= 9 Cin, the padding of the last tile, are dropped).
template <int NC, int STAGES, int TCOLS>
__global__ void __launch_bounds__(128) k_conv3x3_wgrad_tc(const __grid_constant__ CUtensorMap tmX,
                                                          const __grid_constant__ CUtensorMap tmG,
                                                          float *__restrict__ dW, int P, int H, int W, int Cin,
                                                          int Cout, int chunk, int *err) {
  constexpr int BOX = 64 * 64;                   // 64 pixels x 64 bytes
  constexpr int A_BYTES = 4 * BOX, B_BYTES = (NC / 32) * BOX, STAGE = A_BYTES + B_BYTES;
  static_assert(NC % 32 == 0 && NC >= 32 && NC <= 256, "UMMA N for M = 128");
  static_assert(TCOLS >= NC && (TCOLS & (TCOLS - 1)) == 0, "tensor-memory allocation");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  unsigned char *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K9 = 9 * Cin;
  const int k_base = blockIdx.x * 128, n0 = blockIdx.y * NC;
  const int p_begin = blockIdx.z * chunk;
  const int nst = (min(P, p_begin + chunk) - p_begin + 63) / 64;

  if (tid == 0) {
    for (int s2 = 0; s2 < STAGES; ++s2) {
      tc::mbar_init(&full[s2], 1);
      tc::mbar_init(&empty[s2], 1);
    }
    tc::mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (tid == 0) {  // producer
    for (int st = 0; st < nst && ok; ++st) {
      const int buf = st % STAGES;
      if (st >= STAGES) ok = tc::mbar_wait(&empty[buf], (uint32_t)(st / STAGES - 1) & 1u);
      if (!ok) break;
      const int p0 = p_begin + 64 * st;
      const int px = p0 % W, py = (p0 / W) % H, pn = p0 / (W * H);
      unsigned char *sa = smem + buf * STAGE;
      tc::mbar_expect_tx(&full[buf], (uint32_t)STAGE);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kj = k_base + 32 * j;
        // rows past 9 Cin: a box entirely outside the image, i.e. zeros
        const int tap = kj < K9 ? kj / Cin : 0, ci0 = kj < K9 ? kj - tap * Cin : 0;
        const int xo = kj < K9 ? tap % 3 - 1 : 2 * W;
        tc::tma_load_4d(sa + j * BOX, &tmX, ci0, px + xo, py + tap / 3 - 1, pn, &full[buf]);
      }
#pragma unroll
      for (int j = 0; j < NC / 32; ++j) tc::tma_load_2d(sa + A_BYTES + j * BOX, &tmG, n0 + 32 * j, p0, &full[buf]);
    }
  } else if (tid == 32) {  // MMA issuer
    // instruction descriptor: FP32 D, BF16 A and B, both MN-major
    constexpr uint32_t IDESC = tc::instr_desc<128, NC>() | (1u << 15) | (1u << 16);
    for (int st = 0; st < nst && ok; ++st) {
      const int buf = st % STAGES;
      ok = tc::mbar_wait(&full[buf], (uint32_t)(st / STAGES) & 1u);
      if (!ok) break;
      tc::fence_after();
      const uint32_t a0 = smem_addr(smem + buf * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)  // K = 16 pixels per MMA: two 8-row groups (1024 bytes)
        tc::mma(tmem, smem_desc_sw64_mn(a0 + 1024 * ks, BOX), smem_desc_sw64_mn(b0 + 1024 * ks, BOX), IDESC,
                (st > 0 || ks > 0) ? 1u : 0u);
      tc::commit(&empty[buf]);
    }
    if (ok) tc::commit(&done);
  }
  if (ok) ok = tc::mbar_wait(&done, 0);
  const bool failed = __syncthreads_or(!ok);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else if (nst > 0) {
    tc::fence_after();
    const int k = k_base + warp * 32 + lane;  // TMEM lane = row k
#pragma unroll 1
    for (int c0 = 0; c0 < NC; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (k < K9) {
        float4 *dst = reinterpret_cast<float4 *>(dW + (long long)k * Cout + n0 + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// ---------------------------------------------------------------------------
// elementwise kernels (grid-stride)
#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
                               i += (long long)gridDim.x * blockDim.x)

// x fp32 [P][cin] -> bf16 [P][cpad] (zero padded channels)
// Eight BF16 channels (16 bytes) per thread in the kernels below; every
// channel count is a multiple of 32.
__device__ __forceinline__ void unpack8(const uint4 &u, float f[8]) {
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 t = __bfloat1622float2(h[k]);
    f[2 * k] = t.x;
    f[2 * k + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float f[8]) {
  uint4 u;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
  return u;
}
#define GRID_STRIDE_U(i, n) for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// x fp32 [P][cin] -> bf16 [P][cpad] (zero padded channels); chunks of 8
__global__ void k_pack_input(const float *x, bf16 *y, unsigned P, int cin, int cpad) {
  const unsigned cc = (unsigned)cpad / 8;
  GRID_STRIDE_U(e, P * cc) {
    const unsigned p = e / cc, c0 = (e % cc) * 8;
    float f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = (int)c0 + k < cin ? x[(long long)p * cin + c0 + k] : 0.f;
    reinterpret_cast<uint4 *>(y)[e] = pack8(f);
  }
}
// y[n][H/2][W/2][C] = mean of the 2 x 2 block
__global__ void k_avgpool(const bf16 *x, bf16 *y, int nimg, int H, int W, int C) {
  const unsigned Ho = H / 2, Wo = W / 2, cc = C / 8;
  GRID_STRIDE_U(e, (unsigned)nimg * Ho * Wo * cc) {
    const unsigned c = e % cc, q = e / cc;
    const unsigned xo = q % Wo, yo = (q / Wo) % Ho, n = q / (Wo * Ho);
    const uint4 *src = reinterpret_cast<const uint4 *>(x + (((long long)n * H + 2 * yo) * W + 2 * xo) * C) + c;
    const long long row = (long long)W * C / 8;
    float a[8], b2[8], c2[8], d[8], o[8];
    unpack8(src[0], a);
    unpack8(src[C / 8], b2);
    unpack8(src[row], c2);
    unpack8(src[row + C / 8], d);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = 0.25f * (a[k] + b2[k] + c2[k] + d[k]);
    reinterpret_cast<uint4 *>(y)[e] = pack8(o);
  }
}
// gradient of avgpool, added into gx (which already holds the skip gradient)
__global__ void k_avgpool_bwd_add(const bf16 *gy, bf16 *gx, int nimg, int H, int W, int C) {
  const unsigned Ho = H / 2, Wo = W / 2, cc = C / 8;
  GRID_STRIDE_U(e, (unsigned)nimg * H * W * cc) {
    const unsigned c = e % cc, q = e / cc;
    const unsigned x = q % W, y = (q / W) % H, n = q / (W * H);
    float gv[8], xv[8];
    unpack8(reinterpret_cast<const uint4 *>(gy + (((long long)n * Ho + y / 2) * Wo + x / 2) * C)[c], gv);
    unpack8(reinterpret_cast<const uint4 *>(gx)[e], xv);
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] += 0.25f * gv[k];
    reinterpret_cast<uint4 *>(gx)[e] = pack8(xv);
  }
}
// out [n][2H][2W][C1 + C2] = [upsample(a) (C1) | skip (C2)]
__global__ void k_upsample_concat(const bf16 *a, const bf16 *skip, bf16 *out, int nimg, int H, int W, int C1, int C2) {
  const unsigned Ho = 2 * H, Wo = 2 * W, cc = (C1 + C2) / 8, c1 = C1 / 8;
  GRID_STRIDE_U(e, (unsigned)nimg * Ho * Wo * cc) {
    const unsigned c = e % cc, q = e / cc;
    const unsigned x = q % Wo, y = (q / Wo) % Ho, n = q / (Wo * Ho);
    const uint4 v = c < c1 ? reinterpret_cast<const uint4 *>(a + (((long long)n * H + y / 2) * W + x / 2) * C1)[c]
                           : reinterpret_cast<const uint4 *>(skip + (long long)q * C2)[c - c1];
    reinterpret_cast<uint4 *>(out)[e] = v;
  }
}
// split the gradient of the concatenation: ga = upsample^T of the first C1
// channels (H x W output), gs = the remaining C2 channels
__global__ void k_upsample_concat_bwd(const bf16 *g, bf16 *ga, bf16 *gs, int nimg, int H, int W, int C1, int C2) {
  const unsigned Ho = 2 * H, Wo = 2 * W, cc = (C1 + C2) / 8, c1 = C1 / 8, c2 = C2 / 8;
  GRID_STRIDE_U(e, (unsigned)nimg * H * W * c1) {
    const unsigned c = e % c1, q = e / c1;
    const unsigned x = q % W, y = (q / W) % H, n = q / (W * H);
    const uint4 *src = reinterpret_cast<const uint4 *>(g) + ((long long)(n * Ho + 2 * y) * Wo + 2 * x) * cc + c;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, t[8];
#pragma unroll
    for (int dq = 0; dq < 4; ++dq) {
      unpack8(src[((long long)(dq >> 1) * Wo + (dq & 1)) * cc], t);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += t[k];
    }
    reinterpret_cast<uint4 *>(ga)[e] = pack8(s);
  }
  GRID_STRIDE_U(e2, (unsigned)nimg * Ho * Wo * c2) {
    const unsigned c = e2 % c2, q = e2 / c2;
    reinterpret_cast<uint4 *>(gs)[e2] = reinterpret_cast<const uint4 *>(g)[(long long)q * cc + c1 + c];
  }
}
// db[c] += sum over pixels of g[p][c]
// With y given, the ReLU mask is applied on the way: g[p][c] = 0 where
// y[p][c] <= 0, written back, and the sums taken of the masked gradient.
__global__ void k_bias_grad(bf16 *g, const bf16 *y, float *db, long long P, int C) {
  // a thread reads one 8-channel chunk (16 bytes) per pixel; the grid's
  // thread count is a multiple of the C / 8 chunks, so it always sums the
  // same chunk, in registers, then per block in shared memory
  extern __shared__ float red[];  // [C]
  for (int t = threadIdx.x; t < C; t += blockDim.x) red[t] = 0.f;
  __syncthreads();
  const int nch = C / 8;
  const int c = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) % nch);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  GRID_STRIDE(e, P * nch) {
    float v[8];
    unpack8(reinterpret_cast<const uint4 *>(g)[e], v);
    if (y) {
      float yv[8];
      unpack8(reinterpret_cast<const uint4 *>(y)[e], yv);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(yv[k] > 0.f)) v[k] = 0.f;
      reinterpret_cast<uint4 *>(g)[e] = pack8(v);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += v[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) atomicAdd(&red[c * 8 + k], acc[k]);
  __syncthreads();
  for (int t = threadIdx.x; t < C; t += blockDim.x) atomicAdd(db + t, red[t]);
}
// head: y[p][o] = b[o] + sum_i W[i][o] x[p][i] (FP32 out); one pixel per
// thread, W and b staged in shared memory (dynamic, Ci * CO + CO floats), Ci
// a multiple of 8
template <int CO>
__global__ void __launch_bounds__(256) k_head_fwd(const bf16 *x, const float *Wh, const float *bh, float *y,
                                                  unsigned P, int Ci) {
  extern __shared__ float sw[];
  for (int t = threadIdx.x; t < Ci * CO + CO; t += blockDim.x) sw[t] = t < Ci * CO ? Wh[t] : bh[t - Ci * CO];
  __syncthreads();
  GRID_STRIDE_U(p, P) {
    float acc[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[o] = sw[Ci * CO + o];
    const uint4 *xp = reinterpret_cast<const uint4 *>(x + (long long)p * Ci);
    for (int c = 0; c < Ci / 8; ++c) {
      float xv[8];
      unpack8(xp[c], xv);
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int o = 0; o < CO; ++o) acc[o] = fmaf(sw[(c * 8 + k) * CO + o], xv[k], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < CO; ++o) y[(long long)p * CO + o] = acc[o];
  }
}
// loss: sum of squared errors (one atomic per block) and gy = 2 (y - t) / count
__global__ void __launch_bounds__(256) k_mse(const float *y, const float *t, float *gy, long long n,
                                             float *loss_sum) {
  __shared__ float red[8];
  float s = 0.f;
  const float sc = 2.0f / (float)n;
  GRID_STRIDE(e, n) {
    const float d = y[e] - t[e];
    s += d * d;
    gy[e] = sc * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
    atomicAdd(loss_sum, b);
  }
}
// head backward: gx[p][i] = sum_o W[i][o] gy[p][o] (bf16); dW, db.  A thread
// takes one 8-channel chunk of a pixel (16-byte loads and stores, a warp
// covering consecutive chunks); the grid's thread count is a multiple of the
// Ci / 8 chunks, so every thread keeps one chunk and sums its dW in registers,
// then per block in shared memory, then atomically.  Shared memory (dynamic):
// W [Ci * CO], partial sums [Ci * CO + CO].
template <int CO>
__global__ void __launch_bounds__(256) k_head_bwd(const bf16 *x, const float *gy, const float *Wh, bf16 *gx,
                                                  float *dWh, float *dbh, long long P, int Ci) {
  extern __shared__ float sm[];
  float *sw = sm, *part = sm + Ci * CO;
  for (int t = threadIdx.x; t < Ci * CO; t += blockDim.x) sw[t] = Wh[t];
  for (int t = threadIdx.x; t < Ci * CO + CO; t += blockDim.x) part[t] = 0.f;
  __syncthreads();
  const int nch = Ci / 8;
  const int c = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) % nch);
  float aw[8][CO], ab[CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    ab[o] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) aw[k][o] = 0.f;
  }
  GRID_STRIDE(e, P * nch) {
    const long long p = e / nch;
    float g[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) g[o] = gy[p * CO + o];
    float xv[8], gv[8];
    unpack8(reinterpret_cast<const uint4 *>(x)[e], xv);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float sk = 0.f;
#pragma unroll
      for (int o = 0; o < CO; ++o) {
        sk = fmaf(sw[(c * 8 + k) * CO + o], g[o], sk);
        aw[k][o] = fmaf(xv[k], g[o], aw[k][o]);
      }
      gv[k] = sk;
    }
#pragma unroll
    for (int o = 0; o < CO; ++o) ab[o] += g[o];
    reinterpret_cast<uint4 *>(gx)[e] = pack8(gv);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int o = 0; o < CO; ++o) atomicAdd(&part[(c * 8 + k) * CO + o], aw[k][o]);
  if (c == 0)
#pragma unroll
    for (int o = 0; o < CO; ++o) atomicAdd(&part[Ci * CO + o], ab[o]);
  __syncthreads();
  for (int t = threadIdx.x; t < Ci * CO; t += blockDim.x) atomicAdd(dWh + t, part[t]);
  for (int t = threadIdx.x; t < CO; t += blockDim.x) atomicAdd(dbh + t, part[Ci * CO + t]);
}
// Adam (Kingma & Ba) on FP32 parameters; bias corrections c1 = 1 - b1^t,
// c2 = 1 - b2^t passed in
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  GRID_STRIDE(e, n) {
    const float ge = g[e];
    const float mn = b1 * m[e] + (1.f - b1) * ge;
    const float vn = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = mn;
    v[e] = vn;
    p[e] -= lr * (mn / c1) / (sqrtf(vn / c2) + eps);
  }
}
// BF16 copies of a conv layer's weights, K-major for the tensor cores:
// forward wf[co][tap * Cin + ci] and data-gradient wd[ci][tap' * Cout + co]
// with tap' = 8 - tap (the data gradient of a 'same' 3x3 convolution is the
// convolution of the output gradient with the flipped, transposed kernel).
__global__ void k_weights_bf16(const float *w, bf16 *wf, bf16 *wd, int Cin_real, int Cin, int Cout) {
  GRID_STRIDE(e, 9LL * Cin * Cout) {
    const int co = (int)(e % Cout);
    const int ci = (int)((e / Cout) % Cin);
    const int tap = (int)(e / ((long long)Cout * Cin));
    const float val = ci < Cin_real ? w[((long long)tap * Cin_real + ci) * Cout + co] : 0.f;
    const bf16 b = __float2bfloat16_rn(val);
    wf[(long long)co * 9 * Cin + (long long)tap * Cin + ci] = b;
    wd[(long long)ci * 9 * Cout + (long long)(8 - tap) * Cout + co] = b;
  }
}
// gradient of the padded first layer back to the real input channels
__global__ void k_unpad_wgrad(const float *gpad, float *g, int Cin_real, int Cin, int Cout) {
  GRID_STRIDE(e, 9LL * Cin_real * Cout) {
    const int co = (int)(e % Cout);
    const int ci = (int)((e / Cout) % Cin_real);
    const int tap = (int)(e / ((long long)Cout * Cin_real));
    g[e] = gpad[((long long)tap * Cin + ci) * Cout + co];
  }
}

unsigned grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

// The head for CO output channels (compile time: its sums stay in registers).
template <int CO>
cudaError_t head_launch(const bf16 *x, const float *Wh, const float *bh, float *y, const bf16 *xb, const float *gy,
                        bf16 *gx, float *dWh, float *dbh, long long P, int Ci, bool backward, cudaStream_t s) {
  if (!backward) {
    k_head_fwd<CO><<<grid_for(P), 256, (Ci * CO + CO) * sizeof(float), s>>>(x, Wh, bh, y, (unsigned)P, Ci);
  } else {
    // a bounded grid: each thread loops over many pixels with its sums in
    // registers before the per-block reduction
    k_head_bwd<CO><<<std::min<unsigned>(grid_for(P * (Ci / 8)), 1216u), 256, (2 * Ci * CO + CO) * sizeof(float),
                     s>>>(xb, gy, Wh, gx, dWh, dbh, P, Ci);
  }
  return cudaGetLastError();
}
cudaError_t head_dispatch(int Co, const bf16 *x, const float *Wh, const float *bh, float *y, const bf16 *xb,
                          const float *gy, bf16 *gx, float *dWh, float *dbh, long long P, int Ci, bool backward,
                          cudaStream_t s) {
  switch (Co) {
    case 1: return head_launch<1>(x, Wh, bh, y, xb, gy, gx, dWh, dbh, P, Ci, backward, s);
    case 2: return head_launch<2>(x, Wh, bh, y, xb, gy, gx, dWh, dbh, P, Ci, backward, s);
    case 3: return head_launch<3>(x, Wh, bh, y, xb, gy, gx, dWh, dbh, P, Ci, backward, s);
    case 4: return head_launch<4>(x, Wh, bh, y, xb, gy, gx, dWh, dbh, P, Ci, backward, s);
    case 8: return head_launch<8>(x, Wh, bh, y, xb, gy, gx, dWh, dbh, P, Ci, backward, s);
    case 16: return head_launch<16>(x, Wh, bh, y, xb, gy, gx, dWh, dbh, P, Ci, backward, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t head_fwd(const bf16 *x, const float *Wh, const float *bh, float *y, long long P, int Ci, int Co,
                     cudaStream_t s) {
  return head_dispatch(Co, x, Wh, bh, y, nullptr, nullptr, nullptr, nullptr, nullptr, P, Ci, false, s);
}
cudaError_t head_bwd(const bf16 *x, const float *gy, const float *Wh, bf16 *gx, float *dWh, float *dbh, long long P,
                     int Ci, int Co, cudaStream_t s) {
  return head_dispatch(Co, nullptr, Wh, nullptr, nullptr, x, gy, gx, dWh, dbh, P, Ci, true, s);
}

}  // namespace

// ===========================================================================
// Host-side network object.
struct ConvLayer {
  int cin_real, cin, cout;
  long long w_off, b_off;    // in the FP32 parameter vector
  long long wpad_elems;      // 9 * cin * cout
  bf16 *wf = nullptr, *wd = nullptr;
  float *dwpad = nullptr;    // FP32 weight gradient in padded layout (first layer)
};

struct tacchi_nn {
  cudaStream_t stream = nullptr;
  int L = 0;
  std::vector<int> widths;
  int cin_real = 0, cin = 0, cout = 0, H = 0, W = 0, max_batch = 0;
  std::vector<ConvLayer> convs;  // execution order (enc0a, enc0b, ..., dec0b)
  long long head_w = 0, head_b = 0, nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 params, grads, Adam moments
  int t = 0;
  // activations (bf16) and their gradients, per conv layer input/output
  std::vector<bf16 *> act;    // act[0] = packed input; act[k+1] = output of conv k
  std::vector<bf16 *> gact;   // gradients, same shapes
  std::vector<long long> act_elems;
  std::vector<int> act_h, act_c;
  std::vector<bf16 *> pooled, gpooled;  // per encoder level < L-1
  std::vector<bf16 *> cat, gcat, gup;   // per decoder level
  float *out = nullptr, *gout = nullptr, *loss = nullptr, *h_loss = nullptr;
  int *err = nullptr;  // device: a tensor-core wait gave up
  size_t device_bytes = 0;
};

namespace {

template <typename T>
cudaError_t nalloc(tacchi_nn *n, T **ptr, size_t count) {
  cudaError_t e = cudaMalloc((void **)ptr, sizeof(T) * std::max<size_t>(count, 1));
  if (e == cudaSuccess) n->device_bytes += sizeof(T) * count;
  return e;
}

tacchi_status st_of(cudaError_t e) { return e == cudaSuccess ? TACCHI_OK : TACCHI_ERR_CUDA; }

// Synchronise the network's stream and report a tensor-core wait that gave up
// (sticky until the network is destroyed).
tacchi_status nn_sync(tacchi_nn *n) {
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) return TACCHI_ERR_CUDA;
  int e = 0;
  if (cudaMemcpy(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TACCHI_ERR_CUDA;
  return e ? TACCHI_ERR_TIMEOUT : TACCHI_OK;
}
#define NCK(x)                                 \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return st_of(e_);   \
  } while (0)

// Ring depth per tile width.  A tile is a few small loads re-read from L2
// (nine taps of 8 KB for C_in = 32), so the layer is bound by the loads in
// flight per SM: a shallow ring lets more CTAs share an SM (N <= 64: 31-38 KB
// of shared memory, five to seven CTAs; N = 128: four), as long as their
// tensor-memory columns fit its 512 (N >= 192: two CTAs of 256 columns).
template <int N>
constexpr int conv_stages() {
  return N <= 64 ? 3 : (N == 128 ? 3 : 4);
}
template <int N>
constexpr int conv_tcols() {
  return N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
}
template <int N>
constexpr int conv_smem() {
  return conv_stages<N>() * (128 * 32 * 2 + N * 32 * 2) + 1024;  // + alignment slack
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the CUDA runtime).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

template <int N>
cudaError_t conv_launch(const bf16 *X, const bf16 *Wk, const float *bias, bf16 *Y, int nimg, int H, int W, int Cin,
                        int Cout, int relu, int *err, cudaStream_t s) {
  constexpr int S = conv_stages<N>(), TC = conv_tcols<N>();
  static bool ready = false;  // the dynamic shared memory limit, once per instantiation
  if (!ready) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_conv3x3_tc<N, S, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem<N>());
    if (e != cudaSuccess) return e;
    ready = true;
  }
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  // the 128-pixel box of a tile: whole image rows (W and H are powers of two)
  const int wb = W < 128 ? W : 128;
  const int hb = H < 128 / wb ? H : 128 / wb;
  const int nb = 128 / (wb * hb);
  if (wb * hb * nb != 128 || W % wb || H % hb) return cudaErrorInvalidValue;
  CUtensorMap tmX, tmW;
  const cuuint64_t gdX[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nimg};
  const cuuint64_t gsX[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
  const cuuint32_t bxX[4] = {32, (cuuint32_t)wb, (cuuint32_t)hb, (cuuint32_t)nb}, es[4] = {1, 1, 1, 1};
  const cuuint64_t gdW[2] = {(cuuint64_t)9 * Cin, (cuuint64_t)Cout};
  const cuuint64_t gsW[1] = {(cuuint64_t)9 * Cin * 2};
  const cuuint32_t bxW[2] = {32, (cuuint32_t)N};
  if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)X, gdX, gsX, bxX, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS ||
      enc(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)Wk, gdW, gsW, bxW, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const long long M = (long long)nimg * H * W;
  dim3 grid((unsigned)((M + 127) / 128), (unsigned)(Cout / N));
  k_conv3x3_tc<N, S, TC><<<grid, 128, conv_smem<N>(), s>>>(tmX, tmW, bias, Y, nimg, H, W, Cin, Cout, relu, err);
  return cudaGetLastError();
}

// Output-channel tile: the largest UMMA width (a multiple of 16, at most 256)
// that divides Cout (a multiple of 32).
cudaError_t conv_fwd(const bf16 *X, const bf16 *Wk, const float *bias, bf16 *Y, int nimg, int H, int W, int Cin,
                     int Cout, int relu, int *err, cudaStream_t s) {
  if (Cout % 256 == 0) return conv_launch<256>(X, Wk, bias, Y, nimg, H, W, Cin, Cout, relu, err, s);
  if (Cout % 192 == 0) return conv_launch<192>(X, Wk, bias, Y, nimg, H, W, Cin, Cout, relu, err, s);
  if (Cout % 128 == 0) return conv_launch<128>(X, Wk, bias, Y, nimg, H, W, Cin, Cout, relu, err, s);
  if (Cout % 96 == 0) return conv_launch<96>(X, Wk, bias, Y, nimg, H, W, Cin, Cout, relu, err, s);
  if (Cout % 64 == 0) return conv_launch<64>(X, Wk, bias, Y, nimg, H, W, Cin, Cout, relu, err, s);
  return conv_launch<32>(X, Wk, bias, Y, nimg, H, W, Cin, Cout, relu, err, s);
}

template <int NC>
cudaError_t wgrad_launch(const CUtensorMap &tmX, const CUtensorMap &tmG, float *dW, int P, int H, int W, int Cin,
                         int Cout, int *err, cudaStream_t s) {
  constexpr int S = 2;  // a shallow ring: more CTAs per SM hide the load latency better
  constexpr int TC = NC <= 32 ? 32 : (NC <= 64 ? 64 : (NC <= 128 ? 128 : 256));
  constexpr int SMEM = S * (4 + NC / 32) * 4096 + 1024;
  static bool ready = false;
  if (!ready) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_conv3x3_wgrad_tc<NC, S, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    ready = true;
  }
  const int mt = (9 * Cin + 127) / 128, ny = Cout / NC;
  // pixel chunks (multiples of 64) so that the grid gives every SM about
  // four CTAs; each CTA adds its partial sums to dW
  const long long stages = ((long long)P + 63) / 64;
  long long want = (152LL * 4 + (long long)mt * ny - 1) / ((long long)mt * ny);
  if (want < 1) want = 1;
  long long per = (stages + want - 1) / want;
  if (per < 4) per = 4;
  const int chunk = (int)(per * 64);
  dim3 grid((unsigned)mt, (unsigned)ny, (unsigned)((P + chunk - 1) / chunk));
  k_conv3x3_wgrad_tc<NC, S, TC><<<grid, 128, SMEM, s>>>(tmX, tmG, dW, P, H, W, Cin, Cout, chunk, err);
  return cudaGetLastError();
}

// dW (FP32, [9 Cin][Cout], accumulated into) += the weight gradient of a 3x3
// 'same' convolution with input X [nimg][H][W][Cin] and output gradient
// G [nimg][H][W][Cout] (BF16).
cudaError_t conv_wgrad(const bf16 *X, const bf16 *G, float *dW, int nimg, int H, int W, int Cin, int Cout, int *err,
                       cudaStream_t s) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const int P = nimg * H * W;
  // 64-pixel boxes of whole image rows (W and H are powers of two)
  const int wb = W < 64 ? W : 64;
  const int hb = H < 64 / wb ? H : 64 / wb;
  const int nb = 64 / (wb * hb);
  if (wb * hb * nb != 64 || W % wb || H % hb) return cudaErrorInvalidValue;
  CUtensorMap tmX, tmG;
  const cuuint64_t gdX[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nimg};
  const cuuint64_t gsX[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
  const cuuint32_t bxX[4] = {32, (cuuint32_t)wb, (cuuint32_t)hb, (cuuint32_t)nb}, es[4] = {1, 1, 1, 1};
  const cuuint64_t gdG[2] = {(cuuint64_t)Cout, (cuuint64_t)P};
  const cuuint64_t gsG[1] = {(cuuint64_t)Cout * 2};
  const cuuint32_t bxG[2] = {32, 64};
  if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)X, gdX, gsX, bxX, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS ||
      enc(&tmG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)G, gdG, gsG, bxG, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if (Cout % 256 == 0) return wgrad_launch<256>(tmX, tmG, dW, P, H, W, Cin, Cout, err, s);
  if (Cout % 128 == 0) return wgrad_launch<128>(tmX, tmG, dW, P, H, W, Cin, Cout, err, s);
  if (Cout % 64 == 0) return wgrad_launch<64>(tmX, tmG, dW, P, H, W, Cin, Cout, err, s);
  return wgrad_launch<32>(tmX, tmG, dW, P, H, W, Cin, Cout, err, s);
}

// db += sum over pixels of G; with Y, G is first masked by ReLU'(Y) in place
cudaError_t mask_bias_grad(bf16 *G, const bf16 *Y, float *db, long long P, int C, cudaStream_t s) {
  const int nch = C / 8;
  if (C % 8 || nch < 1 || nch > 1024) return cudaErrorInvalidValue;
  const int threads = nch * (256 / nch > 0 ? 256 / nch : 1);  // a multiple of the chunks
  k_bias_grad<<<512, threads, C * sizeof(float), s>>>(G, Y, db, P, C);
  return cudaGetLastError();
}

cudaError_t refresh_weights(tacchi_nn *n) {
  for (auto &cl : n->convs) {
    k_weights_bf16<<<grid_for(cl.wpad_elems), 256, 0, n->stream>>>(n->p + cl.w_off, cl.wf, cl.wd, cl.cin_real,
                                                                   cl.cin, cl.cout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void release_nn(tacchi_nn *n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  for (auto &cl : n->convs) {
    cudaFree(cl.wf);
    cudaFree(cl.wd);
    cudaFree(cl.dwpad);
  }
  for (auto *q : n->act) cudaFree(q);
  for (auto *q : n->gact) cudaFree(q);
  for (auto *q : n->pooled) cudaFree(q);
  for (auto *q : n->gpooled) cudaFree(q);
  for (auto *q : n->cat) cudaFree(q);
  for (auto *q : n->gcat) cudaFree(q);
  for (auto *q : n->gup) cudaFree(q);
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->out);
  cudaFree(n->gout);
  cudaFree(n->loss);
  cudaFree(n->err);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  delete n;
}

// Forward pass for `batch` images; x fp32 [batch][H][W][cin_real] (device).
tacchi_status forward(tacchi_nn *n, int batch, const float *x) {
  cudaStream_t s = n->stream;
  const long long P0 = (long long)batch * n->H * n->W;
  k_pack_input<<<grid_for(P0 * n->cin / 8), 256, 0, s>>>(x, n->act[0], (unsigned)P0, n->cin_real, n->cin);
  NCK(cudaGetLastError());
  int k = 0;
  int H = n->H, W = n->W;
  const bf16 *in = n->act[0];
  for (int l = 0; l < n->L; ++l) {
    for (int q = 0; q < 2; ++q, ++k) {
      ConvLayer &cl = n->convs[k];
      NCK(conv_fwd(in, cl.wf, n->p + cl.b_off, n->act[k + 1], batch, H, W, cl.cin, cl.cout, 1, n->err, s));
      in = n->act[k + 1];
    }
    if (l < n->L - 1) {
      k_avgpool<<<grid_for((long long)batch * H * W * n->widths[l] / 32), 256, 0, s>>>(in, n->pooled[l], batch, H, W,
                                                                                       n->widths[l]);
      NCK(cudaGetLastError());
      in = n->pooled[l];
      H /= 2;
      W /= 2;
    }
  }
  for (int l = n->L - 2; l >= 0; --l) {
    const int C1 = n->widths[l + 1], C2 = n->widths[l];
    const bf16 *skip = n->act[2 * l + 2];  // output of enc{l}b
    k_upsample_concat<<<grid_for((long long)batch * 4 * H * W * (C1 + C2) / 8), 256, 0, s>>>(in, skip, n->cat[l], batch, H,
                                                                                         W, C1, C2);
    NCK(cudaGetLastError());
    H *= 2;
    W *= 2;
    in = n->cat[l];
    for (int q = 0; q < 2; ++q, ++k) {
      ConvLayer &cl = n->convs[k];
      NCK(conv_fwd(in, cl.wf, n->p + cl.b_off, n->act[k + 1], batch, H, W, cl.cin, cl.cout, 1, n->err, s));
      in = n->act[k + 1];
    }
  }
  NCK(head_fwd(in, n->p + n->head_w, n->p + n->head_b, n->out, P0, n->widths[0], n->cout, s));
  return TACCHI_OK;
}

// Loss and gradients of every parameter into n->g (zeroed first).
tacchi_status backward(tacchi_nn *n, int batch, const float *target) {
  cudaStream_t s = n->stream;
  const long long P0 = (long long)batch * n->H * n->W;
  NCK(cudaMemsetAsync(n->g, 0, sizeof(float) * n->nparams, s));
  NCK(cudaMemsetAsync(n->loss, 0, sizeof(float), s));
  k_mse<<<std::min<unsigned>(grid_for(P0 * n->cout), 1216u), 256, 0, s>>>(n->out, target, n->gout, P0 * n->cout,
                                                                          n->loss);
  NCK(cudaGetLastError());
  const int nk = (int)n->convs.size();
  const int C0 = n->widths[0];
  NCK(head_bwd(n->act[nk], n->gout, n->p + n->head_w, n->gact[nk], n->g + n->head_w, n->g + n->head_b, P0, C0,
               n->cout, s));

  // layer k's input activation and the gradient buffer of that input
  int H = n->H, W = n->W;
  int k = nk - 1;
  bf16 *gcur = n->gact[nk];  // gradient of the output of conv k
  // decoder, level 0 first
  for (int l = 0; l <= n->L - 2; ++l) {
    for (int q = 0; q < 2; ++q, --k) {
      ConvLayer &cl = n->convs[k];
      const long long P = (long long)batch * H * W;
      // ReLU mask and bias gradient in one pass over the output gradient
      NCK(mask_bias_grad(gcur, n->act[k + 1], n->g + cl.b_off, P, cl.cout, s));
      const bf16 *xin = q == 0 ? n->act[k] : n->cat[l];
      bf16 *gin = q == 0 ? n->gact[k] : n->gcat[l];
      NCK(conv_wgrad(xin, gcur, n->g + cl.w_off, batch, H, W, cl.cin, cl.cout, n->err, s));
      NCK(conv_fwd(gcur, cl.wd, nullptr, gin, batch, H, W, cl.cout, cl.cin, 0, n->err, s));
      gcur = gin;
    }
    // split the concatenation gradient: upsampled part and skip part
    const int C1 = n->widths[l + 1], C2 = n->widths[l];
    bf16 *gskip = n->gact[2 * l + 2];  // gradient of enc{l}b output (skip part first)
    k_upsample_concat_bwd<<<grid_for((long long)batch * H * W * C2 / 8), 256, 0, s>>>(gcur, n->gup[l], gskip, batch, H / 2,
                                                                                  W / 2, C1, C2);
    NCK(cudaGetLastError());
    gcur = n->gup[l];  // gradient of the level l+1 output (decoder or bottom)
    H /= 2;
    W /= 2;
  }
  // encoder, bottom level first
  k = 2 * n->L - 1;
  for (int l = n->L - 1; l >= 0; --l) {
    if (l < n->L - 1) {
      // gradient of enc{l}b output = skip gradient (already in gact) + pool^T
      bf16 *genc = n->gact[2 * l + 2];
      k_avgpool_bwd_add<<<grid_for((long long)batch * H * W * n->widths[l] / 8), 256, 0, s>>>(gcur, genc, batch, H, W,
                                                                                         n->widths[l]);
      NCK(cudaGetLastError());
      gcur = genc;
    } else {
      // bottom: gradient arrives in gup[L-2]; copy it to the bottom output's buffer
      const long long P = (long long)batch * H * W;
      if (gcur != n->gact[2 * l + 2])
        NCK(cudaMemcpyAsync(n->gact[2 * l + 2], gcur, sizeof(bf16) * P * n->widths[l], cudaMemcpyDeviceToDevice, s));
      gcur = n->gact[2 * l + 2];
    }
    for (int q = 0; q < 2; ++q, --k) {
      ConvLayer &cl = n->convs[k];
      const long long P = (long long)batch * H * W;
      NCK(mask_bias_grad(gcur, n->act[k + 1], n->g + cl.b_off, P, cl.cout, s));
      const bf16 *xin = (q == 1 && l > 0) ? n->pooled[l - 1] : n->act[k];
      float *dW = (k == 0) ? n->convs[0].dwpad : n->g + cl.w_off;
      if (k == 0) NCK(cudaMemsetAsync(dW, 0, sizeof(float) * cl.wpad_elems, s));
      NCK(conv_wgrad(xin, gcur, dW, batch, H, W, cl.cin, cl.cout, n->err, s));
      if (k == 0) {
        k_unpad_wgrad<<<grid_for(9LL * cl.cin_real * cl.cout), 256, 0, s>>>(dW, n->g + cl.w_off, cl.cin_real, cl.cin,
                                                                            cl.cout);
        NCK(cudaGetLastError());
      } else {
        bf16 *gin = q == 0 ? n->gact[k] : n->gpooled[l - 1];
        NCK(conv_fwd(gcur, cl.wd, nullptr, gin, batch, H, W, cl.cout, cl.cin, 0, n->err, s));
        gcur = gin;
      }
    }
    if (l > 0) {
      H *= 2;
      W *= 2;
    }
  }
  return TACCHI_OK;
}

}  // namespace

extern "C" {

tacchi_status tacchi_nn_create(int levels, const int *widths, int in_channels, int out_channels, int height,
                               int width, int max_batch, uint64_t seed, void *stream, tacchi_nn_handle *out) {
  if (!out || !widths || levels < 1 || levels > 6 || in_channels < 1 || in_channels > 32 || out_channels < 1 ||
      out_channels > 16 || (out_channels > 4 && out_channels != 8 && out_channels != 16) || max_batch < 1 ||
      height < 1 || width < 1)
    return TACCHI_ERR_INVALID_ARG;
  *out = nullptr;
  if (height % (1 << (levels - 1)) || width % (1 << (levels - 1))) return TACCHI_ERR_INVALID_ARG;
  if (256 % widths[0]) return TACCHI_ERR_INVALID_ARG;  // the head kernel keeps one channel per thread
  for (int l = 0; l < levels; ++l)
    if (widths[l] < 32 || widths[l] % 32 || widths[l] > 1024) return TACCHI_ERR_INVALID_ARG;
  // elementwise kernels index 8-channel chunks of a level's tensors with
  // 32-bit integers: every level (with its concatenation) stays below 2^32
  for (int l = 0; l < levels; ++l) {
    const double P = (double)max_batch * (height >> l) * (width >> l);
    const int c = widths[l] + (l + 1 < levels ? widths[l + 1] : 0);
    if (P * c > 4.0e9) return TACCHI_ERR_INVALID_ARG;
  }
  tacchi_nn *n = new (std::nothrow) tacchi_nn();
  if (!n) return TACCHI_ERR_OOM;
  n->stream = (cudaStream_t)stream;
  n->L = levels;
  n->widths.assign(widths, widths + levels);
  n->cin_real = in_channels;
  n->cin = 32;
  n->cout = out_channels;
  n->H = height;
  n->W = width;
  n->max_batch = max_batch;
  // parameter layout: per conv (execution order) W [3][3][cin_real][cout] then
  // b [cout]; then head W [widths0][cout], b [cout]
  long long off = 0;
  auto add_conv = [&](int cin_real, int cin, int cout) {
    ConvLayer cl;
    cl.cin_real = cin_real;
    cl.cin = cin;
    cl.cout = cout;
    cl.w_off = off;
    off += 9LL * cin_real * cout;
    cl.b_off = off;
    off += cout;
    cl.wpad_elems = 9LL * cin * cout;
    n->convs.push_back(cl);
  };
  for (int l = 0; l < levels; ++l) {
    if (l == 0) add_conv(in_channels, 32, widths[0]);
    else add_conv(widths[l - 1], widths[l - 1], widths[l]);
    add_conv(widths[l], widths[l], widths[l]);
  }
  for (int l = levels - 2; l >= 0; --l) {
    add_conv(widths[l + 1] + widths[l], widths[l + 1] + widths[l], widths[l]);
    add_conv(widths[l], widths[l], widths[l]);
  }
  n->head_w = off;
  off += (long long)widths[0] * out_channels;
  n->head_b = off;
  off += out_channels;
  n->nparams = off;
  auto fail = [&](tacchi_status s) {
    release_nn(n);
    return s;
  };
  bool ok = nalloc(n, &n->p, off) == cudaSuccess && nalloc(n, &n->g, off) == cudaSuccess &&
            nalloc(n, &n->m, off) == cudaSuccess && nalloc(n, &n->v, off) == cudaSuccess;
  for (auto &cl : n->convs)
    ok = ok && nalloc(n, &cl.wf, cl.wpad_elems) == cudaSuccess && nalloc(n, &cl.wd, cl.wpad_elems) == cudaSuccess;
  ok = ok && nalloc(n, &n->convs[0].dwpad, n->convs[0].wpad_elems) == cudaSuccess;
  // activations: act[0] input (32 ch), act[k+1] output of conv k
  const long long B = max_batch;
  int H = height, W = width;
  std::vector<long long> sizes;
  sizes.push_back(B * H * W * 32);
  for (int l = 0; l < levels; ++l) {
    sizes.push_back(B * H * W * widths[l]);
    sizes.push_back(B * H * W * widths[l]);
    if (l < levels - 1) {
      H /= 2;
      W /= 2;
    }
  }
  for (int l = levels - 2; l >= 0; --l) {
    H *= 2;
    W *= 2;
    sizes.push_back(B * H * W * widths[l]);
    sizes.push_back(B * H * W * widths[l]);
  }
  for (long long sz : sizes) {
    bf16 *a = nullptr, *ga = nullptr;
    ok = ok && nalloc(n, &a, sz) == cudaSuccess && nalloc(n, &ga, sz) == cudaSuccess;
    n->act.push_back(a);
    n->gact.push_back(ga);
  }
  H = height;
  W = width;
  n->pooled.assign(levels, nullptr);
  n->gpooled.assign(levels, nullptr);
  n->cat.assign(levels, nullptr);
  n->gcat.assign(levels, nullptr);
  n->gup.assign(levels, nullptr);
  for (int l = 0; l < levels - 1; ++l) {
    const long long hw = (long long)(H >> l) * (W >> l);
    ok = ok && nalloc(n, &n->pooled[l], B * hw / 4 * widths[l]) == cudaSuccess &&
         nalloc(n, &n->gpooled[l], B * hw / 4 * widths[l]) == cudaSuccess &&
         nalloc(n, &n->cat[l], B * hw * (widths[l] + widths[l + 1])) == cudaSuccess &&
         nalloc(n, &n->gcat[l], B * hw * (widths[l] + widths[l + 1])) == cudaSuccess &&
         nalloc(n, &n->gup[l], B * hw / 4 * widths[l + 1]) == cudaSuccess;
  }
  ok = ok && nalloc(n, &n->out, B * height * width * out_channels) == cudaSuccess &&
       nalloc(n, &n->gout, B * height * width * out_channels) == cudaSuccess &&
       nalloc(n, &n->loss, 1) == cudaSuccess && nalloc(n, &n->err, 1) == cudaSuccess &&
       cudaMallocHost((void **)&n->h_loss, sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return fail(TACCHI_ERR_OOM);
  }
  // He-normal initialisation from splitmix64 + Box-Muller (host, FP64)
  std::vector<float> hp(off, 0.f);
  uint64_t ctr = 0;
  auto uni = [&]() {
    uint64_t z = seed + (++ctr) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * 0x1.0p-53;
  };
  auto gauss = [&]() { return std::sqrt(-2.0 * std::log(uni())) * std::cos(6.283185307179586 * uni()); };
  for (auto &cl : n->convs) {
    const double sd = std::sqrt(2.0 / (9.0 * cl.cin_real));
    for (long long e = 0; e < 9LL * cl.cin_real * cl.cout; ++e) hp[cl.w_off + e] = (float)(sd * gauss());
  }
  const double sdh = std::sqrt(1.0 / widths[0]);
  for (long long e = 0; e < (long long)widths[0] * out_channels; ++e) hp[n->head_w + e] = (float)(sdh * gauss());
  if (cudaMemcpy(n->p, hp.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->m, 0, sizeof(float) * off) != cudaSuccess || cudaMemset(n->v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(n->err, 0, sizeof(int)) != cudaSuccess ||
      refresh_weights(n) != cudaSuccess || cudaStreamSynchronize(n->stream) != cudaSuccess)
    return fail(TACCHI_ERR_CUDA);
  *out = n;
  return TACCHI_OK;
}

void tacchi_nn_destroy(tacchi_nn_handle n) { release_nn(n); }

tacchi_status tacchi_nn_num_params(tacchi_nn_handle n, int64_t *out) {
  if (!n || !out) return TACCHI_ERR_INVALID_ARG;
  *out = n->nparams;
  return TACCHI_OK;
}

tacchi_status tacchi_nn_get_params(tacchi_nn_handle n, int which, float *host) {
  if (!n || !host || which < 0 || which > 1) return TACCHI_ERR_INVALID_ARG;
  NCK(cudaMemcpyAsync(host, which ? n->g : n->p, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost, n->stream));
  return nn_sync(n);
}

tacchi_status tacchi_nn_set_params(tacchi_nn_handle n, const float *host) {
  if (!n || !host) return TACCHI_ERR_INVALID_ARG;
  NCK(cudaMemcpyAsync(n->p, host, sizeof(float) * n->nparams, cudaMemcpyHostToDevice, n->stream));
  NCK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparams, n->stream));
  NCK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparams, n->stream));
  n->t = 0;
  NCK(refresh_weights(n));
  return nn_sync(n);
}

tacchi_status tacchi_nn_forward(tacchi_nn_handle n, int batch, const float *x_dev, float *y_dev) {
  nvtxRangePushA("tacchi_nn_forward");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  if (!n || !x_dev || !y_dev || batch < 1 || batch > n->max_batch) return TACCHI_ERR_INVALID_ARG;
  tacchi_status s = forward(n, batch, x_dev);
  if (s != TACCHI_OK) return s;
  NCK(cudaMemcpyAsync(y_dev, n->out, sizeof(float) * batch * n->H * n->W * n->cout, cudaMemcpyDeviceToDevice,
                      n->stream));
  return TACCHI_OK;
}

tacchi_status tacchi_nn_gradients(tacchi_nn_handle n, int batch, const float *x_dev, const float *target_dev,
                                  float *loss_host) {
  if (!n || !x_dev || !target_dev || batch < 1 || batch > n->max_batch) return TACCHI_ERR_INVALID_ARG;
  tacchi_status s = forward(n, batch, x_dev);
  if (s == TACCHI_OK) s = backward(n, batch, target_dev);
  if (s != TACCHI_OK) return s;
  if (loss_host) {
    NCK(cudaMemcpyAsync(n->h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    const tacchi_status st = nn_sync(n);
    if (st != TACCHI_OK) return st;
    *loss_host = *n->h_loss / (float)((long long)batch * n->H * n->W * n->cout);
  }
  return TACCHI_OK;
}

tacchi_status tacchi_nn_train_step(tacchi_nn_handle n, int batch, const float *x_dev, const float *target_dev,
                                   float lr, float *loss_host) {
  nvtxRangePushA("tacchi_nn_train_step");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  if (!n || !(lr > 0) || !std::isfinite(lr)) return TACCHI_ERR_INVALID_ARG;
  tacchi_status s = tacchi_nn_gradients(n, batch, x_dev, target_dev, nullptr);
  if (s != TACCHI_OK) return s;
  n->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, n->t)), c2 = (float)(1.0 - std::pow(0.999, n->t));
  k_adam<<<grid_for(n->nparams), 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, n->nparams, lr, b1, b2, 1e-8f, c1, c2);
  NCK(cudaGetLastError());
  NCK(refresh_weights(n));
  if (loss_host) {
    NCK(cudaMemcpyAsync(n->h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    const tacchi_status st = nn_sync(n);
    if (st != TACCHI_OK) return st;
    *loss_host = *n->h_loss / (float)((long long)batch * n->H * n->W * n->cout);
  }
  return TACCHI_OK;
}

}  // extern "C"
