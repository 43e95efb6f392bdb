// peak.cu -- FP32 FMA throughput of the current GPU, measured.
//
// The fused MLS-MPM transfer does about 15 FP32 operations per byte it moves,
// so its roofline is the FP32 ALU peak rather than HBM.  This kernel measures
// that peak: every thread runs 8 independent chains of fused multiply-adds,
// in scalar FFMA and in the packed two-lane FFMA2 form, on a grid of whole
// waves over every SM; the rate is 2 flop per FMA lane over the CUDA-event
// time of the launch.
#include <cuda_runtime.h>

#include "tacchi.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, float a, float b, float *sink) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-7f + c, blockIdx.x * 1e-7f - c);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (PACKED) {
        x[c] = __ffma2_rn(x[c], a2, b2);
      } else {
        x[c].x = fmaf(x[c].x, a, b);
        x[c].y = fmaf(x[c].y, a, b);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 1.2345678e-9f) *sink = s;  // keeps the chains live; never taken
}

}  // namespace

extern "C" tacchi_status tacchi_measure_fp32_peak(double *tflops, int *sm_count, int *sm_clock_khz) {
  if (!tflops) return TACCHI_ERR_INVALID_ARG;
  int dev = 0, sms = 0, clk = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TACCHI_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return TACCHI_ERR_CUDA;
  if (cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev) != cudaSuccess) clk = 0;
  if (sm_count) *sm_count = sms;
  if (sm_clock_khz) *sm_clock_khz = clk;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<true>, kThreads, 0) != cudaSuccess ||
      per_sm <= 0)
    return TACCHI_ERR_CUDA;
  float *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  tacchi_status status = TACCHI_OK;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return TACCHI_ERR_OOM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    status = TACCHI_ERR_CUDA;
  const int grid = sms * per_sm * 4;  // four full waves
  const int iters = 1 << 14;
  double best = 0.0;
  for (int variant = 0; variant < 2 && status == TACCHI_OK; ++variant) {
    for (int rep = 0; rep < 4 && status == TACCHI_OK; ++rep) {  // the first run is a warm-up
      cudaEventRecord(e0, st);
      if (variant == 0)
        k_fma_peak<false><<<grid, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f, sink);
      else
        k_fma_peak<true><<<grid, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f, sink);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
        status = TACCHI_ERR_CUDA;
        break;
      }
      const double flop = 2.0 * 2.0 * kChains * (double)iters * kThreads * grid;  // two lanes per chain
      if (rep > 0 && flop / (ms * 1e-3) / 1e12 > best) best = flop / (ms * 1e-3) / 1e12;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(sink);
  if (status == TACCHI_OK) *tflops = best;
  return status;
}
