// peak.cu -- the FP64 FMA throughput of the current GPU, measured by the library itself.  The
// stiff integrator is bound by the FP64 pipe; its roofline needs the rate that pipe sustains on
// this part, which no vendor table lists for GB300.  The kernel runs independent FP64 FMA chains
// (enough per thread and threads per SM to keep the pipe full) and the host times it with CUDA
// events: FMA count x 2 flops / time.
#include <cstdio>

#include "../../include/chem.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) dfma_chains(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-9 * (threadIdx.x + i);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  out[blockIdx.x * kBlock + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" int chem_measure_fp64_peak(double* tflops, int32_t reps, void* stream) {
  if (!tflops || reps < 1) return CHEM_EINVAL;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CHEM_ECUDA;
  const int grid = sms * 4;   // 32 warps per SM
  const int iters = 4096;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = CHEM_OK;
  if (cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(double) * grid * kBlock, st) != cudaSuccess)
    return CHEM_ENOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = CHEM_ECUDA;
  float best = 0.0f;
  for (int r = 0; r <= reps && rc == CHEM_OK; ++r) {   // the first launch warms up
    cudaEventRecord(e0, st);
    dfma_chains<<<grid, kBlock, 0, st>>>(out, iters, 1.0000000001, 1e-12);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = CHEM_ECUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (rc == CHEM_OK && best > 0.0f)
    *tflops = 2.0 * kChains * static_cast<double>(iters) * grid * kBlock / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  return rc;
}
