// layout.cu -- the state load of the bulk phase under three storage layouts (Sec. 3.1, the
// column-major argument around Algorithm 1): a cell's record is (rho, T, Y_0 .. Y_{ns-1}), nv =
// ns + 2 floats, and the kernel computes p = rho R T sum_k Y_k / W_k from it, the same
// all-components-of-one-cell access as the integrators' load.  Layouts:
//   SoA    X[v * ld + i]                          component-major, the library's own layout;
//   AoS    X[i * nv + v]                          cell-major, each thread walks its own record;
//   AoS, staged                                   the same bytes, but a CTA first copies its 128
//                                                 records (contiguous) into shared memory with
//                                                 coalesced 16-byte loads, then reads them there;
//   AoSoA  X[(i / 32) * 32 nv + v * 32 + i % 32]  tiles of 32 cells, component-major inside.
// Each kernel reads nv * 4 bytes and writes 4 bytes per cell; one thread per cell, grid-stride.
#include <cstdint>

#include <cuda_runtime.h>

#include "chem.h"

namespace {

constexpr float kRgasL = 8.314462618f;
constexpr int kLayoutBlock = 128;

struct InvW {
  float v[128];
};

// element v of cell i
template <int L>
__device__ __forceinline__ long long at(long long i, int v, long long ld, int nv) {
  if (L == CHEM_LAYOUT_SOA) return static_cast<long long>(v) * ld + i;
  if (L == CHEM_LAYOUT_AOS) return i * nv + v;
  return (i >> 5) * (32LL * nv) + v * 32 + (i & 31);   // CHEM_LAYOUT_AOSOA
}

template <int NS, int L>
__global__ void __launch_bounds__(kLayoutBlock) p_direct(const float* __restrict__ X, long long ld, long long n,
                                                          float* __restrict__ p, const __grid_constant__ InvW w) {
  constexpr int NV = NS + 2;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < NS; ++k) s = fmaf(X[at<L>(i, 2 + k, ld, NV)], w.v[k], s);
    p[i] = X[at<L>(i, 0, ld, NV)] * kRgasL * X[at<L>(i, 1, ld, NV)] * s;
  }
}

// AoS through shared memory: the 128 records of a CTA are one contiguous run of 128 * NV floats
// (16-byte aligned when the array is), copied with float4 loads, then read per thread (NV odd or
// even, the row stride of NV words keeps the 32 lanes of a warp on distinct banks for odd NV)
template <int NS>
__global__ void __launch_bounds__(kLayoutBlock) p_aos_staged(const float* __restrict__ X, long long n,
                                                              float* __restrict__ p, const __grid_constant__ InvW w) {
  constexpr int NV = NS + 2;
  __shared__ __align__(16) float tile[kLayoutBlock * NV];
  for (long long base = static_cast<long long>(blockIdx.x) * kLayoutBlock; base < n;
       base += static_cast<long long>(gridDim.x) * kLayoutBlock) {
    const long long cells = n - base < kLayoutBlock ? n - base : kLayoutBlock;
    const long long words = cells * NV;
    const float* src = X + base * NV;
    if (cells == kLayoutBlock) {   // full tile: 128 * NV words, a multiple of 4
      const float4* s4 = reinterpret_cast<const float4*>(src);
      float4* d4 = reinterpret_cast<float4*>(tile);
      for (int j = threadIdx.x; j < kLayoutBlock * NV / 4; j += kLayoutBlock) d4[j] = s4[j];
    } else {
      for (long long j = threadIdx.x; j < words; j += kLayoutBlock) tile[j] = src[j];
    }
    __syncthreads();
    if (threadIdx.x < cells) {
      const float* rec = tile + threadIdx.x * NV;
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < NS; ++k) s = fmaf(rec[2 + k], w.v[k], s);
      p[base + threadIdx.x] = rec[0] * kRgasL * rec[1] * s;
    }
    __syncthreads();
  }
}

template <int NS>
int launch_layout(int layout, const float* X, long long ld, long long n, float* p, const InvW& w, int grid,
                  cudaStream_t s) {
  switch (layout) {
    case CHEM_LAYOUT_SOA: p_direct<NS, CHEM_LAYOUT_SOA><<<grid, kLayoutBlock, 0, s>>>(X, ld, n, p, w); break;
    case CHEM_LAYOUT_AOS: p_direct<NS, CHEM_LAYOUT_AOS><<<grid, kLayoutBlock, 0, s>>>(X, ld, n, p, w); break;
    case CHEM_LAYOUT_AOSOA: p_direct<NS, CHEM_LAYOUT_AOSOA><<<grid, kLayoutBlock, 0, s>>>(X, ld, n, p, w); break;
    case CHEM_LAYOUT_AOS_STAGED: p_aos_staged<NS><<<grid, kLayoutBlock, 0, s>>>(X, n, p, w); break;
    default: return CHEM_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? CHEM_OK : CHEM_ECUDA;
}

}  // namespace

extern "C" int chem_pressure_layout(int32_t ns, const double* W, int32_t layout, const float* X, int64_t ld,
                                    int64_t n, float* p, void* stream) {
  if (!W || n < 0 || (n > 0 && (!X || !p))) return CHEM_EINVAL;
  if (layout < CHEM_LAYOUT_SOA || layout > CHEM_LAYOUT_AOS_STAGED) return CHEM_EINVAL;
  if (layout == CHEM_LAYOUT_SOA && ld < n) return CHEM_EINVAL;
  if (layout == CHEM_LAYOUT_AOS_STAGED && (reinterpret_cast<uintptr_t>(X) & 15u)) return CHEM_EINVAL;
  if (ns != 9 && ns != 53) return CHEM_EUNSUPPORTED;
  if (n == 0) return CHEM_OK;
  InvW w{};
  for (int k = 0; k < ns; ++k) {
    if (!(W[k] > 0.0)) return CHEM_EINVAL;
    w.v[k] = static_cast<float>(1.0 / W[k]);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (n + kLayoutBlock - 1) / kLayoutBlock;
  const long long cap = static_cast<long long>(sms > 0 ? sms : 1) * 16;   // 16 CTAs of 128 per SM
  const int grid = static_cast<int>(want < cap ? want : cap);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return ns == 9 ? launch_layout<9>(layout, X, ld, n, p, w, grid, s) : launch_layout<53>(layout, X, ld, n, p, w, grid, s);
}
