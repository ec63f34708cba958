// mlp.cu -- BF16 tensor-core GEMM (tcgen05, FP32 accumulation in TMEM) used by the surrogate's
// training and inference kernels, with fused epilogues (bias, GELU, atomic accumulation).
//
//   C[m, n] = epi( sum_k A(m, k) * B(n, k) ),   A(m, k) = A[m*sam + k*sak], B(n, k) = B[n*sbn + k*sbk]
//
// A and B are FP32 in global memory and are rounded to BF16 while they are staged into shared
// memory in the K-major core-matrix layout (tc.cuh); arbitrary strides let the same kernel serve
// X W^T (forward), dZ W (backward, data) and dZ^T X (backward, weights).  One CTA (4 warps) owns
// 128 rows of C and the whole N (<= 256) extent; K runs in chunks of 64 (4 MMAs of K = 16 per
// chunk, one commit, one bounded mbarrier wait).  gridDim.y splits K; split partial sums are
// added with atomics (EPI_ATOMIC).
#include <cmath>
#include <cstdio>

#include "../../include/chem.h"
#include "internal.h"
#include "tc.cuh"

namespace chem {

enum : int { kEpiStore = 0, kEpiBias = 1, kEpiBiasGelu = 2, kEpiAtomic = 3 };

struct GemmArgs {
  const float* A;
  long long sam, sak;
  const float* B;
  long long sbn, sbk;
  float* C;          // C[m * ldc + n]
  long long ldc;
  float* C2;         // kEpiBiasGelu: gelu(z) here, z in C (may be null)
  const float* bias; // [N]
  int M, N, K, k_per_split, epi;
  int* status;       // error flag (bit 32) on a wait timeout
};

constexpr int kTileM = 128;
constexpr int kChunkK = 64;

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// rows r0.. of an R x 64 chunk (k from k0) into the K-major layout at dst; zero outside [0,R)x[k0,ke)
__device__ __forceinline__ void stage_chunk(unsigned char* dst, const float* src, long long s_row, long long s_k,
                                            int row0, int nrows_valid, int R, int k0, int ke) {
  for (int idx = threadIdx.x; idx < R * (kChunkK / 8); idx += blockDim.x) {
    const int r = idx % R, c = idx / R;   // consecutive threads: consecutive rows
    const int row = row0 + r;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float v2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + c * 8 + 2 * j + h;
        v2[h] = (r < nrows_valid && k < ke) ? src[static_cast<long long>(row) * s_row + static_cast<long long>(k) * s_k]
                                            : 0.0f;
      }
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(v2[0], v2[1]);
      w[j] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(r, c * 8, kChunkK)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t s_taddr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM;
  const int kb = blockIdx.y * g.k_per_split;
  const int ke = min(g.K, kb + g.k_per_split);
  if (kb >= ke) return;   // uniform over the CTA
  const int Npad = (g.N + 15) & ~15;
  const uint32_t ncols = Npad <= 32 ? 32u : (Npad <= 64 ? 64u : (Npad <= 128 ? 128u : 256u));
  unsigned char* sA = smem;
  unsigned char* sB = smem + kTileM * kChunkK * 2;
  if (warp == 0) tc::tmem_alloc(&s_taddr, ncols);
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = tc::idesc_bf16_f32(kTileM, Npad);
  uint32_t phase = 0;
  bool ok = true;
  bool first = true;
  for (int k0 = kb; k0 < ke; k0 += kChunkK) {
    stage_chunk(sA, g.A, g.sam, g.sak, m0, min(kTileM, g.M - m0), kTileM, k0, ke);
    stage_chunk(sB, g.B, g.sbn, g.sbk, 0, g.N, Npad, k0, ke);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kChunkK / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(sA) + kk * 256, 128, (kChunkK / 8) * 128);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + kk * 256, 128, (kChunkK / 8) * 128);
        tc::mma_bf16(taddr, ad, bd, idesc, !(first && kk == 0));
      }
      tc::mma_commit(&bar);
    }
    ok = ok && tc::mbar_wait(&bar, phase);
    phase ^= 1u;
    first = false;
    __syncthreads();
  }
  if (!__syncthreads_and(ok)) {
    // an MMA did not signal completion in time: record it, give it a second bounded chance to
    // finish, free the accumulator and leave without reading it
    if (threadIdx.x == 0) atomicOr(g.status, 32);
    tc::mbar_wait(&bar, phase ^ 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
    return;
  }
  tc::fence_after_sync();
  const int row = m0 + warp * 32 + lane;
  const uint32_t lane_addr = taddr + (static_cast<uint32_t>(warp * 32) << 16);
  for (int n0 = 0; n0 < Npad; n0 += 16) {
    float v[16];
    tc::tmem_ld16(lane_addr + n0, v);
    if (row < g.M) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + j;
        if (n < g.N) {
          float z = v[j];
          float* dst = g.C + static_cast<long long>(row) * g.ldc + n;
          if (g.epi == kEpiAtomic) {
            atomicAdd(dst, z);
          } else {
            if (g.epi != kEpiStore && g.bias) z += g.bias[n];
            *dst = z;
            if (g.epi == kEpiBiasGelu && g.C2) g.C2[static_cast<long long>(row) * g.ldc + n] = gelu_erf(z);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

size_t gemm_smem_bytes(int N) {
  const int Npad = (N + 15) & ~15;
  const size_t need = static_cast<size_t>(kTileM) * kChunkK * 2 + static_cast<size_t>(Npad) * kChunkK * 2;
  // at most 512 / ncols CTAs per SM, so that TMEM allocations of resident CTAs always fit
  const size_t ncols = Npad <= 32 ? 32 : (Npad <= 64 ? 64 : (Npad <= 128 ? 128 : 256));
  const size_t floor_bytes = ncols * 448;
  return need > floor_bytes ? need : floor_bytes;
}

int launch_gemm(const GemmArgs& g, int ksplit, cudaStream_t s) {
  if (g.M < 1 || g.N < 1 || g.N > 256 || g.K < 1 || ksplit < 1) return static_cast<int>(cudaErrorInvalidValue);
  GemmArgs a = g;
  a.k_per_split = (((g.K + ksplit - 1) / ksplit) + kChunkK - 1) / kChunkK * kChunkK;
  const int ysplit = (g.K + a.k_per_split - 1) / a.k_per_split;
  dim3 grid((g.M + kTileM - 1) / kTileM, ysplit);
  const size_t smem = gemm_smem_bytes(g.N);
  cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  gemm_tc_kernel<<<grid, 128, smem, s>>>(a);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace chem

using namespace chem;

extern "C" int chem_tc_gemm(const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbn, int64_t sbk,
                            float* C, int64_t ldc, const float* bias, float* C2, int32_t M, int32_t N, int32_t K,
                            int32_t epi, int32_t ksplit, int32_t* status, void* stream) {
  if (!A || !B || !C || !status || M < 1 || N < 1 || N > 256 || K < 1 || epi < 0 || epi > 3 || ksplit < 1 ||
      ldc < N || ((epi == kEpiBias || epi == kEpiBiasGelu) && !bias) || (epi != kEpiAtomic && ksplit != 1))
    return CHEM_EINVAL;
  GemmArgs g{};
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbn = sbn;
  g.sbk = sbk;
  g.C = C;
  g.ldc = ldc;
  g.C2 = C2;
  g.bias = bias;
  g.M = M;
  g.N = N;
  g.K = K;
  g.epi = epi;
  g.status = status;
  const int r = launch_gemm(g, ksplit, static_cast<cudaStream_t>(stream));
  if (r) {
    std::fprintf(stderr, "libchem: gemm launch: %s\n", cudaGetErrorString(static_cast<cudaError_t>(r)));
    return CHEM_ECUDA;
  }
  return CHEM_OK;
}
