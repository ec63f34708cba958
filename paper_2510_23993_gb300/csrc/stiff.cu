// stiff.cu -- the stiff kernel of the dense table layout (its body is stiff_body.cuh): the packed
// mechanism tables are staged into shared memory once per CTA and read by the table-driven
// kinetics and thermodynamics of chem_device.cuh.
#include "chem_device.cuh"
#include "internal.h"
#include "stiff_body.cuh"

namespace chem {

// Mechanism policy over the staged tables (MechView).
template <int NS_>
struct TableMech {
  static constexpr int NS = NS_;
  static constexpr int NJ = NS_;
  MechView v;
  __device__ __forceinline__ int na() const { return v.nact; }
  __device__ __forceinline__ double temperature(const double* y, double e0, double T, bool* ok, double* cv,
                                                double tol) const {
    return temperature_from_energy<NS>(v, y, e0, T, ok, cv, tol);
  }
  __device__ __forceinline__ void jacobian(float rho, float T, const float* Y, float cvR, float (&J)[NJ][NJ]) const {
    chem::jacobian<NS>(v, rho, T, Y, cvR, J);
  }
  __device__ __forceinline__ bool rates(float rho, float T, const float* Y, float* f) const {
    return chem::rates<NS, float>(v, rho, T, Y, f);
  }
  __device__ __forceinline__ void rates64(float rho, double T, const double* y, float* f) const {
    rates_fp64_fallback<NS>(v, rho, T, y, f);
  }
  __device__ __forceinline__ double invW64(int k) const { return v.e64[(1 * NS + k) * 8 + 6]; }
};

// One instantiation per CTA size the tuner may pick (64, 128, 256 threads): the per-thread matrix
// stride is a compile-time constant in each, which keeps the shared-memory addressing in immediates.
template <int NS, typename S, int BLK>
__global__ void __launch_bounds__(BLK) stiff_kernel(const AdvanceArgs<S> a, unsigned blob_pad) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, a.blob, a.blob_bytes, &bar, &a.ws->status)) return;
  TableMech<NS> m;
  m.v = make_view(smem);
  stiff_body<TableMech<NS>, S, BLK>(a, m, smem, blob_pad);
}

// ------------------------------------------------------------------ launchers

#define CHEM_FOR_EACH_NS(X) X(9)

static unsigned pad128(unsigned b) { return (b + 127u) & ~127u; }

size_t stiff_smem_bytes(int ns, unsigned blob_bytes, int nbox, int block) {
  return pad128(blob_bytes) + box_smem_bytes(nbox) + stiff_matrix_bytes(ns, block);
}

// Launch a stiff kernel (function symbol or cudaKernel_t) with its argument list.  The
// continuation pass waits on grid barriers, so it is a cooperative launch whose grid is capped at
// the CTAs that fit at once for this kernel and shared-memory size (box offsets included).
static int launch_stiff_fn(const void* fn, void** args, size_t smem, int grid, int block, bool coop, cudaStream_t s) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  if (coop) {
    int bps = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, block, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long fit = static_cast<long long>(bps > 0 ? bps : 1) * (sms > 0 ? sms : 1);
    if (grid > fit) grid = static_cast<int>(fit);
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  return static_cast<int>(cudaLaunchKernelExC(&cfg, fn, args));
}

template <int NS, typename S>
static const void* stiff_fn(int block) {
  switch (block) {
    case 64: return reinterpret_cast<const void*>(stiff_kernel<NS, S, 64>);
    case 128: return reinterpret_cast<const void*>(stiff_kernel<NS, S, 128>);
    case 256: return reinterpret_cast<const void*>(stiff_kernel<NS, S, 256>);
    default: return nullptr;
  }
}

template <int NS, typename S>
static int stiff_launch_t(const AdvanceArgs<S>& a, int grid, int block, cudaStream_t s) {
  const void* fn = stiff_fn<NS, S>(block);
  if (!fn) return static_cast<int>(cudaErrorInvalidValue);
  const size_t smem = stiff_smem_bytes(NS, a.blob_bytes, a.nbox, block);
  AdvanceArgs<S> arg = a;
  unsigned pad = pad128(a.blob_bytes);
  void* args[] = {&arg, &pad};
  return launch_stiff_fn(fn, args, smem, grid, block, a.pass == 2, s);
}

int launch_stiff_f32(int ns, const AdvanceArgs<float>& a, int grid, int block, cudaStream_t s) {
#define X(N) \
  if (ns == N) return stiff_launch_t<N, float>(a, grid, block, s);
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int launch_stiff_f64(int ns, const AdvanceArgs<double>& a, int grid, int block, cudaStream_t s) {
#define X(N) \
  if (ns == N) return stiff_launch_t<N, double>(a, grid, block, s);
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int stiff_occupancy(int ns, unsigned blob_bytes, int block, int* blocks_per_sm) {
#define X(N)                                                                                     \
  if (ns == N) {                                                                                 \
    const void* fn = stiff_fn<N, float>(block);                                                  \
    if (!fn) return static_cast<int>(cudaErrorInvalidValue);                                     \
    const size_t smem = stiff_smem_bytes(N, blob_bytes, 0, block);                               \
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)); \
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem)); \
  }
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

}  // namespace chem
