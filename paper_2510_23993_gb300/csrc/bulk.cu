// bulk.cu -- the bulk phase of the bulk-sparse integration (Algorithm 3, sections 1 and 2,
// plus the compaction of section 3) and small per-cell utility kernels.
//
// One persistent grid-stride pass over all cells.  Per cell: coalesced SoA loads of rho, e,
// T, Y; input validation; the activity test T >= T_min (Algorithm 2/3); the FP64 temperature
// inversion; k_bulk explicit Heun steps of dt/k_bulk with FP32 matrix-form rates, an embedded
// error test and the relative-change rule of Sec. 2.1; accepted cells are written back,
// failed cells are compacted into the stiff queue with one warp ballot and one atomic per warp
// (replacing the host round trip of the counter in Algorithm 3).
#include "chem_device.cuh"
#include "internal.h"

namespace chem {

template <typename S>
__device__ __forceinline__ bool finite_(S x) { return isfinite(x); }

template <int NS, typename S>
__global__ void __launch_bounds__(kBulkBlock) bulk_kernel(const AdvanceArgs<S> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, a.blob, a.blob_bytes, &bar, &a.ws->status)) return;
  const MechView m = make_view(smem);
  int* soff = reinterpret_cast<int*>(smem + ((a.blob_bytes + 127u) & ~127u));
  if (a.nbox > 0) stage_box_offsets(soff, a.box_off, a.nbox);
  const int lane = threadIdx.x & 31;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  unsigned long long c_skip = 0, c_bulk = 0, c_inv = 0;
  const int kb = a.prm.k_bulk;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < a.n;
       base += stride) {
    const long long g = base + lane;
    bool enqueue = false;
    int bucket = 0;
    if (g < a.n && !(a.skip && a.skip[g])) {
      const CellRef<S> cr = locate(a, soff, g);
      const long long i = cr.i;
      const double dt = cr.dt;
      const float h = static_cast<float>(dt / kb);
      const S rho = cr.rho[i], e = cr.e[i], T = cr.T[i];
      S y[NS];
      bool valid = finite_(rho) && rho > S(0) && finite_(e) && finite_(T) && T > S(0);
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        y[k] = cr.Y[k * cr.ld + i];
        valid = valid && finite_(y[k]) && y[k] > S(-1e-6);
      }
      if (!valid) {
        cr.sub[i] = -1;
        ++c_inv;
      } else if (T < static_cast<S>(a.prm.T_min)) {
        cr.sub[i] = 0;
        ++c_skip;
      } else {
        bool pass;
        float cost = 0.0f;   // dt * sum_k |dY_k/dt| at the first bulk substep (queue ordering key)
        double Tn = temperature_from_energy<NS>(m, y, static_cast<double>(e), static_cast<double>(T), &pass);
        const float rhof = static_cast<float>(rho);
        for (int s = 0; s < kb && pass; ++s) {
          float yf[NS], f0[NS], f1[NS];
#pragma unroll
          for (int k = 0; k < NS; ++k) yf[k] = static_cast<float>(y[k]);
          pass = rates<NS, float>(m, rhof, static_cast<float>(Tn), yf, f0);
          if (s == 0) {
#pragma unroll
            for (int k = 0; k < NS; ++k) cost += fabsf(f0[k]);
            cost *= static_cast<float>(dt);
          }
          S y1[NS];
          float chg = 0.0f;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const float d = h * f0[k];
            y1[k] = y[k] + static_cast<S>(d);
            yf[k] = static_cast<float>(y1[k]);
            chg = fmaxf(chg, fabsf(d) / fmaxf(fabsf(static_cast<float>(y[k])), a.prm.y_floor));
          }
          bool ok1;
          const double T1 = temperature_from_energy<NS>(m, y1, static_cast<double>(e), Tn, &ok1);
          pass = pass && ok1 && rates<NS, float>(m, rhof, static_cast<float>(T1), yf, f1);
          float err = 0.0f;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const S yh = y[k] + static_cast<S>(0.5f * h * (f0[k] + f1[k]));
            const float est = 0.5f * h * fabsf(f1[k] - f0[k]);
            const float w = a.prm.atol + a.prm.rtol * fmaxf(fabsf(static_cast<float>(y[k])), fabsf(static_cast<float>(yh)));
            err = fmaxf(err, est / w);
            y[k] = yh;
          }
          pass = pass && (err <= 1.0f) && (chg <= a.prm.bulk_frac);
          if (pass) {
            bool okT;
            Tn = temperature_from_energy<NS>(m, y, static_cast<double>(e), T1, &okT);
            pass = okT;
          }
        }
        if (pass) {
          double sw = 0.0;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            cr.Y[k * cr.ld + i] = y[k];
            sw = fma(static_cast<double>(y[k]), static_cast<double>(m.invW[k]), sw);
          }
          cr.T[i] = static_cast<S>(Tn);
          if (cr.p) cr.p[i] = static_cast<S>(static_cast<double>(rho) * kR * Tn * sw);
          cr.sub[i] = kb;
          ++c_bulk;
        } else {
          enqueue = true;
          if (a.qkey) {
            float lk;
            if (a.prm.flags & kFlagOrderPrev) {   // substep count of the previous call on this cell
              const int prev = cr.sub[i];
              lk = 4.0f * __log2f(static_cast<float>(prev > 0 ? (prev < (1 << 24) ? prev : (1 << 24)) : 1));
            } else {                               // explicit rate magnitude over dt
              lk = 2.0f * __log2f(fmaxf(cost, 1e-30f)) + 32.0f;
            }
            bucket = static_cast<int>(fminf(fmaxf(lk, 0.0f), static_cast<float>(kNumBuckets - 1)));
          }
        }
      }
    }
    // warp-level compaction of the failed cells (Algorithm 3, section 3, with one atomic per warp)
    const unsigned mask = __ballot_sync(0xffffffffu, enqueue);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      int off = 0;
      if (lane == leader) off = atomicAdd(&a.ws->qcount, __popc(mask));
      off = __shfl_sync(0xffffffffu, off, leader);
      if (enqueue) {
        const int slot = off + __popc(mask & ((1u << lane) - 1u));
        a.queue[slot] = static_cast<int>(g);
        if (a.qkey) a.qkey[slot] = static_cast<unsigned char>(bucket);
      }
    }
  }
  // counters: warp reduction, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_skip += __shfl_down_sync(0xffffffffu, c_skip, o);
    c_bulk += __shfl_down_sync(0xffffffffu, c_bulk, o);
    c_inv += __shfl_down_sync(0xffffffffu, c_inv, o);
  }
  if (lane == 0) {
    if (c_skip) atomicAdd(&a.ws->nskipped, c_skip);
    if (c_bulk) atomicAdd(&a.ws->nbulk, c_bulk);
    if (c_inv) {
      atomicAdd(&a.ws->ninvalid, c_inv);
      atomicOr(&a.ws->status, kFlagInvalid);
    }
  }
}

// Counting sort of the stiff queue by cost bucket, most expensive bucket first (one block): a
// longest-first order shortens the tail of the persistent stiff kernel, whose duration is set
// by the cells that start last.
__global__ void __launch_bounds__(1024) order_queue_kernel(Workspace* ws, const int* queue, const unsigned char* qkey,
                                                           int* queue_out, long long n, bool continuations) {
  __shared__ int hist[kNumBuckets];
  __shared__ int off[kNumBuckets];
  const int* count = continuations ? &ws->cont_count : &ws->qcount;
  const int qn = static_cast<int>(min(static_cast<long long>(*reinterpret_cast<volatile const int*>(count)), n));
  for (int b = threadIdx.x; b < kNumBuckets; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < qn; i += blockDim.x) atomicAdd(&hist[qkey[i] & (kNumBuckets - 1)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = kNumBuckets - 1; b >= 0; --b) {
      off[b] = acc;
      acc += hist[b];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < qn; i += blockDim.x) {
    const int pos = atomicAdd(&off[qkey[i] & (kNumBuckets - 1)], 1);
    queue_out[pos] = queue[i];
  }
}

int launch_order_queue(Workspace* ws, const int* queue, const unsigned char* qkey, int* queue_out, long long n,
                       cudaStream_t s, bool continuations) {
  order_queue_kernel<<<1, 1024, 0, s>>>(ws, queue, qkey, queue_out, n, continuations);
  return static_cast<int>(cudaGetLastError());
}

// The thermo view of a blob whose first `bytes` are staged in shared memory: the large layout
// keeps its FP64 thermo coefficients in the global tail, read from there through L1.
__device__ __forceinline__ MechView thermo_view(const unsigned char* smem, const unsigned char* blob, unsigned bytes) {
  MechView m = make_view(smem);
  const MechHdr* h = reinterpret_cast<const MechHdr*>(smem);
  if (static_cast<unsigned>(h->off_e64) >= bytes) m.e64 = reinterpret_cast<const double*>(blob + h->off_e64);
  return m;
}

// rho = p / (R T sum Y/W), e = R * e/R(T) (FP64)
template <int NS, typename S>
__global__ void __launch_bounds__(kBulkBlock) state_kernel(const unsigned char* blob, unsigned bytes, const S* T,
                                                           const S* p, const S* Y, long long ld, long long n,
                                                           S* rho, S* e, int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, blob, bytes, &bar, status)) return;
  const MechView m = thermo_view(smem, blob, bytes);
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double t = static_cast<double>(T[i]);
    double y[NS], sw = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      y[k] = static_cast<double>(Y[k * ld + i]);
      sw = fma(y[k], static_cast<double>(m.e64[(1 * NS + k) * 8 + 6]), sw);   // 1/W
    }
    double E[6];
    mixture64<NS>(m, regime_of(static_cast<float>(t), m.T_lo, m.T_hi), y, E);
    const double eR = fma(t, fma(t, fma(t, fma(t, fma(t, E[5], E[4]), E[3]), E[2]), E[1]), E[0]);
    rho[i] = static_cast<S>(static_cast<double>(p[i]) / (kR * t * sw));
    e[i] = static_cast<S>(kR * eR);
  }
}

template <int NS>
__global__ void __launch_bounds__(kBulkBlock) temperature_kernel(const unsigned char* blob, unsigned bytes, const float* Y,
                                                                 long long ld, const float* e, long long n, float* T,
                                                                 int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, blob, bytes, &bar, status)) return;
  const MechView m = thermo_view(smem, blob, bytes);
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    float y[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) y[k] = Y[k * ld + i];
    bool ok;
    const double t = temperature_from_energy<NS>(m, y, static_cast<double>(e[i]), static_cast<double>(T[i]), &ok);
    if (!ok) atomicOr(status, kFlagTemp);
    T[i] = static_cast<float>(t);
  }
}

template <int NS>
__global__ void __launch_bounds__(kBulkBlock) rates_kernel(const unsigned char* blob, unsigned bytes, const float* rho,
                                                           const float* T, const float* Y, long long ld, long long n,
                                                           float* dYdt, int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, blob, bytes, &bar, status)) return;
  const MechView m = make_view(smem);
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    double y[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) y[k] = static_cast<double>(Y[k * ld + i]);
    float f[NS];
    rates_safe<NS>(m, rho[i], static_cast<double>(T[i]), y, f);
#pragma unroll
    for (int k = 0; k < NS; ++k) dYdt[k * ld + i] = f[k];
  }
}

// ------------------------------------------------------------------ launchers

#define CHEM_FOR_EACH_NS(X) X(9)
// species counts of the thread-per-cell thermo helpers (state_kernel, temperature_kernel): also
// the large mechanisms, whose blobs carry the same thermo layout (their FP64 coefficients in the
// global tail)
#define CHEM_FOR_EACH_NS_THERMO(X) X(9) X(53)

size_t bulk_smem_bytes(unsigned blob_bytes, int nbox) {
  return ((blob_bytes + 127u) & ~127u) + box_smem_bytes(nbox);
}

static int grid_for(long long n) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + kBulkBlock - 1) / kBulkBlock;
  long long cap = static_cast<long long>(sms) * 8;
  if (blocks > cap) blocks = cap;
  return static_cast<int>(blocks < 1 ? 1 : blocks);
}

template <int NS, typename S>
static int bulk_launch_t(const AdvanceArgs<S>& a, int grid, cudaStream_t s) {
  auto k = bulk_kernel<NS, S>;
  const size_t smem = bulk_smem_bytes(a.blob_bytes, a.nbox);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  k<<<grid, kBulkBlock, smem, s>>>(a);
  return static_cast<int>(cudaGetLastError());
}

int launch_bulk_f32(int ns, const AdvanceArgs<float>& a, int grid, cudaStream_t s) {
#define X(N) \
  if (ns == N) return bulk_launch_t<N, float>(a, grid, s);
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int launch_bulk_f64(int ns, const AdvanceArgs<double>& a, int grid, cudaStream_t s) {
#define X(N) \
  if (ns == N) return bulk_launch_t<N, double>(a, grid, s);
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int bulk_occupancy(int ns, bool f64, unsigned blob_bytes, int* blocks_per_sm) {
#define X(N)                                                                                          \
  if (ns == N) {                                                                                      \
    if (f64)                                                                                          \
      return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(                         \
          blocks_per_sm, bulk_kernel<N, double>, kBulkBlock, blob_bytes));                            \
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(                           \
        blocks_per_sm, bulk_kernel<N, float>, kBulkBlock, blob_bytes));                               \
  }
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int launch_state_from_TpY_f32(int ns, const unsigned char* blob, unsigned bytes, const float* T, const float* p,
                              const float* Y, long long ld, long long n, float* rho, float* e, int* status,
                              cudaStream_t s) {
#define X(N)                                                                                           \
  if (ns == N) {                                                                                       \
    cudaFuncSetAttribute(state_kernel<N, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);  \
    state_kernel<N, float><<<grid_for(n), kBulkBlock, bytes, s>>>(blob, bytes, T, p, Y, ld, n, rho, e, \
                                                                  status);                             \
    return static_cast<int>(cudaGetLastError());                                                       \
  }
  CHEM_FOR_EACH_NS_THERMO(X)
#undef X
  return -1;
}

int launch_state_from_TpY_f64(int ns, const unsigned char* blob, unsigned bytes, const double* T, const double* p,
                              const double* Y, long long ld, long long n, double* rho, double* e, int* status,
                              cudaStream_t s) {
#define X(N)                                                                                            \
  if (ns == N) {                                                                                        \
    cudaFuncSetAttribute(state_kernel<N, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);  \
    state_kernel<N, double><<<grid_for(n), kBulkBlock, bytes, s>>>(blob, bytes, T, p, Y, ld, n, rho, e, \
                                                                   status);                             \
    return static_cast<int>(cudaGetLastError());                                                        \
  }
  CHEM_FOR_EACH_NS_THERMO(X)
#undef X
  return -1;
}

int launch_temperature(int ns, const unsigned char* blob, unsigned bytes, const float* Y, long long ld,
                       const float* e, long long n, float* T, int* status, cudaStream_t s) {
#define X(N)                                                                                       \
  if (ns == N) {                                                                                   \
    cudaFuncSetAttribute(temperature_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);  \
    temperature_kernel<N><<<grid_for(n), kBulkBlock, bytes, s>>>(blob, bytes, Y, ld, e, n, T, status); \
    return static_cast<int>(cudaGetLastError());                                                   \
  }
  CHEM_FOR_EACH_NS_THERMO(X)
#undef X
  return -1;
}

int launch_rates(int ns, const unsigned char* blob, unsigned bytes, const float* rho, const float* T,
                 const float* Y, long long ld, long long n, float* dYdt, int* status, cudaStream_t s) {
#define X(N)                                                                                                \
  if (ns == N) {                                                                                            \
    rates_kernel<N><<<grid_for(n), kBulkBlock, bytes, s>>>(blob, bytes, rho, T, Y, ld, n, dYdt, status);    \
    return static_cast<int>(cudaGetLastError());                                                            \
  }
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

}  // namespace chem
