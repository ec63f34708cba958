// explicit.cu -- the paper's own integration loop, kept as the comparison point of the implicit
// bulk-sparse path: the explicit first-order adaptive scheme of Sec. 2.1 (each substep as long as
// keeps every mass fraction within bulk_frac of its value, the "1-5%" rule, with |Y_k| floored at
// y_floor, and never past the end of the step) driven by Algorithm 3: a counting launch over all
// cells (section 1), bulk launches over all cells of at most K substeps per cell while the active
// count read back on the host exceeds N* (section 2), then one launch over the compacted active
// cells with at most k_max substeps each (section 3).  One thread per cell; FP64 state, time and
// temperature inversion after every substep; rates in FP32 (FP64 with CHEM_FLAG_FP64_RATES).
#include "chem_device.cuh"
#include "internal.h"

namespace chem {

// mode kExInit: section 1 (time 0 or dt, T from e, count and list the active cells);
// mode kExBulk: every cell still short of dt takes up to max_sub substeps, survivors are listed;
// mode kExSparse: the listed cells take up to max_sub substeps, survivors fail.
// x[(ns + 2) n] carries each active cell's time, temperature and mass fractions in FP64 between
// launches (SoA: t, T, Y_0 .. Y_{ns-1}), so that a cell's sequence of substeps does not depend on
// how the launches split it; the FP32 arrays receive the state when a cell finishes or fails.
// The active list is a.queue / a.ws->qcount.
template <int NS>
__global__ void __launch_bounds__(kBulkBlock) explicit_kernel(const AdvanceArgs<float> a, double* x, int mode,
                                                               int max_sub) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, a.blob, a.blob_bytes, &bar, &a.ws->status)) return;
  const MechView m = make_view(smem);
  const long long cnt = mode == kExSparse ? static_cast<long long>(a.ws->qcount) : a.n;
  const long long n = a.n;
  const double dt = a.dt;
  const bool fp64 = (a.prm.flags & 1) != 0;   // CHEM_FLAG_FP64_RATES
  unsigned long long c_sub = 0, c_skip = 0, c_inv = 0, c_fail = 0, c_done = 0;
  int flags = 0;
  const int lane = threadIdx.x & 31;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < cnt;
       base += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long q = base + lane;
    bool active = false;
    long long i = -1;
    if (q < cnt) {
      i = mode == kExSparse ? a.queue[q] : q;
      if (mode == kExInit) {
        const float rho = a.rho[i], e = a.e[i], T = a.T[i];
        bool valid = isfinite(rho) && rho > 0.0f && isfinite(e) && isfinite(T) && T > 0.0f;
        double y[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const float yk = a.Y[k * a.ld + i];
          valid = valid && isfinite(yk) && yk > -1e-6f;
          y[k] = yk;
        }
        if (!valid) {
          a.substeps[i] = -1;
          ++c_inv;
        } else if (T < a.prm.T_min) {
          a.substeps[i] = 0;
          ++c_skip;
        } else {
          bool ok;
          const double T0 = temperature_from_energy<NS>(m, y, static_cast<double>(e), static_cast<double>(T), &ok);
          a.substeps[i] = ok ? 0 : -1;
          active = ok;
          if (ok) {
            x[n + i] = T0;
#pragma unroll
            for (int k = 0; k < NS; ++k) x[(2 + k) * n + i] = y[k];
          } else {
            ++c_fail;
            flags |= kFlagTemp;
          }
        }
        x[i] = active ? 0.0 : dt;
      } else if (x[i] < dt) {
        double t = x[i], T = x[n + i];
        const float rho = a.rho[i];
        const double e = a.e[i];
        double y[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) y[k] = x[(2 + k) * n + i];
        bool ok = true;
        int s = 0;
#pragma unroll 1
        for (; s < max_sub && ok && t < dt; ++s) {
          double f[NS], y1[NS];
          if (fp64) {
            rates<NS, double>(m, static_cast<double>(rho), T, y, f);
          } else {   // FP32 rates (FP64 where the FP32 log-rates overflow)
            float ff[NS];
            rates_safe<NS>(m, rho, T, y, ff);
#pragma unroll
            for (int k = 0; k < NS; ++k) f[k] = ff[k];
          }
          // the longest substep that changes no Y_k by more than bulk_frac of max(|Y_k|, y_floor)
          const double rem = dt - t;
          double h = rem;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const double af = fabs(f[k]);
            if (af > 0.0) h = fmin(h, static_cast<double>(a.prm.bulk_frac) * fmax(fabs(y[k]), static_cast<double>(a.prm.y_floor)) / af);
          }
#pragma unroll
          for (int k = 0; k < NS; ++k) y1[k] = fma(h, f[k], y[k]);
          bool okT;
          const double T1 = temperature_from_energy<NS>(m, y1, e, T, &okT);
          ok = okT;
          if (ok) {
#pragma unroll
            for (int k = 0; k < NS; ++k) y[k] = y1[k];
            T = T1;
            t = h >= rem ? dt : t + h;
          }
        }
        c_sub += s;
        active = ok && t < dt;
        const bool fail = !ok || (active && mode == kExSparse);   // T(e) lost, or k_max reached
        if (fail) {
          flags |= ok ? kFlagMaxSteps : kFlagTemp;
          a.substeps[i] = -1;
          t = dt;
          active = false;
          ++c_fail;
        } else {
          a.substeps[i] += s;
          if (!active && mode == kExBulk) ++c_done;
        }
        x[i] = t;
        if (active) {
          x[n + i] = T;
#pragma unroll
          for (int k = 0; k < NS; ++k) x[(2 + k) * n + i] = y[k];
        } else {   // finished or failed: the state reached goes to the FP32 arrays
          double sw = 0.0;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            a.Y[k * a.ld + i] = static_cast<float>(y[k]);
            sw = fma(y[k], static_cast<double>(m.invW[k]), sw);
          }
          a.T[i] = static_cast<float>(T);
          if (a.p) a.p[i] = static_cast<float>(static_cast<double>(rho) * kR * T * sw);
        }
      }
    }
    // compaction of the cells still active, one atomic per warp (section 3's index list)
    if (mode != kExSparse) {
      const unsigned mask = __ballot_sync(0xffffffffu, active);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        int off = 0;
        if (lane == leader) off = atomicAdd(&a.ws->qcount, __popc(mask));
        off = __shfl_sync(0xffffffffu, off, leader);
        if (active) a.queue[off + __popc(mask & ((1u << lane) - 1u))] = static_cast<int>(i);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_sub += __shfl_down_sync(0xffffffffu, c_sub, o);
    c_skip += __shfl_down_sync(0xffffffffu, c_skip, o);
    c_inv += __shfl_down_sync(0xffffffffu, c_inv, o);
    c_fail += __shfl_down_sync(0xffffffffu, c_fail, o);
    c_done += __shfl_down_sync(0xffffffffu, c_done, o);
    flags |= __shfl_down_sync(0xffffffffu, flags, o);
  }
  if (lane == 0) {
    if (c_sub) {
      atomicAdd(&a.ws->substeps, c_sub);
      atomicAdd(&a.ws->attempts, c_sub);
    }
    if (c_skip) atomicAdd(&a.ws->nskipped, c_skip);
    if (c_done) atomicAdd(&a.ws->nbulk, c_done);
    if (c_inv) {
      atomicAdd(&a.ws->ninvalid, c_inv);
      atomicOr(&a.ws->status, kFlagInvalid);
    }
    if (c_fail) atomicAdd(&a.ws->nfailed, c_fail);
    if (flags) atomicOr(&a.ws->status, flags);
  }
}

int launch_explicit(int ns, const AdvanceArgs<float>& a, double* x, int mode, int max_sub, int grid,
                    cudaStream_t s) {
  if (ns != 9) return -1;
  const size_t smem = (a.blob_bytes + 127u) & ~127u;
  cudaError_t e = cudaFuncSetAttribute(explicit_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  explicit_kernel<9><<<grid, kBulkBlock, smem, s>>>(a, x, mode, max_sub);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace chem
