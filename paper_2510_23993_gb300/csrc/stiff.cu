// stiff.cu -- the sparse phase of the bulk-sparse integration (Algorithm 3, section 3) with an
// implicit integrator: every cell the bulk kernel compacted into the queue is integrated from
// its original state over [0, dt] by an L-stable, stiffly accurate 3-stage SDIRK method of
// order 3 (Alexander's DIRK3) with an embedded 2nd-order solution for error control.  Each
// stage solves Y_i = y_n + h sum_{j<i} a_ij k_j + gamma h f(Y_i) by simplified Newton with the
// dense iteration matrix I - gamma h J: J analytic in FP32, its LU factorisation with partial
// pivoting and the triangular solves in FP64 (shared memory), the state in FP64, the
// temperature from the internal energy by the FP64 inversion.  The error estimate is filtered
// through (I - gamma h J)^-1 so that stiff components do not inflate it.
//
// The kernel is persistent (grid = SMs x resident blocks).  Each lane owns one cell at a time
// and pulls the next one from the device queue as soon as its cell finishes (warp-aggregated
// atomic on the queue head), so lanes of a warp stay busy on different cells while executing
// the same substep code; this removes the warp-divergence and idle-thread costs that the paper
// attributes to Algorithm 2, without any host round trip.
#include "chem_device.cuh"
#include "internal.h"

namespace chem {

constexpr int kNewtMax = 6;
constexpr double kNewtTol = 0.03;   // predicted remaining Newton error below 3% of the error weight

// Alexander's L-stable DIRK3: c = (g, (1+g)/2, 1), A = [[g,0,0],[(1-g)/2,g,0],[b1,b2,g]], b = last
// row; g is the root of the order-3 condition sum b c^2 = 1/3 in (1/3, 1/2).  Embedded order-2
// weights bh = (1 - bh2, bh2, 0) satisfy sum bh = 1, sum bh c = 1/2.
constexpr double kG = 0.43586652150845895;
constexpr double kA21 = 0.5 * (1.0 - kG);
constexpr double kB1 = 1.2084966491760099;
constexpr double kB2 = -0.6443631706844688;
constexpr double kBh1 = 0.7726301276675509;
constexpr double kBh2 = 0.2273698723324491;
constexpr double kC2 = 0.5 * (1.0 + kG);

// Per-thread FP64 iteration matrix and one FP64 vector in shared memory: element (r, c) of
// thread t at M[(r * NS + c) * B + t], vector element k at V[k * B + t], so consecutive threads
// hit consecutive banks.  The factorisation and the solves index them dynamically in rolled
// loops: the FP64 pipe, not the instruction count, bounds these loops, and the rolled code keeps
// the kernel's instruction footprint small enough for the instruction caches.
template <int NS>
struct Smem {
  double* M;
  double* V;
  int t, B;
  __device__ double& mm(int r, int c) const { return M[(r * NS + c) * B + t]; }
  __device__ double& vv(int k) const { return V[k * B + t]; }
};

// M = I - hh * J from the FP32 Jacobian in registers (FP64 in shared memory).  The product
// hh * J is formed in FP32: J carries FP32 rounding already, so the FP64 product would add no
// accuracy, and it saves NS^2 FP64 multiplies per attempt; the identity is added in FP64.
template <int NS>
__device__ __forceinline__ void store_iteration_matrix(const Smem<NS>& s, const float (&J)[NS][NS], double hh) {
  const float mh = static_cast<float>(-hh);
#pragma unroll
  for (int r = 0; r < NS; ++r)
#pragma unroll
    for (int c = 0; c < NS; ++c) {
      const double v = static_cast<double>(mh * J[r][c]);
      s.mm(r, c) = r == c ? 1.0 + v : v;
    }
}

// LU with partial pivoting in place (unit-lower L below the diagonal, U above, reciprocal of
// U's diagonal on it); pivot rows packed 4 bits each into *piv.
template <int NS>
__device__ __forceinline__ bool lu_factor(const Smem<NS>& s, uint64_t* piv) {
  uint64_t pv = 0;
#pragma unroll 1
  for (int k = 0; k < NS; ++k) {
    int p = k;
    double best = fabs(s.mm(k, k));
#pragma unroll 1
    for (int i = k + 1; i < NS; ++i) {
      const double v = fabs(s.mm(i, k));
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (!(best > 0.0)) return false;
    pv |= static_cast<uint64_t>(p) << (4 * k);
    if (p != k) {
#pragma unroll 1
      for (int c = 0; c < NS; ++c) {
        const double t = s.mm(k, c);
        s.mm(k, c) = s.mm(p, c);
        s.mm(p, c) = t;
      }
    }
    const double inv = 1.0 / s.mm(k, k);
    s.mm(k, k) = inv;
#pragma unroll 1
    for (int i = k + 1; i < NS; ++i) {
      const double l = s.mm(i, k) * inv;
      s.mm(i, k) = l;
#pragma unroll 2
      for (int c = k + 1; c < NS; ++c) s.mm(i, c) = fma(-l, s.mm(k, c), s.mm(i, c));
    }
  }
  *piv = pv;
  return true;
}

// Solve M x = b with the factors of lu_factor (b in registers, in and out; the permutation and
// the substitutions run on the shared-memory vector).
template <int NS>
__device__ __forceinline__ void lu_solve(const Smem<NS>& s, uint64_t piv, double (&b)[NS]) {
#pragma unroll
  for (int k = 0; k < NS; ++k) s.vv(k) = b[k];
#pragma unroll 1
  for (int k = 0; k < NS; ++k) {
    const int p = static_cast<int>((piv >> (4 * k)) & 15u);
    if (p != k) {
      const double t = s.vv(k);
      s.vv(k) = s.vv(p);
      s.vv(p) = t;
    }
  }
#pragma unroll 1
  for (int i = 1; i < NS; ++i) {
    double acc = s.vv(i);
#pragma unroll 1
    for (int j = 0; j < i; ++j) acc = fma(-s.mm(i, j), s.vv(j), acc);
    s.vv(i) = acc;
  }
#pragma unroll 1
  for (int i = NS - 1; i >= 0; --i) {
    double acc = s.vv(i);
#pragma unroll 1
    for (int j = i + 1; j < NS; ++j) acc = fma(-s.mm(i, j), s.vv(j), acc);
    s.vv(i) = acc * s.mm(i, i);
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) b[k] = s.vv(k);
}

struct CellCtx {
  float rho, rtol, atol;
  double e0;
  bool fp64_rates;
};

// Solve the stage equation z = yb + hh f(z) by simplified Newton (iteration matrix factored in
// shared memory) from the initial guess in z.  Tz: temperature guess in, temperature of the
// last evaluated iterate out.  Convergence is judged on the weighted RMS norm of the update and
// the contraction rate theta of the iteration: the iterate is accepted when the remaining error
// predicted from theta, eta * |dz| with eta = theta / (1 - theta), is below kNewtTol.  eta
// carries over between the stages of a step (first iteration of a stage uses the last value).
template <int NS>
__device__ __forceinline__ bool stage_newton(const MechView& m, const Smem<NS>& s, uint64_t piv, const CellCtx& c,
                                             const double (&yb)[NS], double hh, double (&z)[NS], double& Tz,
                                             double& eta, unsigned long long& n_it) {
  double prev = 0.0;
#pragma unroll 1
  for (int it = 0; it < kNewtMax; ++it) {
    ++n_it;
    bool ok;
    Tz = temperature_from_energy<NS>(m, z, c.e0, Tz, &ok);
    if (!ok) return false;
    float F[NS], Zf[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) Zf[k] = static_cast<float>(z[k]);
    bool use64 = c.fp64_rates;
    // FP32 rates; the FP64 instance (one copy in the code) when they overflow
    if (!use64) use64 = !rates<NS, float>(m, c.rho, static_cast<float>(Tz), Zf, F);
    if (use64) rates_fp64_fallback<NS>(m, c.rho, Tz, z, F);
    const float mhh = static_cast<float>(hh);
    double b[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) b[k] = (yb[k] - z[k]) + static_cast<double>(mhh * F[k]);
    lu_solve<NS>(s, piv, b);
    float ss = 0.0f;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      z[k] += b[k];
      const float bf = static_cast<float>(b[k]);
      const float w = c.atol + c.rtol * fabsf(Zf[k] + bf);
      const float r = bf / w;
      ss = fmaf(r, r, ss);
    }
    const double nrm = sqrt(static_cast<double>(ss) * (1.0 / NS));
    if (!(nrm == nrm)) return false;
    if (it > 0) {
      const double theta = nrm / prev;
      if (theta >= 1.0) {
        // not contracting: accept only at the FP32 noise floor (below half the error weight)
        if (nrm <= 0.5 && theta < 2.0) return true;
        return false;
      }
      eta = theta / (1.0 - theta);
    }
    if (eta * nrm <= kNewtTol || nrm <= 1e-3) return true;
    prev = nrm;
  }
  return false;
}

template <int NS, typename S>
__global__ void __launch_bounds__(kStiffBlock) stiff_kernel(const AdvanceArgs<S> a, unsigned blob_pad) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, a.blob, a.blob_bytes, &bar, &a.ws->status)) return;
  const MechView m = make_view(smem);
  int* soff = reinterpret_cast<int*>(smem + blob_pad);
  if (a.nbox > 0) stage_box_offsets(soff, a.box_off, a.nbox);
  Smem<NS> sm;
  sm.t = threadIdx.x;
  sm.B = kStiffBlock;
  sm.M = reinterpret_cast<double*>(smem + blob_pad + box_smem_bytes(a.nbox));
  sm.V = sm.M + NS * NS * kStiffBlock;

  const int lane = threadIdx.x & 31;
  // probe and single passes take cells from the stiff queue; the continuation pass takes the
  // queue slots the probe pass left unfinished, in their sorted order
  const int pass = a.pass;
  const int qn = pass == 2 ? min(*reinterpret_cast<volatile int*>(&a.ws->cont_count), static_cast<int>(a.n))
                           : min(*reinterpret_cast<volatile int*>(&a.ws->qcount), static_cast<int>(a.n));
  int* head = pass == 2 ? &a.ws->head2 : &a.ws->head;
  const long long cc = a.cont_cap;
  double* const cst = a.cont;   // continuation state, SoA by queue slot
  CellCtx c;
  c.rtol = a.prm.rtol;
  c.atol = a.prm.atol;
  c.fp64_rates = (a.prm.flags & 1) != 0;

  int cell = -1, qpos = -1;
  bool done = false;
  double dt = 0.0;
  double y[NS], t = 0.0, h = 0.0, Tc = 0.0;
  float cvR = 1.0f;
  int nst = 0, natt = 0;
  double eta_cell = 1.0;   // Newton contraction estimate carried from step to step
  unsigned long long c_sub = 0, c_fail = 0, c_att = 0, c_newt = 0;
  int flags = 0;

  while (true) {
    // ---- refill idle lanes from the queue
    const bool need = (cell < 0) && !done;
    const unsigned needm = __ballot_sync(0xffffffffu, need);
    if (needm) {
      const int leader = __ffs(needm) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(head, __popc(needm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const int q = base + __popc(needm & ((1u << lane) - 1u));
        if (q < qn) {
          qpos = pass == 2 ? a.cont_sorted[q] : q;
          cell = a.queue[qpos];
          const CellRef<S> cr = locate(a, soff, cell);
          const long long i = cr.i;
          dt = cr.dt;
          c.rho = static_cast<float>(cr.rho[i]);
          c.e0 = static_cast<double>(cr.e[i]);
          if (pass == 2) {   // resume where the probe pass stopped
#pragma unroll
            for (int k = 0; k < NS; ++k) y[k] = cst[k * cc + qpos];
            t = cst[NS * cc + qpos];
            h = cst[(NS + 1) * cc + qpos];
            Tc = cst[(NS + 2) * cc + qpos];
            eta_cell = cst[(NS + 3) * cc + qpos];
            const float* cf = reinterpret_cast<const float*>(cst + (NS + 4) * cc);
            const int* ci = reinterpret_cast<const int*>(cf + cc);
            cvR = cf[qpos];
            nst = ci[qpos];
            natt = ci[cc + qpos];
          } else {
#pragma unroll
            for (int k = 0; k < NS; ++k) y[k] = static_cast<double>(cr.Y[k * cr.ld + i]);
            bool ok;
            double cvd;
            Tc = temperature_from_energy<NS>(m, y, c.e0, static_cast<double>(cr.T[i]), &ok, &cvd);
            cvR = static_cast<float>(cvd);
            t = 0.0;
            nst = 0;
            natt = 0;
            h = 1e-6 * dt;   // the controller grows it by up to 5x per accepted step
            eta_cell = 1.0;
            if (!ok) {       // temperature not invertible: fail the cell right away
              cr.sub[i] = -1;
              ++c_fail;
              flags |= kFlagTemp;
              cell = -1;
            }
          }
        } else {
          done = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, cell < 0)) break;
    if (cell < 0) continue;

    // ---- one attempted SDIRK3 step for this lane's cell
    ++natt;
    ++c_att;
    const double gh = kG * h;
    uint64_t piv;
    bool conv;
    {
      float Yf[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) Yf[k] = static_cast<float>(y[k]);
      float J[NS][NS];
      jacobian<NS>(m, c.rho, static_cast<float>(Tc), Yf, cvR, J);
      store_iteration_matrix<NS>(sm, J, gh);
    }
    conv = lu_factor<NS>(sm, &piv);
    // stage s solves Y_s = y + sum_j A_sj hk_j + g h f(Y_s), hk_j = h k_j, starting from
    // y + sum_j P_sj hk_j (extrapolation of the previous stages to c_s)
    double hk1[NS], hk2[NS], z[NS], base[NS];
    double Tz = Tc;
    double eta = eta_cell;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      hk1[k] = 0.0;
      hk2[k] = 0.0;
    }
#pragma unroll 1
    for (int st = 0; st < 3 && conv; ++st) {
      const double a1 = st == 1 ? kA21 : (st == 2 ? kB1 : 0.0);
      const double a2 = st == 2 ? kB2 : 0.0;
      const double p1 = st == 1 ? kC2 : (st == 2 ? kA21 / kC2 : 0.0);
      const double p2 = st == 2 ? kG / kC2 : 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        base[k] = y[k] + a1 * hk1[k] + a2 * hk2[k];
        z[k] = y[k] + p1 * hk1[k] + p2 * hk2[k];
      }
      conv = stage_newton<NS>(m, sm, piv, c, base, gh, z, Tz, eta, c_newt);
      if (st < 2) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const double hk = (z[k] - base[k]) * (1.0 / kG);
          if (st == 0) hk1[k] = hk; else hk2[k] = hk;
        }
      }
    }
    eta_cell = fmax(eta, 0.05);
    bool finished = false, failed = false;
    if (!conv) {
      h *= 0.25;
      eta_cell = 1.0;
    } else {
      // y_new = Y3 (stiffly accurate); error = (b - bh) . hk, filtered through (I - g h J)^-1
      double er[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const double hk3 = (z[k] - base[k]) * (1.0 / kG);
        er[k] = (kB1 - kBh1) * hk1[k] + (kB2 - kBh2) * hk2[k] + kG * hk3;
      }
      lu_solve<NS>(sm, piv, er);
      double err = 0.0;
      bool neg = false;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const double w = static_cast<double>(c.atol) + static_cast<double>(c.rtol) * fmax(fabs(y[k]), fabs(z[k]));
        err = fmax(err, fabs(er[k]) / w);
        neg = neg || z[k] < -10.0 * static_cast<double>(c.atol);
      }
      // a solution with a clearly negative mass fraction is rejected: an overshoot that the main
      // and the embedded solution share is invisible to the error estimate
      if (neg) err = fmax(err, 4.0);
      if (err <= 1.0) {
        bool ok;
        double cvd;
        const double Tn = temperature_from_energy<NS>(m, z, c.e0, Tz, &ok, &cvd);
        if (ok) {
#pragma unroll
          for (int k = 0; k < NS; ++k) y[k] = z[k];
          Tc = Tn;
          cvR = static_cast<float>(cvd);
          t += h;
          ++nst;
          if (t >= dt * (1.0 - 1e-12)) finished = true;
        } else {
          err = 4.0;   // treat as a rejected step
        }
      }
      double fac = 0.9 * rcbrt(fmax(err, 1e-12));   // embedded order 2: error ~ h^3
      fac = fmin(5.0, fmax(0.2, fac));
      h *= fac;
    }
    if (!finished) {
      if (t + h > dt) h = dt - t;
      if (h < 1e-24 * dt || h < 1e-30) { failed = true; flags |= kFlagNoConv; }
      if (nst >= a.prm.k_max || natt >= 4 * a.prm.k_max) { failed = true; flags |= kFlagMaxSteps; }
    }
    if (!finished && !failed && pass == 1 && natt >= kProbeAttempts) {
      // probe pass: park the cell with its integration state and the remaining-work estimate
#pragma unroll
      for (int k = 0; k < NS; ++k) cst[k * cc + qpos] = y[k];
      cst[NS * cc + qpos] = t;
      cst[(NS + 1) * cc + qpos] = h;
      cst[(NS + 2) * cc + qpos] = Tc;
      cst[(NS + 3) * cc + qpos] = eta_cell;
      float* cf = reinterpret_cast<float*>(cst + (NS + 4) * cc);
      int* ci = reinterpret_cast<int*>(cf + cc);
      cf[qpos] = cvR;
      ci[qpos] = nst;
      ci[cc + qpos] = natt;
      const int pos = atomicAdd(&a.ws->cont_count, 1);
      a.cont_list[pos] = qpos;
      const float rest = static_cast<float>((dt - t) / h);   // steps left at the current step size
      a.cont_key[pos] = static_cast<unsigned char>(fminf(fmaxf(4.0f * __log2f(rest + 1.0f), 0.0f),
                                                         static_cast<float>(kNumBuckets - 1)));
      cell = -1;
    }
    if (finished) {
      const CellRef<S> cr = locate(a, soff, cell);   // recomputed: keeps the loop's registers free
      const long long i = cr.i;
      double sw = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        cr.Y[k * cr.ld + i] = static_cast<S>(y[k]);
        sw = fma(y[k], m.e64[(1 * NS + k) * 8 + 6], sw);
      }
      cr.T[i] = static_cast<S>(Tc);
      if (cr.p) cr.p[i] = static_cast<S>(static_cast<double>(cr.rho[i]) * kR * Tc * sw);
      cr.sub[i] = a.prm.k_bulk + nst;
      c_sub += nst;
      cell = -1;
    } else if (failed) {
      const CellRef<S> cr = locate(a, soff, cell);
      cr.sub[cr.i] = -1;
      ++c_fail;
      cell = -1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_sub += __shfl_down_sync(0xffffffffu, c_sub, o);
    c_fail += __shfl_down_sync(0xffffffffu, c_fail, o);
    c_att += __shfl_down_sync(0xffffffffu, c_att, o);
    c_newt += __shfl_down_sync(0xffffffffu, c_newt, o);
    flags |= __shfl_down_sync(0xffffffffu, flags, o);
  }
  if (lane == 0) {
    if (c_att) atomicAdd(&a.ws->attempts, c_att);
    if (c_newt) atomicAdd(&a.ws->newton, c_newt);
    if (c_sub) atomicAdd(&a.ws->substeps, c_sub);
    if (c_fail) atomicAdd(&a.ws->nfailed, c_fail);
    if (flags) atomicOr(&a.ws->status, flags);
  }
}

// ------------------------------------------------------------------ launchers

#define CHEM_FOR_EACH_NS(X) X(9)

static unsigned pad128(unsigned b) { return (b + 127u) & ~127u; }

size_t stiff_smem_bytes(int ns, unsigned blob_bytes, int nbox) {
  return pad128(blob_bytes) + box_smem_bytes(nbox) + static_cast<size_t>(ns) * (ns + 1) * kStiffBlock * sizeof(double);
}

template <int NS, typename S>
static int stiff_launch_t(const AdvanceArgs<S>& a, int grid, cudaStream_t s) {
  const size_t smem = stiff_smem_bytes(NS, a.blob_bytes, a.nbox);
  auto k = stiff_kernel<NS, S>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  k<<<grid, kStiffBlock, smem, s>>>(a, pad128(a.blob_bytes));
  return static_cast<int>(cudaGetLastError());
}

int launch_stiff_f32(int ns, const AdvanceArgs<float>& a, int grid, cudaStream_t s) {
#define X(N) \
  if (ns == N) return stiff_launch_t<N, float>(a, grid, s);
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int launch_stiff_f64(int ns, const AdvanceArgs<double>& a, int grid, cudaStream_t s) {
#define X(N) \
  if (ns == N) return stiff_launch_t<N, double>(a, grid, s);
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

int stiff_occupancy(int ns, unsigned blob_bytes, int* blocks_per_sm) {
#define X(N)                                                                                     \
  if (ns == N) {                                                                                 \
    const size_t smem = stiff_smem_bytes(N, blob_bytes, 0);                                      \
    cudaFuncSetAttribute(stiff_kernel<N, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                         static_cast<int>(smem));                                                \
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(                      \
        blocks_per_sm, stiff_kernel<N, float>, kStiffBlock, smem));                              \
  }
  CHEM_FOR_EACH_NS(X)
#undef X
  return -1;
}

}  // namespace chem
