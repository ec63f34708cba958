// stiff_body.cuh -- the sparse phase of the bulk-sparse integration (Algorithm 3, section 3) with an
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
//
// The body is a template over the mechanism policy P, which supplies the kinetics and the
// thermodynamics of one cell:
//   P::NS                 species; P::NJ rows and columns of the Jacobian array it fills
//   na()                  species in the leading block of the iteration matrix (the others are
//                         trailing inert species with identity rows and zero right-hand sides)
//   temperature(y, e0, T, &ok, &cv, tol)  FP64 T(e) inversion (Sec. 2.1), Newton steps down to tol T
//   jacobian(rho, T, Yf, cvR, J)          analytic FP32 Jacobian, leading NJ x NJ block
//   rates(rho, T, Yf, f) -> bool          FP32 rates, false if a log-rate left the FP32 range
//   rates64(rho, T, y, f)                 the same rates in FP64 (rounded to FP32)
//   invW64(k)                             1/W_k in FP64 (pressure of the written state)
// stiff.cu instantiates it with the packed tables staged in shared memory.
#pragma once

namespace chem {

constexpr int kNewtMax = 6;
constexpr double kNewtTol = 0.03;   // predicted remaining Newton error below 3% of the error weight
// Stopping tolerance of the T(e) inversions (FP64 Newton, Sec. 2.1).  The temperatures of Newton
// iterates only feed the FP32 rates: a last step |dT| <= 1e-5 T leaves T within ~1e-11 of the root,
// far below the FP32 resolution of those rates, and saves the confirming iteration of the strict
// test.  Temperatures of accepted states (written, and the next step's Jacobian), and every
// temperature of the FP64-rate mode, use 3e-8 T (error ~1e-14 T).
constexpr double kTeIterateTol = 1e-5;
constexpr double kTeStateTol = 3e-8;

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

// Per-thread FP64 iteration matrix (NJ x NJ) and one FP64 vector (NJ) in shared memory: element
// (r, c) of thread t at M[(r * NJ + c) * B + t], vector element k at V[k * B + t], so consecutive
// threads hit consecutive banks.  The factorisation and the solves index them dynamically in
// rolled loops: the FP64 pipe, not the instruction count, bounds these loops, and the rolled code
// keeps the kernel's instruction footprint small enough for the instruction caches.
template <int NJ>
struct Smem {
  double* M;
  double* V;
  int t, B;
  __device__ double& mm(int r, int c) const { return M[(r * NJ + c) * B + t]; }
  __device__ double& vv(int k) const { return V[k * B + t]; }
};

// 1 / x for a pivot: the hardware approximation of the reciprocal (PTX rcp.approx.ftz.f64, relative
// error below 2^-22 for normal x) refined by two Newton-Raphson steps r <- r + r (1 - x r), each of
// which squares the relative error, to within an ulp or two of the FP64 reciprocal.  Four FP64
// FMAs instead of the longer correctly rounded division sequence; an LU needs an accurate pivot
// reciprocal, not a correctly rounded one.  x is a finite nonzero pivot (lu_factor checks it).
__device__ __forceinline__ double pivot_reciprocal(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// |x| as an unsigned integer: for finite values it orders like |x|, so the pivot search compares
// integers (integer pipe) instead of FP64 values (FP64 pipe) and picks the same pivot.
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// M = I - hh * J from the FP32 Jacobian in registers (FP64 in shared memory).  The product
// hh * J is formed in FP32: J carries FP32 rounding already, so the FP64 product would add no
// accuracy, and it saves NJ^2 FP64 multiplies per attempt; the identity is added in FP64.
template <int NJ>
__device__ __forceinline__ void store_iteration_matrix(const Smem<NJ>& s, const float (&J)[NJ][NJ], double hh,
                                                       int na) {
  const float mh = static_cast<float>(-hh);
#pragma unroll
  for (int r = 0; r < NJ; ++r)
#pragma unroll
    for (int c = 0; c < NJ; ++c) {
      if (r < na && c < na) {
        const double v = f32_to_f64_exact(mh * J[r][c]);
        s.mm(r, c) = r == c ? 1.0 + v : v;
      }
    }
}

// LU with partial pivoting in place (unit-lower L below the diagonal, U above, reciprocal of
// U's diagonal on it); pivot rows packed 4 bits each into *piv.  Only the leading na x na block
// is factored: the rows of the trailing inert species are rows of the identity (their rates
// vanish identically), so with a zero right-hand side there the solution of the full system
// is the block's solution extended by zeros, bit for bit.
template <int NJ>
__device__ __forceinline__ bool lu_factor(const Smem<NJ>& s, unsigned long long* piv, int na) {
  unsigned long long pv = 0;
#pragma unroll 1
  for (int k = 0; k < na; ++k) {
    int p = k;
    unsigned long long best = abs_key(s.mm(k, k));
#pragma unroll 1
    for (int i = k + 1; i < na; ++i) {
      const unsigned long long v = abs_key(s.mm(i, k));
      if (v > best) {
        best = v;
        p = i;
      }
    }
    // zero pivot (or NaN): the step fails and is retried smaller
    if (best == 0ull || best > 0x7ff0000000000000ull) return false;
    pv |= static_cast<unsigned long long>(p) << (4 * k);
    if (p != k) {
#pragma unroll 1
      for (int c = 0; c < na; ++c) {
        const double t = s.mm(k, c);
        s.mm(k, c) = s.mm(p, c);
        s.mm(p, c) = t;
      }
    }
    const double inv = pivot_reciprocal(s.mm(k, k));
    s.mm(k, k) = inv;
#pragma unroll 1
    for (int i = k + 1; i < na; ++i) {
      const double l = s.mm(i, k) * inv;
      s.mm(i, k) = l;
#pragma unroll 2
      for (int c = k + 1; c < na; ++c) s.mm(i, c) = fma(-l, s.mm(k, c), s.mm(i, c));
    }
  }
  *piv = pv;
  return true;
}

// Solve M x = b with the factors of lu_factor (b in registers, in and out; the permutation and
// the substitutions run on the shared-memory vector).  Entries na.. of b (the inert species,
// zero) pass through unchanged.
template <int NJ, int NS>
__device__ __forceinline__ void lu_solve(const Smem<NJ>& s, unsigned long long piv, double (&b)[NS], int na) {
#pragma unroll
  for (int k = 0; k < NJ; ++k) s.vv(k) = b[k];
#pragma unroll 1
  for (int k = 0; k < na; ++k) {
    const int p = static_cast<int>((piv >> (4 * k)) & 15u);
    if (p != k) {
      const double t = s.vv(k);
      s.vv(k) = s.vv(p);
      s.vv(p) = t;
    }
  }
#pragma unroll 1
  for (int i = 1; i < na; ++i) {
    double acc = s.vv(i);
#pragma unroll 1
    for (int j = 0; j < i; ++j) acc = fma(-s.mm(i, j), s.vv(j), acc);
    s.vv(i) = acc;
  }
#pragma unroll 1
  for (int i = na - 1; i >= 0; --i) {
    double acc = s.vv(i);
#pragma unroll 1
    for (int j = i + 1; j < na; ++j) acc = fma(-s.mm(i, j), s.vv(j), acc);
    s.vv(i) = acc * s.mm(i, i);
  }
#pragma unroll
  for (int k = 0; k < NJ; ++k) b[k] = s.vv(k);
}

struct CellCtx {
  float rho, rtol, atol;
  double e0;
  bool fp64_rates;
};

// One simplified-Newton iteration of the stage equation z = yb + hh f(z) (iteration matrix
// factored in shared memory).  Tz: temperature guess in, temperature of the evaluated iterate
// out.  Convergence is judged on the weighted RMS norm of the update and the contraction rate
// theta of the iteration: the iterate is accepted when the remaining error predicted from theta,
// eta * |dz| with eta = theta / (1 - theta), is below kNewtTol.  eta carries over between the
// stages of a step (the first iteration of a stage uses the last value).  it and prev hold the
// stage's iteration count and last norm.  known_T: z is the step's initial state and Tz its
// temperature (inverted at the state tolerance), so the iterate's inversion is skipped.  Returns
// 1 when the stage has converged, 0 to iterate again, -1 on failure (T(e) lost, non-finite or
// diverging update, kNewtMax iterations).
template <class P>
__device__ __forceinline__ int newton_iteration(const P& m, const Smem<P::NJ>& s, unsigned long long piv,
                                                const CellCtx& c, const double (&yb)[P::NS], double hh,
                                                double (&z)[P::NS], double& Tz, float& eta, float& prev, int& it,
                                                unsigned long long& n_it, bool known_T) {
  constexpr int NS = P::NS;
  ++n_it;
  if (__builtin_expect(!known_T, 1)) {
    bool ok;
    // FP64 rates (CHEM_FLAG_FP64_RATES) resolve T beyond FP32: their iterates keep the strict tolerance
    Tz = m.temperature(z, c.e0, Tz, &ok, nullptr, c.fp64_rates ? kTeStateTol : kTeIterateTol);
    if (!ok) return -1;
  }
  float F[NS], Zf[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) Zf[k] = static_cast<float>(z[k]);
  bool use64 = c.fp64_rates;
  // FP32 rates; the FP64 instance (one copy in the code) when they overflow
  if (!use64) use64 = !m.rates(c.rho, static_cast<float>(Tz), Zf, F);
  if (use64) m.rates64(c.rho, Tz, z, F);
  const float mhh = static_cast<float>(hh);
  // species na.. (trailing inert ones) have zero rates and zero residual: their update is exactly
  // zero, so their FP64 work is skipped (the same bits as doing it)
  const int na = m.na();
  double b[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) b[k] = k < na ? (yb[k] - z[k]) + static_cast<double>(mhh * F[k]) : 0.0;
  lu_solve<P::NJ, NS>(s, piv, b, na);
  float ss = 0.0f;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (k < na) {
      z[k] += b[k];
      const float bf = static_cast<float>(b[k]);
      const float w = c.atol + c.rtol * fabsf(Zf[k] + bf);
      const float r = bf / w;
      ss = fmaf(r, r, ss);
    }
  }
  // the convergence control (norm, contraction rate) is FP32: it only decides when to stop
  const float nrm = sqrtf(ss * (1.0f / NS));
  if (!(nrm == nrm)) return -1;
  if (it > 0) {
    const float theta = nrm / prev;
    if (theta >= 1.0f) {
      // not contracting: accept only at the FP32 noise floor (below half the error weight)
      return (nrm <= 0.5f && theta < 2.0f) ? 1 : -1;
    }
    eta = theta / (1.0f - theta);
  }
  if (eta * nrm <= static_cast<float>(kNewtTol) || nrm <= 1e-3f) return 1;
  prev = nrm;
  return ++it < kNewtMax ? 0 : -1;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier between the continuation rounds (the launch is cooperative, so every CTA is
// resident).  The wait is bounded: after 4 s of wall time the CTA records kFlagStage and returns
// false, and the kernel ends.
__device__ __forceinline__ bool grid_barrier(Workspace* ws) {
  __shared__ int ok_s;
  __threadfence();   // this thread's list entries and parked states, visible device-wide
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &ws->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&ws->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&ws->bar_count, 0u);
      __threadfence();
      atomicAdd(&ws->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        __nanosleep(256);
        if (global_ns() - t0 > 4000000000ull) {
          ok = 0;
          atomicOr(&ws->status, kFlagStage);
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Shared memory of the stiff kernel after the staged tables (tab_bytes, 128-aligned): the box
// offsets, then the per-thread iteration matrices and vectors.
__host__ __device__ constexpr unsigned long long stiff_matrix_bytes(int nj, int block) {
  return static_cast<unsigned long long>(nj) * (nj + 1) * block * 8ull;
}

// The kernel body (BLK threads per CTA).  smem: dynamic shared memory; tab_pad: bytes at its start
// taken by the staged tables (0 for a policy with compiled-in constants).
template <class P, typename S, int BLK>
__device__ __forceinline__ void stiff_body(const AdvanceArgs<S>& a, const P& m, unsigned char* smem,
                                           unsigned tab_pad) {
  constexpr int NS = P::NS;
  constexpr int NJ = P::NJ;
  int* soff = reinterpret_cast<int*>(smem + tab_pad);
  if (a.nbox > 0) stage_box_offsets(soff, a.box_off, a.nbox);
  Smem<NJ> sm;
  sm.t = threadIdx.x;
  sm.B = BLK;
  sm.M = reinterpret_cast<double*>(smem + tab_pad + box_smem_bytes(a.nbox));
  sm.V = sm.M + NJ * NJ * BLK;
  const int na = m.na();

  const int lane = threadIdx.x & 31;
  // probe and single passes take cells from the stiff queue through an atomic head.  The
  // continuation pass runs in rounds.  Round 0 takes the sorted unfinished cells from a shared
  // queue (longest remaining first) and runs them to completion until the queue is empty; from
  // then on a lane parks its cell after a.round_att more steps.  Round r >= 1 gives every
  // parked cell up to a.round_att steps and lists those still unfinished for round r + 1; slot
  // q of its list belongs to lane q % 32 of warp q / 32 mod W, warps numbered across the CTAs
  // first, so that the cells still running fill whole warps spread over all SMs.
  const int pass = a.pass;
  int qn = pass == 2 ? min(*reinterpret_cast<volatile int*>(&a.ws->cont_count), static_cast<int>(a.n))
                     : min(*reinterpret_cast<volatile int*>(&a.ws->qcount), static_cast<int>(a.n));
  int* head = pass == 2 ? &a.ws->head2 : &a.ws->head;
  // round r >= 1 reads cont_list (r odd) or cont_sorted (r even) and writes the other one;
  // natt_r: steps in the round (round 0: steps since the queue ran empty, -1 before)
  int round = 0, kr = 0, natt_r = 0;
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
  float eta_cell = 1.0f;   // Newton contraction estimate carried from step to step
  unsigned long long c_sub = 0, c_fail = 0, c_att = 0, c_newt = 0;
  int flags = 0;

  while (true) {
    // ---- refill idle lanes from the queue
    const bool need = (cell < 0) && !done;
    const unsigned needm = __ballot_sync(0xffffffffu, need);
    if (needm) {
      int base = 0;
      if (pass != 2 || round == 0) {
        const int leader = __ffs(needm) - 1;
        if (lane == leader) base = atomicAdd(head, __popc(needm));
        base = __shfl_sync(0xffffffffu, base, leader);
      }
      if (need) {
        long long q;
        if (pass == 2 && round > 0) {
          const long long wg = static_cast<long long>(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
          q = (wg + static_cast<long long>(kr) * gridDim.x * (BLK / 32)) * 32 + lane;
          ++kr;
        } else {
          q = base + __popc(needm & ((1u << lane) - 1u));
        }
        if (q < qn) {
          natt_r = (pass == 2 && round == 0) ? -1 : 0;
          // lists and parked states of the continuation rounds are written by other CTAs during
          // this launch: read them past L1 (ld.global.cg)
          qpos = pass == 2 ? __ldcg(((round & 1) ? a.cont_list : a.cont_sorted) + q) : static_cast<int>(q);
          cell = a.queue[qpos];
          const CellRef<S> cr = locate(a, soff, cell);
          const long long i = cr.i;
          dt = cr.dt;
          c.rho = static_cast<float>(cr.rho[i]);
          c.e0 = static_cast<double>(cr.e[i]);
          if (pass == 2) {   // resume where the previous pass or round stopped
#pragma unroll
            for (int k = 0; k < NS; ++k) y[k] = __ldcg(cst + k * cc + qpos);
            t = __ldcg(cst + NS * cc + qpos);
            h = __ldcg(cst + (NS + 1) * cc + qpos);
            Tc = __ldcg(cst + (NS + 2) * cc + qpos);
            eta_cell = static_cast<float>(__ldcg(cst + (NS + 3) * cc + qpos));
            const float* cf = reinterpret_cast<const float*>(cst + (NS + 4) * cc);
            const int* ci = reinterpret_cast<const int*>(cf + cc);
            cvR = __ldcg(cf + qpos);
            nst = __ldcg(ci + qpos);
            natt = __ldcg(ci + cc + qpos);
          } else {
#pragma unroll
            for (int k = 0; k < NS; ++k) y[k] = static_cast<double>(cr.Y[k * cr.ld + i]);
            bool ok;
            double cvd;
            Tc = m.temperature(y, c.e0, static_cast<double>(cr.T[i]), &ok, &cvd, kTeStateTol);
            cvR = static_cast<float>(cvd);
            t = 0.0;
            nst = 0;
            natt = 0;
            h = 1e-6 * dt;   // the controller grows it by up to 5x per accepted step
            eta_cell = 1.0f;
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
    if (__all_sync(0xffffffffu, cell < 0)) {
      if (pass != 2) break;
      // end of a continuation round: wait for every CTA, then take the survivors' list
      if (!grid_barrier(a.ws)) break;
      const int next = min(*reinterpret_cast<volatile int*>(&a.ws->rc[round % 3]), static_cast<int>(a.n));
      if (next == 0) break;
      ++round;
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&a.ws->rc[(round + 1) % 3], 0);   // output of round + 1
      qn = next;
      kr = 0;
      done = false;
      continue;
    }
    const unsigned work = __ballot_sync(0xffffffffu, cell >= 0);   // the lanes that take a step
    if (cell < 0) continue;

    // ---- one attempted SDIRK3 step for this lane's cell
    ++natt;
    ++c_att;
    if (pass == 2) {
      if (natt_r < 0 && *reinterpret_cast<volatile const int*>(head) >= qn) natt_r = 0;   // queue empty
      if (natt_r >= 0) ++natt_r;
    }
    const double gh = kG * h;
    unsigned long long piv;
    bool conv;
    {
      float Yf[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) Yf[k] = static_cast<float>(y[k]);
      float J[NJ][NJ];
      m.jacobian(c.rho, static_cast<float>(Tc), Yf, cvR, J);
      store_iteration_matrix<NJ>(sm, J, gh, na);
    }
    conv = lu_factor<NJ>(sm, &piv, na);
    double hk1[NS], hk2[NS], z[NS], base[NS];
    double Tz = Tc;
    float eta = eta_cell;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      hk1[k] = 0.0;
      hk2[k] = 0.0;
    }
    // the three stages run as one flat sequence of Newton iterations per lane, so that a lane
    // whose stage converges early starts its next stage instead of waiting for the slowest lane:
    // the warp pays max over lanes of the step's iterations rather than the sum over stages of
    // the per-stage maxima.  Stage s solves Y_s = y + sum_j A_sj hk_j + g h f(Y_s), hk_j = h k_j,
    // starting from y + sum_j P_sj hk_j (extrapolation of the previous stages to c_s).
    int st = 0, it = 0;
    float prev = 0.0f;
    bool act = conv;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      base[k] = y[k];
      z[k] = y[k];
    }
#pragma unroll 1
    while (__any_sync(work, act)) {
      if (act) {
        // the first iterate of stage 1 is y itself, whose temperature Tc is known
        const int r = newton_iteration<P>(m, sm, piv, c, base, gh, z, Tz, eta, prev, it, c_newt, st == 0 && it == 0);
        if (r < 0) {
          conv = false;
          act = false;
        } else if (r > 0) {
          // the inert species keep hk = 0 and base = z = y (their stage increments are exactly zero)
          if (st < 2) {
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              if (k < na) {
                const double hk = (z[k] - base[k]) * (1.0 / kG);
                if (st == 0) hk1[k] = hk; else hk2[k] = hk;
              }
            }
          }
          ++st;
          if (st == 3) {
            act = false;
          } else {
            if (st == 1) {   // stage 2 starts from y + a21 hk1 (its hk2 term is zero)
#pragma unroll
              for (int k = 0; k < NS; ++k) {
                if (k < na) {
                  base[k] = y[k] + kA21 * hk1[k];
                  z[k] = y[k] + kC2 * hk1[k];
                }
              }
            } else {
#pragma unroll
              for (int k = 0; k < NS; ++k) {
                if (k < na) {
                  base[k] = y[k] + kB1 * hk1[k] + kB2 * hk2[k];
                  z[k] = y[k] + (kA21 / kC2) * hk1[k] + (kG / kC2) * hk2[k];
                }
              }
            }
            it = 0;
            prev = 0.0f;
          }
        }
      }
    }
    eta_cell = fmaxf(eta, 0.05f);
    bool finished = false, failed = false;
    if (!conv) {
      h *= 0.25;
      eta_cell = 1.0f;
    } else {
      // y_new = Y3 (stiffly accurate); error = (b - bh) . hk, filtered through (I - g h J)^-1
      double er[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (k < na) {
          const double hk3 = (z[k] - base[k]) * (1.0 / kG);
          er[k] = (kB1 - kBh1) * hk1[k] + (kB2 - kBh2) * hk2[k] + kG * hk3;
        } else {
          er[k] = 0.0;
        }
      }
      lu_solve<NJ, NS>(sm, piv, er, na);
      // the weighted error norm is a step-size control quantity: FP32 (the inert species add 0)
      float err = 0.0f;
      bool neg = false;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (k < na) {
          const float zk = static_cast<float>(z[k]);
          const float w = c.atol + c.rtol * fmaxf(fabsf(static_cast<float>(y[k])), fabsf(zk));
          err = fmaxf(err, fabsf(static_cast<float>(er[k])) / w);
          neg = neg || zk < -10.0f * c.atol;
        }
      }
      // a solution with a clearly negative mass fraction is rejected: an overshoot that the main
      // and the embedded solution share is invisible to the error estimate
      if (neg) err = fmaxf(err, 4.0f);
      if (err <= 1.0f) {
        bool ok;
        double cvd;
        const double Tn = m.temperature(z, c.e0, Tz, &ok, &cvd, kTeStateTol);
        if (ok) {
#pragma unroll
          for (int k = 0; k < NS; ++k) y[k] = z[k];
          Tc = Tn;
          cvR = static_cast<float>(cvd);
          t += h;
          ++nst;
          if (t >= dt * (1.0 - 1e-12)) finished = true;
        } else {
          err = 4.0f;   // treat as a rejected step
        }
      }
      float fac = 0.9f * rcbrtf(fmaxf(err, 1e-12f));   // embedded order 2: error ~ h^3
      fac = fminf(5.0f, fmaxf(0.2f, fac));
      h *= static_cast<double>(fac);
    }
    if (!finished) {
      if (t + h > dt) h = dt - t;
      if (h < 1e-24 * dt || h < 1e-30) { failed = true; flags |= kFlagNoConv; }
      if (nst >= a.prm.k_max || natt >= 4 * a.prm.k_max) { failed = true; flags |= kFlagMaxSteps; }
    }
    if (!finished && !failed &&
        ((pass == 1 && natt >= a.probe_att) || (pass == 2 && natt_r >= a.round_att))) {
      // park the cell with its integration state (probe pass: for the sort and round 0; later:
      // for the next round)
#pragma unroll
      for (int k = 0; k < NS; ++k) cst[k * cc + qpos] = y[k];
      cst[NS * cc + qpos] = t;
      cst[(NS + 1) * cc + qpos] = h;
      cst[(NS + 2) * cc + qpos] = Tc;
      cst[(NS + 3) * cc + qpos] = static_cast<double>(eta_cell);
      float* cf = reinterpret_cast<float*>(cst + (NS + 4) * cc);
      int* ci = reinterpret_cast<int*>(cf + cc);
      cf[qpos] = cvR;
      ci[qpos] = nst;
      ci[cc + qpos] = natt;
      if (pass == 1) {
        const int pos = atomicAdd(&a.ws->cont_count, 1);
        a.cont_list[pos] = qpos;
        const float rest = static_cast<float>((dt - t) / h);   // steps left at the current step size
        a.cont_key[pos] = static_cast<unsigned char>(fminf(fmaxf(4.0f * __log2f(rest + 1.0f), 0.0f),
                                                           static_cast<float>(kNumBuckets - 1)));
      } else {
        ((round & 1) ? a.cont_sorted : a.cont_list)[atomicAdd(&a.ws->rc[round % 3], 1)] = qpos;
      }
      cell = -1;
    }
    if (finished) {
      const CellRef<S> cr = locate(a, soff, cell);   // recomputed: keeps the loop's registers free
      const long long i = cr.i;
      double sw = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        cr.Y[k * cr.ld + i] = static_cast<S>(y[k]);
        sw = fma(y[k], m.invW64(k), sw);
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

}  // namespace chem
