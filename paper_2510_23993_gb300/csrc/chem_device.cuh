// chem_device.cuh -- device-side building blocks of the chemistry kernels (sm_103a).
//
// * MechView: the mechanism tables, packed on the host by chem_init into one 16-byte aligned
//   blob and staged once per CTA into shared memory with a TMA bulk copy (cp.async.bulk +
//   mbarrier, bounded wait).
// * temperature_from_energy: FP64 Newton inversion of e(T) = sum_k Y_k u_k(T) at fixed Y
//   (Sec. 2.1), on per-regime mixture polynomial coefficients.
// * rates: the matrix form of the kinetics (Sec. 1/3.2: log-concentrations times the
//   stoichiometric matrix plus the Arrhenius terms, then exp), FP32, with an FP64 instance of
//   the same code for cells whose log-rates leave the FP32 range.
// * jacobian: analytic dense d(dY/dt)/dY of Eq. 5 in FP32, with the temperature eliminated
//   through dT/dY_k = -u_k / c_v (constant e and rho).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace chem {

constexpr double kR = 8.314462618;     // J/mol/K
constexpr double kP0 = 101325.0;       // Pa, standard pressure of K_p
constexpr double kLnP0R = 9.408091968961747;   // ln(p0 / R)
constexpr float kLnZero = -1.0e4f;     // ln C used for C <= 0 (exp() of any rate with it is 0)
constexpr float kLnQMax = 87.0f;       // FP32 exp overflow guard
constexpr double kTbrLo = 50.0, kTbrHi = 20000.0;   // bracket of the T(e) inversion

// status bits accumulated in the device status word
enum : int { kFlagInvalid = 1, kFlagMaxSteps = 2, kFlagNoConv = 4, kFlagStage = 8, kFlagTemp = 16 };

// Layout of the packed mechanism blob (byte offsets, all multiples of 16).
struct MechHdr {
  int ns, nr, ntb, nsp;          // nsp = ns rounded up to 4
  float T_lo, T_hi, lnP0R;       // lnP0R = ln(p0 / R)
  int nact;                      // species before the trailing run of inert ones (no net
                                 //   stoichiometry in any reaction); 0 = all species
  int off_arr, off_nuf, off_nur, off_dnu;
  int off_eff, off_rinfo, off_W, off_invW;
  int off_gam, off_hco, off_hsp, off_e64;
  int off_arr64, off_gam64, off_eff64, bytes;
  // large-mechanism layout (large != 0, large.cu): sparse stoichiometry instead of the dense
  // rows, a species -> reaction index, and the thermo regimes below / above the fit range in a
  // global-only tail after the `prefix` bytes that are staged into shared memory
  int off_sto, off_cptr, off_cent, off_gamg;
  int off_hcog, prefix, nnz, large;
};

// Device view of the (staged) tables.
struct MechView {
  int ns, nr, nsp, nact;
  float T_lo, T_hi, lnP0R;
  const float4* arr;     // [nr] lnA, b, Ea/R, sum dnu
  const float* nuf;      // [nr][nsp]
  const float* nur;      // [nr][nsp]
  const float* dnu;      // [nr][nsp]
  const float* eff;      // [ntb][nsp]
  const int* rinfo;      // [nr] bit0 reversible, (tb row + 1) << 8
  const float* W;        // [nsp]
  const float* invW;     // [nsp]
  const float* gam;      // [3][nr][8] dG/RT = sum_j gam_j phi_j(T), phi = (1-lnT, T, T^2, T^3, T^4, 1/T, 1)
  const float* hco;      // [3][nr][8] dH/RT = sum_j hco_j psi_j(T), psi = (1, T, T^2, T^3, T^4, 1/T)
  const float* hsp;      // [3][ns][8] h_k/RT = sum_j hsp_j psi_j(T)
  const double* e64;     // [3][ns][8] e/R per mass = sum_j c_j T^j (j = 0..5), c_6 = 1/W
  const double* arr64;   // [nr][4] FP64 copy of arr (used by the FP64 rate instance)
  const double* gam64;   // [3][nr][8] FP64 copy of gam
  const double* eff64;   // [ntb][nsp] FP64 copy of eff
};

__device__ __forceinline__ MechView make_view(const unsigned char* base) {
  const MechHdr* h = reinterpret_cast<const MechHdr*>(base);
  MechView v;
  v.ns = h->ns;
  v.nr = h->nr;
  v.nsp = h->nsp;
  v.nact = h->nact > 0 ? h->nact : h->ns;
  v.T_lo = h->T_lo;
  v.T_hi = h->T_hi;
  v.lnP0R = h->lnP0R;
  v.arr = reinterpret_cast<const float4*>(base + h->off_arr);
  v.nuf = reinterpret_cast<const float*>(base + h->off_nuf);
  v.nur = reinterpret_cast<const float*>(base + h->off_nur);
  v.dnu = reinterpret_cast<const float*>(base + h->off_dnu);
  v.eff = reinterpret_cast<const float*>(base + h->off_eff);
  v.rinfo = reinterpret_cast<const int*>(base + h->off_rinfo);
  v.W = reinterpret_cast<const float*>(base + h->off_W);
  v.invW = reinterpret_cast<const float*>(base + h->off_invW);
  v.gam = reinterpret_cast<const float*>(base + h->off_gam);
  v.hco = reinterpret_cast<const float*>(base + h->off_hco);
  v.hsp = reinterpret_cast<const float*>(base + h->off_hsp);
  v.e64 = reinterpret_cast<const double*>(base + h->off_e64);
  v.arr64 = reinterpret_cast<const double*>(base + h->off_arr64);
  v.gam64 = reinterpret_cast<const double*>(base + h->off_gam64);
  v.eff64 = reinterpret_cast<const double*>(base + h->off_eff64);
  return v;
}

// ------------------------------------------------------------------ TMA staging

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global memory into this
// CTA's shared memory with one bulk async copy completed on an mbarrier.  All threads of the
// block must call it.  Returns false (block-uniform) if the copy did not complete within the
// spin limit; the error is recorded in *status and the caller must return without touching
// the destination.
__device__ __forceinline__ bool stage_to_smem(void* dst, const void* src, unsigned bytes,
                                              uint64_t* bar, int* status) {
  const unsigned bar_a = static_cast<unsigned>(__cvta_generic_to_shared(bar));
  const unsigned dst_a = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_a),
        "l"(src), "r"(bytes), "r"(bar_a)
        : "memory");
  }
  unsigned done = 0;
  for (int spin = 0; spin < (1 << 20) && !done; ++spin) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar_a), "r"(0u)
        : "memory");
  }
  const bool failed = __syncthreads_or(!done);
  if (failed) {
    if (threadIdx.x == 0) atomicOr(status, kFlagStage);
    // give a copy still in flight a bounded second chance to land before the CTA exits
    for (int spin = 0; spin < (1 << 20) && !done; ++spin) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(bar_a), "r"(0u)
          : "memory");
    }
    return false;
  }
  return true;
}

// ------------------------------------------------------------------ thermodynamics

__device__ __forceinline__ int regime_of(float T, float T_lo, float T_hi) {
  return T < T_lo ? 0 : (T > T_hi ? 2 : 1);
}

// FP64 mixture coefficients E_j = sum_k Y_k c_jk (j = 0..5) and S = sum_k Y_k / W_k.  Outside the
// fit range (regimes 0 and 2) c_p is frozen, so c_jk = 0 for j >= 2 and only E_0, E_1 are summed.
template <int NS, typename Y_t>
__device__ __forceinline__ void mixture64(const MechView& m, int reg, const Y_t* Y, double E[6]) {
  const double* c = m.e64 + reg * NS * 8;
#pragma unroll
  for (int j = 0; j < 6; ++j) E[j] = 0.0;
  if (reg == 1) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double y = static_cast<double>(Y[k]);
#pragma unroll
      for (int j = 0; j < 6; ++j) E[j] = fma(y, c[k * 8 + j], E[j]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double y = static_cast<double>(Y[k]);
      E[0] = fma(y, c[k * 8 + 0], E[0]);
      E[1] = fma(y, c[k * 8 + 1], E[1]);
    }
  }
}

// T such that e(T, Y) = e0 (FP64 Newton on the mixture polynomial, bisection safeguard).
// mix(reg, E) fills E_j = sum_k Y_k c_jk of regime reg (the caller's mixture coefficients).
// Returns the temperature; *ok is cleared if the root was not found inside [50, 20000] K.
// *cv_out (optional) receives c_v / R at the solution (J/kg/K divided by R).  The iteration stops
// after a Newton step |dT| <= tol T; the error left is then ~1e-7 |dT| (FP32 reciprocal of c_v)
// plus the quadratic term (c_v'/2c_v) dT^2 with c_v'/c_v ~ 1e-4 / K: below 1e-14 T for the default
// tol = 3e-8, below 1e-11 T for tol = 1e-5.
template <class Mix>
__device__ __forceinline__ double temperature_newton(const Mix& mix, float T_lo, float T_hi, double e0, double T,
                                                     bool* ok, double* cv_out, double tol = 3e-8) {
  const double eR = e0 * (1.0 / kR);
  double lo = kTbrLo, hi = kTbrHi;
  if (!(T > lo && T < hi)) T = 1000.0;
  int reg = regime_of(static_cast<float>(T), T_lo, T_hi);
  double E[6], D[4];   // D: the coefficients of de/dT, computed once per regime
  mix(reg, E);
  D[0] = 2.0 * E[2];
  D[1] = 3.0 * E[3];
  D[2] = 4.0 * E[4];
  D[3] = 5.0 * E[5];
  double cv = 0.0;
  bool conv = false;
#pragma unroll 1
  for (int it = 0; it < 60; ++it) {
    const double f = fma(T, fma(T, fma(T, fma(T, fma(T, E[5], E[4]), E[3]), E[2]), E[1]), E[0]) - eR;
    cv = fma(T, fma(T, fma(T, fma(T, D[3], D[2]), D[1]), D[0]), E[1]);
    if (f > 0.0) hi = T; else lo = T;
    // Newton step with an FP32 reciprocal of c_v: the step is exact to ~1e-7 relative, so the
    // iteration still converges to the FP64 root (the residual f is FP64).
    double Tn = (cv > 0.0) ? T - f * static_cast<double>(__frcp_rn(static_cast<float>(cv))) : 0.5 * (lo + hi);
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    const double dT = Tn - T;
    T = Tn;
    const int nreg = regime_of(static_cast<float>(T), T_lo, T_hi);
    if (nreg != reg) {
      reg = nreg;
      mix(reg, E);
      D[0] = 2.0 * E[2];
      D[1] = 3.0 * E[3];
      D[2] = 4.0 * E[4];
      D[3] = 5.0 * E[5];
      continue;
    }
    if (fabs(dT) <= tol * T) { conv = true; break; }
  }
  if (cv_out) *cv_out = cv;
  *ok = conv && (T > kTbrLo) && (T < kTbrHi);
  return T;
}

// The mixture coefficients of the staged tables.
template <int NS, typename Y_t>
struct TableMix {
  const MechView& m;
  const Y_t* Y;
  __device__ __forceinline__ void operator()(int reg, double* E) const { mixture64<NS>(m, reg, Y, E); }
};

// T(e) over the staged tables.
template <int NS, typename Y_t>
__device__ double temperature_from_energy(const MechView& m, const Y_t* Y, double e0, double T,
                                          bool* ok, double* cv_out = nullptr, double tol = 3e-8) {
  const TableMix<NS, Y_t> mix{m, Y};
  return temperature_newton(mix, m.T_lo, m.T_hi, e0, T, ok, cv_out, tol);
}

// Exact FP32 -> FP64 conversion with integer operations.  On GB300 a conversion instruction
// occupies the FP64 pipe (about as long as an FP64 FMA), and the FP64 pipe bounds the stiff
// kernels; the bit assembly runs on the integer pipe instead.  Zeros, subnormals, infinities and NaNs take the
// conversion instruction.  The result is the same value as static_cast<double>.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return static_cast<double>(x);
  const unsigned m = u & 0x7fffffu;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3);   // 896 = 1023 - 127
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(m << 29));
}

// ------------------------------------------------------------------ kinetics

template <typename R> __device__ __forceinline__ R r_exp(R x);
template <> __device__ __forceinline__ float r_exp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double r_exp<double>(double x) { return exp(x); }
template <typename R> __device__ __forceinline__ R r_log(R x);
template <> __device__ __forceinline__ float r_log<float>(float x) { return __logf(x); }
template <> __device__ __forceinline__ double r_log<double>(double x) { return log(x); }

// Arrhenius and Gibbs coefficients of reaction r in the precision of the rate instance R
// (FP32 tables for the FP32 path, FP64 tables for the FP64 path).
template <typename R> struct Coef;
template <> struct Coef<float> {
  __device__ static float4 arr(const MechView& m, int r) { return m.arr[r]; }
  __device__ static const float* gam(const MechView& m, int reg, int r) { return m.gam + (reg * m.nr + r) * 8; }
  __device__ static const float* eff(const MechView& m, int tb) { return m.eff + tb * m.nsp; }
  __device__ static float invW(const MechView& m, int ns, int k) { return m.invW[k]; }
  __device__ static float W(const MechView& m, int ns, int k) { return m.W[k]; }
};
template <> struct Coef<double> {
  __device__ static double4 arr(const MechView& m, int r) {
    const double* a = m.arr64 + 4 * r;
    return make_double4(a[0], a[1], a[2], a[3]);
  }
  __device__ static const double* gam(const MechView& m, int reg, int r) { return m.gam64 + (reg * m.nr + r) * 8; }
  __device__ static const double* eff(const MechView& m, int tb) { return m.eff64 + tb * m.nsp; }
  __device__ static double invW(const MechView& m, int ns, int k) { return m.e64[(ns + k) * 8 + 6]; }
  __device__ static double W(const MechView& m, int ns, int k) { return 1.0 / m.e64[(ns + k) * 8 + 6]; }
};

// Per-cell kinetics workspace kept in registers.
template <int NS, typename R>
struct KinState {
  R C[NS], lnC[NS];
  R lnT, invT, lnP0RT;
  int reg;
};

template <int NS, typename R>
__device__ __forceinline__ void kin_prepare(const MechView& m, R rho, R T, const R* Y, KinState<NS, R>& s) {
  s.lnT = r_log<R>(T);
  s.invT = R(1) / T;
  s.lnP0RT = static_cast<R>(kLnP0R) - s.lnT;   // ln(p0 / (R T))
  s.reg = regime_of(static_cast<float>(T), m.T_lo, m.T_hi);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    s.C[k] = rho * Y[k] * Coef<R>::invW(m, NS, k);
    s.lnC[k] = s.C[k] > R(0) ? r_log<R>(s.C[k]) : static_cast<R>(kLnZero);
  }
}

// ln k_f, ln q_f and ln q_r of reaction r (without third-body factor).
template <int NS, typename R>
__device__ __forceinline__ void log_rates(const MechView& m, const KinState<NS, R>& s, R T, int r,
                                          R& lnkf, R& lnqf, R& lnqr, bool& rev) {
  const auto a = Coef<R>::arr(m, r);
  lnkf = static_cast<R>(a.x) + static_cast<R>(a.y) * s.lnT - static_cast<R>(a.z) * s.invT;
  const float* nf = m.nuf + r * m.nsp;
  R sf = R(0);
#pragma unroll
  for (int k = 0; k < NS; ++k) sf += static_cast<R>(nf[k]) * s.lnC[k];
  lnqf = lnkf + sf;
  rev = (m.rinfo[r] & 1) != 0;
  lnqr = static_cast<R>(kLnZero);
  if (rev) {
    const auto* g = Coef<R>::gam(m, s.reg, r);
    const R T2 = T * T;
    const R dG = static_cast<R>(g[0]) * (R(1) - s.lnT) +
                 T * (static_cast<R>(g[1]) + T * static_cast<R>(g[2]) + T2 * (static_cast<R>(g[3]) + T * static_cast<R>(g[4]))) +
                 static_cast<R>(g[5]) * s.invT + static_cast<R>(g[6]);
    const R lnKc = -dG + static_cast<R>(a.w) * s.lnP0RT;
    const float* nb = m.nur + r * m.nsp;
    R sr = R(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) sr += static_cast<R>(nb[k]) * s.lnC[k];
    lnqr = lnkf - lnKc + sr;
  }
}

// dY/dt of Eq. 5.  Returns false if a log-rate exceeded the FP32 exp range (then f is not
// usable and the caller re-evaluates in FP64).
template <int NS, typename R>
__device__ __forceinline__ bool rates(const MechView& m, R rho, R T, const R* Y, R* f) {
  KinState<NS, R> s;
  kin_prepare<NS, R>(m, rho, T, Y, s);
  R w[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) w[k] = R(0);
  bool fine = true;
#pragma unroll 1
  for (int r = 0; r < m.nr; ++r) {
    R lnkf, lnqf, lnqr;
    bool rev;
    log_rates<NS, R>(m, s, T, r, lnkf, lnqf, lnqr, rev);
    if (sizeof(R) == 4) fine &= (lnqf < static_cast<R>(kLnQMax)) & (lnqr < static_cast<R>(kLnQMax));
    R q = r_exp<R>(lnqf) - r_exp<R>(lnqr);
    const int tb = (m.rinfo[r] >> 8) - 1;
    if (tb >= 0) {
      const auto* ef = Coef<R>::eff(m, tb);
      R M = R(0);
#pragma unroll
      for (int k = 0; k < NS; ++k) M += static_cast<R>(ef[k]) * (s.C[k] > R(0) ? s.C[k] : R(0));
      q *= M;
    }
    const float* dn = m.dnu + r * m.nsp;
#pragma unroll
    for (int k = 0; k < NS; ++k) w[k] += static_cast<R>(dn[k]) * q;
  }
  const R irho = R(1) / rho;
#pragma unroll
  for (int k = 0; k < NS; ++k) f[k] = w[k] * Coef<R>::W(m, NS, k) * irho;
  return fine;
}

// FP64 instance of the rates: it only runs for cells whose FP32 log-rates overflow.
template <int NS>
__device__ __forceinline__ void rates_fp64_fallback(const MechView& m, float rho, double T, const double* y, float* f) {
  double fd[NS];
  rates<NS, double>(m, static_cast<double>(rho), T, y, fd);
#pragma unroll
  for (int k = 0; k < NS; ++k) f[k] = static_cast<float>(fd[k]);
}

// FP32 rates with the FP64 instance as fallback when FP32 log-rates overflow.
template <int NS>
__device__ __forceinline__ void rates_safe(const MechView& m, float rho, double T, const double* y, float* f) {
  float Yf[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) Yf[k] = static_cast<float>(y[k]);
  if (!rates<NS, float>(m, rho, static_cast<float>(T), Yf, f)) rates_fp64_fallback<NS>(m, rho, T, y, f);
}

// Analytic Jacobian of dY/dt (FP32) at (rho, T, Y) with T = T(e, Y):
//   J_kj = (W_k / W_j) sum_r dnu_kr dq_r/dC_j  +  g_k dT/dY_j,
//   g_k = (W_k / rho) sum_r dnu_kr dq_r/dT,  dT/dY_j = -u_j / c_v.
// Row-major NS x NS into J (registers of the caller).
template <int NS>
__device__ __forceinline__ void jacobian(const MechView& m, float rho, float T, const float* Y, float cvR,
                                         float (&J)[NS][NS]) {
  KinState<NS, float> s;
  kin_prepare<NS, float>(m, rho, T, Y, s);
  float invC[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) invC[k] = s.C[k] > 1e-30f ? 1.0f / s.C[k] : 0.0f;
  float g[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    g[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < NS; ++j) J[k][j] = 0.0f;
  }
  const float T2 = T * T;
#pragma unroll 1
  for (int r = 0; r < m.nr; ++r) {
    float lnkf, lnqf, lnqr;
    bool rev;
    log_rates<NS, float>(m, s, T, r, lnkf, lnqf, lnqr, rev);
    lnqf = fminf(lnqf, kLnQMax);
    lnqr = fminf(lnqr, kLnQMax);
    const float qf = __expf(lnqf), qr = __expf(lnqr);
    const float4 a = m.arr[r];
    const float dlnkf = (a.y + a.z * s.invT) * s.invT;
    float dlnKc = 0.0f;
    if (rev) {
      const float* hc = m.hco + (s.reg * m.nr + r) * 8;
      const float dH = hc[0] + T * (hc[1] + T * hc[2] + T2 * (hc[3] + T * hc[4])) + hc[5] * s.invT;
      dlnKc = (dH - a.w) * s.invT;
    }
    float M = 1.0f;
    const int tb = (m.rinfo[r] >> 8) - 1;
    const float* ef = m.eff + (tb >= 0 ? tb : 0) * m.nsp;
    if (tb >= 0) {
      M = 0.0f;
#pragma unroll
      for (int k = 0; k < NS; ++k) M += ef[k] * fmaxf(s.C[k], 0.0f);
    }
    const float dqdT = M * (qf * dlnkf - qr * (dlnkf - dlnKc));
    const float* nf = m.nuf + r * m.nsp;
    const float* nb = m.nur + r * m.nsp;
    const float* dn = m.dnu + r * m.nsp;
    float D[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      float d;
      if (invC[j] != 0.0f) {
        d = (nf[j] * qf - nb[j] * qr) * invC[j];
      } else {   // C_j ~ 0: the derivative of C_j^1 * (others) is (others) = q / C_j in log form
        d = (nf[j] != 0.0f ? nf[j] * __expf(fminf(lnqf - s.lnC[j], kLnQMax)) : 0.0f) -
            (nb[j] != 0.0f ? nb[j] * __expf(fminf(lnqr - s.lnC[j], kLnQMax)) : 0.0f);
      }
      D[j] = M * d + (tb >= 0 ? ef[j] * (qf - qr) : 0.0f);
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float dk = dn[k];
      if (dk != 0.0f) {
        g[k] += dk * dqdT;
#pragma unroll
        for (int j = 0; j < NS; ++j) J[k][j] += dk * D[j];
      }
    }
  }
  // temperature column: u_j = R T (h_j/RT - 1) / W_j, dT/dY_j = -u_j / c_v
  const float* hs = m.hsp + s.reg * NS * 8;
  const float irho = 1.0f / rho;
  const float icv = 1.0f / cvR;   // c_v / R -> u/R / (c_v/R)
  float dTdY[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const float* h = hs + j * 8;
    const float hRT = h[0] + T * (h[1] + T * h[2] + T2 * (h[3] + T * h[4])) + h[5] * s.invT;
    dTdY[j] = -(T * (hRT - 1.0f) * m.invW[j]) * icv;
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const float Wk = m.W[k];
    const float gk = g[k] * Wk * irho;
#pragma unroll
    for (int j = 0; j < NS; ++j) J[k][j] = J[k][j] * Wk * m.invW[j] + gk * dTdY[j];
  }
}

}  // namespace chem
