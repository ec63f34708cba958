// large.cu -- the bulk-sparse integration for mechanisms too large for one thread per cell
// (the 53-species / 325-reaction hydrocarbon-shaped mechanism): one warp per cell.
//
// Same method as bulk.cu / stiff.cu (Eq. 5 closed by T(e); Algorithm 3: a bulk Heun step with an
// error test for every cell, compaction of the failures, SDIRK3 with simplified Newton on the
// dense Jacobian and an FP64 LU for them), laid out for a warp:
//   * the mechanism is sparse (<= 3 reactant and <= 3 product species per reaction, packed 9 bits
//     each) with a species -> (reaction, dnu) index, so the staged tables take ~40 KB of shared
//     memory (the per-reaction thermo coefficients stay in global memory, cached in L1);
//   * a cell's state is spread over the lanes (species k on lane k mod 32); rates are computed
//     lane-parallel over reactions into a per-warp array of rates of progress, then reduced per
//     species over that species' reactions in a fixed order (deterministic, no atomics);
//   * the Jacobian rows are built the same way (lane k owns row k), converted to the FP64 iteration
//     matrix I - gamma h J in per-warp shared memory, factored by the warp with partial pivoting
//     (warp argmax, lane-owned columns in the rank-1 updates) and solved with column sweeps;
//   * T(e) reduces the mixture coefficients over the lanes in FP64 and runs the scalar Newton
//     identically on every lane, so all control flow of a warp is uniform.
// Every scalar decision (convergence, step acceptance) derives from warp-reduced values.
#include <cstdio>

#include "../../include/chem.h"
#include "chem_device.cuh"
#include "internal.h"

namespace chem {
namespace lg {

// cells in flight per CTA of the stiff kernel: as many warps as the shared memory holds (7 for
// the 53-species tables), at most this many
constexpr int kStiffWarpsMax = 8;
constexpr int kBulkWarps = 8;    // cells in flight per CTA of the bulk kernel
constexpr int kNewtMax = 6;
constexpr double kNewtTol = 0.03;
// reuse of the factored iteration matrix across steps (stiff_kernel_lg): hold h while the
// controller's growth factor is within [1, kHoldMax] and the Newton contraction estimate
// eta = theta / (1 - theta) is at most kEtaReuse, for at most kLuMaxAge steps per factorisation
constexpr double kHoldMax = 1.2;
constexpr double kEtaReuse = 0.1;
constexpr int kLuMaxAge = 16;
// Alexander's L-stable DIRK3 (as in stiff.cu)
constexpr double kG = 0.43586652150845895;
constexpr double kA21 = 0.5 * (1.0 - kG);
constexpr double kB1 = 1.2084966491760099;
constexpr double kB2 = -0.6443631706844688;
constexpr double kBh1 = 0.7726301276675509;
constexpr double kBh2 = 0.2273698723324491;
constexpr double kC2 = 0.5 * (1.0 + kG);

__device__ __forceinline__ int sto_sp(int packed, int s) { return (packed >> (9 * s)) & 127; }
__device__ __forceinline__ int sto_c(int packed, int s) { return (packed >> (9 * s + 7)) & 3; }

struct LView {
  int ns, nr, ntb, nsp;
  float T_lo, T_hi, lnP0R;
  const float4* arr;    // [nr] lnA, b, Ea/R, sum dnu
  const int* rinfo;     // [nr] bit 0 reversible, (third-body row + 1) << 8
  const float* W;
  const float* invW;
  const float* eff;     // [ntb][nsp]
  const float* hsp;     // [3][ns][8] species h/RT coefficients
  const int2* sto;      // [nr] packed reactants, products (global memory)
  const int* cptr;      // [ns + 1]
  const int* cent;      // [nnz] reaction | dnu << 16
  const float* gamg;    // [3][nr][8] all regimes (global memory)
  const float* hcog;
  MechView mv;          // e64 (global memory) and the fit range for the temperature inversion
};

__device__ __forceinline__ LView make_lview(const unsigned char* sm, const unsigned char* gl) {
  const MechHdr* h = reinterpret_cast<const MechHdr*>(sm);
  LView v;
  v.ns = h->ns;
  v.nr = h->nr;
  v.ntb = h->ntb;
  v.nsp = h->nsp;
  v.T_lo = h->T_lo;
  v.T_hi = h->T_hi;
  v.lnP0R = h->lnP0R;
  v.arr = reinterpret_cast<const float4*>(sm + h->off_arr);
  v.rinfo = reinterpret_cast<const int*>(sm + h->off_rinfo);
  v.W = reinterpret_cast<const float*>(sm + h->off_W);
  v.invW = reinterpret_cast<const float*>(sm + h->off_invW);
  v.eff = reinterpret_cast<const float*>(sm + h->off_eff);
  v.hsp = reinterpret_cast<const float*>(sm + h->off_hsp);
  v.sto = reinterpret_cast<const int2*>(gl + h->off_sto);
  v.cptr = reinterpret_cast<const int*>(sm + h->off_cptr);
  v.cent = reinterpret_cast<const int*>(sm + h->off_cent);
  v.gamg = reinterpret_cast<const float*>(gl + h->off_gamg);
  v.hcog = reinterpret_cast<const float*>(gl + h->off_hcog);
  v.mv = make_view(sm);
  v.mv.e64 = reinterpret_cast<const double*>(gl + h->off_e64);
  return v;
}

// per-reaction Gibbs / enthalpy coefficients (global, read through L1)
__device__ __forceinline__ const float* gam_of(const LView& m, int reg, int r) { return m.gamg + (reg * m.nr + r) * 8; }
__device__ __forceinline__ const float* hco_of(const LView& m, int reg, int r) { return m.hcog + (reg * m.nr + r) * 8; }

// ---- per-warp scratch in shared memory.  J holds the rates of progress; in the stiff layout M
// holds the FP64 iteration matrix and its factors, and while the Jacobian is built, the FP32
// Jacobian in its first half and the per-reaction slopes behind it (the matrix is widened to FP64
// in place afterwards).
__host__ __device__ inline unsigned jac_slopes_offset(int ns) { return 4u * ((ns * ns + 3u) & ~3u); }
struct ScratchLayout {
  unsigned C, lnC, dT, Mtb, piv, v, J, M, bytes;
};
__host__ __device__ inline ScratchLayout scratch_layout(int ns, int nr, int ntb, bool stiff, int na = 0) {
  ScratchLayout l;
  const unsigned nsp = (ns + 3) & ~3;
  const unsigned mtb = ((ntb > 0 ? ntb : 1) + 3) & ~3;
  l.C = 0;
  l.lnC = l.C + 4 * nsp;
  l.dT = l.lnC + 4 * nsp;
  l.Mtb = l.dT + 4 * nsp;
  l.piv = l.Mtb + 4 * mtb;
  l.v = (l.piv + 4 * nsp + 15) & ~15u;
  l.J = l.v + 8 * nsp;
  const unsigned jb = 8u * nr;   // rates of progress (FP64 at most)
  l.M = (l.J + jb + 15) & ~15u;
  unsigned mb = 0;
  if (stiff) {
    // the leading na x na block (na: species before the trailing inert ones) with row stride na
    const int nj = na > 0 ? na : ns;
    mb = 8u * nj * nj;
    // FP32 Jacobian, then per reaction 6 slopes, dq/dT and qf - qr
    const unsigned jac = jac_slopes_offset(nj) + 4u * 8 * nr;
    if (jac > mb) mb = jac;
  }
  l.bytes = (l.M + mb + 127) & ~127u;
  return l;
}

struct Scratch {
  float* C;
  float* lnC;
  float* dT;
  float* Mtb;
  int* piv;
  double* v;
  float* J;
  double* M;
};

__device__ __forceinline__ Scratch make_scratch(unsigned char* base, const ScratchLayout& l) {
  Scratch s;
  s.C = reinterpret_cast<float*>(base + l.C);
  s.lnC = reinterpret_cast<float*>(base + l.lnC);
  s.dT = reinterpret_cast<float*>(base + l.dT);
  s.Mtb = reinterpret_cast<float*>(base + l.Mtb);
  s.piv = reinterpret_cast<int*>(base + l.piv);
  s.v = reinterpret_cast<double*>(base + l.v);
  s.J = reinterpret_cast<float*>(base + l.J);
  s.M = reinterpret_cast<double*>(base + l.M);
  return s;
}

// ---- warp reductions
__device__ __forceinline__ float wsum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double wsum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ float wmax(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// ---- temperature from internal energy: lanes reduce the FP64 mixture coefficients, every lane
// runs the same scalar Newton iteration (bisection safeguard), as temperature_from_energy does.
// The six sums over the warp: each of the first three butterfly levels halves the values a lane
// carries (it keeps one half and hands its partner the other), so a lane does 4 + 2 + 1 + 1 + 1
// FP64 additions instead of 6 x 5; lane l ends with the sum of value 4 b4 + 2 b3 + b2 (bits 4, 3
// and 2 of l; values 6 and 7 are zero padding), and six broadcasts hand the sums to every lane.
// Newton iterates stop at tol = 1e-5 T (their temperatures only feed the FP32 rates: the last
// step leaves T within ~1e-11 of the root), accepted states at 3e-8 T.
constexpr double kTeIterateTol = 1e-5;
constexpr double kTeStateTol = 3e-8;

template <int NS, typename Y_t>
__device__ double warp_temperature(const LView& m, const Y_t (&y)[2], double e0, double T, bool* ok,
                                   double* cv_out = nullptr, double tol = kTeStateTol) {
  const int lane = threadIdx.x & 31;
  const double eR = e0 * (1.0 / kR);
  double lo = kTbrLo, hi = kTbrHi;
  if (!(T > lo && T < hi)) T = 1000.0;
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
  auto mixture = [&](int reg, double (&E)[6], double (&D)[4]) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.0;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = lane + 32 * kk;
      if (k < NS) {
        const double* c = m.mv.e64 + (reg * NS + k) * 8;
        const double yk = static_cast<double>(y[kk]);
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = fma(yk, c[j], v[j]);
      }
    }
    double w4[4], w2[2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      w4[i] = (b4 ? v[4 + i] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[4 + i], 16);
#pragma unroll
    for (int i = 0; i < 2; ++i)
      w2[i] = (b3 ? w4[2 + i] : w4[i]) + __shfl_xor_sync(0xffffffffu, b3 ? w4[i] : w4[2 + i], 8);
    double w = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? w2[0] : w2[1], 4);
    w += __shfl_xor_sync(0xffffffffu, w, 2);
    w += __shfl_xor_sync(0xffffffffu, w, 1);
#pragma unroll
    for (int j = 0; j < 6; ++j) E[j] = __shfl_sync(0xffffffffu, w, ((j & 4) << 2) | ((j & 2) << 2) | ((j & 1) << 2));
    D[0] = 2.0 * E[2];
    D[1] = 3.0 * E[3];
    D[2] = 4.0 * E[4];
    D[3] = 5.0 * E[5];
  };
  int reg = regime_of(static_cast<float>(T), m.T_lo, m.T_hi);
  double E[6], D[4];   // D: the coefficients of de/dT, once per regime
  mixture(reg, E, D);
  double cv = 0.0;
  bool conv = false;
#pragma unroll 1
  for (int it = 0; it < 60; ++it) {
    const double f = fma(T, fma(T, fma(T, fma(T, fma(T, E[5], E[4]), E[3]), E[2]), E[1]), E[0]) - eR;
    cv = fma(T, fma(T, fma(T, fma(T, D[3], D[2]), D[1]), D[0]), E[1]);
    if (f > 0.0) hi = T; else lo = T;
    double Tn = (cv > 0.0) ? T - f * static_cast<double>(__frcp_rn(static_cast<float>(cv))) : 0.5 * (lo + hi);
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    const double dT = Tn - T;
    T = Tn;
    const int nreg = regime_of(static_cast<float>(T), m.T_lo, m.T_hi);
    if (nreg != reg) {
      reg = nreg;
      mixture(reg, E, D);
      continue;
    }
    if (fabs(dT) <= tol * T) {
      conv = true;
      break;
    }
  }
  if (cv_out) *cv_out = cv;
  *ok = conv && (T > kTbrLo) && (T < kTbrHi);
  return T;
}

// concentrations, their logarithms and the third-body sums into the warp's scratch
template <int NS>
__device__ __forceinline__ void kin_prepare_warp(const LView& m, const Scratch& s, float rho, const float (&Yl)[2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k = lane + 32 * kk;
    if (k < NS) {
      const float C = rho * Yl[kk] * m.invW[k];
      s.C[k] = C;
      s.lnC[k] = C > 0.0f ? __logf(C) : kLnZero;
    }
  }
  __syncwarp();
  for (int tb = lane; tb < m.ntb; tb += 32) {
    const float* ef = m.eff + tb * m.nsp;
    float M = 0.0f;
#pragma unroll 4
    for (int k = 0; k < NS; ++k) M = fmaf(ef[k], fmaxf(s.C[k], 0.0f), M);
    s.Mtb[tb] = M;
  }
  __syncwarp();
}

// ln k_f, ln q_f, ln q_r of reaction r (third-body factor excluded)
__device__ __forceinline__ void log_rates_lg(const LView& m, const Scratch& s, float lnT, float invT, float lnP0RT,
                                             float T, int reg, int r, float& lnkf, float& lnqf, float& lnqr,
                                             bool& rev) {
  const float4 a = m.arr[r];
  lnkf = a.x + a.y * lnT - a.z * invT;
  const int2 st = m.sto[r];
  float sf = 0.0f, sr = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int cf = sto_c(st.x, j), cr = sto_c(st.y, j);
    if (cf) sf = fmaf(static_cast<float>(cf), s.lnC[sto_sp(st.x, j)], sf);
    if (cr) sr = fmaf(static_cast<float>(cr), s.lnC[sto_sp(st.y, j)], sr);
  }
  lnqf = lnkf + sf;
  rev = (m.rinfo[r] & 1) != 0;
  lnqr = kLnZero;
  if (rev) {
    const float* g = gam_of(m, reg, r);
    const float T2 = T * T;
    const float dG = g[0] * (1.0f - lnT) + T * (g[1] + T * g[2] + T2 * (g[3] + T * g[4])) + g[5] * invT + g[6];
    const float lnKc = -dG + a.w * lnP0RT;
    lnqr = lnkf - lnKc + sr;
  }
}

// dY/dt of Eq. 5 for the warp's cell; rates of progress in precision Q (float, or double when
// a float log-rate would overflow exp).  Yl / fl: this lane's species lane and lane + 32.
template <int NS, typename Q>
__device__ bool warp_rates(const LView& m, const Scratch& s, float rho, float T, const float (&Yl)[2], float (&fl)[2]) {
  const int lane = threadIdx.x & 31;
  kin_prepare_warp<NS>(m, s, rho, Yl);
  const float lnT = __logf(T), invT = 1.0f / T;
  const float lnP0RT = m.lnP0R - lnT;
  const int reg = regime_of(T, m.T_lo, m.T_hi);
  Q* q = reinterpret_cast<Q*>(s.J);
  bool fine = true;
  for (int r = lane; r < m.nr; r += 32) {
    float lnkf, lnqf, lnqr;
    bool rev;
    log_rates_lg(m, s, lnT, invT, lnP0RT, T, reg, r, lnkf, lnqf, lnqr, rev);
    Q qv;
    if (sizeof(Q) == 4) {
      fine &= (lnqf < kLnQMax) & (lnqr < kLnQMax);
      qv = static_cast<Q>(__expf(lnqf) - __expf(lnqr));
    } else {
      qv = static_cast<Q>(exp(static_cast<double>(lnqf)) - exp(static_cast<double>(lnqr)));
    }
    const int tb = (m.rinfo[r] >> 8) - 1;
    if (tb >= 0) qv *= static_cast<Q>(s.Mtb[tb]);
    q[r] = qv;
  }
  fine = __all_sync(0xffffffffu, fine);
  __syncwarp();
  if (fine) {
    const Q irho = static_cast<Q>(1) / static_cast<Q>(rho);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = lane + 32 * kk;
      fl[kk] = 0.0f;
      if (k < NS) {
        Q w = 0;
        for (int e = m.cptr[k]; e < m.cptr[k + 1]; ++e) {
          const int ent = m.cent[e];
          w += static_cast<Q>(ent >> 16) * q[ent & 0xFFFF];
        }
        fl[kk] = static_cast<float>(w * static_cast<Q>(m.W[k]) * irho);
      }
    }
  }
  __syncwarp();   // q lives in the Jacobian area
  return fine;
}

template <int NS>
__device__ __forceinline__ void warp_rates_safe(const LView& m, const Scratch& s, float rho, float T,
                                                const float (&Yl)[2], float (&fl)[2]) {
  if (!warp_rates<NS, float>(m, s, rho, T, Yl, fl)) warp_rates<NS, double>(m, s, rho, T, Yl, fl);
}

// Analytic FP32 Jacobian of dY/dt with T eliminated (dT/dY_j = -u_j / c_v), row k on lane k mod 32,
// its leading na x na block (the rows and columns of the non-inert species; row stride na) as FP32
// at the start of the matrix area (the factors of the previous matrix are overwritten).  Per reaction the lanes store the slopes dq/dC_j of its (<= 6) species, dq/dT and
// qf - qr (third-body rows) behind it; each row then sums its reactions in order.
template <int NS>
__device__ void warp_jacobian(const LView& m, const Scratch& s, float rho, float T, const float (&Yl)[2], float cvR) {
  const int lane = threadIdx.x & 31;
  kin_prepare_warp<NS>(m, s, rho, Yl);
  const float lnT = __logf(T), invT = 1.0f / T;
  const float lnP0RT = m.lnP0R - lnT;
  const int reg = regime_of(T, m.T_lo, m.T_hi);
  const float T2 = T * T;
  float* const Jf = reinterpret_cast<float*>(s.M);                                  // [NS][NS]
  const int na = m.mv.nact;
  float* D = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s.M) + jac_slopes_offset(na));   // [nr][6]
  float* dqT = D + 6 * m.nr;                  // [nr]
  float* qd = dqT + m.nr;                     // [nr]
  for (int r = lane; r < m.nr; r += 32) {
    float lnkf, lnqf, lnqr;
    bool rev;
    log_rates_lg(m, s, lnT, invT, lnP0RT, T, reg, r, lnkf, lnqf, lnqr, rev);
    lnqf = fminf(lnqf, kLnQMax);
    lnqr = fminf(lnqr, kLnQMax);
    const float qf = __expf(lnqf), qr = rev ? __expf(lnqr) : 0.0f;
    const float4 a = m.arr[r];
    const float dlnkf = (a.y + a.z * invT) * invT;
    float dlnKc = 0.0f;
    if (rev) {
      const float* hc = hco_of(m, reg, r);
      const float dH = hc[0] + T * (hc[1] + T * hc[2] + T2 * (hc[3] + T * hc[4])) + hc[5] * invT;
      dlnKc = (dH - a.w) * invT;
    }
    const int tb = (m.rinfo[r] >> 8) - 1;
    const float Mf = tb >= 0 ? s.Mtb[tb] : 1.0f;
    dqT[r] = Mf * (qf * dlnkf - qr * (dlnkf - dlnKc));
    qd[r] = tb >= 0 ? qf - qr : 0.0f;
    const int2 st = m.sto[r];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // d(C^c * rest)/dC = c * C^(c-1) * rest = c * exp(ln q - ln C): also right at C -> 0
      const int cf = sto_c(st.x, j), cb = sto_c(st.y, j);
      D[r * 6 + j] = cf ? Mf * cf * __expf(fminf(lnqf - s.lnC[sto_sp(st.x, j)], kLnQMax)) : 0.0f;
      D[r * 6 + 3 + j] = (cb && rev) ? -Mf * cb * __expf(fminf(lnqr - s.lnC[sto_sp(st.y, j)], kLnQMax)) : 0.0f;
    }
  }
  // dT/dY_j = -u_j / c_v with u_j / R = T (h_j/RT - 1) / W_j
  const float icv = 1.0f / cvR;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int j = lane + 32 * kk;
    if (j < NS) {
      const float* h = m.hsp + (reg * NS + j) * 8;
      const float hRT = h[0] + T * (h[1] + T * h[2] + T2 * (h[3] + T * h[4])) + h[5] * invT;
      s.dT[j] = -(T * (hRT - 1.0f) * m.invW[j]) * icv;
    }
  }
  __syncwarp();
  const float irho = 1.0f / rho;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k = lane + 32 * kk;
    if (k < na) {
      float* Jk = Jf + k * na;
#pragma unroll 4
      for (int j = 0; j < na; ++j) Jk[j] = 0.0f;
      float g = 0.0f;
      for (int e = m.cptr[k]; e < m.cptr[k + 1]; ++e) {
        const int ent = m.cent[e];
        const int r = ent & 0xFFFF;
        const float dn = static_cast<float>(ent >> 16);
        g = fmaf(dn, dqT[r], g);
        const int2 st = m.sto[r];
#pragma unroll
        for (int j = 0; j < 3; ++j) {   // (an inert species' column is not kept)
          const int sf = sto_sp(st.x, j), sb = sto_sp(st.y, j);
          if (sto_c(st.x, j) && sf < na) Jk[sf] += dn * D[r * 6 + j];
          if (sto_c(st.y, j) && sb < na) Jk[sb] += dn * D[r * 6 + 3 + j];
        }
        const int tb = (m.rinfo[r] >> 8) - 1;
        if (tb >= 0) {   // d[M]/dC_j = eff_j: a dense row contribution
          const float dq = dn * qd[r];
          const float* ef = m.eff + tb * m.nsp;
#pragma unroll 4
          for (int j = 0; j < na; ++j) Jk[j] = fmaf(dq, ef[j], Jk[j]);
        }
      }
      const float Wk = m.W[k];
      const float gk = g * Wk * irho;
#pragma unroll 4
      for (int j = 0; j < na; ++j) Jk[j] = Jk[j] * Wk * m.invW[j] + gk * s.dT[j];
    }
  }
  __syncwarp();
}

// M = I - hh J (FP64, from the FP32 product as in stiff.cu), widened in place from the FP32
// Jacobian at the start of the same area.  Element idx is read at float offset idx and written at
// float offsets 2 idx and 2 idx + 1.  The warp walks the matrix from its end in chunks of 32
// elements: the chunk starting at c0 reads offsets [c0, c0 + 32) and then (after the __syncwarp)
// writes [2 c0, 2 c0 + 64), which lies above everything the chunks below still read ([0, c0)) and
// below what the chunks above wrote ([2 c0 + 64, ...)).  The widening is the exact integer-pipe
// conversion, and the identity is added to the diagonal afterwards (1 + v either way), so the
// walk issues no FP64 instruction.
template <int NS>
__device__ __forceinline__ void warp_iteration_matrix(const Scratch& s, double hh, int na) {
  const int lane = threadIdx.x & 31;
  const float mh = static_cast<float>(-hh);
  const float* Jf = reinterpret_cast<const float*>(s.M);
  const int n2 = na * na;
#pragma unroll 1
  for (int c0 = ((n2 - 1) / 32) * 32; c0 >= 0; c0 -= 32) {
    const int idx = c0 + lane;
    const float j = idx < n2 ? Jf[idx] : 0.0f;
    __syncwarp();
    if (idx < n2) s.M[idx] = f32_to_f64_exact(mh * j);
    __syncwarp();
  }
  for (int i = lane; i < na; i += 32) s.M[i * na + i] += 1.0;
  __syncwarp();
}

// LU with partial pivoting by the warp (unit-lower L; U stored as D^-1 U, unit upper, with the
// reciprocals D^-1 of its pivots on the diagonal; s.piv holds the composite row permutation: row
// k of the factors is row s.piv[k] of the original matrix).  Scaling U's rows once here lets every
// solve apply D^-1 to its right-hand side in one step instead of a one-lane multiply per row.
// Only the leading na x na block is factored: the trailing inert species (no reaction changes
// them) have identity rows, zero residuals and zero updates, so their rows and columns take no
// part in the solves, and their rows never win a pivot search before column na.
// Returns false (warp-uniform) for a singular matrix.
// |x| as an unsigned integer: for finite values it orders like |x|, so the pivot search compares
// integers instead of FP64 values and picks the same pivot
__device__ __forceinline__ unsigned long long abs_key64(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// 1 / x for a finite nonzero pivot: the hardware approximation (rcp.approx.ftz.f64, relative
// error below 2^-22 for normal x) and two Newton-Raphson steps r <- r + r (1 - x r), to within
// an ulp or two of the FP64 reciprocal, in four FMAs instead of a correctly rounded division
__device__ __forceinline__ double pivot_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

template <int NS>
__device__ bool warp_lu(const Scratch& s, int na) {
  const int lane = threadIdx.x & 31;
  double* M = s.M;
  for (int i = lane; i < NS; i += 32) s.piv[i] = i;
  __syncwarp();
#pragma unroll 1
  for (int k = 0; k < na; ++k) {
    // the pivot search on integer keys of |M_ik| (integer pipe instead of FP64 compares)
    unsigned long long best = 0ull;
    int p = NS;
    for (int i = k + lane; i < na; i += 32) {
      const unsigned long long v = abs_key64(M[i * na + k]);
      if (p == NS || v > best) {
        best = v;
        p = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (op < NS && (p == NS || ob > best || (ob == best && op < p))) {
        best = ob;
        p = op;
      }
    }
    // zero pivot or NaN: singular
    if (best == 0ull || best > 0x7ff0000000000000ull) return false;
    if (p != k) {
      if (lane == 0) {
        const int t = s.piv[k];
        s.piv[k] = s.piv[p];
        s.piv[p] = t;
      }
      for (int c = lane; c < na; c += 32) {
        const double t = M[k * na + c];
        M[k * na + c] = M[p * na + c];
        M[p * na + c] = t;
      }
    }
    __syncwarp();
    const double inv = pivot_rcp(M[k * na + k]);
    for (int i = k + 1 + lane; i < na; i += 32) M[i * na + k] *= inv;
    __syncwarp();
    // rank-1 update of the trailing m x m block, spread over the lanes element by element
    // (row-major order), so that all 32 lanes work until the block is smaller than the warp;
    // every element takes the same single FMA as in a column-per-lane sweep
    if (k < na - 1) {
      const int m = na - 1 - k;
      const int q = 32 / m, r = 32 - q * m;   // a stride of 32 elements: q rows and r columns
      int ii = lane / m, cc = lane - (lane / m) * m;
      for (int e = lane; e < m * m; e += 32) {
        const int i = k + 1 + ii, c = k + 1 + cc;
        M[i * na + c] = fma(-M[i * na + k], M[k * na + c], M[i * na + c]);
        ii += q;
        cc += r;
        if (cc >= m) {
          cc -= m;
          ++ii;
        }
      }
    }
    __syncwarp();
    if (lane == 0) M[k * na + k] = inv;
    __syncwarp();
  }
  // U -> D^-1 U: row i of the strict upper triangle times its pivot's reciprocal
#pragma unroll 1
  for (int i = 0; i < na - 1; ++i) {
    const double d = M[i * na + i];
    for (int c = i + 1 + lane; c < na; c += 32) M[i * na + c] *= d;
  }
  __syncwarp();
  return true;
}

// x = M^-1 b with the factors of warp_lu; b / x: this lane's entries lane and lane + 32 (the
// entries of the inert species na.. come back zero).  The permuted right-hand side is gathered
// through shared memory; the substitutions keep x in registers (up to two rows per lane) and
// broadcast each finished entry with a shuffle (column sweeps: unit-lower L forward, then the
// unit upper D^-1 U backward on D^-1 y).  With na > 32 each sweep lays its rows over the lanes so
// that the rows still to update at column j fill as few warp instructions as possible: forward,
// rows R.. (R = na - 32) on the first register and rows 0..R-1 on the second, so the first
// register's rows all lie below every column at which the second has any; backward, rows 0-31
// and 32-, so the first register's rows all lie above every column at which the second has any.
// Past that point a column takes one FP64 instruction instead of two, no FP64 instruction runs
// with every lane predicated off (it would still take its turn on the FP64 pipe), and every row
// takes its updates in the order of a plain column sweep.
template <int NS>
__device__ void warp_solve(const Scratch& s, double (&b)[2], int na) {
  static_assert(NS > 32 && NS <= 64, "two entries per lane");
  const int lane = threadIdx.x & 31;
  const double* M = s.M;
  double* v = s.v;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k = lane + 32 * kk;
    if (k < na) v[k] = b[kk];
  }
  __syncwarp();
  const int i0 = lane, i1 = lane + 32;
  double x[2];
  if (na <= 32) {   // one row per lane
    x[0] = i0 < na ? v[s.piv[i0]] : 0.0;
    __syncwarp();
#pragma unroll 1
    for (int j = 0; j < na - 1; ++j) {
      const double vj = __shfl_sync(0xffffffffu, x[0], j);
      if (i0 > j && i0 < na) x[0] = fma(-M[i0 * na + j], vj, x[0]);
    }
    if (i0 < na) x[0] *= M[i0 * na + i0];
#pragma unroll 1
    for (int j = na - 1; j >= 1; --j) {
      const double vj = __shfl_sync(0xffffffffu, x[0], j);
      if (i0 < j) x[0] = fma(-M[i0 * na + j], vj, x[0]);
    }
    b[0] = i0 < na ? x[0] : 0.0;
    b[1] = 0.0;
    return;
  }
  const int R = na - 32;
  const int f0 = R + lane, f1 = lane;   // forward layout
  x[0] = v[s.piv[f0]];
  x[1] = f1 < R ? v[s.piv[f1]] : 0.0;
  __syncwarp();
#pragma unroll 1
  for (int j = 0; j < R - 1; ++j) {   // rows below j on both registers (all of the first)
    const double vj = __shfl_sync(0xffffffffu, x[1], j);
    x[0] = fma(-M[f0 * na + j], vj, x[0]);
    if (f1 > j && f1 < R) x[1] = fma(-M[f1 * na + j], vj, x[1]);
  }
#pragma unroll 1
  for (int j = R - 1; j < na - 1; ++j) {   // rows below j only on the first register
    const double src = j < R ? x[1] : x[0];
    const double vj = __shfl_sync(0xffffffffu, src, j < R ? j : j - R);
    if (f0 > j) x[0] = fma(-M[f0 * na + j], vj, x[0]);
  }
  // to the backward layout through shared memory
  v[f0] = x[0];
  if (f1 < R) v[f1] = x[1];
  __syncwarp();
  x[0] = v[i0];
  x[1] = i1 < na ? v[i1] : 0.0;
  __syncwarp();
  x[0] *= M[i0 * na + i0];
  if (i1 < na) x[1] *= M[i1 * na + i1];
#pragma unroll 1
  for (int j = na - 1; j > 32; --j) {   // rows above j on both registers (all of the first)
    const double vj = __shfl_sync(0xffffffffu, x[1], j - 32);
    x[0] = fma(-M[i0 * na + j], vj, x[0]);
    if (i1 < j) x[1] = fma(-M[i1 * na + j], vj, x[1]);
  }
#pragma unroll 1
  for (int j = 32; j >= 1; --j) {   // rows above j only on the first register (none above row 0)
    const double src = j < 32 ? x[0] : x[1];
    const double vj = __shfl_sync(0xffffffffu, src, j & 31);
    if (i0 < j) x[0] = fma(-M[i0 * na + j], vj, x[0]);
  }
  b[0] = x[0];
  b[1] = i1 < na ? x[1] : 0.0;
}

struct CellCtx {
  float rho, rtol, atol;
  double e0;
};

// stage equation z = yb + hh f(z) by simplified Newton (as stage_newton in stiff.cu)
// known_T: the start iterate z is the step's initial state and Tz its temperature (inverted at the
// state tolerance), so the first iteration skips the inversion.
template <int NS>
__device__ bool warp_stage_newton(const LView& m, const Scratch& s, const CellCtx& c, const double (&yb)[2],
                                  double hh, double (&z)[2], double& Tz, float& eta, unsigned long long& n_it,
                                  bool known_T) {
  const int lane = threadIdx.x & 31;
  // the convergence control (norm, contraction rate) is FP32: it only decides when to stop
  float prev = 0.0f;
#pragma unroll 1
  for (int it = 0; it < kNewtMax; ++it) {
    ++n_it;
    if (it > 0 || !known_T) {
      bool ok;
      Tz = warp_temperature<NS>(m, z, c.e0, Tz, &ok, nullptr, kTeIterateTol);
      if (!ok) return false;
    }
    float Zf[2], F[2];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) Zf[kk] = static_cast<float>(z[kk]);
    warp_rates_safe<NS>(m, s, c.rho, static_cast<float>(Tz), Zf, F);
    const float mhh = static_cast<float>(hh);
    double b[2];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
      b[kk] = (lane + 32 * kk < NS) ? (yb[kk] - z[kk]) + static_cast<double>(mhh * F[kk]) : 0.0;
    warp_solve<NS>(s, b, m.mv.nact);
    float ss = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      if (lane + 32 * kk < NS) {
        z[kk] += b[kk];
        const float bf = static_cast<float>(b[kk]);
        const float w = c.atol + c.rtol * fabsf(Zf[kk] + bf);
        const float r = bf / w;
        ss = fmaf(r, r, ss);
      }
    }
    const float nrm = sqrtf(wsum(ss) * (1.0f / NS));
    if (!(nrm == nrm)) return false;
    if (it > 0) {
      const float theta = nrm / prev;
      if (theta >= 1.0f) return nrm <= 0.5f && theta < 2.0f;
      eta = theta / (1.0f - theta);
    }
    if (eta * nrm <= static_cast<float>(kNewtTol) || nrm <= 1e-3f) return true;
    prev = nrm;
  }
  return false;
}

// ------------------------------------------------------------------ bulk kernel (warp per cell)

template <int NS>
__global__ void __launch_bounds__(32 * kBulkWarps) bulk_kernel_lg(const AdvanceArgs<float> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, a.blob, a.blob_bytes, &bar, &a.ws->status)) return;
  const LView m = make_lview(smem, a.blob);
  const unsigned pre = (a.blob_bytes + 127u) & ~127u;
  int* soff = reinterpret_cast<int*>(smem + pre);
  if (a.nbox > 0) stage_box_offsets(soff, a.box_off, a.nbox);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ScratchLayout L = scratch_layout(NS, m.nr, m.ntb, false);
  const Scratch s = make_scratch(smem + pre + box_smem_bytes(a.nbox) + warp * L.bytes, L);
  unsigned long long c_skip = 0, c_bulk = 0, c_inv = 0;
  const int kb = a.prm.k_bulk;
  for (long long g = static_cast<long long>(blockIdx.x) * kBulkWarps + warp; g < a.n;
       g += static_cast<long long>(gridDim.x) * kBulkWarps) {
    if (a.skip && a.skip[g]) continue;
    const CellRef<float> cr = locate(a, soff, g);
    const long long i = cr.i;
    const double dt = cr.dt;
    const float h = static_cast<float>(dt / kb);
    const float rho = cr.rho[i], e = cr.e[i], T = cr.T[i];
    float y[2];
    bool valid = isfinite(rho) && rho > 0.0f && isfinite(e) && isfinite(T) && T > 0.0f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = lane + 32 * kk;
      y[kk] = k < NS ? cr.Y[k * cr.ld + i] : 0.0f;
      if (k < NS) valid = valid && isfinite(y[kk]) && y[kk] > -1e-6f;
    }
    valid = __all_sync(0xffffffffu, valid);
    if (!valid) {
      if (lane == 0) {
        cr.sub[i] = -1;
        ++c_inv;
      }
      continue;
    }
    if (T < a.prm.T_min) {
      if (lane == 0) {
        cr.sub[i] = 0;
        ++c_skip;
      }
      continue;
    }
    bool pass;
    float cost = 0.0f;
    double Tn = warp_temperature<NS>(m, y, static_cast<double>(e), static_cast<double>(T), &pass);
    for (int st = 0; st < kb && pass; ++st) {
      float f0[2], f1[2], y1[2];
      warp_rates_safe<NS>(m, s, rho, static_cast<float>(Tn), y, f0);
      float chg = 0.0f, c0 = 0.0f;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const float d = h * f0[kk];
        y1[kk] = y[kk] + d;
        c0 += fabsf(f0[kk]);
        if (lane + 32 * kk < NS) chg = fmaxf(chg, fabsf(d) / fmaxf(fabsf(y[kk]), a.prm.y_floor));
      }
      if (st == 0) cost = wsum(c0) * static_cast<float>(dt);
      chg = wmax(chg);
      bool ok1;
      const double T1 = warp_temperature<NS>(m, y1, static_cast<double>(e), Tn, &ok1);
      pass = pass && ok1;
      if (pass) warp_rates_safe<NS>(m, s, rho, static_cast<float>(T1), y1, f1);
      float err = 0.0f;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        if (lane + 32 * kk < NS && pass) {
          const float yh = y[kk] + 0.5f * h * (f0[kk] + f1[kk]);
          const float est = 0.5f * h * fabsf(f1[kk] - f0[kk]);
          const float w = a.prm.atol + a.prm.rtol * fmaxf(fabsf(y[kk]), fabsf(yh));
          err = fmaxf(err, est / w);
          y[kk] = yh;
        }
      }
      err = wmax(err);
      pass = pass && (err <= 1.0f) && (chg <= a.prm.bulk_frac);
      if (pass) {
        bool okT;
        Tn = warp_temperature<NS>(m, y, static_cast<double>(e), T1, &okT);
        pass = okT;
      }
    }
    if (pass) {
      double sw = 0.0;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int k = lane + 32 * kk;
        if (k < NS) {
          cr.Y[k * cr.ld + i] = y[kk];
          sw = fma(static_cast<double>(y[kk]), m.mv.e64[k * 8 + 6], sw);
        }
      }
      sw = wsum(sw);
      if (lane == 0) {
        cr.T[i] = static_cast<float>(Tn);
        if (cr.p) cr.p[i] = static_cast<float>(static_cast<double>(rho) * kR * Tn * sw);
        cr.sub[i] = kb;
        ++c_bulk;
      }
    } else if (lane == 0) {
      const int pos = atomicAdd(&a.ws->qcount, 1);
      a.queue[pos] = static_cast<int>(g);
      if (a.qkey) {
        const float lk = 2.0f * __log2f(fmaxf(cost, 1e-30f)) + 32.0f;
        a.qkey[pos] = static_cast<unsigned char>(fminf(fmaxf(lk, 0.0f), static_cast<float>(kNumBuckets - 1)));
      }
    }
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

// ------------------------------------------------------------------ stiff kernel (warp per cell)

template <int NS>
__global__ void __launch_bounds__(32 * kStiffWarpsMax, 1) stiff_kernel_lg(const AdvanceArgs<float> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, a.blob, a.blob_bytes, &bar, &a.ws->status)) return;
  const LView m = make_lview(smem, a.blob);
  const unsigned pre = (a.blob_bytes + 127u) & ~127u;
  int* soff = reinterpret_cast<int*>(smem + pre);
  if (a.nbox > 0) stage_box_offsets(soff, a.box_off, a.nbox);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ScratchLayout L = scratch_layout(NS, m.nr, m.ntb, true, m.mv.nact);
  const Scratch s = make_scratch(smem + pre + box_smem_bytes(a.nbox) + warp * L.bytes, L);
  const int qn = min(*reinterpret_cast<volatile int*>(&a.ws->qcount), static_cast<int>(a.n));
  CellCtx c;
  c.rtol = a.prm.rtol;
  c.atol = a.prm.atol;
  unsigned long long c_sub = 0, c_fail = 0, c_att = 0, c_newt = 0, c_lu = 0;
  int flags = 0;
  // every warp's first cell is queue position warp * gridDim.x + blockIdx.x (interleaved over
  // the CTAs, so that a queue shorter than the warp slots, ordered most expensive first, spreads
  // evenly over the SMs); later cells come from the shared counter, after those slots
  const int slots = static_cast<int>(gridDim.x) * static_cast<int>(blockDim.x >> 5);
  bool first = true;
#pragma unroll 1
  while (true) {
    int q = 0;
    if (first) {
      q = warp * static_cast<int>(gridDim.x) + static_cast<int>(blockIdx.x);
      first = false;
    } else {
      if (lane == 0) q = slots + atomicAdd(&a.ws->head, 1);
      q = __shfl_sync(0xffffffffu, q, 0);
    }
    if (q >= qn) break;
    const int cell = a.queue[q];
    double dt, y[2], Tc;
    float cvR;
    {
      const CellRef<float> cr = locate(a, soff, cell);
      const long long i = cr.i;
      dt = cr.dt;
      c.rho = cr.rho[i];
      c.e0 = static_cast<double>(cr.e[i]);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int k = lane + 32 * kk;
        y[kk] = k < NS ? static_cast<double>(cr.Y[k * cr.ld + i]) : 0.0;
      }
      bool ok;
      double cvd;
      Tc = warp_temperature<NS>(m, y, c.e0, static_cast<double>(cr.T[i]), &ok, &cvd);
      cvR = static_cast<float>(cvd);
      if (!ok) {
        if (lane == 0) {
          cr.sub[i] = -1;
          ++c_fail;
          flags |= kFlagTemp;
        }
        continue;
      }
    }
    double t = 0.0, h = 1e-6 * dt;
    float eta_cell = 1.0f;
    int nst = 0, natt = 0;
    bool finished = false, failed = false;
    // the factored iteration matrix of the last attempt, reused while the step size is held and
    // Newton keeps contracting fast (the 53 x 53 LU is most of an attempt's FP64 work)
    bool lu_valid = false;
    double h_lu = 0.0;
    int lu_age = 0;
#pragma unroll 1
    while (!finished && !failed) {
      ++natt;
      ++c_att;
      const double gh = kG * h;
      const bool reuse = lu_valid && h == h_lu && lu_age < kLuMaxAge;
      bool conv = true;
      if (reuse) {
        ++lu_age;
      } else {
        float Yf[2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) Yf[kk] = static_cast<float>(y[kk]);
        warp_jacobian<NS>(m, s, c.rho, static_cast<float>(Tc), Yf, cvR);
        warp_iteration_matrix<NS>(s, gh, m.mv.nact);
        conv = warp_lu<NS>(s, m.mv.nact);
        ++c_lu;
        lu_valid = conv;
        h_lu = h;
        lu_age = 0;
      }
      double hk1[2] = {0.0, 0.0}, hk2[2] = {0.0, 0.0}, z[2], base[2];
      double Tz = Tc;
      float eta = eta_cell;
#pragma unroll 1
      for (int st = 0; st < 3 && conv; ++st) {
        const double a1 = st == 1 ? kA21 : (st == 2 ? kB1 : 0.0);
        const double a2 = st == 2 ? kB2 : 0.0;
        const double p1 = st == 1 ? kC2 : (st == 2 ? kA21 / kC2 : 0.0);
        const double p2 = st == 2 ? kG / kC2 : 0.0;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          base[kk] = y[kk] + a1 * hk1[kk] + a2 * hk2[kk];
          z[kk] = y[kk] + p1 * hk1[kk] + p2 * hk2[kk];
        }
        conv = warp_stage_newton<NS>(m, s, c, base, gh, z, Tz, eta, c_newt, st == 0);
        if (st < 2) {
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const double hk = (z[kk] - base[kk]) * (1.0 / kG);
            if (st == 0) hk1[kk] = hk; else hk2[kk] = hk;
          }
        }
      }
      eta_cell = fmaxf(eta, 0.05f);
      if (!conv) {
        // Newton failed: with a reused (older) iteration matrix retry the same step with a fresh
        // Jacobian, otherwise shrink the step
        if (!reuse) h *= 0.25;
        lu_valid = false;
        eta_cell = 1.0f;
      } else {
        double er[2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const double hk3 = (z[kk] - base[kk]) * (1.0 / kG);
          er[kk] = (kB1 - kBh1) * hk1[kk] + (kB2 - kBh2) * hk2[kk] + kG * hk3;
        }
        warp_solve<NS>(s, er, m.mv.nact);
        // the weighted error norm is a step-size control quantity: FP32
        float errl = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          if (lane + 32 * kk < NS) {
            const float zk = static_cast<float>(z[kk]);
            const float w = c.atol + c.rtol * fmaxf(fabsf(static_cast<float>(y[kk])), fabsf(zk));
            errl = fmaxf(errl, fabsf(static_cast<float>(er[kk])) / w);
            // a clearly negative mass fraction rejects the step (see stiff.cu)
            if (zk < -10.0f * c.atol) errl = fmaxf(errl, 4.0f);
          }
        }
        float err = wmax(errl);
        if (err <= 1.0f) {
          bool ok;
          double cvd;
          const double Tn = warp_temperature<NS>(m, z, c.e0, Tz, &ok, &cvd);
          if (ok) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) y[kk] = z[kk];
            Tc = Tn;
            cvR = static_cast<float>(cvd);
            t += h;
            ++nst;
            if (t >= dt * (1.0 - 1e-12)) finished = true;
          } else {
            err = 4.0f;
          }
        }
        float fac = 0.9f * rcbrtf(fmaxf(err, 1e-12f));
        fac = fminf(5.0f, fmaxf(0.2f, fac));
        // hold the step size (and so the factored matrix) when the controller would grow it by at
        // most kHoldMax and Newton contracts fast; any other factor refactors at the next attempt
        if (!(err <= 1.0f && fac >= 1.0f && fac <= static_cast<float>(kHoldMax) && eta <= static_cast<float>(kEtaReuse)))
          h *= static_cast<double>(fac);
      }
      if (!finished) {
        if (t + h > dt) h = dt - t;
        if (h < 1e-24 * dt || h < 1e-30) {
          failed = true;
          flags |= kFlagNoConv;
        }
        if (nst >= a.prm.k_max || natt >= 4 * a.prm.k_max) {
          failed = true;
          flags |= kFlagMaxSteps;
        }
      }
    }
    const CellRef<float> cr = locate(a, soff, cell);
    const long long i = cr.i;
    if (finished) {
      double sw = 0.0;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int k = lane + 32 * kk;
        if (k < NS) {
          cr.Y[k * cr.ld + i] = static_cast<float>(y[kk]);
          sw = fma(y[kk], m.mv.e64[k * 8 + 6], sw);
        }
      }
      sw = wsum(sw);
      if (lane == 0) {
        cr.T[i] = static_cast<float>(Tc);
        if (cr.p) cr.p[i] = static_cast<float>(static_cast<double>(cr.rho[i]) * kR * Tc * sw);
        cr.sub[i] = a.prm.k_bulk + nst;
        c_sub += nst;
      }
    } else if (lane == 0) {
      cr.sub[i] = -1;
      ++c_fail;
    }
  }
  if (lane == 0) {
    if (c_att) atomicAdd(&a.ws->attempts, c_att);
    if (c_newt) atomicAdd(&a.ws->newton, c_newt);
    if (c_lu) atomicAdd(&a.ws->factorizations, c_lu);
    if (c_sub) atomicAdd(&a.ws->substeps, c_sub);
    if (c_fail) atomicAdd(&a.ws->nfailed, c_fail);
    if (flags) atomicOr(&a.ws->status, flags);
  }
}

// dY/dt for the chem_rates helper (one warp per cell)
template <int NS>
__global__ void __launch_bounds__(32 * kBulkWarps) rates_kernel_lg(const unsigned char* blob, unsigned bytes,
                                                                    const float* rho, const float* T, const float* Y,
                                                                    long long ld, long long n, float* dYdt,
                                                                    int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar;
  if (!stage_to_smem(smem, blob, bytes, &bar, status)) return;
  const LView m = make_lview(smem, blob);
  const unsigned pre = (bytes + 127u) & ~127u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ScratchLayout L = scratch_layout(NS, m.nr, m.ntb, false);
  const Scratch s = make_scratch(smem + pre + warp * L.bytes, L);
  for (long long i = static_cast<long long>(blockIdx.x) * kBulkWarps + warp; i < n;
       i += static_cast<long long>(gridDim.x) * kBulkWarps) {
    float y[2], f[2];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = lane + 32 * kk;
      y[kk] = k < NS ? Y[k * ld + i] : 0.0f;
    }
    warp_rates_safe<NS>(m, s, rho[i], T[i], y, f);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = lane + 32 * kk;
      if (k < NS) dYdt[k * ld + i] = f[kk];
    }
  }
}

}  // namespace lg

// ------------------------------------------------------------------ launchers (ns = 53)

#define CHEM_FOR_EACH_NS_LARGE(X) X(53)

static unsigned pad128(unsigned b) { return (b + 127u) & ~127u; }

size_t bulk_smem_bytes_lg(int ns, int nr, int ntb, unsigned prefix, int nbox) {
  return pad128(prefix) + box_smem_bytes(nbox) + lg::kBulkWarps * lg::scratch_layout(ns, nr, ntb, false).bytes;
}
size_t stiff_smem_bytes_lg(int ns, int na, int nr, int ntb, unsigned prefix, int nbox, int warps) {
  return pad128(prefix) + box_smem_bytes(nbox) + warps * lg::scratch_layout(ns, nr, ntb, true, na).bytes;
}

// Warps per CTA of the stiff kernel: as many per-warp scratch areas as fit next to the staged
// tables in the device's opt-in shared memory per block (1 KB kept for the kernel's static shared
// memory), between 1 and kStiffWarpsMax.
static int stiff_warps_lg(int ns, int na, int nr, int ntb, unsigned prefix, int nbox) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 1;
  const long long room = static_cast<long long>(optin) - 1024 -
                         static_cast<long long>(stiff_smem_bytes_lg(ns, na, nr, ntb, prefix, nbox, 0));
  const long long w = room / static_cast<long long>(lg::scratch_layout(ns, nr, ntb, true, na).bytes);
  return w < 1 ? 1 : (w > lg::kStiffWarpsMax ? lg::kStiffWarpsMax : static_cast<int>(w));
}

int launch_bulk_lg(int ns, int nr, int ntb, const AdvanceArgs<float>& a, int grid, cudaStream_t s) {
#define X(N)                                                                                     \
  if (ns == N) {                                                                                 \
    const size_t smem = bulk_smem_bytes_lg(N, nr, ntb, a.blob_bytes, a.nbox);                    \
    cudaFuncSetAttribute(lg::bulk_kernel_lg<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                         static_cast<int>(smem));                                                \
    lg::bulk_kernel_lg<N><<<grid, 32 * lg::kBulkWarps, smem, s>>>(a);                            \
    return static_cast<int>(cudaGetLastError());                                                 \
  }
  CHEM_FOR_EACH_NS_LARGE(X)
#undef X
  return -1;
}

int launch_stiff_lg(int ns, int na, int nr, int ntb, const AdvanceArgs<float>& a, int grid, cudaStream_t s) {
#define X(N)                                                                                     \
  if (ns == N) {                                                                                 \
    const int w = stiff_warps_lg(N, na, nr, ntb, a.blob_bytes, a.nbox);                          \
    const size_t smem = stiff_smem_bytes_lg(N, na, nr, ntb, a.blob_bytes, a.nbox, w);            \
    cudaFuncSetAttribute(lg::stiff_kernel_lg<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                         static_cast<int>(smem));                                                \
    lg::stiff_kernel_lg<N><<<grid, 32 * w, smem, s>>>(a);                                        \
    return static_cast<int>(cudaGetLastError());                                                 \
  }
  CHEM_FOR_EACH_NS_LARGE(X)
#undef X
  return -1;
}

int launch_rates_lg(int ns, int nr, int ntb, const unsigned char* blob, unsigned bytes, const float* rho,
                    const float* T, const float* Y, long long ld, long long n, float* dYdt, int* status,
                    cudaStream_t s) {
#define X(N)                                                                                          \
  if (ns == N) {                                                                                      \
    const size_t smem = pad128(bytes) + lg::kBulkWarps * lg::scratch_layout(N, nr, ntb, false).bytes; \
    cudaFuncSetAttribute(lg::rates_kernel_lg<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                         static_cast<int>(smem));                                                     \
    long long blocks = (n + lg::kBulkWarps - 1) / lg::kBulkWarps;                                     \
    if (blocks > 4096) blocks = 4096;                                                                 \
    lg::rates_kernel_lg<N><<<static_cast<int>(blocks), 32 * lg::kBulkWarps, smem, s>>>(               \
        blob, bytes, rho, T, Y, ld, n, dYdt, status);                                                 \
    return static_cast<int>(cudaGetLastError());                                                      \
  }
  CHEM_FOR_EACH_NS_LARGE(X)
#undef X
  return -1;
}

int occupancy_lg(int ns, int na, int nr, int ntb, unsigned prefix, bool stiff, int* blocks_per_sm) {
#define X(N)                                                                                          \
  if (ns == N) {                                                                                      \
    if (stiff) {                                                                                      \
      const int w = stiff_warps_lg(N, na, nr, ntb, prefix, 0);                                        \
      const size_t smem = stiff_smem_bytes_lg(N, na, nr, ntb, prefix, 0, w);                          \
      cudaFuncSetAttribute(lg::stiff_kernel_lg<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                           static_cast<int>(smem));                                                   \
      return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(                          \
          blocks_per_sm, lg::stiff_kernel_lg<N>, 32 * w, smem));                                      \
    }                                                                                                 \
    const size_t smem = bulk_smem_bytes_lg(N, nr, ntb, prefix, 0);                                    \
    cudaFuncSetAttribute(lg::bulk_kernel_lg<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                         static_cast<int>(smem));                                                     \
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(                            \
        blocks_per_sm, lg::bulk_kernel_lg<N>, 32 * lg::kBulkWarps, smem));                            \
  }
  CHEM_FOR_EACH_NS_LARGE(X)
#undef X
  return -1;
}

bool compiled_large(int ns) {
#define X(N) \
  if (ns == N) return true;
  CHEM_FOR_EACH_NS_LARGE(X)
#undef X
  return false;
}

}  // namespace chem
