// pack.cu -- host-side checks of a mechanism and of the integration parameters, and the packing
// of the mechanism into the device table layout of chem_device.cuh (MechHdr).  Shared by
// chem_init (abi.cu) and chem_advance_noalloc (noalloc.cu), so both entry points accept the same
// inputs and the kernels see the same tables.  The dense layout allocates nothing on the host.
#include <cmath>
#include <cstring>
#include <vector>

#include "chem_device.cuh"
#include "internal.h"

namespace chem {

namespace {

unsigned align16(unsigned x) { return (x + 15u) & ~15u; }

// Table layout of m: every offset of the header and the total byte count (h.bytes).
MechHdr layout(const chem_mechanism* m, bool large) {
  const int ns = m->ns, nr = m->nr;
  const int nsp = (ns + 3) & ~3;
  int ntb = 0;
  for (int r = 0; r < nr; ++r) ntb += m->third_body[r] ? 1 : 0;
  int nnz = 0;
  for (int r = 0; r < nr; ++r)
    for (int k = 0; k < ns; ++k) nnz += (m->nu_r[r * ns + k] != m->nu_f[r * ns + k]) ? 1 : 0;
  MechHdr h{};
  h.ns = ns;
  h.nr = nr;
  h.ntb = ntb;
  h.nsp = nsp;
  h.large = large ? 1 : 0;
  h.nnz = nnz;
  // trailing species that no reaction changes (a bath gas such as N2): the stiff kernel leaves
  // them out of the Newton linear algebra, where their rows are those of the identity
  int nact = ns;
  while (nact > 1) {
    bool inert = true;
    for (int r = 0; r < nr && inert; ++r) inert = m->nu_r[r * ns + nact - 1] == m->nu_f[r * ns + nact - 1];
    if (!inert) break;
    --nact;
  }
  h.nact = nact;
  h.T_lo = static_cast<float>(m->thermo[7]);
  h.T_hi = static_cast<float>(m->thermo[8]);
  h.lnP0R = static_cast<float>(std::log(kP0 / kR));
  const int nreg = large ? 0 : 3;   // regimes of gam / hco in the staged part (large: none, all global)
  unsigned off = align16(sizeof(MechHdr));
  h.off_arr = off; off = align16(off + 16u * nr);
  if (!large) {
    h.off_nuf = off; off = align16(off + 4u * nr * nsp);
    h.off_nur = off; off = align16(off + 4u * nr * nsp);
    h.off_dnu = off; off = align16(off + 4u * nr * nsp);
  }
  h.off_eff = off; off = align16(off + 4u * (ntb > 0 ? ntb : 1) * nsp);
  h.off_rinfo = off; off = align16(off + 4u * nr);
  h.off_W = off; off = align16(off + 4u * nsp);
  h.off_invW = off; off = align16(off + 4u * nsp);
  h.off_gam = off; off = align16(off + 4u * nreg * nr * 8);
  h.off_hco = off; off = align16(off + 4u * nreg * nr * 8);
  h.off_hsp = off; off = align16(off + 4u * 3 * ns * 8);
  if (!large) {
    h.off_e64 = off; off = align16(off + 8u * 3 * ns * 8);
    h.off_arr64 = off; off = align16(off + 8u * 4 * nr);
    h.off_gam64 = off; off = align16(off + 8u * 3 * nr * 8);
    h.off_eff64 = off; off = align16(off + 8u * (ntb > 0 ? ntb : 1) * nsp);
    h.prefix = off;
  } else {
    // staged: the species -> reaction index; global tail (read through L1): the per-reaction
    // Gibbs / enthalpy coefficients, the FP64 thermo coefficients and the packed stoichiometry,
    // so that the shared memory holds more cells of the stiff kernel
    h.off_cptr = off; off = align16(off + 4u * (ns + 1));
    h.off_cent = off; off = align16(off + 4u * nnz);
    h.prefix = off;
    h.off_gamg = off; off = align16(off + 4u * 3 * nr * 8);
    h.off_hcog = off; off = align16(off + 4u * 3 * nr * 8);
    h.off_e64 = off; off = align16(off + 8u * 3 * ns * 8);
    h.off_sto = off; off = align16(off + 8u * nr);
  }
  h.bytes = static_cast<int>(off);
  return h;
}

}  // namespace

int check_mechanism(const chem_mechanism* m) {
  if (!m || m->ns < 1 || m->ns > 127 || m->nr < 1 || !m->W || !m->thermo || !m->nu_f || !m->nu_r || !m->A ||
      !m->b || !m->Ea || !m->reversible || !m->third_body)
    return CHEM_EINVAL;
  bool any_tb = false;
  for (int r = 0; r < m->nr; ++r) any_tb |= m->third_body[r] != 0;
  if (any_tb && !m->eff) return CHEM_EINVAL;
  const double T_lo = m->thermo[7], T_hi = m->thermo[8];
  if (!(T_lo > 0 && T_hi > T_lo)) return CHEM_EINVAL;
  for (int k = 0; k < m->ns; ++k) {
    if (!(m->W[k] > 0) || !std::isfinite(m->W[k])) return CHEM_EINVAL;
    for (int j = 0; j < 7; ++j)
      if (!std::isfinite(m->thermo[9 * k + j])) return CHEM_EINVAL;
    if (m->thermo[9 * k + 7] != T_lo || m->thermo[9 * k + 8] != T_hi) return CHEM_EINVAL;
  }
  for (int r = 0; r < m->nr; ++r) {
    if (!(m->A[r] > 0) || !std::isfinite(m->A[r]) || !std::isfinite(m->b[r]) || !std::isfinite(m->Ea[r]))
      return CHEM_EINVAL;
    for (int k = 0; k < m->ns; ++k) {
      const int f = m->nu_f[r * m->ns + k], b = m->nu_r[r * m->ns + k];
      if (f < 0 || f > 3 || b < 0 || b > 3) return CHEM_EINVAL;
      if (m->third_body[r] && !(m->eff[r * m->ns + k] >= 0)) return CHEM_EINVAL;
    }
  }
  return CHEM_OK;
}

int check_params(const chem_params* p) {
  if (!p) return CHEM_EINVAL;
  if (!(p->rtol > 0 && p->rtol < 1) || !(p->atol > 0 && p->atol < 1) || !std::isfinite(p->T_min) ||
      !(p->bulk_frac > 0) || !(p->y_floor > 0) || p->k_bulk < 1 || p->k_bulk > 64 || p->k_max < 1 ||
      (p->flags & ~(CHEM_FLAG_FP64_RATES | CHEM_FLAG_TIMING | CHEM_FLAG_ORDER_RATE | CHEM_FLAG_ORDER_PREV |
                    CHEM_FLAG_TWO_PASS)) != 0)
    return CHEM_EINVAL;
  return CHEM_OK;
}

unsigned packed_bytes(const chem_mechanism* m, bool large) { return static_cast<unsigned>(layout(m, large).bytes); }

// The dense layout (ns <= kDenseMaxNs) holds full stoichiometric rows and FP64 copies of the rate
// tables; the large layout (large.cu) holds packed sparse stoichiometry and a species -> reaction
// index instead, and keeps the per-reaction Gibbs and enthalpy coefficients in a tail that is not
// staged (read through L1), which leaves shared memory for more cells in flight.
int pack_mechanism(const chem_mechanism* m, bool large, unsigned char* out, size_t cap, int* ntb_out) {
  const int ns = m->ns, nr = m->nr;
  if (!large && ns > kDenseMaxNs) return CHEM_EUNSUPPORTED;
  const MechHdr h = layout(m, large);
  const int nsp = h.nsp, ntb = h.ntb;
  const unsigned off = static_cast<unsigned>(h.bytes);
  if (off > cap) return CHEM_ENOMEM;
  const double T_lo = m->thermo[7], T_hi = m->thermo[8];
  std::memset(out, 0, off);
  std::memcpy(out, &h, sizeof(h));
  auto F = [&](int o) { return reinterpret_cast<float*>(out + o); };
  float* arr = F(h.off_arr);
  float* eff = F(h.off_eff);
  int* rinfo = reinterpret_cast<int*>(out + h.off_rinfo);
  float *W = F(h.off_W), *invW = F(h.off_invW), *hsp = F(h.off_hsp);
  double* e64 = reinterpret_cast<double*>(out + h.off_e64);
  // dense layout: the rows and the FP64 copies go straight into the tables; large layout: they are
  // only intermediates, and all regimes of gam / hco go to the unstaged tail
  std::vector<float> scratch_rows(large ? 3u * nr * nsp : 0u);
  std::vector<double> scratch64(large ? 4u * nr + 3u * nr * 8 + (ntb > 0 ? ntb : 1) * nsp : 0u);
  float* nuf = large ? scratch_rows.data() : F(h.off_nuf);
  float* nur = large ? scratch_rows.data() + nr * nsp : F(h.off_nur);
  float* dnu = large ? scratch_rows.data() + 2 * nr * nsp : F(h.off_dnu);
  float* gam = large ? F(h.off_gamg) : F(h.off_gam);
  float* hco = large ? F(h.off_hcog) : F(h.off_hco);
  double* arr64 = large ? scratch64.data() : reinterpret_cast<double*>(out + h.off_arr64);
  double* gam64 = large ? scratch64.data() + 4 * nr : reinterpret_cast<double*>(out + h.off_gam64);
  double* eff64 = large ? scratch64.data() + 4 * nr + 3 * nr * 8 : reinterpret_cast<double*>(out + h.off_eff64);
  for (int k = 0; k < ns; ++k) {
    W[k] = static_cast<float>(m->W[k]);
    invW[k] = static_cast<float>(1.0 / m->W[k]);
  }
  // per-species coefficients per regime (0: T < T_lo, 1: in range, 2: T > T_hi), FP64; fixed
  // arrays for the dense layout, heap vectors only for the large one
  double Gd[3 * kDenseMaxNs * 7], Hd[3 * kDenseMaxNs * 6], Ed[3 * kDenseMaxNs * 6];
  std::vector<double> Gv(large ? 3 * ns * 7 : 0), Hv(large ? 3 * ns * 6 : 0), Ev(large ? 3 * ns * 6 : 0);
  double* G = large ? Gv.data() : Gd;
  double* H = large ? Hv.data() : Hd;
  double* E = large ? Ev.data() : Ed;
  for (int k = 0; k < ns; ++k) {
    const double* a = m->thermo + 9 * k;
    // in range
    double* g = &G[(1 * ns + k) * 7];
    g[0] = a[0]; g[1] = -a[1] / 2; g[2] = -a[2] / 6; g[3] = -a[3] / 12; g[4] = -a[4] / 20; g[5] = a[5]; g[6] = -a[6];
    double* hh = &H[(1 * ns + k) * 6];
    hh[0] = a[0]; hh[1] = a[1] / 2; hh[2] = a[2] / 3; hh[3] = a[3] / 4; hh[4] = a[4] / 5; hh[5] = a[5];
    double* ee = &E[(1 * ns + k) * 6];
    ee[0] = a[5] / m->W[k]; ee[1] = (a[0] - 1.0) / m->W[k]; ee[2] = a[1] / 2 / m->W[k];
    ee[3] = a[2] / 3 / m->W[k]; ee[4] = a[3] / 4 / m->W[k]; ee[5] = a[4] / 5 / m->W[k];
    // extrapolated regimes: cp frozen at the boundary value
    for (int side = 0; side < 2; ++side) {
      const int reg = side == 0 ? 0 : 2;
      const double Tb = side == 0 ? T_lo : T_hi;
      const double cpb = a[0] + Tb * (a[1] + Tb * (a[2] + Tb * (a[3] + Tb * a[4])));
      const double hb = Tb * (a[0] + Tb * (a[1] / 2 + Tb * (a[2] / 3 + Tb * (a[3] / 4 + Tb * a[4] / 5)))) + a[5];
      const double sb = a[0] * std::log(Tb) + Tb * (a[1] + Tb * (a[2] / 2 + Tb * (a[3] / 3 + Tb * a[4] / 4))) + a[6];
      double* g2 = &G[(reg * ns + k) * 7];
      g2[0] = cpb; g2[1] = g2[2] = g2[3] = g2[4] = 0.0; g2[5] = hb - cpb * Tb; g2[6] = cpb * std::log(Tb) - sb;
      double* h2 = &H[(reg * ns + k) * 6];
      h2[0] = cpb; h2[1] = h2[2] = h2[3] = h2[4] = 0.0; h2[5] = hb - cpb * Tb;
      double* e2 = &E[(reg * ns + k) * 6];
      e2[0] = (hb - cpb * Tb) / m->W[k]; e2[1] = (cpb - 1.0) / m->W[k]; e2[2] = e2[3] = e2[4] = e2[5] = 0.0;
    }
  }
  for (int reg = 0; reg < 3; ++reg)
    for (int k = 0; k < ns; ++k) {
      for (int j = 0; j < 6; ++j) {
        e64[(reg * ns + k) * 8 + j] = E[(reg * ns + k) * 6 + j];
        hsp[(reg * ns + k) * 8 + j] = static_cast<float>(H[(reg * ns + k) * 6 + j]);
      }
      e64[(reg * ns + k) * 8 + 6] = 1.0 / m->W[k];
    }
  int tbrow = 0;
  for (int r = 0; r < nr; ++r) {
    double dn = 0.0;
    for (int k = 0; k < ns; ++k) {
      const int f = m->nu_f[r * ns + k], b = m->nu_r[r * ns + k];
      nuf[r * nsp + k] = static_cast<float>(f);
      nur[r * nsp + k] = static_cast<float>(b);
      dnu[r * nsp + k] = static_cast<float>(b - f);
      dn += b - f;
    }
    arr64[4 * r + 0] = std::log(m->A[r]);
    arr64[4 * r + 1] = m->b[r];
    arr64[4 * r + 2] = m->Ea[r] / kR;
    arr64[4 * r + 3] = dn;
    for (int j = 0; j < 4; ++j) arr[4 * r + j] = static_cast<float>(arr64[4 * r + j]);
    int info = m->reversible[r] ? 1 : 0;
    if (m->third_body[r]) {
      for (int k = 0; k < ns; ++k) {
        eff[tbrow * nsp + k] = static_cast<float>(m->eff[r * ns + k]);
        eff64[tbrow * nsp + k] = m->eff[r * ns + k];
      }
      info |= (tbrow + 1) << 8;
      ++tbrow;
    }
    rinfo[r] = info;
    // reaction Gibbs / enthalpy coefficients, contracted with dnu in FP64 (no device cancellation)
    for (int reg = 0; reg < 3; ++reg) {
      for (int j = 0; j < 7; ++j) {
        double sg = 0.0;
        for (int k = 0; k < ns; ++k) sg += (m->nu_r[r * ns + k] - m->nu_f[r * ns + k]) * G[(reg * ns + k) * 7 + j];
        gam[(reg * nr + r) * 8 + j] = static_cast<float>(sg);
        gam64[(reg * nr + r) * 8 + j] = sg;
      }
      for (int j = 0; j < 6; ++j) {
        double sh = 0.0;
        for (int k = 0; k < ns; ++k) sh += (m->nu_r[r * ns + k] - m->nu_f[r * ns + k]) * H[(reg * ns + k) * 6 + j];
        hco[(reg * nr + r) * 8 + j] = static_cast<float>(sh);
      }
    }
  }
  if (large) {
    // packed sparse stoichiometry: up to 3 (species, coefficient) pairs per side, 9 bits each
    int2* sto = reinterpret_cast<int2*>(out + h.off_sto);
    for (int r = 0; r < nr; ++r) {
      int packed[2] = {0, 0}, cnt[2] = {0, 0};
      for (int k = 0; k < ns; ++k)
        for (int side = 0; side < 2; ++side) {
          const int c = side == 0 ? m->nu_f[r * ns + k] : m->nu_r[r * ns + k];
          if (c == 0) continue;
          if (cnt[side] >= 3 || c > 3 || k > 127) return CHEM_EUNSUPPORTED;
          packed[side] |= (k | (c << 7)) << (9 * cnt[side]);
          ++cnt[side];
        }
      sto[r] = make_int2(packed[0], packed[1]);
    }
    // species -> (reaction, dnu), reactions in increasing order
    int* cptr = reinterpret_cast<int*>(out + h.off_cptr);
    int* cent = reinterpret_cast<int*>(out + h.off_cent);
    int e = 0;
    for (int k = 0; k < ns; ++k) {
      cptr[k] = e;
      for (int r = 0; r < nr; ++r) {
        const int d = m->nu_r[r * ns + k] - m->nu_f[r * ns + k];
        if (d != 0) cent[e++] = (r & 0xFFFF) | (d * 65536);
      }
    }
    cptr[ns] = e;
    if (nr > 65535) return CHEM_EUNSUPPORTED;
  }
  if (ntb_out) *ntb_out = ntb;
  return CHEM_OK;
}

}  // namespace chem
