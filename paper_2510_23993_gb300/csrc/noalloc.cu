// noalloc.cu -- chem_advance_noalloc: the bulk-sparse advance of chem_advance for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted -- inside a host
// callback or a real-time loop that must not block on the allocator, plugins of a host
// application that owns all device memory and hands out only its own buffers, or processes
// whose allocator is capped.  chem_init cannot be used there: it allocates the mechanism tables
// and the workspace.  This entry point takes the mechanism from host memory on every call and
// keeps both the tables and its scratch (the counters and the stiff-cell queue) in file-scope
// device arrays of fixed size, loaded with the library and held by every GPU that uses it until
// the process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
//
// Limits: at most kMaxCells cells per call and kTableBytes of packed mechanism tables.  All calls
// share the arrays, which keep the last call's contents: the counters are cleared at the start
// of each call, and calls that overlap on the GPU (other streams, other host threads) race.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/chem.h"
#include "chem_device.cuh"
#include "internal.h"

using namespace chem;

namespace {

constexpr long long kMaxCells = 1LL << 21;           // 2,097,152 cells -> 8 MiB of queue
constexpr size_t kTableBytes = 64u << 10;             // 64 KiB of mechanism tables
constexpr size_t kCounterBytes = 256;                 // Workspace, padded
constexpr int kMaxDevices = 64;
static_assert(sizeof(Workspace) <= kCounterBytes, "counter block too small");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterBytes + 4 * kMaxCells];
static __device__ __align__(256) unsigned char g_noalloc_tables[kTableBytes];

namespace {

struct DeviceSlot {
  bool ready = false;
  unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch on this device
  unsigned char* tables = nullptr;    // device address of g_noalloc_tables on this device
  int sms = 0;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

int fail(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CHEM_OK;
  std::fprintf(stderr, "libchem (noalloc): %s: %s\n", what, cudaGetErrorString(e));
  return CHEM_ECUDA;
}

// Set-up once per device, with that device current: the device addresses of the two arrays.
int setup(int dev, DeviceSlot** out) {
  if (dev < 0 || dev >= kMaxDevices) return CHEM_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* p = nullptr;
    int rc = fail(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
    if (rc) return rc;
    s.scratch = static_cast<unsigned char*>(p);
    rc = fail(cudaGetSymbolAddress(&p, g_noalloc_tables), "cudaGetSymbolAddress(tables)");
    if (rc) return rc;
    s.tables = static_cast<unsigned char*>(p);
    rc = fail(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (rc) return rc;
    s.ready = true;
  }
  *out = &s;
  return CHEM_OK;
}

unsigned al16(unsigned x) { return (x + 15u) & ~15u; }

// The table layout of chem_device.cuh (MechHdr), written into a caller buffer without allocating.
// Returns the byte count, or 0 if the mechanism does not fit in cap bytes or is inconsistent.
unsigned pack_into(const chem_mechanism* m, unsigned char* out, size_t cap) {
  const int ns = m->ns, nr = m->nr, nsp = (ns + 3) & ~3;
  if (ns < 1 || ns > 15 || nr < 1) return 0;
  int ntb = 0;
  for (int r = 0; r < nr; ++r) ntb += m->third_body[r] ? 1 : 0;
  MechHdr h{};
  h.ns = ns;
  h.nr = nr;
  h.ntb = ntb;
  h.nsp = nsp;
  // trailing species that no reaction changes: left out of the stiff kernel's linear algebra
  int nact = ns;
  while (nact > 1) {
    bool inert = true;
    for (int r = 0; r < nr && inert; ++r) inert = m->nu_r[r * ns + nact - 1] == m->nu_f[r * ns + nact - 1];
    if (!inert) break;
    --nact;
  }
  h.nact = nact;
  const double T_lo = m->thermo[7], T_hi = m->thermo[8];
  h.T_lo = static_cast<float>(T_lo);
  h.T_hi = static_cast<float>(T_hi);
  h.lnP0R = static_cast<float>(std::log(kP0 / kR));
  unsigned off = al16(sizeof(MechHdr));
  h.off_arr = off; off = al16(off + 16u * nr);
  h.off_nuf = off; off = al16(off + 4u * nr * nsp);
  h.off_nur = off; off = al16(off + 4u * nr * nsp);
  h.off_dnu = off; off = al16(off + 4u * nr * nsp);
  h.off_eff = off; off = al16(off + 4u * (ntb > 0 ? ntb : 1) * nsp);
  h.off_rinfo = off; off = al16(off + 4u * nr);
  h.off_W = off; off = al16(off + 4u * nsp);
  h.off_invW = off; off = al16(off + 4u * nsp);
  h.off_gam = off; off = al16(off + 4u * 3 * nr * 8);
  h.off_hco = off; off = al16(off + 4u * 3 * nr * 8);
  h.off_hsp = off; off = al16(off + 4u * 3 * ns * 8);
  h.off_e64 = off; off = al16(off + 8u * 3 * ns * 8);
  h.off_arr64 = off; off = al16(off + 8u * 4 * nr);
  h.off_gam64 = off; off = al16(off + 8u * 3 * nr * 8);
  h.off_eff64 = off; off = al16(off + 8u * (ntb > 0 ? ntb : 1) * nsp);
  h.bytes = off;
  if (off > cap) return 0;
  std::memset(out, 0, off);
  std::memcpy(out, &h, sizeof(h));
  auto F = [&](int o) { return reinterpret_cast<float*>(out + o); };
  auto D = [&](int o) { return reinterpret_cast<double*>(out + o); };
  float *arr = F(h.off_arr), *nuf = F(h.off_nuf), *nur = F(h.off_nur), *dnu = F(h.off_dnu), *eff = F(h.off_eff);
  int* rinfo = reinterpret_cast<int*>(out + h.off_rinfo);
  float *W = F(h.off_W), *invW = F(h.off_invW), *gam = F(h.off_gam), *hco = F(h.off_hco), *hsp = F(h.off_hsp);
  double *e64 = D(h.off_e64), *arr64 = D(h.off_arr64), *gam64 = D(h.off_gam64), *eff64 = D(h.off_eff64);
  for (int k = 0; k < ns; ++k) {
    W[k] = static_cast<float>(m->W[k]);
    invW[k] = static_cast<float>(1.0 / m->W[k]);
  }
  // per species and regime: Gibbs (7), enthalpy (6) and mass-specific energy (6) coefficients
  double G[3][15][7], H[3][15][6], E[3][15][6];
  for (int k = 0; k < ns; ++k) {
    const double* a = m->thermo + 9 * k;
    const double Wk = m->W[k];
    const double g1[7] = {a[0], -a[1] / 2, -a[2] / 6, -a[3] / 12, -a[4] / 20, a[5], -a[6]};
    const double h1[6] = {a[0], a[1] / 2, a[2] / 3, a[3] / 4, a[4] / 5, a[5]};
    const double e1[6] = {a[5] / Wk, (a[0] - 1.0) / Wk, a[1] / 2 / Wk, a[2] / 3 / Wk, a[3] / 4 / Wk, a[4] / 5 / Wk};
    for (int j = 0; j < 7; ++j) G[1][k][j] = g1[j];
    for (int j = 0; j < 6; ++j) { H[1][k][j] = h1[j]; E[1][k][j] = e1[j]; }
    for (int side = 0; side < 2; ++side) {
      const int reg = side == 0 ? 0 : 2;
      const double Tb = side == 0 ? T_lo : T_hi;
      const double cpb = a[0] + Tb * (a[1] + Tb * (a[2] + Tb * (a[3] + Tb * a[4])));
      const double hb = Tb * (a[0] + Tb * (a[1] / 2 + Tb * (a[2] / 3 + Tb * (a[3] / 4 + Tb * a[4] / 5)))) + a[5];
      const double sb = a[0] * std::log(Tb) + Tb * (a[1] + Tb * (a[2] / 2 + Tb * (a[3] / 3 + Tb * a[4] / 4))) + a[6];
      for (int j = 0; j < 7; ++j) G[reg][k][j] = 0.0;
      for (int j = 0; j < 6; ++j) { H[reg][k][j] = 0.0; E[reg][k][j] = 0.0; }
      G[reg][k][0] = cpb; G[reg][k][5] = hb - cpb * Tb; G[reg][k][6] = cpb * std::log(Tb) - sb;
      H[reg][k][0] = cpb; H[reg][k][5] = hb - cpb * Tb;
      E[reg][k][0] = (hb - cpb * Tb) / Wk; E[reg][k][1] = (cpb - 1.0) / Wk;
    }
  }
  for (int reg = 0; reg < 3; ++reg)
    for (int k = 0; k < ns; ++k) {
      for (int j = 0; j < 6; ++j) {
        e64[(reg * ns + k) * 8 + j] = E[reg][k][j];
        hsp[(reg * ns + k) * 8 + j] = static_cast<float>(H[reg][k][j]);
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
    for (int reg = 0; reg < 3; ++reg) {
      for (int j = 0; j < 7; ++j) {
        double sg = 0.0;
        for (int k = 0; k < ns; ++k) sg += (m->nu_r[r * ns + k] - m->nu_f[r * ns + k]) * G[reg][k][j];
        gam[(reg * nr + r) * 8 + j] = static_cast<float>(sg);
        gam64[(reg * nr + r) * 8 + j] = sg;
      }
      for (int j = 0; j < 6; ++j) {
        double sh = 0.0;
        for (int k = 0; k < ns; ++k) sh += (m->nu_r[r * ns + k] - m->nu_f[r * ns + k]) * H[reg][k][j];
        hco[(reg * nr + r) * 8 + j] = static_cast<float>(sh);
      }
    }
  }
  return off;
}

}  // namespace

extern "C" int chem_advance_noalloc(const chem_mechanism* mech, const chem_params* params, float* T, float* p,
                                    float* Y, int64_t ld, const float* rho, const float* e, int64_t n, double dt,
                                    int32_t* substeps, chem_stats* stats, void* stream) {
  if (!mech || !mech->W || !mech->thermo || !mech->nu_f || !mech->nu_r || !mech->A || !mech->b || !mech->Ea ||
      !mech->reversible || !mech->third_body || n < 0 || !(dt > 0) || !std::isfinite(dt))
    return CHEM_EINVAL;
  if (n > kMaxCells) {
    std::fprintf(stderr, "libchem (noalloc): %lld cells exceed the static limit of %lld\n",
                 static_cast<long long>(n), kMaxCells);
    return CHEM_ENOMEM;
  }
  if (n > 0 && (!T || !Y || !rho || !e || !substeps || ld < n)) return CHEM_EINVAL;
  if (mech->ns != 9) return CHEM_EUNSUPPORTED;
  for (int r = 0; r < mech->nr; ++r)
    if (mech->third_body[r] && !mech->eff) return CHEM_EINVAL;
  chem_params prm;
  chem_default_params(&prm);
  if (params) prm = *params;
  if (!(prm.rtol > 0 && prm.rtol < 1) || !(prm.atol > 0 && prm.atol < 1) || prm.k_bulk < 1 || prm.k_bulk > 64 ||
      prm.k_max < 1 || !(prm.bulk_frac > 0) || !(prm.y_floor > 0))
    return CHEM_EINVAL;

  int dev = 0;
  int rc = fail(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  DeviceSlot* slot = nullptr;
  if ((rc = setup(dev, &slot))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  unsigned char blob[kTableBytes];   // host stack: packed tables, copied into the static array
  const unsigned bytes = pack_into(mech, blob, sizeof(blob));
  if (bytes == 0) return CHEM_ENOMEM;
  // pageable source: the copy is staged before cudaMemcpyAsync returns, so the stack buffer may go
  if ((rc = fail(cudaMemcpyAsync(slot->tables, blob, bytes, cudaMemcpyHostToDevice, st), "copy tables"))) return rc;
  Workspace* ws = reinterpret_cast<Workspace*>(slot->scratch);
  int* queue = reinterpret_cast<int*>(slot->scratch + kCounterBytes);
  if ((rc = fail(cudaMemsetAsync(ws, 0, sizeof(Workspace), st), "clear counters"))) return rc;
  if (n > 0) {
    AdvanceArgs<float> a;
    a.blob = slot->tables;
    a.blob_bytes = bytes;
    a.prm.rtol = static_cast<float>(prm.rtol);
    a.prm.atol = static_cast<float>(prm.atol);
    a.prm.T_min = static_cast<float>(prm.T_min);
    a.prm.bulk_frac = static_cast<float>(prm.bulk_frac);
    a.prm.y_floor = static_cast<float>(prm.y_floor);
    a.prm.k_bulk = prm.k_bulk;
    a.prm.k_max = prm.k_max;
    a.prm.flags = prm.flags & CHEM_FLAG_FP64_RATES;
    a.T = T;
    a.p = p;
    a.Y = Y;
    a.ld = ld;
    a.rho = rho;
    a.e = e;
    a.n = n;
    a.dt = dt;
    a.substeps = substeps;
    a.ws = ws;
    a.queue = queue;
    a.qkey = nullptr;   // no cost ordering here: the stiff kernel takes cells in compaction order
    a.boxes = nullptr;
    a.box_off = nullptr;
    a.nbox = 0;
    a.skip = nullptr;
    a.pass = 0;   // single pass: the two-pass mode's continuation storage is not part of the scratch
    a.cont_cap = 0;
    a.cont = nullptr;
    a.cont_list = nullptr;
    a.cont_key = nullptr;
    a.cont_sorted = nullptr;
    int bpsm = 1, spsm = 1;
    if (bulk_occupancy(mech->ns, false, bytes, &bpsm) != 0 || bpsm < 1) bpsm = 1;
    if (stiff_occupancy(mech->ns, bytes, &spsm) != 0 || spsm < 1) spsm = 1;
    long long want = (n + kBulkBlock - 1) / kBulkBlock;
    const long long cap = static_cast<long long>(slot->sms) * bpsm;
    const int bgrid = static_cast<int>(want < cap ? (want < 1 ? 1 : want) : cap);
    int r1 = launch_bulk_f32(mech->ns, a, bgrid, st);
    int r2 = r1 ? r1 : launch_stiff_f32(mech->ns, a, slot->sms * spsm, st);
    if (r1 == -1 || r2 == -1) return CHEM_EUNSUPPORTED;
    if (r1 || r2) return fail(static_cast<cudaError_t>(r1 ? r1 : r2), "kernel launch");
  }
  if (stats) {   // pageable destination: this copy completes before cudaMemcpyAsync returns
    Workspace w;
    if ((rc = fail(cudaMemcpyAsync(&w, ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st), "read counters")))
      return rc;
    if ((rc = fail(cudaStreamSynchronize(st), "cudaStreamSynchronize"))) return rc;
    std::memset(stats, 0, sizeof(*stats));
    stats->ncell = n;
    stats->nskipped = static_cast<int64_t>(w.nskipped);
    stats->nbulk = static_cast<int64_t>(w.nbulk);
    stats->nqueued = w.qcount;
    stats->nfailed = static_cast<int64_t>(w.nfailed);
    stats->ninvalid = static_cast<int64_t>(w.ninvalid);
    stats->substeps = static_cast<int64_t>(w.substeps);
    stats->attempts = static_cast<int64_t>(w.attempts);
    stats->newton = static_cast<int64_t>(w.newton);
    int status = CHEM_OK;
    if (w.status & kFlagInvalid) status = CHEM_EINVAL;
    if (w.status & (kFlagNoConv | kFlagTemp)) status = CHEM_ENOCONV;
    if (w.status & kFlagMaxSteps) status = CHEM_EMAXSTEPS;
    if (w.status & kFlagStage) status = CHEM_ECUDA;
    stats->status = status;
  }
  return CHEM_OK;
}
