// noalloc.cu -- chem_advance_noalloc: the bulk-sparse advance of chem_advance for callers that
// cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- a real-time loop that may not block on the
// allocator, a plugin of a host application that owns all device memory and hands out only its
// own buffers, or a process whose allocator is capped.  chem_init cannot be used there: it
// allocates the mechanism tables and the workspace.  This entry point takes the mechanism from
// host memory on every call and keeps both the tables and its scratch (the counters and the
// stiff-cell queue) in file-scope device arrays of fixed size, loaded with the library and held by
// every GPU that uses it until the process exits.  It calls no cudaMalloc, cudaFree or other
// allocating routine; the tables are packed by the same packer as chem_init's (pack.cu) into a
// static host buffer.
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
std::mutex g_mutex;                 // guards g_slots and g_host_tables
unsigned char g_host_tables[kTableBytes];   // packed tables on the host, copied into the device array

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

}  // namespace

extern "C" int chem_advance_noalloc(const chem_mechanism* mech, const chem_params* params, float* T, float* p,
                                    float* Y, int64_t ld, const float* rho, const float* e, int64_t n, double dt,
                                    int32_t* substeps, chem_stats* stats, void* stream) {
  // the same checks of the mechanism and the parameters as chem_init / chem_set_params
  if (check_mechanism(mech) || (params && check_params(params)) || n < 0 || !(dt > 0) || !std::isfinite(dt))
    return CHEM_EINVAL;
  if (n > kMaxCells) {
    std::fprintf(stderr, "libchem (noalloc): %lld cells exceed the static limit of %lld\n",
                 static_cast<long long>(n), kMaxCells);
    return CHEM_ENOMEM;
  }
  if (n > 0 && (!T || !Y || !rho || !e || !substeps || ld < n)) return CHEM_EINVAL;
  if (mech->ns != 9) return CHEM_EUNSUPPORTED;
  chem_params prm;
  chem_default_params(&prm);
  if (params) prm = *params;

  int dev = 0;
  int rc = fail(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  DeviceSlot* slot = nullptr;
  if ((rc = setup(dev, &slot))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  unsigned bytes = 0;
  {
    // pack into the static host buffer; pageable source: cudaMemcpyAsync returns once the bytes
    // are staged, so the buffer is free again when the lock is released
    std::lock_guard<std::mutex> lock(g_mutex);
    if ((rc = pack_mechanism(mech, false, g_host_tables, sizeof(g_host_tables), nullptr))) return rc;
    bytes = reinterpret_cast<const MechHdr*>(g_host_tables)->prefix;
    if ((rc = fail(cudaMemcpyAsync(slot->tables, g_host_tables, bytes, cudaMemcpyHostToDevice, st), "copy tables")))
      return rc;
  }
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
    if (stiff_occupancy(mech->ns, bytes, kStiffBlock, &spsm) != 0 || spsm < 1) spsm = 1;
    long long want = (n + kBulkBlock - 1) / kBulkBlock;
    const long long cap = static_cast<long long>(slot->sms) * bpsm;
    const int bgrid = static_cast<int>(want < cap ? (want < 1 ? 1 : want) : cap);
    int r1 = launch_bulk_f32(mech->ns, a, bgrid, st);
    int r2 = r1 ? r1 : launch_stiff_f32(mech->ns, a, slot->sms * spsm, kStiffBlock, st);
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
    stats->factorizations = stats->attempts;   // the dense stiff kernel factors on every attempt
    int status = CHEM_OK;
    if (w.status & kFlagInvalid) status = CHEM_EINVAL;
    if (w.status & (kFlagNoConv | kFlagTemp)) status = CHEM_ENOCONV;
    if (w.status & kFlagMaxSteps) status = CHEM_EMAXSTEPS;
    if (w.status & kFlagStage) status = CHEM_ECUDA;
    stats->status = status;
  }
  return CHEM_OK;
}
