// abi.cu -- the C ABI of libchem.so (include/chem.h): argument checks, packing of the
// mechanism tables, workspace management and the launch sequence of one chemistry step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/chem.h"
#include "chem_device.cuh"
#include "internal.h"

namespace chem {
namespace sg {
struct State;
}
void surrogate_release(sg::State* s);   // surrogate.cu
}  // namespace chem

using namespace chem;

struct chem_ctx {
  int dev = 0, sms = 0;
  int ns = 0, nr = 0, ntb = 0;
  int nact = 0;                    // species before the trailing inert ones (packed header)
  unsigned char* blob = nullptr;   // device, 16-byte aligned
  unsigned blob_bytes = 0;
  chem_params prm{};
  int64_t max_cells = 0;
  Workspace* ws = nullptr;         // device
  Workspace* ws_host = nullptr;    // pinned copy of the last call's counters
  int* queue = nullptr;            // device [max_cells]
  int* queue2 = nullptr;           // device [max_cells], the queue in cost order
  unsigned char* qkey = nullptr;   // device [max_cells], cost bucket of each queue entry
  int64_t last_n = 0;
  int bulk_grid = 0, stiff_grid = 0;
  int stiff_block = kStiffBlock;                            // threads per CTA of the dense stiff kernel
  int probe_att = kProbeAttempts, round_att = kRoundAttempts;   // two-pass scheduling quanta
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // CHEM_FLAG_TIMING
  // box table (chem_boxes_set)
  DevBox<float>* boxes = nullptr;
  int* box_off = nullptr;
  int nbox = 0;
  int64_t box_cells = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool timed = false;
  // staging buffers of chem_advance_host (allocated on its first use)
  float* hbuf = nullptr;
  int* hsub = nullptr;
  // host copies of the stoichiometry (the surrogate's conservation constraints)
  std::vector<double> W;
  std::vector<int8_t> nu_f, nu_r;
  bool large = false;              // sparse table layout, one warp per cell (large.cu)
  chem::sg::State* sg = nullptr;   // surrogate (surrogate.cu), created by chem_surrogate_init
  // two-pass stiff integration (CHEM_FLAG_TWO_PASS): continuation state by queue slot
  double* cont = nullptr;
  int* cont_list = nullptr;
  unsigned char* cont_key = nullptr;
  int* cont_sorted = nullptr;
  long long cont_cap = 0;
  // chem_advance_explicit: FP64 time, temperature and mass fractions of each cell (first use)
  double* xcell = nullptr;
  // chem_rates_tc: the tensor-core operand image of a large mechanism (rates_tc.cu)
  unsigned char* tc_img = nullptr;
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CHEM_OK;
  std::fprintf(stderr, "libchem: %s: %s\n", what, cudaGetErrorString(e));
  return CHEM_ECUDA;
}

bool compiled_ns(int ns) { return ns == 9; }

// continuation storage of the two-pass mode, allocated once when the flag is first set
int ensure_two_pass(chem_ctx* c) {
  // the warp-per-cell path of large mechanisms runs the single-pass schedule (flag ignored)
  if (!(c->prm.flags & CHEM_FLAG_TWO_PASS) || c->cont || c->large) return CHEM_OK;
  const long long cap = c->max_cells > 0 ? c->max_cells : 1;
  if (cudaMalloc(&c->cont, static_cast<size_t>(cap * cont_bytes_per_slot(c->ns))) != cudaSuccess ||
      cudaMalloc(&c->cont_list, sizeof(int) * cap) != cudaSuccess || cudaMalloc(&c->cont_key, cap) != cudaSuccess ||
      cudaMalloc(&c->cont_sorted, sizeof(int) * cap) != cudaSuccess) {
    cudaFree(c->cont);
    cudaFree(c->cont_list);
    cudaFree(c->cont_key);
    cudaFree(c->cont_sorted);
    c->cont = nullptr;
    c->cont_list = nullptr;
    c->cont_key = nullptr;
    c->cont_sorted = nullptr;
    return CHEM_ENOMEM;
  }
  c->cont_cap = cap;
  return CHEM_OK;
}

// The stiff phase: one persistent launch, or (two-pass mode) a probe launch, a counting sort of
// the unfinished cells by remaining work, and a cooperative continuation launch: the sorted cells
// run to completion from a shared queue until it is empty, then the cells still running are
// parked and finished in rounds of round_att steps, compacted into full warps between rounds.
template <typename S>
int launch_stiff_phase(chem_ctx* c, AdvanceArgs<S> b, long long n, cudaStream_t st) {
  auto launch = [&](const AdvanceArgs<S>& x) {
    if constexpr (sizeof(S) == 4) return launch_stiff_f32(c->ns, x, c->stiff_grid, c->stiff_block, st);
    else return launch_stiff_f64(c->ns, x, c->stiff_grid, c->stiff_block, st);
  };
  b.probe_att = c->probe_att;
  b.round_att = c->round_att;
  b.pass = 0;
  b.cont_cap = 0;
  b.cont = nullptr;
  b.cont_list = nullptr;
  b.cont_key = nullptr;
  b.cont_sorted = nullptr;
  if (!(c->prm.flags & CHEM_FLAG_TWO_PASS) || !c->cont || n > c->cont_cap) return launch(b);
  b.cont_cap = c->cont_cap;
  b.cont = c->cont;
  b.cont_list = c->cont_list;
  b.cont_key = c->cont_key;
  b.cont_sorted = c->cont_sorted;
  b.pass = 1;
  int r = launch(b);
  if (!r) r = launch_order_queue(c->ws, c->cont_list, c->cont_key, c->cont_sorted, n, st, true);
  b.pass = 2;   // cooperative launch (its grid is capped at the CTAs that fit at once)
  if (!r) r = launch(b);
  return r;
}

KParams kparams(const chem_params& p) {
  KParams k;
  k.rtol = static_cast<float>(p.rtol);
  k.atol = static_cast<float>(p.atol);
  k.T_min = static_cast<float>(p.T_min);
  k.bulk_frac = static_cast<float>(p.bulk_frac);
  k.y_floor = static_cast<float>(p.y_floor);
  k.k_bulk = p.k_bulk;
  k.k_max = p.k_max;
  k.flags = p.flags;
  return k;
}

template <typename S>
int advance_impl(chem_ctx* ctx, S* T, S* p, S* Y, int64_t ld, const S* rho, const S* e, int64_t n, double dt,
                 int32_t* substeps, cudaStream_t st, const unsigned char* skip = nullptr) {
  if (!ctx || n < 0 || !(dt > 0) || !std::isfinite(dt)) return CHEM_EINVAL;
  if (n > ctx->max_cells) return CHEM_ENOMEM;
  if (n > 0 && (!T || !Y || !rho || !e || !substeps || ld < n)) return CHEM_EINVAL;
  int rc = cuda_fail(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (rc) return rc;
  rc = cuda_fail(cudaMemsetAsync(ctx->ws, 0, sizeof(Workspace), st), "cudaMemsetAsync");
  if (rc) return rc;
  ctx->last_n = n;
  ctx->timed = false;
  if (n > 0) {
    AdvanceArgs<S> a;
    a.blob = ctx->blob;
    a.blob_bytes = ctx->blob_bytes;
    a.prm = kparams(ctx->prm);
    a.T = T;
    a.p = p;
    a.Y = Y;
    a.ld = ld;
    a.rho = rho;
    a.e = e;
    a.n = n;
    a.dt = dt;
    a.substeps = substeps;
    a.ws = ctx->ws;
    a.queue = ctx->queue;
    a.boxes = nullptr;
    a.box_off = nullptr;
    a.nbox = 0;
    a.skip = skip;
    const bool order = (ctx->prm.flags & (CHEM_FLAG_ORDER_RATE | CHEM_FLAG_ORDER_PREV)) != 0;
    a.qkey = order ? ctx->qkey : nullptr;
    long long want = (n + kBulkBlock - 1) / kBulkBlock;
    const int bgrid = static_cast<int>(want < ctx->bulk_grid ? (want < 1 ? 1 : want) : ctx->bulk_grid);
    int r1, r2;
    const bool timed = (ctx->prm.flags & CHEM_FLAG_TIMING) != 0;
    ctx->timed = timed;
    if (timed) cudaEventRecord(ctx->ev[0], st);
    AdvanceArgs<S> b = a;   // the stiff kernel reads the cost-ordered queue when ordering is on
    if (order) b.queue = ctx->queue2;
    if (ctx->large) {   // one warp per cell (FP32 state only)
      if constexpr (sizeof(S) == 4) {
        const long long wb = (n + 7) / 8;   // bulk CTAs of 8 warps
        const int lgrid = static_cast<int>(wb < ctx->bulk_grid ? (wb < 1 ? 1 : wb) : ctx->bulk_grid);
        r1 = launch_bulk_lg(ctx->ns, ctx->nr, ctx->ntb, a, lgrid, st);
        if (!r1 && order) r1 = launch_order_queue(ctx->ws, ctx->queue, ctx->qkey, ctx->queue2, n, st);
        if (timed && !r1) cudaEventRecord(ctx->ev[1], st);
        r2 = r1 ? r1 : launch_stiff_lg(ctx->ns, ctx->nact, ctx->nr, ctx->ntb, b, ctx->stiff_grid, st);
      } else {
        return CHEM_EUNSUPPORTED;
      }
    } else {
      if constexpr (sizeof(S) == 4) r1 = launch_bulk_f32(ctx->ns, a, bgrid, st);
      else r1 = launch_bulk_f64(ctx->ns, a, bgrid, st);
      if (!r1 && order) r1 = launch_order_queue(ctx->ws, ctx->queue, ctx->qkey, ctx->queue2, n, st);
      if (timed && !r1) cudaEventRecord(ctx->ev[1], st);
      r2 = r1 ? r1 : launch_stiff_phase<S>(ctx, b, n, st);
    }
    if (timed && !r1 && !r2) cudaEventRecord(ctx->ev[2], st);
    if (r1 == -1 || r2 == -1) return CHEM_EUNSUPPORTED;
    if (r1 || r2) return cuda_fail(static_cast<cudaError_t>(r1 ? r1 : r2), "kernel launch");
  }
  return cuda_fail(cudaMemcpyAsync(ctx->ws_host, ctx->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st),
                   "cudaMemcpyAsync(stats)");
}

}  // namespace

namespace chem {
// launch settings of a context, used by the tuner (tune.cu)
void ctx_get_launch(const chem_ctx* c, int* bulk_grid, int* stiff_grid, int* sms, int* ns, int* nr) {
  *bulk_grid = c->bulk_grid;
  *stiff_grid = c->stiff_grid;
  *sms = c->sms;
  *ns = c->ns;
  *nr = c->nr;
}
void ctx_set_launch(chem_ctx* c, int bulk_grid, int stiff_grid) {
  c->bulk_grid = bulk_grid > 0 ? bulk_grid : 1;
  c->stiff_grid = stiff_grid > 0 ? stiff_grid : 1;
}
void ctx_get_params(const chem_ctx* c, chem_params* p) { *p = c->prm; }
// dense stiff kernel: threads per CTA and the two-pass scheduling quanta (large mechanisms: unused)
void ctx_get_sched(const chem_ctx* c, int* stiff_block, int* probe_att, int* round_att, int* large) {
  *stiff_block = c->stiff_block;
  *probe_att = c->probe_att;
  *round_att = c->round_att;
  *large = c->large ? 1 : 0;
}
void ctx_set_sched(chem_ctx* c, int stiff_block, int probe_att, int round_att) {
  // the CTA sizes the stiff kernel is compiled for; anything else keeps the current one
  if (stiff_block == 64 || stiff_block == 128 || stiff_block == 256) c->stiff_block = stiff_block;
  if (probe_att >= 1) c->probe_att = probe_att;
  if (round_att >= 1) c->round_att = round_att;
}
int occupancy_bulk(const chem_ctx* c) {
  int b = 0;
  const int r = c->large ? occupancy_lg(c->ns, c->nact, c->nr, c->ntb, c->blob_bytes, false, &b)
                         : bulk_occupancy(c->ns, false, c->blob_bytes, &b);
  return (r != 0 || b < 1) ? 1 : b;
}
int occupancy_stiff(const chem_ctx* c) {
  int b = 0;
  const int r = c->large ? occupancy_lg(c->ns, c->nact, c->nr, c->ntb, c->blob_bytes, true, &b)
                         : stiff_occupancy(c->ns, c->blob_bytes, c->stiff_block, &b);
  return (r != 0 || b < 1) ? 1 : b;
}
// surrogate state and the mechanism data it needs (surrogate.cu)
sg::State* ctx_surrogate(chem_ctx* c) { return c->sg; }
void ctx_set_surrogate(chem_ctx* c, sg::State* s) { c->sg = s; }
void ctx_mech_host(const chem_ctx* c, int* ns, int* nr, const double** W, const int8_t** nuf, const int8_t** nur) {
  *ns = c->ns;
  *nr = c->nr;
  *W = c->W.data();
  *nuf = c->nu_f.data();
  *nur = c->nu_r.data();
}
const unsigned char* ctx_blob(const chem_ctx* c, unsigned* bytes) {
  *bytes = c->blob_bytes;
  return c->blob;
}
int ctx_device(const chem_ctx* c) { return c->dev; }
// chem_advance with a skip mask: cells with skip[i] != 0 are left as they are
int ctx_advance_skip(chem_ctx* c, float* T, float* p, float* Y, int64_t ld, const float* rho, const float* e, int64_t n,
                     double dt, int32_t* substeps, const unsigned char* skip, cudaStream_t st) {
  return advance_impl<float>(c, T, p, Y, ld, rho, e, n, dt, substeps, st, skip);
}
}  // namespace chem

extern "C" {

void chem_default_params(chem_params* out) {
  if (!out) return;
  out->rtol = 1e-5;
  out->atol = 1e-10;
  out->T_min = 0.0;
  out->bulk_frac = 0.05;
  out->y_floor = 1e-10;
  out->k_bulk = 1;
  out->k_max = 100000;
  out->flags = CHEM_FLAG_ORDER_RATE;
}

int chem_init(const chem_mechanism* mech, const chem_params* params, int64_t max_cells, chem_ctx** out) {
  if (!out) return CHEM_EINVAL;
  *out = nullptr;
  int rc = check_mechanism(mech);
  if (rc) return rc;
  chem_params prm;
  chem_default_params(&prm);
  if (params) {
    if (check_params(params)) return CHEM_EINVAL;
    prm = *params;
  }
  if (max_cells < 0 || max_cells > 0x7fffffffLL) return CHEM_EINVAL;
  const bool large = mech->ns > 15;
  if (large ? !compiled_large(mech->ns) : !compiled_ns(mech->ns)) return CHEM_EUNSUPPORTED;
  chem_ctx* c = new (std::nothrow) chem_ctx();
  if (!c) return CHEM_ENOMEM;
  c->prm = prm;
  c->max_cells = max_cells;
  c->ns = mech->ns;
  c->nr = mech->nr;
  c->W.assign(mech->W, mech->W + mech->ns);
  c->nu_f.assign(mech->nu_f, mech->nu_f + static_cast<size_t>(mech->nr) * mech->ns);
  c->nu_r.assign(mech->nu_r, mech->nu_r + static_cast<size_t>(mech->nr) * mech->ns);
  c->large = large;
  auto fail = [&](int code) {
    chem_destroy(c);
    return code;
  };
  std::vector<unsigned char> blob(packed_bytes(mech, large));
  if ((rc = pack_mechanism(mech, large, blob.data(), blob.size(), &c->ntb))) return fail(rc);
  const unsigned blob_total = static_cast<unsigned>(blob.size());
  // the staged part: the whole dense blob, or the large layout's prefix (its tail stays global)
  c->blob_bytes = reinterpret_cast<const MechHdr*>(blob.data())->prefix;
  {
    const MechHdr* hdr = reinterpret_cast<const MechHdr*>(blob.data());
    c->nact = hdr->nact > 0 ? hdr->nact : hdr->ns;   // as the kernels' view of the header
  }
  if ((rc = cuda_fail(cudaGetDevice(&c->dev), "cudaGetDevice"))) return fail(rc);
  if ((rc = cuda_fail(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev), "attr"))) return fail(rc);
  if (cudaMalloc(&c->blob, blob_total) != cudaSuccess) return fail(CHEM_ENOMEM);
  if ((rc = cuda_fail(cudaMemcpy(c->blob, blob.data(), blob_total, cudaMemcpyHostToDevice), "copy mechanism")))
    return fail(rc);
  if (cudaMalloc(&c->ws, sizeof(Workspace)) != cudaSuccess) return fail(CHEM_ENOMEM);
  if (cudaMallocHost(&c->ws_host, sizeof(Workspace)) != cudaSuccess) return fail(CHEM_ENOMEM);
  std::memset(c->ws_host, 0, sizeof(Workspace));
  const int64_t qcap = max_cells > 0 ? max_cells : 1;
  if (cudaMalloc(&c->queue, sizeof(int) * qcap) != cudaSuccess) return fail(CHEM_ENOMEM);
  if (cudaMalloc(&c->queue2, sizeof(int) * qcap) != cudaSuccess) return fail(CHEM_ENOMEM);
  if (cudaMalloc(&c->qkey, qcap) != cudaSuccess) return fail(CHEM_ENOMEM);
  c->bulk_grid = c->sms * occupancy_bulk(c);
  c->stiff_grid = c->sms * occupancy_stiff(c);
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(CHEM_ECUDA);
  if ((rc = ensure_two_pass(c))) return fail(rc);
  if (large && rates_tc_supported(c->ns, c->ntb)) {
    const std::vector<unsigned char> img = rates_tc_image(mech, blob.data());
    if (cudaMalloc(&c->tc_img, img.size()) != cudaSuccess) return fail(CHEM_ENOMEM);
    if ((rc = cuda_fail(cudaMemcpy(c->tc_img, img.data(), img.size(), cudaMemcpyHostToDevice), "copy operands")))
      return fail(rc);
  }
  *out = c;
  return CHEM_OK;
}

int chem_set_params(chem_ctx* ctx, const chem_params* params) {
  if (!ctx || check_params(params)) return CHEM_EINVAL;
  const chem_params old = ctx->prm;
  ctx->prm = *params;
  const int rc = ensure_two_pass(ctx);
  if (rc) ctx->prm = old;
  return rc;
}

void chem_destroy(chem_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->dev);
  cudaDeviceSynchronize();
  cudaFree(ctx->blob);
  cudaFree(ctx->ws);
  cudaFreeHost(ctx->ws_host);
  cudaFree(ctx->queue);
  cudaFree(ctx->queue2);
  cudaFree(ctx->qkey);
  cudaFree(ctx->hbuf);
  cudaFree(ctx->hsub);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  cudaFree(ctx->boxes);
  cudaFree(ctx->box_off);
  surrogate_release(ctx->sg);
  cudaFree(ctx->cont);
  cudaFree(ctx->cont_list);
  cudaFree(ctx->cont_key);
  cudaFree(ctx->cont_sorted);
  cudaFree(ctx->xcell);
  cudaFree(ctx->tc_img);
  delete ctx;
}

int chem_advance(chem_ctx* ctx, float* T, float* p, float* Y, int64_t ld, const float* rho, const float* e,
                 int64_t n, double dt, int32_t* substeps, void* stream) {
  return advance_impl<float>(ctx, T, p, Y, ld, rho, e, n, dt, substeps, static_cast<cudaStream_t>(stream));
}

int chem_advance_explicit(chem_ctx* ctx, float* T, float* p, float* Y, int64_t ld, const float* rho, const float* e,
                          int64_t n, double dt, int32_t* substeps, int32_t k_steps, int64_t n_star,
                          int32_t* launches, void* stream) {
  if (launches) *launches = 0;
  if (!ctx || n < 0 || !(dt > 0) || !std::isfinite(dt) || k_steps < 1 || n_star < 0) return CHEM_EINVAL;
  if (ctx->large) return CHEM_EUNSUPPORTED;
  if (n > ctx->max_cells) return CHEM_ENOMEM;
  if (n > 0 && (!T || !Y || !rho || !e || !substeps || ld < n)) return CHEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = cuda_fail(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (rc) return rc;
  if (!ctx->xcell && ctx->max_cells > 0) {
    rc = cuda_fail(cudaMalloc(&ctx->xcell, sizeof(double) * (ctx->ns + 2) * ctx->max_cells), "cudaMalloc(xcell)");
    if (rc) return rc;
  }
  rc = cuda_fail(cudaMemsetAsync(ctx->ws, 0, sizeof(Workspace), st), "cudaMemsetAsync");
  if (rc) return rc;
  ctx->last_n = n;
  ctx->timed = false;
  if (n > 0) {
    AdvanceArgs<float> a{};
    a.blob = ctx->blob;
    a.blob_bytes = ctx->blob_bytes;
    a.prm = kparams(ctx->prm);
    a.T = T;
    a.p = p;
    a.Y = Y;
    a.ld = ld;
    a.rho = rho;
    a.e = e;
    a.n = n;
    a.dt = dt;
    a.substeps = substeps;
    a.ws = ctx->ws;
    a.queue = ctx->queue;
    const long long want = (n + kBulkBlock - 1) / kBulkBlock;
    const int grid = static_cast<int>(want < ctx->bulk_grid ? want : ctx->bulk_grid);
    // the active count after a launch, copied to the host (Algorithm 3, copy_device2host)
    auto active = [&](long long* out) {
      int r = cuda_fail(cudaMemcpyAsync(&ctx->ws_host->qcount, &ctx->ws->qcount, sizeof(int), cudaMemcpyDeviceToHost, st),
                        "cudaMemcpyAsync(count)");
      if (!r) r = cuda_fail(cudaStreamSynchronize(st), "cudaStreamSynchronize");
      *out = ctx->ws_host->qcount;
      return r;
    };
    // section 1: times, activity test, first active list
    int r = launch_explicit(ctx->ns, a, ctx->xcell, kExInit, 0, grid, st);
    if (r == -1) return CHEM_EUNSUPPORTED;
    if (r) return cuda_fail(static_cast<cudaError_t>(r), "kernel launch");
    long long n_active = 0;
    rc = active(&n_active);
    if (rc) return rc;
    // section 2: bulk launches of at most k_steps substeps per cell while N_active > N*; the
    // launches are capped so that no cell takes more than k_max substeps in this phase
    const long long cap = (static_cast<long long>(ctx->prm.k_max) + k_steps - 1) / k_steps;
    long long nl = 0;
    while (n_active > n_star && nl < cap) {
      rc = cuda_fail(cudaMemsetAsync(&ctx->ws->qcount, 0, sizeof(int), st), "cudaMemsetAsync");
      if (rc) return rc;
      r = launch_explicit(ctx->ns, a, ctx->xcell, kExBulk, k_steps, grid, st);
      if (r) return cuda_fail(static_cast<cudaError_t>(r), "kernel launch");
      ++nl;
      rc = active(&n_active);
      if (rc) return rc;
    }
    if (launches) *launches = static_cast<int32_t>(nl);
    // section 3: the listed active cells, at most k_max substeps each
    if (n_active > 0) {
      const long long sg = (n_active + kBulkBlock - 1) / kBulkBlock;
      r = launch_explicit(ctx->ns, a, ctx->xcell, kExSparse, ctx->prm.k_max, static_cast<int>(sg), st);
      if (r) return cuda_fail(static_cast<cudaError_t>(r), "kernel launch");
    }
  }
  rc = cuda_fail(cudaMemcpyAsync(ctx->ws_host, ctx->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync(stats)");
  if (rc) return rc;
  return cuda_fail(cudaStreamSynchronize(st), "cudaStreamSynchronize");
}

int chem_advance_f64(chem_ctx* ctx, double* T, double* p, double* Y, int64_t ld, const double* rho,
                     const double* e, int64_t n, double dt, int32_t* substeps, void* stream) {
  return advance_impl<double>(ctx, T, p, Y, ld, rho, e, n, dt, substeps, static_cast<cudaStream_t>(stream));
}

int chem_advance_host(chem_ctx* ctx, float* T, float* p, float* Y, const float* rho, const float* e, int64_t n,
                      double dt, int32_t* substeps, void* stream) {
  if (!ctx || n < 0) return CHEM_EINVAL;
  if (n > ctx->max_cells) return CHEM_ENOMEM;
  if (n == 0) return CHEM_OK;
  if (!T || !Y || !rho || !e || !substeps) return CHEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = cuda_fail(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (rc) return rc;
  const int64_t cap = ctx->max_cells;
  if (!ctx->hbuf) {
    if (cudaMalloc(&ctx->hbuf, sizeof(float) * cap * (ctx->ns + 4)) != cudaSuccess) return CHEM_ENOMEM;
    if (cudaMalloc(&ctx->hsub, sizeof(int) * cap) != cudaSuccess) return CHEM_ENOMEM;
  }
  float* dT = ctx->hbuf;
  float* dp = dT + cap;
  float* drho = dp + cap;
  float* de = drho + cap;
  float* dY = de + cap;
  const size_t b = sizeof(float) * n;
  if ((rc = cuda_fail(cudaMemcpyAsync(dT, T, b, cudaMemcpyHostToDevice, st), "H2D T"))) return rc;
  if ((rc = cuda_fail(cudaMemcpyAsync(drho, rho, b, cudaMemcpyHostToDevice, st), "H2D rho"))) return rc;
  if ((rc = cuda_fail(cudaMemcpyAsync(de, e, b, cudaMemcpyHostToDevice, st), "H2D e"))) return rc;
  if ((rc = cuda_fail(cudaMemcpyAsync(dY, Y, b * ctx->ns, cudaMemcpyHostToDevice, st), "H2D Y"))) return rc;
  if (p && (rc = cuda_fail(cudaMemcpyAsync(dp, p, b, cudaMemcpyHostToDevice, st), "H2D p"))) return rc;
  rc = chem_advance(ctx, dT, p ? dp : nullptr, dY, n, drho, de, n, dt, ctx->hsub, stream);
  if (rc) return rc;
  if ((rc = cuda_fail(cudaMemcpyAsync(T, dT, b, cudaMemcpyDeviceToHost, st), "D2H T"))) return rc;
  if ((rc = cuda_fail(cudaMemcpyAsync(Y, dY, b * ctx->ns, cudaMemcpyDeviceToHost, st), "D2H Y"))) return rc;
  if (p && (rc = cuda_fail(cudaMemcpyAsync(p, dp, b, cudaMemcpyDeviceToHost, st), "D2H p"))) return rc;
  if ((rc = cuda_fail(cudaMemcpyAsync(substeps, ctx->hsub, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "D2H n")))
    return rc;
  return cuda_fail(cudaStreamSynchronize(st), "cudaStreamSynchronize");
}

int chem_boxes_set(chem_ctx* ctx, const chem_box* boxes, int32_t nbox) {
  if (!ctx || nbox < 1 || nbox > kMaxBoxes || !boxes) return CHEM_EINVAL;
  std::vector<DevBox<float>> tab(nbox);
  std::vector<int> off(nbox + 1);
  int64_t total = 0;
  for (int b = 0; b < nbox; ++b) {
    const chem_box& x = boxes[b];
    if (x.n < 0 || (x.n > 0 && (!x.T || !x.Y || !x.rho || !x.e || !x.substeps || x.ld < x.n)) || !(x.dt > 0) ||
        !std::isfinite(x.dt))
      return CHEM_EINVAL;
    tab[b].T = x.T;
    tab[b].p = x.p;
    tab[b].Y = x.Y;
    tab[b].rho = x.rho;
    tab[b].e = x.e;
    tab[b].substeps = x.substeps;
    tab[b].ld = x.ld;
    tab[b].n = x.n;
    tab[b].off = total;
    tab[b].dt = x.dt;
    tab[b].level = x.level;
    tab[b].pad = 0;
    off[b] = static_cast<int>(total);
    total += x.n;
    if (total > ctx->max_cells) return CHEM_ENOMEM;
  }
  off[nbox] = static_cast<int>(total);
  int rc = cuda_fail(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (rc) return rc;
  cudaDeviceSynchronize();   // the previous table may be in use by queued work
  if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  cudaFree(ctx->boxes);
  cudaFree(ctx->box_off);
  ctx->boxes = nullptr;
  ctx->box_off = nullptr;
  ctx->nbox = 0;
  if (cudaMalloc(&ctx->boxes, sizeof(DevBox<float>) * nbox) != cudaSuccess) return CHEM_ENOMEM;
  if (cudaMalloc(&ctx->box_off, sizeof(int) * (nbox + 1)) != cudaSuccess) return CHEM_ENOMEM;
  if ((rc = cuda_fail(cudaMemcpy(ctx->boxes, tab.data(), sizeof(DevBox<float>) * nbox, cudaMemcpyHostToDevice),
                      "copy box table")))
    return rc;
  if ((rc = cuda_fail(cudaMemcpy(ctx->box_off, off.data(), sizeof(int) * (nbox + 1), cudaMemcpyHostToDevice),
                      "copy box offsets")))
    return rc;
  ctx->nbox = nbox;
  ctx->box_cells = total;
  return CHEM_OK;
}

int chem_advance_boxes(chem_ctx* ctx, void* stream) {
  if (!ctx || ctx->nbox < 1) return CHEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = cuda_fail(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (rc) return rc;
  if ((rc = cuda_fail(cudaMemsetAsync(ctx->ws, 0, sizeof(Workspace), st), "cudaMemsetAsync"))) return rc;
  ctx->last_n = ctx->box_cells;
  ctx->timed = false;
  const int64_t n = ctx->box_cells;
  if (n > 0) {
    AdvanceArgs<float> a{};
    a.blob = ctx->blob;
    a.blob_bytes = ctx->blob_bytes;
    a.prm = kparams(ctx->prm);
    a.n = n;
    a.ws = ctx->ws;
    a.queue = ctx->queue;
    a.boxes = ctx->boxes;
    a.box_off = ctx->box_off;
    a.nbox = ctx->nbox;
    const bool order = (ctx->prm.flags & (CHEM_FLAG_ORDER_RATE | CHEM_FLAG_ORDER_PREV)) != 0;
    a.qkey = order ? ctx->qkey : nullptr;
    AdvanceArgs<float> b = a;
    if (order) b.queue = ctx->queue2;
    long long want = (n + kBulkBlock - 1) / kBulkBlock;
    const int bgrid = static_cast<int>(want < ctx->bulk_grid ? (want < 1 ? 1 : want) : ctx->bulk_grid);
    int r1, r2;
    if (ctx->large) {
      const long long wb = (n + 7) / 8;
      const int lgrid = static_cast<int>(wb < ctx->bulk_grid ? (wb < 1 ? 1 : wb) : ctx->bulk_grid);
      r1 = launch_bulk_lg(ctx->ns, ctx->nr, ctx->ntb, a, lgrid, st);
      if (!r1 && order) r1 = launch_order_queue(ctx->ws, ctx->queue, ctx->qkey, ctx->queue2, n, st);
      r2 = r1 ? r1 : launch_stiff_lg(ctx->ns, ctx->nact, ctx->nr, ctx->ntb, b, ctx->stiff_grid, st);
    } else {
      r1 = launch_bulk_f32(ctx->ns, a, bgrid, st);
      if (!r1 && order) r1 = launch_order_queue(ctx->ws, ctx->queue, ctx->qkey, ctx->queue2, n, st);
      r2 = r1 ? r1 : launch_stiff_phase<float>(ctx, b, n, st);
    }
    if (r1 == -1 || r2 == -1) return CHEM_EUNSUPPORTED;
    if (r1 || r2) return cuda_fail(static_cast<cudaError_t>(r1 ? r1 : r2), "kernel launch");
  }
  return cuda_fail(cudaMemcpyAsync(ctx->ws_host, ctx->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st),
                   "cudaMemcpyAsync(stats)");
}

int chem_boxes_capture(chem_ctx* ctx, void* stream) {
  if (!ctx || ctx->nbox < 1 || (ctx->prm.flags & CHEM_FLAG_TIMING)) return CHEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) return CHEM_EINVAL;   // capture needs a non-default stream
  int rc = cuda_fail(cudaSetDevice(ctx->dev), "cudaSetDevice");
  if (rc) return rc;
  if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  if ((rc = cuda_fail(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"))) return rc;
  const int adv = chem_advance_boxes(ctx, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &g);
  if (adv) {
    if (g) cudaGraphDestroy(g);
    return adv;
  }
  if ((rc = cuda_fail(ec, "end capture"))) return rc;
  ctx->graph = g;
  return cuda_fail(cudaGraphInstantiate(&ctx->graph_exec, g, 0), "graph instantiate");
}

int chem_boxes_launch(chem_ctx* ctx, void* stream) {
  if (!ctx || !ctx->graph_exec) return CHEM_EINVAL;
  ctx->last_n = ctx->box_cells;
  ctx->timed = false;
  return cuda_fail(cudaGraphLaunch(ctx->graph_exec, static_cast<cudaStream_t>(stream)), "graph launch");
}

int chem_state_from_TpY(chem_ctx* ctx, const float* T, const float* p, const float* Y, int64_t ld, int64_t n,
                        float* rho, float* e, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!T || !p || !Y || !rho || !e || ld < n))) return CHEM_EINVAL;
  if (n == 0) return CHEM_OK;
  const int r = launch_state_from_TpY_f32(ctx->ns, ctx->blob, ctx->blob_bytes, T, p, Y, ld, n, rho, e,
                                          &ctx->ws->status, static_cast<cudaStream_t>(stream));
  return r == -1 ? CHEM_EUNSUPPORTED : cuda_fail(static_cast<cudaError_t>(r), "state kernel");
}

int chem_state_from_TpY_f64(chem_ctx* ctx, const double* T, const double* p, const double* Y, int64_t ld,
                            int64_t n, double* rho, double* e, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!T || !p || !Y || !rho || !e || ld < n))) return CHEM_EINVAL;
  if (n == 0) return CHEM_OK;
  const int r = launch_state_from_TpY_f64(ctx->ns, ctx->blob, ctx->blob_bytes, T, p, Y, ld, n, rho, e,
                                          &ctx->ws->status, static_cast<cudaStream_t>(stream));
  return r == -1 ? CHEM_EUNSUPPORTED : cuda_fail(static_cast<cudaError_t>(r), "state kernel");
}

int chem_temperature(chem_ctx* ctx, const float* Y, int64_t ld, const float* e, int64_t n, float* T, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!Y || !e || !T || ld < n))) return CHEM_EINVAL;
  if (n == 0) return CHEM_OK;
  const int r = launch_temperature(ctx->ns, ctx->blob, ctx->blob_bytes, Y, ld, e, n, T, &ctx->ws->status,
                                   static_cast<cudaStream_t>(stream));
  return r == -1 ? CHEM_EUNSUPPORTED : cuda_fail(static_cast<cudaError_t>(r), "temperature kernel");
}

int chem_rates(chem_ctx* ctx, const float* rho, const float* T, const float* Y, int64_t ld, int64_t n, float* dYdt,
               void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!rho || !T || !Y || !dYdt || ld < n))) return CHEM_EINVAL;
  if (n == 0) return CHEM_OK;
  const int r = ctx->large ? launch_rates_lg(ctx->ns, ctx->nr, ctx->ntb, ctx->blob, ctx->blob_bytes, rho, T, Y, ld, n,
                                             dYdt, &ctx->ws->status, static_cast<cudaStream_t>(stream))
                           : launch_rates(ctx->ns, ctx->blob, ctx->blob_bytes, rho, T, Y, ld, n, dYdt,
                                          &ctx->ws->status, static_cast<cudaStream_t>(stream));
  return r == -1 ? CHEM_EUNSUPPORTED : cuda_fail(static_cast<cudaError_t>(r), "rates kernel");
}

int chem_rates_tc(chem_ctx* ctx, const float* rho, const float* T, const float* Y, int64_t ld, int64_t n,
                  float* dYdt, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!rho || !T || !Y || !dYdt || ld < n))) return CHEM_EINVAL;
  if (!ctx->tc_img) return CHEM_EUNSUPPORTED;
  if (n == 0) return CHEM_OK;
  const int r = launch_rates_tc(ctx->ns, ctx->nr, ctx->ntb, ctx->tc_img, ctx->blob, rho, T, Y, ld, n, dYdt, &ctx->ws->status,
                                static_cast<cudaStream_t>(stream));
  return r == -1 ? CHEM_EUNSUPPORTED : cuda_fail(static_cast<cudaError_t>(r), "tensor-core rates kernel");
}

int chem_status(chem_ctx* ctx, void* stream, chem_stats* out) {
  if (!ctx || !out) return CHEM_EINVAL;
  int rc = cuda_fail(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "cudaStreamSynchronize");
  if (rc) return rc;
  const Workspace& w = *ctx->ws_host;
  out->ncell = ctx->last_n;
  out->nskipped = static_cast<int64_t>(w.nskipped);
  out->nbulk = static_cast<int64_t>(w.nbulk);
  out->nqueued = w.qcount;
  out->nfailed = static_cast<int64_t>(w.nfailed);
  out->ninvalid = static_cast<int64_t>(w.ninvalid);
  out->substeps = static_cast<int64_t>(w.substeps);
  out->attempts = static_cast<int64_t>(w.attempts);
  out->newton = static_cast<int64_t>(w.newton);
  // the dense stiff kernel factors on every attempt; the large one counts what it factors
  out->factorizations = ctx->large ? static_cast<int64_t>(w.factorizations) : out->attempts;
  out->bulk_ms = 0.0f;
  out->stiff_ms = 0.0f;
  if (ctx->timed) {
    cudaEventElapsedTime(&out->bulk_ms, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&out->stiff_ms, ctx->ev[1], ctx->ev[2]);
  }
  int status = CHEM_OK;
  if (w.status & kFlagInvalid) status = CHEM_EINVAL;
  if (w.status & (kFlagNoConv | kFlagTemp)) status = CHEM_ENOCONV;
  if (w.status & kFlagMaxSteps) status = CHEM_EMAXSTEPS;
  if (w.status & kFlagStage) status = CHEM_ECUDA;
  out->status = status;
  return CHEM_OK;
}

const char* chem_strerror(int code) {
  switch (code) {
    case CHEM_OK: return "ok";
    case CHEM_EINVAL: return "invalid argument or input cell";
    case CHEM_ENOMEM: return "more cells than max_cells, or device allocation failed";
    case CHEM_EMAXSTEPS: return "a stiff cell reached k_max substeps";
    case CHEM_ENOCONV: return "a stiff cell did not converge (step size collapsed or T(e) failed)";
    case CHEM_ECUDA: return "CUDA runtime error";
    case CHEM_EUNSUPPORTED: return "no kernel compiled for this mechanism shape";
    default: return "unknown status";
  }
}

}  // extern "C"
