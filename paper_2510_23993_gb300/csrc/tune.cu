// tune.cu -- chem_tune: pick the launch configuration of chem_advance by timed trials.
//
// The paper tuned its bulk-step count (K_max = 5) and its bulk-to-sparse threshold by hand
// (Sec. 3.2, App. D).  Here the knobs are the explicit bulk substeps per cell (k_bulk), the
// order in which stiff cells are handed to the persistent kernel (none, by rate, by rate with the
// two-pass probe/continuation schedule), the resident blocks per SM of both kernels, and for the
// dense stiff kernel its CTA size (64, 128 or 256 threads, one cell per thread) and the
// scheduling quantum of the two-pass schedule (attempts per cell in the probe pass and in each
// continuation round: 16, 32 or 64).  None of them changes a cell's result, only the launch
// shape and the order of work.  The tuner times chem_advance on the caller's field for each candidate
// (coordinate descent, best of two repetitions, inputs restored between trials), keeps the
// fastest, and can cache the choice in a text file keyed by mechanism shape, field size and GPU.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/chem.h"
#include "internal.h"

struct chem_ctx;
namespace chem {
// accessors of the context's launch settings (abi.cu)
void ctx_get_launch(const chem_ctx* c, int* bulk_grid, int* stiff_grid, int* sms, int* ns, int* nr);
void ctx_set_launch(chem_ctx* c, int bulk_grid, int stiff_grid);
void ctx_get_params(const chem_ctx* c, chem_params* p);
void ctx_get_sched(const chem_ctx* c, int* stiff_block, int* probe_att, int* round_att, int* large);
void ctx_set_sched(chem_ctx* c, int stiff_block, int probe_att, int round_att);
int occupancy_bulk(const chem_ctx* c);
int occupancy_stiff(const chem_ctx* c);
}  // namespace chem

namespace {

struct Choice {
  int k_bulk, order_flags, bulk_bpsm, stiff_bpsm, stiff_block, quantum;
};

std::string cache_key(int ns, int nr, int64_t n, double dt) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  std::string name(prop.name);
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  std::snprintf(buf, sizeof(buf), "ns=%d nr=%d log2n=%d dt=%.3e dev=%s", ns, nr,
                static_cast<int>(std::floor(std::log2(static_cast<double>(n > 1 ? n : 1)))), dt, name.c_str());
  return std::string(buf);
}

bool cache_lookup(const char* path, const std::string& key, Choice* c) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    const char* bar = std::strstr(line, " | ");
    if (!bar || std::string(line, bar - line) != key) continue;
    Choice t;
    if (std::sscanf(bar + 3, "k_bulk=%d order=%d bulk_bpsm=%d stiff_bpsm=%d stiff_block=%d quantum=%d", &t.k_bulk,
                    &t.order_flags, &t.bulk_bpsm, &t.stiff_bpsm, &t.stiff_block, &t.quantum) == 6) {
      // a hand-edited line with a CTA size or quantum the kernel does not offer is ignored
      if ((t.stiff_block == 64 || t.stiff_block == 128 || t.stiff_block == 256) && t.quantum >= 1 &&
          t.quantum <= 1024 && t.stiff_bpsm >= 1 && t.bulk_bpsm >= 1) {
        *c = t;
        found = true;   // the last matching line wins
      }
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const Choice& c) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s | k_bulk=%d order=%d bulk_bpsm=%d stiff_bpsm=%d stiff_block=%d quantum=%d\n", key.c_str(),
               c.k_bulk, c.order_flags, c.bulk_bpsm, c.stiff_bpsm, c.stiff_block, c.quantum);
  std::fclose(f);
}

}  // namespace

extern "C" int chem_tune(chem_ctx* ctx, float* T, float* p, float* Y, int64_t ld, const float* rho, const float* e,
                         int64_t n, double dt, int32_t* substeps, const char* cache_path, chem_tune_result* out,
                         void* stream) {
  using namespace chem;
  if (!ctx || !out || n < 1 || !T || !Y || !rho || !e || !substeps || ld < n || !(dt > 0)) return CHEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int bulk_grid0, stiff_grid0, sms, ns, nr;
  ctx_get_launch(ctx, &bulk_grid0, &stiff_grid0, &sms, &ns, &nr);
  chem_params prm0;
  ctx_get_params(ctx, &prm0);
  int block0, probe0, round0, large;
  ctx_get_sched(ctx, &block0, &probe0, &round0, &large);
  const int occ_b = occupancy_bulk(ctx), occ_s = occupancy_stiff(ctx);
  std::memset(out, 0, sizeof(*out));
  const std::string key = cache_key(ns, nr, n, dt);
  auto apply = [&](const Choice& c) {
    chem_params p = prm0;
    p.k_bulk = c.k_bulk;
    p.flags = (prm0.flags & ~(CHEM_FLAG_ORDER_RATE | CHEM_FLAG_ORDER_PREV | CHEM_FLAG_TWO_PASS)) | c.order_flags;
    if (chem_set_params(ctx, &p) != CHEM_OK) {   // two-pass storage unavailable: keep the one-pass order
      p.flags &= ~CHEM_FLAG_TWO_PASS;
      chem_set_params(ctx, &p);
    }
    ctx_set_sched(ctx, c.stiff_block, c.quantum, c.quantum);
    ctx_set_launch(ctx, sms * c.bulk_bpsm, sms * c.stiff_bpsm);
  };
  Choice best{prm0.k_bulk, prm0.flags & (CHEM_FLAG_ORDER_RATE | CHEM_FLAG_ORDER_PREV | CHEM_FLAG_TWO_PASS),
              bulk_grid0 / sms, stiff_grid0 / sms, block0, probe0};
  if (cache_lookup(cache_path, key, &best)) {
    apply(best);
    out->k_bulk = best.k_bulk;
    out->flags = best.order_flags;
    out->bulk_blocks_per_sm = best.bulk_bpsm;
    out->stiff_blocks_per_sm = best.stiff_bpsm;
    out->stiff_block = best.stiff_block;
    out->quantum = best.quantum;
    out->from_cache = 1;
    return CHEM_OK;
  }
  // backups of the in/out state so that every trial starts from the caller's input
  float *bT = nullptr, *bY = nullptr, *bp = nullptr;
  const size_t nb = sizeof(float) * static_cast<size_t>(n);
  auto cleanup = [&]() {
    cudaFree(bT);
    cudaFree(bY);
    cudaFree(bp);
  };
  if (cudaMalloc(&bT, nb) != cudaSuccess || cudaMalloc(&bY, sizeof(float) * static_cast<size_t>(ld) * ns) != cudaSuccess ||
      (p && cudaMalloc(&bp, nb) != cudaSuccess)) {
    cleanup();
    return CHEM_ENOMEM;
  }
  cudaMemcpyAsync(bT, T, nb, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(bY, Y, sizeof(float) * static_cast<size_t>(ld) * ns, cudaMemcpyDeviceToDevice, st);
  if (p) cudaMemcpyAsync(bp, p, nb, cudaMemcpyDeviceToDevice, st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto restore = [&]() {
    cudaMemcpyAsync(T, bT, nb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(Y, bY, sizeof(float) * static_cast<size_t>(ld) * ns, cudaMemcpyDeviceToDevice, st);
    if (p) cudaMemcpyAsync(p, bp, nb, cudaMemcpyDeviceToDevice, st);
  };
  int rc = CHEM_OK;
  auto time_choice = [&](const Choice& c) -> float {
    apply(c);
    float bestms = 1e30f;
    for (int rep = 0; rep < 2 && rc == CHEM_OK; ++rep) {
      restore();
      cudaEventRecord(e0, st);
      rc = chem_advance(ctx, T, p, Y, ld, rho, e, n, dt, substeps, stream);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = CHEM_ECUDA;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < bestms) bestms = ms;
      ++out->trials;
    }
    return bestms;
  };
  const float t_default = time_choice(best);
  float t_best = t_default;
  auto consider = [&](Choice c) {
    if (rc != CHEM_OK) return;
    const float t = time_choice(c);
    if (t < t_best) {
      t_best = t;
      best = c;
    }
  };
  // coordinate descent over the knobs, most influential first
  for (int s = 1; s <= occ_s; ++s)
    if (s != best.stiff_bpsm) {
      Choice c = best;
      c.stiff_bpsm = s;
      consider(c);
    }
  for (int ord : {0, static_cast<int>(CHEM_FLAG_ORDER_RATE), static_cast<int>(CHEM_FLAG_ORDER_RATE | CHEM_FLAG_TWO_PASS)})
    if (ord != best.order_flags) {
      Choice c = best;
      c.order_flags = ord;
      consider(c);
    }
  for (int kb = 1; kb <= 3; ++kb)
    if (kb != best.k_bulk) {
      Choice c = best;
      c.k_bulk = kb;
      consider(c);
    }
  for (int b : {occ_b, occ_b > 1 ? occ_b / 2 : 1, 2 * occ_b})
    if (b != best.bulk_bpsm) {
      Choice c = best;
      c.bulk_bpsm = b;
      consider(c);
    }
  if (!large) {
    // CTA size of the stiff kernel, each with the most resident blocks that fit
    for (int blk : {64, 128, 256})
      if (blk != best.stiff_block) {
        Choice c = best;
        c.stiff_block = blk;
        ctx_set_sched(ctx, blk, c.quantum, c.quantum);
        c.stiff_bpsm = occupancy_stiff(ctx);
        consider(c);
      }
    // scheduling quantum of the two-pass schedule
    if (best.order_flags & CHEM_FLAG_TWO_PASS)
      for (int qa : {16, 32, 64})
        if (qa != best.quantum) {
          Choice c = best;
          c.quantum = qa;
          consider(c);
        }
  }
  apply(best);
  restore();   // leave the caller's state as it came in
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cleanup();
  if (rc != CHEM_OK) return rc;
  cache_store(cache_path, key, best);
  out->k_bulk = best.k_bulk;
  out->flags = best.order_flags;
  out->bulk_blocks_per_sm = best.bulk_bpsm;
  out->stiff_blocks_per_sm = best.stiff_bpsm;
  out->stiff_block = best.stiff_block;
  out->quantum = best.quantum;
  out->best_ms = t_best;
  out->default_ms = t_default;
  return CHEM_OK;
}
