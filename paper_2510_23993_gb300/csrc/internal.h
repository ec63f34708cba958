// internal.h -- host/device contract between the C ABI (abi.cu) and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace chem {

// Device workspace of one context (counters of the current call; zeroed before each call).
struct Workspace {
  int qcount;                    // cells compacted into the stiff queue by the bulk kernel
  int head;                      // next queue slot handed out by the stiff kernel
  int status;                    // OR of kFlag* bits
  int pad;
  unsigned long long nskipped, nbulk, ninvalid, nfailed, substeps, attempts, newton;
};

struct KParams {
  float rtol, atol, T_min, bulk_frac, y_floor;
  int k_bulk, k_max, flags;
};

template <typename S>
struct AdvanceArgs {
  const unsigned char* blob;     // packed mechanism (global, 16-byte aligned)
  unsigned blob_bytes;           // multiple of 16
  KParams prm;
  S* T;
  S* p;
  S* Y;
  long long ld;
  const S* rho;
  const S* e;
  long long n;
  double dt;
  int* substeps;
  Workspace* ws;
  int* queue;                    // [max_cells]
  unsigned char* qkey;           // [max_cells] cost bucket of each queue entry, or null (no ordering)
};

// cost keys of the stiff queue (chem_params.flags bits, see include/chem.h)
constexpr int kFlagOrderRate = 4;   // bucket of log2(dt * sum_k |dY_k/dt|) at the bulk step
constexpr int kFlagOrderPrev = 8;   // bucket of log2 of the cell's substep count of the previous call
constexpr int kNumBuckets = 64;

constexpr int kBulkBlock = 128;
constexpr int kStiffBlock = 128;

// launchers (kernels.cu / stiff.cu); return cudaError_t as int, or -1 for unsupported ns
int launch_bulk_f32(int ns, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_bulk_f64(int ns, const AdvanceArgs<double>& a, int grid, cudaStream_t s);
int launch_stiff_f32(int ns, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_stiff_f64(int ns, const AdvanceArgs<double>& a, int grid, cudaStream_t s);
size_t stiff_smem_bytes(int ns, unsigned blob_bytes);
// counting sort of the queue by cost bucket, most expensive first: queue -> queue_out
int launch_order_queue(Workspace* ws, const int* queue, const unsigned char* qkey, int* queue_out,
                       long long n, cudaStream_t s);
size_t bulk_smem_bytes(unsigned blob_bytes);
int stiff_occupancy(int ns, unsigned blob_bytes, int* blocks_per_sm);
int bulk_occupancy(int ns, bool f64, unsigned blob_bytes, int* blocks_per_sm);

int launch_state_from_TpY_f32(int ns, const unsigned char* blob, unsigned blob_bytes, const float* T,
                              const float* p, const float* Y, long long ld, long long n, float* rho,
                              float* e, int* status, cudaStream_t s);
int launch_state_from_TpY_f64(int ns, const unsigned char* blob, unsigned blob_bytes, const double* T,
                              const double* p, const double* Y, long long ld, long long n,
                              double* rho, double* e, int* status, cudaStream_t s);
int launch_temperature(int ns, const unsigned char* blob, unsigned blob_bytes, const float* Y,
                       long long ld, const float* e, long long n, float* T, int* status,
                       cudaStream_t s);
int launch_rates(int ns, const unsigned char* blob, unsigned blob_bytes, const float* rho,
                 const float* T, const float* Y, long long ld, long long n, float* dYdt,
                 int* status, cudaStream_t s);

}  // namespace chem
