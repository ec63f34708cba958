// internal.h -- host/device contract between the C ABI (abi.cu) and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/chem.h"

namespace chem {

// Device workspace of one context (counters of the current call; zeroed before each call).
struct Workspace {
  int qcount;                    // cells compacted into the stiff queue by the bulk kernel
  int head;                      // next queue slot handed out by the stiff kernel
  int status;                    // OR of kFlag* bits
  int cont_count;                // two-pass mode: cells the probe pass left unfinished
  int head2;                     // two-pass mode: next slot of the sorted continuation list (round 0)
  int rc[3];                     // two-pass mode: cells left after continuation round r, in rc[r % 3]
  unsigned bar_count, bar_gen;   // grid barrier of the continuation rounds
  unsigned long long nskipped, nbulk, ninvalid, nfailed, substeps, attempts, newton;
};

struct KParams {
  float rtol, atol, T_min, bulk_frac, y_floor;
  int k_bulk, k_max, flags;
};

// One AMR box of a box-table advance: the box's own SoA arrays and its chemistry step.
template <typename S>
struct DevBox {
  S* T;
  S* p;
  S* Y;
  const S* rho;
  const S* e;
  int* substeps;
  long long ld, n, off;          // leading dimension, cells, first global cell index
  double dt;                     // chemistry step of the box (dt0 / r^level under subcycling)
  int level, pad;
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
  const DevBox<S>* boxes;        // box table (nbox > 0): global cell g lives in the box whose
  const int* box_off;            //   [off_b, off_b + n_b) range; box_off[b] = off_b, b <= nbox
  int nbox;                      // 0: flat arrays T, p, Y, rho, e, substeps of n cells, step dt
  const unsigned char* skip;     // [n] or null: cells with skip[g] != 0 are left untouched (their
                                 //   step was taken elsewhere, e.g. by the surrogate)
  // two-pass stiff integration (0: single pass; 1: probe pass; 2: continuation rounds)
  int pass;
  long long cont_cap;            // capacity of the continuation arrays (queue slots)
  double* cont;                  // SoA continuation state by queue slot: y[NS], t, h, T, eta
                                 //   (each [cont_cap] doubles), then float c_v/R, int nst, int natt
  int* cont_list;                // [cont_cap] queue slots of the unfinished cells (probe pass),
                                 //   later the input of odd continuation rounds
  unsigned char* cont_key;       // [cont_cap] their remaining-work bucket
  int* cont_sorted;              // [cont_cap] the same slots, longest remaining first: the input of
                                 //   round 0, later of even rounds
};

constexpr int kMaxBoxes = 4096;

// Where cell g lives: flat arrays, or the box found by binary search over the box offsets
// (staged in shared memory as soff[0..nbox]).
template <typename S>
struct CellRef {
  S* T;
  S* p;
  S* Y;
  const S* rho;
  const S* e;
  int* sub;
  long long ld, i;
  double dt;
};

template <typename S>
__device__ __forceinline__ CellRef<S> locate(const AdvanceArgs<S>& a, const int* soff, long long g) {
  CellRef<S> r;
  if (a.nbox == 0) {
    r.T = a.T;
    r.p = a.p;
    r.Y = a.Y;
    r.rho = a.rho;
    r.e = a.e;
    r.sub = a.substeps;
    r.ld = a.ld;
    r.i = g;
    r.dt = a.dt;
    return r;
  }
  int lo = 0, hi = a.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (static_cast<long long>(soff[mid]) <= g) lo = mid; else hi = mid - 1;
  }
  const DevBox<S>& b = a.boxes[lo];
  r.T = b.T;
  r.p = b.p;
  r.Y = b.Y;
  r.rho = b.rho;
  r.e = b.e;
  r.sub = b.substeps;
  r.ld = b.ld;
  r.i = g - soff[lo];
  r.dt = b.dt;
  return r;
}

// Copy the box offsets into shared memory (all threads of the block call it).
__device__ __forceinline__ void stage_box_offsets(int* soff, const int* off, int nbox) {
  for (int b = threadIdx.x; b <= nbox; b += blockDim.x) soff[b] = off[b];
  __syncthreads();
}

__host__ __device__ inline unsigned box_smem_bytes(int nbox) { return nbox > 0 ? ((4u * (nbox + 1) + 127u) & ~127u) : 0u; }

// cost keys of the stiff queue (chem_params.flags bits, see include/chem.h)
constexpr int kFlagOrderRate = 4;   // bucket of log2(dt * sum_k |dY_k/dt|) at the bulk step
constexpr int kFlagOrderPrev = 8;   // bucket of log2 of the cell's substep count of the previous call
constexpr int kFlagTwoPass = 16;    // two-pass stiff integration
constexpr int kNumBuckets = 64;
constexpr int kProbeAttempts = 32;  // implicit steps per cell in the probe pass
constexpr int kRoundAttempts = 32;  // implicit steps per cell and continuation round

// bytes of continuation state per queue slot
__host__ __device__ constexpr long long cont_bytes_per_slot(int ns) { return 8LL * (ns + 4) + 12; }

constexpr int kBulkBlock = 128;
constexpr int kStiffBlock = 128;

// species count up to which a mechanism uses the dense table layout (thread per cell); larger
// mechanisms use the sparse layout and the warp-per-cell kernels of large.cu
constexpr int kDenseMaxNs = 15;

// host-side checks and table packing (pack.cu), shared by every entry point that takes a mechanism
int check_mechanism(const chem_mechanism* m);   // CHEM_OK or CHEM_EINVAL
int check_params(const chem_params* p);         // CHEM_OK or CHEM_EINVAL
unsigned packed_bytes(const chem_mechanism* m, bool large);
// Writes the tables of m (dense or large layout) into out[0, packed_bytes) after zeroing it.
// CHEM_ENOMEM if cap is too small, CHEM_EUNSUPPORTED for a shape the layout cannot hold; *ntb_out
// (may be null) receives the number of third-body reactions.
int pack_mechanism(const chem_mechanism* m, bool large, unsigned char* out, size_t cap, int* ntb_out);

// launchers (kernels.cu / stiff.cu); return cudaError_t as int, or -1 for unsupported ns
int launch_bulk_f32(int ns, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_bulk_f64(int ns, const AdvanceArgs<double>& a, int grid, cudaStream_t s);
int launch_stiff_f32(int ns, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_stiff_f64(int ns, const AdvanceArgs<double>& a, int grid, cudaStream_t s);
size_t stiff_smem_bytes(int ns, unsigned blob_bytes, int nbox);
// counting sort of the queue by cost bucket, most expensive first: queue -> queue_out
int launch_order_queue(Workspace* ws, const int* queue, const unsigned char* qkey, int* queue_out,
                       long long n, cudaStream_t s, bool continuations = false);
size_t bulk_smem_bytes(unsigned blob_bytes, int nbox);
int stiff_occupancy(int ns, unsigned blob_bytes, int* blocks_per_sm);
int bulk_occupancy(int ns, bool f64, unsigned blob_bytes, int* blocks_per_sm);

// the paper's explicit integration loop (explicit.cu)
constexpr int kExInit = 0, kExBulk = 1, kExSparse = 2;
int launch_explicit(int ns, const AdvanceArgs<float>& a, double* tcell, int mode, int max_sub, int grid,
                    cudaStream_t s);

// large mechanisms (large.cu): one warp per cell, sparse stoichiometry
bool compiled_large(int ns);
int launch_bulk_lg(int ns, int nr, int ntb, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_stiff_lg(int ns, int nr, int ntb, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_rates_lg(int ns, int nr, int ntb, const unsigned char* blob, unsigned bytes, const float* rho,
                    const float* T, const float* Y, long long ld, long long n, float* dYdt, int* status,
                    cudaStream_t s);
int occupancy_lg(int ns, int nr, int ntb, unsigned prefix, bool stiff, int* blocks_per_sm);

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
