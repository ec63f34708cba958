// kernel_abi.cuh -- the structures the host passes to the chemistry kernels (counters, launch
// parameters, box table) and the device helpers that read them.  Self-contained (no host headers).
#pragma once

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
  unsigned long long factorizations;   // LU factorisations (the large kernel reuses some across steps)
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

// default scheduling quanta of the two-pass stiff integration (chem_tune may change them; the
// results do not depend on them)
constexpr int kProbeAttempts = 32;  // implicit steps per cell in the probe pass
constexpr int kRoundAttempts = 32;  // implicit steps per cell and continuation round

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
  int probe_att = kProbeAttempts;   // attempts per cell in the probe pass
  int round_att = kRoundAttempts;   // attempts per cell and continuation round
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

// bytes of continuation state per queue slot
__host__ __device__ constexpr long long cont_bytes_per_slot(int ns) { return 8LL * (ns + 4) + 12; }

constexpr int kBulkBlock = 128;
constexpr int kStiffBlock = 128;      // default threads per CTA of the dense stiff kernel
constexpr int kStiffBlockMax = 256;   // largest CTA the tuner may choose (64, 128 or 256)

}  // namespace chem
