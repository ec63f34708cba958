// internal.h -- host/device contract between the C ABI (abi.cu) and the kernels.
#pragma once
#include <vector>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/chem.h"
#include "kernel_abi.cuh"

namespace chem {

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
int launch_stiff_f32(int ns, const AdvanceArgs<float>& a, int grid, int block, cudaStream_t s);
int launch_stiff_f64(int ns, const AdvanceArgs<double>& a, int grid, int block, cudaStream_t s);
size_t stiff_smem_bytes(int ns, unsigned blob_bytes, int nbox, int block);
// counting sort of the queue by cost bucket, most expensive first: queue -> queue_out
int launch_order_queue(Workspace* ws, const int* queue, const unsigned char* qkey, int* queue_out,
                       long long n, cudaStream_t s, bool continuations = false);
size_t bulk_smem_bytes(unsigned blob_bytes, int nbox);
int stiff_occupancy(int ns, unsigned blob_bytes, int block, int* blocks_per_sm);
int bulk_occupancy(int ns, bool f64, unsigned blob_bytes, int* blocks_per_sm);

// the paper's explicit integration loop (explicit.cu)
constexpr int kExInit = 0, kExBulk = 1, kExSparse = 2;
int launch_explicit(int ns, const AdvanceArgs<float>& a, double* tcell, int mode, int max_sub, int grid,
                    cudaStream_t s);

// large mechanisms (large.cu): one warp per cell, sparse stoichiometry
bool compiled_large(int ns);
int launch_bulk_lg(int ns, int nr, int ntb, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_stiff_lg(int ns, int na, int nr, int ntb, const AdvanceArgs<float>& a, int grid, cudaStream_t s);
int launch_rates_lg(int ns, int nr, int ntb, const unsigned char* blob, unsigned bytes, const float* rho,
                    const float* T, const float* Y, long long ld, long long n, float* dYdt, int* status,
                    cudaStream_t s);
int occupancy_lg(int ns, int na, int nr, int ntb, unsigned prefix, bool stiff, int* blocks_per_sm);

// large mechanisms, rates with the stoichiometric contractions on the tensor cores (rates_tc.cu)
bool rates_tc_supported(int ns, int ntb);
std::vector<unsigned char> rates_tc_image(const chem_mechanism* m, const unsigned char* blob);
int launch_rates_tc(int ns, int nr, int ntb, const unsigned char* img, const unsigned char* blob, const float* rho,
                    const float* T, const float* Y, long long ld, long long n, float* dYdt, int* status,
                    cudaStream_t s);

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
