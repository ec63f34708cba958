// multikernel.cu -- the multi-kernel, library-GEMM evaluation of the species production rates that
// the paper compares its single fused kernel against (Sec. 3.2.1, the baseline strategy of its
// Fig. 2A; App. C): per grid, a short sequence of launches parallel over cells x species or
// cells x reactions, with the stoichiometric products done by cuBLAS SGEMM:
//   1. prep (cells):            lnC_k = ln(rho Y_k / W_k), C_k = max(rho Y_k / W_k, 0), per-cell
//                               ln T, 1/T, ln(p0 / RT), 1/rho, T;
//   2. GEMM:                    Lf = lnC . nu_f^T   (n x nr),  Lr = lnC . nu_r^T;
//   3. GEMM (third-body rows):  M = C . eff^T       (n x ntb);
//   4. progress (cells x nr):   ln k_f = ln A + b ln T - Ea/(R T); ln K_c from the reaction's
//                               combined NASA-7 differences; q = (exp(ln k_f + Lf)
//                               - exp(ln k_f - ln K_c + Lr)) [M] / rho, written over Lf;
//   5. GEMM:                    dY/dt = q . (dnu W)  (n x ns), written straight into dYdt.
// Four to five launches per grid against one for chem_rates over all grids.  FP32 throughout
// (the same precision as chem_rates), GEMMs in plain FP32 (no TF32).  cuBLAS is opened at run
// time (dlopen), so the rest of the library does not depend on it.
#include <dlfcn.h>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include <cublas_v2.h>

#include "chem.h"

namespace {

constexpr double kRgas = 8.314462618;
constexpr double kPref = 101325.0;
constexpr float kLnZeroMk = -1.0e4f;   // ln C of an absent species: exp underflows to 0

// the cuBLAS entry points used here, resolved at run time
struct Blas {
  void* so = nullptr;
  cublasStatus_t (*create)(cublasHandle_t*) = nullptr;
  cublasStatus_t (*destroy)(cublasHandle_t) = nullptr;
  cublasStatus_t (*set_stream)(cublasHandle_t, cudaStream_t) = nullptr;
  cublasStatus_t (*set_math)(cublasHandle_t, cublasMath_t) = nullptr;
  cublasStatus_t (*sgemm)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int, int, const float*,
                          const float*, int, const float*, int, const float*, float*, int) = nullptr;
};

bool open_blas(Blas& b) {
  const char* names[] = {"libcublas.so.13", "libcublas.so", "/usr/local/cuda/lib64/libcublas.so.13"};
  for (const char* n : names) {
    b.so = dlopen(n, RTLD_NOW | RTLD_LOCAL);
    if (b.so) break;
  }
  if (!b.so) return false;
  b.create = reinterpret_cast<decltype(b.create)>(dlsym(b.so, "cublasCreate_v2"));
  b.destroy = reinterpret_cast<decltype(b.destroy)>(dlsym(b.so, "cublasDestroy_v2"));
  b.set_stream = reinterpret_cast<decltype(b.set_stream)>(dlsym(b.so, "cublasSetStream_v2"));
  b.set_math = reinterpret_cast<decltype(b.set_math)>(dlsym(b.so, "cublasSetMathMode"));
  b.sgemm = reinterpret_cast<decltype(b.sgemm)>(dlsym(b.so, "cublasSgemm_v2"));
  return b.create && b.destroy && b.set_stream && b.set_math && b.sgemm;
}

// per reaction: ln A, b, Ea / R, sum of dnu, reversible, third-body row (-1 if none), and the
// seven NASA-7 coefficient differences sum_k dnu_k a_k (for dCp, dH, dS), T_lo, T_hi
struct MkReaction {
  float lnA, b, EaR, dn;
  int rev, tb;
  float da[7];
  float Tlo, Thi;
};

__global__ void mk_prep(const float* __restrict__ rho, const float* __restrict__ T, const float* __restrict__ Y,
                        long long ld, long long n, int ns, const float* __restrict__ invW, float* lnC, float* C,
                        float* cellv) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float r = rho[i], t = T[i];
  for (int k = 0; k < ns; ++k) {
    const float c = r * Y[k * ld + i] * invW[k];
    lnC[k * n + i] = c > 0.0f ? logf(c) : kLnZeroMk;
    C[k * n + i] = c > 0.0f ? c : 0.0f;
  }
  cellv[i] = logf(t);
  cellv[n + i] = 1.0f / t;
  cellv[2 * n + i] = logf(static_cast<float>(kPref / kRgas) / t);
  cellv[3 * n + i] = 1.0f / r;
  cellv[4 * n + i] = t;
}

// dG/RT of one reaction at T from the combined NASA-7 differences, cp held constant outside
// [T_lo, T_hi] (the mechanism's thermo convention)
__device__ __forceinline__ float mk_dg_rt(const MkReaction& q, float T, float lnT) {
  const float Te = fminf(fmaxf(T, q.Tlo), q.Thi);
  const float* a = q.da;
  const float dcp = a[0] + Te * (a[1] + Te * (a[2] + Te * (a[3] + Te * a[4])));
  float dh = Te * (a[0] + Te * (a[1] * 0.5f + Te * (a[2] * (1.0f / 3.0f) + Te * (a[3] * 0.25f + Te * a[4] * 0.2f)))) + a[5];
  const float lnTe = Te == T ? lnT : logf(Te);
  float ds = a[0] * lnTe + Te * (a[1] + Te * (a[2] * 0.5f + Te * (a[3] * (1.0f / 3.0f) + Te * a[4] * 0.25f))) + a[6];
  if (Te != T) {
    dh += dcp * (T - Te);
    ds += dcp * (lnT - lnTe);
  }
  return dh / T - ds;
}

__global__ void mk_progress(const MkReaction* __restrict__ rx, int nr, long long n, const float* __restrict__ cellv,
                            float* Lf, const float* __restrict__ Lr, const float* __restrict__ M, float* q_out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= n || r >= nr) return;
  const MkReaction q = rx[r];
  const float lnT = cellv[i], invT = cellv[n + i], lnP0RT = cellv[2 * n + i], irho = cellv[3 * n + i];
  const float T = cellv[4 * n + i];
  const float lnkf = q.lnA + q.b * lnT - q.EaR * invT;
  float v = expf(lnkf + Lf[r * n + i]);
  if (q.rev) {
    const float lnKc = -mk_dg_rt(q, T, lnT) + q.dn * lnP0RT;
    v -= expf(lnkf - lnKc + Lr[r * n + i]);
  }
  if (q.tb >= 0) v *= M[q.tb * n + i];
  q_out[r * n + i] = v * irho;
}

}  // namespace

struct chem_mk {
  Blas blas;
  cublasHandle_t h = nullptr;
  int ns = 0, nr = 0, ntb = 0;
  long long cap = 0;
  float *NF = nullptr, *NR = nullptr, *E = nullptr, *DW = nullptr, *invW = nullptr;
  MkReaction* rx = nullptr;
  float *lnC = nullptr, *C = nullptr, *cellv = nullptr, *Lf = nullptr, *Lr = nullptr, *M = nullptr;
};

extern "C" {

void chem_mk_destroy(chem_mk* mk) {
  if (!mk) return;
  cudaDeviceSynchronize();
  for (void* p : {static_cast<void*>(mk->NF), static_cast<void*>(mk->NR), static_cast<void*>(mk->E),
                  static_cast<void*>(mk->DW), static_cast<void*>(mk->invW), static_cast<void*>(mk->rx),
                  static_cast<void*>(mk->lnC), static_cast<void*>(mk->C), static_cast<void*>(mk->cellv),
                  static_cast<void*>(mk->Lf), static_cast<void*>(mk->Lr), static_cast<void*>(mk->M)})
    cudaFree(p);
  if (mk->h) mk->blas.destroy(mk->h);
  if (mk->blas.so) dlclose(mk->blas.so);
  delete mk;
}

int chem_mk_create(const chem_mechanism* m, int64_t max_cells, chem_mk** out) {
  if (!out) return CHEM_EINVAL;
  *out = nullptr;
  if (!m || m->ns < 1 || m->nr < 1 || m->ns > 127 || !m->W || !m->thermo || !m->nu_f || !m->nu_r || !m->A ||
      !m->b || !m->Ea || !m->reversible || !m->third_body || !m->eff || max_cells < 0 || max_cells > 0x7fffffffLL)
    return CHEM_EINVAL;
  if (m->nr > 65535) return CHEM_EUNSUPPORTED;   // reactions index the grid's y dimension
  chem_mk* mk = new (std::nothrow) chem_mk();
  if (!mk) return CHEM_ENOMEM;
  if (!open_blas(mk->blas)) {
    chem_mk_destroy(mk);
    return CHEM_EUNSUPPORTED;
  }
  if (mk->blas.create(&mk->h) != CUBLAS_STATUS_SUCCESS) {
    mk->h = nullptr;
    chem_mk_destroy(mk);
    return CHEM_ECUDA;
  }
  if (mk->blas.set_math(mk->h, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS) {
    chem_mk_destroy(mk);
    return CHEM_ECUDA;
  }
  const int ns = m->ns, nr = m->nr;
  mk->ns = ns;
  mk->nr = nr;
  mk->cap = max_cells;
  // host tables: nu_f, nu_r as column-major ns x nr (the [nr][ns] arrays as stored), eff^T for the
  // third-body rows (ns x ntb), dnu_rk W_k as column-major ns x nr (used transposed)
  std::vector<float> nf(static_cast<size_t>(nr) * ns), nb(nf.size()), dw(nf.size()), iw(ns), eff;
  std::vector<MkReaction> rx(nr);
  int ntb = 0;
  for (int r = 0; r < nr; ++r) {
    MkReaction& q = rx[r];
    double dn = 0.0, da[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < ns; ++k) {
      const size_t o = static_cast<size_t>(r) * ns + k;
      const int d = m->nu_r[o] - m->nu_f[o];
      nf[o] = static_cast<float>(m->nu_f[o]);
      nb[o] = static_cast<float>(m->nu_r[o]);
      dw[o] = static_cast<float>(d * m->W[k]);
      dn += d;
      for (int j = 0; j < 7; ++j) da[j] += d * m->thermo[9 * k + j];
    }
    q.lnA = static_cast<float>(std::log(m->A[r]));
    q.b = static_cast<float>(m->b[r]);
    q.EaR = static_cast<float>(m->Ea[r] / kRgas);
    q.dn = static_cast<float>(dn);
    q.rev = m->reversible[r] ? 1 : 0;
    q.tb = -1;
    for (int j = 0; j < 7; ++j) q.da[j] = static_cast<float>(da[j]);
    q.Tlo = static_cast<float>(m->thermo[7]);
    q.Thi = static_cast<float>(m->thermo[8]);
    if (m->third_body[r]) {
      q.tb = ntb++;
      for (int k = 0; k < ns; ++k) eff.push_back(static_cast<float>(m->eff[static_cast<size_t>(r) * ns + k]));
    }
  }
  for (int k = 0; k < ns; ++k) iw[k] = static_cast<float>(1.0 / m->W[k]);
  mk->ntb = ntb;
  auto up = [](float** d, const std::vector<float>& h) {
    if (h.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(d, h.size() * sizeof(float));
    return e ? e : cudaMemcpy(*d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
  };
  cudaError_t e = up(&mk->NF, nf);
  if (!e) e = up(&mk->NR, nb);
  if (!e) e = up(&mk->DW, dw);
  if (!e) e = up(&mk->invW, iw);
  if (!e) e = up(&mk->E, eff);
  if (!e) e = cudaMalloc(&mk->rx, sizeof(MkReaction) * nr);
  if (!e) e = cudaMemcpy(mk->rx, rx.data(), sizeof(MkReaction) * nr, cudaMemcpyHostToDevice);
  const size_t n = static_cast<size_t>(max_cells > 0 ? max_cells : 1);
  if (!e) e = cudaMalloc(&mk->lnC, sizeof(float) * ns * n);
  if (!e) e = cudaMalloc(&mk->C, sizeof(float) * ns * n);
  if (!e) e = cudaMalloc(&mk->cellv, sizeof(float) * 5 * n);
  if (!e) e = cudaMalloc(&mk->Lf, sizeof(float) * nr * n);
  if (!e) e = cudaMalloc(&mk->Lr, sizeof(float) * nr * n);
  if (!e && ntb > 0) e = cudaMalloc(&mk->M, sizeof(float) * ntb * n);
  if (e) {
    std::fprintf(stderr, "libchem: chem_mk_create: %s\n", cudaGetErrorString(e));
    chem_mk_destroy(mk);
    return e == cudaErrorMemoryAllocation ? CHEM_ENOMEM : CHEM_ECUDA;
  }
  *out = mk;
  return CHEM_OK;
}

int chem_mk_rates(chem_mk* mk, const float* rho, const float* T, const float* Y, int64_t ld, int64_t n, float* dYdt,
                  void* stream) {
  if (!mk || n < 0 || (n > 0 && (!rho || !T || !Y || !dYdt || ld < n))) return CHEM_EINVAL;
  if (n > mk->cap) return CHEM_ENOMEM;
  if (n == 0) return CHEM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ns = mk->ns, nr = mk->nr, ni = static_cast<int>(n);
  const float one = 1.0f, zero = 0.0f;
  mk_prep<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(rho, T, Y, ld, n, ns, mk->invW, mk->lnC, mk->C,
                                                                  mk->cellv);
  if (cudaGetLastError() != cudaSuccess) return CHEM_ECUDA;
  if (mk->blas.set_stream(mk->h, st) != CUBLAS_STATUS_SUCCESS) return CHEM_ECUDA;
  // Lf (n x nr) = lnC (n x ns) . NF (ns x nr); Lr likewise; M (n x ntb) = C (n x ns) . E (ns x ntb)
  cublasStatus_t s = mk->blas.sgemm(mk->h, CUBLAS_OP_N, CUBLAS_OP_N, ni, nr, ns, &one, mk->lnC, ni, mk->NF, ns, &zero,
                                    mk->Lf, ni);
  if (s == CUBLAS_STATUS_SUCCESS)
    s = mk->blas.sgemm(mk->h, CUBLAS_OP_N, CUBLAS_OP_N, ni, nr, ns, &one, mk->lnC, ni, mk->NR, ns, &zero, mk->Lr, ni);
  if (s == CUBLAS_STATUS_SUCCESS && mk->ntb > 0)
    s = mk->blas.sgemm(mk->h, CUBLAS_OP_N, CUBLAS_OP_N, ni, mk->ntb, ns, &one, mk->C, ni, mk->E, ns, &zero, mk->M, ni);
  if (s != CUBLAS_STATUS_SUCCESS) return CHEM_ECUDA;
  mk_progress<<<dim3(static_cast<unsigned>((n + 255) / 256), nr), 256, 0, st>>>(mk->rx, nr, n, mk->cellv, mk->Lf,
                                                                                mk->Lr, mk->M, mk->Lf);
  if (cudaGetLastError() != cudaSuccess) return CHEM_ECUDA;
  // dY/dt (n x ns, leading dimension ld) = q (n x nr) . (dnu W) (nr x ns)
  s = mk->blas.sgemm(mk->h, CUBLAS_OP_N, CUBLAS_OP_T, ni, ns, nr, &one, mk->Lf, ni, mk->DW, ns, &zero, dYdt,
                     static_cast<int>(ld));
  return s == CUBLAS_STATUS_SUCCESS ? CHEM_OK : CHEM_ECUDA;
}

}  // extern "C"
