// rates_tc.cu -- the matrix form of the kinetics (Sec. 3.2: species log-concentrations times the
// stoichiometric matrices, plus the Arrhenius and equilibrium terms, then exp; the rates of
// progress times the net stoichiometry) with its contractions on the 5th-generation tensor cores,
// for the large mechanisms (53 species / 325 reactions), where the stoichiometric matrices are
// wide enough for the tensor cores to pay.
//
// One CTA owns tiles of 128 cells (one TMEM lane per cell).  Per tile:
//   M   = C  . eff^T   third-body concentrations [128 x 32]
//   S_f = lnC . nu_f^T and S_r = lnC . nu_r^T, reaction chunk by chunk [128 x 48 each]
//   q   = exp(ln k_f + S_f) - exp(ln k_f - ln K_c + S_r), times M for third-body reactions,
//         per cell and reaction on the CUDA cores (FP32; FP64 for a cell with a |q| beyond 1e37)
//   w  += q . dnu   chunk by chunk into TMEM [128 x 64]
//   dY/dt = w W / rho
// The operands enter the BF16 tensor cores split into three BF16 parts each, x = b0 + b1 + b2
// (b0 = bf16(x), b1 = bf16(x - b0), b2 = bf16(x - b0 - b1)): 24 significant bits, so the
// contractions keep FP32 accuracy (FP32 accumulation in TMEM).  The stoichiometric coefficients
// (small integers) are exact in BF16; the third-body efficiencies are split like the
// concentrations and the six largest of the nine split products are summed.
//
// Reactions are permuted on the host so that the third-body ones come first, in their row order:
// reaction j < ntb of the first chunk takes its [M] from TMEM column j of the M product.  Each
// reaction's constants (Arrhenius, Gibbs coefficients of the three thermo regimes) are one
// 48-byte record in global memory, read through L1 (every thread of a warp reads the same record
// at the same time); padding reactions have records whose rates are exactly 0.
//
// Three groups of four warps share the tile: warps w, w + 4, w + 8 read the same 32 TMEM lanes
// (cells) and take 16 of each chunk's 48 reactions, which triples the warps that hide the
// latency of the per-reaction arithmetic.  S is double-buffered in TMEM and issued two chunks
// ahead, and the dnu product of a chunk completes while the next chunk's rates are computed, so
// the CUDA cores wait on the tensor cores only at the start and the end of a tile.  The
// tensor-core operand images (~138 KB) are built once per context and copied into each CTA's
// shared memory with one bulk async copy.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/chem.h"
#include "chem_device.cuh"
#include "internal.h"
#include "tc.cuh"

namespace chem {
namespace rtc {

constexpr int kTile = 128;    // cells per tile (TMEM lanes)
constexpr int kKS = 64;       // species padded (K of the lnC / C products, N of the dnu product)
constexpr int kChunk = 48;    // reactions per chunk (N of the lnC products, K of the dnu product)
constexpr int kTB = 32;       // third-body reactions padded
constexpr int kGroups = 3;    // thread groups of 128, 16 reactions of each chunk per group
constexpr int kThreads = kTile * kGroups;
static_assert(kChunk == 16 * kGroups, "one 16-column slice of each chunk per group");
// largest |q| kept in FP32: a few such terms still sum below the FP32 maximum (3.4e38)
constexpr float kQFinite = 1.0e37f;
// log-rate offset of the records' padding and irreversible reactions: exp() of it is 0
constexpr float kLnOff = -2.0e4f;
// TMEM columns of the accumulators: two S buffers (S_f at +0, S_r at +kSr), then M and w
constexpr uint32_t kColS = 0, kSBuf = 128, kSr = 64, kColM = 256, kColW = 320, kTmemCols = 512;

__host__ __device__ constexpr int nr_padded(int nr) { return (nr + kChunk - 1) / kChunk * kChunk; }

// byte layout of the operand image: BF16 tensor-core operands (K-major core matrices of tc.cuh),
// staged into shared memory, then the reaction records, read from global memory
struct ImgLayout {
  int nrp;         // reactions padded to whole chunks
  unsigned bf;     // nu_f  [nrp rows][kKS]
  unsigned br;     // nu_r  [nrp rows][kKS]
  unsigned bw;     // dnu^T [kKS rows][nrp]
  unsigned be;     // eff split s at be + s * kTB * kKS * 2, [kTB rows][kKS]
  unsigned staged; // bytes copied into shared memory
  unsigned rec;    // float4 [3 regimes][nrp][3]: (lnA, b, Ea/R, sum dnu), (g0..g3), (g4, g5, g6', 0)
  unsigned perm;   // int [nrp]: original index of permuted reaction j (-1 for padding)
  unsigned bytes;
};

__host__ __device__ inline ImgLayout img_layout(int nr) {
  ImgLayout L;
  L.nrp = nr_padded(nr);
  L.bf = 0;
  L.br = L.bf + static_cast<unsigned>(L.nrp) * kKS * 2;
  L.bw = L.br + static_cast<unsigned>(L.nrp) * kKS * 2;
  L.be = L.bw + static_cast<unsigned>(kKS) * L.nrp * 2;
  L.staged = L.be + 3u * kTB * kKS * 2;
  L.rec = L.staged;
  L.perm = L.rec + 3u * L.nrp * 48;
  L.bytes = L.perm + 4u * L.nrp;
  return L;
}

// shared memory: [staged image][X: 3 splits of 128 x 64][Q: 3 splits of 128 x kChunk]
constexpr unsigned kXBytes = kTile * kKS * 2;
constexpr unsigned kQBytes = kTile * kChunk * 2;
__host__ __device__ inline unsigned x_offset(int nr) { return (img_layout(nr).staged + 127u) & ~127u; }
__host__ __device__ inline unsigned smem_bytes(int nr) { return x_offset(nr) + 3u * kXBytes + 3u * kQBytes; }

// x = b0 + b1 + b2 in BF16, for a pair of values at once; returns the three bf16x2 words
__device__ __forceinline__ void split3_pair(float x, float y, uint32_t (&w)[3]) {
  const __nv_bfloat162 p0 = __floats2bfloat162_rn(x, y);
  const float rx = x - __low2float(p0), ry = y - __high2float(p0);
  const __nv_bfloat162 p1 = __floats2bfloat162_rn(rx, ry);
  const __nv_bfloat162 p2 = __floats2bfloat162_rn(rx - __low2float(p1), ry - __high2float(p1));
  w[0] = *reinterpret_cast<const uint32_t*>(&p0);
  w[1] = *reinterpret_cast<const uint32_t*>(&p1);
  w[2] = *reinterpret_cast<const uint32_t*>(&p2);
}

// eight consecutive K columns [k8, k8 + 8) of row t of the three split tiles (K columns per row)
__device__ __forceinline__ void store_split8(unsigned char* base, unsigned split_bytes, int t, int k8, int K,
                                             const float* v) {
  uint32_t w[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t p[3];
    split3_pair(v[2 * j], v[2 * j + 1], p);
    w[0][j] = p[0];
    w[1][j] = p[1];
    w[2][j] = p[2];
  }
  const uint32_t off = tc::kmajor_offset(t, k8, K);
#pragma unroll
  for (int s = 0; s < 3; ++s)
    *reinterpret_cast<uint4*>(base + s * split_bytes + off) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// tensor-core products into TMEM: D (+)= A . B^T over K = 16 * ksteps (both K-major)
__device__ __forceinline__ void mma_k(uint32_t tmem, const unsigned char* A, int Ka, const unsigned char* B, int Kb,
                                      int ksteps, int N, bool acc) {
  const uint32_t idesc = tc::idesc_bf16_f32(kTile, N);
  for (int kk = 0; kk < ksteps; ++kk) {
    const uint64_t ad = tc::smem_desc(tc::smem_u32(A) + kk * 256, 128, (Ka / 8) * 128);
    const uint64_t bd = tc::smem_desc(tc::smem_u32(B) + kk * 256, 128, (Kb / 8) * 128);
    tc::mma_bf16(tmem, ad, bd, idesc, acc || kk > 0);
  }
}

struct RatesArgs {
  const unsigned char* img;    // operand image (global)
  const unsigned char* blob;   // packed large-layout tables (global; FP64 fallback)
  int nr, ntb;
  const float* rho;
  const float* T;
  const float* Y;
  long long ld, n;
  float* dYdt;
  int* status;
};

// the packed tables, as used by the FP64 fallback
struct RView {
  const float4* arr;
  const int* rinfo;
  const float* W;
  const float* invW;
  const float* gamg;    // [3][nr][8] Gibbs coefficients per regime
  const float* eff;     // [ntb][nsp]
  const int2* sto;      // packed sparse stoichiometry
  float T_lo, T_hi, lnP0R;
  int nr, nsp;
};

__device__ __forceinline__ RView make_rview(const unsigned char* b) {
  const MechHdr* h = reinterpret_cast<const MechHdr*>(b);
  RView v;
  v.arr = reinterpret_cast<const float4*>(b + h->off_arr);
  v.rinfo = reinterpret_cast<const int*>(b + h->off_rinfo);
  v.W = reinterpret_cast<const float*>(b + h->off_W);
  v.invW = reinterpret_cast<const float*>(b + h->off_invW);
  v.gamg = reinterpret_cast<const float*>(b + h->off_gamg);
  v.eff = reinterpret_cast<const float*>(b + h->off_eff);
  v.sto = reinterpret_cast<const int2*>(b + h->off_sto);
  v.T_lo = h->T_lo;
  v.T_hi = h->T_hi;
  v.lnP0R = h->lnP0R;
  v.nr = h->nr;
  v.nsp = h->nsp;
  return v;
}

// dY/dt of one cell with FP64 rates of progress (a cell with a rate beyond the FP32 range): the
// log-rates in FP32 as in the tensor-core path, sparse products from the packed stoichiometry
template <int NS>
__device__ void rates_fp64_cell(const RView& m, float rho, float T, const float* Y, long long ld, long long i,
                                float* out) {
  float C[NS], lnC[NS];
#pragma unroll 1
  for (int k = 0; k < NS; ++k) {
    C[k] = rho * Y[k * ld + i] * m.invW[k];
    lnC[k] = C[k] > 0.0f ? __logf(C[k]) : kLnZero;
  }
  const float lnT = __logf(T), invT = 1.0f / T, lnP0RT = m.lnP0R - lnT;
  const int reg = regime_of(T, m.T_lo, m.T_hi);
  double w[NS];
#pragma unroll 1
  for (int k = 0; k < NS; ++k) w[k] = 0.0;
#pragma unroll 1
  for (int r = 0; r < m.nr; ++r) {
    const float4 a = __ldg(m.arr + r);
    const float lnkf = a.x + a.y * lnT - a.z * invT;
    const int2 st = __ldg(m.sto + r);
    float sf = 0.0f, sr = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int cf = (st.x >> (9 * j + 7)) & 3, cr = (st.y >> (9 * j + 7)) & 3;
      if (cf) sf = fmaf(static_cast<float>(cf), lnC[(st.x >> (9 * j)) & 127], sf);
      if (cr) sr = fmaf(static_cast<float>(cr), lnC[(st.y >> (9 * j)) & 127], sr);
    }
    const float lnqf = lnkf + sf;
    const int info = __ldg(m.rinfo + r);
    float lnqr = kLnZero;
    if (info & 1) {
      const float* g = m.gamg + (reg * m.nr + r) * 8;
      const float T2 = T * T;
      const float dG = __ldg(g) * (1.0f - lnT) +
                       T * (__ldg(g + 1) + T * __ldg(g + 2) + T2 * (__ldg(g + 3) + T * __ldg(g + 4))) +
                       __ldg(g + 5) * invT + __ldg(g + 6);
      lnqr = lnkf - (-dG + a.w * lnP0RT) + sr;
    }
    double q = exp(static_cast<double>(lnqf)) - exp(static_cast<double>(lnqr));
    const int tb = (info >> 8) - 1;
    if (tb >= 0) {
      float M = 0.0f;
#pragma unroll 1
      for (int k = 0; k < NS; ++k) M = fmaf(__ldg(m.eff + tb * m.nsp + k), fmaxf(C[k], 0.0f), M);
      q *= static_cast<double>(M);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int cf = (st.x >> (9 * j + 7)) & 3, cr = (st.y >> (9 * j + 7)) & 3;
      if (cf) w[(st.x >> (9 * j)) & 127] -= cf * q;
      if (cr) w[(st.y >> (9 * j)) & 127] += cr * q;
    }
  }
  const double irho = 1.0 / static_cast<double>(rho);
#pragma unroll 1
  for (int k = 0; k < NS; ++k) out[k * ld + i] = static_cast<float>(w[k] * static_cast<double>(m.W[k]) * irho);
}

template <int NS>
__global__ void __launch_bounds__(kThreads, 1) rates_tc_kernel(const RatesArgs a) {
  static_assert(NS <= kKS, "species exceed the padded K");
  extern __shared__ __align__(128) unsigned char smem[];
  // completion barriers of the tensor-core products: M, the two S buffers, dnu, and the final
  // drain after a timeout
  __shared__ uint64_t bar_img, bar_m, bar_s[2], bar_w, bar_f;
  __shared__ uint32_t s_taddr;
  __shared__ int s_bad[kTile];   // cells with a rate of progress beyond the FP32 range
  const ImgLayout L = img_layout(a.nr);
  unsigned char* sI = smem;
  unsigned char* sX = smem + x_offset(a.nr);
  unsigned char* sQ = sX + 3 * kXBytes;
  if (!stage_to_smem(sI, a.img, L.staged, &bar_img, a.status)) return;
  const float4* rec = reinterpret_cast<const float4*>(a.img + L.rec);
  const RView m = make_rview(a.blob);
  const int warp = threadIdx.x >> 5;
  const int grp = warp >> 2;                                   // reactions 16 grp .. 16 grp + 15 of each chunk
  const int row = (warp & 3) * 32 + (threadIdx.x & 31);        // the cell (TMEM lane) of this thread
  const bool issuer = threadIdx.x == 0;
  if (warp == 0) tc::tmem_alloc(&s_taddr, kTmemCols);
  if (issuer) {
    tc::mbar_init(&bar_m, 1);
    tc::mbar_init(&bar_s[0], 1);
    tc::mbar_init(&bar_s[1], 1);
    tc::mbar_init(&bar_w, 1);
    tc::mbar_init(&bar_f, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = s_taddr;
  const uint32_t lane_addr = taddr + (static_cast<uint32_t>((warp & 3) * 32) << 16);
  const int nchunk = L.nrp / kChunk;
  uint32_t pm = 0, ps0 = 0, ps1 = 0, pw = 0;   // phase parities of the barriers
  bool ok = true;
  // S_f, S_r of chunk c into buffer b (issuer), completion on bar_s[b]
  auto issue_s = [&](int c, int b) {
    const unsigned off = static_cast<unsigned>(c) * kChunk * kKS * 2;   // rows of chunk c
    const uint32_t col = kColS + b * kSBuf;
    for (int s = 0; s < 3; ++s) {
      mma_k(taddr + col, sX + s * kXBytes, kKS, sI + L.bf + off, kKS, kKS / 16, kChunk, s > 0);
      mma_k(taddr + col + kSr, sX + s * kXBytes, kKS, sI + L.br + off, kKS, kKS / 16, kChunk, s > 0);
    }
    tc::mma_commit(&bar_s[b]);
  };
  const long long ntiles = (a.n + kTile - 1) / kTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kTile + row;
    const bool valid = i < a.n;
    const float rho = valid ? a.rho[i] : 1.0f;
    const float T = valid ? a.T[i] : 1000.0f;
    if (grp == 0) s_bad[row] = 0;
    // ---- this group's species blocks of X: C splits first (for M), then lnC splits
    float Cv[3][8];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int k8 = 8 * (grp + kGroups * b);
      if (k8 < kKS) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = k8 + j;
          Cv[b][j] = (valid && k < NS) ? rho * __ldcs(a.Y + k * a.ld + i) * __ldg(m.invW + k) : 0.0f;
        }
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaxf(Cv[b][j], 0.0f);
        store_split8(sX, kXBytes, row, k8, kKS, v);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (issuer) {
      tc::fence_after_sync();
      const unsigned char* Be = sI + L.be;
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};   // the six largest split products
      for (int p = 0; p < 6; ++p)
        mma_k(taddr + kColM, sX + pa[p] * kXBytes, kKS, Be + pb[p] * kTB * kKS * 2, kKS, kKS / 16, kTB, p > 0);
      tc::mma_commit(&bar_m);
    }
    ok = ok && tc::mbar_wait(&bar_m, pm);
    pm ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int k8 = 8 * (grp + kGroups * b);
      if (k8 < kKS) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float C = Cv[b][j];
          v[j] = C > 0.0f ? fmaxf(__logf(C), kLnZero) : kLnZero;   // finite: 0 * lnC must be 0
        }
        store_split8(sX, kXBytes, row, k8, kKS, v);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (issuer) {
      tc::fence_after_sync();
      issue_s(0, 0);
      if (nchunk > 1) issue_s(1, 1);
    }
    // per-cell basis of the log-rates
    const float lnT = __logf(T), invT = 1.0f / T, lnP0RT = m.lnP0R - lnT;
    const float T2 = T * T, T3 = T2 * T, T4 = T2 * T2, omlnT = 1.0f - lnT;
    const int reg = regime_of(T, m.T_lo, m.T_hi);
    const float4* recg = rec + static_cast<long long>(reg) * L.nrp * 3;
    bool fine = true;
#pragma unroll 1
    for (int c = 0; c < nchunk; ++c) {
      const int b = c & 1;
      // S of chunk c (issued two chunks ahead)
      if (b == 0) {
        ok = ok && tc::mbar_wait(&bar_s[0], ps0);
        ps0 ^= 1u;
      } else {
        ok = ok && tc::mbar_wait(&bar_s[1], ps1);
        ps1 ^= 1u;
      }
      tc::fence_after_sync();
      const int col = 16 * grp;
      const int r0 = c * kChunk + col;
      const uint32_t scol = kColS + b * kSBuf + col;
      float sf[16], sr[16];
      tc::tmem_ld16(lane_addr + scol, sf);
      tc::tmem_ld16(lane_addr + scol + kSr, sr);
      float Mv[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) Mv[j] = 1.0f;
      if (r0 < a.ntb) {   // the third-body reactions (first in the permuted order)
        float t16[16];
        tc::tmem_ld16(lane_addr + kColM + r0, t16);
#pragma unroll
        for (int j = 0; j < 16; ++j) Mv[j] = r0 + j < a.ntb ? t16[j] : 1.0f;
      }
      float q[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float4* rr = recg + (r0 + j) * 3;
        const float4 ar = __ldg(rr), g03 = __ldg(rr + 1), g46 = __ldg(rr + 2);
        const float lnkf = fmaf(ar.y, lnT, fmaf(-ar.z, invT, ar.x));
        const float lnqf = lnkf + sf[j];
        const float dG = fmaf(g03.x, omlnT, fmaf(g03.y, T, fmaf(g03.z, T2, fmaf(g03.w, T3,
                         fmaf(g46.x, T4, fmaf(g46.y, invT, g46.z))))));
        const float lnqr = fmaf(-ar.w, lnP0RT, lnkf + dG) + sr[j];
        const float qv = (__expf(lnqf) - __expf(lnqr)) * Mv[j];
        fine &= fabsf(qv) <= kQFinite;   // also false for inf and NaN
        q[j] = qv;
      }
      if (c > 0) {   // the dnu product of chunk c - 1 has read Q
        ok = ok && tc::mbar_wait(&bar_w, pw);
        pw ^= 1u;
      }
      float v8[8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v8[j] = (fine && valid) ? q[8 * h + j] : 0.0f;
        store_split8(sQ, kQBytes, row, col + 8 * h, kChunk, v8);
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      if (!__syncthreads_and(ok)) { ok = false; break; }
      if (issuer) {
        tc::fence_after_sync();
        const unsigned char* Bw = sI + L.bw + static_cast<unsigned>(c) * (kChunk / 8) * 128;   // K offset of chunk c
        const uint32_t idesc = tc::idesc_bf16_f32(kTile, kKS);
        for (int s = 0; s < 3; ++s) {
          for (int kk = 0; kk < kChunk / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(tc::smem_u32(sQ + s * kQBytes) + kk * 256, 128, (kChunk / 8) * 128);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(Bw) + kk * 256, 128, (L.nrp / 8) * 128);
            tc::mma_bf16(taddr + kColW, ad, bd, idesc, c > 0 || s > 0 || kk > 0);
          }
        }
        tc::mma_commit(&bar_w);
        if (c + 2 < nchunk) issue_s(c + 2, b);   // buffer b has been read by every thread
      }
    }
    if (!ok) break;
    if (!fine) s_bad[row] = 1;
    ok = ok && tc::mbar_wait(&bar_w, pw);   // the last dnu product
    pw ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
    // ---- dY/dt = w W / rho: species columns 16 g (and 48 for group 0)
    const bool bad = s_bad[row] != 0;
    const float irho = 1.0f / rho;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int c16 = 16 * (grp + kGroups * b);
      if (c16 < kKS) {
        float w[16];
        tc::tmem_ld16(lane_addr + kColW + c16, w);
        if (valid && !bad) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int k = c16 + j;
            if (k < NS) __stcs(a.dYdt + k * a.ld + i, w[j] * __ldg(m.W + k) * irho);
          }
        }
      }
    }
    if (grp == 0 && valid && bad) rates_fp64_cell<NS>(m, rho, T, a.Y, a.ld, i, a.dYdt);
    tc::fence_before_sync();
    __syncthreads();   // TMEM columns, X, Q and s_bad are reused by the next tile
  }
  if (!ok) {
    // a tensor-core completion did not arrive in time: record it, then wait (bounded) for every
    // product this CTA issued before the accumulator is freed
    if (issuer) {
      atomicOr(a.status, kFlagStage);
      tc::mma_commit(&bar_f);
    }
    tc::mbar_wait(&bar_f, 0);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

}  // namespace rtc

// ------------------------------------------------------------------ host side

namespace {

// K-major core-matrix offset (tc.cuh) on the host
unsigned kmajor(int r, int k, int K) {
  return static_cast<unsigned>((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

uint16_t bf16_bits(float x) {   // round to nearest even (finite inputs)
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

// Operand image of a large mechanism (host), from the mechanism and its packed tables (blob,
// the large layout of pack_mechanism, whose FP32 constants the records copy): nu_f, nu_r and
// dnu^T in BF16 (exact small integers), the efficiencies of the third-body reactions split into
// three BF16 parts, and the reaction records, all in the permuted order (third-body first).
std::vector<unsigned char> rates_tc_image(const chem_mechanism* m, const unsigned char* blob) {
  using namespace rtc;
  const int ns = m->ns, nr = m->nr;
  const ImgLayout L = img_layout(nr);
  const MechHdr* h = reinterpret_cast<const MechHdr*>(blob);
  const float* arr = reinterpret_cast<const float*>(blob + h->off_arr);
  const int* rinfo = reinterpret_cast<const int*>(blob + h->off_rinfo);
  const float* gamg = reinterpret_cast<const float*>(blob + h->off_gamg);
  std::vector<int> perm;
  for (int r = 0; r < nr; ++r)
    if (m->third_body[r]) perm.push_back(r);
  for (int r = 0; r < nr; ++r)
    if (!m->third_body[r]) perm.push_back(r);
  std::vector<unsigned char> img(L.bytes, 0);
  auto put = [&](unsigned base, int r, int k, int K, float v) {
    const uint16_t b = bf16_bits(v);
    std::memcpy(img.data() + base + kmajor(r, k, K), &b, 2);
  };
  float* rec = reinterpret_cast<float*>(img.data() + L.rec);
  int* pidx = reinterpret_cast<int*>(img.data() + L.perm);
  for (int j = 0; j < L.nrp; ++j) {
    pidx[j] = j < nr ? perm[j] : -1;
    for (int reg = 0; reg < 3; ++reg) {
      float* R = rec + (static_cast<size_t>(reg) * L.nrp + j) * 12;
      if (j >= nr) {   // padding: q_f = q_r = 0
        R[0] = kLnOff;
        R[10] = kLnOff;
        continue;
      }
      const int r = perm[j];
      for (int c = 0; c < 4; ++c) R[c] = arr[4 * r + c];
      const float* g = gamg + (static_cast<size_t>(reg) * nr + r) * 8;
      for (int c = 0; c < 7; ++c) R[4 + c] = g[c];
      if (!(rinfo[r] & 1)) {   // irreversible: q_r = 0
        for (int c = 4; c < 10; ++c) R[c] = 0.0f;
        R[3] = 0.0f;
        R[10] = kLnOff;
      }
    }
  }
  for (int j = 0; j < nr; ++j) {
    const int r = perm[j];
    for (int k = 0; k < ns; ++k) {
      const int f = m->nu_f[r * ns + k], b = m->nu_r[r * ns + k];
      if (f) put(L.bf, j, k, kKS, static_cast<float>(f));
      if (b) put(L.br, j, k, kKS, static_cast<float>(b));
      if (b != f) put(L.bw, k, j, L.nrp, static_cast<float>(b - f));
    }
    if (m->third_body[r]) {   // j is the third-body row
      for (int k = 0; k < ns; ++k) {
        const float e = static_cast<float>(m->eff[r * ns + k]);
        const uint16_t b0 = bf16_bits(e);
        const float r1 = e - bf16_value(b0);
        const uint16_t b1 = bf16_bits(r1);
        const uint16_t b2 = bf16_bits(r1 - bf16_value(b1));
        const uint16_t parts[3] = {b0, b1, b2};
        for (int s = 0; s < 3; ++s)
          std::memcpy(img.data() + L.be + s * kTB * kKS * 2 + kmajor(j, k, kKS), &parts[s], 2);
      }
    }
  }
  return img;
}

bool rates_tc_supported(int ns, int ntb) { return ns == 53 && ntb <= rtc::kTB; }

int launch_rates_tc(int ns, int nr, int ntb, const unsigned char* img, const unsigned char* blob, const float* rho,
                    const float* T, const float* Y, long long ld, long long n, float* dYdt, int* status,
                    cudaStream_t s) {
  if (ns != 53 || ntb > rtc::kTB) return -1;
  rtc::RatesArgs a;
  a.img = img;
  a.blob = blob;
  a.nr = nr;
  a.ntb = ntb;
  a.rho = rho;
  a.T = T;
  a.Y = Y;
  a.ld = ld;
  a.n = n;
  a.dYdt = dYdt;
  a.status = status;
  const unsigned smem = rtc::smem_bytes(nr);
  auto k = rtc::rates_tc_kernel<53>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (n + rtc::kTile - 1) / rtc::kTile;
  const int grid = static_cast<int>(tiles < sms ? tiles : sms);
  k<<<grid, rtc::kThreads, smem, s>>>(a);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace chem
