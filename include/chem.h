/*
 * chem.h -- C ABI of the GB300 (sm_103a) per-cell stiff-chemistry library (libchem.so).
 *
 * The library advances every cell of a reacting-flow field over one flow time step dt as a
 * constant-volume, adiabatic 0-D reactor (arxiv 2510.23993, Sec. 2.1, Eq. 5: dY_k/dt =
 * W_k omega_k / rho; temperature from the internal energy at fixed rho by Newton iteration),
 * with the bulk-sparse strategy of Algorithm 3 (Sec. 3.2): every active cell takes one bulk
 * step with an error test, and only the cells that fail are compacted into a device queue and
 * substepped implicitly (an L-stable 3-stage SDIRK method of order 3 whose stages are solved by
 * Newton iterations on a dense per-cell Jacobian, with embedded error control).  Rates use the
 * matrix (log-concentration) form of the kinetics in FP32; the Newton LU/solve of stiff cells
 * and the temperature inversion run in FP64.
 *
 * Conventions for every entry point:
 *   - arrays are structure-of-arrays (Sec. 3.1): a field F of n cells is F[i], i < n; the mass
 *     fractions are Y[k * ld + i] for species k < ns and cell i < n, with ld >= n;
 *   - "device" pointers are CUDA device memory owned by the caller; "host" pointers are host
 *     memory owned by the caller; the library never frees caller memory;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream); work is enqueued
 *     asynchronously, nothing synchronizes unless the entry point says so;
 *   - the return value is CHEM_OK (0) or a negative CHEM_E* code; argument errors are detected
 *     on the host before anything is enqueued; per-cell failures are reported through the
 *     per-cell substep counts and the counters that chem_status returns.
 * The library allocates device memory only in chem_init (tables and workspace sized by
 * max_cells) and frees it in chem_destroy.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CHEM_OK 0
#define CHEM_EINVAL (-1)       /* bad argument, or non-finite / non-physical input cells */
#define CHEM_ENOMEM (-2)       /* n > max_cells, or a device allocation failed */
#define CHEM_EMAXSTEPS (-3)    /* a stiff cell reached k_max substeps (its count is -1) */
#define CHEM_ENOCONV (-4)      /* a stiff cell's Newton iteration / step size collapsed */
#define CHEM_ECUDA (-5)        /* a CUDA runtime call failed */
#define CHEM_EUNSUPPORTED (-6) /* mechanism shape without a compiled kernel (ns) */

/* Opaque context: device copy of the mechanism tables and the stiff-cell workspace. */
typedef struct chem_ctx chem_ctx;

/* Reaction mechanism (host memory, read by chem_init only; SI units).
 * Thermo per species: NASA-7 a1..a7 then T_lo, T_hi (cp/R = a1 + a2 T + ... + a5 T^4,
 * h/R = a1 T + a2 T^2/2 + ... + a5 T^5/5 + a6, s/R = a1 ln T + ... + a5 T^4/4 + a7); outside
 * [T_lo, T_hi] cp is held at its boundary value.  All species must share T_lo and T_hi.
 * Rate constant k_f = A T^b exp(-Ea / (R T)); reverse k_r = k_f / K_c (Sec. 2.1). */
typedef struct {
  int32_t ns, nr;               /* species, reactions */
  const double *W;              /* [ns] molar masses, kg/mol */
  const double *thermo;         /* [ns][9] */
  const int8_t *nu_f, *nu_r;    /* [nr][ns] reactant / product coefficients, 0..2 */
  const double *A, *b, *Ea;     /* [nr] SI pre-exponential, temperature exponent, J/mol */
  const uint8_t *reversible;    /* [nr] 0/1 */
  const uint8_t *third_body;    /* [nr] 0/1: rate multiplied by [M] = sum_k eff_k C_k */
  const double *eff;            /* [nr][ns] third-body efficiencies (read for third-body rows) */
} chem_mechanism;

/* Integration parameters (copied by chem_init; can be changed with chem_set_params). */
typedef struct {
  double rtol;       /* relative tolerance of the bulk test and of the stiff integrator */
  double atol;       /* absolute tolerance on mass fractions */
  double T_min;      /* activity threshold (Algorithm 2/3 T_reaction_min): T < T_min is skipped */
  double bulk_frac;  /* max relative change of any Y_k in one bulk step (Sec. 2.1, 1-5%) */
  double y_floor;    /* floor of |Y_k| in the relative-change rule */
  int32_t k_bulk;    /* explicit bulk substeps attempted per cell (Algorithm 3 K_max, 1..5) */
  int32_t k_max;     /* cap of implicit substeps per stiff cell (Algorithm 3, 1e5) */
  int32_t flags;     /* CHEM_FLAG_* bits, 0 by default */
} chem_params;

/* chem_params.flags: evaluate the rates of the stiff integrator in FP64 (FP64 tables) instead of
 * FP32 (a precision reference for the mixed-precision default; the Jacobian stays FP32). */
#define CHEM_FLAG_FP64_RATES 1
/* chem_params.flags: record CUDA events around the bulk and the stiff kernel of each advance call
 * (on the call's stream); chem_status then reports their durations.  Not for graph capture. */
#define CHEM_FLAG_TIMING 2
/* chem_params.flags: hand the stiff cells to the persistent stiff kernel most expensive first
 * (counting sort by a cost bucket between the two kernels), which shortens the tail of that
 * kernel.  ORDER_RATE keys on dt * sum_k |dY_k/dt| at the bulk step; ORDER_PREV keys on the
 * substep count that the previous call left in substeps[i] (the array is then read on entry:
 * pass the previous call's output, e.g. in a time-stepping loop). */
#define CHEM_FLAG_ORDER_RATE 4
#define CHEM_FLAG_ORDER_PREV 8
/* chem_params.flags: integrate the stiff cells in two passes.  The first pass gives every queued
 * cell up to 32 implicit steps and saves the state of the cells it did not finish; those are
 * sorted by their estimated remaining steps, (dt - t) / h at the current step size.  The second,
 * cooperative launch takes them longest first from a shared queue; once the queue is empty, each
 * cell still running is parked after 32 more steps and the parked cells are finished in rounds of
 * up to 32 steps separated by grid-wide barriers, relisted after each round so that they always
 * fill whole warps (an FP64 warp instruction costs the same with one active lane as with 32)
 * spread over all SMs.  Results are bit-identical to the single pass.  Needs 8 * ns + 53 bytes
 * of device memory per cell of max_cells, allocated when the flag is first set (chem_init or
 * chem_set_params); ignored by chem_advance_noalloc and by mechanisms of more than 15 species.
 * A barrier wait longer than 4 s ends the launch and the call reports CHEM_ECUDA. */
#define CHEM_FLAG_TWO_PASS 16

/* Counters of the last advance call (see chem_status). */
typedef struct {
  int64_t ncell;      /* cells in the call */
  int64_t nskipped;   /* T < T_min */
  int64_t nbulk;      /* accepted by the bulk step */
  int64_t nqueued;    /* compacted into the stiff queue */
  int64_t nfailed;    /* stiff cells that hit k_max or whose step size collapsed */
  int64_t ninvalid;   /* non-finite or non-physical inputs (count -1, state untouched) */
  int64_t substeps;   /* total implicit substeps of the stiff cells */
  int64_t attempts;   /* attempted implicit steps (accepted + rejected) */
  int64_t newton;     /* Newton iterations of the stage solves (rates + T(e) + solve each) */
  int32_t status;     /* CHEM_OK or the most severe per-cell error code */
  float bulk_ms;      /* bulk kernel duration (CHEM_FLAG_TIMING), else 0 */
  float stiff_ms;     /* stiff kernel duration (CHEM_FLAG_TIMING), else 0 */
  int64_t factorizations; /* Jacobians formed and iteration matrices factored: one per attempt in
                             the one-thread-per-cell kernel; the warp-per-cell kernel of the large
                             mechanisms keeps a factored matrix over up to 16 steps of unchanged
                             size */
} chem_stats;

/* Defaults: rtol 1e-5, atol 1e-10, T_min 0, bulk_frac 0.05, y_floor 1e-10, k_bulk 1,
 * k_max 100000, flags CHEM_FLAG_ORDER_RATE. */
void chem_default_params(chem_params *out);

/* Create a context for one mechanism on the current CUDA device.  Copies the mechanism into
 * device tables and allocates the workspace of up to max_cells cells (stiff queue, counters).
 * Returns CHEM_EINVAL for an inconsistent mechanism, CHEM_EUNSUPPORTED if no kernel is compiled
 * for ns, CHEM_ENOMEM / CHEM_ECUDA on allocation failure.  *out is NULL on failure. */
int chem_init(const chem_mechanism *mech, const chem_params *params, int64_t max_cells,
              chem_ctx **out);

/* Replace the integration parameters used by later calls. */
int chem_set_params(chem_ctx *ctx, const chem_params *params);

/* Free the context and its device memory (synchronizes the device). NULL is ignored. */
void chem_destroy(chem_ctx *ctx);

/* Advance n cells over dt (Sec. 2.1 Eq. 5; Algorithm 3), FP32 state.  Device pointers.
 *   T[n]      in: temperature guess (K); out: temperature consistent with e and the new Y
 *   p[n]      out: pressure rho R T sum_k Y_k / W_k (Pa); may be NULL
 *   Y[ns*ld]  in/out: mass fractions, SoA with leading dimension ld
 *   rho[n]    in: density (kg/m^3), e[n] in: mass-specific internal energy (J/kg), both constant
 *   substeps[n] out: 0 skipped (T < T_min), k_bulk accepted by the bulk step, > k_bulk stiff
 *             (k_bulk + implicit substeps), -1 invalid input or failed cell (state untouched)
 * Cells that are skipped, invalid or failed keep T, p, Y unchanged.  Returns CHEM_ENOMEM if
 * n > max_cells.  Asynchronous on `stream`; graph-capturable. */
int chem_advance(chem_ctx *ctx, float *T, float *p, float *Y, int64_t ld, const float *rho,
                 const float *e, int64_t n, double dt, int32_t *substeps, void *stream);

/* Same as chem_advance with FP64 state arrays (state arithmetic of the bulk step and of the
 * stiff solver in FP64; rates still FP32). */
int chem_advance_f64(chem_ctx *ctx, double *T, double *p, double *Y, int64_t ld,
                     const double *rho, const double *e, int64_t n, double dt,
                     int32_t *substeps, void *stream);

/* End-to-end variant of chem_advance on HOST buffers (same layout, ld = n): copies the inputs
 * to the context's device staging buffers, advances, copies T, p, Y, substeps back, and
 * synchronizes `stream`.  Host buffers should be pinned for full copy bandwidth. */
int chem_advance_host(chem_ctx *ctx, float *T, float *p, float *Y, const float *rho,
                      const float *e, int64_t n, double dt, int32_t *substeps, void *stream);

/* The paper's own integration method, kept as the comparison point of chem_advance: the explicit
 * first-order adaptive scheme of Sec. 2.1 (Algorithm 2's per-cell loop: each substep as long as
 * keeps every |dY_k| within params.bulk_frac * max(|Y_k|, params.y_floor), the "1-5%" rule, and
 * never past dt; T from e by the FP64 inversion after every substep) under the bulk / sparse
 * control of Algorithm 3:
 *   section 1: one launch over all cells sets each cell's time to 0 (active) or dt (T < T_min,
 *              invalid), solves its temperature from e and counts the active cells;
 *   section 2: while the active count, copied to the host after every launch, exceeds n_star
 *              (the paper's N* = 1e4), one launch over all cells in which each active cell takes
 *              at most k_steps substeps (the paper's bulk K_max = 5);
 *   section 3: one launch over the compacted list of the remaining active cells, each taking at
 *              most params.k_max substeps (the paper's 1e5).
 * The bulk phase ends after ceil(k_max / k_steps) launches even if more than n_star cells are
 * still active (a bound the paper does not state).  Device pointers, FP32 state, same layout as
 * chem_advance.  substeps[n] out: 0 skipped, the number of explicit substeps, or -1 for invalid
 * input or a failed cell (k_max reached in section 3, or T(e) lost); unlike chem_advance, a failed
 * cell keeps the state it had reached.  chem_status reports nbulk = cells finished in section 2,
 * nqueued = cells entering section 3, substeps = attempts = explicit substeps.  *launches (may be
 * NULL) receives the number of section-2 launches.  Synchronizes `stream` after every launch (the
 * host reads the active count), so it is not graph-capturable.  Allocates 8 * (ns + 2) * max_cells
 * bytes on first use (each cell's time, temperature and Y in FP64 between launches).  FP64 state
 * arithmetic; rates in FP32, or FP64 with CHEM_FLAG_FP64_RATES.  Dense mechanisms only (CHEM_EUNSUPPORTED for the warp-per-cell path); CHEM_EINVAL
 * for k_steps < 1 or n_star < 0. */
int chem_advance_explicit(chem_ctx *ctx, float *T, float *p, float *Y, int64_t ld, const float *rho,
                          const float *e, int64_t n, double dt, int32_t *substeps, int32_t k_steps,
                          int64_t n_star, int32_t *launches, void *stream);

/* The multi-kernel, library-GEMM rate evaluation that the paper's fused kernel replaces (Sec.
 * 3.2.1 and its Fig. 2A baseline; App. C): per call, a cell-parallel preparation kernel, cuBLAS
 * SGEMMs for the stoichiometric products (ln C . nu_f^T, ln C . nu_r^T, C . eff^T for the
 * third-body rows), a cells x reactions kernel for the rates of progress, and a final SGEMM
 * q . (dnu W) that writes dY/dt.  Same inputs, output and precision (FP32) as chem_rates; kept
 * as the comparison point of the single-kernel strategy, per grid.  chem_mk_create copies the
 * mechanism, opens cuBLAS at run time (CHEM_EUNSUPPORTED if libcublas cannot be loaded or the
 * mechanism has more than 65535 reactions) and
 * allocates 4 * (2 ns + 2 nr + ntb + 5) bytes per cell of max_cells (ntb: third-body reactions).
 * chem_mk_rates: device pointers, asynchronous on `stream`, CHEM_ENOMEM if n > max_cells; not
 * thread-safe (one scratch per object).  chem_mk_destroy synchronizes the device. */
typedef struct chem_mk chem_mk;
int chem_mk_create(const chem_mechanism *mech, int64_t max_cells, chem_mk **out);
int chem_mk_rates(chem_mk *mk, const float *rho, const float *T, const float *Y, int64_t ld, int64_t n,
                  float *dYdt, void *stream);
void chem_mk_destroy(chem_mk *mk);

/* Storage layouts of a per-cell state record (rho, T, Y_0 .. Y_{ns-1}), nv = ns + 2 floats, for
 * chem_pressure_layout (the layout question of Sec. 3.1 / Algorithm 1):
 *   CHEM_LAYOUT_SOA        X[v * ld + i]  (component-major; ld >= n; the library's own layout)
 *   CHEM_LAYOUT_AOS        X[i * nv + v]  (cell-major), each thread reads its own record
 *   CHEM_LAYOUT_AOSOA      X[(i / 32) * 32 * nv + v * 32 + i % 32]  (tiles of 32 cells; the
 *                          array holds ceil(n / 32) full tiles)
 *   CHEM_LAYOUT_AOS_STAGED the AoS array, read through shared memory: each CTA copies its 128
 *                          contiguous records with 16-byte loads (X must be 16-byte aligned) */
#define CHEM_LAYOUT_SOA 0
#define CHEM_LAYOUT_AOS 1
#define CHEM_LAYOUT_AOSOA 2
#define CHEM_LAYOUT_AOS_STAGED 3

/* p[i] = rho R T sum_k Y_k / W_k from the state records X of n cells in the given layout: the
 * all-components-of-one-cell load of the integrators, one thread per cell, under each layout
 * (W: host array of ns molar masses, kg/mol).  Device pointers X, p; asynchronous on `stream`
 * of the current device.  ns must be 9 or 53 (CHEM_EUNSUPPORTED otherwise); CHEM_EINVAL for an
 * unknown layout, ld < n (SoA), a misaligned X (staged AoS) or a non-positive W. */
int chem_pressure_layout(int32_t ns, const double *W, int32_t layout, const float *X, int64_t ld,
                         int64_t n, float *p, void *stream);

/* One box of a block-structured AMR hierarchy (Sec. 2.3): its own SoA arrays (device memory,
 * caller-owned; the same meaning and layout as the arguments of chem_advance) and its chemistry
 * step dt (under temporal subcycling a level-l box advances dt0 / r^l).  level is informational. */
typedef struct {
  float *T, *p, *Y;          /* p may be NULL */
  int64_t ld;                /* leading dimension of Y (>= n) */
  const float *rho, *e;
  int32_t *substeps;
  int64_t n;                 /* cells in the box */
  double dt;                 /* s */
  int32_t level;
} chem_box;

/* Register the box table used by chem_advance_boxes (a set-up call: it synchronizes the device
 * and allocates the device copy of the table; the boxes' arrays are referenced, not copied).
 * At most 4096 boxes and max_cells cells in total (else CHEM_EINVAL / CHEM_ENOMEM).  A
 * previously captured graph is released. */
int chem_boxes_set(chem_ctx *ctx, const chem_box *boxes, int32_t nbox);

/* Advance every cell of every registered box over its box's dt in one bulk launch and one
 * persistent stiff launch over all boxes (the multigrid kernel fusion of Sec. 3.2 / App. E: cells
 * find their box through a prefix sum of box sizes, no data is copied).  Same per-cell semantics
 * and status reporting as chem_advance.  Asynchronous, no host synchronization. */
int chem_advance_boxes(chem_ctx *ctx, void *stream);

/* Capture chem_advance_boxes on `stream` (a non-default stream) into a CUDA graph kept by the
 * context; chem_boxes_launch then replays the whole chemistry step as one graph launch.  The
 * graph refers to the registered box arrays: refill them in place between launches.  Not with
 * CHEM_FLAG_TIMING. */
int chem_boxes_capture(chem_ctx *ctx, void *stream);
int chem_boxes_launch(chem_ctx *ctx, void *stream);

/* Density and internal energy from (T, p, Y) (ideal gas; e = sum_k Y_k u_k(T)), computed in
 * FP64 and rounded to the output type.  Device pointers; asynchronous. */
int chem_state_from_TpY(chem_ctx *ctx, const float *T, const float *p, const float *Y,
                        int64_t ld, int64_t n, float *rho, float *e, void *stream);
int chem_state_from_TpY_f64(chem_ctx *ctx, const double *T, const double *p, const double *Y,
                            int64_t ld, int64_t n, double *rho, double *e, void *stream);

/* Temperature from internal energy at fixed Y (the FP64 Newton inversion used by the
 * integrators; Sec. 2.1).  T[n] in: guess, out: solution.  Device pointers; asynchronous. */
int chem_temperature(chem_ctx *ctx, const float *Y, int64_t ld, const float *e, int64_t n,
                     float *T, void *stream);

/* dY/dt of Eq. 5 at given (rho, T, Y), evaluated with the FP32 matrix-form kinetics of the
 * integrators.  dYdt[ns*ld] out.  Device pointers; asynchronous. */
int chem_rates(chem_ctx *ctx, const float *rho, const float *T, const float *Y, int64_t ld,
               int64_t n, float *dYdt, void *stream);

/* chem_rates for the 53-species mechanisms with the stoichiometric contractions of the matrix
 * form (Sec. 3.2; App. C weighs library GEMMs against a hand-written product) on the tensor
 * cores: per tile of 128 cells, ln C . nu_f^T, ln C . nu_r^T and C . eff^T (third-body
 * concentrations) are BF16 tensor-core products accumulated in FP32, the rates of progress are
 * formed per cell and reaction in FP32 on the CUDA cores, and q . dnu is a fourth tensor-core
 * product.  Each FP32 operand enters as three BF16 parts (x = b0 + b1 + b2, 24 significant bits),
 * so the result has the precision of chem_rates (FP32); a cell with a rate of progress above
 * 1e37 in magnitude (or not finite) is redone with FP64 rates of progress.  Same arguments, layout and
 * output as chem_rates (device pointers, Y and dYdt [ns][ld], asynchronous on `stream`).
 * CHEM_EUNSUPPORTED for a context whose mechanism is not a 53-species one with at most 32
 * third-body reactions (the operand image, ~140 KB, is built by chem_init).  A tensor-core
 * completion that does not arrive within the spin limit sets the status that chem_status
 * reports as CHEM_ECUDA. */
int chem_rates_tc(chem_ctx *ctx, const float *rho, const float *T, const float *Y, int64_t ld,
                  int64_t n, float *dYdt, void *stream);

/* chem_advance for callers that cannot allocate device memory (no counterpart in the paper).
 * Real-time loops that may not block on the allocator, plugins that may only use the buffers
 * handed to them, or processes with a capped allocator cannot call chem_init, which allocates.
 * This entry point takes the mechanism from host memory on every call (same layout, same checks
 * and the same packed tables as chem_init, so the results equal chem_advance's) and keeps
 * the packed tables (at most 64 KiB) and its scratch -- the counters and the stiff-cell queue --
 * in fixed-size device arrays that every GPU loading the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree or other allocating routine; the caller passes the device
 * inputs and outputs exactly as for chem_advance (ns = 9 kernels; params NULL = defaults;
 * CHEM_FLAG_TIMING is ignored).
 *   - at most 2,097,152 cells per call: more returns CHEM_ENOMEM with a message on stderr;
 *   - the first call on a device looks up the device addresses of the arrays
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *   - the host copy of the tables synchronizes `stream` before it starts;
 *   - every call shares the arrays and overwrites them (the counters are cleared first): calls
 *     that overlap on the GPU -- other streams, other threads -- race;
 *   - stats (may be NULL) receives this call's counters and status; filling it synchronizes
 *     `stream`.  Without stats a device-side failure shows only in the per-cell counts (-1). */
int chem_advance_noalloc(const chem_mechanism *mech, const chem_params *params, float *T, float *p,
                         float *Y, int64_t ld, const float *rho, const float *e, int64_t n,
                         double dt, int32_t *substeps, chem_stats *stats, void *stream);

/* Measurement utility (no counterpart in the paper): the FP64 FMA throughput of the current GPU in
 * TFLOP/s (2 flops per FMA), from independent FMA chains filling every SM, best of `reps` timed
 * launches after one warm-up launch.  The roofline of the stiff integrator, which the FP64 pipe
 * bounds, is stated against it.  Allocates and frees a small device buffer (stream-ordered) and
 * synchronizes `stream`.  *tflops (host) receives the result; CHEM_EINVAL for a null pointer or
 * reps < 1. */
int chem_measure_fp64_peak(double *tflops, int32_t reps, void *stream);

/* Result of chem_tune. */
typedef struct {
  int32_t k_bulk;                /* chosen explicit bulk substeps per cell */
  int32_t flags;                 /* chosen queue-order flag (0 or CHEM_FLAG_ORDER_RATE) */
  int32_t bulk_blocks_per_sm;    /* resident blocks per SM of the bulk kernel grid */
  int32_t stiff_blocks_per_sm;   /* resident blocks per SM of the persistent stiff kernel */
  float best_ms, default_ms;     /* timed advance with the chosen / the incoming settings */
  int32_t trials;                /* timed advances run */
  int32_t from_cache;            /* 1 if the choice came from the cache file */
  int32_t stiff_block;           /* threads per CTA of the dense stiff kernel (64, 128, 256) */
  int32_t quantum;               /* attempts per cell in the probe pass and in each continuation
                                    round of the two-pass schedule (16, 32, 64) */
} chem_tune_result;

/* Autotuner of the launch configuration (the paper tuned K_max and the bulk-to-sparse threshold
 * by hand, Sec. 3.2 / App. D): times chem_advance on the caller's field (device arrays as for
 * chem_advance) for candidate values of k_bulk (1..3), the stiff-queue order, the resident
 * blocks per SM of both kernels and, for the dense (one cell per thread) stiff kernel, its CTA
 * size and the two-pass scheduling quantum (coordinate descent, best of two repetitions; no
 * candidate changes a cell's result), applies the
 * fastest to the context and returns it.  T, p, Y are restored to their input values on return
 * (the advanced state is discarded).  A set-up call: it allocates temporary device copies of T,
 * p, Y and synchronizes `stream`.  cache_path (may be NULL) names a text file: a matching entry
 * (mechanism shape, log2 of the cell count, dt, GPU name) is applied without trials, and a tuned
 * choice is appended. */
int chem_tune(chem_ctx *ctx, float *T, float *p, float *Y, int64_t ld, const float *rho,
              const float *e, int64_t n, double dt, int32_t *substeps, const char *cache_path,
              chem_tune_result *out, void *stream);

/* The BF16 tensor-core GEMM (tcgen05, FP32 accumulation) that the surrogate's kernels are built
 * on, exposed for verification:
 *   C[m*ldc + n] = epi( sum_k A[m*sam + k*sak] * B[n*sbn + k*sbk] ),  m < M, n < N (<= 256), k < K
 * A and B are FP32 device arrays, rounded to BF16 on load.  epi: 0 store, 1 + bias[n], 2 + bias[n]
 * with gelu(z) also stored in C2 (same layout), 3 atomic add into C (required when ksplit > 1,
 * K split over ksplit CTAs).  *status (device int) gets bit 32 if an MMA completion wait timed out.
 * Asynchronous on `stream`. */
int chem_tc_gemm(const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbn, int64_t sbk,
                 float *C, int64_t ldc, const float *bias, float *C2, int32_t M, int32_t N, int32_t K,
                 int32_t epi, int32_t ksplit, int32_t *status, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Learned surrogate of the chemistry step with a per-cell error gate.  The paper has no
 * counterpart (its outlook, Sec. 6, mentions machine learning only for performance prediction).  The network
 * (compiled for ns = 9 and ns = 53) maps x = (T, ln p, ln dt, ln(Y_k + 1e-6)), standardised, through four
 * GELU layers of 128 to ns + 2 outputs: the standardised encodings a = asinh(u / 1e-8) of
 * u_k = ln((Y1_k + 1e-6) / (max(Y_k, 0) + 1e-6)) and u_T = ln(T1 / T) for the state (Y1, T1)
 * after dt (decoded with u clamped so that 0 <= Y1 <= 1 and T / 10 <= T1 <= 10 T), and an error head
 * (log10 of the predicted relative error of the state the gate would write).  BF16 weights on
 * the tensor cores, FP32 accumulation and FP32 master weights.  All state (weights, AdamW
 * moments, normalisation, scratch) is owned by the context and freed by chem_destroy.
 * --------------------------------------------------------------------------------------------- */

/* Training configuration (chem_surrogate_train). */
typedef struct {
  int32_t epochs;       /* passes over the data set */
  int32_t batch;        /* samples per step, a multiple of 128 (4096 by default) */
  double lr;            /* peak AdamW learning rate, cosine-decayed to 0 over all steps */
  double weight_decay;  /* decoupled weight decay */
  double err_weight;    /* weight of the error-head term of the loss */
  uint64_t seed;        /* shuffling seed */
} chem_train_cfg;

/* Create (or re-initialise) the context's surrogate: He-initialised weights from `seed`, zero
 * AdamW moments, an empty training box (nothing is accepted until it is trained or loaded) and
 * the conserved directions of the mechanism (the complement of the span of the reaction vectors
 * W .* (nu_r - nu_f)).  CHEM_EUNSUPPORTED if ns is not 9 or 53, or more than 8 directions are
 * conserved. */
int chem_surrogate_init(chem_ctx *ctx, uint64_t seed);

/* Number of FP32 parameters of the network for a mechanism of ns species (weights and biases of
 * the five layers, W_l row-major [out][in] followed by b_l, layer by layer): 52,619 for ns = 9,
 * 63,927 for ns = 53; CHEM_EUNSUPPORTED for other species counts. */
int chem_surrogate_nparams(int32_t ns);

/* Train on n samples (device arrays): X [n][ns + 3] rows (T [K], p [Pa], dt [s], Y_1..Y_ns) and
 * Yt [n][ns + 1] rows (Y1_1..Y1_ns, T1), the state after dt.  Sets the normalisation (mean and
 * standard deviation of every feature and target encoding; a standard deviation below 1e-12 is
 * replaced by 1) and the training box (range of every feature) from the data, then runs
 * cfg->epochs epochs of shuffled full batches: forward and backward on the tensor cores, then one
 * AdamW update per batch, m = 0.9 m + 0.1 g, v = 0.999 v + 0.001 g^2,
 * w -= lr_s (m / (1 - 0.9^t) / (sqrt(v / (1 - 0.999^t)) + 1e-8) + weight_decay w), with t the
 * optimiser step count since chem_surrogate_init and lr_s = cfg->lr (1 + cos(pi s / S)) / 2 for
 * step s = 0 .. S - 1 of this call (S = epochs x n / batch).  loss_per_epoch (host, [epochs], or
 * null) receives the mean batch loss of each epoch.  Synchronous; returns CHEM_ECUDA if a
 * tensor-core wait timed out. */
int chem_surrogate_train(chem_ctx *ctx, const float *X, const float *Yt, int64_t n, const chem_train_cfg *cfg,
                         float *loss_per_epoch, void *stream);

/* Gradient of the training loss of one batch of n samples (n a multiple of 128; layouts as in
 * chem_surrogate_train, normalisation as set by the last training or load) with respect to the
 * FP32 parameters: grads (device, [nparams]) and the batch loss (device, [1]).  The loss is
 * mean_b [ sum_j (o_bj - t_bj)^2 + err_weight (o_b,err - e*_b)^2 ], with t the standardised target
 * encodings and e*_b = log10(E_b + 1e-12) held constant, E_b = max over species of
 * |Y1'_k - Y1_k| / max(|Y1_k|, 1e-6) and |T1' - T1| / T1 for the corrected prediction (Y1', T1').  Synchronous. */
int chem_surrogate_grads(chem_ctx *ctx, const float *X, const float *Yt, int32_t n, float err_weight,
                         float *grads, float *loss, void *stream);

/* Network outputs (standardised, [n][ns + 2], device) of the GEMM path for X [n][ns + 3] (device). */
int chem_surrogate_forward(chem_ctx *ctx, const float *X, int32_t n, float *out, void *stream);

/* Network outputs of the fused inference kernel of chem_advance_gated for n cells in the SoA
 * layout of chem_advance (T, Y [ns][ld], rho, e on the device; p is derived), [n][ns + 2] into
 * out.  The state is not modified.  Synchronous. */
int chem_surrogate_infer(chem_ctx *ctx, const float *T, const float *Y, int64_t ld, const float *rho,
                         const float *e, int64_t n, double dt, float *out, void *stream);

/* Copy the FP32 parameters out to dst and/or in from src (host or device, [nparams]). */
int chem_surrogate_params(chem_ctx *ctx, float *dst, const float *src, void *stream);

/* Serialise the surrogate (versioned header, normalisation, FP32 parameters) into buf (host).
 * With buf null only *size is set. */
int chem_surrogate_save(chem_ctx *ctx, void *buf, size_t cap, size_t *size);

/* Load a surrogate saved by chem_surrogate_save for the same mechanism shape. */
int chem_surrogate_load(chem_ctx *ctx, const void *buf, size_t size);

/* One chemistry step with the surrogate in front of the method.  Every cell first goes through
 * the fused inference kernel; the gate accepts a cell only if (i) every feature lies within its
 * range over the training set (widened by 1e-3 of the range) and Y >= -1e-10, (ii) the error head predicts a relative error <= gate_tol, and
 * (iii) after a conservative correction of Y1 - Y (the smallest change, weighted by
 * max(|Y1_k|, 1e-6), that keeps every conserved element mass) the mass fractions stay in
 * [-1e-10, 1 + 1e-6], |sum (Y1 - Y)| <= 1e-7 and T(e, Y1) agrees with the network's T1 to 1e-4.  Accepted cells are written
 * (T from e, p from the ideal gas law, substeps 0, accepted[i] = 1); all other cells
 * (accepted[i] = 0) take the plain bulk / stiff path of chem_advance; the counters of
 * chem_status cover those cells only.  *n_accepted (host, optional; the call then synchronizes)
 * receives the number of accepted cells.  Arguments otherwise as chem_advance. */
int chem_advance_gated(chem_ctx *ctx, float *T, float *p, float *Y, int64_t ld, const float *rho,
                       const float *e, int64_t n, double dt, double gate_tol, uint8_t *accepted,
                       int32_t *substeps, int64_t *n_accepted, void *stream);

/* Synchronize `stream` and return the counters of the last advance call on this context. */
int chem_status(chem_ctx *ctx, void *stream, chem_stats *out);

/* Static description of a status code. */
const char *chem_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CHEM_H */
