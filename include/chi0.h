/*
 * chi0.h - C ABI of libchi0: the RPA polarizability hot path of
 * "Towards Fully Converged GW Calculations for Large Systems" on one GPU.
 *
 *   chi0_{G,G'}(q,w) = 1/2 sum_{v,c} M_vc(q,G) conj(M_vc(q,G'))
 *                       x [1/(E_v - E_c - w + i d) + 1/(E_v - E_c + w + i d)]   (Eq. 1)
 *
 * with M_vc(q,G) = <v,k+q| exp(i(q+G).r) |c,k> (definition following Eq. 1),
 * and its accelerated form (Eq. 3 with the energy quadrature of Eq. 4), in
 * which the conduction bands above N0 are replaced by one state per energy
 * grid point carrying the weight g(E_i) dE_i and the denominator E_v - E_i.
 *
 * Conventions used by every entry point
 *   - Pointers marked (device) must point to memory of the device that was
 *     current when the plan was created; (host) pointers are read before the
 *     call returns and may be reused afterwards.  The caller owns every buffer.
 *   - Complex numbers are interleaved (re, im).  "complex" below means
 *     complex128 (double2) for a CHI0_FP64 plan and complex64 (float2) for the
 *     split-precision plans; energies, weights and chi0 are always FP64.
 *   - Real-space grids are [band][i1][i2][i3] with i3 fastest (n1*n2*n3
 *     points, r = (i1/n1, i2/n2, i3/n3) in lattice coordinates).
 *   - A pair index is p = iv * n_c + ic (valence-major) over the bands passed
 *     to the call.  chi0 is [n_freq][N_G][N_G] complex128, row G, column G'.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute
 *     calls only enqueue work; they return after host-side validation.
 *   - Every call returns a chi0_status and never aborts.  Argument errors are
 *     reported before any work is enqueued.  A device-side failure (a bounded
 *     wait that ran out) is recorded in a device status word and reported as
 *     CHI0_ERR_TIMEOUT by chi0_sync_status().
 *   - A plan is not safe for concurrent use from several host threads.
 */
#ifndef CHI0_H
#define CHI0_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CHI0_OK = 0,
  CHI0_ERR_INVALID = 1,      /* bad argument; nothing was enqueued */
  CHI0_ERR_OOM = 2,          /* device allocation failed */
  CHI0_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  CHI0_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
  CHI0_ERR_UNSUPPORTED = 5,  /* no kernel for this device / shape */
  CHI0_ERR_SINGULAR = 6      /* chi0_epsilon_inverse met a zero pivot (reported by chi0_sync_status) */
} chi0_status;

typedef enum {
  CHI0_FP64 = 0,        /* FP64 end to end (CUDA-core DFMA contraction) */
  CHI0_SPLIT_BF16 = 1,  /* FP32 pair stage; contraction on tcgen05 with hi+lo BF16 operands */
  CHI0_SPLIT_FP16 = 2   /* FP32 pair stage; contraction on tcgen05 with hi+lo FP16 operands */
} chi0_precision;

typedef struct chi0_plan_s* chi0_plan;

/* Plan description.  All arrays are (host) and are copied by chi0_plan_create. */
typedef struct {
  int n1, n2, n3;            /* real-space FFT grid */
  int n_q;                   /* number of q-points */
  const int32_t* n_G;        /* [n_q] dielectric-sphere size per q (>= 1) */
  const int32_t* gvec;       /* [sum n_G][3] integer G vectors of each sphere, q after q;
                                each sphere must span fewer than n_k points along axis k */
  int npw;                   /* size of the wavefunction plane-wave sphere */
  const int32_t* gw;         /* [npw][3] integer g of the wavefunction sphere */
  int n_freq;                /* number of frequencies (>= 1) */
  const double* freq_re;     /* [n_freq] Re(omega), Hartree */
  const double* freq_im;     /* [n_freq] Im(omega), Hartree */
  double delta;              /* broadening d of Eq. 1, Hartree */
  chi0_precision precision;
  int n_products;            /* 16-bit terms and products per real product: 3 = two terms t0+t1,
                                products t0t0+t0t1+t1t0; 4 = two terms, adds t1t1; 6 = three terms
                                t0+t1+t2, products t_i t_j with i+j <= 2.  0 = 6 for BF16 (three
                                BF16 terms carry 24 bits), 3 for FP16; ignored for FP64 */
  int64_t max_pairs;         /* pairs per internal block of chi0_build / chi0_accumulate; 0 = default
                                (8192 for split precisions).  Split plans add each launch's FP32
                                chain sums into chi0 once; the diagonal sum_p f_p |M_p(G)|^2 (terms
                                of one phase) is summed apart on the CUDA cores, so the launch length
                                barely shows: max|d chi0| / max|chi0| 2-3e-8 at 8192 and at 16384 */
  int chain_pairs;           /* pairs accumulated in tensor memory before they are added into FP32
                                registers (multiple of 32).  The tensor cores round each MMA result
                                toward zero, which shrinks each chain's sum by about 1.4e-8 per pair
                                of chain length (the diagonal excepted); 0 = 32 (default) */
  int hermitian;             /* split precisions: contract chi0 = (1 + i t) H1 + i H2 with the Hermitian
                                parts H1 = sum Re(f_p) M_p M_p^H and H2 = sum g_p M_p M_p^H,
                                g_p = Im f_p - t Re f_p (f_p the factor of Eq. 1), only tiles on or above
                                the diagonal, the lower triangle written as the conjugate transpose.
                                Per frequency and pair block, t is the midrange of Im f / Re f over the
                                block (0 when that does not shrink the H2 weights) and rho bounds
                                max|g| / max|Re f|: H2 takes one product where rho <= 2^-11 (FP16
                                operands in both precisions), three where rho <= 2^-6, else n_products
                                (its error scales with rho).  0 = automatic: on except for n_products 4 and except where
                                a launch would leave SMs idle (with T = ceil(n_G / 128) tiles, plain
                                mode has n_freq T^2 work items, Hermitian mode n_freq T (T + 1) / 2, each
                                a quarter dearer; the mode with fewer estimated waves over the SMs
                                wins); 1 = on, -1 = off.  chi0_plan_hermitian reports the choice */
} chi0_plan_desc;

/* Create a plan: validates the description, analyses each G sphere for the
 * pruned transforms, uploads index maps and twiddle tables and allocates the
 * plan's workspace on the current device.  *out is NULL on failure; the
 * reason is available from chi0_last_error(NULL). */
chi0_status chi0_plan_create(chi0_plan* out, const chi0_plan_desc* desc);

/* Release a plan and its workspace (synchronises the device first).  NULL is a no-op. */
chi0_status chi0_plan_destroy(chi0_plan plan);

/* *on = 1 when the plan contracts the Hermitian parts H1, H2 (the hermitian field
 * of the description, with its automatic choice resolved), else 0. */
chi0_status chi0_plan_hermitian(chi0_plan plan, int* on);

/* Text of the last error of this plan (plan-owned, valid until the next call
 * on the plan), or of the last failed plan creation when plan is NULL. */
const char* chi0_last_error(chi0_plan plan);

/* Bytes of device workspace held by the plan. */
size_t chi0_workspace_bytes(chi0_plan plan);

/* Synchronise `stream` and report device-side failures recorded since the
 * last call (CHI0_ERR_TIMEOUT if a bounded wait ran out, CHI0_ERR_CUDA if the
 * stream reports an error).  Clears the recorded status. */
chi0_status chi0_sync_status(chi0_plan plan, void* stream);

/* Wavefunctions on the grid (plane-wave expansion used by M after Eq. 1):
 *   psi[b][r] = sum_{g in wavefunction sphere} coeff[b][g] exp(2 pi i g.r).
 * coeff: (device) [nb][npw] complex128 in the order of desc.gw.
 * psi:   (device) [nb][n1*n2*n3] complex (complex64 for split plans). */
chi0_status chi0_wfn_to_grid(chi0_plan plan, const void* coeff, int nb, void* psi, void* stream);

/* Pair matrix elements (definition following Eq. 1), pruned to sphere iq:
 *   M[p][j] = (1/N_r) sum_r conj(psi_v[v(iv)][r]) psi_c[c(ic)][r] exp(2 pi i G_j.r)
 * for iv < n_v, ic < n_c, p = iv*n_c + ic.
 * psi_v, psi_c: (device) grids as written by chi0_wfn_to_grid.
 * v_idx, c_idx: (device) int32 [n_v] / [n_c] band rows to use, or NULL for 0..n-1.
 * M: (device) [n_v*n_c][n_G[iq]] complex. */
chi0_status chi0_pairs(chi0_plan plan, int iq, const void* psi_v, const int32_t* v_idx, int n_v,
                       const void* psi_c, const int32_t* c_idx, int n_c, void* M, void* stream);

/* Contraction of Eq. 1 / Eq. 3-4 for one set of pairs, added into chi0:
 *   chi0[w][G][G'] += sum_p f_p(w) M[p][G] conj(M[p][G'])
 *   f_p(w) = (w_p/2) [1/(dE_p - w + i d) + 1/(dE_p + w + i d)],
 *   dE_p = E_v[iv] - E_col[ic],  w_p = w_col[ic] (1 when w_col is NULL).
 * For the explicit bands E_col = E_c and w_col = 1; for an energy-grid state
 * of Eq. 4, E_col = E_i and w_col = g(E_i) dE_i.
 * M: (device) [n_v*n_c][n_G[iq]] complex; E_v (device) [n_v]; E_col, w_col (device) [n_c];
 * chi0: (device) [n_freq][n_G[iq]][n_G[iq]] complex128, accumulated in place (caller zeroes it). */
chi0_status chi0_accumulate(chi0_plan plan, int iq, const void* M, int n_v, int n_c,
                            const double* E_v, const double* E_col, const double* w_col,
                            void* chi0, void* stream);

/* The whole hot path for one q-point: for blocks of conduction columns,
 * chi0_pairs into plan workspace followed by chi0_accumulate, so M is never
 * held for all pairs at once.  Arguments as for chi0_pairs/chi0_accumulate
 * (valence rows 0..n_v-1 of psi_v; conduction rows c_idx[ic] of psi_c).
 * Split plans with more than one block pipeline the blocks: the pair stage and
 * packing of block k+1 run on a low-priority plan-owned stream beside the
 * contraction of block k on a high-priority one, with a second workspace set
 * allocated on the first such call (chi0_workspace_bytes grows by it; if it
 * cannot be had the build stays serial).  Both streams are joined back into
 * `stream` before the call returns, so ordering on `stream` is as for a
 * serial build. */
chi0_status chi0_build(chi0_plan plan, int iq, const void* psi_v, int n_v, const double* E_v,
                       const void* psi_c, const int32_t* c_idx, int n_c,
                       const double* E_col, const double* w_col, void* chi0, void* stream);

/* Batched build of every q-point of the plan (Eq. 1 per q-point, q-points with
 * different sphere sizes): for each block of conduction columns, the pair
 * elements and factors of every q-point are formed and ONE persistent
 * tensor-core launch contracts all (q-point, frequency, tile) work items.
 * psi_v, E_v, chi0: (host) arrays [n_q] of (device) pointers: the valence grids
 * at k+q ([n_v][N_r] complex), their energies [n_v] and chi0[q]
 * ([n_freq][n_G[q]][n_G[q]] complex128, accumulated).  psi_c, c_idx, n_c,
 * E_col, w_col as for chi0_build (shared by all q-points).
 * use_graph != 0: the enqueued work is captured into a CUDA graph on a
 * plan-owned stream the first time these arguments are seen and the graph is
 * launched on `stream`; later calls with the same arguments relaunch it.
 * FP64 plans run the q-points one after another.  At most 16 q-points. */
chi0_status chi0_build_batched(chi0_plan plan, const void* const* psi_v, int n_v, const double* const* E_v,
                               const void* psi_c, const int32_t* c_idx, int n_c, const double* E_col,
                               const double* w_col, void* const* chi0, int use_graph, void* stream);

/* Adjoint of chi0_accumulate (derived from Eq. 1).  For a real loss L with
 * upstream gradient Gamma_w = dL/dRe chi0[w] + i dL/dIm chi0[w]:
 *   grad_M[p]    = sum_w conj(f_p(w)) Gamma_w M_p + f_p(w) Gamma_w^H M_p
 *   grad dE_p    = sum_w Re( f'_p(w) conj(M_p^H Gamma_w M_p) ),
 *   f'_p(w)      = -(w_p/2) [(dE_p - w + i d)^-2 + (dE_p + w + i d)^-2],
 *   grad_Ev[iv]  = sum_ic grad dE_p,   grad_Ecol[ic] = -sum_iv grad dE_p.
 * Complex gradients use the dL/dRe + i dL/dIm convention.  Give exactly one of
 *   grad_chi0 (device) [n_freq][n_G][n_G] complex128: dense Gamma (FP64 CUDA-core products), or
 *   diag_g    (device) [n_freq][n_G] double: Gamma_w = diag(diag_g[w]) (one fused pass; n_freq <= 64).
 * M, E_v, E_col, w_col as for chi0_accumulate.  Outputs (written, not accumulated):
 * grad_M (device) [n_v*n_c][n_G] complex (the plan's complex type), grad_Ev (device) [n_v],
 * grad_Ecol (device) [n_c].  Deterministic (no atomics). */
chi0_status chi0_backward(chi0_plan plan, int iq, const void* M, int n_v, int n_c, const double* E_v,
                          const double* E_col, const double* w_col, const void* grad_chi0,
                          const double* diag_g, void* grad_M, double* grad_Ev, double* grad_Ecol,
                          void* stream);

/* First-order error estimate of Eq. 3/4's energy substitution (derived from Eq. 1 and
 * Eq. 4): when every conduction band above N0 is given the energy E_i of its Eq. 4
 * grid point in the denominators, a loss L changes by
 *   dL ~ sum_{c >= N0} dL/dE_c (E_i(c) - E_c),
 * with dL/dE_c the grad_Ecol of chi0_backward over the full band sum.  E_i(c) is the
 * midpoint of the step [e_k, e_k+1) holding E_c, e_k = min(E_0 + k dE, E_max),
 * E_0 = E_c[N0-1], k = 0..N_E-1, N_E = ceil((E_max - E_0)/dE) (the steps of
 * chi0_select_accelerated; the last step is closed and energies outside [E_0, E_max]
 * go to the end steps); bands below N0 keep E_c.  Computed on the device, reduced in
 * a fixed order (deterministic).
 * E_c, grad_Ecol: (device) [n_c] FP64, E_c sorted ascending; E_sub: (device) [n_c]
 * receives E_i(c) (E_c for c < N0), or NULL; *estimate (host) receives the sum.
 * Uses one double of the plan's workspace and synchronises `stream`. */
chi0_status chi0_energy_substitution_estimate(chi0_plan plan, const double* E_c, const double* grad_Ecol, int n_c,
                                              int N0, double dE, double E_max, double* E_sub, double* estimate,
                                              void* stream);

/* Host version of the band-to-grid-energy map above (host arrays, host computation):
 * E_out[c] = E_i(c) for c >= N0, E_c[c] otherwise.  Returns 0, or -1 for bad arguments. */
int chi0_grid_energies(const double* E_c, int n_c, int N0, double dE, double E_max, double* E_out);

/* Diagnostic (not part of the method): enqueue a one-thread wait on a barrier
 * that nothing releases, bounded by budget_ms (0 < budget_ms <= 1000), through
 * the same bounded-wait code the tensor-core kernels use.  The wait runs out,
 * records the failure in the plan's device status word and returns, so the
 * next chi0_sync_status reports CHI0_ERR_TIMEOUT and the plan stays usable. */
chi0_status chi0_selftest_wait(chi0_plan plan, double budget_ms, void* stream);

/* Diagnostic (not part of the method): throughput of the CUDA-core fused
 * multiply-add pipes, FP32 (kind 0) or FP64 (kind 1).  One launch of 8 CTAs of
 * 256 threads per SM, each thread `iters` x 8 independent FMA chains, timed with
 * CUDA events on `stream` (synchronised).  *ms (host) receives the device time,
 * *flops (host) the flops executed (2 per FMA).  CHI0_ERR_INVALID unless
 * kind is 0 or 1 and 1 <= iters <= 2^20.  Needs no plan. */
chi0_status chi0_peak_fma(int kind, int iters, double* ms, double* flops, void* stream);

/* Autotuner of the tensor-core contraction (split plans): times the kernel
 * variant (single CTAs with 128 x 128 tiles, or CTA pairs sharing one
 * tcgen05.mma.cta_group::2 over 256 x 128 tiles), the raster group of the
 * persistent work list (1, 2, 4, 8, 16 or all tile rows) and the pairs per
 * launch (2048, 4096, ... up to max_pairs) on synthetic operands
 * written into the plan's workspace for sphere iq (a scratch chi0 is
 * allocated and freed; every candidate over two launches, the three fastest
 * again by their median over nine launches), keeps the fastest in the plan and appends it to the
 * text cache named by the environment variable CHI0_TUNE_CACHE (default
 * $HOME/.cache/chi0_tune.txt).  Unless flags & 1, a cached entry for the same
 * device, sphere size, frequency count, precision, products and Hermitian mode is applied
 * instead of timing; chi0_plan_create applies one for sphere 0.  Before tuning,
 * the environment variable CHI0_TC_PAIR (0 or 1) read at plan creation selects
 * the variant.
 * *best_us_per_pair (may be NULL) receives the best time per pair, -1 if cached.
 * Synchronises the stream. */
chi0_status chi0_autotune(chi0_plan plan, int iq, int flags, double* best_us_per_pair, void* stream);
chi0_status chi0_get_tuning(chi0_plan plan, int* group, int64_t* block_pairs, int* cta_pair);

/* Kernel families counted and timed by the plan's instrumentation. */
typedef enum {
  CHI0_K_WFN = 0,        /* wavefunctions on the grid */
  CHI0_K_PAIR_PLANES,    /* pair products + transforms along i3, i2 */
  CHI0_K_PAIR_GATHER,    /* transform along i1 on the G sphere */
  CHI0_K_WEIGHTS,        /* FP64 frequency factors */
  CHI0_K_PACK,           /* operand scaling + 16-bit split (split plans) */
  CHI0_K_CONTRACT_TC,    /* tcgen05 contraction + FP64 merge (split plans) */
  CHI0_K_CONTRACT_F64,   /* DFMA contraction (FP64 plans) */
  CHI0_K_EPS,            /* dielectric matrix and precision conversions */
  CHI0_K_INV_PANEL,      /* Gauss-Jordan panels, row swaps, column permutation */
  CHI0_K_INV_UPDATE,     /* Gauss-Jordan trailing updates */
  CHI0_K_COUNT
} chi0_kernel;

/* Instrumentation (not part of the method).  With timing enabled, every
 * launch of a family is bracketed by CUDA events recorded on the launching
 * stream.  chi0_profile_read synchronises the recorded events and returns,
 * per family, the summed device time (ms, may be NULL) and the number of
 * kernel launches since the last reset (launches are always counted).
 * total_ms and launches are (host) arrays of CHI0_K_COUNT entries. */
chi0_status chi0_profile_enable(chi0_plan plan, int timing_on);
chi0_status chi0_profile_reset(chi0_plan plan);
chi0_status chi0_profile_read(chi0_plan plan, double* total_ms, int64_t* launches);

/* Allocation-free FP64 accumulate.  The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory when they need chi0
 * (code embedded in a framework that owns all device memory through its own
 * pool, or a loop that must not risk the device-wide synchronisation and
 * out-of-memory failures of cudaMalloc).  It needs no plan and allocates
 * nothing; it computes what chi0_accumulate computes for a CHI0_FP64 plan:
 *   chi0[w][G][G'] += sum_p f_p(w) M[p][G] conj(M[p][G']),  p = iv*n_c + ic,
 * with f_p, E_v, E_col and w_col as for chi0_accumulate (w_col may be NULL).
 * M: (device) [n_v*n_c][n_G] complex128; E_v (device) [n_v]; E_col, w_col
 * (device) [n_c]; freq_re, freq_im (host) [n_freq], copied into the launch;
 * chi0: (device) [n_freq][n_G][n_G] complex128, accumulated in place.
 * Limits: 1 <= n_freq <= 64 and 1 <= n_G <= 65536, otherwise CHI0_ERR_INVALID
 * with the reason in chi0_last_error(NULL).  Any number of pairs is accepted.
 * Scratch: a fixed 4 MiB array of FP64 frequency factors in the library's
 * device image, held by every device that loads the library until the process
 * exits.  The first call on a device looks up that array's device address
 * (with the device current) and should come before any stream capture; so does
 * the first call in a new context on that device (after cudaDeviceReset, or a
 * context made current through the driver API), which has its own copy of the
 * array at its own address and is recognised by its context id.  All
 * calls share the array and it keeps the last call's contents; every entry a
 * call reads is written earlier in the same call, so nothing needs clearing,
 * but calls whose work can overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. */
chi0_status chi0_accumulate_fp64_noalloc(int n_G, const void* M, int n_v, int n_c, const double* E_v,
                                         const double* E_col, const double* w_col, int n_freq,
                                         const double* freq_re, const double* freq_im, double delta,
                                         void* chi0, void* stream);

/* Non-uniform and higher-order quadrature of the Eq. 3 integral (the text
 * after Eq. 4 allows uniform or non-uniform grids and higher-order rules), with
 * several states per node (host arrays, host computation).  Columns
 * 0..N0-1 are the explicit bands (own energy, weight 1).  The interval
 * [E_0, E_max], E_0 = E_c[N0-1], is cut into N_E = ceil((E_max-E_0)/dE) bins:
 *   grid 0: edges E_0 + k dE, the last clipped at E_max (Eq. 4);
 *   grid 1: equal counts of g between neighbouring edges, i.e.
 *           A c (e_k - V0)^(3/2) = A c (E_0 - V0)^(3/2) + k/N_E [A c (E_max - V0)^(3/2) - A c (E_0 - V0)^(3/2)],
 *           c = 2 sqrt(2)/3, the integral of g(E) = A sqrt(2 (E - V0)).
 * Nodes and raw weights per bin [a, b], h = b - a:
 *   rule 0: midpoint (a+b)/2, h (Eq. 4);
 *   rule 1: Simpson a, (a+b)/2, b with h/6, 4h/6, h/6 (shared ends merged into one node);
 *   rule 2: two-point Gauss-Legendre (a+b)/2 -+ h/(2 sqrt 3), h/2 each.
 * Each node E_k with weight W_k = g(E_k) x raw weight contributes `states`
 * columns: the bands above N0 nearest in energy to E_k (ties to the lower
 * index, in order of distance), each with energy E_k and weight W_k / states
 * (all bands above N0 if there are fewer).  grid 0, rule 0, states 1 gives
 * exactly chi0_select_accelerated.  Returns the number of columns written to
 * c_sel (host int32), E_sel, w_sel (host double), or -1 for bad arguments,
 * unsorted E_c or more than cap columns. */
int chi0_select_quadrature(const double* E_c, int n_c, int N0, double dE, double dos_A, double dos_V0,
                           double E_max, int grid, int rule, int states, int32_t* c_sel, double* E_sel,
                           double* w_sel, int cap);

/* Adaptive grid for the Eq. 3 integral driven by the adjoint (host arrays,
 * host computation).  sens (host) [n_c] holds dL/dE_c for some loss L (e.g.
 * grad_Ecol of chi0_backward on a cheap proxy of the workload).  Starting
 * from the uniform grid of step dE on [E_0, E_max] (as chi0_select_accelerated),
 * the bin [a, b) with the largest first-order estimate of the error of Eq. 4's
 * energy substitution,  |sum_{N0 <= c, a <= E_c < b} sens[c] ((a+b)/2 - E_c)|
 * (the last bin closed at E_max), is halved, n_split times (ties: the lowest
 * bin).  Each bin then contributes the midpoint node with weight g(E_k) (b - a)
 * shared by its `states` nearest bands above N0, as chi0_select_quadrature.
 * n_split = 0 gives chi0_select_accelerated.  Returns the number of columns,
 * or -1 for bad arguments, unsorted E_c or more than cap columns. */
int chi0_select_adaptive(const double* E_c, int n_c, int N0, const double* sens, double dE, double dos_A,
                         double dos_V0, double E_max, int n_split, int states, int32_t* c_sel, double* E_sel,
                         double* w_sel, int cap);

/* ---- Dielectric matrix (section II: eps = 1 - v chi0, W = eps^-1 v; Table III:
 * eps_inf = 1 / [eps^-1]_{00}(q -> 0, omega = 0)).  Hartree atomic units. ---- */

/* Bare Coulomb interaction on sphere iq (host computation):
 *   v_out[j] = 4 pi / (Omega |q + G_j|^2),  q + G_j = (q_frac + g_j) . B,
 * with B the reciprocal lattice (rows b_i, a_i . b_j = 2 pi delta_ij) of the
 * direct lattice `lattice` (host [3][3], rows a_i in bohr) and Omega = |det A|.
 * q_frac (host [3]) is q in reciprocal-lattice units; v_out (host) [n_G[iq]].
 * CHI0_ERR_INVALID for a singular lattice or q + G_j = 0. */
chi0_status chi0_coulomb(chi0_plan plan, int iq, const double* lattice, const double* q_frac, double* v_out);

/* eps[w][G][G'] = delta_GG' - v[G] chi0[w][G][G']                     (symmetric = 0)
 *             or delta_GG' - v[G]^1/2 chi0[w][G][G'] v[G']^1/2        (symmetric = 1; same
 * eigenvalues and same diagonal of the inverse, Hermitian when chi0 is).
 * chi0, eps: (device) [n_freq][n_G[iq]][n_G[iq]] complex128, may be the same buffer;
 * v: (device) [n_G[iq]] FP64 (e.g. from chi0_coulomb). */
chi0_status chi0_epsilon(chi0_plan plan, int iq, const void* chi0, const double* v, int symmetric, void* eps,
                         void* stream);

/* In-place inverse of the n_freq matrices eps[w] ((device) [n_freq][n_G[iq]][n_G[iq]]
 * complex128, row-major) by blocked Gauss-Jordan elimination with partial
 * pivoting (largest |re| + |im| in the column).  FP64 plans compute in FP64;
 * split plans compute in FP32 on a complex64 copy and write the result back
 * as complex128 (forward error about cond(eps) x 1e-7).  Workspace (the
 * complex64 copy for split plans, panel buffers) is allocated at the first
 * call for a sphere this large and kept by the plan.  A zero pivot (singular
 * matrix) leaves non-finite values and makes the next chi0_sync_status return
 * CHI0_ERR_SINGULAR. */
chi0_status chi0_epsilon_inverse(chi0_plan plan, int iq, void* eps, void* stream);

/* eps_inf[w] = 1 / eps_inv[w][i0][i0] with i0 the index of G = 0 in sphere iq.
 * eps_inv: (device) as returned by chi0_epsilon_inverse; out: (host) [n_freq]
 * complex128 (re, im interleaved).  Synchronises `stream`.  CHI0_ERR_INVALID
 * if the sphere does not contain G = 0. */
chi0_status chi0_eps_inf(chi0_plan plan, int iq, const void* eps_inv, double* out, void* stream);

/* ---- Coulomb-hole self-energy of Eq. 2 with the Hybertsen-Louie plasmon-pole
 * model (the paper's extension of the static eps^-1 to finite frequencies). ---- */

/* Plasmon-pole parameters of sphere iq:
 *   Omega2[G][G'] = w_p^2 [(q+G).(q+G') / |q+G|^2] rho(G - G') / rho(0),  w_p^2 = 4 pi n_el / Omega,
 *   wt[G][G']     = sqrt(Omega2 / (delta_GG' - eps_inv[G][G']))  (principal branch; 0 where the
 *                   denominator vanishes),
 * with rho(d) the Fourier coefficient exp(-i d.r) of the density 2 sum_v |psi_v(r)|^2 at the
 * distinct differences d = G - G' (a transform pruned to the offsets they span).
 * psi_v: (device) [n_v][N_r] valence grids (plan complex type); eps_inv: (device) [N_G][N_G]
 * complex128, the inverse of the plain static eps (chi0_epsilon with symmetric = 0);
 * lattice, q_frac (host) as for chi0_coulomb; n_el electrons per cell; Omega2, wt: (device)
 * [N_G][N_G] complex128 outputs.  Allocates temporaries and synchronises `stream`. */
chi0_status chi0_gpp(chi0_plan plan, int iq, const void* psi_v, int n_v, const void* eps_inv,
                     const double* lattice, const double* q_frac, double n_el, void* Omega2, void* wt,
                     void* stream);

/* Diagonal COH self-energy of target bands t with the plasmon-pole model (Eq. 2 with its
 * frequency integral done in closed form):
 *   sigma[t] = sum_b w[b] sum_{G,G'} m[t][b][G] K_GG'(x[t][b]) conj(m[t][b][G']),
 *   K_GG'(x) = Omega2[G][G'] v[G'] / (2 wt[G][G'] (x - wt[G][G'] + i delta)),  0 where wt or Omega2 is 0,
 * m: (device) [n_t * n_b][N_G] complex, the pair elements <t| e^{iG.r} |b> of chi0_pairs with the
 * targets as the first band set and the bands b (explicit, or the columns of an Eq. 3 selection)
 * as the second; x: (device) [n_t][n_b] FP64, E_t - E_b (E_b the grid energy for an energy-grid
 * state); w: (device) [n_b] FP64 or NULL (= 1); Omega2, wt from chi0_gpp; v: (device) [N_G] FP64;
 * sigma: (host) [n_t] complex128.  Split plans compute the terms in FP32 and sum them in FP64,
 * FP64 plans in FP64; the tile sums are added on the host in a fixed order.  Allocates a
 * workspace (two N_G x N_G tables) and synchronises `stream`. */
chi0_status chi0_sigma_coh(chi0_plan plan, int iq, const void* m, int n_t, int n_b, const double* x,
                           const double* w, const void* Omega2, const void* wt, const double* v,
                           double* sigma, void* stream);

/* Band selection of Eq. 3 / Eq. 4 (host arrays, host computation).
 * E_c (host) [n_c] sorted ascending.  Columns 0..N0-1 are bands 0..N0-1 with
 * their own energy and weight 1.  E_0 = E_c[N0-1]; the interval (E_0, E_max]
 * is cut into N_E = ceil((E_max-E_0)/dE) steps of width dE (the last one
 * clipped at E_max); grid point E_i is the midpoint of step i, dE_i its width,
 * its state is the band above N0 nearest in energy to E_i (ties to the lower
 * index), its energy E_i and its weight g(E_i) dE_i with
 * g(E) = dos_A * sqrt(2 (E - dos_V0)) (zero below dos_V0).
 * Writes up to cap columns to c_sel (host int32), E_sel, w_sel (host double).
 * Returns the number of columns N0 + N_E, or -1 on invalid input or when cap is too small. */
int chi0_select_accelerated(const double* E_c, int n_c, int N0, double dE, double dos_A,
                            double dos_V0, double E_max, int32_t* c_sel, double* E_sel,
                            double* w_sel, int cap);

#ifdef __cplusplus
}
#endif

#endif /* CHI0_H */
