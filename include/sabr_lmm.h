/* sabr_lmm.h -- C-ABI of the B300 (sm_103a) SABR/LIBOR calibration library.
 *
 * The library evaluates, on one GPU, the calibration objective of the SABR/LIBOR market models
 * of Ferreiro, Garcia, Lopez-Salas and Vazquez (arXiv 2408.01470, Sections 2-3), and runs the
 * parallel simulated-annealing search of Section 3 (thousands of Metropolis chains per
 * temperature, a minimum over the chains' end points, the start point broadcast to the next
 * level), followed by an optional Levenberg-Marquardt polish.
 *
 * Conventions for every call:
 *   - Plain pointers only.  "host" pointers are read during the call and may be freed after it;
 *     "device" pointers must be CUDA global memory of the current device, owned by the caller.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *     that take a stream only enqueue work; the caller synchronises before reading outputs.
 *     sabr_lmm_anneal synchronises its own stream before returning.
 *   - Every call returns a sabr_lmm_status.  On any status other than SABR_LMM_OK a message is
 *     available from sabr_lmm_last_error() (thread-local, valid until the next call on the same
 *     thread) and no output has been written, except for SABR_LMM_ECUDA and SABR_LMM_ETIMEOUT
 *     raised after launch, where device outputs are unspecified.
 *   - A parameter point whose model vol for some instrument is not a finite positive number is
 *     infeasible: its objective is +inf.  That is a value, not an error.
 *   - Device-side failure detection: every wait of a kernel on its own asynchronous copies is
 *     bounded.  A wait that gives up raises the market's error word, the affected outputs are set
 *     to NaN (an annealing chain of the affected CTA ends the level with f = +inf), and the kernel
 *     returns normally.  The word is reported, and then cleared, by the next sabr_lmm_sync,
 *     sabr_lmm_anneal_fetch or sabr_lmm_anneal on that market, which returns SABR_LMM_ETIMEOUT
 *     once; stream-ordered calls (objective, residuals, model_vols, objective_grad, lm_polish)
 *     return SABR_LMM_OK at enqueue time and are checked by sabr_lmm_sync.
 */
#ifndef SABR_LMM_H
#define SABR_LMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SABR_LMM_OK = 0,
  SABR_LMM_EINVAL = 1,    /* invalid argument or market description */
  SABR_LMM_ENOMEM = 2,    /* device or host allocation failed */
  SABR_LMM_ECUDA = 3,     /* a CUDA call or kernel failed */
  SABR_LMM_ETIMEOUT = 4,  /* a bounded device-side wait gave up (the context stays usable) */
  SABR_LMM_ENOTSUP = 5    /* valid but not supported by this build (e.g. quad_nodes != 8) */
} sabr_lmm_status;

/* Arithmetic of the hot path.
 *   FP64      : every price, integral and sum in FP64 (the plain form).
 *   FP32      : integrals, SABR vols and Black prices in FP32; the squared residuals summed per
 *               lane and across a warp's lanes in FP32 (markets with swaptions: the warps' sums
 *               added in float-float, a 48-bit significand); the Metropolis test in FP32 and
 *               repeated in FP64 whenever the uniform falls inside the FP32 error band (so the
 *               decision equals the FP64 decision on the same objective values); chain state
 *               in FP32.  Outputs (f, vols, best points) are returned as FP64.
 *   FP32_BF16X3 : FP32, with the pair-integral Grams of the swaption forms (S3) contracted on the
 *               tensor cores (tcgen05) on a split (hi + lo bf16) operand, accumulated in FP32;
 *               markets whose panel tables fit one MMA tile (ENOTSUP otherwise).
 *   The value 2 is not a precision of this library (EINVAL).                                 */
typedef enum {
  SABR_LMM_FP64 = 0,
  SABR_LMM_FP32 = 1,
  SABR_LMM_FP32_BF16X3 = 3
} sabr_lmm_prec;

/* Models (Section 2).
 *   SMILE    : one SABR smile; parameters [alpha, rho, nu] shared by every caplet; beta fixed.
 *   REBONATO : the Rebonato SABR/LIBOR model (Section 2.3), 12 parameter slots
 *              [a, b, c, d, alpha_h, beta_h, gamma_h, delta_h, phi, lambda1, lambda2, lambda3]:
 *              g(u) = (a + b u) e^{-c u} + d and h(u) = (alpha_h + beta_h u) e^{-gamma_h u} + delta_h
 *              at time-to-fixing u, kappa = 1, phi_ii = phi, and the correlations of
 *              Eqs. (rhoij), (thetaij), (phiij) with eta1 = eta2 = 0.
 *   MERCURIO_MORINI : the Mercurio & Morini SABR/LIBOR model (Section 2.2), caplets only, at
 *              most 15 forwards, 2 n_fwd + 1 slots [phi_0..phi_{M-1}, sigma, alpha_0..alpha_{M-1}]:
 *              forward i's smile has rho = phi_i, nu = sigma and the alpha of
 *              Eq. (haganForMercurio), alpha_i exp(-sigma sum_{j <= i} tau_j phi_j alpha_j
 *              F_j^b T_j / (1 + tau_j F_j)) (the drift integral between fixing dates, forward j
 *              fixing at T_j).  The reverse sweep, the Levenberg-Marquardt polish and
 *              sabr_lmm_anneal_noalloc cover at most 12 slots (ENOTSUP); the Nelder-Mead polish
 *              covers every model.                                                          */
typedef enum { SABR_LMM_MODEL_SMILE = 0, SABR_LMM_MODEL_REBONATO = 1, SABR_LMM_MODEL_MERCURIO_MORINI = 2 } sabr_lmm_model;

/* SABR implied-vol formula.
 *   HAGAN2002 : Hagan, Kumar, Lesniewski, Woodward (2002) lognormal expansion with z/x(z) and
 *               the first-order expiry correction (the formula Section 2.1 attributes to Hagan).
 *   PAPER     : Eq. (sigmaHagan) exactly as printed (no expiry dependence).                */
typedef enum { SABR_LMM_HAGAN2002 = 0, SABR_LMM_PAPER = 1 } sabr_lmm_formula;

/* A market: a tenor structure, caplet and swaption quotes, and the parameter box.
 * All arrays are host memory, read during sabr_lmm_load_market only.
 *   T[n_fwd+1]   : T[k] is the fixing time of forward k (years, strictly increasing, > 0);
 *                  T[n_fwd] is the payment time of the last forward.  Accrual tau_k = T[k+1]-T[k].
 *   P[n_fwd+1]   : discount factors P(0, T[k]) > 0.  Forward k is (P[k]/P[k+1] - 1) / tau_k.
 *   cap_fwd[n_cap], cap_K[n_cap], cap_vol[n_cap] : caplet on forward cap_fwd[k] (expiry T[k],
 *                  paid at T[k+1]) struck at cap_K[k] > 0, quoted at Black vol cap_vol[k] > 0.
 *   cap_w        : NULL -> weight 1/vega^2 at the quoted vol; else caller weights >= 0.
 *   swp_start/swp_end/swp_K/swp_vol[n_swp] : swaption expiring at T[swp_start] on the swap
 *                  over forwards [swp_start, swp_end) (annuity sum tau_k P[k+1], frozen weights).
 *   swp_w        : as cap_w.
 *   lo/hi[n_param], free_mask[n_param] : search box and the slots the annealer moves (1) or
 *                  keeps (0).  n_param must be 3 (SMILE), 12 (REBONATO) or 2 n_fwd + 1
 *                  (MERCURIO_MORINI).
 *   panel        : quadrature panel width (years); for REBONATO every T[k] must be a whole
 *                  multiple of it.  quad_nodes: Gauss-Legendre nodes per panel (8 only).
 * Quotes are vols: the library prices them with Black's formula (the out-of-the-money option:
 * a put below the forward, a call at or above it) to get the market prices.                  */
typedef struct {
  int32_t model;
  int32_t formula;
  double beta;
  int32_t n_fwd;
  const double* T;
  const double* P;
  int32_t n_cap;
  const int32_t* cap_fwd;
  const double* cap_K;
  const double* cap_vol;
  const double* cap_w;
  int32_t n_swp;
  const int32_t* swp_start;
  const int32_t* swp_end;
  const double* swp_K;
  const double* swp_vol;
  const double* swp_w;
  int32_t n_param;
  const double* lo;
  const double* hi;
  const uint8_t* free_mask;
  double panel;
  int32_t quad_nodes;
} sabr_lmm_market_desc;

typedef struct sabr_lmm_market sabr_lmm_market; /* opaque, library-owned device arena */

/* Validate n_markets descriptions (d[0..n_markets-1]), copy them to the device once and
 * precompute every market-only constant there (forwards, discounts, annuities, swap rates,
 * frozen weights, market prices, vega weights, log-moneyness).  Paper: the problem statement
 * of Section 3 (cost functions f_c and f_s).  Allocates device memory (freed by
 * sabr_lmm_free_market).  Errors: EINVAL (message names the field), ENOMEM, ENOTSUP, ECUDA.  */
sabr_lmm_status sabr_lmm_load_market(const sabr_lmm_market_desc* d, int32_t n_markets,
                                     void* stream, sabr_lmm_market** out);
void sabr_lmm_free_market(sabr_lmm_market* m);

/* f[i] = sum_k w_k (P_k(X[i]) - P_k^mkt)^2 over every caplet and swaption of market
 * `market_idx`, for n parameter sets X (device, row-major n x n_param, FP64).  f: device [n],
 * FP64.  Paper: f_c and f_s of Section 3, the SABR vols of Eq. (sigmaHagan) or Hagan (2002)
 * with the model mappings of Eq. (haganForRebonato).  Errors: EINVAL (n < 0, bad index or
 * precision, NULL pointers with n > 0), ECUDA.                                                */
sabr_lmm_status sabr_lmm_objective(const sabr_lmm_market* m, int32_t market_idx, const double* X,
                                   int64_t n, int32_t prec, double* f, void* stream);

/* The weighted residuals r_k = sqrt(w_k) (P_k(X[i]) - P_k^mkt) of every instrument (caplets first,
 * then swaptions) for n parameter sets: res device [n x (n_cap + n_swp)], FP64, row-major; f
 * (device [n] or NULL) receives sum_k r_k^2 as sabr_lmm_objective would.  The residuals come from
 * the same pricer the annealer's objective runs at this precision (in FP32 the packed-pair
 * pricer), so they are the per-price terms of f.  With the default weights w_k = 1/vega_k^2 at the
 * quoted vol, r_k is the price error in vol units to first order.  Entries whose model vol is not
 * a finite positive number are NaN.  Paper: the terms of f_c and f_s of Section 3.  Same errors
 * as sabr_lmm_objective.                                                                     */
sabr_lmm_status sabr_lmm_residuals(const sabr_lmm_market* m, int32_t market_idx, const double* X,
                                   int64_t n, int32_t prec, double* f, double* res, void* stream);

/* Model Black vols of every instrument (caplets first, then swaptions) for n parameter sets:
 * vols device [n x (n_cap + n_swp)], FP64.  Infeasible entries are NaN.  Same errors.        */
sabr_lmm_status sabr_lmm_model_vols(const sabr_lmm_market* m, int32_t market_idx, const double* X,
                                    int64_t n, int32_t prec, double* vols, void* stream);

/* f[i] and its gradient G[i, :] = df/dtheta (device [n x n_param], FP64, every slot, free or
 * not) by a hand-written reverse-mode (adjoint) sweep through pricing, SABR, the model mapping
 * and the quadrature; for markets with swaptions also through the swap-rate SABR parameters,
 * the quadratic forms of each expiry group, the window integrals, the prefix tables along the
 * diagonals, the pair Grams and the correlation tables (one CTA per point).  Arithmetic per `prec`
 * on caplet markets (FP64, or FP32 accumulating the parameter adjoints in FP64); markets with
 * swaptions are differentiated in FP64 whatever `prec`.  Paper: derivative of the cost functions
 * of Section 3.  Same errors, and ENOTSUP if a market's reverse sweep does not fit one CTA's
 * shared memory, or for a Mercurio & Morini market (the sweep covers the smile and Rebonato
 * models, at most 12 slots).                                                                  */
sabr_lmm_status sabr_lmm_objective_grad(const sabr_lmm_market* m, int32_t market_idx,
                                        const double* X, int64_t n, int32_t prec, double* f,
                                        double* G, void* stream);

/* Simulated annealing (Section 3, one-GPU parallel form).
 * Level l runs at T_l = T0 cooling^l (T_{l+1} = cooling T_l).  Every chain starts the level at
 * the shared start point and runs steps_per_level Metropolis steps: each free slot moves by
 * s_l (hi - lo)(2u - 1), reflected once at the bound it crosses and clamped, with
 * s_l = max(step_frac sqrt(T_l / T0), step_floor); the move is accepted if the objective drops
 * or u < exp(-dE / T_l).  The next start point is the end point with the lowest objective
 * (ties to the lowest chain index).  Uniforms: Philox4x64-10 keyed (seed, 0), counter
 * (block, step, level, chain | market << 32), u = (word >> 11) 2^-53, words 0..n_param-1 move
 * slots 0..n_param-1 and word n_param decides acceptance.  Every chain evaluates f(x0) once,
 * so C (L N + 1) objective evaluations are made.
 *   T0 <= 0  -> T0 = f(x0) (1 if that is not a finite positive number).
 *   x0 NULL  -> box centre.  x0 is host memory [n_markets x n_param], finite, inside the box on
 *   the free slots (EINVAL otherwise; fixed slots keep their given values).
 *   lm_top_k > 0 -> Levenberg-Marquardt polish of the lm_top_k lowest best-ever chain points
 *   (at most lm_max_iter trials; with target_rmse_volpt > 0 a point stops at the target and the
 *   polish ends once any point has reached it), the best polished point returned. */
typedef struct {
  int32_t n_chains;
  int32_t n_levels;
  int32_t steps_per_level;
  double T0;
  double cooling;
  double step_frac;
  double step_floor;
  uint64_t seed;
  const double* x0;
  int32_t prec;
  int32_t lm_top_k;
  int32_t lm_max_iter;
  double target_rmse_volpt;
  int32_t warps_per_block; /* chains (warps) per CTA of the caplet level kernel, 0..28; 0 -> FP32: one
                              CTA of up to 28 chains per SM, FP64: 4 (FP64 is capped at 4); batch:
                              0 -> autotuned CTA size, >= 8 -> 256 threads, else 128; a single
                              market with swaptions: 0..4 -> 128-thread CTAs (one per chain; the
                              faster form), else 256 threads (the tensor-core form always 256) */
  int32_t use_graph;       /* 1 -> the level loop is captured once and replayed as a CUDA graph */
  int32_t record_accepts;  /* 1 -> fill sabr_lmm_result.accept_bits (market 0; small runs)     */
  int32_t polish_nm;       /* 1 -> the lm_top_k points are polished by Nelder-Mead (the paper's
                              hybrid; lm_max_iter iterations, step 0.02, ftol 1e-12) instead of
                              Levenberg-Marquardt                                               */
} sabr_lmm_anneal_opts;

/* Results, per market, in caller-allocated host arrays (any may be NULL).
 *   x_best [n_markets x n_param], f_best, rmse_volpt [n_markets]: best point found (after the
 *   polish when enabled), its objective and its vol RMSE in vol points.
 *   trace_f [n_markets x n_levels]: the start objective of each next level (the per-level min).
 *   accept_bits [n_chains x n_levels x steps] (market 0 only; for tests, small runs).
 *   n_evals: objective evaluations made by the annealer (C (L N + 1) per market).
 *   seconds: device time of the annealing loop; lm_seconds: device time of the polish.
 *   trace_x [n_markets x n_levels x n_param]: the start point of each next level (the best end
 *   point of the level; before any polish).
 *   trace_seconds [n_markets x n_levels]: device time from the search's start (f(x0)) to the end
 *   of each level, read from the GPU's global timer by the CTA that closes the level.          */
typedef struct {
  double* x_best;
  double* f_best;
  double* rmse_volpt;
  double* trace_f;
  uint8_t* accept_bits;
  int64_t n_evals;
  double seconds;
  double lm_seconds;
  double T0_used;
  double* trace_x;
  double* trace_seconds;
} sabr_lmm_result;

sabr_lmm_status sabr_lmm_anneal(const sabr_lmm_market* m, const sabr_lmm_anneal_opts* opts,
                                sabr_lmm_result* out);

/* The same search split for callers that time or overlap it: prepare allocates the chain state
 * and plans the launches; launch enqueues the whole search on `stream` (no host sync); fetch
 * synchronises that stream and copies results; free releases the plan.                      */
typedef struct sabr_lmm_anneal_plan sabr_lmm_anneal_plan;
sabr_lmm_status sabr_lmm_anneal_prepare(const sabr_lmm_market* m, const sabr_lmm_anneal_opts* opts,
                                        void* stream, sabr_lmm_anneal_plan** plan);
sabr_lmm_status sabr_lmm_anneal_launch(sabr_lmm_anneal_plan* plan, void* stream);
sabr_lmm_status sabr_lmm_anneal_fetch(sabr_lmm_anneal_plan* plan, sabr_lmm_result* out);
void sabr_lmm_anneal_plan_free(sabr_lmm_anneal_plan* plan);

/* The launch configuration a plan chose (the autotuners' choices).  Caplet markets: chains (warps)
 * per CTA of the level kernel and its grid; in FP32 with warps_per_block = 0 the chains per CTA are
 * autotuned at prepare time (28, 16, 14, 8, 7, 4 or the one-wave count, each timed on one level of
 * the search's length, at most 100 steps; the one-wave count stays unless another is 2 % faster;
 * every choice runs the same search bit for bit).  Markets with swaptions: threads per CTA (128
 * unless warps_per_block asks for 256; not tuned, since the CTA size orders the partial sums).  A batch: per shared-memory bucket its markets, CTA size, persistent grid and CTAs per SM
 * (the first 16 buckets).  out is host memory.                                                */
typedef struct {
  int32_t chains_per_cta, grid, cta_threads_swaptions, n_buckets;
  int32_t bucket_markets[16], bucket_threads[16], bucket_grid[16], bucket_ctas_per_sm[16];
} sabr_lmm_plan_config;
sabr_lmm_status sabr_lmm_anneal_plan_config(const sabr_lmm_anneal_plan* plan, sabr_lmm_plan_config* out);

/* Synchronise `stream`, then read and clear the error word of every market of m: returns
 * SABR_LMM_ETIMEOUT if a bounded device-side wait of a call on these markets gave up since the
 * word was last read (the outputs of that call are NaN), else SABR_LMM_OK.  The check for the
 * stream-ordered calls.                                                                      */
sabr_lmm_status sabr_lmm_sync(const sabr_lmm_market* m, void* stream);

/* Test hook of the failure detection: raises market_idx's error word on `stream` (stream-ordered)
 * as a device wait that gave up would, without any device wait.  The next sabr_lmm_sync,
 * sabr_lmm_anneal_fetch or sabr_lmm_anneal on the market then reports SABR_LMM_ETIMEOUT once.  */
sabr_lmm_status sabr_lmm_test_raise_error(const sabr_lmm_market* m, int32_t market_idx, void* stream);

/* The annealing search for callers that cannot allocate device memory.  The paper has no
 * counterpart to this call; it exists for code that is not allowed to call cudaMalloc: for
 * example a service that hands the whole device memory to its own pool at start-up, a plug-in
 * host that gives a library a stream but no allocator, or a latency-critical loop where
 * cudaMalloc's implicit device synchronisation would stall other work.
 *   It runs the same search as sabr_lmm_anneal on market `market_idx` (caplet markets and markets
 *   with swaptions; same options, same uniforms, same kernels, so the same result), keeping all of
 *   its working state in one fixed-size array inside the library's device image: 3,637,760 bytes
 *   (3.64 MB), loaded with the library on every GPU that uses it and held until the process exits.
 *   It calls no cudaMalloc, cudaFree or other allocating routine, and enqueues no host copy (the
 *   start point travels as a kernel argument).
 *   Limits: n_chains <= 16384, n_levels <= 4096 (EINVAL names the limit otherwise); lm_top_k and
 *   record_accepts must be 0; the market must fit one CTA's shared memory at `prec` (ENOTSUP, as
 *   for sabr_lmm_anneal).  x0 is host memory [n_param] or NULL (box centre).
 *   Outputs (device, caller-owned): x_best [n_param], f_best [1], trace_f [n_levels] or NULL.
 *   Stream-ordered: it only enqueues work on `stream`; synchronise before reading the outputs.
 *   The first call on a device looks up the array's device address (once per device, with that
 *   device current); make that first call before any stream capture.
 *   Every call uses the same array: two calls whose work overlaps on the GPU (different streams,
 *   or different host threads on one device) race and both results are undefined.  Calls on one
 *   stream are ordered and safe; each call re-initialises everything it reads.                */
sabr_lmm_status sabr_lmm_anneal_noalloc(const sabr_lmm_market* m, int32_t market_idx,
                                        const sabr_lmm_anneal_opts* opts, double* x_best,
                                        double* f_best, double* trace_f, void* stream);

/* Levenberg-Marquardt polish of n points X (device [n x n_param], FP64, updated in place):
 * J by forward differences over the free slots (step 1e-7 max(|theta_p|, 1)), (J^T J + mu diag
 * J^T J) d = -J^T r by Cholesky (J^T r from the reverse sweep of sabr_lmm_objective_grad, run
 * beside the difference stencil; from J where the reverse sweep does not fit a CTA), projection
 * on the box, mu /10 on success, x10 on failure; a
 * point stops at target_rmse_volpt (if > 0) or once mu exceeds 1e16.  f, rmse: device [n] or
 * NULL, those of the final points.  ENOTSUP for a Mercurio & Morini market (it needs the
 * reverse sweep; sabr_lmm_nm_polish covers every model).  Paper: the local polish of the hybrid
 * scheme, Section 3.                                                                          */
sabr_lmm_status sabr_lmm_lm_polish(const sabr_lmm_market* m, int32_t market_idx, double* X,
                                   int64_t n, int32_t max_iter, double target_rmse_volpt,
                                   double* f, double* rmse, void* stream);

/* Nelder-Mead polish of n points X (device [n x n_param], FP64, updated in place): the local search
 * of the paper's hybrid scheme (Section 3), on the free slots, with the standard coefficients
 * (reflection 1, expansion 2, contraction 1/2, shrink 1/2) and every trial point projected onto the
 * box.  The initial simplex is X[i] and, per free slot k, X[i] + step (hi_k - lo_k) e_k (taken
 * downwards where it would leave the box); vertices are ordered by f with a stable sort of the
 * previous order; a point stops after max_iter iterations or once f_worst - f_best <= ftol
 * |f_best|.  f: device [n], the objective of the returned points; evals: device [n] (objective
 * evaluations made) or NULL.  One warp per point on caplet markets, one CTA per point on markets
 * with swaptions.  Errors: EINVAL (max_iter < 0, step not in (0, 1], ftol < 0, NULL pointers with
 * n > 0), ENOTSUP, ECUDA.                                                                     */
sabr_lmm_status sabr_lmm_nm_polish(const sabr_lmm_market* m, int32_t market_idx, double* X, int64_t n,
                                   int32_t max_iter, double step, double ftol, double* f,
                                   int32_t* evals, void* stream);

/* Introspection: the geometry of market market_idx and what its kernels need per CTA.
 *   n_panels, n_diag: absolute 0.5y panels and forward-index diagonals of the swaption tables;
 *   n_swap: distinct swaps behind the swaptions; max_window: most forwards in one expiry group;
 *   smem_fp64, smem_fp32: dynamic shared memory per CTA (one chain per CTA with swaptions, four
 *   chains per CTA for caplet markets); batch_ctas_per_sm_*: 256-thread CTAs of the batch kernel
 *   that fit one SM at that precision (0 if the market does not fit).  out is host memory.  */
typedef struct {
  int32_t n_fwd, n_cap, n_swp, n_swap, n_panels, n_diag, max_window;
  uint32_t smem_fp64, smem_fp32;
  int32_t batch_ctas_per_sm_fp64, batch_ctas_per_sm_fp32;
} sabr_lmm_market_info_t;
sabr_lmm_status sabr_lmm_market_info(const sabr_lmm_market* m, int32_t market_idx,
                                     sabr_lmm_market_info_t* out);

/* Check of the device-side failure detection: one CTA waits, with the library's bounded mbarrier
 * wait limited to `polls` polls (1..2^24), on a phase that never completes (16 bytes announced,
 * none sent).  The wait gives up, raises its error word and the call returns SABR_LMM_ETIMEOUT
 * (SABR_LMM_OK would mean the wait did not give up).  Nothing faults or hangs and the CUDA
 * context stays usable.  Synchronises `stream`.                                              */
sabr_lmm_status sabr_lmm_selftest_wait(int64_t polls, void* stream);

/* Introspection: the Gauss-Legendre rule the kernels use (nodes on [-1,1], weights), q = 8. */
sabr_lmm_status sabr_lmm_quadrature_rule(int32_t q, double* x, double* w);

const char* sabr_lmm_last_error(void);
const char* sabr_lmm_version(void);

/* ---------------------------------------------------------------- Monte Carlo pricer
 * The Hagan SABR/LIBOR model (Section 2.1, Eqs. dinamicasHagan1-2) simulated under the spot
 * measure with the drifts of Section 2.1 (h(t) the first forward not yet fixed), for the Monte
 * Carlo pricing of caplets and swaptions of Section 3 (Table tab:haganMCpricer).
 *   T[n_fwd+1], P[n_fwd+1] : tenor grid and discounts as in a market description: forward k fixes
 *                  at T[k] and is paid at T[k+1], accrual tau_k = T[k+1] - T[k].
 *   beta in [0, 1]; per forward alpha[k] = V_k(0) > 0, sigma[k] >= 0 (vol of vol), phi[k] = phi_kk
 *                  in [-1, 1]; eta1, lambda1, eta2, lambda2, lambda3 of Eqs. (rhoij), (thetaij),
 *                  (phiij): corr(W_i, W_j) = rho_ij, corr(Z_i, Z_j) = theta_ij, corr(W_i, Z_j) =
 *                  sign(phi_ii) sqrt(|phi_ii phi_jj|) e^{-lambda3 |T_i - T_j|}.  An indefinite
 *                  correlation matrix (the printed form makes one when the phi_kk differ in sign)
 *                  is replaced by the nearest correlation matrix in the spectral sense (negative
 *                  eigenvalues set to zero, rows rescaled to unit length), everywhere (increments
 *                  and drifts).
 *   caplets  : cap_fwd[n_cap], cap_K[n_cap] >= 0: tau_k (F_k(T_k) - K)^+ paid at T[k+1].
 *   swaptions: swp_start/swp_end/swp_K[n_swp]: the payer swaption expiring at T[start] on the
 *                  swap over forwards [start, end): A (S - K)^+ at expiry, A and S from the
 *                  forwards at expiry.
 * The instruments may reach at most 16 forwards (cap_fwd < 16, swp_end <= 16; ENOTSUP beyond);
 * at most 4096 instruments.  All arrays are host memory, read during sabr_lmm_mc_prepare.     */
typedef struct {
  int32_t n_fwd;
  const double* T;
  const double* P;
  double beta;
  const double* alpha;
  const double* sigma;
  const double* phi;
  double eta1, lambda1, eta2, lambda2, lambda3;
  int32_t n_cap;
  const int32_t* cap_fwd;
  const double* cap_K;
  int32_t n_swp;
  const int32_t* swp_start;
  const int32_t* swp_end;
  const double* swp_K;
  int32_t model;   /* SABR_LMM_MODEL_SMILE (0): the Hagan dynamics above; SABR_LMM_MODEL_MERCURIO_MORINI
                    * (2): the one-factor volatility of Section 2.2, dF_i = mu_i dt + alpha_i V F_i^beta
                    * dW_i, dV = sigma V dZ, V(0) = 1, with sigma[0] the common vol of vol, phi[i] =
                    * corr(W_i, Z), corr(W_i, W_j) = rho_ij (eta1, lambda1) and mu_i the spot-measure
                    * drift alpha_i V F_i^beta sum_{j<=i} rho_ij tau_j alpha_j V F_j^beta / (1 + tau_j
                    * F_j); eta2, lambda2, lambda3 and sigma[1..] unused.  Others: EINVAL.         */
} sabr_lmm_mc_desc;

/* n_paths in [1, 2^40]; dt > 0: every interval between fixings (and [0, T[0]]) is cut into
 * ceil(len / dt) equal steps; seed: the key of the paths' Philox4x32-10 streams (path p, step s,
 * block b at counter (b, s, p low, p high)); prec: FP64 or FP32 (the path arithmetic and the
 * payoffs with their sums over a warp's 32 paths; the warp sums accumulated in FP64); grid: CTAs (0: enough for every path, at most one wave per SM, the rest looped); a CTA
 * takes 512 paths in FP32 and 128 in FP64 (fewer, in whole warps, when the paths do not fill one
 * such CTA per SM), halved while its per-warp sums (16 bytes per instrument and warp) would not
 * fit in 227 KB of shared memory.                                                              */
typedef struct {
  int64_t n_paths;
  double dt;
  uint64_t seed;
  int32_t prec;
  int32_t grid;
} sabr_lmm_mc_opts;

typedef struct sabr_lmm_mc_plan sabr_lmm_mc_plan; /* opaque: the model constants and device buffers */

/* Validate, build the time grid and the model constants (host, FP64: the correlation matrix, its
 * spectral repair and Cholesky factor), allocate the plan's device buffers.  Synchronises
 * `stream` once.  Errors: EINVAL (message names the field), ENOTSUP, ENOMEM, ECUDA.            */
sabr_lmm_status sabr_lmm_mc_prepare(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o, void* stream,
                                    sabr_lmm_mc_plan** out);
/* Enqueue one pricing on `stream` (the device of the plan): every path (one thread each) steps
 * F by Euler (absorbed at zero: the CEV forward with beta < 1 reaches it) and ln V by log-Euler,
 * the drifts frozen over a step, the increments L xi from Box-Muller normals; at each fixing the
 * instruments fixing there are paid and deflated by the spot numeraire B(T_{k+1}) =
 * prod_{j <= k} (1 + tau_j F_j(T_j)) / P(0, T_0).  A path whose F or ln V is not finite at a
 * fixing pays nothing from there on and is counted in n_bad.  Outputs (device, caller-owned, or
 * all NULL to keep them in the plan): price[n_cap + n_swp] (caplets, then swaptions, in the
 * order given) = mean deflated payoff over n_paths, stderr_out[same] = its standard error,
 * n_bad[1].  Asynchronous; calls on one plan must not overlap on the GPU.                      */
sabr_lmm_status sabr_lmm_mc_launch(sabr_lmm_mc_plan* p, double* price, double* stderr_out,
                                   long long* n_bad, void* stream);
void sabr_lmm_mc_plan_free(sabr_lmm_mc_plan* p);
/* prepare + launch + copy back: price, stderr_out (or NULL), n_bad (or NULL) are host memory.
 * Synchronous.                                                                                 */
sabr_lmm_status sabr_lmm_mc_price(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o, double* price,
                                  double* stderr_out, int64_t* n_bad, void* stream);

/* The swaption calibration of Section 3 by simulated annealing over a Monte Carlo objective: the
 * correlation parameters y = (eta1, lambda1, eta2, lambda2, lambda3) minimise
 *   f_s(y) = sum_k (P_k^Black - P_k^MC(y))^2
 * over the description's instruments (caplets, then swaptions), with its alpha, sigma, phi fixed
 * (the caplet calibration's result) and its own correlation fields ignored.  P_k^Black: Black's
 * formula at quote_vol[k] (host, [n_cap + n_swp], > 0): caplet on forward i with discount
 * tau_i P(0, T[i+1]) and forward F_i(0); payer swaption over [a, b) with annuity sum tau_k
 * P(0, T[k+1]) and swap rate (P(0, T[a]) - P(0, T[b])) / annuity; expiry T[i] or T[a].
 * P_k^MC(y): sabr_lmm_mc_launch's price with `mc` (n_paths, dt, seed, prec) at y; the same seed at
 * every y (common random numbers), so f_s is a deterministic function of y.
 * The search: the annealing loop of sabr_lmm_anneal on the 5-slot box lo/hi/free_mask (0 <= lo <=
 * hi, eta's <= 1), from y0 (or the box centre), T0 (<= 0: f_s(y0)), the same neighbour rule and
 * Philox4x64-10 uniforms (word k moves slot k, word 5 decides, chain c at counter (block, step,
 * level, c) under key (seed, 0)).  Every step evaluates the n_chains proposals in one launch (a
 * CTA grid per proposal, its constants staged in shared memory); the proposals' correlation
 * factors are built by a pool of host threads that lives for the call, the Metropolis decisions
 * taken on the host in FP64.
 * Synchronous; allocates device and pinned host memory for the search.                       */
typedef struct {
  int32_t n_chains, n_levels, steps_per_level;
  double T0, cooling, step_frac, step_floor;
  uint64_t seed;
  const double* y0;             /* [5] or NULL */
  const double* lo;             /* [5] */
  const double* hi;             /* [5] */
  const uint8_t* free_mask;     /* [5] */
} sabr_lmm_mc_anneal_opts;

typedef struct {
  double y_best[5];             /* the best point ever accepted */
  double f_best;
  double T0_used;
  int64_t n_evals;              /* Monte Carlo objective evaluations: n_chains n_levels steps + 1 */
  double seconds;               /* host wall time of the search */
  double* trace_f;              /* caller [n_levels] or NULL: each level's best end value */
  double* trace_y;              /* caller [n_levels x 5] or NULL: each next level's start point */
} sabr_lmm_mc_anneal_result;

sabr_lmm_status sabr_lmm_mc_anneal(const sabr_lmm_mc_desc* d, const double* quote_vol, const sabr_lmm_mc_opts* mc,
                                   const sabr_lmm_mc_anneal_opts* o, sabr_lmm_mc_anneal_result* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SABR_LMM_H */
