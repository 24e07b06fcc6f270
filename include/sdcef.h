/*
 * sdcef.h - C ABI of the batched GB300 solver for the implicit electron-density /
 * electric-potential system of the MISDC method (Esclapez, Ricchiuti, Bell,
 * Day, arXiv:1904.08510, Sec. 3.2).
 *
 * Every call solves, or evaluates pieces of, the backward-Euler system of
 * Eq. nls for many independent 1D columns:
 *
 *   F_e   = -n_e + f_e - dt div( n_e v - D_e grad n_e )                     = 0
 *   F_phi = -n_e + f_phi + (eps0 eps_r / e) lap(phi)                         = 0
 *
 * with f_e = n_e^n + dt I_Re, f_phi = sum_m nu_m n_m (provisional ion number
 * densities times valence), electron velocity v = U + mu grad(phi)
 * (mu = |kappa_e|, Sec. 2.2) and Einstein diffusivity D_e = mu k_B T / e
 * (Sec. 2.1). Space: uniform cell-centred finite volumes, Scharfetter-Gummel
 * electron face fluxes, Dirichlet potentials V_L, V_R at the electrodes
 * (second-order one-sided face gradient), electrons absorbed by the
 * electrodes (drift outflow only) or, as a test mode, zero-gradient.
 * The solve is the Jacobian-free Newton-Krylov iteration of Algorithm 2:
 * scaled Newton (Eq. newton_sc), GMRES with the finite-difference
 * Jacobian-vector product of Eq. jf_dfapprox, the Schur-factorised
 * preconditioner of Eq. prec / Eq. prec_recast, and a backtracking line search.
 *
 * Memory: all array arguments are DEVICE pointers unless marked HOST. The
 * caller owns every array; the library owns only the workspace it allocates
 * in sdcef_create. Per-cell arrays hold the columns back to back: the cells
 * of column c are [col_off[c], col_off[c+1]).
 *
 * Streams: calls are enqueued on the stream given to sdcef_create and return
 * without synchronising, except where stated. sdcef_solve_batch allocates
 * nothing and does not synchronise.
 *
 * Errors: functions return SDCEF_SUCCESS (0) or a negative SDCEF_ERR_* code;
 * sdcef_last_error() gives a message. Per-column outcomes are reported in the
 * status array (SDCEF_STATUS_*); a failed column's outputs hold its last
 * iterate.
 */
#ifndef SDCEF_H
#define SDCEF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SDCEF_SUCCESS 0
#define SDCEF_ERR_INVALID (-1)     /* bad argument (null pointer, size, range)   */
#define SDCEF_ERR_CUDA (-2)        /* a CUDA runtime call failed                 */
#define SDCEF_ERR_CAPACITY (-3)    /* batch larger than the sizes given at create */
#define SDCEF_ERR_NOMEM (-4)       /* workspace allocation failed                */

/* per-column status */
#define SDCEF_STATUS_OK 0              /* ||S_F^-1 F||_inf < eps_F (then the error
                                          test of eps_E), or step < eps_X         */
#define SDCEF_STATUS_MAX_NEWTON 1      /* Newton iteration cap reached                */
#define SDCEF_STATUS_MAX_KRYLOV 2      /* GMRES cap reached and line search failed    */
#define SDCEF_STATUS_LINESEARCH_FAIL 3 /* no sufficient decrease after max halvings   */
#define SDCEF_STATUS_NONFINITE 4       /* a residual or pivot became NaN/Inf          */
#define SDCEF_STATUS_BAD_INPUT 5       /* < 2 cells, too many cells, T <= 0, dt <= 0, NaN */

/* precision of the Krylov solve and preconditioner (Sec. 3.2 has no stated
 * precision; FP64 everywhere is the reference mode) */
#define SDCEF_FP64 0       /* everything in FP64                                   */
#define SDCEF_MIXED 1      /* GMRES basis, Arnoldi and preconditioner in FP32;
                              residuals, JVP differencing, Newton update and the
                              stopping test in FP64                                */
#define SDCEF_MIXED_DF 2   /* preconditioner (factorisation and solves) in
                              double-float arithmetic (pairs of FP32 numbers,
                              ~48-bit significand, FP32 exponent range); GMRES
                              basis, Arnoldi, residuals, JVP, Newton update and
                              the stopping test in FP64                            */

/* preconditioner (Sec. 3.2) */
#define SDCEF_PREC_EXACT 0   /* Eq. prec with the exact Schur complement:
                                P^-1 = J^-1, applied in 1D as a block-tridiagonal
                                solve on the cell-interleaved (n_i, phi_i) unknowns */
#define SDCEF_PREC_RECAST 1  /* Eq. prec_recast: three tridiagonal solves with the
                                approximate Schur complement S~ = L + I_e dt D_r   */
#define SDCEF_PREC_NONE 2    /* no preconditioner (diagnostics)                    */
#define SDCEF_PREC_MG 3      /* Eq. prec_recast with the (dt D_f - I) and S~ blocks
                                solved by geometric multigrid V-cycles to the
                                tolerances mg_gamma_A / mg_gamma_S (Sec. 4.2:
                                two red-black Gauss-Seidel relaxations going down
                                and up every level); SDCEF_FP64 precision only    */

/* multigrid grid transfers (SDCEF_PREC_MG; the paper does not name them) */
#define SDCEF_MG_OPERATOR 0  /* operator-dependent (black-box multigrid): a fine-only
                                unknown i interpolates -T[i][k]/T[i][i] from its
                                coarse neighbour k and restricts with -T[k][i]/T[i][i];
                                coarse operator R T P                               */
#define SDCEF_MG_LINEAR 1    /* linear interpolation (1/2, 1/2), R = P^T, coarse
                                operator R T P                                      */

/* electron transport model (Sec. 2.2) */
#define SDCEF_TRANSPORT_CONSTANT 0  /* constant mobility, Einstein diffusivity mu k_B T / e */
#define SDCEF_TRANSPORT_TABLE 1     /* mu and D from tables over the progress variable
                                       c = (T - T_in)/(T_max - T_in) and the reduced field
                                       |E|/N (sdcef_set_transport_table); FP64 with the
                                       exact, recast or no preconditioner; 128 threads per
                                       column; needs batch->rho                          */

/* provisional charged species between SDC iterations (sdcef_sdc_sweep) */
#define SDCEF_ION_DRIFT_UPWIND 0  /* electric drift only, first-order upwind, explicit */
#define SDCEF_ION_GODUNOV 1       /* the transport of Sec. 3.1 / Algorithm 1: effective-
                                     velocity advection by a second-order Godunov scheme,
                                     implicit diffusion, SDC diffusion correction      */

/* electron boundary condition at the electrodes (the paper states none) */
#define SDCEF_BC_ABSORBING 0      /* drift outflow only, no emission, no diffusion */
#define SDCEF_BC_ZERO_GRADIENT 1  /* boundary flux v n_edge in both directions     */

typedef struct sdcef_ctx sdcef_ctx;

typedef struct {
  double eps_F;       /* Newton stop: ||S_F^-1 F(X)||_inf < eps_F (Sec. 3.2); 1e-10   */
  double eps_X;       /* Newton stop on the scaled step, 0 = off (Sec. 3.2)           */
  double gamma;       /* GMRES forcing term ||J dX + F|| < gamma ||F|| (Table 1: 1e-4) */
  double mobility;    /* electron mobility magnitude mu [m^2/(V s)] (Sec. 2.2: 0.4)   */
  double ls_alpha;    /* sufficient-decrease constant of the line search; 1e-4        */
  double eps_r;       /* relative permittivity (Sec. 2.1: 1)                          */
  int restart_m;      /* GMRES restart length, 1..SDCEF_MAX_RESTART                   */
  int max_newton;     /* Newton iteration cap                                         */
  int max_krylov;     /* GMRES iteration cap per Newton step                          */
  int max_linesearch; /* line-search halvings before LINESEARCH_FAIL                  */
  int precision;      /* SDCEF_FP64 | SDCEF_MIXED | SDCEF_MIXED_DF                    */
  int precond;        /* SDCEF_PREC_EXACT | SDCEF_PREC_RECAST | SDCEF_PREC_NONE       */
  int bc_electron;    /* SDCEF_BC_ABSORBING | SDCEF_BC_ZERO_GRADIENT                  */
  int threads_per_column; /* 0 = chosen per column length; else 32, 64, 128 or 256;
                             SDCEF_PREC_MG always runs 128                         */
  int guess_newton_cap; /* Newton steps allowed from a supplied start (ne_guess /
                           phi_guess) before that column restarts from the plain
                           start X^n with the remaining budget; 0 = never restart  */
  double guess_reject_ratio; /* a supplied start whose scaled residual 2-norm exceeds
                           this multiple of the plain start's is replaced by X^n
                           before the first Newton step; 0 = never                  */
  double mg_gamma_A;  /* SDCEF_PREC_MG: V-cycles of the (dt D_f - I) block stop at
                         ||b - A x||_2 <= mg_gamma_A ||b||_2 (Sec. 4.2: gamma_MG);
                         <= 0 solves that block exactly (partitioned Thomas)    */
  double mg_gamma_S;  /* SDCEF_PREC_MG: the same for the S~ block                 */
  int mg_max_cycles;  /* SDCEF_PREC_MG: V-cycles per block solve, 1..1000; a cycle
                         that does not lower the residual also ends the solve  */
  int mg_transfer;    /* SDCEF_PREC_MG: SDCEF_MG_OPERATOR | SDCEF_MG_LINEAR       */
  int ion_scheme;     /* provisional ions of sdcef_sdc_sweep: SDCEF_ION_GODUNOV |
                         SDCEF_ION_DRIFT_UPWIND                                 */
  int transport;      /* SDCEF_TRANSPORT_CONSTANT | SDCEF_TRANSPORT_TABLE         */
  double gas_molar_mass; /* kg/mol; background gas number density N = rho N_A / W */
  double eps_E;       /* error test at the stop, 0 = off. Sec. 3.2 asks that the
                         tolerances keep the solution error small; the residual
                         test alone bounds it only through the conditioning of the
                         scaled Jacobian. Once ||S_F^-1 F||_inf < eps_F holds, the
                         Newton correction P^-1 F(X) of the last Newton step's
                         preconditioner (P = J for SDCEF_PREC_EXACT) estimates the
                         error of X; the column stops only if, per field, its
                         max-norm is <= eps_E times the field's max-norm, else it
                         takes up to 2 more Newton steps (full steps, accepted on
                         sufficient decrease or if the residual test still holds;
                         a rejected one ends the solve at X). Default 5e-10.    */
  double stall_ratio; /* a GMRES restart cycle whose recomputed linear residual
                         exceeds stall_ratio times the residual at its start
                         ends the GMRES solve of that Newton step with the
                         correction reached (stagnation, e.g. at the attainable
                         accuracy of FP32 Krylov vectors); 0 = never. In [0, 1);
                         default 0.9. The paper states no GMRES cap; this and
                         max_krylov are safeguards of this implementation.     */
  int krylov_on_chip; /* 1: the Krylov vectors of a column (Algorithm 2's
                         GMRES: w, v_0, z_0 = P^-1 v_0, the error test's
                         correction, the correction sum, then v_i, z_i in order)
                         that fit in the shared memory the solver kernel leaves
                         unused at its occupancy live there for the whole solve
                         of that column, the others in its workspace slot;
                         0 (default): all in the slot. Results are bit-identical
                         either way; the shared memory is taken from the L1
                         cache, so which is faster depends on the batch:
                         sdcef_autotune_on_chip measures it.                    */
  double guess_progress; /* a supplied start whose Newton step leaves the scaled
                         residual max-norm above this fraction of the previous
                         step's (while the residual test does not hold) is
                         judged to wander and restarts from X^n, as after
                         guess_newton_cap steps (which must be > 0); 0 = never.
                         In [0, 1].                                             */
  int sdc_poisson_start; /* sdcef_sdc_sweep, iterations k >= 2: 1 (default) starts
                         from the previous iterate's n_e with the potential of
                         its charge under the new provisional ions (the root of
                         F_phi, which is linear in phi); 0 starts from the
                         previous iterate as it is. The root is the same.      */
} sdcef_params;

#define SDCEF_MAX_RESTART 32
#define SDCEF_MAX_SPECIES 16

/* One batch of independent columns (Sec. 3.2, Eq. pnp / Eq. nls inputs). */
typedef struct {
  int64_t ncol;              /* number of columns                                   */
  const int64_t* col_off;    /* [ncol+1] cell offsets, col_off[0] = 0               */
  const double* length;      /* [ncol] column length L [m]                          */
  const double* dt;          /* [ncol] backward-Euler step dt [s]                   */
  const double* v_left;      /* [ncol] electrode potential at x = 0 [V]             */
  const double* v_right;     /* [ncol] electrode potential at x = L [V]             */
  const double* ne_old;      /* [cells] n_e^n [m^-3]                                 */
  const double* phi_old;     /* [cells] phi^n [V]; with ne_old, the scaling point   */
  int n_species;             /* charged species in f_phi, 0..SDCEF_MAX_SPECIES      */
  const int* valence;        /* HOST [n_species] charge number nu_m                 */
  const double* n_ion;       /* [n_species][cells] provisional ion densities [m^-3] */
  const double* T;           /* [cells] temperature [K]                             */
  const double* rho;         /* [cells] density [kg/m^3]; not used by the constant-
                                mobility transport model, may be NULL              */
  const double* u_adv;       /* [cells] advective velocity [m/s] or NULL (= 0)      */
  const double* i_re;        /* [cells] electron source [m^-3 s^-1] or NULL (= 0)   */
  const double* ne_guess;    /* [cells] Newton start or NULL (start = ne_old)       */
  const double* phi_guess;   /* [cells] Newton start or NULL (start = phi_old)      */
} sdcef_batch;

/* Per-column results; every pointer may be NULL except ne_out and phi_out. */
typedef struct {
  double* ne_out;     /* [cells] converged n_e; may alias ne_old / ne_guess   */
  double* phi_out;    /* [cells] converged phi; may alias phi_old / phi_guess */
  int* status;        /* [ncol] SDCEF_STATUS_*                                */
  int* newton_it;     /* [ncol] Newton updates taken                          */
  int* krylov_it;     /* [ncol] GMRES iterations (operator applications)      */
  int* res_evals;     /* [ncol] residual evaluations                          */
  double* final_res;  /* [ncol] ||S_F^-1 F||_inf at exit                      */
  int* mg_cycles;     /* [ncol] V-cycles of all multigrid block solves
                         (SDCEF_PREC_MG; 0 otherwise)                         */
} sdcef_result;

/* Fill p with the defaults: eps_F 1e-10, eps_X 0, eps_E 5e-10, stall_ratio 0.9,
 * Krylov vectors in the slot (krylov_on_chip 0),
 * gamma 1e-4 (Table 1),
 * mobility 0.4 (Sec. 2.2), ls_alpha 1e-4, eps_r 1, restart 8, 50 Newton
 * steps, 200 Krylov iterations per step, 20 halvings, FP64, exact Schur
 * preconditioner, absorbing electrodes, automatic threads per column, and a
 * supplied start rejected if its residual is over 30x the plain start's,
 * restarted from X^n after a step that leaves its residual above 0.3x the
 * previous one and judged after 8 Newton steps; for SDCEF_PREC_MG, gamma_MG = 1e-4 on both
 * blocks (the optimum of Sec. 4.2), at most 50 V-cycles per block solve and
 * operator-dependent transfers; the paper's ion transport in the SDC sweep
 * (SDCEF_ION_GODUNOV), whose later iterations start from the potential of the
 * previous charge under the new ions (sdc_poisson_start 1); constant electron
 * transport, gas molar mass 0.028 kg/mol. */
void sdcef_default_params(sdcef_params* p);

/* Electron transport tables for SDCEF_TRANSPORT_TABLE (Sec. 2.2: mobility
 * and diffusion coefficient tabulated against the progress variable c and the
 * reduced field |E|/N, interpolated during the solve). mu, D: HOST arrays
 * [nc][nx], row k at c = k/(nc - 1), column j at E/N = j en_max_td/(nx - 1)
 * Td (1 Td = 1e-21 V m^2), m^2/(V s) and m^2/s, finite and positive; c of a
 * cell is (T - T_in)/(T_max - T_in) clamped to [0, 1]. Bilinear interpolation,
 * clamped at the table edges; a face takes the means of its cells' c and N and
 * E/N = |dphi/dx| / N at the face. The finite-difference Jacobian-vector
 * product carries the field dependence, and the preconditioner's analytic
 * Jacobian includes the slopes of the interpolant in E/N. The tables are copied to the
 * device (allocated here, replacing earlier ones). nc, nx >= 2, en_max_td > 0,
 * T_max > T_in; SDCEF_ERR_INVALID otherwise. */
int sdcef_set_transport_table(sdcef_ctx* ctx, int nc, int nx, double en_max_td, double T_in,
                              double T_max, const double* mu, const double* D);

/* Create a solver context. max_cols, max_cells and max_col_cells bound every
 * later batch (columns, total cells, cells of the longest column); the
 * workspace is sized from them and allocated here, on the current device.
 * stream is a cudaStream_t (NULL = legacy default stream). Returns
 * SDCEF_ERR_INVALID for bad sizes/params and SDCEF_ERR_NOMEM / _CUDA on
 * allocation failure; *out is set only on success. */
int sdcef_create(sdcef_ctx** out, const sdcef_params* p, int64_t max_cols,
                 int64_t max_cells, int max_col_cells, void* stream);

/* Release the context and its workspace (synchronises its stream). NULL is a no-op. */
int sdcef_destroy(sdcef_ctx* ctx);

/* Replace the parameters of an existing context (same validation as create;
 * restart_m may not exceed the value given at create). */
int sdcef_set_params(sdcef_ctx* ctx, const sdcef_params* p);

/* Solve F(X) = 0 for every column of the batch (Algorithm 2). Device
 * pointers; enqueued on the context stream; no allocation, no host sync, so
 * it can be captured in a CUDA graph. Argument errors are detected on the
 * host and return before launching. */
int sdcef_solve_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const sdcef_result* out);

/* The same solve with every pointer in HOST memory (n_ion, T, ... and all
 * outputs): copies the inputs into a staging area owned by the context,
 * solves, copies the results back and synchronises the stream. */
int sdcef_solve_batch_host(sdcef_ctx* ctx, const sdcef_batch* batch, const sdcef_result* out);

/* Solve nbatch batches given in host memory, one after another, with the
 * copies overlapping the solves: the inputs of batch k + 1 go to the device
 * and the results of batch k - 1 come back while batch k is solved (two
 * staging halves owned by the context, one copy stream each way). batches[k]
 * and out[k] follow the rules of sdcef_solve_batch_host; every batch fits the
 * context (max_cols, max_cells, max_col_cells). Returns when all results are in
 * host memory; on an error the batches not yet solved are not solved. Host
 * buffers should be pinned for the copies to overlap. Not part of the paper:
 * the serving form of the batched solve. */
int sdcef_solve_batches_host(sdcef_ctx* ctx, int nbatch, const sdcef_batch* batches,
                             const sdcef_result* out);

/* Evaluate the residual F(X) of Eq. nls at X = (ne, phi) for every column
 * (device pointers, [cells] each). Enqueued on the context stream. */
int sdcef_residual_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* ne,
                         const double* phi, double* F_e, double* F_phi);

/* The Bernoulli function of the Scharfetter-Gummel electron flux (Sec. 3.1),
 * B(x) = x / (e^x - 1), and its derivative B'(x), evaluated exactly as the
 * residual kernel evaluates them (series for |x| < 1e-3, otherwise a
 * table-driven e^|x| - 1 and B(-a) = a + B(a)). x, b, db: device arrays of n
 * doubles; b and db are written. Enqueued on the context stream. Returns
 * SDCEF_ERR_INVALID for NULL arrays or n < 0. */
int sdcef_bernoulli_batch(sdcef_ctx* ctx, const double* x, double* b, double* db, int64_t n);

/* Bounds-checking build (the library compiled with -DSDCEF_CHECKS; not an
 * operation of the paper: the stand-in for a device memory checker). In that
 * build every plane, level, shared-memory and global index the kernels form is
 * tested before use; a failing test records its site number (a code of
 * csrc/checks.cuh) in the check word of the context or MLP handle, the first
 * failure winning, and the access is redirected inside its array; nothing
 * traps. sdcef_checks_compiled returns 1 in that build, 0 otherwise.
 * sdcef_check_word / sdcef_mlp_check_word synchronise the stream, store the
 * word in *word (HOST; 0 = no failed test) and clear it; in the normal build
 * the word stays 0. They return SDCEF_ERR_INVALID for NULL arguments. */
int sdcef_checks_compiled(void);
int sdcef_check_word(sdcef_ctx* ctx, unsigned* word);

/* Measurement aid, not an operation of the paper: the FP64 (precision =
 * SDCEF_FP64) or FP32 (SDCEF_MIXED) FMA throughput of this GPU, the
 * denominator of the solver kernel's ALU roofline. Runs 8 independent FMA
 * chains per thread, 16 FMAs per chain per loop trip, `iters` trips, on a grid
 * of (SMs x resident blocks) x 256 threads on `stream` (a cudaStream_t, NULL =
 * default), once as warm-up and 5 times timed with CUDA events; *tflops (HOST)
 * receives the best rate in TFLOP/s (2 flops per FMA). Allocates a small output
 * buffer and synchronises: not for use inside a stream capture. Returns
 * SDCEF_ERR_INVALID for another precision, iters < 1 or tflops NULL. */
int sdcef_fma_peak_probe(int precision, int iters, void* stream, double* tflops);

/* Apply the configured preconditioner, built at X = (ne, phi), to the
 * residual-space vector (r_e, r_phi) in physical (unscaled) units:
 * x = P^-1 r with P^-1 from Eq. prec (SDCEF_PREC_EXACT: x = J^-1 r) or
 * Eq. prec_recast (SDCEF_PREC_RECAST; SDCEF_PREC_MG with multigrid block
 * solves), using the precision of the context. Device pointers, [cells] each;
 * mg_cycles ([ncol], may be NULL) receives the V-cycles of each column's
 * multigrid block solves. Enqueued on the context stream. */
int sdcef_precond_apply_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* ne,
                              const double* phi, const double* r_e, const double* r_phi,
                              double* x_e, double* x_phi, int* mg_cycles);

/* Autotuner: times sdcef_solve_batch on this batch with 32, 64, 128 and 256
 * threads per column (one warm-up and `reps` timed solves each, CUDA events on
 * the context stream), keeps the fastest as the context's threads_per_column
 * and returns it in *tpb_out (ms_out, if not NULL, receives the 4 mean times).
 * Synchronises the stream; call it before any stream capture. Not part of the
 * paper (the paper solves one 1D problem at a time). */
int sdcef_autotune(sdcef_ctx* ctx, const sdcef_batch* batch, const sdcef_result* out, int reps,
                   int* tpb_out, float* ms_out);

/* Autotuner for the Krylov storage: times sdcef_solve_batch on this batch with
 * krylov_on_chip 0 and 1 at the context's threads per column (one warm-up and
 * `reps` timed solves each), keeps the faster in the context's parameters and
 * returns it in *on_chip_out (ms_out, if not NULL, receives the 2 mean times,
 * slot first). Synchronises the stream; call it before any stream capture. */
int sdcef_autotune_on_chip(sdcef_ctx* ctx, const sdcef_batch* batch, const sdcef_result* out,
                           int reps, int* on_chip_out, float* ms_out);

/* Provisional charged species of an SDC iteration: the electric-drift part of
 * the provisional rho Y~ that Algorithm 1 hands to the electric solve (the
 * effective ion velocity U_ef,m = U - nu_m kappa_m grad(phi) of Sec. 3.1 with
 * U = 0; advection, diffusion and reactions of the ions are outside this
 * library). One explicit first-order upwind step of length dt per column:
 *   n~_i = n_i - (dt/h) (Phi_{i+1/2} - Phi_{i-1/2}),  Phi = w n_upwind,
 *   w = -nu kappa_ion dphi/dx at the face (second-order one-sided gradient at
 *   the electrodes, which absorb outgoing ions and emit none).
 * Stable for kappa_ion |E| dt / h <= 1. Reads batch->n_ion and the potential
 * phi ([cells]); writes n_ion_out ([n_species][cells], device). */
int sdcef_ion_update_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* phi,
                           double kappa_ion, double* n_ion_out);

/* Provisional charged species of an SDC iteration with the paper's transport
 * (Sec. 3.1, Algorithm 1; SDCEF_ION_GODUNOV): for each species
 *   (I - dt D) n~ = n^n + dt A^{n+1/2} + (dt/2)(D n^n - D n^(k)),
 * A the advection with the effective velocity U_ef,m = U + nu_m kappa_ion E
 * (E = -dphi/dx of phi) by a second-order Godunov (MUSCL) scheme: the face
 * state is the upwind cell value extrapolated to the face and to t^{n+1/2}
 * with its monotonized-central limited difference; electrodes pass outgoing
 * drift only. D: diffusion with D_m = kappa_ion k_B T / (|nu_m| e), no flux
 * through the electrodes. n^(k) = n_prev ([n_species][cells], NULL: n^n, the
 * first SDC iteration, where the correction vanishes). No reactions (the
 * columns carry no chemistry). n^n = batch->n_ion; scratch: [n_species][cells]
 * device doubles; n_ion_out: [n_species][cells] device (may not alias n^n or
 * n_prev). Enqueued on the context stream. */
int sdcef_ion_provisional_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* phi,
                                const double* n_prev, double kappa_ion, double* scratch,
                                double* n_ion_out);

/* Charge flux density through every face (Sec. 4.4, the current of the i-V
 * curves): J_m = nu_m e Gamma_m summed into J+ (positive ions) and J-
 * (negative ions and electrons), J = J+ + J- [A/m^2]; the current through a
 * cross-section S is i = J S. Electrons carry the Scharfetter-Gummel flux of
 * the residual (electrode faces by the context's electron boundary
 * condition); each ion species drifts with U + nu_m kappa_ion E (E =
 * -dphi/dx, upwind cell value) and diffuses with D_m = kappa_ion k_B T /
 * (|nu_m| e) (face mean of T); an electrode passes only outgoing ion drift.
 * ne, phi: the state [cells] (device); ions from batch->n_ion; j_pos, j_neg:
 * [cells + ncol] device outputs, the N + 1 faces of column c at offsets
 * col_off[c] + c .. col_off[c+1] + c (face 0 on the x = 0 electrode).
 * Enqueued on the context stream. Returns SDCEF_ERR_INVALID for NULL arrays
 * or a negative / non-finite kappa_ion. */
int sdcef_current_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* ne,
                        const double* phi, double kappa_ion, double* j_pos, double* j_neg);

/* The electric part of one MISDC time step (Algorithm 1, SDC iterations
 * k = 1..k_max; the paper uses k_max = 4, Table 1): for each k the provisional
 * ions are advanced from batch->n_ion in the field of the previous iterate
 * (phi^n for k = 1) and Eq. nls is solved from the previous iterate (from
 * X^n, or batch->ne_guess / phi_guess, for k = 1). The provisional ions come
 * from sdcef_ion_provisional_batch (params ion_scheme SDCEF_ION_GODUNOV, with
 * the previous iteration's provisional ions as n^(k)) or from
 * sdcef_ion_update_batch (SDCEF_ION_DRIFT_UPWIND). n_ion_work is caller-owned
 * device scratch of 3 n_species x max_cells doubles (Godunov; max_cells
 * of sdcef_create: the library does not read the cell count on the host) or
 * n_species x cells (drift-only). The results of the last iteration are
 * written to out; enqueued on the context stream with no allocation and no
 * synchronisation, so the sweep can be captured in a CUDA graph. */
int sdcef_sdc_sweep(sdcef_ctx* ctx, const sdcef_batch* batch, int k_max, double kappa_ion,
                    double* n_ion_work, const sdcef_result* out);

/* Allocation-free solve. The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc when they solve, for example an
 * application whose device memory is handed out entirely by its own arena
 * allocator, or a time-stepping code that forbids allocation after start-up so
 * that its memory footprint stays fixed. It needs no context: it runs the same
 * solver kernel as sdcef_solve_batch, with its workspace (column slots, work
 * queue, column order) in one file-scope device array of
 * SDCEF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits. It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Arguments: p as for sdcef_create (validated the same way); batch and out as
 * for sdcef_solve_batch (device pointers); max_col_cells bounds the longest
 * column of the batch (cells of a longer column are reported as
 * SDCEF_STATUS_BAD_INPUT); stream is a cudaStream_t (NULL = legacy default).
 * Limits: ncol <= SDCEF_NOALLOC_MAX_COLS and max_col_cells <=
 * SDCEF_NOALLOC_MAX_COL_CELLS, else SDCEF_ERR_CAPACITY with a message; fewer
 * columns run concurrently than with a context (as many slots as fit in the
 * array), so throughput is lower.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so the entry point stays
 * valid after cudaDeviceReset. The first call on a device may load the
 * library's device code there; make that first call before any stream
 * capture. Every call on a device shares the one array and
 * leaves its contents behind (the call itself zeroes the work-queue counter,
 * the only part that must start at zero): calls that overlap on the GPU, on
 * different streams or threads, race and give wrong results. Enqueued on
 * `stream`; does not synchronise. */
#define SDCEF_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
#define SDCEF_NOALLOC_MAX_COLS 65536
#define SDCEF_NOALLOC_MAX_COL_CELLS 4096
int sdcef_solve_batch_noalloc(const sdcef_params* p, const sdcef_batch* batch,
                              const sdcef_result* out, int max_col_cells, void* stream);

/* ---------------------------------------------------------------------------
 * Learned Newton initial guess. Not part of the paper: a small MLP predicts,
 * from stencil and column features of the plain start X^n, the scaled
 * increment to the converged solution; Algorithm 2 then starts from the guess
 * and still decides convergence with its own residual test, so the guess
 * changes only the iteration count, never the accepted root.
 *   features of cell i (BF16, row-major [cells][32]; s_n, s_phi are the
 *   per-column scales of Eq. newton_sc):
 *   0..24: for stencil offsets -2..2 (indices mirrored at the column ends)
 *     n_e^n/s_n, phi^n/s_phi, f_phi/s_n, T/2000 K, E h/s_phi with
 *     E h = -(phi_{k+1} - phi_{k-1})/2;
 *   25..31, the column context: (i + 1/2)/N, log10(s_n / 1 m^-3) - 16,
 *     (V_R - V_L)/1000 V, (log2 N - 10)/2, log10(dt / 1 s) + 5,
 *     asinh(phi_ion,i/s_phi), asinh(E_ion,i L/s_phi), where phi_ion is the
 *     root of the Poisson residual F_phi (Sec. 2) with n_e = 0, electrodes at
 *     0 V and eps_r = 1 (the potential of the ion charge alone) and E_ion,i is
 *     minus the mean of its two face gradients at cell i (0 for N = 1).
 *   network: y = W3 silu(W2 silu(W1 x + b1) + b2) + b3 (32 -> 128 -> 128 -> 2),
 *   BF16 weights and activations on the tensor cores, FP32 accumulation.
 *   parameters: FP32 flat array of SDCEF_MLP_NPARAM values, in order
 *   W1[128][32], b1[128], W2[128][128], b2[128], W3[2][128], b3[2].
 *   training: mean-squared error against y* = ((n* - n^n)/s_n, (phi* - phi^n)/s_phi),
 *   Adam (beta 0.9 / 0.999, eps 1e-8) on the FP32 master parameters.
 * All array arguments are device pointers; calls are enqueued on the stream
 * given to sdcef_mlp_create (set/get_params synchronise it). */
#define SDCEF_MLP_NPARAM 20994
typedef struct sdcef_mlp sdcef_mlp;
/* Allocate parameters, Adam state and activation buffers for up to max_rows cells. */
int sdcef_mlp_create(sdcef_mlp** out, int64_t max_rows, void* stream);
int sdcef_mlp_destroy(sdcef_mlp* mlp);
/* Copy SDCEF_MLP_NPARAM FP32 parameters from HOST memory; resets the Adam state. */
int sdcef_mlp_set_params(sdcef_mlp* mlp, const float* params_host);
/* Copy the FP32 parameters to HOST memory. */
int sdcef_mlp_get_params(sdcef_mlp* mlp, float* params_host);
/* Training checkpoint: the FP32 parameters, the Adam moments m and v (each
 * SDCEF_MLP_NPARAM floats, HOST memory) and the Adam step count. get copies
 * them out (synchronises the stream); set restores them, so that training
 * resumed from a checkpoint continues with the same update as an
 * uninterrupted run. Not part of the paper (the learned guess is not in it). */
int sdcef_mlp_get_state(sdcef_mlp* mlp, float* params_host, float* m_host, float* v_host,
                        int64_t* step);
int sdcef_mlp_set_state(sdcef_mlp* mlp, const float* params_host, const float* m_host,
                        const float* v_host, int64_t step);
/* Features of every cell of the batch into X_bf16 ([cells][32] bfloat16). */
int sdcef_mlp_features(sdcef_mlp* mlp, const sdcef_batch* batch, void* X_bf16);
/* Training targets y* ([cells][2] FP32) from converged (ne_star, phi_star). */
int sdcef_mlp_targets(sdcef_mlp* mlp, const sdcef_batch* batch, const double* ne_star,
                      const double* phi_star, float* targets);
/* Network output Y ([n][2] FP32) for n feature rows (n <= max_rows). */
int sdcef_mlp_forward(sdcef_mlp* mlp, const void* X_bf16, int64_t n, float* Y);
/* Gradient of the mean-squared loss over n rows (no update): grads
 * [SDCEF_MLP_NPARAM] FP32 and loss [1] FP32, both device pointers (may be NULL). */
int sdcef_mlp_grad(sdcef_mlp* mlp, const void* X_bf16, const float* targets, int64_t n,
                   float* grads, float* loss);
/* One Adam step on n rows with learning rate lr; loss [1] FP32 device (may be NULL). */
int sdcef_mlp_train_step(sdcef_mlp* mlp, const void* X_bf16, const float* targets, int64_t n,
                         float lr, float* loss);
/* Newton start for every cell of the batch: features, network, and the
 * start written to ne_guess / phi_guess ([cells] FP64). ncells is the
 * batch's total cell count (<= max_rows). components is a bit set:
 *   SDCEF_GUESS_NE: n_e = n_e^n + s_n y_0 (else n_e^n);
 *   SDCEF_GUESS_PHI: phi = phi^n + s_phi y_1 (else phi^n);
 *   SDCEF_GUESS_PHI_POISSON: phi = the root of the Poisson residual F_phi at
 *     the start's n_e (the potential consistent with the guessed charge;
 *     eps_r = 1, electrodes at V_L, V_R); it takes precedence over
 *     SDCEF_GUESS_PHI. Columns of one cell keep phi^n.
 * Returns SDCEF_ERR_INVALID for components outside 0..7. */
#define SDCEF_GUESS_NE 1
#define SDCEF_GUESS_PHI 2
#define SDCEF_GUESS_PHI_POISSON 4
int sdcef_mlp_guess(sdcef_mlp* mlp, const sdcef_batch* batch, int64_t ncells, int components,
                    double* ne_guess, double* phi_guess);
/* Kernel launches enqueued by the last forward / grad / train_step / guess call. */
int sdcef_mlp_last_launch_count(const sdcef_mlp* mlp);
/* Synchronises the stream and reports whether a tensor-core wait of an earlier
 * forward / grad / train_step / guess call ran out (its kernels bound every
 * wait; the affected rows were written as NaN): SDCEF_ERR_CUDA with a message
 * if so, SDCEF_SUCCESS otherwise. Clears the condition. */
int sdcef_mlp_check(sdcef_mlp* mlp);

/* Failure-path test hook, not an operation of the paper: the number of polls
 * of the main bounded mbarrier waits of this handle's tensor-core kernels
 * (forward, grad, train_step, guess); polls < 0 restores the default (2^22).
 * With polls = 0 every such wait gives up at once, as a wait that ran out would:
 * the kernel sets the error word that sdcef_mlp_check reports, writes NaN for
 * the rows it was computing and skips the rest of its work; its clean-up wait,
 * which lets an issued MMA finish before the tensor memory is freed, keeps the
 * default bound. Takes effect from the next call; no GPU work. */
int sdcef_mlp_set_wait_polls(sdcef_mlp* mlp, int polls);

/* The MLP handle's check word of the bounds-checking build (see
 * sdcef_check_word). */
int sdcef_mlp_check_word(sdcef_mlp* mlp, unsigned* word);

/* Message of the last error on this thread (static storage). */
const char* sdcef_last_error(void);

/* Number of kernel launches the last solve/residual/precond call enqueued. */
int sdcef_last_launch_count(const sdcef_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SDCEF_H */
