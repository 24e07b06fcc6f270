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
#define SDCEF_STATUS_OK 0              /* ||S_F^-1 F||_inf < eps_F (or step < eps_X)  */
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

/* preconditioner (Sec. 3.2) */
#define SDCEF_PREC_EXACT 0   /* Eq. prec with the exact Schur complement:
                                P^-1 = J^-1, applied in 1D as a block-tridiagonal
                                solve on the cell-interleaved (n_i, phi_i) unknowns */
#define SDCEF_PREC_RECAST 1  /* Eq. prec_recast: three tridiagonal solves with the
                                approximate Schur complement S~ = L + I_e dt D_r   */
#define SDCEF_PREC_NONE 2    /* no preconditioner (diagnostics)                    */

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
  int precision;      /* SDCEF_FP64 | SDCEF_MIXED                                     */
  int precond;        /* SDCEF_PREC_EXACT | SDCEF_PREC_RECAST | SDCEF_PREC_NONE       */
  int bc_electron;    /* SDCEF_BC_ABSORBING | SDCEF_BC_ZERO_GRADIENT                  */
  int threads_per_column; /* 0 = chosen per column length; else 32, 64, 128 or 256    */
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
} sdcef_result;

/* Fill p with the defaults: eps_F 1e-10, eps_X 0, gamma 1e-4 (Table 1),
 * mobility 0.4 (Sec. 2.2), ls_alpha 1e-4, eps_r 1, restart 8, 50 Newton
 * steps, 200 Krylov iterations per step, 20 halvings, FP64, exact Schur
 * preconditioner, absorbing electrodes, automatic threads per column. */
void sdcef_default_params(sdcef_params* p);

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

/* Evaluate the residual F(X) of Eq. nls at X = (ne, phi) for every column
 * (device pointers, [cells] each). Enqueued on the context stream. */
int sdcef_residual_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* ne,
                         const double* phi, double* F_e, double* F_phi);

/* Apply the configured preconditioner, built at X = (ne, phi), to the
 * residual-space vector (r_e, r_phi) in physical (unscaled) units:
 * x = P^-1 r with P^-1 from Eq. prec (SDCEF_PREC_EXACT: x = J^-1 r) or
 * Eq. prec_recast (SDCEF_PREC_RECAST), using the precision of the context.
 * Device pointers, [cells] each. Enqueued on the context stream. */
int sdcef_precond_apply_batch(sdcef_ctx* ctx, const sdcef_batch* batch, const double* ne,
                              const double* phi, const double* r_e, const double* r_phi,
                              double* x_e, double* x_phi);

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
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture. Every call on a device shares the one array and
 * leaves its contents behind (the call itself zeroes the work-queue counter,
 * the only part that must start at zero): calls that overlap on the GPU, on
 * different streams or threads, race and give wrong results. Enqueued on
 * `stream`; does not synchronise. */
#define SDCEF_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
#define SDCEF_NOALLOC_MAX_COLS 65536
#define SDCEF_NOALLOC_MAX_COL_CELLS 4096
int sdcef_solve_batch_noalloc(const sdcef_params* p, const sdcef_batch* batch,
                              const sdcef_result* out, int max_col_cells, void* stream);

/* Message of the last error on this thread (static storage). */
const char* sdcef_last_error(void);

/* Number of kernel launches the last solve/residual/precond call enqueued. */
int sdcef_last_launch_count(const sdcef_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SDCEF_H */
