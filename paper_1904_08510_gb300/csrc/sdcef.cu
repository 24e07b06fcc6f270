// C ABI of the batched JFNK solver (host side): argument validation,
// workspace ownership, launch configuration and the host-buffer entry point.
// The kernels are in solver.cuh / kern_inst.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sdcef.h"
#include "fields.cuh"
#include "solver.cuh"

using namespace sdcef_impl;

namespace {

// NVTX range over an entry point (host side; visible to profilers that
// collect NVTX, free otherwise, and harmless inside a stream capture).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
thread_local std::string g_err;
int set_err(int code, const std::string& m) {
  g_err = m;
  return code;
}
}  // namespace

// ============================================================================
// Host side
// ============================================================================
struct sdcef_ctx {
  sdcef_params p;
  int64_t max_cols, max_cells;
  int max_col_cells;
  int m_cap;
  cudaStream_t stream;
  int device, sms;
  char* ws;
  size_t ws_bytes;
  int nslots;
  int* queue;     // 4 ints: [0] work-queue counter, [3] check word of the bounds-checking build
  int* order;     // max_cols ints
  int launches;
  // host-call staging
  char* stage;
  size_t stage_bytes;
  // double-buffered host calls: copy streams (host to device, device to host)
  // and, per staging half, inputs staged / solved / half free again
  cudaStream_t cs[2];
  cudaEvent_t ev_in[2], ev_done[2], ev_free[2];
  bool pipe;
  // electron transport tables (mu then D, [nc][nx] each), device
  double* tab;
  int tab_nc, tab_nx;
  double tab_en_max, tab_T_in, tab_T_max;
};

namespace {

int tpb_for(const sdcef_params& p, int max_col_cells) {
  if (p.precond == SDCEF_PREC_MG) return kMgTPB;   // the multigrid kernel's fixed width
  if (p.transport == SDCEF_TRANSPORT_TABLE) return kMgTPB;   // the table kernel's
  if (p.threads_per_column) return p.threads_per_column;
  (void)max_col_cells;
  return 128;
}


int check_params(const sdcef_params* p, int m_cap) {
  if (!p) return set_err(SDCEF_ERR_INVALID, "params is NULL");
  if (!(p->eps_F > 0.0) || !(p->gamma > 0.0 && p->gamma < 1.0) || !(p->mobility > 0.0) ||
      !(p->ls_alpha >= 0.0 && p->ls_alpha < 1.0) || !(p->eps_r > 0.0) || !(p->eps_X >= 0.0) ||
      !(p->eps_E >= 0.0) || !std::isfinite(p->eps_E) ||
      !(p->stall_ratio >= 0.0 && p->stall_ratio < 1.0))
    return set_err(SDCEF_ERR_INVALID,
                   "params: eps_F, eps_X, eps_E, stall_ratio, gamma, mobility, ls_alpha, eps_r out of range");
  if (p->krylov_on_chip != 0 && p->krylov_on_chip != 1)
    return set_err(SDCEF_ERR_INVALID, "params: krylov_on_chip must be 0 or 1");
  if (p->sdc_poisson_start != 0 && p->sdc_poisson_start != 1)
    return set_err(SDCEF_ERR_INVALID, "params: sdc_poisson_start must be 0 or 1");
  if (p->restart_m < 1 || p->restart_m > SDCEF_MAX_RESTART || (m_cap > 0 && p->restart_m > m_cap))
    return set_err(SDCEF_ERR_INVALID, "params: restart_m out of range");
  if (p->max_newton < 0 || p->max_krylov < 1 || p->max_linesearch < 0 || p->guess_newton_cap < 0 ||
      !(p->guess_reject_ratio >= 0.0) || !(p->guess_progress >= 0.0 && p->guess_progress <= 1.0))
    return set_err(SDCEF_ERR_INVALID, "params: iteration caps out of range");
  if (p->precision != SDCEF_FP64 && p->precision != SDCEF_MIXED && p->precision != SDCEF_MIXED_DF)
    return set_err(SDCEF_ERR_INVALID, "params: precision");
  if (p->precond != SDCEF_PREC_EXACT && p->precond != SDCEF_PREC_RECAST &&
      p->precond != SDCEF_PREC_NONE && p->precond != SDCEF_PREC_MG)
    return set_err(SDCEF_ERR_INVALID, "params: precond");
  if (p->precond == SDCEF_PREC_MG) {
    if (p->precision != SDCEF_FP64)
      return set_err(SDCEF_ERR_INVALID, "params: the multigrid preconditioner needs precision FP64");
    if (!std::isfinite(p->mg_gamma_A) || !std::isfinite(p->mg_gamma_S) || p->mg_gamma_A >= 1.0 ||
        p->mg_gamma_S >= 1.0)
      return set_err(SDCEF_ERR_INVALID, "params: mg_gamma_A / mg_gamma_S");
    if (p->mg_max_cycles < 1 || p->mg_max_cycles > 1000)
      return set_err(SDCEF_ERR_INVALID, "params: mg_max_cycles");
    if (p->mg_transfer != SDCEF_MG_OPERATOR && p->mg_transfer != SDCEF_MG_LINEAR)
      return set_err(SDCEF_ERR_INVALID, "params: mg_transfer");
  }
  if (p->ion_scheme != SDCEF_ION_GODUNOV && p->ion_scheme != SDCEF_ION_DRIFT_UPWIND)
    return set_err(SDCEF_ERR_INVALID, "params: ion_scheme");
  if (p->transport != SDCEF_TRANSPORT_CONSTANT && p->transport != SDCEF_TRANSPORT_TABLE)
    return set_err(SDCEF_ERR_INVALID, "params: transport");
  if (p->transport == SDCEF_TRANSPORT_TABLE) {
    if (p->precision != SDCEF_FP64)
      return set_err(SDCEF_ERR_INVALID, "params: transport tables need precision FP64");
    if (p->precond == SDCEF_PREC_MG)
      return set_err(SDCEF_ERR_INVALID, "params: transport tables with the multigrid preconditioner");
    if (!(p->gas_molar_mass > 0.0) || !std::isfinite(p->gas_molar_mass))
      return set_err(SDCEF_ERR_INVALID, "params: gas_molar_mass");
  }
  if (p->bc_electron != SDCEF_BC_ABSORBING && p->bc_electron != SDCEF_BC_ZERO_GRADIENT)
    return set_err(SDCEF_ERR_INVALID, "params: bc_electron");
  int t = p->threads_per_column;
  if (t != 0 && t != 32 && t != 64 && t != 128 && t != 256)
    return set_err(SDCEF_ERR_INVALID, "params: threads_per_column must be 0, 32, 64, 128 or 256");
  return SDCEF_SUCCESS;
}

int validate_batch(const sdcef_ctx* ctx, const sdcef_batch* b, bool need_solve_inputs) {
  if (!b) return set_err(SDCEF_ERR_INVALID, "batch is NULL");
  if (b->ncol < 0) return set_err(SDCEF_ERR_INVALID, "batch: ncol < 0");
  if (b->ncol > ctx->max_cols) return set_err(SDCEF_ERR_CAPACITY, "batch: ncol exceeds max_cols");
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!b->col_off || !b->length || !b->dt || !b->v_left || !b->v_right || !b->T)
    return set_err(SDCEF_ERR_INVALID, "batch: required pointer is NULL");
  if (need_solve_inputs && (!b->ne_old || !b->phi_old))
    return set_err(SDCEF_ERR_INVALID, "batch: ne_old / phi_old is NULL");
  if (b->n_species < 0 || b->n_species > SDCEF_MAX_SPECIES)
    return set_err(SDCEF_ERR_INVALID, "batch: n_species out of range");
  if (b->n_species > 0 && (!b->valence || !b->n_ion))
    return set_err(SDCEF_ERR_INVALID, "batch: valence / n_ion is NULL");
  return SDCEF_SUCCESS;
}

// Fill kernel args shared by all modes.
unsigned* check_word(sdcef_ctx* ctx) { return reinterpret_cast<unsigned*>(ctx->queue + 3); }

KArgs base_args(sdcef_ctx* ctx, const sdcef_batch* b, int tpb) {
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.chk = check_word(ctx);
  a.ncol = b->ncol;
  a.col_off = b->col_off;
  a.length = b->length;
  a.dt = b->dt;
  a.vl = b->v_left;
  a.vr = b->v_right;
  a.ne_old = b->ne_old;
  a.phi_old = b->phi_old;
  a.nsp = b->n_species;
  for (int s = 0; s < b->n_species; ++s) a.val[s] = b->valence[s];
  a.n_ion = b->n_ion;
  a.T = b->T;
  a.u = b->u_adv;
  a.ire = b->i_re;
  a.ne_g = b->ne_guess;
  a.phi_g = b->phi_guess;
  a.ws = ctx->ws;
  const int kmax = (ctx->max_col_cells + tpb - 1) / tpb;
  a.kmax = kmax;
  a.PL = (size_t)kmax * tpb;
  a.slot_bytes = slot_bytes_prec(ctx->p.precision, a.PL, ctx->m_cap, tpb, ctx->p.precond);
  a.max_col_cells = ctx->max_col_cells;
  a.queue = ctx->queue;
  const sdcef_params& p = ctx->p;
  a.p.eps_F = p.eps_F;
  a.p.eps_X = p.eps_X;
  a.p.eps_E = p.eps_E;
  a.p.stall = p.stall_ratio > 0.0 ? p.stall_ratio : 2.0;
  a.p.gamma = p.gamma;
  a.p.mu = p.mobility;
  a.p.ls_alpha = p.ls_alpha;
  a.p.kap = kEps0 * p.eps_r / kQe;
  a.p.m = ctx->m_cap;   // plane layout uses the capacity; iteration uses restart_m
  a.p.max_newton = p.max_newton;
  a.p.max_krylov = p.max_krylov;
  a.p.max_ls = p.max_linesearch;
  a.p.bc = p.bc_electron;
  a.p.precond = p.precond;
  a.p.guess_cap = p.guess_newton_cap;
  a.p.guess_ratio = p.guess_reject_ratio;
  a.p.guess_prog = p.guess_progress;
  a.p.mg_gA = p.mg_gamma_A;
  a.p.mg_gS = p.mg_gamma_S;
  a.p.mg_maxc = p.mg_max_cycles;
  a.p.mg_transfer = p.mg_transfer;
  a.p.transport = p.transport;
  a.rho = b->rho;
  a.tt.tab = ctx->tab;
  a.tt.nc = ctx->tab_nc;
  a.tt.nx = ctx->tab_nx;
  a.tt.en_max_td = ctx->tab_en_max;
  a.tt.T_in = ctx->tab_T_in;
  a.tt.inv_dT = ctx->tab_T_max > ctx->tab_T_in ? 1.0 / (ctx->tab_T_max - ctx->tab_T_in) : 0.0;
  a.tt.gas_W = p.gas_molar_mass;
  return a;
}

int run(sdcef_ctx* ctx, KArgs& a, int tpb) {
  const int prec = ctx->p.precision;
  if (ctx->p.transport == SDCEF_TRANSPORT_TABLE && (!ctx->tab || !a.rho))
    return set_err(SDCEF_ERR_INVALID, "transport tables: no table set, or batch->rho is NULL");
  // restart length used by the iteration (planes are laid out for m_cap)
  const int m_run = ctx->p.restart_m;
  a.p.m = m_run;
  size_t smem = smem_bytes_prec(prec, tpb, m_run);
  // slot layout must use the same m as the device code: recompute with m_run
  a.slot_bytes = slot_bytes_prec(prec, a.PL, m_run, tpb, ctx->p.precond);
  int per_sm = occupancy_prec(prec, tpb, smem, ctx->p.precond, ctx->p.transport);
  if (ctx->p.krylov_on_chip)
    smem = krylov_arena(prec, tpb, smem, per_sm, ctx->p.precond, ctx->p.transport, &a);
  int64_t slots_fit = (int64_t)(ctx->ws_bytes / a.slot_bytes);
  int grid = (int)std::min<int64_t>({(int64_t)per_sm * ctx->sms, a.ncol, slots_fit});
  if (grid < 1) return set_err(SDCEF_ERR_CAPACITY, "workspace too small for one column slot");
  cudaError_t e = cudaMemsetAsync(ctx->queue, 0, sizeof(int), ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  ctx->launches = 0;
  if (a.mode == MODE_SOLVE && a.ncol > 1) {
    int shift = 4;
    while ((ctx->max_col_cells >> shift) + 1 > 4096) ++shift;
    const int nbins = (ctx->max_col_cells >> shift) + 1;
    e = launch_order(a.col_off, a.ncol, nbins, shift, ctx->order, ctx->stream);
    if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
    a.order = ctx->order;
    ++ctx->launches;
  }
  e = launch_prec(prec, tpb, a, grid, smem, ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  ++ctx->launches;
  return SDCEF_SUCCESS;
}

}  // namespace

// Shared with the allocation-free entry point (noalloc.cu).
namespace sdcef_impl {
int report_error(int code, const char* msg) { return set_err(code, msg); }
// mlp.cu: the potential of a given electron density (root of F_phi) per column
cudaError_t launch_poisson_start(const sdcef_batch* b, const double* ne, const double* n_ion,
                                 double kappa, double* phi_out, cudaStream_t st);
int validate_params(const sdcef_params* p) { return check_params(p, 0); }
}  // namespace sdcef_impl

extern "C" {

void sdcef_default_params(sdcef_params* p) {
  if (!p) return;
  p->eps_F = 1e-10;
  p->eps_X = 0.0;
  p->eps_E = 5e-10;
  p->stall_ratio = 0.9;
  p->krylov_on_chip = 0;
  p->gamma = 1e-4;
  p->mobility = 0.4;
  p->ls_alpha = 1e-4;
  p->eps_r = 1.0;
  p->restart_m = 8;
  p->max_newton = 50;
  p->max_krylov = 200;
  p->max_linesearch = 20;
  p->precision = SDCEF_FP64;
  p->precond = SDCEF_PREC_EXACT;
  p->mg_gamma_A = 1e-4;
  p->mg_gamma_S = 1e-4;
  p->mg_max_cycles = 50;
  p->mg_transfer = SDCEF_MG_OPERATOR;
  p->ion_scheme = SDCEF_ION_GODUNOV;
  p->transport = SDCEF_TRANSPORT_CONSTANT;
  p->gas_molar_mass = 0.028;
  p->bc_electron = SDCEF_BC_ABSORBING;
  p->threads_per_column = 0;
  p->guess_newton_cap = 8;
  p->guess_reject_ratio = 30.0;
  p->guess_progress = 0.3;
  p->sdc_poisson_start = 1;
}

const char* sdcef_last_error(void) { return g_err.c_str(); }

int sdcef_create(sdcef_ctx** out, const sdcef_params* p, int64_t max_cols, int64_t max_cells,
                 int max_col_cells, void* stream) {
  if (!out) return set_err(SDCEF_ERR_INVALID, "out is NULL");
  int rc = check_params(p, 0);
  if (rc) return rc;
  if (max_cols < 1 || max_cells < 2 || max_col_cells < 2 || max_col_cells > (1 << 20) ||
      (int64_t)max_col_cells > max_cells)
    return set_err(SDCEF_ERR_INVALID, "create: sizes out of range");
  sdcef_ctx* c = new sdcef_ctx();
  memset(c, 0, sizeof(*c));
  c->p = *p;
  c->max_cols = max_cols;
  c->max_cells = max_cells;
  c->max_col_cells = max_col_cells;
  c->m_cap = p->restart_m;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  }
  // workspace: enough slots for the widest configuration at 2 CTAs per SM
  // (FP64 planes, smallest thread count gives the largest per-slot size)
  size_t best = 0;
  for (int tpb : {32, 64, 128, 256}) {
    const size_t PL = (size_t)((max_col_cells + tpb - 1) / tpb) * tpb;
    best = std::max(best, slot_bytes_prec(SDCEF_FP64, PL, c->m_cap, tpb, p->precond));
  }
  int64_t nslots = std::min<int64_t>((int64_t)c->sms * 4, max_cols);
  c->nslots = (int)nslots;
  c->ws_bytes = best * (size_t)nslots;
  e = cudaMalloc((void**)&c->ws, c->ws_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->queue, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->queue, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->order, sizeof(int) * (size_t)max_cols);
  if (e != cudaSuccess) {
    if (c->ws) cudaFree(c->ws);
    if (c->queue) cudaFree(c->queue);
    if (c->order) cudaFree(c->order);
    delete c;
    return set_err(SDCEF_ERR_NOMEM, cudaGetErrorString(e));
  }
  *out = c;
  return SDCEF_SUCCESS;
}

int sdcef_set_params(sdcef_ctx* ctx, const sdcef_params* p) {
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = check_params(p, ctx->m_cap);
  if (rc) return rc;
  ctx->p = *p;
  return SDCEF_SUCCESS;
}

int sdcef_destroy(sdcef_ctx* ctx) {
  if (!ctx) return SDCEF_SUCCESS;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->ws);
  cudaFree(ctx->queue);
  cudaFree(ctx->order);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->tab) cudaFree(ctx->tab);
  if (ctx->pipe) {
    for (int i = 0; i < 2; ++i) {
      cudaStreamSynchronize(ctx->cs[i]);
      cudaStreamDestroy(ctx->cs[i]);
      cudaEventDestroy(ctx->ev_in[i]);
      cudaEventDestroy(ctx->ev_done[i]);
      cudaEventDestroy(ctx->ev_free[i]);
    }
  }
  delete ctx;
  return SDCEF_SUCCESS;
}

int sdcef_set_transport_table(sdcef_ctx* ctx, int nc, int nx, double en_max_td, double T_in,
                              double T_max, const double* mu, const double* D) {
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  if (nc < 2 || nx < 2 || nc > 4096 || nx > 65536 || !(en_max_td > 0.0) || !std::isfinite(en_max_td) ||
      !std::isfinite(T_in) || !std::isfinite(T_max) || !(T_max > T_in) || !mu || !D)
    return set_err(SDCEF_ERR_INVALID, "transport table: bad arguments");
  const size_t n = (size_t)nc * nx;
  for (size_t i = 0; i < n; ++i)
    if (!(mu[i] > 0.0) || !(D[i] > 0.0) || !std::isfinite(mu[i]) || !std::isfinite(D[i]))
      return set_err(SDCEF_ERR_INVALID, "transport table: entries must be finite and positive");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);   // no solve may still read the old table
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  if (ctx->tab) cudaFree(ctx->tab);
  ctx->tab = nullptr;
  e = cudaMalloc((void**)&ctx->tab, 2 * n * sizeof(double));
  if (e != cudaSuccess) return set_err(SDCEF_ERR_NOMEM, cudaGetErrorString(e));
  e = cudaMemcpy(ctx->tab, mu, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->tab + n, D, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  ctx->tab_nc = nc;
  ctx->tab_nx = nx;
  ctx->tab_en_max = en_max_td;
  ctx->tab_T_in = T_in;
  ctx->tab_T_max = T_max;
  return SDCEF_SUCCESS;
}

int sdcef_last_launch_count(const sdcef_ctx* ctx) { return ctx ? ctx->launches : 0; }

int sdcef_checks_compiled(void) {
#ifdef SDCEF_CHECKS
  return 1;
#else
  return 0;
#endif
}

int sdcef_check_word(sdcef_ctx* ctx, unsigned* word) {
  if (!ctx || !word) return set_err(SDCEF_ERR_INVALID, "check_word: NULL argument");
  unsigned w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, check_word(ctx), sizeof(unsigned), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(check_word(ctx), 0, sizeof(unsigned), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  *word = w;
  return SDCEF_SUCCESS;
}

int sdcef_solve_batch(sdcef_ctx* ctx, const sdcef_batch* b, const sdcef_result* out) {
  Range range_("sdcef_solve_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, true);
  if (rc) return rc;
  if (b->ncol == 0) { ctx->launches = 0; return SDCEF_SUCCESS; }
  if (!out || !out->ne_out || !out->phi_out) return set_err(SDCEF_ERR_INVALID, "result: ne_out / phi_out is NULL");
  const int tpb = tpb_for(ctx->p, ctx->max_col_cells);
  KArgs a = base_args(ctx, b, tpb);
  a.mode = MODE_SOLVE;
  a.ne_out = out->ne_out;
  a.phi_out = out->phi_out;
  a.status = out->status;
  a.newton_it = out->newton_it;
  a.krylov_it = out->krylov_it;
  a.res_evals = out->res_evals;
  a.mg_cycles = out->mg_cycles;
  a.final_res = out->final_res;
  return run(ctx, a, tpb);
}

int sdcef_autotune(sdcef_ctx* ctx, const sdcef_batch* b, const sdcef_result* out, int reps,
                   int* tpb_out, float* ms_out) {
  Range range_("sdcef_autotune");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  if (reps < 1 || reps > 100) return set_err(SDCEF_ERR_INVALID, "autotune: reps out of range");
  const int cands[4] = {32, 64, 128, 256};
  const sdcef_params saved = ctx->p;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  int best = 0;
  float best_ms = 0.0f;
  int rc = SDCEF_SUCCESS;
  for (int ci = 0; ci < 4 && rc == SDCEF_SUCCESS; ++ci) {
    ctx->p.threads_per_column = cands[ci];
    rc = sdcef_solve_batch(ctx, b, out);   // warm-up (also loads the kernel)
    if (rc) break;
    float tot = 0.0f;
    for (int r = 0; r < reps && rc == SDCEF_SUCCESS; ++r) {
      e = cudaEventRecord(e0, ctx->stream);
      if (e == cudaSuccess) rc = sdcef_solve_batch(ctx, b, out);
      if (e == cudaSuccess && rc == SDCEF_SUCCESS) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess && rc == SDCEF_SUCCESS) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess && rc == SDCEF_SUCCESS) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
      tot += ms;
    }
    if (rc == SDCEF_SUCCESS) {
      const float ms = tot / reps;
      if (ms_out) ms_out[ci] = ms;
      if (best == 0 || ms < best_ms) { best = cands[ci]; best_ms = ms; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->p = saved;
  if (rc) return rc;
  ctx->p.threads_per_column = best;
  if (tpb_out) *tpb_out = best;
  return SDCEF_SUCCESS;
}

int sdcef_autotune_on_chip(sdcef_ctx* ctx, const sdcef_batch* b, const sdcef_result* out,
                           int reps, int* on_chip_out, float* ms_out) {
  Range range_("sdcef_autotune_on_chip");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  if (reps < 1 || reps > 100) return set_err(SDCEF_ERR_INVALID, "autotune: reps out of range");
  const sdcef_params saved = ctx->p;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  float t[2] = {0.0f, 0.0f};
  int rc = SDCEF_SUCCESS;
  for (int oc = 0; oc < 2 && rc == SDCEF_SUCCESS; ++oc) {
    ctx->p.krylov_on_chip = oc;
    rc = sdcef_solve_batch(ctx, b, out);   // warm-up
    for (int r = 0; r < reps && rc == SDCEF_SUCCESS; ++r) {
      e = cudaEventRecord(e0, ctx->stream);
      if (e == cudaSuccess) rc = sdcef_solve_batch(ctx, b, out);
      if (e == cudaSuccess && rc == SDCEF_SUCCESS) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess && rc == SDCEF_SUCCESS) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess && rc == SDCEF_SUCCESS) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
      t[oc] += ms / reps;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->p = saved;
  if (rc) return rc;
  ctx->p.krylov_on_chip = t[1] < t[0] ? 1 : 0;
  if (on_chip_out) *on_chip_out = ctx->p.krylov_on_chip;
  if (ms_out) { ms_out[0] = t[0]; ms_out[1] = t[1]; }
  return SDCEF_SUCCESS;
}

int sdcef_bernoulli_batch(sdcef_ctx* ctx, const double* x, double* b, double* db, int64_t n) {
  Range range_("sdcef_bernoulli_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  if (n < 0 || (n > 0 && (!x || !b || !db))) return set_err(SDCEF_ERR_INVALID, "bernoulli: bad arguments");
  if (n == 0) return SDCEF_SUCCESS;
  cudaError_t e = launch_bernoulli(x, b, db, n, ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  return SDCEF_SUCCESS;
}

int sdcef_ion_update_batch(sdcef_ctx* ctx, const sdcef_batch* b, const double* phi,
                           double kappa_ion, double* n_ion_out) {
  Range range_("sdcef_ion_update_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, false);
  if (rc) return rc;
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!phi || !n_ion_out || !(kappa_ion >= 0.0)) return set_err(SDCEF_ERR_INVALID, "ion_update: bad arguments");
  if (b->n_species == 0) return SDCEF_SUCCESS;
  IonArgs a;
  memset(&a, 0, sizeof(a));
  a.ncol = b->ncol;
  a.col_off = b->col_off;
  a.length = b->length;
  a.dt = b->dt;
  a.vl = b->v_left;
  a.vr = b->v_right;
  a.phi = phi;
  a.n_in = b->n_ion;
  a.n_out = n_ion_out;
  a.nsp = b->n_species;
  for (int s = 0; s < b->n_species; ++s) a.val[s] = b->valence[s];
  a.kappa = kappa_ion;
  a.chk = check_word(ctx);
  cudaError_t e = launch_ion_update(a, ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  return SDCEF_SUCCESS;
}

int sdcef_ion_provisional_batch(sdcef_ctx* ctx, const sdcef_batch* b, const double* phi,
                                const double* n_prev, double kappa_ion, double* scratch,
                                double* n_ion_out) {
  Range range_("sdcef_ion_provisional_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, false);
  if (rc) return rc;
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!phi || !n_ion_out || !scratch || !(kappa_ion >= 0.0) || !std::isfinite(kappa_ion))
    return set_err(SDCEF_ERR_INVALID, "ion_provisional: bad arguments");
  if (b->n_species == 0) return SDCEF_SUCCESS;
  if (n_ion_out == b->n_ion || (n_prev && n_ion_out == n_prev))
    return set_err(SDCEF_ERR_INVALID, "ion_provisional: n_ion_out aliases an input");
  if (b->ncol > 0x7fffffff) return set_err(SDCEF_ERR_INVALID, "ion_provisional: too many columns");
  IonProvArgs a;
  memset(&a, 0, sizeof(a));
  a.ncol = b->ncol;
  a.col_off = b->col_off;
  a.length = b->length;
  a.dt = b->dt;
  a.vl = b->v_left;
  a.vr = b->v_right;
  a.T = b->T;
  a.u = b->u_adv;
  a.phi = phi;
  a.n0 = b->n_ion;
  a.nk = n_prev;
  a.n_out = n_ion_out;
  a.scratch = scratch;
  a.nsp = b->n_species;
  for (int s = 0; s < b->n_species; ++s) a.val[s] = b->valence[s];
  a.kappa = kappa_ion;
  a.chk = check_word(ctx);
  cudaError_t e = launch_ion_provisional(a, ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  return SDCEF_SUCCESS;
}

int sdcef_current_batch(sdcef_ctx* ctx, const sdcef_batch* b, const double* ne,
                        const double* phi, double kappa_ion, double* j_pos, double* j_neg) {
  Range range_("sdcef_current_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, false);
  if (rc) return rc;
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!ne || !phi || !j_pos || !j_neg || !(kappa_ion >= 0.0) || !std::isfinite(kappa_ion))
    return set_err(SDCEF_ERR_INVALID, "current: bad arguments");
  if (b->ncol > 0x7fffffff) return set_err(SDCEF_ERR_INVALID, "current: too many columns");
  CurrentArgs a;
  memset(&a, 0, sizeof(a));
  a.ncol = b->ncol;
  a.col_off = b->col_off;
  a.length = b->length;
  a.vl = b->v_left;
  a.vr = b->v_right;
  a.T = b->T;
  a.u = b->u_adv;
  a.ne = ne;
  a.phi = phi;
  a.n_ion = b->n_ion;
  a.jp = j_pos;
  a.jn = j_neg;
  a.nsp = b->n_species;
  for (int s = 0; s < b->n_species; ++s) a.val[s] = b->valence[s];
  a.kappa = kappa_ion;
  a.chk = check_word(ctx);
  a.mu = ctx->p.mobility;
  a.bc = ctx->p.bc_electron;
  if (ctx->p.transport == SDCEF_TRANSPORT_TABLE) {
    if (!ctx->tab || !b->rho)
      return set_err(SDCEF_ERR_INVALID, "current: transport tables need a table and batch->rho");
    a.tab = ctx->tab;
    a.tnc = ctx->tab_nc;
    a.tnx = ctx->tab_nx;
    a.ten_max_td = ctx->tab_en_max;
    a.tT_in = ctx->tab_T_in;
    a.tinv_dT = 1.0 / (ctx->tab_T_max - ctx->tab_T_in);
    a.tgas_W = ctx->p.gas_molar_mass;
    a.rho = b->rho;
  }
  cudaError_t e = launch_current(a, ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  ctx->launches = 1;
  return SDCEF_SUCCESS;
}

int sdcef_sdc_sweep(sdcef_ctx* ctx, const sdcef_batch* b, int k_max, double kappa_ion,
                    double* n_ion_work, const sdcef_result* out) {
  Range range_("sdcef_sdc_sweep");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, true);
  if (rc) return rc;
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (k_max < 1 || k_max > 64 || !n_ion_work || !(kappa_ion >= 0.0))
    return set_err(SDCEF_ERR_INVALID, "sdc_sweep: bad arguments");
  if (!out || !out->ne_out || !out->phi_out) return set_err(SDCEF_ERR_INVALID, "result: ne_out / phi_out is NULL");
  int launches = 0;
  const bool godunov = ctx->p.ion_scheme == SDCEF_ION_GODUNOV;
  // buffer stride from the context capacity: the cell count lives on the device
  const size_t plane = (size_t)b->n_species * (size_t)ctx->max_cells;
  for (int k = 0; k < k_max; ++k) {
    Range it_("sdc iteration");
    const double* phi_field = (k == 0) ? b->phi_old : out->phi_out;
    // Godunov: provisional ions ping-pong between the first two thirds of the
    // work buffer (the previous iteration's are n^(k)); the Thomas scratch follows
    double* prov = godunov ? n_ion_work + (size_t)(k & 1) * plane : n_ion_work;
    if (godunov)
      rc = sdcef_ion_provisional_batch(ctx, b, phi_field,
                                       k == 0 ? nullptr : n_ion_work + (size_t)((k - 1) & 1) * plane,
                                       kappa_ion, n_ion_work + 2 * plane, prov);
    else
      rc = sdcef_ion_update_batch(ctx, b, phi_field, kappa_ion, prov);
    if (rc) return rc;
    sdcef_batch bk = *b;
    bk.n_ion = b->n_species > 0 ? prov : b->n_ion;
    int extra = 0;
    if (k > 0) {
      bk.ne_guess = out->ne_out;
      bk.phi_guess = out->phi_out;
      if (ctx->p.sdc_poisson_start) {
        // the previous iterate's potential is that of its own charge: re-solve
        // F_phi = 0 for the new provisional ions (in place: it reads n_e only)
        cudaError_t e = sdcef_impl::launch_poisson_start(&bk, out->ne_out, bk.n_ion,
                                                         kEps0 * ctx->p.eps_r / kQe,
                                                         out->phi_out, ctx->stream);
        if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
        extra = 1;
      }
    }
    rc = sdcef_solve_batch(ctx, &bk, out);
    if (rc) return rc;
    launches += ctx->launches + (b->n_species > 0 ? 1 : 0) + extra;
  }
  ctx->launches = launches;
  return SDCEF_SUCCESS;
}

int sdcef_residual_batch(sdcef_ctx* ctx, const sdcef_batch* b, const double* ne, const double* phi,
                         double* F_e, double* F_phi) {
  Range range_("sdcef_residual_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, false);
  if (rc) return rc;
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!ne || !phi || !F_e || !F_phi) return set_err(SDCEF_ERR_INVALID, "residual: NULL array");
  const int tpb = tpb_for(ctx->p, ctx->max_col_cells);
  KArgs a = base_args(ctx, b, tpb);
  // set-up reads ne_old / phi_old; point them at X when absent
  if (!a.ne_old) a.ne_old = ne;
  if (!a.phi_old) a.phi_old = phi;
  a.mode = MODE_RESIDUAL;
  a.x_ne = ne;
  a.x_phi = phi;
  a.o1 = F_e;
  a.o2 = F_phi;
  return run(ctx, a, tpb);
}

int sdcef_precond_apply_batch(sdcef_ctx* ctx, const sdcef_batch* b, const double* ne,
                              const double* phi, const double* r_e, const double* r_phi,
                              double* x_e, double* x_phi, int* mg_cycles) {
  Range range_("sdcef_precond_apply_batch");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = validate_batch(ctx, b, true);
  if (rc) return rc;
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!ne || !phi || !r_e || !r_phi || !x_e || !x_phi)
    return set_err(SDCEF_ERR_INVALID, "precond: NULL array");
  const int tpb = tpb_for(ctx->p, ctx->max_col_cells);
  KArgs a = base_args(ctx, b, tpb);
  a.mode = MODE_PRECOND;
  a.x_ne = ne;
  a.x_phi = phi;
  a.r_e = r_e;
  a.r_phi = r_phi;
  a.o1 = x_e;
  a.o2 = x_phi;
  a.mg_cycles = mg_cycles;
  return run(ctx, a, tpb);
}

}  // extern "C"

namespace {

// Layout of one host batch in a device staging area: inputs, then results
// (byte offsets, each 256-byte aligned).
struct Stage {
  size_t off, len, dt, vl, vr, ne, ph, ion, T, u, ir, ng, pg, neo, pho, st, nt, kt, re, fr, mg;
  size_t need;
};

Stage stage_layout(const sdcef_batch* hb) {
  Stage L;
  size_t need = 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t ncol = hb->ncol, cells = hb->col_off[ncol];
  const size_t c8 = (size_t)cells * 8, n8 = (size_t)ncol * 8, n4 = (size_t)ncol * 4;
  const int nsp = hb->n_species;
  L.off = need; need += al((size_t)(ncol + 1) * 8);
  L.len = need; need += al(n8);
  L.dt = need; need += al(n8);
  L.vl = need; need += al(n8);
  L.vr = need; need += al(n8);
  L.ne = need; need += al(c8);
  L.ph = need; need += al(c8);
  L.ion = need; need += al(c8 * (size_t)std::max(nsp, 1));
  L.T = need; need += al(c8);
  L.u = need; if (hb->u_adv) need += al(c8);
  L.ir = need; if (hb->i_re) need += al(c8);
  L.ng = need; if (hb->ne_guess) need += al(c8);
  L.pg = need; if (hb->phi_guess) need += al(c8);
  L.neo = need; need += al(c8);
  L.pho = need; need += al(c8);
  L.st = need; need += al(n4);
  L.nt = need; need += al(n4);
  L.kt = need; need += al(n4);
  L.re = need; need += al(n4);
  L.fr = need; need += al(n8);
  L.mg = need; need += al(n4);
  L.need = need;
  return L;
}

// host -> staging copies of the batch's inputs on stream st
cudaError_t stage_in(const Stage& L, char* d, const sdcef_batch* hb, cudaStream_t st) {
  const int64_t ncol = hb->ncol, cells = hb->col_off[ncol];
  const size_t c8 = (size_t)cells * 8, n8 = (size_t)ncol * 8;
  auto h2d = [&](size_t o, const void* src, size_t bytes) {
    return cudaMemcpyAsync(d + o, src, bytes, cudaMemcpyHostToDevice, st);
  };
  cudaError_t e = h2d(L.off, hb->col_off, (size_t)(ncol + 1) * 8);
  if (e == cudaSuccess) e = h2d(L.len, hb->length, n8);
  if (e == cudaSuccess) e = h2d(L.dt, hb->dt, n8);
  if (e == cudaSuccess) e = h2d(L.vl, hb->v_left, n8);
  if (e == cudaSuccess) e = h2d(L.vr, hb->v_right, n8);
  if (e == cudaSuccess) e = h2d(L.ne, hb->ne_old, c8);
  if (e == cudaSuccess) e = h2d(L.ph, hb->phi_old, c8);
  if (e == cudaSuccess && hb->n_species > 0) e = h2d(L.ion, hb->n_ion, c8 * hb->n_species);
  if (e == cudaSuccess) e = h2d(L.T, hb->T, c8);
  if (e == cudaSuccess && hb->u_adv) e = h2d(L.u, hb->u_adv, c8);
  if (e == cudaSuccess && hb->i_re) e = h2d(L.ir, hb->i_re, c8);
  if (e == cudaSuccess && hb->ne_guess) e = h2d(L.ng, hb->ne_guess, c8);
  if (e == cudaSuccess && hb->phi_guess) e = h2d(L.pg, hb->phi_guess, c8);
  return e;
}

// the device views of the staged batch and of its result slots
void stage_views(const Stage& L, char* d, const sdcef_batch* hb, sdcef_batch* db,
                 sdcef_result* dr) {
  *db = *hb;
  db->col_off = (const int64_t*)(d + L.off);
  db->length = (const double*)(d + L.len);
  db->dt = (const double*)(d + L.dt);
  db->v_left = (const double*)(d + L.vl);
  db->v_right = (const double*)(d + L.vr);
  db->ne_old = (const double*)(d + L.ne);
  db->phi_old = (const double*)(d + L.ph);
  db->n_ion = hb->n_species > 0 ? (const double*)(d + L.ion) : nullptr;
  db->T = (const double*)(d + L.T);
  db->rho = nullptr;
  db->u_adv = hb->u_adv ? (const double*)(d + L.u) : nullptr;
  db->i_re = hb->i_re ? (const double*)(d + L.ir) : nullptr;
  db->ne_guess = hb->ne_guess ? (const double*)(d + L.ng) : nullptr;
  db->phi_guess = hb->phi_guess ? (const double*)(d + L.pg) : nullptr;
  dr->ne_out = (double*)(d + L.neo);
  dr->phi_out = (double*)(d + L.pho);
  dr->status = (int*)(d + L.st);
  dr->newton_it = (int*)(d + L.nt);
  dr->krylov_it = (int*)(d + L.kt);
  dr->res_evals = (int*)(d + L.re);
  dr->final_res = (double*)(d + L.fr);
  dr->mg_cycles = (int*)(d + L.mg);
}

// staging -> host copies of the results the caller asked for, on stream st
cudaError_t stage_out(const Stage& L, char* d, const sdcef_batch* hb, const sdcef_result* ho,
                      cudaStream_t st) {
  const int64_t ncol = hb->ncol, cells = hb->col_off[ncol];
  const size_t c8 = (size_t)cells * 8, n8 = (size_t)ncol * 8, n4 = (size_t)ncol * 4;
  auto d2h = [&](void* dst, size_t o, size_t bytes) {
    return dst ? cudaMemcpyAsync(dst, d + o, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
  };
  cudaError_t e = d2h(ho->ne_out, L.neo, c8);
  if (e == cudaSuccess) e = d2h(ho->phi_out, L.pho, c8);
  if (e == cudaSuccess) e = d2h(ho->status, L.st, n4);
  if (e == cudaSuccess) e = d2h(ho->newton_it, L.nt, n4);
  if (e == cudaSuccess) e = d2h(ho->krylov_it, L.kt, n4);
  if (e == cudaSuccess) e = d2h(ho->res_evals, L.re, n4);
  if (e == cudaSuccess) e = d2h(ho->final_res, L.fr, n8);
  if (e == cudaSuccess) e = d2h(ho->mg_cycles, L.mg, n4);
  return e;
}

// the host batch is solvable by this context and the result pointers are usable
int check_host_batch(sdcef_ctx* ctx, const sdcef_batch* hb, const sdcef_result* ho) {
  int rc = validate_batch(ctx, hb, true);
  if (rc) return rc;
  if (!ho || !ho->ne_out || !ho->phi_out)
    return set_err(SDCEF_ERR_INVALID, "result: ne_out / phi_out is NULL");
  const int64_t cells = hb->ncol > 0 ? hb->col_off[hb->ncol] : 0;
  if (cells > ctx->max_cells || cells < 0)
    return set_err(SDCEF_ERR_CAPACITY, "batch: cells exceed max_cells");
  return SDCEF_SUCCESS;
}

// staging area of at least `bytes`; grown to twice the request so that
// later calls do not reallocate
int stage_reserve(sdcef_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->stage_bytes) return SDCEF_SUCCESS;
  if (ctx->stage) {
    cudaError_t e = cudaDeviceSynchronize();   // no copy or solve may still use the old area
    if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
    cudaFree(ctx->stage);
  }
  ctx->stage = nullptr;
  ctx->stage_bytes = 0;
  cudaError_t e = cudaMalloc((void**)&ctx->stage, bytes * 2);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_NOMEM, cudaGetErrorString(e));
  ctx->stage_bytes = bytes * 2;
  return SDCEF_SUCCESS;
}

}  // namespace

extern "C" {

int sdcef_solve_batch_host(sdcef_ctx* ctx, const sdcef_batch* hb, const sdcef_result* ho) {
  Range range_("sdcef_solve_batch_host");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  int rc = check_host_batch(ctx, hb, ho);
  if (rc) return rc;
  if (hb->ncol == 0) return SDCEF_SUCCESS;
  const Stage L = stage_layout(hb);
  if ((rc = stage_reserve(ctx, L.need))) return rc;
  char* d = ctx->stage;
  cudaError_t e = stage_in(L, d, hb, ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  sdcef_batch db;
  sdcef_result dr;
  stage_views(L, d, hb, &db, &dr);
  rc = sdcef_solve_batch(ctx, &db, &dr);
  if (rc) return rc;
  e = stage_out(L, d, hb, ho, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  return SDCEF_SUCCESS;
}

int sdcef_solve_batches_host(sdcef_ctx* ctx, int nbatch, const sdcef_batch* hbs,
                             const sdcef_result* hos) {
  Range range_("sdcef_solve_batches_host");
  if (!ctx) return set_err(SDCEF_ERR_INVALID, "ctx is NULL");
  if (nbatch < 0 || (nbatch > 0 && (!hbs || !hos)))
    return set_err(SDCEF_ERR_INVALID, "batches: nbatch < 0 or NULL arrays");
  size_t half = 0;
  for (int k = 0; k < nbatch; ++k) {
    int rc = check_host_batch(ctx, &hbs[k], &hos[k]);
    if (rc) return rc;
    if (hbs[k].ncol > 0) half = std::max(half, (stage_layout(&hbs[k]).need + 255) & ~(size_t)255);
  }
  if (half == 0) return SDCEF_SUCCESS;
  int rc = stage_reserve(ctx, 2 * half);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!ctx->pipe) {
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&ctx->cs[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_free[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
    ctx->pipe = true;
  }
  // copies start after the work already enqueued on the context stream
  e = cudaEventRecord(ctx->ev_free[0], ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_free[1], ctx->stream);
  for (int k = 0; k < nbatch && e == cudaSuccess; ++k) {
    const sdcef_batch* hb = &hbs[k];
    if (hb->ncol == 0) continue;
    const int h = k & 1;
    char* d = ctx->stage + (size_t)h * half;
    const Stage L = stage_layout(hb);
    // inputs of batch k once this half's previous batch has been solved and read back
    e = cudaStreamWaitEvent(ctx->cs[0], ctx->ev_free[h], 0);
    if (e == cudaSuccess) e = stage_in(L, d, hb, ctx->cs[0]);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in[h], ctx->cs[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_in[h], 0);
    if (e != cudaSuccess) break;
    sdcef_batch db;
    sdcef_result dr;
    stage_views(L, d, hb, &db, &dr);
    if ((rc = sdcef_solve_batch(ctx, &db, &dr))) break;
    e = cudaEventRecord(ctx->ev_done[h], ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cs[1], ctx->ev_done[h], 0);
    if (e == cudaSuccess) e = stage_out(L, d, hb, &hos[k], ctx->cs[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_free[h], ctx->cs[1]);
  }
  // every copy and solve has finished before the call returns (also on an error)
  cudaError_t e2 = cudaStreamSynchronize(ctx->cs[0]);
  cudaError_t e3 = cudaStreamSynchronize(ctx->stream);
  cudaError_t e4 = cudaStreamSynchronize(ctx->cs[1]);
  if (rc) return rc;
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
  if (e != cudaSuccess) return set_err(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  return SDCEF_SUCCESS;
}

}  // extern "C"
