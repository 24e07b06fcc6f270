// Allocation-free variant of sdcef_solve_batch (see include/sdcef.h).
//
// Some callers cannot call cudaMalloc at solve time: an application whose
// device memory is handed out entirely by its own arena allocator, or a
// time-stepping code that forbids allocation after start-up so its memory
// footprint stays fixed. This entry point runs the same persistent solver
// kernel as sdcef_solve_batch, but its workspace (the per-CTA column slots,
// the work-queue counter and the column order) lives in one file-scope
// device array of fixed size instead of memory allocated by sdcef_create.
// Every GPU that loads the library holds this array until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/sdcef.h"
#include "solver.cuh"

namespace sdcef_impl {
int report_error(int code, const char* msg);
int validate_params(const sdcef_params* p);
}  // namespace sdcef_impl

using namespace sdcef_impl;

namespace {

constexpr size_t kHeaderBytes = 256 + sizeof(int) * (size_t)SDCEF_NOALLOC_MAX_COLS;
constexpr size_t kHeaderAligned = (kHeaderBytes + 255) & ~(size_t)255;

// The scratch array. In host code `g_scratch` names a host-side stand-in, not
// a device address; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[SDCEF_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device and its SM count,
// looked up on every call (neither allocates): an address kept from an earlier
// call would go stale after cudaDeviceReset or a new primary context.
int scratch_for_current_device(unsigned char** ptr, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  int n = 0;
  e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  *ptr = (unsigned char*)p;
  *sms = n;
  return SDCEF_SUCCESS;
}

}  // namespace

extern "C" int sdcef_solve_batch_noalloc(const sdcef_params* p, const sdcef_batch* b,
                                         const sdcef_result* out, int max_col_cells,
                                         void* stream) {
  int rc = validate_params(p);
  if (rc) return rc;
  if (p->transport != SDCEF_TRANSPORT_CONSTANT)
    return report_error(SDCEF_ERR_INVALID, "noalloc: transport tables need a context");
  if (!b) return report_error(SDCEF_ERR_INVALID, "noalloc: batch is NULL");
  if (b->ncol < 0) return report_error(SDCEF_ERR_INVALID, "noalloc: ncol < 0");
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (b->ncol > SDCEF_NOALLOC_MAX_COLS)
    return report_error(SDCEF_ERR_CAPACITY, "noalloc: ncol exceeds SDCEF_NOALLOC_MAX_COLS");
  if (max_col_cells < 2 || max_col_cells > SDCEF_NOALLOC_MAX_COL_CELLS)
    return report_error(SDCEF_ERR_CAPACITY,
                        "noalloc: max_col_cells must be in [2, SDCEF_NOALLOC_MAX_COL_CELLS]");
  if (!b->col_off || !b->length || !b->dt || !b->v_left || !b->v_right || !b->T || !b->ne_old ||
      !b->phi_old)
    return report_error(SDCEF_ERR_INVALID, "noalloc: required batch pointer is NULL");
  if (b->n_species < 0 || b->n_species > SDCEF_MAX_SPECIES ||
      (b->n_species > 0 && (!b->valence || !b->n_ion)))
    return report_error(SDCEF_ERR_INVALID, "noalloc: ion species arguments");
  if (!out || !out->ne_out || !out->phi_out)
    return report_error(SDCEF_ERR_INVALID, "noalloc: ne_out / phi_out is NULL");

  unsigned char* base = nullptr;
  int sms = 0;
  rc = scratch_for_current_device(&base, &sms);
  if (rc) return rc;

  const int tpb = p->precond == SDCEF_PREC_MG ? kMgTPB
                  : (p->threads_per_column ? p->threads_per_column : 128);
  const int prec = p->precision;
  const int m = p->restart_m;
  const int kmax = (max_col_cells + tpb - 1) / tpb;
  const size_t PL = (size_t)kmax * tpb;
  const size_t slot = slot_bytes_prec(prec, PL, m, tpb, p->precond);
  const size_t avail = SDCEF_NOALLOC_SCRATCH_BYTES - kHeaderAligned;
  const int64_t nslots = (int64_t)(avail / slot);
  if (nslots < 1)
    return report_error(SDCEF_ERR_CAPACITY, "noalloc: one column slot does not fit the scratch array");

  KArgs a;
  memset(&a, 0, sizeof(a));
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
  a.ne_out = out->ne_out;
  a.phi_out = out->phi_out;
  a.status = out->status;
  a.newton_it = out->newton_it;
  a.krylov_it = out->krylov_it;
  a.res_evals = out->res_evals;
  a.mg_cycles = out->mg_cycles;
  a.final_res = out->final_res;
  a.queue = (int*)base;                        // bytes [0, 4): work-queue counter
  int* order = (int*)(base + 256);             // SDCEF_NOALLOC_MAX_COLS ints
  a.ws = (char*)(base + kHeaderAligned);       // column slots
  a.kmax = kmax;
  a.PL = PL;
  a.slot_bytes = slot;
  a.max_col_cells = max_col_cells;
  a.p.eps_F = p->eps_F;
  a.p.eps_X = p->eps_X;
  a.p.eps_E = p->eps_E;
  a.p.stall = p->stall_ratio > 0.0 ? p->stall_ratio : 2.0;
  a.p.gamma = p->gamma;
  a.p.mu = p->mobility;
  a.p.ls_alpha = p->ls_alpha;
  a.p.kap = kEps0 * p->eps_r / kQe;
  a.p.m = m;
  a.p.max_newton = p->max_newton;
  a.p.max_krylov = p->max_krylov;
  a.p.max_ls = p->max_linesearch;
  a.p.bc = p->bc_electron;
  a.p.precond = p->precond;
  a.p.guess_cap = p->guess_newton_cap;
  a.p.guess_ratio = p->guess_reject_ratio;
  a.p.guess_prog = p->guess_progress;
  a.p.mg_gA = p->mg_gamma_A;
  a.p.mg_gS = p->mg_gamma_S;
  a.p.mg_maxc = p->mg_max_cycles;
  a.p.mg_transfer = p->mg_transfer;
  a.mode = MODE_SOLVE;

  cudaStream_t st = (cudaStream_t)stream;
  size_t smem = smem_bytes_prec(prec, tpb, m);
  const int per_sm = occupancy_prec(prec, tpb, smem, p->precond, SDCEF_TRANSPORT_CONSTANT);
  if (p->krylov_on_chip)
    smem = krylov_arena(prec, tpb, smem, per_sm, p->precond, SDCEF_TRANSPORT_CONSTANT, &a);
  const int grid = (int)std::min<int64_t>({(int64_t)per_sm * sms, a.ncol, nslots});
  // the queue counter must start at zero; everything else a call reads it writes first
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  if (a.ncol > 1) {
    int shift = 4;
    while ((max_col_cells >> shift) + 1 > 4096) ++shift;
    const int nbins = (max_col_cells >> shift) + 1;
    e = launch_order(a.col_off, a.ncol, nbins, shift, order, st);
    if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
    a.order = order;
  }
  e = launch_prec(prec, tpb, a, grid, smem, st);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  return SDCEF_SUCCESS;
}
