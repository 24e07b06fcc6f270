// Kernels on the column fields around the solve: the provisional charged
// species of an SDC iteration (electric drift only, or the paper's transport)
// and the charge flux through every face. Argument blocks and launchers;
// the kernels are in fields.cu.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/sdcef.h"

namespace sdcef_impl {

// Provisional charged species of one SDC iteration (electric drift only).
struct IonArgs {
  int64_t ncol;
  const int64_t* col_off;
  const double *length, *dt, *vl, *vr, *phi, *n_in;
  double* n_out;
  int nsp;
  int val[SDCEF_MAX_SPECIES];
  double kappa;
  unsigned* chk;   // check word of the bounds-checking build (may be null)
};
cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t st);

// Provisional ions with the paper's transport (second-order Godunov
// advection, implicit diffusion, SDC diffusion correction).
struct IonProvArgs {
  int64_t ncol;
  const int64_t* col_off;
  const double *length, *dt, *vl, *vr, *T, *u, *phi, *n0, *nk;
  double *n_out, *scratch;
  int nsp;
  int val[SDCEF_MAX_SPECIES];
  double kappa;
  unsigned* chk;   // check word of the bounds-checking build (may be null)
};
cudaError_t launch_ion_provisional(const IonProvArgs& a, cudaStream_t st);

// Charge flux through every face of every column (Sec. 4.4).
struct CurrentArgs {
  int64_t ncol;
  const int64_t* col_off;
  const double *length, *vl, *vr, *T, *u, *ne, *phi, *n_ion;
  double *jp, *jn;
  int nsp, bc;
  int val[SDCEF_MAX_SPECIES];
  double kappa, mu;
  const double* tab;    // transport tables (mu then D), or null: constant mobility, Einstein D
  int tnc, tnx;
  double ten_max_td, tT_in, tinv_dT, tgas_W;
  const double* rho;
  unsigned* chk;   // check word of the bounds-checking build (may be null)
};
cudaError_t launch_current(const CurrentArgs& a, cudaStream_t st);
// B(x) and B'(x) of the Scharfetter-Gummel flux, as the residual evaluates them.

}  // namespace sdcef_impl
