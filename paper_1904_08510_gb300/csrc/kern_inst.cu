// Explicit instantiation of the solver kernel for one (threads per column,
// Krylov type, preconditioner type) triple, selected with -DSDCEF_TPB=...
// -DSDCEF_KR=... -DSDCEF_PR=..., or of the multigrid-preconditioner kernel
// with -DSDCEF_MG; the order kernel is built in the TU compiled with
// -DSDCEF_WITH_ORDER.
#define SDCEF_KERNEL_TU
#include "solver.cuh"

namespace sdcef_impl {
#if defined(SDCEF_MG)
// the multigrid-preconditioner kernel (FP64, kMgTPB threads per column)
cudaError_t launch_mg(const KArgs& a, int grid, size_t smem, cudaStream_t st) {
  return launch_mg_t(a, grid, smem, st);
}
int occupancy_mg(size_t smem) { return occupancy_mg_t(smem); }
#elif defined(SDCEF_TAB)
// the transport-table kernel (FP64, kMgTPB threads per column)
cudaError_t launch_tab(const KArgs& a, int grid, size_t smem, cudaStream_t st) {
  return launch_tab_t(a, grid, smem, st);
}
int occupancy_tab(size_t smem) { return occupancy_tab_t(smem); }
#else
template cudaError_t launch_t<SDCEF_TPB, SDCEF_KR, SDCEF_PR>(const KArgs&, int, size_t, cudaStream_t);
template int occupancy_t<SDCEF_TPB, SDCEF_KR, SDCEF_PR>(size_t);
#endif
#ifdef SDCEF_WITH_ORDER
cudaError_t launch_order(const int64_t* col_off, int64_t ncol, int nbins, int shift, int* order,
                         cudaStream_t st) {
  order_kernel<<<1, 1024, nbins * sizeof(int), st>>>(col_off, ncol, nbins, shift, order);
  return cudaGetLastError();
}
cudaError_t launch_bernoulli(const double* x, double* b, double* db, int64_t n, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  bernoulli_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(x, b, db, n);
  return cudaGetLastError();
}
#endif
}  // namespace sdcef_impl
