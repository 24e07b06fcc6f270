// Bounds checks of the debug build (compiled with -DSDCEF_CHECKS), the
// stand-in for a device memory checker: every plane, level, shared-memory and
// global index the kernels form is tested before it is used. A failing test
// records its site number in the call's check word (the first failure wins)
// and the access is redirected to element 0 of the same array, so nothing
// outside an array is read or written and nothing traps. The host reads and
// clears the word after the call (sdcef_check_word, sdcef_mlp_check_word).
// Without SDCEF_CHECKS every test is the constant true and compiles away.
#pragma once
#include <cuda_runtime.h>

namespace sdcef_chk {

// Site numbers recorded in the check word.
enum Site : unsigned {
  kIx = 101,        // plane row j < rows per thread, thread < threads per column
  kPlane = 102,     // FP64 plane number < PD_COUNT
  kKrylov = 103,    // Krylov basis vector / component
  kZk = 104,        // flexible-GMRES z_i vector / component
  kCell = 105,      // global cell index inside the column
  kCol = 106,       // column index from the queue or the column order
  kRed = 107,       // block-reduction scratch
  kHess = 108,      // Hessenberg / Arnoldi scratch
  kFacPlane = 201,  // factor plane number or row of the block solver
  kScal = 202,      // per-thread scalar of the block solver
  kRedRow = 203,    // row of the reduced (separator) system in shared memory
  kScr = 204,       // block-solver right-hand side / scratch / output row
  kMgLevel = 301,   // multigrid level offset + size inside its region
  kIonCell = 401,   // column cells of the ion / current kernels inside the batch
  kMlpRow = 501,    // row of an MLP kernel inside its matrix
  kMlpStage = 502,  // guess kernel: staged feature values inside their buffer
  kMlpSmem = 503,   // MLP kernels: shared-memory operand offset
};

#ifdef SDCEF_CHECKS
// check word and rows per thread of the running solver kernel (set by thread 0
// at its entry, read by the index helpers of the solver and the block solver)
static __shared__ unsigned* s_word;
static __shared__ int s_kmax;

__device__ __forceinline__ bool hit(unsigned* word, unsigned site) {
  if (word) atomicCAS(word, 0u, site);
  return false;
}
#endif

}  // namespace sdcef_chk

#ifdef SDCEF_CHECKS
// true if cond holds; else records site in *word (or the solver kernel's word)
#define SDCEF_CHECK_W(word, cond, site) ((cond) ? true : sdcef_chk::hit((word), (site)))
#define SDCEF_CHECK(cond, site) SDCEF_CHECK_W(sdcef_chk::s_word, cond, site)
#else
#define SDCEF_CHECK_W(word, cond, site) true
#define SDCEF_CHECK(cond, site) true
#endif
