// Device code of the batched JFNK solver: kernel arguments, workspace layout,
// residual (Eq. nls), finite-difference Jacobian-vector product
// (Eq. jf_dfapprox), preconditioner factorisation/application (Eq. prec,
// Eq. prec_recast), right-preconditioned GMRES and the Newton driver of
// Algorithm 2. Kernel templates are instantiated in kern_inst.cu, one
// translation unit per (threads per column, Krylov precision).
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "../../include/sdcef.h"
#include "checks.cuh"
#include "blockalg.cuh"
#include "expm1_table.cuh"
#include "mg.cuh"

namespace sdcef_impl {
using namespace sdcef;

// SI constants (CODATA 2018)
constexpr double kQe = 1.602176634e-19;
constexpr double kKb = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kNA = 6.02214076e23;
// lambda_FD = eps_mach^(1/3) for IEEE double (Eq. jf_dfapprox)
constexpr double kLambdaFD = 6.0554544523933395e-06;
// Newton steps a column may take for the error test after the residual test holds
constexpr int kMaxPolish = 2;
constexpr double kErrMargin = 10.0;   // error_test: a pass this close to the bar is re-taken


// --------------------------------------------------------------------------
// Kernel arguments
// --------------------------------------------------------------------------
struct DevParams {
  double eps_F, eps_X, gamma, mu, ls_alpha, kap;   // kap = eps0 eps_r / e
  double eps_E;         // error test at the stop (relative, per field); 0 = off
  double stall;         // GMRES restart-cycle stagnation ratio (> 1: never)
  int m, max_newton, max_krylov, max_ls, bc, precond;
  int guess_cap;   // Newton steps from a supplied start before restarting from X^n (0 = never)
  double guess_ratio;   // reject a supplied start with ||Fhat|| > ratio ||Fhat(X^n)|| (0 = never)
  double guess_prog;    // restart a supplied start whose step keeps ||Fhat||_inf above this fraction (0 = never)
  double mg_gA, mg_gS;  // multigrid tolerances of the two blocks (<= 0: exact block solve)
  int mg_maxc, mg_transfer;
  int transport;        // SDCEF_TRANSPORT_*
};

// Electron transport tables (SDCEF_TRANSPORT_TABLE): mu then D, each [nc][nx]
// over c_k = k/(nc-1) and E/N_j = j en_max/(nx-1) Td.
struct TransportTab {
  const double* tab;
  int nc, nx;
  double en_max_td, T_in, inv_dT, gas_W;
};

enum { MODE_SOLVE = 0, MODE_RESIDUAL = 1, MODE_PRECOND = 2 };

// Solver kernel variants (template parameter VAR): the base kernel, the one
// carrying the multigrid preconditioner, and the one with field-dependent
// electron transport from tables. Each is its own instantiation so that the
// base kernel compiles without the others' code.
enum { kVarBase = 0, kVarMG = 1, kVarTable = 2 };

struct KArgs {
  int64_t ncol;
  const int64_t* col_off;
  const double *length, *dt, *vl, *vr, *ne_old, *phi_old;
  int nsp;
  int val[SDCEF_MAX_SPECIES];
  const double *n_ion, *T, *u, *ire, *ne_g, *phi_g;
  double *ne_out, *phi_out;
  int *status, *newton_it, *krylov_it, *res_evals, *mg_cycles;
  double* final_res;
  // workspace
  char* ws;
  size_t slot_bytes;
  size_t PL;          // elements per plane (kmax * TPB)
  int kmax;           // rows per thread capacity
  int max_col_cells;
  int* queue;
  const int* order;
  DevParams p;
  int mode;
  // on-chip Krylov planes: byte offset and size of their region in the dynamic
  // shared memory (size 0: every Krylov plane is in the slot)
  unsigned arena_off, arena_bytes;
  // test modes: state X, residual-space vector r, outputs
  const double *x_ne, *x_phi, *r_e, *r_phi;
  double *o1, *o2;
  // field-dependent transport
  TransportTab tt;
  const double* rho;
  unsigned* chk;      // check word of the bounds-checking build (may be null)
};

// FP64 planes of a slot
enum {
  // PD_MUHD: mu / D_f per face; PD_PE0: (u_f + mu g0) h / D_f, the face Peclet number
  // at dpsi/dx = 0, so that Pe = PD_PE0 + PD_MUHD (psi_{i+1} - psi_i) is one FMA
  // (the transport-table kernel keeps its E/N index factor in PD_MUHD instead)
  PD_N = 0, PD_PSI, PD_FE0, PD_FP0, PD_FE1, PD_FP1, PD_FEX, PD_FPHI, PD_DH, PD_MUHD, PD_PE0, PD_PREF,
  // 3 planes per set: r dGam/dn_i, r dGam/dn_{i+1} (times s_n / s_Fe) and
  // r dGam/dpsi_{i+1} (= -r dGam/dpsi_i, times s_psi / s_Fe) of face i+1/2
  PD_FACE0,
  PD_FACE1 = PD_FACE0 + 3,
  // state (n, psi) of set 1; set 0 is PD_N, PD_PSI. The state of set s is the
  // X whose residual is in (PD_FE0, PD_FP0) + 2 s and whose face derivatives are
  // face set s, so a line-search trial writes its state into the other set and
  // accepting it only switches sets.
  PD_N1 = PD_FACE1 + 3, PD_PSI1,
  PD_COUNT
};
__device__ __forceinline__ int pd_n(int set) { return set ? PD_N1 : PD_N; }
__device__ __forceinline__ int pd_psi(int set) { return set ? PD_PSI1 : PD_PSI; }
// Krylov planes (type KR): V[(m+1)*2], W[2], Z[2], XH[2], T[2], ZK[m*2]
// Preconditioner planes (type PR): 20 factor planes + 2 scratch planes for the
// forward/backward sweeps of a solve; per-thread scalars (type PR).
constexpr int kFactorPlanes = 22;
constexpr int kScrPlane = 20;
constexpr int kScalPerThread = FIdx<2>::NSCAL;   // >= 2 * FIdx<1>::NSCAL for the recast form

template <typename KR, typename PR>
__host__ __device__ inline size_t slot_bytes_for(size_t PL, int m, int tpb) {
  size_t b = (size_t)PD_COUNT * PL * sizeof(double);
  b += (size_t)(2 * (m + 1) + 8 + 2 * m) * PL * sizeof(KR);
  b = (b + 15) & ~(size_t)15;
  b += (size_t)kFactorPlanes * PL * sizeof(PR);
  b += (size_t)kScalPerThread * tpb * sizeof(PR);
  return (b + 255) & ~(size_t)255;
}
// Dynamic shared memory of the solver kernel: reduction scratch, halo,
// Hessenberg / Givens state (FP64) and the block-solver exchange area (PR).
inline size_t smem_bytes_for(int tpb, int m, size_t pr_bytes) {
  const int nw = tpb / 32;
  size_t d = (size_t)(nw + 1) * 40 + 4 * tpb + (m + 1) * m + (m + 1) + 3 * m + m + 2;
  return d * sizeof(double) + 12 * (size_t)tpb * pr_bytes + 64;
}


// Launch / occupancy entry points, one instantiation per kernel TU.
template <int TPB, typename KR, typename PR>
cudaError_t launch_t(const KArgs& a, int grid, size_t smem, cudaStream_t st);
template <int TPB, typename KR, typename PR>
int occupancy_t(size_t smem);
// the multigrid preconditioner runs in its own FP64 kernel instantiation
constexpr int kMgTPB = 128;
cudaError_t launch_mg(const KArgs& a, int grid, size_t smem, cudaStream_t st);
int occupancy_mg(size_t smem);
// field-dependent transport: its own FP64 instantiation, kMgTPB threads per column
cudaError_t launch_tab(const KArgs& a, int grid, size_t smem, cudaStream_t st);
int occupancy_tab(size_t smem);

// Precision modes as (Krylov type KR, preconditioner type PR):
//   SDCEF_FP64 (double, double), SDCEF_MIXED (float, float),
//   SDCEF_MIXED_DF (double, dfloat).
// The multigrid preconditioner (FP64 only) appends its region to the slot.
inline size_t slot_bytes_prec(int precision, size_t PL, int m, int tpb, int precond) {
  if (precision == SDCEF_MIXED) return slot_bytes_for<float, float>(PL, m, tpb);
  if (precision == SDCEF_MIXED_DF) return slot_bytes_for<double, dfloat>(PL, m, tpb);
  const size_t mg = precond == SDCEF_PREC_MG ? mg_region_doubles(PL) * sizeof(double) : 0;
  return slot_bytes_for<double, double>(PL, m, tpb) + mg;
}
inline size_t smem_bytes_prec(int precision, int tpb, int m) {
  return smem_bytes_for(tpb, m, precision == SDCEF_MIXED ? sizeof(float) : 8);
}
#ifndef SDCEF_KERNEL_TU
// Host dispatch (host translation units only: in a kernel unit these bodies
// would instantiate every kernel).
template <typename KR, typename PR>
inline cudaError_t launch_tpb(int tpb, const KArgs& a, int grid, size_t smem, cudaStream_t st) {
  switch (tpb) {
    case 32: return launch_t<32, KR, PR>(a, grid, smem, st);
    case 64: return launch_t<64, KR, PR>(a, grid, smem, st);
    case 128: return launch_t<128, KR, PR>(a, grid, smem, st);
    case 256: return launch_t<256, KR, PR>(a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}
template <typename KR, typename PR>
inline int occupancy_tpb(int tpb, size_t smem) {
  switch (tpb) {
    case 32: return occupancy_t<32, KR, PR>(smem);
    case 64: return occupancy_t<64, KR, PR>(smem);
    case 128: return occupancy_t<128, KR, PR>(smem);
    case 256: return occupancy_t<256, KR, PR>(smem);
  }
  return 1;
}
inline cudaError_t launch_prec(int precision, int tpb, const KArgs& a, int grid, size_t smem,
                               cudaStream_t st) {
  if (a.p.precond == SDCEF_PREC_MG) return launch_mg(a, grid, smem, st);
  if (a.p.transport == SDCEF_TRANSPORT_TABLE) return launch_tab(a, grid, smem, st);
  if (precision == SDCEF_MIXED) return launch_tpb<float, float>(tpb, a, grid, smem, st);
  if (precision == SDCEF_MIXED_DF) return launch_tpb<double, dfloat>(tpb, a, grid, smem, st);
  return launch_tpb<double, double>(tpb, a, grid, smem, st);
}
inline int occupancy_prec(int precision, int tpb, size_t smem, int precond, int transport) {
  if (precond == SDCEF_PREC_MG) return occupancy_mg(smem);
  if (transport == SDCEF_TRANSPORT_TABLE) return occupancy_tab(smem);
  if (precision == SDCEF_MIXED) return occupancy_tpb<float, float>(tpb, smem);
  if (precision == SDCEF_MIXED_DF) return occupancy_tpb<double, dfloat>(tpb, smem);
  return occupancy_tpb<double, double>(tpb, smem);
}
// Region for on-chip Krylov planes: the shared memory an SM has left when
// per_sm CTAs of the kernel (registers decide per_sm) each hold smem bytes,
// split evenly between them, so that the region does not lower the occupancy.
// Sets a->arena_off / arena_bytes and returns the launch's dynamic shared
// memory (smem when no region fits).
inline size_t krylov_arena(int precision, int tpb, size_t smem, int per_sm, int precond,
                           int transport, KArgs* a) {
  a->arena_off = 0;
  a->arena_bytes = 0;
  int dev = 0, per_sm_bytes = 0, reserved = 0, optin = 0;
  if (per_sm < 1 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return smem;
  const size_t off = (smem + 255) & ~(size_t)255;
  long long avail = std::min<long long>((long long)per_sm_bytes / per_sm - reserved, optin);
  avail = (avail - (long long)off) & ~255LL;
  // the kernel's static shared memory also counts: step down until the
  // occupancy holds
  for (; avail >= 4096; avail -= 256) {
    if (occupancy_prec(precision, tpb, off + (size_t)avail, precond, transport) >= per_sm) {
      a->arena_off = (unsigned)off;
      a->arena_bytes = (unsigned)avail;
      return off + (size_t)avail;
    }
  }
  return smem;
}
#endif  // SDCEF_KERNEL_TU
cudaError_t launch_order(const int64_t* col_off, int64_t ncol, int nbins, int shift, int* order,
                         cudaStream_t st);

cudaError_t launch_bernoulli(const double* x, double* b, double* db, int64_t n, cudaStream_t st);

#ifdef SDCEF_KERNEL_TU
// --------------------------------------------------------------------------
// Block reductions
// --------------------------------------------------------------------------
template <int TPB>
__device__ __forceinline__ void block_reduce(double* v, int nv, bool is_max, double* red) {
  constexpr int NW = TPB / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (!SDCEF_CHECK(nv >= 0 && nv <= 40, sdcef_chk::kRed)) nv = 0;
  for (int k = 0; k < nv; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = is_max ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[w * 40 + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double x = red[threadIdx.x];
    for (int q = 1; q < NW; ++q) {
      double y = red[q * 40 + threadIdx.x];
      x = is_max ? fmax(x, y) : x + y;
    }
    red[NW * 40 + threadIdx.x] = x;
  }
  __syncthreads();
  for (int k = 0; k < nv; ++k) v[k] = red[NW * 40 + k];
  __syncthreads();
}

// --------------------------------------------------------------------------
// Bernoulli function of the Scharfetter-Gummel flux. For a = |Pe| >= 0:
// b = B(a) = a / (e^a - 1) and the derivative B'(a) = (1 - a - b) / (e^a - 1).
// B(-a) = a + B(a) and B'(-a) = -1 - B'(a) give the other branch without
// cancellation, so one expm1 and one division serve both.
// --------------------------------------------------------------------------
// Order tests on non-negative doubles run on the integer pipe: for x, y >= 0 the
// IEEE bit patterns order like the values (NaN patterns sort above +inf).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
constexpr long long kBits1em3 = 0x3F50624DD2F1A9FCLL;   // bit pattern of 1e-3

// e^a - 1 for a >= 1e-3 (+inf for a >= 709 and for NaN), FP64, after the
// table-driven method of P. T. P. Tang (ACM TOMS 15, 1989, for exp; ACM TOMS
// 18, 1992, for expm1), with a table of 1024 entries:
//   k = round(1024 a / ln 2) = 1024 M + j,  r = a - k ln2/1024 (|r| <= ln2/2048),
//   e^a = 2^M 2^(j/1024) e^r,  e^r - 1 = p(r) = r + r^2 (1/2 + r/6 + r^2/24)
//   (Taylor; truncation below 4e-20 on |r| <= ln2/2048),
//   e^a - 1 = (2^M T_hi - 1) + 2^M (T_lo + T_hi p),  2^(j/1024) = T_hi + T_lo.
// k comes from the shifter trick (a * 1024/ln2 + 1.5 2^52 rounds to an integer
// held in the low bits) and 2^M from the exponent bits, so the whole
// evaluation is 11 FP64 operations; the 16 KB table is read through L1. For a
// in [709, inf) the Bernoulli function underflows (a / (e^a - 1) < 1e-305) and
// +inf gives B = 0.
__device__ __forceinline__ double expm1_pos(double a) {
  constexpr long long kBits709 = 0x4086280000000000LL;   // bit pattern of 709.0
  if (dbits(a) >= kBits709) return __longlong_as_double(0x7FF0000000000000LL);
  constexpr double kShift = 0x1.8p52;
  constexpr int kMask = (1 << kExpTabBits) - 1;
  const double t = fma(a, kExpInvL, kShift);
  const int k = __double2loint(t);
  const double kd = t - kShift;
  double r = fma(-kd, kExpL1, a);
  r = fma(-kd, kExpL2, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(r * r, q, r);
  const double2 T = __ldg(&kExp2Tab[k & kMask]);
  const double u = fma(T.x, p, T.y);
  const double s = __longlong_as_double((long long)((k >> kExpTabBits) + 1023) << 52);
  return fma(s, u, fma(s, T.x, -1.0));
}

// DERIV = false skips B'(a): the finite-difference JVP needs fluxes only.
// 1/E for E >= 1e-3: the hardware's approximate reciprocal y (relative error
// ~1e-6) refined by one Newton-Raphson step that keeps the second-order term,
// y (1 + e + e^2) with e = 1 - E y (the series 1/E = y / (1 - e) cut after e^2),
// so the result's error is the seed's cubed, below rounding. E = +inf (a >= 709)
// gives 0, as 1/E does.
__device__ __forceinline__ double rcp_pos(double E) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(E));
  const double e = fma(-E, y, 1.0);
  const double r = fma(y, fma(e, e, e), y);
  return dbits(E) >= 0x7FF0000000000000LL ? 0.0 : r;
}
template <bool DERIV>
__device__ __forceinline__ void bern_pos(double a, double* b, double* db) {
  if (dbits(a) < kBits1em3) {
    double a2 = a * a;
    *b = 1.0 - 0.5 * a + a2 * (1.0 / 12.0) - a2 * a2 * (1.0 / 720.0);
    if (DERIV) *db = -0.5 + a * (1.0 / 6.0) - a * a2 * (1.0 / 180.0);
  } else {
    double E = expm1_pos(a);
    double iE = rcp_pos(E);
    *b = a * iE;
    if (DERIV) *db = (1.0 - a - *b) * iE;
  }
}

// --------------------------------------------------------------------------
// Per-CTA column context (shared memory) and per-thread geometry
// --------------------------------------------------------------------------
struct ColShared {
  int64_t col, off;
  int N, K, tact, bad;
  double h, inv_h, dt, vl, vr, g0, ubl, ubr;
  double sn, sp, sFe, sFp;
  // reciprocals / ratios of the scales, set once per column
  double isn, isp, isFe, isFp, r_a, r_b, r_c, r_l, r_rho;
  double vL[2], vR[2];      // electrode-face electron velocities of face sets 0/1
  double xnorm;
  int flag;
  double gam, beta0;
  int conv, stop;
  double scal[8];
  double pref0, dpref;                  // phi_ref at cell i: pref0 + dpref * i
  // scaled Poisson stencil of the Jacobian rows: kap/h^2 s_phi/s_Fphi and multiples
  double kh2, m2kh2, m4kh2, kh2_43;
  double vald[SDCEF_MAX_SPECIES];       // ion valences as doubles
  int mgc;                              // V-cycles of this column's multigrid block solves
  // error test: factors of an earlier Newton step are in the slot; Newton steps
  // taken for the error test; the current step is one of them
  int have_prec, polished;
  // transport tables: table coordinates of the electrode faces (c index, and
  // the factor turning |G| into the E/N index) and dv/dG = mu + G mu'(G) there
  double tcL, sxL, tcR, sxR, muL[2], muR[2];
};

struct Geo {
  int tid, kt, t0, N, K, tact;
};

// Component pointers of the running column's Krylov pairs, by slot position
// (set per column by krylov_table).
constexpr int kMaxKPairs = 2 * SDCEF_MAX_RESTART + 5;
static __shared__ void* s_kptr[2 * kMaxKPairs];

template <int TPB, typename KR, typename PR>
struct Slot {
  double* d;    // FP64 planes
  KR* k;        // Krylov planes
  PR* f;        // preconditioner planes
  PR* s;        // per-thread scalars
  size_t PL;
  int m;
  __device__ double* pd(int i) const {
    if (!SDCEF_CHECK(i >= 0 && i < PD_COUNT, sdcef_chk::kPlane)) i = 0;
    return d + (size_t)i * PL;
  }
  // Krylov pairs by slot position: V_0..V_m, W, Z, XH, T, ZK_0..ZK_{m-1}; the
  // component pointers come from the column's table (on chip or in the slot)
  __device__ KR* kp(int pos, int comp) const {
    return static_cast<KR*>(s_kptr[2 * pos + comp]);
  }
  __device__ KR* V(int i, int comp) const {
    if (!SDCEF_CHECK(i >= 0 && i <= m && (comp == 0 || comp == 1), sdcef_chk::kKrylov)) i = comp = 0;
    return kp(i, comp);
  }
  __device__ KR* W(int comp) const { return kp(m + 1, cmp(comp)); }
  __device__ KR* Z(int comp) const { return kp(m + 2, cmp(comp)); }
  __device__ KR* XH(int comp) const { return kp(m + 3, cmp(comp)); }
  __device__ KR* T(int comp) const { return kp(m + 4, cmp(comp)); }
  // a component number, 0 (n) or 1 (psi)
  __device__ static int cmp(int comp) {
    if (!SDCEF_CHECK(comp == 0 || comp == 1, sdcef_chk::kKrylov)) comp = 0;
    return comp;
  }
  // Mhat^{-1} V_i of the current GMRES cycle (flexible-GMRES storage)
  __device__ KR* ZK(int i, int comp) const {
    if (!SDCEF_CHECK(i >= 0 && i < m && (comp == 0 || comp == 1), sdcef_chk::kZk)) i = comp = 0;
    return kp(m + 5 + i, comp);
  }
};

template <int TPB, typename KR, typename PR>
__device__ Slot<TPB, KR, PR> make_slot(const KArgs& a, int slot) {
  Slot<TPB, KR, PR> s;
  char* base = a.ws + (size_t)slot * a.slot_bytes;
  s.PL = a.PL;
  s.m = a.p.m;
  s.d = (double*)base;
  s.k = (KR*)(base + (size_t)PD_COUNT * a.PL * sizeof(double));
  size_t kb = (size_t)PD_COUNT * a.PL * sizeof(double) +
              (size_t)(2 * (a.p.m + 1) + 8 + 2 * a.p.m) * a.PL * sizeof(KR);
  kb = (kb + 15) & ~(size_t)15;
  s.f = (PR*)(base + kb);
  s.s = s.f + (size_t)kFactorPlanes * a.PL;
  return s;
}

// Element of row j of thread tid in a slot plane (every plane holds kmax * TPB
// elements).
__device__ __forceinline__ size_t ix(int j, int tid, int TPB) {
#ifdef SDCEF_CHECKS
  if (!SDCEF_CHECK(j >= 0 && j < sdcef_chk::s_kmax && tid >= 0 && tid < TPB, sdcef_chk::kIx))
    j = tid = 0;
#endif
  return (size_t)j * TPB + tid;
}

// Global index of row j of this thread inside the column [off, off + N).
__device__ __forceinline__ int64_t cell_ix(int64_t off, const Geo& g, int j) {
#ifdef SDCEF_CHECKS
  if (!SDCEF_CHECK(j >= 0 && g.t0 + j < g.N, sdcef_chk::kCell)) return off;
#endif
  return off + g.t0 + j;
}

// Bilinear interpolation of the mobility and diffusivity tables at table
// coordinates (tc, tx) (fractional node indices), clamped to the table; with
// dmu non-null also the slopes d/dtx of the interpolant (zero where tx is
// clamped).
__device__ __forceinline__ void tab_mu_d(const TransportTab& T, double tc, double tx, double* mu,
                                         double* D, double* dmu = nullptr, double* dD = nullptr) {
  const bool inside = tx >= 0.0 && tx <= (double)(T.nx - 1);
  tc = fmin(fmax(tc, 0.0), (double)(T.nc - 1));
  tx = fmin(fmax(tx, 0.0), (double)(T.nx - 1));
  const int ic = min((int)tc, T.nc - 2), jx = min((int)tx, T.nx - 2);
  const double wc = tc - ic, wx = tx - jx;
  const double* r0 = T.tab + (size_t)ic * T.nx + jx;
  const double* r1 = r0 + T.nx;
  const size_t dofs = (size_t)T.nc * T.nx;
  const double m00 = __ldg(r0), m01 = __ldg(r0 + 1), m10 = __ldg(r1), m11 = __ldg(r1 + 1);
  const double d00 = __ldg(r0 + dofs), d01 = __ldg(r0 + dofs + 1), d10 = __ldg(r1 + dofs),
               d11 = __ldg(r1 + dofs + 1);
  *mu = (1.0 - wc) * ((1.0 - wx) * m00 + wx * m01) + wc * ((1.0 - wx) * m10 + wx * m11);
  *D = (1.0 - wc) * ((1.0 - wx) * d00 + wx * d01) + wc * ((1.0 - wx) * d10 + wx * d11);
  if (dmu) {
    *dmu = inside ? (1.0 - wc) * (m01 - m00) + wc * (m11 - m10) : 0.0;
    *dD = inside ? (1.0 - wc) * (d01 - d00) + wc * (d11 - d10) : 0.0;
  }
}

// The multigrid region follows the slot's planes (SDCEF_PREC_MG only).
template <int TPB, typename KR, typename PR>
__device__ __forceinline__ MgArea mg_slot_area(const Slot<TPB, KR, PR>& S) {
  return mg_area((double*)((char*)S.d + slot_bytes_for<KR, PR>(S.PL, S.m, TPB)), S.PL);
}

// --------------------------------------------------------------------------
// Residual F(X) of Eq. nls on (n, psi), phi = phi_ref + psi.
// State of local row j: n = nb[j] + cn * dn[j], psi = pb[j] + cp * dp[j]
// (dn/dp may be null). Output modes:
//   OUT_F:   write F to (fe_o, fp_o), face derivative set `fs`, electrode
//            velocities; returns raw max|F_e|, max|F_phi|, sum F_e^2, sum F_phi^2
//   OUT_JVP: w = (F - F_ref) / (eps S_F) into Krylov planes (we, wp)
// --------------------------------------------------------------------------
enum { OUT_F = 0, OUT_JVP = 1 };

template <int TPB, typename KR, typename PR, int VAR>
__device__ __noinline__ void residual(const KArgs& a, const Geo& g, ColShared& cs, const Slot<TPB, KR, PR>& S,
                         const double* nb, const double* pb, const KR* dn, const KR* dp,
                         double cn, double cp, int out_mode, double* fe_o, double* fp_o, int fs,
                         const double* fe_ref, const double* fp_ref, KR* we, KR* wp, double ieps,
                         double* halo, double* red, double* norms, double* n_o = nullptr,
                         double* p_o = nullptr) {
  const int tid = g.tid, kt = g.kt, N = g.N;
  const double ih = cs.inv_h, dt = cs.dt, g0 = cs.g0, mu = a.p.mu, kap = a.p.kap;
  const double r = dt * ih;
  // the face derivatives are stored in the Jacobian's scaled units: the n
  // derivatives times r s_n / s_Fe, the psi derivative times r s_psi / s_Fe
  const double ra = r * cs.r_a, rbi = r * cs.r_b * ih, rbm = rbi * mu;
  // face differences dd: psi_{i+1} - psi_i (RAW, 1/h folded into PD_MUHD and the
  // Poisson constant), or the gradient dpsi/dx for the transport-table kernel
  constexpr bool RAW = VAR != kVarTable;
  const double dsc = RAW ? 1.0 : ih;              // dd -> dd as the kernel keeps it
  const double kpo = RAW ? kap * ih * ih : kap * ih;   // Poisson: kpo (dd_{i+1/2} - dd_{i-1/2})
  const double ie_e = ieps * cs.isFe, ie_p = ieps * cs.isFp;   // JVP output scaling
  const double* FEX = S.pd(PD_FEX);
  const double* FPHI = S.pd(PD_FPHI);
  const double* DH = S.pd(PD_DH);
  const double* MUHD = S.pd(PD_MUHD);
  const double* PE0 = S.pd(PD_PE0);
  double* face = S.pd(PD_FACE0 + 3 * fs);
  auto st_n = [&](int j) {
    double v = nb[ix(j, tid, TPB)];
    if (dn) v = fma(cn, (double)dn[ix(j, tid, TPB)], v);
    return v;
  };
  auto st_p = [&](int j) {
    double v = pb[ix(j, tid, TPB)];
    if (dp) v = fma(cp, (double)dp[ix(j, tid, TPB)], v);
    return v;
  };
  // 1. halo: first and last cell state of each thread
  if (kt > 0) {
    halo[0 * TPB + tid] = st_n(0);
    halo[1 * TPB + tid] = st_p(0);
    halo[2 * TPB + tid] = st_n(kt - 1);
    halo[3 * TPB + tid] = st_p(kt - 1);
  }
  __syncthreads();
  long long mxe = 0, mxp = 0;   // bit patterns of max |F_e|, max |F_phi|
  double sse = 0.0, ssp = 0.0;
  constexpr long long kAbs = 0x7FFFFFFFFFFFFFFFLL;
  double gam_left = 0.0, d_left = 0.0;   // left-face values of row 0 (thread 0 only)
  double pend_e = 0.0, pend_p = 0.0;     // row-0 partial residuals
  double gam_prev = 0.0, d_prev = 0.0, last_gam = 0.0, last_d = 0.0;
  if (kt > 0) {
    double n_i = st_n(0), p_i = st_p(0);
    if (g.t0 == 0) {
      // left electrode face: G_L - g0 = (9 psi_0 - psi_1) / (3h)
      double p1 = kt >= 2 ? st_p(1) : halo[1 * TPB + tid + 1];
      double dL = (9.0 * p_i - p1) * (dsc * (1.0 / 3.0));
      const double GL = g0 + (RAW ? dL * ih : dL);
      double muL = mu;
      if constexpr (VAR == kVarTable) {
        double Dd, dmu_x, dDd;
        const double G = GL;
        tab_mu_d(a.tt, cs.tcL, fabs(G) * cs.sxL, &muL, &Dd, &dmu_x, &dDd);
        // dv/dG = mu + G mu'(G) for the Jacobian row
        if (out_mode == OUT_F) cs.muL[fs] = fma(G, dmu_x * (G < 0.0 ? -cs.sxL : cs.sxL), muL);
      }
      double vL = cs.ubl + muL * GL;
      bool act = a.p.bc == SDCEF_BC_ZERO_GRADIENT || vL < 0.0;
      gam_left = act ? vL * n_i : 0.0;
      d_left = dL;
      if (out_mode == OUT_F) cs.vL[fs] = vL;
    }
    for (int j = 0; j < kt; ++j) {
      const int i = g.t0 + j;
      if (n_o) {   // the evaluated state, kept for the line search's accepted trial
        n_o[ix(j, tid, TPB)] = n_i;
        p_o[ix(j, tid, TPB)] = p_i;
      }
      double n_n, p_n, gam, dd;
      if (i < N - 1) {
        n_n = (j + 1 < kt) ? st_n(j + 1) : halo[0 * TPB + tid + 1];
        p_n = (j + 1 < kt) ? st_p(j + 1) : halo[1 * TPB + tid + 1];
        dd = (p_n - p_i) * dsc;
        double Pe, dh, muf;
        double dPe_dG = 0.0, dD_dG = 0.0;   // table mode, OUT_F: slopes of the interpolant
        if constexpr (VAR == kVarTable) {
          // mu, D from the tables at the face's c and E/N = |G| / N
          const double G = g0 + dd;
          const double sx = MUHD[ix(j, tid, TPB)];
          double Df;
          if (out_mode == OUT_F) {
            double dmu_x, dD_x;
            tab_mu_d(a.tt, DH[ix(j, tid, TPB)], fabs(G) * sx, &muf, &Df, &dmu_x, &dD_x);
            const double sg = G < 0.0 ? -sx : sx;   // d tx / dG
            const double dmu = dmu_x * sg;
            dD_dG = dD_x * sg;
            const double v = fma(muf, G, PE0[ix(j, tid, TPB)]);
            // dPe/dG = h ((mu + G mu') D - v D') / D^2
            dPe_dG = cs.h * (fma(G, dmu, muf) * Df - v * dD_dG) / (Df * Df);
          } else {
            tab_mu_d(a.tt, DH[ix(j, tid, TPB)], fabs(G) * sx, &muf, &Df);
          }
          Pe = fma(muf, G, PE0[ix(j, tid, TPB)]) * cs.h / Df;
          dh = Df * ih;
        } else {
          // Pe = (u_f + mu (g0 + dpsi/dx)) h / D_f = PE0 + (mu / D_f) (psi_{i+1} - psi_i)
          Pe = fma(MUHD[ix(j, tid, TPB)], dd, PE0[ix(j, tid, TPB)]);
          dh = DH[ix(j, tid, TPB)];
          muf = mu;
        }
        double aa = fabs(Pe), b, db = 0.0;
        if (out_mode == OUT_F) bern_pos<true>(aa, &b, &db);   // CTA-uniform branch
        else bern_pos<false>(aa, &b, &db);
        const bool pos = dbits(Pe) >= 0;   // sign bit clear
        const double Bp = pos ? b : aa + b, Bm = pos ? aa + b : b;   // B(Pe), B(-Pe)
        gam = dh * (Bm * n_i - Bp * n_n);
        if (out_mode == OUT_F) {
          const double dBp = pos ? db : -1.0 - db, dBm = pos ? -1.0 - db : db;
          // scaled r dGam/dn_i, r dGam/dn_{i+1} and r dGam/dpsi_{i+1}
          const double rdh = ra * dh;
          double dg_p1;
          if constexpr (VAR == kVarTable) {
            // dGam/dG = (D'/h)(B(-Pe) n_i - B(Pe) n_{i+1}) + (D/h)(-B'(-Pe) n_i - B'(Pe) n_{i+1}) dPe/dG
            const double dGam = dD_dG * ih * (Bm * n_i - Bp * n_n) +
                                dh * (-dBm * n_i - dBp * n_n) * dPe_dG;
            dg_p1 = rbi * dGam;
          } else {
            dg_p1 = rbm * (-dBm * n_i - dBp * n_n);
          }
          face[0 * a.PL + ix(j, tid, TPB)] = rdh * Bm;
          face[1 * a.PL + ix(j, tid, TPB)] = -rdh * Bp;
          face[2 * a.PL + ix(j, tid, TPB)] = dg_p1;
        }
      } else {
        // right electrode face: G_R - g0 = (-9 psi_{N-1} + psi_{N-2}) / (3h)
        double pm = (j >= 1) ? st_p(j - 1) : halo[3 * TPB + tid - 1];
        dd = (-9.0 * p_i + pm) * (dsc * (1.0 / 3.0));
        const double GR = g0 + (RAW ? dd * ih : dd);
        double muR = mu;
        if constexpr (VAR == kVarTable) {
          double Dd, dmu_x, dDd;
          const double G = GR;
          tab_mu_d(a.tt, cs.tcR, fabs(G) * cs.sxR, &muR, &Dd, &dmu_x, &dDd);
          if (out_mode == OUT_F) cs.muR[fs] = fma(G, dmu_x * (G < 0.0 ? -cs.sxR : cs.sxR), muR);
        }
        double vR = cs.ubr + muR * GR;
        bool act = a.p.bc == SDCEF_BC_ZERO_GRADIENT || vR > 0.0;
        gam = act ? vR * n_i : 0.0;
        if (out_mode == OUT_F) cs.vR[fs] = vR;
        n_n = 0.0;
        p_n = 0.0;
      }
      const double fex = FEX[ix(j, tid, TPB)], fph = FPHI[ix(j, tid, TPB)];
      double Fe, Fp;
      if (j == 0) {
        Fe = -n_i + fex - r * gam;     // + r * gam_left later
        Fp = -n_i + fph + kpo * dd;
        pend_e = Fe;
        pend_p = Fp;
      } else {
        Fe = -n_i + fex - r * (gam - gam_prev);
        Fp = -n_i + fph + kpo * (dd - d_prev);
        if (out_mode == OUT_F) {
          fe_o[ix(j, tid, TPB)] = Fe;
          fp_o[ix(j, tid, TPB)] = Fp;
          mxe = max(mxe, dbits(Fe) & kAbs);
          mxp = max(mxp, dbits(Fp) & kAbs);
          sse += Fe * Fe;
          ssp += Fp * Fp;
        } else {
          we[ix(j, tid, TPB)] = (KR)((Fe - fe_ref[ix(j, tid, TPB)]) * ie_e);
          wp[ix(j, tid, TPB)] = (KR)((Fp - fp_ref[ix(j, tid, TPB)]) * ie_p);
        }
      }
      gam_prev = gam;
      d_prev = dd;
      n_i = n_n;
      p_i = p_n;
    }
    last_gam = gam_prev;
    last_d = d_prev;
  }
  __syncthreads();   // halo reads done
  if (kt > 0) {
    halo[0 * TPB + tid] = last_gam;
    halo[1 * TPB + tid] = last_d;
  }
  __syncthreads();
  if (kt > 0) {
    if (g.t0 > 0) {
      gam_left = halo[0 * TPB + tid - 1];
      d_left = halo[1 * TPB + tid - 1];
    }
    double Fe = pend_e + r * gam_left;
    double Fp = pend_p - kpo * d_left;
    if (out_mode == OUT_F) {
      fe_o[ix(0, tid, TPB)] = Fe;
      fp_o[ix(0, tid, TPB)] = Fp;
      mxe = max(mxe, dbits(Fe) & kAbs);
      mxp = max(mxp, dbits(Fp) & kAbs);
      sse += Fe * Fe;
      ssp += Fp * Fp;
    } else {
      we[ix(0, tid, TPB)] = (KR)((Fe - fe_ref[ix(0, tid, TPB)]) * ie_e);
      wp[ix(0, tid, TPB)] = (KR)((Fp - fp_ref[ix(0, tid, TPB)]) * ie_p);
    }
  }
  if (out_mode == OUT_F) {
    double mx[2] = {__longlong_as_double(mxe), __longlong_as_double(mxp)};
    // NaN-propagating max: fmax drops NaN, so fold non-finite into +inf
    if (!(mx[0] <= 1.79e308)) mx[0] = INFINITY;
    if (!(mx[1] <= 1.79e308)) mx[1] = INFINITY;
    block_reduce<TPB>(mx, 2, true, red);
    double ss[2] = {sse, ssp};
    block_reduce<TPB>(ss, 2, false, red);
    norms[0] = mx[0];
    norms[1] = mx[1];
    norms[2] = ss[0];
    norms[3] = ss[1];
  } else {
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Scaled Jacobian row blocks (Eq. linear_nls), built from the stored face
// derivatives of face set fs. Unknown order per cell: (n, psi).
//   A = dF_e/dn, B = dF_e/dpsi, C = dF_phi/dn = -I, L = dF_phi/dpsi,
// scaled: Ahat = A s_n/s_Fe, Bhat = B s_phi/s_Fe, Chat = -s_n/s_Fphi, Lhat = L s_phi/s_Fphi.
// --------------------------------------------------------------------------
struct RowJ {
  double As, Ad, Au, Bs, Bd, Bu, Ls, Ld, Lu, C;
};

template <int TPB, typename KR, typename PR, int VAR>
__device__ __forceinline__ RowJ jac_row(const KArgs& a, const Geo& g, const ColShared& cs,
                                        const Slot<TPB, KR, PR>& S, int fs, int j,
                                        const double* lf /*left face's 3 derivatives*/,
                                        const double* rf /*right face's 3 derivatives*/,
                                        double n_0, double n_last) {
  const int i = g.t0 + j, N = g.N;
  const double ih = cs.inv_h, r = cs.dt * ih, mu = a.p.mu;
  RowJ R;
  R.As = R.Au = R.Bs = R.Bu = 0.0;
  const double sa = cs.r_a, sb = cs.r_b;
  R.Ad = -sa;
  R.Bd = 0.0;
  R.C = -cs.r_c;
  // right face (row i carries -r Gam_{i+1/2})
  if (i < N - 1) {
    R.Ad -= rf[0];
    R.Au -= rf[1];
    const double t = rf[2];   // dGam/dpsi_i = -dGam/dpsi_{i+1}
    R.Bd += t;
    R.Bu -= t;
  } else {
    double vR = cs.vR[fs];
    double muR = mu;
    if constexpr (VAR == kVarTable) muR = cs.muR[fs];
    if (a.p.bc == SDCEF_BC_ZERO_GRADIENT || vR > 0.0) {
      R.Ad -= r * vR * sa;
      R.Bd -= r * n_last * muR * (-3.0 * ih) * sb;
      R.Bs -= r * n_last * muR * (ih * (1.0 / 3.0)) * sb;
    }
  }
  // left face (row i carries +r Gam_{i-1/2})
  if (i > 0) {
    R.As += lf[0];
    R.Ad += lf[1];
    const double t = lf[2];
    R.Bs -= t;
    R.Bd += t;
  } else {
    double vL = cs.vL[fs];
    double muL = mu;
    if constexpr (VAR == kVarTable) muL = cs.muL[fs];
    if (a.p.bc == SDCEF_BC_ZERO_GRADIENT || vL < 0.0) {
      R.Ad += r * vL * sa;
      R.Bd += r * n_0 * muL * (3.0 * ih) * sb;
      R.Bu += r * n_0 * muL * (-ih * (1.0 / 3.0)) * sb;
    }
  }
  // Poisson stencil with the second-order electrode closure
  if (i == 0) {
    R.Ls = 0.0;
    R.Ld = cs.m4kh2;
    R.Lu = cs.kh2_43;
  } else if (i == N - 1) {
    R.Ls = cs.kh2_43;
    R.Ld = cs.m4kh2;
    R.Lu = 0.0;
  } else {
    R.Ls = cs.kh2;
    R.Ld = cs.m2kh2;
    R.Lu = cs.kh2;
  }
  return R;
}

// --------------------------------------------------------------------------
// Preconditioner: factorisation and application (scaled units).
// --------------------------------------------------------------------------
template <int TPB, typename KR, typename PR, int VAR>
__device__ __noinline__ void prec_factor(const KArgs& a, const Geo& g, ColShared& cs, const Slot<TPB, KR, PR>& S,
                            int fs, PR* sh, double* halo, bool* bad) {
  const int tid = g.tid, kt = g.kt;
  // left-face derivatives of each thread's first row = previous thread's last face
  if (kt > 0) {
    const double* face = S.pd(PD_FACE0 + 3 * fs);
#pragma unroll
    for (int q = 0; q < 3; ++q) halo[q * TPB + tid] = face[q * a.PL + ix(kt - 1, tid, TPB)];
  }
  __syncthreads();
  double lf0[3] = {0, 0, 0};
  if (kt > 0 && tid > 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) lf0[q] = halo[q * TPB + tid - 1];
  }
  const double* NP = S.pd(pd_n(fs));
  const double n0 = (g.t0 == 0 && kt > 0) ? NP[ix(0, tid, TPB)] : 0.0;
  const double nlast = (kt > 0 && g.t0 + kt == g.N) ? NP[ix(kt - 1, tid, TPB)] : 0.0;
  const double* face = S.pd(PD_FACE0 + 3 * fs);
  // the left and right faces' derivatives of row j; rows come in order, so the
  // right face of row j - 1 is carried over as the left face of row j
  double cf[3] = {0.0, 0.0, 0.0};
  int cj = -2;
  auto faces = [&](int j, double* lf, double* rf) {
    if (j == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) lf[q] = lf0[q];
    } else if (j == cj + 1) {
#pragma unroll
      for (int q = 0; q < 3; ++q) lf[q] = cf[q];
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) lf[q] = face[q * a.PL + ix(j - 1, tid, TPB)];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      rf[q] = face[q * a.PL + ix(j, tid, TPB)];
      cf[q] = rf[q];
    }
    cj = j;
  };
  if (a.p.precond == SDCEF_PREC_EXACT) {
    Planes<2, PR, TPB> F{S.f, S.PL};
    Scal<2, PR, TPB> Sc{S.s};
    auto rowf = [&](int j, Mat<2, PR>& M, Mat<2, PR>& D, Mat<2, PR>& U) {
      double lf[3], rf[3];
      faces(j, lf, rf);
      RowJ R = jac_row<TPB, KR, PR, VAR>(a, g, cs, S, fs, j, lf, rf, n0, nlast);
      M.a[0] = conv<PR>(R.As); M.a[1] = conv<PR>(R.Bs); M.a[2] = PR(0); M.a[3] = conv<PR>(R.Ls);
      D.a[0] = conv<PR>(R.Ad); D.a[1] = conv<PR>(R.Bd); D.a[2] = conv<PR>(R.C); D.a[3] = conv<PR>(R.Ld);
      U.a[0] = conv<PR>(R.Au); U.a[1] = conv<PR>(R.Bu); U.a[2] = PR(0); U.a[3] = conv<PR>(R.Lu);
    };
    part_factor<2, PR, TPB, true>(F, Sc, kt, tid, g.tact, rowf, sh, bad);
  } else if (a.p.precond == SDCEF_PREC_RECAST) {
    // system 1: Ahat; system 2: S~hat = Lhat - (s_Fe/s_Fphi) Bhat; Bhat kept for the matvec
    Planes<1, PR, TPB> F1{S.f, S.PL};
    Planes<1, PR, TPB> F2{S.f + 5 * S.PL, S.PL};
    PR* Bpl = S.f + 10 * S.PL;   // 3 planes: sub, dia, sup
    Scal<1, PR, TPB> S1{S.s};
    Scal<1, PR, TPB> S2{S.s + FIdx<1>::NSCAL * TPB};
    const double rho = cs.r_rho;
    auto row1 = [&](int j, Mat<1, PR>& M, Mat<1, PR>& D, Mat<1, PR>& U) {
      double lf[3], rf[3];
      faces(j, lf, rf);
      RowJ R = jac_row<TPB, KR, PR, VAR>(a, g, cs, S, fs, j, lf, rf, n0, nlast);
      M.a[0] = conv<PR>(R.As); D.a[0] = conv<PR>(R.Ad); U.a[0] = conv<PR>(R.Au);
      Bpl[0 * S.PL + ix(j, tid, TPB)] = conv<PR>(R.Bs);
      Bpl[1 * S.PL + ix(j, tid, TPB)] = conv<PR>(R.Bd);
      Bpl[2 * S.PL + ix(j, tid, TPB)] = conv<PR>(R.Bu);
    };
    part_factor<1, PR, TPB, false>(F1, S1, kt, tid, g.tact, row1, sh, bad);
    auto row2 = [&](int j, Mat<1, PR>& M, Mat<1, PR>& D, Mat<1, PR>& U) {
      double lf[3], rf[3];
      faces(j, lf, rf);
      RowJ R = jac_row<TPB, KR, PR, VAR>(a, g, cs, S, fs, j, lf, rf, n0, nlast);
      M.a[0] = conv<PR>(R.Ls - rho * R.Bs);
      D.a[0] = conv<PR>(R.Ld - rho * R.Bd);
      U.a[0] = conv<PR>(R.Lu - rho * R.Bu);
    };
    part_factor<1, PR, TPB, false>(F2, S2, kt, tid, g.tact, row2, sh, bad);
  } else if (a.p.precond == SDCEF_PREC_MG) {
    if constexpr (VAR == kVarMG && std::is_same<KR, double>::value && std::is_same<PR, double>::value) {
      // level 0 of both blocks in natural row order (Ahat, S~hat = Lhat - rho Bhat),
      // Bhat kept for the matvec as in the recast form
      const MgArea M = mg_slot_area(S);
      PR* Bpl = S.f + 10 * S.PL;
      const double rho = cs.r_rho;
      for (int j = 0; j < kt; ++j) {
        double lf[3], rf[3];
        faces(j, lf, rf);
        RowJ R = jac_row<TPB, KR, PR, VAR>(a, g, cs, S, fs, j, lf, rf, n0, nlast);
        const int i = g.t0 + j;
        M.op[0].sub[i] = R.As;
        M.op[0].dia[i] = R.Ad;
        M.op[0].sup[i] = R.Au;
        M.op[1].sub[i] = R.Ls - rho * R.Bs;
        M.op[1].dia[i] = R.Ld - rho * R.Bd;
        M.op[1].sup[i] = R.Lu - rho * R.Bu;
        Bpl[0 * S.PL + ix(j, tid, TPB)] = R.Bs;
        Bpl[1 * S.PL + ix(j, tid, TPB)] = R.Bd;
        Bpl[2 * S.PL + ix(j, tid, TPB)] = R.Bu;
      }
      __syncthreads();
      for (int blk = 0; blk < 2; ++blk) {
        const MgOp& T = M.op[blk];
        if ((blk == 0 ? a.p.mg_gA : a.p.mg_gS) > 0.0) {
          mg_build<TPB>(T, g.N, a.p.mg_transfer, bad);
        } else {
          // this block is solved exactly: partitioned Thomas factorisation
          Planes<1, PR, TPB> F{S.f + (size_t)(5 * blk) * S.PL, S.PL};
          Scal<1, PR, TPB> Sc{S.s + (size_t)blk * FIdx<1>::NSCAL * TPB};
          auto row = [&](int j, Mat<1, PR>& Ml, Mat<1, PR>& D, Mat<1, PR>& U) {
            const int i = g.t0 + j;
            Ml.a[0] = T.sub[i];
            D.a[0] = T.dia[i];
            U.a[0] = T.sup[i];
          };
          part_factor<1, PR, TPB, false>(F, Sc, kt, tid, g.tact, row, sh, bad);
        }
      }
    }
  }
  __syncthreads();
}

// x = T^{-1} r for block blk of the multigrid area by V-cycles (Sec. 4.2) from
// x = 0 until ||r - T x||_2 <= gamma_MG ||r||_2, the cycle cap, or a cycle that
// does not lower the residual (undone). in/out in the Krylov plane layout (may
// alias). Returns the cycles run; uniform over the CTA.
template <int TPB>
__device__ __noinline__ int mg_solve(const KArgs& a, const Geo& g, const MgArea& M, int blk,
                                     const double* in, double* out, double* red) {
  const int tid = g.tid, kt = g.kt, N = g.N;
  const MgOp& T = M.op[blk];
  const double gam = blk == 0 ? a.p.mg_gA : a.p.mg_gS;
  double s = 0.0;
  for (int j = 0; j < kt; ++j) {
    const double v = in[ix(j, tid, TPB)];
    M.b[g.t0 + j] = v;
    M.x[g.t0 + j] = 0.0;
    s = fma(v, v, s);
  }
  block_reduce<TPB>(&s, 1, false, red);
  const double nb2 = s;
  const double tol2 = gam * gam * nb2;
  const MgLev F0 = mg_lev(T, 0, N);
  double prev = nb2;
  int k = 0;
  while (nb2 > 0.0 && k < a.p.mg_maxc) {
    for (int i = tid; i < N; i += TPB) M.xp[i] = M.x[i];
    __syncthreads();
    mg_vcycle<TPB>(T, N, M.x, M.b, a.p.mg_transfer);
    ++k;
    double r2 = 0.0;
    for (int i = tid; i < N; i += TPB) {
      const double r = mg_res(F0, M.x, M.b, i);
      r2 = fma(r, r, r2);
    }
    block_reduce<TPB>(&r2, 1, false, red);
    if (!(r2 < prev)) {
      for (int i = tid; i < N; i += TPB) M.x[i] = M.xp[i];
      __syncthreads();
      break;
    }
    prev = r2;
    if (r2 <= tol2) break;
  }
  for (int j = 0; j < kt; ++j) out[ix(j, tid, TPB)] = M.x[g.t0 + j];
  __syncthreads();
  return k;
}

// z = Mhat^{-1} r (scaled units); in/out are Krylov planes (2 components each).
// Returns ||z||_2^2 (block-reduced) if want_norm.
template <int TPB, typename KR, typename PR, int VAR>
__device__ __noinline__ double prec_apply(const KArgs& a, const Geo& g, ColShared& cs,
                             const Slot<TPB, KR, PR>& S, KR* re, KR* rp, KR* ze, KR* zp, PR* sh,
                             double* red, bool want_norm) {
  const int tid = g.tid, kt = g.kt;
  double s = 0.0;                 // this thread's part of ||z||_2^2 (want_norm)
  bool have_s = false;
  if (a.p.precond == SDCEF_PREC_EXACT) {
    Planes<2, PR, TPB> F{S.f, S.PL};
    Scal<2, PR, TPB> Sc{S.s};
    KR* rin[2] = {re, rp};
    KR* out[2] = {ze, zp};
    PR* scr = S.f + (size_t)kScrPlane * S.PL;   // two planes, a row's pair contiguous
    part_solve<2, PR, KR, TPB, true>(F, Sc, rin, out, scr, kt, tid, g.tact, sh,
                                     want_norm ? &s : nullptr);
    have_s = true;
  } else if (a.p.precond == SDCEF_PREC_RECAST) {
    Planes<1, PR, TPB> F1{S.f, S.PL};
    Planes<1, PR, TPB> F2{S.f + 5 * S.PL, S.PL};
    const PR* Bpl = S.f + 10 * S.PL;
    PR* scr = S.f + (size_t)kScrPlane * S.PL;
    Scal<1, PR, TPB> S1{S.s};
    Scal<1, PR, TPB> S2{S.s + FIdx<1>::NSCAL * TPB};
    const KR cfac = (KR)cs.r_c;   // -Chat
    // z1 = Ahat^{-1} r_e (into ze)
    {
      KR* rin[1] = {re};
      KR* out[1] = {ze};
      part_solve<1, PR, KR, TPB, false>(F1, S1, rin, out, scr, kt, tid, g.tact, sh);
    }
    // z2 = S~^{-1} (r_phi - Chat z1) (into zp)
    for (int j = 0; j < kt; ++j) zp[ix(j, tid, TPB)] = rp[ix(j, tid, TPB)] + cfac * ze[ix(j, tid, TPB)];
    {
      KR* rin[1] = {zp};
      KR* out[1] = {zp};
      part_solve<1, PR, KR, TPB, false>(F2, S2, rin, out, scr, kt, tid, g.tact, sh);
    }
    // t = Bhat z2 (tridiagonal matvec with halo), then x1 = z1 - Ahat^{-1} t
    KR* tpl = S.T(0);
    {
      KR* hb = reinterpret_cast<KR*>(sh);
      if (kt > 0) {
        hb[tid] = zp[ix(0, tid, TPB)];
        hb[TPB + tid] = zp[ix(kt - 1, tid, TPB)];
      }
      __syncthreads();
      for (int j = 0; j < kt; ++j) {
        const int i = g.t0 + j;
        KR zc = zp[ix(j, tid, TPB)];
        KR zl = (i == 0) ? KR(0) : (j > 0 ? zp[ix(j - 1, tid, TPB)] : hb[TPB + tid - 1]);
        KR zr = (i == g.N - 1) ? KR(0) : (j + 1 < kt ? zp[ix(j + 1, tid, TPB)] : hb[tid + 1]);
        tpl[ix(j, tid, TPB)] = conv<KR>(Bpl[0 * S.PL + ix(j, tid, TPB)]) * zl +
                               conv<KR>(Bpl[1 * S.PL + ix(j, tid, TPB)]) * zc +
                               conv<KR>(Bpl[2 * S.PL + ix(j, tid, TPB)]) * zr;
      }
      __syncthreads();
    }
    {
      KR* rin[1] = {tpl};
      KR* out[1] = {tpl};
      part_solve<1, PR, KR, TPB, false>(F1, S1, rin, out, scr, kt, tid, g.tact, sh);
    }
    for (int j = 0; j < kt; ++j) ze[ix(j, tid, TPB)] = ze[ix(j, tid, TPB)] - tpl[ix(j, tid, TPB)];
  } else if (a.p.precond == SDCEF_PREC_MG) {
    if constexpr (VAR == kVarMG && std::is_same<KR, double>::value && std::is_same<PR, double>::value) {
      // Eq. prec_recast as in the recast form, each block solve by V-cycles
      // (or exactly, where that block's tolerance is <= 0)
      const MgArea M = mg_slot_area(S);
      const PR* Bpl = S.f + 10 * S.PL;
      PR* scr = S.f + (size_t)kScrPlane * S.PL;
      auto blk_solve = [&](int blk, KR* rin_, KR* out_) {
        if ((blk == 0 ? a.p.mg_gA : a.p.mg_gS) > 0.0) {
          const int k = mg_solve<TPB>(a, g, M, blk, rin_, out_, red);
          if (tid == 0) cs.mgc += k;
        } else {
          Planes<1, PR, TPB> F{S.f + (size_t)(5 * blk) * S.PL, S.PL};
          Scal<1, PR, TPB> Sc{S.s + (size_t)blk * FIdx<1>::NSCAL * TPB};
          KR* rin[1] = {rin_};
          KR* out[1] = {out_};
          part_solve<1, PR, KR, TPB, false>(F, Sc, rin, out, scr, kt, tid, g.tact, sh);
        }
      };
      const KR cfac = (KR)cs.r_c;   // -Chat
      blk_solve(0, re, ze);                                   // z1 = Ahat^{-1} r_e
      for (int j = 0; j < kt; ++j) zp[ix(j, tid, TPB)] = rp[ix(j, tid, TPB)] + cfac * ze[ix(j, tid, TPB)];
      __syncthreads();
      blk_solve(1, zp, zp);                                   // z2 = S~^{-1}(r_phi - Chat z1)
      KR* tpl = S.T(0);
      {
        KR* hb = reinterpret_cast<KR*>(sh);
        if (kt > 0) {
          hb[tid] = zp[ix(0, tid, TPB)];
          hb[TPB + tid] = zp[ix(kt - 1, tid, TPB)];
        }
        __syncthreads();
        for (int j = 0; j < kt; ++j) {
          const int i = g.t0 + j;
          KR zc = zp[ix(j, tid, TPB)];
          KR zl = (i == 0) ? KR(0) : (j > 0 ? zp[ix(j - 1, tid, TPB)] : hb[TPB + tid - 1]);
          KR zr = (i == g.N - 1) ? KR(0) : (j + 1 < kt ? zp[ix(j + 1, tid, TPB)] : hb[tid + 1]);
          tpl[ix(j, tid, TPB)] = Bpl[0 * S.PL + ix(j, tid, TPB)] * zl +
                                 Bpl[1 * S.PL + ix(j, tid, TPB)] * zc +
                                 Bpl[2 * S.PL + ix(j, tid, TPB)] * zr;
        }
        __syncthreads();
      }
      blk_solve(0, tpl, tpl);                                 // Ahat^{-1} Bhat z2
      for (int j = 0; j < kt; ++j) ze[ix(j, tid, TPB)] = ze[ix(j, tid, TPB)] - tpl[ix(j, tid, TPB)];
    }
  } else {
    for (int j = 0; j < kt; ++j) {
      ze[ix(j, tid, TPB)] = re[ix(j, tid, TPB)];
      zp[ix(j, tid, TPB)] = rp[ix(j, tid, TPB)];
    }
  }
  double nz = 0.0;
  if (want_norm) {
    if (!have_s)
      for (int j = 0; j < kt; ++j) {
        double x = ze[ix(j, tid, TPB)], y = zp[ix(j, tid, TPB)];
        s += x * x + y * y;
      }
    block_reduce<TPB>(&s, 1, false, red);
    nz = s;
  } else {
    __syncthreads();
  }
  return nz;
}

// --------------------------------------------------------------------------
// Column set-up: inputs into the slot, scaling, initial state.
// Returns false if the column is rejected (BAD_INPUT).
// --------------------------------------------------------------------------
// Krylov pointer table of the column. Pairs go on chip in the order W, V_0,
// ZK_0, Z, XH, V_1, ZK_1, ..., V_{m-1}, ZK_{m-1}, V_m, T (the vectors of a
// one-iteration GMRES solve and of the error test first) while they fit the
// region, a plane there holding the column's K * TPB elements; the others stay
// at their slot planes. All threads call it after column_setup.
template <int TPB, typename KR, typename PR>
__device__ void krylov_table(const KArgs& a, const Geo& g, const Slot<TPB, KR, PR>& S,
                             unsigned char* smem_raw) {
  const int m = S.m, npair = 2 * m + 5;
  const size_t PLs = (size_t)g.K * TPB;
  const int nks = (int)min((size_t)npair, (size_t)a.arena_bytes / (2 * PLs * sizeof(KR)));
  KR* ks = reinterpret_cast<KR*>(smem_raw + a.arena_off);
  for (int e = g.tid; e < 2 * npair; e += TPB) {
    const int pos = e >> 1, comp = e & 1;
    int r;   // on-chip rank of slot position pos
    if (pos == 0) r = 1;                        // V_0
    else if (pos <= m) r = 2 * pos + 3;         // V_1 .. V_m
    else if (pos == m + 1) r = 0;               // W
    else if (pos == m + 2) r = 3;               // Z
    else if (pos == m + 3) r = 4;               // XH
    else if (pos == m + 4) r = 2 * m + 4;       // T
    else r = pos == m + 5 ? 2 : 2 * (pos - m - 5) + 4;   // ZK_i
    s_kptr[e] = r < nks ? static_cast<void*>(ks + (size_t)(2 * r + comp) * PLs)
                        : static_cast<void*>(S.k + (size_t)(2 * pos + comp) * S.PL);
  }
  __syncthreads();
}

template <int TPB, typename KR, typename PR, int VAR>
__device__ __noinline__ bool column_setup(const KArgs& a, Geo& g, ColShared& cs, const Slot<TPB, KR, PR>& S,
                             double* halo, double* red) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    int64_t off = a.col_off[cs.col];
    int64_t N = a.col_off[cs.col + 1] - off;
    cs.off = off;
    int bad = 0;
    if (N < 2 || N > a.max_col_cells) bad = 1;
    double L = a.length[cs.col], dt = a.dt[cs.col];
    if (!(L > 0.0) || !isfinite(L) || !(dt > 0.0) || !isfinite(dt)) bad = 1;
    double vl = a.vl[cs.col], vr = a.vr[cs.col];
    if (!isfinite(vl) || !isfinite(vr)) bad = 1;
    int Ni = bad ? 2 : (int)N;
    cs.N = Ni;
    cs.K = (Ni + TPB - 1) / TPB;
    cs.tact = (Ni + cs.K - 1) / cs.K;
    cs.h = L / Ni;
    cs.inv_h = 1.0 / cs.h;
    cs.dt = dt;
    cs.vl = vl;
    cs.vr = vr;
    cs.g0 = (vr - vl) / (Ni * cs.h);
    cs.dpref = (vr - vl) / Ni;
    cs.pref0 = fma(0.5, cs.dpref, vl);
    for (int sp = 0; sp < a.nsp; ++sp) cs.vald[sp] = (double)a.val[sp];
    cs.bad = bad;
    cs.N = bad ? 0 : Ni;
    cs.mgc = 0;
  }
  __syncthreads();
  if (cs.bad) return false;
  g.tid = tid;
  g.N = cs.N;
  g.K = cs.K;
  g.tact = cs.tact;
  g.t0 = tid * g.K;
  g.kt = max(0, min(g.K, g.N - g.t0));
  const int64_t off = cs.off;
  const int64_t ncell_tot = a.col_off[a.ncol];
  double* NP = S.pd(PD_N);
  double* PP = S.pd(PD_PSI);
  double* FEX = S.pd(PD_FEX);
  double* FPHI = S.pd(PD_FPHI);
  double* DH = S.pd(PD_DH);
  double* MUHD = S.pd(PD_MUHD);
  double* UF = S.pd(PD_PE0);   // cell velocities first, then the face Peclet offsets
  const double mu = a.p.mu;
  // finiteness tests and maxima of |x| on the bit patterns (integer pipe):
  // |x| orders like its bit pattern, and NaN/Inf have the all-ones exponent
  constexpr long long kAbs = 0x7FFFFFFFFFFFFFFFLL, kExp = 0x7FF0000000000000LL;
  auto nonfinite = [&](double x) { return (dbits(x) & kExp) == kExp; };
  int bad = 0;
  long long m_n = 0, m_fphi = 0, m_phi = 0, m_fe = 0;
  // D at this thread's first cell, for the neighbour's last face
  for (int j = 0; j < g.kt; ++j) {
    const int64_t gi = cell_ix(off, g, j);
    double T = a.T[gi];
    if (dbits(T) <= 0 || nonfinite(T)) bad = 1;   // T <= 0 (incl. -0), NaN or Inf
    double D = mu * (kKb / kQe) * T;
    if constexpr (VAR == kVarTable) {
      // progress variable and gas number density in place of D
      const double rh = a.rho[gi];
      if (!(rh > 0.0) || nonfinite(rh)) bad = 1;
      D = fmin(fmax((T - a.tt.T_in) * a.tt.inv_dT, 0.0), 1.0);
      const double Ng = rh * (kNA / a.tt.gas_W);
      MUHD[ix(j, tid, TPB)] = Ng;
      if (j == 0) halo[2 * TPB + tid] = Ng;
      const double sx = (double)(a.tt.nx - 1) / (a.tt.en_max_td * 1e-21 * Ng);
      if (g.t0 + j == 0) {
        cs.tcL = D * (a.tt.nc - 1);
        cs.sxL = sx;
      }
      if (g.t0 + j == g.N - 1) {
        cs.tcR = D * (a.tt.nc - 1);
        cs.sxR = sx;
      }
    }
    if (j == 0) halo[tid] = D;
    if (a.u && j == 0) halo[TPB + tid] = a.u[gi];
    double neo = a.ne_old[gi], pho = a.phi_old[gi];
    double fe = neo + (a.ire ? cs.dt * a.ire[gi] : 0.0);
    double q = 0.0;
    for (int s = 0; s < a.nsp; ++s) q = fma(cs.vald[s], a.n_ion[(int64_t)s * ncell_tot + gi], q);
    double n0 = a.ne_g ? a.ne_g[gi] : neo;
    double p0 = a.phi_g ? a.phi_g[gi] : pho;
    if (nonfinite(neo) || nonfinite(pho) || nonfinite(fe) || nonfinite(q) || nonfinite(n0) ||
        nonfinite(p0))
      bad = 1;
    FEX[ix(j, tid, TPB)] = fe;
    FPHI[ix(j, tid, TPB)] = q;
    const double pref = fma(cs.dpref, (double)(g.t0 + j), cs.pref0);
    S.pd(PD_PREF)[ix(j, tid, TPB)] = pref;
    NP[ix(j, tid, TPB)] = n0;
    PP[ix(j, tid, TPB)] = p0 - pref;
    // face D (right face) stored temporarily as D_i; fixed below
    DH[ix(j, tid, TPB)] = D;
    if (a.u) UF[ix(j, tid, TPB)] = a.u[gi];
    m_n = max(m_n, dbits(neo) & kAbs);
    m_fphi = max(m_fphi, dbits(q) & kAbs);
    m_phi = max(m_phi, dbits(pho) & kAbs);
    m_fe = max(m_fe, dbits(fe) & kAbs);
  }
  __syncthreads();
  for (int j = 0; j < g.kt; ++j) {
    const int i = g.t0 + j;
    if (i < g.N - 1) {
      double Dn = (j + 1 < g.kt) ? DH[ix(j + 1, tid, TPB)] : halo[tid + 1];
      double Df = 0.5 * (DH[ix(j, tid, TPB)] + Dn);
      double uf = 0.0;
      if (a.u) {
        double un = (j + 1 < g.kt) ? UF[ix(j + 1, tid, TPB)] : halo[TPB + tid + 1];
        uf = 0.5 * (UF[ix(j, tid, TPB)] + un);
      }
      if constexpr (VAR == kVarTable) {
        // table coordinates of the face: c index, |G| -> E/N index factor; face velocity
        const double Nn = (j + 1 < g.kt) ? MUHD[ix(j + 1, tid, TPB)] : halo[2 * TPB + tid + 1];
        const double Nf = 0.5 * (MUHD[ix(j, tid, TPB)] + Nn);
        DH[ix(j, tid, TPB)] = Df * (a.tt.nc - 1);
        MUHD[ix(j, tid, TPB)] = (double)(a.tt.nx - 1) / (a.tt.en_max_td * 1e-21 * Nf);
        UF[ix(j, tid, TPB)] = uf;
      } else {
        const double hd = cs.h / Df;
        DH[ix(j, tid, TPB)] = Df * cs.inv_h;
        MUHD[ix(j, tid, TPB)] = mu / Df;
        UF[ix(j, tid, TPB)] = (uf + mu * cs.g0) * hd;
      }
    }
  }
  if (tid == 0) cs.ubl = a.u ? a.u[off] : 0.0;
  if (g.kt > 0 && g.t0 + g.kt == g.N) cs.ubr = a.u ? a.u[off + g.N - 1] : 0.0;
  double mx[5] = {__longlong_as_double(m_n), __longlong_as_double(m_fphi), __longlong_as_double(m_phi),
                  __longlong_as_double(m_fe), (double)bad};
  block_reduce<TPB>(mx, 5, true, red);
  if (mx[4] != 0.0) return false;
  if (tid == 0) {
    cs.sn = fmax(fmax(mx[0], mx[1]), 1.0);
    cs.sp = fmax(fmax(mx[2], fmax(fabs(cs.vl), fabs(cs.vr))), 1.0);
    cs.scal[0] = mx[3];
    cs.scal[1] = mx[1];
  }
  __syncthreads();
  return true;
}

// --------------------------------------------------------------------------
// Error test at the stop (eps_E > 0). Sec. 3.2 asks that the tolerances keep
// the solution error of the nonlinear system small; the residual test bounds
// that error only through the conditioning of S_F^-1 J S_X, which is large for
// columns whose potential scale (a few volts) is small beside their space
// charge. The Newton correction ehat = Mhat^-1 Fhat of the current factors (the
// last Newton step's, with the exact Schur form P = J) estimates the scaled
// error of the iterate. True if max|s_n ehat_n| <= eps_E max|n| and
// max|s_phi ehat_phi| <= eps_E max|phi| over the column, or if the estimate is
// not finite (no estimate: the residual test alone decides). Returns 0 (fails),
// 1 (passes) or 2 (passes within a factor kErrMargin of the bar: from a
// supplied start an estimate on factors of the previous iterate is then taken
// again at X^(l), since the change of J over a large last step, as a learned
// start can end with, can misjudge it; from X^n the last step is small).
// --------------------------------------------------------------------------
template <int TPB, typename KR, typename PR, int VAR>
__device__ __noinline__ int error_test(const KArgs& a, const Geo& g, ColShared& cs,
                                        const Slot<TPB, KR, PR>& S, int cur, PR* sh,
                                        double* red) {
  const int tid = g.tid, kt = g.kt;
  const double* Fe = S.pd(PD_FE0 + 2 * cur);
  const double* Fp = S.pd(PD_FP0 + 2 * cur);
  const double* NP = S.pd(pd_n(cur));
  const double* PP = S.pd(pd_psi(cur));
  const double* PR_ = S.pd(PD_PREF);
  KR* re = S.W(0);
  KR* rp = S.W(1);
  for (int j = 0; j < kt; ++j) {
    re[ix(j, tid, TPB)] = (KR)(Fe[ix(j, tid, TPB)] * cs.isFe);
    rp[ix(j, tid, TPB)] = (KR)(Fp[ix(j, tid, TPB)] * cs.isFp);
  }
  __syncthreads();
  prec_apply<TPB, KR, PR, VAR>(a, g, cs, S, re, rp, S.Z(0), S.Z(1), sh, red, false);
  // maxima of |.| on the bit patterns (integer pipe): non-negative doubles
  // order as their patterns; a NaN counts as 0, as fmax would ignore it
  auto absb = [](double x) {
    const long long b = dbits(x) & 0x7FFFFFFFFFFFFFFFLL;
    return b > 0x7FF0000000000000LL ? 0LL : b;
  };
  long long m[4] = {0, 0, 0, 0};
  for (int j = 0; j < kt; ++j) {
    m[0] = max(m[0], absb((double)S.Z(0)[ix(j, tid, TPB)]));
    m[1] = max(m[1], absb((double)S.Z(1)[ix(j, tid, TPB)]));
    m[2] = max(m[2], absb(NP[ix(j, tid, TPB)]));
    m[3] = max(m[3], absb(PP[ix(j, tid, TPB)] + PR_[ix(j, tid, TPB)]));
  }
  double v[4];
  for (int q = 0; q < 4; ++q) v[q] = __longlong_as_double(m[q]);
  block_reduce<TPB>(v, 4, true, red);
  const double en = v[0] * cs.sn, ep = v[1] * cs.sp;
  if (!(en <= 1.79e308) || !(ep <= 1.79e308)) return 1;
  if (!(en <= a.p.eps_E * v[2] && ep <= a.p.eps_E * v[3])) return 0;
  const double lo = a.p.eps_E * (1.0 / kErrMargin);
  return (en > lo * v[2] || ep > lo * v[3]) ? 2 : 1;
}

// --------------------------------------------------------------------------
// The persistent solver kernel.
// --------------------------------------------------------------------------
// VAR: kVarBase, kVarMG (the multigrid preconditioner, SDCEF_PREC_MG) or
// kVarTable (transport tables, SDCEF_TRANSPORT_TABLE).
template <int TPB, typename KR, typename PR, int VAR>
__global__ void __launch_bounds__(TPB, VAR == kVarBase ? 512 / TPB : 1) jfnk_kernel(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ColShared cs;
  constexpr int NW = TPB / 32;
  double* red = (double*)smem_raw;                          // (NW+1) * 40
  double* halo = red + (NW + 1) * 40;                       // 4 * TPB
  double* Hm = halo + 4 * TPB;                              // (m+1) * m Hessenberg
  const int m = a.p.m;
  double* gv = Hm + (m + 1) * m;                            // m+1
  double* cs_ = gv + (m + 1);                               // m
  double* sn_ = cs_ + m;                                    // m
  double* yv = sn_ + m;                                     // m
  double* hv = yv + m;                                      // m+2 scratch
  PR* sh = (PR*)(hv + m + 2);                               // 12 * TPB (PCR / exchange)
  const int tid = threadIdx.x;
#ifdef SDCEF_CHECKS
  if (tid == 0) {
    sdcef_chk::s_word = a.chk;
    sdcef_chk::s_kmax = a.kmax;
  }
  __syncthreads();
#endif
  Slot<TPB, KR, PR> S = make_slot<TPB, KR, PR>(a, blockIdx.x);

  for (;;) {
    if (tid == 0) {
      int q = atomicAdd(a.queue, 1);
      cs.col = (q < a.ncol) ? (a.order ? a.order[q] : q) : -1;
      if (q < a.ncol && !SDCEF_CHECK(cs.col >= 0 && cs.col < a.ncol, sdcef_chk::kCol)) cs.col = -1;
    }
    __syncthreads();
    if (cs.col < 0) break;
    Geo g;
    bool ok = column_setup<TPB, KR, PR, VAR>(a, g, cs, S, halo, red);
    const int64_t col = cs.col;
    if (!ok) {
      if (tid == 0) {
        if (a.mode == MODE_SOLVE) {
          if (a.status) a.status[col] = SDCEF_STATUS_BAD_INPUT;
          if (a.newton_it) a.newton_it[col] = 0;
          if (a.krylov_it) a.krylov_it[col] = 0;
          if (a.res_evals) a.res_evals[col] = 0;
          if (a.mg_cycles) a.mg_cycles[col] = 0;
          if (a.final_res) a.final_res[col] = NAN;
        }
      }
      // copy the start state through so outputs are defined
      int64_t off = a.col_off[col], N = a.col_off[col + 1] - off;
      if (a.mode == MODE_SOLVE)
        for (int64_t i = tid; i < N; i += TPB) {
          double n0 = a.ne_g ? a.ne_g[off + i] : a.ne_old[off + i];
          double p0 = a.phi_g ? a.phi_g[off + i] : a.phi_old[off + i];
          a.ne_out[off + i] = n0;
          a.phi_out[off + i] = p0;
        }
      __syncthreads();
      continue;
    }
    krylov_table<TPB, KR, PR>(a, g, S, smem_raw);
    const int kt = g.kt;
    const int64_t off = cs.off;
    double* NP = S.pd(PD_N);
    double* PP = S.pd(PD_PSI);
    double norms[4];
    int res_evals = 0;

    // ---- test modes -------------------------------------------------------
    if (a.mode == MODE_RESIDUAL) {
      for (int j = 0; j < kt; ++j) {
        const int64_t gi = cell_ix(off, g, j);
        const double pref = S.pd(PD_PREF)[ix(j, tid, TPB)];
        NP[ix(j, tid, TPB)] = a.x_ne[gi];
        PP[ix(j, tid, TPB)] = a.x_phi[gi] - pref;
      }
      if (tid == 0) { cs.sFe = 1.0; cs.sFp = 1.0; cs.r_a = 1.0; cs.r_b = 1.0; }
      __syncthreads();
      residual<TPB, KR, PR, VAR>(a, g, cs, S, NP, PP, nullptr, nullptr, 0, 0, OUT_F, S.pd(PD_FE0),
                        S.pd(PD_FP0), 0, nullptr, nullptr, nullptr, nullptr, 0, halo, red, norms);
      for (int j = 0; j < kt; ++j) {
        const int64_t gi = cell_ix(off, g, j);
        a.o1[gi] = S.pd(PD_FE0)[ix(j, tid, TPB)];
        a.o2[gi] = S.pd(PD_FP0)[ix(j, tid, TPB)];
      }
      __syncthreads();
      continue;
    }

    // scaling: typical values at the plain start X^n (Eq. newton_sc, Algorithm 2
    // first line), whatever the Newton start is
    const bool start_differs = (a.mode == MODE_PRECOND) || a.ne_g || a.phi_g;
    if (tid == 0) { cs.sFe = 1.0; cs.sFp = 1.0; cs.r_a = 1.0; cs.r_b = 1.0; }
    if (start_differs) {
      double* tn = S.pd(PD_FE1);
      double* tp = S.pd(PD_FP1);
      for (int j = 0; j < kt; ++j) {
        const int64_t gi = cell_ix(off, g, j);
        const double pref = S.pd(PD_PREF)[ix(j, tid, TPB)];
        tn[ix(j, tid, TPB)] = a.ne_old[gi];
        tp[ix(j, tid, TPB)] = a.phi_old[gi] - pref;
      }
      __syncthreads();
      residual<TPB, KR, PR, VAR>(a, g, cs, S, tn, tp, nullptr, nullptr, 0, 0, OUT_F, S.pd(PD_FE0),
                        S.pd(PD_FP0), 0, nullptr, nullptr, nullptr, nullptr, 0, halo, red, norms);
    } else {
      __syncthreads();
      residual<TPB, KR, PR, VAR>(a, g, cs, S, NP, PP, nullptr, nullptr, 0, 0, OUT_F, S.pd(PD_FE0),
                        S.pd(PD_FP0), 0, nullptr, nullptr, nullptr, nullptr, 0, halo, red, norms);
    }
    ++res_evals;
    double norms_n[4] = {norms[0], norms[1], norms[2], norms[3]};   // F at X^n
    if (tid == 0) {
      cs.sFe = fmax(fmax(norms[0], cs.scal[0]), 1e-12 * cs.sn);
      cs.sFp = fmax(fmax(norms[1], cs.scal[1]), 1e-12 * cs.sn);
      if (!(cs.sFe <= 1.79e308)) cs.sFe = 1.0;
      if (!(cs.sFp <= 1.79e308)) cs.sFp = 1.0;
      cs.isn = 1.0 / cs.sn;
      cs.isp = 1.0 / cs.sp;
      cs.isFe = 1.0 / cs.sFe;
      cs.isFp = 1.0 / cs.sFp;
      cs.r_a = cs.sn / cs.sFe;
      cs.r_b = cs.sp / cs.sFe;
      cs.r_c = cs.sn / cs.sFp;
      cs.r_l = cs.sp / cs.sFp;
      cs.r_rho = cs.sFe / cs.sFp;
      cs.kh2 = a.p.kap * cs.inv_h * cs.inv_h * cs.r_l;
      cs.m2kh2 = -2.0 * cs.kh2;
      cs.m4kh2 = -4.0 * cs.kh2;
      cs.kh2_43 = (4.0 / 3.0) * cs.kh2;
      cs.have_prec = 0;
      cs.polished = 0;
    }
    if (start_differs) {
      if (a.mode == MODE_PRECOND) {
        for (int j = 0; j < kt; ++j) {
          const int64_t gi = cell_ix(off, g, j);
          const double pref = S.pd(PD_PREF)[ix(j, tid, TPB)];
          NP[ix(j, tid, TPB)] = a.x_ne[gi];
          PP[ix(j, tid, TPB)] = a.x_phi[gi] - pref;
        }
      }
      __syncthreads();
      residual<TPB, KR, PR, VAR>(a, g, cs, S, NP, PP, nullptr, nullptr, 0, 0, OUT_F, S.pd(PD_FE0),
                        S.pd(PD_FP0), 0, nullptr, nullptr, nullptr, nullptr, 0, halo, red, norms);
      ++res_evals;
    } else {
      // the face derivatives at X^n were stored before the scales were known
      __syncthreads();
      const double fa = cs.r_a, fb = cs.r_b;
      double* f0 = S.pd(PD_FACE0);
      for (int j = 0; j < kt; ++j) {
        f0[0 * a.PL + ix(j, tid, TPB)] *= fa;
        f0[1 * a.PL + ix(j, tid, TPB)] *= fa;
        f0[2 * a.PL + ix(j, tid, TPB)] *= fb;
      }
    }
    __syncthreads();
    int cur = 0;   // current F / face set
    bool bad = false;

    if (a.mode == MODE_PRECOND) {
      prec_factor<TPB, KR, PR, VAR>(a, g, cs, S, cur, sh, halo, &bad);
      // r (physical) -> rhat = r / S_F -> z = Mhat^{-1} rhat -> x = S_X z
      KR* re = S.W(0);
      KR* rp = S.W(1);
      for (int j = 0; j < kt; ++j) {
        const int64_t gi = cell_ix(off, g, j);
        re[ix(j, tid, TPB)] = (KR)(a.r_e[gi] * cs.isFe);
        rp[ix(j, tid, TPB)] = (KR)(a.r_phi[gi] * cs.isFp);
      }
      __syncthreads();
      prec_apply<TPB, KR, PR, VAR>(a, g, cs, S, re, rp, S.Z(0), S.Z(1), sh, red, false);
      for (int j = 0; j < kt; ++j) {
        const int64_t gi = cell_ix(off, g, j);
        a.o1[gi] = (double)S.Z(0)[ix(j, tid, TPB)] * cs.sn;
        a.o2[gi] = (double)S.Z(1)[ix(j, tid, TPB)] * cs.sp;
      }
      if (tid == 0 && a.mg_cycles) a.mg_cycles[col] = cs.mgc;
      __syncthreads();
      continue;
    }

    // ---- Newton loop (Algorithm 2) ---------------------------------------
    auto scaled_inf = [&](const double* nr) { return fmax(nr[0] / cs.sFe, nr[1] / cs.sFp); };
    auto scaled_two = [&](const double* nr) {
      return sqrt(nr[2] / (cs.sFe * cs.sFe) + nr[3] / (cs.sFp * cs.sFp));
    };
    double fninf = scaled_inf(norms), fn2 = scaled_two(norms);
    int status = SDCEF_STATUS_MAX_NEWTON, newton = 0, krylov = 0;
    const double gam = a.p.gamma;
    // A supplied start is judged twice: before the first Newton step (its scaled
    // residual against the plain start's) and by the iteration itself (if it
    // has not converged within guess_cap steps). A rejected start is replaced by
    // X^n, which then gets the remaining Newton budget.
    const bool supplied = a.ne_g || a.phi_g;
    const bool guessed = supplied && a.p.guess_cap > 0;
    const bool reject = supplied && a.p.guess_ratio > 0.0 &&
                        !(fn2 <= a.p.guess_ratio * scaled_two(norms_n));
    const int n_att = (guessed || reject) ? 2 : 1;
    for (int attempt = reject ? 1 : 0; attempt < n_att; ++attempt) {
    if (attempt == 1) {
      if (tid == 0) cs.have_prec = 0;
      // restart from the plain start X^n (state set 0)
      for (int j = 0; j < kt; ++j) {
        const int64_t gi = cell_ix(off, g, j);
        S.pd(PD_N)[ix(j, tid, TPB)] = a.ne_old[gi];
        S.pd(PD_PSI)[ix(j, tid, TPB)] = a.phi_old[gi] - S.pd(PD_PREF)[ix(j, tid, TPB)];
      }
      cur = 0;
      bad = false;
      __syncthreads();
      residual<TPB, KR, PR, VAR>(a, g, cs, S, S.pd(pd_n(cur)), S.pd(pd_psi(cur)), nullptr, nullptr, 0, 0, OUT_F, S.pd(PD_FE0),
                        S.pd(PD_FP0), 0, nullptr, nullptr, nullptr, nullptr, 0, halo, red, norms);
      ++res_evals;
      fninf = scaled_inf(norms);
      fn2 = scaled_two(norms);
    }
    const int cap = (guessed && attempt == 0) ? min(a.p.guess_cap, a.p.max_newton)
                                              : a.p.max_newton - newton;
    status = SDCEF_STATUS_MAX_NEWTON;
    bool prec_cur = false;   // the factors were built at the current iterate (CTA-uniform)
    bool polish = false;     // this step serves the error test (CTA-uniform)
    const bool from_guess = supplied && attempt == 0;   // the start is the supplied one
    for (int l = 0;; ++l) {
      if (!(fninf <= 1.79e308)) { status = SDCEF_STATUS_NONFINITE; break; }
      // polish: this step is taken after the residual test held, for the
      // error test (the line search reads it again). The error test and its polish steps are bounded by the Newton budget,
      // not by the cap of a supplied start: a start that passes the residual
      // test within the cap is judged like any other.
      if (fninf < a.p.eps_F) {
        if (!(a.p.eps_E > 0.0) || newton >= a.p.max_newton || cs.polished >= kMaxPolish) {
          status = SDCEF_STATUS_OK;
          break;
        }
        // (a bad pivot leaves a non-finite estimate, which passes: the residual
        // test then decides; a polish step reports it through bad)
        if (!cs.have_prec) {   // no Newton step yet: factors at X^(l)
          prec_factor<TPB, KR, PR, VAR>(a, g, cs, S, cur, sh, halo, &bad);
          prec_cur = true;
        }
        int et;
        for (;;) {   // a marginal pass on the last step's factors is taken again at X^(l)
          et = error_test<TPB, KR, PR, VAR>(a, g, cs, S, cur, sh, red);
          if (et != 2 || prec_cur || !from_guess) break;
          prec_factor<TPB, KR, PR, VAR>(a, g, cs, S, cur, sh, halo, &bad);
          prec_cur = true;
        }
        if (et != 0) {
          status = SDCEF_STATUS_OK;
          break;
        }
        polish = true;
      } else {
        polish = false;
      }
      if (l >= cap && !polish) { status = SDCEF_STATUS_MAX_NEWTON; break; }
      // preconditioner at X^(l) (unless the error test built it there) and
      // ||S_X^{-1} X||_2 (X = (n, phi))
      if (!prec_cur) prec_factor<TPB, KR, PR, VAR>(a, g, cs, S, cur, sh, halo, &bad);
      if (tid == 0) cs.have_prec = 1;
      {
        double s = 0.0;
        for (int j = 0; j < kt; ++j) {
          const double pref = S.pd(PD_PREF)[ix(j, tid, TPB)];
          double xn = S.pd(pd_n(cur))[ix(j, tid, TPB)] * cs.isn;
          double xp = (S.pd(pd_psi(cur))[ix(j, tid, TPB)] + pref) * cs.isp;
          s += xn * xn + xp * xp;
        }
        double v[2] = {s, bad ? 1.0 : 0.0};
        block_reduce<TPB>(v, 2, false, red);
        if (tid == 0) cs.xnorm = sqrt(v[0]);
        if (v[1] != 0.0) { status = SDCEF_STATUS_NONFINITE; break; }
      }
      const double* Fe = S.pd(PD_FE0 + 2 * cur);
      const double* Fp = S.pd(PD_FP0 + 2 * cur);
      // ---- GMRES(m), right-preconditioned: Jhat Mhat^{-1} y = -Fhat --------
      // With the fixed preconditioner the correction Mhat^{-1} V y is accumulated
      // from the stored z_i = Mhat^{-1} V_i (flexible-GMRES storage), which saves
      // the final preconditioner application.
      KR* XHe = S.XH(0);
      KR* XHp = S.XH(1);
      // the correction is dcoef * (DXe, DXp): y_0 z_0 in place when one Krylov
      // vector sufficed in the first cycle (the common case with the exact
      // preconditioner), else the sum accumulated in XH
      const KR* DXe = XHe;
      const KR* DXp = XHp;
      double dcoef = 1.0;
      bool first_cycle = true;
      double beta = fn2;                 // ||Fhat||_2
      const double beta0 = fn2;
      int its = 0;
      bool converged = (beta0 == 0.0);
      // V0 = -Fhat / beta
      if (!converged) {
        const double ve = -cs.isFe / beta, vp = -cs.isFp / beta;
        for (int j = 0; j < kt; ++j) {
          S.V(0, 0)[ix(j, tid, TPB)] = (KR)(Fe[ix(j, tid, TPB)] * ve);
          S.V(0, 1)[ix(j, tid, TPB)] = (KR)(Fp[ix(j, tid, TPB)] * vp);
        }
      }
      __syncthreads();
      while (!converged && its < a.p.max_krylov) {
        const double beta_cycle = beta;   // residual at the start of this cycle
        if (tid == 0) {
          for (int q = 0; q <= m; ++q) gv[q] = 0.0;
          gv[0] = beta;
        }
        __syncthreads();
        int kdim = 0;
        for (int jj = 0; jj < m && its < a.p.max_krylov; ++jj) {
          // the Arnoldi scratch below holds jj + 2 <= 34 values
          if (!SDCEF_CHECK(jj + 2 <= 34, sdcef_chk::kHess)) { bad = true; break; }
          // z_jj = Mhat^{-1} V_jj (kept), w = Jhat z_jj
          double zz = prec_apply<TPB, KR, PR, VAR>(a, g, cs, S, S.V(jj, 0), S.V(jj, 1), S.ZK(jj, 0),
                                          S.ZK(jj, 1), sh, red, true);
          double zn = sqrt(zz);
          double eps = kLambdaFD * (kLambdaFD + cs.xnorm / zn);
          if (!(zn > 0.0)) eps = 1.0;
          residual<TPB, KR, PR, VAR>(a, g, cs, S, S.pd(pd_n(cur)), S.pd(pd_psi(cur)), S.ZK(jj, 0), S.ZK(jj, 1), eps * cs.sn,
                            eps * cs.sp, OUT_JVP, nullptr, nullptr, 0, Fe, Fp, S.W(0), S.W(1),
                            1.0 / eps, halo, red, norms);
          ++res_evals;
          ++its;
          // CGS with one re-orthogonalisation. Pass 1: d = V^T w, w -= V d. Pass 2
          // reduces d2 = V^T w together with ||w||^2: the re-orthogonalised vector
          // has ||w - V d2||^2 = ||w||^2 - ||d2||^2 (V has orthonormal columns, and
          // after pass 1 d2 is small beside w), and its update below writes
          // V_{jj+1} = (w - V d2) / hn directly.
          // First basis vector: CGS2 in closed form from one pass. With d0 = V0.w,
          // the second pass gives d2 = d0 (1 - |V0|^2), so h = d0 + d2 and
          // |w - h V0|^2 = |w|^2 - 2 h d0 + h^2 |V0|^2. The subtraction cancels as
          // w nears span(V0) but errs by at most a few ulp of |w|^2, i.e. by
          // ~1e-8 |w| in hn, far below the gamma = 1e-4 test; if this step
          // converges (the common case with the exact preconditioner) V_1 is not
          // needed, else the explicit passes below run.
          if (jj == 0) {
            double v3[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < kt; ++j) {
              const double we = S.W(0)[ix(j, tid, TPB)], wp = S.W(1)[ix(j, tid, TPB)];
              const double ve = S.V(0, 0)[ix(j, tid, TPB)], vp = S.V(0, 1)[ix(j, tid, TPB)];
              v3[0] = fma(ve, we, fma(vp, wp, v3[0]));
              v3[1] = fma(we, we, fma(wp, wp, v3[1]));
              v3[2] = fma(ve, ve, fma(vp, vp, v3[2]));
            }
            block_reduce<TPB>(v3, 3, false, red);
            const double d0 = v3[0];
            const double h = fma(d0, 1.0 - v3[2], d0);
            const double hn0 = sqrt(fmax(fma(h * v3[2], h, fma(-2.0 * h, d0, v3[1])), 0.0));
            // the rotation and residual estimate exactly as the Givens step below
            const double rho = sqrt(fma(h, h, hn0 * hn0));
            const double sn0 = rho == 0.0 ? 0.0 : hn0 * (1.0 / rho);
            const double est = fabs(-sn0 * gv[0]);
            if (est <= gam * beta0 && hn0 > 0.0 && isfinite(est)) {
              if (tid == 0) {
                Hm[0] = rho;
                Hm[m] = 0.0;
                cs_[0] = h * (1.0 / rho);
                sn_[0] = sn0;
                gv[1] = -sn0 * gv[0];
                gv[0] = cs_[0] * gv[0];
              }
              __syncthreads();
              kdim = 1;
              converged = true;
              break;
            }
          }
          double hcur[34];
          {
            double d[34];
            for (int q = 0; q <= jj; ++q) d[q] = 0.0;
            for (int j = 0; j < kt; ++j) {
              double we = S.W(0)[ix(j, tid, TPB)], wp = S.W(1)[ix(j, tid, TPB)];
              for (int q = 0; q <= jj; ++q)
                d[q] += (double)S.V(q, 0)[ix(j, tid, TPB)] * we +
                        (double)S.V(q, 1)[ix(j, tid, TPB)] * wp;
            }
            block_reduce<TPB>(d, jj + 1, false, red);
            for (int j = 0; j < kt; ++j) {
              double we = S.W(0)[ix(j, tid, TPB)], wp = S.W(1)[ix(j, tid, TPB)];
              for (int q = 0; q <= jj; ++q) {
                we -= d[q] * (double)S.V(q, 0)[ix(j, tid, TPB)];
                wp -= d[q] * (double)S.V(q, 1)[ix(j, tid, TPB)];
              }
              S.W(0)[ix(j, tid, TPB)] = (KR)we;
              S.W(1)[ix(j, tid, TPB)] = (KR)wp;
            }
            for (int q = 0; q <= jj; ++q) hcur[q] = d[q];
          }
          double d2[35];
          for (int q = 0; q <= jj + 1; ++q) d2[q] = 0.0;
          for (int j = 0; j < kt; ++j) {
            double we = S.W(0)[ix(j, tid, TPB)], wp = S.W(1)[ix(j, tid, TPB)];
            for (int q = 0; q <= jj; ++q)
              d2[q] += (double)S.V(q, 0)[ix(j, tid, TPB)] * we +
                       (double)S.V(q, 1)[ix(j, tid, TPB)] * wp;
            d2[jj + 1] += we * we + wp * wp;
          }
          block_reduce<TPB>(d2, jj + 2, false, red);
          double s2 = 0.0;
          for (int q = 0; q <= jj; ++q) {
            s2 += d2[q] * d2[q];
            hcur[q] += d2[q];
          }
          const double hn = sqrt(fmax(d2[jj + 1] - s2, 0.0));
          if (tid == 0) {
            for (int q = 0; q <= jj; ++q) Hm[q * m + jj] = hcur[q];
            Hm[(jj + 1) * m + jj] = hn;
            for (int q = 0; q < jj; ++q) {
              double x0 = Hm[q * m + jj], x1 = Hm[(q + 1) * m + jj];
              Hm[q * m + jj] = cs_[q] * x0 + sn_[q] * x1;
              Hm[(q + 1) * m + jj] = -sn_[q] * x0 + cs_[q] * x1;
            }
            double x0 = Hm[jj * m + jj], x1 = Hm[(jj + 1) * m + jj];
            const double rho = sqrt(fma(x0, x0, x1 * x1));
            const double irho = 1.0 / rho;
            cs_[jj] = rho == 0.0 ? 1.0 : x0 * irho;
            sn_[jj] = rho == 0.0 ? 0.0 : x1 * irho;
            Hm[jj * m + jj] = rho;
            Hm[(jj + 1) * m + jj] = 0.0;
            gv[jj + 1] = -sn_[jj] * gv[jj];
            gv[jj] = cs_[jj] * gv[jj];
            double est = fabs(gv[jj + 1]);
            cs.conv = (est <= gam * beta0 || !(hn > 0.0) || !isfinite(est)) ? 1 : 0;
            if (!isfinite(est)) cs.conv = 2;
          }
          __syncthreads();
          kdim = jj + 1;
          const int cv = cs.conv;
          if (cv == 2) { bad = true; break; }
          if (cv) { converged = true; break; }
          if (jj + 1 < m) {
            // pass 2's update and the normalisation: V_{jj+1} = (w - V d2) / hn
            const double ihn = 1.0 / hn;
            for (int j = 0; j < kt; ++j) {
              double we = S.W(0)[ix(j, tid, TPB)], wp = S.W(1)[ix(j, tid, TPB)];
              for (int q = 0; q <= jj; ++q) {
                we -= d2[q] * (double)S.V(q, 0)[ix(j, tid, TPB)];
                wp -= d2[q] * (double)S.V(q, 1)[ix(j, tid, TPB)];
              }
              S.V(jj + 1, 0)[ix(j, tid, TPB)] = (KR)(we * ihn);
              S.V(jj + 1, 1)[ix(j, tid, TPB)] = (KR)(wp * ihn);
            }
          }
          __syncthreads();
        }
        if (bad) break;
        // y = H^{-1} g; the correction delta-hat += sum_q y_q z_q
        if (tid == 0) {
          for (int q = kdim - 1; q >= 0; --q) {
            double s = gv[q];
            for (int p2 = q + 1; p2 < kdim; ++p2) s -= Hm[q * m + p2] * yv[p2];
            yv[q] = Hm[q * m + q] != 0.0 ? s / Hm[q * m + q] : 0.0;
          }
        }
        __syncthreads();
        // ||delta-hat||^2 is needed only by a restart (its FD epsilon)
        const bool restart = !(converged || its >= a.p.max_krylov);
        if (first_cycle && !restart && kdim == 1) {
          DXe = S.ZK(0, 0);
          DXp = S.ZK(0, 1);
          dcoef = yv[0];
          first_cycle = false;
          break;
        }
        double dd = 0.0;
        for (int j = 0; j < kt; ++j) {
          double xe = first_cycle ? 0.0 : (double)XHe[ix(j, tid, TPB)];
          double xp = first_cycle ? 0.0 : (double)XHp[ix(j, tid, TPB)];
          for (int q = 0; q < kdim; ++q) {
            xe += yv[q] * (double)S.ZK(q, 0)[ix(j, tid, TPB)];
            xp += yv[q] * (double)S.ZK(q, 1)[ix(j, tid, TPB)];
          }
          XHe[ix(j, tid, TPB)] = (KR)xe;
          XHp[ix(j, tid, TPB)] = (KR)xp;
          if (restart) dd += xe * xe + xp * xp;
        }
        first_cycle = false;
        __syncthreads();
        if (!restart) break;
        // restart: r = -Fhat - Jhat delta-hat
        block_reduce<TPB>(&dd, 1, false, red);
        double zn = sqrt(dd);
        double eps = (zn > 0.0) ? kLambdaFD * (kLambdaFD + cs.xnorm / zn) : 1.0;
        residual<TPB, KR, PR, VAR>(a, g, cs, S, S.pd(pd_n(cur)), S.pd(pd_psi(cur)), XHe, XHp, eps * cs.sn, eps * cs.sp, OUT_JVP,
                          nullptr, nullptr, 0, Fe, Fp, S.W(0), S.W(1), 1.0 / eps, halo, red, norms);
        ++res_evals;
        ++its;
        double rs = 0.0;
        for (int j = 0; j < kt; ++j) {
          double re = -Fe[ix(j, tid, TPB)] * cs.isFe - (double)S.W(0)[ix(j, tid, TPB)];
          double rp = -Fp[ix(j, tid, TPB)] * cs.isFp - (double)S.W(1)[ix(j, tid, TPB)];
          S.W(0)[ix(j, tid, TPB)] = (KR)re;
          S.W(1)[ix(j, tid, TPB)] = (KR)rp;
          rs += re * re + rp * rp;
        }
        block_reduce<TPB>(&rs, 1, false, red);
        beta = sqrt(rs);
        if (beta <= gam * beta0) { converged = true; break; }
        // stagnation: a full cycle that leaves more than stall_ratio of its
        // starting true residual ends the solve with the correction reached
        // (the line search still judges the step); GMRES(m) stalls this way
        // near the attainable accuracy of FP32 Krylov vectors on
        // ill-conditioned columns
        if (beta > a.p.stall * beta_cycle) break;
        const double ib = 1.0 / beta;
        for (int j = 0; j < kt; ++j) {
          S.V(0, 0)[ix(j, tid, TPB)] = (KR)((double)S.W(0)[ix(j, tid, TPB)] * ib);
          S.V(0, 1)[ix(j, tid, TPB)] = (KR)((double)S.W(1)[ix(j, tid, TPB)] * ib);
        }
        __syncthreads();
      }
      krylov += its;
      if (bad) { status = SDCEF_STATUS_NONFINITE; break; }
      if (first_cycle) {   // no GMRES cycle ran (Fhat = 0): a zero correction
        for (int j = 0; j < kt; ++j) { XHe[ix(j, tid, TPB)] = KR(0); XHp[ix(j, tid, TPB)] = KR(0); }
        __syncthreads();
      }
      // delta-hat is in XH (sum of y_q Mhat^{-1} V_q over the cycles)
      // ---- backtracking line search ----------------------------------------
      // A step taken for the error test tries lam = 1 only and is also accepted
      // if the new iterate still passes the residual test (near the rounding
      // floor of F the sufficient decrease of the scaled 2-norm, dominated by
      // the Poisson block's floor, can fail while the step removes the error);
      // otherwise the column keeps X^(l), which passed the residual test.
      double lam = 1.0;
      bool accepted = false;
      const int nxt = 1 - cur;
      const int max_ls = polish ? 0 : a.p.max_ls;
      double tnorm[4];
      for (int t = 0; t <= max_ls; ++t) {
        residual<TPB, KR, PR, VAR>(a, g, cs, S, S.pd(pd_n(cur)), S.pd(pd_psi(cur)), DXe, DXp, lam * dcoef * cs.sn,
                          lam * dcoef * cs.sp, OUT_F,
                          S.pd(PD_FE0 + 2 * nxt), S.pd(PD_FP0 + 2 * nxt), nxt, nullptr, nullptr,
                          nullptr, nullptr, 0, halo, red, tnorm, S.pd(pd_n(nxt)),
                          S.pd(pd_psi(nxt)));
        ++res_evals;
        double t2 = scaled_two(tnorm);
        if (t2 <= 1.79e308 && (t2 <= (1.0 - a.p.ls_alpha * lam * (1.0 - gam)) * fn2 ||
                               (polish && scaled_inf(tnorm) < a.p.eps_F))) {
          accepted = true;
          break;
        }
        if (t < max_ls) lam *= 0.5;
      }
      if (!accepted && polish) { status = SDCEF_STATUS_OK; break; }
      if (!accepted) {
        status = converged ? SDCEF_STATUS_LINESEARCH_FAIL : SDCEF_STATUS_MAX_KRYLOV;
        break;
      }
      // X += lam S_X delta-hat: the accepted trial's state is in set nxt;
      // the step size for the eps_X test
      double smax = 0.0;
      if (a.p.eps_X > 0.0)
        for (int j = 0; j < kt; ++j) {
          double dn = (double)DXe[ix(j, tid, TPB)], dp = (double)DXp[ix(j, tid, TPB)];
          smax = fmax(smax, fabs(dcoef) * fmax(fabs(dn), fabs(dp)));
        }
      cur = nxt;
      const double fprev = fninf;
      fninf = scaled_inf(tnorm);
      fn2 = scaled_two(tnorm);
      ++newton;
      prec_cur = false;
      if (tid == 0) cs.polished += polish ? 1 : 0;
      // a supplied start whose step keeps the residual above guess_prog times
      // the previous one wanders: restart from X^n (CTA-uniform)
      if (guessed && attempt == 0 && a.p.guess_prog > 0.0 && !(fninf < a.p.eps_F) &&
          fninf > a.p.guess_prog * fprev) {
        __syncthreads();
        status = SDCEF_STATUS_MAX_NEWTON;
        break;
      }
      if (a.p.eps_X > 0.0) {
        block_reduce<TPB>(&smax, 1, true, red);
        if (lam * smax < a.p.eps_X && fninf >= a.p.eps_F) { status = SDCEF_STATUS_OK; break; }
      } else {
        __syncthreads();
      }
    }
    if (status == SDCEF_STATUS_OK || !guessed || attempt == 1) break;
    }   // attempts
    // ---- outputs ----------------------------------------------------------
    for (int j = 0; j < kt; ++j) {
      const int64_t gi = cell_ix(off, g, j);
      const double pref = S.pd(PD_PREF)[ix(j, tid, TPB)];
      a.ne_out[gi] = S.pd(pd_n(cur))[ix(j, tid, TPB)];
      a.phi_out[gi] = pref + S.pd(pd_psi(cur))[ix(j, tid, TPB)];
    }
    if (tid == 0) {
      if (a.status) a.status[col] = status;
      if (a.newton_it) a.newton_it[col] = newton;
      if (a.krylov_it) a.krylov_it[col] = krylov;
      if (a.res_evals) a.res_evals[col] = res_evals;
      if (a.mg_cycles) a.mg_cycles[col] = cs.mgc;
      if (a.final_res) a.final_res[col] = fninf;
    }
    __syncthreads();
  }
}

#ifdef SDCEF_WITH_ORDER
// Longest-first order of the columns (counting sort on length, descending).
__global__ void order_kernel(const int64_t* col_off, int64_t ncol, int nbins, int shift,
                             int* order) {
  extern __shared__ int sh_hist[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh_hist[b] = 0;
  __syncthreads();
  for (int64_t c = threadIdx.x; c < ncol; c += blockDim.x) {
    int64_t n = col_off[c + 1] - col_off[c];
    long long nn = n < 0 ? 0 : (long long)n;
    long long bb = nn >> shift;
    int b = (int)(bb < nbins - 1 ? bb : nbins - 1);
    atomicAdd(&sh_hist[nbins - 1 - b], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int b = 0; b < nbins; ++b) {
      int c = sh_hist[b];
      sh_hist[b] = s;
      s += c;
    }
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < ncol; c += blockDim.x) {
    int64_t n = col_off[c + 1] - col_off[c];
    long long nn = n < 0 ? 0 : (long long)n;
    long long bb = nn >> shift;
    int b = (int)(bb < nbins - 1 ? bb : nbins - 1);
    int pos = atomicAdd(&sh_hist[nbins - 1 - b], 1);
    order[pos] = (int)c;
  }
}



// B(x) = x / (e^x - 1) and B'(x) for any sign of x, through bern_pos and
// B(-a) = a + B(a), B'(-a) = -1 - B'(a), exactly as the residual forms them.
__global__ void bernoulli_kernel(const double* x, double* b, double* db, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i], aa = fabs(v);
    double bp, dbp;
    bern_pos<true>(aa, &bp, &dbp);
    const bool pos = dbits(v) >= 0;
    b[i] = pos ? bp : aa + bp;
    db[i] = pos ? dbp : -1.0 - dbp;
  }
}

#endif  // SDCEF_WITH_ORDER

template <int TPB, typename KR, typename PR>
cudaError_t launch_t(const KArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto k = jfnk_kernel<TPB, KR, PR, kVarBase>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, TPB, smem, st>>>(a);
  return cudaGetLastError();
}

template <int TPB, typename KR, typename PR>
int occupancy_t(size_t smem) {
  int nb = 0;
  auto k = jfnk_kernel<TPB, KR, PR, kVarBase>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, TPB, smem) != cudaSuccess) return 1;
  return nb < 1 ? 1 : nb;
}

#ifdef SDCEF_MG
// The multigrid instantiation: FP64, kMgTPB threads per column.
inline cudaError_t launch_mg_t(const KArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto k = jfnk_kernel<kMgTPB, double, double, kVarMG>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kMgTPB, smem, st>>>(a);
  return cudaGetLastError();
}
inline int occupancy_mg_t(size_t smem) {
  int nb = 0;
  auto k = jfnk_kernel<kMgTPB, double, double, kVarMG>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kMgTPB, smem) != cudaSuccess) return 1;
  return nb < 1 ? 1 : nb;
}
#endif  // SDCEF_MG
#ifdef SDCEF_TAB
// The transport-table instantiation: FP64, kMgTPB threads per column.
inline cudaError_t launch_tab_t(const KArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto k = jfnk_kernel<kMgTPB, double, double, kVarTable>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kMgTPB, smem, st>>>(a);
  return cudaGetLastError();
}
inline int occupancy_tab_t(size_t smem) {
  int nb = 0;
  auto k = jfnk_kernel<kMgTPB, double, double, kVarTable>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kMgTPB, smem) != cudaSuccess) return 1;
  return nb < 1 ? 1 : nb;
}
#endif  // SDCEF_TAB
#endif  // SDCEF_KERNEL_TU

}  // namespace sdcef_impl
