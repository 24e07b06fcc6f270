// Geometric multigrid for the two tridiagonal blocks of the recast Schur
// preconditioner (Eq. prec_recast), the block solver of Sec. 4.2: V-cycles with
// two red-black Gauss-Seidel relaxations on every level going down and two going
// up, repeated from x = 0 until ||b - T x||_2 <= gamma_MG ||b||_2, a cycle cap,
// or a cycle that does not lower the residual (that cycle is undone).
//
// One column per CTA, FP64. Storage (per column slot, after the Krylov and
// factor planes): for each block the level matrices (sub, dia, sup, 1/dia),
// levels back to back in natural row order; shared iterate and right-hand side
// vectors of all levels; one copy of the finest iterate.
//
// Hierarchy: coarse unknown I sits on fine unknown 2I+1, n_c = floor(n_f / 2);
// the even unknowns (relaxed first, "red") are the fine-only ones; coarsening
// stops at kMgCoarse unknowns or fewer, solved by Thomas on one thread. Coarse
// operator R T P (Galerkin). Transfers:
//   SDCEF_MG_OPERATOR: black-box (operator-dependent) interpolation from T and
//     restriction from T^T: fine-only unknown i takes -T[i][k] / T[i][i] of its
//     coarse neighbour on fine k and passes -T[k][i] / T[i][i] of its residual
//     to it; coarse unknowns are injected both ways. On a 3-point operator this
//     makes R T P the Schur complement onto the coarse unknowns.
//   SDCEF_MG_LINEAR: linear interpolation (1/2 from each coarse neighbour) and
//     R = P^T.
// Every loop runs over thread-strided rows with a block barrier between
// dependent passes; block reductions give every thread the same norms, so the
// cycle loop's control flow is uniform over the CTA.
#pragma once
#include <cuda_runtime.h>

#include "../../include/sdcef.h"
#include "checks.cuh"

namespace sdcef_impl {

constexpr int kMgCoarse = 8;
constexpr int kMgMaxLev = 24;   // 2^24 * kMgCoarse rows would be needed to exceed it

// FP64 doubles of the multigrid region of a slot with plane length PL (>= N):
// 2 blocks x 4 level arrays x 2 PL, iterate and right-hand side 2 PL each, the
// saved iterate PL.
__host__ __device__ inline size_t mg_region_doubles(size_t PL) { return 21 * PL; }

struct MgOp {
  double *sub, *dia, *sup, *dinv;
  size_t cap;   // elements of each level array (all levels of the block)
};
struct MgArea {
  MgOp op[2];
  double *x, *b, *xp;
  size_t cap;   // elements of x and b (all levels)
};

__device__ inline MgArea mg_area(double* base, size_t PL) {
  MgArea m;
  for (int k = 0; k < 2; ++k) {
    m.op[k].sub = base + (size_t)(8 * k + 0) * PL;
    m.op[k].dia = base + (size_t)(8 * k + 2) * PL;
    m.op[k].sup = base + (size_t)(8 * k + 4) * PL;
    m.op[k].dinv = base + (size_t)(8 * k + 6) * PL;
    m.op[k].cap = 2 * PL;
  }
  m.x = base + 16 * PL;
  m.b = base + 18 * PL;
  m.xp = base + 20 * PL;
  m.cap = 2 * PL;
  return m;
}

// Level l has N >> l unknowns (n_{l+1} = floor(n_l / 2)) and starts at
// offset sum_{j<l} (N >> j); the last level is the first with at most
// kMgCoarse unknowns.
__device__ inline int mg_nlev(int N) {
  int l = 0;
  while ((N >> l) > kMgCoarse && l + 1 < kMgMaxLev) ++l;
  return l + 1;
}

// Level view: operator rows [0, n) of one level.
struct MgLev {
  const double *sub, *dia, *sup, *dinv;
  int n;
  __device__ double at(int i, int k) const {
    if (i < 0 || i >= n || k < 0 || k >= n) return 0.0;
    if (k == i - 1) return sub[i];
    if (k == i) return dia[i];
    if (k == i + 1) return sup[i];
    return 0.0;
  }
};

__device__ inline MgLev mg_lev(const MgOp& T, int off, int n) {
  if (!SDCEF_CHECK(off >= 0 && n >= 0 && (size_t)off + n <= T.cap, sdcef_chk::kMgLevel))
    off = n = 0;
  return MgLev{T.sub + off, T.dia + off, T.sup + off, T.dinv + off, n};
}

// P[i][J] of level F's prolongation (coarse unknown J on fine 2J+1)
__device__ inline double mg_pw(const MgLev& F, int transfer, int i, int J) {
  const int nc = F.n / 2;
  if (i < 0 || i >= F.n || J < 0 || J >= nc) return 0.0;
  if (i & 1) return J == (i - 1) / 2 ? 1.0 : 0.0;
  const int k = 2 * J + 1;
  if (k != i - 1 && k != i + 1) return 0.0;
  return transfer == SDCEF_MG_LINEAR ? 0.5 : -F.at(i, k) * F.dinv[i];
}
// R[J][i] of level F's restriction
__device__ inline double mg_rw(const MgLev& F, int transfer, int J, int i) {
  const int nc = F.n / 2;
  if (i < 0 || i >= F.n || J < 0 || J >= nc) return 0.0;
  if (i & 1) return J == (i - 1) / 2 ? 1.0 : 0.0;
  const int k = 2 * J + 1;
  if (k != i - 1 && k != i + 1) return 0.0;
  return transfer == SDCEF_MG_LINEAR ? 0.5 : -F.at(k, i) * F.dinv[i];
}

// Galerkin entry (R T P)[I][J], I and J coarse
__device__ inline double mg_galerkin(const MgLev& F, int transfer, int I, int J) {
  double s = 0.0;
  for (int i = 2 * I; i <= 2 * I + 2; ++i) {
    const double r = mg_rw(F, transfer, I, i);
    if (r == 0.0) continue;
    for (int k = i - 1; k <= i + 1; ++k) {
      const double p = mg_pw(F, transfer, k, J);
      if (p == 0.0) continue;
      s = fma(r * F.at(i, k), p, s);
    }
  }
  return s;
}

// Build the levels of block T from its level-0 rows (already written):
// 1/dia of every level and the Galerkin coarse operators. Sets *bad if a
// diagonal entry is zero or not finite.
template <int TPB>
__device__ __noinline__ void mg_build(const MgOp& T, int N, int transfer, bool* bad) {
  const int nlev = mg_nlev(N);
  bool ok = true;
  int o = 0;
  for (int l = 0;; ++l) {
    const int n = N >> l;
    // this level and the next coarser one inside the level arrays
    if (!SDCEF_CHECK((size_t)o + n + (N >> (l + 1)) <= T.cap, sdcef_chk::kMgLevel)) {
      ok = false;
      break;
    }
    for (int i = threadIdx.x; i < n; i += TPB) {
      const double d = T.dia[o + i];
      ok = ok && (d != 0.0) && isfinite(d);
      T.dinv[o + i] = 1.0 / d;
    }
    __syncthreads();
    if (l + 1 == nlev) break;
    const MgLev F = mg_lev(T, o, n);
    const int oc = o + n, nc = N >> (l + 1);
    for (int I = threadIdx.x; I < nc; I += TPB) {
      T.sub[oc + I] = I > 0 ? mg_galerkin(F, transfer, I, I - 1) : 0.0;
      T.dia[oc + I] = mg_galerkin(F, transfer, I, I);
      T.sup[oc + I] = I + 1 < nc ? mg_galerkin(F, transfer, I, I + 1) : 0.0;
    }
    __syncthreads();
    o = oc;
  }
  if (!ok) *bad = true;
}

// One red-black Gauss-Seidel relaxation of level F on (x, b).
template <int TPB>
__device__ __forceinline__ void mg_rbgs(const MgLev& F, double* x, const double* b) {
#pragma unroll 1
  for (int colour = 0; colour < 2; ++colour) {
    for (int i = 2 * threadIdx.x + colour; i < F.n; i += 2 * TPB) {
      double s = b[i];
      if (i > 0) s = fma(-F.sub[i], x[i - 1], s);
      if (i + 1 < F.n) s = fma(-F.sup[i], x[i + 1], s);
      x[i] = s * F.dinv[i];
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double mg_res(const MgLev& F, const double* x, const double* b, int i) {
  double s = F.dia[i] * x[i];
  if (i > 0) s = fma(F.sub[i], x[i - 1], s);
  if (i + 1 < F.n) s = fma(F.sup[i], x[i + 1], s);
  return b[i] - s;
}

// One V-cycle on level 0 of block T for the vectors X, B (every level's
// vector at the offset of its operator).
template <int TPB>
__device__ __noinline__ void mg_vcycle(const MgOp& T, int N, double* X, double* B, int transfer) {
  const int tid = threadIdx.x;
  const int nlev = mg_nlev(N);
  int o = 0, l = 0;
  for (; l + 1 < nlev; ++l) {
    const int n = N >> l, nc = N >> (l + 1), oc = o + n;
    // the vectors X, B of this level and the next share the operator's offsets
    if (!SDCEF_CHECK((size_t)oc + nc <= T.cap, sdcef_chk::kMgLevel)) return;
    const MgLev F = mg_lev(T, o, n);
    double* x = X + o;
    const double* b = B + o;
    mg_rbgs<TPB>(F, x, b);
    mg_rbgs<TPB>(F, x, b);
    for (int I = tid; I < nc; I += TPB) {
      double s = 0.0;
      for (int i = 2 * I; i <= 2 * I + 2 && i < n; ++i)
        s = fma(mg_rw(F, transfer, I, i), mg_res(F, x, b, i), s);
      B[oc + I] = s;
      X[oc + I] = 0.0;
    }
    __syncthreads();
    o = oc;
  }
  // coarsest level: Thomas on one thread (at most kMgCoarse rows); the
  // eliminated super-diagonal goes into this level's right-hand side (rebuilt
  // by the next restriction) and the modified right-hand side into x
  if (tid == 0) {
    const int n = N >> l;
    const MgLev C = mg_lev(T, o, n);
    double* x = X + o;
    double* b = B + o;
    double piv = C.dia[0];
    x[0] = b[0] / piv;
    b[0] = C.sup[0] / piv;
    for (int i = 1; i < n; ++i) {
      piv = C.dia[i] - C.sub[i] * b[i - 1];
      x[i] = (b[i] - C.sub[i] * x[i - 1]) / piv;
      b[i] = C.sup[i] / piv;
    }
    for (int i = n - 2; i >= 0; --i) x[i] = x[i] - b[i] * x[i + 1];
  }
  __syncthreads();
  for (--l; l >= 0; --l) {
    const int n = N >> l, nc = N >> (l + 1), of = o - n;
    const MgLev F = mg_lev(T, of, n);
    double* x = X + of;
    const double* b = B + of;
    const double* xc = X + o;
    for (int i = tid; i < n; i += TPB) {
      double s = 0.0;
      for (int J = i / 2 - 1; J <= i / 2; ++J)
        if (J >= 0 && J < nc) s = fma(mg_pw(F, transfer, i, J), xc[J], s);
      x[i] += s;
    }
    __syncthreads();
    mg_rbgs<TPB>(F, x, b);
    mg_rbgs<TPB>(F, x, b);
    o = of;
  }
}

}  // namespace sdcef_impl
