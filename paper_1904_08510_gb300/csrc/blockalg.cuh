// Small dense block algebra (1x1 and 2x2) and the CTA-wide partitioned
// block-tridiagonal solver used by both preconditioner forms of Sec. 3.2:
// the exact Schur factorisation (Eq. prec, 2x2 blocks on the cell-interleaved
// (n_i, phi_i) unknowns) and the recast form (Eq. prec_recast, scalar
// tridiagonal blocks of dt D_f - I and of the approximate Schur complement).
//
// Partition scheme. A CTA of TPB threads owns one column; thread t owns the
// contiguous rows [t*K, t*K + kt). The last row of each chunk is a separator,
// the kt - 1 rows before it are interior rows. Interior rows are eliminated by
// block Thomas with two "spike" couplings (to the previous chunk's separator
// X_L and to the chunk's own separator X_R):
//     x_j = y_j + P_j X_L + Q_j X_R .
// Substituting into the separator rows gives a block-tridiagonal system with
// one unknown per active thread. It is reduced by cyclic reduction (CR, half
// of the rows eliminated per level, compact thread mapping) until at most 32
// rows remain, which warp 0 solves by parallel cyclic reduction (PCR) with
// register shuffles; CR back-substitution then recovers the eliminated rows.
// The factorisation (matrix-only work) is done once per Newton step; each
// solve then costs a forward/backward sweep, the CR/PCR passes on the
// right-hand side only, and the spike reconstruction.
//
// Cost model. On this part every FP64 warp instruction occupies the FP64 pipe
// for the same time whatever the number of active lanes, so the reduced solve
// is organised to keep the number of FP64 warp instructions small: CR touches
// T/2 + T/4 + ... rows on compact lanes, and the PCR tail runs on one warp,
// where PCR over all T rows would issue log2(T) levels on every warp. Products
// with the coupling blocks skip their structural zeros (the lower-left entry
// of the 2x2 off-diagonal blocks of Eq. linear_nls is zero because
// dF_phi/dn is diagonal) and every multiply-accumulate is one FMA chain.
#pragma once
#include <cstring>
#include <cuda_runtime.h>

#include "checks.cuh"
#include "dfloat.cuh"

namespace sdcef {
using ::fma;

template <int NB, typename R>
struct Mat {
  R a[NB * NB];
};
template <int NB, typename R>
struct Vec {
  R a[NB];
};

template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mzero() {
  Mat<NB, R> m;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) m.a[k] = R(0);
  return m;
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mident() {
  Mat<NB, R> m = mzero<NB, R>();
#pragma unroll
  for (int k = 0; k < NB; ++k) m.a[k * NB + k] = R(1);
  return m;
}
template <int NB, typename R>
__device__ __forceinline__ Vec<NB, R> vzero() {
  Vec<NB, R> v;
#pragma unroll
  for (int k = 0; k < NB; ++k) v.a[k] = R(0);
  return v;
}

// Block product with optional accumulator and sign, skipping structural zeros:
//   r = (ACC ? acc : 0) + SG * x y,
// XU / YU: x / y is upper triangular (entries below the diagonal are zero and
// are never read). The first term of an entry without accumulator is a plain
// multiply; the rest are FMAs.
template <int SG, bool ACC, bool XU, bool YU, int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mprod(const Mat<NB, R>& acc, const Mat<NB, R>& x,
                                            const Mat<NB, R>& y) {
  Mat<NB, R> r;
#pragma unroll
  for (int i = 0; i < NB; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      R s = ACC ? acc.a[i * NB + j] : R(0);
      bool first = !ACC;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if ((XU && i > k) || (YU && k > j)) continue;
        const R xv = SG > 0 ? x.a[i * NB + k] : -x.a[i * NB + k];
        if (first) {
          s = xv * y.a[k * NB + j];
          first = false;
        } else {
          s = fma(xv, y.a[k * NB + j], s);
        }
      }
      r.a[i * NB + j] = s;
    }
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mmul(const Mat<NB, R>& x, const Mat<NB, R>& y) {
  return mprod<1, false, false, false>(x, x, y);
}
// r = (ACC ? acc : 0) + SG * x v (x upper triangular if XU)
template <int SG, bool ACC, bool XU, int NB, typename R>
__device__ __forceinline__ Vec<NB, R> vprod(const Vec<NB, R>& acc, const Mat<NB, R>& x,
                                            const Vec<NB, R>& v) {
  Vec<NB, R> r;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    R s = ACC ? acc.a[i] : R(0);
    bool first = !ACC;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (XU && i > k) continue;
      const R xv = SG > 0 ? x.a[i * NB + k] : -x.a[i * NB + k];
      if (first) {
        s = xv * v.a[k];
        first = false;
      } else {
        s = fma(xv, v.a[k], s);
      }
    }
    r.a[i] = s;
  }
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Vec<NB, R> mvec(const Mat<NB, R>& x, const Vec<NB, R>& v) {
  return vprod<1, false, false>(v, x, v);
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mneg(const Mat<NB, R>& x) {
  Mat<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) r.a[k] = -x.a[k];
  return r;
}

// Pivot checks on the bit patterns (integer pipe): zero or non-finite.
__device__ __forceinline__ bool bad_pivot(double det, double inv) {
  const long long d = __double_as_longlong(det), v = __double_as_longlong(inv);
  return (d & 0x7FFFFFFFFFFFFFFFLL) == 0 || (v & 0x7FF0000000000000LL) == 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool bad_pivot(float det, float inv) {
  const int d = __float_as_int(det), v = __float_as_int(inv);
  return (d & 0x7FFFFFFF) == 0 || (v & 0x7F800000) == 0x7F800000;
}
// Reciprocal of a pivot. FP64: the hardware's approximate reciprocal y
// (relative error ~1e-6) refined by one Newton-Raphson step that keeps the
// second-order term, y (1 + e + e^2) with e = 1 - x y (the series
// 1/x = y / (1 - e) cut after e^2), so the error is the seed's cubed, below
// rounding. A zero, subnormal or non-finite x gives a non-finite result, which
// the pivot check flags. Other types divide.
template <typename R>
__device__ __forceinline__ R recip(R x) {
  return R(1) / x;
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
// Inverse; *bad is set when the pivot is zero or the inverse not finite.
template <typename R>
__device__ __forceinline__ Mat<1, R> minv(const Mat<1, R>& x, bool* bad) {
  Mat<1, R> r;
  r.a[0] = recip(x.a[0]);
  if (bad_pivot(x.a[0], r.a[0])) *bad = true;
  return r;
}
template <typename R>
__device__ __forceinline__ Mat<2, R> minv(const Mat<2, R>& x, bool* bad) {
  const R det = fma(x.a[0], x.a[3], -(x.a[1] * x.a[2]));
  const R id = recip(det);
  Mat<2, R> r;
  r.a[0] = x.a[3] * id;
  r.a[1] = -x.a[1] * id;
  r.a[2] = -x.a[2] * id;
  r.a[3] = x.a[0] * id;
  if (bad_pivot(det, id)) *bad = true;
  return r;
}

template <int NB> struct FIdx;

// Factor storage: NB x NB blocks, one per (row j, thread t), in groups of
// NB^2 planes: the block of group k0 for row j of thread t holds its NB^2
// values contiguously at k0 PL + (j TPB + t) NB^2, so that a warp reads a row's
// blocks as one contiguous run and a 2 x 2 block of 8-byte values is two
// 16-byte loads (a block smaller than 16 bytes is read value by value).
template <int NB, typename R, int TPB>
struct Planes {
  R* p;
  size_t PL;   // elements per plane
  static constexpr int NN = NB * NB;
  static constexpr bool kVec = (NN * sizeof(R)) % 16 == 0 && sizeof(Mat<NB, R>) == NN * sizeof(R);
  // checked element offset of block (k0, row j, thread t): k0 .. k0 + NB^2 - 1
  // must be factor planes and j * TPB + t an element of a plane
  __device__ __forceinline__ size_t at(int k0, int j, int t) const {
    if (!SDCEF_CHECK(k0 >= 0 && k0 + NN <= FIdx<NB>::NPLANES && j >= 0 && t >= 0 &&
                         t < TPB && (size_t)j * TPB + t < PL,
                     sdcef_chk::kFacPlane))
      return 0;
    return (size_t)k0 * PL + ((size_t)j * TPB + t) * NN;
  }
  __device__ __forceinline__ Mat<NB, R> ldm(int k0, int j, int t) const {
    Mat<NB, R> m;
    const size_t o = at(k0, j, t);
    if constexpr (kVec) {
      constexpr int NV = NN * sizeof(R) / 16;
      const uint4* s = reinterpret_cast<const uint4*>(p + o);
      uint4 u[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) u[i] = s[i];
      memcpy(&m, u, sizeof(m));
    } else {
#pragma unroll
      for (int k = 0; k < NN; ++k) m.a[k] = p[o + k];
    }
    return m;
  }
  __device__ __forceinline__ void stm(int k0, int j, int t, const Mat<NB, R>& m) const {
    const size_t o = at(k0, j, t);
    if constexpr (kVec) {
      constexpr int NV = NN * sizeof(R) / 16;
      uint4 u[NV];
      memcpy(u, &m, sizeof(m));
      uint4* d = reinterpret_cast<uint4*>(p + o);
#pragma unroll
      for (int i = 0; i < NV; ++i) d[i] = u[i];
    } else {
#pragma unroll
      for (int k = 0; k < NN; ++k) p[o + k] = m.a[k];
    }
  }
};

// Per-thread scalar area: entry k of thread t at k*TPB + t.
template <int NB, typename R, int TPB>
struct Scal {
  R* p;
  __device__ __forceinline__ int at(int k0, int t) const {
    if (!SDCEF_CHECK(k0 >= 0 && k0 + NB * NB <= FIdx<NB>::NSCAL && t >= 0 && t < TPB,
                     sdcef_chk::kScal))
      return 0;
    return k0 * TPB + t;
  }
  __device__ __forceinline__ Mat<NB, R> ldm(int k0, int t) const {
    Mat<NB, R> m;
    const int o = at(k0, t);
#pragma unroll
    for (int k = 0; k < NB * NB; ++k) m.a[k] = p[o + k * TPB];
    return m;
  }
  __device__ __forceinline__ void stm(int k0, int t, const Mat<NB, R>& m) const {
    const int o = at(k0, t);
#pragma unroll
    for (int k = 0; k < NB * NB; ++k) p[o + k * TPB] = m.a[k];
  }
};

// Reduced-system levels: CR while more than 32 rows remain (at most 3 levels
// for TPB <= 256), then PCR on at most 32 rows (at most 5 levels).
constexpr int kMaxCR = 3, kMaxPCR = 5;

// Factor planes per interior row: Winv, G = Winv M, Cp = Winv U, P, Q.
template <int NB> struct FIdx {
  static constexpr int NN = NB * NB;
  static constexpr int WINV = 0, G = NN, CP = 2 * NN, P = 3 * NN, Q = 4 * NN, NPLANES = 5 * NN;
  // per-thread scalars: separator row blocks Me, Ue; final PCR pivot inverse;
  // per CR level: eliminated row (Binv, A, C) and surviving row (alpha, gamma);
  // per PCR level: (alpha, gamma)
  static constexpr int ME = 0, UE = NN, BINV = 2 * NN, CR0 = 3 * NN, CRSTEP = 5 * NN,
                       PCR0 = CR0 + kMaxCR * CRSTEP, NSCAL = PCR0 + 2 * NN * kMaxPCR;
};

// Shuffle a block from lane - s (up) or lane + s (down) within a full warp.
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> shfl_up_m(const Mat<NB, R>& x, int s) {
  Mat<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) r.a[k] = shfl_up_v(x.a[k], s);
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> shfl_down_m(const Mat<NB, R>& x, int s) {
  Mat<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) r.a[k] = shfl_down_v(x.a[k], s);
  return r;
}

// Factorise the reduced system Ab_t X_{t-1} + Bb_t X_t + Cb_t X_{t+1} = rb_t
// (t < T; Ab_0 = 0 and Cb_{T-1} = 0). All threads call it; sh must hold
// 3 * NB * NB * TPB values of R.
template <int NB, typename R, int TPB>
__device__ void red_factor(Scal<NB, R, TPB> S, int tid, int T, const Mat<NB, R>& Ab,
                           const Mat<NB, R>& Bb, const Mat<NB, R>& Cb, R* sh, bool* bad) {
  using FI = FIdx<NB>;
  constexpr int NN = NB * NB;
  R* sA = sh;
  R* sB = sh + NN * TPB;
  R* sC = sh + 2 * NN * TPB;
  auto row = [&](int i) {   // a row of the shared reduced system
    if (!SDCEF_CHECK(i >= 0 && i < TPB, sdcef_chk::kRedRow)) i = 0;
    return i;
  };
  auto ld = [&](const R* b, int i) {
    Mat<NB, R> m;
    i = row(i);
#pragma unroll
    for (int k = 0; k < NN; ++k) m.a[k] = b[k * TPB + i];
    return m;
  };
  auto st = [&](R* b, int i, const Mat<NB, R>& m) {
    i = row(i);
#pragma unroll
    for (int k = 0; k < NN; ++k) b[k * TPB + i] = m.a[k];
  };
  if (tid < T) {
    st(sA, tid, Ab);
    st(sB, tid, Bb);
    st(sC, tid, Cb);
  }
  __syncthreads();
  int n = T, l = 0;
  for (; n > 32; ++l, n >>= 1) {
    const int ne = (n + 1) >> 1, ns = n >> 1;
    const int base = FI::CR0 + FI::CRSTEP * l;
    // rows q = 2t leave the system: invert their pivot in place (only the
    // surviving neighbours read it, after the barrier)
    if (tid < ne) {
      const int q = 2 * tid;
      const Mat<NB, R> Bi = minv(ld(sB, q), bad);
      st(sB, q, Bi);
      S.stm(base, tid, Bi);
      S.stm(base + NN, tid, ld(sA, q));
      S.stm(base + 2 * NN, tid, ld(sC, q));
    }
    __syncthreads();
    Mat<NB, R> An = mzero<NB, R>(), Bn = mident<NB, R>(), Cn = mzero<NB, R>();
    if (tid < ns) {
      const int q = 2 * tid + 1;   // q - 1 >= 0 always exists
      const Mat<NB, R> al = mprod<-1, false, false, false>(Ab, ld(sA, q), ld(sB, q - 1));
      Bn = mprod<1, true, false, false>(ld(sB, q), al, ld(sC, q - 1));
      An = mmul(al, ld(sA, q - 1));
      Mat<NB, R> ga = mzero<NB, R>();
      if (q + 1 < n) {
        ga = mprod<-1, false, false, false>(Ab, ld(sC, q), ld(sB, q + 1));
        Bn = mprod<1, true, false, false>(Bn, ga, ld(sA, q + 1));
        Cn = mmul(ga, ld(sC, q + 1));
      }
      S.stm(base + 3 * NN, tid, al);
      S.stm(base + 4 * NN, tid, ga);
    }
    __syncthreads();
    if (tid < ns) {
      st(sA, tid, An);
      st(sB, tid, Bn);
      st(sC, tid, Cn);
    }
    __syncthreads();
  }
  // PCR on the remaining n <= 32 rows in warp 0; lanes >= n are identity rows
  if (tid < 32) {
    Mat<NB, R> A = mzero<NB, R>(), B = mident<NB, R>(), C = mzero<NB, R>();
    if (tid < n) {
      A = ld(sA, tid);
      B = ld(sB, tid);
      C = ld(sC, tid);
    }
    int k = 0;
    for (int s = 1; s < n; s <<= 1, ++k) {
      Mat<NB, R> Al = shfl_up_m(A, s), Bl = shfl_up_m(B, s), Cl = shfl_up_m(C, s);
      Mat<NB, R> Ar = shfl_down_m(A, s), Br = shfl_down_m(B, s), Cr = shfl_down_m(C, s);
      if (tid < s) {
        Al = mzero<NB, R>();
        Bl = mident<NB, R>();
        Cl = mzero<NB, R>();
      }
      if (tid + s >= n) {
        Ar = mzero<NB, R>();
        Br = mident<NB, R>();
        Cr = mzero<NB, R>();
      }
      const Mat<NB, R> al = mprod<-1, false, false, false>(A, A, minv(Bl, bad));
      const Mat<NB, R> ga = mprod<-1, false, false, false>(C, C, minv(Br, bad));
      B = mprod<1, true, false, false>(mprod<1, true, false, false>(B, al, Cl), ga, Ar);
      A = mmul(al, Al);
      C = mmul(ga, Cr);
      if (tid < n) {
        S.stm(FI::PCR0 + 2 * NN * k, tid, al);
        S.stm(FI::PCR0 + 2 * NN * k + NN, tid, ga);
      }
    }
    if (tid < n) S.stm(FI::BINV, tid, minv(B, bad));
  }
  __syncthreads();   // sh is free again
}

// Solve the factorised reduced system for rb (thread t < T holds rb_t).
// sr must hold 2 * NB * TPB values of R. On return (after a barrier) the
// solution X_t of every row sits at sr[k * T + t], k < NB.
template <int NB, typename R, int TPB>
__device__ void red_solve(Scal<NB, R, TPB> S, int tid, int T, const Vec<NB, R>& rb, R* sr) {
  using FI = FIdx<NB>;
  constexpr int NN = NB * NB;
  // level l occupies sr[o_l + k * n_l + i], o_l = NB * (T + T/2 + ... ) before it
  // the levels occupy at most NB (T + T/2 + ...) < 2 NB TPB values of sr
  auto el = [&](int o, int n, int i) {
    if (!SDCEF_CHECK(o >= 0 && i >= 0 && i < n && o + NB * n <= 2 * NB * TPB, sdcef_chk::kRedRow))
      return 0;
    return o + i;
  };
  auto ld = [&](int o, int n, int i) {
    Vec<NB, R> v;
    const int e = el(o, n, i);
#pragma unroll
    for (int k = 0; k < NB; ++k) v.a[k] = sr[e + k * n];
    return v;
  };
  auto st = [&](int o, int n, int i, const Vec<NB, R>& v) {
    const int e = el(o, n, i);
#pragma unroll
    for (int k = 0; k < NB; ++k) sr[e + k * n] = v.a[k];
  };
  if (tid < T) st(0, T, tid, rb);
  __syncthreads();
  int n = T, l = 0, o = 0;
  for (; n > 32; ++l) {
    const int ns = n >> 1;
    const int base = FI::CR0 + FI::CRSTEP * l;
    if (tid < ns) {
      const int q = 2 * tid + 1;
      Vec<NB, R> r = vprod<1, true, false>(ld(o, n, q), S.ldm(base + 3 * NN, tid), ld(o, n, q - 1));
      if (q + 1 < n) r = vprod<1, true, false>(r, S.ldm(base + 4 * NN, tid), ld(o, n, q + 1));
      st(o + NB * n, ns, tid, r);
    }
    __syncthreads();
    o += NB * n;
    n = ns;
  }
  const int L = l;
  if (tid < 32) {
    Vec<NB, R> r = vzero<NB, R>();
    if (tid < n) r = ld(o, n, tid);
    int k = 0;
    for (int s = 1; s < n; s <<= 1, ++k) {
      Vec<NB, R> rl, rr;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        rl.a[c] = shfl_up_v(r.a[c], s);
        rr.a[c] = shfl_down_v(r.a[c], s);
      }
      if (tid < n) {
        if (tid >= s) r = vprod<1, true, false>(r, S.ldm(FI::PCR0 + 2 * NN * k, tid), rl);
        if (tid + s < n) r = vprod<1, true, false>(r, S.ldm(FI::PCR0 + 2 * NN * k + NN, tid), rr);
      }
    }
    if (tid < n) st(o, n, tid, mvec(S.ldm(FI::BINV, tid), r));
  }
  __syncthreads();
  // CR back-substitution, coarsest level first
  for (l = L - 1; l >= 0; --l) {
    const int nl = T >> l, ns = nl >> 1, ne = (nl + 1) >> 1;
    o -= NB * nl;
    const int o1 = o + NB * nl;
    const int base = FI::CR0 + FI::CRSTEP * l;
    Vec<NB, R> xs = vzero<NB, R>();
    if (tid < ns) xs = ld(o1, ns, tid);
    if (tid < ne) {
      const int q = 2 * tid;
      Vec<NB, R> r = ld(o, nl, q);
      if (tid >= 1) r = vprod<-1, true, false>(r, S.ldm(base + NN, tid), ld(o1, ns, tid - 1));
      if (tid < ns) r = vprod<-1, true, false>(r, S.ldm(base + 2 * NN, tid), xs);
      st(o, nl, q, mvec(S.ldm(base, tid), r));
    }
    if (tid < ns) st(o, nl, 2 * tid + 1, xs);
    __syncthreads();
  }
}

// Factorise the column's block-tridiagonal matrix. rowf(j, M, D, U) yields the
// blocks of the thread's local row j (M couples row-1, U couples row+1); UT
// states that M and U are upper triangular. sh must hold TPB * 3 * NB * NB
// values of R. All threads of the CTA call it.
template <int NB, typename R, int TPB, bool UT, class RowF>
__device__ void part_factor(Planes<NB, R, TPB> F, Scal<NB, R, TPB> S, int kt, int tid,
                            int tact, RowF rowf, R* sh, bool* bad) {
  using FI = FIdx<NB>;
  const int m = kt - 1;   // interior rows of this thread (-1 if inactive)
  Mat<NB, R> Pfirst = mzero<NB, R>(), Qfirst = mident<NB, R>();
  Mat<NB, R> Plast = mident<NB, R>(), Qlast = mzero<NB, R>();
  Mat<NB, R> Me = mzero<NB, R>(), De = mident<NB, R>(), Ue = mzero<NB, R>();
  if (kt > 0) {
    Mat<NB, R> Cp_prev = mzero<NB, R>(), Pg_prev = mzero<NB, R>();
    for (int j = 0; j < m; ++j) {
      Mat<NB, R> M, D, U;
      rowf(j, M, D, U);
      const Mat<NB, R> W = (j == 0) ? D : mprod<-1, true, UT, false>(D, M, Cp_prev);
      const Mat<NB, R> Wi = minv(W, bad);
      const Mat<NB, R> G = mprod<1, false, false, UT>(Wi, Wi, M);
      const Mat<NB, R> Cp = mprod<1, false, false, UT>(Wi, Wi, U);
      const Mat<NB, R> Pg = (j == 0) ? mneg(G) : mprod<-1, false, false, false>(G, G, Pg_prev);
      F.stm(FI::WINV, j, tid, Wi);
      F.stm(FI::G, j, tid, G);
      F.stm(FI::CP, j, tid, Cp);
      F.stm(FI::P, j, tid, Pg);
      Cp_prev = Cp;
      Pg_prev = Pg;
    }
    if (m > 0) {
      // backward: P_j = Pg_j - Cp_j P_{j+1}; Q_{m-1} = -Cp_{m-1}; Q_j = -Cp_j Q_{j+1}
      Mat<NB, R> Pn = Pg_prev;
      Mat<NB, R> Qn = mneg(Cp_prev);
      Plast = Pn;
      Qlast = Qn;
      F.stm(FI::Q, m - 1, tid, Qn);
      if (m >= 2) {
        // row j - 1's operands are loaded before row j is computed and stored
        Mat<NB, R> Cn = F.ldm(FI::CP, m - 2, tid), Pgn = F.ldm(FI::P, m - 2, tid);
        for (int j = m - 2; j >= 0; --j) {
          const Mat<NB, R> Cp = Cn, Pg = Pgn;
          if (j >= 1) {
            Cn = F.ldm(FI::CP, j - 1, tid);
            Pgn = F.ldm(FI::P, j - 1, tid);
          }
          const Mat<NB, R> Pj = mprod<-1, true, false, false>(Pg, Cp, Pn);
          const Mat<NB, R> Qj = mprod<-1, false, false, false>(Cp, Cp, Qn);
          F.stm(FI::P, j, tid, Pj);
          F.stm(FI::Q, j, tid, Qj);
          Pn = Pj;
          Qn = Qj;
        }
      }
      Pfirst = Pn;
      Qfirst = Qn;
    }
    rowf(m, Me, De, Ue);
    S.stm(FI::ME, tid, Me);
    S.stm(FI::UE, tid, Ue);
  }
  // exchange the first interior spikes with the previous thread
  constexpr int NN = NB * NB;
#pragma unroll
  for (int k = 0; k < NN; ++k) {
    sh[k * TPB + tid] = Pfirst.a[k];
    sh[(NN + k) * TPB + tid] = Qfirst.a[k];
  }
  __syncthreads();
  Mat<NB, R> Pn1 = mzero<NB, R>(), Qn1 = mident<NB, R>();
  if (tid + 1 < tact) {
#pragma unroll
    for (int k = 0; k < NN; ++k) {
      Pn1.a[k] = sh[k * TPB + tid + 1];
      Qn1.a[k] = sh[(NN + k) * TPB + tid + 1];
    }
  }
  __syncthreads();
  // reduced row: Abar X_{t-1} + Bbar X_t + Cbar X_{t+1} = rbar
  Mat<NB, R> Ab = mzero<NB, R>(), Bb = mident<NB, R>(), Cb = mzero<NB, R>();
  if (kt > 0) {
    Ab = mprod<1, false, UT, false>(Me, Me, Plast);
    Bb = mprod<1, true, UT, false>(mprod<1, true, UT, false>(De, Me, Qlast), Ue, Pn1);
    Cb = mprod<1, false, UT, false>(Ue, Ue, Qn1);
  }
  red_factor<NB, R, TPB>(S, tid, tact, Ab, Bb, Cb, sh, bad);
}

// Solve with the factors of part_factor. rhs and out are NB planes each of the
// caller's type IO (row j of thread t at j*TPB + t; out may alias rhs); scr is
// the scratch of the intermediate sweeps, NB planes of R holding the NB values
// of row j of thread t contiguously at (j TPB + t) NB (one 16-byte access where
// they fill 16 bytes). sh must hold 3 * TPB * NB values of R. UT as for
// part_factor.
template <int NB, typename R, typename IO, int TPB, bool UT>
__device__ void part_solve(Planes<NB, R, TPB> F, Scal<NB, R, TPB> S, IO* const* rhs,
                           IO* const* out, R* scr, int kt, int tid, int tact, R* sh,
                           double* nrm2 = nullptr) {
  using FI = FIdx<NB>;
  const int m = kt - 1;
  // element of row j of this thread in a right-hand side, scratch or output plane
  auto el = [&](int j) {
    if (!SDCEF_CHECK(j >= 0 && tid >= 0 && tid < TPB && (size_t)j * TPB + tid < F.PL,
                     sdcef_chk::kScr))
      return (size_t)0;
    return (size_t)j * TPB + tid;
  };
  auto ldin = [&](int j) {
    Vec<NB, R> v;
    const size_t e = el(j);
#pragma unroll
    for (int k = 0; k < NB; ++k) v.a[k] = conv<R>(rhs[k][e]);
    return v;
  };
  constexpr bool kVecS = NB * sizeof(R) == 16 && sizeof(Vec<NB, R>) == 16;
  auto lds = [&](int j) {
    Vec<NB, R> v;
    const size_t e = el(j) * NB;
    if constexpr (kVecS) {
      const uint4 u = *reinterpret_cast<const uint4*>(scr + e);
      memcpy(&v, &u, sizeof(v));
    } else {
#pragma unroll
      for (int k = 0; k < NB; ++k) v.a[k] = scr[e + k];
    }
    return v;
  };
  auto sts = [&](int j, const Vec<NB, R>& v) {
    const size_t e = el(j) * NB;
    if constexpr (kVecS) {
      uint4 u;
      memcpy(&u, &v, sizeof(v));
      *reinterpret_cast<uint4*>(scr + e) = u;
    } else {
#pragma unroll
      for (int k = 0; k < NB; ++k) scr[e + k] = v.a[k];
    }
  };
  // stores a row of the solution; with nrm2, also adds the squares of the
  // stored values (this thread's part of ||out||_2^2)
  double acc = 0.0;
  auto stout = [&](int j, const Vec<NB, R>& v) {
    const size_t e = el(j);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const IO o = conv<IO>(v.a[k]);
      out[k][e] = o;
      if (nrm2) acc = fma((double)o, (double)o, acc);
    }
  };
  // Each sweep loads the operands of its next row before it computes and
  // stores the current one (rows differ, so no store can change a loaded value),
  // so that the loads of one row overlap the arithmetic of the previous row.
  Vec<NB, R> yfirst = vzero<NB, R>(), ylast = vzero<NB, R>(), rsep = vzero<NB, R>();
  if (kt > 0) {
    rsep = ldin(m);
    Vec<NB, R> g = vzero<NB, R>();
    if (m > 0) {
      Mat<NB, R> Wn = F.ldm(FI::WINV, 0, tid), Gn = mzero<NB, R>();
      Vec<NB, R> rn = ldin(0);
      for (int j = 0; j < m; ++j) {
        const Mat<NB, R> Wc = Wn, Gc = Gn;
        const Vec<NB, R> rc = rn;
        if (j + 1 < m) {
          Wn = F.ldm(FI::WINV, j + 1, tid);
          Gn = F.ldm(FI::G, j + 1, tid);
          rn = ldin(j + 1);
        }
        Vec<NB, R> gn = mvec(Wc, rc);
        if (j > 0) gn = vprod<-1, true, false>(gn, Gc, g);
        sts(j, gn);
        g = gn;
      }
      Vec<NB, R> yn = g;
      ylast = yn;
      if (m >= 2) {
        Mat<NB, R> Cn = F.ldm(FI::CP, m - 2, tid);
        Vec<NB, R> sn = lds(m - 2);
        for (int j = m - 2; j >= 0; --j) {
          const Mat<NB, R> Cc = Cn;
          const Vec<NB, R> sc = sn;
          if (j >= 1) {
            Cn = F.ldm(FI::CP, j - 1, tid);
            sn = lds(j - 1);
          }
          const Vec<NB, R> yj = vprod<-1, true, false>(sc, Cc, yn);
          sts(j, yj);
          yn = yj;
        }
      }
      yfirst = yn;
    }
  }
#pragma unroll
  for (int k = 0; k < NB; ++k) sh[k * TPB + tid] = yfirst.a[k];
  __syncthreads();
  Vec<NB, R> ynext = vzero<NB, R>();
  if (tid + 1 < tact) {
#pragma unroll
    for (int k = 0; k < NB; ++k) ynext.a[k] = sh[k * TPB + tid + 1];
  }
  Vec<NB, R> rb = vzero<NB, R>();
  if (kt > 0) {
    rb = vprod<-1, true, UT>(vprod<-1, true, UT>(rsep, S.ldm(FI::ME, tid), ylast),
                             S.ldm(FI::UE, tid), ynext);
  }
  R* sr = sh + NB * TPB;
  red_solve<NB, R, TPB>(S, tid, tact, rb, sr);
  if (kt > 0) {
    Vec<NB, R> xsep, xl = vzero<NB, R>();
#pragma unroll
    for (int k = 0; k < NB; ++k) xsep.a[k] = sr[k * tact + tid];
    if (tid > 0) {
#pragma unroll
      for (int k = 0; k < NB; ++k) xl.a[k] = sr[k * tact + tid - 1];
    }
    if (m > 0) {
      Mat<NB, R> Pn = F.ldm(FI::P, 0, tid), Qn = F.ldm(FI::Q, 0, tid);
      Vec<NB, R> sn = lds(0);
      for (int j = 0; j < m; ++j) {
        const Mat<NB, R> Pc = Pn, Qc = Qn;
        const Vec<NB, R> sc = sn;
        if (j + 1 < m) {
          Pn = F.ldm(FI::P, j + 1, tid);
          Qn = F.ldm(FI::Q, j + 1, tid);
          sn = lds(j + 1);
        }
        Vec<NB, R> xj = vprod<1, true, false>(sc, Pc, xl);
        xj = vprod<1, true, false>(xj, Qc, xsep);
        stout(j, xj);
      }
    }
    stout(m, xsep);
  }
  if (nrm2) *nrm2 = acc;
  __syncthreads();   // the caller may reuse sh
}

}  // namespace sdcef
