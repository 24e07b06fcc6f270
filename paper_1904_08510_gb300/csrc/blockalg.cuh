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
// one unknown per thread, solved by parallel cyclic reduction (PCR) in shared
// memory. The factorisation (matrix-only work) is done once per Newton step;
// each solve then costs a forward/backward sweep, log2(threads) PCR levels on
// the right-hand side only, and the spike reconstruction.
#pragma once
#include <cuda_runtime.h>

namespace sdcef {

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
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mmul(const Mat<NB, R>& x, const Mat<NB, R>& y) {
  Mat<NB, R> r;
#pragma unroll
  for (int i = 0; i < NB; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < NB; ++k) s = fma(x.a[i * NB + k], y.a[k * NB + j], s);
      r.a[i * NB + j] = s;
    }
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Vec<NB, R> mvec(const Mat<NB, R>& x, const Vec<NB, R>& v) {
  Vec<NB, R> r;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) s = fma(x.a[i * NB + k], v.a[k], s);
    r.a[i] = s;
  }
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> madd(const Mat<NB, R>& x, const Mat<NB, R>& y) {
  Mat<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) r.a[k] = x.a[k] + y.a[k];
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> msub(const Mat<NB, R>& x, const Mat<NB, R>& y) {
  Mat<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) r.a[k] = x.a[k] - y.a[k];
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Mat<NB, R> mneg(const Mat<NB, R>& x) {
  Mat<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) r.a[k] = -x.a[k];
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Vec<NB, R> vsub(const Vec<NB, R>& x, const Vec<NB, R>& y) {
  Vec<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB; ++k) r.a[k] = x.a[k] - y.a[k];
  return r;
}
template <int NB, typename R>
__device__ __forceinline__ Vec<NB, R> vadd(const Vec<NB, R>& x, const Vec<NB, R>& y) {
  Vec<NB, R> r;
#pragma unroll
  for (int k = 0; k < NB; ++k) r.a[k] = x.a[k] + y.a[k];
  return r;
}
// Inverse; *bad is set when the pivot is zero or not finite.
__device__ __forceinline__ Mat<1, double> minv(const Mat<1, double>& x, bool* bad) {
  Mat<1, double> r;
  r.a[0] = 1.0 / x.a[0];
  if (!(x.a[0] != 0.0) || !isfinite(r.a[0])) *bad = true;
  return r;
}
__device__ __forceinline__ Mat<1, float> minv(const Mat<1, float>& x, bool* bad) {
  Mat<1, float> r;
  r.a[0] = 1.0f / x.a[0];
  if (!(x.a[0] != 0.0f) || !isfinite(r.a[0])) *bad = true;
  return r;
}
template <typename R>
__device__ __forceinline__ Mat<2, R> minv(const Mat<2, R>& x, bool* bad) {
  R det = x.a[0] * x.a[3] - x.a[1] * x.a[2];
  R id = R(1) / det;
  Mat<2, R> r;
  r.a[0] = x.a[3] * id;
  r.a[1] = -x.a[1] * id;
  r.a[2] = -x.a[2] * id;
  r.a[3] = x.a[0] * id;
  if (!(det != R(0)) || !isfinite(id)) *bad = true;
  return r;
}

// Plane storage: a plane holds one value per (row j, thread t) at j*TPB + t.
template <int NB, typename R, int TPB>
struct Planes {
  R* p;
  size_t PL;   // elements per plane
  __device__ __forceinline__ Mat<NB, R> ldm(int k0, int j, int t) const {
    Mat<NB, R> m;
#pragma unroll
    for (int k = 0; k < NB * NB; ++k) m.a[k] = p[(size_t)(k0 + k) * PL + (size_t)j * TPB + t];
    return m;
  }
  __device__ __forceinline__ void stm(int k0, int j, int t, const Mat<NB, R>& m) const {
#pragma unroll
    for (int k = 0; k < NB * NB; ++k) p[(size_t)(k0 + k) * PL + (size_t)j * TPB + t] = m.a[k];
  }
};

// Per-thread scalar area: entry k of thread t at k*TPB + t.
template <int NB, typename R, int TPB>
struct Scal {
  R* p;
  __device__ __forceinline__ Mat<NB, R> ldm(int k0, int t) const {
    Mat<NB, R> m;
#pragma unroll
    for (int k = 0; k < NB * NB; ++k) m.a[k] = p[(k0 + k) * TPB + t];
    return m;
  }
  __device__ __forceinline__ void stm(int k0, int t, const Mat<NB, R>& m) const {
#pragma unroll
    for (int k = 0; k < NB * NB; ++k) p[(k0 + k) * TPB + t] = m.a[k];
  }
};

// Factor planes per interior row: Winv, G = Winv M, Cp = Winv U, P, Q.
template <int NB> struct FIdx {
  static constexpr int WINV = 0, G = NB * NB, CP = 2 * NB * NB, P = 3 * NB * NB,
                       Q = 4 * NB * NB, NPLANES = 5 * NB * NB;
  // per-thread scalars: Me, Ue, Binv, then per PCR level alpha, gamma
  static constexpr int ME = 0, UE = NB * NB, BINV = 2 * NB * NB, LVL = 3 * NB * NB;
  static __host__ __device__ constexpr int nscal(int levels) { return 3 * NB * NB + 2 * NB * NB * levels; }
};

// Number of PCR levels for a reduced system of `tact` unknowns.
__device__ __forceinline__ int pcr_levels(int tact) {
  int l = 0;
  while ((1 << l) < tact) ++l;
  return l;
}

// Factorise the column's block-tridiagonal matrix. rowf(j, M, D, U) yields the
// blocks of the thread's local row j (M couples row-1, U couples row+1).
// sh must hold TPB * 3 * NB * NB values of R. All threads of the CTA call it.
template <int NB, typename R, int TPB, class RowF>
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
      Mat<NB, R> W = (j == 0) ? D : msub(D, mmul(M, Cp_prev));
      Mat<NB, R> Wi = minv(W, bad);
      Mat<NB, R> G = mmul(Wi, M);
      Mat<NB, R> Cp = mmul(Wi, U);
      Mat<NB, R> Pg = (j == 0) ? mneg(G) : mneg(mmul(G, Pg_prev));
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
      for (int j = m - 2; j >= 0; --j) {
        Mat<NB, R> Cp = F.ldm(FI::CP, j, tid);
        Mat<NB, R> Pj = msub(F.ldm(FI::P, j, tid), mmul(Cp, Pn));
        Mat<NB, R> Qj = mneg(mmul(Cp, Qn));
        F.stm(FI::P, j, tid, Pj);
        F.stm(FI::Q, j, tid, Qj);
        Pn = Pj;
        Qn = Qj;
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
    Ab = mmul(Me, Plast);
    Bb = madd(madd(De, mmul(Me, Qlast)), mmul(Ue, Pn1));
    Cb = mmul(Ue, Qn1);
  }
  const int L = pcr_levels(tact);
  for (int l = 0; l < L; ++l) {
    const int s = 1 << l;
#pragma unroll
    for (int k = 0; k < NN; ++k) {
      sh[k * TPB + tid] = Ab.a[k];
      sh[(NN + k) * TPB + tid] = Bb.a[k];
      sh[(2 * NN + k) * TPB + tid] = Cb.a[k];
    }
    __syncthreads();
    Mat<NB, R> Al, Bl, Cl, Ar, Br, Cr;
    const bool hl = tid - s >= 0, hr = tid + s < TPB;
#pragma unroll
    for (int k = 0; k < NN; ++k) {
      Al.a[k] = hl ? sh[k * TPB + tid - s] : R(0);
      Bl.a[k] = hl ? sh[(NN + k) * TPB + tid - s] : R(k % (NB + 1) == 0);
      Cl.a[k] = hl ? sh[(2 * NN + k) * TPB + tid - s] : R(0);
      Ar.a[k] = hr ? sh[k * TPB + tid + s] : R(0);
      Br.a[k] = hr ? sh[(NN + k) * TPB + tid + s] : R(k % (NB + 1) == 0);
      Cr.a[k] = hr ? sh[(2 * NN + k) * TPB + tid + s] : R(0);
    }
    __syncthreads();
    Mat<NB, R> al = hl ? mneg(mmul(Ab, minv(Bl, bad))) : mzero<NB, R>();
    Mat<NB, R> ga = hr ? mneg(mmul(Cb, minv(Br, bad))) : mzero<NB, R>();
    Mat<NB, R> Bn = Bb;
    if (hl) Bn = madd(Bn, mmul(al, Cl));
    if (hr) Bn = madd(Bn, mmul(ga, Ar));
    Ab = hl ? mmul(al, Al) : mzero<NB, R>();
    Cb = hr ? mmul(ga, Cr) : mzero<NB, R>();
    Bb = Bn;
    S.stm(FI::LVL + 2 * NN * l, tid, al);
    S.stm(FI::LVL + 2 * NN * l + NN, tid, ga);
  }
  S.stm(FI::BINV, tid, minv(Bb, bad));
}

// Solve with the factors of part_factor. rhs and out are NB planes each
// (row j of thread t at j*TPB + t); out may alias rhs. sh must hold
// 2 * TPB * NB values of R.
template <int NB, typename R, int TPB>
__device__ void part_solve(Planes<NB, R, TPB> F, Scal<NB, R, TPB> S, R* const* rhs,
                           R* const* out, int kt, int tid, int tact, R* sh) {
  using FI = FIdx<NB>;
  const int m = kt - 1;
  const size_t PL = F.PL;
  (void)PL;
  auto ldv = [&](R* const* pl, int j) {
    Vec<NB, R> v;
#pragma unroll
    for (int k = 0; k < NB; ++k) v.a[k] = pl[k][(size_t)j * TPB + tid];
    return v;
  };
  auto stv = [&](R* const* pl, int j, const Vec<NB, R>& v) {
#pragma unroll
    for (int k = 0; k < NB; ++k) pl[k][(size_t)j * TPB + tid] = v.a[k];
  };
  Vec<NB, R> yfirst = vzero<NB, R>(), ylast = vzero<NB, R>(), rsep = vzero<NB, R>();
  if (kt > 0) {
    rsep = ldv(rhs, m);
    Vec<NB, R> g = vzero<NB, R>();
    for (int j = 0; j < m; ++j) {
      Vec<NB, R> r = ldv(rhs, j);
      Vec<NB, R> gn = mvec(F.ldm(FI::WINV, j, tid), r);
      if (j > 0) gn = vsub(gn, mvec(F.ldm(FI::G, j, tid), g));
      stv(out, j, gn);
      g = gn;
    }
    if (m > 0) {
      Vec<NB, R> yn = g;
      ylast = yn;
      for (int j = m - 2; j >= 0; --j) {
        Vec<NB, R> yj = vsub(ldv(out, j), mvec(F.ldm(FI::CP, j, tid), yn));
        stv(out, j, yj);
        yn = yj;
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
    rb = vsub(vsub(rsep, mvec(S.ldm(FI::ME, tid), ylast)), mvec(S.ldm(FI::UE, tid), ynext));
  }
  const int L = pcr_levels(tact);
  constexpr int NN = NB * NB;
  for (int l = 0; l < L; ++l) {
    const int s = 1 << l;
    R* buf = sh + ((l + 1) & 1) * (NB * TPB);   // level 0 uses buffer 1 (buffer 0 held y)
#pragma unroll
    for (int k = 0; k < NB; ++k) buf[k * TPB + tid] = rb.a[k];
    __syncthreads();
    Vec<NB, R> rl = vzero<NB, R>(), rr = vzero<NB, R>();
    if (tid - s >= 0) {
#pragma unroll
      for (int k = 0; k < NB; ++k) rl.a[k] = buf[k * TPB + tid - s];
    }
    if (tid + s < TPB) {
#pragma unroll
      for (int k = 0; k < NB; ++k) rr.a[k] = buf[k * TPB + tid + s];
    }
    Mat<NB, R> al = S.ldm(FI::LVL + 2 * NN * l, tid);
    Mat<NB, R> ga = S.ldm(FI::LVL + 2 * NN * l + NN, tid);
    rb = vadd(rb, vadd(mvec(al, rl), mvec(ga, rr)));
  }
  Vec<NB, R> xsep = mvec(S.ldm(FI::BINV, tid), rb);
  R* xb = sh + ((L + 1) & 1) * (NB * TPB);
  __syncthreads();   // everyone done reading the last PCR buffer
#pragma unroll
  for (int k = 0; k < NB; ++k) xb[k * TPB + tid] = xsep.a[k];
  __syncthreads();
  if (kt > 0) {
    Vec<NB, R> xl = vzero<NB, R>();
    if (tid > 0) {
#pragma unroll
      for (int k = 0; k < NB; ++k) xl.a[k] = xb[k * TPB + tid - 1];
    }
    for (int j = 0; j < m; ++j) {
      Vec<NB, R> xj = vadd(ldv(out, j),
                           vadd(mvec(F.ldm(FI::P, j, tid), xl), mvec(F.ldm(FI::Q, j, tid), xsep)));
      stv(out, j, xj);
    }
    stv(out, m, xsep);
  }
  __syncthreads();   // the caller may reuse sh
}

}  // namespace sdcef
