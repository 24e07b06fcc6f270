// Kernels on the column fields around the solve (see fields.cuh): the
// provisional charged species of an SDC iteration and the charge flux.
// The device helpers (Bernoulli function, transport-table lookup, physical
// constants) are the solver's own, so the electron flux here is the one the
// residual forms.
#define SDCEF_KERNEL_TU
#include "fields.cuh"
#include "solver.cuh"

namespace sdcef_impl {

// The cells [off, off + N) of column c lie inside the batch's cells (checked
// build: records the site and reports the column as empty otherwise).
__device__ __forceinline__ bool col_in_batch(unsigned* chk, int64_t off, int64_t N, int64_t cells) {
  return SDCEF_CHECK_W(chk, off >= 0 && N >= 0 && off + N <= cells, sdcef_chk::kIonCell);
}

// n~_i = n_i - (dt/h) (Phi_{i+1/2} - Phi_{i-1/2}), Phi = w n_upwind with the
// drift velocity w = nu kappa E at the face (E = -dphi/dx; the electrode faces
// use the second-order one-sided gradient); electrodes absorb outgoing ions
// and emit none. One CTA per column.
__global__ void ion_update_kernel(IonArgs a) {
  const int64_t c = blockIdx.x;
  if (c >= a.ncol) return;
  const int64_t off = a.col_off[c];
  const int N = (int)(a.col_off[c + 1] - off);
  if (N < 2) return;
  const int64_t cells = a.col_off[a.ncol];
  if (!col_in_batch(a.chk, off, N, cells)) return;
  const double h = a.length[c] / N, ih = 1.0 / h, r = a.dt[c] * ih;
  const double* p = a.phi + off;
  const double GL = (-8.0 * a.vl[c] + 9.0 * p[0] - p[1]) * (ih * (1.0 / 3.0));
  const double GR = (8.0 * a.vr[c] - 9.0 * p[N - 1] + p[N - 2]) * (ih * (1.0 / 3.0));
  for (int s = 0; s < a.nsp; ++s) {
    const double* ni = a.n_in + (int64_t)s * cells + off;
    double* no = a.n_out + (int64_t)s * cells + off;
    const double nk = (double)a.val[s] * a.kappa;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      double fl, fr;
      if (i == 0) {
        double w = -nk * GL;
        fl = w < 0.0 ? w * ni[0] : 0.0;
      } else {
        double w = -nk * (p[i] - p[i - 1]) * ih;
        fl = w * (w > 0.0 ? ni[i - 1] : ni[i]);
      }
      if (i == N - 1) {
        double w = -nk * GR;
        fr = w > 0.0 ? w * ni[N - 1] : 0.0;
      } else {
        double w = -nk * (p[i + 1] - p[i]) * ih;
        fr = w * (w > 0.0 ? ni[i] : ni[i + 1]);
      }
      no[i] = ni[i] - r * (fr - fl);
    }
  }
}

// Provisional ion densities of an SDC iteration (Sec. 3.1, Algorithm 1), per
// species: (I - dt D) n~ = n^n - (dt/h)(F_{i+1/2} - F_{i-1/2}) + (dt/2)(D n^n
// - D n^(k)). F = w n_face with the effective velocity w = U_f + nu kappa E_f
// and the second-order Godunov (MUSCL) face state: the upwind cell value
// extrapolated by (1 -+ w dt/h)/2 times its monotonized-central limited
// difference (zero in the end cells); electrodes pass the outgoing drift of
// the edge cell only. D: Einstein diffusivity kappa k_B T_f / (|nu| e), no
// flux through the electrodes. ion_provisional_kernel forms the right-hand
// side (one CTA per column, thread-strided cells); ion_diffusion_kernel then
// solves (I - dt D) n~ = rhs by Thomas with one thread per (column, species),
// so every column's elimination chain runs at once (eliminated
// super-diagonal in scratch, right-hand side in place).
__device__ __forceinline__ double mc_limited(double dm, double dp) {
  if (dm * dp <= 0.0) return 0.0;
  double m = fmin(2.0 * fabs(dm), 2.0 * fabs(dp));
  m = fmin(m, 0.5 * fabs(dm + dp));
  return dm > 0.0 ? m : -m;
}

__global__ void ion_provisional_kernel(IonProvArgs a) {
  const int64_t c = blockIdx.x;
  if (c >= a.ncol) return;
  const int64_t off = a.col_off[c];
  const int N = (int)(a.col_off[c + 1] - off);
  const int64_t cells = a.col_off[a.ncol];
  if (!col_in_batch(a.chk, off, N, cells)) return;
  if (N < 2) {
    for (int s = 0; s < a.nsp; ++s)
      for (int i = threadIdx.x; i < N; i += blockDim.x)
        a.n_out[(int64_t)s * cells + off + i] = a.n0[(int64_t)s * cells + off + i];
    return;
  }
  const double h = a.length[c] / N, dt = a.dt[c];
  const double ih = 1.0 / h, dtih = dt * ih, ih2 = ih * ih;
  const double* p = a.phi + off;
  const double* T = a.T + off;
  const double* U = a.u ? a.u + off : nullptr;
  const double GL = (-8.0 * a.vl[c] + 9.0 * p[0] - p[1]) * (ih * (1.0 / 3.0));
  const double GR = (8.0 * a.vr[c] - 9.0 * p[N - 1] + p[N - 2]) * (ih * (1.0 / 3.0));
  for (int s = 0; s < a.nsp; ++s) {
    const double* n0 = a.n0 + (int64_t)s * cells + off;
    const double* nk = a.nk ? a.nk + (int64_t)s * cells + off : n0;
    double* out = a.n_out + (int64_t)s * cells + off;
    // interior face fluxes F_{f}, f = 1..N-1, computed once each (scratch
    // entry f - 1; the diffusion solve reuses the scratch afterwards)
    double* Fi = a.scratch + (int64_t)s * cells + off;
    const double nu = (double)a.val[s];
    const double nk_ = nu * a.kappa;
    const double Dc = nu != 0.0 ? a.kappa * kKb / (fabs(nu) * kQe) : 0.0;
    auto slope = [&](int i) {
      return (i == 0 || i == N - 1) ? 0.0 : mc_limited(n0[i] - n0[i - 1], n0[i + 1] - n0[i]);
    };
    for (int f = 1 + threadIdx.x; f < N; f += blockDim.x) {
      const int i = f - 1;
      const double w = (U ? 0.5 * (U[i] + U[i + 1]) : 0.0) - nk_ * ((p[i + 1] - p[i]) * ih);
      const double cfl = w * dtih;
      const double nf = w >= 0.0 ? n0[i] + 0.5 * (1.0 - cfl) * slope(i)
                                 : n0[i + 1] - 0.5 * (1.0 + cfl) * slope(i + 1);
      Fi[i] = w * nf;
    }
    __syncthreads();
    auto flux = [&](int f) {
      if (f == 0 || f == N) {
        const double w = (U ? U[f == 0 ? 0 : N - 1] : 0.0) + nk_ * (f == 0 ? -GL : -GR);
        const bool out_ = f == 0 ? w < 0.0 : w > 0.0;
        return out_ ? w * (f == 0 ? n0[0] : n0[N - 1]) : 0.0;
      }
      return Fi[f - 1];
    };
    auto dface = [&](int f) { return (f == 0 || f == N) ? 0.0 : Dc * 0.5 * (T[f - 1] + T[f]); };
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double Dl = dface(i), Dr = dface(i + 1);
      const double dn0 = (Dr * ((i + 1 < N ? n0[i + 1] : n0[i]) - n0[i]) -
                          Dl * (n0[i] - (i > 0 ? n0[i - 1] : n0[i]))) * ih2;
      const double dnk = (Dr * ((i + 1 < N ? nk[i + 1] : nk[i]) - nk[i]) -
                          Dl * (nk[i] - (i > 0 ? nk[i - 1] : nk[i]))) * ih2;
      out[i] = n0[i] - dtih * (flux(i + 1) - flux(i)) + 0.5 * dt * (dn0 - dnk);
    }
    __syncthreads();   // the next species writes its own scratch slice; keep passes ordered
  }
}

__global__ void ion_diffusion_kernel(IonProvArgs a) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.ncol * a.nsp) return;
  const int64_t c = q / a.nsp;
  const int s = (int)(q - c * a.nsp);
  const int64_t off = a.col_off[c];
  const int N = (int)(a.col_off[c + 1] - off);
  if (N < 2) return;
  const int64_t cells = a.col_off[a.ncol];
  if (!col_in_batch(a.chk, off, N, cells)) return;
  const double nu = (double)a.val[s];
  const double Dc = nu != 0.0 ? a.kappa * kKb / (fabs(nu) * kQe) : 0.0;
  const double h = a.length[c] / N, dt = a.dt[c];
  const double* __restrict__ T = a.T + off;
  double* __restrict__ out = a.n_out + (int64_t)s * cells + off;
  double* __restrict__ cp = a.scratch + (int64_t)s * cells + off;
  const double k = dt / (h * h);
  // face diffusivities D_{i+1/2} = Dc (T_i + T_{i+1}) / 2; zero at the
  // electrodes; one reciprocal of the pivot per row
  double Tl = T[0], Tr = T[1];
  double sub = 0.0, sup = -k * (Dc * 0.5 * (Tl + Tr));
  double rp = 1.0 / (1.0 - sub - sup);
  cp[0] = sup * rp;
  double dprev = out[0] * rp;
  out[0] = dprev;
  for (int i = 1; i < N; ++i) {
    sub = sup;                                  // the face shared with row i - 1
    Tl = Tr;
    sup = i + 1 < N ? -k * (Dc * 0.5 * (Tl + (Tr = T[i + 1]))) : 0.0;
    rp = 1.0 / ((1.0 - sub - sup) - sub * cp[i - 1]);
    cp[i] = sup * rp;
    dprev = (out[i] - sub * dprev) * rp;
    out[i] = dprev;
  }
  double xn = dprev;
  for (int i = N - 2; i >= 0; --i) {
    xn = out[i] - cp[i] * xn;
    out[i] = xn;
  }
}

// Charge flux J = J+ + J- through the N + 1 faces of a column (Sec. 4.4):
// J_m = nu_m e Gamma_m, Gamma_m the number flux. Electrons: the
// Scharfetter-Gummel flux of the residual (electrode faces by the electron
// boundary condition). Ions: drift with U + nu_m kappa E (E = -dphi/dx) on the
// upwind cell value plus diffusion -D_m dn/dx, D_m = kappa k_B T / (|nu_m| e)
// with the face mean of T; at an electrode only outgoing drift. One CTA per
// column, one thread per face; faces of column c start at col_off[c] + c.
__global__ void current_kernel(CurrentArgs a) {
  const int64_t c = blockIdx.x;
  if (c >= a.ncol) return;
  const int64_t off = a.col_off[c];
  const int N = (int)(a.col_off[c + 1] - off);
  const int64_t f0 = off + c;
  if (!col_in_batch(a.chk, off, N, a.col_off[a.ncol])) return;
  if (N < 2) {
    for (int f = threadIdx.x; f <= N; f += blockDim.x) {
      a.jp[f0 + f] = 0.0;
      a.jn[f0 + f] = 0.0;
    }
    return;
  }
  const int64_t cells = a.col_off[a.ncol];
  const double h = a.length[c] / N, ih = 1.0 / h, mu = a.mu;
  const double* p = a.phi + off;
  const double* x = a.ne + off;
  const double* T = a.T + off;
  const double* U = a.u ? a.u + off : nullptr;
  const double GL = (-8.0 * a.vl[c] + 9.0 * p[0] - p[1]) / (3.0 * h);
  const double GR = (8.0 * a.vr[c] - 9.0 * p[N - 1] + p[N - 2]) / (3.0 * h);
  const double kbe = kKb / kQe;
  const TransportTab tt{a.tab, a.tnc, a.tnx, a.ten_max_td, a.tT_in, a.tinv_dT, a.tgas_W};
  for (int f = threadIdx.x; f <= N; f += blockDim.x) {
    double jp = 0.0, jn = 0.0;
    const bool edge = (f == 0 || f == N);
    const int i = f - 1;   // interior face between cells i and i + 1
    double gam;            // electrons
    // table coordinates (c index, |G| -> E/N index factor) of a face between cells i and k
    auto tab_coord = [&](int i, int k, double* tc, double* sx) {
      const double ci = fmin(fmax((T[i] - tt.T_in) * tt.inv_dT, 0.0), 1.0);
      const double ck = fmin(fmax((T[k] - tt.T_in) * tt.inv_dT, 0.0), 1.0);
      const double Nf = 0.5 * (a.rho[off + i] + a.rho[off + k]) * (kNA / tt.gas_W);
      *tc = 0.5 * (ci + ck) * (tt.nc - 1);
      *sx = (double)(tt.nx - 1) / (tt.en_max_td * 1e-21 * Nf);
    };
    if (edge) {
      const int k = f == 0 ? 0 : N - 1;
      const double G = f == 0 ? GL : GR;
      double mub = mu;
      if (tt.tab) {
        double tc, sx, Dd;
        tab_coord(k, k, &tc, &sx);
        tab_mu_d(tt, tc, fabs(G) * sx, &mub, &Dd);
      }
      const double v = (U ? U[k] : 0.0) + mub * G;
      const double ned = f == 0 ? x[0] : x[N - 1];
      const bool out = f == 0 ? v < 0.0 : v > 0.0;
      gam = (a.bc == SDCEF_BC_ZERO_GRADIENT || out) ? v * ned : 0.0;
    } else {
      double Df = 0.5 * (mu * kbe * T[i] + mu * kbe * T[i + 1]), muf = mu;
      const double G = (p[i + 1] - p[i]) * ih;
      if (tt.tab) {
        double tc, sx;
        tab_coord(i, i + 1, &tc, &sx);
        tab_mu_d(tt, tc, fabs(G) * sx, &muf, &Df);
      }
      const double uf = U ? 0.5 * (U[i] + U[i + 1]) : 0.0;
      const double v = uf + muf * G;
      const double Pe = v * h / Df;
      const double aa = fabs(Pe);
      double bb, dbb;
      bern_pos<false>(aa, &bb, &dbb);
      const double bpos = Pe >= 0.0 ? bb : aa + bb;    // B(Pe)
      const double bneg = Pe >= 0.0 ? aa + bb : bb;    // B(-Pe)
      gam = (Df * ih) * (bneg * x[i] - bpos * x[i + 1]);
    }
    jn -= kQe * gam;
    for (int s = 0; s < a.nsp; ++s) {
      const double nu = (double)a.val[s];
      if (nu == 0.0) continue;
      const double* ni = a.n_ion + (int64_t)s * cells + off;
      double g;
      if (edge) {
        const double E = f == 0 ? -GL : -GR;
        const double w = (U ? U[f == 0 ? 0 : N - 1] : 0.0) + nu * a.kappa * E;
        const bool out = f == 0 ? w < 0.0 : w > 0.0;
        g = out ? w * (f == 0 ? ni[0] : ni[N - 1]) : 0.0;
      } else {
        const double E = -(p[i + 1] - p[i]) * ih;
        const double w = (U ? 0.5 * (U[i] + U[i + 1]) : 0.0) + nu * a.kappa * E;
        const double Di = 0.5 * (T[i] + T[i + 1]) * a.kappa * kKb / (fabs(nu) * kQe);
        g = w * (w > 0.0 ? ni[i] : ni[i + 1]) - Di * (ni[i + 1] - ni[i]) * ih;
      }
      if (nu > 0.0) jp += nu * kQe * g;
      else jn += nu * kQe * g;
    }
    a.jp[f0 + f] = jp;
    a.jn[f0 + f] = jn;
  }
}


cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t st) {
  ion_update_kernel<<<(unsigned)a.ncol, 128, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_ion_provisional(const IonProvArgs& a, cudaStream_t st) {
  ion_provisional_kernel<<<(unsigned)a.ncol, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nthr = a.ncol * a.nsp;
  ion_diffusion_kernel<<<(unsigned)((nthr + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_current(const CurrentArgs& a, cudaStream_t st) {
  current_kernel<<<(unsigned)a.ncol, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdcef_impl
