// Learned Newton initial guess: feature extraction; training on the tcgen05
// tensor cores (BF16 operands, FP32 accumulators in TMEM): forward, MSE loss
// and backpropagation fused in one persistent kernel whose weight gradients
// accumulate in TMEM, and Adam over the kernel's per-CTA partial gradients;
// the inference forward; and the fused inference kernel (mlp_tc.cuh) that
// assembles the guess. The network maps the
// 5-cell stencil features and the column context of a cell to the scaled
// Newton increment ((n* - n^n)/s_n, (phi* - phi^n)/s_phi); the JFNK of
// Algorithm 2 then starts from the guess instead of X^n and still decides
// convergence. The guess may take as potential the root of the Poisson
// residual at the guessed electron density (poisson_column).
//
// Shapes: 32 (25 stencil + 7 column features) -> 128 -> 128 -> 2, SiLU activations.
// Parameters (FP32 master copy, flat): W1[128][32], b1[128], W2[128][128],
// b2[128], W3[2][128], b3[2]; BF16 copies of W1, W2, W3 feed the tensor cores.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>

#include "../../include/sdcef.h"
#include "checks.cuh"
#include "mlp_tc.cuh"

namespace sdcef_impl {
int report_error(int code, const char* msg);
}
using sdcef_impl::report_error;

namespace {

constexpr int kIn = 32, kFeat = 25, kHid = 128, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid,
              kNParam = kOffB3 + kOut;
static_assert(kNParam == SDCEF_MLP_NPARAM, "parameter count");

// SiLU and its derivative through the hardware tanh approximation:
// silu(z) = z/2 (1 + tanh(z/2)), silu'(z) = s (1 + z (1 - s)) with the sigmoid
// s = (1 + tanh(z/2)) / 2 -- one special-function operation for both instead
// of an exponential and a reciprocal (the training kernel forms them together).
// The ~2^-11 relative error of tanh.approx is below the BF16 rounding of the
// activation or gradient that follows, and training and inference evaluate
// the same activation.
__device__ __forceinline__ float tanh_fast(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}
__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_fast(h), h);
}

// --------------------------------------------------------------------------
// Features: one CTA per column (block max-reductions for s_n, s_phi).
// --------------------------------------------------------------------------
struct FeatArgs {
  int64_t ncol;
  const int64_t* col_off;
  const double *length, *dt, *v_left, *v_right, *ne, *phi, *n_ion, *T;
  int nsp;
  int val[SDCEF_MAX_SPECIES];
  __nv_bfloat16* X;     // [cells][32]
  // optional targets / guess
  const double *ne_star, *phi_star;
  float* Tgt;           // [cells][2]
  double *ne_g, *phi_g;
  unsigned* chk;        // check word of the bounds-checking build (may be null)
  int mode;             // 0 features, 1 targets
  int comps;            // guess: bit 0 n_e increment, bit 1 phi increment, bit 2 Poisson phi
};

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = sh[0];
  for (int q = 1; q < nw; ++q) r = fmax(r, sh[q]);
  return r;
}

// eps_0 / e (eps_r = 1), the Poisson constant of the column features and of
// the Poisson start (CODATA 2018 values)
constexpr double kKapGuess = 8.8541878128e-12 / 1.602176634e-19;

// Exclusive prefix sum of v over threads t = 0..W-1 (W a multiple of 32, at
// most 32 warps), all of which call it; *total gets the sum over all threads
// (the same value, summed in the same order, on every thread). red holds W/32
// values of type T in shared memory; bar() synchronises the W threads.
template <typename T, class Bar>
__device__ __forceinline__ T excl_scan(T v, int t, int W, T* red, Bar bar, T* total) {
  const int lane = t & 31, w = t >> 5, nw = W >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  T ex = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) ex = T(0);
  if (lane == 31) red[w] = x;
  bar();
  T base = T(0), tot = T(0);
  for (int q = 0; q < nw; ++q) {
    const T r = red[q];
    if (q < w) base += r;
    tot += r;
  }
  bar();
  *total = tot;
  return base + ex;
}

// Root of the Poisson residual of one column (N >= 2 cells),
//   F_phi,i = -n_i + f_i + kappa (G_{i+1/2} - G_{i-1/2}) / h = 0,
// interior faces G = (phi_{i+1} - phi_i)/h, electrode faces
// G_{-1/2} = (9 phi_0 - phi_1 - 8 V_L)/(3h), G_{N-1/2} = (8 V_R - 9 phi_{N-1} + phi_{N-2})/(3h),
// for the cell sources s_i = (h^2/kappa)(n_i - f_i), by two prefix sums instead
// of a tridiagonal solve: with the face differences D_i = h G_{i+1/2}, row i
// reads D_i - D_{i-1} = s_i, so D_i = D_{-1} + S_i (S_i = s_0 + ... + s_i) and
// phi_i = phi_0 + i D_{-1} + T_i (T_i = S_0 + ... + S_{i-1}); the two electrode
// faces give phi_0 = V_L + D_{-1}/2 + S_0/8 and
//   D_{-1} = (8 (V_R - V_L) - S_0 - 8 T_{N-1} - S_{N-2} - 3 S_{N-1}) / (8 N).
// Thread t of W takes a contiguous run of cells; src(i) is s_i (called twice
// per cell and once more for cells 0 and N-1); emit(i, phi_i, S_{i-1}, S_i, D_{-1})
// per cell. Every thread of the W calls it. R is the arithmetic type: double for
// a potential that starts Newton, float for the ion-field features (their
// sources share one sign for cations only, and the features are rounded to BF16).
template <typename R, class Src, class Emit, class Bar>
__device__ __forceinline__ void poisson_column(int N, R vl, R vr, int t, int W, R* red, Bar bar,
                                               Src src, Emit emit) {
  const int run = (N + W - 1) / W;
  const int lo = min(t * run, N), hi = min(lo + run, N);
  R sig = R(0), tau = R(0);
  for (int k = lo; k < hi; ++k) {
    sig += src(k);
    tau += sig;
  }
  R s_tot, t_tot;
  const R s_before = excl_scan<R>(sig, t, W, red, bar, &s_tot);
  const R t_before = excl_scan<R>(R(hi - lo) * s_before + tau, t, W, red, bar, &t_tot);
  const R S0 = src(0), SN1 = s_tot, SN2 = s_tot - src(N - 1), TN1 = t_tot - s_tot;
  const R D = (R(8) * (vr - vl) - S0 - R(8) * TN1 - SN2 - R(3) * SN1) / (R(8) * R(N));
  const R p0 = vl + R(0.5) * D + R(0.125) * S0;
  R S = s_before, T = t_before, pk = fma(R(lo), D, p0);   // pk = phi_0 + k D_{-1}
  for (int k = lo; k < hi; ++k) {
    const R Sn = S + src(k);
    emit(k, pk + T, S, Sn, D);
    T += Sn;
    S = Sn;
    pk += D;
  }
}

// Column-context features 26..29 of a column (once per column, in FP64, so
// that a feature that is 0, as log10(dt) + 5 at dt = 1e-5 s, stays near 0).
struct ColCtx {
  float f[4];
};
__device__ __forceinline__ ColCtx col_context(double sn, int N, double vl, double vr, double dt) {
  ColCtx c;
  c.f[0] = (float)(log10(sn) - 16.0);
  c.f[1] = (float)((vr - vl) * 1e-3);
  c.f[2] = (float)((log2((double)N) - 10.0) * 0.5);
  c.f[3] = (float)(log10(dt) + 5.0);
  return c;
}

// Feature 25: the cell position x_i / L = (i + 1/2) / N.
__device__ __forceinline__ float ctx_pos(int i, int N) {
  return ((float)i + 0.5f) / (float)N;
}

// Features 30, 31 of cell i from the ion potential phi_i = phi_ion,i and the
// face sums of poisson_column: E_ion,i = -(D_{i-1} + D_i) / (2h), in FP32 (the
// features are rounded to BF16).
__device__ __forceinline__ void ion_features(float phi_i, float S_prev, float S_i, float D,
                                             float L2h_isp, float isp, float* f30, float* f31) {
  *f30 = asinhf(phi_i * isp);
  *f31 = asinhf(-(2.0f * D + S_prev + S_i) * L2h_isp);
}

// f_phi = sum_s nu_s n_s of batch cell gi (one unit cation: the density itself)
__device__ __forceinline__ double fphi_cell(const FeatArgs& a, int64_t cells, int64_t gi) {
  if (a.nsp == 1 && a.val[0] == 1) return a.n_ion[gi];
  double q = 0.0;
  for (int s = 0; s < a.nsp; ++s) q += (double)a.val[s] * a.n_ion[(int64_t)s * cells + gi];
  return q;
}

// |x| as an ordered bit pattern (non-negative doubles order as their patterns,
// so maxima run on the integer pipe); a NaN counts as 0, as fmax ignores it
__device__ __forceinline__ long long abs_bits(double x) {
  const long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  return b > 0x7FF0000000000000LL ? 0LL : b;
}

// Per-thread maxima of |n_e|, |f_phi|, |phi| of a column over cells t, t+W, ...
__device__ __forceinline__ void col_maxima(const FeatArgs& a, int64_t cells, int64_t off, int N,
                                           int t, int W, double* m) {
  long long mn = 0, mq = 0, mp = 0;
  for (int i = t; i < N; i += W) {
    mn = max(mn, abs_bits(a.ne[off + i]));
    mq = max(mq, abs_bits(fphi_cell(a, cells, off + i)));
    mp = max(mp, abs_bits(a.phi[off + i]));
  }
  m[0] = __longlong_as_double(mn);
  m[1] = __longlong_as_double(mq);
  m[2] = __longlong_as_double(mp);
}

// The five per-cell quantities of the stencil features of cell i (FP32):
// n_e/s_n, phi/s_phi, f_phi/s_n, T/2000 K and E h/s_phi = -(phi_{i+1} -
// phi_{i-1}) / (2 s_phi) with mirrored neighbours; each value is rounded to
// FP32 and scaled in FP32 (the neighbour difference is taken in FP64).
__device__ __forceinline__ void cell_quantities(const FeatArgs& a, int64_t cells, int64_t off, int N,
                                                int i, float isn, float isp, float* v) {
  const int kp = (i + 1 < N) ? i + 1 : N - 1;
  const int km = (i >= 1) ? i - 1 : 0;
  v[0] = (float)a.ne[off + i] * isn;
  v[1] = (float)a.phi[off + i] * isp;
  v[2] = (float)fphi_cell(a, cells, off + i) * isn;
  v[3] = (float)a.T[off + i] * (1.0f / 2000.0f);
  v[4] = (float)(a.phi[off + kp] - a.phi[off + km]) * (-0.5f * isp);
}

__global__ void feat_kernel(FeatArgs a) {
  __shared__ double sh[32];
  const int64_t c = blockIdx.x;
  if (c >= a.ncol) return;
  const int64_t off = a.col_off[c];
  const int N = (int)(a.col_off[c + 1] - off);
  const int64_t cells = a.col_off[a.ncol];
  if (!SDCEF_CHECK_W(a.chk, off >= 0 && N >= 0 && off + N <= cells, sdcef_chk::kMlpRow)) return;
  double m[3];
  col_maxima(a, cells, off, N, (int)threadIdx.x, (int)blockDim.x, m);
  const double mn = block_max(m[0], sh), mq = block_max(m[1], sh), mp = block_max(m[2], sh);
  const double sn = fmax(fmax(mn, mq), 1.0);
  const double sp = fmax(fmax(mp, fmax(fabs(a.v_left[c]), fabs(a.v_right[c]))), 1.0);
  if (N < 1) return;
  if (a.mode == 1) {
    const double isn = 1.0 / sn, isp = 1.0 / sp;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int64_t gi = off + i;
      a.Tgt[gi * 2 + 0] = (float)((a.ne_star[gi] - a.ne[gi]) * isn);
      a.Tgt[gi * 2 + 1] = (float)((a.phi_star[gi] - a.phi[gi]) * isp);
    }
    return;
  }
  const float isn = (float)(1.0 / sn), isp = (float)(1.0 / sp);
  auto mir = [&](int j) {
    if (j < 0) j = -j - 1;
    if (j >= N) j = 2 * N - 1 - j;
    return min(max(j, 0), N - 1);
  };
  const ColCtx cx = col_context(sn, N, a.v_left[c], a.v_right[c], a.dt[c]);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    __nv_bfloat16* x = a.X + (off + i) * kIn;
    for (int o = -2; o <= 2; ++o) {
      float v[5];
      cell_quantities(a, cells, off, N, mir(i + o), isn, isp, v);
      for (int q = 0; q < 5; ++q) x[5 * (o + 2) + q] = __float2bfloat16(v[q]);
    }
    x[kFeat] = __float2bfloat16(ctx_pos(i, N));
    for (int q = 0; q < 4; ++q) x[kFeat + 1 + q] = __float2bfloat16(cx.f[q]);
    if (N < 2) {
      x[kFeat + 5] = __float2bfloat16(0.0f);
      x[kFeat + 6] = __float2bfloat16(0.0f);
    }
  }
  if (N < 2) return;
  // features 30, 31: the potential and field of the ion charge alone
  __syncthreads();   // sh is free again (last read by block_max)
  // sources -(h^2/kappa) f_i = -(h^2 s_n/kappa) (f_i/s_n), the second factor
  // being the staged FP32 quantity of the stencil features
  const double L = a.length[c];
  const float hks = (float)((L / N) * (L / N) / kKapGuess * sn);
  const float L2h_isp = 0.5f * (float)N * isp;
  poisson_column<float>(
      N, 0.0f, 0.0f, (int)threadIdx.x, (int)blockDim.x, reinterpret_cast<float*>(sh),
      [] { __syncthreads(); },
      [&](int i) { return -hks * ((float)fphi_cell(a, cells, off + i) * isn); },
      [&](int i, float phi_i, float S_prev, float S_i, float D) {
        float f30, f31;
        ion_features(phi_i, S_prev, S_i, D, L2h_isp, isp, &f30, &f31);
        __nv_bfloat16* x = a.X + (off + i) * kIn;
        x[kFeat + 5] = __float2bfloat16(f30);
        x[kFeat + 6] = __float2bfloat16(f31);
      });
}

// Potential of the given electron density: for every column of two or more
// cells, phi = the root of the Poisson residual at n_e = a.ne with the ion
// densities a.n_ion (kappa = eps_0 eps_r / e), written to phi_out; columns of
// one cell are left as they are. One CTA per column (grid-stride over columns).
__global__ void poisson_start_kernel(FeatArgs a, double kappa, double* phi_out) {
  __shared__ double red[32];
  const int64_t cells = a.col_off[a.ncol];
  for (int64_t c = blockIdx.x; c < a.ncol; c += gridDim.x) {
    const int64_t off = a.col_off[c];
    const int N = (int)(a.col_off[c + 1] - off);
    if (!SDCEF_CHECK_W(a.chk, off >= 0 && N >= 0 && off + N <= cells, sdcef_chk::kMlpRow)) continue;
    if (N < 2) continue;
    const double L = a.length[c], hk = (L / N) * (L / N) / kappa;
    poisson_column(
        N, a.v_left[c], a.v_right[c], (int)threadIdx.x, (int)blockDim.x, red,
        [] { __syncthreads(); },
        [&](int i) { return hk * (a.ne[off + i] - fphi_cell(a, cells, off + i)); },
        [&](int i, double phi_i, double, double, double) { phi_out[off + i] = phi_i; });
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// --------------------------------------------------------------------------
// Helpers of the tensor-core kernels: operand staging in the K-major
// core-matrix layout of mlp_tc.cuh (16-byte asynchronous copies).
// --------------------------------------------------------------------------
constexpr int kGemmThreads = 256;   // two warps per TMEM lane quadrant

__device__ __forceinline__ uint32_t pack_u16(uint16_t lo, uint16_t hi) {
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// 16-byte asynchronous global -> shared copy; an invalid chunk is zero-filled
// without reading global memory (the source then only names a valid address)
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::saddr(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}


__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// K-contiguous operand X(r, k) = X[r sr + k]: rows rbase.. rbase + R - 1 (valid
// below rmax), k in [k0, k0 + 8 kc) (valid below kend). Item e fills bytes
// [16 e, 16 e + 16) of S, i.e. core matrix e / 8, row e % 8: asynchronously
// where the chunk's 8 k are all valid or all beyond the matrix, element by
// element where it straddles the edge or the rows are not 16-byte aligned.
template <int NT = kGemmThreads>
__device__ __forceinline__ void stage_k(unsigned char* S, const uint16_t* X, int64_t sr, bool vec,
                                        int64_t rbase, int64_t rmax, int R, int k0, int kend,
                                        int kc, int tid) {
  const int items = R * kc;
#pragma unroll 4
  for (int e = tid; e < items; e += NT) {
    const int grp = e / (8 * kc), w = e - grp * 8 * kc;
    const int64_t gr = rbase + grp * 8 + (w & 7);
    const int gk = k0 + (w >> 3) * 8;
    const bool none = gr >= rmax || gk >= kend;
    if (none || (vec && gk + 8 <= kend)) {
      cp16(S + (size_t)e * 16, none ? (const void*)X : (const void*)(X + gr * sr + gk), !none);
    } else {
      uint16_t u[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) u[j] = (gk + j < kend) ? X[gr * sr + gk + j] : 0;
      *reinterpret_cast<uint4*>(S + (size_t)e * 16) =
          make_uint4(pack_u16(u[0], u[1]), pack_u16(u[2], u[3]), pack_u16(u[4], u[5]),
                     pack_u16(u[6], u[7]));
    }
  }
}


// Chunk-major core-matrix layout of a tile of R rows (the training kernel's X
// and weights): the 8-value chunk c of row r (values 8c .. 8c + 7) at byte
// c R 16 + r 16, so chunk c of all R rows is one 16 R-byte block. A K-major
// descriptor steps along K by R 16 bytes (leading offset) and along the rows by
// 128 bytes (stride offset); read MN-major, K runs along the rows (leading
// offset 128) and M / N along the chunks (stride offset R 16). This is the
// layout a TMA box of 8 values x R rows writes (one box per chunk).
//
// Staging into it by 16-byte asynchronous copies (when the tensor-map copy is
// not available): rows rbase .. rbase + R - 1 (zero at and beyond rmax), kc
// chunks of 8 values of X(r, k) = X[r sr + k].
template <int NT>
__device__ __forceinline__ void stage_cm(unsigned char* S, const uint16_t* X, int64_t sr, bool vec,
                                         int64_t rbase, int64_t rmax, int R, int kc, int tid) {
  for (int e = tid; e < R * kc; e += NT) {
    const int c = e / R, r = e - c * R;
    const int64_t gr = rbase + r;
    const bool none = gr >= rmax;
    if (none || vec) {
      cp16(S + (size_t)e * 16, none ? (const void*)X : (const void*)(X + gr * sr + 8 * c), !none);
    } else {
      uint16_t u[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) u[j] = X[gr * sr + 8 * c + j];
      *reinterpret_cast<uint4*>(S + (size_t)e * 16) =
          make_uint4(pack_u16(u[0], u[1]), pack_u16(u[2], u[3]), pack_u16(u[4], u[5]),
                     pack_u16(u[6], u[7]));
    }
  }
}

// TMA: one box of 8 BF16 values (x: the first value, a multiple of 8) by the
// map's box rows (y: the first row) into dst, completing on mbarrier mb; rows
// beyond the matrix arrive as zeros.
__device__ __forceinline__ void tma_box(unsigned char* dst, const CUtensorMap* map, int x, int y,
                                        uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(tc::saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mb)
      : "memory");
}
__device__ __forceinline__ void expect_tx(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
               : "memory");
}

// --------------------------------------------------------------------------
// Inference forward, all three layers in one launch: a CTA of 256 threads
// takes 128 rows of X, stages X and the BF16 weights in the K-major
// core-matrix layout (cp.async), and chains the layers on the tensor core
// through one 128-column TMEM accumulator. After each hidden layer the 8-warp
// epilogue (two warps per TMEM lane quadrant, each on half of the columns)
// adds the bias and writes H = silu(Z) (BF16) into shared memory as the A
// operand of the next layer; the output layer accumulates in TMEM columns of
// its own and Y (FP32) is the only result written. Every wait on the mbarrier
// is bounded; a CTA whose MMAs do not complete sets the error word and writes
// NaN instead of its results.
// --------------------------------------------------------------------------
struct FwdArgs {
  int64_t n;
  const uint16_t* X;                  // [n][32] BF16
  const uint16_t *w1, *w2, *w3;       // [128][32], [128][128], [2][128] BF16
  const float* p;                     // FP32 parameters (biases)
  float* Y;                           // [n][2] FP32
  int* err;
  int polls;                          // polls of the layer waits (clean-up: the default)
  unsigned* chk;                      // check word of the bounds-checking build (may be null)
};

constexpr uint32_t kFwW1 = kHid * kIn * 2, kFwW2 = kHid * kHid * 2, kFwW3 = 16 * kHid * 2,
                   kFwX = 128 * kIn * 2, kFwH = 128 * kHid * 2;
constexpr uint32_t kFwSmem = kFwW1 + kFwW2 + kFwW3 + kFwX + kFwH;

__global__ void __launch_bounds__(kGemmThreads) fwd_tc_kernel(FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  unsigned char* sW1 = gsm;
  unsigned char* sW2 = sW1 + kFwW1;
  unsigned char* sW3 = sW2 + kFwW2;
  unsigned char* sX = sW3 + kFwW3;
  unsigned char* sH = sX + kFwX;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float sb[2 * kHid + kOut];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  // the CTA's rows inside the batch (before any barrier or allocation)
  if (!SDCEF_CHECK_W(a.chk, m0 < a.n, sdcef_chk::kMlpRow)) return;
  const bool vecX = (reinterpret_cast<uintptr_t>(a.X) & 15) == 0;
  stage_k(sX, a.X, kIn, vecX, m0, a.n, 128, 0, kIn, kIn / 8, tid);
  stage_k(sW1, a.w1, kIn, true, 0, kHid, kHid, 0, kIn, kIn / 8, tid);
  stage_k(sW2, a.w2, kHid, true, 0, kHid, kHid, 0, kHid, kHid / 8, tid);
  stage_k(sW3, a.w3, kHid, true, 0, kOut, 16, 0, kHid, kHid / 8, tid);   // rows 2..15 zero
  cp_commit();
  for (int i = tid; i < kHid; i += kGemmThreads) {
    sb[i] = a.p[kOffB1 + i];
    sb[kHid + i] = a.p[kOffB2 + i];
  }
  if (tid < kOut) sb[2 * kHid + tid] = a.p[kOffB3 + tid];
  if (warp == 0) {   // columns 0..127: hidden layers; 128..143: output layer
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        tc::saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar)) : "memory");
  cp_wait<0>();
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tmem_base, s_mbar = tc::saddr(&mbar);
  const int quad = warp & 3, half = warp >> 2;
  const uint32_t lane_addr = tm + ((uint32_t)(quad * 32) << 16);
  const int r = quad * 32 + lane;                  // this thread's row of the tile (TMEM lane)
  const int64_t row = m0 + r;
  const bool live = row < a.n;
  uint32_t phase = 0;
  // one layer: the MMAs (K = 16 each) by thread 0, a bounded wait by all
  auto layer = [&](const unsigned char* A, const unsigned char* B, int kc, uint32_t idesc,
                   uint32_t dcol) {
    if (tid == 0) {
      tc::fence_after();
      const uint32_t aA = tc::saddr(A), aB = tc::saddr(B);
      for (int kk = 0; kk < kc / 2; ++kk)
        tc::mma(tm + dcol, tc::smem_desc(aA + kk * 256, 128, kc * 128),
                tc::smem_desc(aB + kk * 256, 128, kc * 128), idesc, kk > 0 ? 1u : 0u);
      tc::commit(s_mbar);
    }
    const bool w = tc::wait_phase(s_mbar, phase, a.polls);
    phase ^= 1u;
    const bool bad = __syncthreads_or(!w);
    tc::fence_after();
    return !bad;
  };
  // hidden-layer epilogue: H = silu(acc + bias) into sH
  auto hidden = [&](bool ok, const float* bias) {
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
      float v[32];
      if (ok) {
        tc::ld32(lane_addr + c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __int_as_float(0x7fffffff);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += bias[c0 + j];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sH + tc::cm_off(r, c0 + 8 * q, kHid / 8)) =
            make_uint4(pack_bf16(silu_fast(v[8 * q]), silu_fast(v[8 * q + 1])),
                       pack_bf16(silu_fast(v[8 * q + 2]), silu_fast(v[8 * q + 3])),
                       pack_bf16(silu_fast(v[8 * q + 4]), silu_fast(v[8 * q + 5])),
                       pack_bf16(silu_fast(v[8 * q + 6]), silu_fast(v[8 * q + 7])));
    }
    // sH complete (and the accumulator read) before the next layer's MMAs
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  };
  constexpr uint32_t kIdH = tc::idesc_bf16(128, 128), kIdO = tc::idesc_bf16(128, 16);
  bool ok = layer(sX, sW1, kIn / 8, kIdH, 0);
  hidden(ok, sb);
  if (ok) ok = layer(sH, sW2, kHid / 8, kIdH, 0);
  hidden(ok, sb + kHid);
  if (ok) ok = layer(sH, sW3, kHid / 8, kIdO, 128);
  if (half == 0) {
    const float qnan = __int_as_float(0x7fffffff);
    float y[2] = {qnan, qnan};
    if (ok) tc::ld2(lane_addr + 128, y);
    if (live) {
      a.Y[row * kOut] = y[0] + sb[2 * kHid];
      a.Y[row * kOut + 1] = y[1] + sb[2 * kHid + 1];
    }
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // an MMA may still be in flight: one more bounded wait before TMEM is freed
    tc::wait_phase(s_mbar, phase ^ 1u);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tm));
}

// --------------------------------------------------------------------------
// Training step, forward and backward fused in one persistent kernel. A CTA of
// 512 threads (four warps per TMEM lane quadrant, each on 32 of the columns)
// walks tiles of 128 samples; for each it chains on the tensor core
//   Z1 = X W1^T, Z2 = H1 W2^T, Y = H2 W3^T            (forward, K-major operands)
//   dH1 = dZ2 W2                                        (W2 read MN-major)
//   gW2 += dZ2^T H1, gW3^T += H2^T dY, gW1 += dZ1^T X,
//   gb2 += dZ2^T 1, gb1 += dZ1^T 1                      (contraction over the
//                                                        tile's samples: both
//                                                        operands MN-major)
// with H = silu(Z + b), dY = (Y - T) / n, dZ2 = (dY W3) * silu'(Z2 + b2) and
// dZ1 = dH1 * silu'(Z1 + b1); the hidden-layer epilogues store silu' (BF16)
// beside H from the same tanh, and the backward epilogues turn it into dZ in
// place. Every operand stays in shared memory in the one core-matrix layout
// its producer writes ([sample][unit], 16-byte chunks of 8 units): read
// K-major by the next layer and MN-major (transposed) by the weight and bias
// gradients, so nothing is transposed and no activation leaves the chip. The
// weight and bias gradients accumulate in TMEM across the CTA's tiles, the
// loss and gb3 in shared memory; at the end the CTA writes one partial
// gradient vector (parameter order, then the loss) that the Adam or reduction
// kernel sums over the CTAs in a fixed order, so that a step is deterministic. Every mbarrier wait is bounded; a CTA whose MMAs
// do not complete sets the error word, writes NaN as its partial and frees its
// TMEM after one more bounded wait.
// --------------------------------------------------------------------------
constexpr int kPart = kNParam + 2;   // partial: gradient, loss, one pad (16-byte rows)
static_assert(kPart % 4 == 0, "partials in 16-byte rows");
constexpr int kTrThreads = 512;      // four warps per TMEM lane quadrant

struct TrainArgs {
  int64_t n;
  int ntiles;
  const uint16_t* X;                  // [n][32] BF16
  const uint16_t *w1, *w2, *w3;       // [128][32], [128][128], [2][128] BF16
  const float* p;                     // FP32 parameters (biases)
  const float* T;                     // [n][2] FP32 targets
  float inv_n;                        // 1 / n
  float* part;                        // [gridDim.x][kPart]
  int* err;
  int polls;                          // polls of the main waits (clean-up: the default)
  unsigned* chk;                      // check word of the bounds-checking build (may be null)
  int tma;                            // 1: X and the weights by TMA (tensor maps of the launch)
};

constexpr uint32_t kTrW1 = kHid * kIn * 2, kTrW2 = kHid * kHid * 2, kTrW3 = 16 * kHid * 2,
                   kTrX = 128 * kIn * 2, kTrA = 128 * kHid * 2, kTrN16 = 128 * 16 * 2;
// buffers: W1, W2, W3, X (two), H1, H2, G1 (silu'(Z1), then dZ1), G2 (silu'(Z2),
// then dZ2), dY, ones
constexpr uint32_t kTrOffW2 = kTrW1, kTrOffW3 = kTrOffW2 + kTrW2, kTrOffX = kTrOffW3 + kTrW3,
                   kTrOffH1 = kTrOffX + 2 * kTrX, kTrOffH2 = kTrOffH1 + kTrA,
                   kTrOffG1 = kTrOffH2 + kTrA, kTrOffG2 = kTrOffG1 + kTrA,
                   kTrOffDY = kTrOffG2 + kTrA, kTrOffOne = kTrOffDY + kTrN16,
                   kTrSmem = kTrOffOne + kTrN16;
// TMEM columns: Z1; Z2, then dH1; gW2; gW1; Y; gW3^T; gb2; gb1
constexpr uint32_t kCZ1 = 0, kCZ2 = 128, kCG2 = 256, kCG1 = 384, kCY = 416, kCG3 = 432,
                   kCB2 = 448, kCB1 = 464;
// instruction-descriptor bits: A / B read MN-major (transposed)
constexpr uint32_t kTransA = 1u << 15, kTransB = 1u << 16;

__global__ void __launch_bounds__(kTrThreads, 1)
    train_tc_kernel(TrainArgs a, const __grid_constant__ CUtensorMap mX,
                    const __grid_constant__ CUtensorMap mW1, const __grid_constant__ CUtensorMap mW2,
                    const __grid_constant__ CUtensorMap mW3) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sW1 = tsm;
  unsigned char* sW2 = tsm + kTrOffW2;
  unsigned char* sW3 = tsm + kTrOffW3;
  unsigned char* sX0 = tsm + kTrOffX;
  unsigned char* sH1 = tsm + kTrOffH1;
  unsigned char* sH2 = tsm + kTrOffH2;
  unsigned char* sG1 = tsm + kTrOffG1;   // silu'(Z1 + b1), then dZ1 in place
  unsigned char* sG2 = tsm + kTrOffG2;   // silu'(Z2 + b2), then dZ2 in place
  unsigned char* sDY = tsm + kTrOffDY;
  unsigned char* sOne = tsm + kTrOffOne;
  // mbar[0]: the layers and gW1 / gb1; mbar[1]: dH1; mbar[2]: gW2, gW3, gb2,
  // so that the dZ1 epilogue runs while the weight-gradient MMAs do; mbar[3]:
  // the TMA copies. A barrier never has more than one arrival that is not
  // waited for: a parity wait cannot tell a phase from the one two later
  __shared__ __align__(8) uint64_t mbar[4];
  __shared__ uint32_t tmem_base;
  __shared__ float sb[2 * kHid + kOut];
  __shared__ float sw3[kOut][kHid];   // the BF16 W3 as FP32 (the dY W3 product)
  __shared__ float sacc[4][3];        // per lane quadrant: loss, gb3 (one writer each)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cta = blockIdx.x, G = gridDim.x;
  // The kernel may be launched early behind the previous kernel of the stream
  // (programmatic dependent launch): until griddepcontrol.wait it touches only
  // its own shared and tensor memory, nothing that kernel reads or writes.
  // A CTA without a tile (the host sizes the grid so that there is none)
  // contributes a zero partial.
  if (cta >= a.ntiles) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    (void)SDCEF_CHECK_W(a.chk, false, sdcef_chk::kMlpRow);
    for (int i = tid; i < kPart; i += kTrThreads) a.part[(size_t)cta * kPart + i] = 0.0f;
    return;
  }
  // dY (units 2..15 stay zero) and the ones operand (unit 0 one, the rest zero),
  // [sample][16] in the core-matrix layout; TMEM; the barriers
  for (int i = tid; i < (int)(kTrN16 / 16); i += kTrThreads) {
    reinterpret_cast<uint4*>(sDY)[i] = make_uint4(0u, 0u, 0u, 0u);
    reinterpret_cast<uint4*>(sOne)[i] = make_uint4((i & 8) ? 0u : 0x3F80u, 0u, 0u, 0u);
  }
  if (tid < 12) sacc[tid / 3][tid % 3] = 0.0f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        tc::saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < 4)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[tid])) : "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool vecX = (reinterpret_cast<uintptr_t>(a.X) & 15) == 0;
  auto sX = [&](int t) { return sX0 + (size_t)((t / G) & 1) * kTrX; };
  // X and the weights in the chunk-major layout: by TMA once the barriers
  // exist (below), else by asynchronous copies here
  if (!a.tma) {
    stage_cm<kTrThreads>(sX(cta), a.X, kIn, vecX, (int64_t)cta * 128, a.n, 128, kIn / 8, tid);
    stage_cm<kTrThreads>(sW1, a.w1, kIn, true, 0, kHid, 128, kIn / 8, tid);
    stage_cm<kTrThreads>(sW2, a.w2, kHid, true, 0, kHid, 128, kHid / 8, tid);
    stage_cm<kTrThreads>(sW3, a.w3, kHid, true, 0, kOut, 16, kHid / 8, tid);   // rows 2..15 zero
    cp_commit();
  }
  for (int i = tid; i < kHid; i += kTrThreads) {
    sb[i] = a.p[kOffB1 + i];
    sb[kHid + i] = a.p[kOffB2 + i];
  }
  if (tid < kOut) sb[2 * kHid + tid] = a.p[kOffB3 + tid];
  for (int i = tid; i < kOut * kHid; i += kTrThreads)
    sw3[i / kHid][i % kHid] = __uint_as_float((uint32_t)a.w3[i] << 16);
  cp_wait<0>();
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tmem_base, s_bar[4] = {tc::saddr(&mbar[0]), tc::saddr(&mbar[1]),
                                             tc::saddr(&mbar[2]), tc::saddr(&mbar[3])};
  const int quad = warp & 3, part4 = warp >> 2;   // lane quadrant; 32-column group
  const uint32_t lane_addr = tm + ((uint32_t)(quad * 32) << 16);
  const int r = quad * 32 + lane;   // this thread's row of a tile (TMEM lane)
  const int c0 = part4 * 32;        // this thread's 32 columns of a 128-column result
  const float qnan = __int_as_float(0x7fffffff);
  // commits issued and waited for on each mbarrier (every thread counts them
  // alike); phases complete in issue order, each is waited for in turn
  uint32_t issued[4] = {0u, 0u, 0u, 0u}, waited[4] = {0u, 0u, 0u, 0u};
  int failed = -1;   // the barrier of a wait that gave up
  bool ok = true;
  auto commit = [&](int b) {
    if (tid == 0) tc::commit(s_bar[b]);
    ++issued[b];
  };
  // bounded wait for the oldest unwaited commit of barrier b, by all threads;
  // false once any thread gave up
  auto wait_bar = [&](int b) {
    const bool w = tc::wait_phase(s_bar[b], waited[b] & 1u, a.polls);
    ++waited[b];
    const bool bad = __syncthreads_or(!w);
    tc::fence_after();
    if (bad) failed = b;
    return !bad;
  };
  // K-major operand [rows][kc chunks]: K-step kk (16 values) starts 256 bytes on
  auto kdesc = [](const unsigned char* s, int kk, int kc) {
    return tc::smem_desc(tc::saddr(s) + kk * 256, 128, kc * 128);
  };
  // chunk-major tile of R rows (X, the weights), read K-major or MN-major
  auto ckdesc = [](const unsigned char* s, int kk, int R) {
    return tc::smem_desc(tc::saddr(s) + kk * 2 * R * 16, R * 16, 128);
  };
  auto cmdesc = [](const unsigned char* s, int kk, int R) {
    return tc::smem_desc(tc::saddr(s) + kk * 256, 128, R * 16);
  };
  // X of tile t by TMA: one box of 8 values x 128 rows per chunk
  auto tma_x = [&](int t) {
    if (tid == 0) {
      expect_tx(s_bar[3], kTrX);
      for (int c = 0; c < kIn / 8; ++c) tma_box(sX(t) + c * 2048, &mX, 8 * c, t * 128, s_bar[3]);
    }
    ++issued[3];
  };
  // the same storage read MN-major, K = its rows (the samples): K-step kk
  // starts 2 core-matrix rows (2 kc 128 bytes) on; the leading offset steps
  // along K, the stride offset along M / N (8 units, 128 bytes)
  auto mdesc = [](const unsigned char* s, int kk, int kc) {
    return tc::smem_desc(tc::saddr(s) + kk * 256 * kc, kc * 128, 128);
  };
  constexpr uint32_t kIdH = tc::idesc_bf16(128, 128), kIdO = tc::idesc_bf16(128, 16),
                     kIdG1 = tc::idesc_bf16(128, 32) | kTransA | kTransB,
                     kIdG2 = kIdH | kTransA | kTransB, kIdG16 = kIdO | kTransA | kTransB,
                     kIdDH = kIdH | kTransB;
  if (a.tma) {
    // the weights (W3 as its 16-row zero-padded copy) and the first X tile
    if (tid == 0) {
      expect_tx(s_bar[3], kTrW1 + kTrW2 + kTrW3 + kTrX);
      for (int c = 0; c < kIn / 8; ++c) tma_box(sW1 + c * 2048, &mW1, 8 * c, 0, s_bar[3]);
      for (int c = 0; c < kHid / 8; ++c) tma_box(sW2 + c * 2048, &mW2, 8 * c, 0, s_bar[3]);
      for (int c = 0; c < kHid / 8; ++c) tma_box(sW3 + c * 256, &mW3, 8 * c, 0, s_bar[3]);
      for (int c = 0; c < kIn / 8; ++c)
        tma_box(sX(cta) + c * 2048, &mX, 8 * c, cta * 128, s_bar[3]);
    }
    ++issued[3];
    ok = wait_bar(3);
  }
  // layer 1 of the first tile
  if (ok) {
    if (tid == 0) {
      tc::fence_after();
      for (int kk = 0; kk < kIn / 16; ++kk)
        tc::mma(tm + kCZ1, ckdesc(sX(cta), kk, 128), ckdesc(sW1, kk, 128), kIdH, kk > 0);
    }
    commit(0);
  }
  // hidden-layer epilogue: with t = tanh((acc + bias) / 2), H = silu and
  // G = silu' (sigmoid s = (1 + t) / 2, silu' = s (1 + z (1 - s))) into their operands
  auto hidden = [&](uint32_t col, const float* bias, unsigned char* H, unsigned char* Gd) {
    float v[32];
    tc::ld32(lane_addr + col + c0, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float h[8], g[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float z = v[8 * q + j] + bias[c0 + 8 * q + j];
        const float hz = 0.5f * z, t = tanh_fast(hz);
        const float sg = fmaf(0.5f, t, 0.5f);
        h[j] = fmaf(hz, t, hz);
        g[j] = sg * fmaf(z, 1.0f - sg, 1.0f);
      }
      const uint32_t off = tc::cm_off(r, c0 + 8 * q, kHid / 8);
      *reinterpret_cast<uint4*>(H + off) =
          make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                     pack_bf16(h[6], h[7]));
      *reinterpret_cast<uint4*>(Gd + off) =
          make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                     pack_bf16(g[6], g[7]));
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  };
  // 8 BF16 of an operand chunk <-> FP32
  auto unpack8 = [](const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      f[2 * j] = __uint_as_float(w[j] << 16);
      f[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
    }
  };
  bool first = true;
#pragma unroll 1
  for (int t = cta; t < a.ntiles && ok; t += G) {
    const int64_t row = (int64_t)t * 128 + r;
    const bool live = row < a.n;
    // this row's targets, loaded while the MMAs run
    const float t0 = live ? a.T[row * kOut] : 0.0f, t1 = live ? a.T[row * kOut + 1] : 0.0f;
    // the previous tile's weight gradients, then its gW1 / gb1 and this tile's layer 1
    if (!first && !(ok = wait_bar(2))) break;
    if (!(ok = wait_bar(0))) break;
    // the next tile's X into the other buffer (its last reader, gW1 two tiles
    // back, has completed)
    const int tn = t + G;
    if (tn < a.ntiles) {
      if (a.tma) {
        tma_x(tn);
      } else {
        stage_cm<kTrThreads>(sX(tn), a.X, kIn, vecX, (int64_t)tn * 128, a.n, 128, kIn / 8, tid);
        cp_commit();
      }
    }
    hidden(kCZ1, sb, sH1, sG1);
    if (tid == 0) {
      tc::fence_after();
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc::mma(tm + kCZ2, kdesc(sH1, kk, kHid / 8), ckdesc(sW2, kk, 128), kIdH, kk > 0);
    }
    commit(0);
    if (!(ok = wait_bar(0))) break;
    hidden(kCZ2, sb + kHid, sH2, sG2);
    if (tid == 0) {
      tc::fence_after();
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc::mma(tm + kCY, kdesc(sH2, kk, kHid / 8), ckdesc(sW3, kk, 16), kIdO, kk > 0);
    }
    commit(0);
    if (!(ok = wait_bar(0))) break;
    // output layer and dY = (Y - T) / n (BF16), by every thread for its row;
    // the first column group writes the dY operand and sums the loss and gb3
    float dy0, dy1;
    {
      float y[2];
      tc::ld2(lane_addr + kCY, y);
      const float d0 = live ? y[0] + sb[2 * kHid] - t0 : 0.0f;
      const float d1 = live ? y[1] + sb[2 * kHid + 1] - t1 : 0.0f;
      const float e0 = d0 * a.inv_n, e1 = d1 * a.inv_n;
      const __nv_bfloat16 q0 = __float2bfloat16(e0), q1 = __float2bfloat16(e1);
      dy0 = __bfloat162float(q0);
      dy1 = __bfloat162float(q1);
      if (part4 == 0) {
        *reinterpret_cast<uint4*>(sDY + tc::cm_off(r, 0, 2)) =
            make_uint4((uint32_t)__bfloat16_as_ushort(q0) | ((uint32_t)__bfloat16_as_ushort(q1) << 16),
                       0u, 0u, 0u);
        float l = d0 * d0 + d1 * d1, g0 = e0, g1 = e1;
        for (int o = 16; o > 0; o >>= 1) {
          l += __shfl_xor_sync(0xffffffffu, l, o);
          g0 += __shfl_xor_sync(0xffffffffu, g0, o);
          g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        }
        if (lane == 0) {   // the quadrant's one writer: a fixed summation order
          sacc[quad][0] += l;
          sacc[quad][1] += g0;
          sacc[quad][2] += g1;
        }
      }
    }
    // dZ2 = (dY W3) * silu'(Z2 + b2), in place of silu'
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + 8 * q;
      uint4* pp = reinterpret_cast<uint4*>(sG2 + tc::cm_off(r, c, kHid / 8));
      float g[8];
      unpack8(*pp, g);
#pragma unroll
      for (int j = 0; j < 8; ++j) g[j] *= fmaf(dy1, sw3[1][c + j], dy0 * sw3[0][c + j]);
      *pp = make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                       pack_bf16(g[6], g[7]));
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    // dH1 = dZ2 W2 (over Z2; barrier 1), then gW2 += dZ2^T H1, gW3^T += H2^T dY,
    // gb2 += dZ2^T 1 (barrier 2, waited for before the next tile's epilogues)
    if (tid == 0) {
      tc::fence_after();
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc::mma(tm + kCZ2, kdesc(sG2, kk, kHid / 8), cmdesc(sW2, kk, 128), kIdDH, kk > 0);
    }
    commit(1);
    if (tid == 0) {
      for (int kk = 0; kk < 128 / 16; ++kk) {
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        tc::mma(tm + kCG2, mdesc(sG2, kk, kHid / 8), mdesc(sH1, kk, kHid / 8), kIdG2, acc);
        tc::mma(tm + kCG3, mdesc(sH2, kk, kHid / 8), mdesc(sDY, kk, 2), kIdG16, acc);
        tc::mma(tm + kCB2, mdesc(sG2, kk, kHid / 8), mdesc(sOne, kk, 2), kIdG16, acc);
      }
    }
    commit(2);
    if (!(ok = wait_bar(1))) break;
    // dZ1 = dH1 * silu'(Z1 + b1), in place of silu' (the weight-gradient MMAs
    // read neither)
    {
      float v[32];
      tc::ld32(lane_addr + kCZ2 + c0, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint4* pp = reinterpret_cast<uint4*>(sG1 + tc::cm_off(r, c0 + 8 * q, kHid / 8));
        float g[8];
        unpack8(*pp, g);
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = live ? g[j] * v[8 * q + j] : 0.0f;
        *pp = make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                         pack_bf16(g[6], g[7]));
      }
    }
    if (tn < a.ntiles) {   // the next tile's X has landed
      if (a.tma) {
        if (!(ok = wait_bar(3))) break;
      } else {
        cp_wait<0>();
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    // gW1 += dZ1^T X; gb1 += dZ1^T 1; then the next tile's layer 1 (one commit)
    if (tid == 0) {
      tc::fence_after();
      for (int kk = 0; kk < 128 / 16; ++kk) {
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        tc::mma(tm + kCG1, mdesc(sG1, kk, kHid / 8), cmdesc(sX(t), kk, 128), kIdG1, acc);
        tc::mma(tm + kCB1, mdesc(sG1, kk, kHid / 8), mdesc(sOne, kk, 2), kIdG16, acc);
      }
      if (tn < a.ntiles)
        for (int kk = 0; kk < kIn / 16; ++kk)
          tc::mma(tm + kCZ1, ckdesc(sX(tn), kk, 128), ckdesc(sW1, kk, 128), kIdH, kk > 0);
    }
    commit(0);
    first = false;
  }
  // the last tile's weight gradients and gW1 / gb1 are still to be waited for
  if (ok && waited[2] < issued[2]) ok = wait_bar(2);
  if (ok && waited[0] < issued[0]) ok = wait_bar(0);
  float* part = a.part + (size_t)cta * kPart;
  if (ok) {
    // gW2 [c][h]: TMEM lane c, column h; gW1 [h][f]: lane h, column f;
    // gW3 [o][c]: lane c, column o; gb2, gb1: lane c (h), column 0
    {
      float v[32];
      tc::ld32(lane_addr + kCG2 + c0, v);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(part + kOffW2 + r * kHid + c0 + 4 * q) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (part4 == 0) {
      float v[32];
      tc::ld32(lane_addr + kCG1, v);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(part + kOffW1 + r * kIn + 4 * q) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if (part4 == 1) {
      float y[2];
      tc::ld2(lane_addr + kCG3, y);
      part[kOffW3 + r] = y[0];
      part[kOffW3 + kHid + r] = y[1];
    } else if (part4 == 2) {
      float y[2];
      tc::ld2(lane_addr + kCB2, y);
      part[kOffB2 + r] = y[0];
    } else {
      float y[2];
      tc::ld2(lane_addr + kCB1, y);
      part[kOffB1 + r] = y[0];
    }
    if (tid == 0) {
      float v[3];
      for (int k = 0; k < 3; ++k) v[k] = (sacc[0][k] + sacc[1][k]) + (sacc[2][k] + sacc[3][k]);
      part[kOffB3] = v[1];
      part[kOffB3 + 1] = v[2];
      part[kNParam] = v[0] * 0.5f * a.inv_n;
      part[kNParam + 1] = 0.0f;
    }
  } else {
    if (tid == 0) atomicExch(a.err, 1);
    for (int i = tid; i < kPart; i += kTrThreads) part[i] = qnan;
    // MMAs may still be in flight: bounded waits, in order, for every commit
    // not seen to complete (the one a wait gave up on included) before TMEM is freed
    for (int b = 0; b < 4; ++b)
      for (uint32_t w = waited[b] - (b == failed ? 1u : 0u); w < issued[b]; ++w)
        tc::wait_phase(s_bar[b], w & 1u);
  }
  // the partial is written: the summing kernel may launch (it still waits for
  // this grid to complete before it reads)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm));
}

// Sum of the CTAs' partials: 32 parameters per block of 256 threads, each of
// the 8 row groups of a parameter summing every 8th partial. ADAM: the Adam
// update (and the BF16 weight copies); otherwise g = the gradient. The loss
// (entry kNParam) goes to *loss.
template <bool ADAM>
__global__ void __launch_bounds__(256) part_reduce_kernel(const float* part, int nparts, float* g,
                                                          float* loss, float* p, float* m, float* v,
                                                          float lr, float b1, float b2, float eps,
                                                          float c1, float c2, __nv_bfloat16* w1,
                                                          __nv_bfloat16* w2, __nv_bfloat16* w3) {
  __shared__ float s[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + tx;
  asm volatile("griddepcontrol.wait;" ::: "memory");   // the training kernel has completed
  // the next training step may launch; it waits for this kernel before it reads
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  float acc = 0.0f;
  if (i < kNParam + 1) {
    // four independent loads in flight per thread; the order of the sums is fixed
    float q[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int b = ty;
    for (; b + 24 < nparts; b += 32) {
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] += part[(size_t)(b + 8 * u) * kPart + i];
    }
    for (; b < nparts; b += 8) q[0] += part[(size_t)b * kPart + i];
    acc = (q[0] + q[1]) + (q[2] + q[3]);
  }
  s[ty][tx] = acc;
  __syncthreads();
  if (ty != 0 || i > kNParam) return;
  float gi = 0.0f;
  for (int q = 0; q < 8; ++q) gi += s[q][tx];
  if (i == kNParam) {
    *loss = gi;
    return;
  }
  if (!ADAM) {
    g[i] = gi;
    return;
  }
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (i >= kOffW1 && i < kOffB1) w1[i - kOffW1] = __float2bfloat16(pi);
  else if (i >= kOffW2 && i < kOffB2) w2[i - kOffW2] = __float2bfloat16(pi);
  else if (i >= kOffW3 && i < kOffB3) w3[i - kOffW3] = __float2bfloat16(pi);
}

// --------------------------------------------------------------------------
// Fused guess: features -> 3 layers -> X^n + S_X y, one pass per column, on
// the tcgen05 tensor cores (BF16 operands in shared memory, FP32 accumulators
// in tensor memory); the kernel's organisation is described in mlp_tc.cuh.
// --------------------------------------------------------------------------
// per cell of the stage: the 5 stencil quantities, then features 30 and 31
constexpr int kStageW = 7;

struct GuessArgs {
  FeatArgs f;
  const float* p;                  // FP32 parameters (biases read from here)
  const __nv_bfloat16 *w1, *w2, *w3;
  int* queue;
  float* stage;                    // [cells][kStageW] per-cell values (FP32)
  int64_t stage_cap;               // floats the stage buffer holds
  int* err;                        // set when a tensor-core wait times out
  int polls;                       // polls of the layer waits (clean-up: the default)
};

// TMEM lane -> bias + SiLU -> BF16 row of the next layer's A operand
__device__ __forceinline__ void tc_epilogue(uint32_t taddr, const float* bias, unsigned char* A,
                                            int row, int ch_begin) {
#pragma unroll 1
  for (int ch = ch_begin; ch < ch_begin + 2; ++ch) {
    float v[32];
    tc::ld32(taddr + ch * 32, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k0 = ch * 32 + q * 8;
      uint4 w;
      w.x = pack_bf16(silu_fast(v[q * 8 + 0] + bias[k0 + 0]), silu_fast(v[q * 8 + 1] + bias[k0 + 1]));
      w.y = pack_bf16(silu_fast(v[q * 8 + 2] + bias[k0 + 2]), silu_fast(v[q * 8 + 3] + bias[k0 + 3]));
      w.z = pack_bf16(silu_fast(v[q * 8 + 4] + bias[k0 + 4]), silu_fast(v[q * 8 + 5] + bias[k0 + 5]));
      w.w = pack_bf16(silu_fast(v[q * 8 + 6] + bias[k0 + 6]), silu_fast(v[q * 8 + 7] + bias[k0 + 7]));
      *reinterpret_cast<uint4*>(A + tc::cm_off(row, k0, kHid / 8)) = w;
    }
  }
}

__global__ void __launch_bounds__(tc::kGuessThreads, 2) guess_tc_kernel(GuessArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sW1 = tc_smem;
  unsigned char* sW2 = sW1 + tc::kW1Bytes;
  unsigned char* sW3 = sW2 + tc::kW2Bytes;
  float* sb = reinterpret_cast<float*>(sW3 + tc::kW3Bytes + 2 * tc::kABytes);   // b1, b2, b3
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ double red_s[2][8];
  __shared__ int col_s[2];
  __shared__ float cx_s[2][4];     // features 26..29 of each worker's column
  const FeatArgs& a = g.f;
  const int tid = threadIdx.x;
  // weights in the core-matrix layout; W3 padded with zero rows to N = 16
  for (int e = tid; e < kHid * kIn; e += tc::kGuessThreads)
    *reinterpret_cast<__nv_bfloat16*>(sW1 + tc::cm_off(e / kIn, e % kIn, kIn / 8)) = g.w1[e];
  for (int e = tid; e < kHid * kHid; e += tc::kGuessThreads)
    *reinterpret_cast<__nv_bfloat16*>(sW2 + tc::cm_off(e / kHid, e % kHid, kHid / 8)) = g.w2[e];
  for (int e = tid; e < 16 * kHid; e += tc::kGuessThreads) {
    const int n = e / kHid;
    *reinterpret_cast<__nv_bfloat16*>(sW3 + tc::cm_off(n, e % kHid, kHid / 8)) =
        n < kOut ? g.w3[e] : __float2bfloat16(0.0f);
  }
  for (int e = tid; e < kHid; e += tc::kGuessThreads) {
    sb[e] = g.p[kOffB1 + e];
    sb[kHid + e] = g.p[kOffB2 + e];
  }
  if (tid < kOut) sb[2 * kHid + tid] = g.p[kOffB3 + tid];
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::saddr(&tmem_base)),
                 "n"(tc::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[1])) : "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  // ---- this worker (two warpgroups): warp lw of the worker reads TMEM lane
  // quadrant lw % 4 (rows 32 (lw % 4) + lane of the tile) in column half lw / 4
  const int wg = tid / tc::kWorkerThreads, t = tid % tc::kWorkerThreads, lane = t & 31, lw = t >> 5;
  const int quad = lw & 3, half = lw >> 2, r = quad * 32 + lane;   // r: this thread's tile row
  constexpr int W = tc::kWorkerThreads;
  const int barid = 1 + wg;                       // named barrier of the worker (0 is the CTA's)
  unsigned char* sA = sW3 + tc::kW3Bytes + wg * tc::kABytes;
  double* red = red_s[wg];
  const uint32_t s_mbar = tc::saddr(&mbar[wg]);
  const uint32_t tm = tmem_base;
  const uint32_t dcol = tm + 128u * (uint32_t)wg;                     // accumulator columns
  const uint32_t lane_addr = dcol + ((uint32_t)(quad * 32) << 16);   // TMEM lane of row r
  const uint32_t aA = tc::saddr(sA), aW1 = tc::saddr(sW1), aW2 = tc::saddr(sW2),
                 aW3 = tc::saddr(sW3);
  constexpr uint32_t kId1 = tc::idesc_bf16(128, 128), kId3 = tc::idesc_bf16(128, 16);
  const int64_t cells = a.col_off[a.ncol];
  uint32_t phase = 0;
  bool failed = false;
  // the worker's first thread issues a layer once the A operand is published;
  // everyone waits, and the outcome is made uniform over the worker
  auto run_layer = [&](int layer) -> bool {
    tc::fence_async_smem();
    tc::fence_before();
    tc::bar(barid, W);
    if (t == 0) {
      tc::fence_after();
      if (layer == 1) {
#pragma unroll
        for (int k = 0; k < kIn / 16; ++k)
          tc::mma(dcol, tc::smem_desc(aA + k * 256, 128, (kIn / 8) * 128),
                  tc::smem_desc(aW1 + k * 256, 128, (kIn / 8) * 128), kId1, k > 0);
      } else {
        const uint32_t b = layer == 2 ? aW2 : aW3;
#pragma unroll
        for (int k = 0; k < kHid / 16; ++k)
          tc::mma(dcol, tc::smem_desc(aA + k * 256, 128, (kHid / 8) * 128),
                  tc::smem_desc(b + k * 256, 128, (kHid / 8) * 128), layer == 2 ? kId1 : kId3,
                  k > 0);
      }
      tc::commit(s_mbar);
    }
    const bool ok = tc::wait_phase(s_mbar, phase, g.polls);
    phase ^= 1u;
    const bool bad = tc::bar_or(barid, W, !ok);
    tc::fence_after();
    return !bad;
  };
  for (;;) {
    tc::bar(barid, W);
    if (t == 0) col_s[wg] = atomicAdd(g.queue, 1);
    tc::bar(barid, W);
    const int64_t c = col_s[wg];
    if (c >= a.ncol || failed) break;
    const int64_t off = a.col_off[c];
    const int N = (int)(a.col_off[c + 1] - off);
    // the column inside the batch and its staged features inside the stage
    // buffer (uniform over the worker: a failed column is skipped by all)
    if (!SDCEF_CHECK_W(a.chk, off >= 0 && N >= 0 && off + N <= cells &&
                                  (off + N) * kStageW <= g.stage_cap,
                       sdcef_chk::kMlpStage))
      continue;
    double mx[3];
    col_maxima(a, cells, off, N, t, W, mx);
    for (int k = 0; k < 3; ++k) {
      double v = mx[k];
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) red[lw] = v;
      tc::bar(barid, W);
      mx[k] = fmax(fmax(fmax(red[0], red[1]), fmax(red[2], red[3])),
                   fmax(fmax(red[4], red[5]), fmax(red[6], red[7])));
      tc::bar(barid, W);
    }
    const double sn = fmax(fmax(mx[0], mx[1]), 1.0);
    const double sp = fmax(fmax(mx[2], fmax(fabs(a.v_left[c]), fabs(a.v_right[c]))), 1.0);
    if (N < 1) continue;
    const float isn = (float)(1.0 / sn), isp = (float)(1.0 / sp);
    // the five per-cell quantities of the stencil features and features 30, 31
    // (ion potential and field, poisson_column), staged once in FP32
    float* st = g.stage + off * kStageW;
    if (t == 0) {
      const ColCtx cx = col_context(sn, N, a.v_left[c], a.v_right[c], a.dt[c]);
      for (int q = 0; q < 4; ++q) cx_s[wg][q] = cx.f[q];
    }
    auto wbar = [&] { tc::bar(barid, W); };
    for (int i = t; i < N; i += W) {
      float v[5];
      cell_quantities(a, cells, off, N, i, isn, isp, v);
#pragma unroll
      for (int q = 0; q < 5; ++q) st[i * kStageW + q] = v[q];
      if (N < 2) st[i * kStageW + 5] = st[i * kStageW + 6] = 0.0f;
    }
    if (N >= 2) {
      tc::bar(barid, W);   // the staged quantities of every cell of the column
      const double L = a.length[c];
      const float hks = (float)((L / N) * (L / N) / kKapGuess * sn);
      const float L2h_isp = 0.5f * (float)N * isp;
      poisson_column<float>(
          N, 0.0f, 0.0f, t, W, reinterpret_cast<float*>(red), wbar,
          [&](int i) { return -hks * st[i * kStageW + 2]; },
          [&](int i, float phi_i, float S_prev, float S_i, float D) {
            ion_features(phi_i, S_prev, S_i, D, L2h_isp, isp, &st[i * kStageW + 5],
                         &st[i * kStageW + 6]);
          });
    }
    tc::bar(barid, W);
    auto mir = [&](int j) {
      if (j < 0) j = -j - 1;
      if (j >= N) j = 2 * N - 1 - j;
      return min(max(j, 0), N - 1);
    };
    // row r of A: the 25 stencil features of cell i (f = 5 o + q: quantity q
    // of cell i + o - 2) and the 7 of the column context; thread half H of row
    // r builds features 16 H .. 16 H + 15 (the feature index is a compile-time
    // constant in each instance)
    auto build_row = [&](int i, auto hc) {
      constexpr int H = decltype(hc)::value;
#pragma unroll
      for (int cl = 0; cl < 2; ++cl) {
        const int ch = 2 * H + cl;
        float f8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int f = ch * 8 + u;
          if (f < kFeat) f8[u] = st[mir(i + f / 5 - 2) * kStageW + f % 5];
          else if (f == kFeat) f8[u] = ctx_pos(i, N);
          else if (f < kFeat + 5) f8[u] = cx_s[wg][f - kFeat - 1];
          else f8[u] = st[i * kStageW + (f - kFeat)];
        }
        uint4 w;
        w.x = pack_bf16(f8[0], f8[1]);
        w.y = pack_bf16(f8[2], f8[3]);
        w.z = pack_bf16(f8[4], f8[5]);
        w.w = pack_bf16(f8[6], f8[7]);
        uint32_t ao = tc::cm_off(r, ch * 8, kIn / 8);
        if (!SDCEF_CHECK_W(a.chk, ao + 16 <= tc::kABytes, sdcef_chk::kMlpSmem)) ao = 0;
        *reinterpret_cast<uint4*>(sA + ao) = w;
      }
    };
    const bool poisson = (a.comps & 4) && N >= 2;
    for (int r0 = 0; r0 < N; r0 += tc::kTile) {
      const int i = min(r0 + r, N - 1);
      if (half == 0) build_row(i, std::integral_constant<int, 0>{});
      else build_row(i, std::integral_constant<int, 1>{});
      bool ok = run_layer(1);
      if (ok) {
        tc_epilogue(lane_addr, sb, sA, r, 2 * half);
        ok = run_layer(2);
      }
      if (ok) {
        tc_epilogue(lane_addr, sb + kHid, sA, r, 2 * half);
        ok = run_layer(3);
      }
      float y[2] = {NAN, NAN};
      if (ok && half == 0) tc::ld2(lane_addr, y);
      const int row = r0 + r;
      if (half == 0 && row < N) {
        const int64_t gi = off + row;
        const float yn = y[0] + sb[2 * kHid], yp = y[1] + sb[2 * kHid + 1];
        a.ne_g[gi] = a.ne[gi] + ((a.comps & 1) ? sn * (double)yn : (ok ? 0.0 : (double)NAN));
        if (!poisson)
          a.phi_g[gi] = a.phi[gi] + ((a.comps & 6) == 2 ? sp * (double)yp : 0.0);
      }
      // the next tile's layer 1 overwrites these TMEM columns after the barrier
      tc::fence_before();
      if (!ok) {
        failed = true;
        if (t == 0) atomicExch(g.err, 1);
        // an MMA may still be in flight: one more bounded wait before TMEM is freed
        tc::wait_phase(s_mbar, phase ^ 1u);
        break;
      }
    }
    // the potential at the guessed n_e: root of the Poisson residual
    // (uniform over the worker: failed and poisson are)
    if (poisson && !failed) {
      tc::bar(barid, W);   // every n_e of the column written
      const double L = a.length[c], hk = (L / N) * (L / N) / kKapGuess;
      poisson_column(
          N, a.v_left[c], a.v_right[c], t, W, red, wbar,
          [&](int i) { return hk * (a.ne_g[off + i] - fphi_cell(a, cells, off + i)); },
          [&](int i, double phi_i, double, double, double) { a.phi_g[off + i] = phi_i; });
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm),
                 "n"(tc::kTmemCols));
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* w1, __nv_bfloat16* w2,
                               __nv_bfloat16* w3) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
    if (i >= kOffW1 && i < kOffB1) w1[i - kOffW1] = __float2bfloat16(p[i]);
    else if (i >= kOffW2 && i < kOffB2) w2[i - kOffW2] = __float2bfloat16(p[i]);
    else if (i >= kOffW3 && i < kOffB3) w3[i - kOffW3] = __float2bfloat16(p[i]);
  }
}

}  // namespace

// ============================================================================
struct sdcef_mlp {
  int64_t max_rows;
  cudaStream_t st;
  float *p, *g, *m, *v;                 // FP32 parameters, gradients, Adam moments
  __nv_bfloat16 *w1, *w2, *w3;          // BF16 weight copies (W3 zero-padded to 16 rows)
  CUtensorMap mw[3];                    // tensor maps of W1, W2, W3 (TMA boxes of 8 values)
  int tma_w;                            // the weight maps could be encoded
  float *Y, *loss;                      // output, loss (FP32)
  float* part;                          // [sms][kPart] per-CTA partials of the training kernel
  __nv_bfloat16* X;                     // [max_rows][32] staging area of the guess
  int step;
  int launches;
  int sms;                              // multiprocessors of the device
  int polls;                            // polls of the kernels' main bounded waits
};

namespace {
// check word of the bounds-checking build: a spare word of the loss buffer
unsigned* mlp_chk(sdcef_mlp* h) { return reinterpret_cast<unsigned*>(h->loss) + 6; }
}  // namespace

namespace {

int cuda_fail(cudaError_t e) { return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e)); }

// Tensor map of a row-major BF16 matrix [rows][cols], read in boxes of 8
// values (16 bytes) x box_rows rows: box c of a tile lands as box_rows 16-byte
// rows, the chunk-major layout of the training kernel; rows beyond the matrix
// arrive as zeros. False if it cannot be encoded (the kernel then stages by
// cp.async).
bool tma_rows(CUtensorMap* m, const void* base, int64_t rows, int cols, int box_rows) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  memset(m, 0, sizeof(*m));
  if (!encode || (reinterpret_cast<uintptr_t>(base) & 15) || ((cols * 2) & 15) || rows < 1 ||
      cols % 8)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {8, (cuuint32_t)box_rows}, estr[2] = {1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// forward through the three layers for n rows of X: Y (FP32 [n][2])
cudaError_t forward(sdcef_mlp* h, const __nv_bfloat16* X, int64_t n, float* Y) {
  if (n <= 0) return cudaSuccess;
  FwdArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.X = reinterpret_cast<const uint16_t*>(X);
  a.w1 = reinterpret_cast<const uint16_t*>(h->w1);
  a.w2 = reinterpret_cast<const uint16_t*>(h->w2);
  a.w3 = reinterpret_cast<const uint16_t*>(h->w3);
  a.p = h->p;
  a.Y = Y;
  a.err = (int*)h->loss + 5;
  a.polls = h->polls;
  a.chk = mlp_chk(h);
  fwd_tc_kernel<<<(unsigned)((n + 127) / 128), kGemmThreads, kFwSmem, h->st>>>(a);
  ++h->launches;
  return cudaGetLastError();
}

// A launch that may start while the previous kernel of the stream finishes
// (programmatic dependent launch; the kernel waits for it with
// griddepcontrol.wait before it reads that kernel's results). Falls back to a
// plain launch where the attribute is refused.
template <typename... KT, typename... AT>
cudaError_t launch_early(void (*k)(KT...), unsigned grid, unsigned block, size_t smem,
                         cudaStream_t st, AT... args) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k, args...) == cudaSuccess) return cudaSuccess;
  (void)cudaGetLastError();
  k<<<grid, block, smem, st>>>(args...);
  return cudaGetLastError();
}

// forward, loss and backward over n rows (train_tc_kernel), then the sum of
// the CTAs' partials: the Adam step (adam) or the gradient into h->g; the loss
// into h->loss[0]. The grid spreads the 128-row tiles evenly over at most one
// CTA per multiprocessor.
cudaError_t train(sdcef_mlp* h, const __nv_bfloat16* X, const float* T, int64_t n, bool adam,
                  float lr) {
  const int64_t ntiles = (n + 127) / 128;
  const int64_t per = (ntiles + h->sms - 1) / h->sms;
  const int grid = (int)((ntiles + per - 1) / per);
  TrainArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.ntiles = (int)ntiles;
  a.X = reinterpret_cast<const uint16_t*>(X);
  a.w1 = reinterpret_cast<const uint16_t*>(h->w1);
  a.w2 = reinterpret_cast<const uint16_t*>(h->w2);
  a.w3 = reinterpret_cast<const uint16_t*>(h->w3);
  a.p = h->p;
  a.T = T;
  a.inv_n = 1.0f / (float)n;
  a.part = h->part;
  a.err = (int*)h->loss + 5;
  a.polls = h->polls;
  a.chk = mlp_chk(h);
  CUtensorMap mx;
  a.tma = (h->tma_w && tma_rows(&mx, X, n, kIn, 128)) ? 1 : 0;
  cudaError_t e = launch_early(train_tc_kernel, (unsigned)grid, kTrThreads, kTrSmem, h->st, a, mx,
                               h->mw[0], h->mw[1], h->mw[2]);
  ++h->launches;
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((kNParam + 1 + 31) / 32);
  if (adam) {
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)h->step), c2 = 1.0f - powf(b2, (float)h->step);
    e = launch_early(part_reduce_kernel<true>, blocks, 256, 0, h->st, (const float*)h->part, grid,
                     h->g, h->loss, h->p, h->m, h->v, lr, b1, b2, 1e-8f, c1, c2, h->w1, h->w2,
                     h->w3);
  } else {
    e = launch_early(part_reduce_kernel<false>, blocks, 256, 0, h->st, (const float*)h->part, grid,
                     h->g, h->loss, (float*)nullptr, (float*)nullptr, (float*)nullptr, 0.0f, 0.0f,
                     0.0f, 0.0f, 0.0f, 0.0f, (__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr,
                     (__nv_bfloat16*)nullptr);
  }
  ++h->launches;
  return e;
}

FeatArgs feat_args(const sdcef_batch* b) {
  FeatArgs a;
  memset(&a, 0, sizeof(a));
  a.ncol = b->ncol;
  a.col_off = b->col_off;
  a.length = b->length;
  a.dt = b->dt;
  a.v_left = b->v_left;
  a.v_right = b->v_right;
  a.ne = b->ne_old;
  a.phi = b->phi_old;
  a.n_ion = b->n_ion;
  a.T = b->T;
  a.nsp = b->n_species;
  for (int s = 0; s < b->n_species; ++s) a.val[s] = b->valence[s];
  return a;
}

int check_batch(const sdcef_batch* b) {
  if (!b || b->ncol < 0) return report_error(SDCEF_ERR_INVALID, "mlp: batch is NULL or ncol < 0");
  if (b->ncol == 0) return SDCEF_SUCCESS;
  if (!b->col_off || !b->v_left || !b->v_right || !b->ne_old || !b->phi_old || !b->T)
    return report_error(SDCEF_ERR_INVALID, "mlp: required batch pointer is NULL");
  if (b->n_species < 0 || b->n_species > SDCEF_MAX_SPECIES || (b->n_species > 0 && (!b->valence || !b->n_ion)))
    return report_error(SDCEF_ERR_INVALID, "mlp: ion species arguments");
  return SDCEF_SUCCESS;
}

}  // namespace

extern "C" {

int sdcef_mlp_create(sdcef_mlp** out, int64_t max_rows, void* stream) {
  if (!out || max_rows < 1) return report_error(SDCEF_ERR_INVALID, "mlp_create: bad arguments");
  sdcef_mlp* h = new sdcef_mlp();
  memset(h, 0, sizeof(*h));
  h->max_rows = max_rows;
  h->polls = tc::kWaitPolls;
  h->st = (cudaStream_t)stream;
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kFwSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTrSmem);
    if (e != cudaSuccess) {
      delete h;
      return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
    }
    h->sms = std::max(h->sms, 1);
  }
  const size_t R = (size_t)max_rows;
  struct Alloc { void** p; size_t bytes; } al[] = {
      {(void**)&h->p, kNParam * 4}, {(void**)&h->g, kNParam * 4}, {(void**)&h->m, kNParam * 4},
      {(void**)&h->v, kNParam * 4}, {(void**)&h->w1, kHid * kIn * 2}, {(void**)&h->w2, kHid * kHid * 2},
      {(void**)&h->w3, 16 * kHid * 2}, {(void**)&h->Y, R * kOut * 4}, {(void**)&h->loss, 64},
      {(void**)&h->part, (size_t)h->sms * kPart * 4}, {(void**)&h->X, R * kIn * 2}};
  for (auto& a : al) {
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e == cudaSuccess) e = cudaMemset(*a.p, 0, a.bytes);
    if (e != cudaSuccess) {
      for (auto& b : al) if (*b.p) cudaFree(*b.p);
      delete h;
      return report_error(SDCEF_ERR_NOMEM, cudaGetErrorString(e));
    }
  }
  h->tma_w = tma_rows(&h->mw[0], h->w1, kHid, kIn, 128) && tma_rows(&h->mw[1], h->w2, kHid, kHid, 128) &&
             tma_rows(&h->mw[2], h->w3, 16, kHid, 16);
  *out = h;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_destroy(sdcef_mlp* h) {
  if (!h) return SDCEF_SUCCESS;
  cudaStreamSynchronize(h->st);
  void* ps[] = {h->p, h->g, h->m, h->v, h->w1, h->w2, h->w3, h->Y, h->loss, h->part, h->X};
  for (void* p : ps) cudaFree(p);
  delete h;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_set_params(sdcef_mlp* h, const float* params_host) {
  if (!h || !params_host) return report_error(SDCEF_ERR_INVALID, "mlp_set_params: NULL");
  cudaError_t e = cudaMemcpyAsync(h->p, params_host, kNParam * 4, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->m, 0, kNParam * 4, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->v, 0, kNParam * 4, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->g, 0, kNParam * 4, h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  to_bf16_kernel<<<64, 256, 0, h->st>>>(h->p, h->w1, h->w2, h->w3);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  h->step = 0;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_get_params(sdcef_mlp* h, float* params_host) {
  if (!h || !params_host) return report_error(SDCEF_ERR_INVALID, "mlp_get_params: NULL");
  cudaError_t e = cudaMemcpyAsync(params_host, h->p, kNParam * 4, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_get_state(sdcef_mlp* h, float* params_host, float* m_host, float* v_host,
                        int64_t* step) {
  if (!h || !params_host || !m_host || !v_host || !step)
    return report_error(SDCEF_ERR_INVALID, "mlp_get_state: NULL");
  cudaError_t e = cudaMemcpyAsync(params_host, h->p, kNParam * 4, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m_host, h->m, kNParam * 4, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v_host, h->v, kNParam * 4, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  *step = h->step;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_set_state(sdcef_mlp* h, const float* params_host, const float* m_host,
                        const float* v_host, int64_t step) {
  if (!h || !params_host || !m_host || !v_host || step < 0 || step > 0x7fffffff)
    return report_error(SDCEF_ERR_INVALID, "mlp_set_state: bad arguments");
  cudaError_t e = cudaMemcpyAsync(h->p, params_host, kNParam * 4, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->m, m_host, kNParam * 4, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->v, v_host, kNParam * 4, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->g, 0, kNParam * 4, h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  to_bf16_kernel<<<64, 256, 0, h->st>>>(h->p, h->w1, h->w2, h->w3);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  h->step = (int)step;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_features(sdcef_mlp* h, const sdcef_batch* b, void* X_bf16) {
  if (!h || !X_bf16) return report_error(SDCEF_ERR_INVALID, "mlp_features: NULL");
  int rc = check_batch(b);
  if (rc || b->ncol == 0) return rc;
  FeatArgs a = feat_args(b);
  a.chk = mlp_chk(h);
  a.X = (__nv_bfloat16*)X_bf16;
  a.mode = 0;
  feat_kernel<<<(unsigned)b->ncol, 128, 0, h->st>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_targets(sdcef_mlp* h, const sdcef_batch* b, const double* ne_star,
                      const double* phi_star, float* targets) {
  if (!h || !ne_star || !phi_star || !targets) return report_error(SDCEF_ERR_INVALID, "mlp_targets: NULL");
  int rc = check_batch(b);
  if (rc || b->ncol == 0) return rc;
  FeatArgs a = feat_args(b);
  a.chk = mlp_chk(h);
  a.ne_star = ne_star;
  a.phi_star = phi_star;
  a.Tgt = targets;
  a.mode = 1;
  feat_kernel<<<(unsigned)b->ncol, 128, 0, h->st>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_forward(sdcef_mlp* h, const void* X_bf16, int64_t n, float* Y) {
  if (!h || !X_bf16 || n < 0) return report_error(SDCEF_ERR_INVALID, "mlp_forward: bad arguments");
  if (n > h->max_rows) return report_error(SDCEF_ERR_CAPACITY, "mlp_forward: n exceeds max_rows");
  if (n == 0) return SDCEF_SUCCESS;
  h->launches = 0;
  cudaError_t e = forward(h, (const __nv_bfloat16*)X_bf16, n, Y ? Y : h->Y);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_grad(sdcef_mlp* h, const void* X_bf16, const float* T, int64_t n, float* grads,
                   float* loss) {
  if (!h || !X_bf16 || !T || n < 1) return report_error(SDCEF_ERR_INVALID, "mlp_grad: bad arguments");
  if (n > h->max_rows) return report_error(SDCEF_ERR_CAPACITY, "mlp_grad: n exceeds max_rows");
  h->launches = 0;
  cudaError_t e = train(h, (const __nv_bfloat16*)X_bf16, T, n, false, 0.0f);
  if (e == cudaSuccess && grads)
    e = cudaMemcpyAsync(grads, h->g, kNParam * 4, cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, h->loss, 4, cudaMemcpyDeviceToDevice, h->st);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_train_step(sdcef_mlp* h, const void* X_bf16, const float* T, int64_t n, float lr,
                         float* loss) {
  if (!h || !X_bf16 || !T || n < 1 || !(lr > 0.0f))
    return report_error(SDCEF_ERR_INVALID, "mlp_train_step: bad arguments");
  if (n > h->max_rows) return report_error(SDCEF_ERR_CAPACITY, "mlp_train_step: n exceeds max_rows");
  h->launches = 0;
  cudaError_t e = train(h, (const __nv_bfloat16*)X_bf16, T, n, true, lr);
  if (e != cudaSuccess) return cuda_fail(e);
  if (loss) e = cudaMemcpyAsync(loss, h->loss, 4, cudaMemcpyDeviceToDevice, h->st);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_guess(sdcef_mlp* h, const sdcef_batch* b, int64_t ncells, int components,
                    double* ne_guess, double* phi_guess) {
  if (!h || !ne_guess || !phi_guess || ncells < 0 || components < 0 || components > 7)
    return report_error(SDCEF_ERR_INVALID, "mlp_guess: bad arguments");
  int rc = check_batch(b);
  if (rc || b->ncol == 0) return rc;
  h->launches = 0;
  GuessArgs g;
  memset(&g, 0, sizeof(g));
  g.f = feat_args(b);
  g.f.chk = mlp_chk(h);
  g.f.comps = components;
  g.f.ne_g = ne_guess;
  g.f.phi_g = phi_guess;
  g.p = h->p;
  g.w1 = h->w1;
  g.w2 = h->w2;
  g.w3 = h->w3;
  g.queue = (int*)h->loss + 4;   // spare words of the loss buffer
  g.err = (int*)h->loss + 5;
  g.polls = h->polls;
  if (ncells > h->max_rows || ncells * kStageW > h->max_rows * (kIn / 2))
    return report_error(SDCEF_ERR_CAPACITY, "mlp_guess: ncells exceeds max_rows");
  g.stage = (float*)h->X;        // [cells][kStageW] FP32 inside the [max_rows][32] BF16 buffer
  g.stage_cap = h->max_rows * (kIn / 2);
  cudaError_t e = cudaMemsetAsync(g.queue, 0, sizeof(int), h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // two CTAs (four column workers) per SM: 2 x 256 TMEM columns fill the SM's tensor memory
  const int grid = (int)std::min<int64_t>((b->ncol + 1) / 2, (int64_t)std::max(sms, 1) * 2);
  e = cudaFuncSetAttribute(guess_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc::kSmemBytes);
  if (e != cudaSuccess) return cuda_fail(e);
  guess_tc_kernel<<<grid, tc::kGuessThreads, tc::kSmemBytes, h->st>>>(g);
  ++h->launches;
  e = cudaGetLastError();
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_last_launch_count(const sdcef_mlp* h) { return h ? h->launches : 0; }

}  // extern "C"

namespace sdcef_impl {
// The potential consistent with an electron density (poisson_start_kernel),
// enqueued on st: batch geometry, electrode potentials and valences from b,
// ion densities n_ion ([n_species][cells], device), n_e ne (device); phi_out
// (device) may alias nothing the kernel reads. The SDC sweep starts its later
// iterations from it.
cudaError_t launch_poisson_start(const sdcef_batch* b, const double* ne, const double* n_ion,
                                 double kappa, double* phi_out, cudaStream_t st) {
  FeatArgs a = feat_args(b);
  a.ne = ne;
  a.n_ion = n_ion;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(b->ncol, (int64_t)std::max(sms, 1) * 8);
  poisson_start_kernel<<<grid, 256, 0, st>>>(a, kappa, phi_out);
  return cudaGetLastError();
}
}  // namespace sdcef_impl

extern "C" {

int sdcef_mlp_check_word(sdcef_mlp* h, unsigned* word) {
  if (!h || !word) return report_error(SDCEF_ERR_INVALID, "mlp_check_word: NULL argument");
  unsigned w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, mlp_chk(h), sizeof(unsigned), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(mlp_chk(h), 0, sizeof(unsigned), h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  *word = w;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_set_wait_polls(sdcef_mlp* h, int polls) {
  if (!h) return report_error(SDCEF_ERR_INVALID, "mlp_set_wait_polls: NULL");
  h->polls = polls < 0 ? tc::kWaitPolls : polls;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_check(sdcef_mlp* h) {
  if (!h) return report_error(SDCEF_ERR_INVALID, "mlp_check: NULL");
  int* word = (int*)h->loss + 5;
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, word, sizeof(int), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(word, 0, sizeof(int), h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  return flag ? report_error(SDCEF_ERR_CUDA, "mlp: a tensor-core wait timed out (outputs set to NaN)")
              : SDCEF_SUCCESS;
}

}  // extern "C"
