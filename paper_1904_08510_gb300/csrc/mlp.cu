// Learned Newton initial guess: feature extraction; training on the tcgen05
// tensor cores (BF16 operands, FP32 accumulators in TMEM): the three-layer
// forward fused in one kernel, the MSE loss, backpropagation through a BF16
// GEMM with fused SiLU-derivative and split-K weight-gradient epilogues, and
// Adam; and the fused inference kernel (mlp_tc.cuh) that assembles the
// guess. The network maps the
// 5-cell stencil features of a cell to the scaled Newton increment
// ((n* - n^n)/s_n, (phi* - phi^n)/s_phi); the JFNK of Algorithm 2 then starts
// from X^n + S_X y instead of X^n and still decides convergence.
//
// Shapes: 32 (25 features, zero-padded) -> 128 -> 128 -> 2, SiLU activations.
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
// s = (1 + tanh(z/2)) / 2 -- one special-function operation each instead of an
// exponential and a reciprocal. The ~2^-11 relative error of tanh.approx is
// below the BF16 rounding of the activation or gradient that follows, and
// training and inference evaluate the same activation.
__device__ __forceinline__ float tanh_fast(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}
__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_fast(h), h);
}
__device__ __forceinline__ float silu_grad(float z) {
  const float s = fmaf(0.5f, tanh_fast(0.5f * z), 0.5f);
  return s * fmaf(z, 1.0f - s, 1.0f);
}

// --------------------------------------------------------------------------
// Features: one CTA per column (block max-reductions for s_n, s_phi).
// --------------------------------------------------------------------------
struct FeatArgs {
  int64_t ncol;
  const int64_t* col_off;
  const double *v_left, *v_right, *ne, *phi, *n_ion, *T;
  int nsp;
  int val[SDCEF_MAX_SPECIES];
  __nv_bfloat16* X;     // [cells][32]
  // optional targets / guess
  const double *ne_star, *phi_star;
  float* Tgt;           // [cells][2]
  const float* Y;       // [cells][2] network output (guess mode)
  double *ne_g, *phi_g;
  unsigned* chk;        // check word of the bounds-checking build (may be null)
  int mode;             // 0 features, 1 targets, 2 guess
  int comps;            // guess: bit 0 applies the n_e increment, bit 1 the phi increment
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

__global__ void feat_kernel(FeatArgs a) {
  __shared__ double sh[32];
  const int64_t c = blockIdx.x;
  if (c >= a.ncol) return;
  const int64_t off = a.col_off[c];
  const int N = (int)(a.col_off[c + 1] - off);
  const int64_t cells = a.col_off[a.ncol];
  if (!SDCEF_CHECK_W(a.chk, off >= 0 && N >= 0 && off + N <= cells, sdcef_chk::kMlpRow)) return;
  auto fphi = [&](int i) {
    double q = 0.0;
    for (int s = 0; s < a.nsp; ++s) q += (double)a.val[s] * a.n_ion[(int64_t)s * cells + off + i];
    return q;
  };
  double mn = 0.0, mq = 0.0, mp = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    mn = fmax(mn, fabs(a.ne[off + i]));
    mq = fmax(mq, fabs(fphi(i)));
    mp = fmax(mp, fabs(a.phi[off + i]));
  }
  mn = block_max(mn, sh);
  mq = block_max(mq, sh);
  mp = block_max(mp, sh);
  const double sn = fmax(fmax(mn, mq), 1.0);
  const double sp = fmax(fmax(mp, fmax(fabs(a.v_left[c]), fabs(a.v_right[c]))), 1.0);
  const double isn = 1.0 / sn, isp = 1.0 / sp;
  if (N < 1) return;
  auto mir = [&](int j) {
    if (j < 0) j = -j - 1;
    if (j >= N) j = 2 * N - 1 - j;
    return min(max(j, 0), N - 1);
  };
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int64_t gi = off + i;
    if (a.mode == 0) {
      __nv_bfloat16* x = a.X + gi * kIn;
      for (int o = -2; o <= 2; ++o) {
        int k = mir(i + o), kp = mir(k + 1), km = mir(k - 1);
        int base = 5 * (o + 2);
        x[base + 0] = __float2bfloat16((float)(a.ne[off + k] * isn));
        x[base + 1] = __float2bfloat16((float)(a.phi[off + k] * isp));
        x[base + 2] = __float2bfloat16((float)(fphi(k) * isn));
        x[base + 3] = __float2bfloat16((float)(a.T[off + k] * (1.0 / 2000.0)));
        x[base + 4] = __float2bfloat16((float)(-(a.phi[off + kp] - a.phi[off + km]) * 0.5 * isp));
      }
      for (int f = kFeat; f < kIn; ++f) x[f] = __float2bfloat16(0.0f);
    } else if (a.mode == 1) {
      a.Tgt[gi * 2 + 0] = (float)((a.ne_star[gi] - a.ne[gi]) * isn);
      a.Tgt[gi * 2 + 1] = (float)((a.phi_star[gi] - a.phi[gi]) * isp);
    } else {
      a.ne_g[gi] = a.ne[gi] + ((a.comps & 1) ? sn * (double)a.Y[gi * 2 + 0] : 0.0);
      a.phi_g[gi] = a.phi[gi] + ((a.comps & 2) ? sp * (double)a.Y[gi * 2 + 1] : 0.0);
    }
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// --------------------------------------------------------------------------
// Training GEMMs on the tcgen05 tensor cores: C[m][n] = sum_k A(m,k) B(k,n)
// with A(m,k) = transA ? A[k*lda+m] : A[m*lda+k] and
// B(k,n) = transB ? B[n*ldb+k] : B[k*ldb+n] (BF16), FP32 accumulators in TMEM.
// Epilogues: kEpiAccumulate adds C with atomics (split-K weight gradients);
// kEpiSiluGrad writes dZ = acc * G (BF16; G = silu'(Z) in BF16, stored by the
// forward) and adds the column sums of
// dZ to colsum (the forward runs fused, fwd_tc_kernel below).
//
// A CTA of 256 threads computes 128 rows of C (row m0 + r in TMEM lane r) by
// all N <= 128 columns (the MMA's N is N rounded up to 16) over its share of
// K, in slabs of up to 64 k, two of them in flight while the tensor core
// multiplies the current one. Each operand is staged in the K-major
// core-matrix layout of mlp_tc.cuh, zero outside the matrix: a K-contiguous
// operand by 16-byte asynchronous copies (cp.async) that land in core-matrix
// order (two buffers); an operand whose rows are contiguous into one of two
// row-major slots, which ldmatrix.trans then transposes into the operand
// buffer (one, or two when the other operand is K-contiguous) after the
// previous slab's MMAs have read it. The row-major slots of operands with 128
// values per row are filled by TMA (two 64 x 64 boxes with 128-byte swizzle,
// completing on a per-slot mbarrier), narrower ones by cp.async. The
// epilogue runs on all 8 warps: two per 32-lane quadrant of TMEM, each on
// half of the columns.
// Every wait on an mbarrier is bounded; a CTA whose MMAs do not complete sets
// the error word and writes NaN instead of its results.
// --------------------------------------------------------------------------
struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;
  int lda, transA;
  const __nv_bfloat16* B;
  int ldb, transB;
  float* C;
  int ldc;
  int epi;
  __nv_bfloat16* H;
  int ldh;
  const __nv_bfloat16* Gin;
  int ldgin;
  float* colsum;
};

// the kernel's form: operand X(r, k) = X[r * sr + k * sk] with sr == 1 or sk == 1
struct TcGemm {
  int M, N, K, kchunk, epi;
  const uint16_t* A;
  int64_t sam, sak;
  const uint16_t* B;
  int64_t sbn, sbk;
  float* C;
  int64_t scm, scn;
  __nv_bfloat16* H;
  int64_t ldh;
  const __nv_bfloat16* Gin;
  int64_t ldgin;
  float* colsum;
  int* err;
  int tmaA, tmaB;   // the operand's slabs come by TMA (tensor maps of the launch)
  int polls;        // polls of the main bounded waits (the clean-up waits use the default)
  unsigned* chk;    // check word of the bounds-checking build (may be null)
};

constexpr int kEpiAccumulate = 0, kEpiSiluGrad = 2;         // GemmArgs::epi
constexpr int kGemmThreads = 256;                           // two warps per TMEM lane quadrant
constexpr int kSlabK = 64;                                  // k per slab
constexpr uint32_t kOpBytes = 128 * kSlabK * 2;             // one operand slab
__host__ __device__ constexpr uint32_t nat_pitch(int R) { return (uint32_t)(2 * R + 16); }
__host__ __device__ constexpr uint32_t nat_bytes(int R) { return kSlabK * nat_pitch(R); }
constexpr uint32_t kGemmSmemMax = 4 * kOpBytes + 4 * nat_bytes(128) + 1024;   // + alignment slack
constexpr int kHPitch = 80;                                 // epilogue staging pitch (BF16 rows)
constexpr uint32_t kStageBytes = 2 * 32 * kHPitch;
static_assert(kGemmThreads / 32 * kStageBytes <= 4 * kOpBytes, "staging tiles fit the operand buffers");

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
__device__ __forceinline__ void stage_k(unsigned char* S, const uint16_t* X, int64_t sr, bool vec,
                                        int64_t rbase, int64_t rmax, int R, int k0, int kend,
                                        int kc, int tid) {
  const int items = R * kc;
#pragma unroll 4
  for (int e = tid; e < items; e += kGemmThreads) {
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

// row-contiguous operand X(r, k) = X[r + k sk]: copy the slab row-major into
// nat (row k at k * pitch, 16 bytes = 8 consecutive r per item)
__device__ __forceinline__ void stage_nat(unsigned char* nat, uint32_t pitch, const uint16_t* X,
                                          int64_t sk, bool vec, int64_t rbase, int64_t rmax,
                                          int R, int k0, int kend, int ks, int tid) {
  const int rc = R >> 3, items = ks * rc;
#pragma unroll 4
  for (int e = tid; e < items; e += kGemmThreads) {
    const int k = e / rc, c = e - k * rc;
    const int64_t gr = rbase + c * 8, gk = k0 + k;
    unsigned char* d = nat + (size_t)k * pitch + c * 16;
    const bool none = gr >= rmax || gk >= kend;
    if (none || (vec && gr + 8 <= rmax)) {
      cp16(d, none ? (const void*)X : (const void*)(X + gk * sk + gr), !none);
    } else {
      uint16_t u[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) u[j] = (gr + j < rmax) ? X[gk * sk + gr + j] : 0;
      *reinterpret_cast<uint4*>(d) = make_uint4(pack_u16(u[0], u[1]), pack_u16(u[2], u[3]),
                                                pack_u16(u[4], u[5]), pack_u16(u[6], u[7]));
    }
  }
}

// TMA: a 64 x 64 BF16 box (64 k rows of 128 bytes) of a row-major operand
// with 128-byte swizzle: the 16-byte chunk j of row k lands at chunk j ^ (k % 8)
// of the row (the box's base is 1024-byte aligned). Completion on mbarrier mb.
constexpr uint32_t kTmaBoxBytes = 64 * 128;
__device__ __forceinline__ void tma_box(unsigned char* dst, const CUtensorMap* map, int x, int y,
                                        uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(tc::saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mb)
      : "memory");
}

// two swizzled boxes (r 0..63 and 64..127 of 64 k rows) -> K-major core matrices,
// as nat_to_k: core matrix i = c kc + kk holds rows 8c.. of k 8kk..
__device__ __forceinline__ void nat_sw_to_k(unsigned char* S, const unsigned char* nat, int kc,
                                            int warp, int lane) {
  const int mats = 16 * kc;
  for (int g = warp; g * 4 < mats; g += kGemmThreads / 32) {
    const int i = g * 4 + (lane >> 3);
    const int c = i / kc, kk = i - c * kc;
    const int k = kk * 8 + (lane & 7);
    const uint32_t src =
        tc::saddr(nat + (c >> 3) * kTmaBoxBytes + k * 128 + (((c & 7) ^ (k & 7)) << 4));
    uint32_t r0, r1, r2, r3;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(src));
    uint32_t* d = reinterpret_cast<uint32_t*>(S + (size_t)g * 4 * 128) + lane;
    d[0] = r0;
    d[32] = r1;
    d[64] = r2;
    d[96] = r3;
  }
}

// nat (k rows, r contiguous) -> K-major core matrices. Core matrix i = c kc + kk
// holds rows 8c.. of k 8kk..; ldmatrix.trans hands lane l the pair
// (k = 8kk + 2 (l%4) + {0,1}, r = 8c + l/4), which sits at byte 4 l of it.
__device__ __forceinline__ void nat_to_k(unsigned char* S, const unsigned char* nat,
                                         uint32_t pitch, int R, int kc, int warp, int lane) {
  const int mats = (R >> 3) * kc;   // a multiple of 4 (R >= 16, kc >= 2)
  for (int g = warp; g * 4 < mats; g += kGemmThreads / 32) {
    const int i = g * 4 + (lane >> 3);   // the matrix whose row address this lane gives
    const int c = i / kc, kk = i - c * kc;
    const uint32_t src = tc::saddr(nat + (size_t)(kk * 8 + (lane & 7)) * pitch + c * 16);
    uint32_t r0, r1, r2, r3;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(src));
    uint32_t* d = reinterpret_cast<uint32_t*>(S + (size_t)g * 4 * 128) + lane;
    d[0] = r0;
    d[32] = r1;
    d[64] = r2;
    d[96] = r3;
  }
}

// lane l ends with the sum over the warp of v[l]
__device__ __forceinline__ float warp_colsum32(float* v, int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < s; ++j) {
      const float send = up ? v[j] : v[j + s];
      const float keep = up ? v[j + s] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// EPI: the epilogue; AMN / BMN: operand A / B has contiguous rows
// (staged through the row-major copy and ldmatrix.trans) rather than contiguous k
template <int EPI, bool AMN, bool BMN>
__global__ void __launch_bounds__(kGemmThreads) gemm_tc_kernel(TcGemm g,
                                                               const __grid_constant__ CUtensorMap tmA,
                                                               const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  // 1024-byte aligned base (the swizzled TMA boxes need it; the launch adds 1 KB)
  unsigned char* gsm = gsm_raw + ((1024u - (tc::saddr(gsm_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t lbar[2];   // TMA slabs, one per row-major slot
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int kbeg = blockIdx.y * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  // the CTA's rows and its share of K inside the matrices (before any
  // barrier, tensor-memory allocation or copy)
  if (!SDCEF_CHECK_W(g.chk, m0 < g.M && kbeg >= 0 && kbeg < kend && kend <= g.K &&
                                g.N >= 1 && g.N <= 128,
                     sdcef_chk::kMlpRow))
    return;
  const int Np = (g.N + 15) & ~15;
  constexpr bool amn = AMN, bmn = BMN;
  // operand buffers: two per operand, except when both operands go through the
  // row-major copies: then the copies carry the next slab and one buffer each
  // (written after the previous slab's MMAs have finished) suffices
  constexpr int NB = (AMN && BMN) ? 1 : 2;
  unsigned char* opA = gsm;
  unsigned char* opB = gsm + NB * kOpBytes;
  // two slots of row-major copies per such operand, so that two slabs are in
  // flight; every slot starts on a 1024-byte boundary (17408 = 17 KB)
  constexpr uint32_t natA_sz = amn ? nat_bytes(128) : 0;
  const uint32_t natB_sz = bmn ? nat_bytes(Np) : 0;
  unsigned char* natA0 = gsm + 2 * NB * kOpBytes;
  unsigned char* natB0 = natA0 + 2 * natA_sz;
  const bool tmaA = amn && g.tmaA, tmaB = bmn && g.tmaB;
  auto l_bar = [&](int s) { return tc::saddr(&lbar[s & 1]); };
  const bool vecA = ((reinterpret_cast<uintptr_t>(g.A) & 15) == 0) && (((amn ? g.sak : g.sam) & 7) == 0);
  const bool vecB = ((reinterpret_cast<uintptr_t>(g.B) & 15) == 0) && (((bmn ? g.sbk : g.sbn) & 7) == 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        tc::saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[1])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&lbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&lbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tmem_base;
  const uint32_t idesc = tc::idesc_bf16(128, Np);
  const int nslab = (kend - kbeg + kSlabK - 1) / kSlabK;   // >= 1 (the host keeps kbeg < K)
  constexpr int L = 2;   // slabs in flight
  // the mbarrier that slab s's MMAs complete, and the parity of that completion
  auto bar_of = [&](int s) { return tc::saddr(&mbar[NB == 2 ? (s & 1) : 0]); };
  auto par_of = [&](int s) { return (uint32_t)(NB == 2 ? ((s >> 1) & 1) : (s & 1)); };
  auto issue = [&](int s) {
    const int b = NB == 2 ? (s & 1) : 0, k0 = kbeg + s * kSlabK;
    const int ks = min(kSlabK, (kend - k0 + 15) & ~15), kc = ks >> 3;
    unsigned char* natA = natA0 + (s & 1) * natA_sz;
    unsigned char* natB = natB0 + (s & 1) * natB_sz;
    if ((tmaA || tmaB) && tid == 0) {
      // two 64-row boxes per TMA operand (rows past the matrix arrive as zeros)
      const uint32_t bytes = (tmaA ? 2 : 0) * kTmaBoxBytes + (tmaB ? 2 : 0) * kTmaBoxBytes;
      const uint32_t lb = l_bar(s);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lb), "r"(bytes)
                   : "memory");
      if (tmaA) {
        tma_box(natA, &tmA, (int)m0, k0, lb);
        tma_box(natA + kTmaBoxBytes, &tmA, (int)m0 + 64, k0, lb);
      }
      if (tmaB) {
        tma_box(natB, &tmB, 0, k0, lb);
        tma_box(natB + kTmaBoxBytes, &tmB, 64, k0, lb);
      }
    }
    if (!amn) stage_k(opA + b * kOpBytes, g.A, g.sam, vecA, m0, g.M, 128, k0, kend, kc, tid);
    else if (!tmaA) stage_nat(natA, nat_pitch(128), g.A, g.sak, vecA, m0, g.M, 128, k0, kend, ks, tid);
    if (!bmn) stage_k(opB + b * kOpBytes, g.B, g.sbn, vecB, 0, g.N, Np, k0, kend, kc, tid);
    else if (!tmaB) stage_nat(natB, nat_pitch(Np), g.B, g.sbk, vecB, 0, g.N, Np, k0, kend, ks, tid);
    cp_commit();
  };
  for (int j = 0; j < min(L, nslab); ++j) issue(j);
  bool ok = true;
  int last = -1;                                           // last slab whose MMAs were committed
  for (int s = 0; s < nslab; ++s) {
    const int b = NB == 2 ? (s & 1) : 0, k0 = kbeg + s * kSlabK;
    const int ks = min(kSlabK, (kend - k0 + 15) & ~15), kc = ks >> 3;
    if (L == 2 && s + 1 < nslab) cp_wait<1>();
    else cp_wait<0>();
    unsigned char* sA = opA + b * kOpBytes;
    unsigned char* sB = opB + b * kOpBytes;
    unsigned char* natA = natA0 + (s & 1) * natA_sz;
    unsigned char* natB = natB0 + (s & 1) * natB_sz;
    if (amn || bmn) {
      if (tmaA || tmaB) {   // slab s's boxes: completion (s >> 1) of its slot's mbarrier
        const bool w = tc::wait_phase(l_bar(s), (uint32_t)((s >> 1) & 1), g.polls);
        if (__syncthreads_or(!w)) {
          ok = false;
          break;
        }
      }
      __syncthreads();
      if (NB == 1 && s >= 1) {   // the single buffers: slab s - 1's MMAs have read them
        const bool w = tc::wait_phase(bar_of(s - 1), par_of(s - 1), g.polls);
        if (__syncthreads_or(!w)) {
          ok = false;
          break;
        }
      }
      if (tmaA) nat_sw_to_k(sA, natA, kc, warp, lane);
      else if (amn) nat_to_k(sA, natA, nat_pitch(128), 128, kc, warp, lane);
      if (tmaB) nat_sw_to_k(sB, natB, kc, warp, lane);
      else if (bmn) nat_to_k(sB, natB, nat_pitch(Np), Np, kc, warp, lane);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t aA = tc::saddr(sA), aB = tc::saddr(sB);
      for (int kk = 0; kk < ks / 16; ++kk)
        tc::mma(tm, tc::smem_desc(aA + kk * 256, 128, kc * 128),
                tc::smem_desc(aB + kk * 256, 128, kc * 128), idesc, (s > 0 || kk > 0) ? 1u : 0u);
      tc::commit(bar_of(s));
    }
    last = s;
    const int nxt = s + L;
    if (nxt < nslab) {
      // with two buffers, buffer nxt & 1 was last read by the MMAs of slab nxt - 2
      if (NB == 2 && nxt >= 2) {
        const bool w = tc::wait_phase(bar_of(nxt - 2), par_of(nxt - 2), g.polls);
        if (__syncthreads_or(!w)) {
          ok = false;
          break;
        }
      }
      issue(nxt);
    }
  }
  if (ok) {   // the last commit covers every MMA issued before it
    const bool w = tc::wait_phase(bar_of(last), par_of(last), g.polls);
    ok = !__syncthreads_or(!w);
  }
  tc::fence_after();
  // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) + lane (row m0 + 32 (w % 4)
  // + lane) in columns 64 (w / 4) .. 64 (w / 4) + 63 ----
  const int quad = warp & 3, half = warp >> 2;
  const uint32_t lane_addr = tm + ((uint32_t)(quad * 32) << 16);
  const int64_t row = m0 + quad * 32 + lane;
  const bool live = row < g.M;
  // the operand buffers are free now: each warp gets two staging tiles of 32
  // rows x 32 BF16 (pitch 80 B, at which a quarter-warp's 16-byte accesses hit
  // distinct banks), one for G coming in and one for dZ going out
  const int64_t rbase = m0 + quad * 32;
  const int64_t rows_left = (int64_t)g.M - rbase;
  const int nrows = rows_left <= 0 ? 0 : (rows_left < 32 ? (int)rows_left : 32);
  unsigned char* gt = gsm + warp * kStageBytes;
  unsigned char* ht = gt + 32 * kHPitch;
  const bool tiled =
      (g.ldh & 7) == 0 && (g.ldgin & 7) == 0 &&
      ((reinterpret_cast<uintptr_t>(g.H) | reinterpret_cast<uintptr_t>(g.Gin)) & 15) == 0;
  for (int c0 = half * 64; c0 < min(Np, half * 64 + 64); c0 += 32) {
    float v[32];
    if (ok) {
      tc::ld32(lane_addr + c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = __int_as_float(0x7fffffff);
    }
    const bool full = c0 + 32 <= g.N;
    if (EPI == kEpiAccumulate) {
      if (live) {
        float* Cr = g.C + row * g.scm;
        if (full && g.scn == 1 && ((reinterpret_cast<uintptr_t>(Cr + c0) & 15) == 0)) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            atomicAdd(reinterpret_cast<float4*>(Cr + c0 + 4 * q),
                      make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < g.N) atomicAdd(Cr + (c0 + j) * g.scn, v[j]);
        }
      }
    } else {
      float z[32];   // the multiplier G of this thread's row
      if (full && tiled) {
        // G rows in with whole-row loads (8 rows x 64 B per instruction) through the staging tile
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = i * 32 + lane, r = e >> 2, p = e & 3;
          uint4 t = make_uint4(0, 0, 0, 0);
          if (r < nrows)
            t = __ldg(reinterpret_cast<const uint4*>(g.Gin + (rbase + r) * g.ldgin + c0 + 8 * p));
          *reinterpret_cast<uint4*>(gt + r * kHPitch + 16 * p) = t;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 t = *reinterpret_cast<const uint4*>(gt + lane * kHPitch + 16 * q);
          const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            z[8 * q + 2 * u] = __uint_as_float(w[u] << 16);
            z[8 * q + 2 * u + 1] = __uint_as_float(w[u] & 0xffff0000u);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          z[j] = (live && c0 + j < g.N) ? __bfloat162float(g.Gin[row * g.ldgin + c0 + j]) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = (live && c0 + j < g.N) ? v[j] * z[j] : 0.0f;
      if (full && tiled) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(ht + lane * kHPitch + 16 * q) =
              make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                         pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = i * 32 + lane, r = e >> 2, p = e & 3;
          if (r < nrows)
            *reinterpret_cast<uint4*>(g.H + (rbase + r) * g.ldh + c0 + 8 * p) =
                *reinterpret_cast<const uint4*>(ht + r * kHPitch + 16 * p);
        }
        __syncwarp();
      } else if (live) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < g.N) g.H[row * g.ldh + c0 + j] = __float2bfloat16(v[j]);
      }
      const float cs = warp_colsum32(v, lane);
      if (c0 + lane < g.N) atomicAdd(&g.colsum[c0 + lane], cs);
    }
  }
  if (!ok) {
    cp_wait<0>();
    if (tid == 0) atomicExch(g.err, 1);
    // boxes of issued slabs may still be landing: bounded waits
    if (tmaA || tmaB)
      for (int q = last + 1; q < min(nslab, last + 1 + L); ++q)
        tc::wait_phase(l_bar(q), (uint32_t)((q >> 1) & 1));
    // an MMA may still be in flight: one more bounded wait before TMEM is freed
    if (last >= 0) tc::wait_phase(bar_of(last), par_of(last));
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tm));
}

// --------------------------------------------------------------------------
// Training forward, all three layers in one launch: a CTA of 256 threads
// takes 128 rows of X, stages X and the BF16 weights in the K-major
// core-matrix layout (cp.async), and chains the layers on the tensor core
// through one 128-column TMEM accumulator. After each hidden layer the 8-warp
// epilogue (two warps per TMEM lane quadrant, each on half of the columns)
// adds the bias, writes H = silu(Z) (BF16) to global memory (and in training
// silu'(Z1) in BF16, the factor of the layer-1 backward product, instead of
// Z1), and writes H into shared memory as the A operand of the next layer,
// so H1 and H2 are not read back from global memory. The output layer
// accumulates in TMEM columns of its own, so that in training the same
// kernel goes on from Y to the loss against T (dY = (Y - T) / n, the loss and
// the bias gradient of the output layer) and to the first backward product
// dZ2 = (dY W3) * silu'(Z2), read straight from the layer-2 accumulator:
// Z2 never goes to global memory. Every wait on the mbarrier is bounded; a
// CTA whose MMAs do not complete sets the error word and writes NaN instead
// of its results.
// --------------------------------------------------------------------------
struct FwdArgs {
  int64_t n;
  const uint16_t* X;                  // [n][32] BF16
  const uint16_t *w1, *w2, *w3;       // [128][32], [128][128], [2][128] BF16
  const float* p;                     // FP32 parameters (biases)
  __nv_bfloat16* G1;                  // [n][128] silu'(Z1) in BF16 (training)
  __nv_bfloat16 *H1, *H2;             // [n][128] BF16
  float* Y;                           // [n][2] FP32, nullable
  // training (T != nullptr): the MSE loss and the first backward step
  const float* T;                     // [n][2] FP32 targets
  float inv_n;                        // 1 / n
  __nv_bfloat16 *dY, *dZ2;            // [n][2], [n][128] BF16
  float *loss, *gb2, *gb3;            // accumulated with atomics
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
  __shared__ float sw3[kOut][kHid];   // the BF16 W3 as FP32 (dZ2 product)
  __shared__ float sdy[128][kOut];    // the BF16-rounded dY of the tile's rows
  __shared__ float sred[4][3];        // per-warp loss and output-bias partials
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
  for (int i = tid; i < kOut * kHid; i += kGemmThreads)
    sw3[i / kHid][i % kHid] = __uint_as_float((uint32_t)a.w3[i] << 16);
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
  // hidden-layer epilogue: Z = acc + bias, H = silu(Z) to global and to sH,
  // and (training, layer 1) G = silu'(Z) for the backward pass
  auto hidden = [&](bool ok, const float* bias, __nv_bfloat16* G, __nv_bfloat16* H) {
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
      if (live && G) {
        uint4* gp = reinterpret_cast<uint4*>(G + row * kHid + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          gp[q] = make_uint4(pack_bf16(silu_grad(v[8 * q]), silu_grad(v[8 * q + 1])),
                             pack_bf16(silu_grad(v[8 * q + 2]), silu_grad(v[8 * q + 3])),
                             pack_bf16(silu_grad(v[8 * q + 4]), silu_grad(v[8 * q + 5])),
                             pack_bf16(silu_grad(v[8 * q + 6]), silu_grad(v[8 * q + 7])));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 hq = make_uint4(pack_bf16(silu_fast(v[8 * q]), silu_fast(v[8 * q + 1])),
                                    pack_bf16(silu_fast(v[8 * q + 2]), silu_fast(v[8 * q + 3])),
                                    pack_bf16(silu_fast(v[8 * q + 4]), silu_fast(v[8 * q + 5])),
                                    pack_bf16(silu_fast(v[8 * q + 6]), silu_fast(v[8 * q + 7])));
        if (live) *reinterpret_cast<uint4*>(H + row * kHid + c0 + 8 * q) = hq;
        *reinterpret_cast<uint4*>(sH + tc::cm_off(r, c0 + 8 * q, kHid / 8)) = hq;
      }
    }
    // sH complete (and the accumulator read) before the next layer's MMAs
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  };
  constexpr uint32_t kIdH = tc::idesc_bf16(128, 128), kIdO = tc::idesc_bf16(128, 16);
  bool ok = layer(sX, sW1, kIn / 8, kIdH, 0);
  hidden(ok, sb, a.G1, a.H1);
  if (ok) ok = layer(sH, sW2, kHid / 8, kIdH, 0);
  hidden(ok, sb + kHid, nullptr, a.H2);   // Z2 stays in TMEM
  if (ok) ok = layer(sH, sW3, kHid / 8, kIdO, 128);
  const float qnan = __int_as_float(0x7fffffff);
  if (half == 0) {
    float y[2] = {qnan, qnan};
    if (ok) tc::ld2(lane_addr + 128, y);
    y[0] += sb[2 * kHid];
    y[1] += sb[2 * kHid + 1];
    if (live && a.Y) {
      a.Y[row * kOut] = y[0];
      a.Y[row * kOut + 1] = y[1];
    }
    if (a.T) {
      // MSE loss 1/(2n) sum |Y - T|^2: dY = (Y - T) / n in BF16 for the
      // backward GEMMs, the output-layer bias gradient from the FP32 values
      const float d0 = live ? y[0] - a.T[row * kOut] : 0.0f;
      const float d1 = live ? y[1] - a.T[row * kOut + 1] : 0.0f;
      const float e0 = d0 * a.inv_n, e1 = d1 * a.inv_n;
      const __nv_bfloat16 q0 = __float2bfloat16(e0), q1 = __float2bfloat16(e1);
      if (live) {
        a.dY[row * kOut] = q0;
        a.dY[row * kOut + 1] = q1;
      }
      sdy[r][0] = __bfloat162float(q0);
      sdy[r][1] = __bfloat162float(q1);
      float l = d0 * d0 + d1 * d1, g0 = e0, g1 = e1;
      for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, o);
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
      }
      if (lane == 0) {
        sred[quad][0] = l;
        sred[quad][1] = g0;
        sred[quad][2] = g1;
      }
    }
  }
  __syncthreads();
  if (a.T) {
    if (tid < 3) {
      const float v = sred[0][tid] + sred[1][tid] + sred[2][tid] + sred[3][tid];
      atomicAdd(tid == 0 ? a.loss : a.gb3 + (tid - 1), tid == 0 ? v * 0.5f * a.inv_n : v);
    }
    // dZ2 = (dY W3) * silu'(Z2), Z2 = layer-2 accumulator + b2; the column
    // sums of dZ2 are the layer-2 bias gradient
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
      float v[32];
      if (ok) {
        tc::ld32(lane_addr + c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = qnan;
      }
      const float dy0 = sdy[r][0], dy1 = sdy[r][1];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        const float g = fmaf(dy1, sw3[1][c], dy0 * sw3[0][c]);
        v[j] = live ? g * silu_grad(v[j] + sb[kHid + c]) : 0.0f;
      }
      if (live) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(a.dZ2 + row * kHid + c0 + 8 * q) =
              make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                         pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
      }
      const float cs = warp_colsum32(v, lane);
      atomicAdd(&a.gb2[c0 + lane], cs);
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
// Fused guess: features -> 3 layers -> X^n + S_X y, one pass per column, on
// the tcgen05 tensor cores (BF16 operands in shared memory, FP32 accumulators
// in tensor memory); the kernel's organisation is described in mlp_tc.cuh.
// --------------------------------------------------------------------------
struct GuessArgs {
  FeatArgs f;
  const float* p;                  // FP32 parameters (biases read from here)
  const __nv_bfloat16 *w1, *w2, *w3;
  int* queue;
  float* stage;                    // [cells][5] per-cell feature values (FP32)
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
                                  (off + N) * 5 <= g.stage_cap,
                       sdcef_chk::kMlpStage))
      continue;
    auto fphi = [&](int i) {
      double q = 0.0;
      for (int s = 0; s < a.nsp; ++s) q += (double)a.val[s] * a.n_ion[(int64_t)s * cells + off + i];
      return q;
    };
    double mn = 0.0, mq = 0.0, mp = 0.0;
    for (int i = t; i < N; i += W) {
      mn = fmax(mn, fabs(a.ne[off + i]));
      mq = fmax(mq, fabs(fphi(i)));
      mp = fmax(mp, fabs(a.phi[off + i]));
    }
    double mx[3] = {mn, mq, mp};
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
    const double isn = 1.0 / sn, isp = 1.0 / sp;
    if (N < 1) continue;
    auto mir = [&](int j) {
      if (j < 0) j = -j - 1;
      if (j >= N) j = 2 * N - 1 - j;
      return min(max(j, 0), N - 1);
    };
    // the five per-cell values of the features, staged once in FP32
    float* st = g.stage + off * 5;
    for (int i = t; i < N; i += W) {
      const int kp = (i + 1 < N) ? i + 1 : N - 1;
      const int km = (i >= 1) ? i - 1 : 0;
      st[i * 5 + 0] = (float)(a.ne[off + i] * isn);
      st[i * 5 + 1] = (float)(a.phi[off + i] * isp);
      st[i * 5 + 2] = (float)(fphi(i) * isn);
      st[i * 5 + 3] = (float)(a.T[off + i] * (1.0 / 2000.0));
      st[i * 5 + 4] = (float)(-(a.phi[off + kp] - a.phi[off + km]) * 0.5 * isp);
    }
    tc::bar(barid, W);
    for (int r0 = 0; r0 < N; r0 += tc::kTile) {
      // row r of A: the 25 stencil features of cell i (f = 5 o + q: quantity q
      // of cell i + o - 2), zero-padded to K = 32; the worker's two threads of
      // row r build features 0..15 and 16..31
      const int i = min(r0 + r, N - 1);
#pragma unroll
      for (int ch = 2 * half; ch < 2 * half + 2; ++ch) {
        float f8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int f = ch * 8 + u;
          f8[u] = f < kFeat ? st[mir(i + f / 5 - 2) * 5 + f % 5] : 0.0f;
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
        a.phi_g[gi] = a.phi[gi] + ((a.comps & 2) ? sp * (double)yp : 0.0);
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
  }
  tc::fence_before();
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm),
                 "n"(tc::kTmemCols));
}

// Adam (Kingma & Ba 2015) with bias correction; refreshes the BF16 weight
// copies and clears the gradient for the next step.
__global__ void adam_kernel(float* p, float* g, float* m, float* v, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2, __nv_bfloat16* w1,
                            __nv_bfloat16* w2, __nv_bfloat16* w3) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    g[i] = 0.0f;
    if (i >= kOffW1 && i < kOffB1) w1[i - kOffW1] = __float2bfloat16(pi);
    else if (i >= kOffW2 && i < kOffB2) w2[i - kOffW2] = __float2bfloat16(pi);
    else if (i >= kOffW3 && i < kOffB3) w3[i - kOffW3] = __float2bfloat16(pi);
  }
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
  __nv_bfloat16 *w1, *w2, *w3;          // BF16 weight copies
  float *Y, *loss;                      // output, loss (FP32)
  __nv_bfloat16 *G1, *H1, *H2, *dY, *dZ2, *dZ1, *X;   // BF16 silu'(Z1), activations, features
  int step;
  int launches;
  int sms;                              // multiprocessors of the device
  cudaStream_t aux;                     // weight gradients beside the dZ chain
  cudaEvent_t ev[2];
  int polls;                            // polls of the kernels' main bounded waits
};

namespace {
// check word of the bounds-checking build: a spare word of the loss buffer
unsigned* mlp_chk(sdcef_mlp* h) { return reinterpret_cast<unsigned*>(h->loss) + 6; }
}  // namespace

namespace {

int cuda_fail(cudaError_t e) { return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e)); }

// tensor map of a row-major BF16 operand (inner: values per k row, outer: k),
// read in 64 x 64 boxes with 128-byte swizzle; false if it cannot be encoded
// (the kernel then stages the operand with cp.async)
bool tma_map(CUtensorMap* m, const uint16_t* base, int64_t inner, int64_t outer, int64_t row_bytes) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode || (reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || outer < 1) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {64, 64}, estr[2] = {1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(base), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t gemm(sdcef_mlp* h, const GemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  TcGemm g;
  memset(&g, 0, sizeof(g));
  g.M = a.M; g.N = a.N; g.K = a.K; g.epi = a.epi;
  g.A = reinterpret_cast<const uint16_t*>(a.A);
  g.sam = a.transA ? 1 : a.lda; g.sak = a.transA ? a.lda : 1;
  g.B = reinterpret_cast<const uint16_t*>(a.B);
  g.sbn = a.transB ? a.ldb : 1; g.sbk = a.transB ? 1 : a.ldb;
  g.C = a.C; g.scm = a.ldc; g.scn = 1;
  g.H = a.H; g.ldh = a.ldh; g.Gin = a.Gin; g.ldgin = a.ldgin; g.colsum = a.colsum;
  g.err = (int*)h->loss + 5;
  g.polls = h->polls;
  g.chk = mlp_chk(h);
  if (g.epi == kEpiAccumulate && g.M < 64 && g.N > g.M) {
    // C^T = B^T A^T: the long side of the product goes on the 128 TMEM lanes
    std::swap(g.M, g.N); std::swap(g.A, g.B); std::swap(g.sam, g.sbn); std::swap(g.sak, g.sbk);
    std::swap(g.scm, g.scn);
  }
  if (g.N > 128 || (g.sam != 1 && g.sak != 1) || (g.sbn != 1 && g.sbk != 1))
    return cudaErrorInvalidValue;
  const int tiles = (g.M + 127) / 128, Np = (g.N + 15) & ~15;
  int splits = 1;
  g.kchunk = (g.K + kSlabK - 1) / kSlabK * kSlabK;
  if (g.epi == kEpiAccumulate) {
    // split K (the sample dimension of the weight gradients) over about two
    // CTAs per SM, at least two slabs each; partial sums meet in C by atomics
    const int want = std::max(1, 2 * h->sms / tiles);
    const int kc = (g.K + want - 1) / want;
    g.kchunk = std::max((kc + kSlabK - 1) / kSlabK * kSlabK, 2 * kSlabK);
    splits = (g.K + g.kchunk - 1) / g.kchunk;
  }
  const bool amn = g.sak != 1, bmn = g.sbk != 1;
  const uint32_t smem = ((amn && bmn) ? 2 : 4) * kOpBytes + 2 * (amn ? nat_bytes(128) : 0) +
                        2 * (bmn ? nat_bytes(Np) : 0) + 1024;
  // row-major operands of 128 values per k row go by TMA (two swizzled 64 x 64 boxes per slab)
  CUtensorMap mapA, mapB;
  memset(&mapA, 0, sizeof(mapA));
  memset(&mapB, 0, sizeof(mapB));
  g.tmaA = amn && g.M == 128 && tma_map(&mapA, g.A, 128, g.K, g.sak * 2);
  g.tmaB = bmn && g.N == 128 && tma_map(&mapB, g.B, 128, g.K, g.sbk * 2);
  // M (the sample dimension of the layer GEMMs) on grid.x, whose limit is 2^31 - 1
  const dim3 grid(tiles, splits);
  if (g.epi == kEpiAccumulate && amn && bmn)
    gemm_tc_kernel<kEpiAccumulate, true, true><<<grid, kGemmThreads, smem, st>>>(g, mapA, mapB);
  else if (g.epi == kEpiSiluGrad && !amn && bmn)
    gemm_tc_kernel<kEpiSiluGrad, false, true><<<grid, kGemmThreads, smem, st>>>(g, mapA, mapB);
  else
    return cudaErrorInvalidValue;   // a form the training step does not use
  ++h->launches;
  return cudaGetLastError();
}

GemmArgs ga() {
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  return g;
}

// forward through the three layers for n rows of X. Inference (T == nullptr):
// Y (FP32 [n][2]) only. Training: silu'(Z1), H1, H2 for the backward GEMMs, and the
// loss, dY, dZ2 and the bias gradients of layers 2 and 3 (into h->g).
cudaError_t forward(sdcef_mlp* h, const __nv_bfloat16* X, const float* T, int64_t n, float* Y) {
  if (n <= 0) return cudaSuccess;
  FwdArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.X = reinterpret_cast<const uint16_t*>(X);
  a.w1 = reinterpret_cast<const uint16_t*>(h->w1);
  a.w2 = reinterpret_cast<const uint16_t*>(h->w2);
  a.w3 = reinterpret_cast<const uint16_t*>(h->w3);
  a.p = h->p;
  a.H1 = h->H1;
  a.H2 = h->H2;
  a.Y = Y;
  if (T) {
    a.G1 = h->G1;
    a.T = T;
    a.inv_n = 1.0f / (float)n;
    a.dY = h->dY;
    a.dZ2 = h->dZ2;
    a.loss = h->loss;
    a.gb2 = h->g + kOffB2;
    a.gb3 = h->g + kOffB3;
  }
  a.err = (int*)h->loss + 5;
  a.polls = h->polls;
  a.chk = mlp_chk(h);
  fwd_tc_kernel<<<(unsigned)((n + 127) / 128), kGemmThreads, kFwSmem, h->st>>>(a);
  ++h->launches;
  return cudaGetLastError();
}

// gradients of the mean-squared loss over n rows into h->g (accumulated),
// after forward(.., T, ..) produced dY, dZ2 and the layer-2/3 bias gradients
cudaError_t backward(sdcef_mlp* h, const __nv_bfloat16* X, int64_t n) {
  // the weight gradients of layers 3 and 2 (split-K over the samples) run on
  // the auxiliary stream beside dZ1 and gW1
  cudaError_t e = cudaEventRecord(h->ev[0], h->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev[0], 0);
  if (e != cudaSuccess) return e;
  // gW3 = dY^T H2
  GemmArgs g = ga();
  g.M = kOut; g.N = kHid; g.K = (int)n;
  g.A = h->dY; g.lda = kOut; g.transA = 1; g.B = h->H2; g.ldb = kHid;
  g.C = h->g + kOffW3; g.ldc = kHid; g.epi = kEpiAccumulate;
  if ((e = gemm(h, g, h->aux)) != cudaSuccess) return e;
  // gW2 = dZ2^T H1
  g = ga();
  g.M = kHid; g.N = kHid; g.K = (int)n;
  g.A = h->dZ2; g.lda = kHid; g.transA = 1; g.B = h->H1; g.ldb = kHid;
  g.C = h->g + kOffW2; g.ldc = kHid;
  if ((e = gemm(h, g, h->aux)) != cudaSuccess) return e;
  // dZ1 = (dZ2 W2) * silu'(Z1), silu'(Z1) stored by the forward; gb1 += colsum
  g = ga();
  g.M = (int)n; g.N = kHid; g.K = kHid;
  g.A = h->dZ2; g.lda = kHid; g.B = h->w2; g.ldb = kHid;
  g.epi = kEpiSiluGrad; g.Gin = h->G1; g.ldgin = kHid; g.H = h->dZ1; g.ldh = kHid; g.colsum = h->g + kOffB1;
  if ((e = gemm(h, g, h->st)) != cudaSuccess) return e;
  // gW1 = dZ1^T X
  g = ga();
  g.M = kHid; g.N = kIn; g.K = (int)n;
  g.A = h->dZ1; g.lda = kHid; g.transA = 1; g.B = X; g.ldb = kIn;
  g.C = h->g + kOffW1; g.ldc = kIn;
  if ((e = gemm(h, g, h->st)) != cudaSuccess) return e;
  // join: the gradient is complete on the caller's stream
  if ((e = cudaEventRecord(h->ev[1], h->aux)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(h->st, h->ev[1], 0);
}

FeatArgs feat_args(const sdcef_batch* b) {
  FeatArgs a;
  memset(&a, 0, sizeof(a));
  a.ncol = b->ncol;
  a.col_off = b->col_off;
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
      e = cudaFuncSetAttribute(gemm_tc_kernel<kEpiAccumulate, true, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_tc_kernel<kEpiSiluGrad, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kFwSmem);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (cudaEvent_t ev : h->ev) if (ev) cudaEventDestroy(ev);
      if (h->aux) cudaStreamDestroy(h->aux);
      delete h;
      return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
    }
    h->sms = std::max(h->sms, 1);
  }
  const size_t R = (size_t)max_rows;
  struct Alloc { void** p; size_t bytes; } al[] = {
      {(void**)&h->p, kNParam * 4}, {(void**)&h->g, kNParam * 4}, {(void**)&h->m, kNParam * 4},
      {(void**)&h->v, kNParam * 4}, {(void**)&h->w1, kHid * kIn * 2}, {(void**)&h->w2, kHid * kHid * 2},
      {(void**)&h->w3, kOut * kHid * 2}, {(void**)&h->G1, R * kHid * 2},
      {(void**)&h->Y, R * kOut * 4}, {(void**)&h->loss, 64}, {(void**)&h->H1, R * kHid * 2},
      {(void**)&h->H2, R * kHid * 2}, {(void**)&h->dY, R * kOut * 2}, {(void**)&h->dZ2, R * kHid * 2},
      {(void**)&h->dZ1, R * kHid * 2}, {(void**)&h->X, R * kIn * 2}};
  for (auto& a : al) {
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e == cudaSuccess) e = cudaMemset(*a.p, 0, a.bytes);
    if (e != cudaSuccess) {
      for (auto& b : al) if (*b.p) cudaFree(*b.p);
      for (cudaEvent_t ev : h->ev) cudaEventDestroy(ev);
      cudaStreamDestroy(h->aux);
      delete h;
      return report_error(SDCEF_ERR_NOMEM, cudaGetErrorString(e));
    }
  }
  *out = h;
  return SDCEF_SUCCESS;
}

int sdcef_mlp_destroy(sdcef_mlp* h) {
  if (!h) return SDCEF_SUCCESS;
  cudaStreamSynchronize(h->st);
  cudaStreamSynchronize(h->aux);
  for (cudaEvent_t ev : h->ev) cudaEventDestroy(ev);
  cudaStreamDestroy(h->aux);
  void* ps[] = {h->p, h->g, h->m, h->v, h->w1, h->w2, h->w3, h->G1, h->Y, h->loss,
                h->H1, h->H2, h->dY, h->dZ2, h->dZ1, h->X};
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
  cudaError_t e = forward(h, (const __nv_bfloat16*)X_bf16, nullptr, n, Y ? Y : h->Y);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_grad(sdcef_mlp* h, const void* X_bf16, const float* T, int64_t n, float* grads,
                   float* loss) {
  if (!h || !X_bf16 || !T || n < 1) return report_error(SDCEF_ERR_INVALID, "mlp_grad: bad arguments");
  if (n > h->max_rows) return report_error(SDCEF_ERR_CAPACITY, "mlp_grad: n exceeds max_rows");
  h->launches = 0;
  cudaError_t e = cudaMemsetAsync(h->g, 0, kNParam * 4, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->loss, 0, 4, h->st);
  if (e == cudaSuccess) e = forward(h, (const __nv_bfloat16*)X_bf16, T, n, nullptr);
  if (e == cudaSuccess) e = backward(h, (const __nv_bfloat16*)X_bf16, n);
  if (e == cudaSuccess && grads)
    e = cudaMemcpyAsync(grads, h->g, kNParam * 4, cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, h->loss, 4, cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->g, 0, kNParam * 4, h->st);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_train_step(sdcef_mlp* h, const void* X_bf16, const float* T, int64_t n, float lr,
                         float* loss) {
  if (!h || !X_bf16 || !T || n < 1 || !(lr > 0.0f))
    return report_error(SDCEF_ERR_INVALID, "mlp_train_step: bad arguments");
  if (n > h->max_rows) return report_error(SDCEF_ERR_CAPACITY, "mlp_train_step: n exceeds max_rows");
  h->launches = 0;
  cudaError_t e = cudaMemsetAsync(h->loss, 0, 4, h->st);
  if (e == cudaSuccess) e = forward(h, (const __nv_bfloat16*)X_bf16, T, n, nullptr);
  if (e == cudaSuccess) e = backward(h, (const __nv_bfloat16*)X_bf16, n);
  if (e != cudaSuccess) return cuda_fail(e);
  h->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)h->step), c2 = 1.0f - powf(b2, (float)h->step);
  adam_kernel<<<64, 256, 0, h->st>>>(h->p, h->g, h->m, h->v, kNParam, lr, b1, b2, 1e-8f, c1, c2,
                                      h->w1, h->w2, h->w3);
  ++h->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  if (loss) e = cudaMemcpyAsync(loss, h->loss, 4, cudaMemcpyDeviceToDevice, h->st);
  return e == cudaSuccess ? SDCEF_SUCCESS : cuda_fail(e);
}

int sdcef_mlp_guess(sdcef_mlp* h, const sdcef_batch* b, int64_t ncells, int components,
                    double* ne_guess, double* phi_guess) {
  if (!h || !ne_guess || !phi_guess || ncells < 0 || components < 0 || components > 3)
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
  if (ncells * 5 > h->max_rows * (kIn / 2))
    return report_error(SDCEF_ERR_CAPACITY, "mlp_guess: ncells exceeds max_rows");
  g.stage = (float*)h->X;        // [cells][5] FP32 inside the [max_rows][32] BF16 buffer
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

int sdcef_mlp_check_word(sdcef_mlp* h, unsigned* word) {
  if (!h || !word) return report_error(SDCEF_ERR_INVALID, "mlp_check_word: NULL argument");
  unsigned w = 0;
  cudaError_t e = cudaStreamSynchronize(h->aux);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&w, mlp_chk(h), sizeof(unsigned), cudaMemcpyDeviceToHost, h->st);
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
  cudaError_t e = cudaStreamSynchronize(h->aux);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, word, sizeof(int), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(word, 0, sizeof(int), h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e);
  return flag ? report_error(SDCEF_ERR_CUDA, "mlp: a tensor-core wait timed out (outputs set to NaN)")
              : SDCEF_SUCCESS;
}

}  // extern "C"
