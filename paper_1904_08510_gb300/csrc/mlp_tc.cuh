// Fused learned-guess inference on the 5th-generation tensor cores (tcgen05):
// features -> 32x128 -> SiLU -> 128x128 -> SiLU -> 128x2 per cell, BF16
// operands in shared memory, FP32 accumulators in tensor memory (TMEM).
//
// A CTA of 512 threads holds the weights once in shared memory and runs two
// independent workers of 256 threads (two warpgroups) each: a worker takes
// columns from a persistent queue and walks its column in tiles of 128 cells,
// with its own A-operand buffer, its own 128 TMEM accumulator columns, its own
// mbarrier and a named barrier of its 256 threads. Row r of a tile belongs to
// two threads of the worker (warps w and w + 4 reach the same TMEM lane
// quadrant w mod 4): each builds half of row r's features in the A operand,
// the worker's first thread issues the MMAs (M = 128, K = 16 each) and
// commits them to the worker's mbarrier, and after each layer each of the two
// reads its half of TMEM lane r back with tcgen05.ld for the bias + SiLU
// epilogue, which writes the next layer's A operand into the worker's buffer
// (the MMA that read it has completed). Two CTAs per SM keep 32 warps and
// four independent MMA chains resident per SM and fill its 512 TMEM columns.
// Before its tiles the worker stages the column's per-cell quantities and the
// ion-field features (two prefix sums); after them, for the Poisson start, it
// solves for the potential of the guessed charge (two more).
//
// Shared-memory operand layout: K-major, no swizzle, in 8 x 16-byte core
// matrices (8 rows x 8 BF16 of K): element (r, k) of a matrix with K/8 = kc
// chunks at ((r/8) kc + k/8) * 128 + (r%8) * 16 + (k%8) * 2 bytes, so the
// descriptor's leading-byte offset (next K chunk) is 128 B and its stride-byte
// offset (next 8-row group) is kc * 128 B; one MMA of K = 16 spans two chunks.
//
// Every wait on the mbarrier is bounded; a CTA whose MMA does not complete
// sets an error flag, writes NaN to its outputs, releases its TMEM and stops.
#pragma once
#include <cstdint>

namespace tc {

constexpr int kTile = 128;              // rows per tile = TMEM lanes
constexpr int kWorkerThreads = 256;     // two threads per row: two warps per TMEM lane quadrant
constexpr int kGuessThreads = 2 * kWorkerThreads;
constexpr uint32_t kTmemCols = 256;     // two workers: 128 accumulator columns each
constexpr uint32_t kW1Bytes = 128 * 32 * 2, kW2Bytes = 128 * 128 * 2, kW3Bytes = 16 * 128 * 2,
                   kABytes = 128 * 128 * 2;
constexpr uint32_t kSmemBytes = kW1Bytes + kW2Bytes + kW3Bytes + 2 * kABytes + 260 * 4;

__device__ __forceinline__ uint32_t cm_off(int r, int k, int kc) {
  return (uint32_t)((((r >> 3) * kc + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start, leading- and stride-byte offsets
// (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

// default number of polls of a bounded wait
constexpr int kWaitPolls = 1 << 22;

// bounded wait for the completion of phase `parity`: at most `polls` polls;
// false on timeout (polls = 0 gives up at once: the failure path's test)
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, int polls = kWaitPolls) {
  for (int it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// named barrier `id` over `n` threads, and its OR-reduction form
__device__ __forceinline__ void bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool bar_or(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, %2, %3, q;\n"
      " selp.u32 %0, 1, 0, o;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes visible to the tensor core's async proxy
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
// the first two columns of this thread's TMEM lane
__device__ __forceinline__ void ld2(uint32_t taddr, float* v) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
}

}  // namespace tc
