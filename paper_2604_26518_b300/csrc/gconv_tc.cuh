// Forward gather convolution of the learned initializer on the 5th-generation tensor cores
// (tcgen05): out[n][co] = act(b[co] + add[n][co] + sum_t sum_ci W[t][ci][co] x[tab[n][t]][ci])
// as an implicit GEMM, D (128 rows x N) = A (128 x 27 cin) B (27 cin x N), with FP16
// operands staged in shared memory and the FP32 accumulator in tensor memory (TMEM).
//
// One CTA of 128 threads owns 128 output rows (one TMEM lane each, the MMA's M = 128) and
// all N <= 128 output channels. It walks the (tap, 32-channel chunk) stages that any of its
// rows uses; per stage every thread gathers its row's 32 input channels (FP16 activations,
// 64 bytes) into the A tile, the CTA copies the stage's prepared FP16 weight image into the
// B tile, and
// one thread issues two K = 16 MMAs and commits them to the stage buffer's mbarrier. Two
// buffers: the gather of stage k overlaps the MMAs of stage k - 1, and buffer k & 1 is
// refilled only after the MMAs of stage k - 2 have completed. Every wait is bounded; a wait
// that runs out records a status, and the CTA stops issuing, waits (bounded) for its
// MMAs in flight, frees its TMEM and returns.
//
// Shared-memory operand layout (no swizzle, K-major core matrices of 8 rows x 16 bytes):
// element (row r, channel c) of a 32-channel stage sits at byte
//     (c / 16) * 4096 + (r / 8) * 256 + ((c % 16) / 8) * 128 + (r % 8) * 16 + (c % 8) * 2,
// so one MMA (16 channels) reads a 4 KB block whose core matrices are 128 bytes apart along
// K (the descriptor's leading byte offset) and 256 bytes apart along M or N (its stride
// byte offset). The same layout holds B with the output channel as the row.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

namespace gmt {

constexpr int TC_ROWS = 128;        // output rows per CTA = TMEM lanes = MMA M
constexpr int TC_KC = 32;           // input channels per stage (two K = 16 MMAs)
constexpr int TC_TILE = 8192;       // bytes of one A stage tile (and of a B tile at N = 128)

__host__ __device__ constexpr int tc_npad(int cout) { return (cout + 15) / 16 * 16; }
__host__ __device__ constexpr int tc_cols(int npad) {
  return npad <= 32 ? 32 : (npad <= 64 ? 64 : 128);
}
// byte offset of (row, channel) in an A stage tile
__host__ __device__ constexpr int tc_offset(int r, int c) {
  return (c / 16) * 4096 + (r / 8) * 256 + ((c % 16) / 8) * 128 + (r % 8) * 16 + (c % 8) * 2;
}

// shared-memory matrix descriptor: start address, leading byte offset (K direction), stride
// byte offset (M/N direction), descriptor version 1 at bits 46-47, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B in FP16 (bits 7-9
// and 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// true once the phase of parity `parity` of the barrier has completed; gives up after
// about `budget` clock cycles (false)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
    __nanosleep(64);
  }
}

__device__ __forceinline__ void tc_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// warp-wide: allocate `ncols` TMEM columns (the base address goes to shared memory at slot)
__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D (+)= A B for one K = 16 step, issued by one thread
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the barrier's phase completes once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  // the loaded registers are valid after the wait: passing them through it orders every
  // later use after the wait
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace gmt
