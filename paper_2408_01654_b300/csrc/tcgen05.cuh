// Fifth-generation tensor-core helpers (tcgen05, sm_100 family) as inline PTX:
// tensor-memory allocation, shared-memory matrix descriptors, the TF32 MMA
// with its accumulator in tensor memory, completion through an mbarrier with
// a bounded wait, and tensor-memory loads for the epilogue.
//
// Operand layout used here: K-major, no swizzle.  A "core matrix" is 8 rows x
// 16 bytes (8 x 4 TF32 values) stored contiguously (128 B); an operand of R
// rows and K columns is stored as core matrices (g, c) (g = row / 8,
// c = k / 4) at byte offset (g * (K / 4) + c) * 128, so adjacent core
// matrices along K are 128 B apart (the descriptor's leading byte offset) and
// adjacent 8-row groups K * 32 B apart (its stride byte offset).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// byte offset of element (row, k) in the K-major, no-swizzle core-matrix layout
__device__ __forceinline__ uint32_t tc_core_offset(int row, int k, int K) {
  return (uint32_t)(((row >> 3) * (K >> 2) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading byte offset (K
// direction), stride byte offset (M/N direction), version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for this architecture
  return d;                // base offset 0, absolute LBO mode, swizzle none
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32 and K-major,
// M x N tile (M = 64 or 128, N a multiple of 16 up to 256 for M = 128).
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4)                          // D format: F32
         | (2u << 7)                        // A format: TF32
         | (2u << 10)                       // B format: TF32
         | ((uint32_t)(N >> 3) << 17)       // N / 8
         | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// --- tensor memory (one warp, all lanes) -----------------------------------
__device__ __forceinline__ void tc_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_addr(smem_dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// --- MMA (one thread) -------------------------------------------------------
// D[tmem] (+)= A * B^T with A: M x 8 and B: N x 8 (K = 8 TF32 values per MMA)
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            int accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on the mbarrier once every MMA issued so far by this thread completed
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tc_smem_addr(mbar))
               : "memory");
}

// --- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void tc_mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_addr(mbar)), "r"(count) : "memory");
}
// Wait for phase `parity` to complete; false after `timeout` cycles.
// The bound on a wait for this CTA's own bulk copies or MMAs: the caller's
// budget for waits on other CTAs, but never less than ~0.1 s at 2 GHz.  Such
// an operation completes in microseconds, and abandoning it while it is still
// in flight would let the CTA release shared or tensor memory under it; a
// short budget (for waits on other CTAs) must not cut these waits short.
constexpr long long TC_HW_WAIT_MIN = 200000000LL;
__device__ __forceinline__ long long tc_hw_bound(long long timeout) {
  return timeout > TC_HW_WAIT_MIN ? timeout : TC_HW_WAIT_MIN;
}

__device__ __forceinline__ bool tc_mbar_wait(uint64_t* mbar, uint32_t parity, long long timeout) {
  const uint32_t a = tc_smem_addr(mbar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > timeout) return false;
  }
}

// --- fences -----------------------------------------------------------------
// generic-proxy shared-memory writes -> visible to the tensor cores
__device__ __forceinline__ void tc_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// --- tensor memory -> registers ---------------------------------------------
// 32 lanes x 32 consecutive 32-bit columns: lane l of the warp gets row
// (lane base + l), columns col..col+31.  The warp may only read the 32 lanes
// 32 * (warp id % 4) ...
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// split x into its nearest TF32 value and the nearest TF32 value of the rest
// (x - hi is exact in FP32): x = hi + lo up to 2^-22 |x|, with round-to-
// nearest (unbiased) errors.  The three products hi*hi + hi*lo + lo*hi then
// carry a product to about FP32 accuracy (lo*lo is below 2^-22 of it).
__device__ __forceinline__ void tc_split(float x, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  const float rest = x - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rest));
  hi = __uint_as_float(h);
  lo = __uint_as_float(l);
}

// --- bulk copies (async proxy) ------------------------------------------------
// the mbarrier's current phase completes once `bytes` more bytes have landed
// (and the one expected arrival, this call, has been made)
__device__ __forceinline__ void tc_mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem_addr(mbar)), "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (multiple of 16; both addresses 16-byte
// aligned) that completes its bytes on the mbarrier
__device__ __forceinline__ void tc_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc_smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(tc_smem_addr(mbar))
               : "memory");
}
// generic-proxy global writes <-> async-proxy (bulk copy) reads
__device__ __forceinline__ void tc_fence_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
