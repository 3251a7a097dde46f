// The pair-integral Gram sums of the swaption forms (S3) on the 5th-generation tensor cores.
//
// Per chain the pair tables are Gram sums Y Y^T of the matrix Y[A][k] (absolute panel A, 80
// quadrature columns, see swaption.cuh).  With the split y = hi + lo, hi = bf16(y), lo =
// bf16(y - hi), the CTA stores the operand U = [hi rows; lo rows] (128 x 96, bf16, K-major, no
// swizzle) in shared memory and one thread issues, per Gram,
//     D  = U * hi^T  (+)  U * lo^T          (tcgen05.mma, M = 128, N = 16..64, K = 16 per step)
// into a TMEM accumulator: rows 0..63 of D hold hi (hi + lo)^T and rows 64..127 hold
// lo (hi + lo)^T, so their sum is (hi + lo)(hi + lo)^T, the Gram of the 16-bit-significand
// representation of Y, accumulated in FP32.  The three Grams (outer g nodes, outer h nodes, inner
// g h products) occupy K columns [0, 8), [16, 24) and [32, 96) of U and TMEM columns [0, N),
// [N, 2N), [2N, 3N).  Warps 0-3 read their TMEM lane quarters back (tcgen05.ld) and write the band
// |A - B| < ND of each Gram into the pair tables.
//
// Operand layout (canonical K-major, SWIZZLE_NONE): core matrices of 8 rows x 16 bytes (8 bf16),
// element (row, k) at byte (row / 8) * SBO + (k / 8) * LBO + (row % 8) * 16 + (k % 8) * 2 with
// LBO = 128 (K-adjacent core matrices contiguous) and SBO = 12 * 128 (next 8-row group).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace sabr {

constexpr int kTcRows = 128, kTcK = 96;
constexpr uint32_t kTcLBO = 128, kTcSBO = (kTcK / 8) * 128;      // 1536 bytes
constexpr uint32_t kTcBytes = kTcRows / 8 * kTcSBO;              // 24 KB
constexpr uint32_t kTcCols = 256;                                 // TMEM columns per CTA

__device__ __forceinline__ uint32_t tc_offset(int row, int k) {
  return (uint32_t)(row >> 3) * kTcSBO + (uint32_t)(k >> 3) * kTcLBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// K column of U for quadrature column k of Y (0..79).
__device__ __forceinline__ int tc_kcol(int k) { return k < 8 ? k : (k < 16 ? 16 + (k - 8) : 32 + (k - 16)); }

// Shared-memory matrix descriptor (SM100 layout): start address >> 4 in bits [0,14), LBO >> 4 in
// [16,30), SBO >> 4 in [32,46), version 1 in [46,48), base offset 0, layout SWIZZLE_NONE (0).
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kTcLBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kTcSBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D F32 (bits [4,6) = 1), A and B BF16 (bits [7,10) and
// [10,13) = 1), both K-major, N >> 3 in bits [17,23), M >> 4 in bits [24,29).
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar_saddr) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_saddr) : "memory");
}

// TMEM allocation of kTcCols columns by warp 0; the address lands in *slot (shared memory).
__device__ __forceinline__ void tc_alloc(uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(kTcCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr) {
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Per-CTA tensor-core state: operand buffer, TMEM base, completion barrier and its phase.
struct TcState {
  unsigned char* U;      // kTcBytes, 16-byte aligned
  uint32_t tmem;         // TMEM base address (lane 0, column base)
  uint64_t* mbar;        // completion barrier of the MMAs
  uint32_t phase;        // parity expected by the next wait
  int* err;
};

// Store y (row A of Y, quadrature column k) as hi at row A and lo at row 64 + A.
__device__ __forceinline__ void tc_put(const TcState& tc, int A, int k, float y) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(y);
  const __nv_bfloat16 lo = __float2bfloat16_rn(y - __bfloat162float(hi));
  const int kk = tc_kcol(k);
  *(__nv_bfloat16*)(tc.U + tc_offset(A, kk)) = hi;
  *(__nv_bfloat16*)(tc.U + tc_offset(64 + A, kk)) = lo;
}

// Issue the 12 MMAs of the three Grams and wait for them (every thread calls; bounded wait).
// Returns false if the wait gave up (error word raised).
__device__ __forceinline__ bool tc_gram(TcState& tc, int N) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // U writes -> tensor-core reads
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t u = (uint32_t)__cvta_generic_to_shared(tc.U);
    const uint32_t idesc = tc_idesc(kTcRows, N);
    const uint32_t b_lo = 64u / 8u * kTcSBO;   // rows 64.. of U
    for (int g = 0; g < 3; ++g) {
      const uint32_t d = tc.tmem + (uint32_t)(g * N);
      const int s0 = g == 0 ? 0 : (g == 1 ? 1 : 2), s1 = g == 2 ? 6 : s0 + 1;
      for (int s = s0; s < s1; ++s) {
        const uint32_t koff = (uint32_t)s * 2u * kTcLBO;   // 16 K columns = 2 core matrices
        const uint64_t a = tc_smem_desc(u + koff);
        tc_mma(d, a, tc_smem_desc(u + koff), idesc, s > s0);
        tc_mma(d, a, tc_smem_desc(u + b_lo + koff), idesc, true);
      }
    }
    tc_commit((uint32_t)__cvta_generic_to_shared(tc.mbar));
  }
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(tc.mbar);
  uint32_t done = 0;
  long long it = 0;
  while (!done) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(tc.phase) : "memory");
    if (!done && ++it > (1LL << 24)) break;
  }
  if (!done) {
    atomicOr(tc.err, 2);
    // let the MMAs in flight land before the caller goes on (and, eventually, frees TMEM)
    it = 0;
    while (!done && ++it < (1LL << 24)) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(done) : "r"(bar), "r"(tc.phase) : "memory");
    }
    tc.phase ^= 1u;
    return false;
  }
  tc.phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

}  // namespace sabr
