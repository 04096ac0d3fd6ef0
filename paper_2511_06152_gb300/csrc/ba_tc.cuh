// Fifth-generation tensor cores (tcgen05) for binary64-accurate products of
// double-float matrices, as inline PTX for sm_103a.
//
// Products C = A B^T of matrices stored as double-float (hi + lo binary32
// pairs, about 48 significant bits) are computed exactly in pieces on the
// bf16 tensor cores, after Ozaki, Ogita, Oishi and Rump (2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications"): every row of A and of B is scaled
// by a power of two 2^E (its own), written as a 48-bit fixed-point integer
// and cut into kSlices digits of 8 bits,
//   x = sign * 2^E * sum_t d_t 2^(-8 t),   0 <= d_t <= 255,
// each digit exact in bf16.  The products of digit matrices are sums of
// integers below 2^16; with K = 32 terms per product and at most six
// products per accumulator, every partial sum stays below 2^24 and the
// binary32 accumulation in tensor memory is exact.  Products whose weight
// 2^(-8 (t + u)) lies below 2^-56 are dropped (t + u > kSlices + 1), which
// leaves about 2^-48 of |row of A| |row of B| K: the double-float rounding.
//
// Operand layout in shared memory ("canonical K-major, no swizzle"): the
// matrix is a grid of core matrices of 8 rows x 16 bytes (8 bf16 along K),
// each stored as 128 contiguous bytes (row r at 16 r); core matrices along K
// are kLbo bytes apart, groups of 8 rows kSbo bytes apart.  With K = 32 a
// group holds four core matrices: [group][k chunk][row][8 bf16].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ba_bulk.cuh"
#include "ba_dfloat.cuh"
#include "ba_internal.h"

namespace bagpu {

constexpr int kSlices = 6;            // 8-bit digits of a 48-bit double-float
constexpr int kTcK = 32;              // inner dimension of one product
constexpr int kDiags = 2 * kSlices - (kSlices + 1) + 1;  // accumulators: t + u = 2 .. kSlices + 1
constexpr uint32_t kLbo = 128;        // bytes between core matrices along K
constexpr uint32_t kSbo = 512;        // bytes between groups of 8 rows (4 core matrices of K)
constexpr uint32_t kGroupBytes = 512; // one group of 8 rows x 32 K in bf16
static_assert(kDiags == kSlices, "one accumulator per weight 2^-8c, c = 2 .. kSlices + 1");
static_assert(kSlices == kSlicesHost, "digit buffers are sized on the host with kSlicesHost");

// ---------------------------------------------------------------- digits

// Smallest E with |hi + lo| < 2^E for a double-float whose high word is hi
// (|lo| <= ulp(hi) / 2 keeps the sum below the next power of two); zero
// gives a very small E so that it never sets a row's scale.
__device__ __forceinline__ int df_exp_bound(float hi) {
  const uint32_t b = __float_as_uint(hi) & 0x7fffffffu;
  if (b == 0) return -100000;
  const int be = (int)(b >> 23);
  return (be == 0 ? -126 : be - 127) + 1;
}

// |v| * 2^(48 - E) truncated toward zero, for a binary32 v with |v| < 2^E
// (as a signed 64-bit integer).
__device__ __forceinline__ long long fixed48(float v, int E) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t mag = b & 0x7fffffffu;
  if (mag == 0) return 0;
  const int be = (int)(mag >> 23);
  const uint32_t m = be == 0 ? (mag & 0x7fffffu) : ((mag & 0x7fffffu) | 0x800000u);
  const int e = be == 0 ? -126 : be - 127;  // v = m 2^(e - 23)
  const int sh = e - 23 + 48 - E;           // v 2^(48 - E) = m 2^sh, sh <= 24
  long long q;
  if (sh >= 0) q = (long long)m << sh;
  else q = (-sh >= 32) ? 0 : (long long)(m >> (-sh));
  return (b >> 31) ? -q : q;
}

// bf16 bit pattern of sign * d for an integer 0 <= d <= 255 (exact: d has at
// most 8 significant bits; the binary32 value's low half is zero).
__device__ __forceinline__ uint16_t digit_bf16(uint32_t d, uint32_t sign) {
  const float f = __fsub_rn(__uint_as_float(0x4B000000u | d), 8388608.0f);
  return (uint16_t)((__float_as_uint(f) >> 16) | (sign << 15));
}

// The kSlices digits of a double-float x relative to 2^E (|x| < 2^E), as bf16
// bit patterns (sign applied to every digit).
__device__ __forceinline__ void df_digits(dfl x, int E, uint16_t (&dg)[kSlices]) {
  const long long q = fixed48(x.hi, E) + fixed48(x.lo, E);
  const uint32_t sign = q < 0 ? 1u : 0u;
  const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
#pragma unroll
  for (int t = 0; t < kSlices; ++t) dg[t] = digit_bf16((uint32_t)(a >> (40 - 8 * t)) & 0xffu, sign);
}

// Byte offset of element (row r, k) of one digit matrix in the canonical
// layout (32 K values per row).
__device__ __forceinline__ uint32_t canon_off(int r, int k) {
  return (uint32_t)((r >> 3) * kGroupBytes + (k >> 3) * kLbo + (r & 7) * 16 + (k & 7) * 2);
}

// 2^e as binary32 for -126 <= e <= 127, else the nearest end (the callers'
// scales stay far inside the range).
__device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __uint_as_float((uint32_t)(e + 127) << 23);
}

// x * 2^e for a double-float, as two exact power-of-two steps (e may lie
// outside the binary32 exponent range by up to a factor of two).
__device__ __forceinline__ dfl df_ldexp(dfl x, int e) {
  const int e1 = e / 2, e2 = e - e1;
  const float s1 = pow2f(e1), s2 = pow2f(e2);
  return dfl{__fmul_rn(__fmul_rn(x.hi, s1), s2), __fmul_rn(__fmul_rn(x.lo, s1), s2)};
}

// sum_c acc[c] 2^(-8 (c + 2)) as a double-float (every acc is an integer
// below 2^24 in magnitude: each term is exact; TwoSum accumulation from the
// smallest weight up).
__device__ __forceinline__ dfl combine_diags(const float (&acc)[kDiags]) {
  dfl s = dfl{__fmul_rn(acc[kDiags - 1], pow2f(-8 * (kDiags + 1))), 0.0f};
#pragma unroll
  for (int c = kDiags - 2; c >= 0; --c) s = df_add_f(s, __fmul_rn(acc[c], pow2f(-8 * (c + 2))));
  return s;
}

// ---------------------------------------------------------------- tcgen05

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((kLbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((kSbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);  // no swizzle
}

// kind::f16 instruction descriptor: bf16 A and B, binary32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Allocate ncols tensor-memory columns (one full warp); the base address is
// written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A B^T, one instruction (K = 16 for bf16), issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on the mbarrier once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 8 consecutive columns of this thread's tensor-memory lane (32x32b shape:
// thread i of the warp reads lane (warp's lane base) + i).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Issue the digit products of one tile: for every pair of digits (t, u)
// with t + u <= kSlices + 1, D_(t+u) += A_t B_u^T over K = 32 (two
// instructions of K = 16).  a_base / b_base: shared addresses of digit
// matrix 0 of A / B; a_step / b_step: bytes between digit matrices.
// Accumulator c (weight 2^(-8 (c + 2))) sits at tmem + c * N columns.
template <int M, int N>
__device__ __forceinline__ void issue_digit_products(uint32_t tmem, uint32_t a_base, uint32_t a_step,
                                                     uint32_t b_base, uint32_t b_step) {
  constexpr uint32_t idesc = idesc_bf16(M, N);
#pragma unroll
  for (int c = 0; c < kDiags; ++c) {
    const int s = c + 2;  // t + u
    bool first = true;
#pragma unroll
    for (int t = 1; t <= kSlices; ++t) {
      const int u = s - t;
      if (u < 1 || u > kSlices) continue;
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint64_t ad = smem_desc(a_base + (uint32_t)(t - 1) * a_step + (uint32_t)kk * 2 * kLbo);
        const uint64_t bd = smem_desc(b_base + (uint32_t)(u - 1) * b_step + (uint32_t)kk * 2 * kLbo);
        mma_bf16(tmem + (uint32_t)(c * N), ad, bd, idesc, first ? 0u : 1u);
        first = false;
      }
    }
  }
}

}  // namespace bagpu
