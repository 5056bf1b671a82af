// tcgen05 / TMEM / mbarrier helpers and exact-digit conversions shared by the
// tensor-core kernels (split-precision Gram and TTM).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tk {
namespace tc {

// Bounded mbarrier waits.  mbar_wait polls (each try_wait may block for a
// short hardware-defined time) for at most kTcWaitLimit tries: the choice
// for waits on which a whole CTA's pipeline turns.  mbar_try with a suspend
// hint lets the thread sleep until the phase completes, for at most
// kTcSuspendNs per try, so that a single waiting lane of a role warp takes
// no issue slots from the working warps; its callers give up after
// kTcWaitNs of globaltimer time (or kTcWaitLimit tries).  Expiry is
// reported, never waited past.
constexpr long long kTcWaitLimit = 1ll << 22;
constexpr uint32_t kTcSuspendNs = 20000;
constexpr unsigned long long kTcWaitNs = 2000000000ull;

// tcgen05 instruction descriptor for kind::f16: D = F32, A = B = BF16, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// tcgen05 instruction descriptor for kind::f8f6f4: D = F32, A = B = E4M3
// (format code 0), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, LBO, SBO (bytes), version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: rows of 128 bytes (64 bf16 along K), 8-row atoms of 1 KB at
// stride `sbo`, the 16-byte chunk c of row r stored at chunk c ^ (r % 8).  The
// atoms must be 1024-byte aligned; `addr` may step through a row in 32-byte
// K-steps.  The leading-byte offset is unused for this layout (set to 16).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr, uint32_t sbo) {
  return smem_desc(addr, 16, sbo) | ((uint64_t)2 << 61);
}

// D (TMEM) = A B^T (+ D when accumulate != 0), A and B from shared-memory
// descriptors, kind::f16 with instruction descriptor idesc.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The same with kind::f8f6f4 (8-bit operands, K = 32 per instruction).
__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One try: true once the phase with the given parity has completed; the
// thread may be suspended meanwhile (up to kTcSuspendNs).
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity), "r"(kTcSuspendNs)
      : "memory");
  return ok != 0;
}

// Bounded polling wait for the phase with the given parity; false on expiry.
// one arrival (release semantics at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Tensor-map box loads into shared memory (coordinates innermost first),
// completion counted on mbar in bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit TMEM columns per warp.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 lanes x 8 consecutive 32-bit TMEM columns per warp.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// hi + lo += x (x exact in float), error-free TwoSum then renormalisation.
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  const float l = __fadd_rn(lo, e);
  const float t = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(t, s));
  hi = t;
}

// round(|y| 2^(21 - E)) with the sign of y, from the bits (no float64 math);
// requires |y| < 2^E.
__device__ __forceinline__ int scaled_int(double y, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int shift = 31 + E - (ex - 1023);  // >= 32 because |y| < 2^E
  int v = 0;
  if (shift < 64) v = (int)((mant + (1ull << (shift - 1))) >> shift);
  return (b >> 63) ? -v : v;
}

__device__ __forceinline__ int scaled_int(float y, int E) {
  const unsigned b = __float_as_uint(y);
  const int ex = (int)((b >> 23) & 0xFF);
  if (ex == 0) return 0;
  const unsigned mant = (b & 0x7FFFFFu) | 0x800000u;
  const int shift = 2 + E - (ex - 127);  // >= 3 because |y| < 2^E
  const int v = (shift < 32) ? (int)((mant + (1u << (shift - 1))) >> shift) : 0;
  return (b >> 31) ? -v : v;
}

// Magnitude bits (sign cleared): ordered like the magnitudes.
__device__ __forceinline__ unsigned long long mag_bits(double y) {
  return (unsigned long long)__double_as_longlong(y) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long mag_bits(float y) { return __float_as_uint(y) & 0x7FFFFFFFu; }
// Exponent E with max < 2^E from the largest magnitude's bits; very small for 0.
__device__ __forceinline__ int exp_above(unsigned long long bits, bool is_f64) {
  if (is_f64) {
    const int ex = (int)(bits >> 52);
    return ex == 0 ? -4000 : ex - 1023 + 1;
  }
  const int ex = (int)(bits >> 23);
  return ex == 0 ? -4000 : ex - 127 + 1;
}

// Magnitude of an entry as far as its exponent goes: the high word of a
// double (sign cleared), the bits of a float.  Ordered like the magnitude up
// to ties within a binade, which is all the exponent table needs.
__device__ __forceinline__ unsigned hi_mag(double v) {
  return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7FFFFFFFu;
}
__device__ __forceinline__ unsigned hi_mag(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }
// back to the bit pattern exp_above() reads
__device__ __forceinline__ unsigned long long mag_pattern(unsigned m, bool is_f64) {
  return is_f64 ? (unsigned long long)m << 32 : (unsigned long long)m;
}

// Exact float of an integer |n| < 2^22, without a conversion instruction.
__device__ __forceinline__ float small_int_float(int n) {
  return __fsub_rn(__int_as_float(0x4B400000 + n), 12582912.0f);
}
// round-to-nearest integer of |x| < 2^22 as a float
__device__ __forceinline__ float round_float(float x) { return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f); }

// Two floats that BF16 holds exactly (at most 8 significant bits), packed.
__device__ __forceinline__ uint32_t bf16_pair(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);  // high halves of a and b
}


}  // namespace tc
}  // namespace tk
