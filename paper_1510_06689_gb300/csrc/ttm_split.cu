// Split-precision mode-n product on the 5th-generation tensor cores.
//
// The TTM step of Algorithm 1 (Y <- Y x_n U_n^T, Sec. 2.1 and 2.2) computes
// y'_rc = sum_j U[j, r] y_jc for every column c of the unfolding.  On GB300
// the float64 pipe makes it the largest phase once the Gram runs on the
// tensor cores, so it moves there too, with the exact-digit scheme of the
// split Gram:
//
//   * U's column r is scaled by 2^(28 - e_r) (2^e_r above its largest
//     magnitude) and every column c of Y (its J entries, all inside one tile)
//     by 2^(28 - f_c); both are rounded to integers and split into four
//     digits v = s1 2^21 + s2 2^14 + s3 2^7 + s4, exact in BF16 (U's
//     balanced, |s1| <= 128, |s2..s4| <= 64; Y's with |s1|, |s3| <= 128).  The TTM output feeds every later mode
//     and the core, so it keeps 28 bits (21 were measurably too few).
//   * D = U_a Y_b^T products of levels a + b = 2..5 go to four exact TMEM
//     accumulators:
//       acc0 = U1 Y1^T,  acc1 = U1 Y2^T + U2 Y1^T,
//       acc2 = U1 Y3^T + U2 Y2^T + U3 Y1^T,
//       acc3 = U1 Y4^T + U2 Y3^T + U3 Y2^T + U4 Y1^T.
//     Y's digits come from a 14-bit split of v (below), so its third digit
//     reaches 128 too; with J <= 128 every level stays below 2^22 (acc2,
//     acc3 <= 128 (3 2^13 + 2^12)), so all four are exact integers.  Levels 6..8 (products of two low
//     digits of different entries, zero-mean) are dropped: at most ~2^-27 of
//     sum_j |U_jr| |y_jc|.
//   * Each output is assembled exactly in int64,
//     v = 2^28 acc0 + 2^21 acc1 + 2^14 acc2 + 2^7 acc3 (< 2^50),
//     converted to float64 and scaled by 2^(e_r + f_c - 42).
//
// The product is that of U and Y rounded to 28 bits below their local powers
// of two (zero-mean rounding), up to the dropped levels: a relative
// perturbation of ~1e-8 of each output column.
// A CTA keeps U's digits in shared memory and streams tiles of 128 columns
// through two operand stages (see the kernel comment below).  Waits are bounded and
// CTA-uniform; on expiry the kernel flags an error, waits (bounded) for its
// MMAs, frees TMEM and returns.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tk {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kM = 128;           // output rows r (R zero-padded)
constexpr int kMaxJp = 128;       // contraction length of one kernel pass, padded to a multiple of 16
constexpr int kMaxSplitJ = 512;   // longer contractions run in passes of kMaxJp rows
constexpr int kATiles = 4;        // U1..U4
constexpr int kBTiles = 4;        // Y1..Y4

// round(|y| 2^(28 - E)) with the sign of y; requires |y| < 2^E.
__device__ __forceinline__ int scaled_int28(double y, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int shift = 24 + E - (ex - 1023);  // >= 25
  const int v = shift < 64 ? (int)((mant + (1ull << (shift - 1))) >> shift) : 0;
  return (b >> 63) ? -v : v;
}
__device__ __forceinline__ int scaled_int28(float y, int E) {
  const unsigned b = __float_as_uint(y);
  const int ex = (int)((b >> 23) & 0xFF);
  if (ex == 0) return 0;
  const unsigned long long mant = (b & 0x7FFFFFu) | 0x800000u;
  const int shift = E - (ex - 127) - 5;  // >= -4
  int v;
  if (shift <= 0) v = (int)(mant << (-shift));
  else v = shift < 64 ? (int)((mant + (1ull << (shift - 1))) >> shift) : 0;
  return (b >> 31) ? -v : v;
}

__device__ __forceinline__ void digits4(int v, int (&d)[4]) {
  d[0] = (v + (1 << 20)) >> 21;
  const int r1 = v - (d[0] << 21);
  d[1] = (r1 + (1 << 13)) >> 14;
  const int r2 = r1 - (d[1] << 14);
  d[2] = (r2 + 64) >> 7;
  d[3] = r2 - (d[2] << 7);
}

// v 2^sc as a float64, assembled from the bits (v has at most 50 significant
// bits, so the conversion is exact); results below the normal range flush to 0.
__device__ __forceinline__ double scaled_ll_to_double(long long v, int sc) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(a);
  const int ex = 63 - lz;                                       // a in [2^ex, 2^(ex+1))
  const unsigned long long frac = ((a << lz) << 1) >> 12;        // the 52 bits after the leading 1
  const int be = ex + 1023 + sc;
  if (be <= 0) return 0.0;
  if (be >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | frac));
}

// v = round(|y| 2^(28 - f)) (ties away from zero) for |y| < 2^f, as four
// digits v = d0 2^21 + d1 2^14 + d2 2^7 + d3 carrying y's sign, as exact
// floats (|d0|, |d2| <= 128, |d1|, |d3| <= 64).  With m29 the leading 29 bits
// of the significand (its 24 bits, shifted, for float) and sh the distance of
// y's exponent below f (>= 0), t = m29 >> sh and v = (t + 1) >> 1: the
// dropped bits decide no rounding the kept ones do not.  The integer part is
// kept short (the integer pipe is the busy one in this kernel): v's top and
// low 14 bits become exact floats by placing them below the exponent bits of
// 2^23 (with y's sign) and subtracting 2^23, and each splits into two base-128
// digits by round-to-nearest on the float pipe.  Zeros and subnormals give 0.
__device__ __forceinline__ void digits28_from_t(unsigned t, unsigned sign, float (&d)[4]) {
  const unsigned t1 = t + 1u;
  const unsigned M = sign | 0x4B000000u;  // the bits of +-2^23
  const float mf = __uint_as_float(M);
  const float fh = __fsub_rn(__uint_as_float((t1 >> 15) | M), mf);             // +-(v >> 14) <= 2^14
  const float fl = __fsub_rn(__uint_as_float(((t1 >> 1) & 0x3FFFu) | M), mf);  // +-(v mod 2^14)
  constexpr float kRound = 12582912.0f;                                        // 1.5 2^23
  d[0] = __fsub_rn(__fmaf_rn(fh, 0x1p-7f, kRound), kRound);
  d[1] = __fmaf_rn(d[0], -128.0f, fh);
  d[2] = __fsub_rn(__fmaf_rn(fl, 0x1p-7f, kRound), kRound);
  d[3] = __fmaf_rn(d[2], -128.0f, fl);
}
// the pair (a, b) as BF16 (a in the low half), by the conversion instruction;
// exact for values with at most 8 significant bits
__device__ __forceinline__ uint32_t bf16_pack(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
__device__ __forceinline__ unsigned shr_clamped(unsigned x, unsigned sh) {  // x >> sh, 0 for sh >= 32
  unsigned r;
  asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(sh));
  return r;
}
// f1022 = f + 1022
__device__ __forceinline__ void digits28(double y, int f1022, float (&d)[4]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned ex = (hi >> 20) & 0x7FFu;
  const unsigned m29 = __funnelshift_l(lo, (hi & 0xFFFFFu) | 0x100000u, 8);  // (m53 >> 24)
  unsigned t = shr_clamped(m29, (unsigned)(f1022 - (int)ex));
  t = ex ? t : 0u;
  digits28_from_t(t, hi & 0x80000000u, d);
}
__device__ __forceinline__ void digits28(float y, int f1022, float (&d)[4]) {
  const unsigned b = __float_as_uint(y);
  const unsigned ex = (b >> 23) & 0xFFu;
  const unsigned m29 = ((b & 0x7FFFFFu) | 0x800000u) << 5;
  unsigned t = shr_clamped(m29, (unsigned)(f1022 - 896 - (int)ex));  // f + 126 - ex
  t = ex ? t : 0u;
  digits28_from_t(t, b & 0x80000000u, d);
}

// sum_k a_k 2^(28 - 7k) 2^sc as a float64, from four float accumulators that
// hold integers |a_k| < 2^22 (the levels 2..5 of a digit product): the
// integers come out of the floats exactly by magic-number addition, pairs
// combine in 32 bits (|a0 2^7 + a1| < 2^30, likewise a2, a3), and one wide
// multiply-add forms w = (a0 2^7 + a1) 2^14 + a2 2^7 + a3, the sum over
// 2^7 (|w| < 2^45, exact in float64, where it is converted).  The
// power-of-two scale 2^(sc + 7) is either a float64 multiply (kFp64Scale:
// where the integer pipe is the busy one and the float64 pipe, narrow on
// this part, has room for a second instruction) or an integer add to the
// exponent field; both are exact while the result stays normal (w's
// exponent is at most 44, so -1022 <= sc + 7 <= 979 suffices).  Other scales
// take the exact bit assembly.
template <bool kFp64Scale>
__device__ __forceinline__ double levels_to_double(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, int sc) {
  constexpr unsigned kMagic = 0x4B400000u;  // the bits of 1.5 2^23
  const unsigned u0 = __float_as_uint(__fadd_rn(__uint_as_float(a0), 12582912.0f));
  const unsigned u1 = __float_as_uint(__fadd_rn(__uint_as_float(a1), 12582912.0f));
  const unsigned u2 = __float_as_uint(__fadd_rn(__uint_as_float(a2), 12582912.0f));
  const unsigned u3 = __float_as_uint(__fadd_rn(__uint_as_float(a3), 12582912.0f));
  // two's-complement wrap-around: the results are the signed pair values
  const int hi = (int)((u0 - kMagic) * 128u + (u1 - kMagic));
  const int lo = (int)((u2 - kMagic) * 128u + (u3 - kMagic));
  const long long w = (long long)hi * 16384 + lo;
  const int s7 = sc + 7;
  if (s7 >= -1022 && s7 <= 979) {
    if (kFp64Scale) return __dmul_rn((double)w, __longlong_as_double((long long)(s7 + 1023) << 52));
    const long long b = __double_as_longlong((double)w);
    return w ? __longlong_as_double(b + ((long long)s7 << 52)) : 0.0;
  }
  return scaled_ll_to_double(w, s7);
}

// ---------------------------------------------------------------------------
// The 128 columns of a tile are the M = 128 rows of the MMA (A = Y's digits)
// and the factor is the N operand (B = U's digits, N = R rounded up to 16).  One MMA then covers 128 columns, each column's exponent belongs
// to one TMEM lane, and no MMA rows are padding.  The contraction (J) runs in
// k-parts of 64 (32 when R > 64) through two operand stages; a tile's entries
// are loaded into registers first, for the column exponents, and converted
// part by part.  With R <= 64 two TMEM accumulator sets let the previous tile
// drain while the tensor cores work on the next one.
// ---------------------------------------------------------------------------
constexpr int kM2 = 128;

struct TtmSplit2Plan {
  int J, Jp, R, Rp, KH, parts, sets, tmem_cols;
  int64_t K, ntiles;
  int grid;
  size_t smem;
  // a part of a longer contraction (J > 128): Y's rows and U's rows are J of
  // ldj (Y's view (L, ldj, B) and U ldu x R, both offset by the caller) and
  // accum adds the part's product to Z instead of storing it
  int64_t ldj, ldu;
  int accum;
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_ttm_split2(const T *__restrict__ y, int64_t L, int64_t B,
                                                            const double *__restrict__ U, TtmSplit2Plan p,
                                                            double *__restrict__ z, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long mbar[2];   // operand stages
  __shared__ __align__(8) unsigned long long tbar[2];   // accumulator sets (tile done)
  __shared__ unsigned colmax[kM2];
  __shared__ int colexp[2][kM2];
  __shared__ int64_t colout[2][kM2];
  __shared__ int rowexp[kM];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  constexpr bool kF64 = sizeof(T) == 8;
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  const int Jp = p.Jp, Rp = p.Rp, KH = p.KH;
  const int u_tile = p.Rp * Jp * 2;          // bytes of one U digit tile (B: Rp rows x Jp)
  const int a_tile = kM2 * KH * 2;           // bytes of one Y digit tile (A: 128 rows x KH)
  const uint32_t sbo_u = (uint32_t)(Jp / 8) * 128u, sbo_a = (uint32_t)(KH / 8) * 128u;
  unsigned char *Ut = base;                          // 4 tiles
  unsigned char *Ast = base + 4 * u_tile;            // 2 stages x 4 tiles
  const uint32_t idesc = idesc_bf16(kM2, Rp);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_addr(&mbar[k]), 1);
      mbar_init(smem_addr(&tbar[k]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
  }
  if (tid < kM) {
    unsigned long long m = 0ull;
    if (tid < p.R)
      for (int j = 0; j < p.J; ++j) m = max(m, mag_bits(U[j + p.ldu * tid]));
    rowexp[tid] = exp_above(m, true);
  }
  __syncthreads();
  // U's digit tiles (B operands: row r, k = j)
  for (int u = tid; u < Rp * (Jp / 8); u += kThreads) {
    const int r = u / (Jp / 8), jg = u % (Jp / 8);
    uint32_t w[kATiles][4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      int d[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 8 * jg + k + h;
        const double v = (r < p.R && j < p.J) ? U[j + p.ldu * r] : 0.0;
        digits4(scaled_int28(v, rowexp[r]), d[h]);
      }
#pragma unroll
      for (int t = 0; t < kATiles; ++t) w[t][k >> 1] = bf16_pair((float)d[0][t], (float)d[1][t]);
    }
    const int off = (r >> 3) * (int)sbo_u + jg * 128 + (r & 7) * 16;
#pragma unroll
    for (int t = 0; t < kATiles; ++t)
      *reinterpret_cast<uint4 *>(Ut + t * u_tile + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const int64_t in_b = L * p.ldj, out_b = L * (int64_t)p.R;
  const int ngr = Jp / 8;                       // 8-row groups of a column
  const int upt = (kM2 * ngr + kThreads - 1) / kThreads;  // load units per thread (<= 4)
  const int my_c = tid % kM2;
  const int jg0 = tid / kM2;                    // units jg0, jg0 + 4, jg0 + 8, jg0 + 12

  T raw[4][8];
  int64_t my_in = -1;
  auto load_tile = [&](int64_t t) {
    const int64_t c = t * kM2 + my_c;
    my_in = -1;
    if (c < p.K) {
      const int64_t b = c / L, l = c - b * L;
      my_in = l + in_b * b;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int jg = jg0 + 4 * k;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * jg + e;
        raw[k][e] = (k < upt && jg < ngr && my_in >= 0 && j < p.J) ? __ldg(y + my_in + L * (int64_t)j) : T(0);
      }
    }
  };

  auto drain = [&](int64_t t, int set, int dcount) {
    // the dcount-th tile on this set completes that barrier's phase dcount
    if (tid == 0 && !mbar_wait(smem_addr(&tbar[set]), dcount & 1)) stop = 1;
    __syncthreads();
    if (!stop) {
      fence_after();
      const int q = warp & 3, g = warp >> 2;         // lanes 32 q.., r-quarter g
      const int c = 32 * q + lane;
      const int64_t ob = colout[set][c];
      const int rq = Rp / 4;
      const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(set * 4 * Rp);
      for (int r0 = g * rq; r0 < (g + 1) * rq; r0 += 4) {
        uint32_t a[4][4];
#pragma unroll
        for (int lev = 0; lev < 4; ++lev) {
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(a[lev][0]), "=r"(a[lev][1]), "=r"(a[lev][2]), "=r"(a[lev][3])
                       : "r"(tb + (uint32_t)(lev * Rp + r0)));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ob >= 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int r = r0 + e;
            if (r >= p.R) continue;
            const double v = levels_to_double<false>(a[0][e], a[1][e], a[2][e], a[3][e], rowexp[r] + colexp[set][c] - 42);
            double *zp = z + ob + L * (int64_t)r;
            *zp = p.accum ? *zp + v : v;
          }
        }
      }
    }
    fence_before();
    __syncthreads();
  };

  int64_t unit = 0;          // (tile, part) units issued so far
  int tcount[2] = {0, 0};    // tiles committed per accumulator set
  int64_t prev_t = -1;
  int prev_set = 0, it = 0;
  int64_t t = blockIdx.x;
  if (t < p.ntiles) load_tile(t);
  for (; t < p.ntiles; t += gridDim.x, ++it) {
    const int set = (p.sets == 2) ? (it & 1) : 0;
    // column exponents and output addresses of this tile
    if (tid < kM2) colmax[tid] = 0u;
    __syncthreads();
    {
      unsigned m = 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int e = 0; e < 8; ++e) m = max(m, hi_mag(raw[k][e]));
      atomicMax(&colmax[my_c], m);
    }
    if (tid < kM2) {
      const int64_t c = t * kM2 + tid;
      int64_t ob = -1;
      if (c < p.K) {
        const int64_t b = c / L, l = c - b * L;
        ob = l + out_b * b;
      }
      colout[set][tid] = ob;
    }
    __syncthreads();
    if (tid < kM2) colexp[set][tid] = exp_above(mag_pattern(colmax[tid], kF64), kF64);
    __syncthreads();
    const int e_col = colexp[set][my_c];
    for (int part = 0; part < p.parts; ++part, ++unit) {
      const int stg = (int)(unit & 1);
      if (unit >= 2 && tid == 0 && !mbar_wait(smem_addr(&mbar[stg]), (int)(((unit - 2) >> 1) & 1))) stop = 1;
      __syncthreads();
      if (stop) break;
      unsigned char *st = Ast + stg * 4 * a_tile;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int jg = jg0 + 4 * k;
        if (k >= upt || jg >= ngr || jg / (KH / 8) != part) continue;
        uint32_t w[kBTiles][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          float d0[4], d1[4];
          digits28(raw[k][e], e_col + 1022, d0);
          digits28(raw[k][e + 1], e_col + 1022, d1);
#pragma unroll
          for (int q = 0; q < kBTiles; ++q) w[q][e >> 1] = bf16_pair(d0[q], d1[q]);
        }
        const int jl = jg % (KH / 8);
        const int off = (my_c >> 3) * (int)sbo_a + jl * 128 + (my_c & 7) * 16;
#pragma unroll
        for (int q = 0; q < kBTiles; ++q)
          *reinterpret_cast<uint4 *>(st + q * a_tile + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        fence_after();
        const uint32_t ab = smem_addr(st), ub = smem_addr(Ut);
        const uint32_t d0 = tmem + (uint32_t)(set * 4 * Rp);
        for (int ks = 0; ks < KH / 16; ++ks) {
          const uint32_t acc = (part == 0 && ks == 0) ? 0u : 1u;
          uint64_t ya[kBTiles], ub4[kATiles];
#pragma unroll
          for (int q = 0; q < kBTiles; ++q) ya[q] = smem_desc(ab + q * a_tile + 256 * ks, 128, sbo_a);
#pragma unroll
          for (int q = 0; q < kATiles; ++q)
            ub4[q] = smem_desc(ub + q * u_tile + (uint32_t)(part * (KH / 8) * 128) + 256 * ks, 128, sbo_u);
          mma_bf16(d0 + 0 * Rp, ya[0], ub4[0], idesc, acc);
          mma_bf16(d0 + 1 * Rp, ya[0], ub4[1], idesc, acc);
          mma_bf16(d0 + 1 * Rp, ya[1], ub4[0], idesc, 1u);
          mma_bf16(d0 + 2 * Rp, ya[0], ub4[2], idesc, acc);
          mma_bf16(d0 + 2 * Rp, ya[1], ub4[1], idesc, 1u);
          mma_bf16(d0 + 2 * Rp, ya[2], ub4[0], idesc, 1u);
          mma_bf16(d0 + 3 * Rp, ya[0], ub4[3], idesc, acc);
          mma_bf16(d0 + 3 * Rp, ya[1], ub4[2], idesc, 1u);
          mma_bf16(d0 + 3 * Rp, ya[2], ub4[1], idesc, 1u);
          mma_bf16(d0 + 3 * Rp, ya[3], ub4[0], idesc, 1u);
        }
        mma_commit(smem_addr(&mbar[stg]));
        if (part == p.parts - 1) mma_commit(smem_addr(&tbar[set]));
      }
    }
    if (stop) break;
    const int my_count = tcount[set]++;
    // prefetch the next tile, then drain (the previous tile, or this one with a single set)
    if (t + gridDim.x < p.ntiles) load_tile(t + gridDim.x);
    if (p.sets == 2) {
      if (prev_t >= 0) drain(prev_t, prev_set, tcount[prev_set] - 1);
      prev_t = t;
      prev_set = set;
    } else {
      drain(t, set, my_count);
    }
    if (stop) break;
  }
  if (!stop && p.sets == 2 && prev_t >= 0) drain(prev_t, prev_set, tcount[prev_set] - 1);
  if (stop && tid == 0) {  // let our own MMAs finish before TMEM is released
    if (unit >= 1) mbar_wait(smem_addr(&mbar[(unit - 1) & 1]), (int)(((unit - 1) >> 1) & 1));
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
  if (stop && tid == 0) atomicExch(err, 1);
}

TtmSplit2Plan ttm_split2_plan(int64_t L, int64_t J, int64_t B, int64_t R, const DeviceInfo &dev) {
  TtmSplit2Plan p{};
  p.J = (int)J;
  p.Jp = (int)((J + 15) / 16 * 16);
  p.R = (int)R;
  p.Rp = (int)((R + 15) / 16 * 16);
  p.KH = (p.Rp <= 64) ? std::min(64, p.Jp) : std::min(32, p.Jp);
  if (p.Jp % p.KH) p.KH = 16;
  p.parts = p.Jp / p.KH;
  p.sets = (8 * p.Rp <= 512) ? 2 : 1;
  int cols = p.sets * 4 * p.Rp;
  p.tmem_cols = 32;
  while (p.tmem_cols < cols) p.tmem_cols <<= 1;
  p.K = L * B;
  p.ntiles = (p.K + kM2 - 1) / kM2;
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(dev.sms, p.ntiles));
  p.smem = (size_t)4 * p.Rp * p.Jp * 2 + (size_t)2 * 4 * kM2 * p.KH * 2 + 1024;
  p.ldj = J;
  p.ldu = J;
  p.accum = 0;
  return p;
}

// ---------------------------------------------------------------------------
// L == 1 (the first mode of the natural layout): column c of the unfolding
// is the contiguous vector y[c J .. c J + J - 1].  The CTA's warps have
// fixed roles and meet only at mbarriers, so conversion, tensor-core work
// and the drain of the previous tile overlap:
//   16 converter warps take whole columns (8 per warp per tile) in halves of
//      64 entries (the K-parts of the MMA): lanes read consecutive 16-byte
//      pairs (coalesced), scale them by the column exponent (from the
//      exponent pass, or a pass of its own) and write each digit row to a
//      128-byte swizzled K-major tile (one row per store instruction, no
//      bank conflicts).  All first halves of a tile are written before the
//      second halves, so the MMAs of one half run while the other is
//      converted; eight half-columns per warp are in flight in registers;
//   1 MMA warp issues each half's MMAs (columns are the M = 128 rows, U the
//      N operand: 4 MMAs per k-step, one per digit of Y against U's stacked
//      digit tiles) into one of two TMEM accumulator sets;
//   8 drain warps (two per TMEM lane quarter) assemble each output exactly
//      from the four levels and store it from registers (a thread's four
//      consecutive outputs of one column fill one 32-byte sector).
// Barriers: part_full[2] (converters -> MMA: a half's digits written),
// part_free[2] (MMA commit: a half's digits read), acc_full[2] (MMA commit:
// a set holds a finished tile), acc_free[2] (drain -> MMA: set read out).
// Every wait is bounded and also gives up once another role has flagged an
// error.
// ---------------------------------------------------------------------------
struct TtmL1Plan {
  int J, Jp, R, Rp, parts, tmem_cols;
  int64_t K, ntiles;
  int grid;
  size_t u_bytes, a_bytes, smem;
};

constexpr int kL1Conv = 16;                             // converter warps
constexpr int kL1Drain = 8;                             // drain warps (two per TMEM lane quarter)
constexpr int kL1Threads = (kL1Conv + kL1Drain + 1) * 32;
constexpr int kL1ColsPerWarp = kM2 / kL1Conv;           // 8

// round(|y| 2^(28 - f)) etc. are above; the two roles' bounded wait:
// true once the phase of `parity` has completed, false on expiry (which
// raises *stop) or when another role has raised *stop.
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile int *stop) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*stop) return false;
    if (global_ns() - t0 > kTcWaitNs) break;
  }
  *stop = 1;
  return false;
}

// P: K-parts of 64 entries (1 for J <= 64, else 2); colexp: the exponent
// above each column's largest magnitude.
template <typename T, int P>
__global__ void __launch_bounds__(kL1Threads, 1) k_ttm_split_l1(const T *__restrict__ y, const double *__restrict__ U,
                                                              const int *__restrict__ colexp, TtmL1Plan p,
                                                              double *__restrict__ z, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long part_full[2], part_free[2], acc_full[2], acc_free[2];
  __shared__ int rowexp[kM];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int stop;
  constexpr bool kF64 = sizeof(T) == 8;
  using V2 = typename std::conditional<kF64, double2, float2>::type;
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char *At = base;                                  // 4 digit tiles, SW128 K-major
  unsigned char *Ut = base + p.a_bytes;                      // 4 digit tiles, no swizzle
  const int a_tile = P * kM2 * 128;
  const int u_tile = p.Rp * p.Jp * 2;
  const uint32_t sbo_u = (uint32_t)(p.Jp / 8) * 128u;
  uint32_t idesc_q[kBTiles];  // N = (4 - q) Rp: digit q of Y against U1 .. U(4-q)
#pragma unroll
  for (int q = 0; q < kBTiles; ++q) idesc_q[q] = idesc_bf16(kM2, (kBTiles - q) * p.Rp);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_addr(&part_full[k]), kL1Conv);
      mbar_init(smem_addr(&part_free[k]), 1);
      mbar_init(smem_addr(&acc_full[k]), 1);
      mbar_init(smem_addr(&acc_free[k]), kL1Drain);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
  }
  if (tid < kM) {
    unsigned long long m = 0ull;
    if (tid < p.R)
      for (int j = 0; j < p.J; ++j) m = max(m, mag_bits(U[j + (int64_t)p.J * tid]));
    rowexp[tid] = exp_above(m, true);
  }
  __syncthreads();
  // U's digit tiles (B operands: row r, k = j), as in the general kernel
  for (int u = tid; u < p.Rp * (p.Jp / 8); u += kL1Threads) {
    const int r = u / (p.Jp / 8), jg = u % (p.Jp / 8);
    uint32_t w[kATiles][4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      int d[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 8 * jg + k + h;
        const double v = (r < p.R && j < p.J) ? U[j + (int64_t)p.J * r] : 0.0;
        digits4(scaled_int28(v, rowexp[r]), d[h]);
      }
#pragma unroll
      for (int t = 0; t < kATiles; ++t) w[t][k >> 1] = bf16_pair((float)d[0][t], (float)d[1][t]);
    }
    const int off = (r >> 3) * (int)sbo_u + jg * 128 + (r & 7) * 16;
#pragma unroll
    for (int t = 0; t < kATiles; ++t)
      *reinterpret_cast<uint4 *>(Ut + t * u_tile + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
  // zero the A tiles once: K columns past Jp (up to the 64-wide part) stay zero
  for (int e = tid; e < (int)(p.a_bytes / 16); e += kL1Threads) reinterpret_cast<uint4 *>(At)[e] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const int64_t t0 = blockIdx.x, tstride = gridDim.x;
  const int ntc = t0 < p.ntiles ? (int)((p.ntiles - t0 + tstride - 1) / tstride) : 0;

  if (warp < kL1Conv) {
    // ---------------- converters ----------------
    // tile it seen from this warp: its first column (warp) as a pointer to
    // this lane's pair of entries (j = 2 lane) and to the column's exponent,
    // and how many of the tile's columns lie from that one on; slot k (column
    // warp + 16 k) holds data while 16 k < cols.  The next tile's view is
    // formed once per tile (at its last half, so that the two views are not
    // held at once), and a load is an offset from a view and one compare.
    struct View {
      const T *yp;
      const int *ep;
      int cols;
    };
    auto view_of = [&](int it) {
      View v;
      const int64_t c0 = (t0 + (int64_t)it * tstride) * kM2 + warp;
      v.yp = y + c0 * (int64_t)p.J + 2 * lane;
      v.ep = colexp + c0;
      const int64_t left = it < ntc ? p.K - c0 : 0;
      v.cols = (int)(left < kM2 ? (left > 0 ? left : 0) : kM2);
      return v;
    };
    const int slot_elems = kL1Conv * p.J;  // entries between a warp's consecutive columns
    bool jok[P];
#pragma unroll
    for (int h = 0; h < P; ++h) jok[h] = 2 * lane + 64 * h < p.J;
    // half h (entries j = 2 lane + 64 h, a pair) of slot k's column
    auto load_half = [&](const View &t, int k, int h, V2 &v) {
      if (kL1Conv * k < t.cols && jok[h])
        v = __ldg(reinterpret_cast<const V2 *>(t.yp + k * slot_elems + 64 * h));
      else
        v.x = v.y = T(0);
    };
    auto load_exp = [&](const View &t, int k) { return kL1Conv * k < t.cols ? __ldg(t.ep + kL1Conv * k) : 0; };
    // slot k holds column warp + 16 k: its current half, and its exponent
    V2 cb[kL1ColsPerWarp];
    int fx[kL1ColsPerWarp];
    View cur = view_of(0);
#pragma unroll
    for (int k = 0; k < kL1ColsPerWarp; ++k) {
      load_half(cur, k, 0, cb[k]);
      fx[k] = load_exp(cur, k);
    }
    // this lane's byte offset within a digit row: 16-byte chunk lane / 4 of the
    // 128-byte row, XOR-swizzled by the row's index mod 8 (= warp mod 8 for
    // every column of this warp)
    const int lane_off = (((lane >> 2) ^ (warp & 7)) << 4) + (lane & 3) * 4;
    bool ok = true;
    for (int it = 0; it < ntc && ok; ++it) {
      View nxt = cur;
#pragma unroll
      for (int h = 0; h < P; ++h) {
        if (h == P - 1) nxt = view_of(it + 1);  // after the last use of cur's pointer
        if (it >= 1) {  // the previous tile's MMAs have read this half
          int w = 0;
          if (lane == 0) w = role_wait(smem_addr(&part_free[h]), (uint32_t)((it - 1) & 1), &stop);
          if (!__shfl_sync(0xffffffffu, w, 0)) {
            ok = false;
            break;
          }
        }
        unsigned char *Ah = At + h * (kM2 * 128) + lane_off;
#pragma unroll
        for (int k = 0; k < kL1ColsPerWarp; ++k) {
          const int m = warp + kL1Conv * k;
          if (2 * lane + 64 * h < p.Jp) {
            const int f1022 = fx[k] + 1022;
            float d0[4], d1[4];
            digits28(cb[k].x, f1022, d0);
            digits28(cb[k].y, f1022, d1);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              *reinterpret_cast<uint32_t *>(Ah + q * a_tile + m * 128) = bf16_pack(d0[q], d1[q]);
          }
          // refill: the next half of this column, or the first half of the
          // column this slot takes in the next tile (with its exponent)
          if (h + 1 < P) {
            load_half(cur, k, h + 1, cb[k]);
          } else {
            load_half(nxt, k, 0, cb[k]);
            fx[k] = load_exp(nxt, k);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&part_full[h]));
      }
      cur = nxt;
    }
  } else if (warp < kL1Conv + kL1Drain) {
    // ---------------- drain ----------------
    const int dw = warp - kL1Conv;
    const int q = warp & 3;           // the TMEM lane quarter this warp may read
    const int half = dw >> 2;         // which half of the r range
    const int m = 32 * q + lane;      // this thread's column of the tile
    const int rh = p.Rp / 2;          // a multiple of 8
    const bool vec = (p.R % 2) == 0 && (reinterpret_cast<uintptr_t>(z) & 15) == 0;
    auto col_of = [&](int it) { return (t0 + (int64_t)it * tstride) * kM2 + m; };
    int fnext = (ntc > 0 && col_of(0) < p.K) ? __ldg(colexp + col_of(0)) : 0;
    for (int it = 0; it < ntc; ++it) {
      const int set = it & 1;
      int w = 0;
      if (lane == 0) w = role_wait(smem_addr(&acc_full[set]), (uint32_t)((it >> 1) & 1), &stop);
      if (!__shfl_sync(0xffffffffu, w, 0)) break;
      fence_after();
      const int64_t c = col_of(it);
      const bool valid = c < p.K;
      const int fcol = fnext;
      fnext = (it + 1 < ntc && col_of(it + 1) < p.K) ? __ldg(colexp + col_of(it + 1)) : 0;
      double *zc = z + c * (int64_t)p.R;
      const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(set * 4 * p.Rp);
      for (int r0 = half * rh; r0 < (half + 1) * rh; r0 += 4) {
        uint32_t a[4][4];
#pragma unroll
        for (int lev = 0; lev < 4; ++lev)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(a[lev][0]), "=r"(a[lev][1]), "=r"(a[lev][2]), "=r"(a[lev][3])
                       : "r"(tb + (uint32_t)(lev * p.Rp + r0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid && r0 < p.R) {
          double o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            o[e] = levels_to_double<true>(a[0][e], a[1][e], a[2][e], a[3][e], rowexp[r0 + e] + fcol - 42);
          if (vec) {  // R even: (r0, r0 + 1) and (r0 + 2, r0 + 3) are whole pairs or past R
            *reinterpret_cast<double2 *>(zc + r0) = make_double2(o[0], o[1]);
            if (r0 + 2 < p.R) *reinterpret_cast<double2 *>(zc + r0 + 2) = make_double2(o[2], o[3]);
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (r0 + e < p.R) zc[r0 + e] = o[e];
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&acc_free[set]));  // this warp's reads of the set are complete
    }
  } else if (lane == 0) {
    // ---------------- MMA issue ----------------
    const uint32_t ab = smem_addr(At), ub = smem_addr(Ut);
    const int nks = p.Jp / 16;
    int last_h = -1, last_par = 0;  // the last commit of part_free: no MMA of ours runs past it
    for (int it = 0; it < ntc; ++it) {
      const int set = it & 1;
      if (it >= 2 && !role_wait(smem_addr(&acc_free[set]), (uint32_t)(((it - 2) >> 1) & 1), &stop)) break;
      // U's four digit tiles are stacked rows of one K-major operand (U1 first),
      // so the MMA of Y's digit q against its first (4 - q) Rp rows, written
      // at column q Rp of the set, adds Y_q U_a into level q + a for every
      // a <= 3 - q at once: 4 MMAs per k-step carry the 10 digit products.
      const uint32_t d0 = tmem + (uint32_t)(set * 4 * p.Rp);
      bool ok = true;
#pragma unroll
      for (int h = 0; h < P; ++h) {
        if (!role_wait(smem_addr(&part_full[h]), (uint32_t)(it & 1), &stop)) {
          ok = false;
          break;
        }
        fence_after();
        for (int ks = 4 * h; ks < nks && ks < 4 * h + 4; ++ks) {
          const uint32_t koff = (uint32_t)(h * (kM2 * 128) + (ks & 3) * 32);
          const uint64_t ucat = smem_desc(ub + 256 * ks, 128, sbo_u);
#pragma unroll
          for (int q = 0; q < kBTiles; ++q) {
            const uint64_t ya = smem_desc_sw128(ab + q * a_tile + koff, 1024);
            // levels q..3 start accumulating at the first k-step of digit q = 0;
            // later digits add into levels the q = 0 MMA has already initialised
            mma_bf16(d0 + q * p.Rp, ya, ucat, idesc_q[q], (ks == 0 && q == 0) ? 0u : 1u);
          }
        }
        mma_commit(smem_addr(&part_free[h]));
        last_h = h;
        last_par = it & 1;
      }
      if (!ok) break;
      mma_commit(smem_addr(&acc_full[set]));
    }
    // no MMA of ours may still run when TMEM is released (a commit tracks all
    // earlier MMAs of this thread)
    if (last_h >= 0) mbar_wait(smem_addr(&part_free[last_h]), (uint32_t)last_par);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
  if (stop && tid == 0) atomicExch(err, 1);
}

// The plan, or parts == 0 when the shape does not suit this kernel.
TtmL1Plan ttm_l1_plan(int64_t J, int64_t B, int64_t R, const void *y, tucker_dtype dt, const DeviceInfo &dev) {
  TtmL1Plan p{};
  p.J = (int)J;
  p.Jp = (int)((J + 15) / 16 * 16);
  p.R = (int)R;
  p.Rp = (int)((R + 15) / 16 * 16);
  p.parts = (p.Jp + 63) / 64;
  const int cols = 2 * 4 * p.Rp;  // two accumulator sets of four levels
  p.tmem_cols = 32;
  while (p.tmem_cols < cols) p.tmem_cols <<= 1;
  p.K = B;
  p.ntiles = (p.K + kM2 - 1) / kM2;
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(dev.sms, p.ntiles));
  p.a_bytes = (size_t)4 * p.parts * kM2 * 128;
  p.u_bytes = (size_t)4 * p.Rp * p.Jp * 2;
  p.smem = 1024 + p.a_bytes + p.u_bytes;
  const size_t elem = dt == TUCKER_F64 ? 8 : 4;
  const bool ok = J % 2 == 0 && J <= kMaxJp && cols <= 512 && reinterpret_cast<uintptr_t>(y) % (2 * elem) == 0 &&
                  p.smem + 4096 <= (size_t)dev.smem_optin;
  if (!ok) p.parts = 0;
  return p;
}

// ---------------------------------------------------------------------------
// L > 1 through tensor-map tiles.  The unfolding's column (l, b) is J entries
// L apart; a tile is 128 consecutive l of one b (L >= 128) or floor(128 / L)
// whole runs of L (L < 128), i.e. one box {BL, 32, BB} of the 3-D tensor
// map over Y (L, J, B) per K-part of 32 rows (j), copied by the
// tensor-memory accelerator into a ring of shared-memory slots (rows j >= J
// and columns past L or B arrive as zeros).  The column exponents come from
// the exponent pass over the same Y (every column's largest magnitude over
// all J rows), so a part can be converted as soon as it lands.  The warps
// have fixed roles and meet only at mbarriers (as in the L == 1 kernel):
//   16 converter warps: thread (column m, rows 8 (tid / 128) ..) reads its
//      8 entries of a part with constant offsets, forms the four 28-bit
//      digits and stores one 16-byte K-major row unit per digit tile into
//      one of two operand stages (a_full: stage written and slot read);
//   1 control thread issues the copies (a slot is refilled as soon as the
//      converters have read it) and, per part, four MMAs per K-step against
//      U's stacked digit tiles into one of two TMEM accumulator sets
//      (mma_done: stage free; acc_full: a tile's levels complete);
//   8 drain warps assemble each output exactly from the four levels and
//      write it (coalesced runs of l) while the next tile's MMAs run
//      (acc_free: set read out).
// Every wait is bounded and gives up once another role has flagged an error.
// ---------------------------------------------------------------------------
constexpr int kTmKH = 32;  // contraction rows per part (one box)

struct TtmTmaPlan {
  int J, Jp32, R, Rp, parts, BL, BB, slots, tmem_cols, grid;
  int64_t L, B, tiles_per_b, ntiles;
  size_t u_bytes, raw_slot, smem;
};

constexpr int kTmConv = 16;                                // converter warps
constexpr int kTmDrain = 8;                                // drain warps (two per TMEM lane quarter)
constexpr int kTmThreads = (kTmConv + kTmDrain + 1) * 32;  // and the control warp

template <typename T>
__global__ void __launch_bounds__(kTmThreads, 1) k_ttm_split_tma(const __grid_constant__ CUtensorMap ymap,
                                                                 const double *__restrict__ U, TtmTmaPlan p,
                                                                 const int *__restrict__ colexp,
                                                                 double *__restrict__ z, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long raw_full[4], a_full[2], mma_done[2], acc_full[2], acc_free[2];
  __shared__ int rowexp[kM];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int stop;
  __shared__ int drain_go;
  unsigned char *base = dsmem + ((1024u - (smem_addr(dsmem) & 1023u)) & 1023u);
  unsigned char *Ut = base;                                 // 4 stacked digit tiles of U (Rp x Jp32)
  unsigned char *Ast = Ut + p.u_bytes;                      // 2 stages x 4 digit tiles (128 x 32)
  constexpr int kATile = kM2 * kTmKH * 2;                   // 8 KB
  unsigned char *ring = Ast + 2 * 4 * kATile;               // p.slots raw slots
  const int u_tile = p.Rp * p.Jp32 * 2;
  const uint32_t sbo_u = (uint32_t)(p.Jp32 / 8) * 128u;
  constexpr uint32_t kSboA = (kTmKH / 8) * 128u;            // 512
  uint32_t idesc_q[kBTiles];
#pragma unroll
  for (int q = 0; q < kBTiles; ++q) idesc_q[q] = idesc_bf16(kM2, (kBTiles - q) * p.Rp);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int k = 0; k < p.slots; ++k) mbar_init(smem_addr(&raw_full[k]), 1);
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_addr(&a_full[k]), kTmConv);
      mbar_init(smem_addr(&mma_done[k]), 1);
      mbar_init(smem_addr(&acc_full[k]), 1);
      mbar_init(smem_addr(&acc_free[k]), kTmDrain);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
  }
  if (tid < kM) {
    unsigned long long m = 0ull;
    if (tid < p.R)
      for (int j = 0; j < p.J; ++j) m = max(m, mag_bits(U[j + (int64_t)p.J * tid]));
    rowexp[tid] = exp_above(m, true);
  }
  __syncthreads();
  for (int u = tid; u < p.Rp * (p.Jp32 / 8); u += kTmThreads) {  // U's digit tiles (row r, k = j)
    const int r = u / (p.Jp32 / 8), jg = u % (p.Jp32 / 8);
    uint32_t w[kATiles][4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      int d[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 8 * jg + k + h;
        const double v = (r < p.R && j < p.J) ? U[j + (int64_t)p.J * r] : 0.0;
        digits4(scaled_int28(v, rowexp[r]), d[h]);
      }
#pragma unroll
      for (int t = 0; t < kATiles; ++t) w[t][k >> 1] = bf16_pair((float)d[0][t], (float)d[1][t]);
    }
    const int off = (r >> 3) * (int)sbo_u + jg * 128 + (r & 7) * 16;
#pragma unroll
    for (int t = 0; t < kATiles; ++t)
      *reinterpret_cast<uint4 *>(Ut + t * u_tile + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }

  const int64_t t0 = blockIdx.x, tstride = gridDim.x;
  const int ntc = t0 < p.ntiles ? (int)((p.ntiles - t0 + tstride - 1) / tstride) : 0;
  const int nunits = ntc * p.parts;
  // tile it's box origin: (l0, b0)
  auto tile_origin = [&](int it, int64_t &l0, int64_t &b0) {
    const int64_t tg = t0 + (int64_t)it * tstride;
    if (p.BB == 1) {
      b0 = tg / p.tiles_per_b;
      l0 = (tg - b0 * p.tiles_per_b) * kM2;
    } else {
      b0 = tg * p.BB;
      l0 = 0;
    }
  };
  // the column exponent of the tile row at box position (s, lo), i.e. row
  // s BL + lo (-4000 past the tile's columns: such a column converts to
  // zeros and is not written)
  auto col_exp = [&](int it, int s, int lo) -> int {
    int64_t l0, b0;
    tile_origin(it, l0, b0);
    const int64_t l = l0 + lo, b = b0 + s;
    return (s < p.BB && l < p.L && b < p.B) ? colexp[l + p.L * b] : -4000;
  };
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp < kTmConv) {
    // ---------------- converters: thread (column m, rows 8 jq ..) of each part ----------------
    const int m = tid & (kM2 - 1), jq = tid >> 7;
    const int s_m = m / p.BL, loff = m - s_m * p.BL;
    const bool m_in_box = s_m < p.BB;
    const int raw_off = (s_m * kTmKH + 8 * jq) * p.BL + loff;  // element (m, 8 jq) of a slot
    const int off = (m >> 3) * (int)kSboA + jq * 128 + (m & 7) * 16;
    int f1022 = 0;
    // unit u is part pp of tile it in ring slot `slot` (its phase slot_par):
    // counters, not divisions, on this per-unit path
    int it = 0, pp = 0, slot = 0;
    uint32_t slot_par = 0;
    for (int u = 0; u < nunits; ++u) {
      const int stg = u & 1;
      if (pp == 0) f1022 = col_exp(it, s_m, loff) + 1022;
      int ok = 1;
      if (lane == 0) {
        ok = role_wait(smem_addr(&raw_full[slot]), slot_par, &stop);
        if (ok && u >= 2) ok = role_wait(smem_addr(&mma_done[stg]), (uint32_t)(((u - 2) >> 1) & 1), &stop);
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      const T *raw = reinterpret_cast<const T *>(ring + (size_t)slot * p.raw_slot) + raw_off;
      uint32_t w[kBTiles][4];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        float d0[4], d1[4];
        const T y0 = m_in_box ? raw[k * p.BL] : T(0), y1 = m_in_box ? raw[(k + 1) * p.BL] : T(0);
        digits28(y0, f1022, d0);
        digits28(y1, f1022, d1);
#pragma unroll
        for (int qq = 0; qq < kBTiles; ++qq) w[qq][k >> 1] = bf16_pair(d0[qq], d1[qq]);
      }
      unsigned char *st = Ast + stg * 4 * kATile;
#pragma unroll
      for (int qq = 0; qq < kBTiles; ++qq)
        *reinterpret_cast<uint4 *>(st + qq * kATile + off) = make_uint4(w[qq][0], w[qq][1], w[qq][2], w[qq][3]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&a_full[stg]));  // this warp has read slot u and written stage stg
      if (++pp == p.parts) {
        pp = 0;
        ++it;
      }
      if (++slot == p.slots) {
        slot = 0;
        slot_par ^= 1u;
      }
    }
  } else if (warp < kTmConv + kTmDrain) {
    // ---------------- drain: TMEM lanes 32 q.. (columns), half of the rows ----------------
    const int dw = warp - kTmConv, q = warp & 3, half = dw >> 2;
    const int mm = 32 * q + lane;
    const int sm2 = mm / p.BL, lo2 = mm - sm2 * p.BL;
    const int rh = p.Rp / 2;  // a multiple of 8
    for (int it = 0; it < ntc; ++it) {
      const int set = it & 1;
      if (dw == 0 && lane == 0) drain_go = role_wait(smem_addr(&acc_full[set]), (uint32_t)((it >> 1) & 1), &stop);
      asm volatile("bar.sync 1, %0;" ::"n"(kTmDrain * 32) : "memory");
      if (!drain_go) break;
      fence_after();
      int64_t l0, b0;
      tile_origin(it, l0, b0);
      const int64_t l = l0 + lo2, b = b0 + sm2;
      const bool valid = sm2 < p.BB && l < p.L && b < p.B;
      const int fc = valid ? colexp[l + p.L * b] : 0;
      double *zc = z + l + p.L * (int64_t)p.R * b;
      const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(set * 4 * p.Rp);
      for (int r0 = half * rh; r0 < (half + 1) * rh; r0 += 4) {
        uint32_t a[4][4];
#pragma unroll
        for (int lev = 0; lev < 4; ++lev)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(a[lev][0]), "=r"(a[lev][1]), "=r"(a[lev][2]), "=r"(a[lev][3])
                       : "r"(tb + (uint32_t)(lev * p.Rp + r0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int r = r0 + e;
            if (r < p.R) zc[p.L * (int64_t)r] = levels_to_double<false>(a[0][e], a[1][e], a[2][e], a[3][e], rowexp[r] + fc - 42);
          }
        }
      }
      fence_before();
      asm volatile("bar.sync 1, %0;" ::"n"(kTmDrain * 32) : "memory");
      if (lane == 0) mbar_arrive(smem_addr(&acc_free[set]));  // this warp's reads of the set are complete
    }
  } else if (lane == 0) {
    // ---------------- control: copies and MMAs ----------------
    // copy number `issued` is part c_pp of tile c_it into slot c_slot
    int c_it = 0, c_pp = 0, c_slot = 0;
    int64_t c_l0 = 0, c_b0 = 0;
    tile_origin(0, c_l0, c_b0);
    auto issue_copy = [&]() {
      const uint32_t bar = smem_addr(&raw_full[c_slot]);
      mbar_expect_tx(bar, (uint32_t)p.raw_slot);
      tma_load_3d(smem_addr(ring + (size_t)c_slot * p.raw_slot), &ymap, (int)c_l0, kTmKH * c_pp, (int)c_b0, bar);
      if (++c_pp == p.parts) {
        c_pp = 0;
        tile_origin(++c_it, c_l0, c_b0);
      }
      if (++c_slot == p.slots) c_slot = 0;
    };
    int issued = 0, last = -1;
    for (; issued < p.slots && issued < nunits; ++issued) issue_copy();
    const uint32_t ub = smem_addr(Ut);
    int it = 0, pp = 0;  // unit u is part pp of tile it
    for (int u = 0; u < nunits; ++u, ++pp) {
      if (pp == p.parts) {
        pp = 0;
        ++it;
      }
      const int stg = u & 1, set = it & 1;
      if (!role_wait(smem_addr(&a_full[stg]), (uint32_t)((u >> 1) & 1), &stop)) break;
      if (issued < nunits) {  // slot u % slots has been read by every converter
        issue_copy();
        ++issued;
      }
      if (pp == 0 && it >= 2 && !role_wait(smem_addr(&acc_free[set]), (uint32_t)(((it - 2) >> 1) & 1), &stop)) break;
      fence_after();
      const uint32_t ab = smem_addr(Ast + stg * 4 * kATile);
      const uint32_t d0 = tmem + (uint32_t)(set * 4 * p.Rp);
#pragma unroll
      for (int ks = 0; ks < kTmKH / 16; ++ks) {
        const uint64_t ucat = smem_desc(ub + (uint32_t)(((kTmKH / 8) * pp + 2 * ks) * 128), 128, sbo_u);
#pragma unroll
        for (int qq = 0; qq < kBTiles; ++qq) {
          const uint64_t ya = smem_desc(ab + qq * kATile + 256 * ks, 128, kSboA);
          mma_bf16(d0 + qq * p.Rp, ya, ucat, idesc_q[qq], (pp == 0 && ks == 0 && qq == 0) ? 0u : 1u);
        }
      }
      mma_commit(smem_addr(&mma_done[stg]));
      if (pp == p.parts - 1) mma_commit(smem_addr(&acc_full[set]));
      last = u;
    }
    // no MMA or copy of ours may still run when TMEM and shared memory go
    if (last >= 0) mbar_wait(smem_addr(&mma_done[last & 1]), (uint32_t)((last >> 1) & 1));
    for (int c = max(0, issued - p.slots); c < issued; ++c)
      mbar_wait(smem_addr(&raw_full[c % p.slots]), (uint32_t)((c / p.slots) & 1));
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
  if (stop && tid == 0) atomicExch(err, 1);
}

// column exponents of Y (L, J, B) for the tensor-map kernel when no exponent
// pass has run: thread per column (consecutive l: coalesced)
template <typename T>
__global__ void __launch_bounds__(256) k_colexp(const T *__restrict__ y, int64_t L, int J, int64_t K,
                                                int *__restrict__ colexp) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= K) return;
  const int64_t b = c / L, l = c - b * L;
  const T *p = y + l + L * (int64_t)J * b;
  unsigned mx = 0u;
  for (int j = 0; j < J; ++j) mx = max(mx, hi_mag(__ldg(p + L * (int64_t)j)));
  colexp[c] = exp_above(mag_pattern(mx, sizeof(T) == 8), sizeof(T) == 8);
}


// column exponents of contiguous columns (L == 1) when no exponent pass has
// run: a warp per column, its lanes over the column's entries (coalesced)
template <typename T>
__global__ void __launch_bounds__(256) k_colexp_l1(const T *__restrict__ y, int J, int64_t B,
                                                   int *__restrict__ colexp) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < B; c += nw) {
    unsigned mx = 0u;
    for (int j = lane; j < J; j += 32) mx = max(mx, hi_mag(__ldg(y + c * (int64_t)J + j)));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) colexp[c] = exp_above(mag_pattern(mx, sizeof(T) == 8), sizeof(T) == 8);
  }
}

template <typename T>
int run_ttm_l1(const void *y, const double *U, const int *d_colexp, const TtmL1Plan &q, double *z, int *d_err,
               cudaStream_t s) {
  if (q.parts == 1) {
    TK_CUDA(allow_max_smem(k_ttm_split_l1<T, 1>));
    k_ttm_split_l1<T, 1><<<q.grid, kL1Threads, q.smem, s>>>(static_cast<const T *>(y), U, d_colexp, q, z, d_err);
  } else {
    TK_CUDA(allow_max_smem(k_ttm_split_l1<T, 2>));
    k_ttm_split_l1<T, 2><<<q.grid, kL1Threads, q.smem, s>>>(static_cast<const T *>(y), U, d_colexp, q, z, d_err);
  }
  TK_LAUNCHED();
  return TUCKER_OK;
}

// The plan, or parts == 0 when the shape does not suit the tensor-map kernel.
TtmTmaPlan ttm_tma_plan(int64_t L, int64_t J, int64_t B, int64_t R, tucker_dtype dt, const void *y,
                        const DeviceInfo &dev) {
  TtmTmaPlan p{};
  const size_t esz = dt == TUCKER_F64 ? 8 : 4;
  p.J = (int)J;
  p.R = (int)R;
  p.Rp = (int)((R + 15) / 16 * 16);
  p.Jp32 = (int)((J + 31) / 32 * 32);
  p.parts = p.Jp32 / kTmKH;
  p.L = L;
  p.B = B;
  if (L >= kM2) {
    p.BL = kM2;
    p.BB = 1;
    p.tiles_per_b = (L + kM2 - 1) / kM2;
    p.ntiles = B * p.tiles_per_b;
  } else {
    p.BL = (int)L;
    p.BB = (int)(kM2 / L);
    p.tiles_per_b = 1;
    p.ntiles = (B + p.BB - 1) / p.BB;
  }
  p.raw_slot = (size_t)p.BL * kTmKH * p.BB * esz;
  p.u_bytes = (size_t)4 * p.Rp * p.Jp32 * 2;
  const int cols = 2 * 4 * p.Rp;
  p.tmem_cols = 32;
  while (p.tmem_cols < cols) p.tmem_cols <<= 1;
  const size_t fixed = 1024 + p.u_bytes + (size_t)2 * 4 * kM2 * kTmKH * 2;
  const size_t avail = (size_t)dev.smem_optin > fixed + 4096 ? (size_t)dev.smem_optin - fixed - 4096 : 0;
  p.slots = (int)std::min<size_t>(4, avail / std::max<size_t>(p.raw_slot, 1));
  p.smem = fixed + (size_t)p.slots * p.raw_slot;
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(dev.sms, p.ntiles));
  const bool ok = L > 1 && J <= kMaxJp && R <= 64 && R <= J && (L * (int64_t)esz) % 16 == 0 &&
                  reinterpret_cast<uintptr_t>(y) % 16 == 0 && cols <= 512 && p.slots >= 2 && L < (1ll << 31) &&
                  B < (1ll << 31) && p.ntiles >= 1;
  if (!ok) p.parts = 0;
  return p;
}

bool ttm_tma_map(CUtensorMap *map, const void *y, int64_t L, int64_t J, int64_t B, const TtmTmaPlan &p, bool f64) {
  const size_t esz = f64 ? 8 : 4;
  const uint64_t dims[3] = {(uint64_t)L, (uint64_t)J, (uint64_t)B};
  const uint64_t strides[2] = {(uint64_t)L * esz, (uint64_t)L * J * esz};
  const uint32_t box[3] = {(uint32_t)p.BL, (uint32_t)kTmKH, (uint32_t)p.BB};
  return encode_tmap(map, f64, y, 3, dims, strides, box);
}

template <typename T>
int run_ttm_tma(const CUtensorMap &map, const void *y, int64_t L, int64_t J, int64_t B, const double *U,
                const TtmTmaPlan &p, const int *d_colexp, double *z, int *d_err, cudaStream_t s) {
  const int64_t K = L * B;
  int *tmp = nullptr;
  if (!d_colexp) {  // no exponent pass ran: the column exponents first
    TK_CUDA(cudaMallocAsync(&tmp, sizeof(int) * (size_t)K, s));
    k_colexp<T><<<(unsigned)((K + 255) / 256), 256, 0, s>>>(static_cast<const T *>(y), L, (int)J, K, tmp);
    TK_LAUNCHED();
    d_colexp = tmp;
  }
  TK_CUDA(allow_max_smem(k_ttm_split_tma<T>));
  k_ttm_split_tma<T><<<p.grid, kTmThreads, p.smem, s>>>(map, U, p, d_colexp, z, d_err);
  TK_LAUNCHED();
  if (tmp) TK_CUDA(cudaFreeAsync(tmp, s));
  return TUCKER_OK;
}

}  // namespace

int launch_ttm_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *U, int64_t R,
                     double *z, int *d_err, const DeviceInfo &dev, cudaStream_t s, Prof *prof,
                     const int *d_colexp) {
  if (J > kMaxSplitJ || R > kM || R > J) {
    set_error("split-precision TTM supports R <= J <= %d and R <= %d (got J = %lld, R = %lld)", kMaxSplitJ, kM,
              (long long)J, (long long)R);
    return TUCKER_EUNSUPPORTED;
  }
  const double flops = 2.0 * J * R * (double)(L * B);
  const double bytes = (double)(L * B) * (J * (dt == TUCKER_F64 ? 8.0 : 4.0) + R * 8.0) + J * R * 8.0;
  if (J > kMaxJp) {
    // Z = sum over parts of 128 rows of Y_part x_n U_part^T: each part is the
    // register-staged product (its columns scaled by their own part's
    // exponents), the later ones added to Z in float64
    if (prof) prof->begin(L == 1 ? TUCKER_PHASE_TTM_L1 : TUCKER_PHASE_TTM);
    const size_t es = dt == TUCKER_F64 ? 8 : 4;
    int launches = 0;
    for (int64_t j0 = 0; j0 < J; j0 += kMaxJp) {
      TtmSplit2Plan p = ttm_split2_plan(L, std::min<int64_t>(kMaxJp, J - j0), B, R, dev);
      p.ldj = J;
      p.ldu = J;
      p.accum = j0 > 0;
      const void *yp = static_cast<const char *>(y) + (size_t)(L * j0) * es;
      if (dt == TUCKER_F64) {
        TK_CUDA(allow_max_smem(k_ttm_split2<double>));
        k_ttm_split2<double><<<p.grid, kThreads, p.smem, s>>>(static_cast<const double *>(yp), L, B, U + j0, p, z,
                                                              d_err);
      } else {
        TK_CUDA(allow_max_smem(k_ttm_split2<float>));
        k_ttm_split2<float><<<p.grid, kThreads, p.smem, s>>>(static_cast<const float *>(yp), L, B, U + j0, p, z,
                                                             d_err);
      }
      TK_LAUNCHED();
      ++launches;
    }
    if (prof) prof->end(flops, bytes, launches);
    return TUCKER_OK;
  }
  if (L == 1) {
    const TtmL1Plan q = ttm_l1_plan(J, B, R, y, dt, dev);
    if (q.parts > 0) {
      if (prof) prof->begin(TUCKER_PHASE_TTM_L1);
      int *tmp = nullptr;
      int launches = 1;
      if (!d_colexp) {  // no exponent pass ran: the column exponents first
        TK_CUDA(cudaMallocAsync(&tmp, sizeof(int) * (size_t)B, s));
        const unsigned blocks = (unsigned)std::min<int64_t>((B + 7) / 8, (int64_t)dev.sms * 16);
        if (dt == TUCKER_F64)
          k_colexp_l1<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(y), (int)J, B, tmp);
        else
          k_colexp_l1<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(y), (int)J, B, tmp);
        TK_LAUNCHED();
        d_colexp = tmp;
        ++launches;
      }
      if (dt == TUCKER_F64) TK_CHECK(run_ttm_l1<double>(y, U, d_colexp, q, z, d_err, s));
      else TK_CHECK(run_ttm_l1<float>(y, U, d_colexp, q, z, d_err, s));
      if (tmp) TK_CUDA(cudaFreeAsync(tmp, s));
      if (prof) prof->end(flops, bytes, launches);
      return TUCKER_OK;
    }
  }
  if (L > 1) {
    static const bool legacy = [] {  // TUCKER_TTM_SPLIT_KERNEL=regs: the register-staged kernel
      const char *e = std::getenv("TUCKER_TTM_SPLIT_KERNEL");
      return e && std::strcmp(e, "regs") == 0;
    }();
    const TtmTmaPlan q = ttm_tma_plan(L, J, B, R, dt, y, dev);
    CUtensorMap map;
    if (q.parts > 0 && !legacy && ttm_tma_map(&map, y, L, J, B, q, dt == TUCKER_F64)) {
      if (prof) prof->begin(TUCKER_PHASE_TTM);
      if (dt == TUCKER_F64) TK_CHECK(run_ttm_tma<double>(map, y, L, J, B, U, q, d_colexp, z, d_err, s));
      else TK_CHECK(run_ttm_tma<float>(map, y, L, J, B, U, q, d_colexp, z, d_err, s));
      if (prof) prof->end(flops, bytes, 1);
      return TUCKER_OK;
    }
  }
  const TtmSplit2Plan p = ttm_split2_plan(L, J, B, R, dev);
  if (prof) prof->begin(TUCKER_PHASE_TTM);
  if (dt == TUCKER_F64) {
    TK_CUDA(allow_max_smem(k_ttm_split2<double>));
    k_ttm_split2<double><<<p.grid, kThreads, p.smem, s>>>(static_cast<const double *>(y), L, B, U, p, z, d_err);
  } else {
    TK_CUDA(allow_max_smem(k_ttm_split2<float>));
    k_ttm_split2<float><<<p.grid, kThreads, p.smem, s>>>(static_cast<const float *>(y), L, B, U, p, z, d_err);
  }
  TK_LAUNCHED();
  if (prof) prof->end(flops, bytes, 1);
  return TUCKER_OK;
}

}  // namespace tk
