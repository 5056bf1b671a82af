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
//     balanced digits v = s1 2^21 + s2 2^14 + s3 2^7 + s4 (|s1| <= 128,
//     |s2..s4| <= 64), exact in BF16.  The TTM output feeds every later mode
//     and the core, so it keeps 28 bits (21 were measurably too few).
//   * D = U_a Y_b^T products of levels a + b = 2..5 go to four exact TMEM
//     accumulators:
//       acc0 = U1 Y1^T,  acc1 = U1 Y2^T + U2 Y1^T,
//       acc2 = U1 Y3^T + U2 Y2^T + U3 Y1^T,
//       acc3 = U1 Y4^T + U2 Y3^T + U3 Y2^T + U4 Y1^T.
//     With J <= 128 every level stays below 2^22 (acc3 <= 128 (2 2^13 + 2 2^12)),
//     so all four are exact integers.  Levels 6..8 (products of two low
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
#include <type_traits>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tk {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kM = 128;           // output rows r (R zero-padded)
constexpr int kMaxJp = 128;       // contraction length, padded to a multiple of 16
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
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_ttm_split2(const T *__restrict__ y, int64_t L, int64_t B,
                                                            const double *__restrict__ U, TtmSplit2Plan p,
                                                            double *__restrict__ z, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long mbar[2];   // operand stages
  __shared__ __align__(8) unsigned long long tbar[2];   // accumulator sets (tile done)
  __shared__ unsigned long long colmax[kM2];
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
      for (int j = 0; j < p.J; ++j) m = max(m, mag_bits(U[j + (int64_t)p.J * tid]));
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
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const int64_t in_b = L * (int64_t)p.J, out_b = L * (int64_t)p.R;
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
            const long long v = ((long long)__float2int_rn(__uint_as_float(a[0][e])) << 28) +
                                ((long long)__float2int_rn(__uint_as_float(a[1][e])) << 21) +
                                ((long long)__float2int_rn(__uint_as_float(a[2][e])) << 14) +
                                ((long long)__float2int_rn(__uint_as_float(a[3][e])) << 7);
            z[ob + L * (int64_t)r] = scaled_ll_to_double(v, rowexp[r] + colexp[set][c] - 42);
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
    if (tid < kM2) colmax[tid] = 0ull;
    __syncthreads();
    {
      unsigned long long m = 0ull;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int e = 0; e < 8; ++e) m = max(m, mag_bits(raw[k][e]));
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
    if (tid < kM2) colexp[set][tid] = exp_above(colmax[tid], kF64);
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
          int d[2][4];
          digits4(scaled_int28(raw[k][e], e_col), d[0]);
          digits4(scaled_int28(raw[k][e + 1], e_col), d[1]);
#pragma unroll
          for (int q = 0; q < kBTiles; ++q) w[q][e >> 1] = bf16_pair((float)d[0][q], (float)d[1][q]);
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
  return p;
}

// ---------------------------------------------------------------------------
// L == 1 (the first mode of the natural layout): column c of the unfolding
// is the contiguous vector y[c J .. c J + J - 1].  A warp takes whole columns,
// its lanes reading consecutive 16-byte pairs (fully coalesced), finds the
// column exponent with a warp reduction, and writes each digit row into a
// 128-byte swizzled K-major tile (one row per store instruction, no bank
// conflicts).  Each warp keeps four columns in flight in registers.  Two TMEM
// accumulator sets (R <= 64) let a tile's MMAs run while the previous tile
// drains; the drain stages the outputs of a
// tile (R contiguous doubles per column, so the tile's output is one
// contiguous block) in shared memory and writes them out row by row.
// ---------------------------------------------------------------------------
struct TtmL1Plan {
  int J, Jp, R, Rp, parts, Rs, tmem_cols;
  int64_t K, ntiles;
  int grid;
  size_t u_bytes, a_bytes, stg_bytes, smem;
};

constexpr int kL1ColsPerWarp = kM2 / (kThreads / 32);  // 8
constexpr int kL1Depth = 4;                             // columns in flight per warp

// round(|y| 2^(28 - f)) with the sign of y, from the bits in 32-bit integer
// arithmetic (ties away from zero); f1022 = f + 1022 and |y| < 2^f.  With m29
// the leading 29 bits of the significand, v = (m29 + 2^sh) >> (sh + 1) for
// sh = f + 1022 - exponent field; the lower bits cannot change the result.
__device__ __forceinline__ int scaled_int28_bits(double y, int f1022) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const unsigned m29 = (((hi & 0xFFFFFu) | 0x100000u) << 8) | (lo >> 24);
  const int sh = max(min(f1022 - ex, 30), 0);
  unsigned v = (m29 + (1u << sh)) >> (sh + 1);
  v = ex ? v : 0u;
  const int sgn = (int)hi >> 31;
  return ((int)v ^ sgn) - sgn;
}
__device__ __forceinline__ int scaled_int28_bits(float y, int f1022) {
  return scaled_int28(y, f1022 - 1022);
}

// the four balanced digits of v (|v| <= 2^28) as exact floats
__device__ __forceinline__ void digits4_float(int v, float (&d)[4]) {
  const int h = (v + 64) >> 7;  // |h| <= 2^21
  d[3] = small_int_float(v - (h << 7));
  const float hf = small_int_float(h);
  d[0] = round_float(hf * 0x1p-14f);
  const float r = __fmaf_rn(d[0], -16384.0f, hf);
  d[1] = round_float(r * 0x1p-7f);
  d[2] = __fmaf_rn(d[1], -128.0f, r);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_ttm_split_l1(const T *__restrict__ y, const double *__restrict__ U,
                                                              TtmL1Plan p, double *__restrict__ z,
                                                              int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long done_bar;  // a tile's MMAs have completed
  __shared__ int colexp[2][kM2];
  __shared__ int rowexp[kM];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  constexpr bool kF64 = sizeof(T) == 8;
  using V2 = typename std::conditional<kF64, double2, float2>::type;
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char *At = base;                                  // 4 digit tiles, SW128 K-major
  unsigned char *Ut = base + p.a_bytes;                      // 4 digit tiles, no swizzle
  double *stg = reinterpret_cast<double *>(Ut + p.u_bytes);  // 128 x Rs output staging
  const int a_tile = p.parts * kM2 * 128;
  const int u_tile = p.Rp * p.Jp * 2;
  const uint32_t sbo_u = (uint32_t)(p.Jp / 8) * 128u;
  const uint32_t idesc = idesc_bf16(kM2, p.Rp);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_addr(&done_bar), 1);
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
  for (int u = tid; u < p.Rp * (p.Jp / 8); u += kThreads) {
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
  // zero the A tiles once: K columns past J (up to the 64-wide part) stay zero
  for (int e = tid; e < (int)(p.a_bytes / 16); e += kThreads) reinterpret_cast<uint4 *>(At)[e] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  // column m of tile t, entries j = 2 lane + 64 h (h < 2) as two pairs
  auto load_col = [&](int64_t t, int m, V2 (&v)[2]) {
    const int64_t c = t * kM2 + m;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * lane + 64 * h;
      if (t < p.ntiles && c < p.K && j < p.J)
        v[h] = __ldg(reinterpret_cast<const V2 *>(y + c * (int64_t)p.J + j));
      else
        v[h].x = v[h].y = T(0);
    }
  };

  // drain tile t from accumulator set `set` into z
  auto drain = [&](int64_t t, int set) {
    fence_after();
    const int q = warp & 3, g = warp >> 2;
    const int m = 32 * q + lane;
    const int rq = p.Rp / 4;
    const int fcol = colexp[set][m];
    const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(set * 4 * p.Rp);
    for (int r0 = g * rq; r0 < (g + 1) * rq; r0 += 4) {
      uint32_t a[4][4];
#pragma unroll
      for (int lev = 0; lev < 4; ++lev)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(a[lev][0]), "=r"(a[lev][1]), "=r"(a[lev][2]), "=r"(a[lev][3])
                     : "r"(tb + (uint32_t)(lev * p.Rp + r0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + e;
        if (r < p.R) {
          const long long v = ((long long)__float2int_rn(__uint_as_float(a[0][e])) << 28) +
                              ((long long)__float2int_rn(__uint_as_float(a[1][e])) << 21) +
                              ((long long)__float2int_rn(__uint_as_float(a[2][e])) << 14) +
                              ((long long)__float2int_rn(__uint_as_float(a[3][e])) << 7);
          stg[m * p.Rs + r] = scaled_ll_to_double(v, rowexp[r] + fcol - 42);
        }
      }
    }
    fence_before();
    __syncthreads();
    // the tile's output is z[t 128 R ..]: rows of R contiguous doubles
    double *zt = z + t * kM2 * (int64_t)p.R;
    const int nvalid = (int)(p.K - t * kM2 < kM2 ? p.K - t * kM2 : kM2);
    for (int mm = warp; mm < nvalid; mm += kThreads / 32)
      for (int r = lane; r < p.R; r += 32) zt[(int64_t)mm * p.R + r] = stg[mm * p.Rs + r];
  };

  V2 cb[kL1Depth][2];
  const int64_t t0 = blockIdx.x;
#pragma unroll
  for (int k = 0; k < kL1Depth; ++k) load_col(t0, warp + 16 * k, cb[k]);
  int64_t prev_t = -1;
  int it = 0;
  for (int64_t t = t0; t < p.ntiles; t += gridDim.x, ++it) {
    const int set = it & 1;
    // the A tiles are free once the previous tile's MMAs have completed
    if (it >= 1 && tid == 0 && !mbar_wait(smem_addr(&done_bar), (it - 1) & 1)) stop = 1;
    __syncthreads();
    if (stop) break;
#pragma unroll
    for (int k = 0; k < kL1ColsPerWarp; ++k) {
      const int m = warp + 16 * k;
      V2 (&v)[2] = cb[k % kL1Depth];
      // column exponent: the largest magnitude over the column's J entries
      unsigned mx = max(max(hi_mag(v[0].x), hi_mag(v[0].y)), max(hi_mag(v[1].x), hi_mag(v[1].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int f = exp_above(kF64 ? (unsigned long long)mx << 32 : (unsigned long long)mx, kF64);
      if (lane == 0) colexp[set][m] = f;
      const int f1022 = f + 1022;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (2 * lane + 64 * h < p.Jp) {
          float d0[4], d1[4];
          digits4_float(scaled_int28_bits(v[h].x, f1022), d0);
          digits4_float(scaled_int28_bits(v[h].y, f1022), d1);
          const int off = h * (kM2 * 128) + m * 128 + (((lane >> 2) ^ (m & 7)) << 4) + (lane & 3) * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q) *reinterpret_cast<uint32_t *>(At + q * a_tile + off) = bf16_pair(d0[q], d1[q]);
        }
      }
      // refill: the column kL1Depth ahead (possibly of this CTA's next tile)
      const int kn = k + kL1Depth;
      if (kn < kL1ColsPerWarp) load_col(t, warp + 16 * kn, v);
      else load_col(t + gridDim.x, warp + 16 * (kn - kL1ColsPerWarp), v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t ab = smem_addr(At), ub = smem_addr(Ut);
      const uint32_t d0 = tmem + (uint32_t)(set * 4 * p.Rp);
      for (int ks = 0; ks < p.Jp / 16; ++ks) {
        const uint32_t acc = ks == 0 ? 0u : 1u;
        const uint32_t koff = (uint32_t)((ks >> 2) * (kM2 * 128) + (ks & 3) * 32);
        uint64_t ya[kBTiles], ub4[kATiles];
#pragma unroll
        for (int q = 0; q < kBTiles; ++q) ya[q] = smem_desc_sw128(ab + q * a_tile + koff, 1024);
#pragma unroll
        for (int q = 0; q < kATiles; ++q) ub4[q] = smem_desc(ub + q * u_tile + 256 * ks, 128, sbo_u);
        mma_bf16(d0 + 0 * p.Rp, ya[0], ub4[0], idesc, acc);
        mma_bf16(d0 + 1 * p.Rp, ya[0], ub4[1], idesc, acc);
        mma_bf16(d0 + 1 * p.Rp, ya[1], ub4[0], idesc, 1u);
        mma_bf16(d0 + 2 * p.Rp, ya[0], ub4[2], idesc, acc);
        mma_bf16(d0 + 2 * p.Rp, ya[1], ub4[1], idesc, 1u);
        mma_bf16(d0 + 2 * p.Rp, ya[2], ub4[0], idesc, 1u);
        mma_bf16(d0 + 3 * p.Rp, ya[0], ub4[3], idesc, acc);
        mma_bf16(d0 + 3 * p.Rp, ya[1], ub4[2], idesc, 1u);
        mma_bf16(d0 + 3 * p.Rp, ya[2], ub4[1], idesc, 1u);
        mma_bf16(d0 + 3 * p.Rp, ya[3], ub4[0], idesc, 1u);
      }
      mma_commit(smem_addr(&done_bar));
    }
    // drain the previous tile while the tensor cores work on this one
    if (prev_t >= 0) drain(prev_t, set ^ 1);
    prev_t = t;
  }
  // the last tile
  if (!stop && prev_t >= 0) {
    if (tid == 0 && !mbar_wait(smem_addr(&done_bar), (it - 1) & 1)) stop = 1;
    __syncthreads();
    if (!stop) drain(prev_t, (it - 1) & 1);
  } else if (stop && it >= 1 && tid == 0) {
    mbar_wait(smem_addr(&done_bar), (it - 1) & 1);  // let our own MMAs finish before TMEM is released
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
  p.Rs = p.R | 1;
  const int cols = 2 * 4 * p.Rp;  // two accumulator sets of four levels
  p.tmem_cols = 32;
  while (p.tmem_cols < cols) p.tmem_cols <<= 1;
  p.K = B;
  p.ntiles = (p.K + kM2 - 1) / kM2;
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(dev.sms, p.ntiles));
  p.a_bytes = (size_t)4 * p.parts * kM2 * 128;
  p.u_bytes = (size_t)4 * p.Rp * p.Jp * 2;
  p.stg_bytes = (size_t)kM2 * p.Rs * 8;
  p.smem = 1024 + p.a_bytes + p.u_bytes + p.stg_bytes;
  const size_t elem = dt == TUCKER_F64 ? 8 : 4;
  const bool ok = J % 2 == 0 && cols <= 512 && reinterpret_cast<uintptr_t>(y) % (2 * elem) == 0 &&
                  p.smem + 4096 <= (size_t)dev.smem_optin;
  if (!ok) p.parts = 0;
  return p;
}

}  // namespace

int launch_ttm_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *U, int64_t R,
                     double *z, int *d_err, const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (J > kMaxJp || R > kM || R > J) {
    set_error("split-precision TTM supports R <= J <= %d (got J = %lld, R = %lld)", kMaxJp, (long long)J,
              (long long)R);
    return TUCKER_EUNSUPPORTED;
  }
  const double flops = 2.0 * J * R * (double)(L * B);
  const double bytes = (double)(L * B) * (J * (dt == TUCKER_F64 ? 8.0 : 4.0) + R * 8.0) + J * R * 8.0;
  if (L == 1) {
    const TtmL1Plan q = ttm_l1_plan(J, B, R, y, dt, dev);
    if (q.parts > 0) {
      if (prof) prof->begin(TUCKER_PHASE_TTM_L1);
      if (dt == TUCKER_F64) {
        TK_CUDA(cudaFuncSetAttribute(k_ttm_split_l1<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem));
        k_ttm_split_l1<double><<<q.grid, kThreads, q.smem, s>>>(static_cast<const double *>(y), U, q, z, d_err);
      } else {
        TK_CUDA(cudaFuncSetAttribute(k_ttm_split_l1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem));
        k_ttm_split_l1<float><<<q.grid, kThreads, q.smem, s>>>(static_cast<const float *>(y), U, q, z, d_err);
      }
      TK_LAUNCHED();
      if (prof) prof->end(flops, bytes, 1);
      return TUCKER_OK;
    }
  }
  const TtmSplit2Plan p = ttm_split2_plan(L, J, B, R, dev);
  if (prof) prof->begin(TUCKER_PHASE_TTM);
  if (dt == TUCKER_F64) {
    TK_CUDA(cudaFuncSetAttribute(k_ttm_split2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_ttm_split2<double><<<p.grid, kThreads, p.smem, s>>>(static_cast<const double *>(y), L, B, U, p, z, d_err);
  } else {
    TK_CUDA(cudaFuncSetAttribute(k_ttm_split2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_ttm_split2<float><<<p.grid, kThreads, p.smem, s>>>(static_cast<const float *>(y), L, B, U, p, z, d_err);
  }
  TK_LAUNCHED();
  if (prof) prof->end(flops, bytes, 1);
  return TUCKER_OK;
}

}  // namespace tk
