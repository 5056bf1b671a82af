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

}  // namespace

int launch_ttm_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *U, int64_t R,
                     double *z, int *d_err, const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (J > kMaxJp || R > kM || R > J) {
    set_error("split-precision TTM supports R <= J <= %d (got J = %lld, R = %lld)", kMaxJp, (long long)J,
              (long long)R);
    return TUCKER_EUNSUPPORTED;
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
  if (prof)
    prof->end(2.0 * J * R * (double)p.K, (double)p.K * (J * (dt == TUCKER_F64 ? 8.0 : 4.0) + R * 8.0) + J * R * 8.0,
              1);
  return TUCKER_OK;
}

}  // namespace tk
