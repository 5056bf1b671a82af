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
// A CTA keeps U's digits in shared memory, streams tiles of 32 columns
// through two operand stages and two TMEM accumulator sets, and drains tile
// t - 1 while the tensor cores work on tile t.  Waits are bounded and
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
constexpr int kN = 32;            // columns per tile
constexpr int kMaxJp = 128;       // contraction length, padded to a multiple of 16
constexpr int kATiles = 4;        // U1..U4
constexpr int kBTiles = 4;        // Y1..Y4
constexpr int kTmemCols = 256;    // two sets x four levels x 32 columns
constexpr uint32_t kIdesc = idesc_bf16(kM, kN);

struct TtmSplitPlan {
  int J, Jp, R;
  int64_t K;       // columns of the unfolding (L * B)
  int64_t ntiles;
  int grid;
  size_t smem;
};

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

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_ttm_split(const T *__restrict__ y, int64_t L, int64_t B,
                                                           const double *__restrict__ U, TtmSplitPlan p,
                                                           double *__restrict__ z, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long mbar[2];
  // per-tile column metadata, three slots (tile it uses slot it % 3): the
  // next tile's loads fill one slot while the previous tile drains from another
  __shared__ unsigned long long colmax[3][kN];
  __shared__ int colexp[3][kN];
  __shared__ int64_t colin[3][kN], colout[3][kN];
  __shared__ int rowexp[kM];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  constexpr bool kF64 = sizeof(T) == 8;
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  const int Jp = p.Jp;
  const int a_tile = kM * Jp * 2;        // bytes of one U digit tile
  const int b_tile = kN * Jp * 2;        // bytes of one Y digit tile
  const uint32_t sbo = (uint32_t)(Jp / 8) * 128u;
  unsigned char *A = base;                         // 4 tiles
  unsigned char *Bst = base + kATiles * a_tile;    // 2 stages x 4 tiles

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_addr(&mbar[0]), 1);
    mbar_init(smem_addr(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
  }
  // exponents of U's columns (output rows)
  if (tid < kM) {
    unsigned long long m = 0ull;
    if (tid < p.R)
      for (int j = 0; j < p.J; ++j) m = max(m, mag_bits(U[j + (int64_t)p.J * tid]));
    rowexp[tid] = exp_above(m, true);
  }
  __syncthreads();
  // U's digit tiles (A operands: row r, k = j), 8 consecutive j per unit
  for (int u = tid; u < kM * (Jp / 8); u += kThreads) {
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
    const int off = (r >> 3) * (int)sbo + jg * 128 + (r & 7) * 16;
#pragma unroll
    for (int t = 0; t < kATiles; ++t)
      *reinterpret_cast<uint4 *>(A + t * a_tile + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const int64_t in_b = L * (int64_t)p.J, out_b = L * (int64_t)p.R;
  const int ngroups = Jp / 8;
  const int units = kN * ngroups;
  // load unit: column my_c (= lane) and 8 consecutive j; lanes write consecutive
  // 16-byte core-matrix rows, so the operand stores are free of bank conflicts
  const int my_c = tid % kN, my_jg = tid / kN;
  const bool loader = tid < units;

  // --- load phase of a tile: column addresses, then the raw entries into registers
  T raw[8];
  auto load_tile = [&](int64_t t, int slot) {
    if (tid < kN) {
      colmax[slot][tid] = 0ull;
      const int64_t c = t * kN + tid;
      int64_t bi = -1, bo = -1;
      if (c < p.K) {
        const int64_t b = c / L, l = c - b * L;
        bi = l + in_b * b;
        bo = l + out_b * b;
      }
      colin[slot][tid] = bi;
      colout[slot][tid] = bo;
    }
    __syncthreads();
    if (loader) {
      const int64_t bi = colin[slot][my_c];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int j = 8 * my_jg + k;
        raw[k] = (bi >= 0 && j < p.J) ? __ldg(y + bi + L * (int64_t)j) : T(0);
      }
    }
  };

  // --- drain of a finished tile: all 16 warps, warp w reads TMEM lanes
  // 32 (w % 4) .. +31 and columns 8 (w / 4) .. +7 of the four levels
  auto drain = [&](int done_it) {
    const int dset = done_it & 1, dm = done_it % 3;
    if (tid == 0 && !mbar_wait(smem_addr(&mbar[dset]), (done_it >> 1) & 1)) stop = 1;
    __syncthreads();
    const int q = warp & 3, cg = warp >> 2;
    if (!stop && 32 * q < p.R) {
      fence_after();
      const int r = 32 * q + lane;
      const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(dset * 128 + 8 * cg);
      uint32_t a[4][8];
#pragma unroll
      for (int lev = 0; lev < 4; ++lev) tmem_ld8(tb + (uint32_t)(32 * lev), a[lev]);
      if (r < p.R) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int c = 8 * cg + e;
          const int64_t ob = colout[dm][c];
          if (ob < 0) continue;
          const long long v = ((long long)__float2int_rn(__uint_as_float(a[0][e])) << 28) +
                              ((long long)__float2int_rn(__uint_as_float(a[1][e])) << 21) +
                              ((long long)__float2int_rn(__uint_as_float(a[2][e])) << 14) +
                              ((long long)__float2int_rn(__uint_as_float(a[3][e])) << 7);
          z[ob + L * (int64_t)r] = scaled_ll_to_double(v, rowexp[r] + colexp[dm][c] - 42);
        }
      }
    }
    fence_before();
    __syncthreads();
  };

  int last_it = -1;
  int it = 0;
  int64_t t = blockIdx.x;
  if (t < p.ntiles) load_tile(t, 0);
  for (; t < p.ntiles; t += gridDim.x, ++it) {
    const int set = it & 1, ms = it % 3;
    // column exponents of this tile
    if (loader) {
      unsigned long long m = 0ull;
#pragma unroll
      for (int k = 0; k < 8; ++k) m = max(m, mag_bits(raw[k]));
      atomicMax(&colmax[ms][my_c], m);
    }
    // operand stage `set` is free once the MMAs of tile it - 2 have finished
    if (it >= 2 && tid == 0 && !mbar_wait(smem_addr(&mbar[set]), ((it - 2) >> 1) & 1)) stop = 1;
    __syncthreads();
    if (stop) break;
    if (tid < kN) colexp[ms][tid] = exp_above(colmax[ms][tid], kF64);
    __syncthreads();
    if (loader) {
      const int e = colexp[ms][my_c];
      uint32_t w[kBTiles][4];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        int d[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) digits4(scaled_int28(raw[k + h], e), d[h]);
#pragma unroll
        for (int q = 0; q < kBTiles; ++q) w[q][k >> 1] = bf16_pair((float)d[0][q], (float)d[1][q]);
      }
      unsigned char *st = Bst + set * kBTiles * b_tile;
      const int off = (my_c >> 3) * (int)sbo + my_jg * 128 + (my_c & 7) * 16;
#pragma unroll
      for (int q = 0; q < kBTiles; ++q)
        *reinterpret_cast<uint4 *>(st + q * b_tile + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t ab = smem_addr(A), bb = smem_addr(Bst + set * kBTiles * b_tile);
      const uint32_t d0 = tmem + (uint32_t)(set * 128);
      for (int ks = 0; ks < Jp / 16; ++ks) {
        const uint32_t acc = ks ? 1u : 0u;
        uint64_t ua[kATiles], yb[kBTiles];
#pragma unroll
        for (int q = 0; q < kATiles; ++q) ua[q] = smem_desc(ab + q * a_tile + 256 * ks, 128, sbo);
#pragma unroll
        for (int q = 0; q < kBTiles; ++q) yb[q] = smem_desc(bb + q * b_tile + 256 * ks, 128, sbo);
        mma_bf16(d0 + 0, ua[0], yb[0], kIdesc, acc);
        mma_bf16(d0 + 32, ua[0], yb[1], kIdesc, acc);
        mma_bf16(d0 + 32, ua[1], yb[0], kIdesc, 1u);
        mma_bf16(d0 + 64, ua[0], yb[2], kIdesc, acc);
        mma_bf16(d0 + 64, ua[1], yb[1], kIdesc, 1u);
        mma_bf16(d0 + 64, ua[2], yb[0], kIdesc, 1u);
        mma_bf16(d0 + 96, ua[0], yb[3], kIdesc, acc);
        mma_bf16(d0 + 96, ua[1], yb[2], kIdesc, 1u);
        mma_bf16(d0 + 96, ua[2], yb[1], kIdesc, 1u);
        mma_bf16(d0 + 96, ua[3], yb[0], kIdesc, 1u);
      }
      mma_commit(smem_addr(&mbar[set]));
    }
    last_it = it;
    // loads of the next tile are in flight while the previous tile drains
    if (t + gridDim.x < p.ntiles) load_tile(t + gridDim.x, (it + 1) % 3);
    if (it >= 1) drain(it - 1);
    if (stop) break;
  }
  if (!stop && it >= 1) drain(it - 1);
  if (stop && tid == 0 && last_it >= 0)  // let our own MMAs finish before TMEM is released
    mbar_wait(smem_addr(&mbar[last_it & 1]), (last_it >> 1) & 1);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (stop && tid == 0) atomicExch(err, 1);
}

TtmSplitPlan ttm_split_plan(int64_t L, int64_t J, int64_t B, int64_t R, const DeviceInfo &dev) {
  TtmSplitPlan p{};
  p.J = (int)J;
  p.Jp = (int)((J + 15) / 16 * 16);
  p.R = (int)R;
  p.K = L * B;
  p.ntiles = (p.K + kN - 1) / kN;
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(dev.sms, p.ntiles));
  p.smem = (size_t)kATiles * kM * p.Jp * 2 + (size_t)2 * kBTiles * kN * p.Jp * 2 + 1024;
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
  const TtmSplitPlan p = ttm_split_plan(L, J, B, R, dev);
  if (prof) prof->begin(TUCKER_PHASE_TTM);
  if (dt == TUCKER_F64) {
    TK_CUDA(cudaFuncSetAttribute(k_ttm_split<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_ttm_split<double><<<p.grid, kThreads, p.smem, s>>>(static_cast<const double *>(y), L, B, U, p, z, d_err);
  } else {
    TK_CUDA(cudaFuncSetAttribute(k_ttm_split<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_ttm_split<float><<<p.grid, kThreads, p.smem, s>>>(static_cast<const float *>(y), L, B, U, p, z, d_err);
  }
  TK_LAUNCHED();
  if (prof)
    prof->end(2.0 * J * R * (double)p.K, (double)p.K * (J * (dt == TUCKER_F64 ? 8.0 : 4.0) + R * 8.0) + J * R * 8.0,
              1);
  return TUCKER_OK;
}

}  // namespace tk
