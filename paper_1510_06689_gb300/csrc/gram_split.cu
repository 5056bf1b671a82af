// Split-precision Gram on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// The Gram step of Algorithm 1 (S = Y_(n) Y_(n)^T, Sec. 2.2) dominates the
// flops; GB300 runs float64 at ~1.2 TFLOP/s but BF16 tensor MMAs at ~1.9
// PFLOP/s.  This kernel forms the Gram from exact integer digits:
//
//   * Columns are taken in groups of 512.  A first pass (k_rowgroup_exp)
//     tabulates, for row i of group g, the exponent E_ig of the smallest
//     power of two above the row's largest magnitude in the group, and the
//     largest magnitude overall.  Every entry then becomes
//     v = round(y 2^(21 - E_ig)), |v| <= 2^21, split into three balanced
//     digits v = s1 2^14 + s2 2^7 + s3 (|s1| <= 128, |s2|, |s3| <= 64); the
//     digits and 2 s3 are exact in BF16.  Scaling per row and per group keeps
//     21 significant bits relative to the local magnitude, so rows and regions
//     of small entries keep their relative precision.
//   * Digit products are grouped by level p + q (weight 2^(7 (6 - p - q))),
//     and only the symmetric part of each accumulator counts (S is formed
//     from C + C^T below):
//       acc0 = A1 A1^T                                (level 2)
//       acc1 = A1 A2^T                                (level 3)
//       acc2 = A1 (2 A3)^T + A2 A2^T                  (level 4)
//       acc3 = A2 (2 A3)^T + (2 A3) (A3 / 256)^T      (levels 5 and 6)
//     Digit products of levels 2..5 are integers of at most 2^14; FP32 sums
//     of integers stay exact below 2^24 and acc0..acc2 do over a group
//     (acc2 <= 512 (128 128 + 64 64) < 2^24).  acc3 carries level 6 in units
//     of 2^-7 with ordinary FP32 rounding; its weight is 2^-21 of level 2, so
//     that rounding is ~2^-45 of the result.
//   * At the end of each group the accumulators are drained:
//     C += (2^28 acc0 + 2^22 acc1 + 2^14 acc2 + 2^7 acc3) 2^(E_ig + E_jg - 2 E)
//     into per-thread double-float (FP32 pair) accumulators, with 2^E above
//     the global largest magnitude; S = (C + C^T) 2^(2E - 43) after a
//     fixed-order float64 reduction of the per-CTA partials.  The four
//     128 x 128 accumulators fill TMEM's 512 columns; the double-float C
//     (128 KB) sits in shared memory beside two 32-column digit stages, so
//     the converting threads keep their registers for a two-chunk prefetch.
//
// Both exponents are read on the device, so the step needs no host round
// trip.  The result is the Gram of Y rounded to 21 bits below each local
// power of two (zero-mean rounding); the noise this adds to the tail
// eigenvalues is ~ (J - R)/J 2^-42/12 (2^E_ig / rms)^2 of ||Y||^2, a few
// 1e-13 for smooth data.  Operand tiles use the K-major, no-swizzle canonical
// layout of tcgen05 shared-memory descriptors (8-row x 16-byte core
// matrices; LBO = 128 B between core matrices along K, SBO = 512 B between
// 8-row groups).  Every mbarrier wait is bounded and CTA-uniform; on expiry
// the kernel raises an error flag, waits (bounded) for its own MMAs, frees
// its TMEM and returns.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tk {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kRows = 128;         // M = N = 128 (J <= 128, zero padded)
constexpr int kChunk = 32;         // columns staged per stage
constexpr int kTiles = 4;          // digit tiles A1, A2, 2 A3, A3 / 256
constexpr int kTileBytes = kRows * kChunk * 2;
constexpr int kSbo = kChunk / 8 * 128;  // bytes between 8-row core-matrix groups
constexpr int kStageBytes = kTiles * kTileBytes;
constexpr int kStages = 2;
constexpr int kGroup = 512;        // columns per exponent group and per exact accumulation
constexpr int kDrainChunks = kGroup / kChunk;
constexpr int kTmemCols = 512;
constexpr int kAccPerThread = kRows * kRows / kThreads;  // C entries each thread drains (32)
constexpr int kZeroExp = -4000;    // exponent of an all-zero row (see exp_above)
constexpr uint32_t kIdesc = idesc_bf16(kRows, kRows);

struct SplitPlan {
  int J;
  int64_t K;
  int64_t cols_per_split;  // a multiple of kGroup, so groups never straddle CTAs
  int nsplit;
  int64_t ngroups;
};

// round(|y| 2^(21 - E)) with the sign of y (ties away from zero) from the
// bits, in 32-bit integer arithmetic; e1022 = E + 1022 and |y| < 2^E.  With
// m22 the leading 22 bits of the significand, v = (m22 + 2^sh) >> (sh + 1),
// sh = E + 1022 - exponent field; the bits below m22 cannot change the result.
__device__ __forceinline__ int scaled_int21(double y, int e1022) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const unsigned m22 = (__funnelshift_l(lo, hi, 1) & 0x1FFFFFu) | 0x200000u;
  const int sh = max(min(e1022 - ex, 30), 0);
  unsigned v = (m22 + (1u << sh)) >> (sh + 1);
  v = ex ? v : 0u;  // zero or subnormal
  const int sgn = (int)hi >> 31;
  return ((int)v ^ sgn) - sgn;
}

// Same for float: e1022 = E + 1022 as above; v = round(m24 / 2^sh) with
// sh = E + 129 - exponent field >= 3.
__device__ __forceinline__ int scaled_int21(float y, int e1022) {
  const unsigned b = __float_as_uint(y);
  const int ex = (int)((b >> 23) & 0xFFu);
  const unsigned mant = (b & 0x7FFFFFu) | 0x800000u;
  const int sh = max(min(e1022 - 893 - ex, 31), 1);
  unsigned v = (mant + (1u << (sh - 1))) >> sh;
  v = ex ? v : 0u;
  const int sgn = (int)b >> 31;
  return ((int)v ^ sgn) - sgn;
}

// How a unit of 8 consecutive columns of one row is addressed in the
// (L, J, B) view, where column c = l + L b of row i is y[l + L i + L J b]:
//   kColsStrided   L == 1: the 8 entries are J apart;
//   kColsContig    L % 8 == 0 and y 16-byte aligned: units start at l % 8 == 0,
//                  never cross a run of L, and are read as 16-byte vectors;
//   kColsGeneric   anything else, entry by entry.
enum { kColsGeneric = 0, kColsStrided = 1, kColsContig = 2 };

// Position (l, b) of a column, advanced without divisions.
struct ColPos {
  int64_t l, b;
  __device__ __forceinline__ void init(int64_t c, int64_t L) {
    b = c / L;
    l = c - b * L;
  }
  __device__ __forceinline__ void advance(int64_t n, int64_t L) {
    l += n;
    while (l >= L) {  // at most n / L + 1 times
      l -= L;
      ++b;
    }
  }
};

template <typename T>
__device__ __forceinline__ void load8_vec(const T *__restrict__ p, T (&raw)[8]) {
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + k);
      raw[2 * k] = v.x;
      raw[2 * k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + k);
      raw[4 * k] = v.x;
      raw[4 * k + 1] = v.y;
      raw[4 * k + 2] = v.z;
      raw[4 * k + 3] = v.w;
    }
  }
}

// Columns c .. c + 7 of row i (zero past c_end or past J); pos is column c's
// position (used by kColsContig only).
template <typename T, int kMode>
__device__ __forceinline__ void load_unit(const T *__restrict__ y, int64_t L, int J, int64_t stride_b, int i,
                                          int64_t c, int64_t c_end, const ColPos &pos, T (&raw)[8]) {
  if (i >= J || c >= c_end) {
#pragma unroll
    for (int k = 0; k < 8; ++k) raw[k] = T(0);
    return;
  }
  const bool full = c + 8 <= c_end;
  if constexpr (kMode == kColsStrided) {
    const T *p = y + i + (int64_t)J * c;
#pragma unroll
    for (int k = 0; k < 8; ++k) raw[k] = (full || c + k < c_end) ? __ldg(p + (int64_t)J * k) : T(0);
  } else if constexpr (kMode == kColsContig) {
    const T *p = y + pos.l + L * (int64_t)i + stride_b * pos.b;
    if (full) {
      load8_vec(p, raw);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) raw[k] = (c + k < c_end) ? __ldg(p + k) : T(0);
    }
  } else {
    int64_t b = c / L, l = c - b * L;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      raw[k] = (c + k < c_end) ? __ldg(y + l + stride_b * b + L * (int64_t)i) : T(0);
      if (++l == L) {
        l = 0;
        ++b;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Exponent table: E[g J + i] = exponent of the power of two above max |y_ic|
// over the columns c of group g; the largest magnitude of all goes to *gmax
// as a bit pattern ordered like the magnitude.  One CTA of 256 threads per
// group.  With L == 1 (J dividing 512, J even) the group is one contiguous
// block read as 16-byte vectors, each thread meeting the same two rows
// throughout; otherwise each warp takes whole rows, its lanes spread over the
// group's columns (consecutive columns are consecutive entries within a run
// of L).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_rowgroup_exp(const T *__restrict__ y, int64_t L, int J, int64_t K,
                                                      int contig_pairs, int *__restrict__ E,
                                                      unsigned long long *__restrict__ gmax) {
  __shared__ unsigned rmax[kRows];
  constexpr bool kF64 = sizeof(T) == 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t g = blockIdx.x;
  const int64_t c0 = g * kGroup, c1 = min(K, c0 + kGroup);
  const int ncols = (int)(c1 - c0);
  if (contig_pairs) {
    for (int i = tid; i < kRows; i += 256) rmax[i] = 0u;
    __syncthreads();
    using V2 = typename std::conditional<kF64, double2, float2>::type;
    const V2 *base = reinterpret_cast<const V2 *>(y + c0 * (int64_t)J);
    const int n2 = ncols * J / 2;  // pairs; pair e covers rows (2e) % J and (2e) % J + 1
    const int r0 = (2 * tid) % J;
    unsigned m0 = 0u, m1 = 0u;
    int e = tid;
    for (; e + 3 * 256 < n2; e += 4 * 256) {
      V2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(base + e + u * 256);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        m0 = max(m0, hi_mag(v[u].x));
        m1 = max(m1, hi_mag(v[u].y));
      }
    }
    for (; e < n2; e += 256) {
      const V2 v = __ldg(base + e);
      m0 = max(m0, hi_mag(v.x));
      m1 = max(m1, hi_mag(v.y));
    }
    atomicMax(&rmax[r0], m0);
    atomicMax(&rmax[r0 + 1], m1);
  } else {
    // lane `lane` reads columns c0 + lane + 32 k, k < 16; their offsets are
    // computed once and reused for every row
    const int64_t stride_b = L * (int64_t)J;
    int64_t off[kGroup / 32];
#pragma unroll
    for (int k = 0; k < kGroup / 32; ++k) {
      const int cc = lane + 32 * k;
      const int64_t c = c0 + cc, b = c / L, l = c - b * L;
      off[k] = cc < ncols ? l + stride_b * b : -1;
    }
    for (int i = warp; i < J; i += 8) {
      unsigned m = 0u;
#pragma unroll
      for (int k = 0; k < kGroup / 32; ++k)
        if (off[k] >= 0) m = max(m, hi_mag(__ldg(y + off[k] + L * (int64_t)i)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) rmax[i] = m;
    }
  }
  __syncthreads();
  unsigned gm = 0u;
  for (int i = tid; i < J; i += 256) {
    E[g * J + i] = exp_above(mag_pattern(rmax[i], kF64), kF64);
    gm = max(gm, rmax[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  if (lane == 0 && gm != 0u) atomicMax(gmax, mag_pattern(gm, kF64));
}

template <typename T, int kMode>
__global__ void __launch_bounds__(kThreads, 1) k_gram_split(const T *__restrict__ y, int64_t L, SplitPlan p,
                                                            const int *__restrict__ Etab,
                                                            const unsigned long long *__restrict__ gmax,
                                                            double *__restrict__ ws, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long mbar[kStages];
  __shared__ int rowexp[kRows];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  unsigned char *stage_base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  // double-float accumulators of C, element e of thread t at [e][t]
  float2 *cacc = reinterpret_cast<float2 *>(stage_base + kStages * kStageBytes);
  constexpr bool kF64 = sizeof(T) == 8;

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
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) cacc[e * kThreads + tid] = make_float2(0.f, 0.f);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const int Eref = exp_above(*gmax, kF64);

  const int64_t c_begin = (int64_t)blockIdx.x * p.cols_per_split;
  const int64_t c_end = min(p.K, c_begin + p.cols_per_split);
  const int nchunks = (int)((c_end - c_begin + kChunk - 1) / kChunk);
  const int64_t stride_b = L * (int64_t)p.J;

  // converter role: row `row`, columns 8 kg .. 8 kg + 7 of each chunk
  const int row = tid % kRows;
  const int kg = tid / kRows;
  // drain role: TMEM lanes 32 q .. 32 q + 31, columns 32 cb .. 32 cb + 31
  const int q = warp & 3, cb = warp >> 2;
  const int drow = 32 * q + lane;

  int last_committed = -1;
  int my_e1022 = 0;

  // One chunk: convert `raw` (this chunk's unit) to digits, issue its MMAs,
  // refill `raw` with the unit two chunks ahead, and drain at a group's end.
  // Returns false when a bounded wait expired (stop is then set CTA-wide).
  auto chunk = [&](int ch, T(&raw)[8], ColPos &pos) -> bool {
    const int buf = ch & 1;
    const int in_group = ch % kDrainChunks;
    if (in_group == 0 && tid < kRows) {
      const int64_t g = (c_begin + (int64_t)ch * kChunk) / kGroup;
      rowexp[tid] = tid < p.J ? Etab[g * p.J + tid] : kZeroExp;
    }
    // stage `buf` is free once the MMAs of chunk ch - 2 have completed; one
    // thread waits (bounded) and the barrier hands the outcome to all
    if (ch >= 2 && tid == 0 && !mbar_wait(smem_addr(&mbar[buf]), ((ch - 2) >> 1) & 1)) stop = 1;
    __syncthreads();
    if (stop) return false;
    if (in_group == 0) my_e1022 = rowexp[row] + 1022;
    unsigned char *st = stage_base + buf * kStageBytes;
    {
      uint32_t w[kTiles][4];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        float d[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float v = small_int_float(scaled_int21(raw[k + h], my_e1022));
          const float s1 = round_float(v * 0x1p-14f);
          const float r1 = __fmaf_rn(s1, -16384.0f, v);
          const float s2 = round_float(r1 * 0x1p-7f);
          const float s3 = __fmaf_rn(s2, -128.0f, r1);
          d[h][0] = s1;
          d[h][1] = s2;
          d[h][2] = s3 + s3;
          d[h][3] = s3 * 0x1p-8f;
        }
        const int j = k >> 1;
#pragma unroll
        for (int t = 0; t < kTiles; ++t) w[t][j] = bf16_pair(d[0][t], d[1][t]);
      }
      const int off = (row >> 3) * kSbo + kg * 128 + (row & 7) * 16;
#pragma unroll
      for (int t = 0; t < kTiles; ++t)
        *reinterpret_cast<uint4 *>(st + t * kTileBytes + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t base = smem_addr(st);
#pragma unroll
      for (int s = 0; s < kChunk / 16; ++s) {
        const uint32_t acc = (in_group == 0 && s == 0) ? 0u : 1u;
        const uint64_t a1 = smem_desc(base + 0 * kTileBytes + 256 * s, 128, kSbo);
        const uint64_t a2 = smem_desc(base + 1 * kTileBytes + 256 * s, 128, kSbo);
        const uint64_t a3x2 = smem_desc(base + 2 * kTileBytes + 256 * s, 128, kSbo);
        const uint64_t a3q = smem_desc(base + 3 * kTileBytes + 256 * s, 128, kSbo);
        mma_bf16(tmem + 0, a1, a1, kIdesc, acc);
        mma_bf16(tmem + 128, a1, a2, kIdesc, acc);
        mma_bf16(tmem + 256, a1, a3x2, kIdesc, acc);
        mma_bf16(tmem + 256, a2, a2, kIdesc, 1u);
        mma_bf16(tmem + 384, a2, a3x2, kIdesc, acc);
        mma_bf16(tmem + 384, a3x2, a3q, kIdesc, 1u);
      }
      mma_commit(smem_addr(&mbar[buf]));
    }
    last_committed = ch;
    // refill with the unit two chunks ahead while the tensor cores work
    if constexpr (kMode == kColsContig) pos.advance(2 * kChunk, L);
    load_unit<T, kMode>(y, L, p.J, stride_b, row, c_begin + (int64_t)(ch + 2) * kChunk + 8 * kg, c_end, pos, raw);
    if (in_group == kDrainChunks - 1 || ch == nchunks - 1) {
      if (tid == 0 && !mbar_wait(smem_addr(&mbar[buf]), (ch >> 1) & 1)) stop = 1;
      __syncthreads();
      if (!stop) {  // uniform across the CTA, so the .sync.aligned loads below never diverge
        fence_after();
        const float wts[4] = {0x1p28f, 0x1p22f, 0x1p14f, 0x1p7f};  // 2^28, 2 2^21, 2^14, 2^7
        const int ei = rowexp[drow] - Eref;
#pragma unroll
        for (int part = 0; part < 4; ++part) {
          float sc[8], hi[8], lo[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int x = ei + rowexp[32 * cb + 8 * part + e] - Eref;  // <= 0
            sc[e] = x < -120 ? 0.f : __int_as_float((127 + x) << 23);
            const float2 a = cacc[(8 * part + e) * kThreads + tid];
            hi[e] = a.x;
            lo[e] = a.y;
          }
#pragma unroll
          for (int lev = 0; lev < 4; ++lev) {
            uint32_t r[8];
            tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * lev + 32 * cb + 8 * part), r);
#pragma unroll
            for (int e = 0; e < 8; ++e) df_add(hi[e], lo[e], __uint_as_float(r[e]) * wts[lev] * sc[e]);
          }
#pragma unroll
          for (int e = 0; e < 8; ++e) cacc[(8 * part + e) * kThreads + tid] = make_float2(hi[e], lo[e]);
        }
      }
      fence_before();
      __syncthreads();
      if (stop) return false;
    }
    return true;
  };

  T raw0[8], raw1[8];
  ColPos pos0{0, 0}, pos1{0, 0};
  if constexpr (kMode == kColsContig) {
    pos0.init(c_begin + 8 * kg, L);
    pos1.init(c_begin + kChunk + 8 * kg, L);
  }
  load_unit<T, kMode>(y, L, p.J, stride_b, row, c_begin + 8 * kg, c_end, pos0, raw0);
  load_unit<T, kMode>(y, L, p.J, stride_b, row, c_begin + kChunk + 8 * kg, c_end, pos1, raw1);
  for (int ch = 0; ch < nchunks; ch += 2) {
    if (!chunk(ch, raw0, pos0)) break;
    if (ch + 1 < nchunks && !chunk(ch + 1, raw1, pos1)) break;
  }
  // make sure no MMA of ours is still running before TMEM is released
  if (stop && last_committed >= 0 && tid == 0)
    mbar_wait(smem_addr(&mbar[last_committed & 1]), (last_committed >> 1) & 1);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (stop) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  // per-CTA C (not yet symmetrised), row-major 128 x 128
  double *dst = ws + (size_t)blockIdx.x * kRows * kRows + (size_t)drow * kRows + 32 * cb;
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) {
    const float2 a = cacc[e * kThreads + tid];
    dst[e] = (double)a.x + (double)a.y;
  }
}

// S = (sum of the per-CTA C + C^T) 2^(2E - 43); NaN throughout when the
// largest magnitude is not finite (Y holds Inf or NaN).
__global__ void __launch_bounds__(256) k_gram_split_reduce(const double *__restrict__ ws, int nsplit, int J,
                                                           const unsigned long long *__restrict__ gmax, int is_f64,
                                                           double *__restrict__ S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= J * J) return;
  const int i = idx % J, j = idx / J;
  double s = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) {
    const double *c = ws + (size_t)sp * kRows * kRows;
    s += c[i * kRows + j] + c[j * kRows + i];
  }
  const unsigned long long gm = *gmax;
  const bool finite = is_f64 ? gm < 0x7FF0000000000000ull : gm < 0x7F800000ull;
  const int E = exp_above(gm, is_f64 != 0);
  S[i + (int64_t)J * j] = !finite ? __longlong_as_double(0x7FF8000000000000ll) : (E == kZeroExp ? 0.0 : ldexp(s, 2 * E - 43));
}

constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + (size_t)kRows * kRows * sizeof(float2) + 1024;

SplitPlan split_plan(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev) {
  SplitPlan p{};
  p.J = (int)J;
  p.K = L * B;
  p.ngroups = (p.K + kGroup - 1) / kGroup;
  const int64_t ns = std::max<int64_t>(1, std::min<int64_t>(dev.sms, p.ngroups));
  const int64_t groups_per = (p.ngroups + ns - 1) / ns;
  p.cols_per_split = groups_per * kGroup;
  p.nsplit = (int)((p.K + p.cols_per_split - 1) / p.cols_per_split);
  return p;
}

// workspace (in doubles): per-CTA partials | exponent table (ints) | gmax | error flag
struct SplitWs {
  double *partials;
  int *table;
  unsigned long long *gmax;
  int *err;
};

SplitWs split_ws(double *d_ws, const SplitPlan &p) {
  const int64_t np = (int64_t)p.nsplit * kRows * kRows;
  const int64_t tab = (p.ngroups * p.J + 1) / 2;
  SplitWs w;
  w.partials = d_ws;
  w.table = reinterpret_cast<int *>(d_ws + np);
  w.gmax = reinterpret_cast<unsigned long long *>(d_ws + np + tab);
  w.err = reinterpret_cast<int *>(d_ws + np + tab + 1);
  return w;
}

template <typename T, int kMode>
int run_gram_split(const void *y, int64_t L, const SplitPlan &p, const SplitWs &w, const DeviceInfo &dev,
                   cudaStream_t s) {
  (void)dev;
  TK_CUDA(cudaFuncSetAttribute(k_gram_split<T, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  k_gram_split<T, kMode><<<p.nsplit, kThreads, kSmemBytes, s>>>(static_cast<const T *>(y), L, p, w.table, w.gmax,
                                                                w.partials, w.err);
  TK_LAUNCHED();
  return TUCKER_OK;
}

}  // namespace

int64_t gram_split_workspace_doubles(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev) {
  const SplitPlan p = split_plan(L, J, B, dev);
  return (int64_t)p.nsplit * kRows * kRows + (p.ngroups * p.J + 1) / 2 + 4;
}

int launch_gram_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *d_S, double *d_ws,
                      const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (J > kRows) {
    set_error("split-precision Gram supports J <= %d (got %lld)", kRows, (long long)J);
    return TUCKER_EUNSUPPORTED;
  }
  const SplitPlan p = split_plan(L, J, B, dev);
  if (p.ngroups > 0x7FFFFFFFll) {
    set_error("split-precision Gram: too many column groups (%lld)", (long long)p.ngroups);
    return TUCKER_EUNSUPPORTED;
  }
  const SplitWs w = split_ws(d_ws, p);
  const bool f64 = dt == TUCKER_F64;
  const double in_bytes = (double)p.K * J * (f64 ? 8 : 4);
  TK_CUDA(cudaMemsetAsync(w.gmax, 0, 2 * sizeof(double), s));  // gmax and the error flag
  const int contig_pairs = L == 1 && (2 * 256) % J == 0 && J % 2 == 0 &&
                           reinterpret_cast<uintptr_t>(y) % (f64 ? 16 : 8) == 0;
  const int mode = L == 1 ? kColsStrided
                          : (L % 8 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0) ? kColsContig : kColsGeneric;
  if (prof) prof->begin(TUCKER_PHASE_SCALE);
  if (f64)
    k_rowgroup_exp<double><<<(unsigned)p.ngroups, 256, 0, s>>>(static_cast<const double *>(y), L, (int)J, p.K,
                                                               contig_pairs, w.table, w.gmax);
  else
    k_rowgroup_exp<float><<<(unsigned)p.ngroups, 256, 0, s>>>(static_cast<const float *>(y), L, (int)J, p.K,
                                                              contig_pairs, w.table, w.gmax);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, in_bytes, 1);
  if (prof) prof->begin(TUCKER_PHASE_GRAM);
  if (f64) {
    if (mode == kColsStrided) TK_CHECK((run_gram_split<double, kColsStrided>(y, L, p, w, dev, s)));
    else if (mode == kColsContig) TK_CHECK((run_gram_split<double, kColsContig>(y, L, p, w, dev, s)));
    else TK_CHECK((run_gram_split<double, kColsGeneric>(y, L, p, w, dev, s)));
  } else {
    if (mode == kColsStrided) TK_CHECK((run_gram_split<float, kColsStrided>(y, L, p, w, dev, s)));
    else if (mode == kColsContig) TK_CHECK((run_gram_split<float, kColsContig>(y, L, p, w, dev, s)));
    else TK_CHECK((run_gram_split<float, kColsGeneric>(y, L, p, w, dev, s)));
  }
  if (prof) prof->end((double)J * (J + 1) * (double)p.K, in_bytes, 1);
  if (prof) prof->begin(TUCKER_PHASE_GRAM_REDUCE);
  k_gram_split_reduce<<<(unsigned)((J * J + 255) / 256), 256, 0, s>>>(w.partials, p.nsplit, (int)J, w.gmax, f64,
                                                                      d_S);
  TK_LAUNCHED();
  if (prof) prof->end((double)p.nsplit * J * J * 2, (double)p.nsplit * kRows * kRows * 8, 1);
  return TUCKER_OK;
}

int gram_split_error(const double *d_ws, int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, int *h_err,
                     cudaStream_t s) {
  const SplitPlan p = split_plan(L, J, B, dev);
  const SplitWs w = split_ws(const_cast<double *>(d_ws), p);
  TK_CUDA(cudaMemcpyAsync(h_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return TUCKER_OK;
}

}  // namespace tk
