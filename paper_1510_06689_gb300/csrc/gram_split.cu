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
//     C += (2^28 acc0 + 2^22 acc1 + 2^14 acc2 + 2^7 acc3)
//          2^(E_ig - ref_i + E_jg - ref_j)
//     into per-thread double-float (FP32 pair) accumulators, with ref_i the
//     largest E_ig over the CTA's groups; S_ij = sum over CTAs of
//     (C_ij + C_ji) 2^(ref_i + ref_j - 43) by a fixed-order float64
//     reduction.  The four 128 x 128 accumulators fill TMEM's 512 columns.
//     In the register-staged kernel the double-float C (128 KB) sits in
//     shared memory beside two 32-column digit stages, so the converting
//     threads keep their registers for a two-chunk prefetch; the tensor-map
//     kernel keeps C in registers and its raw input in a ring of
//     shared-memory slots.  It takes L == 1 (32 consecutive columns a chunk)
//     and float64 L > 1 with L a multiple of 8, where a chunk is a box of
//     nl octets of consecutive l times 4 / nl consecutive b (the Gram sums
//     over columns in any order), nl chosen to pad the fewest columns.
//
// The exponents are read on the device, so the step needs no host round
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
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tk {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kRows = 128;         // M = N = 128: one block of rows (J zero padded to blocks of 128)
constexpr int kMaxRows = 512;      // largest J: up to four row blocks, Grams of their pairs
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

// Row exponent as the table stores it: E with max |y| < 2^E, raised to a
// floor (float64: 2^-850, whose square is already below the smallest float64
// subnormal; float32: 2^-100, so rows below it are rounded on the 2^-121
// grid), or kZeroExp for an all-zero row.  The reference exponent of the
// drain uses the same rule, so every scale 2^(E_i + E_j - 2 E) stays <= 1.
__device__ __forceinline__ int table_exp(unsigned long long pattern, bool f64) {
  const int e = exp_above(pattern, f64);
  return e == kZeroExp ? e : max(e, f64 ? -850 : -100);
}

// Reference exponent of row i for this CTA: the largest table exponent of the
// row over the CTA's groups [g_begin, g_end) (kZeroExp for a row that is zero
// there).  The drain scales group g's products by 2^(E_ig - ref_i + E_jg -
// ref_j) <= 1, so only a row's own range over the CTA's columns limits the
// float32 exponent range of the double-float accumulators; the per-CTA
// partial carries the factor 2^(ref_i + ref_j) to the reduction.  All threads
// call it; ends with a barrier.  The rows are r0 .. r0 + rows - 1 of the
// table (J per group).
__device__ void cta_row_ref(const int *__restrict__ Etab, int J, int r0, int rows, int64_t g_begin, int64_t g_end,
                            int *ref, int *__restrict__ ref_out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < kRows) ref[tid] = kZeroExp;
  __syncthreads();
  const int i = tid % kRows;
  if (i < rows) {
    int m = kZeroExp;
    for (int64_t g = g_begin + tid / kRows; g < g_end; g += nt / kRows) m = max(m, __ldg(Etab + g * J + r0 + i));
    atomicMax(&ref[i], m);
  }
  __syncthreads();
  if (tid < kRows) ref_out[tid] = ref[tid];
}
__device__ void cta_row_ref(const int *__restrict__ Etab, int J, int64_t g_begin, int64_t g_end, int *ref,
                            int *__restrict__ ref_out) {
  cta_row_ref(Etab, J, 0, J, g_begin, g_end, ref, ref_out);
}

struct SplitPlan {
  int J;
  int64_t K;               // columns (L > 1 tiled path: 32 per chunk of 8 l x 4 b)
  int64_t cols_per_split;  // a multiple of kGroup, so groups never straddle CTAs
  int nsplit;
  int64_t ngroups;
  int nrb;                 // row blocks of 128 (J > 128: the diagonal blocks' CTAs are split x block)
  int npair;               // off-diagonal block pairs (the pair kernel's CTAs are split x pair)
  int nsplit_pair;         // column ranges of the pair kernel, each of cols_per_split_pair columns
  int64_t cols_per_split_pair;
  // tiled path (L > 1): a chunk is nl octets of l (8 l each) x nb = 4 / nl
  // consecutive b; chunk ch covers octets nl (ch % nL) .. and b from nb (ch / nL)
  int64_t nL;              // chunks along l (0: not the tiled path)
  int nl, nb;
  int64_t B;
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
// throughout.  Otherwise each warp takes rows two at a time, its lanes spread
// over the group's columns (consecutive columns are consecutive entries
// within a run of L), loading only the high 32-bit word of each float64 (all
// the magnitude order needs) with 32 loads in flight per lane; with colexp
// given, the exponent above each column's largest magnitude (over all J rows:
// the per-column scale of the split mode product) is written too.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ unsigned ldg_mag(const T *p) {
  if constexpr (sizeof(T) == 8) return __ldg(reinterpret_cast<const unsigned *>(p) + 1) & 0x7FFFFFFFu;
  else return __ldg(reinterpret_cast<const unsigned *>(p)) & 0x7FFFFFFFu;
}

// Contiguous columns of J = 64 HP entries (L == 1), also taking each
// column's largest magnitude: warp w reads columns w kC + 8 kC i .. + kC - 1
// (kC = 8 / HP columns, eight 16-byte pairs per lane in flight), lane l
// holding rows 2 l + 64 h and 2 l + 64 h + 1 (h < HP) throughout, so the
// row maxima stay in registers until one atomic per row at the end and a
// column's maximum is one warp reduction (no atomics).  cmax[cc] gets the
// magnitude bits of column c0 + cc (cc < ncols); rmax must be zeroed.
template <typename T, int HP>
__device__ __forceinline__ void exp_cols_contig(const T *__restrict__ y, int64_t c0, int ncols, unsigned *rmax,
                                                unsigned *cmax, int lane, int warp) {
  using V2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  constexpr int kC = 8 / HP;
  unsigned rm[2 * HP];
#pragma unroll
  for (int h = 0; h < 2 * HP; ++h) rm[h] = 0u;
  for (int cb = warp * kC; cb < ncols; cb += 8 * kC) {  // warp-uniform
    V2 v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int cc = cb + s / HP, h = s % HP;
      if (cc < ncols) {
        v[s] = __ldg(reinterpret_cast<const V2 *>(y + (c0 + cc) * (int64_t)(64 * HP) + 2 * lane + 64 * h));
      } else {
        v[s].x = v[s].y = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < kC; ++u) {
      unsigned cm = 0u;
#pragma unroll
      for (int h = 0; h < HP; ++h) {
        const unsigned a = hi_mag(v[u * HP + h].x), b = hi_mag(v[u * HP + h].y);
        rm[2 * h] = max(rm[2 * h], a);
        rm[2 * h + 1] = max(rm[2 * h + 1], b);
        cm = max(cm, max(a, b));
      }
      cm = __reduce_max_sync(0xffffffffu, cm);
      if (lane == 0 && cb + u < ncols) cmax[cb + u] = cm;
    }
  }
#pragma unroll
  for (int h = 0; h < HP; ++h) {
    atomicMax(&rmax[2 * lane + 64 * h], rm[2 * h]);
    atomicMax(&rmax[2 * lane + 64 * h + 1], rm[2 * h + 1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rowgroup_exp(const T *__restrict__ y, int64_t L, int J, int64_t K,
                                                      int contig_pairs, int *__restrict__ E,
                                                      unsigned long long *__restrict__ gmax,
                                                      int *__restrict__ colexp) {
  __shared__ unsigned rmax[kMaxRows];
  __shared__ unsigned cmax[kGroup];
  constexpr bool kF64 = sizeof(T) == 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t g = blockIdx.x;
  const int64_t c0 = g * kGroup, c1 = min(K, c0 + kGroup);
  const int ncols = (int)(c1 - c0);
  if (contig_pairs && colexp && J % 64 == 0) {
    // column exponents too: warps over whole columns
    for (int i = tid; i < kMaxRows; i += 256) rmax[i] = 0u;
    __syncthreads();
    switch (J / 64) {
      case 1: exp_cols_contig<T, 1>(y, c0, ncols, rmax, cmax, lane, warp); break;
      case 2: exp_cols_contig<T, 2>(y, c0, ncols, rmax, cmax, lane, warp); break;
      case 4: exp_cols_contig<T, 4>(y, c0, ncols, rmax, cmax, lane, warp); break;
      default: exp_cols_contig<T, 8>(y, c0, ncols, rmax, cmax, lane, warp); break;
    }
    __syncthreads();
    for (int cc = tid; cc < ncols; cc += 256) colexp[c0 + cc] = exp_above(mag_pattern(cmax[cc], kF64), kF64);
  } else if (contig_pairs) {
    for (int i = tid; i < kMaxRows; i += 256) rmax[i] = 0u;
    if (colexp)
      for (int cc = tid; cc < kGroup; cc += 256) cmax[cc] = 0u;
    __syncthreads();
    using V2 = typename std::conditional<kF64, double2, float2>::type;
    const V2 *base = reinterpret_cast<const V2 *>(y + c0 * (int64_t)J);
    const int n2 = ncols * J / 2;  // pairs; pair e covers rows (2e) % J and (2e) % J + 1 of column (2e) / J
    const int r0 = (2 * tid) % J;
    unsigned m0 = 0u, m1 = 0u;
    int e = tid;
    for (; e + 3 * 256 < n2; e += 4 * 256) {
      V2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(base + e + u * 256);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned a = hi_mag(v[u].x), b = hi_mag(v[u].y);
        m0 = max(m0, a);
        m1 = max(m1, b);
        if (colexp) atomicMax(&cmax[(2 * (e + u * 256)) / J], max(a, b));  // J < 64 only
      }
    }
    for (; e < n2; e += 256) {
      const V2 v = __ldg(base + e);
      const unsigned a = hi_mag(v.x), b = hi_mag(v.y);
      m0 = max(m0, a);
      m1 = max(m1, b);
      if (colexp) atomicMax(&cmax[(2 * e) / J], max(a, b));
    }
    atomicMax(&rmax[r0], m0);
    atomicMax(&rmax[r0 + 1], m1);
    if (colexp) {
      __syncthreads();
      for (int cc = tid; cc < ncols; cc += 256) colexp[c0 + cc] = exp_above(mag_pattern(cmax[cc], kF64), kF64);
    }
  } else {
    // lane `lane` reads columns c0 + lane + 32 k, k < 16; their offsets are
    // computed once and reused for every row
    const int64_t stride_b = L * (int64_t)J;
    constexpr int kPer = kGroup / 32;
    int64_t off[kPer];
    unsigned colm[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int cc = lane + 32 * k;
      const int64_t c = c0 + cc, b = c / L, l = c - b * L;
      off[k] = cc < ncols ? l + stride_b * b : -1;
      colm[k] = 0u;
    }
    for (int i = warp; i < J; i += 16) {  // rows i and i + 8
      const int i2 = i + 8;
      unsigned a[kPer], b2[kPer];
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        a[k] = off[k] >= 0 ? ldg_mag(y + off[k] + L * (int64_t)i) : 0u;
        b2[k] = (off[k] >= 0 && i2 < J) ? ldg_mag(y + off[k] + L * (int64_t)i2) : 0u;
      }
      unsigned ma = 0u, mb = 0u;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        ma = max(ma, a[k]);
        mb = max(mb, b2[k]);
        colm[k] = max(colm[k], max(a[k], b2[k]));
      }
      ma = __reduce_max_sync(0xffffffffu, ma);
      mb = __reduce_max_sync(0xffffffffu, mb);
      if (lane == 0) {
        rmax[i] = ma;
        if (i2 < J) rmax[i2] = mb;
      }
    }
    if (colexp) {
      for (int cc = tid; cc < kGroup; cc += 256) cmax[cc] = 0u;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kPer; ++k) atomicMax(&cmax[lane + 32 * k], colm[k]);
      __syncthreads();
      for (int cc = tid; cc < ncols; cc += 256) colexp[c0 + cc] = exp_above(mag_pattern(cmax[cc], kF64), kF64);
    }
  }
  __syncthreads();
  unsigned gm = 0u;
  for (int i = tid; i < J; i += 256) {
    E[g * J + i] = table_exp(mag_pattern(rmax[i], kF64), kF64);
    gm = max(gm, rmax[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  if (lane == 0 && gm != 0u) atomicMax(gmax, mag_pattern(gm, kF64));
}

// The exponent pass for L > 1 with 16-byte column strides (L sizeof(T) a
// multiple of 16, Y 16-byte aligned): a group's rows pass through shared
// memory in stages of RS rows, each thread copying 16-byte chunks (2 float64
// or 4 float32 of consecutive columns, never straddling a run of L) with
// cp.async, two stages in flight; a thread reads back only its own chunks,
// so the stream needs no barrier until the per-column maxima are combined.
// kOct (float64): the group is 16 consecutive chunks of the tiled Gram (nl
// octets of consecutive l times nb = 4 / nl consecutive b each; chunk ch
// starts at octet nl (ch % nL) and at b = nb (ch / nL)), so its exponents are
// the ones that kernel's groups need.
template <typename T, bool kOct>
__global__ void __launch_bounds__(512) k_rowgroup_exp_async(const T *__restrict__ y, int64_t L, int J, int64_t K,
                                                            int64_t nL, int nl, int64_t B, int *__restrict__ E,
                                                            unsigned long long *__restrict__ gmax,
                                                            int *__restrict__ colexp) {
  constexpr bool kF64 = sizeof(T) == 8;
  static_assert(!kOct || kF64, "the tiled groups take float64");
  constexpr int V = 16 / (int)sizeof(T);  // entries per chunk
  constexpr int NQ = kGroup / V;          // chunks per row of a group
  constexpr int RT = 512 / NQ;            // threads per chunk column
  constexpr int RS = 4 * RT;              // rows per stage: four chunks per thread
  extern __shared__ uint4 stg[];          // 2 stages x RS x NQ chunks
  __shared__ unsigned rmax[kMaxRows];
  __shared__ unsigned cmax[kGroup];
  const int tid = threadIdx.x, lane = tid & 31;
  const int q = tid % NQ, r0 = tid / NQ;
  const int64_t c0 = (int64_t)blockIdx.x * kGroup;
  const int ncols = (int)min((int64_t)kGroup, K - c0);
  // the chunk q's first column (l, b) and its offset
  auto chunk_col = [&](int qq, int64_t &l, int64_t &b) -> bool {
    if (kOct) {
      const int64_t ch = c0 / 32 + (qq >> 4);
      const int w = qq & 15, kg = w >> 2;  // kg: the box's line block (b offset kg / nl, octet kg % nl)
      const int64_t bb = ch / nL;
      b = (4 / nl) * bb + kg / nl;
      l = 8 * (nl * (ch - bb * nL) + kg % nl) + 2 * (w & 3);
      return V * qq < ncols && b < B && l < L;
    }
    const int64_t c = c0 + V * qq;
    b = c / L;
    l = c - b * L;
    return V * qq < ncols;
  };
  int64_t lq = 0, bq = 0;
  const bool valid = chunk_col(q, lq, bq);
  const int64_t goff = valid ? lq + L * (int64_t)J * bq : 0;
  for (int i = tid; i < kMaxRows; i += 512) rmax[i] = 0u;
  for (int i = tid; i < kGroup; i += 512) cmax[i] = 0u;
  __syncthreads();
  const int nst = (J + RS - 1) / RS;
  auto issue = [&](int st) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = st * RS + r0 + RT * u;
      if (valid && i < J) {
        const uint32_t dst = smem_addr(&stg[((st & 1) * RS + r0 + RT * u) * NQ + q]);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(y + goff + L * (int64_t)i)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  unsigned colm[V];
#pragma unroll
  for (int v = 0; v < V; ++v) colm[v] = 0u;
  issue(0);
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) issue(st + 1);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // stage st has landed (this thread's copies)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = st * RS + r0 + RT * u;  // uniform across the warp (a warp has one r0)
      if (i >= J) continue;
      unsigned mr = 0u;
      if (valid) {
        const uint4 w = stg[((st & 1) * RS + r0 + RT * u) * NQ + q];
        const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const unsigned mv = hi_mag(e[v]);
          mr = max(mr, mv);
          colm[v] = max(colm[v], mv);
        }
      }
      mr = __reduce_max_sync(0xffffffffu, mr);
      if (lane == 0) atomicMax(&rmax[i], mr);
    }
  }
  if (valid)
#pragma unroll
    for (int v = 0; v < V; ++v) atomicMax(&cmax[V * q + v], colm[v]);
  __syncthreads();
  if (colexp)
    for (int cc = tid; cc < ncols; cc += 512) {
      int64_t l, b;
      if (chunk_col(cc / V, l, b)) colexp[l + cc % V + L * b] = exp_above(mag_pattern(cmax[cc], kF64), kF64);
    }
  unsigned gm = 0u;
  for (int i = tid; i < J; i += 512) {
    E[(int64_t)blockIdx.x * J + i] = table_exp(mag_pattern(rmax[i], kF64), kF64);
    gm = max(gm, rmax[i]);
  }
  gm = __reduce_max_sync(0xffffffffu, gm);
  if (lane == 0 && gm != 0u) atomicMax(gmax, mag_pattern(gm, kF64));
}

// E4M3 variant (kF8): every entry is rounded to v = round(y 2^(15 - E_ig)),
// |v| <= 2^15, and split into four balanced base-16 digits
// v = d1 2^12 + d2 2^8 + d3 2^4 + d4 (|d| <= 8, exact in E4M3, and so are
// 2 d, 16 d and 32 d).  Level L = p + q of a digit product has weight
// 2^(4 (8 - L)); with only the symmetric part of C counting, four
// accumulators hold exact integer sums over a 512-column group:
//   acc0 = 16 L2 + L3 = D1 (16 D1)^T + D1 (2 D2)^T
//   acc1 = 16 L4 + L5 = D1 (32 D3)^T + D2 (16 D2)^T + D1 (2 D4)^T + D2 (2 D3)^T
//   acc2 = 16 L6 + L7 = D2 (32 D4)^T + D3 (16 D3)^T + D3 (2 D4)^T
//   acc3 = L8         = D4 D4^T
// (per column at most 1152, 3328, 3200 and 64: far below 2^24 over a group),
// drained with weights 2^20, 2^12, 2^4, 2^0, so that S = (C + C^T) 2^(E_i +
// E_j - 31).  The B operands lie as stacked pairs [16 D1; 32 D3], [2 D2; 2 D4],
// [16 D2; 32 D4] (N = 256), then 2 D3, 16 D3, and the A operands D1..D4
// (D4 is also the B operand of acc3): seven MMAs of K = 32 per chunk.
constexpr int kF8Tiles = 12;
constexpr int kF8TileBytes = kRows * kChunk;      // 128 rows x 32 one-byte digits
constexpr int kF8Sbo = kChunk / 16 * 128;         // two 16-byte core matrices per 8-row group
constexpr int kF8StageBytes = kF8Tiles * kF8TileBytes;
constexpr uint32_t kIdescF8 = idesc_e4m3(kRows, kRows);
constexpr uint32_t kIdescF8x256 = idesc_e4m3(kRows, 2 * kRows);

// Two floats holding small integers (|x| <= 448) as E4M3 bytes: a in the low byte.
__device__ __forceinline__ uint32_t e4m3_pair(float a, float b) {
  unsigned short d;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(b), "f"(a));
  return d;
}

template <typename T, int kMode, bool kF8>
__global__ void __launch_bounds__(kThreads, 1) k_gram_split(const T *__restrict__ y, int64_t L, SplitPlan p,
                                                            const int *__restrict__ Etab,
                                                            int *__restrict__ refs, double *__restrict__ ws,
                                                            int *__restrict__ err) {
  constexpr int kStage = kF8 ? kF8StageBytes : kStageBytes;
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long mbar[kStages];
  __shared__ int rowexp[kRows];
  __shared__ int ref[kRows];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  unsigned char *stage_base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  // double-float accumulators of C, element e of thread t at [e][t]
  float2 *cacc = reinterpret_cast<float2 *>(stage_base + kStages * kStage);

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

  const int64_t c_begin = (int64_t)blockIdx.x * p.cols_per_split;
  const int64_t c_end = min(p.K, c_begin + p.cols_per_split);
  const int nchunks = (int)((c_end - c_begin + kChunk - 1) / kChunk);
  const int64_t stride_b = L * (int64_t)p.J;
  cta_row_ref(Etab, p.J, c_begin / kGroup, (c_end + kGroup - 1) / kGroup, ref, refs + blockIdx.x * kRows);

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
    if (in_group == 0) my_e1022 = rowexp[row] + 1022 + (kF8 ? 6 : 0);  // 15 bits: round(y 2^(21 - (E + 6)))
    unsigned char *st = stage_base + buf * kStage;
    if constexpr (kF8) {
      // tiles: 0 16D1, 1 32D3, 2 2D2, 3 2D4, 4 16D2, 5 32D4, 6 2D3, 7 16D3, 8 D1, 9 D2, 10 D3, 11 D4
      uint32_t w[kF8Tiles][2];
#pragma unroll
      for (int k = 0; k < 8; k += 4) {
        float d[4][4];  // [column][digit]
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float v = small_int_float(scaled_int21(raw[k + h], my_e1022));
          const float d1 = round_float(v * 0x1p-12f);
          const float r1 = __fmaf_rn(d1, -4096.0f, v);
          const float d2 = round_float(r1 * 0x1p-8f);
          const float r2 = __fmaf_rn(d2, -256.0f, r1);
          const float d3 = round_float(r2 * 0x1p-4f);
          d[h][0] = d1;
          d[h][1] = d2;
          d[h][2] = d3;
          d[h][3] = __fmaf_rn(d3, -16.0f, r2);
        }
        const float sc[kF8Tiles] = {16.f, 32.f, 2.f, 2.f, 16.f, 32.f, 2.f, 16.f, 1.f, 1.f, 1.f, 1.f};
        const int dig[kF8Tiles] = {0, 2, 1, 3, 1, 3, 2, 2, 0, 1, 2, 3};
#pragma unroll
        for (int t = 0; t < kF8Tiles; ++t)
          w[t][k >> 2] = e4m3_pair(d[0][dig[t]] * sc[t], d[1][dig[t]] * sc[t]) |
                         (e4m3_pair(d[2][dig[t]] * sc[t], d[3][dig[t]] * sc[t]) << 16);
      }
      const int off = (row >> 3) * kF8Sbo + (kg >> 1) * 128 + (row & 7) * 16 + (kg & 1) * 8;
#pragma unroll
      for (int t = 0; t < kF8Tiles; ++t)
        *reinterpret_cast<uint2 *>(st + t * kF8TileBytes + off) = make_uint2(w[t][0], w[t][1]);
    } else {
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
    if (kF8 && tid == 0) {
      fence_after();
      const uint32_t base = smem_addr(st);
      const uint32_t acc = in_group == 0 ? 0u : 1u;
      auto dsc = [&](int t) { return smem_desc(base + t * kF8TileBytes, 128, kF8Sbo); };
      // each accumulator's first MMA of a group carries `acc` (0: overwrite)
      mma_f8(tmem + 0, dsc(8), dsc(0), kIdescF8x256, acc);    // acc0 (+)= D1 16D1, acc1 (+)= D1 32D3
      mma_f8(tmem + 0, dsc(8), dsc(2), kIdescF8x256, 1u);     // acc0 += D1 2D2,    acc1 += D1 2D4
      mma_f8(tmem + 256, dsc(10), dsc(7), kIdescF8, acc);     // acc2 (+)= D3 16D3
      mma_f8(tmem + 128, dsc(9), dsc(4), kIdescF8x256, 1u);   // acc1 += D2 16D2,   acc2 += D2 32D4
      mma_f8(tmem + 128, dsc(9), dsc(6), kIdescF8, 1u);       // acc1 += D2 2D3
      mma_f8(tmem + 256, dsc(10), dsc(3), kIdescF8, 1u);      // acc2 += D3 2D4
      mma_f8(tmem + 384, dsc(11), dsc(11), kIdescF8, acc);    // acc3 (+)= D4 D4
      mma_commit(smem_addr(&mbar[buf]));
    } else if (tid == 0) {
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
        // bf16: 2^28, 2 2^21, 2^14, 2^7; e4m3: 2^20, 2^12, 2^4, 2^0
        const float wts[4] = {kF8 ? 0x1p20f : 0x1p28f, kF8 ? 0x1p12f : 0x1p22f, kF8 ? 0x1p4f : 0x1p14f,
                              kF8 ? 1.0f : 0x1p7f};
        const int ei = rowexp[drow] - ref[drow];
#pragma unroll
        for (int part = 0; part < 4; ++part) {
          float sc[8], hi[8], lo[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int x = ei + rowexp[32 * cb + 8 * part + e] - ref[32 * cb + 8 * part + e];  // <= 0
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
  // per-CTA C (not yet symmetrised) as double-float pairs, row-major 128 x 128
  float2 *dst = reinterpret_cast<float2 *>(ws) + (size_t)blockIdx.x * kRows * kRows + (size_t)drow * kRows + 32 * cb;
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) dst[e] = cacc[e * kThreads + tid];
}

// ---------------------------------------------------------------------------
// L == 1 with 16-byte column strides (J sizeof(T) a multiple of 16, Y 16-byte
// aligned): the unfolding is a 2-D tensor of K columns of J contiguous
// entries.  The tensor-memory accelerator copies each chunk as one 128 x 32
// box (cp.async.bulk.tensor; rows >= J and columns >= K arrive as zeros) into
// a ring of kRing shared-memory slots, completion counted in bytes on the
// slot's mbarrier: the loads in flight are not bounded by registers, every
// shared load of the conversion has a constant offset and the ragged edges
// need no predicates.  The 16 warps form two groups of eight that convert
// alternate chunks into their own digit stage; a group's leader refills the
// slot its group has read and issues the chunk's MMAs once the other group's
// previous chunk has completed (one in-order accumulator stream).
// A thread converts row t % 128 and 16 columns (t / 128 of the halves, t the
// index within its group) of its group's chunks from shared memory:
//   * f = |y| 2^(21 - E) is built as a float straight from the bits (the
//     exponent field rebased by one integer subtraction clamped at zero, the
//     significand cut to 24 bits with the last bit set, i.e. rounded to odd,
//     so that rounding f to an integer is the correct rounding of y 2^(21-E),
//     ties away from zero);
//   * digits s1 = rn(f 2^-14), s2 = rn((f - 2^14 s1) 2^-7), s3 = rn(rest) by
//     magic-number rounding, packed to BF16 pairs; 2 s3 and s3 / 256 are
//     exact BF16 pair products of the packed s3.
// The digit tiles A1, A2, 2 A3, A3 / 256 lie back to back with one
// row-group stride, so [A1; A2] and [A2; 2 A3] are N = 256 operands and a
// K-step takes four MMAs:
//   D[0, 256)   = A1 [A1; A2]^T           (acc0, acc1)
//   D[256, 512) = A2 [A2; 2 A3]^T         (acc2 part, acc3 part)
//   D[256, 384) += A1 (2 A3)^T            (acc2)
//   D[384, 512) += (2 A3) (A3 / 256)^T    (acc3)
// At a group's end each thread folds its 32 entries into double-float
// registers: the exact levels are merged into p 2^28 + r 2^7 with p an exact
// integer below 2^24 (digit carries moved up by magic-number rounding), so
// one TwoSum per entry and group replaces one per level.
// ---------------------------------------------------------------------------
constexpr int kRing = 4;                                  // raw slots
constexpr int kRawBytes = kChunk * kRows * 8;             // one slot: 32 columns of J <= 128 entries
constexpr size_t kBulkSmemBytes = (size_t)kRing * kRawBytes + (size_t)kStages * kStageBytes + 1024;
constexpr uint32_t kIdesc256 = idesc_bf16(kRows, 2 * kRows);
constexpr float kMagic = 12582912.0f;                     // 1.5 2^23: adding it rounds |x| < 2^22 to an integer

// f = |y| 2^(21 - E) with the sign of y, rounded to odd at 24 bits (see above).
// cvt = (E + 875) << 20, or 2047 << 20 for an all-zero row (every entry then
// gives |f| < 2^-126).  Entries below 2^(E - 23) give |f| < 1/4.
__device__ __forceinline__ float scaled_float(double y, int cvt) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int x = max((int)(hi & 0x7FFFFFFFu) - cvt, 0);
  return __uint_as_float(__funnelshift_l(lo, (unsigned)x, 3) | 1u | (hi & 0x80000000u));
}
// float: cvt = (21 - E) << 23, or -(255 << 23) for an all-zero row; values
// that would fall below 1/16 become 1/16 (then rounded to 0).
__device__ __forceinline__ float scaled_float(float y, int cvt) {
  const unsigned b = __float_as_uint(y);
  const int x = max((int)(b & 0x7FFFFFFFu) + cvt, 0x3D800000);
  return __uint_as_float((unsigned)x | 1u | (b & 0x80000000u));
}
template <typename T>
__device__ __forceinline__ int scaled_float_param(int e) {
  if constexpr (sizeof(T) == 8) return e == kZeroExp ? (2047 << 20) : (e + 875) << 20;
  else return e == kZeroExp ? -(255 << 23) : (21 - e) << 23;
}

// balanced digits of rn(f): f - rn(f) = r - s3 exactly, |s1| <= 128, |s2|, |s3| <= 64
__device__ __forceinline__ void split3(float f, float &s1, float &s2, float &s3) {
  s1 = __fsub_rn(__fmaf_rn(f, 0x1p-14f, kMagic), kMagic);
  const float r1 = __fmaf_rn(s1, -16384.0f, f);
  s2 = __fsub_rn(__fmaf_rn(r1, 0x1p-7f, kMagic), kMagic);
  const float r2 = __fmaf_rn(s2, -128.0f, r1);
  s3 = __fsub_rn(__fadd_rn(r2, kMagic), kMagic);
}

__device__ __forceinline__ uint32_t bf16x2_mul(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Row `row`, columns 8 kg .. 8 kg + 7 of the chunk in `raw` (column c of row
// i at raw[c 128 + i]) as digits into the four tiles at st.
template <typename T>
__device__ __forceinline__ void convert_bulk(const T *raw, int row, int kg, int cvt, unsigned char *st) {
  uint32_t w[kTiles][4];
  const T *src = raw + row + 8 * kg * kRows;
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    float a1, a2, a3, b1, b2, b3;
    split3(scaled_float(src[k * kRows], cvt), a1, a2, a3);
    split3(scaled_float(src[(k + 1) * kRows], cvt), b1, b2, b3);
    const uint32_t p3 = bf16_pair(a3, b3);
    w[0][k >> 1] = bf16_pair(a1, b1);
    w[1][k >> 1] = bf16_pair(a2, b2);
    w[2][k >> 1] = bf16x2_mul(p3, 0x40004000u);  // 2 s3
    w[3][k >> 1] = bf16x2_mul(p3, 0x3B803B80u);  // s3 / 256
  }
  const int off = (row >> 3) * kSbo + kg * 128 + (row & 7) * 16;
#pragma unroll
  for (int t = 0; t < kTiles; ++t)
    *reinterpret_cast<uint4 *>(st + t * kTileBytes + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// (H, Lo) += (2^28 a0 + 2^22 a1 + 2^14 a2 + 2^7 a3) 2^x with sc28 = 2^(28 + x).
// a0, a1, a2 are exact integers (|a0| <= 2^23, |a1| <= 2^22, |a2| < 10.5e6):
// a1 = 64 a1h + a1l and 256 a1l + a2 = 2^14 qh + ql move their high parts
// into p2 = a0 + a1h + qh (exact, < 2^24); r = 128 ql + a3 is the one rounded
// step (its error is ~2^-45 of the group's largest term).
__device__ __forceinline__ void drain_entry(float a0, float a1, float a2, float a3, float sc28, float &H,
                                            float &Lo) {
  const float a1h = __fsub_rn(__fmaf_rn(a1, 0x1p-6f, kMagic), kMagic);
  const float a1l = __fmaf_rn(a1h, -64.0f, a1);
  const float q = __fmaf_rn(a1l, 256.0f, a2);
  const float qh = __fsub_rn(__fmaf_rn(q, 0x1p-14f, kMagic), kMagic);
  const float ql = __fmaf_rn(qh, -16384.0f, q);
  const float p2 = __fadd_rn(__fadd_rn(a0, a1h), qh);
  const float r = __fmaf_rn(ql, 128.0f, a3);
  const float hg = __fmul_rn(p2, sc28);
  const float lg = __fmul_rn(r, __fmul_rn(sc28, 0x1p-21f));
  const float s = __fadd_rn(H, hg);  // TwoSum(H, hg)
  const float bp = __fsub_rn(s, H);
  const float e = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bp)), __fsub_rn(hg, bp));
  const float l = __fadd_rn(Lo, __fadd_rn(e, lg));
  const float t = __fadd_rn(s, l);  // renormalise
  Lo = __fsub_rn(l, __fsub_rn(t, s));
  H = t;
}

// four 32-lane x 4-column TMEM loads (the four levels of 4 entries), then the wait
__device__ __forceinline__ void tmem_ld4x4(uint32_t taddr, uint32_t (&r)[4][4]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%17];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%18];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%19];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]),
        "=r"(r[1][3]), "=r"(r[2][0]), "=r"(r[2][1]), "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[3][0]), "=r"(r[3][1]),
        "=r"(r[3][2]), "=r"(r[3][3])
      : "r"(taddr), "r"(taddr + 128), "r"(taddr + 256), "r"(taddr + 384)
      : "memory");
}

// Row `row`, chunk columns of b offset kg (8 consecutive l) from a box
// {8 l, 128 rows, 4 b} stored with the 64-byte swizzle: the 16-byte piece u of
// line (kg 128 + row) sits at piece u ^ ((row >> 1) & 3), so each quarter-warp's
// 16-byte loads hit eight distinct bank groups.
__device__ __forceinline__ void convert_oct(const unsigned char *raw, int row, int kg, int cvt, unsigned char *st) {
  uint32_t w[kTiles][4];
  const unsigned char *line = raw + (kg * kRows + row) * 64;
  const int sw = (row >> 1) & 3;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 y2 = *reinterpret_cast<const double2 *>(line + ((u ^ sw) << 4));
    float a1, a2, a3, b1, b2, b3;
    split3(scaled_float(y2.x, cvt), a1, a2, a3);
    split3(scaled_float(y2.y, cvt), b1, b2, b3);
    const uint32_t p3 = bf16_pair(a3, b3);
    w[0][u] = bf16_pair(a1, b1);
    w[1][u] = bf16_pair(a2, b2);
    w[2][u] = bf16x2_mul(p3, 0x40004000u);
    w[3][u] = bf16x2_mul(p3, 0x3B803B80u);
  }
  const int off = (row >> 3) * kSbo + kg * 128 + (row & 7) * 16;
#pragma unroll
  for (int t = 0; t < kTiles; ++t)
    *reinterpret_cast<uint4 *>(st + t * kTileBytes + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

template <typename T, bool kOct>
__global__ void __launch_bounds__(kThreads, 1) k_gram_split_bulk(const __grid_constant__ CUtensorMap ymap, SplitPlan p,
                                                                 const int *__restrict__ Etab,
                                                                 int *__restrict__ refs, double *__restrict__ ws,
                                                                 int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long raw_full[kRing];
  __shared__ __align__(8) unsigned long long mma_done[kStages];
  __shared__ __align__(16) int rowexp[2][kRows];  // E_ig of the current and the next group
  __shared__ __align__(16) int relexp[2][kRows];  // E_ig - ref_i
  __shared__ int ref[kRows];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  __shared__ int n_issued;  // copies issued so far (the group leaders, atomically)
  // offsets from dsmem keep the shared address space visible (shared loads and stores)
  unsigned char *ring = dsmem + ((1024u - (smem_addr(dsmem) & 1023u)) & 1023u);
  unsigned char *stages = ring + kRing * kRawBytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int J = p.J;
  // CTA = (column range, diagonal block of 128 rows r0 ..): J > 128 has p.nrb blocks
  const int rb = (int)(blockIdx.x % (unsigned)p.nrb);
  const int r0 = kRows * rb, Jb = min(kRows, J - r0);
  const int64_t c_begin = (int64_t)(blockIdx.x / (unsigned)p.nrb) * p.cols_per_split;
  const int64_t c_end = min(p.K, c_begin + p.cols_per_split);
  const int nchunks = (int)((c_end - c_begin + kChunk - 1) / kChunk);
  const int64_t g0 = c_begin / kGroup;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kRing; ++s) mbar_init(smem_addr(&raw_full[s]), 1);
    for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&mma_done[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
    n_issued = 0;
  }
  cta_row_ref(Etab, J, r0, Jb, g0, (c_end + kGroup - 1) / kGroup, ref, refs + blockIdx.x * kRows);
  // exponents of column group gi go to buffer gi & 1 (threads < kRows, one
  // row each); the next group's are loaded at a group's start into a
  // register and stored at its drain, so no thread waits on the load
  auto fetch_exp = [&](int gi) -> int { return tid < Jb ? Etab[(g0 + gi) * J + r0 + tid] : kZeroExp; };
  auto store_exp = [&](int gi, int e) {
    rowexp[gi & 1][tid] = e;
    relexp[gi & 1][tid] = e - ref[tid];
  };
  if (tid < kRows) store_exp(0, fetch_exp(0));
  int next_exp = 0;        // threads < kRows: the next group's exponent, in flight
  bool next_pending = false;
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  // chunk ch -> slot ch % kRing as the box at (row 0, column c_begin + 32 ch)
  // (thread 0 for the first ring, then the leader of the group that converts
  // the chunk the slot held)
  auto issue_copy = [&](int ch) {
    const int slot = ch % kRing;
    const uint32_t bar = smem_addr(&raw_full[slot]);
    mbar_expect_tx(bar, (uint32_t)(kChunk * kRows * sizeof(T)));
    if (kOct) {  // chunk indices stay below 2^31 (the plan checks it): 32-bit division
      const uint32_t gch = (uint32_t)(c_begin / kChunk) + (uint32_t)ch, nL = (uint32_t)p.nL, bb = gch / nL;
      tma_load_4d(smem_addr(ring + slot * kRawBytes), &ymap, 0, r0, (int)((uint32_t)p.nl * (gch - bb * nL)),
                  (int)((uint32_t)p.nb * bb), bar);
    } else {
      tma_load_2d(smem_addr(ring + slot * kRawBytes), &ymap, r0, (int)(c_begin + (int64_t)ch * kChunk), bar);
    }
  };
  if (tid == 0) {
    int c = 0;
    for (; c < kRing && c < nchunks; ++c) issue_copy(c);
    atomicMax(&n_issued, c);  // the leaders raise it too; read on the error path
  }

  // converter role: two groups of 8 warps take alternate chunks (group grp the
  // chunks with ch & 1 == grp, into digit stage grp); thread (row, 16-column
  // half kh of the chunk); gtid == 0 is the group's leader
  const int grp = warp >> 3, gtid = tid & 255;
  const int row = gtid & (kRows - 1), kh = gtid >> 7;
  const int q = warp & 3, cb = warp >> 2;                  // drain role: TMEM lanes 32 q.., columns 32 cb..
  const int drow = 32 * q + lane;
  const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cb);
  float H[kAccPerThread], Lo[kAccPerThread];
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) H[e] = Lo[e] = 0.f;

  bool bad = false;   // this thread met a failed (expired) wait
  bool halt = false;  // some thread did: every thread stops at the same drain barrier
  // fold the group's four levels into the double-float registers (warp-uniform `ok`)
  // every MMA up to chunk `last` complete: chunk c's commit completes phase
  // c >> 1 of mma_done[c & 1].  A thread waits first on its own group's stage
  // (whose every phase it has waited on in turn) for its group's last chunk,
  // which implies all earlier chunks (a leader issues only after the previous
  // chunk completed), so the other stage's barrier is at most one phase
  // behind the one awaited next.
  auto all_done = [&](int last) -> bool {
    if (bad) return false;
    const int mine = (last & 1) == grp ? last : last - 1;
    if (mine >= 0 && !mbar_wait(smem_addr(&mma_done[mine & 1]), (uint32_t)(mine >> 1) & 1u)) return false;
    if (mine != last && !mbar_wait(smem_addr(&mma_done[last & 1]), (uint32_t)(last >> 1) & 1u)) return false;
    return true;
  };
  auto drain = [&](int gi, bool ok) {
    if (ok) {  // warp-uniform, so the .sync.aligned loads below never diverge
      fence_after();
      const int xi = relexp[gi & 1][drow] + 155;  // exponent field of 2^(28 + E_ig - ref_i)
#pragma unroll
      for (int part = 0; part < 8; ++part) {
        uint32_t r[4][4];
        tmem_ld4x4(taddr + 4 * part, r);
        const int4 ej = *reinterpret_cast<const int4 *>(&relexp[gi & 1][32 * cb + 4 * part]);
        const int ejs[4] = {ej.x, ej.y, ej.z, ej.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float sc28 = __int_as_float(max(xi + ejs[e], 0) << 23);
          drain_entry(__uint_as_float(r[0][e]), __uint_as_float(r[1][e]), __uint_as_float(r[2][e]),
                      __uint_as_float(r[3][e]), sc28, H[4 * part + e], Lo[4 * part + e]);
        }
      }
    } else {
      bad = true;
    }
    if (next_pending) {  // the other buffer, read only after the barrier below
      store_exp(gi + 1, next_exp);
      next_pending = false;
    }
    fence_before();
    // the column group's one block barrier; a failed wait anywhere stops every thread here
    if (__syncthreads_or(bad ? 1 : 0)) halt = true;
  };

  // Chunks go four at a time (the ring depth), so slot, stage and every
  // mbarrier parity below are compile-time constants: chunk ch0 + u uses slot
  // u, digit stage u & 1 (converter group u & 1), the ring phase (ch0 / 4) & 1
  // and, for the stage, commit number (ch0 + u) >> 1 (parity (u >> 1) & 1, as
  // ch0 / 2 is even).  A group converts its chunk, meets at its own named
  // barrier, and its leader waits for the other group's previous chunk's MMAs
  // (so the MMAs stay in chunk order in one accumulator stream), refills the
  // slot and issues the chunk's MMAs; meanwhile the other group converts the
  // next chunk.  The one block barrier is the drain's, once per 512-column
  // group (16 chunks: a column group starts only at u == 0 and ends at u == 3,
  // or at the last chunk, drained after the loop).  After a failed wait a
  // thread skips its work but keeps its barriers, so every thread reaches
  // every drain barrier; the failure stops all of them there.
  int cvt = 0, last_committed = -1;
  bool tail_drain = false;
  for (int ch0 = 0; ch0 < nchunks && !halt; ch0 += kRing) {
    const uint32_t ring_par = (uint32_t)(ch0 / kRing) & 1u;
#pragma unroll
    for (int u = 0; u < kRing; ++u) {
      const int ch = ch0 + u;
      if (ch >= nchunks) break;
      const int in_group = ch % kDrainChunks, gi = ch / kDrainChunks;
      if (u == 0 && in_group == 0) {
        cvt = scaled_float_param<T>(rowexp[gi & 1][row]);
        // the next column group's exponents go to the other buffer at this group's drain
        if (tid < kRows && ch + kDrainChunks < nchunks) {
          next_exp = fetch_exp(gi + 1);
          next_pending = true;
        }
      }
      if ((u & 1) == grp) {
        if (!bad) bad = !mbar_wait(smem_addr(&raw_full[u]), ring_par);
        if (!bad && ch >= 2) bad = !mbar_wait(smem_addr(&mma_done[u & 1]), (uint32_t)(((u + 2) >> 1) & 1));
        if (!bad) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int kg = 2 * kh + h;
            if constexpr (kOct) convert_oct(ring + u * kRawBytes, row, kg, cvt, stages + (u & 1) * kStageBytes);
            else convert_bulk<T>(reinterpret_cast<const T *>(ring + u * kRawBytes), row, kg, cvt, stages + (u & 1) * kStageBytes);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("bar.sync %0, 256;" ::"r"(1 + grp) : "memory");
        if (gtid == 0 && !bad) {
          // the other group's chunk ch - 1 goes first in the accumulators
          if (ch >= 1) bad = !mbar_wait(smem_addr(&mma_done[(u + 1) & 1]), (uint32_t)(((u + 3) >> 1) & 1));
          if (!bad) {
            if (ch + kRing < nchunks) {  // slot u has been read by this group
              issue_copy(ch + kRing);
              atomicMax(&n_issued, ch + kRing + 1);
            }
            fence_after();
            const uint32_t base = smem_addr(stages + (u & 1) * kStageBytes);
#pragma unroll
            for (int k = 0; k < kChunk / 16; ++k) {
              const uint32_t acc = (u == 0 && in_group == 0 && k == 0) ? 0u : 1u;
              const uint64_t a1 = smem_desc(base + 0 * kTileBytes + 256 * k, 128, kSbo);
              const uint64_t a2 = smem_desc(base + 1 * kTileBytes + 256 * k, 128, kSbo);
              const uint64_t a3x2 = smem_desc(base + 2 * kTileBytes + 256 * k, 128, kSbo);
              const uint64_t a3q = smem_desc(base + 3 * kTileBytes + 256 * k, 128, kSbo);
              mma_bf16(tmem + 0, a1, a1, kIdesc256, acc);
              mma_bf16(tmem + 256, a2, a2, kIdesc256, acc);
              mma_bf16(tmem + 256, a1, a3x2, kIdesc, 1u);
              mma_bf16(tmem + 384, a3x2, a3q, kIdesc, 1u);
            }
            mma_commit(smem_addr(&mma_done[u & 1]));
            last_committed = ch;
          }
        }
      }
      if (u == kRing - 1 && in_group == kDrainChunks - 1) {
        drain(gi, __all_sync(0xffffffffu, all_done(ch)));
        if (halt) break;
      } else if (ch == nchunks - 1) {
        tail_drain = true;
      }
    }
  }
  if (tail_drain && !halt) {
    const int ch = nchunks - 1;
    drain(ch / kDrainChunks, __all_sync(0xffffffffu, all_done(ch)));
  }
  if (halt && tid == 0) stop = 1;
  __syncthreads();
  if (stop && gtid == 0 && last_committed >= 0)  // each leader: its own MMAs finish before TMEM goes
    mbar_wait(smem_addr(&mma_done[last_committed & 1]), (uint32_t)(last_committed >> 1) & 1u);
  if (stop && tid == 0) {
    // let the bulk copies finish (bounded) before shared memory goes
    const int issued = n_issued;
    for (int c = max(0, issued - kRing); c < issued; ++c)
      mbar_wait(smem_addr(&raw_full[c % kRing]), (uint32_t)(c / kRing) & 1u);
  }
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
  // per-CTA C (not yet symmetrised) as double-float pairs, row-major 128 x 128
  float2 *dst = reinterpret_cast<float2 *>(ws) + (size_t)blockIdx.x * kRows * kRows + (size_t)drow * kRows + 32 * cb;
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) dst[e] = make_float2(H[e], Lo[e]);
}

// ---------------------------------------------------------------------------
// Off-diagonal blocks for 128 < J <= 512: S_ab = Y_a Y_b^T for row blocks a <
// b of 128 rows (the diagonal blocks are k_gram_split_bulk's, with a row
// offset).  A CTA takes one block pair and a column range and streams it in
// half-chunks of 16 columns: two tensor-map boxes per half (the rows of
// block a and of block b), a ring of kPRing slots, two digit stages.  The
// tiled (kOct) path splits each 32-column chunk of the exponent pass into
// its two halves (16 of its 32 columns: the same groups, so the same
// exponents).  The digits are those of the diagonal kernel (21 bits below
// each (row, group) power of two, three balanced digits), but no symmetry
// folds the levels, so four accumulators hold
//   acc0 = A1 B1^T                       (level 2, weight 2^28)
//   acc1 = A1 B2^T + A2 B1^T             (level 3, 2^21)
//   acc2 = A1 B3^T + A2 B2^T + A3 B1^T   (level 4, 2^14)
//   acc3 = A2 B3^T + A3 B2^T + A3 (B3 / 128)^T   (levels 5 and 6, 2^7)
// from six MMAs per half: A1, A2 and A3 against the stacked [B1; B2] (N =
// 256: two levels each) and A1, A2, A3 against B3, B3 and B3 / 128.  Per
// 512-column group acc0, acc1 <= 2^23 and acc2 < 10.5e6 are exact integer
// sums; acc3's level-6 part is rounded as in the diagonal kernel.  The
// partial is C itself (S_ab = sum over CTAs of C 2^(ref_a + ref_b - 42)).
// ---------------------------------------------------------------------------
constexpr int kPH = 16;                                   // columns per half-chunk
constexpr int kPTile = kRows * kPH * 2;                   // one BF16 digit tile: 128 rows x 16 columns
constexpr int kPSbo = kPH / 8 * 128;                      // bytes between 8-row core-matrix groups
constexpr int kPStage = 7 * kPTile;                       // B1, B2, B3, B3/128, A1, A2, A3
constexpr int kPRawBox = kRows * kPH * 8;                 // one box (sized for float64)
constexpr int kPSlot = 2 * kPRawBox;                      // the two blocks' boxes
constexpr int kPRing = 4;
constexpr int kPGroupHalves = kGroup / kPH;               // 32
constexpr size_t kPairSmemBytes = (size_t)kPRing * kPSlot + (size_t)kStages * kPStage + 1024;

// (H, Lo) += (2^28 a0 + 2^21 a1 + 2^14 a2 + 2^7 a3) 2^x with sc28 = 2^(28 + x)
// for an off-diagonal block: a1 = 128 a1h + a1l and 128 a1l + a2 = 2^14 qh + ql
// move the high parts into p2 = a0 + a1h + qh (exact, < 2^24); r = 128 ql + a3
// is the one rounded step.
__device__ __forceinline__ void drain_entry_off(float a0, float a1, float a2, float a3, float sc28, float &H,
                                                float &Lo) {
  const float a1h = __fsub_rn(__fmaf_rn(a1, 0x1p-7f, kMagic), kMagic);
  const float a1l = __fmaf_rn(a1h, -128.0f, a1);
  const float q = __fmaf_rn(a1l, 128.0f, a2);
  const float qh = __fsub_rn(__fmaf_rn(q, 0x1p-14f, kMagic), kMagic);
  const float ql = __fmaf_rn(qh, -16384.0f, q);
  const float p2 = __fadd_rn(__fadd_rn(a0, a1h), qh);
  const float r = __fmaf_rn(ql, 128.0f, a3);
  const float hg = __fmul_rn(p2, sc28);
  const float lg = __fmul_rn(r, __fmul_rn(sc28, 0x1p-21f));
  const float s = __fadd_rn(H, hg);  // TwoSum(H, hg)
  const float bp = __fsub_rn(s, H);
  const float e = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bp)), __fsub_rn(hg, bp));
  const float l = __fadd_rn(Lo, __fadd_rn(e, lg));
  const float t = __fadd_rn(s, l);  // renormalise
  Lo = __fsub_rn(l, __fsub_rn(t, s));
  H = t;
}

// The three digits (s1, s2, s3) of 8 columns of one row as BF16 pairs: from a
// 128 x kPH box of a 2-D map (column c of row i at raw[c 128 + i]) ...
template <typename T>
__device__ __forceinline__ void digits8_box(const T *raw, int row, int kg, int cvt, uint32_t (&w)[3][4]) {
  const T *src = raw + row + 8 * kg * kRows;
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    float a1, a2, a3, b1, b2, b3;
    split3(scaled_float(src[k * kRows], cvt), a1, a2, a3);
    split3(scaled_float(src[(k + 1) * kRows], cvt), b1, b2, b3);
    w[0][k >> 1] = bf16_pair(a1, b1);
    w[1][k >> 1] = bf16_pair(a2, b2);
    w[2][k >> 1] = bf16_pair(a3, b3);
  }
}
// ... or from line kg of a 64-byte swizzled box of 8 l per line (as convert_oct).
__device__ __forceinline__ void digits8_oct(const unsigned char *raw, int row, int kg, int cvt, uint32_t (&w)[3][4]) {
  const unsigned char *line = raw + (kg * kRows + row) * 64;
  const int sw = (row >> 1) & 3;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 y2 = *reinterpret_cast<const double2 *>(line + ((u ^ sw) << 4));
    float a1, a2, a3, b1, b2, b3;
    split3(scaled_float(y2.x, cvt), a1, a2, a3);
    split3(scaled_float(y2.y, cvt), b1, b2, b3);
    w[0][u] = bf16_pair(a1, b1);
    w[1][u] = bf16_pair(a2, b2);
    w[2][u] = bf16_pair(a3, b3);
  }
}

template <typename T, bool kOct>
__global__ void __launch_bounds__(kThreads, 1) k_gram_split_pair(const __grid_constant__ CUtensorMap ymap, SplitPlan p,
                                                                 const int *__restrict__ Etab,
                                                                 int *__restrict__ refs, double *__restrict__ ws,
                                                                 int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long raw_full[kPRing];
  __shared__ __align__(8) unsigned long long mma_done[kStages];
  __shared__ __align__(16) int rowexp[2][2][kRows];  // [group buffer][block a, b][row]: E_ig
  __shared__ __align__(16) int relexp[2][2][kRows];  // E_ig - ref_i
  __shared__ int ref[2][kRows];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  __shared__ int n_issued;
  unsigned char *ring = dsmem + ((1024u - (smem_addr(dsmem) & 1023u)) & 1023u);
  unsigned char *stages = ring + kPRing * kPSlot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int J = p.J;
  int pi = (int)(blockIdx.x % (unsigned)p.npair), ba = 0;
  while (pi >= p.nrb - 1 - ba) {  // pairs (a, b), a < b, in the order (0,1), (0,2), .., (1,2), ..
    pi -= p.nrb - 1 - ba;
    ++ba;
  }
  const int bb = ba + 1 + pi;
  const int rA = kRows * ba, rB = kRows * bb;
  const int JA = min(kRows, J - rA), JB = min(kRows, J - rB);
  const int64_t c_begin = (int64_t)(blockIdx.x / (unsigned)p.npair) * p.cols_per_split;
  const int64_t c_end = min(p.K, c_begin + p.cols_per_split);
  const int nh = 2 * (int)((c_end - c_begin + kChunk - 1) / kChunk);
  const int64_t g0 = c_begin / kGroup;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kPRing; ++s) mbar_init(smem_addr(&raw_full[s]), 1);
    for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&mma_done[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
  }
  const int64_t g1 = (c_end + kGroup - 1) / kGroup;
  cta_row_ref(Etab, J, rA, JA, g0, g1, ref[0], refs + (int64_t)blockIdx.x * 2 * kRows);
  cta_row_ref(Etab, J, rB, JB, g0, g1, ref[1], refs + (int64_t)blockIdx.x * 2 * kRows + kRows);
  auto load_exps = [&](int hc) {  // the group starting at half hc -> buffer (hc / 32) & 1
    if (tid < 2 * kRows) {
      const int gi = hc / kPGroupHalves, side = tid >> 7, i = tid & (kRows - 1);
      const int e = i < (side ? JB : JA) ? Etab[(g0 + gi) * J + (side ? rB : rA) + i] : kZeroExp;
      rowexp[gi & 1][side][i] = e;
      relexp[gi & 1][side][i] = e - ref[side][i];
    }
  };
  load_exps(0);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  // half hc -> slot hc % kPRing: block a's box, then block b's
  auto issue_copy = [&](int hc) {
    const int slot = hc % kPRing;
    const uint32_t bar = smem_addr(&raw_full[slot]);
    const uint32_t dst = smem_addr(ring + slot * kPSlot);
    mbar_expect_tx(bar, (uint32_t)(2 * kPH * kRows * sizeof(T)));
    if (kOct) {
      const uint32_t gch = (uint32_t)(c_begin / kChunk) + (uint32_t)(hc >> 1), h = (uint32_t)(hc & 1);
      const uint32_t nL = (uint32_t)p.nL, bq = gch / nL;
      const int oct = (int)((uint32_t)p.nl * (gch - bq * nL) + (p.nl == 4 ? 2 * h : 0u));
      const int b = (int)((uint32_t)p.nb * bq + (p.nl == 4 ? 0u : h * (uint32_t)(p.nb / 2)));
      tma_load_4d(dst, &ymap, 0, rA, oct, b, bar);
      tma_load_4d(dst + kPRawBox, &ymap, 0, rB, oct, b, bar);
    } else {
      const int col = (int)(c_begin + (int64_t)hc * kPH);
      tma_load_2d(dst, &ymap, rA, col, bar);
      tma_load_2d(dst + kPRawBox, &ymap, rB, col, bar);
    }
  };
  if (tid == 0) {
    int c = 0;
    for (; c < kPRing && c < nh; ++c) issue_copy(c);
    n_issued = c;
  }

  const int side = tid >> 8, row = tid & (kRows - 1), kg = (tid >> 7) & 1;  // converter role
  const int q = warp & 3, cb = warp >> 2;                                    // drain role
  const int drow = 32 * q + lane;
  const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cb);
  float H[kAccPerThread], Lo[kAccPerThread];
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) H[e] = Lo[e] = 0.f;

  auto drain = [&](int gi, bool ok) {
    if (ok) {  // warp-uniform
      fence_after();
      const int xi = relexp[gi & 1][0][drow] + 155;  // exponent field of 2^(28 + E_ia - ref_a)
#pragma unroll
      for (int part = 0; part < 8; ++part) {
        uint32_t r[4][4];
        tmem_ld4x4(taddr + 4 * part, r);
        const int4 ej = *reinterpret_cast<const int4 *>(&relexp[gi & 1][1][32 * cb + 4 * part]);
        const int ejs[4] = {ej.x, ej.y, ej.z, ej.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float sc28 = __int_as_float(max(xi + ejs[e], 0) << 23);
          drain_entry_off(__uint_as_float(r[0][e]), __uint_as_float(r[1][e]), __uint_as_float(r[2][e]),
                          __uint_as_float(r[3][e]), sc28, H[4 * part + e], Lo[4 * part + e]);
        }
      }
    } else {
      stop = 1;
    }
    fence_before();
    __syncthreads();
  };

  int cvt = 0, last_committed = -1;
  for (int hc = 0; hc < nh && !stop; ++hc) {
    const int slot = hc % kPRing, st = hc & 1;
    const int in_group = hc % kPGroupHalves, gi = hc / kPGroupHalves;
    if (in_group == 0) {
      cvt = scaled_float_param<T>(rowexp[gi & 1][side][row]);
      if (hc + kPGroupHalves < nh) load_exps(hc + kPGroupHalves);  // the other buffer, read after later barriers
    }
    bool ok = mbar_wait(smem_addr(&raw_full[slot]), (uint32_t)(hc / kPRing) & 1u);
    if (ok && hc >= 2) ok = mbar_wait(smem_addr(&mma_done[st]), (uint32_t)((hc - 2) >> 1) & 1u);
    if (ok) {
      uint32_t w[3][4];
      const unsigned char *raw = ring + slot * kPSlot + side * kPRawBox;
      if constexpr (kOct) digits8_oct(raw, row, kg, cvt, w);
      else digits8_box<T>(reinterpret_cast<const T *>(raw), row, kg, cvt, w);
      unsigned char *stg = stages + st * kPStage;
      const int off = (row >> 3) * kPSbo + kg * 128 + (row & 7) * 16;
      if (side == 0) {  // A1, A2, A3 at tiles 4, 5, 6
#pragma unroll
        for (int t = 0; t < 3; ++t)
          *reinterpret_cast<uint4 *>(stg + (4 + t) * kPTile + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
      } else {  // B1, B2, B3, B3 / 128 at tiles 0 .. 3
#pragma unroll
        for (int t = 0; t < 3; ++t)
          *reinterpret_cast<uint4 *>(stg + t * kPTile + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
        *reinterpret_cast<uint4 *>(stg + 3 * kPTile + off) =
            make_uint4(bf16x2_mul(w[2][0], 0x3C003C00u), bf16x2_mul(w[2][1], 0x3C003C00u),
                       bf16x2_mul(w[2][2], 0x3C003C00u), bf16x2_mul(w[2][3], 0x3C003C00u));
      }
    } else {
      stop = 1;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (stop) break;
    if (tid == 32 && hc + kPRing < nh) {  // slot `slot` has been read by every thread
      issue_copy(hc + kPRing);
      n_issued = hc + kPRing + 1;
    }
    if (tid == 0) {
      fence_after();
      const uint32_t base = smem_addr(stages + st * kPStage);
      auto dsc = [&](int t) { return smem_desc(base + t * kPTile, 128, kPSbo); };
      const uint32_t acc = in_group == 0 ? 0u : 1u;  // each accumulator's first MMA of a group overwrites
      mma_bf16(tmem + 0, dsc(4), dsc(0), kIdesc256, acc);    // acc0 (+)= A1 B1, acc1 (+)= A1 B2
      mma_bf16(tmem + 256, dsc(4), dsc(2), kIdesc, acc);     // acc2 (+)= A1 B3
      mma_bf16(tmem + 384, dsc(5), dsc(2), kIdesc, acc);     // acc3 (+)= A2 B3
      mma_bf16(tmem + 128, dsc(5), dsc(0), kIdesc256, 1u);   // acc1 += A2 B1, acc2 += A2 B2
      mma_bf16(tmem + 256, dsc(6), dsc(0), kIdesc256, 1u);   // acc2 += A3 B1, acc3 += A3 B2
      mma_bf16(tmem + 384, dsc(6), dsc(3), kIdesc, 1u);      // acc3 += A3 B3 / 128
      mma_commit(smem_addr(&mma_done[st]));
    }
    last_committed = hc;
    if (in_group == kPGroupHalves - 1 || hc == nh - 1) {
      drain(gi, __all_sync(0xffffffffu, mbar_wait(smem_addr(&mma_done[st]), (uint32_t)(hc >> 1) & 1u)));
      if (stop) break;
    }
  }
  if (stop && tid == 0) {
    if (last_committed >= 0) mbar_wait(smem_addr(&mma_done[last_committed & 1]), (uint32_t)(last_committed >> 1) & 1u);
    const int issued = n_issued;
    for (int c = max(0, issued - kPRing); c < issued; ++c)
      mbar_wait(smem_addr(&raw_full[c % kPRing]), (uint32_t)(c / kPRing) & 1u);
  }
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
  float2 *dst = reinterpret_cast<float2 *>(ws) + (size_t)blockIdx.x * kRows * kRows + (size_t)drow * kRows + 32 * cb;
#pragma unroll
  for (int e = 0; e < kAccPerThread; ++e) dst[e] = make_float2(H[e], Lo[e]);
}

// S_ij = sum over CTAs of (C_ij + C_ji) 2^(ref_i + ref_j - off) for i and j in
// one diagonal block of 128 rows (off = 43 for the BF16 digits: 2 x 21 bits
// and the doubled symmetric part), or of C_ab 2^(ref_a + ref_b - off + 1)
// from the block pair's partials (J > 128); NaN throughout when the largest
// magnitude is not finite (Y holds Inf or NaN).  Partials: the diagonal
// CTAs' (split s, block r) at s nrb + r, then the pair CTAs' (split s, pair
// t) at nsd nrb + s npair + t; refs likewise (128 per diagonal CTA, 256 per
// pair CTA: block a's rows, then block b's).  Eight threads per entry take
// every eighth partial and combine by a fixed shuffle tree, so the result is
// the same on every run, and S_ij and S_ji are the same value.
__global__ void __launch_bounds__(256) k_gram_split_reduce(const double *__restrict__ ws, const int *__restrict__ refs,
                                                           int nsd, int nso, int nrb, int npair, int J,
                                                           const unsigned long long *__restrict__ gmax, int is_f64,
                                                           int scale_off, double *__restrict__ S) {
  const int idx = blockIdx.x * (blockDim.x / 8) + (threadIdx.x >> 3), sub = threadIdx.x & 7;
  const bool live = idx < J * J;
  const int i = live ? idx % J : 0, j = live ? idx / J : 0;
  const int bi = i / kRows, bj = j / kRows, ii = i % kRows, jj = j % kRows;
  double s = 0.0;
  if (live && bi == bj) {
    for (int sp = sub; sp < nsd; sp += 8) {
      const int c = sp * nrb + bi;
      const float2 *cp = reinterpret_cast<const float2 *>(ws) + (size_t)c * kRows * kRows;
      const float2 a = cp[ii * kRows + jj], b = cp[jj * kRows + ii];
      const int ri = refs[c * kRows + ii], rj = refs[c * kRows + jj];
      if (ri != kZeroExp && rj != kZeroExp)
        s += ldexp(((double)a.x + (double)a.y) + ((double)b.x + (double)b.y), ri + rj - scale_off);
    }
  } else if (live) {
    const int a = min(bi, bj), b = max(bi, bj);
    const int ia = bi < bj ? ii : jj, jb = bi < bj ? jj : ii;
    const int t = a * nrb - a * (a + 1) / 2 + (b - a - 1);  // pairs (0,1), (0,2), .., (1,2), ..
    const int64_t c0 = (int64_t)nsd * nrb;
    const int *rp = refs + c0 * kRows;
    for (int sp = sub; sp < nso; sp += 8) {
      const int64_t c = (int64_t)sp * npair + t;
      const float2 v = (reinterpret_cast<const float2 *>(ws) + (size_t)(c0 + c) * kRows * kRows)[ia * kRows + jb];
      const int ra = rp[c * 2 * kRows + ia], rb = rp[c * 2 * kRows + kRows + jb];
      if (ra != kZeroExp && rb != kZeroExp) s += ldexp((double)v.x + (double)v.y, ra + rb - scale_off + 1);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (!live || sub != 0) return;
  const unsigned long long gm = *gmax;
  const bool finite = is_f64 ? gm < 0x7FF0000000000000ull : gm < 0x7F800000ull;
  S[i + (int64_t)J * j] = finite ? s : __longlong_as_double(0x7FF8000000000000ll);
}

constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + (size_t)kRows * kRows * sizeof(float2) + 1024;
constexpr size_t kSmemBytesF8 = (size_t)kStages * kF8StageBytes + (size_t)kRows * kRows * sizeof(float2) + 1024;

// oct: the tiled L > 1 path, whose columns are counted as 32 per chunk of
// 8 l x 4 b (a ragged last quad of b reads zeros past B)
SplitPlan split_plan(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, bool oct = false) {
  SplitPlan p{};
  p.J = (int)J;
  p.B = B;
  p.nl = 1;
  p.nb = 4;
  p.nL = 0;
  if (oct) {
    // the chunk shape with the fewest padded columns; among equals, the longest runs of l
    int64_t best = -1;
    for (int nl = 1; nl <= 4; nl *= 2) {
      const int64_t nL = (L / 8 + nl - 1) / nl, nB = (B + 4 / nl - 1) / (4 / nl);
      if (best < 0 || nL * nB <= best) {
        best = nL * nB;
        p.nl = nl;
        p.nb = 4 / nl;
        p.nL = nL;
      }
    }
    p.K = best * kChunk;
  } else {
    p.K = L * B;
  }
  p.ngroups = (p.K + kGroup - 1) / kGroup;
  // about one wave of CTAs for the diagonal blocks (split x block) and one for the pairs
  p.nrb = (int)((J + kRows - 1) / kRows);
  p.npair = p.nrb * (p.nrb - 1) / 2;
  auto splits = [&](int per, int &nsplit, int64_t &cols) {
    const int64_t ns = std::max<int64_t>(1, std::min<int64_t>((dev.sms + per - 1) / per, p.ngroups));
    const int64_t groups_per = (p.ngroups + ns - 1) / ns;
    cols = groups_per * kGroup;
    nsplit = (int)((p.K + cols - 1) / cols);
  };
  splits(p.nrb, p.nsplit, p.cols_per_split);
  if (p.npair > 0) splits(p.npair, p.nsplit_pair, p.cols_per_split_pair);
  return p;
}

// workspace (in doubles): gmax | error flag | (2 spare) | per-CTA partials
// (double-float pairs) | exponent table (ints) | per-CTA row reference
// exponents (ints)
struct SplitWs {
  double *partials;
  int *table;
  int *refs;
  unsigned long long *gmax;
  int *err;
  void *unfolded;  // J > 128 with a layout the tensor maps cannot read: the explicit unfolding
};

// The explicit mode-n unfolding of Y viewed as (L, J, B): out[j + ld c] =
// y[l + L (j + J b)] with c = l + L b (the column order of the exponent
// table's groups), by 32 x 32 tiles through shared memory (reads coalesced
// along l, writes along j).  Block (x, y): x = the tile of l and the b, y =
// the tile of j.
template <typename T>
__global__ void __launch_bounds__(256) k_unfold(const T *__restrict__ y, int64_t L, int J, int64_t B, int64_t ld,
                                                int64_t nlt, T *__restrict__ out) {
  __shared__ T t[32][33];
  const int64_t lt = blockIdx.x % nlt, b = blockIdx.x / nlt;
  const int jt = blockIdx.y, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t l = lt * 32 + tx;
    const int j = jt * 32 + ty + 8 * k;
    t[ty + 8 * k][tx] = (l < L && j < J) ? y[l + L * (j + (int64_t)J * b)] : T(0);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t l = lt * 32 + ty + 8 * k;
    const int j = jt * 32 + tx;
    if (l < L && j < J) out[j + ld * (l + L * b)] = t[tx][ty + 8 * k];
  }
}

// Column stride of the unfolding: J rounded up to 16 bytes.
int64_t unfold_ld(int64_t J, size_t es) {
  const int64_t q = 16 / (int64_t)es;
  return (J + q - 1) / q * q;
}

// True when J > 128 and neither tensor-map path reads Y in place: L == 1 needs
// 16-byte columns, L > 1 float64 with L a multiple of 8.
bool needs_unfold(int64_t L, int64_t J, tucker_dtype dt, const void *y) {
  const size_t es = dt == TUCKER_F64 ? 8 : 4;
  if (J <= kRows) return false;
  const bool aligned = reinterpret_cast<uintptr_t>(y) % 16 == 0;
  if (L == 1) return !((J * (int64_t)es) % 16 == 0 && aligned);
  return !(dt == TUCKER_F64 && L % 8 == 0 && aligned);
}

int64_t split_ws_doubles(const SplitPlan &p);

// partial blocks: the diagonal CTAs' then the pair CTAs'
int64_t split_partials(const SplitPlan &p) { return (int64_t)p.nsplit * p.nrb + (int64_t)p.nsplit_pair * p.npair; }

SplitWs split_ws(double *d_ws, const SplitPlan &p) {
  const int64_t np = split_partials(p) * kRows * kRows;
  const int64_t tab = (p.ngroups * p.J + 1) / 2;
  SplitWs w;
  w.gmax = reinterpret_cast<unsigned long long *>(d_ws);
  w.err = reinterpret_cast<int *>(d_ws + 1);
  w.partials = d_ws + 4;
  w.table = reinterpret_cast<int *>(d_ws + 4 + np);
  w.refs = reinterpret_cast<int *>(d_ws + 4 + np + tab);
  w.unfolded = d_ws + split_ws_doubles(p);
  return w;
}

int64_t split_ws_doubles(const SplitPlan &p) {
  const int64_t refs = (int64_t)p.nsplit * p.nrb * kRows + (int64_t)p.nsplit_pair * p.npair * 2 * kRows;
  const int64_t n = 4 + split_partials(p) * kRows * kRows + (p.ngroups * p.J + 1) / 2 + refs / 2 + 1;
  return (n + 31) / 32 * 32;  // the unfolding (when needed) starts 256-byte aligned after this
}

// the tiled L > 1 path: float64, L a multiple of 8, 16-byte aligned Y
bool use_oct(const void *y, tucker_dtype dt, int64_t L, int64_t B) {
  static const bool regs = [] {
    const char *e = std::getenv("TUCKER_GRAM_SPLIT_KERNEL");
    return e && std::strcmp(e, "regs") == 0;
  }();
  return !regs && dt == TUCKER_F64 && L > 1 && L % 8 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0 &&
         L < (1ll << 31) && (B + 3) / 4 * 4 < (1ll << 31);
}

template <typename T, int kMode, bool kF8 = false>
int run_gram_split(const void *y, int64_t L, const SplitPlan &p, const SplitWs &w, const DeviceInfo &dev,
                   cudaStream_t s) {
  (void)dev;
  TK_CUDA(allow_max_smem(k_gram_split<T, kMode, kF8>));
  k_gram_split<T, kMode, kF8><<<p.nsplit, kThreads, kF8 ? kSmemBytesF8 : kSmemBytes, s>>>(
      static_cast<const T *>(y), L, p, w.table, w.refs, w.partials, w.err);
  TK_LAUNCHED();
  return TUCKER_OK;
}

// The off-diagonal block pairs (J > 128): CTAs (split, pair) after the
// diagonal CTAs' partials and references.
template <typename T, bool kOct>
int run_gram_split_pair(const CUtensorMap &pmap, const SplitPlan &p, const SplitWs &w, cudaStream_t s) {
  SplitPlan pp = p;
  pp.cols_per_split = p.cols_per_split_pair;
  const int64_t nd = (int64_t)p.nsplit * p.nrb;
  TK_CUDA(allow_max_smem(k_gram_split_pair<T, kOct>));
  k_gram_split_pair<T, kOct><<<p.nsplit_pair * p.npair, kThreads, kPairSmemBytes, s>>>(
      pmap, pp, w.table, w.refs + nd * kRows, w.partials + nd * kRows * kRows, w.err);
  TK_LAUNCHED();
  return TUCKER_OK;
}

// The tensor-map kernel takes L == 1 with 16-byte column strides, a 16-byte
// aligned Y and K < 2^31; TUCKER_GRAM_SPLIT_KERNEL=regs forces the
// register-staged kernel.  Returns 1 when it ran, 0 when it does not apply.
template <typename T>
int run_gram_split_bulk(const void *y, const SplitPlan &p, const SplitWs &w, cudaStream_t s, bool *ran,
                        int64_t ld = 0) {
  static const bool regs = [] {
    const char *e = std::getenv("TUCKER_GRAM_SPLIT_KERNEL");
    return e && std::strcmp(e, "regs") == 0;
  }();
  *ran = false;
  const uint64_t col_bytes = (uint64_t)(ld > 0 ? ld : p.J) * sizeof(T);
  if (regs || col_bytes % 16 != 0 || reinterpret_cast<uintptr_t>(y) % 16 != 0 || p.K >= (1ll << 31)) return TUCKER_OK;
  CUtensorMap map;
  const uint64_t dims[2] = {(uint64_t)p.J, (uint64_t)p.K};
  const uint64_t strides[1] = {col_bytes};
  const uint32_t box[2] = {kRows, kChunk};
  if (!encode_tmap(&map, sizeof(T) == 8, y, 2, dims, strides, box)) return TUCKER_OK;
  CUtensorMap pmap;
  const uint32_t pbox[2] = {kRows, kPH};
  if (p.npair > 0 && !encode_tmap(&pmap, sizeof(T) == 8, y, 2, dims, strides, pbox)) return TUCKER_OK;
  TK_CUDA(allow_max_smem(k_gram_split_bulk<T, false>));
  k_gram_split_bulk<T, false><<<p.nsplit * p.nrb, kThreads, kBulkSmemBytes, s>>>(map, p, w.table, w.refs, w.partials,
                                                                                w.err);
  TK_LAUNCHED();
  if (p.npair > 0) TK_CHECK((run_gram_split_pair<T, false>(pmap, p, w, s)));
  *ran = true;
  return TUCKER_OK;
}

// the tiled L > 1 kernel: boxes {8 l, 128 rows, nl octets, nb b} of the 4-D
// map over Y viewed as (l % 8, j, l / 8, b), 64-byte swizzle
int run_gram_split_oct(const void *y, int64_t L, const SplitPlan &p, const SplitWs &w, cudaStream_t s, bool *ran) {
  *ran = false;
  CUtensorMap map;
  const uint64_t dims[4] = {8, (uint64_t)p.J, (uint64_t)(L / 8), (uint64_t)p.B};
  const uint64_t strides[3] = {(uint64_t)L * 8, 64, (uint64_t)L * p.J * 8};
  const uint32_t box[4] = {8, kRows, (uint32_t)p.nl, (uint32_t)p.nb};
  if (!encode_tmap(&map, true, y, 4, dims, strides, box, 64)) return TUCKER_OK;
  // the pair kernel's half-chunk: 16 of the chunk's 32 columns (2 octets of one b when nl = 4, else half the b)
  CUtensorMap pmap;
  const uint32_t pbox[4] = {8, kRows, p.nl == 4 ? 2u : (uint32_t)p.nl, p.nl == 4 ? 1u : (uint32_t)(p.nb / 2)};
  if (p.npair > 0 && !encode_tmap(&pmap, true, y, 4, dims, strides, pbox, 64)) return TUCKER_OK;
  TK_CUDA(allow_max_smem(k_gram_split_bulk<double, true>));
  k_gram_split_bulk<double, true><<<p.nsplit * p.nrb, kThreads, kBulkSmemBytes, s>>>(map, p, w.table, w.refs,
                                                                                    w.partials, w.err);
  TK_LAUNCHED();
  if (p.npair > 0) TK_CHECK((run_gram_split_pair<double, true>(pmap, p, w, s)));
  *ran = true;
  return TUCKER_OK;
}

}  // namespace

bool encode_tmap(CUtensorMap *map, bool f64, const void *base, int rank, const uint64_t *dims,
                 const uint64_t *strides_bytes, const uint32_t *box, int swizzle) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode || rank < 1 || rank > 5) return false;
  cuuint64_t gdim[5], gstride[4];
  cuuint32_t bx[5], estride[5];
  for (int k = 0; k < rank; ++k) {
    gdim[k] = dims[k];
    bx[k] = box[k];
    estride[k] = 1;
    if (k + 1 < rank) gstride[k] = strides_bytes[k];
  }
  return encode(map, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                const_cast<void *>(base), gdim, gstride, bx, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swizzle == 64    ? CU_TENSOR_MAP_SWIZZLE_64B
                : swizzle == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t gram_split_workspace_doubles(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, tucker_dtype dt,
                                     const void *y) {
  int64_t n = split_ws_doubles(split_plan(L, J, B, dev));
  if (L > 1 && L % 8 == 0) n = std::max(n, split_ws_doubles(split_plan(L, J, B, dev, true)));
  if (needs_unfold(L, J, dt, y)) {  // room for the explicit unfolding after the non-tiled plan's workspace
    const size_t es = dt == TUCKER_F64 ? 8 : 4;
    n = std::max(n, split_ws_doubles(split_plan(L, J, B, dev)) + (unfold_ld(J, es) * L * B * (int64_t)es + 7) / 8);
  }
  return n;
}

int launch_gram_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *d_S, double *d_ws,
                      const DeviceInfo &dev, cudaStream_t s, Prof *prof, int *d_colexp, bool f8) {
  const bool oct = !f8 && use_oct(y, dt, L, B);  // the E4M3 digits run in the register-staged kernel
  if (J > kMaxRows || (f8 && J > kRows)) {
    set_error("split-precision Gram supports J <= %d (got %lld)", f8 ? kRows : kMaxRows, (long long)J);
    return TUCKER_EUNSUPPORTED;
  }
  // J > 128: row blocks and their pairs in the tensor-map kernels, on Y in
  // place or on its explicit unfolding (then read as L == 1)
  const bool unfold = !oct && needs_unfold(L, J, dt, y);
  if (J > kRows && L * B >= (1ll << 31)) {
    set_error("split-precision Gram with J = %lld > %d needs fewer than 2^31 columns", (long long)J, kRows);
    return TUCKER_EUNSUPPORTED;
  }
  const SplitPlan p = split_plan(L, J, B, dev, oct);
  if (p.ngroups > 0x7FFFFFFFll) {
    set_error("split-precision Gram: too many column groups (%lld)", (long long)p.ngroups);
    return TUCKER_EUNSUPPORTED;
  }
  const SplitWs w = split_ws(d_ws, p);
  const bool f64 = dt == TUCKER_F64;
  const double in_bytes = (double)L * B * J * (f64 ? 8 : 4);
  TK_CUDA(cudaMemsetAsync(w.gmax, 0, 2 * sizeof(double), s));  // gmax and the error flag
  const int contig_pairs = L == 1 && (2 * 256) % J == 0 && J % 2 == 0 &&
                           reinterpret_cast<uintptr_t>(y) % (f64 ? 16 : 8) == 0;
  const int mode = L == 1 ? kColsStrided
                          : (L % 8 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0) ? kColsContig : kColsGeneric;
  if (prof) prof->begin(TUCKER_PHASE_SCALE);
  const bool async_exp = L > 1 && (L * (int64_t)(f64 ? 8 : 4)) % 16 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0;
  if (async_exp) {
    constexpr size_t kExpSmem = (size_t)2 * 8 * 256 * 16;  // 2 stages x RS x NQ chunks (the same for both types)
    if (oct) {
      TK_CUDA(allow_max_smem(k_rowgroup_exp_async<double, true>));
      k_rowgroup_exp_async<double, true><<<(unsigned)p.ngroups, 512, kExpSmem, s>>>(
          static_cast<const double *>(y), L, (int)J, p.K, p.nL, p.nl, B, w.table, w.gmax, d_colexp);
    } else if (f64) {
      TK_CUDA(allow_max_smem(k_rowgroup_exp_async<double, false>));
      k_rowgroup_exp_async<double, false><<<(unsigned)p.ngroups, 512, kExpSmem, s>>>(
          static_cast<const double *>(y), L, (int)J, p.K, 1, 1, B, w.table, w.gmax, d_colexp);
    } else {
      TK_CUDA(allow_max_smem(k_rowgroup_exp_async<float, false>));
      k_rowgroup_exp_async<float, false><<<(unsigned)p.ngroups, 512, kExpSmem, s>>>(
          static_cast<const float *>(y), L, (int)J, p.K, 1, 1, B, w.table, w.gmax, d_colexp);
    }
  } else if (f64)
    k_rowgroup_exp<double><<<(unsigned)p.ngroups, 256, 0, s>>>(static_cast<const double *>(y), L, (int)J, p.K,
                                                               contig_pairs, w.table, w.gmax, d_colexp);
  else
    k_rowgroup_exp<float><<<(unsigned)p.ngroups, 256, 0, s>>>(static_cast<const float *>(y), L, (int)J, p.K,
                                                              contig_pairs, w.table, w.gmax, d_colexp);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, in_bytes, 1);
  if (unfold) {  // the explicit unfolding (counted with the exponent pass: data movement before the Gram)
    const size_t es = f64 ? 8 : 4;
    const int64_t ld = unfold_ld(J, es), nlt = (L + 31) / 32;
    if (prof) prof->begin(TUCKER_PHASE_SCALE);
    const dim3 grid((unsigned)(nlt * B), (unsigned)((J + 31) / 32));
    if (f64)
      k_unfold<double><<<grid, 256, 0, s>>>(static_cast<const double *>(y), L, (int)J, B, ld, nlt,
                                            static_cast<double *>(w.unfolded));
    else
      k_unfold<float><<<grid, 256, 0, s>>>(static_cast<const float *>(y), L, (int)J, B, ld, nlt,
                                           static_cast<float *>(w.unfolded));
    TK_LAUNCHED();
    if (prof) prof->end(0.0, 2 * in_bytes, 1);
  }
  if (prof) prof->begin(TUCKER_PHASE_GRAM);
  bool ran = false;
  if (unfold) {
    const int64_t ld = unfold_ld(J, f64 ? 8 : 4);
    if (f64) TK_CHECK(run_gram_split_bulk<double>(w.unfolded, p, w, s, &ran, ld));
    else TK_CHECK(run_gram_split_bulk<float>(w.unfolded, p, w, s, &ran, ld));
  } else if (f8) {
    if (f64) {
      if (mode == kColsStrided) TK_CHECK((run_gram_split<double, kColsStrided, true>(y, L, p, w, dev, s)));
      else if (mode == kColsContig) TK_CHECK((run_gram_split<double, kColsContig, true>(y, L, p, w, dev, s)));
      else TK_CHECK((run_gram_split<double, kColsGeneric, true>(y, L, p, w, dev, s)));
    } else {
      if (mode == kColsStrided) TK_CHECK((run_gram_split<float, kColsStrided, true>(y, L, p, w, dev, s)));
      else if (mode == kColsContig) TK_CHECK((run_gram_split<float, kColsContig, true>(y, L, p, w, dev, s)));
      else TK_CHECK((run_gram_split<float, kColsGeneric, true>(y, L, p, w, dev, s)));
    }
    ran = true;
  } else if (L == 1) {
    if (f64) TK_CHECK(run_gram_split_bulk<double>(y, p, w, s, &ran));
    else TK_CHECK(run_gram_split_bulk<float>(y, p, w, s, &ran));
  } else if (oct) {
    TK_CHECK(run_gram_split_oct(y, L, p, w, s, &ran));
    if (!ran) {
      set_error("split-precision Gram: the tensor map of the tiled path was refused");
      return TUCKER_ECUDA;
    }
  }
  if (!ran && J > kRows) {
    set_error("split-precision Gram: the tensor map for J = %lld was refused", (long long)J);
    return TUCKER_ECUDA;
  }
  if (!ran && f64) {
    if (mode == kColsStrided) TK_CHECK((run_gram_split<double, kColsStrided>(y, L, p, w, dev, s)));
    else if (mode == kColsContig) TK_CHECK((run_gram_split<double, kColsContig>(y, L, p, w, dev, s)));
    else TK_CHECK((run_gram_split<double, kColsGeneric>(y, L, p, w, dev, s)));
  } else if (!ran) {
    if (mode == kColsStrided) TK_CHECK((run_gram_split<float, kColsStrided>(y, L, p, w, dev, s)));
    else if (mode == kColsContig) TK_CHECK((run_gram_split<float, kColsContig>(y, L, p, w, dev, s)));
    else TK_CHECK((run_gram_split<float, kColsGeneric>(y, L, p, w, dev, s)));
  }
  if (prof) prof->end((double)J * (J + 1) * (double)L * B, in_bytes, 1);
  if (prof) prof->begin(TUCKER_PHASE_GRAM_REDUCE);
  // S = (C + C^T) 2^(ref_i + ref_j - off): off = 2 x 21 + 1 for the BF16 digits, 2 x 15 + 1 for E4M3
  k_gram_split_reduce<<<(unsigned)((J * J + 31) / 32), 256, 0, s>>>(w.partials, w.refs, p.nsplit, p.nsplit_pair,
                                                                      p.nrb, p.npair, (int)J, w.gmax, f64,
                                                                      f8 ? 31 : 43, d_S);
  TK_LAUNCHED();
  if (prof)
    prof->end((double)split_partials(p) * kRows * kRows * 2, (double)split_partials(p) * kRows * kRows * 8, 1);
  return TUCKER_OK;
}

int gram_split_error(const double *d_ws, int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, int *h_err,
                     cudaStream_t s) {
  (void)L;
  (void)J;
  (void)B;
  (void)dev;
  // the error flag sits at the same place for every plan (split_ws)
  TK_CUDA(cudaMemcpyAsync(h_err, reinterpret_cast<const int *>(d_ws + 1), sizeof(int), cudaMemcpyDeviceToHost, s));
  return TUCKER_OK;
}

}  // namespace tk
