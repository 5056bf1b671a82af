// Split-precision Gram on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// The Gram step of Algorithm 1 (S = Y_(n) Y_(n)^T, Sec. 2.2) dominates the
// flops; GB300 runs float64 at ~1.2 TFLOP/s but BF16 tensor MMAs at ~1.9
// PFLOP/s.  This kernel forms the Gram from exact integer digits:
//
//   * Columns are taken in groups of 512.  For row i of group g, with
//     2^E_ig the smallest power of two above the row's largest magnitude in
//     the group, every entry becomes v = round(y 2^(21 - E_ig)), |v| <= 2^21,
//     split into three balanced digits v = s1 2^14 + s2 2^7 + s3 with
//     |s1| <= 128 and |s2|, |s3| <= 64.  Every digit (and 2 s3, s3 / 128) is
//     exact in BF16.  Scaling per row and per group keeps 21 significant bits
//     relative to the local magnitude, so rows and regions of small entries
//     keep their relative precision.
//   * Products are grouped by level p + q (weight 2^(7 (6 - p - q))):
//       acc0 = A1 A1^T                       (level 2, exact)
//       acc1 = A1 A2^T                       (level 3, exact, counted twice)
//       acc2 = A1 (2 A3)^T + A2 A2^T         (level 4, exact)
//       acc3 = A2 (2 A3)^T + A3 (A3 / 128)^T (levels 5 and 6)
//     Digit products are integers below 2^15; FP32 sums of integers stay
//     exact below 2^24, so acc0..acc2 are exact over a 512-column group
//     (acc2 <= 512 (128^2 + 64^2) < 2^24).  acc3 carries the two lowest
//     levels with ordinary FP32 rounding: its relative weight is 2^-21, so its
//     rounding error is ~2^-45 of the result.
//   * At the end of each group the four accumulators are drained:
//     C += (2^28 acc0 + 2^22 acc1 + 2^14 acc2 + 2^7 acc3) 2^(E_ig + E_jg - 2 E)
//     into per-thread double-float (FP32 pair) accumulators, E the exponent of
//     the global bound 2^E > max|Y|.  Every product of every level is counted,
//     and S = (C + C^T) 2^(2E - 43) after a fixed-order float64 reduction of
//     the per-CTA partials.  The four 128 x 128 accumulators fill TMEM's 512
//     columns.
//
// The result is the Gram of Y rounded to 21 bits below each local power of
// two (zero-mean rounding); the noise this adds to the tail eigenvalues is
// ~ (J - R)/J 2^-42/12 (2^E_ig / rms)^2 of ||Y||^2, a few 1e-13 for smooth
// data.  Operand tiles use the K-major, no-swizzle canonical layout of tcgen05
// shared-memory descriptors (8-row x 16-byte core matrices; LBO = 128 B
// between core matrices along K, SBO = 1024 B between 8-row groups).  Every
// mbarrier wait is bounded and CTA-uniform; on expiry the kernel raises an
// error flag, waits (bounded) for its own MMAs, frees its TMEM and returns.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tk {

namespace {

constexpr int kThreads = 512;
constexpr int kRows = 128;         // M = N = 128 (J <= 128, zero padded)
constexpr int kChunk = 64;         // columns staged per stage
constexpr int kTiles = 5;          // A1, A2, A3, 2*A3, A3/128
constexpr int kTileBytes = kRows * kChunk * 2;
constexpr int kStageBytes = kTiles * kTileBytes;
constexpr int kStages = 2;
constexpr int kDrainChunks = 8;    // 512 columns between drains
constexpr int kTmemCols = 512;

using namespace tc;
constexpr uint32_t kIdesc = idesc_bf16(kRows, kRows);

struct SplitPlan {
  int J;
  int E;
  int64_t K;
  int64_t cols_per_split;
  int nsplit;
};

template <typename T>
__device__ __forceinline__ void load_unit(const T *__restrict__ y, int64_t L, int J, int64_t K, int64_t stride_b,
                                          int i, int64_t c, int64_t c_end, T (&raw)[8]) {
  // columns c .. c + 7 of row i (zero past the range or past J)
  if (i >= J || c >= c_end) {
#pragma unroll
    for (int k = 0; k < 8; ++k) raw[k] = T(0);
    return;
  }
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

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_gram_split(const T *__restrict__ y, int64_t L, SplitPlan p,
                                                            double *__restrict__ ws, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  __shared__ __align__(8) unsigned long long mbar[kStages];
  __shared__ unsigned long long rowmax[kRows];
  __shared__ int rowexp[kRows];
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  unsigned char *stage_base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
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
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  const int64_t c_begin = (int64_t)blockIdx.x * p.cols_per_split;
  const int64_t c_end = min(p.K, c_begin + p.cols_per_split);
  const int nchunks = (int)((c_end - c_begin + kChunk - 1) / kChunk);
  const int64_t stride_b = L * (int64_t)p.J;

  // loader/converter role: row `row`, column groups kg0 and kg0 + 4 of a chunk
  const int row = tid % kRows;
  const int kg0 = tid / kRows;
  // drain role: TMEM lanes 32 q .. 32 q + 31, columns 32 cb .. 32 cb + 31
  const int q = warp & 3, cb = warp >> 2;
  const int drow = 32 * q + lane;
  float acc_hi[32], acc_lo[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) acc_hi[e] = acc_lo[e] = 0.f;

  T raw[2][8];
  int last_committed = -1;
  int my_exp = 0;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    const int in_group = ch % kDrainChunks;
    if (in_group == 0) {
      // exponent of each row over this group's columns (the re-read below hits L2)
      if (tid < kRows) rowmax[tid] = 0ull;
      __syncthreads();
      unsigned long long m = 0ull;
      const int last = min(nchunks, ch + kDrainChunks);
      for (int c2 = ch; c2 < last; ++c2) {
        const int64_t cc = c_begin + (int64_t)c2 * kChunk;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          load_unit(y, L, p.J, p.K, stride_b, row, cc + 8 * (kg0 + 4 * u), c_end, raw[u]);
#pragma unroll
          for (int k = 0; k < 8; ++k) m = max(m, mag_bits(raw[u][k]));
        }
      }
      atomicMax(&rowmax[row], m);
      __syncthreads();
      if (tid < kRows) rowexp[tid] = exp_above(rowmax[tid], kF64);
      __syncthreads();
      my_exp = rowexp[row];
      const int64_t cc = c_begin + (int64_t)ch * kChunk;
      load_unit(y, L, p.J, p.K, stride_b, row, cc + 8 * kg0, c_end, raw[0]);
      load_unit(y, L, p.J, p.K, stride_b, row, cc + 8 * (kg0 + 4), c_end, raw[1]);
    }
    // stage `buf` is free once the MMAs of chunk ch - 2 have completed; one
    // thread waits (bounded) and the barrier hands the outcome to all
    if (ch >= 2) {
      if (tid == 0 && !mbar_wait(smem_addr(&mbar[buf]), ((ch - 2) >> 1) & 1)) stop = 1;
      __syncthreads();
      if (stop) break;
    }
    unsigned char *st = stage_base + buf * kStageBytes;
    // convert the two units to digits and store one 16-byte core-matrix row per tile
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int kg = kg0 + 4 * u;
      uint32_t w[kTiles][4];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        int d1[2], d2[2], d3[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int v = scaled_int(raw[u][k + h], my_exp);
          const int s1 = (v + (1 << 13)) >> 14;
          const int r1 = v - (s1 << 14);
          const int s2 = (r1 + 64) >> 7;
          d1[h] = s1;
          d2[h] = s2;
          d3[h] = r1 - (s2 << 7);
        }
        const int j = k >> 1;
        w[0][j] = bf16_pair((float)d1[0], (float)d1[1]);
        w[1][j] = bf16_pair((float)d2[0], (float)d2[1]);
        w[2][j] = bf16_pair((float)d3[0], (float)d3[1]);
        w[3][j] = bf16_pair((float)(2 * d3[0]), (float)(2 * d3[1]));
        w[4][j] = bf16_pair((float)d3[0] * 0x1p-7f, (float)d3[1] * 0x1p-7f);
      }
      const int off = (row >> 3) * 1024 + kg * 128 + (row & 7) * 16;
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
        const uint64_t a1 = smem_desc(base + 0 * kTileBytes + 256 * s, 128, 1024);
        const uint64_t a2 = smem_desc(base + 1 * kTileBytes + 256 * s, 128, 1024);
        const uint64_t a3 = smem_desc(base + 2 * kTileBytes + 256 * s, 128, 1024);
        const uint64_t a3x2 = smem_desc(base + 3 * kTileBytes + 256 * s, 128, 1024);
        const uint64_t a3s = smem_desc(base + 4 * kTileBytes + 256 * s, 128, 1024);
        mma_bf16(tmem + 0, a1, a1, kIdesc, acc);
        mma_bf16(tmem + 128, a1, a2, kIdesc, acc);
        mma_bf16(tmem + 256, a1, a3x2, kIdesc, acc);
        mma_bf16(tmem + 256, a2, a2, kIdesc, 1u);
        mma_bf16(tmem + 384, a2, a3x2, kIdesc, acc);
        mma_bf16(tmem + 384, a3, a3s, kIdesc, 1u);
      }
      mma_commit(smem_addr(&mbar[buf]));
    }
    last_committed = ch;
    if (in_group == kDrainChunks - 1 || ch == nchunks - 1) {
      if (tid == 0 && !mbar_wait(smem_addr(&mbar[buf]), (ch >> 1) & 1)) stop = 1;
      __syncthreads();
      if (!stop) {  // uniform across the CTA, so the .sync.aligned loads below never diverge
        fence_after();
        const float wts[4] = {0x1p28f, 0x1p22f, 0x1p14f, 0x1p7f};  // 2^28, 2 2^21, 2^14, 2^7
        const int ei = rowexp[drow] - p.E;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float sc[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int x = ei + rowexp[32 * cb + 16 * half + e] - p.E;  // <= 0
            sc[e] = x < -120 ? 0.f : __int_as_float((127 + x) << 23);
          }
#pragma unroll
          for (int lev = 0; lev < 4; ++lev) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * lev + 32 * cb + 16 * half), r);
#pragma unroll
            for (int e = 0; e < 16; ++e)
              df_add(acc_hi[16 * half + e], acc_lo[16 * half + e], __uint_as_float(r[e]) * wts[lev] * sc[e]);
          }
        }
      }
      fence_before();
      __syncthreads();
      if (stop) break;
    }
    // prefetch the next chunk of this group while the tensor cores work
    if (ch + 1 < nchunks && (ch + 1) % kDrainChunks != 0) {
      const int64_t cn = c_begin + (int64_t)(ch + 1) * kChunk;
      load_unit(y, L, p.J, p.K, stride_b, row, cn + 8 * kg0, c_end, raw[0]);
      load_unit(y, L, p.J, p.K, stride_b, row, cn + 8 * (kg0 + 4), c_end, raw[1]);
    }
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
  for (int e = 0; e < 32; ++e) dst[e] = (double)acc_hi[e] + (double)acc_lo[e];
}

__global__ void __launch_bounds__(256) k_gram_split_reduce(const double *__restrict__ ws, int nsplit, int J,
                                                           double scale, double *__restrict__ S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= J * J) return;
  const int i = idx % J, j = idx / J;
  double s = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) {
    const double *c = ws + (size_t)sp * kRows * kRows;
    s += c[i * kRows + j] + c[j * kRows + i];
  }
  S[i + (int64_t)J * j] = s * scale;
}

__global__ void __launch_bounds__(256) k_maxabs_partial(const void *__restrict__ x, int is_f64, int64_t n,
                                                        double *__restrict__ partial) {
  __shared__ double red[256];
  double m = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = is_f64 ? fabs(__ldg(static_cast<const double *>(x) + i))
                            : (double)fabsf(__ldg(static_cast<const float *>(x) + i));
    m = fmax(m, v);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_maxabs_final(const double *__restrict__ partial, int n, double *__restrict__ out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, partial[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 1024;

SplitPlan split_plan(int64_t L, int64_t J, int64_t B, double maxabs, const DeviceInfo &dev) {
  SplitPlan p{};
  p.J = (int)J;
  p.K = L * B;
  int e = 0;
  if (maxabs > 0.0) std::frexp(maxabs, &e);  // maxabs < 2^e
  p.E = e;
  const int64_t chunks = (p.K + kChunk - 1) / kChunk;
  const int64_t ns = std::max<int64_t>(1, std::min<int64_t>(dev.sms, chunks));
  const int64_t chunks_per = (chunks + ns - 1) / ns;
  p.cols_per_split = chunks_per * kChunk;
  p.nsplit = (int)((p.K + p.cols_per_split - 1) / p.cols_per_split);
  return p;
}

}  // namespace

int64_t maxabs_partials() { return 1024; }

int launch_maxabs(const void *x, tucker_dtype dt, int64_t n, double *d_partials, double *d_out, cudaStream_t s,
                  Prof *prof) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (n + 1023) / 1024));
  if (prof) prof->begin(TUCKER_PHASE_SCALE);
  k_maxabs_partial<<<blocks, 256, 0, s>>>(x, dt == TUCKER_F64, n, d_partials);
  TK_LAUNCHED();
  k_maxabs_final<<<1, 256, 0, s>>>(d_partials, blocks, d_out);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, (double)n * (dt == TUCKER_F64 ? 8 : 4), 2);
  return TUCKER_OK;
}

int64_t gram_split_workspace_doubles(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev) {
  const SplitPlan p = split_plan(L, J, B, 1.0, dev);
  return (int64_t)p.nsplit * kRows * kRows + 8;
}

int launch_gram_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double maxabs, double *d_S,
                      double *d_ws, const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (J > kRows) {
    set_error("split-precision Gram supports J <= %d (got %lld)", kRows, (long long)J);
    return TUCKER_EUNSUPPORTED;
  }
  const SplitPlan p = split_plan(L, J, B, maxabs, dev);
  int *d_err = reinterpret_cast<int *>(d_ws + (int64_t)p.nsplit * kRows * kRows);
  TK_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  if (prof) prof->begin(TUCKER_PHASE_GRAM);
  if (dt == TUCKER_F64) {
    TK_CUDA(cudaFuncSetAttribute(k_gram_split<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    k_gram_split<double><<<p.nsplit, kThreads, kSmemBytes, s>>>(static_cast<const double *>(y), L, p, d_ws, d_err);
  } else {
    TK_CUDA(cudaFuncSetAttribute(k_gram_split<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    k_gram_split<float><<<p.nsplit, kThreads, kSmemBytes, s>>>(static_cast<const float *>(y), L, p, d_ws, d_err);
  }
  TK_LAUNCHED();
  if (prof) prof->end((double)J * (J + 1) * (double)p.K, (double)p.K * J * (dt == TUCKER_F64 ? 8 : 4), 1);
  if (prof) prof->begin(TUCKER_PHASE_GRAM_REDUCE);
  const double scale = std::ldexp(1.0, 2 * p.E - 43);
  k_gram_split_reduce<<<(unsigned)((J * J + 255) / 256), 256, 0, s>>>(d_ws, p.nsplit, (int)J, scale, d_S);
  TK_LAUNCHED();
  if (prof) prof->end((double)p.nsplit * J * J * 2, (double)p.nsplit * kRows * kRows * 8, 1);
  return TUCKER_OK;
}

int gram_split_error(const double *d_ws, int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, int *h_err,
                     cudaStream_t s) {
  const SplitPlan p = split_plan(L, J, B, 1.0, dev);
  TK_CUDA(cudaMemcpyAsync(h_err, d_ws + (int64_t)p.nsplit * kRows * kRows, sizeof(int), cudaMemcpyDeviceToHost, s));
  return TUCKER_OK;
}

}  // namespace tk
