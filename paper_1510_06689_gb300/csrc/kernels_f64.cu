// Float64 kernels of the ST-HOSVD hot path: sum of squares (Sec. 2.1 norm),
// the split-K symmetric Gram of the mode-n unfolding (Algorithm 1, Gram step)
// and the mode-n product (Algorithm 1, TTM step; Eq. reconstruct).
//
// All three read the tensor in place through the (L, J, B) view of the
// natural layout: entry (l, j, b) at l + L (j + J b), column c = l + L b of
// the unfolding.  On GB300 the float64 pipe (about 1.2 TFLOP/s) bounds these
// kernels, far below what HBM could feed, so the design goal is to spend no
// float64 instruction that the algorithm does not need (the Gram computes
// the upper triangle only) and to keep every SM's float64 pipe busy with one
// balanced wave of CTAs.  Loads are plain coalesced loads staged in shared
// memory.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "common.cuh"

namespace tk {

namespace {

constexpr int kMaxCols = 64;  // columns staged per chunk (upper bound)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction (result valid in thread 0).
__device__ double block_sum(double v) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (warp == 0) v = warp_sum(v);
  return v;
}

template <typename T>
__device__ __forceinline__ double ldg(const T *p) {
  return static_cast<double>(__ldg(p));
}

// ---------------------------------------------------------------------------
// sum of squares
// ---------------------------------------------------------------------------
constexpr int kNormThreads = 256;
constexpr int kNormBlocks = 2048;  // fixed, so the summation order depends only on n

template <typename T>
__global__ void __launch_bounds__(kNormThreads) k_sumsq(const T *__restrict__ x, int64_t n,
                                                        double *__restrict__ partial) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const double v0 = ldg(x + i), v1 = ldg(x + i + stride);
    const double v2 = ldg(x + i + 2 * stride), v3 = ldg(x + i + 3 * stride);
    a0 = fma(v0, v0, a0);
    a1 = fma(v1, v1, a1);
    a2 = fma(v2, v2, a2);
    a3 = fma(v3, v3, a3);
  }
  for (; i < n; i += stride) {
    const double v = ldg(x + i);
    a0 = fma(v, v, a0);
  }
  const double s = block_sum((a0 + a1) + (a2 + a3));
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// One block sums `count` partials in a fixed order.
__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ partial, int64_t count,
                                                      double *__restrict__ out) {
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) a += partial[i];
  a = block_sum(a);
  if (threadIdx.x == 0) out[0] = a;
}

// ---------------------------------------------------------------------------
// chunk loader shared by the Gram and TTM kernels: rows [0, J) of columns
// [c0, c0 + kc) of the (L, J, B) view into sm[kk * ld + i] (zero fill).
// colbase[kk] = l + L J b of column c0 + kk, or -1 past the range.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void load_chunk(const T *__restrict__ y, int64_t L, int J, int rows_pad, int kc,
                                           const int64_t *colbase, double *sm, int ld_row, int ld_col) {
  const int total = rows_pad * kc;
  if (L == 1) {  // a column is J contiguous elements: threads run along i
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int i = e % rows_pad, kk = e / rows_pad;
      const int64_t base = colbase[kk];
      sm[kk * ld_col + i * ld_row] = (i < J && base >= 0) ? ldg(y + base + i) : 0.0;
    }
  } else {  // a row segment is contiguous along l: threads run along kk
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int kk = e % kc, i = e / kc;
      const int64_t base = colbase[kk];
      sm[kk * ld_col + i * ld_row] = (i < J && base >= 0) ? ldg(y + base + L * (int64_t)i) : 0.0;
    }
  }
}

__device__ __forceinline__ void set_colbase(int64_t c0, int64_t c_end, int kc, int64_t L, int64_t stride_b,
                                            int64_t *colbase) {
  for (int t = threadIdx.x; t < kc; t += blockDim.x) {
    const int64_t c = c0 + t;
    int64_t v = -1;
    if (c < c_end) {
      const int64_t b = c / L;
      v = (c - b * L) + stride_b * b;
    }
    colbase[t] = v;
  }
}

// ---------------------------------------------------------------------------
// Gram (symmetric, split-K).  The J x J result is covered by 4 x 4 micro-tiles
// (a, b) with a <= b; micro-tile m = b (b + 1) / 2 + a.  CTA (g, split) owns
// the micro-tiles [g * per_group, (g + 1) * per_group) (one per thread) and
// the columns of its split, and writes its 16 partial sums per micro-tile to
// ws[(split * n_micro + m) * 16 + 4 r + c].  k_gram_reduce adds the splits in
// order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
struct GramPlan {
  int J, Jp, n_micro, groups, per_group, threads, kc, nsplit;
  int64_t cols_per_split, K;
  size_t smem;
};

__host__ __device__ __forceinline__ void decode_upper(int m, int &a, int &b) {
  int bb = (int)((sqrt(8.0 * m + 1.0) - 1.0) * 0.5);
  while ((bb + 1) * (bb + 2) / 2 <= m) ++bb;
  while (bb * (bb + 1) / 2 > m) --bb;
  b = bb;
  a = m - bb * (bb + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(512) k_gram_partial(const T *__restrict__ y, int64_t L, int64_t B, GramPlan p,
                                                      double *__restrict__ ws) {
  extern __shared__ __align__(16) double sm[];  // [kc][Jp]
  __shared__ int64_t colbase[kMaxCols];
  const int split = blockIdx.y;
  const int64_t c_begin = (int64_t)split * p.cols_per_split;
  const int64_t c_end = min(p.K, c_begin + p.cols_per_split);
  const int m = blockIdx.x * p.per_group + threadIdx.x;
  const bool active = threadIdx.x < p.per_group && m < p.n_micro;
  int ta = 0, tb = 0;
  if (active) decode_upper(m, ta, tb);
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const int64_t stride_b = L * (int64_t)p.J;
  for (int64_t c0 = c_begin; c0 < c_end; c0 += p.kc) {
    set_colbase(c0, c_end, p.kc, L, stride_b, colbase);
    __syncthreads();
    load_chunk(y, L, p.J, p.Jp, p.kc, colbase, sm, 1, p.Jp);
    __syncthreads();
    if (active) {
      const double *pa = sm + 4 * ta;
      const double *pb = sm + 4 * tb;
#pragma unroll 4
      for (int kk = 0; kk < p.kc; ++kk) {
        const double2 a01 = *reinterpret_cast<const double2 *>(pa + kk * p.Jp);
        const double2 a23 = *reinterpret_cast<const double2 *>(pa + kk * p.Jp + 2);
        const double2 b01 = *reinterpret_cast<const double2 *>(pb + kk * p.Jp);
        const double2 b23 = *reinterpret_cast<const double2 *>(pb + kk * p.Jp + 2);
        const double av[4] = {a01.x, a01.y, a23.x, a23.y};
        const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
      }
    }
    __syncthreads();
  }
  if (active) {
    double *dst = ws + ((size_t)split * p.n_micro + m) * 16;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[4 * r + c] = acc[r][c];
  }
}

__global__ void __launch_bounds__(256) k_gram_reduce(const double *__restrict__ ws, GramPlan p,
                                                     double *__restrict__ S) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_split = (int64_t)p.n_micro * 16;
  if (idx >= per_split) return;
  double s = 0.0;
  for (int sp = 0; sp < p.nsplit; ++sp) s += ws[sp * per_split + idx];
  const int m = (int)(idx >> 4), e = (int)(idx & 15);
  int a, b;
  decode_upper(m, a, b);
  const int i = 4 * a + (e >> 2), j = 4 * b + (e & 3);
  if (i < p.J && j < p.J && i <= j) {
    S[i + (int64_t)p.J * j] = s;
    S[j + (int64_t)p.J * i] = s;
  }
}

// Resident CTAs per SM for a launch shape; the dynamic shared memory limit is
// raised to exactly `smem` first.  Failures of these optional queries are
// cleared so they cannot surface as a later launch error.
template <typename K>
int occupancy(K kernel, int threads, size_t smem) {
  int occ = 1;
  if (allow_max_smem(kernel) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess)
    occ = 1;
  cudaGetLastError();
  return occ < 1 ? 1 : occ;
}

GramPlan gram_plan(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev) {
  GramPlan p{};
  p.J = (int)J;
  p.Jp = (int)((J + 3) / 4 * 4);
  const int nmt = p.Jp / 4;
  p.n_micro = nmt * (nmt + 1) / 2;
  p.groups = (p.n_micro + 511) / 512;
  p.per_group = (p.n_micro + p.groups - 1) / p.groups;
  p.threads = (p.per_group + 31) / 32 * 32;
  p.kc = std::max(8, std::min(kMaxCols, (4096 / p.Jp) / 4 * 4));
  p.smem = (size_t)p.kc * p.Jp * sizeof(double);
  p.K = L * B;
  // One balanced wave: as many splits as resident CTAs allow, never more
  // splits than column chunks.
  int occ = occupancy(k_gram_partial<double>, p.threads, p.smem);
  const int64_t slots = (int64_t)dev.sms * occ;
  const int64_t chunks = (p.K + p.kc - 1) / p.kc;
  int64_t ns = std::max<int64_t>(1, slots / p.groups);
  ns = std::min(ns, chunks);
  const int64_t chunks_per = (chunks + ns - 1) / ns;
  p.cols_per_split = chunks_per * p.kc;
  p.nsplit = (int)((p.K + p.cols_per_split - 1) / p.cols_per_split);
  return p;
}

// ---------------------------------------------------------------------------
// mode-n product Z(L, K, B) = sum_j A[k, j] Y(L, J, B).  CTA (xsplit, ktile)
// stages A[k0 .. k0 + kt, :] (as As[j][kl]) once and then streams its column
// range in chunks of kc columns (Ys[j][kk]); each thread owns 4 k x 4
// columns.  For long contractions (J > kTtmWholeJ) the j range is streamed
// too, jc rows of A and Y at a time with the accumulators kept in registers,
// so that shared memory no longer limits the tile to a few warps.  The DIFF
// variant reads X instead of writing Z and accumulates (x - z)^2 per CTA
// (fixed grid, fixed order).
// ---------------------------------------------------------------------------
constexpr int kTtmWholeJ = 128;   // up to this J, A's tile stays in shared memory for the whole run
constexpr int kTtmMaxCols = 128;  // columns per chunk (upper bound)
struct TtmPlan {
  int J, K, kt, ktp, kc, nkg, ncg, threads, ktiles, xsplit, jc;
  int64_t cols_per_cta, Kc;
  size_t smem;
};

template <typename T, typename TX, bool DIFF>
__global__ void __launch_bounds__(512) k_ttm(const T *__restrict__ y, int64_t L, int64_t B,
                                             const double *__restrict__ a, int64_t ak, int64_t aj, TtmPlan p,
                                             double *__restrict__ z, const TX *__restrict__ x,
                                             double *__restrict__ partial) {
  extern __shared__ __align__(16) double sm[];
  double *As = sm;                             // [jc][ktp]
  double *Ys = sm + (size_t)p.jc * p.ktp;      // [jc][kc]
  __shared__ int64_t colin[kTtmMaxCols], colout[kTtmMaxCols];
  const int k0 = blockIdx.y * p.kt;
  const int kt = min(p.kt, p.K - k0);
  const bool stream_j = p.jc < p.J;
  // rows j0 .. j0 + nj of A's tile into As
  auto load_a = [&](int j0, int nj) {
    for (int e = threadIdx.x; e < nj * p.ktp; e += blockDim.x) {
      const int j = e / p.ktp, kl = e - j * p.ktp;
      As[e] = (kl < kt) ? a[(int64_t)(k0 + kl) * ak + (int64_t)(j0 + j) * aj] : 0.0;
    }
  };
  if (!stream_j) load_a(0, p.J);
  int kg, cg;
  if (L == 1) {
    kg = threadIdx.x % p.nkg;
    cg = threadIdx.x / p.nkg;
  } else {
    cg = threadIdx.x % p.ncg;
    kg = threadIdx.x / p.ncg;
  }
  const bool active = threadIdx.x < p.nkg * p.ncg;
  const int64_t c_begin = (int64_t)blockIdx.x * p.cols_per_cta;
  const int64_t c_end = min(p.Kc, c_begin + p.cols_per_cta);
  const int64_t in_b = L * (int64_t)p.J, out_b = L * (int64_t)p.K;
  double dacc = 0.0;
  for (int64_t c0 = c_begin; c0 < c_end; c0 += p.kc) {
    for (int t = threadIdx.x; t < p.kc; t += blockDim.x) {
      const int64_t c = c0 + t;
      int64_t vi = -1, vo = -1;
      if (c < c_end) {
        const int64_t b = c / L, l = c - b * L;
        vi = l + in_b * b;
        vo = l + out_b * b;
      }
      colin[t] = vi;
      colout[t] = vo;
    }
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
    for (int j0 = 0; j0 < p.J; j0 += p.jc) {
      const int nj = min(p.jc, p.J - j0);
      __syncthreads();  // colin / colout written; the previous stage's reads done
      if (stream_j) load_a(j0, nj);
      load_chunk(y + (L == 1 ? (int64_t)j0 : L * (int64_t)j0), L, nj, nj, p.kc, colin, Ys, p.kc, 1);
      __syncthreads();
      if (active) {
        const double *pa = As + 4 * kg;
        const double *py = Ys + 4 * cg;
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
          const double2 a01 = *reinterpret_cast<const double2 *>(pa + j * p.ktp);
          const double2 a23 = *reinterpret_cast<const double2 *>(pa + j * p.ktp + 2);
          const double2 y01 = *reinterpret_cast<const double2 *>(py + j * p.kc);
          const double2 y23 = *reinterpret_cast<const double2 *>(py + j * p.kc + 2);
          const double av[4] = {a01.x, a01.y, a23.x, a23.y};
          const double yv[4] = {y01.x, y01.y, y23.x, y23.y};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], yv[c], acc[r][c]);
        }
      }
    }
    if (active) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t base = colout[4 * cg + c];
        if (base < 0) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int k = 4 * kg + r;
          if (k < kt) {
            const int64_t addr = base + L * (int64_t)(k0 + k);
            if constexpr (DIFF) {
              const double d = ldg(x + addr) - acc[r][c];
              dacc = fma(d, d, dacc);
            } else {
              z[addr] = acc[r][c];
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if constexpr (DIFF) {
    const double s = block_sum(dacc);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

template <typename T, typename TX, bool DIFF>
TtmPlan ttm_plan(int64_t L, int64_t J, int64_t B, int64_t K, const DeviceInfo &dev) {
  TtmPlan p{};
  p.J = (int)J;
  p.K = (int)K;
  p.Kc = L * B;
  // k tile: As must fit in ~96 KB; at most 128 outputs per tile.
  if (J <= kTtmWholeJ) {
    p.jc = (int)J;
    int ktp_max = std::max(4, std::min(128, (int)(12288 / J) / 4 * 4));
    const int ktiles = (int)((K + ktp_max - 1) / ktp_max);
    p.kt = (int)((K + ktiles - 1) / ktiles);
    p.ktp = (p.kt + 3) / 4 * 4;
    p.ktiles = ktiles;
    p.nkg = p.ktp / 4;
    // column chunk: Ys within ~64 KB, threads <= 512.
    p.kc = std::max(4, std::min(kMaxCols, (int)(8192 / J) / 4 * 4));
    while ((p.kc / 4) * p.nkg > 512 && p.kc > 4) p.kc -= 4;
  } else {
    // streamed j: at most 64 outputs a tile, columns enough for 256..512 threads, 64 rows a stage
    p.jc = 64;
    const int ktiles = (int)((K + 63) / 64);
    p.kt = (int)((K + ktiles - 1) / ktiles);
    p.ktp = (p.kt + 3) / 4 * 4;
    p.ktiles = ktiles;
    p.nkg = p.ktp / 4;
    p.kc = 4 * std::max(8, std::min(kTtmMaxCols / 4, 512 / p.nkg));
  }
  p.ncg = p.kc / 4;
  p.threads = (p.nkg * p.ncg + 31) / 32 * 32;
  p.smem = ((size_t)p.jc * p.ktp + (size_t)p.jc * p.kc) * sizeof(double);
  int occ = occupancy(k_ttm<T, TX, DIFF>, p.threads, p.smem);
  const int64_t slots = (int64_t)dev.sms * occ;
  const int64_t chunks = (p.Kc + p.kc - 1) / p.kc;
  int64_t xs = std::max<int64_t>(1, slots / p.ktiles);
  xs = std::min(xs, chunks);
  const int64_t chunks_per = (chunks + xs - 1) / xs;
  p.cols_per_cta = chunks_per * p.kc;
  p.xsplit = (int)((p.Kc + p.cols_per_cta - 1) / p.cols_per_cta);
  return p;
}

template <typename K>
int set_smem(K kernel, size_t bytes, const DeviceInfo &dev) {
  if (bytes > (size_t)dev.smem_optin) {
    set_error("kernel needs %zu bytes of shared memory, device allows %d", bytes, dev.smem_optin);
    return TUCKER_EUNSUPPORTED;
  }
  TK_CUDA(allow_max_smem(kernel));
  return TUCKER_OK;
}

template <typename T>
int gram_typed(const T *y, int64_t L, int64_t J, int64_t B, double *d_S, double *d_ws, const DeviceInfo &dev,
               cudaStream_t s, Prof *prof) {
  GramPlan p = gram_plan(L, J, B, dev);
  TK_CHECK(set_smem(k_gram_partial<T>, p.smem, dev));
  const double flops = (double)J * (double)(J + 1) * (double)p.K;
  if (prof) prof->begin(TUCKER_PHASE_GRAM);
  if (p.K > 0) {
    k_gram_partial<T><<<dim3(p.groups, p.nsplit), p.threads, p.smem, s>>>(y, L, B, p, d_ws);
    TK_LAUNCHED();
  } else {
    TK_CUDA(cudaMemsetAsync(d_ws, 0, sizeof(double) * p.n_micro * 16, s));
    p.nsplit = 1;
  }
  if (prof) prof->end(flops, (double)p.K * J * sizeof(T) + (double)p.nsplit * p.n_micro * 16 * 8, 1);
  if (prof) prof->begin(TUCKER_PHASE_GRAM_REDUCE);
  const int64_t n = (int64_t)p.n_micro * 16;
  k_gram_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_ws, p, d_S);
  TK_LAUNCHED();
  if (prof) prof->end((double)p.nsplit * n, (double)p.nsplit * n * 8 + (double)J * J * 8, 1);
  return TUCKER_OK;
}

template <typename T>
int ttm_typed(const T *y, int64_t L, int64_t J, int64_t B, const double *a, int64_t ak, int64_t aj, int64_t K,
              double *z, const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  TtmPlan p = ttm_plan<T, double, false>(L, J, B, K, dev);
  TK_CHECK(set_smem(k_ttm<T, double, false>, p.smem, dev));
  if (prof) prof->begin(TUCKER_PHASE_TTM);
  if (p.Kc > 0) {
    k_ttm<T, double, false><<<dim3(p.xsplit, p.ktiles), p.threads, p.smem, s>>>(y, L, B, a, ak, aj, p, z,
                                                                                nullptr, nullptr);
    TK_LAUNCHED();
  }
  if (prof)
    prof->end(2.0 * J * K * (double)p.Kc, (double)p.Kc * (J * sizeof(T) + K * 8.0) + (double)J * K * 8, 1);
  return TUCKER_OK;
}

template <typename TX>
int ttm_diff_typed(const double *y, int64_t L, int64_t J, int64_t B, const double *a, int64_t ak, int64_t aj,
                   int64_t K, const TX *x, double *d_partials, double *d_out, const DeviceInfo &dev,
                   cudaStream_t s, Prof *prof) {
  TtmPlan p = ttm_plan<double, TX, true>(L, J, B, K, dev);
  TK_CHECK(set_smem(k_ttm<double, TX, true>, p.smem, dev));
  if (prof) prof->begin(TUCKER_PHASE_TTM);
  const int64_t np = (int64_t)p.xsplit * p.ktiles;
  if (p.Kc > 0) {
    k_ttm<double, TX, true><<<dim3(p.xsplit, p.ktiles), p.threads, p.smem, s>>>(y, L, B, a, ak, aj, p, nullptr,
                                                                                x, d_partials);
    TK_LAUNCHED();
  }
  k_sum_partials<<<1, 256, 0, s>>>(d_partials, p.Kc > 0 ? np : 0, d_out);
  TK_LAUNCHED();
  if (prof)
    prof->end(2.0 * J * K * (double)p.Kc + 3.0 * K * (double)p.Kc,
              (double)p.Kc * (J * 8.0 + K * sizeof(TX)) + (double)J * K * 8, 2);
  return TUCKER_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int64_t norm2_partials() { return kNormBlocks; }

int launch_norm2(const void *x, tucker_dtype dt, int64_t n, double *d_partials, double *d_out, cudaStream_t s,
                 Prof *prof) {
  const int64_t per_block = (int64_t)kNormThreads * 4;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(kNormBlocks, (n + per_block - 1) / per_block));
  if (prof) prof->begin(TUCKER_PHASE_NORM);
  if (dt == TUCKER_F64)
    k_sumsq<double><<<blocks, kNormThreads, 0, s>>>(static_cast<const double *>(x), n, d_partials);
  else
    k_sumsq<float><<<blocks, kNormThreads, 0, s>>>(static_cast<const float *>(x), n, d_partials);
  TK_LAUNCHED();
  k_sum_partials<<<1, 256, 0, s>>>(d_partials, blocks, d_out);
  TK_LAUNCHED();
  if (prof) prof->end(2.0 * n, (double)n * (dt == TUCKER_F64 ? 8 : 4), 2);
  return TUCKER_OK;
}

// ---------------------------------------------------------------------------
// float64 throughput probe: kPeakChains independent fused multiply-add chains
// per thread in registers (no memory traffic inside the loop), enough in
// flight to hide the pipe's latency; x <- x m + c with m < 1 stays bounded.
// The sum is stored so the loop is not removed.
// ---------------------------------------------------------------------------
namespace {
constexpr int kPeakChains = 8;
constexpr int kPeakIters = 4096;
constexpr int kPeakThreads = 512;

__global__ void __launch_bounds__(kPeakThreads) k_fp64_peak(double m, double c, double *__restrict__ out) {
  double x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 4
  for (int it = 0; it < kPeakIters; ++it)
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = fma(x[k], m, c);
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) t += x[k];
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}
}  // namespace

int fp64_peak(double *tflops, double *ms_out, const DeviceInfo &dev, cudaStream_t s) {
  int occ = 0;
  TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fp64_peak, kPeakThreads, 0));
  const int blocks = dev.sms * std::max(occ, 1) * 4;  // four full waves
  double *out = nullptr;
  TK_CUDA(cudaMallocAsync(&out, sizeof(double) * blocks, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = TUCKER_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("cudaEventCreate failed");
    st = TUCKER_ECUDA;
  }
  float ms = 0.f;
  for (int rep = 0; rep < 2 && st == TUCKER_OK; ++rep) {  // the first launch is untimed
    cudaEventRecord(e0, s);
    k_fp64_peak<<<blocks, kPeakThreads, 0, s>>>(0.999999, 1e-7, out);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("float64 probe launch failed");
      st = TUCKER_ECUDA;
      break;
    }
    bump_launches();
    cudaEventRecord(e1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      set_error("float64 probe timing failed");
      st = TUCKER_ECUDA;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (st != TUCKER_OK) return st;
  const double flops = 2.0 * kPeakChains * (double)kPeakIters * kPeakThreads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return TUCKER_OK;
}

int64_t gram_workspace_doubles(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev) {
  GramPlan p = gram_plan(L, J, B, dev);
  return (int64_t)std::max(p.nsplit, 1) * p.n_micro * 16;
}

int launch_gram(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *d_S, double *d_ws,
                const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (dt == TUCKER_F64) return gram_typed(static_cast<const double *>(y), L, J, B, d_S, d_ws, dev, s, prof);
  return gram_typed(static_cast<const float *>(y), L, J, B, d_S, d_ws, dev, s, prof);
}

int launch_ttm(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *a, int64_t ak,
               int64_t aj, int64_t K, double *z, const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (dt == TUCKER_F64)
    return ttm_typed(static_cast<const double *>(y), L, J, B, a, ak, aj, K, z, dev, s, prof);
  return ttm_typed(static_cast<const float *>(y), L, J, B, a, ak, aj, K, z, dev, s, prof);
}

int64_t ttm_diff_partials(int64_t L, int64_t J, int64_t B, int64_t K, const DeviceInfo &dev) {
  TtmPlan p = ttm_plan<double, double, true>(L, J, B, K, dev);
  TtmPlan q = ttm_plan<double, float, true>(L, J, B, K, dev);
  return std::max<int64_t>(1, std::max((int64_t)p.xsplit * p.ktiles, (int64_t)q.xsplit * q.ktiles));
}

int launch_ttm_diff(const double *y, int64_t L, int64_t J, int64_t B, const double *a, int64_t ak, int64_t aj,
                    int64_t K, const void *x, tucker_dtype xdt, double *d_partials, double *d_out,
                    const DeviceInfo &dev, cudaStream_t s, Prof *prof) {
  if (xdt == TUCKER_F64)
    return ttm_diff_typed(y, L, J, B, a, ak, aj, K, static_cast<const double *>(x), d_partials, d_out, dev, s,
                          prof);
  return ttm_diff_typed(y, L, J, B, a, ak, aj, K, static_cast<const float *>(x), d_partials, d_out, dev, s,
                        prof);
}

}  // namespace tk

// ---------------------------------------------------------------------------
// Gram step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose framework has already
// reserved nearly all of the GPU's memory for its own pool (a library
// allocation then fails or takes memory the pool counts on), and code that
// must not trigger the device-wide synchronisation cudaMalloc/cudaFree can
// cause.  tucker_gram_noalloc runs the same two kernels as tucker_gram, with
// the split-K partial sums in the file-scope array below instead of an
// allocation.  The array is TUCKER_NOALLOC_SCRATCH_BYTES (16 MiB) of device
// memory that every GPU which loads this library holds until the process
// exits.  Every call on a device shares it and it keeps the last call's
// partial sums; nothing in it has to start at zero, because each call writes
// every slot its reduction reads before reading it.  Two calls whose kernels
// overlap on the GPU (other streams, or other host threads) race on the
// array: order them on one stream or serialise them.
// ---------------------------------------------------------------------------
namespace tk {
namespace {

constexpr int64_t kNoallocDoubles = TUCKER_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array for the current device.  In host code
// the symbol names a host-side stand-in, so the address is looked up once per
// device (the first call on that device does it) and cached.
int noalloc_scratch(double **out) {
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return TUCKER_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the Gram scratch failed on device %d: %s", dev, cudaGetErrorString(e));
      return TUCKER_ECUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return TUCKER_OK;
}

template <typename T>
int gram_noalloc_typed(const T *y, int64_t L, int64_t J, int64_t B, double *d_S, const DeviceInfo &dev,
                       cudaStream_t s) {
  GramPlan p = gram_plan(L, J, B, dev);
  const int64_t per_split = (int64_t)p.n_micro * 16;
  const int64_t max_splits = kNoallocDoubles / per_split;
  if (max_splits < 1) {
    set_error("tucker_gram_noalloc: J = %lld needs %lld bytes of scratch for one split, the static scratch holds %lld",
              (long long)J, (long long)(per_split * 8), (long long)TUCKER_NOALLOC_SCRATCH_BYTES);
    return TUCKER_EINVAL;
  }
  const int planned = p.nsplit;
  if (p.nsplit > max_splits) {  // fewer, longer column ranges so the partials fit
    const int64_t chunks = (p.K + p.kc - 1) / p.kc;
    const int64_t chunks_per = (chunks + max_splits - 1) / max_splits;
    p.cols_per_split = chunks_per * p.kc;
    p.nsplit = (int)((p.K + p.cols_per_split - 1) / p.cols_per_split);
  }
  // TUCKER_NOALLOC_TRACE=1 prints the split plan (tests use it to reach the capped case)
  const char *trace = getenv("TUCKER_NOALLOC_TRACE");
  if (trace && trace[0] == '1')
    fprintf(stderr, "tucker_gram_noalloc: J=%lld planned_splits=%d scratch_fits=%lld used_splits=%d\n",
            (long long)J, planned, (long long)max_splits, p.nsplit);
  double *ws = nullptr;
  TK_CHECK(noalloc_scratch(&ws));
  TK_CHECK(set_smem(k_gram_partial<T>, p.smem, dev));
  k_gram_partial<T><<<dim3(p.groups, p.nsplit), p.threads, p.smem, s>>>(y, L, B, p, ws);
  TK_LAUNCHED();
  const int64_t n = per_split;
  k_gram_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ws, p, d_S);
  TK_LAUNCHED();
  return TUCKER_OK;
}

}  // namespace

}  // namespace tk

extern "C" int tucker_gram_noalloc(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S,
                                   void *stream) {
  using namespace tk;
  if (!Y || !S || L < 1 || B < 1 || (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("invalid arguments to tucker_gram_noalloc");
    return TUCKER_EINVAL;
  }
  if (J < 1 || J > TUCKER_MAX_DIM) {
    set_error("tucker_gram_noalloc: J = %lld outside [1, %d] (the static scratch is sized for J <= %d)",
              (long long)J, TUCKER_MAX_DIM, TUCKER_MAX_DIM);
    return TUCKER_EINVAL;
  }
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dt == TUCKER_F64) return gram_noalloc_typed(static_cast<const double *>(Y), L, J, B, S, dev, s);
  return gram_noalloc_typed(static_cast<const float *>(Y), L, J, B, S, dev, s);
}
