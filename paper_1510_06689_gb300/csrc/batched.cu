// Batched ST-HOSVD (Algorithm 1 on many independent small tensors) as a
// device pipeline: for each mode, every tensor's step runs in one launch per
// phase, and nothing returns to the host until all modes are done.
//
//   plan    one CTA: each tensor's view (L, J, B) of its current Y from the
//           ranks already chosen on the device, the work list of (tensor,
//           column range) items and each item's partial-sum slot
//   gram    persistent CTAs over the work list: float64 partial Grams of the
//           items (4 x 4 micro-tiles of the upper triangle, columns staged
//           in shared memory)
//   reduce  one CTA per tensor: S_t = sum of its items' partials (fixed
//           order), mirrored; at the first mode ||X_t||^2 = trace(S_t) and
//           the threshold eps^2 ||X_t||^2 / N
//   eig     one CTA per tensor and stage: float32 Jacobi, two float64
//           Newton-Schulz steps and X^T S X, float64 Jacobi (a few sweeps on
//           the nearly diagonal matrix), V = X W with the sign rule
//   rank    one thread per tensor: the rank rule of Algorithm 1 on the
//           eigenvalues, written into the tensor's current dims
//   ttm     persistent CTAs over the same work list: Y' = U^T Y for the
//           chosen R columns of U (U staged in shared memory)
//
// The launch shapes are fixed by host-side bounds (no truncation) and the
// kernels read the actual shapes from device memory, so the whole pipeline
// can be captured in one CUDA graph.  The columns per work item and the
// persistent grid are picked by a small autotuner on the first call for a
// batch shape (timed candidates on the first mode's Gram), then reused.
// Tensors with a mode longer than 128 take the per-tensor path instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace tk {

namespace {

constexpr int kBtMaxJ = 128;     // every mode of a batched tensor (the one-CTA Jacobi's limit)
constexpr int kBtThreads = 256;
constexpr int kBtStage = 32;     // columns staged in shared memory at a time
constexpr size_t kBtGramSmem = (size_t)2 * kBtStage * kBtMaxJ * sizeof(double);
static_assert(kBtThreads == 256 && kBtStage == 32 && kBtMaxJ <= 128,
              "the stage loader's fixed trip counts assume 8 warps, 32 columns and J <= 128");
constexpr int kBtMaxModes = TUCKER_MAX_MODES;

struct BtItem {
  int t;        // tensor
  int pad;
  int64_t c0, c1;  // columns [c0, c1) of the tensor's current unfolding
  int64_t poff;    // partial-sum slot (J_t^2 doubles)
};

// Per-tensor state on the device.
struct BtTensor {
  const void *x;      // input (dtype of the batch)
  int64_t yoff;       // offset of the tensor's region in each ping-pong buffer
  int dims[kBtMaxModes];
  int cur[kBtMaxModes];  // current dims: ranks of the modes done, dims of the others
  double nx2, thr;
  double tail[kBtMaxModes];
  int64_t L, J, B;    // the current mode's view
  int first, nitems;  // the current mode's items
  int keep_all;
};

// ---------------------------------------------------------------------------
// plan: one CTA of 1024 threads; items of tensor t are contiguous, in tensor
// order.  Writes the item count to *nitems (and an overflow flag past cap).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_bt_plan(BtTensor *__restrict__ T, int count, int N, int k, int64_t kc,
                                                  BtItem *__restrict__ items, int cap, int *__restrict__ nitems,
                                                  int *__restrict__ overflow) {
  __shared__ int64_t scan_i[1024], scan_p[1024];
  __shared__ int64_t base_i, base_p;
  const int tid = threadIdx.x;
  if (tid == 0) {
    base_i = 0;
    base_p = 0;
  }
  __syncthreads();
  for (int t0 = 0; t0 < count; t0 += 1024) {
    const int t = t0 + tid;
    int64_t ni = 0, np = 0, L = 1, B = 1, J = 1;
    if (t < count) {
      BtTensor &d = T[t];
      for (int m = 0; m < k; ++m) L *= d.cur[m];
      for (int m = k + 1; m < N; ++m) B *= d.cur[m];
      J = d.dims[k];
      ni = (L * B + kc - 1) / kc;
      np = ni * J * J;
      d.L = L;
      d.J = J;
      d.B = B;
    }
    scan_i[tid] = ni;
    scan_p[tid] = np;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scans
      const int64_t a = tid >= o ? scan_i[tid - o] : 0, b = tid >= o ? scan_p[tid - o] : 0;
      __syncthreads();
      scan_i[tid] += a;
      scan_p[tid] += b;
      __syncthreads();
    }
    if (t < count) {
      const int64_t first = base_i + scan_i[tid] - ni, poff0 = base_p + scan_p[tid] - np;
      BtTensor &d = T[t];
      d.first = (int)first;
      d.nitems = (int)ni;
      const int64_t K = L * B;
      for (int64_t i = 0; i < ni; ++i) {
        if (first + i >= cap) {
          *overflow = 1;
          break;
        }
        BtItem it;
        it.t = t;
        it.pad = 0;
        it.c0 = i * kc;
        it.c1 = min(K, (i + 1) * kc);
        it.poff = poff0 + i * J * J;
        items[first + i] = it;
      }
    }
    __syncthreads();
    if (tid == 1023) {
      base_i += scan_i[1023];
      base_p += scan_p[1023];
    }
    __syncthreads();
  }
  if (tid == 0) *nitems = (int)(base_i < cap ? base_i : (int64_t)cap);
}

// Columns kk of a stage as Ys[kk * ld + j] (j < J, zero up to ld), column c
// of the view at y + (c % L) + L J (c / L).
template <typename T>
__device__ __forceinline__ void bt_load_stage(const T *__restrict__ y, int64_t L, int J, int ld, int64_t c0,
                                              int64_t c1, double *Ys, int64_t *colbase) {
  const int tid = threadIdx.x;
  if (tid < kBtStage) {
    const int64_t c = c0 + tid;
    int64_t v = -1;
    if (c < c1) {
      const int64_t b = c / L;
      v = (c - b * L) + L * (int64_t)J * b;
    }
    colbase[tid] = v;
  }
  __syncthreads();
  // 16 loads in flight per thread before their shared-memory stores (ld <= 128)
  if (L == 1) {  // a column is J contiguous entries: a warp per column, lanes along j
    const int w = tid >> 5, lane = tid & 31;
    double v[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t base = colbase[w + 8 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = lane + 32 * i;
        v[q][i] = (j < J && base >= 0) ? (double)y[base + j] : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (lane + 32 * i < ld) Ys[(w + 8 * q) * ld + lane + 32 * i] = v[q][i];
  } else {  // a row segment runs along l: threads along the columns, rows j = tid / 32 + 8 i
    const int kk = tid & (kBtStage - 1), j0 = tid / kBtStage;
    const int64_t base = colbase[kk];
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int j = j0 + 8 * i;
      v[i] = (j < J && base >= 0) ? (double)y[base + L * (int64_t)j] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (j0 + 8 * i < ld) Ys[kk * ld + j0 + 8 * i] = v[i];
  }
  __syncthreads();
}

// The same stage in two halves, so that the next stage's loads are in flight
// while the current one is used: bt_fetch loads a thread's 16 entries of the
// stage at columns [c0, c1) into registers (the layout of bt_load_stage),
// bt_put stores them into Ys (row stride ld).
template <typename T>
__device__ __forceinline__ void bt_fetch(const T *__restrict__ y, int64_t L, int J, int64_t c0, int64_t c1,
                                         double (&v)[16]) {
  const int tid = threadIdx.x;
  if (L == 1) {
    const int w = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t c = c0 + w + 8 * q;
      const bool ok = c < c1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = lane + 32 * i;
        v[4 * q + i] = (ok && j < J) ? (double)y[c * (int64_t)J + j] : 0.0;
      }
    }
  } else {
    const int kk = tid & (kBtStage - 1), j0 = tid / kBtStage;
    const int64_t c = c0 + kk;
    const bool ok = c < c1;
    int64_t base = 0;
    if (ok) {
      const int64_t b = c / L;
      base = (c - b * L) + L * (int64_t)J * b;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int j = j0 + 8 * i;
      v[i] = (ok && j < J) ? (double)y[base + L * (int64_t)j] : 0.0;
    }
  }
}
__device__ __forceinline__ void bt_put(int64_t L, int ld, const double (&v)[16], double *Ys) {
  const int tid = threadIdx.x;
  if (L == 1) {
    const int w = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (lane + 32 * i < ld) Ys[(w + 8 * q) * ld + lane + 32 * i] = v[4 * q + i];
  } else {
    const int kk = tid & (kBtStage - 1), j0 = tid / kBtStage;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (j0 + 8 * i < ld) Ys[kk * ld + j0 + 8 * i] = v[i];
  }
}

// ---------------------------------------------------------------------------
// gram: persistent CTAs over the items.  Thread x owns the 4 x 4 micro-tiles
// x, x + 256, x + 512 of the upper triangle (at most 528 for J <= 128) and
// accumulates them over the item's columns, 32 at a time from shared memory;
// the item's partial is written in full 4 x 4 tiles (J x J, column-major).
// first_mode: the first mode reads the input (dtype T) in place, later modes
// the float64 Y of the previous mode (T = double).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBtThreads) k_bt_gram(const BtTensor *__restrict__ Tn, const BtItem *__restrict__ items,
                                                        const int *__restrict__ nitems, const double *__restrict__ ybuf,
                                                        int first_mode, double *__restrict__ partials) {
  extern __shared__ __align__(16) double gram_sm[];  // two stages (kBtGramSmem): one used, the next being filled
  const int n = *nitems, tid = threadIdx.x;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const BtItem item = items[it];
    const BtTensor &d = Tn[item.t];
    const int J = (int)d.J, Jp = (J + 3) & ~3, nmt = (Jp / 4) * (Jp / 4 + 1) / 2;
    const T *y = first_mode ? static_cast<const T *>(d.x) : reinterpret_cast<const T *>(ybuf + d.yoff);
    int ma[3], mb[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {  // micro-tile tid + 256 u -> (block row a <= block column b)
      const int m = tid + kBtThreads * u;
      ma[u] = mb[u] = -1;
      if (m < nmt) {
        int b = (int)((sqrtf(8.0f * (float)m + 1.0f) - 1.0f) * 0.5f);
        while ((b + 1) * (b + 2) / 2 <= m) ++b;
        while (b * (b + 1) / 2 > m) --b;
        ma[u] = m - b * (b + 1) / 2;
        mb[u] = b;
      }
    }
    double acc[3][16];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[u][e] = 0.0;
    // stage st is stored into buffer st & 1 after the barrier that ends the
    // use of stage st - 2 there (every thread has passed stage st - 1's barrier)
    double v[16];
    bt_fetch<T>(y, d.L, J, item.c0, min(item.c1, item.c0 + kBtStage), v);
    __syncthreads();  // the previous item's stages are read out
    int st = 0;
    for (int64_t c0 = item.c0; c0 < item.c1; c0 += kBtStage, ++st) {
      double *Ys = gram_sm + (st & 1) * (kBtStage * kBtMaxJ);
      bt_put(d.L, Jp, v, Ys);
      __syncthreads();
      if (c0 + kBtStage < item.c1)  // the next stage's loads run under this stage's FMAs
        bt_fetch<T>(y, d.L, J, c0 + kBtStage, min(item.c1, c0 + 2 * kBtStage), v);
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if (ma[u] < 0) continue;
        const double *pa = Ys + 4 * ma[u], *pb = Ys + 4 * mb[u];
        for (int kk = 0; kk < kBtStage; ++kk) {
          const double2 a01 = *reinterpret_cast<const double2 *>(pa + kk * Jp);
          const double2 a23 = *reinterpret_cast<const double2 *>(pa + kk * Jp + 2);
          const double2 b01 = *reinterpret_cast<const double2 *>(pb + kk * Jp);
          const double2 b23 = *reinterpret_cast<const double2 *>(pb + kk * Jp + 2);
          const double av[4] = {a01.x, a01.y, a23.x, a23.y}, bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[u][4 * r + c] = fma(av[r], bv[c], acc[u][4 * r + c]);
        }
      }
    }
    double *P = partials + item.poff;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (ma[u] < 0) continue;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = 4 * ma[u] + r, j = 4 * mb[u] + c;
          if (i < J && j < J) P[i + (int64_t)J * j] = acc[u][4 * r + c];
        }
    }
  }
}

// reduce: CTA t forms S_t (ld J, both triangles) from its items' partials in
// item order; at the first mode also ||X_t||^2 = trace(S_t), the threshold,
// and the eigensolver's budget (the threshold; -1 when every rank is kept).
__global__ void __launch_bounds__(kBtThreads) k_bt_reduce(BtTensor *__restrict__ Tn, const double *__restrict__ partials,
                                                          const BtItem *__restrict__ items, double *__restrict__ S,
                                                          int first_mode, double eps2_over_n,
                                                          double *__restrict__ budget) {
  __shared__ double red[kBtThreads / 32];
  BtTensor &d = Tn[blockIdx.x];
  const int J = (int)d.J;
  double *St = S + (int64_t)blockIdx.x * kBtMaxJ * kBtMaxJ;
  for (int e = threadIdx.x; e < J * J; e += kBtThreads) {
    const int i = e % J, j = e / J;
    if (i > j) continue;
    double v = 0.0;
    for (int q = 0; q < d.nitems; ++q) v += partials[items[d.first + q].poff + e];
    St[i + (int64_t)J * j] = v;
    St[j + (int64_t)J * i] = v;
  }
  if (!first_mode) return;
  __syncthreads();
  double t = 0.0;
  for (int i = threadIdx.x; i < J; i += kBtThreads) {
    double v = 0.0;
    for (int q = 0; q < d.nitems; ++q) v += partials[items[d.first + q].poff + i + (int64_t)J * i];
    t += v;
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBtThreads / 32; ++w) s += red[w];
    d.nx2 = s;
    d.thr = d.keep_all ? 0.0 : eps2_over_n * s;
    budget[blockIdx.x] = d.keep_all ? -1.0 : d.thr;
  }
}

// rank: thread t applies the rank rule of Algorithm 1 to tensor t's
// eigenvalues (descending) at mode k and makes R the mode's current dim.
__global__ void k_bt_rank(BtTensor *__restrict__ Tn, int count, int k, const double *__restrict__ lam) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  BtTensor &d = Tn[t];
  const int J = (int)d.J;
  const double *l = lam + (int64_t)t * kBtMaxJ;
  int best = J;
  double best_tail = 0.0;
  if (!d.keep_all) {
    double acc = 0.0;
    for (int r = J - 1; r >= 1; --r) {
      acc += fmax(l[r], 0.0);
      if (acc <= d.thr) {
        best = r;
        best_tail = acc;
      } else {
        break;
      }
    }
  }
  d.cur[k] = best;
  d.tail[k] = best_tail;
}

// ---------------------------------------------------------------------------
// ttm: persistent CTAs over the items: Y'_t[l + L (r + R b)] = sum_j U[j, r]
// Y_t[l + L (j + J b)] for r < R (R the tensor's rank at this mode, U the
// leading R eigenvectors).  U^T is staged as Us[j][r] (dynamic shared
// memory), the columns 32 at a time as in the Gram; thread x owns the 4 x 4
// output tile (rows 4 (x / 8) .., columns 4 (x % 8) ..) of a stage.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBtThreads) k_bt_ttm(const BtTensor *__restrict__ Tn, const BtItem *__restrict__ items,
                                                       const int *__restrict__ nitems, int k,
                                                       const double *__restrict__ ybuf_in, int first_mode,
                                                       const double *__restrict__ V, double *__restrict__ ybuf_out) {
  extern __shared__ __align__(16) double Us[];  // [J][Rp]
  __shared__ __align__(16) double Ys[kBtStage * kBtMaxJ];
  __shared__ int64_t colbase[kBtStage];
  const int n = *nitems, tid = threadIdx.x;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const BtItem item = items[it];
    const BtTensor &d = Tn[item.t];
    const int J = (int)d.J, Jp = (J + 3) & ~3, R = d.cur[k], Rp = (R + 3) & ~3;
    const int64_t L = d.L;
    const T *y = first_mode ? static_cast<const T *>(d.x) : reinterpret_cast<const T *>(ybuf_in + d.yoff);
    double *z = ybuf_out + d.yoff;
    const double *Ut = V + (int64_t)item.t * kBtMaxJ * kBtMaxJ;
    __syncthreads();  // the previous item's reads of Us are done
    for (int e = tid; e < J * Rp; e += kBtThreads) {
      const int j = e / Rp, r = e - j * Rp;
      Us[e] = r < R ? Ut[j + (int64_t)J * r] : 0.0;
    }
    // thread (split sp, rows 4 rt.., stage columns 4 ct..): with few rows the
    // contraction over j is split sp_n ways so that every thread works, the
    // partial tiles summed through shared memory in split order
    const int combos = ((R + 3) >> 2) * 8;
    int sp_n = 1;
    while (sp_n < 8 && 2 * sp_n * combos <= kBtThreads) sp_n *= 2;
    const int sp = tid / combos, rest = tid - sp * combos;
    const int rt = rest >> 3, ct = rest & 7;  // 4 rows r, 4 stage columns
    const bool active = sp < sp_n;
    const int jlo = J * sp / sp_n, jhi = J * (sp + 1) / sp_n;
    for (int64_t c0 = item.c0; c0 < item.c1; c0 += kBtStage) {
      bt_load_stage<T>(y, L, J, Jp, c0, min(item.c1, c0 + kBtStage), Ys, colbase);  // (its barriers cover Us too)
      double acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
      if (active) {
        const double *pu = Us + 4 * rt;
        const double *py = Ys + 4 * ct * Jp;
        for (int j = jlo; j < jhi; ++j) {
          const double2 u01 = *reinterpret_cast<const double2 *>(pu + j * Rp);
          const double2 u23 = *reinterpret_cast<const double2 *>(pu + j * Rp + 2);
          const double uv[4] = {u01.x, u01.y, u23.x, u23.y};
          const double yv[4] = {py[j], py[Jp + j], py[2 * Jp + j], py[3 * Jp + j]};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(uv[a], yv[b], acc[a][b]);
        }
      }
      if (sp_n > 1) {  // uniform over the CTA (one item at a time)
        __syncthreads();  // the stage has been read: its buffer takes the partial tiles
        double *red = Ys;  // sp_n x combos tiles of 16 <= kBtStage x kBtMaxJ doubles
        if (active && sp > 0)
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) red[(sp * combos + rest) * 16 + 4 * a + b] = acc[a][b];
        __syncthreads();
        if (sp == 0)
          for (int s2 = 1; s2 < sp_n; ++s2)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) acc[a][b] += red[(s2 * combos + rest) * 16 + 4 * a + b];
      }
      if (active && sp == 0) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int64_t c = c0 + 4 * ct + b;
          if (c >= item.c1) continue;
          const int64_t bb = c / L, l = c - bb * L;
          const int64_t ob = l + L * (int64_t)R * bb;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int r = 4 * rt + a;
            if (r < R) z[ob + L * (int64_t)r] = acc[a][b];
          }
        }
      }
      __syncthreads();
    }
  }
}

// C = op(A) B for J x J matrices (ld J) by the whole CTA, entries spread over
// its threads; op(A) = A^T when transA.  Operands may have been written
// earlier by this CTA (plain loads, after a barrier).
// C = op(A) B for J x J column-major matrices (J <= 128; op(A) = A or A^T),
// by the whole CTA: panels of 32 k of op(A) and B pass through shared memory
// k-major (row stride J4 + 2 = padded J rounded to 4, plus 2), and each thread
// accumulates up to four 4 x 4 tiles of C in registers (8 shared loads per 16
// FMAs), so the float64 pipe, not the loads, bounds it.  `sm` holds 2 x 32 x
// (J4 + 2) doubles.  Ends with a barrier (C complete).
constexpr int kGemmK = 32;
constexpr size_t kGemmSmem = (size_t)2 * kGemmK * (kBtMaxJ + 2) * sizeof(double);
__device__ void bt_gemm(int J, const double *A, int transA, const double *B, double *C, double *sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int J4 = (J + 3) & ~3, ld = J4 + 2, tn = J4 / 4, ntiles = tn * tn;
  double *Ap = sm, *Bp = sm + kGemmK * ld;
  double acc[4][16];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[u][e] = 0.0;
  for (int k0 = 0; k0 < J4; k0 += kGemmK) {
    __syncthreads();  // the previous panels are read out
    for (int e = tid; e < kGemmK * J4; e += nt) {
      // op(A)[i][k0 + kk] -> Ap[kk][i]: k fastest for A^T (contiguous in memory), i fastest for A
      int i, kk;
      if (transA) {
        i = e / kGemmK;
        kk = e - i * kGemmK;
      } else {
        kk = e / J4;
        i = e - kk * J4;
      }
      const int k = k0 + kk;
      double a = 0.0;
      if (i < J && k < J) a = transA ? A[k + (int64_t)J * i] : A[i + (int64_t)J * k];
      Ap[kk * ld + i] = a;
    }
    for (int e = tid; e < kGemmK * J4; e += nt) {  // B[k0 + kk][j] -> Bp[kk][j], k fastest
      const int j = e / kGemmK, kk = e - j * kGemmK, k = k0 + kk;
      Bp[kk * ld + j] = (j < J && k < J) ? B[k + (int64_t)J * j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int tile = tid + u * nt;
      if (tile >= ntiles) break;
      const int ti = tile % tn, tj = tile / tn;
      const double *pa = Ap + 4 * ti, *pb = Bp + 4 * tj;
#pragma unroll 4
      for (int kk = 0; kk < kGemmK; ++kk) {
        const double2 a01 = *reinterpret_cast<const double2 *>(pa + kk * ld);
        const double2 a23 = *reinterpret_cast<const double2 *>(pa + kk * ld + 2);
        const double2 b01 = *reinterpret_cast<const double2 *>(pb + kk * ld);
        const double2 b23 = *reinterpret_cast<const double2 *>(pb + kk * ld + 2);
        const double av[4] = {a01.x, a01.y, a23.x, a23.y}, bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[u][4 * c + r] = fma(av[r], bv[c], acc[u][4 * c + r]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int tile = tid + u * nt;
    if (tile >= ntiles) break;
    const int ti = tile % tn, tj = tile / tn;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = 4 * ti + r, j = 4 * tj + c;
        if (i < J && j < J) C[i + (int64_t)J * j] = acc[u][4 * c + r];
      }
  }
  __syncthreads();
}

// Between the float32 and float64 Jacobi stages, CTA t: X (the float32
// stage's vectors, orthonormal to ~1e-6) gets two Newton-Schulz steps
// X <- X (3 I - X^T X) / 2 in float64 (orthonormal to rounding: the similarity
// below then keeps the eigenvalues), and S2 = X^T S X, nearly diagonal, for
// the float64 Jacobi, which then needs few sweeps.  W is scratch.
__global__ void __launch_bounds__(kBtThreads) k_bt_presolve(const BtTensor *__restrict__ Tn, const double *__restrict__ S,
                                                            double *__restrict__ X, double *__restrict__ W,
                                                            double *__restrict__ S2) {
  extern __shared__ __align__(16) double gsm[];
  const int t = blockIdx.x, J = (int)Tn[t].J;
  const int64_t o = (int64_t)t * kBtMaxJ * kBtMaxJ;
  double *Xt = X + o, *Wt = W + o, *S2t = S2 + o;
  const double *St = S + o;
  for (int it = 0; it < 2; ++it) {
    bt_gemm(J, Xt, 1, Xt, Wt, gsm);  // P = X^T X
    for (int e = threadIdx.x; e < J * J; e += blockDim.x) Wt[e] = (e % J == e / J ? 1.5 : 0.0) - 0.5 * Wt[e];
    __syncthreads();
    bt_gemm(J, Xt, 0, Wt, S2t, gsm);  // X P into S2, then back to X
    for (int e = threadIdx.x; e < J * J; e += blockDim.x) Xt[e] = S2t[e];
    __syncthreads();
  }
  bt_gemm(J, St, 0, Xt, Wt, gsm);   // S X
  bt_gemm(J, Xt, 1, Wt, S2t, gsm);  // X^T S X
}

// After the float64 Jacobi (W = its eigenvectors of S2, sorted with their
// eigenvalues, descending): V = X W, then the sign rule (the largest-magnitude
// entry of a column positive, the lowest row on ties).
__global__ void __launch_bounds__(kBtThreads) k_bt_backsolve(const BtTensor *__restrict__ Tn, const double *__restrict__ X,
                                                             const double *__restrict__ W, double *__restrict__ V) {
  extern __shared__ __align__(16) double gsm[];
  const int t = blockIdx.x, J = (int)Tn[t].J;
  const int64_t o = (int64_t)t * kBtMaxJ * kBtMaxJ;
  double *Vt = V + o;
  bt_gemm(J, X + o, 0, W + o, Vt, gsm);
  for (int r = threadIdx.x; r < J; r += blockDim.x) {
    double *col = Vt + (int64_t)J * r;
    double best = -1.0;
    int br = 0;
    for (int i = 0; i < J; ++i) {
      const double v = fabs(col[i]);
      if (v > best) {
        best = v;
        br = i;
      }
    }
    if (col[br] < 0.0)
      for (int i = 0; i < J; ++i) col[i] = -col[i];
  }
}

// collect: CTA t copies its core (the final Y, prod R doubles) and every
// factor U_k = the first R_k columns of mode k's eigenvectors (I_k x R_k,
// column-major) into the result block at the host-given offsets.
__global__ void __launch_bounds__(kBtThreads) k_bt_collect(const BtTensor *__restrict__ Tn, int N,
                                                           const double *__restrict__ ybuf_final,
                                                           const double *__restrict__ Vall, int64_t vstride,
                                                           const int64_t *__restrict__ offs, double *__restrict__ block) {
  const int t = blockIdx.x;
  const BtTensor &d = Tn[t];
  const int64_t *o = offs + (int64_t)t * (N + 1);
  int64_t ncore = 1;
  for (int m = 0; m < N; ++m) ncore *= d.cur[m];
  for (int64_t e = threadIdx.x; e < ncore; e += kBtThreads) block[o[0] + e] = ybuf_final[d.yoff + e];
  for (int m = 0; m < N; ++m) {
    const int I = d.dims[m], R = d.cur[m];
    const double *Vm = Vall + m * vstride + (int64_t)t * kBtMaxJ * kBtMaxJ;
    for (int e = threadIdx.x; e < I * R; e += kBtThreads) block[o[m + 1] + e] = Vm[e];  // ld I: columns contiguous
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
namespace {

struct BtTuning {
  int64_t kc = 2048;  // columns per work item
  int grid = 0;       // persistent CTAs of the Gram and TTM
  float ms[6] = {0};  // the candidates' times (kc 512 / 2048 / 8192 x grid 2 / 4 per SM)
};
std::mutex g_bt_mu;
std::map<std::tuple<int, int, int64_t, int>, BtTuning> g_bt_tuned;  // (count, N, total size, max dim)
BtTuning g_bt_last;

struct BtArena {
  BtTensor *T;
  BtItem *items;
  int *nitems, *overflow;
  double *partials, *ybuf[2], *S, *lam, *V;
  double *X, *W, *S2;  // the eigensolver's float32-stage vectors, scratch, and X^T S X
  int *info;       // 4 ints per tensor and mode (launch_eig_batched)
  double *budget;  // per tensor: the rank rule's threshold, -1 when every rank is kept
  const double **Sp, **S2p;
  double **lamp, **Xp, **Wp;
  int *Js;
  // the eigensolver's size classes: mode k, class c covers J in (32 c, 32 (c + 1)]:
  // tensors cidx[coff[k][c] .. coff[k][c + 1])
  int *cidx;
  std::vector<std::vector<int>> coff;
};
constexpr int kBtClasses = 4;
constexpr int kBtEigThreads = 256;

template <typename T>
int bt_run_mode(const BtArena &a, int count, int N, int k, int64_t kc, int cap, int grid, size_t ttm_smem,
                double eps2_over_n, int maxJk, cudaStream_t s, Prof *prof) {
  if (prof) prof->begin(TUCKER_PHASE_GRAM);
  k_bt_plan<<<1, 1024, 0, s>>>(a.T, count, N, k, kc, a.items, cap, a.nitems, a.overflow);
  TK_LAUNCHED();
  const double *yin = k == 0 ? nullptr : a.ybuf[(k - 1) & 1];
  if (k == 0) k_bt_gram<T><<<grid, kBtThreads, kBtGramSmem, s>>>(a.T, a.items, a.nitems, yin, 1, a.partials);
  else k_bt_gram<double><<<grid, kBtThreads, kBtGramSmem, s>>>(a.T, a.items, a.nitems, yin, 0, a.partials);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, 0.0, 2);
  if (prof) prof->begin(TUCKER_PHASE_GRAM_REDUCE);
  k_bt_reduce<<<count, kBtThreads, 0, s>>>(a.T, a.partials, a.items, a.S, k == 0, eps2_over_n, a.budget);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, 0.0, 1);
  if (prof) prof->begin(TUCKER_PHASE_EIG);
  // float32 Jacobi -> float64 orthonormalisation and X^T S X -> float64 Jacobi -> V = X W
  const int *Jk = a.Js + (int64_t)k * count;
  (void)maxJk;
  // per size class: CTAs sized for the class (several per SM for small J)
  for (int c = 0; c < kBtClasses; ++c) {
    const int n = a.coff[k][c + 1] - a.coff[k][c];
    if (n > 0)
      TK_CHECK(launch_jacobi32_batched(a.Sp, Jk, a.Xp, n, 32 * (c + 1), s, a.cidx + a.coff[k][c], kBtEigThreads));
  }
  k_bt_presolve<<<count, kBtThreads, kGemmSmem, s>>>(a.T, a.S, a.X, a.W, a.S2);
  TK_LAUNCHED();
  for (int c = 0; c < kBtClasses; ++c) {
    const int n = a.coff[k][c + 1] - a.coff[k][c];
    if (n > 0)
      TK_CHECK(launch_eig_batched(a.S2p, Jk, a.lamp + (int64_t)k * count, a.Wp, a.info + (int64_t)k * 4 * count, n,
                                  32 * (c + 1), s, a.cidx + a.coff[k][c], kBtEigThreads, a.budget));
  }
  k_bt_backsolve<<<count, kBtThreads, kGemmSmem, s>>>(a.T, a.X, a.W, a.V + (int64_t)k * count * kBtMaxJ * kBtMaxJ);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, 0.0, 4);
  if (prof) prof->begin(TUCKER_PHASE_RANK);
  k_bt_rank<<<(count + 127) / 128, 128, 0, s>>>(a.T, count, k, a.lam + (int64_t)k * count * kBtMaxJ);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, 0.0, 1);
  if (prof) prof->begin(TUCKER_PHASE_TTM);
  const double *Vk = a.V + (int64_t)k * count * kBtMaxJ * kBtMaxJ;
  if (k == 0) k_bt_ttm<T><<<grid, kBtThreads, ttm_smem, s>>>(a.T, a.items, a.nitems, k, yin, 1, Vk, a.ybuf[k & 1]);
  else k_bt_ttm<double><<<grid, kBtThreads, ttm_smem, s>>>(a.T, a.items, a.nitems, k, yin, 0, Vk, a.ybuf[k & 1]);
  TK_LAUNCHED();
  if (prof) prof->end(0.0, 0.0, 1);
  return TUCKER_OK;
}

template <typename T>
int bt_impl(const void *const *X, tucker_dtype dt, const int64_t *dims, int N, int count, double eps, cudaStream_t s,
            tucker_result *out) {
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  // host-side bounds: no truncation
  int64_t total = 0, maxI = 1;
  int maxJ = 1;
  std::vector<int64_t> yoff(count);
  std::vector<int> maxJk(N, 1);
  for (int t = 0; t < count; ++t) {
    int64_t I = 1;
    for (int m = 0; m < N; ++m) {
      I *= dims[(int64_t)t * N + m];
      maxJ = std::max(maxJ, (int)dims[(int64_t)t * N + m]);
      maxJk[m] = std::max(maxJk[m], (int)dims[(int64_t)t * N + m]);
    }
    yoff[t] = total;
    total += I;
    maxI = std::max(maxI, I);
  }
  constexpr int64_t kCands[3] = {512, 2048, 8192};
  auto bounds = [&](int64_t kc, int64_t *cap, int64_t *pcap) {
    *cap = *pcap = 0;
    for (int m = 0; m < N; ++m) {
      int64_t ci = 0, cp = 0;
      for (int t = 0; t < count; ++t) {
        int64_t I = 1;
        for (int q = 0; q < N; ++q) I *= dims[(int64_t)t * N + q];
        const int64_t J = dims[(int64_t)t * N + m], K = I / J, ni = (K + kc - 1) / kc;
        ci += ni;
        cp += ni * J * J;
      }
      *cap = std::max(*cap, ci);
      *pcap = std::max(*pcap, cp);
    }
  };
  int64_t cap = 0, pcap = 0;
  bounds(kCands[0], &cap, &pcap);  // the smallest items need the most slots
  if (cap > 0x7FFFFFFFll) {
    set_error("batched ST-HOSVD: too many work items");
    return TUCKER_EUNSUPPORTED;
  }
  // one arena for the pipeline
  auto al = [](int64_t bytes) { return (bytes + 255) / 256 * 256; };
  const int64_t mats = (int64_t)count * kBtMaxJ * kBtMaxJ;
  const int64_t sz_T = al(sizeof(BtTensor) * count), sz_items = al(sizeof(BtItem) * cap), sz_ints = 256,
                sz_part = al(8 * pcap), sz_y = al(8 * total), sz_S = al(8 * mats), sz_lam = al(8 * (int64_t)N * count * kBtMaxJ),
                sz_V = al(8 * (int64_t)N * mats), sz_info = al(4 * 4 * (int64_t)N * count), sz_budget = al(8 * (int64_t)count),
                sz_ptr = al(8 * (int64_t)count), sz_ptrN = al(8 * (int64_t)N * count), sz_Js = al(4 * (int64_t)N * count),
                sz_offs = al(8 * (int64_t)count * (N + 1)), sz_cidx = al(4 * (int64_t)N * count);
  const int64_t bytes = sz_T + sz_items + sz_ints + sz_part + 2 * sz_y + 4 * sz_S + sz_lam + sz_V + sz_info + sz_budget +
                        4 * sz_ptr + sz_ptrN + sz_Js + sz_offs + sz_cidx;
  char *base = nullptr;
  {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("batched ST-HOSVD: cudaMallocAsync(%lld bytes) failed: %s", (long long)bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA;
    }
  }
  struct Free {
    void *p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } guard{base, s};
  BtArena a;
  char *q = base;
  auto take = [&](int64_t n) {
    char *r = q;
    q += n;
    return r;
  };
  a.T = reinterpret_cast<BtTensor *>(take(sz_T));
  a.items = reinterpret_cast<BtItem *>(take(sz_items));
  a.nitems = reinterpret_cast<int *>(take(sz_ints));
  a.overflow = a.nitems + 1;
  a.partials = reinterpret_cast<double *>(take(sz_part));
  a.ybuf[0] = reinterpret_cast<double *>(take(sz_y));
  a.ybuf[1] = reinterpret_cast<double *>(take(sz_y));
  a.S = reinterpret_cast<double *>(take(sz_S));
  a.X = reinterpret_cast<double *>(take(sz_S));
  a.W = reinterpret_cast<double *>(take(sz_S));
  a.S2 = reinterpret_cast<double *>(take(sz_S));
  a.lam = reinterpret_cast<double *>(take(sz_lam));
  a.V = reinterpret_cast<double *>(take(sz_V));
  a.info = reinterpret_cast<int *>(take(sz_info));
  a.budget = reinterpret_cast<double *>(take(sz_budget));
  a.Sp = reinterpret_cast<const double **>(take(sz_ptr));
  a.S2p = reinterpret_cast<const double **>(take(sz_ptr));
  a.Xp = reinterpret_cast<double **>(take(sz_ptr));
  a.Wp = reinterpret_cast<double **>(take(sz_ptr));
  a.lamp = reinterpret_cast<double **>(take(sz_ptrN));
  a.Js = reinterpret_cast<int *>(take(sz_Js));
  int64_t *doffs = reinterpret_cast<int64_t *>(take(sz_offs));
  a.cidx = reinterpret_cast<int *>(take(sz_cidx));
  // tensors and the eigensolver's per-matrix arrays
  {
    std::vector<BtTensor> ht(count);
    std::vector<const double *> sp(count), s2p(count);
    std::vector<double *> xp(count), wp(count), lp((size_t)N * count);
    std::vector<int> js((size_t)N * count);
    for (int t = 0; t < count; ++t) {
      BtTensor &d = ht[t];
      memset(&d, 0, sizeof d);
      d.x = X[t];
      d.yoff = yoff[t];
      for (int m = 0; m < N; ++m) d.dims[m] = d.cur[m] = (int)dims[(int64_t)t * N + m];
      d.keep_all = !(eps > 0.0);
      const int64_t o = (int64_t)t * kBtMaxJ * kBtMaxJ;
      sp[t] = a.S + o;
      s2p[t] = a.S2 + o;
      xp[t] = a.X + o;
      wp[t] = a.W + o;
      for (int m = 0; m < N; ++m) {
        lp[(size_t)m * count + t] = a.lam + ((int64_t)m * count + t) * kBtMaxJ;
        js[(size_t)m * count + t] = d.dims[m];
      }
    }
    TK_CUDA(cudaMemcpyAsync(a.T, ht.data(), sizeof(BtTensor) * count, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(a.Sp, sp.data(), sizeof(void *) * count, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(a.S2p, s2p.data(), sizeof(void *) * count, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(a.Xp, xp.data(), sizeof(void *) * count, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(a.Wp, wp.data(), sizeof(void *) * count, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(a.lamp, lp.data(), sizeof(void *) * N * count, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(a.Js, js.data(), sizeof(int) * N * count, cudaMemcpyHostToDevice, s));
    // size classes of every mode (the dims, not the ranks, fix them)
    std::vector<int> cidx;
    a.coff.assign(N, std::vector<int>(kBtClasses + 1, 0));
    for (int m = 0; m < N; ++m) {
      for (int c = 0; c < kBtClasses; ++c) {
        a.coff[m][c] = (int)cidx.size();
        for (int t = 0; t < count; ++t) {
          const int J = ht[t].dims[m];
          if (J > 32 * c && J <= 32 * (c + 1)) cidx.push_back(t);
        }
      }
      a.coff[m][kBtClasses] = (int)cidx.size();
    }
    TK_CUDA(cudaMemcpyAsync(a.cidx, cidx.data(), sizeof(int) * cidx.size(), cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemsetAsync(a.overflow, 0, sizeof(int), s));
    TK_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  }
  const size_t ttm_smem = (size_t)maxJ * ((maxJ + 3) & ~3) * sizeof(double);
  TK_CUDA(cudaFuncSetAttribute(k_bt_ttm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ttm_smem));
  TK_CUDA(cudaFuncSetAttribute(k_bt_ttm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ttm_smem));
  TK_CUDA(cudaFuncSetAttribute(k_bt_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBtGramSmem));
  TK_CUDA(cudaFuncSetAttribute(k_bt_gram<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBtGramSmem));
  TK_CUDA(cudaFuncSetAttribute(k_bt_presolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
  TK_CUDA(cudaFuncSetAttribute(k_bt_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
  const double eps2_over_n = eps > 0.0 ? eps * eps / N : 0.0;

  // autotuner: columns per item and persistent grid, timed on the first mode's Gram
  BtTuning tune;
  const auto key = std::make_tuple(count, N, total, maxJ);
  {
    std::lock_guard<std::mutex> lock(g_bt_mu);
    auto it = g_bt_tuned.find(key);
    if (it != g_bt_tuned.end()) tune = it->second;
  }
  if (tune.grid == 0) {
    cudaEvent_t e0, e1;
    TK_CUDA(cudaEventCreate(&e0));
    TK_CUDA(cudaEventCreate(&e1));
    float best = -1.f;
    int ci = 0;
    for (int64_t kc : kCands)
      for (int per : {2, 4}) {
        const int grid = dev.sms * per;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {  // the second run is timed
          cudaEventRecord(e0, s);
          k_bt_plan<<<1, 1024, 0, s>>>(a.T, count, N, 0, kc, a.items, (int)cap, a.nitems, a.overflow);
          k_bt_gram<T><<<grid, kBtThreads, kBtGramSmem, s>>>(a.T, a.items, a.nitems, nullptr, 1, a.partials);
          cudaEventRecord(e1, s);
          bump_launches(2);
          TK_CUDA(cudaGetLastError());
          TK_CUDA(cudaEventSynchronize(e1));
          TK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        }
        tune.ms[ci++] = ms;
        if (best < 0.f || ms < best) {
          best = ms;
          tune.kc = kc;
          tune.grid = grid;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_bt_mu);
    g_bt_tuned[key] = tune;
  }
  {
    std::lock_guard<std::mutex> lock(g_bt_mu);
    g_bt_last = tune;
  }

  // the pipeline: every mode's phases, captured in one graph (launched directly if
  // capture fails, or with phase timing on)
  Prof prof(s);
  auto enqueue = [&](Prof *pr) -> int {
    for (int k = 0; k < N; ++k)
      TK_CHECK(bt_run_mode<T>(a, count, N, k, tune.kc, (int)cap, tune.grid, ttm_smem, eps2_over_n, maxJk[k], s, pr));
    return TUCKER_OK;
  };
  bool done = false;
  if (prof.on) {
    TK_CHECK(enqueue(&prof));
    done = true;
  } else {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int st = enqueue(nullptr);
      const cudaError_t ce = cudaStreamEndCapture(s, &g);
      cudaGraphExec_t ge = nullptr;
      if (st == TUCKER_OK && ce == cudaSuccess && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
        done = cudaGraphLaunch(ge, s) == cudaSuccess;
        cudaGraphExecDestroy(ge);
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
  }
  if (!done) TK_CHECK(enqueue(nullptr));

  // results: ranks and spectra to the host, then one block for every core and factor
  std::vector<BtTensor> ht(count);
  std::vector<double> hlam((size_t)N * count * kBtMaxJ);
  std::vector<int> hinfo((size_t)4 * N * count);
  int overflow = 0;
  TK_CUDA(cudaMemcpyAsync(ht.data(), a.T, sizeof(BtTensor) * count, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(hlam.data(), a.lam, sizeof(double) * hlam.size(), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(hinfo.data(), a.info, sizeof(int) * hinfo.size(), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(&overflow, a.overflow, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (overflow) {
    set_error("batched ST-HOSVD: work list overflow");
    return TUCKER_ECUDA;
  }
  for (int m = 0; m < N; ++m)
    for (int t = 0; t < count; ++t)
      if (hinfo[4 * ((size_t)m * count + t) + 1] != 0) {
        set_error("batched ST-HOSVD: Jacobi did not converge (tensor %d, mode %d)", t, m);
        return TUCKER_ENOCONV;
      }
  std::vector<int64_t> offs((size_t)count * (N + 1));
  int64_t btotal = 0;
  for (int t = 0; t < count; ++t) {
    int64_t nc = 1;
    for (int m = 0; m < N; ++m) nc *= ht[t].cur[m];
    offs[(size_t)t * (N + 1)] = btotal;
    btotal += nc;
    for (int m = 0; m < N; ++m) {
      offs[(size_t)t * (N + 1) + m + 1] = btotal;
      btotal += (int64_t)ht[t].dims[m] * ht[t].cur[m];
    }
  }
  void *blk = nullptr;
  {
    cudaError_t e = cudaMalloc(&blk, sizeof(double) * std::max<int64_t>(btotal, 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("batched ST-HOSVD: result allocation failed: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA;
    }
  }
  std::shared_ptr<void> block(blk, [](void *p) { cudaFree(p); });
  TK_CUDA(cudaMemcpyAsync(doffs, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice, s));
  k_bt_collect<<<count, kBtThreads, 0, s>>>(a.T, N, a.ybuf[(N - 1) & 1], a.V, (int64_t)count * kBtMaxJ * kBtMaxJ,
                                            doffs, static_cast<double *>(blk));
  TK_LAUNCHED();
  TK_CUDA(cudaStreamSynchronize(s));
  int device = 0;
  cudaGetDevice(&device);
  for (int t = 0; t < count; ++t) {
    tucker_result &r = out[t];
    memset(&r, 0, sizeof r);
    r.N = N;
    r.on_host = 0;
    r.norm2_x = ht[t].nx2;
    r.threshold = ht[t].thr;
    r.core = static_cast<double *>(blk) + offs[(size_t)t * (N + 1)];
    for (int m = 0; m < N; ++m) {
      const int I = ht[t].dims[m];
      r.dims[m] = I;
      r.ranks[m] = ht[t].cur[m];
      r.mode_order[m] = m;
      r.sweeps[m] = hinfo[4 * ((size_t)m * count + t)];
      r.tail[m] = ht[t].tail[m];
      r.eig_path[m] = TUCKER_EIG_JACOBI;
      r.eig_resolved[m] = I - hinfo[4 * ((size_t)m * count + t) + 2];
      r.factors[m] = static_cast<double *>(blk) + offs[(size_t)t * (N + 1) + m + 1];
      r.eigvals[m] = static_cast<double *>(malloc(sizeof(double) * I));
      if (!r.eigvals[m]) {
        set_error("host allocation failed");
        return TUCKER_ENOMEM;  // the caller releases out[]
      }
      memcpy(r.eigvals[m], hlam.data() + ((size_t)m * count + t) * kBtMaxJ, sizeof(double) * I);
    }
    ResultPriv *pv = new ResultPriv;
    pv->device = device;
    pv->block = block;
    r.priv = pv;
  }
  return TUCKER_OK;
}

}  // namespace

int sthosvd_batched_device(const void *const *X, tucker_dtype dt, const int64_t *dims, int N, int count, double eps,
                           cudaStream_t s, tucker_result *out, int *handled) {
  *handled = 0;
  const char *e = getenv("TUCKER_BATCH");
  if (e && strcmp(e, "threads") == 0) return TUCKER_OK;  // the per-tensor path on host worker threads
  if (count < 1 || N > kBtMaxModes) return TUCKER_OK;
  for (int64_t i = 0; i < (int64_t)count * N; ++i)
    if (dims[i] > kBtMaxJ) return TUCKER_OK;
  *handled = 1;
  if (dt == TUCKER_F64) return bt_impl<double>(X, dt, dims, N, count, eps, s, out);
  return bt_impl<float>(X, dt, dims, N, count, eps, s, out);
}

// The last batched call's tuning: columns per work item, persistent CTAs and
// the candidates' times (ms).
void batched_last_tuning(int64_t *kc, int *grid, float *ms6) {
  std::lock_guard<std::mutex> lock(g_bt_mu);
  if (kc) *kc = g_bt_last.kc;
  if (grid) *grid = g_bt_last.grid;
  if (ms6) memcpy(ms6, g_bt_last.ms, sizeof g_bt_last.ms);
}

}  // namespace tk
