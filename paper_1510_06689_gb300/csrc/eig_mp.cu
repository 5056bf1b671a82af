// Mixed-precision eigensolver for the eigenvector step of Algorithm 1
// (Sec. 2.2; the paper calls LAPACK's dsyevx, Sec. 4.4, Algorithm 5).
//
// GB300's float64 pipe issues ~2 FMAs per clock per SM, so a float64 Jacobi
// of a 128 x 128 Gram (18 sweeps of 127 dependent steps) is bound by latency
// and float64 throughput at once.  This solver moves the sweeps to float32
// and restores float64 accuracy with matrix products spread over all SMs:
//
//   level(A):  (A symmetric m x m, float64)
//     1. X = eigenvectors of A / max|A| by a float32 parallel-order Jacobi
//        (one CTA, shared memory; accurate to ~2^-24 max|A| / gap).
//     2. Iterative refinement of X in float64 (the symmetric-eigenproblem
//        refinement step of Ogita and Aishima): with R = I - X^T X and
//        S = X^T A X, the approximations l_i = s_ii / (1 - r_ii) and the
//        correction X <- X + X E, where
//          E_ij = (s_ij + l_j r_ij) / (l_j - l_i)   i, j in different clusters
//          E_ij = r_ij / 2                          i, j in the same cluster,
//        converge quadratically for separated eigenvalues.  Clusters are
//        fixed once per level from the first step: sorted approximations
//        whose neighbouring gaps are at most
//          delta = 64 (||off(S)||_F + ||A||_F ||R||_F + m u ||A_top||_F),
//        i.e. well above what float32 resolved (u = 2^-53).
//     3. Each cluster of size > 1 is a smaller problem C = X_c^T A X_c,
//        solved recursively and rotated in (X_c <- X_c Q); a level whose A is
//        a multiple of I up to the float64 noise of the top problem keeps
//        X = I.  Graded spectra thus descend ~7 decimal orders per level.
//     4. Two more refinement steps with the same clusters (orthonormality,
//        and rotations between clusters, to float64 accuracy).
//   Finally the eigenvalues are the Rayleigh quotients, sorted descending
//   (ties by index) with the sign rule of the Jacobi path, and the result is
//   verified on the device: max |A x - l x| <= 16 m u |l|_max and
//   max |X^T X - I| <= 16 m u.  A result that fails is discarded and the
//   float64 Jacobi runs instead, so this path never returns a less accurate
//   answer than that one would.
//
// All products are float64 (a small tiled GEMM over many CTAs).  The host
// reads the cluster layout once per level (a few synchronisations per mode).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace tk {

namespace {

constexpr int kMpMaxJ = 128;
constexpr int kJ32Threads = 1024;
constexpr int kJ32MaxSweeps = 40;
constexpr int kMaxDepth = 5;
constexpr double kU = DBL_EPSILON / 2;
constexpr double kClusterC = 64.0;
constexpr int kRefineSteps = 3;
constexpr int kPolishSteps = 2;

__device__ __forceinline__ int pidx32(int i, int j) {
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  return j * (j + 1) / 2 + i;
}

// ---------------------------------------------------------------------------
// float32 parallel-order cyclic Jacobi on A / max|A| (one CTA).  The packed
// upper triangle of S and V live in shared memory; each step applies the
// m/2 disjoint rotations of the round-robin tournament (every pair meets
// once in m - 1 steps).  A rotation is taken when |s_pq| exceeds 2^-23 times
// the largest diagonal magnitude at the start of the sweep (an absolute
// criterion: the float64 refinement that follows needs no more).  Writes
// X = V (float64, unsorted columns) and the number of sweeps.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kJ32Threads) k_jacobi32(const double *__restrict__ A, int lda, int n,
                                                           double *__restrict__ X, int ldx, int *__restrict__ sweeps) {
  extern __shared__ __align__(16) float sm32[];
  __shared__ float cs[kMpMaxJ / 2], sn[kMpMaxJ / 2];
  __shared__ int pp[kMpMaxJ / 2], qq[kMpMaxJ / 2];
  __shared__ float red[kJ32Threads / 32];
  __shared__ float scale_s, tol_s;
  __shared__ int rotated;
  const int m = n + (n & 1), np = m / 2;
  const int packed = m * (m + 1) / 2;
  float *Sp = sm32;
  float *V = Sp + packed;
  short *blkP = reinterpret_cast<short *>(V + m * m);
  short *blkQ = blkP + np * (np + 1) / 2;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = np * (np + 1) / 2;

  // scale
  float mx = 0.f;
  for (int e = tid; e < n * n; e += nt) mx = fmaxf(mx, (float)fabs(A[(e % n) + (int64_t)lda * (e / n)]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
    for (int w = 0; w < nt / 32; ++w) v = fmaxf(v, red[w]);
    scale_s = v;
  }
  __syncthreads();
  const double inv = scale_s > 0.f ? 1.0 / (double)scale_s : 0.0;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, j = e / m;
    if (i <= j) Sp[pidx32(i, j)] = (j < n) ? (float)(A[i + (int64_t)lda * j] * inv) : 0.f;
    V[e] = (i == j) ? 1.f : 0.f;
  }
  for (int e = tid; e < nblk; e += nt) {  // pair-block table: e -> (P <= Q)
    int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) / 2 <= e) ++q;
    while (q * (q + 1) / 2 > e) --q;
    blkQ[e] = (short)q;
    blkP[e] = (short)(e - q * (q + 1) / 2);
  }
  __syncthreads();

  int sweep = 0;
  for (; sweep < kJ32MaxSweeps; ++sweep) {
    if (tid < 32) {
      float d = 0.f;
      for (int i = tid; i < m; i += 32) d = fmaxf(d, fabsf(Sp[pidx32(i, i)]));
      for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
      if (tid == 0) {
        tol_s = FLT_EPSILON * fmaxf(d, FLT_MIN);
        rotated = 0;
      }
    }
    __syncthreads();
    const float tol = tol_s;
    for (int step = 0; step < m - 1; ++step) {
      for (int t = tid; t < np; t += nt) {
        int p = (t == 0) ? 0 : ((t - 1 + step) % (m - 1)) + 1;
        int q = ((m - 2 - t + step) % (m - 1)) + 1;
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        float c = 1.f, s = 0.f;
        const float b = Sp[pidx32(p, q)];
        if (fabsf(b) > tol) {
          const float a = Sp[pidx32(p, p)], d = Sp[pidx32(q, q)];
          const float tau = (d - a) / (2.f * b);
          const float at = fabsf(tau);
          const float tt = at > 1e18f ? 0.5f / tau : copysignf(1.f, tau) / (at + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + tt * tt);
          s = tt * c;
          if (s != 0.f) rotated = 1;
        }
        cs[t] = c;
        sn[t] = s;
        pp[t] = p;
        qq[t] = q;
      }
      __syncthreads();
      for (int e = tid; e < nblk; e += nt) {
        const int P = blkP[e], Q = blkQ[e];
        const float s1 = sn[P], s2 = sn[Q];
        const int p1 = pp[P], q1 = qq[P];
        if (P == Q) {
          if (s1 != 0.f) {
            const float t1 = s1 / cs[P];
            const int ipq = pidx32(p1, q1), ipp = pidx32(p1, p1), iqq = pidx32(q1, q1);
            const float b = Sp[ipq];
            Sp[ipp] = Sp[ipp] - t1 * b;
            Sp[iqq] = Sp[iqq] + t1 * b;
            Sp[ipq] = 0.f;
          }
          continue;
        }
        if (s1 == 0.f && s2 == 0.f) continue;
        const float c1 = cs[P], c2 = cs[Q];
        const int p2 = pp[Q], q2 = qq[Q];
        const int i11 = pidx32(p1, p2), i12 = pidx32(p1, q2), i21 = pidx32(q1, p2), i22 = pidx32(q1, q2);
        const float x11 = Sp[i11], x12 = Sp[i12], x21 = Sp[i21], x22 = Sp[i22];
        const float y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
        const float y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
        Sp[i11] = y11 * c2 - y12 * s2;
        Sp[i12] = y11 * s2 + y12 * c2;
        Sp[i21] = y21 * c2 - y22 * s2;
        Sp[i22] = y21 * s2 + y22 * c2;
      }
      for (int e = tid; e < np * m; e += nt) {
        const int t = e / m, i = e - t * m;
        const float s = sn[t];
        if (s == 0.f) continue;
        const float c = cs[t];
        float *vp = V + pp[t] * m + i;
        float *vq = V + qq[t] * m + i;
        const float a = *vp, b = *vq;
        *vp = c * a - s * b;
        *vq = s * a + c * b;
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) {
      ++sweep;
      break;
    }
  }
  for (int e = tid; e < n * n; e += nt) {
    const int i = e % n, j = e / n;
    X[i + (int64_t)ldx * j] = (double)V[j * m + i];
  }
  if (tid == 0 && sweeps) *sweeps = sweep;
}

// ---------------------------------------------------------------------------
// C (M x N) = op(A) B (+ D), float64, column-major.  op(A) = A (M x K, lda) or
// A^T (A is K x M).  8 x 8 outputs per CTA of 64 threads; the CTA's rows of
// op(A) and columns of B (K <= 256) are staged in shared memory.  C may alias
// neither A nor B; D may be C.
// ---------------------------------------------------------------------------
constexpr int kGT = 8;
__global__ void __launch_bounds__(kGT *kGT) k_dgemm_small(int M, int N, int K, const double *__restrict__ A, int lda,
                                                          int transA, const double *__restrict__ B, int ldb,
                                                          const double *D, int ldd, double *C, int ldc) {
  __shared__ double As[kGT][kMpMaxJ * 2 + 1];
  __shared__ double Bs[kGT][kMpMaxJ * 2 + 1];
  const int m0 = blockIdx.x * kGT, n0 = blockIdx.y * kGT;
  const int tx = threadIdx.x % kGT, ty = threadIdx.x / kGT;
  for (int e = threadIdx.x; e < kGT * K; e += kGT * kGT) {
    const int r = e % kGT, k = e / kGT;
    const int i = m0 + r;
    double a = 0.0;
    if (i < M) a = transA ? A[k + (int64_t)lda * i] : A[i + (int64_t)lda * k];
    As[r][k] = a;
    const int j = n0 + r;
    Bs[r][k] = j < N ? B[k + (int64_t)ldb * j] : 0.0;
  }
  __syncthreads();
  const int i = m0 + tx, j = n0 + ty;
  if (i >= M || j >= N) return;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) acc = fma(As[tx][k], Bs[ty][k], acc);
  if (D) acc += D[i + (int64_t)ldd * j];
  C[i + (int64_t)ldc * j] = acc;
}

// ---------------------------------------------------------------------------
// Refinement step kernels.  G = X^T [A X | X] (m x 2m): S = G[:, :m],
// X^T X = G[:, m:].  Everything here is one CTA (m <= 128).
// ---------------------------------------------------------------------------
struct LevelInfo {
  double norm_a;   // ||A||_F of the level's matrix
  int nclusters;
  int degenerate;  // A is a multiple of I up to the noise floor
  int start[kMpMaxJ + 1];
};

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];  // fixed order
  return s;
}

// First step of a level: eigenvalue approximations, clusters (sorted order),
// the permuted X (Xp = X P) and E in the permuted basis.  noise < 0 stands
// for ||A||_F (the top level).
__global__ void __launch_bounds__(1024) k_oa_partition(const double *__restrict__ G, int m, const double *__restrict__ A,
                                                       int lda, const double *__restrict__ X, int ldx, double noise,
                                                       double *__restrict__ Xp, double *__restrict__ E,
                                                       int *__restrict__ label, LevelInfo *__restrict__ info) {
  __shared__ double lam[kMpMaxJ];
  __shared__ int perm[kMpMaxJ], lab[kMpMaxJ];
  __shared__ double red[32];
  __shared__ double delta_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ldg = m;
  const double *S = G;
  const double *P = G + (int64_t)m * m;  // X^T X
  double off2 = 0.0, r2 = 0.0, a2 = 0.0, dev2 = 0.0;
  double tr = 0.0;
  for (int i = tid; i < m; i += nt) tr += A[i + (int64_t)lda * i];
  tr = block_sum(tr, red);
  const double mu = tr / m;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, j = e / m;
    const double s = S[i + ldg * j];
    const double r = (i == j ? 1.0 : 0.0) - P[i + ldg * j];
    if (i != j) off2 += s * s;
    r2 += r * r;
    const double a = A[i + (int64_t)lda * j];
    a2 += a * a;
    const double d = a - (i == j ? mu : 0.0);
    dev2 += d * d;
  }
  off2 = block_sum(off2, red);
  r2 = block_sum(r2, red);
  a2 = block_sum(a2, red);
  dev2 = block_sum(dev2, red);
  for (int i = tid; i < m; i += nt) lam[i] = S[i + ldg * i] / P[i + ldg * i];  // s_ii / (1 - r_ii)
  if (noise < 0.0) noise = sqrt(a2);
  if (tid == 0) delta_s = kClusterC * (sqrt(off2) + sqrt(a2) * sqrt(r2) + m * kU * noise);
  __syncthreads();
  // descending order, ties by index
  for (int i = tid; i < m; i += nt) {
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (lam[j] > lam[i]) || (lam[j] == lam[i] && j < i);
    perm[rank] = i;
  }
  __syncthreads();
  if (tid == 0) {
    const double delta = delta_s;
    int k = 0;
    info->start[0] = 0;
    lab[0] = 0;
    for (int a = 1; a < m; ++a) {
      if (lam[perm[a - 1]] - lam[perm[a]] > delta) info->start[++k] = a;
      lab[a] = k;
    }
    info->nclusters = k + 1;
    info->norm_a = sqrt(a2);
    info->start[k + 1] = m;
    info->degenerate = sqrt(dev2) <= kClusterC * m * kU * noise;
  }
  __syncthreads();
  for (int a = tid; a < m; a += nt) label[a] = lab[a];
  for (int e = tid; e < m * m; e += nt) {
    const int a = e % m, b = e / m;
    Xp[a + (int64_t)ldx * b] = X[a + (int64_t)ldx * perm[b]];
    const int i = perm[a], j = perm[b];
    const double r = (i == j ? 1.0 : 0.0) - P[i + ldg * j];
    double v;
    if (a == b || lab[a] == lab[b]) v = 0.5 * r;
    else v = (S[i + ldg * j] + lam[j] * r) / (lam[j] - lam[i]);
    E[a + (int64_t)m * b] = v;
  }
}

// Later steps: E from G with the clusters fixed.
__global__ void __launch_bounds__(1024) k_oa_update(const double *__restrict__ G, int m, const int *__restrict__ label,
                                                    double *__restrict__ E) {
  __shared__ double lam[kMpMaxJ];
  __shared__ int lab[kMpMaxJ];
  const double *S = G;
  const double *P = G + (int64_t)m * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    lam[i] = S[i + (int64_t)m * i] / P[i + (int64_t)m * i];
    lab[i] = label[i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    const double r = (i == j ? 1.0 : 0.0) - P[i + (int64_t)m * j];
    double v;
    if (i == j || lab[i] == lab[j]) v = 0.5 * r;
    else v = (S[i + (int64_t)m * j] + lam[j] * r) / (lam[j] - lam[i]);
    E[e] = v;
  }
}

__global__ void k_set_identity(double *X, int ldx, int m) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;
    X[i + (int64_t)ldx * j] = i == j ? 1.0 : 0.0;
  }
}

__global__ void k_copy_cols(const double *__restrict__ src, int lds, double *__restrict__ dst, int ldd, int rows,
                            int cols) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
    const int i = e % rows, j = e / rows;
    dst[i + (int64_t)ldd * j] = src[i + (int64_t)lds * j];
  }
}

// Rayleigh quotients, verification and output: lam (descending, ties by
// index), V (sign rule: the largest-magnitude entry of a column is positive,
// the lowest row on ties), check[0] = max |A x - l x|, check[1] = max
// |X^T X - I|, check[2] = max |l|.
__global__ void __launch_bounds__(1024) k_mp_finalize(const double *__restrict__ G, const double *__restrict__ T,
                                                      const double *__restrict__ X, int m, double *__restrict__ lam_out,
                                                      double *__restrict__ V_out, double *__restrict__ check) {
  __shared__ double lam[kMpMaxJ];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double *S = G;
  const double *P = G + (int64_t)m * m;
  for (int i = tid; i < m; i += nt) lam[i] = S[i + (int64_t)m * i] / P[i + (int64_t)m * i];
  __syncthreads();
  double res = 0.0, orth = 0.0, lmax = 0.0;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, j = e / m;
    res = fmax(res, fabs(T[e] - X[e] * lam[j]));
    orth = fmax(orth, fabs(P[e] - (i == j ? 1.0 : 0.0)));
    if (!(T[e] == T[e]) || !(P[e] == P[e])) res = INFINITY;  // NaN fails the check
  }
  for (int i = tid; i < m; i += nt) lmax = fmax(lmax, fabs(lam[i]));
  for (int o = 16; o > 0; o >>= 1) {
    res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
    orth = fmax(orth, __shfl_xor_sync(0xffffffffu, orth, o));
    lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  const int lane = tid & 31, warp = tid >> 5;
  __shared__ double rr[32], oo[32], ll[32];
  if (lane == 0) {
    rr[warp] = res;
    oo[warp] = orth;
    ll[warp] = lmax;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < nt / 32; ++w) {
      a = fmax(a, rr[w]);
      b = fmax(b, oo[w]);
      c = fmax(c, ll[w]);
    }
    check[0] = a;
    check[1] = b;
    check[2] = c;
  }
  for (int i = tid; i < m; i += nt) {
    const double di = lam[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (lam[j] > di) || (lam[j] == di && j < i);
    lam_out[rank] = di;
    const double *col = X + (int64_t)m * i;
    double best = -1.0;
    int br = 0;
    for (int r = 0; r < m; ++r) {
      const double v = fabs(col[r]);
      if (v > best) {
        best = v;
        br = r;
      }
    }
    const double sg = col[br] < 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < m; ++r) V_out[r + (int64_t)m * rank] = sg * col[r];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct MpWork {
  // per depth: TX0, TX1 (m x 2m: [A X | X]), G (m x 2m), E, C, T (m x m)
  double *base = nullptr;
  int J = 0;
  double *tx(int d, int k) const { return base + (size_t)d * 9 * J * J + (size_t)k * 2 * J * J; }
  double *g(int d) const { return base + (size_t)d * 9 * J * J + (size_t)4 * J * J; }
  double *e(int d) const { return base + (size_t)d * 9 * J * J + (size_t)6 * J * J; }
  double *c(int d) const { return base + (size_t)d * 9 * J * J + (size_t)7 * J * J; }
  double *t(int d) const { return base + (size_t)d * 9 * J * J + (size_t)8 * J * J; }
  int *labels = nullptr;      // per depth, J ints
  LevelInfo *info = nullptr;  // per depth (device)
  double *check = nullptr;    // 4 doubles
  int *sweeps = nullptr;      // 1 int
};

int gemm(int M, int N, int K, const double *A, int lda, int transA, const double *B, int ldb, const double *D, int ldd,
         double *C, int ldc, cudaStream_t s) {
  dim3 grid((M + kGT - 1) / kGT, (N + kGT - 1) / kGT);
  k_dgemm_small<<<grid, kGT * kGT, 0, s>>>(M, N, K, A, lda, transA, B, ldb, D, ldd, C, ldc);
  TK_LAUNCHED();
  return TUCKER_OK;
}

// G = X^T [A X | X] for X stored in tx[:, m:2m] (ld m); A X goes to tx[:, :m].
int products(const double *A, int lda, int m, double *tx, double *G, cudaStream_t s) {
  double *X = tx + (size_t)m * m;
  TK_CHECK(gemm(m, m, m, A, lda, 0, X, m, nullptr, 0, tx, m, s));
  TK_CHECK(gemm(m, 2 * m, m, X, m, 1, tx, m, nullptr, 0, G, m, s));
  return TUCKER_OK;
}

// One level: eigenvectors of A (m x m, lda) into out (m x m, ld m).
int mp_level(const double *A, int lda, int m, double noise, int depth, const MpWork &w, double *out, cudaStream_t s) {
  double *tx0 = w.tx(depth, 0), *tx1 = w.tx(depth, 1);
  double *G = w.g(depth), *E = w.e(depth);
  int *label = w.labels + depth * w.J;
  LevelInfo *dinfo = w.info + depth;
  const size_t smem32 = (size_t)((m + 1) / 2 * 2) * ((m + 1) / 2 * 2 + 1) / 2 * sizeof(float) +
                        (size_t)((m + 1) / 2 * 2) * ((m + 1) / 2 * 2) * sizeof(float) +
                        (size_t)((m + 1) / 2) * ((m + 1) / 2 + 1) * sizeof(short) + 16;
  TK_CUDA(cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
  k_jacobi32<<<1, kJ32Threads, smem32, s>>>(A, lda, m, tx0 + (size_t)m * m, m, depth == 0 ? w.sweeps : nullptr);
  TK_LAUNCHED();
  // first refinement step: clusters and the permuted basis
  TK_CHECK(products(A, lda, m, tx0, G, s));
  k_oa_partition<<<1, 1024, 0, s>>>(G, m, A, lda, tx0 + (size_t)m * m, m, noise, tx1 + (size_t)m * m, E, label,
                                    dinfo);
  TK_LAUNCHED();
  double *cur = tx1, *nxt = tx0;
  // X <- X + X E
  auto apply = [&]() -> int {
    const double *X = cur + (size_t)m * m;
    TK_CHECK(gemm(m, m, m, X, m, 0, E, m, X, m, nxt + (size_t)m * m, m, s));
    std::swap(cur, nxt);
    return TUCKER_OK;
  };
  auto refine = [&]() -> int {
    TK_CHECK(products(A, lda, m, cur, G, s));
    k_oa_update<<<1, 1024, 0, s>>>(G, m, label, E);
    TK_LAUNCHED();
    return apply();
  };
  TK_CHECK(apply());
  for (int k = 1; k < kRefineSteps; ++k) TK_CHECK(refine());
  LevelInfo h;
  TK_CUDA(cudaMemcpyAsync(&h, dinfo, sizeof h, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (noise < 0.0) noise = h.norm_a;  // the top level fixes the noise floor for its descendants
  if (h.degenerate) {
    k_set_identity<<<(m * m + 255) / 256, 256, 0, s>>>(out, m, m);
    TK_LAUNCHED();
    return TUCKER_OK;
  }
  double *X = cur + (size_t)m * m;
  for (int k = 0; k < h.nclusters; ++k) {
    const int c0 = h.start[k], mc = h.start[k + 1] - c0;
    if (mc < 2 || depth + 1 >= kMaxDepth) continue;
    // C = X_c^T A X_c
    double *T = w.t(depth), *C = w.c(depth);
    TK_CHECK(gemm(m, mc, m, A, lda, 0, X + (size_t)m * c0, m, nullptr, 0, T, m, s));
    TK_CHECK(gemm(mc, mc, m, X + (size_t)m * c0, m, 1, T, m, nullptr, 0, C, mc, s));
    double *Q = w.e(depth + 1);  // the child's E is free until it runs; Q is copied out first
    double *Qc = w.t(depth + 1);
    TK_CHECK(mp_level(C, mc, mc, noise, depth + 1, w, Qc, s));
    // X_c <- X_c Q
    TK_CHECK(gemm(m, mc, mc, X + (size_t)m * c0, m, 0, Qc, mc, nullptr, 0, Q, m, s));
    k_copy_cols<<<(m * mc + 255) / 256, 256, 0, s>>>(Q, m, X + (size_t)m * c0, m, m, mc);
    TK_LAUNCHED();
  }
  for (int k = 0; k < kPolishSteps; ++k) TK_CHECK(refine());
  k_copy_cols<<<(m * m + 255) / 256, 256, 0, s>>>(cur + (size_t)m * m, m, out, m, m, m);
  TK_LAUNCHED();
  return TUCKER_OK;
}

}  // namespace

// Returns TUCKER_OK with *verified = 1 when lam / V hold a verified result;
// *verified = 0 leaves them to the float64 Jacobi.
int launch_eig_mp(const double *d_S, int64_t J, double *d_lam, double *d_V, int *d_info, int *verified,
                  cudaStream_t s, Prof *prof) {
  *verified = 0;
  if (J < 1 || J > kMpMaxJ) return TUCKER_OK;
  const int m = (int)J;
  MpWork w;
  w.J = m;
  const size_t doubles = (size_t)kMaxDepth * 9 * m * m + 8;
  const size_t bytes = doubles * sizeof(double) + (size_t)kMaxDepth * m * sizeof(int) +
                       (size_t)kMaxDepth * sizeof(LevelInfo) + 64;
  void *mem = nullptr;
  TK_CUDA(cudaMallocAsync(&mem, bytes, s));
  struct Free {
    void *p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } guard{mem, s};
  w.base = static_cast<double *>(mem);
  w.check = w.base + (size_t)kMaxDepth * 9 * m * m;
  w.sweeps = reinterpret_cast<int *>(w.check + 4);
  w.labels = reinterpret_cast<int *>(w.check + 8);
  w.info = reinterpret_cast<LevelInfo *>(
      (reinterpret_cast<uintptr_t>(w.labels + kMaxDepth * m) + 15) & ~static_cast<uintptr_t>(15));

  if (prof) prof->begin(TUCKER_PHASE_EIG);
  double *X = w.c(kMaxDepth - 1);  // never a cluster block: the deepest level takes no clusters
  TK_CHECK(mp_level(d_S, m, m, -1.0, 0, w, X, s));
  // final products, Rayleigh quotients, verification, output
  double *tx0 = w.tx(0, 0);
  k_copy_cols<<<(m * m + 255) / 256, 256, 0, s>>>(X, m, tx0 + (size_t)m * m, m, m, m);
  TK_LAUNCHED();
  TK_CHECK(products(d_S, m, m, tx0, w.g(0), s));
  k_mp_finalize<<<1, 1024, 0, s>>>(w.g(0), tx0, tx0 + (size_t)m * m, m, d_lam, d_V, w.check);
  TK_LAUNCHED();
  double chk[3];
  int sw = 0;
  TK_CUDA(cudaMemcpyAsync(chk, w.check, sizeof chk, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(&sw, w.sweeps, sizeof sw, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (prof) prof->end(0.0, (double)J * J * 8, 1);
  const double tol_res = 16.0 * m * kU * chk[2], tol_orth = 16.0 * m * kU;
  if (chk[0] <= tol_res && chk[1] <= tol_orth) {
    const int info[2] = {sw, 0};
    TK_CUDA(cudaMemcpyAsync(d_info, info, sizeof info, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaStreamSynchronize(s));
    *verified = 1;
  }
  return TUCKER_OK;
}

}  // namespace tk
