// Mixed-precision eigensolver for the eigenvector step of Algorithm 1
// (Sec. 2.2; the paper calls LAPACK's dsyevx, Sec. 5.4, Algorithm 5).
//
// GB300's float64 pipe issues ~2 FMAs per clock per SM, so a float64 Jacobi
// of a 128 x 128 Gram (18 sweeps of 127 dependent steps) is bound by latency
// and float64 throughput at once.  This solver finds the eigenvectors in
// float32 and restores float64 accuracy with matrix products spread over all
// SMs:
//
//   level(A):  (A symmetric m x m, float64)
//     1. X = eigenvectors of A in float32, scaled by a power of two so that
//        its largest magnitude is in [1/2, 1) (one CTA, shared memory;
//        accurate to ~2^-24 max|A| / gap): Householder tridiagonalization,
//        multisection, inverse iteration, orthonormalisation by Householder
//        QR and back-transformation (k_eig32_tri), or with
//        TUCKER_EIG32=jacobi the parallel-order Jacobi sweeps (k_jacobi32).
//     2. Iterative refinement of X in float64 (the symmetric-eigenproblem
//        refinement step of Ogita and Aishima): with R = I - X^T X and
//        S = X^T A X, the approximations l_i = s_ii / (1 - r_ii) and the
//        correction X <- X + X E, where
//          E_ij = (s_ij + l_j r_ij) / (l_j - l_i)   i, j in different clusters
//          E_ij = r_ij / 2                          i, j in the same cluster,
//        converge quadratically for separated eigenvalues (two steps from
//        the float32 stage's ~1e-7).  Clusters are
//        fixed once per level from the first step: sorted approximations
//        whose neighbouring gaps are at most
//          delta = 64 (||off(S)||_F + ||A||_F ||R||_F + m u ||A_top||_F),
//        i.e. well above what float32 resolved (u = 2^-53).
//     3. Each cluster of size > 1 is a smaller problem C = X_c^T A X_c,
//        solved recursively and rotated in (X_c <- X_c Q); a level whose A is
//        a multiple of I up to the float64 noise of the top problem keeps
//        X = I.  Graded spectra thus descend ~7 decimal orders per level.
//     4. One more refinement step with the same clusters (orthonormality,
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
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"

namespace tk {

namespace {

constexpr int kTriMaxJ = 128;   // float32 stages with the whole matrix in shared memory
constexpr int kWideMaxJ = 256;  // the wide float32 stage (packed triangle in shared memory)
constexpr int kMpMaxJ = 512;    // the solver as a whole (cluster float32 Jacobi above kWideMaxJ)
constexpr int kGemmMaxK = 256;  // contraction rows the small float64 products stage at a time
constexpr int kJ32Threads = 1024;
constexpr int kJ32MaxSweeps = 40;
constexpr int kMaxDepth = 5;
constexpr double kU = DBL_EPSILON / 2;
constexpr double kClusterC = 64.0;
constexpr int kRefineSteps = 2;
constexpr int kPolishSteps = 1;

// ---------------------------------------------------------------------------
// float32 parallel-order cyclic Jacobi on A / max|A| (one CTA).  S (full,
// row-major, kept symmetric) and V (column-major) live in shared memory,
// padded with zero rows and columns to m = n rounded up to a multiple of 4.
// Each step applies the m/2 disjoint rotations of the round-robin tournament
// (every pair meets once in m - 1 steps): S is updated in 2 x 2 blocks
// {p_P, q_P} x {p_Q, q_Q} as R_P^T B R_Q (one block per pair of pairs P <= Q,
// mirrored), V by 16-byte column vectors.  A rotation is taken when |s_pq|
// exceeds 2^-23 times the largest diagonal magnitude at the start of the
// sweep (an absolute criterion: the float64 refinement that follows needs no
// more).  Writes X = V (float64, unsorted columns) and the number of sweeps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void jacobi32_body(const double *__restrict__ A, int lda, int n, double *__restrict__ X,
                                              int ldx, int *__restrict__ sweeps);

__global__ void __launch_bounds__(kJ32Threads) k_jacobi32(const double *__restrict__ A, int lda, int n,
                                                           double *__restrict__ X, int ldx, int *__restrict__ sweeps) {
  jacobi32_body(A, lda, n, X, ldx, sweeps);
}

// Many matrices at once, one CTA each (J_b <= 128; J_b = 0 skips the CTA):
// A_b (ld J_b) in, X_b = V (float64, ld J_b, unsorted columns) out.
__global__ void __launch_bounds__(kJ32Threads) k_jacobi32_batched(const double *const *__restrict__ A,
                                                                   const int *__restrict__ Js,
                                                                   double *const *__restrict__ X,
                                                                   const int *__restrict__ idx) {
  const int b = idx ? idx[blockIdx.x] : (int)blockIdx.x, J = Js[b];
  if (J > 0) jacobi32_body(A[b], J, J, X[b], J, nullptr);
}

__device__ __forceinline__ void jacobi32_body(const double *__restrict__ A, int lda, int n, double *__restrict__ X,
                                              int ldx, int *__restrict__ sweeps) {
  extern __shared__ __align__(16) float sm32[];
  __shared__ float4 rot[kTriMaxJ / 2];  // per pair: c, s, t = s / c, (p | q << 16) as bits
  __shared__ float red[kJ32Threads / 32];
  __shared__ float scale_s, tol_s;
  __shared__ int rotated;
  const int m = (n + 3) & ~3, np = m / 2;
  const int ld = m + 1;    // odd row stride: S[i ld + j] and its mirror S[j ld + i] fall in different banks
  float *S = sm32;         // m x ld
  float *V = S + ((m * ld + 3) & ~3);  // m x m, column j at V + j m (16-byte aligned)
  int *blk = reinterpret_cast<int *>(V + m * m);  // pair block e -> P | Q << 16, P <= Q
  const int nblk = np * (np + 1) / 2;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;

  float mx = 0.f;
  for (int e = tid; e < n * n; e += nt) mx = fmaxf(mx, (float)fabs(A[(e % n) + (int64_t)lda * (e / n)]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
    for (int w = 0; w < nwarps; ++w) v = fmaxf(v, red[w]);
    scale_s = v;
  }
  __syncthreads();
  const double inv = scale_s > 0.f ? 1.0 / (double)scale_s : 0.0;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - (e / m) * m;
    const int lo = min(i, j), hi = max(i, j);  // read the upper triangle, mirror it
    S[i * ld + j] = (hi < n) ? (float)(A[lo + (int64_t)lda * hi] * inv) : 0.f;
    V[e] = (i == j) ? 1.f : 0.f;
  }
  for (int e = tid; e < nblk; e += nt) {
    int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) / 2 <= e) ++q;
    while (q * (q + 1) / 2 > e) --q;
    blk[e] = (e - q * (q + 1) / 2) | (q << 16);
  }
  __syncthreads();

  int sweep = 0;
  for (; sweep < kJ32MaxSweeps; ++sweep) {
    if (warp == 0) {
      float d = 0.f;
      for (int i = lane; i < m; i += 32) d = fmaxf(d, fabsf(S[i * ld + i]));
      for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
      if (lane == 0) {
        tol_s = FLT_EPSILON * fmaxf(d, FLT_MIN);
        rotated = 0;
      }
    }
    __syncthreads();
    const float tol = tol_s;
    for (int step = 0; step < m - 1; ++step) {
      if (tid < np) {
        const int t = tid;
        int p = (t == 0) ? 0 : ((t - 1 + step) % (m - 1)) + 1;
        int q = ((m - 2 - t + step) % (m - 1)) + 1;
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        // rotation annihilating s_pq (approximate reciprocals and roots are
        // enough: c and s = t c stay orthonormal to rounding, and s_pq is
        // then set to zero exactly)
        float c = 1.f, sv = 0.f, tt = 0.f;
        const float b = S[p * ld + q];
        if (fabsf(b) > tol) {
          const float a = S[p * ld + p], d = S[q * ld + q];
          const float tau = __fdividef(d - a, 2.f * b);
          const float at = fabsf(tau);
          const float h = fmaf(tau, tau, 1.f);
          tt = at > 1e18f ? __fdividef(0.5f, tau) : copysignf(__fdividef(1.f, at + h * rsqrtf(h)), tau);
          c = rsqrtf(fmaf(tt, tt, 1.f));
          sv = tt * c;
          if (sv != 0.f) rotated = 1;
        }
        rot[t] = make_float4(c, sv, tt, __int_as_float(p | (q << 16)));
      }
      __syncthreads();
      for (int e = tid; e < nblk; e += nt) {
        const int pq = blk[e];
        const int P = pq & 0xFFFF, Q = pq >> 16;
        const float4 rP = rot[P];
        if (P == Q) {
          if (rP.y == 0.f) continue;
          const int k = __float_as_int(rP.w), p1 = k & 0xFFFF, q1 = k >> 16;
          const float b = S[p1 * ld + q1];
          S[p1 * ld + p1] -= rP.z * b;
          S[q1 * ld + q1] += rP.z * b;
          S[p1 * ld + q1] = 0.f;
          S[q1 * ld + p1] = 0.f;
          continue;
        }
        const float4 rQ = rot[Q];
        const float s1 = rP.y, s2 = rQ.y;
        if (s1 == 0.f && s2 == 0.f) continue;
        const float c1 = rP.x, c2 = rQ.x;
        const int kP = __float_as_int(rP.w), kQ = __float_as_int(rQ.w);
        const int p1 = kP & 0xFFFF, q1 = kP >> 16, p2 = kQ & 0xFFFF, q2 = kQ >> 16;
        const float x11 = S[p1 * ld + p2], x12 = S[p1 * ld + q2], x21 = S[q1 * ld + p2], x22 = S[q1 * ld + q2];
        const float y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
        const float y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
        const float z11 = y11 * c2 - y12 * s2, z12 = y11 * s2 + y12 * c2;
        const float z21 = y21 * c2 - y22 * s2, z22 = y21 * s2 + y22 * c2;
        S[p1 * ld + p2] = z11;
        S[p2 * ld + p1] = z11;
        S[p1 * ld + q2] = z12;
        S[q2 * ld + p1] = z12;
        S[q1 * ld + p2] = z21;
        S[p2 * ld + q1] = z21;
        S[q1 * ld + q2] = z22;
        S[q2 * ld + q1] = z22;
      }
      for (int t = warp; t < np; t += nwarps) {
        const float4 r = rot[t];
        if (r.y == 0.f || 4 * lane >= m) continue;
        const float c = r.x, sv = r.y;
        const int k = __float_as_int(r.w);
        float4 *vp = reinterpret_cast<float4 *>(V + (k & 0xFFFF) * m) + lane;
        float4 *vq = reinterpret_cast<float4 *>(V + (k >> 16) * m) + lane;
        const float4 a = *vp, b = *vq;
        *vp = make_float4(c * a.x - sv * b.x, c * a.y - sv * b.y, c * a.z - sv * b.z, c * a.w - sv * b.w);
        *vq = make_float4(sv * a.x + c * b.x, sv * a.y + c * b.y, sv * a.z + c * b.z, sv * a.w + c * b.w);
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

size_t jacobi32_smem(int n) {
  const int m = (n + 3) & ~3, np = m / 2;
  return (size_t)(((m * (m + 1) + 3) & ~3) + m * m) * sizeof(float) + (size_t)np * (np + 1) / 2 * sizeof(int) + 16;
}

}  // namespace

// The float32 Jacobi stage on `count` matrices (one CTA each, J <= 128).
int launch_jacobi32_batched(const double *const *d_A, const int *d_J, double *const *d_X, int count, int maxJ,
                            cudaStream_t s, const int *d_idx, int threads) {
  if (maxJ > kTriMaxJ) {
    set_error("batched float32 Jacobi takes J <= %d (got %d)", kTriMaxJ, maxJ);
    return TUCKER_EUNSUPPORTED;
  }
  TK_CUDA(allow_max_smem(k_jacobi32_batched));
  if (count > 0) {
    k_jacobi32_batched<<<count, threads > 0 ? threads : kJ32Threads, jacobi32_smem(maxJ), s>>>(d_A, d_J, d_X, d_idx);
    TK_LAUNCHED();
  }
  return TUCKER_OK;
}

namespace {

// ---------------------------------------------------------------------------
// float32 tridiagonal eigensolver on A scaled by a power of two (largest
// magnitude in [1/2, 1); one CTA of kT32Threads),
// the first stage of a level in place of the Jacobi sweeps: O(n^3) work once
// instead of per sweep, every phase data-parallel over rows, columns or
// eigenvalues, with 2-3 block barriers per reflector.
//   1. Householder tridiagonalization T = Q1^T A Q1 (H_k = I - tau_k v_k v_k^T,
//      v_k(0) = 1, acting on rows k+1..n-1), blocked as LAPACK's sytrd/latrd:
//      within a panel of kNb columns the trailing block's updates
//      A22 -= v w^T + w v^T (w = tau A22 v - (tau/2)(tau v^T A22 v) v, with
//      A22 v corrected for the panel's earlier columns) are deferred and
//      applied at the panel's end as one rank-2 kNb update.  v_k is kept
//      below the subdiagonal of column k.
//   2. Eigenvalues of T by multisection on Sturm counts (four threads per
//      eigenvalue, five sub-intervals per round, 12 rounds: below 2^-26 ||T||).
//   3. Eigenvectors of T by two steps of inverse iteration (thread i solves
//      (T - l_i I) z = b with the LDL^T factorization of T - l_i I, pivots
//      kept above 2^-23 ||T||, first from a fixed pseudo-random b).
//   4. Inverse iteration leaves vectors of close eigenvalues far from
//      orthogonal (~2^-23 ||T|| / gap; nearly parallel below the float32
//      resolution), and the float64 refinement's cluster width grows with
//      ||I - X^T X||, so the vectors, in descending eigenvalue order, are
//      replaced by the Q factor of their Householder QR (signs kept): each
//      keeps its direction up to the components along larger ones, and
//      vectors that were nearly dependent become an orthonormal basis of the
//      complement of the others.
//   5. X = Q1 Z by the tridiagonalization's reflectors in reverse order.
// Steps 4 and 5 apply reflectors kNb at a time in compact WY form,
// H_j0 ... H_j0+nb-1 = I - V T V^T (T upper triangular, LAPACK's larft),
// as two register-tiled products through shared memory: a reflector costs
// a fraction of a matrix pass instead of two passes and two barriers.
// Accuracy is float32's (~2^-23 ||A|| / gap), as the Jacobi sweeps gave; the
// float64 refinement that follows does not depend on which one ran.
// Writes X (float64, columns in descending eigenvalue order).
// ---------------------------------------------------------------------------
constexpr int kT32Threads = 512;
constexpr int kNb = 8;  // reflectors per compact WY block

// row stride of Z and W: a multiple of 4 floats (16-byte rows for vector
// loads) and 4 more, so that column walks spread over 8 banks
__host__ __device__ __forceinline__ int tri32_ld(int n) { return ((n + 3) & ~3) + 4; }

// float offsets of the shared-memory regions, each 16-byte aligned:
// A (n x (n+1)), Z and W (n x ld), WY partials (4 x kNb x 128), the T
// factors of the reflector blocks and 8 n-vectors
struct Tri32Layout {
  int z, w, part, tf, vec, total;
  __host__ __device__ explicit Tri32Layout(int n) {
    auto up = [](int v) { return (v + 3) & ~3; };
    const int ld = tri32_ld(n);
    z = up(n * (n + 1));
    w = z + up(n * ld);
    part = w + up(n * ld);
    tf = part + 4 * kNb * kTriMaxJ;
    vec = tf + ((n + kNb - 1) / kNb) * kNb * kNb;
    total = vec + 8 * n;
  }
};
size_t tri32_smem(int n) { return (size_t)Tri32Layout(n).total * sizeof(float) + 64; }

__device__ __forceinline__ float warp_sum32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// fixed pseudo-random start vector entry in [-1, 1) (integer hash of i, k)
__device__ __forceinline__ float start_entry(int i, int k) {
  uint32_t h = (uint32_t)i * 0x9E3779B1u ^ ((uint32_t)k + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return (float)(int)(h >> 8) * 0x1p-23f - 1.0f;
}

__device__ __forceinline__ float4 fma4(float a, float4 b, float4 c) {
  return make_float4(fmaf(a, b.x, c.x), fmaf(a, b.y, c.y), fmaf(a, b.z, c.z), fmaf(a, b.w, c.w));
}

// Column i of T (kNb x kNb, upper triangular) of a block of reflectors from
// G(k, l) = v_k^T v_l (k < l, row-major kNb x kNb) and the block's taus
// (zero past its last reflector): T = (diag(1 / tau) + striu(G))^-1 by back
// substitution, x_i = tau_i, x_k = -tau_k sum_{l=k+1..i} G(k, l) x_l, which
// stays valid (a zero row and column) for tau = 0.  Equals LAPACK's larft
// recurrence T(0:i, i) = -tau_i T(0:i, 0:i) V(:, 0:i)^T v_i.
__device__ __forceinline__ void wy_t_column(const float *__restrict__ G, const float *__restrict__ taus, int i,
                                            float *__restrict__ T) {
  float x[kNb];
#pragma unroll
  for (int k = kNb - 1; k >= 0; --k) {
    float acc = 0.f;
#pragma unroll
    for (int l = k + 1; l < kNb; ++l) acc = l <= i ? fmaf(G[k * kNb + l], x[l], acc) : acc;
    x[k] = k > i ? 0.f : (k == i ? taus[k] : -taus[k] * acc);
  }
#pragma unroll
  for (int k = 0; k < kNb; ++k) T[k * kNb + i] = x[k];
}

// T factors of the nblk blocks of kNb reflectors in columns 0, kNb, ... of V
// (ldv; explicit unit entries and zeros above them; block b's rows start at
// r0 + b kNb): all the G = V_b^T V_b products at once (a warp per entry),
// then a thread per column of T.  taus[j] for reflector j (j < nref); the T
// factors go to Tf + b kNb^2 and G to Gs (nblk kNb^2 floats).  Ends with a
// barrier.
__device__ void form_wy_ts(const float *__restrict__ V, int ldv, int nblk, int nref, int r0, int n,
                           const float *__restrict__ taus, float *__restrict__ Tf, float *__restrict__ Gs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = warp; e < nblk * kNb * kNb; e += nw) {  // warp-uniform
    const int b = e / (kNb * kNb), k = (e / kNb) % kNb, i = e % kNb, j0 = b * kNb;
    if (k >= i) continue;
    float g = 0.f;
    for (int r = r0 + j0 + lane; r < n; r += 32) g = fmaf(V[r * ldv + j0 + k], V[r * ldv + j0 + i], g);
    g = warp_sum32(g);
    if (lane == 0) Gs[e] = g;
  }
  __syncthreads();
  for (int t = tid; t < nblk * kNb; t += blockDim.x) {
    const int b = t / kNb, i = t % kNb;
    float tb[kNb];
#pragma unroll
    for (int k = 0; k < kNb; ++k) tb[k] = b * kNb + k < nref ? taus[b * kNb + k] : 0.f;
    wy_t_column(Gs + b * kNb * kNb, tb, i, Tf + b * kNb * kNb);
  }
  __syncthreads();
}

// M[r0:n, c0:n] <- (I - V op(T) V^T) M[r0:n, c0:n], op(T) = T or T^T, for
// the kNb reflectors in columns j0.. of V (rows r0 .. n-1, zeros above each
// unit diagonal entry, zero columns past the block's last reflector).  M is
// row-major with a row stride ldm that is a multiple of 4 (16-byte rows).
// Three phases, each ending with a barrier:
//   A. part[p][j][c] = sum over rows r = r0 + p (mod 4) of V[r][j] M[r][c]
//      (thread: a column quad, a pair of reflectors and a row class);
//   B. P = op(T) sum_p part[p] (thread: a column);
//   C. M[r][c] -= sum_j V[r][j] P[j][c] (thread: a column quad and every
//      16th row; V's row is two 16-byte loads, P sits in registers).
__device__ void apply_wy(float *__restrict__ M, int ldm, int n, int r0, int c0, const float *__restrict__ V, int ldv,
                         int j0, const float *__restrict__ T, bool trans, float *__restrict__ part) {
  const int tid = threadIdx.x;
  const int q0 = c0 >> 2, nq = (n + 3) >> 2;
  {
    const int q = q0 + (tid & 31), g = (tid >> 5) & 3, p = tid >> 7;
    if (q < nq) {
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
#pragma unroll 4
      for (int r = r0 + p; r < n; r += 4) {
        const float4 m = *reinterpret_cast<const float4 *>(M + r * ldm + 4 * q);
        const float2 v = *reinterpret_cast<const float2 *>(V + r * ldv + j0 + 2 * g);
        a0 = fma4(v.x, m, a0);
        a1 = fma4(v.y, m, a1);
      }
      *reinterpret_cast<float4 *>(part + (p * kNb + 2 * g) * kTriMaxJ + 4 * q) = a0;
      *reinterpret_cast<float4 *>(part + (p * kNb + 2 * g + 1) * kTriMaxJ + 4 * q) = a1;
    }
  }
  __syncthreads();
  if (tid < kTriMaxJ && tid >= 4 * q0 && tid < 4 * nq) {
    const int c = tid;
    float P[kNb];
#pragma unroll
    for (int j = 0; j < kNb; ++j)
      P[j] = (part[j * kTriMaxJ + c] + part[(kNb + j) * kTriMaxJ + c]) +
             (part[(2 * kNb + j) * kTriMaxJ + c] + part[(3 * kNb + j) * kTriMaxJ + c]);
#pragma unroll
    for (int i = 0; i < kNb; ++i) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < kNb; ++k) t = fmaf(trans ? T[k * kNb + i] : T[i * kNb + k], P[k], t);
      part[i * kTriMaxJ + c] = t;
    }
  }
  __syncthreads();
  {
    const int q = q0 + (tid & 31), p = tid >> 5;
    if (q < nq) {
      float4 P[kNb];
#pragma unroll
      for (int j = 0; j < kNb; ++j) P[j] = *reinterpret_cast<const float4 *>(part + j * kTriMaxJ + 4 * q);
      const bool whole = 4 * q >= c0;
#pragma unroll 2
      for (int r = r0 + p; r < n; r += 16) {
        float4 m = *reinterpret_cast<const float4 *>(M + r * ldm + 4 * q);
        const float4 va = *reinterpret_cast<const float4 *>(V + r * ldv + j0);
        const float4 vb = *reinterpret_cast<const float4 *>(V + r * ldv + j0 + 4);
        m = fma4(-va.x, P[0], m);
        m = fma4(-va.y, P[1], m);
        m = fma4(-va.z, P[2], m);
        m = fma4(-va.w, P[3], m);
        m = fma4(-vb.x, P[4], m);
        m = fma4(-vb.y, P[5], m);
        m = fma4(-vb.z, P[6], m);
        m = fma4(-vb.w, P[7], m);
        float *dst = M + r * ldm + 4 * q;
        if (whole) {
          *reinterpret_cast<float4 *>(dst) = m;
        } else {  // the quad that straddles c0
          const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (4 * q + u >= c0) dst[u] = mv[u];
        }
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void load8(const float *__restrict__ p, float (&x)[kNb]) {
  const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
  x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w, x[4] = b.x, x[5] = b.y, x[6] = b.z, x[7] = b.w;
}

// The tridiagonalization's per-column work runs on warps 0..3 (threads
// 0..127, one row each), synchronised among themselves by named barrier 1.
// The functions below take no __restrict__ pointers: the barrier is inline
// assembly, and a restrict-qualified access could be moved across it.
__device__ __forceinline__ void bar128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Threads 0..127: the reflector of column j (panel position i) of the
// tridiagonalization from its up-to-date entries (thread l holds a = A(j + l,
// j), zero past row n - 1): d[j] = a_j, and for rows j+1 .. n-1 LAPACK's
// larfg (H x = beta e_1, v(i) = x(i) / (alpha - beta), tau = (beta - alpha)
// / beta; tau = 0 when x(1..) ~ 0; e[j] = beta, tau[j]).  v (unit entry at row
// j + 1) goes to Vp's column i, below row j + 1 to A's column j, and from row
// j + 1 on to the contiguous vs for the next A22 v.  Entries below 2^-100
// (the inputs are scaled to at most 1) count as zero, which also keeps
// 1 / max finite.  The norm is the plain sum of squares when max|x| >= 2^-40,
// and otherwise formed from x / max|x|, so that squares that matter never
// fall into the subnormal range (where beta^2 would no longer be alpha^2 +
// ||x(1..)||^2 and H would not be orthogonal).  red: 24 floats of scratch.
// Returns tau (the same in every thread).
__device__ float tri_reflect(float a, int n, int j, int i, float *Af, int ld, float *Vp, float *vs, int tid,
                             float *red, float *d, float *e, float *tau) {
  const int lane = tid & 31, w4 = tid >> 5;
  float mx = tid >= 2 ? fabsf(a) : 0.f, sq = tid >= 2 ? a * a : 0.f;  // rows j + 2 ..
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if (lane == 0) {
    red[w4] = mx;
    red[4 + w4] = sq;
  }
  if (tid == 1) red[8] = a;  // alpha: row j + 1
  bar128();
  mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
  sq = (red[4] + red[5]) + (red[6] + red[7]);
  const float alpha = red[8];
  float t = 0.f, scal = 0.f, beta = alpha;
  if (mx > 0x1p-100f) {  // uniform
    float nrm;
    if (mx >= 0x1p-40f) {  // uniform: alpha^2 + sum x^2 as it stands
      nrm = sqrtf(fmaf(alpha, alpha, sq));
    } else {
      const float s = fmaxf(mx, fabsf(alpha)), sx = 1.f / s;
      const float v = tid >= 2 ? a * sx : 0.f;
      float sg = warp_sum32(v * v);
      if (lane == 0) red[12 + w4] = sg;
      bar128();
      sg = (red[12] + red[13]) + (red[14] + red[15]);
      const float aa = alpha * sx;
      nrm = s * sqrtf(fmaf(aa, aa, sg));
    }
    beta = alpha >= 0.f ? -nrm : nrm;
    // tau = (beta - alpha) / beta = 1 - alpha / beta and 1 / (alpha - beta),
    // from two independent correctly rounded reciprocals
    const float rb = __frcp_rn(beta), rd = __frcp_rn(alpha - beta);
    t = fmaf(-alpha, rb, 1.f);
    scal = rd;
  }
  const int r = j + tid;
  if (tid == 0) {
    d[j] = a;
    e[j] = beta;
    tau[j] = t;
  }
  if (tid >= 1 && r < n) {  // every thread read vs before the first barrier above
    const float v = tid == 1 ? 1.f : a * scal;
    Vp[r * kNb + i] = v;
    vs[tid - 1] = v;
    if (tid >= 2) Af[r * ld + j] = v;
  }
  return t;
}

// Threads 0..127: column j (panel position 0) as it stands, and its reflector.
__device__ float tri_column0(float *Af, int ld, int n, int j, float *Vp, float *vs, int tid, float *red, float *d,
                             float *e, float *tau) {
  const int r = j + tid;
  const float a = Af[min(r, n - 1) * ld + j];
  return tri_reflect(r < n ? a : 0.f, n, j, 0, Af, ld, Vp, vs, tid, red, d, e, tau);
}

// Threads 0..127, after the partial products pd of A22 v for column j
// (panel position i; A22 = rows and columns j+1.., as at the panel's start;
// thread c takes row j + 1 + c): y1 = W^T v and y2 = V^T v over the panel's
// earlier columns (from the extra columns of the partial products when they
// fitted, else reduced here), w = tau (A22 v - V y1 - W y2) - (tau / 2)
// (w^T v) v with w^T v = tau (v^T A22 v - 2 y1 . y2) (LAPACK's latrd), to
// Wp's column i.  Then, if next, column j + 1 on the same rows brought up
// to date with the panel's reflectors 0 .. i, a_r = A(r, j+1) - sum_u
// (V(r, u) W(j+1, u) + W(r, u) V(j+1, u)), and its reflector.  Loads are
// unconditional (rows clamped into range, values past the end zeroed).
// Returns that reflector's tau.
__device__ float tri_step(const float *pd, float *Af, int ld, int n, int j, int i, float t, bool next, float *Vp,
                          float *Wp, float *vs, int tid, float *red, float *d, float *e, float *tau) {
  const int lane = tid & 31, w4 = tid >> 5;
  const int m = n - j - 1;  // >= 2
  const bool has_y = m + 2 * kNb <= kTriMaxJ;
  const int c = tid, cc = min(c, m - 1), r = j + 1 + cc;
  float vr[kNb], wr[kNb];
  load8(Vp + r * kNb, vr);
  load8(Wp + r * kNb, wr);
  const float pp = (pd[cc] + pd[kTriMaxJ + cc]) + (pd[2 * kTriMaxJ + cc] + pd[3 * kTriMaxJ + cc]);
  const float vv = vs[cc];
  const float pq = c < m ? pp : 0.f, v = c < m ? vv : 0.f;
  float y1[kNb], y2[kNb];
  {
    const int c0 = has_y ? m : 0;
#pragma unroll
    for (int u = 0; u < kNb; ++u) {
      const float s2 = (pd[c0 + u] + pd[kTriMaxJ + c0 + u]) + (pd[2 * kTriMaxJ + c0 + u] + pd[3 * kTriMaxJ + c0 + u]);
      const int cy = c0 + kNb + u;
      const float s1 = (pd[cy] + pd[kTriMaxJ + cy]) + (pd[2 * kTriMaxJ + cy] + pd[3 * kTriMaxJ + cy]);
      y1[u] = has_y && u < i ? s1 : 0.f;
      y2[u] = has_y && u < i ? s2 : 0.f;
    }
  }
  if (!has_y) {  // uniform: reduced here over the 128 rows
#pragma unroll
    for (int u = 0; u < kNb; ++u) {
      y1[u] = u < i ? wr[u] * v : 0.f;
      y2[u] = u < i ? vr[u] * v : 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < kNb; ++u)
        if (u < i) {
          y1[u] += __shfl_xor_sync(0xffffffffu, y1[u], o);
          y2[u] += __shfl_xor_sync(0xffffffffu, y2[u], o);
        }
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < kNb; ++u) {
        red[32 + w4 * 2 * kNb + u] = y1[u];
        red[32 + w4 * 2 * kNb + kNb + u] = y2[u];
      }
    bar128();
#pragma unroll
    for (int u = 0; u < kNb; ++u) {
      y1[u] = (red[32 + u] + red[32 + 2 * kNb + u]) + (red[32 + 4 * kNb + u] + red[32 + 6 * kNb + u]);
      y2[u] = (red[32 + kNb + u] + red[32 + 3 * kNb + u]) + (red[32 + 5 * kNb + u] + red[32 + 7 * kNb + u]);
      if (u >= i) y1[u] = y2[u] = 0.f;
    }
  }
  float x = pq;
#pragma unroll
  for (int u = 0; u < kNb; ++u)
    if (u < i) x = fmaf(-vr[u], y1[u], fmaf(-wr[u], y2[u], x));
  float pv = warp_sum32(pq * v);
  if (lane == 0) red[16 + w4] = pv;
  bar128();
  pv = (red[16] + red[17]) + (red[18] + red[19]);
  float y12 = 0.f;
#pragma unroll
  for (int u = 0; u < kNb; ++u) y12 = fmaf(y1[u], y2[u], y12);
  const float kk = 0.5f * t * t * (pv - 2.f * y12);
  const float w = fmaf(-kk, v, t * x);  // zero past row n - 1 (v and x are)
  if (c < m) Wp[(j + 1 + c) * kNb + i] = w;
  if (!next) return 0.f;
  // row j + 1 of V and W: columns u < i as stored; column i is v = 1 there
  // and w as thread 0 has it, recomputed here from the same values (so no
  // barrier is needed before the column update)
  const int j1 = j + 1;
  float vj[kNb], wj[kNb];
  load8(Vp + j1 * kNb, vj);
  load8(Wp + j1 * kNb, wj);
  float x0 = (pd[0] + pd[kTriMaxJ]) + (pd[2 * kTriMaxJ] + pd[3 * kTriMaxJ]);
#pragma unroll
  for (int u = 0; u < kNb; ++u)
    if (u < i) x0 = fmaf(-vj[u], y1[u], fmaf(-wj[u], y2[u], x0));
  const float wji = fmaf(-kk, 1.f, t * x0);
  float a = Af[r * ld + j1];
#pragma unroll
  for (int u = 0; u < kNb; ++u)
    if (u < i) a = fmaf(-vr[u], wj[u], fmaf(-wr[u], vj[u], a));
  a = fmaf(-v, wji, fmaf(-w, 1.f, a));
  return tri_reflect(c < m ? a : 0.f, n, j1, i + 1, Af, ld, Vp, vs, tid, red, d, e, tau);
}

// One warp factors the panel of columns j0 .. j0 + nbk - 1 (rows j0 .. n-1)
// of Z (row-major, lz) in registers: lane l holds rows j0 + l + 32 i.  Per
// column the reflector as in tri_column (norm from x / max|x|), then its
// application to the panel's later columns (their dot products reduced
// together).  Writes the reflectors to W's panel columns (unit diagonal,
// zeros above; the rows above j0 are already zero), taus and R's diagonal
// signs, and the panel's T factor.  No block barrier.
__device__ void qr_panel(const float *__restrict__ Z, int lz, float *__restrict__ W, int n, int j0, int nbk, int lane,
                         float *__restrict__ qtau, float *__restrict__ sgn, float *__restrict__ T) {
  constexpr int kR = kTriMaxJ / 32;
  const int mrows = n - j0;
  float P[kR][kNb];
#pragma unroll
  for (int i = 0; i < kR; ++i) {
    const int row = lane + 32 * i;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (row < mrows) {
      a = *reinterpret_cast<const float4 *>(Z + (j0 + row) * lz + j0);
      b = *reinterpret_cast<const float4 *>(Z + (j0 + row) * lz + j0 + 4);
    }
    P[i][0] = a.x, P[i][1] = a.y, P[i][2] = a.z, P[i][3] = a.w;
    P[i][4] = b.x, P[i][5] = b.y, P[i][6] = b.z, P[i][7] = b.w;
  }
  float tv[kNb];
#pragma unroll
  for (int jj = 0; jj < kNb; ++jj) {
    tv[jj] = 0.f;
    if (jj >= nbk) continue;  // uniform
    const float alpha = __shfl_sync(0xffffffffu, P[0][jj], jj);
    float mx = 0.f, sq = 0.f;  // the reflector as in tri_reflect
#pragma unroll
    for (int i = 0; i < kR; ++i)
      if (lane + 32 * i > jj) {
        mx = fmaxf(mx, fabsf(P[i][jj]));
        sq = fmaf(P[i][jj], P[i][jj], sq);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    float t = 0.f, scal = 0.f, beta = alpha;
    if (mx > 0x1p-100f) {  // uniform
      float nrm;
      if (mx >= 0x1p-40f) {  // uniform
        nrm = sqrtf(fmaf(alpha, alpha, sq));
      } else {
        const float sm = fmaxf(mx, fabsf(alpha)), sx = 1.f / sm;
        float sg = 0.f;
#pragma unroll
        for (int i = 0; i < kR; ++i)
          if (lane + 32 * i > jj) {
            const float v = P[i][jj] * sx;
            sg = fmaf(v, v, sg);
          }
        sg = warp_sum32(sg);
        const float a = alpha * sx;
        nrm = sm * sqrtf(fmaf(a, a, sg));
      }
      beta = alpha >= 0.f ? -nrm : nrm;
      const float rb = __frcp_rn(beta), rd = __frcp_rn(alpha - beta);
      t = fmaf(-alpha, rb, 1.f);
      scal = rd;
    }
    tv[jj] = t;
    if (lane == 0) {
      qtau[j0 + jj] = t;
      sgn[j0 + jj] = beta < 0.f ? -1.f : 1.f;
    }
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      const int row = lane + 32 * i;
      P[i][jj] = row == jj ? 1.f : (row > jj && t != 0.f ? P[i][jj] * scal : 0.f);
    }
    if (t != 0.f) {
      float dd[kNb];
#pragma unroll
      for (int c = 0; c < kNb; ++c) {
        dd[c] = 0.f;
        if (c > jj)
#pragma unroll
          for (int i = 0; i < kR; ++i) dd[c] = fmaf(P[i][jj], P[i][c], dd[c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < kNb; ++c)
          if (c > jj) dd[c] += __shfl_xor_sync(0xffffffffu, dd[c], o);
#pragma unroll
      for (int c = 0; c < kNb; ++c)
        if (c > jj)
#pragma unroll
          for (int i = 0; i < kR; ++i) P[i][c] = fmaf(-t * dd[c], P[i][jj], P[i][c]);
    }
  }
#pragma unroll
  for (int i = 0; i < kR; ++i) {
    const int row = lane + 32 * i;
    if (row < mrows) {
      *reinterpret_cast<float4 *>(W + (j0 + row) * lz + j0) = make_float4(P[i][0], P[i][1], P[i][2], P[i][3]);
      *reinterpret_cast<float4 *>(W + (j0 + row) * lz + j0 + 4) = make_float4(P[i][4], P[i][5], P[i][6], P[i][7]);
    }
  }
  // G = V^T V (upper part) in every lane, then lane i < kNb forms T's column i
  float G[kNb * kNb];
#pragma unroll
  for (int k = 0; k < kNb; ++k)
#pragma unroll
    for (int l = 0; l < kNb; ++l) {
      G[k * kNb + l] = 0.f;
      if (k < l)
#pragma unroll
        for (int i = 0; i < kR; ++i) G[k * kNb + l] = fmaf(P[i][k], P[i][l], G[k * kNb + l]);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < kNb; ++k)
#pragma unroll
      for (int l = k + 1; l < kNb; ++l) G[k * kNb + l] += __shfl_xor_sync(0xffffffffu, G[k * kNb + l], o);
  if (lane < kNb) wy_t_column(G, tv, lane, T);
  __syncwarp();
}

__global__ void __launch_bounds__(kT32Threads, 1) k_eig32_tri(const double *__restrict__ A, int lda, int n,
                                                           double *__restrict__ X, int ldx) {
  extern __shared__ __align__(16) float smt[];
  const int ld = n + 1, lz = tri32_ld(n);
  const Tri32Layout lay(n);
  float *Af = smt;             // n x ld, row-major
  float *Z = smt + lay.z;      // n x lz, Z[k lz + c]: row k of eigenvector c of T
  float *W = smt + lay.w;      // W[k n + i]: L factor of T - l_i I; then reflectors, n x lz (column j: v_j)
  float *part = smt + lay.part;  // WY partial products; 4 x 128 partial sums in step 1
  float *pd = part;
  float *Tf = smt + lay.tf;
  float *d = smt + lay.vec, *e = d + n, *e2 = e + n, *tau = e2 + n, *lam = tau + n, *qtau = lam + n,
        *sgn = qtau + n;
  __shared__ float red[96];
  __shared__ float sc[4];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  // ---- load A * 2^-s (upper triangle, mirrored), s such that the largest
  // magnitude lands in [1/2, 1): thread idx reads entry (r, c) = (idx % n,
  // idx / n) for r <= c, consecutive threads down a column.  The float is
  // built from the float64 bits in integer arithmetic (the exponent rebased,
  // the significand truncated to 23 bits, entries 2^-126 below the largest
  // flushed to zero), so the float64 pipe does no work here.
  unsigned mhi = 0u;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    if (r <= c) mhi = max(mhi, (unsigned)(__double_as_longlong(A[r + (int64_t)lda * c]) >> 32) & 0x7FFFFFFFu);
  }
  mhi = __reduce_max_sync(0xffffffffu, mhi);
  if (lane == 0) red[warp] = __uint_as_float(mhi);
  __syncthreads();
  if (tid == 0) {
    unsigned v = 0u;
    for (int w = 0; w < nw; ++w) v = max(v, __float_as_uint(red[w]));
    sc[0] = __uint_as_float(v);
  }
  __syncthreads();
  const unsigned amax = __float_as_uint(sc[0]);
  // exponent field e of a float64 maps to e - (emax - 126) of a float32
  const int rebase = (int)(amax >> 20) - 126;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    if (r <= c) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(A[r + (int64_t)lda * c]);
      const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b, mag = hi & 0x7FFFFFFFu;
      const int x = max((int)mag - (rebase << 20), 0);
      const unsigned f = (amax == 0u || mag == 0u) ? 0u : ((hi & 0x80000000u) | __funnelshift_l(lo, (unsigned)x, 3));
      const float v = __uint_as_float(f);
      Af[r * ld + c] = v;
      Af[c * ld + r] = v;
    }
  }
  __syncthreads();

  // ---- 1. tridiagonalization, kNb columns a panel (LAPACK's latrd, lower):
  // the panel's reflectors V and the vectors W (columns of the n x kNb
  // row-major Vp, Wp) stand for its updates of the trailing matrix until the
  // panel ends, when A22 -= V W^T + W V^T in one pass.  Per column: the
  // block's threads form the partial products of A22 v (A22 as at the
  // panel's start), then warp 0 completes w and brings the next column up to
  // date and forms its reflector.
  float *Vp = W, *Wp = Z;  // both free until step 3
  float *vs = part + 4 * kTriMaxJ;  // the current v, contiguous (16-byte aligned)
  float tcur = 0.f;        // threads 0..127: tau of the current column
  for (int k0 = 0; k0 + 2 < n; k0 += kNb) {
    const int nbk = min(kNb, n - 2 - k0);
    for (int idx = tid; idx < n * kNb; idx += nt) {
      Vp[idx] = 0.f;
      Wp[idx] = 0.f;
    }
    __syncthreads();
    if (tid < 128) tcur = tri_column0(Af, ld, n, k0, Vp, vs, tid, red, d, e, tau);
    __syncthreads();
    for (int i = 0; i < nbk; ++i) {
      const int j = k0 + i, m = n - j - 1;
      {  // partial A22 v: thread (column c, part) sums a quarter of the rows
         // (a multiple of 4, for 16-byte loads of v); when they fit, the
         // threads of columns m .. m + 15 form V^T v and W^T v the same way
        const int c = tid & (kTriMaxJ - 1), part = tid >> 7;
        const int rb = ((m + 15) >> 4) << 2, r1 = min(m, part * rb + rb);
        const float *X = nullptr;
        int xs = 0;
        if (c < m) {
          X = Af + (j + 1) * ld + (j + 1 + c);
          xs = ld;
        } else if (m + 2 * kNb <= kTriMaxJ && c < m + 2 * kNb) {
          const int u = c - m;
          X = (u < kNb ? Vp + u : Wp + (u - kNb)) + (j + 1) * kNb;
          xs = kNb;
        }
        float acc = 0.f, acc2 = 0.f;
        if (X) {
          int r = part * rb;
          for (; r + 3 < r1; r += 4) {
            const float4 v4 = *reinterpret_cast<const float4 *>(vs + r);
            const float a0 = X[r * xs], a1 = X[(r + 1) * xs], a2 = X[(r + 2) * xs], a3 = X[(r + 3) * xs];
            acc = fmaf(a0, v4.x, fmaf(a2, v4.z, acc));
            acc2 = fmaf(a1, v4.y, fmaf(a3, v4.w, acc2));
          }
          for (; r < r1; ++r) acc = fmaf(X[r * xs], vs[r], acc);
        }
        pd[part * kTriMaxJ + c] = acc + acc2;
      }
      __syncthreads();
      if (tid < 128) tcur = tri_step(pd, Af, ld, n, j, i, tcur, i + 1 < nbk, Vp, Wp, vs, tid, red, d, e, tau);
      __syncthreads();
    }
    // A22 -= V W^T + W V^T on rows and columns t0 .. n-1: thread (column c,
    // part) keeps row c of V and W and takes rows part, part + 4, ...
    const int t0 = k0 + nbk, mt = n - t0;
    {
      const int c = tid & (kTriMaxJ - 1), part = tid >> 7;
      if (c < mt) {
        float vc[kNb], wc[kNb];
        load8(Vp + (t0 + c) * kNb, vc);
        load8(Wp + (t0 + c) * kNb, wc);
        for (int r = part; r < mt; r += 4) {
          float vr[kNb], wr[kNb];
          load8(Vp + (t0 + r) * kNb, vr);
          load8(Wp + (t0 + r) * kNb, wr);
          float a = Af[(t0 + r) * ld + t0 + c];
#pragma unroll
          for (int q = 0; q < kNb; ++q) a = fmaf(-vr[q], wc[q], fmaf(-wr[q], vc[q], a));
          Af[(t0 + r) * ld + t0 + c] = a;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = Af[(n - 2) * ld + (n - 2)];
      e[n - 2] = Af[(n - 1) * ld + (n - 2)];
      tau[n - 2] = 0.f;
    }
    d[n - 1] = Af[(n - 1) * ld + (n - 1)];
    e[n - 1] = 0.f;
    tau[n - 1] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) e2[i] = e[i] * e[i];
  if (warp == 0) {  // Gershgorin bounds and ||T||
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int i = lane; i < n; i += 32) {
      const float r = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
      lo = fminf(lo, d[i] - r);
      hi = fmaxf(hi, d[i] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const float tn = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), FLT_MIN);
      sc[0] = lo - 0x1p-20f * tn;
      sc[1] = hi + 0x1p-20f * tn;
      sc[2] = tn;
    }
  }
  __syncthreads();
  const float gl = sc[0], gu = sc[1], tn = sc[2];
  const float piv = 0x1p-23f * tn;  // smallest pivot magnitude kept

  // ---- 2. multisection: threads 4 i .. 4 i + 3 find the i-th smallest eigenvalue
  {
    const int i = tid >> 2, sub = tid & 3;
    float lo = gl, hi = gu;
    // 12 rounds shrink the interval 5^12 > 2^27 times (all lanes take part in the shuffles)
    for (int it = 0; it < 12; ++it) {
      const float x = lo + (hi - lo) * (0.2f * (float)(sub + 1));
      int cnt = 0;
      if (i < n) {
        float q = d[0] - x;
        for (int k = 0;; ++k) {
          if (fabsf(q) < piv) q = -piv;
          cnt += q < 0.f;
          if (k + 1 >= n) break;
          q = d[k + 1] - x - __fdividef(e2[k], q);
        }
      }
      // counts grow with x: new lo = largest point with count <= i, new hi = smallest with count > i
      float nlo = lo, nhi = hi;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int cs = __shfl_sync(0xffffffffu, cnt, (lane & ~3) | s);
        const float xs = __shfl_sync(0xffffffffu, x, (lane & ~3) | s);
        if (cs <= i) nlo = fmaxf(nlo, xs);
        else nhi = fminf(nhi, xs);
      }
      lo = nlo;
      hi = nhi;
    }
    if (i < n && sub == 0) lam[n - 1 - i] = 0.5f * (lo + hi);  // descending order
  }
  __syncthreads();

  // ---- 3. inverse iteration: thread c solves (T - l_c I) z = b twice
  for (int c = tid; c < n; c += nt) {
    const float s = lam[c];
    float D = d[0] - s;
    for (int k = 0; k + 1 < n; ++k) {
      if (fabsf(D) < piv) D = D < 0.f ? -piv : piv;
      const float L = __fdividef(e[k], D);
      W[k * n + c] = L;
      D = d[k + 1] - s - L * e[k];
    }
    for (int pass = 0; pass < 2; ++pass) {
      float Dk = d[0] - s, y = 0.f;
      for (int k = 0; k < n; ++k) {  // forward: y = L^-1 b, z = D^-1 y
        if (k > 0) Dk = d[k] - s - W[(k - 1) * n + c] * e[k - 1];
        if (fabsf(Dk) < piv) Dk = Dk < 0.f ? -piv : piv;
        const float b = pass == 0 ? start_entry(c, k) : Z[k * lz + c];
        y = k == 0 ? b : b - W[(k - 1) * n + c] * y;
        Z[k * lz + c] = __fdividef(y, Dk);
      }
      float xn = Z[(n - 1) * lz + c], nrm = xn * xn;
      for (int k = n - 2; k >= 0; --k) {  // backward: x = L^-T z
        xn = Z[k * lz + c] - W[k * n + c] * xn;
        Z[k * lz + c] = xn;
        nrm = fmaf(xn, xn, nrm);
      }
      // a solve that overflowed (or vanished) restarts from e_c
      const bool good = nrm > 0.f && nrm <= FLT_MAX;
      const float r = good ? rsqrtf(nrm) : 0.f;
      for (int k = 0; k < n; ++k) Z[k * lz + c] = good ? Z[k * lz + c] * r : (k == c ? 1.f : 0.f);
    }
  }
  __syncthreads();

  // ---- 4. Z <- Q of Z = Q R (Householder), columns in descending eigenvalue order.
  // Panels of kNb columns, each factored by one warp in registers (its
  // reflectors to W with unit diagonal and zeros above, its T factor kept);
  // the trailing columns take the panel at once as (I - V T^T V^T).
  for (int idx = tid; idx < n * lz; idx += nt) {
    const int r = idx / lz, c = idx - r * lz;
    if (c >= n) Z[idx] = 0.f;  // padding columns stay zero (and finite)
    W[idx] = 0.f;
  }
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += kNb) {
    const int nbk = min(kNb, n - j0);
    float *Tb = Tf + (j0 / kNb) * kNb * kNb;
    if (warp == 0) qr_panel(Z, lz, W, n, j0, nbk, lane, qtau, sgn, Tb);
    __syncthreads();
    if (j0 + nbk < n) apply_wy(Z, lz, n, j0, j0 + nbk, W, lz, j0, Tb, true, part);
  }
  // explicit Q: the blocks applied to I in reverse order (block b leaves
  // columns before its first one at the identity), then signs so that
  // column j points along the j-th input vector
  for (int idx = tid; idx < n * lz; idx += nt) {
    const int r = idx / lz, c = idx - r * lz;
    Z[idx] = r == c ? 1.f : 0.f;
  }
  __syncthreads();
  for (int j0 = ((n - 1) / kNb) * kNb; j0 >= 0; j0 -= kNb)
    apply_wy(Z, lz, n, j0, j0, W, lz, j0, Tf + (j0 / kNb) * kNb * kNb, false, part);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx / n, c = idx - r * n;
    Z[r * lz + c] *= sgn[c];
  }
  __syncthreads();

  // ---- 5. X = Q1 Z: the tridiagonalization's reflectors (v_k below the
  // subdiagonal of A's column k, unit entry at row k + 1) copied to W, blocks
  // from the last to the first
  const int nref = max(n - 2, 0);
  for (int idx = tid; idx < n * lz; idx += nt) {
    const int r = idx / lz, k = idx - r * lz;
    W[idx] = k < nref ? (r == k + 1 ? 1.f : (r > k + 1 && tau[k] != 0.f ? Af[r * ld + k] : 0.f)) : 0.f;
  }
  __syncthreads();
  const int nblk = (nref + kNb - 1) / kNb;
  if (nblk > 0) form_wy_ts(W, lz, nblk, nref, 1, n, tau, Tf, part);  // the QR blocks' T factors are spent
  for (int j0 = (nblk - 1) * kNb; j0 >= 0; j0 -= kNb)
    apply_wy(Z, lz, n, j0 + 1, 0, W, lz, j0, Tf + (j0 / kNb) * kNb * kNb, false, part);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    X[r + (int64_t)ldx * c] = (double)Z[r * lz + c];
  }
}

// ---------------------------------------------------------------------------
// First stage for kTriMaxJ < n <= kWideMaxJ (one CTA of kW32Threads), the steps
// of k_eig32_tri with a matrix too large for a full float32 copy in shared
// memory.  The lower triangle is packed by columns in shared memory (column
// j holds rows j..n-1 from offset j n - j (j - 1) / 2: 129 KB at n = 256);
// the eigenvector passes use two n x tri32_ld(n) float arrays in global
// memory (they stay in L2), Zg[k ld + c] (row k of vector c) and Lg (the L
// factors of the inverse iteration, then the reflectors of steps 4 and 5).
//   1. Householder tridiagonalization one reflector at a time: the reflector
//      of column k (v(0) = 1, beta = -sign(alpha) ||x||, tau = (beta -
//      alpha) / beta), p = tau A22 v (four threads per row of the packed
//      triangle), w = p - (tau / 2)(p^T v) v, A22 -= v w^T + w v^T.  v stays
//      in column k below the subdiagonal.
//   2. Eigenvalues by multisection on Sturm counts (four threads each).
//   3. Inverse iteration, thread c for the c-th largest eigenvalue.
//   4. The Q factor of the vectors' Householder QR in descending eigenvalue
//      order, signs kept, as in k_eig32_tri: vectors of a cluster become an
//      orthonormal basis of the complement of the larger ones.  (Modified
//      Gram-Schmidt, even twice, loses orthogonality on strongly graded
//      spectra, where many vectors come out nearly parallel.)
//   5. X = Q1 Q by the reflectors from the last to the first.
// Steps 4 and 5 go kNb reflectors at a time in compact WY form, as in
// k_eig32_tri (a warp factors each QR panel in registers; a block of
// reflectors is three register-tiled passes and three barriers instead of
// kNb passes and 2 kNb barriers).  The tridiagonalization's reflectors are
// LAPACK's larfg with the scaled norm of tri_reflect.
// Writes X (float64, columns in descending eigenvalue order).
// ---------------------------------------------------------------------------
constexpr int kW32Threads = 1024;

__host__ __device__ __forceinline__ int packed_col(int n, int j) { return j * n - j * (j - 1) / 2; }

// float offsets of the wide stage's shared-memory regions, each 16-byte
// aligned: the packed triangle, 6 n-vectors, the WY partial products and the
// T factors of the reflector blocks
struct WideLayout {
  int vec, part, tf, total;
  __host__ __device__ explicit WideLayout(int n) {
    auto up = [](int v) { return (v + 3) & ~3; };
    vec = up(n * (n + 1) / 2);
    part = vec + up(6 * n);
    tf = part + 4 * kNb * kWideMaxJ;
    total = tf + ((n + kNb - 1) / kNb) * kNb * kNb;
  }
};
size_t wide32_smem(int n) { return (size_t)WideLayout(n).total * sizeof(float) + 64; }

// Sum over the block of one value per thread; every thread gets the result.
// Uses red[0..32]; callers separate consecutive uses by a barrier.
__device__ __forceinline__ float block_sum32(float v, float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum32(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float t = lane < nw ? red[lane] : 0.f;
    t = warp_sum32(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ float block_max32(float v, float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float t = lane < nw ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

struct Refl {
  float t, beta, scal;
};

// LAPACK's larfg for x[0..m-1] in shared memory (m <= blockDim), every
// thread taking part and getting the same result: H x = beta e_1 with
// H = I - t v v^T, v(0) = 1, v(1..) = x(1..) scal.  As in tri_reflect,
// entries of x(1..) below 2^-100 count as zero (t = 0), and below 2^-40 the
// norm is formed from x / max|x|, so that no square that matters is
// subnormal (H stays orthogonal).  x[0] is read before the first barrier:
// the caller may overwrite x once this returns.
__device__ Refl wide_larfg(const float *x, int m, float *red) {
  const int tid = threadIdx.x;
  const float alpha = x[0];
  const float xi = (tid >= 1 && tid < m) ? x[tid] : 0.f;
  const float mx = block_max32(fabsf(xi), red);
  const float sq = block_sum32(xi * xi, red);
  Refl h{0.f, alpha, 0.f};
  if (mx > 0x1p-100f) {  // the same in every thread
    float nrm;
    if (mx >= 0x1p-40f) {
      nrm = sqrtf(fmaf(alpha, alpha, sq));
    } else {
      const float sv = fmaxf(mx, fabsf(alpha)), sx = 1.f / sv;
      const float v = xi * sx;
      const float sg = block_sum32(v * v, red);
      const float aa = alpha * sx;
      nrm = sv * sqrtf(fmaf(aa, aa, sg));
    }
    h.beta = alpha >= 0.f ? -nrm : nrm;
    h.t = fmaf(-alpha, __frcp_rn(h.beta), 1.f);
    h.scal = __frcp_rn(alpha - h.beta);
  }
  return h;
}

// The compact-WY steps of k_eig32_tri for n <= kWideMaxJ, on row-major
// matrices in global memory (L2-resident) with a row stride that is a
// multiple of 4 (16-byte rows), by kW32Threads threads.  As apply_wy:
// M[r0:n, c0:n] <- (I - V op(T) V^T) M[r0:n, c0:n] for the kNb reflectors in
// columns j0.. of V, in three phases ending with barriers (part: 4 x kNb x
// kWideMaxJ floats of shared memory).
__device__ void apply_wy_wide(float *__restrict__ M, int ldm, int n, int r0, int c0, const float *__restrict__ V,
                              int ldv, int j0, const float *__restrict__ T, bool trans, float *__restrict__ part) {
  const int tid = threadIdx.x;
  const int q0 = c0 >> 2, nq = (n + 3) >> 2;
  {
    const int q = q0 + (tid & 63), g = (tid >> 6) & 3, p = tid >> 8;
    if (q < nq) {
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
#pragma unroll 4
      for (int r = r0 + p; r < n; r += 4) {
        const float4 m = __ldcg(reinterpret_cast<const float4 *>(M + (int64_t)r * ldm + 4 * q));
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(V + (int64_t)r * ldv + j0 + 2 * g));
        a0 = fma4(v.x, m, a0);
        a1 = fma4(v.y, m, a1);
      }
      *reinterpret_cast<float4 *>(part + (p * kNb + 2 * g) * kWideMaxJ + 4 * q) = a0;
      *reinterpret_cast<float4 *>(part + (p * kNb + 2 * g + 1) * kWideMaxJ + 4 * q) = a1;
    }
  }
  __syncthreads();
  if (tid < kWideMaxJ && tid >= 4 * q0 && tid < 4 * nq) {
    const int c = tid;
    float P[kNb];
#pragma unroll
    for (int j = 0; j < kNb; ++j)
      P[j] = (part[j * kWideMaxJ + c] + part[(kNb + j) * kWideMaxJ + c]) +
             (part[(2 * kNb + j) * kWideMaxJ + c] + part[(3 * kNb + j) * kWideMaxJ + c]);
#pragma unroll
    for (int i = 0; i < kNb; ++i) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < kNb; ++k) t = fmaf(trans ? T[k * kNb + i] : T[i * kNb + k], P[k], t);
      part[i * kWideMaxJ + c] = t;
    }
  }
  __syncthreads();
  {
    const int q = q0 + (tid & 63), p = tid >> 6;
    if (q < nq) {
      float4 P[kNb];
#pragma unroll
      for (int j = 0; j < kNb; ++j) P[j] = *reinterpret_cast<const float4 *>(part + j * kWideMaxJ + 4 * q);
      const bool whole = 4 * q >= c0;
#pragma unroll 2
      for (int r = r0 + p; r < n; r += 16) {
        float *dst = M + (int64_t)r * ldm + 4 * q;
        float4 m = __ldcg(reinterpret_cast<const float4 *>(dst));
        const float4 va = __ldcg(reinterpret_cast<const float4 *>(V + (int64_t)r * ldv + j0));
        const float4 vb = __ldcg(reinterpret_cast<const float4 *>(V + (int64_t)r * ldv + j0 + 4));
        m = fma4(-va.x, P[0], m);
        m = fma4(-va.y, P[1], m);
        m = fma4(-va.z, P[2], m);
        m = fma4(-va.w, P[3], m);
        m = fma4(-vb.x, P[4], m);
        m = fma4(-vb.y, P[5], m);
        m = fma4(-vb.z, P[6], m);
        m = fma4(-vb.w, P[7], m);
        if (whole) {
          __stcg(reinterpret_cast<float4 *>(dst), m);
        } else {  // the quad that straddles c0
          const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (4 * q + u >= c0) __stcg(dst + u, mv[u]);
        }
      }
    }
  }
  __syncthreads();
}

// qr_panel for n <= kWideMaxJ: one warp factors columns j0 .. j0 + nbk - 1
// (rows j0 .. n-1) of Z in registers (lane l: rows j0 + l + 32 i) and writes
// the reflectors to W's panel columns, the taus, R's diagonal signs and the
// panel's T factor.  No block barrier.
__device__ void qr_panel_wide(const float *__restrict__ Z, int lz, float *__restrict__ W, int n, int j0, int nbk,
                              int lane, float *__restrict__ qtau, float *__restrict__ sgn, float *__restrict__ T) {
  constexpr int kR = kWideMaxJ / 32;
  const int mrows = n - j0;
  float P[kR][kNb];
#pragma unroll
  for (int i = 0; i < kR; ++i) {
    const int row = lane + 32 * i;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (row < mrows) {
      a = __ldcg(reinterpret_cast<const float4 *>(Z + (int64_t)(j0 + row) * lz + j0));
      b = __ldcg(reinterpret_cast<const float4 *>(Z + (int64_t)(j0 + row) * lz + j0 + 4));
    }
    P[i][0] = a.x, P[i][1] = a.y, P[i][2] = a.z, P[i][3] = a.w;
    P[i][4] = b.x, P[i][5] = b.y, P[i][6] = b.z, P[i][7] = b.w;
  }
  float tv[kNb];
#pragma unroll
  for (int jj = 0; jj < kNb; ++jj) {
    tv[jj] = 0.f;
    if (jj >= nbk) continue;  // uniform
    const float alpha = __shfl_sync(0xffffffffu, P[0][jj], jj);
    float mx = 0.f, sq = 0.f;
#pragma unroll
    for (int i = 0; i < kR; ++i)
      if (lane + 32 * i > jj) {
        mx = fmaxf(mx, fabsf(P[i][jj]));
        sq = fmaf(P[i][jj], P[i][jj], sq);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    float t = 0.f, scal = 0.f, beta = alpha;
    if (mx > 0x1p-100f) {  // uniform
      float nrm;
      if (mx >= 0x1p-40f) {  // uniform
        nrm = sqrtf(fmaf(alpha, alpha, sq));
      } else {
        const float sm = fmaxf(mx, fabsf(alpha)), sx = 1.f / sm;
        float sg = 0.f;
#pragma unroll
        for (int i = 0; i < kR; ++i)
          if (lane + 32 * i > jj) {
            const float v = P[i][jj] * sx;
            sg = fmaf(v, v, sg);
          }
        sg = warp_sum32(sg);
        const float a = alpha * sx;
        nrm = sm * sqrtf(fmaf(a, a, sg));
      }
      beta = alpha >= 0.f ? -nrm : nrm;
      const float rb = __frcp_rn(beta), rd = __frcp_rn(alpha - beta);
      t = fmaf(-alpha, rb, 1.f);
      scal = rd;
    }
    tv[jj] = t;
    if (lane == 0) {
      qtau[j0 + jj] = t;
      sgn[j0 + jj] = beta < 0.f ? -1.f : 1.f;
    }
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      const int row = lane + 32 * i;
      P[i][jj] = row == jj ? 1.f : (row > jj && t != 0.f ? P[i][jj] * scal : 0.f);
    }
    if (t != 0.f) {
      float dd[kNb];
#pragma unroll
      for (int c = 0; c < kNb; ++c) {
        dd[c] = 0.f;
        if (c > jj)
#pragma unroll
          for (int i = 0; i < kR; ++i) dd[c] = fmaf(P[i][jj], P[i][c], dd[c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < kNb; ++c)
          if (c > jj) dd[c] += __shfl_xor_sync(0xffffffffu, dd[c], o);
#pragma unroll
      for (int c = 0; c < kNb; ++c)
        if (c > jj)
#pragma unroll
          for (int i = 0; i < kR; ++i) P[i][c] = fmaf(-t * dd[c], P[i][jj], P[i][c]);
    }
  }
#pragma unroll
  for (int i = 0; i < kR; ++i) {
    const int row = lane + 32 * i;
    if (row < mrows) {
      __stcg(reinterpret_cast<float4 *>(W + (int64_t)(j0 + row) * lz + j0), make_float4(P[i][0], P[i][1], P[i][2], P[i][3]));
      __stcg(reinterpret_cast<float4 *>(W + (int64_t)(j0 + row) * lz + j0 + 4), make_float4(P[i][4], P[i][5], P[i][6], P[i][7]));
    }
  }
  float G[kNb * kNb];
#pragma unroll
  for (int k = 0; k < kNb; ++k)
#pragma unroll
    for (int l = 0; l < kNb; ++l) {
      G[k * kNb + l] = 0.f;
      if (k < l)
#pragma unroll
        for (int i = 0; i < kR; ++i) G[k * kNb + l] = fmaf(P[i][k], P[i][l], G[k * kNb + l]);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < kNb; ++k)
#pragma unroll
      for (int l = k + 1; l < kNb; ++l) G[k * kNb + l] += __shfl_xor_sync(0xffffffffu, G[k * kNb + l], o);
  if (lane < kNb) wy_t_column(G, tv, lane, T);
  __syncwarp();
}

__global__ void __launch_bounds__(kW32Threads, 1) k_eig32_wide(const double *__restrict__ A, int lda, int n,
                                                             double *__restrict__ X, int ldx,
                                                             float *__restrict__ Zg, float *__restrict__ Lg) {
  extern __shared__ __align__(16) float smw[];
  float *Ap = smw;
  const WideLayout lay(n);
  float *d = smw + lay.vec, *e = d + n, *e2 = e + n, *tau = e2 + n, *lam = tau + n, *pv = lam + n;
  float *part = smw + lay.part;  // WY partial products (4 x kNb x kWideMaxJ)
  float *Tf = smw + lay.tf;      // T factors of the reflector blocks
  const int lz = tri32_ld(n);    // row stride of Zg and Lg
  __shared__ float red[33];
  __shared__ float sc[4];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  // ---- load A * 2^-s into the packed lower triangle (the upper triangle of
  // A read, as in k_eig32_tri: largest magnitude in [1/2, 1), entries 2^-126
  // below it flushed to zero, floats built from the float64 bits)
  unsigned mhi = 0u;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    if (r <= c) mhi = max(mhi, (unsigned)(__double_as_longlong(A[r + (int64_t)lda * c]) >> 32) & 0x7FFFFFFFu);
  }
  mhi = __reduce_max_sync(0xffffffffu, mhi);
  if (lane == 0) red[warp] = __uint_as_float(mhi);
  __syncthreads();
  if (tid == 0) {
    unsigned v = 0u;
    for (int w = 0; w < nw; ++w) v = max(v, __float_as_uint(red[w]));
    sc[0] = __uint_as_float(v);
  }
  __syncthreads();
  const unsigned amax = __float_as_uint(sc[0]);
  const int rebase = (int)(amax >> 20) - 126;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    if (r <= c) {  // A(r, c) = A(c, r): row c of packed column r
      const unsigned long long b = (unsigned long long)__double_as_longlong(A[r + (int64_t)lda * c]);
      const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b, mag = hi & 0x7FFFFFFFu;
      const int x = max((int)mag - (rebase << 20), 0);
      const unsigned f = (amax == 0u || mag == 0u) ? 0u : ((hi & 0x80000000u) | __funnelshift_l(lo, (unsigned)x, 3));
      Ap[packed_col(n, r) + (c - r)] = __uint_as_float(f);
    }
  }
  __syncthreads();

  // ---- 1. tridiagonalization
  for (int k = 0; k + 2 < n; ++k) {
    float *colk = Ap + packed_col(n, k);  // rows k..n-1 of column k
    const int m = n - k - 1;              // rows k+1..n-1: x, then v
    const Refl h = wide_larfg(colk + 1, m, red);
    if (tid == 0) {
      d[k] = colk[0];
      e[k] = h.beta;
      tau[k] = h.t;
    }
    if (tid < m) colk[1 + tid] = tid == 0 ? 1.f : colk[1 + tid] * h.scal;
    __syncthreads();
    const float t = h.t;
    const float *v = colk + 1;  // v[a], row k + 1 + a
    // p = t A22 v: four threads per row a, columns b = part (mod 4)
    {
      const int a = tid >> 2, part = tid & 3;
      float acc = 0.f;
      if (a < m) {
        const int ga = k + 1 + a;
        for (int b = part; b < m; b += 4) {
          const int gb = k + 1 + b;
          const float aab = b <= a ? Ap[packed_col(n, gb) + (ga - gb)] : Ap[packed_col(n, ga) + (gb - ga)];
          acc = fmaf(aab, v[b], acc);
        }
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (a < m && part == 0) pv[a] = t * acc;
    }
    __syncthreads();
    const float pvv = block_sum32(tid < m ? pv[tid] * v[tid] : 0.f, red);
    const float half = 0.5f * t * pvv;
    if (tid < m) pv[tid] = fmaf(-half, v[tid], pv[tid]);  // w
    __syncthreads();
    // A22 -= v w^T + w v^T on the packed lower triangle: warp per column b
    for (int b = warp; b < m; b += nw) {
      float *col = Ap + packed_col(n, k + 1 + b);  // rows k+1+b..: local rows a >= b
      const float vb = v[b], wb = pv[b];
      for (int a = b + lane; a < m; a += 32) col[a - b] -= fmaf(v[a], wb, pv[a] * vb);
    }
    __syncthreads();
  }
  if (tid == 0) {
    d[n - 2] = Ap[packed_col(n, n - 2)];
    e[n - 2] = Ap[packed_col(n, n - 2) + 1];
    d[n - 1] = Ap[packed_col(n, n - 1)];
    e[n - 1] = 0.f;
    tau[n - 2] = 0.f;
    tau[n - 1] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) e2[i] = e[i] * e[i];
  if (warp == 0) {  // Gershgorin bounds and ||T||
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int i = lane; i < n; i += 32) {
      const float r = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
      lo = fminf(lo, d[i] - r);
      hi = fmaxf(hi, d[i] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const float tn = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), FLT_MIN);
      sc[0] = lo - 0x1p-20f * tn;
      sc[1] = hi + 0x1p-20f * tn;
      sc[2] = tn;
    }
  }
  __syncthreads();
  const float gl = sc[0], gu = sc[1], tn = sc[2];
  const float piv = 0x1p-23f * tn;

  // ---- 2. multisection: threads 4 i .. 4 i + 3 find the i-th smallest eigenvalue
  {
    const int i = tid >> 2, sub = tid & 3;
    float lo = gl, hi = gu;
    for (int it = 0; it < 12; ++it) {
      const float x = lo + (hi - lo) * (0.2f * (float)(sub + 1));
      int cnt = 0;
      if (i < n) {
        float q = d[0] - x;
        for (int k = 0;; ++k) {
          if (fabsf(q) < piv) q = -piv;
          cnt += q < 0.f;
          if (k + 1 >= n) break;
          q = d[k + 1] - x - __fdividef(e2[k], q);
        }
      }
      float nlo = lo, nhi = hi;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int cs = __shfl_sync(0xffffffffu, cnt, (lane & ~3) | s);
        const float xs = __shfl_sync(0xffffffffu, x, (lane & ~3) | s);
        if (cs <= i) nlo = fmaxf(nlo, xs);
        else nhi = fminf(nhi, xs);
      }
      lo = nlo;
      hi = nhi;
    }
    if (i < n && sub == 0) lam[n - 1 - i] = 0.5f * (lo + hi);  // descending order
  }
  __syncthreads();

  // ---- 3. inverse iteration: thread c solves (T - l_c I) z = b twice
  for (int c = tid; c < n; c += nt) {
    const float s = lam[c];
    float D = d[0] - s;
    for (int k = 0; k + 1 < n; ++k) {
      if (fabsf(D) < piv) D = D < 0.f ? -piv : piv;
      const float L = __fdividef(e[k], D);
      Lg[k * lz + c] = L;
      D = d[k + 1] - s - L * e[k];
    }
    for (int pass = 0; pass < 2; ++pass) {
      float Dk = d[0] - s, y = 0.f;
      for (int k = 0; k < n; ++k) {  // forward: y = L^-1 b, z = D^-1 y
        if (k > 0) Dk = d[k] - s - Lg[(k - 1) * lz + c] * e[k - 1];
        if (fabsf(Dk) < piv) Dk = Dk < 0.f ? -piv : piv;
        const float b = pass == 0 ? start_entry(c, k) : Zg[k * lz + c];
        y = k == 0 ? b : b - Lg[(k - 1) * lz + c] * y;
        Zg[k * lz + c] = __fdividef(y, Dk);
      }
      float xn = Zg[(n - 1) * lz + c], nrm = xn * xn;
      for (int k = n - 2; k >= 0; --k) {  // backward: x = L^-T z
        xn = Zg[k * lz + c] - Lg[k * lz + c] * xn;
        Zg[k * lz + c] = xn;
        nrm = fmaf(xn, xn, nrm);
      }
      const bool good = nrm > 0.f && nrm <= FLT_MAX;
      const float r = good ? rsqrtf(nrm) : 0.f;
      for (int k = 0; k < n; ++k) Zg[k * lz + c] = good ? Zg[k * lz + c] * r : (k == c ? 1.f : 0.f);
    }
  }
  __syncthreads();

  // ---- 4. Zg <- Q of Zg = Q R (Householder), columns in descending eigenvalue
  // order, signs kept, in compact WY blocks of kNb as in k_eig32_tri: a warp
  // factors each panel in registers (reflectors to Lg, the L factors being
  // spent), the trailing columns take the panel at once; then the explicit Q
  // in Zg by the blocks applied to I in reverse order.
  float *qtau = lam, *sgn = e2;  // spent after steps 2 and 3
  float *W = Lg;
  for (int idx = tid; idx < n * lz; idx += nt) {
    const int r = idx / lz, c = idx - r * lz;
    if (c >= n) Zg[idx] = 0.f;  // padding columns stay zero (and finite)
    W[idx] = 0.f;
  }
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += kNb) {
    const int nbk = min(kNb, n - j0);
    float *Tb = Tf + (j0 / kNb) * kNb * kNb;
    if (warp == 0) qr_panel_wide(Zg, lz, W, n, j0, nbk, lane, qtau, sgn, Tb);
    __syncthreads();
    if (j0 + nbk < n) apply_wy_wide(Zg, lz, n, j0, j0 + nbk, W, lz, j0, Tb, true, part);
  }
  for (int idx = tid; idx < n * lz; idx += nt) {
    const int r = idx / lz, c = idx - r * lz;
    Zg[idx] = r == c ? 1.f : 0.f;
  }
  __syncthreads();
  for (int j0 = ((n - 1) / kNb) * kNb; j0 >= 0; j0 -= kNb)
    apply_wy_wide(Zg, lz, n, j0, j0, W, lz, j0, Tf + (j0 / kNb) * kNb * kNb, false, part);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx / n, c = idx - r * n;
    Zg[r * lz + c] *= sgn[c];
  }
  __syncthreads();

  // ---- 5. X = Q1 Zg: the tridiagonalization's reflectors (v_k in packed
  // column k below the subdiagonal, unit entry at row k + 1) copied to W,
  // their T factors, and the blocks from the last to the first
  const int nref = max(n - 2, 0);
  for (int idx = tid; idx < n * lz; idx += nt) {
    const int r = idx / lz, k = idx - r * lz;
    float v = 0.f;
    if (k < nref) v = r == k + 1 ? 1.f : (r > k + 1 && tau[k] != 0.f ? Ap[packed_col(n, k) + (r - k)] : 0.f);
    W[idx] = v;
  }
  __syncthreads();
  const int nblk = (nref + kNb - 1) / kNb;
  if (nblk > 0) form_wy_ts(W, lz, nblk, nref, 1, n, tau, Tf, part);  // the QR blocks' T factors are spent
  for (int j0 = (nblk - 1) * kNb; j0 >= 0; j0 -= kNb)
    apply_wy_wide(Zg, lz, n, j0 + 1, 0, W, lz, j0, Tf + (j0 / kNb) * kNb * kNb, false, part);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx % n, c = idx / n;
    X[r + (int64_t)ldx * c] = (double)__ldcg(Zg + (int64_t)r * lz + c);
  }
}

// ---------------------------------------------------------------------------
// First stage for kWideMaxJ < n <= kMpMaxJ: float32 parallel-order cyclic
// Jacobi on A / max|A| over a cluster of kJ32ClCtas CTAs.  The float32 S
// (full, row-major, kept symmetric) and V (column-major) of m = n rounded up
// to a multiple of 4 live in global memory (4 MB at n = 512: L2-resident)
// and are updated in place.  Each step of the round-robin tournament (every
// pair meets once in m - 1 steps): every CTA forms the step's m/2 rotations
// from S's current entries (the same values in every CTA), applies its fixed
// share of the 2 x 2 blocks {p_P, q_P} x {p_Q, q_Q} of S (P <= Q, mirrored)
// and of V's column pairs.  The cluster meets at two barriers per step (after
// the rotations are read, so that no CTA overwrites an entry another is still
// reading, and after the updates), whose release/acquire order makes the
// step's writes visible to the next step.
// S and V are read and written at L2 (ld.global.cg): no stale L1 line of
// another CTA's data is ever read.  A rotation is taken while |s_pq|
// exceeds 2^-23 times the largest diagonal magnitude at the start of the
// sweep, as in k_jacobi32; the sweeps stop when a whole sweep takes none
// (the cluster agrees through per-CTA flags) or after kJ32MaxSweeps.
// Writes X = V (float64, unsorted columns) and the number of sweeps.
// ---------------------------------------------------------------------------
constexpr int kJ32ClCtas = 16;
constexpr int kJ32ClThreads = 1024;
constexpr int kJ32ClBlocksPerThread = (kMpMaxJ / 2) * (kMpMaxJ / 2 + 1) / 2 / (kJ32ClCtas * kJ32ClThreads) + 1;
constexpr int kJ32ClVPerThread = (kMpMaxJ / 2) * (kMpMaxJ / 4) / (kJ32ClCtas * kJ32ClThreads);

__global__ void __launch_bounds__(kJ32ClThreads)
    k_jacobi32_cl(const double *__restrict__ A, int lda, int n, float *S, float *V, int *flags,
                  double *__restrict__ X, int ldx, int *__restrict__ sweeps) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ float4 rot[kMpMaxJ / 2];  // per pair: c, s, t = s / c, (p | q << 16) as bits
  __shared__ float red[kJ32ClThreads / 32];
  __shared__ float scale_s, tol_s;
  __shared__ int rotated;
  const int m = (n + 3) & ~3, np = m / 2;
  const int nblk = np * (np + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = (int)cl.block_rank();
  const int gt = rank * kJ32ClThreads + tid, gstride = kJ32ClCtas * kJ32ClThreads;

  // scale: every CTA finds max|A| itself
  float mx = 0.f;
  for (int e = tid; e < n * n; e += kJ32ClThreads) mx = fmaxf(mx, (float)fabs(A[(e % n) + (int64_t)lda * (e / n)]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
    for (int w = 0; w < kJ32ClThreads / 32; ++w) v = fmaxf(v, red[w]);
    scale_s = v;
  }
  __syncthreads();
  const double inv = scale_s > 0.f ? 1.0 / (double)scale_s : 0.0;
  for (int e = gt; e < m * m; e += gstride) {
    const int i = e / m, j = e - (e / m) * m;
    const int lo = min(i, j), hi = max(i, j);  // read the upper triangle, mirror it
    __stcg(S + e, (hi < n) ? (float)(A[lo + (int64_t)lda * hi] * inv) : 0.f);
    __stcg(V + e, (i == j) ? 1.f : 0.f);
  }
  // this thread's blocks (P, Q), P <= Q, fixed for the whole run
  int myblk[kJ32ClBlocksPerThread];
#pragma unroll
  for (int k = 0; k < kJ32ClBlocksPerThread; ++k) {
    const int e = gt + k * gstride;
    myblk[k] = -1;
    if (e < nblk) {
      int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((q + 1) * (q + 2) / 2 <= e) ++q;
      while (q * (q + 1) / 2 > e) --q;
      myblk[k] = (e - q * (q + 1) / 2) | (q << 16);
    }
  }
  cl.sync();

  int sweep = 0;
  for (; sweep < kJ32MaxSweeps; ++sweep) {
    if (warp == 0) {
      float d = 0.f;
      for (int i = lane; i < m; i += 32) d = fmaxf(d, fabsf(__ldcg(S + (int64_t)i * m + i)));
      for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
      if (lane == 0) {
        tol_s = FLT_EPSILON * fmaxf(d, FLT_MIN);
        rotated = 0;
      }
    }
    __syncthreads();
    const float tol = tol_s;
    for (int step = 0; step < m - 1; ++step) {
      if (tid < np) {
        const int t = tid;
        int p = (t == 0) ? 0 : ((t - 1 + step) % (m - 1)) + 1;
        int q = ((m - 2 - t + step) % (m - 1)) + 1;
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        float c = 1.f, sv = 0.f, tt = 0.f;
        // the three entries in one round trip
        const float b = __ldcg(S + (int64_t)p * m + q), a = __ldcg(S + (int64_t)p * m + p),
                    d = __ldcg(S + (int64_t)q * m + q);
        if (fabsf(b) > tol) {
          const float tau = __fdividef(d - a, 2.f * b);
          const float at = fabsf(tau);
          const float h = fmaf(tau, tau, 1.f);
          tt = at > 1e18f ? __fdividef(0.5f, tau) : copysignf(__fdividef(1.f, at + h * rsqrtf(h)), tau);
          c = rsqrtf(fmaf(tt, tt, 1.f));
          sv = tt * c;
          if (sv != 0.f) rotated = 1;
        }
        rot[t] = make_float4(c, sv, tt, __int_as_float(p | (q << 16)));
      }
      // every CTA has read the entries its rotations come from before any CTA
      // overwrites them (the diagonal blocks' owners zero s_pq)
      cl.sync();
      // Every entry of S belongs to one 2 x 2 block and every V column pair to
      // one unit, each applied by one thread: all of this thread's loads go
      // first (one round trip to L2), then the updates and stores.
      float4 xs[kJ32ClBlocksPerThread];
      bool live[kJ32ClBlocksPerThread];
#pragma unroll
      for (int k = 0; k < kJ32ClBlocksPerThread; ++k) {
        const int pq = myblk[k];
        live[k] = false;
        xs[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pq < 0) continue;
        const int P = pq & 0xFFFF, Q = pq >> 16;
        const float4 rP = rot[P], rQ = rot[Q];
        const int kP = __float_as_int(rP.w), kQ = __float_as_int(rQ.w);
        const int64_t p1 = kP & 0xFFFF, q1 = kP >> 16, p2 = kQ & 0xFFFF, q2 = kQ >> 16;
        if (P == Q) {
          if (rP.y == 0.f) continue;
          live[k] = true;  // s_pq, s_pp, s_qq
          xs[k] = make_float4(__ldcg(S + p1 * m + q1), __ldcg(S + p1 * m + p1), __ldcg(S + q1 * m + q1), 0.f);
        } else {
          if (rP.y == 0.f && rQ.y == 0.f) continue;
          live[k] = true;
          xs[k] = make_float4(__ldcg(S + p1 * m + p2), __ldcg(S + p1 * m + q2), __ldcg(S + q1 * m + p2),
                              __ldcg(S + q1 * m + q2));
        }
      }
      const int nq = m / 4;  // V's column pairs: unit u = (pair t, row quad r4)
      float4 va[kJ32ClVPerThread + 1], vb[kJ32ClVPerThread + 1];
#pragma unroll
      for (int k = 0; k <= kJ32ClVPerThread; ++k) {
        const int u = gt + k * gstride;
        va[k] = vb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u >= np * nq) continue;
        const int t = u / nq, r4 = u - t * nq;
        const float4 r = rot[t];
        if (r.y == 0.f) continue;
        const int kk = __float_as_int(r.w);
        va[k] = __ldcg(reinterpret_cast<const float4 *>(V + (int64_t)(kk & 0xFFFF) * m) + r4);
        vb[k] = __ldcg(reinterpret_cast<const float4 *>(V + (int64_t)(kk >> 16) * m) + r4);
      }
#pragma unroll
      for (int k = 0; k < kJ32ClBlocksPerThread; ++k) {
        if (!live[k]) continue;
        const int pq = myblk[k];
        const int P = pq & 0xFFFF, Q = pq >> 16;
        const float4 rP = rot[P];
        const int kP = __float_as_int(rP.w);
        const int64_t p1 = kP & 0xFFFF, q1 = kP >> 16;
        if (P == Q) {
          const float b = xs[k].x;
          __stcg(S + p1 * m + p1, xs[k].y - rP.z * b);
          __stcg(S + q1 * m + q1, xs[k].z + rP.z * b);
          __stcg(S + p1 * m + q1, 0.f);
          __stcg(S + q1 * m + p1, 0.f);
          continue;
        }
        const float4 rQ = rot[Q];
        const float s1 = rP.y, s2 = rQ.y, c1 = rP.x, c2 = rQ.x;
        const int kQ = __float_as_int(rQ.w);
        const int64_t p2 = kQ & 0xFFFF, q2 = kQ >> 16;
        const float x11 = xs[k].x, x12 = xs[k].y, x21 = xs[k].z, x22 = xs[k].w;
        const float y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
        const float y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
        const float z11 = y11 * c2 - y12 * s2, z12 = y11 * s2 + y12 * c2;
        const float z21 = y21 * c2 - y22 * s2, z22 = y21 * s2 + y22 * c2;
        __stcg(S + p1 * m + p2, z11);
        __stcg(S + p2 * m + p1, z11);
        __stcg(S + p1 * m + q2, z12);
        __stcg(S + q2 * m + p1, z12);
        __stcg(S + q1 * m + p2, z21);
        __stcg(S + p2 * m + q1, z21);
        __stcg(S + q1 * m + q2, z22);
        __stcg(S + q2 * m + q1, z22);
      }
#pragma unroll
      for (int k = 0; k <= kJ32ClVPerThread; ++k) {
        const int u = gt + k * gstride;
        if (u >= np * nq) continue;
        const int t = u / nq, r4 = u - t * nq;
        const float4 r = rot[t];
        if (r.y == 0.f) continue;
        const float c = r.x, sv = r.y;
        const int kk = __float_as_int(r.w);
        float4 *vp = reinterpret_cast<float4 *>(V + (int64_t)(kk & 0xFFFF) * m) + r4;
        float4 *vq = reinterpret_cast<float4 *>(V + (int64_t)(kk >> 16) * m) + r4;
        const float4 a = va[k], b = vb[k];
        __stcg(vp, make_float4(c * a.x - sv * b.x, c * a.y - sv * b.y, c * a.z - sv * b.z, c * a.w - sv * b.w));
        __stcg(vq, make_float4(sv * a.x + c * b.x, sv * a.y + c * b.y, sv * a.z + c * b.z, sv * a.w + c * b.w));
      }
      cl.sync();
    }
    // the cluster agrees on whether any CTA rotated during the sweep
    if (tid == 0) __stcg(flags + (sweep & 1) * kJ32ClCtas + rank, rotated);
    cl.sync();
    int any = 0;
    for (int r = 0; r < kJ32ClCtas; ++r) any |= __ldcg(flags + (sweep & 1) * kJ32ClCtas + r);
    if (!any) {
      ++sweep;
      break;
    }
  }
  for (int e = gt; e < n * n; e += gstride) {
    const int i = e % n, j = e / n;
    X[i + (int64_t)ldx * j] = (double)__ldcg(V + (int64_t)j * m + i);
  }
  if (rank == 0 && tid == 0 && sweeps) *sweeps = sweep;
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
  __shared__ double As[kGT][kGemmMaxK + 1];
  __shared__ double Bs[kGT][kGemmMaxK + 1];
  const int m0 = blockIdx.x * kGT, n0 = blockIdx.y * kGT;
  const int tx = threadIdx.x % kGT, ty = threadIdx.x / kGT;
  const int i = m0 + tx, j = n0 + ty;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += kGemmMaxK) {  // contraction rows in stages of kGemmMaxK
    const int kn = min(kGemmMaxK, K - k0);
    if (k0 > 0) __syncthreads();
    for (int e = threadIdx.x; e < kGT * kn; e += kGT * kGT) {
      const int r = e % kGT, k = k0 + e / kGT;
      const int ii = m0 + r;
      double a = 0.0;
      if (ii < M) a = transA ? A[k + (int64_t)lda * ii] : A[ii + (int64_t)lda * k];
      As[r][k - k0] = a;
      const int jj = n0 + r;
      Bs[r][k - k0] = jj < N ? B[k + (int64_t)ldb * jj] : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < kn; ++k) acc = fma(As[tx][k], Bs[ty][k], acc);
  }
  if (i >= M || j >= N) return;
  if (D) acc += D[i + (int64_t)ldd * j];
  C[i + (int64_t)ldc * j] = acc;
}

// ---------------------------------------------------------------------------
// Refinement step kernels.  G = X^T [A X | X] (m x 2m): S = G[:, :m],
// X^T X = G[:, m:].  The m^2-sized passes run on many CTAs (the float64 pipe
// of one SM would take tens of microseconds); the partition is one CTA.
// ---------------------------------------------------------------------------
constexpr int kStatBlocks = 64;
constexpr int kStatThreads = 256;

struct LevelInfo {
  double norm_a;   // ||A||_F of the level's matrix
  double delta;    // cluster gap: eigenvalue approximations are this accurate
  int nclusters;
  int start[kMpMaxJ + 1];
  double csum[kMpMaxJ];  // per cluster, the sum of its eigenvalue approximations
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

// Per-CTA partial sums: part[3 b + 0] = ||off(S)||^2, [1] = ||I - X^T X||^2,
// [2] = ||A||^2 (with G == nullptr: [0] = ||A - mu I||^2, [1] = mu = tr(A) / m).
__global__ void __launch_bounds__(kStatThreads) k_oa_stats(const double *__restrict__ G, int m,
                                                           const double *__restrict__ A, int lda,
                                                           double *__restrict__ part) {
  __shared__ double red[kStatThreads / 32];
  __shared__ double mu_s;
  if (!G) {
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int i = threadIdx.x; i < m; i += 32) t += A[i + (int64_t)lda * i];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) mu_s = t / m;
    }
    __syncthreads();
  }
  const double mu = G ? 0.0 : mu_s;
  double off2 = 0.0, r2 = 0.0, a2 = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int j = e / m, i = e - j * m;
    const double a = A[i + (int64_t)lda * j];
    a2 += a * a;
    if (!G) {
      const double d = a - (i == j ? mu : 0.0);
      off2 += d * d;
      continue;
    }
    const double sv = G[e];
    const double r = (i == j ? 1.0 : 0.0) - G[(int64_t)m * m + e];
    if (i != j) off2 += sv * sv;
    r2 += r * r;
  }
  off2 = block_sum(off2, red);
  r2 = block_sum(r2, red);
  a2 = block_sum(a2, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = off2;
    part[3 * blockIdx.x + 1] = G ? r2 : mu;  // without G: the mean of the diagonal
    part[3 * blockIdx.x + 2] = a2;
  }
}

// A <- A - mu I (m x m, ld lda).
__global__ void k_shift_diag(double *A, int lda, int m, double mu) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) A[i + (int64_t)lda * i] -= mu;
}

// A total order on doubles as unsigned integers (finite values and +-0).
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// First step of a level: eigenvalue approximations l_i = s_ii / (X^T X)_ii,
// sorted descending (ties by index) into perm, and clusters of the sorted
// order (label per position, starts in info).  noise < 0 stands for ||A||_F
// (the top level).
__global__ void __launch_bounds__(256) k_oa_partition(const double *__restrict__ G, int m,
                                                      const double *__restrict__ part, double noise,
                                                      int *__restrict__ perm_out, int *__restrict__ label,
                                                      LevelInfo *__restrict__ info) {
  __shared__ double lam[kMpMaxJ];
  __shared__ unsigned long long key[kMpMaxJ];
  __shared__ int perm[kMpMaxJ];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m; i += nt) {
    lam[i] = G[i + (int64_t)m * i] / G[(int64_t)m * m + i + (int64_t)m * i];
    key[i] = order_key(lam[i]);
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    int rank = 0;
    const unsigned long long ki = key[i];
    for (int j = 0; j < m; ++j) rank += (key[j] > ki) || (key[j] == ki && j < i);
    perm[rank] = i;
  }
  __syncthreads();
  if (tid == 0) {
    double off2 = 0.0, r2 = 0.0, a2 = 0.0;
    for (int b = 0; b < kStatBlocks; ++b) {  // fixed order
      off2 += part[3 * b];
      r2 += part[3 * b + 1];
      a2 += part[3 * b + 2];
    }
    if (noise < 0.0) noise = sqrt(a2);
    const double delta = kClusterC * (sqrt(off2) + sqrt(a2) * sqrt(r2) + m * kU * noise);
    int k = 0;
    info->start[0] = 0;
    label[0] = 0;
    double cs = lam[perm[0]];
    for (int a = 1; a < m; ++a) {
      if (lam[perm[a - 1]] - lam[perm[a]] > delta) {
        info->csum[k] = cs;
        cs = 0.0;
        info->start[++k] = a;
      }
      cs += lam[perm[a]];
      label[a] = k;
    }
    info->csum[k] = cs;
    info->nclusters = k + 1;
    info->start[k + 1] = m;
    info->norm_a = sqrt(a2);
    info->delta = delta;
  }
  for (int a = tid; a < m; a += nt) perm_out[a] = perm[a];
}

// E of a refinement step, in the basis permuted by perm (nullptr: identity),
// with the clusters `label` of the permuted positions; with Xp != nullptr
// also Xp = X perm.
__global__ void __launch_bounds__(kStatThreads) k_oa_E(const double *__restrict__ G, int m,
                                                       const int *__restrict__ perm, const int *__restrict__ label,
                                                       const double *__restrict__ X, double *__restrict__ Xp,
                                                       double *__restrict__ E) {
  __shared__ double lam[kMpMaxJ];
  __shared__ int lab[kMpMaxJ], pm[kMpMaxJ];
  const double *S = G;
  const double *P = G + (int64_t)m * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    lam[i] = S[i + (int64_t)m * i] / P[i + (int64_t)m * i];
    lab[i] = label[i];
    pm[i] = perm ? perm[i] : i;
  }
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int b = e / m, a = e - b * m;
    const int i = pm[a], j = pm[b];
    if (Xp) Xp[e] = X[a + (int64_t)m * j];
    const double r = (i == j ? 1.0 : 0.0) - P[i + (int64_t)m * j];
    double v;
    // S = X^T A X is symmetric in exact arithmetic; its computed form is not
    // (rounding of order m u ||A||).  Only its symmetric part enters E:
    // otherwise that asymmetry, divided by the gap lam_j - lam_i, leaves
    // E + E^T != R and the step cannot restore orthogonality.
    if (a == b || lab[a] == lab[b]) v = 0.5 * r;
    else v = (0.5 * (S[i + (int64_t)m * j] + S[j + (int64_t)m * i]) + lam[j] * r) / (lam[j] - lam[i]);
    E[e] = v;
  }
}

// P <- (3 I - P) / 2 (the Newton-Schulz coefficient matrix; P is m x m).
__global__ void k_ns_coef(double *P, int m) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;
    P[e] = (i == j ? 1.5 : 0.0) - 0.5 * P[e];
  }
}

// the eigensolver's info record: sweeps, not converged, path, resolved count
__global__ void k_set_info(int *info, int sweeps, int noconv, int path, int resolved) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  info[0] = sweeps;
  info[1] = noconv;
  info[2] = path;
  info[3] = resolved;
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
                                                      const double *__restrict__ X, int m, int u0,
                                                      double *__restrict__ lam_out, double *__restrict__ V_out,
                                                      double *__restrict__ check) {
  __shared__ double lam[kMpMaxJ];
  __shared__ int rk[kMpMaxJ];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double *S = G;
  const double *P = G + (int64_t)m * m;
  for (int i = tid; i < m; i += nt) lam[i] = S[i + (int64_t)m * i] / P[i + (int64_t)m * i];
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const double di = lam[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (lam[j] > di) || (lam[j] == di && j < i);
    rk[i] = rank;
  }
  __syncthreads();
  // The check's maxima are of magnitudes, so they are taken on the bit
  // patterns (ordered like the values for non-negative doubles) on the
  // integer pipe; the float64 pipe (2 lanes per clock per SM here) does only
  // the residual's multiply-subtract and the diagonal's subtraction.  A NaN
  // in T or P makes the residual infinite, so the result fails the check.
  constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  const int lane = tid & 31, warp = tid >> 5;
  unsigned long long res = 0ull, orth = 0ull, lmax = 0ull;
  for (int j = warp; j < m; j += nt / 32) {
    const bool resolved = rk[j] < u0;  // columns sorted at or past u0 span the unresolved tail clusters
    const double lj = lam[j];
    for (int i = lane; i < m; i += 32) {
      const int64_t e = i + (int64_t)m * j;
      const double t = T[e], p = P[e];
      const unsigned long long tb = (unsigned long long)__double_as_longlong(t) & kMag;
      const unsigned long long pb = (unsigned long long)__double_as_longlong(p) & kMag;
      if (resolved) res = max(res, (unsigned long long)__double_as_longlong(t - X[e] * lj) & kMag);
      orth = max(orth, i == j ? (unsigned long long)__double_as_longlong(p - 1.0) & kMag : pb);
      if (tb > kInf || pb > kInf) res = kInf;  // NaN
    }
  }
  for (int i = tid; i < m; i += nt) lmax = max(lmax, (unsigned long long)__double_as_longlong(lam[i]) & kMag);
  for (int o = 16; o > 0; o >>= 1) {
    res = max(res, __shfl_xor_sync(0xffffffffu, res, o));
    orth = max(orth, __shfl_xor_sync(0xffffffffu, orth, o));
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  __shared__ unsigned long long rr[32], oo[32], ll[32];
  if (lane == 0) {
    rr[warp] = res;
    oo[warp] = orth;
    ll[warp] = lmax;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0ull, b = 0ull, c = 0ull;
    for (int w = 0; w < nt / 32; ++w) {
      a = max(a, rr[w]);
      b = max(b, oo[w]);
      c = max(c, ll[w]);
    }
    // a residual of NaN (from X or lam) stays NaN: it fails the check too
    check[0] = __longlong_as_double((long long)a);
    check[1] = __longlong_as_double((long long)b);
    check[2] = __longlong_as_double((long long)c);
  }
  // column i, sorted to position rk[i], signed so that its first entry of
  // largest magnitude is positive: a warp per column, lanes over rows
  // (coalesced), the first maximum by a (magnitude, row) reduction
  for (int i = warp; i < m; i += nt / 32) {
    const int rank = rk[i];
    if (lane == 0) lam_out[rank] = lam[i];
    const double *col = X + (int64_t)m * i;
    double best = -1.0;
    int br = m;
    for (int r = lane; r < m; r += 32) {
      const double v = fabs(col[r]);
      if (v > best) {  // NaN never wins, as in a scan over the rows
        best = v;
        br = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int orr = __shfl_xor_sync(0xffffffffu, br, o);
      if (ob > best || (ob == best && orr < br)) {
        best = ob;
        br = orr;
      }
    }
    const double sg = (br < m && col[br] < 0.0) ? -1.0 : 1.0;
    for (int r = lane; r < m; r += 32) V_out[r + (int64_t)m * rank] = sg * col[r];
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
  double *part = nullptr;     // 3 kStatBlocks partial sums
  double *check = nullptr;    // 4 doubles
  int *sweeps = nullptr;      // 1 int
  int *labels = nullptr;      // per depth, J ints
  int *perms = nullptr;       // per depth, J ints
  LevelInfo *info = nullptr;  // per depth (device)
  static size_t bytes(int J) {
    return ((size_t)kMaxDepth * 9 * J * J + 3 * kStatBlocks + 8) * sizeof(double) +
           (size_t)2 * kMaxDepth * J * sizeof(int) + (size_t)kMaxDepth * sizeof(LevelInfo) + 64;
  }
  void carve(void *mem, int J_) {
    J = J_;
    base = static_cast<double *>(mem);
    part = base + (size_t)kMaxDepth * 9 * J * J;
    check = part + 3 * kStatBlocks;
    sweeps = reinterpret_cast<int *>(check + 4);
    labels = reinterpret_cast<int *>(check + 8);
    perms = labels + kMaxDepth * J;
    info = reinterpret_cast<LevelInfo *>((reinterpret_cast<uintptr_t>(perms + kMaxDepth * J) + 15) &
                                         ~static_cast<uintptr_t>(15));
  }
};

// The cluster Jacobi stage on a 16-CTA cluster (non-portable size, allowed
// explicitly).  tx (float64, ld m) receives V.
int launch_jacobi32_cl(const double *A, int lda, int m, float *S32, float *V32, int *flags, double *X, int ldx,
                       int *sweeps, cudaStream_t s) {
  static const bool ok = [] {
    if (cudaFuncSetAttribute(k_jacobi32_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  }();
  if (!ok) {
    set_error("the eigensolver's 16-CTA cluster is not available on this device");
    return TUCKER_EUNSUPPORTED;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kJ32ClCtas);
  cfg.blockDim = dim3(kJ32ClThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kJ32ClCtas;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  TK_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi32_cl, A, lda, m, S32, V32, flags, X, ldx, sweeps));
  TK_LAUNCHED();
  return TUCKER_OK;
}

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

// ||A - mu I||_F (mu = tr(A) / m) and ||A||_F, on the host.
int scalar_deviation(const double *A, int lda, int m, const MpWork &w, cudaStream_t s, double *dev, double *norm,
                     double *mean = nullptr) {
  k_oa_stats<<<kStatBlocks, kStatThreads, 0, s>>>(nullptr, m, A, lda, w.part);
  TK_LAUNCHED();
  double h[3 * kStatBlocks];
  TK_CUDA(cudaMemcpyAsync(h, w.part, sizeof h, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  double d2 = 0.0, a2 = 0.0;
  for (int b = 0; b < kStatBlocks; ++b) {
    d2 += h[3 * b];
    a2 += h[3 * b + 2];
  }
  *dev = std::sqrt(d2);
  if (norm) *norm = std::sqrt(a2);
  if (mean) *mean = h[1];
  return TUCKER_OK;
}

// One level: eigenvectors of A (m x m, lda) into out (m x m, ld m).  noise is
// ||A||_F of the top problem: the float64 noise floor of every level.
// budget >= 0: clusters whose eigenvalues, with everything after them in
// descending order (tail_after this level's matrix, accurate to tail_err),
// sum to at most budget are left unresolved; their column count goes to
// *skipped.
int mp_level(const double *A, int lda, int m, double noise, int depth, const MpWork &w, double *out, cudaStream_t s,
             double budget, double tail_after, double tail_err, int *skipped, double shift = 0.0) {
  double *tx0 = w.tx(depth, 0), *tx1 = w.tx(depth, 1);
  double *G = w.g(depth), *E = w.e(depth);
  int *label = w.labels + depth * w.J, *perm = w.perms + depth * w.J;
  LevelInfo *dinfo = w.info + depth;
  // float32 first stage: the tridiagonal solver, or the Jacobi sweeps with
  // TUCKER_EIG32=jacobi (same accuracy; kept for comparison)
  static const bool use_jacobi = [] {
    const char *e = std::getenv("TUCKER_EIG32");
    return e && std::strcmp(e, "jacobi") == 0;
  }();
  if (m > kWideMaxJ) {  // the cluster Jacobi stage: S, V and the flags in this depth's (free) tx1 region
    const int mp = (m + 3) & ~3;
    float *f = reinterpret_cast<float *>(w.tx(depth, 1));
    f += (4 - (reinterpret_cast<uintptr_t>(f) / sizeof(float)) % 4) % 4;  // 16-byte aligned
    float *S32 = f, *V32 = f + (size_t)mp * mp;
    int *flags = reinterpret_cast<int *>(V32 + (size_t)mp * mp);
    TK_CHECK(launch_jacobi32_cl(A, lda, m, S32, V32, flags, tx0 + (size_t)m * m, m, depth == 0 ? w.sweeps : nullptr,
                                s));
    // Thousands of float32 rotations per column leave ||I - X^T X|| near
    // 1e-5 at m = 512, and the refinement's cluster width grows with it
    // (the ||A|| ||R|| term): two Newton-Schulz steps X <- X (3 I - X^T X) / 2
    // in float64 bring it to rounding level first (R -> ~(3/4) R^2 each).
    double *X = tx0 + (size_t)m * m, *Xn = tx1 + (size_t)m * m;
    for (int it = 0; it < 2; ++it) {
      TK_CHECK(gemm(m, m, m, X, m, 1, X, m, nullptr, 0, E, m, s));
      k_ns_coef<<<(m * m + 255) / 256, 256, 0, s>>>(E, m);
      TK_LAUNCHED();
      TK_CHECK(gemm(m, m, m, X, m, 0, E, m, nullptr, 0, Xn, m, s));
      k_copy_cols<<<(m * m + 255) / 256, 256, 0, s>>>(Xn, m, X, m, m, m);
      TK_LAUNCHED();
    }
  } else if (m > kTriMaxJ) {
    // the wide stage; G (m x 2m float64, free until the refinement) holds its
    // two m x tri32_ld(m) float arrays, which it reads and writes as 16-byte
    // vectors: the workspace's regions start at 8-byte multiples only (odd J),
    // so the arrays start at G rounded up to 16 bytes (G has 16 J^2 bytes; the
    // arrays need 8 m (m + 8))
    const size_t smemw = wide32_smem(m);
    TK_CUDA(allow_max_smem(k_eig32_wide));
    float *zs = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(G) + 15) & ~static_cast<uintptr_t>(15));
    if ((reinterpret_cast<uintptr_t>(zs) & 15) != 0 || ((size_t)m * tri32_ld(m) * sizeof(float)) % 16 != 0) {
      set_error("wide eigensolver stage: unaligned scratch");
      return TUCKER_ECUDA;
    }
    k_eig32_wide<<<1, kW32Threads, smemw, s>>>(A, lda, m, tx0 + (size_t)m * m, m, zs, zs + (size_t)m * tri32_ld(m));
  } else if (use_jacobi) {
    const size_t smem32 = jacobi32_smem(m);
    TK_CUDA(allow_max_smem(k_jacobi32));
    k_jacobi32<<<1, kJ32Threads, smem32, s>>>(A, lda, m, tx0 + (size_t)m * m, m, depth == 0 ? w.sweeps : nullptr);
  } else {
    const size_t smemt = tri32_smem(m);
    TK_CUDA(allow_max_smem(k_eig32_tri));
    k_eig32_tri<<<1, kT32Threads, smemt, s>>>(A, lda, m, tx0 + (size_t)m * m, m);
  }
  TK_LAUNCHED();
  // first refinement step: clusters and the permuted basis
  TK_CHECK(products(A, lda, m, tx0, G, s));
  k_oa_stats<<<kStatBlocks, kStatThreads, 0, s>>>(G, m, A, lda, w.part);
  TK_LAUNCHED();
  k_oa_partition<<<1, 256, 0, s>>>(G, m, w.part, noise, perm, label, dinfo);
  TK_LAUNCHED();
  k_oa_E<<<kStatBlocks, kStatThreads, 0, s>>>(G, m, perm, label, tx0 + (size_t)m * m, tx1 + (size_t)m * m, E);
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
    k_oa_E<<<kStatBlocks, kStatThreads, 0, s>>>(G, m, nullptr, label, nullptr, nullptr, E);
    TK_LAUNCHED();
    return apply();
  };
  TK_CHECK(apply());
  for (int k = 1; k < kRefineSteps; ++k) TK_CHECK(refine());
  LevelInfo h;
  TK_CUDA(cudaMemcpyAsync(&h, dinfo, sizeof h, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  double *X = cur + (size_t)m * m;
  // suffix sums of the clusters' eigenvalue approximations; the first
  // cluster whose suffix (with its error) fits the budget, and all after it,
  // stay unresolved: a rank cut never falls inside them
  double suffix[kMpMaxJ + 1];
  suffix[h.nclusters] = 0.0;
  // (this level's matrix is the original one shifted by -shift)
  for (int k = h.nclusters - 1; k >= 0; --k)
    suffix[k] = suffix[k + 1] + h.csum[k] + shift * (double)(h.start[k + 1] - h.start[k]);
  int first_skip = h.nclusters;
  if (budget >= 0.0)
    for (int k = 0; k < h.nclusters; ++k)
      if (suffix[k] + tail_after + tail_err + (double)(m - h.start[k]) * h.delta <= budget) {
        first_skip = k;
        break;
      }
  if (first_skip < h.nclusters) *skipped += m - h.start[first_skip];
  for (int k = 0; k < first_skip; ++k) {
    const int c0 = h.start[k], mc = h.start[k + 1] - c0;
    if (mc < 2 || depth + 1 >= kMaxDepth) continue;
    // C = X_c^T A X_c; a multiple of I up to the noise floor needs no rotation
    double *T = w.t(depth), *C = w.c(depth);
    TK_CHECK(gemm(m, mc, m, A, lda, 0, X + (size_t)m * c0, m, nullptr, 0, T, m, s));
    TK_CHECK(gemm(mc, mc, m, X + (size_t)m * c0, m, 1, T, m, nullptr, 0, C, mc, s));
    double dev = 0.0, mu = 0.0;
    TK_CHECK(scalar_deviation(C, mc, mc, w, s, &dev, nullptr, &mu));
    if (dev <= kClusterC * mc * kU * noise) continue;
    // The child solves C - mu I (same eigenvectors): its float32 stage then
    // resolves the cluster's spread rather than its magnitude, and its cluster
    // width scales with ||C - mu I||.  Without the shift a tight cluster of
    // large eigenvalues (say 200 within 10%) stays one cluster at every depth.
    k_shift_diag<<<(mc + 255) / 256, 256, 0, s>>>(C, mc, mc, mu);
    TK_LAUNCHED();
    double *Q = w.e(depth + 1);  // the child's E is free once it has returned
    double *Qc = w.t(depth + 1);
    TK_CHECK(mp_level(C, mc, mc, noise, depth + 1, w, Qc, s, budget, tail_after + suffix[k + 1],
                      tail_err + (double)(m - h.start[k + 1]) * h.delta, skipped, shift + mu));
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
static thread_local double g_mp_check[5];

const double *mp_last_check() { return g_mp_check; }

int mp_max_j() {
  // J above kTriMaxJ takes the wide float32 stage (up to kWideMaxJ) or the
  // cluster float32 Jacobi (up to kMpMaxJ); TUCKER_EIG_WIDE=0 restricts the
  // mixed-precision solver to J <= kTriMaxJ (the float64 Jacobi above)
  static const int lim = [] {
    const char *e = std::getenv("TUCKER_EIG_WIDE");
    return e && e[0] == '0' ? kTriMaxJ : kMpMaxJ;
  }();
  return lim;
}

int launch_eig_mp(const double *d_S, int64_t J, double *d_lam, double *d_V, int *d_info, int *verified,
                  cudaStream_t s, Prof *prof, double tail_budget) {
  *verified = 0;
  if (J < 1 || J > mp_max_j()) return TUCKER_OK;
  const int m = (int)J;
  void *mem = nullptr;
  TK_CUDA(cudaMallocAsync(&mem, MpWork::bytes(m), s));
  struct Free {
    void *p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } guard{mem, s};
  MpWork w;
  w.carve(mem, m);

  if (prof) prof->begin(TUCKER_PHASE_EIG);
  double dev = 0.0, noise = 0.0;
  TK_CHECK(scalar_deviation(d_S, m, m, w, s, &dev, &noise));
  double *X = w.c(kMaxDepth - 1);  // never a cluster block: the deepest level takes no clusters
  int sw = 0, skipped = 0;
  TK_CUDA(cudaMemsetAsync(w.sweeps, 0, sizeof(int), s));
  if (dev <= kClusterC * m * kU * noise) {
    k_set_identity<<<(m * m + 255) / 256, 256, 0, s>>>(X, m, m);  // a multiple of I: V = I
    TK_LAUNCHED();
  } else {
    TK_CHECK(mp_level(d_S, m, m, noise, 0, w, X, s, tail_budget, 0.0, 0.0, &skipped));
  }
  // final products, Rayleigh quotients, verification, output
  double *tx0 = w.tx(0, 0);
  k_copy_cols<<<(m * m + 255) / 256, 256, 0, s>>>(X, m, tx0 + (size_t)m * m, m, m, m);
  TK_LAUNCHED();
  TK_CHECK(products(d_S, m, m, tx0, w.g(0), s));
  k_mp_finalize<<<1, 1024, 0, s>>>(w.g(0), tx0, tx0 + (size_t)m * m, m, m - skipped, d_lam, d_V, w.check);
  TK_LAUNCHED();
  double chk[3];
  TK_CUDA(cudaMemcpyAsync(chk, w.check, sizeof chk, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(&sw, w.sweeps, sizeof sw, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  // the paper's flop count of the eigenvector step (10/3 J^3, Sec. 5.4); bytes: S read, V written
  if (prof) prof->end(10.0 / 3.0 * (double)J * J * J, (double)J * J * 16, 1);
  const double tol_res = 16.0 * m * kU * chk[2], tol_orth = 16.0 * m * kU;
  g_mp_check[0] = chk[0];
  g_mp_check[1] = tol_res;
  g_mp_check[2] = chk[1];
  g_mp_check[3] = tol_orth;
  g_mp_check[4] = skipped;
  if (chk[0] <= tol_res && chk[1] <= tol_orth) {
    // written on the stream (a copy from the host stack would wait for it)
    k_set_info<<<1, 32, 0, s>>>(d_info, sw, 0, TUCKER_EIG_MIXED, m - skipped);
    TK_LAUNCHED();
    *verified = 1;
  }
  return TUCKER_OK;
}

}  // namespace tk
