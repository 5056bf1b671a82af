// Eigenvector and rank steps of Algorithm 1 (Sec. 2.2): all eigenpairs of the
// symmetric Gram matrix S by cyclic Jacobi in float64, then the error rule
// that picks R_n.
//
// The paper calls LAPACK's dsyevx redundantly on every process (Sec. 5.4,
// Algorithm 5) and notes the cost is negligible.  Here one CTA runs a
// parallel-order Jacobi: each step applies m/2 disjoint rotations chosen by
// the round-robin (circle) tournament over the m = J rounded-up-to-even
// indices, so that after m - 1 steps every pair has met once (one sweep).
// S is kept as its packed upper triangle; with the rotations of a step fixed,
// every 2 x 2 block {p_P, q_P} x {p_Q, q_Q} of S is updated independently as
// R_P^T B R_Q, and the rotations accumulate into V.  A dummy zero row and
// column pad odd J; rotations that involve it are never taken.  For J <= 128
// S and V live in shared memory (194 KB at J = 128); larger J use a global
// workspace.  A rotation is taken when |s_pq| > eps_mach * sqrt(|s_pp s_qq|)
// and |s_pq| exceeds a tiny absolute floor; a sweep without rotations ends
// the iteration, and the sweep cap ends it with a "not converged" flag (no
// unbounded loop on the device).
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace tk {

namespace {

constexpr int kEigThreads = 1024;
constexpr int kMaxSweeps = 60;
constexpr int kSmemMaxJ = 128;
constexpr int kMaxPairs = TUCKER_MAX_DIM / 2;

__device__ __forceinline__ int64_t pidx(int i, int j) {
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  return (int64_t)j * (j + 1) / 2 + i;
}

__device__ __forceinline__ void decode_pair_block(int e, int &P, int &Q) {
  int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((q + 1) * (q + 2) / 2 <= e) ++q;
  while (q * (q + 1) / 2 > e) --q;
  Q = q;
  P = e - q * (q + 1) / 2;
}

// The body of the one-CTA Jacobi (below), also run by the batched kernel (one
// CTA per matrix).
__device__ __forceinline__ void jacobi_body(const double *__restrict__ S_in, int J, double *__restrict__ lam,
                                            double *__restrict__ V_out, double *__restrict__ gws,
                                            int *__restrict__ info, double floor_rel = 0.0, double budget = -1.0);

__global__ void __launch_bounds__(kEigThreads) k_jacobi(const double *__restrict__ S_in, int J,
                                                         double *__restrict__ lam, double *__restrict__ V_out,
                                                         double *__restrict__ gws, int *__restrict__ info) {
  jacobi_body(S_in, J, lam, V_out, gws, info);
}

// Many matrices at once: CTA b solves matrix b (J_b <= kSmemMaxJ, S and V in
// shared memory) from the descriptor arrays; a J_b of 0 skips the CTA.
__global__ void __launch_bounds__(kEigThreads) k_jacobi_batched(const double *const *__restrict__ S, const int *__restrict__ Js,
                                                                 double *const *__restrict__ lam,
                                                                 double *const *__restrict__ V,
                                                                 int *__restrict__ info, const int *__restrict__ idx,
                                                                 const double *__restrict__ budget) {
  const int b = idx ? idx[blockIdx.x] : (int)blockIdx.x, J = Js[b];
  // absolute floor u max|s_ii|: eigenvalues to within ~J u ||S|| (backward
  // stable, as LAPACK's), without resolving tiny eigenvalues to relative
  // accuracy; with a budget, the tail the rank rule discards is left unresolved
  const double bud = budget ? budget[b] : -1.0;
  if (J > 0) jacobi_body(S[b], J, lam[b], V[b], nullptr, info + 4 * b, DBL_EPSILON, bud);
  if (threadIdx.x == 0 && !(bud >= 0.0)) info[4 * b + 2] = 0;  // no tail
}

__device__ __forceinline__ void jacobi_body(const double *__restrict__ S_in, int J, double *__restrict__ lam,
                                            double *__restrict__ V_out, double *__restrict__ gws,
                                            int *__restrict__ info, double floor_rel, double budget) {
  // budget >= 0 (S positive semidefinite): at each sweep's start the tail set
  // is the longest run of the smallest diagonal entries whose sum tau (negative
  // ones as 0) is at most budget / 2 and at most the next diagonal entry above
  // the run; rotations between two tail indices are skipped.  The tail block
  // is a principal submatrix, so its eigenvalues lie in [0, tau]: below every
  // other eigenvalue, with a sum below the threshold, so every rank cut with
  // that threshold discards the whole tail and nothing it would not discard
  // with resolved eigenvalues; the tail's trace (the discarded sum) does not
  // depend on rotations inside it.  The ranks, the retained vectors and the
  // discarded sum are those of the fully resolved problem; the tail's values
  // are Rayleigh quotients.  info[2] = the tail's size at the end.
  __shared__ unsigned char in_tail[TUCKER_MAX_DIM];
  __shared__ int tail_len;
  extern __shared__ __align__(16) double dyn[];
  __shared__ double cs[kMaxPairs], sn[kMaxPairs];
  __shared__ int pp[kMaxPairs], qq[kMaxPairs];
  __shared__ int rotated;
  __shared__ double abs_floor;
  const int m = J + (J & 1);
  const int np = m / 2;
  const int64_t packed = (int64_t)m * (m + 1) / 2;
  double *Sp = gws ? gws : dyn;
  double *V = Sp + packed;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i <= j) Sp[pidx(i, j)] = (j < J) ? S_in[i + (int64_t)J * j] : 0.0;
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < J; ++i) mx = fmax(mx, fabs(S_in[i + (int64_t)J * i]));
    abs_floor = mx * (floor_rel > 0.0 ? floor_rel : DBL_EPSILON * DBL_EPSILON) + DBL_MIN;
  }
  __syncthreads();

  int sweep = 0;
  bool converged = false;
  const int nblk = np * (np + 1) / 2;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) {
      rotated = 0;
      tail_len = 0;
    }
    __syncthreads();
    if (budget >= 0.0) {
      // over the J entries (not the zero padding row): ascending order (ties:
      // the higher index first); entry i closes the run of the k_i smallest
      // entries, with sum acc and the next entry above nxt
      for (int i = tid; i < J; i += nt) {
        const double di = Sp[pidx(i, i)];
        double acc = 0.0, nxt = INFINITY;
        int k = 0;
        for (int j = 0; j < J; ++j) {
          const double dj = Sp[pidx(j, j)];
          if (dj < di || (dj == di && j >= i)) {
            acc += fmax(dj, 0.0);
            ++k;
          } else {
            nxt = fmin(nxt, dj);
          }
        }
        if (k < J && acc <= 0.5 * budget && acc <= nxt) atomicMax(&tail_len, k);  // one index stays resolved
      }
      __syncthreads();
      for (int i = tid; i < m; i += nt) {  // the run of the tail_len smallest entries (and the padding row)
        const double di = Sp[pidx(i, i)];
        int k = 0;
        for (int j = 0; j < J; ++j) {
          const double dj = Sp[pidx(j, j)];
          k += dj < di || (dj == di && j >= i);
        }
        in_tail[i] = i >= J || k <= tail_len;
      }
      __syncthreads();
    }
    for (int step = 0; step < m - 1; ++step) {
      for (int t = tid; t < np; t += nt) {
        int p = (t == 0) ? 0 : ((t - 1 + step) % (m - 1)) + 1;
        int q = ((m - 2 - t + step) % (m - 1)) + 1;  // position m - 1 - t
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        double c = 1.0, s = 0.0;
        const double b = (budget >= 0.0 && in_tail[p] && in_tail[q]) ? 0.0 : Sp[pidx(p, q)];
        if (b != 0.0) {
          const double a = Sp[pidx(p, p)], d = Sp[pidx(q, q)];
          const double ab = fabs(b);
          if (ab > DBL_EPSILON * sqrt(fabs(a)) * sqrt(fabs(d)) && ab > abs_floor) {
            const double tau = (d - a) / (2.0 * b);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            rotated = 1;
          }
        }
        cs[t] = c;
        sn[t] = s;
        pp[t] = p;
        qq[t] = q;
      }
      __syncthreads();
      for (int e = tid; e < nblk; e += nt) {
        int P, Q;
        decode_pair_block(e, P, Q);
        const double s1 = sn[P], s2 = sn[Q];
        const int p1 = pp[P], q1 = qq[P];
        if (P == Q) {
          if (s1 != 0.0) {
            const double t1 = s1 / cs[P];
            const int64_t ipq = pidx(p1, q1), ipp = pidx(p1, p1), iqq = pidx(q1, q1);
            const double b = Sp[ipq];
            Sp[ipp] = Sp[ipp] - t1 * b;
            Sp[iqq] = Sp[iqq] + t1 * b;
            Sp[ipq] = 0.0;
          }
          continue;
        }
        if (s1 == 0.0 && s2 == 0.0) continue;
        const double c1 = cs[P], c2 = cs[Q];
        const int p2 = pp[Q], q2 = qq[Q];
        const int64_t i11 = pidx(p1, p2), i12 = pidx(p1, q2), i21 = pidx(q1, p2), i22 = pidx(q1, q2);
        const double x11 = Sp[i11], x12 = Sp[i12], x21 = Sp[i21], x22 = Sp[i22];
        // R_P^T B with R = [[c, s], [-s, c]]
        const double y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
        const double y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
        // (.) R_Q
        Sp[i11] = y11 * c2 - y12 * s2;
        Sp[i12] = y11 * s2 + y12 * c2;
        Sp[i21] = y21 * c2 - y22 * s2;
        Sp[i22] = y21 * s2 + y22 * c2;
      }
      for (int e = tid; e < np * m; e += nt) {
        const int t = e / m, i = e - t * m;
        const double s = sn[t];
        if (s == 0.0) continue;
        const double c = cs[t];
        double *vp = V + (int64_t)pp[t] * m + i;
        double *vq = V + (int64_t)qq[t] * m + i;
        const double a = *vp, b = *vq;
        *vp = c * a - s * b;
        *vq = s * a + c * b;
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) {
      converged = true;
      break;
    }
  }

  // Sort descending (ties: lower index first), sign-normalise, write out.
  for (int i = tid; i < J; i += nt) {
    const double di = Sp[pidx(i, i)];
    int rank = 0;
    for (int j = 0; j < J; ++j) {
      const double dj = Sp[pidx(j, j)];
      rank += (dj > di) || (dj == di && j < i);
    }
    lam[rank] = di;
    const double *col = V + (int64_t)i * m;
    double best = -1.0;
    int br = 0;
    for (int r = 0; r < J; ++r) {
      const double v = fabs(col[r]);
      if (v > best) {
        best = v;
        br = r;
      }
    }
    const double sg = col[br] < 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < J; ++r) V_out[r + (int64_t)J * rank] = sg * col[r];
  }
  if (tid == 0) {
    info[0] = converged ? sweep + 1 : kMaxSweeps;
    info[1] = converged ? 0 : 1;
    if (budget >= 0.0) info[2] = tail_len;
  }
}

// ---------------------------------------------------------------------------
// Cluster Jacobi: the same parallel-order sweeps, spread over the CTAs of one
// thread-block cluster (up to 16 SMs) so that the float64 work of a step runs
// on all of them.  S (packed upper triangle), V and the rotation parameters
// live in a global workspace that stays in L2; loads bypass L1 (__ldcg) so a
// CTA never reads a line another CTA rewrote.  Each step is two phases
// separated by hardware cluster barriers: (A) every pair's rotation from the
// current diagonal entries, (B) the 2 x 2 block updates of S and the column
// updates of V.  Rotation flags are kept per sweep, so no flag is reset while
// another CTA may still read it.
// ---------------------------------------------------------------------------
constexpr int kClusterThreads = 1024;

__global__ void __launch_bounds__(kClusterThreads) k_jacobi_cluster(const double *__restrict__ S_in, int J,
                                                                      double *__restrict__ lam,
                                                                      double *__restrict__ V_out,
                                                                      double *__restrict__ ws,
                                                                      int *__restrict__ info) {
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ double cs[kMaxPairs], sn[kMaxPairs];
  __shared__ int pp[kMaxPairs], qq[kMaxPairs];
  const int m = J + (J & 1);
  const int np = m / 2;
  const int64_t packed = (int64_t)m * (m + 1) / 2;
  double *Sp = ws;
  double *V = Sp + packed;
  double *par = V + (int64_t)m * m;                       // np x {c, s}
  int *flags = reinterpret_cast<int *>(par + 2 * np);     // one per sweep
  const int rank = (int)cluster.block_rank();
  const int nct = (int)cluster.num_blocks();
  const int gtid = rank * blockDim.x + threadIdx.x;
  const int gthreads = nct * blockDim.x;

  for (int64_t e = gtid; e < (int64_t)m * m; e += gthreads) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i <= j) Sp[pidx(i, j)] = (j < J) ? S_in[i + (int64_t)J * j] : 0.0;
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  for (int k = gtid; k < kMaxSweeps; k += gthreads) flags[k] = 0;
  double mx = 0.0;
  for (int i = 0; i < J; ++i) mx = fmax(mx, fabs(S_in[i + (int64_t)J * i]));
  const double abs_floor = mx * (DBL_EPSILON * DBL_EPSILON) + DBL_MIN;
  cluster.sync();

  const int nblk = np * (np + 1) / 2;
  const int64_t items = (int64_t)nblk + (int64_t)np * m;
  int sweep = 0;
  bool converged = false;
  for (; sweep < kMaxSweeps; ++sweep) {
    for (int step = 0; step < m - 1; ++step) {
      // (A) rotations of this step
      for (int t = gtid; t < np; t += gthreads) {
        int p = (t == 0) ? 0 : ((t - 1 + step) % (m - 1)) + 1;
        int q = ((m - 2 - t + step) % (m - 1)) + 1;
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        double c = 1.0, s = 0.0;
        const double b = __ldcg(Sp + pidx(p, q));
        if (b != 0.0) {
          const double a = __ldcg(Sp + pidx(p, p)), d = __ldcg(Sp + pidx(q, q));
          const double ab = fabs(b);
          if (ab > DBL_EPSILON * sqrt(fabs(a)) * sqrt(fabs(d)) && ab > abs_floor) {
            const double tau = (d - a) / (2.0 * b);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            flags[sweep] = 1;
          }
        }
        __stcg(par + 2 * t, c);
        __stcg(par + 2 * t + 1, s);
      }
      cluster.sync();
      for (int t = threadIdx.x; t < np; t += blockDim.x) {
        int p = (t == 0) ? 0 : ((t - 1 + step) % (m - 1)) + 1;
        int q = ((m - 2 - t + step) % (m - 1)) + 1;
        pp[t] = min(p, q);
        qq[t] = max(p, q);
        cs[t] = __ldcg(par + 2 * t);
        sn[t] = __ldcg(par + 2 * t + 1);
      }
      __syncthreads();
      // (B) block updates of S, then column updates of V; every CTA takes an
      // equal contiguous share of each kind
      const int64_t b0 = (int64_t)nblk * rank / nct, b1 = (int64_t)nblk * (rank + 1) / nct;
      const int64_t v0 = (int64_t)np * m * rank / nct, v1 = (int64_t)np * m * (rank + 1) / nct;
      const int64_t mine = (b1 - b0) + (v1 - v0);
      for (int64_t k = threadIdx.x; k < mine; k += blockDim.x) {
        const int64_t e = k < b1 - b0 ? b0 + k : nblk + v0 + (k - (b1 - b0));
        if (e < nblk) {
          int P, Q;
          decode_pair_block((int)e, P, Q);
          const double s1 = sn[P], s2 = sn[Q];
          const int p1 = pp[P], q1 = qq[P];
          if (P == Q) {
            if (s1 != 0.0) {
              const double t1 = s1 / cs[P];
              const int64_t ipq = pidx(p1, q1), ipp = pidx(p1, p1), iqq = pidx(q1, q1);
              const double b = __ldcg(Sp + ipq);
              __stcg(Sp + ipp, __ldcg(Sp + ipp) - t1 * b);
              __stcg(Sp + iqq, __ldcg(Sp + iqq) + t1 * b);
              __stcg(Sp + ipq, 0.0);
            }
            continue;
          }
          if (s1 == 0.0 && s2 == 0.0) continue;
          const double c1 = cs[P], c2 = cs[Q];
          const int p2 = pp[Q], q2 = qq[Q];
          const int64_t i11 = pidx(p1, p2), i12 = pidx(p1, q2), i21 = pidx(q1, p2), i22 = pidx(q1, q2);
          const double x11 = __ldcg(Sp + i11), x12 = __ldcg(Sp + i12);
          const double x21 = __ldcg(Sp + i21), x22 = __ldcg(Sp + i22);
          const double y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
          const double y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
          __stcg(Sp + i11, y11 * c2 - y12 * s2);
          __stcg(Sp + i12, y11 * s2 + y12 * c2);
          __stcg(Sp + i21, y21 * c2 - y22 * s2);
          __stcg(Sp + i22, y21 * s2 + y22 * c2);
        } else {
          const int64_t r = e - nblk;
          const int t = (int)(r / m), i = (int)(r - (int64_t)t * m);
          const double s = sn[t];
          if (s == 0.0) continue;
          const double c = cs[t];
          double *vp = V + (int64_t)pp[t] * m + i;
          double *vq = V + (int64_t)qq[t] * m + i;
          const double a = __ldcg(vp), b = __ldcg(vq);
          __stcg(vp, c * a - s * b);
          __stcg(vq, s * a + c * b);
        }
      }
      cluster.sync();
    }
    if (__ldcg(flags + sweep) == 0) {
      converged = true;
      break;
    }
  }

  for (int i = gtid; i < J; i += gthreads) {
    const double di = __ldcg(Sp + pidx(i, i));
    int rk = 0;
    for (int j = 0; j < J; ++j) {
      const double dj = __ldcg(Sp + pidx(j, j));
      rk += (dj > di) || (dj == di && j < i);
    }
    lam[rk] = di;
    const double *col = V + (int64_t)i * m;
    double best = -1.0;
    int br = 0;
    for (int r = 0; r < J; ++r) {
      const double v = fabs(__ldcg(col + r));
      if (v > best) {
        best = v;
        br = r;
      }
    }
    const double sg = __ldcg(col + br) < 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < J; ++r) V_out[r + (int64_t)J * rk] = sg * __ldcg(col + r);
  }
  if (gtid == 0) {
    info[0] = converged ? sweep + 1 : kMaxSweeps;
    info[1] = converged ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// Distributed-shared-memory Jacobi (J up to 512): the same rotations as the
// kernels above, with S (packed upper triangle) and V spread over the shared
// memory of a 16-CTA cluster (element e lives in CTA e mod 16) and ONE cluster
// barrier per step.  The barrier count halves because every step also
// computes the next step's rotations: each next-step pair {a, b} lies in
// exactly one 2 x 2 block of the current step (consecutive rounds of the
// tournament never repeat a pair), so the thread that rewrites that block
// knows s'_ab, and the next diagonal follows in closed form from the current
// one (d_p - t b, d_q + t b).  It broadcasts (c, s) and the new diagonal
// entries into every CTA's shared memory; after the barrier each CTA holds
// the whole step locally.  Distributed shared memory keeps each step's
// remote accesses at shared-memory-network latency instead of L2 round trips.
// ---------------------------------------------------------------------------
constexpr int kDsmThreads = 1024;
constexpr int kDsmMaxJ = 512;

// Element e of the distributed S / V array: in distributed shared memory
// (CTA e mod 16, slot e / 16) or, for kL2, at ws[e] in global memory with all
// loads bypassing L1 (other CTAs rewrite those lines every step).
template <bool kL2>
struct MatView {
  cg::cluster_group cl;
  double *local;
  double *ws;
  int lg, mask;
  __device__ double *at(int64_t e) const {
    if (kL2) return ws + e;
    return cl.map_shared_rank(local + (e >> lg), (int)(e & mask));
  }
  __device__ double ld(int64_t e) const {
    if (kL2) return __ldcg(ws + e);
    return *at(e);
  }
  __device__ void st(int64_t e, double v) const {
    if (kL2) __stcg(ws + e, v);
    else *at(e) = v;
  }
};

__device__ __forceinline__ int tour_player(int pos, int step, int m) {
  return pos == 0 ? 0 : ((pos - 1 + step) % (m - 1)) + 1;
}
__device__ __forceinline__ int tour_pos(int player, int step, int m) {
  return player == 0 ? 0 : ((player - 1 - step) % (m - 1) + (m - 1)) % (m - 1) + 1;
}

// Rotation annihilating b of [[a, b], [b, d]] (same rule as the other kernels).
__device__ __forceinline__ bool jacobi_rotation(double a, double b, double d, double abs_floor, double &c,
                                                double &s, double &na, double &nd) {
  c = 1.0;
  s = 0.0;
  na = a;
  nd = d;
  if (b == 0.0) return false;
  const double ab = fabs(b);
  if (!(ab > DBL_EPSILON * sqrt(fabs(a)) * sqrt(fabs(d)) && ab > abs_floor)) return false;
  const double tau = (d - a) / (2.0 * b);
  const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + tt * tt);
  s = tt * c;
  na = a - tt * b;
  nd = d + tt * b;
  return true;
}

template <bool kL2>
__global__ void __launch_bounds__(kDsmThreads) k_jacobi_dsm(const double *__restrict__ S_in, int J,
                                                           double *__restrict__ lam, double *__restrict__ V_out,
                                                           double *__restrict__ ws, int *__restrict__ info) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double dyn[];
  // the step's rotations and new diagonal, gathered into every CTA
  __shared__ double cpar[kDsmMaxJ / 2], spar[kDsmMaxJ / 2];
  __shared__ double dnew[kDsmMaxJ];
  // home slots (this CTA's share, two step parities): pair t lives in CTA
  // t mod 16 at t / 16, diagonal entry i in CTA i mod 16 at i / 16
  __shared__ double hc[2][kDsmMaxJ / 32], hs[2][kDsmMaxJ / 32], hd[2][kDsmMaxJ / 16];
  __shared__ int flags[kMaxSweeps + 2];
  // this step's pairs and, for every index, its next-step partner and pair
  __shared__ short spp[kDsmMaxJ / 2], sqq[kDsmMaxJ / 2], npart[kDsmMaxJ], npair[kDsmMaxJ];
  const int nct = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int lg = __ffs(nct) - 1;
  const int mask = nct - 1;
  MatView<kL2> D{cl, dyn, ws, lg, mask};
  const int m = J + (J & 1);
  const int np = m / 2;
  const int64_t packed = (int64_t)m * (m + 1) / 2;
  const int64_t total = packed + (int64_t)m * m;
  const int tid = threadIdx.x;
  const int gtid = rank * blockDim.x + tid, gthreads = nct * blockDim.x;

  for (int k = tid; k < kMaxSweeps + 2; k += blockDim.x) flags[k] = 0;
  for (int64_t e = gtid; e < total; e += gthreads) {
    double v;
    if (e < packed) {
      int j = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
      while ((int64_t)(j + 1) * (j + 2) / 2 <= e) ++j;
      while ((int64_t)j * (j + 1) / 2 > e) --j;
      const int i = (int)(e - (int64_t)j * (j + 1) / 2);
      v = (j < J) ? S_in[i + (int64_t)J * j] : 0.0;
    } else {
      const int64_t f = e - packed;
      v = (f % m == f / m) ? 1.0 : 0.0;
    }
    D.st(e, v);
  }
  double mx = 0.0;
  for (int i = 0; i < J; ++i) mx = fmax(mx, fabs(S_in[i + (int64_t)J * i]));
  const double abs_floor = mx * (DBL_EPSILON * DBL_EPSILON) + DBL_MIN;
  cl.sync();

  // one remote store per value, to its home CTA; the sweep flag goes to CTA 0
  auto publish = [&](int buf, int t, int p, int q, double c, double s, double na, double nd) {
    *cl.map_shared_rank(&hc[buf][t >> lg], t & mask) = c;
    *cl.map_shared_rank(&hs[buf][t >> lg], t & mask) = s;
    *cl.map_shared_rank(&hd[buf][p >> lg], p & mask) = na;
    *cl.map_shared_rank(&hd[buf][q >> lg], q & mask) = nd;
  };
  for (int t = gtid; t < np; t += gthreads) {
    int p = tour_player(t, 0, m), q = tour_player(m - 1 - t, 0, m);
    if (p > q) {
      const int x = p;
      p = q;
      q = x;
    }
    double c, s, na, nd;
    const bool rot = jacobi_rotation(D.ld(pidx(p, p)), D.ld(pidx(p, q)), D.ld(pidx(q, q)), abs_floor, c, s, na, nd);
    publish(0, t, p, q, c, s, na, nd);
    if (rot) *cl.map_shared_rank(&flags[0], 0) = 1;
  }
  cl.sync();

  const int nblk = np * (np + 1) / 2;
  const int64_t items = (int64_t)nblk + (int64_t)np * m;
  int sweep = 0;
  bool converged = false;
  int64_t gstep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    for (int step = 0; step < m - 1; ++step, ++gstep) {
      const int cur = (int)(gstep & 1), nxt = cur ^ 1;
      const int nstep = (step + 1) % (m - 1);
      const int nsweep = (step + 1 == m - 1) ? sweep + 1 : sweep;
      // gather this step's rotations and diagonal; tabulate the pairings once
      for (int k = tid; k < np + m; k += blockDim.x) {
        if (k < np) {
          cpar[k] = *cl.map_shared_rank(&hc[cur][k >> lg], k & mask);
          spar[k] = *cl.map_shared_rank(&hs[cur][k >> lg], k & mask);
          const int p = tour_player(k, step, m), q = tour_player(m - 1 - k, step, m);
          spp[k] = (short)min(p, q);
          sqq[k] = (short)max(p, q);
        } else {
          const int i = k - np;
          dnew[i] = *cl.map_shared_rank(&hd[cur][i >> lg], i & mask);
          const int pa = tour_pos(i, nstep, m);
          npart[i] = (short)tour_player(m - 1 - pa, nstep, m);
          npair[i] = (short)min(pa, m - 1 - pa);
        }
      }
      __syncthreads();
      // every CTA takes an equal contiguous share of the 2 x 2 blocks and of the
      // V rows (a global stride would put all block work on the first CTAs)
      const int64_t b0 = (int64_t)nblk * rank / nct, b1 = (int64_t)nblk * (rank + 1) / nct;
      const int64_t v0 = (int64_t)np * m * rank / nct, v1 = (int64_t)np * m * (rank + 1) / nct;
      const int64_t mine = (b1 - b0) + (v1 - v0);
      for (int64_t k = tid; k < mine; k += blockDim.x) {
        const int64_t e = k < b1 - b0 ? b0 + k : nblk + v0 + (k - (b1 - b0));
        if (e < nblk) {
          int P, Q;
          decode_pair_block((int)e, P, Q);
          const int p1 = spp[P], q1 = sqq[P];
          if (P == Q) {
            if (spar[P] != 0.0) {
              D.st(pidx(p1, p1), dnew[p1]);
              D.st(pidx(q1, q1), dnew[q1]);
              D.st(pidx(p1, q1), 0.0);
            }
            continue;
          }
          const int p2 = spp[Q], q2 = sqq[Q];
          const double c1 = cpar[P], s1 = spar[P], c2 = cpar[Q], s2 = spar[Q];
          const int64_t i11 = pidx(p1, p2), i12 = pidx(p1, q2), i21 = pidx(q1, p2), i22 = pidx(q1, q2);
          double x11 = D.ld(i11), x12 = D.ld(i12), x21 = D.ld(i21), x22 = D.ld(i22);
          if (s1 != 0.0 || s2 != 0.0) {
            const double y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
            const double y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
            x11 = y11 * c2 - y12 * s2;
            x12 = y11 * s2 + y12 * c2;
            x21 = y21 * c2 - y22 * s2;
            x22 = y21 * s2 + y22 * c2;
            D.st(i11, x11);
            D.st(i12, x12);
            D.st(i21, x21);
            D.st(i22, x22);
          }
          // any of the four elements a next-step pair?  Then its rotation is made here.
          const int rows[2] = {p1, q1}, cols[2] = {p2, q2};
          const double vals[2][2] = {{x11, x12}, {x21, x22}};
#pragma unroll
          for (int ri = 0; ri < 2; ++ri)
#pragma unroll
            for (int ci = 0; ci < 2; ++ci) {
              const int a = rows[ri], b = cols[ci];
              if (npart[a] != b) continue;
              const int t = npair[a];
              const int lo = min(a, b), hi = max(a, b);
              double c, s, na, nd;
              const bool rot = jacobi_rotation(dnew[lo], vals[ri][ci], dnew[hi], abs_floor, c, s, na, nd);
              publish(nxt, t, lo, hi, c, s, na, nd);
              if (rot) *cl.map_shared_rank(&flags[nsweep], 0) = 1;
            }
        } else {
          const int64_t r = e - nblk;
          const int t = (int)(r / m), i = (int)(r - (int64_t)t * m);
          const double s = spar[t];
          if (s == 0.0) continue;
          const double c = cpar[t];
          const int64_t ep = packed + (int64_t)spp[t] * m + i, eq = packed + (int64_t)sqq[t] * m + i;
          const double a = D.ld(ep), b = D.ld(eq);
          D.st(ep, c * a - s * b);
          D.st(eq, s * a + c * b);
        }
      }
      cl.sync();
    }
    if (*cl.map_shared_rank(&flags[sweep], 0) == 0) {
      converged = true;
      break;
    }
  }

  // eigenvalues: the diagonal after the last applied step (dnew of that step)
  for (int i = gtid; i < J; i += gthreads) {
    const double di = dnew[i];
    int rk = 0;
    for (int j = 0; j < J; ++j) {
      const double dj = dnew[j];
      rk += (dj > di) || (dj == di && j < i);
    }
    lam[rk] = di;
    double best = -1.0, sgv = 0.0;
    for (int r = 0; r < J; ++r) {
      const double v = D.ld(packed + (int64_t)i * m + r);
      if (fabs(v) > best) {
        best = fabs(v);
        sgv = v;
      }
    }
    const double sg = sgv < 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < J; ++r) V_out[r + (int64_t)J * rk] = sg * D.ld(packed + (int64_t)i * m + r);
  }
  if (gtid == 0) {
    info[0] = converged ? sweep + 1 : kMaxSweeps;
    info[1] = converged ? 0 : 1;
  }
  cl.sync();  // no CTA may exit while others still read its shared memory
}

// Rank rule of Algorithm 1: tails[r] = sum_{k >= r} max(lam[k], 0) accumulated
// from the smallest eigenvalue upward; R = smallest r in [1, J] with
// tails[r] <= threshold.
__global__ void k_rank_cut(const double *__restrict__ lam, int J, double threshold, int keep_all,
                           int64_t *__restrict__ R, double *__restrict__ tail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (keep_all) {
    R[0] = J;
    tail[0] = 0.0;
    return;
  }
  double acc = 0.0;
  int best = J;
  double best_tail = 0.0;
  for (int r = J - 1; r >= 1; --r) {
    acc += fmax(lam[r], 0.0);
    if (acc <= threshold) {
      best = r;
      best_tail = acc;
    } else {
      break;
    }
  }
  R[0] = best;
  tail[0] = best_tail;
}

}  // namespace

// Float64 Jacobi on many matrices (J <= 128 each), one CTA per matrix; the
// arrays are device arrays indexed by matrix (info: 4 ints per matrix: sweeps,
// not converged, unresolved tail size (with a budget), spare); with d_idx, CTA
// b solves matrix d_idx[b] (count of them), each CTA `threads` wide with
// shared memory for J <= maxJ; with d_budget (per matrix, < 0: none) the
// rank rule's tail within that budget is left unresolved.
int launch_eig_batched(const double *const *d_S, const int *d_J, double *const *d_lam, double *const *d_V,
                       int *d_info, int count, int maxJ, cudaStream_t s, const int *d_idx, int threads,
                       const double *d_budget) {
  if (maxJ > kSmemMaxJ) {
    set_error("batched eigensolver takes J <= %d (got %d)", kSmemMaxJ, maxJ);
    return TUCKER_EUNSUPPORTED;
  }
  const int m = maxJ + (maxJ & 1);
  const size_t smem = (size_t)(m * (m + 1) / 2 + m * m) * sizeof(double);
  TK_CUDA(allow_max_smem(k_jacobi_batched));
  if (count > 0) {
    k_jacobi_batched<<<count, threads > 0 ? threads : kEigThreads, smem, s>>>(d_S, d_J, d_lam, d_V, d_info, d_idx,
                                                                              d_budget);
    TK_LAUNCHED();
  }
  return TUCKER_OK;
}

// J up to this size runs in one CTA with S and V in shared memory; larger J
// run on a cluster.
constexpr int kOneCtaMaxJ = 32;

int64_t eig_workspace_doubles(int64_t J) {
  const int64_t m = J + (J & 1);
  if (J <= kOneCtaMaxJ) return 0;
  return m * (m + 1) / 2 + m * m + m + kMaxSweeps;  // S, V, rotations, flags
}

// Largest cluster (16 with the non-portable opt-in, else 8) the device can
// co-schedule for k_jacobi_cluster.
static int cluster_size_for_eig() {
  static int cached = 0;
  if (cached) return cached;
  int best = 8;
  if (cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClusterThreads);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 16;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_jacobi_cluster, &cfg) == cudaSuccess && n >= 1) best = 16;
  }
  cudaGetLastError();
  cached = best;
  return best;
}

// True if a 16-CTA cluster of k_jacobi_dsm with `dsmem` bytes of dynamic
// shared memory per CTA can be co-scheduled on this device.
template <bool kL2>
static bool dsm_cluster_ok(size_t dsmem) {
  if (cudaFuncSetAttribute(k_jacobi_dsm<kL2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      allow_max_smem(k_jacobi_dsm<kL2>) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(kDsmThreads);
  cfg.dynamicSmemBytes = dsmem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 16;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&n, k_jacobi_dsm<kL2>, &cfg) == cudaSuccess && n >= 1;
  cudaGetLastError();
  return ok;
}

namespace {
__global__ void k_eig_tag(int *info, int path, int resolved) {
  if (threadIdx.x == 0) {
    info[2] = path;
    info[3] = resolved;
  }
}
}  // namespace

int launch_eig(const double *d_S, int64_t J, double *d_lam, double *d_V, double *d_ws, int *d_info,
               cudaStream_t s, Prof *prof, double tail_budget) {
  const int64_t m = J + (J & 1);
  // "mp" (default: mixed precision, J <= 256 (J <= 128 with TUCKER_EIG_WIDE=0),
  // float64 Jacobi if unverified) |
  // "jacobi" (float64 Jacobi only) | "dsm" | "l2m" | "l2" (cluster variants)
  const char *ev = getenv("TUCKER_EIG_KERNEL");
  const bool use_dsm = ev && !strcmp(ev, "dsm");
  const bool use_l2 = ev && !strcmp(ev, "l2");
  const bool jacobi_only = ev && (use_dsm || use_l2 || !strcmp(ev, "jacobi") || !strcmp(ev, "l2m"));
  // d_info[2] records which solver ran (tucker_eig_path), d_info[3] how many
  // leading eigenvalues were resolved one by one (the mixed-precision path
  // writes both itself)
  const int path_jacobi[1] = {TUCKER_EIG_JACOBI}, path_fallback[1] = {TUCKER_EIG_JACOBI_FALLBACK};
  const int *path = path_jacobi;
  if (!jacobi_only && J <= mp_max_j()) {
    int verified = 0;
    TK_CHECK(launch_eig_mp(d_S, J, d_lam, d_V, d_info, &verified, s, prof, tail_budget));
    if (verified) return TUCKER_OK;
    const char *strict = getenv("TUCKER_EIG_MP_STRICT");  // tests: report instead of falling back
    if (strict && strict[0] == '1') {
      const double *c = mp_last_check();
      set_error("mixed-precision eigensolver failed its check (J = %lld): residual %.3g (bound %.3g), "
                "orthogonality %.3g (bound %.3g), %d tail columns unresolved",
                (long long)J, c[0], c[1], c[2], c[3], (int)c[4]);
      return TUCKER_ENOCONV;
    }
    path = path_fallback;
  }
  k_eig_tag<<<1, 32, 0, s>>>(d_info, path[0], (int)J);
  TK_LAUNCHED();
  if (J > kOneCtaMaxJ && J <= kDsmMaxJ && !use_l2 && (use_dsm || d_ws)) {
    const size_t dsmem = use_dsm ? (size_t)((m * (m + 1) / 2 + m * m + 15) / 16) * sizeof(double) : 0;
    if (use_dsm ? dsm_cluster_ok<false>(dsmem) : dsm_cluster_ok<true>(0)) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kDsmThreads);
      cfg.dynamicSmemBytes = dsmem;
      cfg.stream = s;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = 16;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      if (prof) prof->begin(TUCKER_PHASE_EIG);
      if (use_dsm)
        TK_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi_dsm<false>, d_S, (int)J, d_lam, d_V, (double *)nullptr, d_info));
      else
        TK_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi_dsm<true>, d_S, (int)J, d_lam, d_V, d_ws, d_info));
      TK_LAUNCHED();
      if (prof) prof->end(10.0 / 3.0 * (double)J * J * J, (double)J * J * 16, 1);  // flops: the paper's count, Sec. 5.4
      return TUCKER_OK;
    }
  }
  if (J > kOneCtaMaxJ) {
    if (!d_ws) {
      set_error("eigensolver workspace missing for J = %lld", (long long)J);
      return TUCKER_EINVAL;
    }
    const int csize = cluster_size_for_eig();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = csize;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (prof) prof->begin(TUCKER_PHASE_EIG);
    TK_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi_cluster, d_S, (int)J, d_lam, d_V, d_ws, d_info));
    TK_LAUNCHED();
    if (prof) prof->end(10.0 / 3.0 * (double)J * J * J, (double)J * J * 16, 1);  // flops: the paper's count, Sec. 5.4
    return TUCKER_OK;
  }
  size_t smem = 0;
  double *ws = nullptr;
  if (J <= kSmemMaxJ) {
    smem = (size_t)(m * (m + 1) / 2 + m * m) * sizeof(double);
    TK_CUDA(allow_max_smem(k_jacobi));
  } else {
    ws = d_ws;
    if (!ws) {
      set_error("eigensolver workspace missing for J = %lld", (long long)J);
      return TUCKER_EINVAL;
    }
  }
  if (prof) prof->begin(TUCKER_PHASE_EIG);
  k_jacobi<<<1, kEigThreads, smem, s>>>(d_S, (int)J, d_lam, d_V, ws, d_info);
  TK_LAUNCHED();
  if (prof) prof->end(10.0 / 3.0 * (double)J * J * J, (double)J * J * 16, 1);  // flops: the paper's count, Sec. 5.4
  return TUCKER_OK;
}

int launch_rank_cut(const double *d_lam, int64_t J, double threshold, int keep_all, int64_t *d_rank,
                    double *d_tail, cudaStream_t s, Prof *prof) {
  if (prof) prof->begin(TUCKER_PHASE_RANK);
  k_rank_cut<<<1, 32, 0, s>>>(d_lam, (int)J, threshold, keep_all, d_rank, d_tail);
  TK_LAUNCHED();
  if (prof) prof->end((double)J, (double)J * 8, 1);
  return TUCKER_OK;
}

}  // namespace tk
