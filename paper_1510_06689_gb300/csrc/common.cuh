// Shared declarations of the ST-HOSVD CUDA library (host driver + kernels).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <vector>

#include "../../include/tucker.h"

namespace tk {

// ---------------------------------------------------------------------------
// error reporting (host)
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
int64_t bump_launches(int64_t n = 1);

#define TK_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::tk::set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__,             \
                      cudaGetErrorString(e_));                                         \
      return e_ == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA;           \
    }                                                                                  \
  } while (0)

#define TK_LAUNCHED()                                                                  \
  do {                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess) {                                                           \
      ::tk::set_error("kernel launch failed at %s:%d: %s", __FILE__, __LINE__,         \
                      cudaGetErrorString(e_));                                         \
      return TUCKER_ECUDA;                                                             \
    }                                                                                  \
    ::tk::bump_launches();                                                             \
  } while (0)

#define TK_CHECK(st)                                                                   \
  do {                                                                                 \
    int s_ = (st);                                                                     \
    if (s_ != TUCKER_OK) return s_;                                                    \
  } while (0)

// Library bookkeeping behind tucker_result.priv: the device; for results of
// the batched pipeline the device block their core and factors live in
// (released when the last result that shares it is freed); for host results
// the pinned block holding core and factors (returned to the host block
// cache when the result is freed).
struct ResultPriv {
  int device = 0;
  std::shared_ptr<void> block;
  void *host_block = nullptr;
  size_t host_bytes = 0;
};

// The batched device pipeline (every I_n <= 128): fills out[0..count) like
// tucker_sthosvd with the identity mode order, in float64.  *handled = 0
// when the batch does not suit it (the caller then takes the per-tensor path).
int sthosvd_batched_device(const void *const *X, tucker_dtype dt, const int64_t *dims, int N, int count, double eps,
                           cudaStream_t s, tucker_result *out, int *handled);

void batched_last_tuning(int64_t *kc, int *grid, float *ms6);

// ---------------------------------------------------------------------------
// device description (cached per device)
// ---------------------------------------------------------------------------
struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int smem_optin = 0;
};
int device_info(DeviceInfo *out);

// The device's opt-in shared memory per block (cached per device).
int smem_optin_bytes();

// Lets `kernel` take as much dynamic shared memory as the device allows next
// to its static shared memory.  Kernels get this fixed limit, never a
// launch's own size: host threads running ST-HOSVDs of different shapes at
// once would otherwise lower the limit between another thread's setting and
// its launch.
template <typename K>
cudaError_t allow_max_smem(K kernel) {
  cudaFuncAttributes a;
  const cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin_bytes() - (int)a.sharedSizeBytes);
}

// ---------------------------------------------------------------------------
// phase timing: CUDA events on the launching stream, resolved after the
// caller's stream has been synchronised.
// ---------------------------------------------------------------------------
struct Prof {
  struct Rec {
    int phase;
    cudaEvent_t a, b;
    double flops, bytes;
    int launches;
  };
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<Rec> recs;
  explicit Prof(cudaStream_t stream);
  ~Prof();
  void begin(int phase);
  void end(double flops, double bytes, int launches);
  // Adds the elapsed times of all recorded phases to the process counters;
  // call only after `s` has been synchronised.
  void flush();
};

// ---------------------------------------------------------------------------
// kernel launchers (return tucker_status)
// ---------------------------------------------------------------------------

// Sum of squares of n elements into *d_out (device double).  d_partials holds
// norm2_partials() doubles.
int64_t norm2_partials();
int launch_norm2(const void *x, tucker_dtype dt, int64_t n, double *d_partials, double *d_out,
                 cudaStream_t s, Prof *prof);

// Gram of the (L, J, B) view into d_S (J x J, both triangles).  d_ws holds
// gram_workspace_doubles() doubles of split-K partials.
int64_t gram_workspace_doubles(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev);
int launch_gram(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *d_S, double *d_ws,
                const DeviceInfo &dev, cudaStream_t s, Prof *prof);

// Mode product Z(L,K,B) = sum_j A[k,j] Y(L,J,B) with A[k,j] = a[k*ak + j*aj].
int launch_ttm(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *a, int64_t ak,
               int64_t aj, int64_t K, double *z, const DeviceInfo &dev, cudaStream_t s, Prof *prof);
// Same product, not stored: sum over all entries of (x - z)^2 into *d_out,
// with x of the (L, K, B) shape.  d_partials holds ttm_diff_partials() doubles.
int64_t ttm_diff_partials(int64_t L, int64_t J, int64_t B, int64_t K, const DeviceInfo &dev);
int launch_ttm_diff(const double *y, int64_t L, int64_t J, int64_t B, const double *a, int64_t ak, int64_t aj,
                    int64_t K, const void *x, tucker_dtype xdt, double *d_partials, double *d_out,
                    const DeviceInfo &dev, cudaStream_t s, Prof *prof);

// Split-precision Gram (tcgen05, exact integer digits; J <= 128).  Takes its
// exponents from a first pass over Y on the device (no host round trip).  d_ws
// holds gram_split_workspace_doubles() doubles, including an error flag read
// back by gram_split_error().  With L > 1 and d_colexp given (L B ints), the
// first pass also writes every column's exponent (the scale the split mode
// product of the same Y needs).
int64_t gram_split_workspace_doubles(int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, tucker_dtype dt,
                                     const void *y);
// Tiled tensor map of a float64 (f64) or float32 array: rank dimensions
// (innermost first), byte strides of dimensions 1..rank-1 (multiples of 16),
// box extents; swizzle 0 (none), 64 or 128 (bytes); out-of-range elements
// read as zero.  Calls
// cuTensorMapEncodeTiled through the runtime's driver entry point; false when
// it is unavailable or refuses the map.
bool encode_tmap(CUtensorMap *map, bool f64, const void *base, int rank, const uint64_t *dims,
                 const uint64_t *strides_bytes, const uint32_t *box, int swizzle = 0);
// f8: E4M3 digits (four base-16 digits of 15-bit entries, kind::f8f6f4) instead of BF16 ones.
int launch_gram_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *d_S, double *d_ws,
                      const DeviceInfo &dev, cudaStream_t s, Prof *prof, int *d_colexp = nullptr, bool f8 = false);
// *d_out = trace of the J x J matrix S (column-major), summed in index order.
int launch_trace(const double *d_S, int64_t J, double *d_out, cudaStream_t s);
int gram_split_error(const double *d_ws, int64_t L, int64_t J, int64_t B, const DeviceInfo &dev, int *h_err,
                     cudaStream_t s);
// Split-precision mode product Z(L,R,B) = U^T Y(L,J,B) on tcgen05 (R <= J <= 128);
// U is J x R column-major float64.  *d_err becomes 1 if a bounded wait expired.
// With L > 1, d_colexp (L B ints, from launch_gram_split's exponent pass over
// the same Y) saves a pass over Y; without it the kernel computes them.
int launch_ttm_split(const void *y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *U, int64_t R,
                     double *z, int *d_err, const DeviceInfo &dev, cudaStream_t s, Prof *prof,
                     const int *d_colexp = nullptr);
// Eigensolver.  d_ws holds eig_workspace_doubles(J) doubles (0 when the
// matrix fits in shared memory).  d_info holds 4 ints: [0] Jacobi sweeps,
// [1] 0 if converged else 1, [2] the tucker_eig_path that ran, [3] the
// number of leading eigenvalues resolved one by one.
int64_t eig_workspace_doubles(int64_t J);
// tail_budget >= 0 (the rank rule's threshold) lets the mixed-precision
// solver leave clusters unresolved whose eigenvalues, with all smaller ones,
// sum to at most tail_budget: their columns span the clusters' invariant
// subspace and their values are Rayleigh quotients (every sum from such a
// cluster's first index on is exact, so the rank rule's cut is unchanged);
// the default resolves every eigenpair.
int launch_eig(const double *d_S, int64_t J, double *d_lam, double *d_V, double *d_ws, int *d_info,
               cudaStream_t s, Prof *prof, double tail_budget = -1.0);
// Mixed-precision eigensolver (float32 first stage + float64 refinement,
// J <= 128): *verified = 1 when lam, V and d_info hold a result that passed the
// device check; otherwise the caller runs the float64 Jacobi.  Synchronises s.
int launch_eig_mp(const double *d_S, int64_t J, double *d_lam, double *d_V, int *d_info, int *verified,
                  cudaStream_t s, Prof *prof, double tail_budget = -1.0);
// The calling thread's last mixed-precision check: residual and its bound,
// orthogonality and its bound, and the number of unresolved tail columns.
const double *mp_last_check();
// Largest J the mixed-precision eigensolver takes: 512 (float32 stages: the
// tridiagonal one up to 128, the wide one up to 256, a cluster Jacobi up to
// 512), or 128 with TUCKER_EIG_WIDE=0.
int mp_max_j();
// Float64 fused multiply-add throughput of the device (TFLOP/s) and the timed
// launch's duration; synchronises s.
int fp64_peak(double *tflops, double *ms, const DeviceInfo &dev, cudaStream_t s);
// Float64 Jacobi on `count` matrices at once (one CTA each, J <= 128); device
// arrays of per-matrix pointers and sizes; d_info holds 4 ints per matrix.
int launch_eig_batched(const double *const *d_S, const int *d_J, double *const *d_lam, double *const *d_V,
                       int *d_info, int count, int maxJ, cudaStream_t s, const int *d_idx = nullptr,
                       int threads = 0, const double *d_budget = nullptr);
// Float32 parallel-order Jacobi on `count` matrices (one CTA each, J <= 128):
// X_b = the unsorted float32 eigenvectors of A_b as float64 (ld J_b).
int launch_jacobi32_batched(const double *const *d_A, const int *d_J, double *const *d_X, int count, int maxJ,
                            cudaStream_t s, const int *d_idx = nullptr, int threads = 0);
// Rank rule: *d_rank = R, *d_tail = discarded sum.
int launch_rank_cut(const double *d_lam, int64_t J, double threshold, int keep_all, int64_t *d_rank,
                    double *d_tail, cudaStream_t s, Prof *prof);

}  // namespace tk
