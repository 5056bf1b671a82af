// Host driver and C ABI of the ST-HOSVD library (declarations in include/tucker.h).
//
// tucker_sthosvd sequences Algorithm 1 (Sec. 2.2) on one GPU:
//   ||X||^2 (sum-of-squares kernel; the split-precision path takes the trace
//   of its first Gram instead) -> threshold eps^2 ||X||^2 / N,
//   then for each mode n of the order:
//     Gram of the (L, J_n, B) view   (float64 split-K kernel, or the
//                                     tensor-core digit Gram)
//     eigensolve                     (mixed-precision solver for J <= 128,
//                                     float64 Jacobi otherwise or as fallback)
//     rank rule                      (one thread)
//     copy R_n, tail and eigenvalues to pinned host memory; synchronise
//     factor U_n = first R_n eigenvector columns
//     TTM  Y <- Y x_n U_n^T          (into a fresh stream-ordered buffer)
// The rank, which fixes the shape of the next launch, is the main host<->device
// round trip per mode (the mixed-precision eigensolver adds a few small ones).
// All device memory is stream-ordered (cudaMallocAsync on the caller's stream).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace tk {

// ---------------------------------------------------------------------------
// errors, counters, device info
// ---------------------------------------------------------------------------
static thread_local char g_err[1024];
static std::atomic<int64_t> g_launches{0};

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

int64_t bump_launches(int64_t n) { return g_launches.fetch_add(n) + n; }

int smem_optin_bytes() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cache[dev].load();
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) v = 48 * 1024;
    cache[dev].store(v);
  }
  return v;
}

int device_info(DeviceInfo *out) {
  static std::mutex mu;
  static DeviceInfo cache[64];
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return TUCKER_EINVAL;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev].device != dev) {
    DeviceInfo d;
    d.device = dev;
    TK_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    TK_CUDA(cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // Keep freed stream-ordered memory in the pool across calls (up to 64 GB)
    // so repeated compressions do not return it to the driver each time.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = 64ull << 30;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cache[dev] = d;
  }
  *out = cache[dev];
  return TUCKER_OK;
}

// ---------------------------------------------------------------------------
// profiling
// ---------------------------------------------------------------------------
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};
static tucker_profile g_prof;

// Timing events are reused across calls (per device): creating and
// destroying two per phase would put host work between the launches of a
// profiled run.  Never destroyed, like the host block cache.
struct EventPool {
  std::mutex mu;
  std::vector<cudaEvent_t> free[64];
};
static EventPool &event_pool() {
  static EventPool *p = new EventPool;
  return *p;
}
static bool event_get(cudaEvent_t *e) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  EventPool &p = event_pool();
  {
    std::lock_guard<std::mutex> lock(p.mu);
    if (!p.free[dev].empty()) {
      *e = p.free[dev].back();
      p.free[dev].pop_back();
      return true;
    }
  }
  return cudaEventCreate(e) == cudaSuccess;
}
static void event_put(cudaEvent_t e) {
  int dev = 0;
  if (!e) return;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaEventDestroy(e);
    return;
  }
  EventPool &p = event_pool();
  std::lock_guard<std::mutex> lock(p.mu);
  p.free[dev].push_back(e);
}

Prof::Prof(cudaStream_t stream) : on(g_prof_on.load()), s(stream) {}

Prof::~Prof() {
  for (auto &r : recs) {
    event_put(r.a);
    event_put(r.b);
  }
}

void Prof::begin(int phase) {
  if (!on) return;
  Rec r{phase, nullptr, nullptr, 0, 0, 0};
  if (!event_get(&r.a) || !event_get(&r.b)) {
    event_put(r.a);
    on = false;
    return;
  }
  cudaEventRecord(r.a, s);
  recs.push_back(r);
}

void Prof::end(double flops, double bytes, int launches) {
  if (!on || recs.empty()) return;
  Rec &r = recs.back();
  r.flops = flops;
  r.bytes = bytes;
  r.launches = launches;
  cudaEventRecord(r.b, s);
}

void Prof::flush() {
  if (!on) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  for (auto &r : recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_prof.ms[r.phase] += ms;
      g_prof.launches[r.phase] += r.launches;
      g_prof.flops[r.phase] += r.flops;
      g_prof.bytes[r.phase] += r.bytes;
    }
    event_put(r.a);
    event_put(r.b);
  }
  recs.clear();
}

// ---------------------------------------------------------------------------
// small RAII helpers for stream-ordered device memory and pinned staging
// ---------------------------------------------------------------------------
struct DevBuf {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { reset(); }
  int alloc(size_t bytes, cudaStream_t stream) {
    reset();
    s = stream;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA;
    }
    return TUCKER_OK;
  }
  void reset() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  void *release() {
    void *q = p;
    p = nullptr;
    return q;
  }
  template <typename T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

// Per-thread pinned staging area for the per-mode device->host copies.
struct Pinned {
  void *p = nullptr;
  size_t n = 0;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
static thread_local Pinned g_pinned;

static int pinned(size_t bytes, void **out) {
  if (g_pinned.n < bytes) {
    if (g_pinned.p) cudaFreeHost(g_pinned.p);
    g_pinned.p = nullptr;
    g_pinned.n = 0;
    TK_CUDA(cudaMallocHost(&g_pinned.p, bytes));
    g_pinned.n = bytes;
  }
  *out = g_pinned.p;
  return TUCKER_OK;
}

static int fault_injection(const char *what) {
  const char *f = getenv("TUCKER_FAULT");
  return f && strcmp(f, what) == 0;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static int check_dims(const int64_t *dims, int N) {
  if (!dims || N < 1 || N > TUCKER_MAX_MODES) {
    set_error("N must be in [1, %d] and dims non-null", TUCKER_MAX_MODES);
    return TUCKER_EINVAL;
  }
  double total = 1.0;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1 || dims[n] > TUCKER_MAX_DIM) {
      set_error("dims[%d] = %lld outside [1, %d]", n, (long long)dims[n], TUCKER_MAX_DIM);
      return TUCKER_EINVAL;
    }
    total *= (double)dims[n];
  }
  if (total > 9.0e18) {
    set_error("tensor too large");
    return TUCKER_EINVAL;
  }
  return TUCKER_OK;
}

static int check_order(const int *order, int N, int *out) {
  if (!order) {
    for (int n = 0; n < N; ++n) out[n] = n;
    return TUCKER_OK;
  }
  bool seen[TUCKER_MAX_MODES] = {false};
  for (int k = 0; k < N; ++k) {
    const int n = order[k];
    if (n < 0 || n >= N || seen[n]) {
      set_error("mode_order is not a permutation of 0..%d", N - 1);
      return TUCKER_EINVAL;
    }
    seen[n] = true;
    out[k] = n;
  }
  return TUCKER_OK;
}

static size_t elem_size(tucker_dtype dt) { return dt == TUCKER_F64 ? 8 : 4; }

using Priv = ResultPriv;

// Pinned host blocks for results returned in host memory.  A freed result's
// block is kept (up to kHostCacheCap bytes in all) for the next result of a
// similar size, so repeated host calls neither pin new pages nor fault fresh
// pageable ones in, and their device-to-host copies run at DMA speed.  The
// cache is never destroyed: no CUDA call runs during process teardown.
struct HostBlockCache {
  std::mutex mu;
  std::multimap<size_t, void *> blocks;  // bytes -> block
  size_t bytes = 0;
};
static constexpr size_t kHostCacheCap = size_t(4) << 30;

static HostBlockCache &host_cache() {
  static HostBlockCache *c = new HostBlockCache;
  return *c;
}

// A pinned block of at least `bytes` bytes (*got: its size), or nullptr.  A
// cached block serves if it is at most twice the request.
static void *host_block_get(size_t bytes, size_t *got) {
  bytes = std::max<size_t>(bytes, 16);
  HostBlockCache &c = host_cache();
  {
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.blocks.lower_bound(bytes);
    if (it != c.blocks.end() && it->first / 2 <= bytes) {
      void *p = it->second;
      *got = it->first;
      c.bytes -= it->first;
      c.blocks.erase(it);
      return p;
    }
  }
  void *p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *got = bytes;
  return p;
}

static void host_block_put(void *p, size_t bytes) {
  if (!p) return;
  HostBlockCache &c = host_cache();
  {
    std::lock_guard<std::mutex> lock(c.mu);
    if (c.bytes + bytes <= kHostCacheCap) {
      c.blocks.emplace(bytes, p);
      c.bytes += bytes;
      return;
    }
  }
  cudaFreeHost(p);
}

static size_t host_cache_bytes() {
  HostBlockCache &c = host_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  return c.bytes;
}

// `own`: the stream that issued every use of r's device buffers (they are
// freed on it, in stream order, without a device synchronisation), or nullptr.
static void free_result_device(tucker_result *r, cudaStream_t *own = nullptr) {
  const Priv *pv = static_cast<const Priv *>(r->priv);
  if (pv && pv->block) {  // core and factors live in a block shared by a batch (freed with its last result)
    r->core = nullptr;
    for (int n = 0; n < TUCKER_MAX_MODES; ++n) r->factors[n] = nullptr;
    return;
  }
  if (r->on_host) {
    // core and factors share one pinned block, which goes back to the cache
    if (pv) host_block_put(pv->host_block, pv->host_bytes);
  } else {
    bool any = r->core != nullptr;
    for (int n = 0; n < TUCKER_MAX_MODES; ++n) any = any || r->factors[n] != nullptr;
    if (!any) return;
    // stream-ordered allocations go back to their pool with cudaFreeAsync
    // (freed with cudaFree, the pool's in-use count kept growing by every
    // freed result), after the device synchronisation tucker_result_free
    // promises unless the caller names the buffers' own stream; on the
    // result's own device when the caller has another one current
    int cur = -1;
    cudaGetDevice(&cur);
    const bool other = pv && !own && cur >= 0 && pv->device != cur;
    if (other) cudaSetDevice(pv->device);
    cudaStream_t fs = own ? *own : cudaStreamLegacy;
    if (!own) cudaDeviceSynchronize();
    if (r->core) cudaFreeAsync(r->core, fs);
    for (int n = 0; n < TUCKER_MAX_MODES; ++n)
      if (r->factors[n]) cudaFreeAsync(r->factors[n], fs);
    if (other) cudaSetDevice(cur);
  }
  r->core = nullptr;
  for (int n = 0; n < TUCKER_MAX_MODES; ++n) r->factors[n] = nullptr;
}

namespace {
// trace of a J x J column-major matrix, summed in index order (one thread)
__global__ void k_trace(const double *__restrict__ S, int J, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < J; ++i) t += S[i + (int64_t)J * i];
  *out = t;
}

// S = sum over c < n of the c-th J x J Gram in Sc (the Grams of the column
// chunks of one unfolding), added in chunk order
__global__ void k_sum_grams(const double *__restrict__ Sc, int n, int64_t JJ, double *__restrict__ S) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= JJ) return;
  double t = Sc[i];
  for (int c = 1; c < n; ++c) t += Sc[(int64_t)c * JJ + i];
  S[i] = t;
}
}  // namespace

// X arriving in column chunks of its first unfolding (the host entry
// point's copy): chunk c holds columns col[c] .. col[c + 1] - 1 once event
// ev[c] has completed.
constexpr int kMaxFeedChunks = 8;
struct HostFeed {
  int n = 0;
  cudaEvent_t ev[kMaxFeedChunks] = {};
  int64_t col[kMaxFeedChunks + 1] = {};
};

int launch_trace(const double *d_S, int64_t J, double *d_out, cudaStream_t s) {
  k_trace<<<1, 32, 0, s>>>(d_S, (int)J, d_out);
  TK_LAUNCHED();
  return TUCKER_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------
// `feed`: X is still arriving (see HostFeed); only with the BF16 digits and
// mode 1 processed first, whose Gram then runs chunk by chunk as the columns
// land (Sec. 2.2: the Gram is a sum over columns).
static int sthosvd_impl(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps, const int *order,
                        tucker_precision prec, cudaStream_t s, tucker_result *out, const HostFeed *feed = nullptr) {
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  const int64_t I = [&] {
    int64_t t = 1;
    for (int n = 0; n < N; ++n) t *= dims[n];
    return t;
  }();
  int64_t maxJ = 1;
  for (int n = 0; n < N; ++n) maxJ = std::max(maxJ, dims[n]);

  // small device scratch: norm partials, ||X||^2, S, lam, V, eig info, rank/tail
  DevBuf partials, scal, S, lam, V, eigws, gramws;
  TK_CHECK(partials.alloc(sizeof(double) * norm2_partials(), s));
  TK_CHECK(scal.alloc(64, s));
  TK_CHECK(S.alloc(sizeof(double) * maxJ * maxJ, s));
  TK_CHECK(lam.alloc(sizeof(double) * maxJ, s));
  TK_CHECK(V.alloc(sizeof(double) * maxJ * maxJ, s));
  // scal: ||X||^2 | tail | rank | eigensolver info (4 ints) | spare | TTM error flag
  double *d_nx2 = scal.as<double>();
  double *d_tail = d_nx2 + 1;
  int64_t *d_rank = reinterpret_cast<int64_t *>(d_nx2 + 2);
  int *d_info = reinterpret_cast<int *>(d_nx2 + 3);
  int *d_terr = reinterpret_cast<int *>(d_nx2 + 6);
  TK_CUDA(cudaMemsetAsync(d_terr, 0, sizeof(int), s));
  const bool split = prec != TUCKER_PREC_FP64;  // tensor-core digits for the Gram and the mode product
  const bool f8 = prec == TUCKER_PREC_E4M3X4;
  if (split) {  // the tensor-core kernels' limits (row blocks of 128 up to 512; the E4M3 Gram one block)
    const int64_t lim = f8 ? 128 : 512;
    for (int n = 0; n < N; ++n)
      if (dims[n] > lim) {
        set_error("%s split precision needs every I_n <= %lld (I_%d = %lld)", f8 ? "E4M3" : "BF16", (long long)lim, n,
                  (long long)dims[n]);
        return TUCKER_EUNSUPPORTED;
      }
  }

  void *host = nullptr;
  TK_CHECK(pinned(sizeof(double) * (8 + maxJ) + sizeof(int) * kMaxFeedChunks, &host));
  double *h = static_cast<double *>(host);
  int *h_chunk_err = reinterpret_cast<int *>(h + 8 + maxJ);  // the fed first Gram's per-chunk error flags
  int n_chunk_err = 0;
  if (feed && (prec != TUCKER_PREC_BF16X4 || order[0] != 0 || feed->n < 1 || feed->n > kMaxFeedChunks)) {
    set_error("internal: a chunked input needs the BF16 digits with mode 1 first");
    return TUCKER_EINVAL;
  }

  // ||X||^2 and the threshold of the rank rule.  The split-precision path
  // takes ||X||^2 as the trace of its first Gram (equal in exact arithmetic;
  // the 21-bit rounding of the Gram moves it by ~1e-10 relative), saving a
  // float64-bound pass over X; it is read back after the first Gram.
  // (the E4M3 Gram rounds entries to 15 bits: its trace is too coarse for the threshold)
  const bool norm_from_trace = prec == TUCKER_PREC_BF16X4;
  const int keep_all = !(eps > 0.0);
  double nx2 = 0.0, threshold = 0.0;
  auto set_norm = [&](double v) -> int {
    nx2 = v;
    if (!std::isfinite(nx2) || fault_injection("nan")) {
      set_error("||X||^2 is not finite (%g): the input holds Inf or NaN", nx2);
      return TUCKER_ENONFINITE;
    }
    threshold = keep_all ? 0.0 : eps * eps * nx2 / N;
    out->norm2_x = nx2;
    out->threshold = threshold;
    return TUCKER_OK;
  };
  if (!norm_from_trace) {
    TK_CHECK(launch_norm2(X, dt, I, partials.as<double>(), d_nx2, s, &prof));
    TK_CUDA(cudaMemcpyAsync(h, d_nx2, sizeof(double), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    TK_CHECK(set_norm(h[0]));
  }

  out->N = N;
  out->on_host = 0;
  for (int n = 0; n < N; ++n) {
    out->dims[n] = dims[n];
    out->mode_order[n] = order[n];
  }

  int64_t cur[TUCKER_MAX_MODES];
  for (int n = 0; n < N; ++n) cur[n] = dims[n];
  const void *Y = X;
  tucker_dtype ydt = dt;
  DevBuf ybuf;  // owns Y when Y != X
  DevBuf factor_bufs[TUCKER_MAX_MODES];
  std::vector<double *> eig_host(N, nullptr);
  struct EigFree {
    std::vector<double *> &v;
    bool keep = false;
    ~EigFree() {
      if (!keep)
        for (double *p : v) free(p);
    }
  } eig_guard{eig_host};

  for (int k = 0; k < N; ++k) {
    const int n = order[k];
    int64_t L = 1, B = 1;
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < N; ++m) B *= cur[m];
    const int64_t J = cur[n];

    // Gram step (its exponent pass also leaves the column exponents the TTM needs)
    DevBuf colexp;
    const bool want_colexp = L > 1 || J <= 128;  // longer contiguous columns: the TTM scales its parts itself
    if (split && k == 0 && feed) {
      // mode 1 (L = 1) while X arrives: each chunk of columns gets its own
      // exponent pass and Gram (with its own workspace and error flag) as
      // soon as it has landed, and the chunks' Grams are added in order; the
      // 512-column exponent groups are the same as in one pass over X
      const int nc = feed->n;
      const size_t es = ydt == TUCKER_F64 ? 8 : 4;
      auto chunk_y = [&](int c) { return static_cast<const void *>(static_cast<const char *>(Y) + es * J * feed->col[c]); };
      int64_t gws = 0;
      for (int c = 0; c < nc; ++c)
        gws = std::max(gws, gram_split_workspace_doubles(1, J, feed->col[c + 1] - feed->col[c], dev, ydt, chunk_y(c)));
      TK_CHECK(gramws.alloc(sizeof(double) * gws * nc, s));
      if (want_colexp) TK_CHECK(colexp.alloc(sizeof(int) * L * B, s));
      DevBuf Sc;
      TK_CHECK(Sc.alloc(sizeof(double) * J * J * nc, s));
      reinterpret_cast<int *>(h + 5)[0] = 0;  // no single-pass flag this mode
      for (int c = 0; c < nc; ++c) {
        const int64_t c0 = feed->col[c], bc = feed->col[c + 1] - c0;
        double *wsc = gramws.as<double>() + gws * c;
        TK_CUDA(cudaStreamWaitEvent(s, feed->ev[c], 0));
        TK_CHECK(launch_gram_split(chunk_y(c), ydt, 1, J, bc, Sc.as<double>() + J * J * c, wsc, dev, s, &prof,
                                   want_colexp ? colexp.as<int>() + c0 : nullptr, f8));
        TK_CHECK(gram_split_error(wsc, 1, J, bc, dev, h_chunk_err + c, s));
      }
      n_chunk_err = nc;
      const int64_t JJ = J * J;
      k_sum_grams<<<(unsigned)((JJ + 255) / 256), 256, 0, s>>>(Sc.as<double>(), nc, JJ, S.as<double>());
      TK_LAUNCHED();
      TK_CHECK(launch_trace(S.as<double>(), J, d_nx2, s));
      TK_CUDA(cudaMemcpyAsync(h, d_nx2, sizeof(double), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      TK_CHECK(set_norm(h[0]));
    } else if (split) {
      const int64_t gws = gram_split_workspace_doubles(L, J, B, dev, ydt, Y);
      TK_CHECK(gramws.alloc(sizeof(double) * gws, s));
      if (want_colexp) TK_CHECK(colexp.alloc(sizeof(int) * L * B, s));
      TK_CHECK(launch_gram_split(Y, ydt, L, J, B, S.as<double>(), gramws.as<double>(), dev, s, &prof,
                                 want_colexp ? colexp.as<int>() : nullptr, f8));
      TK_CHECK(gram_split_error(gramws.as<double>(), L, J, B, dev, reinterpret_cast<int *>(h + 5), s));
      if (k == 0 && norm_from_trace) {
        TK_CHECK(launch_trace(S.as<double>(), J, d_nx2, s));
        TK_CUDA(cudaMemcpyAsync(h, d_nx2, sizeof(double), cudaMemcpyDeviceToHost, s));
        TK_CUDA(cudaStreamSynchronize(s));
        TK_CHECK(set_norm(h[0]));
      }
    } else {
      const int64_t gws = gram_workspace_doubles(L, J, B, dev);
      TK_CHECK(gramws.alloc(sizeof(double) * gws, s));
      TK_CHECK(launch_gram(Y, ydt, L, J, B, S.as<double>(), gramws.as<double>(), dev, s, &prof));
    }
    // eigenvector step
    const int64_t ews = eig_workspace_doubles(J);
    if (ews > 0) TK_CHECK(eigws.alloc(sizeof(double) * ews, s));
    TK_CHECK(launch_eig(S.as<double>(), J, lam.as<double>(), V.as<double>(), ews > 0 ? eigws.as<double>() : nullptr,
                        d_info, s, &prof, keep_all ? -1.0 : threshold));
    // rank step
    TK_CHECK(launch_rank_cut(lam.as<double>(), J, threshold, keep_all, d_rank, d_tail, s, &prof));
    TK_CUDA(cudaMemcpyAsync(h, d_tail, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaMemcpyAsync(h + 8, lam.as<double>(), sizeof(double) * J, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    bool gram_expired = split && reinterpret_cast<int *>(h + 5)[0] != 0;
    for (int c = 0; c < n_chunk_err; ++c) gram_expired = gram_expired || h_chunk_err[c] != 0;
    n_chunk_err = 0;
    if (gram_expired) {
      set_error("split-precision Gram: a bounded tensor-core wait expired (mode %d)", n);
      return TUCKER_ETIMEOUT;
    }
    const double tail = h[0];
    int64_t R;
    int info[4];  // sweeps, not converged, eigensolver path, resolved count
    memcpy(&R, h + 1, sizeof R);
    memcpy(info, h + 2, sizeof info);
    if (info[1] != 0 || fault_injection("noconv")) {
      set_error("Jacobi eigensolver did not converge for mode %d (J = %lld) within %d sweeps", n, (long long)J,
                info[0]);
      return TUCKER_ENOCONV;
    }
    if (R < 1 || R > J) {
      set_error("rank rule returned R = %lld outside [1, %lld]", (long long)R, (long long)J);
      return TUCKER_ECUDA;
    }
    eig_host[n] = static_cast<double *>(malloc(sizeof(double) * J));
    if (!eig_host[n]) {
      set_error("host allocation failed");
      return TUCKER_ENOMEM;
    }
    memcpy(eig_host[n], h + 8, sizeof(double) * J);
    out->ranks[n] = R;
    out->tail[n] = tail;
    out->sweeps[n] = info[0];
    out->eig_path[n] = info[2];
    out->eig_resolved[n] = info[3];

    // factor U_n = leading R eigenvectors (first R columns of V)
    TK_CHECK(factor_bufs[n].alloc(sizeof(double) * J * R, s));
    TK_CUDA(cudaMemcpyAsync(factor_bufs[n].p, V.p, sizeof(double) * J * R, cudaMemcpyDeviceToDevice, s));

    // TTM step Y <- Y x_n U_n^T
    if (fault_injection("alloc")) {
      set_error("injected allocation failure");
      return TUCKER_ENOMEM;
    }
    DevBuf ynew;
    TK_CHECK(ynew.alloc(sizeof(double) * L * R * B, s));
    if (split)
      TK_CHECK(launch_ttm_split(Y, ydt, L, J, B, factor_bufs[n].as<double>(), R, ynew.as<double>(), d_terr, dev, s,
                                &prof, want_colexp ? colexp.as<int>() : nullptr));
    else
      TK_CHECK(launch_ttm(Y, ydt, L, J, B, factor_bufs[n].as<double>(), /*ak=*/J, /*aj=*/1, R, ynew.as<double>(),
                          dev, s, &prof));
    // TUCKER_FAULT=timeout: raise the error flag a tensor-core wait raises on
    // expiry (host-side injection; no kernel is made to stall)
    if (fault_injection("timeout")) TK_CUDA(cudaMemsetAsync(d_terr, 1, 1, s));
    ybuf.reset();
    ybuf.p = ynew.release();
    ybuf.s = s;
    Y = ybuf.p;
    ydt = TUCKER_F64;
    cur[n] = R;
  }
  int terr = 0;
  TK_CUDA(cudaMemcpyAsync(&terr, d_terr, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (terr) {
    set_error("a bounded tensor-core wait expired (split-precision mode product)%s",
              fault_injection("timeout") ? " [injected by TUCKER_FAULT=timeout]" : "");
    return TUCKER_ETIMEOUT;
  }
  out->core = static_cast<double *>(ybuf.release());
  for (int n = 0; n < N; ++n) {
    out->factors[n] = factor_bufs[n].as<double>();
    factor_bufs[n].release();
    out->eigvals[n] = eig_host[n];
  }
  eig_guard.keep = true;
  Priv *pv = new Priv;
  pv->device = dev.device;
  out->priv = pv;
  return TUCKER_OK;
}

// Expands core x {U_n} over every mode except `skip` (or all when skip < 0),
// smallest growth first; returns the buffer and its current dims.  With lo
// and hi (both or neither), mode n expands to rows lo[n] .. hi[n]-1 of U_n
// only: a subtensor of X~ (Sec. 2.3, subsets of rows of the factors).
static int expand_modes(const tucker_result *r, int skip, double *final_out, DevBuf &hold, const double **res,
                        int64_t *cur, const DeviceInfo &dev, cudaStream_t s, Prof *prof, const int64_t *lo = nullptr,
                        const int64_t *hi = nullptr) {
  const int N = r->N;
  for (int n = 0; n < N; ++n) cur[n] = r->ranks[n];
  auto rows = [&](int n) -> int64_t { return lo ? hi[n] - lo[n] : r->dims[n]; };
  int seq[TUCKER_MAX_MODES], cnt = 0;
  for (int n = 0; n < N; ++n)
    if (n != skip) seq[cnt++] = n;
  for (int a = 1; a < cnt; ++a)  // insertion sort by growth rows_n / R_n
    for (int b = a; b > 0; --b) {
      const double gb = (double)rows(seq[b]) / r->ranks[seq[b]];
      const double ga = (double)rows(seq[b - 1]) / r->ranks[seq[b - 1]];
      if (gb < ga) std::swap(seq[b], seq[b - 1]);
    }
  const double *y = r->core;
  DevBuf tmp;
  for (int k = 0; k < cnt; ++k) {
    const int n = seq[k];
    int64_t L = 1, B = 1;
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < N; ++m) B *= cur[m];
    const int64_t J = cur[n], K = rows(n);
    double *z;
    DevBuf next;
    if (final_out && k == cnt - 1) {
      z = final_out;
    } else {
      TK_CHECK(next.alloc(sizeof(double) * L * K * B, s));
      z = next.as<double>();
    }
    // A = rows lo[n].. of U_n (I_n x J, column-major): A[k, j] = U[lo + k + I_n j]
    TK_CHECK(launch_ttm(y, TUCKER_F64, L, J, B, r->factors[n] + (lo ? lo[n] : 0), /*ak=*/1, /*aj=*/r->dims[n], K, z,
                        dev, s, prof));
    if (!(final_out && k == cnt - 1)) {
      tmp.reset();
      tmp.p = next.release();
      tmp.s = s;
    }
    y = z;
    cur[n] = K;
  }
  if (cnt == 0 && final_out) {
    int64_t tot = 1;
    for (int n = 0; n < N; ++n) tot *= cur[n];
    TK_CUDA(cudaMemcpyAsync(final_out, r->core, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    y = final_out;
  }
  hold.reset();
  hold.p = tmp.release();
  hold.s = s;
  *res = y;
  return TUCKER_OK;
}

// Algorithm 2 (HOOI) after Algorithm 1 has filled `out` (ranks fixed).
// Each iteration: for n = 0..N-1, Y = X x {U_m^T}_{m != n} with the factors
// as updated so far (formed from a shared partial product, below),
// S = Y_(n) Y_(n)^T, U_n = leading R_n eigenvectors of S; then
// G = Y x_{N-1} U_{N-1}^T from the last Y.  fit[k] = ||X||^2 - ||G||^2.
static int hooi_iterate(const void *X, tucker_dtype dt, int max_iters, double tol, tucker_precision prec,
                        cudaStream_t s, tucker_result *out, int *iters, double *fit) {
  const int N = out->N;
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  int64_t maxJ = 1, ncore = 1;
  for (int n = 0; n < N; ++n) {
    maxJ = std::max(maxJ, out->dims[n]);
    ncore *= out->ranks[n];
  }
  DevBuf S, lam, V, eigws, gramws, partials, scal;
  TK_CHECK(S.alloc(sizeof(double) * maxJ * maxJ, s));
  TK_CHECK(lam.alloc(sizeof(double) * maxJ, s));
  TK_CHECK(V.alloc(sizeof(double) * maxJ * maxJ, s));
  TK_CHECK(partials.alloc(sizeof(double) * norm2_partials(), s));
  TK_CHECK(scal.alloc(64, s));
  double *d_g2 = scal.as<double>();
  int *d_info = reinterpret_cast<int *>(d_g2 + 1);  // 4 ints
  int *d_terr = reinterpret_cast<int *>(d_g2 + 4);
  TK_CUDA(cudaMemsetAsync(d_terr, 0, sizeof(int), s));
  const double nx2 = out->norm2_x;
  auto core_fit = [&](double *f) -> int {
    TK_CHECK(launch_norm2(out->core, TUCKER_F64, ncore, partials.as<double>(), d_g2, s, &prof));
    double g2 = 0.0;
    TK_CUDA(cudaMemcpyAsync(&g2, d_g2, sizeof(double), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    *f = nx2 - g2;
    return TUCKER_OK;
  };
  double prev = 0.0;
  TK_CHECK(core_fit(&prev));
  if (fit) fit[0] = prev;
  *iters = 0;
  // Y <- src x {U_m^T : m in modes}, the largest reductions I_m / R_m first.
  // cur holds src's dims on entry and Y's on return; hold owns Y unless no
  // mode applies (then Y is src).
  auto contract = [&](const void *src, tucker_dtype sdt, int64_t *cur, int *modes, int cnt, DevBuf &hold,
                      const void **res, tucker_dtype *rdt) -> int {
    std::stable_sort(modes, modes + cnt, [&](int a, int b) {
      return (double)out->dims[a] / out->ranks[a] > (double)out->dims[b] / out->ranks[b];
    });
    const void *Y = src;
    tucker_dtype ydt = sdt;
    DevBuf ybuf;
    for (int k = 0; k < cnt; ++k) {
      const int m = modes[k];
      int64_t L = 1, B = 1;
      for (int q = 0; q < m; ++q) L *= cur[q];
      for (int q = m + 1; q < N; ++q) B *= cur[q];
      const int64_t J = cur[m], R = out->ranks[m];
      DevBuf ynew;
      TK_CHECK(ynew.alloc(sizeof(double) * L * R * B, s));
      if (prec != TUCKER_PREC_FP64)
        TK_CHECK(launch_ttm_split(Y, ydt, L, J, B, out->factors[m], R, ynew.as<double>(), d_terr, dev, s, &prof));
      else
        TK_CHECK(launch_ttm(Y, ydt, L, J, B, out->factors[m], /*ak=*/J, /*aj=*/1, R, ynew.as<double>(), dev, s,
                            &prof));
      ybuf.reset();
      ybuf.p = ynew.release();
      ybuf.s = s;
      Y = ybuf.p;
      ydt = TUCKER_F64;
      cur[m] = R;
    }
    hold.reset();
    hold.p = ybuf.release();
    hold.s = s;
    *res = Y;
    *rdt = ydt;
    return TUCKER_OK;
  };
  // Two-level reuse of the products with X: the modes split into a first
  // half F = {0..h-1} and the rest.  While F's factors are updated, every Y
  // shares Z_F = X x {U_m^T : m >= h} (those factors do not change until F is
  // done); the later modes share Z = X x {U_m^T : m < h} with F's new factors.
  // Each iteration reads X twice instead of N times; the products are those of
  // Algorithm 2 with the contractions associated differently.
  const int h = N / 2;
  for (int it = 0; it < max_iters; ++it) {
    DevBuf zbuf;
    const void *Z = X;
    tucker_dtype zdt = dt;
    int64_t zcur[TUCKER_MAX_MODES];
    for (int n = 0; n < N; ++n) {
      if (n == 0 || n == h) {  // Z for this half: contract the other half's modes of X
        int other[TUCKER_MAX_MODES], cnt = 0;
        for (int m = 0; m < N; ++m)
          if ((m < h) != (n < h)) other[cnt++] = m;
        for (int m = 0; m < N; ++m) zcur[m] = out->dims[m];
        zbuf.reset();
        TK_CHECK(contract(X, dt, zcur, other, cnt, zbuf, &Z, &zdt));
      }
      int seq[TUCKER_MAX_MODES], cnt = 0;
      for (int m = 0; m < N; ++m)
        if (m != n && (m < h) == (n < h)) seq[cnt++] = m;
      int64_t cur[TUCKER_MAX_MODES];
      for (int m = 0; m < N; ++m) cur[m] = zcur[m];
      const void *Y = nullptr;
      tucker_dtype ydt = zdt;
      DevBuf ybuf;
      TK_CHECK(contract(Z, zdt, cur, seq, cnt, ybuf, &Y, &ydt));
      int64_t L = 1, B = 1;
      for (int q = 0; q < n; ++q) L *= cur[q];
      for (int q = n + 1; q < N; ++q) B *= cur[q];
      const int64_t J = out->dims[n], R = out->ranks[n];
      TK_CHECK(gramws.alloc(sizeof(double) * gram_workspace_doubles(L, J, B, dev), s));
      TK_CHECK(launch_gram(Y, ydt, L, J, B, S.as<double>(), gramws.as<double>(), dev, s, &prof));
      const int64_t ews = eig_workspace_doubles(J);
      if (ews > 0) TK_CHECK(eigws.alloc(sizeof(double) * ews, s));
      TK_CHECK(launch_eig(S.as<double>(), J, lam.as<double>(), V.as<double>(), ews > 0 ? eigws.as<double>() : nullptr,
                          d_info, s, &prof, -1.0));
      int info[2];
      TK_CUDA(cudaMemcpyAsync(info, d_info, sizeof info, cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      if (info[1] != 0) {
        set_error("HOOI: the eigensolver did not converge for mode %d (J = %lld)", n, (long long)J);
        return TUCKER_ENOCONV;
      }
      TK_CUDA(cudaMemcpyAsync(out->factors[n], V.p, sizeof(double) * J * R, cudaMemcpyDeviceToDevice, s));
      if (n == N - 1) {  // G = Y x_{N-1} U_{N-1}^T
        TK_CHECK(launch_ttm(Y, ydt, L, J, B, out->factors[n], /*ak=*/J, /*aj=*/1, R, out->core, dev, s, &prof));
      }
    }
    double f = 0.0;
    TK_CHECK(core_fit(&f));
    *iters = it + 1;
    if (fit) fit[it + 1] = f;
    const bool done = prev - f <= tol * nx2;
    prev = f;
    if (done) break;
  }
  int terr = 0;
  TK_CUDA(cudaMemcpyAsync(&terr, d_terr, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (terr) {
    set_error("split-precision TTM: a bounded tensor-core wait expired");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

// Flops of Algorithm 1 in a mode order (the ST-HOSVD cost of Sec. 6.1 with
// one process): the step on mode n, with J the product of the current
// dimensions, costs 2 I_n J (Gram) + 2 R_n J (TTM) + 10/3 I_n^3 (eigenvectors).
static double step_flops(const int64_t *dims, const int64_t *ranks, const int64_t *cur, int N, int n) {
  double j = 1.0;
  for (int m = 0; m < N; ++m) j *= (double)cur[m];
  return 2.0 * (double)dims[n] * j + 2.0 * (double)ranks[n] * j + 10.0 / 3.0 * std::pow((double)dims[n], 3.0);
}

static double order_flops(const int64_t *dims, const int64_t *ranks, int N, const int *order) {
  int64_t cur[TUCKER_MAX_MODES];
  for (int m = 0; m < N; ++m) cur[m] = dims[m];
  double total = 0.0;
  for (int k = 0; k < N; ++k) {
    total += step_flops(dims, ranks, cur, N, order[k]);
    cur[order[k]] = ranks[order[k]];
  }
  return total;
}

static int check_result(const tucker_result *r) {
  if (!r || r->N < 1 || r->N > TUCKER_MAX_MODES || !r->core) {
    set_error("result is empty or invalid");
    return TUCKER_EINVAL;
  }
  if (r->on_host) {
    set_error("result lives on the host; device entry points need a device result");
    return TUCKER_EINVAL;
  }
  for (int n = 0; n < r->N; ++n)
    if (!r->factors[n] || r->ranks[n] < 1 || r->ranks[n] > r->dims[n]) {
      set_error("result factor %d is invalid", n);
      return TUCKER_EINVAL;
    }
  return TUCKER_OK;
}

}  // namespace tk

using namespace tk;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *tucker_status_string(int status) {
  switch (status) {
    case TUCKER_OK: return "ok";
    case TUCKER_EINVAL: return "invalid argument";
    case TUCKER_ENOMEM: return "out of memory";
    case TUCKER_ECUDA: return "CUDA error";
    case TUCKER_ENOCONV: return "eigensolver did not converge";
    case TUCKER_ETIMEOUT: return "device wait timed out";
    case TUCKER_ENONFINITE: return "input is not finite";
    case TUCKER_EUNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char *tucker_last_error(void) { return g_err; }

int64_t tucker_launch_count(void) { return g_launches.load(); }

int tucker_memory_stats(int64_t *pool_used, int64_t *pool_reserved, int64_t *host_cached) {
  g_err[0] = 0;
  if (pool_used || pool_reserved) {
    int dev = 0;
    TK_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    TK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t v = 0;
    if (pool_used) {
      TK_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
      *pool_used = (int64_t)v;
    }
    if (pool_reserved) {
      TK_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v));
      *pool_reserved = (int64_t)v;
    }
  }
  if (host_cached) *host_cached = (int64_t)host_cache_bytes();
  return TUCKER_OK;
}

int tucker_memory_trim(void) {
  g_err[0] = 0;
  TK_CUDA(cudaDeviceSynchronize());
  std::multimap<size_t, void *> blocks;
  {
    HostBlockCache &c = host_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    blocks.swap(c.blocks);
    c.bytes = 0;
  }
  for (auto &b : blocks) TK_CUDA(cudaFreeHost(b.second));
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  TK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  TK_CUDA(cudaMemPoolTrimTo(pool, 0));
  return TUCKER_OK;
}

void tucker_batched_tuning(int64_t *cols_per_item, int *ctas, float *candidate_ms) {
  batched_last_tuning(cols_per_item, ctas, candidate_ms);
}

int tucker_fp64_peak(double *tflops, double *ms, void *stream) {
  g_err[0] = 0;
  if (!tflops) {
    set_error("tflops is NULL");
    return TUCKER_EINVAL;
  }
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  return fp64_peak(tflops, ms, dev, static_cast<cudaStream_t>(stream));
}

void tucker_profile_enable(int on) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (on) memset(&g_prof, 0, sizeof g_prof);
  g_prof_on = on != 0;
}

void tucker_profile_read(tucker_profile *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  *p = g_prof;
}

static int sthosvd_entry(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps,
                         const int *mode_order, tucker_precision prec, void *stream, tucker_result *out,
                         const HostFeed *feed);

int tucker_sthosvd(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps, const int *mode_order,
                   tucker_precision prec, void *stream, tucker_result *out) {
  return sthosvd_entry(X, dt, dims, N, eps, mode_order, prec, stream, out, nullptr);
}

static int sthosvd_entry(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps,
                         const int *mode_order, tucker_precision prec, void *stream, tucker_result *out,
                         const HostFeed *feed) {
  g_err[0] = 0;
  if (!out) {
    set_error("out is NULL");
    return TUCKER_EINVAL;
  }
  memset(out, 0, sizeof *out);
  if (!X) {
    set_error("X is NULL");
    return TUCKER_EINVAL;
  }
  if (dt != TUCKER_F64 && dt != TUCKER_F32) {
    set_error("unknown dtype %d", (int)dt);
    return TUCKER_EINVAL;
  }
  if (prec != TUCKER_PREC_FP64 && prec != TUCKER_PREC_BF16X4 && prec != TUCKER_PREC_E4M3X4) {
    set_error("unknown precision %d", (int)prec);
    return TUCKER_EINVAL;
  }
  if (std::isnan(eps)) {
    set_error("eps is NaN");
    return TUCKER_EINVAL;
  }
  TK_CHECK(check_dims(dims, N));
  int order[TUCKER_MAX_MODES];
  TK_CHECK(check_order(mode_order, N, order));
  if (feed && (prec != TUCKER_PREC_BF16X4 || order[0] != 0)) {  // no chunked first Gram: wait for the whole copy
    TK_CUDA(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), feed->ev[feed->n - 1], 0));
    feed = nullptr;
  }
  int st = sthosvd_impl(X, dt, dims, N, eps, order, prec, static_cast<cudaStream_t>(stream), out, feed);
  if (st != TUCKER_OK) {
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    memset(out, 0, sizeof *out);
  }
  return st;
}

// ---------------------------------------------------------------------------
// host entry points: X copied in, results copied out
// ---------------------------------------------------------------------------
// The copy of a host tensor goes on a stream of the library's own, one event
// per chunk.  With the BF16 digits and mode 1 first (and at least two
// 512-column groups) it goes in up to eight chunks of whole groups of the
// mode-1 unfolding and mode 1's Gram starts on each chunk as it lands
// (feed->n = chunks); otherwise in one piece, marked by ev[0] (feed->n = 0:
// the compute waits for all of it).
struct Copier {
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[2][kMaxFeedChunks] = {};  // one set per device buffer
  bool open() {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      cs = nullptr;
      cudaGetLastError();
      return false;
    }
    for (auto &set : ev)
      for (auto &e : set)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
          e = nullptr;
          cudaGetLastError();
          close();
          return false;
        }
    return true;
  }
  // stream and events are released once their pending work has completed
  void close() {
    for (auto &set : ev)
      for (auto &e : set)
        if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
    cs = nullptr;
    for (auto &set : ev)
      for (auto &e : set) e = nullptr;
  }
};

// Issues X_host -> dX on the copier's stream with event set `set`; fills
// *feed and *last (the event after the whole copy).
static int issue_copy(const void *X_host, void *dX, tucker_dtype dt, const int64_t *dims, int64_t I,
                      tucker_precision prec, const int *order, Copier &cp, int set, HostFeed *feed,
                      cudaEvent_t *last) {
  const int64_t B0 = I / dims[0];
  const size_t col_bytes = elem_size(dt) * (size_t)dims[0];
  feed->n = 0;
  if (prec == TUCKER_PREC_BF16X4 && order[0] == 0 && B0 >= 2 * 512) {
    // chunks of ceil(B0 / 8) columns rounded up to whole groups: at most eight
    const int64_t per = std::max<int64_t>(512, ((B0 + kMaxFeedChunks - 1) / kMaxFeedChunks + 511) / 512 * 512);
    const int nc = (int)((B0 + per - 1) / per);
    if (nc >= 2 && nc <= kMaxFeedChunks) {
      for (int c = 0; c < nc; ++c) {
        feed->col[c] = per * c;
        feed->col[c + 1] = std::min(B0, per * (c + 1));
        feed->ev[c] = cp.ev[set][c];
        const size_t off = col_bytes * (size_t)feed->col[c];
        const size_t bytes = col_bytes * (size_t)(feed->col[c + 1] - feed->col[c]);
        TK_CUDA(cudaMemcpyAsync(static_cast<char *>(dX) + off, static_cast<const char *>(X_host) + off, bytes,
                                cudaMemcpyHostToDevice, cp.cs));
        TK_CUDA(cudaEventRecord(cp.ev[set][c], cp.cs));
      }
      feed->n = nc;
      *last = cp.ev[set][nc - 1];
      return TUCKER_OK;
    }
  }
  TK_CUDA(cudaMemcpyAsync(dX, X_host, elem_size(dt) * I, cudaMemcpyHostToDevice, cp.cs));
  TK_CUDA(cudaEventRecord(cp.ev[set][0], cp.cs));
  *last = cp.ev[set][0];
  return TUCKER_OK;
}

// The ST-HOSVD of the tensor in dX once its copy (feed, last) has landed,
// with core and factors copied to one pinned host block (out->on_host = 1).
static int sthosvd_to_host(void *dX, tucker_dtype dt, const int64_t *dims, int N, double eps, const int *mode_order,
                           tucker_precision prec, cudaStream_t s, const HostFeed *feed, cudaEvent_t last,
                           tucker_result *out) {
  memset(out, 0, sizeof *out);
  if (feed->n == 0 && last) TK_CUDA(cudaStreamWaitEvent(s, last, 0));
  tucker_result dres;
  const int st = sthosvd_entry(dX, dt, dims, N, eps, mode_order, prec, s, &dres, feed->n > 0 ? feed : nullptr);
  if (st != TUCKER_OK) return st;
  *out = dres;
  out->on_host = 1;
  out->core = nullptr;
  for (int n = 0; n < TUCKER_MAX_MODES; ++n) out->factors[n] = nullptr;
  // core and factors in one pinned block: core first, then U_1 .. U_N
  int64_t total = 1;
  for (int n = 0; n < N; ++n) total *= dres.ranks[n];
  const int64_t G = total;
  for (int n = 0; n < N; ++n) total += dims[n] * dres.ranks[n];
  size_t got = 0;
  double *hb = static_cast<double *>(host_block_get(sizeof(double) * total, &got));
  Priv *pv = static_cast<Priv *>(out->priv);
  pv->host_block = hb;
  pv->host_bytes = got;
  cudaError_t e = cudaSuccess;
  if (hb) {
    out->core = hb;
    int64_t off = G;
    for (int n = 0; n < N; ++n) {
      out->factors[n] = hb + off;
      off += dims[n] * dres.ranks[n];
    }
    e = cudaMemcpyAsync(out->core, dres.core, sizeof(double) * G, cudaMemcpyDeviceToHost, s);
    for (int n = 0; n < N && e == cudaSuccess; ++n)
      e = cudaMemcpyAsync(out->factors[n], dres.factors[n], sizeof(double) * dims[n] * dres.ranks[n],
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  // release the device copies (eigenvalues and priv now belong to *out)
  for (int n = 0; n < TUCKER_MAX_MODES; ++n) dres.eigvals[n] = nullptr;
  dres.priv = nullptr;
  free_result_device(&dres, &s);  // produced and copied on s only
  if (!hb || e != cudaSuccess) {
    if (!hb) set_error("pinned host allocation of %lld bytes failed", (long long)(sizeof(double) * total));
    else set_error("device-to-host copy failed: %s", cudaGetErrorString(e));
    tucker_result_free(out);
    return hb ? TUCKER_ECUDA : TUCKER_ENOMEM;
  }
  return TUCKER_OK;
}

static int check_host_args(const void *const *X, int count, tucker_dtype dt, const int64_t *dims, int N,
                           const int *mode_order, tucker_result *out, int *order) {
  if (!out || !X || count < 0) {
    set_error("X_host and out must be non-null and count >= 0");
    return TUCKER_EINVAL;
  }
  memset(out, 0, sizeof(tucker_result) * (size_t)count);
  for (int k = 0; k < count; ++k)
    if (!X[k]) {
      set_error("host tensor %d is NULL", k);
      return TUCKER_EINVAL;
    }
  if (dt != TUCKER_F64 && dt != TUCKER_F32) {
    set_error("unknown dtype %d", (int)dt);
    return TUCKER_EINVAL;
  }
  TK_CHECK(check_dims(dims, N));
  return check_order(mode_order, N, order);
}

// `count` host tensors of one shape in turn through two device buffers: the
// copy of tensor k + 1 runs while tensor k is compressed.
static int sthosvd_host_run(const void *const *X, int count, tucker_dtype dt, const int64_t *dims, int N, double eps,
                            const int *mode_order, tucker_precision prec, cudaStream_t s, tucker_result *out) {
  int order[TUCKER_MAX_MODES];
  TK_CHECK(check_host_args(X, count, dt, dims, N, mode_order, out, order));
  if (count == 0) return TUCKER_OK;
  int64_t I = 1;
  for (int n = 0; n < N; ++n) I *= dims[n];
  DevBuf dX[2];
  const int nbuf = count > 1 ? 2 : 1;
  for (int b = 0; b < nbuf; ++b) TK_CHECK(dX[b].alloc(elem_size(dt) * I, s));
  Copier cp;
  if (!cp.open()) {  // no copy stream: copy and compress one tensor at a time on the caller's stream
    for (int k = 0; k < count; ++k) {
      TK_CUDA(cudaMemcpyAsync(dX[0].p, X[k], elem_size(dt) * I, cudaMemcpyHostToDevice, s));
      const HostFeed none;
      const int st = sthosvd_to_host(dX[0].p, dt, dims, N, eps, mode_order, prec, s, &none, nullptr, out + k);
      if (st != TUCKER_OK) {
        for (int j = 0; j < k; ++j) tucker_result_free(out + j);
        return st;
      }
    }
    return TUCKER_OK;
  }
  cudaEvent_t ready = nullptr;  // the buffers' stream-ordered allocations are usable on the copy stream
  int st = TUCKER_OK;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ready, s) != cudaSuccess || cudaStreamWaitEvent(cp.cs, ready, 0) != cudaSuccess) {
    cudaGetLastError();
    set_error("could not order the copy stream after the buffers' allocation");
    st = TUCKER_ECUDA;
  }
  if (ready) cudaEventDestroy(ready);
  HostFeed feed[2];
  cudaEvent_t last[2] = {nullptr, nullptr}, issued = nullptr;
  if (st == TUCKER_OK) st = issue_copy(X[0], dX[0].p, dt, dims, I, prec, order, cp, 0, &feed[0], &last[0]);
  if (st == TUCKER_OK) issued = last[0];
  int k = 0;
  for (; k < count && st == TUCKER_OK; ++k) {
    const int b = k & 1;
    // the other buffer's tensor (k - 1) is done: its call returned
    if (k + 1 < count) {
      st = issue_copy(X[k + 1], dX[b ^ 1].p, dt, dims, I, prec, order, cp, b ^ 1, &feed[b ^ 1], &last[b ^ 1]);
      if (st != TUCKER_OK) break;
      issued = last[b ^ 1];
    }
    st = sthosvd_to_host(dX[b].p, dt, dims, N, eps, mode_order, prec, s, &feed[b], last[b], out + k);
  }
  // the buffers are freed on the caller's stream: after every copy issued, whatever path ran
  if (issued) cudaStreamWaitEvent(s, issued, 0);
  cp.close();
  if (st != TUCKER_OK)
    for (int j = 0; j < count; ++j) tucker_result_free(out + j);
  return st;
}

int tucker_sthosvd_host(const void *X_host, tucker_dtype dt, const int64_t *dims, int N, double eps,
                        const int *mode_order, tucker_precision prec, void *stream, tucker_result *out) {
  g_err[0] = 0;
  return sthosvd_host_run(&X_host, 1, dt, dims, N, eps, mode_order, prec, static_cast<cudaStream_t>(stream), out);
}

int tucker_sthosvd_host_many(const void *const *X_hosts, int count, tucker_dtype dt, const int64_t *dims, int N,
                             double eps, const int *mode_order, tucker_precision prec, void *stream,
                             tucker_result *out) {
  g_err[0] = 0;
  return sthosvd_host_run(X_hosts, count, dt, dims, N, eps, mode_order, prec, static_cast<cudaStream_t>(stream),
                          out);
}

int tucker_reconstruct(const tucker_result *r, double *Xhat, void *stream) {
  g_err[0] = 0;
  TK_CHECK(check_result(r));
  if (!Xhat) {
    set_error("Xhat is NULL");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  DevBuf hold;
  const double *res = nullptr;
  int64_t cur[TUCKER_MAX_MODES];
  int st = expand_modes(r, -1, Xhat, hold, &res, cur, dev, s, &prof);
  if (st != TUCKER_OK) return st;
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  return TUCKER_OK;
}

int tucker_reconstruct_sub(const tucker_result *r, const int64_t *lo, const int64_t *hi, double *Xsub,
                           void *stream) {
  g_err[0] = 0;
  TK_CHECK(check_result(r));
  if (!Xsub || !lo || !hi) {
    set_error("Xsub, lo and hi must be non-null");
    return TUCKER_EINVAL;
  }
  for (int n = 0; n < r->N; ++n)
    if (lo[n] < 0 || hi[n] <= lo[n] || hi[n] > r->dims[n]) {
      set_error("mode %d: need 0 <= lo < hi <= %lld (got %lld, %lld)", n, (long long)r->dims[n], (long long)lo[n],
                (long long)hi[n]);
      return TUCKER_EINVAL;
    }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  DevBuf hold;
  const double *res = nullptr;
  int64_t cur[TUCKER_MAX_MODES];
  int st = expand_modes(r, -1, Xsub, hold, &res, cur, dev, s, &prof, lo, hi);
  if (st != TUCKER_OK) return st;
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  return TUCKER_OK;
}

int tucker_hooi(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps, int max_iters, double tol,
                tucker_precision prec, void *stream, tucker_result *out, int *iters, double *fit) {
  g_err[0] = 0;
  if (!out || !iters || max_iters < 0 || !(tol >= 0.0)) {
    set_error("tucker_hooi: out and iters must be non-null, max_iters >= 0 and tol >= 0");
    return TUCKER_EINVAL;
  }
  *iters = 0;
  TK_CHECK(tucker_sthosvd(X, dt, dims, N, eps, nullptr, prec, stream, out));
  const int st = hooi_iterate(X, dt, max_iters, tol, prec, static_cast<cudaStream_t>(stream), out, iters, fit);
  if (st != TUCKER_OK) tucker_result_free(out);
  return st;
}

int tucker_sthosvd_batched(const void *const *X, tucker_dtype dt, const int64_t *dims, int N, int count, double eps,
                           tucker_precision prec, int workers, void *stream, tucker_result *out) {
  g_err[0] = 0;
  if (!X || !dims || !out || count < 0 || workers < 0 || workers > 64) {
    set_error("tucker_sthosvd_batched: X, dims and out must be non-null, count >= 0, 0 <= workers <= 64");
    return TUCKER_EINVAL;
  }
  memset(out, 0, sizeof(tucker_result) * (size_t)count);
  if (count == 0) return TUCKER_OK;
  for (int i = 0; i < count; ++i) {
    TK_CHECK(check_dims(dims + (int64_t)i * N, N));
    if (!X[i]) {
      set_error("tensor %d is NULL", i);
      return TUCKER_EINVAL;
    }
  }
  {  // every I_n <= 128: the batched device pipeline (float64), no host round trip between phases
    int handled = 0;
    const int st = sthosvd_batched_device(X, dt, dims, N, count, eps, static_cast<cudaStream_t>(stream), out, &handled);
    if (handled) {
      if (st != TUCKER_OK) {
        const std::string msg = tucker_last_error();
        for (int i = 0; i < count; ++i) tucker_result_free(&out[i]);
        set_error("%s", msg.c_str());
      }
      return st;
    }
  }
  if (workers == 0) workers = 8;
  workers = std::min(workers, count);
  int device = 0;
  TK_CUDA(cudaGetDevice(&device));
  // the workers' streams start after everything already queued on `stream`
  cudaEvent_t ready;
  TK_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  TK_CUDA(cudaEventRecord(ready, static_cast<cudaStream_t>(stream)));
  std::atomic<int> next{0};
  std::atomic<int> status{TUCKER_OK};
  std::mutex mu;
  std::string first_err;
  auto work = [&]() {
    cudaStream_t s = nullptr;
    int st = cudaSetDevice(device) == cudaSuccess && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
                     cudaStreamWaitEvent(s, ready, 0) == cudaSuccess
                 ? TUCKER_OK
                 : TUCKER_ECUDA;
    if (st != TUCKER_OK) set_error("tucker_sthosvd_batched: worker stream setup failed");
    while (st == TUCKER_OK && status.load() == TUCKER_OK) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      st = tucker_sthosvd(X[i], dt, dims + (int64_t)i * N, N, eps, nullptr, prec, s, &out[i]);
      if (st != TUCKER_OK) {
        const std::string msg = std::string("tensor ") + std::to_string(i) + ": " + tucker_last_error();
        std::lock_guard<std::mutex> lk(mu);
        if (status.load() == TUCKER_OK) {
          first_err = msg;
          status.store(st);
        }
      }
    }
    if (st != TUCKER_OK && status.load() == TUCKER_OK) {
      std::lock_guard<std::mutex> lk(mu);
      if (status.load() == TUCKER_OK) {
        first_err = tucker_last_error();
        status.store(st);
      }
    }
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  };
  std::vector<std::thread> pool;
  pool.reserve((size_t)workers);
  for (int w = 0; w < workers; ++w) pool.emplace_back(work);
  for (auto &t : pool) t.join();
  cudaEventDestroy(ready);
  if (status.load() != TUCKER_OK) {
    for (int i = 0; i < count; ++i) tucker_result_free(&out[i]);
    set_error("%s", first_err.c_str());
    return status.load();
  }
  return TUCKER_OK;
}

int tucker_order_flops(const int64_t *dims, const int64_t *ranks, int N, const int *order, double *flops) {
  g_err[0] = 0;
  int ord[TUCKER_MAX_MODES];
  if (!ranks || !flops) {
    set_error("tucker_order_flops: ranks and flops must be non-null");
    return TUCKER_EINVAL;
  }
  TK_CHECK(check_dims(dims, N));
  TK_CHECK(check_order(order, N, ord));
  for (int n = 0; n < N; ++n)
    if (ranks[n] < 1 || ranks[n] > dims[n]) {
      set_error("rank %d out of [1, I_n]", n);
      return TUCKER_EINVAL;
    }
  *flops = order_flops(dims, ranks, N, ord);
  return TUCKER_OK;
}

int tucker_mode_order(const int64_t *dims, const int64_t *ranks, int N, int rule, int *order) {
  g_err[0] = 0;
  if (!ranks || !order) {
    set_error("tucker_mode_order: ranks and order must be non-null");
    return TUCKER_EINVAL;
  }
  TK_CHECK(check_dims(dims, N));
  for (int n = 0; n < N; ++n)
    if (ranks[n] < 1 || ranks[n] > dims[n]) {
      set_error("rank %d out of [1, I_n]", n);
      return TUCKER_EINVAL;
    }
  if (rule == TUCKER_ORDER_EXHAUSTIVE) {
    if (N > 9) {
      set_error("exhaustive mode order search takes N <= 9 (got %d)", N);
      return TUCKER_EINVAL;
    }
    int perm[TUCKER_MAX_MODES];
    for (int n = 0; n < N; ++n) perm[n] = n;
    double best = 0.0;
    bool have = false;
    do {  // lexicographic: the first of equal-cost orders wins
      const double f = order_flops(dims, ranks, N, perm);
      if (!have || f < best) {
        best = f;
        have = true;
        memcpy(order, perm, sizeof(int) * N);
      }
    } while (std::next_permutation(perm, perm + N));
    return TUCKER_OK;
  }
  if (rule != TUCKER_ORDER_GREEDY_FLOPS && rule != TUCKER_ORDER_GREEDY_RATIO) {
    set_error("unknown mode order rule %d", rule);
    return TUCKER_EINVAL;
  }
  int64_t cur[TUCKER_MAX_MODES];
  bool used[TUCKER_MAX_MODES] = {};
  for (int n = 0; n < N; ++n) cur[n] = dims[n];
  for (int k = 0; k < N; ++k) {
    int pick = -1;
    double key = 0.0;
    for (int n = 0; n < N; ++n) {
      if (used[n]) continue;
      const double v = rule == TUCKER_ORDER_GREEDY_FLOPS ? step_flops(dims, ranks, cur, N, n)
                                                          : -(double)dims[n] / (double)ranks[n];
      if (pick < 0 || v < key) {  // strict: ties keep the lower mode index
        pick = n;
        key = v;
      }
    }
    used[pick] = true;
    order[k] = pick;
    cur[pick] = ranks[pick];
  }
  return TUCKER_OK;
}

int tucker_rel_error(const void *X, tucker_dtype dt, const tucker_result *r, double *rel_out, void *stream) {
  g_err[0] = 0;
  TK_CHECK(check_result(r));
  if (!X || !rel_out || (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("X and rel_out must be non-null and dt valid");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  const int N = r->N;
  // the last (fused) expansion is the mode with the largest growth
  int last = 0;
  for (int n = 1; n < N; ++n)
    if ((double)r->dims[n] / r->ranks[n] >= (double)r->dims[last] / r->ranks[last]) last = n;
  DevBuf hold, scal, partials;
  const double *y = nullptr;
  int64_t cur[TUCKER_MAX_MODES];
  TK_CHECK(expand_modes(r, last, nullptr, hold, &y, cur, dev, s, &prof));
  int64_t L = 1, B = 1, I = 1;
  for (int m = 0; m < last; ++m) L *= cur[m];
  for (int m = last + 1; m < N; ++m) B *= cur[m];
  for (int m = 0; m < N; ++m) I *= r->dims[m];
  const int64_t J = cur[last], K = r->dims[last];
  TK_CHECK(scal.alloc(2 * sizeof(double), s));
  const int64_t np = std::max(norm2_partials(), ttm_diff_partials(L, J, B, K, dev));
  TK_CHECK(partials.alloc(sizeof(double) * np, s));
  TK_CHECK(launch_ttm_diff(y, L, J, B, r->factors[last], 1, K, K, X, dt, partials.as<double>(), scal.as<double>(),
                           dev, s, &prof));
  TK_CHECK(launch_norm2(X, dt, I, partials.as<double>(), scal.as<double>() + 1, s, &prof));
  double h[2];
  TK_CUDA(cudaMemcpyAsync(h, scal.p, sizeof h, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (h[1] == 0.0) *rel_out = (h[0] == 0.0) ? 0.0 : INFINITY;
  else *rel_out = std::sqrt(h[0] / h[1]);
  return TUCKER_OK;
}

void tucker_result_free(tucker_result *r) {
  if (!r) return;
  free_result_device(r);
  for (int n = 0; n < TUCKER_MAX_MODES; ++n) {
    free(r->eigvals[n]);
    r->eigvals[n] = nullptr;
  }
  delete static_cast<Priv *>(r->priv);
  memset(r, 0, sizeof *r);
}

int tucker_norm2(const void *X, tucker_dtype dt, int64_t n, double *out, void *stream) {
  g_err[0] = 0;
  if ((!X && n > 0) || !out || n < 0 || (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("invalid arguments to tucker_norm2");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Prof prof(s);
  DevBuf partials, scal;
  TK_CHECK(partials.alloc(sizeof(double) * norm2_partials(), s));
  TK_CHECK(scal.alloc(sizeof(double), s));
  TK_CHECK(launch_norm2(X, dt, n, partials.as<double>(), scal.as<double>(), s, &prof));
  TK_CUDA(cudaMemcpyAsync(out, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  return TUCKER_OK;
}

int tucker_gram(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S, void *stream) {
  g_err[0] = 0;
  if (!Y || !S || L < 1 || B < 1 || J < 1 || J > TUCKER_MAX_DIM || (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("invalid arguments to tucker_gram");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  DevBuf ws;
  TK_CHECK(ws.alloc(sizeof(double) * gram_workspace_doubles(L, J, B, dev), s));
  TK_CHECK(launch_gram(Y, dt, L, J, B, S, ws.as<double>(), dev, s, &prof));
  if (prof.on) {
    TK_CUDA(cudaStreamSynchronize(s));
    prof.flush();
  }
  return TUCKER_OK;
}

static int gram_split_entry(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S, void *stream,
                            bool f8);

int tucker_gram_split(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S, void *stream) {
  return gram_split_entry(Y, dt, L, J, B, S, stream, false);
}

int tucker_gram_split_e4m3(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S,
                           void *stream) {
  return gram_split_entry(Y, dt, L, J, B, S, stream, true);
}

static int gram_split_entry(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S, void *stream,
                            bool f8) {
  g_err[0] = 0;
  if (!Y || !S || L < 1 || B < 1 || J < 1 || (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("invalid arguments to tucker_gram_split");
    return TUCKER_EINVAL;
  }
  if (J > (f8 ? 128 : 512)) {
    set_error("tucker_gram_split%s supports J <= %d (got %lld)", f8 ? "_e4m3" : "", f8 ? 128 : 512, (long long)J);
    return TUCKER_EUNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  DevBuf ws;
  TK_CHECK(ws.alloc(sizeof(double) * gram_split_workspace_doubles(L, J, B, dev, dt, Y), s));
  TK_CHECK(launch_gram_split(Y, dt, L, J, B, S, ws.as<double>(), dev, s, &prof, nullptr, f8));
  int herr = 0;
  TK_CHECK(gram_split_error(ws.as<double>(), L, J, B, dev, &herr, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (herr) {
    set_error("tucker_gram_split: a bounded tensor-core wait expired");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

int tucker_ttm_split(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *U, int64_t R,
                     double *Z, void *stream) {
  g_err[0] = 0;
  if (!Y || !U || !Z || L < 1 || B < 1 || J < 1 || R < 1 || (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("invalid arguments to tucker_ttm_split");
    return TUCKER_EINVAL;
  }
  if (J > 512 || R > J || R > 128) {
    set_error("tucker_ttm_split supports R <= J <= 512 with R <= 128 (got J = %lld, R = %lld)", (long long)J,
              (long long)R);
    return TUCKER_EUNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  DevBuf e;
  TK_CHECK(e.alloc(sizeof(int), s));
  TK_CUDA(cudaMemsetAsync(e.p, 0, sizeof(int), s));
  TK_CHECK(launch_ttm_split(Y, dt, L, J, B, U, R, Z, e.as<int>(), dev, s, &prof));
  int herr = 0;
  TK_CUDA(cudaMemcpyAsync(&herr, e.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (herr) {
    set_error("tucker_ttm_split: a bounded tensor-core wait expired");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

int tucker_eig(const double *S, int64_t J, double *lam, double *V, int *sweeps, void *stream) {
  g_err[0] = 0;
  if (!S || !lam || !V || J < 1 || J > TUCKER_MAX_DIM) {
    set_error("invalid arguments to tucker_eig");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Prof prof(s);
  DevBuf ws, info;
  const int64_t ews = eig_workspace_doubles(J);
  if (ews > 0) TK_CHECK(ws.alloc(sizeof(double) * ews, s));
  TK_CHECK(info.alloc(4 * sizeof(int), s));
  TK_CHECK(launch_eig(S, J, lam, V, ews > 0 ? ws.as<double>() : nullptr, info.as<int>(), s, &prof));
  int h[2];
  TK_CUDA(cudaMemcpyAsync(h, info.p, sizeof h, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  if (sweeps) *sweeps = h[0];
  if (h[1] != 0) {
    set_error("Jacobi eigensolver did not converge within %d sweeps", h[0]);
    return TUCKER_ENOCONV;
  }
  return TUCKER_OK;
}

int tucker_rank_cut(const double *lam, int64_t J, double threshold, int keep_all, int64_t *R, double *tail,
                    void *stream) {
  g_err[0] = 0;
  if (!lam || !R || !tail || J < 1 || J > TUCKER_MAX_DIM || std::isnan(threshold)) {
    set_error("invalid arguments to tucker_rank_cut");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Prof prof(s);
  DevBuf buf;
  TK_CHECK(buf.alloc(2 * sizeof(double), s));
  TK_CHECK(launch_rank_cut(lam, J, threshold, keep_all, reinterpret_cast<int64_t *>(buf.as<double>()),
                           buf.as<double>() + 1, s, &prof));
  double h[2];
  TK_CUDA(cudaMemcpyAsync(h, buf.p, sizeof h, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  prof.flush();
  memcpy(R, h, sizeof *R);
  *tail = h[1];
  return TUCKER_OK;
}

int tucker_ttm(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *M, int64_t K,
               int trans_m, double *Z, void *stream) {
  g_err[0] = 0;
  if (!Y || !M || !Z || L < 1 || B < 1 || J < 1 || K < 1 || J > TUCKER_MAX_DIM || K > TUCKER_MAX_DIM ||
      (dt != TUCKER_F64 && dt != TUCKER_F32)) {
    set_error("invalid arguments to tucker_ttm");
    return TUCKER_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  TK_CHECK(device_info(&dev));
  Prof prof(s);
  const int64_t ak = trans_m ? J : 1, aj = trans_m ? 1 : K;
  TK_CHECK(launch_ttm(Y, dt, L, J, B, M, ak, aj, K, Z, dev, s, &prof));
  if (prof.on) {
    TK_CUDA(cudaStreamSynchronize(s));
    prof.flush();
  }
  return TUCKER_OK;
}

}  // extern "C"
