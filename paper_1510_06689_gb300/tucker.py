"""ctypes binding of the C ABI in ``include/tucker.h`` (argument marshalling only).

Every computation happens in the CUDA library ``libtucker_gb300.so``; this
module converts torch tensors to pointers and sizes, passes the caller's
current CUDA stream, and turns status codes into exceptions.  If the library
has not been built, ``load()`` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

MAX_MODES = 16
HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtucker_gb300.so")

F64, F32 = 0, 1
PREC = {"fp64": 0, "bf16x4": 1, "e4m3x4": 2}
PHASES = ("norm", "gram", "gram_reduce", "eig", "rank", "ttm", "scale", "ttm_l1")

# Every symbol include/tucker.h declares (checked by the CPU test suite).
EXPORTS = (
    "tucker_sthosvd", "tucker_sthosvd_host", "tucker_reconstruct", "tucker_reconstruct_sub", "tucker_rel_error",
    "tucker_result_free",
    "tucker_norm2", "tucker_gram", "tucker_eig", "tucker_rank_cut", "tucker_ttm", "tucker_status_string",
    "tucker_last_error", "tucker_launch_count", "tucker_profile_enable", "tucker_profile_read",
    "tucker_gram_noalloc", "tucker_gram_split", "tucker_ttm_split", "tucker_hooi", "tucker_order_flops",
    "tucker_mode_order", "tucker_sthosvd_batched", "tucker_fp64_peak", "tucker_gram_split_e4m3",
    "tucker_batched_tuning", "tucker_memory_stats", "tucker_memory_trim", "tucker_sthosvd_host_many",
)
EIG_PATHS = ("mixed", "jacobi", "jacobi_fallback")
ORDER_RULES = {"flops": 0, "ratio": 1, "exhaustive": 2}


class TuckerError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


class _Result(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int),
        ("on_host", ctypes.c_int),
        ("dims", ctypes.c_int64 * MAX_MODES),
        ("ranks", ctypes.c_int64 * MAX_MODES),
        ("mode_order", ctypes.c_int * MAX_MODES),
        ("sweeps", ctypes.c_int * MAX_MODES),
        ("core", ctypes.c_void_p),
        ("factors", ctypes.c_void_p * MAX_MODES),
        ("eigvals", ctypes.POINTER(ctypes.c_double) * MAX_MODES),
        ("tail", ctypes.c_double * MAX_MODES),
        ("norm2_x", ctypes.c_double),
        ("threshold", ctypes.c_double),
        ("eig_path", ctypes.c_int * MAX_MODES),
        ("eig_resolved", ctypes.c_int * MAX_MODES),
        ("priv", ctypes.c_void_p),
    ]


class _Profile(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_double * len(PHASES)),
        ("launches", ctypes.c_int64 * len(PHASES)),
        ("flops", ctypes.c_double * len(PHASES)),
        ("bytes", ctypes.c_double * len(PHASES)),
    ]


_lib = None


def load(path=LIB_PATH):
    """Load the CUDA library (raises if it is missing: build it with ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} not built; run paper_1510_06689_gb300.build.build()")
    lib = ctypes.CDLL(path)
    i64, vp, i32, dbl = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pi64, pdbl, pi32 = ctypes.POINTER(i64), ctypes.POINTER(dbl), ctypes.POINTER(i32)
    pres = ctypes.POINTER(_Result)
    sig = {
        "tucker_sthosvd": (i32, [vp, i32, pi64, i32, dbl, pi32, i32, vp, pres]),
        "tucker_sthosvd_host": (i32, [vp, i32, pi64, i32, dbl, pi32, i32, vp, pres]),
        "tucker_sthosvd_host_many": (i32, [ctypes.POINTER(vp), i32, i32, pi64, i32, dbl, pi32, i32, vp, pres]),
        "tucker_reconstruct": (i32, [pres, vp, vp]),
        "tucker_reconstruct_sub": (i32, [pres, pi64, pi64, vp, vp]),
        "tucker_hooi": (i32, [vp, i32, pi64, i32, dbl, i32, dbl, i32, vp, pres, pi32, pdbl]),
        "tucker_order_flops": (i32, [pi64, pi64, i32, pi32, pdbl]),
        "tucker_sthosvd_batched": (i32, [ctypes.POINTER(vp), i32, pi64, i32, i32, dbl, i32, i32, vp, pres]),
        "tucker_mode_order": (i32, [pi64, pi64, i32, i32, pi32]),
        "tucker_rel_error": (i32, [vp, i32, pres, pdbl, vp]),
        "tucker_result_free": (None, [pres]),
        "tucker_norm2": (i32, [vp, i32, i64, pdbl, vp]),
        "tucker_gram": (i32, [vp, i32, i64, i64, i64, vp, vp]),
        "tucker_eig": (i32, [vp, i64, vp, vp, pi32, vp]),
        "tucker_rank_cut": (i32, [vp, i64, dbl, i32, pi64, pdbl, vp]),
        "tucker_ttm": (i32, [vp, i32, i64, i64, i64, vp, i64, i32, vp, vp]),
        "tucker_gram_noalloc": (i32, [vp, i32, i64, i64, i64, vp, vp]),
        "tucker_gram_split": (i32, [vp, i32, i64, i64, i64, vp, vp]),
        "tucker_gram_split_e4m3": (i32, [vp, i32, i64, i64, i64, vp, vp]),
        "tucker_ttm_split": (i32, [vp, i32, i64, i64, i64, vp, i64, vp, vp]),
        "tucker_status_string": (ctypes.c_char_p, [i32]),
        "tucker_last_error": (ctypes.c_char_p, []),
        "tucker_launch_count": (i64, []),
        "tucker_profile_enable": (None, [i32]),
        "tucker_profile_read": (None, [ctypes.POINTER(_Profile)]),
        "tucker_fp64_peak": (i32, [pdbl, pdbl, vp]),
        "tucker_batched_tuning": (None, [pi64, pi32, ctypes.POINTER(ctypes.c_float)]),
        "tucker_memory_stats": (i32, [pi64, pi64, pi64]),
        "tucker_memory_trim": (i32, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        lib = load()
        msg = lib.tucker_last_error().decode() or lib.tucker_status_string(status).decode()
        raise TuckerError(status, msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t):
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"tensor dtype {t.dtype} not supported (float64 or float32)")


def _dev_ptr(t, what):
    if t.numel() == 0:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class _DevArray:
    """Minimal __cuda_array_interface__ over library-owned device memory."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _copy_out(ptr, n):
    if n == 0 or not ptr:
        return torch.empty(0, dtype=torch.float64, device="cuda")
    return torch.as_tensor(_DevArray(ptr, (n,)), device="cuda").clone()


def _doubles(ptr, count):
    """`count` doubles at a library pointer as a list (one slice, not per-element indexing)."""
    if not ptr or count <= 0:
        return []
    return ptr[:count]


class Result:
    """An ST-HOSVD result (core, factors, ranks, eigenvalues) owned by the library."""

    def __init__(self, raw):
        self._raw = raw
        n = raw.N
        self.N = n
        self.dims = tuple(raw.dims[:n])
        self.ranks = tuple(raw.ranks[:n])
        self.mode_order = tuple(raw.mode_order[:n])
        self.sweeps = tuple(raw.sweeps[:n])
        self.tails = tuple(raw.tail[:n])
        self.norm2 = raw.norm2_x
        self.threshold = raw.threshold
        self.on_host = bool(raw.on_host)
        self._eigvals = None
        self.eig_paths = tuple(EIG_PATHS[p] for p in raw.eig_path[:n])
        self.eig_resolved = tuple(raw.eig_resolved[:n])

    @property
    def eigvals(self):
        """The I_n eigenvalues of each mode's Gram, descending (read from the result on first use)."""
        if self._eigvals is None:
            raw = self._raw
            self._eigvals = [_doubles(raw.eigvals[i], self.dims[i]) if raw is not None else [] for i in range(self.N)]
        return self._eigvals

    @property
    def raw(self):
        return self._raw

    def core(self):
        """Core as a flat float64 tensor (natural layout), copied out of the library."""
        n = math.prod(self.ranks)
        if self.on_host:
            buf = (ctypes.c_double * n).from_address(self._raw.core)
            return torch.frombuffer(buf, dtype=torch.float64).clone()
        return _copy_out(self._raw.core, n)

    def factor(self, n):
        """U_n as an (I_n, R_n) float64 tensor."""
        i, r = self.dims[n], self.ranks[n]
        if self.on_host:
            buf = (ctypes.c_double * (i * r)).from_address(self._raw.factors[n])
            flat = torch.frombuffer(buf, dtype=torch.float64).clone()
        else:
            flat = _copy_out(self._raw.factors[n], i * r)
        return flat.view(r, i).t().contiguous()  # column-major storage

    def factors(self):
        return [self.factor(n) for n in range(self.N)]

    def free(self):
        if self._raw is not None and _lib is not None:
            self.eigvals  # noqa: B018 - read before the library releases them (they stay readable)
            _lib.tucker_result_free(ctypes.byref(self._raw))
        self._raw = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def _dims_arg(dims):
    dims = tuple(int(d) for d in dims)
    return dims, (ctypes.c_int64 * len(dims))(*dims)


def _order_arg(order, n):
    if order is None:
        return None
    order = tuple(int(o) for o in order)
    if len(order) != n:
        raise ValueError("mode_order must have one entry per mode")
    return (ctypes.c_int * n)(*order)


def sthosvd(x, dims, eps, mode_order=None, precision="fp64", stream=None):
    """Algorithm 1 on a device tensor x (flat, natural layout, float64 or float32)."""
    lib = load()
    dims, cd = _dims_arg(dims)
    if x.numel() != math.prod(dims):
        raise ValueError("x.numel() does not match dims")
    raw = _Result()
    _check(lib.tucker_sthosvd(_dev_ptr(x, "x"), _dtype_code(x), cd, len(dims), float(eps),
                              _order_arg(mode_order, len(dims)), PREC[precision], _stream(stream),
                              ctypes.byref(raw)))
    return Result(raw)


def sthosvd_host(x, dims, eps, mode_order=None, precision="fp64", stream=None):
    """Algorithm 1 on a host tensor (pinned recommended); result lives on the host."""
    lib = load()
    dims, cd = _dims_arg(dims)
    if x.is_cuda or not x.is_contiguous() or x.numel() != math.prod(dims):
        raise ValueError("x must be a contiguous host tensor with prod(dims) elements")
    raw = _Result()
    _check(lib.tucker_sthosvd_host(ctypes.c_void_p(x.data_ptr()), _dtype_code(x), cd, len(dims), float(eps),
                                   _order_arg(mode_order, len(dims)), PREC[precision], _stream(stream),
                                   ctypes.byref(raw)))
    return Result(raw)


def sthosvd_host_many(xs, dims, eps, mode_order=None, precision="fp64", stream=None):
    """Algorithm 1 on several host tensors of one shape in turn, the copy of the
    next running while the current one is compressed; results on the host."""
    lib = load()
    dims, cd = _dims_arg(dims)
    if not xs:
        return []
    code = _dtype_code(xs[0])
    for x in xs:
        if x.is_cuda or not x.is_contiguous() or x.numel() != math.prod(dims) or _dtype_code(x) != code:
            raise ValueError("xs must be contiguous host tensors of one dtype with prod(dims) elements each")
    count = len(xs)
    ptrs = (ctypes.c_void_p * count)(*[x.data_ptr() for x in xs])
    raws = (_Result * count)()
    _check(lib.tucker_sthosvd_host_many(ptrs, count, code, cd, len(dims), float(eps),
                                        _order_arg(mode_order, len(dims)), PREC[precision], _stream(stream), raws))
    return [Result(raws[i]) for i in range(count)]


def reconstruct(result, out=None, stream=None):
    """X~ = G x {U_n} as a flat float64 device tensor."""
    lib = load()
    n = math.prod(result.dims)
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(lib.tucker_reconstruct(ctypes.byref(result.raw), _dev_ptr(out, "out"), _stream(stream)))
    return out


def hooi(x, dims, eps, max_iters=10, tol=0.0, precision="fp64", stream=None):
    """Algorithm 2 (HOOI) from Algorithm 1: returns (Result, iterations, fit history)."""
    lib = load()
    dims, cd = _dims_arg(dims)
    if x.numel() != math.prod(dims):
        raise ValueError("x must hold prod(dims) elements")
    raw = _Result()
    iters = ctypes.c_int(0)
    fit = (ctypes.c_double * (int(max_iters) + 1))()
    _check(lib.tucker_hooi(_dev_ptr(x, "x"), _dtype_code(x), cd, len(dims), float(eps), int(max_iters), float(tol),
                           PREC[precision], _stream(stream), ctypes.byref(raw), ctypes.byref(iters), fit))
    return Result(raw), iters.value, list(fit[: iters.value + 1])


def sthosvd_batched(xs, dims_list, eps, precision="fp64", workers=0, stream=None):
    """Algorithm 1 on many independent device tensors of the same order N and dtype."""
    lib = load()
    count = len(xs)
    if count != len(dims_list) or count == 0:
        raise ValueError("one dims tuple per tensor, at least one tensor")
    n = len(dims_list[0])
    if any(len(d) != n for d in dims_list):
        raise ValueError("every tensor needs the same number of modes")
    code = _dtype_code(xs[0])
    addrs = []
    for x, d in zip(xs, dims_list):
        if _dtype_code(x) != code or x.numel() != math.prod(d):
            raise ValueError("tensors need one dtype and prod(dims) elements each")
        addrs.append(_dev_ptr(x, "x").value)
    ptrs = (ctypes.c_void_p * count)(*addrs)
    flat = (ctypes.c_int64 * (count * n))(*[int(v) for d in dims_list for v in d])
    raws = (_Result * count)()
    _check(lib.tucker_sthosvd_batched(ptrs, code, flat, n, count, float(eps), PREC[precision], int(workers),
                                      _stream(stream), raws))
    # each Result views its element of `raws` (the view keeps the array alive)
    return [Result(raws[i]) for i in range(count)]


def order_flops(dims, ranks, order=None):
    """Flops of Algorithm 1 in a mode order (host-only cost model)."""
    lib = load()
    n = len(dims)
    cd, cr = (ctypes.c_int64 * n)(*dims), (ctypes.c_int64 * n)(*ranks)
    out = ctypes.c_double()
    _check(lib.tucker_order_flops(cd, cr, n, _order_arg(order, n), ctypes.byref(out)))
    return out.value


def mode_order(dims, ranks, rule="flops"):
    """A mode order by a heuristic of the paper ("flops", "ratio") or exhaustive search."""
    lib = load()
    n = len(dims)
    cd, cr = (ctypes.c_int64 * n)(*dims), (ctypes.c_int64 * n)(*ranks)
    out = (ctypes.c_int * n)()
    _check(lib.tucker_mode_order(cd, cr, n, ORDER_RULES[rule], out))
    return list(out)


def reconstruct_sub(result, lo, hi, out=None, stream=None):
    """X~[lo_1:hi_1, ..., lo_N:hi_N] (natural layout) from row subsets of the factors."""
    lib = load()
    lo = [int(v) for v in lo]
    hi = [int(v) for v in hi]
    if len(lo) != len(result.dims) or len(hi) != len(result.dims):
        raise ValueError("lo and hi need one index per mode")
    n = math.prod(max(h - l, 0) for l, h in zip(lo, hi))
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    clo, chi = (ctypes.c_int64 * len(lo))(*lo), (ctypes.c_int64 * len(hi))(*hi)
    _check(lib.tucker_reconstruct_sub(ctypes.byref(result.raw), clo, chi, _dev_ptr(out, "out"), _stream(stream)))
    return out[:n]


def rel_error(x, result, stream=None):
    """||X - X~|| / ||X|| with the difference fused into the last expansion."""
    lib = load()
    rel = ctypes.c_double()
    _check(lib.tucker_rel_error(_dev_ptr(x, "x"), _dtype_code(x), ctypes.byref(result.raw), ctypes.byref(rel),
                                _stream(stream)))
    return rel.value


def norm2(x, stream=None):
    lib = load()
    out = ctypes.c_double()
    _check(lib.tucker_norm2(_dev_ptr(x, "x"), _dtype_code(x), x.numel(), ctypes.byref(out), _stream(stream)))
    return out.value


def gram(y, L, J, B, stream=None):
    """S (J x J) of the (L, J, B) view; returned as a (J, J) tensor (symmetric)."""
    lib = load()
    s = torch.empty((J, J), dtype=torch.float64, device="cuda")
    _check(lib.tucker_gram(_dev_ptr(y, "y"), _dtype_code(y), int(L), int(J), int(B), _dev_ptr(s, "S"),
                           _stream(stream)))
    return s.t()  # column-major storage -> logical S


def gram_noalloc(y, L, J, B, out=None, stream=None):
    """Same result as :func:`gram`, computed without any device allocation by the
    library (its split-K scratch is a static device array).  ``out`` (J x J
    float64, caller-allocated) receives S when given."""
    lib = load()
    L, J, B = int(L), int(J), int(B)
    # the C side cannot see a tensor's type or size: a wrong `out` or a short `y`
    # would become an out-of-bounds device access, so they are checked here
    if y.numel() < L * J * B:
        raise TuckerError(-1, f"y holds {y.numel()} elements, the ({L}, {J}, {B}) view needs {L * J * B}")
    if out is not None:
        if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() or out.numel() != J * J:
            raise TuckerError(-1, "out must be a contiguous float64 CUDA tensor of J*J elements")
    s = out if out is not None else torch.empty((J, J), dtype=torch.float64, device="cuda")
    _check(lib.tucker_gram_noalloc(_dev_ptr(y, "y"), _dtype_code(y), int(L), int(J), int(B), _dev_ptr(s, "S"),
                                   _stream(stream)))
    return s.t()


def gram_split(y, L, J, B, stream=None):
    """Split-precision Gram on the tensor cores (J <= 128); same layout as :func:`gram`."""
    lib = load()
    s = torch.empty((J, J), dtype=torch.float64, device="cuda")
    _check(lib.tucker_gram_split(_dev_ptr(y, "y"), _dtype_code(y), int(L), int(J), int(B), _dev_ptr(s, "S"),
                                 _stream(stream)))
    return s.t()


def gram_split_e4m3(y, L, J, B, stream=None):
    """Split-precision Gram from E4M3 digits on the FP8 tensor cores (J <= 128)."""
    lib = load()
    s = torch.empty((J, J), dtype=torch.float64, device="cuda")
    _check(lib.tucker_gram_split_e4m3(_dev_ptr(y, "y"), _dtype_code(y), int(L), int(J), int(B), _dev_ptr(s, "S"),
                                      _stream(stream)))
    return s.t()


def eig(s, stream=None):
    """(lam descending, V with eigenvectors as columns, sweeps) of a symmetric (J, J) tensor."""
    lib = load()
    j = s.shape[0]
    sc = s.t().contiguous()  # column-major
    lam = torch.empty(j, dtype=torch.float64, device="cuda")
    v = torch.empty((j, j), dtype=torch.float64, device="cuda")
    sweeps = ctypes.c_int()
    _check(lib.tucker_eig(_dev_ptr(sc, "S"), j, _dev_ptr(lam, "lam"), _dev_ptr(v, "V"), ctypes.byref(sweeps),
                          _stream(stream)))
    return lam, v.t(), sweeps.value


def rank_cut(lam, threshold, keep_all=False, stream=None):
    lib = load()
    r, tail = ctypes.c_int64(), ctypes.c_double()
    _check(lib.tucker_rank_cut(_dev_ptr(lam, "lam"), lam.numel(), float(threshold), int(bool(keep_all)),
                               ctypes.byref(r), ctypes.byref(tail), _stream(stream)))
    return r.value, tail.value


def ttm(y, L, J, B, m, transpose=False, stream=None):
    """Z(L, K, B) = sum_j M[k, j] Y(L, J, B); m is (K, J), or (J, K) used transposed."""
    lib = load()
    if transpose:
        jj, k = m.shape
    else:
        k, jj = m.shape
    if jj != J:
        raise ValueError("matrix does not match J")
    mc = m.t().contiguous()  # column-major storage of the given matrix
    z = torch.empty(int(L) * k * int(B), dtype=torch.float64, device="cuda")
    _check(lib.tucker_ttm(_dev_ptr(y, "y"), _dtype_code(y), int(L), int(J), int(B), _dev_ptr(mc, "M"), k,
                          int(bool(transpose)), _dev_ptr(z, "Z"), _stream(stream)))
    return z


def ttm_split(y, L, J, B, u, stream=None):
    """Z(L, R, B) = Y x_n U^T on the tensor cores; u is the (J, R) factor."""
    lib = load()
    jj, r = u.shape
    if jj != J:
        raise ValueError("u does not match J")
    uc = u.t().contiguous()  # column-major storage of u
    z = torch.empty(int(L) * r * int(B), dtype=torch.float64, device="cuda")
    _check(lib.tucker_ttm_split(_dev_ptr(y, "y"), _dtype_code(y), int(L), int(J), int(B), _dev_ptr(uc, "U"), r,
                                _dev_ptr(z, "Z"), _stream(stream)))
    return z


def profile_enable(on=True):
    load().tucker_profile_enable(int(bool(on)))


def profile_read():
    p = _Profile()
    load().tucker_profile_read(ctypes.byref(p))
    return {name: {"ms": p.ms[i], "launches": p.launches[i], "flops": p.flops[i], "bytes": p.bytes[i]}
            for i, name in enumerate(PHASES)}


def launch_count():
    return int(load().tucker_launch_count())


def batched_tuning():
    """(columns per work item, persistent CTAs, candidate ms) of the last batched device pipeline."""
    kc, grid = ctypes.c_int64(), ctypes.c_int()
    ms = (ctypes.c_float * 6)()
    load().tucker_batched_tuning(ctypes.byref(kc), ctypes.byref(grid), ms)
    return kc.value, grid.value, list(ms)


def memory_stats():
    """Bytes held between calls: the device pool in use and reserved, and cached pinned host blocks."""
    used, res, host = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().tucker_memory_stats(ctypes.byref(used), ctypes.byref(res), ctypes.byref(host)))
    return {"pool_used": used.value, "pool_reserved": res.value, "host_cached": host.value}


def memory_trim():
    """Return cached pinned host blocks and unused pool memory to the driver (synchronises the device)."""
    _check(load().tucker_memory_trim())


def fp64_peak(stream=None):
    """(TFLOP/s, ms) of the library's float64 fused multiply-add probe on the current GPU."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().tucker_fp64_peak(ctypes.byref(tf), ctypes.byref(ms), _stream(stream)))
    return tf.value, ms.value
