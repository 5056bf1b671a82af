"""Seeded synthetic inputs for the ST-HOSVD tests and benchmarks.

This module only *builds inputs*: a dense tensor in Tucker form plus
Gaussian noise, shaped like the combustion workloads of Sec. 7 (space x
space x space x variables x time, per-variable normalised so entries are
roughly N(0,1) scale, Sec. 7.1).  It holds none of the compression method's
arithmetic: no Gram matrices, eigensolves, rank cuts or truncations.  Both
the CUDA path and the CPU oracle consume the arrays it returns; neither
imports the other.

Layout convention (used everywhere in this repository): a tensor of
dimensions (I_1, ..., I_N) is stored flat in *natural layout*, first index
fastest (the column-major mode-1 unfolding of Sec. 4.1).  In numpy that is
``X.ravel(order="F")``; in torch it is a contiguous tensor whose shape is the
reversed dimension tuple.

Recipe (the readings of the workload descriptions are stated here once):

* core G of size R_1 x ... x R_N with i.i.d. N(0,1) entries, optionally
  multiplied by exp(-decay * (i_1 + ... + i_N)) with 0-based indices;
* factor U_n = Q of the Householder QR of an I_n x R_n i.i.d. N(0,1) matrix
  (diag(R) > 0), optionally smoothed first along its row (grid) index by a
  centred 5-point moving average over the in-range neighbours;
* X_clean = G x_1 U_1 ... x_N U_N (the Tucker form of Sec. 2.2);
* noise E i.i.d. N(0,1), rescaled so that ||E|| = noise * ||X_clean||;
* X = X_clean + E, optionally rounded to float32.

Two back ends draw the numbers: numpy (``default_rng([seed, tensor, array])``)
for host arrays of test size, and torch on a CUDA device for the
tens-of-gigabyte workloads.  They use different streams, so the same seed
gives different (equally distributed) tensors on the two back ends.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "tucker_tensor_np",
    "tucker_tensor_torch",
    "tucker_prefix_np",
    "random_dims_ranks",
]

# Array ids inside one tensor's random stream.
_CORE, _NOISE = 1, 2
_FACTOR0 = 100


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: shape, generating ranks, noise and eps values."""

    name: str
    dims: tuple
    ranks: tuple
    decay: float
    smooth: bool
    noise: float
    eps: tuple
    dtype: str = "f64"
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def numel(self) -> int:
        return math.prod(self.dims)

    @property
    def nbytes(self) -> int:
        return self.numel * (8 if self.dtype == "f64" else 4)


WORKLOADS = {
    # 3-way 64^3, core 8^3 N(0,1), noise 1e-4, eps 1e-3, order 1,2,3.
    "cube64": Workload("cube64", (64, 64, 64), (8, 8, 8), 0.0, False, 1e-4, (1e-3,)),
    # 5-way combustion-shaped 128^3 x 48 x 32 (25.8 GB), decaying core.
    "combustion5": Workload(
        "combustion5", (128, 128, 128, 48, 32), (40, 40, 40, 20, 10), 0.15, True, 1e-6, (1e-5, 1e-3)
    ),
    # Same generator at 96^3 x 32 x 24 stored in float32.
    "combustion5_f32": Workload(
        "combustion5_f32", (96, 96, 96, 32, 24), (40, 40, 40, 20, 10), 0.15, True, 1e-6, (1e-4,), "f32"
    ),
    # 4-way 512^2 x 256 x 64 (34.4 GB).
    "large4": Workload("large4", (512, 512, 256, 64), (64, 64, 48, 16), 0.15, True, 1e-6, (1e-4,)),
}


def _smooth_rows(a: np.ndarray) -> np.ndarray:
    """Centred 5-point moving average along axis 0, truncated at the ends."""
    n = a.shape[0]
    out = np.empty_like(a)
    for i in range(n):
        lo, hi = max(0, i - 2), min(n, i + 3)
        out[i] = a[lo:hi].mean(axis=0)
    return out


def _qr_positive(a: np.ndarray) -> np.ndarray:
    q, r = np.linalg.qr(a)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def _decay_weights(ranks, decay: float) -> np.ndarray:
    """exp(-decay * sum of 0-based indices), natural layout, shape ranks (F order)."""
    w = np.ones(1)
    for r in ranks:  # first index fastest
        w = np.concatenate([w * math.exp(-decay * i) for i in range(r)])
    return w


def _rng(seed: int, tensor: int, array: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tensor), int(array)])


def _factors_np(dims, ranks, seed, tensor, smooth):
    us = []
    for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
        g = _rng(seed, tensor, _FACTOR0 + n).standard_normal((i_n, r_n))
        if smooth:
            g = _smooth_rows(g)
        us.append(_qr_positive(g))
    return us


def _expand_np(core_flat: np.ndarray, ranks, factors) -> np.ndarray:
    """G x {U_n} with numpy matmuls on the flat natural layout.

    Mode n views the buffer as the C-ordered array (B, R_n, L) (L = product of
    the earlier dimensions, B of the later ones) and multiplies by U_n on the
    left; the modes with the smallest growth go first.
    """
    cur = list(ranks)
    t = np.asarray(core_flat, dtype=np.float64)
    for n in sorted(range(len(cur)), key=lambda m: factors[m].shape[0] / cur[m]):
        u = factors[n]
        lo, hi = math.prod(cur[:n]), math.prod(cur[n + 1:])
        if lo == 1:
            t = (t.reshape(hi, cur[n]) @ u.T).reshape(-1)
        elif hi == 1:
            t = (u @ t.reshape(cur[n], lo)).reshape(-1)
        else:
            t = np.matmul(u, t.reshape(hi, cur[n], lo)).reshape(-1)
        cur[n] = u.shape[0]
    return t


def tucker_tensor_np(dims, ranks, seed=0, *, decay=0.0, smooth=False, noise=0.0, tensor=0,
                     dtype="f64", return_parts=False):
    """Host tensor in Tucker form plus noise, flat natural layout (float64 or float32).

    With ``return_parts`` also returns (core_flat, factors, X_clean_flat).
    """
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    if len(dims) != len(ranks) or any(r > d or r < 1 for d, r in zip(dims, ranks)):
        raise ValueError("need 1 <= ranks[n] <= dims[n]")
    core = _rng(seed, tensor, _CORE).standard_normal(math.prod(ranks))
    if decay:
        core = core * _decay_weights(ranks, decay)
    us = _factors_np(dims, ranks, seed, tensor, smooth)
    clean = _expand_np(core, ranks, us)
    x = clean.copy()
    if noise:
        e = _rng(seed, tensor, _NOISE).standard_normal(x.size)
        e *= noise * np.linalg.norm(clean) / np.linalg.norm(e)
        x += e
    if dtype == "f32":
        x = x.astype(np.float32)
    if return_parts:
        return x, (core, us, clean)
    return x


def tucker_tensor_torch(dims, ranks, seed=0, *, decay=0.0, smooth=False, noise=0.0, tensor=0,
                        dtype="f64", device="cuda", chunk=1 << 27):
    """Device tensor in Tucker form plus noise, flat natural layout.

    Same recipe as :func:`tucker_tensor_np`; factors and core are drawn on the
    host with numpy (they are small), the expansion and the noise run on the
    device with torch so that tensors of tens of GB are built in seconds.
    Returns a 1-D contiguous torch tensor of prod(dims) elements.
    """
    import torch

    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    core = _rng(seed, tensor, _CORE).standard_normal(math.prod(ranks))
    if decay:
        core = core * _decay_weights(ranks, decay)
    us = _factors_np(dims, ranks, seed, tensor, smooth)
    cur = list(ranks)
    t = torch.from_numpy(core).to(device)
    # Expand the modes with the smallest growth first so the big buffer is made once.
    for n in sorted(range(len(dims)), key=lambda m: dims[m] / ranks[m]):
        lo = math.prod(cur[:n])
        hi = math.prod(cur[n + 1:])
        u = torch.from_numpy(us[n]).to(device)
        t3 = t.view(hi, cur[n], lo)
        t = torch.matmul(u, t3).reshape(-1)  # (hi, I_n, lo): natural layout
        del t3
        cur[n] = dims[n]
    x = t
    if noise:
        g = torch.Generator(device=device)
        norm_clean = float(torch.linalg.vector_norm(x))
        sq = 0.0
        for k, off in enumerate(range(0, x.numel(), chunk)):
            g.manual_seed(int(seed) * 1000003 + int(tensor) * 7919 + k)
            e = torch.randn(min(chunk, x.numel() - off), generator=g, device=device, dtype=torch.float64)
            sq += float(torch.dot(e, e))
        scale = noise * norm_clean / math.sqrt(sq)
        for k, off in enumerate(range(0, x.numel(), chunk)):
            g.manual_seed(int(seed) * 1000003 + int(tensor) * 7919 + k)
            e = torch.randn(min(chunk, x.numel() - off), generator=g, device=device, dtype=torch.float64)
            x[off:off + e.numel()].add_(e, alpha=scale)
            del e
    if dtype == "f32":
        x = x.to(torch.float32)
    return x


def tucker_prefix_np(dims, ranks, slices, seed=0, *, decay=0.0, smooth=False, noise=0.0, tensor=0):
    """The first ``slices`` indices of the last mode of the workload ``dims``.

    Because the last mode is the slowest in natural layout, this is a
    contiguous prefix of the full tensor's buffer: the same core and factors
    (the last factor's leading rows), with i.i.d. noise at the full tensor's
    per-entry scale noise * ||X_clean|| / sqrt(prod(dims)), where
    ||X_clean|| = ||G|| since the factors are orthonormal.  Used for bounded
    CPU samples of workloads too large for the host oracle.
    """
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    core = _rng(seed, tensor, _CORE).standard_normal(math.prod(ranks))
    if decay:
        core = core * _decay_weights(ranks, decay)
    us = _factors_np(dims, ranks, seed, tensor, smooth)
    us[-1] = us[-1][:slices]
    x = _expand_np(core, ranks, us)
    if noise:
        scale = noise * float(np.linalg.norm(core)) / math.sqrt(math.prod(dims))
        x += scale * _rng(seed, tensor, _NOISE).standard_normal(x.size)
    return x, dims[:-1] + (int(slices),)


def random_dims_ranks(count, seed=0, dim_range=(16, 128), rank_range=(4, 16), n_modes=3):
    """Per-tensor dims and ranks for the batched workload (inclusive uniform integer draws)."""
    rng = _rng(seed, 0, 9)
    dims = rng.integers(dim_range[0], dim_range[1] + 1, size=(count, n_modes))
    ranks = rng.integers(rank_range[0], rank_range[1] + 1, size=(count, n_modes))
    ranks = np.minimum(ranks, dims)
    return [tuple(map(int, d)) for d in dims], [tuple(map(int, r)) for r in ranks]
