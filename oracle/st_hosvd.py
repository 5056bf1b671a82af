"""Plain, slow CPU oracle for the sequentially-truncated HOSVD, in float64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline leg and ``--impl reference``) may use it.  It shares no code with
the CUDA library.

Every step follows the paper's definitions in the order of Algorithm 1
(ST-HOSVD, Sec. 2.2), written for a reader to check by eye.  Library
routines serve as single steps where the step *is* that routine: a matrix
product for the Gram matrix and the mode-n product, LAPACK's symmetric
eigensolver (``numpy.linalg.eigh``) for "leading eigenvectors of S", as the
paper itself uses LAPACK's ``dsyevx`` there (Sec. 5.4).

Readings of points the paper leaves open:

* Unfolding (Sec. 2.1): the printed column-index formula is garbled (it uses
  I/I_k where prefix products are meant).  We use the standard map
  j = sum_{k != n} i_k prod_{m<k, m != n} I_m (0-based), which is the order in
  which the natural (first-index-fastest) layout of Sec. 4.1 stores the
  columns.
* Rank rule (Algorithm 1, Sec. 7.2): R_n is the smallest R in [1, I_n] with
  sum_{r>R} lambda_r <= eps^2 ||X||^2 / N, where ||X|| is the norm of the
  *original* tensor, negative eigenvalues (rounding) count as 0, and the tail
  sums are accumulated from the smallest eigenvalue upward.  eps <= 0 keeps
  every index (R_n = I_n).
* Eigenvector sign and tie order: eigenvalues in descending order, ties by
  lower index; each eigenvector is negated if needed so that its entry of
  largest magnitude is positive (ties: lowest row).
* Mode order (Sec. 2.2: "any arbitrary order"): ``order`` is a 0-based
  permutation; the core keeps the original mode positions, and factor n is
  always I_n x R_n.
* Reconstruction (Eq. reconstruct, Sec. 2.3): X~ = G x {U_n}, and the
  normalised RMS error is ||X - X~|| / ||X||, formed from the explicit
  difference.  A subtensor uses the same product with row subsets of the
  factors (Sec. 2.3).
* HOOI (Sec. 2.2; Algorithm 2 is the source): alternating best rank-R_n
  subspaces, each factor the leading left singular subspace of X projected on
  the other factors' latest values; ranks fixed by the ST-HOSVD that starts
  it; the core is X projected on all factors.  The stopping test
  "||X||^2 - ||G||^2 ceases to decrease" is read as: stop after an iteration
  whose decrease is at most tol ||X||^2 (tol = 0: no decrease at all), or
  after max_iters.
* Mode-order flop model (the ST-HOSVD cost of Sec. 6.1 with P = 1): the step on
  mode n, with J the product of the current dimensions, costs
  2 I_n J (Gram) + 2 R_n J (TTM) + 10/3 I_n^3 (eigenvectors); J then shrinks
  by R_n / I_n.  The two heuristics of Sec. 8.3 pick, at each step, the mode
  with the fewest flops in that step, or the largest I_n / R_n (ties: lower
  mode index).

Parity pins for every function here live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "as_tensor",
    "unfold",
    "fold",
    "norm2",
    "gram",
    "leading_eigenpairs",
    "rank_from_eps",
    "ttm",
    "sthosvd",
    "reconstruct",
    "rel_error",
    "reconstruct_sub",
    "hooi",
    "order_flops",
    "greedy_order",
    "best_order",
    "compression_ratio",
]


def as_tensor(x_flat, dims):
    """View a flat natural-layout buffer (first index fastest) as an N-way array."""
    return np.asarray(x_flat, dtype=np.float64).reshape(tuple(dims), order="F")


def unfold(x, n):
    """Mode-n unfolding X_(n) (Sec. 2.1): an I_n x (I / I_n) matrix.

    Column j of X_(n) holds the fibre with the other indices ordered first
    index fastest, i.e. the reading of the index map stated in the module
    docstring.
    """
    x = np.asarray(x)
    return np.moveaxis(x, n, 0).reshape(x.shape[n], -1, order="F")


def fold(m, n, shape):
    """Inverse of :func:`unfold`: rebuild the tensor of ``shape`` from X_(n)."""
    shape = tuple(shape)
    moved = (shape[n],) + shape[:n] + shape[n + 1:]
    return np.moveaxis(np.asarray(m).reshape(moved, order="F"), 0, n)


def norm2(x):
    """||X||^2: the sum of squares of all entries (Sec. 2.1)."""
    v = np.asarray(x, dtype=np.float64).ravel(order="K")
    return float(np.dot(v, v))


def gram(y, n):
    """S = Y_(n) Y_(n)^T (Algorithm 1, Gram step)."""
    yn = unfold(y, n)
    return yn @ yn.T


def leading_eigenpairs(s):
    """All eigenpairs of the symmetric S, sorted descending, sign-normalised.

    Returns (lam, V) with S V = V diag(lam); ties in lam keep the lower index
    first; each column of V has its largest-magnitude entry positive.
    """
    s = np.asarray(s, dtype=np.float64)
    lam, v = np.linalg.eigh(0.5 * (s + s.T))
    order = sorted(range(len(lam)), key=lambda i: (-lam[i], i))
    lam = lam[order]
    v = v[:, order]
    for c in range(v.shape[1]):
        col = v[:, c]
        r = int(np.argmax(np.abs(col)))  # first (lowest) row on ties
        if col[r] < 0:
            v[:, c] = -col
    return lam, v


def rank_from_eps(lam, threshold, keep_all=False):
    """Smallest R in [1, len(lam)] with sum_{r>R} max(lam_r, 0) <= threshold.

    ``lam`` is sorted descending.  Returns (R, tail) where tail is the
    discarded sum for that R.  Tail sums run from the smallest eigenvalue
    upward (Algorithm 1, rank step; Sec. 7.2).
    """
    j = len(lam)
    if keep_all:
        return j, 0.0
    tails = [0.0] * (j + 1)  # tails[R] = sum of lam[R:], clamped at 0
    acc = 0.0
    for r in range(j - 1, -1, -1):
        acc += max(float(lam[r]), 0.0)
        tails[r] = acc
    for r in range(1, j + 1):
        if tails[r] <= threshold:
            return r, tails[r]
    return j, 0.0


def ttm(y, n, m):
    """Mode-n product Y x_n M for M of size K x J_n: (Y x_n M)_(n) = M Y_(n) (Sec. 2.1)."""
    y = np.asarray(y)
    shape = list(y.shape)
    shape[n] = m.shape[0]
    return fold(m @ unfold(y, n), n, shape)


def sthosvd(x_flat, dims, eps, order=None):
    """Algorithm 1 (ST-HOSVD).

    Parameters are a flat natural-layout float64 (or float32, promoted
    exactly) buffer, its dimensions, the relative error target eps and an
    optional 0-based mode order.  Returns a dict with the core (flat natural
    layout), the factors (list of I_n x R_n arrays), the ranks, the per-mode
    eigenvalues and discarded tails, ||X||^2 and the threshold.
    """
    dims = tuple(int(d) for d in dims)
    n_modes = len(dims)
    order = list(range(n_modes)) if order is None else [int(o) for o in order]
    if sorted(order) != list(range(n_modes)):
        raise ValueError("order must be a permutation of the modes")
    x = as_tensor(x_flat, dims)
    nx2 = norm2(x)
    keep_all = not (eps > 0)
    threshold = (eps * eps) * nx2 / n_modes if not keep_all else 0.0

    y = x
    ranks = list(dims)
    factors = [None] * n_modes
    eigvals = [None] * n_modes
    tails = [0.0] * n_modes
    for n in order:
        s = gram(y, n)
        lam, v = leading_eigenpairs(s)
        r, tail = rank_from_eps(lam, threshold, keep_all)
        u = v[:, :r].copy()
        y = ttm(y, n, u.T)
        ranks[n] = r
        factors[n] = u
        eigvals[n] = lam
        tails[n] = tail
    core = np.asarray(y).ravel(order="F").copy()
    return {
        "core": core,
        "factors": factors,
        "ranks": tuple(ranks),
        "eigvals": eigvals,
        "tails": tails,
        "norm2": nx2,
        "threshold": threshold,
        "order": tuple(order),
        "dims": dims,
    }


def reconstruct(core_flat, ranks, factors):
    """X~ = G x {U_n} (Eq. reconstruct, Sec. 2.3), flat natural layout."""
    g = as_tensor(core_flat, ranks)
    for n, u in enumerate(factors):
        g = ttm(g, n, u)
    return np.asarray(g).ravel(order="F")


def rel_error(x_flat, core_flat, ranks, factors):
    """||X - X~|| / ||X|| from the explicit difference (Sec. 7.2, normalised RMS error)."""
    x = np.asarray(x_flat, dtype=np.float64).ravel()
    d = x - reconstruct(core_flat, ranks, factors)
    nx2 = float(np.dot(x, x))
    if nx2 == 0.0:
        return 0.0 if not d.any() else math.inf
    return math.sqrt(float(np.dot(d, d)) / nx2)


def reconstruct_sub(core_flat, ranks, factors, lo, hi):
    """X~[lo_1:hi_1, ..., lo_N:hi_N] = G x {U_n[lo_n:hi_n, :]} (Sec. 2.3), flat natural layout."""
    g = as_tensor(core_flat, ranks)
    for n, u in enumerate(factors):
        g = ttm(g, n, np.asarray(u)[int(lo[n]):int(hi[n]), :])
    return np.asarray(g).ravel(order="F")


def _project(x, factors, skip=None):
    """X x_m U_m^T over every mode m except `skip` (Sec. 2.1 mode products)."""
    y = x
    for m, u in enumerate(factors):
        if m != skip:
            y = ttm(y, m, u.T)
    return y


def hooi(x_flat, dims, eps, max_iters=10, tol=0.0, order=None):
    """HOOI (Sec. 2.2, Algorithm 2), started from Algorithm 1 with the same eps.

    HOOI maximises ||G|| = ||X x_1 U_1^T ... x_N U_N^T|| over factors with
    orthonormal columns, one factor at a time.  With every other factor
    fixed, the best U_n is the leading R_n-dimensional left singular subspace
    of W_(n), W = X x_{m != n} U_m^T, i.e. the leading eigenvectors of the
    Gram W_(n) W_(n)^T.  One iteration updates U_1, ..., U_N in turn, each
    against the others' latest values; the core for the final factors is the
    projection G = X x {U_m^T}.  Since ||X - X~||^2 = ||X||^2 - ||G||^2 for
    orthonormal factors, the fit ||X||^2 - ||G||^2 never increases.

    Returns the ST-HOSVD dict updated with the refined core and factors, the
    fit history ||X||^2 - ||G||^2 (one value for the start and one per
    iteration) and the number of iterations run.
    """
    res = sthosvd(x_flat, dims, eps, order)
    dims = res["dims"]
    n_modes = len(dims)
    ranks = res["ranks"]
    x = as_tensor(x_flat, dims)
    nx2 = res["norm2"]
    factors = [u.copy() for u in res["factors"]]
    history = [nx2 - norm2(as_tensor(res["core"], ranks))]
    iters = 0
    for _ in range(max_iters):
        for n in range(n_modes):
            w = _project(x, factors, skip=n)
            _, v = leading_eigenpairs(gram(w, n))
            factors[n] = v[:, : ranks[n]].copy()
        core = _project(x, factors)
        iters += 1
        history.append(nx2 - norm2(core))
        if history[-2] - history[-1] <= tol * nx2:
            break
    out = dict(res)
    out["factors"] = factors
    if iters:
        out["core"] = np.asarray(core).ravel(order="F").copy()
    out["history"] = history
    out["iters"] = iters
    return out


def order_flops(dims, ranks, order):
    """Flops of Algorithm 1 in the given mode order (Sec. 6.1 cost model, P = 1)."""
    cur = [int(d) for d in dims]
    total = 0.0
    for n in order:
        j = math.prod(cur)
        total += 2.0 * dims[n] * j + 2.0 * ranks[n] * j + 10.0 / 3.0 * float(dims[n]) ** 3
        cur[n] = int(ranks[n])
    return total


def greedy_order(dims, ranks, rule):
    """The mode orders of the Sec. 8.3 heuristics: rule "flops" or "ratio"."""
    left = list(range(len(dims)))
    cur = [int(d) for d in dims]
    order = []
    while left:
        if rule == "flops":
            j = math.prod(cur)
            cost = {n: 2.0 * dims[n] * j + 2.0 * ranks[n] * j + 10.0 / 3.0 * float(dims[n]) ** 3 for n in left}
            pick = min(left, key=lambda n: (cost[n], n))
        elif rule == "ratio":
            pick = min(left, key=lambda n: (-dims[n] / ranks[n], n))
        else:
            raise ValueError("rule must be 'flops' or 'ratio'")
        order.append(pick)
        left.remove(pick)
        cur[pick] = int(ranks[pick])
    return order


def best_order(dims, ranks):
    """The order of fewest flops by trying every permutation (ties: lexicographically first)."""
    best = None
    for perm in itertools.permutations(range(len(dims))):
        f = order_flops(dims, ranks, perm)
        if best is None or f < best[0]:
            best = (f, list(perm))
    return best[1]


def compression_ratio(dims, ranks):
    """C = prod I_n / (prod R_n + sum I_n R_n) (Sec. 7.2)."""
    return math.prod(dims) / (math.prod(ranks) + sum(i * r for i, r in zip(dims, ranks)))
