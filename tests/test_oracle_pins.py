"""Pins for the CPU oracle, against facts fixed by the paper and the mathematics.

None of these checks re-runs the oracle's own formula: they use brute force
over the printed index map, LAPACK's SVD (a different routine from the
oracle's eigensolver), closed forms, the paper's printed Table 2, and
invariants of ST-HOSVD.  ``test_planted_mistakes_are_caught`` plants
plausible mistakes in the oracle and checks that some pin fails.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import st_hosvd as osth
from synthetic import tucker_tensor_np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# brute-force helpers (pure Python loops over the unfolding's index map)
# ----------------------------------------------------------------------------

def _flat_index(idx, dims):
    """Natural layout (first index fastest)."""
    off, stride = 0, 1
    for i, d in zip(idx, dims):
        off += i * stride
        stride *= d
    return off


def _column_index(idx, dims, n):
    """Column of X_(n) holding element idx: j = sum_{k!=n} i_k prod_{m<k, m!=n} I_m (0-based)."""
    j, stride = 0, 1
    for k, (i, d) in enumerate(zip(idx, dims)):
        if k == n:
            continue
        j += i * stride
        stride *= d
    return j


def brute_unfold(x_flat, dims, n):
    cols = math.prod(dims) // dims[n]
    m = np.zeros((dims[n], cols))
    for idx in itertools.product(*[range(d) for d in dims]):
        m[idx[n], _column_index(idx, dims, n)] = x_flat[_flat_index(idx, dims)]
    return m


def brute_ttm(y_flat, dims, n, mat):
    """Z = Y x_n M by explicit loops: Z[.., k, ..] = sum_i M[k, i] Y[.., i, ..]."""
    out_dims = list(dims)
    out_dims[n] = mat.shape[0]
    z = np.zeros(math.prod(out_dims))
    for idx in itertools.product(*[range(d) for d in out_dims]):
        acc = 0.0
        for i in range(dims[n]):
            src = list(idx)
            src[n] = i
            acc += mat[idx[n], i] * y_flat[_flat_index(src, dims)]
        z[_flat_index(idx, out_dims)] = acc
    return z, tuple(out_dims)


def principal_sines(a, b):
    """Sines of the principal angles between span(a) and span(b) (orthonormal columns).

    Taken from the part of b outside span(a), which keeps small angles
    accurate (1 - cos^2 would lose them below sqrt(u)).
    """
    return np.linalg.svd(b - a @ (a.T @ b), compute_uv=False)


def svd_factor(m, r):
    """Leading r left singular vectors of m via LAPACK's SVD, with the sign rule."""
    u, sv, _ = np.linalg.svd(m, full_matrices=False)
    u = u[:, :r].copy()
    for c in range(r):
        k = int(np.argmax(np.abs(u[:, c])))
        if u[k, c] < 0:
            u[:, c] *= -1
    return u, sv


# ----------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------

TINY = [(3, 4, 5), (2, 3, 4, 5), (5, 1, 3), (1, 1, 7), (4, 6)]


@pytest.mark.parametrize("dims", TINY)
def test_unfold_matches_index_map(dims):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(math.prod(dims))
    t = oracle.as_tensor(x, dims)
    for n in range(len(dims)):
        np.testing.assert_array_equal(oracle.unfold(t, n), brute_unfold(x, dims, n))
        np.testing.assert_array_equal(oracle.fold(oracle.unfold(t, n), n, dims), t)


@pytest.mark.parametrize("dims", TINY)
def test_gram_eigs_match_svd_of_explicit_unfolding(dims):
    rng = np.random.default_rng(2)
    x = rng.standard_normal(math.prod(dims))
    t = oracle.as_tensor(x, dims)
    for n in range(len(dims)):
        m = brute_unfold(x, dims, n)
        lam, v = oracle.leading_eigenpairs(oracle.gram(t, n))
        u, sv, _ = np.linalg.svd(m, full_matrices=True)
        sig2 = np.zeros(dims[n])
        sig2[: len(sv)] = sv ** 2
        np.testing.assert_allclose(lam, sig2, rtol=0, atol=1e-13 * max(1.0, sig2[0]))
        # leading eigenvector subspaces agree where the spectrum separates them
        for r in range(1, dims[n]):
            if sig2[r - 1] - sig2[r] > 1e-6 * sig2[0]:
                assert principal_sines(v[:, :r], u[:, :r]).max() < 1e-10


def test_matrix_case_is_truncated_svd():
    """N = 2: ST-HOSVD is the truncated SVD; Eckart-Young gives the error exactly."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((30, 7)) @ np.diag(2.0 ** -np.arange(7)) @ rng.standard_normal((7, 20))
    a += 1e-3 * rng.standard_normal((30, 20))
    x = a.ravel(order="F")
    eps = 0.05
    res = oracle.sthosvd(x, (30, 20), eps)
    sv = np.linalg.svd(a, compute_uv=False)
    nx2 = float((sv ** 2).sum())
    thr = eps * eps * nx2 / 2
    # the rank the rule must pick for mode 1, straight from the singular values
    r1 = next(r for r in range(1, 21) if (sv[r:] ** 2).sum() <= thr)
    assert res["ranks"][0] == r1
    xr = oracle.reconstruct(res["core"], res["ranks"], res["factors"])
    err2 = float(((x - xr) ** 2).sum())
    r = min(res["ranks"])
    np.testing.assert_allclose(err2, (sv[r:] ** 2).sum(), rtol=1e-9)
    u, _ = svd_factor(a, res["ranks"][0])
    assert principal_sines(res["factors"][0], u).max() < 1e-10


@pytest.mark.parametrize("dims,ranks,order", [
    ((12, 10, 9), (3, 4, 2), None),
    ((8, 7, 6, 5), (2, 3, 2, 4), (3, 1, 0, 2)),
    ((20, 5), (4, 4), (1, 0)),
])
def test_exact_recovery_of_known_multilinear_rank(dims, ranks, order):
    x = tucker_tensor_np(dims, ranks, seed=4)
    res = oracle.sthosvd(x, dims, 1e-6, order)
    assert res["ranks"] == tuple(ranks)
    assert oracle.rel_error(x, res["core"], res["ranks"], res["factors"]) < 1e-13


def _check_invariants(x, dims, eps, order=None):
    res = oracle.sthosvd(x, dims, eps, order)
    for u in res["factors"]:
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-14 * u.shape[0])
    xr = oracle.reconstruct(res["core"], res["ranks"], res["factors"])
    err2 = float(((x - xr) ** 2).sum())
    nx2 = float((x ** 2).sum())
    g2 = float((res["core"] ** 2).sum())
    # Pythagoras for ST-HOSVD: the discarded pieces are mutually orthogonal
    np.testing.assert_allclose(err2, sum(res["tails"]), rtol=1e-9, atol=1e-13 * nx2)
    np.testing.assert_allclose(err2, nx2 - g2, rtol=1e-6, atol=1e-12 * nx2)
    assert math.sqrt(err2 / nx2) <= eps * (1 + 1e-12)
    for n, t in enumerate(res["tails"]):
        assert t <= res["threshold"] * (1 + 1e-12) + 1e-300
    return res


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_invariants_noisy(seed):
    dims, ranks = (14, 12, 10, 6), (5, 4, 6, 3)
    x = tucker_tensor_np(dims, ranks, seed=seed, decay=0.3, smooth=True, noise=1e-2)
    for eps in (3e-2, 1e-1, 0.3):
        _check_invariants(x, dims, eps)
        _check_invariants(x, dims, eps, (2, 0, 3, 1))


def test_trace_of_each_gram_is_current_norm():
    dims, ranks = (9, 8, 7), (3, 3, 3)
    x = tucker_tensor_np(dims, ranks, seed=5, noise=0.05)
    res = oracle.sthosvd(x, dims, 0.02)
    # ||Y||^2 before mode n equals trace(S_n) = sum of that mode's eigenvalues
    y = oracle.as_tensor(x, dims)
    for n in range(3):
        np.testing.assert_allclose(res["eigvals"][n].sum(), (np.asarray(y) ** 2).sum(), rtol=1e-12)
        y = oracle.ttm(y, n, res["factors"][n].T)


def test_permutation_equivariance():
    dims, ranks = (10, 8, 6), (4, 3, 2)
    x = tucker_tensor_np(dims, ranks, seed=6, noise=0.02)
    perm = (2, 0, 1)  # new mode k is old mode perm[k]
    xt = oracle.as_tensor(x, dims).transpose(perm)
    xp = np.asfortranarray(xt).ravel(order="F")
    dims_p = tuple(dims[p] for p in perm)
    order = (0, 1, 2)
    order_p = tuple(perm.index(o) for o in order)  # same old-mode sequence
    a = oracle.sthosvd(x, dims, 0.05, order)
    b = oracle.sthosvd(xp, dims_p, 0.05, order_p)
    for k, p in enumerate(perm):
        assert b["ranks"][k] == a["ranks"][p]
        np.testing.assert_allclose(b["factors"][k], a["factors"][p], atol=1e-12)
    ga = oracle.as_tensor(a["core"], a["ranks"]).transpose(perm)
    gb = oracle.as_tensor(b["core"], b["ranks"])
    np.testing.assert_allclose(gb, ga, atol=1e-12)


def test_orthogonal_and_scale_equivariance():
    dims, ranks = (9, 7, 6), (3, 2, 3)
    x = tucker_tensor_np(dims, ranks, seed=7, noise=0.02)
    q, _ = np.linalg.qr(np.random.default_rng(8).standard_normal((7, 7)))
    xq = np.asarray(oracle.ttm(oracle.as_tensor(x, dims), 1, q)).ravel(order="F")
    a = oracle.sthosvd(x, dims, 0.05)
    b = oracle.sthosvd(xq, dims, 0.05)
    assert a["ranks"] == b["ranks"]
    assert principal_sines(q @ a["factors"][1], b["factors"][1]).max() < 1e-10
    c = oracle.sthosvd(3.5 * x, dims, 0.05)
    assert c["ranks"] == a["ranks"]
    np.testing.assert_allclose(c["core"], 3.5 * a["core"], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("eps", [0.08, 0.0])
def test_brute_force_sthosvd_tiny(eps):
    """Algorithm 1 by loops: explicit unfoldings, SVD for the factors, loop TTMs.

    eps = 0 keeps every index, so each factor is a full (non-symmetric)
    orthogonal matrix and the core pins the orientation of the TTM (U^T, not U).
    """
    dims = (4, 3, 5)
    x = tucker_tensor_np(dims, (2, 2, 3), seed=9, noise=0.05)
    res = oracle.sthosvd(x, dims, eps, (1, 2, 0))
    nx2 = sum(v * v for v in x)
    thr = eps * eps * nx2 / 3
    y, cur = x.copy(), dims
    for n in (1, 2, 0):
        m = brute_unfold(y, cur, n)
        _, sv = svd_factor(m, 1)
        sig2 = np.zeros(cur[n])
        sig2[: len(sv)] = sv ** 2
        r = next(r for r in range(1, cur[n] + 1) if sig2[r:].sum() <= thr)
        assert res["ranks"][n] == r
        u, _ = svd_factor(m, r)
        np.testing.assert_allclose(res["factors"][n], u, atol=1e-10)
        y, cur = brute_ttm(y, cur, n, u.T)
    np.testing.assert_allclose(res["core"], y, atol=1e-10)


def test_superdiagonal_closed_form():
    """X = 3 e1 o e1 o e1 + 1 e2 o e2 o e2: every Gram is diag(9, 1), ||X||^2 = 10.

    eps = 0.6: threshold 0.36 * 10 / 3 = 1.2 >= 1, so mode 1 drops e2 and
    R = (1, 1, 1), core = [3], error 1/sqrt(10).  eps = 0.5: threshold
    0.8333 < 1, nothing is dropped, core = X.
    """
    x = np.zeros(8)
    x[0], x[7] = 3.0, 1.0
    res = oracle.sthosvd(x, (2, 2, 2), 0.6)
    assert res["ranks"] == (1, 1, 1)
    np.testing.assert_allclose(res["core"], [3.0], atol=1e-15)
    assert res["tails"][0] == pytest.approx(1.0)
    assert oracle.rel_error(x, res["core"], res["ranks"], res["factors"]) == pytest.approx(1 / math.sqrt(10))
    res = oracle.sthosvd(x, (2, 2, 2), 0.5)
    assert res["ranks"] == (2, 2, 2)
    np.testing.assert_allclose(res["core"], x, atol=1e-15)


def test_threshold_uses_original_norm_closed_form():
    """Superdiagonal 3x3x3 with diagonal (3, 1, 0.8), eps = 0.54.

    ||X||^2 = 10.64 and every Gram of X is diag(9, 1, 0.64).  The threshold is
    0.54^2 * 10.64 / 3 = 1.0342.  Mode 1 keeps two indices (tail(1) = 1.64 >
    1.0342, tail(2) = 0.64).  After it, Y holds 3 and 1 on its diagonal, so
    mode 2 sees diag(9, 1, 0) and drops the 1 (1 <= 1.0342), and mode 3 keeps
    one index.  A threshold taken from ||Y||^2 = 10 (0.972) would keep the 1.
    """
    x = np.zeros(27)
    x[0], x[13], x[26] = 3.0, 1.0, 0.8
    res = oracle.sthosvd(x, (3, 3, 3), 0.54)
    assert res["ranks"] == (2, 1, 1)
    np.testing.assert_allclose(res["core"], [3.0, 0.0], atol=1e-14)
    np.testing.assert_allclose(res["tails"], [0.64, 1.0, 0.0], atol=1e-14)
    assert oracle.rel_error(x, res["core"], res["ranks"], res["factors"]) == pytest.approx(math.sqrt(1.64 / 10.64))


def test_rank_one_closed_form():
    """X = a o b o c: R = (1, 1, 1), U_n = +-v/||v||, |G| = ||a|| ||b|| ||c||."""
    a, b, c = np.array([1.0, -2.0, 2.0]), np.array([3.0, 4.0]), np.array([0.0, -1.0, 0.0, 0.0])
    x = np.einsum("i,j,k->kji", a, b, c).ravel()  # C order of reversed axes = natural layout
    res = oracle.sthosvd(x, (3, 2, 4), 1e-3)
    assert res["ranks"] == (1, 1, 1)
    for u, v in zip(res["factors"], (a, b, c)):
        w = v / np.linalg.norm(v)
        k = int(np.argmax(np.abs(w)))
        np.testing.assert_allclose(u[:, 0], w * np.sign(w[k]), atol=1e-14)
    # the sign rule makes each factor's largest entry positive: a -> -a/3, b -> b/5, c -> -c
    np.testing.assert_allclose(res["core"], [3.0 * 5.0 * 1.0], atol=1e-13)


def test_rank_rule_edges():
    lam = np.array([4.0, 1.0, 1.0, -1e-17])
    assert osth.rank_from_eps(lam, 1.0) == (2, 1.0)  # tail(2) = 1 <= 1 (inequality is <=)
    assert osth.rank_from_eps(lam, 0.999)[0] == 3
    assert osth.rank_from_eps(lam, 0.0)[0] == 3  # negative eigenvalue clamps to 0
    assert osth.rank_from_eps(lam, 100.0)[0] == 1  # never below 1
    assert osth.rank_from_eps(lam, 0.0, keep_all=True)[0] == 4
    # clamping decides here: unclamped, tail(1) = 1 - 0.5 would pass 0.6
    assert osth.rank_from_eps(np.array([4.0, 1.0, -0.5]), 0.6)[0] == 2
    res = oracle.sthosvd(np.zeros(24), (2, 3, 4), 1e-3)
    assert res["ranks"] == (1, 1, 1)
    assert not res["core"].any()
    x = tucker_tensor_np((5, 4, 3), (2, 2, 2), seed=1, noise=0.1)
    assert oracle.sthosvd(x, (5, 4, 3), 0.0)["ranks"] == (5, 4, 3)
    assert oracle.sthosvd(x, (5, 4, 3), -1.0)["ranks"] == (5, 4, 3)


def test_cube64_closed_form():
    """64^3, core 8^3 N(0,1), noise 1e-4 ||X_clean||, eps 1e-3.

    The retained subspace holds a fraction (8/64)^3 of the white noise, so the
    error is 1e-4 sqrt(1 - 1/512) / sqrt(1 + 1e-8) of ||X||, within a few
    percent for one Gaussian draw; the rank gap is huge (lambda_8 ~ 5e-2
    ||X||^2 against a threshold of 3.3e-7 ||X||^2).
    """
    x = tucker_tensor_np((64, 64, 64), (8, 8, 8), seed=0, noise=1e-4)
    res = oracle.sthosvd(x, (64, 64, 64), 1e-3)
    assert res["ranks"] == (8, 8, 8)
    rel = oracle.rel_error(x, res["core"], res["ranks"], res["factors"])
    assert rel == pytest.approx(1e-4 * math.sqrt(1 - 1 / 512), rel=0.02)


def test_compression_ratio_table2():
    with open(os.path.join(GOLDEN, "table2_compression.json")) as f:
        rows = json.load(f)["rows"]
    for row in rows:
        c = oracle.compression_ratio(row["dims"], row["ranks"])
        assert round(c) == row["printed_ratio"], row["dataset"]
        assert row["st_hosvd_nrms"] <= row["eps"]  # Eq. error_bound: below the target


# ----------------------------------------------------------------------------
# partial reconstruction (Sec. 2.3), HOOI (Algorithm 2), mode-order cost model
# ----------------------------------------------------------------------------

def test_subtensor_is_the_slice_of_the_full_reconstruction():
    """Row subsets of the factors give exactly that block of X~ (Sec. 2.3)."""
    dims, ranks = (7, 6, 5, 4), (3, 2, 4, 2)
    x = tucker_tensor_np(dims, ranks, seed=5, noise=1e-2)
    res = oracle.sthosvd(x, dims, 0.05)
    full = osth.as_tensor(oracle.reconstruct(res["core"], res["ranks"], res["factors"]), dims)
    for lo, hi in [((0, 0, 0, 0), dims), ((2, 1, 3, 0), (5, 6, 4, 3)), ((6, 5, 4, 3), (7, 6, 5, 4))]:
        sub = oracle.reconstruct_sub(res["core"], res["ranks"], res["factors"], lo, hi)
        block = full[tuple(slice(a, b) for a, b in zip(lo, hi))]
        assert np.allclose(sub, np.asarray(block).ravel(order="F"), rtol=0, atol=1e-13)


def _top_subspace_angle(u, m, r):
    """sin of the largest principal angle between span(u) and the top-r left singular subspace of m."""
    w = np.linalg.svd(m, full_matrices=False)[0][:, :r]
    return float(np.linalg.norm(w - u @ (u.T @ w), 2))


def test_hooi_exact_rank_returns_sthosvd():
    dims, ranks = (6, 5, 7), (2, 3, 2)
    x = tucker_tensor_np(dims, ranks, seed=9, noise=0.0)
    h = oracle.hooi(x, dims, 1e-6, max_iters=3)
    assert h["ranks"] == ranks
    assert h["history"][-1] <= 1e-12 * h["norm2"]
    x_hat = oracle.reconstruct(h["core"], h["ranks"], h["factors"])
    assert np.linalg.norm(x_hat - x) <= 1e-12 * math.sqrt(h["norm2"])


def test_hooi_matrix_case_keeps_the_eckart_young_optimum():
    """N = 2: ST-HOSVD already gives the truncated SVD, HOOI cannot improve it."""
    rng = np.random.default_rng(4)
    a = rng.standard_normal((9, 7))
    h = oracle.hooi(a.ravel(order="F"), (9, 7), 0.3, max_iters=4)
    r = h["ranks"][0]
    sv = np.linalg.svd(a, compute_uv=False)
    tail = float(np.sum(sv[r:] ** 2))
    assert h["ranks"][1] == r
    for f in h["history"]:
        assert abs(f - tail) <= 1e-10 * h["norm2"]


def test_hooi_noisy_monotone_stationary_and_pythagorean():
    dims, ranks = (8, 7, 6), (3, 3, 2)
    x = tucker_tensor_np(dims, ranks, seed=3, noise=0.3)
    st = oracle.sthosvd(x, dims, 0.2)
    h = oracle.hooi(x, dims, 0.2, max_iters=200, tol=0.0)
    hist = h["history"]
    assert h["ranks"] == st["ranks"]
    assert all(b <= a + 1e-12 * h["norm2"] for a, b in zip(hist, hist[1:]))  # Algorithm 2 never increases the fit
    assert hist[-1] <= hist[0]
    # the fit is ||X - X~||^2 (orthogonal projections)
    x_hat = oracle.reconstruct(h["core"], h["ranks"], h["factors"])
    assert abs(float(np.sum((x - x_hat) ** 2)) - hist[-1]) <= 1e-10 * h["norm2"]
    # at the fixed point each U_n spans the top R_n left singular vectors of (X x {U_m^T}_{m != n})_(n)
    xt = osth.as_tensor(x, dims)
    for n in range(3):
        y = xt
        for m in range(3):
            if m != n:
                y = osth.ttm(y, m, h["factors"][m].T)
        assert _top_subspace_angle(h["factors"][n], osth.unfold(y, n), h["ranks"][n]) < 1e-6
        assert np.allclose(h["factors"][n].T @ h["factors"][n], np.eye(h["ranks"][n]), atol=1e-13)


def test_order_flops_hand_count():
    # dims (4, 6), ranks (2, 3).  Order (0, 1): J = 24 then 12:
    #   2*4*24 + 2*2*24 + 10/3*64 = 501.33..., then 2*6*12 + 2*3*12 + 10/3*216 = 936
    assert osth.order_flops((4, 6), (2, 3), (0, 1)) == pytest.approx(192 + 96 + 640 / 3 + 144 + 72 + 720)
    # order (1, 0): 2*6*24 + 2*3*24 + 720, then 2*4*12 + 2*2*12 + 640/3
    assert osth.order_flops((4, 6), (2, 3), (1, 0)) == pytest.approx(288 + 144 + 720 + 96 + 48 + 640 / 3)
    assert osth.best_order((4, 6), (2, 3)) == [0, 1]


def test_greedy_flops_order_hand_count():
    # dims (5, 4, 3), ranks (1, 4, 2): the cost of a step on mode n is
    # 2 I_n J + 2 R_n J + 10/3 I_n^3 with J the product of the current dims.
    # Step 1, J = 60: mode 0: 600 + 120 + 416.67 = 1136.67; mode 1: 480 + 480 +
    #   213.33 = 1173.33; mode 2: 360 + 240 + 90 = 690 -> mode 2, J becomes 5*4*2 = 40.
    # Step 2, J = 40: mode 0: 400 + 80 + 416.67 = 896.67; mode 1: 320 + 320 +
    #   213.33 = 853.33 -> mode 1 (with J left at 60 it would be mode 0).
    # Step 3: mode 0.
    assert osth.greedy_order((5, 4, 3), (1, 4, 2), "flops") == [2, 1, 0]
    # step 3 at J = 5*4*2 = 40: 400 + 80 + 416.67; total 690 + 853.33 + 896.67 = 2440
    assert osth.order_flops((5, 4, 3), (1, 4, 2), (2, 1, 0)) == pytest.approx(2440.0)
    # ratio rule: I_n / R_n = 5, 1, 1.5 -> 0, then 2, then 1
    assert osth.greedy_order((5, 4, 3), (1, 4, 2), "ratio") == [0, 2, 1]


def test_order_heuristics_on_the_papers_mode_order_problem():
    # Sec. 8.3: 25 x 250 x 250 x 250 with core 10 x 10 x 100 x 100; the second
    # mode has by far the largest compression ratio I_n / R_n = 25
    dims, ranks = (25, 250, 250, 250), (10, 10, 100, 100)
    assert osth.greedy_order(dims, ranks, "ratio") == [1, 0, 2, 3]
    # fewest flops in the first step: mode 0 (smallest I_n + R_n), as the paper says
    # that heuristic starts there
    assert osth.greedy_order(dims, ranks, "flops")[0] == 0
    best = osth.best_order(dims, ranks)
    costs = {p: osth.order_flops(dims, ranks, p) for p in itertools.permutations(range(4))}
    assert osth.order_flops(dims, ranks, best) == min(costs.values())


# ----------------------------------------------------------------------------
# planted mistakes: each must break at least one pin above
# ----------------------------------------------------------------------------

def _pins_pass():
    checks = [
        lambda: test_matrix_case_is_truncated_svd(),
        lambda: test_exact_recovery_of_known_multilinear_rank((8, 7, 6, 5), (2, 3, 2, 4), (3, 1, 0, 2)),
        lambda: test_invariants_noisy(0),
        lambda: test_brute_force_sthosvd_tiny(0.08),
        lambda: test_brute_force_sthosvd_tiny(0.0),
        lambda: test_superdiagonal_closed_form(),
        lambda: test_threshold_uses_original_norm_closed_form(),
        lambda: test_rank_one_closed_form(),
        lambda: test_permutation_equivariance(),
        lambda: test_rank_rule_edges(),
        lambda: test_unfold_matches_index_map((2, 3, 4, 5)),
        lambda: test_subtensor_is_the_slice_of_the_full_reconstruction(),
        lambda: test_hooi_noisy_monotone_stationary_and_pythagorean(),
        lambda: test_order_flops_hand_count(),
        lambda: test_order_heuristics_on_the_papers_mode_order_problem(),
        lambda: test_greedy_flops_order_hand_count(),
    ]
    for c in checks:
        try:
            c()
        except Exception:  # noqa: BLE001 - any failure counts as caught
            return False
    return True


def _mut_threshold_without_n(x_flat, dims, eps, order=None, _orig=osth.sthosvd):
    return _orig(x_flat, dims, eps * math.sqrt(len(dims)), order)


def _mut_unfold_c_order(x, n):
    x = np.asarray(x)
    return np.moveaxis(x, n, 0).reshape(x.shape[n], -1, order="C")


def _mut_fold_c_order(m, n, shape):
    shape = tuple(shape)
    moved = (shape[n],) + shape[:n] + shape[n + 1:]
    return np.moveaxis(np.asarray(m).reshape(moved, order="C"), 0, n)


def _mut_ascending(s, _orig=osth.leading_eigenpairs):
    lam, v = _orig(s)
    return lam[::-1].copy(), v[:, ::-1].copy()


def _mut_tail_off_by_one(lam, threshold, keep_all=False):
    j = len(lam)
    if keep_all:
        return j, 0.0
    for r in range(1, j + 1):
        t = float(np.clip(lam[r - 1:], 0, None).sum())  # includes lambda_R itself
        if t <= threshold:
            return r, t
    return j, 0.0


def _mut_no_clamp(lam, threshold, keep_all=False):
    j = len(lam)
    if keep_all:
        return j, 0.0
    for r in range(1, j + 1):
        t = float(np.sum(lam[r:]))
        if t <= threshold:
            return r, t
    return j, 0.0


def _mut_ttm_transposed(y, n, m, _orig=osth.ttm):
    if m.shape[0] == m.shape[1]:
        return _orig(y, n, m.T)
    return _orig(y, n, m)


def _mut_current_norm_threshold(x_flat, dims, eps, order=None):
    # threshold recomputed from the shrinking Y at every mode instead of X
    dims = tuple(dims)
    order = list(range(len(dims))) if order is None else list(order)
    y = osth.as_tensor(x_flat, dims)
    ranks, factors, eigvals, tails = list(dims), [None] * len(dims), [None] * len(dims), [0.0] * len(dims)
    for n in order:
        thr = eps * eps * osth.norm2(y) / len(dims)
        lam, v = osth.leading_eigenpairs(osth.gram(y, n))
        r, t = osth.rank_from_eps(lam, thr, not eps > 0)
        factors[n], ranks[n], eigvals[n], tails[n] = v[:, :r].copy(), r, lam, t
        y = osth.ttm(y, n, factors[n].T)
    nx2 = osth.norm2(osth.as_tensor(x_flat, dims))
    return {"core": np.asarray(y).ravel(order="F"), "factors": factors, "ranks": tuple(ranks),
            "eigvals": eigvals, "tails": tails, "norm2": nx2, "threshold": eps * eps * nx2 / len(dims),
            "order": tuple(order), "dims": dims}


def _mut_sub_ignores_lo(core_flat, ranks, factors, lo, hi, _orig=osth.reconstruct_sub):
    return _orig(core_flat, ranks, factors, [0] * len(lo), [b - a for a, b in zip(lo, hi)])


def _mut_hooi_no_update(x_flat, dims, eps, max_iters=10, tol=0.0, order=None):
    res = osth.sthosvd(x_flat, dims, eps, order)
    core = osth.as_tensor(res["core"], res["ranks"])
    out = dict(res)
    out["history"] = [res["norm2"] - osth.norm2(core)] * 2
    out["iters"] = 1
    return out


def _mut_ttm_flops_with_i(dims, ranks, order):
    cur = [int(d) for d in dims]
    total = 0.0
    for n in order:
        j = math.prod(cur)
        total += 4.0 * dims[n] * j + 10.0 / 3.0 * float(dims[n]) ** 3
        cur[n] = int(ranks[n])
    return total


def _mut_greedy_max(dims, ranks, rule, _orig=osth.greedy_order):
    return _orig(dims, ranks, rule)[::-1]


def _mut_greedy_no_shrink(dims, ranks, rule):
    # the current dims are never updated after a pick
    left = list(range(len(dims)))
    cur = [int(d) for d in dims]
    order = []
    while left:
        if rule == "flops":
            j = math.prod(cur)
            pick = min(left, key=lambda n: (2.0 * dims[n] * j + 2.0 * ranks[n] * j + 10.0 / 3.0 * float(dims[n]) ** 3,
                                            n))
        else:
            pick = min(left, key=lambda n: (-dims[n] / ranks[n], n))
        order.append(pick)
        left.remove(pick)
    return order


MUTATIONS = {
    "subtensor_ignores_lo": ("reconstruct_sub", _mut_sub_ignores_lo),
    "hooi_never_updates": ("hooi", _mut_hooi_no_update),
    "ttm_flops_with_I": ("order_flops", _mut_ttm_flops_with_i),
    "greedy_reversed": ("greedy_order", _mut_greedy_max),
    "greedy_no_shrink": ("greedy_order", _mut_greedy_no_shrink),
    "threshold_without_N": ("sthosvd", _mut_threshold_without_n),
    "unfold_column_order": ("unfold", _mut_unfold_c_order),
    "fold_column_order": ("fold", _mut_fold_c_order),
    "trailing_eigenvectors": ("leading_eigenpairs", _mut_ascending),
    "tail_off_by_one": ("rank_from_eps", _mut_tail_off_by_one),
    "negative_eigs_not_clamped": ("rank_from_eps", _mut_no_clamp),
    "ttm_square_transposed": ("ttm", _mut_ttm_transposed),
    "threshold_from_current_Y": ("sthosvd", _mut_current_norm_threshold),
}


def test_pins_pass_unmutated():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(osth, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    assert not _pins_pass(), f"planted mistake {name} escaped every pin"
