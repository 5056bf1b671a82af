"""GPU parity: every step of the CUDA path against the CPU oracle, through the C ABI.

Tolerances (derived from the float64 arithmetic; u = 2^-53):

* Gram and TTM entries: the rigorous dot-product bound gamma_K * (|A||B|)_ij
  for each side, K the contraction length, gamma_K = K u / (1 - K u).
* Eigenvalues: |lam_gpu - lam_oracle| <= 64 J u ||S||_2 (both are backward
  stable to a few J u ||S||); eigenvectors by residual, orthogonality and
  Davis-Kahan subspace angles sin(theta) <= 64 J u ||S|| / gap.
* Rank rule: bit-exact (it is a decision on identical eigenvalues).
* End to end: identical ranks, |rel_gpu - rel_oracle| <= 1e-12 and principal
  angles <= 1e-8 between factor subspaces wherever the retained and discarded
  eigenvalues are separated by (lam_R - lam_{R+1}) / lam_1 >= 1e-4; closer
  gaps get the Davis-Kahan bound 10 * 1e-14 * lam_1 / gap.  The core is
  compared after aligning factor signs, to 1e-10 ||G||.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synthetic import tucker_tensor_np

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def gamma(k):
    return k * U / (1 - k * U)


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def principal_sines(a, b):
    return np.linalg.svd(b - a @ (a.T @ b), compute_uv=False)


def view3(x_flat, dims, n):
    l = math.prod(dims[:n])
    b = math.prod(dims[n + 1:])
    return l, dims[n], b


# ---------------------------------------------------------------------------
# a1: ||X||^2
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 7, 1000, 262144 + 13, 3_000_001])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_norm2(gpu_lib, n, dtype):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    if dtype == "f32":
        x = x.astype(np.float32)
    ref = float(np.dot(x.astype(np.float64), x.astype(np.float64)))
    got = gpu_lib.norm2(dev(x))
    assert abs(got - ref) <= gamma(max(n, 1)) * ref + 1e-300


# ---------------------------------------------------------------------------
# a2: Gram of the (L, J, B) view, read in place
# ---------------------------------------------------------------------------
GRAM_SHAPES = [
    (1, 1, 1), (1, 5, 3), (1, 64, 4096), (7, 13, 5), (40, 128, 33), (1600, 48, 3),
    (64000 // 100, 32, 1), (1, 129, 257), (3, 200, 17), (2, 512, 40), (1, 1024, 3),
]


@pytest.mark.parametrize("L,J,B", GRAM_SHAPES)
def test_gram(gpu_lib, L, J, B):
    rng = np.random.default_rng(L * 7 + J * 3 + B)
    y = rng.standard_normal(L * J * B)
    s = gpu_lib.gram(dev(y), L, J, B).cpu().numpy()
    t = y.reshape((L, J, B), order="F")
    yn = oracle.unfold(t, 1)  # J x (L B) mode-2 unfolding of the 3-way view
    ref = oracle.gram(t, 1)
    assert np.array_equal(s, s.T)
    k = L * B
    bound = 2 * gamma(k) * (np.abs(yn) @ np.abs(yn).T)
    assert np.all(np.abs(s - ref) <= bound + 1e-300)


def test_gram_f32_input(gpu_lib):
    rng = np.random.default_rng(5)
    L, J, B = 9, 24, 31
    y = rng.standard_normal(L * J * B).astype(np.float32)
    s = gpu_lib.gram(dev(y), L, J, B).cpu().numpy()
    t = y.astype(np.float64).reshape((L, J, B), order="F")
    yn = oracle.unfold(t, 1)
    ref = oracle.gram(t, 1)
    assert np.all(np.abs(s - ref) <= 2 * gamma(L * B) * (np.abs(yn) @ np.abs(yn).T))


def test_gram_deterministic(gpu_lib):
    rng = np.random.default_rng(6)
    L, J, B = 33, 96, 700
    y = dev(rng.standard_normal(L * J * B))
    a = gpu_lib.gram(y, L, J, B).cpu().numpy()
    b = gpu_lib.gram(y, L, J, B).cpu().numpy()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# a3: eigenpairs
# ---------------------------------------------------------------------------
@pytest.fixture(params=["mp", "jacobi"])
def eig_path(request, monkeypatch):
    """Both eigensolvers: mixed precision (strict: no silent fallback) and float64 Jacobi."""
    monkeypatch.setenv("TUCKER_EIG_KERNEL", request.param)
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1" if request.param == "mp" else "0")
    return request.param


def _check_eig(gpu_lib, s):
    import torch

    j = s.shape[0]
    lam, v, sweeps = gpu_lib.eig(torch.from_numpy(s).cuda())
    lam = lam.cpu().numpy()
    v = v.cpu().numpy()
    ref_lam, ref_v = oracle.leading_eigenpairs(s)
    nrm = max(np.linalg.norm(s, 2), 1e-300)
    tol = 64 * j * U * nrm
    assert np.all(np.diff(lam) <= 0)
    assert np.abs(lam - ref_lam).max() <= tol
    assert np.abs(s @ v - v * lam).max() <= tol
    assert np.abs(v.T @ v - np.eye(j)).max() <= 64 * j * U
    # sign rule: largest-magnitude entry of each column is positive
    for c in range(j):
        col = v[:, c]
        assert col[int(np.argmax(np.abs(col)))] > 0
    # Davis-Kahan on every separated leading subspace
    for r in range(1, j):
        gap = ref_lam[r - 1] - ref_lam[r]
        if gap > 1e-6 * nrm:
            assert principal_sines(ref_v[:, :r], v[:, :r]).max() <= tol / gap + 1e-15
    return sweeps


@pytest.mark.parametrize("j", [1, 2, 3, 8, 17, 64, 127, 128, 129, 200])
def test_eig_random_psd(gpu_lib, eig_path, j):
    rng = np.random.default_rng(j)
    a = rng.standard_normal((j, 2 * j + 3)) * (0.7 ** np.arange(j))[:, None]
    _check_eig(gpu_lib, a @ a.T)


WIDE = pytest.mark.skipif(os.environ.get("TUCKER_EIG_WIDE") == "0",
                          reason="the wide float32 stage (128 < J <= 256) is switched off: TUCKER_EIG_WIDE=0")


@WIDE
@pytest.mark.parametrize("j,r,floor", [(160, 40, 1e-12), (200, 20, 1e-12), (250, 100, 1e-12), (256, 10, 1e-6)])
def test_eig_wide_tucker_grams(gpu_lib, monkeypatch, j, r, floor):
    """The wide float32 stage under the strict check (no fallback) on Grams
    shaped like Tucker modes: r signal eigenvalues within about 10% of each
    other over a noise floor holding `floor` of the energy."""
    monkeypatch.setenv("TUCKER_EIG_KERNEL", "mp")
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1")
    rng = np.random.default_rng(j)
    q, _ = np.linalg.qr(rng.standard_normal((j, j)))
    sig = 1e4 * (1 + 0.1 * rng.standard_normal(r))
    lam = np.concatenate([sig, floor * sig.sum() / j * (1 + 0.1 * rng.random(j - r))])
    s = (q * lam) @ q.T
    _check_eig(gpu_lib, 0.5 * (s + s.T))


@WIDE
def test_sthosvd_wide_dims(gpu_lib, monkeypatch):
    """ST-HOSVD with a mode of 200 (the wide stage, strict) against the oracle."""
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1")
    dims, ranks = (200, 24, 20), (10, 5, 4)
    x = tucker_tensor_np(dims, ranks, seed=7, noise=1e-4)
    compare_sthosvd(gpu_lib, x, dims, 1e-3)


@pytest.mark.parametrize("j", [5, 48, 130])
def test_eig_special(gpu_lib, eig_path, j):
    import torch

    # identity: every eigenvalue equal, ties keep index order, V = I
    lam, v, _ = gpu_lib.eig(torch.eye(j, dtype=torch.float64).cuda())
    assert np.array_equal(lam.cpu().numpy(), np.ones(j))
    assert np.array_equal(v.cpu().numpy(), np.eye(j))
    # zero matrix
    lam, v, _ = gpu_lib.eig(torch.zeros((j, j), dtype=torch.float64).cuda())
    assert not lam.cpu().numpy().any()
    # rank-deficient and indefinite diagonal-plus-low-rank
    rng = np.random.default_rng(j)
    a = rng.standard_normal((j, 3))
    _check_eig(gpu_lib, a @ a.T)
    d = np.diag(np.linspace(-1, 1, j))
    _check_eig(gpu_lib, d + 1e-3 * (a @ a.T))


@pytest.mark.parametrize("seed", [0, 3])
def test_eig_mp_on_tucker_grams(gpu_lib, monkeypatch, seed):
    """Graded spectra with a noise cluster (the Grams ST-HOSVD meets): the
    mixed-precision solver must pass on its own, without the float64 fallback."""
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1")
    dims, ranks = (128, 64, 48, 16), (40, 40, 20, 10)
    x = tucker_tensor_np(dims, ranks, seed=seed, decay=0.15, smooth=True, noise=1e-6)
    t = oracle.as_tensor(x, dims)
    for n in range(len(dims)):
        _check_eig(gpu_lib, oracle.gram(t, n))


@pytest.mark.parametrize("j", [257, 300, 384, 512])
def test_eig_cluster_stage(gpu_lib, eig_path, j):
    """256 < J <= 512: the mixed-precision solver's first stage is the float32
    Jacobi on a 16-CTA cluster (strict: no fallback), and the float64 Jacobi."""
    rng = np.random.default_rng(j)
    a = rng.standard_normal((j, j + 40)) * (0.97 ** np.arange(j))[:, None]
    _check_eig(gpu_lib, a @ a.T)


@pytest.mark.parametrize("j,r,floor", [(300, 60, 1e-12), (512, 64, 1e-12), (512, 200, 1e-8), (512, 300, 1e-8),
                                       (400, 200, 1e-12), (256, 200, 1e-8), (256, 120, 1e-8)])
def test_eig_cluster_stage_tucker_grams(gpu_lib, monkeypatch, j, r, floor):
    """Strict solves of Tucker-like Grams: r signal eigenvalues within 10% of
    each other over a noise cluster holding `floor` of the energy.  Clusters
    of more than 128 large, close eigenvalues are solved shifted by their
    mean at the next level (without the shift they stayed one cluster at
    every depth); J > 256 takes the cluster float32 stage."""
    monkeypatch.setenv("TUCKER_EIG_KERNEL", "mp")
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1")
    rng = np.random.default_rng(j + r)
    q, _ = np.linalg.qr(rng.standard_normal((j, j)))
    sig = 1e4 * (1 + 0.1 * rng.standard_normal(r))
    lam = np.concatenate([sig, floor * sig.sum() / j * (1 + 0.1 * rng.random(j - r))])
    s = (q * lam) @ q.T
    _check_eig(gpu_lib, 0.5 * (s + s.T))


def test_eig_large_dim(gpu_lib):
    rng = np.random.default_rng(9)
    j = 512
    a = rng.standard_normal((j, 600)) * (0.97 ** np.arange(j))[:, None]
    _check_eig(gpu_lib, a @ a.T)


# ---------------------------------------------------------------------------
# a4: rank rule (bit-exact)
# ---------------------------------------------------------------------------
def test_rank_cut_bit_exact(gpu_lib):
    import torch

    rng = np.random.default_rng(11)
    for j in (1, 2, 7, 64, 300, 1024):
        lam = np.sort(rng.standard_normal(j) ** 4)[::-1].copy()
        lam[-1] = -abs(lam[-1]) * 1e-3  # a rounding-negative eigenvalue
        total = float(np.clip(lam, 0, None).sum())
        for thr in (0.0, 1e-12 * total, 1e-3 * total, 0.1 * total, total, 10 * total):
            r, tail = gpu_lib.rank_cut(torch.from_numpy(lam).cuda(), thr)
            rr, tt = oracle.rank_from_eps(lam, thr)
            assert (r, tail) == (rr, tt)
        assert gpu_lib.rank_cut(torch.from_numpy(lam).cuda(), 1.0, keep_all=True)[0] == j
    # equality case: tail == threshold is kept (<=)
    lam = np.array([4.0, 1.0, 0.5, 0.5])
    assert gpu_lib.rank_cut(torch.from_numpy(lam).cuda(), 1.0) == (2, 1.0)


# ---------------------------------------------------------------------------
# a6 / a8: mode products (shrinking with U^T, expanding with U)
# ---------------------------------------------------------------------------
TTM_SHAPES = [(1, 64, 4096, 8), (40, 128, 33, 40), (7, 13, 5, 13), (1600, 48, 3, 20), (1, 1, 9, 1),
              (3, 200, 17, 64), (2, 512, 6, 16), (5, 16, 7, 512), (1, 9, 1000, 1024)]


@pytest.mark.parametrize("L,J,B,K", TTM_SHAPES)
@pytest.mark.parametrize("transpose", [True, False])
def test_ttm(gpu_lib, L, J, B, K, transpose):
    import torch

    rng = np.random.default_rng(L + J + B + K)
    y = rng.standard_normal(L * J * B)
    m = rng.standard_normal((J, K) if transpose else (K, J))
    mk = m.T if transpose else m
    z = gpu_lib.ttm(dev(y), L, J, B, torch.from_numpy(m).cuda(), transpose=transpose).cpu().numpy()
    t = y.reshape((L, J, B), order="F")
    ref = np.asarray(oracle.ttm(t, 1, mk)).ravel(order="F")
    absref = np.asarray(oracle.ttm(np.abs(t), 1, np.abs(mk))).ravel(order="F")
    assert np.all(np.abs(z - ref) <= 2 * gamma(J) * absref + 1e-300)


def test_ttm_f32_input(gpu_lib):
    import torch

    rng = np.random.default_rng(3)
    L, J, B, K = 6, 20, 11, 7
    y = rng.standard_normal(L * J * B).astype(np.float32)
    m = rng.standard_normal((J, K))
    z = gpu_lib.ttm(dev(y), L, J, B, torch.from_numpy(m).cuda(), transpose=True).cpu().numpy()
    t = y.astype(np.float64).reshape((L, J, B), order="F")
    ref = np.asarray(oracle.ttm(t, 1, m.T)).ravel(order="F")
    absref = np.asarray(oracle.ttm(np.abs(t), 1, np.abs(m.T))).ravel(order="F")
    assert np.all(np.abs(z - ref) <= 2 * gamma(J) * absref)


# ---------------------------------------------------------------------------
# end to end: Algorithm 1, reconstruction and relative error
# ---------------------------------------------------------------------------
def compare_sthosvd(gpu_lib, x, dims, eps, order=None, dtype="f64"):
    xin = x.astype(np.float32) if dtype == "f32" else x
    xo = xin.astype(np.float64)
    ref = oracle.sthosvd(xo, dims, eps, order)
    xd = dev(xin)
    res = gpu_lib.sthosvd(xd, dims, eps, order)
    assert res.ranks == ref["ranks"]
    assert res.norm2 == pytest.approx(ref["norm2"], rel=1e-13)
    n_modes = len(dims)
    flips = []
    for n in range(n_modes):
        u = res.factor(n).cpu().numpy()
        v = ref["factors"][n]
        lam = ref["eigvals"][n]
        r = ref["ranks"][n]
        assert np.abs(u.T @ u - np.eye(r)).max() <= 1e-13 * dims[n]
        # eigenvalues: the retained ones individually; past the cut the solver may leave a
        # cluster unresolved (Rayleigh quotients of its basis), so the discarded sum is compared
        got = np.asarray(res.eigvals[n])
        assert np.abs(got[:r] - lam[:r]).max(initial=0.0) <= 1e-12 * max(lam[0], 1e-300)
        # each eigenvalue is within 1e-12 lam_1 (the retained ones are checked so above); a sum of
        # the J - R discarded ones is within (J - R) 1e-12 lam_1 (Lidskii: the differences of the
        # eigenvalue vectors are majorised by the eigenvalues of the perturbation)
        n_tail = max(dims[n] - r, 1)
        assert abs(res.tails[n] - lam[r:].sum()) <= 1e-12 * max(lam[0], 1e-300) * n_tail
        assert abs(got[r:].sum() - lam[r:].sum()) <= 1e-12 * max(lam[0], 1e-300) * n_tail
        assert 1 <= res.eig_resolved[n] <= dims[n] and res.eig_resolved[n] >= r
        gap = (lam[r - 1] - lam[r]) if r < dims[n] else lam[r - 1]
        lim = 1e-8 if gap >= 1e-4 * lam[0] else max(1e-8, 10 * 1e-14 * lam[0] / max(gap, 1e-300))
        if r < dims[n]:
            assert principal_sines(v, u).max() <= lim, (n, gap / lam[0])
        flips.append(np.sign(np.sum(u * v, axis=0)))
    # core after aligning signs column by column
    g = res.core().cpu().numpy().reshape(res.ranks, order="F")
    for n, f in enumerate(flips):
        shape = [1] * n_modes
        shape[n] = -1
        g = g * f.reshape(shape)
    gref = ref["core"].reshape(ref["ranks"], order="F")
    gn = max(np.linalg.norm(gref), 1e-300)
    if all(
        (ref["eigvals"][n][ref["ranks"][n] - 1] - (ref["eigvals"][n][ref["ranks"][n]] if ref["ranks"][n] < dims[n]
                                                     else 0.0)) >= 1e-4 * ref["eigvals"][n][0]
        for n in range(n_modes)
    ):
        # within-subspace rotations are fixed only where the retained eigenvalues are separated
        sep = all(np.min(-np.diff(ref["eigvals"][n][: ref["ranks"][n]]), initial=np.inf) >= 1e-6 * ref["eigvals"][n][0]
                  for n in range(n_modes))
        if sep:
            assert np.abs(g - gref).max() <= 1e-10 * gn
    rel = gpu_lib.rel_error(xd, res)
    rel_ref = oracle.rel_error(xo, ref["core"], ref["ranks"], ref["factors"])
    assert abs(rel - rel_ref) <= 1e-12, (rel, rel_ref)
    if eps > 0:
        assert rel <= eps * (1 + 1e-9)
    return res, ref


def test_cube64(gpu_lib):
    """64^3, core 8^3, noise 1e-4, eps 1e-3, order 1,2,3."""
    dims = (64, 64, 64)
    x = tucker_tensor_np(dims, (8, 8, 8), seed=0, noise=1e-4)
    res, ref = compare_sthosvd(gpu_lib, x, dims, 1e-3, (0, 1, 2))
    assert res.ranks == (8, 8, 8)


@pytest.mark.parametrize("order", [(0, 1, 2, 3, 4), (4, 3, 2, 1, 0), (2, 0, 4, 1, 3)])
@pytest.mark.parametrize("eps", [1e-5, 1e-3])
def test_combustion_shaped_small(gpu_lib, order, eps):
    """The 5-way generator (decaying core, smoothed factors) at a size the oracle runs in a second."""
    dims, ranks = (40, 36, 32, 12, 10), (12, 12, 12, 6, 4)
    x = tucker_tensor_np(dims, ranks, seed=1, decay=0.15, smooth=True, noise=1e-6)
    compare_sthosvd(gpu_lib, x, dims, eps, order)


def test_f32_input(gpu_lib):
    dims, ranks = (30, 28, 26, 10, 8), (10, 10, 10, 5, 3)
    x = tucker_tensor_np(dims, ranks, seed=2, decay=0.15, smooth=True, noise=1e-6)
    compare_sthosvd(gpu_lib, x, dims, 1e-4, None, dtype="f32")


@pytest.mark.parametrize("dims,ranks,eps", [
    ((37,), (1,), 0.5),                  # N = 1
    ((50, 33), (6, 6), 1e-3),            # matrix: truncated SVD
    ((1, 9, 1, 7), (1, 3, 1, 2), 1e-2),  # unit modes
    ((17, 13, 11), (4, 5, 3), 0.0),      # eps = 0 keeps everything
    ((17, 13, 11), (4, 5, 3), -1.0),
    ((129, 5, 6), (7, 3, 2), 1e-3),      # J above the shared-memory eigensolver
    ((3, 2, 300), (2, 2, 4), 1e-3),
])
def test_edge_shapes(gpu_lib, dims, ranks, eps):
    x = tucker_tensor_np(dims, ranks, seed=3, noise=1e-3)
    res, _ = compare_sthosvd(gpu_lib, x, dims, eps)
    if eps <= 0:
        assert res.ranks == dims


def test_exact_low_rank_recovery(gpu_lib):
    dims, ranks = (20, 18, 16, 9), (3, 4, 2, 3)
    x = tucker_tensor_np(dims, ranks, seed=4)
    res, _ = compare_sthosvd(gpu_lib, x, dims, 1e-6)
    assert res.ranks == ranks
    assert gpu_lib.rel_error(dev(x), res) < 1e-13


def test_zero_tensor(gpu_lib):
    dims = (6, 5, 4)
    x = np.zeros(math.prod(dims))
    res = gpu_lib.sthosvd(dev(x), dims, 1e-3)
    assert res.ranks == (1, 1, 1)
    assert not res.core().cpu().numpy().any()
    assert gpu_lib.rel_error(dev(x), res) == 0.0


def test_reconstruct_matches_oracle(gpu_lib):
    dims, ranks = (21, 19, 17, 5), (4, 6, 3, 2)
    x = tucker_tensor_np(dims, ranks, seed=5, noise=1e-2)
    xd = dev(x)
    res = gpu_lib.sthosvd(xd, dims, 5e-2)
    xr = gpu_lib.reconstruct(res).cpu().numpy()
    xr_ref = oracle.reconstruct(res.core().cpu().numpy(), res.ranks, [f.cpu().numpy() for f in res.factors()])
    assert np.abs(xr - xr_ref).max() <= 1e-13 * np.abs(x).max()
    # Pythagoras: ||X - X~||^2 = sum of discarded tails (Sec. 7.2 bound, tight for ST-HOSVD)
    err2 = float(((x - xr) ** 2).sum())
    assert err2 == pytest.approx(sum(res.tails), rel=1e-8)


def test_reconstruct_sub_matches_oracle_and_full(gpu_lib):
    """Subtensors from row subsets of the factors (Sec. 2.3)."""
    dims, ranks = (21, 19, 17, 5), (4, 6, 3, 2)
    x = tucker_tensor_np(dims, ranks, seed=8, noise=1e-2)
    res = gpu_lib.sthosvd(dev(x), dims, 5e-2)
    full = gpu_lib.reconstruct(res).cpu().numpy().reshape(dims, order="F")
    core, facs = res.core().cpu().numpy(), [f.cpu().numpy() for f in res.factors()]
    for lo, hi in [((0, 0, 0, 0), dims), ((3, 0, 5, 1), (9, 19, 6, 4)), ((20, 18, 16, 4), dims), ((0, 2, 0, 0), (21, 3, 17, 5))]:
        sub = gpu_lib.reconstruct_sub(res, lo, hi).cpu().numpy()
        ref = oracle.reconstruct_sub(core, res.ranks, facs, lo, hi)
        assert np.abs(sub - ref).max() <= 1e-13 * np.abs(x).max()
        block = full[tuple(slice(a, b) for a, b in zip(lo, hi))].ravel(order="F")
        assert np.abs(sub - block).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("precision", ["fp64", "bf16x4"])
def test_hooi_matches_oracle(gpu_lib, precision):
    """Algorithm 2: same ranks, the same fit history within the path's tolerance,
    and factors spanning the oracle's subspaces (where they are separated)."""
    dims, ranks = (24, 20, 18, 10), (5, 4, 4, 3)
    x = tucker_tensor_np(dims, ranks, seed=12, noise=0.2)
    eps = 0.15
    ref = oracle.hooi(x, dims, eps, max_iters=6, tol=0.0)
    res, iters, fit = gpu_lib.hooi(dev(x), dims, eps, max_iters=6, tol=0.0, precision=precision)
    assert res.ranks == ref["ranks"]
    nx2 = ref["norm2"]
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert len(fit) == iters + 1
    for a, b in zip(fit, ref["history"]):
        assert abs(a - b) <= tol * nx2
    assert all(b <= a + tol * nx2 for a, b in zip(fit, fit[1:]))
    x_hat = gpu_lib.reconstruct(res).cpu().numpy()
    assert abs(float(((x - x_hat) ** 2).sum()) - fit[-1]) <= max(tol, 1e-9) * nx2
    for n in range(len(dims)):
        s = principal_sines(res.factor(n).cpu().numpy(), ref["factors"][n])
        assert s.max() < (1e-6 if precision == "fp64" else 1e-3)


@pytest.mark.parametrize("dims,ranks,eps", [((40,), (1,), 0.1), ((30, 22), (4, 4), 0.2),
                                             ((18, 16, 14), (4, 3, 3), 0.15),
                                             ((10, 9, 8, 7, 6), (3, 3, 2, 2, 2), 0.15)])
def test_hooi_shared_products_any_order(gpu_lib, dims, ranks, eps):
    """HOOI forms every mode's Y from a product shared by its half of the
    modes (first half, then the rest); for N = 1, 2, 3 and 5 the fit history
    still equals Algorithm 2's printed form, where each Y starts from X.  The
    oracle's rank cuts sit at least 2.7e-3 relative from the threshold here."""
    x = tucker_tensor_np(dims, ranks, seed=21, noise=0.2)
    ref = oracle.hooi(x, dims, eps, max_iters=4, tol=0.0)
    res, iters, fit = gpu_lib.hooi(dev(x), dims, eps, max_iters=4, tol=0.0)
    assert res.ranks == ref["ranks"]
    nx2 = ref["norm2"]
    assert len(fit) == iters + 1
    # stagnant fits (N <= 2) may stop one iteration apart: compare the common prefix
    for a, b in zip(fit, ref["history"]):
        assert abs(a - b) <= 1e-10 * nx2
    x_hat = gpu_lib.reconstruct(res).cpu().numpy()
    assert abs(float(((x - x_hat) ** 2).sum()) - fit[-1]) <= 1e-9 * nx2
    for n in range(len(dims)):
        u = res.factor(n).cpu().numpy()
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 64 * dims[n] * U


def test_hooi_zero_iterations_is_sthosvd(gpu_lib):
    dims, ranks = (16, 12, 10), (3, 3, 2)
    x = dev(tucker_tensor_np(dims, ranks, seed=2, noise=1e-2))
    a = gpu_lib.sthosvd(x, dims, 5e-2)
    b, iters, fit = gpu_lib.hooi(x, dims, 5e-2, max_iters=0)
    assert iters == 0 and len(fit) == 1 and b.ranks == a.ranks
    assert np.array_equal(a.core().cpu().numpy(), b.core().cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "bf16x4"])
def test_batched_thread_path_matches_single_calls(gpu_lib, monkeypatch, precision):
    """The per-tensor batched path (host worker threads, TUCKER_BATCH=threads):
    each result equals the single-tensor call bit for bit."""
    from synthetic import random_dims_ranks

    monkeypatch.setenv("TUCKER_BATCH", "threads")
    dims_list, ranks_list = random_dims_ranks(16, seed=3, dim_range=(16, 48), rank_range=(4, 10))
    xs = [dev(tucker_tensor_np(d, r, seed=4, tensor=i, noise=1e-4)) for i, (d, r) in enumerate(zip(dims_list, ranks_list))]
    res = gpu_lib.sthosvd_batched(xs, dims_list, 1e-3, precision=precision, workers=4)
    for x, d, r in zip(xs, dims_list, res):
        one = gpu_lib.sthosvd(x, d, 1e-3, precision=precision)
        assert r.ranks == one.ranks
        assert np.array_equal(r.core().cpu().numpy(), one.core().cpu().numpy())


def _check_batched_against_oracle(gpu_lib, xs_np, xs, dims_list, res, eps):
    for x_np, x, d, r in zip(xs_np, xs, dims_list, res):
        ref = oracle.sthosvd(x_np.astype(np.float64), d, eps)
        assert r.ranks == ref["ranks"], (d, r.ranks, ref["ranks"])
        assert r.norm2 == pytest.approx(ref["norm2"], rel=1e-13)
        for n in range(len(d)):
            u = r.factor(n).cpu().numpy()
            v = ref["factors"][n]
            lam = ref["eigvals"][n]
            k = ref["ranks"][n]
            assert np.abs(u.T @ u - np.eye(k)).max() <= 1e-13 * d[n]
            # the retained eigenvalues individually; the discarded ones the solver may leave
            # unresolved (Rayleigh quotients of a basis of their subspace): their sum, and each
            # in [0, their sum] as the eigenvalues of a positive semidefinite block are
            got = np.asarray(r.eigvals[n])
            tol = 1e-12 * max(lam[0], 1e-300)
            n_tail = max(d[n] - k, 1)
            res_n = r.eig_resolved[n]
            assert k <= res_n <= d[n]
            assert np.abs(got[:res_n] - lam[:res_n]).max(initial=0.0) <= tol
            assert abs(got[k:].sum() - lam[k:].sum()) <= tol * n_tail
            assert abs(r.tails[n] - lam[k:].sum()) <= tol * n_tail
            assert np.all(got[res_n:] >= -tol) and np.all(got[res_n:] <= got[res_n:].sum() + tol)
            if eps == 0.0:
                assert res_n == d[n]
            gap = (lam[k - 1] - lam[k]) if k < d[n] else lam[k - 1]
            if k < d[n] and gap >= 1e-4 * lam[0]:
                assert principal_sines(v, u).max() <= 1e-8
        rel = gpu_lib.rel_error(x, r)
        rel_ref = oracle.rel_error(x_np.astype(np.float64), ref["core"], ref["ranks"], ref["factors"])
        assert abs(rel - rel_ref) <= 1e-12, (rel, rel_ref)


@pytest.mark.parametrize("precision", ["fp64", "bf16x4"])
def test_batched_device_pipeline_matches_oracle(gpu_lib, precision):
    """Many small tensors of mixed sizes (the batched workload's mix, smaller) in
    the device pipeline: each tensor's ranks, eigenvalues, factor subspaces and
    error against the float64 oracle (the pipeline computes in float64)."""
    from synthetic import random_dims_ranks

    dims_list, ranks_list = random_dims_ranks(40, seed=3, dim_range=(16, 64), rank_range=(4, 12))
    xs_np = [tucker_tensor_np(d, r, seed=4, tensor=i, noise=1e-4) for i, (d, r) in enumerate(zip(dims_list, ranks_list))]
    xs = [dev(x) for x in xs_np]
    res = gpu_lib.sthosvd_batched(xs, dims_list, 1e-3, precision=precision)
    assert len(res) == len(xs)
    assert all(p == "jacobi" for r in res for p in r.eig_paths)
    _check_batched_against_oracle(gpu_lib, xs_np, xs, dims_list, res, 1e-3)
    kc, ctas, ms = gpu_lib.batched_tuning()
    assert kc in (512, 2048, 8192) and ctas > 0 and min(ms) > 0


def test_batched_device_pipeline_edges(gpu_lib):
    """Four-way float32 tensors, keep-all (eps = 0), modes of length 1 and 128,
    a batch of one, and results freed in any order (they share one block)."""
    rng = np.random.default_rng(8)
    dims_list = [(12, 9, 7, 5), (1, 20, 3, 2), (128, 4, 3, 2), (17, 16, 15, 14)]
    xs_np = [rng.standard_normal(int(np.prod(d))).astype(np.float32) for d in dims_list]
    xs = [dev(x) for x in xs_np]
    res = gpu_lib.sthosvd_batched(xs, dims_list, 0.0)
    for d, r in zip(dims_list, res):
        assert r.ranks == d
    _check_batched_against_oracle(gpu_lib, xs_np, xs, dims_list, res, 0.0)
    res[0].free()
    res[2].free()
    g = res[3].core().cpu().numpy()  # the shared block is still held by the others
    assert np.isfinite(g).all()
    one = gpu_lib.sthosvd_batched([xs[1]], [dims_list[1]], 0.5)
    ref = oracle.sthosvd(xs_np[1].astype(np.float64), dims_list[1], 0.5)
    assert one[0].ranks == ref["ranks"]


def test_host_entry_point(gpu_lib):
    import torch

    dims, ranks = (24, 20, 18), (5, 4, 3)
    x = tucker_tensor_np(dims, ranks, seed=6, noise=1e-3)
    xh = torch.from_numpy(x).pin_memory()
    res_h = gpu_lib.sthosvd_host(xh, dims, 1e-2)
    res_d = gpu_lib.sthosvd(dev(x), dims, 1e-2)
    assert res_h.on_host and res_h.ranks == res_d.ranks
    assert torch.equal(res_h.core(), res_d.core().cpu())
    for n in range(3):
        assert torch.equal(res_h.factor(n), res_d.factor(n).cpu())


def test_host_entry_point_chunked_bf16(gpu_lib):
    """BF16 digits with mode 1 first: the host entry point copies X in column
    chunks (here 8: seven of 1024 columns and a ragged one of 32) and runs
    mode 1's Gram chunk by chunk.  Ranks equal the device call's, the result
    equals it up to the rounding of the chunk sum, and repeated calls agree
    bit for bit."""
    import torch

    dims, ranks = (64, 40, 30, 6), (6, 5, 4, 3)
    x = tucker_tensor_np(dims, ranks, seed=21, noise=1e-4)
    xh = torch.from_numpy(x).pin_memory()
    a = gpu_lib.sthosvd_host(xh, dims, 1e-3, precision="bf16x4")
    b = gpu_lib.sthosvd_host(xh, dims, 1e-3, precision="bf16x4")
    d = gpu_lib.sthosvd(dev(x), dims, 1e-3, precision="bf16x4")
    assert a.ranks == b.ranks == d.ranks
    assert torch.equal(a.core(), b.core())
    core_d = d.core().cpu()
    assert (a.core() - core_d).abs().max() <= 1e-9 * core_d.abs().max()
    for n in range(len(dims)):
        assert (a.factor(n) - d.factor(n).cpu()).abs().max() <= 1e-8
        assert a.tails[n] == pytest.approx(d.tails[n], rel=1e-9, abs=1e-15 * d.norm2)
    assert a.norm2 == pytest.approx(d.norm2, rel=1e-14)
    # pageable host memory: the chunk copies are staged by the driver, same result
    pg = gpu_lib.sthosvd_host(torch.from_numpy(x.copy()), dims, 1e-3, precision="bf16x4")
    assert pg.ranks == a.ranks and torch.equal(pg.core(), a.core())
    # float32 input takes the same chunked path
    x32 = x.astype(np.float32)
    h32 = gpu_lib.sthosvd_host(torch.from_numpy(x32).pin_memory(), dims, 1e-3, precision="bf16x4")
    d32 = gpu_lib.sthosvd(dev(x32), dims, 1e-3, precision="bf16x4")
    assert h32.ranks == d32.ranks
    c32 = d32.core().cpu()
    assert (h32.core() - c32).abs().max() <= 1e-9 * c32.abs().max()
    # mode 1 not first: one copy, the device call bit for bit
    order = (1, 0, 2, 3)
    h2 = gpu_lib.sthosvd_host(xh, dims, 1e-3, mode_order=order, precision="bf16x4")
    d2 = gpu_lib.sthosvd(dev(x), dims, 1e-3, mode_order=order, precision="bf16x4")
    assert h2.ranks == d2.ranks
    assert torch.equal(h2.core(), d2.core().cpu())


@pytest.mark.parametrize("dims", [(200, 40, 30), (65, 40, 30)])
def test_host_entry_point_chunked_other_grams(gpu_lib, dims):
    """The chunked first Gram on the other Gram paths: J = 200 (row blocks
    and their pairs) and J = 65 (520-byte columns, which the tensor map does
    not take: the register-staged kernel); 1200 columns make three chunks,
    the last one ragged."""
    import torch

    ranks = (8, 6, 5)
    x = tucker_tensor_np(dims, ranks, seed=22, noise=1e-4)
    a = gpu_lib.sthosvd_host(torch.from_numpy(x).pin_memory(), dims, 1e-3, precision="bf16x4")
    d = gpu_lib.sthosvd(dev(x), dims, 1e-3, precision="bf16x4")
    assert a.ranks == d.ranks
    core_d = d.core().cpu()
    assert (a.core() - core_d).abs().max() <= 1e-9 * core_d.abs().max()
    assert a.norm2 == pytest.approx(d.norm2, rel=1e-14)


@pytest.mark.parametrize("precision", ["bf16x4", "fp64"])
def test_host_many_matches_single_calls(gpu_lib, precision):
    """tucker_sthosvd_host_many on three different tensors (two device buffers
    in turn, each copy running while the previous tensor is compressed):
    every result is the single host call's, bit for bit."""
    import torch

    dims, ranks = (64, 40, 30, 6), (6, 5, 4, 3)
    xs = [torch.from_numpy(tucker_tensor_np(dims, ranks, seed=30 + k, noise=1e-4)).pin_memory() for k in range(3)]
    many = gpu_lib.sthosvd_host_many(xs, dims, 1e-3, precision=precision)
    assert len(many) == 3
    for x, m in zip(xs, many):
        one = gpu_lib.sthosvd_host(x, dims, 1e-3, precision=precision)
        assert m.on_host and m.ranks == one.ranks
        assert torch.equal(m.core(), one.core())
        for n in range(len(dims)):
            assert torch.equal(m.factor(n), one.factor(n))
    assert gpu_lib.sthosvd_host_many([], dims, 1e-3) == []
    single = gpu_lib.sthosvd_host_many(xs[:1], dims, 1e-3, precision=precision)
    assert torch.equal(single[0].core(), many[0].core())


def test_results_return_their_memory(gpu_lib):
    """A freed device result goes back to the stream-ordered pool and a freed
    host result's pinned block to the host block cache, so repeated calls hold
    no more memory than one."""
    import gc

    import torch

    dims, ranks = (40, 36, 30), (6, 5, 4)
    x = tucker_tensor_np(dims, ranks, seed=16, noise=1e-3)
    xd = dev(x)
    gpu_lib.sthosvd(xd, dims, 1e-2).free()
    gc.collect()
    torch.cuda.synchronize()
    before = gpu_lib.memory_stats()["pool_used"]
    for _ in range(6):
        r = gpu_lib.sthosvd(xd, dims, 1e-2)
        res_bytes = 8 * (math.prod(r.ranks) + sum(d * k for d, k in zip(dims, r.ranks)))
        held = gpu_lib.memory_stats()["pool_used"]
        r.free()
    assert held >= before + res_bytes  # a live result's core and factors are in the pool
    assert gpu_lib.memory_stats()["pool_used"] <= before

    xh = torch.from_numpy(x).pin_memory()
    first = gpu_lib.sthosvd_host(xh, dims, 1e-2)
    core0 = first.core()
    first.free()
    cached = gpu_lib.memory_stats()["host_cached"]
    assert cached >= res_bytes
    for _ in range(3):
        r = gpu_lib.sthosvd_host(xh, dims, 1e-2)
        assert gpu_lib.memory_stats()["host_cached"] < cached  # the block came from the cache
        assert torch.equal(r.core(), core0)
        r.free()
        assert gpu_lib.memory_stats()["host_cached"] == cached
    gpu_lib.memory_trim()
    assert gpu_lib.memory_stats()["host_cached"] == 0


def test_run_to_run_identical(gpu_lib):
    dims, ranks = (48, 40, 30, 12), (8, 8, 6, 4)
    x = dev(tucker_tensor_np(dims, ranks, seed=7, decay=0.1, noise=1e-5))
    a = gpu_lib.sthosvd(x, dims, 1e-4)
    b = gpu_lib.sthosvd(x, dims, 1e-4)
    assert a.ranks == b.ranks
    assert np.array_equal(a.core().cpu().numpy(), b.core().cpu().numpy())


def test_nonfinite_input_is_reported(gpu_lib):
    x = np.ones(60)
    x[17] = np.nan
    with pytest.raises(gpu_lib.TuckerError) as e:
        gpu_lib.sthosvd(dev(x), (3, 4, 5), 1e-3)
    assert e.value.status == -6


def test_host_side_fault_injection(gpu_lib, monkeypatch):
    dims = (6, 5, 4)
    xh = tucker_tensor_np(dims, (2, 2, 2), seed=8, noise=1e-3)
    x = dev(xh)
    for fault, status in (("noconv", -4), ("alloc", -2), ("nan", -6), ("timeout", -5)):
        monkeypatch.setenv("TUCKER_FAULT", fault)
        with pytest.raises(gpu_lib.TuckerError) as e:
            gpu_lib.sthosvd(x, dims, 5e-2)
        assert e.value.status == status
    monkeypatch.delenv("TUCKER_FAULT")
    # the context is still usable and the next call is correct
    assert gpu_lib.sthosvd(x, dims, 5e-2).ranks == oracle.sthosvd(xh, dims, 5e-2)["ranks"] == (2, 2, 2)


def test_timeout_flag_reported_and_next_call_succeeds(gpu_lib, monkeypatch):
    """TUCKER_FAULT=timeout raises, on the host, the device error flag that a
    tensor-core wait raises when it expires: the split-precision call returns
    TUCKER_ETIMEOUT, repeatedly, and the next call (whose tensor-core kernels
    allocate and free tensor memory again) succeeds with the oracle's ranks.
    No kernel is made to stall: a real expiry is not produced on the GPU."""
    dims = (24, 20, 16)
    xh = tucker_tensor_np(dims, (5, 4, 6), seed=2, noise=1e-4)
    x = dev(xh)
    monkeypatch.setenv("TUCKER_FAULT", "timeout")
    for _ in range(3):
        with pytest.raises(gpu_lib.TuckerError) as e:
            gpu_lib.sthosvd(x, dims, 1e-3, precision="bf16x4")
        assert e.value.status == -5
        assert "TUCKER_FAULT=timeout" in str(e.value)
    monkeypatch.delenv("TUCKER_FAULT")
    ref = oracle.sthosvd(xh, dims, 1e-3)
    for prec in ("bf16x4", "fp64"):
        r = gpu_lib.sthosvd(x, dims, 1e-3, precision=prec)
        assert r.ranks == ref["ranks"]
        r.free()


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "bf16x4"])
def test_small_modes_take_the_mixed_precision_solver(gpu_lib, seed, prec):
    """The modes of small Tucker-like tensors (J = 10..25) are solved by the
    verified mixed-precision solver, with no float64 Jacobi fallback."""
    dims, ranks = (24, 20, 16, 10), (5, 4, 6, 3)
    x = tucker_tensor_np(dims, ranks, seed=seed, decay=0.15, smooth=True, noise=1e-4)
    r = gpu_lib.sthosvd(dev(x), dims, 1e-3, precision=prec)
    assert r.eig_paths == ("mixed",) * 4, r.eig_paths
    r.free()
    dims, ranks = (25, 40, 30), (10, 10, 8)
    x = tucker_tensor_np(dims, ranks, seed=seed, noise=1e-6)
    r = gpu_lib.sthosvd(dev(x), dims, 1e-4, precision=prec)
    assert r.eig_paths == ("mixed",) * 3, r.eig_paths
    r.free()


@pytest.mark.parametrize("j", [10, 16, 20, 24, 25])
def test_eig_mp_strict_small_tucker_grams(gpu_lib, monkeypatch, j):
    """Strict mixed-precision solves (no fallback) of small Tucker-like Grams:
    a few signal eigenvalues within 10% of each other over a noise floor."""
    monkeypatch.setenv("TUCKER_EIG_KERNEL", "mp")
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1")
    rng = np.random.default_rng(100 + j)
    q, _ = np.linalg.qr(rng.standard_normal((j, j)))
    r = max(2, j // 3)
    sig = 1e3 * (1 + 0.1 * rng.standard_normal(r))
    lam = np.concatenate([sig, 1e-9 * sig.sum() * (1 + 0.1 * rng.random(j - r))])
    s = (q * lam) @ q.T
    _check_eig(gpu_lib, 0.5 * (s + s.T))


def test_eig_mp_strict_fifteen_wide_cluster(gpu_lib, monkeypatch):
    """Strict mixed-precision solve with 15 eigenvalues within 10% of each
    other at 1e-9 of the largest (a cluster the refinement must resolve)."""
    monkeypatch.setenv("TUCKER_EIG_KERNEL", "mp")
    monkeypatch.setenv("TUCKER_EIG_MP_STRICT", "1")
    rng = np.random.default_rng(15)
    j = 64
    q, _ = np.linalg.qr(rng.standard_normal((j, j)))
    lam = np.concatenate([0.7 ** np.arange(20), 1e-9 * (1 + 0.1 * rng.random(15)), 1e-13 * rng.random(j - 35)])
    s = (q * lam) @ q.T
    _check_eig(gpu_lib, 0.5 * (s + s.T))


def test_fp64_peak_probe(gpu_lib):
    """The float64 throughput probe lands in a plausible range for GB300
    (152 SMs x 2 float64 FMA per clock: ~1.26 TFLOP/s at 2.07 GHz)."""
    tf, ms = gpu_lib.fp64_peak()
    assert 0.3 < tf < 2.0, tf
    assert ms > 0
