"""The Gram entry point that allocates nothing (tucker_gram_noalloc).

It exists for callers that cannot allocate device memory themselves, such
as a process whose framework has already reserved nearly all of the GPU's
memory for its own pool, or code that must not trigger the device-wide
synchronisation an allocation can cause.  Its split-K scratch is a static
device array shared by every call, so these checks call it twice in a row
on each shape and compare both results with tucker_gram, within the Gram
tolerance of the parity tests (twice the rigorous dot-product bound
gamma_K (|Y||Y|^T)_ij, one bound per computed side).

This file is collected last so that a failure here cannot hide another
test's result in a run that stops at the first failure; it must also pass
when run alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _bound(y, L, J, B):
    t = y.reshape((L, J, B), order="F")
    yn = np.moveaxis(t, 1, 0).reshape(J, -1, order="F")
    k = L * B
    g = k * U / (1 - k * U)
    return 2 * g * (np.abs(yn) @ np.abs(yn).T)


@pytest.mark.parametrize("L,J,B", [(1, 128, 5000), (40, 128, 33), (7, 13, 5), (2, 512, 40), (1, 1, 1)])
def test_noalloc_gram_matches_gram_twice(gpu_lib, L, J, B):
    import torch

    rng = np.random.default_rng(L * 131 + J * 7 + B)
    y = rng.standard_normal(L * J * B)
    yd = torch.from_numpy(y).cuda()
    ref = gpu_lib.gram(yd, L, J, B).cpu().numpy()
    bound = _bound(y, L, J, B)
    for _ in range(2):
        got = gpu_lib.gram_noalloc(yd, L, J, B).cpu().numpy()
        assert np.array_equal(got, got.T)
        assert np.all(np.abs(got - ref) <= bound + 1e-300)


def test_noalloc_gram_float32_and_reuse_after_larger_call(gpu_lib):
    import torch

    rng = np.random.default_rng(3)
    big = torch.from_numpy(rng.standard_normal(2 * 512 * 40)).cuda()
    gpu_lib.gram_noalloc(big, 2, 512, 40)  # leaves large partial sums in the shared scratch
    L, J, B = 9, 24, 31
    y = rng.standard_normal(L * J * B).astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    ref = gpu_lib.gram(yd, L, J, B).cpu().numpy()
    for _ in range(2):
        got = gpu_lib.gram_noalloc(yd, L, J, B).cpu().numpy()
        assert np.all(np.abs(got - ref) <= _bound(y.astype(np.float64), L, J, B))


def test_noalloc_gram_rejects_oversize(gpu_lib):
    import torch

    y = torch.zeros(1025 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.TuckerError) as e:
        gpu_lib.gram_noalloc(y, 1, 1025, 2, out=torch.empty((1025, 1025), dtype=torch.float64, device="cuda"))
    assert e.value.status == -1
    assert "1025" in str(e.value)


CAP_SHAPES = [(1, 1024, 4000), (1, 256, 20000), (1, 512, 8000)]


def _run_capped(gpu_lib, monkeypatch, capfd, L, J, B):
    """Two noalloc calls against tucker_gram; returns whether the split plan
    needed more partial sums than the static scratch holds."""
    import torch

    rng = np.random.default_rng(J + B)
    y = rng.standard_normal(L * J * B)
    yd = torch.from_numpy(y).cuda()
    ref = gpu_lib.gram(yd, L, J, B).cpu().numpy()
    bound = _bound(y, L, J, B)
    monkeypatch.setenv("TUCKER_NOALLOC_TRACE", "1")
    for _ in range(2):
        got = gpu_lib.gram_noalloc(yd, L, J, B).cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound + 1e-300)
    monkeypatch.delenv("TUCKER_NOALLOC_TRACE")
    err = capfd.readouterr().err
    line = [ln for ln in err.splitlines() if ln.startswith("tucker_gram_noalloc:")][-1]
    kv = dict(tok.split("=") for tok in line.split()[1:])
    assert int(kv["used_splits"]) <= int(kv["scratch_fits"])
    return int(kv["planned_splits"]) > int(kv["scratch_fits"])


@pytest.mark.parametrize("L,J,B", CAP_SHAPES)
def test_noalloc_gram_caps_splits_to_the_scratch(gpu_lib, monkeypatch, capfd, L, J, B):
    """Shapes whose split plan can need more partial sums than the static
    scratch holds: the call then runs fewer, longer column ranges and still
    matches tucker_gram (checked twice in a row)."""
    _run_capped(gpu_lib, monkeypatch, capfd, L, J, B)


def test_noalloc_cap_is_reached(gpu_lib, monkeypatch, capfd):
    """At least one of those shapes takes the capped branch on this GPU."""
    assert any(_run_capped(gpu_lib, monkeypatch, capfd, *shape) for shape in CAP_SHAPES)
