"""CPU checks of the C ABI: the library loads, exports what the header declares,
and rejects invalid arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_06689_gb300 import build, tucker

    build.build()
    return tucker.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "tucker.h")).read()
    return sorted(set(re.findall(r"TUCKER_API[^;(]*?\b(tucker_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("tucker_sthosvd", "tucker_reconstruct", "tucker_rel_error", "tucker_result_free"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1510_06689_gb300 import tucker

    names = header_functions()
    assert sorted(tucker.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.tucker_status_string(0) == b"ok"
    assert lib.tucker_status_string(-1) == b"invalid argument"
    assert lib.tucker_status_string(-4) == b"eigensolver did not converge"
    assert lib.tucker_status_string(12345) == b"unknown status"


def test_invalid_arguments_are_rejected_on_host(lib):
    from paper_1510_06689_gb300 import tucker

    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    res = tucker._Result()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    # NULL tensor
    assert lib.tucker_sthosvd(None, 0, dims, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    assert b"NULL" in lib.tucker_last_error()
    # bad N, bad dims, NaN eps, bad order, bad dtype, bad precision
    assert lib.tucker_sthosvd(fake, 0, dims, 0, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    bad = (ctypes.c_int64 * 3)(4, 0, 6)
    assert lib.tucker_sthosvd(fake, 0, bad, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    big = (ctypes.c_int64 * 3)(4, 5000, 6)
    assert lib.tucker_sthosvd(fake, 0, big, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    assert lib.tucker_sthosvd(fake, 0, dims, 3, float("nan"), None, 0, None, ctypes.byref(res)) == -1
    order = (ctypes.c_int * 3)(0, 0, 2)
    assert lib.tucker_sthosvd(fake, 0, dims, 3, 1e-3, order, 0, None, ctypes.byref(res)) == -1
    assert b"permutation" in lib.tucker_last_error()
    assert lib.tucker_sthosvd(fake, 7, dims, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    assert lib.tucker_sthosvd(fake, 0, dims, 3, 1e-3, None, 9, None, ctypes.byref(res)) == -1
    assert lib.tucker_sthosvd(fake, 0, dims, 3, 1e-3, None, 0, None, None) == -1
    # step entry points
    out = ctypes.c_double()
    assert lib.tucker_norm2(None, 0, 10, ctypes.byref(out), None) == -1
    assert lib.tucker_gram(fake, 0, 1, 0, 1, fake, None) == -1
    assert lib.tucker_gram(fake, 0, 1, 2000, 1, fake, None) == -1
    assert lib.tucker_eig(fake, 0, fake, fake, None, None) == -1
    r, t = ctypes.c_int64(), ctypes.c_double()
    assert lib.tucker_rank_cut(fake, 4, float("nan"), 0, ctypes.byref(r), ctypes.byref(t), None) == -1
    assert lib.tucker_ttm(fake, 0, 1, 3, 1, fake, 0, 1, fake, None) == -1
    # results
    assert lib.tucker_reconstruct(ctypes.byref(res), fake, None) == -1
    rel = ctypes.c_double()
    assert lib.tucker_rel_error(fake, 0, ctypes.byref(res), ctypes.byref(rel), None) == -1
    lib.tucker_result_free(ctypes.byref(res))  # safe on an empty result
    lib.tucker_result_free(None)


def test_profile_counters_without_gpu(lib):
    from paper_1510_06689_gb300 import tucker

    tucker.profile_enable(True)
    p = tucker.profile_read()
    assert set(p) == set(tucker.PHASES)
    assert all(v["ms"] == 0 and v["launches"] == 0 for v in p.values())
    tucker.profile_enable(False)
    assert tucker.launch_count() >= 0


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1510_06689_gb300 import tucker

    saved = tucker._lib
    tucker._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            tucker.load(str(tmp_path / "missing.so"))
    finally:
        tucker._lib = saved


def test_mode_order_and_flops_match_the_oracle(lib):
    """Host-only entry points of the mode-order heuristics (Sec. 8.3) against the oracle."""
    import numpy as np

    from oracle import st_hosvd as osth
    from paper_1510_06689_gb300 import tucker

    rng = np.random.default_rng(0)
    cases = [((25, 250, 250, 250), (10, 10, 100, 100)), ((128, 128, 128, 48, 32), (40, 40, 40, 20, 10)),
             ((4, 6), (2, 3)), ((7,), (3,))]
    for _ in range(20):
        n = int(rng.integers(2, 7))
        dims = tuple(int(d) for d in rng.integers(2, 300, n))
        ranks = tuple(int(rng.integers(1, d + 1)) for d in dims)
        cases.append((dims, ranks))
    for dims, ranks in cases:
        for rule in ("flops", "ratio"):
            assert tucker.mode_order(dims, ranks, rule) == osth.greedy_order(dims, ranks, rule), (dims, ranks, rule)
        assert tucker.mode_order(dims, ranks, "exhaustive") == osth.best_order(dims, ranks)
        for order in (None, tucker.mode_order(dims, ranks, "ratio")):
            ref = osth.order_flops(dims, ranks, list(range(len(dims))) if order is None else order)
            assert tucker.order_flops(dims, ranks, order) == pytest.approx(ref, rel=1e-12)


def test_hooi_subtensor_and_order_arguments_rejected_on_host(lib):
    from paper_1510_06689_gb300 import tucker

    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    ranks = (ctypes.c_int64 * 3)(2, 6, 3)  # rank 6 > I_2 = 5
    order = (ctypes.c_int * 3)()
    flops = ctypes.c_double()
    assert lib.tucker_mode_order(dims, ranks, 3, 0, order) == -1
    good = (ctypes.c_int64 * 3)(2, 2, 3)
    assert lib.tucker_mode_order(dims, good, 3, 7, order) == -1  # unknown rule
    assert lib.tucker_mode_order(dims, good, 3, 0, None) == -1
    bad_order = (ctypes.c_int * 3)(0, 0, 2)
    assert lib.tucker_order_flops(dims, good, 3, bad_order, ctypes.byref(flops)) == -1
    res = tucker._Result()
    iters = ctypes.c_int()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    assert lib.tucker_hooi(fake, 0, dims, 3, 1e-3, -1, 0.0, 0, None, ctypes.byref(res), ctypes.byref(iters), None) == -1
    assert lib.tucker_hooi(fake, 0, dims, 3, 1e-3, 2, float("nan"), 0, None, ctypes.byref(res), ctypes.byref(iters),
                           None) == -1
    lo = (ctypes.c_int64 * 3)(0, 0, 0)
    assert lib.tucker_reconstruct_sub(ctypes.byref(res), lo, lo, fake, None) == -1  # empty result


def test_batched_arguments_rejected_on_host(lib):
    from paper_1510_06689_gb300 import tucker

    res = (tucker._Result * 2)()
    dims = (ctypes.c_int64 * 6)(4, 5, 6, 4, 0, 6)  # second tensor has a zero size
    fake = (ctypes.c_void_p * 2)(0x1000, 0x2000)   # never dereferenced: validation fails first
    assert lib.tucker_sthosvd_batched(fake, 0, dims, 3, 2, 1e-3, 0, 0, None, res) == -1
    good = (ctypes.c_int64 * 6)(4, 5, 6, 4, 5, 6)
    null_x = (ctypes.c_void_p * 2)(0x1000, None)
    assert lib.tucker_sthosvd_batched(null_x, 0, good, 3, 2, 1e-3, 0, 0, None, res) == -1
    assert lib.tucker_sthosvd_batched(fake, 0, good, 3, 2, 1e-3, 0, 65, None, res) == -1  # too many workers
    assert lib.tucker_sthosvd_batched(fake, 0, good, 3, 0, 1e-3, 0, 0, None, res) == 0    # nothing to do


def test_gram_noalloc_binding_checks_buffers_before_the_call(lib):
    """The C side cannot see a tensor's type or size, so the binding rejects a
    wrong output buffer or a short input before calling it."""
    import torch

    from paper_1510_06689_gb300 import tucker

    y = torch.zeros(4 * 5 * 6, dtype=torch.float64)
    with pytest.raises(tucker.TuckerError, match="elements"):
        tucker.gram_noalloc(y[:-1], 4, 5, 6)
    for bad in (torch.zeros((5, 5), dtype=torch.float32), torch.zeros((4, 5), dtype=torch.float64),
                torch.zeros((5, 5), dtype=torch.float64), torch.zeros((5, 10), dtype=torch.float64)[:, ::2]):
        with pytest.raises(tucker.TuckerError, match="out must be"):
            tucker.gram_noalloc(y, 4, 5, 6, out=bad)
