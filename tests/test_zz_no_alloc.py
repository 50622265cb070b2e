"""The allocation-free RPY product (gdc_rpy_apply_noalloc) against the context-based one.

gdc_rpy_apply_noalloc serves callers that cannot allocate device memory (a program that
owns all device memory through its own fixed pool, or a loop that cannot afford the
synchronisation of cudaMalloc/cudaFree): it uses a fixed scratch array inside the
library.  This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test; it passes alone or after the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_blob_context(lib, r):
    """Context of single-blob bodies at positions r: its FP32 RPY product is the reference."""
    templates = [np.zeros((1, 3))]
    n = r.shape[0]
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    return lib.Context(lib.Params(autotune=0), templates, np.zeros(n, dtype=np.int32), np.array([0, n]), r, q)


def _call_noalloc(lib, r_dev, lam_dev, u_dev, n, torch):
    clib = lib.load_library()
    s = torch.cuda.current_stream()
    st = clib.gdc_rpy_apply_noalloc(ctypes.c_void_p(r_dev.data_ptr()), ctypes.c_void_p(lam_dev.data_ptr()),
                                    ctypes.c_void_p(u_dev.data_ptr()), n, 1.0, 1.0, ctypes.c_void_p(s.cuda_stream))
    return st


def _cloud(rng, n, kind):
    if kind == "clump":
        # every blob within 0.8a of the centre: all pairs closer than 2a, more than the 32
        # near pairs a blob's list holds, so the product searches the whole suspension
        v = rng.standard_normal((n, 3))
        return 0.8 * v / np.linalg.norm(v, axis=1, keepdims=True) * rng.uniform(0, 1, size=(n, 1)) ** (1 / 3)
    # a dense random cloud: many pairs closer than 2a, so the overlap branch is exercised
    return rng.uniform(0.0, 1.6 * max(n, 1) ** (1.0 / 3.0), size=(n, 3))


@pytest.mark.parametrize("sizes", [((3000, "cloud"), (1337, "cloud")),
                                   ((16384, "cloud"), (1, "cloud")),
                                   ((40, "clump"), (700, "cloud"))])
def test_noalloc_matches_context_product_on_two_calls(lib, sizes):
    """Two calls in a row (the second after a larger or smaller first call) against the
    context-based products; sizes up to GDC_NOALLOC_MAX_BLOBS, a single blob, and a clump
    whose blobs all overlap."""
    import torch
    rng = np.random.default_rng(31)
    for call, (n, kind) in enumerate(sizes):
        r = _cloud(rng, n, kind)
        lam = rng.standard_normal(3 * n)
        ctx = _free_blob_context(lib, r)
        ref32 = ctx.rpy_apply(lam, lib.FP32_MIXED)
        ref64 = ctx.rpy_apply(lam, lib.FP64)
        r_dev = torch.as_tensor(r.reshape(-1), device="cuda")
        lam_dev = torch.as_tensor(lam, device="cuda")
        u_dev = torch.full_like(lam_dev, float("nan"))
        assert _call_noalloc(lib, r_dev, lam_dev, u_dev, n, torch) == 0, lib.load_library().gdc_last_error(None)
        torch.cuda.synchronize()
        assert torch.isfinite(u_dev).all()
        err32 = ((u_dev - ref32).norm() / ref32.norm()).item()
        err64 = ((u_dev - ref64).norm() / ref64.norm()).item()
        assert err32 < 2e-6, (call, n, err32)
        assert err64 < 2e-6, (call, n, err64)
        # the Python wrapper gives the same result
        u2 = lib.rpy_apply_noalloc(r_dev, lam_dev)
        torch.cuda.synchronize()
        assert torch.equal(u2, u_dev)


def test_noalloc_timeout_shows_as_nan_and_the_next_call_is_clean(lib):
    """A pair-kernel wait that runs out (forced with gdc_debug_wait_polls) makes every entry
    of u NaN, since the asynchronous call cannot return a status; the next call clears the
    flag and is correct again."""
    import torch
    rng = np.random.default_rng(33)
    n = 2000
    r = _cloud(rng, n, "cloud")
    lam = rng.standard_normal(3 * n)
    ref64 = _free_blob_context(lib, r).rpy_apply(lam, lib.FP64)
    r_dev = torch.as_tensor(r.reshape(-1), device="cuda")
    lam_dev = torch.as_tensor(lam, device="cuda")
    u_dev = torch.zeros_like(lam_dev)
    try:
        lib.debug_wait_polls(-1)
        assert _call_noalloc(lib, r_dev, lam_dev, u_dev, n, torch) == 0
        torch.cuda.synchronize()
    finally:
        lib.debug_wait_polls(0)
    assert torch.isnan(u_dev).all()
    assert _call_noalloc(lib, r_dev, lam_dev, u_dev, n, torch) == 0
    torch.cuda.synchronize()
    assert ((u_dev - ref64).norm() / ref64.norm()).item() < 2e-6


def test_noalloc_wrapper_rejects_mismatched_tensors(lib):
    import torch
    r = torch.zeros(30, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        lib.rpy_apply_noalloc(r, torch.zeros(30, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        lib.rpy_apply_noalloc(r, torch.zeros(27, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        lib.rpy_apply_noalloc(torch.zeros(31, dtype=torch.float64, device="cuda"),
                              torch.zeros(31, dtype=torch.float64, device="cuda"))


def test_noalloc_rejects_oversized_input(lib):
    import torch
    n = lib.NOALLOC_MAX_BLOBS + 1
    r = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    st = _call_noalloc(lib, r, r, r, n, torch)
    assert st == 1
    assert b"n_blobs must be in [1, 16384]" in lib.load_library().gdc_last_error(None)
