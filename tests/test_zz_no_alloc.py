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


@pytest.mark.parametrize("sizes", [(3000, 1337)])
def test_noalloc_matches_context_product_on_two_calls(lib, sizes):
    import torch
    rng = np.random.default_rng(31)
    for call, n in enumerate(sizes):
        # a dense random cloud: many pairs closer than 2a, so the overlap branch is exercised
        r = rng.uniform(0.0, 1.6 * n ** (1.0 / 3.0), size=(n, 3))
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
        assert err32 < 2e-6, (call, err32)
        assert err64 < 2e-6, (call, err64)


def test_noalloc_rejects_oversized_input(lib):
    import torch
    n = lib.NOALLOC_MAX_BLOBS + 1
    r = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    st = _call_noalloc(lib, r, r, r, n, torch)
    assert st == 1
    assert b"n_blobs must be in [1, 16384]" in lib.load_library().gdc_last_error(None)
