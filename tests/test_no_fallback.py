"""Host side: the product path has no CPU or library fallback.

Without the in-tree CUDA library, or without a CUDA device, every entry point of the binding
raises instead of computing something else.  Runs without a GPU.
"""
import numpy as np
import pytest
import torch

import paper_2106_00449_gb300 as g


@pytest.fixture(scope="module")
def built():
    """The in-tree library, built here if needed (no device calls are made)."""
    import os
    from paper_2106_00449_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "libgdc.so"))
    with pytest.raises(ImportError, match="is missing"):
        g.load_library()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_contexts_refuse_to_run_without_a_cuda_device():
    with pytest.raises(RuntimeError, match="needs a CUDA device"):
        g.Fcm(32, 10.0, 0.5642, 3.0, max_blobs=4)
    with pytest.raises(RuntimeError, match="needs a CUDA device"):
        g.Context(g.Params(), [np.zeros((1, 3))], np.zeros(1, np.int32), np.array([0, 1], np.int64),
                  np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0, 0.0]]))


def test_device_entry_points_reject_host_tensors(built):
    r = torch.zeros(6, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensors"):
        g.rpy_apply_noalloc(r, r.clone())
    with pytest.raises(ValueError, match="CUDA tensor"):
        g.fma_probe(torch.zeros(256, dtype=torch.float32))
