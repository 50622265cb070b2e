"""The FP32 FMA throughput probe (the measured denominator of the pair kernels' roofline):
its chains converge to the fixed point of x <- a x + b, and the scalar, packed and mixed
forms compute the same values bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_modes_agree_and_reach_the_fixed_point(lib):
    import torch
    outs = []
    for mode in (0, 1, 2):
        out = torch.empty(2 * 256, dtype=torch.float32, device="cuda")
        assert lib.fma_probe(out, mode, iters=20000) == 2 * 256 * 20000 * 32
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    # after 20,000 steps a^n < 1e-8: every chain sits at b / (1 - a) = 1 in both lanes
    np.testing.assert_allclose(outs[0], np.full(512, 16.0), rtol=1e-3)
    with pytest.raises(RuntimeError):
        lib.fma_probe(torch.empty(256, dtype=torch.float32, device="cuda"), 3)
