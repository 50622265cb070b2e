"""Bounded waits of the FP32 pair kernels run out and are reported, without any GPU fault.

gdc_debug_wait_polls(-1) makes the pair kernels' first wait for each source-tile copy give
up without polling, as a copy that never lands would.  The kernel then waits, with the
normal bound, for its copies in flight, flags the context's status word and returns early;
the call reports GDC_ERR_TIMEOUT, a host-driven step leaves the state unchanged, and once
the default bound is restored the same context computes correct products and steps again.
"""
import numpy as np
import pytest

from synthetic import workloads as WL

from gpu_common import dense_state, rel, susp_layout

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", [1, 2])
def test_pair_kernel_timeout_is_reported_and_the_context_recovers(lib, kernel):
    wl = WL.mixed_small(40, seed=1)
    ctx = lib.context_from_workload(wl, autotune=0, pair_kernel=kernel, precision=lib.FP32_MIXED, graph=0,
                                    rfd_delta=1e-3, lanczos_max_iter=16, gmres_max_iter=40)
    lam = np.random.default_rng(41).standard_normal(3 * wl.n_blobs)
    Y0, q0, s0 = ctx.get_state()
    try:
        lib.debug_wait_polls(-1)
        with pytest.raises(lib.GdcError) as ei:
            ctx.rpy_apply(lam, lib.FP32_MIXED)
        assert ei.value.status == 5
        with pytest.raises(lib.GdcError) as ei:
            ctx.step(1)
        assert ei.value.status == 5
        Y1, q1, s1 = ctx.get_state()
        assert s1 == s0
        np.testing.assert_array_equal(Y1, Y0)
        np.testing.assert_array_equal(q1, q0)
    finally:
        lib.debug_wait_polls(0)
    u = ctx.rpy_apply(lam, lib.FP32_MIXED).cpu().numpy()
    lay, Y, q = susp_layout(wl, 0)
    r, M, K, B = dense_state(lay, Y, q)
    assert rel(u, M @ lam) < 2e-6
    info = ctx.step(1)[0]
    assert info["solve"]["converged"]
    assert ctx.get_state()[2] == s0 + 1
