"""GPU: the step replayed as one CUDA graph (Lanczos and GMRES loops as conditional WHILE
nodes) against the host-driven step, through the C ABI.

The graph runs the same kernels in the same order with the same arguments, only with the
Krylov iteration index read from device memory, so states, iteration counts, residuals
and nu must agree bit for bit.  Failures must leave the state where it was, as the
host-driven path does by returning early.
"""
import dataclasses

import numpy as np
import pytest

from synthetic import workloads as WL

pytestmark = pytest.mark.gpu


def _pair(lib, wl, **kw):
    return (lib.context_from_workload(wl, graph=1, **kw), lib.context_from_workload(wl, graph=0, **kw))


def _same_info(a, b):
    for k in ("step", "lanczos_iters", "lanczos_err", "nu_min", "nu_max", "pair_evals"):
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("iterations", "cycles", "matvecs_fp32", "matvecs_fp64", "residual", "converged"):
        assert a["solve"][k] == b["solve"][k], (k, a["solve"][k], b["solve"][k])


@pytest.mark.parametrize("case", ["c1_fp64", "mix_fp32", "batch_fp32", "rod_fp32", "mix_em_fp64", "mix_fp32_restart4"])
def test_graph_step_is_bitwise_the_host_driven_step(lib, case):
    if case == "c1_fp64":
        wl, kw = WL.c1(), dict(precision=0, gmres_tol=1e-10, lanczos_tol=1e-8)
    elif case == "mix_fp32":
        wl, kw = WL.mixed_small(40, seed=1), dict(precision=1, rfd_delta=1e-3)
    elif case == "batch_fp32":
        wl, kw = WL.batch_small(6, seed=3), dict(precision=1, rfd_delta=1e-3)
    elif case == "rod_fp32":
        wl, kw = WL.c2(seed=2, n_rods=60, box=37.0), dict(precision=1, rfd_delta=1e-3)
    elif case == "mix_em_fp64":
        wl, kw = WL.mixed_small(40, seed=1), dict(precision=0, scheme=1)
    else:   # short restarts: cycles with residual updates (the graph's IF/ELSE node)
        wl, kw = WL.mixed_small(40, seed=1), dict(precision=1, rfd_delta=1e-3, gmres_restart=4, gmres_max_iter=800)
    g, e = _pair(lib, wl, **kw)
    ig = g.step(3)
    ie = e.step(3)
    for a, b in zip(ig, ie):
        _same_info(a, b)
    Yg, qg, sg = g.get_state()
    Ye, qe, se = e.get_state()
    assert sg == se == 3
    np.testing.assert_array_equal(Yg, Ye)
    np.testing.assert_array_equal(qg, qe)


def test_graph_trace_and_parameter_changes(lib):
    wl = WL.batch_small(6, seed=3)
    g, e = _pair(lib, wl, precision=1, rfd_delta=1e-3)
    g.step(1)
    e.step(1)
    # a trace set after the first capture is honoured (the graph is captured again)
    tg, te = g.set_trace(True), e.set_trace(True)
    g.step(1)
    e.step(1)
    for k in tg:
        np.testing.assert_array_equal(tg[k].cpu().numpy(), te[k].cpu().numpy())
    # so is a parameter change
    for ctx in (g, e):
        ctx.set_params(dataclasses.replace(ctx.params, dt=0.5 * ctx.params.dt, gmres_tol=1e-7))
    _same_info(g.step(1)[0], e.step(1)[0])
    np.testing.assert_array_equal(g.get_state()[0], e.get_state()[0])
    np.testing.assert_array_equal(g.get_state()[1], e.get_state()[1])


def test_graph_step_after_host_driven_steps_and_set_state(lib):
    # the step counter the draws use follows set_state and host-driven steps
    wl = WL.mixed_small(40, seed=1)
    g, e = _pair(lib, wl, precision=1, rfd_delta=1e-3)
    Y0, q0, _ = g.get_state()
    g.profile(True)          # profiling uses the host-driven path
    g.step(1)
    g.profile(False)
    g.step(1)
    e.step(2)
    np.testing.assert_array_equal(g.get_state()[0], e.get_state()[0])
    g.set_state(Y0, q0, 5)
    e.set_state(Y0, q0, 5)
    _same_info(g.step(1)[0], e.step(1)[0])
    np.testing.assert_array_equal(g.get_state()[1], e.get_state()[1])


@pytest.mark.parametrize("which", ["gmres", "lanczos"])
def test_graph_failure_leaves_the_state(lib, which):
    wl = WL.c1()
    bad = dict(gmres_tol=1e-15, gmres_max_iter=2) if which == "gmres" else dict(lanczos_tol=1e-15, lanczos_max_iter=2)
    ctx = lib.context_from_workload(wl, graph=1, precision=0, **bad)
    Y0, q0, s0 = ctx.get_state()
    with pytest.raises(lib.GdcError) as ei:
        ctx.step(1)
    assert ei.value.status == 3   # GDC_ERR_NOT_CONVERGED
    Y1, q1, s1 = ctx.get_state()
    assert s1 == s0
    np.testing.assert_array_equal(Y0, Y1)
    np.testing.assert_array_equal(q0, q1)
    # usable afterwards, with sane parameters (kT = 0: no Lanczos, whose basis size is fixed at init)
    ok = lib.context_from_workload(wl, graph=0, precision=0, kT=0.0, lanczos_max_iter=ctx.params.lanczos_max_iter)
    ctx.set_params(dataclasses.replace(ok.params, graph=1))
    _same_info(ctx.step(1)[0], ok.step(1)[0])
    np.testing.assert_array_equal(ctx.get_state()[0], ok.get_state()[0])


def test_graph_kernel_count(lib):
    """Executed kernels = host-driven kernels + the loop-control kernels of the graph.

    kT = 0 leaves only the GMRES loops: per step 3 step-level kernels (report reset, ok
    flag, report), and for the solve one reset, one finish, a check per cycle boundary
    (cycles + 1), a cycle start per cycle, a loop-control kernel per inner iteration and a
    counter per accurate residual product.
    """
    wl = WL.mixed_small(40, seed=1)
    g, e = _pair(lib, wl, precision=1, kT=0.0)
    g.step(1)
    e.step(1)
    counts = []
    for ctx in (g, e):
        ctx.profile(False)   # resets the counter, keeps the graph path
        inf = ctx.step(1)[0]
        counts.append((ctx.profile_read()["launches"], inf))
    (ng, ig), (ne, ie) = counts
    _same_info(ig, ie)
    cyc, it, acc = ig["solve"]["cycles"], ig["solve"]["iterations"], ig["solve"]["matvecs_fp64"]
    assert ng - ne == 3 + 1 + 1 + (cyc + 1) + cyc + it + acc, (ng, ne, cyc, it, acc)
