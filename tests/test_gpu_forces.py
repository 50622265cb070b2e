"""GPU: pair forces between blobs of different bodies, through the C ABI.

The soft sphere of Sec. 6.3 and the repel-attract / repel-attract-repel potentials of
Sec. 6.4, summed over every pair in tiles or over the cell list, against the dense oracle
(oracle.forces); at 65,520 blobs on sampled bodies the oracle sums one blob at a time
(oracle.matfree).  The cell list and the tiles must agree on every configuration: blobs
closer than 2a, pairs in the wells and beyond the cutoff, several suspensions.
"""
import dataclasses

import numpy as np
import pytest

from oracle import forces, geometry as G, matfree, philox
from oracle import gdc as ogdc
from synthetic import shapes
from synthetic import workloads as WL

from gpu_common import oracle_params, rel, rot_err, susp_layout

pytestmark = pytest.mark.gpu

WELLS = dict(well_A=5.0, well_lambda=0.5)   # Sec. 6.4 with kT = a = 1


def _host(t):
    return t.detach().cpu().numpy()


def _with(wl, **params):
    return dataclasses.replace(wl, params=dict(wl.params, **params))


def _overlapping():
    """A mixed suspension with bodies moved onto their neighbours (blobs closer than 2a)."""
    wl = WL.mixed_small(40, seed=5)
    Y = wl.Y.copy()
    for p in range(0, 12, 2):
        Y[p + 1] = Y[p] + np.array([0.9, 0.4, -0.3]) * (1 + p / 12)
    return dataclasses.replace(wl, Y=Y)


def _oracle_FT(wl):
    pp = wl.params
    out = []
    for s in range(wl.n_susp):
        lay, Y, q = susp_layout(wl, s)
        r = G.blob_positions(lay, Y, q)
        f = forces.blob_forces(r, lay.blob_body, pp["rep_A"], pp["rep_b"], pp["a"], pp.get("potential", 0),
                               pp.get("well_A", 0.0), pp.get("well_lambda", 0.5))
        out.append(forces.body_force_torque(r, Y, lay.blob_body, f))
    return np.concatenate(out)


def _gpu_FT(lib, wl, prec, method):
    ctx = lib.context_from_workload(wl, precision=prec, force_method=method)
    return _host(ctx.forces())


@pytest.mark.parametrize("potential", [0, 1, 2])
@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_forces_match_oracle(lib, prec, method, potential):
    wl = _with(_overlapping(), potential=potential, **WELLS)
    lay, Y, q = susp_layout(wl, 0)
    r = G.blob_positions(lay, Y, q)
    d = np.linalg.norm(r[:, None] - r[None], axis=2)[lay.blob_body[:, None] != lay.blob_body[None]]
    assert d.min() < 2.0 and ((d > 2.5) & (d < 4.0)).sum() > 100   # overlaps and well pairs present
    ref = _oracle_FT(wl)
    got = _gpu_FT(lib, wl, prec, method)
    assert np.abs(ref).max() > 0
    assert rel(got, ref) < (1e-12 if prec == 0 else 1e-5), rel(got, ref)


@pytest.mark.parametrize("method", [1, 2])
def test_forces_batched_suspensions(lib, method):
    # several suspensions share the cell hash table: no pair may cross suspensions
    wl = _with(WL.batch_small(6, seed=3), potential=2, rep_A=40.0, rep_b=0.5, **WELLS)
    ref = _oracle_FT(wl)
    got = _gpu_FT(lib, wl, 0, method)
    assert np.abs(ref).max() > 0
    assert rel(got, ref) < 1e-12, rel(got, ref)


@pytest.mark.parametrize("potential", [0, 2])
def test_cell_list_equals_all_pairs_at_2560_blobs(lib, potential):
    wl = _with(WL.c2(seed=4), potential=potential, **WELLS)
    ref = _oracle_FT(wl)
    for prec, tol in ((0, 1e-12), (1, 1e-5)):
        cell = _gpu_FT(lib, wl, prec, 2)
        pairs = _gpu_FT(lib, wl, prec, 1)
        assert rel(cell, ref) < tol and rel(pairs, ref) < tol, (prec, rel(cell, ref), rel(pairs, ref))
        if prec == 0:
            assert rel(cell, pairs) < 1e-13


def test_forces_without_neighbours_are_zero(lib):
    # bodies further apart than the cutoff: every cell search comes back empty
    wl = WL.c1()
    wl = dataclasses.replace(_with(wl, rep_A=4.0, potential=1, **WELLS), Y=wl.Y * 10.0)
    for method in (1, 2):
        assert np.abs(_gpu_FT(lib, wl, 0, method)).max() == 0.0


def test_forces_sampled_bodies_65k(lib):
    """The bench's workload with the repel-attract wells: the cell list (chosen at this size)."""
    wl = _with(WL.c3_65k(), potential=1, **WELLS)
    ctx = lib.context_from_workload(wl, precision=lib.FP32_MIXED, autotune=0)
    FT = _host(ctx.forces()).reshape(-1, 6)
    lay, Y, q = susp_layout(wl, 0)
    r = G.blob_positions(lay, Y, q)
    rng = np.random.default_rng(31)
    bodies = np.concatenate([[0, wl.n_bodies - 1], rng.choice(wl.n_bodies, 22, replace=False)])
    boff = np.concatenate([[0], np.cumsum(wl.tmpl_nblobs[wl.body_tmpl])])
    pp = wl.params
    ref = []
    for p in bodies:
        rows = np.arange(boff[p], boff[p + 1])
        f = matfree.repulsion_rows(r, lay.blob_body, rows, pp["rep_A"], pp["rep_b"], 1.0, 1, WELLS["well_A"],
                                   WELLS["well_lambda"])
        ref.append(np.concatenate([f.sum(axis=0), np.cross(r[rows] - Y[p], f).sum(axis=0)]))
    ref = np.array(ref)
    assert np.abs(ref).max() > 0
    err = np.abs(FT[bodies] - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err


def test_step_with_repel_attract_repel_matches_oracle(lib):
    wl = _with(WL.mixed_small(40, seed=1), potential=2, rep_A=40.0, rep_b=0.5, **WELLS)
    seed = 77
    ctx = lib.context_from_workload(wl, precision=0, seed=seed, gmres_tol=1e-12, lanczos_tol=1e-11,
                                    gmres_max_iter=1000, lanczos_max_iter=128, force_method=2)
    info = ctx.step(1)[0]
    assert info["solve"]["converged"]
    Y1, q1, _ = ctx.get_state()
    lay, Y, q = susp_layout(wl, 0)
    W = philox.normals(seed, 0, 0, 0, 3 * lay.n_blobs)
    Wt = philox.normals(seed, 0, 0, 1, 6 * lay.n_bodies)
    ora = ogdc.gdc_step(lay, Y, q, W, Wt, oracle_params(wl))
    # the wells act in this configuration
    r = G.blob_positions(lay, Y, q)
    f = forces.blob_forces(r, lay.blob_body, 40.0, 0.5, 1.0, 2, **WELLS)
    f_soft = forces.blob_forces(r, lay.blob_body, 40.0, 0.5, 1.0, 0)
    assert np.abs(f - f_soft).max() > 0.1
    assert rel(Y1 - Y, ora["Y1"] - Y) < 1e-6
    assert rot_err(q1, ora["q1"]) < 1e-9


def _pile():
    """Twelve 42-blob icospheres around nearly one centre: most blobs have more than the
    list's 32 partners closer than 2a (the FP32 product then searches the suspension)."""
    rng = np.random.default_rng(8)
    n = 12
    return WL.Workload("overlap_pile", [shapes.icosphere42()], np.zeros(n, dtype=np.int32),
                       np.array([0, n], dtype=np.int64), rng.uniform(-0.3, 0.3, size=(n, 3)),
                       WL.random_unit_quaternions(rng, n), dict(WL.c1().params), np.array([10.0]))


def _overlapping_65k():
    wl = WL.c3_65k()
    Y = wl.Y.copy()
    for p in range(0, 400, 2):
        Y[p + 1] = Y[p] + np.array([0.9, 0.4, -0.3]) * (1 + p / 400)
    return dataclasses.replace(wl, Y=Y)


@pytest.mark.parametrize("which", ["pairs", "pile", "65k"])
def test_near_pair_lists_do_not_depend_on_the_search(lib, which):
    """The FP32 product corrects the pairs closer than 2a from per-blob lists; the cell list
    must build the lists the all-pairs search builds, so that the products agree bit for bit."""
    import torch
    wl = {"pairs": _overlapping, "pile": _pile, "65k": _overlapping_65k}[which]()
    rng = np.random.default_rng(41)
    lam = torch.as_tensor(rng.standard_normal(3 * wl.n_blobs), device="cuda")
    out = []
    for method in (1, 2):
        ctx = lib.context_from_workload(wl, precision=lib.FP32_MIXED, autotune=0, pair_kernel=2, force_method=method)
        out.append(ctx.rpy_apply(lam, lib.FP32_MIXED).clone())
    assert torch.equal(out[0], out[1])
