"""GPU: fluctuating FCM of Sec. 4.2 in a periodic cube, through the C ABI, against the oracle.

The library's grid arithmetic is FP32: spreading sums, three FFT passes of log2 N radix-2
stages each way and the averaging rows carry relative rounding errors of a few 1e-7 each,
so products agree with the FP64 oracle to about 1e-6; the tests allow 2e-5.  The stress
draws are the same Philox numbers on both sides (stream 2), so the Brownian velocities are
compared sample for sample.
"""
import numpy as np
import pytest

from oracle import fcm

from gpu_common import rel

pytestmark = pytest.mark.gpu

SIGMA = 1.0 / np.sqrt(np.pi)     # a = 1
TOL = 2e-5

# (N, L, R_t, blobs): two binning cells per side, a few, many; sigma/h from 1.8 to 1.8 at 128^3
CASES = [(16, 5.0, 2.0, 7), (32, 10.0, 3.0, 40), (64, 20.0, 3.0, 300), (128, 40.0, 3.0, 3000)]


def _host(t):
    return t.detach().cpu().numpy()


def _positions(n, L, seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, L, size=(n, 3))
    r[: n // 5] += L * rng.integers(-2, 3, size=(n // 5, 3))    # outside the cube: wrapped by both sides
    return r


@pytest.mark.parametrize("N,L,R_t,n", CASES)
def test_fcm_product_matches_oracle(lib, N, L, R_t, n):
    r = _positions(n, L, N)
    lam = np.random.default_rng(N + 1).standard_normal((n, 3))
    F = lib.Fcm(N, L, SIGMA, R_t, max_blobs=n)
    u = _host(F.apply(r, lam))
    ref = fcm.mobility_apply(fcm.Grid(N, L, SIGMA, R_t), r, lam)
    assert rel(u, ref) < TOL, rel(u, ref)
    # deterministic: the gather and the fixed summation orders repeat bit for bit
    np.testing.assert_array_equal(_host(F.apply(r, lam)), u)


@pytest.mark.parametrize("N,L,R_t,n", CASES[:3])
def test_fcm_brownian_matches_oracle(lib, N, L, R_t, n):
    g = fcm.Grid(N, L, SIGMA, R_t)
    r = _positions(n, L, N + 2)
    seed, owner, step, kT, dt = 2024, 3, 17, 1.3, 0.01
    F = lib.Fcm(N, L, SIGMA, R_t, max_blobs=n)
    v = _host(F.brownian(r, seed, owner, step, kT, dt))
    ref, u_ref = fcm.brownian_velocity(g, r, seed, owner, step, kT, dt)
    assert rel(v, ref) < TOL, rel(v, ref)
    # the field stays on the grid: re-averaging at moved positions (Sec. 5) needs no new solve
    r2 = r + 0.4 * np.random.default_rng(5).standard_normal(r.shape)
    v2 = _host(F.average(r2))
    assert rel(v2, fcm.average(g, r2, u_ref)) < TOL
    # a deterministic product in between leaves the fluctuating field alone
    F.apply(r, np.ones((n, 3)))
    np.testing.assert_array_equal(_host(F.average(r2)), v2)


def test_fcm_rejects_bad_input(lib):
    with pytest.raises(lib.GdcError):
        lib.Fcm(24, 10.0, SIGMA, 3.0)            # not a power of two
    with pytest.raises(lib.GdcError):
        lib.Fcm(32, 10.0, SIGMA, 5.0)            # truncation reaches the periodic image
    F = lib.Fcm(32, 10.0, SIGMA, 3.0, max_blobs=4)
    with pytest.raises(lib.GdcError):
        F.average(np.zeros((2, 3)))              # no fluctuating field yet
    with pytest.raises(lib.GdcError):
        F.apply(np.zeros((5, 3)), np.zeros((5, 3)))   # more blobs than max_blobs
    before = F.launches
    F.apply(np.ones((3, 3)), np.ones((3, 3)))
    assert F.launches > before
