"""The allocation-free moment call (kite_moments_1d_static).

It exists for callers that cannot allocate device memory when they need moments -- a host
framework whose caching allocator already holds the GPU's memory, or a latency-critical
loop that must not wait on the allocator.  It must give the same moments as the regular
kite_moments_1d (same kernels; the tolerance the other tests use: 1e-12 in FP64, 1e-6 in
FP32 between two GPU paths), also on the second of two calls in a row, since every call
reuses the same fixed device array and must clear what it needs.  This file is collected
last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture(scope="module")
def ctx():
    c = kite.Context(0)
    yield c
    c.close()


CASES = [
    (dict(lattice=kite.HONEYCOMB, Lx=64, Ly=64, t=-2.7, W=1.0, seed=1), 256, 4, kite.FP64, 1e-12),
    (dict(lattice=kite.HONEYCOMB, Lx=70, Ly=41, t=-2.7, W=2.0, p_vac=0.01, seed=3), 200, 8, kite.FP32, 1e-6),
    (dict(lattice=kite.SQUARE, Lx=130, Ly=50, t=-1.0, W=3.0, seed=5), 128, 3, kite.FP32, 1e-6),
]
# several realisations with vacancies: N_eff differs between them, and each realisation's
# moments are normalised by its own
CASES_S = [
    (dict(lattice=kite.HONEYCOMB, Lx=50, Ly=37, t=-2.7, W=1.5, p_vac=0.03, seed=11), 96, 4, 3, kite.FP64, 1e-12),
    (dict(lattice=kite.SQUARE, Lx=61, Ly=44, t=-1.0, W=2.0, p_vac=0.05, seed=12), 150, 5, 3, kite.FP32, 1e-6),
]


@pytest.mark.parametrize("d,M,R,prec,tol", CASES)
def test_static_call_matches_regular_call_twice(ctx, d, M, R, prec, tol):
    system = kite.make_system(**d)
    ref = np.zeros(M)
    kite.moments_1d(ctx, system, kite.make_kpm(M, R, 2, prec), ref)
    for _ in range(2):  # the second call reuses the array the first one left behind
        mu = np.zeros(M)
        kite.moments_1d_static(system, kite.make_kpm(M, R, 2, prec), mu)
        assert np.max(np.abs(mu - ref)) <= tol


@pytest.mark.parametrize("d,M,R,S,prec,tol", CASES_S)
def test_static_call_with_several_realisations_and_vacancies(ctx, d, M, R, S, prec, tol):
    system = kite.make_system(**d)
    ref = np.zeros(M)
    kite.moments_1d(ctx, system, kite.make_kpm(M, R, S, prec), ref)
    mu = np.zeros(M)
    kite.moments_1d_static(system, kite.make_kpm(M, R, S, prec), mu)
    assert np.max(np.abs(mu - ref)) <= tol


def test_static_call_allocates_no_device_memory(ctx):
    """After the first call on the device (which reserves the fixed array and loads the
    kernels' code), further calls leave the device's free memory unchanged."""
    import torch
    system = kite.make_system(kite.HONEYCOMB, 64, 48, -2.7, 1.0, 0.0, 0.02, 21)
    kpm = kite.make_kpm(128, 4, 2, kite.FP32)
    mu = np.zeros(128)
    kite.moments_1d_static(system, kpm, mu)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        kite.moments_1d_static(system, kpm, mu)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_call_rejects_systems_beyond_its_array():
    system = kite.make_system(kite.HONEYCOMB, 2048, 2048, -2.7, 1.0)
    mu = np.zeros(16)
    with pytest.raises(kite.KiteError) as e:
        kite.moments_1d_static(system, kite.make_kpm(16, 8, 1, kite.FP32), mu)
    assert e.value.status == kite.ERR_ARG and "KiB" in str(e.value)
