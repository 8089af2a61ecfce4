"""GPU parity of Gaussian on-site disorder (the 'Gaussian' kind of the paper's Python
interface, Sec. 3d) against the oracle.

The device draws V = W sqrt(-2 ln(1 - u)) cos(2 pi u2) with CUDA's FP64 log, sqrt and cos
and the oracle with the host's libm: the two agree to an ulp or two, so the bars are the
ones the tests against the plain FP64 definition use (1e-12 with FP64 vectors, 1e-5 with
FP32 vectors); vacancies (the third Philox word) and N_eff are exact.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture(scope="module")
def ctx():
    c = kite.Context(0)
    yield c
    c.close()


def both(**d):
    return (kite.make_system(disorder=kite.DISORDER_GAUSSIAN, **d),
            oracle.make_system(disorder=oracle.GAUSSIAN, **d))


def test_bounds_cover_the_largest_gaussian_draw():
    for lat in (oracle.HONEYCOMB, oracle.SQUARE):
        k, o = both(lattice=lat, Lx=16, Ly=16, t=-2.7, W=0.6, delta=0.2 if lat == 0 else 0.0, seed=3)
        lo, hi = kite.bounds(k)
        olo, ohi = oracle.bounds_auto(o)
        assert lo == olo and hi == ohi


def test_exact_trace_pins_the_device_draws(ctx):
    """Basis start vectors give the exact trace: mu_1 = mean(V~) and mu_2 carry the device's
    Gaussian on-site energies and vacancies; FP64 against the oracle's draws."""
    k, o = both(lattice=oracle.SQUARE, Lx=9, Ly=7, t=-1.0, W=1.3, p_vac=0.1, seed=19)
    n = oracle.norb(o)
    eye = np.eye(n, dtype=np.complex128)
    r0a = np.ascontiguousarray(np.stack([eye.real, eye.imag], -1))
    muv = np.zeros((n, 20, 2))
    st = kite.moments_1d(ctx, k, kite.make_kpm(20, n, 1, kite.FP64, r0=r0a), np.zeros(20), muv)
    ref = oracle.moments_1d(o, 20, n, r0=eye)
    got = muv[..., 0] + 1j * muv[..., 1]
    assert np.max(np.abs(got.sum(0) - ref.sum(0))) <= 1e-12
    _, vac = oracle.disorder(o)
    assert st.n_eff == int((vac == 0).sum())


@pytest.mark.parametrize("prec,bar", [(kite.FP64, 1e-12), (kite.FP32, 1e-5)])
def test_gaussian_moments_match_oracle(ctx, prec, bar):
    k, o = both(lattice=oracle.HONEYCOMB, Lx=64, Ly=48, t=-2.7, W=0.8, delta=0.3, p_vac=0.02, seed=23)
    M, R, S = 128, 3, 2
    mu = np.zeros(M)
    muv = np.zeros((S * R, M, 2))
    kite.moments_1d(ctx, k, kite.make_kpm(M, R, S, prec), mu, muv)
    ref = np.concatenate([oracle.moments_1d(o, M, R, realisation=s) for s in range(S)], 0)
    assert np.max(np.abs(muv[..., 0] + 1j * muv[..., 1] - ref)) <= bar
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar


def test_gaussian_batched_and_static_paths(ctx):
    """The batched sweep (moment doubling) and the allocation-free call draw the same
    Gaussian disorder."""
    specs = [(40, 0.5, 11), (72, 1.5, 12)]
    pairs = [both(lattice=oracle.SQUARE, Lx=L, Ly=L, t=-1.0, W=W, seed=sd) for L, W, sd in specs]
    M, R = 64, 4
    mus = [np.zeros(M) for _ in pairs]
    kite.moments_1d_batched(ctx, [p[0] for p in pairs], [kite.make_kpm(M, R, 1, kite.FP32, doubling=True)
                                                        for _ in pairs], mus)
    for (k, o), mu in zip(pairs, mus):
        ref = oracle.moments_1d(o, M, R).real.mean(0)
        assert np.max(np.abs(mu - ref)) <= 1e-5
    k, o = pairs[0]
    mu_s, mu_r = np.zeros(M), np.zeros(M)
    kite.moments_1d_static(k, kite.make_kpm(M, R, 2, kite.FP64), mu_s)
    kite.moments_1d(ctx, k, kite.make_kpm(M, R, 2, kite.FP64), mu_r)
    assert np.max(np.abs(mu_s - mu_r)) <= 1e-12


def test_unknown_disorder_kind_is_rejected(ctx):
    s = kite.make_system(kite.HONEYCOMB, 8, 8, -2.7, 1.0, disorder=7)
    with pytest.raises(kite.KiteError) as e:
        kite.moments_1d(ctx, s, kite.make_kpm(8, 1, 1, kite.FP32), np.zeros(8))
    assert e.value.status == kite.ERR_ARG
