"""GPU parity with open boundaries (the configuration's boundaries flag): the bonds that
would wrap around the torus along an open direction are absent.  The oracle's open
lattice is pinned by the geometric wrap classes of its bonds and the standing-wave
spectrum of the open square lattice.

Bars: iterates bit-exact against the oracle's fixed-rounding replica (FP32 and FP64: the
kernel reads a zero neighbour across the boundary, the replica adds the same zero);
moments 1e-12 (FP64) / 1e-5 (FP32) against the plain definition; 2D moments 1e-5 of
max |mu|; time evolution 1e-10 (FP64).  Open lattices run one recursion step per launch
(a pinned two-step pass falls back to it).
"""
import contextlib
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture(scope="module")
def ctx():
    c = kite.Context(0)
    yield c
    c.close()


@contextlib.contextmanager
def pass_steps(v):
    old = os.environ.get("KITE_PASS_STEPS")
    os.environ["KITE_PASS_STEPS"] = v
    try:
        yield
    finally:
        if old is None:
            del os.environ["KITE_PASS_STEPS"]
        else:
            os.environ["KITE_PASS_STEPS"] = old


CASES = [
    # (lattice, Lx, Ly, W, p_vac, R, M, open_x, open_y)
    (oracle.HONEYCOMB, 37, 29, 2.0, 0.02, 3, 48, 1, 0),   # ragged strip, open x
    (oracle.HONEYCOMB, 37, 29, 2.0, 0.02, 3, 48, 0, 1),   # open y
    (oracle.HONEYCOMB, 70, 9, 1.0, 0.0, 8, 33, 1, 1),     # 3 strips, odd M, both open
    (oracle.SQUARE, 300, 5, 3.0, 0.05, 1, 40, 1, 1),      # C=1, TX=256, ragged
    (oracle.SQUARE, 17, 40, 0.0, 0.0, 6, 25, 1, 0),       # padded batch
    (oracle.HONEYCOMB, 3, 2, 1.0, 0.1, 2, 16, 1, 1),      # tiny lattice
    (oracle.HONEYCOMB, 1, 3, 1.0, 0.0, 2, 9, 1, 0),       # one cell column, open x
    (oracle.SQUARE, 5, 1, 2.0, 0.0, 4, 12, 0, 1),         # one row, open y
]


def sysd(case, seed):
    lat, Lx, Ly, W, p, R, M, ox, oy = case
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    return dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, p_vac=p, seed=seed, open_x=ox, open_y=oy), R, M


def run(ctx, d, M, R, precision=kite.FP32, r0=None, want_last=False, doubling=False):
    n = oracle.norb(oracle.make_system(**d))
    r0a = None if r0 is None else np.ascontiguousarray(np.stack([r0.real, r0.imag], -1))
    dt = np.complex64 if precision == kite.FP32 else np.complex128
    last = np.zeros((R, 2, n), dt) if want_last else None
    kpm = kite.make_kpm(M, R, 1, precision, 0.0, 0.0, r0a, last, doubling=doubling)
    mu = np.zeros(M)
    muv = np.zeros((R, M, 2))
    st = kite.moments_1d(ctx, kite.make_system(**d), kpm, mu, muv)
    return mu, muv[..., 0] + 1j * muv[..., 1], last, st


@pytest.mark.parametrize("steps", ["1", "2"])
@pytest.mark.parametrize("case", CASES)
def test_open_fp32_iterates_bit_exact_against_replica(ctx, case, steps):
    d, R, M = sysd(case, 41)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=d["Lx"] * 100 + d["Ly"])
    with pass_steps(steps):
        mu, muv, last, st = run(ctx, d, M, R, r0=r0, want_last=True)
    assert st.steps_per_pass == 1
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 0, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint32), last_ref.view(np.uint32))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-6


@pytest.mark.parametrize("steps", ["1", "2"])
@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3], CASES[6]])
def test_open_fp64_iterates_bit_exact_against_replica(ctx, case, steps):
    d, R, M = sysd(case, 42)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=3)
    with pass_steps(steps):
        _, muv, last, st = run(ctx, d, M, R, precision=kite.FP64, r0=r0, want_last=True)
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 1, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint64), last_ref.view(np.uint64))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-12


@pytest.mark.parametrize("doubling", [False, True])
@pytest.mark.parametrize("prec,bar", [(kite.FP64, 1e-12), (kite.FP32, 1e-5)])
def test_open_moments_match_the_plain_definition(ctx, prec, bar, doubling):
    d = dict(lattice=oracle.HONEYCOMB, Lx=48, Ly=40, t=-2.7, W=1.5, delta=0.3, p_vac=0.02, seed=9,
             open_x=1, open_y=1)
    M, R = 96, 3
    mu, muv, _, _ = run(ctx, d, M, R, precision=prec, doubling=doubling)
    ref = oracle.moments_1d(oracle.make_system(**d), M, R)
    assert np.max(np.abs(muv - ref)) <= bar
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar


@pytest.mark.parametrize("prec,bar", [(kite.FP64, 1e-12), (kite.FP32, 1e-5)])
def test_field_on_an_open_strip(ctx, prec, bar):
    """With y open the flux need not fit the torus (0.1 per cell on a 24-row strip)."""
    for lat, t in ((oracle.HONEYCOMB, -2.7), (oracle.SQUARE, -1.0)):
        d = dict(lattice=lat, Lx=40, Ly=24, t=t, W=1.0, p_vac=0.02, seed=5, flux=0.1, open_y=1)
        M, R = 64, 2
        _, muv, _, _ = run(ctx, d, M, R, precision=prec)
        ref = oracle.moments_1d(oracle.make_system(**d), M, R)
        assert np.max(np.abs(muv - ref)) <= bar
    assert kite.flux_nearest(kite.make_system(kite.HONEYCOMB, 40, 24, -2.7, 0.0, flux=0.1, open_y=1), 0.1) == 0.1


@pytest.mark.parametrize("alpha,beta", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("lat", [oracle.HONEYCOMB, oracle.SQUARE])
def test_open_2d_moments_match_oracle(ctx, lat, alpha, beta):
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    d = dict(lattice=lat, Lx=37, Ly=20, t=t, W=1.0, p_vac=0.02, seed=4, open_x=1, open_y=1)
    M, R = 40, 2
    mu = np.zeros((M, M, 2))
    kite.moments_2d(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, kite.FP32), mu, alpha, beta)
    ref = oracle.moments_2d(oracle.make_system(**d), M, R, alpha=alpha, beta=beta)
    got = mu[..., 0] + 1j * mu[..., 1]
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_open_2d_moments_with_a_field(ctx):
    d = dict(lattice=oracle.HONEYCOMB, Lx=30, Ly=16, t=-2.7, W=0.5, seed=6, flux=0.05, open_y=1)
    M, R = 32, 2
    mu = np.zeros((M, M, 2))
    kite.moments_2d(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, kite.FP32), mu, 0, 1)
    ref = oracle.moments_2d(oracle.make_system(**d), M, R, alpha=0, beta=1)
    assert np.max(np.abs(mu[..., 0] + 1j * mu[..., 1] - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_open_time_evolution_matches_oracle(ctx):
    d = dict(lattice=oracle.SQUARE, Lx=33, Ly=21, t=-1.0, W=0.5, seed=3, open_x=1, open_y=1)
    o = oracle.make_system(**d)
    n = oracle.norb(o)
    psi0 = synth.unit_phase_vectors(n, 1, seed=8)[0] / np.sqrt(n)
    dt, steps, M = 0.7, 3, 40
    psi = np.ascontiguousarray(np.stack([psi0.real, psi0.imag], -1)[None])
    kite.propagate(ctx, kite.make_system(**d), kite.make_kpm(M, 1, 1, kite.FP64), dt, steps, psi)
    ref = oracle.propagate(o, psi0, dt, steps, M)[-1]
    assert np.max(np.abs(psi[0, :, 0] + 1j * psi[0, :, 1] - ref)) <= 1e-10


def test_calls_without_open_boundaries_refuse_them(ctx):
    s = kite.make_system(kite.SQUARE, 16, 16, -1.0, 0.0, open_x=1)
    with pytest.raises(kite.KiteError):
        kite.moments_1d_batched(ctx, [s], [kite.make_kpm(8, 2, 1, kite.FP32)], [np.zeros(8)])
    with pytest.raises(kite.KiteError):
        kite.moments_1d_static(s, kite.make_kpm(8, 2, 1, kite.FP32), np.zeros(8))
    bad = kite.make_system(kite.SQUARE, 16, 16, -1.0, 0.0)
    bad.open_x = 2  # neither periodic (0) nor open (1)
    with pytest.raises(kite.KiteError) as e:
        kite.moments_1d(ctx, bad, kite.make_kpm(8, 1, 1, kite.FP32), np.zeros(8))
    assert e.value.status == kite.ERR_ARG
