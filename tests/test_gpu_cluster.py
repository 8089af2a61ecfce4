"""GPU parity of the small-lattice cluster sweep (kite_moments_1d with the iterates held on
chip, one thread-block cluster per real recursion): KITE_CLUSTER=1 forces it where it
applies, KITE_CLUSTER_CTAS pins the CTAs per cluster (2 to 16).

Bars (as for the streaming kernels):
  * iterates: bit-exact against the oracle's fixed-rounding replica (FP32 and FP64), on
    ragged row splits, one row per CTA, vacancies and open boundaries;
  * moments: <= 1e-12 (FP64) and <= 1e-5 (FP32) against the plain FP64 definition, plain
    and with moment doubling, complex and real start vectors, several vector batches and
    realisations, more clusters than fit on the GPU at once;
  * the imaginary part of each moment is not formed (it vanishes for a real symmetric H~)
    and is reported as exactly 0.
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
def env(**kv):
    old = {k: os.environ.get(k) for k in kv}
    for k, v in kv.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    try:
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def run(ctx, d, M, R, S=1, precision=kite.FP32, r0=None, want_last=False, doubling=False,
        real_vectors=False, e_min=0.0, e_max=0.0, ctas=None, force="1"):
    n = oracle.norb(oracle.make_system(**d))
    r0a = None if r0 is None else np.ascontiguousarray(np.stack([r0.real, r0.imag], -1))
    dt = np.complex64 if precision == kite.FP32 else np.complex128
    last = np.zeros((S * R, 2, n), dt) if want_last else None
    kpm = kite.make_kpm(M, R, S, precision, e_min, e_max, r0a, last, doubling=doubling,
                        real_vectors=real_vectors)
    mu = np.zeros(M)
    muv = np.zeros((S * R, M, 2))
    with env(KITE_CLUSTER=force, KITE_CLUSTER_CTAS=None if ctas is None else str(ctas)):
        st = kite.moments_1d(ctx, kite.make_system(**d), kpm, mu, muv)
    return mu, muv[..., 0] + 1j * muv[..., 1], last, st


def sysd(lat, Lx, Ly, W=1.0, delta=0.0, p=0.0, seed=7, **kw):
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    return dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, delta=delta, p_vac=p, seed=seed, **kw)


BITWISE = [
    # (system, R, M, CTAs per cluster)
    (sysd(oracle.HONEYCOMB, 37, 29, W=2.0, p=0.02), 3, 48, 16),   # 29 rows over 16: 2 and 1
    (sysd(oracle.HONEYCOMB, 37, 29, W=2.0, p=0.02), 3, 48, 8),
    (sysd(oracle.HONEYCOMB, 37, 29, W=2.0, p=0.02), 3, 48, 12),
    (sysd(oracle.SQUARE, 17, 40), 6, 25, 5),                      # odd cluster size
    (sysd(oracle.HONEYCOMB, 70, 9, delta=0.5), 8, 33, 8),         # 9 rows over 8
    (sysd(oracle.SQUARE, 17, 40), 6, 25, 16),
    (sysd(oracle.SQUARE, 64, 16, W=3.0, p=0.05), 1, 40, 16),      # one row per CTA
    (sysd(oracle.HONEYCOMB, 64, 64), 4, 64, 16),                  # the 64 x 64 workload's lattice
    (sysd(oracle.HONEYCOMB, 1, 12, p=0.1), 2, 20, 8),             # one cell per row: x wraps onto itself
]


@pytest.mark.parametrize("precision", [kite.FP32, kite.FP64])
@pytest.mark.parametrize("case", BITWISE)
def test_cluster_iterates_bit_exact_against_replica(ctx, case, precision):
    d, R, M, cs = case
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=d["Lx"] * 1000 + d["Ly"])
    mu, muv, last, st = run(ctx, d, M, R, precision=precision, r0=r0, want_last=True, ctas=cs)
    assert st.cluster_ctas == cs and st.steps_per_pass == M - 1
    fp64 = precision == kite.FP64
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 1 if fp64 else 0, r0=r0,
                                         want_last=True)
    u = np.uint64 if fp64 else np.uint32
    assert np.array_equal(last.view(u), last_ref.view(u))
    assert np.max(np.abs(muv.real - mu_ref.real)) <= (1e-12 if fp64 else 1e-6)
    assert np.all(muv.imag == 0.0)
    _, vac = oracle.disorder(oracle.make_system(**d))
    assert st.n_eff == int((vac == 0).sum())


OPEN = [
    (sysd(oracle.HONEYCOMB, 33, 20, W=2.0, p=0.03, open_x=1, open_y=0), 3, 40, 16),
    (sysd(oracle.HONEYCOMB, 33, 20, W=2.0, p=0.03, open_x=0, open_y=1), 3, 40, 8),
    (sysd(oracle.SQUARE, 40, 17, W=1.0, open_x=1, open_y=1), 5, 30, 16),
]


@pytest.mark.parametrize("case", OPEN)
def test_cluster_open_boundaries_bit_exact_against_replica(ctx, case):
    d, R, M, cs = case
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=99)
    mu, muv, last, st = run(ctx, d, M, R, r0=r0, want_last=True, ctas=cs)
    assert st.cluster_ctas == cs
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 0, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint32), last_ref.view(np.uint32))
    assert np.max(np.abs(muv.real - mu_ref.real)) <= 1e-6


MOMENTS = [
    # (system, M, R, S, precision, doubling, real vectors, bar)
    (sysd(oracle.HONEYCOMB, 64, 64, seed=1), 256, 4, 1, kite.FP64, False, False, 1e-12),
    (sysd(oracle.HONEYCOMB, 64, 64, seed=1), 256, 4, 1, kite.FP64, True, False, 1e-12),
    (sysd(oracle.HONEYCOMB, 96, 80, W=2.0, p=0.005, seed=2), 512, 8, 1, kite.FP32, False, False, 1e-5),
    (sysd(oracle.HONEYCOMB, 37, 29, W=2.0, delta=0.5, p=0.02, seed=8), 3, 3, 1, kite.FP64, True, False, 1e-12),
    (sysd(oracle.SQUARE, 17, 40, seed=3), 2, 1, 1, kite.FP32, True, False, 1e-5),
    (sysd(oracle.SQUARE, 17, 40, seed=3), 1, 1, 1, kite.FP64, False, False, 1e-12),
    (sysd(oracle.SQUARE, 17, 40, seed=3), 1, 1, 1, kite.FP64, True, False, 1e-12),
    (sysd(oracle.HONEYCOMB, 24, 20, W=2.0, p=0.02, seed=9), 65, 6, 2, kite.FP64, False, False, 1e-12),
    (sysd(oracle.HONEYCOMB, 24, 20, W=2.0, p=0.02, seed=9), 65, 6, 2, kite.FP32, True, False, 1e-5),
    # real vectors: 8 FP64 lanes; 16 FP32 lanes x 16 CTAs, more clusters than fit at once
    (sysd(oracle.HONEYCOMB, 64, 64, seed=1), 256, 8, 1, kite.FP64, False, True, 1e-12),
    (sysd(oracle.HONEYCOMB, 40, 32, W=2.0, p=0.01, seed=4), 200, 16, 1, kite.FP32, False, True, 1e-5),
    (sysd(oracle.SQUARE, 30, 24, W=1.0, seed=5), 97, 19, 1, kite.FP32, True, True, 1e-5),
]


@pytest.mark.parametrize("case", MOMENTS)
def test_cluster_moments_match_oracle(ctx, case):
    d, M, R, S, prec, dbl, realv, bar = case
    o = oracle.make_system(**d)
    mu, muv, _, st = run(ctx, d, M, R, S=S, precision=prec, doubling=dbl, real_vectors=realv)
    assert 2 <= st.cluster_ctas <= 16
    per_batch = (16 if prec == kite.FP32 else 8) if realv else (8 if prec == kite.FP32 else 4)
    batches = S * -(-R // per_batch)
    assert st.step_launches == batches
    assert st.steps_per_pass == ((M + 1) // 2 if dbl else M - 1)
    refs = []
    for s in range(S):
        r0 = oracle.random_real(o, R, s) if realv else None
        refs.append(oracle.moments_1d(o, M, R, realisation=s, r0=r0))
    ref = np.concatenate(refs, 0)
    assert np.max(np.abs(muv.real - ref.real)) <= bar
    assert np.all(muv.imag == 0.0)
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar


def test_cluster_sweep_is_deterministic_and_matches_the_streaming_kernels(ctx):
    d = sysd(oracle.HONEYCOMB, 64, 64, seed=1)
    b = (3 * 2.7 + 0.5) * 1.01
    a = run(ctx, d, 256, 4, precision=kite.FP64, e_min=-b, e_max=b)
    a2 = run(ctx, d, 256, 4, precision=kite.FP64, e_min=-b, e_max=b)
    s = run(ctx, d, 256, 4, precision=kite.FP64, e_min=-b, e_max=b, force="0")
    assert a[3].cluster_ctas > 0 and s[3].cluster_ctas == 0
    assert np.array_equal(a[0], a2[0])
    # the same iterates, the moment sums in another order
    assert np.max(np.abs(a[0] - s[0])) <= 1e-14


def test_cluster_sweep_needs_four_rows_and_no_field(ctx):
    d = sysd(oracle.SQUARE, 300, 3, W=3.0, p=0.05)
    mu, muv, _, st = run(ctx, d, 33, 2)
    assert st.cluster_ctas == 0  # 3 rows: the streaming kernels
    ref = oracle.moments_1d(oracle.make_system(**d), 33, 2)
    assert np.max(np.abs(muv - ref)) <= 1e-5
    k = kite.make_system(kite.HONEYCOMB, 32, 32, -2.7, 1.0, 0.0, 0.0, 3)
    k = kite.make_system(kite.HONEYCOMB, 32, 32, -2.7, 1.0, 0.0, 0.0, 3, flux=kite.flux_nearest(k, 1.0 / 8))
    mu = np.zeros(16)
    with env(KITE_CLUSTER="1"):
        st = kite.moments_1d(ctx, k, kite.make_kpm(16, 2, 1, kite.FP64), mu)
    assert st.cluster_ctas == 0  # complex H~: the field sweep


def test_autotuned_choice_on_the_64x64_workload(ctx):
    """Unforced, the autotuner picks the cluster sweep or the streaming kernels by measured
    time; either way the moments hold the FP64 bar."""
    d = sysd(oracle.HONEYCOMB, 64, 64, seed=1)
    b = (3 * 2.7 + 0.5) * 1.01
    for dbl in (False, True):
        mu, muv, _, st = run(ctx, d, 256, 4, precision=kite.FP64, e_min=-b, e_max=b, doubling=dbl, force=None)
        ref = oracle.moments_1d(oracle.make_system(**d), 256, 4, e_min=-b, e_max=b)
        print(f"64x64 FP64 M=256 R=4 doubling={dbl}: cluster CTAs {st.cluster_ctas}, "
              f"{st.seconds * 1e3:.3f} ms, {st.step_seconds * 1e3:.3f} ms in the steps")
        assert np.max(np.abs(muv.real - ref.real)) <= 1e-12


@pytest.mark.parametrize("prec,M,bar,dbl", [(kite.FP64, 1500, 1e-12, False), (kite.FP64, 1501, 1e-12, True),
                                           (kite.FP32, 2048, 1e-5, False)])
def test_cluster_long_sweeps_against_oracle(ctx, prec, M, bar, dbl):
    """Long sweeps on chip (many 16-moment transposes, a partial last one): FP64 within 1e-12
    of the oracle, FP32 at the large-DOS workload's order within 1e-5."""
    d = sysd(oracle.HONEYCOMB, 64, 48, W=2.0, p=0.005, seed=6)
    mu, muv, _, st = run(ctx, d, M, 4, precision=prec, doubling=dbl)
    assert st.cluster_ctas >= 2
    ref = oracle.moments_1d(oracle.make_system(**d), M, 4)
    assert np.max(np.abs(muv.real - ref.real)) <= bar
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar
