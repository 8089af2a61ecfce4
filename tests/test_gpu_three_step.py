"""GPU parity of the three-step pass (temporal blocking of depth three: Eq. e6 applied
three times per pass, r_{n+1} kept on chip, the moments of Eqs. e7/e8 of all three
iterates fused in).  KITE_PASS_STEPS=3 pins it for the call; the last one or two steps of
a sweep take the one-step kernel or the two-step pass.

Bars (as for the two-step pass):
  * iterates: bit-exact against the oracle's fixed-rounding replica, FP32 and FP64, halo
    sites of both on-chip levels included;
  * moments: <= 1e-6 against the replica's moments (FP32 partials), <= 1e-12 for FP64,
    <= 1e-5 against the plain FP64 definition.
Lattices cover ragged right strips, lattices narrower than the three-cell halo (it wraps
more than once), a single row, every remainder of M - 2 modulo 3, padded and real batches.
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


def run(ctx, d, M, R, precision=kite.FP32, r0=None, want_last=False, real_vectors=False, S=1, steps="3"):
    s = kite.make_system(**d)
    n = oracle.norb(oracle.make_system(**d))
    r0a = None
    if r0 is not None:
        r0a = np.ascontiguousarray(np.stack([r0.real, r0.imag], -1).astype(np.float64))
    dt = np.complex64 if precision == kite.FP32 else np.complex128
    last = np.zeros((S * R, 2, n), dt) if want_last else None
    kpm = kite.make_kpm(M, R, S, precision, 0.0, 0.0, r0a, last, real_vectors=real_vectors)
    mu = np.zeros(M, np.float64)
    muv = np.zeros((S * R, M, 2), np.float64)
    with pass_steps(steps):
        st = kite.moments_1d(ctx, s, kpm, mu, muv)
    return mu, muv[..., 0] + 1j * muv[..., 1], last, st


CASES = [
    # (lattice, Lx, Ly, W, delta, p_vac, R, M)      M - 2 mod 3: remainder after the passes
    (oracle.HONEYCOMB, 37, 29, 2.0, 0.0, 0.02, 3, 48),   # 1: one-step remainder; C=2, ragged
    (oracle.HONEYCOMB, 70, 9, 1.0, 0.5, 0.0, 8, 33),     # 1; C=4, 3 strips
    (oracle.SQUARE, 300, 5, 3.0, 0.0, 0.05, 1, 40),      # 2: two-step remainder; C=1, TX=256
    (oracle.SQUARE, 17, 40, 0.0, 0.0, 0.0, 6, 29),       # 0: passes only; C=4 (6 padded to 8)
    (oracle.HONEYCOMB, 3, 2, 1.0, 0.0, 0.1, 2, 16),      # 2; narrower than the halo
    (oracle.HONEYCOMB, 1, 3, 1.0, 0.0, 0.0, 2, 9),       # 1; one cell column
    (oracle.SQUARE, 5, 1, 2.0, 0.0, 0.0, 4, 12),         # 1; one row
    (oracle.SQUARE, 2, 2, 1.0, 0.0, 0.0, 1, 5),          # 0; M = 5: one pass
    (oracle.HONEYCOMB, 64, 300, 2.0, 0.0, 0.01, 8, 26),  # 0; many rows per CTA (FP32 flushes)
    (oracle.HONEYCOMB, 6, 7, 1.5, 0.0, 0.05, 4, 8),      # 0; six cells: the wrap's modulo path
    (oracle.HONEYCOMB, 7, 11, 1.5, 0.0, 0.05, 4, 13),    # 2; seven cells: the fast wrap
]


def sysd(case, seed):
    lat, Lx, Ly, W, delta, p, R, M = case
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    return dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, delta=delta, p_vac=p, seed=seed), R, M


@pytest.mark.parametrize("case", CASES)
def test_three_step_fp32_iterates_bit_exact_against_replica(ctx, case):
    d, R, M = sysd(case, 77)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=d["Lx"] * 1000 + d["Ly"])
    mu, muv, last, st = run(ctx, d, M, R, r0=r0, want_last=True)
    assert st.steps_per_pass == 3
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 0, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint32), last_ref.view(np.uint32))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-6
    _, vac = oracle.disorder(oracle.make_system(**d))
    assert st.n_eff == int((vac == 0).sum())
    # launches: the first step, (M - 2) // 3 passes, one remainder launch if M - 2 is not a
    # multiple of three
    assert st.step_launches == 1 + (M - 2) // 3 + ((M - 2) % 3 != 0)


@pytest.mark.parametrize("case", CASES[:3] + CASES[5:7] + CASES[9:])
def test_three_step_fp64_iterates_bit_exact_against_replica(ctx, case):
    d, R, M = sysd(case, 78)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=5)
    mu, muv, last, st = run(ctx, d, M, R, precision=kite.FP64, r0=r0, want_last=True)
    assert st.steps_per_pass == 3
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 1, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint64), last_ref.view(np.uint64))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-12


@pytest.mark.parametrize("case", CASES[:4] + CASES[8:9])
def test_three_step_moments_bit_identical_to_one_step_on_the_same_grid(ctx, case):
    """Where both sweeps launch one CTA per row unit (lattices with fewer units than
    resident CTAs), the same rows feed the same FP32 partials: identical moments."""
    d, R, M = sysd(case, 79)
    mu1, muv1, _, st1 = run(ctx, d, M, R, steps="1")
    mu3, muv3, _, st3 = run(ctx, d, M, R, steps="3")
    assert st1.steps_per_pass == 1 and st3.steps_per_pass == 3
    if st1.grid == st3.grid:
        assert np.array_equal(muv1, muv3) and np.array_equal(mu1, mu3)
    else:
        assert np.max(np.abs(muv1 - muv3)) <= 1e-7


def test_three_step_fp32_moments_within_1e5_of_the_fp64_oracle(ctx):
    """Complex FP32, several CTAs per strip, against the plain FP64 definition."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=96, Ly=80, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 512, 8
    mu, muv, _, st = run(ctx, d, M, R)
    assert st.steps_per_pass == 3
    ref = oracle.moments_1d(oracle.make_system(**d), M, R)
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-5
    assert np.max(np.abs(muv - ref)) <= 1e-5


def test_three_step_at_the_large_dos_order_within_1e5_of_the_fp64_oracle(ctx):
    """The large-DOS workload's order and vectors (M = 2048, R = 8, W = 2 eV, 0.5 %
    vacancies) on a 256 x 256 honeycomb lattice through the three-step pass."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=256, Ly=256, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 2048, 8
    mu, muv, _, st = run(ctx, d, M, R)
    assert st.steps_per_pass == 3
    ref = oracle.moments_1d(oracle.make_system(**d), M, R)
    err = np.max(np.abs(muv - ref))
    print(f"M = 2048, R = 8 FP32, three steps per pass: max |dmu| per vector {err:.2e}")
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-5
    assert err <= 1e-5


@pytest.mark.parametrize("prec,R,S,bar", [("fp32", 16, 1, 1e-5), ("fp32", 19, 2, 1e-5), ("fp64", 6, 1, 1e-12)])
def test_three_step_real_vectors_match_oracle(ctx, prec, R, S, bar):
    """Real +-1 start vectors through the pass (four FP32 / two FP64 per chunk)."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=37, Ly=29, t=-2.7, W=2.0, delta=0.5, p_vac=0.02, seed=8)
    M = 65
    precision = kite.FP64 if prec == "fp64" else kite.FP32
    mu, muv, _, st = run(ctx, d, M, R, precision=precision, real_vectors=True, S=S)
    assert st.steps_per_pass == 3
    s = oracle.make_system(**d)
    ref = np.concatenate([oracle.moments_1d(s, M, R, realisation=k, r0=oracle.random_real(s, R, k))
                          for k in range(S)], 0)
    assert np.max(np.abs(muv - ref)) <= bar
    assert np.max(np.abs(muv.imag)) == 0.0
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar


def test_three_step_full_size_iterates_identical_to_one_step(ctx):
    """The bench's lattice (4096 x 4096 honeycomb, R = 8, FP32): the last two iterates after
    the three-step sweep equal the one-step sweep's bit for bit; moments agree to FP32
    regrouping (the grids differ)."""
    torch = pytest.importorskip("torch")
    d = dict(lattice=oracle.HONEYCOMB, Lx=4096, Ly=4096, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 13, 8  # M - 2 = 11: three passes and a two-step remainder
    n = 2 * 4096 * 4096
    out = {}
    for v in ("1", "3"):
        last = torch.zeros((R, 2, n), dtype=torch.complex64, device="cuda")
        mu = torch.zeros(M, dtype=torch.float64, device="cuda")
        with pass_steps(v):
            st = kite.moments_1d(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, kite.FP32, r_last=last), mu)
        assert st.steps_per_pass == int(v)
        out[v] = (last, mu.cpu().numpy(), st)
    assert torch.equal(out["1"][0].view(torch.float32), out["3"][0].view(torch.float32))
    assert np.max(np.abs(out["1"][1] - out["3"][1])) <= 1e-7
