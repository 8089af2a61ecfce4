"""GPU parity of the two-step pass: temporal blocking of the recursion (Eq. e6 applied
twice per pass over the iterates, the moments <r_0|r_{n+1}> and <r_0|r_{n+2}> of Eqs.
e7/e8 fused into the same pass).  KITE_PASS_STEPS pins the pass (1 or 2) for the call.

Bars (written in each test):
  * iterates: bit-exact against the oracle's fixed-rounding replica (the pass computes each
    site with the one-step rounding sequence, halo sites included), FP32 and FP64;
  * moments: <= 1e-6 against the replica's moments (FP32 products summed in FP32 over at
    most 32 rows), <= 1e-12 for FP64, <= 1e-5 against the plain FP64 definition;
  * same grid as the one-step sweep: moments bit-identical to it (the same rows feed the
    same FP32 partials in the same order).
Lattices cover tiles with ragged right strips, a single cell column and row (the two-cell
halo wraps more than once), odd and even M (odd remainder step) and padded batches.
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


def run(ctx, d, M, R, precision=kite.FP32, r0=None, want_last=False, real_vectors=False, S=1, doubling=False):
    s = kite.make_system(**d)
    n = oracle.norb(oracle.make_system(**d))
    r0a = None
    if r0 is not None:
        r0a = np.ascontiguousarray(np.stack([r0.real, r0.imag], -1).astype(np.float64))
    dt = np.complex64 if precision == kite.FP32 else np.complex128
    last = np.zeros((S * R, 2, n), dt) if want_last else None
    kpm = kite.make_kpm(M, R, S, precision, 0.0, 0.0, r0a, last, real_vectors=real_vectors, doubling=doubling)
    mu = np.zeros(M, np.float64)
    muv = np.zeros((S * R, M, 2), np.float64)
    st = kite.moments_1d(ctx, s, kpm, mu, muv)
    return mu, muv[..., 0] + 1j * muv[..., 1], last, st


CASES = [
    # (lattice, Lx, Ly, W, delta, p_vac, R, M)
    (oracle.HONEYCOMB, 37, 29, 2.0, 0.0, 0.02, 3, 48),   # C=2, ragged strip, even M
    (oracle.HONEYCOMB, 70, 9, 1.0, 0.5, 0.0, 8, 33),     # C=4, 3 strips, odd M (remainder step)
    (oracle.SQUARE, 300, 5, 3.0, 0.0, 0.05, 1, 40),      # C=1, TX=256, ragged
    (oracle.SQUARE, 17, 40, 0.0, 0.0, 0.0, 6, 25),       # C=4 (6 padded to 8)
    (oracle.HONEYCOMB, 3, 2, 1.0, 0.0, 0.1, 2, 16),      # tiny lattice, wrap-around
    (oracle.HONEYCOMB, 1, 3, 1.0, 0.0, 0.0, 2, 9),       # one cell column: the halo wraps twice
    (oracle.SQUARE, 5, 1, 2.0, 0.0, 0.0, 4, 12),         # one row: rows y-1, y, y+1 coincide
    (oracle.SQUARE, 2, 2, 1.0, 0.0, 0.0, 1, 4),          # M = 4: one pass, no remainder
    (oracle.HONEYCOMB, 64, 300, 2.0, 0.0, 0.01, 8, 21),  # many rows per CTA (FP32 flushes)
]


def sysd(case, seed):
    lat, Lx, Ly, W, delta, p, R, M = case
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    return dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, delta=delta, p_vac=p, seed=seed), R, M


@pytest.mark.parametrize("case", CASES)
def test_two_step_fp32_iterates_bit_exact_against_replica(ctx, case):
    d, R, M = sysd(case, 77)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=d["Lx"] * 1000 + d["Ly"])
    with pass_steps("2"):
        mu, muv, last, st = run(ctx, d, M, R, r0=r0, want_last=True)
    assert st.steps_per_pass == 2
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 0, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint32), last_ref.view(np.uint32))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-6
    _, vac = oracle.disorder(oracle.make_system(**d))
    assert st.n_eff == int((vac == 0).sum())


@pytest.mark.parametrize("case", CASES[:3] + CASES[5:7])
def test_two_step_fp64_iterates_bit_exact_against_replica(ctx, case):
    d, R, M = sysd(case, 78)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=5)
    with pass_steps("2"):
        mu, muv, last, st = run(ctx, d, M, R, precision=kite.FP64, r0=r0, want_last=True)
    assert st.steps_per_pass == 2
    mu_ref, last_ref = oracle.replica_1d(oracle.make_system(**d), M, R, 1, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint64), last_ref.view(np.uint64))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-12


@pytest.mark.parametrize("case", CASES[:8])
def test_two_step_moments_bit_identical_to_one_step_on_the_same_grid(ctx, case):
    """Small lattices have fewer row units than resident CTAs: both sweeps launch one CTA
    per unit, so the moments must agree bit for bit."""
    d, R, M = sysd(case, 79)
    with pass_steps("1"):
        mu1, muv1, _, st1 = run(ctx, d, M, R)
    with pass_steps("2"):
        mu2, muv2, _, st2 = run(ctx, d, M, R)
    assert st1.steps_per_pass == 1 and st2.steps_per_pass == 2
    assert st1.grid == st2.grid
    assert np.array_equal(muv1, muv2) and np.array_equal(mu1, mu2)
    # launches: one first step, (M - 2) // 2 passes, one remainder step for odd M - 2
    assert st2.step_launches == 1 + (M - 2) // 2 + (M - 2) % 2


def test_two_step_fp32_moments_within_1e5_of_the_fp64_oracle(ctx):
    """Complex FP32, several CTAs per strip, against the plain FP64 definition."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=96, Ly=80, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 512, 8
    with pass_steps("2"):
        mu, muv, _, st = run(ctx, d, M, R)
    assert st.steps_per_pass == 2
    ref = oracle.moments_1d(oracle.make_system(**d), M, R)
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-5
    assert np.max(np.abs(muv - ref)) <= 1e-5


@pytest.mark.parametrize("steps", ["2", None])
def test_fp32_at_the_large_dos_order_within_1e5_of_the_fp64_oracle(ctx, steps):
    """The large-DOS workload's order and vectors (M = 2048, R = 8, W = 2 eV, 0.5 % vacancies,
    complex FP32 recursion with FP64 moment sums) on a 256 x 256 honeycomb lattice that the
    oracle finishes in seconds: rounding accumulated over 2047 steps stays within 1e-5 of
    the plain FP64 definition, through the two-step pass and through whatever the autotuner
    picks."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=256, Ly=256, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 2048, 8
    with pass_steps(steps) if steps else contextlib.nullcontext():
        mu, muv, _, st = run(ctx, d, M, R)
    if steps:
        assert st.steps_per_pass == 2
    ref = oracle.moments_1d(oracle.make_system(**d), M, R)
    err = np.max(np.abs(muv - ref))
    print(f"M = 2048, R = 8 FP32 ({st.steps_per_pass} steps per pass): max |dmu| per vector {err:.2e}, "
          f"average {np.max(np.abs(mu - ref.real.mean(0))):.2e}")
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-5
    assert err <= 1e-5


@pytest.mark.parametrize("prec,R,S,bar", [("fp32", 16, 1, 1e-5), ("fp32", 19, 2, 1e-5), ("fp64", 6, 1, 1e-12)])
def test_two_step_real_vectors_match_oracle(ctx, prec, R, S, bar):
    """Real +-1 start vectors through the pass (four FP32 / two FP64 per chunk)."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=37, Ly=29, t=-2.7, W=2.0, delta=0.5, p_vac=0.02, seed=8)
    M = 65
    precision = kite.FP64 if prec == "fp64" else kite.FP32
    with pass_steps("2"):
        mu, muv, _, st = run(ctx, d, M, R, precision=precision, real_vectors=True, S=S)
    assert st.steps_per_pass == 2
    s = oracle.make_system(**d)
    ref = np.concatenate([oracle.moments_1d(s, M, R, realisation=k, r0=oracle.random_real(s, R, k))
                          for k in range(S)], 0)
    assert np.max(np.abs(muv - ref)) <= bar
    assert np.max(np.abs(muv.imag)) == 0.0
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar


def test_two_step_full_size_sampled_sites_match_window_oracle(ctx):
    """The bench's lattice (4096 x 4096 honeycomb, R = 8, FP32) through the pass: iterates
    at sampled sites bit-identical to the one-step sweep's and within 1e-5 of the
    light-cone window replica (device phases from CUDA's sincos), N_eff exact."""
    torch = pytest.importorskip("torch")
    d = dict(lattice=oracle.HONEYCOMB, Lx=4096, Ly=4096, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 13, 8  # odd M - 2: five passes and a remainder step
    n = 2 * 4096 * 4096
    out = {}
    for v in ("1", "2"):
        last = torch.zeros((R, 2, n), dtype=torch.complex64, device="cuda")
        mu = torch.zeros(M, dtype=torch.float64, device="cuda")
        with pass_steps(v):
            st = kite.moments_1d(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, kite.FP32, r_last=last), mu)
        assert st.steps_per_pass == int(v)
        out[v] = (last, mu.cpu().numpy(), st)
    assert torch.equal(out["1"][0].view(torch.float32), out["2"][0].view(torch.float32))
    s = oracle.make_system(**d)
    rng = np.random.default_rng(1)
    sites = [(0, 0), (4095, 4095), (31, 32), (32, 31), (2047, 2048)]
    sites += [tuple(int(v) for v in rng.integers(0, 4096, 2)) for _ in range(5)]
    last = out["2"][0]
    for (x0, y0) in sites:
        ref = oracle.replica_window(s, M, R, 0, x0, y0)
        o = 2 * (y0 * 4096 + x0)
        got = last[:, :, o:o + 2].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-5, (x0, y0)
    _, vac = oracle.disorder(s)
    assert out["2"][2].n_eff == int((vac == 0).sum())
    # the grids differ (occupancy of the two kernels): moments agree to FP32 regrouping
    assert np.max(np.abs(out["1"][1] - out["2"][1])) <= 1e-7
    assert abs(out["2"][1][0] - 1.0) <= 1e-6


DOUBLING = [
    # (case, precision, real vectors, S, bar): M odd and even, passes with and without an
    # odd remainder step, padded batches, realisations
    (CASES[0], "fp32", False, 1, 1e-5), (CASES[1], "fp32", False, 2, 1e-5), (CASES[3], "fp64", False, 1, 1e-12),
    (CASES[4], "fp32", False, 1, 1e-5), (CASES[5], "fp64", False, 1, 1e-12), (CASES[8], "fp32", False, 1, 1e-5),
    (CASES[0], "fp32", True, 1, 1e-5), (CASES[2], "fp64", True, 2, 1e-12),
]


@pytest.mark.parametrize("case,prec,realv,S,bar", DOUBLING)
def test_two_step_doubling_against_oracle_and_one_step(ctx, case, prec, realv, S, bar):
    """Moment doubling through the two-step pass (slots <r_n|r_n>, <r_n|r_{n+1}>,
    <r_{n+1}|r_{n+1}>, <r_{n+1}|r_{n+2}> per pass, no r_0 read): against the oracle's plain
    moments, and bit-identical to the one-step doubling sweep where both launch one CTA per
    row unit."""
    d, R, M = sysd(case, 81)
    if M < 5:
        pytest.skip("no pass")
    precision = kite.FP64 if prec == "fp64" else kite.FP32
    with pass_steps("2"):
        mu2, muv2, _, st2 = run(ctx, d, M, R, precision=precision, real_vectors=realv, S=S, doubling=True)
    with pass_steps("1"):
        mu1, muv1, _, st1 = run(ctx, d, M, R, precision=precision, real_vectors=realv, S=S, doubling=True)
    assert st2.steps_per_pass == 2 and st1.steps_per_pass == 1
    steps = (M + 1) // 2
    max_batch = (16 if realv else 8) if prec == "fp32" else (8 if realv else 4)
    batches = S * -(-R // max_batch)
    assert st2.step_launches == batches * (1 + (steps - 1) // 2 + (steps - 1) % 2)
    s = oracle.make_system(**d)
    ref = np.concatenate([oracle.moments_1d(s, M, R, realisation=k,
                                            r0=oracle.random_real(s, R, k) if realv else None)
                          for k in range(S)], 0)
    assert np.max(np.abs(muv2 - ref)) <= bar
    assert np.max(np.abs(mu2 - ref.real.mean(0))) <= bar
    if st1.grid == st2.grid:
        assert np.array_equal(muv1, muv2)
    else:
        assert np.max(np.abs(muv1 - muv2)) <= (1e-7 if prec == "fp32" else 1e-13)
