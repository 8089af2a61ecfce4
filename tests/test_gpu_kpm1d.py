"""GPU parity of the 1D moment path (kite_moments_1d) against the CPU oracle.

Bars (written in each test):
  * recursion iterates: bit-exact against the oracle's fixed-rounding replica, FP32 and
    FP64, when both sides start from the same seeded vectors;
  * moments: |mu_gpu - mu_oracle| <= 1e-5 (FP32 recursion, FP64 accumulation above 32
    terms) and <= 1e-12 (FP64) against the plain FP64 definition;
  * integer work (vacancy draws -> N_eff): exact.
Sizes span several CTA tiles and ragged row tails (Lx not a multiple of the tile).
"""
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


def osys(**kw):
    return oracle.make_system(**kw)


def ksys(**kw):
    return kite.make_system(**kw)


def run_gpu(ctx, sysd, M, R, S=1, precision=kite.FP32, r0=None, want_last=False, e_min=0.0,
            e_max=0.0, doubling=False, real_vectors=False):
    s = ksys(**sysd)
    n = oracle.norb(osys(**sysd))
    r0a = None
    if r0 is not None:
        r0a = np.ascontiguousarray(np.stack([r0.real, r0.imag], -1).astype(np.float64))
    dt = np.complex64 if precision == kite.FP32 else np.complex128
    last = np.zeros((S * R, 2, n), dt) if want_last else None
    kpm = kite.make_kpm(M, R, S, precision, e_min, e_max, r0a, last, doubling=doubling,
                        real_vectors=real_vectors)
    mu = np.zeros(M, np.float64)
    muv = np.zeros((S * R, M, 2), np.float64)
    st = kite.moments_1d(ctx, s, kpm, mu, muv)
    return mu, muv[..., 0] + 1j * muv[..., 1], last, st


CASES_BITWISE = [
    # (lattice, Lx, Ly, W, delta, p_vac, R, M)
    (oracle.HONEYCOMB, 37, 29, 2.0, 0.0, 0.02, 3, 48),   # C=2, ragged strip (TX=64)
    (oracle.HONEYCOMB, 70, 9, 1.0, 0.5, 0.0, 8, 33),     # C=4, TX=32, 3 strips, ragged
    (oracle.SQUARE, 300, 5, 3.0, 0.0, 0.05, 1, 40),      # C=1, TX=256, ragged
    (oracle.SQUARE, 17, 40, 0.0, 0.0, 0.0, 6, 25),       # C=4 (6 padded to 8)
    (oracle.HONEYCOMB, 3, 2, 1.0, 0.0, 0.1, 2, 16),      # tiny lattice, wrap-around
]


@pytest.mark.parametrize("case", CASES_BITWISE)
def test_fp32_iterates_bit_exact_against_replica(ctx, case):
    lat, Lx, Ly, W, delta, p, R, M = case
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    d = dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, delta=delta, p_vac=p, seed=77)
    n = oracle.norb(osys(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=Lx * 1000 + Ly)
    mu, muv, last, st = run_gpu(ctx, d, M, R, r0=r0, want_last=True)
    mu_ref, last_ref = oracle.replica_1d(osys(**d), M, R, 0, r0=r0, want_last=True)
    assert last.dtype == last_ref.dtype
    assert np.array_equal(last.view(np.uint32), last_ref.view(np.uint32))
    # moments of the same iterates: FP32 products summed in FP32 over <= 32 rows
    assert np.max(np.abs(muv - mu_ref)) <= 1e-6
    _, vac = oracle.disorder(osys(**d))
    assert st.n_eff == int((vac == 0).sum())


@pytest.mark.parametrize("case", CASES_BITWISE[:3])
def test_fp64_iterates_bit_exact_against_replica(ctx, case):
    lat, Lx, Ly, W, delta, p, R, M = case
    t = -2.7 if lat == oracle.HONEYCOMB else -1.0
    d = dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, delta=delta, p_vac=p, seed=78)
    n = oracle.norb(osys(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=5)
    mu, muv, last, st = run_gpu(ctx, d, M, R, precision=kite.FP64, r0=r0, want_last=True)
    mu_ref, last_ref = oracle.replica_1d(osys(**d), M, R, 1, r0=r0, want_last=True)
    assert np.array_equal(last.view(np.uint64), last_ref.view(np.uint64))
    assert np.max(np.abs(muv - mu_ref)) <= 1e-12


def test_random_phase_start_vectors_match_oracle(ctx):
    """M = 1: both r_last slots hold r_0 as generated on the device from the seed."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=40, Ly=33, t=-2.7, W=1.0, p_vac=0.03, seed=123)
    R = 5
    _, _, last64, _ = run_gpu(ctx, d, 1, R, precision=kite.FP64, want_last=True)
    ref = oracle.random_phase(osys(**d), R)
    assert np.max(np.abs(last64[:, 0] - ref)) <= 4e-16
    _, _, last32, _ = run_gpu(ctx, d, 1, R, precision=kite.FP32, want_last=True)
    ref32 = ref.astype(np.complex64)
    ulp = np.spacing(np.abs(ref32.real).astype(np.float32)) + np.spacing(np.abs(ref32.imag).astype(np.float32))
    assert np.all(np.abs(last32[:, 0] - ref32) <= ulp)


def test_config_small_fp64_moments(ctx):
    """Honeycomb 64x64, t=-2.7 eV, V in [-0.5, 0.5] eV, bounds +-(3|t|+0.5)*1.01, M=256,
    4 random-phase vectors, complex FP64: <= 1e-12 against the FP64 oracle."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=64, Ly=64, t=-2.7, W=1.0, seed=1)
    b = (3 * 2.7 + 0.5) * 1.01
    mu, muv, _, st = run_gpu(ctx, d, 256, 4, precision=kite.FP64, e_min=-b, e_max=b)
    ref = oracle.moments_1d(osys(**d), 256, 4, e_min=-b, e_max=b)
    assert np.max(np.abs(muv - ref)) <= 1e-12
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-12
    assert abs(mu[0] - 1.0) <= 1e-14


def test_fp32_moments_within_1e5_of_the_fp64_oracle(ctx):
    """Complex FP32 recursion, FP64 accumulation: max_n |mu_n - mu_n^oracle| <= 1e-5."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=96, Ly=80, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 512, 8
    mu, muv, _, st = run_gpu(ctx, d, M, R)
    ref = oracle.moments_1d(osys(**d), M, R)
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-5
    assert np.max(np.abs(muv - ref)) <= 1e-5


DOUBLING_CASES = [
    # (system, M, R, S, precision, bar): bars as for the plain path
    (dict(lattice=oracle.HONEYCOMB, Lx=64, Ly=64, t=-2.7, W=1.0, seed=1), 256, 4, 1, "fp64", 1e-12),
    (dict(lattice=oracle.HONEYCOMB, Lx=96, Ly=80, t=-2.7, W=2.0, p_vac=0.005, seed=2), 512, 8, 1,
     "fp32", 1e-5),
    (dict(lattice=oracle.SQUARE, Lx=300, Ly=5, t=-1.0, W=3.0, p_vac=0.05, seed=5), 33, 6, 2, "fp32", 1e-5),
    (dict(lattice=oracle.HONEYCOMB, Lx=37, Ly=29, t=-2.7, W=2.0, delta=0.5, p_vac=0.02, seed=8), 3, 3,
     1, "fp64", 1e-12),
    (dict(lattice=oracle.SQUARE, Lx=17, Ly=40, t=-1.0, W=1.0, seed=3), 2, 1, 1, "fp32", 1e-5),
    (dict(lattice=oracle.SQUARE, Lx=17, Ly=40, t=-1.0, W=1.0, seed=3), 1, 1, 1, "fp64", 1e-12),
]


@pytest.mark.parametrize("case", DOUBLING_CASES)
def test_moment_doubling_matches_oracle(ctx, case):
    """Moment doubling (mu_2n = 2<r_n|r_n> - mu_0, mu_2n+1 = 2<r_n|r_n+1> - mu_1) against the
    oracle's plain mu_n = <r_0|T_n r_0>: same bars as the plain path, ceil(M/2) steps, odd
    and tiny M, realisations and padded vector batches included."""
    d, M, R, S, prec, bar = case
    precision = kite.FP64 if prec == "fp64" else kite.FP32
    mu, muv, _, st = run_gpu(ctx, d, M, R, S=S, precision=precision, doubling=True)
    ref = np.concatenate([oracle.moments_1d(osys(**d), M, R, realisation=s) for s in range(S)], 0)
    assert np.max(np.abs(muv - ref)) <= bar
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar
    batches = S * ((R + (7 if prec == "fp32" else 3)) // (8 if prec == "fp32" else 4))
    if st.cluster_ctas:  # small lattice held on chip: one launch of ceil(M/2) steps per batch
        assert st.step_launches == batches and st.steps_per_pass == (M + 1) // 2
    else:
        assert st.step_launches == batches * ((M + 1) // 2)


REAL_CASES = [
    # (system, M, R, S, precision, doubling, bar)
    (dict(lattice=oracle.HONEYCOMB, Lx=64, Ly=64, t=-2.7, W=1.0, seed=1), 256, 4, 1, "fp64", False, 1e-12),
    (dict(lattice=oracle.HONEYCOMB, Lx=96, Ly=80, t=-2.7, W=2.0, p_vac=0.005, seed=2), 512, 16, 1,
     "fp32", False, 1e-5),
    (dict(lattice=oracle.SQUARE, Lx=300, Ly=5, t=-1.0, W=3.0, p_vac=0.05, seed=5), 33, 5, 2, "fp32", False, 1e-5),
    (dict(lattice=oracle.HONEYCOMB, Lx=37, Ly=29, t=-2.7, W=2.0, delta=0.5, p_vac=0.02, seed=8), 65, 19, 1,
     "fp32", True, 1e-5),
    (dict(lattice=oracle.SQUARE, Lx=17, Ly=40, t=-1.0, W=1.0, seed=3), 40, 6, 1, "fp64", True, 1e-12),
]


@pytest.mark.parametrize("case", REAL_CASES)
def test_real_vectors_match_oracle(ctx, case):
    """Real +-1 start vectors (16 FP32 / 8 FP64 per batch): device draws and moments
    against the oracle's plain definition on the same vectors, plain and doubling, full
    and padded batches, several batches (R = 19) and realisations."""
    d, M, R, S, prec, dbl, bar = case
    precision = kite.FP64 if prec == "fp64" else kite.FP32
    mu, muv, _, st = run_gpu(ctx, d, M, R, S=S, precision=precision, doubling=dbl, real_vectors=True)
    ref = np.concatenate([oracle.moments_1d(osys(**d), M, R, realisation=s,
                                            r0=oracle.random_real(osys(**d), R, s)) for s in range(S)], 0)
    assert np.max(np.abs(muv - ref)) <= bar
    assert np.max(np.abs(muv.imag)) == 0.0
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar


def test_exact_trace_with_basis_vectors_pins_device_draws(ctx):
    """Basis start vectors give the exact trace: pins the device's disorder and vacancy
    draws against the oracle's (FP64 path, <= 1e-12)."""
    d = dict(lattice=oracle.SQUARE, Lx=9, Ly=7, t=-1.0, W=3.0, p_vac=0.1, seed=19)
    n = oracle.norb(osys(**d))
    eye = np.eye(n, dtype=np.complex128)
    mu, muv, _, st = run_gpu(ctx, d, 20, n, precision=kite.FP64, r0=eye)
    ref = oracle.moments_1d(osys(**d), 20, n, r0=eye)
    assert np.max(np.abs(muv.sum(0) - ref.sum(0))) <= 1e-12


def test_realisations_average(ctx):
    d = dict(lattice=oracle.HONEYCOMB, Lx=24, Ly=20, t=-2.7, W=2.0, p_vac=0.02, seed=9)
    M, R, S = 64, 2, 3
    mu, muv, _, st = run_gpu(ctx, d, M, R, S=S, precision=kite.FP64)
    refs = [oracle.moments_1d(osys(**d), M, R, realisation=s) for s in range(S)]
    ref = np.concatenate(refs, axis=0)
    assert np.max(np.abs(muv - ref)) <= 1e-12
    assert np.max(np.abs(mu - ref.real.mean(0))) <= 1e-12


def test_device_pointers_and_determinism(ctx):
    torch = pytest.importorskip("torch")
    d = dict(lattice=oracle.HONEYCOMB, Lx=50, Ly=50, t=-2.7, W=1.0, seed=4)
    s = ksys(**d)
    kpm = kite.make_kpm(128, 4, 1, kite.FP32)
    mu1 = torch.zeros(128, dtype=torch.float64, device="cuda")
    mu2 = torch.zeros(128, dtype=torch.float64, device="cuda")
    kite.moments_1d(ctx, s, kpm, mu1)
    kite.moments_1d(ctx, s, kpm, mu2)
    assert torch.equal(mu1, mu2)  # fixed-order reductions: run-to-run identical
    ref = oracle.moments_1d(osys(**d), 128, 4).real.mean(0)
    assert np.max(np.abs(mu1.cpu().numpy() - ref)) <= 1e-5


def test_bounds_violation_is_reported(ctx):
    """Bounds tighter than the spectrum make T_n grow: KITE_ERR_BOUNDS, no result."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=16, Ly=16, t=-2.7, W=0.0, seed=1)
    with pytest.raises(kite.KiteError) as e:
        run_gpu(ctx, d, 256, 2, e_min=-4.0, e_max=4.0)
    assert e.value.status == kite.ERR_BOUNDS


def test_dos_reconstruction_matches_oracle(ctx):
    d = dict(lattice=oracle.HONEYCOMB, Lx=32, Ly=32, t=-2.7, W=1.0, seed=3)
    M = 300
    mu, _, _, st = run_gpu(ctx, d, M, 2, precision=kite.FP64)
    lo, hi = st.e_min, st.e_max
    E = np.linspace(lo * 1.05, hi * 1.05, 1001)
    for kern, par, g in ((kite.KERNEL_JACKSON, 0.0, oracle.kernel_jackson(200)),
                         (kite.KERNEL_LORENTZ, 4.0, oracle.kernel_lorentz(200, 4.0)),
                         (kite.KERNEL_NONE, 0.0, None)):
        rho = np.zeros_like(E)
        kite.reconstruct_dos(ctx, mu, M, 200, kern, par, lo, hi, E, E.size, rho)
        ref = oracle.dos(mu[:200], E, lo, hi, g)
        assert np.max(np.abs(rho - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_bounded_wait_timeout_is_reported_and_context_survives(ctx):
    """A barrier armed for bytes that never arrive: the bounded wait gives up, the call
    returns KITE_ERR_TIMEOUT, and the next call on the same context is correct."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=64, Ly=48, t=-2.7, W=1.0, seed=6)
    kite.debug_stall_once(ctx)
    with pytest.raises(kite.KiteError) as e:
        run_gpu(ctx, d, 32, 4)
    assert e.value.status == kite.ERR_TIMEOUT
    mu, _, _, _ = run_gpu(ctx, d, 32, 4)
    ref = oracle.moments_1d(osys(**d), 32, 4).real.mean(0)
    assert np.max(np.abs(mu - ref)) <= 1e-5


def test_full_size_launch_sampled_sites_match_window_oracle(ctx):
    """The bench's lattice (4096 x 4096 honeycomb, R = 8, FP32) and launch configuration,
    with few moments: iterates at sampled sites against the light-cone window replica,
    N_eff exact, mu_0 = 1."""
    torch = pytest.importorskip("torch")
    d = dict(lattice=oracle.HONEYCOMB, Lx=4096, Ly=4096, t=-2.7, W=2.0, p_vac=0.005, seed=2)
    M, R = 12, 8
    n = 2 * 4096 * 4096
    last = torch.zeros((R, 2, n), dtype=torch.complex64, device="cuda")
    mu = torch.zeros(M, dtype=torch.float64, device="cuda")
    st = kite.moments_1d(ctx, ksys(**d), kite.make_kpm(M, R, 1, kite.FP32, r_last=last), mu)
    s = osys(**d)
    rng = np.random.default_rng(0)
    sites = [(0, 0), (4095, 4095), (4095, 0), (0, 4095), (31, 32), (32, 31), (2047, 2048)]
    sites += [tuple(int(v) for v in rng.integers(0, 4096, 2)) for _ in range(9)]
    exact, total = 0, 0
    for (x0, y0) in sites:
        ref = oracle.replica_window(s, M, R, 0, x0, y0)  # [R][2][2]
        o = 2 * (y0 * 4096 + x0)
        got = last[:, :, o:o + 2].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-5, (x0, y0)
        exact += int(np.sum(got == ref))
        total += got.size
    # device random phases use CUDA's FP64 sincos, the oracle libm's: they round to the
    # same FP32 value except at rare ties, so nearly every iterate is bit-identical
    assert exact >= 0.98 * total
    _, vac = oracle.disorder(s)
    assert st.n_eff == int((vac == 0).sum())
    mu_h = mu.cpu().numpy()
    assert abs(mu_h[0] - 1.0) <= 1e-6
    assert np.all(np.abs(mu_h) <= 1.0)


def test_start_vectors_from_pageable_pinned_and_device_memory_agree(ctx):
    """Caller start vectors in pageable host memory (staged), page-locked host memory (read
    in place by the kernels across the host link) and device memory: the same moments bit
    for bit, twice in a row (the staging buffer is reused)."""
    torch = pytest.importorskip("torch")
    d = dict(lattice=oracle.HONEYCOMB, Lx=70, Ly=41, t=-2.7, W=2.0, p_vac=0.01, seed=21)
    M, R = 40, 5
    n = oracle.norb(osys(**d))
    r0 = synth.unit_phase_vectors(n, R, seed=8)
    r0a = np.ascontiguousarray(np.stack([r0.real, r0.imag], -1).astype(np.float64))
    pinned = torch.from_numpy(r0a).pin_memory()
    device = torch.from_numpy(r0a).cuda()
    out = []
    for src in (r0a, pinned, device, r0a):
        muv = np.zeros((R, M, 2))
        kite.moments_1d(ctx, ksys(**d), kite.make_kpm(M, R, 1, kite.FP32, r0=src), np.zeros(M), muv)
        out.append(muv)
    for o in out[1:]:
        assert np.array_equal(o, out[0])
    ref = oracle.moments_1d(osys(**d), M, R, r0=r0)
    assert np.max(np.abs(out[0][..., 0] + 1j * out[0][..., 1] - ref)) <= 1e-5
