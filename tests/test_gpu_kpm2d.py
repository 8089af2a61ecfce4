"""GPU parity of the 2D Kubo-Bastin moments (kite_moments_2d) against the oracle's
plain FP64 triple loop over the stored families.

Bar: max |mu_gpu - mu_oracle| <= 1e-5 * max |mu_oracle| (FP32 recursion, split-BF16
tensor-core contraction with FP32 sums inside 512-product sub-chunks and over 16 of them,
FP64 above), for every pair of velocity directions (x, y)."""
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


def run2d(ctx, d, M, R, S=1, r0=None, alpha=0, beta=0):
    n = oracle.norb(oracle.make_system(**d))
    r0a = None
    if r0 is not None:
        r0a = np.ascontiguousarray(np.stack([r0.real, r0.imag], -1).astype(np.float64))
    mu = np.zeros((M, M, 2), np.float64)
    st = kite.moments_2d(ctx, kite.make_system(**d), kite.make_kpm(M, R, S, kite.FP32, r0=r0a), mu,
                         alpha, beta)
    return mu[..., 0] + 1j * mu[..., 1], st


@pytest.mark.parametrize("d,M,R", [
    (dict(lattice=0, Lx=24, Ly=20, t=-2.7, W=1.0, p_vac=0.02, seed=4), 32, 3),
    (dict(lattice=0, Lx=37, Ly=9, t=-2.7, W=2.0, delta=0.4, seed=5), 130, 2),
    (dict(lattice=1, Lx=33, Ly=17, t=-1.0, W=3.0, p_vac=0.03, seed=6), 48, 1),
])
def test_small_lattices_against_triple_loop(ctx, d, M, R):
    mu, st = run2d(ctx, d, M, R)
    ref = oracle.moments_2d(oracle.make_system(**d), M, R)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(mu - ref)) <= 1e-5 * scale
    _, vac = oracle.disorder(oracle.make_system(**d))
    assert st.n_eff == int((vac == 0).sum())


@pytest.mark.parametrize("alpha,beta", [(1, 1), (0, 1), (1, 0)])
@pytest.mark.parametrize("d,M,R", [
    (dict(lattice=0, Lx=24, Ly=20, t=-2.7, W=1.0, p_vac=0.02, seed=4), 32, 3),
    (dict(lattice=1, Lx=33, Ly=17, t=-1.0, W=3.0, p_vac=0.03, seed=6), 48, 1),
])
def test_y_and_mixed_directions_against_triple_loop(ctx, d, M, R, alpha, beta):
    """mu^{yy}, mu^{xy}, mu^{yx} (sigma_yy and the Hall pair) against the oracle."""
    mu, st = run2d(ctx, d, M, R, alpha=alpha, beta=beta)
    ref = oracle.moments_2d(oracle.make_system(**d), M, R, alpha=alpha, beta=beta)
    assert np.max(np.abs(mu - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_caller_start_vectors(ctx):
    d = dict(lattice=0, Lx=16, Ly=16, t=-2.7, W=1.5, seed=8)
    n = oracle.norb(oracle.make_system(**d))
    r0 = synth.unit_phase_vectors(n, 2, seed=99)
    mu, _ = run2d(ctx, d, 24, 2, r0=r0)
    ref = oracle.moments_2d(oracle.make_system(**d), 24, 2, r0=r0)
    assert np.max(np.abs(mu - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_full_lattice_few_moments(ctx):
    """The 1024 x 1024 honeycomb lattice of the optical-conductivity workload (W = 1 eV,
    the launch configuration of the full run) with M = 8: every moment against the
    oracle; mu_00 = <h r|h r>/N close to its exact trace t~^2/2."""
    d = dict(lattice=0, Lx=1024, Ly=1024, t=-2.7, W=1.0, seed=4)
    M = 8
    mu, st = run2d(ctx, d, M, 1)
    ref = oracle.moments_2d(oracle.make_system(**d), M, 1)
    assert np.max(np.abs(mu - ref)) <= 1e-5 * np.max(np.abs(ref))
    lo, hi = oracle.bounds_auto(oracle.make_system(**d))
    tt = -2.7 / (0.5 * (hi - lo))
    assert abs(mu[0, 0].real - 0.5 * tt * tt) <= 0.01 * 0.5 * tt * tt


def test_full_size_panels_match_oracle(ctx):
    """The optical-conductivity workload at full size and order (1024 x 1024 honeycomb,
    W = 1 eV, M = 1024, one random vector, FP32 families and the split-BF16 tensor-core
    contraction over K = 4.2M): eight whole rows and eight whole columns of mu_nm, chosen
    across tile boundaries and split-K blocks, against the oracle's panels (the plain
    recursion dotted with stored a_n or b_m, Eq. Gammanm) within 1e-5 max|mu|."""
    d = dict(lattice=0, Lx=1024, Ly=1024, t=-2.7, W=1.0, seed=4)
    M = 1024
    mu, st = run2d(ctx, d, M, 1)
    rows = [0, 1, 127, 128, 511, 640, 1000, 1023]
    cols = [0, 2, 129, 255, 256, 513, 767, 1023]
    pr, pc = oracle.moments_2d_panels(oracle.make_system(**d), M, 1, rows, cols)
    scale = np.max(np.abs(mu))
    er, ec = np.max(np.abs(mu[rows, :] - pr)), np.max(np.abs(mu[:, cols] - pc))
    print(f"full-size panels: max|mu| {scale:.4e}, row error {er / scale:.2e}, column error {ec / scale:.2e}")
    assert er <= 1e-5 * scale and ec <= 1e-5 * scale


def test_family_streams_do_not_change_the_moments(ctx, monkeypatch):
    """The A and B families on two streams side by side (default) or in sequence on one
    (KITE_FAM_STREAMS=1): independent recursions into separate buffers, so the moments are
    bit-identical; R = 5 runs three vector batches (the fork and join every batch), S = 2
    two realisations, and a context rebound to another stream keeps its second stream."""
    d = dict(lattice=0, Lx=40, Ly=24, t=-2.7, W=1.5, p_vac=0.01, seed=9)
    mu2, _ = run2d(ctx, d, 24, 5, S=2)
    monkeypatch.setenv("KITE_FAM_STREAMS", "1")
    mu1, _ = run2d(ctx, d, 24, 5, S=2)
    assert np.array_equal(mu1, mu2)
    monkeypatch.delenv("KITE_FAM_STREAMS")
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    ctx.set_stream(s.cuda_stream)
    try:
        mu3, _ = run2d(ctx, d, 24, 5, S=2)
    finally:
        ctx.set_stream(None)
    assert np.array_equal(mu3, mu2)
