"""GPU parity of the optical conductivity reconstruction (kite_reconstruct_sigma) against
the oracle's sigma_xx, given the same 2D moments, and the clean-graphene plateau."""
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


@pytest.fixture(scope="module")
def moments():
    d = dict(lattice=0, Lx=6, Ly=5, t=-2.7, W=1.5, seed=12)
    s = oracle.make_system(**d)
    n = oracle.norb(s)
    mu = oracle.moments_2d(s, 96, n, r0=np.eye(n, dtype=np.complex128)) * n
    lo, hi = oracle.bounds_auto(s)
    return mu, lo, hi


@pytest.mark.parametrize("kernel,eta,kT,M_use", [(None, 0.3, 0.0, 96), ("jackson", 1e-5, 0.0, 96),
                                                   (None, 0.2, 0.05, 80), ("jackson", 1e-5, 0.1, 64)])
def test_sigma_matches_oracle(ctx, moments, kernel, eta, kT, M_use):
    mu, lo, hi = moments
    omega = np.linspace(0.1, 9.0, 37)
    E_F = 0.4
    sig = np.zeros((omega.size, 2))
    mu_in = np.ascontiguousarray(np.stack([mu.real, mu.imag], -1))
    kite.reconstruct_sigma(ctx, mu_in, 96, M_use, kite.HONEYCOMB,
                           kite.KERNEL_JACKSON if kernel else kite.KERNEL_NONE, lo, hi, E_F, kT, eta,
                           omega, omega.size, sig, 0)
    got = sig[:, 0] + 1j * sig[:, 1]
    ref = oracle.sigma_xx(mu[:M_use, :M_use], omega, lo, hi, E_F, eta, oracle.HONEYCOMB,
                          kernel=kernel, kT=kT)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_clean_graphene_universal_plateau(ctx):
    """Clean honeycomb, E_F = 0: in the window broadening << hbar omega << |t| the
    absorptive conductivity of the spinless model is e^2/(8 hbar) (both valleys), with
    corrections of order (hbar omega / t)^2.  The finite lattice's level spacing makes
    single frequencies ripple, so the window average is checked (loose physics check, 3 %)."""
    torch = pytest.importorskip("torch")
    d = dict(lattice=0, Lx=1024, Ly=1024, t=-2.7, W=0.0, seed=21)
    M = 512
    mu = torch.zeros((M, M, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = kite.moments_2d(ctx, kite.make_system(**d), kite.make_kpm(M, 1, 1, kite.FP32), mu)
    omega = np.linspace(0.5, 1.2, 29)
    sig = np.zeros((omega.size, 2))
    kite.reconstruct_sigma(ctx, mu, M, M, kite.HONEYCOMB, kite.KERNEL_JACKSON, st.e_min, st.e_max,
                           0.0, 0.0, 1e-5, omega, omega.size, sig, 0)
    assert abs(np.mean(sig[:, 0]) / 0.125 - 1.0) < 0.03, sig[:, 0]
    assert np.all(sig[:, 0] > 0.0)
