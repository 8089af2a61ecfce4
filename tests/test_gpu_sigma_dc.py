"""GPU parity of the T = 0 longitudinal DC conductivity (Kubo-Greenwood from the 2D
moments) against the oracle, whose formula is pinned by the eigenstate Kubo-Greenwood sum
and by the zero-frequency limit of the optical conductivity.  Both sides compute in FP64
from the same moments: bar 1e-12 relative.  The end-to-end case feeds the device's own 2D
moments of a disordered lattice."""
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


KERNELS = [(kite.KERNEL_JACKSON, 0.0, "jackson"), (kite.KERNEL_NONE, 0.0, None),
           (kite.KERNEL_LORENTZ, 3.0, "lorentz")]


@pytest.mark.parametrize("lattice", [oracle.HONEYCOMB, oracle.SQUARE])
@pytest.mark.parametrize("kern", KERNELS, ids=[k[2] or "none" for k in KERNELS])
def test_sigma_dc_matches_oracle(ctx, lattice, kern):
    kid, param, name = kern
    t = -2.7 if lattice == oracle.HONEYCOMB else -1.0
    o = oracle.make_system(lattice=lattice, Lx=6, Ly=5, t=t, W=2.0, p_vac=0.05, seed=4)
    lo, hi = oracle.bounds_auto(o)
    n = oracle.norb(o)
    M_avail, M_use = 90, 80
    mu = oracle.moments_2d(o, M_avail, n, r0=np.eye(n, dtype=np.complex128)) * n
    E = np.concatenate([np.linspace(lo * 0.99, hi * 0.99, 57), [lo - 0.5, hi + 0.5]])
    ref = oracle.sigma_dc(mu[:M_use, :M_use], E, lo, hi, lattice, kernel=name or "none", lam=param)
    mu_il = np.ascontiguousarray(np.stack([mu.real, mu.imag], -1))
    out = np.zeros(E.size)
    kite.reconstruct_sigma_dc(ctx, mu_il, M_avail, M_use, lattice, kid, param, lo, hi, E, E.size, out)
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert out[-1] == 0.0 and out[-2] == 0.0
    torch = pytest.importorskip("torch")
    dev = torch.zeros(E.size, dtype=torch.float64, device="cuda")
    kite.reconstruct_sigma_dc(ctx, torch.from_numpy(mu_il).cuda(), M_avail, M_use, lattice, kid, param, lo, hi,
                              torch.from_numpy(E).cuda(), E.size, dev)
    assert np.array_equal(dev.cpu().numpy(), out)


def test_sigma_dc_from_device_moments(ctx):
    """Disordered honeycomb 48 x 40: the device's 2D moments (FP32 recursion, split-BF16
    contraction) through the device reconstruction, against the oracle's moments of the
    same start vectors through the oracle's formula; the bar follows the 2D moments' own
    (1e-5 of max |mu|) scaled by the delta coefficients."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=48, Ly=40, t=-2.7, W=2.5, seed=9)
    k, o = kite.make_system(**d), oracle.make_system(**d)
    M, R = 128, 2
    n = oracle.norb(o)
    import synth
    r0 = synth.unit_phase_vectors(n, R, seed=3)
    r0a = np.ascontiguousarray(np.stack([r0.real, r0.imag], -1))
    mu_dev = np.zeros((M, M, 2))
    kite.moments_2d(ctx, k, kite.make_kpm(M, R, 1, kite.FP32, r0=r0a), mu_dev)
    mu_ref = oracle.moments_2d(o, M, R, r0=r0)
    lo, hi = oracle.bounds_auto(o)
    E = np.linspace(-6.0, 6.0, 49)
    out = np.zeros(E.size)
    kite.reconstruct_sigma_dc(ctx, mu_dev, M, M, oracle.HONEYCOMB, kite.KERNEL_JACKSON, 0.0, lo, hi, E, E.size, out)
    ref = oracle.sigma_dc(mu_ref, E, lo, hi, oracle.HONEYCOMB)
    assert np.max(np.abs(out - ref)) <= 2e-3 * np.max(np.abs(ref))
    assert np.all(ref > 0)


def test_sigma_dc_rejects_bad_arguments(ctx):
    mu = np.zeros((4, 4, 2))
    out = np.zeros(3)
    E = np.zeros(3)
    with pytest.raises(kite.KiteError):
        kite.reconstruct_sigma_dc(ctx, mu, 4, 5, oracle.HONEYCOMB, kite.KERNEL_JACKSON, 0.0, -1, 1, E, 3, out)
    with pytest.raises(kite.KiteError):
        kite.reconstruct_sigma_dc(ctx, mu, 4, 4, 7, kite.KERNEL_JACKSON, 0.0, -1, 1, E, 3, out)
    with pytest.raises(kite.KiteError):
        kite.reconstruct_sigma_dc(ctx, mu, 4, 4, oracle.HONEYCOMB, kite.KERNEL_LORENTZ, 0.0, -1, 1, E, 3, out)
