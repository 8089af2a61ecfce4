"""GPU parity of the Green's function reconstruction (kite_reconstruct_green) against the
oracle's plain CPGF sum (Eqs. green_function_cheb_expansion/b): bar 1e-10 relative to
max |G| (FP64 on both sides; the GPU builds the coefficients by the geometric recurrence
q^n, whose rounding grows ~n ulp), for every kernel, host and device buffers, energies
inside and outside the spectrum; and the eta-broadened density against -Im G / pi."""
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
    d = dict(lattice=oracle.HONEYCOMB, Lx=40, Ly=36, t=-2.7, W=1.5, p_vac=0.01, seed=17)
    s = oracle.make_system(**d)
    lo, hi = oracle.bounds_auto(s)
    mu = oracle.moments_1d(s, 2000, 2, e_min=lo, e_max=hi).real.mean(0)
    return mu, lo, hi


@pytest.mark.parametrize("kernel,param", [(0, 0.0), (1, 0.0), (2, 4.0)])
@pytest.mark.parametrize("eta", [0.05, 0.3])
def test_green_matches_oracle(ctx, moments, kernel, param, eta):
    mu, lo, hi = moments
    M_use = 1500
    E = np.linspace(lo * 1.2, hi * 1.2, 777)  # includes energies outside the window
    G = np.zeros((E.size, 2))
    rho = np.zeros(E.size)
    kite.reconstruct_green(ctx, mu, mu.size, M_use, kernel, param, lo, hi, eta, E, E.size, G, rho)
    g = {0: None, 1: oracle.kernel_jackson(M_use), 2: oracle.kernel_lorentz(M_use, param)}[kernel]
    ref = oracle.green(mu[:M_use], E, lo, hi, eta, g)
    Gc = G[:, 0] + 1j * G[:, 1]
    assert np.max(np.abs(Gc - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(rho + ref.imag / np.pi)) <= 1e-10 * np.max(np.abs(ref))


def test_green_device_buffers_and_rho_only(ctx, moments):
    torch = pytest.importorskip("torch")
    mu, lo, hi = moments
    E = np.linspace(lo, hi, 301)
    mu_d = torch.from_numpy(mu).cuda()
    E_d = torch.from_numpy(E).cuda()
    rho_d = torch.zeros(E.size, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    kite.reconstruct_green(ctx, mu_d, mu.size, 1000, 1, 0.0, lo, hi, 0.1, E_d, E.size, None, rho_d)
    ref = -oracle.green(mu[:1000], E, lo, hi, 0.1, oracle.kernel_jackson(1000)).imag / np.pi
    assert np.max(np.abs(rho_d.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
    with pytest.raises(kite.KiteError):
        kite.reconstruct_green(ctx, mu, mu.size, 10, 0, 0.0, lo, hi, 0.0, E, E.size, None, rho_d)
