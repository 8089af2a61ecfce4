"""GPU parity of the DC Hall conductivity: the 2D moments in a magnetic field (the velocity
h~ = [r, H~] with the Hamiltonian's Peierls phases) and the Kubo-Bastin reconstruction with
its Fermi-sea term, against the oracle, whose field velocity is pinned by the position
commutator and whose Bastin formula is pinned by the eigenbasis integral and the TKNN sum.

Bars: the 2D moments as for the field-free path (1e-5 of max |mu|: FP32 recursion,
split-BF16 contraction); the reconstruction 1e-10 of max |sigma| (both FP64 from the same
moments, the same Gauss-Legendre nodes); the plateau of graphene in a field to 3 % of
e^2/h per spin (stochastic trace over 4 vectors of 32768 orbitals, finite M and eta).
"""
import math

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


FIELD_CASES = [
    # honeycomb with disorder, vacancies and staggering; ragged strips
    dict(lattice=0, Lx=37, Ly=16, t=-2.7, W=1.0, delta=0.3, p_vac=0.03, seed=4, flux=2 / 16),
    # square lattice, flux * Ly = 3
    dict(lattice=1, Lx=33, Ly=20, t=-1.0, W=2.0, p_vac=0.02, seed=6, flux=3 / 20),
]


def run2d(ctx, d, M, R, alpha, beta, r0=None):
    r0a = None if r0 is None else np.ascontiguousarray(np.stack([r0.real, r0.imag], -1))
    mu = np.zeros((M, M, 2))
    st = kite.moments_2d(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, kite.FP32, r0=r0a), mu, alpha, beta)
    return mu[..., 0] + 1j * mu[..., 1], st


@pytest.mark.parametrize("alpha,beta", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("d", FIELD_CASES, ids=["honeycomb", "square"])
def test_field_2d_moments_match_oracle(ctx, d, alpha, beta):
    M, R = 48, 3
    mu, st = run2d(ctx, d, M, R, alpha, beta)
    ref = oracle.moments_2d(oracle.make_system(**d), M, R, alpha=alpha, beta=beta)
    assert np.max(np.abs(mu - ref)) <= 1e-5 * np.max(np.abs(ref))
    _, vac = oracle.disorder(oracle.make_system(**d))
    assert st.n_eff == int((vac == 0).sum())


def test_field_exact_trace_xy_moments(ctx):
    """Basis start vectors: the exact trace Tr[v_x T_n v_y T_m]/N of a small honeycomb in a
    field, a Hermitian matrix in (n, m) with an imaginary part only because of the field."""
    d = dict(lattice=0, Lx=6, Ly=8, t=-2.7, W=0.5, seed=2, flux=0.25)
    o = oracle.make_system(**d)
    n = oracle.norb(o)
    eye = np.eye(n, dtype=np.complex128)
    M = 40
    mu, _ = run2d(ctx, d, M, n, 0, 1, r0=eye)
    ref = oracle.moments_2d(o, M, n, r0=eye, alpha=0, beta=1)
    assert np.max(np.abs(mu - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert np.max(np.abs(ref - ref.conj().T)) < 1e-12
    assert np.max(np.abs(ref.imag)) > 1e-3 * np.max(np.abs(ref))


KERNELS = [(kite.KERNEL_JACKSON, 0.0, "jackson"), (kite.KERNEL_NONE, 0.0, None),
           (kite.KERNEL_LORENTZ, 3.0, "lorentz")]


@pytest.mark.parametrize("kern", KERNELS, ids=[k[2] or "none" for k in KERNELS])
@pytest.mark.parametrize("kT", [0.0, 0.2])
def test_bastin_reconstruction_matches_oracle(ctx, kern, kT):
    """Same moments (the oracle's exact trace of a disordered honeycomb in a field) through
    both reconstructions; energies across the band and outside it, M_use < M_avail."""
    kid, param, name = kern
    o = oracle.make_system(lattice=0, Lx=6, Ly=4, t=-2.7, W=1.5, p_vac=0.05, seed=8, flux=0.5)
    lo, hi = oracle.bounds_auto(o)
    n = oracle.norb(o)
    M_avail, M_use, eta = 72, 64, 0.05
    mu = oracle.moments_2d(o, M_avail, n, r0=np.eye(n, dtype=np.complex128), alpha=0, beta=1) * n
    E = np.concatenate([np.linspace(lo * 0.98, hi * 0.98, 13), [lo - 0.5, hi + 0.5]])
    ref = oracle.sigma_dc_bastin(mu[:M_use, :M_use], E, lo, hi, eta, oracle.HONEYCOMB,
                                 kernel=name or "none", lam=param, n_quad=200, kT=kT)
    mu_il = np.ascontiguousarray(np.stack([mu.real, mu.imag], -1))
    out = np.zeros(E.size)
    kite.reconstruct_sigma_dc_bastin(ctx, mu_il, M_avail, M_use, oracle.HONEYCOMB, kid, param, lo, hi, eta, kT,
                                     E, E.size, out, n_quad=200)
    assert np.max(np.abs(out - ref)) <= 1e-10 * np.max(np.abs(ref)), (out, ref)
    if kT == 0.0:
        assert out[-2] == 0.0  # below the band: an empty Fermi sea
    torch = pytest.importorskip("torch")
    dev = torch.zeros(E.size, dtype=torch.float64, device="cuda")
    kite.reconstruct_sigma_dc_bastin(ctx, torch.from_numpy(mu_il).cuda(), M_avail, M_use, oracle.HONEYCOMB, kid,
                                     param, lo, hi, eta, kT, torch.from_numpy(E).cuda(), E.size, dev, n_quad=200)
    assert np.array_equal(dev.cpu().numpy(), out)


def test_bastin_from_device_moments_matches_oracle(ctx):
    """End to end on a disordered square lattice in a field: the device's 2D moments and
    reconstruction against the oracle's moments (same start vectors) and formula."""
    d = dict(lattice=1, Lx=40, Ly=32, t=-1.0, W=1.0, seed=9, flux=4 / 32)
    k, o = kite.make_system(**d), oracle.make_system(**d)
    M, R = 96, 2
    n = oracle.norb(o)
    r0 = synth.unit_phase_vectors(n, R, seed=5)
    lo, hi = oracle.bounds_auto(o)
    E = np.linspace(-3.0, 3.0, 11)
    mu_dev, _ = run2d(ctx, d, M, R, 0, 1, r0=r0)
    mu_il = np.ascontiguousarray(np.stack([mu_dev.real, mu_dev.imag], -1))
    out = np.zeros(E.size)
    kite.reconstruct_sigma_dc_bastin(ctx, mu_il, M, M, oracle.SQUARE, kite.KERNEL_JACKSON, 0.0, lo, hi, 0.02, 0.0,
                                     E, E.size, out)
    ref = oracle.sigma_dc_bastin(oracle.moments_2d(o, M, R, r0=r0, alpha=0, beta=1), E, lo, hi, 0.02,
                                 oracle.SQUARE)
    assert np.max(np.abs(out - ref)) <= 2e-3 * np.max(np.abs(ref)), (out, ref)


def test_quantum_hall_plateau_on_the_device(ctx):
    """Graphene 128 x 128 at 1/8 flux quantum per cell: with E_F in the gap between the
    n = 0 and n = 1 Landau levels (0.26 - 2.44 eV) sigma_xy = -e^2/h per spin
    (-1/(2 pi) e^2/hbar), +e^2/h in the mirror gap below zero, flat across the gap, and
    sigma_xx vanishes there; in the gaps near the band edges (1 and 2 of the 16 subbands
    filled, or 2 and 1 empty) the Chern numbers of the Diophantine equation, -1, -2 and
    +2, +1 e^2/h."""
    s = kite.make_system(kite.HONEYCOMB, 128, 128, -2.7, 0.0, flux=0.125)
    lo, hi = kite.bounds(s)
    M, R = 256, 4
    E = np.array([-1.8, -1.35, -0.8, 0.8, 1.35, 1.8])
    edge_E, edge_sigma = np.array([-6.95, -5.9, 5.9, 6.95]), np.array([-1.0, -2.0, 2.0, 1.0])
    E = np.concatenate([E, edge_E])
    out = {}
    for a, b in ((0, 1), (0, 0)):
        mu = np.zeros((M, M, 2))
        kite.moments_2d(ctx, s, kite.make_kpm(M, R, 1, kite.FP32), mu, a, b)
        sig = np.zeros(E.size)
        kite.reconstruct_sigma_dc_bastin(ctx, mu, M, M, kite.HONEYCOMB, kite.KERNEL_JACKSON, 0.0, lo, hi, 0.01, 0.0,
                                         E, E.size, sig)
        out[(a, b)] = sig * 2 * math.pi
    q = out[(0, 1)]
    assert np.all(np.abs(q[:3] - 1.0) < 0.03) and np.all(np.abs(q[3:6] + 1.0) < 0.03), q
    assert np.all(np.abs(q[6:] - edge_sigma) < 0.06), q
    assert np.max(np.abs(out[(0, 0)][:6])) < 0.05, out[(0, 0)]


def test_bastin_rejects_bad_arguments(ctx):
    mu = np.zeros((4, 4, 2))
    out = np.zeros(3)
    E = np.zeros(3)
    for args in ((4, 4, 0, kite.KERNEL_JACKSON, 0.0, -1.0, 1.0, 0.0, 0.0),    # eta = 0
                 (4, 4, 0, kite.KERNEL_JACKSON, 0.0, -1.0, 1.0, 0.1, -1.0),   # kT < 0
                 (4, 5, 0, kite.KERNEL_JACKSON, 0.0, -1.0, 1.0, 0.1, 0.0),    # M_use > M_avail
                 (4, 4, 0, kite.KERNEL_LORENTZ, 0.0, -1.0, 1.0, 0.1, 0.0),    # lambda = 0
                 (4, 4, 0, kite.KERNEL_JACKSON, 0.0, 1.0, 1.0, 0.1, 0.0)):    # empty window
        with pytest.raises(kite.KiteError) as e:
            kite.reconstruct_sigma_dc_bastin(ctx, mu, *args, E, 3, out)
        assert e.value.status == kite.ERR_ARG
    with pytest.raises(kite.KiteError):
        kite.reconstruct_sigma_dc_bastin(ctx, mu, 4, 4, 0, kite.KERNEL_JACKSON, 0.0, -1.0, 1.0, 0.1, 0.0,
                                         np.array([0.0, np.nan, 0.0]), 3, out)
