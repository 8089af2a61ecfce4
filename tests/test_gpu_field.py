"""GPU parity of the 1D moments in a perpendicular magnetic field (Peierls substitution,
Sec. "Magnetic Field") against the oracle, whose phases are pinned by Hermiticity, the
gauge-independent loop traces and the pi-flux spectrum.

Device phases come from CUDA's FP64 sincos and the oracle's from libm (an ulp apart), so
the bars are those against the plain FP64 definition: 1e-12 with FP64 vectors, 1e-5 with
FP32 vectors.  Also: the Landau levels of graphene appear where the continuum theory puts
them, and the calls that take no field refuse one.
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


CASES = [
    # (lattice, Lx, Ly, t, W, delta, p_vac, flux)
    (oracle.HONEYCOMB, 32, 16, -2.7, 1.0, 0.2, 0.02, 2 / 16),   # flux * Ly = 2 (even)
    (oracle.HONEYCOMB, 70, 24, -2.7, 0.5, 0.0, 0.0, 6 / 24),    # ragged strips, several CTAs
    (oracle.SQUARE, 24, 20, -1.0, 2.0, 0.0, 0.05, 3 / 20),      # flux * Ly = 3
    (oracle.SQUARE, 300, 6, -1.0, 0.0, 0.0, 0.0, 0.5),          # pi flux, ragged strip
]


def pair(case, seed):
    lat, Lx, Ly, t, W, delta, p, flux = case
    d = dict(lattice=lat, Lx=Lx, Ly=Ly, t=t, W=W, delta=delta, p_vac=p, seed=seed, flux=flux)
    return kite.make_system(**d), oracle.make_system(**d)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,bar,doubling", [(kite.FP64, 1e-12, False), (kite.FP32, 1e-5, False),
                                               (kite.FP32, 1e-5, True)])
def test_field_moments_match_oracle(ctx, case, prec, bar, doubling):
    k, o = pair(case, 31)
    M, R, S = 96, 3, 2
    mu = np.zeros(M)
    muv = np.zeros((S * R, M, 2))
    st = kite.moments_1d(ctx, k, kite.make_kpm(M, R, S, prec, doubling=doubling), mu, muv)
    ref = np.concatenate([oracle.moments_1d(o, M, R, realisation=s) for s in range(S)], 0)
    assert np.max(np.abs(muv[..., 0] + 1j * muv[..., 1] - ref)) <= bar
    assert np.max(np.abs(mu - ref.real.mean(0))) <= bar
    assert st.steps_per_pass == 1
    _, vac = oracle.disorder(o, S - 1)
    assert st.n_eff == int((vac == 0).sum())


def test_field_exact_trace_and_last_iterates(ctx):
    """Basis start vectors (exact trace) in FP64, and the last two iterates against the
    oracle's Chebyshev sums T_{M-2} r, T_{M-1} r for one random start vector."""
    k, o = pair((oracle.HONEYCOMB, 6, 8, -2.7, 1.5, 0.0, 0.1, 0.25), 5)
    n = oracle.norb(o)
    eye = np.eye(n, dtype=np.complex128)
    r0a = np.ascontiguousarray(np.stack([eye.real, eye.imag], -1))
    M = 24
    muv = np.zeros((n, M, 2))
    kite.moments_1d(ctx, k, kite.make_kpm(M, n, 1, kite.FP64, r0=r0a), np.zeros(M), muv)
    ref = oracle.moments_1d(o, M, n, r0=eye)
    assert np.max(np.abs((muv[..., 0] + 1j * muv[..., 1]).sum(0) - ref.sum(0))) <= 1e-12
    r = np.exp(2j * np.pi * np.random.default_rng(3).random(n))
    last = np.zeros((1, 2, n), np.complex128)
    ra = np.ascontiguousarray(np.stack([r.real, r.imag], -1)[None])
    kite.moments_1d(ctx, k, kite.make_kpm(M, 1, 1, kite.FP64, r0=ra, r_last=last), np.zeros(M))
    _, vac = oracle.disorder(o)
    rr = np.where(vac == 0, r, 0)
    for slot, m in ((0, M - 2), (1, M - 1)):
        c = np.zeros(m + 1, complex)
        c[m] = 1.0
        assert np.max(np.abs(last[0, slot] - oracle.chebyshev_sum(o, c, rr))) <= 1e-12


def test_graphene_landau_levels_in_the_dos(ctx):
    """Clean graphene at 1/128 flux quantum per cell (about 300 T for a = 2.46 A): the DOS
    peaks at E_n = |t| sqrt(2 sqrt(3) pi flux n) (the continuum Landau levels, n = 1, 2)
    within the lattice corrections (of order flux * n: 6 % for n = 2 at flux 1/32, measured),
    and the n = 0 level at E = 0 holds 2 flux N_cells states (both valleys), i.e. a fraction
    flux of the orbitals."""
    L, flux, t = 256, 1 / 128, -2.7
    s = kite.make_system(kite.HONEYCOMB, L, L, t, 0.0, flux=flux)
    M, R = 2048, 8
    lo, hi = kite.bounds(s)
    mu = np.zeros(M)
    kite.moments_1d(ctx, s, kite.make_kpm(M, R, 1, kite.FP32, doubling=True), mu)
    E = np.linspace(-3.0, 3.0, 6001)
    rho = np.zeros(E.size)
    kite.reconstruct_dos(ctx, mu, M, M, kite.KERNEL_JACKSON, 0.0, lo, hi, E, E.size, rho)
    for n in (1, 2):
        En = abs(t) * math.sqrt(2 * math.sqrt(3) * math.pi * flux * n)
        w = (E > 0.92 * En) & (E < 1.08 * En)  # between the neighbouring levels (En +- 15 % or more)
        peak = E[w][np.argmax(rho[w])]
        assert abs(peak - En) <= 0.03 * En and 0.94 * En < peak < 1.06 * En, (n, peak, En)
    # weight of the zero level: integral of rho per orbital between the n = 0 and n = +-1
    # levels' midpoints = (2 flux N_cells) / (2 N_cells) = flux
    E1 = abs(t) * math.sqrt(2 * math.sqrt(3) * math.pi * flux)
    w0 = np.abs(E) < 0.5 * E1
    Ew, rw = E[w0], rho[w0]
    weight = float(np.sum(0.5 * (rw[1:] + rw[:-1]) * np.diff(Ew)))
    assert abs(weight - flux) <= 0.15 * flux


def test_flux_that_does_not_fit_is_refused_with_the_nearest(ctx):
    s = kite.make_system(kite.HONEYCOMB, 16, 16, -2.7, 0.0, flux=0.1)
    with pytest.raises(kite.KiteError) as e:
        kite.moments_1d(ctx, s, kite.make_kpm(8, 1, 1, kite.FP32), np.zeros(8))
    assert e.value.status == kite.ERR_ARG and "nearest: 0.125" in str(e.value)
    assert kite.flux_nearest(s, 0.1) == 0.125


def test_calls_without_field_support_refuse_a_field(ctx):
    s = kite.make_system(kite.SQUARE, 16, 16, -1.0, 0.0, flux=0.25)
    with pytest.raises(kite.KiteError):
        kite.moments_1d(ctx, s, kite.make_kpm(8, 2, 1, kite.FP32, real_vectors=True), np.zeros(8))
    with pytest.raises(kite.KiteError):
        kite.moments_1d_static(s, kite.make_kpm(8, 2, 1, kite.FP32), np.zeros(8))


@pytest.mark.parametrize("prec,bar", [(kite.FP64, 1e-10), (kite.FP32, 2e-5)])
@pytest.mark.parametrize("lattice,Ly,flux,oy", [(oracle.HONEYCOMB, 16, 2 / 16, 0), (oracle.SQUARE, 20, 3 / 20, 0),
                                                 (oracle.SQUARE, 15, 0.07, 1)])
def test_wave_packet_evolution_in_a_field(ctx, lattice, Ly, flux, oy, prec, bar):
    """exp(-i H dt) with the Peierls phases (and with y open, a flux that does not fit the
    torus) against the oracle's Chebyshev propagator on its own field Hamiltonian; the
    norm is conserved."""
    t = -2.7 if lattice == oracle.HONEYCOMB else -1.0
    d = dict(lattice=lattice, Lx=30, Ly=Ly, t=t, W=0.5, p_vac=0.02, seed=12, flux=flux, open_y=oy)
    o = oracle.make_system(**d)
    n = oracle.norb(o)
    R, dt, steps, M = 2, 0.6, 3, 48
    psi0 = synth.unit_phase_vectors(n, R, seed=4) / np.sqrt(n)
    psi = np.ascontiguousarray(np.stack([psi0.real, psi0.imag], -1))
    norms = np.zeros((steps, R))
    kite.propagate(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, prec), dt, steps, psi, norms)
    for r in range(R):
        ref = oracle.propagate(o, psi0[r], dt, steps, M)
        assert np.max(np.abs(psi[r, :, 0] + 1j * psi[r, :, 1] - ref[-1])) <= bar * max(1.0, np.max(np.abs(ref[-1])))
        assert np.max(np.abs(norms[:, r] - np.sum(np.abs(ref) ** 2, axis=1))) <= (1e-10 if prec == kite.FP64 else 1e-5)


@pytest.mark.parametrize("doubling", [False, True])
def test_batched_sweep_with_fields(ctx, doubling):
    """One persistent launch over systems with different fluxes (one without a field, whose
    phases are identity rotations): each against the oracle's plain moments in its field."""
    specs = [(40, 20, 0.15, 1.0, 11), (24, 10, 0.0, 2.0, 12), (96, 8, 0.5, 0.5, 13), (16, 16, 0.25, 1.5, 14)]
    pairs = []
    for Lx, Ly, flux, W, seed in specs:
        d = dict(lattice=oracle.SQUARE, Lx=Lx, Ly=Ly, t=-1.0, W=W, p_vac=0.02, seed=seed, flux=flux)
        pairs.append((kite.make_system(**d), oracle.make_system(**d)))
    M, R = 64, 4
    mus = [np.zeros(M) for _ in pairs]
    kite.moments_1d_batched(ctx, [p[0] for p in pairs],
                            [kite.make_kpm(M, R, 1, kite.FP32, doubling=doubling) for _ in pairs], mus)
    for (k, o), mu in zip(pairs, mus):
        ref = oracle.moments_1d(o, M, R).real.mean(0)
        assert np.max(np.abs(mu - ref)) <= 1e-5
