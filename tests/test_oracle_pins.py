"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form
(Bloch dispersion of the clean lattice), a library routine (dense
``numpy.linalg.eigh``), an exact low-order trace identity, the white-noise
statistics the paper asks of the random vectors (Sec. 2c), or an exact quadrature
rule.  A dropped term, a wrong sign, a transposed index or an inverted prefactor in
the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle

T_EV = -2.7


def cheb_T(n_max, x):
    """T_0..T_{n_max-1} at x via cos(n arccos x) (closed form, not the recursion)."""
    x = np.clip(np.asarray(x, np.float64), -1.0, 1.0)
    th = np.arccos(x)
    n = np.arange(n_max)[:, None]
    return np.cos(n * th[None, :])


def dense_h(sys, realisation=0, e_min=None, e_max=None):
    """Dense rescaled Hamiltonian on the non-vacant orbitals (uses oracle geometry and
    draws, which the Bloch test pins independently)."""
    n = oracle.norb(sys)
    lo, hi = (oracle.bounds_auto(sys) if e_min is None else (e_min, e_max))
    dp, dm = 0.5 * (hi + lo), 0.5 * (hi - lo)
    V, vac = oracle.disorder(sys, realisation)
    H = np.zeros((n, n))
    for o in range(n):
        if vac[o]:
            continue
        H[o, o] = (V[o] - dp) / dm
        for j in oracle.neighbours(sys, o):
            if not vac[j]:
                H[o, j] += sys.t / dm
    keep = np.where(vac == 0)[0]
    return H[np.ix_(keep, keep)], keep, vac


def exact_trace_moments(sys, M, realisation=0, e_min=None, e_max=None):
    """Oracle run with every basis vector as a start vector: sum over vectors of
    <e_o|T_n|e_o>/N_eff = Tr T_n(H~)/N_eff."""
    n = oracle.norb(sys)
    r0 = np.eye(n, dtype=np.complex128)
    mu = oracle.moments_1d(sys, M, n, realisation=realisation, e_min=e_min, e_max=e_max, r0=r0)
    return mu.sum(axis=0)


# --------------------------------------------------------------------------- RNG


def test_philox_white_noise_statistics():
    """Uniform draws: chi-square flat over 64 bins, independent words, distinct
    counters give distinct blocks (Sec. 2c asks for white-noise variables only)."""
    words = np.array([oracle.philox([i, 0, 7, 1], [123, 0]) for i in range(20000)], np.uint64)
    u = ((words[:, 0] << np.uint64(21)) | (words[:, 1] >> np.uint64(11))).astype(np.float64) * 2.0**-53
    counts, _ = np.histogram(u, bins=64, range=(0.0, 1.0))
    exp = len(u) / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 120.0  # 63 dof: mean 63, sd 11
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))
    # each output bit is balanced
    bits = ((words[:, 2][:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    assert np.all(np.abs(bits.mean(0) - 0.5) < 5 * 0.5 / math.sqrt(len(u)))
    # words of one block are uncorrelated
    f = words.astype(np.float64) / 2**32
    c = np.corrcoef(f.T)
    assert np.all(np.abs(c - np.eye(4)) < 5 / math.sqrt(len(u)))
    assert len({tuple(w) for w in words.tolist()}) == len(words)
    # the key changes the stream
    assert oracle.philox([0, 0, 7, 1], [123, 0]) != oracle.philox([0, 0, 7, 1], [124, 0])


def test_philox_known_answer_vectors():
    """The generator's published known-answer vectors (all-zero, all-ones and pi-digit
    blocks; Salmon et al., SC'11) reproduced word for word: a wrong multiplier, Weyl
    constant, round count or word order changes every output word."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        assert oracle.philox(w[0:4], w[4:6]) == w[6:10], r


def test_disorder_distribution_and_vacancies():
    """V uniform in [-W/2, W/2] +/- delta/2 (Sec. 4b); vacancies Bernoulli(p)."""
    W, delta, p = 2.0, 0.6, 0.05
    sys = oracle.make_system(Lx=128, Ly=96, W=W, delta=delta, p_vac=p, seed=11)
    V, vac = oracle.disorder(sys)
    n = V.size
    VA, VB = V[0::2] - delta / 2, V[1::2] + delta / 2
    for v in (VA, VB):
        assert v.min() >= -W / 2 and v.max() < W / 2
        assert abs(v.mean()) < 5 * W / math.sqrt(12 * v.size)
        assert abs(v.var() - W * W / 12) < 0.02 * W * W / 12 + 5 * W * W / 12 / math.sqrt(v.size)
    frac = vac.mean()
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n)
    sys0 = oracle.make_system(Lx=16, Ly=16, W=0.0, p_vac=0.0)
    V0, vac0 = oracle.disorder(sys0)
    assert np.all(V0 == 0.0) and np.all(vac0 == 0)
    sys1 = oracle.make_system(Lx=8, Ly=8, p_vac=1.0)
    assert np.all(oracle.disorder(sys1)[1] == 1)


def test_gaussian_disorder_distribution_and_bound():
    """Gaussian disorder (the Python interface's 'Gaussian' kind, Sec. 3d): V ~ N(0, W^2)
    +/- delta/2 per sublattice: mean, variance and kurtosis of 131k draws within their
    sampling errors, normal quantiles within a few per cent, every draw inside the
    transform's largest value sqrt(106 ln 2) W, vacancies as for uniform disorder, and
    the Gershgorin bounds built from that largest value."""
    W, delta, p = 0.7, 0.4, 0.03
    sys = oracle.make_system(Lx=256, Ly=256, W=W, delta=delta, p_vac=p, seed=12,
                             disorder=oracle.GAUSSIAN)
    V, vac = oracle.disorder(sys)
    for v in (V[0::2] - delta / 2, V[1::2] + delta / 2):
        n = v.size
        z = v / W
        assert abs(z.mean()) < 5 / math.sqrt(n)
        assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
        assert abs(np.mean(z ** 4) / z.var() ** 2 - 3.0) < 5 * math.sqrt(24.0 / n)
        # P(|z| < 1) = erf(1/sqrt 2) = 0.6826895, P(|z| < 2) = 0.9544997
        assert abs(np.mean(np.abs(z) < 1.0) - 0.6826895) < 0.01
        assert abs(np.mean(np.abs(z) < 2.0) - 0.9544997) < 0.005
        assert np.max(np.abs(z)) <= math.sqrt(106 * math.log(2))
    assert abs(vac.mean() - p) < 5 * math.sqrt(p * (1 - p) / V.size)
    lo, hi = oracle.bounds_auto(sys)
    assert abs(hi - (3 * 2.7 + 8.58 * W + delta / 2) * 1.01) < 1e-12 and lo == -hi
    # same seed, uniform kind: the same vacancies (third word), other on-site values
    Vu, vacu = oracle.disorder(oracle.make_system(Lx=256, Ly=256, W=W, delta=delta, p_vac=p, seed=12))
    assert np.array_equal(vacu, vac) and not np.allclose(Vu, V)


def test_gaussian_disorder_enters_the_second_moment():
    """Exact trace with Gaussian disorder (no vacancies): mu_2 = 2 Tr(H~^2)/N - 1 with
    Tr(H~^2)/N = 3 t~^2 + <V~^2>, and <V^2> within its sampling error of W^2 + delta^2/4."""
    W, delta = 0.9, 0.3
    sys = oracle.make_system(Lx=8, Ly=6, W=W, delta=delta, seed=13, disorder=oracle.GAUSSIAN)
    n = oracle.norb(sys)
    lo, hi = oracle.bounds_auto(sys)
    mu = oracle.moments_1d(sys, 3, n, r0=np.eye(n, dtype=np.complex128)).real.sum(0)
    V, _ = oracle.disorder(sys)
    tt = 2.7 / hi
    assert abs(mu[0] - 1.0) < 1e-12 and abs(mu[1] - np.mean(V) / hi) < 1e-12
    assert abs(mu[2] - (2 * (3 * tt * tt + np.mean((V / hi) ** 2)) - 1)) < 1e-12
    big, _ = oracle.disorder(oracle.make_system(Lx=256, Ly=256, W=W, delta=delta, seed=14,
                                                disorder=oracle.GAUSSIAN))
    assert abs(np.mean(big ** 2) - (W * W + delta * delta / 4)) < 5 * W * W * math.sqrt(2.0 / big.size) + 0.01


def dense_from_operator(sys):
    """The oracle's own rescaled Hamiltonian as a dense matrix, column j = H~ e_j (its
    Chebyshev sum with coefficients (0, 1))."""
    n = oracle.norb(sys)
    eye = np.eye(n, dtype=np.complex128)
    return np.array([oracle.chebyshev_sum(sys, np.array([0.0, 1.0], complex), eye[:, j])
                     for j in range(n)]).T


def power_traces(sys, kmax):
    """<x^k> = Tr(H~^k)/N for k <= kmax from exact-trace Chebyshev moments."""
    mu = exact_trace_moments(sys, kmax + 1).real
    # x^k in Chebyshev polynomials: coefficients from numpy's conversion
    out = []
    for k in range(kmax + 1):
        c = np.polynomial.chebyshev.poly2cheb([0] * k + [1])
        out.append(float(np.dot(c, mu[:k + 1])))
    return np.array(out)


@pytest.mark.parametrize("lattice,flux", [(oracle.SQUARE, 0.25), (oracle.SQUARE, 0.375),
                                          (oracle.HONEYCOMB, 0.25), (oracle.HONEYCOMB, 0.5)])
def test_peierls_phases_hermitian_and_loop_traces(lattice, flux):
    """Magnetic field by Peierls substitution (Sec. "Magnetic Field"): H~ stays Hermitian
    on the torus, |H~_ij| = |t~|, and the flux enters only through closed loops: the
    smallest loops enclose one unit cell (square plaquette: 4 bonds, 8 walks per site;
    honeycomb hexagon: 6 bonds, 6 walks per site), so <x^4> (square) and <x^6>
    (honeycomb) move by 8 t~^4 (cos 2 pi flux - 1) and 6 t~^6 (cos 2 pi flux - 1), and
    the lower traces do not move.  Gauge-independent closed forms."""
    t = -1.0 if lattice == oracle.SQUARE else T_EV
    base = dict(lattice=lattice, Lx=8, Ly=8, t=t)
    sysB = oracle.make_system(flux=flux, **base)
    sys0 = oracle.make_system(**base)
    H = dense_from_operator(sysB)
    assert np.max(np.abs(H - H.conj().T)) < 1e-15
    lo, hi = oracle.bounds_auto(sysB)
    tt = abs(t) / hi
    off = np.abs(H[~np.eye(H.shape[0], dtype=bool)])
    assert np.all((off < 1e-15) | (np.abs(off - tt) < 1e-15))
    pB, p0 = power_traces(sysB, 6), power_traces(sys0, 6)
    c = math.cos(2 * math.pi * flux) - 1.0
    if lattice == oracle.SQUARE:
        assert np.max(np.abs(pB[:4] - p0[:4])) < 1e-13
        assert abs(pB[4] - p0[4] - 8 * tt ** 4 * c) < 1e-13
    else:
        assert np.max(np.abs(pB[:6] - p0[:6])) < 1e-13
        assert abs(pB[6] - p0[6] - 6 * tt ** 6 * c) < 1e-13


def test_pi_flux_square_lattice_spectrum():
    """Half a flux quantum per plaquette on the square lattice: the closed-form spectrum
    E = +-2|t| sqrt(cos^2 kx + cos^2 ky), kx = 2 pi a/Lx, ky = 2 pi b/Ly, b < Ly/2
    (two-row magnetic cell), against dense diagonalisation of the oracle's operator."""
    Lx, Ly, t = 6, 8, -1.0
    sys = oracle.make_system(lattice=oracle.SQUARE, Lx=Lx, Ly=Ly, t=t, flux=0.5)
    lo, hi = oracle.bounds_auto(sys)
    lam = np.sort(np.linalg.eigvalsh(dense_from_operator(sys)) * hi)
    kx = 2 * np.pi * np.arange(Lx) / Lx
    ky = 2 * np.pi * np.arange(Ly // 2) / Ly
    KX, KY = np.meshgrid(kx, ky, indexing="ij")
    e = (2 * abs(t) * np.sqrt(np.cos(KX) ** 2 + np.cos(KY) ** 2)).ravel()
    ref = np.sort(np.concatenate([e, -e]))
    assert np.max(np.abs(lam - ref)) < 1e-12


def test_flux_must_fit_the_torus():
    """The Landau-gauge phases repeat after Ly rows only for flux * Ly even (honeycomb)
    or integer (square); other fluxes are refused."""
    with pytest.raises(ValueError):
        oracle.moments_1d(oracle.make_system(lattice=oracle.SQUARE, Lx=8, Ly=8, t=-1.0, flux=0.3), 4, 1)
    with pytest.raises(ValueError):
        oracle.moments_1d(oracle.make_system(Lx=8, Ly=8, flux=0.125), 4, 1)  # 0.125 * 8 = 1: odd
    oracle.moments_1d(oracle.make_system(Lx=8, Ly=8, flux=0.25), 4, 1)


def wrap_classes(sys):
    """For every pair of orbitals, which periodic images separate them at the shortest
    distance: (m, n) with r_i - r_j + m T1 + n T2 minimal, T1 = Lx a1, T2 = Ly a2.  A bond
    with m != 0 wraps around x, n != 0 around y (positions from the orbital set-up)."""
    P = oracle.orbital_positions(sys)
    if sys.lattice == oracle.HONEYCOMB:
        T1, T2 = np.array([sys.Lx, 0.0]), np.array([0.5 * sys.Ly, 0.5 * math.sqrt(3.0) * sys.Ly])
    else:
        T1, T2 = np.array([sys.Lx, 0.0]), np.array([0.0, sys.Ly])
    d0 = P[:, None, :] - P[None, :, :]
    best = np.sum(d0 * d0, -1)
    cls = np.zeros(best.shape + (2,), int)
    for m in (-1, 0, 1):
        for k in (-1, 0, 1):
            c = d0 + m * T1 + k * T2
            dd = np.sum(c * c, -1)
            better = dd < best - 1e-9
            best[better] = dd[better]
            cls[better] = (m, k)
    return cls


@pytest.mark.parametrize("lattice", [oracle.HONEYCOMB, oracle.SQUARE])
@pytest.mark.parametrize("ox,oy", [(1, 0), (0, 1), (1, 1)])
def test_open_boundaries_remove_exactly_the_wrapping_bonds(lattice, ox, oy):
    """Open boundaries (the configuration's boundaries flag): H~ of the open lattice is the
    periodic H~ (pinned by the Bloch tests) without the bonds that wrap around the torus
    along the open directions, those bonds found geometrically from the orbital positions
    and the torus periods; disorder, vacancies and every other bond unchanged."""
    t = -1.0 if lattice == oracle.SQUARE else T_EV
    base = dict(lattice=lattice, Lx=5, Ly=4, t=t, W=1.0, p_vac=0.05, seed=6)
    per = oracle.make_system(**base)
    opn = oracle.make_system(open_x=ox, open_y=oy, **base)
    Hp, Ho = dense_from_operator(per), dense_from_operator(opn)
    cls = wrap_classes(per)
    cut = ((cls[..., 0] != 0) & bool(ox)) | ((cls[..., 1] != 0) & bool(oy))
    expect = np.where(cut, 0.0, Hp)
    assert np.max(np.abs(Ho - expect)) == 0.0
    assert np.count_nonzero(Hp[cut]) > 0  # the test removes something
    for d in (0, 1):  # the velocity loses the same bonds
        assert np.max(np.abs(dense_v(opn, d) - np.where(cut, 0.0, dense_v(per, d)))) == 0.0


def test_open_square_lattice_spectrum():
    """Clean square lattice with open boundaries: standing waves, E = 2t cos(pi m/(L+1))
    along an open direction and 2t cos(2 pi k/L) along a periodic one (textbook)."""
    for ox, oy in ((1, 0), (1, 1)):
        Lx, Ly, t = 7, 6, -1.0
        sys = oracle.make_system(lattice=oracle.SQUARE, Lx=Lx, Ly=Ly, t=t, open_x=ox, open_y=oy)
        lo, hi = oracle.bounds_auto(sys)
        lam = np.sort(np.linalg.eigvalsh(dense_from_operator(sys)) * hi)
        ex = 2 * t * np.cos(np.pi * np.arange(1, Lx + 1) / (Lx + 1))
        ey = (2 * t * np.cos(np.pi * np.arange(1, Ly + 1) / (Ly + 1)) if oy
              else 2 * t * np.cos(2 * np.pi * np.arange(Ly) / Ly))
        ref = np.sort((ex[:, None] + ey[None, :]).ravel())
        assert np.max(np.abs(lam - ref)) < 1e-12


def test_field_with_an_open_boundary():
    """A field on a lattice open along y needs no commensurate flux (no bond wraps in y):
    H~ stays Hermitian and every plaquette inside encloses the flux, so <x^4> of the square
    lattice moves by 8 t~^4 (cos 2 pi flux - 1) per plaquette, Lx (Ly - 1) of them."""
    Lx, Ly, t, flux = 6, 5, -1.0, 0.1
    sysB = oracle.make_system(lattice=oracle.SQUARE, Lx=Lx, Ly=Ly, t=t, flux=flux, open_y=1)
    sys0 = oracle.make_system(lattice=oracle.SQUARE, Lx=Lx, Ly=Ly, t=t, open_y=1)
    H = dense_from_operator(sysB)
    assert np.max(np.abs(H - H.conj().T)) < 1e-15
    lo, hi = oracle.bounds_auto(sysB)
    tt = abs(t) / hi
    n = Lx * Ly
    pB, p0 = power_traces(sysB, 4), power_traces(sys0, 4)
    assert np.max(np.abs(pB[:4] - p0[:4])) < 1e-13
    shift = 8 * tt ** 4 * (math.cos(2 * math.pi * flux) - 1) * Lx * (Ly - 1) / n
    assert abs(pB[4] - p0[4] - shift) < 1e-13
    with pytest.raises(ValueError):  # periodic in y, the same flux does not fit
        oracle.moments_1d(oracle.make_system(lattice=oracle.SQUARE, Lx=Lx, Ly=Ly, t=t, flux=flux), 4, 1)


def test_random_phase_is_white_noise():
    """|xi| = 1 off vacancies, 0 on them; <xi> = 0, <xi xi> = 0, <|xi|^2> = 1 (Sec. 2c)."""
    sys = oracle.make_system(Lx=64, Ly=64, p_vac=0.02, seed=3)
    xi = oracle.random_phase(sys, R=4)
    _, vac = oracle.disorder(sys)
    on = vac == 0
    assert np.all(xi[:, ~on] == 0)
    assert np.allclose(np.abs(xi[:, on]), 1.0, atol=1e-15)
    z = xi[:, on].ravel()
    tol = 5 / math.sqrt(z.size)
    assert abs(z.mean()) < tol
    assert abs((z * z).mean()) < tol
    # different vectors are independent
    assert abs(np.vdot(xi[0, on], xi[1, on]) / on.sum()) < tol * 2


# --------------------------------------------------------------- 1D moments


def bloch_moments(lattice, Lx, Ly, t, M, e_min, e_max):
    """Exact-trace moments of the clean periodic lattice from its Bloch dispersion."""
    dm = 0.5 * (e_max - e_min)
    dp = 0.5 * (e_max + e_min)
    k1 = 2 * np.pi * np.arange(Lx) / Lx
    k2 = 2 * np.pi * np.arange(Ly) / Ly
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    if lattice == oracle.HONEYCOMB:
        # A(x,y) couples to B(x,y), B(x+1,y-1), B(x,y-1)  (Listing 1 hoppings)
        f = t * (1 + np.exp(1j * (K1 - K2)) + np.exp(-1j * K2))
        E = np.concatenate([np.abs(f).ravel(), -np.abs(f).ravel()])
    else:
        E = (2 * t * (np.cos(K1) + np.cos(K2))).ravel()
    x = (E - dp) / dm
    return cheb_T(M, x).mean(axis=1)


@pytest.mark.parametrize("lattice,Lx,Ly", [(oracle.HONEYCOMB, 4, 3), (oracle.HONEYCOMB, 5, 7),
                                            (oracle.SQUARE, 6, 5), (oracle.SQUARE, 3, 8)])
def test_exact_trace_matches_bloch_dispersion(lattice, Lx, Ly):
    t = T_EV if lattice == oracle.HONEYCOMB else -1.0
    sys = oracle.make_system(lattice=lattice, Lx=Lx, Ly=Ly, t=t)
    lo, hi = oracle.bounds_auto(sys)
    M = 40
    mu = exact_trace_moments(sys, M)
    ref = bloch_moments(lattice, Lx, Ly, t, M, lo, hi)
    assert np.max(np.abs(mu.real - ref)) < 1e-12
    assert np.max(np.abs(mu.imag)) < 1e-12
    if lattice == oracle.HONEYCOMB:  # bipartite: odd moments vanish
        assert np.max(np.abs(mu.real[1::2])) < 1e-12


def test_exact_trace_matches_dense_diagonalisation_with_disorder():
    sys = oracle.make_system(Lx=5, Ly=4, W=2.0, delta=0.4, p_vac=0.1, seed=21)
    M = 32
    H, keep, _ = dense_h(sys)
    lam = np.linalg.eigvalsh(H)
    assert np.all(np.abs(lam) <= 1.0)  # Gershgorin bounds hold (Sec. 2a, ||X|| <= 1)
    ref = cheb_T(M, lam).mean(axis=1)
    mu = exact_trace_moments(sys, M)
    assert np.max(np.abs(mu.real - ref)) < 1e-12


def test_low_order_exact_trace_identities():
    """mu_0 = 1, mu_1 = mean V~, mu_2 = 2 mean(Z_i t~^2 + V~_i^2) - 1 on non-vacant
    orbitals, Z_i counting non-vacant neighbours."""
    sys = oracle.make_system(lattice=oracle.SQUARE, Lx=6, Ly=5, t=-1.0, W=3.0, p_vac=0.15, seed=4)
    lo, hi = -7.0, 6.0  # asymmetric bounds: exercises de_plus
    mu = exact_trace_moments(sys, 3, e_min=lo, e_max=hi).real
    V, vac = oracle.disorder(sys)
    dp, dm = 0.5 * (hi + lo), 0.5 * (hi - lo)
    on = np.where(vac == 0)[0]
    Vt = (V[on] - dp) / dm
    Z = np.array([sum(1 for j in oracle.neighbours(sys, o) if not vac[j]) for o in on])
    tt = sys.t / dm
    assert abs(mu[0] - 1.0) < 1e-14
    assert abs(mu[1] - Vt.mean()) < 1e-14
    assert abs(mu[2] - (2 * np.mean(Z * tt * tt + Vt * Vt) - 1)) < 1e-13


def test_stochastic_estimate_within_trace_variance():
    """Random-phase estimate vs exact trace: the STE variance for unit-modulus phases
    is sum_{i!=j}|A_ij|^2 / N_eff^2 per vector (Sec. 2c)."""
    sys = oracle.make_system(Lx=6, Ly=6, W=1.0, p_vac=0.05, seed=8)
    M, R = 24, 6
    H, keep, _ = dense_h(sys)
    lam, U = np.linalg.eigh(H)
    Tn = cheb_T(M, lam)
    mu = oracle.moments_1d(sys, M, R).real.mean(axis=0)
    ne = H.shape[0]
    for n in range(M):
        A = (U * Tn[n]) @ U.T
        exact = np.trace(A) / ne
        var = (np.sum(A * A) - np.sum(np.diag(A) ** 2)) / ne**2 / R
        assert abs(mu[n] - exact) <= 5 * math.sqrt(var) + 1e-13, n


def test_replica_agrees_with_definition():
    sys = oracle.make_system(Lx=8, Ly=6, W=1.0, p_vac=0.03, seed=9)
    M, R = 64, 2
    mu = oracle.moments_1d(sys, M, R)
    mu64, last64 = oracle.replica_1d(sys, M, R, precision=1, want_last=True)
    mu32, last32 = oracle.replica_1d(sys, M, R, precision=0, want_last=True)
    assert np.max(np.abs(mu64 - mu)) < 1e-12
    assert np.max(np.abs(mu32 - mu)) < 5e-6
    assert np.max(np.abs(last32 - last64)) < 1e-4
    _, vac = oracle.disorder(sys)
    assert np.all(last32[:, :, vac == 1] == 0)


def test_replica_is_exact_on_dyadic_inputs():
    """With t~ = 1/8, no disorder and +-1 start vectors every iterate is a dyadic
    rational that fits in FP32 for the first steps: FP32, FP64 and the plain
    definition must then agree exactly."""
    sys = oracle.make_system(lattice=oracle.SQUARE, Lx=5, Ly=4, t=-1.0)
    n = oracle.norb(sys)
    rng = np.random.default_rng(0)
    r0 = rng.choice([-1.0, 1.0], size=(1, n)).astype(np.complex128)
    r0 = r0 + 1j * rng.choice([-1.0, 1.0], size=(1, n))
    kw = dict(e_min=-8.0, e_max=8.0, r0=r0)
    mu = oracle.moments_1d(sys, 6, 1, **kw)
    m32, l32 = oracle.replica_1d(sys, 6, 1, 0, want_last=True, **kw)
    m64, l64 = oracle.replica_1d(sys, 6, 1, 1, want_last=True, **kw)
    assert np.array_equal(l32.astype(np.complex128), l64)
    assert np.array_equal(m32, mu) and np.array_equal(m64, mu)


# ------------------------------------------------------------ reconstruction


def test_jackson_kernel_properties():
    for M in (8, 64, 1000):
        g = oracle.kernel_jackson(M)
        assert abs(g[0] - 1.0) < 1e-15
        assert np.all(np.diff(g) < 0) and g[-1] > 0
    # the Jackson-damped expansion of a delta function has variance ~ (pi/M)^2
    # at the band centre (Weisse et al. 2006): check with the exact moments of x0=0
    M = 256
    g = oracle.kernel_jackson(M)
    mu = cheb_T(M, np.array([0.0]))[:, 0]
    xs = np.cos(np.pi * (np.arange(4096) + 0.5) / 4096)
    rho = oracle.dos(mu, xs, -1.0, 1.0, g)
    w = np.pi / 4096 * np.sqrt(1 - xs**2) * rho
    var = np.sum(w * xs**2)
    assert abs(var / (np.pi / M) ** 2 - 1.0) < 0.05


def test_dos_quadrature_sum_rules():
    """On K Gauss-Chebyshev nodes (exact for these polynomial degrees),
    (pi/K) sum sqrt(1-e^2) rho(e) T_j(e) = int rho T_j = g_j mu_j for every j, by the
    orthogonality of Eq. e4.  This fixes the (2 - delta_n0) weight of the delta-function
    expansion (the printed (1+delta_n0)/2 of Eq. e8 would give g_j mu_j / 4 for j >= 1)."""
    sys = oracle.make_system(Lx=6, Ly=5, W=1.5, seed=2)
    lo, hi = oracle.bounds_auto(sys)
    M = 48
    mu = exact_trace_moments(sys, M).real
    g = oracle.kernel_jackson(M)
    K = 512
    eps = np.cos(np.pi * (np.arange(K) + 0.5) / K)
    E = eps * 0.5 * (hi - lo) + 0.5 * (hi + lo)
    rho = oracle.dos(mu, E, lo, hi, g) * 0.5 * (hi - lo)  # per unit eps
    w = np.pi / K * np.sqrt(1 - eps**2) * rho
    Tj = cheb_T(6, eps)
    assert abs(w.sum() - g[0] * mu[0]) < 1e-12
    for j in range(1, 6):
        assert abs(np.sum(w * Tj[j]) - g[j] * mu[j]) < 1e-12
    assert np.all(rho > -1e-12)  # Jackson kernel keeps the exact-trace DOS positive


def test_dos_matches_broadened_spectrum():
    """Jackson DOS of exact-trace moments vs the dense spectrum smeared by the same
    kernel evaluated in closed form."""
    sys = oracle.make_system(Lx=6, Ly=6, W=2.0, seed=5)
    lo, hi = oracle.bounds_auto(sys)
    M = 64
    H, _, _ = dense_h(sys)
    lam = np.linalg.eigvalsh(H)
    g = oracle.kernel_jackson(M)
    eps = np.linspace(-0.95, 0.95, 77)
    Te = cheb_T(M, eps)
    Tl = cheb_T(M, lam)
    coef = g * (2.0 - (np.arange(M) == 0))
    ref = (coef[:, None] * Te * Tl.mean(axis=1)[:, None]).sum(0) / (np.pi * np.sqrt(1 - eps**2))
    mu = exact_trace_moments(sys, M).real
    dm = 0.5 * (hi - lo)
    rho = oracle.dos(mu, eps * dm, lo, hi, g) * dm
    assert np.max(np.abs(rho - ref)) < 1e-11


def test_cpgf_coefficients_resum_the_resolvent():
    """sum_n g_n(eps) T_n(x)/(1+delta_n0) -> 1/(eps - x + i sigma eta) (Eqs.
    green_function_cheb_expansion/b), uniformly in x for fixed eta."""
    eta = 0.05
    M = 1500
    for sigma in (+1, -1):
        for eps in (-0.7, 0.0, 0.33):
            gn = np.array([oracle.cpgf_coeff(n, eps, eta, sigma) for n in range(M)])
            gn[0] *= 0.5
            for x in (-0.9, -0.2, 0.1, 0.8):
                s = np.sum(gn * cheb_T(M, np.array([x]))[:, 0])
                ref = 1.0 / (eps - x + 1j * sigma * eta)
                assert abs(s - ref) < 1e-6 * abs(ref), (sigma, eps, x)


def test_lorentz_kernel_definition():
    g = oracle.kernel_lorentz(100, 4.0)
    assert abs(g[0] - 1.0) < 1e-15
    assert abs(g[50] - math.sinh(2.0) / math.sinh(4.0)) < 1e-15


# ---------------------------------------------------------------- 2D moments


def dense_vx(sys, vac, tt):
    n = oracle.norb(sys)
    cols = [oracle.velocity_x(sys, vac, tt, np.eye(n)[j]) for j in range(n)]
    return np.array(cols).T.real


def test_velocity_operator_is_antisymmetric_with_bond_weights():
    """h~x = [x, H]: real antisymmetric; sum_j (x_i-x_j)^2 = 1/2 per honeycomb site
    (bond x-offsets 0, +-a/2 from Listing 1) and 2 per square site."""
    for lat, expect in ((oracle.HONEYCOMB, 0.5), (oracle.SQUARE, 2.0)):
        sys = oracle.make_system(lattice=lat, Lx=5, Ly=4, t=1.0)
        n = oracle.norb(sys)
        hx = dense_vx(sys, np.zeros(n, np.uint8), 1.0)
        assert np.array_equal(hx, -hx.T)
        assert np.allclose((hx * hx).sum(axis=1), expect)


def test_exact_trace_2d_moments_match_bloch_velocity():
    """Clean honeycomb: mu_nm = (1/N) sum_k Tr[v(k) T_n(H(k)) v(k) T_m(H(k))] with the
    Bloch velocity v(k) = dH(k)/dk_x (v = -i h~ = i[H,x]); the offsets of the bonds to
    B(x+1,y-1) and B(x,y-1) are a1-a2 and -a2, whose x-components are +a/2 and -a/2."""
    Lx, Ly, M = 4, 3, 10
    sys = oracle.make_system(Lx=Lx, Ly=Ly, t=T_EV)
    lo, hi = oracle.bounds_auto(sys)
    dm = 0.5 * (hi - lo)
    tt = T_EV / dm
    n = oracle.norb(sys)
    mu = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128)) * n
    ref = np.zeros((M, M), np.complex128)
    for m1 in range(Lx):
        for m2 in range(Ly):
            k1, k2 = 2 * np.pi * m1 / Lx, 2 * np.pi * m2 / Ly
            p1, p2 = np.exp(1j * (k1 - k2)), np.exp(-1j * k2)
            f = tt * (1 + p1 + p2)
            df = tt * (0.5j * p1 - 0.5j * p2)  # d/dk_x with x in units of a
            Hk = np.array([[0, f], [np.conj(f), 0]])
            vk = np.array([[0, df], [np.conj(df), 0]])
            lam, U = np.linalg.eigh(Hk)
            Tn = cheb_T(M, lam)
            vv = U.conj().T @ vk @ U
            for a in range(2):
                for b in range(2):
                    ref += abs(vv[a, b]) ** 2 * np.outer(Tn[:, b], Tn[:, a])
    ref /= n
    assert np.max(np.abs(mu - ref)) < 1e-12
    assert np.max(np.abs(mu.imag)) < 1e-12
    assert np.max(np.abs(mu - mu.T)) < 1e-12
    assert abs(mu[0, 0].real - 0.5 * tt * tt) < 1e-14


def test_y_velocity_is_antisymmetric_with_bond_weights():
    """h~y = [y, H]: real antisymmetric; sum_j (y_i-y_j)^2 = a_cc^2 + 2 (a_cc/2)^2 = 1/2 per
    honeycomb site (a_cc = a/sqrt(3), orbital positions of the lattice set-up listing) and
    2 per square site; and sum_j (x_i-x_j)(y_i-y_j) = 0 (no preferred diagonal)."""
    for lat, expect in ((oracle.HONEYCOMB, 0.5), (oracle.SQUARE, 2.0)):
        sys = oracle.make_system(lattice=lat, Lx=5, Ly=4, t=1.0)
        n = oracle.norb(sys)
        zero = np.zeros(n, np.uint8)
        hy = np.array([oracle.velocity(sys, zero, 1.0, np.eye(n)[j], 1) for j in range(n)]).T.real
        hx = dense_vx(sys, zero, 1.0)
        assert np.array_equal(hy, -hy.T)
        assert np.allclose((hy * hy).sum(axis=1), expect)
        assert np.allclose((hx * hy).sum(axis=1), 0.0)


def bloch_2d_moments(Lx, Ly, M, tt, alpha, beta):
    """(1/N) sum_k Tr[v_alpha(k) T_n(H(k)) v_beta(k) T_m(H(k))] for the clean honeycomb
    lattice in the atomic gauge: H_AB(k) = t~ sum_d exp(i k.d) over the three bond vectors
    d = r_B - r_A = (0, a_cc), (a/2, -a_cc/2), (-a/2, -a_cc/2), v(k) = dH/dk (v = i[H, r])."""
    acc = 1.0 / np.sqrt(3.0)
    bonds = np.array([[0.0, acc], [0.5, -0.5 * acc], [-0.5, -0.5 * acc]])
    ref = np.zeros((M, M), np.complex128)
    for m1 in range(Lx):
        for m2 in range(Ly):
            k1, k2 = 2 * np.pi * m1 / Lx, 2 * np.pi * m2 / Ly  # k.a1, k.a2
            k = np.array([k1, (2.0 * k2 - k1) / np.sqrt(3.0)])
            ph = np.exp(1j * bonds @ k)
            f = tt * ph.sum()
            Hk = np.array([[0, f], [np.conj(f), 0]])
            vs = []
            for d in (alpha, beta):
                df = tt * np.sum(1j * bonds[:, d] * ph)
                vs.append(np.array([[0, df], [np.conj(df), 0]]))
            lam, U = np.linalg.eigh(Hk)
            Tn = cheb_T(M, lam)
            va, vb = (U.conj().T @ v @ U for v in vs)
            for a in range(2):
                for b in range(2):
                    ref += va[a, b] * vb[b, a] * np.outer(Tn[:, b], Tn[:, a])
    return ref / (2 * Lx * Ly)


@pytest.mark.parametrize("alpha,beta", [(0, 0), (1, 1), (0, 1), (1, 0)])
def test_exact_trace_2d_moments_match_bloch_velocity_all_directions(alpha, beta):
    """The four tensor components against the Bloch velocities dH/dk_x, dH/dk_y."""
    Lx, Ly, M = 4, 3, 10
    sys = oracle.make_system(Lx=Lx, Ly=Ly, t=T_EV)
    lo, hi = oracle.bounds_auto(sys)
    tt = T_EV / (0.5 * (hi - lo))
    n = oracle.norb(sys)
    mu = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128), alpha=alpha, beta=beta) * n
    ref = bloch_2d_moments(Lx, Ly, M, tt, alpha, beta)
    assert np.max(np.abs(mu - ref)) < 1e-12


def test_clean_honeycomb_response_is_isotropic():
    """On the clean L x L torus (a 120-degree rotation and the mirror x -> -x map it to
    itself) Tr[h T_n h T_m] is isotropic: mu^yy = mu^xx and mu^xy = mu^yx = 0."""
    sys = oracle.make_system(Lx=4, Ly=4, t=T_EV)
    n = oracle.norb(sys)
    eye = np.eye(n, dtype=np.complex128)
    mu = {(a, b): oracle.moments_2d(sys, 9, n, r0=eye, alpha=a, beta=b) * n for a in (0, 1) for b in (0, 1)}
    assert np.max(np.abs(mu[(1, 1)] - mu[(0, 0)])) < 1e-12
    assert np.max(np.abs(mu[(0, 1)])) < 1e-12 and np.max(np.abs(mu[(1, 0)])) < 1e-12
    assert np.max(np.abs(mu[(0, 0)])) > 1e-3


@pytest.mark.parametrize("alpha,beta", [(0, 0), (1, 1), (0, 1)])
def test_2d_moments_with_disorder_match_dense_diagonalisation(alpha, beta):
    sys = oracle.make_system(Lx=4, Ly=4, W=2.0, p_vac=0.1, seed=31)
    M = 12
    lo, hi = oracle.bounds_auto(sys)
    dm = 0.5 * (hi - lo)
    n = oracle.norb(sys)
    H, keep, vac = dense_h(sys)
    vel = []
    for d in (alpha, beta):
        h = np.array([oracle.velocity(sys, vac, sys.t / dm, np.eye(n)[j], d) for j in range(n)]).T.real
        vel.append(-1j * h[np.ix_(keep, keep)])
    lam, U = np.linalg.eigh(H)
    Tn = cheb_T(M, lam)
    va, vb = (U.conj().T @ v @ U for v in vel)
    ref = np.einsum("ab,ba,nb,ma->nm", va, vb, Tn, Tn) / len(keep)
    mu = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128), alpha=alpha, beta=beta) * n
    assert np.max(np.abs(mu - ref)) < 1e-12


def test_2d_stochastic_estimate_is_close():
    sys = oracle.make_system(Lx=16, Ly=16, W=1.0, seed=12)
    M = 8
    mu_st = oracle.moments_2d(sys, M, 4)
    n = oracle.norb(sys)
    # basis vectors: the vector average times n is the exact trace Tr[v T_n v T_m]/N
    mu_ex = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128)) * n
    scale = np.max(np.abs(mu_ex))
    assert np.max(np.abs(mu_st - mu_ex)) < 0.1 * scale


@pytest.mark.parametrize("lattice", [oracle.HONEYCOMB, oracle.SQUARE])
def test_light_cone_window_reproduces_full_replica(lattice):
    """T_n r at a site depends only on orbitals within n hops: the window replica equals
    the full-lattice replica bit for bit at sampled sites, corners included."""
    Lx, Ly = (40, 36) if lattice == oracle.HONEYCOMB else (45, 33)
    t = T_EV if lattice == oracle.HONEYCOMB else -1.0
    s = oracle.make_system(lattice=lattice, Lx=Lx, Ly=Ly, t=t, W=2.0, p_vac=0.03, seed=5,
                           delta=0.3 if lattice == oracle.HONEYCOMB else 0.0)
    M, R = 12, 2
    sorb = 2 if lattice == oracle.HONEYCOMB else 1
    for prec in (0, 1):
        _, full = oracle.replica_1d(s, M, R, prec, want_last=True)
        for (x0, y0) in ((0, 0), (Lx - 1, Ly - 1), (17, 5), (3, Ly - 2)):
            w = oracle.replica_window(s, M, R, prec, x0, y0)
            o = (y0 * Lx + x0) * sorb
            assert np.array_equal(w, full[:, :, o:o + sorb])


def test_cpgf_vectorised_matches_scalar_definition():
    eps = np.array([-0.8, -0.1, 0.3, 0.95, 1.2])
    for sigma in (+1, -1):
        G = oracle.cpgf_coeffs(20, eps, 0.03, sigma)
        for n in (0, 1, 7, 19):
            for k, e in enumerate(eps):
                assert abs(G[n, k] - oracle.cpgf_coeff(n, e, 0.03, sigma)) < 1e-13 * max(1, abs(G[n, k]))


def test_sigma_matches_eigenstate_kubo_bastin():
    """Kubo-Bastin sigma_xx at T = 0 in the eigenbasis of a tiny disordered lattice
    (Eq. cond 1st order): with G = Tr[h~ T h~ T]/N = -(1/N) sum_ab |v_ab|^2 ..., the
    reconstruction must equal
      sigma = +i (n_orb a^2/Omega_c)/w * (1/N) sum_ab |v_ab|^2 [ I1_ab + I2_ab ],
      I1_ab = int_{-1}^{eF} d_M(e - e_a) / (e + w - e_b + i eta) de,
      I2_ab = int_{-1}^{eF} d_M(e - e_b) / (e - w - e_a - i eta) de,
    where d_M is the M-term Chebyshev expansion of the delta function (the Delta_m series
    of Sec. 2a).  The reference uses the exact resolvent (eta > 0 makes the CPGF series
    converge exponentially) and brute-force Simpson quadrature in theta, so it checks the
    sign conventions of Gamma_nm, the Lambda_nm formula, the CPGF coefficients and the
    contraction independently of the oracle's Gauss-Legendre/Gamma route."""
    sys = oracle.make_system(Lx=4, Ly=3, t=T_EV, W=1.0, seed=3)
    lo, hi = oracle.bounds_auto(sys)
    dm = 0.5 * (hi - lo)
    n = oracle.norb(sys)
    M = 300
    mu = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128)) * n
    H, keep, vac = dense_h(sys)
    hx = dense_vx(sys, vac, sys.t / dm)
    lam, U = np.linalg.eigh(H)
    P = np.abs(U.conj().T @ (-1j * hx) @ U) ** 2
    E_F, eta = 0.3, 0.6  # eV
    eF, et = E_F / dm, eta / dm
    thF = np.arccos(eF)
    K = 20001
    th = np.linspace(thF, np.pi, K)
    wk = np.full(K, 2.0)
    wk[1:-1:2] = 4.0
    wk[0] = wk[-1] = 1.0
    wk *= (th[1] - th[0]) / 3.0
    e = np.cos(th)
    Tl = cheb_T(M, lam)                            # [m][a]
    cm = np.where(np.arange(M) == 0, 0.5, 1.0)
    Dk = (2.0 / np.pi) * np.cos(np.arange(M)[:, None] * th[None, :])  # Delta_m de / d theta
    dM = (Tl * cm[:, None]).T @ Dk                 # [a][k] = d_M(e_k - e_a) de/dtheta
    omegas = np.array([0.5, 1.5, 3.0, 6.0])
    sig = oracle.sigma_xx(mu, omegas, lo, hi, E_F, eta, oracle.HONEYCOMB, kernel=None, n_quad=2000)
    c = oracle.unit_cell_factor(oracle.HONEYCOMB)
    for i, om in enumerate(omegas):
        w = om / dm
        G1 = 1.0 / (e[None, :] + w - lam[:, None] + 1j * et)     # [b][k]
        G2 = 1.0 / (e[None, :] - w - lam[:, None] - 1j * et)     # [a][k]
        S1 = np.sum(wk[None, :] * dM * (P @ G1))                 # sum_a d_M(e-e_a) sum_b P_ab G1
        S2 = np.sum(wk[None, :] * dM * (P.T @ G2))               # sum_b d_M(e-e_b) sum_a P_ab G2
        ref = 1j * c / w * (S1 + S2) / n
        assert abs(sig[i] - ref) < 1e-7 * abs(ref), (om, sig[i], ref)
        assert sig[i].real > 0  # absorption


def test_dc_conductivity_matches_eigenstate_kubo_greenwood():
    """Kubo-Greenwood at T = 0 in the eigenbasis of a tiny disordered lattice:
      sigma(E) = pi (n_orb a^2/Omega_c) (1/N) sum_ab |v_ab|^2 d_M(e - e_a) d_M(e - e_b),
    with d_M the M-term kernel-damped Chebyshev delta function (Sec. 2a) evaluated from the
    exact eigenvalues and velocity matrix elements, against the oracle's contraction of the
    exact-trace 2D moments; positive (Jackson deltas are positive), and symmetric in E for
    the clean bipartite honeycomb."""
    for W, sym in ((1.5, False), (0.0, True)):
        sys = oracle.make_system(Lx=4, Ly=3, t=T_EV, W=W, seed=8)
        lo, hi = oracle.bounds_auto(sys)
        dm = 0.5 * (hi - lo)
        n = oracle.norb(sys)
        M = 120
        mu = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128)) * n
        H, keep, vac = dense_h(sys)
        hx = dense_vx(sys, vac, sys.t / dm)
        lam, U = np.linalg.eigh(H)
        P = np.abs(U.conj().T @ (-1j * hx) @ U) ** 2
        E = np.linspace(-0.8 * hi, 0.8 * hi, 41)
        sig = oracle.sigma_dc(mu, E, lo, hi, oracle.HONEYCOMB)
        g = oracle.kernel_jackson(M)
        w = np.where(np.arange(M) == 0, 1.0, 2.0) * g
        Tl = cheb_T(M, lam)                                          # [n][a]
        for k, Ek in enumerate(E):
            e = Ek / dm
            d = (w * cheb_T(M, np.array([e]))[:, 0]) @ Tl / (np.pi * math.sqrt(1 - e * e))  # [a]
            ref = np.pi * oracle.unit_cell_factor(oracle.HONEYCOMB) * (d @ P @ d) / n
            assert abs(sig[k] - ref) <= 1e-10 * max(1.0, abs(ref)), (W, Ek, sig[k], ref)
        assert np.all(sig >= -1e-12)
        if sym:
            assert np.max(np.abs(sig - sig[::-1])) < 1e-10
    assert np.all(oracle.sigma_dc(mu, np.array([lo - 1.0, hi + 1.0]), lo, hi, oracle.HONEYCOMB) == 0.0)


def test_dc_conductivity_is_the_zero_frequency_limit_of_the_optical_one():
    """The DC formula's prefactor against the independently pinned optical conductivity
    (eigenstate Kubo-Bastin and the graphene plateau): on a disordered lattice, Re sigma(w)
    of the Kubo-Bastin route with Jackson damping tends to sigma_DC as w and eta shrink
    (2-5 % apart at w = 0.02 eV, eta = 0.005 eV where states exist at E_F)."""
    sys = oracle.make_system(Lx=12, Ly=12, t=T_EV, W=3.0, seed=8)
    lo, hi = oracle.bounds_auto(sys)
    n = oracle.norb(sys)
    M = 256
    mu = oracle.moments_2d(sys, M, n, r0=np.eye(n, dtype=np.complex128)) * n
    for E_F in (-1.5, 2.0):
        dc = oracle.sigma_dc(mu, np.array([E_F]), lo, hi, oracle.HONEYCOMB)[0]
        opt = oracle.sigma_xx(mu, np.array([0.02]), lo, hi, E_F, 0.005, oracle.HONEYCOMB)[0].real
        assert dc > 0.1 and abs(opt / dc - 1.0) < 0.1, (E_F, dc, opt)


def dense_v(sys, direction):
    """v~ = -i h~ (h~ = [r_dir, H~]) of the oracle as a dense matrix, with its field phases."""
    lo, hi = oracle.bounds_auto(sys)
    n = oracle.norb(sys)
    _, vac = oracle.disorder(sys)
    eye = np.eye(n, dtype=np.complex128)
    cols = [oracle.velocity(sys, vac, sys.t / (0.5 * (hi - lo)), eye[:, j], direction) for j in range(n)]
    return -1j * np.array(cols).T


def tknn_sigma_xy(H, vx, vy, eF, ucf):
    """T = 0 Kubo formula in the eigenbasis (the textbook TKNN sum),
    sigma_xy = -2 (n_orb a^2/Omega_c)/N sum_{a occupied, b empty} Im[(vx)_ab (vy)_ba] / (e_a - e_b)^2,
    in units of e^2/hbar (rescaled energies and velocities: the ratio is scale free)."""
    lam, U = np.linalg.eigh(H)
    X, Y = U.conj().T @ vx @ U, U.conj().T @ vy @ U
    a, b = np.where(lam < eF)[0], np.where(lam >= eF)[0]
    d = lam[a][:, None] - lam[b][None, :]
    return -2.0 * ucf / H.shape[0] * float(np.sum(np.imag(X[np.ix_(a, b)] * Y[np.ix_(b, a)].T) / d ** 2))


@pytest.mark.parametrize("lattice,flux", [(oracle.HONEYCOMB, 0.25), (oracle.SQUARE, 0.375)])
def test_velocity_in_a_field_is_the_position_commutator(lattice, flux):
    """v = i[H, r]/hbar holds with the Peierls phases: every element of h~ = [r, H~] is the
    minimum-image bond vector r_i - r_j times the element of the oracle's rescaled H~ (taken
    from its recursion, with disorder and vacancies), so the velocity carries the same
    phases as the Hamiltonian; built from the orbital positions, not the bond tables."""
    t = -1.0 if lattice == oracle.SQUARE else T_EV
    sys = oracle.make_system(lattice=lattice, Lx=6, Ly=8, t=t, W=1.0, p_vac=0.05, seed=4, flux=flux)
    H = dense_from_operator(sys)
    P = oracle.orbital_positions(sys)
    if lattice == oracle.HONEYCOMB:
        T1, T2 = np.array([sys.Lx, 0.0]), np.array([0.5 * sys.Ly, 0.5 * math.sqrt(3.0) * sys.Ly])
    else:
        T1, T2 = np.array([sys.Lx, 0.0]), np.array([0.0, sys.Ly])
    d0 = P[:, None, :] - P[None, :, :]
    best = d0.copy()
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            c = d0 + i * T1 + j * T2
            shorter = np.sum(c * c, -1) < np.sum(best * best, -1)
            best[shorter] = c[shorter]
    for direction in (0, 1):
        h = 1j * dense_v(sys, direction)
        assert np.max(np.abs(h - best[..., direction] * H)) < 1e-14
        assert np.max(np.abs(h + h.conj().T)) < 1e-15


def bastin_eigenbasis(H, vx, vy, eF, eta, M, ucf, kT=0.0, dm=1.0, K=20001):
    """sigma_xy of the Kubo-Bastin formula with the exact broadened resolvent derivative
    -1/(e +- i eta - e_a)^2 and the M-term Chebyshev delta function (no kernel), in the
    eigenbasis; Simpson quadrature in theta over the Fermi sea (kT > 0: the whole band
    with Fermi weights, energies in units of dm)."""
    n = H.shape[0]
    lam, U = np.linalg.eigh(H)
    X = (U.conj().T @ vx @ U) * (U.conj().T @ vy @ U).T      # X_ab = (vx)_ab (vy)_ba
    thF = np.arccos(eF) if kT <= 0.0 else 0.0
    th = np.linspace(thF, np.pi, K)
    wk = np.full(K, 2.0)
    wk[1:-1:2] = 4.0
    wk[0] = wk[-1] = 1.0
    wk *= (th[1] - th[0]) / 3.0
    e = np.cos(th)
    if kT > 0.0:
        wk = wk / (1.0 + np.exp((e - eF) * dm / kT))
    cm = np.where(np.arange(M) == 0, 1.0, 2.0) / np.pi
    Dk = (cheb_T(M, lam) * cm[:, None]).T @ np.cos(np.arange(M)[:, None] * th[None, :]) * wk[None, :]
    GR = -1.0 / (e[None, :] + 1j * eta - lam[:, None]) ** 2
    GA = -1.0 / (e[None, :] - 1j * eta - lam[:, None]) ** 2
    T1 = np.sum(GR * (X @ Dk))
    T2 = np.sum(Dk * (X @ GA))
    return float(np.real(1j * ucf / n * (T1 - T2)))


def test_bastin_dc_matches_eigenstate_formula():
    """DC Kubo-Bastin (sigma_xy and sigma_xx, T = 0 and kT > 0) of a tiny disordered
    honeycomb in a field against the eigenbasis evaluation with exact resolvent
    derivatives: the CPGF derivative coefficients, the Delta_n series, the order of the
    velocities in mu_nm and the Fermi-sea limits are all checked at once (the broadening
    makes the CPGF series converge exponentially: M = 400 terms are exact to about 1e-11)."""
    sys = oracle.make_system(Lx=4, Ly=4, t=T_EV, W=1.0, seed=3, flux=0.5)
    lo, hi = oracle.bounds_auto(sys)
    dm = 0.5 * (hi - lo)
    n = oracle.norb(sys)
    M, eta = 400, 0.6
    H = dense_from_operator(sys)
    vx, vy = dense_v(sys, 0), dense_v(sys, 1)
    ucf = oracle.unit_cell_factor(oracle.HONEYCOMB)
    eye = np.eye(n, dtype=np.complex128)
    for (a, b), (A, B) in (((0, 1), (vx, vy)), ((0, 0), (vx, vx))):
        mu = oracle.moments_2d(sys, M, n, r0=eye, alpha=a, beta=b) * n
        for E_F, kT in ((-2.0, 0.0), (0.7, 0.0), (0.7, 0.3)):
            got = oracle.sigma_dc_bastin(mu, [E_F], lo, hi, eta, oracle.HONEYCOMB, kernel=None,
                                         n_quad=1000, kT=kT)[0]
            ref = bastin_eigenbasis(H, A, B, E_F / dm, eta / dm, M, ucf, kT=kT, dm=dm)
            assert abs(got - ref) <= 2e-10, ((a, b), E_F, kT, got, ref)
    assert oracle.sigma_dc_bastin(mu, [lo - 1.0], lo, hi, eta, oracle.HONEYCOMB)[0] == 0.0


def test_quantum_hall_plateau():
    """Graphene in a field with E_F in the gap above the zero Landau level: the textbook
    Kubo (TKNN) sum on the oracle's dense H~ and field velocities gives sigma_xy = -e^2/h
    per spin (one filled level of the Dirac sequence (2n + 1) e^2/h per spin, valleys
    summed; 1/(2 pi) in units of e^2/hbar) to 0.5 % on a 16 x 16 torus, and +e^2/h
    mirrored below it; every other gap of the spectrum carries the Chern number of the
    Diophantine equation; the Kubo-Bastin reconstruction from the exact-trace moments of an
    8 x 16 torus converges to that torus's TKNN value as M grows (Jackson kernel, small
    eta), and sigma_xx vanishes in the gap."""
    ucf = oracle.unit_cell_factor(oracle.HONEYCOMB)
    big = oracle.make_system(Lx=16, Ly=16, t=T_EV, flux=0.125)
    lo, hi = oracle.bounds_auto(big)
    dm = 0.5 * (hi - lo)
    Hb, vxb, vyb = dense_from_operator(big), dense_v(big, 0), dense_v(big, 1)
    for E_F, sign in ((1.35, -1.0), (-1.35, 1.0)):   # the gap spans 0.26 - 2.44 eV
        q = tknn_sigma_xy(Hb, vxb, vyb, E_F / dm, ucf) * 2 * math.pi
        assert abs(q - sign) < 5e-3, (E_F, q)
    # every gap of the flux-1/8 spectrum: with r of the 2q = 16 subbands per cell filled, the
    # Diophantine equation r = q s + p t (p/q = 1/8, |t| <= q/2) fixes the Chern number t,
    # and sigma_xy = -t e^2/h per spin (TKNN 1982)
    lam = np.sort(np.linalg.eigvalsh(Hb))
    n_cells = 16 * 16
    for r in (1, 2, 7, 9, 14, 15):
        k = r * n_cells // 8  # states below the gap: r subbands of n_cells / q states
        assert lam[k] - lam[k - 1] > 0.05, r  # a gap
        t_r = next(t for t in range(-4, 5) if (r - t) % 8 == 0)
        q = tknn_sigma_xy(Hb, vxb, vyb, 0.5 * (lam[k] + lam[k - 1]), ucf) * 2 * math.pi
        assert abs(q + t_r) < 1e-2, (r, q, t_r)
    sys = oracle.make_system(Lx=8, Ly=16, t=T_EV, flux=0.125)
    n = oracle.norb(sys)
    H, vx, vy = dense_from_operator(sys), dense_v(sys, 0), dense_v(sys, 1)
    ref = tknn_sigma_xy(H, vx, vy, 1.35 / dm, ucf)
    eye = np.eye(n, dtype=np.complex128)
    err = []
    for M in (96, 192):
        mu = oracle.moments_2d(sys, M, n, r0=eye, alpha=0, beta=1) * n
        err.append(abs(oracle.sigma_dc_bastin(mu, [1.35], lo, hi, 0.01, oracle.HONEYCOMB)[0] / ref - 1))
    assert err[1] < 0.03 and err[1] < 0.7 * err[0], err
    mu = oracle.moments_2d(sys, 192, n, r0=eye) * n
    sxx = oracle.sigma_dc_bastin(mu, [1.35], lo, hi, 0.01, oracle.HONEYCOMB)[0]
    assert abs(sxx) < 0.02 * abs(ref), sxx


def test_mlp_gradient_matches_finite_differences():
    """The reference MLP's analytic gradient against central differences in FP64 (small
    widths; points kept away from the ReLU and |.| kinks)."""
    from oracle import mlp
    ni, nh, no = 7, 9, 5
    p = mlp.init_params(3, ni, nh, no) + 0.01
    g = np.random.Generator(np.random.PCG64(4))
    X = g.standard_normal((6, ni))
    T = g.standard_normal((6, no)) * 3.0
    an = mlp.grad(p, X, T, ni, nh, no)
    h = 1e-6
    idx = g.choice(p.size, 60, replace=False)
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(p + e, X, T, ni, nh, no) - mlp.loss(p - e, X, T, ni, nh, no)) / (2 * h)
        assert abs(fd - an[k]) <= 1e-6 * max(1.0, abs(an[k])), k


def test_mlp_adamw_first_step_is_sign_step():
    """First AdamW step with bias correction moves each parameter by lr*(sign(g) + wd*p)
    (up to eps): the definition's fixed point."""
    from oracle import mlp
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 2.0])
    p1, m, v = mlp.adamw_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.1, eps=1e-12)
    assert np.allclose(p1, p - 0.01 * (np.sign(g) + 0.1 * p), atol=1e-10)


def test_mlp_adamw_constant_gradient_moves_by_lr_every_step():
    """A constant gradient g with no weight decay: m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2
    exactly, so both bias corrections recover g and g^2 and every step moves each parameter
    by lr * sign(g) (up to eps) -- at t = 1, 2, 3, 10 and 100.  Correcting only m, or with
    the wrong power of b2, leaves a factor sqrt(1 - b2^t) that this catches."""
    from oracle import mlp
    g = np.array([0.7, -3e-3, 2.0, -40.0])
    p = np.array([1.0, -2.0, 0.5, 0.0])
    m, v = np.zeros(4), np.zeros(4)
    lr = 0.01
    for t in range(1, 101):
        p_new, m, v = mlp.adamw_step(p, g, m, v, t, lr=lr, wd=0.0, eps=1e-14)
        if t in (1, 2, 3, 10, 100):
            assert np.allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
            assert np.allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)
            assert np.allclose(p_new - p, -lr * np.sign(g), rtol=1e-9, atol=0)
        p = p_new


def test_mlp_adamw_two_steps_by_hand():
    """g = 1 then g = 0 (no weight decay), worked by hand: after step 2 the bias-corrected
    moments are m^ = b1 (1 - b1) / (1 - b1^2) = b1 / (1 + b1) = 9/19 and
    v^ = b2 (1 - b2) / (1 - b2^2) = b2 / (1 + b2) = 999/1999, so the second step moves the
    parameter by lr (9/19) / sqrt(999/1999)."""
    from oracle import mlp
    lr = 0.1
    p1, m, v = mlp.adamw_step(np.array([0.0]), np.array([1.0]), np.zeros(1), np.zeros(1), 1, lr=lr, wd=0.0,
                              eps=0.0)
    assert p1[0] == pytest.approx(-lr, rel=1e-15)
    p2, m, v = mlp.adamw_step(p1, np.array([0.0]), m, v, 2, lr=lr, wd=0.0, eps=0.0)
    assert m[0] == pytest.approx(0.9 * 0.1, rel=1e-14)
    assert v[0] == pytest.approx(0.999 * 0.001, rel=1e-14)
    assert p2[0] - p1[0] == pytest.approx(-lr * (9.0 / 19.0) / math.sqrt(999.0 / 1999.0), rel=1e-12)


def test_mlp_adamw_weight_decay_is_decoupled():
    """With a zero gradient the moments stay zero and only the decoupled decay acts:
    p -> p (1 - lr wd).  Decay folded into the gradient (L2 regularisation through Adam)
    would instead move every parameter by lr sign(p)."""
    from oracle import mlp
    p = np.array([1.0, -2.0, 0.5])
    p1, m, v = mlp.adamw_step(p, np.zeros(3), np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.1)
    assert np.all(m == 0) and np.all(v == 0)
    assert np.allclose(p1, p * (1 - 0.01 * 0.1), rtol=1e-15)


def test_mlp_cosine_schedule_closed_form():
    """The learning rate of step t of T (t = 1..T) falls from lr as lr (1 + cos(pi (t-1)/T))/2:
    lr at t = 1, lr/2 half way (t = T/2 + 1), lr (2 + sqrt2)/4 a quarter of the way, and it
    decreases strictly towards 0 (reached one step after the last)."""
    from oracle import mlp
    T, lr = 40, 3e-3
    assert mlp.cosine_lr(1, T, lr) == lr
    assert mlp.cosine_lr(T // 2 + 1, T, lr) == pytest.approx(lr / 2, rel=1e-14)
    assert mlp.cosine_lr(T // 4 + 1, T, lr) == pytest.approx(lr * (2 + math.sqrt(2)) / 4, rel=1e-14)
    seq = [mlp.cosine_lr(t, T, lr) for t in range(1, T + 2)]
    assert all(a > b for a, b in zip(seq, seq[1:]))
    assert seq[-1] == pytest.approx(0.0, abs=1e-18)


def test_bf16_rounding_ties_to_even_and_matches_torch():
    """round_bf16: 8 significant bits, ties to even (1 + 2^-8 -> 1, 1 + 3*2^-8 -> 1 + 2^-6),
    and the same values as torch's float32 -> bfloat16 conversion on random inputs."""
    from oracle import mlp
    assert mlp.round_bf16(1.0 + 2.0**-8) == 1.0
    assert mlp.round_bf16(1.0 + 3 * 2.0**-8) == 1.0 + 2.0**-6
    assert mlp.round_bf16(1.0 + 2.0**-8 + 2.0**-20) == 1.0 + 2.0**-7
    assert mlp.round_bf16(-3.0) == -3.0
    torch = pytest.importorskip("torch")
    x = np.random.Generator(np.random.PCG64(12)).standard_normal(4096).astype(np.float32) * 10.0
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.round_bf16(x), ref)


def test_mlp_activation_rounding_moves_only_the_stored_values():
    """With act_round the forward pass equals the plain one evaluated layer by layer on the
    rounded activations, and the masks follow the stored (rounded) activations."""
    from oracle import mlp
    ni, nh, no = 6, 10, 4
    p = mlp.init_params(5, ni, nh, no) + 0.003
    X = np.random.Generator(np.random.PCG64(6)).standard_normal((5, ni))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, ni, nh, no)
    H1 = mlp.round_bf16(np.maximum(X @ W1.T + b1, 0))
    H2 = mlp.round_bf16(np.maximum(H1 @ W2.T + b2, 0))
    Y, _ = mlp.forward(p, X, ni, nh, no, act_round=mlp.round_bf16)
    assert np.array_equal(Y, H2 @ W3.T + b3)
    Yp, _ = mlp.forward(p, X, ni, nh, no)
    assert 0 < np.max(np.abs(Y - Yp)) <= 1e-2 * np.max(np.abs(Yp))


@pytest.mark.parametrize("alpha,beta", [(0, 0), (0, 1)])
def test_moments_2d_panels_equal_the_triple_loop(alpha, beta):
    """The panel routine (rows and columns of mu_nm from the streamed recursion, for
    lattices whose families do not fit in memory) gives the same numbers as the plain
    triple loop over stored families, which the exact-diagonalisation and Bloch-velocity
    pins fix; vacancies, several vectors, rows and columns at both ends."""
    s = oracle.make_system(lattice=oracle.HONEYCOMB, Lx=11, Ly=9, t=T_EV, W=1.0, p_vac=0.03, seed=5)
    M = 37
    full = oracle.moments_2d(s, M, 3, alpha=alpha, beta=beta)
    rows, cols = [0, 1, 17, 36], [0, 5, 35, 36]
    pr, pc = oracle.moments_2d_panels(s, M, 3, rows, cols, alpha=alpha, beta=beta)
    scale = np.max(np.abs(full))
    assert np.max(np.abs(pr - full[rows, :])) <= 1e-13 * scale
    assert np.max(np.abs(pc - full[:, cols])) <= 1e-13 * scale


def test_mlp_delta_rounding_moves_only_the_stored_deltas():
    """With delta_round the gradient equals the chain rule written out layer by layer on the
    rounded deltas (weight gradients = stored deltas times stored activations), and it moves
    the gradient by no more than the rounding of those deltas."""
    from oracle import mlp
    ni, nh, no = 6, 10, 4
    p = mlp.init_params(7, ni, nh, no) + 0.003
    g = np.random.Generator(np.random.PCG64(8))
    X = g.standard_normal((5, ni))
    T = g.standard_normal((5, no)) * 4.0
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, ni, nh, no)
    r = mlp.round_bf16
    H1 = r(np.maximum(X @ W1.T + b1, 0))
    H2 = r(np.maximum(H1 @ W2.T + b2, 0))
    Y = H2 @ W3.T + b3
    dY = r(np.sign(Y - T) / Y.size)
    dZ2 = r((dY @ W3) * (H2 > 0))
    dZ1 = r((dZ2 @ W2) * (H1 > 0))
    want = np.concatenate([a.ravel() for a in (dZ1.T @ X, dZ1.sum(0), dZ2.T @ H1, dZ2.sum(0), dY.T @ H2, dY.sum(0))])
    got = mlp.grad(p, X, T, ni, nh, no, act_round=r, delta_round=r)
    assert np.array_equal(got, want)
    plain = mlp.grad(p, X, T, ni, nh, no, act_round=r)
    assert 0 < np.max(np.abs(got - plain)) <= 1e-2 * np.max(np.abs(plain))


def test_mlp_prior_closed_forms():
    """The residual prior (Jackson reconstruction on the midpoint grid): mu = (1, 0, ...)
    gives 1/(pi a sqrt(1 - eps^2)) exactly (g_0 = 1); moments of a point spectrum
    mu_k = T_k(x0) give a broadened peak at x0 whose midpoint-rule weight is 1."""
    from oracle import mlp
    e_min, e_max = -3.0, 5.0
    a = 0.5 * (e_max - e_min)
    eps = mlp.midpoint_eps(256)
    mu = np.zeros(64)
    mu[0] = 1.0
    rho = mlp.prior(mu, e_min, e_max, n_out=256)[0]
    assert np.allclose(rho, 1.0 / (np.pi * a * np.sqrt(1.0 - eps**2)), rtol=1e-13, atol=0)
    x0 = 0.3
    mu = np.cos(np.arange(64) * np.arccos(x0))
    rho = mlp.prior(mu, e_min, e_max, n_out=1024)[0]
    assert abs(np.sum(rho) * a * 2.0 / 1024 - 1.0) < 1e-3
    assert abs(mlp.midpoint_eps(1024)[np.argmax(rho)] - x0) < 4.0 / 1024


def test_green_function_matches_exact_resolvent_trace():
    """G(E + i eta) from exact-trace moments of a small disordered lattice equals the
    resolvent trace (1/N) sum_k 1/(E - E_k + i eta) of its eigenvalues once the CPGF
    series has converged (M >> de_minus / eta); its -Im/pi integrates to ~1."""
    sys_ = oracle.make_system(lattice=oracle.HONEYCOMB, Lx=4, Ly=3, t=-2.7, W=2.0, p_vac=0.1, seed=21)
    lo, hi = oracle.bounds_auto(sys_)
    M = 3000
    mu = exact_trace_moments(sys_, M).real
    H, keep, vac = dense_h(sys_)
    Ek = np.linalg.eigvalsh(H) * 0.5 * (hi - lo) + 0.5 * (hi + lo)  # back to eV
    eta = 0.15
    E = np.linspace(lo * 0.95, hi * 0.95, 41)
    G = oracle.green(mu, E, lo, hi, eta)
    ref = np.array([np.mean(1.0 / (e - Ek + 1j * eta)) for e in E])
    assert np.max(np.abs(G - ref)) < 1e-8 * np.max(np.abs(ref))
    Ef = np.linspace(lo, hi, 20001)
    rho = -oracle.green(mu, Ef, lo, hi, eta).imag / np.pi
    assert abs(np.trapezoid(rho, Ef) - 1.0) < 0.05  # Lorentzian tails beyond the window


def test_real_random_vectors_are_white_noise_and_unbiased():
    """Real start vectors (Sec. 2c allows real white noise): entries +-1 off the
    vacancies, balanced, uncorrelated between vectors; averaged over many vectors the
    moments converge to the exact trace (real symmetric H~), within the STE error."""
    s = oracle.make_system(lattice=oracle.HONEYCOMB, Lx=6, Ly=5, t=T_EV, W=2.0, p_vac=0.1, seed=41)
    _, vac = oracle.disorder(s)
    R = 4000
    xi = oracle.random_real(s, R)
    keep = vac == 0
    assert np.all(xi.imag == 0) and np.all(xi[:, ~keep] == 0)
    assert np.all(np.abs(xi[:, keep].real) == 1.0)
    x = xi[:, keep].real
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    c = (x[:-1] * x[1:]).mean()  # neighbouring vectors uncorrelated
    assert abs(c) < 5 / np.sqrt(x.size)
    # the same draw decides the sign and the phase: sign = +1 exactly when phase < pi
    ph = oracle.random_phase(s, 8)
    xr = oracle.random_real(s, 8)
    ang = np.mod(np.angle(ph[:, keep]), 2 * np.pi)
    assert np.array_equal(xr[:, keep].real > 0, ang < np.pi)
    M = 12
    ex = exact_trace_moments(s, M).real
    mu = oracle.moments_1d(s, M, 400, r0=oracle.random_real(s, 400)).real
    err = np.abs(mu.mean(0) - ex)
    sd = mu.std(0) / np.sqrt(mu.shape[0])
    assert np.all(err <= 5 * sd + 1e-12)


def test_spectral_function_moments_match_bloch_bands():
    """k-resolved moments (1/N)<k|T_n(H~)|k> of the clean honeycomb lattice with the
    plane-wave start vector of the spectral-function section: for k on the torus grid,
    |k> = sum_a w_a |k, a> decomposes into the two Bloch bands, so the moments equal
    sum_b |<psi_b(k)|w>|^2 T_n(eps_b(k)) / SORB with the 2x2 Bloch Hamiltonian in the
    atomic gauge (bond vectors of the lattice set-up listing); with random orbital
    weights averaged (<w_a* w_b> = delta_ab) every band gets weight 1/2."""
    Lx, Ly, M = 6, 5, 14
    s = oracle.make_system(Lx=Lx, Ly=Ly, t=T_EV)
    lo, hi = oracle.bounds_auto(s)
    tt = T_EV / (0.5 * (hi - lo))
    n = oracle.norb(s)
    acc = 1.0 / np.sqrt(3.0)
    bonds = np.array([[0.0, acc], [0.5, -0.5 * acc], [-0.5, -0.5 * acc]])
    for m1, m2 in ((0, 0), (1, 2), (3, 4), (5, 1)):
        k1, k2 = 2 * np.pi * m1 / Lx, 2 * np.pi * m2 / Ly
        k = np.array([k1, (2.0 * k2 - k1) / np.sqrt(3.0)])
        f = tt * np.exp(1j * bonds @ k).sum()
        lam, U = np.linalg.eigh(np.array([[0, f], [np.conj(f), 0]]))
        for w in (np.array([1.0, 1.0]), np.array([0.3 + 0.4j, -1.1])):
            v = oracle.bloch_vector(s, k, w)
            mu = oracle.moments_1d(s, M, 1, r0=v[None, :])[0] * (n / np.vdot(v, v).real)
            ov = np.abs(U.conj().T @ w) ** 2 / np.sum(np.abs(w) ** 2)
            ref = (ov[None, :] * cheb_T(M, lam)).sum(1)
            assert np.max(np.abs(mu - ref)) < 1e-12, (m1, m2, w)


@pytest.mark.parametrize("lattice,flux,oy", [(oracle.HONEYCOMB, 0.25, 0), (oracle.SQUARE, 0.13, 1)])
def test_wave_packet_propagation_in_a_field_matches_dense_exponential(lattice, flux, oy):
    """The propagator with the Peierls Hamiltonian (complex H, pinned by the loop traces and
    the position commutator) against scipy's matrix exponential of the same dense H~, on a
    torus and on a strip open in y with an incommensurate flux; the norm is conserved."""
    from scipy.linalg import expm
    t = -1.0 if lattice == oracle.SQUARE else T_EV
    s = oracle.make_system(lattice=lattice, Lx=6, Ly=8, t=t, W=1.0, seed=45, flux=flux, open_y=oy)
    lo, hi = oracle.bounds_auto(s)
    H = dense_from_operator(s)
    n = H.shape[0]
    Hphys = H * 0.5 * (hi - lo) + np.eye(n) * 0.5 * (hi + lo)
    g = np.random.Generator(np.random.PCG64(6))
    psi0 = g.standard_normal(n) + 1j * g.standard_normal(n)
    psi0 /= np.linalg.norm(psi0)
    dt, steps, M = 0.6, 3, 60
    out = oracle.propagate(s, psi0, dt, steps, M)
    U = expm(-1j * Hphys * dt)
    ref = psi0
    for k in range(steps):
        ref = U @ ref
        assert np.max(np.abs(out[k] - ref)) < 1e-11
        assert abs(np.linalg.norm(out[k]) - 1.0) < 1e-11


def test_wave_packet_propagation_matches_dense_exponential():
    """Time evolution by the Chebyshev series of the wave-packet section against the dense
    matrix exponential exp(-i H t) of a small disordered lattice (hbar = 1, t in hbar/eV),
    several steps; the norm is conserved.  A (-1)^n coefficient (the printed form) fails."""
    from scipy.linalg import expm
    s = oracle.make_system(lattice=oracle.HONEYCOMB, Lx=5, Ly=4, t=T_EV, W=1.5, p_vac=0.1, seed=44)
    lo, hi = oracle.bounds_auto(s)
    H, keep, vac = dense_h(s)
    Hphys = H * 0.5 * (hi - lo) + np.eye(len(keep)) * 0.5 * (hi + lo)
    n = oracle.norb(s)
    g = np.random.Generator(np.random.PCG64(5))
    psi0 = np.zeros(n, np.complex128)
    psi0[keep] = g.standard_normal(len(keep)) + 1j * g.standard_normal(len(keep))
    psi0 /= np.linalg.norm(psi0)
    dt, steps, M = 0.7, 4, 60
    out = oracle.propagate(s, psi0, dt, steps, M)
    U = expm(-1j * Hphys * dt)
    ref = psi0[keep]
    for k in range(steps):
        ref = U @ ref
        assert np.max(np.abs(out[k][keep] - ref)) < 1e-11
        assert abs(np.linalg.norm(out[k]) - 1.0) < 1e-11
        assert np.all(out[k][vac != 0] == 0)
    from scipy.special import jv
    nn = np.arange(M)
    printed = np.exp(-1j * 0.5 * (hi + lo) * dt) * np.where(nn == 0, 1.0, 2.0) * (-1.0) ** nn * jv(nn, 0.5 * (hi - lo) * dt)
    bad = oracle.chebyshev_sum(s, printed, psi0)
    assert np.max(np.abs(bad[keep] - U @ psi0[keep])) > 1e-3


@pytest.mark.parametrize("lattice", [oracle.HONEYCOMB, oracle.SQUARE])
def test_complex_moments_split_into_real_and_imaginary_recursions(lattice):
    """With no field H~ is real and symmetric, so for r_0 = a + i b the moment
    <r_0|T_n(H~)|r_0> equals <a|T_n a> + <b|T_n b> and its imaginary part vanishes: the
    reading behind the on-chip cluster sweep (one real recursion per part) and the FP64
    sweeps (imaginary part not formed), checked on the plain FP64 definition."""
    s = oracle.make_system(lattice=lattice, Lx=7, Ly=5, t=-2.7 if lattice == oracle.HONEYCOMB else -1.0,
                           W=2.0, delta=0.3 if lattice == oracle.HONEYCOMB else 0.0, p_vac=0.1, seed=13)
    n = oracle.norb(s)
    _, vac = oracle.disorder(s)
    rng = np.random.default_rng(4)
    z = (rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))) * (vac == 0)
    M = 40
    mu = oracle.moments_1d(s, M, 3, r0=z)
    mu_a = oracle.moments_1d(s, M, 3, r0=z.real.astype(complex))
    mu_b = oracle.moments_1d(s, M, 3, r0=z.imag.astype(complex))
    scale = np.max(np.abs(mu))
    assert np.max(np.abs(mu.imag)) <= 1e-13 * scale
    assert np.max(np.abs(mu.real - (mu_a.real + mu_b.real))) <= 1e-13 * scale
    # and in a field (complex Hermitian H~) the split fails while Im still vanishes
    f = oracle.make_system(lattice=lattice, Lx=7, Ly=6, t=-2.7 if lattice == oracle.HONEYCOMB else -1.0,
                           W=2.0, p_vac=0.0, seed=13, flux=2 / 6 if lattice == oracle.HONEYCOMB else 1 / 6)
    nf = oracle.norb(f)
    zf = rng.standard_normal((2, nf)) + 1j * rng.standard_normal((2, nf))
    mf = oracle.moments_1d(f, M, 2, r0=zf)
    mfa = oracle.moments_1d(f, M, 2, r0=zf.real.astype(complex))
    mfb = oracle.moments_1d(f, M, 2, r0=zf.imag.astype(complex))
    sf = np.max(np.abs(mf))
    assert np.max(np.abs(mf.imag)) <= 1e-13 * sf
    assert np.max(np.abs(mf.real - (mfa.real + mfb.real))) > 1e-6 * sf
