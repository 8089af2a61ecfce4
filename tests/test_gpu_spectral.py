"""GPU parity of the k-resolved spectral-function moments (kite_spectral_k) against the
oracle's plain moments of the same plane-wave start vector (the spectral-function section):
bars 1e-12 (FP64) and 1e-5 (FP32) relative to mu_0(k); k-points on and off the torus grid,
both lattices, orbital weights, vacancies and several realisations."""
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


def oracle_spectral(d, M, kpts, w, S=1):
    s = oracle.make_system(**d)
    out = []
    for k in kpts:
        acc = 0.0
        for r in range(S):
            v = oracle.bloch_vector(s, k, w, realisation=r)
            acc = acc + oracle.moments_1d(s, M, 1, realisation=r, r0=v[None, :])[0]
        out.append(acc / S)
    return np.array(out)


@pytest.mark.parametrize("d,M,prec,S,w,dbl", [
    (dict(lattice=oracle.HONEYCOMB, Lx=24, Ly=20, t=-2.7, W=1.0, p_vac=0.02, seed=4), 96, "fp64", 1,
     [1.0, 1.0], False),
    (dict(lattice=oracle.HONEYCOMB, Lx=37, Ly=9, t=-2.7, W=2.0, delta=0.4, seed=5), 64, "fp32", 2,
     [0.3 + 0.4j, -1.1], False),
    (dict(lattice=oracle.SQUARE, Lx=33, Ly=17, t=-1.0, W=3.0, p_vac=0.03, seed=6), 50, "fp32", 1, [1.0], True),
    (dict(lattice=oracle.SQUARE, Lx=16, Ly=16, t=-1.0, W=0.5, seed=7), 40, "fp64", 3, [2.0j], True),
])
def test_spectral_moments_match_oracle(ctx, d, M, prec, S, w, dbl):
    g = np.random.Generator(np.random.PCG64(M))
    kpts = np.concatenate([g.uniform(-np.pi, np.pi, (9, 2)), [[0.0, 0.0], [np.pi, 0.0]]])
    nk = len(kpts)
    mu = np.zeros((nk, M, 2))
    wa = np.ascontiguousarray(np.stack([np.real(w), np.imag(w)], -1).astype(np.float64))
    kite.spectral_k(ctx, kite.make_system(**d), kite.make_kpm(M, 1, S, kite.FP64 if prec == "fp64" else kite.FP32,
                                                              doubling=dbl),
                    np.ascontiguousarray(kpts), nk, mu, weights=wa)
    got = mu[..., 0] + 1j * mu[..., 1]
    ref = oracle_spectral(d, M, kpts, w, S)
    bar = 1e-12 if prec == "fp64" else 1e-5
    scale = np.abs(ref[:, :1])
    assert np.max(np.abs(got - ref) / scale) <= bar


@pytest.mark.parametrize("d,M,prec,dbl", [
    (dict(lattice=oracle.HONEYCOMB, Lx=40, Ly=36, t=-2.7, W=1.0, p_vac=0.02, seed=4), 128, "fp64", False),
    (dict(lattice=oracle.SQUARE, Lx=33, Ly=17, t=-1.0, W=3.0, p_vac=0.03, seed=6), 80, "fp32", True),
])
def test_ldos_matches_oracle_basis_vectors(ctx, d, M, prec, dbl):
    """LDOS moments <i|T_n|i> of chosen orbitals (vacant ones included) against the oracle
    with the same basis start vectors (its moments times N_eff)."""
    s = oracle.make_system(**d)
    n = oracle.norb(s)
    _, vac = oracle.disorder(s)
    vacant = np.nonzero(vac)[0]
    orbs = np.array([0, 1, n // 2, n - 1, 7, 123] + ([int(vacant[0])] if len(vacant) else []), np.int64)
    mu = np.zeros((len(orbs), M, 2))
    kite.ldos(ctx, kite.make_system(**d), kite.make_kpm(M, 1, 1, kite.FP64 if prec == "fp64" else kite.FP32,
                                                        doubling=dbl), orbs, len(orbs), mu)
    got = mu[..., 0] + 1j * mu[..., 1]
    n_eff = int((vac == 0).sum())
    eye = np.zeros((len(orbs), n), np.complex128)
    eye[np.arange(len(orbs)), orbs] = 1.0
    ref = oracle.moments_1d(s, M, len(orbs), r0=eye) * n_eff
    bar = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(got - ref)) <= bar
    for j, o in enumerate(orbs):
        assert got[j, 0].real == (0.0 if vac[o] else 1.0) or abs(got[j, 0].real - (0.0 if vac[o] else 1.0)) <= bar
