"""GPU parity of the wave-packet propagation (kite_propagate) against the oracle's
Chebyshev series on the same start states (the wave-packet section): bars 1e-10 (FP64)
and 2e-5 relative to max|psi| (FP32, whose accumulated series carries ~M ulp); the norm
is conserved; several wave functions (more than one batch), vacancies, both lattices."""
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


@pytest.mark.parametrize("d,R,dt,steps,M,prec", [
    (dict(lattice=oracle.HONEYCOMB, Lx=24, Ly=20, t=-2.7, W=1.0, p_vac=0.02, seed=4), 3, 0.5, 3, 40, "fp64"),
    (dict(lattice=oracle.HONEYCOMB, Lx=37, Ly=9, t=-2.7, W=2.0, delta=0.4, seed=5), 6, 1.2, 2, 60, "fp64"),
    (dict(lattice=oracle.SQUARE, Lx=33, Ly=17, t=-1.0, W=3.0, p_vac=0.03, seed=6), 5, 0.8, 3, 40, "fp32"),
    (dict(lattice=oracle.SQUARE, Lx=16, Ly=16, t=-1.0, W=0.5, seed=7), 1, 2.0, 1, 1, "fp64"),
])
def test_propagation_matches_oracle(ctx, d, R, dt, steps, M, prec):
    s = oracle.make_system(**d)
    n = oracle.norb(s)
    psi0 = synth.gaussian_vectors(n, R, seed=R * 31 + M)
    psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
    psi = np.ascontiguousarray(np.stack([psi0.real, psi0.imag], -1))
    norms = np.zeros((steps, R))
    kite.propagate(ctx, kite.make_system(**d), kite.make_kpm(M, R, 1, kite.FP64 if prec == "fp64" else kite.FP32),
                   dt, steps, psi, norms)
    got = psi[..., 0] + 1j * psi[..., 1]
    _, vac = oracle.disorder(s)
    for r in range(R):
        ref = oracle.propagate(s, psi0[r], dt, steps, M)
        bar = 1e-10 if prec == "fp64" else 2e-5
        assert np.max(np.abs(got[r] - ref[-1])) <= bar * max(1.0, np.max(np.abs(ref[-1]))), r
        ref_norms = np.sum(np.abs(ref) ** 2, axis=1)
        assert np.max(np.abs(norms[:, r] - ref_norms)) <= (1e-10 if prec == "fp64" else 1e-5)
    assert np.all(got[:, vac != 0] == 0)


def test_long_step_is_unitary(ctx):
    """A long time step with enough terms (de_minus dt = 87, M = 140) keeps the norm."""
    d = dict(lattice=oracle.HONEYCOMB, Lx=64, Ly=64, t=-2.7, W=1.0, seed=9)
    s = oracle.make_system(**d)
    n = oracle.norb(s)
    psi0 = synth.unit_phase_vectors(n, 2, seed=3) / np.sqrt(n)
    psi = np.ascontiguousarray(np.stack([psi0.real, psi0.imag], -1))
    norms = np.zeros((4, 2))
    kite.propagate(ctx, kite.make_system(**d), kite.make_kpm(140, 2, 1, kite.FP64), 10.0, 4, psi, norms)
    assert np.max(np.abs(norms - 1.0)) <= 1e-9
