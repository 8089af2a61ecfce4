"""Host-side logic of the library checked on the CPU (no GPU call): the wave-packet
propagator's coefficients against the oracle's (scipy Bessel functions)."""
import numpy as np
import pytest

import oracle

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture(scope="module")
def lib_loaded():
    try:
        kite.lib()
    except Exception as e:  # the shared library is built by the build step
        pytest.skip(f"library not built: {e}")


@pytest.mark.parametrize("M,dt,lo,hi", [(1, 0.3, -1.0, 1.0), (40, 0.5, -8.7, 8.7), (200, 3.0, -10.0, 14.0),
                                        (700, 50.0, -9.0, 9.0), (64, 0.0, -3.0, 3.0)])
def test_evolution_coefficients_match_oracle(lib_loaded, M, dt, lo, hi):
    got = kite.evolution_coeffs(M, dt, lo, hi)
    ref = oracle.evolution_coeffs(M, dt, lo, hi)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
