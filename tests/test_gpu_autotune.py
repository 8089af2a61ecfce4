"""The autotuner (ring depth x resident CTAs per SM x steps per pass) changes only how the
sweep is laid on the GPU: the tuned and the default launch give the same moments to rounding, and the
choice is reported.  The grid decides which rows a thread's FP32 partial (at most 32
rows) groups before the FP64 sums, so the two launches agree to FP32 regrouping error
(bar 1e-7, far inside the 1e-5 bar against the oracle); a repeated launch with the cached
choice is bit-identical."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture()
def ctx():
    c = kite.Context(0)  # a fresh context: an empty tuning cache
    yield c
    c.close()


def with_tuning(flag, fn):
    old = os.environ.get("KITE_AUTOTUNE")
    os.environ["KITE_AUTOTUNE"] = flag
    try:
        return fn()
    finally:
        if old is None:
            del os.environ["KITE_AUTOTUNE"]
        else:
            os.environ["KITE_AUTOTUNE"] = old


@pytest.mark.parametrize("doubling", [False, True])
def test_tuned_sweep_matches_default(ctx, doubling):
    s = kite.make_system(kite.HONEYCOMB, 512, 384, -2.7, 2.0, 0.0, 0.01, 3)
    kpm = kite.make_kpm(96, 8, 1, kite.FP32, doubling=doubling)
    mu_t, mu_d = np.zeros(96), np.zeros(96)
    st_t = with_tuning("1", lambda: kite.moments_1d(ctx, s, kpm, mu_t))
    st_d = with_tuning("0", lambda: kite.moments_1d(ctx, s, kpm, mu_d))
    # one step per pass (4 or 8 stages) or two (5, 6 or 8 stages; plain or doubling)
    assert st_t.ring_stages in (4, 5, 6, 8) and st_t.ctas_per_sm >= 1 and st_t.steps_per_pass in (1, 2)
    assert st_d.ring_stages == 8 and st_d.steps_per_pass == 1
    assert np.max(np.abs(mu_t - mu_d)) <= 1e-7
    st_again = with_tuning("1", lambda: kite.moments_1d(ctx, s, kpm, mu_d))  # cached choice
    assert (st_again.ring_stages, st_again.ctas_per_sm) == (st_t.ring_stages, st_t.ctas_per_sm)
    assert np.array_equal(mu_t, mu_d)  # same launch shape: bit-identical


def test_tuned_batch_matches_default(ctx):
    specs = [(300, 1.0, 96, 11), (40, 2.0, 64, 12), (17, 0.5, 33, 13), (130, 3.0, 128, 14)]
    systems = [kite.make_system(kite.SQUARE, L, L, -1.0, W, 0.0, 0.0, seed) for L, W, M, seed in specs]
    for dbl in (False, True):
        kpms = [kite.make_kpm(M, 4, 1, kite.FP32, doubling=dbl) for _, _, M, _ in specs]
        mus_t = [np.zeros(M) for _, _, M, _ in specs]
        mus_d = [np.zeros(M) for _, _, M, _ in specs]
        st_t = with_tuning("1", lambda: kite.moments_1d_batched(ctx, systems, kpms, mus_t))
        st_d = with_tuning("0", lambda: kite.moments_1d_batched(ctx, systems, kpms, mus_d))
        # one step per pass (4 or 8 stages) or two (5, 6 or 8 stages)
        assert st_t.ring_stages in (4, 5, 6, 8) and st_t.ctas_per_sm >= 1 and st_d.ring_stages == 8
        assert st_t.steps_per_pass in (1, 2) and st_d.steps_per_pass == 1
        for a, b in zip(mus_t, mus_d):
            assert np.max(np.abs(a - b)) <= 1e-7
