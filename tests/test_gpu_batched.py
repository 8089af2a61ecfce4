"""GPU parity of the batched persistent sweep (kite_moments_1d_batched): every system of a
mixed batch against the oracle (FP32 recursion, bar 1e-5), the bounded team barrier, and
the 256-system square-lattice workload (side 64..1024, W 0..4, M in {512..4096}, R = 4) in
its own launch configuration with sampled oracle checks and properties for the rest."""
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


def batch(ctx, specs, R=4, doubling=False, lattice=None):
    lat = kite.SQUARE if lattice is None else lattice
    t = -1.0 if lat == kite.SQUARE else -2.7
    systems = [kite.make_system(lat, sp["L"], sp.get("Ly", sp["L"]), t, sp["W"], 0.0,
                                sp.get("p", 0.0), sp["seed"]) for sp in specs]
    kpms = [kite.make_kpm(sp["M"], R, 1, kite.FP32, doubling=doubling) for sp in specs]
    mus = [np.zeros(sp["M"]) for sp in specs]
    st = kite.moments_1d_batched(ctx, systems, kpms, mus)
    return mus, st


def oracle_mu(sp, R=4, lattice=None):
    lat = oracle.SQUARE if lattice is None else lattice
    t = -1.0 if lat == oracle.SQUARE else -2.7
    s = oracle.make_system(lattice=lat, Lx=sp["L"], Ly=sp.get("Ly", sp["L"]), t=t,
                           W=sp["W"], p_vac=sp.get("p", 0.0), seed=sp["seed"])
    return oracle.moments_1d(s, sp["M"], R).real.mean(0)


def test_mixed_batch_against_oracle(ctx):
    specs = [dict(L=400, Ly=300, W=1.0, M=96, seed=11),  # large: a multi-CTA team
             dict(L=3, W=2.0, M=16, seed=12), dict(L=17, Ly=5, W=0.0, M=33, seed=13),
             dict(L=130, W=4.0, M=64, seed=14, p=0.02), dict(L=64, W=2.5, M=128, seed=15),
             dict(L=257, Ly=40, W=3.0, M=48, seed=16), dict(L=9, W=1.0, M=1, seed=17),
             dict(L=100, W=0.5, M=2, seed=18), dict(L=77, W=3.5, M=200, seed=19)]
    mus, st = batch(ctx, specs)
    for sp, mu in zip(specs, mus):
        ref = oracle_mu(sp)
        assert np.max(np.abs(mu - ref)) <= 1e-5, sp
    assert st.grid >= 2 and st.seconds > 0


@pytest.mark.parametrize("R", [4, 1])
def test_mixed_batch_with_moment_doubling(ctx, R):
    """The same mixed batch with moment doubling (two moments per step, odd and tiny M,
    multi-CTA and packed teams): same 1e-5 bar against the oracle's plain moments."""
    specs = [dict(L=400, Ly=300, W=1.0, M=96, seed=11), dict(L=3, W=2.0, M=16, seed=12),
             dict(L=17, Ly=5, W=0.0, M=33, seed=13), dict(L=130, W=4.0, M=64, seed=14, p=0.02),
             dict(L=9, W=1.0, M=1, seed=17), dict(L=100, W=0.5, M=2, seed=18),
             dict(L=77, W=3.5, M=201, seed=19)]
    mus, st = batch(ctx, specs, R=R, doubling=True)
    for sp, mu in zip(specs, mus):
        assert np.max(np.abs(mu - oracle_mu(sp, R))) <= 1e-5, sp
    with pytest.raises(kite.KiteError):  # doubling must be uniform over a batch
        systems = [kite.make_system(kite.SQUARE, 8, 8, -1.0, 1.0, 0.0, 0.0, 1)] * 2
        kite.moments_1d_batched(ctx, systems, [kite.make_kpm(8, 1, 1, kite.FP32, doubling=d)
                                               for d in (True, False)], [np.zeros(8), np.zeros(8)])


@pytest.mark.parametrize("steps", ["1", "2"])
def test_mixed_batch_pinned_steps_per_pass(ctx, steps, monkeypatch):
    """KITE_PASS_STEPS pins one recursion step per pass (k_batched) or two (a first-step
    launch, then k_batched2's passes with an odd last step run as a whole pass): every
    system within 1e-5 of the oracle, multi-CTA and packed teams, odd and even M."""
    specs = [dict(L=400, Ly=300, W=1.0, M=96, seed=11), dict(L=17, Ly=5, W=0.0, M=33, seed=13),
             dict(L=130, W=4.0, M=64, seed=14, p=0.02), dict(L=64, W=2.5, M=128, seed=15),
             dict(L=257, Ly=40, W=3.0, M=48, seed=16), dict(L=9, W=1.0, M=4, seed=17),
             dict(L=77, W=3.5, M=201, seed=19), dict(L=31, W=2.0, M=5, seed=20)]
    monkeypatch.setenv("KITE_PASS_STEPS", steps)
    mus, st = batch(ctx, specs)
    assert st.steps_per_pass == int(steps)
    for sp, mu in zip(specs, mus):
        assert np.max(np.abs(mu - oracle_mu(sp))) <= 1e-5, sp


@pytest.mark.parametrize("steps,doubling,R", [("1", False, 8), ("2", False, 8), ("2", False, 3),
                                              (None, True, 8)])
def test_honeycomb_batch_against_oracle(ctx, steps, doubling, R, monkeypatch):
    """A honeycomb batch (two sublattices per cell; R = 8: four chunks per orbital, R = 3:
    a padded batch) with one or two steps per pass or moment doubling, vacancies, a
    multi-CTA team and packed teams: every system within 1e-5 of the oracle."""
    specs = [dict(L=300, Ly=200, W=2.0, M=64, seed=31, p=0.01), dict(L=24, Ly=9, W=1.0, M=33, seed=32),
             dict(L=70, W=3.0, M=50, seed=33, p=0.02), dict(L=13, W=0.5, M=8, seed=34),
             dict(L=45, Ly=30, W=1.5, M=97, seed=35)]
    if steps is not None:
        monkeypatch.setenv("KITE_PASS_STEPS", steps)
    mus, st = batch(ctx, specs, R=R, doubling=doubling, lattice=kite.HONEYCOMB)
    if steps is not None:
        assert st.steps_per_pass == int(steps)
    for sp, mu in zip(specs, mus):
        assert np.max(np.abs(mu - oracle_mu(sp, R, lattice=oracle.HONEYCOMB))) <= 1e-5, sp


@pytest.mark.parametrize("steps", ["1", "2"])
def test_doubling_batch_pinned_steps_per_pass(ctx, steps, monkeypatch):
    """Moment doubling with one step per pass or two (the doubling form of the two-step
    pass: slots 2n .. 2n+3 per pass, an odd last step run as a whole pass): every system
    within 1e-5 of the oracle's plain moments."""
    specs = [dict(L=400, Ly=300, W=1.0, M=96, seed=11), dict(L=17, Ly=5, W=0.0, M=33, seed=13),
             dict(L=130, W=4.0, M=64, seed=14, p=0.02), dict(L=64, W=2.5, M=127, seed=15),
             dict(L=257, Ly=40, W=3.0, M=48, seed=16), dict(L=9, W=1.0, M=5, seed=17),
             dict(L=77, W=3.5, M=201, seed=19), dict(L=31, W=2.0, M=6, seed=20)]
    monkeypatch.setenv("KITE_PASS_STEPS", steps)
    mus, st = batch(ctx, specs, doubling=True)
    assert st.steps_per_pass == int(steps)
    for sp, mu in zip(specs, mus):
        assert np.max(np.abs(mu - oracle_mu(sp))) <= 1e-5, sp


def test_team_barrier_timeout_is_reported(ctx):
    specs = [dict(L=600, W=1.0, M=24, seed=21), dict(L=20, W=1.0, M=8, seed=22)]
    kite.debug_stall_once(ctx)
    with pytest.raises(kite.KiteError) as e:
        batch(ctx, specs)
    assert e.value.status == kite.ERR_TIMEOUT
    mus, _ = batch(ctx, specs)  # the context stays usable
    assert np.max(np.abs(mus[1] - oracle_mu(specs[1]))) <= 1e-5


def test_256_system_workload(ctx):
    specs = synth.batched_square_systems(256, seed=3)
    mus, st = batch(ctx, specs)
    print(f"256 systems: {st.updates:.3e} updates in {st.seconds:.3f} s = "
          f"{st.updates / st.seconds:.3e} updates/s, grid {st.grid}")
    for sp, mu in zip(specs, mus):
        # |mu_n| <= 1 in exact arithmetic (|T_n| <= 1 on the rescaled spectrum, unit-norm
        # vectors); the FP32 partial sums round at ~1e-7, hence the same 1e-6 as for mu_0
        assert abs(mu[0] - 1.0) <= 1e-6
        assert np.all(np.abs(mu) <= 1.0 + 1e-6)
    # the systems the CPU oracle finishes quickly: every moment
    cheap = sorted(range(256), key=lambda i: specs[i]["L"] ** 2 * specs[i]["M"])[:6]
    for i in cheap:
        assert np.max(np.abs(mus[i] - oracle_mu(specs[i]))) <= 1e-5, specs[i]
    # the same workload with moment doubling: half the steps, same moments
    mus_d, st_d = batch(ctx, specs, doubling=True)
    print(f"256 systems, doubling: {st_d.updates / st_d.seconds:.3e} updates/s in {st_d.seconds:.3f} s")
    for i in range(256):
        assert np.max(np.abs(mus_d[i] - mus[i])) <= 2e-5, specs[i]
    for i in cheap:
        assert np.max(np.abs(mus_d[i] - oracle_mu(specs[i]))) <= 1e-5, specs[i]
    # the largest system of the batch (side 996, M = 4096: a multi-CTA team through 4095
    # team barriers), every moment against the oracle
    big = max(range(256), key=lambda i: specs[i]["L"] ** 2 * specs[i]["M"])
    assert specs[big]["M"] == 4096
    ref = oracle_mu(specs[big])
    print(f"largest system {specs[big]}: max |dmu| {np.max(np.abs(mus[big] - ref)):.2e} (plain), "
          f"{np.max(np.abs(mus_d[big] - ref)):.2e} (doubling)")
    assert np.max(np.abs(mus[big] - ref)) <= 1e-5
    assert np.max(np.abs(mus_d[big] - ref)) <= 1e-5
