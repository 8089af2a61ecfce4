"""The learned reconstructor's hand-written kernels against the FP64 oracle MLP, and a small
end-to-end training run that must beat the plain 128-moment Jackson reconstruction.

Bars: forward outputs and per-layer gradients within BF16 tolerance of the oracle run on
the kernel's parameters (BF16 weights, FP32 biases) and BF16-stored activations, so that
both sides take the ReLU decisions on the same stored values (relative L2 error <= 2e-2;
BF16 rounding of the stored deltas and activations is ~4e-3 per layer); the residual prior
(a Jackson reconstruction in FP64, stored as FP32) within 1e-6 of the oracle's; after
training, the held-out mean L1 error of the network must be below that of the Jackson
reconstruction from the same 128 moments."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")
from paper_1910_05194_gb300 import learned  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = kite.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def test_param_count_matches_layout():
    assert kite.mlp_param_count() == omlp.n_params()
    assert synth.mlp_init(0).size == omlp.n_params()


def test_forward_and_gradient_match_oracle(ctx):
    n = 64
    p = synth.mlp_init(7)
    p[omlp.n_params() - omlp.OUT:] = 0.01  # nonzero output biases (FP32 on both sides)
    g = np.random.Generator(np.random.PCG64(8))
    X = g.standard_normal((n, omlp.IN)).astype(np.float32)
    Y = np.zeros((n, omlp.OUT), np.float32)
    kite.mlp_forward(ctx, p, X, n, Y)
    pk = omlp.kernel_params(p)
    Xk = omlp.round_bf16(X)
    Yref, _ = omlp.forward(pk, Xk, act_round=omlp.round_bf16)
    assert rel(Y, Yref) <= 2e-2
    # targets far from the outputs so the sign of the residual is the same on both sides
    T = (Yref + np.where(g.random(Yref.shape) < 0.5, -1.0, 1.0) * (0.5 + np.abs(Yref))).astype(np.float32)
    grad = np.zeros(kite.mlp_param_count(), np.float32)
    loss = kite.mlp_gradient(ctx, p, X, T, n, grad)
    gref = omlp.grad(pk, Xk, T, act_round=omlp.round_bf16)
    assert abs(loss - omlp.loss(pk, Xk, T, act_round=omlp.round_bf16)) <= 1e-2 * loss
    off = 0
    for shp in omlp.shapes():
        k = int(np.prod(shp))
        assert rel(grad[off:off + k], gref[off:off + k]) <= 2e-2, shp
        off += k


def test_input_normalisation_matches_oracle(ctx):
    """(x - shift) * scale in FP32 before the BF16 rounding, as the oracle computes it."""
    n = 48
    p = synth.mlp_init(13)
    g = np.random.Generator(np.random.PCG64(14))
    X = (0.3 + 0.05 * g.standard_normal((n, omlp.IN))).astype(np.float32)
    shift = X.mean(0).astype(np.float32)
    scale = (1.0 / X.std(0)).astype(np.float32)
    Y = np.zeros((n, omlp.OUT), np.float32)
    kite.mlp_forward(ctx, p, X, n, Y, shift=shift, scale=scale)
    Xk = omlp.round_bf16((X - shift) * scale)
    Yref, _ = omlp.forward(omlp.kernel_params(p), Xk, act_round=omlp.round_bf16)
    assert rel(Y, Yref) <= 2e-2


def test_jackson_prior_matches_oracle(ctx):
    """With all parameters zero the network adds nothing: the output is the prior alone."""
    n = 40
    e_min, e_max = -10.7, 10.7
    d = dict(lattice=oracle.HONEYCOMB, Lx=24, Ly=24, t=-2.7, W=2.0, delta=0.4, seed=31)
    mu = np.stack([oracle.moments_1d(oracle.make_system(**dict(d, seed=31 + i)), omlp.IN, 1,
                                     e_min=e_min, e_max=e_max).real[0] for i in range(n)])
    X = mu.astype(np.float32)
    Y = np.zeros((n, omlp.OUT), np.float32)
    kite.mlp_forward(ctx, np.zeros(omlp.n_params(), np.float32), X, n, Y,
                     prior=kite.jackson_prior(e_min, e_max))
    ref = omlp.prior(X.astype(np.float64), e_min, e_max)
    assert np.max(np.abs(Y - ref)) <= 1e-6 * np.max(np.abs(ref))
    # and prior + network equals the two parts taken separately
    p = synth.mlp_init(9)
    Yn = np.zeros_like(Y)
    kite.mlp_forward(ctx, p, X, n, Yn)
    Yb = np.zeros_like(Y)
    kite.mlp_forward(ctx, p, X, n, Yb, prior=kite.jackson_prior(e_min, e_max))
    assert np.max(np.abs(Yb - (Yn + Y))) <= 1e-5 * np.max(np.abs(Yb))


def make_dataset(ctx, n, seed, L=48, M_hi=1024, R=2):
    specs = synth.learned_dos_systems(n, seed, L=L)
    systems = learned.to_systems(specs)
    e_min, e_max = learned.window(1.0, 4.0)
    mu, _ = learned.batched_moments(ctx, systems, M_hi, R, e_min, e_max)
    T = learned.jackson_dos(ctx, mu, M_hi, e_min, e_max)
    base = learned.jackson_dos(ctx, mu, omlp.IN, e_min, e_max)
    return mu, T, base, e_min, e_max


def test_training_beats_the_plain_low_order_reconstruction(ctx):
    ntr, nte = 2048, 256
    mu, T, base, e_min, e_max = make_dataset(ctx, ntr + nte, seed=70_000)
    X = mu[:, :omlp.IN].astype(np.float32)
    p = synth.mlp_init(11, head_scale=0.01)
    model, curve = learned.train(ctx, X[:ntr], T[:ntr], e_min, e_max, init=p, epochs=40, batch=128, lr=1e-3,
                                 seed=3)
    assert curve[-1] < curve[0]
    rho, _, _ = learned.infer(ctx, model, mu[ntr:], tol=float("inf"))
    _, flags, dev = learned.infer(ctx, model, mu[ntr:])
    l1_net = np.mean(learned.l1_error(rho, T[ntr:], e_min, e_max))
    l1_base = np.mean(learned.l1_error(base[ntr:], T[ntr:], e_min, e_max))
    print(f"held-out L1: network {l1_net:.4f}, Jackson M=128 {l1_base:.4f}; loss {curve[0]:.4g} -> "
          f"{curve[-1]:.4g}; gate flagged {flags.sum()} median dev {np.median(dev):.3g}")
    assert l1_net < l1_base
    assert np.all(np.isfinite(dev))
    model.close()


def test_adamw_step_matches_oracle(ctx):
    """kite_mlp_adamw_step (the device update of kite_mlp_train) against the oracle's AdamW
    and cosine schedule over five steps of a ten-step schedule, with a fresh gradient each
    step; p, m and v element by element on a ragged length.  FP32 arithmetic on the device:
    m and v within 1e-6 per step of the size of their terms, p within a few ulp plus 1e-5
    of the step size per step."""
    n = 100_003
    g = np.random.Generator(np.random.PCG64(21))
    p = (0.1 * g.standard_normal(n)).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    pr, mr, vr = p.astype(np.float64), np.zeros(n), np.zeros(n)
    mabs = np.zeros(n)  # the first moment's sum of |terms|: its FP32 rounding scale
    lr, wd, total = 3e-3, 1e-2, 10
    for t in range(1, 6):
        grad = (g.standard_normal(n) * 10.0 ** g.uniform(-6, 0, n)).astype(np.float32)
        kite.mlp_adamw_step(ctx, p, grad, m, v, n, t, total, lr, wd)
        pr, mr, vr = omlp.adamw_step(pr, grad.astype(np.float64), mr, vr, t, omlp.cosine_lr(t, total, lr), wd=wd)
        mabs = 0.9 * mabs + 0.1 * np.abs(grad)
        assert np.all(np.abs(m - mr) <= 1e-6 * t * mabs), t
        assert np.all(np.abs(v - vr) <= 1e-6 * t * vr), t
        assert np.all(np.abs(p - pr) <= 4 * np.spacing(np.abs(pr).astype(np.float32)) * t + 1e-5 * lr * t), t


def test_training_steps_match_oracle(ctx):
    """kite_mlp_train, full batch for six optimiser steps (one per epoch, cosine schedule
    over six), against the oracle's gradient and AdamW step by step.  The oracle stores the
    activations and the back-propagated deltas in BF16 as the kernels do, so both sides take
    the same ReLU decisions on the same stored values and the gradients agree to FP32
    accumulation; targets are far from the outputs so every residual keeps its sign.  Each
    parameter's total move must agree within 2 % of the distance travelled (6 lr); the
    parameters whose gradient is below the FP32 noise of its sum may differ in their first
    steps, and at most 1 in 1000 do."""
    n, steps, lr, wd = 64, 6, 1e-3, 1e-4
    p0 = synth.mlp_init(31)
    p0[omlp.n_params() - omlp.OUT:] = 0.01
    g = np.random.Generator(np.random.PCG64(32))
    X = g.standard_normal((n, omlp.IN)).astype(np.float32)
    Y0, _ = omlp.forward(omlp.kernel_params(p0), omlp.round_bf16(X), act_round=omlp.round_bf16)
    T = (Y0 + np.where(g.random(Y0.shape) < 0.5, -1.0, 1.0) * (1.0 + np.abs(Y0))).astype(np.float32)
    p = p0.copy()
    kite.mlp_train(ctx, X, T, n, p, epochs=steps, batch=n, lr=lr, weight_decay=wd, seed=5)
    Xk = omlp.round_bf16(X)
    pr = p0.astype(np.float64)
    m, v = np.zeros_like(pr), np.zeros_like(pr)
    for t in range(1, steps + 1):
        gr = omlp.grad(omlp.kernel_params(pr), Xk, T, act_round=omlp.round_bf16, delta_round=omlp.round_bf16)
        pr, m, v = omlp.adamw_step(pr, gr, m, v, t, omlp.cosine_lr(t, steps, lr), wd=wd)
    d_gpu = p.astype(np.float64) - p0
    d_ref = pr - p0
    bad = np.abs(d_gpu - d_ref) > 0.02 * steps * lr
    print(f"parameters off by more than 2 % of 6 lr: {bad.sum()} of {bad.size}")
    assert bad.mean() <= 1e-3
    assert np.max(np.abs(d_gpu - d_ref)) <= 2 * steps * lr * 1.01
    assert np.linalg.norm(d_gpu - d_ref) <= 0.02 * np.linalg.norm(d_ref)


def test_learned_train_owns_normalisation_and_initial_weights(ctx):
    """kite_learned_train: the model's input shift and scale are the training set's per-moment
    mean and 1/max(std, 1e-4) (population std; numpy in FP64 as the definition), and with no
    initial parameters the weights are drawn on the device: He-uniform within sqrt(6/fan_in)
    (the last layer times head_scale), zero biases, reproducible for a seed.  A learning rate
    of 1e-30 leaves the drawn parameters in place (to 1e-29)."""
    n = 300
    g = np.random.Generator(np.random.PCG64(41))
    X = (g.standard_normal((n, omlp.IN)) * np.linspace(0.01, 2.0, omlp.IN) + np.linspace(-1, 1, omlp.IN))
    X[:, 0] = 1.0  # a constant column: std floored
    X = X.astype(np.float32)
    Y = g.standard_normal((n, omlp.OUT)).astype(np.float32)
    e_min, e_max = -10.0, 10.0
    m1 = kite.learned_train(ctx, X, Y, n, e_min, e_max, epochs=1, batch=n, lr=1e-30, seed=77, head_scale=0.05)
    p, sh, sc, win = m1.export()
    Xd = X.astype(np.float64)
    assert np.allclose(sh, Xd.mean(0), rtol=1e-6, atol=1e-7)
    assert np.allclose(sc, 1.0 / np.maximum(Xd.std(0), 1e-4), rtol=1e-5)
    assert win == (e_min, e_max)
    off = 0
    for k, shp in enumerate(omlp.shapes()):
        size = int(np.prod(shp))
        part = p[off:off + size].astype(np.float64)
        off += size
        if len(shp) == 1:
            assert np.max(np.abs(part)) <= 1e-29
            continue
        lim = np.sqrt(6.0 / shp[1]) * (0.05 if k == 4 else 1.0)
        assert np.max(np.abs(part)) <= lim
        assert abs(part.mean()) <= 5 * lim / np.sqrt(3 * size)
        assert abs(part.var() / (lim * lim / 3) - 1.0) <= 0.02
    m2 = kite.learned_train(ctx, X, Y, n, e_min, e_max, epochs=1, batch=n, lr=1e-30, seed=77, head_scale=0.05)
    m3 = kite.learned_train(ctx, X, Y, n, e_min, e_max, epochs=1, batch=n, lr=1e-30, seed=78, head_scale=0.05)
    assert np.array_equal(m2.export()[0], p)
    assert not np.array_equal(m3.export()[0], p)
    for m in (m1, m2, m3):
        m.close()


def test_learned_dos_network_gate_and_fallback(ctx):
    """kite_learned_dos in its three branches.
    (a) gate off (tol = inf): the output is prior + network of the model's parameters and
        normalisation, against the oracle MLP at the forward bar, and equal to
        kite_mlp_forward of the exported model;
    (b) forced fallback (tol = 0) on the rows' own moments: every row is the Jackson DOS of
        its first M_plain moments, against the oracle's reconstruction (FP32 output) and equal
        to kite_reconstruct_dos;
    (c) forced fallback with the systems: the plain FP64 path reruns each system at M_plain,
        against the oracle's moments and DOS."""
    e_min, e_max = learned.window(1.0, 4.0)
    specs = synth.learned_dos_systems(6, 81_000, L=24)
    systems = learned.to_systems(specs)
    mu, _ = learned.batched_moments(ctx, systems, 256, 2, e_min, e_max)
    T = learned.jackson_dos(ctx, mu, 256, e_min, e_max)
    X = mu[:, :omlp.IN].astype(np.float32)
    model, _ = learned.train(ctx, X, T, e_min, e_max, epochs=3, batch=6, seed=9, head_scale=0.1)
    p, sh, sc, _ = model.export()
    n = len(systems)
    # (a)
    rho, flags, dev = learned.infer(ctx, model, mu, tol=float("inf"))
    assert flags.tolist() == [0] * n and np.all(np.isfinite(dev))
    Yf = np.zeros((n, omlp.OUT), np.float32)
    kite.mlp_forward(ctx, p, X, n, Yf, shift=sh, scale=sc, prior=kite.jackson_prior(e_min, e_max))
    assert np.array_equal(rho, Yf)
    Xk = omlp.round_bf16((X - sh) * sc)
    Yref = omlp.forward(omlp.kernel_params(p), Xk, act_round=omlp.round_bf16)[0] + omlp.prior(X, e_min, e_max)
    assert rel(rho, Yref) <= 2e-2
    # (b)
    M_plain = 192
    rho_b, flags_b, _ = learned.infer(ctx, model, mu, tol=0.0, M_plain=M_plain)
    assert flags_b.tolist() == [1] * n
    E = learned.midpoint_energies(e_min, e_max)
    ref = np.zeros(omlp.OUT)
    for i in range(n):
        kite.reconstruct_dos(ctx, mu[i], mu.shape[1], M_plain, kite.KERNEL_JACKSON, 0.0, e_min, e_max, E, E.size, ref)
        assert np.array_equal(rho_b[i], ref.astype(np.float32))
        o = oracle.dos(mu[i, :M_plain], E, e_min, e_max, oracle.kernel_jackson(M_plain))
        assert np.max(np.abs(rho_b[i] - o)) <= 1e-6 * np.max(np.abs(o))
    # (c)
    rho_c = np.zeros((n, omlp.OUT), np.float32)
    flags_c = np.zeros(n, np.int32)
    kite.learned_dos(ctx, model, mu, mu.shape[1], n, 0.0, 16, M_plain, rho_c, flags_c, systems=systems,
                     plain_kpm=kite.make_kpm(M_plain, 2, 1, kite.FP64))
    assert flags_c.tolist() == [1] * n
    for i, sp in enumerate(specs):
        osys = oracle.make_system(lattice=oracle.HONEYCOMB, Lx=sp["L"], Ly=sp["L"], t=learned.T_HOP, W=sp["W"],
                                  delta=sp["delta"], p_vac=sp["p_vac"], seed=sp["seed"])
        mo = oracle.moments_1d(osys, M_plain, 2, e_min=e_min, e_max=e_max).real.mean(0)
        o = oracle.dos(mo, E, e_min, e_max, oracle.kernel_jackson(M_plain))
        assert np.max(np.abs(rho_c[i] - o)) <= 1e-6 * np.max(np.abs(o)), i
    model.close()


def test_gate_flags_out_of_distribution_inputs(ctx):
    """A density that contradicts its own moments is flagged; the prior alone (the Jackson
    reconstruction of the same moments) passes."""
    e_min, e_max = learned.window(1.0, 4.0)
    d = dict(lattice=oracle.HONEYCOMB, Lx=32, Ly=32, t=-2.7, W=1.0, seed=5)
    mu = oracle.moments_1d(oracle.make_system(**d), 256, 1, e_min=e_min, e_max=e_max).real
    good = omlp.prior(mu[:, :omlp.IN], e_min, e_max).astype(np.float32)
    bad = good.copy()
    bad[0, :omlp.OUT // 2] *= 1.5
    rho = np.concatenate([good, bad])
    mus = np.concatenate([mu, mu])
    flags = np.zeros(2, np.int32)
    dev = np.zeros(2)
    kite.learned_gate(ctx, rho, np.ascontiguousarray(mus), mus.shape[1], 2, 16, e_min, e_max, 0.02, flags, dev)
    assert flags.tolist() == [0, 1], dev


def test_model_import_export_and_argument_errors(ctx):
    """A model rebuilt from its exported parts gives the same densities; the learned calls
    refuse inconsistent arguments with KITE_ERR_ARG and leave the context usable."""
    e_min, e_max = -10.0, 10.0
    g = np.random.Generator(np.random.PCG64(51))
    X = g.standard_normal((64, omlp.IN)).astype(np.float32)
    Y = np.abs(g.standard_normal((64, omlp.OUT))).astype(np.float32)
    m1 = kite.learned_train(ctx, X, Y, 64, e_min, e_max, epochs=2, batch=32, seed=5, head_scale=0.1)
    p, sh, sc, win = m1.export()
    m2 = kite.model_import(ctx, p, win[0], win[1], shift=sh, scale=sc)
    mu = np.zeros((8, 200))
    mu[:, 0] = 1.0
    mu[:, 1:omlp.IN] = 0.01 * g.standard_normal((8, omlp.IN - 1))
    out = []
    for m in (m1, m2):
        rho = np.zeros((8, omlp.OUT), np.float32)
        flags = np.zeros(8, np.int32)
        kite.learned_dos(ctx, m, mu, 200, 8, float("inf"), 16, 64, rho, flags)
        out.append(rho)
    assert np.array_equal(out[0], out[1])
    rho = np.zeros((8, omlp.OUT), np.float32)
    flags = np.zeros(8, np.int32)
    for bad in (dict(mu_ld=100), dict(kcheck=0), dict(M_plain=300), dict(gate_tol=-1.0)):
        a = dict(mu_ld=200, kcheck=16, M_plain=64, gate_tol=0.02)
        a.update(bad)
        with pytest.raises(kite.KiteError) as e:
            kite.learned_dos(ctx, m1, mu, a["mu_ld"], 8, a["gate_tol"], a["kcheck"], a["M_plain"], rho, flags)
        assert e.value.status == kite.ERR_ARG, bad
    with pytest.raises(kite.KiteError) as e:  # systems without the plain path's parameters
        kite.learned_dos(ctx, m1, mu, 200, 8, 0.0, 16, 64, rho, flags,
                         systems=[kite.make_system(kite.HONEYCOMB, 8, 8, -2.7)] * 8)
    assert e.value.status == kite.ERR_ARG
    with pytest.raises(kite.KiteError) as e:
        kite.learned_train(ctx, X, Y, 64, 1.0, -1.0)  # empty window
    assert e.value.status == kite.ERR_ARG
    kite.learned_dos(ctx, m1, mu, 200, 8, float("inf"), 16, 64, rho, flags)  # still usable
    assert np.array_equal(rho, out[0])
    m1.close()
    m2.close()
