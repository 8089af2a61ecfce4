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
    norm, curve = learned.train(ctx, X[:ntr], T[:ntr], e_min, e_max, p, epochs=40, batch=128, lr=1e-3,
                                seed=3)
    assert curve[-1] < curve[0]
    rho, flags, dev = learned.infer(ctx, p, norm, mu[ntr:], e_min, e_max)
    l1_net = np.mean(learned.l1_error(rho, T[ntr:], e_min, e_max))
    l1_base = np.mean(learned.l1_error(base[ntr:], T[ntr:], e_min, e_max))
    print(f"held-out L1: network {l1_net:.4f}, Jackson M=128 {l1_base:.4f}; loss {curve[0]:.4g} -> "
          f"{curve[-1]:.4g}; gate flagged {flags.sum()} median dev {np.median(dev):.3g}")
    assert l1_net < l1_base
    assert np.all(np.isfinite(dev))


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
