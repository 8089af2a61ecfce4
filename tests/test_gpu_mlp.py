"""The learned reconstructor's hand-written kernels against the FP64 oracle MLP, and a small
end-to-end training run that must beat the plain 128-moment Jackson reconstruction.

Bars: forward outputs and per-layer gradients within BF16 tolerance of the oracle run on
the same BF16-rounded weights and inputs (relative L2 error <= 2e-2; BF16 activations
carry ~4e-3 relative rounding per layer); after training, the held-out mean L1 error of
the network must be below that of the Jackson reconstruction from the same 128 moments."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture(scope="module")
def ctx():
    c = kite.Context(0)
    yield c
    c.close()


def bf16(x):
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000  # round to nearest even
    return u.astype(np.uint32).view(np.float32)


def test_param_count_matches_layout():
    assert kite.mlp_param_count() == omlp.n_params()


def test_forward_and_gradient_match_oracle(ctx):
    n = 64
    p = omlp.init_params(7).astype(np.float32)
    g = np.random.Generator(np.random.PCG64(8))
    X = g.standard_normal((n, omlp.IN)).astype(np.float32)
    Y = np.zeros((n, omlp.OUT), np.float32)
    kite.mlp_forward(ctx, p, X, n, Y)
    Yref, _ = omlp.forward(bf16(p).astype(np.float64), bf16(X))
    assert np.linalg.norm(Y - Yref) <= 2e-2 * np.linalg.norm(Yref)
    # targets far from the outputs so the sign of the residual is the same on both sides
    T = (Yref + np.where(g.random(Yref.shape) < 0.5, -1.0, 1.0) * (0.5 + np.abs(Yref))).astype(np.float32)
    grad = np.zeros(kite.mlp_param_count(), np.float32)
    loss = kite.mlp_gradient(ctx, p, X, T, n, grad)
    gref = omlp.grad(bf16(p).astype(np.float64), bf16(X), T)
    assert abs(loss - omlp.loss(bf16(p).astype(np.float64), bf16(X), T)) <= 1e-2 * loss
    off = 0
    for shp in omlp.shapes():
        k = int(np.prod(shp))
        a, b = grad[off:off + k], gref[off:off + k]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b), shp
        off += k


def midpoint_energies(e_min, e_max, K=1024):
    eps = -1.0 + (2.0 * np.arange(K) + 1.0) / K
    return eps * 0.5 * (e_max - e_min) + 0.5 * (e_max + e_min)


def make_dataset(ctx, n, seed, L=40, M_hi=1024, M_in=128):
    g = np.random.Generator(np.random.PCG64(seed))
    bound = (3 * 2.7 + 0.5 + 2.0) * 1.01  # one energy grid for every sample
    systems, kpms, mus = [], [], []
    for i in range(n):
        systems.append(kite.make_system(kite.HONEYCOMB, L, L, -2.7, 4.0 * g.random(), g.random(),
                                        0.02 * g.random(), int(g.integers(1, 2**62))))
        kpms.append(kite.make_kpm(M_hi, 2, 1, kite.FP32, -bound, bound))
        mus.append(np.zeros(M_hi))
    kite.moments_1d_batched(ctx, systems, kpms, mus)
    E = midpoint_energies(-bound, bound)
    Y = np.zeros((n, 1024), np.float32)
    base = np.zeros((n, 1024))
    for i in range(n):
        rho = np.zeros(1024)
        kite.reconstruct_dos(ctx, mus[i], M_hi, M_hi, kite.KERNEL_JACKSON, 0.0, -bound, bound, E, 1024, rho)
        Y[i] = rho
        kite.reconstruct_dos(ctx, mus[i], M_hi, M_in, kite.KERNEL_JACKSON, 0.0, -bound, bound, E, 1024, rho)
        base[i] = rho
    mu_all = np.array(mus)
    return mu_all, Y, base, E, bound


def test_training_beats_the_plain_low_order_reconstruction(ctx):
    mu, Y, base, E, bound = make_dataset(ctx, 640, seed=5)
    X = mu[:, :128].astype(np.float32)
    scale = (1.0 / np.maximum(X[:512].std(0), 1e-3)).astype(np.float32)
    scale[0] = 1.0
    p = omlp.init_params(11).astype(np.float32)
    curve = np.zeros(60, np.float32)
    kite.mlp_train(ctx, X[:512], Y[:512], 512, p, epochs=60, batch=64, lr=2e-3, weight_decay=1e-4,
                   seed=3, scale=scale, loss_curve=curve)
    assert curve[-1] < 0.5 * curve[0]
    pred = np.zeros((128, 1024), np.float32)
    kite.mlp_forward(ctx, p, np.ascontiguousarray(X[512:]), 128, pred, scale=scale)
    dE = E[1] - E[0]
    l1_net = np.mean(np.sum(np.abs(pred - Y[512:]), 1) * dE)
    l1_base = np.mean(np.sum(np.abs(base[512:] - Y[512:]), 1) * dE)
    print(f"held-out L1: network {l1_net:.4f}, Jackson M=128 {l1_base:.4f}")
    assert l1_net < l1_base
    flags = np.zeros(128, np.int32)
    dev = np.zeros(128)
    kite.learned_gate(ctx, pred, np.ascontiguousarray(mu[512:]), mu.shape[1], 128, 8, -bound, bound,
                      0.05, flags, dev)
    assert np.all(np.isfinite(dev))
