"""FP64 reference of the learned DOS reconstructor: a multilayer perceptron
IN -> H -> H -> OUT with ReLU activations, mean-absolute-error loss and AdamW.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).  The network is not in
the paper; it maps a short Chebyshev moment vector to the density of states that the
kernel polynomial reconstruction only reaches with many more moments (the paper notes the
resolution scales as the inverse number of moments, Sec. 2a).  Parameters are one flat
FP32/FP64 vector in the order W1[H][IN], b1[H], W2[H][H], b2[H], W3[OUT][H], b3[OUT]
(row-major), the layout the CUDA kernels use.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 128, 512, 1024


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even) via float32, returned as float64: the
    precision in which the kernels store weights and activations.  Used so that decisions
    taken on stored values (the ReLU masks) are taken on the same values on both sides."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def kernel_params(p, n_in=IN, n_hid=HID, n_out=OUT):
    """The parameters as the kernels use them: weights rounded to bfloat16, biases float32."""
    out, off = [], 0
    for s in shapes(n_in, n_hid, n_out):
        k = int(np.prod(s))
        part = np.asarray(p[off:off + k])
        out.append(round_bf16(part) if len(s) == 2 else part.astype(np.float32).astype(np.float64))
        off += k
    return np.concatenate(out)


def midpoint_eps(n_out=OUT):
    """The output grid in the rescaled energy: eps_j = -1 + (2j+1)/n_out."""
    return -1.0 + (2.0 * np.arange(n_out) + 1.0) / n_out


def prior(mu_in, e_min, e_max, n_out=OUT):
    """The residual prior: the Jackson reconstruction (Eq. e8a with the Jackson kernel of
    order len(mu_in)) from the given moments on the midpoint grid, per eV; rows of mu_in."""
    import oracle
    mu_in = np.atleast_2d(np.asarray(mu_in, np.float64))
    m = mu_in.shape[1]
    g = oracle.kernel_jackson(m)
    E = midpoint_eps(n_out) * 0.5 * (e_max - e_min) + 0.5 * (e_max + e_min)
    return np.stack([oracle.dos(row, E, e_min, e_max, g) for row in mu_in])


def shapes(n_in=IN, n_hid=HID, n_out=OUT):
    return [(n_hid, n_in), (n_hid,), (n_hid, n_hid), (n_hid,), (n_out, n_hid), (n_out,)]


def n_params(n_in=IN, n_hid=HID, n_out=OUT):
    return sum(int(np.prod(s)) for s in shapes(n_in, n_hid, n_out))


def unpack(p, n_in=IN, n_hid=HID, n_out=OUT):
    out, off = [], 0
    for s in shapes(n_in, n_hid, n_out):
        k = int(np.prod(s))
        out.append(np.asarray(p[off:off + k], np.float64).reshape(s))
        off += k
    return out


def forward(p, X, n_in=IN, n_hid=HID, n_out=OUT, act_round=None):
    """Returns (Y, cache): Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per row of X.
    act_round (or None) is applied to the hidden activations after the ReLU, modelling the
    precision in which they are stored; the masks below are taken on the stored values."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hid, n_out)
    rnd = (lambda a: a) if act_round is None else act_round
    X = np.asarray(X, np.float64)
    Z1 = X @ W1.T + b1
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = rnd(np.maximum(Z2, 0.0))
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss(p, X, T, n_in=IN, n_hid=HID, n_out=OUT, act_round=None):
    """Mean absolute error over all outputs of all rows."""
    Y, _ = forward(p, X, n_in, n_hid, n_out, act_round)
    return float(np.mean(np.abs(Y - np.asarray(T, np.float64))))


def grad(p, X, T, n_in=IN, n_hid=HID, n_out=OUT, act_round=None, delta_round=None):
    """Analytic gradient of `loss` by the chain rule (sign(0) taken as 0; the activation
    rounding, if any, is passed through as the identity).  delta_round (or None) is applied
    to the back-propagated deltas dY, dZ2 and dZ1, modelling the precision in which they are
    stored between layers; the weight and bias gradients are then exact sums of the stored
    deltas."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hid, n_out)
    Y, (X, Z1, H1, Z2, H2) = forward(p, X, n_in, n_hid, n_out, act_round)
    rd = (lambda a: a) if delta_round is None else delta_round
    dY = rd(np.sign(Y - np.asarray(T, np.float64)) / Y.size)
    dW3 = dY.T @ H2
    db3 = dY.sum(0)
    dH2 = dY @ W3
    dZ2 = rd(dH2 * (H2 > 0))
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(0)
    dH1 = dZ2 @ W2
    dZ1 = rd(dH1 * (H1 > 0))
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(0)
    return np.concatenate([g.ravel() for g in (dW1, db1, dW2, db2, dW3, db3)])


def init_params(seed, n_in=IN, n_hid=HID, n_out=OUT):
    """He-uniform weights, zero biases, drawn from numpy's PCG64."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for s in shapes(n_in, n_hid, n_out):
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[1])
            parts.append(g.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def adamw_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW update (Loshchilov & Hutter): decoupled weight decay on every parameter."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v


def cosine_lr(t, total, lr):
    """Learning rate of optimiser step t (1-based) of `total` steps: a cosine decay from lr
    towards zero, lr (1 + cos(pi (t - 1) / total)) / 2."""
    return lr * 0.5 * (1.0 + np.cos(np.pi * (t - 1) / max(1, total)))
