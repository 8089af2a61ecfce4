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


def forward(p, X, n_in=IN, n_hid=HID, n_out=OUT):
    """Returns (Y, cache): Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per row of X."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hid, n_out)
    X = np.asarray(X, np.float64)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss(p, X, T, n_in=IN, n_hid=HID, n_out=OUT):
    """Mean absolute error over all outputs of all rows."""
    Y, _ = forward(p, X, n_in, n_hid, n_out)
    return float(np.mean(np.abs(Y - np.asarray(T, np.float64))))


def grad(p, X, T, n_in=IN, n_hid=HID, n_out=OUT):
    """Analytic gradient of `loss` by the chain rule (sign(0) taken as 0)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hid, n_out)
    Y, (X, Z1, H1, Z2, H2) = forward(p, X, n_in, n_hid, n_out)
    dY = np.sign(Y - np.asarray(T, np.float64)) / Y.size
    dW3 = dY.T @ H2
    db3 = dY.sum(0)
    dH2 = dY @ W3
    dZ2 = dH2 * (Z2 > 0)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
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
