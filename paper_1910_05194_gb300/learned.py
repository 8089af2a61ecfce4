"""Learned density-of-states reconstruction on top of the library's C-ABI.

The paper has no learned component.  Its Sec. 2a notes that the energy resolution of a
Chebyshev (kernel polynomial) reconstruction scales as the inverse number of moments, so a
sharp density of states needs many moments.  This module trains the library's perceptron
(kite_mlp_train) to map the first 128 moments of a system to the density that the Jackson
reconstruction reaches with many more (M_hi) moments, as a residual on the Jackson
reconstruction from the same 128 moments (kite_learned_train, which also computes the input
normalisation on the device).  kite_learned_dos then runs the network, the label-free
consistency gate and, for flagged systems, the plain path (moments at a high order and
their Jackson reconstruction) in one call.

Every step runs in the library's kernels; this file only marshals arrays between calls.

    python -m paper_1910_05194_gb300.learned [--n-train 20000 --n-test 2000 --L 256 ...]

runs the whole workflow (dataset, training, held-out evaluation, gate, wall-time
comparison against the plain FP64 path at equal held-out L1 error) and prints one JSON
line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import (FP32, FP64, HONEYCOMB, KERNEL_JACKSON, MLP_IN, MLP_OUT, Context, learned_dos, learned_train,
               make_kpm, make_system, mlp_param_count, moments_1d, moments_1d_batched, reconstruct_dos)

T_HOP = -2.7


def window(delta_hi: float, W_hi: float, t: float = T_HOP):
    """One energy window for every sample (so every density lives on one grid): the
    Gershgorin enclosure of the widest sample, 3|t| + Delta/2 + W/2, widened by 1%."""
    b = (3.0 * abs(t) + 0.5 * delta_hi + 0.5 * W_hi) * 1.01
    return -b, b


def midpoint_energies(e_min: float, e_max: float, K: int = MLP_OUT) -> np.ndarray:
    """E_j for eps_j = -1 + (2j+1)/K, the grid of the network's outputs."""
    eps = -1.0 + (2.0 * np.arange(K) + 1.0) / K
    return eps * 0.5 * (e_max - e_min) + 0.5 * (e_max + e_min)


def to_systems(specs, t: float = T_HOP):
    return [make_system(HONEYCOMB, s["L"], s["L"], t, s["W"], s["delta"], s["p_vac"], s["seed"])
            for s in specs]


def batched_moments(ctx: Context, systems, M: int, R: int, e_min: float, e_max: float,
                    chunk: int = 2000, doubling: bool = True):
    """mu [n][M] (FP64 accumulation of the FP32 recursion) of every system, many systems per
    persistent launch (kite_moments_1d_batched, with moment doubling by default); returns
    (mu, seconds)."""
    n = len(systems)
    mu = np.zeros((n, M))
    secs = 0.0
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        kpms = [make_kpm(M, R, 1, FP32, e_min, e_max, doubling=doubling) for _ in range(a, b)]
        rows = [mu[i] for i in range(a, b)]
        t0 = time.perf_counter()
        moments_1d_batched(ctx, systems[a:b], kpms, rows)
        secs += time.perf_counter() - t0
    return mu, secs


def jackson_dos(ctx: Context, mu, M_use: int, e_min: float, e_max: float) -> np.ndarray:
    """Jackson reconstruction from the first M_use moments of every row on the midpoint
    grid, per eV (kite_reconstruct_dos), as float32 [n][OUT]."""
    E = midpoint_energies(e_min, e_max)
    out = np.zeros((mu.shape[0], MLP_OUT), np.float32)
    rho = np.zeros(MLP_OUT)
    for i in range(mu.shape[0]):
        reconstruct_dos(ctx, mu[i], mu.shape[1], M_use, KERNEL_JACKSON, 0.0, e_min, e_max, E, MLP_OUT, rho)
        out[i] = rho
    return out


def l1_error(rho, ref, e_min: float, e_max: float) -> np.ndarray:
    """Per-row L1 distance int |rho - ref| dE on the midpoint grid."""
    dE = (e_max - e_min) / MLP_OUT
    return np.sum(np.abs(np.asarray(rho, np.float64) - np.asarray(ref, np.float64)), axis=1) * dE


def train(ctx: Context, X, T, e_min: float, e_max: float, init=None, epochs=200, batch=256, lr=1e-3,
          weight_decay=1e-4, seed=0, head_scale=0.01):
    """kite_learned_train: a model trained on X [n][IN] -> T [n][OUT] as a residual on the
    Jackson prior, with its input normalisation computed on the device; returns
    (model, loss curve)."""
    curve = np.zeros(epochs, np.float32)
    model = learned_train(ctx, np.ascontiguousarray(X, np.float32), np.ascontiguousarray(T, np.float32),
                          X.shape[0], e_min, e_max, epochs=epochs, batch=batch, lr=lr, weight_decay=weight_decay,
                          seed=seed, init=init, head_scale=head_scale, loss_curve=curve)
    return model, curve


def infer(ctx: Context, model, mu, kcheck: int = 16, tol: float = 0.02, M_plain: int = None):
    """kite_learned_dos on the moment rows mu [n][M]: densities [n][OUT] (per eV, midpoint
    grid) from the network, gated; flagged rows fall back to the Jackson reconstruction of the
    row's own first M_plain moments (default: all of them).  tol = inf gives the network
    alone.  Returns (rho, flags, deviation)."""
    mu = np.ascontiguousarray(mu, np.float64)
    n, ld = mu.shape
    rho = np.zeros((n, MLP_OUT), np.float32)
    flags = np.zeros(n, np.int32)
    dev = np.zeros(n)
    learned_dos(ctx, model, mu, ld, n, tol, kcheck, M_plain or ld, rho, flags, dev)
    return rho, flags, dev


def plain_dos(ctx: Context, system, M: int, R: int, e_min: float, e_max: float,
              precision=FP64) -> np.ndarray:
    """The plain path for one system: M moments (kite_moments_1d) and their Jackson
    reconstruction on the midpoint grid."""
    mu = np.zeros(M)
    moments_1d(ctx, system, make_kpm(M, R, 1, precision, e_min, e_max), mu)
    return jackson_dos(ctx, mu[None, :], M, e_min, e_max)[0]


def reconstruct(ctx: Context, systems, model, R: int, e_min: float, e_max: float, M_fallback: int,
                kcheck: int = 16, tol: float = 0.02):
    """The learned path with fallback: MLP_IN FP32 moments per system in one batched launch
    (moment doubling), then kite_learned_dos (network, gate, and for flagged systems the plain
    FP64 path at M_fallback: kite_moments_1d + kite_reconstruct_dos).
    Returns (rho [n][OUT], flags)."""
    mu, _ = batched_moments(ctx, systems, MLP_IN, R, e_min, e_max)
    n = len(systems)
    rho = np.zeros((n, MLP_OUT), np.float32)
    flags = np.zeros(n, np.int32)
    learned_dos(ctx, model, mu, MLP_IN, n, tol, kcheck, M_fallback, rho, flags, systems=systems,
                plain_kpm=make_kpm(M_fallback, R, 1, FP64, e_min, e_max))
    return rho, flags


def noise_floor(ctx: Context, systems, M: int, R: int, e_min: float, e_max: float, targets) -> float:
    """Mean L1 error that the R-vector stochastic estimate carries in the targets themselves:
    for each system the per-vector moments (kite_moments_1d) are split into two halves of R/2
    vectors; the Jackson DOS of the two half-averages differ with twice the standard deviation
    of the R-vector average's error, so half their L1 distance estimates the targets' noise.
    No function of the input moments can predict that noise."""
    if R < 2 or R % 2:
        return float("nan")
    out = []
    for i, s in enumerate(systems):
        mu = np.zeros(M)
        per = np.zeros((R, M, 2))
        moments_1d(ctx, s, make_kpm(M, R, 1, FP32, e_min, e_max), mu, per)
        halves = np.stack([per[:R // 2, :, 0].mean(0), per[R // 2:, :, 0].mean(0)])
        d = jackson_dos(ctx, halves, M, e_min, e_max)
        out.append(0.5 * l1_error(d[:1], d[1:], e_min, e_max)[0])
    return float(np.mean(out))


def run(ctx: Context, n_train=20000, n_test=2000, L=256, M_hi=4096, R=4, epochs=200, batch=256, lr=1e-3,
        chunk=4000, time_sample=200, noise_sample=100, seed=5_000_000):
    """The whole workflow on seeded synthetic systems: dataset (batched FP32 moments with
    doubling at M_hi and their Jackson DOS as targets), training (kite_learned_train),
    held-out L1 of the network against the Jackson reconstruction from the same MLP_IN
    moments and the targets' own noise floor, the plain order M_plain that reaches the
    network's held-out L1, the gate, and the wall time of the learned path against the plain
    FP64 path and the batched FP32 path at M_plain.  Returns a dict of the figures."""
    import synth

    e_min, e_max = window(1.0, 4.0)
    specs = synth.learned_dos_systems(n_train + n_test, seed, L=L)
    systems = to_systems(specs)
    t0 = time.perf_counter()
    mu, t_mom = batched_moments(ctx, systems, M_hi, R, e_min, e_max, chunk)
    T = jackson_dos(ctx, mu, M_hi, e_min, e_max)
    t_data = time.perf_counter() - t0
    ntr = n_train
    X = mu[:, :MLP_IN].astype(np.float32)

    params = synth.mlp_init(seed + 1, head_scale=0.01)
    assert params.size == mlp_param_count()
    t0 = time.perf_counter()
    model, curve = train(ctx, X[:ntr], T[:ntr], e_min, e_max, init=params, epochs=epochs, batch=batch, lr=lr,
                         seed=seed)
    t_train = time.perf_counter() - t0

    test_mu, test_T = mu[ntr:], T[ntr:]
    base = jackson_dos(ctx, test_mu, MLP_IN, e_min, e_max)
    rho, _, _ = infer(ctx, model, test_mu, tol=float("inf"))
    _, flags, dev = infer(ctx, model, test_mu)
    l1_net = l1_error(rho, test_T, e_min, e_max)
    l1_base = l1_error(base, test_T, e_min, e_max)
    # the plain path's order that reaches the network's held-out L1 error
    M_list = [m for m in (128, 160, 192, 256, 320, 384, 448, 512, 640, 768, 1024, 1536, 2048, 3072, 4096)
              if m <= M_hi]
    l1_by_M = {}
    M_plain = None
    for m in M_list:
        l1_by_M[m] = float(np.mean(l1_error(jackson_dos(ctx, test_mu, m, e_min, e_max), test_T, e_min, e_max)))
        if M_plain is None and l1_by_M[m] <= float(np.mean(l1_net)):
            M_plain = m
    floor = noise_floor(ctx, systems[ntr:ntr + noise_sample], M_hi, R, e_min, e_max, test_T)
    # wall time on a held-out sample: learned path (batched FP32 M=128 + network + gate)
    # against the plain FP64 path at M_plain (and the batched FP32 path at M_plain)
    ts = systems[ntr:ntr + time_sample]
    res = {}
    if M_plain is not None:
        # each path runs once untimed on the same systems first (the batched sweep plans and
        # times its team schedule on the first call for a batch of this make-up)
        reconstruct(ctx, ts, model, R, e_min, e_max, M_plain)
        t0 = time.perf_counter()
        _, fl = reconstruct(ctx, ts, model, R, e_min, e_max, M_plain)
        res["learned_s"] = time.perf_counter() - t0
        res["learned_flagged"] = int(np.sum(fl))
        plain_dos(ctx, ts[0], M_plain, R, e_min, e_max)
        t0 = time.perf_counter()
        for s in ts:
            plain_dos(ctx, s, M_plain, R, e_min, e_max)
        res["plain_fp64_s"] = time.perf_counter() - t0
        mu_p, _ = batched_moments(ctx, ts, M_plain, R, e_min, e_max)
        t0 = time.perf_counter()
        mu_p, _ = batched_moments(ctx, ts, M_plain, R, e_min, e_max)
        jackson_dos(ctx, mu_p, M_plain, e_min, e_max)
        res["plain_fp32_batched_doubling_s"] = time.perf_counter() - t0
    model.close()
    out = {
        "workload": f"learned_dos_honeycomb_{L}x{L}_train{n_train}_test{n_test}_Mhi{M_hi}_R{R}",
        "window_eV": [e_min, e_max],
        "dataset_s": t_data, "dataset_moment_s": t_mom,
        "dataset_updates": float(len(systems)) * 2 * L * L * M_hi * R,
        "train_s": t_train, "epochs": epochs, "loss_first": float(curve[0]), "loss_last": float(curve[-1]),
        "heldout_l1_network": float(np.mean(l1_net)), "heldout_l1_jackson128": float(np.mean(l1_base)),
        "heldout_l1_noise_floor": floor, "noise_sample": min(noise_sample, n_test),
        "gain": float(np.mean(l1_base) / np.mean(l1_net)),
        "network_better_fraction": float(np.mean(l1_net < l1_base)),
        "gate_tol": 0.02, "gate_flagged": int(np.sum(flags)), "gate_dev_median": float(np.median(dev)),
        "l1_by_M": l1_by_M, "M_plain_equal_l1": M_plain, "time_sample": len(ts), **res,
    }
    if "learned_s" in res:
        out["speedup_vs_plain_fp64"] = res["plain_fp64_s"] / res["learned_s"]
        out["speedup_vs_batched_fp32"] = res["plain_fp32_batched_doubling_s"] / res["learned_s"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--n-test", type=int, default=2000)
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--M-hi", type=int, default=4096)
    ap.add_argument("--R", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--chunk", type=int, default=4000)
    ap.add_argument("--time-sample", type=int, default=200, help="held-out systems timed on each path")
    ap.add_argument("--noise-sample", type=int, default=100, help="held-out systems for the noise floor")
    ap.add_argument("--seed", type=int, default=5_000_000)
    a = ap.parse_args(argv)
    ctx = Context(0)
    out = run(ctx, a.n_train, a.n_test, a.L, a.M_hi, a.R, a.epochs, a.batch, a.lr, a.chunk, a.time_sample,
              a.noise_sample, a.seed)
    print(json.dumps(out), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
