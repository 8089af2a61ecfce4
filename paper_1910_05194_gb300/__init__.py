"""GB300-native stochastic Chebyshev (kernel polynomial) moments of lattice Green's
functions, after KITE (arXiv:1910.05194).

This module is a thin ctypes binding of ``libkite_gb.so``: it marshals structs and
pointers (numpy arrays, torch tensors or raw addresses) and calls the C ABI declared
in ``include/kite_gb.h``.  Every step of the computation runs in the library's CUDA
kernels; there is no Python or CPU fallback.  If the library has not been built, the
first call raises :class:`KiteError` telling how to build it.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkite_gb.so")

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_BOUNDS, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
HONEYCOMB, SQUARE = 0, 1
DISORDER_UNIFORM, DISORDER_GAUSSIAN = 0, 1
FP32, FP64 = 0, 1
KERNEL_NONE, KERNEL_JACKSON, KERNEL_LORENTZ = 0, 1, 2
DIR_X, DIR_Y = 0, 1

EXPORTED = ("kite_create", "kite_destroy", "kite_set_stream", "kite_status_string",
            "kite_last_error", "kite_bounds", "kite_moments_1d", "kite_reconstruct_dos",
            "kite_debug_stall_once", "kite_inner_products", "kite_moments_2d", "kite_reconstruct_green",
            "kite_reconstruct_sigma", "kite_moments_1d_static", "kite_moments_1d_batched",
            "kite_mlp_param_count", "kite_mlp_train", "kite_mlp_forward", "kite_mlp_gradient",
            "kite_learned_gate", "kite_spectral_k", "kite_ldos", "kite_propagate",
            "kite_evolution_coeffs", "kite_flux_nearest", "kite_reconstruct_sigma_dc",
            "kite_reconstruct_sigma_dc_bastin", "kite_mlp_adamw_step", "kite_learned_train",
            "kite_learned_dos", "kite_model_export", "kite_model_import", "kite_model_destroy")
MLP_IN, MLP_HIDDEN, MLP_OUT = 128, 512, 1024


class KiteError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"kite status {status}: {detail}")


class System(ctypes.Structure):
    """``kite_system``: honeycomb/square lattice with disorder, periodic or open."""
    _fields_ = [("lattice", ctypes.c_int32), ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
                ("disorder", ctypes.c_int32), ("t", ctypes.c_double), ("W", ctypes.c_double),
                ("delta", ctypes.c_double), ("p_vac", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("flux", ctypes.c_double), ("open_x", ctypes.c_int32), ("open_y", ctypes.c_int32)]


class KPM(ctypes.Structure):
    """``kite_kpm``: expansion parameters."""
    _fields_ = [("M", ctypes.c_int32), ("R", ctypes.c_int32), ("S", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double), ("r0", ctypes.c_void_p), ("r_last", ctypes.c_void_p),
                ("doubling", ctypes.c_int32), ("real_vectors", ctypes.c_int32)]


class Stats(ctypes.Structure):
    """``kite_stats``: per-call statistics."""
    _fields_ = [("seconds", ctypes.c_double), ("updates", ctypes.c_double),
                ("bytes_moved", ctypes.c_double), ("gbps", ctypes.c_double),
                ("max_abs_imag", ctypes.c_double), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double), ("n_eff", ctypes.c_int64), ("grid", ctypes.c_int32),
                ("block", ctypes.c_int32), ("step_seconds", ctypes.c_double),
                ("step_launches", ctypes.c_int64), ("step_bytes", ctypes.c_double),
                ("gemm_seconds", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("ring_stages", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("steps_per_pass", ctypes.c_int32), ("cluster_ctas", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PRIOR_NONE, PRIOR_JACKSON = 0, 1


class MLPPrior(ctypes.Structure):
    """``kite_mlp_prior``."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double)]


class MLPTrainCfg(ctypes.Structure):
    """``kite_mlp_train_cfg``."""
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("seed", ctypes.c_uint64)]


class LearnedCfg(ctypes.Structure):
    """``kite_learned_cfg``."""
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("seed", ctypes.c_uint64), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double), ("init", ctypes.c_void_p), ("head_scale", ctypes.c_double)]


def make_system(lattice=HONEYCOMB, Lx=64, Ly=64, t=-2.7, W=0.0, delta=0.0, p_vac=0.0, seed=1,
                disorder=0, flux=0.0, open_x=0, open_y=0):
    """W: width of uniform disorder in [-W/2, W/2] (disorder=DISORDER_UNIFORM) or standard
    deviation of Gaussian disorder (disorder=DISORDER_GAUSSIAN); flux: perpendicular
    magnetic flux quanta per unit cell (see flux_nearest); open_x / open_y: open
    boundaries along a1 / a2 (the bonds that wrap around the torus are absent)."""
    return System(int(lattice), int(Lx), int(Ly), int(disorder), float(t), float(W), float(delta),
                  float(p_vac), int(seed), float(flux), int(bool(open_x)), int(bool(open_y)))


def make_kpm(M, R=1, S=1, precision=FP32, e_min=0.0, e_max=0.0, r0=None, r_last=None,
             doubling=False, real_vectors=False):
    return KPM(int(M), int(R), int(S), int(precision), float(e_min), float(e_max),
               _addr(r0), _addr(r_last), int(bool(doubling)), int(bool(real_vectors)))


_LOCK = threading.Lock()
_LIB = None


def lib():
    """The loaded ``libkite_gb.so`` (raises KiteError if it was never built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise KiteError(ERR_UNSUPPORTED,
                                f"{LIB_PATH} is missing; build it with "
                                "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            P, vp, i32, d = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.kite_create.argtypes = [P(vp), i32, vp]
            L.kite_create.restype = i32
            L.kite_destroy.argtypes = [vp]
            L.kite_destroy.restype = None
            L.kite_set_stream.argtypes = [vp, vp]
            L.kite_set_stream.restype = i32
            L.kite_status_string.argtypes = [i32]
            L.kite_status_string.restype = ctypes.c_char_p
            L.kite_last_error.argtypes = [vp]
            L.kite_last_error.restype = ctypes.c_char_p
            L.kite_bounds.argtypes = [P(System), P(d), P(d)]
            L.kite_bounds.restype = i32
            L.kite_flux_nearest.argtypes = [P(System), d, P(d)]
            L.kite_flux_nearest.restype = i32
            L.kite_moments_1d.argtypes = [vp, P(System), P(KPM), vp, vp, P(Stats)]
            L.kite_moments_1d.restype = i32
            L.kite_reconstruct_dos.argtypes = [vp, vp, i32, i32, i32, d, d, d, vp, i32, vp]
            L.kite_reconstruct_dos.restype = i32
            L.kite_reconstruct_sigma.argtypes = [vp, vp, i32, i32, i32, i32, d, d, d, d, d, vp,
                                                 i32, i32, vp]
            L.kite_reconstruct_sigma.restype = i32
            L.kite_reconstruct_sigma_dc.argtypes = [vp, vp, i32, i32, i32, i32, d, d, d, vp, i32, vp]
            L.kite_reconstruct_sigma_dc.restype = i32
            L.kite_reconstruct_sigma_dc_bastin.argtypes = [vp, vp, i32, i32, i32, i32, d, d, d, d, d, vp, i32,
                                                           i32, vp]
            L.kite_reconstruct_sigma_dc_bastin.restype = i32
            L.kite_moments_1d_static.argtypes = [P(System), P(KPM), vp, vp, ctypes.c_char_p, i32]
            L.kite_moments_1d_static.restype = i32
            L.kite_moments_1d_batched.argtypes = [vp, i32, P(System), P(KPM), P(vp), P(Stats)]
            L.kite_moments_1d_batched.restype = i32
            L.kite_mlp_param_count.argtypes = []
            L.kite_mlp_param_count.restype = ctypes.c_int64
            L.kite_mlp_train.argtypes = [vp, vp, vp, i32, vp, vp, P(MLPTrainCfg), vp, vp, P(MLPPrior)]
            L.kite_mlp_train.restype = i32
            L.kite_mlp_forward.argtypes = [vp, vp, vp, i32, vp, vp, vp, P(MLPPrior)]
            L.kite_mlp_forward.restype = i32
            L.kite_mlp_gradient.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, P(d)]
            L.kite_mlp_gradient.restype = i32
            L.kite_learned_gate.argtypes = [vp, vp, vp, i32, i32, i32, d, d, d, vp, vp]
            L.kite_learned_gate.restype = i32
            L.kite_mlp_adamw_step.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int64, i32, i32, d, d]
            L.kite_mlp_adamw_step.restype = i32
            L.kite_learned_train.argtypes = [vp, vp, vp, i32, P(LearnedCfg), P(vp), vp]
            L.kite_learned_train.restype = i32
            L.kite_learned_dos.argtypes = [vp, vp, vp, i32, i32, d, i32, i32, vp, P(KPM), vp, vp, vp]
            L.kite_learned_dos.restype = i32
            L.kite_model_export.argtypes = [vp, vp, vp, vp, vp]
            L.kite_model_export.restype = i32
            L.kite_model_import.argtypes = [vp, vp, vp, vp, d, d, P(vp)]
            L.kite_model_import.restype = i32
            L.kite_model_destroy.argtypes = [vp]
            L.kite_model_destroy.restype = None
            L.kite_moments_2d.argtypes = [vp, P(System), P(KPM), i32, i32, vp, P(Stats)]
            L.kite_moments_2d.restype = i32
            L.kite_reconstruct_green.argtypes = [vp, vp, i32, i32, i32, d, d, d, d, vp, i32, vp, vp]
            L.kite_reconstruct_green.restype = i32
            L.kite_spectral_k.argtypes = [vp, P(System), P(KPM), vp, i32, vp, vp, P(Stats)]
            L.kite_spectral_k.restype = i32
            L.kite_ldos.argtypes = [vp, P(System), P(KPM), vp, i32, vp, P(Stats)]
            L.kite_ldos.restype = i32
            L.kite_propagate.argtypes = [vp, P(System), P(KPM), d, i32, vp, vp, P(Stats)]
            L.kite_propagate.restype = i32
            L.kite_evolution_coeffs.argtypes = [i32, d, d, d, vp]
            L.kite_evolution_coeffs.restype = i32
            L.kite_inner_products.argtypes = [vp, vp, vp, i32, i32, ctypes.c_int64, d, vp, i32, i32, i32]
            L.kite_inner_products.restype = i32
            L.kite_debug_stall_once.argtypes = [vp, i32]
            L.kite_debug_stall_once.restype = i32
            _LIB = L
    return _LIB


def _addr(x):
    """Device/host address of a torch tensor, numpy array or raw int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy.ndarray
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Context:
    """A ``kite_ctx``: one device, one stream, reusable work buffers."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        rc = lib().kite_create(ctypes.byref(self._h), int(device), _stream_handle(stream))
        if rc != OK:
            raise KiteError(rc, lib().kite_status_string(rc).decode())
        self.device = device

    @property
    def handle(self):
        return self._h

    def check(self, rc: int):
        if rc != OK:
            detail = lib().kite_last_error(self._h).decode() or lib().kite_status_string(rc).decode()
            raise KiteError(rc, detail)

    def set_stream(self, stream):
        self.check(lib().kite_set_stream(self._h, _stream_handle(stream)))

    def close(self):
        if self._h:
            lib().kite_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def flux_nearest(system: System, flux: float) -> float:
    """kite_flux_nearest: the admissible flux per unit cell closest to `flux`."""
    out = ctypes.c_double()
    rc = lib().kite_flux_nearest(ctypes.byref(system), ctypes.c_double(flux), ctypes.byref(out))
    if rc != OK:
        raise KiteError(rc, "kite_flux_nearest")
    return out.value


def reconstruct_sigma_dc(ctx: Context, mu_nm, M_avail: int, M_use: int, lattice: int, kernel: int,
                         param: float, e_min: float, e_max: float, E, K: int, sigma):
    """kite_reconstruct_sigma_dc: T = 0 longitudinal DC conductivity (e^2/hbar per spin)
    at the Fermi energies E from the 2D moments mu_nm ([M_avail][M_avail] complex)."""
    ctx.check(lib().kite_reconstruct_sigma_dc(ctx.handle, _addr(mu_nm), int(M_avail), int(M_use), int(lattice),
                                              int(kernel), float(param), float(e_min), float(e_max), _addr(E),
                                              int(K), _addr(sigma)))


def reconstruct_sigma_dc_bastin(ctx: Context, mu_nm, M_avail: int, M_use: int, lattice: int, kernel: int,
                                param: float, e_min: float, e_max: float, eta: float, kT: float, E_F, K: int,
                                sigma, n_quad: int = 0):
    """kite_reconstruct_sigma_dc_bastin: DC sigma_ab (e^2/hbar per spin, Fermi sea included:
    the Hall conductivity for a != b) at the Fermi energies E_F from the 2D moments."""
    ctx.check(lib().kite_reconstruct_sigma_dc_bastin(ctx.handle, _addr(mu_nm), int(M_avail), int(M_use),
                                                     int(lattice), int(kernel), float(param), float(e_min),
                                                     float(e_max), float(eta), float(kT), _addr(E_F), int(K),
                                                     int(n_quad), _addr(sigma)))


def bounds(system: System):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = lib().kite_bounds(ctypes.byref(system), ctypes.byref(lo), ctypes.byref(hi))
    if rc != OK:
        raise KiteError(rc, "kite_bounds")
    return lo.value, hi.value


def moments_1d(ctx: Context, system: System, kpm: KPM, mu, mu_per_vec=None) -> Stats:
    """kite_moments_1d: mu[M] (FP64, host or device), optional mu_per_vec[S*R][M][2]."""
    st = Stats()
    ctx.check(lib().kite_moments_1d(ctx.handle, ctypes.byref(system), ctypes.byref(kpm),
                                    _addr(mu), _addr(mu_per_vec), ctypes.byref(st)))
    return st


def reconstruct_dos(ctx: Context, mu, M_avail: int, M_use: int, kernel: int, param: float,
                    e_min: float, e_max: float, E, K: int, rho):
    """kite_reconstruct_dos: rho[K] per orbital per eV from raw moments (FP64, GPU)."""
    ctx.check(lib().kite_reconstruct_dos(ctx.handle, _addr(mu), int(M_avail), int(M_use),
                                         int(kernel), float(param), float(e_min), float(e_max),
                                         _addr(E), int(K), _addr(rho)))


def debug_stall_once(ctx: Context, enable: bool = True):
    """Test hook: the next kite_moments_1d call's first step times out (KITE_ERR_TIMEOUT)."""
    ctx.check(lib().kite_debug_stall_once(ctx.handle, int(bool(enable))))


def reconstruct_green(ctx: Context, mu, M_avail: int, M_use: int, kernel: int, param: float,
                      e_min: float, e_max: float, eta: float, E, K: int, G=None, rho=None):
    """kite_reconstruct_green: G[K] complex (1/eV) and/or rho[K] = -Im G/pi at E + i eta."""
    ctx.check(lib().kite_reconstruct_green(ctx.handle, _addr(mu), int(M_avail), int(M_use), int(kernel),
                                           float(param), float(e_min), float(e_max), float(eta), _addr(E),
                                           int(K), _addr(G), _addr(rho)))


def spectral_k(ctx: Context, system: System, kpm: KPM, k, nk: int, mu, weights=None) -> Stats:
    """kite_spectral_k: mu[nk][M] complex FP64 moments of the plane-wave start vectors at the
    k-points k[nk][2] (1/a), optional complex orbital weights[SORB] (interleaved)."""
    st = Stats()
    ctx.check(lib().kite_spectral_k(ctx.handle, ctypes.byref(system), ctypes.byref(kpm), _addr(k), int(nk),
                                    _addr(weights), _addr(mu), ctypes.byref(st)))
    return st


def ldos(ctx: Context, system: System, kpm: KPM, orbitals, n: int, mu) -> Stats:
    """kite_ldos: mu[n][M] complex FP64 moments <i|T_n|i> of the orbitals (int64 [n])."""
    st = Stats()
    ctx.check(lib().kite_ldos(ctx.handle, ctypes.byref(system), ctypes.byref(kpm), _addr(orbitals), int(n),
                              _addr(mu), ctypes.byref(st)))
    return st


def propagate(ctx: Context, system: System, kpm: KPM, dt: float, nsteps: int, psi, norms=None) -> Stats:
    """kite_propagate: psi [R][N][2] FP64 (host or device) evolved in place by nsteps steps of
    exp(-i H dt); norms [nsteps][R] (optional)."""
    st = Stats()
    ctx.check(lib().kite_propagate(ctx.handle, ctypes.byref(system), ctypes.byref(kpm), float(dt), int(nsteps),
                                   _addr(psi), _addr(norms), ctypes.byref(st)))
    return st


def evolution_coeffs(M: int, dt: float, e_min: float, e_max: float):
    """kite_evolution_coeffs (host): the propagator's Chebyshev coefficients, complex [M]."""
    import numpy as _np
    c = _np.zeros((int(M), 2))
    rc = lib().kite_evolution_coeffs(int(M), float(dt), float(e_min), float(e_max), _addr(c))
    if rc != 0:
        raise KiteError(rc, "kite_evolution_coeffs")
    return c[:, 0] + 1j * c[:, 1]


def inner_products(ctx: Context, A, B, M: int, M2: int, N: int, scale: float, C, sub_k: int = 0,
                   products: int = 0, fold: int = 0):
    """kite_inner_products: C[n][m] = scale * sum_i conj(A[n][i]) B[m][i] (split-BF16
    tensor cores, FP64 output).  A [M][N], B [M2][N] complex64; C [M][M2] complex128."""
    ctx.check(lib().kite_inner_products(ctx.handle, _addr(A), _addr(B), int(M), int(M2), int(N),
                                        float(scale), _addr(C), int(sub_k), int(products), int(fold)))


def moments_2d(ctx: Context, system: System, kpm: KPM, mu_nm, alpha: int = 0, beta: int = 0) -> Stats:
    """kite_moments_2d: mu_nm[M][M] complex FP64 (host or device) for the velocity
    directions alpha, beta (DIR_X = 0, DIR_Y = 1)."""
    st = Stats()
    ctx.check(lib().kite_moments_2d(ctx.handle, ctypes.byref(system), ctypes.byref(kpm), int(alpha),
                                    int(beta), _addr(mu_nm), ctypes.byref(st)))
    return st


def reconstruct_sigma(ctx: Context, mu_nm, M_avail: int, M_use: int, lattice: int, kernel: int,
                      e_min: float, e_max: float, E_F: float, kT: float, eta: float, omega,
                      K: int, sigma, n_quad: int = 0):
    """kite_reconstruct_sigma: sigma_xx[K] (complex FP64, units e^2/hbar) from mu_nm."""
    ctx.check(lib().kite_reconstruct_sigma(ctx.handle, _addr(mu_nm), int(M_avail), int(M_use),
                                           int(lattice), int(kernel), float(e_min), float(e_max),
                                           float(E_F), float(kT), float(eta), _addr(omega), int(K),
                                           int(n_quad), _addr(sigma)))


def moments_1d_static(system: System, kpm: KPM, mu, stream=None):
    """kite_moments_1d_static: the 1D moments without any device allocation (fixed 32 MiB
    array per GPU, no context).  For callers that cannot allocate at call time."""
    err = ctypes.create_string_buffer(256)
    rc = lib().kite_moments_1d_static(ctypes.byref(system), ctypes.byref(kpm), _addr(mu),
                                      _stream_handle(stream), err, 256)
    if rc != OK:
        raise KiteError(rc, err.value.decode() or lib().kite_status_string(rc).decode())


def moments_1d_batched(ctx: Context, systems, kpms, mus) -> Stats:
    """kite_moments_1d_batched: one persistent graph launch for many systems.
    systems/kpms: sequences of System/KPM; mus: sequence of [M_i] FP64 buffers."""
    n = len(systems)
    sa = (System * n)(*systems)
    ka = (KPM * n)(*kpms)
    pa = (ctypes.c_void_p * n)(*[_addr(m) for m in mus])
    st = Stats()
    ctx.check(lib().kite_moments_1d_batched(ctx.handle, n, sa, ka, pa, ctypes.byref(st)))
    return st


def jackson_prior(e_min: float, e_max: float) -> MLPPrior:
    """The residual prior of kite_mlp_train / kite_mlp_forward on the window [e_min, e_max]."""
    return MLPPrior(PRIOR_JACKSON, 0, float(e_min), float(e_max))


def _prior_ref(prior):
    return ctypes.byref(prior) if prior is not None else None


def mlp_param_count() -> int:
    return int(lib().kite_mlp_param_count())


def mlp_train(ctx: Context, X, T, n: int, params, epochs=50, batch=256, lr=1e-3, weight_decay=1e-4,
              seed=0, scale=None, loss_curve=None, prior=None, shift=None):
    """kite_mlp_train: trains `params` (FP32 [P]) in place on X [n][IN] -> T [n][OUT]."""
    cfg = MLPTrainCfg(int(epochs), int(batch), float(lr), float(weight_decay), int(seed))
    ctx.check(lib().kite_mlp_train(ctx.handle, _addr(X), _addr(T), int(n), _addr(shift), _addr(scale),
                                   ctypes.byref(cfg), _addr(params), _addr(loss_curve),
                                   _prior_ref(prior)))


def mlp_forward(ctx: Context, params, X, n: int, Y, scale=None, prior=None, shift=None):
    ctx.check(lib().kite_mlp_forward(ctx.handle, _addr(params), _addr(X), int(n), _addr(shift), _addr(scale),
                                     _addr(Y), _prior_ref(prior)))


def mlp_gradient(ctx: Context, params, X, T, n: int, grad, scale=None, shift=None) -> float:
    loss = ctypes.c_double()
    ctx.check(lib().kite_mlp_gradient(ctx.handle, _addr(params), _addr(X), _addr(T), int(n),
                                      _addr(shift), _addr(scale), _addr(grad), ctypes.byref(loss)))
    return loss.value


def learned_gate(ctx: Context, rho, mu, mu_ld: int, n: int, kcheck: int, e_min: float, e_max: float,
                 tol: float, flags, deviation=None):
    ctx.check(lib().kite_learned_gate(ctx.handle, _addr(rho), _addr(mu), int(mu_ld), int(n), int(kcheck),
                                      float(e_min), float(e_max), float(tol), _addr(flags),
                                      _addr(deviation)))


def mlp_adamw_step(ctx: Context, params, grad, m, v, n: int, t: int, total: int, lr: float,
                   weight_decay: float):
    """kite_mlp_adamw_step: optimiser step t of `total` (cosine schedule from lr) on FP32
    params, m, v [n] in place, with the gradient grad [n]."""
    ctx.check(lib().kite_mlp_adamw_step(ctx.handle, _addr(params), _addr(grad), _addr(m), _addr(v), int(n),
                                        int(t), int(total), float(lr), float(weight_decay)))


class Model:
    """A ``kite_model``: a trained learned reconstructor owned by the library."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def export(self):
        """(params [P], shift [IN], scale [IN], (e_min, e_max)) copied out of the model."""
        import numpy as _np
        p = _np.zeros(mlp_param_count(), _np.float32)
        sh = _np.zeros(MLP_IN, _np.float32)
        sc = _np.zeros(MLP_IN, _np.float32)
        w = _np.zeros(2)
        rc = lib().kite_model_export(self._h, _addr(p), _addr(sh), _addr(sc), _addr(w))
        if rc != OK:
            raise KiteError(rc, "kite_model_export")
        return p, sh, sc, (float(w[0]), float(w[1]))

    def close(self):
        if self._h:
            lib().kite_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def learned_train(ctx: Context, X, Y, n: int, e_min: float, e_max: float, epochs=200, batch=256, lr=1e-3,
                  weight_decay=1e-4, seed=0, init=None, head_scale=0.0, loss_curve=None) -> Model:
    """kite_learned_train: a model trained on X [n][IN] -> Y [n][OUT] (density per eV on the
    midpoint grid of [e_min, e_max]); init = initial parameters or None (drawn on the device)."""
    cfg = LearnedCfg(int(epochs), int(batch), float(lr), float(weight_decay), int(seed), float(e_min),
                     float(e_max), _addr(init), float(head_scale))
    h = ctypes.c_void_p()
    ctx.check(lib().kite_learned_train(ctx.handle, _addr(X), _addr(Y), int(n), ctypes.byref(cfg), ctypes.byref(h),
                                       _addr(loss_curve)))
    return Model(h)


def model_import(ctx: Context, params, e_min: float, e_max: float, shift=None, scale=None) -> Model:
    """kite_model_import: a model from saved parameters, normalisation and window."""
    h = ctypes.c_void_p()
    ctx.check(lib().kite_model_import(ctx.handle, _addr(params), _addr(shift), _addr(scale), float(e_min),
                                      float(e_max), ctypes.byref(h)))
    return Model(h)


def learned_dos(ctx: Context, model: Model, mu, mu_ld: int, n: int, gate_tol: float, kcheck: int, M_plain: int,
                rho, fell_back, deviation=None, systems=None, plain_kpm: KPM = None):
    """kite_learned_dos: network + consistency gate + plain fallback in one call.
    mu [n][mu_ld] FP64; rho [n][OUT] FP32; fell_back [n] int32; systems: sequence of System
    (the fallback reruns their moments with plain_kpm at M_plain) or None (the fallback uses
    mu's own first M_plain moments)."""
    sa = None
    if systems is not None:
        sa = (System * len(systems))(*systems)
    ctx.check(lib().kite_learned_dos(ctx.handle, model.handle, _addr(mu), int(mu_ld), int(n), float(gate_tol),
                                     int(kcheck), int(M_plain), sa, ctypes.byref(plain_kpm) if plain_kpm else None,
                                     _addr(rho), _addr(fell_back), _addr(deviation)))
