"""FP64 CPU oracle for the stochastic Chebyshev moments of KITE (arXiv:1910.05194).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library and its Python binding never import it, and it never
imports them: the two sides meet only through the definitions in the paper.

The arithmetic lives in ``kite_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module builds it with gcc on first use and wraps it
with numpy-friendly functions.  Section/equation citations are in the C source.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kite_oracle.c")
_HDR = os.path.join(_HERE, "kite_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None

HONEYCOMB = 0
SQUARE = 1


def _source_hash() -> str:
    h = hashlib.sha1()
    for p in (_SRC, _HDR):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle-<hash>.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, f"liboracle-{_source_hash()}.so")
    if os.path.exists(out) and not force:
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class System(ctypes.Structure):
    """Mirror of ``orc_system``: a honeycomb or square lattice with disorder, periodic or
    with open boundaries."""
    _fields_ = [("lattice", ctypes.c_int32), ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
                ("disorder", ctypes.c_int32), ("t", ctypes.c_double), ("W", ctypes.c_double),
                ("delta", ctypes.c_double), ("p_vac", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("flux", ctypes.c_double), ("open_x", ctypes.c_int32),
                ("open_y", ctypes.c_int32)]


UNIFORM, GAUSSIAN = 0, 1


def make_system(lattice=HONEYCOMB, Lx=8, Ly=8, t=-2.7, W=0.0, delta=0.0, p_vac=0.0, seed=1,
                disorder=UNIFORM, flux=0.0, open_x=0, open_y=0):
    """W is the width of uniform disorder in [-W/2, W/2], or the standard deviation of
    Gaussian disorder (disorder=GAUSSIAN); flux is the perpendicular magnetic flux per unit
    cell in flux quanta (Landau gauge: flux * Ly even on the honeycomb, integer on the
    square lattice, when y is periodic); open_x / open_y drop the bonds that wrap around
    the torus along a1 / a2 (open boundaries)."""
    return System(int(lattice), int(Lx), int(Ly), int(disorder), float(t), float(W), float(delta),
                  float(p_vac), int(seed), float(flux), int(bool(open_x)), int(bool(open_y)))


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            vp = ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            L.orc_norb.argtypes = [P(System)]
            L.orc_norb.restype = i64
            L.orc_neighbours.argtypes = [P(System), i64, P(i64)]
            L.orc_neighbours.restype = i32
            L.orc_bounds_auto.argtypes = [P(System), P(d), P(d)]
            L.orc_disorder.argtypes = [P(System), i32, vp, vp]
            L.orc_random_phase.argtypes = [P(System), i32, i32, vp, vp]
            L.orc_random_real.argtypes = [P(System), i32, i32, vp, vp]
            L.orc_moments_1d.argtypes = [P(System), i32, i32, i32, d, d, vp, vp, i32]
            L.orc_moments_1d.restype = i32
            L.orc_replica_1d.argtypes = [P(System), i32, i32, i32, d, d, i32, vp, vp, vp, i32]
            L.orc_replica_1d.restype = i32
            L.orc_replica_window.argtypes = [P(System), i32, i32, i32, d, d, i32, i32, i32, i32, vp]
            L.orc_replica_window.restype = i32
            L.orc_velocity_x.argtypes = [P(System), vp, d, vp, vp]
            L.orc_velocity.argtypes = [P(System), vp, d, i32, vp, vp]
            L.orc_moments_2d.argtypes = [P(System), i32, i32, i32, d, d, vp, vp, vp, vp, i32, i32, i32]
            L.orc_moments_2d.restype = i32
            L.orc_moments_2d_panels.argtypes = [P(System), i32, i32, i32, d, d, vp, i32, vp, i32, i32, i32, vp, vp,
                                                i32]
            L.orc_moments_2d_panels.restype = i32
            L.orc_chebyshev_sum.argtypes = [P(System), i32, d, d, i32, vp, vp, vp]
            L.orc_chebyshev_sum.restype = i32
            L.orc_kernel_jackson.argtypes = [i32, vp]
            L.orc_kernel_lorentz.argtypes = [i32, d, vp]
            L.orc_dos.argtypes = [vp, i32, vp, d, d, vp, i32, vp]
            L.orc_cpgf_coeff.argtypes = [i32, d, d, i32, P(d), P(d)]
            _LIB = L
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def norb(sys: System) -> int:
    return int(lib().orc_norb(ctypes.byref(sys)))


def neighbours(sys: System, o: int):
    """Neighbour orbitals of o (bonds across an open boundary left out)."""
    nb = (ctypes.c_int64 * 4)()
    z = lib().orc_neighbours(ctypes.byref(sys), int(o), nb)
    return [int(nb[k]) for k in range(z) if nb[k] >= 0]


def bounds_auto(sys: System):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    lib().orc_bounds_auto(ctypes.byref(sys), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def disorder(sys: System, realisation: int = 0):
    """Raw on-site energies V (eV) and the vacancy mask of one realisation."""
    n = norb(sys)
    V = np.empty(n, np.float64)
    vac = np.empty(n, np.uint8)
    lib().orc_disorder(ctypes.byref(sys), int(realisation), _ptr(V), _ptr(vac))
    return V, vac


def random_phase(sys: System, R: int, realisation: int = 0):
    """Random-phase start vectors [R][N] complex128 (zero on vacancies)."""
    _, vac = disorder(sys, realisation)
    n = norb(sys)
    out = np.empty((R, n, 2), np.float64)
    lib().orc_random_phase(ctypes.byref(sys), int(realisation), int(R), _ptr(vac), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def random_real(sys: System, R: int, realisation: int = 0):
    """Real random-sign start vectors [R][N] (+-1, zero on vacancies) as complex128."""
    _, vac = disorder(sys, realisation)
    n = norb(sys)
    out = np.empty((R, n, 2), np.float64)
    lib().orc_random_real(ctypes.byref(sys), int(realisation), int(R), _ptr(vac), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def orbital_positions(sys: System):
    """Positions (x, y) of every orbital in units of the lattice constant: honeycomb cell
    (x, y) at x a1 + y a2 with a1 = (1, 0), a2 = (1/2, sqrt(3)/2), A at (0, -a_cc/2) and B
    at (0, +a_cc/2), a_cc = 1/sqrt(3) (the paper's lattice set-up listing); square (x, y)."""
    n = norb(sys)
    o = np.arange(n)
    if sys.lattice == HONEYCOMB:
        cell, s = o // 2, o % 2
        x, y = cell % sys.Lx, cell // sys.Lx
        acc = 1.0 / np.sqrt(3.0)
        return np.stack([x + 0.5 * y, np.sqrt(3.0) / 2.0 * y + np.where(s == 0, -0.5, 0.5) * acc], -1)
    return np.stack([o % sys.Lx, o // sys.Lx], -1).astype(np.float64)


def bloch_vector(sys: System, k, weights, realisation: int = 0):
    """|k> = sum_alpha w_alpha sum_i exp(i k.R_i^alpha) |i, alpha> (Sec. "Spectral
    functions"), zero on vacant orbitals; k = (kx, ky) in 1/a, weights[alpha] complex."""
    R = orbital_positions(sys)
    _, vac = disorder(sys, realisation)
    n = norb(sys)
    sorb = 2 if sys.lattice == HONEYCOMB else 1
    w = np.asarray(weights, np.complex128)[np.arange(n) % sorb]
    v = w * np.exp(1j * (R @ np.asarray(k, np.float64)))
    v[vac != 0] = 0.0
    return v


def _as_r0(r0, R, n):
    if r0 is None:
        return None
    a = np.ascontiguousarray(np.asarray(r0, np.complex128).reshape(R, n))
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1))


def _bounds(sys, e_min, e_max):
    if e_min is None or e_max is None:
        return bounds_auto(sys)
    return float(e_min), float(e_max)


def moments_1d(sys: System, M: int, R: int, realisation: int = 0, e_min=None, e_max=None,
               r0=None, threads: int = 0):
    """Per-vector complex moments mu[r][n] = <r0|T_n(H~)|r0>/N_eff, plain FP64."""
    n = norb(sys)
    lo, hi = _bounds(sys, e_min, e_max)
    r0a = _as_r0(r0, R, n)
    mu = np.empty((R, M, 2), np.float64)
    rc = lib().orc_moments_1d(ctypes.byref(sys), int(realisation), int(M), int(R), lo, hi,
                              _ptr(r0a), _ptr(mu), int(threads))
    if rc != 0:
        raise ValueError(f"orc_moments_1d failed ({rc})")
    return mu[..., 0] + 1j * mu[..., 1]


def replica_1d(sys: System, M: int, R: int, precision: int, realisation: int = 0, e_min=None,
               e_max=None, r0=None, want_last: bool = False, threads: int = 0):
    """Fixed-rounding replica of the recursion (precision 0 = FP32, 1 = FP64).

    Returns (mu[r][n] complex, last) where ``last`` is None or [R][2][N] complex of the
    working precision holding (r_{M-2}, r_{M-1})."""
    n = norb(sys)
    lo, hi = _bounds(sys, e_min, e_max)
    r0a = _as_r0(r0, R, n)
    mu = np.empty((R, M, 2), np.float64)
    dt = np.float32 if precision == 0 else np.float64
    last = np.empty((R, 2, n, 2), dt) if want_last else None
    rc = lib().orc_replica_1d(ctypes.byref(sys), int(realisation), int(M), int(R), lo, hi,
                              int(precision), _ptr(r0a), _ptr(mu), _ptr(last), int(threads))
    if rc != 0:
        raise ValueError(f"orc_replica_1d failed ({rc})")
    muc = mu[..., 0] + 1j * mu[..., 1]
    if last is not None:
        cdt = np.complex64 if precision == 0 else np.complex128
        last = last.view(cdt).reshape(R, 2, n)
    return muc, last


def velocity_x(sys: System, vac, t_scaled: float, vec):
    return velocity(sys, vac, t_scaled, vec, 0)


def velocity(sys: System, vac, t_scaled: float, vec, direction: int = 0):
    """h~ vec with h~ = [r_dir, H~] (direction 0: x, 1: y) on the lattice of `sys`."""
    n = norb(sys)
    v = np.ascontiguousarray(np.stack([np.real(vec), np.imag(vec)], -1).astype(np.float64))
    out = np.empty((n, 2), np.float64)
    lib().orc_velocity(ctypes.byref(sys), _ptr(np.ascontiguousarray(vac, np.uint8)),
                       float(t_scaled), int(direction), _ptr(v), _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def moments_2d(sys: System, M: int, R: int, realisation: int = 0, e_min=None, e_max=None,
               r0=None, want_families: bool = False, threads: int = 0, alpha: int = 0,
               beta: int = 0):
    """mu_nm = <a_n|b_m>/N_eff averaged over R vectors with a_n = T_n h~alpha r and
    b_m = h~beta T_m r (directions 0: x, 1: y), i.e. <r|v_alpha T_n v_beta T_m|r>/N."""
    n = norb(sys)
    lo, hi = _bounds(sys, e_min, e_max)
    r0a = _as_r0(r0, R, n)
    mu = np.empty((M, M, 2), np.float64)
    A = np.empty((M, n, 2), np.float64) if want_families else None
    B = np.empty((M, n, 2), np.float64) if want_families else None
    rc = lib().orc_moments_2d(ctypes.byref(sys), int(realisation), int(M), int(R), lo, hi,
                              _ptr(r0a), _ptr(mu), _ptr(A), _ptr(B), int(alpha), int(beta),
                              int(threads))
    if rc != 0:
        raise ValueError(f"orc_moments_2d failed ({rc})")
    out = mu[..., 0] + 1j * mu[..., 1]
    if want_families:
        return out, A[..., 0] + 1j * A[..., 1], B[..., 0] + 1j * B[..., 1]
    return out


def moments_2d_panels(sys: System, M: int, R: int, rows, cols, realisation: int = 0, e_min=None, e_max=None,
                      threads: int = 0, alpha: int = 0, beta: int = 0):
    """Rows and columns of mu_nm (as moments_2d) without storing the families: returns
    (P_rows [len(rows)][M], P_cols [M][len(cols)]) complex with P_rows[i][m] = mu_{rows[i], m}
    and P_cols[n][j] = mu_{n, cols[j]}."""
    lo, hi = _bounds(sys, e_min, e_max)
    r = np.ascontiguousarray(rows, np.int32)
    c = np.ascontiguousarray(cols, np.int32)
    pr = np.empty((len(r), M, 2), np.float64)
    pc = np.empty((M, len(c), 2), np.float64)
    rc = lib().orc_moments_2d_panels(ctypes.byref(sys), int(realisation), int(M), int(R), lo, hi, _ptr(r), len(r),
                                     _ptr(c), len(c), int(alpha), int(beta), _ptr(pr), _ptr(pc), int(threads))
    if rc != 0:
        raise ValueError(f"orc_moments_2d_panels failed ({rc})")
    return pr[..., 0] + 1j * pr[..., 1], pc[..., 0] + 1j * pc[..., 1]


def kernel_jackson(M: int):
    g = np.empty(M, np.float64)
    lib().orc_kernel_jackson(int(M), _ptr(g))
    return g


def kernel_lorentz(M: int, lam: float):
    g = np.empty(M, np.float64)
    lib().orc_kernel_lorentz(int(M), float(lam), _ptr(g))
    return g


def dos(mu, E, e_min: float, e_max: float, g=None):
    """rho(E) per orbital per eV from raw moments mu[0..M-1] (Eqs. e7/e8a + kernel g)."""
    mu = np.ascontiguousarray(np.real(np.asarray(mu)), np.float64)
    E = np.ascontiguousarray(E, np.float64)
    ga = None if g is None else np.ascontiguousarray(g, np.float64)
    rho = np.empty(E.shape[0], np.float64)
    lib().orc_dos(_ptr(mu), int(mu.shape[0]), _ptr(ga), float(e_min), float(e_max), _ptr(E),
                  int(E.shape[0]), _ptr(rho))
    return rho


def cpgf_coeff(n: int, eps: float, eta: float, sigma: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_cpgf_coeff(int(n), float(eps), float(eta), int(sigma), ctypes.byref(re),
                         ctypes.byref(im))
    return complex(re.value, im.value)


def replica_window(sys: System, M: int, R: int, precision: int, x0: int, y0: int,
                   realisation: int = 0, e_min=None, e_max=None, half=None):
    """(r_{M-2}, r_{M-1}) of the fixed-rounding replica at cell (x0, y0) of a large
    lattice, computed on a light-cone window: [R][2][orbitals per cell] complex."""
    lo, hi = _bounds(sys, e_min, e_max)
    sorb = 2 if sys.lattice == HONEYCOMB else 1
    dt = np.float32 if precision == 0 else np.float64
    out = np.empty((R, 2, sorb, 2), dt)
    h = M if half is None else int(half)
    rc = lib().orc_replica_window(ctypes.byref(sys), int(realisation), int(M), int(R), lo, hi,
                                  int(precision), int(x0), int(y0), h, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_replica_window failed ({rc})")
    cdt = np.complex64 if precision == 0 else np.complex128
    return out.view(cdt).reshape(R, 2, sorb)


def inner_products(A, B, scale: float = 1.0):
    """Plain FP64 definition C[n][m] = scale * sum_i conj(A[n][i]) B[m][i] (the contraction
    of Eq. Gammanm), via a library matrix product."""
    A = np.asarray(A, np.complex128)
    B = np.asarray(B, np.complex128)
    return scale * (np.conj(A) @ B.T)


def cpgf_coeffs(n_max: int, z_real, eta: float, sigma: int):
    """Vectorised CPGF coefficients g_n^{sigma,eta}(eps), n < n_max, at real eps = z_real
    (Eq. green_function_cheb_expansionb): -2 sigma i exp(-sigma i n arccos(eps + i sigma
    eta)) / sqrt(1 - (eps + i sigma eta)^2).  Returns [n_max][len(z_real)]."""
    z = np.asarray(z_real, np.float64) + 1j * sigma * eta
    th = np.arccos(z)
    n = np.arange(n_max)[:, None]
    return -2.0 * sigma * 1j * np.exp(-sigma * 1j * n * th[None, :]) / np.sqrt(1.0 - z * z)[None, :]


def green(mu, E, e_min: float, e_max: float, eta: float, g=None):
    """Average Green's function per orbital G(E + i eta) in 1/eV from raw moments
    (Eqs. green_function_cheb_expansion/b traced as in Eq. e7): with eps = (E - de_plus) /
    de_minus and eta~ = eta / de_minus,
      G(E + i eta) = (1/de_minus) sum_n [g_n mu_n / (1 + delta_n0)] g^{+,eta~}_n(eps),
    optionally damped by a kernel g.  The eta-resolved density is -Im G / pi."""
    mu = np.real(np.asarray(mu, np.float64))
    M = mu.shape[0]
    dm, dp = 0.5 * (e_max - e_min), 0.5 * (e_max + e_min)
    eps = (np.asarray(E, np.float64) - dp) / dm
    w = np.where(np.arange(M) == 0, 0.5, 1.0) * mu
    if g is not None:
        w = w * np.asarray(g, np.float64)
    return (w @ cpgf_coeffs(M, eps, eta / dm, +1)) / dm


def chebyshev_sum(sys: System, coef, vec, realisation: int = 0, e_min=None, e_max=None):
    """sum_n coef_n T_n(H~) vec (complex coef [M], vec [N]); vacant orbitals removed."""
    lo, hi = _bounds(sys, e_min, e_max)
    c = np.ascontiguousarray(np.stack([np.real(coef), np.imag(coef)], -1).astype(np.float64))
    v = np.ascontiguousarray(np.stack([np.real(vec), np.imag(vec)], -1).astype(np.float64))
    out = np.empty_like(v)
    rc = lib().orc_chebyshev_sum(ctypes.byref(sys), int(realisation), lo, hi, int(c.shape[0]), _ptr(c), _ptr(v),
                                 _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_chebyshev_sum failed ({rc})")
    return out[:, 0] + 1j * out[:, 1]


def evolution_coeffs(M: int, dt: float, e_min: float, e_max: float):
    """Chebyshev coefficients of exp(-i H dt) (hbar = 1, dt in hbar/eV) in H~ (the
    wave-packet section, Tal-Ezer and Kosloff): exp(-i de_plus dt) (2 - delta_n0) (-i)^n
    J_n(de_minus dt), the Bessel functions by scipy.  (The paper prints (-1)^n; the
    expansion exp(-i x tau) = J_0(tau) + 2 sum_n (-i)^n J_n(tau) T_n(x) has (-i)^n.)"""
    from scipy.special import jv
    dm, dp = 0.5 * (e_max - e_min), 0.5 * (e_max + e_min)
    n = np.arange(M)
    c = np.where(n == 0, 1.0, 2.0) * (-1j) ** n * jv(n, dm * dt)
    return np.exp(-1j * dp * dt) * c


def propagate(sys: System, psi0, dt: float, nsteps: int, M: int, realisation: int = 0, e_min=None,
              e_max=None):
    """psi(nsteps dt) = U(dt)^nsteps psi0 with the truncated Chebyshev series per step;
    returns the wave function after every step, [nsteps][N]."""
    lo, hi = _bounds(sys, e_min, e_max)
    c = evolution_coeffs(M, dt, lo, hi)
    out, psi = [], np.asarray(psi0, np.complex128)
    for _ in range(nsteps):
        psi = chebyshev_sum(sys, c, psi, realisation, lo, hi)
        out.append(psi)
    return np.array(out)


def unit_cell_factor(lattice: int):
    """(orbitals per cell) * a^2 / Omega_c: honeycomb 2 * 2/sqrt(3), square 1."""
    return 2.0 * 2.0 / np.sqrt(3.0) if lattice == HONEYCOMB else 1.0


def sigma_dc(mu_nm, E, e_min: float, e_max: float, lattice: int, kernel: str = "jackson", lam: float = 4.0):
    """Longitudinal DC conductivity at T = 0 in units of e^2/hbar per spin: the omega -> 0
    limit of the Kubo formula (Eq. conductivity_1st_order), where only states at the Fermi
    energy contribute (Kubo-Greenwood),
      sigma(E) = pi hbar e^2 / Omega Tr[v delta(E - H) v delta(E - H)],
    with v = -i (de_minus a / hbar) h~, delta(E - H) = delta(e - H~)/de_minus and each delta
    function expanded in M Chebyshev terms with the kernel (Sec. 2a):
      sigma(E) = pi (n_orb a^2/Omega_c) sum_nm c_n(e) c_m(e) mu_nm,
      c_n(e) = g_n (2 - d_n0) T_n(e) / (pi sqrt(1 - e^2)),   e = (E - de_plus)/de_minus,
    mu_nm = <r|v T_n v T_m|r>/N the 2D moments (v = -i h~).  0 outside |e| < 1."""
    mu = np.asarray(mu_nm, np.complex128)
    M = mu.shape[0]
    dm, dp = 0.5 * (e_max - e_min), 0.5 * (e_max + e_min)
    if kernel == "jackson":
        g = kernel_jackson(M)
    elif kernel == "lorentz":
        g = kernel_lorentz(M, lam)
    else:
        g = np.ones(M)
    w = np.where(np.arange(M) == 0, 1.0, 2.0) * g
    out = np.zeros(len(E))
    for k, Ek in enumerate(np.asarray(E, np.float64)):
        e = (Ek - dp) / dm
        if not abs(e) < 1.0:
            continue
        c = w * np.cos(np.arange(M) * np.arccos(e)) / (np.pi * np.sqrt(1.0 - e * e))
        out[k] = np.pi * unit_cell_factor(lattice) * float(np.real(c @ mu @ c))
    return out


def sigma_dc_bastin(mu_nm, E_F, e_min: float, e_max: float, eta: float, lattice: int,
                    kernel: str = "jackson", lam: float = 4.0, n_quad: int = 0, kT: float = 0.0):
    """DC conductivity tensor element sigma_ab(E_F) in units of e^2/hbar per spin from the
    Kubo-Bastin formula (the omega -> 0 response of Sec. 2b, full-spectral form of the
    Hall-conductivity example): with f the Fermi function,
      sigma_ab = i hbar e^2/Omega int de f(e) Tr[v_a delta(e - H) v_b dG^R/de
                                                - v_a dG^A/de v_b delta(e - H)],
    rescaled (v = -i (de_minus a/hbar) h~) and expanded in Chebyshev polynomials:
      sigma_ab = Re{ i (n_orb a^2/Omega_c) int de f(e) sum_nm mu_nm
                        [Delta_n(e) dG^R_m(e) - dG^A_n(e) Delta_m(e)] },
      Delta_n(e) = k_n (2 - d_n0) T_n(e) / (pi sqrt(1 - e^2)),
      G^{R/A}_m(e) = k_m g^{+-}_m(e +- i eta) / (1 + d_m0)     (CPGF, Eq. green_function_cheb_expansionb),
      d g_m/dz = g_m(z) [sigma i m / sqrt(1 - z^2) + z / (1 - z^2)],
    mu_nm = <r|v_a T_n v_b T_m|r>/N the 2D moments, k_n the kernel (None: k_n = 1), eta
    (eV) the CPGF broadening that keeps the integrand regular at the band edges.  The
    Fermi sea runs over the rescaled band [-1, e_F] (kT > 0: the whole band weighted by the
    Fermi function), by Gauss-Legendre quadrature in theta, e = cos(theta).  E_F: array."""
    mu = np.asarray(mu_nm, np.complex128)
    M = mu.shape[0]
    dm, dp = 0.5 * (e_max - e_min), 0.5 * (e_max + e_min)
    if kernel == "jackson":
        k = kernel_jackson(M)
    elif kernel == "lorentz":
        k = kernel_lorentz(M, lam)
    else:
        k = np.ones(M)
    n = np.arange(M)
    kw = k * np.where(n == 0, 0.5, 1.0)
    A = mu * kw[:, None] * kw[None, :]   # kernel and 1/(1 + d_n0) of both series
    et = eta / dm
    K = n_quad if n_quad > 0 else 2 * M + 64
    x, w = np.polynomial.legendre.leggauss(K)
    out = np.zeros(len(np.atleast_1d(E_F)))
    for i, Ef in enumerate(np.atleast_1d(np.asarray(E_F, np.float64))):
        eF = (Ef - dp) / dm
        if kT <= 0.0 and eF <= -1.0:
            continue
        thF = np.arccos(min(eF, 1.0)) if kT <= 0.0 else 0.0
        theta = thF + (np.pi - thF) * 0.5 * (x + 1.0)
        wq = w * 0.5 * (np.pi - thF)
        e = np.cos(theta)
        if kT > 0.0:
            wq = wq / (1.0 + np.exp((e * dm + dp - Ef) / kT))
        # Delta_n(e) de without k_n and 1/(1 + d_n0) (those sit in A): (2/pi) cos(n theta) dtheta
        D = (2.0 / np.pi) * np.cos(n[:, None] * theta[None, :]) * wq[None, :]
        dG = []
        for sg in (+1, -1):
            z = e + 1j * sg * et
            s1 = np.sqrt(1.0 - z * z)
            dG.append(cpgf_coeffs(M, e, et, sg) * (sg * 1j * n[:, None] / s1[None, :]
                                                  + (z / (s1 * s1))[None, :]))
        S = np.sum(D * (A @ dG[0])) - np.sum(dG[1] * (A @ D))
        out[i] = float(np.real(1j * unit_cell_factor(lattice) * S))
    return out


def sigma_xx(mu_nm, omega, e_min: float, e_max: float, E_F: float, eta: float, lattice: int,
             kernel: str = "jackson", n_quad: int = 0, gamma_n=None, kT: float = 0.0):
    """First-order optical conductivity sigma_xx(omega) in units of e^2/hbar (T = 0),
    from the 2D moments mu_nm = <r|v T_n v T_m|r>/N, v = -i h~x (Sec. 2b):

      Gamma_nm = -mu_nm / ((1 + d_n0)(1 + d_m0))                      (Eq. Gammanm)
      Lambda_nm(w) = int_{-1}^{eps_F} de [g^R_n(e + w) Delta_m(e) + Delta_n(e) g^A_m(e - w)]
      sigma = -i (n_orb a^2/Omega_c) / w * [sum_n Lambda_n Gamma^xx_n + sum_nm Lambda_nm Gamma_nm]
                                                  (Eq. conductivity_1st_order, rescaled)
    with w = hbar omega / de_minus, eta in eV, Delta_m(e) de = (2/pi) cos(m theta) d theta
    for e = cos theta, and the Fermi-sea integral by Gauss-Legendre quadrature in theta
    (numpy.polynomial.legendre.leggauss); kT > 0 (eV) integrates the whole band weighted
    by the Fermi function.  kernel: "jackson" damps Gamma by g_n g_m;
    None leaves it undamped.  gamma_n (optional) = Gamma^xx_n for the diamagnetic term."""
    mu = np.asarray(mu_nm, np.complex128)
    M = mu.shape[0]
    dm, dp = 0.5 * (e_max - e_min), 0.5 * (e_max + e_min)
    w0 = np.where(np.arange(M) == 0, 0.5, 1.0)
    G = -mu * w0[:, None] * w0[None, :]
    if kernel == "jackson":
        g = kernel_jackson(M)
        G = G * g[:, None] * g[None, :]
    eF = (E_F - dp) / dm
    # T = 0: Fermi sea [-1, eps_F] (theta in [theta_F, pi]); T > 0: the whole band with the
    # Fermi function f(E) = 1/(1 + exp((E - E_F)/kT)) as a weight
    thF = np.arccos(np.clip(eF, -1.0, 1.0)) if kT <= 0.0 else 0.0
    K = n_quad if n_quad > 0 else 2 * M + 64
    x, wq = np.polynomial.legendre.leggauss(K)
    theta = thF + (np.pi - thF) * 0.5 * (x + 1.0)
    wq = wq * 0.5 * (np.pi - thF)
    eps = np.cos(theta)
    if kT > 0.0:
        wq = wq / (1.0 + np.exp((eps * dm + dp - E_F) / kT))
    D = (2.0 / np.pi) * np.cos(np.arange(M)[:, None] * theta[None, :]) * wq[None, :]  # Delta_m de
    eta_t = eta / dm
    U = G @ D        # sum_m Gamma_nm Delta_m(e_k) de_k
    Wm = G.T @ D     # sum_n Delta_n(e_k) de_k Gamma_nm
    out = np.empty(len(omega), np.complex128)
    for i, om in enumerate(np.asarray(omega, np.float64)):
        wt = om / dm
        gR = cpgf_coeffs(M, eps + wt, eta_t, +1)
        gA = cpgf_coeffs(M, eps - wt, eta_t, -1)
        S = np.sum(gR * U) + np.sum(gA * Wm)
        if gamma_n is not None:
            Dn = (2.0 / np.pi) * np.cos(np.arange(len(gamma_n))[:, None] * theta[None, :]) * wq[None, :]
            S += np.sum(np.asarray(gamma_n)[:, None] * Dn)
        out[i] = -1j * unit_cell_factor(lattice) / wt * S
    return out
