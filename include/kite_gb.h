/*
 * kite_gb.h -- C ABI of the GB300-native stochastic Chebyshev (kernel polynomial)
 * expansion of lattice Green's functions described in KITE (arXiv:1910.05194).
 *
 * Every call takes plain pointers and sizes.  A pointer argument documented as
 * "host or device" may point to host memory (pageable or pinned) or to device memory
 * of the context's GPU; the library tells them apart with cudaPointerGetAttributes.
 * The caller owns every input and output buffer.  The library owns its work buffers
 * (grown on demand inside the context, released by kite_destroy).
 *
 * Calls are ordered on the context's stream and return after their results are
 * complete and visible in the caller's buffers.  Device inputs produced on another
 * stream must be complete before the call (bind the context to that stream, or
 * synchronise): the library does not wait on streams it does not own.  Every call returns KITE_OK (0) or a
 * negative status; on failure no output buffer holds a trusted result, and
 * kite_last_error() gives a one-line reason.  Nothing in the library aborts or exits.
 *
 * Notation (Sec. 2 of the paper): H~ = (H - de_plus)/de_minus with
 * de_pm = (E_max +- E_min)/2 (Eqs. rescalingH/rescalingE); T_n are Chebyshev
 * polynomials (Eq. e3, operator form Eq. e6); mu_n = <r|T_n(H~)|r>/N_eff are the
 * moments of the average density of states (Eqs. e7, e8) estimated with random
 * vectors (stochastic trace evaluation, Sec. 2c).
 */
#ifndef KITE_GB_H
#define KITE_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------- */
#define KITE_OK 0
#define KITE_ERR_ARG (-1)         /* invalid argument (sizes, enums, null pointers)     */
#define KITE_ERR_OOM (-2)         /* device allocation failed                           */
#define KITE_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed        */
#define KITE_ERR_BOUNDS (-4)      /* |mu_n| > 1 + 1e-3 or non-finite: spectrum left
                                     [-1,1] (Eq. e6 requires ||H~|| <= 1)               */
#define KITE_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                 */
#define KITE_ERR_UNSUPPORTED (-6) /* valid request the library does not implement      */

/* ---- enums -------------------------------------------------------------------- */
#define KITE_HONEYCOMB 0 /* Listing 1: a1=[a,0], a2=[a/2, a sqrt3/2], two orbitals A, B   */
#define KITE_SQUARE 1    /* one orbital per cell, four nearest neighbours               */
#define KITE_DISORDER_UNIFORM 0
#define KITE_DISORDER_GAUSSIAN 1

#define KITE_FP32 0 /* complex FP32 recursion, FP64 moment accumulation above 32 terms */
#define KITE_FP64 1 /* complex FP64 recursion                                           */

#define KITE_KERNEL_NONE 0
#define KITE_KERNEL_JACKSON 1 /* g_n of Weisse et al. 2006 (the paper's KPM reference)   */
#define KITE_KERNEL_LORENTZ 2 /* g_n = sinh(lambda(1-n/M))/sinh(lambda), Sec. 2a        */

/* ---- problem description -------------------------------------------------------- */

/* A tight-binding lattice with disorder, periodic or open (Sec. 3d, Listings 1-3; Sec. 4b).
 * Orbitals are numbered o = 2*(y*Lx + x) + s for the honeycomb lattice (s = 0 for A,
 * 1 for B) and o = y*Lx + x for the square lattice; N = number of orbitals.
 *   lattice  KITE_HONEYCOMB or KITE_SQUARE
 *   Lx, Ly   unit cells along a1, a2 (>= 1)
 *   t        nearest-neighbour hopping (eV)
 *   disorder KITE_DISORDER_UNIFORM (Anderson, Sec. 4b) or KITE_DISORDER_GAUSSIAN (the
 *            'Gaussian' kind of the Python interface, Sec. 3d)
 *   W        on-site disorder strength (eV), >= 0: V_o uniform in [-W/2, W/2], or
 *            Gaussian with mean 0 and standard deviation W
 *   delta    staggered potential: +delta/2 on A, -delta/2 on B (honeycomb only, eV)
 *   p_vac    probability that an orbital is a vacancy (removed with its bonds), [0,1]
 *   seed     key of the Philox4x32-10 counter-based generator that draws V_o, the
 *            vacancies and the random-phase vectors.  Realisation s, orbital o:
 *            counter (o_lo, o_hi, s, 1); vector v of realisation s: (o_lo, o_hi,
 *            s*R + v, 2).  u = (w0 * 2^21 + (w1 >> 11)) * 2^-53,
 *            V_o = W*(u - 1/2) [+- delta/2] (uniform) or
 *            V_o = W*(sqrt(-2 ln(1 - u)) * cos(2 pi w3 2^-32)) [+- delta/2] (Gaussian,
 *            Box-Muller; |V_o - mean| <= sqrt(106 ln 2) W < 8.58 W), vacant iff
 *            w2 < floor(p_vac * 2^32), phase vector entry exp(2 pi i u) (0 on
 *            vacancies).
 *   flux     perpendicular magnetic field (Sec. "Magnetic Field", Peierls substitution)
 *            as flux quanta h/e per unit cell; 0 = no field.  Landau gauge A = (-B y, 0):
 *            the hopping from orbital j to o, bond offset (dx, dy) = r_o - r_j in units
 *            of a, becomes t exp(i theta), theta = -2 pi (flux/A_cell)(y_o - dy/2) dx,
 *            A_cell = sqrt(3)/2 (honeycomb) or 1 (square), y_o the orbital's y
 *            coordinate (cell (x, y) at x a1 + y a2, a1 = (1, 0), a2 = (1/2, sqrt3/2),
 *            A at (0, -a_cc/2), B at (0, +a_cc/2), a_cc = 1/sqrt3).  With y periodic
 *            flux * Ly must be even (honeycomb) or an integer (square);
 *            kite_flux_nearest gives the nearest such flux; with y open any flux
 *            fits.  Accepted by
 *            kite_moments_1d (complex start vectors), kite_moments_1d_batched (each
 *            system its own flux), kite_moments_2d (the velocity h~ = [r, H~] carries
 *            the same bond phases), kite_spectral_k, kite_ldos and kite_propagate;
 *            kite_moments_1d_static returns KITE_ERR_ARG for a nonzero flux.
 *   open_x, open_y  boundaries along a1, a2 (the configuration's boundaries flag,
 *            Sec. 3d): 0 = periodic, 1 = open (the bonds that would wrap around
 *            the torus are absent: honeycomb A(Lx-1, y) - B(0, y-1) for x, A(x, 0) -
 *            B(x, -1) and A(x, 0) - B(x+1, -1) for y; square the wrapping x or y
 *            bonds).  Orbital indexing and draws are the same as on the torus.
 *            Accepted by kite_moments_1d, kite_moments_2d, kite_spectral_k,
 *            kite_ldos and kite_propagate; kite_moments_1d_batched and
 *            kite_moments_1d_static return KITE_ERR_ARG for an open boundary. */
typedef struct {
  int32_t lattice;
  int32_t Lx, Ly;
  int32_t disorder;
  double t;
  double W;
  double delta;
  double p_vac;
  uint64_t seed;
  double flux;
  int32_t open_x, open_y;
} kite_system;

/* Chebyshev expansion parameters (the calculation settings of Sec. 3d: num_moments,
 * num_random, num_disorder, precision, spectrum range).
 *   M          number of moments mu_0..mu_{M-1} (>= 1)
 *   R          random vectors per disorder realisation (>= 1)
 *   S          disorder realisations (>= 1)
 *   precision  KITE_FP32 or KITE_FP64
 *   e_min, e_max  spectrum endpoints in eV; both 0 selects the Gershgorin enclosure
 *              +-(Z|t| + max|V - mean| + |delta|/2) * 1.01 (kite_bounds)
 *   r0         optional start vectors instead of random phases: [S*R][N] complex FP64,
 *              interleaved (re, im), host or device; entries on vacancies are ignored
 *              (the vacancy is removed from the Hilbert space).  NULL = random phases.
 *              Page-locked host memory is read in place by the kernels (no copy);
 *              pageable host memory is first copied to a context-owned device buffer.
 *              The caller keeps r0 unchanged until the call returns.
 *   r_last     optional output: per vector the last two iterates (T_{M-2} r, T_{M-1} r)
 *              as [S*R][2][N] interleaved complex of the working precision (complex64
 *              for KITE_FP32, complex128 for KITE_FP64), host or device; for M = 1 both
 *              slots hold r.  NULL = not wanted.  Lets a caller check the recursion bit
 *              for bit or checkpoint a run.  Ignored when doubling is set.
 *   doubling   0: mu_n = <r|T_n r> for every n (one recursion step per moment).
 *              1: moment doubling -- T_n^2 = (T_2n + T_0)/2 and T_{n+1} T_n =
 *              (T_{2n+1} + T_1)/2 for the Hermitian H~ give mu_2n = 2<r_n|r_n> - mu_0 and
 *              mu_{2n+1} = 2<r_{n+1}|r_n> - mu_1, so ceil(M/2) steps yield M moments and
 *              r_0 is never re-read (identical in exact arithmetic, not bit for bit).
 *   real_vectors  0: complex unit-modulus random phases exp(2 pi i u) (default).
 *              1: real random signs +-1 (the sign from the same draw, u < 1/2 -> +1) --
 *              the paper allows real or complex white noise (Sec. 2c); for the real
 *              Hamiltonians here both are unbiased.  A real vector takes half the bytes
 *              of a complex one (a batch holds 16 FP32 or 8 FP64 of them) and its trace
 *              estimate has twice the variance of a unit-phase vector (2 sum_{i!=j} A_ij^2
 *              against sum_{i!=j} |A_ij|^2), so the cost per unit of accuracy is the same
 *              at half the memory.  kite_moments_1d only; r_last must be NULL; caller
 *              start vectors (r0) contribute their real parts. */
typedef struct {
  int32_t M;
  int32_t R;
  int32_t S;
  int32_t precision;
  double e_min;
  double e_max;
  const double* r0;
  void* r_last;
  int32_t doubling;
  int32_t real_vectors;
} kite_kpm;

/* Per-call statistics (all optional outputs). */
typedef struct {
  double seconds;       /* device time of the moment sweep (CUDA events)            */
  double updates;       /* orbital * moment * vector updates done (N_eff*(M-1)*R*S)  */
  double bytes_moved;   /* algorithmic HBM bytes of the sweep (iterates read/written + on-site) */
  double gbps;          /* bytes_moved / seconds / 1e9                               */
  double max_abs_imag;  /* max_n |Im mu_n| of the vector average (0 for exact H~; the
                           FP64 sweeps and the on-chip cluster sweep do not form the
                           imaginary part, which vanishes for a Hermitian H~, and read 0) */
  double e_min, e_max;  /* bounds used (eV)                                          */
  int64_t n_eff;        /* non-vacant orbitals of the last realisation               */
  int32_t grid, block;  /* launch shape of the sweep kernel                           */
  double step_seconds;  /* device time of the recursion-step launches alone          */
  int64_t step_launches;/* number of recursion-step launches timed in step_seconds   */
  double step_bytes;    /* algorithmic bytes of those launches                       */
  double gemm_seconds;  /* 2D moments: device time of the tensor-core contraction    */
  double gemm_flops;    /* 2D moments: tensor flops of the contraction (4 BF16 products) */
  int32_t ring_stages;  /* step kernel: shared-memory ring depth used (autotuned)       */
  int32_t ctas_per_sm;  /* step kernel: resident CTAs per SM used (autotuned)           */
  int32_t steps_per_pass; /* step kernel: recursion steps fused per pass over the iterates
                             (1, or 2 with temporal blocking; autotuned; all of them when
                             the cluster sweep ran)                                       */
  int32_t cluster_ctas; /* kite_moments_1d: CTAs per thread-block cluster when the small-
                           lattice sweep held the iterates on chip (one cluster per real
                           recursion, see kite_moments_1d), else 0                      */
} kite_stats;

typedef struct kite_ctx kite_ctx;

/* ---- environment switches ---------------------------------------------------------
 * Read at each call.  The iterates are the same bits whatever the launch shape, and the
 * moments differ only by the regrouping of FP32 partial sums, except where noted (the
 * cluster sweep reports the vanishing imaginary part as 0; KITE_GEMM_PRODUCTS=3).
 *   KITE_AUTOTUNE=0       no timing of launch shapes: 8-stage rings at full occupancy, one
 *                         recursion step per launch, no cluster sweep
 *   KITE_TUNE=SxK[x2|x3]  pins the 1D sweep's ring depth S, CTAs per SM K and steps per pass
 *   KITE_PASS_STEPS=1|2|3 pins the steps per pass (1D and batched sweeps; 3: 1D only)
 *   KITE_CLUSTER=0|1      forbids / forces the on-chip cluster sweep of small lattices
 *                         (KITE_CLUSTER_CTAS=2..16 pins its CTAs per cluster)
 *   KITE_FAM_STREAMS=1    the 2D path's two vector families in sequence on one stream
 *   KITE_FAM_CPS=K        CTAs per SM of the 2D family steps
 *   KITE_GEMM_PRODUCTS=3  drops the lo x lo product of the split-BF16 contraction
 *                         (a quarter less tensor work, ~5e-6 relative bias) */

/* ---- context -------------------------------------------------------------------- */

/* Creates a context on CUDA device `device`, bound to `cuda_stream` (a cudaStream_t;
 * NULL creates a private stream that is ordered with the legacy default stream, so work
 * the caller queued there completes first).  *out receives the handle.
 * Errors: KITE_ERR_ARG (out NULL, bad device), KITE_ERR_CUDA. */
int kite_create(kite_ctx** out, int device, void* cuda_stream);

/* Releases the context, its private stream and work buffers.  NULL is a no-op. */
void kite_destroy(kite_ctx* ctx);

/* Rebinds the context to another stream of the same device (NULL = private stream). */
int kite_set_stream(kite_ctx* ctx, void* cuda_stream);

/* Static, thread-safe description of a status code. */
const char* kite_status_string(int status);

/* Detail of the last failed call on this context ("" if none).  Valid until the next
 * call on the same context. */
const char* kite_last_error(const kite_ctx* ctx);

/* Gershgorin spectrum enclosure used when e_min = e_max = 0 (Eqs. rescalingH/E and the
 * bound warning of Sec. 4b): e_max = -e_min = (Z|t| + Vmax + |delta|/2) * 1.01 with
 * Z = 3 (honeycomb) or 4 (square) and Vmax = W/2 (uniform) or 8.58 W (Gaussian: the
 * largest value its transform can give).  Host-only arithmetic in FP64.
 * Errors: KITE_ERR_ARG. */
int kite_bounds(const kite_system* sys, double* e_min, double* e_max);

/* The flux per unit cell closest to `flux` that the torus of `sys` admits in the Landau
 * gauge (flux * Ly even on the honeycomb, integer on the square lattice); the field KITE
 * "best matches" to a requested one (Sec. "Magnetic Field").  sys->flux is ignored.
 * Host-only.  Errors: KITE_ERR_ARG. */
int kite_flux_nearest(const kite_system* sys, double flux, double* out);

/* ---- 1D moments ----------------------------------------------------------------- */

/* Moments of the average DOS, mu_n = (1/(S R)) sum_{s,r} <r|T_n(H~)|r> / N_eff for
 * n = 0..M-1 (Eqs. e6-e8, stochastic trace of Sec. 2c; cost Z*N*M*R*S, Eq.
 * PcomplexityFactor).  T_1 r = H~ r, T_{n+1} r = 2 H~ T_n r - T_{n-1} r, with H~
 * applied matrix-free (Sec. 3a pattern rules): on-site term and nearest-neighbour
 * hopping, vacancies removed.  Moments are raw (mu_0 = 1); the reconstruction applies
 * the (2 - delta_n0) weight of the delta-function expansion.
 * A lattice too small to keep the GPU busy with one launch per step (fewer than four row
 * segments per SM) and without a magnetic field may instead run the whole sweep on chip,
 * one thread-block cluster per real recursion (the real and imaginary parts of a complex
 * vector evolve independently under a real H~); the autotuner takes that path when it
 * measures it faster, st->cluster_ctas reports it, and the imaginary part of each
 * moment, which vanishes for a real symmetric H~, is then not formed and reads 0.
 * KITE_CLUSTER=0 / 1 in the environment forbids / forces it.
 *   mu          [M] FP64, real part of the average, host or device (required)
 *   mu_per_vec  [S*R][M] complex FP64 interleaved (re, im) per vector, or NULL
 *   st          statistics, or NULL
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_BOUNDS. */
int kite_moments_1d(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, double* mu,
                    double* mu_per_vec, kite_stats* st);

/* Chebyshev moments of the k-resolved spectral function (the paper's spectral-function
 * section, the quantity behind ARPES): the recursion starts from the plane wave
 *   |k> = sum_alpha w_alpha sum_i exp(i k.R_i^alpha) |i, alpha>
 * (zero on vacant orbitals) instead of a random vector, and
 *   mu_n(k) = <k| T_n(H~) |k> / N_eff,
 * averaged over kpm->S disorder realisations, so that rho_k(E) follows from
 * kite_reconstruct_dos applied to the real parts.  Orbital positions R_i^alpha in units of
 * the lattice constant: honeycomb cell (x, y) at x a1 + y a2, a1 = (1, 0),
 * a2 = (1/2, sqrt(3)/2), A at (0, -a_cc/2), B at (0, +a_cc/2), a_cc = 1/sqrt(3) (the
 * paper's lattice set-up); square (x, y).  With random orbital weights averaged
 * (<w_a* w_b> = delta_ab) the clean-lattice result is the band structure with equal
 * weights; fixed weights give the intensities of those weights.
 *   kpm      M, precision, bounds (e_min = e_max = 0: Gershgorin), S realisations; R must
 *            be 1 (one start vector per k-point); r0, r_last NULL; doubling allowed
 *   k        [nk][2] (kx, ky) in 1/a, host or device
 *   weights  [orbitals per cell][2] complex w_alpha, host or device; NULL = all 1
 *   mu       [nk][M] complex FP64 interleaved, host or device
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_BOUNDS, KITE_ERR_TIMEOUT. */
int kite_spectral_k(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const double* k,
                    int nk, const double* weights, double* mu, kite_stats* st);

/* Chebyshev moments of the local density of states (the paper's LDOS section):
 *   mu_n(i) = <i| T_n(H~) |i>  for the orbitals i = orbitals[j],
 * one disorder realisation (kpm->S = 1), the recursion started from the orbital's basis
 * vector on the whole lattice (a sweep batch holds 8 FP32 or 4 FP64 orbitals); rho_i(E)
 * follows from kite_reconstruct_dos on the real parts.  mu_0 = 1 (0 for a vacant orbital).
 * Orbital index = (y Lx + x) * orbitals per cell + sublattice.
 *   kpm       M, precision, bounds, R = 1, S = 1, r0 and r_last NULL, doubling allowed
 *   orbitals  [n] int64, host or device
 *   mu        [n][M] complex FP64 interleaved, host or device
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_BOUNDS, KITE_ERR_TIMEOUT. */
int kite_ldos(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const int64_t* orbitals,
              int n, double* mu, kite_stats* st);

/* Wave-packet time evolution (the paper's spintronics section; hbar = 1, times in hbar/eV,
 * i.e. t_fs = 0.6582 t):
 *   |psi(t + dt)> = exp(-i H dt) |psi(t)>
 *                 = exp(-i de_plus dt) [c_0 + 2 sum_{n=1}^{M-1} c_n T_n(H~)] |psi(t)>,
 *   c_n = (-i)^n J_n(de_minus dt)
 * (the Chebyshev propagator of Tal-Ezer and Kosloff that the paper cites; the printed
 * (-1)^n is read as (-i)^n, which the expansion of exp(-i x tau) has).  M Chebyshev terms
 * per step: the truncation error falls off like J_M(de_minus dt), negligible once
 * M > 1.1 de_minus dt + 20.  Each step runs M - 1 stencil steps that also accumulate the
 * series; vacant orbitals stay 0.  A magnetic field (sys->flux) and open boundaries
 * enter H as in the moment sweeps.
 *   kpm     M terms per step, R wave functions, S = 1, precision (FP32 or FP64
 *           recursion and accumulation), bounds; r0, r_last NULL, doubling 0
 *   psi     [R][N] complex FP64 interleaved, host or device: psi(0) on entry,
 *           psi(nsteps dt) on return
 *   norms   [nsteps][R] FP64 <psi|psi> after every step (unitarity check), or NULL
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_TIMEOUT. */
int kite_propagate(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, double dt,
                   int nsteps, double* psi, double* norms, kite_stats* st);

/* The propagator's coefficients exp(-i de_plus dt) (2 - delta_n0) (-i)^n J_n(de_minus dt),
 * n < M, for the window [e_min, e_max] (host computation, no GPU): coef [M][2] complex.
 * Errors: KITE_ERR_ARG. */
int kite_evolution_coeffs(int M, double dt, double e_min, double e_max, double* coef);

/* Test hook for failure detection (no counterpart in the paper).  When `enable` is
 * non-zero, the first recursion step of the next kite_moments_1d call on this context
 * arms one shared-memory barrier of one CTA for 16 bytes more than it copies, so that
 * CTA's bounded wait gives up (after about a second), it drains its own copies and
 * returns, and the call reports KITE_ERR_TIMEOUT.  Nothing is accessed out of bounds,
 * no wait is unbounded, and the context stays usable.  The hook disarms itself.
 * Errors: KITE_ERR_ARG. */
int kite_debug_stall_once(kite_ctx* ctx, int enable);

/* ---- 2D moments ----------------------------------------------------------------- */

/* Velocity directions of the 2D moments. */
#define KITE_DIR_X 0
#define KITE_DIR_Y 1

/* 2D moments of the first-order Kubo-Bastin conductivity sigma_ab (Sec. 2b,
 * Eqs. cond 1st order, Gammanm, conductivity_1st_order):
 *   mu_nm = (1/(S R)) sum_{s,r} <r| v_a T_n(H~) v_b T_m(H~) |r> / N_eff,   v_d = -i h~d,
 * with h~d = [r_d, H~] applied matrix-free (positions in units of the lattice constant a;
 * honeycomb orbital positions of the paper's lattice set-up: a1 = (1, 0),
 * a2 = (1/2, sqrt(3)/2), A at (0, -a_cc/2), B at (0, a_cc/2), a_cc = 1/sqrt(3), so the
 * bond x-offsets are 0, +-1/2 and the y-offsets a_cc, -a_cc/2; square: +-1).  Computed as
 * mu_nm = <a_n|b_m> with the stored families a_n = T_n h~a r and b_m = h~b T_m r, and
 * contracted on the tensor cores (see kite_inner_products).  The paper's tensor is
 * Gamma^{a,b}_nm = -mu_nm / ((1 + delta_n0)(1 + delta_m0)).
 *   alpha, beta  KITE_DIR_X or KITE_DIR_Y (a and b above)
 *   kpm->precision must be KITE_FP32 (complex FP32 recursion, split-BF16 contraction,
 *   FP64 sums); kpm->r0 may give start vectors; kpm->r_last is ignored.
 *   mu_nm  [M][M] complex FP64 interleaved (re, im), row n, column m; host or device.
 * Work memory: about 24 * M * N bytes per pair of random vectors.
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_TIMEOUT,
 *         KITE_ERR_UNSUPPORTED (precision other than FP32). */
int kite_moments_2d(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, int alpha,
                    int beta, double* mu_nm, kite_stats* st);

/* ---- 2D moments: the contraction primitive ---------------------------------------- */

/* Complex inner products of two vector families, the contraction behind the 2D
 * Kubo-Bastin moments Gamma_nm = Tr[h T_n h T_m]/N (Sec. 2b, Eq. Gammanm):
 *   C[n][m] = scale * sum_{i<N} conj(A[n][i]) * B[m][i],   n < M, m < M2.
 * Runs on the tensor cores (tcgen05.mma): every FP32 input x is split into
 * bf16 hi = bf16(x) and lo = bf16(x - hi); products keep hi*hi + hi*lo + lo*hi
 * (`products` = 3) or also lo*lo (`products` = 4 or 0, the default).  Sums are FP32 inside
 * a K sub-chunk of `sub_k` products (sub_k = 0: default 512; the tensor core's FP32
 * accumulation drifts ~5e-9 per product for one-signed terms), then FP32 over `fold`
 * sub-chunks (fold = 0: default 16; 1 sends every sub-chunk to FP64 directly), and FP64
 * above that.
 *   A  [M][N]  complex FP32 interleaved (re, im), host or device
 *   B  [M2][N] complex FP32 interleaved, host or device
 *   C  [M][M2] complex FP64 interleaved, host or device (overwritten)
 * Device buffers are read and written on the context's stream: order any producer on
 * another stream before the call (e.g. bind the context to that stream).
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_TIMEOUT. */
int kite_inner_products(kite_ctx* ctx, const float* A, const float* B, int M, int M2, int64_t N,
                        double scale, double* C, int sub_k, int products, int fold);

/* Moments of many independent systems in one persistent, graph-captured launch (the S
 * realisations and the independent samples of Eq. PcomplexityFactor, batched).  Each
 * system i gives mu_i[n] = (1/R) sum_r <r|T_n(H~_i)|r>/N_eff,i for n < M_i, as
 * kite_moments_1d with S = 1.  Systems may differ in size, disorder, seed, bounds, M and
 * magnetic flux (a batch with a field in any system runs the Peierls variant of the
 * stencil, flux 0 as identity rotations); they share the lattice kind, R (1..8),
 * periodic boundaries and precision (KITE_FP32).  The CTAs of one
 * resident grid are grouped into teams: large systems get several CTAs that meet at a
 * bounded global barrier after each step, small ones share single-CTA teams.  The
 * set-up kernels, the sweep and the reductions are captured in one CUDA graph.
 *   systems, kpms  [count] arrays; kpms[i].S must be 1, r0 and r_last NULL; doubling
 *                  (0 or 1, see kite_kpm) the same for every system of the batch
 *   mu             [count] pointers, mu[i] -> [M_i] FP64 (host or device)
 *   st             statistics of the graph launch (seconds, updates, bytes), or NULL
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_BOUNDS, KITE_ERR_TIMEOUT,
 *         KITE_ERR_UNSUPPORTED (precision other than FP32). */
int kite_moments_1d_batched(kite_ctx* ctx, int count, const kite_system* systems,
                            const kite_kpm* kpms, double* const* mu, kite_stats* st);

/* ---- learned reconstruction (no counterpart in the paper) -------------------------- */

/* A multilayer perceptron KITE_MLP_IN -> KITE_MLP_HIDDEN -> KITE_MLP_HIDDEN -> KITE_MLP_OUT
 * (ReLU, BF16 weights and activations, FP32 accumulation on the tensor cores) that maps the
 * first KITE_MLP_IN Chebyshev moments of a system to its density of states on
 * KITE_MLP_OUT energies reconstructed from many more moments (the resolution of the
 * reconstruction scales as the inverse number of moments, Sec. 2a).  Parameters are one
 * flat FP32 vector W1[H][IN], b1[H], W2[H][H], b2[H], W3[OUT][H], b3[OUT] (row-major).
 * Inputs are normalised on the device as (x - shift[c]) * scale[c] with per-column
 * `shift` [IN] (NULL = 0) and `scale` [IN] (NULL = 1).  All pointers may be host or
 * device memory. */
#define KITE_MLP_IN 128
#define KITE_MLP_HIDDEN 512
#define KITE_MLP_OUT 1024

/* Optional residual prior of the network (NULL = none).  With KITE_PRIOR_JACKSON the
 * network's output is added to the Jackson reconstruction (Eq. e8a, Jackson kernel of
 * order KITE_MLP_IN) from the same first KITE_MLP_IN moments -- the raw X rows, before
 * shift and scale -- on the midpoint grid eps_j = -1 + (2j+1)/KITE_MLP_OUT of the window
 * [e_min, e_max] (density per eV, as kite_reconstruct_dos), so the network learns only
 * the correction that the many-moment reconstruction adds.  Training subtracts the same
 * prior from the targets. */
#define KITE_PRIOR_NONE 0
#define KITE_PRIOR_JACKSON 1
typedef struct {
  int32_t kind;      /* KITE_PRIOR_NONE or KITE_PRIOR_JACKSON                   */
  int32_t reserved;  /* must be 0                                               */
  double e_min;      /* energy window of the moments and the output grid (eV)   */
  double e_max;
} kite_mlp_prior;

typedef struct {
  int32_t epochs;       /* passes over the training set                      */
  int32_t batch;        /* rows per optimiser step                           */
  double lr;            /* peak learning rate (cosine schedule to zero)      */
  double weight_decay;  /* AdamW decoupled weight decay                      */
  uint64_t seed;        /* shuffling                                         */
} kite_mlp_train_cfg;

/* Number of FP32 parameters of the network. */
int64_t kite_mlp_param_count(void);

/* Trains in place: mean-absolute-error loss over X [n][IN] -> T [n][OUT], AdamW
 * (beta 0.9/0.999, eps 1e-8) on FP32 master weights, hand-written forward and backward
 * kernels.  params [P] holds the initial weights on entry and the trained ones on exit;
 * loss_curve [epochs] (or NULL) receives the mean training loss of each epoch.  prior
 * (or NULL) as above: the loss is taken on prior + network.
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_mlp_train(kite_ctx* ctx, const float* X, const float* T, int n, const float* shift,
                   const float* scale, const kite_mlp_train_cfg* cfg, float* params,
                   float* loss_curve, const kite_mlp_prior* prior);

/* Y [n][OUT] = network((X [n][IN] - shift) * scale) (+ the prior of X, if prior is not
 * NULL).  Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_mlp_forward(kite_ctx* ctx, const float* params, const float* X, int n,
                     const float* shift, const float* scale, float* Y,
                     const kite_mlp_prior* prior);

/* Gradient [P] of the mean absolute error over all n x OUT outputs (for checks), and the
 * loss.  Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_mlp_gradient(kite_ctx* ctx, const float* params, const float* X, const float* T, int n,
                      const float* shift, const float* scale, float* grad, double* loss);

/* Label-free consistency gate of predicted densities rho [n][OUT] (per eV, on the midpoint
 * grid eps_j = -1 + (2j+1)/OUT of the rescaled energy): the Chebyshev moments
 * m_k = int rho(eps) T_k(eps) d eps (midpoint rule) must match the known moments
 * mu [n][mu_ld] for k < kcheck within tol; flags[b] = 1 marks a prediction to replace by
 * the plain reconstruction.  deviation [n] (or NULL) receives max_k |m_k - mu_k|.
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_learned_gate(kite_ctx* ctx, const float* rho, const double* mu, int mu_ld, int n,
                      int kcheck, double e_min, double e_max, double tol, int* flags,
                      double* deviation);

/* One AdamW step of kite_mlp_train on caller arrays (for checks of the optimiser): with
 * the learning rate lr_t = lr (1 + cos(pi (t - 1) / total)) / 2 of step t (1-based) of a
 * cosine schedule over `total` steps and the bias corrections c1 = 1 - 0.9^t,
 * c2 = 1 - 0.999^t, every element i is updated in place as
 *   m = 0.9 m + 0.1 g,  v = 0.999 v + 0.001 g^2,
 *   p = p - lr_t ((m / c1) / (sqrt(v / c2) + 1e-8) + weight_decay p)
 * in FP32 -- the update kite_mlp_train applies after each batch (decoupled weight decay,
 * Loshchilov and Hutter).  params, m, v [n] FP32 (updated), grad [n] FP32; all host or
 * device.  Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_mlp_adamw_step(kite_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t n,
                        int t, int total, double lr, double weight_decay);

/* ---- learned reconstruction: trained model objects ------------------------------- */

/* A trained learned reconstructor owned by the library: its FP32 parameters, its input
 * normalisation (per-moment shift and scale, computed on the device from the training
 * set) and the energy window of its output grid, all in device memory of the GPU it was
 * trained on.  Created by kite_learned_train or kite_model_import, released by
 * kite_model_destroy; usable with any context on that GPU. */
typedef struct kite_model kite_model;

typedef struct {
  int32_t epochs;        /* passes over the training set (>= 1)                          */
  int32_t batch;         /* rows per optimiser step (>= 1)                               */
  double lr;             /* peak learning rate of the cosine schedule (> 0)             */
  double weight_decay;   /* AdamW decoupled weight decay (>= 0)                          */
  uint64_t seed;         /* shuffling; and the initial weights when init is NULL         */
  double e_min, e_max;   /* energy window (eV) of the moments and of the output grid     */
  const float* init;     /* [P] initial parameters (host or device), or NULL: He-uniform
                            weights drawn on the device from `seed` (Philox4x32-10,
                            counter (i_lo, i_hi, 0, 3)), zero biases                      */
  double head_scale;     /* NULL init only: the last layer's weights scaled by this
                            (0 = 1); a small value starts the residual network at its prior */
} kite_learned_cfg;

/* Trains a learned reconstructor on X [n][KITE_MLP_IN] (the first KITE_MLP_IN raw moments
 * mu_k of each training system, FP32) -> Y [n][KITE_MLP_OUT] (its density of states per eV
 * on the midpoint grid eps_j = -1 + (2j+1)/KITE_MLP_OUT of [e_min, e_max], from many more
 * moments).  The inputs are normalised by the training set's per-moment mean and
 * population standard deviation (floored at 1e-4), computed on the device; the network
 * learns the residual on the Jackson reconstruction of the same moments (KITE_PRIOR_JACKSON);
 * training is kite_mlp_train's (mean absolute error, AdamW, cosine schedule).
 *   X, Y        host or device
 *   out         receives the new model (NULL on failure)
 *   loss_curve  [epochs] mean training loss per epoch (host), or NULL
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_learned_train(kite_ctx* ctx, const float* X, const float* Y, int n, const kite_learned_cfg* cfg,
                       kite_model** out, float* loss_curve);

/* Densities of states from moments with the learned reconstructor, gated, with the plain
 * path as fallback -- in one call:
 *   1. rho_i = prior + network of the first KITE_MLP_IN moments of row i of mu;
 *   2. the consistency gate of kite_learned_gate: the first kcheck Chebyshev moments of
 *      rho_i must match mu_i within gate_tol (max abs difference), else row i falls back;
 *   3. a fallen-back row is replaced by the plain path's Jackson DOS from M_plain moments
 *      (Eq. e8a), on the same grid: with `systems` given, kite_moments_1d of systems[i]
 *      with plain_kpm (its M replaced by M_plain and its window by the model's) followed by
 *      kite_reconstruct_dos; with systems NULL, kite_reconstruct_dos of the first M_plain
 *      moments of mu's own row (then M_plain <= mu_ld).
 *   mu        [n][mu_ld] raw moments (FP64), host or device; mu_ld >= max(KITE_MLP_IN, kcheck),
 *             computed on the model's window
 *   gate_tol  >= 0; 0 sends every row whose moments are not reproduced exactly to the
 *             fallback (a forced fallback)
 *   systems   [n] (host) or NULL;  plain_kpm  required with systems (R, S, precision)
 *   rho       [n][KITE_MLP_OUT] FP32 per eV on the model's midpoint grid, host or device
 *   fell_back [n] 1 where the fallback replaced the prediction, host or device
 *   deviation [n] the gate's max |m_k - mu_k| per row, host or device, or NULL
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA, KITE_ERR_BOUNDS, KITE_ERR_TIMEOUT. */
int kite_learned_dos(kite_ctx* ctx, const kite_model* model, const double* mu, int mu_ld, int n,
                     double gate_tol, int kcheck, int M_plain, const kite_system* systems,
                     const kite_kpm* plain_kpm, float* rho, int* fell_back, double* deviation);

/* Copies a model's parameters [P], shift [KITE_MLP_IN], scale [KITE_MLP_IN] (each host or
 * device, or NULL) and window [2] = (e_min, e_max) (host, or NULL) out.
 * Errors: KITE_ERR_ARG, KITE_ERR_CUDA. */
int kite_model_export(const kite_model* model, float* params, float* shift, float* scale, double* window);

/* A model from saved parts (as kite_model_export gives them): params [P], shift and scale
 * [KITE_MLP_IN] (host or device; NULL = 0 and 1), window e_min < e_max.
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_model_import(kite_ctx* ctx, const float* params, const float* shift, const float* scale, double e_min,
                      double e_max, kite_model** out);

/* Releases a model (NULL is a no-op). */
void kite_model_destroy(kite_model* model);

/* ---- 1D moments without allocation (no counterpart in the paper) ------------------ */

/* kite_moments_1d for callers that cannot allocate device memory at the moment they need
 * moments: for example code running inside a host framework whose caching allocator has
 * already reserved the GPU's memory, or a latency-critical loop that must never wait on
 * the allocator.  It runs the same kernels as kite_moments_1d but keeps every intermediate
 * in one fixed 32 MiB array per GPU -- a file-scope __device__ variable of this library,
 * held by every GPU that loads the library until the process exits -- and calls no
 * cudaMalloc, cudaFree or other allocating routine, and needs no kite_ctx.
 *   sys, kpm   as for kite_moments_1d; e_min = e_max = 0 selects the Gershgorin bounds;
 *              R <= 8 (FP32) or 4 (FP64); kpm->r0 and kpm->r_last must be NULL and
 *              kpm->doubling 0
 *   mu         [M] FP64 moments (vector average), host or device, complete on return
 *   cuda_stream  stream the work is queued on (NULL = legacy default stream)
 *   err, err_len optional buffer for a one-line reason when the call fails
 * A system whose intermediates do not fit in 32 MiB is rejected with KITE_ERR_ARG and a
 * message giving the size it needs.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); the CUDA runtime loads the library's device code
 * lazily, so that first call is also when the 32 MiB are reserved on the device (and the
 * kernels' code is loaded): make it once at start-up, before the caller's framework
 * reserves the GPU's memory, and before any stream capture.  The address is looked up
 * again only if the device's context has been replaced (e.g. after cudaDeviceReset).
 * All calls share the array, which keeps the previous call's contents: each call clears
 * what must start at zero, but calls that overlap on the GPU (other streams or host
 * threads) race on it and must be serialised by the caller.
 * Errors: KITE_ERR_ARG, KITE_ERR_CUDA, KITE_ERR_BOUNDS, KITE_ERR_TIMEOUT. */
int kite_moments_1d_static(const kite_system* sys, const kite_kpm* kpm, double* mu,
                           void* cuda_stream, char* err, int err_len);

/* ---- reconstruction ------------------------------------------------------------- */

/* Density of states per orbital and per eV on caller energies (Eqs. e7, e8a with the
 * kernel damping mu_n -> g_n mu_n of Sec. 2a):
 *   eps = (E - de_plus)/de_minus;  rho(E) = [g_0 mu_0 + 2 sum_{n=1}^{M_use-1} g_n mu_n
 *   T_n(eps)] / (pi sqrt(1 - eps^2) de_minus), 0 outside |eps| < 1.
 * Computed in FP64 on the GPU.  M_use <= M_avail moments are used (Sec. 3c: a subset
 * of the computed moments), the kernel built for M = M_use.
 *   mu      [M_avail] FP64 raw moments, host or device
 *   kernel  KITE_KERNEL_NONE / _JACKSON / _LORENTZ (param = lambda for Lorentz)
 *   E       [K] energies (eV), host or device;  rho  [K] FP64 output, host or device
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_reconstruct_dos(kite_ctx* ctx, const double* mu, int M_avail, int M_use, int kernel,
                         double param, double e_min, double e_max, const double* E, int K,
                         double* rho);

/* Average Green's function per orbital at complex energy E + i eta, the eta-resolved
 * companion of the DOS (Eqs. green_function_cheb_expansion/b traced as in Eq. e7):
 *   G(E + i eta) = (1/de_minus) sum_{n<M_use} g_n mu_n / (1 + delta_n0) g^{+,eta~}_n(eps),
 * eps = (E - de_plus)/de_minus, eta~ = eta/de_minus, with the retarded Chebyshev
 * polynomial Green's function coefficients g^{+,eta~}_n(eps) = -2i exp(-i n arccos z) /
 * sqrt(1 - z^2), z = eps + i eta~, and an optional kernel g_n (as kite_reconstruct_dos).
 * FP64 on the GPU.  The series converges for M_use >> de_minus/eta.
 *   mu      [M_avail] raw moments (FP64), host or device
 *   eta     broadening in eV (> 0)
 *   E       [K] energies in eV, host or device
 *   G       [K] complex FP64 interleaved (re, im) in 1/eV, host or device, or NULL
 *   rho     [K] eta-broadened density -Im G / pi per eV, host or device, or NULL
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_reconstruct_green(kite_ctx* ctx, const double* mu, int M_avail, int M_use, int kernel,
                           double param, double e_min, double e_max, double eta,
                           const double* E, int K, double* G, double* rho);

/* Longitudinal DC conductivity at T = 0 in units of e^2/hbar per spin (Kubo-Greenwood:
 * the omega -> 0 limit of Eq. conductivity_1st_order, where only states at the Fermi
 * energy contribute) from the 2D moments mu_nm = <r|v T_n v T_m|r>/N of kite_moments_2d
 * with alpha = beta:
 *   sigma(E) = pi (n_orb a^2/Omega_c) sum_{n,m < M_use} c_n(e) c_m(e) Re mu_nm,
 *   c_n(e) = (2 - delta_n0) g_n T_n(e) / (pi sqrt(1 - e^2)),  e = (E - de_plus)/de_minus,
 * i.e. pi hbar e^2/Omega Tr[v delta(E-H) v delta(E-H)] with both delta functions expanded
 * in M_use kernel-damped Chebyshev terms (Sec. 2a); 0 outside the spectrum window.
 * n_orb a^2/Omega_c = 4/sqrt(3) (honeycomb), 1 (square).  FP64 on the GPU, fixed-order
 * sums.  The Fermi-sea (Hall) term of the DC Kubo-Bastin formula is not part of it: see
 * kite_reconstruct_sigma_dc_bastin.
 *   mu_nm   [M_avail][M_avail] complex FP64, host or device; the leading M_use block is used
 *   kernel  KITE_KERNEL_NONE / _JACKSON / _LORENTZ (param = lambda)
 *   E       [K] Fermi energies (eV), host or device;  sigma  [K] FP64, host or device
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_reconstruct_sigma_dc(kite_ctx* ctx, const double* mu_nm, int M_avail, int M_use, int lattice,
                              int kernel, double param, double e_min, double e_max, const double* E, int K,
                              double* sigma);

/* DC conductivity tensor element sigma_ab(E_F) in units of e^2/hbar per spin from the
 * Kubo-Bastin formula with its Fermi-sea term (the Hall conductivity of the quantum
 * anomalous Hall example and the omega -> 0 limit of Sec. 2b), from the 2D moments
 * mu_nm = <r|v_a T_n v_b T_m|r>/N of kite_moments_2d(alpha = a, beta = b):
 *   sigma_ab = Re{ i (n_orb a^2/Omega_c) int de f(e) sum_nm mu_nm
 *                    [Delta_n(e) dG^R_m(e)/de - dG^A_n(e)/de Delta_m(e)] },
 *   Delta_n(e) = k_n (2 - d_n0) T_n(e) / (pi sqrt(1 - e^2)),
 *   G^{R/A}_m(e) = k_m g^{+-}_m(e +- i eta~) / (1 + d_m0),
 * with the CPGF coefficients g of Eq. green_function_cheb_expansionb, eta~ = eta/de_minus,
 * k_n the kernel (KITE_KERNEL_NONE: 1) and f the Fermi function.  The finite eta keeps
 * the integrand regular at the band edges; the Fermi sea is the rescaled band [-1, e_F]
 * (kT = 0) or the whole band weighted by f (kT > 0, eV), integrated by Gauss-Legendre
 * quadrature in theta (e = cos theta) with n_quad nodes per energy (0: 2 M_use + 64).
 * With a magnetic field in the moments it gives the quantum Hall plateaus.  FP64 on the
 * GPU; two M_use x M_use x n_quad GEMMs per Fermi energy.
 *   mu_nm  [M_avail][M_avail] complex FP64, host or device; the leading M_use block is used
 *   kernel KITE_KERNEL_NONE / _JACKSON / _LORENTZ (param = lambda)
 *   eta    broadening in eV (> 0);  kT  temperature in eV (>= 0)
 *   E_F    [K] Fermi energies (eV), host or device;  sigma  [K] FP64, host or device
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_reconstruct_sigma_dc_bastin(kite_ctx* ctx, const double* mu_nm, int M_avail, int M_use, int lattice,
                                     int kernel, double param, double e_min, double e_max, double eta, double kT,
                                     const double* E_F, int K, int n_quad, double* sigma);

/* First-order optical conductivity sigma_xx(omega) in units of e^2/hbar from the 2D
 * moments of kite_moments_2d (Sec. 2b, Eqs. Gammanm and conductivity_1st_order, in
 * rescaled units w = hbar omega / de_minus, eta in eV):
 *   Gamma_nm = -g_n g_m mu_nm / ((1 + d_n0)(1 + d_m0)),
 *   Lambda_nm(w) = int de f(e) [g^R_n(e + w) Delta_m(e) + Delta_n(e) g^A_m(e - w)],
 *   sigma(w) = -i (n_orb a^2 / Omega_c) / w * sum_nm Lambda_nm(w) Gamma_nm,
 * with the CPGF coefficients g^{R/A}_n of Eq. green_function_cheb_expansionb and the
 * Fermi-sea integral done by Gauss-Legendre quadrature in theta (e = cos theta) with
 * n_quad nodes (0: 2 M_use + 64).  kT = 0 integrates [E_min, E_F]; kT > 0 (eV) weights the
 * whole band by the Fermi function.  n_orb a^2/Omega_c = 4/sqrt(3) (honeycomb), 1 (square).
 * The diamagnetic term sum_n Lambda_n Gamma^xx_n (purely imaginary for omega > 0) is not
 * included: Re sigma is complete, Im sigma lacks it.  kernel = KITE_KERNEL_JACKSON damps
 * both indices (use with eta -> 0, the KPM Kubo-Bastin form); KITE_KERNEL_NONE with
 * eta > 0 is the CPGF form.  All arithmetic FP64 on the GPU.
 *   mu_nm  [M_avail][M_avail] complex FP64, host or device; the leading M_use x M_use
 *          block is used
 *   omega  [K] photon energies hbar*omega (eV, > 0), host or device
 *   sigma  [K] complex FP64 output, host or device
 * Errors: KITE_ERR_ARG, KITE_ERR_OOM, KITE_ERR_CUDA. */
int kite_reconstruct_sigma(kite_ctx* ctx, const double* mu_nm, int M_avail, int M_use,
                           int lattice, int kernel, double e_min, double e_max, double E_F,
                           double kT, double eta, const double* omega, int K, int n_quad,
                           double* sigma);

#ifdef __cplusplus
}
#endif
#endif /* KITE_GB_H */
