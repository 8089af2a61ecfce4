/*
 * kite_oracle.c -- plain FP64 CPU reference for the stochastic Chebyshev moments of
 * KITE (arXiv:1910.05194).  TEST INFRASTRUCTURE ONLY: the CUDA library never links,
 * includes or calls this file; only tests, the smoke check and the benchmark's
 * CPU-baseline leg do.
 *
 * Every routine is a direct transcription of a definition in the paper (cited per
 * function), written for readability, not speed: per-site loops, no blocking, no
 * fusion.  Compile with -ffp-contract=off so that a*b+c is never fused behind the
 * source's back (the FP32/FP64 "replica" below spells out its fused operations).
 */
#include "kite_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------ */
/* Counter-based random numbers.  The paper only asks for white-noise variables    */
/* (Sec. 2c, stochastic trace evaluation); the generator chosen for this project is */
/* Philox4x32-10 from Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as     */
/* easy as 1, 2, 3" (SC'11): 10 rounds of two 32x32->64 multiplies, key bumped by    */
/* the Weyl constants between rounds.                                               */
/* ------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Stream tags: which quantity a Philox block belongs to (fourth counter word). */
#define ORC_TAG_DISORDER 0x1u
#define ORC_TAG_PHASE 0x2u

/* 53-bit uniform in [0,1) from the first two output words. */
static double orc_u53(const uint32_t x[4]) {
  uint64_t k = ((uint64_t)x[0] << 21) | (uint64_t)(x[1] >> 11);
  return (double)k * 0x1p-53;
}

static void orc_draw(const orc_system* sys, uint64_t o, uint32_t word2, uint32_t tag,
                     uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)o, (uint32_t)(o >> 32), word2, tag};
  uint32_t key[2] = {(uint32_t)sys->seed, (uint32_t)(sys->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* Largest |z| a Gaussian draw below can take: u1 >= 2^-53, so
 * |z| <= sqrt(-2 ln 2^-53) = sqrt(106 ln 2) = 8.5717...; bounds use 8.58. */
#define ORC_GAUSS_ZMAX 8.58

/* On-site energy of orbital o from its disorder draw x (Sec. 4b: Anderson disorder,
 * uniform in [-W/2, W/2]; the Python interface of Sec. 3d also offers Gaussian disorder
 * with a mean and a standard deviation).  Gaussian: the Box-Muller transform of the
 * 53-bit uniform u1 = 1 - u (in (0, 1]) and the 32-bit uniform u2 of the fourth word,
 * z = sqrt(-2 ln u1) cos(2 pi u2), V = W z.  The staggered term adds +delta/2 on A and
 * -delta/2 on B (a sublattice mean).  The third word decides vacancies. */
static double orc_onsite(const orc_system* sys, int64_t o, const uint32_t x[4]) {
  double u = orc_u53(x);
  double v;
  if (sys->disorder == 1) {
    double u1 = 1.0 - u;
    double u2 = (double)x[3] * 0x1p-32;
    v = sys->W * (sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  } else {
    v = sys->W * (u - 0.5);
  }
  if (sys->lattice == 0 && sys->delta != 0.0) {
    double half = 0.5 * sys->delta;
    v = v + ((o & 1) == 0 ? half : -half);
  }
  return v;
}

/* ------------------------------------------------------------------------------ */
/* Lattice geometry (Listing 1 of Sec. 3d: honeycomb with a1=[a,0], a2=[a/2,a*sqrt3/2], */
/* A at [0,-acc/2], B at [0,acc/2], hoppings (0,0) A-B, (1,-1) A-B, (0,-1) A-B).       */
/* ------------------------------------------------------------------------------ */
int64_t orc_norb(const orc_system* sys) {
  int64_t cells = (int64_t)sys->Lx * (int64_t)sys->Ly;
  return sys->lattice == 0 ? 2 * cells : cells;
}

static int64_t orc_wrap(int64_t v, int64_t L) {
  int64_t r = v % L;
  return r < 0 ? r + L : r;
}

/* Neighbours of orbital o in a fixed order, with the x-component (in units of a)
 * of the bond vector r_o - r_j used by the velocity operator h~x = [x, H]
 * (Sec. 2b, generalised velocity with n = 1).  Returns the coordination number. */
/* Neighbours of orbital o with the bond offsets (x_o - x_j, y_o - y_j) in units of the
 * lattice constant a.  Honeycomb (the paper's lattice set-up listing): a1 = (1, 0),
 * a2 = (1/2, sqrt(3)/2), A at (0, -a_cc/2) and B at (0, +a_cc/2) in each cell with
 * a_cc = 1/sqrt(3); bonds A(x,y) - B(x+dx1, y+dx2) for cell offsets (0,0), (1,-1), (0,-1).
 * Square: a1 = (1, 0), a2 = (0, 1).  Periodic boundaries wrap the cell indices; with an
 * open boundary (the configuration's boundaries flag set to False, Sec. 3d) a bond whose
 * cell offset leaves [0, L) along that direction is absent: its neighbour index is -1. */
static int orc_neighbours_geo(const orc_system* sys, int64_t o, int64_t nb[4], double dx[4],
                              double dy[4]) {
  int64_t Lx = sys->Lx, Ly = sys->Ly;
  if (sys->lattice == 0) {
    const double acc = 1.0 / sqrt(3.0);
    int64_t cell = o >> 1, s = o & 1;
    int64_t x = cell % Lx, y = cell / Lx;
    const int ox = sys->open_x, oy = sys->open_y;
    if (s == 0) { /* A(x,y) -> B(x,y), B(x+1,y-1), B(x,y-1) */
      nb[0] = 2 * (y * Lx + x) + 1;
      nb[1] = 2 * (orc_wrap(y - 1, Ly) * Lx + orc_wrap(x + 1, Lx)) + 1;
      nb[2] = 2 * (orc_wrap(y - 1, Ly) * Lx + x) + 1;
      if ((ox && x + 1 == Lx) || (oy && y == 0)) nb[1] = -1;
      if (oy && y == 0) nb[2] = -1;
      dx[0] = 0.0;
      dx[1] = -0.5;
      dx[2] = 0.5;
      dy[0] = -acc;
      dy[1] = 0.5 * acc;
      dy[2] = 0.5 * acc;
    } else { /* B(x,y) -> A(x,y), A(x-1,y+1), A(x,y+1) */
      nb[0] = 2 * (y * Lx + x);
      nb[1] = 2 * (orc_wrap(y + 1, Ly) * Lx + orc_wrap(x - 1, Lx));
      nb[2] = 2 * (orc_wrap(y + 1, Ly) * Lx + x);
      if ((ox && x == 0) || (oy && y + 1 == Ly)) nb[1] = -1;
      if (oy && y + 1 == Ly) nb[2] = -1;
      dx[0] = 0.0;
      dx[1] = 0.5;
      dx[2] = -0.5;
      dy[0] = acc;
      dy[1] = -0.5 * acc;
      dy[2] = -0.5 * acc;
    }
    return 3;
  }
  int64_t x = o % Lx, y = o / Lx;
  nb[0] = (sys->open_x && x == 0) ? -1 : y * Lx + orc_wrap(x - 1, Lx);
  nb[1] = (sys->open_x && x + 1 == Lx) ? -1 : y * Lx + orc_wrap(x + 1, Lx);
  nb[2] = (sys->open_y && y == 0) ? -1 : orc_wrap(y - 1, Ly) * Lx + x;
  nb[3] = (sys->open_y && y + 1 == Ly) ? -1 : orc_wrap(y + 1, Ly) * Lx + x;
  dx[0] = 1.0;
  dx[1] = -1.0;
  dx[2] = 0.0;
  dx[3] = 0.0;
  dy[0] = 0.0;
  dy[1] = 0.0;
  dy[2] = 1.0;
  dy[3] = -1.0;
  return 4;
}

int orc_neighbours(const orc_system* sys, int64_t o, int64_t nb[4]) {
  double dx[4], dy[4];
  return orc_neighbours_geo(sys, o, nb, dx, dy);
}

/* Spectral bounds.  The paper rescales H into [-1,1] with the endpoints of the
 * spectrum (Eqs. rescalingH/rescalingE) and warns that estimated endpoints can be
 * wrong (Sec. 4b).  Gershgorin's theorem gives a rigorous enclosure:
 * |E| <= Z|t| + max|V|, with max|V| = W/2 + |delta|/2 (uniform) or
 * ORC_GAUSS_ZMAX W + |delta|/2 (Gaussian: the largest draw the transform can give);
 * a 1% margin is added. */
void orc_bounds_auto(const orc_system* sys, double* e_min, double* e_max) {
  double Z = sys->lattice == 0 ? 3.0 : 4.0;
  double vd = sys->disorder == 1 ? ORC_GAUSS_ZMAX * fabs(sys->W) : 0.5 * fabs(sys->W);
  double vmax = vd + (sys->lattice == 0 ? 0.5 * fabs(sys->delta) : 0.0);
  double b = (Z * fabs(sys->t) + vmax) * 1.01;
  *e_min = -b;
  *e_max = b;
}

/* On-site energies and vacancies for one disorder realisation (orc_onsite).  A vacancy
 * removes the orbital (Sec. 3a: defects as position lists); here each orbital is vacant
 * with probability p_vac. */
void orc_disorder(const orc_system* sys, int realisation, double* V, uint8_t* vac) {
  int64_t N = orc_norb(sys);
  double thr_d = floor(sys->p_vac * 4294967296.0);
  uint64_t thr = sys->p_vac <= 0.0 ? 0 : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
  for (int64_t o = 0; o < N; ++o) {
    uint32_t x[4];
    orc_draw(sys, (uint64_t)o, (uint32_t)realisation, ORC_TAG_DISORDER, x);
    V[o] = orc_onsite(sys, o, x);
    vac[o] = ((uint64_t)x[2] < thr) ? 1 : 0;
  }
}

/* Random-phase vectors |r> = sum_i xi_i |i> with unit-modulus xi_i = exp(2 pi i u)
 * (Sec. 2c, white-noise variables; zero on removed orbitals). */
void orc_random_phase(const orc_system* sys, int realisation, int R, const uint8_t* vac,
                      double* r0) {
  int64_t N = orc_norb(sys);
  const double two_pi = 6.283185307179586;
  for (int r = 0; r < R; ++r) {
    for (int64_t o = 0; o < N; ++o) {
      double* z = r0 + 2 * ((int64_t)r * N + o);
      if (vac[o]) {
        z[0] = 0.0;
        z[1] = 0.0;
        continue;
      }
      uint32_t x[4];
      uint32_t w2 = (uint32_t)realisation * (uint32_t)R + (uint32_t)r;
      orc_draw(sys, (uint64_t)o, w2, ORC_TAG_PHASE, x);
      double phi = two_pi * orc_u53(x);
      z[0] = cos(phi);
      z[1] = sin(phi);
    }
  }
}

/* Real white-noise start vectors (Sec. 2c allows real or complex variables): the sign
 * +-1 of the same draw as the phase, +1 when u < 1/2; 0 on vacant orbitals.  Written as
 * complex values with zero imaginary part, [R][N]. */
void orc_random_real(const orc_system* sys, int realisation, int R, const uint8_t* vac,
                     double* r0) {
  int64_t N = orc_norb(sys);
  for (int r = 0; r < R; ++r) {
    for (int64_t o = 0; o < N; ++o) {
      double* z = r0 + 2 * ((int64_t)r * N + o);
      z[1] = 0.0;
      if (vac[o]) {
        z[0] = 0.0;
        continue;
      }
      uint32_t x[4];
      uint32_t w2 = (uint32_t)realisation * (uint32_t)R + (uint32_t)r;
      orc_draw(sys, (uint64_t)o, w2, ORC_TAG_PHASE, x);
      z[0] = orc_u53(x) < 0.5 ? 1.0 : -1.0;
    }
  }
}

/* ------------------------------------------------------------------------------ */
/* 1D moments: the plain FP64 definition.                                            */
/*   H~ = (H - de_plus)/de_minus                         (Eq. rescalingH)            */
/*   T_0 r = r, T_1 r = H~ r, T_{n+1} r = 2 H~ T_n r - T_{n-1} r     (Eq. e6)         */
/*   mu_n = <r0 | T_n(H~) | r0> / N_eff                  (Eqs. e7-e8, Sec. 2c STE)   */
/* ------------------------------------------------------------------------------ */
typedef struct {
  int64_t N;
  int Z;
  int64_t* nb;   /* [N][4] */
  double* dx;    /* [N][4] bond offsets x_o - x_j */
  double* dy;    /* [N][4] bond offsets y_o - y_j */
  double* Vt;    /* rescaled on-site */
  uint8_t* vac;
  double tt;     /* rescaled hopping */
  int64_t n_eff;
  double* ph;    /* [N][4] (cos, sin) of the Peierls phase of each bond; NULL without field */
} orc_ham;

/* Magnetic field (Sec. "Magnetic Field": Peierls substitution on a periodic lattice).
 * Landau gauge A = (-B y, 0): the hopping from orbital j to orbital o (bond offset
 * (dx, dy) = r_o - r_j) becomes t exp(i theta) with
 *   theta = (2 pi / Phi_0) int_{r_j}^{r_o} A . dl = -2 pi (flux / A_cell) (y_o - dy/2) dx,
 * the line integral along the straight bond (y at its midpoint), flux = B A_cell / Phi_0
 * per unit cell, A_cell = sqrt(3)/2 (honeycomb) or 1 (square) in units of a^2, and y_o
 * the orbital's y coordinate.  The phases repeat after Ly rows only if
 * flux * Ly * |dx| is an integer for every bond (|dx| = 1/2 on the honeycomb, 1 on the
 * square lattice): otherwise the bonds across the y boundary would not be the
 * conjugates of their reverses.  Bonds with dx = 0 carry no phase. */
int orc_flux_fits(const orc_system* sys) {
  if (sys->flux == 0.0 || sys->open_y) return 0; /* no bond wraps in y: any flux fits */
  double q = sys->flux * (double)sys->Ly * (sys->lattice == 0 ? 0.5 : 1.0);
  return fabs(q - nearbyint(q)) <= 1e-9 * fmax(1.0, fabs(q)) ? 0 : -4;
}

static double orc_orbital_y(const orc_system* sys, int64_t o) {
  if (sys->lattice == 0) {
    int64_t cell = o >> 1, s = o & 1;
    double acc = 1.0 / sqrt(3.0);
    return 0.5 * sqrt(3.0) * (double)(cell / sys->Lx) + (s == 0 ? -0.5 : 0.5) * acc;
  }
  return (double)(o / sys->Lx);
}

/* Peierls phases of every bond of h (geometry already filled in), or h->ph = NULL without
 * a field.  0, -2 (allocation) or -4 (flux does not fit the torus). */
static int orc_ham_phases(orc_ham* h, const orc_system* sys) {
  h->ph = NULL;
  if (sys->flux == 0.0) return 0;
  if (orc_flux_fits(sys)) return -4;
  h->ph = (double*)malloc(sizeof(double) * 8 * h->N);
  if (!h->ph) return -2;
  const double cell_area = sys->lattice == 0 ? 0.5 * sqrt(3.0) : 1.0;
  const double k = -2.0 * 3.141592653589793 * sys->flux / cell_area;
  for (int64_t o = 0; o < h->N; ++o) {
    double yo = orc_orbital_y(sys, o);
    for (int b = 0; b < 4; ++b) {
      double th = b < h->Z ? k * (yo - 0.5 * h->dy[4 * o + b]) * h->dx[4 * o + b] : 0.0;
      h->ph[8 * o + 2 * b] = cos(th);
      h->ph[8 * o + 2 * b + 1] = sin(th);
    }
  }
  return 0;
}

static int orc_ham_build(orc_ham* h, const orc_system* sys, int realisation, double e_min,
                         double e_max) {
  h->N = orc_norb(sys);
  h->nb = (int64_t*)malloc(sizeof(int64_t) * 4 * h->N);
  h->dx = (double*)malloc(sizeof(double) * 4 * h->N);
  h->dy = (double*)malloc(sizeof(double) * 4 * h->N);
  h->Vt = (double*)malloc(sizeof(double) * h->N);
  h->vac = (uint8_t*)malloc(h->N);
  if (!h->nb || !h->dx || !h->dy || !h->Vt || !h->vac) return -2;
  double de_plus = 0.5 * (e_max + e_min);
  double de_minus = 0.5 * (e_max - e_min);
  double* V = h->Vt;
  orc_disorder(sys, realisation, V, h->vac);
  h->n_eff = 0;
  for (int64_t o = 0; o < h->N; ++o) {
    h->Z = orc_neighbours_geo(sys, o, h->nb + 4 * o, h->dx + 4 * o, h->dy + 4 * o);
    h->Vt[o] = (V[o] - de_plus) / de_minus;
    if (!h->vac[o]) h->n_eff++;
  }
  h->tt = sys->t / de_minus;
  return orc_ham_phases(h, sys);
}

static void orc_ham_free(orc_ham* h) {
  free(h->nb);
  free(h->dx);
  free(h->dy);
  free(h->Vt);
  free(h->vac);
  free(h->ph);
}

/* y = H~ x on the non-vacant orbitals (vacant rows and columns removed). */
static void orc_apply_h(const orc_ham* h, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t o = 0; o < h->N; ++o) {
    if (h->vac[o]) {
      y[2 * o] = 0.0;
      y[2 * o + 1] = 0.0;
      continue;
    }
    double re = h->Vt[o] * x[2 * o], im = h->Vt[o] * x[2 * o + 1];
    for (int k = 0; k < h->Z; ++k) {
      int64_t j = h->nb[4 * o + k];
      if (j < 0 || h->vac[j]) continue; /* no bond across an open boundary */
      double xr = x[2 * j], xi = x[2 * j + 1];
      if (h->ph) { /* t exp(i theta) x_j */
        double c = h->ph[8 * o + 2 * k], sn = h->ph[8 * o + 2 * k + 1];
        double r2 = c * xr - sn * xi;
        xi = sn * xr + c * xi;
        xr = r2;
      }
      re += h->tt * xr;
      im += h->tt * xi;
    }
    y[2 * o] = re;
    y[2 * o + 1] = im;
  }
}

/* <a|b> = sum conj(a) b over all orbitals. */
static void orc_dot(int64_t N, const double* a, const double* b, double* re, double* im) {
  double sr = 0.0, si = 0.0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
  for (int64_t o = 0; o < N; ++o) {
    sr += a[2 * o] * b[2 * o] + a[2 * o + 1] * b[2 * o + 1];
    si += a[2 * o] * b[2 * o + 1] - a[2 * o + 1] * b[2 * o];
  }
  *re = sr;
  *im = si;
}

static void orc_start_vectors(const orc_system* sys, int realisation, int R, const orc_ham* h,
                              const double* r0_in, double* r0) {
  int64_t N = h->N;
  if (r0_in) {
    memcpy(r0, r0_in, sizeof(double) * 2 * N * R);
    for (int r = 0; r < R; ++r)
      for (int64_t o = 0; o < N; ++o)
        if (h->vac[o]) {
          r0[2 * ((int64_t)r * N + o)] = 0.0;
          r0[2 * ((int64_t)r * N + o) + 1] = 0.0;
        }
  } else {
    orc_random_phase(sys, realisation, R, h->vac, r0);
  }
}

/* out = sum_{n<M} coef_n T_n(H~) in  (complex coef [M][2], in/out [N][2]); the plain
 * recursion of Eq. e6 with vacant orbitals removed.  Used for the time-evolution operator
 * of the wave-packet section: U(t) = exp(-i de_plus t) [c_0 + 2 sum_n c_n T_n(H~)],
 * c_n = (-i)^n J_n(de_minus t). */
int orc_chebyshev_sum(const orc_system* sys, int realisation, double e_min, double e_max, int M,
                      const double* coef, const double* in, double* out) {
  if (M < 1 || !(e_max > e_min)) return -1;
  orc_ham h;
  if (orc_ham_build(&h, sys, realisation, e_min, e_max)) return -2;
  int64_t N = h.N;
  double* prev = (double*)malloc(sizeof(double) * 2 * N);
  double* cur = (double*)malloc(sizeof(double) * 2 * N);
  double* nxt = (double*)malloc(sizeof(double) * 2 * N);
  if (!prev || !cur || !nxt) return -2;
  for (int64_t o = 0; o < N; ++o) {  /* T_0 in, vacancies removed */
    double re = h.vac[o] ? 0.0 : in[2 * o], im = h.vac[o] ? 0.0 : in[2 * o + 1];
    prev[2 * o] = re;
    prev[2 * o + 1] = im;
    out[2 * o] = coef[0] * re - coef[1] * im;
    out[2 * o + 1] = coef[0] * im + coef[1] * re;
  }
  if (M > 1) orc_apply_h(&h, prev, cur);
  for (int n = 1; n < M; ++n) {
    const double cr = coef[2 * n], ci = coef[2 * n + 1];
    for (int64_t o = 0; o < N; ++o) {
      out[2 * o] += cr * cur[2 * o] - ci * cur[2 * o + 1];
      out[2 * o + 1] += cr * cur[2 * o + 1] + ci * cur[2 * o];
    }
    if (n + 1 < M) {
      orc_apply_h(&h, cur, nxt);
      for (int64_t k = 0; k < 2 * N; ++k) nxt[k] = 2.0 * nxt[k] - prev[k];
      double* t = prev;
      prev = cur;
      cur = nxt;
      nxt = t;
    }
  }
  free(prev);
  free(cur);
  free(nxt);
  orc_ham_free(&h);
  return 0;
}

int orc_moments_1d(const orc_system* sys, int realisation, int M, int R, double e_min,
                   double e_max, const double* r0_in, double* mu_per_vec, int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  if (M < 1 || R < 1 || sys->Lx < 1 || sys->Ly < 1 || !(e_max > e_min)) return -1;
  orc_ham h;
  if (orc_ham_build(&h, sys, realisation, e_min, e_max)) return -2;
  int64_t N = h.N;
  double* r0 = (double*)malloc(sizeof(double) * 2 * N * R);
  double* prev = (double*)malloc(sizeof(double) * 2 * N);
  double* cur = (double*)malloc(sizeof(double) * 2 * N);
  double* nxt = (double*)malloc(sizeof(double) * 2 * N);
  if (!r0 || !prev || !cur || !nxt) return -2;
  orc_start_vectors(sys, realisation, R, &h, r0_in, r0);
  double inv = h.n_eff > 0 ? 1.0 / (double)h.n_eff : 0.0;
  for (int r = 0; r < R; ++r) {
    const double* v0 = r0 + 2 * (int64_t)r * N;
    double* mu = mu_per_vec + 2 * (int64_t)r * M;
    double re, im;
    orc_dot(N, v0, v0, &re, &im);
    mu[0] = re * inv;
    mu[1] = im * inv;
    if (M < 2) continue;
    memcpy(prev, v0, sizeof(double) * 2 * N);
    orc_apply_h(&h, prev, cur); /* T_1 r0 = H~ r0 */
    orc_dot(N, v0, cur, &re, &im);
    mu[2] = re * inv;
    mu[3] = im * inv;
    for (int n = 1; n + 1 < M; ++n) {
      orc_apply_h(&h, cur, nxt);
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < 2 * N; ++k) nxt[k] = 2.0 * nxt[k] - prev[k];
      orc_dot(N, v0, nxt, &re, &im);
      mu[2 * (n + 1)] = re * inv;
      mu[2 * (n + 1) + 1] = im * inv;
      double* tmp = prev;
      prev = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
  free(r0);
  free(prev);
  free(cur);
  free(nxt);
  orc_ham_free(&h);
  return 0;
}

/* ------------------------------------------------------------------------------ */
/* Replica of the recursion at a fixed precision with a fixed rounding sequence.    */
/* The paper offers float and double vectors (Sec. 3d, Configuration precision=0/1); */
/* this project pins the order of operations of one site update so that any         */
/* implementation of it can be compared bit for bit:                                */
/*   s  = (nb1 + nb2) + nb3  [+ nb4 on the square lattice], neighbours in the order */
/*        of orc_neighbours_dx, vacant neighbours and absent bonds (open boundaries) */
/*        read as zero;                                                              */
/*   r_1     = fma(t~, s, V~ * r_self)     (one rounding for the product V~*r);     */
/*   r_{n+1} = fma(2t~, s, fma(2V~, r_self, -r_{n-1}))  for n >= 1,                  */
/* i.e. Eq. e6's 2 H~ r_n - r_{n-1} with the factor 2 taken into t~ and V~ (exact    */
/* in binary floating point) and the subtraction fused with the on-site product;   */
/* vacant orbitals stay exactly zero.  V~ and t~ are computed in FP64 and rounded   */
/* once to the working precision; start vectors are rounded once.  Moments are     */
/* accumulated in FP64 (order-free).                                                 */
/* ------------------------------------------------------------------------------ */
#define ORC_REPLICA(REAL, FMA)                                                               \
  static void orc_replica_step_##REAL(const orc_ham* h, REAL tt, const REAL* vt,            \
                                      const REAL* cur, const REAL* prev, REAL* out,          \
                                      int first) {                                           \
    _Pragma("omp parallel for schedule(static)")                                             \
    for (int64_t o = 0; o < h->N; ++o) {                                                     \
      for (int c = 0; c < 2; ++c) {                                                          \
        REAL v;                                                                              \
        if (h->vac[o]) {                                                                     \
          v = (REAL)0;                                                                       \
        } else {                                                                             \
          const int64_t* q = h->nb + 4 * o;                                                  \
          REAL s = (q[0] < 0 ? (REAL)0 : cur[2 * q[0] + c]) +                                \
                   (q[1] < 0 ? (REAL)0 : cur[2 * q[1] + c]);                                 \
          s = s + (q[2] < 0 ? (REAL)0 : cur[2 * q[2] + c]);                                  \
          if (h->Z == 4) s = s + (q[3] < 0 ? (REAL)0 : cur[2 * q[3] + c]);                   \
          if (first) {                                                                       \
            REAL p = vt[o] * cur[2 * o + c];                                                 \
            v = FMA(tt, s, p);                                                               \
          } else {                                                                           \
            REAL tt2 = tt + tt, vt2 = vt[o] + vt[o];                                         \
            v = FMA(tt2, s, FMA(vt2, cur[2 * o + c], -prev[2 * o + c]));                     \
          }                                                                                  \
        }                                                                                    \
        out[2 * o + c] = v;                                                                  \
      }                                                                                      \
    }                                                                                        \
  }                                                                                          \
  static void orc_replica_dot_##REAL(int64_t N, const REAL* a, const REAL* b, double* re,   \
                                     double* im) {                                           \
    double sr = 0.0, si = 0.0;                                                               \
    _Pragma("omp parallel for reduction(+ : sr, si) schedule(static)")                       \
    for (int64_t o = 0; o < N; ++o) {                                                        \
      double ar = a[2 * o], ai = a[2 * o + 1], br = b[2 * o], bi = b[2 * o + 1];             \
      sr += ar * br + ai * bi;                                                               \
      si += ar * bi - ai * br;                                                               \
    }                                                                                        \
    *re = sr;                                                                                \
    *im = si;                                                                                \
  }

ORC_REPLICA(float, fmaf)
ORC_REPLICA(double, fma)

#define ORC_REPLICA_RUN(REAL)                                                                \
  {                                                                                          \
    REAL* vt = (REAL*)malloc(sizeof(REAL) * N);                                              \
    REAL* v0 = (REAL*)malloc(sizeof(REAL) * 2 * N);                                          \
    REAL* a = (REAL*)malloc(sizeof(REAL) * 2 * N);                                           \
    REAL* b = (REAL*)malloc(sizeof(REAL) * 2 * N);                                           \
    REAL* c = (REAL*)malloc(sizeof(REAL) * 2 * N);                                           \
    REAL tt = (REAL)h.tt;                                                                    \
    for (int64_t o = 0; o < N; ++o) vt[o] = h.vac[o] ? (REAL)0 : (REAL)h.Vt[o];            \
    for (int r = 0; r < R; ++r) {                                                            \
      double* mu = mu_per_vec + 2 * (int64_t)r * M;                                          \
      for (int64_t k = 0; k < 2 * N; ++k) v0[k] = (REAL)r0[2 * (int64_t)r * N + k];          \
      REAL *prev = v0, *cur = v0, *nxt = a, *spare = b;                                      \
      double re, im;                                                                         \
      orc_replica_dot_##REAL(N, v0, v0, &re, &im);                                           \
      mu[0] = re * inv;                                                                      \
      mu[1] = im * inv;                                                                      \
      REAL* last_prev = v0;                                                                  \
      REAL* last_cur = v0;                                                                   \
      if (M >= 2) {                                                                          \
        orc_replica_step_##REAL(&h, tt, vt, v0, v0, a, 1);                                   \
        orc_replica_dot_##REAL(N, v0, a, &re, &im);                                          \
        mu[2] = re * inv;                                                                    \
        mu[3] = im * inv;                                                                    \
        prev = v0;                                                                           \
        cur = a;                                                                             \
        nxt = b;                                                                             \
        spare = c;                                                                           \
        for (int n = 1; n + 1 < M; ++n) {                                                    \
          orc_replica_step_##REAL(&h, tt, vt, cur, prev, nxt, 0);                            \
          orc_replica_dot_##REAL(N, v0, nxt, &re, &im);                                      \
          mu[2 * (n + 1)] = re * inv;                                                        \
          mu[2 * (n + 1) + 1] = im * inv;                                                    \
          REAL* freed = (prev == v0) ? spare : prev;                                         \
          prev = cur;                                                                        \
          cur = nxt;                                                                         \
          nxt = freed;                                                                       \
        }                                                                                    \
        last_prev = prev;                                                                    \
        last_cur = cur;                                                                      \
      }                                                                                      \
      if (r_last) {                                                                          \
        REAL* dst = (REAL*)r_last + 4 * (int64_t)r * N;                                      \
        memcpy(dst, last_prev, sizeof(REAL) * 2 * N);                                        \
        memcpy(dst + 2 * N, last_cur, sizeof(REAL) * 2 * N);                                 \
      }                                                                                      \
    }                                                                                        \
    free(vt);                                                                                \
    free(v0);                                                                                \
    free(a);                                                                                 \
    free(b);                                                                                 \
    free(c);                                                                                 \
  }

/* r_last (optional): per vector the last two iterates [r_{M-2}, r_{M-1}] as interleaved
 * complex values of the working precision: r_last[(r*2 + k)*2N ...]. */
int orc_replica_1d(const orc_system* sys, int realisation, int M, int R, double e_min,
                   double e_max, int precision, const double* r0_in, double* mu_per_vec,
                   void* r_last, int threads) {
  if (sys->flux != 0.0) return -3; /* built without Peierls phases */
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  if (M < 1 || R < 1 || sys->Lx < 1 || sys->Ly < 1 || !(e_max > e_min)) return -1;
  if (precision != 0 && precision != 1) return -1;
  orc_ham h;
  if (orc_ham_build(&h, sys, realisation, e_min, e_max)) return -2;
  int64_t N = h.N;
  double* r0 = (double*)malloc(sizeof(double) * 2 * N * R);
  if (!r0) return -2;
  orc_start_vectors(sys, realisation, R, &h, r0_in, r0);
  double inv = h.n_eff > 0 ? 1.0 / (double)h.n_eff : 0.0;
  if (precision == 0) ORC_REPLICA_RUN(float) else ORC_REPLICA_RUN(double)
  free(r0);
  orc_ham_free(&h);
  return 0;
}

/* ------------------------------------------------------------------------------ */
/* Velocity operator and 2D moments.                                                 */
/*   h~x = (i hbar) h^x = [x, H]   (Sec. 2b, Eq. generalized velocity and the tilde  */
/*   convention), so (h~x)_ij = (x_i - x_j) H_ij: real and antisymmetric.  Here x is  */
/*   in units of the lattice constant a and H is the rescaled H~, so physical          */
/*   velocities carry a factor a * de_minus.                                          */
/*   Gamma^{x,x}_nm = Tr[h~ T_n h~ T_m]/N / ((1+d_n0)(1+d_m0))  (Eq. Gammanm)         */
/*   With a_n = T_n(H~) h~ r and b_m = h~ T_m(H~) r and h~^dagger = -h~,              */
/*   <r|h~ T_n h~ T_m|r> = -<a_n|b_m>.  The routine returns                            */
/*   mu_nm = <a_n|b_m>/N_eff averaged over vectors, i.e. <r|v T_n v T_m|r>/N_eff for   */
/*   v = -i h~ (= i[H,x]); Gamma_nm = -mu_nm/((1+d_n0)(1+d_m0)).                       */
/* ------------------------------------------------------------------------------ */
/* y = h~ x with h~ = [r_dir, H~] (dir 0: x, 1: y): (h~)_oj = (r_o - r_j) H~_oj over the
 * bonds (Sec. 2b, the velocity operator v = i[H, r] = -i h~ in units of the lattice
 * constant). */
static void orc_apply_v(const orc_ham* h, int dir, const double* x, double* y) {
  const double* off = dir ? h->dy : h->dx;
#pragma omp parallel for schedule(static)
  for (int64_t o = 0; o < h->N; ++o) {
    double re = 0.0, im = 0.0;
    if (!h->vac[o]) {
      for (int k = 0; k < h->Z; ++k) {
        int64_t j = h->nb[4 * o + k];
        if (j < 0 || h->vac[j]) continue;
        double w = off[4 * o + k] * h->tt;
        double xr = x[2 * j], xi = x[2 * j + 1];
        if (h->ph) { /* [r, H~]_oj = (r_o - r_j) t~ exp(i theta_oj) */
          double c = h->ph[8 * o + 2 * k], sn = h->ph[8 * o + 2 * k + 1];
          double r2 = c * xr - sn * xi;
          xi = sn * xr + c * xi;
          xr = r2;
        }
        re += w * xr;
        im += w * xi;
      }
    }
    y[2 * o] = re;
    y[2 * o + 1] = im;
  }
}

void orc_velocity(const orc_system* sys, const uint8_t* vac, double t_scaled, int dir,
                  const double* in, double* out) {
  orc_ham h;
  h.N = orc_norb(sys);
  h.nb = (int64_t*)malloc(sizeof(int64_t) * 4 * h.N);
  h.dx = (double*)malloc(sizeof(double) * 4 * h.N);
  h.dy = (double*)malloc(sizeof(double) * 4 * h.N);
  h.vac = (uint8_t*)vac;
  h.tt = t_scaled;
  for (int64_t o = 0; o < h.N; ++o)
    h.Z = orc_neighbours_geo(sys, o, h.nb + 4 * o, h.dx + 4 * o, h.dy + 4 * o);
  if (orc_ham_phases(&h, sys) == 0) orc_apply_v(&h, dir, in, out);
  free(h.nb);
  free(h.dx);
  free(h.dy);
  free(h.ph);
}

void orc_velocity_x(const orc_system* sys, const uint8_t* vac, double t_scaled,
                    const double* in, double* out) {
  orc_velocity(sys, vac, t_scaled, 0, in, out);
}

/* Runs the recursion from `start`, storing T_n(H~) start for n < M into fam[n]. */
static void orc_family(const orc_ham* h, int M, const double* start, double* fam,
                       double* work) {
  int64_t N = h->N;
  double* prev = work;
  double* cur = work + 2 * N;
  double* nxt = work + 4 * N;
  memcpy(fam, start, sizeof(double) * 2 * N);
  if (M < 2) return;
  orc_apply_h(h, start, fam + 2 * N);
  memcpy(prev, start, sizeof(double) * 2 * N);
  memcpy(cur, fam + 2 * N, sizeof(double) * 2 * N);
  for (int n = 2; n < M; ++n) {
    orc_apply_h(h, cur, nxt);
    for (int64_t k = 0; k < 2 * N; ++k) nxt[k] = 2.0 * nxt[k] - prev[k];
    memcpy(fam + 2 * N * (int64_t)n, nxt, sizeof(double) * 2 * N);
    double* tmp = prev;
    prev = cur;
    cur = nxt;
    nxt = tmp;
  }
}

/* mu_nm[(n*M + m)*2 + {re,im}]; optional a_fam/b_fam receive the last vector's
 * families [M][N] complex (for inspection in tests). */
int orc_moments_2d(const orc_system* sys, int realisation, int M, int R, double e_min,
                   double e_max, const double* r0_in, double* mu_nm, double* a_fam,
                   double* b_fam, int dir_a, int dir_b, int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  if (M < 1 || R < 1 || sys->Lx < 1 || sys->Ly < 1 || !(e_max > e_min)) return -1;
  orc_ham h;
  if (orc_ham_build(&h, sys, realisation, e_min, e_max)) return -2;
  int64_t N = h.N;
  double* r0 = (double*)malloc(sizeof(double) * 2 * N * R);
  double* A = (double*)malloc(sizeof(double) * 2 * N * M);
  double* B = (double*)malloc(sizeof(double) * 2 * N * M);
  double* T = (double*)malloc(sizeof(double) * 2 * N * M);
  double* work = (double*)malloc(sizeof(double) * 6 * N);
  double* start = (double*)malloc(sizeof(double) * 2 * N);
  if (!r0 || !A || !B || !T || !work || !start) return -2;
  orc_start_vectors(sys, realisation, R, &h, r0_in, r0);
  memset(mu_nm, 0, sizeof(double) * 2 * (int64_t)M * M);
  double inv = h.n_eff > 0 ? 1.0 / ((double)h.n_eff * (double)R) : 0.0;
  for (int r = 0; r < R; ++r) {
    const double* v0 = r0 + 2 * (int64_t)r * N;
    orc_apply_v(&h, dir_a, v0, start);
    orc_family(&h, M, start, A, work); /* a_n = T_n h~a r */
    orc_family(&h, M, v0, T, work);    /* T_m r           */
    for (int m = 0; m < M; ++m) orc_apply_v(&h, dir_b, T + 2 * N * (int64_t)m, B + 2 * N * (int64_t)m);
    /* plain triple loop: mu_nm += sum_o conj(a_n[o]) b_m[o] */
#pragma omp parallel for schedule(static)
    for (int n = 0; n < M; ++n) {
      const double* a = A + 2 * N * (int64_t)n;
      for (int m = 0; m < M; ++m) {
        const double* b = B + 2 * N * (int64_t)m;
        double sr = 0.0, si = 0.0;
        for (int64_t o = 0; o < N; ++o) {
          sr += a[2 * o] * b[2 * o] + a[2 * o + 1] * b[2 * o + 1];
          si += a[2 * o] * b[2 * o + 1] - a[2 * o + 1] * b[2 * o];
        }
        mu_nm[2 * ((int64_t)n * M + m)] += sr * inv;
        mu_nm[2 * ((int64_t)n * M + m) + 1] += si * inv;
      }
    }
    if (r == R - 1) {
      if (a_fam) memcpy(a_fam, A, sizeof(double) * 2 * N * M);
      if (b_fam) memcpy(b_fam, B, sizeof(double) * 2 * N * M);
    }
  }
  free(r0);
  free(A);
  free(B);
  free(T);
  free(work);
  free(start);
  orc_ham_free(&h);
  return 0;
}

/* Selected rows and columns of the same mu_nm, for lattices whose families do not fit
 * in memory: rows[i] < M give out_rows[i][m] = mu_{rows[i], m} for every m < M, and
 * cols[j] < M give out_cols[n][j] = mu_{n, cols[j]} for every n < M.  Per vector, in
 * three passes of the plain recursion: the a-recursion keeps the a_n of the chosen rows;
 * the T_m r recursion forms every b_m = h~b T_m r, dots it with the kept a's and keeps the
 * b_m of the chosen columns; a second a-recursion dots every a_n with the kept b's. */
int orc_moments_2d_panels(const orc_system* sys, int realisation, int M, int R, double e_min,
                          double e_max, const int* rows, int nrows, const int* cols, int ncols,
                          int dir_a, int dir_b, double* out_rows, double* out_cols, int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  if (M < 1 || R < 1 || nrows < 0 || ncols < 0 || !(e_max > e_min)) return -1;
  for (int i = 0; i < nrows; ++i)
    if (rows[i] < 0 || rows[i] >= M) return -1;
  for (int j = 0; j < ncols; ++j)
    if (cols[j] < 0 || cols[j] >= M) return -1;
  orc_ham h;
  if (orc_ham_build(&h, sys, realisation, e_min, e_max)) return -2;
  int64_t N = h.N;
  double* r0 = (double*)malloc(sizeof(double) * 2 * N * R);
  double* keep_a = (double*)malloc(sizeof(double) * 2 * N * (nrows > 0 ? nrows : 1));
  double* keep_b = (double*)malloc(sizeof(double) * 2 * N * (ncols > 0 ? ncols : 1));
  double* start = (double*)malloc(sizeof(double) * 2 * N);
  double* prev = (double*)malloc(sizeof(double) * 2 * N);
  double* cur = (double*)malloc(sizeof(double) * 2 * N);
  double* nxt = (double*)malloc(sizeof(double) * 2 * N);
  double* b = (double*)malloc(sizeof(double) * 2 * N);
  if (!r0 || !keep_a || !keep_b || !start || !prev || !cur || !nxt || !b) return -2;
  orc_start_vectors(sys, realisation, R, &h, NULL, r0);
  memset(out_rows, 0, sizeof(double) * 2 * (int64_t)nrows * M);
  memset(out_cols, 0, sizeof(double) * 2 * (int64_t)M * ncols);
  double inv = h.n_eff > 0 ? 1.0 / ((double)h.n_eff * (double)R) : 0.0;
  for (int r = 0; r < R; ++r) {
    const double* v0 = r0 + 2 * (int64_t)r * N;
    for (int pass = 0; pass < 3; ++pass) {
      /* passes 0 and 2 run T_n (h~a r); pass 1 runs T_m r */
      if (pass == 1) memcpy(start, v0, sizeof(double) * 2 * N);
      else orc_apply_v(&h, dir_a, v0, start);
      memcpy(prev, start, sizeof(double) * 2 * N);
      for (int n = 0; n < M; ++n) {
        const double* x; /* T_n start */
        if (n == 0) {
          x = prev;
        } else if (n == 1) {
          orc_apply_h(&h, prev, cur);
          x = cur;
        } else {
          orc_apply_h(&h, cur, nxt);
          for (int64_t k = 0; k < 2 * N; ++k) nxt[k] = 2.0 * nxt[k] - prev[k];
          double* t = prev;
          prev = cur;
          cur = nxt;
          nxt = t;
          x = cur;
        }
        if (pass == 0) {
          for (int i = 0; i < nrows; ++i)
            if (rows[i] == n) memcpy(keep_a + 2 * N * (int64_t)i, x, sizeof(double) * 2 * N);
        } else if (pass == 1) {
          orc_apply_v(&h, dir_b, x, b); /* b_n = h~b T_n r */
          for (int i = 0; i < nrows; ++i) {
            double sr, si;
            orc_dot(N, keep_a + 2 * N * (int64_t)i, b, &sr, &si);
            out_rows[2 * ((int64_t)i * M + n)] += sr * inv;
            out_rows[2 * ((int64_t)i * M + n) + 1] += si * inv;
          }
          for (int j = 0; j < ncols; ++j)
            if (cols[j] == n) memcpy(keep_b + 2 * N * (int64_t)j, b, sizeof(double) * 2 * N);
        } else {
          for (int j = 0; j < ncols; ++j) {
            double sr, si;
            orc_dot(N, x, keep_b + 2 * N * (int64_t)j, &sr, &si);
            out_cols[2 * ((int64_t)n * ncols + j)] += sr * inv;
            out_cols[2 * ((int64_t)n * ncols + j) + 1] += si * inv;
          }
        }
      }
    }
  }
  free(r0);
  free(keep_a);
  free(keep_b);
  free(start);
  free(prev);
  free(cur);
  free(nxt);
  free(b);
  orc_ham_free(&h);
  return 0;
}

/* ------------------------------------------------------------------------------ */
/* Reconstruction.                                                                   */
/* ------------------------------------------------------------------------------ */

/* Jackson kernel (Weisse et al., Rev. Mod. Phys. 78, 275 (2006), cited by the paper  */
/* for the kernel polynomial method in Sec. 2a):                                      */
/*   g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))] / (M+1).         */
void orc_kernel_jackson(int M, double* g) {
  const double pi = 3.141592653589793;
  double q = pi / (double)(M + 1);
  double cot = cos(q) / sin(q);
  for (int n = 0; n < M; ++n)
    g[n] = ((double)(M - n + 1) * cos(q * n) + sin(q * n) * cot) / (double)(M + 1);
}

/* Lorentz kernel, Sec. 2a: g_n = sinh(lambda (1 - n/M)) / sinh(lambda). */
void orc_kernel_lorentz(int M, double lambda, double* g) {
  for (int n = 0; n < M; ++n) g[n] = sinh(lambda * (1.0 - (double)n / (double)M)) / sinh(lambda);
}

/* Density of states per orbital and per unit energy (Eqs. e7, e8a with the delta-
 * function expansion of Sec. 2a): for eps = (E - de_plus)/de_minus in (-1,1),
 *   rho(eps) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(eps)] / (pi sqrt(1 - eps^2)),
 *   rho(E)   = rho(eps) / de_minus,     rho = 0 outside the band |eps| >= 1.
 * g = NULL means no kernel (g_n = 1).  T_n(eps) follows Eq. e3. */
void orc_dos(const double* mu, int M, const double* g, double e_min, double e_max,
             const double* E, int K, double* rho) {
  const double pi = 3.141592653589793;
  double de_plus = 0.5 * (e_max + e_min), de_minus = 0.5 * (e_max - e_min);
  for (int k = 0; k < K; ++k) {
    double eps = (E[k] - de_plus) / de_minus;
    if (!(eps > -1.0 && eps < 1.0)) {
      rho[k] = 0.0;
      continue;
    }
    double tm1 = 1.0, t = eps;
    double sum = (g ? g[0] : 1.0) * mu[0];
    for (int n = 1; n < M; ++n) {
      sum += 2.0 * (g ? g[n] : 1.0) * mu[n] * t;
      double tn = 2.0 * eps * t - tm1;
      tm1 = t;
      t = tn;
    }
    rho[k] = sum / (pi * sqrt(1.0 - eps * eps)) / de_minus;
  }
}

/* CPGF coefficient of the resolvent expansion (Eq. green_function_cheb_expansionb):
 *   g_n^{sigma,eta}(eps) = -2 sigma i exp(-sigma i n arccos(eps + i sigma eta))
 *                          / sqrt(1 - (eps + i sigma eta)^2),   sigma = +1 (R), -1 (A). */
void orc_cpgf_coeff(int n, double eps, double eta, int sigma, double* re, double* im) {
  double s = (double)sigma;
  double complex z = eps + s * eta * I;
  double complex theta = cacos(z);
  double complex num = cexp(-s * I * (double)n * theta);
  double complex den = csqrt(1.0 - z * z);
  double complex gval = -2.0 * s * I * num / den;
  *re = creal(gval);
  *im = cimag(gval);
}

/* ------------------------------------------------------------------------------ */
/* Replica iterates at one site of a large periodic lattice, computed on a window.   */
/* The stencil couples nearest neighbours only, so T_n(H~) r at an orbital depends   */
/* only on orbitals within n hops (finite propagation of the recursion, Eq. e6).     */
/* Each hop moves the cell by at most one step in x and in y, so a window of          */
/* half-width h >= M cells around (x0, y0), with neighbours outside the window read   */
/* as zero, reproduces the global recursion exactly at its centre.  Draws use the    */
/* global orbital indices, so the window sees the global disorder, vacancies and     */
/* random phases.  out: [R][2][orbitals per cell] complex of the working precision,  */
/* the last two iterates (r_{M-2}, r_{M-1}) at the cell (x0, y0).                    */
/* ------------------------------------------------------------------------------ */
int orc_replica_window(const orc_system* sys, int realisation, int M, int R, double e_min,
                       double e_max, int precision, int x0, int y0, int half, void* out) {
  if (sys->flux != 0.0) return -3; /* built without Peierls phases */
  if (sys->open_x || sys->open_y) return -3; /* periodic lattices only */
  if (M < 1 || R < 1 || half < M || !(e_max > e_min)) return -1;
  if (precision != 0 && precision != 1) return -1;
  const int sorb = sys->lattice == 0 ? 2 : 1;
  const int w = 2 * half + 1;
  const int64_t nw = (int64_t)w * w * sorb;
  double de_plus = 0.5 * (e_max + e_min), de_minus = 0.5 * (e_max - e_min);
  double tt = sys->t / de_minus;
  int64_t* gidx = (int64_t*)malloc(sizeof(int64_t) * nw);
  int64_t* nb = (int64_t*)malloc(sizeof(int64_t) * 4 * nw); /* -1 = outside the window */
  double* vt = (double*)malloc(sizeof(double) * nw);
  uint8_t* vac = (uint8_t*)malloc(nw);
  double* r0 = (double*)malloc(sizeof(double) * 2 * nw * R);
  if (!gidx || !nb || !vt || !vac || !r0) return -2;
  double thr_d = floor(sys->p_vac * 4294967296.0);
  uint64_t thr = sys->p_vac <= 0.0 ? 0 : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
  const double two_pi = 6.283185307179586;
  for (int wy = 0; wy < w; ++wy)
    for (int wx = 0; wx < w; ++wx)
      for (int s = 0; s < sorb; ++s) {
        int64_t l = ((int64_t)wy * w + wx) * sorb + s;
        int64_t gx = orc_wrap((int64_t)x0 - half + wx, sys->Lx);
        int64_t gy = orc_wrap((int64_t)y0 - half + wy, sys->Ly);
        int64_t o = (gy * sys->Lx + gx) * sorb + s;
        gidx[l] = o;
        uint32_t x[4];
        orc_draw(sys, (uint64_t)o, (uint32_t)realisation, ORC_TAG_DISORDER, x);
        double v = orc_onsite(sys, o, x);
        vac[l] = ((uint64_t)x[2] < thr) ? 1 : 0;
        vt[l] = (v - de_plus) / de_minus;
        for (int r = 0; r < R; ++r) {
          double* z = r0 + 2 * ((int64_t)r * nw + l);
          if (vac[l]) {
            z[0] = z[1] = 0.0;
            continue;
          }
          uint32_t y[4];
          orc_draw(sys, (uint64_t)o, (uint32_t)realisation * (uint32_t)R + (uint32_t)r,
                   ORC_TAG_PHASE, y);
          double phi = two_pi * orc_u53(y);
          z[0] = cos(phi);
          z[1] = sin(phi);
        }
        /* neighbours in the order of orc_neighbours_dx, in window coordinates */
        int64_t* q = nb + 4 * l;
        q[0] = q[1] = q[2] = q[3] = -1;
#define ORC_WIN(X, Y, S) (((X) < 0 || (X) >= w || (Y) < 0 || (Y) >= w) ? -1 : (((int64_t)(Y) * w + (X)) * sorb + (S)))
        if (sys->lattice == 0) {
          if (s == 0) {
            q[0] = ORC_WIN(wx, wy, 1);
            q[1] = ORC_WIN(wx + 1, wy - 1, 1);
            q[2] = ORC_WIN(wx, wy - 1, 1);
          } else {
            q[0] = ORC_WIN(wx, wy, 0);
            q[1] = ORC_WIN(wx - 1, wy + 1, 0);
            q[2] = ORC_WIN(wx, wy + 1, 0);
          }
        } else {
          q[0] = ORC_WIN(wx - 1, wy, 0);
          q[1] = ORC_WIN(wx + 1, wy, 0);
          q[2] = ORC_WIN(wx, wy - 1, 0);
          q[3] = ORC_WIN(wx, wy + 1, 0);
        }
#undef ORC_WIN
      }
  const int Z = sys->lattice == 0 ? 3 : 4;
  const int64_t centre = ((int64_t)half * w + half) * sorb;
#define ORC_WINDOW_RUN(REAL, FMA)                                                           \
  {                                                                                         \
    REAL* a = (REAL*)malloc(sizeof(REAL) * 2 * nw);                                         \
    REAL* b = (REAL*)malloc(sizeof(REAL) * 2 * nw);                                         \
    REAL* c = (REAL*)malloc(sizeof(REAL) * 2 * nw);                                         \
    REAL tr = (REAL)tt;                                                                     \
    for (int r = 0; r < R; ++r) {                                                           \
      REAL *prev = a, *cur = b, *nxt = c;                                                   \
      for (int64_t k = 0; k < 2 * nw; ++k) cur[k] = (REAL)r0[2 * (int64_t)r * nw + k];      \
      memcpy(prev, cur, sizeof(REAL) * 2 * nw);                                             \
      for (int n = 0; n + 1 < M; ++n) {                                                     \
        for (int64_t l = 0; l < nw; ++l)                                                    \
          for (int cc = 0; cc < 2; ++cc) {                                                  \
            REAL v;                                                                         \
            if (vac[l]) {                                                                   \
              v = (REAL)0;                                                                  \
            } else {                                                                        \
              const int64_t* q = nb + 4 * l;                                                \
              REAL n1 = q[0] < 0 ? (REAL)0 : cur[2 * q[0] + cc];                            \
              REAL n2 = q[1] < 0 ? (REAL)0 : cur[2 * q[1] + cc];                            \
              REAL n3 = q[2] < 0 ? (REAL)0 : cur[2 * q[2] + cc];                            \
              REAL s = n1 + n2;                                                             \
              s = s + n3;                                                                   \
              if (Z == 4) s = s + (q[3] < 0 ? (REAL)0 : cur[2 * q[3] + cc]);                \
              REAL vr = (REAL)vt[l];                                                        \
              if (n == 0) {                                                                 \
                v = FMA(tr, s, vr * cur[2 * l + cc]);                                       \
              } else {                                                                      \
                REAL tr2 = tr + tr, vr2 = vr + vr;                                          \
                v = FMA(tr2, s, FMA(vr2, cur[2 * l + cc], -prev[2 * l + cc]));              \
              }                                                                             \
            }                                                                               \
            nxt[2 * l + cc] = v;                                                            \
          }                                                                                 \
        REAL* tmp = prev;                                                                   \
        prev = cur;                                                                         \
        cur = nxt;                                                                          \
        nxt = tmp;                                                                          \
      }                                                                                     \
      REAL* dst = (REAL*)out + (int64_t)r * 2 * sorb * 2;                                   \
      for (int s = 0; s < sorb; ++s) {                                                      \
        dst[2 * s] = prev[2 * (centre + s)];                                                \
        dst[2 * s + 1] = prev[2 * (centre + s) + 1];                                        \
        dst[2 * sorb + 2 * s] = cur[2 * (centre + s)];                                      \
        dst[2 * sorb + 2 * s + 1] = cur[2 * (centre + s) + 1];                              \
      }                                                                                     \
    }                                                                                       \
    free(a);                                                                                \
    free(b);                                                                                \
    free(c);                                                                                \
  }
  if (precision == 0) ORC_WINDOW_RUN(float, fmaf) else ORC_WINDOW_RUN(double, fma)
#undef ORC_WINDOW_RUN
  free(gidx);
  free(nb);
  free(vt);
  free(vac);
  free(r0);
  return 0;
}
