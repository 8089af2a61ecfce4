/*
 * kite_oracle.h -- plain, slow, obviously-correct CPU reference for the stochastic
 * Chebyshev (kernel polynomial) moments of KITE (arXiv:1910.05194).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code: only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no header, helper or constant table with the CUDA library; the two sides
 * meet only through the published definitions they both implement.
 *
 * Conventions (each function cites the passage it follows):
 *   - orbital index o = 2*(y*Lx + x) + s (honeycomb, s=0 is A, s=1 is B) or
 *     o = y*Lx + x (square), periodic boundaries in both directions;
 *   - complex vectors are stored as interleaved (re, im) doubles, vector-major:
 *     v[(r*N + o)*2 + {0,1}];
 *   - moments are stored raw, mu_n = <r0|T_n(H~)|r0> / N_eff (mu_0 = 1), the
 *     (2 - delta_n0) weight is applied only in the reconstruction (Sec. 2a, Eqs. e4/e7).
 */
#ifndef KITE_ORACLE_H
#define KITE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t lattice;   /* 0 = honeycomb (Listing 1), 1 = square                          */
  int32_t Lx, Ly;    /* unit cells along a1 and a2                                      */
  int32_t disorder;  /* 0: uniform (Anderson) in [-W/2, W/2]; 1: Gaussian, mean 0, s.d. W */
  double t;          /* nearest-neighbour hopping (eV)                                  */
  double W;          /* on-site disorder strength (eV): uniform width or Gaussian s.d.   */
  double delta;      /* staggered potential +delta/2 on A, -delta/2 on B (eV)          */
  double p_vac;      /* per-orbital vacancy probability                                 */
  uint64_t seed;
  double flux;       /* perpendicular magnetic flux per unit cell, in flux quanta h/e;   */
                     /* flux * Ly must be even (honeycomb) or an integer (square) when   */
                     /* y is periodic                                                    */
  int32_t open_x;    /* 1: open boundary along a1 (the bonds that wrap in x are absent)  */
  int32_t open_y;    /* 1: open boundary along a2 (the bonds that wrap in y are absent)  */
} orc_system;

/* 0 if the flux fits the torus in the Landau gauge (see orc_flux_fits), else -4. */
int orc_flux_fits(const orc_system* sys);

/* Philox4x32-10 counter-based generator (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

int64_t orc_norb(const orc_system* sys);
int orc_neighbours(const orc_system* sys, int64_t o, int64_t nb[4]);
void orc_bounds_auto(const orc_system* sys, double* e_min, double* e_max);
void orc_disorder(const orc_system* sys, int realisation, double* V, uint8_t* vac);
void orc_random_phase(const orc_system* sys, int realisation, int R, const uint8_t* vac,
                      double* r0);
void orc_random_real(const orc_system* sys, int realisation, int R, const uint8_t* vac,
                     double* r0);

int orc_moments_1d(const orc_system* sys, int realisation, int M, int R, double e_min,
                   double e_max, const double* r0_in, double* mu_per_vec, int threads);

int orc_replica_1d(const orc_system* sys, int realisation, int M, int R, double e_min,
                   double e_max, int precision, const double* r0_in, double* mu_per_vec,
                   void* r_last, int threads);

int orc_replica_window(const orc_system* sys, int realisation, int M, int R, double e_min,
                       double e_max, int precision, int x0, int y0, int half, void* out);

void orc_velocity_x(const orc_system* sys, const uint8_t* vac, double t_scaled,
                    const double* in, double* out);
void orc_velocity(const orc_system* sys, const uint8_t* vac, double t_scaled, int dir,
                  const double* in, double* out);
int orc_moments_2d(const orc_system* sys, int realisation, int M, int R, double e_min,
                   double e_max, const double* r0_in, double* mu_nm, double* a_fam,
                   double* b_fam, int dir_a, int dir_b, int threads);
int orc_moments_2d_panels(const orc_system* sys, int realisation, int M, int R, double e_min,
                          double e_max, const int* rows, int nrows, const int* cols, int ncols,
                          int dir_a, int dir_b, double* out_rows, double* out_cols, int threads);

int orc_chebyshev_sum(const orc_system* sys, int realisation, double e_min, double e_max, int M,
                      const double* coef, const double* in, double* out);
void orc_kernel_jackson(int M, double* g);
void orc_kernel_lorentz(int M, double lambda, double* g);
void orc_dos(const double* mu, int M, const double* g, double e_min, double e_max,
             const double* E, int K, double* rho);
void orc_cpgf_coeff(int n, double eps, double eta, int sigma, double* re, double* im);

#ifdef __cplusplus
}
#endif
#endif
