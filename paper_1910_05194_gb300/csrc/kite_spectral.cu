// kite_spectral.cu -- moments from deterministic start vectors: the k-resolved spectral
// function (the paper's spectral-function section, the quantity behind ARPES) and the
// local density of states (its LDOS section).
//
// Instead of a random vector the recursion starts from the plane wave
//   |k> = sum_alpha w_alpha sum_i exp(i k.R_i^alpha) |i, alpha>,
// or from one orbital |i, alpha>, and mu_n = <v|T_n(H~)|v> / norm, so that rho_k(E) and
// rho_i(E) follow from the same Jackson reconstruction as the DOS.  The start vectors are
// written on the device (FP64, the caller-vector layout of the 1D sweep) a batch at a
// time and the sweep itself is the 1D moment path.
#include <math.h>

#include <algorithm>
#include <vector>

#include "kite_internal.h"

namespace kite {

int moments_1d_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
                    double* mu_dev, double* imag_dev, double* mu_vec_dev, kite_stats* st,
                    const double* r0_dev_all);

namespace {

// r0[s][j][o] = w_alpha exp(i k_j . R_o) for the k-points k0 .. k0+nk-1, copied for the S
// realisations.  Orbital positions in units of the lattice constant: honeycomb cell (x, y)
// at x a1 + y a2, a1 = (1, 0), a2 = (1/2, sqrt(3)/2), A at (0, -a_cc/2), B at (0, +a_cc/2),
// a_cc = 1/sqrt(3) (the paper's lattice set-up); square (x, y).
__global__ void k_plane_waves(int lattice, int Lx, int64_t N, const double* __restrict__ k, int k0,
                              int nk, const double* __restrict__ w, int S, double* __restrict__ r0) {
  const int64_t total = (int64_t)nk * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / N);
    const int64_t o = e - (int64_t)j * N;
    double X, Y;
    int alpha = 0;
    if (lattice == KITE_HONEYCOMB) {
      const int64_t cell = o >> 1;
      alpha = (int)(o & 1);
      const double x = (double)(cell % Lx), y = (double)(cell / Lx);
      X = x + 0.5 * y;
      Y = 0.8660254037844386 * y + (alpha == 0 ? -0.5 : 0.5) * 0.5773502691896258;
    } else {
      X = (double)(o % Lx);
      Y = (double)(o / Lx);
    }
    const double kx = k[2 * (k0 + j)], ky = k[2 * (k0 + j) + 1];
    double sn, cs;
    sincos(kx * X + ky * Y, &sn, &cs);
    const double wr = w ? w[2 * alpha] : 1.0, wi = w ? w[2 * alpha + 1] : 0.0;
    const double re = wr * cs - wi * sn, im = wr * sn + wi * cs;
    for (int s = 0; s < S; ++s) {
      double* z = r0 + 2 * (((int64_t)s * nk + j) * N + o);
      z[0] = re;
      z[1] = im;
    }
  }
}

// r0[s][j] = |orbital o_j> (1 at the orbital, 0 elsewhere) for the sites j0 .. j0+n-1
__global__ void k_basis_vectors(int64_t N, const int64_t* __restrict__ orb, int j0, int n, int S,
                                double* __restrict__ r0) {
  const int64_t total = (int64_t)S * n * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e % N;
    const int j = (int)((e / N) % n);
    r0[2 * e] = o == orb[j0 + j] ? 1.0 : 0.0;
    r0[2 * e + 1] = 0.0;
  }
}

// out[k0 + j][n] = scale * (1/S) sum_s mu_vec[s*nk + j][n]  (complex)
__global__ void k_spectral_avg(const double* __restrict__ mu_vec, int S, int nk, int M, int k0,
                               double scale, double* __restrict__ out) {
  const int64_t total = (int64_t)nk * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / M), n = (int)(e - (e / M) * M);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < S; ++s) {
      const double* p = mu_vec + 2 * (((int64_t)s * nk + j) * M + n);
      re += p[0];
      im += p[1];
    }
    out[2 * ((int64_t)(k0 + j) * M + n)] = scale * re / S;
    out[2 * ((int64_t)(k0 + j) * M + n) + 1] = scale * im / S;
  }
}

}  // namespace

// Moments of nv deterministic start vectors, a sweep batch at a time: gen(j0, n, r0) writes
// the S copies of vectors j0 .. j0+n-1 into r0 ([S][n][N][2] FP64); out [nv][M][2] gets
// the realisation average times `scale` (the sweep normalises by N_eff).
template <typename Gen>
int deterministic_moments(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
                          int nv, double scale, Gen gen, double* out, kite_stats* st) {
  const int M = kpm->M, S = kpm->S;
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  const int chunk = kpm->precision == KITE_FP64 ? 4 : 8;  // one sweep batch of vectors
  const int nc = std::min(chunk, nv);
  double* buf = nullptr;
  const size_t r0_n = 2 * (size_t)S * nc * N, mv_n = 2 * (size_t)S * nc * M;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, sizeof(double) * (r0_n + mv_n + 2 * (size_t)M),
                                     ctx->stream));
  double* r0 = buf;
  double* mu_vec = buf + r0_n;
  double* mu_avg = mu_vec + mv_n;
  int rc = KITE_OK;
  kite_stats total{};
  for (int j0 = 0; j0 < nv && rc == KITE_OK; j0 += chunk) {
    const int n = std::min(chunk, nv - j0);
    gen(j0, n, r0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_fail(ctx, e, "start vectors");
      break;
    }
    kite_kpm kk = *kpm;
    kk.R = n;
    kk.r0 = nullptr;  // the device vectors go in through r0_dev_all
    kite_stats one{};
    rc = moments_1d_impl(ctx, sys, &kk, sc, mu_avg, mu_avg + M, mu_vec, &one, r0);
    if (rc != KITE_OK) break;
    const int b2 = (int)std::min<int64_t>(((int64_t)n * M + 255) / 256, (int64_t)ctx->num_sms * 8);
    k_spectral_avg<<<std::max(1, b2), 256, 0, ctx->stream>>>(mu_vec, S, n, M, j0, scale, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "realisation average");
    total.seconds += one.seconds;
    total.updates += one.updates;
    total.bytes_moved += one.bytes_moved;
    total.step_seconds += one.step_seconds;
    total.step_launches += one.step_launches;
    total.step_bytes += one.step_bytes;
    total.n_eff = one.n_eff;
    total.grid = one.grid;
    total.block = one.block;
  }
  cudaFreeAsync(buf, ctx->stream);
  if (st) {
    total.gbps = total.seconds > 0 ? total.bytes_moved / total.seconds * 1e-9 : 0.0;
    total.e_min = sc.e_min;
    total.e_max = sc.e_max;
    *st = total;
  }
  return rc;
}

// k [nk][2], w [SORB][2] (or null), out [nk][M][2]: all device memory.
int spectral_k_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
                    const double* k, int nk, const double* w, double* out, kite_stats* st) {
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  auto gen = [&](int j0, int n, double* r0) {
    const int blocks = (int)std::min<int64_t>(((int64_t)n * N + 255) / 256, (int64_t)ctx->num_sms * 16);
    k_plane_waves<<<std::max(1, blocks), 256, 0, ctx->stream>>>(sys->lattice, sys->Lx, N, k, j0, n, w,
                                                                kpm->S, r0);
  };
  return deterministic_moments(ctx, sys, kpm, sc, nk, 1.0, gen, out, st);
}

static __global__ void k_scale(double* __restrict__ x, int64_t n, double a) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] *= a;
}

// orb [n] orbital indices (device), out [n][M][2]: mu_n(i) = <i|T_n(H~)|i>, the sweep's
// 1/N_eff undone (one realisation): the local density of one orbital, mu_0 = 1 unless the
// orbital is vacant (then all moments are 0).
int ldos_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
              const int64_t* orb, int n, double* out, kite_stats* st) {
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  auto gen = [&](int j0, int m, double* r0) {
    const int blocks = (int)std::min<int64_t>(((int64_t)kpm->S * m * N + 255) / 256, (int64_t)ctx->num_sms * 16);
    k_basis_vectors<<<std::max(1, blocks), 256, 0, ctx->stream>>>(N, orb, j0, m, kpm->S, r0);
  };
  kite_stats local{};
  int rc = deterministic_moments(ctx, sys, kpm, sc, n, 1.0, gen, out, &local);
  if (rc != KITE_OK) return rc;
  const int64_t total = 2 * (int64_t)n * kpm->M;
  k_scale<<<(int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0, ctx->stream>>>(
      out, total, (double)local.n_eff);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  if (st) *st = local;
  return KITE_OK;
}

}  // namespace kite
