// kite_propagate.cu -- wave-packet time evolution (the paper's spintronics section).
//
//   |psi(t + dt)> = U(dt) |psi(t)>,   U(dt) = exp(-i H dt) (hbar = 1, dt in hbar/eV)
//                 = exp(-i de_plus dt) [c_0 + 2 sum_{n>=1} c_n T_n(H~)],
//   c_n = (-i)^n J_n(de_minus dt)    (Tal-Ezer and Kosloff's Chebyshev propagator; the
//                                     paper prints (-1)^n, the expansion has (-i)^n),
// truncated at M terms per time step.  The recursion is the stencil step kernel in
// MODE 4, which adds c_{n+1} T_{n+1} psi into the accumulator while it writes the
// iterate; the accumulator becomes the next step's psi.  Bessel functions by Miller's
// backward recurrence normalised with J_0 + 2 sum_k J_2k = 1.
#include <math.h>

#include <algorithm>
#include <vector>

#include "kite_device.cuh"
#include "kite_internal.h"

#include "kite_step.cuh"

namespace kite {

// J_n(x) for n < M, x >= 0 (Miller's backward recurrence).
void bessel_j(int M, double x, double* J) {
  for (int n = 0; n < M; ++n) J[n] = 0.0;
  if (x == 0.0) {
    J[0] = 1.0;
    return;
  }
  const int top = 2 * ((std::max(M, (int)x) + 16 + (int)sqrt(40.0 * std::max(M, (int)x + 1))) / 2);
  std::vector<double> j(top + 2, 0.0);
  j[top + 1] = 0.0;
  j[top] = 1e-300;
  for (int k = top; k >= 1; --k) {
    j[k - 1] = 2.0 * k / x * j[k] - j[k + 1];
    if (fabs(j[k - 1]) > 1e250) {  // rescale to stay finite
      for (int i = k - 1; i <= top + 1; ++i) j[i] *= 1e-250;
    }
  }
  double norm = j[0];
  for (int k = 2; k <= top; k += 2) norm += 2.0 * j[k];
  for (int n = 0; n < M && n <= top; ++n) J[n] = j[n] / norm;
}

// coef [M][2] = exp(-i de_plus dt) (2 - delta_n0) (-i)^n J_n(de_minus dt)
void evolution_coeffs(int M, double dt, double de_plus, double de_minus, double* coef) {
  std::vector<double> J(M);
  bessel_j(M, de_minus * dt, J.data());
  const double pr = cos(de_plus * dt), pi = -sin(de_plus * dt);
  for (int n = 0; n < M; ++n) {
    const double a = (n == 0 ? 1.0 : 2.0) * J[n];
    double re = 0.0, im = 0.0;  // a * (-i)^n
    switch (n & 3) {
      case 0: re = a; break;
      case 1: im = -a; break;
      case 2: re = -a; break;
      default: im = a; break;
    }
    coef[2 * n] = pr * re - pi * im;
    coef[2 * n + 1] = pr * im + pi * re;
  }
}

namespace {

// acc = c * psi (batch layout, complex per pair of reals)
template <typename Real>
__global__ void k_series_init(int64_t nchunk, const void* __restrict__ psi, void* __restrict__ acc, double cr,
                              double ci) {
  using Ch = Chunk<Real>;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunk;
       q += (int64_t)gridDim.x * blockDim.x) {
    const Ch p = Ch::ldg(psi, q);
    Ch a;
#pragma unroll
    for (int k = 0; k < Ch::kVecs; ++k) {
      a.v[2 * k] = (Real)(cr * (double)p.v[2 * k] - ci * (double)p.v[2 * k + 1]);
      a.v[2 * k + 1] = (Real)(cr * (double)p.v[2 * k + 1] + ci * (double)p.v[2 * k]);
    }
    a.st(acc, q);
  }
}

// per-block partial sums of |psi|^2 per real lane of a chunk: part[block][lane]
template <typename Real>
__global__ void k_norm_partial(int64_t nchunk, int C, const void* __restrict__ psi, double* __restrict__ part) {
  using Ch = Chunk<Real>;
  constexpr int NR = Ch::kReals;
  __shared__ double red[256][4 * NR];
  double acc[4 * NR];
  for (int k = 0; k < 4 * NR; ++k) acc[k] = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunk;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % C);
    const Ch p = Ch::ldg(psi, q);
    for (int k = 0; k < NR; ++k) acc[c * NR + k] += (double)p.v[k] * (double)p.v[k];
  }
  for (int k = 0; k < 4 * NR; ++k) red[threadIdx.x][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < 4 * NR) {
    double s = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) s += red[t][threadIdx.x];
    part[(size_t)blockIdx.x * 4 * NR + threadIdx.x] = s;
  }
}

// norms[v] = sum over blocks of lanes (re, im) of vector v (vec_base + v < R)
template <typename Real>
__global__ void k_norm_final(const double* __restrict__ part, int blocks, int nvec, double* __restrict__ out) {
  constexpr int NR = Chunk<Real>::kReals, VPC = Chunk<Real>::kVecs;
  const int v = threadIdx.x;
  if (v >= nvec) return;
  const int c = v / VPC, k = v % VPC;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b)
    s += part[(size_t)b * 4 * NR + c * NR + 2 * k] + part[(size_t)b * 4 * NR + c * NR + 2 * k + 1];
  out[v] = s;
}

// batch layout -> caller layout psi[vec_base + v][o] (complex FP64)
template <typename Real, int SORB, int C>
__global__ void k_extract64(int64_t ncell, const void* __restrict__ buf, int nvec, int vec_base, int64_t N,
                            double* __restrict__ dst) {
  using Ch = Chunk<Real>;
  const int64_t nchunk = ncell * SORB * C;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunk;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % C);
    const int64_t o = q / C;
    const Ch z = Ch::ldg(buf, q);
#pragma unroll
    for (int k = 0; k < Ch::kVecs; ++k) {
      const int v = c * Ch::kVecs + k;
      if (v >= nvec) continue;
      double* d = dst + 2 * ((int64_t)(vec_base + v) * N + o);
      d[0] = (double)z.v[2 * k];
      d[1] = (double)z.v[2 * k + 1];
    }
  }
}

template <typename Real, int LAT, int C, bool FIELD>
int propagate_typed(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc, double dt,
                    int nsteps, double* psi, double* norms, kite_stats* stats) {
  constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  constexpr int VPC = Chunk<Real>::kVecs;
  using Sh = StepShape<LAT, C>;
  constexpr int SM = Sh::template smem_bytes<4>();
  const int M = kpm->M, R = kpm->R;
  const int64_t ncell = (int64_t)sys->Lx * sys->Ly, N = ncell * SORB;
  const int64_t nchunk = ncell * SORB * C;
  const size_t vb = (size_t)nchunk * 16;
  const long long units = (long long)((sys->Lx + Sh::TX - 1) / Sh::TX) * sys->Ly;
  const int G = grid_for<Real, LAT, C, false, 4, kStages, FIELD>(ctx, units);
  const int nb = (int)std::min<int64_t>((nchunk + 255) / 256, (int64_t)ctx->num_sms * 8);
  Carver probe(nullptr);
  auto lay = [&](Carver& k, Real** vt, void** r0, void** bA, void** bB, void** acc, double** part,
                 unsigned long long** ne, Real** ph) {
    *vt = k.take<Real>(N);
    *ph = FIELD ? k.take<Real>((size_t)sys->Ly * SORB * 4) : nullptr;
    *r0 = k.take<char>(vb);
    *bA = k.take<char>(vb);
    *bB = k.take<char>(vb);
    *acc = k.take<char>(vb);
    *part = k.take<double>((size_t)nb * 4 * Chunk<Real>::kReals + 64);
    *ne = k.take<unsigned long long>(1);
  };
  Real* vt;
  void *r0, *bA, *bB, *acc;
  double* part;
  unsigned long long* ne;
  Real* ph;
  lay(probe, &vt, &r0, &bA, &bB, &acc, &part, &ne, &ph);
  int rc = ensure_ws(ctx, probe.used());
  if (rc != KITE_OK) return rc;
  Carver w(ctx->ws);
  lay(w, &vt, &r0, &bA, &bB, &acc, &part, &ne, &ph);
  cudaStream_t st = ctx->stream;
  if (FIELD) {  // Peierls phases of the bonds with an x component, per row and sublattice
    rc = field_phases(ctx, sys, sizeof(Real) == 8, ph);
    if (rc != KITE_OK) return rc;
  }
  Open open;
  {
    const void* z = nullptr;
    rc = open_zeros(ctx, sys, &z);
    if (rc != KITE_OK) return rc;
    open.zero = static_cast<const unsigned char*>(z);
    open.x = sys->open_x;
    open.y = sys->open_y;
  }
  std::vector<double> coef(2 * (size_t)M);
  evolution_coeffs(M, dt, sc.de_plus, sc.de_minus, coef.data());
  const Real tt = (Real)(sys->t / sc.de_minus);
  const double thr_d = floor(sys->p_vac * 4294967296.0);
  const uint64_t vac_thr =
      sys->p_vac <= 0.0 ? 0ull : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
  const uint32_t k0 = (uint32_t)sys->seed, k1 = (uint32_t)(sys->seed >> 32);
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ne, 0, sizeof(unsigned long long), st));
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  k_onsite<Real><<<nb, 256, 0, st>>>(N, sys->lattice, sys->W, 0.5 * sys->delta, sc.de_plus, sc.de_minus, vac_thr,
                                      0u, k0, k1, vt, ne, sys->disorder);
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, st));
  const int batch = C * VPC;
  double step_s = 0.0;
  int64_t launches = 0;
  for (int base = 0; base < R; base += batch) {
    const int nvec = std::min(batch, R - base);
    k_init_r0<Real, SORB, C><<<nb, 256, 0, st>>>(ncell, vt, base, nvec, 0u, k0, k1, psi, N, r0);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
    void* cur = r0;  // psi(t) in the batch layout
    void* nxt = acc;
    for (int k = 0; k < nsteps; ++k) {
      auto where = [&](int n) -> void* { return n == 0 ? cur : ((n & 1) ? bA : bB); };
      k_series_init<Real><<<nb, 256, 0, st>>>(nchunk, cur, nxt, coef[0], coef[1]);
      if (M >= 2)
        k_step<Real, LAT, C, true, 4, kStages, FIELD><<<G, kBlock, SM, st>>>(
            nullptr, cur, bA, nullptr, vt, tt, sys->Lx, sys->Ly, units, nullptr, nullptr, ctx->d_status, 0, FamOut{},
            0, SeriesOut{nxt, coef[2], coef[3]}, ph, open);
      for (int n = 1; n + 1 < M; ++n)
        k_step<Real, LAT, C, false, 4, kStages, FIELD><<<G, kBlock, SM, st>>>(
            where(n - 1), where(n), where(n + 1), nullptr, vt, tt, sys->Lx, sys->Ly, units, nullptr, nullptr,
            ctx->d_status, 0, FamOut{}, 0, SeriesOut{nxt, coef[2 * (n + 1)], coef[2 * (n + 1) + 1]}, ph, open);
      launches += std::max(0, M - 1);
      KITE_CUDA_TRY(ctx, cudaGetLastError());
      std::swap(cur, nxt);
      if (norms) {
        k_norm_partial<Real><<<nb, 256, 0, st>>>(nchunk, C, cur, part);
        k_norm_final<Real><<<1, 32, 0, st>>>(part, nb, nvec, norms + (size_t)k * R + base);
        KITE_CUDA_TRY(ctx, cudaGetLastError());
      }
    }
    k_extract64<Real, SORB, C><<<nb, 256, 0, st>>>(ncell, cur, nvec, base, N, psi);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, st));
  int status_host = 0;
  unsigned long long ne_host = 0;
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&status_host, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&ne_host, ne, sizeof(ne_host), cudaMemcpyDeviceToHost, st));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (status_host) return fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait gave up in the propagation");
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    step_s = 1e-3 * ms;
    stats->seconds = step_s;
    stats->step_launches = launches;
    stats->updates = (double)ne_host * std::max(0, M - 1) * nsteps * R;
    stats->n_eff = (int64_t)ne_host;
    stats->grid = G;
    stats->block = kBlock;
    stats->e_min = sc.e_min;
    stats->e_max = sc.e_max;
  }
  return KITE_OK;
}

}  // namespace

int propagate_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc, double dt,
                   int nsteps, double* psi, double* norms, kite_stats* st) {
  const bool fp64 = kpm->precision == KITE_FP64;
  const int per = fp64 ? 1 : 2;
  const int c = (std::min(kpm->R, 4 * per) + per - 1) / per;
  const int C = c <= 1 ? 1 : (c <= 2 ? 2 : 4);
#define KITE_P(REAL, LATV, CC)                                                                     \
  (sys->flux != 0.0 ? propagate_typed<REAL, LATV, CC, true>(ctx, sys, kpm, sc, dt, nsteps, psi, norms, st) \
                    : propagate_typed<REAL, LATV, CC, false>(ctx, sys, kpm, sc, dt, nsteps, psi, norms, st))
#define KITE_PC(REAL, LATV) (C == 1 ? KITE_P(REAL, LATV, 1) : (C == 2 ? KITE_P(REAL, LATV, 2) : KITE_P(REAL, LATV, 4)))
  if (sys->lattice == KITE_HONEYCOMB) return fp64 ? KITE_PC(double, KITE_HONEYCOMB) : KITE_PC(float, KITE_HONEYCOMB);
  return fp64 ? KITE_PC(double, KITE_SQUARE) : KITE_PC(float, KITE_SQUARE);
#undef KITE_PC
#undef KITE_P
}

}  // namespace kite
