// kite_kpm1d.cu -- 1D Chebyshev moments of the average density of states.
//
// Path (Sec. 2a-2c of arXiv:1910.05194): on-site energies and vacancies of one
// disorder realisation -> start vectors r_0 (random phases, Sec. 2c) -> recursion
// r_1 = H~ r_0, r_{n+1} = 2 H~ r_n - r_{n-1} (Eq. e6) with H~ applied matrix-free
// (Sec. 3a) and the moment <r_0|r_{n+1}> (Eqs. e7/e8) fused into the same pass ->
// deterministic FP64 reduction of per-CTA partials.
//
// Device layout: a vector batch of up to 8 (FP32) or 4 (FP64) complex vectors is
// interleaved per orbital, [cell = y*Lx + x][sublattice][chunk], one 16-byte chunk
// holding two complex FP32 or one complex FP64 values.  A warp therefore touches
// contiguous 512-byte stretches of a row; x runs fastest (the memory layout along
// a1 used by the paper, Sec. 5).
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "kite_device.cuh"
#include "kite_internal.h"

#include "kite_step.cuh"

namespace kite {
namespace {

// Sums the per-CTA partials of every moment in fixed order and normalises by N_eff:
// mu_vec[(vec_base+v)][n] (complex) for the valid lanes v < nvec.  A lane is (vector,
// re/im) for complex vectors and one real vector (imaginary part 0) for real ones.
__global__ void k_reduce(const double* __restrict__ partial, int M, int G, int Q, int nvec,
                         int vec_base, const unsigned long long* __restrict__ n_eff,
                         double* __restrict__ mu_vec, int realv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * Q) return;
  const int n = idx / Q, q = idx - (idx / Q) * Q;
  const int v = realv ? q : q >> 1, comp = realv ? 0 : q & 1;
  if (v >= nvec) return;
  double sum = 0.0;
  const double* p = partial + (size_t)n * G * Q + q;
  for (int g = 0; g < G; ++g) sum += p[(size_t)g * Q];
  const double ne = (double)*n_eff;
  double* out = mu_vec + ((size_t)(vec_base + v) * M + n) * 2;
  out[comp] = ne > 0.0 ? sum / ne : 0.0;
  if (realv) out[1] = 0.0;
}

// Moment doubling (T_n^2 = (T_2n + T_0)/2, T_{n+1} T_n = (T_{2n+1} + T_1)/2): slot k >= 2
// holds <r_n|r_n> (k = 2n) or <r_n|r_{n+1}> (k = 2n+1); mu_k = 2 slot_k - mu_(k mod 2).
__global__ void k_undouble(double* __restrict__ mu_vec, int M, int nvec, int vec_base) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nvec * M) return;
  const int v = idx / M, n = idx - (idx / M) * M;
  if (n < 2) return;
  double* m = mu_vec + (size_t)(vec_base + v) * M * 2;
  m[2 * n] = 2.0 * m[2 * n] - m[2 * (n & 1)];
  m[2 * n + 1] = 2.0 * m[2 * n + 1] - m[2 * (n & 1) + 1];
}

__global__ void k_average(const double* __restrict__ mu_vec, int nv, int M, double* __restrict__ mu,
                          double* __restrict__ imag) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  double re = 0.0, im = 0.0;
  for (int v = 0; v < nv; ++v) {
    re += mu_vec[((size_t)v * M + n) * 2];
    im += mu_vec[((size_t)v * M + n) * 2 + 1];
  }
  mu[n] = re / nv;
  imag[n] = im / nv;
}

// ------------------------------------------------------------------------------------
// Host driver
// ------------------------------------------------------------------------------------
struct Plan {
  int64_t N, ncell;
  int Lx, Ly, sorb;
  int R, S, M;
  bool fp64;
  bool doubling;  // two moments per step from <r_n|r_n> and <r_n|r_{n+1}>
  bool realv;     // real +-1 start vectors (four FP32 / two FP64 per chunk)
  int max_batch;  // vectors per pass
};

// recursion steps that write r_{n+1}: M - 1 plainly; with doubling, the step from r_n
// also yields mu_2n and mu_2n+1, so steps n = 0 .. ceil(M/2) - 1 suffice
inline int steps_for(const Plan& p) { return p.doubling ? (p.M + 1) / 2 : p.M - 1; }

template <typename Real, int LAT, int C, int NST>
int sweep_batch(kite_ctx* ctx, const Plan& p, const Real* vt, Real tt, void* r0, void* bA,
                void* bB, double* partial, int G, long long units, int nvec, int vec_base,
                const unsigned long long* n_eff, double* mu_vec, void** last_prev,
                void** last_cur, double* step_seconds, int64_t* step_launches) {
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int Q = 2 * C * VPC;
  cudaStream_t st = ctx->stream;
  const int M = p.M;
  // r_0 lives in r0; r_n (n >= 1) lives in bA for odd n and in bB for even n, so
  // r_{n+1} overwrites r_{n-1} in place except at n = 1 (r_0 is kept for the moments).
  auto where = [&](int n) -> void* { return n == 0 ? r0 : ((n & 1) ? bA : bB); };
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
  constexpr int SM = StepShape<LAT, C, NST>::SMEM;
  if (p.doubling) {
    constexpr int SMD = StepShape<LAT, C, NST>::SMEM_NR0;
    // step 0: r_1 = H~ r_0 with <r_0|r_0> -> slot 0 and <r_0|r_1> -> slot 1; step n >= 1
    // (r_{n+1} from r_n, r_{n-1}): <r_n|r_n> -> slot 2n, <r_n|r_{n+1}> -> slot 2n+1
    const int steps = steps_for(p);
    k_step<Real, LAT, C, true, 3, NST><<<G, kBlock, SMD, st>>>(nullptr, r0, bA, nullptr, vt, tt, p.Lx,
                                                         p.Ly, units, partial + (size_t)G * Q,
                                                         partial, ctx->d_status,
                                                         ctx->debug_stall, FamOut{}, p.realv ? 1 : 0);
    ctx->debug_stall = 0;
    for (int n = 1; n < steps; ++n)
      k_step<Real, LAT, C, false, 3, NST><<<G, kBlock, SMD, st>>>(
          where(n - 1), where(n), where(n + 1), nullptr, vt, tt, p.Lx, p.Ly, units,
          partial + (size_t)(2 * n + 1) * G * Q, partial + (size_t)(2 * n) * G * Q, ctx->d_status,
          0, FamOut{}, p.realv ? 1 : 0);
    KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
    KITE_CUDA_TRY(ctx, cudaGetLastError());
    const int total = M * Q;
    k_reduce<<<(total + 255) / 256, 256, 0, st>>>(partial, M, G, Q, nvec, vec_base, n_eff, mu_vec,
                                                 p.realv ? 1 : 0);
    k_undouble<<<(nvec * M + 255) / 256, 256, 0, st>>>(mu_vec, M, nvec, vec_base);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
    float ms = 0.f;
    KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
    KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
    *step_seconds += 1e-3 * ms;
    *step_launches += steps;
    *last_cur = *last_prev = nullptr;
    return KITE_OK;
  }
  if (M >= 2)
    k_step<Real, LAT, C, true, 0, NST><<<G, kBlock, SM, st>>>(nullptr, r0, bA, r0, vt, tt, p.Lx, p.Ly,
                                                      units, partial + (size_t)G * Q, partial,
                                                      ctx->d_status, ctx->debug_stall, FamOut{}, p.realv ? 1 : 0);
  ctx->debug_stall = 0;
  for (int n = 1; n + 1 < M; ++n)
    k_step<Real, LAT, C, false, 0, NST><<<G, kBlock, SM, st>>>(where(n - 1), where(n), where(n + 1), r0,
                                                       vt, tt, p.Lx, p.Ly, units,
                                                       partial + (size_t)(n + 1) * G * Q, nullptr,
                                                       ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0);
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  if (M == 1) {
    // mu_0 alone: one FIRST pass would also write r_1; a plain dot is enough, but the
    // FIRST kernel is cheap and keeps one code path.
    k_step<Real, LAT, C, true, 0, NST><<<G, kBlock, SM, st>>>(nullptr, r0, bA, r0, vt, tt, p.Lx, p.Ly,
                                                      units, partial + (size_t)G * Q, partial,
                                                      ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
  }
  const int total = M * Q;
  k_reduce<<<(total + 255) / 256, 256, 0, st>>>(partial, M, G, Q, nvec, vec_base, n_eff, mu_vec,
                                                 p.realv ? 1 : 0);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  if (M >= 2) {
    float ms = 0.f;
    KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
    KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
    *step_seconds += 1e-3 * ms;
    *step_launches += M - 1;
  }
  *last_cur = where(M - 1);
  *last_prev = where(M >= 2 ? M - 2 : 0);
  return KITE_OK;
}

// ---- autotuner: ring depth x resident CTAs per SM ------------------------------------
// Candidates are timed on the caller's own buffers (a few non-first steps between r_0
// and the two iterate buffers, which the sweep overwrites afterwards) and the fastest is
// cached per (precision, lattice, vectors per orbital, mode, size bucket) on the context.
// KITE_AUTOTUNE=0 keeps the default (8 stages, full occupancy).
struct Tune {
  int nst;  // ring depth: 4 or 8
  int k;    // resident CTAs per SM
};

inline bool autotune_enabled() {
  const char* e = getenv("KITE_AUTOTUNE");
  return !(e && e[0] == '0');
}

template <typename Real, int LAT, int C, int MODE, int NST>
float time_candidate(kite_ctx* ctx, int k, long long units, const Plan& p, const Real* vt, Real tt, void* r0,
                     void* bA, void* bB, double* partial) {
  constexpr int SMEM = StepShape<LAT, C, NST>::template smem_bytes<MODE>();
  constexpr int Q = 2 * C * Chunk<Real>::kVecs;
  const int G = grid_for<Real, LAT, C, false, MODE, NST>(ctx, units, k);
  cudaStream_t st = ctx->stream;
  auto launch = [&]() {
    k_step<Real, LAT, C, false, MODE, NST><<<G, kBlock, SMEM, st>>>(
        r0, bA, bB, MODE == 0 ? r0 : nullptr, vt, tt, p.Lx, p.Ly, units, partial + (size_t)2 * G * Q,
        MODE == 3 ? partial + (size_t)G * Q : nullptr, ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0);
  };
  launch();  // warm-up
  cudaEventRecord(ctx->ev2, st);
  for (int i = 0; i < 3; ++i) launch();
  cudaEventRecord(ctx->ev3, st);
  float ms = 1e30f;
  if (cudaEventSynchronize(ctx->ev3) != cudaSuccess || cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3) != cudaSuccess)
    ms = 1e30f;
  return ms;
}

template <typename Real, int LAT, int C, int MODE>
Tune autotune(kite_ctx* ctx, long long units, const Plan& p, const Real* vt, Real tt, void* r0, void* bA,
              void* bB, double* partial) {
  Tune def{kStages, step_occupancy<Real, LAT, C, MODE, kStages>()};
  if (!autotune_enabled() || units < 4LL * ctx->num_sms) return def;
  int bucket = 0;
  while ((1LL << (bucket + 1)) <= units) ++bucket;
  const uint64_t key = ((uint64_t)1 << 56) | ((uint64_t)sizeof(Real) << 48) | ((uint64_t)LAT << 40) |
                       ((uint64_t)C << 32) | ((uint64_t)MODE << 24) | ((uint64_t)p.realv << 16) | (uint64_t)bucket;
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return Tune{it->second.first, it->second.second};
  Tune best = def;
  float best_ms = 1e30f;
  const int o8 = step_occupancy<Real, LAT, C, MODE, 8>(), o4 = step_occupancy<Real, LAT, C, MODE, 4>();
  for (int k = 1; k <= o8; ++k) {
    const float ms = time_candidate<Real, LAT, C, MODE, 8>(ctx, k, units, p, vt, tt, r0, bA, bB, partial);
    if (ms < best_ms) best_ms = ms, best = Tune{8, k};
  }
  for (int k = 1; k <= o4; ++k) {
    const float ms = time_candidate<Real, LAT, C, MODE, 4>(ctx, k, units, p, vt, tt, r0, bA, bB, partial);
    if (ms < best_ms * 0.98f) best_ms = ms, best = Tune{4, k};  // prefer the deeper ring on a tie
  }
  cudaGetLastError();
  ctx->tune[key] = {best.nst, best.k};
  return best;
}

template <typename Real, int LAT, int MODE>
int max_grid_c(kite_ctx* ctx, int C, long long units) {
  auto g = [&](auto occ8, auto occ4) {
    return (int)std::max(1LL, std::min((long long)ctx->num_sms * std::max(occ8, occ4), units));
  };
  if (C == 1) return g(step_occupancy<Real, LAT, 1, MODE, 8>(), step_occupancy<Real, LAT, 1, MODE, 4>());
  if (C == 2) return g(step_occupancy<Real, LAT, 2, MODE, 8>(), step_occupancy<Real, LAT, 2, MODE, 4>());
  return g(step_occupancy<Real, LAT, 4, MODE, 8>(), step_occupancy<Real, LAT, 4, MODE, 4>());
}

template <typename Real, int LAT>
int run_typed(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
              double* mu_dev, double* imag_dev, double* mu_vec_dev_ext, kite_stats* stats,
              const double* r0_dev_all) {
  constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int kMaxC = 4;
  Plan p;
  p.Lx = sys->Lx;
  p.Ly = sys->Ly;
  p.sorb = SORB;
  p.ncell = (int64_t)sys->Lx * sys->Ly;
  p.N = p.ncell * SORB;
  p.R = kpm->R;
  p.S = kpm->S;
  p.M = kpm->M;
  p.doubling = kpm->doubling != 0;
  p.realv = kpm->real_vectors != 0;
  const int per_chunk = p.realv ? Chunk<Real>::kReals : VPC;  // vectors per 16-byte chunk
  p.max_batch = kMaxC * per_chunk;
  auto chunks_for = [&](int nvec) {
    const int c = (nvec + per_chunk - 1) / per_chunk;
    return c <= 1 ? 1 : (c <= 2 ? 2 : 4);
  };
  auto units_for = [&](int C) {
    const int TX = kBlock / (SORB * C);
    return (long long)((sys->Lx + TX - 1) / TX) * sys->Ly;
  };
  const int Cmax = chunks_for(std::min(p.R, p.max_batch));
  const int Ctail = chunks_for(p.R % p.max_batch == 0 ? std::min(p.R, p.max_batch) : p.R % p.max_batch);
  // partials sized for the widest grid any ring depth may use (the autotuner's choice)
  auto grid_c = [&](int C) {
    return p.doubling ? max_grid_c<Real, LAT, 3>(ctx, C, units_for(C)) : max_grid_c<Real, LAT, 0>(ctx, C, units_for(C));
  };
  const int Gmax = std::max(grid_c(Cmax), grid_c(Ctail));

  // work space
  const size_t vec_bytes = (size_t)p.ncell * SORB * Cmax * 16;
  const size_t nvec_total = (size_t)p.R * p.S;
  Carver cv(nullptr);
  auto plan_ws = [&](Carver& k, Real** vt, void** r0, void** bA, void** bB, double** partial,
                     unsigned long long** ne, double** mu_vec) {
    *vt = k.take<Real>(p.N);
    *r0 = k.take<char>(vec_bytes);
    *bA = k.take<char>(vec_bytes);
    *bB = k.take<char>(vec_bytes);
    *partial = k.take<double>((size_t)(std::max(p.M, 2) + 1) * Gmax * 2 * Cmax * VPC);
    *ne = k.take<unsigned long long>(1);
    *mu_vec = k.take<double>(nvec_total * p.M * 2);
  };
  Real* vt;
  void *r0, *bA, *bB;
  double *partial, *mu_vec;
  unsigned long long* ne;
  plan_ws(cv, &vt, &r0, &bA, &bB, &partial, &ne, &mu_vec);
  int rc = ensure_ws(ctx, cv.used());
  if (rc != KITE_OK) return rc;
  Carver real(ctx->ws);
  plan_ws(real, &vt, &r0, &bA, &bB, &partial, &ne, &mu_vec);
  if (mu_vec_dev_ext) mu_vec = mu_vec_dev_ext;

  const Real tt = (Real)(sys->t / sc.de_minus);
  const double thr_d = floor(sys->p_vac * 4294967296.0);
  const uint64_t vac_thr =
      sys->p_vac <= 0.0 ? 0ull : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
  const uint32_t k0 = (uint32_t)sys->seed, k1 = (uint32_t)(sys->seed >> 32);
  cudaStream_t st = ctx->stream;
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, st));
  int64_t n_eff_last = 0;
  int grid_used = 0;
  Tune tune_used{kStages, 0};
  double step_s = 0.0, step_bytes = 0.0;
  int64_t step_n = 0;
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  for (int s = 0; s < p.S; ++s) {
    KITE_CUDA_TRY(ctx, cudaMemsetAsync(ne, 0, sizeof(unsigned long long), st));
    {
      const int64_t blocks = std::min<int64_t>((p.N + 255) / 256, (int64_t)ctx->num_sms * 16);
      k_onsite<Real><<<(int)std::max<int64_t>(1, blocks), 256, 0, st>>>(
          p.N, sys->lattice, sys->W, 0.5 * sys->delta, sc.de_plus, sc.de_minus, vac_thr,
          (uint32_t)s, k0, k1, vt, ne);
      KITE_CUDA_TRY(ctx, cudaGetLastError());
    }
    for (int base = 0; base < p.R; base += p.max_batch) {
      const int nvec = std::min(p.max_batch, p.R - base);
      const int C = chunks_for(nvec);
      const long long u = units_for(C);
      {
        const int64_t nchunk = p.ncell * SORB * C;
        const int64_t blocks = std::min<int64_t>((nchunk + 255) / 256, (int64_t)ctx->num_sms * 16);
        const double* r0_in = r0_dev_all ? r0_dev_all + (size_t)s * p.R * p.N * 2 : nullptr;
        const uint32_t phase_base = (uint32_t)s * (uint32_t)p.R;
#define KITE_INIT(CC)                                                                       \
  k_init_r0<Real, SORB, CC><<<(int)std::max<int64_t>(1, blocks), 256, 0, st>>>(           \
      p.ncell, vt, base, nvec, phase_base, k0, k1, r0_in, p.N, r0, p.realv ? 1 : 0)
        if (C == 1) KITE_INIT(1);
        else if (C == 2) KITE_INIT(2);
        else KITE_INIT(4);
#undef KITE_INIT
        KITE_CUDA_TRY(ctx, cudaGetLastError());
      }
      void *lp = nullptr, *lc = nullptr;
      const int vec_base = s * p.R + base;
#define KITE_SWEEP(CC)                                                                       \
  do {                                                                                       \
    Tune t = p.doubling ? autotune<Real, LAT, CC, 3>(ctx, u, p, vt, tt, r0, bA, bB, partial)  \
                        : autotune<Real, LAT, CC, 0>(ctx, u, p, vt, tt, r0, bA, bB, partial); \
    const int G = t.nst == 4 ? (p.doubling ? grid_for<Real, LAT, CC, false, 3, 4>(ctx, u, t.k)   \
                                           : grid_for<Real, LAT, CC, false, 0, 4>(ctx, u, t.k))  \
                             : (p.doubling ? grid_for<Real, LAT, CC, false, 3, 8>(ctx, u, t.k)   \
                                           : grid_for<Real, LAT, CC, false, 0, 8>(ctx, u, t.k)); \
    grid_used = G;                                                                           \
    tune_used = t;                                                                           \
    rc = t.nst == 4 ? sweep_batch<Real, LAT, CC, 4>(ctx, p, vt, tt, r0, bA, bB, partial, G, u, nvec,  \
                                                    vec_base, ne, mu_vec, &lp, &lc, &step_s, &step_n) \
                    : sweep_batch<Real, LAT, CC, 8>(ctx, p, vt, tt, r0, bA, bB, partial, G, u, nvec,  \
                                                    vec_base, ne, mu_vec, &lp, &lc, &step_s, &step_n); \
  } while (0)
      if (C == 1) KITE_SWEEP(1);
      else if (C == 2) KITE_SWEEP(2);
      else KITE_SWEEP(4);
#undef KITE_SWEEP
      if (rc != KITE_OK) return rc;
      // algorithmic bytes of this batch's step launches: per orbital and step, read
      // r_{n-1}, r_n, r_0 and write r_{n+1} for each of the batch's 16-byte chunks, and
      // read the shared on-site term (the first step has no r_{n-1} and reads r_0 once)
      if (p.doubling) {
        // doubling never re-reads r_0: r_{n-1}, r_n in, r_{n+1} out per later step
        const double chunk_bytes = 16.0 * SORB * C * (double)p.ncell;
        const int steps = steps_for(p);
        step_bytes += (double)(steps - 1) * (3.0 * chunk_bytes + (double)p.N * sizeof(Real)) +
                      (2.0 * chunk_bytes + (double)p.N * sizeof(Real));
      } else if (p.M >= 2) {
        const double chunk_bytes = 16.0 * SORB * C * (double)p.ncell;
        step_bytes += (double)(p.M - 2) * (4.0 * chunk_bytes + (double)p.N * sizeof(Real)) +
                      (2.0 * chunk_bytes + (double)p.N * sizeof(Real));
      }
      if (kpm->r_last && !p.doubling) {
        // extract into a device staging area or directly into a device destination
        const int64_t nchunk = p.ncell * SORB * C;
        const int64_t blocks = std::min<int64_t>((nchunk + 255) / 256, (int64_t)ctx->num_sms * 16);
        Real* dst = static_cast<Real*>(kpm->r_last);
        Real* stage = nullptr;
        const bool dev_dst = is_device_ptr(kpm->r_last);
        const size_t last_bytes = nvec_total * 2 * (size_t)p.N * 2 * sizeof(Real);
        if (!dev_dst) {
          KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&stage, last_bytes, st));
          dst = stage;
        }
#define KITE_EXTRACT(CC)                                                                     \
  do {                                                                                       \
    k_extract<Real, SORB, CC><<<(int)std::max<int64_t>(1, blocks), 256, 0, st>>>(          \
        p.ncell, lp, nvec, vec_base, 0, p.N, dst);                                           \
    k_extract<Real, SORB, CC><<<(int)std::max<int64_t>(1, blocks), 256, 0, st>>>(          \
        p.ncell, lc, nvec, vec_base, 1, p.N, dst);                                           \
  } while (0)
        if (C == 1) KITE_EXTRACT(1);
        else if (C == 2) KITE_EXTRACT(2);
        else KITE_EXTRACT(4);
#undef KITE_EXTRACT
        KITE_CUDA_TRY(ctx, cudaGetLastError());
        if (!dev_dst) {
          // only this batch's vectors were written; copy them
          const size_t per_vec = 2 * (size_t)p.N * 2 * sizeof(Real);
          KITE_CUDA_TRY(ctx, cudaMemcpyAsync(static_cast<char*>(kpm->r_last) + vec_base * per_vec,
                                             reinterpret_cast<char*>(stage) + vec_base * per_vec,
                                             per_vec * nvec, cudaMemcpyDeviceToHost, st));
          KITE_CUDA_TRY(ctx, cudaFreeAsync(stage, st));
        }
      }
    }
    unsigned long long ne_host = 0;
    int status_host = 0;
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&ne_host, ne, sizeof(ne_host), cudaMemcpyDeviceToHost, st));
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&status_host, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (status_host != 0)
      return fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up in the step kernel");
    n_eff_last = (int64_t)ne_host;
  }
  {
    const int nv = (int)nvec_total;
    k_average<<<(p.M + 255) / 256, 256, 0, st>>>(mu_vec, nv, p.M, mu_dev, imag_dev);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, st));
  KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev1));
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->seconds = ms * 1e-3;
    stats->updates = (double)n_eff_last * p.M * p.R * p.S;
    // algorithmic bytes per orbital and step: read r_{n-1}, r_n, r_0, write r_{n+1}
    // for every vector, plus the shared on-site term
    const double per_orb_step =
        (p.doubling ? 3.0 : 4.0) * (p.realv ? 1.0 : 2.0) * sizeof(Real) * p.R + (double)sizeof(Real);
    stats->bytes_moved = per_orb_step * (double)p.N * (double)steps_for(p) * p.S;
    stats->gbps = stats->seconds > 0 ? stats->bytes_moved / stats->seconds * 1e-9 : 0.0;
    stats->n_eff = n_eff_last;
    stats->grid = grid_used;
    stats->block = kBlock;
    stats->ring_stages = tune_used.nst;
    stats->ctas_per_sm = grid_used / std::max(1, ctx->num_sms);
    stats->step_seconds = step_s;
    stats->step_launches = step_n;
    stats->step_bytes = step_bytes;
  }
  return KITE_OK;
}

}  // namespace

int moments_1d_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
                    double* mu_dev, double* imag_dev, double* mu_vec_dev, kite_stats* st,
                    const double* r0_dev_all) {
  const bool fp64 = kpm->precision == KITE_FP64;
  if (sys->lattice == KITE_HONEYCOMB)
    return fp64 ? run_typed<double, KITE_HONEYCOMB>(ctx, sys, kpm, sc, mu_dev, imag_dev, mu_vec_dev, st, r0_dev_all)
                : run_typed<float, KITE_HONEYCOMB>(ctx, sys, kpm, sc, mu_dev, imag_dev, mu_vec_dev, st, r0_dev_all);
  return fp64 ? run_typed<double, KITE_SQUARE>(ctx, sys, kpm, sc, mu_dev, imag_dev, mu_vec_dev, st, r0_dev_all)
              : run_typed<float, KITE_SQUARE>(ctx, sys, kpm, sc, mu_dev, imag_dev, mu_vec_dev, st, r0_dev_all);
}

}  // namespace kite
