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
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "kite_device.cuh"
#include "kite_internal.h"

#include "kite_step.cuh"
#include "kite_step2.cuh"
#include "kite_step3.cuh"

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
  bool field;     // Peierls phases of a perpendicular magnetic field (kite_field.cu)
  int max_batch;  // vectors per pass
  Open open;      // open boundaries and their zero buffer
};

// recursion steps that write r_{n+1}: M - 1 plainly; with doubling, the step from r_n
// also yields mu_2n and mu_2n+1, so steps n = 0 .. ceil(M/2) - 1 suffice
inline int steps_for(const Plan& p) { return p.doubling ? (p.M + 1) / 2 : p.M - 1; }

template <typename Real, int LAT, int C, int NST>
int sweep_batch(kite_ctx* ctx, const Plan& p, const Real* vt, Real tt, void* r0, void* bA,
                void* bB, double* partial, int G, long long units, int nvec, int vec_base,
                const unsigned long long* n_eff, double* mu_vec, void** last_prev, void** last_cur,
                double* step_seconds, int64_t* step_launches, double* step_bytes) {
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int Q = 2 * C * VPC;
  cudaStream_t st = ctx->stream;
  const int M = p.M;
  // r_0 lives in r0; r_n (n >= 1) lives in bA for odd n and in bB for even n, so
  // r_{n+1} overwrites r_{n-1} in place except at n = 1 (r_0 is kept for the moments).
  auto where = [&](int n) -> void* { return n == 0 ? r0 : ((n & 1) ? bA : bB); };
  // algorithmic bytes of one launch: `vecs` iterate streams of the batch's chunks plus
  // one read of the on-site term
  const double chunk_bytes = 16.0 * StepShape<LAT, C, NST>::SORB * C * (double)p.ncell;
  auto launch_bytes = [&](int vecs) { return vecs * chunk_bytes + (double)p.N * sizeof(Real); };
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
  constexpr int SM = StepShape<LAT, C, NST>::SMEM;
  if (p.doubling) {
    constexpr int SMD = StepShape<LAT, C, NST>::SMEM_NR0;
    // step 0: r_1 = H~ r_0 with <r_0|r_0> -> slot 0 and <r_0|r_1> -> slot 1; step n >= 1
    // (r_{n+1} from r_n, r_{n-1}): <r_n|r_n> -> slot 2n, <r_n|r_{n+1}> -> slot 2n+1
    const int steps = steps_for(p);
    launch_pdl(k_step<Real, LAT, C, true, 3, NST>, G, kBlock, SMD, st,
        nullptr, r0, bA, nullptr, vt, tt, p.Lx, p.Ly, units,
        partial + (size_t)G * Q, partial, ctx->d_status, ctx->debug_stall, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
    ctx->debug_stall = 0;
    for (int n = 1; n < steps; ++n)
      launch_pdl(k_step<Real, LAT, C, false, 3, NST>, G, kBlock, SMD, st,
          where(n - 1), where(n), where(n + 1), nullptr, vt, tt, p.Lx, p.Ly, units,
          partial + (size_t)(2 * n + 1) * G * Q,
          partial + (size_t)(2 * n) * G * Q, ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
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
    // doubling never re-reads r_0: r_{n-1}, r_n in, r_{n+1} out per later step
    *step_bytes += (double)(steps - 1) * launch_bytes(3) + launch_bytes(2);
    *last_cur = *last_prev = nullptr;
    return KITE_OK;
  }
  if (M >= 2)
    launch_pdl(k_step<Real, LAT, C, true, 0, NST>, G, kBlock, SM, st,
        nullptr, r0, bA, r0, vt, tt, p.Lx, p.Ly, units,
        partial + (size_t)G * Q, partial, ctx->d_status, ctx->debug_stall, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
  ctx->debug_stall = 0;
  for (int n = 1; n + 1 < M; ++n)
    launch_pdl(k_step<Real, LAT, C, false, 0, NST>, G, kBlock, SM, st,
        where(n - 1), where(n), where(n + 1), r0, vt, tt, p.Lx, p.Ly, units,
        partial + (size_t)(n + 1) * G * Q, nullptr, ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  if (M == 1) {
    // mu_0 alone: one FIRST pass would also write r_1; a plain dot is enough, but the
    // FIRST kernel is cheap and keeps one code path.
    launch_pdl(k_step<Real, LAT, C, true, 0, NST>, G, kBlock, SM, st,
        nullptr, r0, bA, r0, vt, tt, p.Lx, p.Ly, units,
        partial + (size_t)G * Q, partial, ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
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
    *step_bytes += (double)(M - 2) * launch_bytes(4) + launch_bytes(2);
  }
  *last_cur = where(M - 1);
  *last_prev = where(M >= 2 ? M - 2 : 0);
  return KITE_OK;
}

// Temporal blocking of the plain moment sweep: after the first step, each pass takes
// (r_{n-1}, r_n) to (r_{n+1}, r_{n+2}) and the moments n+1, n+2; an odd remainder takes one
// plain step.  The first and remainder steps use the one-step kernel with a 4-slot ring on
// the same grid (the partials of every moment have the same CTA count).
template <typename Real, int LAT, int C, int NST2>
int sweep_two(kite_ctx* ctx, const Plan& p, const Real* vt, Real tt, void* r0, void* bA, void* bB,
              void* bC, void* bD, double* partial, int G, long long units, int nvec, int vec_base,
              const unsigned long long* n_eff, double* mu_vec, void** last_prev, void** last_cur,
              double* step_seconds, int64_t* step_launches, double* step_bytes) {
  constexpr int NST1 = 4;
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int Q = 2 * C * VPC;
  cudaStream_t st = ctx->stream;
  const int M = p.M;
  const double chunk_bytes = 16.0 * StepShape<LAT, C>::SORB * C * (double)p.ncell;
  auto launch_bytes = [&](int vecs) { return vecs * chunk_bytes + (double)p.N * sizeof(Real); };
  constexpr int SM = StepShape<LAT, C, NST1>::SMEM;
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
  // iterate k >= 1 lives in bufs[k mod 4]: a pass's outputs never alias its inputs
  void* bufs[4] = {bC, bA, bB, bD};
  auto w4 = [&](int n) -> void* { return n == 0 ? r0 : bufs[n & 3]; };
  constexpr int SM2 = Step2Shape<LAT, C, NST2>::SMEM;
  step_occupancy<Real, LAT, C, 0, NST1>();  // sets the kernels' shared-memory limits
  step2_occupancy<Real, LAT, C, NST2>();
  launch_pdl(k_step<Real, LAT, C, true, 0, NST1>, G, kBlock, SM, st,
      nullptr, r0, w4(1), r0, vt, tt, p.Lx, p.Ly, units,
      partial + (size_t)G * Q, partial, ctx->d_status, ctx->debug_stall, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
  ctx->debug_stall = 0;
  int n = 1;
  int64_t launches = 1;
  double bytes = launch_bytes(2);  // r_0 in, r_1 out
  for (; n + 2 <= M - 1; n += 2, ++launches) {
    launch_pdl(k_step2<Real, LAT, C, NST2>, G, kBlock2, SM2, st,
        w4(n - 1), w4(n), w4(n + 1), w4(n + 2), r0, vt, tt, p.Lx, p.Ly, units,
        partial + (size_t)(n + 1) * G * Q,
        partial + (size_t)(n + 2) * G * Q, ctx->d_status, p.realv ? 1 : 0, nullptr, nullptr);
    bytes += launch_bytes(5);  // r_{n-1}, r_n, r_0 in; r_{n+1}, r_{n+2} out
  }
  if (n + 1 <= M - 1) {
    launch_pdl(k_step<Real, LAT, C, false, 0, NST1>, G, kBlock, SM, st,
        w4(n - 1), w4(n), w4(n + 1), r0, vt, tt, p.Lx, p.Ly, units,
        partial + (size_t)(n + 1) * G * Q, nullptr, ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
    ++launches;
    bytes += launch_bytes(4);
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  const int total = M * Q;
  k_reduce<<<(total + 255) / 256, 256, 0, st>>>(partial, M, G, Q, nvec, vec_base, n_eff, mu_vec,
                                                 p.realv ? 1 : 0);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  float ms = 0.f;
  KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
  KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
  *step_seconds += 1e-3 * ms;
  *step_launches += launches;
  *step_bytes += bytes;
  *last_cur = w4(M - 1);
  *last_prev = w4(M - 2);
  return KITE_OK;
}

// Temporal blocking of the doubling sweep: after the first step (r_1, slots 0 and 1), each
// pass takes (r_{n-1}, r_n) to (r_{n+1}, r_{n+2}) with the slots 2n .. 2n+3; an odd
// remainder takes one doubling step.  Four vector streams per two steps instead of six.
template <typename Real, int LAT, int C, int NST2>
int sweep_two_dbl(kite_ctx* ctx, const Plan& p, const Real* vt, Real tt, void* r0, void* bA, void* bB,
                  void* bC, void* bD, double* partial, int G, long long units, int nvec, int vec_base,
                  const unsigned long long* n_eff, double* mu_vec, void** last_prev, void** last_cur,
                  double* step_seconds, int64_t* step_launches, double* step_bytes) {
  constexpr int NST1 = 4;
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int Q = 2 * C * VPC;
  cudaStream_t st = ctx->stream;
  const int M = p.M;
  const int steps = steps_for(p);  // iterates r_1 .. r_steps
  const double chunk_bytes = 16.0 * StepShape<LAT, C>::SORB * C * (double)p.ncell;
  auto launch_bytes = [&](int vecs) { return vecs * chunk_bytes + (double)p.N * sizeof(Real); };
  constexpr int SMD = StepShape<LAT, C, NST1>::SMEM_NR0, SM2 = Step2Shape<LAT, C, NST2, true>::SMEM;
  step_occupancy<Real, LAT, C, 3, NST1>();  // sets the kernels' shared-memory limits
  step2_occupancy<Real, LAT, C, NST2, true>();
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
  void* bufs[4] = {bC, bA, bB, bD};
  auto w4 = [&](int n) -> void* { return n == 0 ? r0 : bufs[n & 3]; };
  auto slot = [&](int k) { return partial + (size_t)k * G * Q; };
  launch_pdl(k_step<Real, LAT, C, true, 3, NST1>, G, kBlock, SMD, st,
      nullptr, r0, w4(1), nullptr, vt, tt, p.Lx, p.Ly, units, slot(1), slot(0), ctx->d_status, ctx->debug_stall,
      FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
  ctx->debug_stall = 0;
  int n = 1;
  int64_t launches = 1;
  double bytes = launch_bytes(2);  // r_0 in, r_1 out
  for (; n + 2 <= steps; n += 2, ++launches) {
    launch_pdl(k_step2<Real, LAT, C, NST2, true>, G, kBlock2, SM2, st,
        w4(n - 1), w4(n), w4(n + 1), w4(n + 2), nullptr, vt, tt, p.Lx, p.Ly, units, slot(2 * n),
        slot(2 * n + 1), ctx->d_status, p.realv ? 1 : 0, slot(2 * n + 2), slot(2 * n + 3));
    bytes += launch_bytes(4);  // r_{n-1}, r_n in; r_{n+1}, r_{n+2} out
  }
  if (n + 1 <= steps) {
    launch_pdl(k_step<Real, LAT, C, false, 3, NST1>, G, kBlock, SMD, st,
        w4(n - 1), w4(n), w4(n + 1), nullptr, vt, tt, p.Lx, p.Ly, units, slot(2 * n + 1), slot(2 * n),
        ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
    ++launches;
    bytes += launch_bytes(3);
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  k_reduce<<<(M * Q + 255) / 256, 256, 0, st>>>(partial, M, G, Q, nvec, vec_base, n_eff, mu_vec,
                                                 p.realv ? 1 : 0);
  k_undouble<<<(nvec * M + 255) / 256, 256, 0, st>>>(mu_vec, M, nvec, vec_base);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  float ms = 0.f;
  KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
  KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
  *step_seconds += 1e-3 * ms;
  *step_launches += launches;
  *step_bytes += bytes;
  *last_cur = *last_prev = nullptr;
  return KITE_OK;
}

// Deeper temporal blocking: after the first step, each pass takes (r_{n-1}, r_n) to
// (r_{n+2}, r_{n+3}) with the moments n+1 .. n+3 (r_{n+1} stays on chip); the last one or
// two steps take the one-step kernel or the two-step pass.  Every launch runs on the same
// grid (the partials of every moment have the same CTA count).
template <typename Real, int LAT, int C, int NST3>
int sweep_three(kite_ctx* ctx, const Plan& p, const Real* vt, Real tt, void* r0, void* bA, void* bB,
                void* bC, void* bD, double* partial, int G, long long units, int nvec, int vec_base,
                const unsigned long long* n_eff, double* mu_vec, void** last_prev, void** last_cur,
                double* step_seconds, int64_t* step_launches, double* step_bytes) {
  constexpr int NST1 = 4, NST2 = 6;
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int Q = 2 * C * VPC;
  cudaStream_t st = ctx->stream;
  const int M = p.M;
  const double chunk_bytes = 16.0 * StepShape<LAT, C>::SORB * C * (double)p.ncell;
  auto launch_bytes = [&](int vecs) { return vecs * chunk_bytes + (double)p.N * sizeof(Real); };
  constexpr int SM1 = StepShape<LAT, C, NST1>::SMEM, SM2 = Step2Shape<LAT, C, NST2>::SMEM,
                SM3 = Step3Shape<LAT, C, NST3>::SMEM;
  step_occupancy<Real, LAT, C, 0, NST1>();  // sets the kernels' shared-memory limits
  step2_occupancy<Real, LAT, C, NST2>();
  step3_occupancy<Real, LAT, C, NST3>();
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
  auto slot = [&](int k) { return partial + (size_t)k * G * Q; };
  // r_0 stays in its own buffer; the iterates move between the four others
  void* prev = r0;
  void* cur = bA;
  void* spare[3] = {bB, bC, bD};
  launch_pdl(k_step<Real, LAT, C, true, 0, NST1>, G, kBlock, SM1, st,
      nullptr, r0, cur, r0, vt, tt, p.Lx, p.Ly, units, slot(1), slot(0), ctx->d_status, ctx->debug_stall,
      FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
  ctx->debug_stall = 0;
  int64_t launches = 1;
  double bytes = launch_bytes(2);
  // buffers free for outputs: the spares, plus prev once it is no longer r_0
  auto take_free = [&](void* keep1, void* keep2, void** o1, void** o2) {
    void* cand[4] = {spare[0], spare[1], spare[2], prev};
    int n = 0;
    for (void* b : cand) {
      if (!b || b == r0 || b == keep1 || b == keep2) continue;
      if (n == 0) *o1 = b;
      else if (n == 1) *o2 = b;
      ++n;
      if (n == 2) break;
    }
  };
  auto rotate = [&](void* np, void* nc) {
    // the new (prev, cur) pair; every other non-r_0 buffer is spare
    void* all[4] = {bA, bB, bC, bD};
    int k = 0;
    for (void* b : all)
      if (b != np && b != nc) spare[k++] = b;
    if (k < 3) spare[2] = nullptr;
    prev = np;
    cur = nc;
  };
  int n = 1;  // r_n = cur
  for (; n + 3 <= M - 1; n += 3, ++launches) {
    void *o2 = nullptr, *o3 = nullptr;
    take_free(prev, cur, &o2, &o3);
    launch_pdl(k_step3<Real, LAT, C, NST3>, G, kBlock3, SM3, st,
        prev, cur, o2, o3, r0, vt, tt, p.Lx, p.Ly, units, slot(n + 1), slot(n + 2), slot(n + 3),
        ctx->d_status, p.realv ? 1 : 0);
    bytes += launch_bytes(5);  // r_{n-1}, r_n, r_0 in; r_{n+2}, r_{n+3} out
    rotate(o2, o3);
  }
  if (n + 2 <= M - 1) {
    void *o1 = nullptr, *o2 = nullptr;
    take_free(prev, cur, &o1, &o2);
    launch_pdl(k_step2<Real, LAT, C, NST2>, G, kBlock2, SM2, st,
        prev, cur, o1, o2, r0, vt, tt, p.Lx, p.Ly, units, slot(n + 1), slot(n + 2), ctx->d_status,
        p.realv ? 1 : 0, nullptr, nullptr);
    bytes += launch_bytes(5);
    rotate(o1, o2);
    n += 2;
    ++launches;
  } else if (n + 1 <= M - 1) {
    void *o1 = nullptr, *o2 = nullptr;
    take_free(prev, cur, &o1, &o2);
    launch_pdl(k_step<Real, LAT, C, false, 0, NST1>, G, kBlock, SM1, st,
        prev, cur, o1, r0, vt, tt, p.Lx, p.Ly, units, slot(n + 1), nullptr, ctx->d_status, 0, FamOut{},
        p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
    bytes += launch_bytes(4);
    rotate(cur, o1);
    n += 1;
    ++launches;
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  const int total = M * Q;
  k_reduce<<<(total + 255) / 256, 256, 0, st>>>(partial, M, G, Q, nvec, vec_base, n_eff, mu_vec,
                                                 p.realv ? 1 : 0);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  float ms = 0.f;
  KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
  KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
  *step_seconds += 1e-3 * ms;
  *step_launches += launches;
  *step_bytes += bytes;
  *last_cur = cur;
  *last_prev = prev;
  return KITE_OK;
}

// ---- autotuner: ring depth x resident CTAs per SM ------------------------------------
// Candidates are timed on the caller's own buffers, which the sweep overwrites afterwards:
// a few non-first steps from two iterate buffers with r_{n+1} written over r_{n-1} (the
// sweep's four streams), and two-step passes from two iterate buffers into the other two.
// The fastest per recursion step is cached per (precision, lattice, vectors per orbital,
// mode, size bucket) on the context.  KITE_AUTOTUNE=0 keeps the default (8 stages, full
// occupancy, one step per pass).
struct Tune {
  int nst;       // ring depth: 4 or 8 (two-step pass: 5, 6 or 8)
  int k;         // resident CTAs per SM
  int two = 0;   // 1: two recursion steps per pass (temporal blocking)
};

inline bool autotune_enabled() {
  const char* e = getenv("KITE_AUTOTUNE");
  return !(e && e[0] == '0');
}

// KITE_PASS_STEPS=1, 2 or 3 pins the steps per pass of the plain moment sweep (the
// autotuner then chooses only the ring depth and occupancy); unset, all are candidates.
inline int pass_steps_pinned() {
  const char* e = getenv("KITE_PASS_STEPS");
  return (e && (e[0] == '1' || e[0] == '2' || e[0] == '3') && e[1] == 0) ? e[0] - '0' : 0;
}

template <typename Real, int LAT, int C, int NST, bool DBL = false>
int step2_grid(kite_ctx* ctx, long long units, int ctas_per_sm = 0) {
  const int occ = std::max(1, step2_occupancy<Real, LAT, C, NST, DBL>());
  const int k = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  return (int)std::max(1LL, std::min((long long)ctx->num_sms * k, units));
}

// Seconds per recursion step of the two-step pass (DBL: its doubling form): three launches
// = six steps.
template <typename Real, int LAT, int C, int NST, bool DBL = false>
float time_candidate2(kite_ctx* ctx, int k, long long units, const Plan& p, const Real* vt, Real tt,
                      void* r0, void* bA, void* bB, void* bC, void* bD, double* partial) {
  constexpr int SMEM = Step2Shape<LAT, C, NST, DBL>::SMEM;
  constexpr int Q = 2 * C * Chunk<Real>::kVecs;
  const int G = step2_grid<Real, LAT, C, NST, DBL>(ctx, units, k);
  cudaStream_t st = ctx->stream;
  auto launch = [&]() {
    launch_pdl(k_step2<Real, LAT, C, NST, DBL>, G, kBlock2, SMEM, st,
        bA, bB, bC, bD, r0, vt, tt, p.Lx, p.Ly, units, partial + (size_t)2 * G * Q,
        partial + (size_t)3 * G * Q, ctx->d_status, p.realv ? 1 : 0,
        DBL ? partial + (size_t)4 * G * Q : nullptr, DBL ? partial + (size_t)5 * G * Q : nullptr);
  };
  launch();  // warm-up
  cudaEventRecord(ctx->ev2, st);
  for (int i = 0; i < 3; ++i) launch();
  cudaEventRecord(ctx->ev3, st);
  float ms = 1e30f;
  if (cudaEventSynchronize(ctx->ev3) != cudaSuccess || cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3) != cudaSuccess)
    return 1e30f;
  return ms / 6.0f;
}

template <typename Real, int LAT, int C, int NST>
int step3_grid(kite_ctx* ctx, long long units, int ctas_per_sm = 0) {
  const int occ = std::max(1, step3_occupancy<Real, LAT, C, NST>());
  const int k = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  return (int)std::max(1LL, std::min((long long)ctx->num_sms * k, units));
}

// Seconds per recursion step of the three-step pass: three launches = nine steps.
template <typename Real, int LAT, int C, int NST>
float time_candidate3(kite_ctx* ctx, int k, long long units, const Plan& p, const Real* vt, Real tt,
                      void* r0, void* bA, void* bB, void* bC, void* bD, double* partial) {
  constexpr int SMEM = Step3Shape<LAT, C, NST>::SMEM;
  constexpr int Q = 2 * C * Chunk<Real>::kVecs;
  const int G = step3_grid<Real, LAT, C, NST>(ctx, units, k);
  cudaStream_t st = ctx->stream;
  auto launch = [&]() {
    launch_pdl(k_step3<Real, LAT, C, NST>, G, kBlock3, SMEM, st,
        bA, bB, bC, bD, r0, vt, tt, p.Lx, p.Ly, units, partial + (size_t)2 * G * Q,
        partial + (size_t)3 * G * Q, partial + (size_t)4 * G * Q, ctx->d_status, p.realv ? 1 : 0);
  };
  launch();  // warm-up
  cudaEventRecord(ctx->ev2, st);
  for (int i = 0; i < 3; ++i) launch();
  cudaEventRecord(ctx->ev3, st);
  float ms = 1e30f;
  if (cudaEventSynchronize(ctx->ev3) != cudaSuccess || cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3) != cudaSuccess)
    return 1e30f;
  return ms / 9.0f;
}

template <typename Real, int LAT, int C, int MODE, int NST>
float time_candidate(kite_ctx* ctx, int k, long long units, const Plan& p, const Real* vt, Real tt, void* r0,
                     void* bA, void* bB, double* partial) {
  constexpr int SMEM = StepShape<LAT, C, NST>::template smem_bytes<MODE>();
  constexpr int Q = 2 * C * Chunk<Real>::kVecs;
  const int G = grid_for<Real, LAT, C, false, MODE, NST>(ctx, units, k);
  cudaStream_t st = ctx->stream;
  auto launch = [&]() {
    // r_{n-1} = bA, r_n = bB, r_{n+1} over r_{n-1} in place, r_0 apart: the sweep's streams
    launch_pdl(k_step<Real, LAT, C, false, MODE, NST>, G, kBlock, SMEM, st,
        bA, bB, bA, MODE == 0 ? r0 : nullptr, vt, tt, p.Lx, p.Ly, units, partial + (size_t)2 * G * Q,
        MODE == 3 ? partial + (size_t)G * Q : nullptr, ctx->d_status, 0, FamOut{}, p.realv ? 1 : 0, SeriesOut{}, nullptr, p.open);
  };
  launch();  // warm-up
  cudaEventRecord(ctx->ev2, st);
  for (int i = 0; i < 3; ++i) launch();
  cudaEventRecord(ctx->ev3, st);
  float ms = 1e30f;
  if (cudaEventSynchronize(ctx->ev3) != cudaSuccess || cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3) != cudaSuccess)
    return 1e30f;
  return ms / 3.0f;  // per recursion step
}

// The two-step pass is a candidate of the plain moment sweep (MODE 0) and of the doubling
// sweep (MODE 3) with enough moments for at least one pass.
template <int MODE>
bool two_step_allowed(const Plan& p) {
  // a field or an open boundary takes the one-step kernel (its variants stage the
  // neighbours the pass would have to rotate or zero in its halo)
  // (doubling: at least one pass after the first step, ceil(M/2) >= 3)
  return (MODE == 0 ? p.M >= 4 : (MODE == 3 && p.M >= 5)) && !p.field && !p.open.x && !p.open.y &&
         pass_steps_pinned() != 1;
}

template <typename Real, int LAT, int C, int MODE>
Tune autotune(kite_ctx* ctx, long long units, const Plan& p, const Real* vt, Real tt, void* r0, void* bA,
              void* bB, void* bC, void* bD, double* partial) {
  const bool two_ok = two_step_allowed<MODE>(p);
  const bool two_only = two_ok && pass_steps_pinned() == 2;
  // the three-step pass (at least one pass after the first step) runs only when pinned
  // (KITE_PASS_STEPS=3 or KITE_TUNE=...x3): on GB300 it measured slower than the two-step
  // pass wherever the two differ (2.5e11 against 3.2e11 updates/s on the 4096^2 workload:
  // at two CTAs per SM its latency is not hidden), so the autotuner does not time it
  const bool three_ok = two_ok && MODE == 0 && p.M >= 5;
  const bool three_only = three_ok && pass_steps_pinned() == 3;
  Tune def{kStages, step_occupancy<Real, LAT, C, MODE, kStages>(), 0};
  constexpr bool DB = MODE == 3;
  if (two_only) def = Tune{5, std::max(1, step2_occupancy<Real, LAT, C, 5, DB>()), 1};
  if (three_only) def = Tune{8, std::max(1, step3_occupancy<Real, LAT, C, 8>()), 2};
  // KITE_TUNE=<stages>x<CTAs per SM>[x2|x3] pins one configuration (reproducible
  // profiles): stages 4 or 8 (5, 6 or 8 for the two-step pass, 7 or 8 for the three-step
  // pass), x2 / x3 = two / three steps per pass
  if (const char* e = getenv("KITE_TUNE")) {
    int nst = 0, k = 0, two = 1;
    if (sscanf(e, "%dx%dx%d", &nst, &k, &two) >= 2) {
      if (two == 3 && three_ok) {
        const int occ = nst == 7 ? step3_occupancy<Real, LAT, C, 7>() : nst == 8 ? step3_occupancy<Real, LAT, C, 8>() : 0;
        if (occ > 0 && k >= 1) return Tune{nst, std::min(k, occ), 2};
      }
      const bool t2 = two == 2 && two_ok;
      const int occ = t2 ? (nst == 5   ? step2_occupancy<Real, LAT, C, 5, DB>()
                            : nst == 6 ? step2_occupancy<Real, LAT, C, 6, DB>()
                            : nst == 8 ? step2_occupancy<Real, LAT, C, 8, DB>() : 0)
                         : (nst == 4   ? step_occupancy<Real, LAT, C, MODE, 4>()
                            : nst == 8 ? step_occupancy<Real, LAT, C, MODE, 8>() : 0);
      if (occ > 0 && k >= 1) return Tune{nst, std::min(k, occ), t2 ? 1 : 0};
    }
  }
  if (!autotune_enabled() || units < 4LL * ctx->num_sms) return def;
  int bucket = 0;
  while ((1LL << (bucket + 1)) <= units) ++bucket;
  const uint64_t key = ((uint64_t)1 << 56) | ((uint64_t)sizeof(Real) << 48) | ((uint64_t)LAT << 40) |
                       ((uint64_t)C << 32) | ((uint64_t)MODE << 24) | ((uint64_t)p.realv << 16) |
                       ((uint64_t)(two_ok ? 1 + two_only : 0) << 20) |
                       ((uint64_t)three_only << 22) | (uint64_t)bucket;
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return Tune{it->second.first & 0xff, it->second.second, it->second.first >> 8};
  Tune best = def;
  float best_ms = 1e30f, best2 = 1e30f;
  if (!two_only && !three_only) {
    const int o8 = step_occupancy<Real, LAT, C, MODE, 8>(), o4 = step_occupancy<Real, LAT, C, MODE, 4>();
    for (int k = 1; k <= o8; ++k) {
      const float ms = time_candidate<Real, LAT, C, MODE, 8>(ctx, k, units, p, vt, tt, r0, bA, bB, partial);
      if (ms < best_ms) best_ms = ms, best = Tune{8, k, 0};
    }
    for (int k = 1; k <= o4; ++k) {
      const float ms = time_candidate<Real, LAT, C, MODE, 4>(ctx, k, units, p, vt, tt, r0, bA, bB, partial);
      if (ms < best_ms * 0.98f) best_ms = ms, best = Tune{4, k, 0};  // prefer the deeper ring on a tie
    }
  }
  if (two_ok && !three_only) {
    // per-step time of the pass against the one-step kernels' (the pass must win clearly:
    // it needs two extra iterate buffers)
    const float bar = two_only ? 1e30f : 0.97f * best_ms;
    best2 = bar;
    const int o8 = step2_occupancy<Real, LAT, C, 8, DB>(), o6 = step2_occupancy<Real, LAT, C, 6, DB>(),
              o5 = step2_occupancy<Real, LAT, C, 5, DB>();
    for (int k = 1; k <= o8; ++k) {
      const float ms = time_candidate2<Real, LAT, C, 8, DB>(ctx, k, units, p, vt, tt, r0, bA, bB, bC, bD, partial);
      if (ms < best2) best2 = ms, best = Tune{8, k, 1};
    }
    for (int k = 1; k <= o6; ++k) {
      const float ms = time_candidate2<Real, LAT, C, 6, DB>(ctx, k, units, p, vt, tt, r0, bA, bB, bC, bD, partial);
      if (ms < best2 * 0.98f) best2 = ms, best = Tune{6, k, 1};
    }
    for (int k = 1; k <= o5; ++k) {
      const float ms = time_candidate2<Real, LAT, C, 5, DB>(ctx, k, units, p, vt, tt, r0, bA, bB, bC, bD, partial);
      if (ms < best2 * 0.98f) best2 = ms, best = Tune{5, k, 1};
    }
  }
  if (three_only) {
    float best3 = 1e30f;
    const int o8 = step3_occupancy<Real, LAT, C, 8>(), o7 = step3_occupancy<Real, LAT, C, 7>();
    for (int k = 1; k <= o8; ++k) {
      const float ms = time_candidate3<Real, LAT, C, 8>(ctx, k, units, p, vt, tt, r0, bA, bB, bC, bD, partial);
      if (ms < best3) best3 = ms, best = Tune{8, k, 2};
    }
    for (int k = 1; k <= o7; ++k) {
      const float ms = time_candidate3<Real, LAT, C, 7>(ctx, k, units, p, vt, tt, r0, bA, bB, bC, bD, partial);
      if (ms < best3 * 0.98f) best3 = ms, best = Tune{7, k, 2};
    }
  }
  cudaGetLastError();
  ctx->tune[key] = {best.nst | (best.two << 8), best.k};
  return best;
}

template <typename Real, int LAT, int MODE>
int max_grid_c(kite_ctx* ctx, int C, long long units) {
  auto g = [&](int occ) { return (int)std::max(1LL, std::min((long long)ctx->num_sms * occ, units)); };
  auto occ = [&](auto cc) {
    constexpr int CC = decltype(cc)::value;
    int o = std::max(step_occupancy<Real, LAT, CC, MODE, 8>(), step_occupancy<Real, LAT, CC, MODE, 4>());
    if (MODE == 0 || MODE == 3)
      o = std::max({o, step2_occupancy<Real, LAT, CC, 8, MODE == 3>(), step2_occupancy<Real, LAT, CC, 6, MODE == 3>(),
                    step2_occupancy<Real, LAT, CC, 5, MODE == 3>()});
    return o;
  };
  if (C == 1) return g(occ(std::integral_constant<int, 1>{}));
  if (C == 2) return g(occ(std::integral_constant<int, 2>{}));
  return g(occ(std::integral_constant<int, 4>{}));
}

// ---- small lattices: the on-chip cluster sweep (kite_cluster.cu) ----------------------
// KITE_CLUSTER=0 never takes it and KITE_CLUSTER=1 takes it whenever the lattice fits
// (KITE_CLUSTER_CTAS=2..16 then pins the cluster size); unset, it is a candidate of the
// autotuner for lattices too small to give the streaming step kernels four work units per
// SM, and runs when it is measured faster per recursion step.  It needs a real H~ (no
// field) and at least 4 rows.
inline int cluster_pinned() {  // 0 unset, 1 off, 2 on
  const char* e = getenv("KITE_CLUSTER");
  return (e && (e[0] == '0' || e[0] == '1') && e[1] == 0) ? e[0] - '0' + 1 : 0;
}
inline int cluster_ctas_pinned() {
  const char* e = getenv("KITE_CLUSTER_CTAS");
  const int v = e ? atoi(e) : 0;
  return (v >= 2 && v <= 16) ? v : 0;
}
constexpr int kClusterTimeSteps = 40;  // longest timing run of the autotuner

// Per-step seconds of the cluster sweep: two timing runs, 8 and 40 steps, so that the
// launch and load cost drops out.
inline float cluster_step_ms(kite_ctx* ctx, ClusterSweep c) {
  if (cluster_sweep(ctx, &c, 8) != KITE_OK) return 1e30f;
  if (cluster_sweep(ctx, &c, 8) != KITE_OK) return 1e30f;
  const double t8 = c.seconds;
  if (cluster_sweep(ctx, &c, kClusterTimeSteps) != KITE_OK) return 1e30f;
  return (float)(1e3 * std::max(0.0, c.seconds - t8) / (kClusterTimeSteps - 8));
}

// Cluster size to run the batch with, 0 for the streaming kernels.  `stream_ms` times the
// streaming kernels' default launch per step (only called when the autotuner compares).
template <typename StreamMs>
int cluster_choice(kite_ctx* ctx, const Plan& p, const ClusterSweep& c, long long units,
                   StreamMs stream_ms) {
  const int pin = cluster_pinned();
  if (pin == 1 || p.field || ctx->debug_stall) return 0;
  // pinning the streaming kernels (KITE_PASS_STEPS, KITE_TUNE) or turning the autotuner off
  // keeps them
  if (pin == 0 && (!autotune_enabled() || pass_steps_pinned() || getenv("KITE_TUNE") ||
                   units >= 4LL * ctx->num_sms))
    return 0;
  // Cluster sizes from 16 CTAs down: more CTAs split the work of a step further, but fewer
  // clusters are resident at once (on GB300 7 of 16 CTAs, 8 of 12, 15 of 8), and a batch
  // with more lanes than that runs in several waves.  The candidates are the largest size
  // for each number of waves (eight FP64 lanes: 16 and 12 CTAs; sixteen FP32 lanes: 16, 12
  // and 6).
  const int fixed = cluster_ctas_pinned();
  const int lanes = c.realv ? c.nvec : 2 * c.nvec;
  int cand[16], nc = 0, one_wave = 0, fewest = 1 << 30;
  for (int cs = 16; cs >= (fixed ? 2 : 4); --cs) {
    if (fixed && cs != fixed) continue;
    const int act = cluster_active(ctx, c, cs);
    if (act < 1) continue;
    const int waves = (lanes + act - 1) / act;
    if (waves >= fewest) continue;
    fewest = waves;
    cand[nc++] = cs;
    if (!one_wave && waves == 1) one_wave = cs;
  }
  if (nc == 0) return 0;
  if (pin == 2) return one_wave ? one_wave : cand[0];
  uint64_t key = 0x6b69746563737470ull;
  for (uint64_t f : {(uint64_t)c.fp64, (uint64_t)c.lattice, (uint64_t)c.doubling, (uint64_t)c.realv,
                     (uint64_t)c.nvec, (uint64_t)c.C, (uint64_t)c.Lx, (uint64_t)c.Ly, (uint64_t)c.open_x,
                     (uint64_t)c.open_y})
    key = (key ^ f) * 0x100000001b3ull;
  key |= 1ull << 63;
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return it->second.first;
  float best = 0.9f * stream_ms();  // the cluster sweep must win clearly
  int pick = 0;
  for (int k = 0; k < nc; ++k) {
    ClusterSweep t = c;
    t.cs = cand[k];
    const float ms = cluster_step_ms(ctx, t);
    if (ms < best) best = ms, pick = cand[k];
  }
  cudaGetLastError();
  ctx->tune[key] = {pick, 0};
  return pick;
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
  p.field = sys->flux != 0.0;
  {
    const void* z = nullptr;
    const int rc = open_zeros(ctx, sys, &z);
    if (rc != KITE_OK) return rc;
    p.open.zero = static_cast<const unsigned char*>(z);
    p.open.x = sys->open_x;
    p.open.y = sys->open_y;
  }
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
  // two more iterate buffers when the two-step pass may run (its outputs never alias its
  // inputs)
  const bool two_possible = (p.doubling ? p.M >= 5 : p.M >= 4) && !p.field && pass_steps_pinned() != 1;
  // the cluster sweep's moment partials (16 CTAs per lane, the larger size)
  const size_t cluster_part =
      (p.field || cluster_pinned() == 1)
          ? 0
          : cluster_part_doubles(p.realv ? p.max_batch : 2 * p.max_batch, 16, p.M, p.doubling, kClusterTimeSteps);
  auto plan_ws = [&](Carver& k, Real** vt, void** r0, void** bA, void** bB, void** bC, void** bD,
                     double** partial, unsigned long long** ne, double** mu_vec, Real** phase) {
    *vt = k.take<Real>(p.N);
    *phase = p.field ? k.take<Real>((size_t)p.Ly * SORB * 4) : nullptr;
    *r0 = k.take<char>(vec_bytes);
    *bA = k.take<char>(vec_bytes);
    *bB = k.take<char>(vec_bytes);
    *bC = two_possible ? k.take<char>(vec_bytes) : nullptr;
    *bD = two_possible ? k.take<char>(vec_bytes) : nullptr;
    *partial = k.take<double>(std::max((size_t)(std::max(p.M, 2) + 1) * Gmax * 2 * Cmax * VPC, cluster_part));
    *ne = k.take<unsigned long long>(1);
    *mu_vec = k.take<double>(nvec_total * p.M * 2);
  };
  Real* vt;
  void *r0, *bA, *bB, *bC, *bD;
  double *partial, *mu_vec;
  unsigned long long* ne;
  Real* phase;
  plan_ws(cv, &vt, &r0, &bA, &bB, &bC, &bD, &partial, &ne, &mu_vec, &phase);
  int rc = ensure_ws(ctx, cv.used());
  if (rc != KITE_OK) return rc;
  Carver real(ctx->ws);
  plan_ws(real, &vt, &r0, &bA, &bB, &bC, &bD, &partial, &ne, &mu_vec, &phase);
  if (p.field) {
    rc = field_phases(ctx, sys, sizeof(Real) == 8, phase);
    if (rc != KITE_OK) return rc;
  }
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
  int cluster_used = 0, steps_used = 0;
  double step_s = 0.0, step_bytes = 0.0;
  int64_t step_n = 0;
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  for (int s = 0; s < p.S; ++s) {
    KITE_CUDA_TRY(ctx, cudaMemsetAsync(ne, 0, sizeof(unsigned long long), st));
    {
      const int64_t blocks = std::min<int64_t>((p.N + 255) / 256, (int64_t)ctx->num_sms * 16);
      k_onsite<Real><<<(int)std::max<int64_t>(1, blocks), 256, 0, st>>>(
          p.N, sys->lattice, sys->W, 0.5 * sys->delta, sc.de_plus, sc.de_minus, vac_thr,
          (uint32_t)s, k0, k1, vt, ne, sys->disorder);
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
#define KITE_SWEEP(CC)                                                                              \
  do {                                                                                              \
    Tune t = p.doubling ? autotune<Real, LAT, CC, 3>(ctx, u, p, vt, tt, r0, bA, bB, bC, bD, partial)  \
                        : autotune<Real, LAT, CC, 0>(ctx, u, p, vt, tt, r0, bA, bB, bC, bD, partial); \
    tune_used = t;                                                                                  \
    if (t.two == 2) {                                                                               \
      const int G = t.nst == 7 ? step3_grid<Real, LAT, CC, 7>(ctx, u, t.k)                          \
                               : step3_grid<Real, LAT, CC, 8>(ctx, u, t.k);                         \
      grid_used = G;                                                                                \
      auto run3 = [&](auto nst) {                                                                   \
        return sweep_three<Real, LAT, CC, decltype(nst)::value>(ctx, p, vt, tt, r0, bA, bB, bC, bD,  \
                                                                 partial, G, u, nvec, vec_base, ne,  \
                                                                 mu_vec, &lp, &lc, &step_s, &step_n, \
                                                                 &step_bytes);                       \
      };                                                                                            \
      rc = t.nst == 7 ? run3(std::integral_constant<int, 7>{}) : run3(std::integral_constant<int, 8>{}); \
    } else if (t.two && p.doubling) {                                                               \
      const int G = t.nst == 5   ? step2_grid<Real, LAT, CC, 5, true>(ctx, u, t.k)                  \
                    : t.nst == 6 ? step2_grid<Real, LAT, CC, 6, true>(ctx, u, t.k)                  \
                                 : step2_grid<Real, LAT, CC, 8, true>(ctx, u, t.k);                 \
      grid_used = G;                                                                                \
      auto run2 = [&](auto nst) {                                                                   \
        return sweep_two_dbl<Real, LAT, CC, decltype(nst)::value>(ctx, p, vt, tt, r0, bA, bB, bC, bD, \
                                                                   partial, G, u, nvec, vec_base, ne, \
                                                                   mu_vec, &lp, &lc, &step_s,        \
                                                                   &step_n, &step_bytes);            \
      };                                                                                            \
      rc = t.nst == 5   ? run2(std::integral_constant<int, 5>{})                                    \
           : t.nst == 6 ? run2(std::integral_constant<int, 6>{})                                    \
                        : run2(std::integral_constant<int, 8>{});                                   \
    } else if (t.two) {                                                                             \
      const int G = t.nst == 5   ? step2_grid<Real, LAT, CC, 5>(ctx, u, t.k)                        \
                    : t.nst == 6 ? step2_grid<Real, LAT, CC, 6>(ctx, u, t.k)                        \
                                 : step2_grid<Real, LAT, CC, 8>(ctx, u, t.k);                       \
      grid_used = G;                                                                                \
      auto run2 = [&](auto nst) {                                                                   \
        return sweep_two<Real, LAT, CC, decltype(nst)::value>(ctx, p, vt, tt, r0, bA, bB, bC, bD,    \
                                                               partial, G, u, nvec, vec_base, ne,    \
                                                               mu_vec, &lp, &lc, &step_s, &step_n,   \
                                                               &step_bytes);                         \
      };                                                                                            \
      rc = t.nst == 5   ? run2(std::integral_constant<int, 5>{})                                    \
           : t.nst == 6 ? run2(std::integral_constant<int, 6>{})                                    \
                        : run2(std::integral_constant<int, 8>{});                                   \
    } else {                                                                                        \
      const int G = t.nst == 4 ? (p.doubling ? grid_for<Real, LAT, CC, false, 3, 4>(ctx, u, t.k)      \
                                             : grid_for<Real, LAT, CC, false, 0, 4>(ctx, u, t.k))     \
                               : (p.doubling ? grid_for<Real, LAT, CC, false, 3, 8>(ctx, u, t.k)      \
                                             : grid_for<Real, LAT, CC, false, 0, 8>(ctx, u, t.k));    \
      grid_used = G;                                                                                \
      rc = t.nst == 4 ? sweep_batch<Real, LAT, CC, 4>(ctx, p, vt, tt, r0, bA, bB, partial, G, u, nvec, \
                                                      vec_base, ne, mu_vec, &lp, &lc, &step_s,       \
                                                      &step_n, &step_bytes)                          \
                      : sweep_batch<Real, LAT, CC, 8>(ctx, p, vt, tt, r0, bA, bB, partial, G, u, nvec, \
                                                      vec_base, ne, mu_vec, &lp, &lc, &step_s,       \
                                                      &step_n, &step_bytes);                         \
    }                                                                                               \
  } while (0)
      ClusterSweep cl{};
      cl.fp64 = sizeof(Real) == 8;
      cl.lattice = LAT;
      cl.doubling = p.doubling;
      cl.realv = p.realv;
      cl.Lx = p.Lx;
      cl.Ly = p.Ly;
      cl.M = p.M;
      cl.C = C;
      cl.per_chunk = per_chunk;
      cl.nvec = nvec;
      cl.open_x = p.open.x;
      cl.open_y = p.open.y;
      cl.r0 = r0;
      cl.vt = vt;
      cl.tt = (double)tt;
      cl.part = partial;
      cl.n_eff = ne;
      cl.mu_vec = mu_vec;
      cl.vec_base = vec_base;
      auto stream_ms = [&]() -> float {
        auto one = [&](auto cc) {
          constexpr int CC = decltype(cc)::value;
          return p.doubling
                     ? time_candidate<Real, LAT, CC, 3, kStages>(ctx, step_occupancy<Real, LAT, CC, 3, kStages>(), u, p,
                                                                 vt, tt, r0, bA, bB, partial)
                     : time_candidate<Real, LAT, CC, 0, kStages>(ctx, step_occupancy<Real, LAT, CC, 0, kStages>(), u, p,
                                                                 vt, tt, r0, bA, bB, partial);
        };
        return C == 1 ? one(std::integral_constant<int, 1>{})
                      : (C == 2 ? one(std::integral_constant<int, 2>{}) : one(std::integral_constant<int, 4>{}));
      };
      const bool want_last = kpm->r_last && !p.doubling;
      cl.last_prev = want_last ? bA : nullptr;
      cl.last_cur = want_last ? bB : nullptr;
      cl.cs = cluster_choice(ctx, p, cl, u, stream_ms);
      if (cl.cs > 0) {
        // small lattice: the whole sweep on chip (kite_cluster.cu)
        rc = cluster_sweep(ctx, &cl, 0);
        if (rc != KITE_OK) return rc;
        step_s += cl.seconds;
        step_n += 1;
        step_bytes += cl.bytes;
        grid_used = cl.grid;
        tune_used = Tune{0, 1, 0};
        cluster_used = cl.cs;
        steps_used = p.doubling ? (p.M + 1) / 2 : p.M - 1;
        lp = bA;
        lc = bB;
      } else if (p.field) {
        // magnetic field: the one-step sweep with Peierls phases (kite_field.cu)
        const int occ = field_occupancy(sizeof(Real) == 8, LAT, C, p.doubling);
        FieldSweep fs{};
        fs.fp64 = sizeof(Real) == 8;
        fs.lattice = LAT;
        fs.C = C;
        fs.doubling = p.doubling;
        fs.Lx = p.Lx;
        fs.Ly = p.Ly;
        fs.M = p.M;
        fs.units = u;
        fs.G = (int)std::max(1LL, std::min({(long long)ctx->num_sms * occ, u, (long long)Gmax}));
        fs.stall = ctx->debug_stall;
        fs.zero = p.open.zero;
        fs.open_x = p.open.x;
        fs.open_y = p.open.y;
        fs.ncell = p.ncell;
        fs.N = p.N;
        fs.vt = vt;
        fs.tt = (double)tt;
        fs.r0 = r0;
        fs.bA = bA;
        fs.bB = bB;
        fs.partial = partial;
        fs.phase = phase;
        ctx->debug_stall = 0;
        rc = field_sweep(ctx, &fs);
        if (rc != KITE_OK) return rc;
        const int Q = 2 * C * VPC;
        k_reduce<<<(p.M * Q + 255) / 256, 256, 0, st>>>(partial, p.M, fs.G, Q, nvec, vec_base, ne, mu_vec,
                                                       0);
        if (p.doubling) k_undouble<<<(nvec * p.M + 255) / 256, 256, 0, st>>>(mu_vec, p.M, nvec, vec_base);
        KITE_CUDA_TRY(ctx, cudaGetLastError());
        lp = fs.last_prev;
        lc = fs.last_cur;
        step_s += fs.seconds;
        step_n += fs.launches;
        step_bytes += fs.bytes;
        grid_used = fs.G;
        tune_used = Tune{8, occ, 0};
      } else if (C == 1) KITE_SWEEP(1);
      else if (C == 2) KITE_SWEEP(2);
      else KITE_SWEEP(4);
#undef KITE_SWEEP
      if (rc != KITE_OK) return rc;
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
  }
  {
    const int nv = (int)nvec_total;
    k_average<<<(p.M + 255) / 256, 256, 0, st>>>(mu_vec, nv, p.M, mu_dev, imag_dev);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, st));
  {
    // one read-back for the whole call: the status word collects every realisation's
    // bounded waits, and `ne` holds the last realisation's N_eff
    unsigned long long ne_host = 0;
    int status_host = 0;
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&ne_host, ne, sizeof(ne_host), cudaMemcpyDeviceToHost, st));
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&status_host, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (status_host != 0)
      return fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up in the step kernel");
    n_eff_last = (int64_t)ne_host;
  }
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->seconds = ms * 1e-3;
    stats->updates = (double)n_eff_last * p.M * p.R * p.S;
    // algorithmic bytes of the step launches as scheduled: per launch, the iterate
    // streams read and written (r_{n-1}, r_n, r_0 in and r_{n+1} out for a plain step;
    // r_{n-1}, r_n, r_0 in and r_{n+1}, r_{n+2} out for a two-step pass; no r_0 with
    // doubling) for each of the batch's 16-byte chunks, plus one read of the on-site term
    stats->bytes_moved = step_bytes;
    stats->gbps = stats->seconds > 0 ? stats->bytes_moved / stats->seconds * 1e-9 : 0.0;
    stats->n_eff = n_eff_last;
    stats->grid = grid_used;
    stats->block = kBlock;
    stats->ring_stages = tune_used.nst;
    stats->steps_per_pass = cluster_used ? steps_used : tune_used.two + 1;
    stats->cluster_ctas = cluster_used;
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
