// kite_field.cu -- the 1D moment sweep in a perpendicular magnetic field (Peierls
// substitution, Sec. "Magnetic Field").
//
// The field only changes the hoppings: t -> t exp(i theta) on every bond with an x
// component, theta = -2 pi (flux/A_cell)(y_o - dy/2) dx in the Landau gauge A = (-B y, 0)
// (bond offset (dx, dy) = r_o - r_j, y_o the orbital's y coordinate), so the phases depend
// on the row and the sublattice only.  k_peierls tabulates them once per call
// ([y][s][bond][cos, sin], FP64 sincos rounded once to the working precision); the sweep
// runs the one-step kernel's FIELD variant, which rotates the neighbours of the two
// x bonds before the stencil sum.  Everything else (start vectors, moments, doubling,
// reductions) is the plain sweep's.  Its kernels live in this translation unit so that the
// field variants do not lengthen the main sweep's build.
#include <algorithm>

#include "kite_device.cuh"
#include "kite_internal.h"

#include "kite_step.cuh"

namespace kite {
namespace {

// Phase table of the bonds with an x component: honeycomb bonds n2 = B(x+1, y-1),
// n3 = B(x, y-1) of A (offsets (-1/2, a_cc/2), (1/2, a_cc/2)) and n2 = A(x-1, y+1),
// n3 = A(x, y+1) of B (the negatives); square bonds n1 = (x-1, y), n2 = (x+1, y)
// (offsets (1, 0), (-1, 0)).  Same operation order as the oracle's FP64 phases.
template <typename Real>
__global__ void k_peierls(int lattice, int Ly, double flux, Real* __restrict__ ph) {
  const int sorb = lattice == KITE_HONEYCOMB ? 2 : 1;
  const int total = Ly * sorb * 2;
  const double sq3 = sqrt(3.0);
  const double acc = __ddiv_rn(1.0, sq3);
  const double area = lattice == KITE_HONEYCOMB ? __dmul_rn(0.5, sq3) : 1.0;
  const double k = __ddiv_rn(__dmul_rn(__dmul_rn(-2.0, 3.141592653589793), flux), area);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int b = e & 1, s = (e >> 1) % sorb, y = (e >> 1) / sorb;
    double dx, dy, yo;
    if (lattice == KITE_HONEYCOMB) {
      dx = s == 0 ? (b == 0 ? -0.5 : 0.5) : (b == 0 ? 0.5 : -0.5);
      dy = __dmul_rn(s == 0 ? 0.5 : -0.5, acc);
      yo = __dadd_rn(__dmul_rn(__dmul_rn(0.5, sq3), (double)y), __dmul_rn(s == 0 ? -0.5 : 0.5, acc));
    } else {
      dx = b == 0 ? 1.0 : -1.0;
      dy = 0.0;
      yo = (double)y;
    }
    const double th = __dmul_rn(__dmul_rn(k, __dsub_rn(yo, __dmul_rn(0.5, dy))), dx);
    double sn, cs;
    sincos(th, &sn, &cs);
    ph[2 * e] = (Real)cs;
    ph[2 * e + 1] = (Real)sn;
  }
}

constexpr int kFieldStages = 8;

template <typename Real, int LAT, int C, int MODE>
int field_occupancy_t() {
  static int occ = -1;
  if (occ < 0) {
    constexpr int SM = StepShape<LAT, C, kFieldStages>::template smem_bytes<MODE>();
    cudaFuncSetAttribute(k_step<Real, LAT, C, true, MODE, kFieldStages, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
    cudaFuncSetAttribute(k_step<Real, LAT, C, false, MODE, kFieldStages, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_step<Real, LAT, C, false, MODE, kFieldStages, true>,
                                                      kBlock, SM) != cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}

// The step launches of one vector batch (the plain sweep's schedule, one step per launch):
// MODE 0 writes the moment partial slots 0 .. M-1, MODE 3 (doubling) the slots 0 .. 2*steps-1.
template <typename Real, int LAT, int C, int MODE>
int sweep_field_t(kite_ctx* ctx, FieldSweep* a) {
  constexpr int NST = kFieldStages;
  constexpr int Q = 2 * C * Chunk<Real>::kVecs;
  constexpr int SM = StepShape<LAT, C, NST>::template smem_bytes<MODE>();
  field_occupancy_t<Real, LAT, C, MODE>();  // sets the shared-memory limits
  cudaStream_t st = ctx->stream;
  const int G = a->G, M = a->M;
  const Real tt = (Real)a->tt;
  const Real* vt = static_cast<const Real*>(a->vt);
  Open open;
  open.zero = static_cast<const unsigned char*>(a->zero);
  open.x = a->open_x;
  open.y = a->open_y;
  auto slot = [&](int k) { return a->partial + (size_t)k * G * Q; };
  // r_0 in r0; r_n (n >= 1) in bA (odd n) or bB (even n); r_{n+1} overwrites r_{n-1}
  auto where = [&](int n) -> void* { return n == 0 ? a->r0 : ((n & 1) ? a->bA : a->bB); };
  const double chunk_bytes = 16.0 * StepShape<LAT, C>::SORB * C * (double)a->ncell;
  auto launch_bytes = [&](int vecs) { return vecs * chunk_bytes + (double)a->N * sizeof(Real); };
  int64_t launches = 0;
  double bytes = 0.0;
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
  if (MODE == 3) {
    const int steps = (M + 1) / 2;
    launch_pdl(k_step<Real, LAT, C, true, 3, NST, true>, G, kBlock, SM, st, nullptr, a->r0, a->bA, nullptr,
               vt, tt, a->Lx, a->Ly, a->units, slot(1), slot(0), ctx->d_status, a->stall, FamOut{}, 0,
               SeriesOut{}, a->phase, open);
    launches = 1;
    bytes = launch_bytes(2);
    for (int n = 1; n < steps; ++n, ++launches) {
      launch_pdl(k_step<Real, LAT, C, false, 3, NST, true>, G, kBlock, SM, st, where(n - 1), where(n),
                 where(n + 1), nullptr, vt, tt, a->Lx, a->Ly, a->units, slot(2 * n + 1), slot(2 * n),
                 ctx->d_status, 0, FamOut{}, 0, SeriesOut{}, a->phase, open);
      bytes += launch_bytes(3);
    }
    a->last_prev = a->last_cur = nullptr;
  } else {
    launch_pdl(k_step<Real, LAT, C, true, 0, NST, true>, G, kBlock, SM, st, nullptr, a->r0, a->bA, a->r0, vt,
               tt, a->Lx, a->Ly, a->units, slot(1), slot(0), ctx->d_status, a->stall, FamOut{}, 0,
               SeriesOut{}, a->phase, open);
    launches = 1;
    bytes = launch_bytes(2);
    for (int n = 1; n + 1 < M; ++n, ++launches) {
      launch_pdl(k_step<Real, LAT, C, false, 0, NST, true>, G, kBlock, SM, st, where(n - 1), where(n),
                 where(n + 1), a->r0, vt, tt, a->Lx, a->Ly, a->units, slot(n + 1), nullptr, ctx->d_status, 0,
                 FamOut{}, 0, SeriesOut{}, a->phase, open);
      bytes += launch_bytes(4);
    }
    a->last_cur = where(M - 1);
    a->last_prev = where(M >= 2 ? M - 2 : 0);
  }
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  float ms = 0.f;
  KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
  KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
  a->seconds = 1e-3 * ms;
  a->launches = launches;
  a->bytes = bytes;
  return KITE_OK;
}

template <typename Real, int LAT, int MODE>
int dispatch_c(kite_ctx* ctx, FieldSweep* a, bool occ_only, int* occ) {
  if (occ_only) {
    *occ = a->C == 1   ? field_occupancy_t<Real, LAT, 1, MODE>()
           : a->C == 2 ? field_occupancy_t<Real, LAT, 2, MODE>()
                       : field_occupancy_t<Real, LAT, 4, MODE>();
    return KITE_OK;
  }
  if (a->C == 1) return sweep_field_t<Real, LAT, 1, MODE>(ctx, a);
  if (a->C == 2) return sweep_field_t<Real, LAT, 2, MODE>(ctx, a);
  return sweep_field_t<Real, LAT, 4, MODE>(ctx, a);
}

int dispatch(kite_ctx* ctx, FieldSweep* a, bool occ_only, int* occ) {
  const bool hc = a->lattice == KITE_HONEYCOMB;
  if (a->fp64) {
    if (a->doubling) return hc ? dispatch_c<double, KITE_HONEYCOMB, 3>(ctx, a, occ_only, occ)
                               : dispatch_c<double, KITE_SQUARE, 3>(ctx, a, occ_only, occ);
    return hc ? dispatch_c<double, KITE_HONEYCOMB, 0>(ctx, a, occ_only, occ)
              : dispatch_c<double, KITE_SQUARE, 0>(ctx, a, occ_only, occ);
  }
  if (a->doubling) return hc ? dispatch_c<float, KITE_HONEYCOMB, 3>(ctx, a, occ_only, occ)
                             : dispatch_c<float, KITE_SQUARE, 3>(ctx, a, occ_only, occ);
  return hc ? dispatch_c<float, KITE_HONEYCOMB, 0>(ctx, a, occ_only, occ)
            : dispatch_c<float, KITE_SQUARE, 0>(ctx, a, occ_only, occ);
}

}  // namespace

int field_phases(kite_ctx* ctx, const kite_system* sys, int fp64, void* table) {
  const int total = sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1) * 2;
  const int blocks = std::max(1, std::min((total + 255) / 256, ctx->num_sms * 4));
  if (fp64)
    k_peierls<double><<<blocks, 256, 0, ctx->stream>>>(sys->lattice, sys->Ly, sys->flux,
                                                        static_cast<double*>(table));
  else
    k_peierls<float><<<blocks, 256, 0, ctx->stream>>>(sys->lattice, sys->Ly, sys->flux,
                                                       static_cast<float*>(table));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

int field_occupancy(int fp64, int lattice, int C, int doubling) {
  FieldSweep a{};
  a.fp64 = fp64;
  a.lattice = lattice;
  a.C = C;
  a.doubling = doubling;
  int occ = 1;
  dispatch(nullptr, &a, true, &occ);
  return occ;
}

int field_sweep(kite_ctx* ctx, FieldSweep* a) { return dispatch(ctx, a, false, nullptr); }

}  // namespace kite
