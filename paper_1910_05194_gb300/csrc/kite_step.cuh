// kite_step.cuh -- device kernels of the Chebyshev recursion shared by the 1D (moment)
// and 2D (vector family) drivers: on-site draws, start vectors, the pipelined stencil
// step and batch/caller layout conversion.  Everything lives in an anonymous namespace,
// so each translation unit instantiates its own copies.
#pragma once

#include <math.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <utility>

#include "kite_device.cuh"
#include "kite_internal.h"

namespace kite {
namespace {

constexpr int kBlock = 256;
constexpr int kFlushRows = 32;  // FP32 moment partials are promoted to FP64 every 32 rows

// ------------------------------------------------------------------------------------
// On-site energies V~_o = (V_o - de_plus)/de_minus of one realisation, a quiet NaN on
// vacancies, and the count of non-vacant orbitals.  Same draws and the same sequence
// of correctly rounded FP64 operations as the problem statement in kite_gb.h.
// ------------------------------------------------------------------------------------
// Gaussian disorder (gaussian != 0): the Box-Muller transform of u1 = 1 - u (in (0, 1])
// and the 32-bit uniform u2 of the fourth word, V = W (sqrt(-2 ln u1) cos(2 pi u2)),
// with CUDA's FP64 log, sqrt and cos (each within an ulp of the host's libm).
template <typename Real>
__global__ void k_onsite(int64_t N, int lattice, double W, double half_delta, double de_plus,
                         double de_minus, uint64_t vac_thr, uint32_t realisation, uint32_t k0,
                         uint32_t k1, Real* __restrict__ vt,
                         unsigned long long* __restrict__ n_eff, int gaussian) {
  unsigned int count = 0;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < N;
       o += (int64_t)gridDim.x * blockDim.x) {
    const Philox4 x = philox4x32_10((uint32_t)o, (uint32_t)((uint64_t)o >> 32), realisation,
                                    kTagDisorder, k0, k1);
    double v;
    if (gaussian) {
      const double u1 = __dsub_rn(1.0, u53(x));
      const double u2 = __dmul_rn((double)x.w[3], 0x1p-32);
      const double radius = sqrt(__dmul_rn(-2.0, log(u1)));
      v = __dmul_rn(W, __dmul_rn(radius, cos(__dmul_rn(6.283185307179586, u2))));
    } else {
      v = __dmul_rn(W, __dsub_rn(u53(x), 0.5));
    }
    if (lattice == KITE_HONEYCOMB && half_delta != 0.0)
      v = __dadd_rn(v, (o & 1) == 0 ? half_delta : -half_delta);
    const bool vacant = (uint64_t)x.w[2] < vac_thr;
    const double vtil = __ddiv_rn(__dsub_rn(v, de_plus), de_minus);
    // stored doubled, 2 V~ (exact: V~ is rounded once to the working precision first), the
    // factor the recursion's 2 H~ r_n needs; the first step halves it back (exact again)
    const Real vr = (Real)vtil;
    vt[o] = vacant ? quiet_nan<Real>() : vr + vr;
    count += vacant ? 0u : 1u;
  }
  // integer sums are order independent: warp-aggregate, one atomic per warp
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) count += __shfl_xor_sync(0xffffffffu, count, d);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(n_eff, (unsigned long long)count);
}

// ------------------------------------------------------------------------------------
// Start vectors of one batch: random phases exp(2 pi i u) or caller vectors (FP64,
// rounded once), zero on vacancies and on padding lanes.
// ------------------------------------------------------------------------------------
// Start vectors of a batch.  Complex (realv = 0): unit-modulus phases exp(2 pi i u), two
// (FP32) or one (FP64) vectors per 16-byte chunk.  Real (realv = 1): +-1 with the sign
// from the same draw (u < 1/2 -> +1), four (FP32) or two (FP64) vectors per chunk.  Both
// are white noise in the sense of Sec. 2c; vacant orbitals get 0.  r0_in (caller vectors,
// complex interleaved) replaces the draws; real batches take its real parts.
template <typename Real, int SORB, int C>
__global__ void k_init_r0(int64_t ncell, const Real* __restrict__ vt, int vec_base, int nvec,
                          uint32_t phase_base, uint32_t k0, uint32_t k1,
                          const double* __restrict__ r0_in, int64_t N, void* __restrict__ r0,
                          int realv = 0) {
  using Ch = Chunk<Real>;
  const int64_t nchunk = ncell * SORB * C;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunk;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % C);
    const int64_t o = q / C;  // orbital index = cell*SORB + s
    const bool vacant = isnan((double)vt[o]);
    Ch out;
    if (realv) {
#pragma unroll
      for (int k = 0; k < Ch::kReals; ++k) {
        const int v = c * Ch::kReals + k;
        double x = 0.0;
        if (v < nvec && !vacant) {
          if (r0_in) {
            x = r0_in[2 * ((int64_t)(vec_base + v) * N + o)];
          } else {
            const Philox4 w = philox4x32_10((uint32_t)o, (uint32_t)((uint64_t)o >> 32),
                                            phase_base + (uint32_t)(vec_base + v), kTagPhase, k0, k1);
            x = u53(w) < 0.5 ? 1.0 : -1.0;
          }
        }
        out.v[k] = (Real)x;
      }
      out.st(r0, q);
      continue;
    }
#pragma unroll
    for (int k = 0; k < Ch::kVecs; ++k) {
      const int v = c * Ch::kVecs + k;  // lane within the batch
      double re = 0.0, im = 0.0;
      if (v < nvec && !vacant) {
        if (r0_in) {
          const double* z = r0_in + 2 * ((int64_t)(vec_base + v) * N + o);
          re = z[0];
          im = z[1];
        } else {
          const Philox4 x = philox4x32_10((uint32_t)o, (uint32_t)((uint64_t)o >> 32),
                                          phase_base + (uint32_t)(vec_base + v), kTagPhase,
                                          k0, k1);
          const double phi = __dmul_rn(6.283185307179586, u53(x));
          sincos(phi, &im, &re);
        }
      }
      out.v[2 * k] = (Real)re;
      out.v[2 * k + 1] = (Real)im;
    }
    out.st(r0, q);
  }
}

// ------------------------------------------------------------------------------------
// One recursion step fused with the moment dot product.
//
// Work unit = one row segment of TX cells (TX*threads-per-cell = 256 threads, one
// 16-byte chunk each).  Each CTA of the persistent grid owns a contiguous range of
// units ordered strip-major, so it marches down the rows of an x-strip; each row of r_n
// is fetched from HBM once per strip (plus one halo row per segment end and one halo
// cell per side) and reused from shared memory by the rows above and below.  Per-site rounding sequence (shared with the oracle's replica):
//   s = (nb1 + nb2) + nb3 [+ nb4];  h = fma(t~, s, V~ * r);
//   first step: out = h;  otherwise out = fma(2, h, -r_prev);  vacancy: out = 0.
// Honeycomb neighbours: A(x,y) <- B(x,y), B(x+1,y-1), B(x,y-1);
//                       B(x,y) <- A(x,y), A(x-1,y+1), A(x,y+1)  (Listing 1 bonds).
// Square neighbours: (x-1,y), (x+1,y), (x,y-1), (x,y+1).
// ------------------------------------------------------------------------------------
// Moment partial of one complex pair: (sr, si) += conj(a) b, as a chain of fused
// multiply-adds (one rounding per product and sum); every kernel that accumulates the
// moments <r_0|r_n> uses it, so the one-step and the two-step sweeps give the same bits.
// The FP64 sweeps, bound by GB300's FP64 pipe, form the real part only: the imaginary
// part of <r|T_n(H~)|r> (and of <r_n|r_n>, <r_n|r_{n+1}>) vanishes for a Hermitian H~, so
// si stays 0 and two of the update's fourteen FP64 operations go.  The FP32 sweeps keep
// it (their ALU work is free under the HBM bound) as a rounding diagnostic.
template <typename Acc, typename Real>
__device__ __forceinline__ void cacc(Acc& sr, Acc& si, Real ar_, Real ai_, Real br_, Real bi_) {
  const Acc ar = ar_, ai = ai_, br = br_, bi = bi_;
  sr = rfma(ar, br, sr);
  sr = rfma(ai, bi, sr);
  if constexpr (sizeof(Real) == 4) {
    si = rfma(ar, bi, si);
    si = rfma(-ai, br, si);
  }
}

template <typename Real>
struct AccT {
  using T = float;
};
template <>
struct AccT<double> {
  using T = double;
};

// Shared-memory ring: kStages slots, each one row segment of the strip.  A slot holds
// r_n of the row with one halo cell on either side (the periodic neighbours x0-1 and
// x0+TX), and for interior rows also r_{n-1} and r_0 of the row.  Computing row y needs
// the slots of rows y-1, y, y+1; the copy of row y+kStages-1 is issued as soon as row
// y-1's slot is free, so ~6 rows (~75 KB per CTA) are always in flight.
constexpr int kStages = 8;  // default ring depth (the autotuner may pick 4)
constexpr int kBarBytes = 128;

template <int LAT, int C, int NST = kStages>
struct StepShape {
  static constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  static constexpr int TPC = SORB * C;              // threads per cell
  static constexpr int TX = kBlock / TPC;           // cells per row segment
  static constexpr int CELLB = SORB * C * 16;       // bytes of one cell of the batch
  static constexpr int ROWB = TX * CELLB;           // bytes of one row segment (4096)
  static constexpr int CURB = (TX + 2) * CELLB;     // r_n row segment with halo cells
  static constexpr int STAGEB = CURB + 2 * ROWB;    // + r_{n-1} and r_0
  static constexpr int SMEM = kBarBytes + NST * STAGEB;
  // modes that never stage r_0 (families, moment doubling) use shorter stages: a third
  // CTA fits on each SM
  static constexpr int STAGEB_NR0 = CURB + ROWB;
  static constexpr int SMEM_NR0 = kBarBytes + NST * STAGEB_NR0;
  template <int MODE>
  static constexpr int stage_bytes() { return MODE == 0 ? STAGEB : STAGEB_NR0; }
  template <int MODE>
  static constexpr int smem_bytes() { return MODE == 0 ? SMEM : SMEM_NR0; }
};

// Vector-family outputs of a step (2D moments, Sec. 2b): per vector of the batch, rows of
// Kp bf16 values (hi = bf16(x), lo = bf16(x - hi)) holding interleaved (re, im) per
// orbital, stored K-blocked (fam_index).  MODE 1 writes the step's output r_{n+1} as row `col` of the A family;
// MODE 2 writes h~x r_n, built from the neighbours already staged for the step, as
// rows `col` (b) and `col + M` (-i b) of the extended B family.  MODE 3 (moment doubling)
// accumulates <r_n|r_{n+1}> and <r_n|r_n> instead of <r_0|r_{n+1}>; r_0 is not staged.
constexpr int kMaxFamVecs = 2;

// Chebyshev-series accumulation of MODE 4 (time evolution, the wave-packet section):
// acc += (cr + i ci) * r_{n+1}, acc in the batch layout of the iterates.
struct SeriesOut {
  void* acc;
  double cr, ci;
};
struct FamOut {
  __nv_bfloat16* hi[kMaxFamVecs];
  __nv_bfloat16* lo[kMaxFamVecs];
  int64_t Kp;
  int rows;    // rows of the family array (M for A, 2M for the extended B)
  int col;
  int M;
  int dir;     // velocity direction of MODE 2: 0 = x, 1 = y
  float tvel;  // t~ times the bond-offset unit of `dir`: honeycomb x t~/2, y t~ a_cc/2
               // (a_cc = 1/sqrt(3)); square t~
};

__device__ __forceinline__ void fam_store(const FamOut& f, int v, int row, int64_t o, float re,
                                          float im) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(re), h1 = __float2bfloat16_rn(im);
  const __nv_bfloat16 l0 = __float2bfloat16_rn(re - __bfloat162float(h0));
  const __nv_bfloat16 l1 = __float2bfloat16_rn(im - __bfloat162float(h1));
  const int64_t idx = fam_index(row, 2 * o, f.rows);
  *reinterpret_cast<__nv_bfloat162*>(f.hi[v] + idx) = __halves2bfloat162(h0, h1);
  *reinterpret_cast<__nv_bfloat162*>(f.lo[v] + idx) = __halves2bfloat162(l0, l1);
}

// Fixed-order CTA sums of per-thread FP64 partials, per 16-byte chunk c = tid % C of the
// kBlock compute threads: a butterfly over the lanes of each warp that hold the same
// chunk (offsets 16 .. C; both partners form the same sum, so every lane agrees), then
// the kBlock/32 warp sums added in warp order.  Threads tid < C*QT write
// out[c*QT + k].  Every thread of the CTA calls it (it synchronises once); `in_warp` is
// false for whole warps that hold no partials.  `red` is free shared scratch of
// (kBlock/32)*C*QT doubles.  The short dependency chain (log2(32/C) + kBlock/32 adds
// instead of kBlock/C) matters for small systems, where a launch covers one row per CTA.
template <int QT, int C>
__device__ __forceinline__ void cta_lane_sums(const double (&d)[QT], bool in_warp, double* red, double* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (in_warp) {
    double v[QT];
#pragma unroll
    for (int k = 0; k < QT; ++k) v[k] = d[k];
#pragma unroll
    for (int off = 16; off >= C; off >>= 1)
#pragma unroll
      for (int k = 0; k < QT; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane < C)
#pragma unroll
      for (int k = 0; k < QT; ++k) red[(warp * C + lane) * QT + k] = v[k];
  }
  __syncthreads();
  if (tid < C * QT) {
    const int cc = tid / QT, k = tid - (tid / QT) * QT;
    double sum = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) sum += red[(w * C + cc) * QT + k];
    out[tid] = sum;
  }
}

// CTA reduction of the per-thread moment partials (the ring is drained, so its memory is
// reused): lane (vector v = c*VPC + q, component) of `partial` for this CTA.
template <int QT, int C, typename Acc>
__device__ __forceinline__ void moment_partials(double (&dacc)[QT], Acc (&facc)[QT],
                                                double (&dacc0)[QT], Acc (&facc0)[QT], bool first,
                                                unsigned char* stages, double* partial,
                                                double* partial0, int cta) {
#pragma unroll
  for (int k = 0; k < QT; ++k) {
    dacc[k] += (double)facc[k];
    if (first) dacc0[k] += (double)facc0[k];
  }
  double* red = reinterpret_cast<double*>(stages);
  constexpr int Q = C * QT;
  cta_lane_sums<QT, C>(dacc, true, red, partial + (size_t)cta * Q);
  if (first) {
    __syncthreads();
    cta_lane_sums<QT, C>(dacc0, true, red, partial0 + (size_t)cta * Q);
  }
}


// Open boundaries (the configuration's boundaries flag set to False): a bond whose cell
// offset leaves the lattice along an open direction is absent.  The kernels stage the
// neighbour cells and rows across such a boundary from `zero` (a device buffer of zeros
// at least one row long, Lx * cells bytes) instead of the wrapped ones, so the stencil
// and the velocity see a zero neighbour.
struct Open {
  const unsigned char* zero = nullptr;
  int x = 0, y = 0;
};

// Work units are row segments of one x-strip, TX cells wide.  They are numbered in band
// order: the rows are cut into bands of B rows, with B the rows per CTA, and within a
// band the units run strip by strip.  A CTA's contiguous share of the units then covers
// about one band of one strip, so neighbouring CTAs walk the same rows of neighbouring
// strips at the same time, and the halo cells a CTA copies from its neighbours' strips
// are read from L2 by whichever of the two comes second.  unit_segment gives the strip,
// first row and row count of the segment that starts at unit u, cut at unit u1.
struct Seg {
  int sx, yb, nr;
};
// Band order pays off for long shares (measured on GB300 with 456 CTAs: 647 and 1150 rows
// per CTA, 1-3 % faster per pass); for shares of up to ~300 rows the plain strip-major
// order (bands of Ly rows) was 2-6 % faster, so band order starts at 512 rows per CTA.
#ifndef KITE_BAND_MIN_ROWS
#define KITE_BAND_MIN_ROWS 512
#endif
__device__ __forceinline__ int band_rows(long long units, int ncta, int Ly) {
  const long long per = max(1LL, (units + ncta - 1) / ncta);
  if (per < KITE_BAND_MIN_ROWS) return Ly;  // short shares: strip-major order
  return (int)min((long long)Ly, per);
}
__device__ __forceinline__ Seg unit_segment(long long u, long long u1, int Ly, long long nstrips, int B) {
  const long long band_units = nstrips * B;
  const int b = (int)(u / band_units);
  const long long w = u - (long long)b * band_units;
  const int y0 = b * B;
  const int bh = min(B, Ly - y0);
  Seg g;
  g.sx = (int)(w / bh);
  const int r = (int)(w - (long long)g.sx * bh);
  g.yb = y0 + r;
  g.nr = (int)min(u1 - u, (long long)(bh - r));
  return g;
}

// Per-CTA state of the shared-memory ring; a persistent launch keeps it across steps.
struct Ring {
  uint64_t* bars;
  unsigned char* stages;
  int* abort;        // shared flag: a bounded wait gave up
  long long gslot;   // slots consumed so far (phase bookkeeping of the ring)
};

// One recursion step over this CTA's share [cta/ncta] of the units.  Returns false if a
// bounded wait gave up (the CTA has drained its copies and set *err; stop using the ring).
// FIELD: Peierls phases of a perpendicular magnetic field (complex vectors only).  phase
// holds, per row y and sublattice s, (cos, sin) of the two bonds with an x component,
// [y][s][bond][2]: honeycomb bonds n2, n3, square bonds n1, n2 in the order of the
// neighbour loads below; the neighbour value is rotated before the sum.
template <typename Real, int LAT, int C, bool FIRST, int MODE, int NST = kStages, bool FIELD = false>
__device__ __forceinline__ bool step_body(Ring& ring, int cta, int ncta, const void* r_prev,
                                          const void* __restrict__ r_cur, void* r_out,
                                          const void* __restrict__ r0, const Real* __restrict__ vt,
                                          Real tt, int Lx, int Ly, long long units,
                                          double* __restrict__ partial, double* __restrict__ partial0,
                                          int* __restrict__ err, int stall, const FamOut& fam,
                                          int realv = 0, const SeriesOut& ser = SeriesOut{},
                                          const Real* __restrict__ phase = nullptr,
                                          const Open& open = Open{}) {
  static_assert(MODE == 0 || MODE == 3 || MODE == 4 || (sizeof(Real) == 4 && C * 2 <= kMaxFamVecs),
                "family modes run on FP32 batches of at most two vectors");
  using Ch = Chunk<Real>;
  using Acc = typename AccT<Real>::T;
  using Sh = StepShape<LAT, C, NST>;
  constexpr int VPC = Ch::kVecs, NR = Ch::kReals;
  constexpr int SORB = Sh::SORB, TPC = Sh::TPC, TX = Sh::TX, CELLB = Sh::CELLB;
  const Real tt2 = tt + tt;  // exact
  constexpr int STG = Sh::template stage_bytes<MODE>();
  constexpr int QT = 2 * VPC;  // (re, im) per complex vector, or one value per real vector
  uint64_t* bars = ring.bars;
  unsigned char* stages = ring.stages;
  int& s_abort = *ring.abort;

  const int tid = threadIdx.x;
  const int xl = tid / TPC;
  const int j = tid - xl * TPC;
  const int s = j / C;
  const int c = j - s * C;
  const int choff = (s * C + c) * 16;             // this thread's chunk inside a cell
  const int nboff = ((1 - s) * C + c) * 16;       // same chunk, other sublattice

  __syncthreads();  // the ring (and its reuse for the previous step's reduction) is free

  const long long u0 = units * (long long)cta / ncta;
  const long long u1 = units * (long long)(cta + 1) / ncta;

  double dacc[QT], dacc0[QT];
  Acc facc[QT], facc0[QT];
#pragma unroll
  for (int k = 0; k < QT; ++k) dacc[k] = dacc0[k] = 0.0, facc[k] = facc0[k] = Acc(0);
  int rows = 0;
  long long gslot = ring.gslot;
  bool aborted = false;

  const int band = band_rows(units, ncta, Ly);
  const long long nstrips = units / Ly;
  for (long long u = u0; u < u1 && !aborted;) {
    // one segment = consecutive rows of one x-strip
    const Seg seg = unit_segment(u, u1, Ly, nstrips, band);
    const int sx = seg.sx, yb = seg.yb, nr = seg.nr;
    const int x0 = sx * TX;
    const int txv = min(TX, Lx - x0);
    const int xlh = (x0 == 0) ? Lx - 1 : x0 - 1;
    const int xrh = (x0 + txv == Lx) ? 0 : x0 + txv;
    const int nslots = nr + 2;

    auto issue = [&](int jj) {  // producer: thread 0 only
      const long long g = gslot + jj;
      const int st = (int)(g % NST);
      unsigned char* base = stages + st * STG;
      int row = yb - 1 + jj;
      const bool wrapped = row < 0 || row >= Ly;
      row = row < 0 ? row + Ly : (row >= Ly ? row - Ly : row);
      const bool interior = !FIRST && jj >= 1 && jj <= nr;
      const uint32_t main_b = (uint32_t)txv * CELLB;
      // r_0 is only staged when moments are accumulated (MODE 0)
      uint32_t bytes = main_b + 2 * CELLB + (interior ? (MODE == 0 ? 2 : 1) * main_b : 0);
      if (stall && cta == 0 && g == 0) bytes += 16;  // test hook: never completes
      mbar_arrive_expect_tx(&bars[st], bytes);
      // a row or halo cell across an open boundary comes from the zero buffer
      const unsigned char* rowp = (open.y && wrapped)
                                      ? open.zero
                                      : static_cast<const unsigned char*>(r_cur) + (size_t)row * Lx * CELLB;
      bulk_g2s(base + CELLB, rowp + (size_t)x0 * CELLB, main_b, &bars[st]);
      bulk_g2s(base, (open.x && x0 == 0) ? open.zero : rowp + (size_t)xlh * CELLB, CELLB, &bars[st]);
      bulk_g2s(base + (size_t)(txv + 1) * CELLB,
               (open.x && x0 + txv == Lx) ? open.zero : rowp + (size_t)xrh * CELLB, CELLB, &bars[st]);
      if (interior) {
        const size_t off = ((size_t)row * Lx + x0) * CELLB;
        bulk_g2s(base + Sh::CURB, static_cast<const unsigned char*>(r_prev) + off, main_b, &bars[st]);
        if (MODE == 0)
          bulk_g2s(base + Sh::CURB + Sh::ROWB, static_cast<const unsigned char*>(r0) + off, main_b,
                   &bars[st]);
      }
    };
    if (tid == 0)
      for (int jj = 0; jj < min(NST, nslots); ++jj) issue(jj);

    const bool active = xl < txv;
    Real vnext = active ? vt[((size_t)yb * Lx + x0 + xl) * SORB + s] : Real(0);
    int i = 0;
    for (; i < nr; ++i) {
      bool ok = true;
      for (int jj = (i == 0 ? 0 : i + 2); jj <= i + 2; ++jj) {
        const long long g = gslot + jj;
        ok = mbar_wait_bounded(&bars[g % NST], (uint32_t)((g / NST) & 1)) && ok;
      }
      if (!ok) s_abort = 1;
      const int y = yb + i;
      const Real v = vnext;
      if (active && i + 1 < nr) vnext = vt[((size_t)(y + 1) * Lx + x0 + xl) * SORB + s];
      Real pc0 = Real(1), ps0 = Real(0), pc1 = Real(1), ps1 = Real(0);
      if constexpr (FIELD) {
        const Real* p4 = phase + ((size_t)y * SORB + s) * 4;
        pc0 = __ldg(p4);
        ps0 = __ldg(p4 + 1);
        pc1 = __ldg(p4 + 2);
        ps1 = __ldg(p4 + 3);
      }
      if (ok && active) {
        const unsigned char* up = stages + (int)((gslot + i) % NST) * STG;
        const unsigned char* mid = stages + (int)((gslot + i + 1) % NST) * STG;
        const unsigned char* dn = stages + (int)((gslot + i + 2) % NST) * STG;
        const Ch me = *reinterpret_cast<const Ch*>(mid + (xl + 1) * CELLB + choff);
        Ch n1, n2, n3, n4;
        if (LAT == KITE_HONEYCOMB) {
          // A(x,y) <- B(x,y), B(x+1,y-1), B(x,y-1);  B(x,y) <- A(x,y), A(x-1,y+1), A(x,y+1)
          const unsigned char* other = s == 0 ? up : dn;
          const int dxi = s == 0 ? xl + 2 : xl;
          n1 = *reinterpret_cast<const Ch*>(mid + (xl + 1) * CELLB + nboff);
          n2 = *reinterpret_cast<const Ch*>(other + dxi * CELLB + nboff);
          n3 = *reinterpret_cast<const Ch*>(other + (xl + 1) * CELLB + nboff);
        } else {
          n1 = *reinterpret_cast<const Ch*>(mid + xl * CELLB + choff);
          n2 = *reinterpret_cast<const Ch*>(mid + (xl + 2) * CELLB + choff);
          n3 = *reinterpret_cast<const Ch*>(up + (xl + 1) * CELLB + choff);
          n4 = *reinterpret_cast<const Ch*>(dn + (xl + 1) * CELLB + choff);
        }
        if constexpr (FIELD) {
          // t exp(i theta) r_j: rotate the neighbours across bonds with an x component
          auto rot = [&](Ch& n, Real cph, Real sph) {
#pragma unroll
            for (int q = 0; q < VPC; ++q) {
              const Real re = n.v[2 * q], im = n.v[2 * q + 1];
              n.v[2 * q] = rfma(cph, re, -rmul(sph, im));
              n.v[2 * q + 1] = rfma(sph, re, rmul(cph, im));
            }
          };
          if (LAT == KITE_HONEYCOMB) {
            rot(n2, pc0, ps0);
            rot(n3, pc1, ps1);
          } else {
            rot(n1, pc0, ps0);
            rot(n2, pc1, ps1);
          }
        }
        Ch pv, z0;
        if (FIRST) {
          z0 = me;
        } else {
          pv = *reinterpret_cast<const Ch*>(mid + Sh::CURB + xl * CELLB + choff);
          if (MODE == 0)
            z0 = *reinterpret_cast<const Ch*>(mid + Sh::CURB + Sh::ROWB + xl * CELLB + choff);
        }
        const bool vacant = is_vacancy(v);
        Ch out;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          Real sum = radd(n1.v[k], n2.v[k]);
          sum = radd(sum, n3.v[k]);
          if (LAT == KITE_SQUARE) sum = radd(sum, n4.v[k]);
          // r_1 = t~ s + V~ r_0; r_{n+1} = 2t~ s + (2V~ r_n - r_{n-1}) (v holds 2V~)
          const Real o = FIRST ? rfma(tt, sum, rmul(Real(0.5) * v, me.v[k]))
                               : rfma(tt2, sum, rfma(v, me.v[k], -pv.v[k]));
          out.v[k] = vacant ? Real(0) : o;
        }
        out.st(r_out, (((size_t)y * Lx + x0 + xl) * SORB + s) * C + c);
        if constexpr (MODE == 4) {
          const size_t qi = (((size_t)y * Lx + x0 + xl) * SORB + s) * C + c;
          Ch a = Ch::ldg(ser.acc, qi);
          const Real cr = (Real)ser.cr, ci = (Real)ser.ci;
#pragma unroll
          for (int q = 0; q < VPC; ++q) {
            const Real br = out.v[2 * q], bi = out.v[2 * q + 1];
            a.v[2 * q] += cr * br - ci * bi;
            a.v[2 * q + 1] += cr * bi + ci * br;
          }
          a.st(ser.acc, qi);
        } else if constexpr (MODE == 3) {
          // moment doubling: <r_n|r_{n+1}> into facc, <r_n|r_n> into facc0
          if (realv) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const Acc a = me.v[k], b = out.v[k];
              facc[k] += a * b;
              facc0[k] += a * a;
            }
          } else {
#pragma unroll
            for (int q = 0; q < VPC; ++q) {
              cacc(facc[2 * q], facc[2 * q + 1], me.v[2 * q], me.v[2 * q + 1], out.v[2 * q], out.v[2 * q + 1]);
              const Acc ar = me.v[2 * q], ai = me.v[2 * q + 1];
              facc0[2 * q] = rfma(ai, ai, rfma(ar, ar, facc0[2 * q]));
            }
          }
          if (++rows == kFlushRows) {
            rows = 0;
#pragma unroll
            for (int k = 0; k < QT; ++k) {
              dacc[k] += (double)facc[k];
              dacc0[k] += (double)facc0[k];
              facc[k] = facc0[k] = Acc(0);
            }
          }
        } else if constexpr (MODE != 0) {
          const int64_t o = ((int64_t)y * Lx + x0 + xl) * SORB + s;
#pragma unroll
          for (int q = 0; q < VPC; ++q) {
            const int vv = c * VPC + q;
            if constexpr (MODE == 1) {
              fam_store(fam, vv, fam.col, o, out.v[2 * q], out.v[2 * q + 1]);
            } else {
              // h~ r at this orbital, h~ = [r_dir, H~]: honeycomb bond offsets (x, y) of the
              // neighbours n1, n2, n3 are (0, -a_cc), (-a/2, a_cc/2), (a/2, a_cc/2) on A
              // and the negatives on B; square (x-1), (x+1), (y-1), (y+1) have x offsets
              // +1, -1 and y offsets +1, -1 for n1, n2 and n3, n4
              float vr, vi;
              if (LAT == KITE_HONEYCOMB) {
                const float sg = s == 0 ? fam.tvel : -fam.tvel;
                if (fam.dir == 0) {
                  vr = sg * (n3.v[2 * q] - n2.v[2 * q]);
                  vi = sg * (n3.v[2 * q + 1] - n2.v[2 * q + 1]);
                } else {
                  vr = sg * ((n2.v[2 * q] + n3.v[2 * q]) - 2.f * n1.v[2 * q]);
                  vi = sg * ((n2.v[2 * q + 1] + n3.v[2 * q + 1]) - 2.f * n1.v[2 * q + 1]);
                }
              } else if (fam.dir == 0) {
                vr = fam.tvel * (n1.v[2 * q] - n2.v[2 * q]);
                vi = fam.tvel * (n1.v[2 * q + 1] - n2.v[2 * q + 1]);
              } else {
                vr = fam.tvel * (n3.v[2 * q] - n4.v[2 * q]);
                vi = fam.tvel * (n3.v[2 * q + 1] - n4.v[2 * q + 1]);
              }
              if (vacant) vr = vi = 0.f;
              fam_store(fam, vv, fam.col, o, vr, vi);
              fam_store(fam, vv, fam.col + fam.M, o, vi, -vr);
            }
          }
        } else {  // MODE 0: fused moment <r_0|r_{n+1}> (and <r_0|r_0> on the first step)
          if (realv) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const Acc a = z0.v[k], b = out.v[k];
              facc[k] += a * b;
              if (FIRST) facc0[k] += a * a;
            }
          } else {
#pragma unroll
            for (int q = 0; q < VPC; ++q) {
              cacc(facc[2 * q], facc[2 * q + 1], z0.v[2 * q], z0.v[2 * q + 1], out.v[2 * q], out.v[2 * q + 1]);
              if (FIRST) {
                const Acc ar = z0.v[2 * q], ai = z0.v[2 * q + 1];
                facc0[2 * q] = rfma(ai, ai, rfma(ar, ar, facc0[2 * q]));
              }
            }
          }
          if (++rows == kFlushRows) {
            rows = 0;
#pragma unroll
            for (int k = 0; k < QT; ++k) {
              dacc[k] += (double)facc[k];
              facc[k] = Acc(0);
              if (FIRST) dacc0[k] += (double)facc0[k], facc0[k] = Acc(0);
            }
          }
        }
      }
      __syncthreads();  // every thread is done with slot i
      if (s_abort) {
        aborted = true;
        break;
      }
      if (tid == 0 && i + NST < nslots) issue(i + NST);
    }
    if (aborted) {
      // drain: wait (bounded) for this CTA's copies still in flight, then give up
      if (tid == 0) {
        const int last = min(nslots, i + NST) - 1;
        for (int jj = i; jj <= last; ++jj) {  // completed phases return at once
          const long long g = gslot + jj;
          mbar_wait_bounded(&bars[g % NST], (uint32_t)((g / NST) & 1));
        }
        atomicExch(err, 1);
      }
      ring.gslot = gslot;
      return false;
    }
    gslot += nslots;
    u += nr;
  }
  ring.gslot = gslot;
  if constexpr (MODE == 0)
    moment_partials<QT, C>(dacc, facc, dacc0, facc0, FIRST, stages, partial, partial0, cta);
  if constexpr (MODE == 3)
    moment_partials<QT, C>(dacc, facc, dacc0, facc0, true, stages, partial, partial0, cta);
  return true;
}

template <typename Real, int LAT, int C, bool FIRST, int MODE = 0, int NST = kStages, bool FIELD = false>
__global__ void __launch_bounds__(kBlock, 2)
    k_step(const void* r_prev, const void* __restrict__ r_cur, void* r_out,
           const void* __restrict__ r0, const Real* __restrict__ vt, Real tt, int Lx, int Ly,
           long long units, double* __restrict__ partial, double* __restrict__ partial0,
           int* __restrict__ err, int stall, const FamOut fam, int realv = 0,
           const SeriesOut ser = SeriesOut{}, const void* phase = nullptr, const Open open = Open{}) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  Ring ring{bars, smem + kBarBytes, &s_abort, 0};
  griddep_wait();  // the previous step's iterates and partials are complete
  griddep_launch_dependents();
  step_body<Real, LAT, C, FIRST, MODE, NST, FIELD>(ring, blockIdx.x, gridDim.x, r_prev, r_cur, r_out, r0,
                                                   vt, tt, Lx, Ly, units, partial, partial0, err, stall,
                                                   fam, realv, ser, static_cast<const Real*>(phase), open);
}

// Launch with programmatic stream serialisation: the kernel's set-up overlaps the end of
// its predecessor on the stream (the step kernels call griddep_wait before any memory
// access).  Arguments are converted to the kernel's parameter types.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Copies one iterate buffer (batch layout) into the caller layout [vec][slot][N].
template <typename Real, int SORB, int C>
__global__ void k_extract(int64_t ncell, const void* __restrict__ buf, int nvec, int vec_base,
                          int slot, int64_t N, Real* __restrict__ dst) {
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
      Real* d = dst + 2 * (((int64_t)(vec_base + v) * 2 + slot) * N + o);
      d[0] = z.v[2 * k];
      d[1] = z.v[2 * k + 1];
    }
  }
}


// Resident CTAs per SM of the step kernel of a mode and ring depth (also sets the
// kernels' dynamic shared-memory limit).
template <typename Real, int LAT, int C, int MODE = 0, int NST = kStages, bool FIELD = false>
int step_occupancy() {
  static int occ = -1;  // per template instance; device-independent enough for one GPU type
  if (occ < 0) {
    int o = 0;
    const int smem = StepShape<LAT, C, NST>::template smem_bytes<MODE>();
    cudaFuncSetAttribute(k_step<Real, LAT, C, true, MODE, NST, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    cudaFuncSetAttribute(k_step<Real, LAT, C, false, MODE, NST, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_step<Real, LAT, C, false, MODE, NST, FIELD>, kBlock,
                                                      smem) != cudaSuccess ||
        o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}

// Persistent grid of the step kernel: min(ctas_per_sm, occupancy) CTAs per SM (0 = the
// occupancy), at most one CTA per unit.
template <typename Real, int LAT, int C, bool FIRST, int MODE = 0, int NST = kStages, bool FIELD = false>
int grid_for(kite_ctx* ctx, long long units, int ctas_per_sm = 0) {
  const int occ = step_occupancy<Real, LAT, C, MODE, NST, FIELD>();
  const int k = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  long long g = (long long)ctx->num_sms * k;
  return (int)std::max(1LL, std::min(g, units));
}


}  // namespace
}  // namespace kite
