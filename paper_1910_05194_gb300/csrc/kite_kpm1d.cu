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

#include <algorithm>
#include <vector>

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
template <typename Real>
__global__ void k_onsite(int64_t N, int lattice, double W, double half_delta, double de_plus,
                         double de_minus, uint64_t vac_thr, uint32_t realisation, uint32_t k0,
                         uint32_t k1, Real* __restrict__ vt,
                         unsigned long long* __restrict__ n_eff) {
  unsigned int count = 0;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < N;
       o += (int64_t)gridDim.x * blockDim.x) {
    const Philox4 x = philox4x32_10((uint32_t)o, (uint32_t)((uint64_t)o >> 32), realisation,
                                    kTagDisorder, k0, k1);
    double v = __dmul_rn(W, __dsub_rn(u53(x), 0.5));
    if (lattice == KITE_HONEYCOMB && half_delta != 0.0)
      v = __dadd_rn(v, (o & 1) == 0 ? half_delta : -half_delta);
    const bool vacant = (uint64_t)x.w[2] < vac_thr;
    const double vtil = __ddiv_rn(__dsub_rn(v, de_plus), de_minus);
    vt[o] = vacant ? quiet_nan<Real>() : (Real)vtil;
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
template <typename Real, int SORB, int C>
__global__ void k_init_r0(int64_t ncell, const Real* __restrict__ vt, int vec_base, int nvec,
                          uint32_t phase_base, uint32_t k0, uint32_t k1,
                          const double* __restrict__ r0_in, int64_t N, void* __restrict__ r0) {
  using Ch = Chunk<Real>;
  const int64_t nchunk = ncell * SORB * C;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunk;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % C);
    const int64_t o = q / C;  // orbital index = cell*SORB + s
    const bool vacant = isnan((double)vt[o]);
    Ch out;
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
constexpr int kStages = 8;
constexpr int kBarBytes = 128;

template <int LAT, int C>
struct StepShape {
  static constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  static constexpr int TPC = SORB * C;              // threads per cell
  static constexpr int TX = kBlock / TPC;           // cells per row segment
  static constexpr int CELLB = SORB * C * 16;       // bytes of one cell of the batch
  static constexpr int ROWB = TX * CELLB;           // bytes of one row segment (4096)
  static constexpr int CURB = (TX + 2) * CELLB;     // r_n row segment with halo cells
  static constexpr int STAGEB = CURB + 2 * ROWB;    // + r_{n-1} and r_0
  static constexpr int SMEM = kBarBytes + kStages * STAGEB;
};

template <typename Real, int LAT, int C, bool FIRST>
__global__ void __launch_bounds__(kBlock, 2)
    k_step(const void* r_prev, const void* __restrict__ r_cur, void* r_out,
           const void* __restrict__ r0, const Real* __restrict__ vt, Real tt, int Lx, int Ly,
           long long units, double* __restrict__ partial, double* __restrict__ partial0,
           int* __restrict__ err, int stall) {
  using Ch = Chunk<Real>;
  using Acc = typename AccT<Real>::T;
  using Sh = StepShape<LAT, C>;
  constexpr int VPC = Ch::kVecs, NR = Ch::kReals;
  constexpr int SORB = Sh::SORB, TPC = Sh::TPC, TX = Sh::TX, CELLB = Sh::CELLB;
  constexpr int QT = 2 * VPC;  // (re, im) per vector held by one thread
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + kBarBytes;
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int xl = tid / TPC;
  const int j = tid - xl * TPC;
  const int s = j / C;
  const int c = j - s * C;
  const int choff = (s * C + c) * 16;             // this thread's chunk inside a cell
  const int nboff = ((1 - s) * C + c) * 16;       // same chunk, other sublattice

  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();

  const long long u0 = units * (long long)blockIdx.x / gridDim.x;
  const long long u1 = units * (long long)(blockIdx.x + 1) / gridDim.x;

  double dacc[QT], dacc0[QT];
  Acc facc[QT], facc0[QT];
#pragma unroll
  for (int k = 0; k < QT; ++k) dacc[k] = dacc0[k] = 0.0, facc[k] = facc0[k] = Acc(0);
  int rows = 0;
  long long gslot = 0;  // slots consumed so far (phase bookkeeping of the ring)
  bool aborted = false;

  for (long long u = u0; u < u1 && !aborted;) {
    // one segment = consecutive rows of one x-strip
    const int sx = (int)(u / Ly);
    const int yb = (int)(u - (long long)sx * Ly);
    const int nr = (int)min(u1 - u, (long long)(Ly - yb));
    const int x0 = sx * TX;
    const int txv = min(TX, Lx - x0);
    const int xlh = (x0 == 0) ? Lx - 1 : x0 - 1;
    const int xrh = (x0 + txv == Lx) ? 0 : x0 + txv;
    const int nslots = nr + 2;

    auto issue = [&](int jj) {  // producer: thread 0 only
      const long long g = gslot + jj;
      const int st = (int)(g % kStages);
      unsigned char* base = stages + st * Sh::STAGEB;
      int row = yb - 1 + jj;
      row = row < 0 ? row + Ly : (row >= Ly ? row - Ly : row);
      const bool interior = !FIRST && jj >= 1 && jj <= nr;
      const uint32_t main_b = (uint32_t)txv * CELLB;
      uint32_t bytes = main_b + 2 * CELLB + (interior ? 2 * main_b : 0);
      if (stall && blockIdx.x == 0 && g == 0) bytes += 16;  // test hook: never completes
      mbar_arrive_expect_tx(&bars[st], bytes);
      const unsigned char* rowp = static_cast<const unsigned char*>(r_cur) + (size_t)row * Lx * CELLB;
      bulk_g2s(base + CELLB, rowp + (size_t)x0 * CELLB, main_b, &bars[st]);
      bulk_g2s(base, rowp + (size_t)xlh * CELLB, CELLB, &bars[st]);
      bulk_g2s(base + (size_t)(txv + 1) * CELLB, rowp + (size_t)xrh * CELLB, CELLB, &bars[st]);
      if (interior) {
        const size_t off = ((size_t)row * Lx + x0) * CELLB;
        bulk_g2s(base + Sh::CURB, static_cast<const unsigned char*>(r_prev) + off, main_b, &bars[st]);
        bulk_g2s(base + Sh::CURB + Sh::ROWB, static_cast<const unsigned char*>(r0) + off, main_b,
                 &bars[st]);
      }
    };
    if (tid == 0)
      for (int jj = 0; jj < min(kStages, nslots); ++jj) issue(jj);

    const bool active = xl < txv;
    Real vnext = active ? vt[((size_t)yb * Lx + x0 + xl) * SORB + s] : Real(0);
    int i = 0;
    for (; i < nr; ++i) {
      bool ok = true;
      for (int jj = (i == 0 ? 0 : i + 2); jj <= i + 2; ++jj) {
        const long long g = gslot + jj;
        ok = mbar_wait_bounded(&bars[g % kStages], (uint32_t)((g / kStages) & 1)) && ok;
      }
      if (!ok) s_abort = 1;
      const int y = yb + i;
      const Real v = vnext;
      if (active && i + 1 < nr) vnext = vt[((size_t)(y + 1) * Lx + x0 + xl) * SORB + s];
      if (ok && active) {
        const unsigned char* up = stages + (int)((gslot + i) % kStages) * Sh::STAGEB;
        const unsigned char* mid = stages + (int)((gslot + i + 1) % kStages) * Sh::STAGEB;
        const unsigned char* dn = stages + (int)((gslot + i + 2) % kStages) * Sh::STAGEB;
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
        Ch pv, z0;
        if (FIRST) {
          z0 = me;
        } else {
          pv = *reinterpret_cast<const Ch*>(mid + Sh::CURB + xl * CELLB + choff);
          z0 = *reinterpret_cast<const Ch*>(mid + Sh::CURB + Sh::ROWB + xl * CELLB + choff);
        }
        const bool vacant = v != v;
        Ch out;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          Real sum = radd(n1.v[k], n2.v[k]);
          sum = radd(sum, n3.v[k]);
          if (LAT == KITE_SQUARE) sum = radd(sum, n4.v[k]);
          const Real h = rfma(tt, sum, rmul(v, me.v[k]));
          const Real o = FIRST ? h : rfma(Real(2), h, -pv.v[k]);
          out.v[k] = vacant ? Real(0) : o;
        }
        out.st(r_out, (((size_t)y * Lx + x0 + xl) * SORB + s) * C + c);
#pragma unroll
        for (int q = 0; q < VPC; ++q) {
          const Acc ar = z0.v[2 * q], ai = z0.v[2 * q + 1];
          const Acc br = out.v[2 * q], bi = out.v[2 * q + 1];
          facc[2 * q] += ar * br + ai * bi;
          facc[2 * q + 1] += ar * bi - ai * br;
          if (FIRST) facc0[2 * q] += ar * ar + ai * ai;
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
      __syncthreads();  // every thread is done with slot i
      if (s_abort) {
        aborted = true;
        break;
      }
      if (tid == 0 && i + kStages < nslots) issue(i + kStages);
    }
    if (aborted) {
      // drain: wait (bounded) for this CTA's copies still in flight, then give up
      if (tid == 0) {
        const int last = min(nslots, i + kStages) - 1;
        for (int jj = i; jj <= last; ++jj) {  // completed phases return at once
          const long long g = gslot + jj;
          mbar_wait_bounded(&bars[g % kStages], (uint32_t)((g / kStages) & 1));
        }
        atomicExch(err, 1);
      }
      return;
    }
    gslot += nslots;
    u += nr;
  }
#pragma unroll
  for (int k = 0; k < QT; ++k) {
    dacc[k] += (double)facc[k];
    if (FIRST) dacc0[k] += (double)facc0[k];
  }

  // CTA reduction in fixed order (the ring is drained, so its memory is reused):
  // lane (vector v = c*VPC + q, component) sums the threads holding chunk c.
  double(*red)[QT] = reinterpret_cast<double(*)[QT]>(stages);
  constexpr int Q = 2 * C * VPC;
#pragma unroll
  for (int k = 0; k < QT; ++k) red[tid][k] = dacc[k];
  __syncthreads();
  if (tid < Q) {
    const int cc = tid / QT, k = tid - (tid / QT) * QT;
    double sum = 0.0;
    for (int t = cc; t < kBlock; t += C) sum += red[t][k];
    partial[(size_t)blockIdx.x * Q + tid] = sum;
  }
  if (FIRST) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < QT; ++k) red[tid][k] = dacc0[k];
    __syncthreads();
    if (tid < Q) {
      const int cc = tid / QT, k = tid - (tid / QT) * QT;
      double sum = 0.0;
      for (int t = cc; t < kBlock; t += C) sum += red[t][k];
      partial0[(size_t)blockIdx.x * Q + tid] = sum;
    }
  }
}

// Sums the per-CTA partials of every moment in fixed order and normalises by N_eff:
// mu_vec[(vec_base+v)][n] (complex) for the valid lanes v < nvec.
__global__ void k_reduce(const double* __restrict__ partial, int M, int G, int Q, int nvec,
                         int vec_base, const unsigned long long* __restrict__ n_eff,
                         double* __restrict__ mu_vec) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * Q) return;
  const int n = idx / Q, q = idx - (idx / Q) * Q;
  const int v = q >> 1, comp = q & 1;
  if (v >= nvec) return;
  double sum = 0.0;
  const double* p = partial + (size_t)n * G * Q + q;
  for (int g = 0; g < G; ++g) sum += p[(size_t)g * Q];
  const double ne = (double)*n_eff;
  mu_vec[((size_t)(vec_base + v) * M + n) * 2 + comp] = ne > 0.0 ? sum / ne : 0.0;
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
template <typename Real, int LAT, int C, bool FIRST>
int grid_for(kite_ctx* ctx, long long units) {
  static int occ = -1;  // per template instance; device-independent enough for one GPU type
  if (occ < 0) {
    int o = 0;
    const int smem = StepShape<LAT, C>::SMEM;
    cudaFuncSetAttribute(k_step<Real, LAT, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_step<Real, LAT, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_step<Real, LAT, C, FIRST>, kBlock, smem) !=
            cudaSuccess ||
        o < 1)
      o = 1;
    occ = o;
  }
  long long g = (long long)ctx->num_sms * occ;
  return (int)std::max(1LL, std::min(g, units));
}

struct Plan {
  int64_t N, ncell;
  int Lx, Ly, sorb;
  int R, S, M;
  bool fp64;
  int max_batch;  // vectors per pass
};

template <typename Real, int LAT, int C>
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
  constexpr int SM = StepShape<LAT, C>::SMEM;
  if (M >= 2)
    k_step<Real, LAT, C, true><<<G, kBlock, SM, st>>>(nullptr, r0, bA, r0, vt, tt, p.Lx, p.Ly,
                                                      units, partial + (size_t)G * Q, partial,
                                                      ctx->d_status, ctx->debug_stall);
  ctx->debug_stall = 0;
  for (int n = 1; n + 1 < M; ++n)
    k_step<Real, LAT, C, false><<<G, kBlock, SM, st>>>(where(n - 1), where(n), where(n + 1), r0,
                                                       vt, tt, p.Lx, p.Ly, units,
                                                       partial + (size_t)(n + 1) * G * Q, nullptr,
                                                       ctx->d_status, 0);
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  if (M == 1) {
    // mu_0 alone: one FIRST pass would also write r_1; a plain dot is enough, but the
    // FIRST kernel is cheap and keeps one code path.
    k_step<Real, LAT, C, true><<<G, kBlock, SM, st>>>(nullptr, r0, bA, r0, vt, tt, p.Lx, p.Ly,
                                                      units, partial + (size_t)G * Q, partial,
                                                      ctx->d_status, 0);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
  }
  const int total = M * Q;
  k_reduce<<<(total + 255) / 256, 256, 0, st>>>(partial, M, G, Q, nvec, vec_base, n_eff, mu_vec);
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

template <typename Real, int LAT>
int grid_for_c(kite_ctx* ctx, int C, long long units) {
  if (C == 1) return grid_for<Real, LAT, 1, false>(ctx, units);
  if (C == 2) return grid_for<Real, LAT, 2, false>(ctx, units);
  return grid_for<Real, LAT, 4, false>(ctx, units);
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
  p.max_batch = kMaxC * VPC;
  auto chunks_for = [&](int nvec) {
    const int c = (nvec + VPC - 1) / VPC;
    return c <= 1 ? 1 : (c <= 2 ? 2 : 4);
  };
  auto units_for = [&](int C) {
    const int TX = kBlock / (SORB * C);
    return (long long)((sys->Lx + TX - 1) / TX) * sys->Ly;
  };
  const int Cmax = chunks_for(std::min(p.R, p.max_batch));
  const int Ctail = chunks_for(p.R % p.max_batch == 0 ? std::min(p.R, p.max_batch) : p.R % p.max_batch);
  const int Gmax = std::max(grid_for_c<Real, LAT>(ctx, Cmax, units_for(Cmax)),
                            grid_for_c<Real, LAT>(ctx, Ctail, units_for(Ctail)));

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
    *partial = k.take<double>((size_t)std::max(p.M, 2) * Gmax * 2 * Cmax * VPC);
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
      p.ncell, vt, base, nvec, phase_base, k0, k1, r0_in, p.N, r0)
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
    const int G = grid_for<Real, LAT, CC, false>(ctx, u);                                    \
    grid_used = G;                                                                           \
    rc = sweep_batch<Real, LAT, CC>(ctx, p, vt, tt, r0, bA, bB, partial, G, u, nvec,         \
                                    vec_base, ne, mu_vec, &lp, &lc, &step_s, &step_n);       \
  } while (0)
      if (C == 1) KITE_SWEEP(1);
      else if (C == 2) KITE_SWEEP(2);
      else KITE_SWEEP(4);
#undef KITE_SWEEP
      if (rc != KITE_OK) return rc;
      // algorithmic bytes of this batch's step launches: per orbital and step, read
      // r_{n-1}, r_n, r_0 and write r_{n+1} for each of the batch's 16-byte chunks, and
      // read the shared on-site term (the first step has no r_{n-1} and reads r_0 once)
      if (p.M >= 2) {
        const double chunk_bytes = 16.0 * SORB * C * (double)p.ncell;
        step_bytes += (double)(p.M - 2) * (4.0 * chunk_bytes + (double)p.N * sizeof(Real)) +
                      (2.0 * chunk_bytes + (double)p.N * sizeof(Real));
      }
      if (kpm->r_last) {
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
    const double per_orb_step = 4.0 * 2.0 * sizeof(Real) * p.R + (double)sizeof(Real);
    stats->bytes_moved = per_orb_step * (double)p.N * (double)(p.M > 1 ? p.M - 1 : 0) * p.S;
    stats->gbps = stats->seconds > 0 ? stats->bytes_moved / stats->seconds * 1e-9 : 0.0;
    stats->n_eff = n_eff_last;
    stats->grid = grid_used;
    stats->block = kBlock;
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
