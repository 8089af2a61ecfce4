// kite_step3.cuh -- three recursion steps per pass (deeper temporal blocking).
//
// From r_{n-1} and r_n one pass computes r_{n+1}, r_{n+2} and r_{n+3} (Eq. e6) and the
// moments <r_0|r_{n+1}>, <r_0|r_{n+2}>, <r_0|r_{n+3}> (Eqs. e7/e8), but writes only
// r_{n+2} and r_{n+3}: the next pass starts from them, and r_{n+1} never leaves shared
// memory.  Per orbital and pass the HBM traffic is r_{n-1}, r_n, r_0 in and two iterates
// out -- the five streams of the two-step pass, now for three steps.
//
// A CTA walks the rows of its share of a strip.  In iteration i it computes row yb-2+i of
// r_{n+1} from the bulk-copied r_n rows (with three halo cells each side), row yb-4+i of
// r_{n+2} from the r_{n+1} rows kept in a five-row tile ring, and row yb-6+i of r_{n+3}
// from the r_{n+2} rows kept in a four-row tile ring; one barrier per iteration.  r_{n+1}
// is computed on the owned cells and two halo cells each side, r_{n+2} on one halo cell
// each side, r_{n+3} on the owned cells; the halo cells of r_{n+1} and r_{n+2} are computed
// by two extra warps (the last thread of the second one also issues the bulk copies).  The
// r_n ring keeps each row's r_0 until its r_{n+3} row is done (slot i-3).  The site update
// is the one-step kernel's rounding sequence, so the iterates are bit-identical to three
// one-step launches.
#pragma once

#include "kite_step.cuh"

namespace kite {
namespace {

template <int LAT, int C, int NST>
struct Step3Shape {
  using S1 = StepShape<LAT, C, NST>;
  static constexpr int SORB = S1::SORB, TPC = S1::TPC, TX = S1::TX, CELLB = S1::CELLB;
  static constexpr int RNB = (TX + 6) * CELLB;  // r_n row, three halo cells each side
  static constexpr int R0B = TX * CELLB;        // r_0 row
  static constexpr int STAGEB = RNB + R0B;
  static constexpr int T1B = (TX + 4) * CELLB;  // r_{n+1} tile row: two halo cells each side
  static constexpr int T2B = (TX + 2) * CELLB;  // r_{n+2} tile row: one halo cell each side
  static constexpr int SMEM = kBarBytes + NST * STAGEB + 5 * T1B + 4 * T2B;
};

// kBlock compute threads (one 16-byte chunk of an owned cell each) and two warps for the
// halo cells: the first computes the four r_{n+1} halo cells, the second the two r_{n+2}
// halo cells and issues the copies.
constexpr int kBlock3 = kBlock + 64;

template <typename Real, int LAT, int C, int NST>
__device__ __forceinline__ bool step3_body(Ring& ring, int cta, int ncta, const void* __restrict__ r_prev,
                                           const void* __restrict__ r_cur, void* __restrict__ out2,
                                           void* __restrict__ out3, const void* __restrict__ r0,
                                           const Real* __restrict__ vt, Real tt, int Lx, int Ly, long long units,
                                           double* __restrict__ partial1, double* __restrict__ partial2,
                                           double* __restrict__ partial3, int* __restrict__ err, int realv) {
  static_assert(NST >= 7, "the ring holds slots i-3 .. i+2 and one row of prefetch");
  using Ch = Chunk<Real>;
  using Acc = typename AccT<Real>::T;
  using Sh = Step3Shape<LAT, C, NST>;
  const Real tt2 = tt + tt;  // exact; the on-site terms vt hold 2 V~
  constexpr int VPC = Ch::kVecs, NR = Ch::kReals;
  constexpr int SORB = Sh::SORB, TPC = Sh::TPC, TX = Sh::TX, CELLB = Sh::CELLB;
  static_assert(4 * TPC <= 32 && 2 * TPC <= 31, "halo cells of one chunk group per warp");
  constexpr int QT = 2 * VPC;
  constexpr int kProducer = kBlock3 - 1;
  uint64_t* bars = ring.bars;
  unsigned char* stages = ring.stages;
  unsigned char* tile1 = stages + NST * Sh::STAGEB;
  unsigned char* tile2 = tile1 + 5 * Sh::T1B;
  int& s_abort = *ring.abort;

  const int tid = threadIdx.x;
  const bool compute = tid < kBlock;
  const int hl = tid - kBlock;  // 0..63 in the halo warps
  const bool halo1 = !compute && hl < 4 * TPC;
  const bool halo2 = !compute && hl >= 32 && hl < 32 + 2 * TPC;
  const int xl = compute ? tid / TPC : 0;
  const int hc1 = halo1 ? hl / TPC : 0;          // r_{n+1} halo cell: 0, 1 left; 2, 3 right
  const int hc2 = halo2 ? (hl - 32) / TPC : 0;   // r_{n+2} halo cell: 0 left, 1 right
  const int j = compute ? tid - xl * TPC : (halo1 ? hl - hc1 * TPC : (halo2 ? hl - 32 - hc2 * TPC : 0));
  const int s = j / C;
  const int c = j - s * C;
  const int choff = (s * C + c) * 16;        // this thread's chunk inside a cell
  const int nboff = ((1 - s) * C + c) * 16;  // same chunk, other sublattice

  __syncthreads();

  const long long u0 = units * (long long)cta / ncta;
  const long long u1 = units * (long long)(cta + 1) / ncta;

  double dacc1[QT], dacc2[QT], dacc3[QT];
  Acc facc1[QT], facc2[QT], facc3[QT];
#pragma unroll
  for (int k = 0; k < QT; ++k)
    dacc1[k] = dacc2[k] = dacc3[k] = 0.0, facc1[k] = facc2[k] = facc3[k] = Acc(0);
  int rows1 = 0, rows2 = 0, rows3 = 0;
  long long gslot = ring.gslot;
  bool aborted = false;

  // periodic cell index of x in [-3, Lx + 2]; lattices of at most six cells, which the halo
  // may wrap more than once, take the modulo
  auto wrapx = [&](int x) {
    if (Lx > 6) return x < 0 ? x + Lx : (x >= Lx ? x - Lx : x);
    x %= Lx;
    return x < 0 ? x + Lx : x;
  };
  auto wrapy = [&](int y) {
    while (y < 0) y += Ly;
    while (y >= Ly) y -= Ly;
    return y;
  };

  // one site of the next iterate from three rows (up, mid, dn: rows y-1, y, y+1 of the
  // current iterate, laid out as cells of CELLB bytes) at cell index si, with on-site term
  // v (2 V~, NaN at a vacancy) and the previous iterate pv of the site
  auto site = [&](const unsigned char* up, const unsigned char* mid, const unsigned char* dn, int si, Real v,
                  const Ch& pv) -> Ch {
    const Ch me = *reinterpret_cast<const Ch*>(mid + si * CELLB + choff);
    Ch n1, n2, n3, n4;
    if (LAT == KITE_HONEYCOMB) {
      const unsigned char* other = s == 0 ? up : dn;
      const int dxi = s == 0 ? si + 1 : si - 1;
      n1 = *reinterpret_cast<const Ch*>(mid + si * CELLB + nboff);
      n2 = *reinterpret_cast<const Ch*>(other + dxi * CELLB + nboff);
      n3 = *reinterpret_cast<const Ch*>(other + si * CELLB + nboff);
    } else {
      n1 = *reinterpret_cast<const Ch*>(mid + (si - 1) * CELLB + choff);
      n2 = *reinterpret_cast<const Ch*>(mid + (si + 1) * CELLB + choff);
      n3 = *reinterpret_cast<const Ch*>(up + si * CELLB + choff);
      n4 = *reinterpret_cast<const Ch*>(dn + si * CELLB + choff);
    }
    // a vacancy holds r = 0 exactly in every iterate: with its hopping and on-site term
    // zeroed, fma(0, s, fma(0, +0, -0)) = +0
    const bool vacant = is_vacancy(v);
    const Real ve = vacant ? Real(0) : v, te = vacant ? Real(0) : tt2;
    Ch out;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      Real sum = radd(n1.v[k], n2.v[k]);
      sum = radd(sum, n3.v[k]);
      if (LAT == KITE_SQUARE) sum = radd(sum, n4.v[k]);
      out.v[k] = rfma(te, sum, rfma(ve, me.v[k], -pv.v[k]));  // 2t~ s + (2V~ r_n - r_{n-1})
    }
    return out;
  };
  auto accumulate = [&](Acc(&facc)[QT], double(&dacc)[QT], int& rows, const Ch& z0, const Ch& out) {
    if (realv) {
#pragma unroll
      for (int k = 0; k < NR; ++k) facc[k] += (Acc)z0.v[k] * (Acc)out.v[k];
    } else {
#pragma unroll
      for (int q = 0; q < VPC; ++q)
        cacc(facc[2 * q], facc[2 * q + 1], z0.v[2 * q], z0.v[2 * q + 1], out.v[2 * q], out.v[2 * q + 1]);
    }
    if (++rows == kFlushRows) {
      rows = 0;
#pragma unroll
      for (int k = 0; k < QT; ++k) dacc[k] += (double)facc[k], facc[k] = Acc(0);
    }
  };

  const int band = band_rows(units, ncta, Ly);
  const long long nstrips = units / Ly;
  for (long long u = u0; u < u1 && !aborted;) {
    const Seg seg = unit_segment(u, u1, Ly, nstrips, band);
    const int sx = seg.sx, yb = seg.yb, nr = seg.nr;
    const int x0 = sx * TX;
    const int txv = min(TX, Lx - x0);
    const int nslots = nr + 6;  // r_n rows yb-3 .. yb+nr+2

    auto copy_cells = [&](unsigned char* dst, const unsigned char* rowp, int x, int ncell, uint64_t* bar) {
      int k = 0;
      while (k < ncell) {
        const int xs = wrapx(x + k);
        const int run = min(ncell - k, Lx - xs);
        bulk_g2s(dst + (size_t)k * CELLB, rowp + (size_t)xs * CELLB, (uint32_t)run * CELLB, bar);
        k += run;
      }
    };
    auto issue = [&](int jj, int st) {  // producer: slot jj (r_n row yb-3+jj) into stage st
      unsigned char* base = stages + st * Sh::STAGEB;
      const int row = wrapy(yb - 3 + jj);
      const bool need_r0 = jj >= 3 && jj <= nr + 2;  // owned rows
      const uint32_t bytes = (uint32_t)(txv + 6) * CELLB + (need_r0 ? (uint32_t)txv * CELLB : 0u);
      mbar_arrive_expect_tx(&bars[st], bytes);
      const size_t roff = (size_t)row * Lx * CELLB;
      copy_cells(base, static_cast<const unsigned char*>(r_cur) + roff, x0 - 3, txv + 6, &bars[st]);
      if (need_r0)
        bulk_g2s(base + Sh::RNB, static_cast<const unsigned char*>(r0) + roff + (size_t)x0 * CELLB,
                 (uint32_t)txv * CELLB, &bars[st]);
    };
    if (tid == kProducer) {
      int st = (int)(gslot % NST);
      for (int jj = 0; jj < min(NST, nslots); ++jj, st = st + 1 == NST ? 0 : st + 1) issue(jj, st);
    }

    const bool active = compute && xl < txv;
    // this thread's r_{n+1} cell: owned (tile cell xl+2) or a halo cell
    const int t1 = active ? xl + 2 : (halo1 ? (hc1 < 2 ? hc1 : txv + hc1) : 0);
    const bool h1ok = halo1;  // halo cells exist whatever txv (wrapped)
    const bool l1 = active || h1ok;
    const int x1 = l1 ? wrapx(x0 - 2 + t1) : 0;  // its global cell
    // the r_{n+2} halo cell of a second-warp thread (tile-2 cell 0 or txv+1)
    const int t2h = hc2 ? txv + 1 : 0;
    const int x2h = halo2 ? wrapx(x0 - 1 + t2h) : 0;
    const Real* vcol1 = vt + (size_t)x1 * SORB + s;
    const Real* vcol2 = vt + (size_t)x2h * SORB + s;
    const uint32_t vrow = (uint32_t)Lx * SORB;
    const size_t pcol = ((size_t)x1 * SORB + s) * C + c;  // r_{n-1} chunk column of the r_{n+1} cell
    const size_t ocol = ((size_t)(x0 + xl) * SORB + s) * C + c;
    const uint32_t orow = (uint32_t)Lx * SORB * C;  // chunks per row
    Real v1 = l1 ? vcol1[(size_t)wrapy(yb - 2) * vrow] : Real(0);
    Ch pv1 = l1 ? Ch::ldg(r_prev, pcol + (size_t)wrapy(yb - 2) * orow) : Ch{};
    Real vm1 = Real(0), vm2 = Real(0), vm3 = Real(0), vm4 = Real(0);  // rows of iterations i-1 .. i-4

    // ring stages of slots i-3 .. i+2 and the phase parities of slots i-1 .. i+2
    int st0 = (int)(gslot % NST);
    auto back = [&](int st, int k) { return st - k < 0 ? st - k + NST : st - k; };
    int sm1 = back(st0, 1), sm2 = back(st0, 2), sm3 = back(st0, 3);
    int st1 = st0 + 1 == NST ? 0 : st0 + 1, st2 = st1 + 1 == NST ? 0 : st1 + 1;
    uint32_t p0 = (uint32_t)((gslot / NST) & 1), p1 = (uint32_t)(((gslot + 1) / NST) & 1),
             p2 = (uint32_t)(((gslot + 2) / NST) & 1);
    uint32_t pm1 = (uint32_t)(((gslot + NST - 1) / NST) & 1) ^ 1u;  // slot -1 (unused at i = 0)
    int a0 = 0, a1 = Sh::T1B, a2 = 2 * Sh::T1B, a3 = 3 * Sh::T1B, a4 = 4 * Sh::T1B;  // tile-1 rows i-4 .. i
    int b0 = 0, b1 = Sh::T2B, b2 = 2 * Sh::T2B, b3 = 3 * Sh::T2B;                   // tile-2 rows i-3 .. i
    int issued = min(NST, nslots);
    int i = 0;
    for (; i < nr + 6; ++i) {
      const bool do1 = i < nr + 4;             // r_{n+1} row yb-2+i
      const bool do2 = i >= 3 && i < nr + 5;   // r_{n+2} row yb-4+i
      const bool do3 = i >= 6;                 // r_{n+3} row yb-6+i
      const int y1 = yb - 2 + i, y2 = yb - 4 + i, y3 = yb - 6 + i;
      const bool more = l1 && i + 1 < nr + 4;
      const Real v1n = more ? vcol1[(size_t)wrapy(y1 + 1) * vrow] : Real(0);
      Ch pvn;
      if (more) pvn = Ch::ldg(r_prev, pcol + (size_t)wrapy(y1 + 1) * orow);
      else pvn = Ch{};
      bool ok = true;
      if (do1 && l1) {
        if (i == 0) {
          ok = mbar_wait_bounded_hint(&bars[st0], p0) && ok;
          ok = mbar_wait_bounded_hint(&bars[st1], p1) && ok;
        }
        ok = mbar_wait_bounded_hint(&bars[st2], p2) && ok;
      }
      if (do2 && halo2) ok = mbar_wait_bounded_hint(&bars[sm1], pm1) && ok;
      const unsigned char* su = stages + st0 * Sh::STAGEB;   // r_n row y1-1
      const unsigned char* sm = stages + st1 * Sh::STAGEB;   // r_n row y1 (and its r_0)
      const unsigned char* sd = stages + st2 * Sh::STAGEB;   // r_n row y1+1
      const unsigned char* sp = stages + sm1 * Sh::STAGEB;   // r_n row y2 (and its r_0)
      const unsigned char* sz = stages + sm3 * Sh::STAGEB;   // r_0 of row y3
      // r_{n+1} row y1 (own or halo cell): stage cell t1+1
      if (do1 && ok && l1) {
        const Ch o = site(su, sm, sd, t1 + 1, v1, pv1);
        *reinterpret_cast<Ch*>(tile1 + a4 + t1 * CELLB + choff) = o;
        if (active && i >= 2 && i <= nr + 1) {
          const Ch z0 = *reinterpret_cast<const Ch*>(sm + Sh::RNB + xl * CELLB + choff);
          accumulate(facc1, dacc1, rows1, z0, o);
        }
      }
      // r_{n+2} row y2: owned cell (tile-2 cell xl+1) or the second warp's halo cell, from
      // tile-1 rows y2-1 .. y2+1 (iterations i-3 .. i-1) and r_n of row y2 (slot i-1)
      if (do2 && ok && (active || halo2)) {
        const int t2 = active ? xl + 1 : t2h;
        const Real v2 = active ? vm2 : vcol2[(size_t)wrapy(y2) * vrow];
        const Ch pv2 = *reinterpret_cast<const Ch*>(sp + (t2 + 2) * CELLB + choff);
        const Ch o = site(tile1 + a1, tile1 + a2, tile1 + a3, t2 + 1, v2, pv2);
        *reinterpret_cast<Ch*>(tile2 + b3 + t2 * CELLB + choff) = o;
        if (active && i >= 4 && i <= nr + 3) {
          o.st(out2, ocol + (size_t)y2 * orow);
          const Ch z0 = *reinterpret_cast<const Ch*>(sp + Sh::RNB + xl * CELLB + choff);
          accumulate(facc2, dacc2, rows2, z0, o);
        }
      }
      // r_{n+3} row y3 (owned cell) from tile-2 rows y3-1 .. y3+1 (iterations i-3 .. i-1)
      // and r_{n+1} of row y3 (tile-1 row of iteration i-4)
      if (do3 && ok && active) {
        const Ch pv3 = *reinterpret_cast<const Ch*>(tile1 + a0 + (xl + 2) * CELLB + choff);
        const Ch o = site(tile2 + b0, tile2 + b1, tile2 + b2, xl + 1, vm4, pv3);
        o.st(out3, ocol + (size_t)y3 * orow);
        const Ch z0 = *reinterpret_cast<const Ch*>(sz + Sh::RNB + xl * CELLB + choff);
        accumulate(facc3, dacc3, rows3, z0, o);
      }
      vm4 = vm3;
      vm3 = vm2;
      vm2 = vm1;
      vm1 = v1;
      v1 = v1n;
      pv1 = pvn;
      if (!ok) s_abort = 1;
      __syncthreads();  // the tile rows are complete; slot i-3 and the oldest tile rows are free
      if (s_abort) {
        aborted = true;
        break;
      }
      if (!compute) {  // warp-uniform: the compute warps skip the producer's test
        if (tid == kProducer && i >= 3 && i - 3 + NST < nslots) {
          issue(i - 3 + NST, sm3);  // slot i-3's stage
          issued = i - 3 + NST + 1;
        }
      }
      // advance: slots, parities (a slot's phase flips when its stage index wraps to 0)
      pm1 = p0;
      const int st3 = st2 + 1 == NST ? 0 : st2 + 1;
      const uint32_t p3 = st3 == 0 ? p2 ^ 1u : p2;
      p0 = p1;
      p1 = p2;
      p2 = p3;
      sm3 = sm2;
      sm2 = sm1;
      sm1 = st0;
      st0 = st1;
      st1 = st2;
      st2 = st3;
      const int fa = a0;  // the oldest tile rows take the next rows
      a0 = a1;
      a1 = a2;
      a2 = a3;
      a3 = a4;
      a4 = fa;
      const int fb = b0;
      b0 = b1;
      b1 = b2;
      b2 = b3;
      b3 = fb;
    }
    if (aborted) {
      if (tid == kProducer) {
        for (int jj = i; jj < issued; ++jj) {  // completed phases return at once
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
  // partial1..3 <- <r_0|r_{n+1..n+3}>: fixed-order sums over the compute threads holding
  // each chunk (the ring is drained; its memory is reused)
#pragma unroll
  for (int k = 0; k < QT; ++k)
    dacc1[k] += (double)facc1[k], dacc2[k] += (double)facc2[k], dacc3[k] += (double)facc3[k];
  double* red = reinterpret_cast<double*>(stages);
  constexpr int Q = C * QT;
  cta_lane_sums<QT, C>(dacc1, compute, red, partial1 + (size_t)cta * Q);
  __syncthreads();
  cta_lane_sums<QT, C>(dacc2, compute, red, partial2 + (size_t)cta * Q);
  __syncthreads();
  cta_lane_sums<QT, C>(dacc3, compute, red, partial3 + (size_t)cta * Q);
  return true;
}

template <typename Real, int LAT, int C, int NST>
__global__ void __launch_bounds__(kBlock3, 2)
    k_step3(const void* r_prev, const void* __restrict__ r_cur, void* out2, void* out3,
            const void* __restrict__ r0, const Real* __restrict__ vt, Real tt, int Lx, int Ly, long long units,
            double* __restrict__ partial1, double* __restrict__ partial2, double* __restrict__ partial3,
            int* __restrict__ err, int realv) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  Ring ring{bars, smem + kBarBytes, &s_abort, 0};
  griddep_wait();  // the previous launch's iterates and partials are complete
  griddep_launch_dependents();
  step3_body<Real, LAT, C, NST>(ring, blockIdx.x, gridDim.x, r_prev, r_cur, out2, out3, r0, vt, tt, Lx, Ly,
                                units, partial1, partial2, partial3, err, realv);
}

template <typename Real, int LAT, int C, int NST>
int step3_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    int o = 0;
    const int smem = Step3Shape<LAT, C, NST>::SMEM;
    if (smem > 227 * 1024 ||
        cudaFuncSetAttribute(k_step3<Real, LAT, C, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_step3<Real, LAT, C, NST>, kBlock3, smem) != cudaSuccess)
      o = 0;
    cudaGetLastError();
    occ = o;
  }
  return occ;
}

}  // namespace
}  // namespace kite
