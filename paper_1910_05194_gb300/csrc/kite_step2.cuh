// kite_step2.cuh -- two recursion steps per pass (temporal blocking of the stencil sweep).
//
// From r_{n-1} and r_n one pass writes r_{n+1} = 2 H~ r_n - r_{n-1} and
// r_{n+2} = 2 H~ r_{n+1} - r_n (Eq. e6) and accumulates <r_0|r_{n+1}> and <r_0|r_{n+2}>
// (Eqs. e7/e8).  A CTA walks the rows of its share of a strip as in the one-step kernel;
// while it computes row y of r_{n+1} it computes row y-1 of r_{n+2} from the three
// r_{n+1} rows it keeps in shared memory.  r_{n+1} is therefore also computed on one
// halo row above and below the CTA's rows and on one halo cell left and right of the
// strip (redundantly: 2 of 34 cells, 2 of ~1700 rows), which needs r_n with a two-cell
// halo.  Per orbital and pass the HBM traffic is r_{n-1}, r_n, r_0 in and r_{n+1},
// r_{n+2} out: 5 vector reads/writes for two steps instead of 8.  The outputs go to two
// buffers distinct from the inputs (the halo reads of neighbouring CTAs need r_n and
// r_{n-1} unchanged during the pass).  Rounding sequence per site as in the one-step
// kernel, so the iterates are bit-identical to two one-step launches.
//
// Staging: the bulk-copy ring holds r_n (with the halo) and r_0 of each row; r_{n-1},
// read once per site by the thread that owns it, is loaded from global memory into
// registers one row ahead, which keeps the stages small enough for a ring of 4-6 rows at
// three CTAs per SM.
#pragma once

#include "kite_step.cuh"

namespace kite {
namespace {

// DBL: the moment-doubling pass (no r_0 staged; four moment slots per pass, their FP64
// partials kept in shared memory: kBlock threads x 4 slots x 4 doubles at most).  SMACC:
// the plain pass with its two FP64 partials in shared memory as well (fewer registers, for
// the persistent batched kernel).
template <int LAT, int C, int NST, bool DBL = false, bool SMACC = false>
struct Step2Shape {
  using S1 = StepShape<LAT, C, NST>;
  static constexpr int SORB = S1::SORB, TPC = S1::TPC, TX = S1::TX, CELLB = S1::CELLB;
  static constexpr int RNB = (TX + 4) * CELLB;  // r_n row, two halo cells each side
  static constexpr int R0B = DBL ? 0 : TX * CELLB;  // r_0 row
  static constexpr int STAGEB = RNB + R0B;      // (r_{n-1} is read once per site: registers)
  static constexpr int TILEB = (TX + 2) * CELLB;  // one r_{n+1} row of the tile ring
  static constexpr int DACCB = (DBL ? 4 : (SMACC ? 2 : 0)) * kBlock * 4 * 8;
  static constexpr int SMEM = kBarBytes + NST * STAGEB + 4 * TILEB + DACCB;
};

// Threads: kBlock compute threads (one 16-byte chunk of an owned cell each, as in the
// one-step kernel) and one more warp that computes the two halo cells of each r_{n+1} row
// (left: tile cell 0, right: tile cell txv+1) and issues the bulk copies, so that the
// compute warps carry equal work between the barriers.
constexpr int kBlock2 = kBlock + 32;

// Plain moments: partial1 <- <r_0|r_{n+1}>, partial2 <- <r_0|r_{n+2}>.  DBL (moment doubling,
// the slots of k_undouble): partial1 <- <r_n|r_n>, partial2 <- <r_n|r_{n+1}>, partial3 <-
// <r_{n+1}|r_{n+1}>, partial4 <- <r_{n+1}|r_{n+2}> (slots 2n .. 2n+3); r0 is not read.
template <typename Real, int LAT, int C, int NST, bool DBL = false, bool SMACC = false>
__device__ __forceinline__ bool step2_body(Ring& ring, int cta, int ncta, const void* __restrict__ r_prev,
                                           const void* __restrict__ r_cur, void* __restrict__ out1,
                                           void* __restrict__ out2, const void* __restrict__ r0,
                                           const Real* __restrict__ vt, Real tt, int Lx, int Ly, long long units,
                                           double* __restrict__ partial1, double* __restrict__ partial2,
                                           int* __restrict__ err, int realv, double* __restrict__ partial3 = nullptr,
                                           double* __restrict__ partial4 = nullptr) {
  using Ch = Chunk<Real>;
  using Acc = typename AccT<Real>::T;
  using Sh = Step2Shape<LAT, C, NST, DBL, SMACC>;
  constexpr bool SMEMSUMS = DBL || SMACC;  // FP64 partials in shared memory
  const Real tt2 = tt + tt;  // exact; the on-site terms vt hold 2 V~
  constexpr int VPC = Ch::kVecs, NR = Ch::kReals;
  constexpr int SORB = Sh::SORB, TPC = Sh::TPC, TX = Sh::TX, CELLB = Sh::CELLB;
  constexpr int QT = 2 * VPC;
  constexpr int kProducer = kBlock2 - 1;
  uint64_t* bars = ring.bars;
  unsigned char* stages = ring.stages;
  unsigned char* tile = stages + NST * Sh::STAGEB;
  int& s_abort = *ring.abort;

  const int tid = threadIdx.x;
  const bool compute = tid < kBlock;
  // compute threads: owned cell xl; halo threads: halo cell hcell (0 left, 1 right)
  const int hl = tid - kBlock;
  const bool halo = !compute && hl < 2 * TPC;
  const int xl = compute ? tid / TPC : 0;
  const int hcell = halo ? hl / TPC : 0;
  const int j = compute ? tid - xl * TPC : (halo ? hl - hcell * TPC : 0);
  const int s = j / C;
  const int c = j - s * C;
  const int choff = (s * C + c) * 16;        // this thread's chunk inside a cell
  const int nboff = ((1 - s) * C + c) * 16;  // same chunk, other sublattice

  __syncthreads();

  const long long u0 = units * (long long)cta / ncta;
  const long long u1 = units * (long long)(cta + 1) / ncta;

  double dacc1[QT], dacc2[QT];
  Acc facc1[QT], facc2[QT];
#pragma unroll
  for (int k = 0; k < QT; ++k) dacc1[k] = dacc2[k] = 0.0, facc1[k] = facc2[k] = Acc(0);
  int rows1 = 0, rows2 = 0;
  // doubling: the <r|r> halves of the two levels in FP32 (facc1/facc2 take <r|r_next>), the
  // FP64 sums of all four slots in this thread's row of shared memory
  Acc gacc1[QT], gacc2[QT];
#pragma unroll
  for (int k = 0; k < QT; ++k) gacc1[k] = gacc2[k] = Acc(0);
  constexpr int NSUM = DBL ? 4 : 2;  // FP64 sums per thread and QT lane
  double* dsm = SMEMSUMS ? reinterpret_cast<double*>(ring.stages + NST * Sh::STAGEB + 4 * Sh::TILEB) +
                               (size_t)(compute ? tid : 0) * NSUM * QT
                         : nullptr;
  if constexpr (SMEMSUMS) {
    if (compute)
#pragma unroll
      for (int k = 0; k < NSUM * QT; ++k) dsm[k] = 0.0;
  }
  long long gslot = ring.gslot;
  bool aborted = false;

  // periodic cell index of x in [-2, Lx + 1] (the copies below start up to two cells left
  // of the lattice and end up to two right of it); lattices of at most four cells, which
  // the halo may wrap more than once, take the modulo
  auto wrapx = [&](int x) {
    if (Lx > 4) return x < 0 ? x + Lx : (x >= Lx ? x - Lx : x);
    x %= Lx;
    return x < 0 ? x + Lx : x;
  };
  auto wrapy = [&](int y) { return y < 0 ? y + Ly : (y >= Ly ? y - Ly : y); };

  const int band = band_rows(units, ncta, Ly);
  const long long nstrips = units / Ly;
  for (long long u = u0; u < u1 && !aborted;) {
    const Seg seg = unit_segment(u, u1, Ly, nstrips, band);
    const int sx = seg.sx, yb = seg.yb, nr = seg.nr;
    const int x0 = sx * TX;
    const int txv = min(TX, Lx - x0);
    const int nslots = nr + 4;  // r_n rows yb-2 .. yb+nr+1

    // copies of `ncell` cells starting at global cell x (wrapped per cell when the run
    // crosses the periodic boundary) into dst
    auto copy_cells = [&](unsigned char* dst, const unsigned char* rowp, int x, int ncell, uint64_t* bar) {
      int k = 0;
      while (k < ncell) {
        const int xs = wrapx(x + k);
        int run = min(ncell - k, Lx - xs);
        bulk_g2s(dst + (size_t)k * CELLB, rowp + (size_t)xs * CELLB, (uint32_t)run * CELLB, bar);
        k += run;
      }
    };
    auto issue = [&](int jj, int st) {  // producer: slot jj (r_n row yb-2+jj) into stage st
      unsigned char* base = stages + st * Sh::STAGEB;
      int row = yb - 2 + jj;
      while (row < 0) row += Ly;
      while (row >= Ly) row -= Ly;
      const bool need_r0 = !DBL && jj >= 2 && jj <= nr + 1;  // owned rows
      const uint32_t bytes = (uint32_t)(txv + 4) * CELLB + (need_r0 ? (uint32_t)txv * CELLB : 0u);
      mbar_arrive_expect_tx(&bars[st], bytes);
      const size_t roff = (size_t)row * Lx * CELLB;
      copy_cells(base, static_cast<const unsigned char*>(r_cur) + roff, x0 - 2, txv + 4, &bars[st]);
      if (need_r0)
        bulk_g2s(base + Sh::RNB, static_cast<const unsigned char*>(r0) + roff + (size_t)x0 * CELLB,
                 (uint32_t)txv * CELLB, &bars[st]);
    };
    if (tid == kProducer) {
      int st = (int)(gslot % NST);
      for (int jj = 0; jj < min(NST, nslots); ++jj, st = st + 1 == NST ? 0 : st + 1) issue(jj, st);
    }

    // one r_{n+1} site: tile cell tx (global x0 - 1 + tx) of row y1 from the stages of
    // rows y1-1, y1, y1+1 (up, mid, dn) and r_{n-1} of the site (pv)
    auto site1 = [&](const unsigned char* up, const unsigned char* mid, const unsigned char* dn, int tx,
                     Real v, const Ch& pv) -> Ch {
      const int si = tx + 1;  // index in the r_n stage (two halo cells on the left)
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
      // a vacancy (v is NaN) holds r = 0 exactly in every iterate, so with its hopping and
      // on-site term zeroed fma(0, s, fma(0, +0, -0)) = +0: the same bits as forcing the
      // output to zero, with two selects per site instead of one per component
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
    // one r_{n+2} site of owned cell xl (tile cell xl+1) of row y2 from the tile rows
    // y2-1, y2, y2+1 (tu, tm, td) and r_n of row y2 (stage mid2)
    auto site2 = [&](const unsigned char* tu, const unsigned char* tm, const unsigned char* td,
                     const unsigned char* mid2, Real v) -> Ch {
      const int tx = xl + 1;
      const Ch me = *reinterpret_cast<const Ch*>(tm + tx * CELLB + choff);
      Ch n1, n2, n3, n4;
      if (LAT == KITE_HONEYCOMB) {
        const unsigned char* other = s == 0 ? tu : td;
        const int dxi = s == 0 ? tx + 1 : tx - 1;
        n1 = *reinterpret_cast<const Ch*>(tm + tx * CELLB + nboff);
        n2 = *reinterpret_cast<const Ch*>(other + dxi * CELLB + nboff);
        n3 = *reinterpret_cast<const Ch*>(other + tx * CELLB + nboff);
      } else {
        n1 = *reinterpret_cast<const Ch*>(tm + (tx - 1) * CELLB + choff);
        n2 = *reinterpret_cast<const Ch*>(tm + (tx + 1) * CELLB + choff);
        n3 = *reinterpret_cast<const Ch*>(tu + tx * CELLB + choff);
        n4 = *reinterpret_cast<const Ch*>(td + tx * CELLB + choff);
      }
      const Ch pv = *reinterpret_cast<const Ch*>(mid2 + (tx + 1) * CELLB + choff);  // r_n, own cell
      // a vacancy (v is NaN) holds r = 0 exactly in every iterate, so with its hopping and
      // on-site term zeroed fma(0, s, fma(0, +0, -0)) = +0: the same bits as forcing the
      // output to zero, with two selects per site instead of one per component
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
        for (int q = 0; q < VPC; ++q) cacc(facc[2 * q], facc[2 * q + 1], z0.v[2 * q], z0.v[2 * q + 1],
                                            out.v[2 * q], out.v[2 * q + 1]);
      }
      if (++rows == kFlushRows) {
        rows = 0;
#pragma unroll
        for (int k = 0; k < QT; ++k) dacc[k] += (double)facc[k], facc[k] = Acc(0);
      }
    };

    // the plain moment with its FP64 sum in this thread's shared-memory slot ks
    auto accumulate_sm = [&](Acc(&facc)[QT], int& rows, int ks, const Ch& z0, const Ch& out) {
      if (realv) {
#pragma unroll
        for (int k = 0; k < NR; ++k) facc[k] += (Acc)z0.v[k] * (Acc)out.v[k];
      } else {
#pragma unroll
        for (int q = 0; q < VPC; ++q) cacc(facc[2 * q], facc[2 * q + 1], z0.v[2 * q], z0.v[2 * q + 1],
                                            out.v[2 * q], out.v[2 * q + 1]);
      }
      if (++rows == kFlushRows) {
        rows = 0;
#pragma unroll
        for (int k = 0; k < QT; ++k) dsm[ks * QT + k] += (double)facc[k], facc[k] = Acc(0);
      }
    };
    // doubling: fr <- <me|out> (complex chain as in the one-step kernel), fg <- <me|me>
    // (real part); every kFlushRows rows both go into this thread's FP64 slots ka, kb
    auto accumulate_dbl = [&](Acc(&fr)[QT], Acc(&fg)[QT], int& rows, int ka, int kb, const Ch& me,
                              const Ch& out) {
      if (realv) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const Acc a = me.v[k], b = out.v[k];
          fr[k] += a * b;
          fg[k] += a * a;
        }
      } else {
#pragma unroll
        for (int q = 0; q < VPC; ++q) {
          cacc(fr[2 * q], fr[2 * q + 1], me.v[2 * q], me.v[2 * q + 1], out.v[2 * q], out.v[2 * q + 1]);
          const Acc ar = me.v[2 * q], ai = me.v[2 * q + 1];
          fg[2 * q] = rfma(ai, ai, rfma(ar, ar, fg[2 * q]));
        }
      }
      if (++rows == kFlushRows) {
        rows = 0;
#pragma unroll
        for (int k = 0; k < QT; ++k) {
          dsm[ka * QT + k] += (double)fg[k];
          dsm[kb * QT + k] += (double)fr[k];
          fr[k] = fg[k] = Acc(0);
        }
      }
    };

    const bool active = compute && xl < txv;
    // on-site terms prefetched one row ahead: the owned (or halo) cell of r_{n+1} row
    // y1 = yb-1+i; r_{n+2} row y2 = y1-1 reuses the previous row's value
    const int xv = active ? x0 + xl : (halo ? wrapx(x0 - 1 + (hcell ? txv + 1 : 0)) : 0);
    const bool loads_v = active || halo;
    const Real* vcol = vt + (size_t)xv * SORB + s;
    const uint32_t vrow = (uint32_t)Lx * SORB;
    auto vload = [&](int y) { return vcol[(size_t)wrapy(y) * vrow]; };
    // this thread's chunk in the outputs: column offset + row * orow chunks (orow fits 32
    // bits; row * orow is formed in 64 bits)
    const size_t ocol = ((size_t)(x0 + xl) * SORB + s) * C + c;
    const uint32_t orow = (uint32_t)Lx * SORB * C;
    Real v1 = loads_v ? vload(yb - 1) : Real(0);
    // r_{n-1} of the same cell, read straight from global memory one row ahead (it is
    // used once, by this thread)
    const size_t pcol = ((size_t)xv * SORB + s) * C + c;
    Ch pv1 = loads_v ? Ch::ldg(r_prev, pcol + (size_t)wrapy(yb - 1) * orow) : Ch{};
    // the prefetch row yn = yb + i of r_{n-1} and the on-site terms, wrapped as it advances
    // (the stored rows yb-1+i and yb-3+i are owned rows whenever they are stored).  The
    // four global streams advance one row per iteration, so their byte addresses are
    // carried across iterations (rows yb-1+i and yb-3+i of the outputs: addresses of rows
    // above the lattice are formed but only dereferenced once they are inside it).
    int yn = yb;
    const long long orowb = (long long)orow * 16;
    unsigned char* po1 = static_cast<unsigned char*>(out1) + (long long)(ocol * 16) + (long long)(yb - 1) * orowb;
    unsigned char* po2 = static_cast<unsigned char*>(out2) + (long long)(ocol * 16) + (long long)(yb - 3) * orowb;
    const unsigned char* pp = static_cast<const unsigned char*>(r_prev) + pcol * 16 + (size_t)yb * orowb;
    const Real* pvt = vcol + (size_t)yb * vrow;
    const long long ly_orowb = (long long)Ly * orowb, ly_vrow = (long long)Ly * vrow;
    // One barrier per row: iteration i computes r_{n+1} row yb-1+i (slots i, i+1, i+2 hold
    // r_n rows yb-2+i .. yb+i) into tile row i mod 4, and r_{n+2} row yb-3+i from the three
    // tile rows written by the previous iterations, with r_n and r_0 of that row from slot
    // i-1.  Slot i-1 is free after iteration i.  (Tile rows rotate as byte offsets: pointers
    // carried around the loop would hide from the compiler that they address shared memory.)
    int st0 = (int)(gslot % NST);           // stage of slot i
    int stm = st0 == 0 ? NST - 1 : st0 - 1;  // stage of slot i-1
    int o0 = 0, o1 = Sh::TILEB, o2 = 2 * Sh::TILEB, o3 = 3 * Sh::TILEB;  // tile rows i-3 .. i
    Real vm1 = Real(0), vm2 = Real(0);  // on-site terms of the rows of iterations i-1, i-2
    int issued = min(NST, nslots);      // slots issued so far (producer's count)
    uint32_t par2 = (uint32_t)(((gslot + 2) / NST) & 1);  // phase parity of slot i+2
    int i = 0;
    for (; i < nr + 3; ++i) {
      const bool do1 = i < nr + 2;  // r_{n+1} row yb-1+i
      const bool do2 = i >= 3;      // r_{n+2} row yb-3+i
      const bool more = loads_v && i + 1 < nr + 2;
      const Real v1n = more ? *pvt : Real(0);
      Ch pvn;
      if (more) pvn = Ch::ldg(pp, 0);
      else pvn = Ch{};
      const int st1 = st0 + 1 == NST ? 0 : st0 + 1;
      const int st2 = st1 + 1 == NST ? 0 : st1 + 1;
      bool ok = true;
      if (do1 && (compute || halo)) {
        if (i == 0)
          for (int jj = 0; jj < 2; ++jj) {
            const long long g = gslot + jj;
            ok = mbar_wait_bounded_hint(&bars[g % NST], (uint32_t)((g / NST) & 1)) && ok;
          }
        ok = mbar_wait_bounded_hint(&bars[st2], par2) && ok;
      }
      const unsigned char* up = stages + st0 * Sh::STAGEB;
      const unsigned char* mid = stages + st1 * Sh::STAGEB;
      const unsigned char* dn = stages + st2 * Sh::STAGEB;
      unsigned char* t3 = tile + o3;
      if (do1 && ok && active) {  // own cell (tile cell xl+1)
        const Ch o = site1(up, mid, dn, xl + 1, v1, pv1);
        *reinterpret_cast<Ch*>(t3 + (xl + 1) * CELLB + choff) = o;
        if (i >= 1 && i <= nr) {
          o.st(po1, 0);
          if constexpr (DBL) {
            const Ch me = *reinterpret_cast<const Ch*>(mid + (xl + 2) * CELLB + choff);  // r_n
            accumulate_dbl(facc1, gacc1, rows1, 0, 1, me, o);
          } else {
            const Ch z0 = *reinterpret_cast<const Ch*>(mid + Sh::RNB + xl * CELLB + choff);
            if constexpr (SMACC) accumulate_sm(facc1, rows1, 0, z0, o);
            else accumulate(facc1, dacc1, rows1, z0, o);
          }
        }
      }
      if (do1 && ok && halo) {  // halo cell left (tile cell 0) or right (tile cell txv+1)
        const int tx = hcell ? txv + 1 : 0;
        *reinterpret_cast<Ch*>(t3 + tx * CELLB + choff) = site1(up, mid, dn, tx, v1, pv1);
      }
      if (do2 && ok && active) {
        // r_{n+2} row y2 = yb-3+i from tile rows y2-1, y2, y2+1 and r_n, r_0 of row y2
        const unsigned char* prev = stages + stm * Sh::STAGEB;
        const Ch o = site2(tile + o0, tile + o1, tile + o2, prev, vm2);
        o.st(po2, 0);
        if constexpr (DBL) {
          const Ch me = *reinterpret_cast<const Ch*>(tile + o1 + (xl + 1) * CELLB + choff);  // r_{n+1}
          accumulate_dbl(facc2, gacc2, rows2, 2, 3, me, o);
        } else {
          const Ch z0 = *reinterpret_cast<const Ch*>(prev + Sh::RNB + xl * CELLB + choff);
          if constexpr (SMACC) accumulate_sm(facc2, rows2, 1, z0, o);
          else accumulate(facc2, dacc2, rows2, z0, o);
        }
      }
      vm2 = vm1;
      vm1 = v1;
      v1 = v1n;
      pv1 = pvn;
      if (st2 == NST - 1) par2 ^= 1u;  // slot i+3 starts the ring's next round
      po1 += orowb;
      po2 += orowb;
      pp += orowb;
      pvt += vrow;
      if (yn + 1 == Ly) {
        pp -= ly_orowb;
        pvt -= ly_vrow;
      }
      yn = yn + 1 == Ly ? 0 : yn + 1;
      const int of = o0;  // the oldest tile row takes the next r_{n+1} row
      o0 = o1;
      o1 = o2;
      o2 = o3;
      o3 = of;
      if (!ok) s_abort = 1;
      __syncthreads();  // the tile row is complete; slot i-1 and the oldest tile row are free
      if (s_abort) {
        aborted = true;
        break;
      }
      if (!compute) {  // warp-uniform: the eight compute warps skip the producer's test
        if (tid == kProducer && i >= 1 && i - 1 + NST < nslots) {
          issue(i - 1 + NST, stm);  // slot i-1's stage
          issued = i + NST;
        }
      }
      stm = st0;
      st0 = st1;
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
  // partial1 <- <r_0|r_{n+1}>, partial2 <- <r_0|r_{n+2}>: fixed-order sums over the compute
  // threads holding each chunk, as in the one-step kernel (the ring is drained; its
  // memory is reused)
  double* red = reinterpret_cast<double*>(stages);
  constexpr int Q = C * QT;
  if constexpr (DBL) {
    // slot k's FP64 sum from shared memory plus the FP32 rows since the last flush
    double* const outs[4] = {partial1, partial2, partial3, partial4};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      double d[QT];
#pragma unroll
      for (int k = 0; k < QT; ++k) {
        const Acc f = kk == 0 ? gacc1[k] : kk == 1 ? facc1[k] : kk == 2 ? gacc2[k] : facc2[k];
        d[k] = compute ? dsm[kk * QT + k] + (double)f : 0.0;
      }
      if (kk) __syncthreads();
      cta_lane_sums<QT, C>(d, compute, red, outs[kk] + (size_t)cta * Q);
    }
    return true;
  }
  if constexpr (SMACC) {
#pragma unroll
    for (int k = 0; k < QT; ++k) {
      dacc1[k] = compute ? dsm[k] : 0.0;
      dacc2[k] = compute ? dsm[QT + k] : 0.0;
    }
  }
#pragma unroll
  for (int k = 0; k < QT; ++k) dacc1[k] += (double)facc1[k], dacc2[k] += (double)facc2[k];
  cta_lane_sums<QT, C>(dacc1, compute, red, partial1 + (size_t)cta * Q);
  __syncthreads();
  cta_lane_sums<QT, C>(dacc2, compute, red, partial2 + (size_t)cta * Q);
  return true;
}

template <typename Real, int LAT, int C, int NST, bool DBL = false>
__global__ void __launch_bounds__(kBlock2, 3 * Step2Shape<LAT, C, NST, DBL>::SMEM <= 227 * 1024 ? 3 : 2)
    k_step2(const void* r_prev, const void* __restrict__ r_cur, void* out1, void* out2,
            const void* __restrict__ r0, const Real* __restrict__ vt, Real tt, int Lx, int Ly, long long units,
            double* __restrict__ partial1, double* __restrict__ partial2, int* __restrict__ err, int realv,
            double* __restrict__ partial3 = nullptr, double* __restrict__ partial4 = nullptr) {
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
  step2_body<Real, LAT, C, NST, DBL>(ring, blockIdx.x, gridDim.x, r_prev, r_cur, out1, out2, r0, vt, tt, Lx, Ly,
                                     units, partial1, partial2, err, realv, partial3, partial4);
}

template <typename Real, int LAT, int C, int NST, bool DBL = false>
int step2_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    int o = 0;
    const int smem = Step2Shape<LAT, C, NST, DBL>::SMEM;
    cudaFuncSetAttribute(k_step2<Real, LAT, C, NST, DBL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_step2<Real, LAT, C, NST, DBL>, kBlock2, smem) !=
        cudaSuccess)
      o = 0;
    occ = o;
  }
  return occ;
}

}  // namespace
}  // namespace kite
