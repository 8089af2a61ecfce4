// kite_gemm.cu -- complex inner products C[n][m] = sum_k A[n][k] * B[m][k] of
// split-BF16 operands on the 5th-generation tensor cores (tcgen05.mma with TMEM
// accumulators, TMA tile loads), FP32 accumulation within a K sub-chunk and FP64 above.
//
// The 2D Kubo-Bastin moments (Sec. 2b, Eq. Gammanm) are mu_nm = <a_n|b_m>/N: a complex
// contraction over all orbitals of two stored Chebyshev vector families.  Written as
// real GEMMs over K = 2N interleaved (re, im) values:
//   Re <a|b> = sum (ar br + ai bi)   = A' . B'
//   Im <a|b> = sum (ar bi - ai br)   = A' . (-i b)'
// so the B operand holds, for every m, the rows b_m and -i b_m (the "extended" B with
// 2M rows) and one real GEMM A' B_ext^T gives both parts.  Each FP32 value x is split
// into hi = bf16(x), lo = bf16(x - hi); the product keeps hi*hi + hi*lo + lo*hi and, by
// default, lo*lo: the dropped lo*lo term is always positive for aligned products (e.g. the
// diagonal <h r|h r>) and would bias them by up to ~5e-6 relative.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "kite_device.cuh"
#include "kite_internal.h"
#include "kite_tc.cuh"

namespace kite {
namespace {

#ifndef KITE_GEMM_BN
#define KITE_GEMM_BN 256
#endif
#ifndef KITE_GEMM_STAGES
#define KITE_GEMM_STAGES 4
#endif
// 32-column stages (64-byte swizzle) in a four-deep ring measured faster than 64-column
// stages in a two-deep one: the same 192 KB in flight, refilled at half the granularity
#ifndef KITE_GEMM_BK
#define KITE_GEMM_BK 32
#endif
constexpr int kBM = 128;                       // rows of A per tile (UMMA M)
constexpr int kBN = KITE_GEMM_BN;              // rows of B per tile (UMMA N)
constexpr int kKB = 64;                        // K columns per block of the K-blocked families
constexpr int kBK = KITE_GEMM_BK;              // K per stage: one 128-byte (64) or 64-byte (32) swizzle row
constexpr int kSub = kKB / kBK;                // stages per family K block
constexpr int kUK = 16;                        // K per tcgen05.mma of kind::f16
static_assert(kBK == 64 || kBK == 32, "stage K must be 64 or 32");
constexpr int kGStages = KITE_GEMM_STAGES;
constexpr int kATile = kBM * kBK * 2;          // 8 KB at kBK = 32
constexpr int kBTile = kBN * kBK * 2;          // 16 KB
constexpr int kStageBytes = 2 * kATile + 2 * kBTile;   // A hi, A lo, B hi, B lo
#ifndef KITE_GEMM_EPI_WARPS
#define KITE_GEMM_EPI_WARPS 8
#endif
constexpr int kEpiWarps = KITE_GEMM_EPI_WARPS;  // 4 or 8: one or two per TMEM lane quarter
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // warp 0 TMA, warp 1 MMA, warps 2.. epilogue
constexpr int kAccCols = kBN;                  // FP32 accumulator columns per buffer
constexpr int kTmemCols = 2 * kAccCols;        // double-buffered accumulator
constexpr int kHalfCols = kAccCols * 4 / kEpiWarps;  // columns of one epilogue warp
static_assert(kHalfCols % 32 == 0, "epilogue works on 32-column blocks");
constexpr int kEpiPitch = 33;                  // floats per transposed row (bank-conflict free)
constexpr int kEpiBytes = kEpiWarps * 32 * kEpiPitch * 4;
constexpr int kGemmSmem = 1024 + kGStages * kStageBytes + kEpiBytes + 256;

// Instruction descriptor of tcgen05.mma kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

// Shared-memory matrix descriptor for a K-major tile written by TMA with 128-byte
// swizzle: start address >> 4 (bits 0-13), leading byte offset (unused with swizzle,
// 16 B), stride byte offset = 1024 B between 8-row groups (bits 32-45), descriptor
// version 1 (bit 46), swizzle mode 2 = 128 B (bits 61-63).
// With a 64-byte swizzle (32-column stages) the 8-row groups are 512 B apart and the
// swizzle mode is 4.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)((8u * kBK * 2u) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(kBK == 64 ? 2 : 4) << 61;
  return d;
}

// One box of a K-blocked family: kBK columns of rows [y, y + box) at stage block kb (family
// K block kb / kSub, columns (kb % kSub) * kBK: a multiple of 32 bf16, 64 bytes).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint64_t* bar,
                                            int y, int kb) {
  const int z = kb / kSub, x = (kb - z * kSub) * kBK;
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

// The same box multicast to the CTAs of `mask` in the cluster: the data lands at the same
// shared-memory offset in each, whose mbarrier at `bar`'s offset receives the bytes.
__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int y, int kb,
                                               uint16_t mask) {
  const int z = kb / kSub, x = (kb - z * kSub) * kBK;
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Arrives on the mbarrier at `bar`'s offset in every CTA of `mask` once this thread's
// tcgen05 operations complete.
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

struct GemmArgs {
  int T;            // output tiles = TM * TN
  int TN;           // tiles along the B rows
  int S;            // K splits
  int items;        // S * T
  int kb_total;     // K blocks of 64
  int kb_per_item;  // K blocks per split
  int sub_kb;       // K blocks per FP32 accumulation sub-chunk (in TMEM)
  int fold;         // sub-chunks summed in FP32 registers before the FP64 partials
  int nprod;        // 3: hi*hi + hi*lo + lo*hi;  4: + lo*lo
  int Mrows;        // rows of A (valid)
  int Nrows;        // rows of B (valid) = columns of C
  double* part;     // [S][Mrows][Nrows] FP64 partial sums
  int* err;
};

// MC: clusters of two CTAs on tiles with the same B rows (tile rows 2p and 2p+1 of A):
// each CTA loads its own A tile and half of the shared B tile, multicast to both, so a
// CTA pulls 2/3 of the operand bytes per stage from L2; a stage is refilled once both
// CTAs' MMAs have released it (their commits arrive on both CTAs' `empty` barriers).
template <bool MC>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_split_bf16(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                      const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                      const GemmArgs a) {
  extern __shared__ unsigned char gsmem_raw[];
  // 1024-byte aligned operand stages (128-byte swizzle atoms repeat every 1024 bytes)
  const uint32_t raw = smem_u32(gsmem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gsmem = gsmem_raw + (base - raw);
  float* epi = reinterpret_cast<float*>(gsmem + kGStages * kStageBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gsmem + kGStages * kStageBytes + kEpiBytes);
  uint64_t* full = bars;                  // [kGStages] TMA -> MMA
  uint64_t* empty = bars + kGStages;      // [kGStages] MMA -> TMA
  uint64_t* tfull = bars + 2 * kGStages;  // [2] MMA -> epilogue
  uint64_t* tempty = bars + 2 * kGStages + 2;  // [2] epilogue -> MMA
  uint64_t* drain = bars + 2 * kGStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kGStages + 5);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // work items: one output tile (MC: a pair of tiles, this CTA's being row 2p + rank) and
  // one K split each, split-major across the persistent grid (MC: across the clusters)
  const int crank = MC ? cluster_rank() : 0;
  const int cid = MC ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int ncl = MC ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int nitems = MC ? a.items / 2 : a.items;
  const int Tw = MC ? a.T / 2 : a.T;  // work tiles per split
  auto coords = [&](int it, int& s, int& tm, int& tn) {
    s = it / Tw;
    const int t = it - s * Tw;
    tm = t / a.TN;
    tn = t - tm * a.TN;
    if (MC) tm = 2 * tm + crank;
  };
  if (threadIdx.x == 0) {
    for (int i = 0; i < kGStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], MC ? 2 : 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 32 * kEpiWarps);
    }
    mbar_init(drain, 1);
    mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 1) {  // the whole warp allocates the accumulator columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if (MC) cluster_sync();  // the peer's barriers are initialised before any multicast arrives
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      int st = 0;
      uint32_t ph = 0;
      bool ok = true;
      int pend[kGStages];  // parity of the last phase issued on each stage (-1: none)
      for (int i = 0; i < kGStages; ++i) pend[i] = -1;
      for (int item = cid; item < nitems && ok; item += ncl) {
        int s, tm, tn;
        coords(item, s, tm, tn);
        const int kb0 = s * a.kb_per_item, kb1 = min(a.kb_total, kb0 + a.kb_per_item);
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!wait_or_abort(&empty[st], ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[st], kStageBytes);
          const uint32_t sb = base + st * kStageBytes;
          tma_load_3d(sb, &tmAh, &full[st], tm * kBM, kb);
          tma_load_3d(sb + kATile, &tmAl, &full[st], tm * kBM, kb);
          if (MC) {  // this CTA's half of the B rows, to both CTAs of the pair
            const uint32_t hoff = (uint32_t)crank * (kBTile / 2);
            tma_load_3d_mc(sb + 2 * kATile + hoff, &tmBh, &full[st], tn * kBN + crank * (kBN / 2), kb, 3);
            tma_load_3d_mc(sb + 2 * kATile + kBTile + hoff, &tmBl, &full[st], tn * kBN + crank * (kBN / 2), kb, 3);
          } else {
            tma_load_3d(sb + 2 * kATile, &tmBh, &full[st], tn * kBN, kb);
            tma_load_3d(sb + 2 * kATile + kBTile, &tmBl, &full[st], tn * kBN, kb);
          }
          pend[st] = (int)ph;
          if (++st == kGStages) st = 0, ph ^= 1u;
        }
      }
      if (!ok) {
        // drain: wait (bounded) until the last copies issued on every stage have landed
        for (int i = 0; i < kGStages; ++i)
          if (pend[i] >= 0) mbar_wait_bounded(&full[i], (uint32_t)pend[i]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      int st = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      for (int item = cid; item < nitems && ok; item += ncl) {
        int s, tm, tn;
        coords(item, s, tm, tn);
        const int kb0 = s * a.kb_per_item, kb1 = min(a.kb_total, kb0 + a.kb_per_item);
        for (int kc = kb0; kc < kb1 && ok; kc += a.sub_kb) {
          if (!wait_or_abort(&tempty[acc], aph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * kAccCols);
          const int kce = min(kb1, kc + a.sub_kb);
          for (int kb = kc; kb < kce; ++kb) {
            if (!wait_or_abort(&full[st], ph, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sb = base + st * kStageBytes;
#pragma unroll
            for (int kk = 0; kk < kBK / kUK; ++kk) {
              const uint32_t koff = kk * kUK * 2;  // bytes along the swizzled row
              const uint64_t ah = desc_sw128(sb + koff);
              const uint64_t al = desc_sw128(sb + kATile + koff);
              const uint64_t bh = desc_sw128(sb + 2 * kATile + koff);
              const uint64_t bl = desc_sw128(sb + 2 * kATile + kBTile + koff);
              umma_bf16(d, ah, bh, (kb > kc || kk > 0) ? 1u : 0u);
              umma_bf16(d, ah, bl, 1u);
              umma_bf16(d, al, bh, 1u);
              if (a.nprod == 4) umma_bf16(d, al, bl, 1u);
            }
            if (MC)
              umma_commit_mc(&empty[st], 3);  // both CTAs' B halves sit in this stage
            else
              umma_commit(&empty[st]);  // stage reusable once these MMAs have read it
            if (++st == kGStages) st = 0, ph ^= 1u;
          }
          if (!ok) break;
          umma_commit(&tfull[acc]);  // accumulator ready for the epilogue
          if (++acc == 2) acc = 0, aph ^= 1u;
        }
      }
      // make sure no MMA is still writing TMEM before the columns are released
      umma_commit(drain);
      const long long t0 = clock64();
      while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {  // ---- epilogue: warps 2.. fold the idle accumulator into FP32 registers
    // Two FP32 levels below FP64: the tensor core sums one sub-chunk (sub_kb K blocks) in
    // TMEM; this warp adds each finished sub-chunk of its 32 rows x 128 columns into d2
    // (registers) and frees the TMEM buffer at once, so the MMA never waits on memory;
    // every `fold` sub-chunks (and at the end of an item) d2 goes into the FP64 partials.
    const int q = warp & 3;                           // TMEM lane quarter this warp may access
    const int half = (warp - 2) / 4;                  // which 128 of the 256 columns
    float* tile = epi + (warp - 2) * 32 * kEpiPitch;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * kHalfCols);
    constexpr int kBlk = kHalfCols / 32;
    float d2[kBlk][32];
    int acc = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int item = cid; item < nitems && ok; item += ncl) {
      int s, tm, tn;
      coords(item, s, tm, tn);
      const int kb0 = s * a.kb_per_item, kb1 = min(a.kb_total, kb0 + a.kb_per_item);
      const int row0 = tm * kBM + q * 32;
      double* pbase = a.part + ((size_t)s * a.Mrows + row0) * a.Nrows;
      bool first = true;
      int nsub = 0;
#pragma unroll
      for (int j = 0; j < kBlk; ++j)
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) d2[j][jj] = 0.f;
      for (int kc = kb0; kc < kb1; kc += a.sub_kb) {
        if (!wait_or_abort(&tfull[acc], aph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int j = 0; j < 2 * kBlk; ++j) {
          uint32_t r[16];
          tmem_ld_32x16(lane_base + (uint32_t)(acc * kAccCols + j * 16), r);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) d2[j >> 1][(j & 1) * 16 + jj] += __uint_as_float(r[jj]);
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc]);  // the MMA may refill this buffer now
        if (++acc == 2) acc = 0, aph ^= 1u;
        if (++nsub < a.fold && kc + a.sub_kb < kb1) continue;
        // flush d2 into the FP64 partials: transpose 32 rows x 32 columns through shared
        // memory so that a warp's FP64 loads and stores run along a row
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) tile[lane * kEpiPitch + jj] = d2[j][jj];
          __syncwarp();
          const int col = tn * kBN + half * kHalfCols + j * 32 + lane;
          const bool colok = col < a.Nrows;
          double* p = pbase + col;
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) d2[j][jj] = 0.f;
#pragma unroll 1  // unrolled, the 32 rows' addresses stay live and the epilogue spills
          for (int h = 0; h < 32; h += 8) {
            double old[8];  // 8 loads in flight before any use
#pragma unroll
            for (int rr = 0; rr < 8; ++rr)
              old[rr] = (!first && colok && row0 + h + rr < a.Mrows) ? p[(size_t)(h + rr) * a.Nrows] : 0.0;
#pragma unroll
            for (int rr = 0; rr < 8; ++rr)
              if (colok && row0 + h + rr < a.Mrows)
                p[(size_t)(h + rr) * a.Nrows] = old[rr] + (double)tile[(h + rr) * kEpiPitch + lane];
          }
          __syncwarp();
        }
        first = false;
        nsub = 0;
      }
    }
  }

  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicExch(a.err, 1);
  // MC: neither CTA leaves while the other may still multicast into it or arrive on its
  // barriers (every wait above is bounded, so both reach this point)
  if (MC) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// Operand preparation and reduction (used by the generic inner-product entry point)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));  // x - hi is exact in FP32
}

// rows [rows][N] complex FP32 -> hi/lo families of `out_rows` rows and K = Kp columns
// (K-blocked, fam_index) holding 2N interleaved (re, im) values.  rot = 1 writes
// -i*z = (im, -re) instead of z.  Columns [2N, Kp) are zero.
__global__ void k_split_rows(const float2* __restrict__ z, int rows, int64_t N, int64_t Kp,
                             int row_off, int out_rows, int rot, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
  const int64_t total = (int64_t)rows * (Kp / 2);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / (Kp / 2));
    const int64_t o = e - (int64_t)r * (Kp / 2);
    float re = 0.f, im = 0.f;
    if (o < N) {
      const float2 v = z[(int64_t)r * N + o];
      re = rot ? v.y : v.x;
      im = rot ? -v.x : v.y;
    }
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(re, h0, l0);
    split_bf16(im, h1, l1);
    const int64_t dst = fam_index(row_off + r, 2 * o, out_rows);
    hi[dst] = h0;
    hi[dst + 1] = h1;
    lo[dst] = l0;
    lo[dst + 1] = l1;
  }
}

// C[n][m] (complex FP64) = sum_s part[s][n][m] + i sum_s part[s][n][M2 + m], scaled.
__global__ void k_reduce_cplx(const double* __restrict__ part, int S, int M, int M2,
                              double scale, double* __restrict__ out, int accumulate) {
  const int64_t total = (int64_t)M * M2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / M2), m = (int)(e - (e / M2) * M2);
    const int ldc = 2 * M2;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < S; ++s) {
      const double* p = part + ((size_t)s * M + n) * ldc;
      re += p[m];
      im += p[M2 + m];
    }
    if (accumulate) {
      out[2 * e] += re * scale;
      out[2 * e + 1] += im * scale;
    } else {
      out[2 * e] = re * scale;
      out[2 * e + 1] = im * scale;
    }
  }
}

// Tensor map of a K-blocked family [Kp/64][rows][64] (bf16): dims {64, rows, Kp/64}.
int make_map(kite_ctx* ctx, CUtensorMap* m, const void* ptr, int64_t Kp, int rows, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(ctx, KITE_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)kKB, (cuuint64_t)rows, (cuuint64_t)(Kp / kKB)};
  cuuint64_t strides[2] = {(cuuint64_t)kKB * 2, (cuuint64_t)rows * kKB * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   kBK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(ctx, KITE_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return KITE_OK;
}

}  // namespace

// Split-BF16 GEMM over operands already in hi/lo form:
//   part[s][n][m] for n < Mrows (A rows), m < Nrows (B rows), K = Kp (multiple of 64).
// Returns the number of splits used in *S_out.  `part` must hold S*Mrows*Nrows doubles;
// plan_gemm_splits() gives S.
int plan_gemm_splits(kite_ctx* ctx, int Mrows, int Nrows, int64_t Kp) {
  const int TM = (Mrows + kBM - 1) / kBM, TN = (Nrows + kBN - 1) / kBN;
  const int T = TM * TN;
  const int kb_total = (int)(Kp / kKB);
  // splits so that items fill whole waves of the persistent grid, at least 2 K blocks each
  int best = 1;
  for (int s = 1; s <= std::max(1, kb_total / 2); ++s) {
    if ((int64_t)s * T > 16LL * ctx->num_sms) break;
    best = s;
    if (((int64_t)s * T) % ctx->num_sms == 0 && (int64_t)s * T >= 4LL * ctx->num_sms) break;
  }
  return best;
}

// The CTA-pair variant (B tiles multicast within a two-CTA cluster, a third fewer operand
// bytes per CTA from L2) gave the same results bit for bit but was not faster on the
// 1024^2, M = 1024 contraction (1690 against 1715 TFLOP/s): the loads are not what holds
// the kernel below the tensor peak.  It stays selectable at build time.
#ifndef KITE_GEMM_MULTICAST
#define KITE_GEMM_MULTICAST 0
#endif

int gemm_split_bf16(kite_ctx* ctx, const void* Ahi, const void* Alo, const void* Bhi,
                    const void* Blo, int Mrows, int Nrows, int64_t Kp, int S, int sub_kb,
                    int fold, int nprod, double* part, int* S_used) {
  if (Kp % kKB != 0) return fail(ctx, KITE_ERR_ARG, "K must be padded to a multiple of 64");
  GemmArgs a;
  a.TN = (Nrows + kBN - 1) / kBN;
  const int TM = (Mrows + kBM - 1) / kBM;
  a.T = TM * a.TN;
  // splits and sub-chunks are planned in family K blocks (64 columns) and run in stages
  const int kb64 = (int)(Kp / kKB);
  a.S = std::max(1, std::min(S, kb64));
  const int per64 = (kb64 + a.S - 1) / a.S;
  a.S = (kb64 + per64 - 1) / per64;  // every split has >= 1 K block
  a.kb_total = kb64 * kSub;
  a.kb_per_item = per64 * kSub;
  a.items = a.S * a.T;
  *S_used = a.S;  // the reduction must sum exactly the splits written here
  a.sub_kb = std::max(1, sub_kb) * kSub;
  a.fold = std::max(1, fold);
  a.nprod = nprod == 3 ? 3 : 4;
  a.Mrows = Mrows;
  a.Nrows = Nrows;
  a.part = part;
  a.err = ctx->d_status;
  // CTA pairs sharing B tiles need an even number of A tile rows and room for whole pairs
  static int max_pairs = -1;
  const bool mc = KITE_GEMM_MULTICAST && TM % 2 == 0 && ctx->num_sms >= 2;
  static bool attr = false;
  if (!attr) {
    KITE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_gemm_split_bf16<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kGemmSmem));
    KITE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_gemm_split_bf16<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kGemmSmem));
    attr = true;
  }
  CUtensorMap mAh, mAl, mBh, mBl;
  int rc;
  const int bbox = mc ? kBN / 2 : kBN;  // each CTA of a pair loads half of the B tile
  if ((rc = make_map(ctx, &mAh, Ahi, Kp, Mrows, kBM)) != KITE_OK) return rc;
  if ((rc = make_map(ctx, &mAl, Alo, Kp, Mrows, kBM)) != KITE_OK) return rc;
  if ((rc = make_map(ctx, &mBh, Bhi, Kp, Nrows, bbox)) != KITE_OK) return rc;
  if ((rc = make_map(ctx, &mBl, Blo, Kp, Nrows, bbox)) != KITE_OK) return rc;
  if (!mc) {
    const int grid = std::min(a.items, ctx->num_sms);
    k_gemm_split_bf16<false><<<grid, kGemmThreads, kGemmSmem, ctx->stream>>>(mAh, mAl, mBh, mBl, a);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
    return KITE_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kGemmThreads);
  cfg.dynamicSmemBytes = kGemmSmem;
  cfg.stream = ctx->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (max_pairs < 0) {  // pairs that can be resident at once (SMs pair up within a GPC)
    int n = 0;
    cfg.gridDim = dim3((unsigned)(ctx->num_sms & ~1));
    if (cudaOccupancyMaxActiveClusters(&n, k_gemm_split_bf16<true>, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = ctx->num_sms / 2;
    }
    max_pairs = n;
  }
  const int pairs = std::max(1, std::min(a.items / 2, std::min(max_pairs, ctx->num_sms / 2)));
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  KITE_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, k_gemm_split_bf16<true>, mAh, mAl, mBh, mBl, a));
  return KITE_OK;
}

int reduce_cplx(kite_ctx* ctx, const double* part, int S, int M, int M2, double scale,
                double* out, bool accumulate) {
  const int64_t total = (int64_t)M * M2;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8);
  k_reduce_cplx<<<std::max(1, blocks), 256, 0, ctx->stream>>>(part, S, M, M2, scale, out,
                                                               accumulate ? 1 : 0);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

// Generic entry: C[n][m] = scale * sum_i conj(A[n][i]) B[m][i], A [M][N], B [M2][N] complex
// FP32 (device), C [M][M2] complex FP64 (device).
int inner_products_impl(kite_ctx* ctx, const float* A, const float* B, int M, int M2, int64_t N,
                        double scale, double* C, int sub_kb, int fold, int nprod) {
  const int64_t Kp = ((2 * N + kKB - 1) / kKB) * kKB;
  const int Nrows = 2 * M2;
  const int S = plan_gemm_splits(ctx, M, Nrows, Kp);
  const size_t a_bytes = (size_t)M * Kp * 2, b_bytes = (size_t)Nrows * Kp * 2;
  const size_t part_n = (size_t)S * M * Nrows;
  Carver cv(nullptr);
  cv.take<char>(a_bytes);
  cv.take<char>(a_bytes);
  cv.take<char>(b_bytes);
  cv.take<char>(b_bytes);
  cv.take<double>(part_n);
  int rc = ensure_ws(ctx, cv.used());
  if (rc != KITE_OK) return rc;
  Carver w(ctx->ws);
  auto* Ahi = w.take<__nv_bfloat16>((size_t)M * Kp);
  auto* Alo = w.take<__nv_bfloat16>((size_t)M * Kp);
  auto* Bhi = w.take<__nv_bfloat16>((size_t)Nrows * Kp);
  auto* Blo = w.take<__nv_bfloat16>((size_t)Nrows * Kp);
  double* part = w.take<double>(part_n);
  const int blocks = ctx->num_sms * 8;
  // A' = conj-free interleave of a (the conjugation lives in the choice of B rows)
  k_split_rows<<<blocks, 256, 0, ctx->stream>>>(reinterpret_cast<const float2*>(A), M, N, Kp, 0, M, 0, Ahi, Alo);
  k_split_rows<<<blocks, 256, 0, ctx->stream>>>(reinterpret_cast<const float2*>(B), M2, N, Kp, 0, Nrows, 0, Bhi,
                                                Blo);
  k_split_rows<<<blocks, 256, 0, ctx->stream>>>(reinterpret_cast<const float2*>(B), M2, N, Kp, M2, Nrows, 1, Bhi,
                                                Blo);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  int S_used = 0;
  rc = gemm_split_bf16(ctx, Ahi, Alo, Bhi, Blo, M, Nrows, Kp, S, sub_kb, fold, nprod, part, &S_used);
  if (rc != KITE_OK) return rc;
  return reduce_cplx(ctx, part, S_used, M, M2, scale, C, false);
}

}  // namespace kite
