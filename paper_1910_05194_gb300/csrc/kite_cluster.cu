// kite_cluster.cu -- the 1D moment sweep of a small lattice held on chip, one thread-block
// cluster per independent real recursion.
//
// A small lattice (honeycomb 64 x 64 is 8,192 orbitals) gives the streaming step kernels
// one row per CTA, and every step then waits on its own chain: the previous launch's
// completion, bulk copies of three rows from L2 and a CTA reduction -- about 5 us per step
// however few orbitals there are.  Here the whole sweep of Eq. e6 runs in one launch and
// the iterates never leave the chip:
//
//   * For a real symmetric H~ (no magnetic field) the real and imaginary parts of a complex
//     start vector r_0 = a_0 + i b_0 evolve independently, T_n(H~) r_0 = T_n(H~) a_0 +
//     i T_n(H~) b_0, and the moment Re <r_0|r_n> = <a_0|a_n> + <b_0|b_n> (Eqs. e7/e8) is a
//     sum of two real dot products.  The imaginary part, <a_0|T_n b_0> - <b_0|T_n a_0>,
//     vanishes for a symmetric T_n(H~) and is not formed.  Each real recursion (one part
//     of one complex vector, or one real vector: a "lane") is independent of the others.
//   * One cluster of CS CTAs (4 to 16, one CTA per SM) runs one lane.  The CTAs split the
//     lattice's rows; each keeps its rows of r_0, r_{n-1}, r_n and the on-site terms in
//     shared memory for the whole sweep and writes r_{n+1} over r_{n-1} in place (site o's
//     r_{n-1} is read by site o alone).
//   * The neighbour row across a CTA boundary is read straight from the adjacent CTA's
//     shared memory (distributed shared memory), and one cluster barrier per step orders
//     the steps: after it, every CTA's r_{n+1} is complete and visible, and no CTA still
//     reads the r_n that the next step overwrites.
//
// The site update is the streaming kernels' own rounding sequence, component by component
// (s = (n1 + n2) + n3 [+ n4]; r_1 = fma(t~, s, V~ * r_0); r_{n+1} = fma(2t~, s, fma(2V~,
// r_n, -r_{n-1})); vacancies 0), so the iterates are the same bits.  The moment of each step is summed per
// thread over its sites, then over the 32 lanes of a warp by a transpose through shared
// memory every 16 moments (two FP64 adds per moment and thread instead of a shuffle tree),
// and the per-warp sums go to global memory; one small kernel adds them in a fixed order
// (deterministic) and divides by N_eff.
//
// The kernel has no spin-waits: the cluster barrier is a hardware barrier over CTAs that
// the launch guarantees to be co-resident, and every CTA of a cluster passes the same
// number of them.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>

#include "kite_device.cuh"
#include "kite_internal.h"

namespace kite {
namespace {

// 512 threads: one CTA per SM, so the SM's latency hiding (FP64 results, shared and
// distributed shared memory) comes from the warps of this CTA alone
#ifndef KITE_CLUSTER_BLOCK
#define KITE_CLUSTER_BLOCK 512
#endif
constexpr int kCBlock = KITE_CLUSTER_BLOCK;
constexpr int kCWarps = kCBlock / 32;
constexpr int kSlots = 16;     // moments per transpose of a warp's buffer
constexpr int kWbStride = 33;  // doubles per moment row of a warp's transpose buffer (padded)
constexpr int kWbBytes = kCWarps * kSlots * kWbStride * 8;

template <typename Real>
struct CAcc {
  using T = float;
};
template <>
struct CAcc<double> {
  using T = double;
};

__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float dsmem_ld(uint32_t a, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double dsmem_ld(uint32_t a, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
// Every thread of every CTA of the cluster arrives (release) and waits (acquire).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
#ifndef KITE_CLUSTER_SPLIT
#define KITE_CLUSTER_SPLIT 1
#endif

// Rows of CTA c when Ly rows are split over n CTAs as evenly as possible.
__device__ __forceinline__ int rows_of(int c, int Ly, int n) { return Ly / n + (c < Ly % n ? 1 : 0); }
__device__ __forceinline__ int row0_of(int c, int Ly, int n) { return c * (Ly / n) + min(c, Ly % n); }

template <typename Real>
struct ClusterArgs {
  const Real* r0;  // the batch's start vectors, 16-byte chunks, C per orbital
  const Real* vt;  // twice the rescaled on-site term per orbital, NaN at a vacancy
  Real tt;         // rescaled hopping
  int Lx, Ly, C;
  int per_chunk;   // vectors per chunk (complex: 2 FP32 / 1 FP64; real: 4 / 2)
  int realv;       // lanes are whole real vectors (1) or parts of complex ones (0)
  int open_x, open_y;
  int steps;       // recursion steps: r_1 .. r_steps
  int slots;       // moment slots per warp row of `part`
  int rows_max;    // rows of the CTA with the most
  double* part;    // [lane][cta][warp][slots] warp sums of the moment slots (null: not stored)
  Real* last_prev;  // optional: r_{steps-1} and r_steps out, in the start vectors' chunk layout
  Real* last_cur;
};

// MODE 0: slot 0 = <r_0|r_0>, slot n+1 = <r_0|r_{n+1}> from step n.
// MODE 3 (moment doubling): slot 0 = <r_0|r_0>, step n gives slot 2n+1 = <r_n|r_{n+1}> and,
// for n >= 1, slot 2n = <r_n|r_n>.
template <typename Real, int LAT, int MODE>
__global__ void __launch_bounds__(kCBlock, 1) k_cluster_sweep(const ClusterArgs<Real> a) {
  using Acc = typename CAcc<Real>::T;
  constexpr int SORB = LAT == KITE_HONEYCOMB ? 2 : 1;
  constexpr int RPC = 16 / (int)sizeof(Real);  // reals per 16-byte chunk
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t rank, ncta, lane_id;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
  asm("mov.u32 %0, %%clusterid.x;" : "=r"(lane_id));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rowlen = a.Lx * SORB;
  const int cap = a.rows_max * rowlen;
  double* wb = reinterpret_cast<double*>(smem) + warp * kSlots * kWbStride;
  Real* Z = reinterpret_cast<Real*>(smem + kWbBytes);  // r_0 (MODE 0)
  Real* B0 = Z + cap;                                  // r_n for even n
  Real* B1 = B0 + cap;                                 // r_n for odd n
  Real* V = B1 + cap;                                  // on-site terms
  const int n_cta = (int)ncta, me_cta = (int)rank;
  const int nr = rows_of(me_cta, a.Ly, n_cta), y0 = row0_of(me_cta, a.Ly, n_cta);
  const int prev = (me_cta + n_cta - 1) % n_cta, next = (me_cta + 1) % n_cta;
  const int prev_last = rows_of(prev, a.Ly, n_cta) - 1;
  const int v = a.realv ? (int)lane_id : (int)(lane_id >> 1);
  const int comp = a.realv ? 0 : (int)(lane_id & 1);
  const int chunk = v / a.per_chunk;
  const int elem = a.realv ? v % a.per_chunk : 2 * (v % a.per_chunk) + comp;
  const int count = nr * rowlen;

  // moment slots: per-thread values -> a warp's transpose buffer -> per-warp sums
  double* part = a.part ? a.part + (((size_t)lane_id * n_cta + me_cta) * kCWarps + warp) * a.slots : nullptr;
  auto flush = [&](int base, int cnt) {
    __syncwarp();
    if (lane < cnt) {
      const double* row = wb + lane * kWbStride;
      double s = 0.0;
#pragma unroll 8
      for (int i = 0; i < 32; ++i) s += row[i];
      if (part) part[base + lane] = s;
    }
    __syncwarp();
  };
  auto emit = [&](int slot, Acc val) {
    wb[(slot % kSlots) * kWbStride + lane] = (double)val;
    if (slot % kSlots == kSlots - 1) flush(slot - (kSlots - 1), kSlots);
  };

  // this CTA's rows of the lane's r_0 and of the on-site terms
  Acc z2 = Acc(0);
  for (int o = tid; o < count; o += kCBlock) {
    const int64_t g = (int64_t)y0 * rowlen + o;  // orbital index cell * SORB + s
    const Real x = a.r0[(g * a.C + chunk) * RPC + elem];
    Z[o] = x;
    B0[o] = x;
    V[o] = a.vt[g];
    z2 = rfma((Acc)x, (Acc)x, z2);
  }
  emit(0, z2);
  cluster_barrier();  // every CTA's rows are in place before the first remote read

  const uint32_t p0 = cluster_addr(B0, prev), p1 = cluster_addr(B1, prev);
  const uint32_t q0 = cluster_addr(B0, next), q1 = cluster_addr(B1, next);
  const uint32_t prow = (uint32_t)(prev_last * rowlen * (int)sizeof(Real));
  const Real tt2 = a.tt + a.tt;  // exact
  // one recursion step; the first (r_1 = H~ r_0) is its own instance so that the other
  // steps carry no select between the two formulas
  auto step = [&](auto first_tag, int n) {
    constexpr bool FIRST = decltype(first_tag)::value;
    const Real* cur = (n & 1) ? B1 : B0;
    Real* out = (n & 1) ? B0 : B1;
    const uint32_t pc = ((n & 1) ? p1 : p0) + prow, qc = (n & 1) ? q1 : q0;
    // r_n at local row rr (-1: the previous CTA's last row, nr: the next CTA's first row)
    auto at = [&](int rr, int ii) -> Real {
      if (rr < 0) return dsmem_ld(pc + (uint32_t)(ii * (int)sizeof(Real)), Real());
      if (rr >= nr) return dsmem_ld(qc + (uint32_t)(ii * (int)sizeof(Real)), Real());
      return cur[rr * rowlen + ii];
    };
    Acc acc = Acc(0), acc2 = Acc(0);
    // One site in two halves: the loads (neighbour sum, r_n, r_{n-1}, on-site term, r_0),
    // then the arithmetic and the store.  Two sites per thread are loaded before either is
    // stored, so that their shared-memory and FP64 latencies overlap.
    struct In {
      Real sum, me, pv, vo, z;
    };
    auto load = [&](int o) -> In {
      const int r = o / rowlen, i = o - r * rowlen;
      const int y = y0 + r;
      In q;
      q.me = cur[o];
      Real n1, n2, n3, n4 = Real(0);
      if (LAT == KITE_HONEYCOMB) {
        const int x = i >> 1;
        if ((i & 1) == 0) {  // A(x,y) <- B(x,y), B(x+1,y-1), B(x,y-1)
          const bool cut = a.open_y && y == 0;
          const int xp = x + 1 == a.Lx ? 0 : x + 1;
          n1 = cur[o + 1];
          n2 = (cut || (a.open_x && x + 1 == a.Lx)) ? Real(0) : at(r - 1, 2 * xp + 1);
          n3 = cut ? Real(0) : at(r - 1, 2 * x + 1);
        } else {  // B(x,y) <- A(x,y), A(x-1,y+1), A(x,y+1)
          const bool cut = a.open_y && y == a.Ly - 1;
          const int xm = x == 0 ? a.Lx - 1 : x - 1;
          n1 = cur[o - 1];
          n2 = (cut || (a.open_x && x == 0)) ? Real(0) : at(r + 1, 2 * xm);
          n3 = cut ? Real(0) : at(r + 1, 2 * x);
        }
      } else {  // (x-1,y), (x+1,y), (x,y-1), (x,y+1)
        const int x = i;
        const int xm = x == 0 ? a.Lx - 1 : x - 1, xp = x + 1 == a.Lx ? 0 : x + 1;
        n1 = (a.open_x && x == 0) ? Real(0) : cur[r * rowlen + xm];
        n2 = (a.open_x && x + 1 == a.Lx) ? Real(0) : cur[r * rowlen + xp];
        n3 = (a.open_y && y == 0) ? Real(0) : at(r - 1, x);
        n4 = (a.open_y && y == a.Ly - 1) ? Real(0) : at(r + 1, x);
      }
      q.sum = radd(n1, n2);
      q.sum = radd(q.sum, n3);
      if (LAT == KITE_SQUARE) q.sum = radd(q.sum, n4);
      q.vo = V[o];
      q.pv = FIRST ? Real(0) : out[o];
      q.z = MODE == 0 ? Z[o] : Real(0);
      return q;
    };
    auto finish = [&](int o, const In& q) {
      // r_1 = t~ s + V~ r_0; r_{n+1} = 2t~ s + (2V~ r_n - r_{n-1}) (V holds 2V~)
      const Real nx = FIRST ? rfma(a.tt, q.sum, rmul(Real(0.5) * q.vo, q.me))
                            : rfma(tt2, q.sum, rfma(q.vo, q.me, -q.pv));
      const Real w = is_vacancy(q.vo) ? Real(0) : nx;
      out[o] = w;
      if (MODE == 0) {
        acc = rfma((Acc)q.z, (Acc)w, acc);
      } else {
        acc = rfma((Acc)q.me, (Acc)w, acc);
        if (!FIRST) acc2 = rfma((Acc)q.me, (Acc)q.me, acc2);  // <r_0|r_0> is slot 0 already
      }
    };
    // sites f(k) for k = tid, tid + kCBlock, ... < cnt, two at a time
    auto sweep = [&](int cnt, auto f) {
      int k = tid;
      for (; k + kCBlock < cnt; k += 2 * kCBlock) {
        const int o1 = f(k), o2 = f(k + kCBlock);
        const In q1 = load(o1);
        const In q2 = load(o2);
        finish(o1, q1);
        finish(o2, q2);
      }
      if (k < cnt) {
        const int o1 = f(k);
        finish(o1, load(o1));
      }
    };
#if KITE_CLUSTER_SPLIT
    // The first and last rows (the only ones the neighbours read, and the only ones that
    // read theirs) first; then arrive on the cluster barrier and update the interior rows
    // while the other CTAs catch up.  The CTA barrier before the wait makes the interior
    // rows, written after the arrival, complete for this CTA's own next step.
    const int nb = (nr == 1 ? 1 : 2) * rowlen;
    sweep(nb, [&](int k) { return k < rowlen ? k : (nr - 1) * rowlen + (k - rowlen); });
    cluster_arrive();
    sweep((nr - 2) * rowlen, [&](int k) { return rowlen + k; });
#else
    sweep(count, [&](int k) { return k; });
#endif
    if (MODE == 0) {
      emit(n + 1, acc);
    } else {
      if (n > 0) emit(2 * n, acc2);
      emit(2 * n + 1, acc);
    }
#if KITE_CLUSTER_SPLIT
    __syncthreads();
    cluster_wait();  // r_{n+1} complete everywhere; nobody reads r_n any more
#else
    cluster_barrier();  // r_{n+1} complete everywhere; nobody reads r_n any more
#endif
  };
  if (a.steps > 0) step(std::true_type{}, 0);
  for (int n = 1; n < a.steps; ++n) step(std::false_type{}, n);
  const int last = MODE == 0 ? a.steps : (a.steps > 0 ? 2 * a.steps - 1 : 0);
  if (last % kSlots != kSlots - 1) flush(last - last % kSlots, last % kSlots + 1);
  if (a.last_cur) {  // the last two iterates (after the final barrier: nothing writes them)
    const Real* rc = (a.steps & 1) ? B1 : B0;
    const Real* rp = a.steps == 0 ? B0 : (((a.steps - 1) & 1) ? B1 : B0);
    for (int o = tid; o < count; o += kCBlock) {
      const size_t q = (size_t)(((int64_t)y0 * rowlen + o) * a.C + chunk) * RPC + elem;
      a.last_prev[q] = rp[o];
      a.last_cur[q] = rc[o];
    }
  }
}

// mu_vec[(vec_base + v)][n] = (sum over the vector's lanes, CTAs and warps of slot n) / N_eff;
// with doubling, mu_n = 2 slot_n - slot_(n mod 2) for n >= 2.  One block per (vector, n):
// the FP64 adds are spread over the whole GPU (a thread per moment would leave them on a
// few SMs of GB300's narrow FP64 pipe).  Fixed order: thread t adds terms t, t + 128, ...,
// then a fixed butterfly within each warp and the four warp sums in order.
constexpr int kRedBlock = 128;
__global__ void __launch_bounds__(kRedBlock) k_cluster_reduce(const double* __restrict__ part, int lanes_per_vec,
                                                              int ncta, int slots, int M, int doubling, int vec_base,
                                                              const unsigned long long* __restrict__ n_eff,
                                                              double* __restrict__ mu_vec) {
  __shared__ double wsum[2][kRedBlock / 32];
  const int v = blockIdx.y, n = blockIdx.x;
  const int per_lane = ncta * kCWarps, terms = lanes_per_vec * per_lane;
  const double* base = part + (size_t)v * terms * slots;  // the vector's lanes are adjacent
  const bool two = doubling && n >= 2;
  double s0 = 0.0, s1 = 0.0;
  for (int g = threadIdx.x; g < terms; g += kRedBlock) {
    s0 += base[(size_t)g * slots + n];
    if (two) s1 += base[(size_t)g * slots + (n & 1)];
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, d);
    s1 += __shfl_xor_sync(0xffffffffu, s1, d);
  }
  if ((threadIdx.x & 31) == 0) {
    wsum[0][threadIdx.x >> 5] = s0;
    wsum[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kRedBlock / 32; ++w) a += wsum[0][w], b += wsum[1][w];
    const double sum = two ? 2.0 * a - b : a;
    const double ne = (double)*n_eff;
    double* out = mu_vec + ((size_t)(vec_base + v) * M + n) * 2;
    out[0] = ne > 0.0 ? sum / ne : 0.0;
    out[1] = 0.0;
  }
}

template <typename Real, int LAT, int MODE>
const void* sweep_kernel() {
  return reinterpret_cast<const void*>(&k_cluster_sweep<Real, LAT, MODE>);
}

const void* kernel_for(int fp64, int lattice, int doubling) {
  if (fp64) {
    if (lattice == KITE_HONEYCOMB)
      return doubling ? sweep_kernel<double, KITE_HONEYCOMB, 3>() : sweep_kernel<double, KITE_HONEYCOMB, 0>();
    return doubling ? sweep_kernel<double, KITE_SQUARE, 3>() : sweep_kernel<double, KITE_SQUARE, 0>();
  }
  if (lattice == KITE_HONEYCOMB)
    return doubling ? sweep_kernel<float, KITE_HONEYCOMB, 3>() : sweep_kernel<float, KITE_HONEYCOMB, 0>();
  return doubling ? sweep_kernel<float, KITE_SQUARE, 3>() : sweep_kernel<float, KITE_SQUARE, 0>();
}

int round32(int x) { return (x + 31) & ~31; }

}  // namespace

int cluster_smem(const ClusterSweep& a, int cs) {
  if (cs < 2 || a.Ly < cs || a.Lx < 1) return 0;
  const int sorb = a.lattice == KITE_HONEYCOMB ? 2 : 1;
  const int rows_max = (a.Ly + cs - 1) / cs;
  const size_t real = a.fp64 ? 8 : 4;
  const size_t need = kWbBytes + 4 * (size_t)rows_max * a.Lx * sorb * real;
  return need <= 227u * 1024u ? (int)need : 0;
}

size_t cluster_part_doubles(int lanes, int cs, int M, int doubling, int timing_steps) {
  const int steps = doubling ? (M + 1) / 2 : M - 1;
  const int last = std::max({doubling ? 2 * steps : steps + 1, 2 * timing_steps, 1});
  return (size_t)lanes * cs * kCWarps * round32(last);
}

namespace {

// Launch shape of cluster size cs: more than half of an SM's shared memory keeps one CTA
// per SM (each CTA gets a whole SM's FP64 pipe).  Returns false if the lattice does not fit.
bool cluster_config(kite_ctx* ctx, const ClusterSweep& a, int cs, cudaLaunchConfig_t* cfg,
                    cudaLaunchAttribute* attr, const void** fn) {
  const int need = cluster_smem(a, cs);
  if (need == 0) return false;
  int per_sm = 0;
  if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device) != cudaSuccess)
    return false;
  const int smem = std::min(227 * 1024, std::max(need, per_sm / 2 + 1024));
  *fn = kernel_for(a.fp64, a.lattice, a.doubling);
  {
    // the kernel attributes once per kernel and device (the shared-memory limit at its
    // maximum: the launch's own request decides the occupancy)
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    if (!done.count({*fn, ctx->device})) {
      if (cudaFuncSetAttribute(*fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess ||
          cudaFuncSetAttribute(*fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return false;
      done.insert({*fn, ctx->device});
    }
  }
  const int lanes = a.realv ? a.nvec : 2 * a.nvec;
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3((unsigned)(lanes * cs), 1, 1);
  cfg->blockDim = dim3(kCBlock, 1, 1);
  cfg->dynamicSmemBytes = (size_t)smem;
  cfg->stream = ctx->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  return true;
}

}  // namespace

int cluster_active(kite_ctx* ctx, const ClusterSweep& a, int cs) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  const void* fn = nullptr;
  if (!cluster_config(ctx, a, cs, &cfg, attr, &fn)) {
    cudaGetLastError();
    return 0;
  }
  // resident clusters of this kernel, size and shared memory, cached per device
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, int> cache;
  const auto key = std::make_tuple(fn, ctx->device, cs, cfg.dynamicSmemBytes);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int active = 0;
  if (cudaOccupancyMaxActiveClusters(&active, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = active;
  }
  return active;
}

int cluster_sweep(kite_ctx* ctx, ClusterSweep* a, int timing_steps) {
  const int sorb = a->lattice == KITE_HONEYCOMB ? 2 : 1;
  const int cs = a->cs;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  const void* fn = nullptr;
  if (!cluster_config(ctx, *a, cs, &cfg, attr, &fn) || cluster_active(ctx, *a, cs) < 1)
    return fail(ctx, KITE_ERR_ARG, "cluster sweep: no cluster of this size fits the lattice and the GPU");
  const int lanes = a->realv ? a->nvec : 2 * a->nvec;
  const int steps = timing_steps > 0 ? timing_steps : (a->doubling ? (a->M + 1) / 2 : a->M - 1);
  const int last = a->doubling ? (steps > 0 ? 2 * steps - 1 : 0) : steps;
  const int slots = round32(last + 1);
  auto launch = [&](auto real_tag, double* part) -> cudaError_t {
    using Real = decltype(real_tag);
    ClusterArgs<Real> args;
    args.r0 = static_cast<const Real*>(a->r0);
    args.vt = static_cast<const Real*>(a->vt);
    args.tt = (Real)a->tt;
    args.Lx = a->Lx;
    args.Ly = a->Ly;
    args.C = a->C;
    args.per_chunk = a->per_chunk;
    args.realv = a->realv;
    args.open_x = a->open_x;
    args.open_y = a->open_y;
    args.steps = steps;
    args.slots = slots;
    args.rows_max = (a->Ly + cs - 1) / cs;
    args.part = part;
    args.last_prev = timing_steps > 0 ? nullptr : static_cast<Real*>(a->last_prev);
    args.last_cur = timing_steps > 0 ? nullptr : static_cast<Real*>(a->last_cur);
    void* kargs[] = {&args};
    return cudaLaunchKernelExC(&cfg, fn, kargs);
  };
  double* part = timing_steps > 0 ? nullptr : a->part;
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, ctx->stream));
  KITE_CUDA_TRY(ctx, a->fp64 ? launch(double(), part) : launch(float(), part));
  KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, ctx->stream));
  if (timing_steps == 0) {
    k_cluster_reduce<<<dim3((unsigned)a->M, (unsigned)a->nvec), kRedBlock, 0, ctx->stream>>>(
        a->part, a->realv ? 1 : 2, cs, slots, a->M, a->doubling, a->vec_base, a->n_eff, a->mu_vec);
    KITE_CUDA_TRY(ctx, cudaGetLastError());
  }
  float ms = 0.f;
  KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
  KITE_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev2, ctx->ev3));
  a->seconds = 1e-3 * ms;
  a->grid = lanes * cs;
  // bytes to and from device memory: each lane's part of r_0 and the on-site terms in, the
  // per-warp moment sums out
  const double n_orb = (double)a->Lx * a->Ly * sorb;
  a->bytes = lanes * n_orb * (a->fp64 ? 16.0 : 8.0) + (double)lanes * cs * kCWarps * slots * 8.0;
  return KITE_OK;
}

}  // namespace kite
