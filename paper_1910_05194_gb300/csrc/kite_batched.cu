// kite_batched.cu -- many independent systems in one persistent, graph-captured launch.
//
// The cost of the DOS path is Z*N*M*R*S (Eq. PcomplexityFactor); independent disorder
// realisations and lattices of uneven size are the natural unit of batching.  The host
// groups the persistent grid's CTAs into teams: a system whose work N*M exceeds the
// target share gets a team of several CTAs that split its rows and meet at a global
// barrier after every recursion step; smaller systems are packed first-fit-decreasing
// into single-CTA teams that run them one after another.  Every CTA of the grid is
// resident at once (cooperative launch), every barrier wait is bounded, and the whole
// batch -- on-site draws, start vectors, the persistent sweep and the fixed-order moment
// reductions -- is captured into one CUDA graph and launched once.
#include <stdlib.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "kite_step.cuh"
#include "kite_step2.cuh"

namespace kite {
namespace {

struct BSys {
  const void* r0;
  void* bA;
  void* bB;
  void* bC;  // two more iterate buffers for the two-step pass (null without it)
  void* bD;
  const float* vt;
  const float* phase;  // Peierls phases [Ly][sublattice][2 bonds][cos, sin] (field batches)
  double* partial;  // [max(M,2)][ncta][Q]
  float tt;
  int Lx, Ly, M;
  long long units;
};

struct BTeam {
  int cta0, ncta;  // CTAs [cta0, cta0 + ncta)
  int sys0, nsys;  // systems order[sys0 .. sys0 + nsys)
};

// Arrive-and-wait of the CTAs of one team (counter counts arrivals monotonically).  The
// writes of this step were made by generic stores; the next step reads them with bulk
// copies, hence the proxy fences around the release/acquire pair.
__device__ __forceinline__ bool team_barrier(unsigned int* ctr, unsigned int target, bool skip_arrive,
                                             int* err, int* abort_flag) {
  asm volatile("fence.proxy.async.global;" ::: "memory");  // each thread's own stores
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (!skip_arrive) atomicAdd(ctr, 1u);
    const long long t0 = clock64();
    for (;;) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if ((int)(v - target) >= 0) break;
      if (clock64() - t0 > kWaitCycles) {
        *abort_flag = 1;
        atomicExch(err, 1);
        break;
      }
      __nanosleep(64);
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();
  return *abort_flag == 0;
}

// DBL: moment doubling for the whole batch (two moments per step, r_0 not re-read):
// step 0 writes <r_0|r_0>, <r_0|r_1> into slots 0, 1; step n >= 1 writes <r_n|r_n>,
// <r_n|r_{n+1}> into slots 2n, 2n+1; k_breduce turns slots into moments.
// NST: ring depth.  mcap > 0 caps every system's steps (the autotuner's probe launches).
// FIELD: a batch with a magnetic field in any system runs the stencil's Peierls variant for
// all of them (a system without a field has the phase table of flux 0: rotations by
// (1, 0), which leave every value unchanged).
template <int LAT, int C, bool DBL, int NST, bool FIELD = false>
__global__ void __launch_bounds__(kBlock, 3)  // <= 85 registers: three CTAs fit when the stages do
    k_batched(const BSys* __restrict__ systems, const BTeam* __restrict__ teams,
              const int* __restrict__ order, const int* __restrict__ cta_team,
              unsigned int* __restrict__ counters, int* __restrict__ err, int stall, int mcap) {
  constexpr int Q = 2 * C * 2;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  Ring ring{bars, smem + kBarBytes, &s_abort, 0};
  const int team = cta_team[blockIdx.x];
  const BTeam T = teams[team];
  const int rank = blockIdx.x - T.cta0;
  unsigned int arrived = 0;
  const FamOut nofam{};
  for (int i = 0; i < T.nsys; ++i) {
    const BSys S = systems[order[T.sys0 + i]];
    auto where = [&](int n) -> void* {
      return n == 0 ? const_cast<void*>(S.r0) : ((n & 1) ? S.bA : S.bB);
    };
    constexpr int MODE = DBL ? 3 : 0;
    const int full = DBL ? (S.M + 1) / 2 : max(S.M - 1, 1);
    const int steps = mcap > 0 ? min(full, mcap) : full;
    for (int n = 0; n < steps; ++n) {
      bool ok;
      if (n == 0)
        ok = step_body<float, LAT, C, true, MODE, NST, FIELD>(ring, rank, T.ncta, nullptr, S.r0, S.bA, S.r0,
                                                         S.vt, S.tt, S.Lx, S.Ly, S.units,
                                                         S.partial + (size_t)T.ncta * Q, S.partial, err, 0,
                                                         nofam, 0, SeriesOut{}, S.phase);
      else if (DBL)
        ok = step_body<float, LAT, C, false, MODE, NST, FIELD>(ring, rank, T.ncta, where(n - 1), where(n),
                                                          where(n + 1), S.r0, S.vt, S.tt, S.Lx, S.Ly, S.units,
                                                          S.partial + (size_t)(2 * n + 1) * T.ncta * Q,
                                                          S.partial + (size_t)(2 * n) * T.ncta * Q, err, 0,
                                                          nofam, 0, SeriesOut{}, S.phase);
      else
        ok = step_body<float, LAT, C, false, MODE, NST, FIELD>(ring, rank, T.ncta, where(n - 1), where(n),
                                                          where(n + 1), S.r0, S.vt, S.tt, S.Lx, S.Ly, S.units,
                                                          S.partial + (size_t)(n + 1) * T.ncta * Q, nullptr,
                                                          err, 0, nofam, 0, SeriesOut{}, S.phase);
      if (!ok) return;
      // step_body reused the ring's shared memory for its reduction (generic-proxy
      // writes); order them before the next step's bulk copies into the same memory
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (T.ncta > 1) {
        arrived += (unsigned int)T.ncta;
        const bool skip = stall && team == 0 && rank == 0 && arrived == (unsigned int)T.ncta;
        if (!team_barrier(counters + team, arrived, skip, err, &s_abort)) return;
      } else {
        // a single-CTA team reads its own previous step through the async proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
      }
    }
  }
}

// The batched sweep with temporal blocking (no field), after a one-step launch of k_batched
// has written every system's r_1 (and the moment slots 0, 1): passes of two steps (r_{n-1},
// r_n) -> (r_{n+1}, r_{n+2}) with the moments n+1, n+2 -- or, with doubling, the slots
// 2n .. 2n+3 -- (the two-step body of kite_step2.cuh) and a team barrier after each.  When
// r_1 .. r_last leaves an odd step, the last pass also computes r_{last+1} (its moment slots
// lie past M - 1, unread), so the kernel holds the two-step body alone.
// Iterate k >= 1 lives in buffer k mod 4 so that a pass's outputs never alias its inputs.
template <int LAT, int C, int NST, bool DBL = false>
struct Batched2Shape {
  static constexpr int SMEM = Step2Shape<LAT, C, NST, DBL, true>::SMEM;
};

// Three CTAs per SM (72 registers): the per-system state that the persistent loop carries
// around the pass costs registers that the one-launch-per-pass kernel takes from its
// parameters, so the pass keeps its FP64 moment sums in shared memory (SMACC).  Measured
// on the 256-system square-lattice batch: 2.46e11 updates/s (2.30e11 at two CTAs per SM;
// 1.35e11 at three with the sums in registers, which spilled).
#ifndef KITE_BATCHED2_MIN_CTAS
#define KITE_BATCHED2_MIN_CTAS 3
#endif
template <int LAT, int C, int NST, bool DBL = false>
__global__ void __launch_bounds__(kBlock2, KITE_BATCHED2_MIN_CTAS)
    k_batched2(const BSys* __restrict__ systems, const BTeam* __restrict__ teams,
               const int* __restrict__ order, const int* __restrict__ cta_team,
               unsigned int* __restrict__ counters, int* __restrict__ err, int stall, int mcap) {
  constexpr int Q = 2 * C * 2;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  Ring ring{bars, smem + kBarBytes, &s_abort, 0};
  const int team = cta_team[blockIdx.x];
  const BTeam T = teams[team];
  const int rank = blockIdx.x - T.cta0;
  unsigned int arrived = 0;
  auto sync_team = [&]() -> bool {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (T.ncta > 1) {
      arrived += (unsigned int)T.ncta;
      const bool skip = stall && team == 0 && rank == 0 && arrived == (unsigned int)T.ncta;
      return team_barrier(counters + team, arrived, skip, err, &s_abort);
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    return true;
  };
  for (int i = 0; i < T.nsys; ++i) {
    const BSys S = systems[order[T.sys0 + i]];
    void* const bufs[4] = {S.bC, S.bA, S.bB, S.bD};
    auto w4 = [&](int n) -> void* { return n == 0 ? const_cast<void*>(S.r0) : bufs[n & 3]; };
    auto slot = [&](int k) { return S.partial + (size_t)k * T.ncta * Q; };
    const int full = DBL ? (S.M + 1) / 2 : max(S.M - 1, 1);
    const int last = mcap > 0 ? min(full, mcap) : full;  // iterates r_1 .. r_last
    for (int n = 1; n + 1 <= last; n += 2) {
      // plain: moments n+1, n+2; doubling: slots 2n .. 2n+3 (<r_n|r_n>, <r_n|r_{n+1}>, ...)
      const bool ok = DBL ? step2_body<float, LAT, C, NST, true>(ring, rank, T.ncta, w4(n - 1), w4(n), w4(n + 1),
                                                                 w4(n + 2), nullptr, S.vt, S.tt, S.Lx, S.Ly,
                                                                 S.units, slot(2 * n), slot(2 * n + 1), err, 0,
                                                                 slot(2 * n + 2), slot(2 * n + 3))
                          : step2_body<float, LAT, C, NST, false, true>(
                                ring, rank, T.ncta, w4(n - 1), w4(n), w4(n + 1), w4(n + 2), S.r0, S.vt, S.tt,
                                S.Lx, S.Ly, S.units, slot(n + 1), slot(n + 2), err, 0);
      if (!ok) return;
      if (!sync_team()) return;
    }
  }
}

// mean over the vectors of slot k's real part, CTA partials summed in fixed order
__device__ double slot_mean(const double* __restrict__ partial, int k, int G, int Q, int nvec, double ne) {
  double acc = 0.0;
  for (int q = 0; q < 2 * nvec; q += 2) {  // real parts, vector by vector, CTA by CTA
    double sum = 0.0;
    const double* p = partial + (size_t)k * G * Q + q;
    for (int g = 0; g < G; ++g) sum += p[(size_t)g * Q];
    acc += ne > 0.0 ? sum / ne : 0.0;
  }
  return acc / nvec;
}

// mu_n from the slots; with doubling mu_n = 2 slot_n - slot_(n mod 2) for n >= 2
__global__ void k_breduce(const double* __restrict__ partial, int M, int G, int Q, int nvec, int dbl,
                          const unsigned long long* __restrict__ n_eff, double* __restrict__ mu) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  const double ne = (double)*n_eff;
  const double v = slot_mean(partial, n, G, Q, nvec, ne);
  mu[n] = (dbl && n >= 2) ? 2.0 * v - slot_mean(partial, n & 1, G, Q, nvec, ne) : v;
}

inline bool autotune_enabled_batched() {
  const char* e = getenv("KITE_AUTOTUNE");
  return !(e && e[0] == '0');
}

struct Schedule {
  std::vector<BTeam> teams;
  std::vector<int> order, cta_team, ncta_of;
  int grid = 0;
};

// Teams for a target per-CTA work T: systems above T get ceil(W/T) CTAs (at most one per
// unit of work), the rest are packed first-fit-decreasing into single-CTA bins.
Schedule plan_teams(const std::vector<double>& work, const std::vector<long long>& units, double T) {
  Schedule sc;
  const int n = (int)work.size();
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return work[a] > work[b]; });
  sc.ncta_of.assign(n, 1);
  std::vector<std::vector<int>> bins;
  std::vector<double> load;
  for (int i : idx) {
    if (work[i] >= T) {
      const int c = (int)std::min<long long>(units[i], (long long)std::ceil(work[i] / T));
      sc.ncta_of[i] = std::max(1, c);
      BTeam t{sc.grid, sc.ncta_of[i], (int)sc.order.size(), 1};
      sc.order.push_back(i);
      sc.teams.push_back(t);
      sc.grid += t.ncta;
    } else {
      size_t b = 0;
      for (; b < bins.size(); ++b)
        if (load[b] + work[i] <= T) break;
      if (b == bins.size()) {
        bins.emplace_back();
        load.push_back(0.0);
      }
      bins[b].push_back(i);
      load[b] += work[i];
    }
  }
  for (auto& bin : bins) {
    BTeam t{sc.grid, 1, (int)sc.order.size(), (int)bin.size()};
    for (int i : bin) sc.order.push_back(i);
    sc.teams.push_back(t);
    sc.grid += 1;
  }
  sc.cta_team.resize(sc.grid);
  for (int t = 0; t < (int)sc.teams.size(); ++t)
    for (int k = 0; k < sc.teams[t].ncta; ++k) sc.cta_team[sc.teams[t].cta0 + k] = t;
  return sc;
}

// One candidate of the batched launch: ring depth, resident CTAs per SM, and the team
// schedule that fits that grid.
struct BPlan {
  int nst = kStages, k = 0;
  int two = 0;  // 1: the two-step kernel (k_batched2)
  Schedule sc;
};

// KITE_PASS_STEPS=1 or 2 pins one or two recursion steps per pass (as for kite_moments_1d)
inline int batched_pass_steps_pinned() {
  const char* e = getenv("KITE_PASS_STEPS");
  return (e && (e[0] == '1' || e[0] == '2') && e[1] == 0) ? e[0] - '0' : 0;
}

template <int LAT, int C, int NST, bool DBL = false>
int batched2_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    constexpr int SMEM = Batched2Shape<LAT, C, NST, DBL>::SMEM;
    int o = 0;
    if (SMEM > 227 * 1024 ||
        cudaFuncSetAttribute(k_batched2<LAT, C, NST, DBL>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batched2<LAT, C, NST, DBL>, kBlock2, SMEM) !=
            cudaSuccess)
      o = 0;
    cudaGetLastError();
    occ = o;
  }
  return occ;
}

template <int LAT, int C, bool DBL, int NST, bool FIELD>
int batched_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    constexpr int SMEM = StepShape<LAT, C, NST>::template smem_bytes<DBL ? 3 : 0>();
    cudaFuncSetAttribute(k_batched<LAT, C, DBL, NST, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batched<LAT, C, DBL, NST, FIELD>, kBlock, SMEM) !=
        cudaSuccess)
      o = 0;
    occ = o;
  }
  return occ;
}

// smallest target share whose schedule fits `gmax` resident CTAs
inline Schedule fit_schedule(const std::vector<double>& work, const std::vector<long long>& units, int gmax) {
  double total = 0.0, wmax = 0.0;
  for (double w : work) total += w, wmax = std::max(wmax, w);
  double lo = total / gmax, hi = std::max(total, wmax) * 1.0001;
  Schedule sc = plan_teams(work, units, hi);
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    Schedule s2 = plan_teams(work, units, mid);
    if (s2.grid <= gmax) {
      hi = mid;
      sc = std::move(s2);
    } else {
      lo = mid;
    }
  }
  return sc;
}

template <int LAT, int C, bool DBL, bool FIELD>
cudaError_t launch_batched(kite_ctx* ctx, const BPlan& pl, const BSys* d_sys, const BTeam* d_teams,
                           const int* d_ints, unsigned int* counters, int stall, int mcap) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.sc.grid);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int* cta_team = d_ints + pl.sc.order.size();
  if constexpr (!FIELD) {
    if (pl.two) {
      // every system's first step with the one-step kernel (capped at one step), then the
      // passes; the team barrier counters start again from zero
      cfg.dynamicSmemBytes = StepShape<LAT, C, 4>::template smem_bytes<DBL ? 3 : 0>();
      cudaError_t ce = cudaLaunchKernelEx(&cfg, k_batched<LAT, C, DBL, 4, false>, d_sys, d_teams, d_ints, cta_team,
                                          counters, ctx->d_status, stall, 1);
      if (ce == cudaSuccess)
        ce = cudaMemsetAsync(counters, 0, sizeof(unsigned int) * pl.sc.teams.size(), ctx->stream);
      if (ce != cudaSuccess) return ce;
      cfg.blockDim = dim3(kBlock2);
      auto go = [&](auto nst) {
        constexpr int NST = decltype(nst)::value;
        cfg.dynamicSmemBytes = Batched2Shape<LAT, C, NST, DBL>::SMEM;
        return cudaLaunchKernelEx(&cfg, k_batched2<LAT, C, NST, DBL>, d_sys, d_teams, d_ints, cta_team, counters,
                                  ctx->d_status, 0, mcap);
      };
      return pl.nst == 5   ? go(std::integral_constant<int, 5>{})
             : pl.nst == 6 ? go(std::integral_constant<int, 6>{})
                           : go(std::integral_constant<int, 8>{});
    }
  }
  if (pl.nst == 4) {
    cfg.dynamicSmemBytes = StepShape<LAT, C, 4>::template smem_bytes<DBL ? 3 : 0>();
    return cudaLaunchKernelEx(&cfg, k_batched<LAT, C, DBL, 4, FIELD>, d_sys, d_teams, d_ints, cta_team, counters,
                              ctx->d_status, stall, mcap);
  }
  cfg.dynamicSmemBytes = StepShape<LAT, C, 8>::template smem_bytes<DBL ? 3 : 0>();
  return cudaLaunchKernelEx(&cfg, k_batched<LAT, C, DBL, 8, FIELD>, d_sys, d_teams, d_ints, cta_team, counters,
                            ctx->d_status, stall, mcap);
}

template <int LAT, int C, bool DBL, bool FIELD>
int run_batched(kite_ctx* ctx, int count, const kite_system* sys, const kite_kpm* kpm,
                const std::vector<Scale>& scales, double* const* mu_out, kite_stats* stats) {
  constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  constexpr int Q = 2 * C * 2;
  using Sh = StepShape<LAT, C>;  // TX and cell sizes do not depend on the ring depth
  cudaStream_t st = ctx->stream;
  const int R = kpm[0].R;
  auto steps_of = [](int M) { return DBL ? (M + 1) / 2 : std::max(M - 1, 1); };
  std::vector<double> work(count);
  std::vector<long long> units(count);
  double total = 0.0;
  for (int i = 0; i < count; ++i) {
    units[i] = (long long)((sys[i].Lx + Sh::TX - 1) / Sh::TX) * sys[i].Ly;
    work[i] = (double)units[i] * Sh::TX * steps_of(kpm[i].M);
    total += work[i];
  }
  // candidate plans: every (ring depth, CTAs per SM) whose grid is resident
  std::vector<BPlan> cands;
  const int occ8 = batched_occupancy<LAT, C, DBL, 8, FIELD>(), occ4 = batched_occupancy<LAT, C, DBL, 4, FIELD>();
  if (occ8 < 1 && occ4 < 1) return fail(ctx, KITE_ERR_CUDA, "occupancy query for the batched kernel failed");
  const bool tune = autotune_enabled_batched() && count > 1;
  const int pin = batched_pass_steps_pinned();
  // the two-step kernel: no field, every system with M >= 4 (doubling: M >= 5)
  bool two_ok = !FIELD && pin != 1;
  for (int i = 0; i < count; ++i) two_ok = two_ok && kpm[i].M >= (DBL ? 5 : 4);
  if (pin != 2 || !two_ok) {
    for (int nst : {8, 4}) {
      const int occ = nst == 8 ? occ8 : occ4;
      for (int k = tune ? 1 : occ; k <= occ; ++k) {
        if (!tune && nst == 4) break;
        BPlan pl;
        pl.nst = nst;
        pl.k = k;
        pl.sc = fit_schedule(work, units, ctx->num_sms * k);
        cands.push_back(std::move(pl));
      }
    }
  }
  if (two_ok && (tune || pin == 2)) {
    for (int nst : {8, 6, 5}) {
      const int occ = nst == 8 ? batched2_occupancy<LAT, C, 8, DBL>()
                               : (nst == 6 ? batched2_occupancy<LAT, C, 6, DBL>() : batched2_occupancy<LAT, C, 5, DBL>());
      // (the first-step launch runs the one-step kernel with four stages on the same grid)
      for (int k = std::min(2, occ); k <= std::min(occ, occ4); ++k) {
        BPlan pl;
        pl.nst = nst;
        pl.k = k;
        pl.two = 1;
        pl.sc = fit_schedule(work, units, ctx->num_sms * k);
        cands.push_back(std::move(pl));
      }
    }
  }
  if (cands.empty()) return fail(ctx, KITE_ERR_CUDA, "no launch configuration of the batched kernel fits");
  const bool has_two = std::any_of(cands.begin(), cands.end(), [](const BPlan& p) { return p.two != 0; });
  // work space: per system vt, three vector buffers, partials for the widest team any
  // candidate gives it, then counters and the schedule tables of the largest candidate
  std::vector<int> max_ncta(count, 1);
  size_t max_teams = 1, max_ints = 1;
  for (const BPlan& pl : cands) {
    for (int i = 0; i < count; ++i) max_ncta[i] = std::max(max_ncta[i], pl.sc.ncta_of[i]);
    max_teams = std::max(max_teams, pl.sc.teams.size());
    max_ints = std::max(max_ints, pl.sc.order.size() + pl.sc.cta_team.size());
  }
  std::vector<size_t> off_vt(count), off_vec(count), off_part(count), off_ph(count, 0);
  auto lay = [&](Carver& k, bool record) {
    for (int i = 0; i < count; ++i) {
      const int64_t ncell = (int64_t)sys[i].Lx * sys[i].Ly, N = ncell * SORB;
      const size_t vb = (size_t)ncell * SORB * C * 16;
      char* a = k.take<char>(sizeof(float) * N);
      if (FIELD) {
        char* ph = k.take<char>(sizeof(float) * (size_t)sys[i].Ly * SORB * 4);
        if (record) off_ph[i] = (size_t)ph;
      }
      char* b = k.take<char>((has_two ? 5 : 3) * vb);
      // (the two-step doubling pass may write slots up to M + 2)
      char* c = k.take<char>(sizeof(double) * (size_t)(std::max(kpm[i].M, 2) + 3) * max_ncta[i] * Q);
      if (record) {
        off_vt[i] = (size_t)a;
        off_vec[i] = (size_t)b;
        off_part[i] = (size_t)c;
      }
    }
  };
  size_t mu_total = 0;
  for (int i = 0; i < count; ++i) mu_total += (size_t)kpm[i].M;
  auto tail = [&](Carver& k) {
    k.take<unsigned long long>(count);  // n_eff
    k.take<unsigned int>(max_teams);    // barrier counters
    k.take<BSys>(count);
    k.take<BTeam>(max_teams);
    k.take<int>(max_ints);
    k.take<double>(mu_total);
  };
  Carver probe(nullptr);
  lay(probe, false);
  tail(probe);
  int rc = ensure_ws(ctx, probe.used());
  if (rc != KITE_OK) return rc;
  Carver w(ctx->ws);
  lay(w, true);
  auto* ne = w.take<unsigned long long>(count);
  auto* counters = w.take<unsigned int>(max_teams);
  auto* d_sys = w.take<BSys>(count);
  auto* d_teams = w.take<BTeam>(max_teams);
  auto* d_ints = w.take<int>(max_ints);
  auto* d_mu = w.take<double>(mu_total);

  std::vector<BSys> hs(count);
  std::vector<size_t> mu_off(count);
  size_t mo = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t ncell = (int64_t)sys[i].Lx * sys[i].Ly;
    const size_t vb = (size_t)ncell * SORB * C * 16;
    char* vec = reinterpret_cast<char*>(off_vec[i]);
    hs[i].vt = reinterpret_cast<const float*>(off_vt[i]);
    hs[i].phase = reinterpret_cast<const float*>(off_ph[i]);
    hs[i].r0 = vec;
    hs[i].bA = vec + vb;
    hs[i].bB = vec + 2 * vb;
    hs[i].bC = has_two ? vec + 3 * vb : nullptr;
    hs[i].bD = has_two ? vec + 4 * vb : nullptr;
    hs[i].partial = reinterpret_cast<double*>(off_part[i]);
    hs[i].tt = (float)(sys[i].t / scales[i].de_minus);
    hs[i].Lx = sys[i].Lx;
    hs[i].Ly = sys[i].Ly;
    hs[i].M = kpm[i].M;
    hs[i].units = units[i];
    mu_off[i] = mo;
    mo += (size_t)kpm[i].M;
  }
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(d_sys, hs.data(), sizeof(BSys) * count, cudaMemcpyHostToDevice, st));
  for (int i = 0; FIELD && i < count; ++i) {  // phase tables (flux 0: the identity rotations)
    rc = field_phases(ctx, &sys[i], 0, const_cast<float*>(hs[i].phase));
    if (rc != KITE_OK) return rc;
  }

  // set-up kernels of every system (on-site draws and start vectors)
  auto setup = [&]() -> cudaError_t {
    cudaError_t ce = cudaMemsetAsync(ne, 0, sizeof(unsigned long long) * count, st);
    for (int i = 0; i < count && ce == cudaSuccess; ++i) {
      const int64_t ncell = (int64_t)sys[i].Lx * sys[i].Ly, N = ncell * SORB;
      const double thr_d = floor(sys[i].p_vac * 4294967296.0);
      const uint64_t vac_thr =
          sys[i].p_vac <= 0.0 ? 0ull : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
      const uint32_t k0 = (uint32_t)sys[i].seed, k1 = (uint32_t)(sys[i].seed >> 32);
      const int blocks = (int)std::min<int64_t>((N + 255) / 256, (int64_t)ctx->num_sms * 16);
      k_onsite<float><<<std::max(1, blocks), 256, 0, st>>>(N, sys[i].lattice, sys[i].W, 0.5 * sys[i].delta,
                                                           scales[i].de_plus, scales[i].de_minus, vac_thr, 0u,
                                                           k0, k1, const_cast<float*>(hs[i].vt), ne + i,
                                                           sys[i].disorder);
      k_init_r0<float, SORB, C><<<std::max(1, blocks), 256, 0, st>>>(ncell, hs[i].vt, 0, R, 0u, k0, k1,
                                                                      nullptr, N, const_cast<void*>(hs[i].r0));
      ce = cudaGetLastError();
    }
    return ce;
  };
  auto upload = [&](const BPlan& pl) -> int {
    std::vector<int> ints(pl.sc.order);
    ints.insert(ints.end(), pl.sc.cta_team.begin(), pl.sc.cta_team.end());
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(d_teams, pl.sc.teams.data(), sizeof(BTeam) * pl.sc.teams.size(),
                                       cudaMemcpyHostToDevice, st));
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, st));
    KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // the host vectors go out of scope
    return KITE_OK;
  };

  // ---- autotune: time every candidate on this batch with capped steps -------------------
  // untuned: 8 stages at full occupancy (the last one-step plan), or the pinned two-step one
  int pick = 0;
  for (int c = 0; c < (int)cands.size(); ++c)
    if (!cands[c].two) pick = c;
  if (cands[pick].two) pick = (int)cands.size() - 1;
  if (tune && cands.size() > 1) {
    double wmax = 0.0;
    for (double x : work) wmax = std::max(wmax, x);
    int b1 = 0, b2 = 0;
    while ((double)(1ULL << (b1 + 1)) <= total) ++b1;
    while ((double)(1ULL << (b2 + 1)) <= wmax) ++b2;
    const uint64_t key = ((uint64_t)2 << 56) | ((uint64_t)LAT << 48) | ((uint64_t)C << 40) | ((uint64_t)DBL << 36) |
                         ((uint64_t)FIELD << 35) | ((uint64_t)(two_ok ? 1 + (pin == 2) : 0) << 32) |
                         ((uint64_t)std::min(count, 4095) << 20) | ((uint64_t)b1 << 10) | (uint64_t)b2;
    auto it = ctx->tune.find(key);
    bool found = false;
    if (it != ctx->tune.end())
      for (int c = 0; c < (int)cands.size(); ++c)
        if ((cands[c].nst | (cands[c].two << 8)) == it->second.first && cands[c].k == it->second.second)
          pick = c, found = true;
    if (!found) {
      KITE_CUDA_TRY(ctx, setup());
      // one capped sweep of candidate c (the first launch warms up, the second is timed)
      auto probe = [&](int c, int mcap, float* ms) -> int {
        if (upload(cands[c]) != KITE_OK) return KITE_ERR_CUDA;
        for (int rep = 0; rep < 2; ++rep) {
          KITE_CUDA_TRY(ctx, cudaMemsetAsync(counters, 0, sizeof(unsigned int) * cands[c].sc.teams.size(), st));
          KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
          cudaError_t ce = launch_batched<LAT, C, DBL, FIELD>(ctx, cands[c], d_sys, d_teams, d_ints, counters, 0, mcap);
          if (ce != cudaSuccess) return cuda_fail(ctx, ce, "autotune probe launch");
          KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
          KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
          KITE_CUDA_TRY(ctx, cudaEventElapsedTime(ms, ctx->ev2, ctx->ev3));
        }
        return KITE_OK;
      };
      // every candidate on a short capped sweep; the best one-step and the best two-step
      // plan are then compared per recursion step (a longer sweep minus the short one), since
      // a short sweep over-weights the two-step kernel's single first step
      const int mshort = DBL ? 4 : 8, mlong = 40;
      float best1 = 1e30f, best2 = 1e30f;
      int pick1 = -1, pick2 = -1;
      for (int c = 0; c < (int)cands.size(); ++c) {
        float ms = 1e30f;
        if (probe(c, mshort, &ms) != KITE_OK) return KITE_ERR_CUDA;
        // prefer the deeper ring and the default occupancy on near-ties
        if (cands[c].two) {
          if (ms < best2 * 0.98f) best2 = ms, pick2 = c;
        } else if (ms < best1 * 0.98f) {
          best1 = ms, pick1 = c;
        }
      }
      pick = pick1 >= 0 ? pick1 : pick2;
      if (pick1 >= 0 && pick2 >= 0) {
        float l1 = 1e30f, l2 = 1e30f;
        if (probe(pick1, mlong, &l1) != KITE_OK || probe(pick2, mlong, &l2) != KITE_OK) return KITE_ERR_CUDA;
        if (l2 - best2 < 0.97f * (l1 - best1)) pick = pick2;
      }
      ctx->tune[key] = {cands[pick].nst | (cands[pick].two << 8), cands[pick].k};
    }
  }
  const BPlan& pl = cands[pick];
  if (upload(pl) != KITE_OK) return KITE_ERR_CUDA;

  // ---- capture the whole batch into one graph ----------------------------------------
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  KITE_CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaMemsetAsync(counters, 0, sizeof(unsigned int) * pl.sc.teams.size(), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
  if (ce == cudaSuccess) ce = setup();
  if (ce == cudaSuccess) {
    const int stall = ctx->debug_stall;
    ctx->debug_stall = 0;
    ce = launch_batched<LAT, C, DBL, FIELD>(ctx, pl, d_sys, d_teams, d_ints, counters, stall, 0);
  }
  for (int i = 0; i < count && ce == cudaSuccess; ++i) {
    const int M = kpm[i].M;
    k_breduce<<<(M + 255) / 256, 256, 0, st>>>(hs[i].partial, M, pl.sc.ncta_of[i], Q, R, DBL ? 1 : 0, ne + i,
                                               d_mu + mu_off[i]);
    ce = cudaGetLastError();
  }
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, ce != cudaSuccess ? ce : ee, "capturing the batched graph");
  }
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "instantiating the batched graph");
  ce = cudaEventRecord(ctx->ev0, st);
  if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, st);
  if (ce == cudaSuccess) ce = cudaEventRecord(ctx->ev1, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(exec);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "running the batched graph");
  int status = 0;
  KITE_CUDA_TRY(ctx, cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status) return fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait gave up in the batched sweep");
  std::vector<unsigned long long> ne_h(count);
  KITE_CUDA_TRY(ctx, cudaMemcpy(ne_h.data(), ne, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost));
  // copy moments out and check them
  std::vector<double> host(mu_total);
  KITE_CUDA_TRY(ctx, cudaMemcpy(host.data(), d_mu, sizeof(double) * mu_total, cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < mu_total; ++k)
    if (!std::isfinite(host[k]) || std::fabs(host[k]) > 1.0 + 1e-3)
      return fail(ctx, KITE_ERR_BOUNDS, "a moment of the batch exceeds 1 or is not finite");
  for (int i = 0; i < count; ++i)
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(mu_out[i], d_mu + mu_off[i], sizeof(double) * kpm[i].M,
                                       cudaMemcpyDefault, st));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    double upd = 0.0, bytes = 0.0;
    for (int i = 0; i < count; ++i) {
      const double N = (double)sys[i].Lx * sys[i].Ly * SORB;
      upd += (double)ne_h[i] * kpm[i].M * R;
      if (pl.two) {
        // first step: r_0 in, r_1 out; a pass: r_{n-1}, r_n (and r_0 without doubling) in,
        // r_{n+1}, r_{n+2} out; the on-site term once per step or pass (an odd last step
        // runs as a whole pass)
        const int last = DBL ? steps_of(kpm[i].M) : std::max(kpm[i].M - 1, 1), passes = last / 2;
        bytes += (2.0 * 8.0 * R + 4.0) * N + passes * ((DBL ? 4.0 : 5.0) * 8.0 * R + 4.0) * N;
      } else {
        // per orbital and step: r_{n-1}, r_n (and r_0 without doubling) in, r_{n+1} out, on-site
        bytes += ((DBL ? 3.0 : 4.0) * 8.0 * R + 4.0) * N * (DBL ? steps_of(kpm[i].M) : std::max(kpm[i].M - 1, 0));
      }
    }
    stats->seconds = 1e-3 * ms;
    stats->updates = upd;
    stats->bytes_moved = bytes;
    stats->gbps = ms > 0 ? bytes / (1e-3 * ms) * 1e-9 : 0.0;
    stats->grid = pl.sc.grid;
    stats->block = pl.two ? kBlock2 : kBlock;
    stats->step_seconds = 1e-3 * ms;
    stats->step_launches = 1;
    stats->step_bytes = bytes;
    stats->n_eff = (int64_t)ne_h[count - 1];
    stats->ring_stages = pl.nst;
    stats->ctas_per_sm = pl.k;
    stats->steps_per_pass = pl.two ? 2 : 1;
  }
  return KITE_OK;
}

}  // namespace

int moments_1d_batched_impl(kite_ctx* ctx, int count, const kite_system* sys, const kite_kpm* kpm,
                            const std::vector<Scale>& scales, double* const* mu, kite_stats* st) {
  const int R = kpm[0].R;
  const int c = (R + 1) / 2;
  const int C = c <= 1 ? 1 : (c <= 2 ? 2 : 4);
  const bool hc = sys[0].lattice == KITE_HONEYCOMB;
  bool field = false;
  for (int i = 0; i < count; ++i) field = field || sys[i].flux != 0.0;
#define KITE_BF(LATV, CC, DB)                                                                 \
  (field ? run_batched<LATV, CC, DB, true>(ctx, count, sys, kpm, scales, mu, st)              \
         : run_batched<LATV, CC, DB, false>(ctx, count, sys, kpm, scales, mu, st))
#define KITE_B(LATV, CC) (kpm[0].doubling ? KITE_BF(LATV, CC, true) : KITE_BF(LATV, CC, false))
  if (hc) return C == 1 ? KITE_B(KITE_HONEYCOMB, 1) : (C == 2 ? KITE_B(KITE_HONEYCOMB, 2) : KITE_B(KITE_HONEYCOMB, 4));
  return C == 1 ? KITE_B(KITE_SQUARE, 1) : (C == 2 ? KITE_B(KITE_SQUARE, 2) : KITE_B(KITE_SQUARE, 4));
#undef KITE_B
#undef KITE_BF
}

}  // namespace kite
