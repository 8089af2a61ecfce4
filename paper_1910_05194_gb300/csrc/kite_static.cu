// kite_static.cu -- a variant of the 1D moment sweep that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need moments: a host
// framework whose caching allocator has already reserved the device's memory budget,
// or a latency-critical loop that must never block in the allocator.  For them,
// kite_moments_1d_static runs the same kernels as kite_moments_1d but keeps every
// intermediate (on-site energies, the three vector buffers, moment partials, counters,
// status words) in one file-scope device array of fixed size, so the call performs no
// cudaMalloc/cudaFree and creates no library context.
//
// The array exists once per GPU that loads the library and lives until the process
// exits.  All calls on a device share it and it keeps the previous call's contents:
// every value that must start at zero is cleared on the stream at the start of a call,
// and calls that overlap on the GPU (two streams, or two host threads) race on it.
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "kite_step.cuh"

namespace kite {
namespace {

// Maximum scratch: 32 MiB per device.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
// device address of g_static_scratch per device, with the id of the context it was taken
// in (0 when the driver cannot report context ids)
struct StaticAddr {
  void* ptr = nullptr;
  unsigned long long ctx_id = 0;
};
StaticAddr g_static_addr[kMaxDevices];

// Error text goes to the caller's buffer (if any) with snprintf: no allocation.
struct ErrBuf {
  char* buf;
  int len;
};
thread_local ErrBuf g_err = {nullptr, 0};

int static_fail(int status, const char* fmt, ...) {
  if (g_err.buf && g_err.len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err.buf, (size_t)g_err.len, fmt, ap);
    va_end(ap);
  }
  return status;
}

// Id of the calling thread's current CUDA context (driver calls cuCtxGetCurrent and
// cuCtxGetId, looked up through the runtime so the library does not link the driver
// library); 0 if unavailable.  A new context on a device (after cudaDeviceReset, for
// example) has a new id, so a cached address is never used across contexts.
unsigned long long current_ctx_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f1);
      get_id = reinterpret_cast<GetId>(f2);
    }
    cudaGetLastError();
    looked_up = true;
  }
  void* c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device.  The first call on a device
// (and the first after that device's context was replaced) resolves it with
// cudaGetSymbolAddress; in host code the symbol is only a stand-in.  On that first call
// the runtime loads this library's device code on the device, which reserves the array.
int static_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return static_fail(KITE_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticAddr& a = g_static_addr[device];
  if (a.ptr && a.ctx_id != 0 && current_ctx_id() == a.ctx_id) {
    *out = a.ptr;
    return KITE_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return static_fail(KITE_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  }
  a.ptr = p;
  a.ctx_id = current_ctx_id();
  *out = p;
  return KITE_OK;
}

__global__ void k_static_reduce(const double* __restrict__ partial, int M, int G, int Q, int nvec,
                                const unsigned long long* __restrict__ n_eff,
                                double* __restrict__ acc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * Q) return;
  const int n = idx / Q, q = idx - (idx / Q) * Q;
  if ((q & 1) || (q >> 1) >= nvec) return;  // real parts of the valid vectors
  double sum = 0.0;
  const double* p = partial + (size_t)n * G * Q + q;
  for (int g = 0; g < G; ++g) sum += p[(size_t)g * Q];
  const double ne = (double)*n_eff;
  acc[(size_t)(q >> 1) * M + n] += ne > 0.0 ? sum / ne : 0.0;
}

__global__ void k_static_finish(const double* __restrict__ acc, int nv_total, int M,
                                double* __restrict__ mu, int* __restrict__ bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  double s = 0.0;
  for (int v = 0; v < 8; ++v) s += acc[(size_t)v * M + n];
  s /= nv_total;
  mu[n] = s;
  if (!(fabs(s) <= 1.0 + 1e-3)) atomicExch(bad, 1);  // also catches NaN
}

template <typename Real, int LAT, int C>
int static_run(const kite_system* sys, const kite_kpm* kpm, double* mu, cudaStream_t st,
               void* scratch, int device) {
  constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  constexpr int VPC = Chunk<Real>::kVecs;
  constexpr int Q = 2 * C * VPC;
  using Sh = StepShape<LAT, C>;
  const int M = kpm->M, R = kpm->R, S = kpm->S;
  const int64_t ncell = (int64_t)sys->Lx * sys->Ly, N = ncell * SORB;
  const long long units = (long long)((sys->Lx + Sh::TX - 1) / Sh::TX) * sys->Ly;
  int sms = 0, occ = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return static_fail(KITE_ERR_CUDA, "cudaDeviceGetAttribute");
  cudaFuncSetAttribute(k_step<Real, LAT, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  cudaFuncSetAttribute(k_step<Real, LAT, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step<Real, LAT, C, false>, kBlock,
                                                    Sh::SMEM) != cudaSuccess || occ < 1)
    occ = 1;
  const int G = (int)std::max(1LL, std::min((long long)sms * occ, units));
  const size_t vec_bytes = (size_t)ncell * SORB * C * 16;
  // carve the fixed array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += bytes;
    return static_cast<unsigned char*>(scratch) + at;
  };
  Real* vt = reinterpret_cast<Real*>(take(sizeof(Real) * N));
  void* r0 = take(vec_bytes);
  void* bA = take(vec_bytes);
  void* bB = take(vec_bytes);
  double* partial = reinterpret_cast<double*>(take(sizeof(double) * (size_t)std::max(M, 2) * G * Q));
  double* acc = reinterpret_cast<double*>(take(sizeof(double) * 8 * (size_t)M));
  double* mu_dev = reinterpret_cast<double*>(take(sizeof(double) * (size_t)M));
  unsigned long long* ne = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long)));
  int* status = reinterpret_cast<int*>(take(2 * sizeof(int)));  // [0] timeout, [1] bounds
  if (off > kStaticScratchBytes)
    return static_fail(KITE_ERR_ARG,
                       "kite_moments_1d_static needs %zu KiB of scratch but its fixed array holds "
                       "%zu KiB: use fewer orbitals, vectors or moments, or kite_moments_1d",
                       off >> 10, kStaticScratchBytes >> 10);
  // clear what must start at zero (the array keeps the previous call's contents)
  if (cudaMemsetAsync(acc, 0, sizeof(double) * 8 * (size_t)M, st) != cudaSuccess ||
      cudaMemsetAsync(status, 0, 2 * sizeof(int), st) != cudaSuccess)
    return static_fail(KITE_ERR_CUDA, "clearing scratch");
  const double de_plus = 0.5 * (kpm->e_max + kpm->e_min), de_minus = 0.5 * (kpm->e_max - kpm->e_min);
  const Real tt = (Real)(sys->t / de_minus);
  const double thr_d = floor(sys->p_vac * 4294967296.0);
  const uint64_t vac_thr =
      sys->p_vac <= 0.0 ? 0ull : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
  const uint32_t k0 = (uint32_t)sys->seed, k1 = (uint32_t)(sys->seed >> 32);
  const int blocks = (int)std::min<int64_t>((N + 255) / 256, (int64_t)sms * 16);
  for (int s = 0; s < S; ++s) {
    if (cudaMemsetAsync(ne, 0, sizeof(unsigned long long), st) != cudaSuccess)
      return static_fail(KITE_ERR_CUDA, "clearing counter");
    k_onsite<Real><<<blocks, 256, 0, st>>>(N, sys->lattice, sys->W, 0.5 * sys->delta, de_plus,
                                           de_minus, vac_thr, (uint32_t)s, k0, k1, vt, ne,
                                           sys->disorder);
    k_init_r0<Real, SORB, C><<<blocks, 256, 0, st>>>(ncell, vt, 0, R, (uint32_t)s * R, k0, k1,
                                                     nullptr, N, r0);
    auto where = [&](int n) -> void* { return n == 0 ? r0 : ((n & 1) ? bA : bB); };
    k_step<Real, LAT, C, true><<<G, kBlock, Sh::SMEM, st>>>(nullptr, r0, bA, r0, vt, tt, sys->Lx, sys->Ly,
                                                         units, partial + (size_t)G * Q, partial,
                                                         status, 0, FamOut{});
    for (int n = 1; n + 1 < M; ++n)
      k_step<Real, LAT, C, false><<<G, kBlock, Sh::SMEM, st>>>(
          where(n - 1), where(n), where(n + 1), r0, vt, tt, sys->Lx, sys->Ly, units,
          partial + (size_t)(n + 1) * G * Q, nullptr, status, 0, FamOut{});
    k_static_reduce<<<(M * Q + 255) / 256, 256, 0, st>>>(partial, M, G, Q, R, ne, acc);
    if (cudaGetLastError() != cudaSuccess) return static_fail(KITE_ERR_CUDA, "kernel launch");
  }
  k_static_finish<<<(M + 255) / 256, 256, 0, st>>>(acc, R * S, M, mu_dev, status + 1);
  int flags[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(mu, mu_dev, sizeof(double) * M, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags, status, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return static_fail(KITE_ERR_CUDA, "moments: %s", cudaGetErrorString(e));
  if (flags[0]) return static_fail(KITE_ERR_TIMEOUT, "a bounded wait gave up in the step kernel");
  if (flags[1]) return static_fail(KITE_ERR_BOUNDS, "a moment exceeds 1 in magnitude or is not finite");
  return KITE_OK;
}

}  // namespace
}  // namespace kite

using namespace kite;

namespace {
int moments_1d_static_checked(const kite_system* sys, const kite_kpm* kpm_in, double* mu,
                              void* cuda_stream);
}

extern "C" int kite_moments_1d_static(const kite_system* sys, const kite_kpm* kpm, double* mu,
                                      void* cuda_stream, char* err, int err_len) {
  g_err = {err, err_len};
  if (err && err_len > 0) err[0] = '\0';
  const int rc = moments_1d_static_checked(sys, kpm, mu, cuda_stream);
  g_err = {nullptr, 0};
  return rc;
}

namespace {
int moments_1d_static_checked(const kite_system* sys, const kite_kpm* kpm_in, double* mu,
                              void* cuda_stream) {
  if (!sys || !kpm_in || !mu) return static_fail(KITE_ERR_ARG, "system, kpm and mu are required");
  kite_kpm kpm_v = *kpm_in;
  const kite_kpm* kpm = &kpm_v;
  if (kpm_v.e_min == 0.0 && kpm_v.e_max == 0.0) {  // Gershgorin enclosure, as kite_moments_1d
    if (kite_bounds(sys, &kpm_v.e_min, &kpm_v.e_max) != KITE_OK)
      return static_fail(KITE_ERR_ARG, "invalid system");
  }
  if (sys->lattice != KITE_HONEYCOMB && sys->lattice != KITE_SQUARE)
    return static_fail(KITE_ERR_ARG, "unknown lattice");
  if (sys->Lx < 1 || sys->Ly < 1 || !(sys->p_vac >= 0.0 && sys->p_vac <= 1.0) || sys->W < 0.0 ||
      (sys->disorder != KITE_DISORDER_UNIFORM && sys->disorder != KITE_DISORDER_GAUSSIAN))
    return static_fail(KITE_ERR_ARG, "invalid system");
  if (sys->flux != 0.0) return static_fail(KITE_ERR_ARG, "the allocation-free call takes no magnetic field");
  if (sys->open_x || sys->open_y)
    return static_fail(KITE_ERR_ARG, "the allocation-free call takes periodic boundaries only");
  if (kpm->M < 1 || kpm->M > 65536 || kpm->R < 1 || kpm->S < 1)
    return static_fail(KITE_ERR_ARG, "need 1 <= M <= 65536, R >= 1, S >= 1");
  if (kpm->r0 || kpm->r_last || kpm->doubling != 0 || kpm->real_vectors != 0)
    return static_fail(KITE_ERR_ARG, "start vectors, r_last and doubling are not available here");
  if (!(kpm->e_max > kpm->e_min)) return static_fail(KITE_ERR_ARG, "e_max must exceed e_min");
  const int max_vec = kpm->precision == KITE_FP64 ? 4 : 8;
  if (kpm->R > max_vec)
    return static_fail(KITE_ERR_ARG, "R is limited to one batch (8 FP32 or 4 FP64 vectors)");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return static_fail(KITE_ERR_CUDA, "cudaGetDevice");
  void* scratch = nullptr;
  int rc = static_scratch(device, &scratch);
  if (rc != KITE_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int VPC = kpm->precision == KITE_FP64 ? 1 : 2;
  const int c = (kpm->R + VPC - 1) / VPC;
  const int C = c <= 1 ? 1 : (c <= 2 ? 2 : 4);
  const bool fp64 = kpm->precision == KITE_FP64;
  if (kpm->precision != KITE_FP32 && !fp64) return static_fail(KITE_ERR_ARG, "unknown precision");
#define KITE_STATIC(REAL, LAT)                                                              \
  (C == 1   ? static_run<REAL, LAT, 1>(sys, kpm, mu, st, scratch, device)                    \
   : C == 2 ? static_run<REAL, LAT, 2>(sys, kpm, mu, st, scratch, device)                    \
            : static_run<REAL, LAT, 4>(sys, kpm, mu, st, scratch, device))
  if (sys->lattice == KITE_HONEYCOMB)
    return fp64 ? KITE_STATIC(double, KITE_HONEYCOMB) : KITE_STATIC(float, KITE_HONEYCOMB);
  return fp64 ? KITE_STATIC(double, KITE_SQUARE) : KITE_STATIC(float, KITE_SQUARE);
#undef KITE_STATIC
}
}  // namespace
