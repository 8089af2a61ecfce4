// kite_device.cuh -- device helpers: counter-based random numbers and the 16-byte
// vector chunks the stencil kernels move.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kite {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11).  Ten rounds; each multiplies counter words 0 and 2 by the
// round constants, crosses the high halves with words 1/3 and the key, and the key
// advances by the Weyl increments between rounds.
struct Philox4 {
  uint32_t w[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  Philox4 r;
  r.w[0] = c0;
  r.w[1] = c1;
  r.w[2] = c2;
  r.w[3] = c3;
  return r;
}

enum : uint32_t { kTagDisorder = 1u, kTagPhase = 2u, kTagInit = 3u };

// 53-bit uniform in [0,1): exact in FP64.
__device__ __forceinline__ double u53(const Philox4& x) {
  const uint64_t k = (uint64_t(x.w[0]) << 21) | uint64_t(x.w[1] >> 11);
  return __dmul_rn(__ull2double_rn(k), 0x1p-53);
}

// A 16-byte chunk of interleaved complex values: two complex FP32 or one complex FP64.
template <typename Real>
struct Chunk;

// 16-byte aligned: every chunk in global or shared memory starts on a 16-byte boundary, and
// the alignment lets the compiler use one 16-byte access per chunk whatever the address
// arithmetic.
template <>
struct alignas(16) Chunk<float> {
  static constexpr int kReals = 4;
  static constexpr int kVecs = 2;
  float v[4];
  __device__ __forceinline__ static Chunk ldg(const void* base, size_t idx) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(base) + idx);
    Chunk c;
    c.v[0] = t.x;
    c.v[1] = t.y;
    c.v[2] = t.z;
    c.v[3] = t.w;
    return c;
  }
  __device__ __forceinline__ static Chunk ld(const void* base, size_t idx) {
    const float4 t = reinterpret_cast<const float4*>(base)[idx];
    Chunk c;
    c.v[0] = t.x;
    c.v[1] = t.y;
    c.v[2] = t.z;
    c.v[3] = t.w;
    return c;
  }
  __device__ __forceinline__ void st(void* base, size_t idx) const {
    reinterpret_cast<float4*>(base)[idx] = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <>
struct alignas(16) Chunk<double> {
  static constexpr int kReals = 2;
  static constexpr int kVecs = 1;
  double v[2];
  __device__ __forceinline__ static Chunk ldg(const void* base, size_t idx) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(base) + idx);
    Chunk c;
    c.v[0] = t.x;
    c.v[1] = t.y;
    return c;
  }
  __device__ __forceinline__ static Chunk ld(const void* base, size_t idx) {
    const double2 t = reinterpret_cast<const double2*>(base)[idx];
    Chunk c;
    c.v[0] = t.x;
    c.v[1] = t.y;
    return c;
  }
  __device__ __forceinline__ void st(void* base, size_t idx) const {
    reinterpret_cast<double2*>(base)[idx] = make_double2(v[0], v[1]);
  }
};

// Rounded arithmetic with no contraction or reassociation, for both precisions.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename Real>
__device__ __forceinline__ Real quiet_nan();
template <>
__device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double quiet_nan<double>() {
  return __longlong_as_double(0x7ff8000000000000ll);
}

// A vacancy's on-site term is a NaN.  In FP64 the test runs on the integer pipe (|bits|
// above the infinity pattern) rather than as an FP64 comparison: GB300's FP64 pipe is the
// bound of the FP64 recursion.
__device__ __forceinline__ bool is_vacancy(float v) { return v != v; }
__device__ __forceinline__ bool is_vacancy(double v) {
  return (unsigned long long)(__double_as_longlong(v) & 0x7fffffffffffffffll) > 0x7ff0000000000000ull;
}

}  // namespace kite

namespace kite {

// ---- shared-memory mbarrier and bulk-copy (TMA engine, 1D) helpers ------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Makes barrier initialisation visible to the asynchronous (bulk-copy) proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity; gives up after ~kWaitCycles SM cycles
// (about a second) and returns false, so that no wait can hang the GPU.
constexpr long long kWaitCycles = 2000000000ll;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// As mbar_wait_bounded, with each try suspending the thread for up to ~20 us (instead of
// the hardware's default limit) while the phase is pending: fewer polling instructions.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded_hint(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait_hint(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait_hint(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic stream
// serialisation may be scheduled while its predecessor on the stream still runs; it must
// wait here, before it reads or writes any memory the predecessor touches, until that grid
// has completed and its writes are visible.  In a kernel launched the ordinary way the wait
// returns at once.  launch_dependents lets the successor be scheduled as soon as every CTA
// of this grid has passed it (it then waits in griddep_wait, on the hardware).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Element (row, k) of a split-BF16 vector family stored K-blocked: the 64 K columns of one
// block for all `rows` rows are contiguous ([K/64][rows][64]), so a TMA box of 64 columns
// by 128 or 256 rows is one contiguous run of memory instead of rows spread Kp apart.
__host__ __device__ __forceinline__ int64_t fam_index(int64_t row, int64_t k, int64_t rows) {
  return ((k >> 6) * rows + row) * 64 + (k & 63);
}

// 1D bulk copy global -> shared, completion counted in bytes on `bar`.  Both addresses
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace kite
