// kite_internal.h -- internal declarations shared by the translation units of
// libkite_gb.so (never installed, never seen by callers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "kite_gb.h"

struct kite_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::string last_error;
  // Work buffer: one growing device allocation carved per call.
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // Small pinned host staging area (moments, status words).
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  // Device copy of pageable caller start vectors (grows on demand, freed at destroy).
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // Device zeros: the neighbour rows and cells across an open boundary (grows on demand).
  void* zeros = nullptr;
  size_t zeros_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  // Second stream for independent launch sequences that run side by side (the 2D path's
  // two vector families), with the events that fork it from and join it to `stream`.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Device status word: kernels set it (never trap) when a bounded wait gives up.
  int* d_status = nullptr;
  int debug_stall = 0;  // test hook, see kite_debug_stall_once
  // Autotuner cache: key (kernel family, precision, lattice, vectors per orbital, mode,
  // size bucket) -> (ring depth, CTAs per SM) measured fastest on this context's GPU.
  std::map<uint64_t, std::pair<int, int>> tune;
};

namespace kite {

// Records a message on the context and returns `status`.
int fail(kite_ctx* ctx, int status, const std::string& msg);
int cuda_fail(kite_ctx* ctx, cudaError_t e, const char* what);

// Ensures at least `bytes` of device work space; returns KITE_OK / KITE_ERR_OOM.
int ensure_ws(kite_ctx* ctx, size_t bytes);
int ensure_pinned(kite_ctx* ctx, size_t bytes);
// Creates the context's second stream and its fork/join events on first use.
int ensure_aux(kite_ctx* ctx);
// Device zeros of the system's open boundaries (one row of the widest cell, 128 bytes per
// cell, plus a margin for narrow lattices): *out = null for a periodic lattice.
int open_zeros(kite_ctx* ctx, const kite_system* sys, const void** out);

// True if p is device (or managed) memory of the current device.
bool is_device_ptr(const void* p);

// Device-side view of `bytes` of caller input: device memory as it is; page-locked host
// memory through its mapped device address (kernels read it across the host link, no
// copy); pageable host memory copied into the context's staging buffer on its stream.
int device_view(kite_ctx* ctx, const void* p, size_t bytes, const void** out);

// Copies `bytes` between caller memory (host or device) and device memory on the
// context stream.
cudaError_t copy_in(kite_ctx* ctx, void* dst_dev, const void* src, size_t bytes);
cudaError_t copy_out(kite_ctx* ctx, void* dst, const void* src_dev, size_t bytes);

// Carves aligned sub-buffers out of the work space.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
  size_t used() const { return (off + 255) & ~size_t(255); }
};

// One vector batch of the 1D sweep in a magnetic field (kite_field.cu): the step launches
// only; the caller reduces the partials as for the plain sweep.
struct FieldSweep {
  int fp64, lattice, C, doubling;
  int Lx, Ly, M;
  long long units;
  int G;       // persistent grid (the partials hold G rows per moment slot)
  int stall;   // test hook of the first launch (kite_debug_stall_once)
  int64_t ncell, N;
  const void* vt;
  double tt;
  void *r0, *bA, *bB;
  double* partial;
  const void* phase;  // [Ly][sublattice][2 bonds][cos, sin] of the working precision
  const void* zero;   // open boundaries: device zeros of at least one row, else null
  int open_x, open_y;
  // outputs
  void *last_prev, *last_cur;
  double seconds, bytes;
  int64_t launches;
};
int field_phases(kite_ctx* ctx, const kite_system* sys, int fp64, void* table);
int field_occupancy(int fp64, int lattice, int C, int doubling);
int field_sweep(kite_ctx* ctx, FieldSweep* a);

// The 1D sweep of a small lattice held on chip, one thread-block cluster of `cs` CTAs per
// independent real recursion (kite_cluster.cu); no magnetic field.
struct ClusterSweep {
  int fp64, lattice, doubling, realv;
  int Lx, Ly, M;
  int C;          // 16-byte chunks per orbital of the start-vector batch
  int per_chunk;  // vectors per chunk
  int nvec;       // vectors of the batch
  int open_x, open_y;
  int cs;         // CTAs per cluster
  const void* r0;
  const void* vt;
  double tt;
  double* part;   // moment partials, cluster_part_doubles(...) doubles
  const unsigned long long* n_eff;
  double* mu_vec;
  int vec_base;
  void* last_prev;  // optional: r_{M-2}, r_{M-1} in the start vectors' chunk layout (no doubling)
  void* last_cur;
  // outputs
  double seconds, bytes;
  int grid;
};
// Dynamic shared memory of one CTA for cluster size cs (0: the lattice does not fit).
int cluster_smem(const ClusterSweep& a, int cs);
// Clusters of size cs that can be resident at once (0: not launchable or does not fit).
int cluster_active(kite_ctx* ctx, const ClusterSweep& a, int cs);
size_t cluster_part_doubles(int lanes, int cs, int M, int doubling, int timing_steps);
// timing_steps > 0: a timing run of that many steps, nothing stored; 0: the whole sweep,
// then the moments into mu_vec.
int cluster_sweep(kite_ctx* ctx, ClusterSweep* a, int timing_steps);

// AdamW step coefficients of the learned reconstructor's training (kite_mlp.cu).
struct AdamwCoeffs {
  float lr, c1, c2;
};
AdamwCoeffs adamw_coeffs(int t, int total, double lr);

// Rescaling of Eqs. rescalingH/rescalingE.
struct Scale {
  double e_min, e_max, de_plus, de_minus;
};
int resolve_bounds(kite_ctx* ctx, const kite_system* sys, double e_min, double e_max, Scale* sc);

}  // namespace kite

#define KITE_CUDA_TRY(ctx, expr)                              \
  do {                                                        \
    cudaError_t kite_e_ = (expr);                             \
    if (kite_e_ != cudaSuccess) return kite::cuda_fail(ctx, kite_e_, #expr); \
  } while (0)

namespace kite {

// Device views of caller buffers: device pointers pass through; host buffers are staged
// in one stream-ordered allocation released at the end of the call.
struct Staging {
  kite_ctx* ctx;
  std::vector<void*> owned;
  ~Staging() {
    for (void* p : owned) cudaFreeAsync(p, ctx->stream);
  }
  template <typename T>
  int in(const T* src, size_t count, const T** out) {
    if (!src || is_device_ptr(src)) {
      *out = src;
      return KITE_OK;
    }
    void* d = nullptr;
    KITE_CUDA_TRY(ctx, cudaMallocAsync(&d, sizeof(T) * std::max<size_t>(count, 1), ctx->stream));
    owned.push_back(d);
    KITE_CUDA_TRY(ctx, copy_in(ctx, d, src, sizeof(T) * count));
    *out = static_cast<const T*>(d);
    return KITE_OK;
  }
  template <typename T>
  int out(T* dst, size_t count, T** dev) {
    if (!dst || is_device_ptr(dst)) {
      *dev = dst;
      return KITE_OK;
    }
    void* d = nullptr;
    KITE_CUDA_TRY(ctx, cudaMallocAsync(&d, sizeof(T) * std::max<size_t>(count, 1), ctx->stream));
    owned.push_back(d);
    *dev = static_cast<T*>(d);
    return KITE_OK;
  }
  template <typename T>
  int scratch(size_t count, T** dev) {
    void* d = nullptr;
    KITE_CUDA_TRY(ctx, cudaMallocAsync(&d, sizeof(T) * std::max<size_t>(count, 1), ctx->stream));
    owned.push_back(d);
    *dev = static_cast<T*>(d);
    return KITE_OK;
  }
  template <typename T>
  int back(T* dst, const T* dev, size_t count) {
    if (!dst || dst == dev) return KITE_OK;
    KITE_CUDA_TRY(ctx, copy_out(ctx, dst, dev, sizeof(T) * count));
    return KITE_OK;
  }
};

}  // namespace kite
