// kite_mlp.cu -- the learned DOS reconstructor: a multilayer perceptron IN -> H -> H -> OUT
// (ReLU, BF16 weights/activations, FP32 accumulation) trained with a mean-absolute-error
// loss and AdamW on FP32 master weights, all in this file's kernels.
//
// The paper has no learned component; its Sec. 2a notes that the energy resolution of the
// Chebyshev reconstruction scales as the inverse number of moments.  The network maps the
// first IN moments of a system to its density of states on OUT energies as reconstructed
// from many more moments.  A label-free consistency gate recomputes the low Chebyshev
// moments of the predicted density and flags predictions that disagree with the input.
//
// Parameter layout (one flat FP32 vector): W1[H][IN], b1[H], W2[H][H], b2[H], W3[OUT][H],
// b3[OUT], row-major.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <random>
#include <vector>

#include "kite_device.cuh"
#include "kite_internal.h"
#include "kite_tc.cuh"

namespace kite {
namespace {

constexpr int IN = KITE_MLP_IN, HID = KITE_MLP_HIDDEN, OUT = KITE_MLP_OUT;
constexpr double kBeta1 = 0.9, kBeta2 = 0.999;
constexpr float kAdamEps = 1e-8f;
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + (int64_t)HID * IN, kOffW2 = kOffB1 + HID,
                  kOffB2 = kOffW2 + (int64_t)HID * HID, kOffW3 = kOffB2 + HID,
                  kOffB3 = kOffW3 + (int64_t)OUT * HID, kParams = kOffB3 + OUT;

// ------------------------------------------------------------------------------------
// GEMM on the 5th-generation tensor cores, BF16 in, FP32 accumulate in TMEM:
//   C[m][n] = sum_k A[m][k] B[n][k]   (A [M][lda], B [N][ldb], both K contiguous)
// Epilogue: alpha * C + bias[n] + add[m][n]; relu; zero where mask[m][n] <= 0; store FP32
// (C32) and/or BF16 (C16) with leading dimension ldc.  One 128 x 128 output tile per CTA:
// warp 0 issues the TMA loads (128-byte swizzle, 64-column K blocks, zero fill outside
// the matrices) into a four-stage ring, warp 1 allocates 128 TMEM columns and one lane
// issues tcgen05.mma (M = N = 128, K = 16), warps 2-5 read the accumulator back
// (tcgen05.ld, one TMEM lane quarter each) and apply the epilogue.  The backward pass
// turns its transposed products into this form with explicit transposes (k_mlp_transpose).
// ------------------------------------------------------------------------------------
struct GemmEpi {
  const float* bias;
  const float* add;  // optional addend [M][ldc] (the residual prior)
  const __nv_bfloat16* mask;
  int relu;
  float* C32;
  __nv_bfloat16* C16;
  int ldc;
  float alpha;
};

constexpr int kTM = 128, kTN = 128, kTK = 64, kTStages = 4;
constexpr int kTATile = kTM * kTK * 2, kTBTile = kTN * kTK * 2;  // 16 KB each
constexpr int kTStage = kTATile + kTBTile;
constexpr int kTThreads = 64 + 128;  // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kTSmem = 1024 + kTStages * kTStage + 256;
constexpr int kTPitch = kTN + 1;  // floats per row of the epilogue's staging tile (conflict-free)
static_assert(kTM * kTPitch * 4 <= kTStages * kTStage, "the epilogue tile reuses the operand stages");
constexpr uint32_t kTIdesc = idesc_bf16_f32(kTM, kTN);

__global__ void __launch_bounds__(kTThreads, 1)
    k_mlp_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int M, int N, int K,
             const GemmEpi ep, int* __restrict__ err) {
  extern __shared__ unsigned char tsmem_raw[];
  const uint32_t raw = smem_u32(tsmem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle atoms repeat every 1024 B
  uint64_t* bars = reinterpret_cast<uint64_t*>(tsmem_raw + (base - raw) + kTStages * kTStage);
  uint64_t* full = bars;
  uint64_t* empty = bars + kTStages;
  uint64_t* tfull = bars + 2 * kTStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTStages + 1);
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = blockIdx.x, tm = blockIdx.y;
  const int nk = (K + kTK - 1) / kTK;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kTStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(tfull, 1);
    mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int pend[kTStages];
      for (int i = 0; i < kTStages; ++i) pend[i] = -1;
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb) {
        const int st = kb % kTStages;
        const uint32_t ph = (uint32_t)((kb / kTStages) & 1);
        if (!wait_or_abort(&empty[st], ph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[st], kTStage);
        const uint32_t sb = base + st * kTStage;
        tma_load_2d(sb, &tA, &full[st], kb * kTK, tm * kTM);
        tma_load_2d(sb + kTATile, &tB, &full[st], kb * kTK, tn * kTN);
        pend[st] = (int)ph;
      }
      if (!ok)  // drain: the last copies issued on every stage land before the CTA exits
        for (int i = 0; i < kTStages; ++i)
          if (pend[i] >= 0) mbar_wait_bounded(&full[i], (uint32_t)pend[i]);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int st = kb % kTStages;
        if (!wait_or_abort(&full[st], (uint32_t)((kb / kTStages) & 1), abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sb = base + st * kTStage;
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk)
          umma_f16(tmem, desc_k128(sb + kk * 32), desc_k128(sb + kTATile + kk * 32), kTIdesc,
                   (kb > 0 || kk > 0) ? 1u : 0u);
        umma_commit(&empty[st]);  // the stage is reusable once these MMAs have read it
      }
      umma_commit(tfull);  // every MMA issued (none if aborted) has completed
    }
  } else {  // epilogue: TMEM lane quarter q holds rows q*32 .. q*32+31 of the tile
    // The accumulator goes through shared memory (the operand stages are free once every
    // MMA has completed), so that the epilogue's loads and stores run along rows: lane l
    // of a warp handles columns l, l+32, l+64, l+96 of each of its quarter's rows.
    const int q = warp & 3;
    float* tile = reinterpret_cast<float*>(tsmem_raw + (base - raw)) + q * 32 * kTPitch;
    if (wait_or_abort(tfull, 0, abort_flag) && !*abort_flag) {
      tc_fence_after();
#pragma unroll 1
      for (int j = 0; j < kTN / 32; ++j) {
        uint32_t r[32];
        tmem_ld_32x32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 32), r);
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) tile[lane * kTPitch + j * 32 + jj] = __uint_as_float(r[jj]);
      }
      __syncwarp();
#pragma unroll 1
      for (int rr = 0; rr < 32; ++rr) {
        const int m = tm * kTM + q * 32 + rr;
        if (m >= M) break;
        const int64_t row = (int64_t)m * ep.ldc;
#pragma unroll
        for (int c4 = 0; c4 < kTN / 32; ++c4) {
          const int cl = c4 * 32 + lane, n = tn * kTN + cl;
          if (n >= N) continue;
          float v = ep.alpha * tile[rr * kTPitch + cl];
          if (ep.bias) v += ep.bias[n];
          if (ep.add) v += ep.add[row + n];
          if (ep.relu) v = fmaxf(v, 0.0f);
          if (ep.mask && !(__bfloat162float(ep.mask[row + n]) > 0.0f)) v = 0.0f;
          if (ep.C32) ep.C32[row + n] = v;
          if (ep.C16) ep.C16[row + n] = __float2bfloat16(v);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN) : "memory");
  }
}

// out[c][r] = in[r][c] for r < rows, c < cols (BF16, 32 x 32 tiles through shared memory)
__global__ void k_mlp_transpose(const __nv_bfloat16* __restrict__ in, int rows, int cols, int ldin,
                                __nv_bfloat16* __restrict__ out, int ldout) {
  __shared__ __nv_bfloat16 t[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    t[k][threadIdx.x] = (r < rows && c < cols) ? in[(int64_t)r * ldin + c] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(int64_t)c * ldout + r] = t[threadIdx.x][k];
  }
}

// Jackson kernel of order IN (Sec. 2a, kernel polynomial method) times the Chebyshev
// weight 2 - delta_k0 of Eq. e8a, computed on the host.
struct PriorCoef {
  double c[IN];
};

PriorCoef prior_coef() {
  PriorCoef pc;
  const double pi = 3.141592653589793, q = pi / (IN + 1);
  for (int k = 0; k < IN; ++k) {
    const double g = ((IN - k + 1) * std::cos(q * k) + std::sin(q * k) * std::cos(q) / std::sin(q)) / (IN + 1);
    pc.c[k] = (k == 0 ? 1.0 : 2.0) * g;
  }
  return pc;
}

// Residual prior P[r][j] = sum_k c_k X[r][k] T_k(eps_j) / (pi a sqrt(1 - eps_j^2)) on the
// midpoint grid eps_j = -1 + (2j+1)/OUT, a = (e_max - e_min)/2: the Jackson density per eV
// from the raw moments X (FP64 sums, forward Chebyshev recurrence).  One block per row.
__global__ void __launch_bounds__(256) k_mlp_prior(const float* __restrict__ X, int rows, const PriorCoef pc,
                                                   double inv_pi_a, float* __restrict__ P) {
  __shared__ double cx[IN];
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    __syncthreads();
    for (int k = threadIdx.x; k < IN; k += blockDim.x) cx[k] = pc.c[k] * (double)X[(int64_t)r * IN + k];
    __syncthreads();
    for (int j = threadIdx.x; j < OUT; j += blockDim.x) {
      const double e = -1.0 + (2.0 * j + 1.0) / OUT;
      double t0 = 1.0, t1 = e, sum = cx[0] + cx[1] * e;
      for (int k = 2; k < IN; ++k) {
        const double t2 = 2.0 * e * t1 - t0;
        sum += cx[k] * t2;
        t0 = t1;
        t1 = t2;
      }
      P[(int64_t)r * OUT + j] = (float)(sum * inv_pi_a / sqrt(1.0 - e * e));
    }
  }
}

// rows of X (FP32, optional per-column shift and scale: (x - shift) * scale) gathered by
// idx -> BF16; targets gathered alongside, minus the prior rows Tsub when given
__global__ void k_mlp_gather(const float* __restrict__ X, const int* __restrict__ idx, int rows, int cols,
                             const float* __restrict__ shift, const float* __restrict__ scale,
                             __nv_bfloat16* __restrict__ out,
                             const float* __restrict__ T, float* __restrict__ Tout, int tcols,
                             const float* __restrict__ Tsub = nullptr) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    const int64_t src = idx ? idx[r] : r;
    out[e] = __float2bfloat16((X[src * cols + c] - (shift ? shift[c] : 0.0f)) * (scale ? scale[c] : 1.0f));
  }
  if (T) {
    const int64_t tt = (int64_t)rows * tcols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tt; e += (int64_t)gridDim.x * blockDim.x) {
      const int r = (int)(e / tcols), c = (int)(e % tcols);
      const int64_t src = idx ? idx[r] : r;
      Tout[e] = T[src * tcols + c] - (Tsub ? Tsub[src * tcols + c] : 0.0f);
    }
  }
}

// dY = sign(Y - T) / count (BF16) and the partial L1 sums per block
__global__ void k_mlp_l1grad(const float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                             float inv_count, __nv_bfloat16* __restrict__ dY, double* __restrict__ lsum) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    dY[e] = __float2bfloat16(d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f));
    s += fabs((double)d);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) lsum[blockIdx.x] = red[0];
}

// db[n] = sum_m D[m][n] in fixed order (one thread per column)
__global__ void k_mlp_colsum(const __nv_bfloat16* __restrict__ D, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += __bfloat162float(D[(int64_t)m * N + n]);
  db[n] = s;
}

// AdamW (decoupled weight decay) on FP32 master weights; refreshes the BF16 copy (if any)
// (1 - b1 and 1 - b2 come from the host, rounded once from FP64: 1 - 0.999f in FP32 would
// be 1.3e-5 away from 0.001.)
__global__ void k_mlp_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int64_t n, float lr,
                            float b1, float omb1, float b2, float omb2, float eps, float wd, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i];
    p[i] -= lr * upd;
    if (pb) pb[i] = __float2bfloat16(p[i]);
  }
}

// Initial parameters drawn on the device: He-uniform weights W ~ U[-lim, lim] with
// lim = sqrt(6 / fan_in) (times head_scale for the last layer), zero biases.  The uniform
// u in [0,1) is the 53-bit draw of Philox4x32-10 at counter (i_lo, i_hi, 0, kTagInit),
// key = seed.
__global__ void k_mlp_init(float* __restrict__ p, uint64_t seed, float head_scale) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kParams; i += (int64_t)gridDim.x * blockDim.x) {
    float lim = 0.0f;
    if (i < kOffB1) lim = sqrtf(6.0f / IN);
    else if (i >= kOffW2 && i < kOffB2) lim = sqrtf(6.0f / HID);
    else if (i >= kOffW3 && i < kOffB3) lim = sqrtf(6.0f / HID) * head_scale;
    if (lim == 0.0f) {
      p[i] = 0.0f;
      continue;
    }
    const Philox4 x = philox4x32_10((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, kTagInit, k0, k1);
    p[i] = (float)((2.0 * u53(x) - 1.0) * (double)lim);
  }
}

// Per-column statistics of X [n][IN] for the input normalisation: shift = mean,
// scale = 1 / max(std, floor) with the population standard deviation, FP64 sums in a fixed
// order (one block per column, a strided partial per thread, then a tree).
__global__ void __launch_bounds__(256) k_mlp_colstats(const float* __restrict__ X, int n, float sd_floor,
                                                      float* __restrict__ shift, float* __restrict__ scale) {
  __shared__ double s1[256], s2[256];
  const int c = blockIdx.x;
  double a = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) a += (double)X[(int64_t)r * IN + c];
  s1[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s1[threadIdx.x] += s1[threadIdx.x + st];
    __syncthreads();
  }
  const double mean = s1[0] / n;
  double b = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double d = (double)X[(int64_t)r * IN + c] - mean;
    b += d * d;
  }
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s2[threadIdx.x] += s2[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    shift[c] = (float)mean;
    scale[c] = (float)(1.0 / fmax(sqrt(s2[0] / n), (double)sd_floor));
  }
}

// X [n][IN] FP32 = the first IN entries of each row of mu [n][mu_ld] (FP64)
__global__ void k_mlp_take_inputs(const double* __restrict__ mu, int mu_ld, int n, float* __restrict__ X) {
  const int64_t total = (int64_t)n * IN;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (float)mu[(e / IN) * mu_ld + e % IN];
}

// dst [K] FP32 = src [K] FP64 (round to nearest)
__global__ void k_mlp_narrow(const double* __restrict__ src, int K, float* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) dst[i] = (float)src[i];
}

__global__ void k_mlp_tobf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Consistency gate: Chebyshev moments of the predicted density on the midpoint grid
// eps_j = -1 + (2j+1)/OUT (rho in units per unit eps): m_k = (2/OUT) sum_j rho_j T_k(eps_j)
// compared with the input moments mu_k for k < kcheck; flag if max |m_k - mu_k| > tol.
__global__ void k_mlp_gate(const float* __restrict__ rho, const double* __restrict__ mu, int mu_ld, int kcheck,
                           double de_minus, double tol, int* __restrict__ flag, double* __restrict__ dev) {
  const int b = blockIdx.x;
  __shared__ double red[128];
  double worst = 0.0;
  for (int k = 0; k < kcheck; ++k) {
    double s = 0.0;
    for (int j = threadIdx.x; j < OUT; j += blockDim.x) {
      const double e = -1.0 + (2.0 * j + 1.0) / OUT;
      s += (double)rho[(int64_t)b * OUT + j] * de_minus * cos(k * acos(e));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
      if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) worst = fmax(worst, fabs(red[0] * 2.0 / OUT - mu[(int64_t)b * mu_ld + k]));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    flag[b] = worst > tol ? 1 : 0;
    if (dev) dev[b] = worst;
  }
}

struct Net {
  __nv_bfloat16* pb;  // bf16 parameters
  __nv_bfloat16 *W2t, *W3t;  // bf16 transposes of W2 [H][H] and W3 [OUT][H]: [H][H], [H][OUT]
  __nv_bfloat16 *X, *H1, *H2, *dY, *dZ2, *dZ1;
  // transposes of the activations and deltas, [features][ldr] with ldr = rows rounded up
  // to a multiple of 8 (the tensor maps' row pitch must be a multiple of 16 bytes)
  __nv_bfloat16 *Xt, *H1t, *H2t, *dYt, *dZ2t, *dZ1t;
  int ldr;
  float *Y, *T, *grad;
};

// Tensor maps of the operands: [rows][cols] bf16 with row pitch ld elements, boxes of 64
// columns x 128 rows, 128-byte swizzle.  Encoding is host work, so maps are cached by
// (address, shape, pitch), which fully determines them.
struct MapKey {
  const void* p;
  int rows, cols, ld;
  bool operator==(const MapKey& o) const { return p == o.p && rows == o.rows && cols == o.cols && ld == o.ld; }
};
struct MapEntry {
  MapKey key;
  CUtensorMap map;
};
std::mutex g_map_mutex;
std::vector<MapEntry> g_maps;

int operand_map(kite_ctx* ctx, const __nv_bfloat16* p, int rows, int cols, int ld, CUtensorMap* out) {
  const MapKey key{p, rows, cols, ld};
  std::lock_guard<std::mutex> lock(g_map_mutex);
  for (const MapEntry& e : g_maps)
    if (e.key == key) {
      *out = e.map;
      return KITE_OK;
    }
  auto enc = tensor_map_encoder();
  if (!enc) return fail(ctx, KITE_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)kTM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, KITE_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  if (g_maps.size() >= 256) g_maps.erase(g_maps.begin());
  g_maps.push_back(MapEntry{key, m});
  *out = m;
  return KITE_OK;
}

// C = A B^T on the tensor cores: A [M][K] (pitch lda), B [N][K] (pitch ldb), see k_mlp_tc.
int gemm(kite_ctx* ctx, cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
         int N, int K, GemmEpi ep) {
  if (M < 1 || N < 1 || K < 1) return KITE_OK;
  static bool attr = false;
  if (!attr) {
    KITE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTSmem));
    attr = true;
  }
  CUtensorMap mA, mB;
  int rc = operand_map(ctx, A, M, K, lda, &mA);
  if (rc == KITE_OK) rc = operand_map(ctx, B, N, K, ldb, &mB);
  if (rc != KITE_OK) return rc;
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
  k_mlp_tc<<<grid, kTThreads, kTSmem, st>>>(mA, mB, M, N, K, ep, ctx->d_status);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

void transpose(cudaStream_t st, const __nv_bfloat16* in, int rows, int cols, int ldin, __nv_bfloat16* out,
               int ldout) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  k_mlp_transpose<<<grid, block, 0, st>>>(in, rows, cols, ldin, out, ldout);
}

// bf16 transposes of W2 and W3 after the bf16 parameters changed
void refresh_wt(cudaStream_t st, const Net& net) {
  transpose(st, net.pb + kOffW2, HID, HID, HID, net.W2t, HID);
  transpose(st, net.pb + kOffW3, OUT, HID, HID, net.W3t, OUT);
}

GemmEpi epi(float* C32, __nv_bfloat16* C16, int ldc, const float* bias = nullptr, int relu = 0,
            const __nv_bfloat16* mask = nullptr) {
  GemmEpi e;
  e.bias = bias;
  e.add = nullptr;
  e.mask = mask;
  e.relu = relu;
  e.C32 = C32;
  e.C16 = C16;
  e.ldc = ldc;
  e.alpha = 1.0f;
  return e;
}

// forward on rows already in net.X (BF16, scaled); writes net.Y (FP32) = network (+ add)
int forward(kite_ctx* ctx, cudaStream_t st, const Net& net, const float* p32, int rows, const float* add = nullptr) {
  int rc = gemm(ctx, st, net.X, IN, net.pb + kOffW1, IN, rows, HID, IN, epi(nullptr, net.H1, HID, p32 + kOffB1, 1));
  if (rc == KITE_OK)
    rc = gemm(ctx, st, net.H1, HID, net.pb + kOffW2, HID, rows, HID, HID, epi(nullptr, net.H2, HID, p32 + kOffB2, 1));
  GemmEpi e3 = epi(net.Y, nullptr, OUT, p32 + kOffB3);
  e3.add = add;
  if (rc == KITE_OK) rc = gemm(ctx, st, net.H2, HID, net.pb + kOffW3, HID, rows, OUT, HID, e3);
  return rc;
}

bool use_prior(const kite_mlp_prior* prior) { return prior && prior->kind == KITE_PRIOR_JACKSON; }

void launch_prior(cudaStream_t st, int num_sms, const float* X, int rows, const kite_mlp_prior* prior, float* P) {
  const double a = 0.5 * (prior->e_max - prior->e_min);
  const int blocks = std::max(1, std::min(rows, num_sms * 8));
  k_mlp_prior<<<blocks, 256, 0, st>>>(X, rows, prior_coef(), 1.0 / (3.141592653589793 * a), P);
}

// backward of the mean L1 loss over rows x OUT; gradient into net.grad.  Each product with
// a transposed operand takes the transposes of activations, deltas or weights, so that
// every GEMM is A B^T with both operands K-contiguous.
int backward(kite_ctx* ctx, cudaStream_t st, const Net& net, int rows, double* lsum, int lblocks) {
  const int64_t n = (int64_t)rows * OUT;
  const int ldr = net.ldr;
  k_mlp_l1grad<<<lblocks, 256, 0, st>>>(net.Y, net.T, n, 1.0f / (float)n, net.dY, lsum);
  float* g = net.grad;
  transpose(st, net.dY, rows, OUT, OUT, net.dYt, ldr);
  transpose(st, net.H2, rows, HID, HID, net.H2t, ldr);
  // dW3 [OUT][H] = dY^T H2
  int rc = gemm(ctx, st, net.dYt, ldr, net.H2t, ldr, OUT, HID, rows, epi(g + kOffW3, nullptr, HID));
  k_mlp_colsum<<<(OUT + 255) / 256, 256, 0, st>>>(net.dY, rows, OUT, g + kOffB3);
  // dZ2 [rows][H] = (dY W3) masked by H2 > 0
  if (rc == KITE_OK)
    rc = gemm(ctx, st, net.dY, OUT, net.W3t, OUT, rows, HID, OUT, epi(nullptr, net.dZ2, HID, nullptr, 0, net.H2));
  transpose(st, net.dZ2, rows, HID, HID, net.dZ2t, ldr);
  transpose(st, net.H1, rows, HID, HID, net.H1t, ldr);
  // dW2 [H][H] = dZ2^T H1
  if (rc == KITE_OK) rc = gemm(ctx, st, net.dZ2t, ldr, net.H1t, ldr, HID, HID, rows, epi(g + kOffW2, nullptr, HID));
  k_mlp_colsum<<<(HID + 255) / 256, 256, 0, st>>>(net.dZ2, rows, HID, g + kOffB2);
  // dZ1 [rows][H] = (dZ2 W2) masked by H1 > 0
  if (rc == KITE_OK)
    rc = gemm(ctx, st, net.dZ2, HID, net.W2t, HID, rows, HID, HID, epi(nullptr, net.dZ1, HID, nullptr, 0, net.H1));
  transpose(st, net.dZ1, rows, HID, HID, net.dZ1t, ldr);
  transpose(st, net.X, rows, IN, IN, net.Xt, ldr);
  // dW1 [H][IN] = dZ1^T X
  if (rc == KITE_OK) rc = gemm(ctx, st, net.dZ1t, ldr, net.Xt, ldr, HID, IN, rows, epi(g + kOffW1, nullptr, IN));
  k_mlp_colsum<<<(HID + 255) / 256, 256, 0, st>>>(net.dZ1, rows, HID, g + kOffB1);
  return rc;
}

// The GEMM kernels set the context's status word when a bounded wait gives up.
int clear_status(kite_ctx* ctx) {
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  return KITE_OK;
}
int read_status(kite_ctx* ctx) {
  int h = 0;
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return h ? fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait gave up in the perceptron's GEMM") : KITE_OK;
}

int carve_net(kite_ctx* ctx, int rows, Net* net, float** extra, size_t extra_floats) {
  Carver probe(nullptr);
  const int ldr = (rows + 7) / 8 * 8;
  auto lay = [&](Carver& k, Net& n, float** ex) {
    n.pb = k.take<__nv_bfloat16>(kParams);
    n.W2t = k.take<__nv_bfloat16>((size_t)HID * HID);
    n.W3t = k.take<__nv_bfloat16>((size_t)HID * OUT);
    n.X = k.take<__nv_bfloat16>((size_t)rows * IN);
    n.H1 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.H2 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.dY = k.take<__nv_bfloat16>((size_t)rows * OUT);
    n.dZ2 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.dZ1 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.ldr = ldr;
    n.Xt = k.take<__nv_bfloat16>((size_t)IN * ldr);
    n.H1t = k.take<__nv_bfloat16>((size_t)HID * ldr);
    n.H2t = k.take<__nv_bfloat16>((size_t)HID * ldr);
    n.dYt = k.take<__nv_bfloat16>((size_t)OUT * ldr);
    n.dZ2t = k.take<__nv_bfloat16>((size_t)HID * ldr);
    n.dZ1t = k.take<__nv_bfloat16>((size_t)HID * ldr);
    n.Y = k.take<float>((size_t)rows * OUT);
    n.T = k.take<float>((size_t)rows * OUT);
    n.grad = k.take<float>(kParams);
    *ex = k.take<float>(extra_floats);
  };
  Net dummy;
  float* dex;
  lay(probe, dummy, &dex);
  int rc = ensure_ws(ctx, probe.used());
  if (rc != KITE_OK) return rc;
  Carver w(ctx->ws);
  lay(w, *net, extra);
  return KITE_OK;
}

}  // namespace

int64_t mlp_param_count() { return kParams; }

// Learning rate and bias corrections of optimiser step t (1-based) of `total`: the cosine
// schedule lr (1 + cos(pi (t - 1) / total)) / 2 and c1 = 1 - b1^t, c2 = 1 - b2^t of AdamW.
AdamwCoeffs adamw_coeffs(int t, int total, double lr) {
  AdamwCoeffs c;
  c.lr = (float)(lr * 0.5 * (1.0 + std::cos(3.141592653589793 * (t - 1) / std::max(1, total))));
  c.c1 = (float)(1.0 - std::pow(kBeta1, t));
  c.c2 = (float)(1.0 - std::pow(kBeta2, t));
  return c;
}

// One optimiser step on device arrays (the update kite_mlp_train applies after each batch).
int mlp_adamw_step_impl(kite_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n, int t, int total,
                        double lr, double wd) {
  const AdamwCoeffs c = adamw_coeffs(t, total, lr);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
  k_mlp_adamw<<<std::max(1, blocks), 256, 0, ctx->stream>>>(p, g, m, v, nullptr, n, c.lr, (float)kBeta1,
                                                             (float)(1.0 - kBeta1), (float)kBeta2,
                                                             (float)(1.0 - kBeta2), kAdamEps, (float)wd, c.c1, c.c2);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

// Full-batch gradient of the mean L1 loss (for checks): params, X [n][IN], T [n][OUT] device.
int mlp_gradient_impl(kite_ctx* ctx, const float* params, const float* X, const float* T, int n,
                      const float* shift, const float* scale, float* grad, double* loss) {
  Net net;
  float* ex;
  int rc = carve_net(ctx, n, &net, &ex, kParams + 4096);
  if (rc != KITE_OK) return rc;
  cudaStream_t st = ctx->stream;
  float* p32 = ex;
  double* lsum = reinterpret_cast<double*>(ex + kParams);
  if ((rc = clear_status(ctx)) != KITE_OK) return rc;
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(p32, params, sizeof(float) * kParams, cudaMemcpyDefault, st));
  k_mlp_tobf16<<<1024, 256, 0, st>>>(p32, net.pb, kParams);
  refresh_wt(st, net);
  k_mlp_gather<<<1024, 256, 0, st>>>(X, nullptr, n, IN, shift, scale, net.X, T, net.T, OUT);
  const int lblocks = 256;
  rc = forward(ctx, st, net, p32, n);
  if (rc == KITE_OK) rc = backward(ctx, st, net, n, lsum, lblocks);
  if (rc != KITE_OK) return rc;
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(grad, net.grad, sizeof(float) * kParams, cudaMemcpyDefault, st));
  std::vector<double> ls(lblocks);
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ls.data(), lsum, sizeof(double) * lblocks, cudaMemcpyDeviceToHost, st));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if ((rc = read_status(ctx)) != KITE_OK) return rc;
  if (loss) *loss = std::accumulate(ls.begin(), ls.end(), 0.0) / ((double)n * OUT);
  return KITE_OK;
}

int mlp_forward_impl(kite_ctx* ctx, const float* params, const float* X, int n, const float* shift,
                     const float* scale, float* Y,
                     const kite_mlp_prior* prior) {
  const int chunk = 4096;
  Net net;
  float* ex;
  const bool pri = use_prior(prior);
  int rc = carve_net(ctx, std::min(n, chunk), &net, &ex, kParams + (pri ? (size_t)std::min(n, chunk) * OUT : 0));
  if (rc != KITE_OK) return rc;
  cudaStream_t st = ctx->stream;
  if ((rc = clear_status(ctx)) != KITE_OK) return rc;
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ex, params, sizeof(float) * kParams, cudaMemcpyDefault, st));
  k_mlp_tobf16<<<1024, 256, 0, st>>>(ex, net.pb, kParams);
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int rows = std::min(chunk, n - r0);
    k_mlp_gather<<<1024, 256, 0, st>>>(X + (int64_t)r0 * IN, nullptr, rows, IN, shift, scale, net.X, nullptr,
                                       nullptr, 0);
    float* P = pri ? ex + kParams : nullptr;
    if (pri) launch_prior(st, ctx->num_sms, X + (int64_t)r0 * IN, rows, prior, P);
    rc = forward(ctx, st, net, ex, rows, P);
    if (rc != KITE_OK) return rc;
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(Y + (int64_t)r0 * OUT, net.Y, sizeof(float) * rows * OUT, cudaMemcpyDefault, st));
  }
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return read_status(ctx);
}

int mlp_train_impl(kite_ctx* ctx, const float* X, const float* T, int n, const float* shift, const float* scale,
                   const kite_mlp_train_cfg* cfg, float* params, float* loss_curve,
                   const kite_mlp_prior* prior) {
  const int bs = std::max(1, std::min(cfg->batch, n));
  Net net;
  float* ex;
  const bool pri = use_prior(prior);
  const size_t lsum_floats = 2 * (size_t)128 * ((n + bs - 1) / bs);  // FP64 partial sums of every step
  const size_t idx_floats = ((size_t)n + 63) / 64 * 64;
  int rc = carve_net(ctx, bs, &net, &ex, 3 * kParams + lsum_floats + idx_floats + (pri ? (size_t)n * OUT : 0));
  if (rc != KITE_OK) return rc;
  cudaStream_t st = ctx->stream;
  float* p32 = ex;
  float* m = ex + kParams;
  float* v = ex + 2 * kParams;
  double* lsum = reinterpret_cast<double*>(ex + 3 * kParams);
  int* d_idx = reinterpret_cast<int*>(ex + 3 * kParams + lsum_floats);
  // the prior of every training row, once; the batches gather T - prior as targets
  float* P = pri ? ex + 3 * kParams + lsum_floats + idx_floats : nullptr;
  if ((rc = clear_status(ctx)) != KITE_OK) return rc;
  if (pri) launch_prior(st, ctx->num_sms, X, n, prior, P);
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(p32, params, sizeof(float) * kParams, cudaMemcpyDefault, st));
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(m, 0, sizeof(float) * 2 * kParams, st));
  k_mlp_tobf16<<<1024, 256, 0, st>>>(p32, net.pb, kParams);
  refresh_wt(st, net);
  std::mt19937_64 rng(cfg->seed);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  const int steps_per_epoch = (n + bs - 1) / bs;
  const int total = cfg->epochs * steps_per_epoch;
  const int lblocks = 128;
  // per epoch: the shuffled order goes up once, every step's partial loss sums stay on the
  // device, and the host reads them (and synchronises) once at the end of the epoch
  std::vector<double> ls((size_t)lblocks * steps_per_epoch);
  int t = 0;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(d_idx, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    for (int b = 0; b < steps_per_epoch; ++b) {
      const int rows = std::min(bs, n - b * bs);
      k_mlp_gather<<<512, 256, 0, st>>>(X, d_idx + (size_t)b * bs, rows, IN, shift, scale, net.X, T, net.T, OUT, P);
      rc = forward(ctx, st, net, p32, rows);
      if (rc == KITE_OK) rc = backward(ctx, st, net, rows, lsum + (size_t)b * lblocks, lblocks);
      if (rc != KITE_OK) return rc;
      ++t;
      const AdamwCoeffs c = adamw_coeffs(t, total, cfg->lr);
      k_mlp_adamw<<<1024, 256, 0, st>>>(p32, net.grad, m, v, net.pb, kParams, c.lr, (float)kBeta1,
                                        (float)(1.0 - kBeta1), (float)kBeta2, (float)(1.0 - kBeta2), kAdamEps,
                                        (float)cfg->weight_decay, c.c1, c.c2);
      refresh_wt(st, net);
      KITE_CUDA_TRY(ctx, cudaGetLastError());
    }
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ls.data(), lsum, sizeof(double) * ls.size(), cudaMemcpyDeviceToHost, st));
    KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // the order buffer and ls are reused
    if (loss_curve) loss_curve[ep] = (float)(std::accumulate(ls.begin(), ls.end(), 0.0) / ((double)n * OUT));
  }
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(params, p32, sizeof(float) * kParams, cudaMemcpyDefault, st));
  return read_status(ctx);
}

int mlp_init_impl(kite_ctx* ctx, uint64_t seed, double head_scale, float* p) {
  k_mlp_init<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(p, seed, (float)head_scale);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

int mlp_norm_impl(kite_ctx* ctx, const float* X, int n, double sd_floor, float* shift, float* scale) {
  k_mlp_colstats<<<IN, 256, 0, ctx->stream>>>(X, n, (float)sd_floor, shift, scale);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

int mlp_take_inputs_impl(kite_ctx* ctx, const double* mu, int mu_ld, int n, float* X) {
  const int blocks = (int)std::min<int64_t>(((int64_t)n * IN + 255) / 256, (int64_t)ctx->num_sms * 8);
  k_mlp_take_inputs<<<std::max(1, blocks), 256, 0, ctx->stream>>>(mu, mu_ld, n, X);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

int mlp_narrow_impl(kite_ctx* ctx, const double* src, int K, float* dst) {
  k_mlp_narrow<<<(K + 255) / 256, 256, 0, ctx->stream>>>(src, K, dst);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

int mlp_gate_impl(kite_ctx* ctx, const float* rho, const double* mu, int mu_ld, int n, int kcheck,
                  double de_minus, double tol, int* flags, double* dev) {
  k_mlp_gate<<<n, 128, 0, ctx->stream>>>(rho, mu, mu_ld, kcheck, de_minus, tol, flags, dev);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

}  // namespace kite
