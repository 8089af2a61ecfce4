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
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "kite_device.cuh"
#include "kite_internal.h"

namespace kite {
namespace {

constexpr int IN = KITE_MLP_IN, HID = KITE_MLP_HIDDEN, OUT = KITE_MLP_OUT;
constexpr double kBeta1 = 0.9, kBeta2 = 0.999;
constexpr float kAdamEps = 1e-8f;
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + (int64_t)HID * IN, kOffW2 = kOffB1 + HID,
                  kOffB2 = kOffW2 + (int64_t)HID * HID, kOffW3 = kOffB2 + HID,
                  kOffB3 = kOffW3 + (int64_t)OUT * HID, kParams = kOffB3 + OUT;

// ------------------------------------------------------------------------------------
// GEMM on the tensor cores (BF16 in, FP32 accumulate): C[m][n] = sum_k A(m,k) B(k,n)
//   A(m,k) = transA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = transB ? B[n*ldb + k] : B[k*ldb + n]
// Epilogue: + bias[n]; relu; mask by mask[m][n] > 0; store FP32 (C32) and/or BF16 (C16).
// 64x64 CTA tile, 4 warps of 32x32 (2x2 WMMA 16x16x16 fragments), K step 32 via smem.
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

__global__ void __launch_bounds__(128) k_mlp_gemm(const __nv_bfloat16* __restrict__ A, int lda, int transA,
                                                  const __nv_bfloat16* __restrict__ B, int ldb, int transB,
                                                  int M, int N, int K, const GemmEpi ep) {
  using namespace nvcuda;
  constexpr int BM = 64, BN = 64, BK = 32, PA = BK + 8, PB = BN + 8, PC = BN + 4;
  __shared__ __align__(32) __nv_bfloat16 As[BM][PA];
  __shared__ __align__(32) __nv_bfloat16 Bs[BK][PB];
  __shared__ __align__(32) float Cs[BM][PC];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) wmma::fill_fragment(acc[i][j], 0.0f);
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = transA ? e % BM : e / BK, c = transA ? e / BM : e % BK;
      const int gm = m0 + r, gk = k0 + c;
      As[r][c] = (gm < M && gk < K) ? (transA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk]) : zero;
    }
    for (int e = tid; e < BK * BN; e += 128) {
      const int r = transB ? e % BK : e / BN, c = transB ? e / BK : e % BN;
      const int gk = k0 + r, gn = n0 + c;
      Bs[r][c] = (gk < K && gn < N) ? (transB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn]) : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> fa[2];
      wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) wmma::load_matrix_sync(fa[i], &As[wm + 16 * i][kk], PA);
#pragma unroll
      for (int j = 0; j < 2; ++j) wmma::load_matrix_sync(fb[j], &Bs[kk][wn + 16 * j], PB);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
      wmma::store_matrix_sync(&Cs[wm + 16 * i][wn + 16 * j], acc[i][j], PC, wmma::mem_row_major);
  __syncthreads();
  for (int e = tid; e < BM * BN; e += 128) {
    const int r = e / BN, c = e % BN, gm = m0 + r, gn = n0 + c;
    if (gm >= M || gn >= N) continue;
    float v = ep.alpha * Cs[r][c];
    if (ep.bias) v += ep.bias[gn];
    if (ep.add) v += ep.add[(int64_t)gm * ep.ldc + gn];
    if (ep.relu) v = fmaxf(v, 0.0f);
    if (ep.mask && !(__bfloat162float(ep.mask[(int64_t)gm * ep.ldc + gn]) > 0.0f)) v = 0.0f;
    if (ep.C32) ep.C32[(int64_t)gm * ep.ldc + gn] = v;
    if (ep.C16) ep.C16[(int64_t)gm * ep.ldc + gn] = __float2bfloat16(v);
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
  __nv_bfloat16 *X, *H1, *H2, *dY, *dZ2, *dZ1;
  float *Y, *T, *grad;
};

void gemm(cudaStream_t st, const __nv_bfloat16* A, int lda, int tA, const __nv_bfloat16* B, int ldb, int tB,
          int M, int N, int K, GemmEpi ep) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_mlp_gemm<<<grid, 128, 0, st>>>(A, lda, tA, B, ldb, tB, M, N, K, ep);
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
void forward(cudaStream_t st, const Net& net, const float* p32, int rows, const float* add = nullptr) {
  gemm(st, net.X, IN, 0, net.pb + kOffW1, IN, 1, rows, HID, IN, epi(nullptr, net.H1, HID, p32 + kOffB1, 1));
  gemm(st, net.H1, HID, 0, net.pb + kOffW2, HID, 1, rows, HID, HID, epi(nullptr, net.H2, HID, p32 + kOffB2, 1));
  GemmEpi e3 = epi(net.Y, nullptr, OUT, p32 + kOffB3);
  e3.add = add;
  gemm(st, net.H2, HID, 0, net.pb + kOffW3, HID, 1, rows, OUT, HID, e3);
}

bool use_prior(const kite_mlp_prior* prior) { return prior && prior->kind == KITE_PRIOR_JACKSON; }

void launch_prior(cudaStream_t st, int num_sms, const float* X, int rows, const kite_mlp_prior* prior, float* P) {
  const double a = 0.5 * (prior->e_max - prior->e_min);
  const int blocks = std::max(1, std::min(rows, num_sms * 8));
  k_mlp_prior<<<blocks, 256, 0, st>>>(X, rows, prior_coef(), 1.0 / (3.141592653589793 * a), P);
}

// backward of the mean L1 loss over rows x OUT; gradient into net.grad
void backward(cudaStream_t st, const Net& net, int rows, double* lsum, int lblocks) {
  const int64_t n = (int64_t)rows * OUT;
  k_mlp_l1grad<<<lblocks, 256, 0, st>>>(net.Y, net.T, n, 1.0f / (float)n, net.dY, lsum);
  float* g = net.grad;
  gemm(st, net.dY, OUT, 1, net.H2, HID, 0, OUT, HID, rows, epi(g + kOffW3, nullptr, HID));
  k_mlp_colsum<<<(OUT + 255) / 256, 256, 0, st>>>(net.dY, rows, OUT, g + kOffB3);
  gemm(st, net.dY, OUT, 0, net.pb + kOffW3, HID, 0, rows, HID, OUT, epi(nullptr, net.dZ2, HID, nullptr, 0, net.H2));
  gemm(st, net.dZ2, HID, 1, net.H1, HID, 0, HID, HID, rows, epi(g + kOffW2, nullptr, HID));
  k_mlp_colsum<<<(HID + 255) / 256, 256, 0, st>>>(net.dZ2, rows, HID, g + kOffB2);
  gemm(st, net.dZ2, HID, 0, net.pb + kOffW2, HID, 0, rows, HID, HID, epi(nullptr, net.dZ1, HID, nullptr, 0, net.H1));
  gemm(st, net.dZ1, HID, 1, net.X, IN, 0, HID, IN, rows, epi(g + kOffW1, nullptr, IN));
  k_mlp_colsum<<<(HID + 255) / 256, 256, 0, st>>>(net.dZ1, rows, HID, g + kOffB1);
}

int carve_net(kite_ctx* ctx, int rows, Net* net, float** extra, size_t extra_floats) {
  Carver probe(nullptr);
  auto lay = [&](Carver& k, Net& n, float** ex) {
    n.pb = k.take<__nv_bfloat16>(kParams);
    n.X = k.take<__nv_bfloat16>((size_t)rows * IN);
    n.H1 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.H2 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.dY = k.take<__nv_bfloat16>((size_t)rows * OUT);
    n.dZ2 = k.take<__nv_bfloat16>((size_t)rows * HID);
    n.dZ1 = k.take<__nv_bfloat16>((size_t)rows * HID);
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
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(p32, params, sizeof(float) * kParams, cudaMemcpyDefault, st));
  k_mlp_tobf16<<<1024, 256, 0, st>>>(p32, net.pb, kParams);
  k_mlp_gather<<<1024, 256, 0, st>>>(X, nullptr, n, IN, shift, scale, net.X, T, net.T, OUT);
  forward(st, net, p32, n);
  const int lblocks = 256;
  backward(st, net, n, lsum, lblocks);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(grad, net.grad, sizeof(float) * kParams, cudaMemcpyDefault, st));
  std::vector<double> ls(lblocks);
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ls.data(), lsum, sizeof(double) * lblocks, cudaMemcpyDeviceToHost, st));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
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
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ex, params, sizeof(float) * kParams, cudaMemcpyDefault, st));
  k_mlp_tobf16<<<1024, 256, 0, st>>>(ex, net.pb, kParams);
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int rows = std::min(chunk, n - r0);
    k_mlp_gather<<<1024, 256, 0, st>>>(X + (int64_t)r0 * IN, nullptr, rows, IN, shift, scale, net.X, nullptr,
                                       nullptr, 0);
    float* P = pri ? ex + kParams : nullptr;
    if (pri) launch_prior(st, ctx->num_sms, X + (int64_t)r0 * IN, rows, prior, P);
    forward(st, net, ex, rows, P);
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(Y + (int64_t)r0 * OUT, net.Y, sizeof(float) * rows * OUT, cudaMemcpyDefault, st));
  }
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return KITE_OK;
}

int mlp_train_impl(kite_ctx* ctx, const float* X, const float* T, int n, const float* shift, const float* scale,
                   const kite_mlp_train_cfg* cfg, float* params, float* loss_curve,
                   const kite_mlp_prior* prior) {
  const int bs = std::max(1, std::min(cfg->batch, n));
  Net net;
  float* ex;
  const bool pri = use_prior(prior);
  int rc = carve_net(ctx, bs, &net, &ex, 3 * kParams + 4096 + (size_t)bs + (pri ? (size_t)n * OUT : 0));
  if (rc != KITE_OK) return rc;
  cudaStream_t st = ctx->stream;
  float* p32 = ex;
  float* m = ex + kParams;
  float* v = ex + 2 * kParams;
  double* lsum = reinterpret_cast<double*>(ex + 3 * kParams);
  int* d_idx = reinterpret_cast<int*>(ex + 3 * kParams + 4096);
  // the prior of every training row, once; the batches gather T - prior as targets
  float* P = pri ? ex + 3 * kParams + 4096 + bs : nullptr;
  if (pri) launch_prior(st, ctx->num_sms, X, n, prior, P);
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(p32, params, sizeof(float) * kParams, cudaMemcpyDefault, st));
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(m, 0, sizeof(float) * 2 * kParams, st));
  k_mlp_tobf16<<<1024, 256, 0, st>>>(p32, net.pb, kParams);
  std::mt19937_64 rng(cfg->seed);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  const int steps_per_epoch = (n + bs - 1) / bs;
  const int total = cfg->epochs * steps_per_epoch;
  const int lblocks = 128;
  std::vector<double> ls(lblocks);
  int t = 0;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    double epoch_loss = 0.0;
    for (int b = 0; b < steps_per_epoch; ++b) {
      const int rows = std::min(bs, n - b * bs);
      KITE_CUDA_TRY(ctx, cudaMemcpyAsync(d_idx, order.data() + (size_t)b * bs, sizeof(int) * rows,
                                         cudaMemcpyHostToDevice, st));
      k_mlp_gather<<<512, 256, 0, st>>>(X, d_idx, rows, IN, shift, scale, net.X, T, net.T, OUT, P);
      forward(st, net, p32, rows);
      backward(st, net, rows, lsum, lblocks);
      ++t;
      const AdamwCoeffs c = adamw_coeffs(t, total, cfg->lr);
      k_mlp_adamw<<<1024, 256, 0, st>>>(p32, net.grad, m, v, net.pb, kParams, c.lr, (float)kBeta1,
                                        (float)(1.0 - kBeta1), (float)kBeta2, (float)(1.0 - kBeta2), kAdamEps,
                                        (float)cfg->weight_decay, c.c1, c.c2);
      KITE_CUDA_TRY(ctx, cudaGetLastError());
      KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ls.data(), lsum, sizeof(double) * lblocks, cudaMemcpyDeviceToHost, st));
      KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // d_idx / order reuse
      epoch_loss += std::accumulate(ls.begin(), ls.end(), 0.0);
    }
    if (loss_curve) loss_curve[ep] = (float)(epoch_loss / ((double)n * OUT));
  }
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(params, p32, sizeof(float) * kParams, cudaMemcpyDefault, st));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return KITE_OK;
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
