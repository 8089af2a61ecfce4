// kite_recon.cu -- FP64 reconstruction of the density of states from raw moments.
//
// rho(E) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(eps)] / (pi sqrt(1-eps^2) de_minus) with
// eps = (E - de_plus)/de_minus: the delta-function expansion of Sec. 2a
// (Delta_n = 2 T_n / (pi sqrt(1-eps^2)), weight 1/(1+delta_n0)) traced as in Eq. e7,
// truncated at M terms (Eq. e8a) and damped by a kernel g_n (Sec. 2a).
#include <math.h>

#include <algorithm>

#include <vector>

#include "kite_internal.h"

namespace kite {
namespace {

// c_n = (2 - delta_n0) g_n mu_n, kernel built for M terms.
__global__ void k_dos_coef(const double* __restrict__ mu, int M, int kernel, double param,
                           double* __restrict__ coef) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  double g = 1.0;
  if (kernel == KITE_KERNEL_JACKSON) {
    // Jackson kernel (Weisse et al., Rev. Mod. Phys. 78, 275 (2006)):
    // g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))] / (M+1)
    const double q = 3.141592653589793 / (double)(M + 1);
    const double cot = cos(q) / sin(q);
    g = ((double)(M - n + 1) * cos(q * n) + sin(q * n) * cot) / (double)(M + 1);
  } else if (kernel == KITE_KERNEL_LORENTZ) {
    g = sinh(param * (1.0 - (double)n / (double)M)) / sinh(param);
  }
  coef[n] = (n == 0 ? 1.0 : 2.0) * g * mu[n];
}

// One thread per energy; the Chebyshev polynomials follow the recurrence of Eq. e3.
// Coefficients are staged through shared memory in tiles.
__global__ void k_dos_eval(const double* __restrict__ coef, int M, double de_plus,
                           double de_minus, const double* __restrict__ E, int K,
                           double* __restrict__ rho) {
  __shared__ double tile[1024];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double eps = 0.0;
  bool inside = false;
  if (k < K) {
    eps = (E[k] - de_plus) / de_minus;
    inside = eps > -1.0 && eps < 1.0;
  }
  double tm1 = 1.0, t = eps, sum = 0.0;
  for (int base = 0; base < M; base += 1024) {
    const int len = min(1024, M - base);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) tile[i] = coef[base + i];
    __syncthreads();
    for (int i = 0; i < len; ++i) {
      const int n = base + i;
      if (n == 0) {
        sum += tile[i];
      } else {
        sum += tile[i] * t;
        const double tn = 2.0 * eps * t - tm1;
        tm1 = t;
        t = tn;
      }
    }
  }
  if (k < K) rho[k] = inside ? sum / (3.141592653589793 * sqrt(1.0 - eps * eps)) / de_minus : 0.0;
}

// Average Green's function G(E + i eta) per eV (Eqs. green_function_cheb_expansion/b traced
// as in Eq. e7): sum_n (c_n / 2) g^{+,eta~}_n(eps) / de_minus with c_n = (2 - d_n0) g_n mu_n
// from k_dos_coef, and the retarded CPGF coefficients g_n = -2i q^n / sqrt(1 - z^2),
// q = z - i sqrt(1 - z^2), z = eps + i eta~ (geometric in n).  One thread per energy.
struct gcplx {
  double re, im;
};
__device__ __forceinline__ gcplx gmul(gcplx a, gcplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ gcplx gsqrt(gcplx z) {  // principal branch
  const double r = hypot(z.re, z.im);
  if (r == 0.0) return {0.0, 0.0};
  if (z.re >= 0.0) {
    const double t = sqrt(0.5 * (r + z.re));
    return {t, z.im / (2.0 * t)};
  }
  const double t = sqrt(0.5 * (r - z.re));
  return {fabs(z.im) / (2.0 * t), z.im >= 0.0 ? t : -t};
}

__global__ void k_green_eval(const double* __restrict__ coef, int M, double de_plus, double de_minus,
                             double eta_t, const double* __restrict__ E, int K, double* __restrict__ G,
                             double* __restrict__ rho) {
  __shared__ double tile[1024];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const double eps = k < K ? (E[k] - de_plus) / de_minus : 0.0;
  const gcplx z = {eps, eta_t};
  const gcplx r = gsqrt({1.0 - (z.re * z.re - z.im * z.im), -2.0 * z.re * z.im});
  const gcplx q = {z.re + r.im, z.im - r.re};  // z - i r
  // g_0 = -2i / r
  const double rr = r.re * r.re + r.im * r.im;
  gcplx g = {-2.0 * r.im / rr, -2.0 * r.re / rr};
  double are = 0.0, aim = 0.0;
  for (int base = 0; base < M; base += 1024) {
    const int len = min(1024, M - base);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) tile[i] = 0.5 * coef[base + i];
    __syncthreads();
    for (int i = 0; i < len; ++i) {
      are += tile[i] * g.re;
      aim += tile[i] * g.im;
      g = gmul(g, q);
    }
  }
  if (k < K) {
    if (G) {
      G[2 * k] = are / de_minus;
      G[2 * k + 1] = aim / de_minus;
    }
    if (rho) rho[k] = -aim / de_minus / 3.141592653589793;
  }
}

}  // namespace

int reconstruct_green_impl(kite_ctx* ctx, const double* mu_dev, int M_use, int kernel, double param,
                           const Scale& sc, double eta, const double* E_dev, int K, double* G_dev,
                           double* rho_dev, double* coef_dev) {
  k_dos_coef<<<(M_use + 255) / 256, 256, 0, ctx->stream>>>(mu_dev, M_use, kernel, param, coef_dev);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  k_green_eval<<<(K + 127) / 128, 128, 0, ctx->stream>>>(coef_dev, M_use, sc.de_plus, sc.de_minus,
                                                         eta / sc.de_minus, E_dev, K, G_dev, rho_dev);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

int reconstruct_dos_impl(kite_ctx* ctx, const double* mu_dev, int M_use, int kernel,
                         double param, const Scale& sc, const double* E_dev, int K,
                         double* rho_dev, double* coef_dev) {
  k_dos_coef<<<(M_use + 255) / 256, 256, 0, ctx->stream>>>(mu_dev, M_use, kernel, param, coef_dev);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  k_dos_eval<<<(K + 127) / 128, 128, 0, ctx->stream>>>(coef_dev, M_use, sc.de_plus, sc.de_minus,
                                                       E_dev, K, rho_dev);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

}  // namespace kite

// ====================================================================================
// First-order optical conductivity sigma_xx(omega) from the 2D moments (Sec. 2b):
//   Gamma_nm = -g_n g_m mu_nm / ((1 + d_n0)(1 + d_m0))            (Eq. Gammanm, damped)
//   S(w) = int de f(e) sum_nm Gamma_nm [g^R_n(e + w) Delta_m(e) + Delta_n(e) g^A_m(e - w)]
//   sigma(w) = -i (n_orb a^2/Omega_c) / w * S(w)   [units e^2/hbar, w = hbar omega/de_minus]
// (Eq. conductivity_1st_order in rescaled units).  With e = cos(theta), Delta_m(e) de =
// (2/pi) cos(m theta) d theta, integrated by Gauss-Legendre quadrature in theta.  Then
// U[n][k] = sum_m Gamma_nm D[m][k] and W[m][k] = sum_n Gamma_nm D[n][k] (two FP64 GEMMs),
// and per frequency S = sum_k sum_n (g^R_n(e_k + w) U[n][k] + g^A_n(e_k - w) W[n][k]).
// The CPGF coefficients (Eq. green_function_cheb_expansionb) are geometric in n:
// g^{s}_n(z) = -2 s i q^n / sqrt(1 - z^2) with q = exp(-s i arccos z) = z - s i sqrt(1 - z^2)
// for the principal branches, so only a complex square root is needed per (w, node).
// ====================================================================================
namespace kite {
namespace {

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// principal square root (Re >= 0), cancellation-free in both half planes
__device__ __forceinline__ cplx csqrt_p(cplx z) {
  const double r = hypot(z.re, z.im);
  if (r == 0.0) return {0.0, 0.0};
  if (z.re >= 0.0) {
    const double t = sqrt(0.5 * (r + z.re));
    return {t, z.im / (2.0 * t)};
  }
  const double t = sqrt(0.5 * (r - z.re));
  return {fabs(z.im) / (2.0 * t), z.im >= 0.0 ? t : -t};
}

__global__ void k_sig_gamma(const double* __restrict__ mu, int M_avail, int M, int kernel,
                            double* __restrict__ gam) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * M) return;
  const int n = (int)(e / M), m = (int)(e - (e / M) * M);
  auto jackson = [&](int k) {
    const double q = 3.141592653589793 / (double)(M + 1);
    return ((double)(M - k + 1) * cos(q * k) + sin(q * k) * (cos(q) / sin(q))) / (double)(M + 1);
  };
  double w = (n == 0 ? 0.5 : 1.0) * (m == 0 ? 0.5 : 1.0);
  if (kernel == KITE_KERNEL_JACKSON) w *= jackson(n) * jackson(m);
  const double* p = mu + 2 * ((int64_t)n * M_avail + m);
  gam[2 * e] = -w * p[0];
  gam[2 * e + 1] = -w * p[1];
}

// D[m][k] = (2/pi) cos(m theta_k) w_k
__global__ void k_sig_dmat(const double* __restrict__ theta, const double* __restrict__ wq, int M,
                           int K, double* __restrict__ D) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * K) return;
  const int m = (int)(e / K), k = (int)(e - (e / K) * K);
  D[e] = 0.6366197723675814 * cos((double)m * theta[k]) * wq[k];
}

// C[i][k] = sum_j A(i,j) B[j][k], A complex [M][M] (A(i,j) = G[i][j] or, if trans, G[j][i]),
// B real [M][K], C complex [M][K].  16x16 tiles through shared memory.
__global__ void k_zgemm_real(const double* __restrict__ G, int trans, const double* __restrict__ B,
                             int M, int K, double* __restrict__ Cm) {
  __shared__ double As_re[16][17], As_im[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * 16 + ty, k = blockIdx.x * 16 + tx;
  double re = 0.0, im = 0.0;
  for (int j0 = 0; j0 < M; j0 += 16) {
    const int ia = blockIdx.y * 16 + ty, ja = j0 + tx;
    double ar = 0.0, ai = 0.0;
    if (ia < M && ja < M) {
      const int64_t idx = trans ? (int64_t)ja * M + ia : (int64_t)ia * M + ja;
      ar = G[2 * idx];
      ai = G[2 * idx + 1];
    }
    As_re[ty][tx] = ar;
    As_im[ty][tx] = ai;
    const int jb = j0 + ty;
    Bs[ty][tx] = (jb < M && k < K) ? B[(int64_t)jb * K + k] : 0.0;
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      re += As_re[ty][jj] * Bs[jj][tx];
      im += As_im[ty][jj] * Bs[jj][tx];
    }
    __syncthreads();
  }
  if (i < M && k < K) {
    Cm[2 * ((int64_t)i * K + k)] = re;
    Cm[2 * ((int64_t)i * K + k) + 1] = im;
  }
}

// One block per frequency: S(w) = sum_k [sum_n gR_n(e_k + w) U[n][k] + gA_n(e_k - w) W[n][k]]
__global__ void k_sig_omega(const double* __restrict__ U, const double* __restrict__ W,
                            const double* __restrict__ theta, int M, int K,
                            const double* __restrict__ wt, double eta_t, double factor,
                            double* __restrict__ sigma) {
  const int iw = blockIdx.x;
  const double w = wt[iw];
  double sre = 0.0, sim = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double e = cos(theta[k]);
    // retarded: z = e + w + i eta, g_n = -2i q^n / sqrt(1 - z^2), q = z - i sqrt(1 - z^2)
    // advanced: z = e - w - i eta, g_n = +2i q^n / sqrt(1 - z^2), q = z + i sqrt(1 - z^2)
    for (int sgn = 0; sgn < 2; ++sgn) {
      const double s = sgn == 0 ? 1.0 : -1.0;
      const cplx z = {e + s * w, s * eta_t};
      const cplx one_m_z2 = {1.0 - (z.re * z.re - z.im * z.im), -2.0 * z.re * z.im};
      const cplx r = csqrt_p(one_m_z2);
      const cplx q = {z.re + s * r.im, z.im - s * r.re};  // z - s i r
      cplx g = cdiv({0.0, -2.0 * s}, r);
      const double* X = sgn == 0 ? U : W;
      double ar = 0.0, ai = 0.0;
      for (int n = 0; n < M; ++n) {
        const double xr = X[2 * ((int64_t)n * K + k)], xi = X[2 * ((int64_t)n * K + k) + 1];
        ar += g.re * xr - g.im * xi;
        ai += g.re * xi + g.im * xr;
        g = cmul(g, q);
      }
      sre += ar;
      sim += ai;
    }
  }
  __shared__ double red_re[256], red_im[256];
  red_re[threadIdx.x] = sre;
  red_im[threadIdx.x] = sim;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      red_re[threadIdx.x] += red_re[threadIdx.x + st];
      red_im[threadIdx.x] += red_im[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // sigma = -i * factor / w * S
    const double Sr = red_re[0], Si = red_im[0];
    sigma[2 * iw] = factor / w * Si;
    sigma[2 * iw + 1] = -factor / w * Sr;
  }
}

// ---- DC conductivity (Kubo-Greenwood, T = 0) ---------------------------------------
// One block per energy (grid-stride): the kernel-damped delta coefficients
// c_n = w_n T_n(e) / (pi sqrt(1 - e^2)), w_n = (2 - delta_n0) g_n, in shared memory; each
// warp contracts whole rows, s = sum_n c_n sum_m Re(mu_nm) c_m, then a fixed-order sum
// over the warps.  sigma_k = pi ucf s (0 outside |e| < 1).  FP64 throughout.
__global__ void k_sigma_dc(const double* __restrict__ mu, int M_avail, int M, const double* __restrict__ w,
                           double de_plus, double de_minus, const double* __restrict__ E, int K, double ucf,
                           double* __restrict__ sigma) {
  extern __shared__ double c[];  // [M] + [blockDim/32]
  double* wsum = c + M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int k = blockIdx.x; k < K; k += gridDim.x) {
    const double e = (E[k] - de_plus) / de_minus;
    if (!(fabs(e) < 1.0)) {
      if (threadIdx.x == 0) sigma[k] = 0.0;
      continue;  // uniform across the block
    }
    const double th = acos(e), den = 3.141592653589793 * sqrt(1.0 - e * e);
    for (int n = threadIdx.x; n < M; n += blockDim.x) c[n] = w[n] * cos((double)n * th) / den;
    __syncthreads();
    double acc = 0.0;
    for (int n = warp; n < M; n += nwarp) {
      const double* row = mu + 2 * (size_t)n * M_avail;
      double r = 0.0;
      for (int m = lane; m < M; m += 32) r += row[2 * m] * c[m];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
      acc += c[n] * r;
    }
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int q = 0; q < nwarp; ++q) sum += wsum[q];
      sigma[k] = 3.141592653589793 * ucf * sum;
    }
    __syncthreads();
  }
}

// w_n = (2 - delta_n0) g_n for the kernel built for M terms
__global__ void k_dc_weights(int M, int kernel, double param, double* __restrict__ w) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  double g = 1.0;
  if (kernel == KITE_KERNEL_JACKSON) {
    const double q = 3.141592653589793 / (double)(M + 1);
    g = ((double)(M - n + 1) * cos(q * n) + sin(q * n) * (cos(q) / sin(q))) / (double)(M + 1);
  } else if (kernel == KITE_KERNEL_LORENTZ) {
    g = sinh(param * (1.0 - (double)n / (double)M)) / sinh(param);
  }
  w[n] = (n == 0 ? 1.0 : 2.0) * g;
}

}  // namespace

// Gauss-Legendre nodes/weights on [-1, 1] (Newton iteration on P_K from the three-term
// recurrence), host FP64.
void gauss_legendre(int K, double* x, double* w) {
  const double pi = 3.141592653589793;
  for (int i = 0; i < (K + 1) / 2; ++i) {
    double z = cos(pi * (i + 0.75) / (K + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= K; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = K * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= K; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = K * (z * p0 - p1) / (z * z - 1.0);
    }
    x[i] = -z;
    x[K - 1 - i] = z;
    w[i] = w[K - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

int reconstruct_sigma_impl(kite_ctx* ctx, const double* mu_dev, int M_avail, int M, int lattice,
                           int kernel, const Scale& sc, double E_F, double kT, double eta,
                           const double* omega_host, int K_w, int n_quad, double* sigma_dev) {
  const int K = n_quad > 0 ? n_quad : 2 * M + 64;
  const double eF = (E_F - sc.de_plus) / sc.de_minus;
  const double thF = kT > 0.0 ? 0.0 : acos(fmin(1.0, fmax(-1.0, eF)));
  std::vector<double> x(K), wq(K), th(K), wts(2 * (size_t)K_w);
  gauss_legendre(K, x.data(), wq.data());
  const double pi = 3.141592653589793;
  for (int k = 0; k < K; ++k) {
    th[k] = thF + (pi - thF) * 0.5 * (x[k] + 1.0);
    wq[k] *= 0.5 * (pi - thF);
    if (kT > 0.0) {
      const double E = cos(th[k]) * sc.de_minus + sc.de_plus;
      wq[k] /= (1.0 + exp((E - E_F) / kT));
    }
  }
  for (int i = 0; i < K_w; ++i) wts[i] = omega_host[i] / sc.de_minus;
  const size_t nG = 2 * (size_t)M * M, nD = (size_t)M * K, nU = 2 * (size_t)M * K;
  double* buf = nullptr;
  const size_t total = nG + nD + 2 * nU + 2 * (size_t)K + K_w;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, total * sizeof(double), ctx->stream));
  double* G = buf;
  double* D = G + nG;
  double* U = D + nD;
  double* W = U + nU;
  double* th_d = W + nU;
  double* wq_d = th_d + K;
  double* wt_d = wq_d + K;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(th_d, th.data(), K * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(wq_d, wq.data(), K * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(wt_d, wts.data(), K_w * sizeof(double), cudaMemcpyHostToDevice, st);
  int rc = e == cudaSuccess ? KITE_OK : cuda_fail(ctx, e, "sigma set-up");
  if (rc == KITE_OK) {
    k_sig_gamma<<<(int)(((int64_t)M * M + 255) / 256), 256, 0, st>>>(mu_dev, M_avail, M, kernel, G);
    k_sig_dmat<<<(int)(((int64_t)M * K + 255) / 256), 256, 0, st>>>(th_d, wq_d, M, K, D);
    dim3 blk(16, 16), grd((K + 15) / 16, (M + 15) / 16);
    k_zgemm_real<<<grd, blk, 0, st>>>(G, 0, D, M, K, U);
    k_zgemm_real<<<grd, blk, 0, st>>>(G, 1, D, M, K, W);
    const double factor = lattice == KITE_HONEYCOMB ? 4.0 / sqrt(3.0) : 1.0;
    k_sig_omega<<<K_w, 256, 0, st>>>(U, W, th_d, M, K, wt_d, eta / sc.de_minus, factor, sigma_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "sigma kernels");
  }
  cudaFreeAsync(buf, st);
  return rc;
}

}  // namespace kite

namespace kite {

// sigma_DC(E_k) for K energies from the leading M x M block of mu_nm (device pointers);
// w is device scratch of M doubles.
int reconstruct_sigma_dc_impl(kite_ctx* ctx, const double* mu_dev, int M_avail, int M, int kernel, double param,
                              int lattice, const Scale& sc, const double* E_dev, int K, double* sigma_dev,
                              double* w) {
  cudaStream_t st = ctx->stream;
  k_dc_weights<<<(M + 255) / 256, 256, 0, st>>>(M, kernel, param, w);
  const int block = 256;
  const size_t smem = sizeof(double) * ((size_t)M + block / 32);
  if (smem > 48 * 1024)
    KITE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sigma_dc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::max(1, std::min(K, ctx->num_sms * 4));
  const double ucf = lattice == KITE_HONEYCOMB ? 2.0 * 2.0 / sqrt(3.0) : 1.0;
  k_sigma_dc<<<grid, block, smem, st>>>(mu_dev, M_avail, M, w, sc.de_plus, sc.de_minus, E_dev, K, ucf,
                                         sigma_dev);
  KITE_CUDA_TRY(ctx, cudaGetLastError());
  return KITE_OK;
}

}  // namespace kite

// ====================================================================================
// DC conductivity tensor from the Kubo-Bastin formula, Fermi sea included (the Hall
// conductivity of the paper's quantum anomalous Hall example, Sec. 2b at omega -> 0):
//   sigma_ab(E_F) = Re{ i ucf int de f(e) sum_nm mu_nm [Delta_n(e) dG^R_m(e) - dG^A_n(e) Delta_m(e)] }
// with Delta_n(e) de = k_n (2 - d_n0)/pi cos(n theta) d theta (e = cos theta), the CPGF
// coefficients G^{R/A}_m(e) = k_m g^{+-}_m(e +- i eta)/(1 + d_m0) (Eq.
// green_function_cheb_expansionb) and their derivatives
//   d g_m/dz = g_m(z) [s i m / sqrt(1 - z^2) + z / (1 - z^2)]   (s = +1 retarded, -1 advanced).
// A_nm = mu_nm k_n k_m / ((1 + d_n0)(1 + d_m0)).  Each Fermi energy has its own
// Gauss-Legendre nodes theta_k on [theta_F, pi] (kT > 0: [0, pi] with Fermi weights);
// D[n][k] = (2/pi) cos(n theta_k) w_k, U = A^T D, W = A D (FP64 GEMMs), and per node
//   F_k = sum_m dG^R_m(e_k) U[m][k] - sum_n dG^A_n(e_k) W[n][k],
// the CPGF terms geometric, g_m = g_0 q^m with q = z - s i sqrt(1 - z^2), summed as
// S0 = sum_m g_m X_m and S1 = sum_m m g_m X_m:  sum_m dg_m X_m = s i S1 / r + z S0 / r^2,
// r = sqrt(1 - z^2).  sigma = Re(i ucf sum_k F_k) = -ucf Im(sum_k F_k), each energy's
// node sum in a fixed order.  Cost: two M x M x (K nodes) GEMMs per energy.
// ====================================================================================
namespace kite {
namespace {

__global__ void k_bastin_gamma(const double* __restrict__ mu, int M_avail, int M, const double* __restrict__ w,
                               double* __restrict__ A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * M) return;
  const int n = (int)(e / M), m = (int)(e - (e / M) * M);
  // w_n = (2 - d_n0) k_n, so w_n / 2 = k_n / (1 + d_n0)
  const double f = 0.25 * w[n] * w[m];
  const double* p = mu + 2 * ((int64_t)n * M_avail + m);
  A[2 * e] = f * p[0];
  A[2 * e + 1] = f * p[1];
}

__global__ void k_bastin_nodes(const double* __restrict__ U, const double* __restrict__ W,
                               const double* __restrict__ theta, int M, int64_t Kt, double eta_t,
                               double* __restrict__ F) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Kt; k += (int64_t)gridDim.x * blockDim.x) {
    const double e = cos(theta[k]);
    cplx tot = {0.0, 0.0};
    for (int sgn = 0; sgn < 2; ++sgn) {
      const double s = sgn == 0 ? 1.0 : -1.0;
      const cplx z = {e, s * eta_t};
      const cplx r = csqrt_p({1.0 - (z.re * z.re - z.im * z.im), -2.0 * z.re * z.im});
      const cplx q = {z.re + s * r.im, z.im - s * r.re};  // z - s i r
      cplx g = cdiv({0.0, -2.0 * s}, r);
      const double* X = sgn == 0 ? U : W;
      cplx S0 = {0.0, 0.0}, S1 = {0.0, 0.0};
      for (int m = 0; m < M; ++m) {
        const cplx x = {X[2 * ((int64_t)m * Kt + k)], X[2 * ((int64_t)m * Kt + k) + 1]};
        const cplx gx = cmul(g, x);
        S0.re += gx.re;
        S0.im += gx.im;
        S1.re += (double)m * gx.re;
        S1.im += (double)m * gx.im;
        g = cmul(g, q);
      }
      const cplx a = cdiv(S1, r);
      const cplx b = cdiv(cmul(z, S0), cmul(r, r));
      const cplx d = {-s * a.im + b.re, s * a.re + b.im};  // s i a + b
      tot.re += s * d.re;
      tot.im += s * d.im;
    }
    F[2 * k] = tot.re;
    F[2 * k + 1] = tot.im;
  }
}

// one block per energy: sigma = -ucf * sum_k Im F_k over that energy's K nodes
__global__ void k_bastin_sum(const double* __restrict__ F, int K, double ucf, double* __restrict__ sigma) {
  const double* f = F + 2 * (int64_t)blockIdx.x * K;
  double acc = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) acc += f[2 * k + 1];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) sigma[blockIdx.x] = -ucf * red[0];
}

}  // namespace

int reconstruct_sigma_bastin_impl(kite_ctx* ctx, const double* mu_dev, int M_avail, int M, int lattice,
                                  int kernel, double param, const Scale& sc, double eta, double kT,
                                  const double* E_host, int K_E, int n_quad, double* sigma_dev) {
  const int K = n_quad > 0 ? n_quad : 2 * M + 64;
  std::vector<double> x(K), w0(K);
  gauss_legendre(K, x.data(), w0.data());
  // energies per batch: D (M K), U and W (2 M K each), theta, weights, F (2 K) doubles
  const size_t per_energy = (size_t)K * (5 * (size_t)M + 4);
  const size_t budget = (size_t)1 << 27;  // doubles (1 GiB)
  const int EB = (int)std::max<size_t>(1, std::min<size_t>((size_t)K_E, budget / per_energy));
  const size_t Kt_max = (size_t)EB * K;
  const size_t nA = 2 * (size_t)M * M;
  const size_t total = nA + (size_t)M + Kt_max * (5 * (size_t)M + 4);
  double* buf = nullptr;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, total * sizeof(double), ctx->stream));
  double* A = buf;
  double* wk = A + nA;
  double* D = wk + M;
  double* U = D + (size_t)M * Kt_max;
  double* W = U + 2 * (size_t)M * Kt_max;
  double* th_d = W + 2 * (size_t)M * Kt_max;
  double* wq_d = th_d + Kt_max;
  double* F = wq_d + Kt_max;
  cudaStream_t st = ctx->stream;
  const double pi = 3.141592653589793;
  const double ucf = lattice == KITE_HONEYCOMB ? 4.0 / sqrt(3.0) : 1.0;
  k_dc_weights<<<(M + 255) / 256, 256, 0, st>>>(M, kernel, param, wk);
  k_bastin_gamma<<<(int)(((int64_t)M * M + 255) / 256), 256, 0, st>>>(mu_dev, M_avail, M, wk, A);
  cudaError_t e = cudaGetLastError();
  int rc = e == cudaSuccess ? KITE_OK : cuda_fail(ctx, e, "Bastin set-up");
  std::vector<double> th(Kt_max), wq(Kt_max);
  for (int b = 0; b < K_E && rc == KITE_OK; b += EB) {
    const int nb = std::min(EB, K_E - b);
    const int64_t Kt = (int64_t)nb * K;
    for (int i = 0; i < nb; ++i) {
      const double EF = E_host[b + i];
      const double eF = (EF - sc.de_plus) / sc.de_minus;
      const double thF = kT > 0.0 ? 0.0 : acos(fmin(1.0, fmax(-1.0, eF)));
      for (int k = 0; k < K; ++k) {
        double t = thF + (pi - thF) * 0.5 * (x[k] + 1.0), ww = w0[k] * 0.5 * (pi - thF);
        if (kT > 0.0) ww /= (1.0 + exp((cos(t) * sc.de_minus + sc.de_plus - EF) / kT));
        th[(size_t)i * K + k] = t;
        wq[(size_t)i * K + k] = ww;
      }
    }
    e = cudaMemcpyAsync(th_d, th.data(), Kt * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wq_d, wq.data(), Kt * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      rc = cuda_fail(ctx, e, "Bastin nodes");
      break;
    }
    k_sig_dmat<<<(int)(((int64_t)M * Kt + 255) / 256), 256, 0, st>>>(th_d, wq_d, M, (int)Kt, D);
    dim3 blk(16, 16), grd((unsigned)((Kt + 15) / 16), (unsigned)((M + 15) / 16));
    k_zgemm_real<<<grd, blk, 0, st>>>(A, 1, D, M, (int)Kt, U);  // U[m][k] = sum_n A_nm D[n][k]
    k_zgemm_real<<<grd, blk, 0, st>>>(A, 0, D, M, (int)Kt, W);  // W[n][k] = sum_m A_nm D[m][k]
    const int nblk = (int)std::min<int64_t>((Kt + 255) / 256, (int64_t)ctx->num_sms * 8);
    k_bastin_nodes<<<nblk, 256, 0, st>>>(U, W, th_d, M, Kt, eta / sc.de_minus, F);
    k_bastin_sum<<<nb, 256, 0, st>>>(F, K, ucf, sigma_dev + b);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "Bastin kernels");
    // the host node arrays are refilled next batch: let this batch's copies finish
    if (rc == KITE_OK && b + EB < K_E) {
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "Bastin batch");
    }
  }
  cudaFreeAsync(buf, st);
  return rc;
}

}  // namespace kite
