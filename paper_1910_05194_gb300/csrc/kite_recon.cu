// kite_recon.cu -- FP64 reconstruction of the density of states from raw moments.
//
// rho(E) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(eps)] / (pi sqrt(1-eps^2) de_minus) with
// eps = (E - de_plus)/de_minus: the delta-function expansion of Sec. 2a
// (Delta_n = 2 T_n / (pi sqrt(1-eps^2)), weight 1/(1+delta_n0)) traced as in Eq. e7,
// truncated at M terms (Eq. e8a) and damped by a kernel g_n (Sec. 2a).
#include <math.h>

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

}  // namespace

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
