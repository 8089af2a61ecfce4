// kite_capi.cu -- context, argument validation and the extern "C" entry points of
// libkite_gb.so.  All compute runs in the kernels of the other translation units.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "kite_internal.h"

namespace kite {

int moments_1d_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
                    double* mu_dev, double* imag_dev, double* mu_vec_dev, kite_stats* st,
                    const double* r0_dev_all);
int64_t mlp_param_count();
int mlp_gradient_impl(kite_ctx* ctx, const float* params, const float* X, const float* T, int n,
                      const float* shift, const float* scale, float* grad, double* loss);
int mlp_forward_impl(kite_ctx* ctx, const float* params, const float* X, int n, const float* shift,
                     const float* scale, float* Y, const kite_mlp_prior* prior);
int mlp_train_impl(kite_ctx* ctx, const float* X, const float* T, int n, const float* shift, const float* scale,
                   const kite_mlp_train_cfg* cfg, float* params, float* loss_curve,
                   const kite_mlp_prior* prior);
int mlp_gate_impl(kite_ctx* ctx, const float* rho, const double* mu, int mu_ld, int n, int kcheck,
                  double de_minus, double tol, int* flags, double* dev);
int moments_1d_batched_impl(kite_ctx* ctx, int count, const kite_system* sys, const kite_kpm* kpm,
                            const std::vector<Scale>& scales, double* const* mu, kite_stats* st);
int moments_2d_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc, int alpha,
                    int beta, double* mu_nm_dev, kite_stats* st, const double* r0_dev_all);
int inner_products_impl(kite_ctx* ctx, const float* A, const float* B, int M, int M2, int64_t N,
                        double scale, double* C, int sub_kb, int fold, int nprod);
int reconstruct_sigma_dc_impl(kite_ctx* ctx, const double* mu_dev, int M_avail, int M, int kernel, double param,
                              int lattice, const Scale& sc, const double* E_dev, int K, double* sigma_dev,
                              double* w);
int reconstruct_sigma_bastin_impl(kite_ctx* ctx, const double* mu_dev, int M_avail, int M, int lattice,
                                  int kernel, double param, const Scale& sc, double eta, double kT,
                                  const double* E_host, int K_E, int n_quad, double* sigma_dev);
int reconstruct_sigma_impl(kite_ctx* ctx, const double* mu_dev, int M_avail, int M, int lattice,
                           int kernel, const Scale& sc, double E_F, double kT, double eta,
                           const double* omega_host, int K_w, int n_quad, double* sigma_dev);
int spectral_k_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
                    const double* k, int nk, const double* w, double* out, kite_stats* st);
int ldos_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc,
              const int64_t* orb, int n, double* out, kite_stats* st);
int propagate_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc, double dt,
                   int nsteps, double* psi, double* norms, kite_stats* st);
void evolution_coeffs(int M, double dt, double de_plus, double de_minus, double* coef);
int reconstruct_green_impl(kite_ctx* ctx, const double* mu_dev, int M_use, int kernel, double param,
                           const Scale& sc, double eta, const double* E_dev, int K, double* G_dev,
                           double* rho_dev, double* coef_dev);
int reconstruct_dos_impl(kite_ctx* ctx, const double* mu_dev, int M_use, int kernel,
                         double param, const Scale& sc, const double* E_dev, int K,
                         double* rho_dev, double* coef_dev);

int fail(kite_ctx* ctx, int status, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return status;
}

int cuda_fail(kite_ctx* ctx, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error where possible
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? KITE_ERR_OOM : KITE_ERR_CUDA, m);
}

int ensure_ws(kite_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return KITE_OK;
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&ctx->ws, bytes);
    want = bytes;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(ctx, KITE_ERR_OOM,
                "work space of " + std::to_string(bytes >> 20) + " MiB could not be allocated");
  }
  ctx->ws_bytes = want;
  return KITE_OK;
}

int open_zeros(kite_ctx* ctx, const kite_system* sys, const void** out) {
  *out = nullptr;
  if (!sys->open_x && !sys->open_y) return KITE_OK;
  const size_t bytes = ((size_t)sys->Lx + 64) * 128;
  if (bytes > ctx->zeros_bytes) {
    if (ctx->zeros) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->zeros);
      ctx->zeros = nullptr;
      ctx->zeros_bytes = 0;
    }
    if (cudaMalloc(&ctx->zeros, bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->zeros = nullptr;
      return fail(ctx, KITE_ERR_OOM, "zero row of the open boundaries could not be allocated");
    }
    cudaError_t e = cudaMemsetAsync(ctx->zeros, 0, bytes, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "zero row");
    ctx->zeros_bytes = bytes;
  }
  *out = ctx->zeros;
  return KITE_OK;
}

int ensure_pinned(kite_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->pinned_bytes) return KITE_OK;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  if (cudaMallocHost(&ctx->pinned, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KITE_ERR_OOM, "pinned staging buffer");
  }
  ctx->pinned_bytes = bytes;
  return KITE_OK;
}

int ensure_aux(kite_ctx* ctx) {
  if (ctx->aux) return KITE_OK;
  if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->aux = nullptr;
    cudaGetLastError();
    return fail(ctx, KITE_ERR_CUDA, "second stream");
  }
  if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KITE_ERR_CUDA, "fork/join events");
  }
  return KITE_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int device_view(kite_ctx* ctx, const void* p, size_t bytes, const void** out) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    a.type = cudaMemoryTypeUnregistered;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    *out = p;
    return KITE_OK;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *out = a.devicePointer;
    return KITE_OK;
  }
  if (bytes > ctx->stage_bytes) {
    KITE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    if (cudaMalloc(&ctx->stage, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, KITE_ERR_OOM, "staging buffer for caller start vectors");
    }
    ctx->stage_bytes = bytes;
  }
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->stage, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *out = ctx->stage;
  return KITE_OK;
}

cudaError_t copy_in(kite_ctx* ctx, void* dst_dev, const void* src, size_t bytes) {
  return cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDefault, ctx->stream);
}

cudaError_t copy_out(kite_ctx* ctx, void* dst, const void* src_dev, size_t bytes) {
  return cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, ctx->stream);
}

// Landau-gauge Peierls phases repeat after Ly rows iff flux * Ly * |dx| is an integer for
// every bond: |dx| = 1/2 (honeycomb) or 1 (square), i.e. flux * Ly even or integer.
static double flux_quantum_step(const kite_system* s) {
  return (s->lattice == KITE_HONEYCOMB ? 2.0 : 1.0) / (double)s->Ly;
}
static bool flux_fits(const kite_system* s) {
  if (s->open_y) return true;  // no bond wraps in y: any flux
  const double q = s->flux / flux_quantum_step(s);
  return fabs(q - nearbyint(q)) <= 1e-9 * fmax(1.0, fabs(q));
}
static double nearest_flux(const kite_system* s, double flux) {
  if (s->open_y) return flux;
  const double step = flux_quantum_step(s);
  return nearbyint(flux / step) * step;
}

static int validate_system(kite_ctx* ctx, const kite_system* s) {
  if (!s) return fail(ctx, KITE_ERR_ARG, "system is NULL");
  if (s->lattice != KITE_HONEYCOMB && s->lattice != KITE_SQUARE)
    return fail(ctx, KITE_ERR_ARG, "unknown lattice");
  if (s->Lx < 1 || s->Ly < 1) return fail(ctx, KITE_ERR_ARG, "Lx and Ly must be >= 1");
  if ((s->open_x != 0 && s->open_x != 1) || (s->open_y != 0 && s->open_y != 1))
    return fail(ctx, KITE_ERR_ARG, "open_x and open_y must be 0 (periodic) or 1 (open)");
  const double cells = (double)s->Lx * (double)s->Ly;
  if (cells * (s->lattice == KITE_HONEYCOMB ? 2 : 1) > 4.0e9)
    return fail(ctx, KITE_ERR_ARG, "more than 4e9 orbitals");
  if (!isfinite(s->t) || !isfinite(s->W) || !isfinite(s->delta) || s->W < 0.0)
    return fail(ctx, KITE_ERR_ARG, "t, W, delta must be finite and W >= 0");
  if (!(s->p_vac >= 0.0 && s->p_vac <= 1.0)) return fail(ctx, KITE_ERR_ARG, "p_vac outside [0,1]");
  if (s->disorder != KITE_DISORDER_UNIFORM && s->disorder != KITE_DISORDER_GAUSSIAN)
    return fail(ctx, KITE_ERR_ARG, "disorder must be KITE_DISORDER_UNIFORM or KITE_DISORDER_GAUSSIAN");
  if (!isfinite(s->flux)) return fail(ctx, KITE_ERR_ARG, "flux must be finite");
  if (s->flux != 0.0 && !flux_fits(s)) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "flux %.9g per cell does not fit the torus in the Landau gauge (flux * Ly must be %s); "
             "nearest: %.9g",
             s->flux, s->lattice == KITE_HONEYCOMB ? "even" : "an integer", nearest_flux(s, s->flux));
    return fail(ctx, KITE_ERR_ARG, msg);
  }
  return KITE_OK;
}

static void gershgorin(const kite_system* s, double* lo, double* hi) {
  const double Z = s->lattice == KITE_HONEYCOMB ? 3.0 : 4.0;
  // Gaussian draws satisfy |z| <= sqrt(-2 ln 2^-53) = sqrt(106 ln 2) < 8.58 (k_onsite)
  const double vd = s->disorder == KITE_DISORDER_GAUSSIAN ? 8.58 * fabs(s->W) : 0.5 * fabs(s->W);
  const double vmax = vd + (s->lattice == KITE_HONEYCOMB ? 0.5 * fabs(s->delta) : 0.0);
  const double b = (Z * fabs(s->t) + vmax) * 1.01;
  *lo = -b;
  *hi = b;
}

int resolve_bounds(kite_ctx* ctx, const kite_system* sys, double e_min, double e_max, Scale* sc) {
  if (e_min == 0.0 && e_max == 0.0) {
    gershgorin(sys, &e_min, &e_max);
  }
  if (!(e_max > e_min) || !isfinite(e_min) || !isfinite(e_max))
    return fail(ctx, KITE_ERR_ARG, "e_max must exceed e_min");
  sc->e_min = e_min;
  sc->e_max = e_max;
  sc->de_plus = 0.5 * (e_max + e_min);
  sc->de_minus = 0.5 * (e_max - e_min);
  return KITE_OK;
}

int check_prior(kite_ctx* ctx, const kite_mlp_prior* prior) {
  if (!prior) return KITE_OK;
  if ((prior->kind != KITE_PRIOR_NONE && prior->kind != KITE_PRIOR_JACKSON) || prior->reserved != 0 ||
      !(prior->e_max > prior->e_min) || !std::isfinite(prior->e_min) || !std::isfinite(prior->e_max))
    return fail(ctx, KITE_ERR_ARG, "prior: kind must be KITE_PRIOR_NONE/JACKSON, reserved 0, e_max > e_min");
  return KITE_OK;
}

}  // namespace kite

using namespace kite;

extern "C" {

const char* kite_status_string(int status) {
  switch (status) {
    case KITE_OK: return "ok";
    case KITE_ERR_ARG: return "invalid argument";
    case KITE_ERR_OOM: return "out of device memory";
    case KITE_ERR_CUDA: return "CUDA error";
    case KITE_ERR_BOUNDS: return "moments out of bounds (spectrum outside [-1,1] after rescaling)";
    case KITE_ERR_TIMEOUT: return "device-side wait timed out";
    case KITE_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char* kite_last_error(const kite_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int kite_create(kite_ctx** out, int device, void* cuda_stream) {
  if (!out) return KITE_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return KITE_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return KITE_ERR_CUDA;
  kite_ctx* c = new kite_ctx();
  c->device = device;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return KITE_ERR_CUDA;
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    // a blocking stream: ordered with work the caller left on the legacy default stream
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault) != cudaSuccess) {
      delete c;
      return KITE_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreate(&c->ev2) != cudaSuccess || cudaEventCreate(&c->ev3) != cudaSuccess) {
    delete c;
    return KITE_ERR_CUDA;
  }
  if (cudaMalloc(&c->d_status, 256) != cudaSuccess || cudaMemset(c->d_status, 0, 256) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return KITE_ERR_CUDA;
  }
  // Keep memory freed with cudaFreeAsync cached in the device pool between calls
  // (a per-process setting of this process's pool; nothing outlives the process).
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  *out = c;
  return KITE_OK;
}

void kite_destroy(kite_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->zeros) cudaFree(ctx->zeros);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->ev2) cudaEventDestroy(ctx->ev2);
  if (ctx->ev3) cudaEventDestroy(ctx->ev3);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int kite_set_stream(kite_ctx* ctx, void* cuda_stream) {
  if (!ctx) return KITE_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  ctx->own_stream = false;
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamDefault) != cudaSuccess)
      return fail(ctx, KITE_ERR_CUDA, "stream creation failed");
    ctx->own_stream = true;
  }
  return KITE_OK;
}

int kite_debug_stall_once(kite_ctx* ctx, int enable) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->debug_stall = enable ? 1 : 0;
  return KITE_OK;
}

int kite_bounds(const kite_system* sys, double* e_min, double* e_max) {
  if (!e_min || !e_max) return KITE_ERR_ARG;
  int rc = validate_system(nullptr, sys);
  if (rc != KITE_OK) return rc;
  gershgorin(sys, e_min, e_max);
  return KITE_OK;
}

int kite_flux_nearest(const kite_system* sys, double flux, double* out) {
  if (!sys || !out || !isfinite(flux)) return KITE_ERR_ARG;
  if ((sys->lattice != KITE_HONEYCOMB && sys->lattice != KITE_SQUARE) || sys->Ly < 1) return KITE_ERR_ARG;
  *out = nearest_flux(sys, flux);
  return KITE_OK;
}

int kite_moments_1d(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, double* mu,
                    double* mu_per_vec, kite_stats* st) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  int rc = validate_system(ctx, sys);
  if (rc != KITE_OK) return rc;
  if (!kpm || !mu) return fail(ctx, KITE_ERR_ARG, "kpm and mu are required");
  if (kpm->M < 1 || kpm->R < 1 || kpm->S < 1)
    return fail(ctx, KITE_ERR_ARG, "M, R and S must be >= 1");
  if (kpm->precision != KITE_FP32 && kpm->precision != KITE_FP64)
    return fail(ctx, KITE_ERR_ARG, "precision must be KITE_FP32 or KITE_FP64");
  if ((double)kpm->R * kpm->S > 65536.0) return fail(ctx, KITE_ERR_ARG, "R*S > 65536");
  if (sys->flux != 0.0 && kpm->real_vectors)
    return fail(ctx, KITE_ERR_ARG, "a magnetic field makes H complex: use complex start vectors");
  if ((kpm->doubling != 0 && kpm->doubling != 1) || (kpm->real_vectors != 0 && kpm->real_vectors != 1))
    return fail(ctx, KITE_ERR_ARG, "doubling and real_vectors must be 0 or 1");
  if (kpm->real_vectors && kpm->r_last)
    return fail(ctx, KITE_ERR_ARG, "r_last is not available with real vectors");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc;
  rc = resolve_bounds(ctx, sys, kpm->e_min, kpm->e_max, &sc);
  if (rc != KITE_OK) return rc;

  const int M = kpm->M;
  const size_t nvec = (size_t)kpm->R * kpm->S;
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  // Caller start vectors: read in place (device or page-locked host memory) or staged in a
  // buffer of their own, so the sweep's work space stays put.
  const double* r0_dev = nullptr;
  if (kpm->r0) {
    const void* v = nullptr;
    rc = device_view(ctx, kpm->r0, nvec * (size_t)N * 2 * sizeof(double), &v);
    if (rc != KITE_OK) return rc;
    r0_dev = static_cast<const double*>(v);
  }
  // outputs: device staging for mu, imag and per-vector moments
  double* out_dev = nullptr;
  const size_t out_doubles = 2 * (size_t)M + nvec * (size_t)M * 2;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&out_dev, out_doubles * sizeof(double), ctx->stream));
  double* mu_dev = out_dev;
  double* imag_dev = out_dev + M;
  double* mu_vec_dev = out_dev + 2 * (size_t)M;
  kite_stats local{};
  rc = moments_1d_impl(ctx, sys, kpm, sc, mu_dev, imag_dev, mu_vec_dev, &local, r0_dev);
  if (rc == KITE_OK) {
    std::vector<double> host(2 * (size_t)M);
    cudaError_t e = cudaMemcpyAsync(host.data(), out_dev, 2 * (size_t)M * sizeof(double),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = copy_out(ctx, mu, mu_dev, (size_t)M * sizeof(double));
    if (e == cudaSuccess && mu_per_vec)
      e = copy_out(ctx, mu_per_vec, mu_vec_dev, nvec * (size_t)M * 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(ctx, e, "copying moments out");
    } else {
      double max_im = 0.0;
      bool ok = true;
      for (int n = 0; n < M; ++n) {
        const double re = host[n], im = host[M + n];
        if (!isfinite(re) || !isfinite(im) || fabs(re) > 1.0 + 1e-3) ok = false;
        max_im = fmax(max_im, fabs(im));
      }
      local.max_abs_imag = max_im;
      local.e_min = sc.e_min;
      local.e_max = sc.e_max;
      if (!ok)
        rc = fail(ctx, KITE_ERR_BOUNDS,
                  "a moment is non-finite or exceeds 1 in magnitude: the spectrum of the "
                  "rescaled Hamiltonian is not inside [-1,1]");
    }
  }
  cudaFreeAsync(out_dev, ctx->stream);  // stream-ordered: the copies above have completed
  if (st) *st = local;
  return rc;
}

int64_t kite_mlp_param_count(void) { return mlp_param_count(); }


int kite_mlp_train(kite_ctx* ctx, const float* X, const float* T, int n, const float* shift,
                   const float* scale, const kite_mlp_train_cfg* cfg, float* params, float* loss_curve,
                   const kite_mlp_prior* prior) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!X || !T || !cfg || !params || n < 1 || cfg->epochs < 1 || cfg->batch < 1 || !(cfg->lr > 0.0) ||
      !(cfg->weight_decay >= 0.0))
    return fail(ctx, KITE_ERR_ARG, "need X, T, params, n >= 1 and a valid configuration");
  if (check_prior(ctx, prior) != KITE_OK) return KITE_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Staging sg{ctx, {}};
  const float *Xd, *Td, *Hd, *Sd;
  int rc = sg.in(X, (size_t)n * KITE_MLP_IN, &Xd);
  if (rc == KITE_OK) rc = sg.in(T, (size_t)n * KITE_MLP_OUT, &Td);
  if (rc == KITE_OK) rc = sg.in(shift, KITE_MLP_IN, &Hd);
  if (rc == KITE_OK) rc = sg.in(scale, KITE_MLP_IN, &Sd);
  std::vector<float> curve(cfg->epochs);
  if (rc == KITE_OK) rc = mlp_train_impl(ctx, Xd, Td, n, Hd, Sd, cfg, params, curve.data(), prior);
  if (rc == KITE_OK && loss_curve) std::copy(curve.begin(), curve.end(), loss_curve);
  cudaStreamSynchronize(ctx->stream);
  return rc;
}

int kite_mlp_forward(kite_ctx* ctx, const float* params, const float* X, int n, const float* shift,
                     const float* scale, float* Y, const kite_mlp_prior* prior) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!params || !X || !Y || n < 1) return fail(ctx, KITE_ERR_ARG, "need params, X, Y and n >= 1");
  if (check_prior(ctx, prior) != KITE_OK) return KITE_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Staging sg{ctx, {}};
  const float *Xd, *Hd, *Sd;
  float* Yd;
  int rc = sg.in(X, (size_t)n * KITE_MLP_IN, &Xd);
  if (rc == KITE_OK) rc = sg.in(shift, KITE_MLP_IN, &Hd);
  if (rc == KITE_OK) rc = sg.in(scale, KITE_MLP_IN, &Sd);
  if (rc == KITE_OK) rc = sg.out(Y, (size_t)n * KITE_MLP_OUT, &Yd);
  if (rc == KITE_OK) rc = mlp_forward_impl(ctx, params, Xd, n, Hd, Sd, Yd, prior);
  if (rc == KITE_OK) rc = sg.back(Y, Yd, (size_t)n * KITE_MLP_OUT);
  cudaStreamSynchronize(ctx->stream);
  return rc;
}

int kite_mlp_gradient(kite_ctx* ctx, const float* params, const float* X, const float* T, int n,
                      const float* shift, const float* scale, float* grad, double* loss) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!params || !X || !T || !grad || n < 1) return fail(ctx, KITE_ERR_ARG, "need params, X, T, grad, n >= 1");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Staging sg{ctx, {}};
  const float *Xd, *Td, *Hd, *Sd;
  int rc = sg.in(X, (size_t)n * KITE_MLP_IN, &Xd);
  if (rc == KITE_OK) rc = sg.in(T, (size_t)n * KITE_MLP_OUT, &Td);
  if (rc == KITE_OK) rc = sg.in(shift, KITE_MLP_IN, &Hd);
  if (rc == KITE_OK) rc = sg.in(scale, KITE_MLP_IN, &Sd);
  if (rc == KITE_OK) rc = mlp_gradient_impl(ctx, params, Xd, Td, n, Hd, Sd, grad, loss);
  cudaStreamSynchronize(ctx->stream);
  return rc;
}

int kite_learned_gate(kite_ctx* ctx, const float* rho, const double* mu, int mu_ld, int n,
                      int kcheck, double e_min, double e_max, double tol, int* flags,
                      double* deviation) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!rho || !mu || !flags || n < 1 || kcheck < 1 || mu_ld < kcheck || !(e_max > e_min) || !(tol >= 0.0))
    return fail(ctx, KITE_ERR_ARG, "need rho, mu, flags, n >= 1, 1 <= kcheck <= mu_ld");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Staging sg{ctx, {}};
  const float* rd;
  const double* md;
  int* fd;
  double* dd;
  int rc = sg.in(rho, (size_t)n * KITE_MLP_OUT, &rd);
  if (rc == KITE_OK) rc = sg.in(mu, (size_t)n * mu_ld, &md);
  if (rc == KITE_OK) rc = sg.out(flags, (size_t)n, &fd);
  if (rc == KITE_OK) rc = sg.out(deviation, (size_t)n, &dd);
  if (rc == KITE_OK) rc = mlp_gate_impl(ctx, rd, md, mu_ld, n, kcheck, 0.5 * (e_max - e_min), tol, fd, dd);
  if (rc == KITE_OK) rc = sg.back(flags, fd, (size_t)n);
  if (rc == KITE_OK && deviation) rc = sg.back(deviation, dd, (size_t)n);
  cudaStreamSynchronize(ctx->stream);
  return rc;
}

int kite_spectral_k(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const double* k, int nk,
                    const double* weights, double* mu, kite_stats* st) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  int rc = validate_system(ctx, sys);
  if (rc != KITE_OK) return rc;
  if (!kpm || !k || !mu || nk < 1) return fail(ctx, KITE_ERR_ARG, "kpm, k, mu and nk >= 1 are required");
  if (kpm->M < 1 || kpm->S < 1 || kpm->R != 1 || kpm->S > 4096)
    return fail(ctx, KITE_ERR_ARG, "need M >= 1, R = 1 (one start vector per k) and 1 <= S <= 4096");
  if (kpm->precision != KITE_FP32 && kpm->precision != KITE_FP64)
    return fail(ctx, KITE_ERR_ARG, "precision must be KITE_FP32 or KITE_FP64");
  if (kpm->r0 || kpm->r_last || kpm->real_vectors != 0 || (kpm->doubling != 0 && kpm->doubling != 1))
    return fail(ctx, KITE_ERR_ARG, "no r0/r_last, complex vectors, doubling 0 or 1");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc;
  rc = resolve_bounds(ctx, sys, kpm->e_min, kpm->e_max, &sc);
  if (rc != KITE_OK) return rc;
  const int M = kpm->M;
  const int sorb = sys->lattice == KITE_HONEYCOMB ? 2 : 1;
  Staging sg{ctx, {}};
  const double *kd, *wd;
  double* md;
  rc = sg.in(k, 2 * (size_t)nk, &kd);
  if (rc == KITE_OK) rc = sg.in(weights, 2 * (size_t)sorb, &wd);
  if (rc == KITE_OK) rc = sg.out(mu, 2 * (size_t)nk * M, &md);
  kite_stats local{};
  if (rc == KITE_OK) rc = spectral_k_impl(ctx, sys, kpm, sc, kd, nk, wd, md, &local);
  if (rc == KITE_OK) rc = sg.back(mu, md, 2 * (size_t)nk * M);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "spectral_k");
  if (rc == KITE_OK) {
    // growth check: |mu_n(k)| <= mu_0(k) when the spectrum is inside [-1, 1]
    std::vector<double> h(2 * (size_t)nk * M);
    if (cudaMemcpy(h.data(), md, sizeof(double) * h.size(), cudaMemcpyDefault) == cudaSuccess) {
      for (int j = 0; j < nk && rc == KITE_OK; ++j) {
        const double m0 = h[2 * (size_t)j * M];
        for (int n = 0; n < M; ++n) {
          const double re = h[2 * ((size_t)j * M + n)], im = h[2 * ((size_t)j * M + n) + 1];
          if (!isfinite(re) || !isfinite(im) || hypot(re, im) > fabs(m0) * (1.0 + 1e-3) + 1e-12) {
            rc = fail(ctx, KITE_ERR_BOUNDS, "a spectral moment exceeds mu_0(k): the spectrum is not inside the bounds");
            break;
          }
        }
      }
    }
  }
  if (st) *st = local;
  return rc;
}

int kite_ldos(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const int64_t* orbitals, int n,
              double* mu, kite_stats* st) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  int rc = validate_system(ctx, sys);
  if (rc != KITE_OK) return rc;
  if (!kpm || !orbitals || !mu || n < 1) return fail(ctx, KITE_ERR_ARG, "kpm, orbitals, mu and n >= 1 are required");
  if (kpm->M < 1 || kpm->S != 1 || kpm->R != 1)
    return fail(ctx, KITE_ERR_ARG, "need M >= 1, R = 1 (one start vector per orbital) and S = 1");
  if (kpm->precision != KITE_FP32 && kpm->precision != KITE_FP64)
    return fail(ctx, KITE_ERR_ARG, "precision must be KITE_FP32 or KITE_FP64");
  if (kpm->r0 || kpm->r_last || kpm->real_vectors != 0 || (kpm->doubling != 0 && kpm->doubling != 1))
    return fail(ctx, KITE_ERR_ARG, "no r0/r_last, complex vectors, doubling 0 or 1");
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc;
  rc = resolve_bounds(ctx, sys, kpm->e_min, kpm->e_max, &sc);
  if (rc != KITE_OK) return rc;
  Staging sg{ctx, {}};
  const int64_t* od;
  double* md;
  rc = sg.in(orbitals, (size_t)n, &od);
  if (rc == KITE_OK) {  // range check on the host copy
    std::vector<int64_t> h((size_t)n);
    if (cudaMemcpy(h.data(), od, sizeof(int64_t) * n, cudaMemcpyDefault) != cudaSuccess)
      return fail(ctx, KITE_ERR_CUDA, "reading orbitals");
    for (int64_t o : h)
      if (o < 0 || o >= N) return fail(ctx, KITE_ERR_ARG, "orbital index out of range");
  }
  if (rc == KITE_OK) rc = sg.out(mu, 2 * (size_t)n * kpm->M, &md);
  kite_stats local{};
  if (rc == KITE_OK) rc = ldos_impl(ctx, sys, kpm, sc, od, n, md, &local);
  if (rc == KITE_OK) rc = sg.back(mu, md, 2 * (size_t)n * kpm->M);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "ldos");
  if (rc == KITE_OK) {
    std::vector<double> h(2 * (size_t)n * kpm->M);
    if (cudaMemcpy(h.data(), md, sizeof(double) * h.size(), cudaMemcpyDefault) == cudaSuccess)
      for (double x : h)
        if (!isfinite(x) || fabs(x) > 1.0 + 1e-3) {
          rc = fail(ctx, KITE_ERR_BOUNDS, "an LDOS moment exceeds 1: the spectrum is not inside the bounds");
          break;
        }
  }
  if (st) *st = local;
  return rc;
}

int kite_evolution_coeffs(int M, double dt, double e_min, double e_max, double* coef) {
  if (M < 1 || !coef || !(e_max > e_min) || !isfinite(dt) || dt < 0.0) return KITE_ERR_ARG;
  evolution_coeffs(M, dt, 0.5 * (e_max + e_min), 0.5 * (e_max - e_min), coef);
  return KITE_OK;
}

int kite_propagate(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, double dt, int nsteps, double* psi,
                   double* norms, kite_stats* st) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  int rc = validate_system(ctx, sys);
  if (rc != KITE_OK) return rc;
  if (!kpm || !psi || nsteps < 1 || !isfinite(dt) || dt < 0.0)
    return fail(ctx, KITE_ERR_ARG, "kpm, psi, nsteps >= 1 and dt >= 0 are required");
  if (kpm->M < 1 || kpm->R < 1 || kpm->R > 65536 || kpm->S != 1)
    return fail(ctx, KITE_ERR_ARG, "need M >= 1, 1 <= R <= 65536 wave functions and S = 1");
  if (kpm->precision != KITE_FP32 && kpm->precision != KITE_FP64)
    return fail(ctx, KITE_ERR_ARG, "precision must be KITE_FP32 or KITE_FP64");
  if (kpm->r0 || kpm->r_last || kpm->doubling != 0 || kpm->real_vectors != 0)
    return fail(ctx, KITE_ERR_ARG, "no r0/r_last (psi is the start), doubling 0, complex vectors");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc;
  rc = resolve_bounds(ctx, sys, kpm->e_min, kpm->e_max, &sc);
  if (rc != KITE_OK) return rc;
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  const size_t npsi = 2 * (size_t)kpm->R * N;
  Staging sg{ctx, {}};
  const double* pin;
  double *pd, *nd = nullptr;
  rc = sg.in((const double*)psi, npsi, &pin);
  pd = const_cast<double*>(pin);  // psi is updated in place (staged copy for host memory)
  if (rc == KITE_OK && norms) rc = sg.out(norms, (size_t)nsteps * kpm->R, &nd);
  kite_stats local{};
  if (rc == KITE_OK) rc = propagate_impl(ctx, sys, kpm, sc, dt, nsteps, pd, nd, &local);
  if (rc == KITE_OK) rc = sg.back(psi, (const double*)pd, npsi);
  if (rc == KITE_OK && norms) rc = sg.back(norms, (const double*)nd, (size_t)nsteps * kpm->R);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "propagate");
  if (st) *st = local;
  return rc;
}

int kite_moments_1d_batched(kite_ctx* ctx, int count, const kite_system* systems,
                            const kite_kpm* kpms, double* const* mu, kite_stats* st) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (count < 1 || !systems || !kpms || !mu) return fail(ctx, KITE_ERR_ARG, "need count >= 1 and arrays");
  std::vector<Scale> scales(count);
  for (int i = 0; i < count; ++i) {
    int rc = validate_system(ctx, &systems[i]);
    if (rc != KITE_OK) return rc;
    const kite_kpm& k = kpms[i];
    if (!mu[i]) return fail(ctx, KITE_ERR_ARG, "mu[" + std::to_string(i) + "] is NULL");
    if (systems[i].lattice != systems[0].lattice)
      return fail(ctx, KITE_ERR_ARG, "all systems of a batch must share the lattice kind");
    if (systems[i].open_x || systems[i].open_y)
      return fail(ctx, KITE_ERR_ARG, "the batched sweep takes periodic boundaries only");
    if (k.precision != KITE_FP32) return fail(ctx, KITE_ERR_UNSUPPORTED, "the batched sweep is FP32");
    if (k.R != kpms[0].R || k.R < 1 || k.R > 8)
      return fail(ctx, KITE_ERR_ARG, "all systems need the same R, 1 <= R <= 8");
    if (k.S != 1 || k.r0 || k.r_last || k.real_vectors != 0)
      return fail(ctx, KITE_ERR_ARG, "batched systems take S = 1, no r0/r_last, complex vectors");
    if ((k.doubling != 0 && k.doubling != 1) || k.doubling != kpms[0].doubling)
      return fail(ctx, KITE_ERR_ARG, "all systems of a batch need the same doubling, 0 or 1");
    if (k.M < 1 || k.M > (1 << 20)) return fail(ctx, KITE_ERR_ARG, "M out of range");
    rc = resolve_bounds(ctx, &systems[i], k.e_min, k.e_max, &scales[i]);
    if (rc != KITE_OK) return rc;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  kite_stats local{};
  const int rc = moments_1d_batched_impl(ctx, count, systems, kpms, scales, mu, &local);
  if (st) *st = local;
  return rc;
}

int kite_moments_2d(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, int alpha, int beta,
                    double* mu_nm, kite_stats* st) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  int rc = validate_system(ctx, sys);
  if (rc != KITE_OK) return rc;
  if (!kpm || !mu_nm) return fail(ctx, KITE_ERR_ARG, "kpm and mu_nm are required");
  if (kpm->M < 1 || kpm->R < 1 || kpm->S < 1 || kpm->M > 65536)
    return fail(ctx, KITE_ERR_ARG, "need 1 <= M <= 65536, R >= 1, S >= 1");
  if (kpm->precision != KITE_FP32)
    return fail(ctx, KITE_ERR_UNSUPPORTED, "2D moments run the FP32 recursion only");
  if ((double)kpm->R * kpm->S > 65536.0) return fail(ctx, KITE_ERR_ARG, "R*S > 65536");
  if (kpm->doubling != 0 || kpm->real_vectors != 0)
    return fail(ctx, KITE_ERR_ARG, "the 2D moments take doubling = 0 and complex vectors");
  if ((alpha != KITE_DIR_X && alpha != KITE_DIR_Y) || (beta != KITE_DIR_X && beta != KITE_DIR_Y))
    return fail(ctx, KITE_ERR_ARG, "alpha and beta must be KITE_DIR_X or KITE_DIR_Y");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc;
  rc = resolve_bounds(ctx, sys, kpm->e_min, kpm->e_max, &sc);
  if (rc != KITE_OK) return rc;
  const int M = kpm->M;
  const size_t nvec = (size_t)kpm->R * kpm->S;
  const int64_t N = (int64_t)sys->Lx * sys->Ly * (sys->lattice == KITE_HONEYCOMB ? 2 : 1);
  const double* r0_dev = nullptr;
  if (kpm->r0) {
    const void* v = nullptr;
    rc = device_view(ctx, kpm->r0, nvec * (size_t)N * 2 * sizeof(double), &v);
    if (rc != KITE_OK) return rc;
    r0_dev = static_cast<const double*>(v);
  }
  const bool out_d = is_device_ptr(mu_nm);
  double* out_dev = mu_nm;
  const size_t out_bytes = sizeof(double) * 2 * (size_t)M * M;
  if (!out_d) KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&out_dev, out_bytes, ctx->stream));
  kite_stats local{};
  rc = moments_2d_impl(ctx, sys, kpm, sc, alpha, beta, out_dev, &local, r0_dev);
  if (rc == KITE_OK && !out_d) {
    cudaError_t e = copy_out(ctx, mu_nm, out_dev, out_bytes);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying mu_nm");
  }
  if (!out_d) cudaFreeAsync(out_dev, ctx->stream);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "moments_2d");
  local.e_min = sc.e_min;
  local.e_max = sc.e_max;
  if (st) *st = local;
  return rc;
}

int kite_inner_products(kite_ctx* ctx, const float* A, const float* B, int M, int M2, int64_t N,
                        double scale, double* C, int sub_k, int products, int fold) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!A || !B || !C || M < 1 || M2 < 1 || N < 1 || sub_k < 0 || fold < 0 || !isfinite(scale))
    return fail(ctx, KITE_ERR_ARG, "need A, B, C, M >= 1, M2 >= 1, N >= 1, sub_k >= 0, fold >= 0");
  if (products != 0 && products != 3 && products != 4)
    return fail(ctx, KITE_ERR_ARG, "products must be 0 (default 4), 3 or 4");
  if ((double)M * N > 4.0e10 || (double)M2 * N > 4.0e10)
    return fail(ctx, KITE_ERR_ARG, "families larger than 4e10 complex entries");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  const int sub_kb = sub_k == 0 ? 8 : (sub_k + 63) / 64;
  const size_t a_bytes = (size_t)M * N * 8, b_bytes = (size_t)M2 * N * 8, c_bytes = (size_t)M * M2 * 16;
  const bool a_d = is_device_ptr(A), b_d = is_device_ptr(B), c_d = is_device_ptr(C);
  char* stage = nullptr;
  const size_t st_bytes = (a_d ? 0 : a_bytes) + (b_d ? 0 : b_bytes) + (c_d ? 0 : c_bytes) + 512;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&stage, st_bytes, ctx->stream));
  size_t off = 0;
  const float* Ad = A;
  const float* Bd = B;
  double* Cd = C;
  cudaError_t e = cudaSuccess;
  if (!a_d) { Ad = reinterpret_cast<float*>(stage + off); e = copy_in(ctx, stage + off, A, a_bytes); off += (a_bytes + 255) & ~size_t(255); }
  if (e == cudaSuccess && !b_d) { Bd = reinterpret_cast<float*>(stage + off); e = copy_in(ctx, stage + off, B, b_bytes); off += (b_bytes + 255) & ~size_t(255); }
  if (!c_d) Cd = reinterpret_cast<double*>(stage + off);
  int rc = e == cudaSuccess ? KITE_OK : cuda_fail(ctx, e, "copying A/B");
  if (rc == KITE_OK) rc = inner_products_impl(ctx, Ad, Bd, M, M2, N, scale, Cd, sub_kb,
                                                   fold == 0 ? 16 : fold, products == 3 ? 3 : 4);
  if (rc == KITE_OK && !c_d) {
    e = copy_out(ctx, C, Cd, c_bytes);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying C");
  }
  int status_host = 0;
  if (rc == KITE_OK) {
    e = cudaMemcpyAsync(&status_host, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "status");
  }
  cudaFreeAsync(stage, ctx->stream);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "inner_products");
  if (rc == KITE_OK && status_host != 0)
    rc = fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait gave up in the tensor-core contraction");
  return rc;
}

int kite_reconstruct_dos(kite_ctx* ctx, const double* mu, int M_avail, int M_use, int kernel,
                         double param, double e_min, double e_max, const double* E, int K,
                         double* rho) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!mu || !E || !rho || K < 0 || M_avail < 1 || M_use < 1 || M_use > M_avail)
    return fail(ctx, KITE_ERR_ARG, "need mu, E, rho and 1 <= M_use <= M_avail, K >= 0");
  if (kernel != KITE_KERNEL_NONE && kernel != KITE_KERNEL_JACKSON && kernel != KITE_KERNEL_LORENTZ)
    return fail(ctx, KITE_ERR_ARG, "unknown kernel");
  if (kernel == KITE_KERNEL_LORENTZ && !(param > 0.0))
    return fail(ctx, KITE_ERR_ARG, "Lorentz kernel needs lambda > 0");
  if (!(e_max > e_min)) return fail(ctx, KITE_ERR_ARG, "e_max must exceed e_min");
  if (K == 0) return KITE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc{e_min, e_max, 0.5 * (e_max + e_min), 0.5 * (e_max - e_min)};
  const bool mu_d = is_device_ptr(mu), E_d = is_device_ptr(E), rho_d = is_device_ptr(rho);
  double* buf = nullptr;
  const size_t nbuf = (size_t)M_use * 2 + (size_t)K * 2;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, nbuf * sizeof(double), ctx->stream));
  double* mu_dev = mu_d ? const_cast<double*>(mu) : buf;
  double* coef = buf + M_use;
  double* E_dev = E_d ? const_cast<double*>(E) : buf + 2 * (size_t)M_use;
  double* rho_dev = rho_d ? rho : buf + 2 * (size_t)M_use + K;
  int rc = KITE_OK;
  cudaError_t e = cudaSuccess;
  if (!mu_d) e = copy_in(ctx, mu_dev, mu, (size_t)M_use * sizeof(double));
  if (e == cudaSuccess && !E_d) e = copy_in(ctx, E_dev, E, (size_t)K * sizeof(double));
  if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying inputs");
  if (rc == KITE_OK) rc = reconstruct_dos_impl(ctx, mu_dev, M_use, kernel, param, sc, E_dev, K, rho_dev, coef);
  if (rc == KITE_OK && !rho_d) {
    e = copy_out(ctx, rho, rho_dev, (size_t)K * sizeof(double));
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying rho");
  }
  cudaFreeAsync(buf, ctx->stream);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "reconstruct_dos");
  return rc;
}

int kite_reconstruct_green(kite_ctx* ctx, const double* mu, int M_avail, int M_use, int kernel,
                           double param, double e_min, double e_max, double eta, const double* E, int K,
                           double* G, double* rho) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!mu || !E || (!G && !rho) || K < 0 || M_avail < 1 || M_use < 1 || M_use > M_avail)
    return fail(ctx, KITE_ERR_ARG, "need mu, E, G or rho, and 1 <= M_use <= M_avail, K >= 0");
  if (kernel != KITE_KERNEL_NONE && kernel != KITE_KERNEL_JACKSON && kernel != KITE_KERNEL_LORENTZ)
    return fail(ctx, KITE_ERR_ARG, "unknown kernel");
  if (kernel == KITE_KERNEL_LORENTZ && !(param > 0.0))
    return fail(ctx, KITE_ERR_ARG, "Lorentz kernel needs lambda > 0");
  if (!(e_max > e_min)) return fail(ctx, KITE_ERR_ARG, "e_max must exceed e_min");
  if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ctx, KITE_ERR_ARG, "eta must be > 0");
  if (K == 0) return KITE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc{e_min, e_max, 0.5 * (e_max + e_min), 0.5 * (e_max - e_min)};
  Staging sg{ctx, {}};
  const double *mu_dev, *E_dev;
  double *G_dev = nullptr, *rho_dev = nullptr, *coef = nullptr;
  int rc = sg.in(mu, (size_t)M_use, &mu_dev);
  if (rc == KITE_OK) rc = sg.in(E, (size_t)K, &E_dev);
  if (rc == KITE_OK && G) rc = sg.out(G, 2 * (size_t)K, &G_dev);
  if (rc == KITE_OK && rho) rc = sg.out(rho, (size_t)K, &rho_dev);
  if (rc == KITE_OK) {
    KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&coef, sizeof(double) * (size_t)M_use, ctx->stream));
    rc = reconstruct_green_impl(ctx, mu_dev, M_use, kernel, param, sc, eta, E_dev, K, G_dev, rho_dev, coef);
    cudaFreeAsync(coef, ctx->stream);
  }
  if (rc == KITE_OK && G) rc = sg.back(G, G_dev, 2 * (size_t)K);
  if (rc == KITE_OK && rho) rc = sg.back(rho, rho_dev, (size_t)K);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "reconstruct_green");
  return rc;
}

int kite_reconstruct_sigma_dc(kite_ctx* ctx, const double* mu_nm, int M_avail, int M_use, int lattice,
                              int kernel, double param, double e_min, double e_max, const double* E, int K,
                              double* sigma) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!mu_nm || !E || !sigma || K < 0 || M_avail < 1 || M_use < 1 || M_use > M_avail || M_use > 16384)
    return fail(ctx, KITE_ERR_ARG, "need mu_nm, E, sigma and 1 <= M_use <= min(M_avail, 16384), K >= 0");
  if (lattice != KITE_HONEYCOMB && lattice != KITE_SQUARE) return fail(ctx, KITE_ERR_ARG, "unknown lattice");
  if (kernel != KITE_KERNEL_NONE && kernel != KITE_KERNEL_JACKSON && kernel != KITE_KERNEL_LORENTZ)
    return fail(ctx, KITE_ERR_ARG, "unknown kernel");
  if (kernel == KITE_KERNEL_LORENTZ && !(param > 0.0))
    return fail(ctx, KITE_ERR_ARG, "Lorentz kernel needs lambda > 0");
  if (!(e_max > e_min)) return fail(ctx, KITE_ERR_ARG, "e_max must exceed e_min");
  if (K == 0) return KITE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc{e_min, e_max, 0.5 * (e_max + e_min), 0.5 * (e_max - e_min)};
  const bool mu_d = is_device_ptr(mu_nm), E_d = is_device_ptr(E), s_d = is_device_ptr(sigma);
  const size_t mu_doubles = mu_d ? 0 : 2 * (size_t)M_avail * M_avail;
  double* buf = nullptr;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, sizeof(double) * (mu_doubles + (size_t)M_use + 2 * (size_t)K),
                                     ctx->stream));
  const double* mu_dev = mu_d ? mu_nm : buf;
  double* w = buf + mu_doubles;
  double* E_dev = E_d ? const_cast<double*>(E) : w + M_use;
  double* s_dev = s_d ? sigma : w + M_use + K;
  cudaError_t e = cudaSuccess;
  if (!mu_d) e = copy_in(ctx, buf, mu_nm, mu_doubles * sizeof(double));
  if (e == cudaSuccess && !E_d) e = copy_in(ctx, E_dev, E, (size_t)K * sizeof(double));
  int rc = e == cudaSuccess ? KITE_OK : cuda_fail(ctx, e, "copying inputs");
  if (rc == KITE_OK)
    rc = reconstruct_sigma_dc_impl(ctx, mu_dev, M_avail, M_use, kernel, param, lattice, sc, E_dev, K, s_dev, w);
  if (rc == KITE_OK && !s_d) {
    e = copy_out(ctx, sigma, s_dev, (size_t)K * sizeof(double));
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying sigma");
  }
  cudaFreeAsync(buf, ctx->stream);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "reconstruct_sigma_dc");
  return rc;
}

int kite_reconstruct_sigma_dc_bastin(kite_ctx* ctx, const double* mu_nm, int M_avail, int M_use, int lattice,
                                     int kernel, double param, double e_min, double e_max, double eta, double kT,
                                     const double* E_F, int K, int n_quad, double* sigma) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!mu_nm || !E_F || !sigma || K < 0 || M_avail < 1 || M_use < 1 || M_use > M_avail || M_use > 16384)
    return fail(ctx, KITE_ERR_ARG, "need mu_nm, E_F, sigma and 1 <= M_use <= min(M_avail, 16384), K >= 0");
  if (lattice != KITE_HONEYCOMB && lattice != KITE_SQUARE) return fail(ctx, KITE_ERR_ARG, "unknown lattice");
  if (kernel != KITE_KERNEL_NONE && kernel != KITE_KERNEL_JACKSON && kernel != KITE_KERNEL_LORENTZ)
    return fail(ctx, KITE_ERR_ARG, "unknown kernel");
  if (kernel == KITE_KERNEL_LORENTZ && !(param > 0.0))
    return fail(ctx, KITE_ERR_ARG, "Lorentz kernel needs lambda > 0");
  if (!(e_max > e_min) || !isfinite(e_min) || !isfinite(e_max))
    return fail(ctx, KITE_ERR_ARG, "need finite e_min < e_max");
  if (!(eta > 0.0) || !isfinite(eta)) return fail(ctx, KITE_ERR_ARG, "eta must be finite and > 0");
  if (!(kT >= 0.0) || !isfinite(kT)) return fail(ctx, KITE_ERR_ARG, "kT must be finite and >= 0");
  if (n_quad < 0 || n_quad > (1 << 20)) return fail(ctx, KITE_ERR_ARG, "need 0 <= n_quad <= 2^20");
  if (K == 0) return KITE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Scale sc{e_min, e_max, 0.5 * (e_max + e_min), 0.5 * (e_max - e_min)};
  std::vector<double> E_host((size_t)K);
  const bool mu_d = is_device_ptr(mu_nm), s_d = is_device_ptr(sigma);
  cudaError_t e = cudaMemcpy(E_host.data(), E_F, (size_t)K * sizeof(double), cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading E_F");
  for (int i = 0; i < K; ++i)
    if (!isfinite(E_host[i])) return fail(ctx, KITE_ERR_ARG, "E_F must be finite");
  const size_t mu_doubles = mu_d ? 0 : 2 * (size_t)M_avail * M_avail;
  double* buf = nullptr;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, sizeof(double) * (mu_doubles + (size_t)K), ctx->stream));
  const double* mu_dev = mu_d ? mu_nm : buf;
  double* s_dev = s_d ? sigma : buf + mu_doubles;
  if (!mu_d) e = copy_in(ctx, buf, mu_nm, mu_doubles * sizeof(double));
  int rc = e == cudaSuccess ? KITE_OK : cuda_fail(ctx, e, "copying mu_nm");
  if (rc == KITE_OK)
    rc = reconstruct_sigma_bastin_impl(ctx, mu_dev, M_avail, M_use, lattice, kernel, param, sc, eta, kT,
                                       E_host.data(), K, n_quad, s_dev);
  if (rc == KITE_OK && !s_d) {
    e = copy_out(ctx, sigma, s_dev, (size_t)K * sizeof(double));
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying sigma");
  }
  cudaFreeAsync(buf, ctx->stream);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "reconstruct_sigma_dc_bastin");
  return rc;
}

int kite_reconstruct_sigma(kite_ctx* ctx, const double* mu_nm, int M_avail, int M_use,
                           int lattice, int kernel, double e_min, double e_max, double E_F,
                           double kT, double eta, const double* omega, int K, int n_quad,
                           double* sigma) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!mu_nm || !omega || !sigma || K < 0 || M_avail < 1 || M_use < 1 || M_use > M_avail ||
      n_quad < 0 || n_quad > (1 << 20))
    return fail(ctx, KITE_ERR_ARG, "need mu_nm, omega, sigma and 1 <= M_use <= M_avail");
  if (lattice != KITE_HONEYCOMB && lattice != KITE_SQUARE) return fail(ctx, KITE_ERR_ARG, "unknown lattice");
  if (kernel != KITE_KERNEL_NONE && kernel != KITE_KERNEL_JACKSON)
    return fail(ctx, KITE_ERR_ARG, "sigma supports KITE_KERNEL_NONE and KITE_KERNEL_JACKSON");
  if (!(e_max > e_min) || !(eta > 0.0) || !(kT >= 0.0) || !isfinite(E_F))
    return fail(ctx, KITE_ERR_ARG, "need e_max > e_min, eta > 0, kT >= 0");
  if (K == 0) return KITE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  std::vector<double> om(K);
  cudaError_t e = cudaMemcpy(om.data(), omega, K * sizeof(double), cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading omega");
  for (int i = 0; i < K; ++i)
    if (!(om[i] > 0.0) || !isfinite(om[i])) return fail(ctx, KITE_ERR_ARG, "omega must be > 0");
  Scale sc{e_min, e_max, 0.5 * (e_max + e_min), 0.5 * (e_max - e_min)};
  const bool mu_d = is_device_ptr(mu_nm), s_d = is_device_ptr(sigma);
  const size_t mu_bytes = 2 * sizeof(double) * (size_t)M_avail * M_avail;
  double* stage = nullptr;
  const size_t st_bytes = (mu_d ? 0 : mu_bytes) + (s_d ? 0 : 2 * sizeof(double) * K) + 512;
  KITE_CUDA_TRY(ctx, cudaMallocAsync((void**)&stage, st_bytes, ctx->stream));
  const double* mu_dev = mu_nm;
  double* sig_dev = sigma;
  if (!mu_d) {
    mu_dev = stage;
    e = copy_in(ctx, stage, mu_nm, mu_bytes);
  }
  if (!s_d) sig_dev = stage + (mu_d ? 0 : 2 * (size_t)M_avail * M_avail);
  int rc = e == cudaSuccess ? KITE_OK : cuda_fail(ctx, e, "copying mu_nm");
  if (rc == KITE_OK)
    rc = reconstruct_sigma_impl(ctx, mu_dev, M_avail, M_use, lattice, kernel, sc, E_F, kT, eta,
                                om.data(), K, n_quad, sig_dev);
  if (rc == KITE_OK && !s_d) {
    e = copy_out(ctx, sigma, sig_dev, 2 * sizeof(double) * K);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copying sigma");
  }
  cudaFreeAsync(stage, ctx->stream);
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && es != cudaSuccess) rc = cuda_fail(ctx, es, "reconstruct_sigma");
  return rc;
}

}  // extern "C"
