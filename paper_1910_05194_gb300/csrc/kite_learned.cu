// kite_learned.cu -- the learned reconstructor as library objects: a model (parameters,
// input normalisation and output window, owned in device memory) trained by
// kite_learned_train and applied by kite_learned_dos, which runs the network, the
// consistency gate and the plain fallback in one call.  The kernels are kite_mlp.cu's.
//
// The paper has no learned component.  Its Sec. 2a notes that the resolution of the
// Chebyshev reconstruction scales as the inverse number of moments; the model maps the
// first KITE_MLP_IN moments to the density that many more moments give, and the plain
// Jackson reconstruction (Eq. e8a) is both its fallback and the reference for its error.
#include <math.h>

#include <string>
#include <vector>

#include "kite_internal.h"

struct kite_model {
  int device = 0;
  float* buf = nullptr;  // one device allocation: params [P], shift [IN], scale [IN]
  float* params = nullptr;
  float* shift = nullptr;
  float* scale = nullptr;
  double e_min = 0.0, e_max = 0.0;
};

namespace kite {

int64_t mlp_param_count();
int mlp_train_impl(kite_ctx* ctx, const float* X, const float* T, int n, const float* shift, const float* scale,
                   const kite_mlp_train_cfg* cfg, float* params, float* loss_curve,
                   const kite_mlp_prior* prior);
int mlp_forward_impl(kite_ctx* ctx, const float* params, const float* X, int n, const float* shift,
                     const float* scale, float* Y, const kite_mlp_prior* prior);
int mlp_gate_impl(kite_ctx* ctx, const float* rho, const double* mu, int mu_ld, int n, int kcheck,
                  double de_minus, double tol, int* flags, double* dev);
int mlp_adamw_step_impl(kite_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n, int t, int total,
                        double lr, double wd);
int mlp_init_impl(kite_ctx* ctx, uint64_t seed, double head_scale, float* p);
int mlp_norm_impl(kite_ctx* ctx, const float* X, int n, double sd_floor, float* shift, float* scale);
int mlp_take_inputs_impl(kite_ctx* ctx, const double* mu, int mu_ld, int n, float* X);
int mlp_narrow_impl(kite_ctx* ctx, const double* src, int K, float* dst);

namespace {

constexpr int IN = KITE_MLP_IN, OUT = KITE_MLP_OUT;
constexpr double kSdFloor = 1e-4;

// A model's device buffers (params, shift, scale) in one allocation.
int new_model(kite_ctx* ctx, double e_min, double e_max, kite_model** out) {
  kite_model* m = new kite_model();
  m->device = ctx->device;
  const int64_t P = mlp_param_count();
  if (cudaMalloc((void**)&m->buf, sizeof(float) * (size_t)(P + 2 * IN)) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return fail(ctx, KITE_ERR_OOM, "model parameters could not be allocated");
  }
  m->params = m->buf;
  m->shift = m->buf + P;
  m->scale = m->buf + P + IN;
  m->e_min = e_min;
  m->e_max = e_max;
  *out = m;
  return KITE_OK;
}

kite_mlp_prior model_prior(const kite_model* m) {
  kite_mlp_prior p;
  p.kind = KITE_PRIOR_JACKSON;
  p.reserved = 0;
  p.e_min = m->e_min;
  p.e_max = m->e_max;
  return p;
}

}  // namespace
}  // namespace kite

using namespace kite;

extern "C" {

int kite_mlp_adamw_step(kite_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t n, int t,
                        int total, double lr, double weight_decay) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!params || !grad || !m || !v || n < 1 || t < 1 || total < 1 || !(lr >= 0.0) || !(weight_decay >= 0.0))
    return fail(ctx, KITE_ERR_ARG, "need params, grad, m, v, n >= 1, t >= 1, total >= 1, lr and decay >= 0");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  Staging sg{ctx, {}};
  const float* gd;
  float *pd, *md, *vd;
  int rc = sg.in(grad, (size_t)n, &gd);
  if (rc == KITE_OK) rc = sg.out(params, (size_t)n, &pd);
  if (rc == KITE_OK && pd != params) rc = copy_in(ctx, pd, params, sizeof(float) * n) == cudaSuccess ? KITE_OK
                                                                                           : KITE_ERR_CUDA;
  if (rc == KITE_OK) rc = sg.out(m, (size_t)n, &md);
  if (rc == KITE_OK && md != m) rc = copy_in(ctx, md, m, sizeof(float) * n) == cudaSuccess ? KITE_OK : KITE_ERR_CUDA;
  if (rc == KITE_OK) rc = sg.out(v, (size_t)n, &vd);
  if (rc == KITE_OK && vd != v) rc = copy_in(ctx, vd, v, sizeof(float) * n) == cudaSuccess ? KITE_OK : KITE_ERR_CUDA;
  if (rc == KITE_ERR_CUDA && ctx->last_error.empty()) fail(ctx, rc, "copying the optimiser state in");
  if (rc == KITE_OK) rc = mlp_adamw_step_impl(ctx, pd, gd, md, vd, n, t, total, lr, weight_decay);
  if (rc == KITE_OK) rc = sg.back(params, pd, (size_t)n);
  if (rc == KITE_OK) rc = sg.back(m, md, (size_t)n);
  if (rc == KITE_OK) rc = sg.back(v, vd, (size_t)n);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "kite_mlp_adamw_step");
  return rc;
}

int kite_learned_train(kite_ctx* ctx, const float* X, const float* Y, int n, const kite_learned_cfg* cfg,
                       kite_model** out, float* loss_curve) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!out) return fail(ctx, KITE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!X || !Y || !cfg || n < 1 || cfg->epochs < 1 || cfg->batch < 1 || !(cfg->lr > 0.0) ||
      !(cfg->weight_decay >= 0.0) || !(cfg->e_max > cfg->e_min) || !isfinite(cfg->e_min) || !isfinite(cfg->e_max) ||
      !(cfg->head_scale >= 0.0))
    return fail(ctx, KITE_ERR_ARG,
                "need X, Y, n >= 1, epochs and batch >= 1, lr > 0, decay >= 0, e_max > e_min, head_scale >= 0");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  const int64_t P = mlp_param_count();
  kite_model* m = nullptr;
  int rc = new_model(ctx, cfg->e_min, cfg->e_max, &m);
  if (rc != KITE_OK) return rc;
  {
    Staging sg{ctx, {}};
    const float *Xd, *Yd;
    rc = sg.in(X, (size_t)n * IN, &Xd);
    if (rc == KITE_OK) rc = sg.in(Y, (size_t)n * OUT, &Yd);
    if (rc == KITE_OK) {
      if (cfg->init) {
        if (copy_in(ctx, m->params, cfg->init, sizeof(float) * (size_t)P) != cudaSuccess)
          rc = fail(ctx, KITE_ERR_CUDA, "copying the initial parameters");
      } else {
        rc = mlp_init_impl(ctx, cfg->seed, cfg->head_scale > 0.0 ? cfg->head_scale : 1.0, m->params);
      }
    }
    if (rc == KITE_OK) rc = mlp_norm_impl(ctx, Xd, n, kSdFloor, m->shift, m->scale);
    if (rc == KITE_OK) {
      kite_mlp_train_cfg tc;
      tc.epochs = cfg->epochs;
      tc.batch = cfg->batch;
      tc.lr = cfg->lr;
      tc.weight_decay = cfg->weight_decay;
      tc.seed = cfg->seed;
      const kite_mlp_prior prior = model_prior(m);
      std::vector<float> curve(cfg->epochs);
      rc = mlp_train_impl(ctx, Xd, Yd, n, m->shift, m->scale, &tc, m->params, curve.data(), &prior);
      if (rc == KITE_OK && loss_curve) std::copy(curve.begin(), curve.end(), loss_curve);
    }
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "kite_learned_train");
  if (rc != KITE_OK) {
    kite_model_destroy(m);
    return rc;
  }
  *out = m;
  return KITE_OK;
}

int kite_learned_dos(kite_ctx* ctx, const kite_model* model, const double* mu, int mu_ld, int n, double gate_tol,
                     int kcheck, int M_plain, const kite_system* systems, const kite_kpm* plain_kpm, float* rho,
                     int* fell_back, double* deviation) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!model || !mu || !rho || !fell_back || n < 1 || kcheck < 1 || mu_ld < IN || mu_ld < kcheck ||
      !(gate_tol >= 0.0) || M_plain < 1)
    return fail(ctx, KITE_ERR_ARG,
                "need model, mu, rho, fell_back, n >= 1, kcheck >= 1, mu_ld >= max(KITE_MLP_IN, kcheck), "
                "gate_tol >= 0, M_plain >= 1");
  if (model->device != ctx->device) return fail(ctx, KITE_ERR_ARG, "the model lives on another GPU");
  if (systems && !plain_kpm) return fail(ctx, KITE_ERR_ARG, "plain_kpm is required with systems");
  if (!systems && M_plain > mu_ld)
    return fail(ctx, KITE_ERR_ARG, "without systems the fallback needs M_plain <= mu_ld moments in mu");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  const double de_minus = 0.5 * (model->e_max - model->e_min), de_plus = 0.5 * (model->e_max + model->e_min);
  Staging sg{ctx, {}};
  const double* md;
  float *Xd, *rd;
  int* fd;
  double* dd;
  int rc = sg.in(mu, (size_t)n * mu_ld, &md);
  if (rc == KITE_OK) rc = sg.scratch((size_t)n * IN, &Xd);
  if (rc == KITE_OK) rc = sg.out(rho, (size_t)n * OUT, &rd);
  if (rc == KITE_OK) rc = sg.out(fell_back, (size_t)n, &fd);
  if (rc == KITE_OK) rc = sg.scratch((size_t)n, &dd);
  // 1. the network on the first IN moments, as a residual on their Jackson reconstruction
  if (rc == KITE_OK) rc = mlp_take_inputs_impl(ctx, md, mu_ld, n, Xd);
  const kite_mlp_prior prior = model_prior(model);
  if (rc == KITE_OK) rc = mlp_forward_impl(ctx, model->params, Xd, n, model->shift, model->scale, rd, &prior);
  // 2. the consistency gate
  if (rc == KITE_OK) rc = mlp_gate_impl(ctx, rd, md, mu_ld, n, kcheck, de_minus, gate_tol, fd, dd);
  std::vector<int> flags(n, 0);
  if (rc == KITE_OK && cudaMemcpyAsync(flags.data(), fd, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream) !=
                           cudaSuccess)
    rc = fail(ctx, KITE_ERR_CUDA, "reading the gate's flags");
  if (rc == KITE_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = fail(ctx, KITE_ERR_CUDA, "gate");
  // 3. the plain path for every flagged row, on the model's grid
  int flagged = 0;
  for (int i = 0; i < n; ++i) flagged += flags[i] != 0;
  if (rc == KITE_OK && flagged > 0) {
    double *E, *rho64, *mu_plain = nullptr;
    rc = sg.scratch(OUT, &E);
    if (rc == KITE_OK) rc = sg.scratch(OUT, &rho64);
    if (rc == KITE_OK && systems) rc = sg.scratch((size_t)M_plain, &mu_plain);
    std::vector<double> Eh(OUT);
    for (int j = 0; j < OUT; ++j) Eh[j] = (-1.0 + (2.0 * j + 1.0) / OUT) * de_minus + de_plus;
    if (rc == KITE_OK && copy_in(ctx, E, Eh.data(), sizeof(double) * OUT) != cudaSuccess)
      rc = fail(ctx, KITE_ERR_CUDA, "energy grid");
    if (rc == KITE_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess)  // Eh leaves scope only after the copy
      rc = fail(ctx, KITE_ERR_CUDA, "energy grid");
    for (int i = 0; i < n && rc == KITE_OK; ++i) {
      if (!flags[i]) continue;
      const double* row = md + (size_t)i * mu_ld;
      int M_avail = mu_ld;
      if (systems) {
        kite_kpm kp = *plain_kpm;
        kp.M = M_plain;
        kp.e_min = model->e_min;
        kp.e_max = model->e_max;
        kp.r0 = nullptr;
        kp.r_last = nullptr;
        rc = kite_moments_1d(ctx, &systems[i], &kp, mu_plain, nullptr, nullptr);
        row = mu_plain;
        M_avail = M_plain;
      }
      if (rc == KITE_OK)
        rc = kite_reconstruct_dos(ctx, row, M_avail, M_plain, KITE_KERNEL_JACKSON, 0.0, model->e_min, model->e_max,
                                  E, OUT, rho64);
      if (rc == KITE_OK) rc = mlp_narrow_impl(ctx, rho64, OUT, rd + (size_t)i * OUT);
    }
  }
  if (rc == KITE_OK) rc = sg.back(rho, rd, (size_t)n * OUT);
  if (rc == KITE_OK) rc = sg.back(fell_back, fd, (size_t)n);
  if (rc == KITE_OK && deviation) {
    double* dv;
    rc = sg.out(deviation, (size_t)n, &dv);
    if (rc == KITE_OK && dv != dd && cudaMemcpyAsync(dv, dd, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                                     ctx->stream) != cudaSuccess)
      rc = fail(ctx, KITE_ERR_CUDA, "deviation");
    if (rc == KITE_OK) rc = sg.back(deviation, dv, (size_t)n);
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (rc == KITE_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "kite_learned_dos");
  return rc;
}

int kite_model_export(const kite_model* model, float* params, float* shift, float* scale, double* window) {
  if (!model) return KITE_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(model->device) != cudaSuccess) return KITE_ERR_CUDA;
  const int64_t P = mlp_param_count();
  int rc = KITE_OK;
  if (params && cudaMemcpy(params, model->params, sizeof(float) * (size_t)P, cudaMemcpyDefault) != cudaSuccess)
    rc = KITE_ERR_CUDA;
  if (rc == KITE_OK && shift && cudaMemcpy(shift, model->shift, sizeof(float) * IN, cudaMemcpyDefault) != cudaSuccess)
    rc = KITE_ERR_CUDA;
  if (rc == KITE_OK && scale && cudaMemcpy(scale, model->scale, sizeof(float) * IN, cudaMemcpyDefault) != cudaSuccess)
    rc = KITE_ERR_CUDA;
  if (rc == KITE_OK && window) {
    window[0] = model->e_min;
    window[1] = model->e_max;
  }
  cudaSetDevice(prev);  // the caller's current device is left as it was
  return rc;
}

int kite_model_import(kite_ctx* ctx, const float* params, const float* shift, const float* scale, double e_min,
                      double e_max, kite_model** out) {
  if (!ctx) return KITE_ERR_ARG;
  ctx->last_error.clear();
  if (!out || !params || !(e_max > e_min) || !isfinite(e_min) || !isfinite(e_max))
    return fail(ctx, KITE_ERR_ARG, "need out, params and a window e_min < e_max");
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, KITE_ERR_CUDA, "cudaSetDevice");
  kite_model* m = nullptr;
  int rc = new_model(ctx, e_min, e_max, &m);
  if (rc != KITE_OK) return rc;
  const int64_t P = mlp_param_count();
  std::vector<float> ones(IN, 1.0f), zeros(IN, 0.0f);
  bool ok = copy_in(ctx, m->params, params, sizeof(float) * (size_t)P) == cudaSuccess &&
            copy_in(ctx, m->shift, shift ? shift : zeros.data(), sizeof(float) * IN) == cudaSuccess &&
            copy_in(ctx, m->scale, scale ? scale : ones.data(), sizeof(float) * IN) == cudaSuccess &&
            cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  if (!ok) {
    kite_model_destroy(m);
    return fail(ctx, KITE_ERR_CUDA, "copying the model in");
  }
  *out = m;
  return KITE_OK;
}

void kite_model_destroy(kite_model* model) {
  if (!model) return;
  int prev = 0;
  const bool had = cudaGetDevice(&prev) == cudaSuccess;
  cudaSetDevice(model->device);
  if (model->buf) cudaFree(model->buf);
  if (had) cudaSetDevice(prev);
  delete model;
}

}  // extern "C"
