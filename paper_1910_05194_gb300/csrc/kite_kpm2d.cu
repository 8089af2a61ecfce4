// kite_kpm2d.cu -- 2D Kubo-Bastin moments (Sec. 2b, Eq. Gammanm).
//
//   mu_nm = (1/(S R N_eff)) sum_{s,r} <a_n|b_m>,  a_n = T_n(H~) h~a r,  b_m = h~b T_m(H~) r,
// with h~d = [r_d, H~] for the directions a, b in {x, y} (positions in units of the
// lattice constant).  Because h~ is anti-Hermitian, <r| h~a T_n h~b T_m |r> = -<a_n|b_m>;
// the paper's Gamma^{a,b}_nm is -mu_nm / ((1 + d_n0)(1 + d_m0)) and
// mu_nm = <r|v_a T_n v_b T_m|r>/N for v = -i h~.
//
// Per batch of (up to) two random vectors: the A family is the recursion started from
// a_0 = h~a r_0, each step writing its output row in split-BF16 form; the B family is the
// recursion from r_0, each step writing h~b r_n (from the neighbours it already staged)
// as the rows b_n and -i b_n.  The tensor-core contraction (kite_gemm.cu) then gives
// Re and Im of <a_n|b_m> in one real GEMM per vector.
//
// In a perpendicular magnetic field (Peierls substitution, Sec. "Magnetic Field") both
// H~ and h~ carry the phase exp(i theta_oj) of each bond with an x component:
// h~_oj = (r_o - r_j) t~ exp(i theta_oj), the same gauge as the Hamiltonian, so that
// v = i[H, r]/hbar.  The step kernel's FIELD variant rotates the neighbour values before
// both the stencil sum and the velocity, and k_velocity rotates them the same way.
#include <stdlib.h>

#include "kite_internal.h"
#include "kite_step.cuh"

namespace kite {

int plan_gemm_splits(kite_ctx* ctx, int Mrows, int Nrows, int64_t Kp);
int gemm_split_bf16(kite_ctx* ctx, const void* Ahi, const void* Alo, const void* Bhi,
                    const void* Blo, int Mrows, int Nrows, int64_t Kp, int S, int sub_kb,
                    int fold, int nprod, double* part, int* S_used);
int reduce_cplx(kite_ctx* ctx, const double* part, int S, int M, int M2, double scale,
                double* out, bool accumulate);

namespace {

// Ring depth and CTAs per SM of the family step kernels, measured on the optical
// conductivity workload (1024^2, two vectors per batch): four stages at five CTAs per SM
// moved 5.88 TB/s, eight stages at three 5.55 TB/s, five or six stages at four 5.54-5.75.
// KITE_FAM_CPS=<CTAs per SM> overrides the CTA count (it is capped at the occupancy).
#ifndef KITE_FAM_STAGES
#define KITE_FAM_STAGES 4
#endif
constexpr int kFamStages = KITE_FAM_STAGES;
constexpr int kFamCtasPerSm = 5;
constexpr int kGemmSubKb = 8;   // 512 products per FP32 accumulation sub-chunk (TMEM)
constexpr int kGemmFold = 16;   // sub-chunks summed in FP32 registers before FP64
constexpr int kGemmProducts = 4; // hi*hi + hi*lo + lo*hi + lo*lo
// KITE_GEMM_PRODUCTS=3 drops lo*lo (a quarter less tensor work, a one-signed bias of up to
// ~5e-6 relative on aligned products); the default keeps all four
// The A and B families are independent recursions: by default their step launches run on
// two streams side by side, so that one family's launch fills the ramp and tail of the
// other's (KITE_FAM_STREAMS=1 keeps them in sequence on one stream).
inline bool fam_two_streams() {
  const char* e = getenv("KITE_FAM_STREAMS");
  return !(e && e[0] == '1' && e[1] == 0);
}
inline int gemm_products() {
  const char* e = getenv("KITE_GEMM_PRODUCTS");
  return (e && e[0] == '3' && e[1] == 0) ? 3 : kGemmProducts;
}

// h~ = [r_dir, H~] applied to a whole FP32 batch (one chunk = two vectors).  mode 1: writes
// the result as row `col` of the A family (and to out_vec if given); mode 2: rows `col`
// and `col + M` of the extended B family.  Bond offsets as in the step kernel's MODE 2.
// phase (or null: no field): the step kernel's table [y][s][bond][cos, sin] of the two
// bonds with an x component (honeycomb n2, n3; square n1, n2).
template <int LAT>
__global__ void k_velocity(const float4* __restrict__ in, float4* __restrict__ out_vec,
                           const float* __restrict__ vt, int Lx, int Ly, int mode, const FamOut fam,
                           const float* __restrict__ phase, int open_x, int open_y) {
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto rot = [](float4 n, float c, float sn) {  // exp(i theta) on both vectors of the chunk
    return make_float4(fmaf(c, n.x, -(sn * n.y)), fmaf(sn, n.x, c * n.y), fmaf(c, n.z, -(sn * n.w)),
                       fmaf(sn, n.z, c * n.w));
  };
  constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  const int64_t norb = (int64_t)Lx * Ly * SORB;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < norb;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(o % SORB);
    const int64_t cell = o / SORB;
    const int x = (int)(cell % Lx), y = (int)(cell / Lx);
    const int xm = x == 0 ? Lx - 1 : x - 1, xp = x + 1 == Lx ? 0 : x + 1;
    const int ym = y == 0 ? Ly - 1 : y - 1, yp = y + 1 == Ly ? 0 : y + 1;
    float4 v;
    if (LAT == KITE_HONEYCOMB) {
      // A: n1 = B(x,y), n2 = B(x+1,y-1), n3 = B(x,y-1);  B: n1 = A(x,y), n2 = A(x-1,y+1), n3 = A(x,y+1)
      const int so = 1 - s;
      const int ny = s == 0 ? ym : yp, nx = s == 0 ? xp : xm;
      const float4 n1 = __ldg(in + cell * 2 + so);
      float4 n2 = __ldg(in + ((int64_t)ny * Lx + nx) * 2 + so);
      float4 n3 = __ldg(in + ((int64_t)ny * Lx + x) * 2 + so);
      // bonds across an open boundary: A's n2 leaves at x = Lx-1 or y = 0, n3 at y = 0;
      // B's n2 at x = 0 or y = Ly-1, n3 at y = Ly-1
      const bool cy = open_y && (s == 0 ? y == 0 : y + 1 == Ly);
      if (cy || (open_x && (s == 0 ? x + 1 == Lx : x == 0))) n2 = z4;
      if (cy) n3 = z4;
      if (phase) {
        const float* p4 = phase + ((size_t)y * 2 + s) * 4;
        n2 = rot(n2, __ldg(p4), __ldg(p4 + 1));
        n3 = rot(n3, __ldg(p4 + 2), __ldg(p4 + 3));
      }
      const float sg = s == 0 ? fam.tvel : -fam.tvel;
      if (fam.dir == 0)
        v = make_float4(sg * (n3.x - n2.x), sg * (n3.y - n2.y), sg * (n3.z - n2.z), sg * (n3.w - n2.w));
      else
        v = make_float4(sg * ((n2.x + n3.x) - 2.f * n1.x), sg * ((n2.y + n3.y) - 2.f * n1.y),
                        sg * ((n2.z + n3.z) - 2.f * n1.z), sg * ((n2.w + n3.w) - 2.f * n1.w));
    } else {
      float4 n1 = __ldg(in + (fam.dir == 0 ? (int64_t)y * Lx + xm : (int64_t)ym * Lx + x));
      float4 n2 = __ldg(in + (fam.dir == 0 ? (int64_t)y * Lx + xp : (int64_t)yp * Lx + x));
      if (fam.dir == 0 ? open_x && x == 0 : open_y && y == 0) n1 = z4;
      if (fam.dir == 0 ? open_x && x + 1 == Lx : open_y && y + 1 == Ly) n2 = z4;
      if (phase && fam.dir == 0) {  // the y bonds carry no phase in the Landau gauge
        const float* p4 = phase + (size_t)y * 4;
        n1 = rot(n1, __ldg(p4), __ldg(p4 + 1));
        n2 = rot(n2, __ldg(p4 + 2), __ldg(p4 + 3));
      }
      const float t = fam.tvel;
      v = make_float4(t * (n1.x - n2.x), t * (n1.y - n2.y), t * (n1.z - n2.z), t * (n1.w - n2.w));
    }
    if (vt[o] != vt[o]) v = make_float4(0.f, 0.f, 0.f, 0.f);  // vacancy
    if (out_vec) out_vec[o] = v;
    if (mode == 1) {
      fam_store(fam, 0, fam.col, o, v.x, v.y);
      fam_store(fam, 1, fam.col, o, v.z, v.w);
    } else {
      fam_store(fam, 0, fam.col, o, v.x, v.y);
      fam_store(fam, 0, fam.col + fam.M, o, v.y, -v.x);
      fam_store(fam, 1, fam.col, o, v.z, v.w);
      fam_store(fam, 1, fam.col + fam.M, o, v.w, -v.z);
    }
  }
}

template <int LAT, bool FIELD>
int run_2d(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc, int alpha,
           int beta, double* mu_nm_dev, kite_stats* stats, const double* r0_dev_all) {
  constexpr int SORB = (LAT == KITE_HONEYCOMB) ? 2 : 1;
  constexpr int C = 1;  // two FP32 vectors per 16-byte chunk
  using Sh = StepShape<LAT, C>;
  const int M = kpm->M, R = kpm->R, Sreal = kpm->S;
  const int64_t ncell = (int64_t)sys->Lx * sys->Ly, N = ncell * SORB;
  const int64_t Kp = ((2 * N + 63) / 64) * 64;
  const int VB = 2;
  const char* fam_cps = getenv("KITE_FAM_CPS");
  const int G = grid_for<float, LAT, C, false, 1, kFamStages, FIELD>(
      ctx, (long long)((sys->Lx + Sh::TX - 1) / Sh::TX) * sys->Ly, fam_cps ? atoi(fam_cps) : kFamCtasPerSm);
  const long long units = (long long)((sys->Lx + Sh::TX - 1) / Sh::TX) * sys->Ly;
  const int Sg = plan_gemm_splits(ctx, M, 2 * M, Kp);
  const size_t vec_bytes = (size_t)ncell * SORB * C * 16;
  const size_t famA = (size_t)M * Kp, famB = (size_t)2 * M * Kp;  // bf16 elements per array

  const bool two = fam_two_streams();
  auto layout = [&](Carver& k, float** vt, void** r0, void** bA, void** bB, void** bC, void** bD,
                    __nv_bfloat16** Ah, __nv_bfloat16** Al, __nv_bfloat16** Bh,
                    __nv_bfloat16** Bl, double** part, unsigned long long** ne, float** ph) {
    *vt = k.take<float>(N);
    *ph = FIELD ? k.take<float>((size_t)sys->Ly * SORB * 4) : nullptr;
    *r0 = k.take<char>(vec_bytes);
    *bA = k.take<char>(vec_bytes);
    *bB = k.take<char>(vec_bytes);
    // the B family's own iterates when the families run side by side
    *bC = two ? k.take<char>(vec_bytes) : *bA;
    *bD = two ? k.take<char>(vec_bytes) : *bB;
    for (int v = 0; v < VB; ++v) {
      Ah[v] = k.take<__nv_bfloat16>(famA);
      Al[v] = k.take<__nv_bfloat16>(famA);
      Bh[v] = k.take<__nv_bfloat16>(famB);
      Bl[v] = k.take<__nv_bfloat16>(famB);
    }
    *part = k.take<double>((size_t)Sg * M * 2 * M);
    *ne = k.take<unsigned long long>(1);
  };
  float* vt;
  void *r0, *bA, *bB, *bC, *bD;
  __nv_bfloat16 *Ah[VB], *Al[VB], *Bh[VB], *Bl[VB];
  double* part;
  unsigned long long* ne;
  float* ph;
  {
    Carver probe(nullptr);
    layout(probe, &vt, &r0, &bA, &bB, &bC, &bD, Ah, Al, Bh, Bl, &part, &ne, &ph);
    int rc = ensure_ws(ctx, probe.used());
    if (rc != KITE_OK) return rc;
  }
  Carver w(ctx->ws);
  layout(w, &vt, &r0, &bA, &bB, &bC, &bD, Ah, Al, Bh, Bl, &part, &ne, &ph);
  if (two) {
    const int rc = ensure_aux(ctx);
    if (rc != KITE_OK) return rc;
  }
  cudaStream_t st = ctx->stream;
  if (FIELD) {
    int rc = field_phases(ctx, sys, 0, ph);
    if (rc != KITE_OK) return rc;
  }
  Open open;
  {
    const void* z = nullptr;
    int rc = open_zeros(ctx, sys, &z);
    if (rc != KITE_OK) return rc;
    open.zero = static_cast<const unsigned char*>(z);
    open.x = sys->open_x;
    open.y = sys->open_y;
  }
  if (Kp > 2 * N) {  // zero the K padding (the tail of the last K block of every row) once
    const int64_t k0 = 2 * N;  // first padded column; Kp - k0 < 64, all in the last block
    const size_t width = (size_t)(Kp - k0) * 2;
    for (int v = 0; v < VB; ++v) {
      KITE_CUDA_TRY(ctx, cudaMemset2DAsync(Ah[v] + fam_index(0, k0, M), 128, 0, width, M, st));
      KITE_CUDA_TRY(ctx, cudaMemset2DAsync(Al[v] + fam_index(0, k0, M), 128, 0, width, M, st));
      KITE_CUDA_TRY(ctx, cudaMemset2DAsync(Bh[v] + fam_index(0, k0, 2 * M), 128, 0, width, 2 * M, st));
      KITE_CUDA_TRY(ctx, cudaMemset2DAsync(Bl[v] + fam_index(0, k0, 2 * M), 128, 0, width, 2 * M, st));
    }
  }
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(mu_nm_dev, 0, sizeof(double) * 2 * (size_t)M * M, st));
  KITE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));

  const float tt = (float)(sys->t / sc.de_minus);
  // t~ times the bond-offset unit of each direction (x: a/2, y: a_cc/2 on the honeycomb)
  auto tvel_of = [&](int dir) -> float {
    if (LAT != KITE_HONEYCOMB) return tt;
    return dir == 0 ? 0.5f * tt : (float)(0.5 * (sys->t / sc.de_minus) / sqrt(3.0));
  };
  const double thr_d = floor(sys->p_vac * 4294967296.0);
  const uint64_t vac_thr =
      sys->p_vac <= 0.0 ? 0ull : (thr_d >= 4294967296.0 ? 4294967296ull : (uint64_t)thr_d);
  const uint32_t k0 = (uint32_t)sys->seed, k1 = (uint32_t)(sys->seed >> 32);
  const int blocks = (int)std::min<int64_t>((N + 255) / 256, (int64_t)ctx->num_sms * 16);
  constexpr int SM = StepShape<LAT, C, kFamStages>::SMEM_NR0;  // the family modes never stage r_0
  cudaFuncSetAttribute(k_step<float, LAT, C, true, 1, kFamStages, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       SM);
  cudaFuncSetAttribute(k_step<float, LAT, C, false, 1, kFamStages, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       SM);
  cudaFuncSetAttribute(k_step<float, LAT, C, true, 2, kFamStages, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       SM);
  cudaFuncSetAttribute(k_step<float, LAT, C, false, 2, kFamStages, FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       SM);

  FamOut fa{}, fb{};
  for (int v = 0; v < VB; ++v) {
    fa.hi[v] = Ah[v];
    fa.lo[v] = Al[v];
    fb.hi[v] = Bh[v];
    fb.lo[v] = Bl[v];
  }
  fa.Kp = fb.Kp = Kp;
  fa.rows = M;
  fb.rows = 2 * M;
  fa.M = fb.M = M;
  fa.dir = alpha;
  fb.dir = beta;
  fa.tvel = tvel_of(alpha);
  fb.tvel = tvel_of(beta);

  double gemm_s = 0.0, rec_s = 0.0, fam_bytes = 0.0;
  int64_t n_eff = 0;
  for (int s = 0; s < Sreal; ++s) {
    KITE_CUDA_TRY(ctx, cudaMemsetAsync(ne, 0, sizeof(unsigned long long), st));
    k_onsite<float><<<blocks, 256, 0, st>>>(N, sys->lattice, sys->W, 0.5 * sys->delta, sc.de_plus,
                                            sc.de_minus, vac_thr, (uint32_t)s, k0, k1, vt, ne,
                                            sys->disorder);
    unsigned long long ne_host = 0;
    KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&ne_host, ne, sizeof(ne_host), cudaMemcpyDeviceToHost, st));
    KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    n_eff = (int64_t)ne_host;
    const double scale = n_eff > 0 ? 1.0 / ((double)n_eff * R * Sreal) : 0.0;
    for (int base = 0; base < R; base += VB) {
      const int nvec = std::min(VB, R - base);
      const double* r0_in = r0_dev_all ? r0_dev_all + (size_t)s * R * N * 2 : nullptr;
      k_init_r0<float, SORB, C><<<blocks, 256, 0, st>>>(ncell, vt, base, nvec, (uint32_t)s * R,
                                                         k0, k1, r0_in, N, r0);
      KITE_CUDA_TRY(ctx, cudaGetLastError());
      KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, st));
      // fork: the B family's launches go to the second stream once r_0 is written
      cudaStream_t sb = st;
      if (two) {
        KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, st));
        KITE_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
        sb = ctx->aux;
      }
      // A family: a_0 = h~alpha r_0 (row 0, and the recursion's start vector in bB)
      fa.col = 0;
      k_velocity<LAT><<<blocks, 256, 0, st>>>(static_cast<const float4*>(r0),
                                              static_cast<float4*>(bB), vt, sys->Lx, sys->Ly, 1, fa, ph,
                                              open.x, open.y);
      auto whereA = [&](int n) -> void* { return (n & 1) ? bA : bB; };
      for (int n = 0; n + 1 < M; ++n) {
        fa.col = n + 1;
        if (n == 0)
          launch_pdl(k_step<float, LAT, C, true, 1, kFamStages, FIELD>, G, kBlock, SM, st,
              nullptr, whereA(0), whereA(1), nullptr, vt, tt, sys->Lx, sys->Ly, units, nullptr,
              nullptr, ctx->d_status, 0, fa, 0, SeriesOut{}, ph, open);
        else
          launch_pdl(k_step<float, LAT, C, false, 1, kFamStages, FIELD>, G, kBlock, SM, st,
              whereA(n - 1), whereA(n), whereA(n + 1), nullptr, vt, tt, sys->Lx, sys->Ly, units,
              nullptr, nullptr, ctx->d_status, 0, fa, 0, SeriesOut{}, ph, open);
      }
      // B family: recursion from r_0; step n writes b_n = h~beta r_n
      auto whereB = [&](int n) -> void* { return n == 0 ? r0 : ((n & 1) ? bC : bD); };
      for (int n = 0; n + 1 < M; ++n) {
        fb.col = n;
        if (n == 0)
          launch_pdl(k_step<float, LAT, C, true, 2, kFamStages, FIELD>, G, kBlock, SM, sb,
              nullptr, whereB(0), whereB(1), nullptr, vt, tt, sys->Lx, sys->Ly, units, nullptr,
              nullptr, ctx->d_status, 0, fb, 0, SeriesOut{}, ph, open);
        else
          launch_pdl(k_step<float, LAT, C, false, 2, kFamStages, FIELD>, G, kBlock, SM, sb,
              whereB(n - 1), whereB(n), whereB(n + 1), nullptr, vt, tt, sys->Lx, sys->Ly, units,
              nullptr, nullptr, ctx->d_status, 0, fb, 0, SeriesOut{}, ph, open);
      }
      fb.col = M - 1;
      k_velocity<LAT><<<blocks, 256, 0, sb>>>(static_cast<const float4*>(whereB(M - 1)), nullptr, vt,
                                              sys->Lx, sys->Ly, 2, fb, ph, open.x, open.y);
      KITE_CUDA_TRY(ctx, cudaGetLastError());
      if (two) {  // join: the contraction needs both families
        KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_join, sb));
        KITE_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0));
      }
      KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, st));
      // contraction, one vector at a time, accumulated in FP64
      KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, st));
      for (int v = 0; v < nvec; ++v) {
        int S_used = 0;
        int rc = gemm_split_bf16(ctx, Ah[v], Al[v], Bh[v], Bl[v], M, 2 * M, Kp, Sg, kGemmSubKb, kGemmFold,
                                 gemm_products(), part, &S_used);
        if (rc != KITE_OK) return rc;
        rc = reduce_cplx(ctx, part, S_used, M, M, scale, mu_nm_dev, true);
        if (rc != KITE_OK) return rc;
      }
      KITE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev3, st));
      KITE_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev3));
      float ms_rec = 0.f, ms_gemm = 0.f;
      cudaEventElapsedTime(&ms_rec, ctx->ev0, ctx->ev1);
      cudaEventElapsedTime(&ms_gemm, ctx->ev2, ctx->ev3);
      rec_s += 1e-3 * ms_rec;
      gemm_s += 1e-3 * ms_gemm;
      // algorithmic bytes of the family steps, per orbital and step: the A step reads
      // r_{n-1}, r_n and writes r_{n+1} (8 B each per vector) and a_{n+1} as BF16 hi + lo
      // (8 B per vector); the B step the same three iterates and b_n, -i b_n as hi + lo
      // (16 B per vector); each step reads the on-site term once (4 B)
      fam_bytes += (double)(M > 1 ? M - 1 : 0) * (double)N * ((32.0 + 40.0) * nvec + 2 * 4.0);
    }
  }
  int status_host = 0;
  KITE_CUDA_TRY(ctx, cudaMemcpyAsync(&status_host, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  KITE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (status_host != 0) return fail(ctx, KITE_ERR_TIMEOUT, "a bounded wait gave up in the 2D path");
  if (stats) {
    stats->seconds = rec_s + gemm_s;
    stats->step_seconds = rec_s;
    stats->step_launches = (int64_t)Sreal * ((R + VB - 1) / VB) * 2 * (M > 1 ? M - 1 : 0);
    stats->step_bytes = fam_bytes;
    stats->gemm_seconds = gemm_s;
    // BF16 products (four, or three) of an M x 2M x Kp real GEMM per vector
    stats->gemm_flops = (double)gemm_products() * 2.0 * (double)M * (2.0 * M) * (double)Kp * R * Sreal;
    stats->updates = (double)n_eff * M * R * Sreal * 2.0;
    stats->n_eff = n_eff;
    stats->grid = G;
    stats->block = kBlock;
  }
  return KITE_OK;
}

}  // namespace

int moments_2d_impl(kite_ctx* ctx, const kite_system* sys, const kite_kpm* kpm, const Scale& sc, int alpha,
                    int beta, double* mu_nm_dev, kite_stats* st, const double* r0_dev_all) {
  const bool hc = sys->lattice == KITE_HONEYCOMB;
  if (sys->flux != 0.0)
    return hc ? run_2d<KITE_HONEYCOMB, true>(ctx, sys, kpm, sc, alpha, beta, mu_nm_dev, st, r0_dev_all)
              : run_2d<KITE_SQUARE, true>(ctx, sys, kpm, sc, alpha, beta, mu_nm_dev, st, r0_dev_all);
  return hc ? run_2d<KITE_HONEYCOMB, false>(ctx, sys, kpm, sc, alpha, beta, mu_nm_dev, st, r0_dev_all)
            : run_2d<KITE_SQUARE, false>(ctx, sys, kpm, sc, alpha, beta, mu_nm_dev, st, r0_dev_all);
}

}  // namespace kite
