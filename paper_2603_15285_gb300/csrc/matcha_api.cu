// The C ABI of include/matcha.h: argument checking, plan construction,
// workspace carving and the launch sequence of Algorithm 1.
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <nvtx3/nvToolsExt.h>
#include <functional>
#include <vector>
#include "internal.cuh"

using namespace matcha;

namespace {

thread_local char g_err[512] = "";

matcha_status fail_cuda(cudaError_t e, const char *where) {
  snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
  return MATCHA_ERR_CUDA;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return fail_cuda(e_, #call); \
  } while (0)

Plan *P_(matcha_plan p) { return reinterpret_cast<Plan *>(p); }

// NVTX range over one step's enqueue (visible in timeline profilers; no cost
// without one attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

size_t real_size(const Plan &p) { return p.fp64 ? 8 : 4; }

struct Carve {
  char *base;
  size_t off = 0;
  template <typename X>
  X *take(size_t count) {
    X *r = reinterpret_cast<X *>(base + off);
    off = align_up(off + sizeof(X) * count);
    return r;
  }
};

struct AlignWs {
  void *f, *h, *c, *grid;
  int *cidx, *cflags, *ncand;
  double *ceuler, *cscore;
  int *order, *ticket;  // the cost-sorted Newton queue (one ticket per part start)
  double *ceuler0;      // the autotuner's copy of the refinement's start points
};

size_t carve_align(const Plan &p, int B, int Bt, char *base, AlignWs *w) {
  Carve cv{base};
  size_t rs = real_size(p);
  size_t coefv = (size_t)p.S * p.nlm * 2;
  w->f = cv.take<char>(rs * coefv * B);
  w->h = cv.take<char>(rs * coefv * Bt);
  w->c = cv.take<char>(rs * 4 * (size_t)p.nc * B);
  // the grid itself is only materialised when no fused SOFFT kernel applies
  w->grid = soft_grid_optional(p) ? nullptr : cv.take<char>(rs * (size_t)p.ns * p.ns * p.ns * B);
  w->cidx = cv.take<int>((size_t)B * p.P);
  w->cflags = cv.take<int>((size_t)B * p.P);
  w->ncand = cv.take<int>(B);
  w->ceuler = cv.take<double>((size_t)B * p.P * 3);
  w->cscore = cv.take<double>((size_t)B * p.P);
  w->order = cv.take<int>(B);
  w->ticket = cv.take<int>(B);
  w->ceuler0 = cv.take<double>((size_t)B * p.P * 3);
  return cv.off;
}

bool valid_stride(int s) { return s == 0 || s == 1; }

}  // namespace

namespace matcha {
// Sets the text matcha_last_error() returns on this thread.
void set_error_text(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace matcha

extern "C" {

const char *matcha_status_string(matcha_status s) {
  switch (s) {
    case MATCHA_OK: return "ok";
    case MATCHA_ERR_INVALID_ARG: return "invalid argument";
    case MATCHA_ERR_CUDA: return "CUDA error";
    case MATCHA_ERR_WORKSPACE: return "workspace too small";
    case MATCHA_ERR_TIMEOUT: return "device wait timed out";
    case MATCHA_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *matcha_last_error(void) { return g_err; }

matcha_status matcha_plan_create(const matcha_plan_desc *d, matcha_plan *out) {
  if (!d || !out) return MATCHA_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->box_n < 4 || d->box_n > 512 || d->n_shells < 1 || d->n_shells > 128) return MATCHA_ERR_INVALID_ARG;
  if (d->L0 < 1 || d->L0 > 32 || d->K_oversample < 1 || d->K_oversample > 16) return MATCHA_ERR_INVALID_ARG;
  if (d->P_max < 1 || d->P_max > MATCHA_MAX_P || d->M_iter < 1 || d->M_iter > 32) return MATCHA_ERR_INVALID_ARG;
  if (d->n_levels < 1 || d->n_levels > MATCHA_MAX_LEVELS) return MATCHA_ERR_INVALID_ARG;
  if (d->L_sched[0] != d->L0) return MATCHA_ERR_INVALID_ARG;
  for (int i = 1; i < d->n_levels; ++i)
    if (d->L_sched[i] <= d->L_sched[i - 1]) return MATCHA_ERR_INVALID_ARG;
  if (d->L_sched[d->n_levels - 1] > MATCHA_MAX_L) return MATCHA_ERR_UNSUPPORTED;
  if (d->precision < MATCHA_FP64 || d->precision > MATCHA_BF16) return MATCHA_ERR_INVALID_ARG;
  if (!isfinite(d->r_max) || !isfinite(d->step_tol) || !isfinite(d->accept_tol))
    return MATCHA_ERR_INVALID_ARG;
  if (d->refine != 0 && d->refine != 1) return MATCHA_ERR_INVALID_ARG;
  if (!isfinite(d->ball_lambda) || d->ball_lambda < 0) return MATCHA_ERR_INVALID_ARG;
  if (d->ball_lambda > 0 && d->precision >= MATCHA_TF32) {
    set_error_text("plan: the ball-harmonic radial basis runs on the CUDA-core contraction "
                   "(FP64 and FP32 plans)");
    return MATCHA_ERR_UNSUPPORTED;
  }

  Plan *p = new Plan();
  p->desc = *d;
  p->N = d->box_n; p->S = d->n_shells; p->L0 = d->L0; p->K = d->K_oversample;
  p->P = d->P_max; p->M = d->M_iter; p->nlev = d->n_levels;
  for (int i = 0; i < MATCHA_MAX_LEVELS; ++i) p->Ls[i] = i < d->n_levels ? d->L_sched[i] : 0;
  p->LJ = d->L_sched[d->n_levels - 1];
  p->R = d->r_max > 0 ? d->r_max : 0.5 * d->box_n - 1.0;
  p->fp64 = d->precision == MATCHA_FP64;
  p->refine = d->refine;
  p->tc = d->precision == MATCHA_TF32 ? 1 : d->precision == MATCHA_BF16 ? 2 : 0;
  p->step_tol = d->step_tol > 0 ? d->step_tol : (p->fp64 ? 1e-9 : 1e-6);
  p->accept_tol = d->accept_tol > 0 ? d->accept_tol : (p->fp64 ? 1e-11 : 1e-5);
  p->nt = p->LJ + 1;
  p->np = 2 * p->LJ + 2;
  p->nlm = (p->LJ + 1) * (p->LJ + 2) / 2;
  p->npairs = (p->LJ + 1) * (p->LJ + 1);
  p->npairs0 = (p->L0 + 1) * (p->L0 + 1);
  p->ns = 2 * p->K * (p->L0 + 1);
  // F rows of the analysis: the orders padded to a multiple of 4, plus one, so
  // that the 4-ring x 4-order tiles' stores of consecutive ring quads fall in
  // different banks (an even row stride of 4 Mp complex values would repeat them)
  p->Mp = (p->LJ + 1 + 3) / 4 * 4 + 1;
  p->Qf = (p->LJ + 1) / 2;
  p->Mq = (p->LJ / 2 + 1 + 3) / 4 * 4;
  p->ngroups = (p->LJ + 1) * (p->LJ + 2) / 2;
  p->nc = 2 * group_entries_host(p->LJ);
  p->nc0 = pair_entries_host(p->L0);
  if (!newton_fits(*p)) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "plan: the refinement kernel's shared-memory tables do not fit for P_max = %d, "
             "L_J = %d in this precision", p->P, p->LJ);
    delete p;
    set_error_text(msg);
    return MATCHA_ERR_UNSUPPORTED;
  }
  if (!soft_fits(*p)) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "plan: no SOFFT kernel's shared memory fits L0 = %d with K = %d in this precision "
             "(%d points per angle)", p->L0, p->K, p->ns);
    delete p;
    set_error_text(msg);
    return MATCHA_ERR_UNSUPPORTED;
  }
  if (p->tc && !correlate_tc_fits(p->S, p->LJ, p->tc == 2 ? 2 : 4)) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "plan: the tensor-core contraction takes L_J <= 63 (4(L_J+1) accumulator columns "
             "<= 256); L_J = %d", p->LJ);
    delete p;
    set_error_text(msg);
    return MATCHA_ERR_UNSUPPORTED;
  }
  std::vector<int> base(p->npairs), off0(p->npairs0);
  for (int m = 0; m <= p->LJ; ++m)
    for (int n = -m; n <= m; ++n) {
      int q = m * m + n + m;
      base[q] = (int)pair_base_host(m, n, p->LJ);
      if (m <= p->L0) off0[q] = (int)pair_offset_host(m, n, p->L0);
    }
  size_t rs = real_size(*p);
  size_t sz = 0;
  auto add = [&](size_t bytes) { size_t o = sz; sz = align_up(sz + bytes); return o; };
  size_t o_rs = add(8 * p->S), o_w = add(8 * p->S), o_x = add(8 * p->nt), o_wj = add(8 * p->nt);
  size_t o_pt = add(rs * p->nlm * p->nt), o_phi = add(rs * 2 * p->np), o_tw = add(rs * 2 * p->ns);
  size_t o_sd = add(rs * p->ns * p->nc0), o_rc = add(rs * 4 * p->nc), o_K = add(rs * 4 * p->ngroups);
  size_t o_off = add(4 * p->npairs), o_off0 = add(4 * p->npairs0);
  size_t o_ptl = add(rs * p->nlm * p->nt), o_leg = add(4 * (size_t)p->nlm);
  size_t o_dcs = add(rs * 4 * (size_t)p->Qf * p->Mq);
  size_t o_ring = add(rs * 2 * (size_t)p->S * p->nt);
  size_t o_err = add(sizeof(int));
  size_t o_fft = add(rs * 2 * (size_t)p->N);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { delete p; return fail_cuda(e, "cudaGetDevice"); }
  e = cudaMalloc(&p->base, sz);
  if (e != cudaSuccess) { delete p; return fail_cuda(e, "cudaMalloc(plan tables)"); }
  char *b = (char *)p->base;
  p->rs = (double *)(b + o_rs); p->wrad = (double *)(b + o_w);
  p->xj = (double *)(b + o_x); p->wj = (double *)(b + o_wj);
  p->ptab = b + o_pt; p->phi_cs = b + o_phi; p->soft_tw = b + o_tw; p->soft_d = b + o_sd;
  p->rcoef = b + o_rc; p->seedK = b + o_K;
  p->pair_base = (int *)(b + o_off); p->pair_off0 = (int *)(b + o_off0);
  p->ptab_leg = b + o_ptl; p->leg_lm = (int *)(b + o_leg);
  p->dft_cs = b + o_dcs;
  p->ring = b + o_ring;
  p->dev_err = (int *)(b + o_err);
  p->fft_tw = b + o_fft;
  {  // radices of the box FFT (translation search): 4s first, then 2, 3, 5
    int n = p->N, np = 0;
    while (n % 4 == 0 && np < 16) { p->fft_radix[np++] = 4; n /= 4; }
    while (n % 2 == 0 && np < 16) { p->fft_radix[np++] = 2; n /= 2; }
    while (n % 3 == 0 && np < 16) { p->fft_radix[np++] = 3; n /= 3; }
    while (n % 5 == 0 && np < 16) { p->fft_radix[np++] = 5; n /= 5; }
    p->fft_npass = n == 1 ? np : 0;
  }
  std::vector<double> tw(2 * (size_t)p->N);
  for (int j = 0; j < p->N; ++j) {
    tw[2 * j] = cos(2.0 * M_PI * j / p->N);
    tw[2 * j + 1] = -sin(2.0 * M_PI * j / p->N);
  }
  std::vector<float> twf(tw.begin(), tw.end());
  e = cudaMemset(p->dev_err, 0, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->fft_tw, p->fp64 ? (const void *)tw.data() : (const void *)twf.data(),
                   rs * 2 * (size_t)p->N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->pair_base, base.data(), 4 * p->npairs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->pair_off0, off0.data(), 4 * p->npairs0, cudaMemcpyHostToDevice);
  {  // Legendre items: m ascending, then the parity of l + m, then l
    std::vector<int> leg;
    for (int m = 0; m <= p->LJ; ++m)
      for (int par = 0; par < 2; ++par)
        for (int l = m + par; l <= p->LJ; l += 2) leg.push_back((l << 16) | m);
    if (e == cudaSuccess) e = cudaMemcpy(p->leg_lm, leg.data(), 4 * leg.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = build_tables(*p, 0);
  if (e != cudaSuccess) {
    cudaFree(p->base);
    delete p;
    return fail_cuda(e, "plan tables");
  }
  if (d->ball_lambda > 0) {  // ball-harmonic radial table (host), then uploaded
    p->ball_lambda = d->ball_lambda;
    std::vector<double> r(p->S), w(p->S), W;
    std::vector<int> counts;
    e = cudaMemcpy(r.data(), p->rs, 8 * p->S, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w.data(), p->wrad, 8 * p->S, cudaMemcpyDeviceToHost);
    int kmax = e == cudaSuccess ? ball_tables(p->LJ, p->S, p->R, p->ball_lambda, r.data(), w.data(),
                                              W, counts) : 0;
    if (e == cudaSuccess && (kmax < 1 || kmax > p->S)) {
      char msg[200];
      snprintf(msg, sizeof(msg),
               "plan: Lambda = %g keeps %d radial functions at l = 0; the ball basis needs "
               "1 .. n_shells (%d)", p->ball_lambda, kmax, p->S);
      cudaFree(p->base);
      delete p;
      set_error_text(msg);
      return MATCHA_ERR_UNSUPPORTED;
    }
    p->ball_kmax = kmax;
    const size_t nW = W.size(), oK = align_up(rs * nW);
    if (e == cudaSuccess) e = cudaMalloc(&p->ball_W, oK + sizeof(int) * counts.size());
    if (e == cudaSuccess) {
      p->ball_K = (int *)((char *)p->ball_W + oK);
      std::vector<float> Wf(W.begin(), W.end());
      e = cudaMemcpy(p->ball_W, p->fp64 ? (const void *)W.data() : (const void *)Wf.data(), rs * nW,
                     cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(p->ball_K, counts.data(), sizeof(int) * counts.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      if (p->ball_W) cudaFree(p->ball_W);
      cudaFree(p->base);
      delete p;
      return fail_cuda(e, "plan ball tables");
    }
  }
  *out = reinterpret_cast<matcha_plan>(p);
  return MATCHA_OK;
}

matcha_status matcha_plan_destroy(matcha_plan plan) {
  if (!plan) return MATCHA_OK;
  Plan *p = P_(plan);
  cudaDeviceSynchronize();
  for (auto &ev : p->ev)
    if (ev) cudaEventDestroy(ev);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  for (int i = 0; i < Plan::NSPLIT - 1; ++i) {
    if (p->split_stream[i]) cudaStreamDestroy(p->split_stream[i]);
    if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  destroy_texsets(*p);
  if (p->ball_W) cudaFree(p->ball_W);
  cudaError_t e = cudaFree(p->base);
  delete p;
  if (e != cudaSuccess) return fail_cuda(e, "cudaFree(plan tables)");
  return MATCHA_OK;
}

matcha_status matcha_plan_device_status(matcha_plan plan, int *bits) {
  if (!plan || !bits) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  CK(cudaMemcpy(bits, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (*bits) CK(cudaMemset(p->dev_err, 0, sizeof(int)));
  return *bits ? MATCHA_ERR_TIMEOUT : MATCHA_OK;
}

matcha_status matcha_plan_set_wait_limit(matcha_plan plan, long polls) {
  if (!plan || polls < -1) return MATCHA_ERR_INVALID_ARG;
  P_(plan)->wait_limit = polls;
  return MATCHA_OK;
}

matcha_status matcha_plan_info(matcha_plan plan, matcha_plan_info_t *info) {
  if (!plan || !info) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  info->n_lm = p->nlm;
  info->coeff_count = (long)p->S * p->nlm;
  info->corr_entries = p->nc;
  info->n_pairs = p->npairs;
  info->soft_n = p->ns;
  info->real_bytes = (int)real_size(*p);
  return MATCHA_OK;
}

matcha_status matcha_plan_table(matcha_plan plan, int which, double *host_out, long capacity,
                                long *count) {
  if (!plan || !count || capacity < 0) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  const double *src;
  long n;
  switch (which) {
    case 0: src = p->rs; n = p->S; break;
    case 1: src = p->wrad; n = p->S; break;
    case 2: src = p->xj; n = p->nt; break;
    case 3: src = p->wj; n = p->nt; break;
    default: return MATCHA_ERR_INVALID_ARG;
  }
  *count = n;
  if (host_out && capacity > 0) {
    long k = capacity < n ? capacity : n;
    CK(cudaMemcpy(host_out, src, sizeof(double) * k, cudaMemcpyDeviceToHost));
  }
  return MATCHA_OK;
}

matcha_status matcha_workspace_size(matcha_plan plan, int B, size_t *bytes) {
  if (!plan || !bytes || B < 0) return MATCHA_ERR_INVALID_ARG;
  AlignWs w;
  *bytes = carve_align(*P_(plan), B, B, nullptr, &w);
  return MATCHA_OK;
}

matcha_status matcha_analyze(matcha_plan plan, const float *vols, int B, void *coeffs, void *stream) {
  if (!plan || B < 0 || (B > 0 && (!vols || !coeffs))) return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  Plan *p = P_(plan);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p->fp64 ? launch_analyze<double>(*p, vols, B, (double *)coeffs, st)
                          : launch_analyze<float>(*p, vols, B, (float *)coeffs, st);
  if (e != cudaSuccess) return fail_cuda(e, "analyze");
  return MATCHA_OK;
}

matcha_status matcha_correlate_coeffs(matcha_plan plan, const void *f, const void *h, int B,
                                      int h_batch_stride, void *c, void *stream) {
  if (!plan || B < 0 || !valid_stride(h_batch_stride) || (B > 0 && (!f || !h || !c)))
    return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  Plan *p = P_(plan);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p->fp64 ? launch_correlate<double>(*p, (const double *)f, (const double *)h, B,
                                                     h_batch_stride, (double *)c, st)
                          : launch_correlate<float>(*p, (const float *)f, (const float *)h, B,
                                                    h_batch_stride, (float *)c, st);
  if (e != cudaSuccess) return fail_cuda(e, "correlate_coeffs");
  return MATCHA_OK;
}

matcha_status matcha_soft_search(matcha_plan plan, const void *c, int B, const int *P_per,
                                 void *grid, int *idx, double *euler, double *score, int *n_cand,
                                 void *stream) {
  if (!plan || B < 0 || (B > 0 && (!c || !grid || !idx || !euler || !score || !n_cand)))
    return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  Plan *p = P_(plan);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p->fp64 ? launch_soft<double>(*p, (const double *)c, B, P_per, (double *)grid,
                                                idx, euler, score, n_cand, st)
                          : launch_soft<float>(*p, (const float *)c, B, P_per, (float *)grid, idx,
                                               euler, score, n_cand, st);
  if (e != cudaSuccess) return fail_cuda(e, "soft_search");
  return MATCHA_OK;
}

matcha_status matcha_newton_march(matcha_plan plan, const void *c, int B, const int *n_cand,
                                  double *euler, double *score, int *cflags, long long *work,
                                  void *stream) {
  if (!plan || B < 0 || (B > 0 && (!c || !n_cand || !euler || !score || !cflags)))
    return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p->fp64 ? launch_newton<double>(*p, (const double *)c, B, n_cand, euler, score,
                                                  cflags, work, st)
                          : launch_newton<float>(*p, (const float *)c, B, n_cand, euler, score,
                                                 cflags, work, st);
  if (e != cudaSuccess) return fail_cuda(e, "newton_march");
  return MATCHA_OK;
}

matcha_status matcha_objective(matcha_plan plan, const void *c, int B, int L, int Q,
                               const double *euler, double *out, void *stream) {
  if (!plan || B < 0 || Q < 0) return MATCHA_ERR_INVALID_ARG;
  if (B == 0 || Q == 0) return MATCHA_OK;
  if (!c || !euler || !out) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  if (Q > p->P || L < 0 || L > p->LJ) return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p->fp64 ? launch_objective<double>(*p, (const double *)c, B, L, Q, euler, out, st)
                          : launch_objective<float>(*p, (const float *)c, B, L, Q, euler, out, st);
  if (e != cudaSuccess) return fail_cuda(e, "objective");
  return MATCHA_OK;
}

matcha_status matcha_final_select(matcha_plan plan, int B, const int *P_per, const int *n_cand,
                                  const double *cand_euler, const double *cand_score,
                                  const int *cand_flags, double *euler, double *R, double *score,
                                  int *best_p, int *flags, void *stream) {
  if (!plan || B < 0 || (B > 0 && (!n_cand || !cand_euler || !cand_score || !cand_flags || !euler ||
                                   !R || !score || !best_p || !flags)))
    return MATCHA_ERR_INVALID_ARG;
  cudaError_t e = launch_final_select(*P_(plan), B, P_per, n_cand, cand_euler, cand_score,
                                      cand_flags, euler, R, score, best_p, flags,
                                      (cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(e, "final_select");
  return MATCHA_OK;
}

// Steps a1..a7 for the particle range covered by `w` (workspace arrays already
// offset to the range's first particle); the templates' coefficients are
// analysed here unless `h_ready`.
static matcha_status align_range(matcha_plan plan, const float *particles, const float *templates,
                                 int B, int tstride, bool h_ready, const int *P_per, double *euler,
                                 double *R, double *score, int *best_p, int *flags,
                                 const AlignWs &w, void *stream) {
  Plan *p = P_(plan);
  const int Bt = tstride ? B : 1;
  matcha_status s;
  {
    Range r("a1+a2 analysis");
    if ((s = matcha_analyze(plan, particles, B, w.f, stream))) return s;
    if (!h_ready && (s = matcha_analyze(plan, templates, Bt, w.h, stream))) return s;
  }
  {
    Range r("a3 contraction");
    if ((s = matcha_correlate_coeffs(plan, w.f, w.h, B, tstride, w.c, stream))) return s;
  }
  {
    Range r("a4+a5 SOFFT search");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = p->fp64 ? launch_soft<double>(*p, (const double *)w.c, B, P_per,
                                                  (double *)w.grid, w.cidx, w.ceuler, w.cscore,
                                                  w.ncand, st)
                            : launch_soft<float>(*p, (const float *)w.c, B, P_per, (float *)w.grid,
                                                 w.cidx, w.ceuler, w.cscore, w.ncand, st);
    if (e != cudaSuccess) return fail_cuda(e, "soft_search");
  }
  {
    Range r("a6 Newton march");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->tune_newton == 2) {  // persistent CTAs on the cost-sorted queue
      cudaError_t e = p->fp64 ? launch_newton_queue<double>(*p, (const double *)w.c, B, w.ncand,
                                                            w.ceuler, w.cscore, w.cflags, nullptr,
                                                            w.order, w.ticket, st)
                              : launch_newton_queue<float>(*p, (const float *)w.c, B, w.ncand,
                                                           w.ceuler, w.cscore, w.cflags, nullptr,
                                                           w.order, w.ticket, st);
      if (e != cudaSuccess) return fail_cuda(e, "newton_march");
    } else if ((s = matcha_newton_march(plan, w.c, B, w.ncand, w.ceuler, w.cscore, w.cflags,
                                        nullptr, stream))) {
      return s;
    }
  }
  Range r("a7 final selection");
  return matcha_final_select(plan, B, P_per, w.ncand, w.ceuler, w.cscore, w.cflags, euler, R, score,
                             best_p, flags, stream);
}

// The workspace arrays of `w` advanced to particle b0.
static AlignWs ws_at(const Plan &p, const AlignWs &w, long b0, int tstride) {
  const size_t rs = real_size(p), coefv = (size_t)p.S * p.nlm * 2;
  AlignWs o = w;
  o.f = (char *)w.f + rs * coefv * b0;
  o.h = (char *)w.h + rs * coefv * (tstride ? b0 : 0);
  o.c = (char *)w.c + rs * 4 * (size_t)p.nc * b0;
  o.grid = w.grid ? (char *)w.grid + rs * (size_t)p.ns * p.ns * p.ns * b0 : nullptr;
  o.cidx = w.cidx + b0 * p.P;
  o.order = w.order + b0;
  o.ticket = w.ticket + b0;
  o.cflags = w.cflags + b0 * p.P;
  o.ncand = w.ncand + b0;
  o.ceuler = w.ceuler + 3 * b0 * p.P;
  o.cscore = w.cscore + b0 * p.P;
  return o;
}

matcha_status matcha_align(matcha_plan plan, const float *particles, const float *templates, int B,
                           int tstride, const int *P_per, double *euler, double *R, double *score,
                           int *best_p, int *flags, void *ws, size_t ws_bytes, void *stream) {
  if (!plan || B < 0 || !valid_stride(tstride)) return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  if (!particles || !templates || !euler || !R || !score || !best_p || !flags || !ws)
    return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  const int Bt = tstride ? B : 1;
  AlignWs w;
  size_t need = carve_align(*p, B, Bt, (char *)ws, &w);
  if (ws_bytes < need) return MATCHA_ERR_WORKSPACE;
  Range all("matcha_align");
  // one pass for small batches, and where the SOFFT grid goes through HBM
  // (large L0: its grid and scan kernels gain nothing from the split)
  if (B < 256 || !soft_grid_optional(*p))
    return align_range(plan, particles, templates, B, tstride, false, P_per, euler, R, score,
                       best_p, flags, w, stream);
  // Parts of at least 128 particles on up to NSPLIT streams (the caller's and
  // ones the plan owns), joined back into the caller's stream: each part's
  // kernels fill the others' wave tails.  Every particle's arithmetic is the
  // same as in one pass.
  if (!p->ev_fork) {
    CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    for (int i = 0; i < Plan::NSPLIT - 1; ++i) {
      CK(cudaStreamCreateWithFlags(&p->split_stream[i], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming));
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  matcha_status s;
  bool h_ready = false;
  if (!tstride) {  // one shared template: analysed once, before the fork
    if ((s = matcha_analyze(plan, templates, 1, w.h, stream))) return s;
    h_ready = true;
  }
  int np = B / 128;
  if (np > Plan::NSPLIT) np = Plan::NSPLIT;
  CK(cudaEventRecord(p->ev_fork, st));
  const size_t vox = (size_t)p->N * p->N * p->N;
  // Parts k >= joined (k > 0) have been forked and have recorded their join
  // event.  An error in one part still joins every forked part back into the
  // caller's stream, so no fork is left open (in a capture, or for the
  // ordering of later work on `stream`).
  int joined = np;
  s = MATCHA_OK;
  for (int k = np - 1; k >= 0; --k) {
    const int b0 = (int)((long)B * k / np), b1 = (int)((long)B * (k + 1) / np);
    cudaStream_t sk = k ? p->split_stream[k - 1] : st;
    if (k) {
      cudaError_t e = cudaStreamWaitEvent(sk, p->ev_fork, 0);
      if (e != cudaSuccess) { s = fail_cuda(e, "matcha_align fork"); break; }
    }
    const AlignWs wk = ws_at(*p, w, b0, tstride);
    s = align_range(plan, particles + vox * b0, tstride ? templates + vox * b0 : templates,
                    b1 - b0, tstride, h_ready, P_per ? P_per + b0 : nullptr, euler + 3 * b0,
                    R + 9 * b0, score + b0, best_p + b0, flags + b0, wk, sk);
    if (k) {
      cudaError_t e = cudaEventRecord(p->ev_join[k - 1], sk);
      if (e != cudaSuccess) {
        if (s == MATCHA_OK) s = fail_cuda(e, "matcha_align join");
        break;
      }
      joined = k;
    }
    if (s != MATCHA_OK) break;
  }
  for (int k = joined; k < np; ++k) {
    cudaError_t e = cudaStreamWaitEvent(st, p->ev_join[k - 1], 0);
    if (e != cudaSuccess && s == MATCHA_OK) s = fail_cuda(e, "matcha_align join");
  }
  return s;
}

// Host-buffer path: the batch is split into up to 8 chunks (of at least 128
// particles); chunk i+1 is copied to the device on the plan's copy stream
// while chunk i is aligned on the caller's stream.  Host-to-device bandwidth
// bounds this path, so only the last chunk's alignment is exposed.
static int host_chunk(int B) {
  int ch = (B + 7) / 8;
  return ch < 128 ? (B < 128 ? B : 128) : ch;
}

matcha_status matcha_host_workspace_size(matcha_plan plan, int B, int tstride, size_t *bytes) {
  if (!plan || !bytes || B < 0 || !valid_stride(tstride)) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  AlignWs w;
  const int Bt = tstride ? B : 1, CH = host_chunk(B);
  size_t vox = (size_t)p->N * p->N * p->N;
  size_t sz = align_up(carve_align(*p, CH, tstride ? CH : 1, nullptr, &w));
  sz += align_up(sizeof(float) * vox * B) + align_up(sizeof(float) * vox * Bt);
  sz += align_up(sizeof(double) * 13 * B) + align_up(sizeof(int) * 2 * B);
  *bytes = sz;
  return MATCHA_OK;
}

matcha_status matcha_align_host(matcha_plan plan, const float *particles, const float *templates,
                                int B, int tstride, double *euler, double *R, double *score,
                                int *best_p, int *flags, void *ws, size_t ws_bytes, void *stream) {
  if (!plan || B < 0 || !valid_stride(tstride)) return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  if (!particles || !templates || !euler || !R || !score || !best_p || !flags || !ws)
    return MATCHA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return MATCHA_ERR_INVALID_ARG;
  size_t need;
  matcha_status s = matcha_host_workspace_size(plan, B, tstride, &need);
  if (s) return s;
  if (ws_bytes < need) return MATCHA_ERR_WORKSPACE;
  Plan *p = P_(plan);
  if (!p->copy_stream) {
    CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    for (auto &ev : p->ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  const int Bt = tstride ? B : 1, CH = host_chunk(B);
  AlignWs w;
  size_t inner = align_up(carve_align(*p, CH, tstride ? CH : 1, nullptr, &w));
  Carve cv{(char *)ws + inner};
  size_t vox = (size_t)p->N * p->N * p->N;
  float *dpart = cv.take<float>(vox * B);
  float *dtemp = cv.take<float>(vox * Bt);
  double *dout = cv.take<double>(13 * (size_t)B);
  int *iout = cv.take<int>(2 * (size_t)B);
  cudaStream_t st = (cudaStream_t)stream, cs = p->copy_stream;
  const int nch = (B + CH - 1) / CH;
  // the copies must not overtake earlier work of the caller's stream
  CK(cudaEventRecord(p->ev[8], st));
  CK(cudaStreamWaitEvent(cs, p->ev[8], 0));
  if (!tstride) CK(cudaMemcpyAsync(dtemp, templates, sizeof(float) * vox, cudaMemcpyHostToDevice, cs));
  for (int c = 0; c < nch; ++c) {
    size_t b0 = (size_t)c * CH, nb = (size_t)(B - (int)b0 < CH ? B - (int)b0 : CH);
    CK(cudaMemcpyAsync(dpart + b0 * vox, particles + b0 * vox, sizeof(float) * vox * nb,
                       cudaMemcpyHostToDevice, cs));
    if (tstride)
      CK(cudaMemcpyAsync(dtemp + b0 * vox, templates + b0 * vox, sizeof(float) * vox * nb,
                         cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(p->ev[c], cs));
  }
  for (int c = 0; c < nch; ++c) {
    size_t b0 = (size_t)c * CH;
    int nb = B - (int)b0 < CH ? B - (int)b0 : CH;
    CK(cudaStreamWaitEvent(st, p->ev[c], 0));
    s = matcha_align(plan, dpart + b0 * vox, tstride ? dtemp + b0 * vox : dtemp, nb, tstride,
                     nullptr, dout + 3 * b0, dout + 3 * B + 9 * b0, dout + 12 * B + b0, iout + b0,
                     iout + B + b0, ws, inner, stream);
    if (s) return s;
  }
  CK(cudaMemcpyAsync(euler, dout, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(R, dout + 3 * B, sizeof(double) * 9 * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(score, dout + 12 * B, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(best_p, iout, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(flags, iout + B, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MATCHA_OK;
}

// Autotuning of the tile choices that leave every result bit unchanged.
static float time_ms(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps,
                     const std::function<cudaError_t()> &fn, cudaError_t *err) {
  *err = fn();  // warm-up (and attribute setup)
  if (*err != cudaSuccess) return -1.0f;
  float best = -1.0f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, st);
    *err = fn();
    cudaEventRecord(e1, st);
    if (*err == cudaSuccess) *err = cudaEventSynchronize(e1);
    if (*err != cudaSuccess) return -1.0f;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0 || ms < best) best = ms;
  }
  return best;
}

matcha_status matcha_plan_autotune(matcha_plan plan, const float *particles, const float *templates,
                                   int B, int tstride, const int *P_per, void *ws, size_t ws_bytes,
                                   void *stream, matcha_tune_report *rep) {
  if (!plan || B < 1 || !valid_stride(tstride) || !particles || !templates || !ws || !rep)
    return MATCHA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return MATCHA_ERR_INVALID_ARG;
  size_t need;
  matcha_status s = matcha_workspace_size(plan, B, &need);
  if (s) return s;
  if (ws_bytes < need) return MATCHA_ERR_WORKSPACE;
  Plan *p = P_(plan);
  AlignWs w;
  carve_align(*p, B, tstride ? B : 1, (char *)ws, &w);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t err = cudaSuccess;
  memset(rep, 0, sizeof(*rep));
  const int cand[4] = {1, 2, 4, 8};
  int bestG = 0;
  float bestT = -1.0f;
  for (int i = 0; i < 4; ++i) {
    rep->analyze_ms[i] = -1.0f;
    if (!analyze_shells_ok(*p, cand[i])) continue;
    p->tune_shells = cand[i];
    float t = time_ms(st, e0, e1, 3, [&]() {
      return p->fp64 ? launch_analyze<double>(*p, particles, B, (double *)w.f, st)
                     : launch_analyze<float>(*p, particles, B, (float *)w.f, st);
    }, &err);
    if (err != cudaSuccess) break;
    rep->analyze_ms[i] = t;
    if (bestT < 0 || t < bestT) { bestT = t; bestG = cand[i]; }
  }
  p->tune_shells = bestG;
  rep->analyze_shells = bestG;
  if (err == cudaSuccess && p->tc) {
    const int Bt = tstride ? B : 1;
    err = launch_analyze<float>(*p, particles, B, (float *)w.f, st);
    if (err == cudaSuccess) err = launch_analyze<float>(*p, templates, Bt, (float *)w.h, st);
    int bestC = 0;
    float bc = -1.0f;
    for (int k = 1; k <= 2 && err == cudaSuccess; ++k) {
      p->tune_tc_ctas = k;
      float t = time_ms(st, e0, e1, 3, [&]() {
        return launch_correlate<float>(*p, (const float *)w.f, (const float *)w.h, B, tstride,
                                       (float *)w.c, st);
      }, &err);
      rep->tc_ms[k - 1] = t;
      if (err == cudaSuccess && (bc < 0 || t < bc)) { bc = t; bestC = k; }
    }
    p->tune_tc_ctas = bestC;
    rep->tc_ctas_per_sm = bestC;
  }
  rep->soft_ms[0] = rep->soft_ms[1] = rep->soft_ms[2] = -1.0f;
  if (err == cudaSuccess && (soft_warps_ok(*p) || soft_tile_ok(*p))) {  // 32-bit plans: the SOFFT kernel
    const int Bt = tstride ? B : 1;
    err = launch_analyze<float>(*p, particles, B, (float *)w.f, st);
    if (err == cudaSuccess) err = launch_analyze<float>(*p, templates, Bt, (float *)w.h, st);
    if (err == cudaSuccess)
      err = launch_correlate<float>(*p, (const float *)w.f, (const float *)w.h, B, tstride,
                                    (float *)w.c, st);
    int bestK = 0;
    float bk = -1.0f;
    for (int k = 1; k <= 3 && err == cudaSuccess; ++k) {
      if ((k == 2 && !soft_warps_ok(*p)) || (k == 3 && !soft_tile_ok(*p))) continue;
      p->tune_soft = k;
      float t = time_ms(st, e0, e1, 3, [&]() {
        return launch_soft<float>(*p, (const float *)w.c, B, nullptr, nullptr, w.cidx, w.ceuler,
                                  w.cscore, w.ncand, st);
      }, &err);
      rep->soft_ms[k - 1] = t;
      if (err == cudaSuccess && (bk < 0 || t < bk)) { bk = t; bestK = k; }
    }
    p->tune_soft = bestK;
    rep->soft_kernel = bestK;
  }
  rep->newton_ms[0] = rep->newton_ms[1] = -1.0f;
  if (err == cudaSuccess) {  // the refinement schedule, from the same start points each time
    const int Bt = tstride ? B : 1;
    err = p->fp64 ? launch_analyze<double>(*p, particles, B, (double *)w.f, st)
                  : launch_analyze<float>(*p, particles, B, (float *)w.f, st);
    if (err == cudaSuccess)
      err = p->fp64 ? launch_analyze<double>(*p, templates, Bt, (double *)w.h, st)
                    : launch_analyze<float>(*p, templates, Bt, (float *)w.h, st);
    if (err == cudaSuccess)
      err = p->fp64 ? launch_correlate<double>(*p, (const double *)w.f, (const double *)w.h, B,
                                               tstride, (double *)w.c, st)
                    : launch_correlate<float>(*p, (const float *)w.f, (const float *)w.h, B, tstride,
                                              (float *)w.c, st);
    if (err == cudaSuccess)
      err = p->fp64 ? launch_soft<double>(*p, (const double *)w.c, B, P_per, (double *)w.grid,
                                          w.cidx, w.ceuler, w.cscore, w.ncand, st)
                    : launch_soft<float>(*p, (const float *)w.c, B, P_per, (float *)w.grid, w.cidx,
                                         w.ceuler, w.cscore, w.ncand, st);
    // the refinement overwrites its start points: each timed run starts from a copy
    const size_t eb = sizeof(double) * 3 * (size_t)B * p->P;
    double *start = w.ceuler0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(start, w.ceuler, eb, cudaMemcpyDeviceToDevice, st);
    int bestN = 0;
    float bn = -1.0f;
    for (int k = 1; k <= 2 && err == cudaSuccess; ++k) {
      float t = time_ms(st, e0, e1, 3, [&]() {
        cudaError_t e2 = cudaMemcpyAsync(w.ceuler, start, eb, cudaMemcpyDeviceToDevice, st);
        if (e2 != cudaSuccess) return e2;
        if (k == 1)
          return p->fp64 ? launch_newton<double>(*p, (const double *)w.c, B, w.ncand, w.ceuler,
                                                 w.cscore, w.cflags, nullptr, st)
                         : launch_newton<float>(*p, (const float *)w.c, B, w.ncand, w.ceuler,
                                                w.cscore, w.cflags, nullptr, st);
        return p->fp64 ? launch_newton_queue<double>(*p, (const double *)w.c, B, w.ncand, w.ceuler,
                                                     w.cscore, w.cflags, nullptr, w.order, w.ticket, st)
                       : launch_newton_queue<float>(*p, (const float *)w.c, B, w.ncand, w.ceuler,
                                                    w.cscore, w.cflags, nullptr, w.order, w.ticket, st);
      }, &err);
      rep->newton_ms[k - 1] = t;
      if (err == cudaSuccess && (bn < 0 || t < bn)) { bn = t; bestN = k; }
    }
    p->tune_newton = bestN;
    rep->newton_sched = bestN;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail_cuda(err, "autotune");
  return MATCHA_OK;
}

matcha_status matcha_plan_set_tiles(matcha_plan plan, const matcha_tune_report *ch) {
  if (!plan || !ch) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  if (ch->analyze_shells && !analyze_shells_ok(*p, ch->analyze_shells)) return MATCHA_ERR_INVALID_ARG;
  if (ch->tc_ctas_per_sm && (!p->tc || ch->tc_ctas_per_sm < 1 || ch->tc_ctas_per_sm > 2))
    return MATCHA_ERR_INVALID_ARG;
  if (ch->soft_kernel && (ch->soft_kernel < 1 || ch->soft_kernel > 3 ||
                          (ch->soft_kernel == 2 && !soft_warps_ok(*p)) ||
                          (ch->soft_kernel == 3 && !soft_tile_ok(*p))))
    return MATCHA_ERR_INVALID_ARG;
  if (ch->newton_sched < 0 || ch->newton_sched > 2) return MATCHA_ERR_INVALID_ARG;
  p->tune_shells = ch->analyze_shells;
  p->tune_tc_ctas = ch->tc_ctas_per_sm;
  p->tune_soft = ch->soft_kernel;
  p->tune_newton = ch->newton_sched;
  return MATCHA_OK;
}

// Template gradient of the refined scores: workspace = per-particle shifts
// (v, C) and, for a shared template, the per-particle coefficient gradients
// before their sum.
static size_t grad_ws(const Plan &p, int B, int tstride, double **shift, void **X, char *base) {
  Carve cv{base};
  *shift = cv.take<double>(4 * (size_t)B);
  *X = tstride ? nullptr : cv.take<char>(real_size(p) * 2 * (size_t)p.S * p.nlm * B);
  return cv.off;
}

matcha_status matcha_template_grad_workspace_size(matcha_plan plan, int B, int tstride,
                                                  size_t *bytes) {
  if (!plan || !bytes || B < 0 || !valid_stride(tstride)) return MATCHA_ERR_INVALID_ARG;
  double *sh;
  void *X;
  *bytes = grad_ws(*P_(plan), B, tstride, &sh, &X, nullptr);
  return MATCHA_OK;
}

matcha_status matcha_template_grad(matcha_plan plan, const void *f, const void *c, int B,
                                   int tstride, const double *euler, const double *weight,
                                   void *coef_grad, double *vox_grad, double *shift_out,
                                   int *flags, void *ws, size_t ws_bytes, void *stream) {
  if (!plan || B < 0 || !valid_stride(tstride)) return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  if (!f || !c || !euler || !coef_grad || !ws) return MATCHA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return MATCHA_ERR_INVALID_ARG;
  Plan *p = P_(plan);
  if (!backward_fits(*p)) {
    set_error_text("template gradient: the per-degree tables of this bandwidth exceed shared memory");
    return MATCHA_ERR_UNSUPPORTED;
  }
  if (p->ball_kmax > 0) {
    set_error_text("template gradient: not available with the ball-harmonic radial basis");
    return MATCHA_ERR_UNSUPPORTED;
  }
  if (!p->fp64 && p->LJ > 64) {
    set_error_text("template gradient: the 32-bit gradient recurrences are not rescaled; "
                   "L_J <= 64 (use an FP64 plan above)");
    return MATCHA_ERR_UNSUPPORTED;
  }
  double *shift;
  void *X;
  if (ws_bytes < grad_ws(*p, B, tstride, &shift, &X, nullptr)) return MATCHA_ERR_WORKSPACE;
  grad_ws(*p, B, tstride, &shift, &X, (char *)ws);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e =
      p->fp64 ? launch_template_grad<double>(*p, (const double *)f, (const double *)c, B, tstride,
                                             euler, weight, (double *)X, (double *)coef_grad,
                                             vox_grad, shift, flags, st)
              : launch_template_grad<float>(*p, (const float *)f, (const float *)c, B, tstride,
                                            euler, weight, (float *)X, (float *)coef_grad,
                                            vox_grad, shift, flags, st);
  if (e != cudaSuccess) return fail_cuda(e, "template_grad");
  if (shift_out) CK(cudaMemcpyAsync(shift_out, shift, sizeof(double) * 4 * B, cudaMemcpyDeviceToDevice, st));
  return MATCHA_OK;
}

}  // extern "C"
