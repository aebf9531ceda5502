/*
 * Oracle: the whole rotational-alignment path of Algorithm 1 for a batch of
 * independent (particle, template) pairs.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *   analyse f and h on the shells -> c^l_{mn} up to L_J (Appendix A.5)
 *   -> C_{L0} on the SOFFT grid -> the P strongest local maxima (Section 2.3)
 *   -> Newton march over L_sched (L_sched[0] = L0 is the optional refinement
 *      on C_{L0}) -> argmax_p C_{L_J}, ties to the smaller p (Algorithm 1).
 * Output flags: OR of the candidates' march flags, plus bit 3 when fewer than
 * P local maxima exist.  Particles are independent; OpenMP splits the batch.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Algorithm 1 from the correlation coefficients c^l_mn (complex, the
 * oracle's layout, up to L_J): the SOFFT search, the march, the argmax. */
int orc_align_from_c(const orc_params *p, const double *c, int P_this, double *euler, double *R,
                     double *score, int *best_p, int *flags, int *cand_idx, double *cand_euler0,
                     double *cand_euler, double *cand_score, int *n_cand) {
  int n = orc_soft_n(p->L0, p->K);
  double *grid = (double *)malloc(sizeof(double) * (size_t)n * n * n);
  int P = P_this;
  int idx[P > 0 ? P : 1];
  double sc[P > 0 ? P : 1];

  orc_soft_grid(c, p->L0, p->K, grid);
  int nc = orc_local_maxima_topk(grid, n, P, idx, sc);

  int fl = nc < P ? 8 : 0;
  int best = -1;
  double best_score = -INFINITY;
  for (int q = 0; q < nc; ++q) {
    double abg[3];
    orc_soft_angles(n, idx[q], abg);
    if (cand_euler0) memcpy(cand_euler0 + 3 * q, abg, sizeof(abg));
    double s;
    fl |= orc_refine_march(c, p->L_sched, p->n_levels, p->M_iter, p->step_tol, p->accept_tol, p->refine, abg, &s);
    if (cand_idx) cand_idx[q] = idx[q];
    if (cand_euler) memcpy(cand_euler + 3 * q, abg, sizeof(abg));
    if (cand_score) cand_score[q] = s;
    if (s > best_score) { best_score = s; best = q; }
  }
  for (int q = nc; q < P; ++q) {
    if (cand_idx) cand_idx[q] = -1;
    if (cand_score) cand_score[q] = NAN;
  }
  if (best >= 0) {
    double abg[3];
    if (cand_euler) memcpy(abg, cand_euler + 3 * best, sizeof(abg));
    else {
      orc_soft_angles(n, idx[best], abg);
      double s;
      orc_refine_march(c, p->L_sched, p->n_levels, p->M_iter, p->step_tol, p->accept_tol, p->refine, abg, &s);
    }
    memcpy(euler, abg, sizeof(abg));
    orc_euler_to_matrix(abg[0], abg[1], abg[2], R);
  }
  *score = best_score;
  *best_p = best;
  *flags = fl;
  if (n_cand) *n_cand = nc;
  free(grid);
  return 0;
}

/* Algorithm 1 from the SH coefficients of the particle (f) and the template
 * (h), complex [S][lm] at L_J: everything after the analysis. */
int orc_align_coefs_one(const orc_params *p, const double *f, const double *h, int P_this,
                        double *euler, double *R, double *score, int *best_p, int *flags,
                        int *cand_idx, double *cand_euler0, double *cand_euler,
                        double *cand_score, int *n_cand) {
  int LJ = p->L_sched[p->n_levels - 1];
  double *c = (double *)malloc(sizeof(double) * 2 * (size_t)orc_c_size(LJ));
  orc_correlate(f, h, p->S, p->r_max, LJ, c);
  int rc = orc_align_from_c(p, c, P_this, euler, R, score, best_p, flags, cand_idx, cand_euler0,
                            cand_euler, cand_score, n_cand);
  free(c);
  return rc;
}

int orc_align_one(const orc_params *p, const float *particle, const float *tmpl, int P_this,
                  double *euler, double *R, double *score, int *best_p, int *flags,
                  int *cand_idx, double *cand_euler0, double *cand_euler,
                  double *cand_score, int *n_cand) {
  int LJ = p->L_sched[p->n_levels - 1];
  int nlm = orc_lm_size(LJ);
  double *f = (double *)malloc(sizeof(double) * 2 * (size_t)p->S * nlm);
  double *h = (double *)malloc(sizeof(double) * 2 * (size_t)p->S * nlm);
  orc_analyze_volume(particle, p->N, p->S, p->r_max, LJ, f);
  orc_analyze_volume(tmpl, p->N, p->S, p->r_max, LJ, h);
  int rc = orc_align_coefs_one(p, f, h, P_this, euler, R, score, best_p, flags, cand_idx,
                               cand_euler0, cand_euler, cand_score, n_cand);
  free(f); free(h);
  return rc;
}

/* Batch form of orc_align_coefs_one: f complex [B][S][lm]; h one template
 * (h_stride = 0) or one per particle (h_stride in doubles). */
int orc_align_coefs_batch(const orc_params *p, const double *f, const double *h, long h_stride,
                          int B, double *euler, double *score, int *best_p, int *flags,
                          int n_threads) {
  int LJ = p->L_sched[p->n_levels - 1];
  long per = 2L * p->S * orc_lm_size(LJ);
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int b = 0; b < B; ++b) {
    double R[9];
    orc_align_coefs_one(p, f + b * per, h + b * h_stride, p->P, euler + 3 * b, R, score + b,
                        best_p + b, flags + b, NULL, NULL, NULL, NULL, NULL);
  }
  (void)n_threads;
  return 0;
}

int orc_align_batch(const orc_params *p, const float *particles, const float *templates,
                    int B, long template_stride, const int *P_per,
                    double *euler, double *R, double *score, int *best_p, int *flags,
                    int *cand_idx, double *cand_euler0, double *cand_euler,
                    double *cand_score, int *n_cand, int n_threads) {
  long vox = (long)p->N * p->N * p->N;
  int P = p->P;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int b = 0; b < B; ++b) {
    int Pb = P_per ? P_per[b] : P;
    if (Pb > P) Pb = P;
    orc_align_one(p, particles + b * vox, templates + b * template_stride, Pb,
                  euler + 3 * b, R + 9 * b, score + b, best_p + b, flags + b,
                  cand_idx ? cand_idx + (long)b * P : NULL,
                  cand_euler0 ? cand_euler0 + 3L * b * P : NULL,
                  cand_euler ? cand_euler + 3L * b * P : NULL,
                  cand_score ? cand_score + (long)b * P : NULL,
                  n_cand ? n_cand + b : NULL);
  }
  (void)n_threads;
  return 0;
}
