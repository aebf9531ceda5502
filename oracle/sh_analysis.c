/*
 * Oracle: spherical-harmonic analysis and synthesis on one shell.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The angular part of the ball-harmonic expansion (Appendix A.1): on shell s,
 *   f_lm(r_s) = sum_j sum_k  w_j (2 pi / n_phi) f(r_s w_jk) conj(Y_lm(t_j, p_k)),
 * written here as the plain double sum over the quadrature points.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

void orc_sh_analyze_shell(const double *samples, int L, double *coef) {
  int nt, np;
  double x[L + 1], w[L + 1];
  orc_angular_grid(L, x, w, &nt, &np);
  for (int l = 0; l <= L; ++l)
    for (int m = 0; m <= l; ++m) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < nt; ++j) {
        double p = orc_plm_bar(l, m, x[j]);
        for (int k = 0; k < np; ++k) {
          double ph = 2.0 * M_PI * k / np;
          double wt = w[j] * (2.0 * M_PI / np) * samples[(long)j * np + k] * p;
          /* conj(Y_lm) = Pbar_lm exp(-i m phi) */
          re += wt * cos(m * ph);
          im -= wt * sin(m * ph);
        }
      }
      coef[2 * orc_lm_index(l, m)] = re;
      coef[2 * orc_lm_index(l, m) + 1] = im;
    }
}

/* u(t, p) = sum_{l<=L} sum_{|m|<=l} a_lm Y_lm(t, p) for a real function, whose
 * negative orders follow from a_{l,-m} = (-1)^m conj(a_lm):
 * u = sum_l [ Re(a_l0 Y_l0) + 2 Re sum_{m>0} a_lm Y_lm ].  out[0] = u. */
void orc_sh_synthesize(const double *coef, int L, double theta, double phi, double *out) {
  double x = cos(theta), u = 0.0;
  for (int l = 0; l <= L; ++l)
    for (int m = 0; m <= l; ++m) {
      double p = orc_plm_bar(l, m, x);
      double re = coef[2 * orc_lm_index(l, m)], im = coef[2 * orc_lm_index(l, m) + 1];
      double t = p * (re * cos(m * phi) - im * sin(m * phi));
      u += (m == 0) ? t : 2.0 * t;
    }
  out[0] = u;
}

/* coef[s][lm] for all S shells of one volume. */
void orc_analyze_volume(const float *vol, int N, int S, double R, int L, double *coef) {
  int nt = L + 1, np = 2 * L + 2, nlm = orc_lm_size(L);
  double *smp = (double *)malloc(sizeof(double) * (size_t)S * nt * np);
  orc_sample_shells(vol, N, S, R, L, smp);
  /* shells are independent; inside an already parallel batch this runs on
     the calling thread (no nested parallelism) */
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < S; ++s)
    orc_sh_analyze_shell(smp + (long)s * nt * np, L, coef + 2L * s * nlm);
  free(smp);
}
