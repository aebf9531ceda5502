/*
 * Oracle: the per-degree contraction of Eq. (sigmalmm), Appendix A.5.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *   c^l_{mn} = sum_s w_s f_lm(r_s) conj(h_ln(r_s)),   |m|, |n| <= l <= L,
 *
 * with the radial quadrature weights w_s (r^2 Jacobian included) in place of
 * the ball-harmonic radial index k.  Negative orders of the real volumes come
 * from f_{l,-m} = (-1)^m conj(f_lm).
 */
#include "oracle.h"

static void coef_at(const double *f, int nlm, int s, int l, int m, double *re, double *im) {
  int am = m < 0 ? -m : m;
  long i = 2L * ((long)s * nlm + orc_lm_index(l, am));
  *re = f[i];
  *im = f[i + 1];
  if (m < 0) {
    double sg = (am & 1) ? -1.0 : 1.0;
    *re = sg * *re;
    *im = -sg * *im;
  }
}

void orc_correlate(const double *f, const double *h, int S, double R, int L, double *c) {
  double r[S], w[S];
  orc_radial_nodes(S, R, r, w);
  int nlm = orc_lm_size(L);
  for (int l = 0; l <= L; ++l)
    for (int m = -l; m <= l; ++m)
      for (int n = -l; n <= l; ++n) {
        double re = 0.0, im = 0.0;
        for (int s = 0; s < S; ++s) {
          double fr, fi, hr, hi;
          coef_at(f, nlm, s, l, m, &fr, &fi);
          coef_at(h, nlm, s, l, n, &hr, &hi);
          /* f * conj(h) */
          re += w[s] * (fr * hr + fi * hi);
          im += w[s] * (fi * hr - fr * hi);
        }
        long i = orc_c_index(l, m, n);
        c[2 * i] = re;
        c[2 * i + 1] = im;
      }
}
