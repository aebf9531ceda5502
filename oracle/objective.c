/*
 * Oracle: the bandlimited correlation C_L and its Euler-angle derivatives.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * With (g o h)(x) = h(g^{-1} x) (Section 2) and the rotation rule of the ball
 * harmonics (Appendix A.4), the coefficients of g o h are
 * sum_n D^l_{mn}(g) h_ln, so
 *
 *   C_L(g) = <f, g o h> = sum_{l<=L} sum_{m,n} c^l_{mn} conj(D^l_{mn}(g))
 *          = Re sum c^l_{mn} exp(i(m a + n g)) d^l_{mn}(b)
 *
 * with c^l_{mn} = sum_s w_s f_lm conj(h_ln).  This is Eq. (cc-L) with the
 * conjugate placed on D instead of on sigma, one of the convention choices
 * Appendix A.5 allows; for real f and h the sum is real.  Derivatives
 * (Appendix A.4): d/da brings i m, d/dg brings i n, d/db acts on d^l.
 *
 * grad = (dC/da, dC/db, dC/dg); hess = 3x3 row-major in (a, b, g).
 * Either may be NULL.  imag_part (may be NULL) receives Im of the sum.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

double orc_objective(const double *c, int L, double a, double b, double g,
                     double *grad, double *hess, double *imag_part) {
  long T = orc_c_size(L);
  int want_d = (grad != NULL) || (hess != NULL);
  double *d = (double *)malloc(sizeof(double) * T * (want_d ? 3 : 1));
  double *d1 = want_d ? d + T : NULL, *d2 = want_d ? d + 2 * T : NULL;
  if (want_d) orc_wigner_d_derivs(L, b, d, d1, d2);
  else orc_wigner_d(L, b, d);

  double C = 0.0, Ci = 0.0;
  double ga = 0.0, gb = 0.0, gg = 0.0;
  double haa = 0.0, hab = 0.0, hag = 0.0, hbb = 0.0, hbg = 0.0, hgg = 0.0;
  for (int m = -L; m <= L; ++m)
    for (int n = -L; n <= L; ++n) {
      double ph = m * a + n * g, ep = cos(ph), eq = sin(ph);
      int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
      for (int l = (am > an ? am : an); l <= L; ++l) {
        long i = orc_c_index(l, m, n);
        double cr = c[2 * i], ci = c[2 * i + 1];
        double zr = cr * ep - ci * eq, zi = cr * eq + ci * ep; /* c exp(i ph) */
        C += zr * d[i];
        Ci += zi * d[i];
        if (want_d) {
          ga += -m * zi * d[i];
          gb += zr * d1[i];
          gg += -n * zi * d[i];
          haa += -(double)m * m * zr * d[i];
          hab += -m * zi * d1[i];
          hag += -(double)m * n * zr * d[i];
          hbb += zr * d2[i];
          hbg += -n * zi * d1[i];
          hgg += -(double)n * n * zr * d[i];
        }
      }
    }
  free(d);
  if (grad) { grad[0] = ga; grad[1] = gb; grad[2] = gg; }
  if (hess) {
    hess[0] = haa; hess[1] = hab; hess[2] = hag;
    hess[3] = hab; hess[4] = hbb; hess[5] = hbg;
    hess[6] = hag; hess[7] = hbg; hess[8] = hgg;
  }
  if (imag_part) *imag_part = Ci;
  return C;
}
