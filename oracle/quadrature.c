/*
 * Oracle: quadrature rules and normalised associated Legendre functions.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The correlation of Section 2.1 is an integral over the ball (the inner
 * product of L^2(B_3), Section 2).  The ball is discretised in spherical
 * coordinates: Gauss-Legendre nodes in the radius with the r^2 Jacobian folded
 * into the weights, Gauss-Legendre nodes in cos(theta) and equispaced nodes in
 * phi.  With n_theta = L+1 and n_phi = 2L+2 the angular rule integrates
 * Y_lm conj(Y_l'm') exactly for l, l' <= L.
 */
#include <math.h>
#include "oracle.h"

long orc_c_offset(int l) { return (long)l * (2L * l - 1) * (2L * l + 1) / 3; }
long orc_c_size(int L) { return (long)(L + 1) * (2L * L + 1) * (2L * L + 3) / 3; }
long orc_c_index(int l, int m, int n) {
  return orc_c_offset(l) + (long)(m + l) * (2 * l + 1) + (n + l);
}
int orc_lm_index(int l, int m) { return l * (l + 1) / 2 + m; }
int orc_lm_size(int L) { return (L + 1) * (L + 2) / 2; }

/* Legendre polynomial P_n(x) and P_{n-1}(x) by the three-term recurrence. */
static void legendre_pair(int n, double x, double *pn, double *pn1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1; p1 = p2;
  }
  *pn = p1; *pn1 = p0;
}

/* n-point Gauss-Legendre rule on [-1, 1], nodes ascending. */
void orc_gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn, pn1, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pair(n, z, &pn, &pn1);
      dp = n * (z * pn - pn1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre_pair(n, z, &pn, &pn1);
    dp = n * (z * pn - pn1) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Radial rule on (0, R]: r_s = R (1 + x_s) / 2, weight (R/2) w_s r_s^2. */
void orc_radial_nodes(int S, double R, double *r, double *w) {
  double x[S], wg[S];
  orc_gauss_legendre(S, x, wg);
  for (int s = 0; s < S; ++s) {
    r[s] = 0.5 * R * (1.0 + x[s]);
    w[s] = 0.5 * R * wg[s] * r[s] * r[s];
  }
}

/* Pbar_lm(x) for 0 <= m <= l: Y_lm(t, p) = Pbar_lm(cos t) exp(i m p) is
 * orthonormal on the sphere and carries the Condon-Shortley phase.
 * Seeds Pbar_00 = 1/sqrt(4 pi), Pbar_mm = -sqrt((2m+1)/(2m)) sin(t) Pbar_{m-1,m-1},
 * Pbar_{m+1,m} = sqrt(2m+3) x Pbar_mm, then the standard normalised recurrence
 * in l. */
double orc_plm_bar(int l, int m, double x) {
  double st = sqrt(fmax(0.0, 1.0 - x * x));
  double pmm = 1.0 / sqrt(4.0 * M_PI);
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * st;
  if (l == m) return pmm;
  double p1 = sqrt(2.0 * m + 3.0) * x * pmm;
  if (l == m + 1) return p1;
  double p0 = pmm;
  for (int k = m + 2; k <= l; ++k) {
    double a = sqrt((4.0 * k * k - 1.0) / ((double)k * k - (double)m * m));
    double b = sqrt(((k - 1.0) * (k - 1.0) - (double)m * m) / (4.0 * (k - 1.0) * (k - 1.0) - 1.0));
    double p2 = a * (x * p1 - b * p0);
    p0 = p1; p1 = p2;
  }
  return p1;
}

/* Angular grid for bandwidth L: n_theta = L+1 Gauss-Legendre nodes in cos(theta)
 * (ascending) with weights, n_phi = 2L+2 equispaced phi_k = 2 pi k / n_phi. */
void orc_angular_grid(int L, double *x, double *w, int *n_theta, int *n_phi) {
  *n_theta = L + 1;
  *n_phi = 2 * L + 2;
  orc_gauss_legendre(L + 1, x, w);
}
