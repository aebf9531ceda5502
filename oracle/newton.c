/*
 * Oracle: frequency-marched Newton refinement (Sections 2.2 and 2.4,
 * Algorithm 1, the loop over bandwidth levels).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper's update is theta <- theta - H^{-1} grad C_L in the wrapped ZYZ
 * chart, at most M_iter steps per level.  Its safeguards and stopping
 * tolerances are not given; the reading used on both sides of the parity
 * check is:
 *   1. evaluate C, grad, H at theta on C_{L_j};
 *   2. if -H is positive definite (Cholesky pivots > 1e-12 ||H||_F) then
 *      delta = -H^{-1} grad, else delta = grad / ||H||_F  (flag bit 1);
 *   3. clamp ||delta||_2 <= pi / (2 (L_j + 1));
 *   4. trial theta' = wrap(theta + delta); accept when C_{L_j}(theta') >=
 *      C_{L_j}(theta) - accept_tol |C_{L_j}(theta)|, else halve delta, at
 *      most twice; when no trial is accepted theta stays (flag bit 2).
 *      accept_tol (1e-11 in double) sits above the rounding level of the
 *      Wigner sums, so steps near convergence, whose change of C is below
 *      that level, are not judged on rounding noise;
 *   5. at most M_iter steps per level; the level ends early for a candidate
 *      once ||delta||_2 (after step 2) is below step_tol, the "parameter
 *      increment below a prescribed tolerance" stop of Section 2.4;
 *   a non-finite C, grad or H stops the march (flag bit 0).
 * wrap: alpha, gamma mod 2 pi; beta < 0 -> (a+pi, -b, g+pi); beta > pi ->
 * (a+pi, 2pi-b, g+pi), since r_z(pi) r_y(b) r_z(pi) = r_y(-b).
 */
#include <math.h>
#include <stddef.h>
#include "oracle.h"

static double mod2pi(double x) {
  double t = 2.0 * M_PI;
  double r = x - t * floor(x / t);
  if (r >= t) r -= t;
  if (r < 0) r += t;
  return r;
}

void orc_wrap(double *abg) {
  double a = abg[0], b = abg[1], g = abg[2];
  if (b < 0) { b = -b; a += M_PI; g += M_PI; }
  else if (b > M_PI) { b = 2.0 * M_PI - b; a += M_PI; g += M_PI; }
  abg[0] = mod2pi(a); abg[1] = b; abg[2] = mod2pi(g);
}

/* Returns flag bits (bit 1 when the gradient fallback was used). */
int orc_newton_direction(const double *g, const double *H, int L, double *delta) {
  double hn = 0.0;
  for (int i = 0; i < 9; ++i) hn += H[i] * H[i];
  hn = sqrt(hn);
  double tol = 1e-12 * hn;
  double A[9];
  for (int i = 0; i < 9; ++i) A[i] = -H[i];
  /* Cholesky A = L L^T */
  double l00 = A[0], l11, l22, L00, L10, L20, L11, L21, L22;
  int ok = l00 > tol;
  if (ok) {
    L00 = sqrt(l00); L10 = A[3] / L00; L20 = A[6] / L00;
    l11 = A[4] - L10 * L10;
    ok = l11 > tol;
    if (ok) {
      L11 = sqrt(l11); L21 = (A[7] - L20 * L10) / L11;
      l22 = A[8] - L20 * L20 - L21 * L21;
      ok = l22 > tol;
      if (ok) L22 = sqrt(l22);
    }
  }
  int flags = 0;
  if (ok) {
    /* A delta = g : forward then back substitution */
    double y0 = g[0] / L00;
    double y1 = (g[1] - L10 * y0) / L11;
    double y2 = (g[2] - L20 * y0 - L21 * y1) / L22;
    double x2 = y2 / L22;
    double x1 = (y1 - L21 * x2) / L11;
    double x0 = (y0 - L10 * x1 - L20 * x2) / L00;
    delta[0] = x0; delta[1] = x1; delta[2] = x2;
  } else {
    flags |= 2;
    for (int i = 0; i < 3; ++i) delta[i] = hn > 0 ? g[i] / hn : 0.0;
  }
  double nrm = sqrt(delta[0] * delta[0] + delta[1] * delta[1] + delta[2] * delta[2]);
  double cap = M_PI / (2.0 * (L + 1.0));
  if (nrm > cap) for (int i = 0; i < 3; ++i) delta[i] *= cap / nrm;
  return flags;
}

/* First-order alternative (Section 5.1 compares Newton refinement with a
 * gradient method): delta = grad / ||H||_F, the gradient step with the
 * inverse of a local curvature bound as step size (||H||_2 <= ||H||_F), then
 * the same clamp.  No flag: this direction is the method, not a fallback. */
int orc_gradient_direction(const double *g, const double *H, int L, double *delta) {
  double hn = 0.0;
  for (int i = 0; i < 9; ++i) hn += H[i] * H[i];
  hn = sqrt(hn);
  for (int i = 0; i < 3; ++i) delta[i] = hn > 0 ? g[i] / hn : 0.0;
  double nrm = sqrt(delta[0] * delta[0] + delta[1] * delta[1] + delta[2] * delta[2]);
  double cap = M_PI / (2.0 * (L + 1.0));
  if (nrm > cap) for (int i = 0; i < 3; ++i) delta[i] *= cap / nrm;
  return 0;
}

static int finite_all(double C, const double *g, const double *H) {
  if (!isfinite(C)) return 0;
  for (int i = 0; i < 3; ++i) if (!isfinite(g[i])) return 0;
  for (int i = 0; i < 9; ++i) if (!isfinite(H[i])) return 0;
  return 1;
}

int orc_newton_march(const double *c, const int *L_sched, int n_levels, int M_iter,
                     double step_tol, double accept_tol, double *abg, double *score) {
  return orc_refine_march(c, L_sched, n_levels, M_iter, step_tol, accept_tol, 0, abg, score);
}

/* Refines abg in place through the schedule; *score = C_{L_J}(abg).
 * method 0: Newton steps, 1: gradient steps (orc_gradient_direction); the
 * step control is the same.  Returns flag bits. */
int orc_refine_march(const double *c, const int *L_sched, int n_levels, int M_iter,
                     double step_tol, double accept_tol, int method, double *abg,
                     double *score) {
  int flags = 0;
  double C = NAN;
  for (int lev = 0; lev < n_levels; ++lev) {
    int L = L_sched[lev];
    for (int t = 0; t < M_iter; ++t) {
      double g[3], H[9], delta[3];
      C = orc_objective(c, L, abg[0], abg[1], abg[2], g, H, NULL);
      if (!finite_all(C, g, H)) { *score = C; return flags | 1; }
      flags |= method == 1 ? orc_gradient_direction(g, H, L, delta)
                           : orc_newton_direction(g, H, L, delta);
      if (sqrt(delta[0] * delta[0] + delta[1] * delta[1] + delta[2] * delta[2]) < step_tol) break;
      int accepted = 0;
      for (int h = 0; h < 3 && !accepted; ++h) {
        double trial[3] = {abg[0] + delta[0], abg[1] + delta[1], abg[2] + delta[2]};
        orc_wrap(trial);
        double Ct = orc_objective(c, L, trial[0], trial[1], trial[2], NULL, NULL, NULL);
        if (Ct >= C - accept_tol * fabs(C)) {
          abg[0] = trial[0]; abg[1] = trial[1]; abg[2] = trial[2];
          C = Ct;
          accepted = 1;
        } else {
          for (int i = 0; i < 3; ++i) delta[i] *= 0.5;
        }
      }
      if (!accepted) flags |= 4;
    }
  }
  *score = C;
  return flags;
}
