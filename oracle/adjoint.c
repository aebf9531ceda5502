/*
 * Oracle: gradient of the refined alignment score with respect to the
 * template, through its SH coefficients down to its voxels.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Loss of one particle: Lambda = C_L(theta*), theta* the refined maximiser of
 * C_L (Algorithm 1; Newton on the analytic gradient and Hessian, Section 2.2).
 * The template h enters through c^l_{mn} = sum_s w_s f_lm conj(h_ln)
 * (Eq. sigmalmm), and theta* moves with h so that grad_theta C stays zero.
 * By the implicit function theorem, d(theta*) / dh = -H^{-1} d(grad C) / dh, so
 *
 *   dLambda/dh = dC/dh - (grad C)^T H^{-1} d(grad C)/dh          (at theta*)
 *              = d/dh Re sum_{l,m,n} c^l_{mn} E'^l_{mn}          (v fixed)
 *   E'^l_{mn}  = E^l_{mn} - sum_k v_k dE^l_{mn}/dtheta_k,  v = H^{-1} grad C,
 *   E^l_{mn}   = exp(i(m a + n g)) d^l_{mn}(b)                   (Eq. wigner-D)
 *
 * (d/da brings i m, d/dg brings i n, d/db acts on d^l; Appendix A.4).
 *
 * Complex gradients are written as dLambda/dRe z + i dLambda/dIm z.  The
 * template's stored coefficients are h_ln(r_s), 0 <= n <= l; its negative
 * orders are h_{l,-n} = (-1)^n conj(h_ln), so the gradient of a stored
 * coefficient collects both the n and the -n terms of the sum.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

/* v = H^{-1} grad by Gaussian elimination with partial pivoting (H 3x3
 * row-major).  Returns 1 and v = 0 when a pivot falls below 1e-14 ||H||_F
 * (no isolated maximum: the implicit term is undefined), else 0. */
int orc_implicit_shift(const double *grad, const double *H, double *v) {
  double A[3][4], nf = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      A[i][j] = H[3 * i + j];
      nf += H[3 * i + j] * H[3 * i + j];
    }
    A[i][3] = grad[i];
  }
  nf = sqrt(nf);
  for (int k = 0; k < 3; ++k) {
    int piv = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
    if (!(fabs(A[piv][k]) > 1e-14 * nf)) {
      v[0] = v[1] = v[2] = 0.0;
      return 1;
    }
    if (piv != k)
      for (int j = 0; j < 4; ++j) {
        double t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t;
      }
    for (int i = k + 1; i < 3; ++i) {
      double f = A[i][k] / A[k][k];
      for (int j = k; j < 4; ++j) A[i][j] -= f * A[k][j];
    }
  }
  for (int k = 2; k >= 0; --k) {
    double s = A[k][3];
    for (int j = k + 1; j < 3; ++j) s -= A[k][j] * v[j];
    v[k] = s / A[k][k];
  }
  return 0;
}

/* f_lm(r_s) for any -l <= m <= l from the stored m >= 0 (real volume). */
static void coef_signed(const double *f, int nlm, int s, int l, int m, double *re, double *im) {
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

/* G[s][ln] += wt * dLambda/dh_ln(r_s) for one particle with coefficients f
 * (complex [S][lm]) at the refined rotation abg and implicit shift v (NULL:
 * v = 0, the partial derivative at fixed theta).
 *
 * For every n in [-l, l]:  X_ln(s) = w_s sum_{m=-l..l} f_lm(r_s) E'^l_{mn}
 * (c is linear in conj(h_ln) with coefficient w_s f_lm, and Re(conj(h) X) has
 * gradient X).  The stored coefficient h_ln, n >= 0, also drives
 * h_{l,-n} = (-1)^n conj(h_ln), whose contribution to its gradient is
 * (-1)^n conj(X_{l,-n}); for n = 0 there is only the one term. */
void orc_coef_grad(const double *f, int S, double R, int L, const double *abg, const double *v,
                   double wt, double *G) {
  double r[S], w[S];
  orc_radial_nodes(S, R, r, w);
  int nlm = orc_lm_size(L);
  long T = orc_c_size(L);
  double *d = (double *)malloc(sizeof(double) * 3 * T);
  double *d1 = d + T, *d2 = d + 2 * T;
  orc_wigner_d_derivs(L, abg[1], d, d1, d2);
  double va = v ? v[0] : 0.0, vb = v ? v[1] : 0.0, vg = v ? v[2] : 0.0;
  double *Xr = (double *)malloc(sizeof(double) * 2 * (2 * L + 1));
  double *Xi = Xr + (2 * L + 1);
  for (int s = 0; s < S; ++s)
    for (int l = 0; l <= L; ++l) {
      for (int n = -l; n <= l; ++n) {
        double xr = 0.0, xi = 0.0;
        for (int m = -l; m <= l; ++m) {
          long i = orc_c_index(l, m, n);
          double ph = m * abg[0] + n * abg[2], cp = cos(ph), sp = sin(ph);
          /* E' = exp(i ph) [ d (1 - i (m va + n vg)) - vb d' ] */
          double br = d[i] - vb * d1[i], bi = -(m * va + n * vg) * d[i];
          double er = cp * br - sp * bi, ei = cp * bi + sp * br;
          double fr, fi;
          coef_signed(f, nlm, s, l, m, &fr, &fi);
          xr += fr * er - fi * ei;
          xi += fr * ei + fi * er;
        }
        Xr[n + l] = w[s] * xr;
        Xi[n + l] = w[s] * xi;
      }
      for (int n = 0; n <= l; ++n) {
        double gr = Xr[n + l], gi = Xi[n + l];
        if (n > 0) {
          double sg = (n & 1) ? -1.0 : 1.0;
          gr += sg * Xr[l - n];
          gi -= sg * Xi[l - n];
        }
        long o = 2L * ((long)s * nlm + orc_lm_index(l, n));
        G[o] += wt * gr;
        G[o + 1] += wt * gi;
      }
    }
  free(Xr);
  free(d);
}

/* vox[z][y][x] += dLambda/dvoxel for the coefficient gradient G (complex
 * [S][lm]): the transpose of orc_analyze_volume.  Coefficient h_lm(r_s) is
 * sum_{j,k} w_j (2 pi/n_phi) Pbar_lm(x_j) exp(-i m p_k) u(s,j,k) over the
 * samples u, each a trilinear combination of eight voxels (zero outside the
 * box); a real input x feeding z = a x has dLambda/dx = Re(conj(G_z) a). */
void orc_analysis_adjoint(const double *G, int N, int S, double R, int L, double *vox) {
  double r[S], wr[S], x[L + 1], wx[L + 1];
  int nt, np;
  orc_radial_nodes(S, R, r, wr);
  orc_angular_grid(L, x, wx, &nt, &np);
  int nlm = orc_lm_size(L);
  double c0 = 0.5 * N;
  double *pb = (double *)malloc(sizeof(double) * nlm);
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < nt; ++j) {
      double st = sqrt(1.0 - x[j] * x[j]);
      for (int l = 0; l <= L; ++l)
        for (int m = 0; m <= l; ++m) pb[orc_lm_index(l, m)] = orc_plm_bar(l, m, x[j]);
      for (int k = 0; k < np; ++k) {
        double ph = 2.0 * M_PI * k / np;
        double du = 0.0;
        for (int l = 0; l <= L; ++l)
          for (int m = 0; m <= l; ++m) {
            long o = 2L * ((long)s * nlm + orc_lm_index(l, m));
            double a = wx[j] * (2.0 * M_PI / np) * pb[orc_lm_index(l, m)];
            /* a exp(-i m p): Re(conj(G) a e) = a (Gr cos mp - Gi sin mp) */
            du += a * (G[o] * cos(m * ph) - G[o + 1] * sin(m * ph));
          }
        double px = c0 + r[s] * st * cos(ph);
        double py = c0 + r[s] * st * sin(ph);
        double pz = c0 + r[s] * x[j];
        double fx0 = floor(px), fy0 = floor(py), fz0 = floor(pz);
        long i0 = (long)fx0, j0 = (long)fy0, k0 = (long)fz0;
        double tx = px - fx0, ty = py - fy0, tz = pz - fz0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              long ii = i0 + dx, jj = j0 + dy, kk = k0 + dz;
              if (ii < 0 || jj < 0 || kk < 0 || ii >= N || jj >= N || kk >= N) continue;
              double wgt = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
              vox[(kk * N + jj) * N + ii] += wgt * du;
            }
      }
    }
  free(pb);
}

/* One particle: c from (f, h), then C, grad, Hessian at abg on C_{L_J}, the
 * implicit shift v, and G += wt dLambda/dh.  out4 (may be NULL) receives
 * (v, C).  Returns 1 when the Hessian is singular (v = 0 used), else 0. */
int orc_template_grad_one(const orc_params *p, const double *f, const double *h,
                          const double *abg, double wt, double *G, double *out4) {
  int LJ = p->L_sched[p->n_levels - 1];
  double *c = (double *)malloc(sizeof(double) * 2 * (size_t)orc_c_size(LJ));
  orc_correlate(f, h, p->S, p->r_max, LJ, c);
  double grad[3], H[9], v[3];
  double C = orc_objective(c, LJ, abg[0], abg[1], abg[2], grad, H, NULL);
  int fl = orc_implicit_shift(grad, H, v);
  orc_coef_grad(f, p->S, p->r_max, LJ, abg, v, wt, G);
  if (out4) { out4[0] = v[0]; out4[1] = v[1]; out4[2] = v[2]; out4[3] = C; }
  free(c);
  return fl;
}

/* Batch of particles: G_b = wt_b dLambda_b/dh for each b (complex
 * [B][S][lm]); h holds one template's coefficients (h_stride = 0) or one
 * per particle (h_stride in doubles).  out4 [B][4] may be NULL. */
int orc_template_grad_batch(const orc_params *p, const double *f, const double *h, long h_stride,
                            int B, const double *euler, const double *wt, double *G,
                            double *out4, int *flags, int n_threads) {
  int LJ = p->L_sched[p->n_levels - 1];
  long per = 2L * p->S * orc_lm_size(LJ);
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int b = 0; b < B; ++b) {
    memset(G + b * per, 0, sizeof(double) * per);
    int fl = orc_template_grad_one(p, f + b * per, h + b * h_stride, euler + 3 * b,
                                   wt ? wt[b] : 1.0, G + b * per, out4 ? out4 + 4 * b : NULL);
    if (flags) flags[b] = fl;
  }
  (void)n_threads;
  return 0;
}
