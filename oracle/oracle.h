/*
 * FP64 CPU oracle for Matcha's rotational-alignment path (arXiv 2603.15285).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this code: only the test-suite, the smoke check and the bench's
 * CPU-baseline leg use it.  It shares no source, header, table or helper with
 * the CUDA library; it is written from the paper's definitions, plainly and
 * slowly, in double precision throughout (long double for the cross-check of
 * the Wigner finite sum).
 *
 * Conventions (all fixed by the paper, Section 2 and Appendix A):
 *   - volumes: float32, C order [z][y][x], voxel [k][j][i] at (x,y,z)=(i,j,k),
 *     centre c0 = N/2, trilinear interpolation, zero outside the box;
 *   - Euler angles: ZYZ, g = r_z(alpha) r_y(beta) r_z(gamma)  (Eq. Euler);
 *   - Wigner D: D^l_{mn}(a,b,g) = exp(-i m a) d^l_{mn}(b) exp(-i n g)
 *     (Eq. wigner-D), d^l_{mn}(b) = <l m| exp(-i b J_y) |l n>;
 *   - spherical harmonics Y_lm = Pbar_lm(cos t) exp(i m p), orthonormal on
 *     the sphere, Condon-Shortley phase included;
 *   - complex numbers are stored as interleaved (re, im) doubles.
 *
 * Array layouts:
 *   SH coefficients  f[s][lm],  lm = l(l+1)/2 + m,  0 <= m <= l <= L
 *   correlation      c[off(l) + (m+l)(2l+1) + (n+l)],  off(l) = l(2l-1)(2l+1)/3
 *   Wigner d         same index as c (real)
 *   SOFFT grid       g[(i*n + k)*n + j]  for (alpha_i, beta_k, gamma_j)
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#ifndef MATCHA_ORACLE_H
#define MATCHA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- index helpers ---------------------------------------------------- */
long orc_c_offset(int l);                 /* l(2l-1)(2l+1)/3 = sum_{l'<l} (2l'+1)^2 */
long orc_c_size(int L);                   /* (L+1)(2L+1)(2L+3)/3 */
long orc_c_index(int l, int m, int n);
int  orc_lm_index(int l, int m);          /* l(l+1)/2 + m */
int  orc_lm_size(int L);                  /* (L+1)(L+2)/2 */

/* ---- quadrature (quadrature.c) ----------------------------------------- */
void   orc_gauss_legendre(int n, double *x, double *w);
void   orc_radial_nodes(int S, double R, double *r, double *w);
double orc_plm_bar(int l, int m, double x);
void   orc_angular_grid(int L, double *x, double *w, int *n_theta, int *n_phi);

/* ---- sampling and SH analysis (sampling.c, sh_analysis.c) ------------- */
double orc_trilinear(const float *vol, int N, double px, double py, double pz);
void   orc_sample_shells(const float *vol, int N, int S, double R, int L, double *samples);
void   orc_sh_analyze_shell(const double *samples, int L, double *coef);
void   orc_sh_synthesize(const double *coef, int L, double theta, double phi, double *out);
void   orc_analyze_volume(const float *vol, int N, int S, double R, int L, double *coef);
void   orc_transform_volume(const float *vol, int N, const double *R, const double *s, float *out);

/* ---- contraction (contraction.c) --------------------------------------- */
void orc_correlate(const double *f, const double *h, int S, double R, int L, double *c);

/* ---- Wigner d (wigner.c) ----------------------------------------------- */
void   orc_wigner_d(int L, double beta, double *d);
double orc_wigner_d_finite_sum(int l, int m, int n, double beta);
void   orc_wigner_d_derivs(int L, double beta, double *d, double *d1, double *d2);
void   orc_euler_to_matrix(double a, double b, double g, double *R);
void   orc_matrix_to_euler(const double *R, double *abg);
double orc_rotation_angle(const double *R1, const double *R2);

/* ---- objective (objective.c) -------------------------------------------- */
double orc_objective(const double *c, int L, double a, double b, double g,
                     double *grad, double *hess, double *imag_part);

/* ---- SOFFT grid and candidates (soft.c) -------------------------------- */
int  orc_soft_n(int L0, int K);
void orc_soft_grid(const double *c, int L0, int K, double *grid);
void orc_soft_angles(int n, long idx, double *abg);
int  orc_local_maxima_topk(const double *grid, int n, int P, int *idx, double *score);

/* ---- Newton march (newton.c) ------------------------------------------- */
void orc_wrap(double *abg);
int  orc_newton_direction(const double *g, const double *H, int L, double *delta);
int  orc_newton_march(const double *c, const int *L_sched, int n_levels, int M_iter,
                      double step_tol, double accept_tol, double *abg, double *score);
int  orc_gradient_direction(const double *g, const double *H, int L, double *delta);
int  orc_refine_march(const double *c, const int *L_sched, int n_levels, int M_iter,
                      double step_tol, double accept_tol, int method, double *abg,
                      double *score);

/* ---- full path (align.c) ------------------------------------------------ */
typedef struct {
  int N, S, L0, K, P, M_iter, n_levels;
  int L_sched[16];
  double r_max;
  double step_tol;
  double accept_tol;
  int refine;               /* 0 Newton steps, 1 gradient steps */
} orc_params;

int orc_align_one(const orc_params *p, const float *particle, const float *tmpl, int P_this,
                  double *euler, double *R, double *score, int *best_p, int *flags,
                  int *cand_idx, double *cand_euler0, double *cand_euler,
                  double *cand_score, int *n_cand);
int orc_align_batch(const orc_params *p, const float *particles, const float *templates,
                    int B, long template_stride, const int *P_per,
                    double *euler, double *R, double *score, int *best_p, int *flags,
                    int *cand_idx, double *cand_euler0, double *cand_euler,
                    double *cand_score, int *n_cand, int n_threads);
int orc_align_from_c(const orc_params *p, const double *c, int P_this, double *euler, double *R,
                     double *score, int *best_p, int *flags, int *cand_idx, double *cand_euler0,
                     double *cand_euler, double *cand_score, int *n_cand);
int orc_align_coefs_one(const orc_params *p, const double *f, const double *h, int P_this,
                        double *euler, double *R, double *score, int *best_p, int *flags,
                        int *cand_idx, double *cand_euler0, double *cand_euler,
                        double *cand_score, int *n_cand);
int orc_align_coefs_batch(const orc_params *p, const double *f, const double *h, long h_stride,
                          int B, double *euler, double *score, int *best_p, int *flags,
                          int n_threads);
int orc_max_threads(void);

/* ---- template gradient of the refined score (adjoint.c) ---------------- */
int  orc_implicit_shift(const double *grad, const double *H, double *v);
void orc_coef_grad(const double *f, int S, double R, int L, const double *abg, const double *v,
                   double wt, double *G);
void orc_analysis_adjoint(const double *G, int N, int S, double R, int L, double *vox);
int  orc_template_grad_one(const orc_params *p, const double *f, const double *h,
                           const double *abg, double wt, double *G, double *out4);
int  orc_template_grad_batch(const orc_params *p, const double *f, const double *h, long h_stride,
                             int B, const double *euler, const double *wt, double *G,
                             double *out4, int *flags, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
