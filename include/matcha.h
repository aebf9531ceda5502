/*
 * matcha.h — C ABI of the GB300 (sm_103a) batched rotational-alignment library.
 *
 * The library computes the data-parallel path of Matcha (Kruse, Debarnot,
 * Kishore, Dokmanic, arXiv 2603.15285): for each (particle f, template h)
 * pair it finds g^ = argmax_g C(g), C(g) = <f, g o h>  (Section 2, Eq. maxcc_rot),
 * by Algorithm 1: a SOFFT grid search on the bandlimited correlation C_{L0},
 * the P strongest local maxima as candidates, and Newton steps on C_{L_j} for
 * an increasing bandwidth schedule L_0 < L_1 < ... < L_J.
 *
 * Conventions shared by every entry point:
 *   - all calls that take a `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) are asynchronous on that stream: argument
 *     errors are returned synchronously before anything is enqueued, CUDA
 *     launch errors are returned as MATCHA_ERR_CUDA;
 *   - `*_dev` pointers are device memory owned by the caller; the library never
 *     allocates or frees in those calls (only plan create/destroy do);
 *   - precision: a plan computes either in FP64 throughout (MATCHA_FP64) or
 *     in FP32 with FP64 angles, acceptance tests and final comparisons (MATCHA_FP32);
 *     MATCHA_TF32 and MATCHA_BF16 are FP32 plans whose per-degree contraction
 *     (step a3) runs on the tensor cores (tcgen05) with TF32 or BF16 operands and
 *     FP32 accumulation, for L_J <= 63;
 *     "real" below is double for FP64 plans and float for the others, and a
 *     complex number is two consecutive reals (re, im);
 *   - volumes: float32, C order [z][y][x], N^3 per volume, voxel [k][j][i] at
 *     position (x, y, z) = (i, j, k), rotation centre c0 = N/2, trilinear
 *     interpolation with zero outside the box;
 *   - Euler angles: ZYZ radians, g = r_z(alpha) r_y(beta) r_z(gamma)
 *     (Appendix A.3, Eq. Euler), alpha, gamma in [0, 2pi), beta in [0, pi];
 *     rotation matrices are row-major 3x3 doubles.
 *
 * Layouts:
 *   SH coefficients (matcha_analyze):  [b][s][lm] complex, lm = l(l+1)/2 + m,
 *     0 <= m <= l <= L_J, s < n_shells.  Negative orders of these real volumes
 *     follow from f_{l,-m} = (-1)^m conj(f_{lm}).
 *   correlation coefficients (matcha_correlate_coeffs): per particle, the
 *     order pairs (m, n) with 0 <= m <= L_J and -m <= n <= m, taken two at a
 *     time with equal m: group g = m(m+1)/2 + j (j = 0..m) holds the
 *     partners n_a = 2j - m (slot 0) and n_b = n_a + 1 (slot 1; for j = m
 *     slot 1 is empty and holds zeros).  Group g covers l = m .. L_J; entry
 *     (g, l) is 8 reals starting at real 8 * (goff(m, j) + l - m) with
 *     goff(m, j) = sum_{m' < m} (m'+1)(L_J-m'+1) + j (L_J-m+1), and real
 *     2k + h of it is component k of slot h, k = 0..3 being Re c^l_{mn},
 *     Im c^l_{mn}, Re c^l_{nm}, Im c^l_{nm}.  The partners' equal components
 *     sit side by side so that both advance in one paired operation.
 *     matcha_plan_info() returns corr_entries = 2 * (number of (g, l)
 *     entries), so a particle holds corr_entries * 4 reals.  These pairs and
 *     their images under c^l_{-m,-n} = (-1)^{m+n} conj(c^l_{mn}) give every
 *     coefficient with |m|, |n| <= l <= L_J.
 *   SOFFT grid (workspace): n = 2K(L0+1) points per angle, alpha_i = 2 pi i/n,
 *     beta_k = pi (2k+1)/(2n), gamma_j = 2 pi j/n, linear index (i n + k) n + j.
 */
#ifndef MATCHA_H
#define MATCHA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MATCHA_MAX_LEVELS 16
#define MATCHA_MAX_L 100
#define MATCHA_MAX_P 32

typedef struct matcha_plan_s *matcha_plan;

typedef enum {
  MATCHA_OK = 0,
  MATCHA_ERR_INVALID_ARG = 1, /* bad pointer, size or descriptor field */
  MATCHA_ERR_CUDA = 2,        /* a CUDA call or kernel launch failed */
  MATCHA_ERR_WORKSPACE = 3,   /* workspace smaller than matcha_workspace_size */
  MATCHA_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (matcha_plan_device_status) */
  MATCHA_ERR_UNSUPPORTED = 5  /* valid but not implemented (e.g. a size limit) */
} matcha_status;

typedef enum { MATCHA_FP64 = 0, MATCHA_FP32 = 1, MATCHA_TF32 = 2, MATCHA_BF16 = 3 } matcha_precision;

/* Plan descriptor: the parameters of Algorithm 1 plus the sampling of the ball.
 *   box_n        N, volume edge (4 .. 512)
 *   n_shells     S, Gauss-Legendre radial shells on (0, r_max] (1 .. 128)
 *   r_max        outer shell radius in voxels; <= 0 selects N/2 - 1
 *   L0           SOFFT bandwidth (Section 2.3), 1 .. 32, equal to L_sched[0]
 *   K_oversample SOFFT oversampling K (1 .. 16; grids beyond the fused
 *                kernels go through memory, MATCHA_ERR_UNSUPPORTED when even
 *                that kernel's per-slice tables do not fit)
 *   P_max        candidates kept per particle, 1 .. MATCHA_MAX_P
 *   M_iter       Newton steps per level, 1 .. 32
 *   n_levels     number of bandwidth levels J+1 (L_sched[0] = L0 is the
 *                optional refinement on C_{L0}), 1 .. MATCHA_MAX_LEVELS
 *   L_sched      strictly increasing bandwidths, last = L_J <= MATCHA_MAX_L
 *   precision    matcha_precision
 *   step_tol     Newton early stop (Section 2.4): a level stops for a candidate
 *                once ||delta||_2 < step_tol (radians); <= 0 selects 1e-9 for
 *                FP64 plans and 1e-6 for the 32-bit (FP32, TF32, BF16) plans.
 *   accept_tol   a Newton trial is accepted unless it lowers C_L by more than
 *                accept_tol |C_L|, the rounding level of the Wigner sums;
 *                <= 0 selects 1e-11 (FP64) or 1e-5 (32-bit plans).
 *   refine       0: Newton steps (Section 2.2); 1: gradient steps
 *                delta = grad / ||H||_F with the same clamp and step control,
 *                the first-order method Section 5.1 compares against.
 *   ball_lambda  0: radial shells (c^l_mn = sum_s w_s f_lm(r_s) conj(h_ln(r_s)));
 *                > 0: the ball-harmonic radial basis with the eigenvalue cut
 *                Lambda (Appendix "Ball harmonics expansion and eigenvalue-
 *                based truncation"): radial functions N_lk j_l(lambda_lk r/R),
 *                lambda_lk the zeros of j_l up to Lambda (R = r_max), the
 *                coefficients projected from the shells by the radial rule,
 *                c^l_mn = sum_{k in K_l} f_klm conj(h_kln) (Eq. sigmalmm,
 *                rank <= |K_l|).  Needs 1 <= |K_0| <= n_shells; not with
 *                MATCHA_TF32 / MATCHA_BF16 nor with the template gradient.
 * The angular sampling is n_theta = L_J + 1 Gauss-Legendre nodes in cos(theta)
 * and n_phi = 2 L_J + 2 equispaced phi per shell. */
typedef struct {
  int box_n;
  int n_shells;
  double r_max;
  int L0;
  int K_oversample;
  int P_max;
  int M_iter;
  int n_levels;
  int L_sched[MATCHA_MAX_LEVELS];
  int precision;
  double step_tol;
  double accept_tol;
  int refine;
  double ball_lambda;
} matcha_plan_desc;

/* Sizes derived from a plan. */
typedef struct {
  int n_lm;            /* (L_J+1)(L_J+2)/2 SH coefficients per shell */
  long coeff_count;    /* complex SH coefficients per volume = n_shells * n_lm */
  long corr_entries;   /* (pair slot, l) entries per particle, empty slots included; 2 complex each */
  int n_pairs;         /* (L_J+1)^2 order pairs */
  int soft_n;          /* SOFFT points per angle, 2K(L0+1) */
  int real_bytes;      /* 8 (FP64) or 4 (FP32, TF32, BF16) */
} matcha_plan_info_t;

/* Builds the quadrature, Legendre, twiddle, Wigner-recurrence and SOFFT
 * tables of the plan on the current CUDA device (Appendix A.1-A.5 supply the
 * definitions) and synchronises.  *out receives the plan (NULL on error).
 * Allocates device memory owned by the plan. */
matcha_status matcha_plan_create(const matcha_plan_desc *desc, matcha_plan *out);
/* Frees the plan's tables; NULL is accepted. Synchronises the device. */
matcha_status matcha_plan_destroy(matcha_plan plan);
matcha_status matcha_plan_info(matcha_plan plan, matcha_plan_info_t *info);
/* Reads (synchronously) and clears the plan's device status word: bit 0 is
 * set when a tensor-core kernel's wait for its MMAs reached its iteration
 * limit (that CTA then waits, again bounded, for the MMAs it issued, frees its
 * tensor memory and stops; the output blocks it had not written stay
 * unwritten).  Returns MATCHA_ERR_TIMEOUT when any bit was set, else MATCHA_OK. */
matcha_status matcha_plan_device_status(matcha_plan plan, int *bits);
/* Sets the number of mbarrier polls after which such a wait gives up (-1
 * restores the built-in limit, 2^24 polls).  For tests of the timeout path:
 * with 0 every wait gives up at once. */
matcha_status matcha_plan_set_wait_limit(matcha_plan plan, long polls);

/* Copies one of the plan's FP64 quadrature tables to the host (synchronous):
 * which = 0 radial nodes r_s, 1 radial weights w_s (r^2 Jacobian included),
 * 2 angular nodes cos(theta_j), 3 angular weights w_j.  *count receives the
 * table length; at most `capacity` values are written to host_out (which may
 * be NULL to query the length). */
matcha_status matcha_plan_table(matcha_plan plan, int which, double *host_out, long capacity,
                                long *count);

/* Workspace bytes matcha_align needs for B particles. */
matcha_status matcha_workspace_size(matcha_plan plan, int B, size_t *bytes);

/* a1+a2: shell sampling and SH analysis (Appendix A.1 with radial shells in
 * place of the radial Bessel basis).  vols_dev: B float32 volumes; coeffs_dev:
 * B * coeff_count complex reals, layout above.  Samples are trilinear with
 * zero outside the box.  A batch whose base address and row pitch meet the
 * device's texture alignment rules is read through 2-D texture views of its
 * buffer, created on first use and cached in the plan (up to 16 buffers);
 * replacing a cached view synchronises the device first, and no view is
 * created while `stream` is being captured.  Batches without a view are read
 * with plain loads; the coefficients are bit-identical either way.  The view
 * lookup and the launch that uses it run under a per-plan lock, so host
 * threads sharing a plan take turns there.  The same holds for the analysis
 * inside matcha_align. */
matcha_status matcha_analyze(matcha_plan plan, const float *vols_dev, int B, void *coeffs_dev,
                             void *stream);

/* a3: per-degree contraction, Eq. (sigmalmm):
 *   c^l_{mn} = sum_s w_s f_lm(r_s) conj(h_ln(r_s)).
 * f_dev: B particles' SH coefficients; h_dev: templates' coefficients, with
 * template index b * h_batch_stride (0 = one shared template, 1 = one per
 * particle).  c_dev: B * corr_entries * 2 complex reals. */
matcha_status matcha_correlate_coeffs(matcha_plan plan, const void *f_dev, const void *h_dev,
                                      int B, int h_batch_stride, void *c_dev, void *stream);

/* a4+a5: C_{L0} on the SOFFT grid (Section 2.3, beta transform plus 2-D DFT)
 * and the P strongest local maxima.  P_per_dev (nullable) gives a per-particle
 * P_b <= P_max.  Outputs, [B][P_max] each: idx_dev (linear grid index, -1
 * past n_cand), euler_dev ([B][P_max][3] grid angles), score_dev (grid value);
 * n_cand_dev [B].  grid_dev: B * soft_n^3 reals of scratch. */
matcha_status matcha_soft_search(matcha_plan plan, const void *c_dev, int B, const int *P_per_dev,
                                 void *grid_dev, int *idx_dev, double *euler_dev,
                                 double *score_dev, int *n_cand_dev, void *stream);

/* matcha_soft_search without caller-provided scratch.  The paper has no
 * counterpart: this is a library convenience.  It exists for callers that may
 * not allocate device memory themselves: applications whose device memory is
 * owned by a single allocator (a framework's caching allocator or a pool sized
 * at start-up) and latency-critical loops that cannot afford cudaMalloc and
 * cudaFree, which may synchronise the device.  The caller passes c and the
 * candidate outputs exactly as for matcha_soft_search.  Plans whose SOFFT
 * grid fits the fused on-chip kernels (e.g. L0 = 8, K = 2) need no grid
 * scratch at all and take batches up to 65535, as matcha_soft_search.  Plans
 * whose grid goes through memory (e.g. L0 = 30, K = 2: 124^3 points per
 * particle) keep it in a fixed array of MATCHA_NOALLOC_GRID_BYTES (64 MiB)
 * compiled into the library, which every GPU that loads the library keeps
 * until the process exits; for them B * soft_n^3 * real_bytes must fit in it
 * (8 particles per call in FP32, 4 in FP64 at L0 = 30, K = 2), and larger
 * batches return MATCHA_ERR_UNSUPPORTED with the limit in
 * matcha_last_error().  The call allocates nothing.  For such a plan its
 * first call looks up the array's device address (cudaGetSymbolAddress, with
 * the plan's device current) and keeps it in the plan; make that first call
 * before any stream capture.  All calls on a device share the array: calls
 * that overlap on the GPU (e.g. on different streams) race on it and must be
 * ordered by the caller.  The grid is fully rewritten on each call, so
 * leftover contents of the previous call do not matter. */
#define MATCHA_NOALLOC_GRID_BYTES (64u << 20)
matcha_status matcha_soft_search_noalloc(matcha_plan plan, const void *c_dev, int B,
                                         const int *P_per_dev, int *idx_dev, double *euler_dev,
                                         double *score_dev, int *n_cand_dev, void *stream);

/* a6: frequency-marched Newton refinement of every candidate (Sections
 * 2.2-2.4, Algorithm 1).  euler_dev is read as the start points and
 * overwritten by the refined angles; score_dev receives C_{L_J} at the
 * refined angles; cand_flags_dev [B][P_max] receives bit 0 non-finite value,
 * bit 1 gradient fallback (-H not positive definite), bit 2 a step with no
 * accepted trial.  work_dev (nullable) [B][2] receives, per particle, the
 * number of Wigner recurrence steps (one order pair, one degree, one
 * candidate) taken by evaluations with derivatives and by value-only trial
 * evaluations; it measures the work the march performed.  The 32-bit plans
 * sum C, its gradient and Hessian in FP32 and solve the 3x3 Newton systems of
 * the final level in FP64 (the earlier levels in FP32); angles, acceptance
 * tests and scores are FP64 in every plan. */
matcha_status matcha_newton_march(matcha_plan plan, const void *c_dev, int B,
                                  const int *n_cand_dev, double *euler_dev, double *score_dev,
                                  int *cand_flags_dev, long long *work_dev, void *stream);

/* C_L and its analytic gradient and Hessian in the Euler angles (Section
 * 2.2, Appendix A.4: d/da brings i m, d/dg brings i n, d/db acts on d^l) at
 * Q <= P_max rotations per particle, summed exactly as the refinement sums
 * them (plan precision, per-degree rescaling above L_J = 64 in the 32-bit
 * plans).  euler_dev [B][Q][3]; out_dev [B][Q][10] doubles: C, C_a, C_b,
 * C_g, C_aa, C_ab, C_ag, C_bb, C_bg, C_gg.  0 <= L <= L_J. */
matcha_status matcha_objective(matcha_plan plan, const void *c_dev, int B, int L, int Q,
                               const double *euler_dev, double *out_dev, void *stream);

/* a7: argmax_p C_{L_J} (ties to the smaller p, NaN skipped), Euler -> matrix.
 * flags_dev [B]: OR of the candidates' flags, plus bit 3 when fewer than P_b
 * local maxima existed. */
matcha_status matcha_final_select(matcha_plan plan, int B, const int *P_per_dev,
                                  const int *n_cand_dev, const double *cand_euler_dev,
                                  const double *cand_score_dev, const int *cand_flags_dev,
                                  double *euler_dev, double *R_dev, double *score_dev,
                                  int *best_p_dev, int *flags_dev, void *stream);

/* The whole path (a1..a7) for B pairs: particles_dev B volumes, templates_dev
 * volume b * template_batch_stride (0 or 1).  Outputs euler [B][3], R [B][9],
 * score [B], best_p [B], flags [B].  ws_dev must hold
 * matcha_workspace_size(plan, B) bytes (256-byte aligned).  The call only
 * enqueues kernels on `stream` (no allocation, no synchronisation), so it can
 * be captured into a CUDA graph and replayed with the same buffers; the first
 * call on a plan should be made before capture.  From 256 particles on (for
 * plans whose SOFFT grid stays on chip), the batch runs as up to four
 * concurrent parts, one on `stream` and the others
 * on streams the plan owns (forked from `stream` and joined back into it by
 * events), so the call's work stays ordered on `stream`; calls on one plan
 * from several host threads at once share those streams. */
matcha_status matcha_align(matcha_plan plan, const float *particles_dev, const float *templates_dev,
                           int B, int template_batch_stride, const int *P_per_dev,
                           double *euler_dev, double *R_dev, double *score_dev, int *best_p_dev,
                           int *flags_dev, void *ws_dev, size_t ws_bytes, void *stream);

/* matcha_align on HOST buffers: copies the volumes to the device (into the
 * workspace, which must hold matcha_host_workspace_size bytes), runs the
 * path, copies the results back and synchronises the stream.  The batch is
 * split into up to 8 chunks: chunk i+1 is copied on a copy stream owned by
 * the plan (created on the first call) while chunk i is aligned on `stream`,
 * so host calls on one plan must not run concurrently.  Host buffers may be
 * pageable; pinned buffers give full copy bandwidth and the overlap. */
matcha_status matcha_host_workspace_size(matcha_plan plan, int B, int template_batch_stride,
                                         size_t *bytes);
matcha_status matcha_align_host(matcha_plan plan, const float *particles, const float *templates,
                                int B, int template_batch_stride, double *euler, double *R,
                                double *score, int *best_p, int *flags, void *ws_dev,
                                size_t ws_bytes, void *stream);

/* Autotuning.  Times, on the given batch, the tile choices that leave every
 * result bit unchanged and keeps the fastest in the plan: the shells per
 * analysis CTA (1, 2, 4 or 8, those whose shared memory fits), for TF32 /
 * BF16 plans the tensor-core contraction's CTAs per SM (1 or 2), and for
 * 32-bit plans whose grid fits it the SOFFT search kernel (1: the chunked
 * kernels, 2: one warp per beta slice, 3: the register-tiled chunked kernel,
 * the built-in choice where it applies), and the refinement schedule of
 * matcha_align (1: one CTA per particle, 2: persistent CTAs on a cost-sorted
 * queue, longest processing time first).  P_per_dev (nullable) gives the
 * per-particle candidate counts as for matcha_align.  Uses the matcha_align workspace for
 * its scratch; synchronises `stream` (not graph-capturable: tune first, then
 * capture).  report: the choices and the best time (ms) of each candidate,
 * -1 where a candidate does not apply. */
typedef struct {
  int analyze_shells;
  float analyze_ms[4];     /* candidates 1, 2, 4, 8 shells per CTA */
  int tc_ctas_per_sm;      /* 0 when the plan's contraction runs on the CUDA cores */
  float tc_ms[2];          /* candidates 1, 2 CTAs per SM */
  int soft_kernel;         /* 0 when only one SOFFT kernel serves the plan */
  float soft_ms[3];        /* candidates 1 (chunked), 2 (warp per slice), 3 (register-tiled) */
  int newton_sched;        /* matcha_align's refinement: 1 a CTA per particle in index
                              order, 2 persistent CTAs pulling particles from a queue
                              sorted by decreasing candidate count */
  float newton_ms[2];
} matcha_tune_report;
matcha_status matcha_plan_autotune(matcha_plan plan, const float *particles_dev,
                                   const float *templates_dev, int B, int template_batch_stride,
                                   const int *P_per_dev, void *ws_dev, size_t ws_bytes,
                                   void *stream, matcha_tune_report *report);
/* Sets the plan's tile choices directly (the choice fields of a report:
 * analyze_shells, tc_ctas_per_sm, soft_kernel, newton_sched; 0 restores the
 * built-in rule for that field).  Every choice gives bit-identical results; invalid values
 * return MATCHA_ERR_INVALID_ARG and change nothing. */
matcha_status matcha_plan_set_tiles(matcha_plan plan, const matcha_tune_report *choices);

/* Gradient of the refined scores with respect to the template.
 *
 * Loss Lambda = sum_b w_b C_{L_J}(theta*_b), theta*_b the refined rotation of
 * particle b (Algorithm 1).  The template h enters C through
 * c^l_{mn} = sum_s w_s f_lm(r_s) conj(h_ln(r_s)) (Eq. sigmalmm, Appendix A.5),
 * and theta* moves with h so that grad C stays zero (Section 2.2); by the
 * implicit function theorem
 *   dLambda_b/dh = dC/dh - (grad C)^T H^{-1} d(grad C)/dh   at theta*_b,
 * the second term through the analytic Hessian H.  Wigner d and its
 * derivative are recomputed by the l-recurrence; nothing is kept from the
 * forward pass but its outputs.
 *
 * Inputs (device, plan precision unless stated):
 *   f_dev      particles' SH coefficients [B][S][n_lm][2] (matcha_analyze);
 *   c_dev      correlation coefficients [B][corr_entries][4]
 *              (matcha_correlate_coeffs with the same template);
 *   euler_dev  double [B][3]: the refined rotations (matcha_final_select);
 *   weight_dev double [B]: w_b (the upstream gradient), NULL = all ones;
 *   template_batch_stride 0: one template shared by all particles (the
 *              gradients are summed over b); 1: one template per particle.
 * Outputs (device; n_t = 1 for a shared template, B otherwise):
 *   coef_grad_dev  [n_t][S][n_lm][2], plan precision: dLambda/dRe h_ln(r_s)
 *              and dLambda/dIm h_ln(r_s) of the stored coefficients
 *              (0 <= n <= l), each collecting the terms of its mirror
 *              h_{l,-n} = (-1)^n conj(h_ln);
 *   vox_grad_dev   double [n_t][N][N][N] (C order [z][y][x]): dLambda/dvoxel
 *              through the shell analysis and trilinear sampling; NULL skips
 *              it.  Overwritten (zeroed first); sums by atomic adds, so the
 *              last bits may vary between runs;
 *   shift_dev  double [B][4] or NULL: (v, C) with v = H^{-1} grad C at theta*
 *              and C = C_{L_J}(theta*);
 *   flags_dev  int [B] or NULL: 16 when H is singular at theta* (no isolated
 *              maximum; the implicit term is dropped for that particle), else 0.
 * ws_dev: matcha_template_grad_workspace_size bytes, 256-byte aligned.
 * Asynchronous on `stream`.  MATCHA_ERR_UNSUPPORTED when the per-degree
 * tables do not fit in shared memory (FP64 above L_J = 58). */
matcha_status matcha_template_grad_workspace_size(matcha_plan plan, int B,
                                                  int template_batch_stride, size_t *bytes);
matcha_status matcha_template_grad(matcha_plan plan, const void *f_dev, const void *c_dev, int B,
                                   int template_batch_stride, const double *euler_dev,
                                   const double *weight_dev, void *coef_grad_dev,
                                   double *vox_grad_dev, double *shift_dev, int *flags_dev,
                                   void *ws_dev, size_t ws_bytes, void *stream);

/* 6-D pose: rotation and translation (the appendix "Alternating search over
 * rotations and translations"; T = 3 alternations in Section 5.2).
 *
 * The objective is C(tau, g) = <f, g o S_tau h>, (S_tau h)(x) = h(x - tau).
 * At a fixed g it is the cross-correlation CC(t) = sum_x f(x) u(x - t) of f
 * and the rotated template u = g o h at t = g tau (so tau = R^T t).  CC is
 * the circular correlation a 3-D FFT computes (indices mod N); it is
 * searched on the integer window t in [-max_shift, max_shift]^3, then
 * refined on a grid of 2 floor(0.75 upsample) + 1 points per axis at spacing
 * 1/upsample around the integer peak, where CC is the trigonometric
 * interpolant N^-3 Re sum_k X(k) e^{2 pi i k.t/N}, X = F conj(U), k in
 * [-N/2, N/2)^3 (the upsampled DFT the paper cites for sub-voxel accuracy).
 * Grid maxima: ties to the smaller [z][y][x] index.  Vectors t, tau are
 * (x, y, z) in voxels.  The box edge N must factor into 2, 3 and 5
 * (MATCHA_ERR_UNSUPPORTED otherwise); 0 <= max_shift <= 64 with
 * 2 max_shift + 1 <= N, 1 <= upsample <= 64.  Plan precision: FP64 plans run
 * the FFT and the correlation in FP64, the 32-bit plans in FP32.
 *
 * matcha_transform_volumes: out_b(x) = vol(R_b^T (x - c0) + c0 - shift_b),
 *   trilinear, zero outside, for B volumes (vol_stride 0: one shared input
 *   volume, 1: one per output); R_dev [B][9] row-major and shift_dev [B][3]
 *   are nullable (identity, zero).  precision MATCHA_FP64 interpolates in
 *   FP64, the others in FP32.  With R = I this is the translation S_shift,
 *   with shift = 0 the rotation g o vol about c0. */
matcha_status matcha_transform_volumes(int N, const float *vols_dev, int B, int vol_stride,
                                       const double *R_dev, const double *shift_dev, int precision,
                                       float *out_dev, void *stream);
/* matcha_shift_search: the translation search of particle b against the
 * already rotated template rotated_dev[b] (B volumes each).  Outputs t_dev
 * [B][3], cc_dev [B] (CC at t), flags_dev [B] (set to 32 when the integer
 * peak lies on the window's edge, i.e. the true shift may lie beyond it);
 * with R_dev [B][9] given, tau_dev [B][3] = R^T t (both nullable together).
 * ws_dev: matcha_shift_search_workspace_size bytes, 256-byte aligned. */
matcha_status matcha_shift_search_workspace_size(matcha_plan plan, int B, int max_shift,
                                                 int upsample, size_t *bytes);
matcha_status matcha_shift_search(matcha_plan plan, const float *particles_dev,
                                  const float *rotated_dev, int B, int max_shift, int upsample,
                                  const double *R_dev, double *t_dev, double *tau_dev,
                                  double *cc_dev, int *flags_dev, void *ws_dev, size_t ws_bytes,
                                  void *stream);
/* matcha_align6d: `rounds` alternations starting from tau = 0; round r runs
 * matcha_align on (f, S_tau h) (the template itself in round 0), then
 * matcha_shift_search on u = g o h and sets tau = R^T t.  Outputs the last
 * round's euler [B][3], R [B][9], score [B] (C_{L_J} of the rotation step),
 * tau [B][3], t [B][3], cc [B] and flags [B] (matcha_align's bits, plus 32
 * from the last translation search).  ws_dev: matcha_align6d_workspace_size
 * bytes (it contains matcha_align's workspace), 256-byte aligned.  Only
 * enqueues work on `stream`. */
matcha_status matcha_align6d_workspace_size(matcha_plan plan, int B, int template_batch_stride,
                                            int max_shift, int upsample, size_t *bytes);
matcha_status matcha_align6d(matcha_plan plan, const float *particles_dev,
                             const float *templates_dev, int B, int template_batch_stride,
                             int rounds, int max_shift, int upsample, double *euler_dev,
                             double *R_dev, double *tau_dev, double *t_dev, double *score_dev,
                             double *cc_dev, int *flags_dev, void *ws_dev, size_t ws_bytes,
                             void *stream);

const char *matcha_status_string(matcha_status s);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char *matcha_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MATCHA_H */
