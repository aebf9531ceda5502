// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (see include/matcha.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>
#include <vector>
#include "../../include/matcha.h"

namespace matcha {

// Texture views of a batch of volumes for the analysis gathers: 2-D
// pitch-linear views (x, z N + y) of runs of `vpt` consecutive volumes, so
// one 2x2 texture gather fetches the four x-y corners of a trilinear cell in
// one plane.  A texture object only describes the memory (it owns none), so
// a view stays valid for any later allocation at the same address.
constexpr int TEX_MAX = 256;  // views per batch (kernel parameter array)
struct TexSet {
  const void *base = nullptr;
  int B = 0, vpt = 0, ntex = 0;
  unsigned long long used = 0;
  cudaTextureObject_t t[TEX_MAX] = {};
};
struct TexArgs {  // passed by value to the analysis kernel
  cudaTextureObject_t t[TEX_MAX];
  int vpt;
};

// Plan: descriptor, derived sizes and the device tables it owns.
struct Plan {
  matcha_plan_desc desc;
  int N, S, LJ, L0, K, P, M, nlev;
  int Ls[MATCHA_MAX_LEVELS];
  double R, step_tol, accept_tol;
  bool fp64;
  int refine;    // 0 Newton steps, 1 gradient steps
  int tc;        // contraction on the tensor cores: 0 no, 1 TF32, 2 BF16 (FP32 plans)
  int *dev_err;  // device word: bit 0 = a tensor-core wait reached its limit
  int device = -1;                 // the CUDA device current at plan creation
  void *noalloc_grid = nullptr;    // device address of the allocation-free search's array
  // tile choices set by matcha_plan_autotune (0 = the built-in rule); none of
  // them changes any result bit
  int tune_shells = 0;   // shells per analysis CTA (1, 2, 4, 8)
  int tune_tc_ctas = 0;  // tensor-core contraction CTAs per SM (1, 2)
  int tune_soft = 0;     // SOFFT search kernel: 1 the chunked kernels, 2 warp per slice,
                         // 3 register-tiled
  int tune_newton = 0;   // refinement schedule: 1 a CTA per particle, 2 persistent cost-sorted queue
  long wait_limit = -1;  // mbarrier polls before a wait gives up (-1: the built-in limit)
  int nt, np, nlm, npairs, npairs0, ns;
  int ngroups;  // partner groups of the correlation layout, (L_J+1)(L_J+2)/2
  long nc;      // pair slots x degrees per particle (dummy halves included), 4 reals each
  long nc0;     // (pair, l) entries with m <= L0 and l <= L0 (SOFFT layout)
  // device tables (one allocation)
  void *base = nullptr;
  double *rs, *wrad, *xj, *wj;  // S, S, nt, nt (FP64 always)
  void *ptab;                   // real [nt][nlm]: w_j (2 pi / n_phi) Pbar_lm(x_j)
  void *ptab_leg;               // real [nt][nlm]: ptab with its columns in the Legendre item order
  int *leg_lm;                  // [nlm] (l << 16) | m of Legendre item t: m ascending, then the
                                // parity of l + m, then l (runs of equal m and parity)
  void *phi_cs;                 // real [np][2]: cos, sin (2 pi k / n_phi)
  void *soft_tw;                // real [ns][2]: cos, sin (2 pi t / ns)
  void *soft_d;                 // real [ns][nc0]: d^l_mn(beta_k) in the SOFFT layout
  void *rcoef;                  // real, grouped layout: (a, -b, -e) of the step l -> l+1, -l(l+1)
  void *seedK;                  // real [ngroups][4]: (sqrt(binom(2m, m+n)) of both halves, 0, 0)
  void *dft_cs;                 // real [2][2][Qf][Mq]: folded phi-DFT table (parity, cos|sin, q, column)
  int Mp;                       // analysis F row: orders padded to a multiple of 4, plus 1
  int Qf, Mq;                   // folded DFT rows ceil(L_J/2); columns per order parity, padded to 4
  void *ring;                   // real [S * nt][2]: (r_s sin t_j, N/2 + r_s cos t_j) of ring s * nt + j
  void *fft_tw;                 // real [N][2]: cos, sin (-2 pi j / N), the box FFT's twiddles
  // ball-harmonic radial basis (ball_kmax = 0: radial shells)
  double ball_lambda = 0;       // frequency budget Lambda
  int ball_kmax = 0;            // |K_0|, rows of the projection table
  void *ball_W = nullptr;       // real [L_J+1][ball_kmax][S]: w_s N_lk j_l(lambda_lk r_s / R)
  int *ball_K = nullptr;        // [L_J+1] |K_l| (in the same allocation as ball_W)
  int fft_npass = 0;            // radix passes of the length-N FFT (0: N has a factor > 5)
  int fft_radix[16] = {};       // radices (4, 2, 3, 5) in pass order
  int *pair_base;               // [npairs] first real of pair q in the grouped L_J layout
  int *pair_off0;               // [npairs0] entry offset of pair q in the L0 (SOFFT) layout
  // copy stream and events of matcha_align_host (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev[9] = {};
  // extra streams of matcha_align's concurrent parts and their fork / join events
  static constexpr int NSPLIT = 4;
  cudaStream_t split_stream[NSPLIT - 1] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[NSPLIT - 1] = {};
  // texture views of recently analysed batches (most recently used kept)
  static constexpr int NTEXSET = 16;
  mutable TexSet texsets[NTEXSET];
  mutable unsigned long long tex_clock = 0;
  // held from the view lookup through the analysis launch, so that a view
  // another host thread evicts is never one whose launch is still to come
  mutable std::mutex tex_mu;
};
void destroy_texsets(Plan &p);

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Grouped correlation layout.  The order pairs (m, n), m >= |n|, of one m are
// taken two at a time: group g = m(m+1)/2 + j (j = 0..m) holds the partners
// n_a = 2j - m and n_b = n_a + 1 (half 0 and half 1); for j = m the second
// half is empty (n_b = m + 1 does not exist) and holds zeros.  Group g covers
// the degrees l = m..L, and each (group, l) is 8 reals with the two halves
// interleaved: real 2k + h is component k of half h, k = 0..3 being
// (Re, Im) of c^l_{mn} and (Re, Im) of c^l_{nm}.  Interleaving puts the same
// component of both partners side by side, so one paired (2-wide) operation
// advances both.
inline long group_offset_host(int m, int j, int L) {  // in (group, l) entries
  long o = 0;
  for (int mm = 0; mm < m; ++mm) o += (long)(mm + 1) * (L - mm + 1);
  return o + (long)j * (L - m + 1);
}
inline long group_entries_host(int L) { return group_offset_host(L + 1, 0, L); }
// first real of pair (m, n) in the grouped layout of bandwidth L
inline long pair_base_host(int m, int n, int L) {
  int j = (n + m) >> 1, h = (n + m) & 1;
  return 8 * group_offset_host(m, j, L) + h;
}
// Ungrouped layout of the SOFFT kernels' staged copy and of soft_d:
// off(m, n) = sum_{m'<m} (2m'+1)(L-m'+1) + (n+m)(L-m+1) entries.
inline long pair_offset_host(int m, int n, int L) {
  long o = 0;
  for (int mm = 0; mm < m; ++mm) o += (long)(2 * mm + 1) * (L - mm + 1);
  return o + (long)(n + m) * (L - m + 1);
}
inline long pair_entries_host(int L) {  // sum_{m<=L} (2m+1)(L-m+1)
  return pair_offset_host(L + 1, -(L + 1), L);
}

// Table builders (plan_tables.cu).
cudaError_t build_tables(Plan &p, cudaStream_t st);
// The ball-harmonic radial table on the host (ball.cu): W[l][k][s] =
// w_s N_lk j_l(lambda_lk r_s / R) for k < |K_l| (zero-padded to Kmax), the
// counts |K_l|; returns Kmax = |K_0|.
int ball_tables(int L, int S, double R, double Lam, const double *r, const double *w,
                std::vector<double> &W, std::vector<int> &counts);

// Kernel launchers; each returns cudaGetLastError() after its launches.
template <typename T>
cudaError_t launch_analyze(const Plan &p, const float *vols, int B, T *coef, cudaStream_t st);
template <typename T>
cudaError_t launch_correlate(const Plan &p, const T *f, const T *h, int B, int hstride, T *c,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_soft(const Plan &p, const T *c, int B, const int *P_per, T *grid, int *idx,
                        double *euler, double *score, int *n_cand, cudaStream_t st);
template <typename T>
cudaError_t launch_newton(const Plan &p, const T *c, int B, const int *n_cand, double *euler,
                          double *score, int *cflags, long long *work, cudaStream_t st);
template <typename T>
cudaError_t launch_newton_queue(const Plan &p, const T *c, int B, const int *n_cand, double *euler,
                                double *score, int *cflags, long long *work, int *order,
                                int *ticket, cudaStream_t st);
template <typename T>
cudaError_t launch_objective(const Plan &p, const T *c, int B, int L, int Q, const double *pts,
                             double *out, cudaStream_t st);
template <typename T>
cudaError_t launch_template_grad(const Plan &p, const T *f, const T *c, int B, int tstride,
                                 const double *euler, const double *weight, T *X, T *coef_grad,
                                 double *vox_grad, double *shift, int *flags, cudaStream_t st);
cudaError_t launch_correlate_tc(const Plan &p, const float *f, const float *h, int B, int hstride,
                                float *c, cudaStream_t st);
bool correlate_tc_fits(int S, int L, int bytes);
bool backward_fits(const Plan &p);  // the template-gradient kernel's shared memory fits
bool newton_fits(const Plan &p);  // the refinement kernel's shared memory fits
bool analyze_shells_ok(const Plan &p, int G);  // G shells per analysis CTA fit
bool soft_grid_optional(const Plan &p);  // the SOFFT search can skip writing the grid
bool soft_fits(const Plan &p);           // some SOFFT kernel serves the plan
bool soft_warps_ok(const Plan &p);       // the warp-per-slice SOFFT kernel serves the plan
bool soft_tile_ok(const Plan &p);        // the register-tiled SOFFT kernel serves the plan
// Translation search (translate.cu): volume poses, the box FFT, the cross
// spectrum and the windowed inverse DFT of the correlation.
cudaError_t launch_pose_volumes(int N, const float *vol, int B, long vol_stride, const double *R,
                                const double *shift, bool fp64, float *out, cudaStream_t st);
struct ShiftWs {
  void *Z;        // complex [B][N^3] (plan precision): spectra, then the cross spectrum
  void *Y1, *Y2;  // complex [B][nt][N^2], [B][nt][nt][N]
  void *E;        // complex [B][3][N][nt]: the inverse-DFT factors per axis
  void *CC;       // real [B][nt^3]
  double *t0;     // [B][3] integer peak
};
size_t shift_ws_bytes(const Plan &p, int B, int max_shift, int upsample, char *base, ShiftWs *w);
template <typename T>
cudaError_t launch_shift_search(const Plan &p, const float *f, const float *u, int B,
                                int max_shift, int upsample, const double *R, const ShiftWs &w,
                                double *t, double *tau, double *cc, int *flags, cudaStream_t st);
cudaError_t launch_final_select(const Plan &p, int B, const int *P_per, const int *n_cand,
                                const double *cand_euler, const double *cand_score,
                                const int *cand_flags, double *euler, double *R, double *score,
                                int *best_p, int *flags, cudaStream_t st);

// Small device helpers.
template <typename T> struct Cplx { T x, y; };

// Exact division of small non-negative ints by a runtime divisor without the
// emulated integer divide: a float reciprocal estimate, then one correction.
struct FastDiv {
  int d;
  float inv;
  __device__ __forceinline__ explicit FastDiv(int dd) : d(dd), inv(1.0f / (float)dd) {}
  __device__ __forceinline__ int div(int x) const {
    int q = __float2int_rz(((float)x + 0.5f) * inv);
    if (q * d > x) --q;
    else if ((q + 1) * d <= x) ++q;
    return q;
  }
};

__device__ __forceinline__ int isqrt_floor(int q) {
  int m = (int)sqrtf((float)q);
  while (m * m > q) --m;
  while ((m + 1) * (m + 1) <= q) ++m;
  return m;
}

// Largest m with m(m+1)/2 <= g (the order m of partner group g).
__device__ __forceinline__ int tri_floor(int g) {
  int m = (int)((sqrtf(8.0f * (float)g + 1.0f) - 1.0f) * 0.5f);
  while (m * (m + 1) / 2 > g) --m;
  while ((m + 1) * (m + 2) / 2 <= g) ++m;
  return m;
}

}  // namespace matcha
