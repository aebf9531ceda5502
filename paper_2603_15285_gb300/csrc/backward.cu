// Gradient of the refined alignment score with respect to the template.
//
// Loss Lambda = sum_b w_b C_{L_J}(theta*_b): the refined score of each
// particle (Algorithm 1), weighted by the caller's w_b (the upstream
// gradient).  The template enters through c^l_{mn} = sum_s w_s f_lm
// conj(h_ln) (Eq. sigmalmm); the refined rotation theta* moves with it so
// that grad C stays zero, and the implicit function theorem turns that into
// a shift of the evaluation point (Section 2.2 gives grad and Hessian):
//
//   dLambda_b/dh = d/dh Re sum c^l_{mn} E'^l_{mn},   v = H^{-1} grad C (held fixed),
//   E'^l_{mn} = exp(i(m a + n g)) [ d^l_{mn}(b) (1 - i(m v_a + n v_g)) - v_b d'^l_{mn}(b) ].
//
// Four kernels, Wigner d recomputed by the l-recurrence (nothing stored
// from the forward pass):
//   k_bwd_point  one CTA per particle: C, grad, Hessian at theta* from c, and
//                v = H^{-1} grad (FP64 solve);
//   k_bwd_coef   one CTA per particle: per degree l, E'^l (rows m = -l..l,
//                columns n = 0..l) into shared memory, then
//                X_ln(s) = w_b w_s sum_m f_lm(r_s) E'^l_{mn}, doubled for
//                n > 0 (the stored h_ln also drives h_{l,-n} = (-1)^n
//                conj(h_ln), and that term equals X_ln);
//   k_bwd_reduce sums X over the particles that share one template;
//   k_bwd_synth  one CTA per (template, shell): the transpose of the shell
//                analysis (Legendre sum, then the phi series at the
//                samples) and of the trilinear sampling (FP64 atomic adds
//                into the voxel gradient), on the forward pass's own
//                sample coordinates.
#include <math.h>
#include "internal.cuh"

namespace matcha {
namespace {

constexpr int BWD_THREADS = 256;

// first (group, l) entry of group (m, j) in the grouped layout:
// sum_{m' < m} (m'+1)(L-m'+1) + j (L-m+1)
__device__ __forceinline__ long goff_dev(int m, int j, int L) {
  const long t = (long)m * (m + 1) / 2;
  return (long)(L + 2) * t - (long)m * (m + 1) * (2 * m + 1) / 6 + (long)j * (L - m + 1);
}

// x^k, and 0 for k < 0 (those terms carry a zero integer factor)
template <typename T> __device__ __forceinline__ T pw(T x, int k) {
  if (k < 0) return T(0);
  T r = T(1);
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

// d^m_{mn}(b) and its first two b-derivatives at the seed degree l = m:
// sigma K ch^a sh^c with a = m + n, c = m - n, sigma = (-1)^c, ch = cos(b/2),
// sh = sin(b/2); d/db (ch^a sh^c) = (c ch^{a+1} sh^{c-1} - a ch^{a-1} sh^{c+1}) / 2.
template <typename T>
__device__ __forceinline__ void seed3(int m, int n, T K, T ch, T sh, T &d, T &d1, T &d2) {
  const int a = m + n, c = m - n;
  const T g = (c & 1) ? -K : K;
  d = g * pw(ch, a) * pw(sh, c);
  d1 = g * T(0.5) * (T(c) * pw(ch, a + 1) * pw(sh, c - 1) - T(a) * pw(ch, a - 1) * pw(sh, c + 1));
  d2 = g * T(0.25) *
       (T(c * (c - 1)) * pw(ch, a + 2) * pw(sh, c - 2) -
        T(c * (a + 1) + a * (c + 1)) * pw(ch, a) * pw(sh, c) +
        T(a * (a - 1)) * pw(ch, a - 2) * pw(sh, c + 2));
}

// Adds one image (u, v) with weight W of the sums S0 = sum c d, S1 = sum c d',
// S2 = sum c d'' (complex) to (C, C_a, C_b, C_g, C_aa, C_ab, C_ag, C_bb, C_bg,
// C_gg): the phase exp(i(u a + v g)) brings i u under d/da and i v under d/dg.
__device__ __forceinline__ void add_img(double (&acc)[10], double W, double u, double v, double er,
                                        double ei, double s0r, double s0i, double s1r, double s1i,
                                        double s2r, double s2i) {
  const double zr0 = s0r * er - s0i * ei, zi0 = s0r * ei + s0i * er;
  const double zr1 = s1r * er - s1i * ei, zi1 = s1r * ei + s1i * er;
  const double zr2 = s2r * er - s2i * ei;
  acc[0] += W * zr0;
  acc[1] -= W * u * zi0;
  acc[2] += W * zr1;
  acc[3] -= W * v * zi0;
  acc[4] -= W * u * u * zr0;
  acc[5] -= W * u * zi1;
  acc[6] -= W * u * v * zr0;
  acc[7] += W * zr2;
  acc[8] -= W * v * zi1;
  acc[9] -= W * v * v * zr0;
}

// 3x3 solve H v = g by Gaussian elimination with partial pivoting; false
// (v = 0) when a pivot falls below 1e-14 ||H||_F.
__device__ bool solve3(const double *H, const double *g, double *v) {
  double A[3][4], nf = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      A[i][j] = H[3 * i + j];
      nf += H[3 * i + j] * H[3 * i + j];
    }
    A[i][3] = g[i];
  }
  nf = sqrt(nf);
  for (int k = 0; k < 3; ++k) {
    int piv = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
    if (!(fabs(A[piv][k]) > 1e-14 * nf)) {
      v[0] = v[1] = v[2] = 0.0;
      return false;
    }
    if (piv != k)
      for (int j = 0; j < 4; ++j) {
        const double t = A[k][j];
        A[k][j] = A[piv][j];
        A[piv][j] = t;
      }
    for (int i = k + 1; i < 3; ++i) {
      const double f = A[i][k] / A[k][k];
      for (int j = k; j < 4; ++j) A[i][j] -= f * A[k][j];
    }
  }
  for (int k = 2; k >= 0; --k) {
    double s = A[k][3];
    for (int j = k + 1; j < 3; ++j) s -= A[k][j] * v[j];
    v[k] = s / A[k][k];
  }
  return true;
}

// C, grad, Hessian of C_{L} at theta*_b from the grouped coefficients, then
// shift[b] = (v, C) with v = H^{-1} grad; flags[b] bit 4 when H is singular.
template <typename T>
__global__ void __launch_bounds__(BWD_THREADS)
    k_bwd_point(const T *__restrict__ c, long cper, const T *__restrict__ rcoef,
                const T *__restrict__ seedK, int L, const double *__restrict__ euler,
                double *__restrict__ shift, int *__restrict__ flags) {
  const long b = blockIdx.x;
  const T *cb = c + b * cper;
  const double al = euler[3 * b], be = euler[3 * b + 1], ga = euler[3 * b + 2];
  const T x = (T)cos(be), s = (T)sin(be), ch = (T)cos(0.5 * be), sh = (T)sin(0.5 * be);
  double acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = 0.0;
  const int ng = (L + 1) * (L + 2) / 2;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int m = tri_floor(g), j = g - m * (m + 1) / 2;
    const long e0 = goff_dev(m, j, L);
    for (int h = 0; h < 2; ++h) {
      const int n = 2 * j - m + h;
      if (n > m) break;
      T d, d1, d2, p0 = 0, p1 = 0, p2 = 0;
      seed3<T>(m, n, seedK[4L * g + h], ch, sh, d, d1, d2);
      T s0r = 0, s0i = 0, s1r = 0, s1i = 0, s2r = 0, s2i = 0;  // c_mn sums
      T t0r = 0, t0i = 0, t1r = 0, t1i = 0, t2r = 0, t2i = 0;  // c_nm sums
      for (int l = m; l <= L; ++l) {
        const T *ce = cb + 8 * (e0 + l - m) + h;
        const T cr = ce[0], ci = ce[2], dr = ce[4], di = ce[6];
        s0r += cr * d; s0i += ci * d; s1r += cr * d1; s1i += ci * d1; s2r += cr * d2; s2i += ci * d2;
        t0r += dr * d; t0i += di * d; t1r += dr * d1; t1i += di * d1; t2r += dr * d2; t2i += di * d2;
        if (l < L) {  // d^{l+1} = (a x - b) d^l - e d^{l-1}, differentiated in b
          const T *re = rcoef + 8 * (e0 + l - m) + h;
          const T A = re[0], NB = re[2], NE = re[4];
          const T t = A * x + NB;
          const T n0 = t * d + NE * p0;
          const T n1 = t * d1 - A * s * d + NE * p1;
          const T n2 = t * d2 - T(2) * A * s * d1 - A * x * d + NE * p2;
          p0 = d; p1 = d1; p2 = d2;
          d = n0; d1 = n1; d2 = n2;
        }
      }
      // image (m, n), weight 1 for (0, 0) else 2 (with its conjugate (-m, -n))
      {
        const double ph = m * al + n * ga;
        add_img(acc, (m == 0 && n == 0) ? 1.0 : 2.0, m, n, cos(ph), sin(ph), s0r, s0i, s1r, s1i,
                s2r, s2i);
      }
      // image (n, m): d^l_nm = (-1)^{m-n} d^l_mn; absent for n = +-m
      if (n != m && n != -m) {
        const double ph = n * al + m * ga;
        add_img(acc, ((m - n) & 1) ? -2.0 : 2.0, n, m, cos(ph), sin(ph), t0r, t0i, t1r, t1i, t2r,
                t2i);
      }
    }
  }
  __shared__ double red[BWD_THREADS / 32][10];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[10];
    for (int i = 0; i < 10; ++i) {
      r[i] = 0.0;
      for (int w = 0; w < BWD_THREADS / 32; ++w) r[i] += red[w][i];
    }
    const double grad[3] = {r[1], r[2], r[3]};
    const double H[9] = {r[4], r[5], r[6], r[5], r[7], r[8], r[6], r[8], r[9]};
    double v[3];
    const bool ok = solve3(H, grad, v);
    shift[4 * b] = v[0];
    shift[4 * b + 1] = v[1];
    shift[4 * b + 2] = v[2];
    shift[4 * b + 3] = r[0];
    if (flags) flags[b] = ok ? 0 : 16;
  }
}

// Shared memory of k_bwd_coef, in reals: recurrence state [4][(L+1)^2],
// E' [2L+1][L+1][2], phase tables [4][2L+1].
__host__ __device__ __forceinline__ long bwd_coef_reals(int L) {
  return 4L * (L + 1) * (L + 1) + 2L * (2 * L + 1) * (L + 1) + 4L * (2 * L + 1);
}

template <typename T>
__global__ void __launch_bounds__(BWD_THREADS)
    k_bwd_coef(const T *__restrict__ f, int S, int L, const double *__restrict__ wrad,
               const T *__restrict__ rcoef, const T *__restrict__ seedK,
               const double *__restrict__ euler, const double *__restrict__ shift,
               const double *__restrict__ weight, T *__restrict__ X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long b = blockIdx.x;
  const int np = (L + 1) * (L + 1), nlm = (L + 1) * (L + 2) / 2, R2 = 2 * L + 1;
  T *dc = reinterpret_cast<T *>(smem_raw);  // d^l
  T *dp = dc + np;                           // d^{l-1}
  T *d1c = dp + np;                          // d'^l
  T *d1p = d1c + np;                         // d'^{l-1}
  T *Es = d1p + np;                          // [m + L][n][2]
  T *pa = Es + 2L * R2 * (L + 1);            // cos, sin (k a), k = -L..L
  T *pg = pa + 2 * R2;                       // cos, sin (k g)
  const double al = euler[3 * b], be = euler[3 * b + 1], ga = euler[3 * b + 2];
  const T va = (T)shift[4 * b], vb = (T)shift[4 * b + 1], vg = (T)shift[4 * b + 2];
  const double wb = weight ? weight[b] : 1.0;
  const T x = (T)cos(be), s = (T)sin(be), ch = (T)cos(0.5 * be), sh = (T)sin(0.5 * be);
  for (int k = threadIdx.x; k < R2; k += blockDim.x) {
    const double ka = (k - L) * al, kg = (k - L) * ga;
    pa[2 * k] = (T)cos(ka); pa[2 * k + 1] = (T)sin(ka);
    pg[2 * k] = (T)cos(kg); pg[2 * k + 1] = (T)sin(kg);
  }
  const T *fb = f + 2L * b * S * nlm;
  T *Xb = X + 2L * b * S * nlm;
  __syncthreads();
  for (int l = 0; l <= L; ++l) {
    // 1. d^l, d'^l of every pair (m, n), m = isqrt(q), n = q - m^2 - m, with
    //    m <= l; then E' of its images with a non-negative second index
    for (int q = threadIdx.x; q < (l + 1) * (l + 1); q += blockDim.x) {
      const int m = isqrt_floor(q), n = q - m * m - m;
      const int j = (n + m) >> 1, h = (n + m) & 1;
      T d, d1;
      if (m == l) {
        T d2;
        seed3<T>(m, n, seedK[4L * (m * (m + 1) / 2 + j) + h], ch, sh, d, d1, d2);
        dp[q] = T(0); d1p[q] = T(0);
      } else {  // step l-1 -> l with the coefficients of entry (group, l-1)
        const T *re = rcoef + 8 * (goff_dev(m, j, L) + (l - 1) - m) + h;
        const T A = re[0], NB = re[2], NE = re[4];
        const T t = A * x + NB, od = dc[q], od1 = d1c[q];
        d = t * od + NE * dp[q];
        d1 = t * od1 - A * s * od + NE * d1p[q];
        dp[q] = od; d1p[q] = od1;
      }
      dc[q] = d; d1c[q] = d1;
      // images (u, w) with d^l_uw = sg d^l_mn:
      //   (m, n) sg 1; (n, m) and (-m, -n) sg (-1)^{m-n}; (-n, -m) sg 1
      const T sgm = ((m - n) & 1) ? T(-1) : T(1);
      const int us[4] = {m, n, -m, -n}, ws[4] = {n, m, -n, -m};
      const T sgs[4] = {T(1), sgm, sgm, T(1)};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int u = us[k], w = ws[k];
        if (w < 0) continue;
        const T dd = sgs[k] * d, dd1 = sgs[k] * d1;
        // exp(i(u a + w g)) [dd - vb dd1 - i (u va + w vg) dd]
        const T ar = pa[2 * (u + L)], ai = pa[2 * (u + L) + 1];
        const T gr = pg[2 * (w + L)], gi = pg[2 * (w + L) + 1];
        const T er = ar * gr - ai * gi, ei = ar * gi + ai * gr;
        const T br = dd - vb * dd1, bi = -(T(u) * va + T(w) * vg) * dd;
        T *o = Es + 2 * ((long)(u + L) * (L + 1) + w);
        o[0] = er * br - ei * bi;
        o[1] = er * bi + ei * br;
      }
    }
    __syncthreads();
    // 2. X_ln(s) = w_b w_s (2 if n > 0) sum_{m=-l..l} f_lm(r_s) E'_mn, with
    //    f_{l,-m} = (-1)^m conj(f_lm)
    const int lm0 = l * (l + 1) / 2;
    for (int o = threadIdx.x; o < S * (l + 1); o += blockDim.x) {
      const int sidx = o / (l + 1), n = o - sidx * (l + 1);
      const T *fs = fb + 2L * ((long)sidx * nlm + lm0);
      T xr = 0, xi = 0;
      for (int m = 0; m <= l; ++m) {
        const T fr = fs[2 * m], fi = fs[2 * m + 1];
        const T *ep = Es + 2 * ((long)(m + L) * (L + 1) + n);
        xr += fr * ep[0] - fi * ep[1];
        xi += fr * ep[1] + fi * ep[0];
        if (m > 0) {  // (-1)^m conj(f) E'_{-m, n}
          const T *en = Es + 2 * ((long)(L - m) * (L + 1) + n);
          const T gr = (m & 1) ? -fr : fr, gi = (m & 1) ? fi : -fi;
          xr += gr * en[0] - gi * en[1];
          xi += gr * en[1] + gi * en[0];
        }
      }
      const T sc = (T)(wb * wrad[sidx] * (n > 0 ? 2.0 : 1.0));
      T *xo = Xb + 2L * ((long)sidx * nlm + lm0 + n);
      xo[0] = sc * xr;
      xo[1] = sc * xi;
    }
    __syncthreads();
  }
}

// G[s][lm] = sum_b X[b][s][lm] (FP64 sums, fixed order).
template <typename T>
__global__ void k_bwd_reduce(const T *__restrict__ X, int B, long per, T *__restrict__ G) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per) return;
  double acc = 0.0;
  for (int b = 0; b < B; ++b) acc += (double)X[(long)b * per + i];
  G[i] = (T)acc;
}

// Transpose of the analysis of one shell s of template t: the sample
// gradient du(j, k) = Re sum_m A_m(j) exp(i m phi_k) with
// A_m(j) = sum_l ptab[j][lm] G_lm(r_s), ptab = w_j (2 pi / n_phi) Pbar_lm(x_j),
// then the transpose of the trilinear sampling at the forward pass's own
// coordinates (same clamping of the corner), by FP64 atomic adds.
template <typename T>
__global__ void __launch_bounds__(BWD_THREADS)
    k_bwd_synth(const T *__restrict__ G, int S, int L, int N, const T *__restrict__ ptab,
                const T *__restrict__ phi_cs, const T *__restrict__ ring, double *__restrict__ vox) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int sidx = blockIdx.x;
  const long t = blockIdx.y;
  const int nt = L + 1, nph = 2 * L + 2, nlm = (L + 1) * (L + 2) / 2;
  T *A = reinterpret_cast<T *>(smem_raw);  // [nt][L+1][2]
  T *cs = A + 2 * nt * (L + 1);             // [nph][2]
  const T *Gs = G + 2L * (t * S + sidx) * nlm;
  for (int k = threadIdx.x; k < 2 * nph; k += blockDim.x) cs[k] = phi_cs[k];
  for (int it = threadIdx.x; it < nt * (L + 1); it += blockDim.x) {
    const int j = it / (L + 1), m = it - j * (L + 1);
    T ar = 0, ai = 0;
    for (int l = m; l <= L; ++l) {
      const int lm = l * (l + 1) / 2 + m;
      const T p = ptab[(long)j * nlm + lm];
      ar += p * Gs[2 * lm];
      ai += p * Gs[2 * lm + 1];
    }
    A[2 * it] = ar;
    A[2 * it + 1] = ai;
  }
  __syncthreads();
  const T c0 = (T)(0.5 * N), hi = (T)(N - 1);
  const long NN = (long)N * N;
  double *vt = vox + t * NN * N;
  for (int it = threadIdx.x; it < nt * nph; it += blockDim.x) {
    const int j = it / nph, k = it - j * nph;
    T du = 0;
    int mk = 0;  // m k mod n_phi
    for (int m = 0; m <= L; ++m) {
      du += A[2 * (j * (L + 1) + m)] * cs[2 * mk] - A[2 * (j * (L + 1) + m) + 1] * cs[2 * mk + 1];
      mk += k;
      if (mk >= nph) mk -= nph;
    }
    const T rho = ring[2 * ((long)sidx * nt + j)], pz = ring[2 * ((long)sidx * nt + j) + 1];
    const T px = c0 + rho * cs[2 * k], py = c0 + rho * cs[2 * k + 1];
    const T fx = floor(px), fy = floor(py), fz = floor(pz);
    const bool inside = px >= T(0) && py >= T(0) && pz >= T(0) && px <= hi && py <= hi && pz <= hi;
    int i0, j0, k0;
    T tx, ty, tz;
    if (inside) {
      i0 = min((int)fx, N - 2); j0 = min((int)fy, N - 2); k0 = min((int)fz, N - 2);
      tx = px - (T)i0; ty = py - (T)j0; tz = pz - (T)k0;
    } else {
      i0 = (int)fx; j0 = (int)fy; k0 = (int)fz;
      tx = px - fx; ty = py - fy; tz = pz - fz;
    }
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int ii = i0 + dx, jj = j0 + dy, kk = k0 + dz;
          if (ii < 0 || jj < 0 || kk < 0 || ii >= N || jj >= N || kk >= N) continue;
          const T w = (dx ? tx : T(1) - tx) * (dy ? ty : T(1) - ty) * (dz ? tz : T(1) - tz);
          atomicAdd(vt + (long)kk * NN + (long)jj * N + ii, (double)w * (double)du);
        }
  }
}

}  // namespace

size_t bwd_coef_smem(const Plan &p) { return (p.fp64 ? 8 : 4) * (size_t)bwd_coef_reals(p.LJ); }
bool backward_fits(const Plan &p) { return bwd_coef_smem(p) <= 227 * 1024; }

template <typename T>
cudaError_t launch_template_grad(const Plan &p, const T *f, const T *c, int B, int tstride,
                                 const double *euler, const double *weight, T *X, T *coef_grad,
                                 double *vox_grad, double *shift, int *flags, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const long per = 2L * p.S * p.nlm;
  k_bwd_point<T><<<B, BWD_THREADS, 0, st>>>(c, 4L * p.nc, (const T *)p.rcoef, (const T *)p.seedK,
                                            p.LJ, euler, shift, flags);
  const size_t smem = bwd_coef_smem(p);
  cudaFuncSetAttribute(k_bwd_coef<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  T *Xo = tstride ? coef_grad : X;
  k_bwd_coef<T><<<B, BWD_THREADS, smem, st>>>(f, p.S, p.LJ, p.wrad, (const T *)p.rcoef,
                                              (const T *)p.seedK, euler, shift, weight, Xo);
  const int ntmpl = tstride ? B : 1;
  if (!tstride)
    k_bwd_reduce<T><<<(int)((per + 255) / 256), 256, 0, st>>>(X, B, per, coef_grad);
  if (vox_grad) {
    const long nv = (long)p.N * p.N * p.N * ntmpl;
    cudaError_t e = cudaMemsetAsync(vox_grad, 0, sizeof(double) * nv, st);
    if (e != cudaSuccess) return e;
    const size_t ss = sizeof(T) * (2 * (size_t)(p.LJ + 1) * (p.LJ + 1) + 2 * (size_t)(2 * p.LJ + 2));
    k_bwd_synth<T><<<dim3(p.S, ntmpl), BWD_THREADS, ss, st>>>(coef_grad, p.S, p.LJ, p.N,
                                                              (const T *)p.ptab, (const T *)p.phi_cs,
                                                              (const T *)p.ring, vox_grad);
  }
  return cudaGetLastError();
}

template cudaError_t launch_template_grad<float>(const Plan &, const float *, const float *, int,
                                                 int, const double *, const double *, float *,
                                                 float *, double *, double *, int *, cudaStream_t);
template cudaError_t launch_template_grad<double>(const Plan &, const double *, const double *, int,
                                                  int, const double *, const double *, double *,
                                                  double *, double *, double *, int *, cudaStream_t);

}  // namespace matcha
