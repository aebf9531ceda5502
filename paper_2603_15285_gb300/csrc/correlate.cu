// Step a3: the per-degree contraction of Eq. (sigmalmm), with the radial
// quadrature in place of the ball-harmonic radial index:
//   c^l_{mn} = sum_s w_s f_lm(r_s) conj(h_ln(r_s)).
// Negative orders come from f_{l,-m} = (-1)^m conj(f_lm) (real volumes).
// Output layout: the grouped layout of the plan (pairs (m, n), m >= |n|, taken
// two at a time with equal m, components of the two partners interleaved);
// each (pair, l), l = m..L_J, holds (c^l_{mn}, c^l_{nm}).
#include "internal.cuh"

namespace matcha {

template <typename T>
__device__ __forceinline__ void coef_at(const T *__restrict__ f, int nlm, int s, int l, int m,
                                        T &re, T &im) {
  int am = m < 0 ? -m : m;
  const T *q = f + 2 * ((long)s * nlm + l * (l + 1) / 2 + am);
  re = q[0];
  im = q[1];
  if (m < 0) {
    if (am & 1) re = -re; else im = -im;
  }
}

// One CTA per (particle, degree pair {l, L-l}): the coefficients of both
// degrees (all shells, orders 0..l) are staged in shared memory with the
// template side pre-multiplied by the radial weight, then one thread per
// (degree, order pair (m, n), m >= |n|) produces (c^l_mn, c^l_nm); the two
// degrees share one item loop, so pairing l with L - l balances the
// (l+1)^2 + (L-l+1)^2 items of a CTA.  The signs of the negative order -|n|
// are applied once after the shell sums.
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

//
// With BALL (plans with the ball-harmonic radial basis) the staged rows are
// the projections on the retained radial functions instead of the shells:
// f_klm = sum_s W_lk(s) f_lm(r_s), W_lk(s) = w_s N_lk j_l(lambda_lk r_s / R),
// for k < |K_l| (both sides), and the products run over those |K_l| rows:
// c^l_mn = sum_{k in K_l} f_klm conj(h_kln), Eq. (sigmalmm) itself, i.e. A_l
// through its rank-|K_l| factors, so a degree costs |K_l| (2l+1)^2 products
// instead of S (2l+1)^2.
template <typename T, bool BALL>
__global__ void __launch_bounds__(256)
k_correlate_deg(const T *__restrict__ f, const T *__restrict__ h, int S, int L, long h_stride,
                const double *__restrict__ wrad, const int *__restrict__ pair_base, long nc,
                T *__restrict__ c, const T *__restrict__ ballW, const int *__restrict__ ballK,
                int Kmax) {
  using C2 = typename Cplx<T>::type;
  const long b = blockIdx.y;
  const int nlm = (L + 1) * (L + 2) / 2;
  const T *fb = f + 2 * b * (long)S * nlm;
  const T *hb = h + 2 * (b * h_stride) * (long)S * nlm;
  T *cb = c + 4 * b * nc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2 *sF = reinterpret_cast<C2 *>(smem_raw);
  const int l_lo = blockIdx.x, l_hi = L - blockIdx.x;
  const int npass = l_hi == l_lo ? 1 : 2;
  // stage: degree d's orders 0..l at [S][l+1] (F) and [S][l+1] (w H)
  const int no0 = l_lo + 1, no1 = l_hi + 1;
  const int R0 = BALL ? Kmax : S;  // rows reserved per degree
  C2 *F0 = sF, *H0 = sF + R0 * no0, *F1 = sF + 2 * R0 * no0, *H1 = F1 + R0 * no1;
  // rows summed per degree: the shells, or the retained radial functions
  const int S0 = BALL ? ballK[l_lo] : S, S1 = BALL ? ballK[l_hi] : S;
  for (int d = 0; d < npass; ++d) {
    const int l = d ? l_hi : l_lo, no = l + 1, base = l * (l + 1) / 2;
    C2 *Fd = d ? F1 : F0, *Hd = d ? H1 : H0;
    if (BALL) {
      const int Kl = d ? S1 : S0;
      const T *Wl = ballW + (long)l * Kmax * S;
      for (int t = threadIdx.x; t < Kl * no; t += blockDim.x) {
        const int k = t / no, m = t - k * no;
        C2 fv{T(0), T(0)}, hv{T(0), T(0)};
        for (int s = 0; s < S; ++s) {
          const T w = Wl[k * S + s];
          const long src = 2 * ((long)s * nlm + base + m);
          fv.x = fma(w, fb[src], fv.x); fv.y = fma(w, fb[src + 1], fv.y);
          hv.x = fma(w, hb[src], hv.x); hv.y = fma(w, hb[src + 1], hv.y);
        }
        Fd[t] = fv; Hd[t] = hv;
      }
    } else {
      for (int t = threadIdx.x; t < S * no; t += blockDim.x) {
        int s = t / no, m = t - s * no;
        long src = 2 * ((long)s * nlm + base + m);
        T w = (T)wrad[s];
        C2 fv, hv;
        fv.x = fb[src]; fv.y = fb[src + 1];
        hv.x = w * hb[src]; hv.y = w * hb[src + 1];
        Fd[t] = fv; Hd[t] = hv;
      }
    }
  }
  __syncthreads();
  // Products over the shells for every order pair (a, b), 0 <= a, b <= l:
  //   A = sum f_a.re h_b.re, B = sum f_a.im h_b.im, C = sum f_a.im h_b.re, D = sum f_a.re h_b.im,
  // so that P1 = sum f_a conj(h_b) = (A + B) + i (C - D) and P2 = sum f_a h_b =
  // (A - B) + i (C + D).  With f_{l,-k} = (-1)^k conj(f_{lk}) (real volumes):
  //   c_mn = P1[m][n] (n >= 0),  (-1)^|n| P2[m][|n|] (n < 0),
  //   c_nm = P1[n][m] (n >= 0),  (-1)^|n| conj(P2[|n|][m]) (n < 0).
  // One thread per 2 x 2 block of (a, b): two 128-bit loads per shell feed 16
  // multiply-adds.
  const int h0 = (l_lo + 2) / 2, h1 = (l_hi + 2) / 2;  // blocks per side
  const int t_lo = h0 * h0, t_tot = t_lo + (npass == 2 ? h1 * h1 : 0);
  for (int t = threadIdx.x; t < t_tot; t += blockDim.x) {
    const int d = t < t_lo ? 0 : 1, tt = d ? t - t_lo : t, hh = d ? h1 : h0;
    const int l = d ? l_hi : l_lo, no = l + 1;
    const int a0 = 2 * (tt / hh), b0 = 2 * (tt - (tt / hh) * hh);
    // rows past l read a zero-weighted copy of row l (loaded, never stored)
    const int a1 = a0 + 1 <= l ? a0 + 1 : a0, b1 = b0 + 1 <= l ? b0 + 1 : b0;
    T acc[2][2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[u][v][k] = 0;
    const C2 *F = d ? F1 : F0, *H = d ? H1 : H0;
    const int Sd = d ? S1 : S0;
    for (int s = 0; s < Sd; ++s, F += no, H += no) {
      const C2 fa[2] = {F[a0], F[a1]}, hb[2] = {H[b0], H[b1]};
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          acc[u][v][0] = fma(fa[u].x, hb[v].x, acc[u][v][0]);
          acc[u][v][1] = fma(fa[u].y, hb[v].y, acc[u][v][1]);
          acc[u][v][2] = fma(fa[u].y, hb[v].x, acc[u][v][2]);
          acc[u][v][3] = fma(fa[u].x, hb[v].y, acc[u][v][3]);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int ai = a0 + u, bi = b0 + v;
        if (ai > l || bi > l) continue;
        const T A = acc[u][v][0], B = acc[u][v][1], C = acc[u][v][2], D = acc[u][v][3];
        const T p1r = A + B, p1i = C - D, p2r = A - B, p2i = C + D;
        // P1[ai][bi]: c_mn of pair (ai, bi) when ai >= bi; c_nm of pair (bi, ai) when ai <= bi
        if (ai >= bi) {
          const int m = ai, n = bi, q = m * m + n + m;
          T *o = cb + pair_base[q] + 8L * (l - m);
          o[0] = p1r; o[2] = p1i;
          if (n == m) { o[4] = p1r; o[6] = p1i; o[1] = 0; o[3] = 0; o[5] = 0; o[7] = 0; }
        }
        if (ai < bi) {
          const int m = bi, n = ai, q = m * m + n + m;
          T *o = cb + pair_base[q] + 8L * (l - m);
          o[4] = p1r; o[6] = p1i;
        }
        // P2[ai][bi] with the smaller index k > 0 as |n|: pair (max, -min)
        const int mx = ai > bi ? ai : bi, k = ai > bi ? bi : ai;
        if (k > 0) {
          const T sg = (k & 1) ? T(-1) : T(1);
          const int q = mx * mx - k + mx;
          T *o = cb + pair_base[q] + 8L * (l - mx);
          if (ai >= bi) { o[0] = sg * p2r; o[2] = sg * p2i; }    // c_{m,-k} = (-1)^k P2[m][k]
          if (ai <= bi) { o[4] = sg * p2r; o[6] = -sg * p2i; }   // c_{-k,m} = (-1)^k conj(P2[k][m])
        }
      }
  }
}

template <typename T>
cudaError_t launch_correlate(const Plan &p, const T *f, const T *h, int B, int hstride, T *c,
                             cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  if (sizeof(T) == 4 && p.tc)
    return launch_correlate_tc(p, (const float *)f, (const float *)h, B, hstride, (float *)c, st);
  const bool ball = p.ball_kmax > 0;
  const int rows = ball ? p.ball_kmax : p.S;
  size_t smem = sizeof(T) * 4 * (size_t)rows * (p.LJ + 2);  // both degrees of a pair
  static bool attr[2][2] = {{false, false}, {false, false}};
  if (!attr[ball][sizeof(T) == 8]) {
    cudaFuncSetAttribute(ball ? k_correlate_deg<T, true> : k_correlate_deg<T, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr[ball][sizeof(T) == 8] = true;
  }
  dim3 grid(p.LJ / 2 + 1, B);
  if (ball)
    k_correlate_deg<T, true><<<grid, 256, smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad, p.pair_base,
                                                      p.nc, c, (const T *)p.ball_W, p.ball_K,
                                                      p.ball_kmax);
  else
    k_correlate_deg<T, false><<<grid, 256, smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad,
                                                       p.pair_base, p.nc, c, nullptr, nullptr, 0);
  return cudaGetLastError();
}

template cudaError_t launch_correlate<float>(const Plan &, const float *, const float *, int, int,
                                             float *, cudaStream_t);
template cudaError_t launch_correlate<double>(const Plan &, const double *, const double *, int,
                                              int, double *, cudaStream_t);

}  // namespace matcha
