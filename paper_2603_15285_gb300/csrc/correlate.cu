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

template <typename T>
__global__ void __launch_bounds__(256)
k_correlate_deg(const T *__restrict__ f, const T *__restrict__ h, int S, int L, long h_stride,
                const double *__restrict__ wrad, const int *__restrict__ pair_base, long nc,
                T *__restrict__ c) {
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
  C2 *F0 = sF, *H0 = sF + S * no0, *F1 = sF + 2 * S * no0, *H1 = F1 + S * no1;
  for (int d = 0; d < npass; ++d) {
    const int l = d ? l_hi : l_lo, no = l + 1, base = l * (l + 1) / 2;
    C2 *Fd = d ? F1 : F0, *Hd = d ? H1 : H0;
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
  __syncthreads();
  const int n_lo = (l_lo + 1) * (l_lo + 1), n_tot = n_lo + (npass == 2 ? (l_hi + 1) * (l_hi + 1) : 0);
  for (int t = threadIdx.x; t < n_tot; t += blockDim.x) {
    const int d = t < n_lo ? 0 : 1, q = d ? t - n_lo : t, l = d ? l_hi : l_lo, no = l + 1;
    const int m = isqrt_floor(q), n = q - m * m - m;
    const int an = n < 0 ? -n : n;
    // order -|n| of a real function: f_{l,-|n|} = (-1)^|n| conj(f_{l,|n|})
    const T sr = (n < 0 && (an & 1)) ? T(-1) : T(1);
    const T si = n < 0 ? -sr : sr;
    // c_mn = sum_s f_lm conj(w h_ln), c_nm = sum_s f_ln conj(w h_lm), with the
    // order-n factors' signs (sr, si) taken out of the sums
    T a = 0, bb = 0, cc = 0, dd = 0, e = 0, g = 0, ii = 0, jj = 0;
    const C2 *F = d ? F1 : F0, *H = d ? H1 : H0;
    for (int s = 0; s < S; ++s, F += no, H += no) {
      const C2 fm = F[m], hm = H[m], fn = F[an], hn = H[an];
      a = fma(fm.x, hn.x, a);  bb = fma(fm.y, hn.y, bb);
      cc = fma(fm.y, hn.x, cc); dd = fma(fm.x, hn.y, dd);
      e = fma(fn.x, hm.x, e);  g = fma(fn.y, hm.y, g);
      ii = fma(fn.y, hm.x, ii); jj = fma(fn.x, hm.y, jj);
    }
    T *o = cb + pair_base[q] + 8L * (l - m);
    o[0] = sr * a + si * bb;   // Re c_mn
    o[2] = sr * cc - si * dd;  // Im c_mn
    o[4] = sr * e + si * g;    // Re c_nm
    o[6] = si * ii - sr * jj;  // Im c_nm
    if (n == m) { o[1] = 0; o[3] = 0; o[5] = 0; o[7] = 0; }  // empty partner
  }
}

template <typename T>
cudaError_t launch_correlate(const Plan &p, const T *f, const T *h, int B, int hstride, T *c,
                             cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  size_t smem = sizeof(T) * 4 * (size_t)p.S * (p.LJ + 2);  // both degrees of a pair
  static bool attr[2] = {false, false};
  if (!attr[sizeof(T) == 8]) {
    cudaFuncSetAttribute(k_correlate_deg<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr[sizeof(T) == 8] = true;
  }
  k_correlate_deg<T><<<dim3(p.LJ / 2 + 1, B), 256, smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad,
                                                              p.pair_base, p.nc, c);
  return cudaGetLastError();
}

template cudaError_t launch_correlate<float>(const Plan &, const float *, const float *, int, int,
                                             float *, cudaStream_t);
template cudaError_t launch_correlate<double>(const Plan &, const double *, const double *, int,
                                              int, double *, cudaStream_t);

}  // namespace matcha
