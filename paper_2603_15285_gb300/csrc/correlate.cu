// Step a3: the per-degree contraction of Eq. (sigmalmm), with the radial
// quadrature in place of the ball-harmonic radial index:
//   c^l_{mn} = sum_s w_s f_lm(r_s) conj(h_ln(r_s)).
// Negative orders come from f_{l,-m} = (-1)^m conj(f_lm) (real volumes).
// Output layout: for each order pair (m, n), m >= |n|, the entries l = m..L_J
// hold (c^l_{mn}, c^l_{nm}); one CTA computes the (2m+1)(L_J-m+1) contiguous
// entries of one m for one particle, so its stores are coalesced.
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

template <typename T>
__global__ void __launch_bounds__(256)
k_correlate(const T *__restrict__ f, const T *__restrict__ h, int S, int L, long h_stride,
            const double *__restrict__ wrad, const int *__restrict__ pair_off, long nc,
            T *__restrict__ c) {
  const int m = blockIdx.x;
  const long b = blockIdx.y;
  const int nlm = (L + 1) * (L + 2) / 2;
  const int len = L - m + 1, cnt = (2 * m + 1) * len;
  const T *fb = f + 2 * b * (long)S * nlm;
  const T *hb = h + 2 * (b * h_stride) * (long)S * nlm;
  T *cb = c + 4 * (b * nc + pair_off[m * m]);
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    int nn = e / len;
    int l = m + (e - nn * len);
    int n = nn - m;
    T r1 = 0, i1 = 0, r2 = 0, i2 = 0;
    for (int s = 0; s < S; ++s) {
      T w = (T)wrad[s];
      T fmr, fmi, hmr, hmi, fnr, fni, hnr, hni;
      coef_at(fb, nlm, s, l, m, fmr, fmi);
      coef_at(hb, nlm, s, l, m, hmr, hmi);
      coef_at(fb, nlm, s, l, n, fnr, fni);
      coef_at(hb, nlm, s, l, n, hnr, hni);
      // c_mn += w f_lm conj(h_ln);  c_nm += w f_ln conj(h_lm)
      r1 += w * (fmr * hnr + fmi * hni);
      i1 += w * (fmi * hnr - fmr * hni);
      r2 += w * (fnr * hmr + fni * hmi);
      i2 += w * (fni * hmr - fnr * hmi);
    }
    T *o = cb + 4 * (long)e;
    o[0] = r1; o[1] = i1; o[2] = r2; o[3] = i2;
  }
}

template <typename T>
cudaError_t launch_correlate(const Plan &p, const T *f, const T *h, int B, int hstride, T *c,
                             cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  k_correlate<T><<<dim3(p.LJ + 1, B), 256, 0, st>>>(f, h, p.S, p.LJ, hstride, p.wrad, p.pair_off,
                                                     p.nc, c);
  return cudaGetLastError();
}

template cudaError_t launch_correlate<float>(const Plan &, const float *, const float *, int, int,
                                             float *, cudaStream_t);
template cudaError_t launch_correlate<double>(const Plan &, const double *, const double *, int,
                                              int, double *, cudaStream_t);

}  // namespace matcha
