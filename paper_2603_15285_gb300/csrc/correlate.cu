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
// template side pre-multiplied by the radial weight, then one thread per order
// pair (m, n), m >= |n|, produces (c^l_mn, c^l_nm).  Pairing degree l with
// L - l balances the (l+1)^2 work of a degree.
template <typename T>
__global__ void __launch_bounds__(256)
k_correlate_deg(const T *__restrict__ f, const T *__restrict__ h, int S, int L, long h_stride,
                const double *__restrict__ wrad, const int *__restrict__ pair_base, long nc,
                T *__restrict__ c) {
  const long b = blockIdx.y;
  const int nlm = (L + 1) * (L + 2) / 2;
  const T *fb = f + 2 * b * (long)S * nlm;
  const T *hb = h + 2 * (b * h_stride) * (long)S * nlm;
  T *cb = c + 4 * b * nc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sF = reinterpret_cast<T *>(smem_raw);
  const int l_lo = blockIdx.x, l_hi = L - blockIdx.x;
  for (int pass = 0; pass < 2; ++pass) {
    const int l = pass ? l_hi : l_lo;
    if (pass && l_hi == l_lo) break;
    const int no = l + 1;                    // orders 0..l
    T *Fs = sF;                              // [S][no] complex
    T *Hs = sF + 2 * S * no;                 // [S][no] complex, times w_s
    const int base = l * (l + 1) / 2;
    for (int t = threadIdx.x; t < S * no; t += blockDim.x) {
      int s = t / no, m = t - s * no;
      long src = 2 * ((long)s * nlm + base + m);
      T w = (T)wrad[s];
      Fs[2 * t] = fb[src]; Fs[2 * t + 1] = fb[src + 1];
      Hs[2 * t] = w * hb[src]; Hs[2 * t + 1] = w * hb[src + 1];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < no * no; q += blockDim.x) {
      int m = isqrt_floor(q), n = q - m * m - m;
      int an = n < 0 ? -n : n;
      // order -|n| of a real function: (-1)^n conj(.)
      T sr = (n < 0 && (an & 1)) ? T(-1) : T(1);
      T si = n < 0 ? -sr : sr;
      T r1 = 0, i1 = 0, r2 = 0, i2 = 0;
      for (int s = 0; s < S; ++s) {
        const T *F = Fs + 2 * s * no, *H = Hs + 2 * s * no;
        T fmr = F[2 * m], fmi = F[2 * m + 1];
        T hmr = H[2 * m], hmi = H[2 * m + 1];
        T fnr = sr * F[2 * an], fni = si * F[2 * an + 1];
        T hnr = sr * H[2 * an], hni = si * H[2 * an + 1];
        // c_mn += f_lm conj(w h_ln);  c_nm += f_ln conj(w h_lm)
        r1 = fma(fmr, hnr, fma(fmi, hni, r1));
        i1 = fma(fmi, hnr, fma(-fmr, hni, i1));
        r2 = fma(fnr, hmr, fma(fni, hmi, r2));
        i2 = fma(fni, hmr, fma(-fnr, hmi, i2));
      }
      T *o = cb + pair_base[q] + 8L * (l - m);
      o[0] = r1; o[2] = i1; o[4] = r2; o[6] = i2;
      if (n == m) { o[1] = 0; o[3] = 0; o[5] = 0; o[7] = 0; }  // empty partner
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_correlate(const Plan &p, const T *f, const T *h, int B, int hstride, T *c,
                             cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  size_t smem = sizeof(T) * 4 * (size_t)p.S * (p.LJ + 1);
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
