// Steps a1+a2: shell sampling and spherical-harmonic analysis.
//
// The paper obtains ball-harmonic coefficients with a NUFFT (Section 1.1,
// Appendix A.1-A.2); this path samples each volume on the quadrature points of
// S radial shells instead (Gauss-Legendre in r, Gauss-Legendre in cos(theta),
// equispaced in phi) and analyses every shell:
//   F_m(s, j)  = sum_k f(r_s w_jk) exp(-i m phi_k)                 (phi DFT)
//   f_lm(r_s)  = sum_j w_j (2 pi / n_phi) Pbar_lm(x_j) F_m(s, j)    (Legendre)
// One CTA owns one (volume, shell): it gathers the n_theta * n_phi trilinear
// samples into shared memory, folds the real DFT (pairs k, n_phi - k) and
// runs the Legendre sums against the plan's table.
#include "internal.cuh"

namespace matcha {

template <typename T>
__device__ __forceinline__ T trilinear(const float *__restrict__ vol, int N, T px, T py, T pz) {
  T fx = floor(px), fy = floor(py), fz = floor(pz);
  int i = (int)fx, j = (int)fy, k = (int)fz;
  T tx = px - fx, ty = py - fy, tz = pz - fz;
  T v = 0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    int kk = k + dz;
    bool okz = kk >= 0 && kk < N;
    T wz = dz ? tz : T(1) - tz;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      int jj = j + dy;
      bool oky = okz && jj >= 0 && jj < N;
      T wy = wz * (dy ? ty : T(1) - ty);
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        int ii = i + dx;
        if (oky && ii >= 0 && ii < N) {
          T w = wy * (dx ? tx : T(1) - tx);
          v += w * (T)__ldg(vol + ((long)kk * N + jj) * N + ii);
        }
      }
    }
  }
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_analyze(const float *__restrict__ vols, int N, int S, int L, const double *__restrict__ rs,
          const double *__restrict__ xj, const T *__restrict__ ptab, const T *__restrict__ phi_cs,
          T *__restrict__ out) {
  const int s = blockIdx.x;
  const long b = blockIdx.y;
  const int nt = L + 1, np = 2 * L + 2, nm = L + 1, nlm = (L + 1) * (L + 2) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smp = reinterpret_cast<T *>(smem_raw);  // [nt][np]
  T *F = smp + nt * np;                       // [nt][nm] complex
  const float *vol = vols + b * N * N * N;
  const T r = (T)rs[s];
  const T c0 = (T)(0.5 * N);

  for (int idx = threadIdx.x; idx < nt * np; idx += blockDim.x) {
    int j = idx / np, k = idx - j * np;
    T x = (T)xj[j];
    T st = sqrt(max(T(1) - x * x, T(0)));
    T px = c0 + r * st * phi_cs[2 * k];
    T py = c0 + r * st * phi_cs[2 * k + 1];
    T pz = c0 + r * x;
    smp[idx] = trilinear<T>(vol, N, px, py, pz);
  }
  __syncthreads();

  const int half = np / 2;
  for (int idx = threadIdx.x; idx < nt * nm; idx += blockDim.x) {
    int j = idx / nm, m = idx - j * nm;
    const T *row = smp + j * np;
    T re = row[0] + ((m & 1) ? -row[half] : row[half]);
    T im = 0;
    int t = m;
    for (int k = 1; k < half; ++k) {
      T sp = row[k] + row[np - k], sm = row[k] - row[np - k];
      re = fma(sp, phi_cs[2 * t], re);
      im = fma(-sm, phi_cs[2 * t + 1], im);
      t += m;
      if (t >= np) t -= np;
    }
    F[2 * idx] = re;
    F[2 * idx + 1] = im;
  }
  __syncthreads();

  T *o = out + 2 * ((b * S + s) * (long)nlm);
  for (int lm = threadIdx.x; lm < nlm; lm += blockDim.x) {
    int l = (int)((sqrtf(8.0f * lm + 1.0f) - 1.0f) * 0.5f);
    while (l * (l + 1) / 2 > lm) --l;
    while ((l + 1) * (l + 2) / 2 <= lm) ++l;
    int m = lm - l * (l + 1) / 2;
    const T *pt = ptab + (long)lm * nt;
    T re = 0, im = 0;
    for (int j = 0; j < nt; ++j) {
      T w = pt[j];
      re = fma(w, F[2 * (j * nm + m)], re);
      im = fma(w, F[2 * (j * nm + m) + 1], im);
    }
    o[2 * lm] = re;
    o[2 * lm + 1] = im;
  }
}

template <typename T>
cudaError_t launch_analyze(const Plan &p, const float *vols, int B, T *coef, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  size_t smem = sizeof(T) * ((size_t)p.nt * p.np + 2 * (size_t)p.nt * (p.LJ + 1));
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(T) == 8]) {
    cudaFuncSetAttribute(k_analyze<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set[sizeof(T) == 8] = true;
  }
  k_analyze<T><<<dim3(p.S, B), 256, smem, st>>>(vols, p.N, p.S, p.LJ, p.rs, p.xj, (const T *)p.ptab,
                                                 (const T *)p.phi_cs, coef);
  return cudaGetLastError();
}

template cudaError_t launch_analyze<float>(const Plan &, const float *, int, float *, cudaStream_t);
template cudaError_t launch_analyze<double>(const Plan &, const float *, int, double *, cudaStream_t);

}  // namespace matcha
