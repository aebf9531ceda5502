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

// Trilinear interpolation, zero outside the box.  Corner indices are clamped
// into the box and out-of-box corners get weight 0, so the eight loads are
// unconditional and can all be in flight together.
template <typename T>
__device__ __forceinline__ T trilinear(const float *__restrict__ vol, int N, T px, T py, T pz) {
  T fx = floor(px), fy = floor(py), fz = floor(pz);
  int i = (int)fx, j = (int)fy, k = (int)fz;
  T tx = px - fx, ty = py - fy, tz = pz - fz;
  T wx0 = (i >= 0 && i < N) ? T(1) - tx : T(0), wx1 = (i + 1 >= 0 && i + 1 < N) ? tx : T(0);
  T wy0 = (j >= 0 && j < N) ? T(1) - ty : T(0), wy1 = (j + 1 >= 0 && j + 1 < N) ? ty : T(0);
  T wz0 = (k >= 0 && k < N) ? T(1) - tz : T(0), wz1 = (k + 1 >= 0 && k + 1 < N) ? tz : T(0);
  int i0 = min(max(i, 0), N - 1), i1 = min(max(i + 1, 0), N - 1);
  int j0 = min(max(j, 0), N - 1), j1 = min(max(j + 1, 0), N - 1);
  int k0 = min(max(k, 0), N - 1), k1 = min(max(k + 1, 0), N - 1);
  const float *p00 = vol + ((long)k0 * N + j0) * N, *p01 = vol + ((long)k0 * N + j1) * N;
  const float *p10 = vol + ((long)k1 * N + j0) * N, *p11 = vol + ((long)k1 * N + j1) * N;
  float v000 = __ldg(p00 + i0), v001 = __ldg(p00 + i1), v010 = __ldg(p01 + i0), v011 = __ldg(p01 + i1);
  float v100 = __ldg(p10 + i0), v101 = __ldg(p10 + i1), v110 = __ldg(p11 + i0), v111 = __ldg(p11 + i1);
  T a0 = wy0 * (wx0 * (T)v000 + wx1 * (T)v001) + wy1 * (wx0 * (T)v010 + wx1 * (T)v011);
  T a1 = wy0 * (wx0 * (T)v100 + wx1 * (T)v101) + wy1 * (wx0 * (T)v110 + wx1 * (T)v111);
  return wz0 * a0 + wz1 * a1;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_analyze(const float *__restrict__ vols, int N, int S, int L, const double *__restrict__ rs,
          const double *__restrict__ xj, const T *__restrict__ ptabT, const T *__restrict__ phi_cs,
          T *__restrict__ out) {
  const int s = blockIdx.x;
  const long b = blockIdx.y;
  const int nt = L + 1, np = 2 * L + 2, nm = L + 1, nlm = (L + 1) * (L + 2) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smp = reinterpret_cast<T *>(smem_raw);  // [nt][np]
  T *F = smp + nt * np;                       // [nt][nm] complex
  T *tw = F + 2 * nt * nm;                    // [np][2]
  const float *vol = vols + b * N * N * N;
  const T r = (T)rs[s];
  const T c0 = (T)(0.5 * N);
  for (int k = threadIdx.x; k < 2 * np; k += blockDim.x) tw[k] = phi_cs[k];
  __syncthreads();

  const int total = nt * np, NT = blockDim.x;
  for (int base = threadIdx.x; base < total; base += 2 * NT) {
    int id1 = base + NT;
    int j0 = base / np, k0 = base - j0 * np;
    int id1c = id1 < total ? id1 : base;
    int j1 = id1c / np, k1 = id1c - j1 * np;
    T x0 = (T)xj[j0], x1 = (T)xj[j1];
    T st0 = sqrt(max(T(1) - x0 * x0, T(0))), st1 = sqrt(max(T(1) - x1 * x1, T(0)));
    T v0 = trilinear<T>(vol, N, c0 + r * st0 * tw[2 * k0], c0 + r * st0 * tw[2 * k0 + 1], c0 + r * x0);
    T v1 = trilinear<T>(vol, N, c0 + r * st1 * tw[2 * k1], c0 + r * st1 * tw[2 * k1 + 1], c0 + r * x1);
    smp[base] = v0;
    if (id1 < total) smp[id1] = v1;
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
      re = fma(sp, tw[2 * t], re);
      im = fma(-sm, tw[2 * t + 1], im);
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
    T re = 0, im = 0;
    for (int j = 0; j < nt; ++j) {
      T w = ptabT[(long)j * nlm + lm];
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
  size_t smem = sizeof(T) * ((size_t)p.nt * p.np + 2 * (size_t)p.nt * (p.LJ + 1) + 2 * (size_t)p.np);
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
