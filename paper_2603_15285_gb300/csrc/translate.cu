// Translation search of the 6-D pose (the appendix "Alternating search over
// rotations and translations"; three alternations in Section 5.2).
//
// For a fixed rotation g the objective <f, g o S_tau h> is the
// cross-correlation CC(t) = sum_x f(x) u(x - t) of the particle f and the
// rotated template u = g o h at t = g tau.  CC is the circular correlation a
// 3-D FFT computes:
//   1. Z = FFT3(f + i u): both real volumes in one complex transform
//      (mixed radix 4/2/3/5 Stockham passes along x, y and z, each line held
//      in shared memory, loads and stores coalesced along x);
//   2. X(k) = F(k) conj(U(k)) from Z(k) and Z(-k) (the two spectra of a
//      packed pair), in place, one thread per conjugate pair;
//   3. CC(t) = N^-3 Re sum_k X(k) e^{2 pi i k.t/N} (k in [-N/2, N/2)^3, the
//      trigonometric interpolant of CC) only where it is needed, by three
//      separable partial inverse DFTs (z, then y, then x): first on the
//      integer window [-m, m]^3, then on a grid of 2 floor(0.75 U) + 1
//      points per axis at spacing 1/U around the integer peak (the upsampled
//      DFT of Guizar-Sicairos et al. that the paper cites for sub-voxel
//      accuracy);
//   4. the maximum of each grid (ties to the smaller [z][y][x] index, NaN
//      never wins) gives t, and tau = R^T t.
// A pose kernel makes the rotated template u(x) = h(R^T (x - c0) + c0) and
// the shifted template (S_tau h)(x) = h(x - tau) by trilinear interpolation.
#include <math.h>
#include "internal.cuh"

namespace matcha {

template <typename T> struct alignas(2 * sizeof(T)) C2 { T x, y; };

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }
// s * i * a
template <typename T> __device__ __forceinline__ C2<T> cmuli(C2<T> a, T s) { return {-s * a.y, s * a.x}; }
template <typename T> __device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return {s * a.x, s * a.y}; }

// Rounded multiply and add that the compiler may not contract into an FMA:
// the FP64 pose transform then rounds exactly as the oracle's plain C.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// ---- volume pose ------------------------------------------------------------
// out_b(x) = vol_b(R_b^T (x - c0) + c0 - s_b), trilinear, zero outside, one
// thread per output voxel.  R (row-major [B][9]) and s ([B][3]) are nullable
// (identity, zero).
template <typename T>
__global__ void __launch_bounds__(256)
k_pose_volume(int N, const float *__restrict__ vol, long vstride, const double *__restrict__ R,
              const double *__restrict__ sh, float *__restrict__ out) {
  const long b = blockIdx.y;
  const long N2 = (long)N * N, N3 = N2 * N;
  const long v = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (v >= N3) return;
  const int i = (int)(v % N), j = (int)((v / N) % N), k = (int)(v / N2);
  const float *src = vol + b * vstride;
  T r[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (R)
#pragma unroll
    for (int q = 0; q < 9; ++q) r[q] = (T)R[9 * b + q];
  T s0 = 0, s1 = 0, s2 = 0;
  if (sh) { s0 = (T)sh[3 * b]; s1 = (T)sh[3 * b + 1]; s2 = (T)sh[3 * b + 2]; }
  const T c0 = T(0.5) * (T)N;
  const T x = (T)i - c0, y = (T)j - c0, z = (T)k - c0;
  // column c of R dotted with (x, y, z), then + c0 - s, left to right
  T px = add_rn(add_rn(add_rn(add_rn(mul_rn(r[0], x), mul_rn(r[3], y)), mul_rn(r[6], z)), c0), -s0);
  T py = add_rn(add_rn(add_rn(add_rn(mul_rn(r[1], x), mul_rn(r[4], y)), mul_rn(r[7], z)), c0), -s1);
  T pz = add_rn(add_rn(add_rn(add_rn(mul_rn(r[2], x), mul_rn(r[5], y)), mul_rn(r[8], z)), c0), -s2);
  const T fx0 = floor(px), fy0 = floor(py), fz0 = floor(pz);
  const long i0 = (long)fx0, j0 = (long)fy0, k0 = (long)fz0;
  const T tx = add_rn(px, -fx0), ty = add_rn(py, -fy0), tz = add_rn(pz, -fz0);
  T acc = 0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const T w = mul_rn(mul_rn(dx ? tx : add_rn(T(1), -tx), dy ? ty : add_rn(T(1), -ty)),
                           dz ? tz : add_rn(T(1), -tz));
        const long ii = i0 + dx, jj = j0 + dy, kk = k0 + dz;
        T val = 0;
        if (ii >= 0 && jj >= 0 && kk >= 0 && ii < N && jj < N && kk < N)
          val = (T)__ldg(src + (kk * N + jj) * N + ii);
        acc = add_rn(acc, mul_rn(w, val));
      }
  out[b * N3 + v] = (float)acc;
}

cudaError_t launch_pose_volumes(int N, const float *vol, int B, long vol_stride, const double *R,
                                const double *shift, bool fp64, float *out, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const long N3 = (long)N * N * N;
  dim3 grid((unsigned)((N3 + 255) / 256), B);
  if (fp64) k_pose_volume<double><<<grid, 256, 0, st>>>(N, vol, vol_stride, R, shift, out);
  else k_pose_volume<float><<<grid, 256, 0, st>>>(N, vol, vol_stride, R, shift, out);
  return cudaGetLastError();
}

// ---- box FFT ------------------------------------------------------------------
struct FftDesc {
  int N, npass;
  int radix[16];
};

// Size-R DFT in place, V_q = sum_r v_r e^{sg 2 pi i q r / R} (sg = -1 forward).
template <typename T>
__device__ __forceinline__ void dft2(C2<T> *v, T) {
  C2<T> a = v[0], b = v[1];
  v[0] = cadd(a, b); v[1] = csub(a, b);
}
template <typename T>
__device__ __forceinline__ void dft4(C2<T> *v, T sg) {
  C2<T> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  C2<T> s13 = cadd(v[1], v[3]), d13 = cmuli(csub(v[1], v[3]), sg);
  v[0] = cadd(s02, s13); v[2] = csub(s02, s13);
  v[1] = cadd(d02, d13); v[3] = csub(d02, d13);
}
template <typename T>
__device__ __forceinline__ void dft3(C2<T> *v, T sg) {
  const T h3 = T(0.86602540378443864676);  // sin(2 pi / 3)
  C2<T> t1 = cadd(v[1], v[2]), t2 = cmuli(csub(v[1], v[2]), sg * h3);
  C2<T> a = csub(v[0], cscale(t1, T(0.5)));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(a, t2);
  v[2] = csub(a, t2);
}
template <typename T>
__device__ __forceinline__ void dft5(C2<T> *v, T sg) {
  const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos(2pi/5), cos(4pi/5)
  const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin(2pi/5), sin(4pi/5)
  C2<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  C2<T> t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  C2<T> a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
  C2<T> a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
  C2<T> b1 = cmuli(cadd(cscale(t3, s1), cscale(t4, s2)), sg);
  C2<T> b2 = cmuli(csub(cscale(t3, s2), cscale(t4, s1)), sg);
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, b1); v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2); v[3] = csub(a2, b2);
}

// One Stockham autosort pass of radix R over NB lines (line stride LS) of
// length N: butterfly j of a line reads A[j + r N/R], applies the twiddles
// e^{sg 2 pi i k r / (Ns R)} (k = j mod Ns, Ns = product of earlier radices)
// and writes B[(j / Ns) Ns R + k + r Ns].
template <int R, typename T>
__device__ __forceinline__ void fft_pass(const C2<T> *A, C2<T> *Bv, int N, int LS, int NB, int Ns,
                                         const C2<T> *__restrict__ tw, T sg) {
  const int NR = N / R, span = N / (Ns * R);
  for (int t = threadIdx.x; t < NB * NR; t += blockDim.x) {
    const int line = t / NR, j = t - line * NR;
    const int k = j % Ns;
    const C2<T> *a = A + line * LS;
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[j + r * NR];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2<T> w = tw[k * r * span];  // e^{-2 pi i k r / (Ns R)}
        if (sg > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    if (R == 2) dft2(v, sg);
    else if (R == 3) dft3(v, sg);
    else if (R == 4) dft4(v, sg);
    else dft5(v, sg);
    C2<T> *o = Bv + line * LS + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) o[r * Ns] = v[r];
  }
}

// Length-N transforms of NB lines of each volume along `axis` (0 x, 1 y,
// 2 z), in place.  Axis 0: NB consecutive rows; axes 1 and 2: NB
// consecutive x columns of one z plane (axis 1) or one y plane (axis 2), so
// every global access runs along x.  With fre/fim given (forward x pass
// only) the input is the packed pair fre + i fim of float volumes.
template <typename T>
__global__ void __launch_bounds__(256)
k_fft_axis(C2<T> *__restrict__ data, const float *__restrict__ fre, const float *__restrict__ fim,
           int axis, FftDesc fd, const C2<T> *__restrict__ tw, int NB, T sg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = fd.N, LS = N + 1;
  C2<T> *bufA = reinterpret_cast<C2<T> *>(smem_raw);
  C2<T> *bufB = bufA + NB * LS;
  const long b = blockIdx.y;
  const long N2 = (long)N * N, N3 = N2 * N;
  C2<T> *vol = data + b * N3;
  const int tid = threadIdx.x, NT = blockDim.x;
  const long g = blockIdx.x;
  long row0 = 0, ob = 0, es = 1;
  int x0 = 0;
  if (axis == 0) {
    row0 = g * NB;
  } else {
    const int ntile = (N + NB - 1) / NB;
    const long outer = g / ntile;
    x0 = (int)(g - outer * ntile) * NB;
    es = axis == 1 ? N : N2;
    ob = axis == 1 ? outer * N2 : outer * N;
  }
  // load
  for (int idx = tid; idx < NB * N; idx += NT) {
    int line, e;
    long off;
    bool ok;
    if (axis == 0) {
      line = idx / N; e = idx - line * N;
      ok = row0 + line < N2;
      off = (row0 + line) * N + e;
    } else {
      e = idx / NB; line = idx - e * NB;
      ok = x0 + line < N;
      off = ob + e * es + x0 + line;
    }
    C2<T> v{T(0), T(0)};
    if (ok) {
      if (fre) v = C2<T>{(T)__ldg(fre + b * N3 + off), (T)__ldg(fim + b * N3 + off)};
      else v = vol[off];
    }
    bufA[line * LS + e] = v;
  }
  __syncthreads();
  C2<T> *src = bufA, *dst = bufB;
  int Ns = 1;
  for (int q = 0; q < fd.npass; ++q) {
    const int R = fd.radix[q];
    if (R == 4) fft_pass<4>(src, dst, N, LS, NB, Ns, tw, sg);
    else if (R == 2) fft_pass<2>(src, dst, N, LS, NB, Ns, tw, sg);
    else if (R == 3) fft_pass<3>(src, dst, N, LS, NB, Ns, tw, sg);
    else fft_pass<5>(src, dst, N, LS, NB, Ns, tw, sg);
    __syncthreads();
    C2<T> *tmp = src; src = dst; dst = tmp;
    Ns *= R;
  }
  // store
  for (int idx = tid; idx < NB * N; idx += NT) {
    int line, e;
    long off;
    bool ok;
    if (axis == 0) {
      line = idx / N; e = idx - line * N;
      ok = row0 + line < N2;
      off = (row0 + line) * N + e;
    } else {
      e = idx / NB; line = idx - e * NB;
      ok = x0 + line < N;
      off = ob + e * es + x0 + line;
    }
    if (ok) vol[off] = src[line * LS + e];
  }
}

// X(k) = F(k) conj(U(k)) in place from the packed spectrum Z = FFT(f + i u):
// F = (Z(k) + conj Z(-k)) / 2, U = (Z(k) - conj Z(-k)) / (2i), so
// X(k) = (i/4) (Z(k) + conj Z(-k)) (conj Z(k) - Z(-k)) and X(-k) = conj X(k)
// (CC is real).  One thread per conjugate pair (the smaller linear index).
template <typename T>
__global__ void __launch_bounds__(256) k_cross_spectrum(C2<T> *__restrict__ Z, int N) {
  const long b = blockIdx.y;
  const long N2 = (long)N * N, N3 = N2 * N;
  const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (q >= N3) return;
  const int kx = (int)(q % N), ky = (int)((q / N) % N), kz = (int)(q / N2);
  const int mx = kx ? N - kx : 0, my = ky ? N - ky : 0, mz = kz ? N - kz : 0;
  const long q2 = ((long)mz * N + my) * N + mx;
  if (q2 < q) return;
  C2<T> *zb = Z + b * N3;
  const C2<T> A = zb[q], C = zb[q2];
  const C2<T> s{A.x + C.x, A.y - C.y};    // Z(k) + conj Z(-k)
  const C2<T> d{A.x - C.x, -A.y - C.y};   // conj Z(k) - Z(-k)
  const C2<T> p = cmul(s, d);
  const C2<T> X{-T(0.25) * p.y, T(0.25) * p.x};
  zb[q] = X;
  if (q2 != q) zb[q2] = C2<T>{X.x, -X.y};
}

// Grid point j of axis a of particle b: t = org[b][a] + (j + j0) / den (org
// nullable), rounded as the oracle rounds it.
__device__ __forceinline__ double grid_t(const double *org, long b, int a, int j, int j0, int den) {
  return (org ? org[3 * b + a] : 0.0) + (double)(j + j0) / (double)den;
}

// E[b][a][k][j] = e^{2 pi i kk t / N} at the grid points t, kk = k or k - N
// (the symmetric frequency range); a = 0, 1, 2 for the x, y, z components.
template <typename T>
__global__ void __launch_bounds__(256)
k_idft_factors(C2<T> *__restrict__ E, int N, int nt, int B, const double *__restrict__ org,
               int j0, int den) {
  const long tot = (long)B * 3 * N * nt;
  const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (q >= tot) return;
  const int j = (int)(q % nt);
  const int k = (int)((q / nt) % N);
  const int a = (int)((q / ((long)nt * N)) % 3);
  const long b = q / ((long)3 * N * nt);
  const int kk = k < (N + 1) / 2 ? k : k - N;
  const double t = grid_t(org, b, a, j, j0, den);
  T s, c;
  if (sizeof(T) == 8) {
    double sd, cd;
    sincospi(2.0 * kk * t / N, &sd, &cd);
    s = (T)sd; c = (T)cd;
  } else {
    float sf, cf;
    sincospif((float)(2.0 * kk * t / N), &sf, &cf);
    s = (T)sf; c = (T)cf;
  }
  E[q] = C2<T>{c, s};
}

// out[b][a][j][c] = sum_k in[b][a][k][c] E[b][axis][k][j]: the partial inverse
// DFT along a middle (y) or outer (z) axis.  One CTA per (a, tile of TC
// columns, b); the tile's N x TC inputs and the N x nt factors sit in shared
// memory.
template <typename T>
__global__ void __launch_bounds__(256)
k_idft_mid(const C2<T> *__restrict__ in, C2<T> *__restrict__ out, const C2<T> *__restrict__ E,
           int N, int nt, int A, long C, int TC, int axis) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T> *slab = reinterpret_cast<C2<T> *>(smem_raw);  // [N][TC]
  C2<T> *Es = slab + (long)N * TC;                     // [N][nt]
  const long b = blockIdx.y;
  const long ntile = (C + TC - 1) / TC;
  const long a = blockIdx.x / ntile, c0 = (blockIdx.x - a * ntile) * (long)TC;
  const C2<T> *src = in + (b * A + a) * (long)N * C;
  const C2<T> *eb = E + ((b * 3 + axis) * (long)N) * nt;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int idx = tid; idx < N * TC; idx += NT) {
    const int k = idx / TC, c = idx - k * TC;
    slab[idx] = c0 + c < C ? src[(long)k * C + c0 + c] : C2<T>{T(0), T(0)};
  }
  for (int idx = tid; idx < N * nt; idx += NT) Es[idx] = eb[idx];
  __syncthreads();
  C2<T> *dstb = out + (b * A + a) * (long)nt * C;
  for (int o = tid; o < nt * TC; o += NT) {
    const int j = o / TC, c = o - j * TC;
    if (c0 + c >= C) continue;
    T re = 0, im = 0;
    for (int k = 0; k < N; ++k) {
      const C2<T> v = slab[k * TC + c], e = Es[k * nt + j];
      re += v.x * e.x - v.y * e.y;
      im += v.x * e.y + v.y * e.x;
    }
    dstb[(long)j * C + c0 + c] = C2<T>{re, im};
  }
}

// CC[b][r][j] = scale Re sum_k Y[b][r][k] E[b][0][k][j]: the x stage, rows r =
// (tz, ty).  One CTA per (tile of ROWS rows, b).
template <typename T>
__global__ void __launch_bounds__(256)
k_idft_x(const C2<T> *__restrict__ Y, T *__restrict__ CC, const C2<T> *__restrict__ E, int N,
         int nt, int rows, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ROWS = 8;
  C2<T> *ys = reinterpret_cast<C2<T> *>(smem_raw);  // [ROWS][N]
  C2<T> *Es = ys + ROWS * N;                         // [N][nt]
  const long b = blockIdx.y;
  const int r0 = blockIdx.x * ROWS;
  const int tid = threadIdx.x, NT = blockDim.x;
  const C2<T> *yb = Y + b * (long)rows * N;
  for (int idx = tid; idx < ROWS * N; idx += NT) {
    const int r = idx / N;
    ys[idx] = r0 + r < rows ? yb[(long)r0 * N + idx] : C2<T>{T(0), T(0)};
  }
  const C2<T> *eb = E + (b * 3) * (long)N * nt;
  for (int idx = tid; idx < N * nt; idx += NT) Es[idx] = eb[idx];
  __syncthreads();
  for (int o = tid; o < ROWS * nt; o += NT) {
    const int r = o / nt, j = o - r * nt;
    if (r0 + r >= rows) continue;
    T re = 0;
    for (int k = 0; k < N; ++k) {
      const C2<T> v = ys[r * N + k], e = Es[k * nt + j];
      re += v.x * e.x - v.y * e.y;
    }
    CC[b * (long)rows * nt + (long)(r0 + r) * nt + j] = scale * re;
  }
}

// Maximum of each particle's nt^3 grid (value desc, index asc; NaN never
// wins): its grid point t, the value, flag bit 5 when an integer peak lies on
// the window's edge |t_a| = edge, and tau = R^T t.
template <typename T>
__global__ void __launch_bounds__(256)
k_cc_argmax(const T *__restrict__ CC, int nt, const double *__restrict__ org, int j0, int den,
            int edge, int flag_mode, const double *__restrict__ R, double *__restrict__ t_out,
            double *__restrict__ tau_out, double *__restrict__ cc_out, int *__restrict__ flags) {
  __shared__ T sv[256];
  __shared__ int si[256];
  const long b = blockIdx.x;
  const int n3 = nt * nt * nt, tid = threadIdx.x;
  const T *cb = CC + b * (long)n3;
  T bv = T(0);
  int bi = -1;
  for (int q = tid; q < n3; q += blockDim.x) {
    const T v = cb[q];
    if (v == v && (bi < 0 || v > bv)) { bv = v; bi = q; }  // q ascends: ties keep the first
  }
  sv[tid] = bv; si[tid] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      const T ov = sv[tid + s];
      const int oi = si[tid + s];
      if (oi >= 0 && (si[tid] < 0 || ov > sv[tid] || (ov == sv[tid] && oi < si[tid]))) {
        sv[tid] = ov; si[tid] = oi;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int q = si[0];
    double t[3];
    double v;
    if (q < 0) {
      t[0] = t[1] = t[2] = 0.0;
      v = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      const int jx = q % nt, jy = (q / nt) % nt, jz = q / (nt * nt);
      const int jj[3] = {jx, jy, jz};
      for (int a = 0; a < 3; ++a) t[a] = grid_t(org, b, a, jj[a], j0, den);
      v = (double)sv[0];
    }
    for (int a = 0; a < 3; ++a) t_out[3 * b + a] = t[a];
    if (cc_out) cc_out[b] = v;
    int fl = 0;
    if (edge > 0)
      for (int a = 0; a < 3; ++a)
        if (fabs(t[a]) == (double)edge) fl = 32;
    if (q < 0) fl |= 1;
    if (flag_mode == 1) flags[b] = fl;
    else if (flag_mode == 2) flags[b] |= fl;
    if (tau_out) {
      const double *r = R + 9 * b;
      for (int a = 0; a < 3; ++a) tau_out[3 * b + a] = r[a] * t[0] + r[3 + a] * t[1] + r[6 + a] * t[2];
    }
  }
}

static int fine_points(int upsample) { return 2 * (int)floor(0.75 * upsample) + 1; }

size_t shift_ws_bytes(const Plan &p, int B, int max_shift, int upsample, char *base, ShiftWs *w) {
  const size_t cs = p.fp64 ? 16 : 8, rs = p.fp64 ? 8 : 4;
  const long N = p.N, N2 = N * N, N3 = N2 * N;
  const int nw = 2 * max_shift + 1, nf = fine_points(upsample);
  const long nt = nw > nf ? nw : nf;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *r = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return r;
  };
  ShiftWs tmp;
  ShiftWs *o = w ? w : &tmp;
  o->Z = take(cs * (size_t)B * N3);
  o->Y1 = take(cs * (size_t)B * nt * N2);
  o->Y2 = take(cs * (size_t)B * nt * nt * N);
  o->E = take(cs * (size_t)B * 3 * N * nt);
  o->CC = take(rs * (size_t)B * nt * nt * nt);
  o->t0 = reinterpret_cast<double *>(take(sizeof(double) * 3 * (size_t)B));
  return off;
}

// the three partial inverse-DFT stages and the maximum, on one grid
template <typename T>
static cudaError_t idft_grid(const Plan &p, int B, int nt, const double *org, int j0, int den,
                             int edge, int flag_mode, const double *R, const ShiftWs &w,
                             double *t_out, double *tau_out, double *cc_out, int *flags,
                             cudaStream_t st) {
  const int N = p.N;
  const long N2 = (long)N * N;
  const long nE = (long)B * 3 * N * nt;
  k_idft_factors<T><<<(unsigned)((nE + 255) / 256), 256, 0, st>>>((C2<T> *)w.E, N, nt, B, org, j0, den);
  // z stage: X[b][kz][ky kx] -> Y1[b][tz][ky kx]
  const size_t cs = sizeof(C2<T>);
  int TC = 64;
  while (TC > 8 && cs * ((size_t)N * TC + (size_t)N * nt) > 96 * 1024) TC /= 2;
  size_t smem = cs * ((size_t)N * TC + (size_t)N * nt);
  cudaFuncSetAttribute(k_idft_mid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_idft_mid<T><<<dim3((unsigned)((N2 + TC - 1) / TC), B), 256, smem, st>>>(
      (const C2<T> *)w.Z, (C2<T> *)w.Y1, (const C2<T> *)w.E, N, nt, 1, N2, TC, 2);
  // y stage: Y1[b][tz][ky][kx] -> Y2[b][tz][ty][kx]
  int TCy = TC < N ? TC : N;
  k_idft_mid<T><<<dim3((unsigned)(nt * ((N + TCy - 1) / TCy)), B), 256, smem, st>>>(
      (const C2<T> *)w.Y1, (C2<T> *)w.Y2, (const C2<T> *)w.E, N, nt, nt, N, TCy, 1);
  // x stage: Y2[b][tz ty][kx] -> CC[b][tz ty][tx]
  const int rows = nt * nt;
  size_t smx = cs * (8 * (size_t)N + (size_t)N * nt);
  cudaFuncSetAttribute(k_idft_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx);
  k_idft_x<T><<<dim3((rows + 7) / 8, B), 256, smx, st>>>(
      (const C2<T> *)w.Y2, (T *)w.CC, (const C2<T> *)w.E, N, nt, rows, T(1.0 / ((double)N2 * N)));
  k_cc_argmax<T><<<B, 256, 0, st>>>((const T *)w.CC, nt, org, j0, den, edge, flag_mode, R, t_out,
                                    tau_out, cc_out, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_shift_search(const Plan &p, const float *f, const float *u, int B,
                                int max_shift, int upsample, const double *R, const ShiftWs &w,
                                double *t, double *tau, double *cc, int *flags, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int N = p.N;
  const long N2 = (long)N * N, N3 = N2 * N;
  FftDesc fd;
  fd.N = N;
  fd.npass = p.fft_npass;
  for (int q = 0; q < 16; ++q) fd.radix[q] = p.fft_radix[q];
  const size_t cs = sizeof(C2<T>);
  // lines per CTA: about 4096 elements (a whole 64 x 64 plane), at least 16
  // columns for the strided passes so their rows stay coalesced
  const int NB0 = N * N <= 4096 ? N : (4096 / N > 0 ? 4096 / N : 1);
  const int NB = N <= 64 ? N : (4096 / N > 16 ? 4096 / N : 16);
  size_t sm0 = cs * 2 * (size_t)NB0 * (N + 1), sm1 = cs * 2 * (size_t)NB * (N + 1);
  size_t smax = sm0 > sm1 ? sm0 : sm1;
  cudaFuncSetAttribute(k_fft_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
  C2<T> *Z = (C2<T> *)w.Z;
  const C2<T> *tw = (const C2<T> *)p.fft_tw;
  const T fwd = T(-1);
  k_fft_axis<T><<<dim3((unsigned)((N2 + NB0 - 1) / NB0), B), 256, sm0, st>>>(Z, f, u, 0, fd, tw, NB0, fwd);
  const unsigned tiles = (unsigned)(N * ((N + NB - 1) / NB));
  k_fft_axis<T><<<dim3(tiles, B), 256, sm1, st>>>(Z, nullptr, nullptr, 1, fd, tw, NB, fwd);
  k_fft_axis<T><<<dim3(tiles, B), 256, sm1, st>>>(Z, nullptr, nullptr, 2, fd, tw, NB, fwd);
  k_cross_spectrum<T><<<dim3((unsigned)((N3 + 255) / 256), B), 256, 0, st>>>(Z, N);
  cudaError_t e;
  // integer window [-m, m]^3
  const int nw = 2 * max_shift + 1;
  e = idft_grid<T>(p, B, nw, nullptr, -max_shift, 1, max_shift, 1, nullptr, w, w.t0,
                   nullptr, nullptr, flags, st);
  if (e != cudaSuccess) return e;
  // fine grid around the integer peak
  const int h = (int)floor(0.75 * upsample), nf = 2 * h + 1;
  return idft_grid<T>(p, B, nf, w.t0, -h, upsample, 0, 0, R, w, t, tau,
                      cc, flags, st);
}

template cudaError_t launch_shift_search<float>(const Plan &, const float *, const float *, int,
                                                int, int, const double *, const ShiftWs &,
                                                double *, double *, double *, int *, cudaStream_t);
template cudaError_t launch_shift_search<double>(const Plan &, const float *, const float *, int,
                                                 int, int, const double *, const ShiftWs &,
                                                 double *, double *, double *, int *, cudaStream_t);

}  // namespace matcha
