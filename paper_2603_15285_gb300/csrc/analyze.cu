// Steps a1+a2: shell sampling and spherical-harmonic analysis.
//
// The paper obtains ball-harmonic coefficients with a NUFFT (Section 1.1,
// Appendix A.1-A.2); this path samples each volume on the quadrature points of
// S radial shells instead (Gauss-Legendre in r, Gauss-Legendre in cos(theta),
// equispaced in phi) and analyses every shell:
//   F_m(s, j)  = sum_k f(r_s w_jk) exp(-i m phi_k)                 (phi DFT)
//   f_lm(r_s)  = sum_j w_j (2 pi / n_phi) Pbar_lm(x_j) F_m(s, j)    (Legendre)
// The shell-group kernel (k_analyze2) gives one CTA a volume and G shells: it
// samples the G * n_theta rings into shared memory (texture gathers where the
// batch allows), folds the real DFT (pairs k, n_phi - k) and runs the Legendre
// sums against the plan's table.  The ring-batched kernel (k_analyze) takes
// one shell per CTA a few rings at a time, for bandwidths whose shell does not
// fit in shared memory.
#include <stdlib.h>
#include <algorithm>
#include <type_traits>
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

// The rings are sampled and transformed RB at a time (the samples of RB
// rings, then their phi DFTs into F), so the shared memory holds F and RB
// rings rather than every sample of the shell: this kernel serves the
// bandwidths the shell-group kernel cannot hold (up to L_J = 100 in FP64).
template <typename T>
__global__ void __launch_bounds__(256)
k_analyze(const float *__restrict__ vols, int N, int S, int L, const double *__restrict__ rs,
          const double *__restrict__ xj, const T *__restrict__ ptabT, const T *__restrict__ phi_cs,
          T *__restrict__ out, int RB) {
  const int s = blockIdx.x;
  const long b = blockIdx.y;
  const int nt = L + 1, np = 2 * L + 2, nm = L + 1, nlm = (L + 1) * (L + 2) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *F = reinterpret_cast<T *>(smem_raw);  // [nt][nm] complex
  T *tw = F + 2 * nt * nm;                  // [np][2]
  T *smp = tw + 2 * np;                     // [RB][np]
  const float *vol = vols + b * N * N * N;
  const T r = (T)rs[s];
  const T c0 = (T)(0.5 * N);
  for (int k = threadIdx.x; k < 2 * np; k += blockDim.x) tw[k] = phi_cs[k];
  __syncthreads();

  const int NT = blockDim.x, half = np / 2;
  for (int jr = 0; jr < nt; jr += RB) {
    const int nr = min(RB, nt - jr), total = nr * np;
    for (int base = threadIdx.x; base < total; base += 2 * NT) {
      int id1 = base + NT;
      int j0 = base / np, k0 = base - j0 * np;
      int id1c = id1 < total ? id1 : base;
      int j1 = id1c / np, k1 = id1c - j1 * np;
      T x0 = (T)xj[jr + j0], x1 = (T)xj[jr + j1];
      T st0 = sqrt(max(T(1) - x0 * x0, T(0))), st1 = sqrt(max(T(1) - x1 * x1, T(0)));
      T v0 = trilinear<T>(vol, N, c0 + r * st0 * tw[2 * k0], c0 + r * st0 * tw[2 * k0 + 1], c0 + r * x0);
      T v1 = trilinear<T>(vol, N, c0 + r * st1 * tw[2 * k1], c0 + r * st1 * tw[2 * k1 + 1], c0 + r * x1);
      smp[base] = v0;
      if (id1 < total) smp[id1] = v1;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
      int jj = idx / nm, m = idx - jj * nm;
      const T *row = smp + jj * np;
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
      F[2 * ((jr + jj) * nm + m)] = re;
      F[2 * ((jr + jj) * nm + m) + 1] = im;
    }
    __syncthreads();
  }

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

// Shell-group kernel: one CTA per (volume, group of G shells).
//  1. trilinear samples from per-ring constants (points near or outside the
//     box edge take the bounds-checked path), folded on the fly into
//     SP_k = f_k + f_{np-k}, SM_k = f_k - f_{np-k}, k = 1..np/2-1;
//  2. the folded real DFT as two small matrix products
//       Re F_m = f_0 + (-1)^m f_{np/2} + sum_k SP_k cos(2 pi m k/np)
//       Im F_m = -sum_k SM_k sin(2 pi m k/np)
//     register-tiled 4 rings x 4 orders per thread;
//  3. the Legendre sums, one thread per (l, m) for all shells of the group.
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  typedef float4 type;
};
template <> struct Vec4<double> {
  struct type { double x, y, z, w; };
};

template <typename T>
__device__ __forceinline__ typename Vec4<T>::type ld4(const T *p) {
  return *reinterpret_cast<const typename Vec4<T>::type *>(p);
}
// (re, im) and (cos, sin) pairs move as one 8- or 16-byte shared access
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };
template <typename T>
__device__ __forceinline__ typename Vec2<T>::type ld2(const T *p) {
  return *reinterpret_cast<const typename Vec2<T>::type *>(p);
}
template <typename T>
__device__ __forceinline__ void st2(T *p, typename Vec2<T>::type v) {
  *reinterpret_cast<typename Vec2<T>::type *>(p) = v;
}
template <typename T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4]) {
  typename Vec4<T>::type q;
  q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3];
  *reinterpret_cast<typename Vec4<T>::type *>(p) = q;
}

// TEX: the four x-y corners of each plane of a trilinear cell come from one
// 2x2 texture gather on the 2-D view (x, z N + y) of the volume (texture
// views of runs of ta.vpt volumes); the gathered values are the voxels
// themselves (no filtering), so the samples are bit-identical to the
// eight-load path, and the gathers go through the texture pipe, which serves
// the 2x2 footprints faster than eight scattered loads.
constexpr int ANALYZE_THREADS = 192;
// samples whose texture gathers are in flight together (per thread): two
// keep the kernel within four CTAs per SM; four need 95 registers (three
// CTAs per SM) or spill under a four-CTA bound, and both measure slower
constexpr int GATHER_BATCH = 2;

template <typename T, int G, bool TEX>
__global__ void __launch_bounds__(ANALYZE_THREADS)
k_analyze2(const float *__restrict__ vols, int N, int S, int L,
           const double *__restrict__ rs, const double *__restrict__ xj, const T *__restrict__ phi_cs,
           const T *__restrict__ dcs, int Mp, int Qf, int Mq, const T *__restrict__ ptabT,
           const int *__restrict__ leg, const T *__restrict__ ring, T *__restrict__ out,
           const __grid_constant__ TexArgs ta) {
  constexpr int GB = GATHER_BATCH;
  const int s0 = blockIdx.x * G;
  const long b = blockIdx.y;
  const int Gs = G;  // the launcher picks G dividing S
  const int nt = L + 1, np = 2 * L + 2, half = np / 2, K1 = half - 1;
  const int nlm = (L + 1) * (L + 2) / 2;
  const int R = Gs * nt, Rp = (G * nt + 3) / 4 * 4;
  const int tid = threadIdx.x, NT = blockDim.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *SP = reinterpret_cast<T *>(smem_raw);  // [K1][Rp]
  T *SM = SP + K1 * Rp;                     // [K1][Rp]
  T *E0 = SM + K1 * Rp;                     // [Rp]  f_0
  T *EH = E0 + Rp;                          // [Rp]  f_{np/2}
  T *CS = EH + Rp;                          // [2][2][Qf][Mq] folded DFT table
  T *F = CS + 4 * Qf * Mq;                  // [Rp][Mp] complex
  T *RH = F + 2 * Rp * Mp;                  // [Rp] ring radius r_s sin(t_j)
  T *RZ = RH + Rp;                          // [Rp] ring height c0 + r_s cos(t_j)
  T *PH = RZ + Rp;                          // [np][2] cos, sin phi_k
  const float *vol = vols + b * N * N * N;
  const long NN = (long)N * N;

  for (int t = tid; t < 4 * Qf * Mq; t += NT) CS[t] = dcs[t];
  // per-ring constants from the plan: rho = r_s sin(t_j), z = c0 + r_s cos(t_j)
  const FastDiv dhalf(half);
  for (int r = tid; r < R; r += NT) {
    RH[r] = ring[2 * ((long)s0 * nt + r)];
    RZ[r] = ring[2 * ((long)s0 * nt + r) + 1];
  }
  for (int t = tid; t < 2 * np; t += NT) PH[t] = phi_cs[t];
  __syncthreads();
  const T c0 = (T)(0.5 * N);
  const T hi = (T)(N - 1);
  cudaTextureObject_t tob = 0;
  float yoff = 0.f;  // first row of this volume in its texture view
  if (TEX) {
    const int run = (int)(b / ta.vpt);
    tob = ta.t[run];
    yoff = (float)((b - (long)run * ta.vpt) * NN);
  }
  // trilinear combination of the two gathered planes (components: x (i, j+1),
  // y (i+1, j+1), z (i+1, j), w (i, j)) at cell offsets (tx, ty, tz)
  auto combine = [](const float4 &q0, const float4 &q1, T tx, T ty, T tz) -> T {
    const T v000 = (T)q0.w, v001 = (T)q0.z, v010 = (T)q0.x, v011 = (T)q0.y;
    const T v100 = (T)q1.w, v101 = (T)q1.z, v110 = (T)q1.x, v111 = (T)q1.y;
    T a00 = v000 + tx * (v001 - v000), a01 = v010 + tx * (v011 - v010);
    T a10 = v100 + tx * (v101 - v100), a11 = v110 + tx * (v111 - v110);
    T b0 = a00 + ty * (a01 - a00), b1 = a10 + ty * (a11 - a10);
    return b0 + tz * (b1 - b0);
  };
  // trilinear at (px, py, pz) by plain loads (the load path, and points the
  // texture path finds outside the box); corners clamped so that all eight
  // are in the box when the point is (the value is unchanged), bounds-checked
  // otherwise
  auto sample = [&](T px, T py, T pz) -> T {
    T fx = floor(px), fy = floor(py), fz = floor(pz);
    bool inside = px >= T(0) && py >= T(0) && pz >= T(0) && px <= hi && py <= hi && pz <= hi;
    if (inside) {
      int i = min((int)fx, N - 2), j = min((int)fy, N - 2), k = min((int)fz, N - 2);
      T tx = px - (T)i, ty = py - (T)j, tz = pz - (T)k;
      const float *v = vol + ((long)k * N + j) * N + i;
      const T v000 = (T)__ldg(v), v001 = (T)__ldg(v + 1), v010 = (T)__ldg(v + N),
              v011 = (T)__ldg(v + N + 1), v100 = (T)__ldg(v + NN), v101 = (T)__ldg(v + NN + 1),
              v110 = (T)__ldg(v + NN + N), v111 = (T)__ldg(v + NN + N + 1);
      T a00 = v000 + tx * (v001 - v000), a01 = v010 + tx * (v011 - v010);
      T a10 = v100 + tx * (v101 - v100), a11 = v110 + tx * (v111 - v110);
      T b0 = a00 + ty * (a01 - a00), b1 = a10 + ty * (a11 - a10);
      return b0 + tz * (b1 - b0);
    }
    int i3[3] = {(int)fx, (int)fy, (int)fz};
    T f3[3] = {px - fx, py - fy, pz - fz};
    T acc = 0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          int ii = i3[0] + dx, jj = i3[1] + dy, kk = i3[2] + dz;
          if (ii < 0 || jj < 0 || kk < 0 || ii >= N || jj >= N || kk >= N) continue;
          T wt = (dx ? f3[0] : T(1) - f3[0]) * (dy ? f3[1] : T(1) - f3[1]) * (dz ? f3[2] : T(1) - f3[2]);
          acc += wt * (T)__ldg(vol + ((long)kk * N + jj) * N + ii);
        }
    return acc;
  };
  // 1. samples: item (quad of rings r0..r0+3, kk), kk = 0..half-1, two
  //    samples per ring: kk = 0 -> phi index 0 and np/2 (into E0, EH); kk >= 1
  //    -> kk and np - kk (folded into SP, SM).  A quad's four values go out as
  //    one 16-byte store, so the lanes of a warp (consecutive kk, row stride
  //    Rp) write distinct banks; the padding rings r >= R get zeros.
  const int items = (Rp / 4) * half;
  for (int t = tid; t < items; t += NT) {
    const int q = dhalf.div(t), kk = t - q * half, r0 = 4 * q;
    const int ka = kk, kb = kk ? np - kk : half;
    const typename Vec2<T>::type pa = ld2(PH + 2 * ka), pb = ld2(PH + 2 * kb);
    T va[4], vb[4];
    if constexpr (TEX) {
      // the item's eight samples (a_0, b_0, a_1, b_1, ...) in batches of GB:
      // both gathers of every sample of a batch are issued before the first
      // is combined; a point outside the box (or of a padding ring) gathers
      // at the origin and then takes the bounds-checked path (or zero)
#pragma unroll
      for (int sq = 0; sq < 8; sq += GB) {
        float4 q0[GB], q1[GB];
        T ftx[GB], fty[GB], ftz[GB];
        bool in[GB];
#pragma unroll
        for (int v = 0; v < GB; ++v) {
          const int u = (sq + v) >> 1, r = r0 + u;
          const typename Vec2<T>::type pc = ((sq + v) & 1) ? pb : pa;
          const T rho = r < R ? RH[r] : T(0), pz = r < R ? RZ[r] : T(-1);
          const T px = c0 + rho * pc.x, py = c0 + rho * pc.y;
          in[v] = px >= T(0) && py >= T(0) && pz >= T(0) && px <= hi && py <= hi && pz <= hi;
          const int i = in[v] ? min((int)floor(px), N - 2) : 0;
          const int j = in[v] ? min((int)floor(py), N - 2) : 0;
          const int k = in[v] ? min((int)floor(pz), N - 2) : 0;
          ftx[v] = px - (T)i; fty[v] = py - (T)j; ftz[v] = pz - (T)k;
          const float tx0 = (float)i + 1.f, ty0 = yoff + (float)(k * N + j) + 1.f;
          q0[v] = tex2Dgather<float4>(tob, tx0, ty0, 0);
          q1[v] = tex2Dgather<float4>(tob, tx0, ty0 + (float)N, 0);
        }
#pragma unroll
        for (int v = 0; v < GB; ++v) {
          const int u = (sq + v) >> 1, r = r0 + u;
          T val = combine(q0[v], q1[v], ftx[v], fty[v], ftz[v]);
          if (!in[v]) {
            val = T(0);
            if (r < R) {
              const typename Vec2<T>::type pc = ((sq + v) & 1) ? pb : pa;
              const T rho = RH[r];
              val = sample(c0 + rho * pc.x, c0 + rho * pc.y, RZ[r]);
            }
          }
          if ((sq + v) & 1) vb[u] = val;
          else va[u] = val;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        va[u] = T(0); vb[u] = T(0);
        if (r < R) {
          const T rho = RH[r], pz = RZ[r];
          va[u] = sample(c0 + rho * pa.x, c0 + rho * pa.y, pz);
          vb[u] = sample(c0 + rho * pb.x, c0 + rho * pb.y, pz);
        }
      }
    }
    if (kk == 0) {
      st4(E0 + r0, va);
      st4(EH + r0, vb);
    } else {
      T sp[4], sm[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { sp[u] = va[u] + vb[u]; sm[u] = va[u] - vb[u]; }
      st4(SP + (kk - 1) * Rp + r0, sp);
      st4(SM + (kk - 1) * Rp + r0, sm);
    }
  }
  __syncthreads();
  // 2. phi DFT.  Fold the pairs (q, q') = (q, np/2 - q), q = 1..Qf, in place:
  //    row q-1 <- x_q + x_q', row q'-1 <- x_q - x_q' (a self-paired middle row,
  //    odd L, stays); even orders then read (SP+, SM-), odd orders (SP-, SM+).
  const FastDiv dRp(Rp);
  for (int t = tid; t < (K1 / 2) * Rp; t += NT) {
    int q = dRp.div(t) + 1, r = t - (q - 1) * Rp, q2 = K1 + 1 - q;
    T a = SP[(q - 1) * Rp + r], c = SP[(q2 - 1) * Rp + r];
    SP[(q - 1) * Rp + r] = a + c; SP[(q2 - 1) * Rp + r] = a - c;
    a = SM[(q - 1) * Rp + r]; c = SM[(q2 - 1) * Rp + r];
    SM[(q - 1) * Rp + r] = a + c; SM[(q2 - 1) * Rp + r] = a - c;
  }
  __syncthreads();
  //    4 x 4 tiles of (ring, 4 orders of one parity)
  {
    const int tr = Rp / 4, tc = Mq / 4;
    const FastDiv dtc(2 * tc);
    for (int t = tid; t < tr * 2 * tc; t += NT) {
      int tq = dtc.div(t), rest = t - tq * 2 * tc;
      int par = rest >= tc ? 1 : 0, c0 = (rest - par * tc) * 4, r0 = tq * 4;
      const T *cst = CS + (2 * par) * Qf * Mq + c0, *snt = CS + (2 * par + 1) * Qf * Mq + c0;
      T re[4][4], im[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) { re[u][v] = 0; im[u][v] = 0; }
      for (int q = 1; q <= Qf; ++q) {
        const int rlo = q - 1, rhi = K1 - q;  // rows of x_q + x_q' and x_q - x_q'
        typename Vec4<T>::type sp = ld4(SP + (par ? rhi : rlo) * Rp + r0);
        typename Vec4<T>::type sm = ld4(SM + (par ? rlo : rhi) * Rp + r0);
        typename Vec4<T>::type c = ld4(cst + (q - 1) * Mq), sn = ld4(snt + (q - 1) * Mq);
        T spv[4] = {sp.x, sp.y, sp.z, sp.w}, smv[4] = {sm.x, sm.y, sm.z, sm.w};
        T cv[4] = {c.x, c.y, c.z, c.w}, sv[4] = {sn.x, sn.y, sn.z, sn.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            re[u][v] = fma(spv[u], cv[v], re[u][v]);
            im[u][v] = fma(-smv[u], sv[v], im[u][v]);
          }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        T e0 = E0[r0 + u], eh = EH[r0 + u];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          int m = 2 * (c0 + v) + par;
          if (m <= L) {
            typename Vec2<T>::type o;
            o.x = re[u][v] + e0 + (par ? -eh : eh);
            o.y = im[u][v];
            st2(F + 2 * ((r0 + u) * Mp + m), o);
          }
        }
      }
    }
  }
  __syncthreads();
  // 3. Legendre over the symmetric Gauss nodes: x_{nt-1-j} = -x_j and
  //    Pbar_lm(-x) = (-1)^(l+m) Pbar_lm(x), so rows j and nt-1-j fold to
  //    F(j) + F(nt-1-j) (even l+m, kept in row j) and F(j) - F(nt-1-j) (odd,
  //    in row nt-1-j); the middle node of odd nt serves both.
  const int Jh = (nt + 1) / 2;
  const FastDiv dL1(L + 1), dnh(nt / 2 > 0 ? nt / 2 : 1);
  for (int t = tid; t < Gs * (nt / 2) * (L + 1); t += NT) {
    int gj = dL1.div(t), m = t - gj * (L + 1), g = dnh.div(gj), j = gj - g * (nt / 2);
    T *fa = F + 2 * ((g * nt + j) * Mp + m), *fb = F + 2 * ((g * nt + nt - 1 - j) * Mp + m);
    const typename Vec2<T>::type a = ld2(fa), bq = ld2(fb);
    typename Vec2<T>::type sa, sb;
    sa.x = a.x + bq.x; sa.y = a.y + bq.y;
    sb.x = a.x - bq.x; sb.y = a.y - bq.y;
    st2(fa, sa);
    st2(fb, sb);
  }
  __syncthreads();
  //    Items in the plan's Legendre order (runs of equal m and parity of
  //    l + m): the lanes of a run read the same F value, and the table
  //    (ptabT: columns in item order) is read contiguously.
  for (int t = tid; t < nlm; t += NT) {
    const int lp = leg[t], l = lp >> 16, m = lp & 0xffff, lm = l * (l + 1) / 2 + m;
    const bool odd = (l + m) & 1;
    T ar[G], ai[G];
#pragma unroll
    for (int g = 0; g < G; ++g) { ar[g] = 0; ai[g] = 0; }
    for (int j = 0; j < Jh; ++j) {
      T w = ptabT[(long)j * nlm + t];
      const T *fj = F + 2 * ((odd ? nt - 1 - j : j) * Mp + m);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const typename Vec2<T>::type f = ld2(fj + 2 * g * nt * Mp);
        ar[g] = fma(w, f.x, ar[g]);
        ai[g] = fma(w, f.y, ai[g]);
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      T *o = out + 2 * ((b * S + s0 + g) * (long)nlm + lm);
      o[0] = ar[g];
      o[1] = ai[g];
    }
  }
}

// Texture views for a batch (looked up in, or added to, the plan's cache).
// False when the batch does not qualify (row pitch or base alignment, view
// height, more than TEX_MAX views) or when a new view would have to be made
// while `st` is being captured into a graph; the kernel then reads the
// volumes with plain loads.  Evicting a view synchronises the device first
// (a kernel still queued may use it).  The caller holds p.tex_mu through the
// launch that uses the views.
bool texture_views(const Plan &p, const float *vols, int B, cudaStream_t st, TexArgs &ta) {
  ta.vpt = 1;
  int dev = 0, pitch_al = 0, tex_al = 0, max_w = 0, max_h = 0, max_pitch = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&pitch_al, cudaDevAttrTexturePitchAlignment, dev);
  cudaDeviceGetAttribute(&tex_al, cudaDevAttrTextureAlignment, dev);
  cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture2DLinearWidth, dev);
  cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxTexture2DLinearHeight, dev);
  cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxTexture2DLinearPitch, dev);
  const long N = p.N, NN = N * N, pitch = 4 * N, vbytes = 4 * N * NN;
  if (pitch_al <= 0 || tex_al <= 0 || pitch % pitch_al || pitch > max_pitch || N > max_w ||
      NN > max_h || vbytes % tex_al || reinterpret_cast<uintptr_t>(vols) % tex_al)
    return false;
  const int vpt = (int)std::min<long>(B, max_h / NN), ntex = (B + vpt - 1) / vpt;
  if (ntex > TEX_MAX) return false;
  TexSet *hit = nullptr, *slot = nullptr;
  for (auto &t : p.texsets) {
    if (t.ntex && t.base == vols && t.B == B && t.vpt == vpt) hit = &t;
    if (!slot || !t.ntex || (slot->ntex && t.used < slot->used)) slot = &t;
  }
  if (!hit) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return false;
    if (slot->ntex) {
      cudaDeviceSynchronize();
      for (int i = 0; i < slot->ntex; ++i) cudaDestroyTextureObject(slot->t[i]);
      slot->ntex = 0;
    }
    for (int r = 0; r < ntex; ++r) {
      cudaResourceDesc rd = {};
      rd.resType = cudaResourceTypePitch2D;
      rd.res.pitch2D.devPtr = const_cast<float *>(vols) + (size_t)r * vpt * N * NN;
      rd.res.pitch2D.desc = cudaCreateChannelDesc<float>();
      rd.res.pitch2D.width = N;
      rd.res.pitch2D.height = (size_t)std::min(vpt, B - r * vpt) * NN;
      rd.res.pitch2D.pitchInBytes = pitch;
      cudaTextureDesc td = {};
      td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
      td.filterMode = cudaFilterModePoint;
      td.readMode = cudaReadModeElementType;
      td.normalizedCoords = 0;
      if (cudaCreateTextureObject(&slot->t[r], &rd, &td, nullptr) != cudaSuccess) {
        for (int i = 0; i < r; ++i) cudaDestroyTextureObject(slot->t[i]);
        cudaGetLastError();
        return false;
      }
    }
    slot->base = vols; slot->B = B; slot->vpt = vpt; slot->ntex = ntex;
    hit = slot;
  }
  hit->used = ++p.tex_clock;
  for (int i = 0; i < hit->ntex; ++i) ta.t[i] = hit->t[i];
  ta.vpt = hit->vpt;
  return true;
}

void destroy_texsets(Plan &p) {
  for (auto &t : p.texsets) {
    for (int i = 0; i < t.ntex; ++i) cudaDestroyTextureObject(t.t[i]);
    t.ntex = 0;
  }
}

template <typename T>
size_t analyze2_smem(const Plan &p, int G) {
  int K1 = p.np / 2 - 1, Rp = (G * p.nt + 3) / 4 * 4;
  return sizeof(T) * (2 * (size_t)K1 * Rp + 4 * (size_t)Rp + 4 * (size_t)p.Qf * p.Mq +
                      2 * (size_t)Rp * p.Mp + 2 * (size_t)p.np);
}

template <typename T>
cudaError_t launch_analyze(const Plan &p, const float *vols, int B, T *coef, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  {
    // shells per CTA: a divisor of S in {8, 4, 2, 1} whose shared memory fits;
    // 2 unless the plan was autotuned (matcha_plan_autotune)
    int G = p.tune_shells > 0 ? p.tune_shells : 2;
    G = G >= 8 ? 8 : G >= 4 ? 4 : G >= 2 ? 2 : 1;
    while (G > 1 && (p.S % G != 0 || analyze2_smem<T>(p, G) > 100 * 1024)) G >>= 1;
    size_t smem = analyze2_smem<T>(p, G);
    if (smem <= 200 * 1024) {
      std::lock_guard<std::mutex> lock(p.tex_mu);
      TexArgs ta;
      const bool tex = texture_views(p, vols, B, st, ta);
      auto pick = [&](auto tag) {
        constexpr bool X = decltype(tag)::value;
        return G == 8 ? k_analyze2<T, 8, X> : G == 4 ? k_analyze2<T, 4, X>
             : G == 2 ? k_analyze2<T, 2, X> : k_analyze2<T, 1, X>;
      };
      auto kern = tex ? pick(std::true_type{}) : pick(std::false_type{});
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      // 192 threads: six warps per CTA keep four CTAs resident per SM
      // (measured 1.27 ms per 1,024 batch64 particles against 1.41 with 256
      // threads and 1.59 with 128)
      kern<<<dim3(p.S / G, B), ANALYZE_THREADS, smem, st>>>(vols, p.N, p.S, p.LJ, p.rs, p.xj,
                                                (const T *)p.phi_cs, (const T *)p.dft_cs, p.Mp,
                                                p.Qf, p.Mq, (const T *)p.ptab_leg, p.leg_lm,
                                                (const T *)p.ring,
                                                coef, ta);
      return cudaGetLastError();
    }
  }
  // rings per batch: as many as fit next to F (all of them when they do)
  const size_t fixed = 2 * (size_t)p.nt * (p.LJ + 1) + 2 * (size_t)p.np;
  int RB = p.nt;
  while (RB > 1 && sizeof(T) * (fixed + (size_t)RB * p.np) > 220 * 1024) RB = (RB + 1) / 2;
  size_t smem = sizeof(T) * (fixed + (size_t)RB * p.np);
  if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
  cudaFuncSetAttribute(k_analyze<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_analyze<T><<<dim3(p.S, B), 256, smem, st>>>(vols, p.N, p.S, p.LJ, p.rs, p.xj, (const T *)p.ptab,
                                                 (const T *)p.phi_cs, coef, RB);
  return cudaGetLastError();
}

bool analyze_shells_ok(const Plan &p, int G) {
  if (G != 1 && G != 2 && G != 4 && G != 8) return false;
  if (p.S % G) return false;
  return p.fp64 ? analyze2_smem<double>(p, G) <= 100 * 1024 : analyze2_smem<float>(p, G) <= 100 * 1024;
}

template cudaError_t launch_analyze<float>(const Plan &, const float *, int, float *, cudaStream_t);
template cudaError_t launch_analyze<double>(const Plan &, const float *, int, double *, cudaStream_t);

}  // namespace matcha
