// Steps a4+a5: the SOFFT initialisation (Section 2.3; Algorithm 1, steps 1-2).
//
// C_{L0} on the equiangular grid alpha_i = 2 pi i/n, beta_k = pi(2k+1)/(2n),
// gamma_j = 2 pi j/n, n = 2K(L0+1), is evaluated as the inverse SO(3) Fourier
// transform of Kostelec and Rockmore:
//   S_mn(beta_k)   = sum_{l=max(|m|,|n|)}^{L0} c^l_{mn} d^l_{mn}(beta_k)   (beta transform)
//   C(a_i,b_k,g_j) = Re sum_{m,n} S_mn(beta_k) e^{i(m a_i + n g_j)}       (2-D DFT)
// For real volumes S_{-m,-n} = conj(S_mn), so the alpha sum folds to
// m >= 0.
//
// Candidates: a grid point is a local maximum when it precedes all 26
// neighbours in the order (value desc, index asc), alpha and gamma wrapping
// and beta neighbours outside the grid skipped; the P strongest local maxima
// in that order are kept.
//
// Kernels (the launcher picks one by plan and tuning; all give the same
// candidates):
//   k_soft_grid + k_topk  grids too large for shared memory: one CTA per
//                         (beta_k, particle) writes the grid, then one CTA per
//                         particle compacts its local maxima and selects P of
//                         them by block-wide argmax rounds;
//   k_soft_fused, k_soft_stream, k_soft_chunk
//                         one CTA per particle, the grid kept on chip (whole,
//                         streamed by beta slice, or in passes of beta
//                         slices with a ring of two neighbour slices);
//   k_soft_warps          the chunked passes with a warp per beta slice;
//   k_soft_tile           the chunked passes register-tiled for L0 = 8,
//                         K = 2 in 32-bit plans (the bench configuration).
#include <algorithm>
#include <float.h>
#include <limits.h>
#include "internal.cuh"

namespace matcha {

template <typename T>
__global__ void __launch_bounds__(256)
k_soft_grid(const T *__restrict__ c, long nc, int L0, int ns, const int *__restrict__ pair_base,
            const T *__restrict__ soft_d, const int *__restrict__ pair_off0, long nc0,
            const T *__restrict__ tw, T *__restrict__ grid) {
  const int k = blockIdx.x;
  const long b = blockIdx.y;
  const int W = 2 * L0 + 1, np0 = (L0 + 1) * (L0 + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Sg = reinterpret_cast<T *>(smem_raw);  // [W][W] complex, index (m+L0)*W + n+L0
  T *G = Sg + 2 * W * W;                     // [L0+1][ns] complex
  const T *cb = c + 4 * b * nc;
  const T *dk = soft_d + (long)k * nc0;
  for (int q = threadIdx.x; q < np0; q += blockDim.x) {
    int m = isqrt_floor(q), n = q - m * m - m;
    const T *cp = cb + pair_base[q];
    const T *dp = dk + pair_off0[q];
    T ar = 0, ai = 0, br = 0, bi = 0;
    for (int l = m; l <= L0; ++l) {
      T d = dp[l - m];
      const T *e = cp + 8 * (l - m);
      ar = fma(e[0], d, ar); ai = fma(e[2], d, ai);
      br = fma(e[4], d, br); bi = fma(e[6], d, bi);
    }
    if ((m - n) & 1) { br = -br; bi = -bi; }  // d^l_nm = (-1)^{m-n} d^l_mn
    auto put = [&](int a, int bb, T re, T im) {
      int i = (a + L0) * W + (bb + L0);
      Sg[2 * i] = re; Sg[2 * i + 1] = im;
    };
    put(m, n, ar, ai);
    if (q != 0) put(-m, -n, ar, -ai);
    if (n != m && n != -m) { put(n, m, br, bi); put(-n, -m, br, -bi); }
  }
  __syncthreads();
  // G_m(j) = sum_n S_mn e^{i n g_j}, m = 0..L0; the twiddle index n j mod ns
  // advances by j per term (no integer division in the loop)
  for (int idx = threadIdx.x; idx < (L0 + 1) * ns; idx += blockDim.x) {
    int m = idx / ns, j = idx - m * ns;
    T re = 0, im = 0;
    const T *row = Sg + 2 * (m + L0) * W;
    int t = (int)(((long)(ns - j) * L0) % ns);  // (-L0 j) mod ns
    for (int n = 0; n < W; ++n) {
      T cr = tw[2 * t], ci = tw[2 * t + 1];
      T sr = row[2 * n], si = row[2 * n + 1];
      re += sr * cr - si * ci;
      im += sr * ci + si * cr;
      t += j;
      if (t >= ns) t -= ns;
    }
    G[2 * idx] = re;
    G[2 * idx + 1] = im;
  }
  __syncthreads();
  // C(i, k, j) = Re G_0(j) + 2 Re sum_{m>=1} G_m(j) e^{i m a_i}; four alpha
  // rows per thread share each G_m(j) load
  T *gb = grid + b * (long)ns * ns * ns;
  const int ni4 = (ns + 3) / 4;
  for (int idx = threadIdx.x; idx < ni4 * ns; idx += blockDim.x) {
    const int i0 = 4 * (idx / ns), j = idx - (idx / ns) * ns;
    T acc[4] = {0, 0, 0, 0};
    int t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) t[u] = i0 + u < ns ? i0 + u : 0;  // m i mod ns at m = 1
    for (int m = 1; m <= L0; ++m) {
      const T gr = G[2 * (m * ns + j)], gi = G[2 * (m * ns + j) + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[u] += gr * tw[2 * t[u]] - gi * tw[2 * t[u] + 1];
        t[u] += i0 + u;
        if (t[u] >= ns) t[u] -= ns;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < ns) gb[((long)(i0 + u) * ns + k) * ns + j] = G[2 * j] + 2 * acc[u];
  }
}

// max(a, b) that returns NaN when either is NaN
__device__ __forceinline__ float nan_max(float a, float b) {
  float d;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ double nan_max(double a, double b) {
  return (a != a || a > b) ? a : b;
}

template <typename T>
__device__ __forceinline__ bool precedes(T va, int ia, T vb, int ib) {
  return va > vb || (va == vb && ia < ib);
}

constexpr int TOPK_THREADS = 1024;

// Top-P local maxima of a materialised grid, one CTA per particle.  A point is
// a local maximum when it precedes each of its 26 neighbours in the order
// (value desc, index asc), alpha and gamma wrapping and beta neighbours
// outside the grid skipped; NaN is never one.  One warp per grid row (alpha
// i, beta k), lanes along gamma, so every neighbour load is coalesced; the
// point's own row first, each lane stopping at its first failure.  Each warp
// keeps the best P_max maxima it has seen as a sorted list distributed over
// its lanes (lane r holds rank r), inserting a new maximum only when it
// precedes the list's last entry; the warp lists are merged at the end.  All
// maxima are counted, for n_cand.
template <typename T>
__global__ void __launch_bounds__(TOPK_THREADS)
k_topk(const T *__restrict__ grid, int ns, int P_max, const int *__restrict__ P_per,
       int *__restrict__ idx_out, double *__restrict__ euler_out, double *__restrict__ score_out,
       int *__restrict__ n_cand_out) {
  const long b = blockIdx.x;
  const int tot = ns * ns * ns;
  const T *g = grid + b * (long)tot;
  constexpr int NW = TOPK_THREADS / 32;
  __shared__ int cnt;
  __shared__ T lv[NW * 32];
  __shared__ int li[NW * 32];
  __shared__ T red_v[NW];
  __shared__ int red_i[NW];
  __shared__ T prev_v;
  __shared__ int prev_i;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T wv = T(0);
  int wi = INT_MAX;  // this lane's rank of the warp list (INT_MAX: empty)
  int found = 0;
  for (int ik = warp; ik < ns * ns; ik += NW) {
    const int i = ik / ns, k = ik - i * ns;
    const int im = i == 0 ? ns - 1 : i - 1, ip = i == ns - 1 ? 0 : i + 1;
    const int base = (i * ns + k) * ns;
    // four 32-point chunks of the row at once: four independent load chains
    for (int j00 = 0; j00 < ns; j00 += 128) {
      bool ok[4];
      T v[4];
      int jj[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        jj[c] = j00 + 32 * c + lane;
        ok[c] = jj[c] < ns;
        v[c] = ok[c] ? g[base + jj[c]] : T(0);
        ok[c] = ok[c] && v[c] == v[c];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = jj[c], p = base + j;
        const int jm = j == 0 ? ns - 1 : j - 1, jp = j >= ns - 1 ? 0 : j + 1;
        if (ok[c]) ok[c] = precedes(v[c], p, g[base + jm], base + jm) && precedes(v[c], p, g[base + jp], base + jp);
      }
#pragma unroll
      for (int di = 0; di < 3; ++di) {
        const int ii = di == 0 ? im : (di == 1 ? i : ip);
#pragma unroll
        for (int dk = -1; dk <= 1; ++dk) {
          const int kk = k + dk;
          if (kk < 0 || kk >= ns || (di == 1 && dk == 0)) continue;
          const int rb = (ii * ns + kk) * ns;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (!ok[c]) continue;
            const int j = jj[c], p = base + j;
            const int jm = j == 0 ? ns - 1 : j - 1, jp = j >= ns - 1 ? 0 : j + 1;
            ok[c] = precedes(v[c], p, g[rb + j], rb + j) && precedes(v[c], p, g[rb + jm], rb + jm) &&
                    precedes(v[c], p, g[rb + jp], rb + jp);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        found += ok[c];
        const int p = base + jj[c];
        unsigned m = __ballot_sync(0xffffffffu, ok[c]);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const T cv = __shfl_sync(0xffffffffu, v[c], src);
          const int ci = __shfl_sync(0xffffffffu, p, src);
          const bool before = lane < P_max && wi != INT_MAX && precedes(wv, wi, cv, ci);
          const int pos = __popc(__ballot_sync(0xffffffffu, before));
          const T uv = __shfl_up_sync(0xffffffffu, wv, 1);
          const int ui = __shfl_up_sync(0xffffffffu, wi, 1);
          if (pos < P_max) {
            if (lane > pos && lane < P_max) { wv = uv; wi = ui; }
            if (lane == pos) { wv = cv; wi = ci; }
          }
        }
      }
    }
  }
  atomicAdd(&cnt, found);
  lv[warp * 32 + lane] = wv;
  li[warp * 32 + lane] = lane < P_max ? wi : INT_MAX;
  __syncthreads();
  const int n_max = cnt;
  int Pb = P_per ? min(P_per[b], P_max) : P_max;
  if (Pb < 0) Pb = 0;
  const int kept = min(Pb, n_max);
  // merge: rank r is the best entry of the warp lists that follows rank r-1
  for (int r = 0; r < kept; ++r) {
    const bool have_prev = r > 0;
    const T pv = have_prev ? prev_v : T(0);
    const int pi = have_prev ? prev_i : 0;
    T bv = T(0);
    int bi = INT_MAX;
    for (int t = threadIdx.x; t < NW * 32; t += blockDim.x) {
      const T v = lv[t];
      const int i = li[t];
      if (i == INT_MAX || (have_prev && !precedes(pv, pi, v, i))) continue;
      if (bi == INT_MAX || precedes(v, i, bv, bi)) { bv = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi != INT_MAX && (bi == INT_MAX || precedes(ov, oi, bv, bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T v = red_v[0];
      int i = red_i[0];
      for (int w = 1; w < NW; ++w)
        if (red_i[w] != INT_MAX && (i == INT_MAX || precedes(red_v[w], red_i[w], v, i))) {
          v = red_v[w]; i = red_i[w];
        }
      prev_v = v;
      prev_i = i;
      long o = b * P_max + r;
      idx_out[o] = i;
      score_out[o] = (double)v;
      int ia = i / (ns * ns), kb = (i / ns) % ns, jg = i % ns;
      euler_out[3 * o] = 2.0 * M_PI * ia / ns;
      euler_out[3 * o + 1] = M_PI * (2.0 * kb + 1.0) / (2.0 * ns);
      euler_out[3 * o + 2] = 2.0 * M_PI * jg / ns;
    }
    __syncthreads();
  }
  for (int r = kept + threadIdx.x; r < P_max; r += blockDim.x) {
    long o = b * P_max + r;
    idx_out[o] = -1;
    score_out[o] = __longlong_as_double(0x7ff8000000000000LL);
    euler_out[3 * o] = euler_out[3 * o + 1] = euler_out[3 * o + 2] = 0.0;
  }
  if (threadIdx.x == 0) n_cand_out[b] = kept;
}

// Fused variant for grids that fit in shared memory (FP32, n^3 * 4 bytes plus
// work space <= 227 KB): one CTA per particle computes the grid slice by slice
// (KB beta values at a time) into shared memory, optionally copies it out,
// tests local maxima against shared memory (face neighbours first, the
// cheapest rejection) and selects the top P like k_topk.
constexpr int FUSED_THREADS = 1024;
constexpr int FUSED_KB = 4;

__device__ __forceinline__ bool is_local_max_smem(const float *g, int ns, int p) {
  int i = p / (ns * ns), k = (p / ns) % ns, j = p % ns;
  float v = g[p];
  if (v != v) return false;
  int im = i == 0 ? ns - 1 : i - 1, ip = i == ns - 1 ? 0 : i + 1;
  int jm = j == 0 ? ns - 1 : j - 1, jp = j == ns - 1 ? 0 : j + 1;
  // face neighbours first
  {
    int q;
    q = (im * ns + k) * ns + j; if (!precedes(v, p, g[q], q)) return false;
    q = (ip * ns + k) * ns + j; if (!precedes(v, p, g[q], q)) return false;
    q = (i * ns + k) * ns + jm; if (!precedes(v, p, g[q], q)) return false;
    q = (i * ns + k) * ns + jp; if (!precedes(v, p, g[q], q)) return false;
    if (k > 0) { q = (i * ns + k - 1) * ns + j; if (!precedes(v, p, g[q], q)) return false; }
    if (k < ns - 1) { q = (i * ns + k + 1) * ns + j; if (!precedes(v, p, g[q], q)) return false; }
  }
  const int is[3] = {im, i, ip}, js[3] = {jm, j, jp};
  for (int a = 0; a < 3; ++a)
    for (int dk = -1; dk <= 1; ++dk) {
      int kk = k + dk;
      if (kk < 0 || kk >= ns) continue;
      for (int c = 0; c < 3; ++c) {
        int nz = (a != 1) + (dk != 0) + (c != 1);
        if (nz < 2) continue;  // the centre and the face neighbours are done
        int q = (is[a] * ns + kk) * ns + js[c];
        if (!precedes(v, p, g[q], q)) return false;
      }
    }
  return true;
}

__global__ void __launch_bounds__(FUSED_THREADS)
k_soft_fused(const float *__restrict__ c, long nc, int L0, int ns, const int *__restrict__ pair_base,
             const float *__restrict__ soft_d, const int *__restrict__ pair_off0, long nc0,
             const float *__restrict__ tw, int P_max, const int *__restrict__ P_per,
             float *__restrict__ grid_out, int *__restrict__ idx_out,
             double *__restrict__ euler_out, double *__restrict__ score_out,
             int *__restrict__ n_cand_out) {
  const long b = blockIdx.x;
  const int W = 2 * L0 + 1, np0 = (L0 + 1) * (L0 + 1), tot = ns * ns * ns;
  const int tid = threadIdx.x, NT = blockDim.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *g = reinterpret_cast<float *>(smem_raw);          // [ns^3]
  float *Sg = g + tot;                                       // [KB][W*W] complex
  float *G = Sg + 2 * FUSED_KB * W * W;                      // [KB][(L0+1)*ns] complex
  const float *cb = c + 4 * b * nc;
  for (int k0 = 0; k0 < ns; k0 += FUSED_KB) {
    for (int t = tid; t < FUSED_KB * np0; t += NT) {
      int kk = t / np0, q = t - kk * np0, k = k0 + kk;
      if (k >= ns) continue;
      int m = isqrt_floor(q), n = q - m * m - m;
      const float *cp = cb + pair_base[q];
      const float *dp = soft_d + (long)k * nc0 + pair_off0[q];
      float ar = 0, ai = 0, br = 0, bi = 0;
      for (int l = m; l <= L0; ++l) {
        float d = dp[l - m];
        const float *e = cp + 8 * (l - m);
        ar = fmaf(e[0], d, ar); ai = fmaf(e[2], d, ai);
        br = fmaf(e[4], d, br); bi = fmaf(e[6], d, bi);
      }
      if ((m - n) & 1) { br = -br; bi = -bi; }
      float *S = Sg + 2 * kk * W * W;
      int i0 = (m + L0) * W + (n + L0);
      S[2 * i0] = ar; S[2 * i0 + 1] = ai;
      if (q != 0) { int i1 = (-m + L0) * W + (-n + L0); S[2 * i1] = ar; S[2 * i1 + 1] = -ai; }
      if (n != m && n != -m) {
        int i2 = (n + L0) * W + (m + L0), i3 = (-n + L0) * W + (-m + L0);
        S[2 * i2] = br; S[2 * i2 + 1] = bi;
        S[2 * i3] = br; S[2 * i3 + 1] = -bi;
      }
    }
    __syncthreads();
    const int nG = (L0 + 1) * ns;
    for (int t = tid; t < FUSED_KB * nG; t += NT) {
      int kk = t / nG, r = t - kk * nG;
      if (k0 + kk >= ns) continue;
      int m = r / ns, j = r - m * ns;
      const float *row = Sg + 2 * kk * W * W + 2 * (m + L0) * W;
      float re = 0, im = 0;
      int tt = (int)(((long)(-L0) * j) % ns);
      if (tt < 0) tt += ns;
      for (int n = -L0; n <= L0; ++n) {
        float cr = tw[2 * tt], ci = tw[2 * tt + 1];
        float sr = row[2 * (n + L0)], si = row[2 * (n + L0) + 1];
        re += sr * cr - si * ci;
        im += sr * ci + si * cr;
        tt += j; if (tt >= ns) tt -= ns;
      }
      float *Gk = G + 2 * kk * nG;
      Gk[2 * r] = re; Gk[2 * r + 1] = im;
    }
    __syncthreads();
    for (int t = tid; t < FUSED_KB * ns * ns; t += NT) {
      int kk = t / (ns * ns), r = t - kk * ns * ns, k = k0 + kk;
      if (k >= ns) continue;
      int i = r / ns, j = r - i * ns;
      const float *Gk = G + 2 * kk * nG;
      float acc = 0;
      int tt = i;
      for (int m = 1; m <= L0; ++m) {
        float gr = Gk[2 * (m * ns + j)], gi = Gk[2 * (m * ns + j) + 1];
        acc += gr * tw[2 * tt] - gi * tw[2 * tt + 1];
        tt += i; if (tt >= ns) tt -= ns;
      }
      g[((long)i * ns + k) * ns + j] = Gk[2 * j] + 2 * acc;
    }
    __syncthreads();
  }
  if (grid_out) {
    float *go = grid_out + b * (long)tot;
    for (int t = tid; t < tot; t += NT) go[t] = g[t];
  }
  // candidates: reuse the work space after the grid
  __shared__ int cnt;
  __shared__ float red_v[FUSED_THREADS / 32];
  __shared__ int red_i[FUSED_THREADS / 32];
  __shared__ float prev_v;
  __shared__ int prev_i;
  float *lv = Sg;
  int *li = reinterpret_cast<int *>(Sg) + (FUSED_KB * W * W + FUSED_KB * (L0 + 1) * ns);
  const int cap = FUSED_KB * W * W + FUSED_KB * (L0 + 1) * ns;  // entries of each array
  if (tid == 0) cnt = 0;
  __syncthreads();
  for (int p = tid; p < tot; p += NT) {
    if (is_local_max_smem(g, ns, p)) {
      int pos = atomicAdd(&cnt, 1);
      if (pos < cap) { lv[pos] = g[p]; li[pos] = p; }
    }
  }
  __syncthreads();
  const int n_max = cnt;
  const bool listed = n_max <= cap;
  int Pb = P_per ? min(P_per[b], P_max) : P_max;
  if (Pb < 0) Pb = 0;
  const int kept = min(Pb, n_max);
  const int lane = tid & 31, warp = tid >> 5;
  for (int r = 0; r < kept; ++r) {
    float bv = -INFINITY;
    int bi = INT_MAX;
    bool have_prev = r > 0;
    float pv = have_prev ? prev_v : 0.f;
    int pi = have_prev ? prev_i : 0;
    if (listed) {
      for (int t = tid; t < n_max; t += NT) {
        float v = lv[t];
        int i = li[t];
        if (have_prev && !precedes(pv, pi, v, i)) continue;
        if (bi == INT_MAX || precedes(v, i, bv, bi)) { bv = v; bi = i; }
      }
    } else {
      for (int p = tid; p < tot; p += NT) {
        float v = g[p];
        if (have_prev && !precedes(pv, pi, v, p)) continue;
        if (bi != INT_MAX && !precedes(v, p, bv, bi)) continue;
        if (!is_local_max_smem(g, ns, p)) continue;
        bv = v; bi = p;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi != INT_MAX && (bi == INT_MAX || precedes(ov, oi, bv, bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      float v = red_v[0];
      int i = red_i[0];
      for (int w = 1; w < NT / 32; ++w)
        if (red_i[w] != INT_MAX && (i == INT_MAX || precedes(red_v[w], red_i[w], v, i))) {
          v = red_v[w]; i = red_i[w];
        }
      prev_v = v;
      prev_i = i;
      long o = b * P_max + r;
      idx_out[o] = i;
      score_out[o] = (double)v;
      int ia = i / (ns * ns), kb = (i / ns) % ns, jg = i % ns;
      euler_out[3 * o] = 2.0 * M_PI * ia / ns;
      euler_out[3 * o + 1] = M_PI * (2.0 * kb + 1.0) / (2.0 * ns);
      euler_out[3 * o + 2] = 2.0 * M_PI * jg / ns;
    }
    __syncthreads();
  }
  for (int r = kept + tid; r < P_max; r += NT) {
    long o = b * P_max + r;
    idx_out[o] = -1;
    score_out[o] = __longlong_as_double(0x7ff8000000000000LL);
    euler_out[3 * o] = euler_out[3 * o + 1] = euler_out[3 * o + 2] = 0.0;
  }
  if (tid == 0) n_cand_out[b] = kept;
}

size_t soft_fused_smem(const Plan &p) {
  int W = 2 * p.L0 + 1;
  size_t tot = (size_t)p.ns * p.ns * p.ns;
  return sizeof(float) * (tot + 2 * (size_t)FUSED_KB * W * W + 2 * (size_t)FUSED_KB * (p.L0 + 1) * p.ns);
}

bool soft_fused_ok(const Plan &p) { return !p.fp64 && soft_fused_smem(p) <= 227 * 1024 - 1024; }

// Streaming variant (both precisions): one CTA per particle walks the beta
// slices k = 0..n-1, computing slice k+1 into a ring of three slices in
// shared memory and then testing the local maxima of slice k, which needs
// only slices k-1, k, k+1.  Under a strict total order no two neighbouring
// grid points can both be local maxima, so one slice holds at most
// ceil(n/2)^2 of them; they are merged by one warp into a running, sorted
// list of the best P.  The grid itself never has to leave the chip; it is
// written to grid_out only when that pointer is given.
constexpr int STREAM_THREADS = 256;

template <typename T>
__device__ void stream_slice(const T *cb, int L0, int ns, int k,
                             const int *__restrict__ pair_base, const T *__restrict__ soft_d,
                             const int *__restrict__ pair_off0, long nc0, const T *__restrict__ tw,
                             T *Sg, T *G, T *dst) {
  const int W = 2 * L0 + 1, np0 = (L0 + 1) * (L0 + 1), tid = threadIdx.x, NT = blockDim.x;
  const T *dk = soft_d + (long)k * nc0;
  for (int q = tid; q < np0; q += NT) {
    int m = isqrt_floor(q), n = q - m * m - m;
    const T *cp = cb + 4L * pair_off0[q];  // staged copy, SOFFT layout
    const T *dp = dk + pair_off0[q];
    T ar = 0, ai = 0, br = 0, bi = 0;
    for (int l = m; l <= L0; ++l) {
      T d = dp[l - m];
      const T *e = cp + 4 * (l - m);
      ar = fma(e[0], d, ar); ai = fma(e[1], d, ai);
      br = fma(e[2], d, br); bi = fma(e[3], d, bi);
    }
    if ((m - n) & 1) { br = -br; bi = -bi; }  // d^l_nm = (-1)^{m-n} d^l_mn
    int i0 = (m + L0) * W + (n + L0);
    Sg[2 * i0] = ar; Sg[2 * i0 + 1] = ai;
    if (q != 0) { int i1 = (-m + L0) * W + (-n + L0); Sg[2 * i1] = ar; Sg[2 * i1 + 1] = -ai; }
    if (n != m && n != -m) {
      int i2 = (n + L0) * W + (m + L0), i3 = (-n + L0) * W + (-m + L0);
      Sg[2 * i2] = br; Sg[2 * i2 + 1] = bi;
      Sg[2 * i3] = br; Sg[2 * i3 + 1] = -bi;
    }
  }
  __syncthreads();
  const FastDiv dns(ns);
  for (int t = tid; t < (L0 + 1) * ns; t += NT) {  // G_m(j) = sum_n S_mn e^{i n g_j}
    int m = dns.div(t), j = t - m * ns;
    const T *row = Sg + 2 * (m + L0) * W;
    T re = 0, im = 0;
    int tt = ns - (L0 * j - dns.div(L0 * j) * ns);  // (-L0 j) mod ns
    if (tt >= ns) tt -= ns;
    for (int n = -L0; n <= L0; ++n) {
      T cr = tw[2 * tt], ci = tw[2 * tt + 1];
      T sr = row[2 * (n + L0)], si = row[2 * (n + L0) + 1];
      re += sr * cr - si * ci;
      im += sr * ci + si * cr;
      tt += j; if (tt >= ns) tt -= ns;
    }
    G[2 * t] = re; G[2 * t + 1] = im;
  }
  __syncthreads();
  for (int t = tid; t < ns * ns; t += NT) {  // Re G_0(j) + 2 Re sum_{m>=1} G_m(j) e^{i m a_i}
    int i = dns.div(t), j = t - i * ns;
    T acc = 0;
    int tt = i;
    for (int m = 1; m <= L0; ++m) {
      T gr = G[2 * (m * ns + j)], gi = G[2 * (m * ns + j) + 1];
      acc += gr * tw[2 * tt] - gi * tw[2 * tt + 1];
      tt += i; if (tt >= ns) tt -= ns;
    }
    dst[t] = G[2 * j] + 2 * acc;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS)
k_soft_stream(const T *__restrict__ c, long nc, int L0, int ns, const int *__restrict__ pair_base,
              const T *__restrict__ soft_d, const int *__restrict__ pair_off0, long nc0,
              const T *__restrict__ tw, int P_max, const int *__restrict__ P_per,
              T *__restrict__ grid_out, int *__restrict__ idx_out, double *__restrict__ euler_out,
              double *__restrict__ score_out, int *__restrict__ n_cand_out) {
  const long b = blockIdx.x;
  const int W = 2 * L0 + 1, n2 = ns * ns, tid = threadIdx.x, NT = blockDim.x;
  const int capc = ((ns + 1) / 2) * ((ns + 1) / 2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ring = reinterpret_cast<T *>(smem_raw);  // [3][n2]
  T *Sg = ring + 3 * n2;                       // [W*W] complex
  T *G = Sg + 2 * W * W;                       // [(L0+1)*ns] complex
  T *cv = G + 2 * (L0 + 1) * ns;               // [capc] slice candidates
  T *rv = cv + capc;                           // [32] running best values
  int *ci = reinterpret_cast<int *>(rv + 32);  // [capc]
  int *ri = ci + capc;                         // [32]
  int *counters = ri + 32;                     // [0] slice count, [1] kept
  T *cst = reinterpret_cast<T *>(reinterpret_cast<uintptr_t>(counters + 4) + 15 & ~uintptr_t(15));
  // stage c^l_mn, l <= L0, of this particle in the SOFFT layout [nc0][4]
  {
    const T *cg = c + 4 * b * nc;
    const int np0 = (L0 + 1) * (L0 + 1);
    const FastDiv dl(L0 + 1);
    for (int t = threadIdx.x; t < np0 * (L0 + 1); t += blockDim.x) {
      int q = dl.div(t), e = t - q * (L0 + 1);
      int m = isqrt_floor(q);
      if (e <= L0 - m) {
        const T *src = cg + pair_base[q] + 8L * e;
        T *dst = cst + 4L * (pair_off0[q] + e);
        dst[0] = src[0]; dst[1] = src[2]; dst[2] = src[4]; dst[3] = src[6];
      }
    }
  }
  const T *cb = cst;
  int Pb = P_per ? min(P_per[b], P_max) : P_max;
  if (Pb < 0) Pb = 0;
  if (tid < 32) { rv[tid] = 0; ri[tid] = INT_MAX; }
  if (tid == 0) counters[1] = 0;
  __syncthreads();
  stream_slice(cb, L0, ns, 0, pair_base, soft_d, pair_off0, nc0, tw, Sg, G, ring);
  if (ns > 1) stream_slice(cb, L0, ns, 1, pair_base, soft_d, pair_off0, nc0, tw, Sg, G, ring + n2);
  for (int k = 0; k < ns; ++k) {
    if (k >= 1 && k + 1 < ns)
      stream_slice(cb, L0, ns, k + 1, pair_base, soft_d, pair_off0, nc0, tw, Sg, G,
                   ring + ((k + 1) % 3) * n2);
    const T *cur = ring + (k % 3) * n2;
    const T *sls[3] = {ring + ((k + 2) % 3) * n2, cur, ring + ((k + 1) % 3) * n2};
    const FastDiv dns(ns);
    if (grid_out) {
      T *go = grid_out + b * (long)ns * n2;
      for (int t = tid; t < n2; t += NT) {
        int i = dns.div(t), j = t - i * ns;
        go[((long)i * ns + k) * ns + j] = cur[t];
      }
    }
    if (tid == 0) counters[0] = 0;
    __syncthreads();
    for (int t = tid; t < n2; t += NT) {
      int i = dns.div(t), j = t - i * ns;
      int p = (i * ns + k) * ns + j;
      T v = cur[t];
      bool ok = v == v;
      for (int dk = -1; dk <= 1 && ok; ++dk) {
        int kk = k + dk;
        if (kk < 0 || kk >= ns) continue;
        const T *sl = sls[dk + 1];
        for (int di = -1; di <= 1 && ok; ++di) {
          int ii = i + di; ii = ii < 0 ? ii + ns : (ii >= ns ? ii - ns : ii);
          for (int dj = -1; dj <= 1; ++dj) {
            if (!di && !dk && !dj) continue;
            int jj = j + dj; jj = jj < 0 ? jj + ns : (jj >= ns ? jj - ns : jj);
            int q = (ii * ns + kk) * ns + jj;
            if (!precedes(v, p, sl[ii * ns + jj], q)) { ok = false; break; }
          }
        }
      }
      if (ok) {
        int pos = atomicAdd(&counters[0], 1);
        if (pos < capc) { cv[pos] = v; ci[pos] = p; }
      }
    }
    __syncthreads();
    if (tid < 32) {  // warp 0: insert the slice's maxima into the sorted best-P list
      const int lane = tid;
      T myv = rv[lane];
      int myi = ri[lane];
      int kept = counters[1];
      const int cnt = min(counters[0], capc);
      for (int e = 0; e < cnt; ++e) {
        T v = cv[e];
        int i = ci[e];
        bool before = lane < kept && precedes(myv, myi, v, i);
        int pos = __popc(__ballot_sync(0xffffffffu, before));
        T upv = __shfl_up_sync(0xffffffffu, myv, 1);
        int upi = __shfl_up_sync(0xffffffffu, myi, 1);
        if (pos < Pb) {
          if (lane > pos) { myv = upv; myi = upi; }
          if (lane == pos) { myv = v; myi = i; }
          kept = min(kept + 1, Pb);
        }
      }
      rv[lane] = myv;
      ri[lane] = myi;
      if (lane == 0) counters[1] = kept;
    }
    __syncthreads();
  }
  const int kept = counters[1];
  for (int r = tid; r < P_max; r += NT) {
    long o = b * P_max + r;
    if (r < kept) {
      int i = ri[r];
      idx_out[o] = i;
      score_out[o] = (double)rv[r];
      int ia = i / (ns * ns), kb = (i / ns) % ns, jg = i % ns;
      euler_out[3 * o] = 2.0 * M_PI * ia / ns;
      euler_out[3 * o + 1] = M_PI * (2.0 * kb + 1.0) / (2.0 * ns);
      euler_out[3 * o + 2] = 2.0 * M_PI * jg / ns;
    } else {
      idx_out[o] = -1;
      score_out[o] = __longlong_as_double(0x7ff8000000000000LL);
      euler_out[3 * o] = euler_out[3 * o + 1] = euler_out[3 * o + 2] = 0.0;
    }
  }
  if (tid == 0) n_cand_out[b] = kept;
}

// Chunked streaming variant: each pass computes up to KB+1 new beta slices at
// once (three phases over all of them) into a ring of KB+2 slices, then tests
// the local maxima of KB slices and merges them, so each barrier separates
// KB times more independent work than the one-slice version.
constexpr int CHUNK_THREADS = 512;

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { struct type { double x, y, z, w; }; };
template <typename T>
__device__ __forceinline__ typename Vec4<T>::type ld4(const T *p) {
  return *reinterpret_cast<const typename Vec4<T>::type *>(p);
}

template <typename T, int KB>
__global__ void __launch_bounds__(CHUNK_THREADS, sizeof(T) == 8 ? 1 : 2)
k_soft_chunk(const T *__restrict__ c, long nc, int L0, int ns, const int *__restrict__ pair_base,
             const T *__restrict__ soft_d, const int *__restrict__ pair_off0, long nc0,
             const T *__restrict__ tw, int P_max, const int *__restrict__ P_per,
             T *__restrict__ grid_out, int *__restrict__ idx_out, double *__restrict__ euler_out,
             double *__restrict__ score_out, int *__restrict__ n_cand_out) {
  constexpr int NR = KB + 2;
  const long b = blockIdx.x;
  const int W = 2 * L0 + 1, np0 = (L0 + 1) * (L0 + 1), n2 = ns * ns;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int capc = KB * ((ns + 1) / 2) * ((ns + 1) / 2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // every section starts on a multiple of 4 elements (16-byte vector loads)
  auto al4 = [](long x) { return (x + 3) & ~3L; };
  T *ring = reinterpret_cast<T *>(smem_raw);   // [NR][n2]
  T *mx = ring + al4(NR * n2);                  // [NR][n2] 3x3 (alpha, gamma) maxima
  T *Sg = mx + al4(NR * n2);                    // [KB+1][W*W] complex
  const int nsp = (ns + 3) / 4 * 4, nq4 = nsp / 4;
  T *G = Sg + al4((KB + 1) * 2 * W * W);        // [KB+1][L0+1][re|im][nsp]
  T *Eg = G + al4((KB + 1) * 2 * (L0 + 1) * nsp);  // [W][nsp] complex: e^{i n g_j}
  T *Aa = Eg + al4(2 * W * nsp);                // [2(L0+1)][nsp]: w_m (cos m a_i, -sin m a_i)
  T *cst = Aa + al4(2 * (L0 + 1) * nsp);        // [nc0][4] staged c, l <= L0
  T *cv = cst + 4 * nc0;                        // [capc]
  T *rv = cv + capc;                            // [32]
  int *ci = reinterpret_cast<int *>(rv + 32);   // [capc]
  int *ri = ci + capc;                          // [32]
  int *counters = ri + 32;                      // [0] pass count, [1] kept
  const FastDiv dns(ns), dn2(n2), dnp0(np0), dl(L0 + 1);
  const FastDiv dq4(nq4), dmq((L0 + 1) * nq4), dqq(nq4 * nq4);
  // twiddle tables (angles 2 pi t / ns from the plan's table)
  for (int t = tid; t < W * nsp; t += NT) {
    int n = t / nsp, j = t - n * nsp;
    T er = 0, ei = 0;
    if (j < ns) {
      int tt = ((n - L0) * j) % ns;
      if (tt < 0) tt += ns;
      er = tw[2 * tt]; ei = tw[2 * tt + 1];
    }
    Eg[2 * t] = er; Eg[2 * t + 1] = ei;
  }
  for (int t = tid; t < 2 * (L0 + 1) * nsp; t += NT) {
    int cc = t / nsp, i = t - cc * nsp, m = cc >> 1;
    T v = 0;
    if (i < ns) {
      int tt = (m * i) % ns;
      T w = m == 0 ? T(1) : T(2);
      v = (cc & 1) ? -w * tw[2 * tt + 1] : w * tw[2 * tt];
    }
    Aa[t] = v;
  }
  {
    const T *cg = c + 4 * b * nc;
    for (int t = tid; t < np0 * (L0 + 1); t += NT) {
      int q = dl.div(t), e = t - q * (L0 + 1);
      int m = isqrt_floor(q);
      if (e <= L0 - m) {
        const T *src = cg + pair_base[q] + 8L * e;
        T *dst = cst + 4L * (pair_off0[q] + e);
        dst[0] = src[0]; dst[1] = src[2]; dst[2] = src[4]; dst[3] = src[6];
      }
    }
  }
  int Pb = P_per ? min(P_per[b], P_max) : P_max;
  if (Pb < 0) Pb = 0;
  if (tid < 32) { rv[tid] = 0; ri[tid] = INT_MAX; }
  if (tid == 0) counters[1] = 0;
  __syncthreads();
  int done = 0;  // slices [0, done) computed
  for (int k0 = 0; k0 < ns; k0 += KB) {
    const int hi = min(ns, k0 + KB + 1), ka = done, nk = hi - ka;
    // phase 1: beta transform of slices ka..hi-1
    for (int t = tid; t < nk * np0; t += NT) {
      int kk = dnp0.div(t), q = t - kk * np0, k = ka + kk;
      int m = isqrt_floor(q), n = q - m * m - m;
      const T *cp = cst + 4L * pair_off0[q];
      const T *dp = soft_d + (long)k * nc0 + pair_off0[q];
      T ar = 0, ai = 0, br = 0, bi = 0;
      for (int l = m; l <= L0; ++l) {
        T d = dp[l - m];
        const T *e = cp + 4 * (l - m);
        ar = fma(e[0], d, ar); ai = fma(e[1], d, ai);
        br = fma(e[2], d, br); bi = fma(e[3], d, bi);
      }
      if ((m - n) & 1) { br = -br; bi = -bi; }  // d^l_nm = (-1)^{m-n} d^l_mn
      T *S = Sg + kk * 2 * W * W;
      int i0 = (m + L0) * W + (n + L0);
      S[2 * i0] = ar; S[2 * i0 + 1] = ai;
      if (q != 0) { int i1 = (-m + L0) * W + (-n + L0); S[2 * i1] = ar; S[2 * i1 + 1] = -ai; }
      if (n != m && n != -m) {
        int i2 = (n + L0) * W + (m + L0), i3 = (-n + L0) * W + (-m + L0);
        S[2 * i2] = br; S[2 * i2 + 1] = bi;
        S[2 * i3] = br; S[2 * i3 + 1] = -bi;
      }
    }
    __syncthreads();
    // phase 2: G_m(j) = sum_n S_mn e^{i n g_j}; tiles of one m and 4 j
    for (int t = tid; t < nk * (L0 + 1) * nq4; t += NT) {
      int kk = dmq.div(t), r = t - kk * (L0 + 1) * nq4;
      int m = dq4.div(r), j0 = (r - m * nq4) * 4;
      const T *row = Sg + kk * 2 * W * W + 2 * (m + L0) * W;
      T re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
      for (int n = 0; n < W; ++n) {
        T sr = row[2 * n], si = row[2 * n + 1];
        const T *e = Eg + 2 * (n * nsp + j0);
        typename Vec4<T>::type e01 = ld4(e), e23 = ld4(e + 4);
        T er[4] = {e01.x, e01.z, e23.x, e23.z}, ei[4] = {e01.y, e01.w, e23.y, e23.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          re[u] = fma(sr, er[u], fma(-si, ei[u], re[u]));
          im[u] = fma(sr, ei[u], fma(si, er[u], im[u]));
        }
      }
      T *Gk = G + kk * 2 * (L0 + 1) * nsp + 2 * m * nsp;  // [m][re|im][j]
#pragma unroll
      for (int u = 0; u < 4; ++u) { Gk[j0 + u] = re[u]; Gk[nsp + j0 + u] = im[u]; }
    }
    __syncthreads();
    // phase 3: C(i, k, j) = sum_c A[c][i] B[c][j] with c = (m, re/im),
    // A = w_m (cos m a_i, -sin m a_i), B = (Re G_m(j), Im G_m(j)); 4 x 4 tiles
    for (int t = tid; t < nk * nq4 * nq4; t += NT) {
      int kk = dqq.div(t), r = t - kk * nq4 * nq4;
      int iq = dq4.div(r), i0 = iq * 4, j0 = (r - iq * nq4) * 4;
      const T *Bk = G + kk * 2 * (L0 + 1) * nsp;
      T o[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) o[u][v] = 0;
      for (int cc = 0; cc < 2 * (L0 + 1); ++cc) {
        typename Vec4<T>::type av = ld4(Aa + cc * nsp + i0), bv = ld4(Bk + cc * nsp + j0);
        T a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) o[u][v] = fma(a4[u], b4[v], o[u][v]);
      }
      T *dst = ring + ((ka + kk) % NR) * n2;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (i0 + u < ns && j0 + v < ns) dst[(i0 + u) * ns + j0 + v] = o[u][v];
    }
    __syncthreads();
    // 3x3 maxima over (alpha, gamma), both wrapping, of the new slices;
    // a NaN anywhere in the window makes the maximum NaN.  A thread keeps one
    // (alpha, gamma) position and walks the slices.
    for (int r = tid; r < n2; r += NT) {
      const int i = dns.div(r), j = r - i * ns;
      const int im = (i == 0 ? ns - 1 : i - 1) * ns, ic = i * ns, ip = (i == ns - 1 ? 0 : i + 1) * ns;
      const int jm = j == 0 ? ns - 1 : j - 1, jp = j == ns - 1 ? 0 : j + 1;
      int slot = ka % NR;
      for (int kk = 0; kk < nk; ++kk) {
        const T *sl = ring + slot * n2;
        T m = sl[ic + j];
        m = nan_max(m, sl[ic + jm]); m = nan_max(m, sl[ic + jp]);
        m = nan_max(m, sl[im + jm]); m = nan_max(m, sl[im + j]); m = nan_max(m, sl[im + jp]);
        m = nan_max(m, sl[ip + jm]); m = nan_max(m, sl[ip + j]); m = nan_max(m, sl[ip + jp]);
        mx[slot * n2 + r] = m;
        slot = slot == NR - 1 ? 0 : slot + 1;
      }
    }
    done = hi;
    if (tid == 0) counters[0] = 0;
    __syncthreads();
    const int k1 = min(ns, k0 + KB), nt_ = k1 - k0;
    if (grid_out) {
      T *go = grid_out + b * (long)ns * n2;
      for (int t = tid; t < nt_ * n2; t += NT) {
        int kk = dn2.div(t), r = t - kk * n2;
        int i = dns.div(r), j = r - i * ns, k = k0 + kk;
        go[((long)i * ns + k) * ns + j] = ring[(k % NR) * n2 + r];
      }
    }
    // local maxima of slices k0..k1-1: the 3x3x3 maximum (slices outside the
    // beta range skipped) rules out every point below it; a point equal to it
    // takes the exact test, which also orders equal values by index
    for (int r = tid; r < n2; r += NT) {
      int slot = k0 % NR;
      int prev = slot == 0 ? NR - 1 : slot - 1;
      T mprev = k0 > 0 ? mx[prev * n2 + r] : T(-INFINITY), mcur = mx[slot * n2 + r];
      for (int k = k0; k < k1; ++k) {
        const int next = slot == NR - 1 ? 0 : slot + 1;
        const T mnext = k < ns - 1 ? mx[next * n2 + r] : T(-INFINITY);
        const T v = ring[slot * n2 + r];
        const T m3 = nan_max(nan_max(mprev, mcur), mnext);
        if (v == m3) {
          const int i = dns.div(r), j = r - i * ns;
          const int p = (i * ns + k) * ns + j;
          bool ok = true;
          for (int dk = -1; dk <= 1 && ok; ++dk) {
            int kq = k + dk;
            if (kq < 0 || kq >= ns) continue;
            const T *sl = ring + (kq % NR) * n2;
            for (int di = -1; di <= 1 && ok; ++di) {
              int ii = i + di; ii = ii < 0 ? ii + ns : (ii >= ns ? ii - ns : ii);
              for (int dj = -1; dj <= 1; ++dj) {
                if (!di && !dk && !dj) continue;
                int jj = j + dj; jj = jj < 0 ? jj + ns : (jj >= ns ? jj - ns : jj);
                int q = (ii * ns + kq) * ns + jj;
                if (!precedes(v, p, sl[ii * ns + jj], q)) { ok = false; break; }
              }
            }
          }
          if (ok) {
            int pos = atomicAdd(&counters[0], 1);
            if (pos < capc) { cv[pos] = v; ci[pos] = p; }
          }
        }
        mprev = mcur; mcur = mnext; slot = next;
      }
    }
    __syncthreads();
    if (tid < 32) {  // warp 0: insert into the sorted best-P list
      const int lane = tid;
      T myv = rv[lane];
      int myi = ri[lane];
      int kept = counters[1];
      const int cnt = min(counters[0], capc);
      for (int e = 0; e < cnt; ++e) {
        T v = cv[e];
        int i = ci[e];
        bool before = lane < kept && precedes(myv, myi, v, i);
        int pos = __popc(__ballot_sync(0xffffffffu, before));
        T upv = __shfl_up_sync(0xffffffffu, myv, 1);
        int upi = __shfl_up_sync(0xffffffffu, myi, 1);
        if (pos < Pb) {
          if (lane > pos) { myv = upv; myi = upi; }
          if (lane == pos) { myv = v; myi = i; }
          kept = min(kept + 1, Pb);
        }
      }
      rv[lane] = myv;
      ri[lane] = myi;
      if (lane == 0) counters[1] = kept;
    }
    __syncthreads();
  }
  const int kept = counters[1];
  for (int r = tid; r < P_max; r += NT) {
    long o = b * P_max + r;
    if (r < kept) {
      int i = ri[r];
      idx_out[o] = i;
      score_out[o] = (double)rv[r];
      int ia = i / (ns * ns), kb = (i / ns) % ns, jg = i % ns;
      euler_out[3 * o] = 2.0 * M_PI * ia / ns;
      euler_out[3 * o + 1] = M_PI * (2.0 * kb + 1.0) / (2.0 * ns);
      euler_out[3 * o + 2] = 2.0 * M_PI * jg / ns;
    } else {
      idx_out[o] = -1;
      score_out[o] = __longlong_as_double(0x7ff8000000000000LL);
      euler_out[3 * o] = euler_out[3 * o + 1] = euler_out[3 * o + 2] = 0.0;
    }
  }
  if (tid == 0) n_cand_out[b] = kept;
}

constexpr int SOFT_KB = 4;

// Warp-per-slice variant (32-bit plans, grids of a few tens of points per
// angle): one CTA per particle; in each pass warp w computes beta slice
// p NW + w on its own (beta transform, the two DFT stages, its slice of the
// grid into a ring of NW + 2 slices), separated only by warp barriers; one
// CTA barrier per pass, then the exact 26-neighbour test of every slice whose
// neighbours are ready (early exit on the first neighbour that precedes the
// point), the survivors merged by warp 0 into the sorted best-P list.  The
// per-point arithmetic and its order are those of k_soft_chunk, so the grid,
// the candidates and their order are bit-identical to it.
template <int NW>
__global__ void __launch_bounds__(NW * 32, 2)
k_soft_warps(const float *__restrict__ c, long nc, int L0, int ns, const int *__restrict__ pair_base,
             const float *__restrict__ soft_d, const int *__restrict__ pair_off0, long nc0,
             const float *__restrict__ tw, int P_max, const int *__restrict__ P_per,
             float *__restrict__ grid_out, int *__restrict__ idx_out, double *__restrict__ euler_out,
             double *__restrict__ score_out, int *__restrict__ n_cand_out) {
  using T = float;
  constexpr int NR = NW + 2;
  const long b = blockIdx.x;
  const int W = 2 * L0 + 1, np0 = (L0 + 1) * (L0 + 1), n2 = ns * ns;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int capc = (NW + 1) * ((ns + 1) / 2) * ((ns + 1) / 2);  // maxima of one pass's slices
  const int nsp = (ns + 3) / 4 * 4, nq4 = nsp / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto al4 = [](long x) { return (x + 3) & ~3L; };
  T *ring = reinterpret_cast<T *>(smem_raw);           // [NR][n2]
  const long per_w = al4(2 * W * W) + al4(2 * (L0 + 1) * nsp);
  T *wbuf = ring + al4(NR * n2);                        // [NW][Sg | G]
  T *Eg = wbuf + NW * per_w;                            // [W][nsp] complex
  T *Aa = Eg + al4(2 * W * nsp);                        // [2(L0+1)][nsp]
  T *cst = Aa + al4(2 * (L0 + 1) * nsp);                // [nc0][4]
  T *cv = cst + 4 * nc0;                                // [capc]
  T *rv = cv + capc;                                    // [32]
  int *ci = reinterpret_cast<int *>(rv + 32);           // [capc]
  int *ri = ci + capc;                                  // [32]
  int *counters = ri + 32;                              // [0] pass count, [1] kept
  const FastDiv dns(ns), dq4(nq4);
  for (int t = tid; t < W * nsp; t += NT) {
    int n = t / nsp, j = t - n * nsp;
    T er = 0, ei = 0;
    if (j < ns) {
      int tt = ((n - L0) * j) % ns;
      if (tt < 0) tt += ns;
      er = tw[2 * tt]; ei = tw[2 * tt + 1];
    }
    Eg[2 * t] = er; Eg[2 * t + 1] = ei;
  }
  for (int t = tid; t < 2 * (L0 + 1) * nsp; t += NT) {
    int cc = t / nsp, i = t - cc * nsp, m = cc >> 1;
    T v = 0;
    if (i < ns) {
      int tt = (m * i) % ns;
      T w = m == 0 ? T(1) : T(2);
      v = (cc & 1) ? -w * tw[2 * tt + 1] : w * tw[2 * tt];
    }
    Aa[t] = v;
  }
  {
    const T *cg = c + 4 * b * nc;
    const FastDiv dl(L0 + 1);
    for (int t = tid; t < np0 * (L0 + 1); t += NT) {
      int q = dl.div(t), e = t - q * (L0 + 1);
      int m = isqrt_floor(q);
      if (e <= L0 - m) {
        const T *src = cg + pair_base[q] + 8L * e;
        T *dst = cst + 4L * (pair_off0[q] + e);
        dst[0] = src[0]; dst[1] = src[2]; dst[2] = src[4]; dst[3] = src[6];
      }
    }
  }
  int Pb = P_per ? min(P_per[b], P_max) : P_max;
  if (Pb < 0) Pb = 0;
  if (tid < 32) { rv[tid] = 0; ri[tid] = INT_MAX; }
  if (tid == 0) counters[1] = 0;
  __syncthreads();
  T *Sg = wbuf + warp * per_w;
  T *G = Sg + al4(2 * W * W);
  int tested = 0;  // slices [0, tested) tested
  for (int k0 = 0; k0 < ns; k0 += NW) {
    const int k = k0 + warp;
    if (k < ns) {
      // beta transform of slice k
      for (int q = lane; q < np0; q += 32) {
        int m = isqrt_floor(q), n = q - m * m - m;
        const T *cp = cst + 4L * pair_off0[q];
        const T *dp = soft_d + (long)k * nc0 + pair_off0[q];
        T ar = 0, ai = 0, br = 0, bi = 0;
        for (int l = m; l <= L0; ++l) {
          T d = dp[l - m];
          const T *e = cp + 4 * (l - m);
          ar = fma(e[0], d, ar); ai = fma(e[1], d, ai);
          br = fma(e[2], d, br); bi = fma(e[3], d, bi);
        }
        if ((m - n) & 1) { br = -br; bi = -bi; }
        int i0 = (m + L0) * W + (n + L0);
        Sg[2 * i0] = ar; Sg[2 * i0 + 1] = ai;
        if (q != 0) { int i1 = (-m + L0) * W + (-n + L0); Sg[2 * i1] = ar; Sg[2 * i1 + 1] = -ai; }
        if (n != m && n != -m) {
          int i2 = (n + L0) * W + (m + L0), i3 = (-n + L0) * W + (-m + L0);
          Sg[2 * i2] = br; Sg[2 * i2 + 1] = bi;
          Sg[2 * i3] = br; Sg[2 * i3 + 1] = -bi;
        }
      }
      __syncwarp();
      // G_m(j) = sum_n S_mn e^{i n g_j}; items of one m and 4 j
      for (int t = lane; t < (L0 + 1) * nq4; t += 32) {
        int m = dq4.div(t), j0 = (t - m * nq4) * 4;
        const T *row = Sg + 2 * (m + L0) * W;
        T re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
        for (int n = 0; n < W; ++n) {
          T sr = row[2 * n], si = row[2 * n + 1];
          const T *e = Eg + 2 * (n * nsp + j0);
          float4 e01 = *reinterpret_cast<const float4 *>(e), e23 = *reinterpret_cast<const float4 *>(e + 4);
          T er[4] = {e01.x, e01.z, e23.x, e23.z}, ei[4] = {e01.y, e01.w, e23.y, e23.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            re[u] = fma(sr, er[u], fma(-si, ei[u], re[u]));
            im[u] = fma(sr, ei[u], fma(si, er[u], im[u]));
          }
        }
        T *Gm = G + 2 * m * nsp;  // [m][re|im][j]
#pragma unroll
        for (int u = 0; u < 4; ++u) { Gm[j0 + u] = re[u]; Gm[nsp + j0 + u] = im[u]; }
      }
      __syncwarp();
      // C(i, k, j) = sum_c A[c][i] B[c][j]; 4 x 4 tiles
      T *dst = ring + (k % NR) * n2;
      for (int t = lane; t < nq4 * nq4; t += 32) {
        int iq = dq4.div(t), i0 = iq * 4, j0 = (t - iq * nq4) * 4;
        T o[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) o[u][v] = 0;
        for (int cc = 0; cc < 2 * (L0 + 1); ++cc) {
          float4 av = *reinterpret_cast<const float4 *>(Aa + cc * nsp + i0);
          float4 bv = *reinterpret_cast<const float4 *>(G + cc * nsp + j0);
          T a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u][v] = fma(a4[u], b4[v], o[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (i0 + u < ns && j0 + v < ns) dst[(i0 + u) * ns + j0 + v] = o[u][v];
      }
      if (grid_out) {
        __syncwarp();
        T *go = grid_out + b * (long)ns * n2;
        for (int r = lane; r < n2; r += 32) {
          int i = dns.div(r), j = r - i * ns;
          go[((long)i * ns + k) * ns + j] = dst[r];
        }
      }
    }
    if (tid == 0) counters[0] = 0;
    __syncthreads();
    // slices whose beta neighbours are ready
    const int done = min(ns, k0 + NW);
    const int t1 = done == ns ? ns : done - 1;
    const int nt_ = t1 - tested;
    for (int t = tid; t < nt_ * n2; t += NT) {
      const int kk = t / n2, r = t - kk * n2, kq0 = tested + kk;
      const int i = dns.div(r), j = r - i * ns;
      const T v = ring[(kq0 % NR) * n2 + r];
      if (!(v == v)) continue;
      const int p = (i * ns + kq0) * ns + j;
      bool ok = true;
      for (int dk = -1; dk <= 1 && ok; ++dk) {
        int kq = kq0 + dk;
        if (kq < 0 || kq >= ns) continue;
        const T *sl = ring + (kq % NR) * n2;
        for (int di = -1; di <= 1 && ok; ++di) {
          int ii = i + di; ii = ii < 0 ? ii + ns : (ii >= ns ? ii - ns : ii);
          for (int dj = -1; dj <= 1; ++dj) {
            if (!di && !dk && !dj) continue;
            int jj = j + dj; jj = jj < 0 ? jj + ns : (jj >= ns ? jj - ns : jj);
            int q = (ii * ns + kq) * ns + jj;
            if (!precedes(v, p, sl[ii * ns + jj], q)) { ok = false; break; }
          }
        }
      }
      if (ok) {
        int pos = atomicAdd(&counters[0], 1);
        if (pos < capc) { cv[pos] = v; ci[pos] = p; }
      }
    }
    tested = t1;
    __syncthreads();
    if (tid < 32) {  // warp 0: insert into the sorted best-P list, in (value, index) order
      T myv = rv[lane];
      int myi = ri[lane];
      int kept = counters[1];
      const int cnt = min(counters[0], capc);
      for (int e = 0; e < cnt; ++e) {
        T v = cv[e];
        int i = ci[e];
        bool before = lane < kept && precedes(myv, myi, v, i);
        int pos = __popc(__ballot_sync(0xffffffffu, before));
        T upv = __shfl_up_sync(0xffffffffu, myv, 1);
        int upi = __shfl_up_sync(0xffffffffu, myi, 1);
        if (pos < Pb) {
          if (lane > pos) { myv = upv; myi = upi; }
          if (lane == pos) { myv = v; myi = i; }
          kept = min(kept + 1, Pb);
        }
      }
      rv[lane] = myv;
      ri[lane] = myi;
      if (lane == 0) counters[1] = kept;
    }
    __syncthreads();
  }
  const int kept = counters[1];
  for (int r = tid; r < P_max; r += NT) {
    long o = b * P_max + r;
    if (r < kept) {
      int i = ri[r];
      idx_out[o] = i;
      score_out[o] = (double)rv[r];
      int ia = i / (ns * ns), kb = (i / ns) % ns, jg = i % ns;
      euler_out[3 * o] = 2.0 * M_PI * ia / ns;
      euler_out[3 * o + 1] = M_PI * (2.0 * kb + 1.0) / (2.0 * ns);
      euler_out[3 * o + 2] = 2.0 * M_PI * jg / ns;
    } else {
      idx_out[o] = -1;
      score_out[o] = __longlong_as_double(0x7ff8000000000000LL);
      euler_out[3 * o] = euler_out[3 * o + 1] = euler_out[3 * o + 2] = 0.0;
    }
  }
  if (tid == 0) n_cand_out[b] = kept;
}

template <int NW>
size_t soft_warps_smem(const Plan &p) {
  auto al4 = [](size_t x) { return (x + 3) & ~size_t(3); };
  const size_t W = 2 * p.L0 + 1, n2 = (size_t)p.ns * p.ns, nsp = (p.ns + 3) / 4 * 4;
  const size_t capc = (size_t)(NW + 1) * ((p.ns + 1) / 2) * ((p.ns + 1) / 2);
  const size_t per_w = al4(2 * W * W) + al4(2 * (p.L0 + 1) * nsp);
  return 4 * (al4((NW + 2) * n2) + NW * per_w + al4(2 * W * nsp) + al4(2 * (p.L0 + 1) * nsp) +
              4 * (size_t)p.nc0 + capc + 32) +
         4 * (capc + 32 + 4) + 16;
}

// Register-tiled chunked variant (32-bit plans, soft_n % 4 == 0): the pass
// structure of k_soft_chunk (KB new beta slices per pass into a ring of KB+2,
// then the local maxima of KB slices), with every phase cut into exactly as
// many work items as the CTA has threads for L0 = 8, K = 2 (324 threads: 324
// pairs, 324 (slice, m, 4 gamma) items, 324 4x4 (alpha, gamma) tiles, 324
// quads of the maximum filter and of the test), and the two DFT stages on
// packed FP32x2 operations fed by operand tables laid out in pairs:
//   stage 2: (Re, Im) G_m(j..j+3) += S_mn (e^{i n g_j}), S read as
//            (Re, Re, Im, Im), twiddles as (cos x4, sin x4, -sin x4);
//   stage 3: C(i..i+3, j..j+3) += A[c][i] B[c][j], A read as pairs (a, a).
// Each grid value is the same chain of roundings as in k_soft_chunk (the same
// fused multiply-adds in the same order; x*(-y) equals (-x)*y exactly), so the
// grid, the candidates and their order are bit-identical to it.  The 3x3
// (alpha, gamma) maximum is taken separably over a thread's quad of gamma
// values.  The bandwidth and the grid size are compile-time constants (the
// stage loops unroll); local maxima that cannot enter the best-P list (once
// it holds P_b entries, those that do not precede its last one) are not
// queued for the merge.
template <int KB, int L0, int ns>
__global__ void __launch_bounds__(384, 2)
k_soft_tile(const float *__restrict__ c, long nc, const int *__restrict__ pair_base,
            const float *__restrict__ soft_d, const int *__restrict__ pair_off0, long nc0,
            const float *__restrict__ tw, int P_max, const int *__restrict__ P_per,
            float *__restrict__ grid_out, int *__restrict__ idx_out, double *__restrict__ euler_out,
            double *__restrict__ score_out, int *__restrict__ n_cand_out) {
  constexpr int NR = KB + 2;
  const long b = blockIdx.x;
  static_assert(ns % 4 == 0, "gamma quads");
  constexpr int W = 2 * L0 + 1, M1 = L0 + 1, np0 = M1 * M1, n2 = ns * ns, q4 = ns / 4;
  const int tid = threadIdx.x, NT = blockDim.x;
  constexpr int capc = KB * ((ns + 1) / 2) * ((ns + 1) / 2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto al4 = [](long x) { return (x + 3) & ~3L; };
  float *ring = reinterpret_cast<float *>(smem_raw);  // [NR][n2]
  float *mx = ring + al4(NR * n2);                     // [NR][n2] 3x3 (alpha, gamma) maxima
  float *G = mx + al4(NR * n2);                        // [KB+1][2 M1][ns]: rows (Re, Im) of G_m
  float *Eg = G + al4((KB + 1) * 2 * M1 * ns);         // [W][q4][12]: cos, sin, -sin of 4 gammas
  float *Ad = Eg + al4(W * q4 * 12);                   // [2 M1][ns][2]: (a, a)
  float *cst = Ad + al4(2 * M1 * ns * 2);              // [nc0][4] staged c, l <= L0
  const long sdn = al4(max((long)(KB + 1) * M1 * W * 4, 2L * capc));
  float *Sd = cst + al4(4 * nc0);                      // [KB+1][M1][W][4]: (Re, Re, Im, Im)
  float *cv = Sd;                                      // [capc] candidates (alias of Sd)
  int *ci = reinterpret_cast<int *>(Sd + capc);        // [capc]
  float *rv = Sd + sdn;                                // [32]
  int *ri = reinterpret_cast<int *>(rv + 32);          // [32]
  int *counters = ri + 32;                             // [0] pass count, [1] kept
  struct CDiv {  // division by a compile-time constant
    int d;
    __device__ __forceinline__ int div(int x) const { return x / d; }
  };
  constexpr CDiv dnp0{np0}, dl{M1}, dq4{q4}, dmq{M1 * q4}, dqq{q4 * q4}, dnq{ns * q4};
  // (row, quad) of item r of a rows x q4 grid: the first q4 - 1 quads of every
  // row first, eight consecutive items per row, then the last quad of each row,
  // so that the eight lanes of a 16-byte shared access stay in one row
  // (conflict-free) instead of straddling two
  auto split = [](int r, int rows, int &row, int &quad) {
    constexpr int Q = q4 - 1;
    if (r < Q * rows) { row = r / Q; quad = r - row * Q; }
    else { row = r - Q * rows; quad = Q; }
  };
  for (int t = tid; t < W * q4 * 4; t += NT) {
    const int n = t / (q4 * 4), r = t - n * q4 * 4, j = 4 * (r >> 2) + (r & 3);
    int tt = ((n - L0) * j) % ns;
    if (tt < 0) tt += ns;
    float *e = Eg + (n * q4 + (r >> 2)) * 12 + (r & 3);
    e[0] = tw[2 * tt];
    e[4] = tw[2 * tt + 1];
    e[8] = -tw[2 * tt + 1];
  }
  for (int t = tid; t < 2 * M1 * ns; t += NT) {
    const int cc = t / ns, i = t - cc * ns, m = cc >> 1;
    const int tt = (m * i) % ns;
    const float wgt = m == 0 ? 1.f : 2.f;
    const float v = (cc & 1) ? -wgt * tw[2 * tt + 1] : wgt * tw[2 * tt];
    Ad[2 * t] = v;
    Ad[2 * t + 1] = v;
  }
  {
    const float *cg = c + 4 * b * nc;
    for (int t = tid; t < np0 * M1; t += NT) {
      int q = dl.div(t), e = t - q * M1;
      int m = isqrt_floor(q);
      if (e <= L0 - m) {
        const float *src = cg + pair_base[q] + 8L * e;
        float *dst = cst + 4L * (pair_off0[q] + e);
        dst[0] = src[0]; dst[1] = src[2]; dst[2] = src[4]; dst[3] = src[6];
      }
    }
  }
  int Pb = P_per ? min(P_per[b], P_max) : P_max;
  if (Pb < 0) Pb = 0;
  if (tid < 32) { rv[tid] = 0; ri[tid] = INT_MAX; }
  if (tid == 0) counters[1] = 0;
  __syncthreads();
  int done = 0;  // slices [0, done) computed
  for (int k0 = 0; k0 < ns; k0 += KB) {
    const int hi = min(ns, k0 + KB + 1), ka = done, nk = hi - ka;
    // phase 1: beta transform of slices ka..hi-1 into the rows m >= 0 of S
    for (int t = tid; t < nk * np0; t += NT) {
      int kk = dnp0.div(t), q = t - kk * np0, k = ka + kk;
      int m = isqrt_floor(q), n = q - m * m - m;
      const float *cp = cst + 4L * pair_off0[q];
      const float *dp = soft_d + (long)k * nc0 + pair_off0[q];
      float ar = 0, ai = 0, br = 0, bi = 0;
      for (int l = m; l <= L0; ++l) {
        float d = dp[l - m];
        const float4 e = *reinterpret_cast<const float4 *>(cp + 4 * (l - m));
        ar = fmaf(e.x, d, ar); ai = fmaf(e.y, d, ai);
        br = fmaf(e.z, d, br); bi = fmaf(e.w, d, bi);
      }
      if ((m - n) & 1) { br = -br; bi = -bi; }  // d^l_nm = (-1)^{m-n} d^l_mn
      float *S = Sd + (long)kk * M1 * W * 4;
      *reinterpret_cast<float4 *>(S + 4 * (m * W + n + L0)) = make_float4(ar, ar, ai, ai);
      if (n != m && n != -m) {
        if (n >= 0) *reinterpret_cast<float4 *>(S + 4 * (n * W + m + L0)) = make_float4(br, br, bi, bi);
        if (n <= 0) *reinterpret_cast<float4 *>(S + 4 * (-n * W - m + L0)) = make_float4(br, br, -bi, -bi);
      }
    }
    __syncthreads();
    // phase 2: G_m(j) = sum_n S_mn e^{i n g_j}, items (slice, m, 4 gammas)
    for (int t = tid; t < nk * M1 * q4; t += NT) {
      int kk = dmq.div(t), r = t - kk * M1 * q4, m, jb;
      split(r, M1, m, jb);
      const float *row = Sd + ((long)kk * M1 + m) * W * 4;
      const float *e = Eg + jb * 12;
      float2 re01 = make_float2(0.f, 0.f), re23 = re01, im01 = re01, im23 = re01;
#pragma unroll
      for (int n = 0; n < W; ++n, e += q4 * 12) {
        const float4 s = *reinterpret_cast<const float4 *>(row + 4 * n);
        const float4 er = *reinterpret_cast<const float4 *>(e);
        const float4 ei = *reinterpret_cast<const float4 *>(e + 4);
        const float4 ne = *reinterpret_cast<const float4 *>(e + 8);
        const float2 sr = make_float2(s.x, s.y), si = make_float2(s.z, s.w);
        re01 = __ffma2_rn(sr, make_float2(er.x, er.y), __ffma2_rn(si, make_float2(ne.x, ne.y), re01));
        re23 = __ffma2_rn(sr, make_float2(er.z, er.w), __ffma2_rn(si, make_float2(ne.z, ne.w), re23));
        im01 = __ffma2_rn(sr, make_float2(ei.x, ei.y), __ffma2_rn(si, make_float2(er.x, er.y), im01));
        im23 = __ffma2_rn(sr, make_float2(ei.z, ei.w), __ffma2_rn(si, make_float2(er.z, er.w), im23));
      }
      float *Gk = G + ((long)kk * 2 * M1 + 2 * m) * ns + 4 * jb;
      *reinterpret_cast<float4 *>(Gk) = make_float4(re01.x, re01.y, re23.x, re23.y);
      *reinterpret_cast<float4 *>(Gk + ns) = make_float4(im01.x, im01.y, im23.x, im23.y);
    }
    __syncthreads();
    // phase 3: C(i, k, j) = sum_c A[c][i] B[c][j]; 4 x 4 tiles
    for (int t = tid; t < nk * q4 * q4; t += NT) {
      int kk = dqq.div(t), r = t - kk * q4 * q4, iq, jq;
      split(r, q4, iq, jq);
      const int i0 = iq * 4, j0 = jq * 4;
      const float *Bk = G + (long)kk * 2 * M1 * ns + j0;
      const float *Ai = Ad + 2 * i0;
      float2 o[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) o[u][0] = o[u][1] = make_float2(0.f, 0.f);
#pragma unroll
      for (int cc = 0; cc < 2 * M1; ++cc) {
        const float4 bv = *reinterpret_cast<const float4 *>(Bk + cc * ns);
        const float4 a01 = *reinterpret_cast<const float4 *>(Ai + 2 * cc * ns);
        const float4 a23 = *reinterpret_cast<const float4 *>(Ai + 2 * cc * ns + 4);
        const float2 b01 = make_float2(bv.x, bv.y), b23 = make_float2(bv.z, bv.w);
        const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                             make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          o[u][0] = __ffma2_rn(a[u], b01, o[u][0]);
          o[u][1] = __ffma2_rn(a[u], b23, o[u][1]);
        }
      }
      float *dst = ring + ((ka + kk) % NR) * n2 + i0 * ns + j0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *reinterpret_cast<float4 *>(dst + u * ns) = make_float4(o[u][0].x, o[u][0].y, o[u][1].x, o[u][1].y);
    }
    __syncthreads();
    // 3x3 maxima over (alpha, gamma), both wrapping, of the new slices; a NaN
    // anywhere in the window makes the maximum NaN.  Item (slice, block of 4
    // alpha rows, quad of 4 gammas): the gamma maxima of the 6 rows i0-1..i0+4
    // from 16-byte reads of the quad and its two neighbours, then the maxima
    // over 3 consecutive rows.
    for (int t = tid; t < nk * q4 * q4; t += NT) {
      const int kk = dqq.div(t), r = t - kk * q4 * q4;
      int ib, jq;
      split(r, q4, ib, jq);
      const int i0 = 4 * ib, j0 = 4 * jq;
      const float *sl = ring + ((ka + kk) % NR) * n2;
      const int jl = (jq == 0 ? q4 - 1 : jq - 1) * 4, jr = (jq == q4 - 1 ? 0 : jq + 1) * 4;
      float rm[6][4];
#pragma unroll
      for (int di = 0; di < 6; ++di) {
        int ii = i0 - 1 + di;
        ii = ii < 0 ? ii + ns : (ii >= ns ? ii - ns : ii);
        const float *rw = sl + ii * ns;
        const float4 x = *reinterpret_cast<const float4 *>(rw + j0);
        const float xm = reinterpret_cast<const float4 *>(rw + jl)->w;
        const float xp = reinterpret_cast<const float4 *>(rw + jr)->x;
        rm[di][0] = nan_max(nan_max(xm, x.x), x.y);
        rm[di][1] = nan_max(nan_max(x.x, x.y), x.z);
        rm[di][2] = nan_max(nan_max(x.y, x.z), x.w);
        rm[di][3] = nan_max(nan_max(x.z, x.w), xp);
      }
      float *mo = mx + ((ka + kk) % NR) * n2 + i0 * ns + j0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float m4[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) m4[v] = nan_max(nan_max(rm[u][v], rm[u + 1][v]), rm[u + 2][v]);
        *reinterpret_cast<float4 *>(mo + u * ns) = make_float4(m4[0], m4[1], m4[2], m4[3]);
      }
    }
    done = hi;
    if (tid == 0) counters[0] = 0;
    __syncthreads();
    const int k1 = min(ns, k0 + KB), nt_ = k1 - k0;
    if (grid_out) {
      float *go = grid_out + b * (long)ns * n2;
      for (int t = tid; t < nt_ * n2; t += NT) {
        int kk = t / n2, r = t - kk * n2;
        int i = r / ns, j = r - i * ns, k = k0 + kk;
        go[((long)i * ns + k) * ns + j] = ring[(k % NR) * n2 + r];
      }
    }
    // local maxima of slices k0..k1-1: the 3x3x3 maximum (slices outside the
    // beta range skipped) rules out every point below it; a point equal to it
    // takes the exact test, which also orders equal values by index
    const bool full = counters[1] >= Pb;
    const float thv = full && Pb > 0 ? rv[Pb - 1] : 0.f;
    const int thi = full && Pb > 0 ? ri[Pb - 1] : 0;
    for (int t = tid; t < ns * q4 && !(full && Pb == 0); t += NT) {
      const int i = dq4.div(t), j0 = (t - i * q4) * 4, r = i * ns + j0;
      int slot = k0 % NR;
      const int prev = slot == 0 ? NR - 1 : slot - 1;
      const float4 ninf = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
      float4 mprev = k0 > 0 ? *reinterpret_cast<const float4 *>(mx + prev * n2 + r) : ninf;
      float4 mcur = *reinterpret_cast<const float4 *>(mx + slot * n2 + r);
      for (int k = k0; k < k1; ++k) {
        const int next = slot == NR - 1 ? 0 : slot + 1;
        const float4 mnext = k < ns - 1 ? *reinterpret_cast<const float4 *>(mx + next * n2 + r) : ninf;
        const float4 v4 = *reinterpret_cast<const float4 *>(ring + slot * n2 + r);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
        const float m3[4] = {nan_max(nan_max(mprev.x, mcur.x), mnext.x),
                             nan_max(nan_max(mprev.y, mcur.y), mnext.y),
                             nan_max(nan_max(mprev.z, mcur.z), mnext.z),
                             nan_max(nan_max(mprev.w, mcur.w), mnext.w)};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (vv[u] != m3[u]) continue;
          const float v = vv[u];
          const int j = j0 + u;
          const int p = (i * ns + k) * ns + j;
          if (full && !precedes(v, p, thv, thi)) continue;
          bool ok = true;
          for (int dk = -1; dk <= 1 && ok; ++dk) {
            int kq = k + dk;
            if (kq < 0 || kq >= ns) continue;
            const float *sl = ring + (kq % NR) * n2;
            for (int di = -1; di <= 1 && ok; ++di) {
              int ii = i + di; ii = ii < 0 ? ii + ns : (ii >= ns ? ii - ns : ii);
              for (int dj = -1; dj <= 1; ++dj) {
                if (!di && !dk && !dj) continue;
                int jj = j + dj; jj = jj < 0 ? jj + ns : (jj >= ns ? jj - ns : jj);
                int q = (ii * ns + kq) * ns + jj;
                if (!precedes(v, p, sl[ii * ns + jj], q)) { ok = false; break; }
              }
            }
          }
          if (ok) {
            int pos = atomicAdd(&counters[0], 1);
            if (pos < capc) { cv[pos] = v; ci[pos] = p; }
          }
        }
        mprev = mcur; mcur = mnext; slot = next;
      }
    }
    __syncthreads();
    if (tid < 32) {  // warp 0: insert into the sorted best-P list
      const int lane = tid;
      float myv = rv[lane];
      int myi = ri[lane];
      int kept = counters[1];
      const int cnt = min(counters[0], capc);
      for (int e = 0; e < cnt; ++e) {
        float v = cv[e];
        int i = ci[e];
        bool before = lane < kept && precedes(myv, myi, v, i);
        int pos = __popc(__ballot_sync(0xffffffffu, before));
        float upv = __shfl_up_sync(0xffffffffu, myv, 1);
        int upi = __shfl_up_sync(0xffffffffu, myi, 1);
        if (pos < Pb) {
          if (lane > pos) { myv = upv; myi = upi; }
          if (lane == pos) { myv = v; myi = i; }
          kept = min(kept + 1, Pb);
        }
      }
      rv[lane] = myv;
      ri[lane] = myi;
      if (lane == 0) counters[1] = kept;
    }
    __syncthreads();
  }
  const int kept = counters[1];
  for (int r = tid; r < P_max; r += NT) {
    long o = b * P_max + r;
    if (r < kept) {
      int i = ri[r];
      idx_out[o] = i;
      score_out[o] = (double)rv[r];
      int ia = i / (ns * ns), kb = (i / ns) % ns, jg = i % ns;
      euler_out[3 * o] = 2.0 * M_PI * ia / ns;
      euler_out[3 * o + 1] = M_PI * (2.0 * kb + 1.0) / (2.0 * ns);
      euler_out[3 * o + 2] = 2.0 * M_PI * jg / ns;
    } else {
      idx_out[o] = -1;
      score_out[o] = __longlong_as_double(0x7ff8000000000000LL);
      euler_out[3 * o] = euler_out[3 * o + 1] = euler_out[3 * o + 2] = 0.0;
    }
  }
  if (tid == 0) n_cand_out[b] = kept;
}

constexpr int TILE_KB = 4;

// Shared memory of k_soft_tile (the layout carved at its start).
size_t soft_tile_smem(const Plan &p) {
  auto al4 = [](size_t x) { return (x + 3) & ~size_t(3); };
  const size_t W = 2 * p.L0 + 1, M1 = p.L0 + 1, ns = p.ns, n2 = ns * ns, q4 = ns / 4;
  const size_t capc = (size_t)TILE_KB * ((ns + 1) / 2) * ((ns + 1) / 2);
  const size_t sdn = al4(std::max((TILE_KB + 1) * M1 * W * 4, 2 * capc));
  return 4 * (2 * al4((TILE_KB + 2) * n2) + al4((TILE_KB + 1) * 2 * M1 * ns) + al4(W * q4 * 12) +
              al4(2 * M1 * ns * 2) + al4(4 * (size_t)p.nc0) + sdn + 32 + 32 + 4);
}

// Threads of k_soft_tile: one per 4x4 tile of a pass (324 at L0 = 8, K = 2),
// at least 128 and at most 384.
int soft_tile_threads(const Plan &p) {
  const int q4 = p.ns / 4;
  return std::min(384, std::max(128, TILE_KB * q4 * q4));
}

// Instantiated for L0 = 8, K = 2 (36 points per angle), the SOFFT of every
// 32-bit workload here; other plans take the chunked kernel.
bool soft_tile_ok(const Plan &p) {
  return !p.fp64 && p.L0 == 8 && p.ns == 36 && soft_tile_smem(p) <= 113 * 1024;
}

size_t soft_chunk_smem(const Plan &p, size_t ts) {
  size_t W = 2 * p.L0 + 1, n2 = (size_t)p.ns * p.ns;
  size_t capc = (size_t)SOFT_KB * ((p.ns + 1) / 2) * ((p.ns + 1) / 2);
  size_t nsp = (size_t)(p.ns + 3) / 4 * 4;
  auto al4 = [](size_t x) { return (x + 3) & ~size_t(3); };
  return ts * (2 * al4((SOFT_KB + 2) * n2) + al4((SOFT_KB + 1) * 2 * W * W) +
               al4((SOFT_KB + 1) * 2 * (size_t)(p.L0 + 1) * nsp) + al4(2 * W * nsp) +
               al4(2 * (size_t)(p.L0 + 1) * nsp) + 4 * (size_t)p.nc0 + capc + 32) +
         sizeof(int) * (capc + 32 + 4) + 16;
}

size_t soft_stream_smem(const Plan &p, size_t ts) {
  size_t W = 2 * p.L0 + 1, n2 = (size_t)p.ns * p.ns, capc = (size_t)((p.ns + 1) / 2) * ((p.ns + 1) / 2);
  return ts * (3 * n2 + 2 * W * W + 2 * (size_t)(p.L0 + 1) * p.ns + capc + 32) +
         sizeof(int) * (capc + 32 + 4) + 32 + ts * 4 * (size_t)p.nc0;
}

// True when one of the fused kernels (chunked, streaming or FP32 fused) serves
// the plan, so the full grid need not be materialised.
bool soft_warps_ok(const Plan &p);

bool soft_grid_optional(const Plan &p) {
  const size_t ts = p.fp64 ? 8 : 4;
  return soft_tile_ok(p) || soft_warps_ok(p) || soft_chunk_smem(p, ts) <= 227 * 1024 - 1024 || soft_stream_smem(p, ts) <= 227 * 1024 - 1024 ||
         (!p.fp64 && soft_fused_ok(p));
}

// True when one of the SOFFT kernels serves the plan (the grid kernel's
// per-slice tables grow with the points per angle).
bool soft_fits(const Plan &p) {
  if (soft_grid_optional(p)) return true;
  const size_t ts = p.fp64 ? 8 : 4, W = 2 * p.L0 + 1;
  return ts * (2 * W * W + 2 * (size_t)(p.L0 + 1) * p.ns) <= 227 * 1024 - 1024;
}

constexpr int SOFT_NW = 6;  // slices per pass of k_soft_warps (two CTAs per SM at L0 = 8, K = 2)

bool soft_warps_ok(const Plan &p) {
  return !p.fp64 && soft_warps_smem<SOFT_NW>(p) <= 113 * 1024;
}

template <typename T>
cudaError_t launch_soft(const Plan &p, const T *c, int B, const int *P_per, T *grid, int *idx,
                        double *euler, double *score, int *n_cand, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  // the warp-per-slice kernel only when chosen (autotuner or matcha_plan_set_tiles):
  // measured slower than the chunked kernel at L0 = 8, K = 2 (0.43 against 0.16 ms
  // for 256 particles)
  if (sizeof(T) == 4 && p.tune_soft == 2 && soft_warps_ok(p)) {
    size_t smem = soft_warps_smem<SOFT_NW>(p);
    cudaFuncSetAttribute(k_soft_warps<SOFT_NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_soft_warps<SOFT_NW><<<B, SOFT_NW * 32, smem, st>>>(
        (const float *)c, p.nc, p.L0, p.ns, p.pair_base, (const float *)p.soft_d, p.pair_off0,
        p.nc0, (const float *)p.soft_tw, p.P, P_per, (float *)grid, idx, euler, score, n_cand);
    return cudaGetLastError();
  }
  // the register-tiled kernel unless another was chosen (bit-identical to the chunked one)
  if (sizeof(T) == 4 && (p.tune_soft == 0 || p.tune_soft == 3) && soft_tile_ok(p)) {
    const size_t smem = soft_tile_smem(p);
    cudaFuncSetAttribute(k_soft_tile<TILE_KB, 8, 36>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_soft_tile<TILE_KB, 8, 36><<<B, soft_tile_threads(p), smem, st>>>(
        (const float *)c, p.nc, p.pair_base, (const float *)p.soft_d, p.pair_off0,
        p.nc0, (const float *)p.soft_tw, p.P, P_per, (float *)grid, idx, euler, score, n_cand);
    return cudaGetLastError();
  }
  {
    size_t smem = soft_chunk_smem(p, sizeof(T));
    if (smem <= 227 * 1024 - 1024) {
      cudaFuncSetAttribute(k_soft_chunk<T, SOFT_KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      k_soft_chunk<T, SOFT_KB><<<B, CHUNK_THREADS, smem, st>>>(
          c, p.nc, p.L0, p.ns, p.pair_base, (const T *)p.soft_d, p.pair_off0, p.nc0,
          (const T *)p.soft_tw, p.P, P_per, grid, idx, euler, score, n_cand);
      return cudaGetLastError();
    }
  }
  {
    size_t smem = soft_stream_smem(p, sizeof(T));
    if (smem <= 227 * 1024 - 1024) {
      cudaFuncSetAttribute(k_soft_stream<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_soft_stream<T><<<B, STREAM_THREADS, smem, st>>>(
          c, p.nc, p.L0, p.ns, p.pair_base, (const T *)p.soft_d, p.pair_off0, p.nc0,
          (const T *)p.soft_tw, p.P, P_per, grid, idx, euler, score, n_cand);
      return cudaGetLastError();
    }
  }
  if (sizeof(T) == 4 && soft_fused_ok(p)) {
    size_t smem = soft_fused_smem(p);
    cudaFuncSetAttribute(k_soft_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_soft_fused<<<B, FUSED_THREADS, smem, st>>>(
        (const float *)c, p.nc, p.L0, p.ns, p.pair_base, (const float *)p.soft_d, p.pair_off0,
        p.nc0, (const float *)p.soft_tw, p.P, P_per, (float *)grid, idx, euler, score, n_cand);
    return cudaGetLastError();
  }
  int W = 2 * p.L0 + 1;
  size_t smem = sizeof(T) * (2 * (size_t)W * W + 2 * (size_t)(p.L0 + 1) * p.ns);
  if (smem > 227 * 1024 - 1024) return cudaErrorInvalidConfiguration;
  cudaFuncSetAttribute(k_soft_grid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_soft_grid<T><<<dim3(p.ns, B), 256, smem, st>>>(c, p.nc, p.L0, p.ns, p.pair_base,
                                                   (const T *)p.soft_d, p.pair_off0, p.nc0,
                                                   (const T *)p.soft_tw, grid);
  k_topk<T><<<B, TOPK_THREADS, 0, st>>>(grid, p.ns, p.P, P_per, idx, euler, score, n_cand);
  return cudaGetLastError();
}

template cudaError_t launch_soft<float>(const Plan &, const float *, int, const int *, float *, int *,
                                        double *, double *, int *, cudaStream_t);
template cudaError_t launch_soft<double>(const Plan &, const double *, int, const int *, double *,
                                         int *, double *, double *, int *, cudaStream_t);

}  // namespace matcha
