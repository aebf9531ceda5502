// Step a6: frequency-marched Newton refinement (Sections 2.2-2.4, Algorithm 1)
// and step a7: the final argmax over candidates.
//
// C_L(a,b,g) = Re sum_{l<=L} sum_{m,n} c^l_{mn} e^{i(m a + n g)} d^l_{mn}(b),
// grad and Hessian in (a, b, g): d/da brings i m, d/dg brings i n, d/db acts
// on d^l (Appendix A.4).  Every evaluation runs the three-term l-recurrence
// of d, d' and d'' for each order pair (m, n) with m >= |n| and uses
//   d^l_{nm} = (-1)^{m-n} d^l_{mn}            (transposed image),
//   term(-m,-n) = conj(term(m,n))              (real volumes),
// so one recurrence serves the four orders (m,n), (n,m), (-m,-n), (-n,-m).
//
// Work layout: one CTA per particle holds all P candidates.  A warp is split
// into sub-slots of `cpw` lanes (cpw = P rounded up to a power of two); lane
// p of a sub-slot follows candidate p, and a sub-slot walks one order pair at
// a time, so the coefficient loads c^l and the recurrence coefficients of a
// step are warp broadcasts.  Per-lane partial sums are reduced in a fixed
// order (shuffles, then warps in index order, in FP64), so results do not
// depend on scheduling.
//
// Step rule (the paper gives only the plain update theta - H^{-1} grad):
//   delta = -H^{-1} grad when -H is positive definite (Cholesky pivots
//   > 1e-12 ||H||_F), else grad / ||H||_F (flag bit 1); ||delta|| clamped to
//   pi / (2 (L+1)); the level ends early when ||delta|| < step_tol
//   (Section 2.4); trial theta' = wrap(theta + delta) is accepted when
//   C(theta') >= C(theta) - acc_tol |C(theta)| (acc_tol above the rounding
//   level of the sums), else delta is halved (at most twice); three
//   rejected trials end the level for that candidate (flag bit 2), since a
//   repeated step from the same point would reject again.  Angles, the 3x3
//   solve and the acceptance test are FP64 in both precisions.
#include <math.h>
#include "internal.cuh"

namespace matcha {

constexpr int NEWTON_THREADS = 256;
constexpr int NEWTON_WARPS = NEWTON_THREADS / 32;

enum { ST_RUN = 0, ST_TRIAL = 1, ST_STOP = 2, ST_DEAD = 3 };

struct NewtonArgs {
  int LJ, nlev, M, P, cpw;
  int Ls[MATCHA_MAX_LEVELS];
  double tol, acc_tol;
  long nc;
};

template <typename T>
__device__ __forceinline__ T ipow_t(T x, int e) {
  T r = T(1);
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

template <typename T> __device__ __forceinline__ T tcos(T x);
template <typename T> __device__ __forceinline__ T tsin(T x);
template <> __device__ __forceinline__ float tcos<float>(float x) { return cosf(x); }
template <> __device__ __forceinline__ float tsin<float>(float x) { return sinf(x); }
template <> __device__ __forceinline__ double tcos<double>(double x) { return cos(x); }
template <> __device__ __forceinline__ double tsin<double>(double x) { return sin(x); }

struct SmemLayout {
  double *th, *tr, *del, *Cc, *res, *red;
  int *state, *steps, *tries, *fl;
  void *evp, *ea, *eg, *pw, *stage;
};

// Asynchronous global -> shared copies (no registers involved).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Copies one entry of four reals (16 B in FP32, 32 B in FP64).
template <typename T>
__device__ __forceinline__ void copy_quad(T *dst, const T *src) {
  cp_async16(dst, src);
  if (sizeof(T) == 8) cp_async16(dst + 2, src + 2);
}

// 16-byte (FP32) or 32-byte (FP64) entry of four reals.
template <typename T> struct Quad;
template <> struct Quad<float> {
  float4 v;
  __device__ __forceinline__ void load(const float *p) { v = *reinterpret_cast<const float4 *>(p); }
  __device__ __forceinline__ float x() const { return v.x; }
  __device__ __forceinline__ float y() const { return v.y; }
  __device__ __forceinline__ float z() const { return v.z; }
  __device__ __forceinline__ float w() const { return v.w; }
};
template <> struct Quad<double> {
  double2 a, b;
  __device__ __forceinline__ void load(const double *p) {
    a = *reinterpret_cast<const double2 *>(p);
    b = *(reinterpret_cast<const double2 *>(p) + 1);
  }
  __device__ __forceinline__ double x() const { return a.x; }
  __device__ __forceinline__ double y() const { return a.y; }
  __device__ __forceinline__ double z() const { return b.x; }
  __device__ __forceinline__ double w() const { return b.y; }
};

// Accumulates the contributions of one order pair for NC candidates that
// share the pair's staged entries (one lane carries NC candidates).
// st: the pair's entries staged in shared memory, entry i = degree m+i holds
// (c^l_mn, c^l_nm) in reals 8i..8i+3 and its recurrence coefficients in
// 8i+4..8i+7.  pc[c][k] = cos(b/2)^k, ps[c][k] = sin(b/2)^k of candidate c.
// A[c]: sum_l c^l_mn {d, d', d''} and sum_l c^l_nm {d, d', d''} (complex).
template <typename T, bool FULL, int NC>
__device__ __forceinline__ void pair_sum(const T *st, T K, int m, int n, int L, const T *x,
                                         const T *s, const T *const *pc, const T *const *ps,
                                         T (*A)[12]) {
  // seed at l = m: d = sigma K ch^a sh^b, a = m+n, b = m-n, sigma = (-1)^b
  const int a = m + n, bq = m - n;
  const T gK = ((bq & 1) ? -K : K);
  T d0[NC], d1[NC], d2[NC], p0[NC], p1[NC], p2[NC], ac[NC][12];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    d0[c] = gK * pc[c][a] * ps[c][bq];
    d1[c] = 0; d2[c] = 0;
    if (FULL) {
      // d/db (ch^a sh^b) = (b ch^{a+1} sh^{b-1} - a ch^{a-1} sh^{b+1}) / 2; the
      // second derivative differentiates once more.  Terms with a zero
      // coefficient are skipped, so no negative power is read.
      T t1 = bq >= 1 ? T(bq) * pc[c][a + 1] * ps[c][bq - 1] : T(0);
      T t2 = a >= 1 ? T(a) * pc[c][a - 1] * ps[c][bq + 1] : T(0);
      d1[c] = gK * T(0.5) * (t1 - t2);
      T u1 = bq >= 2 ? T(bq * (bq - 1)) * pc[c][a + 2] * ps[c][bq - 2] : T(0);
      T u2 = T(bq * (a + 1) + a * (bq + 1)) * pc[c][a] * ps[c][bq];
      T u3 = a >= 2 ? T(a * (a - 1)) * pc[c][a - 2] * ps[c][bq + 2] : T(0);
      d2[c] = gK * T(0.25) * (u1 - u2 + u3);
    }
    p0[c] = 0; p1[c] = 0; p2[c] = 0;
#pragma unroll
    for (int q = 0; q < 12; ++q) ac[c][q] = 0;
  }
  const int last = L - m;  // entries 0..last; the recurrence runs for 0..last-1
  if constexpr (sizeof(T) == 4 && NC == 2) {
    // Packed path: both candidates in float2 registers, one FFMA2 per pair of
    // operations.  The sign of each subtracted term is moved into a negated
    // operand, which is exact, so the results equal the scalar path's.
    float2 D0 = make_float2(d0[0], d0[1]), D1 = make_float2(d1[0], d1[1]);
    float2 D2 = make_float2(d2[0], d2[1]);
    float2 P0 = make_float2(0.f, 0.f), P1 = P0, P2 = P0;
    const float2 X = make_float2(x[0], x[1]), Sn = make_float2(-s[0], -s[1]);
    float2 Z[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) Z[q] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int i = 0; i <= last; ++i) {
      Quad<T> e, r;
      e.load(st + 8 * i);
      r.load(st + 8 * i + 4);
      const float2 Cr = make_float2(e.x(), e.x()), Ci = make_float2(e.y(), e.y());
      const float2 Dr = make_float2(e.z(), e.z()), Di = make_float2(e.w(), e.w());
      Z[0] = __ffma2_rn(Cr, D0, Z[0]); Z[1] = __ffma2_rn(Ci, D0, Z[1]);
      Z[2] = __ffma2_rn(Dr, D0, Z[2]); Z[3] = __ffma2_rn(Di, D0, Z[3]);
      if (FULL) {
        Z[4] = __ffma2_rn(Cr, D1, Z[4]); Z[5] = __ffma2_rn(Ci, D1, Z[5]);
        Z[6] = __ffma2_rn(Dr, D1, Z[6]); Z[7] = __ffma2_rn(Di, D1, Z[7]);
        Z[8] = __ffma2_rn(Cr, D2, Z[8]); Z[9] = __ffma2_rn(Ci, D2, Z[9]);
        Z[10] = __ffma2_rn(Dr, D2, Z[10]); Z[11] = __ffma2_rn(Di, D2, Z[11]);
      }
      if (i < last) {
        const float2 Ca = make_float2(r.x(), r.x()), nCb = make_float2(-r.y(), -r.y());
        const float2 nCe = make_float2(-r.z(), -r.z());
        const float2 t = __ffma2_rn(Ca, X, nCb);                      // a x - b
        const float2 N0 = __ffma2_rn(t, D0, __fmul2_rn(nCe, P0));     // t d - e p
        if (FULL) {
          const float2 nAs = __fmul2_rn(Ca, Sn);                      // -a s
          // t d' - (a s d + e p')
          const float2 N1 = __ffma2_rn(t, D1, __ffma2_rn(nAs, D0, __fmul2_rn(nCe, P1)));
          // t d'' - (2 a s d' + a x d + e p'')
          const float2 nAx = make_float2(-r.x() * x[0], -r.x() * x[1]);
          const float2 N2 = __ffma2_rn(
              t, D2, __ffma2_rn(__fadd2_rn(nAs, nAs), D1, __ffma2_rn(nAx, D0, __fmul2_rn(nCe, P2))));
          P1 = D1; D1 = N1;
          P2 = D2; D2 = N2;
        }
        P0 = D0; D0 = N0;
      }
    }
#pragma unroll
    for (int q = 0; q < 12; ++q)
      if (FULL || q < 4) { A[0][q] = Z[q].x; A[1][q] = Z[q].y; }
    return;
  }
#pragma unroll 2
  for (int i = 0; i <= last; ++i) {
    Quad<T> e, r;
    e.load(st + 8 * i);
    r.load(st + 8 * i + 4);
    const T cr = e.x(), ci = e.y(), dr = e.z(), di = e.w();
    const T ca = r.x(), cb = r.y(), ce = r.z();
    const bool step = i < last;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      ac[c][0] = fma(cr, d0[c], ac[c][0]); ac[c][1] = fma(ci, d0[c], ac[c][1]);
      ac[c][2] = fma(dr, d0[c], ac[c][2]); ac[c][3] = fma(di, d0[c], ac[c][3]);
      if (FULL) {
        ac[c][4] = fma(cr, d1[c], ac[c][4]); ac[c][5] = fma(ci, d1[c], ac[c][5]);
        ac[c][6] = fma(dr, d1[c], ac[c][6]); ac[c][7] = fma(di, d1[c], ac[c][7]);
        ac[c][8] = fma(cr, d2[c], ac[c][8]); ac[c][9] = fma(ci, d2[c], ac[c][9]);
        ac[c][10] = fma(dr, d2[c], ac[c][10]); ac[c][11] = fma(di, d2[c], ac[c][11]);
      }
      if (step) {
        T t = fma(ca, x[c], -cb);
        T n0 = fma(t, d0[c], -ce * p0[c]);
        if (FULL) {
          T as = ca * s[c];
          T n1 = fma(t, d1[c], -fma(as, d0[c], ce * p1[c]));
          T n2 = fma(t, d2[c], -fma(as + as, d1[c], fma(ca * x[c], d0[c], ce * p2[c])));
          p1[c] = d1[c]; d1[c] = n1;
          p2[c] = d2[c]; d2[c] = n2;
        }
        p0[c] = d0[c]; d0[c] = n0;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < 12; ++q)
      if (FULL || q < 4) A[c][q] = ac[c][q];
}

template <typename T, bool FULL>
__device__ __forceinline__ void add_image(T *acc, T w, int a, int b, T zr0, T zi0, T zr1, T zi1,
                                          T zr2) {
  acc[0] += w * zr0;
  if (FULL) {
    T fa = T(a), fb = T(b);
    acc[1] += w * (-fa * zi0);
    acc[2] += w * zr1;
    acc[3] += w * (-fb * zi0);
    acc[4] += w * (-fa * fa * zr0);
    acc[5] += w * (-fa * zi1);
    acc[6] += w * (-fa * fb * zr0);
    acc[7] += w * zr2;
    acc[8] += w * (-fb * zi1);
    acc[9] += w * (-fb * fb * zr0);
  }
}

// Evaluates C (and grad, Hessian when FULL) at pts[p] for the candidates with
// need[p] != 0; results in res[p][0..9] (FP64).  Called by the whole CTA.
template <typename T, bool FULL, int NC>
__device__ void evaluate(const NewtonArgs &A, int L, const T *__restrict__ cb,
                         const int *__restrict__ pair_off, const T *__restrict__ rcoef,
                         const T *__restrict__ seedK, const double *pts, const int *need,
                         SmemLayout &sm) {
  const int P = A.P, cpw = A.cpw, W = 2 * L + 1;
  T *evp = (T *)sm.evp;  // [P][8]: x, s, ch, sh, cos a, sin a, cos g, sin g
  T *ea = (T *)sm.ea;    // [P][W][2]: e^{i m a}, m = -L..L
  T *eg = (T *)sm.eg;
  T *pw = (T *)sm.pw;    // [P][2][NPW]: ch^k, sh^k
  const int NPW = 2 * A.LJ + 3;
  const int tid = threadIdx.x;
  if (tid < P && need[tid]) {
    T al = (T)pts[3 * tid], be = (T)pts[3 * tid + 1], ga = (T)pts[3 * tid + 2];
    T *e = evp + 8 * tid;
    e[0] = tcos(be); e[1] = tsin(be);
    e[2] = tcos(be * T(0.5)); e[3] = tsin(be * T(0.5));
    e[4] = tcos(al); e[5] = tsin(al);
    e[6] = tcos(ga); e[7] = tsin(ga);
  }
  __syncthreads();
  const FastDiv dw(2 * L + 3);
  for (int t = tid; t < 2 * P * (2 * L + 3); t += blockDim.x) {
    int pr = dw.div(t), k = t - pr * (2 * L + 3);
    int p = pr >> 1, which = pr & 1;
    if (need[p]) pw[(2 * p + which) * NPW + k] = ipow_t(evp[8 * p + 2 + which], k);
  }
  if (tid < 2 * P) {
    int p = tid >> 1, which = tid & 1;
    if (need[p]) {
      T c1 = evp[8 * p + 4 + 2 * which], s1 = evp[8 * p + 5 + 2 * which];
      T *tab = (which ? eg : ea) + 2 * (long)p * W;
      T cr = 1, ci = 0;
      tab[2 * L] = 1; tab[2 * L + 1] = 0;
      for (int m = 1; m <= L; ++m) {
        T nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
        cr = nr; ci = ni;
        tab[2 * (L + m)] = cr; tab[2 * (L + m) + 1] = ci;
        tab[2 * (L - m)] = cr; tab[2 * (L - m) + 1] = -ci;
      }
    }
  }
  __syncthreads();

  const int lane = tid & 31, warp = tid >> 5;
  const int spw = 32 / cpw;
  const int p = lane & (cpw - 1);
  const int sub = lane / cpw;
  const int slot = warp * spw + sub;
  const int nslots = NEWTON_WARPS * spw;
  const unsigned submask = cpw == 32 ? 0xffffffffu : (((1u << cpw) - 1u) << (sub * cpw));
  // lane carries candidates p, p + cpw, ..., p + (NC-1) cpw
  bool actc[NC];
  bool act = false;
  T xs[NC], ss[NC], acc[NC][10];
  const T *eap[NC], *egp[NC], *pcp[NC], *psp[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int pc = p + c * cpw;
    actc[c] = pc < P && need[pc];
    act = act || actc[c];
    const int pcc = pc < P ? pc : 0;
    xs[c] = evp[8 * pcc]; ss[c] = evp[8 * pcc + 1];
    eap[c] = ea + 2 * (long)pcc * W; egp[c] = eg + 2 * (long)pcc * W;
    pcp[c] = pw + (2 * pcc) * NPW; psp[c] = pw + (2 * pcc + 1) * NPW;
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[c][i] = 0;
  }
  // Each sub-slot walks order pairs q = slot, slot + nslots, ...; the next
  // pair's entries are copied into the other half of the slot's shared
  // buffer while the current pair is processed.
  const int npl = (L + 1) * (L + 1);
  const int BUFE = A.LJ + 1;
  T *stg = (T *)sm.stage + (long)slot * 2 * (BUFE + 1) * 8;
  auto issue = [&](int qq, int half) {
    int mm = isqrt_floor(qq), len = L - mm + 1, off = pair_off[qq];
    T *dst = stg + half * (BUFE + 1) * 8;
    for (int e = p; e < len; e += cpw) {
      copy_quad<T>(dst + 8 * e, cb + 4L * (off + e));
      copy_quad<T>(dst + 8 * e + 4, rcoef + 4L * (off + e));
    }
    if (p == 0) copy_quad<T>(dst + 8 * BUFE, seedK + 4L * qq);  // (K, 0, 0, 0)
  };
  int cur = 0;
  if (slot < npl) issue(slot, 0);
  cp_async_commit();
  for (int q = slot; q < npl; q += nslots) {
    if (q + nslots < npl) issue(q + nslots, cur ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp(submask);
    if (act) {
      int m = isqrt_floor(q), n = q - m * m - m;
      T Acc[NC][12];
      const T *st = stg + cur * (BUFE + 1) * 8;
      pair_sum<T, FULL, NC>(st, st[8 * BUFE], m, n, L, xs, ss, pcp, psp, Acc);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (!actc[c]) continue;
        const T *Ac = Acc[c];
        // image (m, n) and its negation
        {
          T er = eap[c][2 * (m + L)] * egp[c][2 * (n + L)] - eap[c][2 * (m + L) + 1] * egp[c][2 * (n + L) + 1];
          T ei = eap[c][2 * (m + L)] * egp[c][2 * (n + L) + 1] + eap[c][2 * (m + L) + 1] * egp[c][2 * (n + L)];
          T w = q == 0 ? T(1) : T(2);
          T zr0 = Ac[0] * er - Ac[1] * ei, zi0 = Ac[0] * ei + Ac[1] * er;
          T zr1 = 0, zi1 = 0, zr2 = 0;
          if (FULL) {
            zr1 = Ac[4] * er - Ac[5] * ei; zi1 = Ac[4] * ei + Ac[5] * er;
            zr2 = Ac[8] * er - Ac[9] * ei;
          }
          add_image<T, FULL>(acc[c], w, m, n, zr0, zi0, zr1, zi1, zr2);
        }
        if (n != m && n != -m) {
          // image (n, m): c^l_nm d^l_nm e^{i(n a + m g)}, d^l_nm = (-1)^{m-n} d^l_mn
          T sg = ((m - n) & 1) ? T(-2) : T(2);
          T er = eap[c][2 * (n + L)] * egp[c][2 * (m + L)] - eap[c][2 * (n + L) + 1] * egp[c][2 * (m + L) + 1];
          T ei = eap[c][2 * (n + L)] * egp[c][2 * (m + L) + 1] + eap[c][2 * (n + L) + 1] * egp[c][2 * (m + L)];
          T zr0 = Ac[2] * er - Ac[3] * ei, zi0 = Ac[2] * ei + Ac[3] * er;
          T zr1 = 0, zi1 = 0, zr2 = 0;
          if (FULL) {
            zr1 = Ac[6] * er - Ac[7] * ei; zi1 = Ac[6] * ei + Ac[7] * er;
            zr2 = Ac[10] * er - Ac[11] * ei;
          }
          add_image<T, FULL>(acc[c], sg, n, m, zr0, zi0, zr1, zi1, zr2);
        }
      }
    }
    __syncwarp(submask);
    cur ^= 1;
  }
  cp_async_wait<0>();
  // reduce over the sub-slots of the warp that follow the same candidate
  // (in the working precision; the cross-warp sum below is FP64)
  const int nq = FULL ? 10 : 1;
  for (int o = cpw; o < 32; o <<= 1)
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < 10; ++i)
        if (i < nq) acc[c][i] += __shfl_xor_sync(0xffffffffu, acc[c][i], o);
  if (lane < cpw)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int pc = p + c * cpw;
      if (pc < P)
        for (int i = 0; i < nq; ++i) sm.red[(warp * P + pc) * 10 + i] = (double)acc[c][i];
    }
  __syncthreads();
  for (int idx = tid; idx < P * nq; idx += blockDim.x) {
    int pp = idx / nq, i = idx - pp * nq;
    if (need[pp]) {
      double v = 0;
      for (int w = 0; w < NEWTON_WARPS; ++w) v += sm.red[(w * P + pp) * 10 + i];
      sm.res[pp * 10 + i] = v;
    }
  }
  __syncthreads();
}

__device__ double mod2pi_d(double x) {
  const double t = 2.0 * M_PI;
  double r = x - t * floor(x / t);
  if (r >= t) r -= t;
  if (r < 0) r += t;
  return r;
}

__device__ void wrap_d(double *v) {
  double a = v[0], b = v[1], g = v[2];
  if (b < 0) { b = -b; a += M_PI; g += M_PI; }
  else if (b > M_PI) { b = 2.0 * M_PI - b; a += M_PI; g += M_PI; }
  v[0] = mod2pi_d(a); v[1] = b; v[2] = mod2pi_d(g);
}

// Newton direction from grad g and Hessian H (row-major 3x3); returns flag bits.
__device__ int newton_dir(const double *g, const double *H, int L, double *d) {
  double hn = 0;
  for (int i = 0; i < 9; ++i) hn += H[i] * H[i];
  hn = sqrt(hn);
  const double tol = 1e-12 * hn;
  // Cholesky of A = -H
  double a00 = -H[0], a10 = -H[3], a20 = -H[6], a11 = -H[4], a21 = -H[7], a22 = -H[8];
  bool ok = a00 > tol;
  double L00 = 0, L10 = 0, L20 = 0, L11 = 0, L21 = 0, L22 = 0;
  if (ok) {
    L00 = sqrt(a00); L10 = a10 / L00; L20 = a20 / L00;
    double p11 = a11 - L10 * L10;
    ok = p11 > tol;
    if (ok) {
      L11 = sqrt(p11); L21 = (a21 - L20 * L10) / L11;
      double p22 = a22 - L20 * L20 - L21 * L21;
      ok = p22 > tol;
      if (ok) L22 = sqrt(p22);
    }
  }
  int fl = 0;
  if (ok) {
    double y0 = g[0] / L00;
    double y1 = (g[1] - L10 * y0) / L11;
    double y2 = (g[2] - L20 * y0 - L21 * y1) / L22;
    double x2 = y2 / L22;
    double x1 = (y1 - L21 * x2) / L11;
    double x0 = (y0 - L10 * x1 - L20 * x2) / L00;
    d[0] = x0; d[1] = x1; d[2] = x2;
  } else {
    fl = 2;
    for (int i = 0; i < 3; ++i) d[i] = hn > 0 ? g[i] / hn : 0.0;
  }
  double nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double cap = M_PI / (2.0 * (L + 1.0));
  if (nrm > cap)
    for (int i = 0; i < 3; ++i) d[i] *= cap / nrm;
  return fl;
}

// Candidate tid has C, grad, H of its current point in res: record C, stop on
// a non-finite value (flag bit 0), take the Newton direction, stop the level
// when the increment is below step_tol, else prepare the first trial.
__device__ void start_step(int tid, int L, const NewtonArgs &A, SmemLayout &sm) {
  const double *r = sm.res + 10 * tid;
  double C = r[0], g[3] = {r[1], r[2], r[3]};
  double H[9] = {r[4], r[5], r[6], r[5], r[7], r[8], r[6], r[8], r[9]};
  bool fin = isfinite(C);
  for (int i = 0; i < 3; ++i) fin = fin && isfinite(g[i]);
  for (int i = 0; i < 9; ++i) fin = fin && isfinite(H[i]);
  sm.Cc[tid] = C;
  if (!fin) {
    sm.fl[tid] |= 1;
    sm.state[tid] = ST_DEAD;
    return;
  }
  double d[3];
  sm.fl[tid] |= newton_dir(g, H, L, d);
  if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < A.tol) {
    sm.state[tid] = ST_STOP;
    return;
  }
  double tr[3] = {sm.th[3 * tid] + d[0], sm.th[3 * tid + 1] + d[1], sm.th[3 * tid + 2] + d[2]};
  wrap_d(tr);
  for (int i = 0; i < 3; ++i) {
    sm.del[3 * tid + i] = d[i];
    sm.tr[3 * tid + i] = tr[i];
  }
  sm.tries[tid] = 0;
  sm.state[tid] = ST_TRIAL;
}

template <typename T, int NC>
__global__ void __launch_bounds__(NEWTON_THREADS, sizeof(T) == 8 ? 2 : (NC == 1 ? 3 : 2))
k_newton(const T *__restrict__ c, const int *__restrict__ pair_off, const T *__restrict__ rcoef,
         const T *__restrict__ seedK, NewtonArgs A, const int *__restrict__ n_cand,
         double *__restrict__ euler, double *__restrict__ score, int *__restrict__ cflags,
         long long *__restrict__ work) {
  const long b = blockIdx.x;
  const int P = A.P, tid = threadIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout sm;
  double *dp = reinterpret_cast<double *>(smem_raw);
  sm.th = dp; dp += 3 * P;
  sm.tr = dp; dp += 3 * P;
  sm.del = dp; dp += 3 * P;
  sm.Cc = dp; dp += P;
  sm.res = dp; dp += 10 * P;
  sm.red = dp; dp += 10 * P * NEWTON_WARPS;
  int *ip = reinterpret_cast<int *>(dp);
  sm.state = ip; ip += P;
  sm.steps = ip; ip += P;
  sm.tries = ip; ip += P;
  sm.fl = ip; ip += P;
  int *need = ip; ip += P;
  uintptr_t u = reinterpret_cast<uintptr_t>(ip);
  u = (u + 15) & ~uintptr_t(15);
  T *tp = reinterpret_cast<T *>(u);
  const int Wm = 2 * A.LJ + 1;
  sm.evp = tp; tp += 8 * P;
  sm.ea = tp; tp += 2 * P * Wm;
  sm.eg = tp; tp += 2 * P * Wm;
  sm.pw = tp; tp += 2 * P * (2 * A.LJ + 3);
  tp = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(tp) + 31) & ~uintptr_t(31));
  sm.stage = tp;  // [slots][2][L_J+1][8]

  const int nc_b = n_cand[b];
  if (tid < P) {
    double *e = euler + 3 * (b * P + tid);
    sm.th[3 * tid] = e[0]; sm.th[3 * tid + 1] = e[1]; sm.th[3 * tid + 2] = e[2];
    sm.state[tid] = tid < nc_b ? ST_RUN : ST_DEAD;
    sm.fl[tid] = 0;
    sm.Cc[tid] = __longlong_as_double(0x7ff8000000000000LL);
  }
  __syncthreads();
  const T *cb = c + 4 * b * A.nc;
  long long work_full = 0, work_val = 0;  // counted by thread 0

  // A trial point that is accepted is where the next step needs C, grad and
  // H, so trials are evaluated with derivatives except on a level's last
  // step: per level one derivative evaluation at the start point, then one
  // evaluation per trial.  The points, the arithmetic at each point and the
  // decisions are those of "evaluate at theta, step, test the trial".
  for (int lev = 0; lev < A.nlev; ++lev) {
    const int L = A.Ls[lev];
    // recurrence steps of one evaluation: sum_{m<=L} (2m+1)(L-m+1)
    long long steps_L = 0;
    for (int mm = 0; mm <= L; ++mm) steps_L += (long long)(2 * mm + 1) * (L - mm + 1);
    int want = 0;
    if (tid < P) { need[tid] = sm.state[tid] != ST_DEAD; want = need[tid]; }
    if (!__syncthreads_or(want)) break;
    if (tid == 0)
      for (int q = 0; q < P; ++q) work_full += need[q] ? steps_L : 0;
    evaluate<T, true, NC>(A, L, cb, pair_off, rcoef, seedK, sm.th, need, sm);
    if (tid < P && need[tid]) {
      sm.steps[tid] = 0;
      start_step(tid, L, A, sm);
    }
    for (int round = 0; round < 3 * A.M; ++round) {
      int tw = 0, wf = 0;
      if (tid < P) {
        need[tid] = sm.state[tid] == ST_TRIAL;
        tw = need[tid];
        wf = tw && sm.steps[tid] < A.M - 1;
      }
      if (!__syncthreads_or(tw)) break;
      const bool full = __syncthreads_or(wf);
      if (tid == 0)
        for (int q = 0; q < P; ++q) (full ? work_full : work_val) += need[q] ? steps_L : 0;
      if (full) evaluate<T, true, NC>(A, L, cb, pair_off, rcoef, seedK, sm.tr, need, sm);
      else evaluate<T, false, NC>(A, L, cb, pair_off, rcoef, seedK, sm.tr, need, sm);
      if (tid < P && need[tid]) {
        double Ct = sm.res[10 * tid];
        if (Ct >= sm.Cc[tid] - A.acc_tol * fabs(sm.Cc[tid])) {
          for (int i = 0; i < 3; ++i) sm.th[3 * tid + i] = sm.tr[3 * tid + i];
          sm.Cc[tid] = Ct;
          if (sm.steps[tid] < A.M - 1) {
            ++sm.steps[tid];
            start_step(tid, L, A, sm);  // derivatives at the accepted point
          } else {
            sm.state[tid] = ST_STOP;
          }
        } else if (++sm.tries[tid] == 3) {
          sm.fl[tid] |= 4;
          sm.state[tid] = ST_STOP;  // a repeated step from the same point rejects again
        } else {
          double tr[3];
          for (int i = 0; i < 3; ++i) {
            sm.del[3 * tid + i] *= 0.5;
            tr[i] = sm.th[3 * tid + i] + sm.del[3 * tid + i];
          }
          wrap_d(tr);
          for (int i = 0; i < 3; ++i) sm.tr[3 * tid + i] = tr[i];
        }
      }
    }
    __syncthreads();
  }
  if (tid < P) {
    long o = b * P + tid;
    if (tid < nc_b) {
      euler[3 * o] = sm.th[3 * tid];
      euler[3 * o + 1] = sm.th[3 * tid + 1];
      euler[3 * o + 2] = sm.th[3 * tid + 2];
      score[o] = sm.Cc[tid];
    }
    cflags[o] = sm.fl[tid];
  }
  if (tid == 0 && work) {
    work[2 * b] = work_full;
    work[2 * b + 1] = work_val;
  }
}

// Lanes per warp sub-slot: enough that each lane carries at most NC candidates.
static int newton_cpw(int P, int NC) {
  int per = (P + NC - 1) / NC, cpw = 1;
  while (cpw < per) cpw <<= 1;
  return cpw;
}

size_t newton_smem_bytes(const Plan &p, size_t tsize, int NC) {
  size_t P = p.P, W = 2 * p.LJ + 1;
  size_t bytes = sizeof(double) * (3 * P * 3 + P + 10 * P + 10 * P * NEWTON_WARPS);
  bytes += sizeof(int) * 5 * P;
  bytes = (bytes + 15) / 16 * 16;
  bytes += tsize * (8 * P + 4 * P * W + 2 * P * (2 * (size_t)p.LJ + 3)) + 32;
  size_t slots = (size_t)NEWTON_WARPS * (32 / newton_cpw(p.P, NC));
  bytes += tsize * slots * 2 * (p.LJ + 2) * 8;
  return bytes;
}

template <typename T>
cudaError_t launch_newton(const Plan &p, const T *c, int B, const int *n_cand, double *euler,
                          double *score, int *cflags, long long *work, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  // FP32 plans carry two candidates per lane (shared loads, two independent
  // recurrence chains); FP64 plans one (register pressure)
  constexpr int NC = sizeof(T) == 4 ? 2 : 1;
  NewtonArgs A;
  A.LJ = p.LJ; A.nlev = p.nlev; A.M = p.M; A.P = p.P;
  A.cpw = newton_cpw(p.P, NC);
  for (int i = 0; i < MATCHA_MAX_LEVELS; ++i) A.Ls[i] = i < p.nlev ? p.Ls[i] : 0;
  A.tol = p.step_tol;
  A.acc_tol = p.accept_tol;
  A.nc = p.nc;
  size_t smem = newton_smem_bytes(p, sizeof(T), NC);
  cudaFuncSetAttribute(k_newton<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_newton<T, NC><<<B, NEWTON_THREADS, smem, st>>>(c, p.pair_off, (const T *)p.rcoef,
                                                   (const T *)p.seedK, A, n_cand, euler, score,
                                                   cflags, work);
  return cudaGetLastError();
}

template cudaError_t launch_newton<float>(const Plan &, const float *, int, const int *, double *,
                                          double *, int *, long long *, cudaStream_t);
template cudaError_t launch_newton<double>(const Plan &, const double *, int, const int *, double *,
                                           double *, int *, long long *, cudaStream_t);

__global__ void k_final_select(int B, int P, const int *P_per, const int *n_cand,
                               const double *ce, const double *cs, const int *cf, double *euler,
                               double *R, double *score, int *best_p, int *flags) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int nc = n_cand[b];
  int Pb = P_per ? min(P_per[b], P) : P;
  int best = -1, fl = nc < Pb ? 8 : 0;
  double bs = -INFINITY;
  for (int q = 0; q < nc; ++q) {
    double s = cs[(long)b * P + q];
    fl |= cf[(long)b * P + q];
    if (s > bs) { bs = s; best = q; }
  }
  double a = 0, be = 0, g = 0;
  if (best >= 0) {
    const double *e = ce + 3 * ((long)b * P + best);
    a = e[0]; be = e[1]; g = e[2];
  }
  euler[3 * b] = a; euler[3 * b + 1] = be; euler[3 * b + 2] = g;
  // R = r_z(a) r_y(b) r_z(g)
  double ca = cos(a), sa = sin(a), cb = cos(be), sb = sin(be), cg = cos(g), sg = sin(g);
  double *r = R + 9 * b;
  r[0] = ca * cb * cg - sa * sg; r[1] = -ca * cb * sg - sa * cg; r[2] = ca * sb;
  r[3] = sa * cb * cg + ca * sg; r[4] = -sa * cb * sg + ca * cg; r[5] = sa * sb;
  r[6] = -sb * cg;               r[7] = sb * sg;                 r[8] = cb;
  score[b] = best >= 0 ? bs : __longlong_as_double(0x7ff8000000000000LL);
  best_p[b] = best;
  flags[b] = fl;
}

cudaError_t launch_final_select(const Plan &p, int B, const int *P_per, const int *n_cand,
                                const double *cand_euler, const double *cand_score,
                                const int *cand_flags, double *euler, double *R, double *score,
                                int *best_p, int *flags, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  k_final_select<<<(B + 127) / 128, 128, 0, st>>>(B, p.P, P_per, n_cand, cand_euler, cand_score,
                                                  cand_flags, euler, R, score, best_p, flags);
  return cudaGetLastError();
}

}  // namespace matcha
