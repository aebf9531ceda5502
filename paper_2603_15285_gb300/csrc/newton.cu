// Step a6: frequency-marched Newton refinement (Sections 2.2-2.4, Algorithm 1)
// and step a7: the final argmax over candidates.
//
// C_L(a,b,g) = Re sum_{l<=L} sum_{m,n} c^l_{mn} e^{i(m a + n g)} d^l_{mn}(b),
// grad and Hessian in (a, b, g): d/da brings i m, d/dg brings i n, d/db acts
// on d^l (Appendix A.4).  Every evaluation runs the three-term l-recurrence
// of d and d' for each order pair (m, n) with m >= |n|; the second
// derivative comes from the differential equation of the Wigner functions,
//   d'' = -cot(b) d' + ((m^2 + n^2 - 2mn cos b) / sin^2 b - l(l+1)) d,
// applied to the sums over l (the plans with the rescaled 32-bit recurrence
// above L_J = 64 run a third recurrence for d'' instead).  It uses
//   d^l_{nm} = (-1)^{m-n} d^l_{mn}            (transposed image),
//   term(-m,-n) = conj(term(m,n))              (real volumes),
// so one recurrence serves the four orders (m,n), (n,m), (-m,-n), (-n,-m).
//
// Work layout: one CTA per particle holds all P candidates.  A warp is split
// into sub-slots of `cpw` lanes (cpw = P rounded up to a power of two); lane
// p of a sub-slot follows candidate p.  A sub-slot walks partner groups (the
// two order pairs (m, n), (m, n+1) of one m, stored interleaved), and each
// lane advances both pairs of a group with paired (FP32x2 / 2 x FP64)
// operations: c^l, the recurrence coefficients and the recurrence state are
// pairs over the two partners, so no packed operand is a broadcast pair.  The
// entries are staged in shared memory with cp.async, in batches of up to four
// consecutive groups of the sub-slot.  Per-lane partial sums are reduced in a fixed order (the two
// halves, shuffles across sub-slots, then warps in index order), all in the
// plan's working precision and converted to FP64 at the end, so results do
// not depend on scheduling.
//
// Step rule (the paper gives only the plain update theta - H^{-1} grad):
//   delta = -H^{-1} grad when -H is positive definite (Cholesky pivots
//   > 1e-12 ||H||_F for FP64 sums, > 1e-6 ||H||_F for FP32 sums), else
//   grad / ||H||_F (flag bit 1); ||delta|| clamped to pi / (2 (L+1)); the
//   level ends early when ||delta|| < step_tol (Section 2.4); trial
//   theta' = wrap(theta + delta) is accepted when
//   C(theta') >= C(theta) - acc_tol |C(theta)| (acc_tol above the rounding
//   level of the sums), else delta is halved (at most twice); three
//   rejected trials end the level for that candidate (flag bit 2), since a
//   repeated step from the same point would reject again.  Angles, the
//   acceptance test and the scores are FP64 in every plan; the 3x3 solve is
//   FP64 on the final level and in the plan's precision (FP32 for the 32-bit
//   plans) on the earlier levels.
#include <math.h>
#include <algorithm>
#include "internal.cuh"

namespace matcha {

constexpr int NEWTON_THREADS = 256;
constexpr int NEWTON_WARPS = NEWTON_THREADS / 32;

enum { ST_RUN = 0, ST_TRIAL = 1, ST_STOP = 2, ST_DEAD = 3 };

struct NewtonArgs {
  int LJ, nlev, M, P, cpw, nslots;
  int grad;  // 1: gradient steps grad / ||H||_F instead of Newton steps
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
  double *th, *tr, *del, *Cc, *res;
  void *red;  // [warps][P][10] working precision
  int *state, *steps, *tries, *fl;
  void *ea, *pw, *stage;
};

// Asynchronous global -> shared copies (no registers involved).
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Shared-memory addressing: the hot loops address shared memory through
// 32-bit shared-window addresses and ld.shared, so every load is a shared
// load with 32-bit address arithmetic.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16s(unsigned sa, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void lds1(unsigned a, float &x) {
  asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(x) : "r"(a));
}
__device__ __forceinline__ void lds1(unsigned a, double &x) {
  asm volatile("ld.shared.f64 %0, [%1];\n" : "=d"(x) : "r"(a));
}
__device__ __forceinline__ void lds2(unsigned a, float2 &v) {
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
}
__device__ __forceinline__ void lds2(unsigned a, double2 &v) {
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(v.x), "=d"(v.y) : "r"(a));
}
// two pairs: 16 bytes in FP32 (one vector load), 32 bytes in FP64
__device__ __forceinline__ void lds4(unsigned a, float2 &lo, float2 &hi) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(lo.x), "=f"(lo.y), "=f"(hi.x), "=f"(hi.y)
               : "r"(a));
}
__device__ __forceinline__ void lds4(unsigned a, double2 &lo, double2 &hi) {
  lds2(a, lo);
  lds2(a + 16, hi);
}

// Two-wide values: the two halves of a partner group (pairs (m, n) and
// (m, n+1)) advance together.  FP32 uses the packed FP32x2 instructions of the
// sm_100 family (one FFMA2 does both halves); FP64 issues two scalar FMAs.
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using v2 = typename Vec2<T>::type;

__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vmul(double2 a, double2 b) {
  return make_double2(a.x * b.x, a.y * b.y);
}
__device__ __forceinline__ double2 vadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
template <typename T> __device__ __forceinline__ v2<T> vset(T x, T y);
template <> __device__ __forceinline__ float2 vset<float>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 vset<double>(double x, double y) {
  return make_double2(x, y);
}
template <typename T> __device__ __forceinline__ v2<T> vld(unsigned a0, unsigned a1) {
  T x, y;
  lds1(a0, x);
  lds1(a1, y);
  return vset<T>(x, y);
}

struct Group {
  int m, na, off;  // order, first partner's n, offset in (group, l) entries
};
// The groups of a sub-slot come in increasing g: the order m and the offset
// of the first group of m advance with g instead of being solved for.
struct GroupWalk {
  int m = 0, tri = 0, base = 0;  // tri = m(m+1)/2, base = offset of group (m, 0)
  __device__ __forceinline__ Group at(int g, int LJ) {
    while (g >= tri + m + 1) {
      base += (m + 1) * (LJ - m + 1);
      tri += m + 1;
      ++m;
    }
    const int j = g - tri;
    return {m, 2 * j - m, base + j * (LJ - m + 1)};
  }
};

// Staging buffer of one sub-slot, per half (double buffering), in reals: a
// header (below), then per degree entry 16 reals: the 8 c reals of the group
// entry, then its 8 recurrence reals (a_a, a_b, -b_a, -b_b, -e_a, -e_b,
// -l(l+1), -l(l+1)); L_J + 1 entries.
// Batched staging: a half buffer takes a run of up to STAGE_BATCH consecutive
// groups of its sub-slot whose entries fit in L_J + 1 entries; its header
// holds 8 reals per group: (K_a, K_b, 0, 0) from the seed table, then (m,
// n_a, first entry) written by the sub-slot's first lane, then one pad.
constexpr int STAGE_BATCH = 4;
constexpr int STAGE_HDR = 8 * STAGE_BATCH;  // reals
__host__ __device__ __forceinline__ int stage_half(int LJ) { return STAGE_HDR + 16 * (LJ + 1); }

// Per-candidate tables, candidate index fastest with an odd stride
// cand_stride(P) >= P, so the lanes of a sub-slot (one candidate each) read
// distinct banks.  Power table: two rows (cos(b/2)^k, sin(b/2)^k), each
// PW_PAD zeros followed by k = 0 .. 2 L_J + 3.  Phase table: four rows
// (cos k a, sin k a, cos k g, sin k g) for k = -L_J .. L_J + 1 (index k + L_J).
// Element (row r, position k, candidate p) is at (r * row_len + k) * stride + p.
constexpr int PW_PAD = 4;
__host__ __device__ __forceinline__ int pw_row(int LJ) { return PW_PAD + 2 * LJ + 4; }
__host__ __device__ __forceinline__ int ph_row(int LJ) { return 2 * LJ + 2; }
__host__ __device__ __forceinline__ int cand_stride(int P) { return P | 1; }

// Seeds at l = m of both halves: d = sigma K ch^a sh^b with a = m+n,
// b = m-n, sigma = (-1)^b; with FULL also d' and d'' (Appendix A.4 applied to
// the closed form: d/db (ch^a sh^b) = (b ch^{a+1} sh^{b-1} - a ch^{a-1} sh^{b+1})/2).
// The first half has a = aa, b = ba (both even, so sigma = +1); the second
// a = aa + 1, b = ba - 1 (sigma = -1).  pc, ps: shared addresses of ch^aa,
// sh^ba in the padded power tables; a term whose integer coefficient is zero
// may read a zero pad, so it adds exactly 0.  z: bytes between consecutive
// powers in the table.
template <typename T, bool FULL, bool ODE = false>
__device__ __forceinline__ void group_seed(unsigned pc, unsigned ps, unsigned z, v2<T> K, int aa,
                                           int ba, v2<T> &D0, v2<T> &D1, v2<T> &D2) {
  T c0, c1, s0, sm1;
  lds1(pc, c0); lds1(pc + z, c1);
  lds1(ps, s0); lds1(ps - z, sm1);
  const v2<T> mone = vset<T>(T(-1), T(-1));
  const v2<T> GK = vmul(K, vset<T>(T(1), T(-1)));
  const v2<T> pp0 = vmul(vset<T>(c0, c1), vset<T>(s0, sm1));  // ch^a sh^b
  D0 = vmul(GK, pp0);
  if (FULL) {
    T c2, c3, cm1, cm2, s1, s2, sm2, sm3;
    lds1(pc + 2 * z, c2); lds1(pc + 3 * z, c3); lds1(pc - z, cm1); lds1(pc - 2 * z, cm2);
    lds1(ps + z, s1); lds1(ps + 2 * z, s2); lds1(ps - 2 * z, sm2); lds1(ps - 3 * z, sm3);
    const T fa = T(aa), fb = T(ba);
    const v2<T> A = vset<T>(fa, fa + T(1)), B = vset<T>(fb, fb - T(1));
    const v2<T> one = vset<T>(T(1), T(1));
    const v2<T> t1 = vmul(B, vmul(vset<T>(c1, c2), vset<T>(sm1, sm2)));
    const v2<T> t2 = vmul(A, vmul(vset<T>(cm1, c0), vset<T>(s1, s0)));
    D1 = vmul(vmul(GK, vset<T>(T(0.5), T(0.5))), vfma(t2, mone, t1));
    if (ODE) return;  // d'' comes from the differential equation
    // b(b-1) ch^{a+2} sh^{b-2} - (b(a+1) + a(b+1)) ch^a sh^b + a(a-1) ch^{a-2} sh^{b+2}
    const v2<T> u1 = vmul(vmul(B, vadd(B, mone)), vmul(vset<T>(c2, c3), vset<T>(sm2, sm3)));
    const v2<T> u2 = vmul(vfma(B, vadd(A, one), vmul(A, vadd(B, one))), pp0);
    const v2<T> u3 = vmul(vmul(A, vadd(A, mone)), vmul(vset<T>(cm2, cm1), vset<T>(s2, s1)));
    D2 = vmul(vmul(GK, vset<T>(T(0.25), T(0.25))), vfma(u2, mone, vadd(u1, u3)));
  }
}

// 2^e as a float for -126 <= e <= 127, 0 below (values that small times a
// state below 2^32 are far under FP32 resolution of any sum they enter).
__device__ __forceinline__ float pow2f(int e) {
  return e < -126 ? 0.f : __int_as_float((min(e, 127) + 127) << 23);
}

// Extended-range power x^k = mant 2^expo (mant in [0.5, 1), or 0 for x = 0,
// k > 0) by binary powering with the exponent carried as an integer, so
// that powers far below the FP32 range keep their leading bits.
__device__ __forceinline__ void xpow(float x, int k, float &mant, int &expo) {
  int ex;
  float xm = frexpf(x, &ex);
  float rm = 1.f;
  int re = 0;
  while (k) {
    if (k & 1) {
      int t;
      rm = frexpf(rm * xm, &t);
      re += ex + t;
    }
    k >>= 1;
    if (k) {
      int t;
      xm = frexpf(xm * xm, &t);
      ex = 2 * ex + t;
    }
  }
  if (rm == 0.f) re = 0;
  int t;
  mant = frexpf(rm, &t);
  expo = re + t;
}

// Seeds of the rescaled recurrence (32-bit plans above L_J = 64).  The
// powers come as (mantissa, exponent) from the extended-range tables: pc,
// ps address ch^aa and sh^ba, pe is the byte offset of the exponent rows.
// The states D0, D1, D2 of half h are the true seeds divided by 2^E_h,
// E_h = the exponent of K ch^a sh^b, so the state of d starts near 1 however
// small the true seed is; D1 and D2 keep their ratio to D0.
template <bool FULL>
__device__ __forceinline__ void group_seed_rs(unsigned pc, unsigned ps, unsigned pe, unsigned z,
                                              v2<float> K, int aa, int ba, v2<float> &D0,
                                              v2<float> &D1, v2<float> &D2, int &E0, int &E1) {
  auto ldm = [&](unsigned a, float &m, int &e) {
    float ef;
    lds1(a, m);
    lds1(a + pe, ef);
    e = (int)ef;
  };
  float c0, c1, s0, sm1;
  int ec0, ec1, es0, esm1;
  ldm(pc, c0, ec0); ldm(pc + z, c1, ec1);
  ldm(ps, s0, es0); ldm(ps - z, sm1, esm1);
  int kex, key;
  const float kmx = frexpf(K.x, &kex), kmy = frexpf(K.y, &key);
  const int R0 = ec0 + es0, R1 = ec1 + esm1;  // reference exponents of ch^a sh^b
  E0 = kex + R0;
  E1 = key + R1;
  const float g0 = kmx, g1 = -kmy;            // sigma K of both halves, mantissas
  D0 = vset<float>(g0 * c0 * s0, g1 * c1 * sm1);
  if (FULL) {
    float c2, c3, cm1, cm2, s1, s2, sm2, sm3;
    int ec2, ec3, ecm1, ecm2, es1, es2, esm2, esm3;
    ldm(pc + 2 * z, c2, ec2); ldm(pc + 3 * z, c3, ec3);
    ldm(pc - z, cm1, ecm1); ldm(pc - 2 * z, cm2, ecm2);
    ldm(ps + z, s1, es1); ldm(ps + 2 * z, s2, es2);
    ldm(ps - 2 * z, sm2, esm2); ldm(ps - 3 * z, sm3, esm3);
    // ch^i sh^j relative to 2^R
    auto rel = [](float cm, int ce, float sm, int se, int R) { return cm * sm * pow2f(ce + se - R); };
    const float fa = (float)aa, fb = (float)ba;
    // half 0: a = aa, b = ba; half 1: a = aa + 1, b = ba - 1
    const float t1a = fb * rel(c1, ec1, sm1, esm1, R0), t2a = fa * rel(cm1, ecm1, s1, es1, R0);
    const float t1b = (fb - 1.f) * rel(c2, ec2, sm2, esm2, R1), t2b = (fa + 1.f) * rel(c0, ec0, s0, es0, R1);
    D1 = vset<float>(0.5f * g0 * (t1a - t2a), 0.5f * g1 * (t1b - t2b));
    const float A0 = fa, B0 = fb, A1 = fa + 1.f, B1 = fb - 1.f;
    const float u1a = B0 * (B0 - 1.f) * rel(c2, ec2, sm2, esm2, R0);
    const float u2a = (B0 * (A0 + 1.f) + A0 * (B0 + 1.f)) * rel(c0, ec0, s0, es0, R0);
    const float u3a = A0 * (A0 - 1.f) * rel(cm2, ecm2, s2, es2, R0);
    const float u1b = B1 * (B1 - 1.f) * rel(c3, ec3, sm3, esm3, R1);
    const float u2b = (B1 * (A1 + 1.f) + A1 * (B1 + 1.f)) * rel(c1, ec1, sm1, esm1, R1);
    const float u3b = A1 * (A1 - 1.f) * rel(cm1, ecm1, s1, es1, R1);
    D2 = vset<float>(0.25f * g0 * (u1a + u3a - u2a), 0.25f * g1 * (u1b + u3b - u2b));
  }
}

// One staged degree entry of a partner group: c of both halves, the
// recurrence coefficients (a, -b, -e) of the step to the next degree, and
// -l(l+1) of the entry's own degree l.
template <typename T> struct Coef {
  v2<T> CR, CI, DR, DI;
};
template <typename T> struct Rec {
  v2<T> A, NB, NE, NL;
};
template <typename T> __device__ __forceinline__ void load_coef(unsigned a, Coef<T> &e) {
  lds4(a, e.CR, e.CI);
  lds4(a + 4 * sizeof(T), e.DR, e.DI);
}
template <typename T> __device__ __forceinline__ void load_rec(unsigned a, Rec<T> &r) {
  lds4(a + 8 * sizeof(T), r.A, r.NB);
  lds4(a + 12 * sizeof(T), r.NE, r.NL);
}
// Z += c d (and c d', c d'' when FULL) for one entry; with ODE the third
// sums take -l(l+1) c d (passed as D2 = -l(l+1) d) instead of c d''.
template <typename T, bool FULL>
__device__ __forceinline__ void accumulate(const Coef<T> &e, const v2<T> &D0, const v2<T> &D1,
                                           const v2<T> &D2, v2<T> (&Z)[12]) {
  Z[0] = vfma(e.CR, D0, Z[0]); Z[1] = vfma(e.CI, D0, Z[1]);
  Z[2] = vfma(e.DR, D0, Z[2]); Z[3] = vfma(e.DI, D0, Z[3]);
  if (FULL) {
    Z[4] = vfma(e.CR, D1, Z[4]); Z[5] = vfma(e.CI, D1, Z[5]);
    Z[6] = vfma(e.DR, D1, Z[6]); Z[7] = vfma(e.DI, D1, Z[7]);
    Z[8] = vfma(e.CR, D2, Z[8]); Z[9] = vfma(e.CI, D2, Z[9]);
    Z[10] = vfma(e.DR, D2, Z[10]); Z[11] = vfma(e.DI, D2, Z[11]);
  }
}
// One recurrence step from (d^l, d^{l-1}) = (D, P); d^{l+1} overwrites P:
//   d^{l+1} = t d - e p,  t = a x - b,
//   d'^{l+1} = t d' - a s d - e p',  d''^{l+1} = t d'' - 2 a s d' - a x d - e p''.
template <typename T, bool FULL, bool ODE = false>
__device__ __forceinline__ void step_into(const Rec<T> &r, v2<T> X, v2<T> NS, v2<T> NX,
                                          const v2<T> &D0, const v2<T> &D1, const v2<T> &D2,
                                          v2<T> &P0, v2<T> &P1, v2<T> &P2) {
  const v2<T> t = vfma(r.A, X, r.NB);
  P0 = vfma(t, D0, vmul(r.NE, P0));
  if (FULL && ODE) {
    const v2<T> nAs = vmul(r.A, NS);
    P1 = vfma(t, D1, vfma(nAs, D0, vmul(r.NE, P1)));
  } else if (FULL) {
    const v2<T> nAs = vmul(r.A, NS);
    P1 = vfma(t, D1, vfma(nAs, D0, vmul(r.NE, P1)));
    const v2<T> nAx = vmul(r.A, NX);
    P2 = vfma(t, D2, vfma(vadd(nAs, nAs), D1, vfma(nAx, D0, vmul(r.NE, P2))));
  }
}

// Sums over l = m..m+last of one partner group for one candidate: Z[0..3] =
// sum d (Re c_mn, Im c_mn, Re c_nm, Im c_nm), then the same with d' (Z[4..7])
// and d'' (Z[8..11]) when FULL; each a pair over the two halves.  With ODE
// the second-derivative recurrence is not run: Z[8..11] gets -l(l+1) d in
// place of d'' (the caller completes it with the differential equation).
// a: shared address of the group's first staged entry (16 reals per entry).
// The loop takes two degrees per trip with the roles of (D, P) swapped in the
// second; c is loaded one degree ahead of its use, the step coefficients at
// the start of their degree.
template <typename T, bool FULL, bool ODE = false>
__device__ __forceinline__ void group_sum(unsigned a, int last, v2<T> X, v2<T> NS, v2<T> NX,
                                          v2<T> D0, v2<T> D1, v2<T> D2, v2<T> (&Z)[12]) {
  constexpr unsigned ES = 16 * sizeof(T);
  const v2<T> zero = vset<T>(T(0), T(0));
  v2<T> P0, P1 = zero, P2 = zero;
  auto acc = [&](const Coef<T> &e, const v2<T> &S0, const v2<T> &S1, const v2<T> &S2,
                 const v2<T> &NL) {
    if (ODE) accumulate<T, FULL>(e, S0, S1, vmul(NL, S0), Z);
    else accumulate<T, FULL>(e, S0, S1, S2, Z);
  };
  Coef<T> e0, e1;
  Rec<T> r;
  load_coef(a, e0);
  load_rec(a, r);
  // degree m: the sums start from its products (a product rounds as the
  // multiply-add onto zero does)
  {
    const v2<T> S2 = ODE ? vmul(r.NL, D0) : D2;
    Z[0] = vmul(e0.CR, D0); Z[1] = vmul(e0.CI, D0); Z[2] = vmul(e0.DR, D0); Z[3] = vmul(e0.DI, D0);
    if (FULL) {
      Z[4] = vmul(e0.CR, D1); Z[5] = vmul(e0.CI, D1); Z[6] = vmul(e0.DR, D1); Z[7] = vmul(e0.DI, D1);
      Z[8] = vmul(e0.CR, S2); Z[9] = vmul(e0.CI, S2); Z[10] = vmul(e0.DR, S2); Z[11] = vmul(e0.DI, S2);
    } else {
#pragma unroll
      for (int q = 4; q < 12; ++q) Z[q] = zero;
    }
  }
  if (last == 0) return;
  // the step from degree m, whose predecessor state is zero
  {
    const v2<T> t = vfma(r.A, X, r.NB);
    P0 = vmul(t, D0);
    if (FULL) {
      const v2<T> nAs = vmul(r.A, NS);
      P1 = vfma(t, D1, vmul(nAs, D0));
      if (!ODE) {
        const v2<T> nAx = vmul(r.A, NX);
        P2 = vfma(t, D2, vfma(vadd(nAs, nAs), D1, vmul(nAx, D0)));
      }
    }
  }
  a += ES;
  load_coef(a, e1);
  // two degrees per trip: degree i in (P0, P1, P2), degree i + 1 in (D0, D1, D2)
  int i = 1;
  for (; i + 2 <= last; i += 2, a += 2 * ES) {
    load_rec(a, r);
    load_coef(a + ES, e0);
    acc(e1, P0, P1, P2, r.NL);
    step_into<T, FULL, ODE>(r, X, NS, NX, P0, P1, P2, D0, D1, D2);
    load_rec(a + ES, r);
    load_coef(a + 2 * ES, e1);
    acc(e0, D0, D1, D2, r.NL);
    step_into<T, FULL, ODE>(r, X, NS, NX, D0, D1, D2, P0, P1, P2);
  }
  v2<T> nl = zero;
  if (i < last) {  // degrees i (with a step) and last = i + 1
    load_rec(a, r);
    load_coef(a + ES, e0);
    acc(e1, P0, P1, P2, r.NL);
    step_into<T, FULL, ODE>(r, X, NS, NX, P0, P1, P2, D0, D1, D2);
    if (ODE && FULL) lds2(a + ES + 14 * sizeof(T), nl);
    acc(e0, D0, D1, D2, nl);
  } else {         // degree last = i
    if (ODE && FULL) lds2(a + 14 * sizeof(T), nl);
    acc(e1, P0, P1, P2, nl);
  }
}

// group_sum for the rescaled states of group_seed_rs: the true d, d', d'' of
// half h are the states times 2^E_h.  Each accumulation multiplies the state
// by SC = 2^E (0 while the true values are below 2^-126); after each step a
// half whose state has grown past 2^32 while E_h < 0 is scaled down by 2^32
// (exactly) and E_h raised by 32, so the states neither overflow nor lose the
// digits of seeds far below the FP32 range (per-degree rescaling).
__device__ __forceinline__ void rescale_half(float &p0, float &p1, float &p2, float &d0, float &d1,
                                             float &d2, int &E, float &sc) {
  if (E < 0 && fabsf(p0) > 4294967296.f) {
    const float f = 2.3283064365386963e-10f;  // 2^-32
    p0 *= f; p1 *= f; p2 *= f; d0 *= f; d1 *= f; d2 *= f;
    E += 32;
    sc = pow2f(E);
  }
}

template <bool FULL>
__device__ __forceinline__ void group_sum_rs(unsigned a, int last, v2<float> X, v2<float> NS,
                                             v2<float> NX, v2<float> D0, v2<float> D1, v2<float> D2,
                                             int E0, int E1, v2<float> (&Z)[12]) {
  constexpr unsigned ES = 16 * sizeof(float);
  const v2<float> zero = vset<float>(0.f, 0.f);
  v2<float> P0 = zero, P1 = zero, P2 = zero;
#pragma unroll
  for (int q = 0; q < 12; ++q) Z[q] = zero;
  float scx = pow2f(E0), scy = pow2f(E1);
  Coef<float> e;
  Rec<float> r;
  auto acc = [&](const v2<float> &S0, const v2<float> &S1, const v2<float> &S2) {
    const v2<float> SC = vset<float>(scx, scy);
    accumulate<float, FULL>(e, vmul(S0, SC), vmul(S1, SC), vmul(S2, SC), Z);
  };
  for (int i = 0; i <= last; ++i, a += ES) {
    load_coef(a, e);
    if (i & 1) acc(P0, P1, P2);
    else acc(D0, D1, D2);
    if (i == last) break;
    load_rec(a, r);
    if (i & 1) {
      step_into<float, FULL>(r, X, NS, NX, P0, P1, P2, D0, D1, D2);
      rescale_half(D0.x, D1.x, D2.x, P0.x, P1.x, P2.x, E0, scx);
      rescale_half(D0.y, D1.y, D2.y, P0.y, P1.y, P2.y, E1, scy);
    } else {
      step_into<float, FULL>(r, X, NS, NX, D0, D1, D2, P0, P1, P2);
      rescale_half(P0.x, P1.x, P2.x, D0.x, D1.x, D2.x, E0, scx);
      rescale_half(P0.y, P1.y, P2.y, D0.y, D1.y, D2.y, E1, scy);
    }
  }
}

// Adds one image of both halves to the candidate's sums.  The image has phase
// E = e^{i(u a + v g)} and weight W; (zr0, zi0) = S0 E, (zr1, zi1) = S1 E,
// zr2 = Re S2 E for the d, d', d'' sums S0, S1, S2.  d/da brings i u and d/dg
// brings i v, so with AU = -W u, GV = -W v:
//   C += W zr0, C_a += AU zi0, C_b += W zr1, C_g += GV zi0,
//   C_aa += AU u zr0, C_ab += AU zi1, C_ag += AU v zr0, C_bb += W zr2,
//   C_bg += GV zi1, C_gg += GV v zr0.
template <typename T, bool FULL>
__device__ __forceinline__ void add_image(v2<T> (&acc)[10], v2<T> W, v2<T> U, v2<T> V,
                                          const v2<T> &ER, const v2<T> &EI, const v2<T> &NEI,
                                          const v2<T> &S0r, const v2<T> &S0i, const v2<T> &S1r,
                                          const v2<T> &S1i, const v2<T> &S2r, const v2<T> &S2i) {
  const v2<T> zr0 = vfma(S0r, ER, vmul(S0i, NEI));
  acc[0] = vfma(W, zr0, acc[0]);
  if (FULL) {
    const v2<T> mone = vset<T>(T(-1), T(-1));
    const v2<T> zi0 = vfma(S0r, EI, vmul(S0i, ER));
    const v2<T> zr1 = vfma(S1r, ER, vmul(S1i, NEI));
    const v2<T> zi1 = vfma(S1r, EI, vmul(S1i, ER));
    const v2<T> zr2 = vfma(S2r, ER, vmul(S2i, NEI));
    const v2<T> NW = vmul(W, mone);
    const v2<T> AU = vmul(NW, U), GV = vmul(NW, V);
    acc[1] = vfma(AU, zi0, acc[1]);
    acc[2] = vfma(W, zr1, acc[2]);
    acc[3] = vfma(GV, zi0, acc[3]);
    acc[4] = vfma(vmul(AU, U), zr0, acc[4]);
    acc[5] = vfma(AU, zi1, acc[5]);
    acc[6] = vfma(vmul(AU, V), zr0, acc[6]);
    acc[7] = vfma(W, zr2, acc[7]);
    acc[8] = vfma(GV, zi1, acc[8]);
    acc[9] = vfma(vmul(GV, V), zr0, acc[9]);
  }
}

// Phase pair E = (cos, sin) rows product: E = EA EG with EA = (ar + i ai),
// EG = (gr + i gi) pairs; returns Re, Im and -Im.
template <typename T>
__device__ __forceinline__ void phase(v2<T> Ar, v2<T> Ai, v2<T> Gr, v2<T> Gi, v2<T> &ER,
                                      v2<T> &EI, v2<T> &NEI) {
  const v2<T> mone = vset<T>(T(-1), T(-1));
  ER = vfma(Ar, Gr, vmul(vmul(Ai, mone), Gi));
  EI = vfma(Ar, Gi, vmul(Ai, Gr));
  NEI = vmul(EI, mone);
}

// Evaluates C (and grad, Hessian when FULL) at pts[p] for the candidates with
// need[p] != 0; results in res[p][0..9] (FP64).  Called by the whole CTA.
//
// Lane layout: a warp holds 32 / cpw sub-slots of cpw lanes; lane p of a
// sub-slot follows candidate p.  Sub-slot `slot` walks the partner groups of
// bandwidth L in its alternating order; the next batch of its groups is
// copied into the other half of the slot's buffer while the current batch is
// summed, and the lanes of a sub-slot read the same staged entries (one
// shared-memory broadcast per load).
template <typename T, bool FULL, bool RS>
__device__ __forceinline__ void evaluate(const NewtonArgs &A, int L, const T *__restrict__ cb,
                                         const T *__restrict__ rcoef, const T *__restrict__ seedK,
                                         const double *pts, const int *need, SmemLayout &sm) {
  constexpr unsigned z = sizeof(T);
  const int P = A.P, cpw = A.cpw, LJ = A.LJ;
  const int NPW = pw_row(LJ), RW = ph_row(LJ), PS = cand_stride(P);
  T *ph = (T *)sm.ea;    // [4][RW][PS]: cos k a, sin k a, cos k g, sin k g
  T *pw = (T *)sm.pw;    // [2][NPW][PS]: PW_PAD zeros, then ch^k (sh^k), k = 0..2LJ+3
  const int tid = threadIdx.x;
  // Each thread takes the cosines and sines it needs from the point itself
  // (no table and no barrier before the tables below).
  // powers k = 0..2L+3 of cos(beta/2) and sin(beta/2): runs of 8 consecutive
  // powers per item, the first by binary powering, the rest by one product each
  constexpr int RUN = 8;
  const int npk = 2 * L + 4, nrun = (npk + RUN - 1) / RUN;
  const FastDiv dw(nrun);
  for (int t = tid; t < 2 * P * nrun; t += blockDim.x) {
    int pr = dw.div(t), k0 = (t - pr * nrun) * RUN;
    int p = pr >> 1, which = pr & 1;
    if (!need[p]) continue;
    const T hb = (T)pts[3 * p + 1] * T(0.5);
    const T x = which ? tsin(hb) : tcos(hb);
    const int k1 = min(k0 + RUN, npk);
    if (RS) {  // mantissa rows, then exponent rows (2 NPW rows further on)
      for (int k = k0; k < k1; ++k) {
        float mt;
        int ex;
        xpow((float)x, k, mt, ex);
        pw[(which * NPW + PW_PAD + k) * PS + p] = (T)mt;
        pw[((2 + which) * NPW + PW_PAD + k) * PS + p] = (T)ex;
      }
    } else {
      T v = ipow_t(x, k0);
      T *o = pw + (which * NPW + PW_PAD + k0) * PS + p;
      o[0] = v;
      for (int k = k0 + 1; k < k1; ++k) {
        v *= x;
        o += PS;
        o[0] = v;
      }
    }
  }
  // phase rows cos, sin of k alpha and k gamma, k = -L..L+1: eight chains per
  // (candidate, angle), chain q holding k = q, q + 8, ... (start e^{i q x},
  // step e^{8 i x})
  for (int t = tid; t < 16 * P; t += blockDim.x) {
    const int pq = t >> 3, q = t & 7, p = pq >> 1, which = pq & 1;
    if (need[p]) {
      const T ang = (T)pts[3 * p + 2 * which];  // alpha or gamma
      const T c1 = tcos(ang), s1 = tsin(ang);
      T *cr_ = ph + ((2 * which) * RW + LJ) * PS + p, *ci_ = cr_ + RW * PS;
      // e^{2ix}, e^{4ix}, e^{8ix} and e^{iqx} by binary powering
      const T c2 = c1 * c1 - s1 * s1, s2 = T(2) * c1 * s1;
      const T c4 = c2 * c2 - s2 * s2, s4 = T(2) * c2 * s2;
      const T c8 = c4 * c4 - s4 * s4, s8 = T(2) * c4 * s4;
      T cr = 1, ci = 0;
      if (q & 1) { cr = c1; ci = s1; }
      if (q & 2) { const T nr = cr * c2 - ci * s2, ni = cr * s2 + ci * c2; cr = nr; ci = ni; }
      if (q & 4) { const T nr = cr * c4 - ci * s4, ni = cr * s4 + ci * c4; cr = nr; ci = ni; }
      for (int m = q; m <= L + 1; m += 8) {
        cr_[m * PS] = cr; ci_[m * PS] = ci;
        if (m > 0 && m <= L) { cr_[-m * PS] = cr; ci_[-m * PS] = -ci; }
        const T nr = cr * c8 - ci * s8, ni = cr * s8 + ci * c8;
        cr = nr; ci = ni;
      }
    }
  }
  __syncthreads();

  const int lane = tid & 31, warp = tid >> 5;
  const int spw = 32 / cpw;
  const int p = lane & (cpw - 1);
  const int sub = lane / cpw;
  const int slot = warp * spw + sub;
  const int nslots = A.nslots;  // sub-slots with a staging buffer (<= NEWTON_WARPS * spw)
  const unsigned submask = cpw == 32 ? 0xffffffffu : (((1u << cpw) - 1u) << (sub * cpw));
  const bool act = p < P && need[p];
  const int pc = p < P ? p : 0;
  const T bt = (T)pts[3 * pc + 1];
  const T xb = tcos(bt), sb = tsin(bt);
  const v2<T> X = vset<T>(xb, xb), NS = vset<T>(-sb, -sb), NX = vset<T>(-xb, -xb);
  // constants of the differential equation for d'' (the non-rescaled path):
  // 1/sin^2 b and -cot b with sin b floored away from zero, and the pole form
  // of the numerator of Q (sign of n in m -/+ n, and +4 sin^2(b/2) or -4 cos^2(b/2))
  v2<T> IS2, NCOT, QSG, QC4;
  {
    const T sfl = sizeof(T) == 8 ? T(1e-150) : T(1e-18);
    const T se = sb > sfl ? sb : sfl;
    const T is2 = T(1) / (se * se), ncot = -xb / se;
    const T chb = tcos(bt * T(0.5)), shb = tsin(bt * T(0.5));
    const bool north = xb >= T(0);
    const T sg = north ? T(-1) : T(1), c4 = north ? T(4) * shb * shb : T(-4) * chb * chb;
    IS2 = vset<T>(is2, is2); NCOT = vset<T>(ncot, ncot);
    QSG = vset<T>(sg, sg); QC4 = vset<T>(c4, c4);
  }
  // shared addresses of this candidate's tables (index 0 of each row)
  const unsigned zs = z * PS;  // bytes between consecutive positions of a row
  const unsigned pcu = smem_u32(pw + PW_PAD * PS + pc);
  const unsigned psu = pcu + zs * NPW;
  const unsigned eacu = smem_u32(ph + LJ * PS + pc);  // k = 0 of cos k a
  const unsigned easu = eacu + zs * RW, egcu = easu + zs * RW, egsu = egcu + zs * RW;
  v2<T> acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = vset<T>(T(0), T(0));

  const int ng = (L + 1) * (L + 2) / 2;
  const unsigned HB = z * stage_half(LJ);  // bytes per half buffer
  const unsigned stg = smem_u32(sm.stage) + (unsigned)(slot < nslots ? slot : 0) * 2 * HB;
  // Copy duty of this lane: 16-byte chunk `part` of every entry e = e0,
  // e0 + estep, ...; parts below CPE/2 come from c, the rest from the
  // recurrence table.
  constexpr int CH = 16 / (int)sizeof(T), CPE = 16 / CH;  // reals per chunk, chunks per entry
  const int part = p % CPE, e0 = p / CPE, estep = cpw / CPE;
  const T *srcb = (part < CPE / 2 ? cb : rcoef) + CH * (part % (CPE / 2)) + 8 * e0;
  const unsigned dsto = z * (STAGE_HDR + 16 * e0 + CH * part);
  // Sub-slot `slot` takes group k * nslots + slot in even rounds k and
  // k * nslots + (nslots - 1 - slot) in odd ones: groups come in increasing g
  // (non-increasing length), so the alternating order balances the sub-slots
  // while keeping every sum's order fixed.
  auto group_at = [&](int k) {
    return k * nslots + ((k & 1) ? nslots - 1 - slot : slot);
  };
  if (slot < nslots && slot < ng) {
    GroupWalk walk;
    int k = 0;  // next group of this sub-slot's sequence
    // Copies the next batch of groups into half buffer hb; returns its size
    // (0 when the sub-slot has no group left).
    auto issue_batch = [&](unsigned hb) -> int {
      int cnt = 0, eoff = 0;
      while (cnt < STAGE_BATCH) {
        const int g = group_at(k);
        if (g >= ng) break;
        const Group G = walk.at(g, LJ);
        const int len = L - G.m + 1;
        if (cnt > 0 && eoff + len > LJ + 1) break;
        const T *src = srcb + 8L * G.off;
        unsigned dst = hb + dsto + 16 * z * eoff;
        for (int e = e0; e < len; e += estep, src += 8 * estep, dst += 16 * z * estep)
          cp_async16s(dst, src);
        const unsigned hd = hb + z * 8 * cnt;
        if (p < 4 / CH) cp_async16s(hd + 16 * p, seedK + 4L * g + CH * p);
        if (p == 0) {
          T *h = reinterpret_cast<T *>(__cvta_shared_to_generic(hd));
          h[4] = T(G.m); h[5] = T(G.na); h[6] = T(eoff);
        }
        eoff += len;
        ++cnt;
        ++k;
      }
      return cnt;
    };
    int cur = 0;
    int ncur = issue_batch(stg);
    cp_async_commit();
    while (ncur > 0) {
      const int nnext = issue_batch(stg + (cur ^ 1) * HB);
      cp_async_commit();
      cp_async_wait<1>();
      __syncwarp(submask);
      if (act) {
       for (int t = 0; t < ncur; ++t) {
        const unsigned buf = stg + cur * HB, hd = buf + z * 8 * t;
        T hm, hn, he;
        lds1(hd + 4 * z, hm); lds1(hd + 5 * z, hn); lds1(hd + 6 * z, he);
        const int m = (int)hm, na = (int)hn, eoff = (int)he, aa = m + na, ba = m - na;
        const unsigned ent = buf + z * (STAGE_HDR + 16 * eoff);
        v2<T> K, D0, D1, D2, Z[12];
        lds2(hd, K);
        D1 = D2 = vset<T>(T(0), T(0));
        if constexpr (RS) {
          int E0, E1;
          group_seed_rs<FULL>(pcu + zs * aa, psu + zs * ba, zs * 2 * NPW, zs, K, aa, ba, D0, D1,
                              D2, E0, E1);
          group_sum_rs<FULL>(ent, L - m, X, NS, NX, D0, D1, D2, E0, E1, Z);
        } else {
          group_seed<T, FULL, true>(pcu + zs * aa, psu + zs * ba, zs, K, aa, ba, D0, D1, D2);
          group_sum<T, FULL, true>(ent, L - m, X, NS, NX, D0, D1, D2, Z);
          if (FULL) {
            // d'' = -cot(b) d' + (Q - l(l+1)) d with Q = (m^2 + n^2 - 2mn cos b) / sin^2 b,
            // the numerator as (m - n)^2 + 4mn sin^2(b/2) (beta <= pi/2) or
            // (m + n)^2 - 4mn cos^2(b/2) (beta > pi/2), free of cancellation at the pole
            const v2<T> mm = vset<T>(T(m), T(m)), nh = vset<T>(T(na), T(na + 1));
            const v2<T> dd = vfma(nh, QSG, mm);
            const v2<T> Q = vmul(vfma(vmul(mm, nh), QC4, vmul(dd, dd)), IS2);
#pragma unroll
            for (int q = 0; q < 4; ++q) Z[8 + q] = vfma(NCOT, Z[4 + q], vfma(Q, Z[q], Z[8 + q]));
          }
        }
        const T fm = T(m), fa = T(na);
        const v2<T> MM = vset<T>(fm, fm), NN = vset<T>(fa, fa + T(1));
        // image (m, n): phase e^{i(m a + n g)}, weight 1 for (0, 0) else 2
        // (the image (-m, -n) is the conjugate); an empty half has weight 0
        {
          v2<T> ER, EI, NEI;
          T ar, ai;
          lds1(eacu + zs * m, ar);
          lds1(easu + zs * m, ai);
          phase<T>(vset<T>(ar, ar), vset<T>(ai, ai), vld<T>(egcu + zs * na, egcu + zs * (na + 1)),
                   vld<T>(egsu + zs * na, egsu + zs * (na + 1)), ER, EI, NEI);
          const v2<T> Wt = vset<T>(m == 0 ? T(1) : T(2), na < m ? T(2) : T(0));
          add_image<T, FULL>(acc, Wt, MM, NN, ER, EI, NEI, Z[0], Z[1], Z[4], Z[5], Z[8], Z[9]);
        }
        // image (n, m): c^l_nm d^l_nm e^{i(n a + m g)}, d^l_nm = (-1)^{m-n} d^l_mn
        // (m - n even in the first half, odd in the second); absent when n = +-m
        {
          v2<T> ER, EI, NEI;
          T gr, gi;
          lds1(egcu + zs * m, gr);
          lds1(egsu + zs * m, gi);
          phase<T>(vld<T>(eacu + zs * na, eacu + zs * (na + 1)),
                   vld<T>(easu + zs * na, easu + zs * (na + 1)), vset<T>(gr, gr), vset<T>(gi, gi),
                   ER, EI, NEI);
          const v2<T> Wt = vset<T>(na == m || na == -m ? T(0) : T(2), na + 1 < m ? T(-2) : T(0));
          add_image<T, FULL>(acc, Wt, NN, MM, ER, EI, NEI, Z[2], Z[3], Z[6], Z[7], Z[10], Z[11]);
        }
       }
      }
      __syncwarp(submask);
      cur ^= 1;
      ncur = nnext;
    }
    cp_async_wait<0>();
  }
  // both halves, then the sub-slots of the warp that follow the same candidate,
  // then (below) the warps in index order: all in the working precision
  const int nq = FULL ? 10 : 1;
  T r[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) r[i] = acc[i].x + acc[i].y;
  for (int o = cpw; o < 32; o <<= 1)
#pragma unroll
    for (int i = 0; i < 10; ++i)
      if (i < nq) r[i] += __shfl_xor_sync(0xffffffffu, r[i], o);
  if (lane < cpw && p < P)
#pragma unroll
    for (int i = 0; i < 10; ++i)
      if (i < nq) ((T *)sm.red)[(warp * P + p) * 10 + i] = r[i];
  __syncthreads();
  for (int idx = tid; idx < P * nq; idx += blockDim.x) {
    int pp = idx / nq, i = idx - pp * nq;
    if (need[pp]) {
      T v = 0;
      for (int w = 0; w < NEWTON_WARPS; ++w) v += ((const T *)sm.red)[(w * P + pp) * 10 + i];
      sm.res[pp * 10 + i] = (double)v;
    }
  }
  __syncthreads();
}

// x mod 2 pi in [0, 2 pi).  The refinement only meets |x| < 4 pi (a wrapped
// angle plus a clamped step, or plus pi after a reflection of beta), where a
// few compare-and-add steps give the same result as x - 2 pi floor(x / 2 pi)
// without a double-precision division; other inputs take that formula first.
__device__ __forceinline__ double mod2pi_d(double x) {
  const double t = 2.0 * M_PI;
  if (!(x < 4.0 * t && x >= -4.0 * t)) x -= t * floor(x / t);
  for (int k = 0; k < 4 && x >= t; ++k) x -= t;
  for (int k = 0; k < 4 && x < 0.0; ++k) x += t;
  return x;
}

__device__ __forceinline__ void wrap_d(double *v) {
  double a = v[0], b = v[1], g = v[2];
  if (b < 0) { b = -b; a += M_PI; g += M_PI; }
  else if (b > M_PI) { b = 2.0 * M_PI - b; a += M_PI; g += M_PI; }
  v[0] = mod2pi_d(a); v[1] = b; v[2] = mod2pi_d(g);
}

// Newton direction from grad g and Hessian H (row-major 3x3) in the solve
// precision S; returns flag bits.  A Cholesky pivot of -H counts as positive
// above piv_rel ||H||_F, set by the precision H was summed in (1e-12 for FP64
// sums, 1e-6 for FP32 sums: above the rounding level of H's entries).
template <typename S>
__device__ __forceinline__ int newton_dir(const S *g, const S *H, int L, S *d, double piv_rel,
                                          bool grad) {
  S hn = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) hn += H[i] * H[i];
  hn = sqrt(hn);
  const S tol = S(piv_rel) * hn;
  // Cholesky of A = -H
  S a00 = -H[0], a10 = -H[3], a20 = -H[6], a11 = -H[4], a21 = -H[7], a22 = -H[8];
  bool ok = !grad && a00 > tol;  // grad: the gradient method, never the Newton step
  S L00 = 0, L10 = 0, L20 = 0, L11 = 0, L21 = 0, L22 = 0;
  if (ok) {
    L00 = sqrt(a00); L10 = a10 / L00; L20 = a20 / L00;
    S p11 = a11 - L10 * L10;
    ok = p11 > tol;
    if (ok) {
      L11 = sqrt(p11); L21 = (a21 - L20 * L10) / L11;
      S p22 = a22 - L20 * L20 - L21 * L21;
      ok = p22 > tol;
      if (ok) L22 = sqrt(p22);
    }
  }
  int fl = 0;
  if (ok) {
    S y0 = g[0] / L00;
    S y1 = (g[1] - L10 * y0) / L11;
    S y2 = (g[2] - L20 * y0 - L21 * y1) / L22;
    S x2 = y2 / L22;
    S x1 = (y1 - L21 * x2) / L11;
    S x0 = (y0 - L10 * x1 - L20 * x2) / L00;
    d[0] = x0; d[1] = x1; d[2] = x2;
  } else {
    fl = grad ? 0 : 2;
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = hn > 0 ? g[i] / hn : S(0);
  }
  S nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  S cap = S(M_PI / (2.0 * (L + 1.0)));
  if (nrm > cap) {
    S f = cap / nrm;
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] *= f;
  }
  return fl;
}

// Candidate tid has C, grad, H of its current point in res: record C, stop on
// a non-finite value (flag bit 0), take the Newton direction (solved in
// precision S), stop the level when the increment is below step_tol, else
// prepare the first trial (angles in FP64).
template <typename S>
__device__ __forceinline__ void start_step(int tid, int L, const NewtonArgs &A, SmemLayout &sm,
                                           double piv_rel) {
  const double *r = sm.res + 10 * tid;
  const double C = r[0];
  const S g[3] = {S(r[1]), S(r[2]), S(r[3])};
  const S H[9] = {S(r[4]), S(r[5]), S(r[6]), S(r[5]), S(r[7]), S(r[8]), S(r[6]), S(r[8]), S(r[9])};
  bool fin = true;
#pragma unroll
  for (int i = 0; i < 10; ++i) fin = fin && isfinite(r[i]);
  sm.Cc[tid] = C;
  if (!fin) {
    sm.fl[tid] |= 1;
    sm.state[tid] = ST_DEAD;
    return;
  }
  S d[3];
  sm.fl[tid] |= newton_dir<S>(g, H, L, d, piv_rel, A.grad != 0);
  if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < S(A.tol)) {
    sm.state[tid] = ST_STOP;
    return;
  }
  double tr[3] = {sm.th[3 * tid] + (double)d[0], sm.th[3 * tid + 1] + (double)d[1],
                  sm.th[3 * tid + 2] + (double)d[2]};
  wrap_d(tr);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sm.del[3 * tid + i] = (double)d[i];
    sm.tr[3 * tid + i] = tr[i];
  }
  sm.tries[tid] = 0;
  sm.state[tid] = ST_TRIAL;
}

// Carves the refinement kernels' shared memory (layout of newton_smem_bytes).
template <typename T, bool RS>
__device__ __forceinline__ int *carve_smem(unsigned char *smem_raw, int P, int LJ, SmemLayout &sm) {
  double *dp = reinterpret_cast<double *>(smem_raw);
  sm.th = dp; dp += 3 * P;
  sm.tr = dp; dp += 3 * P;
  sm.del = dp; dp += 3 * P;
  sm.Cc = dp; dp += P;
  sm.res = dp; dp += 10 * P;
  int *ip = reinterpret_cast<int *>(dp);
  sm.state = ip; ip += P;
  sm.steps = ip; ip += P;
  sm.tries = ip; ip += P;
  sm.fl = ip; ip += P;
  int *need = ip; ip += P;
  uintptr_t u = reinterpret_cast<uintptr_t>(ip);
  u = (u + 15) & ~uintptr_t(15);
  T *tp = reinterpret_cast<T *>(u);
  sm.red = tp; tp += 10 * P * NEWTON_WARPS;
  sm.ea = tp; tp += 4 * cand_stride(P) * ph_row(LJ);
  sm.pw = tp; tp += (RS ? 4 : 2) * cand_stride(P) * pw_row(LJ);
  tp = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(tp) + 31) & ~uintptr_t(31));
  sm.stage = tp;
  for (int t = threadIdx.x; t < (RS ? 4 : 2) * cand_stride(P) * pw_row(LJ); t += blockDim.x)
    ((T *)sm.pw)[t] = T(0);  // pads
  return need;
}

// C_L, its gradient and Hessian (Section 2.2) at Q given rotations per
// particle: the refinement kernel's evaluation, one CTA per particle.
// out[b][q][10] = (C, C_a, C_b, C_g, C_aa, C_ab, C_ag, C_bb, C_bg, C_gg).
template <typename T, bool RS>
__global__ void __launch_bounds__(NEWTON_THREADS, sizeof(T) == 8 ? 1 : 2)
k_objective(const T *__restrict__ c, const T *__restrict__ rcoef, const T *__restrict__ seedK,
            NewtonArgs A, int L, int Q, const double *__restrict__ pts, double *__restrict__ out) {
  const long b = blockIdx.x;
  const int tid = threadIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout sm;
  int *need = carve_smem<T, RS>(smem_raw, A.P, A.LJ, sm);
  if (tid < A.P) {
    const bool on = tid < Q;
    for (int i = 0; i < 3; ++i) sm.th[3 * tid + i] = on ? pts[3 * (b * Q + tid) + i] : 0.0;
    need[tid] = on;
  }
  __syncthreads();
  evaluate<T, true, RS>(A, L, c + 4 * b * A.nc, rcoef, seedK, sm.th, need, sm);
  for (int t = tid; t < Q * 10; t += blockDim.x) out[10 * b * Q + t] = sm.res[t];
}

// The march of all candidates of particle b by the whole CTA.
template <typename T, bool RS>
__device__ __forceinline__ void newton_particle(const T *__restrict__ c, const T *__restrict__ rcoef,
                                                const T *__restrict__ seedK, const NewtonArgs &A,
                                                const int *__restrict__ n_cand,
                                                double *__restrict__ euler, double *__restrict__ score,
                                                int *__restrict__ cflags, long long *__restrict__ work,
                                                long b, unsigned char *smem_raw) {
  const int P = A.P, tid = threadIdx.x;
  SmemLayout sm;  // staging buffers: [slots][2][stage_half(L_J)]
  int *need = carve_smem<T, RS>(smem_raw, P, A.LJ, sm);
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
  const double piv_rel = sizeof(T) == 8 ? 1e-12 : 1e-6;  // H summed in T
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
    evaluate<T, true, RS>(A, L, cb, rcoef, seedK, sm.th, need, sm);
    // the 3x3 solves of the final level run in FP64 in every plan
    const bool last = lev == A.nlev - 1;
    auto step_from = [&]() {
      if (last) start_step<double>(tid, L, A, sm, piv_rel);
      else start_step<T>(tid, L, A, sm, piv_rel);
    };
    if (tid < P && need[tid]) {
      sm.steps[tid] = 0;
      step_from();
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
      if (full) evaluate<T, true, RS>(A, L, cb, rcoef, seedK, sm.tr, need, sm);
      else evaluate<T, false, RS>(A, L, cb, rcoef, seedK, sm.tr, need, sm);
      if (tid < P && need[tid]) {
        double Ct = sm.res[10 * tid];
        if (Ct >= sm.Cc[tid] - A.acc_tol * fabs(sm.Cc[tid])) {
          for (int i = 0; i < 3; ++i) sm.th[3 * tid + i] = sm.tr[3 * tid + i];
          sm.Cc[tid] = Ct;
          if (sm.steps[tid] < A.M - 1) {
            ++sm.steps[tid];
            step_from();  // derivatives at the accepted point
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

// One CTA per particle, in index order.
template <typename T, bool RS>
__global__ void __launch_bounds__(NEWTON_THREADS, sizeof(T) == 8 ? 1 : 2)
k_newton(const T *__restrict__ c, const T *__restrict__ rcoef,
         const T *__restrict__ seedK, NewtonArgs A, const int *__restrict__ n_cand,
         double *__restrict__ euler, double *__restrict__ score, int *__restrict__ cflags,
         long long *__restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  newton_particle<T, RS>(c, rcoef, seedK, A, n_cand, euler, score, cflags, work, blockIdx.x,
                         smem_raw);
}

// Persistent CTAs (as many as fit on the GPU at once) pulling particles from a
// cost-sorted queue: order[] lists the particles by decreasing refinement cost
// (candidates to march), and a CTA takes the next entry with an atomic ticket,
// so the most expensive particles start first and the cheap ones fill the tail
// (longest processing time first).  Each particle's arithmetic is that of
// k_newton, so the results are bit-identical.
template <typename T, bool RS>
__global__ void __launch_bounds__(NEWTON_THREADS, sizeof(T) == 8 ? 1 : 2)
k_newton_queue(const T *__restrict__ c, const T *__restrict__ rcoef, const T *__restrict__ seedK,
               NewtonArgs A, const int *__restrict__ n_cand, double *__restrict__ euler,
               double *__restrict__ score, int *__restrict__ cflags, long long *__restrict__ work,
               const int *__restrict__ order, int B, int *__restrict__ ticket) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int next;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next = atomicAdd(ticket, 1);
    __syncthreads();
    const int q = next;
    if (q >= B) break;
    newton_particle<T, RS>(c, rcoef, seedK, A, n_cand, euler, score, cflags, work, order[q],
                           smem_raw);
  }
}

// order[] = the particles by decreasing candidate count (stable in the index),
// by a counting sort in one CTA; also resets the queue's ticket.
__global__ void k_cost_order(const int *__restrict__ n_cand, int B, int P, int *__restrict__ order,
                             int *__restrict__ ticket) {
  __shared__ int start[MATCHA_MAX_P + 2];
  const int tid = threadIdx.x;
  if (tid <= P + 1) start[tid] = 0;
  __syncthreads();
  for (int b = tid; b < B; b += blockDim.x) atomicAdd(&start[P - min(max(n_cand[b], 0), P) + 1], 1);
  __syncthreads();
  if (tid == 0) {
    for (int k = 1; k <= P + 1; ++k) start[k] += start[k - 1];
    *ticket = 0;
  }
  __syncthreads();
  // stable placement: each bin is filled in index order by one warp per bin
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int k = warp; k <= P; k += nw) {
    int pos = start[k];
    for (int b0 = 0; b0 < B; b0 += 32) {
      const int b = b0 + lane;
      const bool in = b < B && P - min(max(n_cand[b], 0), P) == k;
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) order[pos + __popc(m & ((1u << lane) - 1u))] = b;
      pos += __popc(m);
    }
  }
}

// Lanes per warp sub-slot: one per candidate, at least 16.
static int newton_cpw(int P) { return P <= 16 ? 16 : 32; }

// Shared memory of k_newton with `slots` staging buffers.
// Above this bandwidth the 32-bit plans run the rescaled recurrence: seeds
// flushed below the FP32 range would otherwise grow into significant terms
// (at L_J = 100 a seed under 2^-126 reaches 2.6e-4).
constexpr int RESCALE_ABOVE_L = 64;
static bool newton_rescaled(const Plan &p, size_t tsize) { return tsize == 4 && p.LJ > RESCALE_ABOVE_L; }

static size_t newton_smem_bytes(const Plan &p, size_t tsize, int slots) {
  size_t P = p.P;
  const size_t pw_rows = newton_rescaled(p, tsize) ? 4 : 2;
  size_t bytes = sizeof(double) * (3 * P * 3 + P + 10 * P);
  bytes += sizeof(int) * 5 * P;
  bytes = (bytes + 15) / 16 * 16;
  const size_t PS = cand_stride(p.P);
  bytes += tsize * (10 * P * NEWTON_WARPS + 4 * PS * ph_row(p.LJ) + pw_rows * PS * pw_row(p.LJ)) + 32;
  bytes += tsize * (size_t)slots * 2 * stage_half(p.LJ);
  return bytes;
}

// Staging buffers that fit: one per sub-slot when possible, else fewer (the
// other sub-slots then idle); 0 when even one does not fit.
static int newton_slots(const Plan &p, size_t tsize) {
  const size_t limit = 227 * 1024;
  int slots = NEWTON_WARPS * (32 / newton_cpw(p.P));
  while (slots > 0 && newton_smem_bytes(p, tsize, slots) > limit) --slots;
  return slots;
}

bool newton_fits(const Plan &p) { return newton_slots(p, p.fp64 ? 8 : 4) > 0; }

template <typename T>
cudaError_t launch_newton(const Plan &p, const T *c, int B, const int *n_cand, double *euler,
                          double *score, int *cflags, long long *work, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  NewtonArgs A;
  A.LJ = p.LJ; A.nlev = p.nlev; A.M = p.M; A.P = p.P;
  A.cpw = newton_cpw(p.P);
  A.nslots = newton_slots(p, sizeof(T));
  if (A.nslots == 0) return cudaErrorInvalidConfiguration;
  for (int i = 0; i < MATCHA_MAX_LEVELS; ++i) A.Ls[i] = i < p.nlev ? p.Ls[i] : 0;
  A.tol = p.step_tol;
  A.acc_tol = p.accept_tol;
  A.grad = p.refine;
  A.nc = p.nc;
  size_t smem = newton_smem_bytes(p, sizeof(T), A.nslots);
  if constexpr (sizeof(T) == 4) {
    if (newton_rescaled(p, sizeof(T))) {
      cudaFuncSetAttribute(k_newton<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_newton<T, true><<<B, NEWTON_THREADS, smem, st>>>(c, (const T *)p.rcoef, (const T *)p.seedK,
                                                         A, n_cand, euler, score, cflags, work);
      return cudaGetLastError();
    }
  }
  cudaFuncSetAttribute(k_newton<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_newton<T, false><<<B, NEWTON_THREADS, smem, st>>>(c, (const T *)p.rcoef, (const T *)p.seedK,
                                                      A, n_cand, euler, score, cflags, work);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_newton_queue(const Plan &p, const T *c, int B, const int *n_cand, double *euler,
                                double *score, int *cflags, long long *work, int *order,
                                int *ticket, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  NewtonArgs A;
  A.LJ = p.LJ; A.nlev = p.nlev; A.M = p.M; A.P = p.P;
  A.cpw = newton_cpw(p.P);
  A.nslots = newton_slots(p, sizeof(T));
  if (A.nslots == 0) return cudaErrorInvalidConfiguration;
  for (int i = 0; i < MATCHA_MAX_LEVELS; ++i) A.Ls[i] = i < p.nlev ? p.Ls[i] : 0;
  A.tol = p.step_tol; A.acc_tol = p.accept_tol; A.grad = p.refine; A.nc = p.nc;
  const size_t smem = newton_smem_bytes(p, sizeof(T), A.nslots);
  k_cost_order<<<1, 1024, 0, st>>>(n_cand, B, p.P, order, ticket);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NEWTON_THREADS, smem);
    const int grid = std::max(1, std::min(B, std::max(per_sm, 1) * sms));
    kern<<<grid, NEWTON_THREADS, smem, st>>>(c, (const T *)p.rcoef, (const T *)p.seedK, A, n_cand,
                                             euler, score, cflags, work, order, B, ticket);
  };
  if constexpr (sizeof(T) == 4) {
    if (newton_rescaled(p, sizeof(T))) { go(k_newton_queue<T, true>); return cudaGetLastError(); }
  }
  go(k_newton_queue<T, false>);
  return cudaGetLastError();
}
template cudaError_t launch_newton_queue<float>(const Plan &, const float *, int, const int *,
                                                double *, double *, int *, long long *, int *,
                                                int *, cudaStream_t);
template cudaError_t launch_newton_queue<double>(const Plan &, const double *, int, const int *,
                                                 double *, double *, int *, long long *, int *,
                                                 int *, cudaStream_t);

template <typename T>
cudaError_t launch_objective(const Plan &p, const T *c, int B, int L, int Q, const double *pts,
                             double *out, cudaStream_t st) {
  if (B == 0 || Q == 0) return cudaSuccess;
  NewtonArgs A;
  A.LJ = p.LJ; A.nlev = p.nlev; A.M = p.M; A.P = p.P;
  A.cpw = newton_cpw(p.P);
  A.nslots = newton_slots(p, sizeof(T));
  if (A.nslots == 0) return cudaErrorInvalidConfiguration;
  for (int i = 0; i < MATCHA_MAX_LEVELS; ++i) A.Ls[i] = i < p.nlev ? p.Ls[i] : 0;
  A.tol = p.step_tol; A.acc_tol = p.accept_tol; A.grad = p.refine; A.nc = p.nc;
  size_t smem = newton_smem_bytes(p, sizeof(T), A.nslots);
  if constexpr (sizeof(T) == 4) {
    if (newton_rescaled(p, sizeof(T))) {
      cudaFuncSetAttribute(k_objective<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_objective<T, true><<<B, NEWTON_THREADS, smem, st>>>(c, (const T *)p.rcoef,
                                                            (const T *)p.seedK, A, L, Q, pts, out);
      return cudaGetLastError();
    }
  }
  cudaFuncSetAttribute(k_objective<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_objective<T, false><<<B, NEWTON_THREADS, smem, st>>>(c, (const T *)p.rcoef, (const T *)p.seedK,
                                                         A, L, Q, pts, out);
  return cudaGetLastError();
}
template cudaError_t launch_objective<float>(const Plan &, const float *, int, int, int,
                                             const double *, double *, cudaStream_t);
template cudaError_t launch_objective<double>(const Plan &, const double *, int, int, int,
                                              const double *, double *, cudaStream_t);

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
