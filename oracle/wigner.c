/*
 * Oracle: Wigner small-d functions, their beta derivatives, and the ZYZ chart.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * d^l_{mn}(b) = <l m| exp(-i b J_y) |l n> are the real functions in the
 * factorisation D^l_{mn}(a,b,g) = exp(-i m a) d^l_{mn}(b) exp(-i n g)
 * (Eq. wigner-D, Appendix A.4).  Three routes are written here:
 *
 *  1. the three-term recurrence in l (Kostelec and Rockmore) seeded at
 *     l = max(|m|,|n|) with the closed form of the corner entries;
 *  2. Wigner's explicit finite sum, in long double (the "explicit expressions
 *     in terms of finite sums" of Appendix A.4), which cancels badly at high l
 *     and is used only to cross-check route 1 at moderate l;
 *  3. beta derivatives from d'(b) = d(b) Y with Y = -i J_y, the real
 *     tridiagonal matrix of the ladder relation (Appendix A.4 notes that the
 *     beta derivatives are finite combinations of neighbouring entries);
 *     applying Y twice gives d''.
 *
 * The ZYZ chart is Eq. (Euler): g(a,b,g) = r_z(a) r_y(b) r_z(g).
 */
#include <math.h>
#include "oracle.h"

static double binom(int a, int b) {
  double r = 1.0;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

static double ipow(double x, int p) {
  double r = 1.0;
  for (int i = 0; i < p; ++i) r *= x;
  return r;
}

/* d^j_{j n}(b) = sqrt(C(2j, j+n)) cos(b/2)^{j+n} (-sin(b/2))^{j-n}. */
static double corner(int j, int n, double beta) {
  double c = cos(0.5 * beta), s = sin(0.5 * beta);
  return sqrt(binom(2 * j, j + n)) * ipow(c, j + n) * ipow(-s, j - n);
}

/* d^j_{mn} at j = max(|m|,|n|), from the corner formula and the symmetries
 * d_{mn} = (-1)^{m-n} d_{nm} = d_{-n,-m}. */
static double seed(int m, int n, double beta) {
  int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
  int j = am > an ? am : an;
  if (m == j) return corner(j, n, beta);
  if (m == -j) return (((j + n) & 1) ? -1.0 : 1.0) * corner(j, -n, beta);
  if (n == j) return (((j - m) & 1) ? -1.0 : 1.0) * corner(j, m, beta);
  return corner(j, -m, beta); /* n == -j */
}

void orc_wigner_d(int L, double beta, double *d) {
  double x = cos(beta);
  for (int l = 0; l <= L; ++l)
    for (int m = -l; m <= l; ++m)
      for (int n = -l; n <= l; ++n) d[orc_c_index(l, m, n)] = 0.0;
  for (int m = -L; m <= L; ++m)
    for (int n = -L; n <= L; ++n) {
      int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
      int l0 = am > an ? am : an;
      double dprev = 0.0, dcur = seed(m, n, beta);
      d[orc_c_index(l0, m, n)] = dcur;
      for (int l = l0; l < L; ++l) {
        double dnext;
        if (l == 0) {
          dnext = x; /* d^1_00 = cos(b) */
        } else {
          double mm = (double)m * m, nn = (double)n * n, l1 = l + 1.0;
          double num_a = (2.0 * l + 1.0) * ((double)l * l1 * x - (double)m * n);
          double num_b = l1 * sqrt(((double)l * l - mm) * ((double)l * l - nn));
          double den = l * sqrt((l1 * l1 - mm) * (l1 * l1 - nn));
          dnext = (num_a * dcur - num_b * dprev) / den;
        }
        dprev = dcur;
        dcur = dnext;
        d[orc_c_index(l + 1, m, n)] = dcur;
      }
    }
}

static long double factl(int k) {
  long double r = 1.0L;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}

/* Wigner's formula, with the bra index m and the ket index n:
 * d^l_{mn}(b) = sum_k (-1)^{k-n+m} sqrt((l+n)!(l-n)!(l+m)!(l-m)!)
 *               / ((l+n-k)! k! (l-k-m)! (k-n+m)!)
 *               cos(b/2)^{2l-2k+n-m} sin(b/2)^{2k-n+m}. */
double orc_wigner_d_finite_sum(int l, int m, int n, double beta) {
  long double c = cosl(0.5L * beta), s = sinl(0.5L * beta);
  long double pre = sqrtl(factl(l + n) * factl(l - n) * factl(l + m) * factl(l - m));
  long double sum = 0.0L;
  for (int k = 0; k <= 2 * l; ++k) {
    int a1 = l + n - k, a2 = l - k - m, a3 = k - n + m;
    if (a1 < 0 || a2 < 0 || a3 < 0) continue;
    long double term = pre / (factl(a1) * factl(k) * factl(a2) * factl(a3));
    int pc = 2 * l - 2 * k + n - m, ps = 2 * k - n + m;
    long double cp = 1.0L, sp = 1.0L;
    for (int i = 0; i < pc; ++i) cp *= c;
    for (int i = 0; i < ps; ++i) sp *= s;
    term *= cp * sp;
    if ((k - n + m) & 1) term = -term;
    sum += term;
  }
  return (double)sum;
}

/* Right-multiply each d^l by Y = -i J_y:
 * (dY)_{mn} = 1/2 [ sqrt((l+n)(l-n+1)) d_{m,n-1} - sqrt((l-n)(l+n+1)) d_{m,n+1} ]. */
static void times_Y(int L, const double *in, double *out) {
  for (int l = 0; l <= L; ++l)
    for (int m = -l; m <= l; ++m)
      for (int n = -l; n <= l; ++n) {
        double v = 0.0;
        if (n - 1 >= -l) v += sqrt((double)(l + n) * (l - n + 1)) * in[orc_c_index(l, m, n - 1)];
        if (n + 1 <= l) v -= sqrt((double)(l - n) * (l + n + 1)) * in[orc_c_index(l, m, n + 1)];
        out[orc_c_index(l, m, n)] = 0.5 * v;
      }
}

void orc_wigner_d_derivs(int L, double beta, double *d, double *d1, double *d2) {
  orc_wigner_d(L, beta, d);
  times_Y(L, d, d1);
  times_Y(L, d1, d2);
}

static void matmul3(const double *A, const double *B, double *C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

/* R = r_z(a) r_y(b) r_z(g), row-major (Eq. Euler). */
void orc_euler_to_matrix(double a, double b, double g, double *R) {
  double rza[9] = {cos(a), -sin(a), 0, sin(a), cos(a), 0, 0, 0, 1};
  double ryb[9] = {cos(b), 0, sin(b), 0, 1, 0, -sin(b), 0, cos(b)};
  double rzg[9] = {cos(g), -sin(g), 0, sin(g), cos(g), 0, 0, 0, 1};
  double t[9];
  matmul3(ryb, rzg, t);
  matmul3(rza, t, R);
}

/* Inverse of the chart on (0, pi) in beta; at beta = 0 or pi, gamma = 0. */
void orc_matrix_to_euler(const double *R, double *abg) {
  double sb = sqrt(R[2] * R[2] + R[5] * R[5]);
  double b = atan2(sb, R[8]);
  double a, g;
  if (sb > 1e-12) {
    a = atan2(R[5], R[2]);
    g = atan2(R[7], -R[6]);
  } else if (R[8] > 0) {
    a = atan2(R[3], R[0]);
    g = 0.0;
  } else {
    a = atan2(-R[3], -R[0]);
    g = 0.0;
  }
  if (a < 0) a += 2 * M_PI;
  if (g < 0) g += 2 * M_PI;
  abg[0] = a; abg[1] = b; abg[2] = g;
}

/* Geodesic angle 2 asin(||R1 - R2||_F / (2 sqrt 2)). */
double orc_rotation_angle(const double *R1, const double *R2) {
  double s = 0.0;
  for (int i = 0; i < 9; ++i) s += (R1[i] - R2[i]) * (R1[i] - R2[i]);
  double t = sqrt(s) / (2.0 * sqrt(2.0));
  if (t > 1.0) t = 1.0;
  return 2.0 * asin(t);
}
