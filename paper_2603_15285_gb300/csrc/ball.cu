// Ball-harmonic radial basis with the eigenvalue truncation (Appendix "Ball
// harmonics expansion and eigenvalue-based truncation"): on the ball of
// radius R the radial functions of degree l are N_lk j_l(lambda_lk r / R),
// lambda_lk the k-th positive zero of the spherical Bessel function j_l
// (Dirichlet condition at r = R), N_lk^2 = 2 / (R^3 j_{l+1}(lambda_lk)^2)
// (unit norm in r^2 dr), and a degree keeps K_l = {k : lambda_lk <= Lambda}.
// The plan's projection table turns the shell SH coefficients into these
// coefficients with the radial Gauss-Legendre rule:
//   f_klm = sum_s w_s N_lk j_l(lambda_lk r_s / R) f_lm(r_s).
// Host code, run once at plan creation.
#include <cmath>
#include "internal.cuh"

namespace matcha {

namespace {

double jl(int l, double x) { return std::sph_bessel((unsigned)l, x); }

// The zero of j_l in (a, b), where j_l changes sign, by bisection to the
// last bit.
double bisect_zero(int l, double a, double b) {
  double fa = jl(l, a);
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    if (m <= a || m >= b) break;
    const double fm = jl(l, m);
    if (fm == 0.0) return m;
    if ((fm < 0) == (fa < 0)) { a = m; fa = fm; }
    else b = m;
  }
  return 0.5 * (a + b);
}

}  // namespace

int ball_tables(int L, int S, double R, double Lam, const double *r, const double *w,
                std::vector<double> &W, std::vector<int> &counts) {
  // zeros of j_0 are k pi; those of j_l interlace those of j_{l-1}:
  // lambda_{l-1,k} < lambda_{l,k} < lambda_{l-1,k+1}.  One more zero beyond
  // the last bracket is found by stepping up until j_l changes sign.
  std::vector<double> prev;
  for (int k = 1; k * M_PI <= Lam + 2 * M_PI; ++k) prev.push_back(k * M_PI);
  std::vector<std::vector<double>> zeros(L + 1);
  zeros[0] = prev;
  for (int l = 1; l <= L; ++l) {
    std::vector<double> cur;
    for (size_t k = 0; k + 1 < prev.size(); ++k) cur.push_back(bisect_zero(l, prev[k], prev[k + 1]));
    if (!prev.empty()) {
      double a = prev.back(), b = a + 0.5;
      while ((jl(l, a) < 0) == (jl(l, b) < 0)) b += 0.5;
      cur.push_back(bisect_zero(l, a, b));
    }
    zeros[l] = cur;
    prev = cur;
  }
  counts.assign(L + 1, 0);
  int kmax = 0;
  for (int l = 0; l <= L; ++l) {
    int n = 0;
    for (double z : zeros[l]) n += z <= Lam;
    counts[l] = n;
    kmax = n > kmax ? n : kmax;
  }
  W.assign((size_t)(L + 1) * (kmax > 0 ? kmax : 1) * S, 0.0);
  for (int l = 0; l <= L; ++l)
    for (int k = 0; k < counts[l]; ++k) {
      const double lam = zeros[l][k];
      const double N = std::sqrt(2.0 / (R * R * R)) / std::fabs(jl(l + 1, lam));
      for (int s = 0; s < S; ++s) W[((size_t)l * kmax + k) * S + s] = w[s] * N * jl(l, lam * r[s] / R);
    }
  return kmax;
}

}  // namespace matcha
