// Plan tables (step a0): quadrature nodes and weights, normalised Legendre
// values, DFT twiddles, the l-recurrence coefficients of the Wigner small-d
// functions and the SOFFT beta table.  All computed on the device in FP64;
// FP32 plans get a rounded copy.
//
// Definitions: Gauss-Legendre rules for the radius and cos(theta) (the ball
// and sphere integrals of Section 2 and Appendix A.1); Pbar_lm normalised so
// that Pbar_lm(cos t) e^{imp} is orthonormal on the sphere with the
// Condon-Shortley phase; Wigner d^l_{mn}(b) = <lm|exp(-i b J_y)|ln>
// (Appendix A.4, Eq. wigner-D) through the three-term recurrence in l
//   d^{l+1} = (a cos b - b') d^l - e d^{l-1},
//   a  = (2l+1)(l+1) / Q_{l+1},  b' = (2l+1) m n / (l Q_{l+1}),
//   e  = (l+1) Q_l / (l Q_{l+1}),  Q_j = sqrt((j^2 - m^2)(j^2 - n^2)),
// seeded at l = m >= |n| by d^m_{mn} = sqrt(C(2m, m+n)) cos(b/2)^{m+n} (-sin(b/2))^{m-n}.
#include <math.h>
#include "internal.cuh"

namespace matcha {

// One thread per node: Newton iteration on P_n, nodes ascending.
__global__ void k_gauss_legendre(int n, double *x, double *w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double z = cos(M_PI * (i + 0.75) / (n + 0.5));
  double p0 = 1, p1 = z, dp = 1;
  for (int it = 0; it < 100; ++it) {
    p0 = 1; p1 = z;
    for (int k = 1; k < n; ++k) { double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1); p0 = p1; p1 = p2; }
    if (n == 1) { p1 = z; p0 = 1; }
    dp = n * (z * p1 - p0) / (z * z - 1);
    double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  p0 = 1; p1 = z;
  for (int k = 1; k < n; ++k) { double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1); p0 = p1; p1 = p2; }
  dp = n * (z * p1 - p0) / (z * z - 1);
  x[n - 1 - i] = z;
  w[n - 1 - i] = 2.0 / ((1 - z * z) * dp * dp);
}

__global__ void k_radial(int S, double R, const double *xg, const double *wg, double *r, double *w) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double rr = 0.5 * R * (1.0 + xg[s]);
  r[s] = rr;
  w[s] = 0.5 * R * wg[s] * rr * rr;
}

__device__ double plm_bar_dev(int l, int m, double x) {
  double st = sqrt(fmax(0.0, 1.0 - x * x));
  double pmm = 0.28209479177387814347;  // 1/sqrt(4 pi)
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * st;
  if (l == m) return pmm;
  double pa = pmm, pb = sqrt(2.0 * m + 3.0) * x * pmm;
  for (int k = m + 2; k <= l; ++k) {
    double a = sqrt((4.0 * k * k - 1.0) / ((double)(k - m) * (k + m)));
    double b = sqrt(((double)(k - 1 - m) * (k - 1 + m)) / (4.0 * (k - 1) * (k - 1) - 1.0));
    double pc = a * (x * pb - b * pa);
    pa = pb; pb = pc;
  }
  return pb;
}

// ptab[j][lm] = w_j (2 pi / n_phi) Pbar_lm(x_j)  (lm fastest)
__global__ void k_ptab(int L, int nt, int np, const double *xj, const double *wj, double *pt) {
  int nlm = (L + 1) * (L + 2) / 2;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlm * nt) return;
  int j = t / nlm, lm = t - j * nlm;
  int l = 0;
  while ((l + 1) * (l + 2) / 2 <= lm) ++l;
  int m = lm - l * (l + 1) / 2;
  pt[t] = wj[j] * (2.0 * M_PI / np) * plm_bar_dev(l, m, xj[j]);
}

__global__ void k_twiddle(int n, double *cs) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi(2.0 * k / n, &s, &c);
  cs[2 * k] = c;
  cs[2 * k + 1] = s;
}

// Recurrence coefficients of every (pair q, l) in the grouped layout: reals
// pair_base[q] + 8 (l - m) + {0, 2, 4, 6} = (a, -b, -e, 0) of the step
// d^{l+1} = (a x - b) d^l - e d^{l-1}; zero at l = L.  The empty half of each
// m's last group (partner of n = m) is zero.
__global__ void k_rcoef(int L, int npairs, const int *pair_base, double *rc) {
  int q = blockIdx.x;
  if (q >= npairs) return;
  int m = 0;
  while ((m + 1) * (m + 1) <= q) ++m;
  int n = q - m * m - m;
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    double a = 0, b = 0, e = 0;
    if (l < L) {
      if (l == 0) {
        a = 1.0;  // d^1_00 = cos(b) d^0_00
      } else {
        double mm = (double)m * m, nn = (double)n * n, l1 = l + 1.0, ll = l;
        double q1 = sqrt((l1 * l1 - mm) * (l1 * l1 - nn));
        double q0 = sqrt((ll * ll - mm) * (ll * ll - nn));
        a = (2 * ll + 1) * l1 / q1;
        b = (2 * ll + 1) * (double)m * n / (ll * q1);
        e = l1 * q0 / (ll * q1);
      }
    }
    double *o = rc + pair_base[q] + 8L * (l - m);
    o[0] = a; o[2] = -b; o[4] = -e; o[6] = -(double)l * (l + 1);  // -l(l+1): the d'' equation
    if (n == m) { o[1] = 0; o[3] = 0; o[5] = 0; o[7] = 0; }
  }
}

__device__ double seed_norm(int m, int n) {
  // sqrt(C(2m, m+n)), C(2m, m+n) = prod_{i=1}^{m-n} (m+n+i)/i
  double c = 1.0;
  for (int i = 1; i <= m - n; ++i) c = c * (m + n + i) / i;
  return sqrt(c);
}

// seedK[g] = (K(m, n_a), K(m, n_b), 0, 0) for partner group g; K of the empty
// half is zero, so its recurrence stays at zero.
__global__ void k_seedK(int ngroups, double *K) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  int m = 0;
  while ((m + 1) * (m + 2) / 2 <= g) ++m;
  int j = g - m * (m + 1) / 2, na = 2 * j - m;
  K[4 * g] = seed_norm(m, na);
  K[4 * g + 1] = na + 1 <= m ? seed_norm(m, na + 1) : 0.0;
  K[4 * g + 2] = K[4 * g + 3] = 0.0;
}

__device__ double ipow_d(double x, int p) {
  double r = 1.0;
  while (p) { if (p & 1) r *= x; x *= x; p >>= 1; }
  return r;
}

// soft_d[k][pair_off0[q] + l - m] = d^l_mn(beta_k), l = m..L0, by the recurrence.
__global__ void k_soft_d(int L0, int ns, int npairs0, const int *pair_base, const int *pair_off0,
                         const double *rc, const double *K, long nc0, double *out) {
  int q = blockIdx.x, k = blockIdx.y;
  if (q >= npairs0 || threadIdx.x != 0) return;
  int m = 0;
  while ((m + 1) * (m + 1) <= q) ++m;
  int n = q - m * m - m;
  int g = m * (m + 1) / 2 + ((n + m) >> 1), h = (n + m) & 1;
  double beta = M_PI * (2.0 * k + 1.0) / (2.0 * ns);
  double ch = cos(0.5 * beta), sh = sin(0.5 * beta), x = cos(beta);
  double d = K[4 * g + h] * ipow_d(ch, m + n) * ipow_d(-sh, m - n), dp = 0.0;
  double *o = out + (long)k * nc0 + pair_off0[q];
  const double *r = rc + pair_base[q];
  for (int l = m; l <= L0; ++l) {
    o[l - m] = d;
    const double *c = r + 8 * (l - m);
    double dn = (c[0] * x + c[2]) * d + c[4] * dp;
    dp = d; d = dn;
  }
}

// Folded phi-DFT table.  With np = n_phi and k' = np/2 - k,
//   cos(2 pi m k'/np) = (-1)^m cos(2 pi m k/np),
//   sin(2 pi m k'/np) = (-1)^(m+1) sin(2 pi m k/np),
// so the sums over k = 1..np/2-1 fold onto q = 1..Qf.  Entry
// cs[p][0][q-1][c] = cos(2 pi m q / np), cs[p][1][q-1][c] = sin(2 pi m q / np)
// for the order m = 2c + p of parity p (zero for m > L).
__global__ void k_dft_cs(int L, int Qf, int Mq, double *cs) {
  const int np = 2 * L + 2;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * Qf * Mq) return;
  int p = t / (Qf * Mq), rem = t - p * Qf * Mq, q = rem / Mq + 1, c = rem - (q - 1) * Mq;
  int m = 2 * c + p;
  double sv = 0.0, cv = 0.0;
  if (m <= L) sincospi(2.0 * ((long)m * q % np) / np, &sv, &cv);
  cs[(2 * p) * Qf * Mq + rem] = cv;
  cs[(2 * p + 1) * Qf * Mq + rem] = sv;
}

// Ring constants of the shell sampling: ring r = s * nt + j lies in the plane
// z = N/2 + r_s cos t_j with radius r_s sin t_j.
__global__ void k_ring(int S, int nt, int N, const double *rs, const double *xj, double *ring) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= S * nt) return;
  int s = r / nt, j = r - s * nt;
  double rr = rs[s], x = xj[j];
  ring[2 * r] = rr * sqrt(fmax(1.0 - x * x, 0.0));
  ring[2 * r + 1] = 0.5 * N + rr * x;
}

__global__ void k_to_float(const double *in, float *out, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// The Legendre table with its columns in the analysis' item order:
// out[j][t] = in[j][lm(t)].
template <typename T>
__global__ void k_ptab_leg(int nt, int nlm, const int *leg, const T *in, T *out) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)nt * nlm) return;
  const int j = (int)(t / nlm), c = (int)(t - (long)j * nlm);
  const int l = leg[c] >> 16, m = leg[c] & 0xffff;
  out[t] = in[(long)j * nlm + l * (l + 1) / 2 + m];
}

cudaError_t build_tables(Plan &p, cudaStream_t st) {
  // scratch for the FP64 versions of the real tables
  size_t n_ptab = (size_t)p.nlm * p.nt, n_phi = 2 * (size_t)p.np, n_tw = 2 * (size_t)p.ns;
  size_t n_softd = (size_t)p.ns * p.nc0, n_rc = 4 * (size_t)p.nc, n_K = 4 * (size_t)p.ngroups;
  size_t n_dcs = 4 * (size_t)p.Qf * p.Mq, n_ring = 2 * (size_t)p.S * p.nt;
  double *gx, *gw;
  cudaError_t e;
  if ((e = cudaMalloc(&gx, sizeof(double) * 2 * p.S))) return e;
  gw = gx + p.S;
  k_gauss_legendre<<<(p.S + 63) / 64, 64, 0, st>>>(p.S, gx, gw);
  k_radial<<<(p.S + 63) / 64, 64, 0, st>>>(p.S, p.R, gx, gw, p.rs, p.wrad);
  k_gauss_legendre<<<(p.nt + 63) / 64, 64, 0, st>>>(p.nt, p.xj, p.wj);
  double *d64 = nullptr;
  size_t tot = n_ptab + n_phi + n_tw + n_softd + n_rc + n_K + n_dcs + n_ring;
  if (!p.fp64) {
    if ((e = cudaMalloc(&d64, sizeof(double) * tot))) { cudaFree(gx); return e; }
  }
  double *ptab = p.fp64 ? (double *)p.ptab : d64;
  double *phi = p.fp64 ? (double *)p.phi_cs : ptab + n_ptab;
  double *tw = p.fp64 ? (double *)p.soft_tw : phi + n_phi;
  double *sd = p.fp64 ? (double *)p.soft_d : tw + n_tw;
  double *rc = p.fp64 ? (double *)p.rcoef : sd + n_softd;
  double *K = p.fp64 ? (double *)p.seedK : rc + n_rc;
  double *dcs = p.fp64 ? (double *)p.dft_cs : K + n_K;
  double *ring = p.fp64 ? (double *)p.ring : dcs + n_dcs;
  k_ptab<<<(unsigned)((n_ptab + 127) / 128), 128, 0, st>>>(p.LJ, p.nt, p.np, p.xj, p.wj, ptab);
  k_twiddle<<<(p.np + 127) / 128, 128, 0, st>>>(p.np, phi);
  k_twiddle<<<(p.ns + 127) / 128, 128, 0, st>>>(p.ns, tw);
  k_rcoef<<<p.npairs, 64, 0, st>>>(p.LJ, p.npairs, p.pair_base, rc);
  k_seedK<<<(p.ngroups + 127) / 128, 128, 0, st>>>(p.ngroups, K);
  k_dft_cs<<<(unsigned)((n_dcs / 2 + 127) / 128), 128, 0, st>>>(p.LJ, p.Qf, p.Mq, dcs);
  k_ring<<<(unsigned)((n_ring / 2 + 127) / 128), 128, 0, st>>>(p.S, p.nt, p.N, p.rs, p.xj, ring);
  k_soft_d<<<dim3(p.npairs0, p.ns), 32, 0, st>>>(p.L0, p.ns, p.npairs0, p.pair_base, p.pair_off0,
                                                 rc, K, p.nc0, sd);
  if (!p.fp64) {
    struct { double *src; void *dst; size_t n; } cp[] = {
        {ptab, p.ptab, n_ptab}, {phi, p.phi_cs, n_phi}, {tw, p.soft_tw, n_tw},
        {sd, p.soft_d, n_softd}, {rc, p.rcoef, n_rc}, {K, p.seedK, n_K},
        {dcs, p.dft_cs, n_dcs}, {ring, p.ring, n_ring}};
    for (auto &c : cp)
      k_to_float<<<(unsigned)((c.n + 255) / 256), 256, 0, st>>>(c.src, (float *)c.dst, (long)c.n);
  }
  {
    const unsigned nb = (unsigned)((n_ptab + 255) / 256);
    if (p.fp64)
      k_ptab_leg<double><<<nb, 256, 0, st>>>(p.nt, p.nlm, p.leg_lm, (const double *)p.ptab,
                                               (double *)p.ptab_leg);
    else
      k_ptab_leg<float><<<nb, 256, 0, st>>>(p.nt, p.nlm, p.leg_lm, (const float *)p.ptab,
                                              (float *)p.ptab_leg);
  }
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (d64) cudaFree(d64);
  cudaFree(gx);
  return e ? e : e2;
}

}  // namespace matcha
