/*
 * Oracle: samples of a voxel volume on the radial shells of the ball.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper expands each volume in ball harmonics through a NUFFT (Section 1.1,
 * Appendix A.1-A.2).  This path instead samples the volume on the quadrature
 * points of the ball: point (s, j, k) sits at c0 + r_s (sin t_j cos p_k,
 * sin t_j sin p_k, cos t_j) in voxel units (x, y, z), c0 = N/2, and its value
 * is the trilinear interpolation of the voxel values (zero outside the box).
 */
#include <math.h>
#include "oracle.h"

static double voxel(const float *vol, int N, long i, long j, long k) {
  if (i < 0 || j < 0 || k < 0 || i >= N || j >= N || k >= N) return 0.0;
  return (double)vol[(k * N + j) * N + i];
}

double orc_trilinear(const float *vol, int N, double px, double py, double pz) {
  double fx0 = floor(px), fy0 = floor(py), fz0 = floor(pz);
  long i = (long)fx0, j = (long)fy0, k = (long)fz0;
  double tx = px - fx0, ty = py - fy0, tz = pz - fz0;
  double v = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double wgt = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
        v += wgt * voxel(vol, N, i + dx, j + dy, k + dz);
      }
  return v;
}

/* samples[s][j][k], s < S, j < n_theta = L+1, k < n_phi = 2L+2. */
void orc_sample_shells(const float *vol, int N, int S, double R, int L, double *samples) {
  double r[S], wr[S], x[L + 1], wx[L + 1];
  int nt, np;
  orc_radial_nodes(S, R, r, wr);
  orc_angular_grid(L, x, wx, &nt, &np);
  double c0 = 0.5 * N;
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < nt; ++j) {
      double st = sqrt(1.0 - x[j] * x[j]);
      for (int k = 0; k < np; ++k) {
        double ph = 2.0 * M_PI * k / np;
        double px = c0 + r[s] * st * cos(ph);
        double py = c0 + r[s] * st * sin(ph);
        double pz = c0 + r[s] * x[j];
        samples[((long)s * nt + j) * np + k] = orc_trilinear(vol, N, px, py, pz);
      }
    }
}

/*
 * Pose of a voxel volume (the appendix on alternating search over rotations
 * and translations): out(x) = vol(R^T (x - c0) + c0 - s) at every voxel
 * centre x, trilinear, zero outside, rounded to float32 like any volume.
 * With R = I this is the translation (S_s vol)(x) = vol(x - s); with s = 0 it
 * is the rotation g o vol about c0.  R is row-major; s = (x, y, z) voxels.
 */
void orc_transform_volume(const float *vol, int N, const double *R, const double *s, float *out) {
  double c0 = 0.5 * N;
  for (long k = 0; k < N; ++k)
    for (long j = 0; j < N; ++j)
      for (long i = 0; i < N; ++i) {
        double x = i - c0, y = j - c0, z = k - c0;
        /* R^T x: column c of R dotted with x */
        double px = R[0] * x + R[3] * y + R[6] * z + c0 - s[0];
        double py = R[1] * x + R[4] * y + R[7] * z + c0 - s[1];
        double pz = R[2] * x + R[5] * y + R[8] * z + c0 - s[2];
        out[(k * N + j) * N + i] = (float)orc_trilinear(vol, N, px, py, pz);
      }
}
