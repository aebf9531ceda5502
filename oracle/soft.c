/*
 * Oracle: the SOFFT initialisation grid and the candidate selection
 * (Section 2.3; Algorithm 1, first two steps).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Grid: the equiangular grid of Kostelec and Rockmore at bandwidth L0+1,
 * oversampled K times: n = 2K(L0+1) points per angle,
 *   alpha_i = 2 pi i / n,  beta_k = pi (2k+1) / (2n),  gamma_j = 2 pi j / n,
 * about (K L0)^3 rotations, linear index (i*n + k)*n + j.  The oracle evaluates
 * C_{L0} by the direct Wigner sum at every grid point (no FFT).
 *
 * Local maxima ("the P strongest local maxima", Section 2.3): a grid point is
 * a local maximum when it precedes each of its 26 neighbours in the order
 * (value descending, index ascending); alpha and gamma wrap, beta neighbours
 * outside [0, n-1] are skipped.  Candidates are the local maxima in that same
 * order, the first P of them.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

int orc_soft_n(int L0, int K) { return 2 * K * (L0 + 1); }

void orc_soft_angles(int n, long idx, double *abg) {
  long i = idx / ((long)n * n), k = (idx / n) % n, j = idx % n;
  abg[0] = 2.0 * M_PI * i / n;
  abg[1] = M_PI * (2.0 * k + 1.0) / (2.0 * n);
  abg[2] = 2.0 * M_PI * j / n;
}

void orc_soft_grid(const double *c, int L0, int K, double *grid) {
  int n = orc_soft_n(L0, K);
  for (long idx = 0; idx < (long)n * n * n; ++idx) {
    double abg[3];
    orc_soft_angles(n, idx, abg);
    grid[idx] = orc_objective(c, L0, abg[0], abg[1], abg[2], NULL, NULL, NULL);
  }
}

/* a precedes b in (value desc, index asc) */
static int precedes(double va, long ia, double vb, long ib) {
  return va > vb || (va == vb && ia < ib);
}

typedef struct { double v; long i; } cand_t;

static int cmp_cand(const void *pa, const void *pb) {
  const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
  if (precedes(a->v, a->i, b->v, b->i)) return -1;
  if (precedes(b->v, b->i, a->v, a->i)) return 1;
  return 0;
}

/* Returns the number of local maxima kept (<= P). */
int orc_local_maxima_topk(const double *grid, int n, int P, int *idx, double *score) {
  long tot = (long)n * n * n, cnt = 0;
  cand_t *cs = (cand_t *)malloc(sizeof(cand_t) * tot);
  for (long p = 0; p < tot; ++p) {
    long i = p / ((long)n * n), k = (p / n) % n, j = p % n;
    double v = grid[p];
    int is_max = !isnan(v);
    for (int di = -1; di <= 1 && is_max; ++di)
      for (int dk = -1; dk <= 1 && is_max; ++dk)
        for (int dj = -1; dj <= 1 && is_max; ++dj) {
          if (!di && !dk && !dj) continue;
          long kk = k + dk;
          if (kk < 0 || kk >= n) continue;
          long ii = (i + di + n) % n, jj = (j + dj + n) % n;
          long q = (ii * n + kk) * n + jj;
          if (!precedes(v, p, grid[q], q)) is_max = 0;
        }
    if (is_max) { cs[cnt].v = v; cs[cnt].i = p; ++cnt; }
  }
  qsort(cs, cnt, sizeof(cand_t), cmp_cand);
  int kept = cnt < P ? (int)cnt : P;
  for (int q = 0; q < kept; ++q) { idx[q] = (int)cs[q].i; score[q] = cs[q].v; }
  free(cs);
  return kept;
}
