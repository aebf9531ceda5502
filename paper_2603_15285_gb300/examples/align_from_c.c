/*
 * Rotational alignment from C through the library's C ABI alone (no Python):
 * reads B particle volumes and B template volumes (raw float32, C order
 * [b][z][y][x], N^3 each), runs Algorithm 1 with matcha_align_host and prints
 * one line per particle: best candidate, score and the ZYZ Euler angles.
 *
 *   align_from_c N S L0 K P M_iter B particles.f32 templates.f32 L_1 ... L_J
 *
 * (L_sched = L0 L_1 ... L_J; FP64 plan; the CUDA runtime supplies the device
 * workspace the caller owns.)
 */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include "matcha.h"

static float *read_f32(const char *path, size_t count) {
  FILE *f = fopen(path, "rb");
  if (!f) return NULL;
  float *buf = (float *)malloc(sizeof(float) * count);
  size_t got = buf ? fread(buf, sizeof(float), count, f) : 0;
  fclose(f);
  if (got != count) { free(buf); return NULL; }
  return buf;
}

int main(int argc, char **argv) {
  if (argc < 11) {
    fprintf(stderr, "usage: %s N S L0 K P M_iter B particles.f32 templates.f32 L_1 ... L_J\n", argv[0]);
    return 2;
  }
  matcha_plan_desc d = {0};
  d.box_n = atoi(argv[1]);
  d.n_shells = atoi(argv[2]);
  d.L0 = atoi(argv[3]);
  d.K_oversample = atoi(argv[4]);
  d.P_max = atoi(argv[5]);
  d.M_iter = atoi(argv[6]);
  const int B = atoi(argv[7]);
  d.n_levels = 1 + (argc - 10);
  if (d.n_levels > MATCHA_MAX_LEVELS) return 2;
  d.L_sched[0] = d.L0;
  for (int i = 10; i < argc; ++i) d.L_sched[i - 9] = atoi(argv[i]);
  d.precision = MATCHA_FP64;
  const size_t vox = (size_t)d.box_n * d.box_n * d.box_n;
  float *parts = read_f32(argv[8], vox * B), *temps = read_f32(argv[9], vox * B);
  if (!parts || !temps) { fprintf(stderr, "cannot read the volumes\n"); return 1; }

  matcha_plan plan;
  matcha_status s = matcha_plan_create(&d, &plan);
  if (s != MATCHA_OK) { fprintf(stderr, "plan: %s (%s)\n", matcha_status_string(s), matcha_last_error()); return 1; }
  size_t wsb = 0;
  matcha_host_workspace_size(plan, B, 1, &wsb);
  void *ws = NULL;
  if (cudaMalloc(&ws, wsb) != cudaSuccess) { fprintf(stderr, "cudaMalloc failed\n"); return 1; }
  double *euler = (double *)malloc(sizeof(double) * 3 * B), *R = (double *)malloc(sizeof(double) * 9 * B);
  double *score = (double *)malloc(sizeof(double) * B);
  int *best = (int *)malloc(sizeof(int) * B), *flags = (int *)malloc(sizeof(int) * B);
  s = matcha_align_host(plan, parts, temps, B, 1, euler, R, score, best, flags, ws, wsb, NULL);
  if (s != MATCHA_OK) { fprintf(stderr, "align: %s (%s)\n", matcha_status_string(s), matcha_last_error()); return 1; }
  for (int b = 0; b < B; ++b)
    printf("%d %d %.17g %.17g %.17g %.17g %d\n", b, best[b], score[b], euler[3 * b], euler[3 * b + 1],
           euler[3 * b + 2], flags[b]);
  cudaFree(ws);
  matcha_plan_destroy(plan);
  free(parts); free(temps); free(euler); free(R); free(score); free(best); free(flags);
  return 0;
}
