/* A plain C client of the library's C ABI (no Python, no PyTorch): a two-mesh Euler system,
 * a periodic 48 x 48 background on [-5, 5)^2 and a 33 x 33 patch on [-1, 1]^2 with interface
 * faces, uniform flow with a small quadratic density perturbation, MRAB order 3 at step ratio 2 for five macro
 * steps from the bootstrap; device buffers from cudaMalloc. Writes both meshes' initial and
 * then final states (the library's layout: 4 planes of nj rows of pitch values, doubles) to the
 * file argv[1], followed by both meshes' donor tables (sbp_get_tables: base, weights).
 * Test program for the ABI; returns non-zero on any failed call. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sbp_mrab.h"

#define TRY(call)                                                                          \
  do {                                                                                     \
    sbp_status st_ = (call);                                                               \
    if (st_ != SBP_OK) {                                                                   \
      fprintf(stderr, "%s: %s (%s)\n", #call, sbp_status_string(st_), sbp_last_error_message()); \
      return 1;                                                                            \
    }                                                                                      \
  } while (0)
#define CTRY(call)                                                      \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));       \
      return 1;                                                         \
    }                                                                   \
  } while (0)

int main(int argc, char **argv) {
  if (argc < 2) {
    fprintf(stderr, "usage: %s out.bin [0: autotuner off] [macro steps, default 5]\n", argv[0]);
    return 2;
  }
  const double gam = 1.4, u0 = 0.5;
  sbp_mesh_desc m[2];
  memset(m, 0, sizeof m);
  m[0].n[0] = m[0].n[1] = 48;
  m[0].periodic[0] = m[0].periodic[1] = 1;
  for (int f = 0; f < 4; ++f) m[0].bc[f] = SBP_BC_PERIODIC;
  m[0].cartesian = 1;
  m[0].lo[0] = m[0].lo[1] = -5.0;
  m[0].h[0] = m[0].h[1] = 10.0 / 48;
  m[0].shift[0] = 10.0;  /* i wrap: (10, 0) */
  m[0].shift[3] = 10.0;  /* j wrap: (0, 10) */
  m[1].n[0] = m[1].n[1] = 33;
  for (int f = 0; f < 4; ++f) m[1].bc[f] = SBP_BC_INTERFACE;
  m[1].cartesian = 1;
  m[1].lo[0] = m[1].lo[1] = -1.0;
  m[1].h[0] = m[1].h[1] = 2.0 / 32;

  sbp_params p;
  memset(&p, 0, sizeof p);
  p.physics = SBP_EULER;
  p.dtype = SBP_F64;
  p.gamma = gam;
  p.pr = 0.72;
  p.twall = 1.0;
  p.omega_corner = 1.0;
  p.sigma_interface = 0.5;
  p.sigma_physical = 1.0;
  p.cfl = 0.5;
  p.qinf[0] = 1.0;
  p.qinf[1] = u0;
  p.qinf[3] = 1.0 / (gam * (gam - 1.0)) + 0.5 * u0 * u0;
  p.order = 3;
  p.hist_len = 3;
  p.step_ratio = 2;
  p.fast_mesh = 1;

  /* argv[4] = "xy": hand over coordinate arrays (lo + i h) instead of lo/h alone */
  double *xy[2][2] = {{NULL, NULL}, {NULL, NULL}};
  if (argc > 4 && strcmp(argv[4], "xy") == 0)
    for (int k = 0; k < 2; ++k) {
      const size_t n = (size_t)m[k].n[0] * m[k].n[1];
      xy[k][0] = (double *)malloc(n * sizeof(double));
      xy[k][1] = (double *)malloc(n * sizeof(double));
      for (int j = 0; j < m[k].n[1]; ++j)
        for (int i = 0; i < m[k].n[0]; ++i) {
          xy[k][0][(size_t)j * m[k].n[0] + i] = m[k].lo[0] + m[k].h[0] * i;
          xy[k][1][(size_t)j * m[k].n[0] + i] = m[k].lo[1] + m[k].h[1] * j;
        }
      m[k].x = xy[k][0];
      m[k].y = xy[k][1];
    }
  sbp_system_t sys = NULL;
  TRY(sbp_system_create(m, 2, &p, &sys));
  FILE *out = fopen(argv[1], "wb");
  if (!out) return 1;
  void *qa[2], *qb[2], *hist[2];
  double *host[2];
  sbp_mesh_info inf[2];
  for (int k = 0; k < 2; ++k) {
    TRY(sbp_mesh_info_get(sys, k, &inf[k]));
    const size_t field = inf[k].field_elems;
    host[k] = (double *)calloc(4 * field, sizeof(double));
    for (int j = 0; j < inf[k].nj; ++j)
      for (int i = 0; i < inf[k].ni; ++i) {
        const double x = m[k].lo[0] + i * m[k].h[0], y = m[k].lo[1] + j * m[k].h[1];
        const double rho = 1.0 + 0.01 * (x * x - y * y) / 25.0;
        const double pr = 1.0 / gam;
        const size_t o = (size_t)j * inf[k].pitch + i;
        host[k][o] = rho;
        host[k][field + o] = rho * u0;
        host[k][2 * field + o] = 0.0;
        host[k][3 * field + o] = pr / (gam - 1.0) + 0.5 * rho * u0 * u0;
      }
    fwrite(host[k], 1, inf[k].state_bytes, out);  /* the initial state, then the final one */
    CTRY(cudaMalloc(&qa[k], inf[k].state_bytes));
    CTRY(cudaMalloc(&qb[k], inf[k].state_bytes));
    CTRY(cudaMalloc(&hist[k], inf[k].hist_bytes));
    CTRY(cudaMemcpy(qa[k], host[k], inf[k].state_bytes, cudaMemcpyHostToDevice));
    TRY(sbp_bind(sys, k, qa[k], qb[k], hist[k]));
  }
  if (argc > 2 && argv[2][0] == '0') TRY(sbp_autotune(sys, 0, NULL));  /* keep the default kernel shapes */
  TRY(sbp_mrab_init(sys, 0.0, NULL));
  TRY(sbp_mrab_step(sys, argc > 3 ? atoi(argv[3]) : 5, NULL));
  TRY(sbp_check(sys, NULL));
  double H = 0.0, t = 0.0;
  TRY(sbp_mrab_time(sys, &H, &t));
  for (int k = 0; k < 2; ++k) {
    void *cur = NULL;
    TRY(sbp_current_state(sys, k, &cur));
    CTRY(cudaMemcpy(host[k], cur, inf[k].state_bytes, cudaMemcpyDeviceToHost));
    fwrite(host[k], 1, inf[k].state_bytes, out);
  }
  /* the donor tables, for comparison with other clients: base (2 ints) and weights (8 doubles)
   * per receiver */
  for (int k = 0; k < 2; ++k) {
    const int nr = inf[k].n_receivers;
    int *base = (int *)calloc(2 * (size_t)nr + 1, sizeof(int));
    double *w = (double *)calloc(8 * (size_t)nr + 1, sizeof(double));
    TRY(sbp_get_tables(sys, k, NULL, NULL, NULL, base, w));
    fwrite(base, sizeof(int), 2 * (size_t)nr, out);
    fwrite(w, sizeof(double), 8 * (size_t)nr, out);
    free(base);
    free(w);
  }
  fclose(out);
  printf("H %.17g t %.17g\n", H, t);
  TRY(sbp_system_destroy(sys));
  for (int k = 0; k < 2; ++k) {
    cudaFree(qa[k]);
    cudaFree(qb[k]);
    cudaFree(hist[k]);
    free(host[k]);
  }
  return 0;
}
