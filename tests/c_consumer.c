/* A plain C99 program that uses the library through include/elas.h alone (no Python, no torch):
 * the Eshelby inclusion cell of Sec. 3.1's validation in its small form (n^3 voxels, a centred
 * sphere of radius r of E = 400 GPa, nu = 0.25 in a matrix of E = 200 GPa, nu = 0.3, strain
 * eps_11 = 1e-3), FP64, point-block Jacobi PCG to Algorithm 2's criterion 1e-10, then the voxel
 * stress and its macroscopic mean.  Device memory comes from the CUDA runtime, as a C caller's
 * would.  Prints "status iters relres_true macro_11 macro_22" and exits 0 when converged.
 * Usage: c_consumer n r */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "elas.h"

int main(int argc, char** argv) {
  const int n = argc > 1 ? atoi(argv[1]) : 12;
  const double r = argc > 2 ? atof(argv[2]) : 3.0;
  const long long N = (long long)n * n * n;
  int32_t* phase = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  double C[72], strain[6] = {1e-3, 0.0, 0.0, 0.0, 0.0, 0.0}, macro[6];
  size_t ws_bytes = 0;
  void* ws = NULL;
  elas_ctx* ctx = NULL;
  elas_solve_info info;
  long long v;
  int rc;
  if (!phase) return 2;
  for (v = 0; v < N; ++v) {
    const double x = (double)(v % n) + 0.5 - 0.5 * n;
    const double y = (double)((v / n) % n) + 0.5 - 0.5 * n;
    const double z = (double)(v / ((long long)n * n)) + 0.5 - 0.5 * n;
    phase[v] = x * x + y * y + z * z <= r * r ? 1 : 0;
  }
  if (elas_isotropic_stiffness(200.0, 0.3, C) != ELAS_OK || elas_isotropic_stiffness(400.0, 0.25, C + 36) != ELAS_OK)
    return 3;
  if (elas_workspace_bytes(n, n, n, 2, ELAS_PREC_FP64, &ws_bytes) != ELAS_OK) return 4;
  if (cudaMalloc(&ws, ws_bytes) != cudaSuccess) return 5;
  rc = elas_create(&ctx, n, n, n, phase, 2, C, NULL, ELAS_PREC_FP64, ws, ws_bytes, NULL);
  if (rc != ELAS_OK) {
    fprintf(stderr, "elas_create: %s\n", elas_last_error(NULL));
    return 6;
  }
  rc = elas_pcg_solve(ctx, strain, 1e-10, 5000, NULL, NULL, &info);
  if (rc != ELAS_OK) {
    fprintf(stderr, "elas_pcg_solve: %s\n", elas_last_error(ctx));
    return 7;
  }
  rc = elas_stress(ctx, strain, NULL, NULL, NULL, macro);
  if (rc != ELAS_OK) {
    fprintf(stderr, "elas_stress: %s\n", elas_last_error(ctx));
    return 8;
  }
  printf("%d %d %.17g %.17g %.17g\n", info.status, info.iters, info.relres_true, macro[0], macro[1]);
  elas_destroy(ctx);
  cudaFree(ws);
  free(phase);
  return info.status == ELAS_CONVERGED ? 0 : 1;
}
