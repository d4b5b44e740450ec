/* Plain-C client of the fetipe C ABI (include/fetipe.h): no Python, no torch.
 *
 * Usage: abi_steps NSUB_X NSUB_Y CELLS ORDER_K N_STEPS PRECISION(0 fp64 | 1 mixed) TOL
 * Builds the uniform partition (the lower half of the subdomain rows poroelastic), the
 * stationary manufactured solution of Test Case 1 with lambda = mu = alpha = c0 = K = mu_f = 1
 * and tau = 1e-3, runs N_STEPS backward-Euler steps and prints, one per line,
 *   "step <n> <iterations> <true relative residual>"   for every step, then
 *   "lambda <n_lambda>" and the multipliers of the last step, one "%.17g" per line.
 * Exit status: 0 on success, otherwise the fp_status of the failing call (its message on
 * stderr).  Without a CUDA device fp_create fails with FP_ERR_CUDA. */
#include <stdio.h>
#include <stdlib.h>

#include "fetipe.h"

static int fail(const char *what, fp_status st, const fp_handle *h) {
  fprintf(stderr, "%s: status %d: %s\n", what, (int)st, fp_last_error(h));
  return (int)st;
}

int main(int argc, char **argv) {
  if (argc != 8) {
    fprintf(stderr, "usage: %s NSUB_X NSUB_Y CELLS ORDER_K N_STEPS PRECISION TOL\n", argv[0]);
    return 1;
  }
  const int nsx = atoi(argv[1]), nsy = atoi(argv[2]), cells = atoi(argv[3]), k = atoi(argv[4]);
  const int n_steps = atoi(argv[5]), precision = atoi(argv[6]);
  const double tol = atof(argv[7]);
  if (nsx < 1 || nsy < 2 || cells < 1 || n_steps < 1) return 1;

  int *cx = (int *)malloc(sizeof(int) * (size_t)nsx), *cy = (int *)malloc(sizeof(int) * (size_t)nsy);
  if (!cx || !cy) return 2;
  for (int i = 0; i < nsx; ++i) cx[i] = cells;
  for (int j = 0; j < nsy; ++j) cy[j] = cells;
  fp_mesh_desc mesh;
  mesh.nsub_x = nsx;
  mesh.nsub_y = nsy;
  mesh.cells_x = cx;
  mesh.cells_y = cy;
  mesh.poro_rows = nsy / 2;
  mesh.order_k = k;

  fp_params par;
  par.lame_lambda = 1.0;
  par.mu = 1.0;
  par.alpha = 1.0;
  par.c0 = 1.0;
  par.perm_k = 1.0;
  par.mu_f = 1.0;
  par.tau = 1e-3;
  par.perm = NULL;
  par.source = FP_SOURCE_MANUFACTURED;
  par.src_i = 0;
  par.src_j = 0;
  par.q_omega = 0.0;
  par.precision = precision ? FP_PREC_MIXED : FP_PREC_FP64;
  par.precond = FP_PRECOND_DIRICHLET;
  par.tol = tol;
  par.max_it = 1000;

  fp_handle *h = NULL;
  fp_status st = fp_create(&mesh, &par, NULL, &h);
  free(cx);
  free(cy);
  if (st != FP_OK) return fail("fp_create", st, NULL);
  if ((st = fp_assemble(h)) != FP_OK) return fail("fp_assemble", st, h);
  if ((st = fp_factor(h)) != FP_OK) return fail("fp_factor", st, h);
  for (int n = 0; n < n_steps; ++n) {
    fp_step_stats stats;
    if ((st = fp_step(h, &stats)) != FP_OK) return fail("fp_step", st, h);
    printf("step %d %d %.6e\n", stats.step, stats.iterations, stats.true_rel_residual);
  }
  fp_sizes sz;
  if ((st = fp_get_sizes(h, &sz)) != FP_OK) return fail("fp_get_sizes", st, h);
  double *lam = (double *)malloc(sizeof(double) * (size_t)(sz.n_lambda > 0 ? sz.n_lambda : 1));
  if (!lam) return 2;
  if ((st = fp_get_lambda(h, lam, 0)) != FP_OK) return fail("fp_get_lambda", st, h);
  printf("lambda %d\n", sz.n_lambda);
  for (int i = 0; i < sz.n_lambda; ++i) printf("%.17g\n", lam[i]);
  free(lam);
  fp_destroy(h);
  return 0;
}
