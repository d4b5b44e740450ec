/*
 * fetipe -- FETI interface solver for quasi-static poroelasticity coupled with elasticity,
 * multiphysics finite elements, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Ge & Wang, "A Parallel Solver with Multiphysics Finite Element Method for
 * Poroelasticity Coupled with Elasticity Model", arXiv 2509.06673.
 *
 * Problem statement (Sec. 2.5, Problem 2.4): given a triangulation of the unit square
 * Omega = Omega^P (y < 1/2, Biot poroelasticity) U Omega^E (y > 1/2, linear elasticity),
 * parameters (Table 2), boundary and initial data, compute for n = 1..N the backward-Euler
 * solution (u_h^n, xi_h^n, eta_h^n, p_h^n) and the interface multiplier lambda_h^n.
 * Each step is solved by FETI (Sec. 3): PCG (Algorithm 1) on F lambda = d with
 * F = sum_s B_s K_s^+ B_s^T (Eq. (3.6)) and the Dirichlet preconditioner (Eq. (3.5)),
 * plus the FETI-1 rigid-mode coarse projection for floating subdomains.
 *
 * Conventions of every call:
 *  - All calls return fp_status; FP_OK is 0.  fp_last_error() gives a message.
 *  - No call aborts the process.  A failed call leaves the handle valid; calls that need
 *    an earlier stage (fp_step before fp_factor, ...) return FP_ERR_STATE.
 *  - Input arrays are copied during the call; the caller keeps ownership.
 *  - Output arrays are caller-owned.  `on_device` = 0: host memory; 1: device memory of
 *    the handle's device (e.g. a torch tensor's data_ptr()).
 *  - One CUDA stream per handle (the `cuda_stream` given to fp_create; NULL = legacy
 *    default stream).  Calls are synchronous with respect to the host unless stated.
 *  - The handle owns all the device memory it allocates; fp_destroy frees it.
 */
#ifndef FETIPE_H
#define FETIPE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fp_handle fp_handle;

typedef enum {
  FP_OK = 0,
  FP_ERR_INVALID = 1,        /* bad argument or inconsistent mesh/partition */
  FP_ERR_OOM = 2,            /* device or host allocation failed */
  FP_ERR_CUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error) */
  FP_ERR_NOT_CONVERGED = 4,  /* max_it reached before the stop test held */
  FP_ERR_BREAKDOWN = 5,      /* PCG breakdown (p^T F p = 0 or non-finite values) */
  FP_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  FP_ERR_STATE = 7           /* call out of order (e.g. fp_step before fp_factor) */
} fp_status;

enum { FP_SOURCE_MANUFACTURED = 0, FP_SOURCE_POINT = 1, FP_SOURCE_MANUFACTURED_T = 2 };
enum { FP_PREC_FP64 = 0, FP_PREC_MIXED = 1 };
/* Preconditioner: DIRICHLET W B S B^T W (Eq. (3.5)); LUMPED W B K_bb B^T W, the interface
 * block of the local 3-field matrices in place of their Schur complement (Sec. 3.3: the M_A
 * of Algorithm 2 reduces to it), no local solve; NONE; AUTO: fp_factor times probe runs of
 * Algorithm 1 with DIRICHLET and LUMPED and keeps the one with the smaller predicted time
 * to the tolerance (see fp_get_tuning). */
enum { FP_PRECOND_DIRICHLET = 0, FP_PRECOND_LUMPED = 1, FP_PRECOND_NONE = 2, FP_PRECOND_AUTO = 3 };

/*
 * Partition and mesh (Sec. 2.4; Sec. 4.1 uses uniform triangulations).  The unit square is
 * cut into nsub_x x nsub_y rectangular subdomains, numbered s = cy * nsub_x + cx from the
 * bottom-left.  Partition column cx has cells_x[cx] cells across, partition row cy has
 * cells_y[cy] cells up, so meshes match on every interface.  Rows cy < poro_rows are
 * poroelastic (poro_rows = nsub_y / 2 puts the P/E interface at y = 1/2).  Every cell is
 * cut by its '/' diagonal into triangles (v00, v10, v11) and (v00, v11, v01); element
 * e = 2 * (j * nx + i) + t within a subdomain.  Displacement: P_k, k = order_k (1 or 2);
 * xi, eta, p: P1 (Sec. 2.4).  u = 0 on the boundary of the square; p = 0 on the outer
 * boundary of Omega^P (no-flux on y = 1/2, Eq. (2.14)).
 */
typedef struct {
  int nsub_x, nsub_y;   /* 1 <= nsub_x <= 4096, 2 <= nsub_y <= 4096 */
  const int *cells_x;   /* [nsub_x], each in [1, 4096] */
  const int *cells_y;   /* [nsub_y], each in [1, 4096] */
  int poro_rows;        /* 1 <= poro_rows < nsub_y */
  int order_k;          /* 1 or 2 */
} fp_mesh_desc;

/*
 * Physical and solver parameters (Table 2 of the paper; the multiphysics constants
 * kappa_1..3 of Sec. 2.2 follow from lame_lambda, alpha, c0).
 *  perm: NULL (uniform perm_k) or one value per element of every subdomain, subdomains in
 *        id order, elements in the order above (host pointer, copied).
 *  source: FP_SOURCE_MANUFACTURED -- the closed-form solution of Test Case 1 (Sec. 4.1)
 *            with its sources; eta^0 is the L2 projection of c0 p + alpha div u.
 *          FP_SOURCE_MANUFACTURED_T -- the same closed form times g(t) = 1 + t (every
 *            source times g(t); z gains g'(t) eta_0); backward Euler is exact in time for it.
 *          FP_SOURCE_POINT -- f = 0 and a point fluid source z = sin(q_omega t) at the P1
 *            vertex with global P1 grid indices (src_i, src_j) (must lie strictly inside
 *            one poroelastic subdomain); zero initial data.
 *  precision: FP_PREC_FP64 -- local factors and solves in FP64.
 *             FP_PREC_MIXED -- local factors and solves in FP32, outer PCG, coarse problem
 *             and refinement residuals in FP64.
 *  tol: PCG stops when ||P(d - F lambda)||_2 <= tol * ||P(d - F lambda_00)||_2.
 */
typedef struct {
  double lame_lambda, mu, alpha, c0;
  double perm_k, mu_f;
  double tau;
  const double *perm;
  int source;
  int src_i, src_j;
  double q_omega;
  int precision;
  int precond;
  double tol;
  int max_it;
} fp_params;

typedef struct {
  int nsub, n_floating, n_lambda, n_lambda_p;
  long long n_dofs;          /* sum of local 3-field dofs (u, xi, p) */
  long long n_unode_total;   /* length of the u field / 2 in fp_get_fields */
  long long n_pnode_total;   /* length of xi, eta, p in fp_get_fields */
  long long factor_bytes;    /* device bytes of all local factors */
  int max_half_band;
} fp_sizes;

typedef struct {
  int step;                  /* n of the step just solved */
  int iterations;            /* PCG iterations */
  double rel_residual;       /* recursive ||P r|| / ||P(d - F lambda_00)|| at exit */
  double true_rel_residual;  /* the same with r recomputed from lambda at exit */
  int lambda0_learned;       /* 1 if the learned guess moved lambda_0 off the lambda^{n-1} guess:
                                the guess selector minimises the true residual over the span of lambda^{n-1},
                                the extrapolation and the network's correction (see
                                fp_learned_use) */
  double guess_res_prev;     /* relative true residual of the lambda^{n-1} guess (-1: not computed) */
  double guess_res_learned;  /* relative true residual of the learned lambda_0 (-1: not computed) */
  int restarts;              /* restarts of Algorithm 1 from the true residual */
  int stagnations;           /* rounds stopped because the recursive residual stalled */
  long long h2d_bytes;       /* host -> device bytes the step copied (per-step scalars, loop flags) */
  long long d2h_bytes;       /* device -> host bytes the step copied (loop flags, scalars, status);
                                the caller's fp_get_* reads are not included */
  long long kernel_launches; /* kernels of the library this step launched ("graph" 1: the kernel
                                nodes of the step graph, of its outer loop body per round and of
                                its inner loop body per execution, counted on the device, plus the
                                sample-recording kernels; -1 with "graph" 0, not counted) */
} fp_step_stats;

/* Copies the mesh description and parameters, builds the dof numbering, band ordering and
 * interface tables on the host and uploads them to the current device.
 * cuda_stream: a cudaStream_t (NULL = default stream).  Errors: FP_ERR_INVALID (bad mesh or
 * parameters), FP_ERR_OOM (host or device allocation), FP_ERR_CUDA (no usable device, or a
 * CUDA call failed; there is no host fallback).  *out is NULL on error; fp_last_error(NULL)
 * gives the message. */
fp_status fp_create(const fp_mesh_desc *mesh, const fp_params *params, void *cuda_stream,
                    fp_handle **out);

/* Assembles every local matrix (the 3-field blocks of Sec. 3.1 with eta eliminated, see
 * below) and load vector on the device, and the coarse matrix G^T G.  Time-invariant
 * (tau is fixed, Sec. 2.5), so called once.  Local 3-field block of a poroelastic
 * subdomain, unknowns (u, xi, p):
 *   [ A        B^T            0                          ]
 *   [ B      -R/lambda       (alpha/lambda) R            ]
 *   [ 0      (alpha/lambda) R  -((c0 + alpha^2/lambda) R + tau A_f) ]
 * obtained from Eq. (2.43) by eta = (p - kappa_1 xi) / kappa_2 (exact since W_h = M_h^P);
 * elastic: [[A, B^T], [B, -R/lambda]]. */
fp_status fp_assemble(fp_handle *h);

/* Factors every local matrix: LDL^T (no pivoting; the 3-field blocks are symmetric
 * quasi-definite) of the Neumann matrix K_s (three displacement dofs fixed on floating
 * subdomains, giving the generalised inverse K_s^+) and of the Dirichlet matrix (K_s with
 * identity rows on the dofs touched by B_s, giving S_s of Eq. (3.5)), and the coarse
 * inverse (G^T G)^{-1}.  Idempotent. */
fp_status fp_factor(fp_handle *h);

/* Solves one backward-Euler step (Problem 2.4) with FETI: right-hand side, d = B K^+ f,
 * lambda_0 from lambda^{n-1} (Algorithm 1) projected onto G^T lambda = e, PCG, recovery of
 * (u, xi, p) per subdomain and eta = (c0 + alpha^2/lambda) p - (alpha/lambda) xi.
 * stats may be NULL.  Returns FP_ERR_NOT_CONVERGED / FP_ERR_BREAKDOWN with the state of
 * the last iterate kept. */
fp_status fp_step(fp_handle *h, fp_step_stats *stats);

/* Initial conditions (Sec. 2.5): replaces the initial state that fp_assemble set (R eta^0
 * from the configured source's closed-form initial data, zero for the point source) by the
 * one of the given nodal fields: eta_0 = c0 p0 + alpha div u0 (Eq. 2.17), R eta^0 =
 * (eta_0, phi_i) over every poroelastic subdomain with u0, p0 interpolated in P_k and P1
 * (every node, Dirichlet nodes included).  u0, p0: host arrays in the layout of
 * fp_get_fields (u 2 per displacement node, p one per P1 node, subdomains in id order),
 * NULL for zero.  Also resets the step counter and the lambda history to zero; the given
 * fields are what fp_get_fields returns until the first step.  After fp_assemble
 * (FP_ERR_STATE before). */
fp_status fp_set_initial(fp_handle *h, const double *u0, const double *p0);

/* Runs n_steps steps back to back (same as calling fp_step n_steps times); stops at the first
 * step that does not return FP_OK and returns its status.  FP_ERR_INVALID for n_steps < 0. */
fp_status fp_run(fp_handle *h, int n_steps, fp_step_stats *last);

/* Sizes of the handle's problem (host struct), valid from fp_create on. */
fp_status fp_get_sizes(const fp_handle *h, fp_sizes *out);

/* Host-only planning: validates mesh and params as fp_create does, builds the dof numbering
 * and interface tables on the host and reports the sizes fp_get_sizes would report for that
 * problem (factor_bytes: the device bytes of the local factors at params->precision), without
 * any CUDA call, so a problem can be sized against device memory before fp_create.
 * lambda_keys: NULL, or [6 * n_lambda] ints that receive the key of every multiplier row in
 * the format and order of fp_get_lambda_keys (call once with NULL to learn n_lambda).
 * Errors: FP_ERR_INVALID, FP_ERR_OOM; fp_last_error(NULL) gives the message. */
fp_status fp_plan(const fp_mesh_desc *mesh, const fp_params *params, fp_sizes *out, int *lambda_keys);

/* lambda^n of the last step, n_lambda doubles.  Multiplier r enforces
 * x_{s_a} - x_{s_b} = 0 on one node component (see fp_get_lambda_keys). */
fp_status fp_get_lambda(const fp_handle *h, double *dst, int on_device);

/* Six ints per multiplier (host): kind (0 displacement, 1 pressure), component (0/1),
 * global grid index I, J (displacement grid of order k for kind 0, P1 grid for kind 1),
 * s_a, s_b (s_a < s_b; the row is +1 on s_a, -1 on s_b). */
fp_status fp_get_lambda_keys(const fp_handle *h, int *keys);

/* Fields of the last step on the subdomain node grids, subdomains in id order:
 * u: 2 doubles per displacement node ((k*ny+1) x (k*nx+1) per subdomain, row-major, x
 * fastest); xi, eta, p: one double per P1 node ((ny+1) x (nx+1) per subdomain); eta and p
 * are zero on elastic subdomains.  Any pointer may be NULL. */
fp_status fp_get_fields(const fp_handle *h, double *u, double *xi, double *eta, double *p,
                        int on_device);

/* The same fields of one subdomain s (0 <= s < nsub_x * nsub_y, id = row * nsub_x + column):
 * u 2 (k*nx+1)(k*ny+1) doubles, xi, eta, p (nx+1)(ny+1) doubles each.  Any pointer may be
 * NULL.  FP_ERR_INVALID for s out of range. */
fp_status fp_get_subdomain(const fp_handle *h, int s, double *u, double *xi, double *eta, double *p,
                           int on_device);

/* Checkpoint / restore of the time-stepping state: step counter, lambda^n, lambda^{n-1},
 * R eta^n, the last fields, the source-signal history, the learned-guess network (its
 * parameters, Adam moments and step, and whether it is in use) and the refinement's
 * measured contraction.  Not stored: matrices and
 * factors (fp_assemble / fp_factor rebuild them bit for bit), options, recorded training
 * samples.  fp_restore needs a handle of the same problem after fp_assemble (FP_ERR_STATE
 * before; FP_ERR_INVALID for a file of another problem, a bad or truncated file); the
 * next fp_step continues exactly where the checkpointed run would have.  Host file I/O,
 * synchronous. */
fp_status fp_checkpoint(const fp_handle *h, const char *path);
fp_status fp_restore(fp_handle *h, const char *path);

/* Operator applications on multiplier vectors of length n_lambda (after fp_factor):
 * out = F v (Eq. (3.6)), out = M^{-1} v (Eq. (3.5), scaled by W = (B B^T)^{-1} on both
 * sides), out = P v (coarse projection).  v and out may not alias. */
fp_status fp_apply_F(fp_handle *h, const double *v, double *out, int on_device);
fp_status fp_apply_precond(fp_handle *h, const double *v, double *out, int on_device);
fp_status fp_apply_projection(fp_handle *h, const double *v, double *out, int on_device);

/* Same result as fp_apply_projection, for callers that cannot allocate device memory at
 * call time: an application that reserves the device's memory for its own pool up front (so
 * a library cudaMalloc fails or breaks its budget), or a latency-bound loop that may not take
 * cudaMalloc's implicit device synchronisation.  The paper has no counterpart: this is a
 * library convenience.  v and out are device pointers of the handle's device (n_lambda
 * doubles; they may alias).  The call allocates nothing: its scratch (two vectors of
 * 3 * n_floating doubles) is a fixed array of 2 * 24576 doubles (384 KiB) compiled into the
 * library and kept on every device that loads it until the process exits; a problem with
 * more than 8192 floating subdomains is rejected with FP_ERR_INVALID (checked first, right
 * after fp_create).  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make that first call
 * before any stream capture, and do not use the library across cudaDeviceReset.  Every call
 * shares the array and leaves its last contents there: calls that overlap on the GPU (other
 * streams, other threads, other handles on the same device) race; serialise them.  The call
 * waits for its kernels (it synchronises the handle's stream) and reports their errors. */
fp_status fp_apply_projection_noalloc(fp_handle *h, const double *v, double *out);

/* Local dof map of subdomain s (host, n_s ints each): field (0 u_x, 1 u_y, 2 xi, 3 p) and
 * node index on the subdomain's grid (displacement grid for u, P1 grid otherwise). */
fp_status fp_get_dof_map(const fp_handle *h, int s, int *field, int *node, int *n_out);

/* Dense copy (host, n_s * n_s doubles, row-major) of the assembled local matrix of
 * subdomain s in its band ordering (lower band mirrored).  For tests of small subdomains. */
fp_status fp_get_local_matrix(const fp_handle *h, int s, double *dense);

/* Device time of the last fp_step split by phase (milliseconds, CUDA events):
 * [0] right-hand side, d and the initial guess, [1] the PCG loop with its restarts,
 * [2] recovery and history; [3] the number of restarts of the step. */
fp_status fp_get_step_timing(const fp_handle *h, double *ms4);

/* ---------------- learned initial guess (not in the paper: a library pattern) ----------
 * A 3-layer MLP (8 -> 256 -> 256 -> 1, ReLU; the 256 x 256 products on tensor cores with
 * bfloat16 operands and FP32 accumulation) maps per-multiplier features (the last increment
 * dl = lambda^{n-1} - lambda^{n-2} and lambda^{n-1}, each divided by its RMS; the ratio rho of
 * the last two increments of the source's time signal; three products of these; kind and
 * component; every input clamped to [-8, 8]) to a correction of the source-scaled
 * extrapolation, in units of s = RMS(dl).  With fp_learned_use on, fp_step forms the
 * directions tc = P(rho dl) and tb = P(s MLP) from lambda_a = lambda_00 + P lambda^{n-1} and
 * takes lambda_0 = lambda_a + a tc + b tb with (a, b) minimising the true projected residual
 * ||P(d - F lambda_0)||_2 (the guess selector: a 2 x 2 least-squares problem, two more accurate F
 * applications); (a, b) = (0, 0), the previous-step guess, is the fallback and never beaten
 * by the result.  Parameters: one flat FP32 array of
 * 68353 values: W1 [8 x 256] row-major, b1 [256], W2 [256 x 256] row-major, b2 [256],
 * W3 [256], b3 [1]. */
/* Recording of training samples: with on = 1, every later fp_step with two earlier steps of
 * history stores per_step (features, target) pairs, multipliers taken at an even stride, in a
 * device store of max_samples pairs (grown, keeping what it holds, when max_samples exceeds
 * its capacity; FP_ERR_OOM if it cannot be); the target is what the extrapolation misses,
 * (lambda^n - lambda^{n-1} - rho dl) / s, the network's output units.  Recording stops silently when the store is full.  on = 0 stops it.
 * FP_ERR_INVALID for max_samples < 0 or per_step < 1. */
fp_status fp_learned_record(fp_handle *h, int on, long long max_samples, int per_step);
/* Use (on = 1) or not the learned guess in fp_step; FP_ERR_STATE while the network has no
 * parameters (fp_mlp_init, fp_mlp_set_params or fp_learned_train first). */
fp_status fp_learned_use(fp_handle *h, int on);
/* Trains the network on the recorded samples with Adam (learning rate lr), `epochs` passes
 * of minibatches of `batch` samples (32 <= batch <= 65536) in a SplitMix64 shuffle from
 * `seed`; initialises the parameters (fp_mlp_init(seed)) if there are none.  last_loss
 * (may be NULL): the mean loss of the last epoch.  FP_ERR_STATE with fewer samples than one
 * batch; FP_ERR_INVALID for epochs < 1 or lr <= 0. */
fp_status fp_learned_train(fp_handle *h, int epochs, int batch, double lr, unsigned long long seed,
                           double *last_loss);
/* Number of recorded samples. */
fp_status fp_learned_num_samples(const fp_handle *h, long long *n);
/* He-uniform W1, W2 from SplitMix64 stream `seed` (value i -> parameter i); W3 and biases 0. */
fp_status fp_mlp_init(fp_handle *h, unsigned long long seed);
/* Copy the flat parameter array in (set) or out (get); n must be 68353 (FP_ERR_INVALID
 * otherwise); get returns FP_ERR_STATE while there are no parameters. */
fp_status fp_mlp_set_params(fp_handle *h, const float *host, int n);
fp_status fp_mlp_get_params(const fp_handle *h, float *host, int n);
/* Forward pass / mean-squared-error loss L = sum((out - y)^2) / (2 rows) and its gradient
 * (68353 floats in the parameter layout), on host arrays of 1 to 65536 rows (x: rows x 8,
 * row-major); FP_ERR_STATE while the network has no parameters.  For checking the kernels
 * against a reference; training uses the same kernels on device-resident samples. */
fp_status fp_mlp_forward(fp_handle *h, const float *x, int rows, float *out);
fp_status fp_mlp_loss_grad(fp_handle *h, const float *x, const float *y, int rows, float *grad,
                           double *loss);

/* Tunables of the solve (defaults in brackets); FP_ERR_INVALID for an unknown key or a value
 * out of range.
 *   "ir_sweeps"    [6]  maximum FP64 refinement sweeps of the accurate local solves (mixed
 *                       precision: d = B K^+ f, the true residual, the recovery), 0..16
 *   "ir_eps"       [0]  refinement stops once ||dx||_2 <= ir_eps ||x||_2 (all subdomains) or
 *                       once the predicted next correction (the last one times the last
 *                       contraction measured on these factors) is below that; 0: 1e-2 tol,
 *                       clamped to [1e-15, 1e-10]
 *   "ir_stag"      [0.5] ... or once ||dx||_2 > ir_stag ||dx_prev||_2 (stagnation at the
 *                       rounding floor), 0 <= ir_stag < 1, 0 never
 *   "inner_ir"     [0]  refinement sweeps of the local solves inside the PCG loop, 0..8
 *   "max_restarts" [8]  restarts of PCG from the true residual, 0..64
 *   "pcg_chunk"    [8]  PCG iterations per body of the device-side loop (per host poll of the
 *                       stop flag when "graph" is 0), 1..256
 *   "solve_kernel" [1]  local solve kernel: 1 blocked sweeps (32-row blocks, inverse diagonal
 *                       blocks), 0 row-step sweeps
 *   "solve_wpc"    [0]  warps per CTA of the local solves, 1..8 (0: autotuned, or chosen
 *                       from the task count when "autotune" is 0)
 *   "solve_chunk"  [0]  bytes per shared-memory stage of the blocked solves, 4096..65536
 *                       (0: autotuned, or 8192)
 *   "solve_cps"    [0]  CTAs per SM of the blocked solves, 1..2 (0: autotuned, or 1)
 *   "factor_nb"    [0]  panel width of the factorisation, 4..64, multiple of 4 (0: autotuned,
 *                       or the widest of 32, 16, 8, 4 whose panel fits in shared memory)
 *   "explicit"     [0]  1: fp_factor also forms the local interface operators explicitly,
 *                       F_s = (K_s^+) restricted to the dofs touched by B_s and the Dirichlet
 *                       Schur complement S_s (dense m_s x m_s per subdomain, the factors'
 *                       precision; m_s = 480 for a 24 x 24-cell P2 poroelastic subdomain with
 *                       four interface sides), by multi-right-hand-side
 *                       band solves; F and the Dirichlet preconditioner are then applied as
 *                       batched dense products.  FP64: F_s, S_s in FP64 for every apply.
 *                       Mixed: F_s is formed in FP64 from the FP64 factorisation (with
 *                       "factor_fp64", the default) and serves every accurate apply, its FP32
 *                       rounding serves the PCG loop; S_s is FP32 from the FP32 factors (without
 *                       "factor_fp64": F_s FP32 for the loop only, accurate applies keep the
 *                       refined band solves).  The right-hand side and the recovery keep full
 *                       band solves.  Needs b + 64 window rows of 32 values in shared memory
 *                       (FP_ERR_INVALID when the band is too wide).  Takes effect at fp_factor.
 *   "explicit_tile" [0] right-hand sides per task of the explicit-operator build: 32 or 16
 *                       (0: 32 where its shared-memory window fits, else 16)
 *   "autotune"     [1]  fp_factor times candidate launch shapes on the handle's own factors
 *                       and keeps the fastest (see fp_get_tuning); explicitly set shape
 *                       options are kept fixed.  Takes effect at the next fp_factor.
 *   "factor_fp64"  [1]  mixed precision: compute the local factors in FP64 (temporary device
 *                       memory) and round the finished factors to FP32 (0: factor in FP32);
 *                       takes effect at the next fp_factor
 *   "graph"        [1]  1: fp_step is one CUDA graph launch: the step is captured once (on
 *                       private streams; re-captured after an option, fp_factor,
 *                       fp_set_profiling or the learned-guess mode changes) with Algorithm 1
 *                       and its restarts as conditional WHILE nodes set by device flags, and
 *                       replayed on the handle's stream; 0: the same kernels launched
 *                       directly, with a host poll every pcg_chunk iterations.  Both give
 *                       bit-identical results.
 *   "stag_window"  [60] a round of Algorithm 1 stops (and restarts from the true residual)
 *                       when its recursive residual has not halved within this many
 *                       iterations; 0 never, 1..100000
 *   "mlp_tc"       [1]  the learned guess's MLP forward pass (fp_step, fp_mlp_forward) as one
 *                       fused kernel with the 256 x 256 layer on the tensor cores (tcgen05,
 *                       bfloat16 operands, FP32 accumulation in tensor memory); 0: the training
 *                       path's kernels (mma.sync).  Training always uses the latter
 *   "factor_tc"    [1]  FP32 factorisations run on the tensor cores: right-looking panels of 32
 *                       columns, the dense trailing updates as tcgen05 TF32 tiles with the
 *                       3xTF32 split (hi*hi + hi*lo + lo*hi, about FP32 accuracy); half
 *                       bandwidth <= 511.  Mixed precision with "factor_fp64": the Dirichlet
 *                       factor (preconditioner only) this way, the Neumann factor in FP64;
 *                       without "factor_fp64": both.  0: CUDA-core factorisation
 *   "precond_bf16" [1]  mixed precision with "explicit": the Dirichlet preconditioner's S_s
 *                       tiles stored in BF16 (half the bytes of the FP32 tiles; products and
 *                       sums stay FP32).  The preconditioner only steers Algorithm 1, so the
 *                       converged result keeps its accuracy (measured on the large workload: the
 *                       same iteration counts as FP32 tiles); 0: FP32 tiles.  Takes effect at
 *                       the next fp_factor
 *   "explicit_2f"  [1]  mixed precision with "explicit" and "factor_fp64": the accurate F applies
 *                       (reference, initial, learned-guess and true residuals) multiply by F_s
 *                       stored as FP32 hi/lo pairs of its upper 32 x 32 tiles (FP32 arithmetic
 *                       with error-free products and sums, ~1e-14 relative) instead of the FP64
 *                       F_s; 0: the FP64 F_s
 *   "explicit_df"  [1]  mixed precision with "explicit" and "factor_fp64": the FP64 F_s (source
 *                       of the accurate applies' tiles) is built in two-float arithmetic on the
 *                       FP32 units from the FP64 factor split into FP32 hi/lo pairs (error-free
 *                       products and sums, ~2^-46 relative per operation); 0: FP64 arithmetic.
 *                       Takes effect at the next fp_factor
 *   "coarse_2f"    [1]  mixed precision: the coarse projection multiplies by (G^T G)^{-1} stored
 *                       as FP32 hi/lo pairs of its upper 32 x 32 tiles (half the bytes, FP32
 *                       arithmetic with error-free products and sums, ~1e-14 relative); 0: the
 *                       dense FP64 product.  The tiles are packed at fp_factor; the FP64 path
 *                       always uses the FP64 product
 *   "tol"          [fp_params.tol] relative projected residual at which Algorithm 1 stops,
 *                       0 < tol < 1; takes effect at the next fp_step
 */
fp_status fp_set_option(fp_handle *h, const char *key, double value);

/* Per-kernel-class timing (CUDA events on the handle's stream around every launch of the
 * class; off by default).  kind 0: Neumann local solves (K_s^+), 1: Dirichlet local solves
 * (the preconditioner).  bytes_per_launch / flops_per_launch are algorithmic figures: every
 * band entry read once per sweep (2 sweeps, entry size of the factor precision) plus the
 * right-hand side / solution traffic (4 doubles per row), and 2 flops per band entry per
 * sweep.  fp_set_profiling(h, 1) also resets the counters. */
typedef struct {
  long long launches;
  double total_ms;
  double bytes_per_launch;
  double flops_per_launch;
} fp_kernel_stats;
fp_status fp_set_profiling(fp_handle *h, int on);
fp_status fp_get_kernel_stats(const fp_handle *h, int kind, fp_kernel_stats *out);

/* Launch shapes chosen by the autotuner at the last fp_factor (FP_ERR_STATE before it).
 * factor_nb: panel width, timed on a factorisation of the 2 x (SM count) largest subdomains
 * after a fresh copy of their band (factor_ms: that time for the chosen width); solve_*:
 * warps per CTA, bytes per shared-memory stage and CTAs per SM of the blocked solves, timed
 * on whole Neumann solves (solve_ms: one solve with the chosen shape; candidates: shapes
 * timed).  With "autotune" 0 the fields hold the shapes in use and the timings are 0. */
typedef struct {
  int factor_nb;
  int solve_wpc, solve_chunk, solve_ctas_per_sm;
  double factor_ms, solve_ms;
  int candidates;
  double explicit_ms;  /* build time of the explicit interface operators (0: not built) */
  int precond;         /* preconditioner in use (FP_PRECOND_*; the AUTO choice) */
  /* AUTO probes (index 0 DIRICHLET, 1 LUMPED; zero when not probed): contraction of the
   * residual norm per iteration over 30 iterations of Algorithm 1 on a seeded random
   * right-hand side in range(P) from lambda_0 = 0, and the time per iteration */
  double precond_rate[2], precond_ms_per_it[2];
  /* kernel instantiations in use after the last fp_factor.  solve_mmax: the band-solve
   * template's window registers per lane (LD / 32 of the widest band, rounded up to 4, 8, 12
   * or 16).  Per explicit operator (index 0 F_s, 1 S_s; zero when not built): the
   * multi-right-hand-side build's rows per thread of the off-block coupling (mrhs_nr: 4, 8,
   * 12 or 16), right-hand sides per tile (mrhs_mt: 32, or 16 where a 32-wide window does
   * not fit in shared memory) and element size in bytes (mrhs_esz: 8 FP64, 4 FP32). */
  int solve_mmax;
  int mrhs_nr[2], mrhs_mt[2], mrhs_esz[2];
  /* device time of the FP32 factorisations on the tensor cores ("factor_tc"; index 0 Neumann,
   * 1 Dirichlet), milliseconds; 0 where that factor was not computed this way */
  double factor_tc_ms[2];
  /* device time of each explicit operator's multi-right-hand-side build (index 0 F_s, 1 S_s;
   * the parts of explicit_ms), milliseconds; 0 where not built */
  double mrhs_ms[2];
  /* arithmetic of each build: 0 FP64, 1 FP32, 2 two-float (FP32 pairs, FP64 result); -1 not built */
  int mrhs_prec[2];
} fp_tuning;
fp_status fp_get_tuning(const fp_handle *h, fp_tuning *out);

/* Message of the last failed call on h; with h = NULL, of the last failed fp_create or
 * fp_plan on the calling thread.  The string is owned by the library and valid until the
 * next call on h (or on the thread). */
const char *fp_last_error(const fp_handle *h);
/* Frees everything the handle owns (device memory, streams, events, graphs); NULL is a no-op.
 * The handle's stream must be idle. */
void fp_destroy(fp_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* FETIPE_H */
