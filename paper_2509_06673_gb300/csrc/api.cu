// C ABI of the fetipe library: handle lifecycle and the orchestration of one
// backward-Euler step (Sec. 2.5) solved by FETI (Sec. 3, Algorithm 1).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <functional>
#include <random>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace fp {
// kernels (defined in the other translation units)
__global__ void k_assemble(DevTopo, DevParams, double *, double *, double *, double *);
__global__ void k_set_initial(DevTopo, DevParams, const double *, const double *, double *);
cudaError_t launch_csr_to_band(bool fp32, DevTopo D, const double *csr_val, void *band, int mode, cudaStream_t s);
__global__ void k_coarse_G(DevTopo, double *, double *);
__global__ void k_coarse_GtG(DevTopo, const double *, const double *, double *);
cudaError_t launch_band_factor(bool fp32, const BandTask *tasks, int ntask, void *base, int NB, int *status,
                               size_t smem, cudaStream_t stream);
cudaError_t launch_band_solve(bool fp32, int mmax, int grid, int wpc, cudaStream_t stream, const BandTask *tasks,
                              int ntask, const void *fac, double *x, int *counter, int *status, const int *done);
cudaError_t launch_band_solve_blk(bool fp32, int mmax, int grid, int wpc, int chunk, cudaStream_t stream,
                                  const BandTask *tasks, int ntask, const void *fac, double *x, int *counter,
                                  int *status, const int *done);
cudaError_t launch_band_linv(bool fp32, const BandTask *tasks, int ntask, const void *fac, void *linv,
                             cudaStream_t stream);
cudaError_t launch_round_to_float(const double *src, float *dst, long long n, cudaStream_t stream);
size_t mrhs_smem_bytes(int prec, int R, int LDp, int mt);
cudaError_t launch_split_df(double *v, long long n, cudaStream_t st);
cudaError_t launch_band_mrhs(int prec, int bmax, int mt, int grid, cudaStream_t st, const int *task_s,
                             const int *task_j0, int ntask, DevTopo D, const void *fac, const void *linv,
                             const long long *linv_off, const double *csr, int kind, void *scratch, long long sstride,
                             int *counter, void *out, const long long *out_off, int R, int LDp);
int mrhs_blocks_per_sm(int prec, int bmax, int mt, int R, int LDp);
int mrhs_nr(int b, int mt);
cudaError_t launch_mrhs_symmetrize(bool fp32, DevTopo D, int S, void *out, const long long *out_off, int mt,
                                   cudaStream_t st);
cudaError_t launch_explicit_apply(bool fp32, DevTopo D, int S, int mmax_bnd, const void *ops, const long long *op_off,
                                  double *xloc, const int *fl, cudaStream_t st);
cudaError_t launch_pack_sym2f(DevTopo D, int S, const double *full, const long long *full_off, float *tiles,
                              const long long *tile_off, cudaStream_t st);
cudaError_t launch_explicit_apply_sym2f(DevTopo D, int S, int mmax_bnd, const float *tiles, const long long *tile_off,
                                        double *xloc, const int *fl, cudaStream_t st);
cudaError_t launch_pack_sym(bool src_fp64, DevTopo D, int S, const void *full, const long long *full_off,
                            void *tiles, const long long *tile_off, cudaStream_t st, bool bf16_out = false);
cudaError_t launch_explicit_apply_sym(DevTopo D, int S, int mmax_bnd, const void *tiles, const long long *tile_off,
                                      double *xloc, const int *fl, cudaStream_t st, const double *vlam,
                                      int skip_fixed, bool bf16);
__global__ void k_gather_wscale(DevTopo, const double *, double *, const int *);
__global__ void k_Gcomb_dot(DevTopo, const double *, const double *, double *, const double *, double *, unsigned *,
                            double *, int *, int);
__global__ void k_dot(const double *, const double *, long long, double *, unsigned *, double *, int *, int,
                      double *, int);
__global__ void k_pcg_update(double *, double *, const double *, const double *, long long, double *, unsigned *,
                             double *, int *);
__global__ void k_pcg_update_w(DevTopo, double *, double *, const double *, const double *, double *, double *,
                               unsigned *, double *, int *);
__global__ void k_pcg_pupdate(double *, const double *, long long, const double *, const int *);
__global__ void k_lincomb(double *, const double *, double, const double *, double, long long, const int *);
__global__ void k_scatter(DevTopo, const double *, double, double *, int, const int *, int);
__global__ void k_gather(DevTopo, const double *, double *, const int *);
__global__ void k_wscale(DevTopo, const double *, double *, const int *);
__global__ void k_halo(DevTopo, const double *, const double *, double *, const int *);
__global__ void k_bnd_apply(DevTopo, const double *, const double *, double *, const int *);
__global__ void k_Gt(DevTopo, const double *, double *, const int *, float *);
__global__ void k_pack_float_g(DevTopo, double *);
cudaError_t launch_gemv(const double *H, const double *y, double *alpha, int nH, const int *fl, cudaStream_t st);
cudaError_t launch_coarse_pack2f(const double *H, int nH, float *tiles, cudaStream_t st);
size_t band_factor_tc_smem(int ldmax, int bmax);
cudaError_t launch_mlp_forward_tc(long long rows, const float *X, const float *P, float *out, int num_sms,
                                  int *status, cudaStream_t st);
cudaError_t launch_band_factor_tc(const BandTask *tasks, int ntask, float *base, int ldmax, int bmax, int num_sms,
                                  int *counter, int *status, cudaStream_t stream);
cudaError_t launch_coarse_apply2f(const float *tiles, int nH, const float *ysplit, double *part, double *alpha,
                                  const int *fl, cudaStream_t st);
__global__ void k_Gcomb(DevTopo, const double *, const double *, double, double *, const int *);
__global__ void k_rhs(DevTopo, DevParams, const double *, const double *, const double *, const double *,
                      const double *, double *, double *);
__global__ void k_loop_arm_outer(cudaGraphConditionalHandle, int *);
__global__ void k_loop_arm_inner(cudaGraphConditionalHandle, int *);
__global__ void k_loop_inner(cudaGraphConditionalHandle, int *, int);
__global__ void k_loop_outer(cudaGraphConditionalHandle, int *, const double *, int);
__global__ void k_copy_if(double *, const double *, long long, const int *);
__global__ void k_recover(DevTopo, DevParams, const double *, const double *, const double *, double *, double *,
                          double *, double *, double *);
cudaError_t launch_band_to_dense(const double *band, int n, int LD, int b, double *out, cudaStream_t s);
__global__ void k_identity(double *, int);
__global__ void k_residual_N(DevTopo, const double *, const double *, const double *, double *, const int *);
__global__ void k_csr_to_sell(DevTopo, const double *, double *);
__global__ void k_local_add(double *, const double *, long long, const int *);
__global__ void k_ir_check(const double *, const double *, long long, double, double *, unsigned *, int *,
                           double *, double, double *);

// learned lambda_0 (learned.cu)
constexpr int MLP_NIN = 8, MLP_NH = 256, MLP_NPARAM = 8 * 256 + 256 + 256 * 256 + 256 + 256 + 1;
constexpr int MLP_OFF_W2 = 8 * 256 + 256, MLP_OFF_B2 = MLP_OFF_W2 + 256 * 256, MLP_OFF_B1 = 8 * 256;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + 256, MLP_OFF_B3 = MLP_OFF_W3 + 256;
cudaError_t launch_gemm_bf16(cudaStream_t s, int M, int N, int K, const float *A, long long sai, long long sak,
                             const float *B, long long sbk, long long sbj, float *C, int ldc, const float *bias,
                             float *z, const float *mask, int relu);
__global__ void k_mlp_l1(int, const float *, const float *, float *, float *);
__global__ void k_mlp_l3(int, const float *, const float *, float *, const float *, float *, double *, float);
__global__ void k_mlp_d2(int, const float *, const float *, const float *, float *);
__global__ void k_colsum(int, int, const float *, int, const float *, float *);
__global__ void k_mlp_dw1(int, const float *, const float *, float *);
__global__ void k_sum_double(const double *, int, double *);
__global__ void k_adam(float *, const float *, float *, float *, int, float, float, float, float, int);
__global__ void k_mlp_init(float *, unsigned long long);
__global__ void k_features(int, const double *, const double *, const double *, const double *, const float *,
                           const int *, const int *, float *, float *);
__global__ void k_guess_dirs(int, const double *, const double *, const float *, const double *, const double *,
                             double *, double *);
__global__ void k_span_solve(const double *, double *, int *);
__global__ void k_span_apply(int, double *, double *, const double *, const double *, const double *,
                             const double *, const double *);
__global__ void k_record(int, const float *, const double *, const double *, const double *, const double *,
                         const double *, int, int, long long, long long, float *, float *);
__global__ void k_gather_rows(int, const int *, const float *, const float *, float *, float *);

}  // namespace fp

using namespace fp;

struct fp_handle {
  Topology T;
  fp_params P{};
  std::vector<double> perm;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 148;
  std::string err;
  int stage = 0;  // 0 created, 1 assembled, 2 factored
  int step_n = 0;
  std::vector<void *> allocs;
  // device topology
  DevTopo D{};
  DevParams DP{};
  // matrices
  double *csr_val = nullptr, *fstat = nullptr, *Zn = nullptr, *E0n = nullptr, *Reta = nullptr;
  double *sell_val = nullptr;  // sliced ELL copy of the Neumann matrices (FP64 residuals)
  void *facN = nullptr, *facD = nullptr, *linvN = nullptr, *linvD = nullptr;
  long long linv_total = 0;
  int solve_kernel = 1;    // 1: blocked sweeps (32-column blocks streamed by TMA), 0: row-step sweeps
  int solve_wpc = 0;       // warps per CTA of the solve kernels (0: autotuned / from the task count)
  int solve_chunk = 0;     // bytes per ring stage of the blocked solve (0: autotuned / 8192)
  int solve_cps = 0;       // CTAs per SM of the blocked solve (0: autotuned / 1)
  int factor_nb = 0;       // panel width of the factorisation (0: autotuned / widest that fits)
  int autotune = 1;        // time candidate shapes at fp_factor and keep the fastest
  struct SolveShape { int wpc, chunk, cps; };
  SolveShape shape{0, 0, 0};  // launch shape of the blocked solves (set at fp_factor)
  fp_tuning tuning{};
  // explicit local interface operators F_s, S_s (dense, per subdomain; option "explicit")
  int precond_req = 0;      // requested preconditioner (FP_PRECOND_AUTO resolved at fp_factor)
  int explicit_ops = 0, ops_ready = 0, opF64_ready = 0;
  int explicit_tile = 0;    // right-hand sides per build task: 0 automatic (32, else 16)
  // the PCG loop's operators: FP64 full m x mp matrices (FP64), FP32 upper 32 x 32 tiles (mixed)
  void *opF = nullptr, *opS = nullptr;
  double *opF64 = nullptr;              // mixed precision: F_s in FP64 for the accurate applies
  float *opF2 = nullptr;                // ... and as two-float (hi/lo FP32) symmetric tiles
  int explicit_2f = 1;                  // option: accurate mixed-precision F applies from opF2
  int explicit_df = 1;                  // option: opF64 built in two-float arithmetic (FP32 units)
  int precond_bf16 = 1;                 // option: mixed precision's S_s tiles in BF16
  int opS_bf16 = 0;                     // the stored S_s tiles are BF16
  const long long *op_off = nullptr, *tile_off = nullptr, *linv_off_dev = nullptr;
  long long op_total = 0, tile_total = 0;
  const int *mrhs_s[2] = {}, *mrhs_j0[2] = {};  // build tasks for tiles of 32 / 16 right-hand sides
  int mrhs_ntask[2] = {0, 0};
  double explicit_build_ms = 0;
  int factor_fp64 = 1;     // mixed precision: factor in FP64, round the finished factor to FP32
  int factor_tc = 1;       // FP32 factors on the tensor cores (3xTF32 trailing updates)
  int mlp_tc = 1;          // MLP inference in the fused tcgen05 kernel
  double *Hband = nullptr, *Hinv = nullptr, *ga = nullptr, *gb = nullptr;
  // mixed precision: (G^T G)^{-1} as hi/lo FP32 upper tiles and the apply's FP64 partials
  float *Htiles = nullptr, *cysplit = nullptr;
  double *Hpart = nullptr;
  int coarse_2f = 1;       // option: two-float tiled coarse product in mixed precision
  int gkernels[3] = {0, 0, 0};  // kernel nodes of the step graph: top level, outer body, inner body
  BandTask *tasksN = nullptr, *tasksD = nullptr, *taskH = nullptr, *tasksHinv = nullptr;
  int ntask = 0, mmax = 4, mmaxH = 4, ldmax = 32;
  int *counter = nullptr, *status = nullptr;
  // vectors
  double *X2 = nullptr, *XB = nullptr, *XP = nullptr, *XY = nullptr;
  double *XF = nullptr, *XA = nullptr, *XR = nullptr;  // rhs, refined solution, residual
  // tunables (fp_set_option)
  int ir_sweeps = 6;       // max refinement sweeps of the accurate local solves (mixed precision)
  double ir_eps = 0.0;     // refinement stops once ||dx|| <= ir_eps ||x|| (0: 1e-2 tol in [1e-15, 1e-10])
  double ir_stag = 0.5;    // ... or once ||dx|| > ir_stag ||dx_prev|| (0: never)
  int inner_ir = 0;        // refinement sweeps inside the PCG loop (mixed precision)
  int max_restarts = 8;    // PCG restarts from the true residual
  int pcg_chunk = 8;       // PCG iterations per body of the device loop (per host poll without graphs)
  int use_graph = 1;       // 1: each time step is one CUDA graph launch (device-side loops)
  int stag_window = 60;    // PCG round stops after this many iterations without halving
  int restarts_last = 0;
  // per-step graph: captured on private streams, launched on `stream`
  cudaStream_t cap[3] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gkey = -1;             // learned-guess variant the graph was captured with
  int gdirty = 1;            // options, profiling or factors changed since the capture
  int capturing = 0, in_body = 0;
  std::vector<cudaEvent_t> gev;  // events recorded by the graph (profiling)
  size_t gev_used = 0;
  double *stepv = nullptr, *h_stepv = nullptr;  // per-step scalars (device, pinned host)
  long long xfer[2] = {0, 0};                    // host->device, device->host bytes of the last fp_step
  int *h_flinit = nullptr;                      // initial PCG flags (pinned host)
  double *lam = nullptr, *lam_prev = nullptr, *lam00 = nullptr, *d = nullptr, *r = nullptr, *z = nullptr,
         *p = nullptr, *q = nullptr, *t1 = nullptr, *t2 = nullptr;
  double *ce = nullptr, *cy = nullptr, *calpha = nullptr;
  double *partial = nullptr, *sc = nullptr, *ir_prev = nullptr;
  unsigned *red_counter = nullptr;
  int *fl = nullptr, *fl_zero = nullptr, *fl_ir = nullptr, *h_fl = nullptr;
  double *h_sc = nullptr;
  double *U = nullptr, *XI = nullptr, *ETA = nullptr, *PP = nullptr;
  cudaEvent_t ev[6] = {};
  double last_ms[4] = {0, 0, 0, 0};
  int nbnd_max = 0;
  // profiling of the local-solve launches
  int profiling = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Pending { int kind; cudaEvent_t e0, e1; };
  std::vector<Pending> pending;   // timed launches of the current step
  std::vector<Pending> gpending;  // timed launches inside the captured graph
  long long prof_launches[2] = {0, 0};
  double prof_ms[2] = {0, 0};
  double bytes_per_solve = 0, flops_per_solve = 0;
  // learned lambda_0
  static constexpr int CH = 65536;             // rows per MLP chunk / max training batch
  float *mlpP = nullptr, *mlpG = nullptr, *mlpM1 = nullptr, *mlpM2 = nullptr;
  float *Xf = nullptr, *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *mout = nullptr, *dout = nullptr,
        *yb = nullptr, *xb = nullptr, *fscale = nullptr;
  double *loss_rows = nullptr, *loss_acc = nullptr, *fsum = nullptr, *nrm = nullptr;
  float *xy_rows = nullptr;
  int *kind_rows = nullptr, *comp_rows = nullptr, *idx_dev = nullptr, *choose_flag = nullptr;
  double *lam_prev2 = nullptr, *lam_b = nullptr, *r_b = nullptr;
  float *SX = nullptr, *SY = nullptr;
  int *train_idx = nullptr;  // shuffled sample indices of fp_learned_train (grown on demand)
  long long train_idx_cap = 0;
  long long n_samples = 0, cap_samples = 0;
  int mlp_ready = 0, learned_use = 0, learned_record = 0, adam_step = 0, hist = 0;
  int record_per_step = 65536;
  double sigma_hist[2] = {0, 0};               // source signal at t_{n-1}, t_{n-2}
  int last_learned = 0;
  double last_res_prev = -1, last_res_learned = -1;
};

namespace {

thread_local std::string g_create_err;

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return e_ == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;           \
    }                                                                             \
  } while (0)

#define CKL()                                                                     \
  do {                                                                            \
    cudaError_t e_ = cudaGetLastError();                                          \
    if (e_ != cudaSuccess) {                                                      \
      h->err = std::string("kernel launch: ") + cudaGetErrorString(e_);           \
      return FP_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)

template <typename V>
fp_status dalloc(fp_handle *h, V **ptr, size_t count) {
  void *p = nullptr;
  CK(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(V)));
  h->allocs.push_back(p);
  *ptr = static_cast<V *>(p);
  return FP_OK;
}

// Frees one allocation made by dalloc (cudaFree waits for the device to finish with it).
void dfree(fp_handle *h, void *p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) h->allocs.erase(it);
  cudaFree(p);
}

template <typename V>
fp_status upload(fp_handle *h, const V **dst, const std::vector<V> &src) {
  V *p = nullptr;
  fp_status st = dalloc(h, &p, src.size());
  if (st) return st;
  if (!src.empty()) CK(cudaMemcpyAsync(p, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice, h->stream));
  *dst = p;
  return FP_OK;
}

#define TRY(x)                 \
  do {                         \
    fp_status s_ = (x);        \
    if (s_ != FP_OK) return s_; \
  } while (0)

unsigned grid_for(long long n, int block) { return (unsigned)std::min<long long>((n + block - 1) / block, 65535LL * 16); }

fp_status build_device(fp_handle *h) {
  Topology &T = h->T;
  // ---- template pool ----
  std::vector<int> pool;
  std::vector<DevTpl> tpls;
  auto put = [&](const std::vector<int> &v) {
    long long off = (long long)pool.size();
    pool.insert(pool.end(), v.begin(), v.end());
    return off;
  };
  for (const Template &t : T.tpl) {
    DevTpl d{};
    d.n = t.n; d.b = t.b; d.LD = t.LD; d.k = t.k; d.poro = t.poro; d.nx = t.nx; d.ny = t.ny;
    d.nux = t.nux; d.nuy = t.nuy; d.npx = t.npx; d.npy = t.npy; d.ndl = t.ndl; d.floating = t.floating;
    d.fixed0 = t.fixed[0]; d.fixed1 = t.fixed[1]; d.fixed2 = t.fixed[2];
    d.nbnd = (int)t.bnd.size(); d.nhalo = (int)t.halo_row.size(); d.nnz = (int)t.csr_col.size();
    d.udof = put(t.udof); d.xidof = put(t.xidof); d.pdof = put(t.pdof);
    d.dof_field = put(t.dof_field); d.dof_node = put(t.dof_node);
    d.csr_ptr = put(t.csr_ptr); d.csr_col = put(t.csr_col);
    d.bnd = put(t.bnd);
    std::vector<int> isb(t.is_bnd.begin(), t.is_bnd.end());
    d.is_bnd = put(isb);
    d.halo_ptr = put(t.halo_ptr); d.halo_row = put(t.halo_row); d.halo_ent = put(t.halo_ent);
    d.elem_dofs = put(t.elem_dofs);
    d.sell_ptr = put(t.sell_ptr); d.sell_col = put(t.sell_col); d.sell_src = put(t.sell_src);
    d.nslice = (int)t.sell_ptr.size() - 1;
    tpls.push_back(d);
    h->nbnd_max = std::max(h->nbnd_max, d.nbnd);
    h->ldmax = std::max(h->ldmax, t.LD);
  }
  DevTopo &D = h->D;
  D.S = T.S; D.NF = T.NF; D.nlam = T.n_lambda; D.nH = T.nH; D.bH = T.bH; D.LDH = T.LDH; D.k = T.k;
  D.nsx = T.nsx; D.nsy = T.nsy;
  TRY(upload(h, &D.tpl, tpls));
  TRY(upload(h, &D.pool, pool));
  TRY(upload(h, &D.sub_tpl, T.sub_tpl));
  TRY(upload(h, &D.sub_x0, T.sub_x0)); TRY(upload(h, &D.sub_y0, T.sub_y0));
  TRY(upload(h, &D.sub_hx, T.sub_hx)); TRY(upload(h, &D.sub_hy, T.sub_hy));
  TRY(upload(h, &D.vec_off, T.vec_off)); TRY(upload(h, &D.fac_off, T.fac_off));
  TRY(upload(h, &D.csr_off, T.csr_off)); TRY(upload(h, &D.sell_off, T.sell_off)); TRY(upload(h, &D.unode_off, T.unode_off));
  TRY(upload(h, &D.pnode_off, T.pnode_off)); TRY(upload(h, &D.elem_off, T.elem_off));
  TRY(upload(h, &D.bsc_off, T.bsc_off));
  TRY(upload(h, &D.sub_I0, T.sub_I0)); TRY(upload(h, &D.sub_J0, T.sub_J0));
  TRY(upload(h, &D.lam_sa, T.lam_sa)); TRY(upload(h, &D.lam_da, T.lam_da));
  TRY(upload(h, &D.lam_sb, T.lam_sb)); TRY(upload(h, &D.lam_db, T.lam_db));
  std::vector<int> kind(T.n_lambda);
  for (int r = 0; r < T.n_lambda; ++r) kind[r] = T.lam_key[6 * r];
  TRY(upload(h, &D.lam_kind, kind));
  TRY(upload(h, &D.wgrp_first, T.wgrp_first)); TRY(upload(h, &D.wgrp_size, T.wgrp_size));
  D.nwgrp = (int)T.wgrp_first.size();
  TRY(upload(h, &D.bsc_row, T.bsc_row)); TRY(upload(h, &D.bsc_sign, T.bsc_sign));
  TRY(upload(h, &D.sub_float, T.sub_float)); TRY(upload(h, &D.float_sub, T.float_sub));
  TRY(upload(h, &D.float_rows_ptr, T.float_rows_ptr)); TRY(upload(h, &D.float_rows, T.float_rows));
  std::vector<int> fa(T.n_lambda), fb(T.n_lambda);
  for (int r = 0; r < T.n_lambda; ++r) { fa[r] = T.sub_float[T.lam_sa[r]]; fb[r] = T.sub_float[T.lam_sb[r]]; }
  TRY(upload(h, &D.lam_fa, fa)); TRY(upload(h, &D.lam_fb, fb));
  TRY(dalloc(h, &h->ga, 3 * (size_t)T.n_lambda));
  TRY(dalloc(h, &h->gb, 3 * (size_t)T.n_lambda));
  D.lam_ga = h->ga; D.lam_gb = h->gb;
  {
    double *fg = nullptr;
    TRY(dalloc(h, &fg, 3 * std::max<size_t>(T.float_rows.size(), 1)));
    D.float_g = fg;
  }
  // params
  DevParams &P = h->DP;
  P.lam = h->P.lame_lambda; P.mu = h->P.mu; P.alpha = h->P.alpha; P.c0 = h->P.c0;
  P.perm_k = h->P.perm_k; P.mu_f = h->P.mu_f; P.tau = h->P.tau; P.q_omega = h->P.q_omega;
  P.source = h->P.source; P.src_sub = T.src_sub; P.src_node = T.src_node;
  P.perm = nullptr;
  if (!h->perm.empty()) {
    const double *pp = nullptr;
    TRY(upload(h, &pp, h->perm));
    P.perm = pp;
  }
  // ---- tasks (cost-sorted, largest first) ----
  std::vector<int> order(T.S);
  for (int s = 0; s < T.S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const Template &ta = T.tpl[T.sub_tpl[a]], &tb = T.tpl[T.sub_tpl[b]];
    return (long long)ta.n * ta.LD > (long long)tb.n * tb.LD;
  });
  std::vector<long long> linv_off(T.S + 1, 0);
  for (int s = 0; s < T.S; ++s) linv_off[s + 1] = linv_off[s] + 1024LL * ((T.tpl[T.sub_tpl[s]].n + 31) / 32);
  h->linv_total = linv_off[T.S];
  TRY(upload(h, &h->linv_off_dev, linv_off));
  {
    // explicit-operator layout (rows padded to a multiple of 4) and build tasks: every
    // subdomain in cost order, tiles of 32 right-hand sides
    std::vector<long long> ooff(T.S + 1, 0), toff(T.S + 1, 0);
    std::vector<int> ms[2], mj[2];
    for (int s = 0; s < T.S; ++s) {
      const long long m = (long long)T.tpl[T.sub_tpl[s]].bnd.size(), nt = (m + 31) / 32;
      ooff[s + 1] = ooff[s] + m * ((m + 3) & ~3LL);
      toff[s + 1] = toff[s] + nt * (nt + 1) / 2 * 1024;
    }
    for (int w = 0; w < 2; ++w)
      for (int s : order) {
        const int m = (int)T.tpl[T.sub_tpl[s]].bnd.size();
        for (int j0 = 0; j0 < m; j0 += (w == 0 ? 32 : 16)) { ms[w].push_back(s); mj[w].push_back(j0); }
      }
    h->op_total = ooff[T.S];
    h->tile_total = toff[T.S];
    TRY(upload(h, &h->op_off, ooff));
    TRY(upload(h, &h->tile_off, toff));
    for (int w = 0; w < 2; ++w) {
      h->mrhs_ntask[w] = (int)ms[w].size();
      TRY(upload(h, &h->mrhs_s[w], ms[w]));
      TRY(upload(h, &h->mrhs_j0[w], mj[w]));
    }
  }
  std::vector<BandTask> tk;
  int mmax = 1;
  for (int s : order) {
    const Template &t = T.tpl[T.sub_tpl[s]];
    tk.push_back({T.fac_off[s], T.vec_off[s], linv_off[s], t.n, t.LD, t.b, 0});
    mmax = std::max(mmax, t.LD / 32);
  }
  if (T.nH > 28672) { h->err = "coarse space above 28672 unknowns is not supported"; return FP_ERR_INVALID; }
  if (mmax > 16) { h->err = "half bandwidth above 511 is not supported"; return FP_ERR_INVALID; }
  h->mmax = mmax <= 4 ? 4 : mmax <= 8 ? 8 : mmax <= 12 ? 12 : 16;
  h->ntask = T.S;
  const BandTask *dt = nullptr;
  TRY(upload(h, &dt, tk));
  h->tasksN = const_cast<BandTask *>(dt);
  h->tasksD = h->tasksN;  // same offsets; the two factors live in separate arrays
  if (T.NF) {
    std::vector<BandTask> th = {{0, 0, 0, T.nH, T.LDH, T.bH, 0}};
    TRY(upload(h, &dt, th));
    h->taskH = const_cast<BandTask *>(dt);
    std::vector<BandTask> ti(T.nH);
    for (int i = 0; i < T.nH; ++i) ti[i] = {0, (long long)i * T.nH, 0, T.nH, T.LDH, T.bH, 0};
    TRY(upload(h, &dt, ti));
    h->tasksHinv = const_cast<BandTask *>(dt);
    const int mh = T.LDH / 32;
    if (mh > 16) { h->err = "coarse band too wide"; return FP_ERR_INVALID; }
    h->mmaxH = mh <= 4 ? 4 : mh <= 8 ? 8 : mh <= 12 ? 12 : 16;
  }
  // ---- work arrays ----
  const long long nv = T.vec_off[T.S], nl = std::max(T.n_lambda, 1);
  TRY(dalloc(h, &h->csr_val, (size_t)T.csr_off[T.S]));
  if (h->P.precision == FP_PREC_MIXED) TRY(dalloc(h, &h->sell_val, (size_t)T.sell_off[T.S]));
  TRY(dalloc(h, &h->fstat, (size_t)nv));
  TRY(dalloc(h, &h->Zn, (size_t)T.pnode_off[T.S]));
  TRY(dalloc(h, &h->E0n, (size_t)T.pnode_off[T.S]));
  TRY(dalloc(h, &h->Reta, (size_t)T.pnode_off[T.S]));
  for (double **v : {&h->X2, &h->XB, &h->XP, &h->XY}) TRY(dalloc(h, v, (size_t)nv));
  if (h->P.precision == FP_PREC_MIXED)
    for (double **v : {&h->XF, &h->XA, &h->XR}) TRY(dalloc(h, v, (size_t)nv));
  for (double **v : {&h->lam, &h->lam_prev, &h->lam00, &h->d, &h->r, &h->z, &h->p, &h->q, &h->t1, &h->t2})
    TRY(dalloc(h, v, (size_t)nl));
  const size_t nc = std::max(T.nH, 1);
  for (double **v : {&h->ce, &h->cy, &h->calpha}) TRY(dalloc(h, v, nc));
  TRY(dalloc(h, &h->partial, 2 * RED_BLOCKS));
  TRY(dalloc(h, &h->sc, SC_N));
  TRY(dalloc(h, &h->ir_prev, 2));  // [0] last correction^2 of the current solve, [1] contraction^2
  TRY(dalloc(h, &h->red_counter, 4));
  TRY(dalloc(h, &h->fl, FL_N));
  TRY(dalloc(h, &h->fl_zero, FL_N));
  TRY(dalloc(h, &h->fl_ir, FL_N));
  TRY(dalloc(h, &h->counter, 4));
  TRY(dalloc(h, &h->status, 4));
  TRY(dalloc(h, &h->U, 2 * (size_t)T.unode_off[T.S]));
  TRY(dalloc(h, &h->XI, (size_t)T.pnode_off[T.S]));
  TRY(dalloc(h, &h->ETA, (size_t)T.pnode_off[T.S]));
  TRY(dalloc(h, &h->PP, (size_t)T.pnode_off[T.S]));
  CK(cudaMemsetAsync(h->red_counter, 0, 4 * sizeof(unsigned), h->stream));
  CK(cudaMemsetAsync(h->fl_zero, 0, FL_N * sizeof(int), h->stream));
  CK(cudaMemsetAsync(h->fl_ir, 0, FL_N * sizeof(int), h->stream));
  // zero every local vector once: kernels write only real rows, so the padding stays zero
  for (double *v : {h->X2, h->XB, h->XP, h->XY, h->XF, h->XA, h->XR})
    if (v) CK(cudaMemsetAsync(v, 0, (size_t)nv * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->status, 0, 4 * sizeof(int), h->stream));
  CK(cudaMemsetAsync(h->lam_prev, 0, nl * sizeof(double), h->stream));
  // learned lambda_0 state (features per multiplier, MLP chunk buffers)
  {
    const int CH = fp_handle::CH;
    TRY(dalloc(h, &h->mlpP, MLP_NPARAM)); TRY(dalloc(h, &h->mlpG, MLP_NPARAM));
    TRY(dalloc(h, &h->mlpM1, MLP_NPARAM)); TRY(dalloc(h, &h->mlpM2, MLP_NPARAM));
    TRY(dalloc(h, &h->Xf, (size_t)nl * MLP_NIN));
    for (float **v : {&h->z1, &h->h1, &h->z2, &h->h2}) TRY(dalloc(h, v, (size_t)CH * MLP_NH));
    for (float **v : {&h->mout, &h->dout, &h->yb}) TRY(dalloc(h, v, (size_t)std::max<long long>(CH, nl)));
    TRY(dalloc(h, &h->xb, (size_t)CH * MLP_NIN));
    TRY(dalloc(h, &h->fscale, 1));
    TRY(dalloc(h, &h->loss_rows, CH)); TRY(dalloc(h, &h->loss_acc, 1));
    TRY(dalloc(h, &h->fsum, 2)); TRY(dalloc(h, &h->nrm, 10));
    TRY(dalloc(h, &h->idx_dev, CH)); TRY(dalloc(h, &h->choose_flag, 1));
    for (double **v : {&h->lam_prev2, &h->lam_b, &h->r_b}) TRY(dalloc(h, v, (size_t)nl));
    CK(cudaMemsetAsync(h->lam_prev2, 0, nl * sizeof(double), h->stream));
    // node coordinates, kind and component of every multiplier (geometry of the keys)
    std::vector<float> xy(2 * (size_t)nl, 0.f);
    std::vector<int> kd(nl, 0), cp(nl, 0);
    std::vector<double> xs(T.nsx + 1, 0), ys(T.nsy + 1, 0);
    for (int r = 0; r < T.n_lambda; ++r) {
      const int kind = T.lam_key[6 * r], comp = T.lam_key[6 * r + 1], I = T.lam_key[6 * r + 2], J = T.lam_key[6 * r + 3];
      const int kk = kind == 0 ? T.k : 1;
      auto coord = [&](int G, const std::vector<int> &cells, int nsub) {
        int base = 0;
        for (int c = 0; c < nsub; ++c) {
          const int w = kk * cells[c];
          if (G <= base + w) return ((double)c + (double)(G - base) / w) / nsub;
          base += w;
        }
        return 1.0;
      };
      xy[2 * r] = (float)coord(I, T.cells_x, T.nsx);
      xy[2 * r + 1] = (float)coord(J, T.cells_y, T.nsy);
      kd[r] = kind;
      cp[r] = comp;
    }
    const float *dxy = nullptr;
    const int *dk = nullptr, *dc = nullptr;
    TRY(upload(h, &dxy, xy)); TRY(upload(h, &dk, kd)); TRY(upload(h, &dc, cp));
    h->xy_rows = const_cast<float *>(dxy); h->kind_rows = const_cast<int *>(dk); h->comp_rows = const_cast<int *>(dc);
  }
  CK(cudaMallocHost(&h->h_fl, FL_N * sizeof(int)));
  CK(cudaMallocHost(&h->h_sc, SC_N * sizeof(double)));
  CK(cudaMallocHost(&h->h_stepv, ST_N * sizeof(double)));
  CK(cudaMallocHost(&h->h_flinit, FL_N * sizeof(int)));
  for (int i = 0; i < FL_N; ++i) h->h_flinit[i] = 0;
  h->h_flinit[FL_MAXIT] = h->P.max_it;
  for (int i = 0; i < ST_N; ++i) h->h_stepv[i] = 0.0;
  TRY(dalloc(h, &h->stepv, ST_N));
  for (auto &c : h->cap) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
  for (auto &e : h->ev) CK(cudaEventCreate(&e));
  return FP_OK;
}

// ------------------------------ building blocks -------------------------------------
// The blocked solve's launch shape made legal for the element size: a stage holds at least
// one column of the widest band; the ring fits the shared memory of one CTA (and of cps CTAs
// per SM).
fp_handle::SolveShape legal_shape(const fp_handle *h, fp_handle::SolveShape sh, bool fp32) {
  const int esz = fp32 ? 4 : 8;
  sh.chunk = std::max(sh.chunk, (std::max(h->ldmax, h->T.LDH) * esz + 1023) / 1024 * 1024);
  while (sh.wpc > 1 && (size_t)sh.wpc * 3 * (sh.chunk + 8) > 200 * 1024) sh.wpc >>= 1;
  if (sh.cps < 1) sh.cps = 1;
  while (sh.cps > 1 && (size_t)sh.cps * sh.wpc * 3 * (sh.chunk + 8) > 220 * 1024) --sh.cps;
  return sh;
}

// shape from the task count when nothing was tuned: warps per CTA double while every SM
// still gets two CTAs' worth of tasks; options pinned by the caller win
fp_handle::SolveShape default_shape(const fp_handle *h, int ntask) {
  fp_handle::SolveShape sh{h->solve_wpc, h->solve_chunk ? h->solve_chunk : 8192, h->solve_cps ? h->solve_cps : 1};
  if (sh.wpc <= 0) {
    sh.wpc = 1;
    while (sh.wpc < 8 && ntask >= 2 * sh.wpc * h->num_sms) sh.wpc *= 2;
  }
  return sh;
}

fp_status launch_solve_shaped(fp_handle *h, bool fp32, const BandTask *tasks, int ntask, const void *fac,
                              double *x, int mmax, const int *done, fp_handle::SolveShape sh) {
  CK(cudaMemsetAsync(h->counter, 0, sizeof(int), h->stream));
  if (h->solve_kernel == 1) {
    sh = legal_shape(h, sh, fp32);
    const int grid = std::max(1, std::min(sh.cps * h->num_sms, (ntask + sh.wpc - 1) / sh.wpc));
    CK(launch_band_solve_blk(fp32, mmax, grid, sh.wpc, sh.chunk, h->stream, tasks, ntask, fac, x, h->counter,
                             h->status, done));
  } else {
    int wpc = ntask >= 4 * h->num_sms ? 4 : (ntask >= 2 * h->num_sms ? 2 : 1);
    if (h->solve_wpc > 0) wpc = std::min(h->solve_wpc, 4);
    const int grid = std::max(1, std::min(h->num_sms, (ntask + wpc - 1) / wpc));
    CK(launch_band_solve(fp32, mmax, grid, wpc, h->stream, tasks, ntask, fac, x, h->counter, h->status, done));
  }
  return FP_OK;
}

fp_status launch_solve(fp_handle *h, bool fp32, const BandTask *tasks, int ntask, const void *fac, double *x,
                       int mmax, const int *done) {
  const fp_handle::SolveShape sh = h->shape.wpc > 0 ? h->shape : default_shape(h, ntask);
  return launch_solve_shaped(h, fp32, tasks, ntask, fac, x, mmax, done, sh);
}

fp_status next_event(fp_handle *h, cudaEvent_t *e) {
  if (h->capturing) {  // events recorded by the graph: created before the capture began
    if (h->gev_used == h->gev.size()) { h->err = "graph profiling: out of events"; return FP_ERR_STATE; }
    *e = h->gev[h->gev_used++];
    return FP_OK;
  }
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t ne;
    CK(cudaEventCreate(&ne));
    h->ev_pool.push_back(ne);
  }
  *e = h->ev_pool[h->ev_used++];
  return FP_OK;
}

fp_status solve_local(fp_handle *h, bool dirichlet, double *x, const int *done) {
  const void *fac = dirichlet ? h->facD : h->facN;
  const BandTask *tasks = dirichlet ? h->tasksD : h->tasksN;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // launches inside a conditional body are not timed (a body may not hold event nodes)
  const bool timed = h->profiling && !h->in_body;
  const unsigned evflags = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (timed) {
    TRY(next_event(h, &e0));
    TRY(next_event(h, &e1));
    CK(cudaEventRecordWithFlags(e0, h->stream, evflags));
  }
  TRY(launch_solve(h, h->P.precision == FP_PREC_MIXED, tasks, h->ntask, fac, x, h->mmax, done));
  if (timed) {
    CK(cudaEventRecordWithFlags(e1, h->stream, evflags));
    (h->capturing ? h->gpending : h->pending).push_back({dirichlet ? 1 : 0, e0, e1});
  }
  return FP_OK;
}

// After a stream synchronisation: fold the pending event pairs into the counters.  A
// launch that returned at once because the PCG had already converged is not counted.
fp_status collect_profile(fp_handle *h) {
  for (auto &pr : h->pending) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, pr.e0, pr.e1));
    if (ms > 0.02f) {
      h->prof_launches[pr.kind] += 1;
      h->prof_ms[pr.kind] += ms;
    }
  }
  h->pending.clear();
  h->ev_used = 0;
  return FP_OK;
}

// x = K^+ b.  FP64: one solve.  Mixed: FP32 solve then `sweeps` refinement sweeps with the
// residual b - K_N x in FP64.  b is kept; x must not alias b unless sweeps == 0 and FP64.
fp_status solve_refined(fp_handle *h, const double *b, double *x, int sweeps, const int *fl) {
  const long long nv = h->T.vec_off[h->T.S];
  if (x != b) CK(cudaMemcpyAsync(x, b, nv * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  TRY(solve_local(h, false, x, fl));
  if (h->P.precision != FP_PREC_MIXED) return FP_OK;
  // adaptive: the skip flag fl_ir[FL_IRSKIP] turns the remaining sweeps into no-ops
  int *skip = h->fl_ir + FL_IRSKIP;
  CK(cudaMemsetAsync(skip, 0, sizeof(int), h->stream));
  CK(cudaMemsetAsync(h->ir_prev, 0, sizeof(double), h->stream));
  for (int it = 0; it < sweeps; ++it) {
    k_residual_N<<<h->T.S, 256, 0, h->stream>>>(h->D, h->sell_val, b, x, h->XR, skip);
    CKL();
    TRY(solve_local(h, false, h->XR, skip));
    k_local_add<<<1184, 256, 0, h->stream>>>(x, h->XR, nv, skip);
    const double eps = h->ir_eps > 0 ? h->ir_eps : std::min(1e-10, std::max(1e-15, 1e-2 * h->P.tol));
    k_ir_check<<<RED_BLOCKS_IR, 256, 0, h->stream>>>(x, h->XR, nv, eps * eps, h->partial,
                                                  h->red_counter + 2, h->fl_ir, h->ir_prev,
                                                  h->ir_stag * h->ir_stag, h->ir_prev + 1);
    CKL();
  }
  (void)fl;
  return FP_OK;
}

// out = P v (FP64 throughout: an FP32 copy of (G^T G)^{-1} in the PCG loop let lambda drift
// off G^T lambda = e far enough to force restarts on config 5)
fp_status apply_P(fp_handle *h, const double *v, double *out, const int *fl) {
  const int nl = h->T.n_lambda;
  if (!h->T.NF) {
    if (out != v) CK(cudaMemcpyAsync(out, v, nl * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return FP_OK;
  }
  const bool two_float = h->Htiles && h->coarse_2f;
  k_Gt<<<(h->T.NF * 32 + 255) / 256, 256, 0, h->stream>>>(h->D, v, h->cy, fl, two_float ? h->cysplit : nullptr);
  CKL();
  if (two_float) CK(launch_coarse_apply2f(h->Htiles, h->T.nH, h->cysplit, h->Hpart, h->calpha, fl, h->stream));
  else CK(launch_gemv(h->Hinv, h->cy, h->calpha, h->T.nH, fl, h->stream));
  k_Gcomb<<<(nl + 255) / 256, 256, 0, h->stream>>>(h->D, h->calpha, v, -1.0, out, fl);
  CKL();
  return FP_OK;
}

fp_status dot(fp_handle *h, const double *a, const double *b, int op, double *slot, const int *check);

// out = P v, then dot(a, out) -> op (Algorithm 1's reductions after a projection; the last
// projection kernel and the reduction are one launch when there is a coarse space)
fp_status apply_P_dot(fp_handle *h, const double *v, double *out, const double *a, int op) {
  const int nl = h->T.n_lambda;
  if (!h->T.NF) {
    if (out != v) CK(cudaMemcpyAsync(out, v, nl * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return dot(h, a, out, op, nullptr, h->fl);
  }
  const bool two_float = h->Htiles && h->coarse_2f;
  k_Gt<<<(h->T.NF * 32 + 255) / 256, 256, 0, h->stream>>>(h->D, v, h->cy, h->fl, two_float ? h->cysplit : nullptr);
  CKL();
  if (two_float) CK(launch_coarse_apply2f(h->Htiles, h->T.nH, h->cysplit, h->Hpart, h->calpha, h->fl, h->stream));
  else CK(launch_gemv(h->Hinv, h->cy, h->calpha, h->T.nH, h->fl, h->stream));
  k_Gcomb_dot<<<RED_BLOCKS, 256, 0, h->stream>>>(h->D, h->calpha, v, out, a, h->partial, h->red_counter, h->sc,
                                                 h->fl, op);
  CKL();
  return FP_OK;
}

// out = F v.  accurate: local solves refined to FP64 accuracy (mixed precision); the
// solution K^+ B^T v is left in xsol(h) (XA for mixed precision, XB for FP64).
double *xsol(fp_handle *h) { return h->P.precision == FP_PREC_MIXED ? h->XA : h->XB; }

fp_status apply_F(fp_handle *h, const double *v, double *out, const int *fl, bool accurate = true) {
  // explicit F_s: every apply in FP64, the loop's inexact apply in mixed precision (only the
  // rows touched by B are formed, so K^+ B^T v is not left in xsol)
  const bool mixed = h->P.precision == FP_PREC_MIXED;
  const void *op = nullptr;
  if (h->ops_ready) op = !mixed || !accurate ? h->opF : (h->opF64_ready ? h->opF64 : nullptr);
  const bool fused = op && mixed && !accurate;  // the tiled FP32 apply forms B^T v itself
  if (!fused) {
    k_scatter<<<h->T.S, 256, 0, h->stream>>>(h->D, v, 1.0, h->XB, 1, fl, op ? 0 : 1);
    CKL();
  }
  if (op) {
    if (fused)
      CK(launch_explicit_apply_sym(h->D, h->T.S, h->nbnd_max, op, h->tile_off, h->XB, fl, h->stream, v, 1, false));
    else if (mixed && h->opF2 && h->explicit_2f)
      CK(launch_explicit_apply_sym2f(h->D, h->T.S, h->nbnd_max, h->opF2, h->tile_off, h->XB, fl, h->stream));
    else
      CK(launch_explicit_apply(false, h->D, h->T.S, h->nbnd_max, op, h->op_off, h->XB, fl, h->stream));
    k_gather<<<(h->T.n_lambda + 255) / 256, 256, 0, h->stream>>>(h->D, h->XB, out, fl);
    CKL();
    return FP_OK;
  }
  double *x = h->XB;
  if (h->P.precision == FP_PREC_MIXED) {
    x = h->XA;
    TRY(solve_refined(h, h->XB, x, accurate ? h->ir_sweeps : h->inner_ir, fl));
  } else {
    TRY(solve_local(h, false, x, fl));
  }
  k_gather<<<(h->T.n_lambda + 255) / 256, 256, 0, h->stream>>>(h->D, x, out, fl);
  CKL();
  return FP_OK;
}

fp_status apply_M_lumped(fp_handle *h, const double *v, double *out, const int *fl, bool w_done);

// out = W B S B^T W v  (Eq. (3.5) with the scaling W).  w_done: t1 already holds W v (the PCG
// update kernel formed it), so the first scaling is skipped.
fp_status apply_M(fp_handle *h, const double *v, double *out, const int *fl, bool w_done = false) {
  const int nl = h->T.n_lambda;
  const int ng = (int)h->T.wgrp_first.size();
  if (h->P.precond == FP_PRECOND_NONE) {
    if (out != v) CK(cudaMemcpyAsync(out, v, nl * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return FP_OK;
  }
  if (h->P.precond == FP_PRECOND_LUMPED) return apply_M_lumped(h, v, out, fl, w_done);
  if (!w_done) k_wscale<<<(ng + 255) / 256, 256, 0, h->stream>>>(h->D, v, h->t1, fl);
  const bool fused = h->ops_ready && h->P.precision == FP_PREC_MIXED;  // tiled apply forms B^T W v itself
  if (!fused) k_scatter<<<h->T.S, 256, 0, h->stream>>>(h->D, h->t1, 1.0, h->XP, 0, fl, h->ops_ready ? 0 : 1);
  CKL();
  if (h->ops_ready) {
    if (fused) {
      CK(launch_explicit_apply_sym(h->D, h->T.S, h->nbnd_max, h->opS, h->tile_off, h->XP, fl, h->stream, h->t1, 0,
                                   h->opS_bf16 != 0));
      k_gather_wscale<<<(ng + 255) / 256, 256, 0, h->stream>>>(h->D, h->XP, out, fl);
      CKL();
      return FP_OK;
    }
    CK(launch_explicit_apply(false, h->D, h->T.S, h->nbnd_max, h->opS, h->op_off, h->XP, fl, h->stream));
  } else {
    k_halo<<<h->T.S, 256, 0, h->stream>>>(h->D, h->csr_val, h->XP, h->XY, fl);
    CKL();
    TRY(solve_local(h, true, h->XY, fl));
    k_bnd_apply<<<h->T.S, 256, h->nbnd_max * sizeof(double), h->stream>>>(h->D, h->csr_val, h->XY, h->XP, fl);
  }
  CKL();
  k_gather<<<(nl + 255) / 256, 256, 0, h->stream>>>(h->D, h->XP, h->t2, fl);
  k_wscale<<<(ng + 255) / 256, 256, 0, h->stream>>>(h->D, h->t2, out, fl);
  CKL();
  return FP_OK;
}

// out = W B K_bb B^T W v: the lumped preconditioner (Sec. 3.3), the local matrices' interface
// block in place of the Schur complement (no local solve)
fp_status apply_M_lumped(fp_handle *h, const double *v, double *out, const int *fl, bool w_done) {
  const int nl = h->T.n_lambda;
  const int ng = (int)h->T.wgrp_first.size();
  if (!w_done) k_wscale<<<(ng + 255) / 256, 256, 0, h->stream>>>(h->D, v, h->t1, fl);
  k_scatter<<<h->T.S, 256, 0, h->stream>>>(h->D, h->t1, 1.0, h->XP, 0, fl, 1);
  k_bnd_apply<<<h->T.S, 256, h->nbnd_max * sizeof(double), h->stream>>>(h->D, h->csr_val, nullptr, h->XP, fl);
  k_gather<<<(nl + 255) / 256, 256, 0, h->stream>>>(h->D, h->XP, h->t2, fl);
  k_wscale<<<(ng + 255) / 256, 256, 0, h->stream>>>(h->D, h->t2, out, fl);
  CKL();
  return FP_OK;
}

fp_status dot(fp_handle *h, const double *a, const double *b, int op, double *slot, const int *check) {
  k_dot<<<RED_BLOCKS, 256, 0, h->stream>>>(a, b, h->T.n_lambda, h->partial, h->red_counter, h->sc, h->fl, op,
                                           slot, check ? 1 : 0);
  CKL();
  return FP_OK;
}

fp_status lincomb(fp_handle *h, double *out, const double *x, double a, const double *y, double b, const int *fl) {
  const int nl = h->T.n_lambda;
  k_lincomb<<<(nl + 255) / 256, 256, 0, h->stream>>>(out, x, a, y, b, nl, fl);
  CKL();
  return FP_OK;
}


// ------------------------------- learned lambda_0 ------------------------------------
double source_signal(const fp_handle *h, double t) {
  if (h->P.source == FP_SOURCE_POINT) return std::sin(h->P.q_omega * t);
  if (h->P.source == FP_SOURCE_MANUFACTURED_T) return 1.0 + t;
  return 1.0;
}

// forward over `rows` feature rows (device X, rows x 8) -> out (device, rows)
fp_status mlp_forward(fp_handle *h, const float *X, long long rows, float *out) {
  const int CH = fp_handle::CH;
  cudaStream_t s = h->stream;
  if (h->mlp_tc) {  // one fused launch, the 256 x 256 layer on tcgen05 (mlp_tc.cu)
    CK(launch_mlp_forward_tc(rows, X, h->mlpP, out, h->num_sms, h->status, s));
    return FP_OK;
  }
  for (long long r0 = 0; r0 < rows; r0 += CH) {
    const int m = (int)std::min<long long>(CH, rows - r0);
    k_mlp_l1<<<(m * MLP_NH + 255) / 256, 256, 0, s>>>(m, X + r0 * MLP_NIN, h->mlpP, nullptr, h->h1);
    CK(launch_gemm_bf16(s, m, MLP_NH, MLP_NH, h->h1, MLP_NH, 1, h->mlpP + MLP_OFF_W2, MLP_NH, 1, h->h2, MLP_NH,
                        h->mlpP + MLP_OFF_B2, nullptr, nullptr, 1));
    k_mlp_l3<<<(m * 32 + 255) / 256, 256, 0, s>>>(m, h->h2, h->mlpP, out + r0, nullptr, nullptr, nullptr, 0.f);
    CKL();
  }
  return FP_OK;
}

// loss (accumulated into loss_acc) and gradient (into mlpG) of m <= CH rows
fp_status mlp_loss_grad(fp_handle *h, const float *X, const float *Y, int m) {
  cudaStream_t s = h->stream;
  float *P = h->mlpP, *G = h->mlpG;
  k_mlp_l1<<<(m * MLP_NH + 255) / 256, 256, 0, s>>>(m, X, P, h->z1, h->h1);
  CK(launch_gemm_bf16(s, m, MLP_NH, MLP_NH, h->h1, MLP_NH, 1, P + MLP_OFF_W2, MLP_NH, 1, h->h2, MLP_NH,
                      P + MLP_OFF_B2, h->z2, nullptr, 1));
  k_mlp_l3<<<(m * 32 + 255) / 256, 256, 0, s>>>(m, h->h2, P, h->mout, Y, h->dout, h->loss_rows, 1.f / m);
  k_colsum<<<(MLP_NH + 31) / 32, 256, 0, s>>>(m, MLP_NH, h->h2, MLP_NH, h->dout, G + MLP_OFF_W3);
  k_colsum<<<1, 256, 0, s>>>(m, 1, h->dout, 1, nullptr, G + MLP_OFF_B3);
  k_mlp_d2<<<(m * MLP_NH + 255) / 256, 256, 0, s>>>(m, h->dout, P, h->z2, h->z2);  // d2 in place of z2
  k_colsum<<<(MLP_NH + 31) / 32, 256, 0, s>>>(m, MLP_NH, h->z2, MLP_NH, nullptr, G + MLP_OFF_B2);
  CKL();
  // dW2 = h1^T d2
  CK(launch_gemm_bf16(s, MLP_NH, MLP_NH, m, h->h1, 1, MLP_NH, h->z2, MLP_NH, 1, G + MLP_OFF_W2, MLP_NH, nullptr,
                      nullptr, nullptr, 0));
  // d1 = (d2 W2^T) * (z1 > 0), into the h2 buffer
  CK(launch_gemm_bf16(s, m, MLP_NH, MLP_NH, h->z2, MLP_NH, 1, P + MLP_OFF_W2, 1, MLP_NH, h->h2, MLP_NH, nullptr,
                      nullptr, h->z1, 0));
  k_colsum<<<(MLP_NH + 31) / 32, 256, 0, s>>>(m, MLP_NH, h->h2, MLP_NH, nullptr, G + MLP_OFF_B1);
  k_mlp_dw1<<<(MLP_NIN * MLP_NH + 255) / 256, 256, 0, s>>>(m, X, h->h2, G);
  k_sum_double<<<1, 256, 0, s>>>(h->loss_rows, m, h->loss_acc);
  CKL();
  return FP_OK;
}

fp_status mlp_ensure_init(fp_handle *h, unsigned long long seed) {
  if (h->mlp_ready) return FP_OK;
  k_mlp_init<<<(MLP_NPARAM + 255) / 256, 256, 0, h->stream>>>(h->mlpP, seed);
  CKL();
  CK(cudaMemsetAsync(h->mlpM1, 0, MLP_NPARAM * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->mlpM2, 0, MLP_NPARAM * sizeof(float), h->stream));
  h->adam_step = 0;
  h->mlp_ready = 1;
  return FP_OK;
}

// features of step n from lambda^{n-1}, lambda^{n-2} and the source signal (the ratio rho in
// stepv[ST_RHO]); fsum gets the sums of squares of the last increment and of lambda^{n-1}
fp_status build_features(fp_handle *h) {
  const int nl = h->T.n_lambda;
  TRY(lincomb(h, h->t1, h->lam_prev, 1.0, h->lam_prev2, -1.0, nullptr));
  TRY(dot(h, h->t1, h->t1, OP_STORE, h->fsum, nullptr));
  TRY(dot(h, h->lam_prev, h->lam_prev, OP_STORE, h->fsum + 1, nullptr));
  k_features<<<(nl + 255) / 256, 256, 0, h->stream>>>(nl, h->lam_prev, h->lam_prev2, h->fsum, h->stepv, h->xy_rows,
                                                      h->kind_rows, h->comp_rows, h->Xf, h->fscale);
  CKL();
  return FP_OK;
}

fp_status choose_nb(fp_handle *h, bool dbl, const BandTask *tasks, void *buf, int *nb_out);
fp_status run_mrhs(fp_handle *h, int prec, const void *fac, const void *linv, int kind, void *out);
fp_status alloc_op(fp_handle *h, void **p, size_t bytes);

// FP32 factorisation on the tensor cores (k_band_factor_tc): usable when the widest band's
// operands fit in shared memory (half bandwidth <= 511)
bool tc_ok(const fp_handle *h) {
  int bmax = 0;
  for (const Template &t : h->T.tpl) bmax = std::max(bmax, t.b);
  return h->factor_tc && bmax <= 511 && band_factor_tc_smem(h->ldmax, bmax) <= 227 * 1024;
}

// band of K_s (mode 0 Neumann, 1 Dirichlet) in FP32, factorised with 3xTF32 tensor-core trailing
// updates, then the inverse diagonal blocks of the solves; timed with events into factor_tc_ms
fp_status factor_fp32_tc(fp_handle *h, const BandTask *tk, float *fac, float *linv, int mode) {
  int bmax = 0;
  for (const Template &t : h->T.tpl) bmax = std::max(bmax, t.b);
  CK(launch_csr_to_band(true, h->D, h->csr_val, fac, mode, h->stream));
  CK(cudaEventRecord(h->ev[4], h->stream));
  CK(launch_band_factor_tc(tk, h->ntask, fac, h->ldmax, bmax, h->num_sms, h->counter, h->status, h->stream));
  CK(cudaEventRecord(h->ev[5], h->stream));
  CK(launch_band_linv(true, tk, h->ntask, fac, linv, h->stream));
  CK(cudaEventSynchronize(h->ev[5]));
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]);
  h->tuning.factor_tc_ms[mode] = ms;
  return FP_OK;
}

template <typename T>
fp_status factor_T(fp_handle *h) {
  Topology &Tp = h->T;
  const size_t nf = (size_t)Tp.fac_off[Tp.S];
  T *fN = nullptr, *fD = nullptr;
  if (!h->facN) {
    T *lN = nullptr, *lD = nullptr;
    TRY(dalloc(h, &fN, nf));
    TRY(dalloc(h, &fD, nf));
    TRY(dalloc(h, &lN, (size_t)h->linv_total));
    TRY(dalloc(h, &lD, (size_t)h->linv_total));
    h->facN = fN; h->facD = fD; h->linvN = lN; h->linvD = lD;
  }
  fN = (T *)h->facN; fD = (T *)h->facD;
  const bool f32 = sizeof(T) == 4;
  if (f32 && h->factor_fp64) {
    // FP64 factorisation in temporary arrays, then one rounding of the finished factor (and of
    // its inverse diagonal blocks, computed in FP64 from the FP64 factor) to FP32
    double *tN = nullptr, *tL = nullptr;
    CK(cudaMalloc(&tN, nf * sizeof(double)));
    cudaError_t e = cudaMalloc(&tL, (size_t)h->linv_total * sizeof(double));
    if (e != cudaSuccess) { cudaFree(tN); h->err = cudaGetErrorString(e); return FP_ERR_OOM; }
    int NB = 32;
    fp_status st = choose_nb(h, true, h->tasksN, tN, &NB);
    h->tuning.factor_nb = NB;
    const size_t smem = (size_t)NB * (h->ldmax + 1) * sizeof(double);
    for (int mode = 0; mode < 2 && st == FP_OK; ++mode) {
      T *dstF = (T *)(mode == 0 ? h->facN : h->facD);
      T *dstL = (T *)(mode == 0 ? h->linvN : h->linvD);
      const BandTask *tk = mode == 0 ? h->tasksN : h->tasksD;
      if (mode == 1 && tc_ok(h)) {
        // the Dirichlet factor serves only the preconditioner (S_s, or its band solves): FP32 on
        // the tensor cores, no FP64 copy
        st = factor_fp32_tc(h, tk, (float *)dstF, (float *)dstL, 1);
        continue;
      }
      cudaError_t ee = launch_csr_to_band(false, h->D, h->csr_val, tN, mode, h->stream);
      if (ee == cudaSuccess) ee = launch_band_factor(false, tk, h->ntask, tN, NB, h->status, smem, h->stream);
      if (ee == cudaSuccess) ee = launch_band_linv(false, tk, h->ntask, tN, tL, h->stream);
      if (ee == cudaSuccess) ee = launch_round_to_float(tN, (float *)dstF, (long long)nf, h->stream);
      if (ee == cudaSuccess) ee = launch_round_to_float(tL, (float *)dstL, h->linv_total, h->stream);
      if (ee != cudaSuccess) { h->err = cudaGetErrorString(ee); st = FP_ERR_CUDA; }
      if (st == FP_OK && mode == 0 && h->explicit_ops) {
        // F_s in FP64 from the FP64 factor (the accurate applies), and its FP32 rounding (the
        // PCG loop's operator)
        st = alloc_op(h, (void **)&h->opF64, (size_t)h->op_total * 8);
        if (st == FP_OK) st = alloc_op(h, &h->opF, (size_t)h->tile_total * 4);
        if (st == FP_OK && h->explicit_df) {
          // two-float arithmetic on the FP32 units: the FP64 factor (already rounded to FP32
          // above) and its inverse blocks split in place
          ee = launch_split_df(tN, (long long)nf, h->stream);
          if (ee == cudaSuccess) ee = launch_split_df(tL, h->linv_total, h->stream);
          if (ee != cudaSuccess) { h->err = cudaGetErrorString(ee); st = FP_ERR_CUDA; }
        }
        if (st == FP_OK) st = run_mrhs(h, h->explicit_df ? MRHS_DF : MRHS_FP64, tN, tL, 0, h->opF64);
        if (st == FP_OK) {
          ee = launch_pack_sym(true, h->D, h->T.S, h->opF64, h->op_off, (float *)h->opF, h->tile_off, h->stream);
          if (ee != cudaSuccess) { h->err = cudaGetErrorString(ee); st = FP_ERR_CUDA; }
        }
        if (st == FP_OK) st = alloc_op(h, (void **)&h->opF2, (size_t)h->tile_total * 8);
        if (st == FP_OK) {
          ee = launch_pack_sym2f(h->D, h->T.S, h->opF64, h->op_off, h->opF2, h->tile_off, h->stream);
          if (ee != cudaSuccess) { h->err = cudaGetErrorString(ee); st = FP_ERR_CUDA; }
        }
        if (st == FP_OK) h->opF64_ready = 1;
      }
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(tN);
    cudaFree(tL);
    return st;
  }
  if (f32 && tc_ok(h)) {
    TRY(factor_fp32_tc(h, h->tasksN, (float *)fN, (float *)h->linvN, 0));
    TRY(factor_fp32_tc(h, h->tasksD, (float *)fD, (float *)h->linvD, 1));
    return FP_OK;
  }
  int NB = 32;
  TRY(choose_nb(h, !f32, h->tasksN, fN, &NB));
  h->tuning.factor_nb = NB;
  CK(launch_csr_to_band(f32, h->D, h->csr_val, fN, 0, h->stream));
  CK(launch_csr_to_band(f32, h->D, h->csr_val, fD, 1, h->stream));
  const size_t smem = (size_t)NB * (h->ldmax + 1) * sizeof(T);
  CK(launch_band_factor(f32, h->tasksN, h->ntask, fN, NB, h->status, smem, h->stream));
  CK(launch_band_factor(f32, h->tasksD, h->ntask, fD, NB, h->status, smem, h->stream));
  CK(launch_band_linv(f32, h->tasksN, h->ntask, fN, h->linvN, h->stream));
  CK(launch_band_linv(f32, h->tasksD, h->ntask, fD, h->linvD, h->stream));
  return FP_OK;
}

fp_status factor_coarse(fp_handle *h) {
  Topology &T = h->T;
  if (!T.NF) return FP_OK;
  if (!h->Hband) {
    TRY(dalloc(h, &h->Hband, (size_t)T.nH * T.LDH));
    TRY(dalloc(h, &h->Hinv, (size_t)T.nH * T.nH));
  }
  k_coarse_G<<<(T.n_lambda + 255) / 256, 256, 0, h->stream>>>(h->D, h->ga, h->gb);
  k_pack_float_g<<<(T.NF + 7) / 8, 256, 0, h->stream>>>(h->D, const_cast<double *>(h->D.float_g));
  CK(cudaMemsetAsync(h->Hband, 0, (size_t)T.nH * T.LDH * sizeof(double), h->stream));
  k_coarse_GtG<<<(T.NF + 127) / 128, 128, 0, h->stream>>>(h->D, h->ga, h->gb, h->Hband);
  CKL();
  int NB = 32;
  while (NB > 4 && (size_t)NB * (T.LDH + 1) * sizeof(double) > 200 * 1024) NB /= 2;
  const size_t smem = (size_t)NB * (T.LDH + 1) * sizeof(double);
  CK(launch_band_factor(false, h->taskH, 1, h->Hband, NB, h->status, smem, h->stream));
  k_identity<<<1024, 256, 0, h->stream>>>(h->Hinv, T.nH);
  CKL();
  TRY(launch_solve(h, false, h->tasksHinv, T.nH, h->Hband, h->Hinv, h->mmaxH, nullptr));
  if (h->P.precision == FP_PREC_MIXED && h->coarse_2f) {
    const long long nt = (T.nH + 31) / 32, ntile = nt * (nt + 1) / 2;
    if (!h->Htiles) {
      TRY(dalloc(h, &h->Htiles, (size_t)ntile * 2048));
      TRY(dalloc(h, &h->Hpart, (size_t)ntile * 64));   // two-float partials: 2 x ntile x 32 float pairs
      TRY(dalloc(h, &h->cysplit, 2 * (size_t)T.nH));
    }
    CK(launch_coarse_pack2f(h->Hinv, T.nH, h->Htiles, h->stream));
  }
  return FP_OK;
}

// ----------------------------------- autotuner -----------------------------------------
// Panel width of the factorisation: each candidate factorises the 2 x num_sms largest tasks
// (the task list is sorted by cost) after a fresh copy of the band; the fastest is kept.
fp_status choose_nb(fp_handle *h, bool dbl, const BandTask *tasks, void *buf, int *nb_out) {
  const size_t esz = dbl ? 8 : 4;
  auto fits = [&](int nb) { return (size_t)nb * (h->ldmax + 1) * esz <= 200 * 1024; };
  if (h->factor_nb > 0) {
    int nb = h->factor_nb;
    while (nb > 4 && !fits(nb)) nb /= 2;
    *nb_out = nb;
    return FP_OK;
  }
  int nb = 64;
  while (nb > 4 && !fits(nb)) nb /= 2;
  if (nb > 32) nb = 32;
  if (!h->autotune) { *nb_out = nb; return FP_OK; }
  const int sub = std::min(h->ntask, 2 * h->num_sms);
  cudaEvent_t e0 = h->ev[4], e1 = h->ev[5];
  float best = 1e30f;
  for (int cand : {8, 16, 32, 64}) {
    if (!fits(cand)) continue;
    CK(launch_csr_to_band(!dbl, h->D, h->csr_val, buf, 0, h->stream));
    CK(cudaEventRecord(e0, h->stream));
    CK(launch_band_factor(!dbl, tasks, sub, buf, cand, h->status, (size_t)cand * (h->ldmax + 1) * esz, h->stream));
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) { best = ms; nb = cand; }
  }
  h->tuning.factor_ms = best;
  *nb_out = nb;
  return FP_OK;
}

// Launch shape of the blocked solves: every legal (warps per CTA, stage bytes, CTAs per SM)
// is timed on a Neumann solve of all subdomains (a zero vector stays zero, so the scratch
// vector is left as it was); the fastest is kept.  Options set by the caller stay fixed.
fp_status autotune_solve(fp_handle *h) {
  const bool fp32 = h->P.precision == FP_PREC_MIXED;
  const fp_handle::SolveShape def = legal_shape(h, default_shape(h, h->ntask), fp32);
  h->shape = def;
  h->tuning.candidates = 0;
  if (h->autotune && h->solve_kernel == 1) {
    std::vector<fp_handle::SolveShape> cands;
    for (int wpc : {1, 2, 4, 8}) {
      if (h->solve_wpc && wpc != h->solve_wpc) continue;
      for (int chunk : {4096, 8192, 16384, 32768}) {
        if (h->solve_chunk && chunk != h->solve_chunk) continue;
        for (int cps : {1, 2}) {
          if (h->solve_cps && cps != h->solve_cps) continue;
          const fp_handle::SolveShape sh = legal_shape(h, {wpc, chunk, cps}, fp32);
          if (sh.wpc != wpc || sh.cps != cps) continue;
          bool dup = false;
          for (auto &c : cands) dup |= c.wpc == sh.wpc && c.chunk == sh.chunk && c.cps == sh.cps;
          if (!dup) cands.push_back(sh);
        }
      }
    }
    const long long nv = h->T.vec_off[h->T.S];
    cudaEvent_t e0 = h->ev[4], e1 = h->ev[5];
    float best = 1e30f;
    for (const auto &sh : cands) {
      float tot = 0.0f;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaMemsetAsync(h->XB, 0, nv * sizeof(double), h->stream));
        CK(cudaEventRecord(e0, h->stream));
        TRY(launch_solve_shaped(h, fp32, h->tasksN, h->ntask, h->facN, h->XB, h->mmax, nullptr, sh));
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tot += ms;
      }
      ++h->tuning.candidates;
      if (tot / 2 < best) { best = tot / 2; h->shape = sh; }
    }
    h->tuning.solve_ms = best;
  }
  h->tuning.solve_wpc = h->shape.wpc;
  h->tuning.solve_chunk = h->shape.chunk;
  h->tuning.solve_ctas_per_sm = h->shape.cps;
  return FP_OK;
}

// ---------------------------- explicit interface operators ------------------------------
// One operator for every subdomain by the multi-right-hand-side band kernel: kind 0 F_s =
// (K_s^+)_{bb} from Neumann factors, kind 1 S_s = K_bb - K_bi K_ii^{-1} K_ib from Dirichlet
// factors, in the arithmetic prec (MRHS_FP64, MRHS_FP32, or MRHS_DF: factors and inverse blocks
// split into two-float values, FP64 operator).  out: op_total entries (FP32 for MRHS_FP32, else FP64).
fp_status run_mrhs(fp_handle *h, int prec, const void *fac, const void *linv, int kind, void *out) {
  const bool fp32 = prec == MRHS_FP32;
  const size_t esz = fp32 ? 4 : 8;
  int bmax = 0, nmax = 0;
  for (const Template &t : h->T.tpl) { bmax = std::max(bmax, t.b); nmax = std::max(nmax, t.n); }
  const int R = (bmax + 64 + 31) / 32 * 32, LDp = h->ldmax + 4;
  // tiles of 32 right-hand sides, or 16 where the 32-wide window does not fit
  int mt = 32, w = 0;
  int bps = h->explicit_tile == 16 ? 0 : mrhs_blocks_per_sm(prec, bmax, 32, R, LDp);
  if (bps < 1 && h->explicit_tile != 32) { mt = 16; w = 1; bps = mrhs_blocks_per_sm(prec, bmax, 16, R, LDp); }
  if (bps < 1) {
    h->err = "explicit operators: the band is too wide for the shared-memory window";
    return FP_ERR_INVALID;
  }
  const int grid = std::min(bps * h->num_sms, std::max(1, h->mrhs_ntask[w]));
  h->tuning.mrhs_nr[kind] = mrhs_nr(bmax, mt);
  h->tuning.mrhs_mt[kind] = mt;
  h->tuning.mrhs_esz[kind] = (int)esz;
  CK(cudaMemsetAsync(out, 0, (size_t)h->op_total * esz, h->stream));
  const long long sstride = (long long)nmax * mt;
  void *scratch = nullptr;
  CK(cudaMalloc(&scratch, (size_t)grid * sstride * esz));
  CK(cudaEventRecord(h->ev[4], h->stream));
  cudaError_t e = cudaMemsetAsync(h->counter, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = launch_band_mrhs(prec, bmax, mt, grid, h->stream, h->mrhs_s[w], h->mrhs_j0[w], h->mrhs_ntask[w], h->D, fac,
                         linv, h->linv_off_dev, h->csr_val, kind, scratch, sstride, h->counter, out, h->op_off, R,
                         LDp);
  if (e == cudaSuccess) e = launch_mrhs_symmetrize(fp32, h->D, h->T.S, out, h->op_off, mt, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev[5], h->stream);
  const cudaError_t es = cudaStreamSynchronize(h->stream);
  cudaFree(scratch);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) { h->err = std::string("explicit operators: ") + cudaGetErrorString(e); return FP_ERR_CUDA; }
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]);
  h->tuning.explicit_ms += ms;
  h->tuning.mrhs_ms[kind] += ms;
  h->tuning.mrhs_prec[kind] = prec;
  return FP_OK;
}

fp_status alloc_op(fp_handle *h, void **p, size_t bytes) {
  if (!*p) {
    CK(cudaMalloc(p, bytes));
    h->allocs.push_back(*p);
  }
  return FP_OK;
}

// FP64: F_s and S_s in FP64, full.  Mixed: the loop's F_s and S_s as FP32 symmetric tiles;
// F_s is the FP64 one of the factorisation rounded when it exists, else formed in FP32;
// S_s is formed in FP32 from the FP32 Dirichlet factors.
fp_status build_explicit(fp_handle *h) {
  const bool need_S = h->precond_req == FP_PRECOND_DIRICHLET || h->precond_req == FP_PRECOND_AUTO;
  if (h->P.precision == FP_PREC_FP64) {
    TRY(alloc_op(h, &h->opF, (size_t)h->op_total * 8));
    TRY(run_mrhs(h, MRHS_FP64, h->facN, h->linvN, 0, h->opF));
    if (need_S) {
      TRY(alloc_op(h, &h->opS, (size_t)h->op_total * 8));
      TRY(run_mrhs(h, MRHS_FP64, h->facD, h->linvD, 1, h->opS));
    }
    h->ops_ready = 1;
    return FP_OK;
  }
  TRY(alloc_op(h, &h->opF, (size_t)h->tile_total * 4));
  if (need_S) TRY(alloc_op(h, &h->opS, (size_t)h->tile_total * 4));
  void *full = nullptr;
  CK(cudaMalloc(&full, (size_t)h->op_total * 4));
  fp_status st = FP_OK;
  if (!h->opF64_ready) {
    st = run_mrhs(h, MRHS_FP32, h->facN, h->linvN, 0, full);
    if (st == FP_OK && launch_pack_sym(false, h->D, h->T.S, full, h->op_off, (float *)h->opF, h->tile_off,
                                       h->stream) != cudaSuccess) {
      h->err = "explicit operators: packing the symmetric tiles of F_s failed";
      st = FP_ERR_CUDA;
    }
  }
  if (st == FP_OK && need_S) st = run_mrhs(h, MRHS_FP32, h->facD, h->linvD, 1, full);
  h->opS_bf16 = h->precond_bf16;
  if (st == FP_OK && need_S &&
      launch_pack_sym(false, h->D, h->T.S, full, h->op_off, h->opS, h->tile_off, h->stream, h->opS_bf16 != 0) !=
          cudaSuccess) {
    h->err = "explicit operators: packing the symmetric tiles of S_s failed";
    st = FP_ERR_CUDA;
  }
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  cudaFree(full);
  if (st != FP_OK) return st;
  if (e != cudaSuccess) { h->err = cudaGetErrorString(e); return FP_ERR_CUDA; }
  h->ops_ready = 1;
  return FP_OK;
}

// ------------------------------ preconditioner autotuning ------------------------------
// A probe run of Algorithm 1 with preconditioner pc: 30 iterations from lambda_0 = 0 on a
// seeded random right-hand side in range(P) (no stop test); returns the contraction of the
// residual norm per iteration and the time per iteration.  Uses only step scratch vectors.
fp_status pcg_start(fp_handle *h);
fp_status pcg_iteration(fp_handle *h);

fp_status probe_precond(fp_handle *h, int pc, double *rho, double *ms_it) {
  const int nl = h->T.n_lambda, N = 30;
  cudaStream_t s = h->stream;
  h->P.precond = pc;
  std::vector<double> v(nl);
  std::mt19937_64 gen(0x5eed5eedULL);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (double &x : v) x = nd(gen);
  CK(cudaMemcpyAsync(h->t2, v.data(), nl * sizeof(double), cudaMemcpyHostToDevice, s));
  TRY(apply_P(h, h->t2, h->r, h->fl_zero));
  CK(cudaMemsetAsync(h->lam, 0, nl * sizeof(double), s));
  int hfl[FL_N] = {};
  hfl[FL_MAXIT] = N + 1;
  CK(cudaMemcpyAsync(h->fl, hfl, sizeof hfl, cudaMemcpyHostToDevice, s));
  const double zero = 0.0, one = 1.0;
  CK(cudaMemcpyAsync(h->sc + SC_TOL2, &zero, sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->sc + SC_REF2, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  TRY(dot(h, h->r, h->r, OP_STORE, h->nrm, nullptr));
  CK(cudaEventRecord(h->ev[4], s));
  TRY(pcg_start(h));
  for (int i = 0; i < N; ++i) TRY(pcg_iteration(h));
  CK(cudaEventRecord(h->ev[5], s));
  double r0 = 0.0;
  CK(cudaMemcpyAsync(&r0, h->nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_fl, h->fl, FL_N * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_sc, h->sc, SC_N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]));
  const int its = h->h_fl[FL_ITER];
  const double r1 = h->h_sc[SC_RNORM2];
  *ms_it = its > 0 ? ms / its : 1e30;
  *rho = (its > 0 && !h->h_fl[FL_STATUS] && r0 > 0 && r1 == r1) ? std::pow(r1 / r0, 0.5 / its) : 1.0;
  return FP_OK;
}

// FP_PRECOND_AUTO: probe DIRICHLET and LUMPED, keep the smaller predicted time to the
// tolerance, log(tol) / log(rho) iterations at the measured time per iteration
fp_status autotune_precond(fp_handle *h) {
  h->tuning.precond_rate[0] = h->tuning.precond_rate[1] = 0.0;
  h->tuning.precond_ms_per_it[0] = h->tuning.precond_ms_per_it[1] = 0.0;
  if (h->precond_req != FP_PRECOND_AUTO) {
    h->P.precond = h->precond_req;
    h->tuning.precond = h->P.precond;
    return FP_OK;
  }
  const int cand[2] = {FP_PRECOND_DIRICHLET, FP_PRECOND_LUMPED};
  double best = 1e300;
  int pick = FP_PRECOND_DIRICHLET;
  for (int c = 0; c < 2; ++c) {
    double rho = 1.0, msi = 0.0;
    TRY(probe_precond(h, cand[c], &rho, &msi));
    h->tuning.precond_rate[c] = rho;
    h->tuning.precond_ms_per_it[c] = msi;
    const double its = rho > 0.0 && rho < 1.0 ? std::log(h->P.tol) / std::log(rho) : 1e300;
    if (its * msi < best) { best = its * msi; pick = cand[c]; }
  }
  h->P.precond = pick;
  h->tuning.precond = pick;
  return FP_OK;
}

fp_status check_status(fp_handle *h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st == DS_ZERO_PIVOT) { h->err = "zero or non-finite pivot in a local LDL^T factorisation"; return FP_ERR_BREAKDOWN; }
  if (st == DS_TIMEOUT) { h->err = "a bounded device wait gave up (TMA copy did not complete)"; return FP_ERR_TIMEOUT; }
  if (st) { h->err = "device status " + std::to_string(st); return FP_ERR_BREAKDOWN; }
  return FP_OK;
}

// ----------------------------------- one time step -----------------------------------
// A step is recorded by pieces shared by the graph path and the stream path:
// step_prologue (right-hand side, d, lambda_00, lambda_0, the reference residual, r_0 and
// the learned guess), the Krylov loop, and step_recovery.  With use_graph the three are
// captured once into a CUDA graph whose Krylov loop is two nested conditional WHILE nodes,
// so a whole step is one graph launch and no host round trip until its end.

fp_status record_event(fp_handle *h, cudaEvent_t e) {
  CK(cudaEventRecordWithFlags(e, h->stream, h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  return FP_OK;
}

fp_status step_prologue(fp_handle *h, bool use_learned) {
  Topology &T = h->T;
  const int nl = T.n_lambda;
  const bool mixed = h->P.precision == FP_PREC_MIXED;
  cudaStream_t s = h->stream;
  // per-step scalars and flags from pinned host memory (read when this point executes)
  CK(cudaMemcpyAsync(h->stepv, h->h_stepv, ST_N * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->fl, h->h_flinit, FL_N * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->sc + SC_TOL2, h->stepv + ST_TOL2, sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
  // right-hand side f, d = B K^+ f (refined), e = R^T f
  double *fbuf = mixed ? h->XF : h->X2;
  k_rhs<<<T.S, 256, 0, s>>>(h->D, h->DP, h->fstat, h->Zn, h->E0n, h->Reta, h->stepv, fbuf, h->ce);
  CKL();
  TRY(solve_refined(h, fbuf, h->X2, h->ir_sweeps, nullptr));
  k_gather<<<(nl + 255) / 256, 256, 0, s>>>(h->D, h->X2, h->d, nullptr);
  CKL();
  // lambda_00 = G (G^T G)^{-1} e ; lambda_0 = lambda_00 + P lambda^{n-1}
  if (T.NF) {
    CK(launch_gemv(h->Hinv, h->ce, h->calpha, T.nH, nullptr, s));
    k_Gcomb<<<(nl + 255) / 256, 256, 0, s>>>(h->D, h->calpha, nullptr, 1.0, h->lam00, nullptr);
    CKL();
  } else {
    CK(cudaMemsetAsync(h->lam00, 0, nl * sizeof(double), s));
  }
  TRY(apply_P(h, h->lam_prev, h->t1, h->fl_zero));
  TRY(lincomb(h, h->lam, h->lam00, 1.0, h->t1, 1.0, nullptr));
  // reference ||P(d - F lambda_00)|| (guess independent)
  if (T.NF) {
    // the reference only scales the stop test: the loop operator's accuracy is plenty
    TRY(apply_F(h, h->lam00, h->t2, h->fl_zero, false));
    TRY(lincomb(h, h->t2, h->d, 1.0, h->t2, -1.0, nullptr));
    TRY(apply_P(h, h->t2, h->t2, h->fl_zero));
    TRY(dot(h, h->t2, h->t2, OP_STORE, h->sc + SC_REF2, nullptr));
  } else {
    TRY(dot(h, h->d, h->d, OP_STORE, h->sc + SC_REF2, nullptr));
  }
  // r_0 = P(d - F lambda_0) with the accurate operator
  TRY(apply_F(h, h->lam, h->q, h->fl_zero));
  TRY(lincomb(h, h->r, h->d, 1.0, h->q, -1.0, nullptr));
  TRY(apply_P(h, h->r, h->r, h->fl_zero));
  // learned lambda_0: the network predicts a correction to the source-scaled extrapolation;
  // the guess selector takes the point of smallest true projected residual on the affine span of
  // lambda_a = lambda_00 + P lambda^{n-1} (the fallback), the extrapolation and the network's
  // correction (two more accurate F applications).  nrm: [0] ||r_a||^2, [1] ||r_0||^2,
  // [2..6] the Gram entries, [7..8] the coefficients.
  if (use_learned) {
    double *tc = h->t2, *tb = h->lam_b, *u = h->q, *w = h->r_b;
    TRY(build_features(h));
    TRY(mlp_forward(h, h->Xf, nl, h->mout));
    k_guess_dirs<<<(nl + 255) / 256, 256, 0, s>>>(nl, h->lam_prev, h->lam_prev2, h->mout, h->stepv, h->fsum, tc,
                                                   tb);
    CKL();
    TRY(apply_P(h, tc, tc, h->fl_zero));
    TRY(apply_P(h, tb, tb, h->fl_zero));
    // the loop operator for the two images: their errors (~1e-7 of |a u|, |b w|, themselves
    // below ||r_a||) stay far below the tolerance; lambda_0 and r_0 stay exact
    TRY(apply_F(h, tc, u, h->fl_zero, false));
    TRY(apply_P(h, u, u, h->fl_zero));
    TRY(apply_F(h, tb, w, h->fl_zero, false));
    TRY(apply_P(h, w, w, h->fl_zero));
    TRY(dot(h, h->r, h->r, OP_STORE, h->nrm, nullptr));
    TRY(dot(h, u, u, OP_STORE, h->nrm + 2, nullptr));
    TRY(dot(h, u, w, OP_STORE, h->nrm + 3, nullptr));
    TRY(dot(h, w, w, OP_STORE, h->nrm + 4, nullptr));
    TRY(dot(h, u, h->r, OP_STORE, h->nrm + 5, nullptr));
    TRY(dot(h, w, h->r, OP_STORE, h->nrm + 6, nullptr));
    k_span_solve<<<1, 1, 0, s>>>(h->nrm + 2, h->nrm + 7, h->choose_flag);
    k_span_apply<<<(nl + 255) / 256, 256, 0, s>>>(nl, h->lam, h->r, tc, tb, u, w, h->nrm + 7);
    CKL();
    TRY(dot(h, h->r, h->r, OP_STORE, h->nrm + 1, nullptr));
  }
  return FP_OK;
}

// z = P M^{-1} r, p = z, (r, z): the start of Algorithm 1 and of every restart
fp_status pcg_start(fp_handle *h) {
  TRY(dot(h, h->r, h->r, OP_RNORM0, nullptr, nullptr));
  TRY(apply_M(h, h->r, h->z, h->fl_zero));
  TRY(apply_P(h, h->z, h->z, h->fl_zero));
  CK(cudaMemcpyAsync(h->p, h->z, h->T.n_lambda * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  TRY(dot(h, h->r, h->z, OP_RZ_INIT, nullptr, nullptr));
  return FP_OK;
}

// one iteration of Algorithm 1; F may use unrefined FP32 solves (mixed precision); every
// kernel is a no-op once the device flag fl[FL_DONE] is set
fp_status pcg_iteration(fp_handle *h) {
  const int nl = h->T.n_lambda;
  cudaStream_t s = h->stream;
  TRY(apply_F(h, h->p, h->q, h->fl, false));
  TRY(apply_P_dot(h, h->q, h->q, h->p, OP_PQ));
  if (h->P.precond == FP_PRECOND_NONE) {
    k_pcg_update<<<RED_BLOCKS, 256, 0, s>>>(h->lam, h->r, h->p, h->q, nl, h->partial, h->red_counter, h->sc, h->fl);
    CKL();
    TRY(apply_M(h, h->r, h->z, h->fl));
  } else {
    // the update also forms t1 = W r, the preconditioner's first step
    k_pcg_update_w<<<RED_BLOCKS, 256, 0, s>>>(h->D, h->lam, h->r, h->p, h->q, h->t1, h->partial, h->red_counter,
                                             h->sc, h->fl);
    CKL();
    TRY(apply_M(h, h->r, h->z, h->fl, true));
  }
  TRY(apply_P_dot(h, h->z, h->z, h->r, OP_RZ));
  k_pcg_pupdate<<<(nl + 255) / 256, 256, 0, s>>>(h->p, h->z, nl, h->sc, h->fl);
  CKL();
  return FP_OK;
}

// ||P(d - F lambda)||^2 into sc[SC_TRUE2] with the accurate operator; leaves F lambda in t2,
// P(d - F lambda) in t1 and K^+ B^T lambda in xsol(h)
fp_status true_residual(fp_handle *h) {
  TRY(apply_F(h, h->lam, h->t2, h->fl_zero));
  TRY(lincomb(h, h->t1, h->d, 1.0, h->t2, -1.0, nullptr));
  TRY(apply_P(h, h->t1, h->t1, h->fl_zero));
  TRY(dot(h, h->t1, h->t1, OP_STORE, h->sc + SC_TRUE2, nullptr));
  return FP_OK;
}

// Algorithm 1 driven from the host: chunks of pcg_chunk iterations between polls of the
// device flags, restarted from the true residual until the true residual meets tol
fp_status krylov_stream(fp_handle *h, int *restarts_out) {
  cudaStream_t s = h->stream;
  const double tol2 = h->P.tol * h->P.tol;
  int restarts = 0;
  for (;;) {
    TRY(pcg_start(h));
    for (int it = 0; it < h->P.max_it; it += h->pcg_chunk) {
      for (int c = 0; c < h->pcg_chunk; ++c) TRY(pcg_iteration(h));
      CK(cudaMemcpyAsync(h->h_fl, h->fl, FL_N * sizeof(int), cudaMemcpyDeviceToHost, s));
      h->xfer[1] += FL_N * sizeof(int);
      CK(cudaStreamSynchronize(s));
      if (h->h_fl[FL_DONE]) break;
    }
    TRY(true_residual(h));
    CK(cudaMemcpyAsync(h->h_fl, h->fl, FL_N * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_sc, h->sc, SC_N * sizeof(double), cudaMemcpyDeviceToHost, s));
    h->xfer[1] += FL_N * sizeof(int) + SC_N * sizeof(double);
    CK(cudaStreamSynchronize(s));
    const bool ok = h->h_sc[SC_TRUE2] <= tol2 * h->h_sc[SC_REF2];
    if (ok || h->h_fl[FL_STATUS] || restarts >= h->max_restarts || h->h_fl[FL_ITER] >= h->P.max_it) break;
    // restart: r = true residual, keep the iteration count
    ++restarts;
    CK(cudaMemcpyAsync(h->r, h->t1, h->T.n_lambda * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(h->fl + FL_DONE, 0, sizeof(int), s));
  }
  *restarts_out = restarts;
  return FP_OK;
}

// Adds, at the capture position of h->stream, a conditional WHILE node: `arm` launches the
// kernel that sets its first condition value, `body` records the body on capture stream
// cap[depth] (the body's last kernel sets the condition for the next round).
using CondFn = std::function<fp_status(cudaGraphConditionalHandle)>;
// kernel nodes of a graph (not those of the bodies of its conditional nodes)
int count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

fp_status capture_while(fp_handle *h, int depth, const CondFn &arm, const CondFn &body) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaGraph_t cg = nullptr;
  CK(cudaStreamGetCaptureInfo(h->stream, &cst, nullptr, &cg, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive || depth < 1 || depth > 2) {
    h->err = "capture_while: stream not capturing";
    return FP_ERR_STATE;
  }
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, cg, 0, 0));
  TRY(arm(hc));
  const cudaGraphNode_t *dp = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->stream, &cst, nullptr, &cg, &dp, nullptr, &nd));
  std::vector<cudaGraphNode_t> deps(dp, dp + nd);
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hc;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, cg, deps.data(), nullptr, deps.size(), &np));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  cudaStream_t outer = h->stream, bs = h->cap[depth];
  CK(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int was_in_body = h->in_body;
  h->stream = bs;
  h->in_body = 1;
  const fp_status st = body(hc);
  h->in_body = was_in_body;
  h->stream = outer;
  cudaGraph_t ended = nullptr;
  const cudaError_t e = cudaStreamEndCapture(bs, &ended);
  if (st != FP_OK) return st;
  if (e != cudaSuccess) { h->err = std::string("capture of a loop body: ") + cudaGetErrorString(e); return FP_ERR_CUDA; }
  h->gkernels[depth] = count_kernel_nodes(bodyg);
  CK(cudaStreamUpdateCaptureDependencies(outer, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return FP_OK;
}

// Algorithm 1 with restarts as two nested WHILE nodes (recorded while capturing)
fp_status krylov_graph(fp_handle *h) {
  const int nl = h->T.n_lambda;
  const int max_body = (h->P.max_it + h->pcg_chunk - 1) / h->pcg_chunk + 1;
  const CondFn arm_outer = [h](cudaGraphConditionalHandle hc) -> fp_status {
    k_loop_arm_outer<<<1, 1, 0, h->stream>>>(hc, h->fl);
    CKL();
    return FP_OK;
  };
  const CondFn arm_inner = [h](cudaGraphConditionalHandle hc) -> fp_status {
    k_loop_arm_inner<<<1, 1, 0, h->stream>>>(hc, h->fl);
    CKL();
    return FP_OK;
  };
  const CondFn body_inner = [h, max_body](cudaGraphConditionalHandle hc) -> fp_status {
    for (int c = 0; c < h->pcg_chunk; ++c) TRY(pcg_iteration(h));
    k_loop_inner<<<1, 1, 0, h->stream>>>(hc, h->fl, max_body);
    CKL();
    return FP_OK;
  };
  const CondFn body_outer = [&](cudaGraphConditionalHandle hc) -> fp_status {
    // restart: r = true residual of the previous round (no-op in the first round)
    k_copy_if<<<grid_for(nl, 256), 256, 0, h->stream>>>(h->r, h->t1, nl, h->fl + FL_PENDING);
    CKL();
    TRY(pcg_start(h));
    TRY(capture_while(h, 2, arm_inner, body_inner));
    TRY(true_residual(h));
    k_loop_outer<<<1, 1, 0, h->stream>>>(hc, h->fl, h->sc, h->max_restarts);
    CKL();
    return FP_OK;
  };
  return capture_while(h, 1, arm_outer, body_outer);
}

// recovery: alpha = (G^T G)^{-1} G^T (F lambda - d); x_s = K^+ f - K^+ B^T lambda + R alpha
fp_status step_recovery(fp_handle *h) {
  Topology &T = h->T;
  cudaStream_t s = h->stream;
  if (T.NF) {
    TRY(lincomb(h, h->t1, h->t2, 1.0, h->d, -1.0, nullptr));
    k_Gt<<<(T.NF * 32 + 255) / 256, 256, 0, s>>>(h->D, h->t1, h->cy, nullptr, nullptr);
    CK(launch_gemv(h->Hinv, h->cy, h->calpha, T.nH, nullptr, s));
    CKL();
  }
  if (h->ops_ready && (h->P.precision == FP_PREC_FP64 || h->opF64_ready)) {
    // the explicit accurate apply formed only the interface rows of K^+ B^T lambda: one full
    // (refined) solve for the recovery
    k_scatter<<<T.S, 256, 0, s>>>(h->D, h->lam, 1.0, h->XB, 1, nullptr, 1);
    CKL();
    if (h->P.precision == FP_PREC_MIXED) TRY(solve_refined(h, h->XB, h->XA, h->ir_sweeps, nullptr));
    else TRY(solve_local(h, false, h->XB, nullptr));
  }
  k_recover<<<T.S, 256, 0, s>>>(h->D, h->DP, h->X2, xsol(h), h->calpha, h->U, h->XI, h->ETA, h->PP, h->Reta);
  CKL();
  return FP_OK;
}

void drop_graph(fp_handle *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  h->gpending.clear();
}

// captures prologue + Krylov loop + recovery of a step into h->gexec
fp_status capture_step(fp_handle *h, bool use_learned) {
  drop_graph(h);
  // events of the timed prologue launches: at most 4 accurate solves of 1 + ir_sweeps launches
  const size_t need = h->profiling ? 2 * 4 * (size_t)(1 + h->ir_sweeps) : 0;
  while (h->gev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->gev.push_back(e);
  }
  h->gev_used = 0;
  cudaStream_t user = h->stream;
  CK(cudaStreamBeginCapture(h->cap[0], cudaStreamCaptureModeThreadLocal));
  h->stream = h->cap[0];
  h->capturing = 1;
  fp_status st = step_prologue(h, use_learned);
  if (st == FP_OK) st = record_event(h, h->ev[1]);
  if (st == FP_OK) st = krylov_graph(h);
  if (st == FP_OK) st = record_event(h, h->ev[2]);
  if (st == FP_OK) st = step_recovery(h);
  h->capturing = 0;
  h->stream = user;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap[0], &g);
  if (st != FP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    h->gpending.clear();
    if (st == FP_OK) { h->err = std::string("capture of a time step: ") + cudaGetErrorString(e); st = FP_ERR_CUDA; }
    cudaGetLastError();
    return st;
  }
  const cudaError_t ei = cudaGraphInstantiate(&h->gexec, g, 0);
  if (ei != cudaSuccess) {
    cudaGraphDestroy(g);
    h->gexec = nullptr;
    h->gpending.clear();
    h->err = std::string("instantiating the step graph: ") + cudaGetErrorString(ei);
    return FP_ERR_CUDA;
  }
  h->graph = g;
  h->gkernels[0] = count_kernel_nodes(g);
  h->gkey = use_learned ? 1 : 0;
  h->gdirty = 0;
  return FP_OK;
}

}  // namespace

// ====================================== ABI ==========================================
// Parameter checks shared by fp_create and fp_plan (precond AUTO already mapped or not).
static bool params_valid(const fp_params &P) {
  return P.lame_lambda > 0 && P.mu > 0 && P.c0 > 0 && P.tau > 0 && P.mu_f > 0 && P.alpha >= 0 && P.tol > 0 &&
         P.max_it >= 1 && (P.precision == FP_PREC_FP64 || P.precision == FP_PREC_MIXED) &&
         P.precond >= FP_PRECOND_DIRICHLET && P.precond <= FP_PRECOND_AUTO;
}

static bool perm_valid(const double *perm, long long n) {
  for (long long e = 0; e < n; ++e)
    if (!(perm[e] > 0) || !std::isfinite(perm[e])) return false;
  return true;
}

static void sizes_of(const Topology &T, int precision, fp_sizes *o) {
  o->nsub = T.S; o->n_floating = T.NF; o->n_lambda = T.n_lambda; o->n_lambda_p = T.n_lambda_p;
  long long nd = 0;
  int bmax = 0;
  for (int s = 0; s < T.S; ++s) { nd += T.tpl[T.sub_tpl[s]].n; bmax = std::max(bmax, T.tpl[T.sub_tpl[s]].b); }
  o->n_dofs = nd;
  o->n_unode_total = T.unode_off[T.S];
  o->n_pnode_total = T.pnode_off[T.S];
  o->factor_bytes = 2LL * T.fac_off[T.S] * (precision == FP_PREC_MIXED ? 4 : 8);
  o->max_half_band = bmax;
}

extern "C" {

fp_status fp_create(const fp_mesh_desc *mesh, const fp_params *params, void *cuda_stream, fp_handle **out) {
  if (!out) return FP_ERR_INVALID;
  *out = nullptr;
  fp_handle *h = new (std::nothrow) fp_handle();
  if (!h) return FP_ERR_OOM;
  if (!params || !mesh) { delete h; return FP_ERR_INVALID; }
  h->P = *params;
  h->precond_req = h->P.precond;
  if (h->P.precond == FP_PRECOND_AUTO) h->P.precond = FP_PRECOND_DIRICHLET;
  if (!params_valid(h->P)) {
    g_create_err = "fp_create: invalid parameters";
    delete h;
    return FP_ERR_INVALID;
  }
  std::string err;
  bool topo_ok = false;
  try {
    topo_ok = build_topology(mesh, params, h->T, err);
  } catch (const std::bad_alloc &) {
    g_create_err = "fp_create: host allocation failed while building the topology";
    delete h;
    return FP_ERR_OOM;
  }
  if (!topo_ok) {
    g_create_err = "fp_create: " + err;
    delete h;
    return FP_ERR_INVALID;
  }
  if (params->perm) {
    if (!perm_valid(params->perm, h->T.elem_off[h->T.S])) {
      g_create_err = "fp_create: perm values must be positive and finite";
      delete h;
      return FP_ERR_INVALID;
    }
    h->perm.assign(params->perm, params->perm + h->T.elem_off[h->T.S]);
  }
  h->P.perm = nullptr;
  h->stream = (cudaStream_t)cuda_stream;
  {
    // no host fallback: without a usable CUDA device the call fails
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce == cudaSuccess && ndev < 1) ce = cudaErrorNoDevice;
    if (ce == cudaSuccess) ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) {
      g_create_err = std::string("fp_create: no usable CUDA device (") + cudaGetErrorString(ce) + ")";
      cudaGetLastError();
      delete h;
      return FP_ERR_CUDA;
    }
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  fp_status st;
  try {
    st = build_device(h);
  } catch (const std::bad_alloc &) {
    h->err = "fp_create: host allocation failed while building the device data";
    st = FP_ERR_OOM;
  }
  if (st != FP_OK) { g_create_err = h->err; fp_destroy(h); return st; }
  {
    const double esz = h->P.precision == FP_PREC_MIXED ? 4.0 : 8.0;
    for (int s = 0; s < h->T.S; ++s) {
      const Template &t = h->T.tpl[h->T.sub_tpl[s]];
      h->bytes_per_solve += 2.0 * t.n * (t.b + 1) * esz + 4.0 * t.n * 8.0;
      h->flops_per_solve += 4.0 * t.n * t.b + t.n;
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) { fp_destroy(h); return FP_ERR_CUDA; }
  *out = h;
  return FP_OK;
}

fp_status fp_assemble(fp_handle *h) {
  if (!h) return FP_ERR_INVALID;
  Topology &T = h->T;
  CK(cudaMemsetAsync(h->csr_val, 0, T.csr_off[T.S] * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->fstat, 0, T.vec_off[T.S] * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->Zn, 0, T.pnode_off[T.S] * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->E0n, 0, T.pnode_off[T.S] * sizeof(double), h->stream));
  k_assemble<<<T.S, 256, 0, h->stream>>>(h->D, h->DP, h->csr_val, h->fstat, h->Zn, h->E0n);
  CKL();
  if (h->sell_val) {
    k_csr_to_sell<<<T.S, 256, 0, h->stream>>>(h->D, h->csr_val, h->sell_val);
    CKL();
  }
  // initial state: R eta^0 = (eta_0, phi_i) (L2 projection), lambda^0 = 0
  CK(cudaMemcpyAsync(h->Reta, h->E0n, T.pnode_off[T.S] * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemsetAsync(h->lam_prev, 0, std::max(T.n_lambda, 1) * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->lam_prev2, 0, std::max(T.n_lambda, 1) * sizeof(double), h->stream));
  h->hist = 0;
  h->sigma_hist[0] = h->sigma_hist[1] = 0.0;
  CK(cudaMemsetAsync(h->U, 0, 2 * T.unode_off[T.S] * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->XI, 0, T.pnode_off[T.S] * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->ETA, 0, T.pnode_off[T.S] * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->PP, 0, T.pnode_off[T.S] * sizeof(double), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->stage = 1;
  h->step_n = 0;
  return FP_OK;
}

fp_status fp_set_initial(fp_handle *h, const double *u0, const double *p0) {
  if (!h) return FP_ERR_INVALID;
  if (h->stage < 1) { h->err = "fp_set_initial before fp_assemble"; return FP_ERR_STATE; }
  const Topology &T = h->T;
  const size_t nu2 = 2 * (size_t)T.unode_off[T.S], np = (size_t)T.pnode_off[T.S];
  cudaStream_t s = h->stream;
  // the initial fields become the reported fields until the first step
  if (u0) CK(cudaMemcpyAsync(h->U, u0, nu2 * sizeof(double), cudaMemcpyHostToDevice, s));
  else CK(cudaMemsetAsync(h->U, 0, nu2 * sizeof(double), s));
  if (p0) CK(cudaMemcpyAsync(h->PP, p0, np * sizeof(double), cudaMemcpyHostToDevice, s));
  else CK(cudaMemsetAsync(h->PP, 0, np * sizeof(double), s));
  CK(cudaMemsetAsync(h->XI, 0, np * sizeof(double), s));
  CK(cudaMemsetAsync(h->ETA, 0, np * sizeof(double), s));
  k_set_initial<<<T.S, 256, 0, s>>>(h->D, h->DP, u0 ? h->U : nullptr, p0 ? h->PP : nullptr, h->Reta);
  CKL();
  const int nl = std::max(T.n_lambda, 1);
  CK(cudaMemsetAsync(h->lam_prev, 0, nl * sizeof(double), s));
  CK(cudaMemsetAsync(h->lam_prev2, 0, nl * sizeof(double), s));
  CK(cudaMemsetAsync(h->lam, 0, nl * sizeof(double), s));
  CK(cudaStreamSynchronize(s));
  h->step_n = 0;
  h->hist = 0;
  h->sigma_hist[0] = h->sigma_hist[1] = 0.0;
  return FP_OK;
}

fp_status fp_factor(fp_handle *h) {
  if (!h) return FP_ERR_INVALID;
  if (h->stage < 1) { h->err = "fp_factor before fp_assemble"; return FP_ERR_STATE; }
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  h->ops_ready = 0;
  h->opF64_ready = 0;
  h->tuning.explicit_ms = 0;
  h->tuning.solve_mmax = h->mmax;
  h->tuning.factor_tc_ms[0] = h->tuning.factor_tc_ms[1] = 0.0;
  for (int k = 0; k < 2; ++k) {
    h->tuning.mrhs_nr[k] = h->tuning.mrhs_mt[k] = h->tuning.mrhs_esz[k] = 0;
    h->tuning.mrhs_ms[k] = 0.0;
    h->tuning.mrhs_prec[k] = -1;
  }
  CK(cudaMemsetAsync(h->ir_prev, 0, 2 * sizeof(double), h->stream));
  TRY(h->P.precision == FP_PREC_MIXED ? factor_T<float>(h) : factor_T<double>(h));
  TRY(factor_coarse(h));
  TRY(check_status(h));
  TRY(autotune_solve(h));
  TRY(check_status(h));
  if (h->explicit_ops) {
    TRY(build_explicit(h));
    TRY(check_status(h));
  }
  TRY(autotune_precond(h));
  TRY(check_status(h));
  h->stage = 2;
  h->gdirty = 1;
  return FP_OK;
}

fp_status fp_step(fp_handle *h, fp_step_stats *stats) {
  if (!h) return FP_ERR_INVALID;
  if (h->stage < 2) { h->err = "fp_step before fp_factor"; return FP_ERR_STATE; }
  Topology &T = h->T;
  const int nl = T.n_lambda;
  const int n = h->step_n + 1;
  const double t_now = n * h->P.tau;
  cudaStream_t s = h->stream;
  // per-step scalars: t_n, the extrapolation ratio of the source signal, tol^2
  const double tol2 = h->P.tol * h->P.tol;
  const double s0 = source_signal(h, t_now), s1 = h->sigma_hist[0], s2 = h->sigma_hist[1];
  double rho = 1.0;
  if (std::fabs(s1 - s2) > 1e-300) rho = std::max(-4.0, std::min(4.0, (s0 - s1) / (s1 - s2)));
  h->h_stepv[ST_T] = t_now;
  h->h_stepv[ST_RHO] = rho;
  h->h_stepv[ST_TOL2] = tol2;
  h->h_flinit[FL_STAGWIN] = h->stag_window;
  const bool use_learned = h->learned_use && h->mlp_ready && h->hist >= 2;
  int restarts = 0;
  // the prologue copies the per-step scalars and the initial loop flags from pinned memory
  // (graph path: as memcpy nodes replayed every launch)
  h->xfer[0] = ST_N * sizeof(double) + FL_N * sizeof(int);
  h->xfer[1] = 0;
  if (h->use_graph) {
    if (!h->gexec || h->gdirty || h->gkey != (use_learned ? 1 : 0)) TRY(capture_step(h, use_learned));
    CK(cudaEventRecord(h->ev[0], s));
    CK(cudaGraphLaunch(h->gexec, s));
    h->pending.insert(h->pending.end(), h->gpending.begin(), h->gpending.end());
  } else {
    CK(cudaEventRecord(h->ev[0], s));
    TRY(step_prologue(h, use_learned));
    CK(cudaEventRecord(h->ev[1], s));
    TRY(krylov_stream(h, &restarts));
    CK(cudaEventRecord(h->ev[2], s));
    TRY(step_recovery(h));
  }
  // training samples: features of this step and target (lambda^n - lambda^{n-1}) / s1
  int extra_launches = 0;
  if (h->learned_record && h->hist >= 2 && h->n_samples < h->cap_samples) {
    if (!use_learned) TRY(build_features(h));
    extra_launches = 1 + (use_learned ? 0 : 4);  // k_record, and build_features' four kernels
    const int per = std::min(h->record_per_step, nl);
    const int stride = std::max(1, nl / per);
    const int r0 = (int)(h->step_n % stride);
    const long long cnt = (nl - r0 + stride - 1) / stride;
    k_record<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(nl, h->Xf, h->lam, h->lam_prev, h->lam_prev2, h->stepv,
                                                           h->fsum, r0, stride, h->n_samples, h->cap_samples, h->SX,
                                                           h->SY);
    CKL();
    h->n_samples = std::min(h->cap_samples, h->n_samples + cnt);
  }
  // history: lambda^{n-2} <- lambda^{n-1} <- lambda^n
  CK(cudaMemcpyAsync(h->lam_prev2, h->lam_prev, nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->lam_prev, h->lam, nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
  h->sigma_hist[1] = h->sigma_hist[0];
  h->sigma_hist[0] = s0;
  h->hist += 1;
  CK(cudaEventRecord(h->ev[3], s));
  CK(cudaMemcpyAsync(h->h_fl, h->fl, FL_N * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_sc, h->sc, SC_N * sizeof(double), cudaMemcpyDeviceToHost, s));
  h->xfer[1] += FL_N * sizeof(int) + SC_N * sizeof(double) + sizeof(int);  // + the status word below
  double hn[2] = {-1, -1};
  int hflag = 0;
  if (use_learned) {
    CK(cudaMemcpyAsync(hn, h->nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hflag, h->choose_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    h->xfer[1] += 2 * sizeof(double) + sizeof(int);
  }
  CK(cudaStreamSynchronize(s));
  TRY(collect_profile(h));
  if (h->use_graph) restarts = h->h_fl[FL_RESTARTS];
  h->restarts_last = restarts;
  float ms01 = 0, ms12 = 0, ms23 = 0;
  cudaEventElapsedTime(&ms01, h->ev[0], h->ev[1]);
  cudaEventElapsedTime(&ms12, h->ev[1], h->ev[2]);
  cudaEventElapsedTime(&ms23, h->ev[2], h->ev[3]);
  h->last_ms[0] = ms01; h->last_ms[1] = ms12; h->last_ms[2] = ms23; h->last_ms[3] = restarts;
  h->step_n = n;
  const double ref2 = h->h_sc[SC_REF2];
  h->last_learned = hflag;
  h->last_res_prev = hn[0] >= 0 && ref2 > 0 ? std::sqrt(hn[0] / ref2) : -1.0;
  h->last_res_learned = hn[1] >= 0 && ref2 > 0 ? std::sqrt(hn[1] / ref2) : -1.0;
  if (stats) {
    stats->step = n;
    stats->iterations = h->h_fl[FL_ITER];
    stats->lambda0_learned = hflag;
    stats->guess_res_prev = h->last_res_prev;
    stats->guess_res_learned = h->last_res_learned;
    stats->rel_residual = ref2 > 0 ? std::sqrt(h->h_sc[SC_RNORM2] / ref2) : 0.0;
    stats->true_rel_residual = ref2 > 0 ? std::sqrt(h->h_sc[SC_TRUE2] / ref2) : 0.0;
    stats->restarts = restarts;
    stats->stagnations = h->h_fl[FL_NSTAG];
    stats->h2d_bytes = h->xfer[0];
    stats->d2h_bytes = h->xfer[1];
    // graph path: the step graph's kernel nodes, the outer body's per round, the inner body's per
    // execution (counted on the device), plus the recording kernels launched after the graph
    stats->kernel_launches = h->use_graph ? h->gkernels[0] + (long long)(restarts + 1) * h->gkernels[1] +
                                                (long long)h->h_fl[FL_NINNER] * h->gkernels[2] + extra_launches
                                          : -1;
  }
  fp_status st = check_status(h);
  if (st) return st;
  if (h->h_fl[FL_STATUS] == DS_BREAKDOWN) { h->err = "PCG breakdown (p^T F p = 0 or non-finite)"; return FP_ERR_BREAKDOWN; }
  if (h->h_fl[FL_STATUS]) { h->err = "non-finite values in PCG"; return FP_ERR_BREAKDOWN; }
  if (!(h->h_sc[SC_TRUE2] <= tol2 * ref2)) { h->err = "PCG did not reach tol within max_it / restarts"; return FP_ERR_NOT_CONVERGED; }
  return FP_OK;
}

fp_status fp_run(fp_handle *h, int n_steps, fp_step_stats *last) {
  if (!h || n_steps < 0) return FP_ERR_INVALID;
  for (int i = 0; i < n_steps; ++i) {
    fp_status st = fp_step(h, last);
    if (st) return st;
  }
  return FP_OK;
}

fp_status fp_get_sizes(const fp_handle *h, fp_sizes *o) {
  if (!h || !o) return FP_ERR_INVALID;
  sizes_of(h->T, h->P.precision, o);
  return FP_OK;
}

fp_status fp_plan(const fp_mesh_desc *mesh, const fp_params *params, fp_sizes *out, int *lambda_keys) {
  if (!mesh || !params || !out) { g_create_err = "fp_plan: null argument"; return FP_ERR_INVALID; }
  if (!params_valid(*params)) { g_create_err = "fp_plan: invalid parameters"; return FP_ERR_INVALID; }
  try {
    Topology T;
    std::string err;
    if (!build_topology(mesh, params, T, err)) { g_create_err = "fp_plan: " + err; return FP_ERR_INVALID; }
    if (params->perm && !perm_valid(params->perm, T.elem_off[T.S])) {
      g_create_err = "fp_plan: perm values must be positive and finite";
      return FP_ERR_INVALID;
    }
    sizes_of(T, params->precision, out);
    if (lambda_keys && T.n_lambda)
      std::memcpy(lambda_keys, T.lam_key.data(), (size_t)6 * T.n_lambda * sizeof(int));
  } catch (const std::bad_alloc &) {
    g_create_err = "fp_plan: host allocation failed";
    return FP_ERR_OOM;
  }
  return FP_OK;
}

static fp_status copy_out(fp_handle *h, void *dst, const void *src, size_t bytes, int on_device) {
  if (!dst) return FP_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FP_OK;
}

fp_status fp_get_lambda(const fp_handle *hc, double *dst, int on_device) {
  fp_handle *h = const_cast<fp_handle *>(hc);
  if (!h || !dst) return FP_ERR_INVALID;
  return copy_out(h, dst, h->lam_prev, h->T.n_lambda * sizeof(double), on_device);
}

fp_status fp_get_lambda_keys(const fp_handle *h, int *keys) {
  if (!h || !keys) return FP_ERR_INVALID;
  std::memcpy(keys, h->T.lam_key.data(), h->T.lam_key.size() * sizeof(int));
  return FP_OK;
}

fp_status fp_get_fields(const fp_handle *hc, double *u, double *xi, double *eta, double *p, int on_device) {
  fp_handle *h = const_cast<fp_handle *>(hc);
  if (!h) return FP_ERR_INVALID;
  const Topology &T = h->T;
  TRY(copy_out(h, u, h->U, 2 * T.unode_off[T.S] * sizeof(double), on_device));
  TRY(copy_out(h, xi, h->XI, T.pnode_off[T.S] * sizeof(double), on_device));
  TRY(copy_out(h, eta, h->ETA, T.pnode_off[T.S] * sizeof(double), on_device));
  TRY(copy_out(h, p, h->PP, T.pnode_off[T.S] * sizeof(double), on_device));
  return FP_OK;
}

fp_status fp_get_subdomain(const fp_handle *hc, int s, double *u, double *xi, double *eta, double *p,
                           int on_device) {
  fp_handle *h = const_cast<fp_handle *>(hc);
  if (!h) return FP_ERR_INVALID;
  const Topology &T = h->T;
  if (s < 0 || s >= T.S) { h->err = "fp_get_subdomain: subdomain out of range"; return FP_ERR_INVALID; }
  const long long u0 = T.unode_off[s], nu = T.unode_off[s + 1] - u0;
  const long long p0 = T.pnode_off[s], np = T.pnode_off[s + 1] - p0;
  TRY(copy_out(h, u, h->U + 2 * u0, 2 * nu * sizeof(double), on_device));
  TRY(copy_out(h, xi, h->XI + p0, np * sizeof(double), on_device));
  TRY(copy_out(h, eta, h->ETA + p0, np * sizeof(double), on_device));
  TRY(copy_out(h, p, h->PP + p0, np * sizeof(double), on_device));
  return FP_OK;
}

// ------------------------------- checkpoint / restore ----------------------------------
// File: magic, version, the sizes that identify the topology, the host scalars of the time
// stepping, then the device arrays in a fixed order (little-endian doubles / floats).
namespace {
constexpr char kCkptMagic[8] = {'F', 'E', 'T', 'I', 'P', 'E', 'C', 'K'};
constexpr int kCkptVersion = 2;
struct CkptHeader {
  char magic[8];
  int version, S, n_lambda, order_k;
  long long nv, np, nu, nparam;
  int step_n, hist, mlp_ready, adam_step, learned_use, pad;
  double sigma0, sigma1;
};

struct CkptArray { void *dev; size_t bytes; };

std::vector<CkptArray> ckpt_arrays(fp_handle *h) {
  const Topology &T = h->T;
  const size_t nl = (size_t)T.n_lambda, np = (size_t)T.pnode_off[T.S], nu = (size_t)T.unode_off[T.S];
  return {{h->lam_prev, nl * 8}, {h->lam_prev2, nl * 8}, {h->lam, nl * 8}, {h->Reta, np * 8},
          {h->U, 2 * nu * 8}, {h->XI, np * 8}, {h->ETA, np * 8}, {h->PP, np * 8},
          {h->mlpP, (size_t)MLP_NPARAM * 4}, {h->mlpM1, (size_t)MLP_NPARAM * 4}, {h->mlpM2, (size_t)MLP_NPARAM * 4},
          {h->ir_prev + 1, sizeof(double)}};
}

CkptHeader ckpt_header(const fp_handle *h) {
  CkptHeader c{};
  std::memcpy(c.magic, kCkptMagic, 8);
  c.version = kCkptVersion;
  c.S = h->T.S; c.n_lambda = h->T.n_lambda; c.order_k = h->T.k;
  c.nv = h->T.vec_off[h->T.S]; c.np = h->T.pnode_off[h->T.S]; c.nu = h->T.unode_off[h->T.S];
  c.nparam = MLP_NPARAM;
  return c;
}
}  // namespace

fp_status fp_checkpoint(const fp_handle *hc, const char *path) {
  fp_handle *h = const_cast<fp_handle *>(hc);
  if (!h || !path) return FP_ERR_INVALID;
  CkptHeader c = ckpt_header(h);
  c.step_n = h->step_n; c.hist = h->hist; c.mlp_ready = h->mlp_ready; c.adam_step = h->adam_step;
  c.learned_use = h->learned_use;
  c.sigma0 = h->sigma_hist[0]; c.sigma1 = h->sigma_hist[1];
  CK(cudaStreamSynchronize(h->stream));
  FILE *f = std::fopen(path, "wb");
  if (!f) { h->err = std::string("fp_checkpoint: cannot open ") + path; return FP_ERR_INVALID; }
  bool ok = std::fwrite(&c, sizeof c, 1, f) == 1;
  std::vector<unsigned char> buf;
  for (const CkptArray &a : ckpt_arrays(h)) {
    if (!ok) break;
    try {
      buf.resize(a.bytes);
    } catch (const std::bad_alloc &) {
      std::fclose(f);
      h->err = "fp_checkpoint: host allocation failed";
      return FP_ERR_OOM;
    }
    if (a.bytes && cudaMemcpy(buf.data(), a.dev, a.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(f);
      h->err = "fp_checkpoint: device read failed";
      return FP_ERR_CUDA;
    }
    ok = a.bytes == 0 || std::fwrite(buf.data(), 1, a.bytes, f) == a.bytes;
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) { h->err = std::string("fp_checkpoint: write failed: ") + path; return FP_ERR_INVALID; }
  return FP_OK;
}

fp_status fp_restore(fp_handle *h, const char *path) {
  if (!h || !path) return FP_ERR_INVALID;
  if (h->stage < 1) { h->err = "fp_restore before fp_assemble"; return FP_ERR_STATE; }
  FILE *f = std::fopen(path, "rb");
  if (!f) { h->err = std::string("fp_restore: cannot open ") + path; return FP_ERR_INVALID; }
  CkptHeader c{};
  const CkptHeader want = ckpt_header(h);
  if (std::fread(&c, sizeof c, 1, f) != 1 || std::memcmp(c.magic, kCkptMagic, 8) != 0 || c.version != kCkptVersion ||
      c.S != want.S || c.n_lambda != want.n_lambda || c.order_k != want.order_k || c.nv != want.nv ||
      c.np != want.np || c.nu != want.nu || c.nparam != want.nparam) {
    std::fclose(f);
    h->err = "fp_restore: not a checkpoint of this problem (magic, version or sizes differ)";
    return FP_ERR_INVALID;
  }
  std::vector<std::vector<unsigned char>> data;
  for (const CkptArray &a : ckpt_arrays(h)) {
    try {
      data.emplace_back(a.bytes);
    } catch (const std::bad_alloc &) {
      std::fclose(f);
      h->err = "fp_restore: host allocation failed";
      return FP_ERR_OOM;
    }
    if (a.bytes && std::fread(data.back().data(), 1, a.bytes, f) != a.bytes) {
      std::fclose(f);
      h->err = "fp_restore: file truncated";
      return FP_ERR_INVALID;
    }
  }
  const bool trailing = std::fgetc(f) != EOF;
  std::fclose(f);
  if (trailing) { h->err = "fp_restore: bytes after the last array (not a checkpoint of this problem)"; return FP_ERR_INVALID; }
  const auto arrays = ckpt_arrays(h);
  CK(cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < arrays.size(); ++i)
    if (arrays[i].bytes) CK(cudaMemcpy(arrays[i].dev, data[i].data(), arrays[i].bytes, cudaMemcpyHostToDevice));
  h->step_n = c.step_n; h->hist = c.hist; h->mlp_ready = c.mlp_ready; h->adam_step = c.adam_step;
  h->learned_use = c.learned_use;
  h->sigma_hist[0] = c.sigma0; h->sigma_hist[1] = c.sigma1;
  h->gdirty = 1;
  return FP_OK;
}

static fp_status apply_op_abi(fp_handle *h, const double *v, double *out, int on_device, int which) {
  if (!h || !v || !out) return FP_ERR_INVALID;
  if (h->stage < 2) { h->err = "operator before fp_factor"; return FP_ERR_STATE; }
  const size_t bytes = h->T.n_lambda * sizeof(double);
  double *vin = h->p;  // scratch copy of the input
  CK(cudaMemcpyAsync(vin, v, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  fp_status st = which == 0 ? apply_F(h, vin, h->q, h->fl_zero)
                 : which == 1 ? apply_M(h, vin, h->q, h->fl_zero)
                              : apply_P(h, vin, h->q, h->fl_zero);
  if (st) return st;
  TRY(copy_out(h, out, h->q, bytes, on_device));
  TRY(collect_profile(h));
  return check_status(h);
}

fp_status fp_apply_F(fp_handle *h, const double *v, double *out, int on_device) { return apply_op_abi(h, v, out, on_device, 0); }
fp_status fp_apply_precond(fp_handle *h, const double *v, double *out, int on_device) { return apply_op_abi(h, v, out, on_device, 1); }
fp_status fp_apply_projection(fp_handle *h, const double *v, double *out, int on_device) { return apply_op_abi(h, v, out, on_device, 2); }

fp_status fp_get_dof_map(const fp_handle *h, int s, int *field, int *node, int *n_out) {
  if (!h || s < 0 || s >= h->T.S) return FP_ERR_INVALID;
  const Template &t = h->T.tpl[h->T.sub_tpl[s]];
  if (n_out) *n_out = t.n;
  if (field) std::memcpy(field, t.dof_field.data(), t.n * sizeof(int));
  if (node) std::memcpy(node, t.dof_node.data(), t.n * sizeof(int));
  return FP_OK;
}

fp_status fp_get_local_matrix(const fp_handle *hc, int s, double *dense) {
  fp_handle *h = const_cast<fp_handle *>(hc);
  if (!h || !dense || s < 0 || s >= h->T.S) return FP_ERR_INVALID;
  if (h->stage < 1) { h->err = "before fp_assemble"; return FP_ERR_STATE; }
  const Template &t = h->T.tpl[h->T.sub_tpl[s]];
  double *band = nullptr, *out = nullptr;
  CK(cudaMalloc(&band, (size_t)t.n * t.LD * sizeof(double)));
  CK(cudaMalloc(&out, (size_t)t.n * t.n * sizeof(double)));
  // rebuild the plain (Neumann, no identity rows) band of s from the CSR values
  std::vector<double> hv(t.csr_col.size());
  cudaMemcpy(hv.data(), h->csr_val + h->T.csr_off[s], hv.size() * sizeof(double), cudaMemcpyDeviceToHost);
  std::vector<double> hb((size_t)t.n * t.LD, 0.0);
  for (int r = 0; r < t.n; ++r)
    for (int e = t.csr_ptr[r]; e < t.csr_ptr[r + 1]; ++e) {
      const int c = t.csr_col[e];
      if (c <= r) hb[(size_t)c * t.LD + r % t.LD] = hv[e];
    }
  cudaMemcpy(band, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice);
  launch_band_to_dense(band, t.n, t.LD, t.b, out, nullptr);
  cudaError_t e = cudaMemcpy(dense, out, (size_t)t.n * t.n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(band);
  cudaFree(out);
  if (e != cudaSuccess) { h->err = cudaGetErrorString(e); return FP_ERR_CUDA; }
  return FP_OK;
}

fp_status fp_get_step_timing(const fp_handle *h, double *ms4) {
  if (!h || !ms4) return FP_ERR_INVALID;
  for (int i = 0; i < 4; ++i) ms4[i] = h->last_ms[i];
  return FP_OK;
}


// ------------------------------- learned lambda_0 ABI --------------------------------
fp_status fp_learned_record(fp_handle *h, int on, long long max_samples, int per_step) {
  if (!h || max_samples < 0 || per_step < 1) return FP_ERR_INVALID;
  if (on && max_samples > h->cap_samples) {
    float *sx = nullptr, *sy = nullptr;
    TRY(dalloc(h, &sx, (size_t)max_samples * MLP_NIN));
    TRY(dalloc(h, &sy, (size_t)max_samples));
    if (h->SX && h->n_samples)
      CK(cudaMemcpyAsync(sx, h->SX, h->n_samples * MLP_NIN * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    if (h->SY && h->n_samples)
      CK(cudaMemcpyAsync(sy, h->SY, h->n_samples * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, h->SX);  // the smaller store it replaces
    dfree(h, h->SY);
    h->SX = sx; h->SY = sy; h->cap_samples = max_samples;
  }
  h->learned_record = on ? 1 : 0;
  h->record_per_step = per_step;
  return FP_OK;
}

fp_status fp_learned_use(fp_handle *h, int on) {
  if (!h) return FP_ERR_INVALID;
  if (on && !h->mlp_ready) { h->err = "fp_learned_use: the network has no parameters (train or set them)"; return FP_ERR_STATE; }
  h->learned_use = on ? 1 : 0;
  return FP_OK;
}

fp_status fp_learned_num_samples(const fp_handle *h, long long *n) {
  if (!h || !n) return FP_ERR_INVALID;
  *n = h->n_samples;
  return FP_OK;
}

fp_status fp_mlp_init(fp_handle *h, unsigned long long seed) {
  if (!h) return FP_ERR_INVALID;
  h->mlp_ready = 0;
  TRY(mlp_ensure_init(h, seed));
  CK(cudaStreamSynchronize(h->stream));
  return FP_OK;
}

fp_status fp_mlp_set_params(fp_handle *h, const float *host, int n) {
  if (!h || !host || n != MLP_NPARAM) return FP_ERR_INVALID;
  CK(cudaMemcpyAsync(h->mlpP, host, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->mlpM1, 0, MLP_NPARAM * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->mlpM2, 0, MLP_NPARAM * sizeof(float), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->adam_step = 0;
  h->mlp_ready = 1;
  return FP_OK;
}

fp_status fp_mlp_get_params(const fp_handle *hc, float *host, int n) {
  fp_handle *h = const_cast<fp_handle *>(hc);
  if (!h || !host || n != MLP_NPARAM) return FP_ERR_INVALID;
  CK(cudaMemcpyAsync(host, h->mlpP, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FP_OK;
}

fp_status fp_mlp_forward(fp_handle *h, const float *x, int rows, float *out) {
  if (!h || !x || !out || rows < 1 || rows > fp_handle::CH) return FP_ERR_INVALID;
  if (!h->mlp_ready) { h->err = "no MLP parameters"; return FP_ERR_STATE; }
  CK(cudaMemcpyAsync(h->xb, x, (size_t)rows * MLP_NIN * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  TRY(mlp_forward(h, h->xb, rows, h->mout));
  CK(cudaMemcpyAsync(out, h->mout, rows * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FP_OK;
}

fp_status fp_mlp_loss_grad(fp_handle *h, const float *x, const float *y, int rows, float *grad, double *loss) {
  if (!h || !x || !y || !grad || rows < 1 || rows > fp_handle::CH) return FP_ERR_INVALID;
  if (!h->mlp_ready) { h->err = "no MLP parameters"; return FP_ERR_STATE; }
  CK(cudaMemcpyAsync(h->xb, x, (size_t)rows * MLP_NIN * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->yb, y, rows * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->loss_acc, 0, sizeof(double), h->stream));
  TRY(mlp_loss_grad(h, h->xb, h->yb, rows));
  CK(cudaMemcpyAsync(grad, h->mlpG, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  double l = 0;
  CK(cudaMemcpyAsync(&l, h->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (loss) *loss = l;
  return FP_OK;
}

// Adam on minibatches of the recorded samples; the order of the samples in every epoch is a
// Fisher-Yates shuffle driven by SplitMix64 (seed, epoch).
fp_status fp_learned_train(fp_handle *h, int epochs, int batch, double lr, unsigned long long seed, double *last_loss) {
  if (!h || epochs < 1 || batch < 32 || batch > fp_handle::CH || !(lr > 0)) return FP_ERR_INVALID;
  if (h->n_samples < batch) { h->err = "fp_learned_train: fewer recorded samples than one batch"; return FP_ERR_STATE; }
  TRY(mlp_ensure_init(h, seed));
  const long long ns = h->n_samples;
  const long long nb = ns / batch;
  std::vector<int> perm(ns);
  if (h->train_idx_cap < ns) {
    if (h->train_idx) cudaFree(h->train_idx);
    h->train_idx = nullptr;
    h->train_idx_cap = 0;
    CK(cudaMalloc(&h->train_idx, (size_t)ns * sizeof(int)));
    h->train_idx_cap = ns;
  }
  int *didx = h->train_idx;
  double epoch_loss = 0;
  for (int e = 0; e < epochs; ++e) {
    for (long long i = 0; i < ns; ++i) perm[i] = (int)i;
    unsigned long long ctr = 0;
    for (long long i = ns - 1; i > 0; --i) {
      unsigned long long z = (seed ^ (0x5851F42D4C957F2DULL * (e + 1))) + (++ctr) * 0x9E3779B97F4A7C15ULL;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
      z ^= z >> 31;
      std::swap(perm[i], perm[z % (unsigned long long)(i + 1)]);
    }
    CK(cudaMemcpyAsync(didx, perm.data(), ns * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->loss_acc, 0, sizeof(double), h->stream));
    for (long long b = 0; b < nb; ++b) {
      k_gather_rows<<<(batch * (MLP_NIN + 1) + 255) / 256, 256, 0, h->stream>>>(batch, didx + b * batch, h->SX, h->SY,
                                                                                h->xb, h->yb);
      CKL();
      TRY(mlp_loss_grad(h, h->xb, h->yb, batch));
      k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, h->stream>>>(h->mlpP, h->mlpG, h->mlpM1, h->mlpM2, MLP_NPARAM,
                                                              (float)lr, 0.9f, 0.999f, 1e-8f, ++h->adam_step);
      CKL();
    }
    double l = 0;
    CK(cudaMemcpyAsync(&l, h->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    epoch_loss = l / nb;
  }
  if (last_loss) *last_loss = epoch_loss;
  return FP_OK;
}

fp_status fp_set_option(fp_handle *h, const char *key, double value) {
  if (!h || !key) return FP_ERR_INVALID;
  const std::string k(key);
  const int v = (int)value;
  auto bad = [&]() { h->err = "fp_set_option: bad value for " + k; return FP_ERR_INVALID; };
  if (k == "ir_sweeps") { if (v < 0 || v > 16) return bad(); h->ir_sweeps = v; }
  else if (k == "inner_ir") { if (v < 0 || v > 8) return bad(); h->inner_ir = v; }
  else if (k == "ir_stag") { if (!(value >= 0.0) || value >= 1.0) return bad(); h->ir_stag = value; }
  else if (k == "ir_eps") { if (value != 0.0 && (!(value >= 1e-17) || value > 1e-2)) return bad(); h->ir_eps = value; }
  else if (k == "max_restarts") { if (v < 0 || v > 64) return bad(); h->max_restarts = v; }
  else if (k == "pcg_chunk") { if (v < 1 || v > 256) return bad(); h->pcg_chunk = v; }
  else if (k == "solve_kernel") { if (v < 0 || v > 1) return bad(); h->solve_kernel = v; }
  else if (k == "solve_wpc") { if (v < 0 || v > 8) return bad(); h->solve_wpc = v; }
  else if (k == "factor_fp64") { if (v < 0 || v > 1) return bad(); h->factor_fp64 = v; }
  else if (k == "graph") { if (v < 0 || v > 1) return bad(); h->use_graph = v; }
  else if (k == "stag_window") { if (v < 0 || v > 100000) return bad(); h->stag_window = v; }
  else if (k == "solve_chunk") { if (v != 0 && (v < 4096 || v > 65536 || v % 1024)) return bad(); h->solve_chunk = v; }
  else if (k == "solve_cps") { if (v < 0 || v > 2) return bad(); h->solve_cps = v; }
  else if (k == "factor_nb") { if (v != 0 && (v < 4 || v > 64 || v % 4)) return bad(); h->factor_nb = v; }
  else if (k == "explicit") { if (v < 0 || v > 1) return bad(); h->explicit_ops = v; }
  else if (k == "explicit_tile") { if (v != 0 && v != 16 && v != 32) return bad(); h->explicit_tile = v; }
  else if (k == "autotune") { if (v < 0 || v > 1) return bad(); h->autotune = v; }
  else if (k == "mlp_tc") { if (v < 0 || v > 1) return bad(); h->mlp_tc = v; }
  else if (k == "factor_tc") { if (v < 0 || v > 1) return bad(); h->factor_tc = v; }
  else if (k == "explicit_df") { if (v < 0 || v > 1) return bad(); h->explicit_df = v; }
  else if (k == "precond_bf16") { if (v < 0 || v > 1) return bad(); h->precond_bf16 = v; }
  else if (k == "explicit_2f") { if (v < 0 || v > 1) return bad(); h->explicit_2f = v; }
  else if (k == "coarse_2f") { if (v < 0 || v > 1) return bad(); h->coarse_2f = v; }
  else if (k == "tol") { if (!(value > 0.0) || !(value < 1.0)) return bad(); h->P.tol = value; }
  else { h->err = "fp_set_option: unknown key " + k; return FP_ERR_INVALID; }
  h->gdirty = 1;
  return FP_OK;
}

fp_status fp_set_profiling(fp_handle *h, int on) {
  if (!h) return FP_ERR_INVALID;
  h->profiling = on ? 1 : 0;
  h->gdirty = 1;
  h->prof_launches[0] = h->prof_launches[1] = 0;
  h->prof_ms[0] = h->prof_ms[1] = 0;
  h->pending.clear();
  h->ev_used = 0;
  return FP_OK;
}

fp_status fp_get_tuning(const fp_handle *h, fp_tuning *out) {
  if (!h || !out) return FP_ERR_INVALID;
  if (h->stage < 2) return FP_ERR_STATE;
  *out = h->tuning;
  return FP_OK;
}

fp_status fp_get_kernel_stats(const fp_handle *h, int kind, fp_kernel_stats *out) {
  if (!h || !out || kind < 0 || kind > 1) return FP_ERR_INVALID;
  out->launches = h->prof_launches[kind];
  out->total_ms = h->prof_ms[kind];
  out->bytes_per_launch = h->bytes_per_solve;
  out->flops_per_launch = h->flops_per_solve;
  return FP_OK;
}

const char *fp_last_error(const fp_handle *h) { return h ? h->err.c_str() : g_create_err.c_str(); }

void fp_destroy(fp_handle *h) {
  if (!h) return;
  if (h->train_idx) cudaFree(h->train_idx);
  drop_graph(h);
  for (auto &c : h->cap)
    if (c) cudaStreamDestroy(c);
  for (auto &e : h->gev) cudaEventDestroy(e);
  if (h->h_stepv) cudaFreeHost(h->h_stepv);
  if (h->h_flinit) cudaFreeHost(h->h_flinit);
  for (void *p : h->allocs) cudaFree(p);
  if (h->h_fl) cudaFreeHost(h->h_fl);
  if (h->h_sc) cudaFreeHost(h->h_sc);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"

// =========================== projection without allocation ==========================
// fp_apply_projection_noalloc: the coarse projection of fp_apply_projection for callers
// that may not allocate device memory at call time -- an embedding application that has
// reserved the device memory for its own pool, or a latency-bound loop that cannot take
// cudaMalloc's implicit device synchronisation.  Its two scratch vectors (G^T v and (G^T G)^{-1} G^T v) live in the
// file-scope array below instead of handle memory, so the call performs no cudaMalloc,
// cudaFree or allocating library call.  The array is fixed at compile time:
// kNoAllocMaxCoarse coarse unknowns (3 per floating subdomain, i.e. up to 8192 floating
// subdomains), 2 * 24576 doubles = 384 KiB on every device that loads this library, held
// until the process exits.  Host code cannot use the array's name as a device address; the
// address is obtained with cudaGetSymbolAddress once per device, with that device current,
// during the first call on the device, and kept for the life of the process (a
// cudaDeviceReset would make it stale, as it does every handle's memory).
namespace {
constexpr int kNoAllocMaxCoarse = 3 * 8192;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxCoarse];
std::mutex g_noalloc_mu;
double *g_noalloc_addr[128] = {nullptr};
}  // namespace

extern "C" fp_status fp_apply_projection_noalloc(fp_handle *h, const double *v, double *out) {
  if (!h) return FP_ERR_INVALID;
  const Topology &T = h->T;
  if (T.nH > kNoAllocMaxCoarse) {
    h->err = "fp_apply_projection_noalloc: " + std::to_string(T.nH) + " coarse unknowns exceed the fixed scratch of " +
             std::to_string(kNoAllocMaxCoarse) + " (8192 floating subdomains); use fp_apply_projection";
    return FP_ERR_INVALID;
  }
  if (!v || !out) { h->err = "fp_apply_projection_noalloc: NULL vector"; return FP_ERR_INVALID; }
  if (h->stage < 2) { h->err = "fp_apply_projection_noalloc before fp_factor"; return FP_ERR_STATE; }
  int prev = -1;
  CK(cudaGetDevice(&prev));
  if (prev != h->device) CK(cudaSetDevice(h->device));
  fp_status st = FP_OK;
  do {
    if (!T.NF) {
      if (out != v) {
        cudaError_t e = cudaMemcpyAsync(out, v, T.n_lambda * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) { h->err = cudaGetErrorString(e); st = FP_ERR_CUDA; break; }
      }
    } else {
      double *scratch = nullptr;
      {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (h->device < 0 || h->device >= 128) { h->err = "device index out of range"; st = FP_ERR_INVALID; break; }
        if (!g_noalloc_addr[h->device]) {
          void *p = nullptr;
          cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
          if (e != cudaSuccess) { h->err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); st = FP_ERR_CUDA; break; }
          g_noalloc_addr[h->device] = static_cast<double *>(p);
        }
        scratch = g_noalloc_addr[h->device];
      }
      double *cy = scratch, *ca = scratch + kNoAllocMaxCoarse;
      k_Gt<<<(T.NF * 32 + 255) / 256, 256, 0, h->stream>>>(h->D, v, cy, h->fl_zero, nullptr);
      cudaError_t e = launch_gemv(h->Hinv, cy, ca, T.nH, h->fl_zero, h->stream);
      if (e != cudaSuccess) { h->err = std::string("kernel launch: ") + cudaGetErrorString(e); st = FP_ERR_CUDA; break; }
      k_Gcomb<<<(T.n_lambda + 255) / 256, 256, 0, h->stream>>>(h->D, ca, v, -1.0, out, h->fl_zero);
      e = cudaGetLastError();
      if (e != cudaSuccess) { h->err = std::string("kernel launch: ") + cudaGetErrorString(e); st = FP_ERR_CUDA; break; }
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); st = FP_ERR_CUDA; }
  } while (0);
  if (prev != h->device) cudaSetDevice(prev);
  return st;
}
