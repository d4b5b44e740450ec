// Device-side views of the topology and small helpers shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fp {

constexpr unsigned FULL = 0xffffffffu;

// Template (per subdomain shape) data, flattened.
struct DevTpl {
  int n, b, LD, k, poro, nx, ny, nux, nuy, npx, npy, ndl, floating;
  int fixed0, fixed1, fixed2;
  int nbnd, nhalo, nnz;
  long long udof, xidof, pdof;          // offsets into the int pool
  long long dof_field, dof_node;
  long long csr_ptr, csr_col;
  long long bnd, is_bnd;
  long long halo_ptr, halo_row, halo_ent;
  long long elem_dofs;
  long long sell_ptr, sell_col, sell_src;  // sliced ELL of the Neumann matrix (see internal.h)
  int nslice;
};

// Everything the kernels need about the partition, by pointer.
struct DevTopo {
  int S, NF, nlam, nH, bH, LDH, k, nsx, nsy;
  const DevTpl *tpl;
  const int *pool;                  // integer pool for template arrays
  const int *sub_tpl;
  const double *sub_x0, *sub_y0, *sub_hx, *sub_hy;
  const long long *vec_off, *fac_off, *csr_off, *unode_off, *pnode_off, *elem_off, *bsc_off, *sell_off;
  const int *sub_I0, *sub_J0;
  // interface
  const int *lam_sa, *lam_da, *lam_sb, *lam_db, *lam_kind;
  const int *wgrp_first, *wgrp_size;
  int nwgrp;
  const int *bsc_row;
  const int8_t *bsc_sign;
  // coarse
  const int *sub_float, *float_sub, *float_rows_ptr, *float_rows;
  const double *float_g;             // [3 * float_rows] G entries of each (floating subdomain, row) pair
  const int *lam_fa, *lam_fb;        // floating index of s_a / s_b or -1
  const double *lam_ga, *lam_gb;     // [3 * nlam] G row entries for s_a / s_b
};

// Physical parameters used inside kernels.
struct DevParams {
  double lam, mu, alpha, c0, perm_k, mu_f, tau, q_omega;
  int source, src_sub, src_node;
  const double *perm;               // per element or null
};

// A batched banded solve/factor task.
struct BandTask {
  long long fac_off;   // element offset of the factor
  long long x_off;     // element offset of the vector
  long long linv_off;  // element offset of the inverse diagonal 32 x 32 blocks
  int n, LD, b, pad;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Two-float ("double-float") arithmetic: a value is an unevaluated sum h + l of two floats.
// Products and sums use error-free transformations (Knuth's TwoSum; TwoProduct by fma), in the
// manner of Ogita, Rump & Oishi's Dot2: sums of a few hundred terms keep ~2^-46 relative error.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (h, l) += (bh, bl), renormalised (by TwoSum: under cancellation of h and bh the collected low
// parts can exceed the new high part)
__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  two_sum(s, e, h, l);
}
// (h, l) = (ah + al) * (xh + xl), dropping al * xl (~2^-48 relative)
__device__ __forceinline__ void df_mul(float ah, float al, float xh, float xl, float &h, float &l) {
  h = ah * xh;
  l = fmaf(ah, xh, -h) + fmaf(ah, xl, al * xh);
}
// (h, l) += (bh, bl) without renormalising: h takes the exact TwoSum, l collects its error and
// the low parts (long sums; df_norm once before the value is used)
__device__ __forceinline__ void df_add_lazy(float &h, float &l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  h = s;
  l += e + bl;
}
// TwoSum, not the cheaper fast form: after cancellation in h the low part can be the larger one
__device__ __forceinline__ void df_norm(float &h, float &l) {
  float s, e;
  two_sum(h, l, s, e);
  h = s;
  l = e;
}
__device__ __forceinline__ void df_split(double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// PCG state kept on the device: scalar slots, integer flags, reduction finalisers
enum ScSlot { SC_RZ = 0, SC_PQ, SC_ALPHA, SC_BETA, SC_RNORM2, SC_REF2, SC_TOL2, SC_TMP, SC_TRUE2, SC_RMIN,
              SC_N = 16 };
// FL_BODY, FL_RESTARTS, FL_PENDING: loop state of the per-step graph (bodies run in the
// current WHILE loop, restarts taken, restart requested by the last true-residual check).
// FL_STAG: iterations since the recursive residual last halved; FL_STAGWIN: the window after
// which the loop stops for a restart (0: never); FL_NSTAG: such stops in this step.
// FL_NINNER: executions of the inner loop body in this step (for the launch count).
enum FlSlot { FL_DONE = 0, FL_ITER, FL_STATUS, FL_MAXIT, FL_IRSKIP, FL_IRSWEEPS, FL_BODY, FL_RESTARTS, FL_PENDING,
              FL_STAG, FL_STAGWIN, FL_NSTAG, FL_NINNER, FL_N = 13 };
// per-step scalars read by kernels from device memory (so one captured graph serves every
// step): time t_n, extrapolation ratio rho of the source signal, squared tolerance
enum StepSlot { ST_T = 0, ST_RHO, ST_TOL2, ST_N = 4 };
enum RedOp { OP_STORE = 0, OP_PQ = 1, OP_RZ_INIT = 2, OP_RZ = 3, OP_RNORM = 4, OP_RNORM0 = 5 };
// fixed grids of the two-stage reductions (deterministic): the PCG reductions and updates stream
// n_lambda-long vectors with dependent (gathered) loads, so they take 8 CTAs per SM of 152; the
// refinement check, whose finishing thread re-adds the first partials serially, keeps fewer
constexpr int RED_BLOCKS = 1216;
constexpr int RED_BLOCKS_IR = 296;

// arithmetic of the explicit operators' multi-right-hand-side build
enum MrhsPrec { MRHS_FP64 = 0, MRHS_FP32 = 1, MRHS_DF = 2 };

// status codes written by kernels (first error wins)
enum DevStatus { DS_OK = 0, DS_ZERO_PIVOT = 1, DS_TIMEOUT = 2, DS_BREAKDOWN = 3, DS_NONFINITE = 4 };

__device__ __forceinline__ void set_status(int *st, int code) {
  if (st) atomicCAS(st, 0, code);
}

}  // namespace fp
