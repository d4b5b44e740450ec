// FETI interface kernels (Sec. 3): jump operator B / B^T, the scaling W = (B B^T)^{-1},
// the sparse parts of the Dirichlet preconditioner (Eq. (3.5)), the FETI-1 coarse
// projection P = I - G (G^T G)^{-1} G^T, per-step right-hand side and recovery, and the
// reductions and vector updates of Algorithm 1 with all scalars kept on the device.
// Every reduction has a fixed order (per-block tree, then the partials in block order), so
// results are bitwise reproducible run to run.
#include <cmath>

#include "device.cuh"

namespace fp {

// ------------------------------------------------------------------------------------

__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// last-block finalisation of a two-stage reduction; returns true in the finishing thread
__device__ bool finish_reduction(double local, double *partial, unsigned *counter, double &total) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double bsum = block_sum(local, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bsum;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  // the last block's first warp adds the block partials: lane l takes partials l, l + 32, ...
  // in order, then a butterfly (a fixed order, so the sum is reproducible)
  if (threadIdx.x < 32) {
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) t += ((volatile double *)partial)[i];
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      total = t;
      *counter = 0u;
      return true;
    }
  }
  return false;
}

__device__ void apply_op(int op, double v, double *sc, int *fl) {
  switch (op) {
    case OP_STORE:
      sc[SC_TMP] = v;
      break;
    case OP_PQ:
      sc[SC_PQ] = v;
      if (!(v != 0.0) || !isfinite(v)) {
        fl[FL_STATUS] = DS_BREAKDOWN;
        fl[FL_DONE] = 1;
      } else {
        sc[SC_ALPHA] = sc[SC_RZ] / v;
      }
      break;
    case OP_RZ_INIT:
      sc[SC_RZ] = v;
      break;
    case OP_RZ:
      if (!isfinite(v)) { fl[FL_STATUS] = DS_NONFINITE; fl[FL_DONE] = 1; }
      sc[SC_BETA] = v / sc[SC_RZ];
      sc[SC_RZ] = v;
      break;
    case OP_RNORM0:
      sc[SC_RNORM2] = v;
      sc[SC_RMIN] = v;
      fl[FL_STAG] = 0;
      if (!isfinite(v)) { fl[FL_STATUS] = DS_NONFINITE; fl[FL_DONE] = 1; }
      else if (v <= sc[SC_TOL2] * sc[SC_REF2]) fl[FL_DONE] = 1;
      break;
    case OP_RNORM:
      sc[SC_RNORM2] = v;
      fl[FL_ITER] += 1;
      if (!isfinite(v)) { fl[FL_STATUS] = DS_NONFINITE; fl[FL_DONE] = 1; }
      else if (v <= sc[SC_TOL2] * sc[SC_REF2]) fl[FL_DONE] = 1;
      else if (fl[FL_ITER] >= fl[FL_MAXIT]) fl[FL_DONE] = 1;
      else if (v < 0.25 * sc[SC_RMIN]) { sc[SC_RMIN] = v; fl[FL_STAG] = 0; }
      else if (fl[FL_STAGWIN] > 0 && ++fl[FL_STAG] >= fl[FL_STAGWIN]) {
        // stagnation (the inexact FP32 operator of the loop can stall the recursion): stop
        // this round; the true-residual check restarts from the true residual
        fl[FL_DONE] = 1;
        fl[FL_NSTAG] += 1;
      }
      break;
  }
}

// dot(a, b) -> op.  If out_slot is given the raw value is also stored there.
__global__ void k_dot(const double *a, const double *b, long long n, double *partial, unsigned *counter,
                      double *sc, int *fl, int op, double *out_slot, int check_done) {
  if (check_done && fl[FL_DONE]) return;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  double tot;
  if (finish_reduction(s, partial, counter, tot)) {
    if (out_slot) *out_slot = tot;
    apply_op(op, tot, sc, fl);
  }
}

// out[0 .. m) = W_g v for one group of W = (B B^T)^{-1}: per node component a chain of m <= 3
// rows whose B B^T is tridiag(-1, 2, -1), its inverse in closed form (multiplications by the
// constant reciprocals: GB300's FP64 divide is a long instruction sequence; 1/4 is exact, 1/3
// rounds once)
__device__ __forceinline__ void wscale_group(const double *v, int m, double *out) {
  constexpr double third = 1.0 / 3.0;
  if (m == 1) {
    out[0] = 0.5 * v[0];
  } else if (m == 2) {
    out[0] = (2 * v[0] + v[1]) * third;
    out[1] = (v[0] + 2 * v[1]) * third;
  } else {
    out[0] = (3 * v[0] + 2 * v[1] + v[2]) * 0.25;
    out[1] = (2 * v[0] + 4 * v[1] + 2 * v[2]) * 0.25;
    out[2] = (v[0] + 2 * v[1] + 3 * v[2]) * 0.25;
  }
}

// lambda += alpha p; r -= alpha q; then ||r||^2 -> stop test (Algorithm 1, lines 5-6)
__global__ void k_pcg_update(double *lam, double *r, const double *p, const double *q, long long n,
                             double *partial, unsigned *counter, double *sc, int *fl) {
  if (fl[FL_DONE]) return;
  const double alpha = sc[SC_ALPHA];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    lam[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  double tot;
  if (finish_reduction(s, partial, counter, tot)) apply_op(OP_RNORM, tot, sc, fl);
}

// k_pcg_update followed by the first step of the preconditioner (Eq. (3.5)): t = W r, one
// thread per group of W (the rows of one node component; the groups partition the
// multipliers), the scaling of k_wscale on the updated residual.  One launch instead of two.
__global__ void k_pcg_update_w(DevTopo D, double *lam, double *r, const double *p, const double *q, double *t,
                               double *partial, unsigned *counter, double *sc, int *fl) {
  if (fl[FL_DONE]) return;
  const double alpha = sc[SC_ALPHA];
  double s = 0.0;
  for (int gidx = blockIdx.x * blockDim.x + threadIdx.x; gidx < D.nwgrp; gidx += gridDim.x * blockDim.x) {
    const int f = D.wgrp_first[gidx], m = D.wgrp_size[gidx];
    double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // static indices keep v in registers
      if (k < m) {
        const int i = f + k;
        lam[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        s += ri * ri;
        v[k] = ri;
      }
    }
    wscale_group(v, m, t + f);
  }
  double tot;
  if (finish_reduction(s, partial, counter, tot)) apply_op(OP_RNORM, tot, sc, fl);
}

// p = z + beta p (Algorithm 1, line 9)
__global__ void k_pcg_pupdate(double *p, const double *z, long long n, const double *sc, const int *fl) {
  if (fl[FL_DONE]) return;
  const double beta = sc[SC_BETA];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// out = a x + b y  (host scalars; y may be null)
__global__ void k_lincomb(double *out, const double *x, double a, const double *y, double b, long long n,
                          const int *fl) {
  if (fl && fl[FL_DONE]) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// ---------------------------------- jump operator -----------------------------------
// Local vectors x_s = scale * B_s^T v on the dofs touched by B_s, zero elsewhere.
// skip_fixed: leave the fixed dofs of floating subdomains at zero (K^+ convention).
// zero_all: clear the whole local vector first (the band solves read every row); without it
// only the rows touched by B are written (the explicit operators read nothing else), fixed
// dofs of floating subdomains as 0
__global__ void k_scatter(DevTopo D, const double *v, double scale, double *xloc, int skip_fixed, const int *fl,
                          int zero_all) {
  if (fl && fl[FL_DONE]) return;
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  double *x = xloc + D.vec_off[s];
  if (zero_all) {
    for (int d = threadIdx.x; d < t.n; d += blockDim.x) x[d] = 0.0;
    __syncthreads();
  }
  const int *bnd = D.pool + t.bnd;
  const long long b0 = D.bsc_off[s];
  for (int q = threadIdx.x; q < t.nbnd; q += blockDim.x) {
    const int d = bnd[q];
    if (skip_fixed && t.floating && (d == t.fixed0 || d == t.fixed1 || d == t.fixed2)) {
      x[d] = 0.0;
      continue;
    }
    double acc = 0.0;
#pragma unroll
    for (int z = 0; z < 3; ++z) {
      const int r = D.bsc_row[3 * (b0 + q) + z];
      if (r >= 0) acc += D.bsc_sign[3 * (b0 + q) + z] * v[r];
    }
    x[d] = scale * acc;
  }
}

// out[r] = x_{s_a}[d_a] - x_{s_b}[d_b]
__global__ void k_gather(DevTopo D, const double *xloc, double *out, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D.nlam) return;
  out[r] = xloc[D.vec_off[D.lam_sa[r]] + D.lam_da[r]] - xloc[D.vec_off[D.lam_sb[r]] + D.lam_db[r]];
}

// out = W (B x): the gather of k_gather followed by the scaling of k_wscale, one thread per
// group of W (the rows of one node component), in one launch.
__global__ void k_gather_wscale(DevTopo D, const double *xloc, double *out, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= D.nwgrp) return;
  const int f = D.wgrp_first[gidx], m = D.wgrp_size[gidx];
  double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // static indices keep g in registers
    const int r = f + k;
    if (k < m) g[k] = xloc[D.vec_off[D.lam_sa[r]] + D.lam_da[r]] - xloc[D.vec_off[D.lam_sb[r]] + D.lam_db[r]];
  }
  wscale_group(g, m, out + f);
}

// out = W v (wscale_group per group of W)
__global__ void k_wscale(DevTopo D, const double *v, double *out, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= D.nwgrp) return;
  const int f = D.wgrp_first[gidx], m = D.wgrp_size[gidx];
  double v3[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < m) v3[k] = v[f + k];
  wscale_group(v3, m, out + f);
}

// ------------------------------ Dirichlet preconditioner -----------------------------
// y_s = -K_{I b} xb_s on the halo rows (rows outside b coupled to b), zero elsewhere.
__global__ void k_halo(DevTopo D, const double *csr_val, const double *xb, double *y, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const double *xs = xb + D.vec_off[s];
  double *ys = y + D.vec_off[s];
  for (int d = threadIdx.x; d < t.n; d += blockDim.x) ys[d] = 0.0;
  __syncthreads();
  const int *hp = D.pool + t.halo_ptr, *hr = D.pool + t.halo_row, *he = D.pool + t.halo_ent;
  const int *ccol = D.pool + t.csr_col;
  const double *val = csr_val + D.csr_off[s];
  for (int h = threadIdx.x; h < t.nhalo; h += blockDim.x) {
    double acc = 0.0;
    for (int e = hp[h]; e < hp[h + 1]; ++e) acc += val[he[e]] * xs[ccol[he[e]]];
    ys[hr[h]] = -acc;
  }
}

// z_b = K_{b .} (y + xb) on the rows of b (the Schur complement S_s xb, since y solves the
// Dirichlet problem); written back into xb at the rows of b.  y = null: z_b = K_bb xb (xb is
// zero off the rows of b), the lumped preconditioner's local operator.
__global__ void k_bnd_apply(DevTopo D, const double *csr_val, const double *y, double *xb, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  extern __shared__ double zsh[];
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const double *ys = y + D.vec_off[s];
  double *xs = xb + D.vec_off[s];
  const int *bnd = D.pool + t.bnd;
  const int *cptr = D.pool + t.csr_ptr, *ccol = D.pool + t.csr_col;
  const double *val = csr_val + D.csr_off[s];
  for (int q = threadIdx.x; q < t.nbnd; q += blockDim.x) {
    const int row = bnd[q];
    double acc = 0.0;
    for (int e = cptr[row]; e < cptr[row + 1]; ++e) {
      const int c = ccol[e];
      acc += val[e] * ((ys ? ys[c] : 0.0) + xs[c]);
    }
    zsh[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < t.nbnd; q += blockDim.x) xs[bnd[q]] = zsh[q];
}

// ------------------------------ iterative refinement ---------------------------------
// Sliced-ELL values of every subdomain from its assembled CSR values (sell_src: CSR entry,
// -1 padding, -2 the unit diagonal of a fixed row).
__global__ void k_csr_to_sell(DevTopo D, const double *__restrict__ csr_val, double *__restrict__ sell_val) {
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int *src = D.pool + t.sell_src;
  const double *cv = csr_val + D.csr_off[s];
  double *sv = sell_val + D.sell_off[s];
  const long long nslot = D.sell_off[s + 1] - D.sell_off[s];
  for (long long i = threadIdx.x; i < nslot; i += blockDim.x) {
    const int e = src[i];
    sv[i] = e >= 0 ? cv[e] : (e == -2 ? 1.0 : 0.0);
  }
}

// FP64 residual r = b - K_N x of the refinement sweeps (mixed precision), K_N the Neumann
// matrix with the generalised-inverse convention (fixed rows and columns replaced by the
// identity).  One CTA per subdomain, one thread per row over the sliced ELL copy, so every
// warp load of values and column indices is one contiguous segment; a row's entries are
// summed in column order.
__global__ void k_residual_N(DevTopo D, const double *__restrict__ sell_val, const double *__restrict__ b,
                             const double *__restrict__ x, double *__restrict__ r, const int *skip) {
  if (skip && *skip) return;
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const long long off = D.vec_off[s];
  const int *sptr = D.pool + t.sell_ptr, *scol = D.pool + t.sell_col;
  const double *val = sell_val + D.sell_off[s];
  const double *xs = x + off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < t.nslice; q += nw) {
    const int row = 32 * q + lane;
    const int p1 = sptr[q + 1];
    double acc = 0.0;
    for (int p = sptr[q] + lane; p < p1; p += 32) acc += val[p] * xs[scol[p]];
    if (row < t.n) r[off + row] = b[off + row] - acc;
  }
}

// Refinement stop test: after x += r (r the correction of this sweep), skip further sweeps
// once ||r|| <= eps ||x|| (2-norms over all subdomains); or once the predicted next
// correction, ||r|| times the contraction ||r|| / ||r_prev|| of the last sweep, is below
// eps ||x|| (a converging sweep multiplies the error by the FP32 solve's relative accuracy,
// so x is then already that accurate); or, with stag2 > 0, once the correction stagnates
// (||r||^2 > stag2 ||r_prev||^2: the rounding floor of the FP64 residual).  prev2 holds
// ||r_prev||^2 (0 before the first sweep).  After the first sweep the contraction is not yet
// known from this solve: rho2 holds the last one measured (a property of the FP32 factor and
// the matrix, the same for every right-hand side; 0 until measured) and, inflated by 4,
// predicts the next correction.  Counts sweeps in fl[FL_IRSWEEPS].
__global__ void k_ir_check(const double *x, const double *r, long long n, double eps2, double *partial,
                           unsigned *counter, int *fl, double *prev2, double stag2, double *rho2) {
  if (fl[FL_IRSKIP]) return;
  double sr = 0.0, sx = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    sr += r[i] * r[i];
    sx += x[i] * x[i];
  }
  // two two-stage reductions: ||r||^2 into partial[0, G), ||x||^2 into partial[G, 2G)
  double tr, tx;
  finish_reduction(sr, partial, counter, tr);
  if (finish_reduction(sx, partial + gridDim.x, counter + 1, tx)) {
    // the block finishing the second reduction re-sums the first partials (all written
    // before any block's second atomic) in the same fixed order
    double t1 = 0.0;
    for (int i = 0; i < (int)gridDim.x; ++i) t1 += ((volatile double *)partial)[i];
    fl[FL_IRSWEEPS] += 1;
    const double p2 = *prev2;
    if (p2 > 0.0 && t1 < p2) *rho2 = t1 / p2;
    if (t1 <= eps2 * tx || !(t1 == t1) || (p2 > 0.0 && t1 * t1 <= eps2 * tx * p2) ||
        (p2 == 0.0 && *rho2 > 0.0 && 4.0 * *rho2 * t1 <= eps2 * tx) ||
        (stag2 > 0.0 && p2 > 0.0 && t1 > stag2 * p2))
      fl[FL_IRSKIP] = 1;
    *prev2 = t1;
  }
}

// x += r over the whole local-vector array
__global__ void k_local_add(double *x, const double *r, long long n, const int *skip) {
  if (skip && *skip) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += r[i];
}

// ------------------------------------ coarse -----------------------------------------
// float_g[3 q ..] = the G row entries (3 rigid modes) that row float_rows[q] has for the
// floating subdomain owning entry q: one warp per floating subdomain (setup, after k_coarse_G)
__global__ void k_pack_float_g(DevTopo D, double *fg) {
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= D.NF) return;
  for (int q = D.float_rows_ptr[f] + lane; q < D.float_rows_ptr[f + 1]; q += 32) {
    const int r = D.float_rows[q];
    const double *g = (D.lam_fa[r] == f ? D.lam_ga : D.lam_gb) + 3 * (long long)r;
    fg[3 * (long long)q] = g[0];
    fg[3 * (long long)q + 1] = g[1];
    fg[3 * (long long)q + 2] = g[2];
  }
}

// y = G^T v : one warp per floating subdomain, lanes stride over its rows (entries packed per
// subdomain: one index and three coefficients per row), fixed-order sum.
__global__ void k_Gt(DevTopo D, const double *v, double *y, const int *fl, float *ysplit) {
  if (fl && fl[FL_DONE]) return;
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= D.NF) return;
  double a0 = 0, a1 = 0, a2 = 0;
  const int q1 = D.float_rows_ptr[f + 1];
#pragma unroll 4
  for (int q = D.float_rows_ptr[f] + lane; q < q1; q += 32) {
    const double vr = v[D.float_rows[q]];
    const double *g = D.float_g + 3 * (long long)q;
    a0 += g[0] * vr; a1 += g[1] * vr; a2 += g[2] * vr;
  }
  a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
  if (lane == 0) { y[3 * f] = a0; y[3 * f + 1] = a1; y[3 * f + 2] = a2; }
  if (ysplit && lane < 3) {  // two-float copy (hi at [i], lo at [nH + i]) for the tiled product
    const double a = lane == 0 ? a0 : lane == 1 ? a1 : a2;
    float h, l;
    df_split(a, h, l);
    ysplit[3 * f + lane] = h;
    ysplit[3 * D.NF + 3 * f + lane] = l;
  }
}

// alpha = H y with H = (G^T G)^{-1} dense nH x nH (row-major, FP64): one warp per row, y
// read through the cache (every row reuses it), four independent partial sums per lane;
// fixed order.  (Measured on config 5 and dropped: staging y in shared memory per CTA, every
// CTA re-reading all of y, 0.40 ms; four warps per row with a fixed-order combine, 0.24 ms;
// this form 0.22 ms for the 1.06 GB matrix.)
__global__ void __launch_bounds__(256) k_gemv(const double *__restrict__ H, const double *__restrict__ y,
                                              double *alpha, int nH, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nH) return;
  const double *h = H + (long long)row * nH;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = lane;
  for (; c + 96 < nH; c += 128) {
    a0 += h[c] * __ldg(y + c);
    a1 += h[c + 32] * __ldg(y + c + 32);
    a2 += h[c + 64] * __ldg(y + c + 64);
    a3 += h[c + 96] * __ldg(y + c + 96);
  }
  for (; c < nH; c += 32) a0 += h[c] * __ldg(y + c);
  const double acc = warp_sum((a0 + a1) + (a2 + a3));
  if (lane == 0) alpha[row] = acc;
}

cudaError_t launch_gemv(const double *H, const double *y, double *alpha, int nH, const int *fl, cudaStream_t st) {
  k_gemv<<<(unsigned)(((long long)nH * 32 + 255) / 256), 256, 0, st>>>(H, y, alpha, nH, fl);
  return cudaGetLastError();
}

// ------------------- (G^T G)^{-1} y from two-float symmetric tiles ---------------------
// The dense inverse H = (G^T G)^{-1} is symmetric.  Its upper 32 x 32 tiles (I <= J; tile
// index start(I) + J - I, start(I) = I nt - I (I - 1) / 2, nt = ceil(nH / 32)) are stored as
// two FP32 tiles, hi = fl32(h) and lo = fl32(h - hi) (2048 floats per tile, row-major, zero past
// nH): half the bytes of the FP64 matrix, and the products run on FP32 units (GB300's FP64
// rate, not HBM, bounds the FP64 product).  Products and sums use error-free transformations
// (Knuth's TwoSum; TwoProduct by fma) in the manner of Ogita, Rump & Oishi's Dot2, so every
// tile's partial sums carry ~2^-46 relative error; partials are added in FP64 in a fixed order.
namespace {
__device__ __forceinline__ int coarse_tile_row(int tile, int nt) {
  // largest I with start(I) <= tile: an FP32 estimate from the quadratic (GB300's FP64 pipe would
  // make this per-tile index, computed by every lane, the kernel's bottleneck), corrected exactly
  const long long b = 2LL * nt + 1;
  const float disc = (float)max(b * b - 8LL * tile, 0LL);
  int I = (int)(((float)b - sqrtf(disc)) * 0.5f);
  I = max(0, min(I, nt - 1));
  while (I > 0 && I * nt - I * (I - 1) / 2 > tile) --I;
  while (I + 1 < nt && (I + 1) * nt - (I + 1) * I / 2 <= tile) ++I;
  return I;
}
}  // namespace

// Packs the upper tiles of H (dense nH x nH FP64, row-major) into hi/lo FP32 tiles.
__global__ void k_coarse_pack2f(const double *H, int nH, float *tiles) {
  const int nt = (nH + 31) / 32;
  const int tile = blockIdx.x;
  const int I = coarse_tile_row(tile, nt);
  const int J = I + tile - (I * nt - I * (I - 1) / 2);
  float *T = tiles + (long long)tile * 2048;
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    const int a = 32 * I + (e >> 5), j = 32 * J + (e & 31);
    const double v = (a < nH && j < nH) ? H[(long long)a * nH + j] : 0.0;
    float h, l;
    df_split(v, h, l);
    T[e] = h;
    T[1024 + e] = l;
  }
}

// One warp per tile (I, J): lane c holds column c (coalesced 128-byte rows of hi and lo), the
// tile taken in two halves of 16 rows (half the registers of a whole tile: more warps per SM to
// cover the memory latency).  Direct product H_IJ y_J -> row block I: per half a transposing
// butterfly over 16 values (offsets 16, 8, 4, 2; lane l ends with row l >> 1 of the half, summed
// over 16 lanes) and a final exchange with lane l ^ 1.  Transposed product H_IJ^T y_I -> row block
// J (I < J only) as per-lane sums.  y comes pre-split into two floats (ys: hi at [i], lo at
// [nH + i]), so the kernel runs no FP64 instruction; sums run unnormalised (df_add_lazy) and are
// renormalised once; partials go to rp[tile] / cp[tile] as two-float pairs.
__global__ void __launch_bounds__(256, 4) k_coarse_apply2f(const float *__restrict__ tiles, int nH,
                                                           const float *__restrict__ ys, float2 *rp, float2 *cp,
                                                           const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int nt = (nH + 31) / 32, ntile = nt * (nt + 1) / 2;
  const int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (tile >= ntile) return;
  const int I = coarse_tile_row(tile, nt);
  const int J = I + tile - (I * nt - I * (I - 1) / 2);
  const float *T = tiles + (long long)tile * 2048;
  const int col = 32 * J + lane;
  const float yh = col < nH ? __ldg(ys + col) : 0.0f, yl = col < nH ? __ldg(ys + nH + col) : 0.0f;
  float sh = 0.0f, sl = 0.0f;  // transposed product, column `lane`
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float vh[16], vl[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      vh[i] = __ldg(T + (16 * half + i) * 32 + lane);
      vl[i] = __ldg(T + 1024 + (16 * half + i) * 32 + lane);
    }
    if (I < J) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int row = 32 * I + 16 * half + i;
        const float xh = row < nH ? __ldg(ys + row) : 0.0f, xl = row < nH ? __ldg(ys + nH + row) : 0.0f;
        float ph, pl;
        df_mul(vh[i], vl[i], xh, xl, ph, pl);
        df_add_lazy(sh, sl, ph, pl);
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float ph, pl;
      df_mul(vh[i], vl[i], yh, yl, ph, pl);
      vh[i] = ph;
      vl[i] = pl;
    }
#pragma unroll
    for (int k = 16, cnt = 8; k >= 2; k >>= 1, cnt >>= 1) {
      const bool up = (lane & k) != 0;
#pragma unroll
      for (int i = 0; i < cnt; ++i) {
        const float sendh = up ? vh[i] : vh[i + cnt], sendl = up ? vl[i] : vl[i + cnt];
        float kh = up ? vh[i + cnt] : vh[i], kl = up ? vl[i + cnt] : vl[i];
        const float rh = __shfl_xor_sync(FULL, sendh, k), rl = __shfl_xor_sync(FULL, sendl, k);
        df_add_lazy(kh, kl, rh, rl);
        vh[i] = kh;
        vl[i] = kl;
      }
    }
    {
      const float rh = __shfl_xor_sync(FULL, vh[0], 1), rl = __shfl_xor_sync(FULL, vl[0], 1);
      df_add_lazy(vh[0], vl[0], rh, rl);
      df_norm(vh[0], vl[0]);
    }
    if ((lane & 1) == 0) rp[(long long)tile * 32 + 16 * half + (lane >> 1)] = make_float2(vh[0], vl[0]);
  }
  if (I < J) {
    df_norm(sh, sl);
    cp[(long long)tile * 32 + lane] = make_float2(sh, sl);
  }
}

// alpha_i = sum_{J >= I} rp[(I, J)][r] + sum_{J < I} cp[(J, I)][r], i = 32 I + r: one block per
// row block I, warp w takes J = w, w + 8, ... (coalesced rows of partials), two-float sums; the
// eight warp sums are added in a fixed order, and the result is rounded once to FP64.
__global__ void __launch_bounds__(256) k_coarse_sum2f(const float2 *rp, const float2 *cp, int nH, double *alpha,
                                                     const int *fl) {
  if (fl && fl[FL_DONE]) return;
  __shared__ float2 part[8][32];
  const int nt = (nH + 31) / 32, I = blockIdx.x, r = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long row0 = (long long)I * nt - (long long)I * (I - 1) / 2;
  float ah = 0.0f, al = 0.0f;
  for (int J = I + w; J < nt; J += 8) {
    const float2 q = rp[(row0 + J - I) * 32 + r];
    df_add_lazy(ah, al, q.x, q.y);
  }
  for (int J = w; J < I; J += 8) {
    const float2 q = cp[((long long)J * nt - (long long)J * (J - 1) / 2 + I - J) * 32 + r];
    df_add_lazy(ah, al, q.x, q.y);
  }
  df_norm(ah, al);
  part[w][r] = make_float2(ah, al);
  __syncthreads();
  if (w == 0) {
    float sh = 0.0f, sl = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) df_add(sh, sl, part[k][r].x, part[k][r].y);
    const int i = 32 * I + r;
    if (i < nH) alpha[i] = (double)sh + (double)sl;
  }
}

cudaError_t launch_coarse_pack2f(const double *H, int nH, float *tiles, cudaStream_t st) {
  const int nt = (nH + 31) / 32;
  k_coarse_pack2f<<<nt * (nt + 1) / 2, 256, 0, st>>>(H, nH, tiles);
  return cudaGetLastError();
}

cudaError_t launch_coarse_apply2f(const float *tiles, int nH, const float *ysplit, double *part, double *alpha,
                                  const int *fl, cudaStream_t st) {
  const int nt = (nH + 31) / 32;
  const long long ntile = (long long)nt * (nt + 1) / 2;
  float2 *rp = reinterpret_cast<float2 *>(part), *cp = rp + ntile * 32;
  k_coarse_apply2f<<<(unsigned)((ntile * 32 + 255) / 256), 256, 0, st>>>(tiles, nH, ysplit, rp, cp, fl);
  k_coarse_sum2f<<<nt, 256, 0, st>>>(rp, cp, nH, alpha, fl);
  return cudaGetLastError();
}

// out = v + sgn * G alpha  (v may be null)
__global__ void k_Gcomb(DevTopo D, const double *alpha, const double *v, double sgn, double *out, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D.nlam) return;
  double acc = 0.0;
  const int fa = D.lam_fa[r], fb = D.lam_fb[r];
  if (fa >= 0) acc += D.lam_ga[3 * r] * alpha[3 * fa] + D.lam_ga[3 * r + 1] * alpha[3 * fa + 1] + D.lam_ga[3 * r + 2] * alpha[3 * fa + 2];
  if (fb >= 0) acc += D.lam_gb[3 * r] * alpha[3 * fb] + D.lam_gb[3 * r + 1] * alpha[3 * fb + 1] + D.lam_gb[3 * r + 2] * alpha[3 * fb + 2];
  out[r] = (v ? v[r] : 0.0) + sgn * acc;
}

// out = v - G alpha and dot(a, out) -> op in one launch (the projection's last step fused with
// the reduction that follows it in Algorithm 1; the grid and the summation order are those of
// k_dot, so the dot product is the same bit for bit).
__global__ void k_Gcomb_dot(DevTopo D, const double *alpha, const double *v, double *out, const double *a,
                            double *partial, unsigned *counter, double *sc, int *fl, int op) {
  if (fl[FL_DONE]) return;
  double s = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < D.nlam;
       r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    const int fa = D.lam_fa[r], fb = D.lam_fb[r];
    if (fa >= 0) acc += D.lam_ga[3 * r] * alpha[3 * fa] + D.lam_ga[3 * r + 1] * alpha[3 * fa + 1] + D.lam_ga[3 * r + 2] * alpha[3 * fa + 2];
    if (fb >= 0) acc += D.lam_gb[3 * r] * alpha[3 * fb] + D.lam_gb[3 * r + 1] * alpha[3 * fb + 1] + D.lam_gb[3 * r + 2] * alpha[3 * fb + 2];
    const double o = v[r] - acc;
    out[r] = o;
    s += a[r] * o;
  }
  double tot;
  if (finish_reduction(s, partial, counter, tot)) apply_op(op, tot, sc, fl);
}

// ------------------------------- right-hand side --------------------------------------
// f_s at time t: u rows the assembled loads (times g(t)), xi rows 0, p rows
// -(R eta^{n-1}) - tau Z(t)
// (Eq. (2.42) with eta eliminated).  Writes f into xf (fixed dofs of floating subdomains
// zeroed, the K^+ convention) and e_f = R_f^T f_f for floating subdomains.
__global__ void k_rhs(DevTopo D, DevParams P, const double *fstat, const double *Zn, const double *E0n,
                      const double *Reta, const double *stepv, double *xf, double *e) {
  const int s = blockIdx.x;
  const double t_now = stepv[ST_T];
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const double *fs = fstat + D.vec_off[s];
  double *x = xf + D.vec_off[s];
  const int *dfield = D.pool + t.dof_field, *dnode = D.pool + t.dof_node;
  const long long pn0 = D.pnode_off[s];
  const double q_t = sin(P.q_omega * t_now);
  // time factor of the time-dependent manufactured variant: g = 1 + t, g' = 1
  const double g = P.source == 2 ? 1.0 + t_now : 1.0, dg = P.source == 2 ? 1.0 : 0.0;
  const int fidx = D.sub_float[s];
  const double hx = D.sub_hx[s], hy = D.sub_hy[s];
  const double xc = D.sub_x0[s] + 0.5 * t.nx * hx, yc = D.sub_y0[s] + 0.5 * t.ny * hy;
  // node spacing and 1 / L once per subdomain (GB300's FP64 divide is a long sequence)
  const double hxk = hx / t.k, hyk = hy / t.k, invL = 1.0 / fmax(t.nx * hx, t.ny * hy);
  double e0 = 0, e1 = 0, e2 = 0;
  for (int d = threadIdx.x; d < t.n; d += blockDim.x) {
    const int f = dfield[d], node = dnode[d];
    double v = 0.0;
    if (f <= 1) {
      v = g * fs[d];
      if (fidx >= 0) {
        const int ni = node % t.nux, nj = node / t.nux;
        const double xx = D.sub_x0[s] + ni * hxk;
        const double yy = D.sub_y0[s] + nj * hyk;
        if (f == 0) { e0 += v; e2 += -(yy - yc) * invL * v; }
        else { e1 += v; e2 += (xx - xc) * invL * v; }
      }
    } else if (f == 3) {
      double z = g * Zn[pn0 + node] + dg * E0n[pn0 + node];
      if (P.source == 1 && s == P.src_sub && node == P.src_node) z += q_t;
      v = -Reta[pn0 + node] - P.tau * z;
    }
    const bool fixed = t.floating && (d == t.fixed0 || d == t.fixed1 || d == t.fixed2);
    x[d] = fixed ? 0.0 : v;
  }
  if (fidx >= 0) {
    __shared__ double sh[32];
    const double s0 = block_sum(e0, sh);
    const double s1 = block_sum(e1, sh);
    const double s2 = block_sum(e2, sh);
    if (threadIdx.x == 0) { e[3 * fidx] = s0; e[3 * fidx + 1] = s1; e[3 * fidx + 2] = s2; }
  }
}

// --------------------------------- recovery -------------------------------------------
// x_s = (K^+ f)_s - (K^+ B^T lambda)_s + R_s alpha_s; canonical fields; eta; R eta.
__global__ void k_recover(DevTopo D, DevParams P, const double *xf, const double *xl, const double *alpha,
                          double *U, double *XI, double *ETA, double *PP, double *Reta) {
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const double *a = xf + D.vec_off[s];
  const double *b = xl + D.vec_off[s];
  const int *dfield = D.pool + t.dof_field, *dnode = D.pool + t.dof_node;
  const long long un0 = D.unode_off[s], pn0 = D.pnode_off[s];
  const int fidx = D.sub_float[s];
  const double hx = D.sub_hx[s], hy = D.sub_hy[s];
  const double xc = D.sub_x0[s] + 0.5 * t.nx * hx, yc = D.sub_y0[s] + 0.5 * t.ny * hy;
  const double hxk = hx / t.k, hyk = hy / t.k, invL = 1.0 / fmax(t.nx * hx, t.ny * hy);
  // Dirichlet nodes carry the (homogeneous) boundary data: zero everything first
  for (int i = threadIdx.x; i < 2 * t.nux * t.nuy; i += blockDim.x) U[2 * un0 + i] = 0.0;
  for (int i = threadIdx.x; i < t.npx * t.npy; i += blockDim.x) {
    XI[pn0 + i] = 0.0;
    PP[pn0 + i] = 0.0;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < t.n; d += blockDim.x) {
    const int f = dfield[d], node = dnode[d];
    double v = a[d] - b[d];
    if (f <= 1) {
      if (fidx >= 0) {
        const double xx = D.sub_x0[s] + (node % t.nux) * hxk;
        const double yy = D.sub_y0[s] + (node / t.nux) * hyk;
        const double *al = alpha + 3 * fidx;
        if (f == 0) v += al[0] - (yy - yc) * invL * al[2];
        else v += al[1] + (xx - xc) * invL * al[2];
      }
      U[2 * (un0 + node) + f] = v;
    } else if (f == 2) {
      XI[pn0 + node] = v;
    } else {
      PP[pn0 + node] = v;
    }
  }
  __syncthreads();
  if (!t.poro) return;
  const double ce = P.c0 + P.alpha * P.alpha / P.lam, cx = P.alpha / P.lam;
  const int np = t.npx * t.npy;
  for (int node = threadIdx.x; node < np; node += blockDim.x)
    ETA[pn0 + node] = ce * PP[pn0 + node] - cx * XI[pn0 + node];
  __syncthreads();
  // R eta, matrix free: every incident triangle adds area/12 (2 eta_n + eta_a + eta_b)
  const double w = 0.5 * hx * hy / 12.0;
  const double *E = ETA + pn0;
  for (int node = threadIdx.x; node < np; node += blockDim.x) {
    const int i = node % t.npx, j = node / t.npx, nx = t.nx, ny = t.ny, W = t.npx;
    auto e = [&](int ii, int jj) { return E[jj * W + ii]; };
    const double en = e(i, j);
    double acc = 0.0;
    if (i >= 1 && j >= 1) {
      acc += 2 * en + e(i - 1, j - 1) + e(i, j - 1);
      acc += 2 * en + e(i - 1, j - 1) + e(i - 1, j);
    }
    if (i < nx && j >= 1) acc += 2 * en + e(i, j - 1) + e(i + 1, j);
    if (i >= 1 && j < ny) acc += 2 * en + e(i - 1, j) + e(i, j + 1);
    if (i < nx && j < ny) {
      acc += 2 * en + e(i + 1, j) + e(i + 1, j + 1);
      acc += 2 * en + e(i + 1, j + 1) + e(i, j + 1);
    }
    Reta[pn0 + node] = w * acc;
  }
}

// Dense copy of one band matrix for tests: out[r * n + c] (both triangles).
template <typename T>
__global__ void k_band_to_dense(const T *band, int n, int LD, int b, double *out) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    const int lo = min(r, c), hi = max(r, c);
    out[e] = (hi - lo <= b) ? double(band[(long long)lo * LD + hi % LD]) : 0.0;
  }
}
cudaError_t launch_band_to_dense(const double *band, int n, int LD, int b, double *out, cudaStream_t s) {
  k_band_to_dense<double><<<256, 256, 0, s>>>(band, n, LD, b, out);
  return cudaGetLastError();
}

// identity columns for the explicit coarse inverse
__global__ void k_identity(double *X, int nH) {
  const long long tot = (long long)nH * nH;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    X[e] = (e / nH == e % nH) ? 1.0 : 0.0;
}

// ------------------------- loop control of the per-step graph -------------------------
// The Krylov loop of a time step runs as two nested conditional WHILE nodes: the outer one
// restarts from the true residual, the inner one runs chunks of PCG iterations.  These
// single-thread kernels set the loop conditions from the device flags; every loop is also
// bounded by a count (restarts, bodies), so the graph ends whatever the flags say.
__global__ void k_loop_arm_outer(cudaGraphConditionalHandle hc, int *fl) {
  fl[FL_RESTARTS] = 0;
  fl[FL_PENDING] = 0;
  cudaGraphSetConditional(hc, 1u);
}

__global__ void k_loop_arm_inner(cudaGraphConditionalHandle hc, int *fl) {
  fl[FL_BODY] = 0;
  cudaGraphSetConditional(hc, fl[FL_DONE] ? 0u : 1u);
}

__global__ void k_loop_inner(cudaGraphConditionalHandle hc, int *fl, int max_body) {
  const int b = ++fl[FL_BODY];
  fl[FL_NINNER] += 1;
  const bool more = !fl[FL_DONE] && fl[FL_ITER] < fl[FL_MAXIT] && b < max_body;
  cudaGraphSetConditional(hc, more ? 1u : 0u);
}

// after the true residual ||P(d - F lambda)||^2 has been stored in SC_TRUE2: restart while it
// misses the tolerance, no breakdown was flagged and the restart and iteration budgets last
__global__ void k_loop_outer(cudaGraphConditionalHandle hc, int *fl, const double *sc, int max_restarts) {
  const bool ok = sc[SC_TRUE2] <= sc[SC_TOL2] * sc[SC_REF2];
  const bool again = !ok && !fl[FL_STATUS] && fl[FL_RESTARTS] < max_restarts && fl[FL_ITER] < fl[FL_MAXIT];
  if (again) {
    fl[FL_RESTARTS] += 1;
    fl[FL_DONE] = 0;
  }
  fl[FL_PENDING] = again ? 1 : 0;
  cudaGraphSetConditional(hc, again ? 1u : 0u);
}

// dst = src when *flag is set (the restart's r = true residual)
__global__ void k_copy_if(double *dst, const double *src, long long n, const int *flag) {
  if (!*flag) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace fp
